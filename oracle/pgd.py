"""Projection, PGD, rounding/check and annealing with ERWA (TEST INFRASTRUCTURE ONLY).

Follows, in the paper's order:
  * Eq. pg1 / pg2 (Methods, "Projected Gradient Descent"): a gradient step
    then proj_D.  The step is taken in coordinates where the reals are divided
    by the instance length scale S (the paper's instances live in [0, 1]), so
    the b-step is eta * S^2 * dC/db; uniform scaling leaves the Euclidean
    projection of the reals unchanged.
  * Def. Projection / Prop. QP: D = [-1, 1]^n x (box of the reals) x (unit
    atomic constraints).  Single-variable unit atoms tighten the box (exact
    clamp); a single-variable equality pins the real.  A multi-variable equality
    is a hyperplane: its Dykstra multiplier is not clamped (the projection onto
    an affine set), the polish returns points to it within the FP32 band, and
    repair_equalities makes it hold exactly before the exact check (a reading).  Multi-variable unit atoms are half-spaces; the projection onto
    box n half-spaces uses Dykstra's alternating projections (Boyle & Dykstra
    1986) with a fixed number of sweeps, half-spaces in constraint order and
    the box last in each sweep, followed by a short feasibility polish so that
    the point lies in D exactly -- the paper names no QP method, so this is a
    documented reading (the projection it approximates is exact in the limit).
  * Step size: Thm. max_step takes eta = 1/L with L proportional to the total
    weight alpha (Prop. Lipschitz); with ERWA growing the weights, the step is
    eta_r = eta |C_sigma| / alpha_r per restart (a documented reading).
  * Eq. grad_map: g = ((a, b) - proj(...)) / eta, measured in the scaled
    coordinates, and the epsilon-critical stopping rule ||g||^2 <= eps^2
    (Eq. critical), applied per restart.
  * Alg. 1 rounding x = sgn(a) with x_i = TRUE (-1) iff a_i < 0, y = b, and the
    exact check of every constraint (Thm. Soundness).
  * Alg. 2: per sigma stage, PGD to a critical point, round, u_c = [c violated],
    h_c <- rho h_c + u_c, and every tau stages w_c <- w_c gamma^h_c, h_c <- 1;
    SAT when #Unsat = 0.  rho = 0.5, gamma = 2, tau = 1 (Methods).
  * Weight rescale (a documented reading for schedules longer than the paper's
    20 stages): with the normalised step, a restart whose mean weight over
    C_sigma exceeded 2^32 during the stage has its updated weights multiplied by
    2^-32.  Alg. 2 grows every weight by at least gamma^rho per stage (h_c is
    reset to 1), so FP32 weights would overflow after some 90 stages; the
    normalised step does not see a common factor of the weights.

Pins (tests/test_oracle_pgd.py): projection idempotent and non-expansive;
Dykstra against an exact active-set enumeration of the QP on small blocks, and
the polish within 8 margins of that exact projection (bit for bit unchanged
where no half-space is within its margin); the descent lemma with eta = 1/L
(Lemma descent, Prop. Lipschitz) at S = 1 and, in the coordinates y/S, at
S = 100; the step's covariance under a change of the reals' unit (atoms, boxes,
sigma and S times 4 give the reals times 4 and the same ||g||^2, bit for bit);
step_sizes by hand on a three-constraint instance and its independence of the
projected atoms' weights; exact check against planted assignments and
single-literal flips; Fig. 2's two minima; the vectorised kind evaluation
against the scalar definition; with equalities, Dykstra against the active-set QP
with the equality rows always active, the polish back onto the hyperplanes within
their band, and the repair's cases by hand.
The annealing trajectory itself is parity unpinned (the paper gives no
trajectory values for a known step size).
"""
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import objective as OBJ
from . import semantics as S


@dataclass
class Config:
    eta: float = 0.01
    eps: float = 1e-2
    t_max: int = 200
    rho: float = 0.5
    gamma: float = 2.0
    tau: int = 1
    sweeps: int = 20
    polish: int = 32
    normalize_eta: bool = True
    policy: int = OBJ.PROJECT
    inv_sigma: list = field(default_factory=lambda: [0.1 * t for t in range(1, 21)])  # times 1/S


POLISH_MARGIN = 2.0 ** -16


def eq_holds_on_device(var, coef, q0, y):
    """The device check's rule for a projected equality at reals y: it counts as holding
    when |q.y - q0| <= 2^-16 (|q0| + sum |q_j y_j|), the polish margin (a candidate
    filter: the exact repair and check on the host decide SAT)."""
    z = sum(Fraction(int(q)) * Fraction(float(y[int(v)])) for v, q in zip(var, coef)) - int(q0)
    mag = abs(int(q0)) + sum(abs(float(q) * float(y[int(v)])) for v, q in zip(var, coef))
    return abs(float(z)) <= POLISH_MARGIN * mag


def eq_band(n, mag):
    """The band within which an equality's residual q.y - q0 is taken as zero in FP32:
    (n + 4) (u mag + 2^-126-ish), u = 2^-24, mag = |q0| + sum |q_j y_j| over its n
    terms (Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., Sec. 3.1,
    the bound of an n-term FP32 dot product, with two terms for the rounding of mag)."""
    return (n + 4) * (2.0 ** -24 * mag + 1e-38)


def step_sizes(inst, w, cfg, policy=None):
    """Per-restart step size.  With normalize_eta, eta_r = eta |C_sigma| / sum_c w_c[r]:
    Thm. max_step takes eta = 1/L with L proportional to alpha = sum_c w_c (Prop.
    Lipschitz), so the step shrinks as ERWA grows the weights."""
    R = w.shape[1]
    if not cfg.normalize_eta:
        return np.full(R, cfg.eta)
    oc = OBJ.objective_constraints(inst, cfg.policy if policy is None else policy)
    if not oc:
        return np.full(R, cfg.eta)
    return cfg.eta * len(oc) / w[oc].sum(0)


# ---------------------------------------------------------------------------
# the feasible set D
# ---------------------------------------------------------------------------
class Domain:
    """Box [lo, hi] of the reals tightened by unit atoms, plus half-spaces q.y <= q0."""

    def __init__(self, inst, policy=OBJ.PROJECT):
        self.lo = np.array(inst.lo, np.float64)
        self.hi = np.array(inst.hi, np.float64)
        self.halfspaces = []  # (vars, coefs float64, q0 float64)
        self.eq = []          # per entry of halfspaces: an equality's hyperplane q.y = q0
        if policy != OBJ.PROJECT:
            return
        for c in range(inst.n_cons):
            if not OBJ.is_unit_atomic(inst, c):
                continue
            l = int(inst.lits(c)[0])
            var, coef, q0, rel = inst.atom((l >> 1) - inst.n_bool)
            if rel == S.EQ:  # an equality unit atom: a pinned real, or a hyperplane
                if l & 1:
                    raise ValueError("a negated equality is not a convex set")
                if len(var) == 1:
                    v = float(Fraction(int(q0), int(coef[0])))
                    j = int(var[0])
                    self.lo[j], self.hi[j] = max(self.lo[j], v), min(self.hi[j], v)
                else:
                    self.halfspaces.append((np.asarray(var, np.int64), np.asarray(coef, np.float64), float(q0)))
                    self.eq.append(True)
                continue
            coef, q0, strict = S.normalized_atom(coef, q0, rel)
            if l & 1:  # not (q.y <= q0)  ->  -q.y <= -q0 (closure of the open half-space)
                coef, q0 = [-c_ for c_ in coef], -q0
            if len(var) == 1:
                j, qj = int(var[0]), coef[0]
                bound = float(Fraction(q0, qj))
                if qj > 0:
                    self.hi[j] = min(self.hi[j], bound)
                else:
                    self.lo[j] = max(self.lo[j], bound)
            else:
                self.halfspaces.append((np.asarray(var, np.int64), np.asarray(coef, np.float64), float(q0)))
                self.eq.append(False)

    def project_b(self, bp, sweeps, polish=32):
        """proj onto box n half-spaces of points bp [m][R] (Dykstra; exact clamp if no half-space).

        After the Dykstra sweeps, up to `polish` passes make the point feasible:
        each half-space q.y <= q0 whose value is above -margin (margin = 2^-16
        (|q0| + sum |q_j y_j|), far above the rounding error of evaluating q.y) is
        projected onto q.y <= q0 - 2 margin along the reals that are not pinned
        at the bound the step would cross, then the box is clamped; a restart
        stops when a pass moves nothing.  The result satisfies every half-space exactly
        whenever the passes settle.

        An equality is a hyperplane: in Dykstra's sweeps its multiplier is not clamped
        at zero (the projection onto an affine set), and in the polish a hyperplane whose
        residual exceeds eq_band is projected back onto it along the reals not pinned at
        the bound the move would cross (FP32 cannot hold most hyperplanes exactly; the
        exact repair on the host, repair_equalities, finishes them)."""
        x = np.clip(bp, self.lo[:, None], self.hi[:, None])
        if not self.halfspaces:
            return x
        J = np.unique(np.concatenate([h[0] for h in self.halfspaces]))
        x[J] = bp[J]
        R = bp.shape[1]
        p_box = np.zeros((len(J), R))
        t_h = [np.zeros(R) for _ in self.halfspaces]
        for _ in range(sweeps):
            for k, (var, q, q0) in enumerate(self.halfspaces):
                yv = x[var] + t_h[k][None, :] * q[:, None]
                viol = (q[:, None] * yv).sum(0) - q0
                t_h[k] = (viol if self.eq[k] else np.maximum(viol, 0.0)) / float((q * q).sum())
                x[var] = yv - t_h[k][None, :] * q[:, None]
            yv = x[J] + p_box
            xn = np.clip(yv, self.lo[J][:, None], self.hi[J][:, None])
            p_box = yv - xn
            x[J] = xn
        for _ in range(polish):
            moved = np.zeros(R, bool)
            for k, (var, q, q0) in enumerate(self.halfspaces):
                xv = x[var]
                v = (q[:, None] * xv).sum(0) - q0
                if self.eq[k]:  # back onto the hyperplane when off it by more than the FP32 band
                    need = np.abs(v) > eq_band(len(var), abs(q0) + (np.abs(q[:, None] * xv)).sum(0))
                    lo, hi = self.lo[var][:, None], self.hi[var][:, None]
                    dirn = np.sign(v)[None, :] * q[:, None]  # the move is -t q_j, t of the sign of v
                    free = ~(((dirn > 0) & (xv <= lo)) | ((dirn < 0) & (xv >= hi)))
                    qq = ((q * q)[:, None] * free).sum(0)
                    need &= qq > 0
                    step = np.where(need, v / np.where(qq > 0, qq, 1.0), 0.0)
                    x[var] = xv - step[None, :] * q[:, None] * free
                    moved |= need
                    continue
                margin = POLISH_MARGIN * (abs(q0) + (np.abs(q[:, None] * xv)).sum(0))
                need = v > -margin
                # the step moves y_j by -t q_j; a real on the bound it would cross stays put
                lo, hi = self.lo[var][:, None], self.hi[var][:, None]
                free = ~(((q[:, None] > 0) & (xv <= lo)) | ((q[:, None] < 0) & (xv >= hi)))
                qq = ((q * q)[:, None] * free).sum(0)
                need &= qq > 0
                step = np.where(need, (v + 2.0 * margin) / np.where(qq > 0, qq, 1.0), 0.0)
                x[var] = xv - step[None, :] * q[:, None] * free
                moved |= need
            x[J] = np.clip(x[J], self.lo[J][:, None], self.hi[J][:, None])
            if not moved.any():
                break
        return x


def repair_equalities(inst, y):
    """Exact repair of the reals y ([m] floats) so that every projected equality unit
    atom holds exactly, before the exact check (the projection leaves a hyperplane only
    within FP32 rounding).  In constraint order, an equality that does not already hold
    is solved for its pivot: the last of its reals with coefficient +-1 that no earlier
    equality used as pivot; y_p = (q0 - sum_{j != p} q_j y_j) / q_p exactly.  Returns the
    reals as Fractions, or None when an equality has no such real or a later pivot broke
    an earlier equality.  (A reading: the paper's exact check has no equalities to hold.)"""
    yv = [Fraction(float(v)) for v in y]
    eqs = []
    for c in range(inst.n_cons):
        if OBJ.is_unit_atomic(inst, c):
            l = int(inst.lits(c)[0])
            var, coef, q0, rel = inst.atom((l >> 1) - inst.n_bool)
            if rel == S.EQ and not l & 1:
                eqs.append(([int(v) for v in var], [int(q) for q in coef], int(q0)))
    pivots = set()

    def residual(var, coef, q0):
        return sum(Fraction(q) * yv[v] for v, q in zip(var, coef)) - q0

    for var, coef, q0 in eqs:
        if residual(var, coef, q0) == 0:
            continue
        cand = [t for t in range(len(var)) if abs(coef[t]) == 1 and var[t] not in pivots]
        if not cand:
            return None
        t = cand[-1]
        rest = sum(Fraction(coef[u]) * yv[var[u]] for u in range(len(var)) if u != t)
        yv[var[t]] = (q0 - rest) / coef[t]
        pivots.add(var[t])
    if any(residual(*e) != 0 for e in eqs):
        return None
    return yv


def pgd_step(a, b, ga, gb, eta, scale, dom, sweeps, polish=32):
    """One PGD step (Eq. pg1, pg2) and ||g||^2 (Eq. grad_map, scaled coordinates).

    eta is a scalar or one step size per restart ([R])."""
    eta = np.asarray(eta, np.float64)
    a_new = np.clip(a - eta * ga, -1.0, 1.0)
    b_new = dom.project_b(b - eta * scale * scale * gb, sweeps, polish)
    gn2 = (((a - a_new) / eta) ** 2).sum(0) + (((b - b_new) / (scale * eta)) ** 2).sum(0)
    return a_new, b_new, gn2


# ---------------------------------------------------------------------------
# rounding and the exact check
# ---------------------------------------------------------------------------
def kind_value_vec(kind, param, T):
    """semantics.kind_value over restarts: T is a bool array [L][R]."""
    if kind == S.OR:
        return T.any(0)
    if kind == S.XOR:
        return T.sum(0) % 2 == 1
    if kind == S.CARD_LE:
        return T.sum(0) <= param
    if kind == S.NAE:
        return T.any(0) & ~T.all(0)
    if kind == S.MUX:
        idx = sum((T[i].astype(np.int64) << i) for i in range(param))
        return np.take_along_axis(T[param:], idx[None, :], 0)[0]
    if kind == S.NEQ_OR:
        P = param
        r = np.zeros(T.shape[1], bool)
        for i in range(P):
            r |= T[2 * i] != T[2 * i + 1]
        return r | T[2 * P:].any(0)
    raise ValueError(kind)


def atom_truth_exact(inst, i, y):
    """Exact truth of atom i at each restart's reals y [m][R]."""
    return S.atom_truth_batch(inst, i, y)


def round_check(inst, a, b, constraints=None):
    """x = sgn(a) (TRUE iff a < 0), y = b; returns (x int8 [n][R], violated bool [C][R])."""
    a = np.asarray(a)
    R = a.shape[1] if a.ndim == 2 else np.asarray(b).shape[1]
    x = np.where(a < 0, -1, 1).astype(np.int8)
    cons = range(inst.n_cons) if constraints is None else constraints
    viol = np.zeros((inst.n_cons, R), bool)
    atom_cache = {}
    for c in cons:
        ls = inst.lits(c)
        T = np.empty((len(ls), R), bool)
        for t, l in enumerate(ls):
            vid, neg = int(l) >> 1, bool(int(l) & 1)
            if vid < inst.n_bool:
                val = x[vid] == -1
            else:
                val = atom_cache.get(vid)
                if val is None:
                    val = atom_cache[vid] = atom_truth_exact(inst, vid - inst.n_bool, b)
            T[t] = val != neg
        viol[c] = ~kind_value_vec(int(inst.con_kind[c]), int(inst.con_param[c]), T)
    return x, viol


W_RESCALE_AT = 2.0 ** 32


def erwa(w, h, u, t, rho, gamma, tau, mean_w=None):
    """Alg. 2's history and weight update for stage index t (1-based); returns (w, h, #Unsat).

    mean_w [R] (optional): each restart's mean weight over C_sigma during the stage;
    restarts above W_RESCALE_AT get their updated weights times 1 / W_RESCALE_AT."""
    h = rho * h + u
    n_unsat = u.sum(0)
    if t % tau == 0:
        w = w * np.power(gamma, h)
        if mean_w is not None:
            w = w * np.where(np.asarray(mean_w) > W_RESCALE_AT, 1.0 / W_RESCALE_AT, 1.0)
        h = np.ones_like(h)
    return w, h, n_unsat


def mean_weight(inst, w, policy):
    """Per-restart mean weight over the constraints of C_sigma (None when there are none)."""
    oc = OBJ.objective_constraints(inst, policy)
    return w[oc].sum(0) / len(oc) if oc else None


# ---------------------------------------------------------------------------
# one annealing stage and the full Alg. 2 loop
# ---------------------------------------------------------------------------
def run_stage(inst, a, b, w, h, sigma, t, cfg: Config, dom=None, diagrams=None, iters=None):
    """PGD at fixed sigma (Alg. 1's while loop, per restart) then rounding, check and ERWA.

    Returns (a, b, w, h, n_unsat [R], iterations_run [R], obj_last [R]).
    """
    dom = dom or Domain(inst, cfg.policy)
    diagrams = diagrams or OBJ.Diagrams(inst)
    a = np.array(a, np.float64)
    b = np.array(b, np.float64)
    R = w.shape[1]
    active = np.ones(R, bool)
    its = np.zeros(R, np.int64)
    obj = np.zeros(R)
    etas = step_sizes(inst, w, cfg)
    mean_w = mean_weight(inst, w, cfg.policy) if cfg.normalize_eta else None
    for _ in range(cfg.t_max if iters is None else iters):
        obj, _, ga, gb = OBJ.evaluate(inst, a, b, w, sigma, cfg.policy, diagrams)
        a_new, b_new, gn2 = pgd_step(a, b, ga, gb, etas, inst.scale, dom, cfg.sweeps, cfg.polish)
        a[:, active] = a_new[:, active]
        b[:, active] = b_new[:, active]
        its += active
        active &= ~(gn2 <= cfg.eps * cfg.eps)
        if not active.any():
            break
    _, viol = round_check(inst, a, b)
    w, h, n_unsat = erwa(w, h, viol.astype(np.float64), t, cfg.rho, cfg.gamma, cfg.tau, mean_w)
    return a, b, w, h, n_unsat, its, obj


def anneal(inst, a, b, cfg: Config, stages=None):
    """Alg. 2 over the sigma schedule for R restarts; returns per-restart first SAT stage (0 = none)."""
    R = a.shape[1]
    w = np.ones((inst.n_cons, R))
    h = np.zeros((inst.n_cons, R))
    dom = Domain(inst, cfg.policy)
    diagrams = OBJ.Diagrams(inst)
    sat_stage = np.zeros(R, np.int64)
    sched = cfg.inv_sigma if stages is None else cfg.inv_sigma[:stages]
    for t, inv in enumerate(sched, start=1):
        sigma = inst.scale / inv
        a, b, w, h, n_unsat, _, _ = run_stage(inst, a, b, w, h, sigma, t, cfg, dom, diagrams)
        newly = (n_unsat == 0) & (sat_stage == 0)
        sat_stage[newly] = t
        if (sat_stage > 0).all():
            break
    return sat_stage, a, b
