"""Seeded synthetic SMT(LRA) instances shaped like the paper's workloads.

This module only *generates* inputs: constraint sets over Boolean variables and
linear atoms, planted satisfying assignments, and seeded initial points. It
holds none of the method's arithmetic (no COP, no gradient, no projection), so
that both the FP64 oracle and the CUDA path can consume exactly the same inputs.

Conventions (shared by every consumer):
  * Boolean variables have ids 0..n_bool-1; an atom with index i has id n_bool+i.
  * A literal is ``2*id + neg``.  A literal is true when its variable/atom is
    true and neg == 0, or when it is false and neg == 1.
  * A Boolean value x is +-1 with -1 meaning TRUE (the paper's convention, Cor. 1).
  * An atom is ``sum_j coef_j * y_j  rel  q0`` with integer coefficients and
    rel in {LE, LT, GE, GT, EQ}; an EQ atom appears only as a unit constraint.
  * Constraint kinds (the Boolean function of the literal truth values):
      OR      at least one literal true
      XOR     an odd number of literals true
      CARD_LE at most ``param`` literals true
      NAE     not all literals equal (at least one true and one false)
      MUX     ``param`` = b selectors, then 2**b data literals; value is the
              data literal indexed by sum_i 2**i [selector i true]
      NEQ_OR  ``param`` = P pairs; true if some pair (l_2t, l_2t+1) differs
              or one of the remaining literals is true
  * A constraint never names the same variable or atom twice.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

# constraint kinds
OR, XOR, CARD_LE, NAE, MUX, NEQ_OR = 0, 1, 2, 3, 4, 5
KIND_NAMES = {OR: "OR", XOR: "XOR", CARD_LE: "CARD_LE", NAE: "NAE", MUX: "MUX", NEQ_OR: "NEQ_OR"}
# atom relations
LE, LT, GE, GT, EQ = 0, 1, 2, 3, 4


@dataclass
class Instance:
    name: str
    n_bool: int
    n_real: int
    # box bounds on the reals (may be +-inf)
    lo: np.ndarray
    hi: np.ndarray
    # atoms, CSR
    atom_ptr: np.ndarray  # int64 [k+1]
    atom_var: np.ndarray  # int32 [nnz]
    atom_coef: np.ndarray  # int64 [nnz]
    atom_q0: np.ndarray  # int64 [k]
    atom_rel: np.ndarray  # int8 [k]
    # constraints, CSR over literals
    con_kind: np.ndarray  # int8 [C]
    con_param: np.ndarray  # int32 [C]
    con_ptr: np.ndarray  # int64 [C+1]
    con_lits: np.ndarray  # int32 [L]
    # a planted satisfying assignment (x in {-1,+1}, y exact as Fractions via float64)
    planted_x: np.ndarray  # int8 [n]
    planted_y: np.ndarray  # float64 [m] (integers or dyadic values: exact)
    # length scale of the reals (used to scale the sigma schedule and the b-step)
    scale: float = 1.0
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return len(self.atom_q0)

    @property
    def n_cons(self) -> int:
        return len(self.con_kind)

    def lits(self, c: int) -> np.ndarray:
        return self.con_lits[self.con_ptr[c]:self.con_ptr[c + 1]]

    def atom(self, i: int):
        s, e = self.atom_ptr[i], self.atom_ptr[i + 1]
        return self.atom_var[s:e], self.atom_coef[s:e], int(self.atom_q0[i]), int(self.atom_rel[i])


class _Builder:
    """Accumulates atoms and constraints, then freezes them into an Instance."""

    def __init__(self, n_bool: int, n_real: int):
        self.n_bool, self.n_real = n_bool, n_real
        self.atom_var, self.atom_coef, self.atom_ptr = [], [], [0]
        self.atom_q0, self.atom_rel = [], []
        self.kind, self.param, self.lits, self.ptr = [], [], [], [0]

    def atom(self, var, coef, q0, rel=LE) -> int:
        var = [int(v) for v in var]
        assert len(set(var)) == len(var) and len(var) > 0
        self.atom_var += var
        self.atom_coef += [int(c) for c in coef]
        self.atom_ptr.append(len(self.atom_var))
        self.atom_q0.append(int(q0))
        self.atom_rel.append(int(rel))
        return self.n_bool + len(self.atom_q0) - 1  # the atom's id

    def con(self, kind, lits, param=0):
        ids = [l >> 1 for l in lits]
        assert len(set(ids)) == len(ids), "a constraint may not repeat a variable"
        self.kind.append(kind)
        self.param.append(int(param))
        self.lits += [int(l) for l in lits]
        self.ptr.append(len(self.lits))

    def atoms_rows(self, var, coef, q0, rel=LE) -> np.ndarray:
        """Appends one atom per row of var / coef (int arrays [m][nnz]) with right-hand
        sides q0[m], as m calls of atom() would; returns the atoms' ids."""
        var = np.asarray(var, np.int64)
        coef = np.asarray(coef, np.int64)
        m, nnz = var.shape
        assert nnz > 0 and (np.sort(var, 1)[:, 1:] != np.sort(var, 1)[:, :-1]).all()
        first = len(self.atom_q0)
        end = self.atom_ptr[-1]
        self.atom_var += var.ravel().tolist()
        self.atom_coef += coef.ravel().tolist()
        self.atom_ptr += (end + nnz * np.arange(1, m + 1)).tolist()
        self.atom_q0 += np.asarray(q0, np.int64).tolist()
        self.atom_rel += [int(rel)] * m
        return self.n_bool + first + np.arange(m)

    def cons_rows(self, kind, lits, param=0):
        """Appends one constraint per row of lits (int array [m][L]), as m calls of con()."""
        lits = np.asarray(lits, np.int64)
        m, L = lits.shape
        ids = np.sort(lits >> 1, 1)
        assert (ids[:, 1:] != ids[:, :-1]).all(), "a constraint may not repeat a variable"
        end = self.ptr[-1]
        self.kind += [kind] * m
        self.param += [int(param)] * m
        self.lits += lits.ravel().tolist()
        self.ptr += (end + L * np.arange(1, m + 1)).tolist()

    def freeze(self, name, lo, hi, px, py, scale, **meta) -> Instance:
        return Instance(
            name=name, n_bool=self.n_bool, n_real=self.n_real,
            lo=np.asarray(lo, np.float64), hi=np.asarray(hi, np.float64),
            atom_ptr=np.asarray(self.atom_ptr, np.int64),
            atom_var=np.asarray(self.atom_var, np.int32),
            atom_coef=np.asarray(self.atom_coef, np.int64),
            atom_q0=np.asarray(self.atom_q0, np.int64),
            atom_rel=np.asarray(self.atom_rel, np.int8),
            con_kind=np.asarray(self.kind, np.int8),
            con_param=np.asarray(self.param, np.int32),
            con_ptr=np.asarray(self.ptr, np.int64),
            con_lits=np.asarray(self.lits, np.int32),
            planted_x=np.asarray(px, np.int8), planted_y=np.asarray(py, np.float64),
            scale=float(scale), meta=meta)


def lit(var_id: int, neg: bool = False) -> int:
    return 2 * int(var_id) + int(bool(neg))


def _ceil_dot(coef, yvals) -> int:
    """ceil(sum coef*y) computed exactly (y are float64, hence dyadic rationals)."""
    s = sum(Fraction(int(c)) * Fraction(float(v)) for c, v in zip(coef, yvals))
    return math.ceil(s)


# ---------------------------------------------------------------------------
# Tiny random SMT(LRA): 20 Booleans, 10 reals in [0,100], 200 clauses of 3 literals
# ---------------------------------------------------------------------------
def tiny_random(seed: int = 1001, n_bool=20, n_real=10, n_cons=200, width=3) -> Instance:
    rng = np.random.default_rng(seed)
    px = rng.choice(np.array([-1, 1], np.int8), n_bool)
    py = rng.uniform(0.0, 100.0, n_real)
    B = _Builder(n_bool, n_real)
    for _ in range(n_cons):
        lits, truth = [], []
        used_bool = set()
        for _t in range(width):
            if rng.random() < 0.5:
                v = int(rng.integers(n_bool))
                while v in used_bool:
                    v = int(rng.integers(n_bool))
                used_bool.add(v)
                neg = bool(rng.integers(2))
                lits.append(lit(v, neg))
                truth.append((px[v] == -1) != neg)
            else:
                nnz = int(rng.integers(2, 5))
                var = rng.choice(n_real, nnz, replace=False)
                coef = rng.integers(1, 11, nnz) * rng.choice([-1, 1], nnz)
                q0 = _ceil_dot(coef, py[var])  # the atom holds at the plant
                aid = B.atom(var, coef, q0, LE)
                neg = bool(rng.integers(2))
                lits.append(lit(aid, neg))
                truth.append(not neg)
        if not any(truth):  # make the plant satisfy the clause
            lits[0] ^= 1
        B.con(OR, lits)
    return B.freeze("tiny_random", np.zeros(n_real), np.full(n_real, 100.0), px, py, 100.0,
                    seed=seed)


# ---------------------------------------------------------------------------
# Job-shop scheduling with Boolean order selectors
# ---------------------------------------------------------------------------
def _jobshop_into(B: _Builder, rng, n_jobs, n_mach, dur_max, bool_base, real_base, px, py, no_wait=0):
    """Adds one job-shop instance to builder B.  Returns (horizon, n_bool_used, n_real_used).

    no_wait: the last no_wait jobs run without waits between their operations (each
    precedence an equality s_k + d_k = s_{k+1}); the plant then runs them one after
    another after every other job."""
    order = [rng.permutation(n_mach) for _ in range(n_jobs)]
    dur = rng.integers(1, dur_max + 1, (n_jobs, n_mach))
    sidx = lambda j, k: real_base + j * n_mach + k  # real var of the k-th operation of job j
    # planted schedule by greedy list scheduling (operation rank major, jobs in random order)
    start = np.zeros((n_jobs, n_mach), np.int64)
    job_ready = np.zeros(n_jobs, np.int64)
    mach_ready = np.zeros(n_mach, np.int64)
    for k in range(n_mach):
        for j in rng.permutation(n_jobs):
            mch = order[j][k]
            s = max(job_ready[j], mach_ready[mch])
            start[j, k] = s
            job_ready[j] = mach_ready[mch] = s + dur[j, k]
    if no_wait:
        t = int(job_ready[:n_jobs - no_wait].max()) if n_jobs > no_wait else 0
        for j in range(n_jobs - no_wait, n_jobs):
            for k in range(n_mach):
                start[j, k] = t
                t += int(dur[j, k])
            job_ready[j] = t
    H = int(math.ceil(1.2 * int(job_ready.max())))
    for j in range(n_jobs):
        for k in range(n_mach):
            py[sidx(j, k)] = float(start[j, k])
    # unit atoms: 0 <= s and s + d <= H
    for j in range(n_jobs):
        for k in range(n_mach):
            a0 = B.atom([sidx(j, k)], [-1], 0, LE)
            B.con(OR, [lit(a0)])
            a1 = B.atom([sidx(j, k)], [1], H - int(dur[j, k]), LE)
            B.con(OR, [lit(a1)])
    # precedence along each job: s_k + d_k <= s_{k+1} (= for the no-wait jobs)
    for j in range(n_jobs):
        for k in range(n_mach - 1):
            rel = EQ if j >= n_jobs - no_wait else LE
            a = B.atom([sidx(j, k), sidx(j, k + 1)], [1, -1], -int(dur[j, k]), rel)
            B.con(OR, [lit(a)])
    # same-machine pairs with an order selector o: o -> (i before j), not o -> (j before i)
    ops_on = [[] for _ in range(n_mach)]
    for j in range(n_jobs):
        for k in range(n_mach):
            ops_on[order[j][k]].append((j, k))
    nb = 0
    for mch in range(n_mach):
        ops = ops_on[mch]
        for u in range(len(ops)):
            for v in range(u + 1, len(ops)):
                (ji, ki), (jj, kj) = ops[u], ops[v]
                o = bool_base + nb
                nb += 1
                si, sj = sidx(ji, ki), sidx(jj, kj)
                di, dj = int(dur[ji, ki]), int(dur[jj, kj])
                a_ij = B.atom([si, sj], [1, -1], -di, LE)  # s_i + d_i <= s_j
                a_ji = B.atom([sj, si], [1, -1], -dj, LE)  # s_j + d_j <= s_i
                B.con(OR, [lit(o, True), lit(a_ij)])
                B.con(OR, [lit(o, False), lit(a_ji)])
                px[o] = -1 if start[ji, ki] < start[jj, kj] else 1
    return H, nb, n_jobs * n_mach


def jobshop(seed: int = 1002, n_jobs=40, n_mach=10, dur_max=20, no_wait=0) -> Instance:
    rng = np.random.default_rng(seed)
    n_bool = n_mach * n_jobs * (n_jobs - 1) // 2
    n_real = n_jobs * n_mach
    B = _Builder(n_bool, n_real)
    px = np.ones(n_bool, np.int8)
    py = np.zeros(n_real)
    H, nb, nr = _jobshop_into(B, rng, n_jobs, n_mach, dur_max, 0, 0, px, py, no_wait)
    assert nb == n_bool and nr == n_real
    lo = np.zeros(n_real)
    hi = np.full(n_real, float(H))
    return B.freeze("jobshop", lo, hi, px, py, float(dur_max), seed=seed, horizon=H,
                    n_jobs=n_jobs, n_mach=n_mach)


def uneven_batch(seed: int = 1004, n_inst=64, jobs=(5, 60), machines=(3, 15), dur_max=20):
    """A list of job-shop instances of very different sizes (one per batch member)."""
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n_inst):
        nj = int(rng.integers(jobs[0], jobs[1] + 1))
        nm = int(rng.integers(machines[0], machines[1] + 1))
        out.append(jobshop(seed * 1000 + t, nj, nm, dur_max))
    return out


# ---------------------------------------------------------------------------
# 2D placement with Boolean selectors
# ---------------------------------------------------------------------------
def placement2d(seed: int = 1003, n_rect=400, dim_max=30, selectors=True) -> Instance:
    redraws = 0
    while True:
        rng = np.random.default_rng(seed + 7919 * redraws)
        w = rng.integers(1, dim_max + 1, n_rect)
        h = rng.integers(1, dim_max + 1, n_rect)
        L = int(math.ceil(math.sqrt(1.3 * float((w * h).sum()))))
        # shelf packing plant: tallest first, left to right, shelves upwards
        order = np.argsort(-h, kind="stable")
        X = np.zeros(n_rect, np.int64)
        Y = np.zeros(n_rect, np.int64)
        cx, cy, shelf_h, ok = 0, 0, 0, True
        for i in order:
            if cx + w[i] > L:
                cy += shelf_h
                cx, shelf_h = 0, 0
            X[i], Y[i] = cx, cy
            cx += w[i]
            shelf_h = max(shelf_h, int(h[i]))
            if cy + h[i] > L:
                ok = False
                break
        if ok:
            break
        redraws += 1
    n_real = 2 * n_rect
    n_pairs = n_rect * (n_rect - 1) // 2
    n_bool = 2 * n_pairs if selectors else 0
    B = _Builder(n_bool, n_real)
    xv = lambda i: 2 * i
    yv = lambda i: 2 * i + 1
    py = np.zeros(n_real)
    for i in range(n_rect):
        py[xv(i)], py[yv(i)] = float(X[i]), float(Y[i])
    px = np.ones(n_bool, np.int8)
    # feasibility: 0 <= x <= L - w, 0 <= y <= L - h  (unit atoms)
    for i in range(n_rect):
        for v, size in ((xv(i), w[i]), (yv(i), h[i])):
            B.con(OR, [lit(B.atom([v], [-1], 0, LE))])
            B.con(OR, [lit(B.atom([v], [1], L - int(size), LE))])
    p = 0
    for i in range(n_rect):
        for j in range(i + 1, n_rect):
            A1 = B.atom([xv(i), xv(j)], [1, -1], -int(w[i]), LE)  # x_i + w_i <= x_j
            A2 = B.atom([xv(j), xv(i)], [1, -1], -int(w[j]), LE)  # x_j + w_j <= x_i
            A3 = B.atom([yv(i), yv(j)], [1, -1], -int(h[i]), LE)  # y_i + h_i <= y_j
            A4 = B.atom([yv(j), yv(i)], [1, -1], -int(h[j]), LE)  # y_j + h_j <= y_i
            holds = [X[i] + w[i] <= X[j], X[j] + w[j] <= X[i], Y[i] + h[i] <= Y[j], Y[j] + h[j] <= Y[i]]
            if selectors:
                u, v = 2 * p, 2 * p + 1
                # ITE(u, ITE(v, A1, A2), ITE(v, A3, A4)) as a MUX with index [u] + 2[v]:
                #   idx 0 (u F, v F) -> A4, 1 (u T, v F) -> A2, 2 (u F, v T) -> A3, 3 (u T, v T) -> A1
                B.con(MUX, [lit(u), lit(v), lit(A4), lit(A2), lit(A3), lit(A1)], param=2)
                k = int(np.argmax(holds))  # which disjunct the plant uses
                uT, vT = {0: (True, True), 1: (True, False), 2: (False, True), 3: (False, False)}[k]
                px[u] = -1 if uT else 1
                px[v] = -1 if vT else 1
            else:
                B.con(OR, [lit(A1), lit(A2), lit(A3), lit(A4)])
            p += 1
    lo = np.zeros(n_real)
    hi = np.full(n_real, float(L))
    return B.freeze("placement2d" + ("" if selectors else "_nosel"), lo, hi, px, py, float(dim_max),
                    seed=seed, redraws=redraws, die=L)


# ---------------------------------------------------------------------------
# 3D placement (macro and layer index bits, routing-aware adjacency)
# ---------------------------------------------------------------------------
P3_MACRO = 20                                  # macro side; every size below is an integer
P3_SIZES = {"large_proc": (8, 8), "small_proc": (4, 4), "large_mem": (2, 2)}


def placement3d(seed: int = 1007, n_macros=64, n_layers=8) -> Instance:
    """The paper's 3D placement encoding (Methods, "3D Placement").

    Modules: n_macros large processes, n_macros*n_layers small processes, n_macros
    large memories and n_macros*n_layers/2 small memories.  Lengths are in units of
    1/20 of the macro side, so that every size is an integer: macro 20 x 20, large
    process 8 x 8, small process 4 x 4, large memory 2 x 2, small memory 2 x 1 or
    1 x 2 (its alignment along x or y drawn per element).  Module j has macro-index
    bits m_{i,j} (log2 n_macros), layer-index bits l_{i,j} (log2 n_layers) and
    macro-relative coordinates x_j, y_j in [0, 20].

    Constraints:
      * feasibility: unit atoms 0 <= x_j <= 20 - w_j, 0 <= y_j <= 20 - d_j;
      * routing-aware, per associated pair (j, j'): for every macro bit i the unit
        clause (m_{i,j} = m_{i,j'}) (an XOR with one literal negated), and the unit
        atoms x_j - x_j' <= w_j', x_j' - x_j <= w_j, y_j - y_j' <= d_j',
        y_j' - y_j <= d_j (the two touch or overlap in both axes; on different
        layers they may stack);
      * non-overlap, per pair of modules: some macro bit differs, or some layer bit
        differs, or one of x_j - x_j' >= w_j', x_j' - x_j >= w_j, y_j - y_j' >= d_j',
        y_j' - y_j >= d_j holds (one disjunction, as an NEQ_OR).
    Association: each large process with one large memory, and each small memory
    with two small processes (n_macros*n_layers small processes and half as many
    small memories pair up only this way).  Module ids are a random permutation.

    Plant, per macro t: its large pair on layer 0 at (0, 0) and (8, 0); its small
    process k on layer k at (10, 10); its small memory q on layer 2q at (14, 10),
    touching process 2q and stacked beside process 2q + 1.
    """
    assert n_macros >= 2 and n_macros & (n_macros - 1) == 0
    assert n_layers >= 2 and n_layers & (n_layers - 1) == 0
    rng = np.random.default_rng(seed)
    bm, bl = n_macros.bit_length() - 1, n_layers.bit_length() - 1
    # modules in plant order: per macro, large process, large memory, small processes, small memories
    size, macro, layer, X, Y, kind = [], [], [], [], [], []
    pairs = []                                          # associated (plant index, plant index)
    for t in range(n_macros):
        base = len(size)
        for name, lay, xy in (("large_proc", 0, (0, 0)), ("large_mem", 0, (8, 0))):
            size.append(P3_SIZES[name]); macro.append(t); layer.append(lay); X.append(xy[0]); Y.append(xy[1])
            kind.append(name)
        pairs.append((base, base + 1))
        procs = []
        for k in range(n_layers):
            procs.append(len(size))
            size.append(P3_SIZES["small_proc"]); macro.append(t); layer.append(k); X.append(10); Y.append(10)
            kind.append("small_proc")
        for q in range(n_layers // 2):
            m = len(size)
            size.append((2, 1) if rng.random() < 0.5 else (1, 2)); macro.append(t); layer.append(2 * q)
            X.append(14); Y.append(10); kind.append("small_mem")
            pairs += [(procs[2 * q], m), (procs[2 * q + 1], m)]
    N = len(size)
    perm = rng.permutation(N)                           # plant index -> module id
    nb = bm + bl
    mbit = lambda j, i: j * nb + i
    lbit = lambda j, i: j * nb + bm + i
    xv = lambda j: 2 * j
    yv = lambda j: 2 * j + 1
    B = _Builder(N * nb, 2 * N)
    px = np.ones(N * nb, np.int8)
    py = np.zeros(2 * N)
    w = np.zeros(N, np.int64)
    d = np.zeros(N, np.int64)
    for s in range(N):
        j = int(perm[s])
        w[j], d[j] = size[s]
        py[xv(j)], py[yv(j)] = float(X[s]), float(Y[s])
        for i in range(bm):
            px[mbit(j, i)] = -1 if (macro[s] >> i) & 1 else 1
        for i in range(bl):
            px[lbit(j, i)] = -1 if (layer[s] >> i) & 1 else 1
    # feasibility
    for j in range(N):
        for v, sz in ((xv(j), w[j]), (yv(j), d[j])):
            B.con(OR, [lit(B.atom([v], [-1], 0, LE))])
            B.con(OR, [lit(B.atom([v], [1], P3_MACRO - int(sz), LE))])
    # routing-aware
    for s, s2 in pairs:
        j, k = int(perm[s]), int(perm[s2])
        for i in range(bm):
            B.con(XOR, [lit(mbit(j, i)), lit(mbit(k, i), neg=True)])
        B.con(OR, [lit(B.atom([xv(j), xv(k)], [1, -1], int(w[k]), LE))])
        B.con(OR, [lit(B.atom([xv(k), xv(j)], [1, -1], int(w[j]), LE))])
        B.con(OR, [lit(B.atom([yv(j), yv(k)], [1, -1], int(d[k]), LE))])
        B.con(OR, [lit(B.atom([yv(k), yv(j)], [1, -1], int(d[j]), LE))])
    # non-overlap for every pair j < k (row-major): the macro-bit and layer-bit XOR
    # pairs, then x_j - x_k >= w_k, x_k - x_j >= w_j, y_j - y_k >= d_k, y_k - y_j >= d_j
    J, K = np.triu_indices(N, 1)
    var = np.stack([2 * K, 2 * J, 2 * J, 2 * K, 2 * K + 1, 2 * J + 1, 2 * J + 1, 2 * K + 1], 1).reshape(-1, 2)
    q0 = np.stack([-w[K], -w[J], -d[K], -d[J]], 1).ravel()
    A = B.atoms_rows(var, np.tile([1, -1], (4 * len(J), 1)), q0).reshape(-1, 4)
    mb = np.stack([J[:, None] * nb + np.arange(bm), K[:, None] * nb + np.arange(bm)], 2).reshape(len(J), 2 * bm)
    lb = np.stack([J[:, None] * nb + bm + np.arange(bl), K[:, None] * nb + bm + np.arange(bl)],
                  2).reshape(len(J), 2 * bl)
    B.cons_rows(NEQ_OR, np.concatenate([2 * mb, 2 * lb, 2 * A], 1), param=nb)
    lo = np.zeros(2 * N)
    hi = np.full(2 * N, float(P3_MACRO))
    kinds = np.array(kind)[np.argsort(perm)]
    return B.freeze("placement3d", lo, hi, px, py, float(P3_MACRO), seed=seed, n_macros=n_macros,
                    n_layers=n_layers, n_modules=N, n_pairs=len(pairs), kinds=kinds.tolist())


# ---------------------------------------------------------------------------
# Large continuous-time scheduling (worker-index bits, pairwise non-overlap)
# ---------------------------------------------------------------------------
def large_scheduling(seed: int = 1005, n_workers=256, n_jobs=1111, dur_max=20,
                     n_late=72, late_max=10, chain_max=3, n_early=0, name="large_scheduling") -> Instance:
    """The paper's scheduling encoding at ~10k variables / ~0.7M constraints.

    Per job j: worker-index bits x_{i,j} (log2 n_workers of them) and a start time y_j.
    Constraints: per-pair non-overlap  OR_i (x_{i,j} xor x_{i,j'}) OR (y_j - y_j' >= t_j')
    OR (y_j' - y_j >= t_j); precedence y_j >= y_j' + t_j' inside short job chains;
    release/deadline unit atoms 0 <= y_j, y_j + t_j <= T; and, for each of ``n_late``
    workers that start late at d_w, per job: (X_j != w) OR (y_j >= d_w).  With
    ``n_early`` > 0, as many workers also close early at e_w (the deadline side of a
    worker's availability window), per job: (X_j != w) OR (y_j + t_j <= e_w); e_w is
    drawn in [0.5, 0.8] x the makespan of the plain greedy plant, and the plant is then
    redone so that no job on such a worker ends after e_w.

    When n_workers is not a power of two the index takes ceil(log2 n_workers) bits and
    each job also gets clauses that keep X_j below n_workers: the unused codes
    [n_workers, 2**bits) are covered by aligned blocks (one per set bit of
    2**bits - n_workers, as in a binary range split), and each block forbids its prefix
    with one OR clause over the prefix bits.
    """
    rng = np.random.default_rng(seed)
    bits = max(1, (n_workers - 1).bit_length())
    assert n_workers >= 2 and n_late <= n_workers
    n_bool = bits * n_jobs
    n_real = n_jobs
    t = rng.integers(1, dur_max + 1, n_jobs)
    d = np.zeros(n_workers, np.int64)
    late = rng.choice(n_workers, n_late, replace=False)
    d[late] = rng.integers(1, late_max + 1, n_late)
    # precedence: jobs form chains of 1..chain_max consecutive jobs
    pred = -np.ones(n_jobs, np.int64)
    j = 0
    while j < n_jobs:
        ln = int(rng.integers(1, chain_max + 1))
        for q in range(j + 1, min(j + ln, n_jobs)):
            pred[q] = q - 1
        j += ln
    # planted greedy schedule: each job to the worker where it can start earliest
    def greedy(close):
        free = d.copy()
        Y = np.zeros(n_jobs, np.int64)
        W = np.zeros(n_jobs, np.int64)
        for j in range(n_jobs):
            ready = 0 if pred[j] < 0 else Y[pred[j]] + t[pred[j]]
            st = np.maximum(free, ready)
            if close is not None:
                st = np.where(st + t[j] <= close, st, np.iinfo(np.int64).max)
            w = int(np.argmin(st))
            Y[j], W[j] = st[w], w
            free[w] = st[w] + t[j]
        return Y, W

    Y, W = greedy(None)
    early, e = np.zeros(0, np.int64), None
    if n_early:
        assert n_early < n_workers
        rng2 = np.random.default_rng([seed, 2])   # its own stream: n_early = 0 draws nothing
        early = rng2.choice(n_workers, n_early, replace=False)
        M = int((Y + t).max())
        e = np.full(n_workers, np.iinfo(np.int64).max // 2)
        e[early] = rng2.integers(int(math.ceil(0.5 * M)), int(math.ceil(0.8 * M)) + 1, n_early)
        Y, W = greedy(e)
    T = int(math.ceil(1.2 * int((Y + t).max())))
    xb = lambda i, j: j * bits + i  # Boolean id of bit i of job j
    B = _Builder(n_bool, n_real)
    px = np.ones(n_bool, np.int8)
    for j in range(n_jobs):
        for i in range(bits):
            px[xb(i, j)] = -1 if (W[j] >> i) & 1 else 1
    py = Y.astype(np.float64)
    # non-overlap for every pair j < k (row-major, as two nested loops would give):
    # OR_i (x_ij xor x_ik) OR A1 OR A2 with A1: y_j - y_k >= t_k, A2: y_k - y_j >= t_j
    J, K = np.triu_indices(n_jobs, 1)
    atom_pairs = B.atoms_rows(np.stack([K, J, J, K], 1).reshape(-1, 2), np.tile([1, -1], (2 * len(J), 1)),
                              np.stack([-t[K], -t[J]], 1).ravel())
    A = atom_pairs.reshape(-1, 2)
    bit_lits = np.stack([2 * (J[:, None] * bits + np.arange(bits)), 2 * (K[:, None] * bits + np.arange(bits))],
                        2).reshape(len(J), 2 * bits)
    B.cons_rows(NEQ_OR, np.concatenate([bit_lits, 2 * A], 1), param=bits)
    # precedence
    for j in range(n_jobs):
        if pred[j] >= 0:
            B.con(OR, [lit(B.atom([int(pred[j]), j], [1, -1], -int(t[pred[j]]), LE))])
    # release / deadline
    for j in range(n_jobs):
        B.con(OR, [lit(B.atom([j], [-1], 0, LE))])
        B.con(OR, [lit(B.atom([j], [1], T - int(t[j]), LE))])
    # worker index in range: for each aligned block [lo, lo + 2**k) of unused codes,
    # NOT(bits >= k of X_j equal those of lo)
    blocks, lo_code = [], n_workers
    while lo_code < (1 << bits):
        k = (lo_code & -lo_code).bit_length() - 1  # largest aligned block starting here
        while lo_code + (1 << k) > (1 << bits):
            k -= 1
        blocks.append((lo_code, k))
        lo_code += 1 << k
    for j in range(n_jobs):
        for code, k in blocks:
            B.con(OR, [lit(xb(i, j), neg=bool((code >> i) & 1)) for i in range(k, bits)])
    # late workers: (X_j != w) OR (y_j >= d_w)
    for w in late:
        for j in range(n_jobs):
            lits = [lit(xb(i, j), neg=bool((int(w) >> i) & 1)) for i in range(bits)]
            lits.append(lit(B.atom([j], [-1], -int(d[w]), LE)))
            B.con(OR, lits)
    # early-closing workers: (X_j != w) OR (y_j + t_j <= e_w)
    for w in early:
        for j in range(n_jobs):
            lits = [lit(xb(i, j), neg=bool((int(w) >> i) & 1)) for i in range(bits)]
            lits.append(lit(B.atom([j], [1], int(e[w]) - int(t[j]), LE)))
            B.con(OR, lits)
    lo = np.zeros(n_real)
    hi = np.full(n_real, float(T))
    return B.freeze(name, lo, hi, px, py, float(dur_max), seed=seed, horizon=T,
                    n_workers=n_workers, n_jobs=n_jobs, n_late=n_late, n_early=n_early,
                    close=(e[early].tolist() if n_early else []))


def concat(instances, name="batch") -> Instance:
    """Block-diagonal union of instances (disjoint variables), for batched solving.

    meta['bool_base'], meta['real_base'], meta['con_base'] give each member's offsets.
    """
    n_bool = sum(I.n_bool for I in instances)
    n_real = sum(I.n_real for I in instances)
    B = _Builder(n_bool, n_real)
    bb, rb, cb = [0], [0], [0]
    for I in instances:
        boff, roff, aoff_new = bb[-1], rb[-1], None
        atom_map = {}
        for i in range(I.n_atoms):
            var, coef, q0, rel = I.atom(i)
            atom_map[I.n_bool + i] = B.atom(var + roff, coef, q0, rel)
        for c in range(I.n_cons):
            ls = []
            for l in I.lits(c):
                vid, neg = int(l) >> 1, int(l) & 1
                nid = vid + boff if vid < I.n_bool else atom_map[vid]
                ls.append(2 * nid + neg)
            B.con(int(I.con_kind[c]), ls, int(I.con_param[c]))
        bb.append(boff + I.n_bool)
        rb.append(roff + I.n_real)
        cb.append(cb[-1] + I.n_cons)
    return B.freeze(name, np.concatenate([I.lo for I in instances]),
                    np.concatenate([I.hi for I in instances]),
                    np.concatenate([I.planted_x for I in instances]),
                    np.concatenate([I.planted_y for I in instances]),
                    max(I.scale for I in instances),
                    bool_base=bb, real_base=rb, con_base=cb, members=len(instances))


# ---------------------------------------------------------------------------
# Seeded initial points (restart-minor layout [var][R], float32)
# ---------------------------------------------------------------------------
def initial_point(inst: Instance, R: int, seed: int = 7):
    """a ~ U(-1,1); b_j ~ U(lo_j, hi_j) (U(0, scale) where a bound is infinite)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, (inst.n_bool, R)).astype(np.float32)
    lo = np.where(np.isfinite(inst.lo), inst.lo, 0.0)
    hi = np.where(np.isfinite(inst.hi), inst.hi, lo + inst.scale)
    b = (lo[:, None] + (hi - lo)[:, None] * rng.random((inst.n_real, R))).astype(np.float32)
    return a, b


# ---------------------------------------------------------------------------
# Random hybrid constraints (cardinality, not-all-equal, parity) over Booleans
# and LRA atoms: the random benchmark of the paper's Results and Methods
# ---------------------------------------------------------------------------
def random_hybrid(seed: int = 1006, n: int = 100) -> Instance:
    """n Booleans, n reals in [0, 1] and n LRA atoms; n/5 cardinality constraints
    (sum of literals <= k) and n/5 not-all-equal constraints of min(50, n/5)
    literals each, and n/50 parity constraints of 50 literals.  A literal is a
    Boolean or an atom, negated at random; literals of one constraint are
    distinct variables.  An atom has 2-4 reals with integer coefficients in
    [-10, 10] \\ {0} and q0 one of round(q.y*) - 1, +0, +1 at a planted point y*, so
    atoms hold or fail there at random.  A planted (x*, y*) satisfies every
    constraint: k is at least the number of true literals (and at least half
    the length), and a not-all-equal or parity constraint that fails at the
    plant has its first literal's polarity flipped."""
    rng = np.random.default_rng(seed)
    px = rng.choice(np.array([-1, 1], np.int8), n)
    py = rng.uniform(0.0, 1.0, n)
    B = _Builder(n, n)
    atom_true = []
    for _ in range(n):
        nnz = int(rng.integers(2, 5))
        var = rng.choice(n, nnz, replace=False)
        coef = rng.integers(1, 11, nnz) * rng.choice([-1, 1], nnz)
        exact = sum(Fraction(int(cf)) * Fraction(float(py[v])) for cf, v in zip(coef, var))
        q0 = int(round(exact)) + int(rng.integers(-1, 2))
        B.atom(var, coef, q0, LE)
        atom_true.append(exact <= q0)

    def literals(length):
        ids = rng.choice(2 * n, length, replace=False)  # 0..n-1 Booleans, n..2n-1 atoms
        lits, truth = [], []
        for v in ids:
            v = int(v)
            neg = bool(rng.integers(2))
            lits.append(lit(v, neg))
            val = (px[v] == -1) if v < n else atom_true[v - n]
            truth.append(bool(val) != neg)
        return lits, truth

    l_cn = min(50, n // 5)
    for _ in range(n // 5):  # cardinality
        lits, truth = literals(l_cn)
        B.con(CARD_LE, lits, param=max(sum(truth), l_cn // 2))
    for _ in range(n // 5):  # not-all-equal
        lits, truth = literals(l_cn)
        if all(truth) or not any(truth):
            lits[0] ^= 1
        B.con(NAE, lits)
    for _ in range(max(1, n // 50)):  # parity
        lits, truth = literals(min(50, 2 * n))
        if sum(truth) % 2 == 0:
            lits[0] ^= 1
        B.con(XOR, lits)
    return B.freeze("random_hybrid", np.zeros(n), np.ones(n), px, py, 1.0, seed=seed, n=n)


CONFIGS = {
    "tiny_random": dict(make=lambda: tiny_random(1001), R=64),
    "jobshop": dict(make=lambda: jobshop(1002), R=256),
    "placement2d": dict(make=lambda: placement2d(1003), R=1024),
    "uneven_batch": dict(make=lambda: concat(uneven_batch(1004), "uneven_batch"), R=32),
    "large_scheduling": dict(make=lambda: large_scheduling(1005), R=512),
    "placement3d": dict(make=lambda: placement3d(1007), R=512),
    "large_scheduling_lit": dict(make=lambda: large_scheduling(1005, n_workers=20, n_jobs=1000, n_late=6), R=512),
    "random_hybrid": dict(make=lambda: random_hybrid(1006, 1000), R=100),
}
