/*
 * fsmt.h -- C ABI of the B300 engine for FourierSMT's hot path (arxiv 2603.22877).
 *
 * The engine evaluates, for R restarts at once, the relaxed objective
 *     C_sigma(a, b) = sum_c w_c (1 - 2 COP_c)
 * where COP_c is the circuit-output probability of constraint c's extended BDD
 * (xBDD) under randomized rounding of the Booleans and Gaussian smoothing of the
 * atoms; its exact gradient by an adjoint sweep; the projected-gradient step; and
 * rounding with an exact satisfaction check.
 *
 * Conventions shared by every entry point
 *   - Boolean variables have ids 0..n_bool-1; atom i has id n_bool + i.
 *     A literal is 2*id + neg.  Boolean value -1 means TRUE (Cor. xWFE).
 *   - Restart-minor device layout, FP32: a[n_bool][R], b[n_real][R],
 *     w[n_cons][R] and h[n_cons][R] indexed by the constraint's id (the order of
 *     fsmt_add_constraint), grad_a[n_bool][R], grad_b[n_real][R].
 *   - "device" pointers are CUDA device memory owned by the caller; the library
 *     never frees them.  "host" pointers are ordinary host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device entry points enqueue work on it and return without synchronising,
 *     unless stated otherwise.
 *   - Every function returns an fsmt_status; nothing throws across the ABI.
 *     On failure fsmt_last_error() returns a message (thread-local).
 *   - fsmt_problem and fsmt_compiled are owned by the library; release them
 *     with fsmt_free_problem / fsmt_free_compiled.
 */
#ifndef FSMT_H
#define FSMT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsmt_problem fsmt_problem;
typedef struct fsmt_compiled fsmt_compiled;

typedef enum {
  FSMT_OK = 0,
  FSMT_EINVAL = -1,   /* invalid argument or unsupported input */
  FSMT_ENOMEM = -2,   /* host or device allocation failed */
  FSMT_ECUDA = -3,    /* a CUDA runtime call or launch failed */
  FSMT_ETIMEOUT = -4, /* a bounded device wait gave up: the persistent stage kernel's
                         grid barrier (fsmt_solve_stage_host) */
  FSMT_ENAN = -5,     /* non-finite state detected (fsmt_solve_stage_host; device calls
                         mark it per restart in n_unsat instead, see fsmt_round_check) */
  FSMT_ESTATE = -6    /* call out of order (e.g. device call before fsmt_upload) */
} fsmt_status;

/* atom relations: sum_j coef_j y_j  rel  q0 (Results "Satisfiability Modulo Theories").
 * An equality (FSMT_EQ) has probability 0 under Gaussian smoothing, so it is accepted
 * only as the positive literal of a unit constraint that the projection enforces
 * (fsmt_compile with FSMT_UNIT_PROJECT); see fsmt_compile and fsmt_repair_equalities. */
enum { FSMT_LE = 0, FSMT_LT = 1, FSMT_GE = 2, FSMT_GT = 3, FSMT_EQ = 4 };

/* constraint kinds (the Boolean function of the literals' truth values)
 *   OR      at least one literal true
 *   XOR     an odd number of literals true (parity, Methods "Random Hybrid")
 *   CARD_LE at most param literals true (cardinality, Methods "Random Hybrid")
 *   NAE     not all literals equal (Methods "Random Hybrid")
 *   MUX     param = b selectors followed by 2^b data literals; the value is the
 *           data literal at index sum_i 2^i [selector i true]
 *   NEQ_OR  param = P pairs: true if a pair (l_2t, l_2t+1) differs or one of the
 *           remaining literals is true (Methods "Scheduling": worker-bit XORs
 *           OR'ed with atoms) */
enum { FSMT_OR = 0, FSMT_XOR = 1, FSMT_CARD_LE = 2, FSMT_NAE = 3, FSMT_MUX = 4, FSMT_NEQ_OR = 5 };

/* what happens to unit atomic constraints (one atom literal, no Boolean; Prop. QP) */
enum { FSMT_UNIT_PROJECT = 0, /* enforced by the projection, left out of C_sigma */
       FSMT_UNIT_SOFT = 1 };  /* kept in C_sigma like any other constraint */

typedef struct {
  int32_t n_bool, n_real, n_atoms, n_cons;
  int32_t n_obj_cons;    /* constraints that enter C_sigma */
  int64_t n_nodes;       /* decision nodes over all constraints */
  int64_t n_obj_nodes;   /* decision nodes of the constraints in C_sigma */
  int32_t max_nodes;     /* largest diagram among the constraints in C_sigma */
  int32_t n_halfspaces;  /* multi-variable unit atoms handled by the projection */
  int32_t n_components;  /* blocks of reals coupled by those half-spaces */
  int32_t n_free_reals;  /* reals with a box constraint only */
  int64_t atom_nnz;      /* nonzero coefficients over all atoms */
  int32_t fused_ok;      /* 1 if the fused kernels accept this instance */
  int32_t n_chunks;      /* chunks of the chunked forward/adjoint kernel (0: warp-per-constraint kernel) */
  int32_t jit_shapes;    /* diagram shapes given run-time generated code at fsmt_upload (0: none) */
  int32_t empty_boxes;   /* reals whose FP32 box is empty after unit-atom tightening (lo > hi): their
                            unit atoms admit no FP32 value (contradictory, or pinning the real to a
                            value FP32 cannot represent), so no restart can pass the exact check */
  int32_t proj_shapes;   /* shapes of blocks of coupled reals given run-time generated projection routines at
                            fsmt_upload (0: none; the generic projection loop serves every block) */
} fsmt_info;

/* One way to run the forward (+ adjoint) pass of C_sigma on an instance at R
 * restarts (fsmt_launch_configs, fsmt_select_config, fsmt_autotune).  The
 * paper fixes none of this: it is the kernel's tile (restarts per lane) and
 * work split (warps per CTA, which kernel, whether a chunk's reals are staged
 * in shared memory). */
enum { FSMT_VARIANT_WARP = 0,     /* one warp per constraint */
       FSMT_VARIANT_CHUNKED = 1,  /* chunked kernel compiled ahead of time (generic diagram pass) */
       FSMT_VARIANT_JIT = 2,      /* chunked kernel with run-time generated per-shape routines */
       FSMT_VARIANT_WIDE = 3 };   /* the same without the generic pass: every constraint has a routine */
typedef struct {
  int32_t variant;         /* FSMT_VARIANT_* */
  int32_t restarts_per_lane;
  int32_t staged_reals;    /* reals of a chunk staged in shared memory per restart tile (0: none) */
  int32_t warps;           /* per CTA */
  int64_t smem_bytes;      /* dynamic shared memory per CTA */
  float ms;                /* fsmt_autotune: measured time of one forward + adjoint (else 0) */
  int32_t reserved;
} fsmt_launch_config;

/* ---------------------------------------------------------------- problem --
 * Builds the constraint set C of Alg. 1 / Alg. 2 (Results "Satisfiability
 * Modulo Theories": F is the conjunction of constraints over Booleans x and
 * reals y; atoms are linear relations, Results "Walsh-Fourier Expansions"). */

/* Creates an empty problem with n_bool >= 0 Booleans and n_real >= 0 reals,
 * all reals unbounded.  EINVAL on negative sizes, ENOMEM on allocation failure. */
fsmt_status fsmt_problem_create(int32_t n_bool, int32_t n_real, fsmt_problem** out);

/* Box bounds lo <= y_j <= hi for real j (+-INFINITY allowed).  Part of the
 * feasible set D of Def. Projection.  EINVAL if j is out of range, lo > hi or
 * a bound is NaN. */
fsmt_status fsmt_set_real_bounds(fsmt_problem* p, int32_t j, double lo, double hi);

/* Adds the atom sum_{t<nnz} coef[t] * y_{var[t]}  rel  q0 (host arrays of length
 * nnz >= 1) and writes its atom index (0-based, its literal id is n_bool + index)
 * to *atom_id_out.  EINVAL if a var is out of range or repeated, a coefficient is
 * 0 or |coef| >= 2^24, |q0| >= 2^53, or rel is not one of FSMT_LE..FSMT_EQ.
 * (The bounds make every coefficient exact in FP32 and q0 exact in FP64, which
 * the exact check relies on.) */
fsmt_status fsmt_add_atom(fsmt_problem* p, int32_t nnz, const int32_t* var, const int64_t* coef,
                          int64_t q0, int32_t rel, int32_t* atom_id_out);

/* Bulk form: count atoms in CSR form (host arrays): atom t has nonzeros
 * ptr[t]..ptr[t+1]-1 of var/coef, right-hand side q0[t], relation rel[t].
 * Same validation as fsmt_add_atom; on error nothing is added. */
fsmt_status fsmt_add_atoms(fsmt_problem* p, int32_t count, const int64_t* ptr, const int32_t* var,
                           const int64_t* coef, const int64_t* q0, const int8_t* rel);

/* Adds a constraint of the given kind over nlits literals (host array).  Its
 * constraint id is the number of constraints added before it.  EINVAL if a
 * literal names an unknown variable/atom, a variable or atom appears twice, the
 * kind is unknown, or param does not fit the kind (CARD_LE: param >= 0; MUX:
 * nlits == param + 2^param with 1 <= param <= 16; NEQ_OR: 0 <= 2*param <= nlits). */
fsmt_status fsmt_add_constraint(fsmt_problem* p, int32_t kind, int32_t nlits, const int32_t* lits,
                                int32_t param);

/* Bulk form: count constraints in CSR form (host arrays): constraint t has kind
 * kind[t], parameter param[t] and literals lits[ptr[t]..ptr[t+1]-1].  On error
 * nothing is added. */
fsmt_status fsmt_add_constraints(fsmt_problem* p, int32_t count, const int8_t* kind, const int32_t* param,
                                 const int64_t* ptr, const int32_t* lits);

void fsmt_free_problem(fsmt_problem* p);

/* Exact check of Alg. 1 (rounded assignment; Thm. Soundness) on the host:
 * x[n_bool] holds +-1 (-1 = TRUE), y[n_real] the reals.  Every atom is decided
 * exactly (y is taken as the exact rational value of each double).  Writes 1 to
 * *sat_out if every constraint holds, else 0 and the id of the first violated
 * constraint to *first_violated_out (-1 when satisfied).  EINVAL on NULL
 * pointers or an x entry other than +-1. */
fsmt_status fsmt_verify_exact(const fsmt_problem* p, const int8_t* x, const double* y,
                              int32_t* sat_out, int32_t* first_violated_out);

/* Exact repair of reals y[n_real] (host, in place) so that every projected equality
 * unit atom holds exactly, before fsmt_verify_exact: the projection leaves a point on
 * a hyperplane only within FP32 rounding.  In constraint order, an equality that does
 * not already hold is solved for its pivot -- the last of its reals with coefficient
 * +-1 that no earlier equality used as pivot -- as y_p = (q0 - sum_{j != p} q_j y_j) / q_p,
 * computed exactly.  Writes 1 to *ok_out when every equality then holds exactly, else 0
 * (an equality with no such real, a pivot value that a double cannot hold exactly, or
 * a later pivot that broke an earlier equality); y is written either way.  Problems
 * without equalities leave y unchanged with *ok_out = 1.  EINVAL on NULL pointers. */
fsmt_status fsmt_repair_equalities(const fsmt_problem* p, double* y, int32_t* ok_out);

/* --------------------------------------------------------------- compile --
 * Compiles every constraint to a reduced ordered xBDD (Def. xBDD: atoms are
 * propositional inputs, no LP pruning; Suppl. Note "Decision Diagrams"), variable
 * order = order of first occurrence in the literal list, flattened in topological
 * order with the TRUE / FALSE terminals last.  With FSMT_UNIT_PROJECT, unit atomic
 * constraints leave the objective: single-variable ones tighten the box (bounds
 * rounded inward to FP32 so that a clamped value satisfies the atom exactly),
 * multi-variable ones become half-spaces of the projection (Prop. QP).  A
 * single-variable equality pins its real (both bounds rounded inward: an empty box
 * when FP32 cannot hold the value); a multi-variable equality becomes a hyperplane of
 * the projection (Dykstra's multiplier unclamped; the polish returns points to it
 * within the FP32 band of an n-term dot product), and the exact check on the device
 * counts it as holding within the polish margin 2^-16 (|q0| + sum |q_j y_j|), a candidate
 * filter for fsmt_repair_equalities and fsmt_verify_exact on the host.  The
 * problem may be freed afterwards.  EINVAL if an equality atom appears anywhere but
 * as the positive literal of a unit constraint under FSMT_UNIT_PROJECT, if a diagram has
 * more than 65,533
 * decision nodes, the total exceeds 2^31 - 1 nodes, or a block of reals coupled
 * by half-spaces needs more than one CTA's shared memory in the projection:
 * 4 * ((2 nv + nh) * 32 + (nh + 1) + 2 nnz + 2 nh + 2 nv) bytes > 225 KB for a block of
 * nv reals, nh half-spaces and nnz nonzeros (a chain of some 500 reals fits). */
fsmt_status fsmt_compile(const fsmt_problem* p, int32_t unit_policy, fsmt_compiled** out);

fsmt_status fsmt_compiled_info(const fsmt_compiled* c, fsmt_info* out);

/* Copies the flattened diagrams out for inspection (host arrays; any may be NULL):
 * con_ptr[n_cons+1] node offsets in schedule order (constraints of C_sigma first),
 * con_id[n_cons] the constraint id at each schedule position, con_root[n_cons] the
 * root index (0, or V / V+1 for a constant diagram with V = 0 nodes),
 * label[n_nodes] the variable or atom id tested by each node, hi/lo[n_nodes] the
 * child indices relative to the constraint's first node (V = TRUE, V+1 = FALSE). */
fsmt_status fsmt_get_diagrams(const fsmt_compiled* c, int32_t* con_ptr, int32_t* con_id, uint8_t* con_root,
                              int32_t* label, uint16_t* hi, uint16_t* lo);

/* The FP32 box of the reals after unit-atom tightening (host arrays [n_real]). */
fsmt_status fsmt_get_bounds(const fsmt_compiled* c, float* lo, float* hi);

/* Copies the compiled arrays to the current CUDA device (library-owned device
 * memory, freed by fsmt_free_compiled).  Must precede every device entry point.
 * Synchronises the stream.  ENOMEM / ECUDA on failure. */
fsmt_status fsmt_upload(fsmt_compiled* c, void* stream);

void fsmt_free_compiled(fsmt_compiled* c);

/* ---------------------------------------------------- relaxed objective --
 * fsmt_forward: Alg. 3 for every constraint of C_sigma and every restart, with
 * the literal probabilities of Alg. 1 (p = (1-a)/2 for Booleans, Eq. rounding;
 * p = erfc(z / (sqrt(2) sigma ||q||)) / 2 for atoms, z = q.b - q0, Eq. sampling;
 * sigma = 0 is the unsmoothed indicator).  Device inputs a[n_bool][R],
 * b[n_real][R], w[n_cons][R]; outputs (device, each may be NULL):
 * cop[n_cons][R] (COP of each constraint of C_sigma; other rows untouched) and
 * obj[R] = C_sigma (overwritten).  R >= 1, sigma >= 0.  One fused kernel, no
 * scratch memory.  EINVAL on bad sizes or an instance the fused kernel rejects
 * (fsmt_info.fused_ok == 0); ESTATE before fsmt_upload; ECUDA on launch errors. */
fsmt_status fsmt_forward(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                         const float* b, float* cop, float* obj, void* stream);

/* fsmt_adjoint: forward plus the adjoint sweep of Alg. 4 in one kernel, returning
 * the exact gradient of C_sigma (Thm. backward; sign as in its proof):
 *   grad_a[i] = sum_c w_c sum_{v tests i} m_td[v] (m_bu[hi v] - m_bu[lo v])
 *   grad_b[j] = sum_c w_c sum_{atom nodes v} m_td[v] (m_bu[hi]-m_bu[lo]) dd/db_j
 * with dd/db_j = sqrt(2) q_j / (sqrt(pi) sigma ||q||) exp(-z^2 / (2 sigma^2 ||q||^2)).
 * grad_a[n_bool][R] and grad_b[n_real][R] (device) are overwritten; obj[R] and
 * cop[n_cons][R] as in fsmt_forward (may be NULL).  Errors as fsmt_forward. */
fsmt_status fsmt_adjoint(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                         const float* b, float* grad_a, float* grad_b, float* obj, float* cop, void* stream);

/* The configurations that can run this instance at R restarts, the default
 * first.  Writes min(cap, count) of them to out (device-free; out may be NULL
 * with cap 0 to count) and the count to *n.  ESTATE before fsmt_upload (the
 * run-time compiled kernels are known only then), EINVAL on R < 1. */
fsmt_status fsmt_launch_configs(const fsmt_compiled* c, int32_t R, fsmt_launch_config* out, int32_t cap,
                                int32_t* n);

/* Pins one of fsmt_launch_configs' configurations (matched on variant,
 * restarts_per_lane and staged_reals) for later fsmt_forward, fsmt_adjoint and
 * stages at this R; cfg NULL returns to the default.  EINVAL if it is not one
 * of them.  A stage graph captured before is re-captured. */
fsmt_status fsmt_select_config(fsmt_compiled* c, int32_t R, const fsmt_launch_config* cfg);

/* Autotuner: times every configuration of fsmt_launch_configs on the caller's
 * inputs (one warm-up and three timed forward + adjoint passes each, CUDA
 * events on `stream`) and pins the fastest as fsmt_select_config does.
 * grad_a, grad_b and obj are scratch of fsmt_adjoint's shapes, zero on return.
 * The chosen configuration, with its time, goes to *best (may be NULL).
 * Synchronises the stream.  Errors as fsmt_adjoint. */
fsmt_status fsmt_autotune(fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                          const float* b, float* grad_a, float* grad_b, float* obj, fsmt_launch_config* best,
                          void* stream);

/* Plain (unfused) form of the same two passes, for comparison: separate
 * kernels for the atom probabilities, the forward pass (which stores every
 * node's top-down message in work) and the adjoint pass (which reads it back).
 * work is a device buffer of fsmt_plain_work_floats(c, R) floats owned by the
 * caller; fsmt_adjoint_plain must see the work written by fsmt_forward_plain at
 * the same (R, sigma, w, a, b).  Outputs and errors as the fused forms. */
fsmt_status fsmt_plain_work_floats(const fsmt_compiled* c, int32_t R, int64_t* n_floats);
fsmt_status fsmt_forward_plain(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* work, float* cop, float* obj, void* stream);
fsmt_status fsmt_adjoint_plain(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* work, float* grad_a, float* grad_b, void* stream);

/* Allocation-free form of the plain pass pair (the paper has no counterpart: this
 * is a deployment convenience).  Some callers cannot call cudaMalloc at this
 * point: programs that reserve all device memory at start-up and must keep a
 * fixed footprint afterwards, and hosts whose device memory is owned by another
 * allocator (for instance a framework's caching pool) that forbids allocations
 * outside its own accounting.  For them this entry point runs fsmt_forward_plain
 * and then fsmt_adjoint_plain with their work memory taken from a fixed 64 MiB
 * array (16 Mi floats) that lives in the library's device image on every GPU
 * that loads the library, until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.  Inputs and outputs are as for the two
 * plain calls (grad_a, grad_b overwritten; cop, obj may be NULL).
 *  - Size limit: EINVAL, with a message, when fsmt_plain_work_floats(c, R) exceeds
 *    16 Mi floats; nothing is launched then.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents behind;
 *    the passes write every value they later read, so no clearing is needed.
 *    Calls that overlap on the GPU (other streams, other threads) race on the
 *    array: serialise them.
 * Errors as the plain calls. */
fsmt_status fsmt_plain_noalloc(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* grad_a, float* grad_b, float* cop, float* obj, void* stream);

/* ------------------------------------------------------------ PGD step --
 * fsmt_weight_sum: wsum[r] = sum over the constraints of C_sigma of w[c][r]
 * (device w[n_cons][R] in, device wsum[R] overwritten) -- alpha of Prop.
 * Lipschitz per restart.  Errors as above.
 *
 * fsmt_pgd_step: Eq. pg1 / pg2 and Eq. grad_map, in coordinates where the reals
 * are divided by b_scale (> 0).  Step of restart r: eta_r = eta, or, when wsum
 * is given, eta_r = eta * n_obj / wsum[r] (Thm. max_step takes eta = 1/L with L
 * proportional to the total weight; the ERWA weights grow every stage).
 * a' = a - eta_r grad_a, b' = b - eta_r b_scale^2 grad_b,
 * (a, b) <- proj_D(a', b') with D = [-1,1]^n x box x half-spaces: clamps, and for
 * each block of reals coupled by half-spaces, `sweeps` sweeps of Dykstra's
 * alternating projections (half-spaces in constraint order, then the box)
 * followed by up to `polish` passes that project each half-space q.y <= q0 with
 * q.y > q0 - m onto q.y <= q0 - 2m, m = 2^-16 (|q0| + sum |q_j y_j|), moving only
 * reals not pinned at the bound the step would cross, then clamp the box, until
 * a pass moves nothing (so the result lies in D exactly once the
 * passes settle); then
 * gnorm2[r] += sum ((a - a_new)/eta_r)^2 + sum ((b - b_new)/(b_scale eta_r))^2.
 * a, b (device, [n][R], [m][R]) are updated in place for restarts with
 * active[r] == 1 (active may be NULL = all; 0 and 2 are stopped restarts, as
 * fsmt_solve_stage writes them); gnorm2[R] (device) is accumulated,
 * so the caller zeroes it first.  eta > 0, sweeps >= 0, polish >= 0; wsum (device
 * [R]) may be NULL.  Errors as above. */
fsmt_status fsmt_weight_sum(const fsmt_compiled* c, int32_t R, const float* w, float* wsum, void* stream);
fsmt_status fsmt_pgd_step(const fsmt_compiled* c, int32_t R, float eta, float b_scale, int32_t sweeps,
                          int32_t polish, float* a, float* b, const float* grad_a, const float* grad_b,
                          const float* wsum, float* gnorm2, const uint8_t* active, void* stream);

/* ------------------------------------------------------- round + check --
 * Alg. 1's rounding x = sgn(a) (x_i = TRUE = -1 iff a_i < 0), y = b, and an exact
 * check of every constraint (each atom's sign decided exactly in fixed point),
 * followed by Alg. 2's ERWA update: u_c = [c violated], h_c <- rho h_c + u_c,
 * n_unsat[r] = sum_c u_c, and if update_w != 0: w_c <- w_c gamma^h_c, h_c <- 1.
 * Device arrays: a, b inputs; n_unsat[R] output (overwritten); x[n_bool][R] (int8,
 * may be NULL), violated[n_cons][R] (uint8, may be NULL), w and h [n_cons][R]
 * (may both be NULL to skip ERWA); wsum[R] (may be NULL): the restarts' total
 * weights over C_sigma as fsmt_weight_sum gave them for the stage.  With wsum, a
 * restart whose mean weight wsum[r] / |C_sigma| exceeds 2^32 has its updated
 * weights multiplied by 2^-32 (exact): ERWA grows every weight geometrically and a
 * step normalised by the total weight (fsmt_pgd_step with wsum) does not see a
 * common factor, so this keeps long schedules inside FP32 (NULL: Alg. 2 as
 * printed).  A restart whose point has a non-finite coordinate that the check
 * reads gets bit 31 of n_unsat[r] set (the value is negative; the low bits still
 * count its violated constraints); the call itself does not synchronise and
 * returns FSMT_OK.  Errors as above. */
fsmt_status fsmt_round_check(const fsmt_compiled* c, int32_t R, const float* a, const float* b, int8_t* x,
                             uint8_t* violated, int32_t* n_unsat, float* w, float* h, float rho, float gamma,
                             int32_t update_w, const float* wsum, void* stream);

/* Alg. 1's rounding alone: x[i][r] = -1 (TRUE) if a[i][r] < 0, else +1, for every
 * Boolean and restart (device a[n_bool][R] in, device int8 x[n_bool][R] out).  The
 * values fsmt_round_check writes to its x.  Errors as above. */
fsmt_status fsmt_round(const fsmt_compiled* c, int32_t R, const float* a, int8_t* x, void* stream);

/* The epsilon rule of Eq. critical after one PGD iteration, per restart, as the
 * stage applies it: for every restart with active[r] == 1, iters[r] += 1; then a
 * non-finite gnorm2[r] stops it with active[r] = 2 and sets bit 0 of ctl[1];
 * gnorm2[r] <= eps^2 stops it with active[r] = 0.  ctl[0] is overwritten with the
 * number of restarts still active (1).  Device arrays gnorm2[R], active[R],
 * iters[R], ctl[2]; eps >= 0.  For callers that drive the iterations themselves
 * (the plain form); fsmt_solve_stage does this inside its graph.  Errors as above. */
fsmt_status fsmt_converge(const fsmt_compiled* c, int32_t R, float eps, const float* gnorm2, uint8_t* active,
                          int32_t* iters, int32_t* ctl, void* stream);

/* Sets bit 31 of n_unsat[r] (device int32[R]) for every restart with active[r] == 2
 * (device uint8[R]): a restart stopped on a non-finite ||g||^2, marked at the check
 * as fsmt_solve_stage marks it.  Call it after fsmt_round_check.  Errors as above. */
fsmt_status fsmt_mark_nonfinite(const fsmt_compiled* c, int32_t R, const uint8_t* active, int32_t* n_unsat,
                                void* stream);

/* ------------------------------------------------------- one sigma stage --
 * One stage of Alg. 2 for all restarts: wsum from fsmt_weight_sum, then up to
 * t_max iterations of
 * [fused forward + adjoint -> PGD step + projection -> ||g||^2 test] with the
 * epsilon rule of Eq. critical applied per restart (an iteration's update is
 * applied, then a restart with ||g||^2 <= eps^2 stops for the rest of the
 * stage), then round + check + ERWA as fsmt_round_check (with the stage's wsum
 * when the step is normalised).  All buffers are caller
 * owned device memory; grad_a/grad_b are work buffers that the stage leaves at
 * zero.  ctl is a device int32[4] control block (ctl[0] = restarts still
 * iterating, ctl[1] = error bits: 1 = non-finite ||g||^2 seen, 4 = the persistent
 * kernel gave up waiting at a grid barrier; ctl[2..3] = that kernel's grid barrier,
 * reset by the stage itself).  With use_graph != 0 the launches of a stage are
 * captured once in a CUDA graph (per compiled object and buffer set) and replayed;
 * the scalar parameters travel in params (a device float[16] buffer), so one graph
 * serves every sigma.
 *
 * With persistent != 0, and when fsmt_stage_form reports the persistent forms for
 * R, Alg. 1's loop body runs fused in one persistent cooperative kernel (forward +
 * adjoint over C_sigma, grid barrier, PGD step + projection of every real and
 * Boolean, grid barrier whose last CTA applies the epsilon test; the forward +
 * adjoint phase is the configuration chosen by fsmt_autotune / fsmt_select_config):
 * persistent = 1 runs all t_max iterations in ONE launch (a stage is five launches
 * -- parameters, stage start, weight sum, iteration start, the stage kernel -- before
 * the round check); persistent = 2 launches the same kernel once per iteration (no
 * loop inside it, so that the forward + adjoint phase is compiled as in its own
 * kernel).  Each barrier waits at most 5 s for the slowest CTA (the environment
 * variable FSMT_STAGE_BARRIER_NS, read at each launch or graph capture, sets another
 * limit in ns); a kernel that gave up sets bit 4 of ctl[1] and ends, and
 * fsmt_solve_stage_host returns FSMT_ETIMEOUT.  Results equal the separate-launch
 * form's up to the order of floating-point atomic additions.  One stage at a time
 * per state (the barrier lives in its ctl). */
typedef struct {
  int32_t R;
  float* a;        /* [n_bool][R] */
  float* b;        /* [n_real][R] */
  float* w;        /* [n_cons][R] */
  float* h;        /* [n_cons][R] */
  float* grad_a;   /* [n_bool][R] work, zero on entry */
  float* grad_b;   /* [n_real][R] work, zero on entry */
  float* obj;      /* [R] C_sigma at the start of the last iteration run */
  float* gnorm2;   /* [R] ||g||^2 of the last iteration run */
  uint8_t* active; /* [R] 1 iterating, 0 stopped by the epsilon test, 2 stopped on a
                      non-finite ||g||^2 (its n_unsat gets bit 31 at the check) */
  int32_t* iters;  /* [R] iterations run in this stage */
  int32_t* n_unsat;/* [R] */
  int32_t* ctl;    /* [4] */
  float* params;   /* [16] */
  float* wsum;     /* [R] total weight of C_sigma per restart, computed at stage start */
} fsmt_state;

typedef struct {
  float sigma, eta, b_scale, eps;
  int32_t t_max, sweeps;
  float rho, gamma;
  int32_t update_w;
  int32_t use_graph;
  int32_t polish;        /* feasibility passes after Dykstra (see fsmt_pgd_step) */
  int32_t normalize_eta; /* 1: eta_r = eta * n_obj / wsum[r] */
  int32_t persistent;    /* 0: separate launches per iteration; 1: one persistent kernel for the
                            stage; 2: one persistent kernel per iteration (where available) */
} fsmt_stage_config;

fsmt_status fsmt_solve_stage(fsmt_compiled* c, const fsmt_stage_config* cfg, fsmt_state* s, void* stream);

/* Whether fsmt_solve_stage with persistent = 1 or 2 runs the persistent kernel at R
 * restarts (1) or falls back to separate launches per iteration (0): the
 * persistent forms need the run-time compiled module (NVRTC; it holds a stage kernel
 * for each run-time compiled chunked configuration and for the warp-per-constraint
 * one, but none for the ahead-of-time chunked kernel), at most 1e11 node visits per
 * iteration, and the largest block of coupled reals within one CTA's shared memory.
 * The stage kernels are compiled at the first call that needs them (this one, or the
 * first persistent fsmt_solve_stage), not at fsmt_upload: make that call before any
 * stream capture of your own.  ESTATE before fsmt_upload. */
fsmt_status fsmt_stage_form(fsmt_compiled* c, int32_t R, int32_t* persistent_out);

/* Per-phase device timestamps of the persistent stage kernel, for profiling (no
 * counterpart in the paper).  With trace != NULL every later persistent stage of c
 * writes global-timer readings (ns) into the caller's device buffer trace, which
 * holds 1 + 2 t_max uint64: [0] the kernel's start, [1 + 2 i] the moment the last CTA
 * finished iteration i's forward + adjoint phase, [2 + 2 i] the moment the last CTA
 * finished its PGD phase and the epsilon test ran; entries of iterations not run keep
 * their old values.  NULL turns it off.  Stages captured in a CUDA graph keep the
 * buffer they were captured with (the graph is keyed by it).  EINVAL for a NULL c. */
fsmt_status fsmt_stage_trace(fsmt_compiled* c, uint64_t* trace);

/* The same stage driven from HOST buffers: copies a[n_bool*R] and b[n_real*R]
 * (host, ideally pinned) into the device state, runs fsmt_solve_stage, and
 * copies n_unsat[R] and obj[R] back to host buffers (may be NULL), and ctl[1].
 * Synchronises the stream before returning.  Errors as fsmt_solve_stage,
 * FSMT_ETIMEOUT when the persistent kernel gave up at a grid barrier, and FSMT_ENAN when
 * n_unsat is copied back and some restart's point is non-finite (bit 31 of its
 * n_unsat, as fsmt_round_check marks it; the outputs are still written). */
fsmt_status fsmt_solve_stage_host(fsmt_compiled* c, const fsmt_stage_config* cfg, fsmt_state* s,
                                  const float* a_host, const float* b_host, int32_t* n_unsat_host,
                                  float* obj_host, void* stream);

/* Thread-local message describing the last error ("" if none). */
const char* fsmt_last_error(void);

/* Library version string. */
const char* fsmt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSMT_H */
