"""The run-time code generator of the chunked kernel, executed on the host.

The generator (fsmt_jit.cpp) writes Alg. 3 and Alg. 4 for one diagram shape as
straight-line code.  Here its source is compiled with g++ together with a small
host stand-in for the handful of device names the routine uses (plain float
arithmetic, a non-atomic add), run on literal probabilities laid out as the kernel's
shared-memory slot rows, and compared with the FP64 oracle's COP and dCOP/dp taken
from their definition (sum over all assignments; the oracle's message passing for the
18-literal scheduling shape).  This checks the generated arithmetic -- message
passing, constant folding, grouped nodes, negated literals, the literal-list
addressing -- with no GPU.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import bdd, cop
from workloads import instances as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_22877_b300", "csrc")
CUDA = "/usr/local/cuda"
SLOT_FLOATS = 64        # floats per slot row: [restart k < 2][lane < 32]
MAX_JIT_NODES = 48      # the generator's largest shape

HARNESS = r'''
#include <cstring>
#include "fsmt_jit.cpp"
namespace fsmt { void set_error(const std::string&) {} }
extern "C" long proj_src(int rank, int nv, int nh, const int32_t* hs_ptr, const int32_t* lvar, const float* coef,
                         const float* inv_qq, const uint8_t* eq, char* out, long cap) {
  fsmt::Compiled C;
  C.comp_var_ptr = {0, nv};
  C.comp_hs_ptr = {0, nh};
  C.hs_ptr.assign(hs_ptr, hs_ptr + nh + 1);
  C.hs_lvar.assign(lvar, lvar + hs_ptr[nh]);
  C.hs_coef.assign(coef, coef + hs_ptr[nh]);
  C.hs_inv_qq.assign(inv_qq, inv_qq + nh);
  C.hs_eq.assign(eq, eq + nh);
  const std::string s = fsmt::proj_routine(rank, C, 0);
  if ((long)s.size() + 1 > cap) return -1;
  std::memcpy(out, s.c_str(), s.size() + 1);
  return (long)s.size();
}
extern "C" long shape_src(int rank, int V, const uint16_t* hi, const uint16_t* lo, const uint16_t* grp,
                          char* out, long cap) {
  const std::string s = fsmt::shape_routine(rank, V, hi, lo, grp);
  if ((long)s.size() + 1 > cap) return -1;
  std::memcpy(out, s.c_str(), s.size() + 1);
  return (long)s.size();
}
'''

SHIM = r'''
#include <cmath>
#include <cstdint>
#define __device__
#define __forceinline__ inline
struct uint4 { unsigned x, y, z, w; };
template <int R> struct Pack { float v[R]; };
static inline float vadd(float a, float b) { return a + b; }
static inline float vsub(float a, float b) { return a - b; }
static inline float vmul(float a, float b) { return a * b; }
static inline float vfma(float a, float b, float c) { return std::fma(a, b, c); }
static inline float atomicAdd(float* p, float v) { const float o = *p; *p = o + v; return o; }
'''


def _gxx():
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    return gxx


@pytest.fixture(scope="module")
def generator(tmp_path_factory):
    """The product's shape-routine generator, built from its source into a host library."""
    from paper_2603_22877_b300 import build as B
    B.write_jit_sources()
    d = tmp_path_factory.mktemp("jitgen")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "harness.so"
    cmd = [_gxx(), "-std=c++17", "-O1", "-shared", "-fPIC", f"-I{CSRC}", f"-I{ROOT}/include", f"-I{CUDA}/include",
           str(src), "-o", str(so), f"-L{CUDA}/lib64", "-lcudart", f"-Wl,-rpath,{CUDA}/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(str(so))
    lib.shape_src.restype = C.c_long
    lib.proj_src.restype = C.c_long

    def source(rank, hi, lo, grp):
        buf = C.create_string_buffer(1 << 20)
        arrs = [np.ascontiguousarray(x, np.uint16) for x in (hi, lo, grp)]
        n = lib.shape_src(rank, len(hi), *[a.ctypes.data_as(C.c_void_p) for a in arrs], buf, 1 << 20)
        assert n > 0
        return buf.value.decode()
    source.lib = lib
    return source, d


def literal_shape(kind, param, lits):
    """The oracle's diagram in literal space (a node testing a negated literal has its
    children swapped; hi = the literal holds), its groups (first node testing the same
    variable) and the variables in order of their group's first node."""
    M, r = bdd.build(kind, param, lits)
    var, hi, lo, root = bdd.flatten(M, r, lits)
    V = len(var)
    neg = {int(l) >> 1: bool(int(l) & 1) for l in lits}
    first, order = {}, []
    h, l_, g = [], [], []
    for v in range(V):
        a, b = hi[v], lo[v]
        if neg[var[v]]:
            a, b = b, a
        h.append(a)
        l_.append(b)
        if var[v] not in first:
            first[var[v]] = v
            order.append(var[v])
        g.append(first[var[v]])
    return V, h, l_, g, order, neg


def test_generated_routines_match_the_definition(generator):
    source, d = generator
    rng = np.random.default_rng(21)
    cases = []
    for kind, L_, params in ((W.OR, 5, [0]), (W.XOR, 4, [0]), (W.NAE, 5, [0]), (W.CARD_LE, 6, [0, 2, 4]),
                             (W.MUX, 6, [2]), (W.MUX, 3, [1]), (W.NEQ_OR, 6, [2]), (W.NEQ_OR, 7, [3]),
                             (W.NEQ_OR, 18, [8])):
        for param in params:
            for _ in range(3):
                ids = rng.choice(40, L_, replace=False)
                lits = [2 * int(i) + int(rng.integers(2)) for i in ids]
                V, hi, lo, grp, order, neg = literal_shape(kind, param, lits)
                if 1 <= V <= MAX_JIT_NODES:
                    cases.append((kind, param, lits, V, hi, lo, grp, order, neg))
    assert len(cases) >= 25
    # one translation unit with every routine and a runner per routine
    body = [SHIM]
    for k, (_, _, _, V, hi, lo, grp, _, _) in enumerate(cases, start=1):
        body.append(source(k, hi, lo, grp))
        body.append(f'extern "C" void run_{k}(int adj, const unsigned* sl, const float* s_p, float* s_g, '
                    f'const float* w, float* out) {{\n  Pack<2> wc{{{{w[0], w[1]}}}}, cp{{}};\n'
                    f'  if (adj) shape_{k}<true, 2>(sl, s_p, s_g, 0, wc, cp); '
                    f'else shape_{k}<false, 2>(sl, s_p, s_g, 0, wc, cp);\n  out[0] = cp.v[0]; out[1] = cp.v[1];\n}}\n')
    src = d / "routines.cpp"
    src.write_text("\n".join(body))
    so = d / "routines.so"
    r = subprocess.run([_gxx(), "-std=c++17", "-O1", "-ffp-contract=off", "-Wno-unknown-pragmas", "-shared", "-fPIC",
                        str(src), "-o", str(so)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[:4000]
    lib = C.CDLL(str(so))
    for k, (kind, param, lits, V, hi, lo, grp, order, neg) in enumerate(cases, start=1):
        n_slots = len(order)
        sl = np.zeros(((n_slots + 3) // 4) * 4, np.uint32)
        sl[:n_slots] = np.arange(n_slots) * SLOT_FLOATS * 4          # byte offsets of the slot rows
        ptrue = {i: rng.uniform(0.02, 0.98, 2) for i in order}       # P[variable TRUE], two restarts
        s_p = np.zeros(n_slots * SLOT_FLOATS, np.float32)
        for j, i in enumerate(order):
            for r_ in range(2):
                s_p[j * SLOT_FLOATS + 32 * r_] = 1.0 - ptrue[i][r_] if neg[i] else ptrue[i][r_]
        w = np.array([1.5, 0.25], np.float32)
        if len(lits) <= 10:                                          # the definition itself
            want = np.asarray(cop.cop_definition(kind, param, lits, ptrue), np.float64)
            dwant = cop.dcop_definition(kind, param, lits, ptrue)
        else:  # 2^18 assignments are slow in Python: the oracle's Alg. 3 / Alg. 4, pinned to it
            M, r = bdd.build(kind, param, lits)
            diagram = bdd.flatten(M, r, lits)
            m_td, want = cop.forward(diagram, ptrue, 2)
            _, dwant = cop.backward(diagram, ptrue, m_td, 2)
        for adj in (0, 1):
            s_g = np.zeros_like(s_p)
            out = np.zeros(2, np.float32)
            getattr(lib, f"run_{k}")(adj, sl.ctypes.data_as(C.c_void_p), s_p.ctypes.data_as(C.c_void_p),
                                     s_g.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p),
                                     out.ctypes.data_as(C.c_void_p))
            np.testing.assert_allclose(out, want, atol=2e-6, err_msg=f"COP kind {kind} lits {lits}")
            if not adj:
                assert not s_g.any()
                continue
            for j, i in enumerate(order):                            # w * dCOP/dq, q the literal's probability
                for r_ in range(2):
                    g = float(dwant[i][r_]) * (-1.0 if neg[i] else 1.0) * float(w[r_])
                    assert abs(s_g[j * SLOT_FLOATS + 32 * r_] - g) <= 2e-5 * max(1.0, abs(g)), (kind, lits, i, r_)


PROJ_SHIM = r'''
#include <cmath>
#include <cstddef>
#define __device__
#define __forceinline__ inline
#define __restrict__
static inline float fmaf_(float a, float b, float c) { return std::fma(a, b, c); }
#define fmaf fmaf_
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static const float kPolishMargin = 1.52587890625e-05f;
static inline float proj_dot(float cf, float x, float th, float dot) { return fmaf(cf, fmaf(th, cf, x), dot); }
static inline float proj_tn(float dot, float iq) { return __fmul_rn(std::fmax(dot, 0.f), iq); }
static inline float proj_tn_eq(float dot, float iq) { return __fmul_rn(dot, iq); }
static inline float proj_eq_band(int n, float mag) { return (float)(n + 4) * std::fma(5.9604645e-8f, mag, 1e-38f); }
static inline float proj_box(float& x, float p, float lo, float hi) {
  const float yv = __fadd_rn(x, p); const float xn = std::fmin(std::fmax(yv, lo), hi); x = xn; return __fsub_rn(yv, xn);
}
static inline float fminf_(float a, float b) { return std::fmin(a, b); }
static inline float fmaxf_(float a, float b) { return std::fmax(a, b); }
static inline float fabsf_(float a) { return std::fabs(a); }
#define fminf fminf_
#define fmaxf fmaxf_
#define fabsf fabsf_
'''


def test_generated_projection_routines_match_the_oracle(generator):
    """The projection routines generated for frequent block shapes (fsmt_jit.cpp,
    proj_routine: Dykstra's sweeps and the feasibility polish of Prop. QP's reading,
    straight-line over registers) compiled for the host and run on precedence chains
    of job-shop instances (blocks of 3, 5 and 9 reals, and a no-wait chain of 6 whose
    links are equalities' hyperplanes), against the oracle's
    Domain.project_b in FP64: the same end points up to FP32 rounding, and the
    squared step lengths summed as ||g||^2 (Eq. grad_map)."""
    from oracle import pgd
    source, d = generator
    lib = source.lib
    rng = np.random.default_rng(8)
    body = [PROJ_SHIM]
    cases = []
    for k, (jobs, machines, no_wait) in enumerate(((4, 3, 0), (5, 5, 0), (3, 9, 0), (4, 6, 4)), start=1):
        inst = W.jobshop(1002, jobs, machines, no_wait=no_wait)
        dom = pgd.Domain(inst)
        hs = dom.halfspaces[:machines - 1]                  # the first job's chain
        eqf = dom.eq[:machines - 1]                         # no-wait: every link an equality
        order = []
        for var, q, q0 in hs:
            for j in var:
                if int(j) not in order:
                    order.append(int(j))
        loc = {j: t for t, j in enumerate(order)}
        ptr, lv, cf, iq = [0], [], [], []
        for var, q, q0 in hs:
            lv += [loc[int(j)] for j in var]
            cf += [float(c) for c in q]
            ptr.append(len(lv))
            iq.append(np.float32(1.0 / float((np.asarray(q) ** 2).sum())))
        arrs = [np.asarray(ptr, np.int32), np.asarray(lv, np.int32), np.asarray(cf, np.float32), np.asarray(iq, np.float32),
                np.asarray(eqf, np.uint8)]
        buf = C.create_string_buffer(1 << 20)
        assert lib.proj_src(k, len(order), len(hs), *[a.ctypes.data_as(C.c_void_p) for a in arrs], buf, 1 << 20) > 0
        body.append(buf.value.decode())
        body.append(f'extern "C" void run_{k}(const float* q0, const float* lo, const float* hi, float* b, float* gb,'
                    f' const int* cvar, float step, float inv, float* part) {{\n'
                    f'  float p = 0.f;\n  proj_{k}(q0, lo, hi, b, gb, cvar, 1, 0, step, inv, 20, 32, 1, true, p);\n'
                    f'  *part = p;\n}}\n')
        cases.append((k, inst, dom, hs, order))
    src = d / "proj.cpp"
    src.write_text("\n".join(body))
    so = d / "proj.so"
    r = subprocess.run([_gxx(), "-std=c++17", "-O1", "-ffp-contract=off", "-shared", "-fPIC", str(src), "-o", str(so)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[:4000]
    rl = C.CDLL(str(so))
    for k, inst, dom, hs, order in cases:
        n = len(order)
        q0 = np.asarray([h[2] for h in hs], np.float32)
        lo = np.asarray([dom.lo[j] for j in order], np.float32)
        hi = np.asarray([dom.hi[j] for j in order], np.float32)
        cvar = np.arange(n, dtype=np.int32)                  # restart 0 of R = 1: b[t]
        for trial in range(6):
            y0 = (inst.planted_y[order] + rng.normal(0, 4.0, n)).astype(np.float32)
            g = rng.normal(0, 1.0, n).astype(np.float32)
            step, inv = np.float32(0.5), np.float32(1.0)
            b = y0.copy()
            gb = g.copy()
            part = np.zeros(1, np.float32)
            getattr(rl, f"run_{k}")(*[a.ctypes.data_as(C.c_void_p) for a in (q0, lo, hi, b, gb, cvar)],
                                    C.c_float(step), C.c_float(inv), part.ctypes.data_as(C.c_void_p))
            assert not gb.any()                              # the gradient is cleared
            full = np.zeros((inst.n_real, 1))
            full[:, 0] = inst.planted_y
            full[order, 0] = y0.astype(np.float64) - 0.5 * g.astype(np.float64)
            # the other reals of the instance do not interact with this chain's block
            ref = dom.project_b(full, 20, 32)[order, 0]
            scale = float(np.abs(ref).max()) + 1.0
            np.testing.assert_allclose(b, ref, atol=2e-5 * scale, err_msg=f"shape {k} trial {trial}")
            want = float(((y0.astype(np.float64) - ref) ** 2).sum())
            assert abs(part[0] - want) <= 1e-4 * want + 1e-3, (part[0], want)


def test_polish_multiplies_only_by_exact_reciprocals(generator):
    """The generated polish replaces the division by qq (the free terms' squared
    coefficients) with a product only when every nonzero qq the flags can give is a
    power of two, where x / 2^k and x * 2^-k round the same real number: unit chains
    (qq in {1, 2}) and coefficients +-2 (qq in {4, 8}) multiply, coefficients (1, 3)
    (qq = 10) divide."""
    source, _ = generator
    lib = source.lib

    def src(coefs):
        arrs = [np.asarray([0, len(coefs)], np.int32), np.arange(len(coefs), dtype=np.int32),
                np.asarray(coefs, np.float32), np.asarray([1.0 / sum(c * c for c in coefs)], np.float32),
                np.zeros(1, np.uint8)]
        buf = C.create_string_buffer(1 << 16)
        assert lib.proj_src(1, len(coefs), 1, *[a.ctypes.data_as(C.c_void_p) for a in arrs], buf, 1 << 16) > 0
        return buf.value.decode()

    unit = src([1.0, -1.0])
    assert "__fdiv_rn" not in unit and "(n1 ? (n0 ? 0x1p-1f : 0x1p+0f)" in unit
    two = src([2.0, -2.0])
    assert "__fdiv_rn" not in two and "0x1p-3f" in two and "0x1p-2f" in two
    assert "__fdiv_rn" in src([1.0, 3.0])
    assert "__fdiv_rn" in src([1.0, 1.0, 1.0, 1.0, 1.0])  # more than four terms: always the division
