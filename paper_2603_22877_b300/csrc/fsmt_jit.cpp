// Run-time specialisation of the chunked forward/adjoint kernel.
//
// Most constraints of an instance share a handful of diagram shapes (in literal
// space, see build_chunks).  For each frequent shape this file writes Alg. 3 and
// Alg. 4 as straight-line CUDA over named registers -- the top-down and bottom-up
// messages never touch shared memory -- compiles it together with the chunked
// kernel (fsmt_chunked.cuh) with NVRTC for the current GPU, and loads the result.
// Constraints of other shapes take the generic path of the same kernel.  NVRTC is
// opened at run time; without it the ahead-of-time kernel is used unchanged.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "fsmt_internal.h"
#include "fsmt_jit_src.inc"  // kJitDevviewSrc, kJitChunkedSrc, kJitProjSrc, kJitStageSrc (generated by build.py)

namespace fsmt {

namespace {

struct Nvrtc {
  bool tried = false, ok = false;
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  if (n.tried) return n;
  n.tried = true;
  const char* names[] = {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"};
  void* h = nullptr;
  for (const char* nm : names)
    if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) return n;
  n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
  n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
  n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
  n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
  n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
  n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
  n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
  n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  return n;
}

// Alg. 3 / Alg. 4 for one shape, straight-line, one restart of the lane at a
// time (the RPL restarts in turn).  Node v tests a literal whose probability q
// comes from its slot; its children (hi: the literal holds) are nodes, or V
// (TRUE) / V+1 (FALSE).  Nodes testing the same literal form a group (grp = its
// first node); each pass reads a group's slot word and q from shared memory
// once, at the group's first node in that pass's order.  The messages t_v
// (Alg. 3, started at w_c instead of 1, so that t_v = w_c m_td[v]) and b_v
// (Alg. 4) live in registers, and the reverse pass sums t_v (b_hi - b_lo) over a
// group -- the group's w_c dC/dq -- and issues the group's one shared-memory
// update at its last node.  The terminals' messages are constants, and every
// operation with a constant operand is folded as the code is generated.
namespace {
struct Ex {  // a message: 0, 1, -1 or a named value
  enum Kind { ZERO, ONE, MONE, VAR } k;
  std::string n;
};
struct Emitter {
  std::ostringstream& o;
  int tmp = 0;
  std::string name(const Ex& e) const {
    return e.k == Ex::ZERO ? "zero" : e.k == Ex::ONE ? "one" : e.k == Ex::MONE ? "mone" : e.n;
  }
  Ex emit(const std::string& expr) {
    const std::string n = "e" + std::to_string(tmp++);
    o << "    const V " << n << " = " << expr << ";\n";
    return {Ex::VAR, n};
  }
  Ex neg(const Ex& x) {
    if (x.k == Ex::ZERO) return x;
    if (x.k == Ex::ONE) return {Ex::MONE, ""};
    if (x.k == Ex::MONE) return {Ex::ONE, ""};
    return emit("vsub(zero, " + x.n + ")");
  }
  Ex add(const Ex& a, const Ex& x) {
    if (x.k == Ex::ZERO) return a;
    if (a.k == Ex::ZERO) return x;
    if (x.k == Ex::MONE) return emit("vsub(" + name(a) + ", one)");
    return emit("vadd(" + name(a) + ", " + name(x) + ")");
  }
  Ex sub(const Ex& a, const Ex& x) {
    if (x.k == Ex::ZERO) return a;
    if (a.k == Ex::ZERO) return neg(x);
    if (a.k == Ex::ONE && x.k == Ex::ONE) return {Ex::ZERO, ""};
    return emit("vsub(" + name(a) + ", " + name(x) + ")");
  }
  Ex mul(const Ex& x, const Ex& y) {
    if (x.k == Ex::ZERO || y.k == Ex::ZERO) return {Ex::ZERO, ""};
    if (x.k == Ex::ONE) return y;
    if (y.k == Ex::ONE) return x;
    if (x.k == Ex::MONE) return neg(y);
    if (y.k == Ex::MONE) return neg(x);
    return emit("vmul(" + x.n + ", " + y.n + ")");
  }
  Ex fma(const Ex& x, const Ex& y, const Ex& a) {  // a + x y
    if (x.k != Ex::VAR || y.k != Ex::VAR) {
      if (x.k == Ex::ONE) return add(a, y);
      if (y.k == Ex::ONE) return add(a, x);
      if (x.k == Ex::MONE) return sub(a, y);
      if (y.k == Ex::MONE) return sub(a, x);
      return a;  // a zero factor
    }
    if (a.k == Ex::ZERO) return mul(x, y);
    return emit("vfma(" + x.n + ", " + y.n + ", " + name(a) + ")");
  }
};
}  // namespace

std::string shape_routine(int rank, int V, const uint16_t* hi, const uint16_t* lo, const uint16_t* grp) {
  std::ostringstream o;
  std::vector<int> last(V, -1), pos(V, -1);  // last node of each group; the group's place in the literal list
  int n_groups = 0;
  for (int v = 0; v < V; ++v) {
    last[grp[v]] = v;
    if (grp[v] == v) pos[v] = n_groups++;
  }
  // sl: the constraint's literal list, 16-byte aligned; each pass fetches it four
  // slot words at a time (F<b> forward, B<b> reverse); word of group g: <block>.<x|y|z|w>
  static const char* comp = "xyzw";
  std::vector<char> fetched_f((n_groups + 3) / 4, 0), fetched_b((n_groups + 3) / 4, 0);
  auto word = [&](int g, bool fwd) {
    const int j = pos[g], blk = j / 4;
    std::string name = std::string(fwd ? "F" : "B") + std::to_string(blk);
    std::vector<char>& f = fwd ? fetched_f : fetched_b;
    if (!f[blk]) {
      o << "    const uint4 " << name << " = *reinterpret_cast<const uint4*>(sl + " << 4 * blk << ");\n";
      f[blk] = 1;
    }
    return name + "." + comp[j % 4];
  };
  // a slot word is the byte offset of the slot's row; pb and gb point at the lane's
  // first restart in the probability and adjoint rows of slot 0
  auto load = [&](int g, bool fwd) {
    const std::string w = word(g, fwd);
    return "*reinterpret_cast<const float*>(pb + " + w + " + 128 * k)";
  };
  o << "template <bool ADJ, int RPL>\n__device__ __forceinline__ void shape_" << rank
    << "(const unsigned* __restrict__ sl, const float* __restrict__ s_p, float* __restrict__ s_g, int lane,"
       " const Pack<RPL>& wc, Pack<RPL>& cp) {\n"
       "  using V = float;\n  const V zero = 0.f, one = 1.f, mone = -1.f;\n"
       "  const char* pb = reinterpret_cast<const char*>(s_p + lane);\n"
       "  char* gb = reinterpret_cast<char*>(s_g + lane);\n#pragma unroll\n"
       "  for (int k = 0; k < RPL; ++k) {\n";
  for (int adj = 1; adj >= 0; --adj) {
    o << (adj ? "  if (ADJ) {\n" : "  } else {\n");
    std::fill(fetched_f.begin(), fetched_f.end(), 0);
    std::fill(fetched_b.begin(), fetched_b.end(), 0);
    Emitter E{o};
    std::vector<Ex> t(V, Ex{Ex::ZERO, ""});
    std::vector<int> loaded(V, 0);  // bit 0: the forward pass holds q of the group in f<g>
    if (adj) {
      // the root's top-down message is w_c instead of 1: every m_td, and so every
      // group's adjoint sum, carries the weight, and no group multiplies by it
      o << "    const V wv = wc.v[k];\n";
      t[0] = {Ex::VAR, "wv"};
      for (int v = 0; v < V; ++v) {  // Alg. 3: push to non-terminal children
        const int g = grp[v];
        if (hi[v] >= V && lo[v] >= V) continue;
        if (!(loaded[g] & 1)) {
          const std::string ld = load(g, true);  // may emit the block fetch first
          o << "    const V f" << g << " = " << ld << ";\n";
          loaded[g] |= 1;
        }
        const Ex q{Ex::VAR, "f" + std::to_string(g)};
        if (hi[v] < V) t[hi[v]] = E.fma(q, t[v], t[hi[v]]);
        if (lo[v] < V) {
          if (!(loaded[g] & 2)) {
            o << "    const V nf" << g << " = vsub(one, f" << g << ");\n";
            loaded[g] |= 2;
          }
          t[lo[v]] = E.fma({Ex::VAR, "nf" + std::to_string(g)}, t[v], t[lo[v]]);
        }
      }
    }
    std::vector<Ex> bm(V), acc(V, Ex{Ex::ZERO, ""});
    auto bu = [&](int ch) -> Ex {
      if (ch == V) return {Ex::ONE, ""};
      if (ch == V + 1) return {Ex::ZERO, ""};
      return bm[ch];
    };
    for (int v = V - 1; v >= 0; --v) {  // Alg. 4, and the adjoint sum of each group
      const int g = grp[v];
      const bool kept = loaded[g] & 1;  // q from the forward pass, still in a register
      if (last[g] == v && !kept) {
        const std::string ld = load(g, false);
        o << "    const V q" << g << " = " << ld << ";\n";
      }
      const Ex q{Ex::VAR, (kept ? "f" : "q") + std::to_string(g)};
      const Ex d = E.sub(bu(hi[v]), bu(lo[v]));
      bm[v] = E.fma(q, d, bu(lo[v]));
      if (adj) {
        acc[g] = E.fma(t[v], d, acc[g]);
        if (g == v && acc[g].k != Ex::ZERO) {
          const std::string wd = word(g, false);  // fetched at the group's last node already
          o << "    atomicAdd(reinterpret_cast<float*>(gb + " << wd << " + 128 * k), " << E.name(acc[g]) << ");\n";
        }
      }
    }
    o << "    cp.v[k] = " << E.name(bm[0]) << ";\n";
  }
  o << "  }\n  }\n}\n\n";
  return o.str();
}

// A float as an exact hexadecimal literal.
std::string flit(float f) {
  char buf[64];
  std::snprintf(buf, sizeof(buf), "%af", (double)f);
  return buf;
}

// The polish divides by qq = sum of the free terms' squared coefficients (FP32, fmaf in
// term order; term e free when flag n<e> is set).  When every nonzero qq that the flags
// can give is a power of two, the quotient equals the product with the exact reciprocal
// 2^-k, and the routine multiplies by a reciprocal picked by the flags instead of
// dividing (bit for bit the same result); returns that selection as an expression, or ""
// (divide) when some qq is not a power of two or the half-space has more than 4 terms.
static std::string polish_reciprocal(const std::vector<float>& cf) {
  const int n = (int)cf.size();
  if (n == 0 || n > 4) return "";
  std::vector<float> rq(1u << n, 1.f);
  for (unsigned m = 1; m < (1u << n); ++m) {
    float qq = 0.f;
    for (int e = 0; e < n; ++e)
      if ((m >> e) & 1u) qq = std::fmaf(cf[e], cf[e], qq);
    if (!(qq > 0.f)) continue;
    int ex;
    if (std::frexp(qq, &ex) != 0.5f || ex - 1 < -126 || ex - 1 > 126) return "";  // qq = 2^(ex-1), normal
    rq[m] = std::ldexp(1.f, 1 - ex);
  }
  // nested selection on n<n-1> ... n0 (mask bit e = flag n<e>)
  std::function<std::string(int, unsigned)> sel = [&](int e, unsigned m) -> std::string {
    if (e < 0) return flit(rq[m]);
    return "(n" + std::to_string(e) + " ? " + sel(e - 1, m | (1u << e)) + " : " + sel(e - 1, m) + ")";
  };
  return sel(n - 1, 0u);
}

// The projection of one (block, restart) for one block shape (fsmt_proj.cuh's
// pgd_comp_body, the same operations in the same order): the block's iterate x<t>,
// box corrections p<t> and half-space multipliers h<q> in registers, the
// coefficients and 1/||q||^2 as constants, the right-hand sides and the box read
// from the warp's staged block.  Representative block c of the shape.
std::string proj_routine(int rank, const Compiled& C, int c) {
  std::ostringstream o;
  const int v0 = C.comp_var_ptr[c], nv = C.comp_var_ptr[c + 1] - v0;
  const int h0 = C.comp_hs_ptr[c], nh = C.comp_hs_ptr[c + 1] - h0;
  auto X = [](int t) { return "x" + std::to_string(t); };
  o << "__device__ __forceinline__ void proj_" << rank
    << "(const float* __restrict__ s_q0, const float* __restrict__ s_lo, const float* __restrict__ s_hi,"
       " float* __restrict__ b, float* __restrict__ gb, const int* __restrict__ cvar, int R, int r, float step,"
       " float inv, int sweeps, int polish, int clear_grad, bool act, float& part) {\n";
  for (int t = 0; t < nv; ++t) o << "  float x" << t << ", p" << t << " = 0.f;\n";
  for (int t = 0; t < nv; ++t)
    o << "  {\n    const size_t k = (size_t)cvar[" << t << "] * R + r;\n    x" << t
      << " = fmaf(-step, gb[k], b[k]);\n    if (clear_grad) gb[k] = 0.f;\n  }\n";
  for (int q = 0; q < nh; ++q) o << "  float h" << q << " = 0.f;\n";
  o << "  for (int sw = 0; sw < sweeps; ++sw) {\n";
  for (int q = 0; q < nh; ++q) {
    const int e0 = C.hs_ptr[h0 + q], e1 = C.hs_ptr[h0 + q + 1];
    o << "    {\n      float dot = -s_q0[" << q << "];\n";
    for (int e = e0; e < e1; ++e)
      o << "      dot = proj_dot(" << flit(C.hs_coef[e]) << ", " << X(C.hs_lvar[e]) << ", h" << q << ", dot);\n";
    o << "      const float tn = " << (C.hs_eq[h0 + q] ? "proj_tn_eq" : "proj_tn") << "(dot, "
      << flit(C.hs_inv_qq[h0 + q]) << ");\n";
    o << "      const float dl = __fsub_rn(h" << q << ", tn);\n";
    for (int e = e0; e < e1; ++e)
      o << "      " << X(C.hs_lvar[e]) << " = fmaf(dl, " << flit(C.hs_coef[e]) << ", " << X(C.hs_lvar[e]) << ");\n";
    o << "      h" << q << " = tn;\n    }\n";
  }
  for (int t = 0; t < nv; ++t)
    o << "    p" << t << " = proj_box(x" << t << ", p" << t << ", s_lo[" << t << "], s_hi[" << t << "]);\n";
  o << "  }\n  if (sweeps == 0) {\n";
  for (int t = 0; t < nv; ++t)
    o << "    x" << t << " = fminf(fmaxf(x" << t << ", s_lo[" << t << "]), s_hi[" << t << "]);\n";
  o << "  }\n  for (int pass = 0; pass < polish; ++pass) {\n    bool moved = false;\n";
  for (int q = 0; q < nh; ++q) {
    const int e0 = C.hs_ptr[h0 + q], e1 = C.hs_ptr[h0 + q + 1];
    o << "    {\n      const float q0 = s_q0[" << q << "];\n      float v = -q0, mag = fabsf(q0);\n";
    for (int e = e0; e < e1; ++e)
      o << "      { const float tm = __fmul_rn(" << flit(C.hs_coef[e]) << ", " << X(C.hs_lvar[e])
        << "); v = __fadd_rn(v, tm); mag = __fadd_rn(mag, fabsf(tm)); }\n";
    if (C.hs_eq[h0 + q]) {  // a hyperplane: back onto it when off by more than the FP32 band
      o << "      if (fabsf(v) > proj_eq_band(" << e1 - e0 << ", mag)) {\n        float qq = 0.f;\n";
      for (int e = e0; e < e1; ++e) {
        const int t = C.hs_lvar[e];
        const float cf = C.hs_coef[e];
        o << "        const bool n" << e - e0 << " = !(((v > 0.f) == " << (cf > 0.f ? "true" : "false") << ") ? "
          << X(t) << " <= s_lo[" << t << "] : " << X(t) << " >= s_hi[" << t << "]);\n        if (n" << e - e0
          << ") qq = fmaf(" << flit(cf) << ", " << flit(cf) << ", qq);\n";
      }
      std::vector<float> cfs(C.hs_coef.begin() + e0, C.hs_coef.begin() + e1);
      const std::string rq = polish_reciprocal(cfs);
      o << "        if (qq > 0.f) {\n          const float tq = "
        << (rq.empty() ? std::string("__fdiv_rn(v, qq)") : "__fmul_rn(v, " + rq + ")") << ";\n";
      for (int e = e0; e < e1; ++e)
        o << "          if (n" << e - e0 << ") " << X(C.hs_lvar[e]) << " = fmaf(-tq, " << flit(C.hs_coef[e]) << ", "
          << X(C.hs_lvar[e]) << ");\n";
      o << "          moved = true;\n        }\n      }\n    }\n";
      continue;
    }
    // with an exact reciprocal the half-space is one straight run of selects (no
    // branch): a real moves where the half-space is within the margin, some real is
    // free (qq > 0) and this real is free -- the generic loop's conditions
    std::vector<float> cfs(C.hs_coef.begin() + e0, C.hs_coef.begin() + e1);
    const std::string rq = polish_reciprocal(cfs);
    o << "      const float mg = __fmul_rn(kPolishMargin, mag);\n";
    o << (rq.empty() ? "      if (v > -mg) {\n" : "      {\n") << "        float qq = 0.f;\n";
    for (int e = e0; e < e1; ++e) {
      const int t = C.hs_lvar[e];
      const float cf = C.hs_coef[e];
      o << "        const bool n" << e - e0 << " = !(" << (cf > 0.f ? X(t) + " <= s_lo[" : X(t) + " >= s_hi[") << t
        << "]);\n        if (n" << e - e0 << ") qq = fmaf(" << flit(cf) << ", " << flit(cf) << ", qq);\n";
    }
    if (rq.empty()) {
      o << "        if (qq > 0.f) {\n          const float tq = __fdiv_rn(__fadd_rn(v, __fmul_rn(2.f, mg)), qq);\n";
      for (int e = e0; e < e1; ++e)
        o << "          if (n" << e - e0 << ") " << X(C.hs_lvar[e]) << " = fmaf(-tq, " << flit(C.hs_coef[e]) << ", "
          << X(C.hs_lvar[e]) << ");\n";
      o << "          moved = true;\n        }\n      }\n    }\n";
    } else {
      o << "        const bool go = v > -mg && qq > 0.f;\n";
      o << "        const float tq = __fmul_rn(__fadd_rn(v, __fmul_rn(2.f, mg)), " << rq << ");\n";
      for (int e = e0; e < e1; ++e)
        o << "        " << X(C.hs_lvar[e]) << " = go && n" << e - e0 << " ? fmaf(-tq, " << flit(C.hs_coef[e]) << ", "
          << X(C.hs_lvar[e]) << ") : " << X(C.hs_lvar[e]) << ";\n";
      o << "        moved |= go;\n      }\n    }\n";
    }
  }
  for (int t = 0; t < nv; ++t)
    o << "    x" << t << " = fminf(fmaxf(x" << t << ", s_lo[" << t << "]), s_hi[" << t << "]);\n";
  o << "    if (!moved) break;\n  }\n";
  for (int t = 0; t < nv; ++t)
    o << "  {\n    const size_t k = (size_t)cvar[" << t << "] * R + r;\n    const float q = __fmul_rn(__fsub_rn(b[k], x"
      << t << "), inv);\n    part = fmaf(q, q, part);\n    if (act) b[k] = x" << t << ";\n  }\n";
  o << "}\n\n";
  return o.str();
}

std::string kernel_name(int wide, int adj, int rpl) {
  return std::string("fsmt_jit_") + (wide ? "wide_" : "") + (adj ? "adj_" : "fwd_") + std::to_string(rpl);
}

// step: one iteration a launch; wide: chunked without (1) / with (0) the generic
// path, or -1 for warp per constraint
std::string stage_kernel_name(int step, int wide, int rpl) {
  const std::string k = step ? "fsmt_jit_step_" : "fsmt_jit_stage_";
  return wide < 0 ? k + "warp" : k + (wide ? "wide_" : "gen_") + std::to_string(rpl);
}

// The device headers and the instance's generated routines, common to both modules.
std::string routines_source(const Compiled& C) {
  std::ostringstream o;
  o << "#define FSMT_JIT_SHAPES 1\n#define FSMT_JIT_PROJ 1\n" << kJitDevviewSrc << "\n" << kJitChunkedSrc << "\n"
    << kJitProjSrc << "\n" << kJitStageSrc << "\nnamespace fsmt {\n\n";
  for (size_t k = 0; k < C.proj_shape_comp.size(); ++k) o << proj_routine((int)k + 1, C, C.proj_shape_comp[k]);
  o << "__device__ __forceinline__ bool proj_dispatch(int shape, const float* s_q0, const float* s_lo,"
       " const float* s_hi, float* b, float* gb, const int* cvar, int R, int r, float step, float inv, int sweeps,"
       " int polish, int clear_grad, bool act, float& part) {\n  switch (shape) {\n";
  for (size_t k = 0; k < C.proj_shape_comp.size(); ++k)
    o << "    case " << k + 1 << ": proj_" << k + 1
      << "(s_q0, s_lo, s_hi, b, gb, cvar, R, r, step, inv, sweeps, polish, clear_grad, act, part); return true;\n";
  o << "    default: return false;\n  }\n}\n\n";
  for (size_t k = 0; k < C.jit_shape.size(); ++k) {
    const int x = C.jit_shape[k];
    const int b = C.shape_ptr[x], V = C.shape_ptr[x + 1] - b;
    o << shape_routine((int)k + 1, V, C.shape_hi.data() + b, C.shape_lo.data() + b, C.shape_grp.data() + b);
  }
  o << "template <bool ADJ, int RPL>\n__device__ __forceinline__ bool shape_dispatch(int shape, const unsigned* sl,"
       " const float* s_p, float* s_g, int lane, const Pack<RPL>& wc, Pack<RPL>& cp) {\n  switch (shape) {\n";
  for (size_t k = 0; k < C.jit_shape.size(); ++k)
    o << "    case " << k + 1 << ": shape_" << k + 1 << "<ADJ, RPL>(sl, s_p, s_g, lane, wc, cp); return true;\n";
  o << "    default: return false;\n  }\n}\n\n}  // namespace fsmt\n\n";
  return o.str();
}

// The module of the forward / adjoint kernels and the projection kernel.
std::string generated_source(const Compiled& C) {
  std::ostringstream o;
  o << routines_source(C);
  for (int wide = 0; wide < 2; ++wide)
    for (int adj = 0; adj < 2; ++adj)
      for (int rpl = 1; rpl <= 2; ++rpl)
        o << "extern \"C\" __global__ void __launch_bounds__(" << (wide ? "fsmt::kChunkThreadsWide" : "fsmt::kChunkThreads")
          << ", 1) " << kernel_name(wide, adj, rpl)
          << "(fsmt::DevView d, int R, float sigma, const float* prm, int vcap, const float* __restrict__ w,"
             " const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ grad_a,"
             " float* __restrict__ grad_b, float* __restrict__ obj, float* __restrict__ cop, const int* ctl) {\n"
          << "  fsmt::chunked_body<" << (adj ? "true" : "false") << ", " << rpl << ", " << (wide ? "false" : "true")
          << ">(d, R, sigma, prm, vcap, w, a, b, grad_a, grad_b, obj, cop, ctl);\n}\n";
  o << "extern \"C\" __global__ void __launch_bounds__(256) fsmt_jit_proj(fsmt::DevView d, int R, float eta,"
       " float bscale, int sweeps, int polish, const float* prm, const float* __restrict__ wsum,"
       " float* __restrict__ b, float* __restrict__ gb, float* __restrict__ gn2,"
       " const uint8_t* __restrict__ active, int clear_grad, const int* ctl, int maxv, int maxh, int maxnz) {\n"
       "  fsmt::pgd_comp_body(d, R, eta, bscale, sweeps, polish, prm, wsum, b, gb, gn2, active, clear_grad, ctl,"
       " maxv, maxh, maxnz);\n}\n";
  return o.str();
}

// The module of the persistent stage kernels, compiled on first use (jit_build_stage).
std::string stage_source(const Compiled& C) {
  std::ostringstream o;
  o << routines_source(C);
  // the persistent stage kernels (fsmt_stage.cuh) around each forward + adjoint body
  // the tuner can choose: chunked with and without the generic path (the latter run
  // only when every constraint has a routine), and warp per constraint; each once for
  // the stage (stage_body) and once per iteration (stage_step_body).  They read the
  // point through L2 (it changes between their phases).  The warp form is held to at
  // most 51 registers, so that five CTAs of its forward + adjoint phase share an SM, as
  // in the warp kernel of its own.
  for (int step = 0; step < 2; ++step) {
    const char* body = step ? "stage_step_body" : "stage_body";
    for (int wide = 0; wide < 2; ++wide)
      for (int rpl = 1; rpl <= 2; ++rpl)
        o << "extern \"C\" __global__ void __launch_bounds__("
          << (wide ? "fsmt::kChunkThreadsWide" : "fsmt::kChunkThreads") << ", 1) "
          << stage_kernel_name(step, wide, rpl) << "(fsmt::StageArgs s) {\n  fsmt::" << body
          << "(s, [&] { fsmt::chunked_body<true, " << rpl << ", " << (wide ? "false" : "true")
          << ", true>(s.d, s.R, 0.f, s.prm, s.vcap, s.w, s.a, s.b, s.ga, s.gb, s.obj, nullptr, nullptr); });\n}\n";
    o << "extern \"C\" __global__ void __launch_bounds__(fsmt::kFusedThreads, 5) " << stage_kernel_name(step, -1, 0)
      << "(fsmt::StageArgs s) {\n  fsmt::" << body
      << "(s, [&] { fsmt::fused_warp_body<true, true>(s.d, s.R, 0.f, s.prm, s.vcap, s.w, s.a, s.b, s.ga, s.gb, s.obj,"
         " nullptr); });\n}\n";
  }
  return o.str();
}

struct Module {
  void* kernel[2][2][2];  // [wide][adjoint][restarts per lane - 1]
  void* proj;             // the projection kernel with generated block routines
};
struct StageModule {
  void* stage_chunk[2][2][2];  // persistent stage kernels: chunked [per iteration][wide][restarts per lane - 1]
  void* stage_warp[2];         // and warp per constraint [per iteration]
};
std::mutex g_mutex;
std::unordered_map<std::string, Module> g_modules;  // by source text; kept for the process lifetime
std::unordered_map<std::string, StageModule> g_stage_modules;

// The device's "-arch=sm_XYa" option, or "" without a device.
std::string device_arch(int& dev) {
  int major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return "";
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return "-arch=sm_" + std::to_string(major) + std::to_string(minor) + "a";
}

// Compiles src with NVRTC and loads it; false (with the error message set) on failure.
bool compile_and_load(const std::string& src, const std::string& arch, cudaLibrary_t& lib) {
  Nvrtc& N = nvrtc();
  nvrtcProgram prog;
  if (N.create(&prog, src.c_str(), "fsmt_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return false;
  const bool verbose = std::getenv("FSMT_JIT_VERBOSE") != nullptr;
  // -default-device: the kernel body's generic lambdas are device code
  const char* opts[] = {arch.c_str(), "-std=c++17", "-default-device", "-lineinfo", "--ptxas-options=-v"};
  const nvrtcResult rc = N.compile(prog, verbose ? 5 : 4, opts);
  size_t ls = 0;
  N.log_size(prog, &ls);
  std::string log(ls, '\0');
  if (ls) N.log(prog, &log[0]);
  if (verbose) std::fprintf(stderr, "%s\n", log.c_str());
  if (rc != NVRTC_SUCCESS) {
    set_error("run-time compilation failed; using the ahead-of-time kernel:\n" + log);
    N.destroy(&prog);
    return false;
  }
  size_t cs = 0;
  N.cubin_size(prog, &cs);
  std::string cubin(cs, '\0');
  N.cubin(prog, &cubin[0]);
  N.destroy(&prog);
  if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    cudaGetLastError();
    set_error("loading the run-time compiled kernels failed; using the ahead-of-time kernel");
    return false;
  }
  return true;
}

}  // namespace

// Builds (or reuses) the specialised kernels for C.  Returns false, leaving C
// on the ahead-of-time kernel, when there is nothing to specialise, NVRTC is
// missing, FSMT_NO_JIT is set, or compilation fails (the reason goes to the
// error message).
bool jit_build(Compiled& C) {
  for (auto& r : C.jit_kernel) r[0] = r[1] = nullptr;
  for (auto& r : C.jit_wide) r[0] = r[1] = nullptr;
  C.jit_shapes = 0;
  C.jit_proj = nullptr;
  C.proj_shapes = 0;
  C.jit_stage_tried = false;
  for (int step = 0; step < 2; ++step) {
    C.jit_stage_warp[step] = nullptr;
    for (int w = 0; w < 2; ++w) C.jit_stage_chunk[step][w][0] = C.jit_stage_chunk[step][w][1] = nullptr;
  }
  const char* off = std::getenv("FSMT_NO_JIT");
  const bool diagrams = !C.jit_shape.empty() && C.chunked_ok, blocks = !C.proj_shape_comp.empty();
  if ((off && *off && *off != '0') || !(diagrams || blocks)) return false;
  if (!nvrtc().ok) return false;
  int dev = 0;
  const std::string arch = device_arch(dev);
  if (arch.empty()) return false;
  const std::string src = generated_source(C);
  std::lock_guard<std::mutex> lock(g_mutex);
  const std::string key = arch + src;
  auto it = g_modules.find(key);
  if (it == g_modules.end()) {
    cudaLibrary_t lib;
    if (!compile_and_load(src, arch, lib)) return false;
    // a failure below leaves no error behind for the next launch check to find
    auto fail = [](const char* what) {
      cudaGetLastError();
      set_error(std::string(what) + "; using the ahead-of-time kernel");
      return false;
    };
    Module m{};
    for (int wide = 0; wide < 2; ++wide)
      for (int adj = 0; adj < 2; ++adj)
        for (int r = 0; r < 2; ++r) {
          cudaKernel_t k;
          if (cudaLibraryGetKernel(&k, lib, kernel_name(wide, adj, r + 1).c_str()) != cudaSuccess ||
              cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
                  cudaSuccess)
            return fail("preparing a run-time compiled chunked kernel failed");
          m.kernel[wide][adj][r] = (void*)k;
        }
    {
      cudaKernel_t k;
      if (cudaLibraryGetKernel(&k, lib, "fsmt_jit_proj") != cudaSuccess ||
          cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(kProjSmemWords * sizeof(float))) != cudaSuccess)
        return fail("preparing the run-time compiled projection kernel failed");
      m.proj = (void*)k;
    }
    it = g_modules.emplace(key, m).first;
  }
  if (diagrams) {
    for (int adj = 0; adj < 2; ++adj)
      for (int r = 0; r < 2; ++r) {
        C.jit_kernel[adj][r] = it->second.kernel[0][adj][r];
        C.jit_wide[adj][r] = C.all_specialized ? it->second.kernel[1][adj][r] : nullptr;
      }
    C.jit_shapes = (int32_t)C.jit_shape.size();
  }
  if (blocks) {
    C.jit_proj = it->second.proj;
    C.proj_shapes = (int32_t)C.proj_shape_comp.size();
  }
  return true;
}

// Builds (or reuses) the persistent stage kernels for C, once per compiled object and
// only when asked for: they double the run-time compilation, which every upload would
// otherwise pay.  Needs the module of jit_build (the same routines).  Returns whether
// the kernels are there.
bool jit_build_stage(Compiled& C) {
  if (C.jit_stage_tried) return C.jit_stage_warp[0] != nullptr;
  C.jit_stage_tried = true;
  if (!C.jit_proj && !C.jit_kernel[1][0]) return false;  // no run-time compiled module
  int dev = 0;
  const std::string arch = device_arch(dev);
  if (arch.empty()) return false;
  const std::string src = stage_source(C);
  std::lock_guard<std::mutex> lock(g_mutex);
  const std::string key = arch + src;
  auto it = g_stage_modules.find(key);
  if (it == g_stage_modules.end()) {
    cudaLibrary_t lib;
    if (!compile_and_load(src, arch, lib)) return false;
    // the stage kernels have static shared memory of their own (barrier and epsilon
    // test): the dynamic part may take what is left of the per-CTA maximum
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto stage_kernel = [&](int step, int wide, int rpl, void*& out) {
      cudaKernel_t k;
      cudaFuncAttributes fa;
      if (cudaLibraryGetKernel(&k, lib, stage_kernel_name(step, wide, rpl).c_str()) != cudaSuccess ||
          cudaFuncGetAttributes(&fa, (const void*)k) != cudaSuccess ||
          cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes) != cudaSuccess)
        return false;
      out = (void*)k;
      return true;
    };
    StageModule m{};
    for (int step = 0; step < 2; ++step) {
      bool ok = stage_kernel(step, -1, 0, m.stage_warp[step]);
      for (int wide = 0; wide < 2; ++wide)
        for (int r = 0; r < 2; ++r) ok = ok && stage_kernel(step, wide, r + 1, m.stage_chunk[step][wide][r]);
      if (!ok) {
        cudaGetLastError();  // leave no error behind for the next launch check to find
        set_error("preparing the persistent stage kernels failed; stages use separate launches");
        return false;
      }
    }
    it = g_stage_modules.emplace(key, m).first;
  }
  for (int step = 0; step < 2; ++step) {
    C.jit_stage_warp[step] = it->second.stage_warp[step];
    for (int r = 0; r < 2; ++r) {
      C.jit_stage_chunk[step][0][r] = C.jit_kernel[1][0] ? it->second.stage_chunk[step][0][r] : nullptr;
      C.jit_stage_chunk[step][1][r] = C.jit_wide[1][0] ? it->second.stage_chunk[step][1][r] : nullptr;
    }
  }
  return true;
}

}  // namespace fsmt
