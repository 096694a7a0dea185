// Device code of the chunked forward/adjoint kernel and the helpers it shares
// with the other kernels.  Written to compile both ahead of time (nvcc, through
// fsmt_device.cu) and at run time (NVRTC), where per-shape specialisations of the
// diagram passes are generated from the compiled diagrams (fsmt_jit.cpp).
#pragma once

namespace fsmt {

constexpr float kTwoOverSqrtPi = 1.1283791670955126f;
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr int kMaxObjSmemR = 4096;
constexpr int kChunkThreadsWide = 1024;  // 32 warps, without the generic path

// stage parameter slots (device float[16])
enum { P_SIGMA = 0, P_ETA, P_BSCALE, P_EPS, P_RHO, P_GAMMA, P_UPDATE_W, P_SWEEPS, P_POLISH, P_NORM };

__device__ __forceinline__ float load_param(const float* prm, int slot, float fallback) {
  return prm ? prm[slot] : fallback;
}

// A read of the restarts' point (a, b).  Kernels that run one pass read it through
// the read-only path; the persistent stage kernel, whose PGD phase rewrites a and b
// between its forward + adjoint phases, reads it through L2 (CO = true), because the
// read-only path is only defined for data that no thread of the kernel writes.
template <bool CO>
__device__ __forceinline__ float ld_state(const float* p) {
  return CO ? __ldcg(p) : __ldg(p);
}

// ------------------------------------------------------- literal probability --
// p = P[variable TRUE]; gz = dd/dz for atoms (0 for Booleans).  Eq. rounding and
// Eq. sampling.  s_inv = 1 / (sqrt 2 sigma); s_inv < 0 stands for sigma = 0, which
// decides the atom exactly; s_inv = 0 for sigma = infinity gives p = 1/2, gz = 0.
template <bool CO = false>
__device__ __forceinline__ void literal_prob(const DevView& d, int lab, int R, int r, bool ok, float s_inv,
                                             const float* __restrict__ a, const float* __restrict__ b, float& p,
                                             float& gz) {
  if (lab < d.n_bool) {
    float av = ok ? ld_state<CO>(a + (size_t)lab * R + r) : 0.f;
    p = 0.5f * (1.f - av);
    gz = 0.f;
    return;
  }
  const int i = lab - d.n_bool;
  const int k0 = __ldg(d.atom_ptr + i), k1 = __ldg(d.atom_ptr + i + 1);
  if (s_inv >= 0.f) {
    float z = -__ldg(d.atom_q0f + i);
    for (int k = k0; k < k1; ++k) {
      float bv = ok ? ld_state<CO>(b + (size_t)__ldg(d.atom_var + k) * R + r) : 0.f;
      z = fmaf(__ldg(d.atom_coef + k), bv, z);
    }
    const float si = __ldg(d.atom_inv_norm + i) * s_inv;  // 1 / (sqrt(2) sigma ||q||)
    const float u = z * si;
    p = 0.5f * erfcf(u);
    gz = kTwoOverSqrtPi * __expf(-u * u) * si;
  } else {
    Fixed320 acc;
    acc.clear();
    for (int k = k0; k < k1; ++k) {
      float bv = ok ? ld_state<CO>(b + (size_t)__ldg(d.atom_var + k) * R + r) : 0.f;
      uint32_t m;
      int e;
      bool neg;
      float_parts(bv, m, e, neg);
      if (m == 0) continue;
      float c = __ldg(d.atom_coef + k);
      bool cneg = c < 0.f;
      acc.add((uint64_t)(cneg ? -c : c) * (uint64_t)m, e + 149, neg != cneg);
    }
    double q0 = __ldg(d.atom_q0d + i);
    if (q0 != 0.0) acc.add((uint64_t)fabs(q0), 149, q0 > 0.0);
    const int sg = acc.sign();
    const bool truth = __ldg(d.atom_strict + i) ? sg < 0 : sg <= 0;
    p = truth ? 1.f : 0.f;
    gz = 0.f;
  }
}

__device__ __forceinline__ void scatter_grad(const DevView& d, int lab, int R, int r, float g, float gz,
                                             float* __restrict__ grad_a, float* __restrict__ grad_b) {
  if (lab < d.n_bool) {
    atomicAdd(grad_a + (size_t)lab * R + r, g);
  } else {
    const int i = lab - d.n_bool;
    const float gg = g * gz;
    if (gg != 0.f) {
      const int k0 = __ldg(d.atom_ptr + i), k1 = __ldg(d.atom_ptr + i + 1);
      for (int k = k0; k < k1; ++k)
        atomicAdd(grad_b + (size_t)__ldg(d.atom_var + k) * R + r, gg * __ldg(d.atom_coef + k));
    }
  }
}


// -------------------------------------------------------- chunked kernel --
// One CTA per chunk of constraints of C_sigma (grid-stride over chunks), looping
// over restart tiles of 32*RPL restarts; each lane carries RPL restarts (lane,
// lane+32, ...), so every global access of a warp is a contiguous 128-byte line.
// Per tile:
//  (1) every slot -- a literal (a Boolean or an atom, with its polarity) used by
//      the chunk -- gets its probability q of holding once (Eq. rounding /
//      Eq. sampling; 1 - p for a negated literal), so the diagram passes work in
//      literal space (a node's hi child: its literal holds) with no polarity
//      logic of their own;
//  (2) each warp runs Alg. 3 then Alg. 4 on its constraints -- through a
//      routine generated for the constraint's diagram shape when there is one
//      (shape_dispatch), else the generic form below -- with p read from
//      shared memory and the messages in the warp's rows: one row per decision
//      node plus two fixed rows for the terminals (the compiler points terminal
//      children there), so the passes have no branches -- the forward pass may
//      push into the terminal rows, which are then set to 1 (TRUE) and 0 (FALSE)
//      for the backward pass; COP_c = m_bu[root] (Lemma backward).  The
//      backward pass adds w_c m_td[v] (m_bu[hi] - m_bu[lo]) to the slot's
//      shared accumulator;
//  (3) each slot's accumulated derivative reaches the global gradient once (for
//      atoms through dd/db_j; negated literals with the sign flipped).
template <int RPL>
struct __align__(4 * RPL) Pack {
  float v[RPL];
};
template <int N>
struct IntC {
  static constexpr int value = N;
};

// Arithmetic of the generated diagram routines: IEEE single operations, never
// contracted with one another.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }

// erfc(x)/2 for the atom probability, by Abramowitz & Stegun 7.1.26 (Hastings):
// erf(x) = 1 - (a1 t + ... + a5 t^5) e^{-x^2} + e(x), t = 1/(1 + 0.3275911 x),
// |e(x)| <= 1.5e-7 for x >= 0; erfc(-x) = 2 - erfc(x).  `ex` is e^{-x^2}.
__device__ __forceinline__ float half_erfc_as(float x, float ex) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.f, fmaf(0.3275911f, ax, 1.f));  // approximate reciprocal, 1 + 0.33|x| >= 1
  float poly = fmaf(t, 1.061405429f, -1.453152027f);
  poly = fmaf(t, poly, 1.421413741f);
  poly = fmaf(t, poly, -0.284496736f);
  poly = fmaf(t, poly, 0.254829592f);
  const float h = 0.5f * t * poly * ex;  // erfc(|x|) / 2
  return x >= 0.f ? h : 1.f - h;
}

// z = q.b - q0 of atom i at restart r (normalised form)
__device__ __forceinline__ float atom_z(const DevView& d, int i, int R, int r, const float* __restrict__ b) {
  const int k0 = __ldg(d.atom_ptr + i), k1 = __ldg(d.atom_ptr + i + 1);
  float z = -__ldg(d.atom_q0f + i);
  for (int k = k0; k < k1; ++k) z = fmaf(__ldg(d.atom_coef + k), __ldg(b + (size_t)__ldg(d.atom_var + k) * R + r), z);
  return z;
}

template <bool ADJ, int RPL>
__device__ __forceinline__ bool shape_dispatch(int shape, const unsigned* sl, const float* s_p, float* s_g, int lane,
                                               const Pack<RPL>& wc, Pack<RPL>& cp);

// GENERIC = false: every constraint has a generated routine, so the generic
// path and its per-warp message rows are left out (more warps fit).
template <bool ADJ, int RPL, bool GENERIC = true, bool CO = false>
__device__ __forceinline__ void chunked_body(const DevView& d, int R, float sigma, const float* prm, int vcap,
                                             const float* __restrict__ w, const float* __restrict__ a,
                                             const float* __restrict__ b, float* __restrict__ grad_a,
                                             float* __restrict__ grad_b, float* __restrict__ obj,
                                             float* __restrict__ cop, const int* ctl) {
  using PK = Pack<RPL>;
  if (ctl && ctl[0] == 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int rows = vcap + 2;  // decision nodes, then TRUE (vcap) and FALSE (vcap + 1)
  uint2* s_node = reinterpret_cast<uint2*>(smem);
  int4* s_con = reinterpret_cast<int4*>(s_node + kChunkMaxNodes);
  unsigned* s_list = reinterpret_cast<unsigned*>(s_con + kChunkMaxCons);  // the constraints' literal lists
  int* s_lab = reinterpret_cast<int*>(s_list + kChunkMaxList);
  int* s_meta = s_lab + kChunkMaxSlots;                            // atom slots: first term << 16 | count
  float* s_q0 = reinterpret_cast<float*>(s_meta + kChunkMaxSlots);  // atom slots: q0
  float* s_si = s_q0 + kChunkMaxSlots;                             // atom slots: 1 / (sqrt(2) sigma ||q||)
  int* s_tvar = reinterpret_cast<int*>(s_si + kChunkMaxSlots);     // the chunk's atom terms
  float* s_tcoef = reinterpret_cast<float*>(s_tvar + kChunkMaxTerms);
  int* s_rid = reinterpret_cast<int*>(s_tcoef + kChunkMaxTerms);  // the chunk's reals
  const int cap = d.chunk_slot_cap;
  // per-slot rows of kSlotStride floats, restart k of lane l at 32 k + l; a node's
  // slot word is the row's byte offset (slot * 4 * kSlotStride)
  float* s_p = reinterpret_cast<float*>(s_rid + kChunkMaxReals);  // probability of the literal
  float* s_g = s_p + cap * kSlotStride;                            // its adjoint
  // reals staged per restart tile (0: atoms read b from global memory instead)
  const int rcap = d.chunk_real_cap;
  float* s_b = s_g + cap * kSlotStride;         // [tile parity][real][RPL][32]: b of the chunk's reals
  float* s_gr = s_b + 2 * rcap * RPL * 32;      // [tile parity][real][RPL][32]: dC/db accumulators
  PK* s_rows = reinterpret_cast<PK*>(s_gr + 2 * rcap * RPL * 32);
  PK* s_m = s_rows + warp * rows * 32 + lane;
  float* obj_s = (R <= kMaxObjSmemR) ? reinterpret_cast<float*>(s_rows + (GENERIC ? W * rows * 32 : 0)) : nullptr;
  if (obj_s)
    for (int r = threadIdx.x; r < R; r += blockDim.x) obj_s[r] = 0.f;
  sigma = load_param(prm, P_SIGMA, sigma);
  const float s_inv = sigma > 0.f ? kInvSqrt2 / sigma : -1.f;  // < 0: sigma = 0, exact; 0: sigma = inf
  const int n_tiles = (R + 32 * RPL - 1) / (32 * RPL);
  for (int q = blockIdx.x; q < d.n_chunks; q += gridDim.x) {
    const int c0 = __ldg(d.chunk_con_ptr + q), nc = __ldg(d.chunk_con_ptr + q + 1) - c0;
    const int n0 = __ldg(d.chunk_node_ptr + q), nn = __ldg(d.chunk_node_ptr + q + 1) - n0;
    const int l0 = __ldg(d.chunk_slot_ptr + q), ns = __ldg(d.chunk_slot_ptr + q + 1) - l0;
    __syncthreads();  // the previous chunk is done with shared memory
    for (int i = threadIdx.x; i < nn; i += blockDim.x) s_node[i] = d.cnodes[n0 + i];
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s_con[i] = d.ccon[c0 + i];
    {
      const int q0l = __ldg(d.chunk_list_ptr + q), nl = __ldg(d.chunk_list_ptr + q + 1) - q0l;
      for (int i = threadIdx.x; i < nl; i += blockDim.x) s_list[i] = __ldg(d.clist + q0l + i);
    }
    const int t0 = __ldg(d.chunk_term_ptr + q), nt = __ldg(d.chunk_term_ptr + q + 1) - t0;
    const int e0 = __ldg(d.chunk_real_ptr + q), nr = __ldg(d.chunk_real_ptr + q + 1) - e0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) s_rid[i] = __ldg(d.real_id + e0 + i);
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const int raw = __ldg(d.slot_label + l0 + i);  // bit 31: the literal is negated
      const int lab = raw & 0x7fffffff;
      s_lab[i] = raw;
      s_meta[i] = __ldg(d.slot_meta + l0 + i);
      if (lab >= d.n_bool) {
        s_q0[i] = __ldg(d.atom_q0f + lab - d.n_bool);
        s_si[i] = __ldg(d.atom_inv_norm + lab - d.n_bool) * s_inv;
      }
    }
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      s_tvar[i] = __ldg(d.term_var + t0 + i);
      s_tcoef[i] = __ldg(d.term_coef + t0 + i);
    }
    const bool staged = rcap > 0;
    const int nre = nr * RPL * 32;  // staged elements per tile
    // b of tile t for the chunk's reals, into buffer t & 1
    auto stage_b = [&](int t) {
      float* dst = s_b + (t & 1) * rcap * RPL * 32;
      for (int e = threadIdx.x; e < nre; e += blockDim.x) {
        const int r = (t * RPL + (e >> 5) % RPL) * 32 + (e & 31);
        dst[e] = r < R ? ld_state<CO>(b + (size_t)__ldg(d.real_id + e0 + e / (RPL * 32)) * R + r) : 0.f;
      }
    };
    // dC/db of tile t: one global update per real and restart, then the buffer is cleared
    auto flush_gr = [&](int t) {
      float* src = s_gr + (t & 1) * rcap * RPL * 32;
      for (int e = threadIdx.x; e < nre; e += blockDim.x) {
        const float g = src[e];
        const int r = (t * RPL + (e >> 5) % RPL) * 32 + (e & 31);
        if (g != 0.f && r < R) atomicAdd(grad_b + (size_t)s_rid[e / (RPL * 32)] * R + r, g);
        src[e] = 0.f;
      }
    };
    if (staged) {
      stage_b(0);
      if (ADJ)
        for (int e = threadIdx.x; e < 2 * nre; e += blockDim.x) s_gr[(e / nre) * rcap * RPL * 32 + e % nre] = 0.f;
    }
    __syncthreads();
    // One pass over the slots: the gradient of tile tf leaves the slot
    // accumulators (a Boolean's for global memory, an atom's through dd/dz and
    // the chain rule into its reals), and the slots get the TRUE-probability p
    // of tile tp.
    auto slot_pass = [&](int tf, int tp) {
      const bool do_f = ADJ && tf >= 0, do_p = tp < n_tiles;
      const float* sbf = s_b + (tf & 1) * rcap * RPL * 32;
      const float* sbp = s_b + (tp & 1) * rcap * RPL * 32;
      float* sgr = s_gr + (tf & 1) * rcap * RPL * 32;
      for (int i = warp; i < ns; i += W) {
        const int raw = s_lab[i], lab = raw & 0x7fffffff;
        const float sg = raw < 0 ? -1.f : 1.f;  // dq/dp
        float* gi = s_g + i * kSlotStride + lane;  // the slot's adjoint dC/dq, restart k at gi[32 k]
        PK pp;
        if (lab < d.n_bool) {  // a Boolean: p = (1 - a) / 2
#pragma unroll
          for (int k = 0; k < RPL; ++k) {
            const int rf = (tf * RPL + k) * 32 + lane, rp = (tp * RPL + k) * 32 + lane;
            if (do_f) {
              const float g = gi[32 * k];
              if (rf < R && g != 0.f) atomicAdd(grad_a + (size_t)lab * R + rf, sg * g);
            }
            if (do_p) pp.v[k] = rp < R ? 0.5f * (1.f - sg * ld_state<CO>(a + (size_t)lab * R + rp)) : 0.f;
          }
        } else if (staged && s_inv >= 0.f) {
          // an atom, its reals staged: z = q.y - q0 of both tiles in one sweep
          // over the terms; past the last restart b reads 0 and the adjoint is 0
          const int meta = s_meta[i], tb = meta >> 16, tc = meta & 0xffff;
          const float q0 = s_q0[i], si = s_si[i];
          // NT terms known at compile time (2, the common case), or tc when NT = 0
          auto atom = [&](auto ntc) {
            constexpr int NT = decltype(ntc)::value;
            const int nt = NT ? NT : tc;
            float zf[RPL], zp[RPL];
#pragma unroll
            for (int k = 0; k < RPL; ++k) zf[k] = zp[k] = -q0;
#pragma unroll
            for (int j = 0; j < nt; ++j) {
              const float cj = s_tcoef[tb + j];
              const int o = s_tvar[tb + j] * RPL * 32 + lane;
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                if (do_f) zf[k] = fmaf(cj, sbf[o + 32 * k], zf[k]);
                if (do_p) zp[k] = fmaf(cj, sbp[o + 32 * k], zp[k]);
              }
            }
            if (do_f) {  // dC/dz = dC/dq dq/dp dp/dz, then dC/db_j = dC/dz q_j into the chunk's reals
              float gz[RPL];
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                const float u = zf[k] * si;
                gz[k] = sg * gi[32 * k] * (kTwoOverSqrtPi * si) * __expf(-u * u);
              }
#pragma unroll
              for (int j = 0; j < nt; ++j) {
                const float cj = s_tcoef[tb + j];
                const int o = s_tvar[tb + j] * RPL * 32 + lane;
#pragma unroll
                for (int k = 0; k < RPL; ++k) atomicAdd(sgr + o + 32 * k, gz[k] * cj);
              }
            }
            if (do_p)
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                const float u = zp[k] * si;
                pp.v[k] = half_erfc_as(sg * u, __expf(-u * u));  // 1 - erfc(u)/2 = erfc(-u)/2
              }
          };
          if (tc == 2)
            atom(IntC<2>{});
          else
            atom(IntC<0>{});
        } else {  // an atom with b in global memory, or sigma = 0
          const int meta = s_meta[i], tb = meta >> 16, tc = meta & 0xffff;
#pragma unroll
          for (int k = 0; k < RPL; ++k) {
            const int rf = (tf * RPL + k) * 32 + lane, rp = (tp * RPL + k) * 32 + lane;
            if (do_f && s_inv >= 0.f) {
              const float g = gi[32 * k];
              if (rf < R && g != 0.f) {
                float z = -s_q0[i];
                for (int j = 0; j < tc; ++j)
                  z = fmaf(s_tcoef[tb + j], ld_state<CO>(b + (size_t)s_rid[s_tvar[tb + j]] * R + rf), z);
                const float si = s_si[i], u = z * si;
                const float gz = sg * g * kTwoOverSqrtPi * __expf(-u * u) * si;  // dC/dz
                for (int j = 0; j < tc; ++j)
                  atomicAdd(grad_b + (size_t)s_rid[s_tvar[tb + j]] * R + rf, gz * s_tcoef[tb + j]);
              }
            }
            if (do_p) {
              const bool ok = rp < R;
              if (s_inv >= 0.f) {
                float z = -s_q0[i];
                for (int j = 0; j < tc; ++j)
                  z = fmaf(s_tcoef[tb + j], ok ? ld_state<CO>(b + (size_t)s_rid[s_tvar[tb + j]] * R + rp) : 0.f, z);
                const float u = z * s_si[i];
                pp.v[k] = half_erfc_as(sg * u, __expf(-u * u));
              } else {
                float p, gz;
                literal_prob<CO>(d, lab, R, rp, ok, -1.f, a, b, p, gz);
                pp.v[k] = raw < 0 ? 1.f - p : p;  // exact: p is 0 or 1
              }
            }
          }
        }
        if (do_p)
#pragma unroll
          for (int k = 0; k < RPL; ++k) {
            s_p[i * kSlotStride + 32 * k + lane] = pp.v[k];
            if (ADJ) gi[32 * k] = 0.f;
          }
      }
    };
    slot_pass(-1, 0);
    for (int t = 0; t < n_tiles; ++t) {
      int rr[RPL];
      bool ok[RPL];
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        rr[k] = (t * RPL + k) * 32 + lane;
        ok[k] = rr[k] < R;
      }
      __syncthreads();  // p of tile t is ready, accumulators are zero
      if (staged) {  // while the DP runs: b of tile t + 1 in, dC/db of tile t - 1 out
        if (t + 1 < n_tiles) stage_b(t + 1);
        if (ADJ && t >= 1) flush_gr(t - 1);
      }
      // Alg. 3 and Alg. 4, one warp per constraint, each warp a contiguous run
      float objacc[RPL];
#pragma unroll
      for (int k = 0; k < RPL; ++k) objacc[k] = 0.f;
      const int c_end = (warp + 1) * nc / W;
      PK wn;  // w of the warp's next constraint, loaded one constraint ahead
      {
        const int c = warp * nc / W;
        const int id = c < c_end ? s_con[c].w : 0;
#pragma unroll
        for (int k = 0; k < RPL; ++k) wn.v[k] = (c < c_end && ok[k]) ? __ldg(w + (size_t)id * R + rr[k]) : 0.f;
      }
      for (int c = warp * nc / W; c < c_end; ++c) {
        const int4 cn = s_con[c];
        const uint2* nd = s_node + cn.x;
        const int V = cn.y & 0xffff;
        const int shape = cn.y >> 16;
        const PK wc = wn;
        PK cp;
        if (c + 1 < c_end) {
          const int id = s_con[c + 1].w;
#pragma unroll
          for (int k = 0; k < RPL; ++k) wn.v[k] = ok[k] ? __ldg(w + (size_t)id * R + rr[k]) : 0.f;
        }
        if ((shape == 0 || !shape_dispatch<ADJ, RPL>(shape, s_list + cn.z, s_p, s_g, lane, wc, cp)) && GENERIC) {
          PK zero, one;
#pragma unroll
          for (int k = 0; k < RPL; ++k) {
            zero.v[k] = 0.f;
            one.v[k] = 1.f;
          }
          if (ADJ && V > 0) {
            s_m[0] = one;  // the root is node 0
            for (int v = 1; v < V; ++v) s_m[v * 32] = zero;
            for (int v = 0; v < V; ++v) {  // Alg. 3, topological order
              const uint2 e = nd[v];
              const int hi = (int)(e.y & 0xffffu) * 32, lo = (int)(e.y >> 16) * 32;
              PK p;
#pragma unroll
              for (int k = 0; k < RPL; ++k) p.v[k] = s_p[(e.x >> 8) * kSlotStride + 32 * k + lane];
              const PK mv = s_m[v * 32];
              PK mh = s_m[hi], ml = s_m[lo];
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                mh.v[k] = fmaf(p.v[k], mv.v[k], mh.v[k]);
                ml.v[k] = fmaf(-p.v[k], mv.v[k], ml.v[k] + mv.v[k]);
              }
              s_m[hi] = mh;
              s_m[lo] = ml;
            }
          }
          s_m[vcap * 32] = one;
          s_m[(vcap + 1) * 32] = zero;
          for (int v = V - 1; v >= 0; --v) {  // Alg. 4, reverse topological order
            const uint2 e = nd[v];
            const int slot = (int)(e.x >> 8);
            const PK mh = s_m[(int)(e.y & 0xffffu) * 32], ml = s_m[(int)(e.y >> 16) * 32];
            PK p;
#pragma unroll
            for (int k = 0; k < RPL; ++k) p.v[k] = s_p[slot * kSlotStride + 32 * k + lane];
            PK nb;
            if (ADJ) {
              const PK td = s_m[v * 32];
              float* gs = s_g + slot * kSlotStride + lane;
#pragma unroll
              for (int k = 0; k < RPL; ++k) {
                const float diff = mh.v[k] - ml.v[k];
                nb.v[k] = fmaf(p.v[k], diff, ml.v[k]);
                const float g = wc.v[k] * td.v[k] * diff;
                if (g != 0.f) atomicAdd(gs + k * 32, g);
              }
            } else {
#pragma unroll
              for (int k = 0; k < RPL; ++k) nb.v[k] = fmaf(p.v[k], mh.v[k] - ml.v[k], ml.v[k]);
            }
            s_m[v * 32] = nb;
          }
          // COP = m_bu[root]; a constant diagram's root is a terminal row
          cp = V > 0 ? s_m[0] : s_m[(cn.z == 0 ? vcap : vcap + 1) * 32];
        }
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          if (!ok[k]) continue;
          if (cop) cop[(size_t)cn.w * R + rr[k]] = cp.v[k];
          objacc[k] = fmaf(wc.v[k], 1.f - 2.f * cp.v[k], objacc[k]);
        }
      }
      if (obj)
#pragma unroll
        for (int k = 0; k < RPL; ++k)
          if (ok[k] && objacc[k] != 0.f) atomicAdd(obj_s ? obj_s + rr[k] : obj + rr[k], objacc[k]);
      __syncthreads();  // the gradient of tile t is complete; p of tile t is no longer read
      slot_pass(t, t + 1);
    }
    if (ADJ && staged) {
      __syncthreads();
      flush_gr(n_tiles - 1);
    }
  }
  if (obj_s && obj) {
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      if (obj_s[r] != 0.f) atomicAdd(obj + r, obj_s[r]);
  }
}


// ---------------------------------------------------- warp per constraint --
// One warp per constraint of C_sigma (grid-stride), looping over restart tiles;
// the constraint's nodes are staged once in the warp's shared memory and reused
// for every tile.  Per lane: Alg. 3 (top-down messages m_td), then, if ADJ,
// Alg. 4 (bottom-up messages m_bu written over m_td in reverse topological
// order, so one array serves both) with the gradient scattered by atomics.
template <bool ADJ, bool CO = false>
__device__ __forceinline__ void fused_warp_body(const DevView& d, int R, float sigma, const float* prm, int vcap,
                                                const float* __restrict__ w, const float* __restrict__ a,
                                                const float* __restrict__ b, float* __restrict__ grad_a,
                                                float* __restrict__ grad_b, float* __restrict__ obj,
                                                float* __restrict__ cop) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const size_t wb = (size_t)vcap * 8 + (size_t)(3 * vcap + 2) * 128;
  uint2* snode = reinterpret_cast<uint2*>(smem + warp * wb);
  float* sp = reinterpret_cast<float*>(snode + vcap);
  float* sg = sp + vcap * 32;
  float* sm = sg + vcap * 32;
  float* obj_s = (R <= kMaxObjSmemR) ? reinterpret_cast<float*>(smem + W * wb) : nullptr;
  if (obj_s) {
    for (int r = threadIdx.x; r < R; r += blockDim.x) obj_s[r] = 0.f;
    __syncthreads();
  }
  sigma = load_param(prm, P_SIGMA, sigma);
  const float s_inv = sigma > 0.f ? kInvSqrt2 / sigma : -1.f;  // < 0: sigma = 0, exact; 0: sigma = inf
  const int n_tiles = (R + 31) >> 5;
  for (int s = blockIdx.x * W + warp; s < d.n_obj; s += gridDim.x * W) {
    const int nb = __ldg(d.con_ptr + s);
    const int V = __ldg(d.con_ptr + s + 1) - nb;
    const int cid = __ldg(d.con_id + s);
    const int root = __ldg(d.con_root + s);
    for (int i = lane; i < V; i += 32) snode[i] = d.nodes[nb + i];
    __syncwarp();
    for (int t = 0; t < n_tiles; ++t) {
      const int r = t * 32 + lane;
      const bool ok = r < R;
      for (int v = 0; v < V + 2; ++v) sm[v * 32 + lane] = 0.f;
      sm[root * 32 + lane] = 1.f;
      for (int v = 0; v < V; ++v) {  // Alg. 3, topological order
        const uint2 nd = snode[v];
        const int hi = nd.y & 0xffff, lo = nd.y >> 16;
        float p, gz;
        literal_prob<CO>(d, (int)nd.x, R, r, ok, s_inv, a, b, p, gz);
        sp[v * 32 + lane] = p;
        if (ADJ) sg[v * 32 + lane] = gz;
        const float mv = sm[v * 32 + lane];
        sm[hi * 32 + lane] = fmaf(p, mv, sm[hi * 32 + lane]);
        sm[lo * 32 + lane] = fmaf(1.f - p, mv, sm[lo * 32 + lane]);
      }
      const float cp = sm[V * 32 + lane];
      const float wc = ok ? __ldg(w + (size_t)cid * R + r) : 0.f;
      if (ok) {
        if (cop) cop[(size_t)cid * R + r] = cp;
        const float contrib = wc * (1.f - 2.f * cp);
        if (obj) {
          if (obj_s)
            atomicAdd(obj_s + r, contrib);
          else
            atomicAdd(obj + r, contrib);
        }
      }
      if (ADJ) {  // Alg. 4, reverse topological order
        sm[V * 32 + lane] = 1.f;
        sm[(V + 1) * 32 + lane] = 0.f;
        for (int v = V - 1; v >= 0; --v) {
          const uint2 nd = snode[v];
          const int hi = nd.y & 0xffff, lo = nd.y >> 16;
          const float mh = sm[hi * 32 + lane], ml = sm[lo * 32 + lane];
          const float p = sp[v * 32 + lane];
          const float td = sm[v * 32 + lane];
          const float diff = mh - ml;
          sm[v * 32 + lane] = fmaf(p, diff, ml);
          if (ok) scatter_grad(d, (int)nd.x, R, r, wc * td * diff, sg[v * 32 + lane], grad_a, grad_b);
        }
      }
    }
    __syncwarp();
  }
  if (obj_s && obj) {
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x)
      if (obj_s[r] != 0.f) atomicAdd(obj + r, obj_s[r]);
  }
}

#ifndef FSMT_JIT_SHAPES
// Ahead-of-time build: no generated routines, every constraint takes the generic path.
template <bool ADJ, int RPL>
__device__ __forceinline__ bool shape_dispatch(int, const unsigned*, const float*, float*, int, const Pack<RPL>&,
                                               Pack<RPL>&) {
  return false;
}
#endif

}  // namespace fsmt
