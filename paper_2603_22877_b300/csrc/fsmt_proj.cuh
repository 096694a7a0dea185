// Device code of the projection of the reals onto D (Def. Projection, Prop. QP):
// Dykstra's alternating projections on each block of reals coupled by
// multi-variable unit atoms, then the feasibility polish, with the per-restart
// ||g||^2 of Eq. grad_map.  Compiled both ahead of time (through fsmt_device.cu)
// and at run time (NVRTC, fsmt_jit.cpp), where straight-line routines with the
// block's iterate in registers are generated for the most frequent block shapes.
//
// The arithmetic is written out with explicit fused multiply-adds and correctly
// rounded operations (no contraction left to the compiler), so that a generated
// routine, which repeats it with the coefficients as constants, gives the same
// bits as the generic loop.
#pragma once

namespace fsmt {

constexpr float kPolishMargin = 1.52587890625e-05f;  // 2^-16

// Sum over the blockDim.y rows of a (32 restarts x rows) block, added to gn2[r].
__device__ __forceinline__ void reduce_rows_add(float part, float* gn2, int r, bool ok) {
  __shared__ float red[8][33];
  red[threadIdx.y][threadIdx.x] = part;
  __syncthreads();
  if (threadIdx.y == 0) {
    float s = 0.f;
    for (int y = 0; y < (int)blockDim.y; ++y) s += red[y][threadIdx.x];
    if (ok && s != 0.f) atomicAdd(gn2 + r, s);
  }
}

// The step of restart r: eta, or eta * n_obj / wsum[r] when the step is normalised
// by the total weight (Thm. max_step with L proportional to the weight, Prop. Lipschitz).
__device__ __forceinline__ float restart_eta(const DevView& d, float eta, const float* prm, const float* wsum,
                                             int r, bool ok) {
  eta = load_param(prm, P_ETA, eta);
  if (prm && prm[P_NORM] == 0.f) wsum = nullptr;
  if (wsum && ok && d.n_obj > 0) {
    const float ws = wsum[r];
    if (ws > 0.f) eta *= (float)d.n_obj / ws;
  }
  return eta;
}

// The arithmetic of one Dykstra half-space term, one box step and one polish term,
// shared by the generic loop and the generated routines.
__device__ __forceinline__ float proj_dot(float cf, float x, float th, float dot) { return fmaf(cf, fmaf(th, cf, x), dot); }
__device__ __forceinline__ float proj_tn(float dot, float iq) { return __fmul_rn(fmaxf(dot, 0.f), iq); }
// Dykstra's multiplier of an equality's hyperplane: not clamped at zero (an affine set).
__device__ __forceinline__ float proj_tn_eq(float dot, float iq) { return __fmul_rn(dot, iq); }
// The band within which an equality's residual counts as zero in FP32: (n + 4) (u mag +
// 2^-126-ish), u = 2^-24 (the bound of an n-term FP32 dot product; Higham, Accuracy and
// Stability of Numerical Algorithms, 2nd ed., Sec. 3.1).
__device__ __forceinline__ float proj_eq_band(int n, float mag) {
  return (float)(n + 4) * fmaf(5.9604645e-8f, mag, 1e-38f);
}
__device__ __forceinline__ float proj_box(float& x, float p, float lo, float hi) {  // returns the new correction
  const float yv = __fadd_rn(x, p);
  const float xn = fminf(fmaxf(yv, lo), hi);
  x = xn;
  return __fsub_rn(yv, xn);
}

// A block shape's generated routine (rank shape >= 1) runs the whole projection of
// one (block, restart) and returns true; false leaves it to the generic loop.
__device__ __forceinline__ bool proj_dispatch(int shape, const float* s_q0, const float* s_lo, const float* s_hi,
                                              float* b, float* gb, const int* cvar, int R, int r, float step,
                                              float inv, int sweeps, int polish, int clear_grad, bool act,
                                              float& part);

// One thread per (block, restart); a warp serves one block for 32 restarts.  Per
// sweep: every half-space in constraint order, then the box.  Then up to `polish`
// passes: each half-space q.y <= q0 whose value is above -margin, margin = 2^-16
// (|q0| + sum |q_j y_j|) (far above the FP32 rounding of q.y), is projected onto
// q.y <= q0 - 2 margin along the reals not pinned at the bound the step would
// cross, then the box is clamped; the thread stops at the first pass that moves
// nothing, so the point it returns satisfies every half-space exactly whenever
// the passes settle.  An equality's hyperplane q.y = q0 takes Dykstra's step with an
// unclamped multiplier, and in the polish it is projected back onto itself (along the
// reals not pinned at the bound the move would cross) while its residual exceeds
// proj_eq_band; the exact repair on the host finishes it.
// Shared memory: the iterate, Dykstra's box corrections and half-space
// multipliers of each (block, restart), one column per thread ([var][thread]:
// conflict-free), sized by the instance's largest block; and per warp the block
// itself (half-space offsets, local reals, coefficients, right-hand sides,
// 1/||q||^2, the box), staged once by the warp's lanes together so that the
// sweeps read it by broadcast instead of through dependent global loads.
// The work of one thread: restart tile `tile`, blocks c0, c0 + cstride, ...; ty is
// the warp's place among the T / 32 warps that share s_col (the columns' stride is
// T).  Returns the thread's part of ||g||^2 for its restart.
__device__ __forceinline__ float pgd_comp_core(const DevView& d, int R, float eta, float bscale, int sweeps,
                                               int polish, const float* prm, const float* __restrict__ wsum,
                                               float* __restrict__ b, float* __restrict__ gb,
                                               const uint8_t* __restrict__ active, int clear_grad, int maxv,
                                               int maxh, int maxnz, int tile, int c0, int cstride, int ty, int T,
                                               float* s_col) {
  const int lane = threadIdx.x & 31;
  const int r = tile * 32 + lane;
  const bool ok = r < R;
  const bool act = ok && (!active || active[r] == 1);
  eta = restart_eta(d, eta, prm, wsum, r, ok);
  bscale = load_param(prm, P_BSCALE, bscale);
  if (prm) {
    sweeps = (int)prm[P_SWEEPS];
    polish = (int)prm[P_POLISH];
  }
  const float step = eta * bscale * bscale, inv = 1.f / (bscale * eta);
  float part = 0.f;
  const int tid = ty * 32 + lane;
  float* xs = s_col + tid;           // x(t) at xs[t * T]
  float* ps = xs + maxv * T;         // pbox(t)
  float* hs = ps + maxv * T;         // th(q)
  // the warp's staged block
  const int wwords = (maxh + 1) + 2 * maxnz + 3 * maxh + 2 * maxv;
  int* s_hp = reinterpret_cast<int*>(s_col + (2 * maxv + maxh) * T) + ty * wwords;  // offsets [nh + 1]
  int* s_lv = s_hp + maxh + 1;                                   // local real of each term
  float* s_cf = reinterpret_cast<float*>(s_lv + maxnz);          // coefficient of each term
  float* s_q0 = s_cf + maxnz;                                    // right-hand sides
  float* s_iq = s_q0 + maxh;                                     // 1 / ||q||^2
  float* s_lo = s_iq + maxh;                                     // the box of each local real
  float* s_hi = s_lo + maxv;
  int* s_eq = reinterpret_cast<int*>(s_hi + maxv);                // 1: an equality's hyperplane
#define x(t) xs[(t) * T]
#define pbox(t) ps[(t) * T]
#define th(q) hs[(q) * T]
  for (int c = c0; c < d.n_comp; c += cstride) {
    const int v0 = d.comp_var_ptr[c], nv = d.comp_var_ptr[c + 1] - v0;
    const int h0 = d.comp_hs_ptr[c], nh = d.comp_hs_ptr[c + 1] - h0;
    const int e_base = d.hs_ptr[h0], nz = d.hs_ptr[h0 + nh] - e_base;
    __syncwarp();  // the previous block's reads are done
    for (int i = lane; i <= nh; i += 32) s_hp[i] = d.hs_ptr[h0 + i] - e_base;
    for (int i = lane; i < nz; i += 32) {
      s_lv[i] = d.hs_lvar[e_base + i];
      s_cf[i] = d.hs_coef[e_base + i];
    }
    for (int i = lane; i < nh; i += 32) {
      s_q0[i] = d.hs_q0[h0 + i];
      s_iq[i] = d.hs_inv_qq[h0 + i];
      s_eq[i] = d.hs_eq[h0 + i];
    }
    for (int i = lane; i < nv; i += 32) {
      const int j = d.comp_var[v0 + i];
      s_lo[i] = d.lo[j];
      s_hi[i] = d.hi[j];
    }
    __syncwarp();
    if (!ok) continue;
    const int shape = d.comp_shape[c];
    if (shape > 0 && proj_dispatch(shape, s_q0, s_lo, s_hi, b, gb, d.comp_var + v0, R, r, step, inv, sweeps, polish,
                                   clear_grad, act, part))
      continue;
    for (int t = 0; t < nv; ++t) {
      const size_t k = (size_t)d.comp_var[v0 + t] * R + r;
      x(t) = fmaf(-step, gb[k], b[k]);
      pbox(t) = 0.f;
      if (clear_grad) gb[k] = 0.f;
    }
    for (int q = 0; q < nh; ++q) th(q) = 0.f;
    for (int sw = 0; sw < sweeps; ++sw) {
      for (int q = 0; q < nh; ++q) {
        const int e0 = s_hp[q], e1 = s_hp[q + 1];
        const float thq = th(q);
        float dot = -s_q0[q];
        for (int e = e0; e < e1; ++e) dot = proj_dot(s_cf[e], x(s_lv[e]), thq, dot);
        const float tn = s_eq[q] ? proj_tn_eq(dot, s_iq[q]) : proj_tn(dot, s_iq[q]);
        const float delta = __fsub_rn(thq, tn);
        for (int e = e0; e < e1; ++e) x(s_lv[e]) = fmaf(delta, s_cf[e], x(s_lv[e]));
        th(q) = tn;
      }
      for (int t = 0; t < nv; ++t) {
        float xt = x(t);
        pbox(t) = proj_box(xt, pbox(t), s_lo[t], s_hi[t]);
        x(t) = xt;
      }
    }
    if (sweeps == 0)
      for (int t = 0; t < nv; ++t) x(t) = fminf(fmaxf(x(t), s_lo[t]), s_hi[t]);
    for (int pass = 0; pass < polish; ++pass) {
      bool moved = false;
      for (int q = 0; q < nh; ++q) {
        const int e0 = s_hp[q], e1 = s_hp[q + 1];
        const float q0 = s_q0[q];
        float v = -q0, mag = fabsf(q0);
        for (int e = e0; e < e1; ++e) {
          const float term = __fmul_rn(s_cf[e], x(s_lv[e]));
          v = __fadd_rn(v, term);
          mag = __fadd_rn(mag, fabsf(term));
        }
        if (s_eq[q]) {  // back onto the hyperplane when off it by more than the FP32 band
          if (fabsf(v) > proj_eq_band(e1 - e0, mag)) {
            float qq = 0.f;
            for (int e = e0; e < e1; ++e) {
              const float cf = s_cf[e];
              const int t = s_lv[e];
              const bool down = (v > 0.f) == (cf > 0.f);  // the move -(v/qq) cf lowers x(t)
              const bool pinned = down ? x(t) <= s_lo[t] : x(t) >= s_hi[t];
              if (!pinned) qq = fmaf(cf, cf, qq);
            }
            if (qq > 0.f) {
              const float tq = __fdiv_rn(v, qq);
              for (int e = e0; e < e1; ++e) {
                const float cf = s_cf[e];
                const int t = s_lv[e];
                const bool down = (v > 0.f) == (cf > 0.f);
                const bool pinned = down ? x(t) <= s_lo[t] : x(t) >= s_hi[t];
                if (!pinned) x(t) = fmaf(-tq, cf, x(t));
              }
              moved = true;
            }
          }
          continue;
        }
        const float margin = __fmul_rn(kPolishMargin, mag);
        if (v > -margin) {
          // move along the reals that are not pinned at the bound the step would cross
          float qq = 0.f;
          for (int e = e0; e < e1; ++e) {
            const float cf = s_cf[e];
            const int t = s_lv[e];
            const bool pinned = (cf > 0.f && x(t) <= s_lo[t]) || (cf < 0.f && x(t) >= s_hi[t]);
            if (!pinned) qq = fmaf(cf, cf, qq);
          }
          if (qq > 0.f) {
            const float tq = __fdiv_rn(__fadd_rn(v, __fmul_rn(2.f, margin)), qq);
            for (int e = e0; e < e1; ++e) {
              const float cf = s_cf[e];
              const int t = s_lv[e];
              const bool pinned = (cf > 0.f && x(t) <= s_lo[t]) || (cf < 0.f && x(t) >= s_hi[t]);
              if (!pinned) x(t) = fmaf(-tq, cf, x(t));
            }
            moved = true;
          }
        }
      }
      for (int t = 0; t < nv; ++t) x(t) = fminf(fmaxf(x(t), s_lo[t]), s_hi[t]);
      if (!moved) break;
    }
    for (int t = 0; t < nv; ++t) {
      const size_t k = (size_t)d.comp_var[v0 + t] * R + r;
      const float q = __fmul_rn(__fsub_rn(b[k], x(t)), inv);  // b still holds the step's starting point
      part = fmaf(q, q, part);
      if (act) b[k] = x(t);
    }
  }
#undef x
#undef pbox
#undef th
  return part;
}

// The projection kernel's body: CTA (32 restarts, blockDim.y blocks of reals), grid
// (restart tiles, groups of blocks); the CTA's ||g||^2 parts summed over its rows.
__device__ __forceinline__ void pgd_comp_body(const DevView& d, int R, float eta, float bscale, int sweeps,
                                              int polish, const float* prm, const float* __restrict__ wsum,
                                              float* __restrict__ b, float* __restrict__ gb,
                                              float* __restrict__ gn2, const uint8_t* __restrict__ active,
                                              int clear_grad, const int* ctl, int maxv, int maxh, int maxnz) {
  if (ctl && ctl[0] == 0) return;
  extern __shared__ float s_col[];
  const int r = blockIdx.x * 32 + threadIdx.x;
  const float part = pgd_comp_core(d, R, eta, bscale, sweeps, polish, prm, wsum, b, gb, active, clear_grad, maxv,
                                   maxh, maxnz, blockIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
                                   gridDim.y * blockDim.y, threadIdx.y, blockDim.x * blockDim.y, s_col);
  reduce_rows_add(part, gn2, r, r < R);
}

#ifndef FSMT_JIT_PROJ
// Ahead-of-time build: no generated projection routines, every block takes the generic loop.
__device__ __forceinline__ bool proj_dispatch(int, const float*, const float*, const float*, float*, float*,
                                              const int*, int, int, float, float, int, int, int, bool, float&) {
  return false;
}
#endif

}  // namespace fsmt
