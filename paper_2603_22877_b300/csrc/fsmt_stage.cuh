// Device code of one annealing stage run as ONE persistent kernel: every iteration
// of the stage (Alg. 1's loop body -- fused forward + adjoint, PGD step with the
// projection, the epsilon test of Eq. critical) inside a single cooperative launch,
// the phases separated by grid-wide barriers.  Compiled both ahead of time (the
// epsilon test, through fsmt_device.cu) and at run time (NVRTC, fsmt_jit.cpp), where
// the stage kernels take the generated diagram and projection routines.
#pragma once

namespace fsmt {

// Eq. critical per restart after an iteration: the iteration just run is counted,
// a restart whose ||g||^2 <= eps^2 stops (active 0); one whose ||g||^2 is not finite
// stops with active 2 and error bit 1 in ctl[1] (its point may already have been
// clamped back into the box, so the round check marks it from active).  ctl[0] =
// restarts still iterating.  All threads of one CTA.
__device__ __forceinline__ void converge_block(int R, float eps, const float* gn2, uint8_t* active, int* iters,
                                               int* ctl) {
  const float eps2 = eps * eps;
  int cnt = 0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (active[r] != 1) continue;
    iters[r] += 1;
    const float g = gn2[r];
    if (!isfinite(g)) {
      active[r] = 2;
      atomicOr(ctl + 1, 1);
    } else if (g <= eps2) {
      active[r] = 0;
    } else {
      ++cnt;
    }
  }
  __shared__ int red[32];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __syncthreads();  // red[] is free (a caller may run this twice in a row)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    ctl[0] = s;
  }
}

// ctl[1] error bit of a grid barrier that gave up waiting
constexpr int kCtlBarrierTimeout = 4;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over the CTAs of a cooperative launch (all co-resident).  ctl[2]
// counts arrivals, ctl[3] is the generation.  After a CTA barrier, one thread per CTA
// fences (cumulatively, for the writes its CTA made before the CTA barrier) and
// arrives; the last CTA to arrive runs serial() with all its threads, resets the
// count and opens the next generation; the others wait for it and fence again before
// their CTA barrier.  The wait is bounded: after limit_ns (or 2^31 polls) the CTA sets
// kCtlBarrierTimeout in ctl[1] and the barrier returns false, and the caller returns at
// once (a CTA that never arrives -- it cannot, in a cooperative launch -- costs the
// others one limit each, never a hang).  The fences make every write before the
// barrier visible to every read after it (weak loads included; the read-only path
// excluded).
template <class F>
__device__ __forceinline__ bool grid_barrier(int* ctl, unsigned long long limit_ns, F&& serial) {
  __shared__ int s_role;  // 1: the last CTA to arrive, 0: released, -1: gave up
  unsigned* cnt = reinterpret_cast<unsigned*>(ctl + 2);
  volatile unsigned* gen = reinterpret_cast<volatile unsigned*>(ctl + 3);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(cnt, 1u) + 1u;
    int role = 0;
    if (arrived == gridDim.x) {
      role = 1;
    } else {
      const unsigned long long t0 = global_ns();
      for (unsigned polls = 0;; ++polls) {
        if (*gen != g0) break;
        if (polls >= (1u << 31) || ((polls & 15u) == 15u && global_ns() - t0 > limit_ns)) {
          atomicOr(ctl + 1, kCtlBarrierTimeout);
          role = -1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_role = role;
  }
  __syncthreads();
  const int role = s_role;
  if (role == 1) {
    serial();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(const_cast<unsigned*>(gen), 1u);
    }
  }
  return role >= 0;
}

// Everything the stage kernel reads; passed by value.
struct StageArgs {
  DevView d;                  // with chunk_real_cap of the forward + adjoint configuration
  int R, t_max, vcap;
  int proj_warps;             // warps per CTA that project blocks of reals (their shared memory fits)
  int maxv, maxh, maxnz;      // the largest block of coupled reals
  unsigned long long barrier_ns;
  const float* prm;           // stage parameters (P_*)
  const float* w;
  const float* wsum;
  float* a;
  float* b;
  float* ga;
  float* gb;
  float* obj;
  float* gn2;
  uint8_t* active;
  int* iters;
  int* ctl;
  unsigned long long* trace;  // NULL, or 1 + 2 t_max device timestamps (ns): see stage_body
  int it0;                    // stage_step_body: the iteration this launch runs
};

// The PGD phase of one iteration (Eqs. pg1, pg2, Def. Projection), the same
// arithmetic as k_pgd_bool, k_pgd_free and the projection kernel: every warp of the
// grid takes (restart tile, row phase) slots of the Booleans and the box-only reals;
// then the first proj_warps warps of each CTA project the blocks of coupled reals,
// the CTAs taking (tile, group of blocks) pairs.  The gradients are cleared as they
// are read; each lane adds its part of ||g||^2 to gn2.
__device__ __forceinline__ void stage_pgd(const StageArgs& s) {
  const DevView& d = s.d;
  const int R = s.R, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int tiles = (R + 31) >> 5;
  const int gw = blockIdx.x * W + warp, nw = gridDim.x * W;
  const int wpt = max(1, nw / tiles);  // warps per restart tile
  const float bscale = load_param(s.prm, P_BSCALE, 1.f);
  float* __restrict__ a = s.a;
  float* __restrict__ ga = s.ga;
  float* __restrict__ b = s.b;
  float* __restrict__ gb = s.gb;
  for (int sl = gw; sl < wpt * tiles; sl += nw) {
    const int tile = sl / wpt, ph = sl - tile * wpt, r = tile * 32 + lane;
    const bool ok = r < R;
    const bool act = ok && s.active[r] == 1;
    const float eta = restart_eta(d, 1.f, s.prm, s.wsum, r, ok);
    const float inv = 1.f / eta;
    const float step = eta * bscale * bscale, inv_b = 1.f / (bscale * eta);
    float part = 0.f;
    if (ok) {
      // kRows rows a pass, their loads issued together (a warp walks many rows)
      constexpr int kRows = 4;
      for (int i0 = ph; i0 < d.n_bool; i0 += kRows * wpt) {
        float av[kRows], g[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          const int i = i0 + u * wpt;
          av[u] = i < d.n_bool ? a[(size_t)i * R + r] : 0.f;
          g[u] = i < d.n_bool ? ga[(size_t)i * R + r] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          const int i = i0 + u * wpt;
          if (i >= d.n_bool) break;
          const size_t k = (size_t)i * R + r;
          const float an = fminf(fmaxf(av[u] - eta * g[u], -1.f), 1.f);
          const float q = (av[u] - an) * inv;
          part = fmaf(q, q, part);
          if (act) a[k] = an;
          ga[k] = 0.f;
        }
      }
      for (int t0 = ph; t0 < d.n_free; t0 += kRows * wpt) {
        float bv[kRows], g[kRows];
        int jj[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          const int t = t0 + u * wpt;
          jj[u] = t < d.n_free ? d.free_var[t] : 0;
          bv[u] = t < d.n_free ? b[(size_t)jj[u] * R + r] : 0.f;
          g[u] = t < d.n_free ? gb[(size_t)jj[u] * R + r] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
          const int t = t0 + u * wpt;
          if (t >= d.n_free) break;
          const int j = jj[u];
          const size_t k = (size_t)j * R + r;
          const float bn = fminf(fmaxf(bv[u] - step * g[u], d.lo[j]), d.hi[j]);
          const float q = (bv[u] - bn) * inv_b;
          part = fmaf(q, q, part);
          if (act) b[k] = bn;
          gb[k] = 0.f;
        }
      }
    }
    if (ok && part != 0.f) atomicAdd(s.gn2 + r, part);
  }
  if (d.n_comp > 0 && warp < s.proj_warps) {
    extern __shared__ float s_col[];
    const int gy = max(1, (int)gridDim.x / tiles);  // CTAs per restart tile
    for (int vb = blockIdx.x; vb < tiles * gy; vb += gridDim.x) {
      const int tile = vb % tiles, yb = vb / tiles;
      const float part = pgd_comp_core(d, R, 1.f, 1.f, 0, 0, s.prm, s.wsum, s.b, s.gb, s.active, 1, s.maxv, s.maxh,
                                       s.maxnz, tile, yb * s.proj_warps + warp, gy * s.proj_warps, warp,
                                       32 * s.proj_warps, s_col);
      const int r = tile * 32 + lane;
      if (r < R && part != 0.f) atomicAdd(s.gn2 + r, part);
    }
  }
}

// The stage's iterations.  Before the launch: obj and gn2 zeroed, ctl[0] = R,
// ctl[2] = 0, wsum taken.  Per iteration: the forward + adjoint phase (fwd_adj(),
// accumulating the gradients and obj), a barrier, the PGD phase (gn2), a barrier
// whose last CTA applies the epsilon test and, when another iteration follows,
// zeroes obj and gn2 for it.  The loop ends when no restart is iterating, after
// t_max iterations, or when a barrier gave up (ctl[1] bit kCtlBarrierTimeout).
// The epsilon test after an iteration (one CTA), and when another iteration follows,
// obj and gn2 zeroed for it.
__device__ __forceinline__ void stage_converge(const StageArgs& s, bool more) {
  converge_block(s.R, load_param(s.prm, P_EPS, 0.f), s.gn2, s.active, s.iters, s.ctl);
  __syncthreads();
  if (more && *(const volatile int*)s.ctl != 0)
    for (int r = threadIdx.x; r < s.R; r += blockDim.x) {
      s.obj[r] = 0.f;
      s.gn2[r] = 0.f;
    }
}

// With s.trace, thread 0 of CTA 0 records the global timer at the start and as each
// barrier opens: trace[0] = start, trace[1 + 2 it] = end of iteration it's forward +
// adjoint phase (its slowest CTA), trace[2 + 2 it] = end of its PGD phase and
// epsilon test.
// One iteration per launch (iteration s.it0 of s.t_max; the stage launches it t_max
// times): the same phases and barriers as stage_body, with no loop around them.
template <class FwdAdj>
__device__ __forceinline__ void stage_step_body(const StageArgs& s, FwdAdj&& fwd_adj) {
  const volatile int* n_iter = s.ctl;
  if (*n_iter == 0) return;  // every restart stopped in an earlier iteration
  const int it = s.it0;
  const bool rec = s.trace && blockIdx.x == 0 && threadIdx.x == 0;
  if (rec && it == 0) s.trace[0] = global_ns();
  fwd_adj();
  if (!grid_barrier(s.ctl, s.barrier_ns, [] {})) return;
  if (rec) s.trace[1 + 2 * it] = global_ns();
  stage_pgd(s);
  const bool more = it + 1 < s.t_max;
  if (!grid_barrier(s.ctl, s.barrier_ns, [&] { stage_converge(s, more); })) return;
  if (rec) s.trace[2 + 2 * it] = global_ns();
}

template <class FwdAdj>
__device__ __forceinline__ void stage_body(const StageArgs& s, FwdAdj&& fwd_adj) {
  const volatile int* n_iter = s.ctl;
  const bool rec = s.trace && blockIdx.x == 0 && threadIdx.x == 0;
  if (rec) s.trace[0] = global_ns();
  for (int it = 0; it < s.t_max; ++it) {
    if (*n_iter == 0) break;
    fwd_adj();
    if (!grid_barrier(s.ctl, s.barrier_ns, [] {})) return;
    if (rec) s.trace[1 + 2 * it] = global_ns();
    stage_pgd(s);
    const bool more = it + 1 < s.t_max;
    const bool ok = grid_barrier(s.ctl, s.barrier_ns, [&] { stage_converge(s, more); });
    if (!ok) return;
    if (rec) s.trace[2 + 2 * it] = global_ns();
  }
}

}  // namespace fsmt
