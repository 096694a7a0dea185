// Device side of the C ABI: upload, the relaxed-objective kernels (fused and
// plain forms), the PGD step with projection, rounding + exact check + ERWA, and
// one annealing stage replayed from a CUDA graph.  sm_103a.
//
// Layout: restart-minor.  Lane l of a warp works on restart 32*t + l of restart
// tile t, so every per-restart access of a warp is one contiguous 128-byte line,
// while the diagram structure a warp reads is the same for all its lanes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "fsmt_internal.h"
#include "fsmt_chunked.cuh"
#include "fsmt_proj.cuh"
#include "fsmt_stage.cuh"

int fsmt_fused_limit_ok(const fsmt::Compiled& C);  // below

namespace fsmt {

namespace {

constexpr int kSmemBudget = 112 * 1024;
// shared memory of the chunked kernel without the per-warp message arrays
inline size_t chunk_fixed_bytes(int rpl, int slot_cap) {
  return (size_t)kChunkMaxNodes * 8 + (size_t)kChunkMaxCons * 16 + (size_t)kChunkMaxSlots * 4 * 4 +
         (size_t)kChunkMaxTerms * 8 + (size_t)kChunkMaxReals * 4 + (size_t)kChunkMaxList * 4 +
         (size_t)slot_cap * kSlotStride * 4 * 2;
}
constexpr size_t kSmemMax = 227 * 1024;


fsmt_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FSMT_ECUDA;
}
fsmt_status cuda_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? FSMT_OK : cuda_fail(e, what); }

#define FSMT_CUDA(call, what)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

inline size_t fused_warp_bytes(int vcap) { return (size_t)vcap * 8 + (size_t)(3 * vcap + 2) * 32 * 4; }

struct FusedShape {
  int warps;
  int vcap;
  size_t smem;
};

FusedShape fused_shape(const Compiled& C, int R) {
  FusedShape f;
  f.vcap = std::max(1, C.max_nodes);
  size_t wb = fused_warp_bytes(f.vcap);
  int w = (int)std::min<size_t>(kFusedThreads / 32, std::max<size_t>(1, kSmemBudget / wb));
  f.warps = w;
  f.smem = wb * w + (R <= kMaxObjSmemR ? (size_t)R * 4 : 0);
  return f;
}

// The floating-point filter of the exact atom test: with z = sum_t c_t y_t - q0 and
// mag = sum_t |c_t y_t| + |q0| accumulated in FP32 over n terms (fused
// multiply-adds, c_t exact, q0 rounded once), sign(z) is certain when |z| exceeds
// (n + 4) (u mag + 2^-126-ish), u = 2^-24 (Higham, Accuracy and Stability of
// Numerical Algorithms, 2nd ed., Sec. 3.1, with two terms for the rounding of
// mag itself and an absolute term for results below the normal range).  Returns
// -1 (z < 0), +1 (z > 0) or 0 (inside the band: the exact test decides).
// the filter's bound on |fl(z) - z| for an n-term FP32 dot product, fn = n + 4
__device__ __forceinline__ float filter_bound(float mag, float fn) { return fn * fmaf(5.9604645e-8f, mag, 1e-38f); }
__device__ __forceinline__ int atom_filter(float z, float mag, int n) {
  if (fabsf(z) > filter_bound(mag, (float)(n + 4))) return z < 0.f ? -1 : 1;
  return 0;
}

// the exact test itself, kept out of line: rare, and register-hungry (320-bit accumulator)
__device__ __noinline__ bool atom_truth_exact_slow(const DevView& d, int lab, int R, int r,
                                                   const float* __restrict__ a, const float* __restrict__ b) {
  float p, gz;
  literal_prob(d, lab, R, r, true, -1.f, a, b, p, gz);
  return p > 0.5f;
}

// bit 31 of n_unsat[r]: restart r's point has a non-finite coordinate that the check
// read (the count in the low bits stays valid; ordering against the counts' atomic
// additions does not matter)
constexpr int kUnsatNonFinite = (int)0x80000000u;

__device__ __forceinline__ bool literal_truth_exact(const DevView& d, int lab, int R, int r,
                                                    const float* __restrict__ a, const float* __restrict__ b,
                                                    bool& bad) {
  if (lab < d.n_bool) {
    const float av = __ldg(a + (size_t)lab * R + r);
    bad |= !isfinite(av);
    return av < 0.f;
  }
  // filtered first; outside the filter's band z != 0, so the atom holds iff z < 0
  // whatever its strictness; inside it the exact path decides
  const int i = lab - d.n_bool;
  const int k0 = __ldg(d.atom_ptr + i), k1 = __ldg(d.atom_ptr + i + 1);
  const float q0 = __ldg(d.atom_q0f + i);
  float z = -q0, mag = fabsf(q0);
  for (int k = k0; k < k1; ++k) {
    const float c = __ldg(d.atom_coef + k), y = __ldg(b + (size_t)__ldg(d.atom_var + k) * R + r);
    bad |= !isfinite(y);
    z = fmaf(c, y, z);
    mag = fmaf(fabsf(c), fabsf(y), mag);
  }
  // an equality (a projected unit atom) counts as holding within the projection's polish
  // margin, 2^-16 (|q0| + sum |q_j y_j|): FP32 reals rarely meet a hyperplane exactly, the
  // polish leaves them within a few FP32 bands of it, and the host repairs them exactly
  // before its verification
  if (__ldg(d.atom_strict + i) == 2) return fabsf(z) <= kPolishMargin * mag;
  const int f = atom_filter(z, mag, k1 - k0);
  if (f != 0) return f < 0;
  return atom_truth_exact_slow(d, lab, R, r, a, b);
}

// ---------------------------------------------------------- fused kernel --
// One warp per constraint of C_sigma (fused_warp_body, fsmt_chunked.cuh).
template <bool ADJ>
__global__ void __launch_bounds__(kFusedThreads) k_fused(DevView d, int R, float sigma, const float* prm, int vcap,
                                                         const float* __restrict__ w, const float* __restrict__ a,
                                                         const float* __restrict__ b, float* __restrict__ grad_a,
                                                         float* __restrict__ grad_b, float* __restrict__ obj,
                                                         float* __restrict__ cop, const int* ctl) {
  if (ctl && ctl[0] == 0) return;
  fused_warp_body<ADJ>(d, R, sigma, prm, vcap, w, a, b, grad_a, grad_b, obj, cop);
}

// The chunked kernel compiled ahead of time (no per-shape routines: the
// default shape_dispatch of fsmt_chunked.cuh declines every shape).
template <bool ADJ, int RPL>
__global__ void __launch_bounds__(kChunkThreads, 1)
    k_chunked(DevView d, int R, float sigma, const float* prm, int vcap, const float* __restrict__ w,
              const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ grad_a,
              float* __restrict__ grad_b, float* __restrict__ obj, float* __restrict__ cop, const int* ctl) {
  chunked_body<ADJ, RPL>(d, R, sigma, prm, vcap, w, a, b, grad_a, grad_b, obj, cop, ctl);
}

// ------------------------------------------------------------ plain form --
// Separate kernels; every node's message lives in global memory (work) between
// the passes: work = m [(n_obj_nodes + 2 n_obj) x R] | p_atom [K x R] | gz [K x R].
__global__ void k_atoms_plain(DevView d, int R, float sigma, const float* __restrict__ b, float* __restrict__ p_atom,
                              float* __restrict__ gz_atom) {
  const int r = blockIdx.x * 32 + threadIdx.x;
  const bool ok = r < R;
  const float s_inv = sigma > 0.f ? kInvSqrt2 / sigma : -1.f;  // < 0: sigma = 0, exact; 0: sigma = inf
  for (int i = blockIdx.y * blockDim.y + threadIdx.y; i < d.n_atoms; i += gridDim.y * blockDim.y) {
    float p, gz;
    literal_prob(d, d.n_bool + i, R, r, ok, s_inv, nullptr, b, p, gz);
    if (ok) {
      p_atom[(size_t)i * R + r] = p;
      gz_atom[(size_t)i * R + r] = gz;
    }
  }
}

__device__ __forceinline__ float plain_prob(const DevView& d, int lab, int R, int r, bool ok, const float* a,
                                            const float* p_atom) {
  if (!ok) return 0.f;
  if (lab < d.n_bool) return 0.5f * (1.f - a[(size_t)lab * R + r]);
  return p_atom[(size_t)(lab - d.n_bool) * R + r];
}

__global__ void k_fwd_plain(DevView d, int R, const float* __restrict__ w, const float* __restrict__ a,
                            const float* __restrict__ p_atom, float* __restrict__ m, float* __restrict__ cop,
                            float* __restrict__ obj) {
  const int lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  const int n_tiles = (R + 31) >> 5;
  for (int s = blockIdx.x * W + (threadIdx.x >> 5); s < d.n_obj; s += gridDim.x * W) {
    const int nb = d.con_ptr[s];
    const int V = d.con_ptr[s + 1] - nb;
    const int cid = d.con_id[s];
    float* ms = m + (size_t)(nb + 2 * s) * R;
    for (int t = 0; t < n_tiles; ++t) {
      const int r = t * 32 + lane;
      const bool ok = r < R;
      if (!ok) continue;
      for (int v = 0; v < V + 2; ++v) ms[(size_t)v * R + r] = 0.f;
      ms[(size_t)d.con_root[s] * R + r] = 1.f;
      for (int v = 0; v < V; ++v) {
        const uint2 nd = d.nodes[nb + v];
        const int hi = nd.y & 0xffff, lo = nd.y >> 16;
        const float p = plain_prob(d, (int)nd.x, R, r, ok, a, p_atom);
        const float mv = ms[(size_t)v * R + r];
        ms[(size_t)hi * R + r] += p * mv;
        ms[(size_t)lo * R + r] += (1.f - p) * mv;
      }
      const float cp = ms[(size_t)V * R + r];
      if (cop) cop[(size_t)cid * R + r] = cp;
      if (obj) atomicAdd(obj + r, w[(size_t)cid * R + r] * (1.f - 2.f * cp));
    }
  }
}

__global__ void k_adj_plain(DevView d, int R, const float* __restrict__ w, const float* __restrict__ a,
                            const float* __restrict__ p_atom, const float* __restrict__ gz_atom,
                            float* __restrict__ m, float* __restrict__ grad_a, float* __restrict__ grad_b) {
  const int lane = threadIdx.x & 31;
  const int W = blockDim.x >> 5;
  const int n_tiles = (R + 31) >> 5;
  for (int s = blockIdx.x * W + (threadIdx.x >> 5); s < d.n_obj; s += gridDim.x * W) {
    const int nb = d.con_ptr[s];
    const int V = d.con_ptr[s + 1] - nb;
    const int cid = d.con_id[s];
    float* ms = m + (size_t)(nb + 2 * s) * R;
    for (int t = 0; t < n_tiles; ++t) {
      const int r = t * 32 + lane;
      if (r >= R) continue;
      const float wc = w[(size_t)cid * R + r];
      ms[(size_t)V * R + r] = 1.f;
      ms[(size_t)(V + 1) * R + r] = 0.f;
      for (int v = V - 1; v >= 0; --v) {
        const uint2 nd = d.nodes[nb + v];
        const int hi = nd.y & 0xffff, lo = nd.y >> 16;
        const float p = plain_prob(d, (int)nd.x, R, r, true, a, p_atom);
        const float mh = ms[(size_t)hi * R + r], ml = ms[(size_t)lo * R + r];
        const float td = ms[(size_t)v * R + r];
        const float diff = mh - ml;
        ms[(size_t)v * R + r] = p * mh + (1.f - p) * ml;
        const int lab = (int)nd.x;
        const float gz = lab < d.n_bool ? 0.f : gz_atom[(size_t)(lab - d.n_bool) * R + r];
        scatter_grad(d, lab, R, r, wc * td * diff, gz, grad_a, grad_b);
      }
    }
  }
}

// ------------------------------------------------------------- PGD step --
// Eq. pg1 / pg2 with the b-step scaled by b_scale^2, projection onto D, and the
// per-restart ||g||^2 of Eq. grad_map.  Block = 32 restarts x 8 row groups.
// With wsum (per-restart total weight of C_sigma) the step of restart r is
// eta * n_obj / wsum[r] (Thm. max_step: eta = 1/L with L proportional to the
// total weight, Prop. Lipschitz).
// reduce_rows_add and restart_eta: fsmt_proj.cuh

__global__ void k_pgd_bool(DevView d, int R, float eta, const float* prm, const float* __restrict__ wsum,
                           float* __restrict__ a, float* __restrict__ ga, float* __restrict__ gn2,
                           const uint8_t* __restrict__ active, int clear_grad, const int* ctl) {
  if (ctl && ctl[0] == 0) return;
  const int r = blockIdx.x * 32 + threadIdx.x;
  const bool ok = r < R;
  const bool act = ok && (!active || active[r] == 1);
  eta = restart_eta(d, eta, prm, wsum, r, ok);
  const float inv = 1.f / eta;
  float part = 0.f;
  if (ok) {
    for (int i = blockIdx.y * blockDim.y + threadIdx.y; i < d.n_bool; i += gridDim.y * blockDim.y) {
      const size_t k = (size_t)i * R + r;
      const float av = a[k];
      const float g = ga[k];
      const float an = fminf(fmaxf(av - eta * g, -1.f), 1.f);
      const float q = (av - an) * inv;
      part = fmaf(q, q, part);
      if (act) a[k] = an;
      if (clear_grad) ga[k] = 0.f;
    }
  }
  reduce_rows_add(part, gn2, r, ok);
}

__global__ void k_pgd_free(DevView d, int R, float eta, float bscale, const float* prm,
                           const float* __restrict__ wsum, float* __restrict__ b, float* __restrict__ gb,
                           float* __restrict__ gn2, const uint8_t* __restrict__ active, int clear_grad,
                           const int* ctl) {
  if (ctl && ctl[0] == 0) return;
  const int r = blockIdx.x * 32 + threadIdx.x;
  const bool ok = r < R;
  const bool act = ok && (!active || active[r] == 1);
  eta = restart_eta(d, eta, prm, wsum, r, ok);
  bscale = load_param(prm, P_BSCALE, bscale);
  const float step = eta * bscale * bscale, inv = 1.f / (bscale * eta);
  float part = 0.f;
  if (ok) {
    for (int t = blockIdx.y * blockDim.y + threadIdx.y; t < d.n_free; t += gridDim.y * blockDim.y) {
      const int j = d.free_var[t];
      const size_t k = (size_t)j * R + r;
      const float bv = b[k];
      const float bn = fminf(fmaxf(bv - step * gb[k], d.lo[j]), d.hi[j]);
      const float q = (bv - bn) * inv;
      part = fmaf(q, q, part);
      if (act) b[k] = bn;
      if (clear_grad) gb[k] = 0.f;
    }
  }
  reduce_rows_add(part, gn2, r, ok);
}

// The projection of the blocks of coupled reals (fsmt_proj.cuh), compiled ahead of
// time: every block takes the generic loop.
__global__ void k_pgd_comp(DevView d, int R, float eta, float bscale, int sweeps, int polish, const float* prm,
                           const float* __restrict__ wsum, float* __restrict__ b, float* __restrict__ gb,
                           float* __restrict__ gn2, const uint8_t* __restrict__ active, int clear_grad,
                           const int* ctl, int maxv, int maxh, int maxnz) {
  pgd_comp_body(d, R, eta, bscale, sweeps, polish, prm, wsum, b, gb, gn2, active, clear_grad, ctl, maxv, maxh, maxnz);
}

// wsum[r] += sum over the constraints of C_sigma of w[c][r] (caller zeroes wsum).
__global__ void k_weight_sum(DevView d, int R, const float* __restrict__ w, float* __restrict__ wsum) {
  const int r = blockIdx.x * 32 + threadIdx.x;
  const bool ok = r < R;
  float part = 0.f;
  if (ok)
    for (int s = blockIdx.y * blockDim.y + threadIdx.y; s < d.n_obj; s += gridDim.y * blockDim.y)
      part += w[(size_t)d.con_id[s] * R + r];
  reduce_rows_add(part, wsum, r, ok);
}

// The same sum for R a multiple of 4, at streaming speed: each warp takes 32 rows of
// C_sigma at a time (their ids in one load, then broadcast) and reads each row as
// float4 columns, 512 restarts a pass (column 4 lane + 128 m of the pass, m < 4),
// two rows in flight; the lane keeps its columns' sums in registers, the CTA's
// warps meet in shared memory, and the CTA adds its sums to wsum once per pass.
constexpr int kWsumCols = 512;
__global__ void __launch_bounds__(256) k_weight_sum_rows(DevView d, int R, const float* __restrict__ w,
                                                        float* __restrict__ wsum) {
  __shared__ float s_sum[kWsumCols];
  const int lane = threadIdx.x & 31, W = blockDim.x >> 5;
  const int gw = blockIdx.x * W + (threadIdx.x >> 5), nw = gridDim.x * W;
  for (int c0 = 0; c0 < R; c0 += kWsumCols) {
    for (int i = threadIdx.x; i < kWsumCols; i += blockDim.x) s_sum[i] = 0.f;
    __syncthreads();
    float4 acc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s0 = gw * 32; s0 < d.n_obj; s0 += nw * 32) {
      const int nrow = min(32, d.n_obj - s0);
      const int myid = lane < nrow ? __ldg(d.con_id + s0 + lane) : 0;
      for (int j = 0; j < nrow; j += 2) {
        float4 v[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int id = __shfl_sync(0xffffffffu, myid, j + u);
          const bool rok = j + u < nrow;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int col = c0 + 4 * lane + 128 * m;
            v[u][m] = rok && col < R ? __ldg(reinterpret_cast<const float4*>(w + (size_t)id * R + col))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            acc[m].x += v[u][m].x;
            acc[m].y += v[u][m].y;
            acc[m].z += v[u][m].z;
            acc[m].w += v[u][m].w;
          }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int cl = 4 * lane + 128 * m;
      if (c0 + cl < R) {
        atomicAdd(s_sum + cl, acc[m].x);
        atomicAdd(s_sum + cl + 1, acc[m].y);
        atomicAdd(s_sum + cl + 2, acc[m].z);
        atomicAdd(s_sum + cl + 3, acc[m].w);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWsumCols && c0 + i < R; i += blockDim.x)
      if (s_sum[i] != 0.f) atomicAdd(wsum + c0 + i, s_sum[i]);
    __syncthreads();
  }
}

// ------------------------------------------------------- stage bookkeeping --
__global__ void k_set_params(float* prm, float sigma, float eta, float bscale, float eps, float rho, float gamma,
                             float update_w, float sweeps, float polish, float norm) {
  prm[P_SIGMA] = sigma;
  prm[P_ETA] = eta;
  prm[P_BSCALE] = bscale;
  prm[P_EPS] = eps;
  prm[P_RHO] = rho;
  prm[P_GAMMA] = gamma;
  prm[P_UPDATE_W] = update_w;
  prm[P_SWEEPS] = sweeps;
  prm[P_POLISH] = polish;
  prm[P_NORM] = norm;
}

__global__ void k_stage_begin(int R, uint8_t* active, int* iters, int* ctl) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    active[r] = 1;
    iters[r] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl[0] = R;
    ctl[1] = 0;
    ctl[2] = 0;  // the persistent stage kernel's barrier: no CTA has arrived
  }
}

__global__ void k_iter_begin(int R, float* obj, float* gn2, const int* ctl) {
  if (ctl[0] == 0) return;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    obj[r] = 0.f;
    gn2[r] = 0.f;
  }
}

// Eq. critical per restart (converge_block, fsmt_stage.cuh).  One block.  gate:
// return at once when ctl[0] is already 0 (the graph's iterations past
// convergence); eps comes from prm when it is given.
__global__ void k_converge(int R, const float* prm, float eps_arg, const float* gn2, uint8_t* active, int* iters,
                           int* ctl, int gate) {
  if (gate && ctl[0] == 0) return;
  __syncthreads();
  converge_block(R, load_param(prm, P_EPS, eps_arg), gn2, active, iters, ctl);
}

// --------------------------------------------------- round + check + ERWA --
// Weight rescale of a restart at the ERWA update: Alg. 2 multiplies every weight by
// gamma^h_c >= gamma^(rho h) each stage, so a long schedule overflows FP32 after some
// 90 stages.  The step is normalised by the restart's total weight, so a common
// factor of the weights leaves the iteration unchanged except for the scale of the
// epsilon test; when the restart's mean weight over C_sigma exceeded 2^32 during the
// stage (wsum, taken at its start), the updated weights are multiplied by 2^-32
// (exact).  No rescale without wsum or when the step is not normalised.
constexpr float kWRescaleAt = 0x1p32f, kWRescale = 0x1p-32f;
__device__ __forceinline__ float erwa_scale(const DevView& d, const float* wsum, const float* prm, int r, bool ok) {
  if (!wsum || !ok || (prm && prm[P_NORM] == 0.f)) return 1.f;
  return wsum[r] > kWRescaleAt * (float)d.n_obj ? kWRescale : 1.f;
}

// Alg. 1 rounding and an exact walk of every constraint's diagram per restart;
// Alg. 2's u_c, h_c, #Unsat and weight update.  One warp per constraint.
__global__ void k_round_check(DevView d, int R, const float* __restrict__ a, const float* __restrict__ b,
                              uint8_t* __restrict__ viol, int* __restrict__ n_unsat, float* __restrict__ w,
                              float* __restrict__ h, float rho, float gamma, int update_w, const float* prm,
                              const float* __restrict__ wsum, const uint8_t* __restrict__ active, int s_begin) {
  extern __shared__ int cnt_s[];
  for (int r = threadIdx.x; r < R; r += blockDim.x) cnt_s[r] = 0;
  __syncthreads();
  if (prm) {
    rho = prm[P_RHO];
    gamma = prm[P_GAMMA];
    update_w = prm[P_UPDATE_W] != 0.f;
  }
  const float lg = log2f(gamma);
  const int lane = threadIdx.x & 31, W = blockDim.x >> 5;
  const int n_tiles = (R + 31) >> 5;
  for (int s = s_begin + blockIdx.x * W + (threadIdx.x >> 5); s < d.n_cons; s += gridDim.x * W) {
    const int nb = __ldg(d.con_ptr + s);
    const int V = __ldg(d.con_ptr + s + 1) - nb;
    const int cid = __ldg(d.con_id + s);
    const int root = __ldg(d.con_root + s);
    for (int t = 0; t < n_tiles; ++t) {
      const int r = t * 32 + lane;
      if (r >= R) continue;
      int v = root;
      bool bad = false;
      while (v < V) {
        const uint2 nd = d.nodes[nb + v];
        v = literal_truth_exact(d, (int)nd.x, R, r, a, b, bad) ? (int)(nd.y & 0xffff) : (int)(nd.y >> 16);
      }
      if (bad) atomicOr(n_unsat + r, kUnsatNonFinite);
      const int u = v != V ? 1 : 0;
      if (viol) viol[(size_t)cid * R + r] = (uint8_t)u;
      if (u) atomicAdd(cnt_s + r, 1);
      if (h) {
        const size_t k = (size_t)cid * R + r;
        float hh = fmaf(rho, h[k], (float)u);
        if (update_w) {
          w[k] = w[k] * exp2f(hh * lg) * erwa_scale(d, wsum, prm, r, true);
          hh = 1.f;
        }
        h[k] = hh;
      }
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (cnt_s[r]) atomicAdd(n_unsat + r, cnt_s[r]);
    if (active && blockIdx.x == 0 && active[r] == 2) atomicOr(n_unsat + r, kUnsatNonFinite);
  }
}

// Round + check of the constraints of C_sigma over the chunk schedule.  Per chunk,
// the restarts in groups of TG tiles of 32 (TG: the least power of two >= the tile
// count, at most 8): (A) every literal slot's truth at
// the rounded point (x = sgn(a), exact atoms) as one 32-bit word per tile: Boolean
// slots two a warp, atom slots one a warp (the chunk's slots fall into the two
// lists as they are staged), the loads of all the group's tiles in flight together,
// the FP32 filter decided per word and the exact test only where it cannot; (B) one
// thread per (constraint, tile) evaluates the diagram bottom up on those words
// (node value = (holds & value(hi)) | (~holds & value(lo)), literal space), all 32
// restarts of the tile at once, and keeps the constraint's violation word; (C) a
// warp per tile counts #Unsat from the words.  Once every group is done, each warp
// streams whole rows of w and h (one constraint, every restart, four restarts a
// lane per vector access when R is a multiple of 4) and applies the ERWA update as
// k_round_check does.
constexpr int kCheckThreads = 512;
constexpr int kCheckTG = 8;  // the largest group: (A) unrolls over its tiles, (B) has one thread per tile
static_assert(kCheckThreads / 32 >= kCheckTG, "(C) takes a warp per tile of the group");
inline int check_group(int R) {  // TG for R restarts
  const int tiles = (R + 31) / 32;
  return tiles >= 5 ? 8 : tiles >= 3 ? 4 : tiles;
}
__host__ __device__ constexpr size_t check_smem_bytes(int R, int TG) {
  return (size_t)kChunkMaxNodes * 8 + (size_t)kChunkMaxCons * 16 + (size_t)kChunkMaxSlots * 12 +
         (size_t)kChunkMaxTerms * 8 + (size_t)kChunkMaxSlots * 4 + (size_t)kChunkMaxSlots * TG * 4 +
         (size_t)kChunkMaxNodes * TG * 4 + (size_t)((R + 31) / 32) * kChunkMaxCons * 4 + (size_t)(R + 2) * 4;
}
template <int TG>
__global__ void __launch_bounds__(kCheckThreads, TG <= 2 ? 3 : 2)
    k_check_chunked(DevView d, int R, int vcap, const float* __restrict__ a, const float* __restrict__ b,
                    uint8_t* __restrict__ viol, int* __restrict__ n_unsat, float* __restrict__ w,
                    float* __restrict__ h, float rho, float gamma, int update_w, const float* prm,
                    const float* __restrict__ wsum, const uint8_t* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint2* s_node = reinterpret_cast<uint2*>(smem);
  int4* s_con = reinterpret_cast<int4*>(s_node + kChunkMaxNodes);
  int* s_lab = reinterpret_cast<int*>(s_con + kChunkMaxCons);
  int* s_meta = s_lab + kChunkMaxSlots;                               // atoms: first term << 16 | count
  float* s_q0 = reinterpret_cast<float*>(s_meta + kChunkMaxSlots);    // atoms: q0 (FP32)
  int* s_tvar = reinterpret_cast<int*>(s_q0 + kChunkMaxSlots);        // the chunk's atom terms: global real id
  float* s_tcoef = reinterpret_cast<float*>(s_tvar + kChunkMaxTerms);
  int* s_list = reinterpret_cast<int*>(s_tcoef + kChunkMaxTerms);     // Boolean slots from the front, atom slots from the back
  unsigned* s_t = reinterpret_cast<unsigned*>(s_list + kChunkMaxSlots);  // [slot][tile of group]: holds, bit per restart
  unsigned* s_val = s_t + kChunkMaxSlots * TG;                          // [node][tile of group]: the node's value
  unsigned* s_u = s_val + kChunkMaxNodes * TG;                          // [tile][constraint]: violated bits
  const int n_tiles = (R + 31) >> 5;
  int* cnt_s = reinterpret_cast<int*>(s_u + n_tiles * kChunkMaxCons);  // [R]: #Unsat of the CTA's chunks
  int& s_nb = cnt_s[R];      // the chunk's Boolean slots
  int& s_na = cnt_s[R + 1];  // and atom slots
  for (int r = threadIdx.x; r < R; r += blockDim.x) cnt_s[r] = 0;
  if (threadIdx.x == 0) s_nb = s_na = 0;
  if (prm) {
    rho = prm[P_RHO];
    gamma = prm[P_GAMMA];
    update_w = prm[P_UPDATE_W] != 0.f;
  }
  const float lg = log2f(gamma);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  // (B) pairs a constraint with ts tiles, ts the least power of two >= min(TG, n_tiles)
  int ts_log = 0;
  while ((1 << ts_log) < min(TG, n_tiles)) ++ts_log;
  const int ts = 1 << ts_log;
  for (int q = blockIdx.x; q < d.n_chunks; q += gridDim.x) {
    const int c0 = __ldg(d.chunk_con_ptr + q), nc = __ldg(d.chunk_con_ptr + q + 1) - c0;
    const int n0 = __ldg(d.chunk_node_ptr + q), nn = __ldg(d.chunk_node_ptr + q + 1) - n0;
    const int l0 = __ldg(d.chunk_slot_ptr + q), ns = __ldg(d.chunk_slot_ptr + q + 1) - l0;
    __syncthreads();  // the previous chunk is done with shared memory
    for (int i = threadIdx.x; i < nn; i += blockDim.x) s_node[i] = d.cnodes[n0 + i];
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s_con[i] = d.ccon[c0 + i];
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
      const int raw = __ldg(d.slot_label + l0 + i), lab = raw & 0x7fffffff;
      s_lab[i] = raw;
      s_meta[i] = __ldg(d.slot_meta + l0 + i);
      if (lab >= d.n_bool) {
        s_q0[i] = __ldg(d.atom_q0f + lab - d.n_bool);
        s_list[ns - 1 - atomicAdd(&s_na, 1)] = i;
      } else {
        s_list[atomicAdd(&s_nb, 1)] = i;
      }
    }
    const int t0 = __ldg(d.chunk_term_ptr + q), nt = __ldg(d.chunk_term_ptr + q + 1) - t0;
    const int e0 = __ldg(d.chunk_real_ptr + q);
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      s_tvar[i] = __ldg(d.real_id + e0 + __ldg(d.term_var + t0 + i));
      s_tcoef[i] = __ldg(d.term_coef + t0 + i);
    }
    for (int g = 0; g < n_tiles; g += TG) {
      const int ng = min(TG, n_tiles - g);
      __syncthreads();  // chunk loaded / the previous group's walks are done with s_t
      // (A) restart r = (g + k) * 32 + lane of tile k of the group; every restart of
      // the group exists when `full`, otherwise loads past R read 0 (bits masked in B)
      const bool full = ng == TG && (R & 31) == 0;
      auto in_r = [&](int k) { return full || (k < ng && (g + k) * 32 + lane < R); };
      const int nb = s_nb, na = s_na;
      // the slot's row of TG words, 16-byte aligned
      auto store_row = [&](int i, const unsigned* word) {
        if constexpr (TG % 4 == 0) {
          uint4* row = reinterpret_cast<uint4*>(s_t + i * TG);
#pragma unroll
          for (int k = 0; k < TG; k += 4) row[k / 4] = make_uint4(word[k], word[k + 1], word[k + 2], word[k + 3]);
        } else {
#pragma unroll
          for (int k = 0; k < TG; ++k) s_t[i * TG + k] = word[k];
        }
      };
      // Booleans (holds: a < 0), two slots a warp at a time
      for (int j = warp; j < nb; j += 2 * W) {
        const bool two = j + W < nb;
        const int i0 = s_list[j], i1 = two ? s_list[j + W] : i0;
        const float* ap0 = a + (size_t)(s_lab[i0] & 0x7fffffff) * R + g * 32 + lane;
        const float* ap1 = a + (size_t)(s_lab[i1] & 0x7fffffff) * R + g * 32 + lane;
        float av0[TG], av1[TG];
#pragma unroll
        for (int k = 0; k < TG; ++k) {
          av0[k] = in_r(k) ? __ldg(ap0 + 32 * k) : 0.f;
          av1[k] = in_r(k) ? __ldg(ap1 + 32 * k) : 0.f;
        }
        const unsigned flip0 = s_lab[i0] < 0 ? 0xffffffffu : 0u, flip1 = s_lab[i1] < 0 ? 0xffffffffu : 0u;
        unsigned w0[TG], w1[TG], badm = 0;  // badm: bit k, this lane's restart of tile k is non-finite
#pragma unroll
        for (int k = 0; k < TG; ++k) {
          w0[k] = __ballot_sync(0xffffffffu, av0[k] < 0.f) ^ flip0;
          w1[k] = __ballot_sync(0xffffffffu, av1[k] < 0.f) ^ flip1;
          if (!isfinite(av0[k]) || !isfinite(av1[k])) badm |= 1u << k;
        }
        if (badm)
#pragma unroll
          for (int k = 0; k < TG; ++k)
            if ((badm >> k) & 1u) atomicOr(n_unsat + (g + k) * 32 + lane, kUnsatNonFinite);
        if (lane == 0) store_row(i0, w0);
        if (lane == 1 && two) store_row(i1, w1);
      }
      // atoms: z = q.y - q0 and the filter's magnitude; the exact test where the filter cannot decide
      for (int j = warp; j < na; j += W) {
        const int i = s_list[ns - 1 - j];
        const int raw = s_lab[i], lab = raw & 0x7fffffff;
        const unsigned flip = raw < 0 ? 0xffffffffu : 0u;
        const int meta = s_meta[i], tb = meta >> 16, tc = meta & 0xffff;
        const float q0 = s_q0[i];
        unsigned word[TG];
        float z[TG], mag[TG];
        // term jj's y at tile k (0 past R)
        auto term_y = [&](int jj, int k) -> float {
          return in_r(k) ? __ldg(b + (size_t)s_tvar[tb + jj] * R + (g + k) * 32 + lane) : 0.f;
        };
        if (tc == 2) {
          const float c0 = s_tcoef[tb], c1 = s_tcoef[tb + 1];
          float y0[TG], y1[TG];
#pragma unroll
          for (int k = 0; k < TG; ++k) {
            y0[k] = term_y(0, k);
            y1[k] = term_y(1, k);
          }
#pragma unroll
          for (int k = 0; k < TG; ++k) {
            z[k] = fmaf(c1, y1[k], fmaf(c0, y0[k], -q0));
            mag[k] = fmaf(fabsf(c1), fabsf(y1[k]), fmaf(fabsf(c0), fabsf(y0[k]), fabsf(q0)));
          }
        } else {
#pragma unroll
          for (int k = 0; k < TG; ++k) {
            z[k] = -q0;
            mag[k] = fabsf(q0);
          }
          for (int jj = 0; jj < tc; ++jj) {
            const float cj = s_tcoef[tb + jj];
            float y[TG];
#pragma unroll
            for (int k = 0; k < TG; ++k) y[k] = term_y(jj, k);
#pragma unroll
            for (int k = 0; k < TG; ++k) {
              z[k] = fmaf(cj, y[k], z[k]);
              mag[k] = fmaf(fabsf(cj), fabsf(y[k]), mag[k]);
            }
          }
        }
        // bit k of uncm: the filter cannot decide this lane's restart of tile k; of badm:
        // its magnitude is non-finite, which a non-finite y makes it
        const float fn = (float)(tc + 4);
        unsigned uncm = 0, badm = 0;
#pragma unroll
        for (int k = 0; k < TG; ++k) {
          word[k] = __ballot_sync(0xffffffffu, z[k] < 0.f) ^ flip;
          if (!(fabsf(z[k]) > filter_bound(mag[k], fn))) uncm |= 1u << k;
          if (!isfinite(mag[k])) badm |= 1u << k;
        }
        if (__any_sync(0xffffffffu, (uncm | badm) != 0)) {  // rare: exact decisions, and which reals are non-finite
#pragma unroll
          for (int k = 0; k < TG; ++k) {
            const int r = (g + k) * 32 + lane;
            const bool ok = in_r(k);
            if (ok && ((badm >> k) & 1u))
              for (int jj = 0; jj < tc; ++jj)
                if (!isfinite(__ldg(b + (size_t)s_tvar[tb + jj] * R + r))) atomicOr(n_unsat + r, kUnsatNonFinite);
            bool holds = ((word[k] ^ flip) >> lane) & 1u;  // z < 0, where the filter decides
            if (ok && ((uncm >> k) & 1u)) holds = atom_truth_exact_slow(d, lab, R, r, a, b);
            word[k] = __ballot_sync(0xffffffffu, holds) ^ flip;
          }
        }
        if (lane == 0) store_row(i, word);
      }
      __syncthreads();
      // (B) thread per (constraint c, tile k of the group)
      for (int p = threadIdx.x; p < nc << ts_log; p += blockDim.x) {
        const int c = p >> ts_log, k = p & (ts - 1), t = g + k;
        if (k >= ng) continue;
        const int4 cn = s_con[c];
        const int V = cn.y & 0xffff;
        unsigned holds_c;
        if (V == 0) {
          holds_c = cn.z == 0 ? 0xffffffffu : 0u;  // constant diagram: 0 TRUE, 1 FALSE
        } else {
          const uint2* nd = s_node + cn.x;
          unsigned* val = s_val + cn.x * TG + k;
          auto value = [&](unsigned ch) -> unsigned {  // the TRUE terminal's row is vcap, FALSE vcap + 1
            return ch < (unsigned)V ? val[ch * TG] : (ch == (unsigned)vcap ? 0xffffffffu : 0u);
          };
          for (int v = V - 1; v >= 0; --v) {
            const uint2 e = nd[v];
            const unsigned m = s_t[(e.x >> 8) * TG + k];
            val[v * TG] = (m & value(e.y & 0xffffu)) | (~m & value(e.y >> 16));
          }
          holds_c = val[0];
        }
        const unsigned valid = t * 32 + 32 <= R ? 0xffffffffu : (1u << (R - t * 32)) - 1u;
        s_u[t * kChunkMaxCons + c] = ~holds_c & valid;
      }
      __syncthreads();
      // (C) the group's #Unsat over the chunk, a warp per tile (W >= TG)
      if (warp < ng) {
        const int t = g + warp, r = t * 32 + lane;
        if (r < R) {
          int cnt = 0;
          for (int c = 0; c < nc; ++c) cnt += (int)((s_u[t * kChunkMaxCons + c] >> lane) & 1u);
          cnt_s[r] += cnt;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_nb = s_na = 0;  // read last by (A); the next chunk counts after the loop-top barrier
    // ERWA per constraint, every restart: u, then h <- rho h + u and, on update, w <- w gamma^h, h <- 1
    auto erwa = [&](size_t k, int rr, int u) {
      if (viol) viol[k] = (uint8_t)u;
      if (h) {
        float hh = fmaf(rho, h[k], (float)u);
        if (update_w) {
          w[k] = w[k] * exp2f(hh * lg) * erwa_scale(d, wsum, prm, rr, true);
          hh = 1.f;
        }
        h[k] = hh;
      }
    };
    if ((R & 3) == 0) {  // rows 16-byte aligned: four restarts per lane and access
      for (int c = warp; c < nc; c += W) {
        const size_t row = (size_t)s_con[c].w * R;
        for (int r4 = 4 * lane; r4 < R; r4 += 128) {
          const unsigned bits = (s_u[(r4 >> 5) * kChunkMaxCons + c] >> (r4 & 31)) & 15u;
          const size_t k = row + r4;
          if (viol)
            *reinterpret_cast<uchar4*>(viol + k) =
                make_uchar4(bits & 1u, (bits >> 1) & 1u, (bits >> 2) & 1u, (bits >> 3) & 1u);
          if (!h) continue;
          float4 hv = *reinterpret_cast<const float4*>(h + k);
          float hs[4] = {hv.x, hv.y, hv.z, hv.w}, ws[4];
          if (update_w) {
            const float4 wv = *reinterpret_cast<const float4*>(w + k);
            ws[0] = wv.x, ws[1] = wv.y, ws[2] = wv.z, ws[3] = wv.w;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float hh = fmaf(rho, hs[j], (float)((bits >> j) & 1u));
            if (update_w) {
              ws[j] = ws[j] * exp2f(hh * lg) * erwa_scale(d, wsum, prm, r4 + j, true);
              hh = 1.f;
            }
            hs[j] = hh;
          }
          *reinterpret_cast<float4*>(h + k) = make_float4(hs[0], hs[1], hs[2], hs[3]);
          if (update_w) *reinterpret_cast<float4*>(w + k) = make_float4(ws[0], ws[1], ws[2], ws[3]);
        }
      }
    } else {
      for (int c = warp; c < nc; c += W) {
        const size_t row = (size_t)s_con[c].w * R;
        for (int rr = lane; rr < R; rr += 32)
          erwa(row + rr, rr, (int)((s_u[(rr >> 5) * kChunkMaxCons + c] >> (rr & 31)) & 1u));
      }
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (cnt_s[r]) atomicAdd(n_unsat + r, cnt_s[r]);
    if (active && blockIdx.x == 0 && active[r] == 2) atomicOr(n_unsat + r, kUnsatNonFinite);
  }
}

// bit 31 of n_unsat[r] for every restart stopped on a non-finite ||g||^2 (active 2)
__global__ void k_mark_nonfinite(int R, const uint8_t* __restrict__ active, int* __restrict__ n_unsat) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
    if (active[r] == 2) n_unsat[r] |= kUnsatNonFinite;
}

__global__ void k_sign(int n, int R, const float* __restrict__ a, int8_t* __restrict__ x) {
  const size_t N = (size_t)n * R;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
    x[k] = a[k] < 0.f ? (int8_t)-1 : (int8_t)1;
}

// ---------------------------------------------------------------- helpers --
int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

fsmt_status check_ready(const fsmt_compiled* c, int R) {
  if (!c) {
    set_error("compiled is NULL");
    return FSMT_EINVAL;
  }
  if (!c->c.uploaded) {
    set_error("fsmt_upload has not been called");
    return FSMT_ESTATE;
  }
  if (R < 1) {
    set_error("R must be >= 1");
    return FSMT_EINVAL;
  }
  return FSMT_OK;
}

fsmt_status launch_fused_warp(const Compiled& C, bool adj, int R, float sigma, const float* prm, const float* w,
                         const float* a, const float* b, float* ga, float* gb, float* obj, float* cop, const int* ctl,
                         cudaStream_t st) {
  if (C.n_obj == 0) return FSMT_OK;
  FusedShape f = fused_shape(C, R);
  if (fused_warp_bytes(f.vcap) + (size_t)R * 4 > 220 * 1024) {
    set_error("a diagram is too large for the fused kernel; use the plain form");
    return FSMT_EINVAL;
  }
  const int threads = f.warps * 32;
  int per_sm = 1;
  if (adj)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<true>, threads, f.smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<false>, threads, f.smem);
  per_sm = std::max(per_sm, 1);
  const long need = (C.n_obj + f.warps - 1) / f.warps;
  const int blocks = (int)std::max<long>(1, std::min<long>(need, (long)sm_count() * per_sm));
  if (adj)
    k_fused<true><<<blocks, threads, f.smem, st>>>(C.view, R, sigma, prm, f.vcap, w, a, b, ga, gb, obj, cop, ctl);
  else
    k_fused<false><<<blocks, threads, f.smem, st>>>(C.view, R, sigma, prm, f.vcap, w, a, b, ga, gb, obj, cop, ctl);
  FSMT_CUDA(cudaGetLastError(), "fused kernel launch");
  return FSMT_OK;
}

// shared memory of the staged reals: b and dC/db, two tiles each
inline size_t staged_bytes(int rpl, int real_cap) { return (size_t)real_cap * rpl * 32 * 4 * 4; }

// The ways to run the forward (+ adjoint) pass on an instance at R restarts
// (the autotuner's candidates), in the order of the default choice.
std::vector<LaunchCfg> launch_candidates(const Compiled& C, int R) {
  std::vector<LaunchCfg> out;
  if (C.n_obj == 0) return out;
  const size_t obj_bytes = R <= kMaxObjSmemR ? (size_t)R * 4 : 0;
  const int vcap = std::max(1, C.max_nodes);
  const int rmax = C.stage_reals ? C.chunk_real_max : 0;
  if (C.chunked_ok) {
    for (int rpl = R > 32 ? 2 : 1; rpl >= 1; --rpl)  // generated routines, no generic path: 32 warps
      if (C.jit_wide[1][rpl - 1])
        for (int rc : {rmax, 0}) {
          const size_t smem = chunk_fixed_bytes(rpl, C.chunk_slot_cap) + staged_bytes(rpl, rc) + obj_bytes;
          if (smem <= kSmemMax) out.push_back({kVariantWide, rpl, rc, kChunkThreadsWide / 32, smem});
          if (rc == 0) break;
        }
    for (int rpl = R > 32 ? 2 : 1; rpl >= 1; --rpl)  // with the generic path's per-warp message rows
      for (int rc : {rmax, 0}) {
        const size_t per_warp = (size_t)(vcap + 2) * 32 * 4 * rpl;
        const size_t fixed = chunk_fixed_bytes(rpl, C.chunk_slot_cap) + staged_bytes(rpl, rc) + obj_bytes;
        if (fixed + per_warp <= kSmemMax) {  // down to one warp: large diagrams' messages still in shared memory
          const int warps = (int)std::min<size_t>(kChunkThreads / 32, (kSmemMax - fixed) / per_warp);
          const LaunchCfg g{kVariantGeneric, rpl, rc, warps, fixed + (size_t)warps * per_warp};
          if (C.jit_kernel[1][rpl - 1]) out.push_back({kVariantJit, rpl, rc, warps, g.smem});
          out.push_back(g);
        }
        if (rc == 0) break;
      }
  }
  if (fsmt_fused_limit_ok(C)) {
    const FusedShape f = fused_shape(C, R);
    out.push_back({kVariantWarp, 1, 0, f.warps, f.smem});
  }
  return out;
}

// The default among the candidates: generated routines without the generic
// path when every constraint has one; else the chunked kernel with two restarts
// per lane while that leaves at least 8 warps (staged reals likewise); else one
// warp per constraint.
LaunchCfg default_config(const Compiled& C, int R) {
  const std::vector<LaunchCfg> all = launch_candidates(C, R);
  LaunchCfg best{-1, 0, 0, 0, 0};
  for (const LaunchCfg& x : all) {
    if (x.variant == kVariantWide) return x;
    if (x.variant == kVariantJit || x.variant == kVariantGeneric) {
      if (best.variant < 0 || (best.warps < 8 && x.warps > best.warps)) best = x;
      continue;
    }
    if (best.variant < 0) best = x;
  }
  return best;
}

const LaunchCfg& chosen_config(const Compiled& C, int R, LaunchCfg& scratch) {
  if (C.tuned_R == R && C.tuned.variant >= 0) return C.tuned;
  scratch = default_config(C, R);
  return scratch;
}

fsmt_status launch_cfg(const Compiled& C, const LaunchCfg& x, bool adj, int R, float sigma, const float* prm,
                       const float* w, const float* a, const float* b, float* ga, float* gb, float* obj, float* cop,
                       const int* ctl, cudaStream_t st) {
  if (x.variant == kVariantWarp) return launch_fused_warp(C, adj, R, sigma, prm, w, a, b, ga, gb, obj, cop, ctl, st);
  int vcap = std::max(1, C.max_nodes);
  const dim3 g(std::max(1, std::min(C.n_chunks, sm_count()))), t(x.warps * 32);
  DevView view = C.view;
  view.chunk_real_cap = x.real_cap;
  void* args[] = {&view, &R, &sigma, (void*)&prm, &vcap, (void*)&w, (void*)&a, (void*)&b,
                  &ga, &gb, &obj, &cop, (void*)&ctl};
  if (x.variant == kVariantWide || x.variant == kVariantJit) {
    void* k = x.variant == kVariantWide ? C.jit_wide[adj ? 1 : 0][x.rpl - 1] : C.jit_kernel[adj ? 1 : 0][x.rpl - 1];
    if (!k) {
      set_error("run-time compiled kernel missing for the selected configuration");
      return FSMT_EINVAL;
    }
    FSMT_CUDA(cudaLaunchKernel((const void*)k, g, t, args, x.smem, st), "specialised kernel launch");
    return FSMT_OK;
  }
  if (x.rpl == 2) {
    if (adj)
      k_chunked<true, 2><<<g, t, x.smem, st>>>(view, R, sigma, prm, vcap, w, a, b, ga, gb, obj, cop, ctl);
    else
      k_chunked<false, 2><<<g, t, x.smem, st>>>(view, R, sigma, prm, vcap, w, a, b, ga, gb, obj, cop, ctl);
  } else {
    if (adj)
      k_chunked<true, 1><<<g, t, x.smem, st>>>(view, R, sigma, prm, vcap, w, a, b, ga, gb, obj, cop, ctl);
    else
      k_chunked<false, 1><<<g, t, x.smem, st>>>(view, R, sigma, prm, vcap, w, a, b, ga, gb, obj, cop, ctl);
  }
  FSMT_CUDA(cudaGetLastError(), "chunked kernel launch");
  return FSMT_OK;
}

fsmt_status launch_fused(const Compiled& C, bool adj, int R, float sigma, const float* prm, const float* w,
                         const float* a, const float* b, float* ga, float* gb, float* obj, float* cop, const int* ctl,
                         cudaStream_t st) {
  if (C.n_obj == 0) return FSMT_OK;
  LaunchCfg scratch;
  const LaunchCfg& x = chosen_config(C, R, scratch);
  if (x.variant < 0) {
    set_error("no kernel configuration fits this instance; use the plain form");
    return FSMT_EINVAL;
  }
  return launch_cfg(C, x, adj, R, sigma, prm, w, a, b, ga, gb, obj, cop, ctl, st);
}

fsmt_status launch_pgd(const Compiled& C, int R, float eta, float bscale, int sweeps, int polish, const float* prm,
                       const float* wsum, float* a, float* b, float* ga, float* gb, float* gn2,
                       const uint8_t* active, int clear, const int* ctl, cudaStream_t st) {
  const int tiles = (R + 31) / 32;
  const dim3 blk(32, 8);
  // enough blocks to fill the GPU a few times; each thread strides over rows
  auto rows = [&](long n) {
    const long cap = std::max<long>(1, 4L * sm_count() * 8 / tiles);
    return (int)std::max<long>(1, std::min<long>(std::min<long>((n + 7) / 8, cap), 65535L));
  };
  if (C.n_bool > 0)
    k_pgd_bool<<<dim3(tiles, rows(C.n_bool)), blk, 0, st>>>(C.view, R, eta, prm, wsum, a, ga, gn2, active, clear,
                                                            ctl);
  if (!C.free_var.empty())
    k_pgd_free<<<dim3(tiles, rows((long)C.free_var.size())), blk, 0, st>>>(C.view, R, eta, bscale, prm, wsum, b, gb,
                                                                           gn2, active, clear, ctl);
  const int ncomp = (int)C.comp_var_ptr.size() - 1;
  if (ncomp > 0) {
    // as many warps per CTA (at most 8) as the largest block's shared memory allows
    auto words = [&](int wy) { return (size_t)proj_block_words(C.comp_max_vars, C.comp_max_hs, C.comp_max_nnz, wy); };
    int wy = 8;
    while (wy > 1 && words(wy) > (size_t)kProjSmemWords) wy /= 2;
    const dim3 cblk(32, wy);
    const long cap = std::max<long>(1, 4L * sm_count() * 8 / tiles);
    const int gy = (int)std::max<long>(1, std::min<long>(std::min<long>((ncomp + wy - 1) / wy, cap), 65535L));
    if (C.jit_proj) {  // generated routines for the frequent block shapes, the generic loop for the rest
      DevView view = C.view;
      int maxv = C.comp_max_vars, maxh = C.comp_max_hs, maxnz = C.comp_max_nnz;
      void* args[] = {&view, &R, &eta, &bscale, &sweeps, &polish, (void*)&prm, (void*)&wsum, &b, &gb, &gn2,
                      (void*)&active, &clear, (void*)&ctl, &maxv, &maxh, &maxnz};
      FSMT_CUDA(cudaLaunchKernel((const void*)C.jit_proj, dim3(tiles, gy), cblk, args, words(wy) * sizeof(float), st),
                "projection kernel launch");
    } else {
      k_pgd_comp<<<dim3(tiles, gy), cblk, words(wy) * sizeof(float), st>>>(
          C.view, R, eta, bscale, sweeps, polish, prm, wsum, b, gb, gn2, active, clear, ctl, C.comp_max_vars,
          C.comp_max_hs, C.comp_max_nnz);
    }
  }
  FSMT_CUDA(cudaGetLastError(), "pgd kernel launch");
  return FSMT_OK;
}

fsmt_status launch_weight_sum(const Compiled& C, int R, const float* w, float* wsum, cudaStream_t st) {
  FSMT_CUDA(cudaMemsetAsync(wsum, 0, sizeof(float) * (size_t)R, st), "memset wsum");
  if (C.n_obj == 0) return FSMT_OK;
  if (R % 4 == 0 && R >= 128) {  // rows 16-byte aligned and at least a warp's float4 width: whole rows
    const int blocks = (int)std::max<long>(1, std::min<long>((C.n_obj + 255) / 256, (long)sm_count() * 4));
    k_weight_sum_rows<<<blocks, 256, 0, st>>>(C.view, R, w, wsum);
    FSMT_CUDA(cudaGetLastError(), "weight sum launch");
    return FSMT_OK;
  }
  const int tiles = (R + 31) / 32;
  const long cap = std::max<long>(1, 4L * sm_count() * 8 / tiles);
  const int gy = (int)std::max<long>(1, std::min<long>(std::min<long>((C.n_obj + 7) / 8, cap), 65535L));
  k_weight_sum<<<dim3(tiles, gy), dim3(32, 8), 0, st>>>(C.view, R, w, wsum);
  FSMT_CUDA(cudaGetLastError(), "weight sum launch");
  return FSMT_OK;
}

fsmt_status launch_round_check(const Compiled& C, int R, const float* a, const float* b, uint8_t* viol, int* n_unsat,
                               float* w, float* h, float rho, float gamma, int update_w, const float* prm,
                               const float* wsum, const uint8_t* active, cudaStream_t st) {
  FSMT_CUDA(cudaMemsetAsync(n_unsat, 0, sizeof(int) * (size_t)R, st), "memset n_unsat");
  if (C.n_cons == 0) return FSMT_OK;
  const int threads = 256;
  const size_t smem = (size_t)R * sizeof(int);
  if (smem > 200 * 1024) {
    set_error("R too large for round_check");
    return FSMT_EINVAL;
  }
  // constraints of C_sigma over the chunk schedule (when it exists), the rest one warp each
  int s_begin = 0;
  const int tg = check_group(R);
  const size_t csmem = check_smem_bytes(R, tg);
  if (C.chunked_ok && C.n_chunks > 0 && csmem <= kSmemMax) {
    const int fit = (int)std::max<size_t>(1, 228 * 1024 / (csmem + 1024));
    const int per_sm = std::min(fit, tg <= 2 ? 3 : 2);
    const int cblocks = std::max(1, std::min(C.n_chunks, sm_count() * per_sm));
    auto kern = tg == 1 ? k_check_chunked<1> : tg == 2 ? k_check_chunked<2> : tg == 4 ? k_check_chunked<4>
                                                                                      : k_check_chunked<8>;
    kern<<<cblocks, kCheckThreads, csmem, st>>>(C.view, R, std::max(1, C.max_nodes), a, b, viol, n_unsat, w, h, rho,
                                                gamma, update_w, prm, wsum, active);
    FSMT_CUDA(cudaGetLastError(), "chunked check launch");
    s_begin = C.n_obj;
  }
  if (s_begin < C.n_cons) {
    const int blocks =
        (int)std::max<long>(1, std::min<long>((C.n_cons - s_begin + 7) / 8, (long)sm_count() * 4));
    k_round_check<<<blocks, threads, smem, st>>>(C.view, R, a, b, viol, n_unsat, w, h, rho, gamma, update_w, prm,
                                                 wsum, active, s_begin);
    FSMT_CUDA(cudaGetLastError(), "round_check launch");
  }
  return FSMT_OK;
}

// ------------------------------------------------- persistent stage kernel --
// The stage's iterations in one cooperative launch (stage_body, fsmt_stage.cuh), or
// one such launch per iteration (stage_step_body), when the instance's run-time
// compiled stage module (jit_build_stage) holds a stage kernel for the chosen
// forward + adjoint configuration.  The PGD phase's projection runs on the first
// proj_warps warps of each CTA, as many as fit in the larger of the forward +
// adjoint phase's shared memory and 32 KB; the grid is every CTA that fits on the
// GPU at once (a cooperative launch refuses more).
struct StagePlan {
  void* kernel = nullptr;
  bool per_iteration = false;  // kernel runs one iteration a launch (the stage launches it t_max times)
  int threads = 0, blocks = 0, proj_warps = 0;
  size_t smem = 0;
  LaunchCfg cfg{-1, 0, 0, 0, 0};
};
// the per-iteration work above which the stage keeps separate launches (a barrier
// waits at most kStageBarrierNs for the slowest CTA of a phase)
constexpr double kStageMaxVisits = 1e11;
constexpr unsigned long long kStageBarrierNs = 5000000000ull;

// Compiles the stage kernels on first use (outside any stream capture: fsmt_solve_stage
// plans before it captures).
bool stage_plan(Compiled& C, int R, bool per_iteration, StagePlan& p) {
  p.per_iteration = per_iteration;
  if (C.n_obj == 0 || (double)C.n_obj_nodes * R > kStageMaxVisits) return false;
  if (!jit_build_stage(C)) return false;
  LaunchCfg scratch;
  const LaunchCfg& x = chosen_config(C, R, scratch);
  if (x.variant < 0) return false;
  int warps = 0;
  size_t smem_a = 0;
  if (x.variant == kVariantWarp) {
    const FusedShape f = fused_shape(C, R);
    p.kernel = C.jit_stage_warp[per_iteration];
    warps = f.warps;
    smem_a = f.smem;
  } else if (x.variant == kVariantWide || x.variant == kVariantJit) {
    p.kernel = C.jit_stage_chunk[per_iteration][x.variant == kVariantWide][x.rpl - 1];
    warps = x.warps;
    smem_a = x.smem;
  }
  if (!p.kernel) return false;
  const int ncomp = (int)C.comp_var_ptr.size() - 1;
  p.smem = smem_a;
  if (ncomp > 0) {
    auto bytes = [&](int wy) {
      return (size_t)proj_block_words(C.comp_max_vars, C.comp_max_hs, C.comp_max_nnz, wy) * sizeof(float);
    };
    const size_t room = std::max<size_t>(smem_a, 32 * 1024);
    int wy = warps;
    while (wy > 1 && bytes(wy) > room) --wy;
    if (bytes(wy) > kSmemMax) return false;
    p.proj_warps = wy;
    p.smem = std::max(smem_a, bytes(wy));
  }
  p.threads = warps * 32;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)p.kernel) != cudaSuccess ||
      p.smem > (size_t)fa.maxDynamicSharedSizeBytes) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)p.kernel, p.threads, p.smem) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  p.blocks = sm_count() * per_sm;
  p.cfg = x;
  return true;
}

fsmt_status launch_stage_kernel(const Compiled& C, const StagePlan& p, int t_max, int it0, fsmt_state* s,
                                cudaStream_t st) {
  StageArgs sa;
  sa.d = C.view;
  sa.d.chunk_real_cap = p.cfg.variant == kVariantWarp ? C.view.chunk_real_cap : p.cfg.real_cap;
  sa.R = s->R;
  sa.t_max = t_max;
  sa.vcap = std::max(1, C.max_nodes);
  sa.proj_warps = p.proj_warps;
  sa.maxv = C.comp_max_vars;
  sa.maxh = C.comp_max_hs;
  sa.maxnz = C.comp_max_nnz;
  sa.barrier_ns = kStageBarrierNs;
  if (const char* e = std::getenv("FSMT_STAGE_BARRIER_NS")) {  // tests of the bounded wait
    const unsigned long long v = std::strtoull(e, nullptr, 10);
    if (v > 0) sa.barrier_ns = v;
  }
  sa.prm = s->params;
  sa.w = s->w;
  sa.wsum = s->wsum;
  sa.a = s->a;
  sa.b = s->b;
  sa.ga = s->grad_a;
  sa.gb = s->grad_b;
  sa.obj = s->obj;
  sa.gn2 = s->gnorm2;
  sa.active = s->active;
  sa.iters = s->iters;
  sa.ctl = s->ctl;
  sa.trace = C.stage_trace;
  sa.it0 = it0;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(p.blocks);
  lc.blockDim = dim3(p.threads);
  lc.dynamicSmemBytes = p.smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  void* args[] = {&sa};
  FSMT_CUDA(cudaLaunchKernelExC(&lc, (const void*)p.kernel, args), "persistent stage kernel launch");
  return FSMT_OK;
}

template <typename T>
size_t push_array(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + std::max<size_t>(v.size() * sizeof(T), 1));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

}  // namespace

}  // namespace fsmt

using namespace fsmt;

int fsmt_fused_limit_ok(const fsmt::Compiled& C) {
  return fused_warp_bytes(std::max(1, C.max_nodes)) <= 200 * 1024 ? 1 : 0;
}

extern "C" {

fsmt_status fsmt_upload(fsmt_compiled* cc, void* stream) {
  if (!cc) {
    set_error("compiled is NULL");
    return FSMT_EINVAL;
  }
  Compiled& C = cc->c;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<unsigned char> blob;
  std::vector<uint2> nodes(C.node_label.size());
  for (size_t i = 0; i < nodes.size(); ++i) nodes[i] = make_uint2(C.node_label[i], C.node_hilo[i]);
  const size_t o_con_ptr = push_array(blob, C.con_ptr), o_con_id = push_array(blob, C.con_id),
               o_con_root = push_array(blob, C.con_root), o_nodes = push_array(blob, nodes),
               o_aptr = push_array(blob, C.atom_ptr), o_avar = push_array(blob, C.atom_var),
               o_acoef = push_array(blob, C.atom_coef), o_aq0f = push_array(blob, C.atom_q0f),
               o_aq0d = push_array(blob, C.atom_q0d), o_ainv = push_array(blob, C.atom_inv_norm),
               o_astr = push_array(blob, C.atom_strict), o_lo = push_array(blob, C.lo), o_hi = push_array(blob, C.hi),
               o_free = push_array(blob, C.free_var), o_cvp = push_array(blob, C.comp_var_ptr),
               o_cv = push_array(blob, C.comp_var), o_chp = push_array(blob, C.comp_hs_ptr),
               o_hsp = push_array(blob, C.hs_ptr), o_hsl = push_array(blob, C.hs_lvar),
               o_hsc = push_array(blob, C.hs_coef), o_hsq = push_array(blob, C.hs_q0),
               o_hsi = push_array(blob, C.hs_inv_qq), o_csh = push_array(blob, C.comp_shape),
               o_hse = push_array(blob, C.hs_eq);
  std::vector<uint2> cnodes(C.cnode_slot.size());
  for (size_t i = 0; i < cnodes.size(); ++i) cnodes[i] = make_uint2(C.cnode_slot[i], C.cnode_hilo[i]);
  const size_t o_ccp = push_array(blob, C.chunk_con_ptr), o_ccon = push_array(blob, C.ccon),
               o_cnp = push_array(blob, C.chunk_node_ptr), o_cnodes = push_array(blob, cnodes),
               o_csp = push_array(blob, C.chunk_slot_ptr), o_slab = push_array(blob, C.slot_label),
               o_smeta = push_array(blob, C.slot_meta), o_ctp = push_array(blob, C.chunk_term_ptr),
               o_tvar = push_array(blob, C.term_var), o_tcoef = push_array(blob, C.term_coef),
               o_crp = push_array(blob, C.chunk_real_ptr), o_rid = push_array(blob, C.real_id),
               o_clp = push_array(blob, C.chunk_list_ptr), o_clist = push_array(blob, C.clist);
  if (C.dev_block) {
    cudaFree(C.dev_block);
    C.dev_block = nullptr;
  }
  cudaError_t e = cudaMalloc(&C.dev_block, blob.size());
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FSMT_ENOMEM : FSMT_ECUDA;
  }
  FSMT_CUDA(cudaMemcpyAsync(C.dev_block, blob.data(), blob.size(), cudaMemcpyHostToDevice, st), "upload copy");
  FSMT_CUDA(cudaStreamSynchronize(st), "upload sync");
  unsigned char* base = (unsigned char*)C.dev_block;
  DevView& v = C.view;
  v.n_bool = C.n_bool;
  v.n_real = C.n_real;
  v.n_atoms = C.n_atoms;
  v.n_cons = C.n_cons;
  v.n_obj = C.n_obj;
  v.con_ptr = (const int32_t*)(base + o_con_ptr);
  v.con_id = (const int32_t*)(base + o_con_id);
  v.con_root = (const uint8_t*)(base + o_con_root);
  v.nodes = (const uint2*)(base + o_nodes);
  v.atom_ptr = (const int32_t*)(base + o_aptr);
  v.atom_var = (const int32_t*)(base + o_avar);
  v.atom_coef = (const float*)(base + o_acoef);
  v.atom_q0f = (const float*)(base + o_aq0f);
  v.atom_q0d = (const double*)(base + o_aq0d);
  v.atom_inv_norm = (const float*)(base + o_ainv);
  v.atom_strict = (const uint8_t*)(base + o_astr);
  v.lo = (const float*)(base + o_lo);
  v.hi = (const float*)(base + o_hi);
  v.n_free = (int32_t)C.free_var.size();
  v.free_var = (const int32_t*)(base + o_free);
  v.n_comp = (int32_t)C.comp_var_ptr.size() - 1;
  v.comp_var_ptr = (const int32_t*)(base + o_cvp);
  v.comp_var = (const int32_t*)(base + o_cv);
  v.comp_hs_ptr = (const int32_t*)(base + o_chp);
  v.hs_ptr = (const int32_t*)(base + o_hsp);
  v.hs_lvar = (const int32_t*)(base + o_hsl);
  v.hs_coef = (const float*)(base + o_hsc);
  v.hs_q0 = (const float*)(base + o_hsq);
  v.hs_inv_qq = (const float*)(base + o_hsi);
  v.comp_shape = (const int32_t*)(base + o_csh);
  v.hs_eq = (const uint8_t*)(base + o_hse);
  v.n_chunks = C.n_chunks;
  v.chunk_slot_cap = C.chunk_slot_cap;
  v.chunk_real_cap = 0;  // set per launch
  v.chunk_con_ptr = (const int32_t*)(base + o_ccp);
  v.ccon = (const int4*)(base + o_ccon);
  v.chunk_node_ptr = (const int32_t*)(base + o_cnp);
  v.cnodes = (const uint2*)(base + o_cnodes);
  v.chunk_slot_ptr = (const int32_t*)(base + o_csp);
  v.slot_label = (const int32_t*)(base + o_slab);
  v.slot_meta = (const int32_t*)(base + o_smeta);
  v.chunk_term_ptr = (const int32_t*)(base + o_ctp);
  v.term_var = (const int32_t*)(base + o_tvar);
  v.term_coef = (const float*)(base + o_tcoef);
  v.chunk_real_ptr = (const int32_t*)(base + o_crp);
  v.real_id = (const int32_t*)(base + o_rid);
  v.chunk_list_ptr = (const int32_t*)(base + o_clp);
  v.clist = (const uint32_t*)(base + o_clist);
  FSMT_CUDA(cudaFuncSetAttribute(k_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_round_check, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  // the block columns and the staged blocks (launch_pgd narrows the CTA when they need more)
  FSMT_CUDA(cudaFuncSetAttribute(k_pgd_comp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kProjSmemWords * sizeof(float))),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_check_chunked<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_check_chunked<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_check_chunked<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_check_chunked<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_chunked<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_chunked<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_chunked<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  FSMT_CUDA(cudaFuncSetAttribute(k_chunked<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
            "smem attribute");
  cudaGetDevice(&C.device);
  C.uploaded = true;
  jit_build(C);  // optional: falls back to the ahead-of-time chunked kernel
  const char* no_stage = std::getenv("FSMT_NO_STAGE");
  C.stage_reals = !(no_stage && no_stage[0] && std::string(no_stage) != "0");
  return FSMT_OK;
}

void fsmt_free_compiled(fsmt_compiled* cc) {
  if (!cc) return;
  if (cc->c.graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)cc->c.graph_exec);
  if (cc->c.capture_stream) cudaStreamDestroy((cudaStream_t)cc->c.capture_stream);
  if (cc->c.dev_block) cudaFree(cc->c.dev_block);
  delete cc;
}

fsmt_status fsmt_forward(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                         const float* b, float* cop, float* obj, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  if (!(sigma >= 0.f) || !w || (c->c.n_bool && !a) || (c->c.n_real && !b)) {
    set_error("invalid sigma or NULL input");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (obj) FSMT_CUDA(cudaMemsetAsync(obj, 0, sizeof(float) * (size_t)R, st), "memset obj");
  return launch_fused(c->c, false, R, sigma, nullptr, w, a, b, nullptr, nullptr, obj, cop, nullptr, st);
}

fsmt_status fsmt_adjoint(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                         const float* b, float* grad_a, float* grad_b, float* obj, float* cop, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (!(sigma >= 0.f) || !w || (C.n_bool && (!a || !grad_a)) || (C.n_real && (!b || !grad_b))) {
    set_error("invalid sigma or NULL argument");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (C.n_bool) FSMT_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(float) * (size_t)C.n_bool * R, st), "memset grad_a");
  if (C.n_real) FSMT_CUDA(cudaMemsetAsync(grad_b, 0, sizeof(float) * (size_t)C.n_real * R, st), "memset grad_b");
  if (obj) FSMT_CUDA(cudaMemsetAsync(obj, 0, sizeof(float) * (size_t)R, st), "memset obj");
  return launch_fused(C, true, R, sigma, nullptr, w, a, b, grad_a, grad_b, obj, cop, nullptr, st);
}

static fsmt_launch_config to_public(const LaunchCfg& x, float ms) {
  fsmt_launch_config o{};
  o.variant = x.variant;
  o.restarts_per_lane = x.rpl;
  o.staged_reals = x.real_cap;
  o.warps = x.warps;
  o.smem_bytes = (int64_t)x.smem;
  o.ms = ms;
  return o;
}

fsmt_status fsmt_launch_configs(const fsmt_compiled* c, int32_t R, fsmt_launch_config* out, int32_t cap,
                                int32_t* n) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  if (!n || cap < 0 || (cap > 0 && !out)) {
    set_error("invalid output arguments");
    return FSMT_EINVAL;
  }
  const std::vector<LaunchCfg> all = launch_candidates(c->c, R);
  // the default first, then the rest in enumeration order
  const LaunchCfg d = default_config(c->c, R);
  std::vector<LaunchCfg> ordered;
  if (d.variant >= 0) ordered.push_back(d);
  for (const LaunchCfg& x : all)
    if (!(x.variant == d.variant && x.rpl == d.rpl && x.real_cap == d.real_cap)) ordered.push_back(x);
  for (int i = 0; i < (int)ordered.size() && i < cap; ++i) out[i] = to_public(ordered[i], 0.f);
  *n = (int32_t)ordered.size();
  return FSMT_OK;
}

fsmt_status fsmt_select_config(fsmt_compiled* c, int32_t R, const fsmt_launch_config* cfg) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  Compiled& C = c->c;
  if (!cfg) {
    C.tuned_R = -1;
    C.tuned.variant = -1;
    return FSMT_OK;
  }
  for (const LaunchCfg& x : launch_candidates(C, R))
    if (x.variant == cfg->variant && x.rpl == cfg->restarts_per_lane && x.real_cap == cfg->staged_reals) {
      C.tuned = x;
      C.tuned_R = R;
      return FSMT_OK;
    }
  set_error("not a configuration of this instance at this R (see fsmt_launch_configs)");
  return FSMT_EINVAL;
}

fsmt_status fsmt_autotune(fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                          const float* b, float* grad_a, float* grad_b, float* obj, fsmt_launch_config* best,
                          void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  Compiled& C = c->c;
  if (!(sigma >= 0.f) || !w || (C.n_bool && (!a || !grad_a)) || (C.n_real && (!b || !grad_b))) {
    set_error("invalid sigma or NULL argument");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const std::vector<LaunchCfg> all = launch_candidates(C, R);
  if (all.empty()) {
    if (best) *best = to_public(LaunchCfg{-1, 0, 0, 0, 0}, 0.f);
    return FSMT_OK;
  }
  cudaEvent_t e0, e1;
  FSMT_CUDA(cudaEventCreate(&e0), "event");
  FSMT_CUDA(cudaEventCreate(&e1), "event");
  float best_ms = 0.f;
  int best_i = -1;
  for (int i = 0; i < (int)all.size(); ++i) {
    fsmt_status e = launch_cfg(C, all[i], true, R, sigma, nullptr, w, a, b, grad_a, grad_b, obj, nullptr, nullptr, st);
    if (e == FSMT_OK) e = cuda_ok(cudaEventRecord(e0, st), "event");
    for (int k = 0; k < 3 && e == FSMT_OK; ++k)
      e = launch_cfg(C, all[i], true, R, sigma, nullptr, w, a, b, grad_a, grad_b, obj, nullptr, nullptr, st);
    if (e == FSMT_OK) e = cuda_ok(cudaEventRecord(e1, st), "event");
    if (e == FSMT_OK) e = cuda_ok(cudaEventSynchronize(e1), "event");
    float ms = 0.f;
    if (e == FSMT_OK) e = cuda_ok(cudaEventElapsedTime(&ms, e0, e1), "event");
    if (e != FSMT_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return e;
    }
    ms /= 3.f;
    if (best_i < 0 || ms < best_ms) {
      best_ms = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  C.tuned = all[best_i];
  C.tuned_R = R;
  if (C.n_bool) FSMT_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(float) * (size_t)C.n_bool * R, st), "memset grad_a");
  if (C.n_real) FSMT_CUDA(cudaMemsetAsync(grad_b, 0, sizeof(float) * (size_t)C.n_real * R, st), "memset grad_b");
  if (obj) FSMT_CUDA(cudaMemsetAsync(obj, 0, sizeof(float) * (size_t)R, st), "memset obj");
  FSMT_CUDA(cudaStreamSynchronize(st), "synchronise");
  if (best) *best = to_public(C.tuned, best_ms);
  return FSMT_OK;
}

fsmt_status fsmt_plain_work_floats(const fsmt_compiled* c, int32_t R, int64_t* n_floats) {
  if (!c || !n_floats || R < 1) {
    set_error("invalid argument");
    return FSMT_EINVAL;
  }
  const Compiled& C = c->c;
  *n_floats = ((int64_t)C.n_obj_nodes + 2LL * C.n_obj + 2LL * C.n_atoms) * R;
  return FSMT_OK;
}

fsmt_status fsmt_forward_plain(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* work, float* cop, float* obj, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (!(sigma >= 0.f) || !w || !work || (C.n_bool && !a) || (C.n_real && !b)) {
    set_error("invalid sigma or NULL argument");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float* m = work;
  float* p_atom = work + ((size_t)C.n_obj_nodes + 2 * (size_t)C.n_obj) * R;
  float* gz_atom = p_atom + (size_t)C.n_atoms * R;
  const int tiles = (R + 31) / 32;
  if (C.n_atoms > 0) {
    k_atoms_plain<<<dim3(tiles, (unsigned)std::min<long>((C.n_atoms + 7) / 8, 4096)), dim3(32, 8), 0, st>>>(
        C.view, R, sigma, b, p_atom, gz_atom);
    FSMT_CUDA(cudaGetLastError(), "atoms kernel launch");
  }
  if (obj) FSMT_CUDA(cudaMemsetAsync(obj, 0, sizeof(float) * (size_t)R, st), "memset obj");
  if (C.n_obj > 0) {
    const int blocks = (int)std::max<long>(1, std::min<long>((C.n_obj + 7) / 8, (long)sm_count() * 8));
    k_fwd_plain<<<blocks, 256, 0, st>>>(C.view, R, w, a, p_atom, m, cop, obj);
    FSMT_CUDA(cudaGetLastError(), "plain forward launch");
  }
  return FSMT_OK;
}

fsmt_status fsmt_adjoint_plain(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* work, float* grad_a, float* grad_b, void* stream) {
  (void)sigma;
  (void)b;
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (!w || !work || (C.n_bool && (!a || !grad_a)) || (C.n_real && !grad_b)) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float* m = work;
  float* p_atom = work + ((size_t)C.n_obj_nodes + 2 * (size_t)C.n_obj) * R;
  float* gz_atom = p_atom + (size_t)C.n_atoms * R;
  if (C.n_bool) FSMT_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(float) * (size_t)C.n_bool * R, st), "memset grad_a");
  if (C.n_real) FSMT_CUDA(cudaMemsetAsync(grad_b, 0, sizeof(float) * (size_t)C.n_real * R, st), "memset grad_b");
  if (C.n_obj > 0) {
    const int blocks = (int)std::max<long>(1, std::min<long>((C.n_obj + 7) / 8, (long)sm_count() * 8));
    k_adj_plain<<<blocks, 256, 0, st>>>(C.view, R, w, a, p_atom, gz_atom, m, grad_a, grad_b);
    FSMT_CUDA(cudaGetLastError(), "plain adjoint launch");
  }
  return FSMT_OK;
}

// ------------------------------------------------ allocation-free variant --
// Work memory of fsmt_plain_noalloc: a fixed array in the library's device image,
// present on every GPU that loads the library until the process exits.  Host
// code must not use the symbol as a pointer: its device address is looked up once
// per device with cudaGetSymbolAddress.
namespace {
constexpr int64_t kNoAllocWorkFloats = int64_t(1) << 24;  // 16 Mi floats = 64 MiB
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace
static __device__ __align__(256) float g_noalloc_work[kNoAllocWorkFloats];

static fsmt_status noalloc_work_ptr(float** out) {
  int dev = 0;
  FSMT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("fsmt_plain_noalloc supports device ordinals below 64");
    return FSMT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    FSMT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_work), "cudaGetSymbolAddress of the work array");
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return FSMT_OK;
}

fsmt_status fsmt_plain_noalloc(const fsmt_compiled* c, int32_t R, float sigma, const float* w, const float* a,
                               const float* b, float* grad_a, float* grad_b, float* cop, float* obj, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  int64_t need = 0;
  s = fsmt_plain_work_floats(c, R, &need);
  if (s != FSMT_OK) return s;
  if (need > kNoAllocWorkFloats) {
    set_error("fsmt_plain_noalloc: this instance needs " + std::to_string(need) +
              " work floats at this R, more than the fixed array of " + std::to_string(kNoAllocWorkFloats) +
              "; use fsmt_forward_plain / fsmt_adjoint_plain with a caller buffer, or fewer restarts");
    return FSMT_EINVAL;
  }
  float* work = nullptr;
  s = noalloc_work_ptr(&work);
  if (s != FSMT_OK) return s;
  s = fsmt_forward_plain(c, R, sigma, w, a, b, work, cop, obj, stream);
  if (s != FSMT_OK) return s;
  return fsmt_adjoint_plain(c, R, sigma, w, a, b, work, grad_a, grad_b, stream);
}

fsmt_status fsmt_weight_sum(const fsmt_compiled* c, int32_t R, const float* w, float* wsum, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  if (!w || !wsum) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  return launch_weight_sum(c->c, R, w, wsum, (cudaStream_t)stream);
}

fsmt_status fsmt_pgd_step(const fsmt_compiled* c, int32_t R, float eta, float b_scale, int32_t sweeps, int32_t polish,
                          float* a, float* b, const float* grad_a, const float* grad_b, const float* wsum,
                          float* gnorm2, const uint8_t* active, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (!(eta > 0.f) || !(b_scale > 0.f) || sweeps < 0 || polish < 0 || !gnorm2 || (C.n_bool && (!a || !grad_a)) ||
      (C.n_real && (!b || !grad_b))) {
    set_error("invalid step parameters or NULL argument");
    return FSMT_EINVAL;
  }
  return launch_pgd(C, R, eta, b_scale, sweeps, polish, nullptr, wsum, a, b, const_cast<float*>(grad_a),
                    const_cast<float*>(grad_b),
                    gnorm2, active, 0, nullptr, (cudaStream_t)stream);
}

fsmt_status fsmt_round_check(const fsmt_compiled* c, int32_t R, const float* a, const float* b, int8_t* x,
                             uint8_t* violated, int32_t* n_unsat, float* w, float* h, float rho, float gamma,
                             int32_t update_w, const float* wsum, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (!n_unsat || (C.n_bool && !a) || (C.n_real && !b) || ((w == nullptr) != (h == nullptr)) ||
      (h && !(gamma > 0.f))) {
    set_error("NULL argument or invalid ERWA parameters");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (x && C.n_bool) {
    k_sign<<<std::min<long>(((long)C.n_bool * R + 255) / 256, 65535L), 256, 0, st>>>(C.n_bool, R, a, x);
    FSMT_CUDA(cudaGetLastError(), "sign launch");
  }
  return launch_round_check(C, R, a, b, violated, n_unsat, w, h, rho, gamma, update_w, nullptr, wsum, nullptr, st);
}

fsmt_status fsmt_round(const fsmt_compiled* c, int32_t R, const float* a, int8_t* x, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  const Compiled& C = c->c;
  if (C.n_bool == 0) return FSMT_OK;
  if (!a || !x) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  k_sign<<<std::min<long>(((long)C.n_bool * R + 255) / 256, 65535L), 256, 0, (cudaStream_t)stream>>>(C.n_bool, R,
                                                                                                        a, x);
  FSMT_CUDA(cudaGetLastError(), "sign launch");
  return FSMT_OK;
}

fsmt_status fsmt_converge(const fsmt_compiled* c, int32_t R, float eps, const float* gnorm2, uint8_t* active,
                          int32_t* iters, int32_t* ctl, void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  if (!gnorm2 || !active || !iters || !ctl || !(eps >= 0.f)) {
    set_error("NULL argument or invalid eps");
    return FSMT_EINVAL;
  }
  k_converge<<<1, 1024, 0, (cudaStream_t)stream>>>(R, nullptr, eps, gnorm2, active, iters, ctl, 0);
  FSMT_CUDA(cudaGetLastError(), "converge launch");
  return FSMT_OK;
}

fsmt_status fsmt_mark_nonfinite(const fsmt_compiled* c, int32_t R, const uint8_t* active, int32_t* n_unsat,
                                void* stream) {
  fsmt_status s = check_ready(c, R);
  if (s != FSMT_OK) return s;
  if (!active || !n_unsat) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  k_mark_nonfinite<<<(R + 255) / 256, 256, 0, (cudaStream_t)stream>>>(R, active, n_unsat);
  FSMT_CUDA(cudaGetLastError(), "mark launch");
  return FSMT_OK;
}

// plan: the persistent stage kernel's launch, or NULL for separate launches per iteration
static fsmt_status enqueue_stage(const Compiled& C, int t_max, fsmt_state* s, const StagePlan* plan,
                                 cudaStream_t st) {
  const int R = s->R;
  k_stage_begin<<<(R + 255) / 256, 256, 0, st>>>(R, s->active, s->iters, s->ctl);
  FSMT_CUDA(cudaGetLastError(), "stage begin");
  fsmt_status ws = launch_weight_sum(C, R, s->w, s->wsum, st);
  if (ws != FSMT_OK) return ws;
  if (plan && t_max > 0) {
    k_iter_begin<<<(R + 255) / 256, 256, 0, st>>>(R, s->obj, s->gnorm2, s->ctl);
    FSMT_CUDA(cudaGetLastError(), "iteration begin");
    for (int it = 0; it < (plan->per_iteration ? t_max : 1); ++it) {
      ws = launch_stage_kernel(C, *plan, t_max, it, s, st);
      if (ws != FSMT_OK) return ws;
    }
    t_max = 0;
  }
  for (int it = 0; it < t_max; ++it) {
    k_iter_begin<<<(R + 255) / 256, 256, 0, st>>>(R, s->obj, s->gnorm2, s->ctl);
    fsmt_status e = launch_fused(C, true, R, 0.f, s->params, s->w, s->a, s->b, s->grad_a, s->grad_b, s->obj, nullptr,
                                 s->ctl, st);
    if (e != FSMT_OK) return e;
    e = launch_pgd(C, R, 1.f, 1.f, 0, 0, s->params, s->wsum, s->a, s->b, s->grad_a, s->grad_b, s->gnorm2, s->active, 1,
                   s->ctl, st);
    if (e != FSMT_OK) return e;
    k_converge<<<1, 1024, 0, st>>>(R, s->params, 0.f, s->gnorm2, s->active, s->iters, s->ctl, 1);
    FSMT_CUDA(cudaGetLastError(), "converge");
  }
  return launch_round_check(C, R, s->a, s->b, nullptr, s->n_unsat, s->w, s->h, 0.f, 2.f, 0, s->params, s->wsum,
                            s->active, st);
}

fsmt_status fsmt_solve_stage(fsmt_compiled* cc, const fsmt_stage_config* cfg, fsmt_state* s, void* stream) {
  if (!cfg || !s) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  fsmt_status e = check_ready(cc, s->R);
  if (e != FSMT_OK) return e;
  Compiled& C = cc->c;
  if (!(cfg->sigma >= 0.f) || !(cfg->eta > 0.f) || !(cfg->b_scale > 0.f) || cfg->t_max < 0 || cfg->sweeps < 0 ||
      cfg->polish < 0 || !(cfg->gamma > 0.f) || !s->w || !s->h || !s->wsum || !s->obj || !s->gnorm2 || !s->active || !s->iters || !s->n_unsat ||
      !s->ctl || !s->params || (C.n_bool && (!s->a || !s->grad_a)) || (C.n_real && (!s->b || !s->grad_b))) {
    set_error("invalid stage configuration or NULL state buffer");
    return FSMT_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  StagePlan plan;
  const bool persistent = cfg->persistent > 0 && stage_plan(C, s->R, cfg->persistent == 2, plan);
  k_set_params<<<1, 1, 0, st>>>(s->params, cfg->sigma, cfg->eta, cfg->b_scale, cfg->eps, cfg->rho, cfg->gamma,
                                (float)cfg->update_w, (float)cfg->sweeps, (float)cfg->polish,
                                (float)cfg->normalize_eta);
  FSMT_CUDA(cudaGetLastError(), "set params");
  if (!cfg->use_graph) return enqueue_stage(C, cfg->t_max, s, persistent ? &plan : nullptr, st);
  // the legacy default stream cannot be captured: use a blocking stream of our own,
  // which the legacy stream's implicit synchronisation orders with the caller's work
  if (st == nullptr || st == cudaStreamLegacy) {
    if (!C.capture_stream) {
      cudaStream_t cs;
      FSMT_CUDA(cudaStreamCreate(&cs), "create capture stream");
      C.capture_stream = cs;
    }
    st = (cudaStream_t)C.capture_stream;
  }
  // one graph per (buffer set, R, t_max)
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
  const void* ptrs[] = {s->a, s->b, s->w, s->h, s->grad_a, s->grad_b, s->obj, s->gnorm2, s->active, s->iters,
                        s->n_unsat, s->ctl, s->params, s->wsum};
  for (const void* p : ptrs) mix((uint64_t)(uintptr_t)p);
  mix((uint64_t)s->R);
  mix((uint64_t)cfg->t_max);
  mix((uint64_t)(C.tuned_R == s->R ? 1 + C.tuned.variant * 64 + C.tuned.rpl * 8 + (C.tuned.real_cap > 0) : 0));
  mix((uint64_t)persistent + 2 * (uint64_t)(persistent && plan.per_iteration));
  mix((uint64_t)(uintptr_t)(persistent ? C.stage_trace : nullptr));
  if (!C.graph_exec || C.graph_key != key) {
    if (C.graph_exec) {
      cudaGraphExecDestroy((cudaGraphExec_t)C.graph_exec);
      C.graph_exec = nullptr;
    }
    cudaGraph_t g;
    FSMT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    fsmt_status q = enqueue_stage(C, cfg->t_max, s, persistent ? &plan : nullptr, st);
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (q != FSMT_OK) return q;
    if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
    cudaGraphExec_t ex;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
    C.graph_exec = ex;
    C.graph_key = key;
  }
  FSMT_CUDA(cudaGraphLaunch((cudaGraphExec_t)C.graph_exec, st), "graph launch");
  return FSMT_OK;
}

fsmt_status fsmt_stage_trace(fsmt_compiled* c, uint64_t* trace) {
  if (!c) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  c->c.stage_trace = reinterpret_cast<unsigned long long*>(trace);
  return FSMT_OK;
}

fsmt_status fsmt_stage_form(fsmt_compiled* c, int32_t R, int32_t* persistent_out) {
  if (!persistent_out) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  fsmt_status e = check_ready(c, R);
  if (e != FSMT_OK) return e;
  StagePlan plan;
  *persistent_out = stage_plan(c->c, R, false, plan) && stage_plan(c->c, R, true, plan) ? 1 : 0;
  return FSMT_OK;
}

fsmt_status fsmt_solve_stage_host(fsmt_compiled* cc, const fsmt_stage_config* cfg, fsmt_state* s,
                                  const float* a_host, const float* b_host, int32_t* n_unsat_host, float* obj_host,
                                  void* stream) {
  if (!cc || !cfg || !s) {
    set_error("NULL argument");
    return FSMT_EINVAL;
  }
  fsmt_status ready = check_ready(cc, s->R);  // before any copy into the state
  if (ready != FSMT_OK) return ready;
  const Compiled& C = cc->c;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t R = (size_t)s->R;
  if (C.n_bool && a_host)
    FSMT_CUDA(cudaMemcpyAsync(s->a, a_host, sizeof(float) * C.n_bool * R, cudaMemcpyHostToDevice, st), "copy a");
  if (C.n_real && b_host)
    FSMT_CUDA(cudaMemcpyAsync(s->b, b_host, sizeof(float) * C.n_real * R, cudaMemcpyHostToDevice, st), "copy b");
  fsmt_status e = fsmt_solve_stage(cc, cfg, s, stream);
  if (e != FSMT_OK) return e;
  if (n_unsat_host)
    FSMT_CUDA(cudaMemcpyAsync(n_unsat_host, s->n_unsat, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, st), "copy n_unsat");
  if (obj_host) FSMT_CUDA(cudaMemcpyAsync(obj_host, s->obj, sizeof(float) * R, cudaMemcpyDeviceToHost, st), "copy obj");
  int32_t err_bits = 0;
  FSMT_CUDA(cudaMemcpyAsync(&err_bits, s->ctl + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy ctl");
  FSMT_CUDA(cudaStreamSynchronize(st), "stage sync");
  if (err_bits & kCtlBarrierTimeout) {
    set_error("the persistent stage kernel gave up waiting at a grid barrier");
    return FSMT_ETIMEOUT;
  }
  if (n_unsat_host)
    for (size_t r = 0; r < R; ++r)
      if (n_unsat_host[r] < 0) {
        set_error("non-finite point in restart " + std::to_string(r));
        return FSMT_ENAN;
      }
  return FSMT_OK;
}

}  // extern "C"
