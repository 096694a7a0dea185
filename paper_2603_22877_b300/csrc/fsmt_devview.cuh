// The view of the compiled instance that every kernel reads, and the exact
// fixed-point sign used by the exact check.  Host- and device-safe; also compiled
// by NVRTC, hence no standard headers there.
#pragma once

#ifdef __CUDACC_RTC__
typedef decltype(sizeof(0)) size_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef unsigned char uint8_t;
typedef signed char int8_t;
#else
#include <cstdint>

#include <vector_types.h>
#endif

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define FSMT_HD __host__ __device__ __forceinline__
#else
#define FSMT_HD inline
#endif

namespace fsmt {

constexpr int kMaxNodesPerDiagram = 65533;  // hi/lo are 16-bit and V, V+1 are the terminals
// Shared memory (4-byte words) of the projection kernel for blocks of coupled reals of
// at most nv reals, nh half-spaces and nnz nonzeros over a block's half-spaces, wy
// warps per CTA: per thread the block's iterate, box corrections and half-space
// multipliers; per warp the staged block (offsets, local reals, coefficients,
// right-hand sides, 1/||q||^2, the box, the equality flags).  A block is accepted when one
// warp's CTA fits.
FSMT_HD long proj_block_words(long nv, long nh, long nnz, long wy) {
  return (2 * nv + nh) * 32 * wy + wy * ((nh + 1) + 2 * nnz + 3 * nh + 2 * nv);
}
constexpr long kProjSmemWords = (227 * 1024 - 2048) / 4;  // a CTA's dynamic shared memory, 2 KB left for static
// chunks of the chunked forward/adjoint kernel
constexpr int kChunkMaxCons = 64;    // constraints per chunk
constexpr int kChunkMaxNodes = 2048; // decision nodes per chunk
constexpr int kChunkMaxSlots = 320;  // distinct variables / atoms per chunk (hard limit)
// the slot limit when the generic DP path may run: its per-warp message rows
// share shared memory with the slot arrays, so smaller chunks keep more warps
constexpr int kChunkSlotsGeneric = 192;
constexpr int kChunkMaxList = 2304;  // words of a chunk's per-constraint literal lists (nodes + padding)
constexpr int kSlotStride = 64;  // floats per slot row of the per-slot shared arrays (two restarts x 32 lanes)
constexpr int kChunkThreads = 512;  // threads of the chunked kernel with the generic path (16 warps)
constexpr int kFusedThreads = 256;  // threads of the warp-per-constraint kernel (8 warps)
constexpr int kChunkMaxTerms = 768;  // nonzeros of the atoms of a chunk
constexpr int kChunkMaxReals = 128;   // reals touched by a chunk's atoms
constexpr int kMaxJitShapes = 16;      // diagram shapes given generated code per instance
constexpr int kMaxJitShapeNodes = 48;  // largest diagram given generated code
constexpr int kMaxProjShapes = 16;     // block shapes given generated projection routines per instance
constexpr int kMaxProjShapeVars = 24;  // largest block given one: reals,
constexpr int kMaxProjShapeHs = 32;    // half-spaces
constexpr int kMaxProjShapeNnz = 96;   // and nonzeros

// Everything the kernels read, as one POD passed by value.
struct DevView {
  int32_t n_bool, n_real, n_atoms, n_cons, n_obj;
  const int32_t* con_ptr;   // [n_cons + 1] node offsets, schedule order
  const int32_t* con_id;    // [n_cons] constraint id of each schedule slot
  const uint8_t* con_root;  // [n_cons] root index (0, or V / V+1 if constant)
  const uint2* nodes;       // {label, hi | lo << 16}
  // atoms in normalised form  sum coef_j y_j - q0 (<= | <) 0
  const int32_t* atom_ptr;  // [n_atoms + 1]
  const int32_t* atom_var;
  const float* atom_coef;       // exact integers (|q| < 2^24)
  const float* atom_q0f;        // q0 rounded to FP32 (relaxation only)
  const double* atom_q0d;       // q0 exact (|q0| < 2^53), for the exact check
  const float* atom_inv_norm;   // 1 / ||q||_2
  const uint8_t* atom_strict;   // 1: strict (<), 2: equality (=, projected unit atoms only), else 0
  // projection
  const float* lo;
  const float* hi;
  int32_t n_free;
  const int32_t* free_var;      // reals that only have a box
  int32_t n_comp;
  const int32_t* comp_var_ptr;  // [n_comp + 1] into comp_var
  const int32_t* comp_var;      // global real ids
  const int32_t* comp_hs_ptr;   // [n_comp + 1] into half-space list
  const int32_t* hs_ptr;        // [n_hs + 1] into hs_lvar / hs_coef
  const int32_t* hs_lvar;       // local index of the real inside its block
  const float* hs_coef;
  const float* hs_q0;
  const float* hs_inv_qq;       // 1 / ||q||^2
  const uint8_t* hs_eq;         // 1: the entry is an equality's hyperplane q.y = q0
  const int32_t* comp_shape;    // [n_comp] rank of the block's generated projection routine (0: none)
  // chunked schedule of the constraints of C_sigma
  int32_t n_chunks;
  int32_t chunk_slot_cap;         // most slots of any chunk: rows of the per-slot shared arrays
  int32_t chunk_real_cap;         // most reals of any chunk when their b is staged in shared memory, else 0
  const int32_t* chunk_con_ptr;   // [n_chunks + 1] into ccon
  const int4* ccon;               // {node offset in chunk, V, root, constraint id}
  const int32_t* chunk_node_ptr;  // [n_chunks + 1] into cnodes
  const uint2* cnodes;            // {slot, hi | lo << 16}
  const int32_t* chunk_slot_ptr;  // [n_chunks + 1] into slot_label
  const int32_t* slot_label;      // variable id (< n_bool) or n_bool + atom index
  const int32_t* slot_meta;       // atom slots: (first term << 16) | term count, chunk-relative; else 0
  const int32_t* chunk_term_ptr;  // [n_chunks + 1] into term_var / term_coef
  const int32_t* term_var;        // chunk-local real of each atom nonzero, chunk by chunk
  const int32_t* chunk_real_ptr;  // [n_chunks + 1] into real_id
  const int32_t* real_id;         // the chunk's reals
  const int32_t* chunk_list_ptr;  // [n_chunks + 1] into clist
  const uint32_t* clist;          // per constraint (16-byte aligned, at ccon.z words into the chunk's
                                  // part): the slot words of its distinct literals in order of first node
  const float* term_coef;         // its (normalised) coefficient
};

// Exact sign of  sum_t c_t * y_t - q0  where c_t are integers with |c_t| < 2^24
// (given as exact floats), y_t are FP32 values and q0 an integer with
// |q0| < 2^53 (given as an exact double).  Every term is an integer multiple of
// 2^-149, so the sum is accumulated exactly in a 320-bit two's-complement fixed
// point with that unit.  Returns -1, 0 or +1.
struct Fixed320 {
  uint64_t limb[5];
  FSMT_HD void clear() {
    for (int i = 0; i < 5; ++i) limb[i] = 0;
  }
  // adds (neg ? -1 : 1) * mag * 2^shift, mag < 2^63, shift < 256
  FSMT_HD void add(uint64_t mag, int shift, bool neg) {
    uint64_t part[5] = {0, 0, 0, 0, 0};
    int w = shift >> 6, s = shift & 63;
    part[w] = mag << s;
    if (s && w + 1 < 5) part[w + 1] = mag >> (64 - s);
    if (neg) {  // two's complement of part
      uint64_t carry = 1;
      for (int i = 0; i < 5; ++i) {
        uint64_t v = ~part[i] + carry;
        carry = (carry && v == 0) ? 1 : 0;
        part[i] = v;
      }
    }
    uint64_t carry = 0;
    for (int i = 0; i < 5; ++i) {
      uint64_t x = limb[i] + part[i];
      uint64_t c1 = x < limb[i] ? 1 : 0;
      uint64_t y = x + carry;
      uint64_t c2 = y < x ? 1 : 0;
      limb[i] = y;
      carry = c1 | c2;
    }
  }
  FSMT_HD int sign() const {
    if (limb[4] >> 63) return -1;
    for (int i = 0; i < 5; ++i)
      if (limb[i]) return 1;
    return 0;
  }
};

// Splits a finite float into (integer mantissa m >= 0, exponent k) with
// value = m * 2^k, k >= -149.
FSMT_HD void float_parts(float y, uint32_t& m, int& k, bool& neg) {
  union {
    float f;
    uint32_t u;
  } v;
  v.f = y;
  neg = (v.u >> 31) != 0;
  uint32_t e = (v.u >> 23) & 0xff;
  uint32_t f = v.u & 0x7fffff;
  if (e == 0) {
    m = f;
    k = -149;
  } else {
    m = f | 0x800000u;
    k = (int)e - 150;
  }
}

// sign(sum_t coef_t * y_t - q0) exactly; coef are exact integers stored as floats.
FSMT_HD int exact_atom_sign(int nnz, const float* coef, const float* y, double q0) {
  Fixed320 acc;
  acc.clear();
  for (int t = 0; t < nnz; ++t) {
    uint32_t m;
    int k;
    bool neg;
    float_parts(y[t], m, k, neg);
    if (m == 0) continue;
    float c = coef[t];
    bool cneg = c < 0.f;
    uint64_t cm = (uint64_t)(cneg ? -c : c);
    acc.add(cm * (uint64_t)m, k + 149, neg != cneg);
  }
  if (q0 != 0.0) {
    bool qneg = q0 < 0.0;
    double aq = qneg ? -q0 : q0;
    uint64_t iq = (uint64_t)aq;
    acc.add(iq, 149, !qneg);
  }
  return acc.sign();
}

}  // namespace fsmt
