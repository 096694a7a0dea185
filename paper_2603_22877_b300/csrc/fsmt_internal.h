// Internal structures shared by the host compiler (fsmt_host.cpp) and the CUDA
// code (fsmt_device.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fsmt.h"
#include "fsmt_devview.cuh"

namespace fsmt {

void set_error(const std::string& msg);
struct Compiled;
bool jit_build(Compiled& C);  // fsmt_jit.cpp
bool jit_build_stage(Compiled& C);  // fsmt_jit.cpp: the persistent stage kernels, on first use

struct Problem {
  int32_t n_bool = 0, n_real = 0;
  std::vector<double> lo, hi;
  std::vector<int64_t> atom_ptr{0};
  std::vector<int32_t> atom_var;
  std::vector<int64_t> atom_coef;
  std::vector<int64_t> atom_q0;
  std::vector<int8_t> atom_rel;
  std::vector<int8_t> con_kind;
  std::vector<int32_t> con_param;
  std::vector<int64_t> con_ptr{0};
  std::vector<int32_t> con_lits;
  int32_t n_atoms() const { return (int32_t)atom_q0.size(); }
  int32_t n_cons() const { return (int32_t)con_kind.size(); }
};

// Host-side compiled form (arrays mirror DevView).
// One way to run the forward (+ adjoint) pass (fsmt_device.cu; the autotuner's unit).
enum { kVariantWarp = 0, kVariantGeneric = 1, kVariantJit = 2, kVariantWide = 3 };
struct LaunchCfg {
  int variant;   // kVariant*: warp per constraint, ahead-of-time chunked, generated with / without the generic path
  int rpl;       // restarts per lane
  int real_cap;  // reals staged in shared memory per chunk (0: b read from global memory)
  int warps;     // per CTA
  size_t smem;   // dynamic shared memory per CTA
};

struct Compiled {
  int32_t n_bool = 0, n_real = 0, n_atoms = 0, n_cons = 0, n_obj = 0;
  int32_t max_nodes = 0;
  int64_t n_obj_nodes = 0;
  std::vector<int32_t> con_ptr, con_id;
  std::vector<uint8_t> con_root;
  std::vector<uint32_t> node_label;
  std::vector<uint32_t> node_hilo;
  std::vector<int32_t> atom_ptr, atom_var;
  std::vector<float> atom_coef, atom_q0f, atom_inv_norm;
  std::vector<double> atom_q0d;
  std::vector<uint8_t> atom_strict;
  std::vector<float> lo, hi;
  std::vector<int32_t> free_var;
  std::vector<int32_t> comp_var_ptr{0}, comp_var, comp_hs_ptr{0}, hs_ptr{0}, hs_lvar;
  std::vector<float> hs_coef, hs_q0, hs_inv_qq;
  std::vector<uint8_t> hs_eq;  // 1: an equality's hyperplane, 0: a half-space
  int32_t comp_max_vars = 0, comp_max_hs = 0;  // the largest block's reals and half-spaces
  int32_t comp_max_nnz = 0;  // the most nonzeros over one block's half-spaces
  std::vector<int32_t> comp_shape;       // per block: rank of its generated projection routine (0: generic)
  std::vector<int32_t> proj_shape_comp;  // per generated routine: a block of that shape
  void* jit_proj = nullptr;              // run-time compiled projection kernel (fsmt_jit.cpp), or none
  int32_t proj_shapes = 0;               // projection routines in it
  int32_t empty_boxes = 0;  // reals with lo > hi after unit-atom tightening (no FP32 point)
  // chunked schedule of C_sigma (see build_chunks in fsmt_host.cpp)
  bool chunked_ok = false;
  int32_t n_chunks = 0;
  int32_t chunk_slot_cap = 0;  // most slots of any chunk
  int32_t chunk_real_max = 0;  // most reals of any chunk
  bool stage_reals = true;     // stage the chunk's reals in shared memory (FSMT_NO_STAGE=1 turns it off)
  int tuned_R = -1;            // restarts the configuration below was chosen for (fsmt_autotune / fsmt_select_config)
  LaunchCfg tuned{-1, 0, 0, 0, 0};
  std::vector<int32_t> chunk_con_ptr{0}, chunk_node_ptr{0}, chunk_slot_ptr{0}, slot_label;
  std::vector<int32_t> slot_meta, chunk_term_ptr{0}, term_var, chunk_real_ptr{0}, real_id;
  std::vector<float> term_coef;
  std::vector<int32_t> ccon;  // 4 ints per constraint
  std::vector<int32_t> chunk_list_ptr{0};
  std::vector<uint32_t> clist;  // per constraint: slot words of its distinct literals (padded to 4)
  std::vector<uint32_t> cnode_slot, cnode_hilo;  // slot | negated-literal bit 31; children
  // diagram shapes in literal space (build_chunks) and those given generated code
  std::vector<int32_t> shape_ptr{0};
  std::vector<uint16_t> shape_hi, shape_lo, shape_grp;  // grp: first node testing the same variable
  std::vector<int64_t> shape_nodes;
  std::vector<int32_t> jit_shape;  // shape index of generated routine k (rank k + 1)
  // run-time compiled chunked kernels (fsmt_jit.cpp): [adjoint][restarts per lane - 1]
  void* jit_kernel[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  void* jit_wide[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // no generic path: all_specialized only
  bool all_specialized = false;  // every constraint of C_sigma has a generated routine
  int32_t jit_shapes = 0;
  // run-time compiled persistent stage kernels (fsmt_stage.cuh), [one iteration a
  // launch] and by the forward + adjoint body they run: chunked [without the generic
  // path (all_specialized only)][restarts per lane - 1], or warp per constraint
  void* jit_stage_chunk[2][2][2] = {};
  void* jit_stage_warp[2] = {nullptr, nullptr};
  bool jit_stage_tried = false;  // jit_build_stage ran (they are built on first use)
  unsigned long long* stage_trace = nullptr;  // the caller's device buffer for fsmt_stage_trace, or none
  // device side
  void* dev_block = nullptr;  // one allocation holding every device array
  DevView view{};
  bool uploaded = false;
  int device = -1;
  // cached CUDA graph of a stage (fsmt_device.cu)
  void* graph_exec = nullptr;
  uint64_t graph_key = 0;
  void* capture_stream = nullptr;  // used when the caller passes the legacy default stream
};

}  // namespace fsmt

struct fsmt_problem {
  fsmt::Problem p;
};
struct fsmt_compiled {
  fsmt::Compiled c;
};
