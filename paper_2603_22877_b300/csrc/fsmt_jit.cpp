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

#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <sstream>
#include <unordered_map>
#include <vector>

#include "fsmt_internal.h"
#include "fsmt_jit_src.inc"  // kJitDevviewSrc, kJitChunkedSrc (generated by build.py)

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

// Alg. 3 / Alg. 4 for one shape, straight-line.  Node v tests literal l_v with
// probability q_v (= p or 1 - p for a negated literal); its children (hi = l_v
// true) are nodes, or V (TRUE) / V+1 (FALSE).  Nodes testing the same variable
// form a group (grp = its first node), so the shape fixes which nodes read
// which variable.  Each pass reads a group's slot word and q from shared
// memory once, at the group's first node in that pass's order; the messages
// t_v (Alg. 3) and b_v (Alg. 4) live in registers; the reverse pass sums
// t_v (b_hi - b_lo) over a group and issues the one shared-memory update of
// its slot at the group's last node.  Short live ranges keep the routine
// within the 64 registers of the 1024-thread kernel.
std::string shape_routine(int rank, int V, const uint16_t* hi, const uint16_t* lo, const uint16_t* grp) {
  std::ostringstream o;
  auto bu = [&](int c) -> std::string {  // m_bu of a child
    if (c == V) return "1.f";
    if (c == V + 1) return "0.f";
    return "b" + std::to_string(c);
  };
  std::vector<int> last(V, -1);  // last node of each group, by index
  for (int v = 0; v < V; ++v) last[grp[v]] = v;
  o << "template <bool ADJ, int RPL>\n__device__ __forceinline__ void shape_" << rank
    << "(const uint2* __restrict__ nd, const float* __restrict__ s_p, float* __restrict__ s_g, int lane,"
       " const Pack<RPL>& wc, Pack<RPL>& cp) {\n";
  o << "#pragma unroll\n  for (int k = 0; k < RPL; ++k) {\n";
  o << "    float t0 = 1.f";
  for (int v = 1; v < V; ++v) o << ", t" << v << " = 0.f";
  o << ";\n    if (ADJ) {\n";
  for (int v = 0; v < V; ++v) {  // Alg. 3: push to non-terminal children
    const int g = grp[v];
    if (g == v) o << "      const float f" << g << " = lit_q<RPL>(nd[" << g << "].x, s_p, lane, k);\n";
    if (hi[v] < V) o << "      t" << hi[v] << " = fmaf(f" << g << ", t" << v << ", t" << hi[v] << ");\n";
    if (lo[v] < V) o << "      t" << lo[v] << " = fmaf(1.f - f" << g << ", t" << v << ", t" << lo[v] << ");\n";
  }
  o << "    }\n";
  for (int v = V - 1; v >= 0; --v) {  // Alg. 4, and the adjoint sum of each group
    const int g = grp[v];
    if (last[g] == v)
      o << "    const float q" << g << " = lit_q<RPL>(nd[" << g << "].x, s_p, lane, k);\n    float acc" << g << " = 0.f;\n";
    o << "    const float d" << v << " = " << bu(hi[v]) << " - " << bu(lo[v]) << ";\n";
    o << "    const float b" << v << " = fmaf(q" << g << ", d" << v << ", " << bu(lo[v]) << ");\n";
    o << "    if (ADJ) acc" << g << " = fmaf(t" << v << ", d" << v << ", acc" << g << ");\n";
    if (g == v)
      o << "    if (ADJ) {\n      const unsigned r = nd[" << g << "].x;\n"
        << "      atomicAdd(s_g + ((int)(r & 0x7fffffffu) * RPL + k) * 32 + lane, (r >> 31) ? -wc.v[k] * acc" << g
        << " : wc.v[k] * acc" << g << ");\n    }\n";
  }
  o << "    cp.v[k] = b0;\n  }\n}\n\n";
  return o.str();
}

std::string kernel_name(int wide, int adj, int rpl) {
  return std::string("fsmt_jit_") + (wide ? "wide_" : "") + (adj ? "adj_" : "fwd_") + std::to_string(rpl);
}

std::string generated_source(const Compiled& C) {
  std::ostringstream o;
  o << "#define FSMT_JIT_SHAPES 1\n" << kJitDevviewSrc << "\n" << kJitChunkedSrc << "\nnamespace fsmt {\n\n";
  o << "// probability of the literal a node tests: p of its slot, or 1 - p when negated (bit 31)\n"
       "template <int RPL>\n__device__ __forceinline__ float lit_q(unsigned r, const float* __restrict__ s_p, int lane,"
       " int k) {\n  const float p = s_p[((r & 0x7fffffffu) * RPL + k) * 32 + lane];\n  return (r >> 31) ? 1.f - p : p;\n}\n\n";
  for (size_t k = 0; k < C.jit_shape.size(); ++k) {
    const int x = C.jit_shape[k];
    const int b = C.shape_ptr[x], V = C.shape_ptr[x + 1] - b;
    o << shape_routine((int)k + 1, V, C.shape_hi.data() + b, C.shape_lo.data() + b, C.shape_grp.data() + b);
  }
  o << "template <bool ADJ, int RPL>\n__device__ __forceinline__ bool shape_dispatch(int shape, const uint2* nd,"
       " const float* s_p, float* s_g, int lane, const Pack<RPL>& wc, Pack<RPL>& cp) {\n  switch (shape) {\n";
  for (size_t k = 0; k < C.jit_shape.size(); ++k)
    o << "    case " << k + 1 << ": shape_" << k + 1 << "<ADJ, RPL>(nd, s_p, s_g, lane, wc, cp); return true;\n";
  o << "    default: return false;\n  }\n}\n\n}  // namespace fsmt\n\n";
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
  return o.str();
}

struct Module {
  void* kernel[2][2][2];  // [wide][adjoint][restarts per lane - 1]
};
std::mutex g_mutex;
std::unordered_map<std::string, Module> g_modules;  // by source text; kept for the process lifetime

}  // namespace

// Builds (or reuses) the specialised kernels for C.  Returns false, leaving C
// on the ahead-of-time kernel, when there is nothing to specialise, NVRTC is
// missing, FSMT_NO_JIT is set, or compilation fails (the reason goes to the
// error message).
bool jit_build(Compiled& C) {
  for (auto& r : C.jit_kernel) r[0] = r[1] = nullptr;
  C.jit_shapes = 0;
  const char* off = std::getenv("FSMT_NO_JIT");
  if ((off && *off && *off != '0') || C.jit_shape.empty() || !C.chunked_ok) return false;
  Nvrtc& N = nvrtc();
  if (!N.ok) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  const std::string src = generated_source(C);
  const std::string arch = "-arch=sm_" + std::to_string(major) + std::to_string(minor) + "a";
  std::lock_guard<std::mutex> lock(g_mutex);
  const std::string key = arch + src;
  auto it = g_modules.find(key);
  if (it == g_modules.end()) {
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "fsmt_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return false;
    const bool verbose = std::getenv("FSMT_JIT_VERBOSE") != nullptr;
    const char* opts[] = {arch.c_str(), "-std=c++17", "-lineinfo", "--ptxas-options=-v"};
    const nvrtcResult rc = N.compile(prog, verbose ? 4 : 3, opts);
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
    cudaLibrary_t lib;
    if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
      set_error("loading the run-time compiled kernels failed; using the ahead-of-time kernel");
      return false;
    }
    Module m{};
    for (int wide = 0; wide < 2; ++wide)
      for (int adj = 0; adj < 2; ++adj)
        for (int r = 0; r < 2; ++r) {
          cudaKernel_t k;
          if (cudaLibraryGetKernel(&k, lib, kernel_name(wide, adj, r + 1).c_str()) != cudaSuccess) return false;
          if (cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
              cudaSuccess)
            return false;
          m.kernel[wide][adj][r] = (void*)k;
        }
    it = g_modules.emplace(key, m).first;
  }
  for (int adj = 0; adj < 2; ++adj)
    for (int r = 0; r < 2; ++r) {
      C.jit_kernel[adj][r] = it->second.kernel[0][adj][r];
      C.jit_wide[adj][r] = C.all_specialized ? it->second.kernel[1][adj][r] : nullptr;
    }
  C.jit_shapes = (int32_t)C.jit_shape.size();
  return true;
}

}  // namespace fsmt
