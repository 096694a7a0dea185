"""The run-time generated CUDA sources compile for sm_103a, checked with no GPU.

At upload the library writes one CUDA source per instance (the device headers, the
diagram and projection routines generated for its shapes, the chunked forward /
adjoint kernels and the projection kernel) and, on first use, a second one with the
persistent stage kernels; on the GPU both go to NVRTC.  Here the generator
(fsmt_jit.cpp) is built into a host library next to libfsmt.so, asked for both
sources of a compiled instance, and each is compiled with nvcc for sm_103a: a
source that NVRTC would refuse fails here first, before any GPU time is spent."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from workloads import instances as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_22877_b300", "csrc")
CUDA = "/usr/local/cuda"

HARNESS = r'''
#include <cstring>
#include "fsmt_jit.cpp"
namespace fsmt { void set_error(const std::string&) {} }
static long put(const std::string& s, char* out, long cap) {
  if ((long)s.size() + 1 > cap) return -1;
  std::memcpy(out, s.c_str(), s.size() + 1);
  return (long)s.size();
}
extern "C" long main_src(const fsmt_compiled* c, char* out, long cap) { return put(fsmt::generated_source(c->c), out, cap); }
extern "C" long stage_src(const fsmt_compiled* c, char* out, long cap) { return put(fsmt::stage_source(c->c), out, cap); }
'''


def test_generated_sources_compile_for_sm103a(tmp_path):
    gxx, nvcc = shutil.which("g++"), shutil.which("nvcc") or os.path.join(CUDA, "bin", "nvcc")
    if gxx is None or not os.path.exists(nvcc):
        pytest.skip("g++ or nvcc is missing")
    from paper_2603_22877_b300 import build as B
    from paper_2603_22877_b300.engine import Problem
    B.write_jit_sources()
    (tmp_path / "harness.cpp").write_text(HARNESS)
    so = tmp_path / "harness.so"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", f"-I{CSRC}", f"-I{ROOT}/include",
                        f"-I{CUDA}/include", str(tmp_path / "harness.cpp"), "-o", str(so), f"-L{CUDA}/lib64",
                        "-lcudart", f"-Wl,-rpath,{CUDA}/lib64"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(str(so), mode=C.RTLD_LOCAL)
    for f in (lib.main_src, lib.stage_src):
        f.restype = C.c_long
        f.argtypes = [C.c_void_p, C.c_char_p, C.c_long]
    # one diagram shape family, atoms, and blocks of reals coupled by precedences
    comp = Problem.from_instance(W.jobshop(1002, 6, 3)).compile()
    assert comp.info["n_chunks"] > 0 and comp.info["n_components"] > 0
    procs = []
    for name, f in (("main", lib.main_src), ("stage", lib.stage_src)):
        buf = C.create_string_buffer(8 << 20)
        n = f(comp.h, buf, len(buf))
        assert n > 0
        src = buf.value.decode()
        kernels = (["fsmt_jit_wide_adj_2", "fsmt_jit_adj_1", "fsmt_jit_proj"] if name == "main" else
                   ["fsmt_jit_stage_wide_2", "fsmt_jit_stage_gen_1", "fsmt_jit_stage_warp", "fsmt_jit_step_wide_2",
                    "fsmt_jit_step_warp"])
        for k in kernels:
            assert f"{k}(" in src, (name, k)
        path = tmp_path / f"{name}.cu"
        path.write_text(src)
        procs.append((name, subprocess.Popen([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                                              "-c", str(path), "-o", str(tmp_path / f"{name}.o")],
                                             stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    for name, p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, (name, err[-4000:])
