"""Builds libfsmt.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2603_22877_b300.build   (or call build())
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfsmt.so")
SOURCES = ["fsmt_device.cu", "fsmt_host.cpp", "fsmt_jit.cpp"]
HEADERS = ["fsmt_internal.h", "fsmt_devview.cuh", "fsmt_chunked.cuh", "fsmt_proj.cuh", "fsmt_stage.cuh", "fsmt_jit_src.inc",
           os.path.join("..", "..", "include", "fsmt.h")]


def nvcc_path():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def needs_rebuild():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


JIT_INC = os.path.join(CSRC, "fsmt_jit_src.inc")


def write_jit_sources():
    """Embeds the device headers as strings, for the run-time compiler (fsmt_jit.cpp)."""
    parts = []
    for var, name in (("kJitDevviewSrc", "fsmt_devview.cuh"), ("kJitChunkedSrc", "fsmt_chunked.cuh"),
                      ("kJitProjSrc", "fsmt_proj.cuh"), ("kJitStageSrc", "fsmt_stage.cuh")):
        text = open(os.path.join(CSRC, name)).read()
        assert ")FSMTSRC" not in text
        parts.append(f'static const char* {var} = R"FSMTSRC(\n{text})FSMTSRC";\n')
    body = ("// generated by build.py from fsmt_devview.cuh, fsmt_chunked.cuh, fsmt_proj.cuh and fsmt_stage.cuh;"
            " do not edit\n" + "".join(parts))
    if not os.path.exists(JIT_INC) or open(JIT_INC).read() != body:
        with open(JIT_INC, "w") as f:
            f.write(body)


def build(force=False, verbose=False):
    write_jit_sources()
    if not force and not needs_rebuild():
        return LIB
    cmd = [nvcc_path(), "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC,-O2", "-shared", "-ldl", "-o", LIB + ".tmp"] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        print(r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
