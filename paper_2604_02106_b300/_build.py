"""In-tree build of libhgrd.so for sm_103a (nvcc; no GPU needed to compile)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhgrd.so")
SOURCES = ["desc.cpp", "kernels.cu", "check.cu", "batch.cu", "mlp.cu", "rank.cu", "jit.cpp"]
HEADERS = ["hgrd_internal.h", "hgrd_host.h", "kernels.cuh", "kcommon.cuh", "expand_body.cuh", "jit.h", os.path.join("..", "..", "include", "hgrd.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-shared", "-cudart", "shared",
         "--expt-relaxed-constexpr"]
LIBS = ["-lnvrtc"]
# device headers handed to the run-time compiler as text (jit.cpp), by the
# name they are included under
JIT_HEADERS = [("hgrd_internal.h", "hgrd_internal.h"), ("kcommon.cuh", "kcommon.cuh"),
               ("expand_body.cuh", "expand_body.cuh")]
JIT_INC = os.path.join(CSRC, "jit_headers.inc")


def _write_jit_headers() -> None:
    delim = "hgrdjit"
    names, texts = [], []
    for name, rel in JIT_HEADERS:
        text = open(os.path.join(CSRC, rel)).read()
        assert f"){delim}\"" not in text
        names.append(f'"{name}"')
        texts.append(f'R"{delim}({text}){delim}"')
    out = ("// written by _build.py: device headers for the run-time compiler\n"
           f"static const char* const kJitHeaderNames[] = {{{', '.join(names)}}};\n"
           f"static const char* const kJitHeaders[] = {{\n{(','+chr(10)).join(texts)}}};\n")
    old = open(JIT_INC).read() if os.path.exists(JIT_INC) else None
    if old != out:
        with open(JIT_INC, "w") as f:
            f.write(out)


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    _write_jit_headers()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, *FLAGS, "-o", tmp, *[os.path.join(CSRC, f) for f in SOURCES], *LIBS]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
