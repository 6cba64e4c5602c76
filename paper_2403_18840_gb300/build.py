"""Build the fdcore shared library for sm_103a with nvcc (no cmake).

Translation units are compiled in parallel and linked into
``paper_2403_18840_gb300/_build/libfdcore.so`` (in-tree, git-ignored).
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfdcore.so")
SOURCES = ["fd_api.cu", "fd_integrand.cu", "fd_flow.cu", "fd_jit.cu", "fd_mcmc.cu", "fd_nsf.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _needs_rebuild():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "fdcore.h"))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _cuda_libdir():
    nvcc = shutil.which(NVCC)
    if not nvcc:
        return ""
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def _embed_runtime_header():
    """The specialised kernels include fd_jit_rt.cuh; the library hands its text
    to the run-time compiler, so it is embedded as a raw string literal."""
    text = open(os.path.join(CSRC, "fd_jit_rt.cuh")).read()
    assert ")FDRT" not in text
    out = os.path.join(BUILD, "fd_jit_rt.inc")
    body = 'R"FDRT(' + text + ')FDRT"\n'
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)


def build(force=False, verbose=False, extra_flags=()):
    """Compile (when sources changed) and return the library path."""
    if not force and not _needs_rebuild():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    _embed_runtime_header()
    extra_flags = list(extra_flags) + ["-I", BUILD, '-DFD_CUDA_LIBDIR="%s"' % _cuda_libdir()]
    objs, procs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [NVCC, *ARCH, *FLAGS, *extra_flags, "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            print(out, flush=True)
        if p.returncode != 0:
            failed.append((src, out))
    if failed:
        msg = "\n".join("%s:\n%s" % f for f in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
