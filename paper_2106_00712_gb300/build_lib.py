"""Build libnmc.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel to paper_2106_00712_gb300/_build/*.o; the
shared library lands beside this file. Rebuilds only when a source or header is newer.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnmc.so")
SOURCES = ["gemm.cu", "gemm_df.cu", "gemm_tc.cu", "stab.cu", "flip.cu", "misc.cu", "nmc_api.cu", "noalloc.cu",
           "nimc.cu", "cgen.cu", "probe.cu", "lattice.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    inc = os.path.join(ROOT, "include")
    files += [os.path.join(inc, f) for f in os.listdir(inc)]
    return files


LIB_DEBUG = os.path.join(HERE, "libnmc_debug.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")


def needs_build(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force=False, verbose=False, extra=(), debug=False):
    """Compile libnmc.so (returns its path); debug=True: the bounds-checked
    libnmc_debug.so (NMC_DEBUG) instead. Raises RuntimeError on a compiler error."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if debug:
        extra = list(extra) + ["-DNMC_DEBUG"]
    if not force and not needs_build(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + ARCH + NVCC_FLAGS + list(extra)
        if src.endswith(".cpp"):
            cmd += ["-x", "c++"]
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                 stderr=subprocess.STDOUT)))
        objs.append(obj)
    errors = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            errors.append(f"{src}:\n{text}")
        elif verbose and text.strip():
            sys.stderr.write(f"[{src}]\n{text}\n")
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib + ".tmp"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    verbose = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=verbose or bool(extra), extra=extra,
                debug="--debug" in sys.argv))
