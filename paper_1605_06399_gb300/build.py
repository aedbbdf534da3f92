"""Build ``libimagecl.so`` (sm_103a) in-tree with nvcc, one job per translation unit.

The tiled conv2d source is compiled once per (filter side, pixel-type group) so the
heavily unrolled kernels build in parallel.  Objects go to ``_build/`` beside this file
and are rebuilt when their source, a header or the flags change.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libimagecl.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                 "-I" + INCLUDE, "-I" + CSRC]

TILED_K = (3, 5, 7, 9, 11, 13, 15)
TILED_GROUPS = (0, 1, 2, 3)
SEP_GROUPS = (0, 1, 2)
SEP_RSETS = (0, 1)
TC_K = (9, 11, 13, 15)
MULTI = ("conv2d_tiled.cu", "sepconv_fused.cu", "conv2d_tc.cu")


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build libimagecl.so")


def units() -> list[tuple[str, list[str], str]]:
    """(source, extra flags, object name) for every translation unit."""
    out = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu") and f not in MULTI:
            out.append((os.path.join(CSRC, f), [], f[:-3] + ".o"))
    for k in TILED_K:
        for g in TILED_GROUPS:
            out.append((os.path.join(CSRC, "conv2d_tiled.cu"),
                        [f"-DIMCL_TILED_K={k}", f"-DIMCL_TILED_GROUP={g}"],
                        f"conv2d_tiled_k{k}_g{g}.o"))
    for k in TC_K:
        out.append((os.path.join(CSRC, "conv2d_tc.cu"), [f"-DIMCL_TC_K={k}"], f"conv2d_tc_k{k}.o"))
    for g in SEP_GROUPS:
        for r in SEP_RSETS:
            out.append((os.path.join(CSRC, "sepconv_fused.cu"),
                        [f"-DIMCL_SEP_GROUP={g}", f"-DIMCL_SEP_RSET={r}"],
                        f"sepconv_fused_g{g}_s{r}.o"))
    return out


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "imagecl.h"))
    return max(os.path.getmtime(h) for h in hs)


def _stamp(flags: list[str]) -> str:
    return hashlib.sha1(" ".join(flags).encode()).hexdigest()[:12]


def _compile(nvcc, src, extra, obj, hdr_mtime, verbose):
    flags = CFLAGS + extra
    stamp_file = obj + ".flags"
    stamp = _stamp(flags)
    if (os.path.exists(obj) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp
            and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_mtime)):
        return obj, False
    cmd = [nvcc] + flags + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr[-6000:]}")
    if verbose and r.stderr.strip():
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return obj, True


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link ``libimagecl.so``."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdr = _headers_mtime()
    todo = units()
    if force:
        for _, _, o in todo:
            p = os.path.join(BUILD, o)
            if os.path.exists(p):
                os.unlink(p)
    jobs = jobs or max(1, os.cpu_count() or 1)
    changed = False
    # longest jobs (tiled, large K, f32) first
    def cost(u):
        src, extra, o = u
        if "conv2d_tiled" in o:
            k = int(o.split("_k")[1].split("_")[0])
            return -(k * k * (3 if o.endswith("g0.o") else 1))
        if "sepconv_fused" in o:
            return -150
        return 0
    todo.sort(key=cost)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, s, e, os.path.join(BUILD, o), hdr, verbose)
                for s, e, o in todo]
        objs = []
        for f in futs:
            o, c = f.result()
            objs.append(o)
            changed |= c
    if changed or force or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
              ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t0 = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(f"built in {time.time() - t0:.1f} s")
