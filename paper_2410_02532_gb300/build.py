"""Compile ``libopo.so`` for sm_103a with nvcc (no torch extension, no cmake).

Each translation unit compiles in parallel to an object file under
``_build/``; the objects link into ``paper_2410_02532_gb300/libopo.so``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libopo.so")
SOURCES = ["opo_abi.cu", "opo_setup.cu", "opo_plain.cu", "opo_fused.cu", "opo_fused2.cu",
           "opo_fused2_f32_f3.cu", "opo_fused2_f32_f2.cu", "opo_fused2_f64_f3.cu",
           "opo_fused2_f64_f2.cu", "opo_fused2_f32_f3_kerr.cu", "opo_fused2_f32_f2_kerr.cu",
           "opo_fused2_f64_f3_kerr.cu", "opo_fused2_f64_f2_kerr.cu", "opo_fused2_f32_f3_nodk.cu",
           "opo_fused2_f32_f2_nodk.cu", "opo_noalloc.cu"]
HEADERS = ["opo_common.cuh", "opo_internal.h", "opo_fused_desc.cuh", "opo_fused2.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
                     "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libopo.so")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Build libopo.so if any source or header is newer than it."""
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "opo.h")]
    flags = NVCC_FLAGS + list(extra_flags or [])
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc(), *flags, "-c", src, "-o", obj])
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
