"""Builds libqvx.so in-tree: the planner and C interface (g++) and the kernels (nvcc, sm_103a)."""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libqvx.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SOURCES = ["planner.cpp", "capi.cpp"]
CUDA_SOURCES = ["kernels.cu", "noalloc.cu", "gemm_tc.cu"]
HEADERS = ["plan.h", "device_program.h", "kernels.h", "plan_handle.h", "device_util.cuh"]


def _cuda_home():
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home:
        return home
    nvcc = shutil.which("nvcc")
    return os.path.dirname(os.path.dirname(nvcc)) if nvcc else "/usr/local/cuda"


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = os.path.join(ROOT, "include")
    deps = [os.path.join(CSRC, f) for f in HOST_SOURCES + CUDA_SOURCES + HEADERS] + [os.path.join(inc, "qvx.h")]
    if not force and not _stale(OUT, deps):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    jobs, objs = [], []
    for f in HOST_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        # no fused multiply-adds in the planner's floating point, so that plans (orders chosen
        # by cost comparisons) are the same on x86 and on Arm hosts
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-pthread", "-Wall", "-I", inc,
               "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
        objs.append(o)
    for f in CUDA_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        cmd = [nvcc] + ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", inc,
                               "-c", os.path.join(CSRC, f), "-o", o]
        jobs.append(cmd)
        objs.append(o)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in jobs]
    failed = []
    for c, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(" ".join(c))
    if failed:
        raise RuntimeError("compile failed:\n" + "\n".join(failed))
    tmp = OUT + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC,-pthread", "-o", tmp] + objs)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
