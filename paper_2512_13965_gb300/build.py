"""Build libgmc.so in-tree with nvcc for sm_103a (GB300).

Each .cu translation unit compiles in parallel to an object file; the objects
link into paper_2512_13965_gb300/_lib/libgmc.so. No torch headers are used:
the library's ABI is plain C (include/gmc.h).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libgmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "gmc.h"))
    cc = nvcc()
    jobs = []
    for src in sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src[:-3] + ".o")
        if force or _stale(o, [s] + headers):
            jobs.append([cc] + ARCH + FLAGS + list(extra) + ["-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            res = list(ex.map(lambda cmd: subprocess.run(cmd, capture_output=True, text=True), jobs))
        failed = [(j, r) for j, r in zip(jobs, res) if r.returncode != 0]
        for j, r in zip(jobs, res):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
        if failed:
            raise RuntimeError("nvcc failed on: " + ", ".join(os.path.basename(j[-3]) for j, _ in failed))
    objs = [os.path.join(OUT, s[:-3] + ".o") for s in sources()]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lcuda"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
