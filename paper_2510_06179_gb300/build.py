"""Build the CUDA library libdmpc.so in-tree for sm_103a (nvcc, no cmake).

Each .cu translation unit compiles in parallel; the objects link into one shared library
with the C-ABI of include/dmpc.h."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libdmpc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
TEAMS = (32, 64, 128, 256)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "177",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(obj, src_deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in src_deps)


def build(verbose=False, jobs=None, extra=()):
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "dmpc.h"))
    cmds, objs = [], []
    for s in _sources():
        src = os.path.join(CSRC, s)
        # kernel units (k_*.cu) are compiled once per team size: more, smaller units in parallel
        variants = [(f"_t{t}", [f"-DDMPC_TEAM={t}"]) for t in TEAMS] if s.startswith("k_") else [("", [])]
        for suffix, defs in variants:
            obj = os.path.join(OUT, s[:-3] + suffix + ".o")
            objs.append(obj)
            if _stale(obj, [src] + headers):
                cmds.append([nvcc, *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj])
    # longest units first (rigid body, mixed, LQ) so the pool finishes early
    weight = lambda c: (2 if any(k in c[-3] for k in ("rigid", "mixed", "lq", "single")) else 1)
    cmds.sort(key=weight, reverse=True)
    for f in os.listdir(OUT):
        if f.endswith(".o") and os.path.join(OUT, f) not in objs:
            os.remove(os.path.join(OUT, f))
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 4))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(" ".join(os.path.basename(c) for c in cmd[-3:]), flush=True)
        return r
    with ThreadPoolExecutor(jobs) as ex:
        list(ex.map(run, cmds))
    if cmds or not os.path.exists(LIB):
        link = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
