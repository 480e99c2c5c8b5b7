"""Build the sm_103a shared library ``liblbm.so`` in-tree with nvcc (no torch extension).

Each translation unit is compiled in parallel, then linked with ``nvcc -shared``.
The output lives next to this file and is git-ignored.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
SOURCES = ["lbm_api.cu", "batch.cu", "mlp.cu", "thermo.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _obj(src):
    return os.path.join(BUILD, os.path.splitext(src)[0] + ".o")


def _stamp(src):
    return _obj(src) + ".flags"


def _cmd(src, obj):
    return [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *EXTRA,
            "-c", os.path.join(CSRC, src), "-o", obj]


def _deps_newer(obj, src):
    if not os.path.exists(obj):
        return True
    try:  # rebuild when the compile flags changed
        with open(_stamp(src)) as f:
            if f.read() != " ".join(_cmd(src, obj)):
                return True
    except OSError:
        return True
    t = os.path.getmtime(obj)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "lbm.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


# Extra nvcc flags for tuning builds (e.g. LBM_NVCC_EXTRA="-DLBM_FEP_STAGES=8"); the default
# build uses none.
EXTRA = os.environ.get("LBM_NVCC_EXTRA", "").split()


def _compile(src, verbose):
    obj = _obj(src)
    cmd = _cmd(src, obj)
    stamp = " ".join(cmd)
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    with open(_stamp(src), "w") as f:
        f.write(stamp)
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    todo = [s for s in SOURCES if force or verbose or _deps_newer(_obj(s), s)]
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=len(todo)) as ex:
            logs = list(ex.map(lambda s: _compile(s, verbose), todo))
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [NVCC, *ARCH, "-shared", *[_obj(s) for s in SOURCES], "-o", tmp, "-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    if verbose:
        for l in logs:
            sys.stderr.write(l)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
