"""Build libdkss.so in-tree with nvcc for sm_103a (no CMake).

Translation units: the C ABI (capi.cu), the host number theory
(host_math.cpp) and one instantiation of the stage kernels per supported
(m, L, LR) triple (inst.cu compiled with -DDKSS_INST_M/_L/_LR), compiled in
parallel and linked into paper_1503_04955_gb300/_build/libdkss.so.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libdkss.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (m, L, LR): ring degree, 32-bit limbs of stored residues, 26-bit limbs of products
TRIPLES = [(m, L, LR) for m in (16, 32, 64) for (L, LR) in ((2, 2), (2, 3), (3, 3), (3, 4), (4, 4), (4, 5))]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdkss")
    return path


def _flags(extra_ptxas=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]
    if extra_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _units():
    units = [("capi.o", os.path.join(CSRC, "capi.cu"), []),
             ("decode_static.o", os.path.join(CSRC, "decode_static.cu"), []),
             ("mersenne.o", os.path.join(CSRC, "mersenne.cu"), []),
             ("batch.o", os.path.join(CSRC, "batch.cu"), []),
             ("mlp.o", os.path.join(CSRC, "mlp.cu"), []),
             ("host_math.o", os.path.join(CSRC, "host_math.cpp"), ["-x", "cu"]),
             ("ntt_bounds.o", os.path.join(CSRC, "ntt_bounds.cpp"), ["-x", "cu"])]
    for m, L, LR in TRIPLES:
        units.append(("inst_m%d_L%d_R%d.o" % (m, L, LR), os.path.join(CSRC, "inst.cu"),
                      ["-DDKSS_INST_M=%d" % m, "-DDKSS_INST_L=%d" % L, "-DDKSS_INST_LR=%d" % LR]))
    return units


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.abspath(__file__)]


def lib_path():
    return os.path.join(OUT_DIR, LIB_NAME)


def build(force=False, verbose=False, ptxas_info=False):
    """Compile and link libdkss.so; skipped when it is newer than every source."""
    out = lib_path()
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(p) for p in _sources())
        if os.path.getmtime(out) >= newest:
            return out
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        obj, src, extra = unit
        cmd = [cc] + _flags(ptxas_info) + extra + ["-c", src, "-o", os.path.join(OUT_DIR, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (obj, " ".join(cmd), r.stderr))
        return obj, r.stderr

    units = _units()
    workers = min(len(units), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(compile_one, units))
    if verbose or ptxas_info:
        for obj, err in results:
            if err.strip():
                sys.stderr.write("== %s\n%s\n" % (obj, err))
    objs = [os.path.join(OUT_DIR, u[0]) for u in units]
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
