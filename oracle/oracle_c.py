"""ctypes wrapper of the C transcription of the oracle (test infrastructure only).

``build()`` compiles ``oracle/dkss_oracle.c`` with gcc into
``oracle/_build/libdkss_oracle.so``; ``load()`` builds on first use.
The functions take and return Python ints / numpy arrays.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dkss_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libdkss_oracle.so")

_lib = None


def build(force=False):
    """Compile the oracle's C part (plain -O2, no target-specific flags), with
    OpenMP over its independent loops when the compiler supports it."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", SRC, "-o", tmp]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_r_mul.argtypes = [ctypes.c_uint32, u64p, u64p, u64p, u64p]
        lib.oracle_fft.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u64p, u64p, u64p, u64p]
        lib.oracle_dkss_mul.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, u64p, u64p, u64p, u64p, u64p,
                                        u64p, u64p, u64p, u64p]
        lib.oracle_fft_alpha_point.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, u64p, u64p, ctypes.c_uint64, u64p]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        for f in (lib.oracle_r_mul, lib.oracle_fft, lib.oracle_dkss_mul, lib.oracle_fft_alpha_point,
                  lib.oracle_set_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(arr):
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def words2(values):
    """Residues (< 2^128) -> flat uint64 array, two little-endian words each."""
    flat = np.zeros(2 * len(values), dtype=np.uint64)
    for k, v in enumerate(values):
        flat[2 * k] = v & 0xFFFFFFFFFFFFFFFF
        flat[2 * k + 1] = v >> 64
    return flat


def from_words2(flat):
    flat = np.asarray(flat, dtype=np.uint64)
    lo = flat[0::2].tolist()
    hi = flat[1::2].tolist()
    return [l | (h << 64) for l, h in zip(lo, hi)]


def set_threads(n):
    """Host threads of the oracle's parallel loops (0: leave as is); returns
    the count in effect (1 without OpenMP)."""
    return load().oracle_set_threads(int(n))


def r_mul(x, y, pz):
    lib = load()
    m = len(x)
    out = np.zeros(2 * m, dtype=np.uint64)
    rc = lib.oracle_r_mul(m, _ptr(words2([pz])), _ptr(words2(x)), _ptr(words2(y)), _ptr(out))
    assert rc == 0
    return from_words2(out)


def fft(a_elems, M, m, pz, rho):
    """Forward DFT with root rho of 2M elements of R (lists of m ints)."""
    lib = load()
    flat_in = words2([v for el in a_elems for v in el])
    out = np.zeros_like(flat_in)
    rc = lib.oracle_fft(M, m, _ptr(words2([pz])), _ptr(words2(rho)), _ptr(flat_in), _ptr(out))
    assert rc == 0
    vals = from_words2(out)
    return [vals[i * m:(i + 1) * m] for i in range(2 * M)]


DUMP_NAMES = ("a_hat", "b_hat", "c_hat", "c")


def dkss_mul(a_limbs, b_limbs, par, rho, dumps=False):
    """c = a*b with the C oracle.  a_limbs, b_limbs: uint64 arrays of
    ceil(N/64) limbs.  Returns (c_limbs, dumps) where dumps maps 'a_hat',
    'b_hat', 'c_hat', 'c' to uint64 arrays of shape (2M, m, 2) or is None.
    dumps may also be a collection of those names (only they are kept)."""
    lib = load()
    nw = (par.n_bits + 63) // 64
    a = np.ascontiguousarray(a_limbs, dtype=np.uint64)
    b = np.ascontiguousarray(b_limbs, dtype=np.uint64)
    assert a.size == nw and b.size == nw
    c = np.zeros(2 * nw, dtype=np.uint64)
    shape = (par.P2, par.m, 2)
    names = DUMP_NAMES if dumps is True else tuple(dumps) if dumps else ()
    d = {k: np.zeros(shape, dtype=np.uint64) for k in names} if names else None
    rc = lib.oracle_dkss_mul(par.n_bits, par.M, par.m, par.u, _ptr(words2([par.pz])),
                             _ptr(words2(rho)), _ptr(a), _ptr(b), _ptr(c),
                             *[_ptr(d[k]) if d and k in d else None for k in DUMP_NAMES])
    assert rc == 0
    return c, d


def fft_alpha_point(a_limbs, par, k):
    """a_hat at frequency k*mu, i.e. sum_j a_j alpha^(k j) (Section 3.2.3: rho^mu = alpha)."""
    lib = load()
    a = np.ascontiguousarray(a_limbs, dtype=np.uint64)
    out = np.zeros(2 * par.m, dtype=np.uint64)
    rc = lib.oracle_fft_alpha_point(par.n_bits, par.M, par.m, par.u, _ptr(words2([par.pz])), _ptr(a), k, _ptr(out))
    assert rc == 0
    return from_words2(out)
