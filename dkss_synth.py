"""Seeded synthetic operands for DKSS_MUL tests and benchmarks.

This module holds no arithmetic of the multiplication method: it only draws
uniform random bits.  Both the CPU oracle and the CUDA path take their inputs
from here, so neither depends on the other.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Its i-th output is a fixed bijective mix of
``seed + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64), so limb i of an operand is
computed independently of the others (counter-based), which lets numpy draw
67M limbs at once.

Operands are little-endian arrays of 64-bit limbs, the number representation of
the thesis (Section 2.1): limb k holds bits [64k, 64k + 64).
"""
import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
BASE_SEED = 0x444B535300000000  # "DKSS" in the top half


def _mix64(z):
    """SplitMix64 output function on a uint64 numpy array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed, count, start=0):
    """Outputs start .. start+count-1 of the SplitMix64 sequence seeded with ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        state = np.uint64(seed % (1 << 64)) + idx * GOLDEN_GAMMA
        return _mix64(state)


def stream_seed(seed, stream):
    """Seed of sub-stream ``stream``: one SplitMix64 output of (seed, stream)."""
    return int(splitmix64(seed, 1, start=stream)[0])


def n_limbs(n_bits):
    return (n_bits + 63) // 64


def operand(n_bits, seed, stream):
    """Uniform random integer in [0, 2^n_bits) as little-endian uint64 limbs."""
    k = n_limbs(n_bits)
    limbs = splitmix64(stream_seed(seed, stream), k)
    top = n_bits - 64 * (k - 1)
    if k and top < 64:
        limbs[-1] &= np.uint64((1 << top) - 1)
    return limbs


def operand_pair(n_bits, seed, product=0):
    """Operands (a, b) of product ``product``: streams 2*product and 2*product+1."""
    return operand(n_bits, seed, 2 * product), operand(n_bits, seed, 2 * product + 1)


def config_seed(index):
    return BASE_SEED + index


def special_operand(n_bits, kind):
    """Fixed edge-case operands: 'zero', 'one', 'ones' (2^N - 1), 'top' (2^(N-1))."""
    k = n_limbs(n_bits)
    x = np.zeros(k, dtype=np.uint64)
    if kind == "zero" or k == 0:
        return x
    if kind == "one":
        x[0] = 1
    elif kind == "ones":
        x[:] = np.uint64(0xFFFFFFFFFFFFFFFF)
        top = n_bits - 64 * (k - 1)
        if top < 64:
            x[-1] = np.uint64((1 << top) - 1)
    elif kind == "top":
        bit = n_bits - 1
        x[bit // 64] = np.uint64(1 << (bit % 64))
    else:
        raise ValueError(kind)
    return x


def log_uniform_lengths(count, seed, lo_exp=14, hi_exp=20):
    """Operand bit-lengths for the batched workload: 2^x with x uniform in
    [lo_exp, hi_exp], rounded up to whole 64-bit limbs."""
    r = splitmix64(seed, count, start=1 << 40)
    x = lo_exp + (hi_exp - lo_exp) * ((r >> np.uint64(11)).astype(np.float64) / float(1 << 53))
    bits = np.exp2(x)
    return (64 * np.ceil(bits / 64.0)).astype(np.int64)


def to_int(limbs):
    """Little-endian uint64 limbs -> Python int (test helper)."""
    return int.from_bytes(np.asarray(limbs, dtype="<u8").tobytes(), "little")


def from_int(x, k):
    """Python int -> k little-endian uint64 limbs (test helper)."""
    return np.frombuffer(int(x).to_bytes(8 * k, "little"), dtype="<u8").copy()


# Workload shapes: (n_bits, M, m, u, p, z) of the single-product cases, named
# by size.  Operands of workload k are drawn with seed config_seed(k).
WORKLOADS = {
    "dkss_65536b": dict(index=0, n_bits=1 << 16, M=512, m=16, u=16, p=12289, z=4),
    "dkss_2p24b": dict(index=1, n_bits=1 << 24, M=1 << 15, m=32, u=32, p=65537, z=6),
    "dkss_2p28b": dict(index=3, n_bits=1 << 28, M=1 << 18, m=64, u=32, p=7340033, z=4),
    "dkss_2p32b": dict(index=4, n_bits=1 << 32, M=1 << 22, m=64, u=32, p=998244353, z=4),
    # the 2^32-bit workload's ring and encoding at 2^26 bits (ncu captures: a
    # few hundred MB on the device, still larger than L2)
    "dkss_2p26b_ring2p32": dict(index=5, n_bits=1 << 26, M=1 << 16, m=64, u=32, p=998244353, z=4),
}
BATCH_WORKLOAD = dict(index=2, count=4096, lo_exp=14, hi_exp=20)


def workload_params(name):
    w = WORKLOADS[name]
    return w["n_bits"], w["M"], w["m"], w["u"], w["p"], w["z"]
