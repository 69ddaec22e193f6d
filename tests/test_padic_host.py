"""The p-adic digit arithmetic of the m = 64 NTT kernels (csrc/padic.cuh) and
its limit check (csrc/ntt_bounds.cpp, pd_lazy_bounds), run on the CPU through
a small host driver (tests/native/padic_host.cu) and compared with exact
integers.

A residue mod p^4 is four base-p digits x = sum_k x_k p^k; digits may exceed
p (lazy).  mmul returns the canonical digits of a b mod p^4, pd_canon those of
x mod p^4, pd_norm digits of a congruent value near p (quotients by a shift),
pd_from_words the digits of a value given as 32-bit words, pd_to_words the
words of a value given as canonical digits.  The primes are those of the 2^28- and 2^32-bit
workloads, one just below 2^30 and a small one.
"""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "padic_host.cu")
BOUNDS = os.path.join(ROOT, "paper_1503_04955_gb300", "csrc", "ntt_bounds.cpp")
PRIMES = [998244353, 7340033, 1073479681, 12289]
W = 1 << 32


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("pd") / "padic_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-gencode",
                    "arch=compute_103a,code=sm_103a", SRC, BOUNDS, "-o", exe], check=True, capture_output=True)
    return exe


def call(driver, lines):
    r = subprocess.run([driver], input="".join(l + "\n" for l in lines), capture_output=True, text=True, check=True)
    return [[int(t) for t in line.split()] for line in r.stdout.strip().split("\n")]


def value(p, ds):
    return sum(d * p ** k for k, d in enumerate(ds))


def digits(p, v):
    return [(v // p ** k) % p for k in range(4)]


def test_primes_are_primes():
    import sympy
    for p in PRIMES:
        assert sympy.isprime(p) and p < 1 << 30


def test_product_is_canonical_and_exact(driver):
    rng = random.Random(7)
    lines, want = [], []
    for p in PRIMES:
        q = p ** 4
        cases = [([0] * 4, [0] * 4), ([p - 1] * 4, [p - 1] * 4), ([W - 1] * 4, [p - 1] * 4),
                 ([W - 1] * 4, [0, 0, 0, p - 1])]
        # lazy first factor (any 32-bit digits), canonical second factor; both lazy below 2p + 2^20
        cases += [([rng.randrange(W) for _ in range(4)], digits(p, rng.randrange(q))) for _ in range(60)]
        cases += [([rng.randrange(2 * p) for _ in range(4)], [rng.randrange(2 * p) for _ in range(4)])
                  for _ in range(30)]
        for a, b in cases:
            lines.append("mul %d %s %s" % (p, " ".join(map(str, a)), " ".join(map(str, b))))
            want.append(digits(p, value(p, a) * value(p, b) % q))
    assert call(driver, lines) == want


def test_fast_carries(driver):
    """floor(2^32/p) = 4 for the 2^32-bit workload's prime and one just below
    2^30: the carries take floor(2^64/p) as 4 2^32 + mu_lo; the product must be
    the same within the limit check's columns (a lazy below 4.3p, b canonical)."""
    rng = random.Random(10)
    lines, want = [], []
    for p in (998244353, 1073479681):
        assert (1 << 32) // p == 4
        q = p ** 4
        cases = [([0] * 4, [0] * 4), ([p - 1] * 4, [p - 1] * 4), ([W - 1] * 4, [p - 1] * 4)]
        cases += [([rng.randrange(W) for _ in range(4)], digits(p, rng.randrange(q))) for _ in range(200)]
        for a, b in cases:
            lines.append("mulf %d %s %s" % (p, " ".join(map(str, a)), " ".join(map(str, b))))
            want.append(digits(p, value(p, a) * value(p, b) % q))
    assert call(driver, lines) == want


def test_norm_and_canon(driver):
    rng = random.Random(8)
    lines, kinds = [], []
    for p in PRIMES:
        # digits whose sums with a carry stay below 2^32
        lim = W - 64 - W // p
        cases = [[0] * 4, [lim] * 4, [p] * 4, [p - 1] * 4] + [[rng.randrange(lim) for _ in range(4)] for _ in range(80)]
        for x in cases:
            lines.append("norm %d %s" % (p, " ".join(map(str, x))))
            lines.append("canon %d %s" % (p, " ".join(map(str, x))))
            kinds.append((p, x))
    got = call(driver, lines)
    for i, (p, x) in enumerate(kinds):
        nrm, can = got[2 * i], got[2 * i + 1]
        q = p ** 4
        assert value(p, nrm) % q == value(p, x) % q
        # pd_norm's quotient is v >> ceil(log2 p): a digit v becomes below v (1 - p / 2^sh) + p
        sh = p.bit_length()
        vmax = max(x) + (max(x) >> sh) + 1
        assert all(d < vmax * ((1 << sh) - p) // (1 << sh) + p + 1 for d in nrm)
        assert can == digits(p, value(p, x) % q)


def test_words_round_trip(driver):
    rng = random.Random(9)
    lines, want = [], []
    for p in PRIMES:
        q = p ** 4
        L = max(2, (q.bit_length() + 31) // 32)
        pw = sum((digits(p, pow(2, 32 * j, q)) for j in range(4)), [])
        for v in [0, 1, q - 1, W ** L - 1] + [rng.randrange(W ** L) for _ in range(50)]:
            words = [(v >> (32 * j)) & (W - 1) for j in range(L)]
            lines.append("from %d %d %s %s" % (p, L, " ".join(map(str, words)), " ".join(map(str, pw))))
            want.append(digits(p, v % q))
        for v in [0, q - 1] + [rng.randrange(q) for _ in range(50)]:
            lines.append("to %d %d %s" % (p, L, " ".join(map(str, digits(p, v)))))
            want.append([(v >> (32 * j)) & (W - 1) for j in range(L)])
    assert call(driver, lines) == want


def test_short_conversion_for_large_p(driver):
    """For p > 2^22 the digits of 2^32 mod p^4 end after the second and those
    of 2^64 after the third: the short conversion leaves those products out
    and must give the same digits for every 4-word value."""
    rng = random.Random(11)
    lines, want = [], []
    for p in (998244353, 1073479681, 754974721, 7340033):
        q = p ** 4
        pw = sum((digits(p, pow(2, 32 * j, q)) for j in range(4)), [])
        assert pw[4 + 2] == pw[4 + 3] == pw[8 + 3] == 0
        for v in [0, 1, q - 1, W ** 4 - 1] + [rng.randrange(W ** 4) for _ in range(50)]:
            words = [(v >> (32 * j)) & (W - 1) for j in range(4)]
            lines.append("from4 %d %s %s" % (p, " ".join(map(str, words)), " ".join(map(str, pw))))
            want.append(digits(p, v % q))
    assert call(driver, lines) == want


def test_limits(driver):
    """The rings of the 2^28- and 2^32-bit workloads pass the limit check;
    primes at or above 2^30, more than four words and tiny primes do not."""
    got = call(driver, ["bounds 998244353 64 4", "bounds 7340033 64 3", "bounds 1073479681 64 4",
                        "bounds 1073741827 64 4", "bounds 998244353 64 5", "bounds 2 64 2"])
    assert got[0][0] == 1 and got[1][0] == 1 and got[2][0] == 1
    assert got[3][0] == 0 and got[4][0] == 0 and got[5][0] == 0
    for g in got[:3]:
        kf, kb = g[1], g[2:8]
        assert kf == 1 and all(1 <= k <= 255 for k in kb)
    # fast carries: floor(2^32/p) = 4 for p = 998244353 and 1073479681, 585 for 7340033
    assert got[0][9] == 1 and got[2][9] == 1 and got[1][9] == 0
    # DFTs on digits (the forward levels keeping digits in HBM) within their limits
    assert got[0][10] == 1 and got[1][10] == 1 and got[2][10] == 1
