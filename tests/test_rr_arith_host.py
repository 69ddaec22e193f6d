"""The limb arithmetic the R-multiplication kernels inline (csrc/rr_arith.cuh,
csrc/ntt_rmul.cuh), run on the CPU through a small host driver
(tests/native/rr_arith_host.cu) and compared with exact integers.

Residues mod q = p^z are LR limbs of 26 bits, R' = 2^(26 LR).  The Montgomery
product of the direct form returns a b R'^-1 mod q, canonical; the lazy one of
the NTT form returns normalised limbs of a value congruent to it and below
a b / R' + q; canon maps a normalised value below 2q to [0, q); lz_norm
carries limbs below 2^32 into 26-bit limbs; neg_rr is q - y mod q; to_rr and
from_rr convert between 32-bit words and 26-bit limbs.  The moduli are those
of the library's plans for every workload.
"""
import os
import random
import shutil
import subprocess

import pytest

import dkss_synth as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "rr_arith_host.cu")
M26 = (1 << 26) - 1


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("rr") / "rr_arith_host")
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-gencode",
                    "arch=compute_103a,code=sm_103a", SRC, "-o", exe], check=True, capture_output=True)
    return exe


@pytest.fixture(scope="module")
def rings():
    """(q, LR) of the library's plans for the workloads and two small rings."""
    import paper_1503_04955_gb300 as pkg
    pkg.buildlib.build()
    cfgs = [syn.workload_params(k) for k in syn.WORKLOADS]
    cfgs += [(4096, 32, 16, 16, 40961, 3), (786432, 2048, 32, 24, 65537, 5)]
    out = []
    for cfg in cfgs:
        _, consts = pkg.plan_rho(*cfg)
        out.append((consts["pz"], consts["LR"]))
    return out


def limbs(v, n):
    return [(v >> (26 * i)) & M26 if i + 1 < n else v >> (26 * i) for i in range(n)]


def value(ls):
    return sum(x << (26 * i) for i, x in enumerate(ls))


def call(driver, reqs):
    text = "".join("%s %d %d %s\n" % (op, lr, npr, " ".join(str(w) for w in q + x + y))
                   for op, lr, npr, q, x, y in reqs)
    r = subprocess.run([driver], input=text, capture_output=True, text=True, check=True)
    return [[int(t) for t in line.split()] for line in r.stdout.strip().split("\n")]


def nprime(q):
    return (-pow(q, -1, 1 << 26)) % (1 << 26)


def test_montgomery_product_direct_form(driver, rings):
    rng = random.Random(1)
    reqs, want = [], []
    for q, lr in rings:
        rinv = pow(1 << (26 * lr), -1, q)
        for a, b in [(0, 0), (q - 1, q - 1), (1, q - 1)] + [(rng.randrange(q), rng.randrange(q)) for _ in range(40)]:
            reqs.append(("mont", lr, nprime(q), limbs(q, lr), limbs(a, lr), limbs(b, lr)))
            want.append(a * b * rinv % q)
    got = call(driver, reqs)
    for (op, lr, _, ql, _, _), g, w in zip(reqs, got, want):
        assert value(g) == w and all(x <= M26 for x in g)


def test_lazy_montgomery_product(driver, rings):
    """Inputs with limbs above 26 bits (lazy sums): the result is congruent to
    a b R'^-1, its limbs are normalised, and it stays below a b / R' + q."""
    rng = random.Random(2)
    reqs, meta = [], []
    for q, lr in rings:
        rp = 1 << (26 * lr)
        for _ in range(60):
            xa = [rng.randrange(1 << 28) for _ in range(lr)]
            xb = [rng.randrange(1 << 28) for _ in range(lr)]
            reqs.append(("mmul", lr, nprime(q), limbs(q, lr), xa, xb))
            meta.append((q, rp, value(xa), value(xb)))
        for a, b in [(q - 1, q - 1), (2 * q - 1, q - 1)]:
            reqs.append(("mmul", lr, nprime(q), limbs(q, lr), limbs(a, lr), limbs(b, lr)))
            meta.append((q, rp, a, b))
    got = call(driver, reqs)
    for (q, rp, a, b), g in zip(meta, got):
        v = value(g)
        assert v % q == a * b * pow(rp, -1, q) % q
        assert all(x <= M26 for x in g[:-1])
        assert v * rp < a * b + q * rp


def test_canon_norm_neg(driver, rings):
    rng = random.Random(3)
    reqs, want = [], []
    for q, lr in rings:
        zero = [0] * lr
        for v in [0, q - 1, q, q + 1, 2 * q - 1] + [rng.randrange(2 * q) for _ in range(30)]:
            reqs.append(("canon", lr, nprime(q), limbs(q, lr), limbs(v, lr), zero))
            want.append(("canon", q, v % q))
        for y in [0, 1, q - 1] + [rng.randrange(q) for _ in range(20)]:
            reqs.append(("neg", lr, nprime(q), limbs(q, lr), limbs(y, lr), zero))
            want.append(("neg", q, (q - y) % q))
        for _ in range(20):
            x = [rng.randrange(1 << 32) for _ in range(lr - 1)] + [rng.randrange(1 << 30)]
            reqs.append(("norm", lr, 0, zero, x, zero))
            want.append(("norm", q, value(x)))
    got = call(driver, reqs)
    for (kind, q, w), g in zip(want, got):
        assert value(g) == w
        assert all(x <= M26 for x in g[:-1])


def test_reduce_raw_of_lazy_values(driver, rings):
    """reduce_raw: a lazy value (limbs up to 32 bits, quotient by q below
    2^12, the plan's limits) to its canonical residue, with the integer
    quotient estimate from q's two top limbs; rings whose top two limbs hold
    at least 2^18 (the plan's condition for using it)."""
    rng = random.Random(5)
    reqs, want = [], []
    for q, lr in rings:
        ql = limbs(q, lr)
        if (ql[-1] << 26) + ql[-2] < (1 << 18):
            continue
        for v in [0, q - 1, q, 2 * q - 1, 3 * q, (1 << 12) * q - 1] + \
                 [rng.randrange((1 << 12) * q) for _ in range(60)]:
            x = limbs(v, lr)
            for i in range(lr - 1):            # move value into lower limbs (lazy form)
                if x[i + 1] and rng.random() < 0.5:
                    d = rng.randrange(1, min(x[i + 1], 32) + 1)
                    x[i + 1] -= d
                    x[i] += d << 26
            assert value(x) == v and all(w < (1 << 32) for w in x)
            reqs.append(("rraw", lr, nprime(q), ql, x, [0] * lr))
            want.append(v % q)
    assert reqs
    got = call(driver, reqs)
    for g, w in zip(got, want):
        assert value(g) == w and all(x <= M26 for x in g[:-1])


@pytest.mark.parametrize("L,LR", [(2, 2), (2, 3), (3, 4), (4, 4), (4, 5)])
def test_word_limb_round_trip(driver, L, LR):
    """to_rr then from_rr of L 32-bit words (value below 2^(26 LR)); the
    driver reads LR words and converts the first L."""
    rng = random.Random(4 + L + LR)
    bits = min(32 * L, 26 * LR)
    reqs, vals = [], []
    for v in [0, (1 << bits) - 1] + [rng.randrange(1 << bits) for _ in range(30)]:
        words = [(v >> (32 * i)) & 0xFFFFFFFF for i in range(L)]
        reqs.append(("rt%d" % L, LR, 0, [0] * LR, (words + [0] * LR)[:LR], [0] * LR))
        vals.append((v, words))
    got = call(driver, reqs)
    for (v, words), g in zip(vals, got):
        rr, back = g[:LR], g[LR:]
        assert value(rr) == v and all(x <= M26 for x in rr)
        assert back == words


def test_lucas_lehmer_fold(driver):
    """The reduction of dkss_ll_step (csrc/mersenne.cuh) on the host:
    s = (c - 2) mod (2^p - 1) for c < 2^(2p), including c = 0, 1, 2, M_p,
    M_p^2, 2^(2p) - 1 and word-boundary exponents."""
    rng = random.Random(5)
    lines, want = [], []
    for p in list(range(3, 200)) + [521, 607, 1277, 1279, 2203, 4423]:
        mp = (1 << p) - 1
        w = (p + 63) // 64
        cases = [0, 1, 2, 3, mp - 1, mp, mp + 1, 2 * mp, mp * mp, (1 << (2 * p)) - 1, 1 << p, (1 << p) + 1]
        cases += [rng.getrandbits(2 * p) for _ in range(12)] + [rng.randrange(mp) ** 2 for _ in range(4)]
        for c in cases:
            words = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(2 * w)]
            lines.append("ll %d %s\n" % (p, " ".join(str(x) for x in words)))
            want.append((c - 2) % mp)
    r = subprocess.run([driver], input="".join(lines), capture_output=True, text=True, check=True)
    got = [sum(int(t) << (64 * i) for i, t in enumerate(line.split())) for line in r.stdout.strip().split("\n")]
    assert got == want
