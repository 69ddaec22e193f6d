"""Pins of the CPU oracle against the thesis and the mathematics (no GPU).

Each check uses something other than the oracle function itself: values the
thesis prints, closed forms, invariants the thesis proves, brute force on tiny
inputs, or the exact integer product.
"""
import os
import random

import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# small parameter sets: (n_bits, M, m, u, p, z); 2M | p-1 and the bound holds
TINY = [
    (32, 8, 4, 2, 17, 2),       # 2M = 16 = 2m*2: one bad-multiplication level
    (24, 4, 4, 3, 17, 3),       # 2M = 8 = 2m: a single alpha-power DFT
    (192, 64, 4, 3, 257, 2),    # 2M = 128 = 8*8*2: recursion two levels deep
    (512, 32, 8, 4, 193, 3),    # 2M = 64 = 16*4: last level shorter than 2m
    (1000, 64, 8, 4, 257, 3),   # N not a multiple of 64, zero-padded top
]


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


def brute_order(g, p):
    x, k = g % p, 1
    while x != 1:
        x = x * g % p
        k += 1
    return k


# ---- input generator --------------------------------------------------------

def test_splitmix64_reference_vectors():
    # SplitMix64 (Steele, Lea, Flood 2014): published first outputs
    assert int(syn.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert [int(v) for v in syn.splitmix64(1234567, 3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_operand_masking_and_specials():
    a = syn.operand(1000, 7, 0)
    assert a.size == 16 and syn.to_int(a) < (1 << 1000)
    assert syn.to_int(syn.special_operand(1000, "ones")) == (1 << 1000) - 1
    assert syn.to_int(syn.special_operand(1000, "top")) == 1 << 999
    assert syn.to_int(syn.special_operand(1000, "one")) == 1


# ---- primality, generators, roots (Section 3.2.2 / 3.2.3, Section 2.8 table) --

def test_lucas_matches_trial_division():
    def trial(n):
        return n >= 2 and all(n % d for d in range(2, int(n ** 0.5) + 1))
    for n in range(0, 3000):
        assert o.lucas_is_prime(n) == trial(n), n
    for n in (561, 1105, 1729, 2465, 65535, 65537 * 3, (1 << 32) + 1):
        assert not o.lucas_is_prime(n)
    for n in (12289, 65537, 7340033, 998244353, 167772161, 469762049):
        assert o.lucas_is_prime(n)


def test_qmul_table_generators_and_roots():
    for bits, p, h, k, g, n, omega in read_golden("qmul_primes_roots.txt"):
        assert p == h * (1 << k) + 1 and n == 1 << k
        assert o.lucas_is_prime(p)
        assert o.smallest_generator(p) == g
        zeta_1 = o.hensel_lift(g, p, 1)            # z = 1: no lifting
        assert pow(zeta_1, (p - 1) // n, p) == omega


def test_smallest_generator_brute_force():
    for p in [q for q in range(3, 800) if o.lucas_is_prime(q)]:
        g = o.smallest_generator(p)
        assert brute_order(g, p) == p - 1
        assert all(brute_order(x, p) < p - 1 for x in range(2, g))


def test_root_example_mod_17():
    for mod, omega, order in read_golden("small_root_example.txt"):
        assert brute_order(omega, mod) == order


@pytest.mark.parametrize("p,z", [(17, 3), (193, 4), (12289, 4), (65537, 6), (7340033, 4), (998244353, 4)])
def test_hensel_is_teichmuller_lift(p, z):
    zeta = o.smallest_generator(p)
    x = o.hensel_lift(zeta, p, z)
    pz = p ** z
    # closed form: the unique (p-1)-th root of unity mod p^z congruent to zeta
    assert x == pow(zeta, p ** (z - 1), pz)
    assert pow(x, p - 1, pz) == 1 and x % p == zeta


ALL_PARAMS = TINY + [syn.workload_params(k) for k in syn.WORKLOADS]


@pytest.mark.parametrize("cfg", ALL_PARAMS)
def test_rho_invariants(cfg):
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    q, m = par.pz, par.m
    alpha = [0, 1] + [0] * (m - 2)
    minus_one = [q - 1] + [0] * (m - 1)
    one = o.r_one(m)
    # omega: principal 2M-th root of unity in P (Section 3.2.2)
    assert pow(r.omega, par.P2, q) == 1 and pow(r.omega, par.M, q) == q - 1
    # gamma^m = -1 (Section 3.2.3)
    assert pow(r.gamma, m, q) == q - 1
    # rho^mu = alpha, rho^M = -1, rho^(2M) = 1
    assert o.r_pow(r.rho, par.mu, q) == alpha
    assert o.r_pow(r.rho, par.M, q) == minus_one
    assert o.r_pow(r.rho, par.P2, q) == one
    # Lagrange data points: rho(gamma^i) = omega^i for odd i
    for i in range(1, 2 * m, 2):
        gi = pow(r.gamma, i, q)
        assert sum(c * pow(gi, k, q) for k, c in enumerate(r.rho)) % q == pow(r.omega, i, q)
    # the interpolation divides by gamma^i - gamma^j (i != j odd): units of P,
    # i.e. not divisible by p (Section 3.2.3)
    pts = [pow(r.gamma, i, q) for i in range(1, 2 * m, 2)]
    assert all((x - y) % par.p != 0 for a, x in enumerate(pts) for y in pts[:a])


@pytest.mark.parametrize("cfg", TINY[:3])
def test_rho_is_principal(cfg):
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    q = par.pz
    for j in range(1, par.P2):
        rj = o.r_pow(r.rho, j, q)
        acc, x = o.r_zero(par.m), o.r_one(par.m)
        for _ in range(par.P2):
            acc = o.r_add(acc, x, q)
            x = o.r_mul(x, rj, q)
        assert acc == o.r_zero(par.m)


# ---- arithmetic in R ----------------------------------------------------------

def alpha_vec(k, m, q):
    """alpha^k written out independently of r_shift."""
    k %= 2 * m
    v = [0] * m
    if k < m:
        v[k] = 1
    else:
        v[k - m] = q - 1
    return v


def test_r_mul_small_closed_form():
    q = 10007
    for _ in range(50):
        x0, x1, y0, y1 = (random.randrange(q) for _ in range(4))
        # (x0 + x1 a)(y0 + y1 a) with a^2 = -1
        assert o.r_mul([x0, x1], [y0, y1], q) == [(x0 * y0 - x1 * y1) % q, (x0 * y1 + x1 * y0) % q]


@pytest.mark.parametrize("cfg", TINY + [syn.workload_params("dkss_2p24b")])
def test_r_mul_evaluation_homomorphism(cfg):
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    q, m = par.pz, par.m
    rng = random.Random(5)
    for _ in range(5):
        x = [rng.randrange(q) for _ in range(m)]
        y = [q - 1 - rng.randrange(3) for _ in range(m)]    # extreme residues
        c = o.r_mul(x, y, q)
        for i in range(1, 2 * m, 2):
            g = pow(r.gamma, i, q)
            ev = lambda v: sum(cf * pow(g, k, q) for k, cf in enumerate(v)) % q
            assert ev(c) == ev(x) * ev(y) % q


def test_r_shift_is_alpha_power_product():
    q, m = 257 ** 2, 8
    rng = random.Random(1)
    x = [rng.randrange(q) for _ in range(m)]
    for k in range(-3, 3 * m):
        assert o.r_shift(x, k, q) == o.r_mul(x, alpha_vec(k, m, q), q)
    assert o.r_shift(x, m, q) == [(-v) % q for v in x]


# ---- FFT (Section 3.2.5) --------------------------------------------------------

@pytest.mark.parametrize("cfg", TINY)
def test_alpha_dft_brute_force(cfg):
    par = o.Params(*cfg).check()
    q, m = par.pz, par.m
    rng = random.Random(2)
    for n in (2, 4, 2 * m):
        step = 2 * m // n
        e = [[rng.randrange(q) for _ in range(m)] for _ in range(n)]
        out = o.alpha_dft(e, step, par)
        for v in range(n):
            acc = o.r_zero(m)
            for j in range(n):
                acc = o.r_add(acc, o.r_mul(e[j], alpha_vec(step * j * v, m, q), q), q)
            assert out[v] == acc


@pytest.mark.parametrize("cfg", TINY)
def test_dkss_fft_brute_force_and_inverse(cfg):
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    q, m = par.pz, par.m
    table = o.rho_table(r.rho, par)
    rng = random.Random(3)
    a = [[rng.randrange(q) for _ in range(m)] for _ in range(par.P2)]
    a_hat = o.dkss_fft(a, table, par)
    for k in range(par.P2):
        rk = o.r_pow(r.rho, k, q)
        acc, x = o.r_zero(m), o.r_one(m)
        for j in range(par.P2):
            acc = o.r_add(acc, o.r_mul(a[j], x, q), q)
            x = o.r_mul(x, rk, q)
        assert a_hat[k] == acc
    assert o.dkss_inverse(a_hat, table, par) == a
    # DFT of x^k is (rho^(ik))_i
    k = 3
    xk = [o.r_zero(m) for _ in range(par.P2)]
    xk[k] = o.r_one(m)
    assert o.dkss_fft(xk, table, par) == [o.r_pow(r.rho, i * k, q) for i in range(par.P2)]


def test_rho_table_and_power():
    par = o.Params(*TINY[2]).check()
    r = o.compute_roots(par)
    table = o.rho_table(r.rho, par)
    for e in range(0, 3 * par.P2, 7):
        assert o.rho_power(e, table, par) == o.r_pow(r.rho, e, par.pz)


# ---- encode / decode / whole product ----------------------------------------

@pytest.mark.parametrize("cfg", TINY)
def test_encode_layout_and_decode(cfg):
    par = o.Params(*cfg).check()
    rng = random.Random(4)
    a = rng.getrandbits(par.n_bits)
    enc = o.encode(a, par)
    assert len(enc) == par.P2
    assert all(el == [0] * par.m for el in enc[par.M:])
    assert all(el[par.h:] == [0] * par.h for el in enc)
    assert all(0 <= v < (1 << par.u) for el in enc for v in el)
    # decode is the weighted sum 2^(u(i h + t)) of Section 3.2.8
    assert o.decode(enc, par) == a


@pytest.mark.parametrize("cfg", TINY)
def test_dkss_mul_exact(cfg):
    par = o.Params(*cfg).check()
    rng = random.Random(6)
    r = o.compute_roots(par)
    N = par.n_bits
    cases = [(rng.getrandbits(N), rng.getrandbits(N)) for _ in range(6)]
    cases += [(0, 0), (1, (1 << N) - 1), ((1 << N) - 1, (1 << N) - 1), (1 << (N - 1), 1 << (N - 1))]
    for a, b in cases:
        assert o.dkss_mul(a, b, par, r) == a * b


def test_dkss_mul_matches_omul():
    par = o.Params(*TINY[4]).check()
    rng = random.Random(8)
    a, b = rng.getrandbits(1000), rng.getrandbits(1000)
    aw = [int(v) for v in syn.from_int(a, 16)]
    bw = [int(v) for v in syn.from_int(b, 16)]
    c = o.omul(aw, bw)
    assert sum(w << (64 * k) for k, w in enumerate(c)) == o.dkss_mul(a, b, par)


def test_coefficient_bound_attained():
    """a = b = 2^N - 1 reaches the inner-coefficient maximum (1/2) M m (2^u-1)^2
    (Section 3.2.2) at outer index M-1, inner index m/2-1."""
    par = o.Params(*TINY[0]).check()
    st = {}
    a = (1 << par.n_bits) - 1
    assert o.dkss_mul(a, a, par, stages=st) == a * a
    peak = par.M * par.h * ((1 << par.u) - 1) ** 2
    assert st["c"][par.M - 1][par.h - 1] == peak
    assert max(v for el in st["c"] for v in el) == peak


def test_dkss_mul_65536_bits_python():
    par = o.Params(*syn.workload_params("dkss_65536b")).check()
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(0))
    a, b = syn.to_int(A), syn.to_int(B)
    assert o.dkss_mul(a, b, par) == a * b


# ---- the C transcription ----------------------------------------------------

def test_c_oracle_r_mul_and_fft_match_python():
    import oracle_c as oc
    for cfg in TINY:
        par = o.Params(*cfg).check()
        r = o.compute_roots(par)
        rng = random.Random(9)
        q, m = par.pz, par.m
        x = [rng.randrange(q) for _ in range(m)]
        y = [q - 1] * m
        assert oc.r_mul(x, y, q) == o.r_mul(x, y, q)
        a = [[rng.randrange(q) for _ in range(m)] for _ in range(par.P2)]
        table = o.rho_table(r.rho, par)
        assert oc.fft(a, par.M, m, q, r.rho) == o.dkss_fft(a, table, par)


@pytest.mark.parametrize("cfg", TINY + [syn.workload_params("dkss_65536b")])
def test_c_oracle_exact_product(cfg):
    import oracle_c as oc
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    nw = syn.n_limbs(par.n_bits)
    rng = random.Random(10)
    N = par.n_bits
    for a, b in [(rng.getrandbits(N), rng.getrandbits(N)), ((1 << N) - 1, (1 << N) - 1), (0, 5)]:
        c, _ = oc.dkss_mul(syn.from_int(a, nw), syn.from_int(b, nw), par, r.rho)
        assert syn.to_int(c) == a * b


def test_c_oracle_stage_dumps_match_python():
    import oracle_c as oc
    par = o.Params(*syn.workload_params("dkss_65536b")).check()
    r = o.compute_roots(par)
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(0))
    st = {}
    o.dkss_mul(syn.to_int(A), syn.to_int(B), par, r, stages=st)
    _, d = oc.dkss_mul(A, B, par, r.rho, dumps=True)
    for key in ("a_hat", "b_hat", "c_hat", "c"):
        got = oc.from_words2(d[key].reshape(-1))
        assert got == [v for el in st[key] for v in el], key


@pytest.mark.slow
def test_c_oracle_2p24_bits_exact():
    import oracle_c as oc
    par = o.Params(*syn.workload_params("dkss_2p24b")).check()
    r = o.compute_roots(par)
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(1))
    c, _ = oc.dkss_mul(A, B, par, r.rho)
    assert syn.to_int(c) == syn.to_int(A) * syn.to_int(B)


@pytest.mark.parametrize("cfg", TINY)
def test_c_oracle_alpha_points_match_full_transform(cfg):
    """a_hat_{k mu} = sum_j a_j alpha^(k j) because rho^mu = alpha (Section 3.2.3)."""
    import oracle_c as oc
    par = o.Params(*cfg).check()
    rng = random.Random(11)
    a = rng.getrandbits(par.n_bits)
    table = o.rho_table(o.compute_roots(par).rho, par)
    full = o.dkss_fft(o.encode(a, par), table, par)
    limbs = syn.from_int(a, syn.n_limbs(par.n_bits))
    for k in range(2 * par.m):
        assert oc.fft_alpha_point(limbs, par, k) == full[k * par.mu]


# ---- cost model of the autotuner (float, outside the product path) ----------

def test_mlp_oracle_gradient_matches_finite_differences():
    import mlp_oracle as mo
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.3, mo.NPARAM)
    x = rng.normal(0, 1, (7, mo.F))
    t = rng.normal(0, 1, 7)
    g = mo.grad(p, x, t)
    h = 1e-6
    for i in rng.choice(mo.NPARAM, 60, replace=False).tolist() + [mo.NPARAM - 1]:
        e = np.zeros(mo.NPARAM)
        e[i] = h
        fd = (mo.loss(p + e, x, t) - mo.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_mlp_oracle_forward_closed_form():
    import mlp_oracle as mo
    # W1 = identity on the first F hidden units, W2 = identity, w3 = ones:
    # y = sum_i relu(x_i + b1_i) + b3 with b2 = 0
    p = np.zeros(mo.NPARAM)
    W1, b1, W2, b2, w3, _ = [a for a in mo.unpack(p)]
    o = 0
    for j in range(mo.F):
        p[o + j * mo.F + j] = 1.0
    o_b1 = mo.H * mo.F
    p[o_b1:o_b1 + mo.H] = 0.5
    o_w2 = o_b1 + mo.H
    for j in range(mo.H):
        p[o_w2 + j * mo.H + j] = 1.0
    o_w3 = o_w2 + mo.H * mo.H + mo.H
    p[o_w3:o_w3 + mo.H] = 1.0
    p[-1] = -2.0
    x = np.array([np.linspace(-1, 1, mo.F)])
    want = np.maximum(x[0] + 0.5, 0).sum() + 0.5 * (mo.H - mo.F) - 2.0
    assert abs(mo.forward(p, x)[0] - want) < 1e-12


def test_mlp_oracle_first_adam_step():
    import mlp_oracle as mo
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p, m1, m2 = mo.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 0.01, 1)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8))


# ---- Lucas-Lehmer system test (implementation chapter) ----------------------

def _is_prime_trial(n):
    if n < 2:
        return False
    f = 2
    while f * f <= n:
        if n % f == 0:
            return False
        f += 1
    return True


def test_lucas_lehmer_small_exponents_by_trial_division():
    """For odd prime p <= 31 the oracle's test says "prime" exactly when trial
    division finds no factor of 2^p - 1."""
    for p in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31):
        assert (o.lucas_lehmer(p) == 0) == _is_prime_trial((1 << p) - 1), p


def test_lucas_lehmer_composites_with_known_factors():
    """Composite Mersenne numbers (a factor divides 2^p - 1) leave a nonzero residue."""
    for p, f in ((37, 223), (41, 13367), (43, 431), (47, 2351), (53, 6361), (59, 179951), (67, 193707721),
                 (71, 228479), (73, 439), (79, 2687), (83, 167), (97, 11447)):
        assert ((1 << p) - 1) % f == 0, p
        assert o.lucas_lehmer(p) != 0, p


def test_lucas_lehmer_primes_by_fermat_tests():
    """2^p - 1 for p = 61, 89, 107, 127 passes Fermat tests to 12 bases and the
    oracle's test calls it prime; p = 521 and 607 are prime exponents too."""
    for p in (61, 89, 107, 127):
        n = (1 << p) - 1
        assert all(pow(b, n - 1, n) == 1 for b in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37))
        assert o.lucas_lehmer(p) == 0
    for p in (521, 607):
        n = (1 << p) - 1
        assert pow(3, n - 1, n) == 1
        assert o.lucas_lehmer(p) == 0
