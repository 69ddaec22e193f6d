"""CPU-only checks of the C-ABI library: it loads, exports every symbol that
include/dkss.h declares, and its host plan math (Section 3.2.2-3.2.3) agrees
with the oracle.  No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dk():
    import paper_1503_04955_gb300 as pkg
    pkg.buildlib.build()
    pkg.load()
    return pkg


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dkss.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dkss_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(dk):
    lib = ctypes.CDLL(dk.lib_path())
    names = declared_symbols()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(dk.EXPORTS)


def test_status_strings(dk):
    lib = dk.load()
    for code in range(8):
        assert lib.dkss_status_str(code)


GPU_SMALL = [
    (2000, 32, 16, 8, 193, 4),
    (26600, 128, 32, 13, 257, 5),
    (131072, 256, 64, 16, 7681, 4),
    (262144, 2048, 16, 16, 12289, 4),
    (786432, 2048, 32, 24, 65537, 5),
    (1 << 22, 1 << 12, 64, 32, 7340033, 4),
    (1 << 24, 1 << 14, 64, 32, 998244353, 4),
]


@pytest.mark.parametrize("cfg", [syn.workload_params(k) for k in syn.WORKLOADS] + GPU_SMALL)
def test_plan_roots_match_oracle(dk, cfg):
    rho, consts = dk.plan_rho(*cfg)
    par = o.Params(*cfg).check()
    r = o.compute_roots(par)
    assert rho == r.rho
    assert consts["zeta"] == r.zeta and consts["omega"] == r.omega and consts["gamma"] == r.gamma
    assert consts["pz"] == par.pz and consts["P2"] == par.P2 and consts["mu"] == par.mu
    # limbs: one spare bit above p^z, and room for m-term sums and their REDC
    L = consts["L"]
    assert par.pz < 1 << (32 * L - 1)
    assert par.m * par.pz ** 2 + (1 << (32 * L)) * par.pz < 1 << (64 * L)
    # 26-bit product limbs: m p^z < 2^(26 LR), so one subtraction ends each REDC,
    # and a 64-bit column holds m*LR limb products of 52 bits
    LR = consts["LR"]
    assert par.m * par.pz < 1 << (26 * LR) and par.m * LR * (1 << 52) < 1 << 63


@pytest.mark.parametrize("bad", [
    (1 << 16, 512, 16, 16, 12287, 4),     # p not prime
    (1 << 16, 512, 16, 16, 13, 4),        # 2M does not divide p-1
    (1 << 16, 512, 16, 16, 12289, 3),     # p^z below the coefficient bound
    (1 << 16, 500, 16, 16, 12289, 4),     # M not a power of two
    (1 << 16, 8, 16, 16, 12289, 4),       # M < m
    (1 << 20, 512, 16, 16, 12289, 4),     # M (m/2) u < N
    (1 << 16, 512, 16, 0, 12289, 4),      # u = 0
    (1 << 16, 512, 16, 33, 12289, 4),     # u above 32
    (0, 512, 16, 16, 12289, 4),           # empty operands
    (1 << 16, 512, 16, 16, 12289, 0),     # z = 0
    (1 << 16, 512, 1, 16, 12289, 4),      # m < 2
])
def test_plan_rejects_invalid_parameters(dk, bad):
    with pytest.raises(dk.DkssError) as e:
        dk.plan_rho(*bad)
    assert e.value.code == 2   # DKSS_EPARAM


def test_plan_unsupported_m(dk):
    # m = 8 is a valid DKSS ring but this build has kernels for m in {16, 32, 64}
    with pytest.raises(dk.DkssError) as e:
        dk.plan_rho(1 << 12, 512, 8, 4, 12289, 3)
    assert e.value.code in (2, 4)


def test_int8_form_needs_m_32(dk):
    # the INT8 tensor-core form gives each element a warp: m = 16 is rejected
    # before any device work
    h = ctypes.c_void_p()
    rc = dk.load().dkss_plan(ctypes.byref(h), 1 << 16, 512, 16, 16, 12289, 4, 2)
    assert rc == 4 and not h.value


def test_rings_take_the_evaluation_map_form(dk):
    """Every workload ring and every tested small ring stays within the lazy
    transform's limits (else the plan falls back to the direct convolution),
    and those with m <= 32 within the limits of the inner levels in
    evaluation coordinates; the m = 16, p^z = 40961^3 ring is one whose
    componentwise products are prescaled."""
    for cfg in [syn.workload_params(k) for k in syn.WORKLOADS] + GPU_SMALL:
        _, consts = dk.plan_rho(*cfg)
        assert consts["rmul"] == 0, cfg
        assert consts["eval_ok"] == (1 if cfg[2] <= 32 else 0), cfg
        assert consts["eval_skip"] & 1, cfg
    _, consts = dk.plan_rho(4096, 32, 16, 16, 40961, 3)
    assert consts["rmul"] == 0 and consts["prescale"] == 1
    _, consts = dk.plan_rho(*syn.workload_params("dkss_2p24b"))
    assert consts["prescale"] == 0


def test_square_and_lucas_lehmer_argument_errors(dk):
    """dkss_sqr and dkss_ll_step reject bad arguments on the host, before any
    launch (DKSS_EINVAL = 1)."""
    lib = dk.load()
    buf = (ctypes.c_uint64 * 64)()
    base = ctypes.addressof(buf)
    assert lib.dkss_sqr(None, base, base + 256, None) == 1            # no plan
    assert lib.dkss_ll_step(None, base, 127, None) == 1               # no c
    assert lib.dkss_ll_step(base, None, 127, None) == 1               # no s
    for p in (0, 1, 2, 1 << 26):                                      # p out of range
        assert lib.dkss_ll_step(base, base + 256, p, None) == 1
    # s overlapping c: c holds 2 ceil(p/64) words, s ceil(p/64)
    assert lib.dkss_ll_step(base, base + 8, 127, None) == 1
    assert lib.dkss_ll_step(base + 16, base + 8, 127, None) == 1


def test_fault_injection_wrong_rho_is_rejected(dk):
    """A perturbed rho fails the plan's checks rho^(2M/2m) = alpha and rho^M = -1
    (Section 3.2.3): DKSS_EPARAM; without the fault the same plan is fine."""
    lib = dk.load()
    cfg = syn.workload_params("dkss_65536b")
    old = lib.dkss_fault_inject(1)
    try:
        with pytest.raises(dk.DkssError) as e:
            dk.plan_rho(*cfg)
        assert e.value.code == 2
        plan = ctypes.c_void_p()
        assert lib.dkss_plan(ctypes.byref(plan), *cfg, 0) == 2 and plan.value is None
    finally:
        lib.dkss_fault_inject(old)
    rho, consts = dk.plan_rho(*cfg)
    assert rho == o.compute_roots(o.Params(*cfg).check()).rho


def test_fault_injection_host_allocation(dk):
    """dkss_plan's host allocation fails: DKSS_ENOMEM, *plan set to NULL."""
    lib = dk.load()
    cfg = syn.workload_params("dkss_65536b")
    plan = ctypes.c_void_p(1)
    old = lib.dkss_fault_inject(2)
    try:
        assert lib.dkss_plan(ctypes.byref(plan), *cfg, 0) == 3
        assert plan.value is None
    finally:
        lib.dkss_fault_inject(old)
    assert lib.dkss_fault_inject(0) == 0


@pytest.mark.parametrize("n_bits", [4096, 65536, 100000, 1 << 20, 3 << 20, 1 << 24, 1 << 28, 1 << 32])
def test_plan_choose_follows_the_thesis_rule(dk, n_bits):
    """dkss_plan_choose with the rule flag (host only): among the valid sets
    (dkss_plan_candidates), u is the largest, M m the smallest, M/m the
    closest to N / log2(N)^3, and p^z the smallest of that kernel shape
    (Section 4.1) -- checked by enumeration; the shape equals the Python
    restatement's."""
    import math
    from paper_1503_04955_gb300 import autotune
    M, m, u, p, z = dk.plan_choose(n_bits, dk.TUNE_RULE)
    cands = dk.plan_candidates(n_bits)
    assert any((c["M"], c["m"], c["u"], c["p"], c["z"]) == (M, m, u, p, z) for c in cands)
    umax = max(c["u"] for c in cands)
    assert u == umax
    best_mm = min(c["M"] * c["m"] for c in cands if c["u"] == umax)
    assert M * m == best_mm
    target = math.log2(n_bits / math.log2(n_bits) ** 3)
    dist = abs(math.log2(M / m) - target)
    assert all(abs(math.log2(c["M"] / c["m"]) - target) >= dist - 1e-12
               for c in cands if c["u"] == umax and c["M"] * c["m"] == best_mm)
    # the same kernel shape as the Python restatement (which keeps one ring per shape)
    r = autotune.rule_choice(n_bits, autotune.candidates(n_bits))
    mine = [c for c in cands if (c["M"], c["m"], c["u"], c["p"], c["z"]) == (M, m, u, p, z)][0]
    assert tuple(r[k] for k in autotune.KEY) == tuple(mine[k] for k in autotune.KEY)
    # and p^z just above the bound: the smallest p^z of that shape
    same = [c for c in cands if all(c[k] == mine[k] for k in autotune.KEY)]
    assert p ** z == min(c["p"] ** c["z"] for c in same)
    o.Params(n_bits, M, m, u, p, z).check()


def test_plan_choose_rule_for_int8_needs_m32(dk):
    for n_bits in (65536, 1 << 24):
        M, m, u, p, z = dk.plan_choose(n_bits, dk.TUNE_RULE | dk.FORM_INT8TC)
        assert m >= 32
    with pytest.raises(dk.DkssError):
        dk.plan_choose(0, dk.TUNE_RULE)


# Proth rings (z = 1, p = h 2^n + 1): the thesis's primes (Section 4.1)
PROTH_SHAPES = [(1 << 16, 512, 16, 16), (1 << 20, 1 << 13, 16, 16), (1 << 24, 1 << 15, 32, 32),
                (1 << 28, 1 << 18, 64, 32), (1 << 32, 1 << 22, 64, 32)]


def test_proth_primality_matches_sympy(dk):
    """dkss_plan_proth_rho rejects exactly the composite h 2^n + 1 (Proth's
    theorem on the host) -- compared with sympy on every odd h below 200 for
    a few n."""
    sympy = pytest.importorskip("sympy")
    M, m, u = 32, 16, 8
    for n in (30, 61, 64, 78, 100):
        for h in range(1, 200, 2):
            p = (h << n) + 1
            try:
                dk.plan_proth_rho(2000, M, m, u, h, n)
                ok = True
            except dk.DkssError as e:
                assert e.code == 2
                ok = False
            assert ok == sympy.isprime(p), (h, n)


@pytest.mark.parametrize("shape", PROTH_SHAPES)
def test_proth_ring_is_the_smallest_valid_prime(dk, shape):
    """dkss_proth_ring: p = h 2^n + 1 prime, 2M | p - 1, above the coefficient
    bound, m p < 2^(26 LR - 2) with the fewest limbs, and no smaller odd h at
    that n gives such a prime (p just above the bound, Section 4.1)."""
    n_bits, M, m, u = shape
    h, n = dk.proth_ring(*shape)
    p = (h << n) + 1
    bound = M * (m // 2) * ((1 << u) - 1) ** 2
    assert o.lucas_is_prime(p) and (p - 1) % (2 * M) == 0 and p > bound
    lr = (n + 25) // 26 + (1 if n % 26 == 0 else 0)
    assert n == max(26 * (lr - 1), (2 * M).bit_length() - 1)
    assert m * p < 1 << (26 * lr - 2)
    for hh in range(max(1, (bound >> n) + 1) | 1, h, 2):
        assert not o.lucas_is_prime((hh << n) + 1) or ((hh << n) + 1) <= bound
    rho, consts = dk.plan_proth_rho(n_bits, M, m, u, h, n)
    assert consts["sparse"] == 1 and consts["LR"] == lr and consts["p"] == p and consts["z"] == 1
    par = o.Params(n_bits, M, m, u, p, 1).check()
    roots = o.compute_roots(par)
    assert rho == roots.rho
    assert (consts["zeta"], consts["omega"], consts["gamma"]) == (roots.zeta, roots.omega, roots.gamma)


def test_proth_plan_argument_checks(dk):
    with pytest.raises(dk.DkssError):
        dk.plan_proth_rho(1 << 24, 1 << 15, 32, 32, 4, 78)      # h even
    with pytest.raises(dk.DkssError):
        dk.plan_proth_rho(1 << 24, 1 << 15, 32, 32, 3, 10)      # 2M does not divide 2^n
    with pytest.raises(dk.DkssError):
        dk.plan_proth_rho(1 << 24, 1 << 15, 32, 32, 1, 20)      # below the coefficient bound


def test_decode_static_size_limit_on_host(dk):
    """The allocation-free decode refuses products beyond its static scratch
    (ceil(N/64) <= 2^27, N <= 2^33) before any device work: N = 2^33 + 64 gives
    DKSS_EUNSUPPORTED, N = 2^33 passes the size check and then needs a device
    (DKSS_ECUDA on this host).  Host only: with a GPU present the accepted
    call would launch kernels on the placeholder pointers, so it is skipped."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("host-only check")
    except ImportError:
        pass
    lib = dk.load()
    c, out = 4096, 8192          # placeholders, never dereferenced on this host
    assert lib.dkss_decode_static(c, (1 << 33) + 64, 1 << 28, 64, 32, 4, out, None) == 4
    assert lib.dkss_decode_static(c, 1 << 33, 1 << 28, 64, 32, 4, out, None) == 5
