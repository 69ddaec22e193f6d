"""Squares (dkss_sqr, and dkss_mul with a == b) and the thesis's system test,
the Lucas-Lehmer test of Mersenne numbers, on the GPU (needs a GPU).

A square runs the forward transform once; its words must equal the exact
square and the oracle's product a*a.  The Lucas-Lehmer test chains p - 2
squares with dkss_ll_step; its last residue must be 0 exactly for the Mersenne
prime exponents and equal the oracle's residue for the others.
"""
import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn
from gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

SQUARE_CONFIGS = [
    (2000, 32, 16, 8, 193, 4),              # m=16, L=2, one radix-2m level
    (4096, 32, 16, 16, 40961, 3),           # LR=2: the NTT form prescales the componentwise products
    (786432, 2048, 32, 24, 65537, 5),       # m=32, L=3, fused levels
    (1 << 22, 1 << 12, 64, 32, 7340033, 4),  # m=64, split levels
]
FORMS = [0, 128, 16]


@pytest.fixture(scope="module")
def dk():
    import torch
    import paper_1503_04955_gb300 as pkg
    assert torch.cuda.is_available()
    pkg.buildlib.build()
    return pkg


@pytest.fixture(scope="module")
def oc():
    import oracle_c
    oracle_c.build()
    return oracle_c


@pytest.mark.parametrize("flags", FORMS)
@pytest.mark.parametrize("cfg", SQUARE_CONFIGS)
def test_square_matches_oracle(dk, oc, cfg, flags):
    par = o.Params(*cfg).check()
    A, _ = syn.operand_pair(cfg[0], 4321, product=SQUARE_CONFIGS.index(cfg))
    want, _ = oc.dkss_mul(A, A, par, o.compute_roots(par).rho)
    assert syn.to_int(want) == syn.to_int(A) ** 2
    with dk.Plan(*cfg, flags=flags) as plan:
        a = to_dev(A)
        sq = to_host(plan.sqr(a))                  # dkss_sqr
        same = to_host(plan.mul(a, a))             # dkss_mul, a == b
        two = to_host(plan.mul(a, to_dev(A)))      # two operands with equal words
        plan.sync_status()
    assert np.array_equal(sq, want)
    assert np.array_equal(same, want)
    assert np.array_equal(two, want)


@pytest.mark.parametrize("cfg", SQUARE_CONFIGS[2:])
def test_square_int8_form(dk, oc, cfg):
    par = o.Params(*cfg).check()
    A, _ = syn.operand_pair(cfg[0], 4322, product=SQUARE_CONFIGS.index(cfg))
    want, _ = oc.dkss_mul(A, A, par, o.compute_roots(par).rho)
    with dk.Plan(*cfg, flags=dk.binding.FORM_INT8TC) as plan:
        got = to_host(plan.sqr(to_dev(A)))
        plan.sync_status()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("kind", ["ones", "top", "one", "zero"])
def test_square_special_operands(dk, oc, kind):
    cfg = SQUARE_CONFIGS[2]
    par = o.Params(*cfg).check()
    A = syn.special_operand(cfg[0], kind)
    want, _ = oc.dkss_mul(A, A, par, o.compute_roots(par).rho)
    with dk.Plan(*cfg) as plan:
        got = to_host(plan.sqr(to_dev(A)))
        plan.sync_status()
    assert np.array_equal(got, want)


def test_square_2p24_bits(dk, oc):
    cfg = syn.workload_params("dkss_2p24b")
    par = o.Params(*cfg).check()
    A, _ = syn.operand_pair(cfg[0], syn.config_seed(1))
    want, _ = oc.dkss_mul(A, A, par, o.compute_roots(par).rho)
    with dk.Plan(*cfg) as plan:
        got = to_host(plan.sqr(to_dev(A)))
        plan.sync_status()
    assert np.array_equal(got, want)


def lucas_lehmer_gpu(dk, p):
    """Last Lucas-Lehmer residue of 2^p - 1 with the library's square and step."""
    import torch
    from paper_1503_04955_gb300 import autotune
    w = (p + 63) // 64
    n_bits = 64 * w
    c = autotune.rule_choice(n_bits, autotune.candidates(n_bits))
    with dk.Plan(n_bits, c["M"], c["m"], c["u"], c["p"], c["z"]) as plan:
        s = torch.zeros(w, dtype=torch.int64, device="cuda")
        s[0] = 4
        sq = torch.empty(2 * w, dtype=torch.int64, device="cuda")
        for _ in range(p - 2):
            plan.sqr(s, sq)
            dk.ll_step(sq, s, p)
        plan.sync_status()
        return syn.to_int(to_host(s))


@pytest.mark.parametrize("p", [521, 607, 1279, 2203, 2281, 3217, 4253, 4423])
def test_lucas_lehmer_mersenne_primes(dk, p):
    assert lucas_lehmer_gpu(dk, p) == 0


@pytest.mark.parametrize("p", [523, 1277, 2207])
def test_lucas_lehmer_composite_residues(dk, p):
    got = lucas_lehmer_gpu(dk, p)
    assert got != 0
    assert got == o.lucas_lehmer(p)


def test_ll_step_rejects_overlap_and_bad_p(dk):
    import torch
    c = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(dk.DkssError):
        dk.ll_step(c, c[:2], 100)
    with pytest.raises(ValueError):
        dk.ll_step(c, torch.zeros(2, dtype=torch.int64, device="cuda"), 200)
