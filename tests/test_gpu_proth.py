"""Products over Proth rings (z = 1, p = h 2^n + 1, dkss_plan_proth) against
the oracle (needs a GPU).

The oracle computes with any modulus below 2^126, so the same comparisons as
for the configured rings apply: product words and the forward transform
a_hat_i = a(rho^i), element by element, on every form; the default form uses
the sparse-modulus Montgomery reduction there (plan info "sparse").
"""
import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn
from gpu_helpers import to_dev, to_host, residues

import bench

pytestmark = pytest.mark.gpu

# (n_bits, M, m, u): every m, one- to three-deep recursion, ragged N, u not dividing 64
SHAPES = [
    (2000, 32, 16, 8),
    (26600, 128, 32, 13),
    (131072, 256, 64, 16),
    (262144, 2048, 16, 16),
    (786432, 2048, 32, 24),
    (1 << 22, 1 << 12, 64, 32),
    (1 << 24, 1 << 15, 32, 32),
]


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


def proth_cfg(dk, shape):
    h, n = dk.proth_ring(*shape)
    return h, n, (h << n) + 1


@pytest.mark.parametrize("flags", [0, 128, 16, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_proth_ring_matches_oracle(dk, oc, shape, flags):
    if flags == 2 and shape[2] < 32:
        pytest.skip("the INT8 form needs m >= 32")
    h, n, p = proth_cfg(dk, shape)
    par = o.Params(*shape, p, 1).check()
    roots = o.compute_roots(par)
    A, B = syn.operand_pair(shape[0], 4242, product=SHAPES.index(shape))
    with dk.Plan.proth(*shape, h, n, flags=flags) as plan:
        info = plan.info()
        assert info["p"] == p and info["z"] == 1 and info["sparse"] == 1
        c = plan.mul(to_dev(A), to_dev(B))
        fwd = plan.forward(to_dev(A))
        sq = plan.mul(to_dev(A), to_dev(A))
        plan.sync_status()
        got, fwd_host, sq_host = to_host(c), fwd.cpu().numpy(), to_host(sq)
    want, dumps = oc.dkss_mul(A, B, par, roots.rho, dumps=("a_hat",))
    assert np.array_equal(got, want)
    assert residues(fwd_host) == residues(dumps["a_hat"])
    assert syn.to_int(sq_host) == syn.to_int(A) ** 2


def test_proth_ring_special_operands(dk, oc):
    shape = SHAPES[4]
    h, n, p = proth_cfg(dk, shape)
    par = o.Params(*shape, p, 1).check()
    roots = o.compute_roots(par)
    ones = syn.special_operand(shape[0], "ones")
    with dk.Plan.proth(*shape, h, n) as plan:
        for kind in ("zero", "one", "ones", "top"):
            A = syn.special_operand(shape[0], kind)
            got = to_host(plan.mul(to_dev(A), to_dev(ones)))
            plan.sync_status()
            want, _ = oc.dkss_mul(A, ones, par, roots.rho)
            assert np.array_equal(got, want), kind


@pytest.mark.parametrize("shape", [(1 << 28, 1 << 18, 64, 32), (1 << 32, 1 << 22, 64, 32)])
def test_proth_ring_large(dk, oc, shape):
    """The 2^28- and 2^32-bit shapes with their Proth rings: product by low
    word, length and residues mod three 31-bit primes; transform at sampled
    frequencies k mu (rho^(k mu) = alpha^k) from the oracle."""
    h, n, p = proth_cfg(dk, shape)
    par = o.Params(*shape, p, 1).check()
    A, B = syn.operand_pair(shape[0], 777)
    with dk.Plan.proth(*shape, h, n) as plan:
        da, db = to_dev(A), to_dev(B)
        got = to_host(plan.mul(da, db))
        plan.sync_status()
        fwd = plan.forward(da)
        ks = list(range(0, 2 * par.m, 16))
        sampled = fwd[[k * par.mu for k in ks]].cpu().numpy()
        del fwd
    assert got.size == 2 * A.size
    assert bench.check_product(got, A, B)      # low word, residues mod three 31-bit primes
    for row, k in zip(sampled, ks):
        assert residues(row) == oc.fft_alpha_point(A, par, k)
