"""The stored oracle results of the large workloads are pinned (CPU).

tests/golden/make_large_digests.py ran the C oracle once on the 2^28- and
2^32-bit workloads and stored digests of its product and forward transform,
with the product's residues mod four random 61-bit primes.  Here those
residues are checked against (a mod q)(b mod q) mod q from the seeded
operands: a product that is wrong anywhere fails them (except with
probability about 2^-240), so the stored digests describe the exact product.
"""
import os
import sys

import pytest

import dkss_synth as syn

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_large_digests as golden  # noqa: E402


@pytest.mark.parametrize("name", ["dkss_2p28b", "dkss_2p32b"])
def test_stored_product_residues(name):
    want = golden.read_golden(name)
    cfg = syn.workload_params(name)
    assert [int(x) for x in want["params"]] == list(cfg)
    assert want["product"][0] == 2 * syn.n_limbs(cfg[0])
    assert want["a_hat"][0] == 2 * cfg[1] * cfg[2] * 2
    assert len(want["product"][2]) == golden.CHUNKS and len(want["a_hat"][2]) == golden.CHUNKS
    A, B = syn.operand_pair(cfg[0], syn.config_seed(syn.WORKLOADS[name]["index"]))
    ia, ib = syn.to_int(A), syn.to_int(B)
    res = want["residues"]
    assert [q for q, _ in res] == golden.random_primes61(4, golden.RESIDUE_SEED)
    for q, r in res:
        assert r == (ia % q) * (ib % q) % q


def test_random_primes61_are_prime():
    sympy = pytest.importorskip("sympy")
    for q in golden.random_primes61(4, golden.RESIDUE_SEED):
        assert (1 << 60) <= q < (1 << 61) and sympy.isprime(q)
