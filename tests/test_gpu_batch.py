"""Batched products of uneven sizes: one persistent kernel for all jobs
(needs a GPU).  Every product is checked against the exact integer product,
and against dkss_mul with the job's size-class parameters."""
import random

import numpy as np
import pytest

import dkss_synth as syn
from gpu_helpers import to_dev, to_host, random_primes61, mod_int

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    import torch
    import paper_1503_04955_gb300 as pkg
    assert torch.cuda.is_available()
    pkg.buildlib.build()
    return pkg


def make_jobs(lengths, seed):
    import torch
    ops = [syn.operand_pair(n, seed, product=j) for j, n in enumerate(lengths)]
    words = [syn.n_limbs(n) for n in lengths]
    total = sum(words)
    a_all = torch.zeros(total, dtype=torch.int64, device="cuda")
    b_all = torch.zeros(total, dtype=torch.int64, device="cuda")
    o_all = torch.zeros(2 * total, dtype=torch.int64, device="cuda")
    a_list, b_list, o_list = [], [], []
    off = 0
    for (A, B), w in zip(ops, words):
        a_all[off:off + w] = to_dev(A)
        b_all[off:off + w] = to_dev(B)
        a_list.append(a_all[off:off + w])
        b_list.append(b_all[off:off + w])
        o_list.append(o_all[2 * off:2 * off + 2 * w])
        off += w
    return ops, a_list, b_list, o_list


SMALL_LENGTHS = [64, 100, 4095, 4096, 4097, 12345, 65536, 70000, 131072, 1000] + \
    [int(x) for x in syn.log_uniform_lengths(20, 77, lo_exp=12, hi_exp=17)]


@pytest.mark.parametrize("flags", [0, 32, 64])      # autotuned + graph, rule, no graph
def test_small_uneven_batch(dk, flags):
    import torch
    ops, a, b, o = make_jobs(SMALL_LENGTHS, 31)
    with dk.Batch(SMALL_LENGTHS, flags=flags) as bt:
        for rep in range(2):
            bt.run(a, b, o)
            torch.cuda.synchronize()
            for (A, B), out in zip(ops, o):
                assert syn.to_int(to_host(out)) == syn.to_int(A) * syn.to_int(B)
            for t in o:
                t.zero_()
        # same products through single plans with each job's class parameters
        for j in (0, 5, 9, len(SMALL_LENGTHS) - 1):
            prm = bt.job_params(j)
            assert prm["graph"] == (0 if flags & 64 else prm["graph"])
            with dk.Plan(SMALL_LENGTHS[j], prm["M"], prm["m"], prm["u"], prm["p"], prm["z"]) as pl:
                A, B = ops[j]
                c = to_host(pl.mul(to_dev(A), to_dev(B)))
                assert syn.to_int(c) == syn.to_int(A) * syn.to_int(B)


def test_mul_batch_convenience_reuses_plan(dk):
    import torch
    lengths = SMALL_LENGTHS[:8]
    ops, a, b, o = make_jobs(lengths, 5)
    for rep in range(2):
        dk.mul_batch(a, b, o, lengths)
        torch.cuda.synchronize()
        for (A, B), out in zip(ops, o):
            assert syn.to_int(to_host(out)) == syn.to_int(A) * syn.to_int(B)


def test_4096_products_log_uniform_2p14_2p20(dk):
    """The batched workload: 4096 products, lengths 2^x, x uniform in [14, 20],
    rounded to 64-bit limbs.  All products: low word and residues mod random
    61-bit primes; 16 sampled products: exact."""
    import torch
    w = syn.BATCH_WORKLOAD
    lengths = [int(n) for n in syn.log_uniform_lengths(w["count"], syn.config_seed(w["index"]),
                                                       w["lo_exp"], w["hi_exp"])]
    ops, a, b, o = make_jobs(lengths, syn.config_seed(w["index"]))
    with dk.Batch(lengths) as bt:
        bt.run(a, b, o)
        torch.cuda.synchronize()
        got = [to_host(t) for t in o]
    qs = random_primes61(2, seed=11)
    for (A, B), g in zip(ops, got):
        assert int(g[0]) == (int(A[0]) * int(B[0])) % (1 << 64)
        for q in qs:
            assert mod_int(g, q) == mod_int(A, q) * mod_int(B, q) % q
    for j in random.Random(3).sample(range(len(lengths)), 16):
        A, B = ops[j]
        assert syn.to_int(got[j]) == syn.to_int(A) * syn.to_int(B)
