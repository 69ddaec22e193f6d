"""Batched products of uneven sizes: one persistent kernel for all jobs
(needs a GPU).  Every product is checked against the exact integer product,
and against dkss_mul with the job's size-class parameters (each class has its
own ring: configured primes or a Proth prime)."""
import random

import numpy as np
import pytest

import dkss_synth as syn
from gpu_helpers import to_dev, to_host

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


# autotuned + graph, rule, no graph, Proth rings, configured rings
@pytest.mark.parametrize("flags", [0, 32, 64, 128, 256])
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
        classes = {}
        for j in range(len(SMALL_LENGTHS)):
            prm = bt.job_params(j)
            classes.setdefault(prm["class_bits"], prm)
            assert prm["graph"] == (0 if flags & 64 else prm["graph"])
            assert prm["proth"] == (1 if flags & 128 else 0 if flags & (32 | 256) else prm["proth"])
        # every class has a valid ring of its own; the same products through single plans
        for prm in classes.values():
            assert (prm["p"] - 1) % (2 * prm["M"]) == 0
        for j in (0, 5, 9, len(SMALL_LENGTHS) - 1):
            with bt.class_plan(j) as pl:
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
    rounded to 64-bit limbs; every product compared with the exact integer
    product."""
    import torch
    w = syn.BATCH_WORKLOAD
    lengths = [int(n) for n in syn.log_uniform_lengths(w["count"], syn.config_seed(w["index"]),
                                                       w["lo_exp"], w["hi_exp"])]
    ops, a, b, o = make_jobs(lengths, syn.config_seed(w["index"]))
    with dk.Batch(lengths) as bt:
        bt.run(a, b, o)
        torch.cuda.synchronize()
        got = [to_host(t) for t in o]
        rings = {bt.job_params(j)["p"] for j in range(len(lengths))}
    assert len(rings) >= 1
    bad = [j for j, ((A, B), g) in enumerate(zip(ops, got)) if syn.to_int(g) != syn.to_int(A) * syn.to_int(B)]
    assert not bad, "products %s differ from the exact products" % bad[:10]
