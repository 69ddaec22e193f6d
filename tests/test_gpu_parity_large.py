"""Bit-exact parity at the two largest workloads (needs a GPU).

2^28 bits (M = 2^18, m = 64, u = 32, p = 7340033, z = 4): the C oracle runs
inside the test (OpenMP over its independent loops, about ten seconds on the
host cores) and the GPU's product words and forward transform
a_hat_i = a(rho^i), i < 2M, natural order, are compared with it element by
element, in the default form, the direct convolution and the INT8
tensor-core form.

2^32 bits (M = 2^22, m = 64, u = 32, p = 998244353, z = 4): the oracle needs
about half an hour and 32 GiB, so tests/golden/make_large_digests.py ran it
once and stored SHA-256 digests of its product words and of its a_hat (the
whole array and 16 equal slices); the GPU's full outputs are hashed the same
way and must match every digest, in the default form (p-adic digits), with
Montgomery products, the direct and the INT8 form.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn
from gpu_helpers import to_dev, to_host

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_large_digests as golden  # noqa: E402

pytestmark = pytest.mark.gpu

FORM_DEFAULT, FORM_DIRECT, FORM_INT8, FORM_MONT = 0, 16, 2, 512


@pytest.fixture(scope="module")
def dk():
    import torch
    import paper_1503_04955_gb300 as pkg
    assert torch.cuda.is_available()
    pkg.buildlib.build()
    return pkg


@pytest.fixture(scope="module")
def c4_oracle():
    """Product words and a_hat of the 2^28-bit workload from the C oracle,
    checked against the stored digests (the oracle gives the same result on
    this host as where the digests were written)."""
    import oracle_c
    oracle_c.build()
    name = "dkss_2p28b"
    cfg = syn.workload_params(name)
    par = o.Params(*cfg).check()
    rho = o.compute_roots(par).rho
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(syn.WORKLOADS[name]["index"]))
    oracle_c.set_threads(os.cpu_count() or 1)
    c, d = oracle_c.dkss_mul(A, B, par, rho, dumps=("a_hat",))
    want = golden.read_golden(name)
    assert golden.digests(c)[0] == want["product"][1]
    assert golden.digests(d["a_hat"])[0] == want["a_hat"][1]
    return cfg, A, B, c, d["a_hat"].reshape(-1)


def first_mismatch(got, want):
    bad = np.flatnonzero(got != want)
    return None if bad.size == 0 else int(bad[0])


@pytest.mark.parametrize("flags", [FORM_DEFAULT, FORM_MONT, FORM_DIRECT, FORM_INT8])
def test_2p28_bits_exact(dk, c4_oracle, flags):
    cfg, A, B, c_want, ahat_want = c4_oracle
    with dk.Plan(*cfg, flags=flags) as plan:
        da, db = to_dev(A), to_dev(B)
        c = to_host(plan.mul(da, db))
        plan.sync_status()
        fwd = plan.forward(da)
        ahat = fwd.cpu().numpy().view(np.uint64).reshape(-1)
        del fwd
    assert c.size == c_want.size
    assert first_mismatch(c, c_want) is None, "product word %s differs" % first_mismatch(c, c_want)
    assert ahat.size == ahat_want.size
    assert first_mismatch(ahat, ahat_want) is None, "a_hat word %s differs" % first_mismatch(ahat, ahat_want)


def device_digests(t, chunks=golden.CHUNKS):
    """Digests of a device int64 tensor as make_large_digests computes them
    (little-endian bytes of the 64-bit words), copied to the host slice by slice."""
    flat = t.reshape(-1)
    assert flat.numel() % chunks == 0
    step = flat.numel() // chunks
    whole = hashlib.sha256()
    parts = []
    for k in range(chunks):
        host = np.ascontiguousarray(flat[k * step:(k + 1) * step].cpu().numpy().view("<u8"))
        b = memoryview(host).cast("B")
        whole.update(b)
        parts.append(hashlib.sha256(b).hexdigest())
    return whole.hexdigest(), parts


def check_digests(got, want, what):
    words, whole, parts = want
    bad = [k for k, (g, w) in enumerate(zip(got[1], parts)) if g != w]
    assert not bad, "%s: slices %s of %d differ from the oracle's" % (what, bad, len(parts))
    assert got[0] == whole


@pytest.mark.parametrize("flags", [FORM_DEFAULT, FORM_MONT, FORM_DIRECT, FORM_INT8])
def test_2p32_bits_exact(dk, flags):
    name = "dkss_2p32b"
    want = golden.read_golden(name)
    cfg = syn.workload_params(name)
    assert [int(x) for x in want["params"]] == list(cfg)
    A, B = syn.operand_pair(cfg[0], syn.config_seed(syn.WORKLOADS[name]["index"]))
    with dk.Plan(*cfg, flags=flags) as plan:
        da, db = to_dev(A), to_dev(B)
        c = plan.mul(da, db)
        plan.sync_status()
        assert c.numel() == want["product"][0]
        check_digests(device_digests(c), want["product"], "product")
        del c
        fwd = plan.forward(da)
        plan.sync_status()
        assert fwd.numel() == want["a_hat"][0]
        check_digests(device_digests(fwd), want["a_hat"], "a_hat")
        del fwd
