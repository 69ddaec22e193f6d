"""dkss_decode_static, the entry point that allocates nothing (needs a GPU).

Callers that cannot allocate device memory when they call -- a latency-bound
loop whose device memory is fixed before it starts, or code inside a framework
that owns the device's memory pool -- decode a product polynomial with scratch
held in a file-scope device array.  Its output must equal what dkss_mul produces for the same product, on
two calls in a row (the scratch keeps the previous call's contents).  The file
sorts last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn
from gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def product_polynomial_words(A, B, par, L):
    """The product polynomial from the C oracle, as 2M x m residues of L 32-bit words."""
    import oracle_c
    roots = o.compute_roots(par)
    _, dumps = oracle_c.dkss_mul(A, B, par, roots.rho, dumps=True)
    c64 = dumps["c"].reshape(-1, 2)                    # residues as two 64-bit words
    words = np.zeros((c64.shape[0], 4), dtype=np.uint32)
    words[:, 0] = (c64[:, 0] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    words[:, 1] = (c64[:, 0] >> np.uint64(32)).astype(np.uint32)
    words[:, 2] = (c64[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    words[:, 3] = (c64[:, 1] >> np.uint64(32)).astype(np.uint32)
    assert not words[:, L:].any()
    return np.ascontiguousarray(words[:, :L]).reshape(-1)


# u = 16 (L = 2), u = 13 (generic windows), u = 32 (L = 3 and L = 4)
NO_ALLOC_CFGS = [syn.workload_params("dkss_65536b"), (26600, 128, 32, 13, 257, 5), (65536, 256, 16, 32, 12289, 6),
                 (1 << 20, 2048, 32, 32, 65537, 6)]


@pytest.mark.parametrize("cfg", NO_ALLOC_CFGS)
def test_decode_static_matches_dkss_mul_twice(cfg):
    import torch
    import oracle_c
    import paper_1503_04955_gb300 as dk
    dk.buildlib.build()
    oracle_c.build()
    par = o.Params(*cfg).check()
    with dk.Plan(*cfg) as plan:
        L = plan.info()["L"]
        for k in range(2):                              # two calls in a row
            A, B = syn.operand_pair(par.n_bits, 4242, product=k)
            want = to_host(plan.mul(to_dev(A), to_dev(B)))
            c = torch.from_numpy(product_polynomial_words(A, B, par, L).view(np.int32)).cuda()
            got = dk.binding.decode_static(c, par.n_bits, par.M, par.m, par.u, L)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(got), want)
            assert syn.to_int(want) == syn.to_int(A) * syn.to_int(B)


def test_decode_static_rejects_oversize():
    import torch
    import paper_1503_04955_gb300 as dk
    c = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    lib = dk.load()
    n_bits = 1 << 34                                     # beyond DKSS_DECODE_STATIC_MAX_TILES
    rc = lib.dkss_decode_static(c.data_ptr(), n_bits, 1 << 29, 64, 32, 4, out.data_ptr(), None)
    assert rc == 4                                       # DKSS_EUNSUPPORTED, nothing launched


@pytest.mark.parametrize("cfg", [NO_ALLOC_CFGS[0], NO_ALLOC_CFGS[3]])
def test_decode_static_unaligned_input(cfg):
    """A product polynomial that starts one word past an aligned address is
    read with word loads instead of vector loads; the result is the same."""
    import torch
    import oracle_c
    import paper_1503_04955_gb300 as dk
    dk.buildlib.build()
    oracle_c.build()
    par = o.Params(*cfg).check()
    with dk.Plan(*cfg) as plan:
        L = plan.info()["L"]
        A, B = syn.operand_pair(par.n_bits, 4343)
        want = to_host(plan.mul(to_dev(A), to_dev(B)))
        words = product_polynomial_words(A, B, par, L).view(np.int32)
        buf = torch.zeros(words.size + 1, dtype=torch.int32, device="cuda")
        buf[1:] = torch.from_numpy(words).cuda()
        got = dk.binding.decode_static(buf[1:], par.n_bits, par.M, par.m, par.u, L)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(got), want)
