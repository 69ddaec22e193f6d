"""Parity of the CUDA DKSS_MUL path with the CPU oracle (needs a GPU).

Bit-exact: the product, and the forward transform a_hat_i = a(rho^i) in
natural order, element by element, on every size the oracle finishes in
seconds; at the 2^28- and 2^32-bit sizes, the product is checked through
properties that hold at any size (its low word, its length, and residues mod
random 61-bit primes) and the transform through sampled outputs the oracle
computes one by one (frequencies k*mu, where rho^(k mu) = alpha^k).
"""
import numpy as np
import pytest

import dkss_oracle as o
import dkss_synth as syn
from gpu_helpers import to_dev, to_host, residues, random_primes61, mod_int

pytestmark = pytest.mark.gpu

# (n_bits, M, m, u, p, z): every (m, L) kind and level structure, ragged N, u not dividing 64
SMALL = [
    (2000, 32, 16, 8, 193, 4),              # m=16, L=2, one radix-2m level, last level 2
    (26600, 128, 32, 13, 257, 5),           # m=32, L=2, u=13 straddles words, last level 4
    (131072, 256, 64, 16, 7681, 4),         # m=64, L=2, last level 4
    (262144, 2048, 16, 16, 12289, 4),       # m=16, two radix-2m levels, last level 4
    (786432, 2048, 32, 24, 65537, 5),       # m=32, L=3, last level 2m
    (1 << 22, 1 << 12, 64, 32, 7340033, 4),  # m=64, L=3 (three REDC subtractions), last level 2m
    (1 << 21, 1 << 14, 64, 16, 998244353, 4),  # m=64, L=4, two radix-2m levels, last level 2; p-adic, fast carries
    (1 << 21, 1 << 14, 64, 16, 754974721, 4),  # m=64, L=4, LR=5: p-adic with the generic carries
    (1 << 21, 1 << 14, 64, 16, 1073479681, 4),  # m=64, p just below 2^30: p-adic, fast carries at their limits
    (4096, 32, 16, 16, 40961, 3),           # m=16, L=2, LR=2: NTT form prescales the componentwise products
    (65536, 256, 16, 32, 12289, 6),         # m=16, L=3: padded shared-memory element stride
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


def check_product(dk, oc, cfg, A, B, with_oracle=True, with_forward=True, flags=0):
    par = o.Params(*cfg).check()
    roots = o.compute_roots(par)
    with dk.Plan(*cfg, flags=flags) as plan:
        # the default runs the evaluation-map form of the R-multiplications on every
        # ring tested here; levels in evaluation coordinates apply for m <= 32
        want = 2 if flags & 2 else 1 if flags & 16 else 3 if (flags & 128 and cfg[2] <= 32) else 0
        info = plan.info()
        assert info["rmul"] == want
        # m = 64 over p^4, p < 2^30: the NTT form computes in p-adic digits unless DKSS_ARITH_MONT,
        # where floor(2^32/p) is a power of two or the Montgomery products need five limbs
        nmu = (1 << 32) // cfg[4]
        fewer = (nmu & (nmu - 1)) == 0 or info["LR"] >= 5
        assert info["padic"] == int(want == 0 and not flags & 512 and cfg[2] == 64 and cfg[5] == 4
                                    and cfg[4] < 1 << 30 and fewer)
        c = plan.mul(to_dev(A), to_dev(B))
        fwd = plan.forward(to_dev(A)) if with_forward else None
        plan.sync_status()
        got = to_host(c)
        fwd_host = fwd.cpu().numpy() if with_forward else None
    assert syn.to_int(got) == syn.to_int(A) * syn.to_int(B)
    if with_oracle:
        want, dumps = oc.dkss_mul(A, B, par, roots.rho, dumps=with_forward)
        assert np.array_equal(got, want)
        if with_forward:
            assert residues(fwd_host) == residues(dumps["a_hat"])


# alpha-shift inner DFTs with R-multiplications through the evaluation map of
# R (default: p-adic digits for m = 64 over p^4), the same with 26-bit-limb
# Montgomery products (DKSS_ARITH_MONT), inner levels in evaluation
# coordinates (DKSS_LEVELS_EVAL), and the direct negacyclic convolution
# (DKSS_RMUL_DIRECT)
FORMS = [0, 512, 128, 16]


@pytest.mark.parametrize("flags", FORMS)
@pytest.mark.parametrize("cfg", SMALL)
def test_small_configs_random(dk, oc, cfg, flags):
    A, B = syn.operand_pair(cfg[0], 1234, product=SMALL.index(cfg))
    check_product(dk, oc, cfg, A, B, flags=flags)


@pytest.mark.parametrize("flags", FORMS)
@pytest.mark.parametrize("kind", ["zero", "one", "ones", "top"])
@pytest.mark.parametrize("cfg", [SMALL[0], SMALL[4], SMALL[6], SMALL[7]])
def test_small_configs_special_operands(dk, oc, cfg, kind, flags):
    A = syn.special_operand(cfg[0], kind)
    B = syn.special_operand(cfg[0], "ones")
    check_product(dk, oc, cfg, A, B, with_forward=(kind == "ones"), flags=flags)


def test_65536_bits_full_parity(dk, oc):
    cfg = syn.workload_params("dkss_65536b")
    A, B = syn.operand_pair(cfg[0], syn.config_seed(0))
    check_product(dk, oc, cfg, A, B)


def test_65536_bits_all_ones_reaches_bound(dk, oc):
    cfg = syn.workload_params("dkss_65536b")
    A = syn.special_operand(cfg[0], "ones")
    check_product(dk, oc, cfg, A, A)


@pytest.mark.parametrize("flags", FORMS)
def test_2p24_bits_full_parity(dk, oc, flags):
    cfg = syn.workload_params("dkss_2p24b")
    A, B = syn.operand_pair(cfg[0], syn.config_seed(1))
    check_product(dk, oc, cfg, A, B, flags=flags)


def test_mul_host_matches_device_path(dk):
    cfg = syn.workload_params("dkss_65536b")
    A, B = syn.operand_pair(cfg[0], syn.config_seed(0), product=3)
    with dk.Plan(*cfg) as plan:
        got = plan.mul_host(A, B)
        again = plan.mul_host(B, A)
    want = syn.to_int(A) * syn.to_int(B)
    assert syn.to_int(got) == want and syn.to_int(again) == want


def test_repeated_calls_reuse_workspace(dk):
    cfg = SMALL[3]
    with dk.Plan(*cfg) as plan:
        for k in range(3):
            A, B = syn.operand_pair(cfg[0], 99, product=k)
            c = plan.mul(to_dev(A), to_dev(B))
            assert syn.to_int(to_host(c)) == syn.to_int(A) * syn.to_int(B)
        plan.sync_status()


def test_aliasing_output_rejected(dk):
    import torch
    cfg = SMALL[0]
    with dk.Plan(*cfg) as plan:
        buf = torch.zeros(3 * plan.words, dtype=torch.int64, device="cuda")
        with pytest.raises(dk.DkssError) as e:
            import ctypes
            lib = dk.load()
            rc = lib.dkss_mul(plan._h, buf.data_ptr(), buf.data_ptr() + 8 * plan.words,
                              buf.data_ptr() + 8 * plan.words, None)
            if rc:
                raise dk.DkssError(rc, "dkss_mul")
        assert e.value.code == 1


def large_checks(dk, oc, name, n_alpha_points, flags=0):
    cfg = syn.workload_params(name)
    par = o.Params(*cfg).check()
    A, B = syn.operand_pair(par.n_bits, syn.config_seed(syn.WORKLOADS[name]["index"]))
    with dk.Plan(*cfg, flags=flags) as plan:
        da, db = to_dev(A), to_dev(B)
        c = plan.mul(da, db)
        plan.sync_status()
        got = to_host(c)
        fwd = plan.forward(da)
        # sampled transform outputs at frequencies k*mu
        ks = list(range(0, 2 * par.m, max(1, 2 * par.m // n_alpha_points)))
        idx = [k * par.mu for k in ks]
        sampled = fwd[idx].cpu().numpy()
        del fwd
    # product: low word, length, residues mod random 61-bit primes
    assert int(got[0]) == (int(A[0]) * int(B[0])) % (1 << 64)
    assert got.size == 2 * A.size
    for q in random_primes61(4, seed=syn.WORKLOADS[name]["index"]):
        assert mod_int(got, q) == mod_int(A, q) * mod_int(B, q) % q
    for row, k in zip(sampled, ks):
        assert residues(row) == oc.fft_alpha_point(A, par, k)


@pytest.mark.parametrize("flags", FORMS)
def test_2p28_bits_properties(dk, oc, flags):
    large_checks(dk, oc, "dkss_2p28b", 8, flags)


def test_2p32_bits_properties(dk, oc):
    large_checks(dk, oc, "dkss_2p32b", 4)


def test_plans_of_one_kind_do_not_interfere(dk):
    """Two live plans of the same (m, L) with different last-level lengths:
    the second plan's set-up must not break the first (kernel attributes are
    shared by all plans of a kind)."""
    big = (1 << 20, 2048, 32, 32, 65537, 5)      # last level 2m = 64
    small = (16384, 64, 32, 16, 65537, 5)        # last level 2
    A, B = syn.operand_pair(big[0], 8)
    with dk.Plan(*big) as p1:
        with dk.Plan(*small) as p2:
            a2, b2 = syn.operand_pair(small[0], 9)
            assert syn.to_int(to_host(p2.mul(to_dev(a2), to_dev(b2)))) == syn.to_int(a2) * syn.to_int(b2)
        c = to_host(p1.mul(to_dev(A), to_dev(B)))
    assert syn.to_int(c) == syn.to_int(A) * syn.to_int(B)


# INT8 tensor-core form (DKSS_FORM_INT8TC): m >= 32, byte counts 6 .. 15
I8_CFGS = [SMALL[1], SMALL[2], SMALL[4], SMALL[5], SMALL[6]]


@pytest.mark.parametrize("cfg", I8_CFGS)
def test_int8_form_small_configs(dk, oc, cfg):
    A, B = syn.operand_pair(cfg[0], 4321, product=I8_CFGS.index(cfg))
    check_product(dk, oc, cfg, A, B, flags=2)
    A = syn.special_operand(cfg[0], "ones")
    check_product(dk, oc, cfg, A, A, with_forward=False, flags=2)


def test_int8_form_2p24_bits(dk, oc):
    cfg = syn.workload_params("dkss_2p24b")
    A, B = syn.operand_pair(cfg[0], syn.config_seed(1))
    check_product(dk, oc, cfg, A, B, flags=2)


def test_int8_form_2p28_bits_properties(dk, oc):
    large_checks(dk, oc, "dkss_2p28b", 8, flags=2)
