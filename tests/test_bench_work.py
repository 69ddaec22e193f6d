"""The algorithmic work counts behind bench.py's rooflines, checked by
enumeration on small transforms (CPU).

A bad twiddle of level d multiplies element (v, l) of a block by
rho^(v l (2m)^d); it is work unless v l = 0 (Section 3.2.5 ii.).  A radix-2
decimation-in-time DFT of n points multiplies by a power of its root in every
butterfly; those with exponent 0 are products by 1 and not work.
"""
import pytest

import bench


def enumerate_nontrivial(P2, m, levels):
    """Bad twiddles with exponent != 0, by level, counted element by element."""
    out, length = [], P2
    for d in range(levels - 1):
        mu_d = length // (2 * m)
        bp = (2 * m) ** d
        n = 0
        for blk in range(P2 // length):
            for v in range(2 * m):
                for l in range(mu_d):
                    if (v * l * bp) % P2 != 0:
                        n += 1
        out.append(n)
        length //= 2 * m
    return out


def enumerate_dit_products(n):
    """Butterflies of an n-point radix-2 DIT whose twiddle exponent is not 0."""
    count, half = 0, 1
    while half < n:
        scale = n // (2 * half)
        for start in range(0, n, 2 * half):
            for k in range(half):
                if (k * scale) % n != 0:
                    count += 1
        half *= 2
    return count


@pytest.mark.parametrize("P2,m", [(64, 4), (256, 4), (512, 8), (2048, 16), (4096, 32)])
def test_nontrivial_twiddles_match_enumeration(P2, m):
    levels = 1
    while P2 // (2 * m) ** (levels - 1) > 2 * m:
        levels += 1
    info = {"P2": P2, "L": 3, "levels": levels, "pz": (1 << 80) + 1}
    brute = enumerate_nontrivial(P2, m, levels)
    r = bench.rmul_imads(m, 3, "ntt")
    work = bench.stage_work(info, m, "ntt")
    assert work["fwd_twiddle"] == (2 * sum(brute) * r, levels - 1)
    assert work["inv_twiddle"] == (sum(brute) * r, levels - 1)
    rd = bench.rmul_imads(m, 3, "direct")
    assert bench.stage_work(info, m, "direct")["fwd_twiddle"][0] == 2 * sum(brute) * rd
    S = 11
    assert bench.stage_work_i8(info, m)["fwd_twiddle"][0] == 2 * sum(brute) * 2 * S * S * m * m


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128])
def test_dit_products_match_enumeration(n):
    assert bench.nontrivial_dft_products(n) == enumerate_dit_products(n)


def test_montgomery_product_count():
    """A Montgomery product of L-limb residues: L^2 limb products (lo and hi
    halves each) and L(L+1) for the reduction's digits and q multiples,
    2 L^2 + L (2L + 1) 32-bit multiply-adds."""
    for L in (2, 3, 4, 5):
        limb_products = 2 * L * L
        reduction = L + 2 * L * L
        assert bench.modmul_imads(L) == limb_products + reduction
    # the NTT form's R-multiplication at m = 32: 80 + 32 + 96 = 208 products
    assert bench.rmul_imads(32, 4, "ntt") == 208 * bench.modmul_imads(4)


def test_limb_residues_match_python_int():
    """bench's product check: vectorised residues mod 31-bit primes equal the
    residues of the Python integer (sizes across the 2^12-limb blocks)."""
    import numpy as np
    import dkss_synth as syn
    for n_bits in (64, 4096 * 64, 4096 * 64 + 64, 100000):
        x = syn.operand(n_bits, 77, 0)
        v = syn.to_int(x)
        assert bench.limb_residues(x) == [v % q for q in bench.CHECK_PRIMES]
    A, B = syn.operand_pair(70000, 3)
    c = syn.from_int(syn.to_int(A) * syn.to_int(B), 2 * A.size)
    assert bench.check_product(c, A, B)
    c[123] ^= np.uint64(1 << 17)
    assert not bench.check_product(c, A, B)


def test_oracle_sample_is_a_valid_plan():
    """The CPU baseline's bounded sample of each workload: the workload itself
    up to 2^23 bits, else 2^23-bit operands with the same ring and encoding,
    which must satisfy the thesis's conditions (Section 3.2 steps 1-2)."""
    import dkss_oracle as o
    import dkss_synth as syn
    for name in syn.WORKLOADS:
        cfg, A, B, desc = bench.oracle_sample(name)
        full = syn.workload_params(name)
        assert cfg[2:] == list(full[2:])
        assert cfg[0] == min(full[0], bench.SAMPLE_MAX_BITS) and A.size == (cfg[0] + 63) // 64
        o.Params(*cfg).check()


@pytest.mark.parametrize("P2,m,levels", [(1024, 16, 3), (4096, 16, 3), (8192, 32, 3), (1 << 15, 64, 3)])
def test_transformed_elements_by_enumeration(P2, m, levels):
    """Elements per level whose bad twiddle is not 1 (the unit the captured
    per-element traffic is scaled by), against enumeration."""
    got = bench.transformed_elements({"P2": P2, "levels": levels}, m)
    assert got == enumerate_nontrivial(P2, m, levels)
