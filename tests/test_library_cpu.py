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
