"""Device-side range checks and library-chosen parameters (needs a GPU).

DKSS_DEBUG_CHECKS runs a range check over every polynomial at the stage
boundaries (every residue in [0, p^z), Section 3.2).  Valid products must pass
it in every form; an out-of-range residue written into the transformed
operand from the host (DKSS_FAULT_RANGE, a host-side injection: no kernel
faults or waits) must be reported as DKSS_EDEVICE by dkss_sync_status.

dkss_plan with M = m = u = p = z = 0 chooses its parameters (the thesis's rule
of Section 4.1, then timing of the best candidates); the products of such
plans must be exact.
"""
import pytest

import dkss_synth as syn
from gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

EDEVICE = 7


@pytest.fixture(scope="module")
def dk():
    import torch
    import paper_1503_04955_gb300 as pkg
    assert torch.cuda.is_available()
    pkg.buildlib.build()
    return pkg


CFGS = [
    (2000, 32, 16, 8, 193, 4),
    (786432, 2048, 32, 24, 65537, 5),
    (1 << 21, 1 << 14, 64, 16, 998244353, 4),
    (1 << 24, 1 << 15, 32, 32, 65537, 6),
]


@pytest.mark.parametrize("form", [0, 128, 16, 2])
@pytest.mark.parametrize("cfg", CFGS)
def test_debug_checks_pass_on_valid_products(dk, cfg, form):
    if form == 2 and cfg[2] < 32:
        pytest.skip("the INT8 form needs m >= 32")
    A, B = syn.operand_pair(cfg[0], 55, product=CFGS.index(cfg))
    with dk.Plan(*cfg, flags=form | dk.DEBUG_CHECKS) as plan:
        c = plan.mul(to_dev(A), to_dev(B))
        plan.sync_status()
        sq = plan.mul(to_dev(A), to_dev(A))
        plan.sync_status()
        assert syn.to_int(to_host(c)) == syn.to_int(A) * syn.to_int(B)
        assert syn.to_int(to_host(sq)) == syn.to_int(A) ** 2
        assert plan.launches > 0


@pytest.mark.parametrize("cfg", [CFGS[0], CFGS[2], CFGS[3]])
def test_debug_checks_report_an_injected_range_fault(dk, cfg):
    lib = dk.load()
    A, B = syn.operand_pair(cfg[0], 56)
    with dk.Plan(*cfg, flags=dk.DEBUG_CHECKS) as plan:
        old = lib.dkss_fault_inject(dk.FAULT_RANGE)
        try:
            plan.mul(to_dev(A), to_dev(B))
            with pytest.raises(dk.DkssError) as e:
                plan.sync_status()
            assert e.value.code == EDEVICE
        finally:
            lib.dkss_fault_inject(old)
        # the status word was cleared by the read; the next product is clean
        c = plan.mul(to_dev(A), to_dev(B))
        plan.sync_status()
        assert syn.to_int(to_host(c)) == syn.to_int(A) * syn.to_int(B)


def test_injected_fault_without_checks_is_not_reported(dk):
    """Without DKSS_DEBUG_CHECKS no range check runs (the flag costs nothing
    when off); the injection then goes unreported by the status word."""
    lib = dk.load()
    cfg = CFGS[0]
    A, B = syn.operand_pair(cfg[0], 57)
    with dk.Plan(*cfg) as plan:
        old = lib.dkss_fault_inject(dk.FAULT_RANGE)
        try:
            plan.mul(to_dev(A), to_dev(B))
            plan.sync_status()
        finally:
            lib.dkss_fault_inject(old)


@pytest.mark.parametrize("n_bits", [5000, 65536, 1 << 20, 3 << 20, 1 << 24])
def test_library_chosen_parameters(dk, n_bits):
    A, B = syn.operand_pair(n_bits, 58)
    want = syn.to_int(A) * syn.to_int(B)
    with dk.Plan(n_bits) as plan:
        params = (plan.M, plan.m, plan.u, plan.p, plan.z)
        assert params == dk.plan_choose(n_bits, 0)          # cached: the same choice
        assert syn.to_int(to_host(plan.mul(to_dev(A), to_dev(B)))) == want
        plan.sync_status()
    rule = dk.plan_choose(n_bits, dk.TUNE_RULE)
    with dk.Plan(n_bits, flags=dk.TUNE_RULE) as plan:
        assert (plan.M, plan.m, plan.u, plan.p, plan.z) == rule
        assert syn.to_int(to_host(plan.mul(to_dev(A), to_dev(B)))) == want


def test_library_chosen_parameters_int8(dk):
    n_bits = 1 << 20
    A, B = syn.operand_pair(n_bits, 59)
    with dk.Plan(n_bits, flags=dk.FORM_INT8TC) as plan:
        assert plan.m >= 32
        assert syn.to_int(to_host(plan.mul(to_dev(A), to_dev(B)))) == syn.to_int(A) * syn.to_int(B)
        plan.sync_status()
