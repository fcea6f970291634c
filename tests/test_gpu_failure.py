"""The error paths, exercised without any GPU fault: a workspace allocation
made to fail on the host (G3PCF_OPT_TEST_FAIL_ALLOC) and a bounded device wait
made to give up early (G3PCF_OPT_TEST_TC_TIMEOUT).  Each call must return its
error code, and the next normal call on the same plan must match the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1709_00086_gb300 as g3  # noqa: E402
from paper_1709_00086_gb300 import catalogs  # noqa: E402

from gpu_util import maxrel, oracle_zeta, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _cat():
    return catalogs.small_case("clustered", 3000, seed=97, box=300.0, nbins=6, rmin=0.0, rmax=60.0, lmax=6)


def _check(plan, cat, ref, tc):
    z, c = plan.compute(*to_dev(cat, torch), fp32_contraction=not tc)
    np.testing.assert_array_equal(c.cpu().numpy(), ref[1])
    assert maxrel(z.cpu().numpy(), ref[0]) < (1e-4 if tc else 1e-5)


def test_injected_allocation_failure_at_every_workspace_growth_then_recovery():
    # the k-th workspace growth of a fresh plan's first forward fails, for every k
    # until the forward needs fewer growths than k; each time the same plan then
    # runs normally and matches the oracle
    cat = _cat()
    ref = oracle_zeta(cat)
    pos, w = to_dev(cat, torch)
    failed = 0
    for k in range(1, 200):
        plan = g3.Plan(**cat.params())
        plan.set_option(g3.OPT_TEST_FAIL_ALLOC, k)
        try:
            plan.compute(pos, w)
        except g3.G3PCFError as e:
            assert e.name == "ERR_ALLOC" and "injected" in str(e)
            failed += 1
            plan.set_option(g3.OPT_TEST_FAIL_ALLOC, 0)
            _check(plan, cat, ref, tc=True)
            if k % 4 == 1:
                _check(plan, cat, ref, tc=False)
            continue
        break  # this forward grew its workspace fewer than k times
    assert failed >= 8, failed


def test_injected_allocation_failure_in_backward():
    cat = _cat()
    plan = g3.Plan(**cat.params())
    pos, w = to_dev(cat, torch)
    plan.compute(pos, w, keep_alm=True)
    dz = torch.zeros((plan.zsize, 2), dtype=torch.float64, device="cuda")
    plan.set_option(g3.OPT_TEST_FAIL_ALLOC, 1)
    with pytest.raises(g3.G3PCFError) as ei:
        plan.backward(dz)
    assert ei.value.name == "ERR_ALLOC"
    dpos, dw = plan.backward(dz)  # zero dL/dzeta: zero gradient
    assert torch.count_nonzero(dpos).item() == 0 and torch.count_nonzero(dw).item() == 0


@pytest.mark.parametrize("operands", [0, 1])
def test_tensor_core_wait_gives_up_then_recovery(operands):
    # operands 1: the contraction kernel that copies the operands written by the
    # pair stage, whose MMA thread waits on the copies instead of the converters
    cat = _cat()
    ref = oracle_zeta(cat)
    plan = g3.Plan(**cat.params())
    plan.set_option(g3.OPT_TC_OPERANDS, operands)
    _check(plan, cat, ref, tc=True)
    assert plan.stats()["tc_operands_from_pairs"] == float(operands)
    plan.set_option(g3.OPT_TEST_TC_TIMEOUT, 1)
    with pytest.raises(g3.G3PCFError) as ei:
        plan.compute(*to_dev(cat, torch))
    assert ei.value.name == "ERR_TIMEOUT"
    plan.set_option(g3.OPT_TEST_TC_TIMEOUT, 0)
    _check(plan, cat, ref, tc=True)
    _check(plan, cat, ref, tc=False)
