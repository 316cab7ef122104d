"""The bounded-wait path of the tensor-core kernels, made to run out on purpose without faulting anything.

Every wait in the tcgen05 M2L / M2M pipeline is bounded by a host-set budget (FMM_OPT_WAIT_BUDGET_NS).
The test hook FMM_OPT_INJECT_STALL makes the MMA issuer of the single-CTA kernel first wait on an mbarrier
that nothing arrives on -- the "flag that nothing sets" -- so the wait runs out after the budget, the CTA
aborts, waits (with its own limit) for the copies it had already issued, frees its TMEM and returns, and
the call reports FMM_ERR_TIMEOUT.  The plan must then evaluate correctly again."""
import numpy as np
import pytest

from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_wait_budget_runs_out_and_the_plan_recovers():
    from paper_2003_13218_gb300.fmm import FMMError, FMMPlan, FMM_OPT_INJECT_STALL, FMM_OPT_WAIT_BUDGET_NS
    b = boxes.ion_in_water(1500, "Na", seed=31)
    pos = torch.from_numpy(b.pos).to(DEV)
    q = torch.from_numpy(b.q).to(DEV)
    d, p = 4, 8
    plan = FMMPlan(b.L, b.N, d, p, precision="mixed", m2l_pair=False)  # single-CTA kernels only
    e_ok, _ = plan.energy(pos, q)
    plan.set_option(FMM_OPT_WAIT_BUDGET_NS, 1_000_000)  # 1 ms
    plan.set_option(FMM_OPT_INJECT_STALL, 1)
    for _ in range(2):
        with pytest.raises(FMMError) as e:
            plan.energy(pos, q)
        assert e.value.code == 5  # FMM_ERR_TIMEOUT
    plan.set_option(FMM_OPT_INJECT_STALL, 0)
    e_again, _ = plan.energy(pos, q)
    assert e_again == e_ok  # the same plan, bitwise
    F = torch.empty((b.N, 3), dtype=torch.float64, device=DEV)
    plan.forces(pos, q, out=F)
    assert torch.isfinite(F).all()
    plan.close()
    fresh = FMMPlan(b.L, b.N, d, p, precision="mixed", m2l_pair=False)
    assert fresh.energy(pos, q)[0] == e_ok
    fresh.close()


def test_wait_options_are_validated():
    from paper_2003_13218_gb300.fmm import FMMError, FMMPlan, FMM_OPT_INJECT_STALL, FMM_OPT_WAIT_BUDGET_NS
    plan = FMMPlan(4.0, 10, 2, 4)
    for key, bad in ((FMM_OPT_WAIT_BUDGET_NS, 999), (FMM_OPT_WAIT_BUDGET_NS, 10 ** 10 + 1),
                     (FMM_OPT_INJECT_STALL, 2), (FMM_OPT_INJECT_STALL, -1)):
        with pytest.raises(FMMError) as e:
            plan.set_option(key, bad)
        assert e.value.code == 1
    plan.close()
