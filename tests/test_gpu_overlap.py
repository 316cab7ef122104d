"""Overlapped execution (FMM_OPT_OVERLAP): the near field on a low-priority stream
forked after the sort, the sparse solute pass of Eq. FMMcalc forked after the
full pass's M2L, both joined before the reductions.  The kernels and their
inputs are the same as in the in-order run, so every result must be bitwise
identical to it: energies, the solute-solvent terms and every force, for the
solute counts that take each branch of the pass (none, one, several, more than
the sparse pass's 64 charges), in both precisions.  A call that returns without
synchronising leaves its results ordered before later work on the caller's
stream."""
import numpy as np
import pytest

from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=dtype)


def _box():
    return boxes.ion_in_water(333333 // 64, "Na", seed=5, L=215.3 / 4)  # N = 15,625, d = 4


def _solute(b, n):
    sol = np.zeros(b.N, np.uint8)
    if n:
        c = b.pos[0]
        dist = np.linalg.norm(np.mod(b.pos - c + b.L / 2, b.L) - b.L / 2, axis=1)
        sol[np.argsort(dist)[:n]] = 1  # the ion and its nearest neighbours
    return sol


def _eval(b, sol, precision, overlap, calls=1):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(b.L, b.N, 4, 10, precision=precision, overlap=overlap)
    F = torch.empty((b.N, 3), dtype=torch.float64, device=DEV)
    out = []
    for _ in range(calls):
        t, uv = plan.evaluate(_t(b.pos), _t(b.q), _t(sol, torch.uint8), forces=F)
        out.append((t, uv, F.cpu().numpy()))
    plan.close()
    return out


@pytest.mark.parametrize("precision,n_solute", [("mixed", 0), ("mixed", 1), ("mixed", 5), ("mixed", 80),
                                                ("fp64", 5)])
def test_overlap_is_bitwise_identical_to_in_order(precision, n_solute):
    b = _box()
    sol = _solute(b, n_solute)
    ref = _eval(b, sol, precision, overlap=False)[0]
    for t, uv, F in _eval(b, sol, precision, overlap=True, calls=3):
        assert t == ref[0]
        assert uv == ref[1]
        assert np.array_equal(F, ref[2])


def test_overlap_without_solute_request():
    """Energy and forces alone: the near field forks, there is no solute pass."""
    from paper_2003_13218_gb300.fmm import FMMPlan
    b = _box()
    res = []
    for overlap in (False, True):
        plan = FMMPlan(b.L, b.N, 4, 10, precision="mixed", overlap=overlap)
        F, e = plan.forces(_t(b.pos), _t(b.q))
        res.append((e, F.cpu().numpy()))
        plan.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_asynchronous_call_is_ordered_on_the_callers_stream():
    from paper_2003_13218_gb300.fmm import FMMPlan
    b = _box()
    pos, q = _t(b.pos), _t(b.q)
    plan = FMMPlan(b.L, b.N, 4, 10, precision="mixed")
    F_ref, _ = plan.forces(pos, q)  # synchronised
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        F = torch.full((b.N, 3), float("nan"), dtype=torch.float64, device=DEV)
        plan.evaluate(pos, q, None, forces=F, want_terms=False)  # returns without synchronising
        G = F.clone()  # ordered after the call's join on s
    s.synchronize()
    assert torch.equal(G, F_ref)
    plan.close()
