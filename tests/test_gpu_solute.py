"""Solute-solvent energy of the reduced far-field scheme (Eq. FMMcalc) on trees
deep enough for the sparse solute-only pass (depth >= 4), against the oracle's
two dense passes.  Cases: one ion (one active cell per level), 16- and 40-atom
solutes spread over several cells (shared targets, merged ancestors), and an
80-atom solute (beyond the sparse pass's 64 charges: the dense pass runs).

In the dense fallback the full-field potential at the solute charges (the A
of Eq. FMMcalc) comes from the mixed full pass (fp16x2 tensor-core M2L, about
2^-22 relative per product); the 80-charge case measured 5e-7 of the scale, so
every case keeps the 1e-5 bound."""
import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("e_uv", "W", "A", "B", "C", "nf_uv", "bc_cross")


def _box():
    return boxes.ion_in_water(333333 // 64, "Na", seed=5, L=215.3 / 4)  # N = 15,625


def _gpu_uv(b, sol, d, p, precision):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(b.L, b.N, d, p, precision=precision)
    dev = "cuda:0"
    _, uv = plan.evaluate(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.q).to(dev),
                          torch.from_numpy(sol).to(dev), forces=None)
    plan.close()
    return uv


@pytest.mark.parametrize("n_solute", [1, 16, 40, 80])
def test_sparse_solute_pass_against_oracle(n_solute):
    b = _box()
    sol = np.zeros(b.N, np.uint8)
    sol[:n_solute] = 1  # the ion and the first waters' atoms
    d, p = 4, 8
    ref = oracle.solute_solvent(b.pos, b.q, sol, b.L, d, p)
    scale = abs(ref["A"]) + abs(ref["C"]) + abs(ref["e_uv"])
    for precision, tol in (("fp64", 1e-11), ("mixed", 1e-5)):
        uv = _gpu_uv(b, sol, d, p, precision)
        for k in KEYS:
            assert abs(uv[k] - ref[k]) <= tol * scale, (precision, k, uv[k], ref[k])
        assert abs((uv["A"] - uv["B"]) - uv["C"]) <= 10 * tol * scale  # reciprocity (P10)


@pytest.mark.parametrize("n_solute", [1, 40])
def test_three_pass_solute_solvent_matches_reduced(n_solute):
    """The conventional scheme (Eq. FMMconv: three full passes, u+v, u alone and v alone, each
    set with its own background) against the reduced far field of Eq. FMMcalc on the GPU and against
    the oracle's E_uv.  The potentials
    are linear in the charges for a fixed tree, so E(u+v) - E(u) - E(v) and (A - B + C)/2 plus
    the near-field and background cross terms are the same quantity, equal up to rounding (FP64
    path)."""
    from paper_2003_13218_gb300.fmm import FMMPlan
    b = _box()
    sol = np.zeros(b.N, np.uint8)
    sol[:n_solute] = 1
    d, p = 4, 8
    dev = "cuda:0"
    plan = FMMPlan(b.L, b.N, d, p, precision="fp64")
    pos = torch.from_numpy(b.pos).to(dev)
    q = torch.from_numpy(b.q).to(dev)
    t, uv = plan.evaluate(pos, q, torch.from_numpy(sol).to(dev), forces=None)
    qu = torch.from_numpy(np.where(sol == 1, b.q, 0.0)).to(dev)
    qv = torch.from_numpy(np.where(sol == 1, 0.0, b.q)).to(dev)
    e_u, _ = plan.energy(pos, qu)
    e_v, _ = plan.energy(pos, qv)
    plan.close()
    three_pass = t["total"] - e_u - e_v
    assert abs(three_pass - uv["e_uv"]) <= 1e-10 * abs(t["total"])
    # and against the oracle's solute-solvent energy (Eq. FMMcalc, two dense FP64 passes on the host):
    # the three-pass difference carries the rounding of three totals of size |E|
    ref = oracle.solute_solvent(b.pos, b.q, sol, b.L, d, p)
    assert abs(three_pass - ref["e_uv"]) <= 1e-10 * abs(t["total"]), (three_pass, ref["e_uv"])
