"""Soft-core solute-solvent near field on the GPU (FMM_OPT_SOFTCORE): the paper's soft-core form for the
solute-solvent LJ term, r -> (alpha lambda A^c + r^c)^(1/c) with alpha = 0.2 and c = 6, which it notes
applies to the electrostatic NF term too (Calculation detail), on the near-field solute-solvent pairs.

Against the oracle (oracle.softcore_nf_uv, pinned in test_oracle_pins.py): the pair sum and its lambda
derivative, FP64 path to 1e-12 relative, mixed path (FP32 coordinates relative to the leaf centres, FP64
arithmetic) to 1e-6; lambda = 0 reproduces the plain NF_uv; the batch's V_lambda and dV/dlambda_C with the
softened pairs against central differences in lambda, with the recorded graph picking up changed lambdas."""
import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ALPHA, C = 0.2, 6


def _box():
    b = boxes.ion_in_water(3000, "Mg", seed=12)  # N = 9,001, depth 3
    sol = b.is_solute.copy()
    sol[1:7] = 1  # the ion and the first two waters: several solute charges, some sharing a leaf
    return b, sol


def _plan_uv(b, sol, d, p, precision, lam, A):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(b.L, b.N, d, p, precision=precision)
    plan.set_softcore(C, A, lam, ALPHA)
    _, uv = plan.evaluate(torch.from_numpy(b.pos).to(DEV), torch.from_numpy(b.q).to(DEV),
                          torch.from_numpy(sol).to(DEV), forces=None)
    plan.close()
    return uv


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("lam,A", [(0.0, 1.5), (0.36, 1.5), (1.0, 2.5)])
def test_softcore_pair_sum_against_oracle(precision, tol, lam, A):
    b, sol = _box()
    d, p = 3, 6
    ref = oracle.softcore_nf_uv(b.pos, b.q, sol, b.L, d, lam, A)
    uv = _plan_uv(b, sol, d, p, precision, lam, A)
    assert abs(uv["nf_sc"] - ref["e_sc"]) <= tol * abs(ref["e_sc"]), (uv["nf_sc"], ref["e_sc"])
    assert abs(uv["dnf_sc"] - ref["de_sc_dlambda"]) <= tol * abs(ref["de_sc_dlambda"]) + 1e-15
    if lam == 0.0:  # no softening: the plain near-field solute-solvent sum
        assert abs(uv["nf_sc"] - uv["nf_uv"]) <= tol * abs(uv["nf_uv"])


def test_softcore_off_leaves_the_uv_terms_unchanged():
    from paper_2003_13218_gb300.fmm import FMMPlan
    b, sol = _box()
    plan = FMMPlan(b.L, b.N, 3, 6, precision="fp64")
    args = (torch.from_numpy(b.pos).to(DEV), torch.from_numpy(b.q).to(DEV), torch.from_numpy(sol).to(DEV))
    _, plain = plan.evaluate(*args, forces=None)
    plan.set_softcore(C, 1.5, 0.5)
    _, soft = plan.evaluate(*args, forces=None)
    plan.set_softcore(0)
    _, off = plan.evaluate(*args, forces=None)
    plan.close()
    for k in ("e_uv", "W", "A", "B", "C", "nf_uv", "bc_cross"):
        assert plain[k] == soft[k] == off[k], k
    assert off["nf_sc"] == 0.0 and off["dnf_sc"] == 0.0 and soft["nf_sc"] != 0.0


def test_softcore_options_are_validated():
    from paper_2003_13218_gb300.fmm import (FMMError, FMMPlan, FMM_OPT_SOFTCORE, FMM_OPT_SOFTCORE_ALPHA,
                                            FMM_OPT_SOFTCORE_LAMBDA)
    plan = FMMPlan(4.0, 10, 2, 4)
    for key, iv, dv in ((FMM_OPT_SOFTCORE, 13, 1.0), (FMM_OPT_SOFTCORE, -1, 1.0), (FMM_OPT_SOFTCORE, 6, 0.0),
                        (FMM_OPT_SOFTCORE, 6, float("nan")), (FMM_OPT_SOFTCORE_LAMBDA, 0, 0.5),
                        (FMM_OPT_SOFTCORE_ALPHA, 0, -0.2)):
        with pytest.raises(FMMError) as e:
            plan.set_option(key, iv, dv)
        assert e.value.code == 1, (key, iv, dv)
    plan.set_option(FMM_OPT_SOFTCORE, 6, 1.0)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(FMMError):
            plan.set_option(FMM_OPT_SOFTCORE_LAMBDA, 0, bad)
    plan.close()


def test_batch_softcore_lambda_derivative_and_graph_replay():
    """V_lambda of every box with the softened near-field pairs: dV/dlambda_C from the batch equals the
    central difference of V_lambda in lambda; a replay of the recorded graph with new lambdas uses
    them (lambda is read from pinned host memory when the call runs)."""
    from paper_2003_13218_gb300.fmm import FMMBatch
    wins = []
    for k, ion in enumerate(("Mg", "Na", "Cl")):
        b = boxes.ion_in_water(1500 + 400 * k, ion, seed=40 + k)
        wins.append(b)
    pos = [torch.from_numpy(b.pos).to(DEV) for b in wins]
    q = [torch.from_numpy(b.q).to(DEV) for b in wins]
    sol = [torch.from_numpy(b.is_solute).to(DEV) for b in wins]
    bt = FMMBatch([b.L for b in wins], [b.N for b in wins], [3] * 3, [8] * 3, precision="fp64")
    bt.set_softcore(C, 2.0, ALPHA)
    lam = np.array([0.2, 0.5, 0.8])
    h = 1e-4
    r0 = bt.lambda_energies(pos, q, sol, lam)      # stream path, then recorded
    rp = bt.lambda_energies(pos, q, sol, lam + h)  # replays
    rm = bt.lambda_energies(pos, q, sol, lam - h)
    assert bt.info(0)["replays"] >= 2
    fd = (rp["v_lambda"] - rm["v_lambda"]) / (2 * h)
    assert np.all(np.abs(fd - r0["dv_dlambda"]) <= 1e-6 * np.abs(r0["dv_dlambda"]) + 1e-9), (fd, r0["dv_dlambda"])
    # at lambda = 0 the softened pairs are plain Coulomb: V_0 = E_total
    rz = bt.lambda_energies(pos, q, sol, np.zeros(3))
    assert np.allclose(rz["v_lambda"], rz["e_total"], rtol=1e-13, atol=0)
    # against the oracle's soft-core sum: V_lambda - (E_total - E_uv) = (1 - lambda)(E_uv - NF_uv + NF_sc)
    for i, b in enumerate(wins):
        sc = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 3, lam[i], 2.0)
        uv = oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, 3, 8)
        want = (1 - lam[i]) * (uv["e_uv"] - uv["nf_uv"] + sc["e_sc"])
        got = r0["v_lambda"][i] - (r0["e_total"][i] - r0["e_uv"][i])
        assert abs(got - want) <= 1e-10 * abs(r0["e_total"][i]), (i, got, want)
    bt.close()
