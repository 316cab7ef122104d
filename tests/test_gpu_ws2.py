"""ws = 2, the paper's own near-field setting (App. B: second-nearest neighbour
leaves): 125-leaf near field, 875-cell interaction lists, a 5^3 block of image
cells left to the M2L levels.  The FP64 GPU path against the oracle at ws = 2
(the oracle's ws = 2 is pinned against Ewald in the CPU tests), the mixed path
(tensor-core M2L with halo width 2, CTA pairs and single CTAs) against the FP64
path, the solute-solvent energy, and the option's validation."""
import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(pos, q, L, d, p, sol=None, **kw):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(L, len(q), d, p, ws=2, **kw)
    F = torch.empty((len(q), 3), dtype=torch.float64, device=DEV)
    t, uv = plan.evaluate(torch.from_numpy(np.ascontiguousarray(pos)).to(DEV), torch.from_numpy(q).to(DEV),
                          None if sol is None else torch.from_numpy(sol).to(DEV), forces=F)
    plan.close()
    return t, uv, F.cpu().numpy()


def _rms_rel(F, ref):
    return float(np.sqrt(np.mean((F - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


@pytest.mark.parametrize("case", ["random", "mg"])
def test_ws2_fp64_against_oracle(case):
    if case == "random":
        pos, q = boxes.random_charges(700, 5.0, seed=21)
        L, d, p = 5.0, 3, 8
    else:
        b, d, p = boxes.workload("mg_3k")
        pos, q, L = b.pos, b.q, b.L
    ref = oracle.fmm(pos, q, L, d, p, ws=2)
    t, _, F = _run(pos, q, L, d, p)
    scale = abs(ref["total"])
    for k in ("near", "far", "charged", "quad_surface", "dipole_surface", "total"):
        assert abs(t[k] - ref[k]) <= 1e-12 * scale, k
    assert _rms_rel(F, ref["forces"]) < 1e-10


def test_ws2_mixed_against_fp64():
    b = boxes.ion_in_water(333333 // 64, "Na", seed=5, L=215.3 / 4)  # N = 15,625, d = 4: CTA pairs at level 4
    d, p = 4, 12
    t64, _, F64 = _run(b.pos, b.q, b.L, d, p)
    for pair in (True, False):
        tm, _, Fm = _run(b.pos, b.q, b.L, d, p, precision="mixed", m2l_pair=pair)
        assert abs(tm["total"] - t64["total"]) <= 1e-6 * abs(t64["total"])
        assert _rms_rel(Fm, F64) < 1e-5


def test_ws2_solute_solvent_against_oracle():
    b, d, p = boxes.workload("mg_3k")
    sol = b.is_solute
    ref = oracle.solute_solvent(b.pos, b.q, sol, b.L, d, p, ws=2)
    scale = abs(ref["A"]) + abs(ref["C"]) + abs(ref["e_uv"])
    _, uv, _ = _run(b.pos, b.q, b.L, d, p, sol=sol)
    for k in ("e_uv", "W", "A", "B", "C", "nf_uv", "bc_cross"):
        assert abs(uv[k] - ref[k]) <= 1e-11 * scale, k


def test_ws2_sparse_solute_pass_against_fp64():
    """depth 4: the sparse solute-only pass with 875-cell lists, mixed against FP64."""
    b = boxes.ion_in_water(333333 // 64, "Mg", seed=6, L=215.3 / 4)
    sol = np.zeros(b.N, np.uint8)
    sol[:16] = 1
    d, p = 4, 10
    _, u64, _ = _run(b.pos, b.q, b.L, d, p, sol=sol)
    _, umx, _ = _run(b.pos, b.q, b.L, d, p, sol=sol, precision="mixed")
    scale = abs(u64["A"]) + abs(u64["C"]) + abs(u64["e_uv"])
    for k in ("e_uv", "A", "B", "C"):
        assert abs(umx[k] - u64[k]) <= 1e-5 * scale, k


def test_ws_option_validation():
    from paper_2003_13218_gb300.fmm import FMMPlan, FMMError, FMM_OPT_WS
    plan = FMMPlan(10.0, 100, 2, 4)
    with pytest.raises(FMMError):
        plan.set_option(FMM_OPT_WS, 2)  # 2^2 = 4 leaves per side: the 5-leaf near field would hold own images
    with pytest.raises(FMMError):
        plan.set_option(FMM_OPT_WS, 3)
    plan.close()
