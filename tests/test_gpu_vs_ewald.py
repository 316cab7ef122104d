"""GPU FMM against the exactly defined quantity it approximates: the Ewald sum of
the point charges plus their neutralising background under the conducting
boundary (Appendix A, the oracle's O1), on the ion-in-water workloads where the
Ewald sum is affordable on the host: Mg2+ + 999 waters (N = 2,998, d = 3) and
Cl- + 33,333 waters (N = 100,000, d = 5).

The 100,000-charge case costs minutes of host time for the Ewald sum (all pairs
in real space) and runs only with FMM_EWALD_100K=1 in the environment.

The FMM differs from Ewald by its truncation at order p (ws = 1); the mixed
path must add nothing visible to that difference.  Bounds: at p = 12 the
truncation error of these boxes is below 1e-6 of the energy (the oracle pins
the same trend on the CPU); at p = 8 below 1e-4.  The measured errors are
printed (run with -s)."""
import os

import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu(b, d, p, precision, forces=True):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(b.L, b.N, d, p, precision=precision)
    dev = "cuda:0"
    F = torch.empty((b.N, 3), dtype=torch.float64, device=dev) if forces else None
    terms, _ = plan.evaluate(torch.from_numpy(b.pos).to(dev), torch.from_numpy(b.q).to(dev), None, forces=F)
    plan.close()
    return terms["total"], (F.cpu().numpy() if forces else None)


def _rms_rel(F, ref):
    return float(np.sqrt(np.mean((F - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


@pytest.mark.parametrize("p,bound", [(8, 1e-4), (12, 1e-6)])
def test_mg_3k_against_ewald(p, bound):
    b, d, _ = boxes.workload("mg_3k")
    ref = oracle.ewald(b.pos, b.q, b.L, forces=True)
    e_ref, F_ref = ref["energy"], ref["forces"]
    out = {}
    for prec in ("fp64", "mixed"):
        e, F = _gpu(b, d, p, prec)
        out[prec] = (abs(e - e_ref) / abs(e_ref), _rms_rel(F, F_ref))
    print("\nEWALD mg_3k d=%d p=%d  fp64: energy %.3e force %.3e  mixed: energy %.3e force %.3e"
          % (d, p, out["fp64"][0], out["fp64"][1], out["mixed"][0], out["mixed"][1]))
    assert out["fp64"][0] < bound
    assert abs(out["mixed"][0] - out["fp64"][0]) < 1e-6  # the mixed path adds < 1e-6 to the truncation
    assert out["mixed"][1] < 10 * out["fp64"][1] + 1e-5


@pytest.mark.skipif(os.environ.get("FMM_EWALD_100K") != "1", reason="minutes of host time; FMM_EWALD_100K=1")
def test_cl_100k_against_ewald():
    b, d, p = boxes.workload("cl_100k")
    e_ref = oracle.ewald(b.pos, b.q, b.L)["energy"]
    e64, _ = _gpu(b, d, p, "fp64", forces=False)
    emx, _ = _gpu(b, d, p, "mixed", forces=False)
    r64, rmx = abs(e64 - e_ref) / abs(e_ref), abs(emx - e_ref) / abs(e_ref)
    print("\nEWALD cl_100k d=%d p=%d N=%d  fp64: energy %.3e  mixed: energy %.3e" % (d, p, b.N, r64, rmx))
    assert r64 < 1e-6
    assert rmx < 2e-6
