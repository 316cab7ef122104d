"""Batched lambda windows (fmm_batch_*): every box of a batch against its own plan
evaluated alone, the recorded CUDA graph against the stream path (same pointers,
data changed in place, a changed solute count), the depth tuner, and the
coupling formula V_lambda = E - lambda_C E_uv of Eq. Vswucheme / Eq. FMMVTI
against the Ewald definition (Appendix A) of the partly decoupled system."""
import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _small_windows(n=6, seed=3):
    out = []
    u = boxes.uniform01(seed, 11, n)
    for b in range(n):
        n_w = 300 + int(u[b] * 2700)
        ion = ("Mg", "Na", "Cl")[b % 3]
        lam = b / (n - 1)
        box = boxes.ion_in_water(n_w, ion, seed=seed * 100 + b, ion_charge=lam * boxes.ION_CHARGE[ion])
        out.append((box, lam))
    return out


def _dev(ws):
    pos = [torch.from_numpy(b.pos).to(DEV) for b, _ in ws]
    q = [torch.from_numpy(b.q).to(DEV) for b, _ in ws]
    sol = [torch.from_numpy(b.is_solute).to(DEV) for b, _ in ws]
    return pos, q, sol


def _single(b, d, p, pos, q, sol, precision="mixed"):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(b.L, b.N, d, p, precision=precision)
    t, uv = plan.evaluate(pos, q, sol, forces=None)
    plan.close()
    return t["total"], uv["e_uv"]


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_matches_single_plans(precision):
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = _small_windows()
    depths = [3 if b.N < 4000 else 4 for b, _ in ws]
    lam = np.array([l for _, l in ws])
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], depths, [10] * len(ws), precision=precision)
    r = bt.lambda_energies(pos, q, sol, lam)
    for i, (b, l) in enumerate(ws):
        e, uv = _single(b, depths[i], 10, pos[i], q[i], sol[i], precision)
        assert _rel(r["e_total"][i], e) < 1e-12
        assert abs(r["e_uv"][i] - uv) <= 1e-12 * abs(e)
        assert r["v_lambda"][i] == pytest.approx(e - l * uv, rel=1e-12, abs=1e-12 * abs(e))
        assert r["dv_dlambda"][i] == -r["e_uv"][i]
    bt.close()


def test_batch_graph_replay_and_fallback():
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = _small_windows(5, seed=4)
    depths = [4] * len(ws)  # depth >= 4: the sparse solute pass, which depends on the solute count
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], depths, [8] * len(ws))
    r1 = bt.lambda_energies(pos, q, sol)
    r2 = bt.lambda_energies(pos, q, sol)
    r3 = bt.lambda_energies(pos, q, sol)
    info = bt.info(0)
    assert info["enqueued"] == 1 and info["replays"] == 2  # recorded once, replayed twice
    for k in ("e_total", "e_uv"):
        assert np.array_equal(r1[k], r2[k]) and np.array_equal(r1[k], r3[k])
    # new coordinates in place: the replay sees them
    g = torch.Generator(device="cpu").manual_seed(5)
    for i in range(len(ws)):
        pos[i].add_((torch.rand(pos[i].shape, generator=g, dtype=torch.float64) - 0.5).to(DEV) * 0.02)
    r4 = bt.lambda_energies(pos, q, sol)
    assert bt.info(0)["replays"] == 3
    for i, (b, _) in enumerate(ws):
        e, uv = _single(b, 4, 8, pos[i], q[i], sol[i])
        assert _rel(r4["e_total"][i], e) < 1e-12 and abs(r4["e_uv"][i] - uv) <= 1e-12 * abs(e)
    # a different solute set (count 1 -> 4) in place: the replay notices and the stream path runs
    sol[2][1:4] = 1
    r5 = bt.lambda_energies(pos, q, sol)
    info = bt.info(0)
    assert info["enqueued"] == 2 and info["replays"] == 4
    e, uv = _single(ws[2][0], 4, 8, pos[2], q[2], sol[2])
    assert _rel(r5["e_total"][2], e) < 1e-12 and abs(r5["e_uv"][2] - uv) <= 1e-12 * abs(e)
    r6 = bt.lambda_energies(pos, q, sol)  # recorded again with the new count
    assert bt.info(0)["replays"] == 5 and np.array_equal(r5["e_uv"], r6["e_uv"])
    bt.close()


def test_batch_depth_tuner():
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = [(boxes.ion_in_water(n, "Na", seed=9 + n), 0.5) for n in (1500, 1700, 14000)]
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], None, [8] * 3)
    r = bt.lambda_energies(pos, q, sol, [0.5] * 3)
    for i, (b, _) in enumerate(ws):
        d = bt.info(i)["depth"]
        d0 = int(round(np.log(b.N / 3.8) / np.log(8.0)))
        assert abs(d - d0) <= 1 and d >= 2
        e, uv = _single(b, d, 8, pos[i], q[i], sol[i])
        assert _rel(r["e_total"][i], e) < 1e-12
    assert bt.info(0)["depth"] == bt.info(1)["depth"]  # one group, one choice
    bt.close()


def _ewald_energy(pos, q, L):
    return oracle.ewald(pos, q, L)["energy"]


@pytest.mark.parametrize("lam", [0.0, 0.36, 1.0])
def test_lambda_coupling_against_ewald(lam):
    """Eq. Vswucheme: V_lambda = E(u+v) - lambda [E(u+v) - E(u) - E(v)], each E the Ewald
    energy of that set of charges with its own neutralising background (the u-v, u-Bv,
    v-Bu and Bu-Bv pairs scaled by 1 - lambda).  The ion sits off the leaf corners so that
    p = 12 converges (the corner case is pinned as a trend in the oracle tests)."""
    from paper_2003_13218_gb300.fmm import FMMBatch
    b, d, _ = boxes.workload("mg_3k")
    b.pos[0] += 0.5 * b.L / 2 ** d
    u = b.is_solute == 1
    e_all = _ewald_energy(b.pos, b.q, b.L)
    e_u = _ewald_energy(b.pos[u], b.q[u], b.L)
    e_v = _ewald_energy(b.pos[~u], b.q[~u], b.L)
    ref = e_all - lam * (e_all - e_u - e_v)
    pos, q, sol = _dev([(b, lam)])
    bt = FMMBatch([b.L], [b.N], [d], [12], precision="fp64")
    r = bt.lambda_energies(pos, q, sol, [lam])
    assert _rel(r["v_lambda"][0], ref) < 1e-6
    assert _rel(-r["dv_dlambda"][0], e_all - e_u - e_v) < 2e-5
    bt.close()
