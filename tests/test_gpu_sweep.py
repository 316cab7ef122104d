"""The persistent sweep of a batch (fmm_batch_*, FMM_BATCH_OPT_SWEEP): the CTA-pair
tensor-core levels (M2L of Eq. Lcoeffdef with the fused L2L) of all boxes in one
launch of persistent CTA pairs pulling (box, level, stage, tile) items from a device
queue.  It must give bitwise the results of the per-level launches, on the stream
path and in the recorded graph, cover exactly the boxes it can (order p of the first
box taking part, a level with full tile pairs), agree with single plans, and stop
cleanly with FMM_ERR_TIMEOUT when a dependency wait runs out."""
import numpy as np
import pytest

from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _windows(sizes, seed=7):
    out = []
    for b, n_w in enumerate(sizes):
        ion = ("Mg", "Na", "Cl")[b % 3]
        lam = (b % 4) / 3.0
        box = boxes.ion_in_water(n_w, ion, seed=seed * 100 + b, ion_charge=lam * boxes.ION_CHARGE[ion])
        out.append((box, lam))
    return out


def _dev(ws):
    pos = [torch.from_numpy(b.pos).to(DEV) for b, _ in ws]
    q = [torch.from_numpy(b.q).to(DEV) for b, _ in ws]
    sol = [torch.from_numpy(b.is_solute).to(DEV) for b, _ in ws]
    return pos, q, sol


# depths 3 (no pair level), 4 (sweep level 4), 5 (levels 4, 5) and 6 (levels 4..6); one box at p = 10
SIZES = [900, 5000, 11000, 16000, 21000, 34000]
DEPTHS = [3, 4, 4, 5, 5, 6]
PS = [12, 12, 10, 12, 12, 12]


def test_sweep_covers_the_pair_levels_and_is_bitwise_the_per_level_path():
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = _windows(SIZES)
    lam = np.array([l for _, l in ws])
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], DEPTHS, PS)
    info = bt.sweep_info()
    # depth 3: no level with full tile pairs; p = 10: another order than the first box taking part
    assert info["first_level"] == [0, 4, 0, 4, 4, 4] and info["boxes"] == 4
    bt.set_graph(False)
    r_on = bt.lambda_energies(pos, q, sol, lam)
    r_on2 = bt.lambda_energies(pos, q, sol, lam)
    bt.set_sweep(False)
    assert bt.sweep_info() == {"boxes": 0, "first_level": [0] * 6}
    r_off = bt.lambda_energies(pos, q, sol, lam)
    for k in ("e_total", "e_uv", "v_lambda", "dv_dlambda"):
        assert np.array_equal(r_on[k], r_off[k]), k
        assert np.array_equal(r_on[k], r_on2[k]), k
    bt.close()


def test_sweep_in_the_recorded_graph_and_against_single_plans():
    from paper_2003_13218_gb300.fmm import FMMBatch, FMMPlan
    ws = _windows(SIZES[1:], seed=8)
    d, p = DEPTHS[1:], [12] * 5
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], d, p)
    assert bt.sweep_info()["boxes"] == 5
    r1 = bt.lambda_energies(pos, q, sol)  # stream path, then recorded
    r2 = bt.lambda_energies(pos, q, sol)  # replay
    r3 = bt.lambda_energies(pos, q, sol)
    assert bt.info(0)["replays"] == 2
    for k in ("e_total", "e_uv"):
        assert np.array_equal(r1[k], r2[k]) and np.array_equal(r1[k], r3[k])
    # coordinates moved in place: the replayed sweep sees them
    g = torch.Generator(device="cpu").manual_seed(3)
    for i in range(len(ws)):
        pos[i].add_((torch.rand(pos[i].shape, generator=g, dtype=torch.float64) - 0.5).to(DEV) * 0.02)
    r4 = bt.lambda_energies(pos, q, sol)
    assert bt.info(0)["replays"] == 3
    for i, (b, _) in enumerate(ws):
        plan = FMMPlan(b.L, b.N, d[i], 12, precision="mixed")
        t, uv = plan.evaluate(pos[i], q[i], sol[i], forces=None)
        plan.close()
        assert abs(r4["e_total"][i] - t["total"]) <= 1e-12 * abs(t["total"])
        assert abs(r4["e_uv"][i] - uv["e_uv"]) <= 1e-12 * abs(t["total"])
    bt.close()


def test_sweep_dependency_wait_runs_out_and_the_batch_recovers():
    from paper_2003_13218_gb300.fmm import (FMM_BATCH_OPT_INJECT_STALL, FMM_BATCH_OPT_WAIT_BUDGET_NS, FMMBatch,
                                            FMMError)
    ws = _windows([5000, 16000, 21000], seed=9)
    pos, q, sol = _dev(ws)
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], [4, 5, 5], [12] * 3)
    ref = bt.lambda_energies(pos, q, sol)
    bt.set_option(FMM_BATCH_OPT_WAIT_BUDGET_NS, 1_000_000)  # 1 ms
    bt.set_option(FMM_BATCH_OPT_INJECT_STALL, 1)
    for _ in range(2):  # the stream path, then the graph recorded with the stall
        with pytest.raises(FMMError) as e:
            bt.lambda_energies(pos, q, sol)
        assert e.value.code == 5  # FMM_ERR_TIMEOUT
    bt.set_option(FMM_BATCH_OPT_INJECT_STALL, 0)
    again = bt.lambda_energies(pos, q, sol)
    again2 = bt.lambda_energies(pos, q, sol)
    for k in ("e_total", "e_uv"):
        assert np.array_equal(again[k], ref[k]) and np.array_equal(again2[k], ref[k])
    for key, bad in ((FMM_BATCH_OPT_WAIT_BUDGET_NS, 999), (FMM_BATCH_OPT_INJECT_STALL, 2), (99, 0)):
        with pytest.raises(FMMError) as e:
            bt.set_option(key, bad)
        assert e.value.code == 1
    bt.close()


def test_tuned_batch_picks_order_within_the_error_budget_and_the_faster_launch_form():
    """fmm_batch_create_tuned: boxes that leave p to the tuner take the smallest order whose energy error
    against FP64 p = 15 on the water test box of every depth group is within the budget (and the error it
    measured shrinks with the order); boxes with a given p keep it; the sweep is in use exactly when it
    replayed faster; the results are those of an untuned batch with the same depths and orders; and each
    box's mixed-precision energy at the tuned order is within 1e-6 of FP64 at the same order.  (The
    criterion is agreement with order 15 on the test boxes: at ws = 1 the FMM itself is not converged to
    1e-6 of the Ewald energy even at p = 15 on some boxes, so no per-box promise against the exact energy
    is made.)"""
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = _windows([4000, 9000, 16000, 21000], seed=12)
    pos, q, sol = _dev(ws)
    tol = 1e-6
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], [4, 4, 5, 5], [-1, -1, -1, 12], energy_rel_tol=tol,
                  sweep="auto")
    info = bt.tune_info()
    err = info["p_err"]
    assert all(err[p] >= 0.0 for p in (6, 8, 10, 12))
    assert err[6] > err[10] and err[8] > err[12]
    expect = next((p for p in (6, 8, 10, 12) if err[p] <= tol), 12)
    assert info["p_chosen"] == expect
    assert [bt.info(i)["p"] for i in range(4)] == [expect, expect, expect, 12]
    assert info["ms_sweep_off"] > 0.0 and info["ms_sweep_on"] > 0.0
    assert info["sweep_on"] == (info["ms_sweep_on"] < info["ms_sweep_off"])
    assert (bt.sweep_info()["boxes"] > 0) == info["sweep_on"]
    r = bt.lambda_energies(pos, q, sol)
    ref = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], [4, 4, 5, 5], [expect, expect, expect, 12])
    r_ref = ref.lambda_energies(pos, q, sol)
    for k in ("e_total", "e_uv"):
        assert np.array_equal(r[k], r_ref[k])
    ref.close()
    from paper_2003_13218_gb300.fmm import FMMPlan
    for i in range(3):
        b = ws[i][0]
        pl = FMMPlan(b.L, b.N, [4, 4, 5, 5][i], expect, precision="fp64")
        e64, _ = pl.energy(pos[i], q[i])
        pl.close()
        assert abs(r["e_total"][i] - e64) <= 1e-6 * abs(e64)
    bt.close()


def test_m2l_brick_option_changes_no_result():
    """FMM_OPT_M2L_BRICK regroups the targets of a level into tiles; every target's sum is the same, so
    energies, forces and E_uv are bitwise those of the default bricks, and bad bricks are refused."""
    from paper_2003_13218_gb300.fmm import FMM_OPT_M2L_BRICK, FMMError, FMMPlan
    b = boxes.ion_in_water(12000, "Cl", seed=5)
    pos = torch.from_numpy(b.pos).to(DEV)
    q = torch.from_numpy(b.q).to(DEV)
    sol = torch.from_numpy(b.is_solute).to(DEV)
    out = []
    for bricks in ([], [(5, 8, 4, 4), (4, 8, 4, 4)], [(5, 16, 4, 2)]):
        plan = FMMPlan(b.L, b.N, 5, 12, precision="mixed")
        for l, x, y, z in bricks:
            plan.set_brick(l, x, y, z)
        F = torch.empty((b.N, 3), dtype=torch.float64, device=DEV)
        t, uv = plan.evaluate(pos, q, sol, forces=F)
        out.append((t["total"], uv["e_uv"], F.cpu().numpy()))
        plan.close()
    for t, u, F in out[1:]:
        assert t == out[0][0] and u == out[0][1] and np.array_equal(F, out[0][2])
    plan = FMMPlan(b.L, b.N, 5, 12, precision="mixed")
    plan.set_brick(5, 16, 8, 1)  # the default brick of level 5 is accepted
    for l, x, y, z in ((5, 8, 8, 8),    # 512 cells
                       (6, 8, 4, 4),    # a level beyond the depth
                       (4, 3, 8, 4),    # does not divide the class side
                       (4, 8, 8, 2),    # fine at level 4 ...
                       (3, 4, 4, 8)):   # ... but level 3 (side 4) has one tile per class: no pairs
        if (l, x, y, z) == (4, 8, 8, 2):
            plan.set_brick(l, x, y, z)
            continue
        with pytest.raises(FMMError) as e:
            plan.set_brick(l, x, y, z)
        assert e.value.code == 1
    plan.close()
    p64 = FMMPlan(b.L, b.N, 5, 12, precision="fp64")
    with pytest.raises(FMMError) as e:
        p64.set_brick(5, 8, 4, 4)
    assert e.value.code == 7  # FMM_ERR_UNSUPPORTED: no tensor-core path
    p64.close()


def test_tuned_bricks_are_shared_by_a_depth_group_and_change_no_result():
    from paper_2003_13218_gb300.fmm import FMMBatch
    ws = _windows([9000, 11000, 16000, 21000], seed=13)
    pos, q, sol = _dev(ws)
    d, p = [4, 4, 5, 5], [12] * 4
    bt = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], d, p, tiles=True)
    br = [bt.brick(i) for i in range(4)]
    assert [l for l, _ in br] == d
    assert br[0][1] == br[1][1] and br[2][1] == br[3][1]
    for _, (x, y, z) in br:
        assert x * y * z == 128 and x >= y >= z
    r = bt.lambda_energies(pos, q, sol)
    ref = FMMBatch([b.L for b, _ in ws], [b.N for b, _ in ws], d, p)
    assert [ref.brick(i)[1] for i in range(4)] == [(8, 8, 2), (8, 8, 2), (16, 8, 1), (16, 8, 1)]
    r_ref = ref.lambda_energies(pos, q, sol)
    for k in ("e_total", "e_uv"):
        assert np.array_equal(r[k], r_ref[k])
    ref.close()
    bt.close()
