"""CPU-side checks of the Python binding's argument marshalling (paper_2003_13218_gb300/fmm.py).

The C ABI takes plain pointers and cannot see what they point to, so the binding checks element
types, element counts and, for outputs, that the buffer is written in place.  These tests drive the
binding's methods against a recording stand-in for the library handle (no GPU, no compute call):
valid host inputs reach the library with the right pointers, and an array that is too short, an
output of the wrong type or layout, or a batch entry that is not a contiguous CUDA tensor is refused
before any call is made."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_13218_gb300 import fmm  # noqa: E402


class _Recorder:
    """Stands in for the loaded library: records each call and returns FMM_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


def _plan(N):
    plan = object.__new__(fmm.FMMPlan)
    plan._lib = _Recorder()
    plan._h = ctypes.c_void_p(0)  # close() is a no-op for a null handle
    plan.N = N
    return plan


def _batch(Ns):
    bt = object.__new__(fmm.FMMBatch)
    bt._lib = _Recorder()
    bt._h = ctypes.c_void_p(0)
    bt.n = len(Ns)
    bt._N = np.asarray(Ns, np.int64)
    return bt


def _inputs(N, seed=0):
    rng = np.random.default_rng(seed)
    return rng.random((N, 3)), rng.random(N) - 0.5, (rng.random(N) < 0.1).astype(np.uint8)


def test_ptr_passes_matching_arrays_without_a_copy():
    a = np.zeros((5, 3))
    p, keep = fmm._ptr(a, 15, "f8", "pos")
    assert keep is a and p.value == a.ctypes.data
    t = torch.zeros(5, 3, dtype=torch.float64)
    p, keep = fmm._ptr(t, 15, "f8", "pos")
    assert keep is t and p.value == t.data_ptr()
    s = torch.zeros(5, dtype=torch.uint8)
    assert fmm._ptr(s, 5, "u1", "is_solute")[1] is s
    assert fmm._ptr(None, 5) == (None, None)


def test_ptr_converts_inputs_of_another_type_or_layout():
    a32 = np.arange(15, dtype=np.float32).reshape(5, 3)
    p, keep = fmm._ptr(a32, 15, "f8", "pos")
    assert keep.dtype == np.float64 and np.array_equal(keep, a32) and p.value == keep.ctypes.data
    t = torch.arange(30, dtype=torch.float64).reshape(5, 6)[:, ::2]  # not contiguous
    p, keep = fmm._ptr(t, 15, "f8", "pos")
    assert keep.is_contiguous() and torch.equal(keep, t)
    b = torch.tensor([True, False, True])
    _, keep = fmm._ptr(b, 3, "u1", "is_solute")
    assert keep.dtype == torch.uint8 and keep.tolist() == [1, 0, 1]


def test_ptr_refuses_short_arrays_and_outputs_it_would_copy():
    with pytest.raises(ValueError):
        fmm._ptr(np.zeros((4, 3)), 15, "f8", "pos")
    with pytest.raises(ValueError):
        fmm._ptr(torch.zeros(4, dtype=torch.float64), 5, "f8", "q")
    with pytest.raises(ValueError):  # float32 output: the library writes doubles
        fmm._ptr(torch.zeros(5, 3, dtype=torch.float32), 15, "f8", "forces", out=True)
    with pytest.raises(ValueError):  # a strided output would receive nothing
        fmm._ptr(torch.zeros(5, 6, dtype=torch.float64)[:, ::2], 15, "f8", "forces", out=True)
    with pytest.raises(ValueError):
        fmm._ptr(np.zeros((5, 3), np.float32), 15, "f8", "forces", out=True)
    ro = np.zeros((5, 3))
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        fmm._ptr(ro, 15, "f8", "forces", out=True)
    with pytest.raises(ValueError):
        fmm._ptr(np.zeros((4, 3)), 15, "f8", "forces", out=True)


def test_plan_methods_pass_valid_host_inputs_through():
    N = 7
    pos, q, sol = _inputs(N)
    plan = _plan(N)
    F = np.empty((N, 3))
    plan.evaluate(pos, q, sol, forces=F)
    plan.energy(pos, q)
    out, _ = plan.forces(pos, q)
    assert out.shape == (N, 3) and out.dtype == np.float64
    phi, _ = plan.potentials(torch.from_numpy(pos), torch.from_numpy(q), forces=torch.empty(N, 3, dtype=torch.float64))
    assert phi.shape == (N,) and phi.dtype == torch.float64
    plan.solute_solvent_energy(pos, q, sol)
    names = [c[0] for c in plan._lib.calls]
    assert names == ["fmm_evaluate", "fmm_energy", "fmm_forces", "fmm_potentials", "fmm_solute_solvent_energy"]
    ev = plan._lib.calls[0][1]
    assert ev[1].value == pos.ctypes.data and ev[2].value == q.ctypes.data
    assert ev[3].value == sol.ctypes.data and ev[4].value == F.ctypes.data


def test_plan_methods_refuse_bad_buffers_before_calling_the_library():
    N = 7
    pos, q, sol = _inputs(N)
    plan = _plan(N)
    bad = [
        lambda: plan.evaluate(pos[:-1], q, sol),
        lambda: plan.evaluate(pos, q[:-1], sol),
        lambda: plan.evaluate(pos, q, sol[:-1]),
        lambda: plan.evaluate(pos, q, sol, forces=np.empty((N, 3), np.float32)),
        lambda: plan.energy(pos, q[:3]),
        lambda: plan.forces(pos, q, out=np.empty((N - 1, 3))),
        lambda: plan.potentials(pos, q, out=np.empty(N, np.float32)),
        lambda: plan.potentials(pos, q, forces=np.empty((N, 3))[:, ::-1]),
        lambda: plan.solute_solvent_energy(pos, q, sol[:2]),
    ]
    for f in bad:
        with pytest.raises(ValueError):
            f()
    assert plan._lib.calls == []


def test_batch_refuses_entries_it_cannot_record_in_its_graph():
    Ns = [4, 6]
    bt = _batch(Ns)
    pos = [torch.zeros(n, 3, dtype=torch.float64) for n in Ns]
    q = [torch.zeros(n, dtype=torch.float64) for n in Ns]
    sol = [torch.zeros(n, dtype=torch.uint8) for n in Ns]
    with pytest.raises(ValueError):  # host tensors: the batch reads device memory only
        bt.lambda_energies(pos, q, sol)
    with pytest.raises(ValueError):  # one box missing
        bt.lambda_energies(pos[:1], q, sol)
    assert bt._lib.calls == []
    ptrs, keep = fmm._batch_ptrs([], [], "f8", "pos")
    assert len(ptrs) == 0 and keep == []
