"""The allocation-free entry point fmm_background_terms_noalloc, through the C ABI.

It serves callers that cannot allocate device memory: an application or
plug-in whose device memory all belongs to another allocator or a fixed
budget, or a loop that cannot pay for an allocation's synchronisation.  Its
output must equal the background-charge terms that fmm_energy reports for the
same input, call after call, although every call reuses the same static
scratch array.  It returns no device-side status, so a NaN input must show up
as non-finite outputs rather than be dropped.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # FP64 on both sides, different summation order
MAX_N = 1 << 22


@pytest.fixture(scope="module")
def lib():
    from paper_2003_13218_gb300 import build
    from paper_2003_13218_gb300.fmm import load_library
    build.build()
    L = load_library()
    f = L.fmm_background_terms_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def _noalloc(lib, pos, q, L, kappa=0.0):
    dpos = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    dq = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.fmm_background_terms_noalloc(ctypes.c_void_p(dpos.data_ptr()), ctypes.c_void_p(dq.data_ptr()),
                                          len(q), L, kappa, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy()


def _reference_terms(pos, q, L, d=3, p=4):
    from paper_2003_13218_gb300.fmm import FMMPlan
    plan = FMMPlan(L, len(q), d, p)
    _, terms = plan.energy(torch.from_numpy(pos).cuda(), torch.from_numpy(q).cuda())
    plan.close()
    return terms


def _close(a, b):
    return abs(a - b) <= TOL * max(abs(b), 1e-300)


def test_noalloc_matches_fmm_energy_on_consecutive_calls(lib):
    # first call: many blocks (N = 100,000); second call: fewer blocks, so rows
    # written by the first call stay in the scratch array and must be ignored
    big = boxes.ion_in_water(33333, "Cl", seed=3)
    small = boxes.ion_in_water(700, "Mg", seed=4, L=30.0)
    small.pos[5] += [40.0, -31.0, 75.0]  # outside the box: wrapped like the plan path
    for b in (big, small):
        rc, out = _noalloc(lib, b.pos, b.q, b.L)
        assert rc == 0
        ref = _reference_terms(b.pos, b.q, b.L)
        assert _close(out[5], ref["charged"])
        assert _close(out[6], ref["quad_surface"])
        assert _close(out[7], ref["dipole_surface"])
        assert _close(out[0], float(np.sum(b.q)))


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    pos, q = boxes.random_charges(16, 2.0, seed=1)
    dpos = torch.from_numpy(pos).cuda()
    dq = torch.from_numpy(q).cuda()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.fmm_background_terms_noalloc(ctypes.c_void_p(dpos.data_ptr()), ctypes.c_void_p(dq.data_ptr()),
                                          MAX_N + 1, 2.0, 0.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0  # nothing was launched


def test_noalloc_nonfinite_input_reaches_the_outputs(lib):
    """A NaN charge (or an infinite coordinate) is not filtered out: the sums that contain it
    come out non-finite, and the next call with clean inputs is exact again."""
    b = boxes.ion_in_water(700, "Mg", seed=4, L=30.0)
    q = b.q.copy()
    q[17] = float("nan")
    rc, out = _noalloc(lib, b.pos, q, b.L)
    assert rc == 0
    assert not np.isfinite(out[0]) and not np.isfinite(out[5]) and not np.isfinite(out[6])
    pos = b.pos.copy()
    pos[3, 1] = float("inf")
    rc, out = _noalloc(lib, pos, b.q, b.L)
    assert rc == 0
    assert np.isfinite(out[0])  # Q does not involve coordinates
    assert not np.isfinite(out[2]) and not np.isfinite(out[7])
    rc, out = _noalloc(lib, b.pos, b.q, b.L)
    assert rc == 0
    ref = _reference_terms(b.pos, b.q, b.L)
    assert _close(out[5], ref["charged"]) and _close(out[6], ref["quad_surface"])
    assert _close(out[7], ref["dipole_surface"])
