"""phi_i = dV/dq_i (fmm_potentials).  V_elec of Eq. Velecfull is a quadratic
form in the charges: the pair terms through the symmetric FMM bilinear form
(near field, M2L / lattice with the charge's own images, exact M2M and L2L of
the truncated expansions), the background terms through Q^2, Q S_2 and mu.mu.
So, in the FP64 path,
  * central differences in q_i are exact up to rounding,
  * sum_i q_i phi_i = 2 V (Euler's theorem for a function homogeneous of degree 2),
and the autograd wrapper's charge gradient is phi.  Host and device pointers,
both boundaries of App. D, and the mixed path against FP64."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=DEV, dtype=torch.float64)


def _plan(b, d, p, **kw):
    from paper_2003_13218_gb300.fmm import FMMPlan
    return FMMPlan(b.L, b.N, d, p, **kw)


@pytest.mark.parametrize("boundary", ["conducting", "vacuum"])
def test_potentials_are_the_charge_gradient(boundary):
    b = boxes.ion_in_water(200, "Mg", seed=8, L=18.0)  # net charge +2: every background term is present
    d, p = 3, 8
    plan = _plan(b, d, p, boundary=boundary)
    phi_d, e = plan.potentials(_t(b.pos), _t(b.q))
    phi = phi_d.cpu().numpy()
    assert abs(float(np.dot(b.q, phi)) - 2.0 * e) <= 1e-11 * float(np.sum(np.abs(b.q * phi)))
    h = 1e-3  # e; the energy is quadratic in q, so the central difference has no truncation error
    worst = 0.0
    for i in (0, 1, 2, 57, 200, 333, b.N - 1):
        qp = b.q.copy()
        qm = b.q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (plan.energy(_t(b.pos), _t(qp))[0] - plan.energy(_t(b.pos), _t(qm))[0]) / (2 * h)
        worst = max(worst, abs(fd - phi[i]) / (1.0 + abs(phi[i])))
    print("\nphi vs central differences in q (%s): max deviation %.2e" % (boundary, worst))
    assert worst < 1e-8
    plan.close()


def test_potentials_host_pointers_forces_and_autograd():
    from paper_2003_13218_gb300.fmm import FmmEnergy
    b = boxes.ion_in_water(200, "Cl", seed=9, L=18.0)
    d, p = 3, 8
    plan = _plan(b, d, p)
    F = torch.empty((b.N, 3), dtype=torch.float64, device=DEV)
    phi_d, e = plan.potentials(_t(b.pos), _t(b.q), forces=F)
    phi_h, e_h = plan.potentials(b.pos, b.q)
    assert e_h == e and np.array_equal(phi_h, phi_d.cpu().numpy())
    F2, e2 = plan.forces(_t(b.pos), _t(b.q))
    assert e2 == e and torch.equal(F2, F)
    x = _t(b.pos).requires_grad_(True)
    qq = _t(b.q).requires_grad_(True)
    E = FmmEnergy.apply(x, qq, plan)
    E.backward()
    assert E.item() == e
    assert torch.equal(qq.grad, phi_d) and torch.equal(x.grad, -F)
    plan.close()


def test_mixed_potentials_against_fp64():
    b = boxes.ion_in_water(1500, "Na", seed=10)
    d, p = 3, 10
    out = {}
    for prec in ("fp64", "mixed"):
        plan = _plan(b, d, p, precision=prec)
        phi, e = plan.potentials(_t(b.pos), _t(b.q))
        out[prec] = (phi.cpu().numpy(), e)
        plan.close()
    ref, e64 = out["fp64"]
    phi_m, em = out["mixed"]
    assert np.sqrt(np.mean((phi_m - ref) ** 2)) < 1e-5 * np.sqrt(np.mean(ref ** 2))
    # the mixed energy sums q_i phi_i with the charges rounded to FP32
    assert abs(float(np.dot(b.q, phi_m)) - 2.0 * em) <= 1e-6 * float(np.sum(np.abs(b.q * phi_m)))


def test_potentials_against_oracle():
    """phi against the oracle's per-charge potentials (near + far) plus the background terms'
    derivatives (the oracle pins this sum against central differences of its energy)."""
    pos, q = boxes.random_charges(700, 5.0, seed=2)
    q[0] += 0.75  # net charge
    L, d, p = 5.0, 3, 8
    ref = oracle.fmm(pos, q, L, d, p, forces=False)
    kappa = oracle.default_kappa(L)
    V = L ** 3
    r = np.mod(pos, L)
    Q, mu, S2 = q.sum(), (q[:, None] * r).sum(0), float((q * (r * r).sum(1)).sum())
    phi_ref = (ref["phi_nf"] + ref["phi_ff"] - math.pi * Q / (V * kappa ** 2)
               + 2 * math.pi / (3 * V) * (S2 + Q * (r * r).sum(1)) - 4 * math.pi / (3 * V) * (r @ mu))
    scale = np.sqrt(np.mean(phi_ref ** 2))
    for prec, tol in (("fp64", 1e-11), ("mixed", 1e-5)):
        from paper_2003_13218_gb300.fmm import FMMPlan
        plan = FMMPlan(L, len(q), d, p, precision=prec)
        phi, _ = plan.potentials(_t(pos), _t(q))
        plan.close()
        err = np.sqrt(np.mean((phi.cpu().numpy() - phi_ref) ** 2)) / scale
        assert err < tol, (prec, err)
