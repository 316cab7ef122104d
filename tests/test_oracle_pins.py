"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names the paper passage the pinned part follows and what fixes the
expected value: a closed form of the definitions, a textbook lattice constant
(tests/golden/lattice_constants.txt), an invariant, or a brute-force sum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2003_13218_gb300 import boxes
from tests.golden.constants import load as load_constants

C = load_constants()
PI = math.pi


def rel(a, b):
    return abs(a - b) / abs(b)


# --------------------------------------------------------------- harmonics
def test_regular_harmonics_closed_forms():
    """R_n^m of Eq. P2M / Eq. EqFF against the explicit low-degree polynomials."""
    x, y, z = 0.3, -0.4, 0.5
    R = oracle.regular(2, [x, y, z])
    h = oracle.hidx
    w = complex(x, y)
    assert R[h(0, 0)] == pytest.approx(1.0)
    assert R[h(1, 0)] == pytest.approx(z)
    assert R[h(1, 1)] == pytest.approx(-w / 2)
    assert R[h(1, -1)] == pytest.approx(w.conjugate() / 2)
    assert R[h(2, 0)] == pytest.approx((2 * z * z - x * x - y * y) / 4)
    assert R[h(2, 1)] == pytest.approx(-z * w / 2)
    assert R[h(2, 2)] == pytest.approx(w * w / 8)


def test_irregular_harmonics_closed_forms():
    """I_n^m of Eq. Lcoeffdef against the explicit low-degree forms."""
    x, y, z = 0.3, -0.4, 0.5
    r = math.sqrt(x * x + y * y + z * z)
    I = oracle.irregular(2, [x, y, z])
    h = oracle.hidx
    w = complex(x, y)
    assert I[h(0, 0)] == pytest.approx(1 / r)
    assert I[h(1, 0)] == pytest.approx(-z / r ** 3)
    assert I[h(1, 1)] == pytest.approx(-w / r ** 3)
    assert I[h(2, 0)] == pytest.approx((2 * z * z - x * x - y * y) / r ** 5)


def test_taylor_identity_of_inverse_distance():
    """1/|D + y| = sum_{N,M} R_N^M(y) I_N^{-M}(D): the identity behind Eq. Lcoeffdef."""
    D = np.array([1.7, -2.1, 0.9])
    yv = np.array([0.25, 0.31, -0.18])
    P = 40
    R = oracle.regular(P, yv)
    I = oracle.irregular(P, D)
    s = sum(R[oracle.hidx(n, m)] * I[oracle.hidx(n, -m)] for n in range(P + 1) for m in range(-n, n + 1))
    assert abs(s.imag) < 1e-14
    assert rel(s.real, 1 / np.linalg.norm(D + yv)) < 1e-14


def test_regular_addition_theorem():
    """R_N^M(a + b) = sum R_n^m(a) R_{N-n}^{M-m}(b): the identity behind M2M and L2L."""
    a = np.array([0.4, -0.2, 0.7])
    b = np.array([-0.3, 0.5, 0.1])
    P = 7
    Ra, Rb, Rab = oracle.regular(P, a), oracle.regular(P, b), oracle.regular(P, a + b)
    h = oracle.hidx
    for N in range(P + 1):
        for M in range(-N, N + 1):
            s = 0
            for n in range(N + 1):
                for m in range(-n, n + 1):
                    if abs(M - m) <= N - n:
                        s += Ra[h(n, m)] * Rb[h(N - n, M - m)]
            assert abs(s - Rab[h(N, M)]) < 1e-14


# --------------------------------------------------------------- operators (P5)
def _cluster(seed, n, centre, half):
    rng = np.random.default_rng(seed)
    return np.asarray(centre) + rng.uniform(-half, half, (n, 3)), rng.uniform(-1, 1, n)


@pytest.mark.parametrize("sep", [3.0, 4.0])
def test_p2m_m2l_l2p_against_direct_sum(sep):
    """Eq. P2M -> Eq. Lcoeffdef -> Eq. EqFF reproduces sum q/r; error decays geometrically in p."""
    src, q = _cluster(0, 20, [0, 0, 0], 0.5)
    tc = np.array([sep, 0.0, 0.0])
    tgt, _ = _cluster(1, 10, tc, 0.5)
    ref = np.array([np.sum(q / np.linalg.norm(t - src, axis=1)) for t in tgt])
    errs = []
    for p in (4, 8, 12, 16):
        M = oracle.p2m(p, src, q, [0, 0, 0])
        L = oracle.m2l(p, M, [0, 0, 0], tc)
        phi = np.array([oracle.l2p(p, L, tc, t)[0] for t in tgt])
        errs.append(np.max(np.abs(phi - ref)) / np.max(np.abs(ref)))
    assert all(errs[i + 1] < 0.05 * errs[i] for i in range(3))
    assert errs[-1] < 1e-10


def test_m2m_is_exact_translation():
    """M2M of child moments equals P2M taken directly about the parent centre."""
    p = 10
    child = np.array([0.25, -0.25, 0.25])
    parent = np.zeros(3)
    src, q = _cluster(2, 7, child, 0.25)
    Mc = oracle.p2m(p, src, q, child)
    Mp = oracle.m2m(p, Mc, child, parent)
    Md = oracle.p2m(p, src, q, parent)
    assert np.max(np.abs(Mp - Md)) < 1e-14 * np.max(np.abs(Md)) * 10


def test_l2l_is_exact_translation():
    """L2L re-expansion gives the same potential (and gradient) as the parent expansion."""
    p = 10
    src, q = _cluster(3, 9, [4.0, 1.0, -1.0], 0.5)
    parent = np.zeros(3)
    child = np.array([-0.25, 0.25, 0.25])
    M = oracle.p2m(p, src, q, [4.0, 1.0, -1.0])
    Lp = oracle.m2l(p, M, [4.0, 1.0, -1.0], parent)
    Lc = oracle.l2l(p, Lp, parent, child)
    r = child + np.array([0.1, -0.07, 0.05])
    f1, g1 = oracle.l2p(p, Lp, parent, r)
    f2, g2 = oracle.l2p(p, Lc, child, r)
    assert rel(f2, f1) < 1e-13
    assert np.max(np.abs(g2 - g1)) < 1e-13 * np.max(np.abs(g1))


def test_l2p_gradient_matches_finite_differences():
    p = 12
    src, q = _cluster(4, 9, [0, 0, 0], 0.5)
    tc = np.array([3.0, 1.0, 0.0])
    L = oracle.m2l(p, oracle.p2m(p, src, q, [0, 0, 0]), [0, 0, 0], tc)
    r = tc + np.array([0.2, -0.1, 0.3])
    _, g = oracle.l2p(p, L, tc, r)
    h = 1e-5
    fd = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd[a] = (oracle.l2p(p, L, tc, r + e)[0] - oracle.l2p(p, L, tc, r - e)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-8 * np.max(np.abs(g))


# --------------------------------------------------------------- lattice (P6)
def _irregular_cartesian(jmax, v):
    """Independent vectorised Cartesian recurrence for I_n^m, m >= 0 (v: [K,3])."""
    x, y, z = v[:, 0], v[:, 1], v[:, 2]
    r2 = x * x + y * y + z * z
    w = x + 1j * y
    T = {}
    T[(0, 0)] = 1 / np.sqrt(r2) + 0j
    for m in range(jmax + 1):
        if m > 0:
            T[(m, m)] = -(2 * m - 1) * w / r2 * T[(m - 1, m - 1)]
        for n in range(m + 1, jmax + 1):
            prev = T.get((n - 2, m), 0)
            # (-1)^(n+m) sign of I folded into the recurrence
            T[(n, m)] = (-(2 * n - 1) * z * T[(n - 1, m)] - (n + m - 1) * (n - m - 1) * prev) / r2
    return T


def test_lattice_odd_and_degree_two_vanish():
    """Cubic lattice: odd degrees vanish by inversion, degree 2 by cubic symmetry."""
    b = 1.0
    S = oracle.lattice(12, b, 2.0 / b)
    scale = np.max(np.abs(S))
    for j in (1, 2, 3, 5, 7, 9, 11):
        for m in range(-j, j + 1):
            assert abs(S[oracle.hidx(j, m)]) < 1e-13 * scale


def test_lattice_degree_four_is_the_cubic_harmonic():
    """Degree 4: only the cubic-invariant combination survives; its m=4 / m=0 ratio is the
    same as for the six axis vectors (the invariant subspace is one-dimensional)."""
    S = oracle.lattice(4, 1.0, 2.0)
    h = oracle.hidx
    for m in (1, 2, 3):
        assert abs(S[h(4, m)]) < 1e-12 * abs(S[h(4, 0)])
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    T = _irregular_cartesian(4, axes)
    ratio_axes = T[(4, 4)].sum() / T[(4, 0)].sum()
    assert abs(S[h(4, 4)] / S[h(4, 0)] - ratio_axes) < 1e-11


@pytest.mark.parametrize("j", [8, 10])
def test_lattice_high_degree_against_direct_sum(j):
    """Degrees j >= 8 converge absolutely: Eq. 12 (minus the near block) equals the direct
    sum over image cells outside the 3^3 block."""
    b, R = 1.3, 30
    g = np.arange(-R, R + 1)
    nu = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    nu = nu[np.max(np.abs(nu), axis=1) > 1].astype(float) * b
    T = _irregular_cartesian(j, nu)
    S = oracle.lattice(j, b, 2.0 / b)
    for m in (0, 4, 8):
        if m > j:
            continue
        direct = T[(j, m)].sum()
        tail = 6 * 4 * R * R * j ** 2 * math.factorial(j) / (R * b) ** (j + 1)  # crude bound
        assert abs(S[oracle.hidx(j, m)] - direct) < max(1e-12 * abs(direct), tail)


@pytest.mark.parametrize("kb", [1.5, 2.0, 3.0])
def test_lattice_monopole_gives_wigner_constant(kb):
    """Degree 0 plus the near block plus the charged term (Eq. 6) is kappa-independent and
    equals the simple-cubic Wigner constant / b (Eq. 12 with its self term 12c)."""
    b = 2.5
    kappa = kb / b
    S = oracle.lattice(0, b, kappa)
    block = sum(1 / (b * math.sqrt(i * i + j * j + k * k)) for i in (-1, 0, 1) for j in (-1, 0, 1)
                for k in (-1, 0, 1) if (i, j, k) != (0, 0, 0))
    val = S[0].real + block - PI / (b ** 3 * kappa ** 2)
    assert rel(val, C["wigner_sc"] / b) < 1e-11


# --------------------------------------------------------------- O1 Ewald
def _nacl(shift=0.25):
    na = [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0)]
    cl = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    return np.array(na + cl, float) + shift, np.array([1.0] * 4 + [-1.0] * 4), 2.0


def test_ewald_nacl_madelung():
    pos, q, b = _nacl()
    assert rel(oracle.ewald(pos, q, b)["energy"], -4 * C["nacl_madelung"]) < 1e-12


def test_ewald_cscl_madelung():
    """CsCl with a cell that carries a dipole: the conducting boundary of Appendix A gives the
    bulk Madelung energy."""
    a = 1.0
    pos = np.array([[0.1, 0.1, 0.1], [0.6, 0.6, 0.6]])
    q = np.array([1.0, -1.0])
    rnn = a * math.sqrt(3) / 2
    assert rel(oracle.ewald(pos, q, a)["energy"], -C["cscl_madelung"] / rnn) < 1e-12


@pytest.mark.parametrize("where", [[0.3, 0.7, 0.2], [0.5, 0.5, 0.5], [0.01, 0.99, 0.5]])
def test_ewald_wigner_single_charge(where):
    q = np.array([1.5])
    b = 1.7
    e = oracle.ewald(np.array([where]) * b, q, b)["energy"]
    assert rel(e, C["wigner_sc"] * q[0] ** 2 / (2 * b)) < 1e-11


def _wigner_crystal(kind, b, q, shift):
    """Charges q on a cubic cell of side b: 2 (body-centred) or 4 (face-centred) per cell."""
    basis = {"bcc": [(0, 0, 0), (0.5, 0.5, 0.5)],
             "fcc": [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]}[kind]
    pos = (np.array(basis) + np.array(shift)) * b
    n = len(basis)
    r_s = (3 * b ** 3 / (4 * PI * n)) ** (1 / 3)
    return pos, np.full(n, q), -n * C["wigner_" + kind] * q * q / r_s


@pytest.mark.parametrize("kind,shift", [("bcc", (0.13, 0.13, 0.13)), ("bcc", (0.71, 0.05, 0.4)),
                                        ("fcc", (0.21, 0.07, 0.33))])
def test_ewald_wigner_crystals(kind, shift):
    """Several equal charges per cell with the background (Q = 2, 4): the total net charge enters
    the charged term squared, and the energy is the published Wigner-crystal constant."""
    pos, q, target = _wigner_crystal(kind, 1.3, 0.7, shift)
    assert rel(oracle.ewald(pos, q, 1.3)["energy"], target) < 1e-11


def test_ewald_kappa_independent_for_charged_box():
    pos, q = boxes.random_charges(30, 3.0, seed=5)
    e = [oracle.ewald(pos, q, 3.0, kappa=k / 1.5)["energy"] for k in (5.0, 6.0, 7.5)]
    assert max(e) - min(e) < 1e-12 * abs(e[0])


def test_ewald_neutral_box_has_no_charged_term():
    pos, q = boxes.random_charges(20, 2.0, seed=6)
    q = np.where(np.arange(20) % 2 == 0, 1.0, -1.0)
    assert oracle.ewald(pos, q, 2.0)["charged"] == 0.0


def test_ewald_forces_match_finite_differences():
    pos, q = boxes.random_charges(12, 2.0, seed=7)
    F = oracle.ewald(pos, q, 2.0, forces=True)["forces"]
    h = 1e-5
    for i in (0, 5):
        for a in range(3):
            pp = pos.copy()
            pm = pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            fd = -(oracle.ewald(pp, q, 2.0)["energy"] - oracle.ewald(pm, q, 2.0)["energy"]) / (2 * h)
            assert abs(fd - F[i, a]) < 1e-6 * (1 + abs(F[i, a]))


# --------------------------------------------------------------- O2 FMM
@pytest.mark.parametrize("where,kb", [([0.3, 0.7, 0.2], 2.0), ([0.62, 0.41, 0.57], 2.0), ([0.12, 0.81, 0.45], 3.0)])
def test_fmm_wigner_single_charge(where, kb):
    """P2: one charge with background.  Isolates the lattice degree-0 entry, the self term
    (12c), the charged term (Eq. 6) and the cancellation of the two surface terms."""
    b = 1.7
    q = np.array([1.5])
    r = oracle.fmm(np.array(where)[None] * b, q, b, 2, 16, kappa=kb / b)
    assert rel(r["total"], C["wigner_sc"] * q[0] ** 2 / (2 * b)) < 2e-9
    assert rel(r["quad_surface"], -r["dipole_surface"]) < 1e-13


def test_fmm_wigner_charge_on_a_cell_corner():
    """A charge at the box centre sits on a leaf corner at every level: the worst case of the
    ws = 1 expansion (ratio (sqrt3/2 + sqrt3/2)/2).  The error still falls with p."""
    b = 1.7
    q = np.array([1.5])
    ref = C["wigner_sc"] * q[0] ** 2 / (2 * b)
    errs = [rel(oracle.fmm(np.array([[0.5, 0.5, 0.5]]) * b, q, b, 2, p, forces=False)["total"], ref)
            for p in (8, 16, 24)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-5


@pytest.mark.parametrize("kind,shift", [("bcc", (0.13, 0.13, 0.13)), ("fcc", (0.21, 0.07, 0.33))])
def test_fmm_wigner_crystals(kind, shift):
    """P2 with several charges per cell: the charged term (Eq. 6) with Q = 2 and 4, and the
    quadrupole and dipole surface terms (Eq. surfchargedend, App. D), which no longer cancel
    term by term, give the published Wigner-crystal energy; the error falls with p."""
    pos, q, target = _wigner_crystal(kind, 1.3, 0.7, shift)
    errs = [rel(oracle.fmm(pos, q, 1.3, 2, p, forces=False)["total"], target) for p in (12, 20)]
    assert errs[1] < 1e-9 and errs[1] < errs[0]


def test_fmm_nacl_madelung():
    """P1: neutral rock salt; BC terms vanish (Q = 0, mu = 0)."""
    pos, q, b = _nacl()
    r = oracle.fmm(pos, q, b, 2, 16)
    assert rel(r["total"], -4 * C["nacl_madelung"]) < 1e-8
    assert r["charged"] == 0.0 and r["quad_surface"] == 0.0


def test_fmm_cscl_dipole_term():
    """Neutral cell with a dipole: only the dipole surface term of Eq. Velecfull (App. D)
    turns the FMM's vacuum boundary into the conducting one."""
    pos = np.array([[0.1, 0.1, 0.1], [0.6, 0.6, 0.6]])
    q = np.array([1.0, -1.0])
    r = oracle.fmm(pos, q, 1.0, 2, 20)
    target = -C["cscl_madelung"] / (math.sqrt(3) / 2)
    assert rel(r["total"], target) < 1e-8
    assert abs(r["dipole_surface"]) > 0.1
    assert rel(r["total"] - r["dipole_surface"], target) > 1e-2


def test_fmm_kappa_independent():
    """P3: kappa of Eq. 12 and of Eq. 6 must be the same; then the total does not depend on it."""
    pos, q = boxes.random_charges(40, 2.0, seed=8)
    e = [oracle.fmm(pos, q, 2.0, 2, 8, kappa=kb / 2.0)["total"] for kb in (1.5, 2.0, 2.5, 3.0)]
    assert max(e) - min(e) < 1e-12 * abs(e[0])


def test_fmm_neutral_box_bc_terms_vanish():
    """P4: with Q_C = 0 the charged and quadrupole terms are exactly zero."""
    pos, _ = boxes.random_charges(24, 2.0, seed=9)
    q = np.where(np.arange(24) % 2 == 0, 0.5, -0.5)
    r = oracle.fmm(pos, q, 2.0, 2, 6)
    assert r["charged"] == 0.0 and r["quad_surface"] == 0.0


def test_fmm_converges_to_ewald_in_p():
    """P7 (the trend of the paper's error figure): log relative error falls with n_max on the
    Mg2+ + 999 water box, d = 3."""
    b, d, _ = boxes.workload("mg_3k")
    e = oracle.ewald(b.pos, b.q, b.L)["energy"]
    errs = [rel(oracle.fmm(b.pos, b.q, b.L, d, p, forces=False)["total"], e) for p in (4, 8, 12)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_fmm_ws2_converges_faster_than_ws1():
    """ws = 2 (the paper's near field of second-nearest neighbour leaves): interaction lists of
    875 cells, 125 near-field leaves, a 5^3 block left to the M2L levels.  Against Ewald on the
    Mg2+ box the error falls with p and stays below the ws = 1 error at the same p (the nearest
    M2L sources are twice as far)."""
    b, d, _ = boxes.workload("mg_3k")
    e = oracle.ewald(b.pos, b.q, b.L)["energy"]
    e1 = [rel(oracle.fmm(b.pos, b.q, b.L, d, p, ws=1, forces=False)["total"], e) for p in (4, 8)]
    e2 = [rel(oracle.fmm(b.pos, b.q, b.L, d, p, ws=2, forces=False)["total"], e) for p in (4, 8)]
    assert e2[0] > e2[1]
    assert e2[0] < e1[0] and e2[1] < e1[1]
    assert e2[1] < 1e-6


@pytest.mark.parametrize("N", [3, 17])
def test_fmm_ws2_tiny_boxes_against_ewald(N):
    """P8 at ws = 2: brute force on tiny net-charged sets, d = 3 (8 > 2 ws + 1), p = 16."""
    pos, q = boxes.random_charges(N, 1.0, seed=300 + N)
    e = oracle.ewald(pos, q, 1.0)["energy"]
    f = oracle.fmm(pos, q, 1.0, 3, 16, ws=2, forces=False)["total"]
    assert rel(f, e) < 2e-7


@pytest.mark.parametrize("N", [2, 5, 11, 24])
def test_fmm_tiny_boxes_against_ewald(N):
    """P8: brute force on tiny net-charged sets, d = 2, p = 20."""
    pos, q = boxes.random_charges(N, 1.0, seed=100 + N)
    e = oracle.ewald(pos, q, 1.0)["energy"]
    f = oracle.fmm(pos, q, 1.0, 2, 20, forces=False)["total"]
    assert rel(f, e) < 2e-7


def test_fmm_wrap_continuity_needs_quadrupole_term():
    """P9: an ion crossing the cell face changes the energy only at truncation level; without
    the quadrupole surface term (Eq. surfchargedend) the energy jumps (results section)."""
    pos, q = boxes.random_charges(30, 2.0, seed=10)
    q[0] = 2.0
    eps = 1e-9
    pa = pos.copy()
    pa[0] = [2.0 - eps, 0.9, 1.1]
    pb = pos.copy()
    pb[0] = [eps, 0.9, 1.1]  # the same point one period over
    ra = oracle.fmm(pa, q, 2.0, 3, 12, forces=False)
    rb = oracle.fmm(pb, q, 2.0, 3, 12, forces=False)
    jump = abs(ra["total"] - rb["total"])
    jump_noquad = abs((ra["total"] - ra["quad_surface"]) - (rb["total"] - rb["quad_surface"]))
    assert jump < 1e-5 * abs(ra["total"])
    assert jump_noquad > 100 * jump


def test_fmm_sampled_matches_full():
    b, d, _ = boxes.workload("mg_3k")
    full = oracle.fmm(b.pos, b.q, b.L, d, 6)
    idx = np.array([0, 17, 1500, 2997])
    s = oracle.fmm_sampled(b.pos, b.q, b.L, d, 6, idx)
    assert np.allclose(s["phi_nf"], full["phi_nf"][idx], rtol=1e-13, atol=0)
    assert np.allclose(s["phi_ff"], full["phi_ff"][idx], rtol=1e-12, atol=1e-14)
    assert np.allclose(s["forces"], full["forces"][idx], rtol=1e-12, atol=1e-13)


def test_fmm_forces_match_finite_differences():
    """P12: analytic forces (L2P gradient + pair forces + background term) equal -dE/dr."""
    pos, q = boxes.random_charges(40, 2.0, seed=11)
    q[0] = 1.7
    d, p = 2, 8
    F = oracle.fmm(pos, q, 2.0, d, p)["forces"]
    h = 1e-4
    leaf = 2.0 / 4
    for i in range(6):
        x = pos[i] / leaf
        if np.min(np.abs(x - np.round(x))) * leaf < 3 * h:
            continue
        for a in range(3):
            pp = pos.copy()
            pm = pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            ep = oracle.fmm(pp, q, 2.0, d, p, forces=False)["total"]
            em = oracle.fmm(pm, q, 2.0, d, p, forces=False)["total"]
            assert abs(-(ep - em) / (2 * h) - F[i, a]) < 1e-6 * (1 + abs(F[i, a]))


def test_fmm_potentials_are_the_charge_gradient():
    """Eq. Velecfull is a quadratic form in the charges, so dE/dq_i is the charge's pair potential
    (near + far, own images included) plus the derivatives of the background terms,
    -pi Q/(V kappa^2) + (2 pi/3V)(S2 + Q r_i^2) - (4 pi/3V) mu.r_i; central differences in q_i are
    exact up to rounding, and sum_i q_i phi_i = 2E (Euler).  This pins the oracle's per-charge
    potentials against its own energy, including the symmetry of the FMM bilinear form."""
    pos, q = boxes.random_charges(40, 2.0, seed=13)
    q[0] = 1.3  # net charge: every background term contributes
    L, d, p = 2.0, 2, 8
    out = oracle.fmm(pos, q, L, d, p, forces=False)
    kappa = oracle.default_kappa(L)
    V = L ** 3
    r = np.mod(pos, L)
    Q, mu, S2 = q.sum(), (q[:, None] * r).sum(0), float((q * (r * r).sum(1)).sum())
    phi = (out["phi_nf"] + out["phi_ff"] - PI * Q / (V * kappa ** 2)
           + 2 * PI / (3 * V) * (S2 + Q * (r * r).sum(1)) - 4 * PI / (3 * V) * (r @ mu))
    assert abs(float(q @ phi) - 2 * out["total"]) <= 1e-12 * float(np.abs(q * phi).sum())
    h = 1e-3
    for i in (0, 1, 7, 39):
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (oracle.fmm(pos, qp, L, d, p, forces=False)["total"] -
              oracle.fmm(pos, qm, L, d, p, forces=False)["total"]) / (2 * h)
        assert abs(fd - phi[i]) < 1e-9 * (1 + abs(phi[i]))


def test_fmm_forces_approach_ewald_forces():
    pos, q = boxes.random_charges(30, 2.0, seed=12)
    Fe = oracle.ewald(pos, q, 2.0, forces=True)["forces"]
    Ff = oracle.fmm(pos, q, 2.0, 2, 16)["forces"]
    assert np.sqrt(np.mean((Ff - Fe) ** 2)) < 1e-5 * np.sqrt(np.mean(Fe ** 2))


# --------------------------------------------------------------- solute-solvent
def _ewald_uv(pos, q, u, L):
    e_all = oracle.ewald(pos, q, L)["energy"]
    e_u = oracle.ewald(pos[u], q[u], L)["energy"]
    e_v = oracle.ewald(pos[~u], q[~u], L)["energy"]
    return e_all - e_u - e_v


def test_solute_solvent_reciprocity_and_ewald():
    """P10: the symmetric FMM bilinear form behind Eq. FMMcalc gives A - B = C; the result
    matches the Ewald interaction energy E(u+v) - E(u) - E(v), each set with its own
    neutralising background.  The ion is moved to a leaf centre, where its expansion is exact
    and the comparison is free of the slow corner convergence."""
    b, d, _ = boxes.workload("mg_3k")
    h = b.L / 2 ** d
    b.pos[0] += 0.5 * h
    p = 12
    r = oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, d, p)
    assert abs((r["A"] - r["B"]) - r["C"]) < 1e-11 * abs(r["C"])
    ref = _ewald_uv(b.pos, b.q, b.is_solute == 1, b.L)
    assert rel(r["e_uv"], ref) < 2e-5
    assert abs(r["bc_cross"]) > 1e-3 * abs(ref)
    r8 = oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, d, 8)
    assert rel(r8["e_uv"], ref) > rel(r["e_uv"], ref)


def test_solute_solvent_charged_solvent_against_ewald():
    """All three background cross terms (charged, quadrupole, dipole) enter when both sets
    carry net charge."""
    pos, q = boxes.random_charges(60, 2.0, seed=21)
    u = np.zeros(60, bool)
    u[:5] = True
    r = oracle.solute_solvent(pos, q, u.astype(np.uint8), 2.0, 2, 16)
    assert abs((r["A"] - r["B"]) - r["C"]) < 1e-11 * abs(r["C"])
    ref = _ewald_uv(pos, q, u, 2.0)
    assert rel(r["e_uv"], ref) < 1e-5


def test_solute_solvent_corner_ion_converges_in_p():
    """The workload ion sits on a leaf corner at every level; E_uv still converges in p."""
    b, d, _ = boxes.workload("mg_3k")
    ref = _ewald_uv(b.pos, b.q, b.is_solute == 1, b.L)
    errs = [rel(oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, d, p)["e_uv"], ref) for p in (6, 12)]
    assert errs[1] < errs[0] and errs[1] < 2e-3


def test_solute_solvent_linear_in_ion_charge():
    """P11: E_uv is linear in the solute charge at fixed coordinates."""
    b1 = boxes.ion_in_water(120, "Na", seed=3, L=16.0)
    b2 = boxes.ion_in_water(120, "Na", seed=3, L=16.0, ion_charge=0.36)
    r1 = oracle.solute_solvent(b1.pos, b1.q, b1.is_solute, b1.L, 2, 8)
    r2 = oracle.solute_solvent(b2.pos, b2.q, b2.is_solute, b2.L, 2, 8)
    assert rel(r2["e_uv"], 0.36 * r1["e_uv"]) < 1e-12


# ---------------------------------------------------------------- soft-core near field
def test_softcore_at_lambda_zero_is_the_plain_near_field():
    """At lambda = 0 the soft-core distance (alpha lambda A^c + r^c)^(1/c) is r: the sum is the plain
    solute-solvent near-field Coulomb sum of Eq. FMMcalc's NF part, whatever A."""
    b = boxes.ion_in_water(200, "Mg", seed=8, L=18.0)
    ref = oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, 3, 4)["nf_uv"]
    for A in (0.5, 1.0, 3.0):
        r = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 3, 0.0, A)
        assert rel(r["e_sc"], ref) < 1e-14
    # A = 0: no softening at any lambda
    r = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 3, 0.7, 0.0)
    assert rel(r["e_sc"], ref) < 1e-14 and r["de_sc_dlambda"] == 0.0


def test_softcore_far_pairs_reduce_to_coulomb():
    """For r >> A the soft-core pair energy is q q' / r (1 - alpha lambda (A/r)^c / c + ...): a single
    solute-solvent pair at r = 2.5 A with A = 0.25 A differs from Coulomb by alpha lambda 1e-6 / 6."""
    L = 12.0
    pos = np.array([[1.0, 1.0, 1.0], [3.5, 1.0, 1.0]])
    q = np.array([1.0, -0.8])
    sol = np.array([1, 0], np.uint8)
    lam, A = 0.5, 0.25
    r = oracle.softcore_nf_uv(pos, q, sol, L, 2, lam, A)
    coul = q[0] * q[1] / 2.5
    assert abs(r["e_sc"] / coul - 1.0 - (-0.2 * lam * (A / 2.5) ** 6 / 6)) < 1e-12
    assert r["e_sc"] > coul  # softening weakens the attraction


def test_softcore_lambda_derivative_matches_central_differences():
    b = boxes.ion_in_water(120, "Na", seed=3, L=16.0)
    A = 1.2
    for lam in (0.1, 0.5, 0.9):
        r = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 2, lam, A)
        h = 1e-5
        ep = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 2, lam + h, A)["e_sc"]
        em = oracle.softcore_nf_uv(b.pos, b.q, b.is_solute, b.L, 2, lam - h, A)["e_sc"]
        assert abs((ep - em) / (2 * h) - r["de_sc_dlambda"]) < 1e-7 * abs(r["de_sc_dlambda"]) + 1e-12


def test_softcore_removes_the_overlap_divergence():
    """The purpose of the soft-core form: a solvent charge on top of the solute charge gives a finite
    energy for lambda > 0, q q' / (alpha lambda A^c)^(1/c)."""
    L = 10.0
    pos = np.array([[2.0, 2.0, 2.0], [2.0, 2.0, 2.0 + 1e-9]])
    q = np.array([1.0, -1.0])
    sol = np.array([1, 0], np.uint8)
    r = oracle.softcore_nf_uv(pos, q, sol, L, 2, 1.0, 1.0)
    assert abs(r["e_sc"] - (-1.0 / 0.2 ** (1 / 6))) < 1e-9
