"""FP64 CPU oracle for the periodic FMM with a neutralising background charge.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: see ``fmm_oracle.c`` for the equations it follows
(Appendix A Ewald sum; Appendix B operators; Eq. 12 lattice sum; Eq. Velecfull;
Eq. FMMcalc).

All lengths in A, charges in e, energies in e^2/A (Gaussian units without
1/(4 pi eps0), as in Appendix A).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build

_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        vp = ctypes.c_void_p
        L.oracle_regular.argtypes = [c_int, vp, vp]
        L.oracle_irregular.argtypes = [c_int, vp, vp]
        L.oracle_p2m.argtypes = [c_int, c_int, vp, vp, vp, vp]
        L.oracle_m2m.argtypes = [c_int, vp, vp, vp, vp]
        L.oracle_m2l.argtypes = [c_int, vp, vp, vp, vp]
        L.oracle_l2l.argtypes = [c_int, vp, vp, vp, vp]
        L.oracle_l2p.argtypes = [c_int, vp, vp, vp, vp, vp]
        L.oracle_lattice.argtypes = [c_int, c_double, c_double, c_int, c_int, c_int, vp]
        L.oracle_fmm.argtypes = [c_int, vp, vp, c_double, c_int, c_int, c_int, c_double, vp, vp, vp, vp]
        L.oracle_fmm.restype = c_int
        L.oracle_fmm_sampled.argtypes = [c_int, vp, vp, c_double, c_int, c_int, c_int, c_double, c_int, vp,
                                         vp, vp, vp]
        L.oracle_fmm_sampled.restype = c_int
        L.oracle_fmm_solute_solvent.argtypes = [c_int, vp, vp, vp, c_double, c_int, c_int, c_int, c_double, vp]
        L.oracle_fmm_solute_solvent.restype = c_int
        L.oracle_softcore_nf_uv.argtypes = [c_int, vp, vp, vp, c_double, c_int, c_int, c_double, c_double, c_double,
                                            c_int, vp]
        L.oracle_softcore_nf_uv.restype = c_int
        L.oracle_ewald.argtypes = [c_int, vp, vp, c_double, c_double, c_double, c_double, vp, vp, vp]
        L.oracle_ewald.restype = c_int
        L.oracle_num_threads.restype = c_int
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def ncoef(p: int) -> int:
    return (p + 1) * (p + 1)


def hidx(n: int, m: int) -> int:
    return n * n + n + m


def num_threads() -> int:
    return lib().oracle_num_threads()


def default_kappa(L: float) -> float:
    """Splitting parameter of the level-0 lattice sum and the charged term: kappa L = 2."""
    return 2.0 / L


# ---------------------------------------------------------------- operators
def regular(p, v):
    out = np.zeros(ncoef(p), np.complex128)
    lib().oracle_regular(p, _ptr(_f64(v, 3)), _ptr(out))
    return out


def irregular(p, v):
    out = np.zeros(ncoef(p), np.complex128)
    lib().oracle_irregular(p, _ptr(_f64(v, 3)), _ptr(out))
    return out


def p2m(p, src, q, centre):
    src = _f64(src, (-1, 3))
    q = _f64(q)
    M = np.zeros(ncoef(p), np.complex128)
    lib().oracle_p2m(p, src.shape[0], _ptr(src), _ptr(q), _ptr(_f64(centre, 3)), _ptr(M))
    return M


def m2m(p, Mc, child, parent):
    Mp = np.zeros(ncoef(p), np.complex128)
    lib().oracle_m2m(p, _ptr(np.ascontiguousarray(Mc, np.complex128)), _ptr(_f64(child, 3)),
                     _ptr(_f64(parent, 3)), _ptr(Mp))
    return Mp


def m2l(p, M, src_centre, tgt_centre):
    L = np.zeros(ncoef(p), np.complex128)
    lib().oracle_m2l(p, _ptr(np.ascontiguousarray(M, np.complex128)), _ptr(_f64(src_centre, 3)),
                     _ptr(_f64(tgt_centre, 3)), _ptr(L))
    return L


def l2l(p, Lp, parent, child):
    Lc = np.zeros(ncoef(p), np.complex128)
    lib().oracle_l2l(p, _ptr(np.ascontiguousarray(Lp, np.complex128)), _ptr(_f64(parent, 3)),
                     _ptr(_f64(child, 3)), _ptr(Lc))
    return Lc


def l2p(p, L, centre, r):
    phi = np.zeros(1)
    g = np.zeros(3)
    lib().oracle_l2p(p, _ptr(np.ascontiguousarray(L, np.complex128)), _ptr(_f64(centre, 3)), _ptr(_f64(r, 3)),
                     _ptr(phi), _ptr(g))
    return phi[0], g


def lattice(jmax, b, kappa, ws=1, nu_max=None, n_kmax=None):
    """Eq. 12 lattice sum of I_j^k over images outside the (2ws+1)^3 block."""
    kb = kappa * b
    if nu_max is None:
        nu_max = int(math.ceil(7.0 / kb)) + ws + 2
    if n_kmax is None:
        n_kmax = int(math.ceil(2.0 * kb * 6.5 / (2 * math.pi))) + 2
    S = np.zeros(ncoef(jmax), np.complex128)
    lib().oracle_lattice(jmax, b, kappa, ws, nu_max, n_kmax, _ptr(S))
    return S


# ---------------------------------------------------------------- O2: FMM
def fmm(pos, q, L, d, p, ws=1, kappa=None, forces=True):
    """Plain FMM energy (Eq. Velecfull) with per-particle potentials and forces."""
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    N = q.shape[0]
    kappa = default_kappa(L) if kappa is None else kappa
    pn = np.zeros(N)
    pf = np.zeros(N)
    F = np.zeros((N, 3)) if forces else None
    terms = np.zeros(6)
    rc = lib().oracle_fmm(N, _ptr(pos), _ptr(q), L, d, p, ws, kappa, _ptr(pn), _ptr(pf), _ptr(F), _ptr(terms))
    if rc:
        raise ValueError("oracle_fmm: invalid arguments")
    names = ["near", "far", "charged", "quad_surface", "dipole_surface", "total"]
    out = dict(zip(names, terms.tolist()))
    out.update(phi_nf=pn, phi_ff=pf, forces=F, energy=terms[5])
    return out


def fmm_sampled(pos, q, L, d, p, idx, ws=1, kappa=None):
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    idx = np.ascontiguousarray(idx, np.int64)
    ns = idx.shape[0]
    kappa = default_kappa(L) if kappa is None else kappa
    pn = np.zeros(ns)
    pf = np.zeros(ns)
    F = np.zeros((ns, 3))
    rc = lib().oracle_fmm_sampled(q.shape[0], _ptr(pos), _ptr(q), L, d, p, ws, kappa, ns, _ptr(idx), _ptr(pn),
                                  _ptr(pf), _ptr(F))
    if rc:
        raise ValueError("oracle_fmm_sampled: invalid arguments")
    return dict(phi_nf=pn, phi_ff=pf, forces=F)


def solute_solvent(pos, q, is_solute, L, d, p, ws=1, kappa=None):
    """Reduced-far-field solute-solvent energy (Eq. FMMcalc) and its parts."""
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    sol = np.ascontiguousarray(is_solute, np.uint8)
    kappa = default_kappa(L) if kappa is None else kappa
    out = np.zeros(8)
    rc = lib().oracle_fmm_solute_solvent(q.shape[0], _ptr(pos), _ptr(q), _ptr(sol), L, d, p, ws, kappa, _ptr(out))
    if rc:
        raise ValueError("oracle_fmm_solute_solvent: invalid arguments")
    names = ["e_uv", "W", "A", "B", "C", "nf_uv", "bc_cross"]
    return dict(zip(names, out[:7].tolist()))


SOFTCORE_ALPHA = 0.2  # the paper's soft-core parameters (Calculation detail)
SOFTCORE_C = 6


def softcore_nf_uv(pos, q, is_solute, L, d, lam, A, ws=1, alpha=SOFTCORE_ALPHA, c=SOFTCORE_C):
    """Soft-core solute-solvent near-field energy and its lambda derivative: r -> (alpha lambda A^c +
    r^c)^(1/c) on the u-v pairs of the near-field stencil (the paper's soft-core form applied to the
    electrostatic NF term, as it remarks after the soft-core LJ equation)."""
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    sol = np.ascontiguousarray(is_solute, np.uint8)
    out = np.zeros(2)
    rc = lib().oracle_softcore_nf_uv(q.shape[0], _ptr(pos), _ptr(q), _ptr(sol), L, d, ws, lam, alpha, A, c,
                                     _ptr(out))
    if rc:
        raise ValueError("oracle_softcore_nf_uv: invalid arguments")
    return {"e_sc": float(out[0]), "de_sc_dlambda": float(out[1])}


# ---------------------------------------------------------------- O1: Ewald
def ewald(pos, q, b, kappa=None, rcut=None, kmax=None, forces=False):
    """Ewald energy of point charges plus background charge, conducting boundary (Appendix A)."""
    pos = _f64(pos, (-1, 3))
    q = _f64(q)
    N = q.shape[0]
    if rcut is None:
        rcut = 0.5 * b
    if kappa is None:
        kappa = 6.0 / rcut
    if kmax is None:
        kmax = 2.0 * kappa * math.sqrt(39.0)
    e = np.zeros(1)
    parts = np.zeros(4)
    F = np.zeros((N, 3)) if forces else None
    rc = lib().oracle_ewald(N, _ptr(pos), _ptr(q), b, kappa, rcut, kmax, _ptr(e), _ptr(F), _ptr(parts))
    if rc:
        raise ValueError("oracle_ewald: invalid arguments")
    return dict(energy=e[0], real=parts[0], reciprocal=parts[1], self=parts[2], charged=parts[3], forces=F)
