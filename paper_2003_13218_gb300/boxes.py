"""Seeded synthetic ion-in-water boxes (input generation only).

This module holds no part of the electrostatics: it only places point charges.
It is the one module both the FP64 oracle tests and the CUDA path read their
inputs from, so that the two sides see bit-identical coordinates and charges.

The composition follows the paper's workload (Calculation detail section: one
ion -- Mg2+, Na+ or Cl- -- dissolved in rigid three-site TIP3P water in a cubic
periodic cell).  The paper's MD snapshots are not available, so boxes are
generated:

* molecule sites on an n^3 lattice, n = smallest integer with n^3 >= N_w + 1,
  spacing a = L/n, coordinate (i + (n mod 2)/2) * a, so that lattice site
  floor(n/2) sits exactly at L/2;
* the ion takes the centre site and is not jittered;
* N_w of the remaining sites are chosen by a seeded random permutation, each
  jittered by U(-0.3, 0.3) A per axis; the water oxygen sits on the site and
  the molecule gets a uniformly random orientation (uniform unit quaternion);
* TIP3P geometry: O-H 0.9572 A, H-O-H 104.52 deg, charges O -0.834 e,
  H +0.417 e;
* all atoms are wrapped into [0, L);
* the box side is L = (N_w / 0.0334)^(1/3) A unless given.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) run as
a counter-based generator, so the streams are identical on every platform.
Atom 0 is the ion; atoms 1.. are water O, H, H per molecule.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WATER_DENSITY = 0.0334  # molecules per A^3
Q_O = -0.834
Q_H = 0.417
R_OH = 0.9572
THETA_HOH = math.radians(104.52)
ION_CHARGE = {"Mg": 2.0, "Na": 1.0, "Cl": -1.0}
COULOMB_KJ_PER_MOL = 1389.35458  # 1 e^2/A in kJ/mol

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """Counter-based SplitMix64: output k = mix(base + (k + 1) * golden)."""
    base = np.uint64((seed * 0x632BE59BD9B4E019 + stream * 0x8CB92BA72F3D8DD7) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = base + (np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def lattice_side(n_sites: int) -> int:
    n = 1
    while n * n * n < n_sites:
        n += 1
    return n


@dataclasses.dataclass
class Box:
    pos: np.ndarray        # [N, 3] float64, wrapped into [0, L)
    q: np.ndarray          # [N] float64, charges in e
    is_solute: np.ndarray  # [N] uint8, 1 for the ion
    L: float               # cubic box side, A
    ion: str
    n_waters: int
    seed: int

    @property
    def N(self) -> int:
        return int(self.q.shape[0])


def _quat_rotations(u1, u2, u3):
    """Uniform random rotation matrices from three uniforms (Shoemake 1992)."""
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((u1.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def ion_in_water(n_waters: int, ion: str = "Na", seed: int = 0, L: float | None = None,
                 jitter: float = 0.3, ion_charge: float | None = None) -> Box:
    """One ion at the box centre plus ``n_waters`` rigid TIP3P waters."""
    if L is None:
        L = (n_waters / WATER_DENSITY) ** (1.0 / 3.0)
    L = float(L)
    n = lattice_side(n_waters + 1)
    a = L / n
    off = 0.5 * (n % 2)
    centre = n // 2
    centre_lin = centre + n * (centre + n * centre)
    # seeded permutation of the other sites (sort of random 64-bit keys)
    keys = splitmix64(seed, 1, n ** 3)
    keys[centre_lin] = np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys, kind="stable")
    order = order[order != centre_lin][:n_waters]
    ix = order % n
    iy = (order // n) % n
    iz = order // (n * n)
    sites = np.stack([(ix + off) * a, (iy + off) * a, (iz + off) * a], axis=1)
    jit = (uniform01(seed, 2, 3 * n_waters).reshape(n_waters, 3) * 2.0 - 1.0) * jitter
    sites = sites + jit
    u = uniform01(seed, 3, 3 * n_waters).reshape(n_waters, 3)
    rot = _quat_rotations(u[:, 0], u[:, 1], u[:, 2])
    h = THETA_HOH / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [R_OH * math.sin(h), 0.0, R_OH * math.cos(h)],
                     [-R_OH * math.sin(h), 0.0, R_OH * math.cos(h)]])
    atoms = sites[:, None, :] + np.einsum("wij,aj->wai", rot, body)
    pos = np.empty((1 + 3 * n_waters, 3))
    pos[0] = (centre + off) * a
    pos[1:] = atoms.reshape(-1, 3)
    pos = pos - L * np.floor(pos / L)
    pos[pos >= L] -= L
    qi = ION_CHARGE[ion] if ion_charge is None else float(ion_charge)
    q = np.empty(1 + 3 * n_waters)
    q[0] = qi
    q[1::3] = Q_O
    q[2::3] = Q_H
    q[3::3] = Q_H
    sol = np.zeros(1 + 3 * n_waters, dtype=np.uint8)
    sol[0] = 1
    return Box(pos=np.ascontiguousarray(pos), q=q, is_solute=sol, L=L, ion=ion,
               n_waters=n_waters, seed=seed)


# Named workloads: sizes, depth d (2^d leaves per side) and order p of the
# runs they are used for.
WORKLOADS = {
    "mg_3k": dict(n_waters=999, ion="Mg", L=31.0, depth=3, p=8),
    "cl_100k": dict(n_waters=33333, ion="Cl", L=None, depth=5, p=12),
    "na_1m": dict(n_waters=333333, ion="Na", L=None, depth=6, p=12),
    "mg_10m": dict(n_waters=3333333, ion="Mg", L=None, depth=7, p=10),
}


def workload(name: str, seed: int = 0) -> tuple[Box, int, int]:
    w = WORKLOADS[name]
    box = ion_in_water(w["n_waters"], w["ion"], seed=seed, L=w["L"])
    return box, w["depth"], w["p"]


def random_charges(N: int, L: float, seed: int = 0, neutral: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Uniformly placed random charges in [0, L)^3 (for small parity cases)."""
    pos = uniform01(seed, 11, 3 * N).reshape(N, 3) * L
    q = uniform01(seed, 12, N) * 2.0 - 1.0
    if neutral:
        q -= q.mean()
    return pos, q


# The batched free-energy workload (lambda windows of uneven size): box b holds
# n_w waters drawn uniformly from 3334..66666 (10,002..199,998 water atoms)
# plus one ion; the species cycles Mg, Na, Cl with b, the coupling is
# lambda_b = (b mod 16) / 15 and the ion's charge is scaled by lambda_b.
LAMBDA_NW_LO, LAMBDA_NW_HI = 3334, 66666
LAMBDA_STREAM = 7


def lambda_windows(nbox: int = 64, seed: int = 0) -> list[tuple[Box, float]]:
    u = uniform01(seed, LAMBDA_STREAM, nbox)
    out = []
    for b in range(nbox):
        n_w = LAMBDA_NW_LO + int(u[b] * (LAMBDA_NW_HI - LAMBDA_NW_LO + 1))
        ion = ("Mg", "Na", "Cl")[b % 3]
        lam = (b % 16) / 15.0
        box = ion_in_water(n_w, ion, seed=seed * 1000 + b, ion_charge=lam * ION_CHARGE[ion])
        out.append((box, lam))
    return out
