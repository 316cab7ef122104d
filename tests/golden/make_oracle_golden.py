"""Write the FP64 oracle's results for the benchmarked workloads to tests/golden/.

Calls only the oracle (oracle/) and the seeded input generator
(paper_2003_13218_gb300.boxes, which holds no electrostatics); nothing here
touches the CUDA library.  The oracle takes minutes at N = 100,000 and most of
an hour at N = 1,000,000 on eight host cores, so its results are stored once
and the GPU parity tests read them.

Each file holds, for one (workload, ws, p):
  * the inputs' identity: seed, N, box, depth, order, ws, kappa, the sha256 of
    the position, charge and membership bytes, and a few input moments (the
    tests regenerate the inputs and check them against these);
  * every term of Eq. Velecfull the oracle reports (near, far, charged,
    quad_surface, dipole_surface, total);
  * every part of the reduced-far-field solute-solvent energy of Eq. FMMcalc
    (e_uv, W, A, B, C, nf_uv, bc_cross);
  * the oracle's forces on 64 seeded sample charges and the RMS force over all
    charges (the normalisation of the relative RMS force error).

Usage: python tests/golden/make_oracle_golden.py [name ...]
       (names: cl_100k_ws1_p12, cl_100k_ws2_p8, na_1m_ws1_p12; default all)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# name -> (workload, ws, p); depth and seed are the workload's
CASES = {
    "cl_100k_ws1_p12": ("cl_100k", 1, 12),
    "cl_100k_ws2_p8": ("cl_100k", 2, 8),
    "na_1m_ws1_p12": ("na_1m", 1, 12),
}
N_SAMPLES = 64
SAMPLE_STREAM = 21  # SplitMix64 stream of the sample indices


def input_identity(b) -> dict:
    """sha256 of the raw input bytes and moments that tolerate last-bit differences in the
    generator's transcendental functions between platforms."""
    h = hashlib.sha256()
    for a in (b.pos, b.q, b.is_solute):
        h.update(np.ascontiguousarray(a).tobytes())
    return {"sha256": h.hexdigest(),
            "sum_pos": np.sum(b.pos, axis=0).tolist(),
            "sum_pos2": float(np.sum(b.pos * b.pos)),
            "sum_q": float(np.sum(b.q)),
            "sum_q_pos": np.sum(b.q[:, None] * b.pos, axis=0).tolist()}


def sample_indices(N: int) -> np.ndarray:
    from paper_2003_13218_gb300 import boxes
    u = boxes.uniform01(0, SAMPLE_STREAM, N_SAMPLES)
    return np.unique((u * N).astype(np.int64))


def path_of(name: str) -> str:
    return os.path.join(HERE, "oracle_%s.json" % name)


def make(name: str) -> dict:
    import oracle
    from paper_2003_13218_gb300 import boxes
    workload, ws, p = CASES[name]
    b, d, _ = boxes.workload(workload, seed=0)
    kappa = oracle.default_kappa(b.L)
    t0 = time.perf_counter()
    full = oracle.fmm(b.pos, b.q, b.L, d, p, ws=ws, kappa=kappa, forces=True)
    t1 = time.perf_counter()
    uv = oracle.solute_solvent(b.pos, b.q, b.is_solute, b.L, d, p, ws=ws, kappa=kappa)
    t2 = time.perf_counter()
    idx = sample_indices(b.N)
    F = full["forces"]
    out = {
        "case": name, "workload": workload, "seed": 0, "N": b.N, "L": b.L, "depth": d, "p": p, "ws": ws,
        "kappa": kappa, "boundary": "conducting",
        "inputs": input_identity(b),
        "terms": {k: full[k] for k in ("near", "far", "charged", "quad_surface", "dipole_surface", "total")},
        "uv": uv,
        "sample_idx": idx.tolist(),
        "sample_forces": F[idx].tolist(),
        "force_rms": float(np.sqrt(np.mean(F * F))),
        "oracle_seconds": {"fmm": t1 - t0, "solute_solvent": t2 - t1, "threads": oracle.num_threads()},
        "written_by": "tests/golden/make_oracle_golden.py (oracle/ only)",
    }
    with open(path_of(name), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for n in names:
        r = make(n)
        print(n, r["terms"]["total"], r["uv"]["e_uv"], r["oracle_seconds"], flush=True)
