"""Thin Python binding of the C ABI in include/fmm_gb300.h (argument marshalling only).

Every step of an evaluation runs in the CUDA library ``libfmm_gb300.so``; this
module only passes pointers, sizes and options.  If the library is missing the
calls fail loudly -- there is no CPU fallback.

Inputs may be CUDA tensors (float64 positions [N, 3], float64 charges [N],
uint8 solute flags [N]) or host NumPy arrays / CPU tensors; host inputs go
through the library's own host<->device copies.  The binding checks what the
C ABI cannot: an input with fewer elements than the call reads is refused, one
of another element type or layout is converted; an output (forces, potentials)
is written in place and must be contiguous, of the right type and long enough.
A batch keeps the addresses of its per-box tensors in its recorded CUDA graph,
so those must already be contiguous CUDA tensors of the right type.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")

FMM_OPT_WS, FMM_OPT_PRECISION, FMM_OPT_KAPPA, FMM_OPT_M2L_SPLIT, FMM_OPT_STREAM, FMM_OPT_TIMINGS = 1, 2, 3, 4, 5, 6
FMM_OPT_M2L_PAIR = 7
FMM_OPT_BOUNDARY = 8
FMM_OPT_OVERLAP = 9
FMM_OPT_M2L_GRADE = 10
FMM_OPT_M2L_ACC_GROUP = 11
FMM_OPT_SOFTCORE, FMM_OPT_SOFTCORE_LAMBDA, FMM_OPT_SOFTCORE_ALPHA = 12, 13, 14
FMM_OPT_WAIT_BUDGET_NS, FMM_OPT_INJECT_STALL = 15, 16
FMM_OPT_M2L_BRICK = 17
FMM_BATCH_OPT_SWEEP, FMM_BATCH_OPT_WAIT_BUDGET_NS, FMM_BATCH_OPT_INJECT_STALL, FMM_BATCH_OPT_SWEEP_PAIRS = 1, 2, 3, 4
BOUNDARY = {"conducting": 0, "vacuum": 1}
PRECISION = {"fp64": 0, "mixed": 1}
SPLIT = {"bf16x3": 0, "bf16x2": 1, "fp32": 2, "bf16a2b3": 3, "fp16x2": 4}
STATUS = ["ok", "invalid argument", "non-finite input", "CUDA error", "out of memory", "timeout",
          "internal error", "unsupported"]


class FMMError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = STATUS[code] if 0 <= code < len(STATUS) else "status %d" % code
        super().__init__("%s: %s (status %d)" % (where, msg, code))


class EnergyTerms(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("near", "far", "charged", "quad_surface", "dipole_surface", "total")]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class UVTerms(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("e_uv", "W", "A", "B", "C", "nf_uv", "bc_cross", "nf_sc", "dnf_sc")]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TunePolicy(ctypes.Structure):
    _fields_ = [("energy_rel_tol", ctypes.c_double), ("sweep", ctypes.c_int), ("tiles", ctypes.c_int)]


class Timings(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("sort", "upward", "lattice", "m2l_l2l", "l2p", "p2p", "solute_pass",
                                              "reduce", "total", "m2l_kernels", "m2l_top")]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def load_library(path: str = LIB_PATH):
    """Load libfmm_gb300.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError("libfmm_gb300.so not found at %s: run paper_2003_13218_gb300/build.py "
                           "(or __graft_entry__.build()) first" % path)
    L = ctypes.CDLL(path)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.fmm_plan_create.argtypes = [dbl, i64, c_int, c_int, ctypes.POINTER(vp)]
    L.fmm_plan_create.restype = c_int
    L.fmm_plan_set_option.argtypes = [vp, c_int, i64, dbl]
    L.fmm_plan_set_option.restype = c_int
    L.fmm_energy.argtypes = [vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(EnergyTerms)]
    L.fmm_energy.restype = c_int
    L.fmm_forces.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl)]
    L.fmm_forces.restype = c_int
    L.fmm_potentials.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(dbl)]
    L.fmm_potentials.restype = c_int
    L.fmm_solute_solvent_energy.argtypes = [vp, vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(UVTerms)]
    L.fmm_solute_solvent_energy.restype = c_int
    L.fmm_evaluate.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(EnergyTerms), ctypes.POINTER(UVTerms)]
    L.fmm_evaluate.restype = c_int
    L.fmm_plan_get_timings.argtypes = [vp, ctypes.POINTER(Timings)]
    L.fmm_plan_get_timings.restype = c_int
    L.fmm_plan_last_launch_count.argtypes = [vp]
    L.fmm_plan_last_launch_count.restype = i64
    L.fmm_plan_m2l_backend.argtypes = [vp, c_int]
    L.fmm_plan_m2l_backend.restype = c_int
    L.fmm_plan_destroy.argtypes = [vp]
    L.fmm_plan_destroy.restype = None
    pp = ctypes.POINTER(vp)
    L.fmm_batch_create.argtypes = [c_int, vp, vp, vp, vp, c_int, ctypes.POINTER(vp)]
    L.fmm_batch_create.restype = c_int
    L.fmm_batch_create_tuned.argtypes = [c_int, vp, vp, vp, vp, c_int, ctypes.POINTER(TunePolicy), ctypes.POINTER(vp)]
    L.fmm_batch_create_tuned.restype = c_int
    L.fmm_batch_tune_info.argtypes = [vp, vp, ctypes.POINTER(c_int), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                      ctypes.POINTER(c_int)]
    L.fmm_batch_tune_info.restype = c_int
    L.fmm_batch_brick_info.argtypes = [vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                       ctypes.POINTER(c_int)]
    L.fmm_batch_brick_info.restype = c_int
    L.fmm_batch_lambda_energies.argtypes = [vp, pp, pp, pp, vp, vp, vp, vp, vp]
    L.fmm_batch_lambda_energies.restype = c_int
    L.fmm_batch_info.argtypes = [vp, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(i64),
                                 ctypes.POINTER(i64)]
    L.fmm_batch_info.restype = c_int
    L.fmm_batch_set_softcore.argtypes = [vp, c_int, dbl, dbl]
    L.fmm_batch_set_softcore.restype = c_int
    L.fmm_batch_set_graph.argtypes = [vp, c_int]
    L.fmm_batch_set_graph.restype = c_int
    L.fmm_batch_set_option.argtypes = [vp, c_int, i64, dbl]
    L.fmm_batch_set_option.restype = c_int
    L.fmm_batch_sweep_info.argtypes = [vp, ctypes.POINTER(c_int), vp]
    L.fmm_batch_sweep_info.restype = c_int
    L.fmm_batch_destroy.argtypes = [vp]
    L.fmm_batch_destroy.restype = None
    L.fmm_status_string.argtypes = [c_int]
    L.fmm_status_string.restype = ctypes.c_char_p
    _LIB = L
    return L


def _check(code, where):
    if code != 0:
        raise FMMError(code, where)


_KIND = {"f8": (torch.float64, np.dtype(np.float64)), "u1": (torch.uint8, np.dtype(np.uint8))}


def _ptr(x, count=None, kind="f8", name="array", out=False):
    """(pointer, keepalive) for a tensor (CUDA or CPU) or NumPy array; None stays None.

    The C ABI takes plain pointers and cannot check what they point to, so the checks are made here:
    `count` is the number of elements the call reads or writes (fewer is a ValueError), `kind` the
    element type ("f8" double, "u1" uint8).  An input of another element type or layout is converted
    (a copy that lives until the call returns); an output is written in place, so it must already be
    contiguous and of the right type."""
    if x is None:
        return None, None
    tdt, ndt = _KIND[kind]
    if isinstance(x, torch.Tensor):
        if out and (x.dtype != tdt or not x.is_contiguous()):
            raise ValueError(f"{name}: an output must be a contiguous {tdt} tensor (got {x.dtype}, "
                             f"contiguous={x.is_contiguous()})")
        if x.dtype != tdt:
            x = x.to(tdt)
        if not x.is_contiguous():
            x = x.contiguous()
        n, ptr = x.numel(), x.data_ptr()
    else:
        if out and not (isinstance(x, np.ndarray) and x.dtype == ndt and x.flags.c_contiguous and x.flags.writeable):
            raise ValueError(f"{name}: an output must be a writeable C-contiguous {ndt} array")
        x = np.ascontiguousarray(x, dtype=ndt)
        n, ptr = x.size, x.ctypes.data
    if count is not None and n < count:
        raise ValueError(f"{name}: {n} elements, the call {'writes' if out else 'reads'} {count}")
    return ctypes.c_void_p(ptr), x


def _batch_ptrs(xs, counts, kind, name):
    """Array of per-box device pointers for fmm_batch_lambda_energies.  The batch replays a recorded
    CUDA graph that holds these addresses, so nothing is converted: every entry must already be a
    contiguous CUDA tensor of the element type with at least counts[i] elements."""
    xs = list(xs)
    if len(xs) != len(counts):
        raise ValueError(f"{name}: {len(xs)} tensors for {len(counts)} boxes")
    tdt = _KIND[kind][0]
    for i, (x, c) in enumerate(zip(xs, counts)):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == tdt and x.is_contiguous()):
            raise ValueError(f"{name}[{i}]: must be a contiguous CUDA {tdt} tensor")
        if x.numel() < c:
            raise ValueError(f"{name}[{i}]: {x.numel()} elements, the box has {c}")
    return (ctypes.c_void_p * len(xs))(*[ctypes.c_void_p(x.data_ptr()) for x in xs]), xs


class FMMPlan:
    """A plan for N charges in a cubic box of side ``box`` (A), depth d, order p."""

    def __init__(self, box: float, N: int, depth: int, p: int, precision: str = "fp64", kappa: float | None = None,
                 split: str = "fp16x2", timings: bool = False, m2l_pair: bool = True, boundary: str = "conducting",
                 ws: int = 1, overlap: bool = True, m2l_grade: tuple[int, int] | None = None,
                 acc_group: int | None = None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.fmm_plan_create(float(box), int(N), int(depth), int(p), ctypes.byref(h)), "fmm_plan_create")
        self._h = h
        self.box, self.N, self.depth, self.p = float(box), int(N), int(depth), int(p)
        if ws != 1:
            self.set_option(FMM_OPT_WS, int(ws))
        if split != "fp16x2":
            self.set_option(FMM_OPT_M2L_SPLIT, SPLIT[split])
        if precision != "fp64":
            self.set_option(FMM_OPT_PRECISION, PRECISION[precision])
        if kappa is not None:
            self.set_option(FMM_OPT_KAPPA, 0, float(kappa))
        if timings:
            self.set_option(FMM_OPT_TIMINGS, 1)
        if not m2l_pair:
            self.set_option(FMM_OPT_M2L_PAIR, 0)
        if boundary != "conducting":
            self.set_option(FMM_OPT_BOUNDARY, BOUNDARY[boundary])
        if not overlap:
            self.set_option(FMM_OPT_OVERLAP, 0)
        if m2l_grade is not None:  # (D2, D1): degrees from which the fp16x2 M2L drops a product / two
            self.set_option(FMM_OPT_M2L_GRADE, int(m2l_grade[0]) | (int(m2l_grade[1]) << 8))
        if acc_group is not None:  # offsets per TMEM accumulator drain of the tensor-core M2L
            self.set_option(FMM_OPT_M2L_ACC_GROUP, int(acc_group))
        self.precision = precision

    def set_option(self, key: int, ival: int = 0, dval: float = 0.0):
        _check(self._lib.fmm_plan_set_option(self._h, int(key), int(ival), float(dval)), "fmm_plan_set_option")

    def set_brick(self, level: int, bx: int, by: int, bz: int):
        """Tile brick of the tensor-core M2L of a level (FMM_OPT_M2L_BRICK)."""
        self.set_option(FMM_OPT_M2L_BRICK, int(level) | (int(bx) << 8) | (int(by) << 16) | (int(bz) << 24))

    def set_softcore(self, c: int, A: float = 0.0, lam: float = 0.0, alpha: float = 0.2):
        """Soft-core solute-solvent near field (FMM_OPT_SOFTCORE): c = 0 turns it off."""
        self.set_option(FMM_OPT_SOFTCORE, int(c), float(A))
        if c > 0:
            self.set_option(FMM_OPT_SOFTCORE_ALPHA, 0, float(alpha))
            self.set_option(FMM_OPT_SOFTCORE_LAMBDA, 0, float(lam))

    def _bind_stream(self, *tensors):
        if any(isinstance(t, torch.Tensor) and t.is_cuda for t in tensors if t is not None):
            s = torch.cuda.current_stream().cuda_stream
            self._lib.fmm_plan_set_option(self._h, FMM_OPT_STREAM, int(s), 0.0)

    def evaluate(self, pos, q, is_solute=None, forces=None, want_terms=True):
        """fmm_evaluate: returns (terms dict or None, uv dict or None); fills ``forces`` if given."""
        self._bind_stream(pos, q, is_solute, forces)
        N = self.N
        pp, kp = _ptr(pos, 3 * N, "f8", "pos")
        pq, kq = _ptr(q, N, "f8", "q")
        ps, ks = _ptr(is_solute, N, "u1", "is_solute")
        pf, kf = _ptr(forces, 3 * N, "f8", "forces", out=True)
        t = EnergyTerms()
        u = UVTerms()
        _check(self._lib.fmm_evaluate(self._h, pp, pq, ps, pf, ctypes.byref(t) if want_terms else None,
                                      ctypes.byref(u) if is_solute is not None else None), "fmm_evaluate")
        return (t.asdict() if want_terms else None), (u.asdict() if is_solute is not None else None)

    def energy(self, pos, q):
        self._bind_stream(pos, q)
        pp, kp = _ptr(pos, 3 * self.N, "f8", "pos")
        pq, kq = _ptr(q, self.N, "f8", "q")
        e = ctypes.c_double()
        t = EnergyTerms()
        _check(self._lib.fmm_energy(self._h, pp, pq, ctypes.byref(e), ctypes.byref(t)), "fmm_energy")
        return e.value, t.asdict()

    def forces(self, pos, q, out=None, with_energy=True):
        if out is None:
            if isinstance(pos, torch.Tensor):
                out = torch.empty((self.N, 3), dtype=torch.float64, device=pos.device)
            else:
                out = np.empty((self.N, 3), dtype=np.float64)
        self._bind_stream(pos, q, out)
        pp, kp = _ptr(pos, 3 * self.N, "f8", "pos")
        pq, kq = _ptr(q, self.N, "f8", "q")
        pf, kf = _ptr(out, 3 * self.N, "f8", "out", out=True)
        e = ctypes.c_double()
        _check(self._lib.fmm_forces(self._h, pp, pq, pf, ctypes.byref(e) if with_energy else None), "fmm_forces")
        return out, (e.value if with_energy else None)

    def potentials(self, pos, q, out=None, forces=None, with_energy=True):
        """fmm_potentials: phi_i = dE/dq_i (and, if `forces` is given, the forces of the same evaluation)."""
        if out is None:
            if isinstance(pos, torch.Tensor):
                out = torch.empty((self.N,), dtype=torch.float64, device=pos.device)
            else:
                out = np.empty((self.N,), dtype=np.float64)
        self._bind_stream(pos, q, out, forces)
        pp, kp = _ptr(pos, 3 * self.N, "f8", "pos")
        pq, kq = _ptr(q, self.N, "f8", "q")
        po, ko = _ptr(out, self.N, "f8", "out", out=True)
        pf, kf = _ptr(forces, 3 * self.N, "f8", "forces", out=True)
        e = ctypes.c_double()
        _check(self._lib.fmm_potentials(self._h, pp, pq, po, pf, ctypes.byref(e) if with_energy else None),
               "fmm_potentials")
        return out, (e.value if with_energy else None)

    def solute_solvent_energy(self, pos, q, is_solute):
        self._bind_stream(pos, q, is_solute)
        pp, kp = _ptr(pos, 3 * self.N, "f8", "pos")
        pq, kq = _ptr(q, self.N, "f8", "q")
        ps, ks = _ptr(is_solute, self.N, "u1", "is_solute")
        e = ctypes.c_double()
        u = UVTerms()
        _check(self._lib.fmm_solute_solvent_energy(self._h, pp, pq, ps, ctypes.byref(e), ctypes.byref(u)),
               "fmm_solute_solvent_energy")
        return e.value, u.asdict()

    def timings(self):
        t = Timings()
        _check(self._lib.fmm_plan_get_timings(self._h, ctypes.byref(t)), "fmm_plan_get_timings")
        return t.asdict()

    def last_launch_count(self) -> int:
        return int(self._lib.fmm_plan_last_launch_count(self._h))

    def m2l_backend(self, level: int) -> str:
        code = int(self._lib.fmm_plan_m2l_backend(self._h, int(level)))
        return {0: "fp64-simt", 1: "fp32-simt", 2: "tcgen05"}.get(code, "invalid")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FMMBatch:
    """Independent boxes evaluated together (fmm_batch_*): per box the total energy, the
    solute-solvent interaction E_uv, V_lambda = E - lambda_C E_uv and dV/dlambda_C = -E_uv.

    Inputs are lists of CUDA tensors; keep the same tensors (updated in place) between
    calls so that the batch can replay its recorded CUDA graph."""

    def __init__(self, boxes, Ns, depths=None, ps=None, precision: str = "mixed", energy_rel_tol: float | None = None,
                 sweep: str | None = None, tiles: bool = False):
        """energy_rel_tol / sweep / tiles given: fmm_batch_create_tuned with that policy (sweep "auto", "on" or
        "off"; boxes with ps[i] < 0 or ps None then take the tuned order; tiles: time the deepest level's tile
        bricks); otherwise fmm_batch_create."""
        self._lib = load_library()
        n = len(boxes)
        self.n = n
        self._box = np.ascontiguousarray(boxes, np.float64)
        self._N = np.ascontiguousarray(Ns, np.int64)
        self._d = None if depths is None else np.ascontiguousarray(depths, np.int32)
        self._p = None if ps is None else np.ascontiguousarray(ps, np.int32)
        h = ctypes.c_void_p()
        args = (n, self._box.ctypes.data, self._N.ctypes.data, None if self._d is None else self._d.ctypes.data,
                None if self._p is None else self._p.ctypes.data, PRECISION[precision])
        if energy_rel_tol is None and sweep is None and not tiles:
            _check(self._lib.fmm_batch_create(*args, ctypes.byref(h)), "fmm_batch_create")
        else:
            pol = TunePolicy(float(energy_rel_tol or 0.0), {"auto": -1, "off": 0, "on": 1}[sweep or "on"],
                             1 if tiles else 0)
            _check(self._lib.fmm_batch_create_tuned(*args, ctypes.byref(pol), ctypes.byref(h)), "fmm_batch_create_tuned")
        self._h = h

    def lambda_energies(self, pos, q, is_solute, lambda_c=None):
        n = self.n
        Ns = [int(v) for v in self._N]
        P, kp = _batch_ptrs(pos, [3 * v for v in Ns], "f8", "pos")
        Q, kq = _batch_ptrs(q, Ns, "f8", "q")
        S, ks = _batch_ptrs(is_solute, Ns, "u1", "is_solute")
        lam = None if lambda_c is None else np.ascontiguousarray(lambda_c, np.float64)
        if lam is not None and lam.size < n:
            raise ValueError(f"lambda_c: {lam.size} values for {n} boxes")
        out = {k: np.zeros(n) for k in ("e_total", "e_uv", "v_lambda", "dv_dlambda")}
        _check(self._lib.fmm_batch_lambda_energies(self._h, P, Q, S, None if lam is None else lam.ctypes.data,
                                                   out["e_total"].ctypes.data, out["e_uv"].ctypes.data,
                                                   out["v_lambda"].ctypes.data, out["dv_dlambda"].ctypes.data),
               "fmm_batch_lambda_energies")
        return out

    def info(self, i: int):
        d, p = ctypes.c_int(), ctypes.c_int()
        r, e = ctypes.c_int64(), ctypes.c_int64()
        _check(self._lib.fmm_batch_info(self._h, i, ctypes.byref(d), ctypes.byref(p), ctypes.byref(r),
                                        ctypes.byref(e)), "fmm_batch_info")
        return {"depth": d.value, "p": p.value, "replays": r.value, "enqueued": e.value}

    def tune_info(self):
        """What the tuner measured: energy errors of p = 6, 8, 10, 12 against p = 15, the order chosen, the graph
        replay times with the sweep off / on, and whether the sweep is in use."""
        err = np.zeros(4)
        pc, on = ctypes.c_int(), ctypes.c_int()
        t0, t1 = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.fmm_batch_tune_info(self._h, err.ctypes.data, ctypes.byref(pc), ctypes.byref(t0),
                                             ctypes.byref(t1), ctypes.byref(on)), "fmm_batch_tune_info")
        return {"p_err": {6: err[0], 8: err[1], 10: err[2], 12: err[3]}, "p_chosen": pc.value,
                "ms_sweep_off": t0.value, "ms_sweep_on": t1.value, "sweep_on": bool(on.value)}

    def brick(self, i: int):
        """The deepest level of box i and its tile brick (bx, by, bz)."""
        l, x, y, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.fmm_batch_brick_info(self._h, i, ctypes.byref(l), ctypes.byref(x), ctypes.byref(y),
                                              ctypes.byref(z)), "fmm_batch_brick_info")
        return l.value, (x.value, y.value, z.value)

    def set_softcore(self, c: int, A: float = 0.0, alpha: float = 0.2):
        _check(self._lib.fmm_batch_set_softcore(self._h, int(c), float(A), float(alpha)), "fmm_batch_set_softcore")

    def set_graph(self, enable: bool):
        _check(self._lib.fmm_batch_set_graph(self._h, 1 if enable else 0), "fmm_batch_set_graph")

    def set_option(self, key: int, ival: int, dval: float = 0.0):
        _check(self._lib.fmm_batch_set_option(self._h, int(key), int(ival), float(dval)), "fmm_batch_set_option")

    def set_sweep(self, enable: bool):
        self.set_option(FMM_BATCH_OPT_SWEEP, 1 if enable else 0)

    def sweep_info(self):
        """Boxes in the persistent sweep and each box's first sweep level (0: not in it)."""
        nb = ctypes.c_int()
        first = np.zeros(self.n, np.int32)
        _check(self._lib.fmm_batch_sweep_info(self._h, ctypes.byref(nb), first.ctypes.data), "fmm_batch_sweep_info")
        return {"boxes": nb.value, "first_level": first.tolist()}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FmmEnergy(torch.autograd.Function):
    """E = V_elec(pos, q) with the hand-written adjoint: dE/dpos = -F (fmm_forces) and, when q needs a
    gradient, dE/dq = phi (fmm_potentials, from the same evaluation)."""

    @staticmethod
    def forward(ctx, pos, q, plan: FMMPlan):
        if ctx.needs_input_grad[1]:
            F = torch.empty((plan.N, 3), dtype=torch.float64, device=pos.device)
            phi, e = plan.potentials(pos.detach(), q.detach(), forces=F)
        else:
            F, e = plan.forces(pos.detach(), q.detach())
            phi = None
        ctx.save_for_backward(F, phi)
        return torch.tensor(e, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, grad_e):
        F, phi = ctx.saved_tensors
        return -F * grad_e, (phi * grad_e if phi is not None else None), None
