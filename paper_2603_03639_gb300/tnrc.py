"""Python binding of the tnrc C ABI (``include/tnrc.h``): argument marshalling
only.  Every step of the evaluation runs in the CUDA library
``lib/libtnrc.so``; there is no fallback, so a missing library is an error."""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TNRC_LIB") or os.path.join(_HERE, "lib", "libtnrc.so")

TNRC_OK = 0
STATUS_NAMES = {0: "TNRC_OK", -1: "TNRC_E_INVALID", -2: "TNRC_E_NOMEM", -3: "TNRC_E_CUDA",
                -4: "TNRC_E_STATE", -5: "TNRC_E_TIMEOUT", -6: "TNRC_E_NUMERIC", -7: "TNRC_E_TOO_LARGE"}

#: every symbol the header declares
EXPORTS = ("tnrc_create", "tnrc_set_controls", "tnrc_sample_noise", "tnrc_set_noise", "tnrc_get_noise",
           "tnrc_fidelity",
           "tnrc_fidelity_grad", "tnrc_get_overlaps", "tnrc_get_stats", "tnrc_set_controls_dev",
           "tnrc_evaluate_dev", "tnrc_sync", "tnrc_footprint", "tnrc_destroy", "tnrc_status_string",
           "tnrc_fidelity_static", "tnrc_set_graphs", "tnrc_last_error", "tnrc_measure_fp64_peak",
           "tnrc_measure_dmma_peak", "tnrc_set_pooled", "tnrc_set_stream", "tnrc_fidelity_grad_plain",
           "tnrc_set_svd_shape")


class TNRCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__("%s failed: %s%s" % (where, _status_string(status), (" (%s)" % detail) if detail else ""))


class Problem(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("n_sites", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("dt", ctypes.c_double), ("chi_max", ctypes.c_int32), ("sv_cutoff", ctypes.c_double),
                ("n_samples", ctypes.c_int32), ("n_controls", ctypes.c_int32), ("n_inputs", ctypes.c_int32),
                ("control_mask", ctypes.POINTER(ctypes.c_uint8)), ("g_fixed", ctypes.POINTER(ctypes.c_double)),
                ("checkpoint_every", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("crosstalk_terms", ctypes.c_int32),
                ("trotter_order", ctypes.c_int32), ("substeps", ctypes.c_int32),
                ("operator_form", ctypes.c_int32)]


class MPSDesc(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("bond_dims", ctypes.POINTER(ctypes.c_int32)),
                ("data", ctypes.POINTER(ctypes.c_double))]


class Stats(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("jacobi_sweeps", ctypes.c_int64), ("max_bond", ctypes.c_int32),
                ("hist_len", ctypes.c_int32), ("bond_hist", ctypes.c_int64 * 65),
                ("discarded_weight", ctypes.c_double), ("last_ms", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("traj_ms", ctypes.c_double), ("traj_launches", ctypes.c_int64),
                ("restarts", ctypes.c_int64), ("phase_cycles", ctypes.c_int64 * 9),
                ("cap_truncations", ctypes.c_int64), ("min_trunc_gap", ctypes.c_double)]


#: trajectory-kernel phases of tnrc_stats.phase_cycles
PHASES = ("contraction", "qr", "truncate", "split", "environments", "gradients", "history", "barriers",
          "jacobi")

_LIB = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("tnrc CUDA library not built (%s missing): run "
                               "paper_2603_03639_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.tnrc_create.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(MPSDesc), ctypes.POINTER(MPSDesc), vp,
                                  ctypes.POINTER(vp)]
        L.tnrc_set_controls.argtypes = [vp, dp, i64]
        L.tnrc_sample_noise.argtypes = [vp, ctypes.c_uint64, i32, ctypes.c_double]
        L.tnrc_set_noise.argtypes = [vp, dp, i64]
        L.tnrc_get_noise.argtypes = [vp, dp, i64]
        L.tnrc_fidelity.argtypes = [vp, dp, dp]
        L.tnrc_fidelity_grad.argtypes = [vp, dp, dp]
        L.tnrc_get_overlaps.argtypes = [vp, dp, i64]
        L.tnrc_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.tnrc_set_controls_dev.argtypes = [vp, vp]
        L.tnrc_evaluate_dev.argtypes = [vp, vp, vp, vp]
        L.tnrc_sync.argtypes = [vp]
        L.tnrc_measure_fp64_peak.argtypes = [vp, ctypes.c_size_t, dp]
        L.tnrc_measure_fp64_peak.restype = i32
        L.tnrc_measure_dmma_peak.argtypes = [vp, ctypes.c_size_t, dp]
        L.tnrc_measure_dmma_peak.restype = i32
        L.tnrc_last_error.argtypes = [vp]
        L.tnrc_last_error.restype = ctypes.c_char_p
        L.tnrc_set_graphs.argtypes = [vp, i32]
        L.tnrc_set_graphs.restype = i32
        L.tnrc_set_pooled.argtypes = [vp, i32]
        L.tnrc_set_pooled.restype = i32
        L.tnrc_set_stream.argtypes = [vp, vp]
        L.tnrc_set_stream.restype = i32
        L.tnrc_fidelity_grad_plain.argtypes = [vp, dp, dp]
        L.tnrc_fidelity_grad_plain.restype = i32
        L.tnrc_set_svd_shape.argtypes = [vp, i32]
        L.tnrc_set_svd_shape.restype = i32
        L.tnrc_footprint.argtypes = [ctypes.POINTER(Problem)]
        L.tnrc_footprint.restype = ctypes.c_size_t
        L.tnrc_destroy.argtypes = [vp]
        L.tnrc_destroy.restype = None
        L.tnrc_fidelity_static.argtypes = [ctypes.POINTER(Problem), ctypes.POINTER(MPSDesc),
                                           ctypes.POINTER(MPSDesc), dp, dp, vp, dp, dp]
        L.tnrc_fidelity_static.restype = i32
        L.tnrc_status_string.argtypes = [i32]
        L.tnrc_status_string.restype = ctypes.c_char_p
        for name in ("tnrc_create", "tnrc_set_controls", "tnrc_sample_noise", "tnrc_set_noise", "tnrc_get_noise",
                     "tnrc_fidelity",
                     "tnrc_fidelity_grad", "tnrc_get_overlaps", "tnrc_get_stats", "tnrc_set_controls_dev",
                     "tnrc_evaluate_dev", "tnrc_sync"):
            getattr(L, name).restype = i32
        _LIB = L
    return _LIB


def _status_string(s: int) -> str:
    try:
        return lib().tnrc_status_string(s).decode()
    except Exception:
        return STATUS_NAMES.get(s, str(s))


def _check(s: int, where: str, handle=None):
    if s != TNRC_OK:
        detail = ""
        if s == -3 and handle is not None and handle.value:
            detail = lib().tnrc_last_error(handle).decode(errors="replace")
        raise TNRCError(s, where, detail)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pack(state):
    """(bond_dims int32, data float64 interleaved) from an object with
    ``pack()`` or a (bond_dims, complex data) pair."""
    dims, data = state.pack() if hasattr(state, "pack") else state
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    data = np.ascontiguousarray(np.asarray(data, dtype=np.complex128)).view(np.float64)
    return dims, data


def make_problem(N, K, dt, chi, M, C, P, cutoff=1e-12, mask=None, g_fixed=None, checkpoint_every=0, warps=0,
                 ctas_per_sm=0, crosstalk=1, order=2, substeps=1, operator=False):
    """A ``Problem`` plus the arrays it points to (keep both alive)."""
    keep = []
    pb = Problem()
    pb.struct_size = ctypes.sizeof(Problem)
    pb.n_sites, pb.n_slices, pb.dt, pb.chi_max, pb.sv_cutoff = N, K, dt, chi, cutoff
    pb.n_samples, pb.n_controls, pb.n_inputs = M, C, P
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        keep.append(m)
        pb.control_mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if g_fixed is not None:
        g = np.ascontiguousarray(g_fixed, dtype=np.float64)
        keep.append(g)
        pb.g_fixed = _dp(g)
    pb.checkpoint_every = checkpoint_every
    pb.warps_per_cta = warps
    pb.ctas_per_sm = ctas_per_sm
    pb.crosstalk_terms = crosstalk
    pb.trotter_order = order
    pb.substeps = substeps
    pb.operator_form = 1 if operator else 0
    return pb, keep


def _descs(states):
    packs = [_pack(s) for s in states]
    descs = (MPSDesc * len(packs))()
    for d, (dims, data) in zip(descs, packs):
        d.n_sites = len(dims) - 1
        d.bond_dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.data = _dp(data)
    return descs, packs


def fidelity_static(N, K, dt, chi, C, inputs, targets, u, J, cutoff=1e-12, mask=None, g_fixed=None,
                    stream=None, per_traj=False, crosstalk=1, order=2, substeps=1, operator=False):
    """F (and per-trajectory |O|^2) through tnrc_fidelity_static, which
    allocates no device memory: for callers that cannot call cudaMalloc.
    Calls must not overlap on the GPU (they share one static array)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    M, P = J.shape[0], len(inputs)
    pb, keep = make_problem(N, K, dt, chi, M, C, P, cutoff, mask, g_fixed, crosstalk=crosstalk, order=order,
                            substeps=substeps, operator=operator)
    ins, kin = _descs(inputs)
    tgs, ktg = _descs(targets)
    F = np.zeros(1)
    pt = np.zeros(M * P) if per_traj else None
    _check(lib().tnrc_fidelity_static(ctypes.byref(pb), ins, tgs, _dp(u), _dp(J), ctypes.c_void_p(stream or 0),
                                      _dp(F), _dp(pt) if pt is not None else None), "tnrc_fidelity_static")
    return (F[0], pt.reshape(M, P)) if per_traj else F[0]


def measure_fp64_peak(scratch_ptr: int, scratch_bytes: int) -> float:
    """FP64 FMA throughput of the current device in GFLOP/s (see the header)."""
    g = np.zeros(1)
    _check(lib().tnrc_measure_fp64_peak(ctypes.c_void_p(scratch_ptr), scratch_bytes, _dp(g)),
           "tnrc_measure_fp64_peak")
    return float(g[0])


def measure_dmma_peak(scratch_ptr: int, scratch_bytes: int) -> float:
    """FP64 tensor-core (DMMA) throughput of the current device in GFLOP/s."""
    g = np.zeros(1)
    _check(lib().tnrc_measure_dmma_peak(ctypes.c_void_p(scratch_ptr), scratch_bytes, _dp(g)),
           "tnrc_measure_dmma_peak")
    return float(g[0])


def footprint(N, K, dt, chi, M, C, P, **kw) -> int:
    pb, _keep = make_problem(N, K, dt, chi, M, C, P, **kw)
    return int(lib().tnrc_footprint(ctypes.byref(pb)))


class Context:
    """One tnrc context: problem, canonical inputs/targets, device arena."""

    def __init__(self, N: int, K: int, dt: float, chi: int, M: int, C: int, inputs: Sequence, targets: Sequence,
                 cutoff: float = 1e-12, mask=None, g_fixed=None, checkpoint_every: int = 0,
                 stream: Optional[int] = None, warps: int = 0, ctas_per_sm: int = 0, crosstalk: int = 1,
                 order: int = 2, substeps: int = 1, operator: bool = False):
        L = lib()
        self.N, self.K, self.C, self.M, self.P = N, K, C, M, len(inputs)
        self.stream = int(stream or 0)
        self.terms = 3 if crosstalk == 3 else 1
        if len(targets) != self.P:
            raise ValueError("inputs and targets differ in length")
        pb, keep = make_problem(N, K, dt, chi, M, C, self.P, cutoff, mask, g_fixed, checkpoint_every, warps,
                                ctas_per_sm, crosstalk, order, substeps, operator)
        packs = [_pack(s) for s in list(inputs) + list(targets)]
        descs = (MPSDesc * len(packs))()
        for d, (dims, data) in zip(descs, packs):
            d.n_sites = len(dims) - 1
            d.bond_dims = dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.data = _dp(data)
        ins = ctypes.cast(ctypes.byref(descs, 0), ctypes.POINTER(MPSDesc))
        tgs = ctypes.cast(ctypes.byref(descs, ctypes.sizeof(MPSDesc) * self.P), ctypes.POINTER(MPSDesc))
        h = ctypes.c_void_p()
        _check(L.tnrc_create(ctypes.byref(pb), ins, tgs, ctypes.c_void_p(stream or 0), ctypes.byref(h)),
               "tnrc_create")
        del keep, packs
        self._h = h

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().tnrc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- inputs --
    def set_controls(self, u: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().tnrc_set_controls(self._h, _dp(u), u.size), "tnrc_set_controls", self._h)

    def set_controls_dev(self, ptr: int):
        _check(lib().tnrc_set_controls_dev(self._h, ctypes.c_void_p(ptr)), "tnrc_set_controls_dev", self._h)

    def sample_noise(self, seed: int, dist: int, scale: float):
        _check(lib().tnrc_sample_noise(self._h, ctypes.c_uint64(seed), dist, scale), "tnrc_sample_noise", self._h)

    def set_noise(self, J: np.ndarray):
        J = np.ascontiguousarray(J, dtype=np.float64)
        _check(lib().tnrc_set_noise(self._h, _dp(J), J.size), "tnrc_set_noise", self._h)

    def get_noise(self) -> np.ndarray:
        J = np.zeros((self.M, self.N - 1) if self.terms == 1 else (self.M, self.N - 1, 3))
        _check(lib().tnrc_get_noise(self._h, _dp(J), J.size), "tnrc_get_noise", self._h)
        return J

    # -- evaluations --
    def fidelity(self, per_traj: bool = False):
        F = np.zeros(1)
        pt = np.zeros(self.M * self.P) if per_traj else None
        _check(lib().tnrc_fidelity(self._h, _dp(F), _dp(pt) if pt is not None else None), "tnrc_fidelity", self._h)
        return (F[0], pt.reshape(self.M, self.P)) if per_traj else F[0]

    def fidelity_grad(self):
        F = np.zeros(1)
        g = np.zeros((self.K, self.C, self.N))
        _check(lib().tnrc_fidelity_grad(self._h, _dp(F), _dp(g)), "tnrc_fidelity_grad", self._h)
        return F[0], g

    def fidelity_grad_plain(self):
        """F and dF/du by the plain one-trajectory-at-a-time GPU path."""
        F = np.zeros(1)
        g = np.zeros((self.K, self.C, self.N))
        _check(lib().tnrc_fidelity_grad_plain(self._h, _dp(F), _dp(g)), "tnrc_fidelity_grad_plain", self._h)
        return F[0], g

    def overlaps(self) -> np.ndarray:
        o = np.zeros(2 * self.M * self.P)
        _check(lib().tnrc_get_overlaps(self._h, _dp(o), o.size), "tnrc_get_overlaps", self._h)
        return o.view(np.complex128).reshape(self.M, self.P)

    def evaluate_dev(self, F_ptr: int, grad_ptr: int = 0, per_traj_ptr: int = 0):
        _check(lib().tnrc_evaluate_dev(self._h, ctypes.c_void_p(F_ptr), ctypes.c_void_p(grad_ptr or None),
                                       ctypes.c_void_p(per_traj_ptr or None)), "tnrc_evaluate_dev", self._h)

    def set_graphs(self, enable: bool = True):
        _check(lib().tnrc_set_graphs(self._h, 1 if enable else 0), "tnrc_set_graphs", self._h)

    def set_stream(self, stream: int):
        """Order later work on another CUDA stream (waits for queued work)."""
        _check(lib().tnrc_set_stream(self._h, ctypes.c_void_p(stream or None)), "tnrc_set_stream", self._h)
        self.stream = int(stream or 0)

    def set_svd_shape(self, pairs: bool = True):
        """Two small SVDs per warp on the half-warps (True) or one per warp."""
        _check(lib().tnrc_set_svd_shape(self._h, 1 if pairs else 0), "tnrc_set_svd_shape", self._h)

    def set_pooled(self, enable: bool = True):
        """One CTA per trajectory with work regions from a pool (see the header)."""
        _check(lib().tnrc_set_pooled(self._h, 1 if enable else 0), "tnrc_set_pooled", self._h)

    def sync(self):
        _check(lib().tnrc_sync(self._h), "tnrc_sync", self._h)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().tnrc_get_stats(self._h, ctypes.byref(s)), "tnrc_get_stats", self._h)
        return {"updates": s.updates, "jacobi_sweeps": s.jacobi_sweeps, "max_bond": s.max_bond,
                "bond_hist": [int(s.bond_hist[i]) for i in range(s.hist_len)],
                "discarded_weight": s.discarded_weight, "last_ms": s.last_ms, "alg_flops": s.alg_flops,
                "traj_ms": s.traj_ms, "traj_launches": s.traj_launches, "restarts": s.restarts,
                "phase_cycles": dict(zip(PHASES, (int(x) for x in s.phase_cycles))),
                "cap_truncations": int(s.cap_truncations), "min_trunc_gap": float(s.min_trunc_gap)}
