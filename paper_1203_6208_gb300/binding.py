"""Thin ctypes binding of libbdgb (C ABI in include/bd.h).

Argument marshalling only: every step of the Brownian-dynamics path runs in
the CUDA library.  Tensors are torch CUDA tensors (torch supplies device
memory and the current stream); the library sees plain pointers.

Layouts (see include/bd.h): positions R are (N, 3) float64; a block of m
3N-vectors is an (m, 3N) float64 tensor (row j = column j of the 3N x m
column-major block); D is a raw byte buffer of ``info.d_bytes``.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbdgb.so")

BD_OK = 0
STATUS_NAMES = {0: "BD_OK", 1: "BD_ERR_INVALID", 2: "BD_ERR_OOM", 3: "BD_ERR_CUDA",
                4: "BD_ERR_NOT_PD", 5: "BD_ERR_FENE_STRETCH", 6: "BD_ERR_CHEB_NOCONV",
                7: "BD_ERR_TIMEOUT", 8: "BD_ERR_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "mixed_f16": 1, "mixed_bf16": 2}
BD_APPLY_REFINE = 1
BD_STEP_DEVICE_COUNTER = 1
BD_STEP_MATRIX_FREE = 2
BD_SHAPE_SYMMETRIC = 3
BD_SHAPE_F64_DOUBLE_FLOAT = 4
BOUNDS_MODES = {"fresh": 0, "lagged": 1, "fixman_dilute": 2, "fixman_semidilute": 3}

EXPORTS = ["bd_plan_create", "bd_plan_destroy", "bd_plan_query", "bd_forces", "bd_build_D",
           "bd_apply_D", "bd_eig_bounds", "bd_chebyshev_sqrt", "bd_step", "bd_wiener",
           "bd_set_phase_events", "bd_kernel_launches", "bd_eig_bounds_noalloc",
           "bd_apply_D_backward", "bd_chebyshev_backward", "bd_plan_autotune", "bd_plan_set_shape",
           "bd_plan_test_stall", "bd_step_capture", "bd_step_replay", "bd_product_timing",
           "bd_plan_set_step_counter", "bd_batch_create", "bd_batch_destroy", "bd_batch_query",
           "bd_batch_step", "bd_chebyshev_sqrt_adaptive", "bd_apply_D_matfree",
           "bd_mesh_fft", "bd_last_error", "bd_version"]
PHASES = ["forces", "build_D", "bounds", "first_product", "chebyshev", "update"]


class BdParams(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int32), ("beads_per_chain", ctypes.c_int32),
                ("box_L", ctypes.c_double), ("a", ctypes.c_double),
                ("alpha", ctypes.c_double), ("r_c", ctypes.c_double),
                ("n2max", ctypes.c_int32), ("overlap_corr", ctypes.c_int32),
                ("spring", ctypes.c_int32), ("fene_b", ctypes.c_double),
                ("ev_on", ctypes.c_int32), ("z_star", ctypes.c_double),
                ("d_star", ctypes.c_double), ("r_ev", ctypes.c_double),
                ("dt", ctypes.c_double), ("precision", ctypes.c_int32),
                ("max_rhs", ctypes.c_int32), ("max_cheb", ctypes.c_int32),
                ("pme_grid", ctypes.c_int32), ("pme_order", ctypes.c_int32)]


class BdPlanInfo(ctypes.Structure):
    _fields_ = [("n3", ctypes.c_int32), ("ld", ctypes.c_int32), ("d_bytes", ctypes.c_int64),
                ("n_kvec", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64)]


class BdStepStats(ctypes.Structure):
    _fields_ = [("d_min", ctypes.c_double), ("d_max", ctypes.c_double),
                ("ef_max", ctypes.c_double), ("n_cheb", ctypes.c_int32),
                ("n_overstretched", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class BdStepOpts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n_cheb", ctypes.c_int32),
                ("lanczos_iters", ctypes.c_int32), ("bound_safety", ctypes.c_double),
                ("dmin_fraction", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("step_index", ctypes.c_uint64), ("bounds_mode", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("ef_tol", ctypes.c_double),
                ("fixman_c", ctypes.c_double)]


STATS_BYTES = ctypes.sizeof(BdStepStats)

_lib = None
_vp = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load libbdgb.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_1203_6208_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(path)
    i32, f64, u64, i64 = ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
    L.bd_plan_create.argtypes = [ctypes.POINTER(BdParams), ctypes.POINTER(_vp)]
    L.bd_plan_destroy.argtypes = [_vp]
    L.bd_plan_destroy.restype = None
    L.bd_plan_query.argtypes = [_vp, ctypes.POINTER(BdPlanInfo)]
    L.bd_forces.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.bd_build_D.argtypes = [_vp, _vp, _vp, _vp]
    L.bd_apply_D.argtypes = [_vp, _vp, _vp, i32, _vp, i32, _vp]
    L.bd_eig_bounds.argtypes = [_vp, _vp, i32, f64, f64, _vp, _vp, _vp]
    L.bd_chebyshev_sqrt.argtypes = [_vp, _vp, _vp, i32, _vp, i32, _vp, _vp, _vp]
    L.bd_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(BdStepOpts), _vp, _vp, _vp, _vp]
    L.bd_step_capture.argtypes = [_vp, _vp, _vp, ctypes.POINTER(BdStepOpts), _vp, _vp, _vp, _vp]
    L.bd_step_replay.argtypes = [_vp, _vp]
    L.bd_wiener.argtypes = [_vp, u64, u64, i64, _vp, _vp]
    L.bd_set_phase_events.argtypes = [_vp, ctypes.POINTER(_vp), i32]
    L.bd_apply_D_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.bd_plan_set_shape.argtypes = [_vp, i32]
    L.bd_plan_set_shape.restype = i32
    L.bd_plan_test_stall.argtypes = [_vp, i32, i32]
    L.bd_plan_autotune.argtypes = [_vp, _vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                                   _vp]
    L.bd_plan_set_step_counter.argtypes = [_vp, u64, _vp]
    L.bd_product_timing.argtypes = [_vp, i32, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
    L.bd_batch_create.argtypes = [ctypes.POINTER(BdParams), i32, ctypes.POINTER(_vp)]
    L.bd_batch_destroy.argtypes = [_vp]
    L.bd_batch_destroy.restype = None
    L.bd_batch_query.argtypes = [_vp, i32, ctypes.POINTER(BdPlanInfo), ctypes.POINTER(i64),
                                 ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.bd_batch_step.argtypes = [_vp, _vp, _vp, ctypes.POINTER(BdStepOpts), _vp, _vp]
    L.bd_chebyshev_backward.argtypes = [_vp, _vp, _vp, _vp, i32, _vp, i32, _vp, _vp, _vp, _vp]
    L.bd_apply_D_matfree.argtypes = [_vp, _vp, _vp, i32, _vp, _vp]
    L.bd_mesh_fft.argtypes = [i32, i32, i32, i32, _vp, _vp, _vp]
    L.bd_chebyshev_sqrt_adaptive.argtypes = [_vp, _vp, _vp, f64, _vp, i32, _vp, _vp,
                                             ctypes.POINTER(i32), _vp]
    L.bd_eig_bounds_noalloc.argtypes = [_vp, i32, i32, i32, f64, f64, _vp, _vp, _vp]
    L.bd_kernel_launches.restype = ctypes.c_uint64
    L.bd_last_error.restype = ctypes.c_char_p
    L.bd_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("bd_plan_destroy", "bd_last_error", "bd_version", "bd_kernel_launches",
                        "bd_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class BDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int):
    if st != BD_OK:
        raise BDError(st, load().bd_last_error().decode())


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_params(p: dict, precision: str = "fp64", max_rhs: int = 16,
                max_cheb: int = 64) -> BdParams:
    return BdParams(n_beads=int(p["n"]), beads_per_chain=int(p["nb"]), box_L=float(p["L"]),
                    a=float(p["a"]), alpha=float(p["alpha"]), r_c=float(p["rc"]),
                    n2max=int(p["n2max"]), overlap_corr=int(p.get("overlap_corr", 1)),
                    spring=int(p.get("spring", 0)), fene_b=float(p.get("fene_b", 0.0)),
                    ev_on=int(p.get("ev_on", 0)), z_star=float(p.get("z_star", 0.0)),
                    d_star=float(p.get("d_star", 1.0)), r_ev=float(p.get("r_ev", 0.0)),
                    dt=float(p.get("dt", 0.0)), precision=PRECISIONS[precision],
                    max_rhs=int(max_rhs), max_cheb=int(max_cheb),
                    pme_grid=int(p.get("pme_grid", 0)), pme_order=int(p.get("pme_order", 0)))


class Plan:
    """One bd_plan on the current CUDA device."""

    def __init__(self, p: dict, precision: str = "fp64", max_rhs: int = 16, max_cheb: int = 64):
        L = load()
        self.params = dict(p)
        self.precision = precision
        self._c_params = make_params(p, precision, max_rhs, max_cheb)
        h = _vp()
        _check(L.bd_plan_create(ctypes.byref(self._c_params), ctypes.byref(h)))
        self._h = h
        info = BdPlanInfo()
        _check(L.bd_plan_query(h, ctypes.byref(info)))
        self.info = info
        self.n3, self.ld = info.n3, info.ld

    def close(self):
        if getattr(self, "_h", None):
            load().bd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers ------------------------------------------------------------
    def alloc_D(self) -> torch.Tensor:
        return torch.empty(self.info.d_bytes, dtype=torch.uint8, device="cuda")

    def D_view(self, D: torch.Tensor, which: str = "main") -> torch.Tensor:
        """(3N, 3N) view of the matrix stored in D (FP64, FP32 or 16-bit)."""
        n3, ld = self.n3, self.ld
        if self.precision == "fp64":
            return D.view(torch.float64).view(n3, ld)[:, :n3]
        if which in ("main", "f32"):
            return D[: n3 * ld * 4].view(torch.float32).view(n3, ld)[:, :n3]
        dt = torch.bfloat16 if self.precision == "mixed_bf16" else torch.float16
        return D[n3 * ld * 4:].view(dt).view(n3, ld)[:, :n3]

    # -- entry points ---------------------------------------------------------
    def forces(self, R, F, n_bad=None, stream=None):
        _check(load().bd_forces(self._h, _p(R), _p(F), _p(n_bad), _stream(stream)))

    def build_D(self, R, D, stream=None):
        _check(load().bd_build_D(self._h, _p(R), _p(D), _stream(stream)))

    def apply(self, D, X, Y, refine: bool = False, stream=None):
        m = X.shape[0] if X.dim() == 2 else 1
        _check(load().bd_apply_D(self._h, _p(D), _p(X), m, _p(Y),
                                 BD_APPLY_REFINE if refine else 0, _stream(stream)))

    def eig_bounds(self, D, iters, safety_max, dmin_fraction, bounds, status=None, stream=None):
        _check(load().bd_eig_bounds(self._h, _p(D), int(iters), float(safety_max),
                                    float(dmin_fraction), _p(bounds), _p(status), _stream(stream)))

    def chebyshev(self, D, bounds, n_cheb, dW, dS, Ef=None, stream=None):
        m = dW.shape[0] if dW.dim() == 2 else 1
        _check(load().bd_chebyshev_sqrt(self._h, _p(D), _p(bounds), int(n_cheb), _p(dW), m,
                                        _p(dS), _p(Ef), _stream(stream)))

    def apply_matfree(self, R, X, Y, stream=None):
        """Y = D(R) X without storing D (matrix-free product)."""
        m = X.shape[0] if X.dim() == 2 else 1
        _check(load().bd_apply_D_matfree(self._h, _p(R), _p(X), m, _p(Y), _stream(stream)))

    def chebyshev_adaptive(self, D, bounds, ef_tol, dW, dS, Ef=None, stream=None):
        """Adaptive N_Ch (synchronising); returns (n_used, converged)."""
        m = dW.shape[0] if dW.dim() == 2 else 1
        n = ctypes.c_int32()
        st = load().bd_chebyshev_sqrt_adaptive(self._h, _p(D), _p(bounds), float(ef_tol), _p(dW),
                                               m, _p(dS), _p(Ef), ctypes.byref(n),
                                               _stream(stream))
        if st == 6:                     # BD_ERR_CHEB_NOCONV: outputs hold max_cheb terms
            return int(n.value), False
        _check(st)
        return int(n.value), True

    def step(self, R, D, dW=None, *, m=1, n_cheb=20, lanczos_iters=30, bound_safety=0.05,
             dmin_fraction=0.5, seed=0, step_index=0, DF=None, dS=None, stats=None,
             bounds_mode=0, flags=0, ef_tol=0.0, fixman_c=0.0, stream=None):
        """n_cheb = 0 selects the adaptive series with ef_tol (synchronising);
        bounds_mode 2/3 = Fixman's dilute / semidilute estimates (fixman_c = C)."""
        o = BdStepOpts(m=int(m), n_cheb=int(n_cheb), lanczos_iters=int(lanczos_iters),
                       bound_safety=float(bound_safety), dmin_fraction=float(dmin_fraction),
                       seed=int(seed), step_index=int(step_index), bounds_mode=int(bounds_mode),
                       flags=int(flags), ef_tol=float(ef_tol), fixman_c=float(fixman_c))
        _check(load().bd_step(self._h, _p(R), _p(D), _p(dW), ctypes.byref(o), _p(DF), _p(dS),
                              _p(stats), _stream(stream)))

    def step_capture(self, R, D, *, m=1, n_cheb=20, lanczos_iters=30, bound_safety=0.05,
                     dmin_fraction=0.5, seed=0, DF=None, dS=None, stats=None, bounds_mode=0,
                     flags=0, fixman_c=0.0, stream=None):
        """bd_step_capture: record one step (noise from the device step counter)
        as a CUDA graph kept by the plan; replay it with step_replay."""
        o = BdStepOpts(m=int(m), n_cheb=int(n_cheb), lanczos_iters=int(lanczos_iters),
                       bound_safety=float(bound_safety), dmin_fraction=float(dmin_fraction),
                       seed=int(seed), step_index=0, bounds_mode=int(bounds_mode),
                       flags=int(flags), ef_tol=0.0, fixman_c=float(fixman_c))
        _check(load().bd_step_capture(self._h, _p(R), _p(D), ctypes.byref(o), _p(DF), _p(dS),
                                      _p(stats), _stream(stream)))

    def step_replay(self, stream=None):
        _check(load().bd_step_replay(self._h, _stream(stream)))

    def apply_backward(self, R, D, F, gY, gR, gF=None, stream=None):
        _check(load().bd_apply_D_backward(self._h, _p(R), _p(D), _p(F), _p(gY), _p(gR), _p(gF),
                                          _stream(stream)))

    def chebyshev_backward(self, R, D, bounds, n_cheb, dW, gS, gR, gdW=None, stream=None):
        m = dW.shape[0] if dW.dim() == 2 else 1
        _check(load().bd_chebyshev_backward(self._h, _p(R), _p(D), _p(bounds), int(n_cheb),
                                            _p(dW), m, _p(gS), _p(gR), _p(gdW), _stream(stream)))

    def product_timing(self, enable: bool):
        """enable=True starts recording; enable=False returns (total_ms, launches)."""
        ms = ctypes.c_float()
        n = ctypes.c_int32()
        _check(load().bd_product_timing(self._h, 1 if enable else 0, ctypes.byref(ms),
                                        ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def set_step_counter(self, value, stream=None):
        _check(load().bd_plan_set_step_counter(self._h, int(value), _stream(stream)))

    def set_shape(self, shape: int):
        """Launch shape of the product.  Mixed plans: 1/2 stream-K CTAs per
        SM, 3 the symmetric kernel over the upper triangle (BD_SHAPE_SYMMETRIC).
        FP64 plans: 0 FP64 multiply-adds, 4 double-float on the FP32 pipe
        (BD_SHAPE_F64_DOUBLE_FLOAT)."""
        _check(load().bd_plan_set_shape(self._h, int(shape)))

    def test_stall(self, cta: int, term: int = 0):
        """bd_plan_test_stall: CTA `cta` of the next symmetric product (term 0)
        or of the term-th product of a Chebyshev series from now takes the
        bounded-wait failure path (a test of the device-side error handling)."""
        _check(load().bd_plan_test_stall(self._h, int(cta), int(term)))

    def autotune(self, D, stream=None):
        sp = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(load().bd_plan_autotune(self._h, _p(D), ctypes.byref(sp), ctypes.byref(ms),
                                       _stream(stream)))
        return int(sp.value), float(ms.value)

    def set_phase_events(self, events):
        """events: list of 7 torch.cuda.Event (enable_timing) or None."""
        if events is None:
            _check(load().bd_set_phase_events(self._h, None, 0))
            return
        for e in events:
            if not e.cuda_event:          # created lazily by torch on first record
                e.record()
        arr = (_vp * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        _check(load().bd_set_phase_events(self._h, arr, len(events)))

    def wiener(self, seed, step_index, out, stream=None):
        _check(load().bd_wiener(self._h, int(seed), int(step_index), out.numel(), _p(out),
                                _stream(stream)))


def eig_bounds_noalloc(D, n3, ld, iters, safety_max, dmin_fraction, bounds, status=None,
                       stream=None):
    """bd_eig_bounds_noalloc: Lanczos bounds of an FP64 D without a plan and
    without any device allocation (fixed-size static scratch, 3N <= 24576)."""
    _check(load().bd_eig_bounds_noalloc(_p(D), int(n3), int(ld), int(iters), float(safety_max),
                                        float(dmin_fraction), _p(bounds), _p(status),
                                        _stream(stream)))


def mesh_fft(K, B, precision, inverse, x, y, stream=None):
    """bd_mesh_fft: B real K^3 meshes <-> their half spectra (unnormalised;
    synchronous).  x and y are device tensors of the input and output."""
    _check(load().bd_mesh_fft(int(K), int(B), PRECISIONS[precision], int(inverse), _p(x), _p(y),
                              _stream(stream)))


class Batch:
    """bd_batch: independent replicas (uneven N), one graph launch per step."""

    def __init__(self, plist, precision: str = "mixed_f16", max_rhs: int = 1, max_cheb: int = 64):
        L = load()
        arr = (BdParams * len(plist))(*[make_params(p, precision, max_rhs, max_cheb)
                                        for p in plist])
        h = _vp()
        _check(L.bd_batch_create(arr, len(plist), ctypes.byref(h)))
        self._h = h
        self.count = len(plist)
        rt, dt = ctypes.c_int64(), ctypes.c_int64()
        _check(L.bd_batch_query(h, -1, None, None, None, ctypes.byref(rt), ctypes.byref(dt)))
        self.r_total, self.d_total = int(rt.value), int(dt.value)
        self.r_off, self.d_off, self.n3 = [], [], []
        for i in range(self.count):
            info = BdPlanInfo()
            ro, do = ctypes.c_int64(), ctypes.c_int64()
            _check(L.bd_batch_query(h, i, ctypes.byref(info), ctypes.byref(ro), ctypes.byref(do),
                                    None, None))
            self.r_off.append(int(ro.value))
            self.d_off.append(int(do.value))
            self.n3.append(int(info.n3))

    def close(self):
        if getattr(self, "_h", None):
            load().bd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_D(self):
        return torch.empty(self.d_total, dtype=torch.uint8, device="cuda")

    def step(self, R, D, *, m=1, n_cheb=20, lanczos_iters=30, bound_safety=0.05,
             dmin_fraction=0.5, seed=0, step_index=0, stats=None, bounds_mode=1, stream=None):
        o = BdStepOpts(m=int(m), n_cheb=int(n_cheb), lanczos_iters=int(lanczos_iters),
                       bound_safety=float(bound_safety), dmin_fraction=float(dmin_fraction),
                       seed=int(seed), step_index=int(step_index), bounds_mode=int(bounds_mode),
                       flags=0)
        _check(load().bd_batch_step(self._h, _p(R), _p(D), ctypes.byref(o), _p(stats),
                                    _stream(stream)))


def kernel_launches() -> int:
    return int(load().bd_kernel_launches())


def read_stats(stats: torch.Tensor) -> dict:
    """Decode a device bd_step_stats buffer (uint8 tensor of STATS_BYTES)."""
    raw = bytes(stats.detach().cpu().numpy().tobytes())
    s = BdStepStats.from_buffer_copy(raw)
    return {f: getattr(s, f) for f, _ in BdStepStats._fields_}


def new_stats() -> torch.Tensor:
    return torch.zeros(STATS_BYTES, dtype=torch.uint8, device="cuda")
