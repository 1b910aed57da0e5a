"""Thin ctypes binding of libhlb (include/hlb.h): argument marshalling only.

Every step of the time step runs in the library's CUDA kernels; this module
converts Python values to the C ABI and raises ``HlbError`` on a non-OK
status.  PyTorch is used by callers only for device memory and streams
(pass ``torch.cuda.current_stream().cuda_stream`` as ``stream``).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhlb.so")

HLB_OK, HLB_EINVAL, HLB_ENOMEM, HLB_ECUDA, HLB_ETIMEOUT, HLB_ENONFINITE, HLB_EUNSUPPORTED = range(7)
HLB_UPWIND2, HLB_WENO5 = 0, 1
HLB_FP64, HLB_FP32, HLB_FP32_TF32X3, HLB_FP32_BF16SPLIT = 0, 1, 2, 3
HLB_ROUND_NEAREST, HLB_ROUND_STOCHASTIC = 0, 1
STATUS_NAMES = {0: "HLB_OK", 1: "HLB_EINVAL", 2: "HLB_ENOMEM", 3: "HLB_ECUDA",
                4: "HLB_ETIMEOUT", 5: "HLB_ENONFINITE", 6: "HLB_EUNSUPPORTED"}


class HlbConfig(C.Structure):
    _fields_ = [("Qx", C.c_int), ("Qy", C.c_int), ("Qz", C.c_int),
                ("Nx_eq", C.c_int), ("Ny_eq", C.c_int), ("Nz_eq", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("stretch_A", C.c_double),
                ("advection", C.c_int), ("precision", C.c_int),
                ("cfl", C.c_double), ("dt", C.c_double),
                ("T_left", C.c_double), ("T_right", C.c_double),
                ("ax", C.c_double), ("ay", C.c_double), ("az", C.c_double),
                ("Kn", C.c_double), ("x_basis", C.c_int)]


class HlbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_LL = C.POINTER(C.c_longlong)
SIGNATURES = {
    "hlb_create": (C.c_int, [C.POINTER(HlbConfig), C.c_int, _P, C.POINTER(_P)]),
    "hlb_destroy": (None, [_P]),
    "hlb_set_walls": (C.c_int, [_P, C.c_int, C.c_double, C.c_double]),
    "hlb_set_force": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_double]),
    "hlb_set_Kn": (C.c_int, [_P, C.c_int, C.c_double]),
    "hlb_init_equilibrium": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double]),
    "hlb_step": (C.c_int, [_P, C.c_long]),
    "hlb_moments": (C.c_int, [_P, _D, _D, _D, _D]),
    "hlb_moments_dev": (C.c_int, [_P, _P, _P, _P, _P]),
    "hlb_moments_noalloc": (C.c_int, [_P, _P, _P, _P, _P]),
    "hlb_sizes": (C.c_int, [_P, _LL, _LL, _LL]),
    "hlb_get_dt": (C.c_int, [_P, C.c_int, _D]),
    "hlb_force_form": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "hlb_set_persistent": (C.c_int, [_P, C.c_int]),
    "hlb_set_rounding": (C.c_int, [_P, C.c_int]),
    "hlb_df_special_check": (C.c_int, [_P, C.c_int, _P, _P]),
    "hlb_fp32_peak": (C.c_int, [C.c_int, _D]),
    "hlb_step_form": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _D]),
    "hlb_get_nsteps": (C.c_int, [_P, _LL]),
    "hlb_get_state": (C.c_int, [_P, _P, C.c_size_t]),
    "hlb_set_state": (C.c_int, [_P, _P, C.c_size_t]),
    "hlb_get_state_dev": (C.c_int, [_P, _P, C.c_size_t]),
    "hlb_set_state_dev": (C.c_int, [_P, _P, C.c_size_t]),
    "hlb_set_force_field": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "hlb_autotune": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "hlb_moments_async": (C.c_int, [_P, _D, _D, _D, _D]),
    "hlb_moments_wait": (C.c_int, [_P]),
    "hlb_prefetch_state": (C.c_int, [_P, _P, C.c_size_t]),
    "hlb_commit_state": (C.c_int, [_P]),
    "hlb_diag": (C.c_int, [_P, _D, _D]),
    "hlb_tables": (C.c_int, [_P, C.c_int] + [_D] * 10),
    "hlb_equilibrium_x": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, _D]),
    "hlb_axis": (C.c_int, [C.c_int, C.c_int, _D, _D, _D]),
    "hlb_set_options": (C.c_int, [_P, C.c_int, C.c_int]),
    "hlb_kernel_times": (C.c_int, [_P, _D, _LL, _D, _LL, C.c_int]),
    "hlb_launch_count": (C.c_int, [_P, _LL, C.c_int]),
    "hlb_set_wait_test": (C.c_int, [_P, C.c_int, C.c_double]),
    "hlb_set_alloc_fail_test": (C.c_int, [C.c_longlong]),
    "hlb_last_error": (C.c_char_p, []),
    "hlb_version": (C.c_char_p, []),
}


def lib():
    """Load libhlb (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhlb is not built ({LIB_PATH} missing); run "
                              "python -m paper_1708_03249_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != HLB_OK:
        raise HlbError(status, lib().hlb_last_error().decode())


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_D)


def make_config(d: dict) -> HlbConfig:
    c = HlbConfig()
    for name, _ in HlbConfig._fields_:
        setattr(c, name, d.get(name, 0) if name == "x_basis" else d[name])
    return c


class Handle:
    """Owns an hlb_handle.  ``cfgs``: one workload dict or a list of them."""

    def __init__(self, cfgs, stream: int | None = None):
        if isinstance(cfgs, dict):
            cfgs = [cfgs]
        self.cfgs = [dict(c) for c in cfgs]
        arr = (HlbConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        h = _P()
        _check(lib().hlb_create(arr, len(cfgs), stream, C.byref(h)))
        self._h = h
        n, v, b = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib().hlb_sizes(self._h, C.byref(n), C.byref(v), C.byref(b)))
        self.nodes, self.values, self.state_bytes = n.value, v.value, b.value
        self.dtype = np.float64 if cfgs[0]["precision"] == HLB_FP64 else np.float32

    def close(self):
        if getattr(self, "_h", None):
            lib().hlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- parameters ------------------------------------------------------------
    def set_walls(self, T_left, T_right, inst=-1):
        _check(lib().hlb_set_walls(self._h, inst, T_left, T_right))

    def set_force(self, ax, ay=0.0, az=0.0, inst=-1):
        _check(lib().hlb_set_force(self._h, inst, ax, ay, az))

    def set_force_field(self, inst, ax=None, ay=None, az=None):
        """hlb_set_force_field: per-node accelerations (arrays of nx * ny, node order), None = zero."""
        keep = []
        c = self.cfgs[inst]
        nodes = int(c["nx"]) * int(c.get("ny", 1))

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            if a.size != nodes:
                raise ValueError(f"acceleration field of instance {inst} needs {nodes} values, got {a.size}")
            keep.append(a)
            return a.ctypes.data_as(_D)
        _check(lib().hlb_set_force_field(self._h, inst, ptr(ax), ptr(ay), ptr(az)))

    def set_Kn(self, Kn, inst=-1):
        _check(lib().hlb_set_Kn(self._h, inst, Kn))

    def set_options(self, use_graphs=True, time_kernels=False):
        _check(lib().hlb_set_options(self._h, int(use_graphs), int(time_kernels)))

    # -- stepping --------------------------------------------------------------
    def init_equilibrium(self, n=1.0, ux=0.0, uy=0.0, T=1.0):
        _check(lib().hlb_init_equilibrium(self._h, n, ux, uy, T))

    def step(self, nsteps=1):
        _check(lib().hlb_step(self._h, int(nsteps)))

    def set_persistent(self, on: bool = True):
        _check(lib().hlb_set_persistent(self._h, 1 if on else 0))

    def set_rounding(self, stochastic: bool):
        """hlb_set_rounding: FP32 stage outputs rounded stochastically or to nearest."""
        _check(lib().hlb_set_rounding(self._h, HLB_ROUND_STOCHASTIC if stochastic else HLB_ROUND_NEAREST))

    def step_form(self, inst=0) -> dict:
        """{"persistent": bool, "segment_cells": int, "ctas": int, "tuned_ms": (persistent, per-stage)}
        of instance inst's group."""
        p, sx, c = C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_double * 2)()
        _check(lib().hlb_step_form(self._h, inst, C.byref(p), C.byref(sx), C.byref(c), ms))
        return {"persistent": bool(p.value), "segment_cells": sx.value, "ctas": c.value,
                "tuned_ms": (ms[0], ms[1])}

    def force_form(self, inst=0) -> int:
        """0: FMA force term; 1: 3xTF32 tensor cores; 2: split-BF16 tensor cores."""
        f = C.c_int(-1)
        _check(lib().hlb_force_form(self._h, inst, C.byref(f)))
        return f.value

    def dt(self, inst=0) -> float:
        d = C.c_double()
        _check(lib().hlb_get_dt(self._h, inst, C.byref(d)))
        return d.value

    def nsteps(self) -> int:
        n = C.c_longlong()
        _check(lib().hlb_get_nsteps(self._h, C.byref(n)))
        return n.value

    # -- outputs ---------------------------------------------------------------
    def moments(self):
        n = np.empty(self.nodes)
        u = np.empty(3 * self.nodes)
        T = np.empty(self.nodes)
        q = np.empty(self.nodes)
        _check(lib().hlb_moments(self._h, _dptr(n), _dptr(u), _dptr(T), _dptr(q)))
        return n, u.reshape(-1, 3), T, q

    def moments_dev(self, n_ptr, u_ptr, T_ptr, q_ptr):
        _check(lib().hlb_moments_dev(self._h, n_ptr, u_ptr, T_ptr, q_ptr))

    def moments_noalloc(self, n_ptr, u_ptr, T_ptr, q_ptr):
        """hlb_moments_dev without any allocation (static device scratch)."""
        _check(lib().hlb_moments_noalloc(self._h, n_ptr, u_ptr, T_ptr, q_ptr))

    def get_state(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.values, dtype=self.dtype)
        _check(lib().hlb_get_state(self._h, out.ctypes.data, out.nbytes))
        return out

    def set_state(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        _check(lib().hlb_set_state(self._h, f.ctypes.data, f.nbytes))

    def get_state_dev(self, ptr: int, nbytes: int):
        _check(lib().hlb_get_state_dev(self._h, ptr, nbytes))

    def set_state_dev(self, ptr: int, nbytes: int):
        _check(lib().hlb_set_state_dev(self._h, ptr, nbytes))

    def moments_async(self, n, u, T, q):
        """hlb_moments_async into caller-owned float64 arrays (page-locked for overlap; keep them alive
        until moments_wait)."""
        ptr = lambda a: None if a is None else a.ctypes.data_as(_D)
        _check(lib().hlb_moments_async(self._h, ptr(n), ptr(u), ptr(T), ptr(q)))

    def moments_wait(self):
        _check(lib().hlb_moments_wait(self._h))

    def autotune(self):
        """hlb_autotune: time segment lengths per velocity-set group, keep the fastest; returns them."""
        out = (C.c_int * len(self.cfgs))(*([-1] * len(self.cfgs)))     # groups <= instances
        _check(lib().hlb_autotune(self._h, out))
        return [v for v in out if v >= 0]

    def prefetch_state(self, ptr: int, nbytes: int):
        """hlb_prefetch_state: stage the host buffer at ptr (keep it alive and unchanged until the commit has run)."""
        _check(lib().hlb_prefetch_state(self._h, ptr, nbytes))

    def commit_state(self):
        _check(lib().hlb_commit_state(self._h))

    def diag(self):
        k = len(self.cfgs)
        N = np.empty(k)
        r = np.empty(k)
        _check(lib().hlb_diag(self._h, _dptr(N), _dptr(r)))
        return N, r

    def tables(self, inst=0):
        c = self.cfgs[inst]
        QX2, VY, VZ = 2 * c["Qx"], max(c["Qy"], 1), max(c["Qz"], 1)
        out = dict(px=np.empty(QX2), py=np.empty(VY), pz=np.empty(VZ), wx=np.empty(QX2),
                   wy=np.empty(VY), wz=np.empty(VZ), Kx=np.empty(QX2 * QX2),
                   Ky=np.empty(VY * VY), Kz=np.empty(VZ * VZ), dx=np.empty(c["nx"]))
        _check(lib().hlb_tables(self._h, inst, *[_dptr(out[k]) for k in
                                                 ("px", "py", "pz", "wx", "wy", "wz", "Kx", "Ky", "Kz", "dx")]))
        out["Kx"] = out["Kx"].reshape(QX2, QX2)
        out["Ky"] = out["Ky"].reshape(VY, VY)
        out["Kz"] = out["Kz"].reshape(VZ, VZ)
        return out

    def kernel_times(self, reset=True):
        sm, wm = C.c_double(), C.c_double()
        sn, wn = C.c_longlong(), C.c_longlong()
        _check(lib().hlb_kernel_times(self._h, C.byref(sm), C.byref(sn), C.byref(wm), C.byref(wn), int(reset)))
        return dict(stage_ms=sm.value, stage_launches=sn.value, wall_ms=wm.value, wall_launches=wn.value)

    def launch_count(self, reset=True) -> int:
        n = C.c_longlong()
        _check(lib().hlb_launch_count(self._h, C.byref(n), int(reset)))
        return n.value

    def set_wait_test(self, withhold_copies: bool, wait_limit_s: float = 0.0):
        _check(lib().hlb_set_wait_test(self._h, int(bool(withhold_copies)), float(wait_limit_s)))


def set_alloc_fail_test(nth: int) -> None:
    """hlb_set_alloc_fail_test: the nth library allocation from now on fails (0 disarms)."""
    _check(lib().hlb_set_alloc_fail_test(int(nth)))


def equilibrium_x(Qx: int, u: float, T: float, Nx_eq: int = -1) -> np.ndarray:
    g = np.empty(2 * Qx)
    _check(lib().hlb_equilibrium_x(Qx, Nx_eq, u, T, _dptr(g)))
    return g


def axis(Q: int, half, laguerre: bool = False):
    """(p, w, K) of a half-range (2Q points; Hermite, or Gauss-Laguerre with
    ``laguerre``) or full-range (Q points) axis, host-built."""
    n = 2 * Q if half else Q
    p, w, K = np.empty(n), np.empty(n), np.empty(n * n)
    _check(lib().hlb_axis(Q, (2 if laguerre else 1) if half else 0, _dptr(p), _dptr(w), _dptr(K)))
    return p, w, K.reshape(n, n)


def fp32_peak(packed: bool = False) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(lib().hlb_fp32_peak(1 if packed else 0, C.byref(t)))
    return t.value


def version() -> str:
    return lib().hlb_version().decode()


def df_special_check(z_ptr: int, n: int, erf_ptr: int, exp_ptr: int):
    """hlb_df_special_check: the node pass's double-float erf(z) and exp(-z^2) (device pointers)."""
    _check(lib().hlb_df_special_check(z_ptr, n, erf_ptr, exp_ptr))
