"""Python binding of libskconv (include/skconv.h): argument marshalling only.

Every step of the convolution runs in the library's CUDA kernels; this module
turns torch CUDA tensors into pointers and streams and raises on error codes.
There is no CPU fallback: without the compiled library (or a GPU) every call
raises.

The operation is the real-space part of the split convolution of Sutter,
Wandelt & Elsner (Sec. 2, Eq. 1): y_o = dOmega sum_{gamma(o,i) <= theta_cut}
K_lin(gamma(o,i)) x_i on HEALPix RING maps, with K_lin the linearly interpolated
kernel table of Sec. 3.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libskconv.so")

SK_OK, SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT, SK_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
NODES_UNIFORM, NODES_BIASED = 0, 1
PATH_AUTO, PATH_GENERAL, PATH_TENSOR, PATH_FP32, PATH_BF16X3 = 0, 1, 2, 3, 4
BELT_FP32, BELT_TENSOR, BELT_BF16X3 = 0, 1, 2
PEAK_FFMA, PEAK_FFMA2, PEAK_TF32 = 0, 1, 2

_ERRNAMES = {SK_EINVAL: "SK_EINVAL", SK_ENOMEM: "SK_ENOMEM", SK_ECUDA: "SK_ECUDA",
             SK_ETIMEOUT: "SK_ETIMEOUT", SK_EUNSUPPORTED: "SK_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class SkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class sk_job(ctypes.Structure):
    _fields_ = [("k", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("batch", ctypes.c_int64), ("map_stride", ctypes.c_int64)]


def _declare(L):
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "sk_create": (I, [PP, I]),
        "sk_destroy": (I, [P]),
        "sk_last_error": (ctypes.c_char_p, []),
        "sk_get_status": (I, [P, P]),
        "sk_npix": (I64, [I64]),
        "sk_geometry_create": (I, [P, I64, PP]),
        "sk_geometry_destroy": (I, [P]),
        "sk_geometry_rings": (I, [P, P, P, P, P, P]),
        "sk_kernel_create": (I, [P, P, P, I64, D, I, PP]),
        "sk_kernel_from_legendre": (I, [P, P, P, I64, I64, I64, D, I, D, P, PP]),
        "sk_kernel_update_values": (I, [P, P]),
        "sk_kernel_update_values_async": (I, [P, P, P]),
        "sk_kernel_destroy": (I, [P]),
        "sk_count_pairs": (I, [P, P, ctypes.POINTER(I64)]),
        "sk_count_pairs_by_path": (I, [P, P, ctypes.POINTER(I64)]),
        "sk_count_pairs_by_launch": (I, [P, P, ctypes.POINTER(I64)]),
        "sk_profile_enable": (I, [P, I]),
        "sk_set_workspace_limit": (I, [P, I64]),
        "sk_profile_read": (I, [P, I, P, P, P, ctypes.POINTER(I)]),
        "sk_convolve": (I, [P, P, P, P, I64, I64, P]),
        "sk_convolve_path": (I, [P, P, P, P, I64, I64, I, P]),
        "sk_convolve_rings": (I, [P, P, P, P, I64, I64, I, I, P]),
        "sk_convolve_rings_sym": (I, [P, P, P, P, I64, I64, I, I, P]),
        "sk_resample": (I, [P, P, P, P, I64, I64, P, I, I, I, P]),
        "sk_resample_plan_create": (I, [P, P, P, I, I, I, PP]),
        "sk_resample_plan_destroy": (I, [P]),
        "sk_resample_plan_info": (I, [P, ctypes.POINTER(I64)]),
        "sk_resample_plan_apply": (I, [P, P, P, I64, I64, P]),
        "sk_convolve_adjoint": (I, [P, P, P, P, I64, I64, P]),
        "sk_grad_table": (I, [P, P, P, P, I64, I64, P, P]),
        "sk_grad_table_noalloc": (I, [P, P, P, P, I64, I64, P, P]),
        "sk_convolve_host": (I, [P, P, P, P, I64, I64, P]),
        "sk_convolve_jobs": (I, [P, ctypes.POINTER(sk_job), I, I, P]),
        "sk_graph_capture": (I, [P, ctypes.POINTER(sk_job), I, I, P, PP]),
        "sk_graph_launch": (I, [P, P]),
        "sk_graph_destroy": (I, [P]),
        "sk_kernel_set_tiles": (I, [P, I, I]),
        "sk_kernel_autotune": (I, [P, P, P, P, I64, I64, ctypes.c_char_p, P, ctypes.POINTER(I)]),
        "sk_selftest_wait_timeout": (I, [P, D, P]),
        "sk_selftest_tc_gemm": (I, [P, P, P, P, I, I, I, P]),
        "sk_selftest_tc_sliding": (I, [P, P, P, P, I, I, I, P]),
        "sk_selftest_tc_sliding_bf16": (I, [P, P, P, P, I, I, P]),
        "sk_kernel_get_tiles": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "sk_kernel_response": (I, [P, P, I, P]),
        "sk_fit_real_kernel": (I, [P, P, I, I, D, I, I, D, D, P, P]),
        "sk_harmonic_create": (I, [P, P, P, I, PP]),
        "sk_harmonic_destroy": (I, [P]),
        "sk_harmonic_table_bytes": (I, [P, ctypes.POINTER(I64)]),
        "sk_harmonic_apply": (I, [P, P, P, P, I64, I64, I, P]),
        "sk_harmonic_spectrum": (I, [P, P, P, I64, I64, P, P]),
        "sk_fourier_create": (I, [P, P, PP]),
        "sk_fourier_destroy": (I, [P]),
        "sk_fourier_info": (I, [P, ctypes.POINTER(I64)]),
        "sk_fourier_apply": (I, [P, P, P, P, I64, I64, P]),
        "sk_measure_peak": (I, [P, I, D, ctypes.POINTER(D), P]),
        "sk_kernel_set_cap_weights": (I, [P, I]),
        "sk_kernel_cap_weight_bytes": (I, [P, ctypes.POINTER(I64)]),
        "sk_kernel_set_belt_form": (I, [P, I]),
        "sk_count_pairs_by_ring": (I, [P, P, P, P]),
        "sk_field_plan": (I, [P, D, D, D, D, P, P]),
        "sk_kernel_get_config": (I, [P, ctypes.POINTER(I64)]),
        "sk_device_info": (I, [P, ctypes.POINTER(I64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    """Load libskconv.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build
            if not _build.up_to_date():
                _build.build()
            _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def _check(rc):
    if rc != SK_OK:
        raise SkError(rc, lib().sk_last_error().decode())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _map_args(t, npix):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
        raise TypeError("maps must be float32 CUDA tensors")
    if t.dim() == 1:
        t = t.view(1, -1)
    if t.dim() != 2 or t.shape[1] < npix or t.stride(1) != 1:
        raise ValueError(f"maps must be [batch, >= {npix}] with unit inner stride")
    return t, t.shape[0], t.stride(0) if t.shape[0] > 1 else max(t.shape[1], npix)


class Context:
    """A library context bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().sk_create(ctypes.byref(self._h), device))
        self.device = device

    def close(self):
        if self._h:
            lib().sk_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        _check(lib().sk_get_status(self._h, _stream_ptr(stream)))

    def selftest_wait_timeout(self, seconds: float = 0.05, stream=None):
        """Launch the bounded-wait self-test kernel (it records SK_ETIMEOUT)."""
        _check(lib().sk_selftest_wait_timeout(self._h, float(seconds), _stream_ptr(stream)))

    def measure_peak(self, kind: int, seconds: float = 2.0, stream=None) -> float:
        """TFLOP/s of one arithmetic form (PEAK_FFMA, PEAK_FFMA2, PEAK_TF32) over about `seconds`."""
        r = ctypes.c_double()
        _check(lib().sk_measure_peak(self._h, kind, float(seconds), ctypes.byref(r), _stream_ptr(stream)))
        return r.value

    def device_info(self) -> dict:
        """SM count, maximum SM clock (kHz), opt-in shared memory per block and L2 bytes."""
        a = (ctypes.c_int64 * 4)()
        _check(lib().sk_device_info(self._h, a))
        return {"sms": int(a[0]), "sm_clock_khz": int(a[1]), "smem_per_block": int(a[2]), "l2_bytes": int(a[3])}

    def set_workspace_limit(self, nbytes: int):
        """Cap the context's on-demand workspace at nbytes (0: no cap); a call that would
        need more fails with SkError(SK_ENOMEM) before launching any kernel."""
        _check(lib().sk_set_workspace_limit(self._h, int(nbytes)))

    def profile(self, on: bool):
        _check(lib().sk_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} of the launches recorded since the last read."""
        m = 32
        names = ctypes.create_string_buffer(32 * m)
        ms = np.zeros(m); cnt = np.zeros(m, np.int32); n = ctypes.c_int()
        _check(lib().sk_profile_read(self._h, m, names, ms.ctypes.data, cnt.ctypes.data, ctypes.byref(n)))
        out = {}
        for i in range(min(n.value, m)):
            nm = names.raw[32 * i: 32 * i + 32].split(b"\0")[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out


class Geometry:
    """HEALPix RING geometry for one Nside, on the device."""

    def __init__(self, ctx: Context, nside: int):
        self.ctx = ctx
        self.nside = int(nside)
        self.npix = 12 * self.nside * self.nside
        self._h = ctypes.c_void_p()
        _check(lib().sk_geometry_create(ctx._h, self.nside, ctypes.byref(self._h)))

    def rings(self):
        nr = 4 * self.nside - 1
        n = np.empty(nr, np.int32); st = np.empty(nr, np.int64); s = np.empty(nr, np.int32)
        z = np.empty(nr); sn = np.empty(nr)
        _check(lib().sk_geometry_rings(self._h, n.ctypes.data, st.ctypes.data, s.ctypes.data,
                                       z.ctypes.data, sn.ctypes.data))
        return n, st, s, z, sn

    def close(self):
        if self._h:
            lib().sk_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Kernel:
    """The operator: a tabulated real-space kernel on [0, theta_cut] for a geometry."""

    def __init__(self, geom: Geometry, values=None, theta_cut: float = None, layout: int = NODES_UNIFORM,
                 _handle=None):
        self.geom = geom
        self.ctx = geom.ctx
        self.theta_cut = float(theta_cut)
        self.layout = int(layout)
        if _handle is not None:
            self._h = _handle
            self.values = None
            return
        v = np.ascontiguousarray(values, dtype=np.float64)
        self.values = v.copy()
        self.n_nodes = len(v)
        self._h = ctypes.c_void_p()
        _check(lib().sk_kernel_create(self.ctx._h, geom._h, v.ctypes.data, len(v), self.theta_cut,
                                      self.layout, ctypes.byref(self._h)))

    @classmethod
    def from_legendre(cls, geom: Geometry, k_ell, lmin: int, lmax: int, n_nodes: int, theta_cut: float,
                      layout: int = NODES_UNIFORM, taper_start: float = 0.9):
        """Tabulate on the device the l in [lmin, lmax] part of sum (2l+1)/(4pi) K_l P_l(cos theta),
        tapered to 0 at theta_cut, and build the operator.  Returns (Kernel, FP64 node values)."""
        kl = np.ascontiguousarray(k_ell, dtype=np.float64)
        if len(kl) < lmax + 1:
            raise ValueError("k_ell shorter than lmax + 1")
        vals = np.empty(n_nodes, np.float64)
        h = ctypes.c_void_p()
        _check(lib().sk_kernel_from_legendre(geom.ctx._h, geom._h, kl.ctypes.data, lmin, lmax, n_nodes,
                                             float(theta_cut), layout, float(taper_start),
                                             vals.ctypes.data, ctypes.byref(h)))
        k = cls(geom, theta_cut=theta_cut, layout=layout, _handle=h)
        k.values = vals
        k.n_nodes = n_nodes
        return k, vals

    @staticmethod
    def tabulate(geom: Geometry, k_ell, lmin, lmax, n_nodes, theta_cut, layout=NODES_UNIFORM,
                 taper_start=0.9):
        """Only the FP64 node values of from_legendre (no operator)."""
        kl = np.ascontiguousarray(k_ell, dtype=np.float64)
        vals = np.empty(n_nodes, np.float64)
        _check(lib().sk_kernel_from_legendre(geom.ctx._h, geom._h, kl.ctypes.data, lmin, lmax, n_nodes,
                                             float(theta_cut), layout, float(taper_start),
                                             vals.ctypes.data, None))
        return vals

    def update_values_async(self, values, stream=None):
        """Take node values from a float64 CUDA tensor on `stream` (no host synchronisation;
        the table and stored cap weights are rebuilt on the device only if the values changed)."""
        import torch
        if not (isinstance(values, torch.Tensor) and values.is_cuda and values.dtype == torch.float64):
            raise TypeError("values must be a float64 CUDA tensor")
        v = values.contiguous()
        if v.numel() != self.n_nodes:
            raise ValueError("node count differs")
        _check(lib().sk_kernel_update_values_async(self._h, ctypes.c_void_p(v.data_ptr()), _stream_ptr(stream)))
        self.values = None                  # the host copy no longer describes the device table
        self._async_values = v              # kept alive until the stream has read it

    def update_values(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        if len(v) != self.n_nodes:
            raise ValueError("node count differs")
        _check(lib().sk_kernel_update_values(self._h, v.ctypes.data))
        self.values = v.copy()

    def count_pairs(self) -> int:
        c = ctypes.c_int64()
        _check(lib().sk_count_pairs(self.ctx._h, self._h, ctypes.byref(c)))
        return c.value

    def count_pairs_by_path(self):
        """(belt, cap, general) in-cut pair counts of the outputs each path evaluates."""
        c = (ctypes.c_int64 * 3)()
        _check(lib().sk_count_pairs_by_path(self.ctx._h, self._h, c))
        return int(c[0]), int(c[1]), int(c[2])

    def count_pairs_by_launch(self):
        """In-cut pairs (belt, caps with narrow windows, caps with wide windows, per-pair general)."""
        a = (ctypes.c_int64 * 4)()
        _check(lib().sk_count_pairs_by_launch(self.ctx._h, self._h, a))
        return [int(v) for v in a]

    def pairs_by_ring(self):
        """(in-cut pairs of each output ring, each ring's path: 0 belt, 1 cap, 2 per-pair,
        3 cap with wide windows) -- sk_count_pairs_by_ring."""
        nr = 4 * self.geom.nside - 1
        pairs = np.zeros(nr, np.int64)
        path = np.zeros(nr, np.uint8)
        _check(lib().sk_count_pairs_by_ring(self.ctx._h, self._h, pairs.ctypes.data, path.ctypes.data))
        return pairs, path

    def autotune(self, x, out=None, cache_path=None, stream=None) -> int:
        """Time the belt forms (FP32 with every tile width, tensor cores) and stored
        against evaluated cap weights on maps x, keep the fastest; returns the FP32
        tile width (the rest: config())."""
        import torch
        x2, b, stride = _map_args(x, self.geom.npix)
        if out is None:
            out = torch.empty_like(x2)
        p = ctypes.c_int()
        cp = cache_path.encode() if cache_path else None
        _check(lib().sk_kernel_autotune(self.ctx._h, self._h, ctypes.c_void_p(x2.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), b, stride, cp, _stream_ptr(stream),
                                        ctypes.byref(p)))
        return p.value

    def set_belt_form(self, form: int):
        """Belt of PATH_AUTO: BELT_FP32, BELT_TENSOR (3xTF32) or BELT_BF16X3 (about 1e-5
        relative: outside the 1e-6 bound); a tensor form evaluates its tiles."""
        _check(lib().sk_kernel_set_belt_form(self._h, int(form)))

    def config(self) -> dict:
        """The operator's settings: FP32 belt tile width, belt form, stored cap weights,
        whether it has a tensor belt form."""
        a = (ctypes.c_int64 * 4)()
        _check(lib().sk_kernel_get_config(self._h, a))
        return {"belt_p": int(a[0]), "belt_form": {BELT_FP32: "fp32", BELT_TENSOR: "tensor",
                                                   BELT_BF16X3: "bf16x3"}[int(a[1])],
                "cap_weights": "stored" if a[2] else "evaluated", "tensor_form_available": bool(a[3] & 1),
                "bf16x3_form_available": bool(a[3] & 2)}

    def set_cap_weights(self, stored: bool):
        """Keep the caps' weights stored on the device (True) or evaluate them per call (False)."""
        _check(lib().sk_kernel_set_cap_weights(self._h, 1 if stored else 0))

    def cap_weight_bytes(self) -> int:
        """Device bytes of the stored cap weights (0 when the caps evaluate per call)."""
        b = ctypes.c_int64()
        _check(lib().sk_kernel_cap_weight_bytes(self._h, ctypes.byref(b)))
        return b.value

    def set_tiles(self, belt_p=0, cap_t=0):
        _check(lib().sk_kernel_set_tiles(self._h, belt_p, cap_t))

    def tiles(self):
        p = ctypes.c_int(); t = ctypes.c_int()
        _check(lib().sk_kernel_get_tiles(self._h, ctypes.byref(p), ctypes.byref(t)))
        return p.value, t.value

    def close(self):
        if self._h:
            lib().sk_kernel_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def convolve(kern: Kernel, x, out=None, path: int = PATH_AUTO, stream=None):
    """y = A x for maps x [batch, npix] (float32 CUDA)."""
    import torch
    x2, b, stride = _map_args(x, kern.geom.npix)
    if out is None:
        out = torch.empty_like(x2)
    o2, b2, stride2 = _map_args(out, kern.geom.npix)
    if b2 != b or stride2 != stride:
        raise ValueError("out must match x in shape and strides")
    _check(lib().sk_convolve_path(kern.ctx._h, kern._h, ctypes.c_void_p(x2.data_ptr()),
                                  ctypes.c_void_p(o2.data_ptr()), b, stride, path, _stream_ptr(stream)))
    return out


def convolve_rings(kern: Kernel, x, ring_lo: int, ring_hi: int, out=None, stream=None):
    """The outputs of rings [ring_lo, ring_hi) (0-based) of y = A x, for a ring-band
    decomposition (see bands.py): x needs valid values on the band's halo rings only (the
    rest finite, e.g. zeros: zero weights meet some pixels outside a window), and out is
    valid on the band only (other rings may hold partial sums)."""
    import torch
    x2, b, stride = _map_args(x, kern.geom.npix)
    if out is None:
        out = torch.empty_like(x2)
    o2, b2, stride2 = _map_args(out, kern.geom.npix)
    if b2 != b or stride2 != stride:
        raise ValueError("out must match x in shape and strides")
    _check(lib().sk_convolve_rings(kern.ctx._h, kern._h, ctypes.c_void_p(x2.data_ptr()),
                                   ctypes.c_void_p(o2.data_ptr()), b, stride, int(ring_lo), int(ring_hi),
                                   _stream_ptr(stream)))
    return out


def rotation_to_pole(theta0: float, phi0: float) -> np.ndarray:
    """The rotation M (3x3, FP64) that takes the north pole to the direction (theta0, phi0):
    M = R_z(phi0) R_y(theta0) (sk_field_plan).  resample(.., M, ..) moves a field centred
    there onto the pole; resample(.., M.T, ..) moves it back."""
    return field_plan(None, theta0, phi0, 1.0, 1.0)[0]


def field_plan(geom, theta0: float, phi0: float, radius: float, theta_cut: float):
    """(rotation, (out_hi, in_hi, sky_lo, sky_hi)) of a partial-sky field (sk_field_plan);
    geom None gives the rotation only."""
    rot = np.empty(9, np.float64)
    rings = np.zeros(4, np.int32)
    _check(lib().sk_field_plan(None if geom is None else geom._h, float(theta0), float(phi0), float(radius),
                               float(theta_cut), rot.ctypes.data, rings.ctypes.data))
    return rot.reshape(3, 3), tuple(int(v) for v in rings)


def resample(geom: Geometry, x, rot, ring_lo: int, ring_hi: int, src_ring_hi: int = None, out=None, stream=None):
    """Nearest-centre resampling of maps under a rotation (sk_resample): output pixel p of
    rings [ring_lo, ring_hi) takes x at the pixel nearest to rot @ v_p (0 if that pixel is
    on a ring >= src_ring_hi).  Other output pixels are left as they are (zeros if out is
    None)."""
    import torch
    x2, b, stride = _map_args(x, geom.npix)
    if out is None:
        out = torch.zeros_like(x2)
    o2, b2, stride2 = _map_args(out, geom.npix)
    if b2 != b or stride2 != stride:
        raise ValueError("out must match x in shape and strides")
    m = np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(9))
    nr = 4 * geom.nside - 1
    src = nr if src_ring_hi is None else int(src_ring_hi)
    _check(lib().sk_resample(geom.ctx._h, geom._h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(o2.data_ptr()),
                             b, stride, m.ctypes.data, int(ring_lo), int(ring_hi), src, _stream_ptr(stream)))
    return out


class ResamplePlan:
    """resample() planned once for a rotation and ring ranges (sk_resample_plan_*): the
    nearest-centre search runs at creation; apply() is a gather with the same result."""

    def __init__(self, geom: Geometry, rot, ring_lo: int, ring_hi: int, src_ring_hi: int = None):
        self.geom = geom
        m = np.ascontiguousarray(np.asarray(rot, dtype=np.float64).reshape(9))
        nr = 4 * geom.nside - 1
        src = nr if src_ring_hi is None else int(src_ring_hi)
        self._h = ctypes.c_void_p()
        _check(lib().sk_resample_plan_create(geom.ctx._h, geom._h, m.ctypes.data, int(ring_lo), int(ring_hi), src,
                                             ctypes.byref(self._h)))

    def info(self):
        out = (ctypes.c_int64 * 3)()
        _check(lib().sk_resample_plan_info(self._h, out))
        return {"pairs": out[0], "pixels": out[1], "bytes": out[2]}

    def apply(self, x, out=None, stream=None):
        import torch
        x2, b, stride = _map_args(x, self.geom.npix)
        if out is None:
            out = torch.zeros_like(x2)
        o2, b2, stride2 = _map_args(out, self.geom.npix)
        if b2 != b or stride2 != stride:
            raise ValueError("out must match x in shape and strides")
        _check(lib().sk_resample_plan_apply(self._h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(o2.data_ptr()),
                                            b, stride, _stream_ptr(stream)))
        return out

    def close(self):
        if self._h:
            lib().sk_resample_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PolarPatch:
    """A partial-sky field (a disc of `radius` around (theta0, phi0)) convolved on the
    polar cap (Sec. 4: re-oriented onto the pole, a field spans few rings).  The map is
    rotated so that the field centre is the pole (nearest-centre resampling of the cap
    rings the sums read), the output rings of the field are summed (convolve_rings, whose
    windows stay on those rings), and the result is rotated back onto the sky rings that
    hold the field; sky pixels whose nearest rotated pixel is outside the summed rings get
    0.  Up to the two resamplings this is the full-sky operator on the field: the kernel
    is radial."""

    def __init__(self, kern: Kernel, theta0: float, phi0: float, radius: float):
        self.kern = kern
        g = kern.geom
        # rotation and rings (sk_field_plan): output rings reach the field radius plus two
        # pixels, input rings theta_cut beyond them, sky rings the field's colatitude band
        self.rot, (self.out_hi, self.in_hi, self.sky_lo, self.sky_hi) = field_plan(g, theta0, phi0, radius,
                                                                                   kern.theta_cut)

        # the two resamplings, planned once (their searches depend on the geometry only)
        self.to_cap = ResamplePlan(g, self.rot, 0, self.in_hi)
        self.to_sky = ResamplePlan(g, self.rot.T, self.sky_lo, self.sky_hi, src_ring_hi=self.out_hi)

    def convolve(self, x, out=None, stream=None, work=None):
        """y on the field's sky rings (other pixels of out untouched; zeros if out is None).
        work: optional pair of scratch maps shaped like x (the rotated input and output; the
        first must hold finite values, e.g. zeros, beyond the cap rings, which it is not
        written on)."""
        import torch
        if work is None:
            x2, _, _ = _map_args(x, self.kern.geom.npix)
            work = (torch.zeros_like(x2), torch.empty_like(x2))
        xr, yr = work
        self.to_cap.apply(x, out=xr, stream=stream)
        convolve_rings(self.kern, xr, 0, self.out_hi, out=yr, stream=stream)
        return self.to_sky.apply(yr, out=out, stream=stream)


def convolve_rings_sym(kern: Kernel, x, ring_lo: int, ring_hi: int, out=None, stream=None):
    """convolve_rings for rings [ring_lo, ring_hi) and their mirrors about the equator (a band
    of bands.symmetric_bands): the polar-cap sums of a ring and its mirror run once."""
    import torch
    x2, b, stride = _map_args(x, kern.geom.npix)
    if out is None:
        out = torch.empty_like(x2)
    o2, b2, stride2 = _map_args(out, kern.geom.npix)
    if b2 != b or stride2 != stride:
        raise ValueError("out must match x in shape and strides")
    _check(lib().sk_convolve_rings_sym(kern.ctx._h, kern._h, ctypes.c_void_p(x2.data_ptr()),
                                       ctypes.c_void_p(o2.data_ptr()), b, stride, int(ring_lo), int(ring_hi),
                                       _stream_ptr(stream)))
    return out


def convolve_adjoint(kern: Kernel, gy, out=None, stream=None):
    """x_bar = A^T y_bar (the same gather: the operator is symmetric)."""
    import torch
    g2, b, stride = _map_args(gy, kern.geom.npix)
    if out is None:
        out = torch.empty_like(g2)
    o2, _, _ = _map_args(out, kern.geom.npix)
    _check(lib().sk_convolve_adjoint(kern.ctx._h, kern._h, ctypes.c_void_p(g2.data_ptr()),
                                     ctypes.c_void_p(o2.data_ptr()), b, stride, _stream_ptr(stream)))
    return out


def grad_table(kern: Kernel, x, gy, out=None, stream=None):
    """dL/dV_n for the table nodes given maps x and dL/dy (float32 [n_nodes])."""
    import torch
    x2, b, stride = _map_args(x, kern.geom.npix)
    g2, b2, stride2 = _map_args(gy, kern.geom.npix)
    if b2 != b or stride2 != stride:
        raise ValueError("x and gy must match")
    if out is None:
        out = torch.empty(kern.n_nodes, dtype=torch.float32, device=x2.device)
    _check(lib().sk_grad_table(kern.ctx._h, kern._h, ctypes.c_void_p(x2.data_ptr()),
                               ctypes.c_void_p(g2.data_ptr()), b, stride,
                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def convolve_host(kern: Kernel, x: np.ndarray, out: np.ndarray = None, stream=None) -> np.ndarray:
    """End to end from host memory: copies in, convolves, copies out (synchronises)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x[None]
    if out is None:
        out = np.empty_like(x)
    _check(lib().sk_convolve_host(kern.ctx._h, kern._h, x.ctypes.data, out.ctypes.data, x.shape[0],
                                  x.shape[1], _stream_ptr(stream)))
    return out


def _jobs_array(jobs):
    arr = (sk_job * len(jobs))()
    keep = []
    for i, (kern, x, y) in enumerate(jobs):
        x2, b, stride = _map_args(x, kern.geom.npix)
        y2, _, _ = _map_args(y, kern.geom.npix)
        keep.append((x2, y2))
        arr[i] = sk_job(kern._h.value, x2.data_ptr(), y2.data_ptr(), b, stride)
    return arr, keep


def convolve_jobs(ctx: Context, jobs, path: int = PATH_AUTO, stream=None):
    """Several (kernel, x, y) jobs with mixed Nside/kernels/batch in one launch per path family."""
    arr, _keep = _jobs_array(jobs)
    _check(lib().sk_convolve_jobs(ctx._h, arr, len(jobs), path, _stream_ptr(stream)))


def kernel_response(kern: Kernel, lmax: int):
    """R_l = 2 pi int K_lin P_l(cos t) sin t dt, l = 0..lmax (FP64 numpy): the harmonic
    content of the real-space part, so that K^_l = K_l - R_l completes the split."""
    R = np.empty(int(lmax) + 1, np.float64)
    _check(lib().sk_kernel_response(kern.ctx._h, kern._h, int(lmax), R.ctypes.data))
    return R


def fit_real_kernel(ctx: Context, k_ell, lcut: int, theta_cut: float, n_basis: int = 257, nt_out: int = None,
                    lfit: int = None, low_weight: float = 1e-3, reg: float = 1e-9):
    """Least-squares real-space part of K_l (see sk_fit_real_kernel): returns
    (node values on nt_out uniform nodes of [0, theta_cut], sigma_rms)."""
    kl = np.ascontiguousarray(np.asarray(k_ell, dtype=np.float64))
    lfit = len(kl) - 1 if lfit is None else int(lfit)
    if nt_out is None:
        nt_out = 32 * (n_basis - 1) + 1
    V = np.empty(int(nt_out), np.float64)
    sig = ctypes.c_double()
    _check(lib().sk_fit_real_kernel(ctx._h, kl.ctypes.data, lfit, int(lcut), float(theta_cut), int(n_basis),
                                    int(nt_out), float(low_weight), float(reg), V.ctypes.data, ctypes.byref(sig)))
    return V, sig.value


class Harmonic:
    """The harmonic half of the split (Sec. 2, Eq. 1): y = sum_{l <= lmax} K^_l a_lm Y_lm
    with a_lm = dOmega sum_q x_q Y*_lm(q), for a geometry and FP64 coefficients K^_l."""

    def __init__(self, ctx: Context, geom: Geometry, k_hat, lmax: int = None):
        import numpy as np
        kl = np.ascontiguousarray(np.asarray(k_hat, dtype=np.float64))
        self.lmax = len(kl) - 1 if lmax is None else int(lmax)
        if len(kl) < self.lmax + 1:
            raise ValueError("k_hat needs lmax + 1 coefficients")
        self.ctx, self.geom = ctx, geom
        self._h = ctypes.c_void_p()
        _check(lib().sk_harmonic_create(ctx._h, geom._h, kl.ctypes.data, self.lmax, ctypes.byref(self._h)))

    def table_bytes(self) -> int:
        n = ctypes.c_int64()
        _check(lib().sk_harmonic_table_bytes(self._h, ctypes.byref(n)))
        return n.value

    def apply(self, x, out=None, accumulate: bool = False, stream=None):
        """out (+)= H x for maps x [batch, npix] (float32 CUDA)."""
        import torch
        x2, b, stride = _map_args(x, self.geom.npix)
        if out is None:
            out = torch.empty_like(x2)
        o2, _, ostride = _map_args(out, self.geom.npix)
        if ostride != stride:
            raise ValueError("input and output maps need the same stride")
        _check(lib().sk_harmonic_apply(self.ctx._h, self._h, ctypes.c_void_p(x2.data_ptr()),
                                       ctypes.c_void_p(o2.data_ptr()), b, stride, 1 if accumulate else 0,
                                       _stream_ptr(stream)))
        return out if out.dim() == x.dim() else out.view_as(x)

    def spectrum(self, x, stream=None):
        """Power spectra C_l = sum_m |a_lm|^2 / (2l + 1), l = 0..lmax, of maps x [batch, npix]
        (float32 CUDA) from the handle's analysis: a float64 CUDA tensor [batch, lmax + 1]."""
        import torch
        x2, b, stride = _map_args(x, self.geom.npix)
        cl = torch.empty(b, self.lmax + 1, dtype=torch.float64, device=x2.device)
        _check(lib().sk_harmonic_spectrum(self.ctx._h, self._h, ctypes.c_void_p(x2.data_ptr()), b, stride,
                                          ctypes.c_void_p(cl.data_ptr()), _stream_ptr(stream)))
        return cl

    def __del__(self):
        try:
            if self._h:
                lib().sk_harmonic_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


class FourierBelt:
    """The real-space convolution of a kernel with its equatorial-zone rings done in the
    rings' Fourier modes (Y_o(m) = sum_i W_oi(m) X_i(m), linear in theta_cut), the other
    rings by the direct paths: for wide theta_cut, where direct sums grow with its square."""

    def __init__(self, kern: Kernel):
        self.kern, self.ctx, self.geom = kern, kern.geom.ctx, kern.geom
        self._h = ctypes.c_void_p()
        _check(lib().sk_fourier_create(self.ctx._h, kern._h, ctypes.byref(self._h)))

    def info(self) -> dict:
        """first_ring, rings (0: none in the Fourier form), H (ring offsets -H..H), bytes of G."""
        v = (ctypes.c_int64 * 4)()
        _check(lib().sk_fourier_info(self._h, v))
        return {"first_ring": v[0], "rings": v[1], "H": v[2], "bytes": v[3]}

    def apply(self, x, out=None, stream=None):
        """out = A x for maps x [batch, npix] (float32 CUDA)."""
        import torch
        x2, b, stride = _map_args(x, self.geom.npix)
        if out is None:
            out = torch.empty_like(x2)
        o2, _, ostride = _map_args(out, self.geom.npix)
        if ostride != stride:
            raise ValueError("input and output maps need the same stride")
        _check(lib().sk_fourier_apply(self.ctx._h, self._h, ctypes.c_void_p(x2.data_ptr()),
                                      ctypes.c_void_p(o2.data_ptr()), b, stride, _stream_ptr(stream)))
        return out if out.dim() == x.dim() else out.view_as(x)

    def __del__(self):
        try:
            if self._h:
                lib().sk_fourier_destroy(self._h)
                self._h = ctypes.c_void_p()
        except Exception:
            pass


def split_convolve(kern: Kernel, harm: Harmonic, x, out=None, stream=None):
    """The whole split convolution (Sec. 2, Eq. 1): the real-space part of kern plus the
    harmonic part of harm, y = A_real x + H x."""
    y = convolve(kern, x, out=out, stream=stream)
    harm.apply(x, out=y, accumulate=True, stream=stream)
    return y


def plan_split(ctx: Context, geom: Geometry, k_ell, target_sigma: float, lcut_options, theta_cut_options,
               alpha: float = 5.0, n_basis: int = 257, lfit: int = None, reps: int = 3):
    """Choose (l_cut, theta_cut) for the split of K_l like the paper's optimiser
    (Sec. 2 and 4: the cheapest split whose Eq. 2 error meets the target), with
    measured costs instead of cost models: for every candidate the real-space part
    is fitted (fit_real_kernel), its error taken as alpha * sigma_rms (Eq. 2), and
    the whole split timed on this GPU (real-space sum with the fitted table plus
    the harmonic part with K^_l = K_l - R_l) on a white-noise map.  Returns
    (best, rows): best is the fastest row meeting the target (None if none does);
    a row is a dict with lcut, theta_cut, sigma, ms_real, ms_harmonic, ms_total."""
    import torch
    kl = np.asarray(k_ell, dtype=np.float64)
    lfit = len(kl) - 1 if lfit is None else int(lfit)
    npix = geom.npix
    x = torch.randn(1, npix, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    y = torch.empty_like(x)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = []
    for lcut in lcut_options:
        for tc in theta_cut_options:
            V, sig = fit_real_kernel(ctx, kl, lcut, tc, n_basis=n_basis, lfit=lfit)
            kern = Kernel(geom, V, tc)
            R = kernel_response(kern, lcut)
            harm = Harmonic(ctx, geom, kl[: lcut + 1] - R, lcut)
            ms_r = timed(lambda: convolve(kern, x, out=y))
            ms_h = timed(lambda: harm.apply(x, out=y, accumulate=True))
            rows.append(dict(lcut=int(lcut), theta_cut=float(tc), sigma=alpha * sig, ms_real=ms_r,
                             ms_harmonic=ms_h, ms_total=ms_r + ms_h))
            del harm, kern
    ok = [r for r in rows if r["sigma"] <= target_sigma]
    best = min(ok, key=lambda r: r["ms_total"]) if ok else None
    return best, rows


class Graph:
    """A CUDA graph of convolve_jobs(jobs) on fixed buffers."""

    def __init__(self, ctx: Context, jobs, path: int = PATH_AUTO, stream=None):
        import torch
        self.ctx = ctx
        self._stream = stream if stream is not None else torch.cuda.Stream()
        arr, self._keep = _jobs_array(jobs)
        self._h = ctypes.c_void_p()
        _check(lib().sk_graph_capture(ctx._h, arr, len(jobs), path, _stream_ptr(self._stream),
                                      ctypes.byref(self._h)))

    def launch(self, stream=None):
        _check(lib().sk_graph_launch(self._h, _stream_ptr(stream)))

    def close(self):
        if self._h:
            lib().sk_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sph_conv(x, table, kern: Kernel):
    """Differentiable y = A(table) x: gradients for the maps (adjoint gather) and for the
    table nodes (binned scatter-add).  `table` is a float64 or float32 tensor of the
    node values; the operator's table is refreshed when the values change."""
    return _SphConv.apply(x, table, kern)


def _make_autograd():
    import torch

    class SphConv(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, table, kern):
            if table.is_cuda:
                # on the device, on the current stream: no host round trip (the kernels
                # rebuild the table only if the values changed)
                kern.update_values_async(table.detach().to(torch.float64))
            else:
                v = table.detach().to(torch.float64).numpy()
                if kern.values is None or not np.array_equal(v, kern.values):
                    kern.update_values(v)
            ctx.kern = kern
            ctx.table_dtype = table.dtype
            ctx.table_device = table.device
            ctx.save_for_backward(x)
            return convolve(kern, x.contiguous())

        @staticmethod
        def backward(ctx, gy):
            (x,) = ctx.saved_tensors
            gy = gy.contiguous()
            gx = convolve_adjoint(ctx.kern, gy) if ctx.needs_input_grad[0] else None
            gt = None
            if ctx.needs_input_grad[1]:
                gt = grad_table(ctx.kern, x.contiguous(), gy).to(device=ctx.table_device,
                                                                  dtype=ctx.table_dtype)
            return gx, gt, None

    return SphConv


class _Lazy:
    _cls = None

    def apply(self, *a):
        if _Lazy._cls is None:
            _Lazy._cls = _make_autograd()
        return _Lazy._cls.apply(*a)


_SphConv = _Lazy()
