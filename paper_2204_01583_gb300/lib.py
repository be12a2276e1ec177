"""Thin ctypes binding of the C ABI in ``include/ov.h``.

Argument marshalling only: tensors are passed as raw pointers with their sizes,
every computation runs in the CUDA library.  Importing this module loads the
in-tree shared library and raises if it is missing (build it with
``python -m paper_2204_01583_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libov_gb300.so"

OV_OK = 0
OV_ERR_INVALID_ARG = 1
OV_ERR_OUT_OF_MEMORY = 2
OV_ERR_NOT_CONVERGED = 3
OV_ERR_BREAKDOWN = 4
OV_ERR_CUDA = 5
OV_ERR_NO_GAUGE = 6
OV_ERR_NO_CONTOUR = 7
OV_ERR_SCRATCH_TOO_SMALL = 8

OV_FP64, OV_FP32 = 0, 1
OV_MODE_FP64, OV_MODE_MIXED, OV_MODE_FP64_2PASS, OV_MODE_FP64_REGEN, OV_MODE_F32X2 = 0, 1, 2, 3, 4
OV_CONTOUR_SINGLE, OV_CONTOUR_PAIR = 0, 1

MODES = {"fp64": OV_MODE_FP64, "mixed": OV_MODE_MIXED, "fp64_2pass": OV_MODE_FP64_2PASS,
         "fp64_regen": OV_MODE_FP64_REGEN, "f32x2": OV_MODE_F32X2}

# every symbol include/ov.h declares
EXPORTS = (
    "ov_create", "ov_destroy", "ov_last_error", "ov_set_gauge", "ov_apply_HW", "ov_set_contour",
    "ov_set_contour_ellipse", "ov_get_contour", "ov_place_contour", "ov_sgn_HW_apply", "ov_overlap_apply",
    "ov_sgn_vjp", "ov_overlap_vjp", "ov_set_kernel_timing", "ov_kernel_times", "ov_version",
    "ov_apply_HW_noalloc", "ov_set_hw32_variant", "ov_hw32_variants", "ov_set_persistent", "ov_overlap_solve",
    "ov_set_concurrency", "ov_zolotarev_rule", "ov_set_contour_zolotarev", "ov_place_zolotarev",
)


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("host_io", ctypes.c_int), ("check_every", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("node_chunk", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refine_rounds", ctypes.c_int),
                ("inner_iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("max_residual", ctypes.c_double), ("error_bound", ctypes.c_double), ("ms", ctypes.c_double),
                ("node_updates", ctypes.c_double), ("launches", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Spectrum(ctypes.Structure):
    _fields_ = [("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("abs_max_bound", ctypes.c_double), ("gap", ctypes.c_double),
                ("predicted_error", ctypes.c_double), ("gamma", ctypes.c_double), ("rho", ctypes.c_double),
                ("alpha", ctypes.c_double), ("steps", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"CUDA library not built: {_LIB_PATH} (run python -m paper_2204_01583_gb300.build)")
    lib = ctypes.CDLL(str(_LIB_PATH))
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "ov_create": [ctypes.POINTER(vp), ip, i, d, d, i],
        "ov_destroy": [vp],
        "ov_set_gauge": [vp, vp, i, vp],
        "ov_apply_HW": [vp, vp, vp, i, i, vp],
        "ov_set_contour": [vp, i, dp, dp, d, d],
        "ov_set_contour_ellipse": [vp, i, d, d, d, i],
        "ov_get_contour": [vp, ip, dp, dp, dp],
        "ov_place_contour": [vp, i, i, ctypes.POINTER(Spectrum), vp],
        "ov_sgn_HW_apply": [vp, vp, vp, i, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), vp],
        "ov_overlap_apply": [vp, d, vp, vp, i, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), vp],
        "ov_sgn_vjp": [vp, vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), vp],
        "ov_overlap_vjp": [vp, d, vp, vp, vp, vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(Stats), vp],
        "ov_set_kernel_timing": [vp, i],
        "ov_kernel_times": [vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong), dp, i],
        "ov_apply_HW_noalloc": [ip, i, d, vp, vp, vp, i, vp],
        "ov_set_hw32_variant": [vp, i],
        "ov_set_persistent": [vp, i],
        "ov_set_concurrency": [vp, i],
        "ov_zolotarev_rule": [i, d, d, dp, dp, dp],
        "ov_set_contour_zolotarev": [vp, i, d, d, dp],
        "ov_place_zolotarev": [vp, i, i, ctypes.POINTER(Spectrum), vp],
        "ov_hw32_variants": [i, ip, ip, ip],
        "ov_overlap_solve": [vp, d, vp, vp, i, ctypes.POINTER(SolveOpts), d, i, ctypes.POINTER(Stats), vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ov_last_error.argtypes = [vp]
    lib.ov_last_error.restype = ctypes.c_char_p
    lib.ov_version.argtypes = []
    lib.ov_version.restype = ctypes.c_char_p
    return lib


_lib = _load()


class OvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ov status {code}: {msg}")
        self.code = code


def _ptr(t):
    """Raw data pointer of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(t.ctypes.data)
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """One lattice geometry on one GPU (ov_create / ov_destroy)."""

    def __init__(self, dims, bc_t=-1, m0=1.6, r=1.0, device=0):
        self.dims = tuple(int(x) for x in dims)
        self.V = int(np.prod(self.dims))
        self.device = device
        h = ctypes.c_void_p()
        rc = _lib.ov_create(ctypes.byref(h), (ctypes.c_int * 4)(*self.dims), int(bc_t), float(m0), float(r),
                            int(device))
        if rc != OV_OK:
            raise OvError(rc, "ov_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ov_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != OV_OK and rc not in allow:
            raise OvError(rc, _lib.ov_last_error(self._h).decode())
        return rc

    def last_error(self):
        return _lib.ov_last_error(self._h).decode()

    # ------------------------------------------------------------ gauge / contour
    def set_gauge(self, U, stream=None):
        """U: complex128 canonical gauge field (torch tensor on the device, or host numpy array)."""
        on_dev = 0 if isinstance(U, np.ndarray) else int(U.is_cuda)
        self._check(_lib.ov_set_gauge(self._h, _ptr(U), on_dev, _stream_ptr(stream) if on_dev else None))

    def set_contour(self, z, c, c0):
        z = np.ascontiguousarray(z, dtype=np.complex128)
        c = np.ascontiguousarray(c, dtype=np.complex128)
        c0 = complex(c0)
        self._check(_lib.ov_set_contour(self._h, len(z), z.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        c.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        c0.real, c0.imag))

    def set_contour_ellipse(self, n_q, gamma, rho, alpha, form=OV_CONTOUR_SINGLE):
        self._check(_lib.ov_set_contour_ellipse(self._h, int(n_q), float(gamma), float(rho), float(alpha), int(form)))

    def get_contour(self):
        n = ctypes.c_int(0)
        self._check(_lib.ov_get_contour(self._h, ctypes.byref(n), None, None, None))
        z = np.zeros(n.value, dtype=np.complex128)
        c = np.zeros(n.value, dtype=np.complex128)
        c0 = np.zeros(2)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(_lib.ov_get_contour(self._h, ctypes.byref(n), z.view(np.float64).ctypes.data_as(dp),
                                        c.view(np.float64).ctypes.data_as(dp), c0.ctypes.data_as(dp)))
        return z, c, complex(c0[0], c0[1])

    def place_contour(self, n_q, steps=100, stream=None):
        sp = Spectrum()
        self._check(_lib.ov_place_contour(self._h, int(n_q), int(steps), ctypes.byref(sp), _stream_ptr(stream)))
        return sp.as_dict()

    # ------------------------------------------------------------------ operators
    def apply_HW(self, psi_in, psi_out, nrhs, precision=OV_FP64, stream=None):
        self._check(_lib.ov_apply_HW(self._h, _ptr(psi_in), _ptr(psi_out), int(nrhs), int(precision),
                                     _stream_ptr(stream)))

    @staticmethod
    def opts(mode="fp64", tol=1e-12, max_iter=20000, host_io=False, check_every=32, use_graph=True, node_chunk=0):
        return SolveOpts(MODES[mode] if isinstance(mode, str) else int(mode), float(tol), int(max_iter),
                         int(bool(host_io)), int(check_every), int(bool(use_graph)), int(node_chunk))

    def sgn(self, b, out, nrhs, opts=None, stream=None, allow_not_converged=False):
        st = Stats()
        o = opts if opts is not None else self.opts()
        stream_p = None if o.host_io and stream is None else _stream_ptr(stream)
        rc = _lib.ov_sgn_HW_apply(self._h, _ptr(b), _ptr(out), int(nrhs), ctypes.byref(o), ctypes.byref(st), stream_p)
        self._check(rc, (OV_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = rc
        return d

    def overlap(self, m_q, b, out, nrhs, opts=None, stream=None, allow_not_converged=False):
        st = Stats()
        o = opts if opts is not None else self.opts()
        stream_p = None if o.host_io and stream is None else _stream_ptr(stream)
        rc = _lib.ov_overlap_apply(self._h, float(m_q), _ptr(b), _ptr(out), int(nrhs), ctypes.byref(o),
                                   ctypes.byref(st), stream_p)
        self._check(rc, (OV_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = rc
        return d

    def overlap_solve(self, m_q, b, x, nrhs, inner=None, tol=1e-10, max_iter=10000, stream=None,
                      allow_not_converged=False):
        """x = D_ov(m_q)^-1 b for nrhs sources (CG on the normal equations; see ov_overlap_solve).
        Returns the stats: iterations = CG iterations, max_residual = true ||b - D x|| / ||b||."""
        st = Stats()
        o = inner if inner is not None else self.opts()
        stream_p = None if o.host_io and stream is None else _stream_ptr(stream)
        rc = _lib.ov_overlap_solve(self._h, float(m_q), _ptr(b), _ptr(x), int(nrhs), ctypes.byref(o), float(tol),
                                   int(max_iter), ctypes.byref(st), stream_p)
        self._check(rc, (OV_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = rc
        return d

    def sgn_vjp(self, eta, b, grad_b=None, grad_links=None, opts=None, stream=None):
        st = Stats()
        o = opts if opts is not None else self.opts()
        rc = _lib.ov_sgn_vjp(self._h, _ptr(eta), _ptr(b), _ptr(grad_b) if grad_b is not None else None,
                             _ptr(grad_links) if grad_links is not None else None, ctypes.byref(o),
                             ctypes.byref(st), _stream_ptr(stream))
        self._check(rc)
        return st.as_dict()

    def overlap_vjp(self, m_q, eta, b, grad_b=None, grad_links=None, opts=None, stream=None):
        st = Stats()
        o = opts if opts is not None else self.opts()
        rc = _lib.ov_overlap_vjp(self._h, float(m_q), _ptr(eta), _ptr(b), _ptr(grad_b) if grad_b is not None else None,
                                 _ptr(grad_links) if grad_links is not None else None, ctypes.byref(o),
                                 ctypes.byref(st), _stream_ptr(stream))
        self._check(rc)
        return st.as_dict()

    def set_persistent(self, enable=True):
        self._check(_lib.ov_set_persistent(self._h, int(bool(enable))))

    def set_hw32_variant(self, k=-1):
        self._check(_lib.ov_set_hw32_variant(self._h, int(k)))

    # ------------------------------------------------------------------ timing
    def set_contour_zolotarev(self, n_poles, lambda_min, lambda_max):
        """Zolotarev node set on [lambda_min, lambda_max]; returns its maximum error delta."""
        dl = ctypes.c_double(0.0)
        self._check(_lib.ov_set_contour_zolotarev(self._h, int(n_poles), float(lambda_min), float(lambda_max),
                                                  ctypes.byref(dl)))
        return dl.value

    def place_zolotarev(self, n_poles, steps=100, stream=None):
        sp = Spectrum()
        self._check(_lib.ov_place_zolotarev(self._h, int(n_poles), int(steps), ctypes.byref(sp), _stream_ptr(stream)))
        return sp.as_dict()

    def set_concurrency(self, groups=0):
        """Parallel graph branches over groups of sources (0 = automatic)."""
        self._check(_lib.ov_set_concurrency(self._h, int(groups)))

    def set_kernel_timing(self, enable=True):
        self._check(_lib.ov_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_times(self):
        cap = 16
        names = (ctypes.c_char_p * cap)()
        launches = (ctypes.c_longlong * cap)()
        ms = (ctypes.c_double * cap)()
        n = _lib.ov_kernel_times(self._h, names, launches, ms, cap)
        return {names[k].decode(): (int(launches[k]), float(ms[k])) for k in range(n)}


def apply_HW_noalloc(dims, bc_t, m0, U, psi_in, psi_out, nrhs, stream=None):
    """ov_apply_HW_noalloc: FP64 H_W on device tensors without any allocation in the
    library (fixed internal scratch).  Returns the ov_status code."""
    return _lib.ov_apply_HW_noalloc((ctypes.c_int * 4)(*[int(x) for x in dims]), int(bc_t), float(m0), _ptr(U),
                                    _ptr(psi_in), _ptr(psi_out), int(nrhs), _stream_ptr(stream))


def hw32_variants():
    """[(rhs_tile, compressed, threads)] of the FP32 stencil variants."""
    n = _lib.ov_hw32_variants(-1, None, None, None)
    out = []
    for k in range(n):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.ov_hw32_variants(k, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        out.append((a.value, b.value, c.value))
    return out


def zolotarev_rule(n_poles, lambda_min, lambda_max):
    """(z, c, c0, delta) of the library's Zolotarev node set (host computation, no GPU)."""
    import numpy as np

    z = np.zeros(2 * int(n_poles), dtype=np.complex128)
    c = np.zeros_like(z)
    dl = ctypes.c_double(0.0)
    rc = _lib.ov_zolotarev_rule(int(n_poles), float(lambda_min), float(lambda_max),
                                z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(dl))
    if rc != 0:
        raise OvError(rc, "ov_zolotarev_rule: bad arguments")
    return z, c, 0.0 + 0.0j, dl.value


def version():
    return _lib.ov_version().decode()
