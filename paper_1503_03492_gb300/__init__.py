"""GB300 (sm_103a) statistical multi-resolution projection (arXiv 1503.03492).

Thin ctypes binding of the C ABI in ``include/smre.h`` (``libsmre.so``).  The
functions keep the C names; every step of the projection runs in the CUDA
kernels of the library, this module only marshals arguments.  Images may be
``torch`` CUDA tensors, ``torch`` CPU tensors or ``numpy`` arrays (float32,
C-contiguous, H x W); CUDA tensors are passed by device pointer, host arrays
by host pointer (the library stages them).

The library must have been built (``python -m paper_1503_03492_gb300.build``
or ``__graft_entry__.build()``); every call raises ImportError when it is
missing.  There is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "SMRE_OK", "SMRE_EINVAL", "SMRE_ENOMEM", "SMRE_ECUDA", "SMRE_ETIMEOUT", "SMRE_ENOTCONVERGED",
    "SMRE_C_PERSET", "SMRE_C_CHI2", "SMRE_C_MAXSTAT", "SMRE_C_EXPLICIT", "SMRE_F_VIOLATION",
    "SMRE_F_GROUP_LAUNCHES", "SMRE_F_SELFTEST_TIMEOUT", "SMRE_F_AUTOTUNE", "SMRE_F_BAND_IN_SMEM",
    "SMRE_SCHED_PERSISTENT",
    "SMRE_SCHED_BATCHED", "SMRE_SCHED_GROUPS", "smre_dykstra_schedule",
    "SmreError", "smre_params", "smre_result", "lib_path", "load",
    "smre_bounds", "smre_dykstra_create", "smre_dykstra_project",
    "smre_dykstra_project_incomplete", "smre_dykstra_set_stopping", "smre_dykstra_bounds",
    "smre_dykstra_history", "smre_dykstra_icd_sweeps", "smre_dykstra_device_bytes",
    "smre_dykstra_destroy", "smre_last_error", "smre_version", "Projector", "EXPORTED",
    "smre_dykstra_kernel_launches", "make_params", "smre_dykstra_project_static",
    "SMRE_Q_FP32", "SMRE_Q_BF16", "SMRE_Q_FP16", "smre_batch_params", "make_batch_params",
    "smre_batch_image_bytes", "smre_batch_create", "smre_batch_submit", "smre_batch_run",
    "smre_batch_poll", "smre_batch_retrieve", "smre_batch_project", "smre_batch_active",
    "smre_batch_item_spread", "SMRE_BF_AUTOTUNE", "SMRE_BF_SPREAD2", "SMRE_BF_SPREAD4",
    "SMRE_BF_PER_SIDE", "smre_batch_per_side",
    "smre_batch_kernel_launches", "smre_batch_device_bytes", "smre_batch_last_error",
    "smre_batch_destroy", "Batch", "smre_server_params", "smre_server_counters",
    "smre_server_create", "smre_server_submit", "smre_server_wait", "smre_server_stats",
    "smre_server_destroy", "Server", "smre_admm_params", "smre_admm_result", "make_admm_params",
    "smre_admm_create", "smre_admm_solve", "smre_admm_kernel_launches", "smre_admm_projector",
    "smre_admm_destroy", "smre_admm_last_error", "Admm",
]

SMRE_OK, SMRE_EINVAL, SMRE_ENOMEM, SMRE_ECUDA, SMRE_ETIMEOUT, SMRE_ENOTCONVERGED = range(6)
SMRE_C_PERSET, SMRE_C_CHI2, SMRE_C_MAXSTAT, SMRE_C_EXPLICIT = range(4)
SMRE_F_VIOLATION = 1
SMRE_F_GROUP_LAUNCHES = 2
SMRE_F_SELFTEST_TIMEOUT = 4
SMRE_F_AUTOTUNE = 8
SMRE_F_BAND_IN_SMEM = 16
SMRE_SCHED_PERSISTENT, SMRE_SCHED_BATCHED, SMRE_SCHED_GROUPS = 1, 2, 3
SMRE_Q_FP32, SMRE_Q_BF16, SMRE_Q_FP16 = range(3)
SMRE_BF_AUTOTUNE, SMRE_BF_SPREAD2, SMRE_BF_SPREAD4, SMRE_BF_PER_SIDE = 1, 2, 4, 8

_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTCONVERGED"}

# every entry point declared in include/smre.h
EXPORTED = (
    "smre_bounds", "smre_dykstra_create", "smre_dykstra_project",
    "smre_dykstra_project_incomplete", "smre_dykstra_set_stopping", "smre_dykstra_bounds",
    "smre_dykstra_history", "smre_dykstra_icd_sweeps", "smre_dykstra_device_bytes",
    "smre_dykstra_destroy", "smre_last_error", "smre_version", "smre_dykstra_kernel_launches",
    "smre_dykstra_project_static", "smre_dykstra_schedule", "smre_batch_image_bytes",
    "smre_batch_create",
    "smre_batch_submit", "smre_batch_run", "smre_batch_poll", "smre_batch_retrieve",
    "smre_batch_project", "smre_batch_active", "smre_batch_item_spread", "smre_batch_per_side",
    "smre_batch_kernel_launches",
    "smre_batch_device_bytes", "smre_batch_last_error", "smre_batch_destroy",
    "smre_server_create", "smre_server_submit", "smre_server_wait", "smre_server_stats",
    "smre_server_destroy", "smre_admm_create", "smre_admm_solve", "smre_admm_kernel_launches",
    "smre_admm_projector", "smre_admm_destroy", "smre_admm_last_error",
)


class SmreError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class smre_params(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int), ("width", ctypes.c_int),
        ("sides", ctypes.POINTER(ctypes.c_int)), ("n_sides", ctypes.c_int),
        ("alpha", ctypes.c_double), ("cmode", ctypes.c_int),
        ("c_explicit", ctypes.POINTER(ctypes.c_double)),
        ("max_cycles", ctypes.c_int), ("tol", ctypes.c_double), ("tol_relative", ctypes.c_int),
        ("q_dtype", ctypes.c_int), ("icd_max_sweeps", ctypes.c_int),
        ("maxstat_draws", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("flags", ctypes.c_int),
        ("max_ctas", ctypes.c_int),
    ]


class smre_batch_params(ctypes.Structure):
    _fields_ = [
        ("sides", ctypes.POINTER(ctypes.c_int)), ("n_sides", ctypes.c_int),
        ("alpha", ctypes.c_double), ("cmode", ctypes.c_int),
        ("c_explicit", ctypes.POINTER(ctypes.c_double)),
        ("max_cycles", ctypes.c_int), ("tol", ctypes.c_double), ("tol_relative", ctypes.c_int),
        ("q_dtype", ctypes.c_int), ("max_images", ctypes.c_int),
        ("device_bytes", ctypes.c_size_t), ("flags", ctypes.c_int),
    ]


class smre_server_params(ctypes.Structure):
    _fields_ = [("batch", smre_batch_params), ("cycles_per_round", ctypes.c_int)]


class smre_server_counters(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
        ("waiting", ctypes.c_int), ("active", ctypes.c_int), ("peak_active", ctypes.c_int),
        ("rounds", ctypes.c_longlong),
        ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("max_s", ctypes.c_double),
        ("mean_s", ctypes.c_double), ("images_per_s", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class smre_admm_params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("radius", ctypes.c_int), ("rho1", ctypes.c_double),
                ("rho2", ctypes.c_double), ("gamma", ctypes.c_double), ("tv_iters", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("delta", ctypes.c_double),
                ("eps_incomplete", ctypes.c_int), ("icd_K", ctypes.c_int), ("icd_tol", ctypes.c_double)]


class smre_admm_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("dx", ctypes.c_double),
                ("residual", ctypes.c_double), ("dykstra_cycles", ctypes.c_longlong),
                ("seconds", ctypes.c_double), ("projection_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class smre_result(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int), ("status", ctypes.c_int),
        ("step", ctypes.c_double), ("rel_step", ctypes.c_double),
        ("max_violation", ctypes.c_double), ("windows", ctypes.c_longlong),
        ("max_tile_sweeps", ctypes.c_int), ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_PKG = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_PKG, "lib", "libsmre.so")


_lib = None


def load():
    """Load libsmre.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = lib_path()
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with `python -m paper_1503_03492_gb300.build`")
    lib = ctypes.CDLL(p)
    H = ctypes.c_void_p
    P = ctypes.POINTER
    st = ctypes.c_int
    sig = {
        "smre_bounds": (st, [P(smre_params), P(ctypes.c_double)]),
        "smre_dykstra_create": (st, [P(smre_params), ctypes.c_void_p, P(H)]),
        "smre_dykstra_project": (st, [H, ctypes.c_void_p, ctypes.c_void_p, P(smre_result)]),
        "smre_dykstra_project_incomplete": (st, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_double, P(smre_result)]),
        "smre_dykstra_set_stopping": (st, [H, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
        "smre_dykstra_bounds": (st, [H, P(ctypes.c_int), P(ctypes.c_double), ctypes.c_int]),
        "smre_dykstra_history": (st, [H, P(ctypes.c_double), ctypes.c_int, P(ctypes.c_int)]),
        "smre_dykstra_icd_sweeps": (st, [H, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]),
        "smre_dykstra_device_bytes": (ctypes.c_size_t, [H]),
        "smre_dykstra_kernel_launches": (ctypes.c_longlong, [H]),
        "smre_dykstra_schedule": (ctypes.c_int, [H]),
        "smre_dykstra_project_static": (st, [P(smre_params), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, P(smre_result)]),
        "smre_dykstra_destroy": (None, [H]),
        "smre_batch_image_bytes": (ctypes.c_size_t, [P(smre_batch_params), ctypes.c_int,
                                                     ctypes.c_int]),
        "smre_batch_create": (st, [P(smre_batch_params), ctypes.c_void_p, P(H)]),
        "smre_batch_submit": (st, [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                   P(ctypes.c_int)]),
        "smre_batch_run": (st, [H, ctypes.c_int]),
        "smre_batch_poll": (st, [H, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int)]),
        "smre_batch_retrieve": (st, [H, ctypes.c_int, ctypes.c_void_p, P(smre_result)]),
        "smre_batch_project": (st, [H, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int),
                                    P(ctypes.c_void_p), P(ctypes.c_void_p), P(smre_result)]),
        "smre_batch_active": (ctypes.c_int, [H]),
        "smre_batch_item_spread": (ctypes.c_int, [H, P(ctypes.c_int)]),
        "smre_batch_per_side": (ctypes.c_int, [H]),
        "smre_batch_kernel_launches": (ctypes.c_longlong, [H]),
        "smre_batch_device_bytes": (ctypes.c_size_t, [H]),
        "smre_batch_last_error": (ctypes.c_char_p, [H]),
        "smre_batch_destroy": (None, [H]),
        "smre_server_create": (st, [P(smre_server_params), ctypes.c_void_p, P(H)]),
        "smre_server_submit": (st, [H, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_void_p, P(ctypes.c_longlong)]),
        "smre_server_wait": (st, [H, ctypes.c_longlong, ctypes.c_double, P(smre_result)]),
        "smre_server_stats": (st, [H, P(smre_server_counters)]),
        "smre_server_destroy": (None, [H]),
        "smre_admm_create": (st, [P(smre_params), P(smre_admm_params), ctypes.c_void_p, P(H)]),
        "smre_admm_solve": (st, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 P(smre_admm_result)]),
        "smre_admm_kernel_launches": (ctypes.c_longlong, [H]),
        "smre_admm_projector": (H, [H]),
        "smre_admm_destroy": (None, [H]),
        "smre_admm_last_error": (ctypes.c_char_p, [H]),
        "smre_last_error": (ctypes.c_char_p, [H]),
        "smre_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------ marshalling

def _ptr(img):
    """(address, keepalive) of a float32 C-contiguous H x W image."""
    try:
        import torch
        if isinstance(img, torch.Tensor):
            if img.dtype != torch.float32 or not img.is_contiguous() or img.dim() != 2:
                raise ValueError("image must be a contiguous 2-D float32 tensor")
            return img.data_ptr(), img
    except ImportError:
        pass
    import numpy as np
    if isinstance(img, np.ndarray):
        if img.dtype != np.float32 or not img.flags.c_contiguous or img.ndim != 2:
            raise ValueError("image must be a C-contiguous 2-D float32 array")
        return img.ctypes.data, img
    raise TypeError(f"unsupported image type {type(img)}")


def _check(status, h=None, ok=(SMRE_OK,)):
    if status not in ok:
        msg = load().smre_last_error(h)
        raise SmreError(status, msg.decode() if msg else "")
    return status


def make_params(H, W, sides, alpha=0.9, cmode=SMRE_C_PERSET, c_explicit=None, max_cycles=200,
                tol=-1.0, tol_relative=False, icd_max_sweeps=0, maxstat_draws=0, seed=0, flags=0,
                max_ctas=0, q_dtype=0):
    """Build an ``smre_params`` (the arrays it points to are kept on the object)."""
    p = smre_params()
    sides_arr = (ctypes.c_int * len(sides))(*[int(s) for s in sides])
    p.height, p.width = int(H), int(W)
    p.sides, p.n_sides = sides_arr, len(sides)
    p.alpha, p.cmode = float(alpha), int(cmode)
    if c_explicit is not None:
        c_arr = (ctypes.c_double * len(c_explicit))(*[float(c) for c in c_explicit])
        p.c_explicit = c_arr
        p._c_keep = c_arr
    p.max_cycles, p.tol, p.tol_relative = int(max_cycles), float(tol), int(bool(tol_relative))
    p.q_dtype, p.icd_max_sweeps, p.maxstat_draws = int(q_dtype), int(icd_max_sweeps), int(maxstat_draws)
    p.seed, p.flags = int(seed), int(flags)
    p.max_ctas = int(max_ctas)
    p._sides_keep = sides_arr
    return p


# ------------------------------------------------------- C-named functions

def smre_version() -> str:
    return load().smre_version().decode()


def smre_last_error(h=None) -> str:
    m = load().smre_last_error(h)
    return m.decode() if m else ""


def smre_bounds(params: smre_params):
    out = (ctypes.c_double * params.n_sides)()
    _check(load().smre_bounds(ctypes.byref(params), out))
    return list(out)


def smre_dykstra_create(params: smre_params, stream=None):
    """Returns an opaque handle (int).  ``stream``: a cudaStream_t as int, a
    ``torch.cuda.Stream``, or None for the legacy default stream."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    _check(load().smre_dykstra_create(ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                      ctypes.byref(h)))
    return h.value


def smre_dykstra_project(h, x0, x, want_result=True):
    p0, k0 = _ptr(x0)
    p1, k1 = _ptr(x)
    res = smre_result()
    st = load().smre_dykstra_project(h, p0, p1, ctypes.byref(res) if want_result else None)
    _check(st, h, ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return res if want_result else None


def smre_dykstra_project_incomplete(h, x0, x, K=-1, tol=1e-3, want_result=True):
    p0, k0 = _ptr(x0)
    p1, k1 = _ptr(x)
    res = smre_result()
    st = load().smre_dykstra_project_incomplete(h, p0, p1, int(K), float(tol),
                                                ctypes.byref(res) if want_result else None)
    _check(st, h)
    return res if want_result else None


def smre_dykstra_set_stopping(h, max_cycles, tol, tol_relative=False):
    _check(load().smre_dykstra_set_stopping(h, int(max_cycles), float(tol), int(bool(tol_relative))), h)


def smre_dykstra_bounds(h, n=64):
    s = (ctypes.c_int * n)()
    c = (ctypes.c_double * n)()
    _check(load().smre_dykstra_bounds(h, s, c, n), h)
    out = {}
    for i in range(n):
        if s[i] <= 0:
            break
        out[s[i]] = c[i]
    return out


def smre_dykstra_history(h, n_max=1 << 20):
    import numpy as np
    n = ctypes.c_int()
    _check(load().smre_dykstra_history(h, None, 0, ctypes.byref(n)), h)
    buf = np.zeros((max(n.value, 1), 2))
    _check(load().smre_dykstra_history(h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       min(n.value, n_max), ctypes.byref(n)), h)
    return buf[:n.value]


def smre_dykstra_icd_sweeps(h):
    import numpy as np
    n = ctypes.c_int()
    _check(load().smre_dykstra_icd_sweeps(h, None, 0, ctypes.byref(n)), h)
    buf = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(load().smre_dykstra_icd_sweeps(h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                          n.value, ctypes.byref(n)), h)
    return buf[:n.value]


def smre_dykstra_device_bytes(h) -> int:
    return int(load().smre_dykstra_device_bytes(h))


def smre_dykstra_project_static(params: smre_params, x0, x, stream=None, want_result=True):
    """Standard projection without any device allocation (the library's static
    16 MiB scratch holds every intermediate buffer); see include/smre.h."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    p0, k0 = _ptr(x0)
    p1, k1 = _ptr(x)
    res = smre_result()
    st = load().smre_dykstra_project_static(ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                            p0, p1, ctypes.byref(res) if want_result else None)
    _check(st, None, ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return res if want_result else None


def smre_dykstra_schedule(h) -> int:
    """SMRE_SCHED_PERSISTENT, SMRE_SCHED_BATCHED or SMRE_SCHED_GROUPS."""
    return int(load().smre_dykstra_schedule(h))


def smre_dykstra_kernel_launches(h) -> int:
    return int(load().smre_dykstra_kernel_launches(h))


def smre_dykstra_destroy(h):
    load().smre_dykstra_destroy(h)


class Projector:
    """RAII wrapper: ``with Projector(H, W, sides, ...) as P: P.project(x0, x)``."""

    def __init__(self, H, W, sides, stream=None, **kw):
        self.params = make_params(H, W, sides, **kw)
        self.h = smre_dykstra_create(self.params, stream)

    def project(self, x0, x, want_result=True):
        return smre_dykstra_project(self.h, x0, x, want_result)

    def project_incomplete(self, x0, x, K=-1, tol=1e-3, want_result=True):
        return smre_dykstra_project_incomplete(self.h, x0, x, K, tol, want_result)

    def set_stopping(self, max_cycles, tol, tol_relative=False):
        smre_dykstra_set_stopping(self.h, max_cycles, tol, tol_relative)

    def bounds(self):
        return smre_dykstra_bounds(self.h)

    def history(self):
        return smre_dykstra_history(self.h)

    def icd_sweeps(self):
        return smre_dykstra_icd_sweeps(self.h)

    def device_bytes(self):
        return smre_dykstra_device_bytes(self.h)

    def kernel_launches(self):
        return smre_dykstra_kernel_launches(self.h)

    def schedule(self):
        return smre_dykstra_schedule(self.h)

    def close(self):
        if self.h:
            smre_dykstra_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batches

def make_batch_params(sides, alpha=0.9, cmode=SMRE_C_PERSET, c_explicit=None, max_cycles=200,
                      tol=-1.0, tol_relative=False, q_dtype=SMRE_Q_FP32, max_images=64,
                      device_bytes=1 << 30, flags=0):
    """Build an ``smre_batch_params`` (the arrays it points to are kept on the object)."""
    p = smre_batch_params()
    sides_arr = (ctypes.c_int * len(sides))(*[int(s) for s in sides])
    p.sides, p.n_sides = sides_arr, len(sides)
    p.alpha, p.cmode = float(alpha), int(cmode)
    if c_explicit is not None:
        c_arr = (ctypes.c_double * len(c_explicit))(*[float(c) for c in c_explicit])
        p.c_explicit = c_arr
        p._c_keep = c_arr
    p.max_cycles, p.tol, p.tol_relative = int(max_cycles), float(tol), int(bool(tol_relative))
    p.q_dtype, p.max_images, p.device_bytes = int(q_dtype), int(max_images), int(device_bytes)
    p.flags = int(flags)
    p._sides_keep = sides_arr
    return p


def _bcheck(status, b=None, ok=(SMRE_OK,)):
    if status not in ok:
        msg = load().smre_batch_last_error(b)
        raise SmreError(status, msg.decode() if msg else "")
    return status


def smre_batch_image_bytes(params: smre_batch_params, H, W) -> int:
    return int(load().smre_batch_image_bytes(ctypes.byref(params), int(H), int(W)))


def smre_batch_create(params: smre_batch_params, stream=None):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    b = ctypes.c_void_p()
    _bcheck(load().smre_batch_create(ctypes.byref(params), ctypes.c_void_p(stream or 0),
                                     ctypes.byref(b)))
    return b.value


def smre_batch_submit(b, x0) -> int:
    """Admit x0 (H x W); returns its slot, or -1 when there is no room now."""
    p0, k0 = _ptr(x0)
    H, W = x0.shape
    slot = ctypes.c_int(-1)
    _bcheck(load().smre_batch_submit(b, int(H), int(W), p0, ctypes.byref(slot)), b)
    return slot.value


def smre_batch_run(b, cycles):
    _bcheck(load().smre_batch_run(b, int(cycles)), b)


def smre_batch_poll(b, max_done=4096):
    done = (ctypes.c_int * max_done)()
    n = ctypes.c_int()
    _bcheck(load().smre_batch_poll(b, done, max_done, ctypes.byref(n)), b)
    return [done[i] for i in range(n.value)]


def smre_batch_retrieve(b, slot, x=None):
    res = smre_result()
    px, kx = _ptr(x) if x is not None else (None, None)
    _bcheck(load().smre_batch_retrieve(b, int(slot), px, ctypes.byref(res)), b,
            ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return res


def smre_batch_project(b, x0s, xs):
    n = len(x0s)
    keep = [_ptr(a) for a in x0s] + [_ptr(a) for a in xs]
    Hs = (ctypes.c_int * n)(*[int(a.shape[0]) for a in x0s])
    Ws = (ctypes.c_int * n)(*[int(a.shape[1]) for a in x0s])
    p0 = (ctypes.c_void_p * n)(*[k[0] for k in keep[:n]])
    p1 = (ctypes.c_void_p * n)(*[k[0] for k in keep[n:]])
    res = (smre_result * n)()
    _bcheck(load().smre_batch_project(b, n, Hs, Ws, p0, p1, res), b,
            ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return list(res)


def smre_batch_active(b) -> int:
    return int(load().smre_batch_active(b))


def smre_batch_item_spread(b):
    """(spread, tuned): the batch's current item spread and whether
    SMRE_BF_AUTOTUNE chose it (1 measured, 2 cached, 0 not tuned)."""
    t = ctypes.c_int(0)
    v = int(load().smre_batch_item_spread(b, ctypes.byref(t)))
    return v, int(t.value)


def smre_batch_per_side(b) -> bool:
    """True when the batch's step launches run one per side (SMRE_BF_PER_SIDE
    or chosen by SMRE_BF_AUTOTUNE)."""
    return bool(load().smre_batch_per_side(b))


def smre_batch_kernel_launches(b) -> int:
    return int(load().smre_batch_kernel_launches(b))


def smre_batch_device_bytes(b) -> int:
    return int(load().smre_batch_device_bytes(b))


def smre_batch_last_error(b=None) -> str:
    m = load().smre_batch_last_error(b)
    return m.decode() if m else ""


def smre_batch_destroy(b):
    load().smre_batch_destroy(b)


class Batch:
    """RAII wrapper over a batch: ``with Batch(sides, ...) as B: B.project([x0...], [x...])``."""

    def __init__(self, sides, stream=None, **kw):
        self.params = make_batch_params(sides, **kw)
        self.b = smre_batch_create(self.params, stream)

    def image_bytes(self, H, W):
        return smre_batch_image_bytes(self.params, H, W)

    def project(self, x0s, xs):
        return smre_batch_project(self.b, x0s, xs)

    def submit(self, x0):
        return smre_batch_submit(self.b, x0)

    def run(self, cycles):
        smre_batch_run(self.b, cycles)

    def poll(self):
        return smre_batch_poll(self.b)

    def retrieve(self, slot, x=None):
        return smre_batch_retrieve(self.b, slot, x)

    def active(self):
        return smre_batch_active(self.b)

    def item_spread(self):
        return smre_batch_item_spread(self.b)

    def per_side(self):
        return smre_batch_per_side(self.b)

    def kernel_launches(self):
        return smre_batch_kernel_launches(self.b)

    def device_bytes(self):
        return smre_batch_device_bytes(self.b)

    def close(self):
        if self.b:
            smre_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

def smre_server_create(batch_params: smre_batch_params, cycles_per_round=4, stream=None):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    p = smre_server_params()
    p.batch = batch_params
    p.cycles_per_round = int(cycles_per_round)
    s = ctypes.c_void_p()
    _check(load().smre_server_create(ctypes.byref(p), ctypes.c_void_p(stream or 0),
                                     ctypes.byref(s)))
    return s.value


def smre_server_submit(s, x0, x) -> int:
    """Queue x0 (H x W); the result lands in x (same shape).  Returns the ticket."""
    p0, k0 = _ptr(x0)
    p1, k1 = _ptr(x)
    H, W = x0.shape
    t = ctypes.c_longlong()
    _check(load().smre_server_submit(s, int(H), int(W), p0, p1, ctypes.byref(t)))
    return t.value


def smre_server_wait(s, ticket, timeout_s=-1.0):
    """Result of a request (None if it did not finish within timeout_s)."""
    res = smre_result()
    st = load().smre_server_wait(s, int(ticket), float(timeout_s), ctypes.byref(res))
    if st == SMRE_ETIMEOUT:
        return None
    _check(st, None, ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return res


def smre_server_stats(s):
    c = smre_server_counters()
    load().smre_server_stats(s, ctypes.byref(c))
    return c


def smre_server_destroy(s):
    load().smre_server_destroy(s)


class Server:
    """Continuous-batching request loop: ``with Server(sides, ...) as S: t = S.submit(x0, x); S.wait(t)``.
    The output arrays passed to ``submit`` are kept alive until their request is waited for."""

    def __init__(self, sides, cycles_per_round=4, stream=None, **batch_kw):
        self.params = make_batch_params(sides, **batch_kw)
        self.s = smre_server_create(self.params, cycles_per_round, stream)
        self._keep = {}

    def submit(self, x0, x):
        t = smre_server_submit(self.s, x0, x)
        self._keep[t] = x
        return t

    def wait(self, ticket, timeout_s=-1.0):
        r = smre_server_wait(self.s, ticket, timeout_s)
        if r is not None:
            self._keep.pop(ticket, None)
        return r

    def stats(self):
        return smre_server_stats(self.s)

    def close(self):
        if self.s:
            smre_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------- ADMM

def make_admm_params(sigma, radius=0, rho1=1.0, rho2=1.0, gamma=0.0, tv_iters=20, max_iters=100,
                     delta=-1.0, eps_incomplete=False, icd_K=-1, icd_tol=1e-3) -> smre_admm_params:
    p = smre_admm_params()
    p.sigma, p.radius = float(sigma), int(radius)
    p.rho1, p.rho2, p.gamma = float(rho1), float(rho2), float(gamma)
    p.tv_iters, p.max_iters, p.delta = int(tv_iters), int(max_iters), float(delta)
    p.eps_incomplete, p.icd_K, p.icd_tol = int(bool(eps_incomplete)), int(icd_K), float(icd_tol)
    return p


def smre_admm_last_error(a=None) -> str:
    m = load().smre_admm_last_error(a)
    return m.decode() if m else ""


def _acheck(status, a=None, ok=(SMRE_OK,)):
    if status not in ok:
        raise SmreError(status, smre_admm_last_error(a))
    return status


def smre_admm_create(proj: smre_params, ap: smre_admm_params, stream=None):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    a = ctypes.c_void_p()
    _acheck(load().smre_admm_create(ctypes.byref(proj), ctypes.byref(ap), ctypes.c_void_p(stream or 0),
                                    ctypes.byref(a)))
    return a.value


def smre_admm_solve(a, I, x, z=None, eps=None):
    """ADMM on the observed image I (device, H x W); the final x (and z, eps when
    given) land in the caller's device images.  Returns an smre_admm_result."""
    pI, kI = _ptr(I)
    px, kx = _ptr(x)
    pz, kz = _ptr(z) if z is not None else (None, None)
    pe, ke = _ptr(eps) if eps is not None else (None, None)
    res = smre_admm_result()
    st = load().smre_admm_solve(a, pI, px, pz, pe, ctypes.byref(res))
    _acheck(st, a, ok=(SMRE_OK, SMRE_ENOTCONVERGED))
    return res


def smre_admm_kernel_launches(a) -> int:
    return load().smre_admm_kernel_launches(a)


def smre_admm_projector(a):
    return load().smre_admm_projector(a)


def smre_admm_destroy(a):
    load().smre_admm_destroy(a)


class Admm:
    """The full estimator: ``with Admm(H, W, sides, sigma=2.0, ...) as A: A.solve(I, x)``.
    Keywords of ``make_params`` set the eps-step's projection (cycle cap,
    tolerance, bounds); those of ``make_admm_params`` the outer loop."""

    _AKEYS = ("radius", "rho1", "rho2", "gamma", "tv_iters", "max_iters", "delta", "eps_incomplete",
              "icd_K", "icd_tol")

    def __init__(self, H, W, sides, sigma, stream=None, **kw):
        akw = {k: kw.pop(k) for k in list(kw) if k in self._AKEYS}
        self.params = make_params(H, W, sides, **kw)
        self.aparams = make_admm_params(sigma, **akw)
        self.a = smre_admm_create(self.params, self.aparams, stream)

    def solve(self, I, x, z=None, eps=None):
        return smre_admm_solve(self.a, I, x, z, eps)

    def kernel_launches(self):
        return smre_admm_kernel_launches(self.a)

    def projection_launches(self):
        return smre_dykstra_kernel_launches(smre_admm_projector(self.a))

    def close(self):
        if self.a:
            smre_admm_destroy(self.a)
            self.a = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
