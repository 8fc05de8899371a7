"""Python binding of libhsma.so, the GB300 HSMA pair-sum library.

Argument marshalling only: every step of an evaluation runs in the library's
CUDA kernels.  The functions carry the names of the C entry points in
``include/hsma.h``; arrays may be NumPy arrays (host) or torch tensors (host
or CUDA), float64 and contiguous.  There is no CPU fallback: without the
compiled library every call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsma.so")

HSMA_OK = 0
HSMA_PENDING = 1
ERRORS = {
    -1: "HSMA_ERR_ARG", -2: "HSMA_ERR_NOT_NEUTRAL", -3: "HSMA_ERR_OUT_OF_SLAB",
    -4: "HSMA_ERR_NOMEM", -5: "HSMA_ERR_BUDGET", -6: "HSMA_ERR_TIMEOUT",
    -7: "HSMA_ERR_CUDA", -8: "HSMA_ERR_NUMERIC",
}

# name -> (restype, argtypes); every symbol include/hsma.h declares
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_int64
SIGNATURES = {
    "hsma_create": (_I, [ctypes.POINTER(_D), _I, _I, _I, _D, _D, ctypes.POINTER(_P)]),
    "hsma_set_option": (_I, [_P, ctypes.c_char_p, _D]),
    "hsma_set_stream": (_I, [_P, _P]),
    "hsma_eval": (_I, [_P, _P, _P, _L, _P, _P]),
    "hsma_eval_ex": (_I, [_P, _P, _P, _L, _P, _P, _P]),
    "hsma_get_info": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_D)]),
    "hsma_get_array": (_I, [_P, ctypes.c_char_p, _P, _L]),
    "hsma_destroy": (None, [_P]),
    "hsma_last_error": (ctypes.c_char_p, [_P]),
    "hsma_server_create": (_I, [_I, _D, _I, ctypes.POINTER(_P)]),
    "hsma_submit": (_I, [_P, _P, _P, _L, ctypes.POINTER(_D), _I, _I, ctypes.POINTER(ctypes.c_uint64)]),
    "hsma_poll": (_I, [_P, ctypes.c_uint64, _P, _P]),
    "hsma_server_step": (_I, [_P]),
    "hsma_geometry_array": (_I, [ctypes.POINTER(_D), _I, _I, _I, _D, _D, _D, _I, _I, _D, _I,
                                 ctypes.c_char_p, _P, _L]),
    "hsma_pair_sum_static": (_I, [_P, _L, _P, _L, _P, _I, _P]),
    "hsma_md_create": (_I, [_P, _P, _P, _P, _L, _D, _D, _D, _D, _D, _D, ctypes.POINTER(_P)]),
    "hsma_md_set_option": (_I, [_P, ctypes.c_char_p, _D]),
    "hsma_md_run": (_I, [_P, _L, _P]),
    "hsma_md_get": (_I, [_P, ctypes.c_char_p, _P, _L]),
    "hsma_md_last_error": (ctypes.c_char_p, [_P]),
    "hsma_md_destroy": (None, [_P]),
}

_lib = None


class HSMAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhsma.so is not built ({LIB_PATH}); run "
                               "paper_2104_05260_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(h, rc):
    if rc < 0:
        msg = lib().hsma_last_error(h)
        raise HSMAError(rc, msg.decode() if msg else "")
    return rc


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, n):
    """Pointer to a contiguous float64 array of at least n elements."""
    if _is_torch(a):
        if a.dtype != __import__("torch").float64 or not a.is_contiguous() or a.numel() < n:
            raise ValueError("torch tensors must be contiguous float64 of the right size")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous or a.size < n:
        raise ValueError("arrays must be contiguous float64 of the right size")
    return ctypes.c_void_p(a.ctypes.data)


def _as_input(a):
    if _is_torch(a):
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _like(a, shape):
    if _is_torch(a):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=a.device)
    return np.empty(shape, dtype=np.float64)


# ---------------------------------------------------------------- C names
def hsma_create(box, dims, p, M, gamma_top=0.0, gamma_bot=0.0):
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    h = ctypes.c_void_p()
    rc = lib().hsma_create(b, int(dims), int(p), int(M), float(gamma_top), float(gamma_bot),
                           ctypes.byref(h))
    if rc != HSMA_OK:
        raise HSMAError(rc, "hsma_create failed")
    return h


def hsma_set_option(h, key, value):
    return _check(h, lib().hsma_set_option(h, key.encode(), float(value)))


def hsma_set_stream(h, stream_ptr):
    return _check(h, lib().hsma_set_stream(h, ctypes.c_void_p(stream_ptr)))


def hsma_eval(h, x, q, forces=True, potential=False):
    """Returns (energy, forces or None, potential or None)."""
    x = _as_input(x)
    q = _as_input(q)
    N = int(q.shape[0])
    e = ctypes.c_double()
    f = _like(x, (N, 3)) if forces else None
    pot = _like(q, (N,)) if potential else None
    rc = lib().hsma_eval_ex(h, _ptr(x, 3 * N), _ptr(q, N), N, ctypes.cast(ctypes.byref(e), ctypes.c_void_p),
                            _ptr(f, 3 * N) if f is not None else None,
                            _ptr(pot, N) if pot is not None else None)
    _check(h, rc)
    return e.value, f, pot


def hsma_eval_into(h, x, q, N, energy_buf, forces_buf):
    """Zero-allocation form of hsma_eval with caller-owned outputs."""
    return _check(h, lib().hsma_eval(h, _ptr(x, 3 * N), _ptr(q, N), int(N), _ptr(energy_buf, 1),
                                     _ptr(forces_buf, 3 * N) if forces_buf is not None else None))


def hsma_get_info(h, key):
    v = ctypes.c_double()
    _check(h, lib().hsma_get_info(h, key.encode(), ctypes.byref(v)))
    return v.value


def hsma_get_array(h, name, n):
    out = np.empty(int(n), dtype=np.float64)
    _check(h, lib().hsma_get_array(h, name.encode(), ctypes.c_void_p(out.ctypes.data), int(n)))
    return out


def hsma_destroy(h):
    if h is not None and h.value:
        lib().hsma_destroy(h)


def hsma_last_error(h):
    m = lib().hsma_last_error(h)
    return m.decode() if m else ""


def hsma_server_create(slots, budget_bytes, precision=1):
    h = ctypes.c_void_p()
    rc = lib().hsma_server_create(int(slots), float(budget_bytes), int(precision), ctypes.byref(h))
    if rc != HSMA_OK:
        raise HSMAError(rc, "hsma_server_create failed")
    return h


def hsma_submit(server, x, q, box, p, M):
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    N = int(q.shape[0])
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    t = ctypes.c_uint64()
    _check(server, lib().hsma_submit(server, _ptr(x, 3 * N), _ptr(q, N), N, b, int(p), int(M),
                                     ctypes.byref(t)))
    return t.value


def hsma_poll(server, ticket, N, out=None):
    """Returns None while pending, else (energy, forces).  out, an (N, 3)
    float64 array, receives the forces; without it one is allocated."""
    e = ctypes.c_double()
    f = out if out is not None else np.empty((N, 3), dtype=np.float64)
    if f.shape != (N, 3) or f.dtype != np.float64 or not f.flags.c_contiguous:
        raise ValueError("out must be a contiguous float64 array of shape (N, 3)")
    rc = lib().hsma_poll(server, ctypes.c_uint64(ticket), ctypes.cast(ctypes.byref(e), ctypes.c_void_p),
                         ctypes.c_void_p(f.ctypes.data))
    if rc == HSMA_PENDING:
        return None
    _check(server, rc)
    return e.value, f


def hsma_server_step(server):
    return _check(server, lib().hsma_server_step(server))


def hsma_geometry_array(box, dims, p, M, name, n, gamma_top=0.0, gamma_bot=0.0, lam=0.0,
                        n_monitor=0, G=0, grad_weight=0.0, surface_rule=0):
    """Host-only geometry array (no GPU); see include/hsma.h."""
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    out = np.empty(int(n), dtype=np.float64)
    rc = lib().hsma_geometry_array(b, int(dims), int(p), int(M), float(gamma_top), float(gamma_bot),
                                   float(lam), int(n_monitor), int(G), float(grad_weight),
                                   int(surface_rule), name.encode(),
                                   ctypes.c_void_p(out.ctypes.data), int(n))
    if rc != HSMA_OK:
        raise HSMAError(rc, "hsma_geometry_array(" + name + ") failed")
    return out


def hsma_pair_sum_static(targets, sources, out, precision=1, stream_ptr=0):
    """Direct pair sum with the library's static scratch (no device allocation).

    targets (n_t, 3), sources (n_s, 4: x, y, z, q) and out (n_t, 4: phi,
    dphi/dx, dphi/dy, dphi/dz) are float64 CUDA tensors on one device; the
    call runs with that device current, the work is enqueued on the given
    stream and is complete when that stream reaches it.
    """
    if not all(_is_torch(a) and a.is_cuda for a in (targets, sources, out)):
        raise ValueError("hsma_pair_sum_static takes CUDA tensors only")
    if not (targets.device == sources.device == out.device):
        raise ValueError("targets, sources and out must be on the same CUDA device")
    import torch
    nt, ns = int(targets.shape[0]), int(sources.shape[0])
    with torch.cuda.device(targets.device):
        rc = lib().hsma_pair_sum_static(_ptr(targets, 3 * nt), nt, _ptr(sources, 4 * ns), ns,
                                        _ptr(out, 4 * nt), int(precision), ctypes.c_void_p(stream_ptr))
    if rc != HSMA_OK:
        raise HSMAError(rc, "hsma_pair_sum_static failed")
    return out


class HSMA:
    """One HSMA set-up (box, order, surface points) bound to a handle."""

    def __init__(self, box, dims=3, p=6, M=800, gamma_top=0.0, gamma_bot=0.0, **options):
        self.h = hsma_create(box, dims, p, M, gamma_top, gamma_bot)
        for k, v in options.items():
            hsma_set_option(self.h, k, v)

    def set_option(self, key, value):
        hsma_set_option(self.h, key, value)

    def eval(self, x, q, forces=True, potential=False):
        return hsma_eval(self.h, x, q, forces, potential)

    def info(self, key):
        return hsma_get_info(self.h, key)

    def array(self, name, n):
        return hsma_get_array(self.h, name, n)

    def close(self):
        if self.h is not None:
            hsma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- MD loop
def _md_check(m, rc):
    if rc < 0:
        msg = lib().hsma_md_last_error(m)
        raise HSMAError(rc, msg.decode() if msg else "")
    return rc


def hsma_md_create(h, x, v, q, mass=1.0, dt=0.01, kT=1.0, tdamp=0.0, lj_sigma=1.0, lj_eps=1.0):
    x, v, q = _as_input(x), _as_input(v), _as_input(q)
    N = q.shape[0] if _is_torch(q) else q.size
    out = ctypes.c_void_p()
    rc = lib().hsma_md_create(h, _ptr(x, 3 * N), _ptr(v, 3 * N), _ptr(q, N), int(N), float(mass), float(dt),
                              float(kT), float(tdamp), float(lj_sigma), float(lj_eps), ctypes.byref(out))
    if rc != HSMA_OK:
        msg = lib().hsma_last_error(h)
        raise HSMAError(rc, "hsma_md_create failed" + (": " + msg.decode() if msg else ""))
    return out


def hsma_md_set_option(m, key, value):
    return _md_check(m, lib().hsma_md_set_option(m, key.encode(), float(value)))


def hsma_md_run(m, steps, thermo=None):
    """Advance steps; thermo (steps x 6, float64, host or CUDA) or None."""
    p = _ptr(thermo, 6 * steps) if thermo is not None else None
    return _md_check(m, lib().hsma_md_run(m, int(steps), p))


def hsma_md_get(m, name, n):
    out = np.empty(int(n), dtype=np.float64)
    _md_check(m, lib().hsma_md_get(m, name.encode(), ctypes.c_void_p(out.ctypes.data), int(n)))
    return out


def hsma_md_destroy(m):
    lib().hsma_md_destroy(m)


class MD:
    """The MD loop of the validation workload (include/hsma.h, hsma_md_*)
    around an HSMA handle."""

    def __init__(self, hsma, x, v, q, **kw):
        self.hsma = hsma
        self.N = len(q)
        self.m = hsma_md_create(hsma.h, x, v, q, **kw)

    def set_option(self, key, value):
        hsma_md_set_option(self.m, key, value)
        if key == "rdf_bins":
            self.rdf_bins = int(value)
        if key == "zhist_bins":
            self.zhist_bins = int(value)

    def run(self, steps):
        t = np.empty((int(steps), 6))
        hsma_md_run(self.m, steps, t if steps > 0 else None)
        return t

    def get(self, name):
        n = {"state": 6}.get(name)
        if name == "rdf":
            n = int(3 * self._rdf_bins())
        if name == "zhist":
            n = int(2 * getattr(self, "zhist_bins", 100))
        return hsma_md_get(self.m, name, n if n else 3 * self.N).reshape(
            (-1, 3) if name in ("x", "v", "x_unwrapped", "forces") else (-1,))

    def _rdf_bins(self):
        return getattr(self, "rdf_bins", 200)

    def close(self):
        if self.m is not None:
            hsma_md_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
