"""ctypes binding of libaniso.so: the C ABI of include/aniso.h under the same
names.  Argument marshalling only -- every step of the method runs in the
library's CUDA kernels; there is no Python or CPU fallback, and loading fails
loudly when the library has not been built."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaniso.so")

# status codes
ANISO_OK = 0
ANISO_ERR_ARG = 1
ANISO_ERR_STATE = 2
ANISO_ERR_CUDA = 3
ANISO_ERR_NONFINITE = 4
ANISO_ERR_TIMEOUT = 5
ANISO_ERR_OOM = 6
ANISO_ERR_UNSUPPORTED = 7
# boundary conditions
ANISO_BC_ZEROFLUX = 0
ANISO_BC_PERIODIC = 1
ANISO_BC_DIRICHLET = 2
# options
ANISO_OPT_PRECISION = 0
ANISO_OPT_FIELD_FP16 = 1
ANISO_OPT_KAHAN = 2
ANISO_OPT_LIMITER = 3
ANISO_OPT_ORDER = 4
ANISO_OPT_STREAM = 5
ANISO_OPT_GRAPH = 6
ANISO_OPT_PROFILE = 7
ANISO_OPT_FAST_PATH = 8
ANISO_OPT_SEGMENT = 9
ANISO_OPT_BLOCK_WARPS = 10
ANISO_OPT_SCHEME = 11
ANISO_OPT_DIAGNOSTICS = 12
ANISO_OPT_TMA_LINES = 13
ANISO_OPT_TMEM = 14
ANISO_OPT_CLUSTER_LINES = 15
ANISO_SCHEME_2STEP = 0
ANISO_SCHEME_4STEP = 1
ANISO_SCHEME_EXPLICIT = 2
ANISO_PREC_FP64 = 0
ANISO_PREC_FP32 = 1
ANISO_LIM_VANLEER = 0
ANISO_LIM_ARITH = 1
ANISO_LIM_MINMOD = 2
ANISO_LIM_MC = 3
ANISO_ORDER_XY = 0
ANISO_ORDER_YX = 1
ANISO_ORDER_ALTERNATE = 2
ANISO_DIR_X = 0
ANISO_DIR_Y = 1
ANISO_KERNEL_XSWEEP = 0
ANISO_KERNEL_YSWEEP = 1
ANISO_KERNEL_TRANSPOSE = 2

EXPORTED = ("aniso_create", "aniso_set_option", "aniso_set_field", "aniso_step", "aniso_sweep",
            "aniso_total", "aniso_get_state", "aniso_set_state", "aniso_sync",
            "aniso_kernel_times", "aniso_destroy", "aniso_last_error", "aniso_batch_create",
            "aniso_step_batched", "aniso_step_batched_host", "aniso_batch_diagnostics", "aniso_batch_destroy",
            "aniso_step_noalloc",
            "aniso_batch_autotune", "aniso_autotune_candidate", "aniso_set_source",
            "aniso_batch_kernel_count", "aniso_set_nonlinear",
            "aniso3_create", "aniso3_set_option", "aniso3_set_field", "aniso3_step",
            "aniso3_total", "aniso3_sync", "aniso3_destroy")


class AnisoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("aniso error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load():
    """Load libaniso.so (built by paper_1008_0861_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libaniso.so is missing at %s: build it with "
                           "paper_1008_0861_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    P = ctypes.POINTER
    sig = {
        "aniso_create": (i, [i, i, d, d, d, d, i, P(vp)]),
        "aniso_set_option": (i, [vp, i, ll]),
        "aniso_set_field": (i, [vp, vp, vp]),
        "aniso_step": (i, [vp, vp, d, i]),
        "aniso_sweep": (i, [vp, i, vp, vp, d]),
        "aniso_total": (i, [vp, vp, P(d), P(d), P(d), P(ll)]),
        "aniso_get_state": (i, [vp, P(ll), vp]),
        "aniso_set_state": (i, [vp, ll, vp]),
        "aniso_sync": (i, [vp]),
        "aniso_kernel_times": (i, [vp, vp, i, P(d), P(ll), i]),
        "aniso_destroy": (None, [vp]),
        "aniso_last_error": (ctypes.c_char_p, []),
        "aniso_batch_create": (i, [i, P(vp), P(vp)]),
        "aniso_step_batched": (i, [vp, P(vp), P(d), P(i)]),
        "aniso_step_batched_host": (i, [vp, P(vp), P(d), P(i)]),
        "aniso_batch_diagnostics": (i, [vp, P(d), ll, P(i)]),
        "aniso_batch_destroy": (None, [vp]),
        "aniso_step_noalloc": (i, [i, i, d, d, d, d, i, i, vp, vp, vp, d, i, vp]),
        "aniso_batch_autotune": (i, [vp, P(vp), P(d), i, i, P(i), P(d)]),
        "aniso_autotune_candidate": (i, [i, P(i), P(i), P(i)]),
        "aniso_set_source": (i, [vp, vp]),
        "aniso_batch_kernel_count": (i, [vp, P(ll)]),
        "aniso_set_nonlinear": (i, [vp, d, d]),
        "aniso3_create": (i, [i, i, i, d, d, d, d, d, i, P(vp)]),
        "aniso3_set_option": (i, [vp, i, ll]),
        "aniso3_set_field": (i, [vp, vp, vp, vp]),
        "aniso3_step": (i, [vp, vp, d, i]),
        "aniso3_total": (i, [vp, vp, P(d), P(d), P(d), P(ll)]),
        "aniso3_sync": (i, [vp]),
        "aniso3_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Device address of a torch tensor (or an int address)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _check(rc):
    if rc != ANISO_OK:
        raise AnisoError(rc, load().aniso_last_error().decode())


def aniso_last_error():
    return load().aniso_last_error().decode()


def aniso_create(nx, ny, dx, dy, chi_par, chi_perp=0.0, bc=ANISO_BC_PERIODIC):
    h = ctypes.c_void_p()
    _check(load().aniso_create(int(nx), int(ny), float(dx), float(dy), float(chi_par),
                               float(chi_perp), int(bc), ctypes.byref(h)))
    return h


def aniso_set_option(h, key, value):
    _check(load().aniso_set_option(h, int(key), int(value)))


def aniso_set_field(h, bx, by):
    _check(load().aniso_set_field(h, _ptr(bx), _ptr(by)))


def aniso_step(h, T, dt, nsteps=1):
    _check(load().aniso_step(h, _ptr(T), float(dt), int(nsteps)))


def aniso_sweep(h, direction, Tin, Tout, dt):
    _check(load().aniso_sweep(h, int(direction), _ptr(Tin), _ptr(Tout), float(dt)))


def aniso_total(h, T):
    """(sum, min, max, nonfinite count) of T, FP64 sum."""
    s, lo, hi, nf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    _check(load().aniso_total(h, _ptr(T), ctypes.byref(s), ctypes.byref(lo), ctypes.byref(hi),
                              ctypes.byref(nf)))
    return s.value, lo.value, hi.value, nf.value


def aniso_get_state(h, lo_out=None):
    c = ctypes.c_longlong()
    _check(load().aniso_get_state(h, ctypes.byref(c), _ptr(lo_out)))
    return c.value


def aniso_set_state(h, step_counter, lo_in=None):
    _check(load().aniso_set_state(h, int(step_counter), _ptr(lo_in)))


def aniso_sync(h):
    _check(load().aniso_sync(h))


def aniso_kernel_times(h=None, batch=None, kind=ANISO_KERNEL_XSWEEP, reset=False):
    ms, n = ctypes.c_double(), ctypes.c_longlong()
    _check(load().aniso_kernel_times(h, batch, int(kind), ctypes.byref(ms), ctypes.byref(n),
                                     int(bool(reset))))
    return ms.value, n.value


def aniso_destroy(h):
    if h:
        load().aniso_destroy(h)


def aniso_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                              for h in handles])
    b = ctypes.c_void_p()
    _check(load().aniso_batch_create(len(handles), arr, ctypes.byref(b)))
    return b


def aniso_step_batched(batch, Ts, dts, nsteps):
    n = len(Ts)
    Tarr = (ctypes.c_void_p * n)(*[t.data_ptr() if hasattr(t, "data_ptr") else int(t) for t in Ts])
    darr = (ctypes.c_double * n)(*[float(x) for x in dts])
    narr = (ctypes.c_int * n)(*[int(x) for x in nsteps])
    _check(load().aniso_step_batched(batch, Tarr, darr, narr))


def aniso_step_batched_host(batch, Ts, dts, nsteps):
    """aniso_step_batched on host arrays (numpy arrays or CPU tensors, pinned
    or not, in the batch's precision); returns when they hold the result."""
    n = len(Ts)
    ptrs = []
    for t in Ts:
        if hasattr(t, "data_ptr"):
            if getattr(t, "is_cuda", False):
                raise ValueError("aniso_step_batched_host takes host arrays")
            ptrs.append(t.data_ptr())
        else:
            ptrs.append(t.ctypes.data)
    Tarr = (ctypes.c_void_p * n)(*ptrs)
    darr = (ctypes.c_double * n)(*[float(x) for x in dts])
    narr = (ctypes.c_int * n)(*[int(x) for x in nsteps])
    _check(load().aniso_step_batched_host(batch, Tarr, darr, narr))


def aniso_batch_diagnostics(batch, n_grids):
    """Per-step (sum, min, max) of the last diagnostics-enabled batched call as
    a numpy array [n_grids, steps, 3] (NaN where a grid took no such step)."""
    import numpy as np
    steps = ctypes.c_int()
    _check(load().aniso_batch_diagnostics(batch, None, 0, ctypes.byref(steps)))
    out = np.empty((n_grids, steps.value, 3), dtype=np.float64)
    _check(load().aniso_batch_diagnostics(batch, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          out.size, ctypes.byref(steps)))
    return out


def aniso_batch_autotune(batch, Ts, dts, nsteps=2, reps=3):
    """Time the batched fast path's block shapes on copies of Ts and keep the
    fastest in every handle of the batch.  Returns (index, ms per call) or
    (-1, 0.0) when no grid is on the fast path."""
    n = len(Ts)
    Tarr = (ctypes.c_void_p * n)(*[t.data_ptr() if hasattr(t, "data_ptr") else int(t) for t in Ts])
    darr = (ctypes.c_double * n)(*[float(x) for x in dts])
    ch, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().aniso_batch_autotune(batch, Tarr, darr, int(nsteps), int(reps), ctypes.byref(ch),
                                       ctypes.byref(ms)))
    return ch.value, ms.value


def aniso_autotune_candidate(index):
    """(fast-path option, warps per block, chunks per lane) of a tuner choice."""
    f, w, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().aniso_autotune_candidate(int(index), ctypes.byref(f), ctypes.byref(w), ctypes.byref(s)))
    return f.value, w.value, s.value


def aniso_set_source(h, Q):
    """Source term Q (device tensor [ny][nx], handle precision) applied as
    T += dt Q before every step; None removes it."""
    _check(load().aniso_set_source(h, _ptr(Q)))


def aniso_set_nonlinear(h, alpha, t_ref=1.0):
    """chi_par * (max(T,0)/t_ref)^alpha with harmonic face averaging (alpha = 0: off)."""
    _check(load().aniso_set_nonlinear(h, float(alpha), float(t_ref)))


def aniso_batch_kernel_count(batch):
    """Kernel launches per aniso_step_batched call of the current plan."""
    k = ctypes.c_longlong()
    _check(load().aniso_batch_kernel_count(batch, ctypes.byref(k)))
    return k.value


def aniso_batch_destroy(batch):
    if batch:
        load().aniso_batch_destroy(batch)


def aniso_step_noalloc(nx, ny, dx, dy, chi_par, chi_perp, bc, precision, bx, by, T, dt, nsteps,
                       stream=None):
    """aniso_step without device allocation (fixed 20 MiB scratch array in
    the library; see include/aniso.h).  For callers that may not allocate GPU
    memory; serialise calls, they share that array."""
    _check(load().aniso_step_noalloc(int(nx), int(ny), float(dx), float(dy), float(chi_par),
                                     float(chi_perp), int(bc), int(precision), _ptr(bx), _ptr(by),
                                     _ptr(T), float(dt), int(nsteps), _ptr(stream)))


# ------------------------------------------------------ three dimensions

def aniso3_create(nx, ny, nz, dx, dy, dz, chi_par, chi_perp=0.0, bc=ANISO_BC_PERIODIC):
    h = ctypes.c_void_p()
    _check(load().aniso3_create(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                float(chi_par), float(chi_perp), int(bc), ctypes.byref(h)))
    return h


def aniso3_set_option(h, key, value):
    _check(load().aniso3_set_option(h, int(key), int(value)))


def aniso3_set_field(h, bx, by, bz):
    _check(load().aniso3_set_field(h, _ptr(bx), _ptr(by), _ptr(bz)))


def aniso3_step(h, T, dt, nsteps=1):
    _check(load().aniso3_step(h, _ptr(T), float(dt), int(nsteps)))


def aniso3_total(h, T):
    """(sum, min, max, nonfinite count) of T, FP64 sum."""
    s, lo, hi, nf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    _check(load().aniso3_total(h, _ptr(T), ctypes.byref(s), ctypes.byref(lo), ctypes.byref(hi),
                               ctypes.byref(nf)))
    return s.value, lo.value, hi.value, nf.value


def aniso3_sync(h):
    _check(load().aniso3_sync(h))


def aniso3_destroy(h):
    if h:
        load().aniso3_destroy(h)
