"""FP64 CPU oracle for the split semi-implicit anisotropic-diffusion step.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the GPU library (``paper_1008_0861_gb300``) and imports nothing from it.

The arithmetic lives in ``aniso_oracle.c`` (plain C, FP64, written from
Section 2 of Sharma & Hammett, arXiv:1008.0861: Eqs. xup and yup, the limited
face differences after them, Eq. vanLeer and Eq. op_2step; the temperature-
dependent diffusivity of Section 3.3 in ``or_step_nl``) and, for the
three-dimensional form of Section 2.1, ``aniso3d_oracle.c``.  This module
marshals numpy arrays to it, composes those sweeps into the 4-step scheme of
Eq. 4step (step4), runs the explicit limited scheme built from the same face
fluxes (explicit_step), and does the one encoding step the paper leaves
to the implementation: rounding stored face coefficients to FP16 with numpy
(round-to-nearest-even) when a test asks for the FP16-field variant.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms (Eqs. amp1/amp2, the 1-D backward-Euler factor), dense
linear algebra on tiny grids, conservation, the extremum property of the
limiter (Section 3.1) and x/y transposition symmetry; step3 by
``tests/test_oracle3d_pins.py`` and step_nl by
``tests/test_oracle_nonlinear_pins.py``.  Parity unpinned: which temperature
feeds the y-update's face factor in step_nl (T*, the reading taken, or T^n:
no pin tells them apart); the ring-test contour shapes and min-T time series
of the paper's figures are printed only as plots and are not compared.
"""
import ctypes

import numpy as np

from . import build as _build

BC_ZEROFLUX = 0
BC_PERIODIC = 1
BC_DIRICHLET = 2   # boundary nodes keep their values (T fixed at the domain edge)

LIM_VANLEER = 0
LIM_ARITH = 1
LIM_MINMOD = 2
LIM_MC = 3

ORDER_XY = 0         # Eq. op_2step: x-update then y-update every step (default)
ORDER_YX = 1         # the reversed order mentioned after Eq. op_2step
ORDER_ALTERNATE = 2  # x then y on even step counters, y then x on odd ones

_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i, d, ll, sz = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
        lib.or_limit4.restype = d
        lib.or_limit4.argtypes = [i, d, d, d, d]
        lib.or_face_coeffs.restype = None
        lib.or_face_coeffs.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, _D]
        lib.or_thomas.restype = i
        lib.or_thomas.argtypes = [i, _D, _D, _D, _D, _D, _D]
        lib.or_cyclic.restype = i
        lib.or_cyclic.argtypes = [i, _D, _D, _D, _D, _D, _D]
        lib.or_xsweep_row.restype = None
        lib.or_xsweep_row.argtypes = [i, i, _D, _D, _D, _D, _D, d, d, i, _D, _D]
        lib.or_ysweep_col.restype = None
        lib.or_ysweep_col.argtypes = [i, i, _D, _D, _D, _D, _D, d, d, i, _D, _D]
        lib.or_xsweep.restype = None
        lib.or_xsweep.argtypes = [i, i, i, _D, _D, d, d, i, _D, _D]
        lib.or_ysweep.restype = None
        lib.or_ysweep.argtypes = [i, i, i, _D, _D, d, d, i, _D, _D]
        lib.or_step.restype = i
        lib.or_step.argtypes = [i, i, i, _D, _D, _D, _D, d, d, d, i, i, ll, i, _D, ctypes.c_void_p, d]
        lib.or_explicit_step.restype = i
        lib.or_explicit_step.argtypes = [i, i, i, _D, _D, _D, _D, d, d, d, i, i, _D]
        lib.or_totals.restype = None
        lib.or_totals.argtypes = [sz, _D, _D, _D, _D]
        lib.or_num_threads.restype = i
        lib.or_num_threads.argtypes = []
        lib.or_set_num_threads.restype = None
        lib.or_set_num_threads.argtypes = [i]
        lib.or_step_nl.restype = i
        lib.or_step_nl.argtypes = [i, i, i, _D, _D, _D, _D, d, d, d, i, d, d, i, _D]
        _D9 = _D * 9
        lib.or3_face_coeffs.restype = None
        lib.or3_face_coeffs.argtypes = [i, i, i, i, d, _D, _D, _D, _D9]
        lib.or3_sweep.restype = None
        lib.or3_sweep.argtypes = [i, i, i, i, i, _D, _D, _D, d, d, d, i, _D, _D]
        lib.or3_step.restype = i
        lib.or3_step.argtypes = [i, i, i, i, _D9, _D, _D, i, i, i, _D]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_D)


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    """Use n OpenMP threads from now on (results do not depend on it)."""
    _load().or_set_num_threads(int(n))


def limit4(a, b, c, d, limiter=LIM_VANLEER) -> float:
    """L(a,b,c,d) = L(L(a,b),L(c,d)) (Eq. vanLeer and the text after it)."""
    return float(_load().or_limit4(int(limiter), float(a), float(b), float(c), float(d)))


class Coeffs:
    """Face coefficients in units of chi_par (x faces: cxx, cxy; y faces:
    cyy, cyx), each [ny, nx] with face i+1/2 / j+1/2 at index i / j."""

    def __init__(self, cxx, cxy, cyy, cyx):
        self.cxx, self.cxy, self.cyy, self.cyx = (_f64(c) for c in (cxx, cxy, cyy, cyx))

    def rounded(self, dtype):
        """Coefficients as stored in a reduced-precision field (the encoding
        is plain round-to-nearest-even of each stored value), widened back
        exactly to FP64."""
        f = lambda c: c.astype(dtype).astype(np.float64)  # noqa: E731
        return Coeffs(f(self.cxx), f(self.cxy), f(self.cyy), f(self.cyx))


def face_coeffs(bx, by, bc, chi_par=1.0, chi_perp=0.0) -> Coeffs:
    """Average the cell-centred unit field to faces (Section 2) and form the
    implicit (normal) and explicit (transverse) coefficients."""
    bx, by = _f64(bx), _f64(by)
    ny, nx = bx.shape
    kappa = float(chi_perp) / float(chi_par)
    out = [np.empty((ny, nx)) for _ in range(4)]
    _load().or_face_coeffs(nx, ny, int(bc), kappa, _p(bx), _p(by), *(_p(o) for o in out))
    return Coeffs(*out)


def thomas(a, b, c, d):
    """Solve a tridiagonal system (a_0, c_{n-1} unused) by Thomas."""
    a, b, c, d = (_f64(v) for v in (a, b, c, d))
    n = len(b)
    x, w = np.empty(n), np.empty(n)
    if _load().or_thomas(n, _p(a), _p(b), _p(c), _p(d), _p(x), _p(w)):
        raise ZeroDivisionError("zero pivot")
    return x


def cyclic(a, b, c, d):
    """Solve a cyclic tridiagonal system (a_0 couples x_{n-1}, c_{n-1}
    couples x_0) by Sherman-Morrison on two Thomas solves."""
    a, b, c, d = (_f64(v) for v in (a, b, c, d))
    n = len(b)
    x, w = np.empty(n), np.empty(4 * n)
    if _load().or_cyclic(n, _p(a), _p(b), _p(c), _p(d), _p(x), _p(w)):
        raise ZeroDivisionError("zero pivot")
    return x


def lambdas(dt, dx, dy, chi_par):
    """(lamx, lamy, mu) = chi dt/dx^2, chi dt/dy^2, chi dt/(dx dy)."""
    return chi_par * dt / (dx * dx), chi_par * dt / (dy * dy), chi_par * dt / (dx * dy)


def xsweep_row(Tm, T0, Tp, cxx_row, cxy_row, lamx, mu, periodic, limiter=LIM_VANLEER):
    """Eq. xup for one row, given rows j-1, j, j+1 of T^n."""
    Tm, T0, Tp, g, e = (_f64(v) for v in (Tm, T0, Tp, cxx_row, cxy_row))
    n = len(T0)
    out, w = np.empty(n), np.empty(9 * n)
    _load().or_xsweep_row(n, int(periodic), _p(Tm), _p(T0), _p(Tp), _p(g), _p(e),
                          float(lamx), float(mu), int(limiter), _p(out), _p(w))
    return out


def ysweep_col(Tl, T0, Tr, cyy_col, cyx_col, lamy, mu, periodic, limiter=LIM_VANLEER):
    """Eq. yup for one column, given columns i-1, i, i+1 of T*."""
    Tl, T0, Tr, g, e = (_f64(v) for v in (Tl, T0, Tr, cyy_col, cyx_col))
    n = len(T0)
    out, w = np.empty(n), np.empty(9 * n)
    _load().or_ysweep_col(n, int(periodic), _p(Tl), _p(T0), _p(Tr), _p(g), _p(e),
                          float(lamy), float(mu), int(limiter), _p(out), _p(w))
    return out


def xsweep(T, co: Coeffs, bc, lamx, mu, limiter=LIM_VANLEER):
    """Eq. xup on every row of T (shape [ny, nx])."""
    T = _f64(T)
    ny, nx = T.shape
    out = np.empty_like(T)
    _load().or_xsweep(nx, ny, int(bc), _p(co.cxx), _p(co.cxy), float(lamx), float(mu),
                      int(limiter), _p(T), _p(out))
    return out


def ysweep(T, co: Coeffs, bc, lamy, mu, limiter=LIM_VANLEER):
    """Eq. yup on every column of T (shape [ny, nx])."""
    T = _f64(T)
    ny, nx = T.shape
    out = np.empty_like(T)
    _load().or_ysweep(nx, ny, int(bc), _p(co.cyy), _p(co.cyx), float(lamy), float(mu),
                      int(limiter), _p(T), _p(out))
    return out


def step(T, co: Coeffs, bc, dt, dx, dy, chi_par, nsteps=1, step0=0,
         order=ORDER_XY, limiter=LIM_VANLEER, Q=None):
    """nsteps steps of Eq. op_2step starting at step counter step0; returns a
    new FP64 array.  Q (optional, [ny][nx]): a source term, added as
    T += dt Q before each step."""
    T = _f64(T).copy()
    ny, nx = T.shape
    lamx, lamy, mu = lambdas(dt, dx, dy, chi_par)
    q = None if Q is None else _f64(Q)
    rc = _load().or_step(nx, ny, int(bc), _p(co.cxx), _p(co.cxy), _p(co.cyy), _p(co.cyx),
                         lamx, lamy, mu, int(limiter), int(order), int(step0), int(nsteps), _p(T),
                         None if q is None else q.ctypes.data_as(ctypes.c_void_p), float(dt))
    if rc:
        raise MemoryError("oracle scratch allocation failed")
    return T


def step4(T, co: Coeffs, bc, dt, dx, dy, chi_par, nsteps=1, step0=0,
          order=ORDER_XY, limiter=LIM_VANLEER):
    """nsteps steps of the 4-step scheme, Eq. 4step:
        T^{n+1} = (1 + dt Dyy/2)^-2 (1 - dt Dyx) (1 + dt Dxx/2)^-2 (1 - dt Dxy) T^n.
    Each direction is the update of Eq. xup / Eq. yup with its implicit (normal)
    part taken over dt/2 and the explicit transverse part over dt, followed by a
    fully implicit dt/2 update of the same direction (no transverse term).
    `order` as in step(): the reversed order swaps the x and y parts."""
    T = _f64(T).copy()
    lamx, lamy, mu = lambdas(dt, dx, dy, chi_par)

    def xpart(U):
        return xsweep(xsweep(U, co, bc, 0.5 * lamx, mu, limiter), co, bc, 0.5 * lamx, 0.0, limiter)

    def ypart(U):
        return ysweep(ysweep(U, co, bc, 0.5 * lamy, mu, limiter), co, bc, 0.5 * lamy, 0.0, limiter)

    for s in range(nsteps):
        k = step0 + s
        x_first = order == ORDER_XY or (order == ORDER_ALTERNATE and k % 2 == 0)
        T = ypart(xpart(T)) if x_first else xpart(ypart(T))
    return T


def step_nl(T, co: Coeffs, bc, dt, dx, dy, chi_par, alpha, t_ref=1.0, nsteps=1, limiter=LIM_VANLEER):
    """nsteps x-then-y steps with chi_par scaled by (max(T,0)/t_ref)^alpha at
    each face: the harmonic mean of the two cells' values, from the input of
    each directional update (Section 3.3 uses alpha = 5/2)."""
    T = _f64(T).copy()
    ny, nx = T.shape
    lamx, lamy, mu = lambdas(dt, dx, dy, chi_par)
    rc = _load().or_step_nl(nx, ny, int(bc), _p(co.cxx), _p(co.cxy), _p(co.cyy), _p(co.cyx),
                            lamx, lamy, mu, int(limiter), float(alpha), float(t_ref), int(nsteps), _p(T))
    if rc:
        raise MemoryError("oracle scratch allocation failed")
    return T


def explicit_step(T, co: Coeffs, bc, dt, dx, dy, chi_par, nsteps=1, limiter=LIM_VANLEER):
    """nsteps steps of the explicit limited scheme: the unsplit explicit form
    of the face fluxes of Eqs. xup and yup, every flux from T^n (the explicit
    method the paper compares against)."""
    T = _f64(T).copy()
    ny, nx = T.shape
    lamx, lamy, mu = lambdas(dt, dx, dy, chi_par)
    rc = _load().or_explicit_step(nx, ny, int(bc), _p(co.cxx), _p(co.cxy), _p(co.cyy), _p(co.cyx),
                                  lamx, lamy, mu, int(limiter), int(nsteps), _p(T))
    if rc:
        raise MemoryError("oracle scratch allocation failed")
    return T


# ------------------------------------------------------------ three dimensions

SCHEME_2STEP = 0   # Eq. op_2step with a third factor: x, y, z updates
SCHEME_4STEP = 1   # Eq. 4step with a third pair of factors


class Coeffs3:
    """The nine face coefficients of a 3-D grid in units of chi_par, each
    [nz, ny, nx] with face f+1/2 along an axis stored at cell f:
    x faces cxx, cxy, cxz; y faces cyy, cyz, cyx; z faces czz, czx, czy."""

    NAMES = ("cxx", "cxy", "cxz", "cyy", "cyz", "cyx", "czz", "czx", "czy")

    def __init__(self, arrays):
        self.arrays = [_f64(a) for a in arrays]
        for name, a in zip(self.NAMES, self.arrays):
            setattr(self, name, a)

    def _ptrs(self):
        return (_D * 9)(*(_p(a) for a in self.arrays))

    def rounded(self, dtype):
        """Coefficients as stored in a reduced-precision field (plain
        round-to-nearest-even of each stored value), widened back exactly."""
        return Coeffs3([a.astype(dtype).astype(np.float64) for a in self.arrays])


def face_coeffs3(bx, by, bz, bc, chi_par=1.0, chi_perp=0.0) -> Coeffs3:
    """Average the cell-centred unit field to the faces of a 3-D grid and form
    the normal and the two transverse coefficients of each face."""
    bx, by, bz = _f64(bx), _f64(by), _f64(bz)
    nz, ny, nx = bx.shape
    kappa = float(chi_perp) / float(chi_par)
    out = [np.empty((nz, ny, nx)) for _ in range(9)]
    c = Coeffs3(out)
    _load().or3_face_coeffs(nx, ny, nz, int(bc), kappa, _p(bx), _p(by), _p(bz), c._ptrs())
    return c


def lambdas3(dt, dx, dy, dz, chi_par):
    """(lam, mu): lam[d] = chi dt / Delta_d^2; mu[2d], mu[2d+1] = chi dt /
    (Delta_d Delta_{d+1}), chi dt / (Delta_d Delta_{d+2}), axes cyclic."""
    D = (dx, dy, dz)
    lam = [chi_par * dt / (D[a] * D[a]) for a in range(3)]
    mu = []
    for a in range(3):
        mu += [chi_par * dt / (D[a] * D[(a + 1) % 3]), chi_par * dt / (D[a] * D[(a + 2) % 3])]
    return lam, mu


def sweep3(T, co: Coeffs3, bc, axis, lam, mua, mub, limiter=LIM_VANLEER):
    """One directional update along `axis` (0 = x, 1 = y, 2 = z) of T
    [nz, ny, nx]: implicit in the face-normal flux, explicit and limited in
    the two transverse ones."""
    T = _f64(T)
    nz, ny, nx = T.shape
    out = np.empty_like(T)
    cn, ca, cb = co.arrays[3 * axis: 3 * axis + 3]
    _load().or3_sweep(nx, ny, nz, int(bc), int(axis), _p(cn), _p(ca), _p(cb), float(lam),
                      float(mua), float(mub), int(limiter), _p(T), _p(out))
    return out


def step3(T, co: Coeffs3, bc, dt, dx, dy, dz, chi_par, nsteps=1, limiter=LIM_VANLEER,
          scheme=SCHEME_2STEP):
    """nsteps 3-D steps (x, y, z updates; SCHEME_4STEP takes each axis as a
    half-coefficient update with the transverse terms followed by a purely
    implicit half-coefficient update); returns a new FP64 array."""
    T = _f64(T).copy()
    nz, ny, nx = T.shape
    lam, mu = lambdas3(dt, dx, dy, dz, chi_par)
    lam_a, mu_a = np.array(lam, dtype=np.float64), np.array(mu, dtype=np.float64)
    rc = _load().or3_step(nx, ny, nz, int(bc), co._ptrs(), _p(lam_a), _p(mu_a), int(limiter),
                          int(scheme), int(nsteps), _p(T))
    if rc:
        raise MemoryError("oracle scratch allocation failed")
    return T


def totals(T):
    """(sum, min, max) of T in FP64."""
    T = _f64(T)
    s, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().or_totals(T.size, _p(T), ctypes.byref(s), ctypes.byref(lo), ctypes.byref(hi))
    return s.value, lo.value, hi.value


__all__ = [n for n in dir() if not n.startswith("_")]
