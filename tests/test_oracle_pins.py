"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form the
paper prints (Eqs. amp1, amp2, amp_sym), an exact reduction to 1-D backward
Euler, dense linear algebra, an invariant (conservation, the extremum property
of limited averaging, x/y transposition symmetry), or a value the paper
reports for the ring test.  A dropped term, a wrong sign or a shifted index in
the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- limiter

def test_vanleer_two_argument_values():
    # Eq. vanLeer: 2ab/(a+b) when ab > 0, else 0 (L(a,b) = L(a,b,a,b)).
    assert O.limit4(1.0, 3.0, 1.0, 3.0) == pytest.approx(1.5)
    assert O.limit4(-2.0, -2.0, -2.0, -2.0) == -2.0
    assert O.limit4(1.0, -1.0, 5.0, 5.0) == 0.0
    assert O.limit4(0.0, 1.0, 1.0, 1.0) == 0.0
    # tiny same-sign differences do not underflow to zero (sign test, not product)
    assert O.limit4(1e-200, 1e-200, 1e-200, 1e-200) == pytest.approx(1e-200, rel=1e-12)


def test_vanleer_four_argument_is_harmonic_mean_and_symmetric():
    rng = np.random.default_rng(1)
    for _ in range(200):
        v = rng.uniform(0.01, 5.0, 4) * rng.choice([-1.0, 1.0])
        got = O.limit4(*v)
        harmonic = 4.0 / np.sum(1.0 / v)        # closed form of the nesting
        assert got == pytest.approx(harmonic, rel=1e-13)
        assert min(v) - 1e-12 <= got <= max(v) + 1e-12
        # the limiter is symmetric in its four arguments (text after Eq. vanLeer)
        for perm in ([1, 0, 2, 3], [2, 3, 0, 1], [0, 2, 1, 3], [3, 1, 2, 0]):
            assert O.limit4(*v[perm]) == pytest.approx(got, rel=1e-13)
    # any sign disagreement gives zero
    assert O.limit4(1.0, 2.0, 3.0, -4.0) == 0.0


# The two other limiters the paper names after Eq. vanLeer (minmod and the
# monotonized central limiter, defined in the limiter literature it cites):
#   minmod(a, b) = s * min(|a|, |b|)
#   MC(a, b)     = s * min(2|a|, 2|b|, |a + b| / 2)
# with s the common sign of a and b, and 0 unless a and b share a strict sign.
# The expected values below were worked out by hand from those definitions;
# L(a, b) is read through L(a, b, a, b) = L(L(a,b), L(a,b)) = L(a, b), which
# holds for all three limiters since L(x, x) = x.

@pytest.mark.parametrize("a,b,want", [
    (1.0, 3.0, 1.0), (3.0, 1.0, 1.0), (-1.0, -3.0, -1.0), (-3.0, -0.5, -0.5),
    (2.5, 2.5, 2.5), (1.0, -3.0, 0.0), (-1.0, 3.0, 0.0), (0.0, 2.0, 0.0), (2.0, 0.0, 0.0),
])
def test_minmod_two_argument_values(a, b, want):
    assert O.limit4(a, b, a, b, O.LIM_MINMOD) == want


@pytest.mark.parametrize("a,b,want", [
    (1.0, 3.0, 2.0),      # 2|a| = 2 binds (|a+b|/2 = 2 too)
    (1.0, 10.0, 2.0),     # 2|a| binds
    (1.0, 1.2, 1.1),      # |a+b|/2 binds: a dropped /2 gives 2, a dropped factor 2 gives 1
    (3.0, 1.0, 2.0),      # 2|b| binds
    (4.0, 6.0, 5.0),
    (-1.0, -3.0, -2.0), (-4.0, -6.0, -5.0), (-1.0, -1.2, -1.1),
    (1.0, -3.0, 0.0), (-2.0, 5.0, 0.0), (0.0, 1.0, 0.0), (1.0, 0.0, 0.0),
])
def test_mc_two_argument_values(a, b, want):
    assert O.limit4(a, b, a, b, O.LIM_MC) == pytest.approx(want, rel=1e-15, abs=0.0)


def test_mc_nesting_pairs_each_cells_differences():
    # L(a,b,c,d) = L(L(a,b), L(c,d)) as written after Eq. vanLeer.  For MC
    # the nesting is not symmetric, so the pairing is visible:
    #   MC(MC(1,3), MC(4,6)) = MC(2, 5)   = min(4, 10, 3.5)  = 3.5
    #   MC(MC(1,4), MC(3,6)) = MC(2, 4.5) = min(4, 9, 3.25)  = 3.25
    #   MC(MC(1,6), MC(3,4)) = MC(2, 3.5) = min(4, 7, 2.75)  = 2.75
    assert O.limit4(1.0, 3.0, 4.0, 6.0, O.LIM_MC) == pytest.approx(3.5, rel=1e-15)
    assert O.limit4(1.0, 4.0, 3.0, 6.0, O.LIM_MC) == pytest.approx(3.25, rel=1e-15)
    assert O.limit4(1.0, 6.0, 3.0, 4.0, O.LIM_MC) == pytest.approx(2.75, rel=1e-15)
    assert O.limit4(-1.0, -3.0, -4.0, -6.0, O.LIM_MC) == pytest.approx(-3.5, rel=1e-15)
    # one pair of mixed sign zeroes the inner level, hence the whole value
    assert O.limit4(1.0, 3.0, 4.0, -6.0, O.LIM_MC) == 0.0
    # minmod nests to the smallest magnitude of the four when all agree
    assert O.limit4(1.0, 3.0, 4.0, 6.0, O.LIM_MINMOD) == 1.0
    assert O.limit4(-6.0, -4.0, -3.0, -2.0, O.LIM_MINMOD) == -2.0


# Slopes (up, down) = (T[i,2] - T[i,1], T[i,1] - T[i,0]) of the five columns
# of a 3-row grid; the middle row is the only one with a non-zero limited
# difference (rows 0 and 2 see a mirrored ghost, so one inner argument is 0).
_SLOPES = [(4.0, 6.0), (1.0, 3.0), (-1.0, 2.0), (-2.0, -6.0), (-1.0, -1.0)]
# Transverse coefficients e at x faces 0..4 of the middle row (face 4 is the
# zero-flux boundary face, stored as 0).
_E = [1.0, 1.0, 1.0, 0.5, 0.0]
# Worked by hand.  Face i+1/2 takes L(L(up_{i+1}, down_{i+1}), L(up_i, down_i))
# (first DeltaT-bar equation after Eq. yup); column 2 is mixed-sign, so faces
# 1 and 2 are 0.  With mu = 0.5 and no implicit part, T* - T at cell i is
# mu (e_i dT_i - e_{i-1} dT_{i-1}):
#   MC:     dT = [MC(MC(1,3),MC(4,6)) = 3.5, 0, 0, MC(-1,-4) = -2, 0]
#           delta = 0.5 [3.5, -3.5, 0, -1, 1]
#   minmod: dT = [minmod(1, 4) = 1, 0, 0, minmod(-1, -2) = -1, 0]
#           delta = 0.5 [1, -1, 0, -0.5, 0.5]
_WANT_DELTA = {
    O.LIM_MC: [1.75, -1.75, 0.0, -0.5, 0.5],
    O.LIM_MINMOD: [0.5, -0.5, 0.0, -0.25, 0.25],
}


def _slope_grid():
    T = np.empty((3, 5))
    for i, (up, down) in enumerate(_SLOPES):
        T[0, i] = 10.0
        T[1, i] = 10.0 + down
        T[2, i] = 10.0 + down + up
    return T


@pytest.mark.parametrize("lim", [O.LIM_MC, O.LIM_MINMOD])
def test_x_update_transverse_term_on_known_slopes(lim):
    T = _slope_grid()
    zero = np.zeros_like(T)
    e = np.zeros_like(T)
    e[1, :] = _E
    e[0, :4] = e[2, :4] = 1.0                # rows 0, 2: limited difference is 0 anyway
    co = O.Coeffs(zero, e, zero, zero)       # no implicit part: T* = T + mu dF
    out = O.xsweep(T, co, O.BC_ZEROFLUX, lamx=7.0, mu=0.5, limiter=lim)
    np.testing.assert_array_equal(out[0], T[0])
    np.testing.assert_array_equal(out[2], T[2])
    np.testing.assert_allclose(out[1] - T[1], _WANT_DELTA[lim], rtol=0, atol=1e-14)


@pytest.mark.parametrize("lim", [O.LIM_MC, O.LIM_MINMOD])
def test_y_update_transverse_term_on_known_slopes(lim):
    # The same numbers through Eq. yup: columns become rows (second
    # DeltaT-bar equation after Eq. yup, x-differences of rows j and j+1).
    T = _slope_grid().T.copy()               # [5][3]: column 1 holds the slopes
    zero = np.zeros_like(T)
    f = np.zeros_like(T)
    f[:, 1] = _E
    f[:4, 0] = f[:4, 2] = 1.0
    co = O.Coeffs(zero, zero, zero, f)
    out = O.ysweep(T, co, O.BC_ZEROFLUX, lamy=7.0, mu=0.5, limiter=lim)
    np.testing.assert_array_equal(out[:, 0], T[:, 0])
    np.testing.assert_array_equal(out[:, 2], T[:, 2])
    np.testing.assert_allclose(out[:, 1] - T[:, 1], _WANT_DELTA[lim], rtol=0, atol=1e-14)


# ------------------------------------------------------- tridiagonal solves

def _dd_system(rng, n):
    a = -rng.uniform(0, 2, n)
    c = -rng.uniform(0, 2, n)
    b = 1.0 - a - c + rng.uniform(0, 0.5, n)
    d = rng.normal(size=n)
    return a, b, c, d


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 12])
def test_thomas_matches_dense_lu(n):
    rng = np.random.default_rng(n)
    a, b, c, d = _dd_system(rng, n)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x = O.thomas(a, b, c, d)
    np.testing.assert_allclose(x, np.linalg.solve(A, d), rtol=1e-13, atol=1e-14)
    assert np.max(np.abs(A @ x - d)) < 1e-14 * max(1.0, np.max(np.abs(d))) * 10


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_cyclic_matches_dense_lu(n):
    rng = np.random.default_rng(100 + n)
    a, b, c, d = _dd_system(rng, n)
    A = np.zeros((n, n))
    for k in range(n):
        A[k, k] += b[k]
        A[k, (k - 1) % n] += a[k]
        A[k, (k + 1) % n] += c[k]
    x = O.cyclic(a, b, c, d)
    np.testing.assert_allclose(x, np.linalg.solve(A, d), rtol=1e-12, atol=1e-13)


# --------------------------------------------- closed-form amplification

@pytest.mark.parametrize("nx,ny,mx,my,alpha,fac", [
    (16, 12, 1, 2, 0.3, 10.0), (16, 16, 3, -5, 2.1, 100.0), (10, 14, 4, 1, -0.7, 1000.0),
    (8, 8, 2, 2, math.pi / 4, 50.0), (12, 9, 5, 3, 1.2, 3.0)])
def test_fourier_mode_amplification_eq_amp(nx, ny, mx, my, alpha, fac):
    """Constant b, periodic, arithmetic-mean transverse average: one step maps
    cos(k.x) to r1 r2 cos(k.x) with r1, r2 of Eqs. amp1/amp2 (Section 2.1)."""
    chi = 0.7
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = fac * W.cfl_dt(dx, dy, chi)
    bxv, byv = math.cos(alpha), math.sin(alpha)
    bx = np.full((ny, nx), bxv)
    by = np.full((ny, nx), byv)
    co = O.face_coeffs(bx, by, O.BC_PERIODIC)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    kx, ky = 2 * math.pi * mx, 2 * math.pi * my
    T0 = np.cos(kx * x[None, :] + ky * y[:, None] + 0.37)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    tx, ty = kx * dx, ky * dy
    num = 1.0 - mu * bxv * byv * math.sin(tx) * math.sin(ty)
    r1 = num / (1.0 + 4.0 * lamx * bxv ** 2 * math.sin(tx / 2) ** 2)
    r2 = num / (1.0 + 4.0 * lamy * byv ** 2 * math.sin(ty / 2) ** 2)
    # Eq. amp_sym, the paper's combined form of r1 r2
    Ax = 2 * math.sqrt(chi * dt) * bxv / dx * math.sin(tx / 2)
    Ay = 2 * math.sqrt(chi * dt) * byv / dy * math.sin(ty / 2)
    r_sym = (1 - Ax * Ay * math.cos(tx / 2) * math.cos(ty / 2)) ** 2 / ((1 + Ax ** 2) * (1 + Ay ** 2))
    assert r1 * r2 == pytest.approx(r_sym, rel=1e-12, abs=1e-15)
    assert abs(r_sym) <= 1.0 + 1e-15          # unconditional stability (Section 2.1)
    for order in (O.ORDER_XY, O.ORDER_YX):
        T1 = O.step(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, order=order, limiter=O.LIM_ARITH)
        np.testing.assert_allclose(T1, r1 * r2 * T0, atol=1e-13)
    # single x-update alone gives r1
    Ts = O.xsweep(T0, co, O.BC_PERIODIC, lamx, mu, limiter=O.LIM_ARITH)
    np.testing.assert_allclose(Ts, r1 * T0, atol=1e-13)


@pytest.mark.parametrize("nx,ny,mx,my,alpha,fac", [
    (16, 12, 1, 2, 0.3, 10.0), (16, 16, 3, -5, 2.1, 100.0), (10, 14, 4, 1, -0.7, 1000.0),
    (12, 9, 5, 3, 1.2, 3.0)])
def test_four_step_fourier_mode_amplification(nx, ny, mx, my, alpha, fac):
    """Eq. 4step on a Fourier mode (constant b, periodic, arithmetic-mean
    transverse average): each direction multiplies by the explicit transverse
    factor of Eqs. amp1/amp2 and divides by its implicit half-step factor
    twice, r = num^2 / ((1 + 2 lamx bx^2 sin^2(tx/2))^2 (1 + 2 lamy by^2 sin^2(ty/2))^2)."""
    chi = 0.7
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = fac * W.cfl_dt(dx, dy, chi)
    bxv, byv = math.cos(alpha), math.sin(alpha)
    co = O.face_coeffs(np.full((ny, nx), bxv), np.full((ny, nx), byv), O.BC_PERIODIC)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    kx, ky = 2 * math.pi * mx, 2 * math.pi * my
    T0 = np.cos(kx * x[None, :] + ky * y[:, None] - 0.9)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    tx, ty = kx * dx, ky * dy
    num = 1.0 - mu * bxv * byv * math.sin(tx) * math.sin(ty)
    rx = num / (1.0 + 2.0 * lamx * bxv ** 2 * math.sin(tx / 2) ** 2) ** 2
    ry = num / (1.0 + 2.0 * lamy * byv ** 2 * math.sin(ty / 2) ** 2) ** 2
    for order in (O.ORDER_XY, O.ORDER_YX):
        T1 = O.step4(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, order=order, limiter=O.LIM_ARITH)
        np.testing.assert_allclose(T1, rx * ry * T0, atol=1e-13)
    # and it differs from the 2-step factor unless the implicit parts vanish
    r2 = num / (1.0 + 4.0 * lamx * bxv ** 2 * math.sin(tx / 2) ** 2) * \
        num / (1.0 + 4.0 * lamy * byv ** 2 * math.sin(ty / 2) ** 2)
    assert abs(rx * ry - r2) > 1e-6


@pytest.mark.parametrize("alpha", [0.25, 1.0, 2.5, -2.0])
@pytest.mark.parametrize("order", [O.ORDER_XY, O.ORDER_YX])
def test_one_dimensional_data_reduces_to_backward_euler(alpha, order):
    """With the van Leer limiter and T depending on y alone, the x-update leaves
    T unchanged (row-constant transverse flux, zero normal gradient) and the
    y-update is 1-D backward Euler: r = 1/(1 + 4 lamy by^2 sin^2(ky dy/2))."""
    nx, ny, my, chi = 12, 20, 3, 0.05
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = 200.0 * W.cfl_dt(dx, dy, chi)
    bxv, byv = math.cos(alpha), math.sin(alpha)
    co = O.face_coeffs(np.full((ny, nx), bxv), np.full((ny, nx), byv), O.BC_PERIODIC)
    y = (np.arange(ny) + 0.5) * dy
    mode = np.cos(2 * math.pi * my * y + 0.1)[:, None] * np.ones((1, nx))
    T0 = 3.0 + mode
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    np.testing.assert_allclose(O.xsweep(T0, co, O.BC_PERIODIC, lamx, mu), T0, atol=1e-14)
    r = 1.0 / (1.0 + 4.0 * lamy * byv ** 2 * math.sin(math.pi * my * dy) ** 2)
    T1 = O.step(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, order=order)
    np.testing.assert_allclose(T1 - 3.0, r * mode, atol=2e-14)
    # and symmetrically for T depending on x alone
    x = (np.arange(nx) + 0.5) * dx
    modex = np.ones((ny, 1)) * np.cos(2 * math.pi * 2 * x + 0.4)[None, :]
    rx = 1.0 / (1.0 + 4.0 * lamx * bxv ** 2 * math.sin(math.pi * 2 * dx) ** 2)
    T1 = O.step(3.0 + modex, co, O.BC_PERIODIC, dt, dx, dy, chi, order=order)
    np.testing.assert_allclose(T1 - 3.0, rx * modex, atol=2e-14)


def test_field_along_x_is_implicit_diffusion_first_order_in_time():
    """b = x: transverse terms vanish and each step is 1-D backward Euler in x
    for any ky; against exp(-chi kx^2 t) the error is first order in dt
    (Section 2.1: the scheme is first order in time)."""
    nx, ny, chi = 64, 8, 1.0
    dx, dy = 1.0 / nx, 1.0 / ny
    co = O.face_coeffs(np.ones((ny, nx)), np.zeros((ny, nx)), O.BC_PERIODIC)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    T0 = np.cos(2 * math.pi * x[None, :] + 2 * math.pi * 3 * y[:, None])
    t_end = 0.02
    errs = []
    for nsteps in (4, 8, 16):
        dt = t_end / nsteps
        lamx = chi * dt / dx ** 2
        T1 = O.step(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, nsteps=nsteps)
        r = 1.0 / (1.0 + 4.0 * lamx * math.sin(math.pi * dx) ** 2)
        np.testing.assert_allclose(T1, r ** nsteps * T0, atol=1e-13)
        errs.append(abs(r ** nsteps - math.exp(-chi * (2 * math.pi) ** 2 * t_end)))
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


# --------------------------------------------------------- dense operator

def _cell(i, j, nx, ny, periodic):
    if periodic:
        return (j % ny) * nx + (i % nx)
    return min(max(j, 0), ny - 1) * nx + min(max(i, 0), nx - 1)   # mirrored ghost


def _dense_step_matrix(nx, ny, bc, co, lamx, lamy, mu, x_first=True, four_step=False):
    """Eq. op_2step assembled densely for the arithmetic-mean transverse
    average: (I+dt Dyy)^-1 (I-dt Dyx) (I+dt Dxx)^-1 (I-dt Dxy); with
    four_step, Eq. 4step: (I+dt Dyy/2)^-2 (I-dt Dyx) (I+dt Dxx/2)^-2 (I-dt Dxy)."""
    if four_step:
        lamx, lamy = 0.5 * lamx, 0.5 * lamy
    per = bc == O.BC_PERIODIC
    N = nx * ny
    Ax, Ex, Ay, Ey = (np.zeros((N, N)) for _ in range(4))
    for j in range(ny):
        for i in range(nx):
            k = j * nx + i
            # x faces i+1/2 (index i) and i-1/2 (index i-1, wrapped or absent)
            gp = co.cxx[j, i] if (per or i < nx - 1) else 0.0
            gm = co.cxx[j, (i - 1) % nx] if (per or i > 0) else 0.0
            ep = co.cxy[j, i] if (per or i < nx - 1) else 0.0
            em = co.cxy[j, (i - 1) % nx] if (per or i > 0) else 0.0
            Ax[k, k] += 1 + lamx * (gp + gm)
            if gp: Ax[k, _cell(i + 1, j, nx, ny, per)] -= lamx * gp
            if gm: Ax[k, _cell(i - 1, j, nx, ny, per)] -= lamx * gm
            Ex[k, k] += 1
            # mean of the four y-differences at face i+1/2: (T[i+1,j+1]-T[i+1,j-1]+T[i,j+1]-T[i,j-1])/4
            for (ii, sgn_face, e) in ((i, +1, ep), (i - 1, -1, em)):
                if not e:
                    continue
                for (ci, cj, s) in ((ii + 1, j + 1, 1), (ii + 1, j - 1, -1), (ii, j + 1, 1), (ii, j - 1, -1)):
                    Ex[k, _cell(ci, cj, nx, ny, per)] += sgn_face * mu * e * 0.25 * s
            # y faces
            gp = co.cyy[j, i] if (per or j < ny - 1) else 0.0
            gm = co.cyy[(j - 1) % ny, i] if (per or j > 0) else 0.0
            ep = co.cyx[j, i] if (per or j < ny - 1) else 0.0
            em = co.cyx[(j - 1) % ny, i] if (per or j > 0) else 0.0
            Ay[k, k] += 1 + lamy * (gp + gm)
            if gp: Ay[k, _cell(i, j + 1, nx, ny, per)] -= lamy * gp
            if gm: Ay[k, _cell(i, j - 1, nx, ny, per)] -= lamy * gm
            Ey[k, k] += 1
            for (jj, sgn_face, e) in ((j, +1, ep), (j - 1, -1, em)):
                if not e:
                    continue
                for (ci, cj, s) in ((i + 1, jj + 1, 1), (i - 1, jj + 1, -1), (i + 1, jj, 1), (i - 1, jj, -1)):
                    Ey[k, _cell(ci, cj, nx, ny, per)] += sgn_face * mu * e * 0.25 * s
    Mx = np.linalg.solve(Ax, Ex)
    My = np.linalg.solve(Ay, Ey)
    if four_step:
        Mx = np.linalg.solve(Ax, Mx)
        My = np.linalg.solve(Ay, My)
    return My @ Mx if x_first else Mx @ My


@pytest.mark.parametrize("nx,ny,bc", [(6, 5, O.BC_PERIODIC), (5, 7, O.BC_ZEROFLUX),
                                      (6, 5, O.BC_ZEROFLUX), (4, 6, O.BC_PERIODIC)])
def test_step_matches_dense_operator(nx, ny, bc):
    rng = np.random.default_rng(nx * 10 + ny + bc)
    ang = rng.uniform(0, 2 * math.pi, (ny, nx))
    co = O.face_coeffs(np.cos(ang), np.sin(ang), bc, chi_par=1.0, chi_perp=0.1)
    dx, dy, chi = 1.0 / nx, 1.3 / ny, 0.4
    dt = 30 * W.cfl_dt(dx, dy, chi)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    T0 = rng.normal(size=(ny, nx))
    for order, xf in ((O.ORDER_XY, True), (O.ORDER_YX, False)):
        M = _dense_step_matrix(nx, ny, bc, co, lamx, lamy, mu, x_first=xf)
        T1 = O.step(T0, co, bc, dt, dx, dy, chi, order=order, limiter=O.LIM_ARITH)
        np.testing.assert_allclose(T1.ravel(), M @ T0.ravel(), atol=1e-12)


@pytest.mark.parametrize("nx,ny,bc", [(6, 5, O.BC_PERIODIC), (5, 7, O.BC_ZEROFLUX), (4, 6, O.BC_ZEROFLUX)])
def test_four_step_matches_dense_operator(nx, ny, bc):
    """Eq. 4step assembled densely (random b, chi_perp > 0, both boundary
    conditions) against step4, both orders."""
    rng = np.random.default_rng(nx * 7 + ny + 3 * bc)
    ang = rng.uniform(0, 2 * math.pi, (ny, nx))
    co = O.face_coeffs(np.cos(ang), np.sin(ang), bc, chi_par=1.0, chi_perp=0.05)
    dx, dy, chi = 1.1 / nx, 1.0 / ny, 0.3
    dt = 40 * W.cfl_dt(dx, dy, chi)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    T0 = rng.normal(size=(ny, nx))
    for order, xf in ((O.ORDER_XY, True), (O.ORDER_YX, False)):
        M = _dense_step_matrix(nx, ny, bc, co, lamx, lamy, mu, x_first=xf, four_step=True)
        T1 = O.step4(T0, co, bc, dt, dx, dy, chi, order=order, limiter=O.LIM_ARITH)
        np.testing.assert_allclose(T1.ravel(), M @ T0.ravel(), atol=1e-12)


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_ZEROFLUX])
def test_four_step_conserves(bc):
    inst = W.random_instance(24, 20, seed=5, dt_factor=500.0) if bc == O.BC_PERIODIC else \
        W.ring_instance(24, ny=20, dt_factor=500.0)
    co = O.face_coeffs(inst.bx, inst.by, bc, inst.chi_par)
    T1 = O.step4(inst.T0, co, bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=5)
    s0, s1 = np.sum(inst.T0), np.sum(T1)
    assert abs(s1 - s0) <= 1e-12 * abs(s0)


def test_alternating_order_follows_step_counter():
    rng = np.random.default_rng(7)
    inst = W.random_instance(10, 8, seed=3)
    co = O.face_coeffs(inst.bx, inst.by, inst.bc)
    T0 = rng.uniform(1, 2, (8, 10))
    a = O.step(inst.T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3, step0=0,
               order=O.ORDER_ALTERNATE)
    b = O.step(inst.T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, order=O.ORDER_XY)
    b = O.step(b, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, order=O.ORDER_YX)
    b = O.step(b, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, order=O.ORDER_XY)
    np.testing.assert_array_equal(a, b)
    c = O.step(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, step0=5,
               order=O.ORDER_ALTERNATE)
    d = O.step(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, order=O.ORDER_YX)
    np.testing.assert_array_equal(c, d)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("which", ["random", "ring"])
def test_conservation(which):
    """Flux form: sum T is unchanged under periodic and zero-flux boundaries."""
    inst = W.random_instance(24, 20, seed=11) if which == "random" else W.ring_instance(32)
    co = O.face_coeffs(inst.bx, inst.by, inst.bc, inst.chi_par)
    s0 = inst.T0.sum()
    T = O.step(inst.T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=12)
    assert abs(T.sum() - s0) / abs(s0) < 1e-12


def test_transverse_term_vanishes_at_extrema():
    """Section 3.1: limited averaging makes the transverse term vanish at a
    temperature extremum.  With cxx = 0 the x-update is T* = T + transverse
    term, so T* = T exactly at every strict extremum along y."""
    rng = np.random.default_rng(5)
    nx, ny = 20, 18
    T = rng.normal(size=(ny, nx))
    zero = np.zeros((ny, nx))
    co = O.Coeffs(zero, rng.uniform(-0.5, 0.5, (ny, nx)), zero, zero)
    Ts = O.xsweep(T, co, O.BC_PERIODIC, 0.0, 3.0)
    up, dn = np.roll(T, -1, axis=0), np.roll(T, 1, axis=0)
    ext = ((T > up) & (T > dn)) | ((T < up) & (T < dn))
    assert ext.sum() > 50
    np.testing.assert_array_equal(Ts[ext], T[ext])
    assert np.any(Ts[~ext] != T[~ext])


def test_transposition_symmetry():
    """Swapping x and y (field components, grid sizes, spacings) and the
    update order gives the transposed result, bit for bit."""
    inst = W.random_instance(14, 9, seed=21)
    co = O.face_coeffs(inst.bx, inst.by, inst.bc, inst.chi_par)
    cot = O.face_coeffs(inst.by.T, inst.bx.T, inst.bc, inst.chi_par)
    dt = 50 * inst.dt
    a = O.step(inst.T0, co, 1, dt, inst.dx, inst.dy, inst.chi_par, nsteps=2, order=O.ORDER_XY)
    b = O.step(inst.T0.T, cot, 1, dt, inst.dy, inst.dx, inst.chi_par, nsteps=2, order=O.ORDER_YX)
    np.testing.assert_array_equal(a, b.T)


def test_first_step_keeps_initial_bounds_on_ring():
    """Section 3.1: with a two-valued initial condition every limited
    difference vanishes, so the first step respects the initial extrema."""
    inst = W.ring_instance(64, t_hot=10.0, t_cold=0.1)
    co = O.face_coeffs(inst.bx, inst.by, inst.bc, inst.chi_par)
    T = O.step(inst.T0, co, 0, 1000 * inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1)
    assert T.min() >= 0.1 - 1e-14 and T.max() <= 10.0 + 1e-14


def test_linear_stability_norm_non_increasing():
    """r <= 1 (Section 2.1): with constant b and the arithmetic-mean
    transverse average the L2 norm never grows, even at large dt."""
    rng = np.random.default_rng(9)
    nx, ny = 16, 16
    co = O.face_coeffs(np.full((ny, nx), 0.6), np.full((ny, nx), 0.8), O.BC_PERIODIC)
    T = rng.normal(size=(ny, nx))
    for _ in range(5):
        T1 = O.step(T, co, O.BC_PERIODIC, 1.0, 1.0 / nx, 1.0 / ny, 10.0, limiter=O.LIM_ARITH)
        assert np.linalg.norm(T1) <= np.linalg.norm(T) * (1 + 1e-13)
        T = T1


# ------------------------------------------------ paper-reported ring values

def test_ring_nonmonotonicity_matches_paper():
    """The values the paper reports for the ring test at 512^2 (Section 3.1,
    Figs. 4-5): relative non-monotonicity about 0.2 at ncfl = 1000, T kept
    positive up to ncfl = 10000, and more non-monotonicity at larger ncfl.
    Stored in tests/golden with the citation.  The paper's update order is
    the fixed x-then-y composition of Eq. op_2step."""
    g = json.load(open(os.path.join(GOLDEN, "ring_paper_values.json")))
    n = g["n"]
    inst = W.ring_instance(n, t_hot=g["T_hot"], t_cold=g["T_cold"], chi_par=g["chi_par"])
    co = O.face_coeffs(inst.bx, inst.by, inst.bc, inst.chi_par)
    rels = []
    for ncfl, check in ((100, "trend"), (g["ncfl"], "nonmono"), (g["positive_up_to_ncfl"], "positive")):
        dt_req = ncfl * inst.dx ** 2 / (4 * inst.chi_par)        # Eq. ncfl
        nsteps = int(math.ceil(g["t_end"] / dt_req))
        dt = g["t_end"] / nsteps
        T = inst.T0
        tmin = T.min()
        for s in range(nsteps):
            T = O.step(T, co, 0, dt, inst.dx, inst.dy, inst.chi_par, nsteps=1, step0=s)
            tmin = min(tmin, T.min())
        rels.append((g["T_cold"] - tmin) / g["T_cold"])
        if check == "nonmono":
            rel = (g["T_cold"] - tmin) / g["T_cold"]
            lo, hi = g["rel_nonmonotonicity_band"]
            assert lo <= rel <= hi, rel
        elif check == "positive":
            assert tmin > 0.0
    assert rels[0] < rels[1] < rels[2]


# ------------------------------------------------- explicit limited step

@pytest.mark.parametrize("nx,ny,mx,my,alpha,fac", [
    (16, 12, 1, 2, 0.3, 0.4), (16, 16, 3, -5, 2.1, 0.25), (10, 14, 4, 1, -0.7, 0.5), (12, 9, 5, 3, 1.2, 5.0)])
def test_explicit_step_fourier_mode(nx, ny, mx, my, alpha, fac):
    """Constant b, periodic, arithmetic-mean transverse average: one explicit
    step multiplies cos(k.x) by 1 - dt (Dxx + Dyy + Dxy + Dyx), whose symbols
    are those of Eqs. amp1/amp2: 4 lamx bx^2 sin^2(tx/2), 4 lamy by^2
    sin^2(ty/2) and mu bx by sin(tx) sin(ty) for each transverse operator."""
    chi = 0.7
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = fac * W.cfl_dt(dx, dy, chi)
    bxv, byv = math.cos(alpha), math.sin(alpha)
    co = O.face_coeffs(np.full((ny, nx), bxv), np.full((ny, nx), byv), O.BC_PERIODIC)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    kx, ky = 2 * math.pi * mx, 2 * math.pi * my
    T0 = np.cos(kx * x[None, :] + ky * y[:, None] + 0.2)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    tx, ty = kx * dx, ky * dy
    r = (1.0 - 4 * lamx * bxv ** 2 * math.sin(tx / 2) ** 2 - 4 * lamy * byv ** 2 * math.sin(ty / 2) ** 2
         - 2 * mu * bxv * byv * math.sin(tx) * math.sin(ty))
    T1 = O.explicit_step(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, limiter=O.LIM_ARITH)
    np.testing.assert_allclose(T1, r * T0, atol=1e-13)


def test_explicit_step_one_dimensional_is_ftcs():
    """b = x, T depending on x only: the textbook FTCS update
    T_i + lam (T_{i+1} - 2 T_i + T_{i-1}), any limiter."""
    nx, ny = 24, 6
    rng = np.random.default_rng(4)
    Tx = rng.normal(size=nx)
    T0 = np.tile(Tx, (ny, 1))
    co = O.face_coeffs(np.ones((ny, nx)), np.zeros((ny, nx)), O.BC_PERIODIC)
    dx, dy, chi, dt = 1.0 / nx, 1.0 / ny, 1.0, 0.3 / nx ** 2
    lam = chi * dt / dx ** 2
    ref = Tx + lam * (np.roll(Tx, -1) - 2 * Tx + np.roll(Tx, 1))
    for lim in (O.LIM_VANLEER, O.LIM_ARITH, O.LIM_MC):
        T1 = O.explicit_step(T0, co, O.BC_PERIODIC, dt, dx, dy, chi, limiter=lim)
        np.testing.assert_allclose(T1, np.tile(ref, (ny, 1)), atol=1e-14)


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_ZEROFLUX])
def test_explicit_step_conserves(bc):
    inst = W.random_instance(20, 16, seed=2, dt_factor=0.4) if bc == O.BC_PERIODIC else \
        W.ring_instance(20, ny=16, dt_factor=0.4)
    co = O.face_coeffs(inst.bx, inst.by, bc, inst.chi_par)
    T1 = O.explicit_step(inst.T0, co, bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=7)
    assert abs(np.sum(T1) - np.sum(inst.T0)) <= 1e-12 * abs(np.sum(inst.T0))


def test_explicit_ring_minimum_matches_paper():
    """Section 3.1, caption of the minimum-temperature figure: the explicit
    method without limiters at ncfl = 1 reaches min T = -0.41 on the 512^2 ring
    (10 / 0.1); with the van Leer limiter there are no oscillations at a
    CFL-stable step.  Stored in tests/golden with the citation."""
    g = json.load(open(os.path.join(GOLDEN, "ring_explicit_paper_values.json")))
    n, chi = g["n"], g["chi_par"]
    inst = W.ring_instance(n, t_hot=g["T_hot"], t_cold=g["T_cold"], chi_par=chi, dt_factor=1.0)
    dt = g["ncfl"] * inst.dx ** 2 / (4 * chi)   # Eq. ncfl
    co = O.face_coeffs(inst.bx, inst.by, O.BC_ZEROFLUX, chi)
    lows = {}
    for lim in (O.LIM_ARITH, O.LIM_VANLEER):
        T, lo = inst.T0.copy(), np.inf
        for _ in range(g["steps_checked"] // 50):
            T = O.explicit_step(T, co, O.BC_ZEROFLUX, dt, inst.dx, inst.dy, chi, nsteps=50, limiter=lim)
            lo = min(lo, T.min())
        lows[lim] = lo
    assert abs(lows[O.LIM_ARITH] - g["min_T_without_limiter"]) < g["min_T_tolerance"]
    assert lows[O.LIM_VANLEER] >= g["T_cold"] * (1 - 1e-12)


# ----------------------------------- fixed boundary nodes and source term

def _pinned_nodes(nx, ny):
    return [j * nx + i for j in range(ny) for i in range(nx) if i in (0, nx - 1) or j in (0, ny - 1)]


@pytest.mark.parametrize("nx,ny", [(6, 7), (7, 5)])
def test_fixed_boundary_step_matches_dense_operator(nx, ny):
    """bc 2 (the convergence test's T = 0 on the boundary): the outer ring of
    nodes are identity rows of every directional operator, and the source is
    an explicit stage: T1 = M (T0 + dt Q) with M = Eq. op_2step assembled
    densely (arithmetic-mean transverse average) with those identity rows."""
    rng = np.random.default_rng(nx + 10 * ny)
    ang = rng.uniform(0, 2 * math.pi, (ny, nx))
    co = O.face_coeffs(np.cos(ang), np.sin(ang), O.BC_DIRICHLET, chi_par=1.0, chi_perp=0.1)
    dx, dy, chi = 1.0 / (nx - 1), 1.0 / (ny - 1), 0.6
    dt = 25 * W.cfl_dt(dx, dy, chi)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    T0 = rng.normal(size=(ny, nx))
    Q = rng.normal(size=(ny, nx))
    pins = _pinned_nodes(nx, ny)
    Q.ravel()[pins] = 0.0
    # the zero-flux assembly gives the interior rows; boundary rows become identity
    M = {}
    for xf in (True, False):
        per = False
        N = nx * ny
        mats = []
        for which in ("x", "y"):
            A, E = np.zeros((N, N)), np.zeros((N, N))
            for j in range(ny):
                for i in range(nx):
                    k = j * nx + i
                    if which == "x":
                        gp = co.cxx[j, i] if i < nx - 1 else 0.0
                        gm = co.cxx[j, i - 1] if i > 0 else 0.0
                        ep = co.cxy[j, i] if i < nx - 1 else 0.0
                        em = co.cxy[j, i - 1] if i > 0 else 0.0
                        A[k, k] += 1 + lamx * (gp + gm)
                        if gp: A[k, _cell(i + 1, j, nx, ny, per)] -= lamx * gp
                        if gm: A[k, _cell(i - 1, j, nx, ny, per)] -= lamx * gm
                        E[k, k] += 1
                        for (ii, sg, e) in ((i, 1, ep), (i - 1, -1, em)):
                            if not e:
                                continue
                            for (ci, cj, sv) in ((ii + 1, j + 1, 1), (ii + 1, j - 1, -1), (ii, j + 1, 1), (ii, j - 1, -1)):
                                E[k, _cell(ci, cj, nx, ny, per)] += sg * mu * e * 0.25 * sv
                    else:
                        gp = co.cyy[j, i] if j < ny - 1 else 0.0
                        gm = co.cyy[j - 1, i] if j > 0 else 0.0
                        ep = co.cyx[j, i] if j < ny - 1 else 0.0
                        em = co.cyx[j - 1, i] if j > 0 else 0.0
                        A[k, k] += 1 + lamy * (gp + gm)
                        if gp: A[k, _cell(i, j + 1, nx, ny, per)] -= lamy * gp
                        if gm: A[k, _cell(i, j - 1, nx, ny, per)] -= lamy * gm
                        E[k, k] += 1
                        for (jj, sg, e) in ((j, 1, ep), (j - 1, -1, em)):
                            if not e:
                                continue
                            for (ci, cj, sv) in ((i + 1, jj + 1, 1), (i - 1, jj + 1, -1), (i + 1, jj, 1), (i - 1, jj, -1)):
                                E[k, _cell(ci, cj, nx, ny, per)] += sg * mu * e * 0.25 * sv
            for k in pins:
                A[k, :] = 0.0
                E[k, :] = 0.0
                A[k, k] = E[k, k] = 1.0
            mats.append(np.linalg.solve(A, E))
        Mx, My = mats
        M[xf] = My @ Mx if xf else Mx @ My
    for order, xf in ((O.ORDER_XY, True), (O.ORDER_YX, False)):
        T1 = O.step(T0, co, O.BC_DIRICHLET, dt, dx, dy, chi, order=order, limiter=O.LIM_ARITH, Q=Q)
        np.testing.assert_allclose(T1.ravel(), M[xf] @ (T0 + dt * Q).ravel(), atol=1e-12)
        np.testing.assert_array_equal(T1.ravel()[pins], (T0 + dt * Q).ravel()[pins])


def _steady_center(inst, co, tol=1e-11):
    T, prev, c = inst.T0.copy(), 0.0, inst.nx // 2
    for _ in range(2000):
        T = O.step(T, co, O.BC_DIRICHLET, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=100, Q=inst.Q)
        v = T[c, c]
        if abs(v - prev) < tol * abs(v):
            return v, T
        prev = v
    raise AssertionError("no steady state")


def test_fixed_boundary_isotropic_steady_state_is_second_order():
    """chi_perp = chi_par makes the operator isotropic: the steady state of
    the convergence test (Q = 2 pi^2 cos(pi x) cos(pi y), T = 0 on the
    boundary) is cos(pi x) cos(pi y), so T(0,0) -> 1; the error falls by 4
    per halving of the spacing (second order) at a fixed ncfl."""
    errs = []
    for n in (9, 17, 33):
        inst = W.sovinec_instance(n, ncfl=1.0, chi_perp=1.0)
        co = O.face_coeffs(inst.bx, inst.by, O.BC_DIRICHLET, inst.chi_par, inst.chi_perp)
        v, T = _steady_center(inst, co)
        errs.append(abs(v - 1.0))
        assert np.all(T[0, :] == 0.0) and np.all(T[:, -1] == 0.0)
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5



def test_results_do_not_depend_on_the_thread_count():
    # Every line is solved independently, so the OpenMP thread count cannot
    # change a bit of the result.
    inst = W.random_instance(96, 64, seed=4, dt_factor=300.0)
    co = O.face_coeffs(inst.bx, inst.by, inst.bc, inst.chi_par)
    nt = O.num_threads()
    try:
        O.set_num_threads(1)
        one = O.step(inst.T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3)
        O.set_num_threads(max(2, nt))
        many = O.step(inst.T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3)
    finally:
        O.set_num_threads(nt)
    assert np.array_equal(one, many)
