"""Pins for the three-dimensional FP64 oracle (Section 2.1) against what the
paper and the mathematics fix.

- The 3-D amplification factor the paper prints for the x-update (r1 of
  Section 2.1) and its y and z analogues, mode by mode, update by update.
- The paper's stability limit of the 2-step scheme in three dimensions,
  chi dt / dx^2 <= 8.25: a grid mode grows at 8.3 and none grows at 8.2.
- The paper's statement that the 4-step scheme (Eq. 4step) is stable in
  three dimensions at any timestep.
- Exact reductions: a field in a coordinate plane with T constant across
  it gives the already pinned 2-D oracle step on every slice; b along z
  gives 1-D backward Euler.
- Invariants: conservation, and mirror symmetry in each axis.
A dropped transverse term, a wrong sign, a swapped axis or a shifted face
index fails at least one of these.
"""
import math

import numpy as np
import pytest

import oracle as O


def _unit(rng, shape):
    b = rng.normal(size=(3,) + shape)
    return b / np.linalg.norm(b, axis=0)


def _const_field(b, shape):
    return [np.full(shape, float(v)) for v in b]


def _r_factors(lam, mu, b, kd, half=False):
    """The paper's r1 and its two analogues for one Fourier mode: kd[d] =
    k_d Delta_d.  half=True gives the 4-step factors (implicit part over
    dt/2, twice)."""
    s = [math.sin(k) for k in kd]
    h = [math.sin(k / 2) ** 2 for k in kd]
    out = []
    for d in range(3):
        a, c = (d + 1) % 3, (d + 2) % 3
        num = 1.0 - mu[2 * d] * b[d] * b[a] * s[d] * s[a] - mu[2 * d + 1] * b[d] * b[c] * s[d] * s[c]
        if half:
            out.append(num / (1.0 + 2.0 * lam[d] * b[d] ** 2 * h[d]) ** 2)
        else:
            out.append(num / (1.0 + 4.0 * lam[d] * b[d] ** 2 * h[d]))
    return out


def _mode(shape, m):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = 2 * np.pi * (m[0] * i / nx + m[1] * j / ny + m[2] * k / nz)
    return np.cos(ph), [2 * np.pi * m[0] / nx, 2 * np.pi * m[1] / ny, 2 * np.pi * m[2] / nz]


# ------------------------------------------------ amplification factors

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_each_update_multiplies_a_mode_by_the_printed_factor(seed):
    # Section 2.1: with constant b and the linear (arithmetic-mean) average,
    # the x-update multiplies a Fourier mode by r1 and the y- and z-updates
    # by its analogues; the grid spacings differ so every mixed factor
    # chi dt / (Delta_d Delta_a) is distinct.
    rng = np.random.default_rng(seed)
    shape = (6, 10, 8)
    b = _unit(rng, ())
    co = O.face_coeffs3(*_const_field(b, shape), O.BC_PERIODIC)
    dx, dy, dz, chi, dt = 0.7, 1.1, 0.9, 1.0, 3.0
    lam, mu = O.lambdas3(dt, dx, dy, dz, chi)
    for m in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 2, 1), (3, 1, 2), (2, 4, 1), (4, 5, 3)]:
        T, kd = _mode(shape, m)
        r = _r_factors(lam, mu, b, kd)
        U = T
        for d in range(3):
            U2 = O.sweep3(U, co, O.BC_PERIODIC, d, lam[d], mu[2 * d], mu[2 * d + 1], O.LIM_ARITH)
            np.testing.assert_allclose(U2, r[d] * U, rtol=0, atol=1e-13)
            U = U2
        full = O.step3(T, co, O.BC_PERIODIC, dt, dx, dy, dz, chi, limiter=O.LIM_ARITH)
        np.testing.assert_allclose(full, r[0] * r[1] * r[2] * T, rtol=0, atol=1e-13)
        four = O.step3(T, co, O.BC_PERIODIC, dt, dx, dy, dz, chi, limiter=O.LIM_ARITH,
                       scheme=O.SCHEME_4STEP)
        r4 = _r_factors(lam, mu, b, kd, half=True)
        np.testing.assert_allclose(four, r4[0] * r4[1] * r4[2] * T, rtol=0, atol=1e-13)


# ---------------------------------------------------- stability limit

_GRID = (12, 12, 28)   # (nz, ny, nx): modes with k_x dx near 0.67, k_y dy and k_z dz near 0.52


def _grid_modes(shape):
    """k_d Delta_d of the grid modes with no zero component, as [mx-1, my-1,
    mz-1] arrays.  A mode with a zero component is a 2-D (or 1-D) mode, for
    which the split is unconditionally stable (Section 2.1)."""
    nz, ny, nx = shape
    kx = 2 * np.pi * np.arange(1, nx) / nx
    ky = 2 * np.pi * np.arange(1, ny) / ny
    kz = 2 * np.pi * np.arange(1, nz) / nz
    return np.meshgrid(kx, ky, kz, indexing="ij")


def _max_r(lam, b, K, half=False):
    bx, by, bz = b
    KX, KY, KZ = K
    sx, sy, sz = np.sin(KX), np.sin(KY), np.sin(KZ)
    hx, hy, hz = np.sin(KX / 2) ** 2, np.sin(KY / 2) ** 2, np.sin(KZ / 2) ** 2
    p, q = (2.0, 2) if half else (4.0, 1)   # 4-step: (1 + 2 lam b^2 h)^2; 2-step: 1 + 4 lam b^2 h
    r1 = (1 - lam * bx * by * sx * sy - lam * bx * bz * sx * sz) / (1 + p * lam * bx * bx * hx) ** q
    r2 = (1 - lam * by * bz * sy * sz - lam * by * bx * sy * sx) / (1 + p * lam * by * by * hy) ** q
    r3 = (1 - lam * bz * bx * sz * sx - lam * bz * by * sz * sy) / (1 + p * lam * bz * bz * hz) ** q
    r = np.abs(r1 * r2 * r3)
    idx = np.unravel_index(np.argmax(r), r.shape)
    return float(r[idx]), idx


def _directions(n=36):
    th = np.linspace(0.02, np.pi - 0.02, n)
    ph = np.linspace(0.0, 2 * np.pi, 2 * n, endpoint=False) + 0.01
    for t in th:
        for p in ph:
            yield (math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t))


def _worst(lam, K, half=False):
    """Largest |r| over the grid modes K and all field directions: a scan of
    the sphere, then a local search from the twenty best directions (the
    growing region is narrow in b)."""
    from scipy.optimize import minimize

    def sph(p):
        return (math.sin(p[0]) * math.cos(p[1]), math.sin(p[0]) * math.sin(p[1]), math.cos(p[0]))

    scan = []
    for b in _directions():
        scan.append((_max_r(lam, b, K, half)[0], b))
    scan.sort(key=lambda t: -t[0])
    best = (0.0, None, None)
    for _, b in scan[:20]:
        p0 = [math.acos(max(-1.0, min(1.0, b[2]))), math.atan2(b[1], b[0])]
        res = minimize(lambda p: -_max_r(lam, sph(p), K, half)[0], p0, method="Nelder-Mead",
                       options=dict(xatol=1e-9, fatol=1e-15, maxiter=2000))
        bb = sph(res.x)
        r, idx = _max_r(lam, bb, K, half)
        if r > best[0]:
            best = (r, bb, idx)
    return best


def test_two_step_3d_stability_limit_brackets_the_papers_8_25():
    # Section 2.1: with dx = dy = dz the 2-step scheme in three dimensions is
    # stable for chi dt / dx^2 up to 8.25.  Over the modes of a 28x12x12
    # periodic grid and a sphere of directions, no mode grows at 8.2 and
    # one does at 8.3; the oracle then reproduces that growth.
    K = _grid_modes(_GRID)
    r_lo, _, _ = _worst(8.2, K)
    assert r_lo < 1.0
    r_hi, b, idx = _worst(8.3, K)
    assert r_hi > 1.0 + 1e-4
    m = (idx[0] + 1, idx[1] + 1, idx[2] + 1)  # (mx, my, mz) of the growing mode
    T, kd = _mode(_GRID, m)
    co = O.face_coeffs3(*_const_field(b, _GRID), O.BC_PERIODIC)
    T1 = O.step3(T, co, O.BC_PERIODIC, 8.3, 1.0, 1.0, 1.0, 1.0, limiter=O.LIM_ARITH)
    ratio = float(np.sum(T1 * T) / np.sum(T * T))
    assert abs(ratio) == pytest.approx(r_hi, rel=1e-10)
    # below the limit the discrete L2 norm never grows (all |r| <= 1 and
    # the Fourier modes are orthogonal)
    rng = np.random.default_rng(5)
    U = rng.normal(size=_GRID)
    n0 = np.linalg.norm(U)
    for _ in range(5):
        U = O.step3(U, co, O.BC_PERIODIC, 8.2, 1.0, 1.0, 1.0, 1.0, limiter=O.LIM_ARITH)
        n1 = np.linalg.norm(U)
        assert n1 <= n0 * (1 + 1e-12)
        n0 = n1


def test_four_step_3d_is_stable_at_large_timesteps():
    # Section 2.1: the 4-step scheme (Eq. 4step) is stable in three
    # dimensions at any timestep.
    K = _grid_modes(_GRID)
    for lam in (8.3, 100.0, 1e4):
        r, _, _ = _worst(lam, K, half=True)
        assert r < 1.0
    rng = np.random.default_rng(6)
    b = _unit(rng, ())
    co = O.face_coeffs3(*_const_field(b, _GRID), O.BC_PERIODIC)
    U = rng.normal(size=_GRID)
    n0 = np.linalg.norm(U)
    for _ in range(4):
        U = O.step3(U, co, O.BC_PERIODIC, 1000.0, 1.0, 1.0, 1.0, 1.0, limiter=O.LIM_ARITH,
                    scheme=O.SCHEME_4STEP)
        n1 = np.linalg.norm(U)
        assert n1 <= n0 * (1 + 1e-12)
        n0 = n1


# ---------------------------------------------------- exact reductions

@pytest.mark.parametrize("bc", [O.BC_ZEROFLUX, O.BC_PERIODIC])
@pytest.mark.parametrize("scheme", [O.SCHEME_2STEP, O.SCHEME_4STEP])
@pytest.mark.parametrize("plane", ["xy", "yz", "zx"])
def test_plane_field_reduces_to_the_2d_step(bc, scheme, plane):
    # b in a coordinate plane and T constant along the third axis: that
    # axis's update is the identity and the other two carry no term along
    # it, so every slice takes the (separately pinned) 2-D step, the two
    # in-plane updates in the order x, y, z; likewise for the 4-step form
    # against the 2-D Eq. 4step.
    rng = np.random.default_rng({"xy": 1, "yz": 2, "zx": 3}[plane] + 10 * bc)
    shape = (5, 6, 7)  # (nz, ny, nx)
    dx, dy, dz, chi, dt = 0.8, 1.3, 1.1, 1.0, 4.0
    if plane == "xy":    # 2-D (x, y) = 3-D (x, y); slices along z
        n2 = (shape[1], shape[2])
        b2 = rng.normal(size=(2,) + n2)
        b2 /= np.linalg.norm(b2, axis=0)
        T2 = rng.uniform(1, 2, n2)
        bx = np.broadcast_to(b2[0], shape).copy()
        by = np.broadcast_to(b2[1], shape).copy()
        bz = np.zeros(shape)
        T = np.broadcast_to(T2, shape).copy()
        d2 = (dx, dy)
        take = lambda U: [U[k] for k in range(shape[0])]  # noqa: E731
    elif plane == "yz":  # 2-D (x, y) = 3-D (y, z); slices along x
        n2 = (shape[0], shape[1])
        b2 = rng.normal(size=(2,) + n2)
        b2 /= np.linalg.norm(b2, axis=0)
        T2 = rng.uniform(1, 2, n2)
        bx = np.zeros(shape)
        by = np.repeat(b2[0][:, :, None], shape[2], axis=2)
        bz = np.repeat(b2[1][:, :, None], shape[2], axis=2)
        T = np.repeat(T2[:, :, None], shape[2], axis=2)
        d2 = (dy, dz)
        take = lambda U: [U[:, :, i] for i in range(shape[2])]  # noqa: E731
    else:                # 2-D (x, y) = 3-D (x, z); slices along y
        n2 = (shape[0], shape[2])
        b2 = rng.normal(size=(2,) + n2)
        b2 /= np.linalg.norm(b2, axis=0)
        T2 = rng.uniform(1, 2, n2)
        bx = np.repeat(b2[0][:, None, :], shape[1], axis=1)
        by = np.zeros(shape)
        bz = np.repeat(b2[1][:, None, :], shape[1], axis=1)
        T = np.repeat(T2[:, None, :], shape[1], axis=1)
        d2 = (dx, dz)
        take = lambda U: [U[:, j, :] for j in range(shape[1])]  # noqa: E731
    co3 = O.face_coeffs3(bx, by, bz, bc)
    got = O.step3(T, co3, bc, dt, dx, dy, dz, chi, nsteps=2, scheme=scheme)
    co2 = O.face_coeffs(b2[0], b2[1], bc)
    two_d = O.step if scheme == O.SCHEME_2STEP else O.step4  # Eq. op_2step / Eq. 4step in 2-D
    want = two_d(T2, co2, bc, dt, d2[0], d2[1], chi, nsteps=2)
    for s in take(got):
        np.testing.assert_allclose(s, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("bc", [O.BC_ZEROFLUX, O.BC_PERIODIC])
def test_field_along_z_is_1d_backward_euler(bc):
    # b = z-hat: only the z-update acts, and it is backward Euler in z; a
    # cosine in z (cell-centred for zero-flux, grid mode for periodic) decays
    # by 1 / (1 + 4 lam_z sin^2(k dz / 2)) per step.
    nz, ny, nx = 16, 4, 8
    dz, chi, dt = 0.5, 1.0, 2.0
    k = np.arange(nz)
    if bc == O.BC_PERIODIC:
        kd = 2 * np.pi * 3 / nz
        prof = np.cos(kd * k)
    else:
        kd = np.pi * 3 / nz
        prof = np.cos(kd * (k + 0.5))
    T = np.broadcast_to(prof[:, None, None], (nz, ny, nx)).copy()
    shape = T.shape
    co = O.face_coeffs3(np.zeros(shape), np.zeros(shape), np.ones(shape), bc)
    got = O.step3(T, co, bc, dt, 1.0, 1.0, dz, chi, nsteps=3)
    lamz = chi * dt / dz ** 2
    np.testing.assert_allclose(got, T / (1 + 4 * lamz * math.sin(kd / 2) ** 2) ** 3, rtol=0, atol=1e-14)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("bc", [O.BC_ZEROFLUX, O.BC_PERIODIC])
@pytest.mark.parametrize("scheme", [O.SCHEME_2STEP, O.SCHEME_4STEP])
@pytest.mark.parametrize("limiter", [O.LIM_VANLEER, O.LIM_MC])
def test_conservation_3d(bc, scheme, limiter):
    # Every face flux leaves one cell and enters its neighbour, and zero-flux
    # boundary faces carry nothing: sum(T) is constant to rounding.
    rng = np.random.default_rng(7 + bc + 2 * scheme + 4 * limiter)
    shape = (8, 9, 10)
    b = _unit(rng, shape)
    co = O.face_coeffs3(*b, bc)
    T = rng.uniform(0.1, 10.0, shape)
    got = O.step3(T, co, bc, 50.0, 1.0, 0.8, 1.2, 1.0, nsteps=3, limiter=limiter, scheme=scheme)
    assert abs(got.sum() - T.sum()) <= 1e-12 * T.sum()


@pytest.mark.parametrize("bc", [O.BC_ZEROFLUX, O.BC_PERIODIC])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry_3d(bc, axis):
    # Reflecting the grid in one axis and reversing that component of b
    # reflects the result: the limiter is odd and symmetric, and face i+1/2
    # maps to face n-2-i+1/2.  A face index off by one breaks this.
    rng = np.random.default_rng(20 + axis + 3 * bc)
    shape = (6, 7, 8)
    b = _unit(rng, shape)
    T = rng.uniform(0.0, 1.0, shape)
    ax = 2 - axis  # numpy axis of x, y, z
    bc_ = O.face_coeffs3(*b, bc)
    got = O.step3(T, bc_, bc, 20.0, 1.0, 1.0, 1.0, 1.0, nsteps=2)
    br = [np.flip(c, axis=ax).copy() for c in b]
    br[axis] = -br[axis]
    cor = O.face_coeffs3(*br, bc)
    got_r = O.step3(np.flip(T, axis=ax).copy(), cor, bc, 20.0, 1.0, 1.0, 1.0, 1.0, nsteps=2)
    np.testing.assert_allclose(np.flip(got_r, axis=ax), got, rtol=0, atol=1e-13)
