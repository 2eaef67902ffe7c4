"""Seeded input generators (no method arithmetic lives here).

Every stream is SplitMix64 with a fixed base seed; instance q of a batch uses
seed BASE_SEED + q.  Draw order within one instance:
  batch only: nx, ny (multiples of 32 in [64, 1024]), log10 chi_par, log10 dt
  factor;
  random field: for kx ascending, ky ascending over 1 <= kx^2+ky^2 <= kmax^2:
    a_k (normal / |k|^2), then phi_k (uniform * 2pi);
  Gaussians: for each of the 16: centre x, centre y, amplitude, width.
Three-dimensional instances (random_instance3d): vector-potential
coefficients for kx, ky, kz ascending over 1 <= |k|^2 <= kmax^2: the three
amplitudes (normal / |k|^2), then phi_k (uniform * 2pi); then 16 Gaussians:
centre x, y, z, amplitude, width.
"""
from dataclasses import dataclass, field
import math

import numpy as np

BASE_SEED = 20100805
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then a 3-step xor-shift /
    multiply finaliser.  Vectorised by drawing the k-th output directly."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.count = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.count + 1, self.count + 1 + n, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            z = self.seed + k * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int = 1) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int = 1) -> np.ndarray:
        """Box-Muller: each normal consumes two uniforms (u1, u2) in that order."""
        u = self.uniform(2 * n).reshape(n, 2)
        r = np.sqrt(-2.0 * np.log(1.0 - u[:, 0]))
        return r * np.cos(2.0 * math.pi * u[:, 1])


@dataclass
class Instance:
    """One grid: cell-centred field (bx, by), initial T, and parameters."""
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    bc: int            # 0 zero-flux, 1 periodic, 2 fixed boundary nodes
    chi_par: float
    chi_perp: float
    dt: float
    nsteps: int
    bx: np.ndarray = field(repr=False)
    by: np.ndarray = field(repr=False)
    T0: np.ndarray = field(repr=False)
    Q: np.ndarray = field(default=None, repr=False)  # source term, or None

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def astype(self, dtype):
        """Copy with bx, by, T0 rounded to `dtype` (the inputs a reduced-
        precision run sees; the oracle widens the same values)."""
        return Instance(self.name, self.nx, self.ny, self.dx, self.dy, self.bc, self.chi_par,
                        self.chi_perp, self.dt, self.nsteps, self.bx.astype(dtype),
                        self.by.astype(dtype), self.T0.astype(dtype),
                        None if self.Q is None else self.Q.astype(dtype))


def cfl_dt(dx: float, dy: float, chi_par: float) -> float:
    """The explicit limit min(dx,dy)^2 / (2 chi_par), the unit of the dt factors."""
    return min(dx, dy) ** 2 / (2.0 * chi_par)


def ring_instance(n: int, t_hot: float = 12.0, t_cold: float = 10.0, chi_par: float = 0.01,
                  dt_factor: float = 10.0, nsteps: int = 250, ny: int = None) -> Instance:
    """Ring test (Section 3.1) on [-1,1]^2 with zero-flux boundaries."""
    nx = n
    ny = n if ny is None else ny
    dx, dy = 2.0 / nx, 2.0 / ny
    x = -1.0 + (np.arange(nx) + 0.5) * dx
    y = -1.0 + (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)                       # [ny, nx]
    r = np.hypot(X, Y)
    theta = np.mod(np.arctan2(Y, X), 2.0 * math.pi)
    hot = (r > 0.5) & (r < 0.7) & (theta > 11.0 * math.pi / 12.0) & (theta < 13.0 * math.pi / 12.0)
    T0 = np.where(hot, t_hot, t_cold).astype(np.float64)
    inside = (r <= 1.0) & (r > 0.0)
    rs = np.where(inside, r, 1.0)
    bx = np.where(inside, -Y / rs, 0.0)
    by = np.where(inside, X / rs, 0.0)
    dt = dt_factor * cfl_dt(dx, dy, chi_par)
    return Instance("ring%dx%d" % (nx, ny), nx, ny, dx, dy, 0, chi_par, 0.0, dt, nsteps,
                    bx, by, T0)


def sovinec_instance(n: int, chi_par: float = 1.0, ncfl: float = 1000.0, chi_perp: float = 0.0,
                     nsteps: int = 0) -> Instance:
    """Convergence test of Section 3.2 (after Sovinec et al.): [-1/2,1/2]^2
    with T = 0 on the boundary, T(0) = 0, source Q = 2 pi^2 cos(pi x) cos(pi y),
    b along the contours of phi = cos(pi x) cos(pi y), i.e. b = z x grad(phi)
    / |grad phi| (b = (1, 0) where |grad phi| < 1e-8).  Nodes x_i = -1/2 +
    i/(n-1): the outer ring sits on the boundary and keeps T = 0 (bc 2); an odd
    n puts a node at the origin, where the steady state is 1/chi_perp,num.
    dt = ncfl dx^2 / (4 chi_par) (Eq. ncfl)."""
    h = 1.0 / (n - 1)
    x = -0.5 + np.arange(n) * h
    X, Y = np.meshgrid(x, x)                       # [ny, nx]
    gx = -math.pi * np.sin(math.pi * X) * np.cos(math.pi * Y)
    gy = -math.pi * np.cos(math.pi * X) * np.sin(math.pi * Y)
    mag = np.hypot(gx, gy)
    small = mag < 1e-8
    safe = np.where(small, 1.0, mag)
    bx = np.where(small, 1.0, -gy / safe)
    by = np.where(small, 0.0, gx / safe)
    Q = 2.0 * math.pi ** 2 * np.cos(math.pi * X) * np.cos(math.pi * Y)
    Q[0, :] = Q[-1, :] = 0.0
    Q[:, 0] = Q[:, -1] = 0.0
    dt = ncfl * h * h / (4.0 * chi_par)
    return Instance("sovinec%d" % n, n, n, h, h, 2, chi_par, chi_perp, dt, nsteps, bx, by,
                    np.zeros((n, n)), Q)


def _random_field(rng: SplitMix64, nx: int, ny: int, kmax: int, chunk_rows: int = 1024):
    """b = z x grad(psi) / |grad psi| for psi = sum a_k cos(2 pi k.x + phi_k),
    evaluated on cell centres ((i+1/2)/nx, (j+1/2)/ny) as a separable sum."""
    ks = np.arange(-kmax, kmax + 1)
    nk = len(ks)
    Cx = np.zeros((nk, nk), dtype=np.complex128)   # [kx, ky]
    Cy = np.zeros((nk, nk), dtype=np.complex128)
    for a_idx, kx in enumerate(ks):
        for b_idx, ky in enumerate(ks):
            k2 = kx * kx + ky * ky
            if k2 < 1 or k2 > kmax * kmax:
                continue
            a = rng.normal(1)[0] / k2
            phi = rng.uniform(1)[0] * 2.0 * math.pi
            w = a * np.exp(1j * phi)
            # d/dx cos(2pi k.x + phi) = -2pi kx sin(.) = Im(-2pi kx e^{i(.)})
            Cx[a_idx, b_idx] = -2.0 * math.pi * kx * w
            Cy[a_idx, b_idx] = -2.0 * math.pi * ky * w
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X = np.exp(2j * math.pi * np.outer(x, ks))     # [nx, nk]
    Y = np.exp(2j * math.pi * np.outer(y, ks))     # [ny, nk]
    bx = np.empty((ny, nx))
    by = np.empty((ny, nx))
    for r0 in range(0, ny, chunk_rows):
        r1 = min(ny, r0 + chunk_rows)
        gx = ((Y[r0:r1] @ Cx.T) @ X.T).imag        # [rows, nx]
        gy = ((Y[r0:r1] @ Cy.T) @ X.T).imag
        mag = np.hypot(gx, gy)
        small = mag < 1e-8
        safe = np.where(small, 1.0, mag)
        bx[r0:r1] = np.where(small, 1.0, -gy / safe)
        by[r0:r1] = np.where(small, 0.0, gx / safe)
    return bx, by


def _gaussians(rng: SplitMix64, nx: int, ny: int, count: int = 16):
    """T = 1 + sum of `count` periodic Gaussians A exp(-r^2 / (2 w^2)) with
    minimum-image distance on the unit torus."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    T = np.ones((ny, nx))
    for _ in range(count):
        cx, cy, ua, uw = rng.uniform(4)
        amp = 0.5 + 1.5 * ua
        w = 0.01 + 0.04 * uw
        ddx = x - cx
        ddx -= np.round(ddx)
        ddy = y - cy
        ddy -= np.round(ddy)
        gx = np.exp(-(ddx * ddx) / (2.0 * w * w))
        gy = np.exp(-(ddy * ddy) / (2.0 * w * w))
        T += amp * np.outer(gy, gx)
    return T


def random_instance(nx: int, ny: int, seed: int = BASE_SEED, kmax: int = 8,
                    chi_par: float = 0.05, dt_factor: float = 100.0, nsteps: int = 100,
                    rng: SplitMix64 = None, name: str = None) -> Instance:
    """Random-field instance on the periodic unit square."""
    rng = SplitMix64(seed) if rng is None else rng
    bx, by = _random_field(rng, nx, ny, kmax)
    T0 = _gaussians(rng, nx, ny)
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = dt_factor * cfl_dt(dx, dy, chi_par)
    return Instance(name or "random%dx%d" % (nx, ny), nx, ny, dx, dy, 1, chi_par, 0.0, dt,
                    nsteps, bx, by, T0)


def batch_instances(count: int = 512, nsteps: int = 200, base_seed: int = BASE_SEED,
                    kmax: int = 8, first: int = 0, size_cap: int = 1024):
    """Uneven batch: instance q draws nx, ny uniformly from the multiples of
    32 in [64, size_cap], chi_par log-uniform in [1e-3, 1e-1] and a dt factor
    log-uniform in [10, 1000] (times the explicit limit), then its own field
    and Gaussians."""
    out = []
    steps = (size_cap - 64) // 32 + 1
    for q in range(first, first + count):
        rng = SplitMix64(base_seed + q)
        u = rng.uniform(4)
        nx = 32 * (2 + int(u[0] * steps))
        ny = 32 * (2 + int(u[1] * steps))
        chi = 10.0 ** (-3.0 + 2.0 * u[2])
        fac = 10.0 ** (1.0 + 2.0 * u[3])
        out.append(random_instance(nx, ny, kmax=kmax, chi_par=chi, dt_factor=fac,
                                   nsteps=nsteps, rng=rng, name="batch%03d" % q))
    return out


# ------------------------------------------------------------ three dimensions

@dataclass
class Instance3:
    """One 3-D grid: cell-centred unit field (bx, by, bz), initial T, all
    [nz][ny][nx], and parameters."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    bc: int            # 0 zero-flux, 1 periodic
    chi_par: float
    chi_perp: float
    dt: float
    nsteps: int
    bx: np.ndarray = field(repr=False)
    by: np.ndarray = field(repr=False)
    bz: np.ndarray = field(repr=False)
    T0: np.ndarray = field(repr=False)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def astype(self, dtype):
        return Instance3(self.name, self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.bc,
                         self.chi_par, self.chi_perp, self.dt, self.nsteps, self.bx.astype(dtype),
                         self.by.astype(dtype), self.bz.astype(dtype), self.T0.astype(dtype))


def _field3d(rng: SplitMix64, nx: int, ny: int, nz: int, kmax: int, guide: float):
    """b = B / |B| with B = guide * z-hat + curl A, A = sum_k a_k cos(2 pi k.x
    + phi_k) (a_k a random vector), so B is divergence-free like a magnetic
    field.  Cell centres ((i+1/2)/nx, ...), evaluated as a separable sum one
    z-plane at a time."""
    ks = np.arange(-kmax, kmax + 1)
    nk = len(ks)
    C = np.zeros((3, nk, nk, nk), dtype=np.complex128)   # B component, [kz, ky, kx]
    for ix, kx in enumerate(ks):
        for iy, ky in enumerate(ks):
            for iz, kz in enumerate(ks):
                k2 = kx * kx + ky * ky + kz * kz
                if k2 < 1 or k2 > kmax * kmax:
                    continue
                a = rng.normal(3) / k2
                phi = rng.uniform(1)[0] * 2.0 * math.pi
                w = np.exp(1j * phi)
                k = 2.0 * math.pi * np.array([kx, ky, kz], dtype=np.float64)
                # curl of a cos(k.x + phi) = -(k x a) sin(k.x + phi) = Im(-(k x a) e^{i(.)})
                C[:, iz, iy, ix] = -np.cross(k, a) * w
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    X = np.exp(2j * math.pi * np.outer(x, ks))     # [nx, nk]
    Y = np.exp(2j * math.pi * np.outer(y, ks))     # [ny, nk]
    Z = np.exp(2j * math.pi * np.outer(z, ks))     # [nz, nk]
    out = np.empty((3, nz, ny, nx))
    for c in range(3):
        CX = np.einsum("zyk,xk->zyx", C[c], X)     # [kz, ky, x]
        for p in range(nz):
            Cz = np.tensordot(Z[p], CX, axes=(0, 0))   # [ky, x]
            out[c, p] = (Y @ Cz).imag                   # [y, x]
    out[2] += guide
    mag = np.sqrt(out[0] ** 2 + out[1] ** 2 + out[2] ** 2)
    small = mag < 1e-8
    safe = np.where(small, 1.0, mag)
    bx = np.where(small, 0.0, out[0] / safe)
    by = np.where(small, 0.0, out[1] / safe)
    bz = np.where(small, 1.0, out[2] / safe)
    return bx, by, bz


def _gaussians3d(rng: SplitMix64, nx: int, ny: int, nz: int, count: int = 16):
    """T = 1 + sum of `count` periodic Gaussians A exp(-r^2 / (2 w^2)) on the
    unit torus (minimum-image distance), A in [0.5, 2], w in [0.02, 0.08]."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    T = np.ones((nz, ny, nx))
    for _ in range(count):
        cx, cy, cz, ua, uw = rng.uniform(5)
        amp = 0.5 + 1.5 * ua
        w = 0.02 + 0.06 * uw
        g = []
        for v, c in ((x, cx), (y, cy), (z, cz)):
            d = v - c
            d -= np.round(d)
            g.append(np.exp(-(d * d) / (2.0 * w * w)))
        T += amp * g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]
    return T


def random_instance3d(nx: int, ny: int, nz: int, seed: int = BASE_SEED, kmax: int = 3,
                      guide: float = 1.0, chi_par: float = 0.05, dt_factor: float = 10.0,
                      nsteps: int = 20, bc: int = 1, chi_perp: float = 0.0) -> Instance3:
    """Random divergence-free field and Gaussian blobs on the unit cube;
    dt = dt_factor * min(dx, dy, dz)^2 / (2 chi_par)."""
    rng = SplitMix64(seed)
    bx, by, bz = _field3d(rng, nx, ny, nz, kmax, guide)
    T0 = _gaussians3d(rng, nx, ny, nz)
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    dt = dt_factor * min(dx, dy, dz) ** 2 / (2.0 * chi_par)
    return Instance3("random3d_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, dx, dy, dz, bc, chi_par,
                     chi_perp, dt, nsteps, bx, by, bz, T0)
