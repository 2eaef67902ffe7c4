"""GPU parity of the three-dimensional split step (Section 2.1) through the
C ABI (aniso3_*) against the FP64 oracle (oracle.step3) on the same seeded
inputs: FP64 within 1e-12 relative per step, FP32 within 1e-4 relative
L-inf (or 3x the problem's own FP32 noise floor where that is larger).
Shapes span several blocks of lines, ragged line counts, the shortest and
the longest lines the kernel takes, and unequal spacings."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
FP64_TOL_PER_STEP = 1e-12
FP32_TOL = 1e-4


def rel_linf(a, ref):
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


class Grid3:
    """One aniso3 handle with its field set and T resident on the device."""

    def __init__(self, P, inst, prec, limiter=0, scheme=0, warps=0, seg=0, fp16=False):
        import torch
        self.P, self.inst = P, inst
        self.dtype = torch.float64 if prec == FP64 else torch.float32
        self.h = P.aniso3_create(inst.nx, inst.ny, inst.nz, inst.dx, inst.dy, inst.dz, inst.chi_par,
                                 inst.chi_perp, inst.bc)
        P.aniso3_set_option(self.h, P.ANISO_OPT_PRECISION, prec)
        if fp16:
            P.aniso3_set_option(self.h, P.ANISO_OPT_FIELD_FP16, 1)
        P.aniso3_set_option(self.h, P.ANISO_OPT_LIMITER, limiter)
        P.aniso3_set_option(self.h, P.ANISO_OPT_SCHEME, scheme)
        if warps:
            P.aniso3_set_option(self.h, P.ANISO_OPT_BLOCK_WARPS, warps)
        if seg:
            P.aniso3_set_option(self.h, P.ANISO_OPT_SEGMENT, seg)
        self.b = [torch.tensor(a, dtype=self.dtype, device="cuda") for a in (inst.bx, inst.by, inst.bz)]
        P.aniso3_set_field(self.h, *self.b)
        self.T = torch.tensor(inst.T0, dtype=self.dtype, device="cuda")

    def step(self, nsteps, dt=None):
        self.P.aniso3_step(self.h, self.T, self.inst.dt if dt is None else dt, nsteps)
        self.P.aniso3_sync(self.h)
        return self.T.double().cpu().numpy()

    def close(self):
        self.P.aniso3_destroy(self.h)


def oracle_run(inst, prec, nsteps, limiter=0, scheme=0, round_each_step=False, fp16=False):
    """The oracle on the inputs the GPU sees (rounded to its precision,
    widened exactly; with fp16, the face coefficients rounded to FP16 as the
    GPU stores them).  round_each_step: round the state to FP32 after every
    step (the FP32 noise floor of the problem)."""
    dt = np.float64 if prec == FP64 else np.float32
    b = [a.astype(dt).astype(np.float64) for a in (inst.bx, inst.by, inst.bz)]
    T = inst.T0.astype(dt).astype(np.float64)
    co = O.face_coeffs3(*b, inst.bc, inst.chi_par, inst.chi_perp)
    if fp16:
        co = co.rounded(np.float16)
    if not round_each_step:
        return O.step3(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.dz, inst.chi_par, nsteps=nsteps,
                       limiter=limiter, scheme=scheme)
    for _ in range(nsteps):
        T = O.step3(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.dz, inst.chi_par, nsteps=1,
                    limiter=limiter, scheme=scheme).astype(np.float32).astype(np.float64)
    return T


def _inst(nx, ny, nz, bc, seed, dt_factor=10.0, nsteps=3, chi_perp=0.0):
    return W.random_instance3d(nx, ny, nz, seed=seed, bc=bc, dt_factor=dt_factor, nsteps=nsteps,
                               chi_perp=chi_perp)


# (nx, ny, nz): multiples of the 16-byte vector in every axis; small and long
# lines, line counts that leave a ragged last block, unequal spacings
SHAPES64 = [(4, 4, 4), (6, 10, 8), (16, 12, 22), (30, 18, 14), (64, 40, 24), (128, 6, 10)]
SHAPES32 = [(8, 8, 8), (8, 12, 20), (32, 28, 16), (64, 36, 44), (128, 16, 24), (12, 96, 8)]


@pytest.mark.parametrize("shape", SHAPES64)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_steps_fp64(lib, shape, bc, scheme):
    inst = _inst(*shape, bc, seed=sum(shape) + bc, nsteps=3)
    ref = oracle_run(inst, FP64, inst.nsteps, scheme=scheme)
    g = Grid3(lib, inst, FP64, scheme=scheme)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < FP64_TOL_PER_STEP * inst.nsteps


@pytest.mark.parametrize("limiter", [0, 1, 2, 3])
@pytest.mark.parametrize("chi_perp", [0.0, 0.01])
def test_limiters_and_chi_perp_fp64(lib, limiter, chi_perp):
    inst = _inst(24, 16, 20, 1, seed=40 + limiter, nsteps=2, chi_perp=chi_perp)
    ref = oracle_run(inst, FP64, inst.nsteps, limiter=limiter)
    g = Grid3(lib, inst, FP64, limiter=limiter)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < FP64_TOL_PER_STEP * inst.nsteps


@pytest.mark.parametrize("shape", SHAPES32)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_steps_fp32(lib, shape, bc, scheme):
    inst = _inst(*shape, bc, seed=3 * sum(shape) + bc, nsteps=4)
    ref = oracle_run(inst, FP32, inst.nsteps, scheme=scheme)
    floor = rel_linf(oracle_run(inst, FP32, inst.nsteps, scheme=scheme, round_each_step=True), ref)
    g = Grid3(lib, inst, FP32, scheme=scheme)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < max(FP32_TOL, 3.0 * floor)


@pytest.mark.parametrize("warps,seg", [(4, 2), (8, 8), (2, 4)])
def test_block_shapes_fp32(lib, warps, seg):
    inst = _inst(64, 32, 48, 1, seed=77, nsteps=2)
    ref = oracle_run(inst, FP32, inst.nsteps)
    g = Grid3(lib, inst, FP32, warps=warps, seg=seg)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < FP32_TOL


@pytest.mark.parametrize("prec,shape", [(FP64, (1024, 4, 6)), (FP64, (6, 4, 1024)), (FP32, (2048, 8, 8)),
                                         (FP32, (8, 2048, 8)), (FP32, (8, 8, 2048))])
def test_longest_lines(lib, prec, shape):
    inst = _inst(*shape, 1, seed=5, nsteps=1)
    ref = oracle_run(inst, prec, 1)
    g = Grid3(lib, inst, prec)
    try:
        got = g.step(1)
    finally:
        g.close()
    assert rel_linf(got, ref) < (FP64_TOL_PER_STEP if prec == FP64 else FP32_TOL)


def test_large_grid_fp32_sampled(lib):
    """128 x 96 x 160 (about 2M cells, many waves of blocks): the whole
    result against the oracle."""
    inst = _inst(128, 96, 160, 1, seed=9, nsteps=2)
    ref = oracle_run(inst, FP32, inst.nsteps)
    g = Grid3(lib, inst, FP32)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < FP32_TOL


@pytest.mark.parametrize("bc", [0, 1])
def test_conservation_fp64(lib, bc):
    inst = _inst(32, 24, 16, bc, seed=11, nsteps=10, dt_factor=30.0)
    g = Grid3(lib, inst, FP64, scheme=1)
    try:
        s0 = lib.aniso3_total(g.h, g.T)[0]
        g.step(inst.nsteps)
        s1, lo, hi, nf = lib.aniso3_total(g.h, g.T)
    finally:
        g.close()
    assert nf == 0
    assert abs(s1 - s0) <= 1e-12 * abs(s0)
    assert s0 == pytest.approx(float(inst.T0.sum()), rel=1e-14)


def test_first_step_stays_within_initial_bounds(lib):
    """With the van Leer limiter a large first step makes no new extrema on
    this smooth problem (the 3-D counterpart of the ring test's bound is not
    claimed by the paper; this checks the GPU keeps the oracle's extrema)."""
    inst = _inst(32, 32, 32, 1, seed=13, nsteps=1, dt_factor=10.0)
    ref = oracle_run(inst, FP64, 1)
    g = Grid3(lib, inst, FP64)
    try:
        got = g.step(1)
    finally:
        g.close()
    assert got.min() == pytest.approx(ref.min(), rel=1e-12)
    assert got.max() == pytest.approx(ref.max(), rel=1e-12)


def test_nonfinite_is_reported(lib):
    import torch
    inst = _inst(16, 8, 8, 1, seed=2, nsteps=1)
    g = Grid3(lib, inst, FP32)
    try:
        g.T[3, 4, 5] = float("nan")
        lib.aniso3_step(g.h, g.T, inst.dt, 1)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso3_sync(g.h)
        assert ei.value.code == lib.ANISO_ERR_NONFINITE
        g.T.copy_(torch.tensor(inst.T0, dtype=torch.float32, device="cuda"))
        g.step(1)  # the flag was cleared; a clean step reports nothing
    finally:
        g.close()


def test_zero_steps_leave_T_untouched(lib):
    import torch
    inst = _inst(8, 8, 8, 1, seed=21, nsteps=0)
    g = Grid3(lib, inst, FP32)
    try:
        before = g.T.clone()
        lib.aniso3_step(g.h, g.T, inst.dt, 0)
        lib.aniso3_sync(g.h)
        assert torch.equal(before, g.T)
    finally:
        g.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_constant_T_is_a_fixed_point(lib, prec):
    """Uniform T: every difference is zero, so every update returns T."""
    inst = _inst(16, 12, 8, 0, seed=22, nsteps=5)
    inst.T0 = np.full_like(inst.T0, 3.25)
    g = Grid3(lib, inst, prec)
    try:
        got = g.step(5)
    finally:
        g.close()
    assert np.max(np.abs(got - 3.25)) <= (1e-15 if prec == FP64 else 2e-6) * 3.25


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_axis_aligned_field_fp64(lib, axis):
    """b exactly along one axis: all transverse coefficients vanish and only
    that axis diffuses (degenerate case of the limiter terms)."""
    inst = _inst(12, 10, 8, 1, seed=23 + axis, nsteps=2)
    b = [np.zeros_like(inst.bx) for _ in range(3)]
    b[axis][:] = 1.0
    inst.bx, inst.by, inst.bz = b
    ref = oracle_run(inst, FP64, 2)
    g = Grid3(lib, inst, FP64)
    try:
        got = g.step(2)
    finally:
        g.close()
    assert rel_linf(got, ref) < 2 * FP64_TOL_PER_STEP


def test_isotropic_limit_fp64(lib):
    """chi_perp = chi_par: the tensor is chi I, the transverse terms vanish."""
    inst = _inst(16, 8, 12, 0, seed=24, nsteps=3, chi_perp=0.05)
    ref = oracle_run(inst, FP64, 3)
    g = Grid3(lib, inst, FP64)
    try:
        got = g.step(3)
    finally:
        g.close()
    assert rel_linf(got, ref) < 3 * FP64_TOL_PER_STEP


def test_stability_limit_on_the_gpu(lib):
    """The paper's 3-D stability limit of the 2-step scheme (chi dt / dx^2 <=
    8.25, Section 2.1) on the GPU: with the linear (arithmetic-mean) average,
    the worst mode of a 28 x 12 x 12 periodic grid grows by the closed-form
    factor at 8.3 and the L2 norm of a random state does not grow at 8.2."""
    import math
    from test_oracle3d_pins import _GRID, _grid_modes, _mode, _worst
    K = _grid_modes(_GRID)
    r_hi, b, idx = _worst(8.3, K)
    nz, ny, nx = _GRID
    T, _ = _mode(_GRID, (idx[0] + 1, idx[1] + 1, idx[2] + 1))
    ones = np.ones(_GRID)

    def run(T0, lam, steps):
        inst = W.Instance3("stability", nx, ny, nz, 1.0, 1.0, 1.0, 1, 1.0, 0.0, lam, steps,
                           b[0] * ones, b[1] * ones, b[2] * ones, T0)
        g = Grid3(lib, inst, FP64, limiter=1)
        try:
            return g.step(steps)
        finally:
            g.close()

    T1 = run(T, 8.3, 1)
    ratio = float(np.sum(T1 * T) / np.sum(T * T))
    assert r_hi > 1.0 + 1e-4
    assert abs(ratio) == pytest.approx(r_hi, rel=1e-10)
    rng = np.random.default_rng(5)
    U = rng.normal(size=_GRID)
    n0 = np.linalg.norm(U)
    U5 = run(U, 8.2, 5)
    assert np.linalg.norm(U5) <= n0 * (1 + 1e-12)
    assert math.isfinite(float(np.linalg.norm(U5)))


@pytest.mark.parametrize("shape", [(32, 28, 16), (64, 36, 44), (8, 12, 20)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_fp16_field_fp32(lib, shape, bc, scheme):
    """FP16 face coefficients (14 instead of 20 bytes per cell and update)
    against the oracle run on the same FP16-rounded coefficients."""
    inst = _inst(*shape, bc, seed=5 * sum(shape) + bc, nsteps=3)
    ref = oracle_run(inst, FP32, inst.nsteps, scheme=scheme, fp16=True)
    floor = rel_linf(oracle_run(inst, FP32, inst.nsteps, scheme=scheme, fp16=True, round_each_step=True), ref)
    g = Grid3(lib, inst, FP32, scheme=scheme, fp16=True)
    try:
        got = g.step(inst.nsteps)
    finally:
        g.close()
    assert rel_linf(got, ref) < max(FP32_TOL, 3.0 * floor)


def test_fp16_field_needs_fp32(lib):
    inst = _inst(8, 8, 8, 1, seed=1, nsteps=1)
    h = lib.aniso3_create(8, 8, 8, inst.dx, inst.dy, inst.dz, inst.chi_par, 0.0, 1)
    try:
        lib.aniso3_set_option(h, lib.ANISO_OPT_FIELD_FP16, 1)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso3_set_field(h, 0x1000, 0x1000, 0x1000)  # FP64 handle: refused before any access
        assert ei.value.code == lib.ANISO_ERR_ARG
    finally:
        lib.aniso3_destroy(h)
