"""GPU parity of the temperature-dependent diffusivity (Section 3.3: chi_par
times (max(T,0)/t_ref)^alpha, harmonic face average from each update's
input) against the oracle's step_nl: FP64 within 1e-12 relative per step,
FP32 within 1e-4 or 3x the problem's own FP32 noise floor.  Also: alpha = 0
is the constant-diffusivity path bit for bit, conservation, and the
combinations outside the supported path are refused."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import FP32_TOL, FP64_TOL_PER_STEP, GpuGrid, oracle_inputs, rel_linf

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1


def _inst(nx, ny, bc, seed, dt_factor=10.0):
    if bc == 1:
        return W.random_instance(nx, ny, seed=seed, dt_factor=dt_factor)
    return W.ring_instance(nx, ny=ny, dt_factor=dt_factor)


def _oracle(inst, T0, co, nsteps, alpha, t_ref, limiter=0, round32=False):
    if not round32:
        return O.step_nl(T0, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, alpha, t_ref=t_ref,
                         nsteps=nsteps, limiter=limiter)
    T = T0
    for _ in range(nsteps):
        T = O.step_nl(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, alpha, t_ref=t_ref,
                      limiter=limiter).astype(np.float32).astype(np.float64)
    return T


@pytest.mark.parametrize("nx,ny", [(64, 48), (96, 160), (544, 72), (1024, 64), (8, 12)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("alpha", [1.0, 2.5])
def test_nonlinear_fp64(lib, nx, ny, bc, alpha):
    inst = _inst(nx, ny, bc, seed=nx + ny)
    T0, co = oracle_inputs(lib, inst, FP64)
    t_ref = float(np.median(T0)) if bc == 0 else 1.0
    g = GpuGrid(lib, inst, FP64, fast=3)
    try:
        lib.aniso_set_nonlinear(g.h, alpha, t_ref)
        got = g.step(3)
    finally:
        g.close()
    ref = _oracle(inst, T0, co, 3, alpha, t_ref)
    assert rel_linf(got, ref) < 3 * FP64_TOL_PER_STEP


@pytest.mark.parametrize("limiter", [1, 2, 3])
def test_nonlinear_limiters_fp64(lib, limiter):
    inst = _inst(160, 96, 1, seed=3)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, limiter=limiter, fast=3)
    try:
        lib.aniso_set_nonlinear(g.h, 2.5, 1.0)
        got = g.step(2)
    finally:
        g.close()
    assert rel_linf(got, _oracle(inst, T0, co, 2, 2.5, 1.0, limiter=limiter)) < 2 * FP64_TOL_PER_STEP


@pytest.mark.parametrize("nx,ny", [(256, 128), (544, 96), (1024, 1024)])
def test_nonlinear_fp32(lib, nx, ny):
    inst = _inst(nx, ny, 1, seed=7 * nx)
    T0, co = oracle_inputs(lib, inst, FP32)
    g = GpuGrid(lib, inst, FP32, fast=3)
    try:
        lib.aniso_set_nonlinear(g.h, 2.5, 1.0)
        got = g.step(4)
    finally:
        g.close()
    ref = _oracle(inst, T0, co, 4, 2.5, 1.0)
    floor = rel_linf(_oracle(inst, T0, co, 4, 2.5, 1.0, round32=True), ref)
    assert rel_linf(got, ref) < max(FP32_TOL, 3.0 * floor)


def test_zero_exponent_is_the_constant_path_bit_for_bit(lib):
    inst = _inst(256, 96, 1, seed=9)
    a = GpuGrid(lib, inst, FP32, fast=3)
    b = GpuGrid(lib, inst, FP32, fast=3)
    try:
        lib.aniso_set_nonlinear(b.h, 2.5, 1.0)
        lib.aniso_set_nonlinear(b.h, 0.0, 1.0)
        assert np.array_equal(a.step(3), b.step(3))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_nonlinear_conservation_fp64(lib, bc):
    inst = _inst(128, 96, bc, seed=11)
    g = GpuGrid(lib, inst, FP64, fast=3)
    try:
        lib.aniso_set_nonlinear(g.h, 2.5, 1.0)
        s0 = lib.aniso_total(g.h, g.T)[0]
        g.step(5)
        s1 = lib.aniso_total(g.h, g.T)[0]
    finally:
        g.close()
    assert abs(s1 - s0) <= 1e-12 * abs(s0)


def test_unsupported_combinations_are_refused(lib):
    import torch
    inst = _inst(64, 48, 1, seed=12)
    g = GpuGrid(lib, inst, FP32, fast=3)
    try:
        lib.aniso_set_nonlinear(g.h, 2.5, 1.0)
        for key, val in ((lib.ANISO_OPT_SCHEME, lib.ANISO_SCHEME_4STEP), (lib.ANISO_OPT_ORDER, lib.ANISO_ORDER_YX),
                         (lib.ANISO_OPT_FAST_PATH, 1)):
            lib.aniso_set_option(g.h, key, val)
            with pytest.raises(lib.AnisoError) as ei:
                lib.aniso_step(g.h, g.T, inst.dt, 1)
            assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
            lib.aniso_set_option(g.h, key, {lib.ANISO_OPT_SCHEME: 0, lib.ANISO_OPT_ORDER: 0,
                                            lib.ANISO_OPT_FAST_PATH: 3}[key])
        out = torch.empty_like(g.T)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_sweep(g.h, lib.ANISO_DIR_X, g.T, out, inst.dt)
        assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_batch_create([g.h])
        assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
        g.step(1)  # the supported path still runs
    finally:
        g.close()
    odd = _inst(50, 48, 1, seed=13)  # 50 cells: not a multiple of the FP32 vector
    g = GpuGrid(lib, odd, FP32)
    try:
        lib.aniso_set_nonlinear(g.h, 2.5, 1.0)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_step(g.h, g.T, odd.dt, 1)
        assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
    finally:
        g.close()
