"""The 4-step scheme (Eq. 4step) on the GPU against the oracle's step4."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import FP64_TOL_PER_STEP, GpuGrid, oracle_inputs, rel_linf

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1


def _inst(nx, ny, bc, seed):
    if bc == 1:
        return W.random_instance(nx, ny, seed=seed, dt_factor=300.0)
    return W.ring_instance(nx, ny=ny, dt_factor=300.0)


def _four(lib, g):
    lib.aniso_set_option(g.h, lib.ANISO_OPT_SCHEME, lib.ANISO_SCHEME_4STEP)


@pytest.mark.parametrize("nx,ny", [(33, 17), (64, 96), (256, 128), (96, 1100), (544, 40)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_four_step_fp64_matches_oracle(lib, nx, ny, bc, order):
    inst = _inst(nx, ny, bc, seed=nx + ny)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, order=order)
    try:
        _four(lib, g)
        got = g.step(3)
        ref = O.step4(T0, co, bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3, order=order)
        assert rel_linf(got, ref) < 3 * 2 * FP64_TOL_PER_STEP
    finally:
        g.close()


@pytest.mark.parametrize("limiter", [0, 1, 2, 3])
def test_four_step_limiters_fp64(lib, limiter):
    inst = W.random_instance(128, 96, seed=4, dt_factor=1000.0)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, limiter=limiter)
    try:
        _four(lib, g)
        ref = O.step4(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=2, limiter=limiter)
        assert rel_linf(g.step(2), ref) < 4 * FP64_TOL_PER_STEP
    finally:
        g.close()


def test_four_step_fp32_and_graph(lib):
    """FP32 within 1e-4 of the oracle on a square grid; graph replay equals
    direct launches bit for bit; the sum is conserved in FP64 to rounding."""
    inst = W.random_instance(256, 256, seed=8, chi_par=0.05, dt_factor=100.0)
    T0, co = oracle_inputs(lib, inst, FP32)
    a = GpuGrid(lib, inst, FP32, graph=True)
    b = GpuGrid(lib, inst, FP32, graph=False)
    try:
        _four(lib, a)
        _four(lib, b)
        ga, gb = a.step(10), b.step(10)
        np.testing.assert_array_equal(ga, gb)
        ref = O.step4(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=10)
        assert rel_linf(ga, ref) < 1e-4
    finally:
        a.close()
        b.close()


def test_four_step_differs_from_two_step(lib):
    inst = W.random_instance(64, 64, seed=9, dt_factor=1000.0)
    a = GpuGrid(lib, inst, FP64)
    b = GpuGrid(lib, inst, FP64)
    try:
        _four(lib, a)
        assert rel_linf(a.step(2), b.step(2)) > 1e-6
    finally:
        a.close()
        b.close()


def test_four_step_option_rules(lib):
    inst = W.random_instance(32, 32, seed=1)
    g = GpuGrid(lib, inst, FP32)
    try:
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_set_option(g.h, lib.ANISO_OPT_SCHEME, 2)
        assert ei.value.code == lib.ANISO_ERR_ARG
        _four(lib, g)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_batch_create([g.h])
        assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
    finally:
        g.close()
    h = lib.aniso_create(32, 32, inst.dx, inst.dy, inst.chi_par, 0.0, 1)
    try:
        lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, FP32)
        lib.aniso_set_option(h, lib.ANISO_OPT_KAHAN, 1)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_set_option(h, lib.ANISO_OPT_SCHEME, lib.ANISO_SCHEME_4STEP)
        assert ei.value.code == lib.ANISO_ERR_UNSUPPORTED
    finally:
        lib.aniso_destroy(h)
