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
            lib.aniso_set_option(g.h, lib.ANISO_OPT_SCHEME, 3)
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


# ------------------------------------------------------- explicit scheme

def _explicit(lib, g):
    lib.aniso_set_option(g.h, lib.ANISO_OPT_SCHEME, lib.ANISO_SCHEME_EXPLICIT)


@pytest.mark.parametrize("nx,ny", [(5, 7), (33, 17), (64, 96), (256, 128), (96, 1100), (40, 3)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nsteps", [1, 4])
def test_explicit_fp64_matches_oracle(lib, nx, ny, bc, nsteps):
    inst = W.random_instance(nx, ny, seed=nx * 3 + ny, dt_factor=0.45) if bc == 1 else \
        W.ring_instance(nx, ny=ny, dt_factor=0.45)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64)
    try:
        _explicit(lib, g)
        got = g.step(nsteps)
        ref = O.explicit_step(T0, co, bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=nsteps)
        assert rel_linf(got, ref) < nsteps * FP64_TOL_PER_STEP
    finally:
        g.close()


@pytest.mark.parametrize("limiter", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_explicit_limiters(lib, limiter, prec):
    inst = W.random_instance(160, 96, seed=6, dt_factor=0.4)
    T0, co = oracle_inputs(lib, inst, prec)
    g = GpuGrid(lib, inst, prec, limiter=limiter)
    try:
        _explicit(lib, g)
        ref = O.explicit_step(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=3, limiter=limiter)
        tol = 3 * FP64_TOL_PER_STEP if prec == FP64 else 1e-5
        assert rel_linf(g.step(3), ref) < tol
    finally:
        g.close()


def test_explicit_fp16_field_and_graph(lib):
    inst = W.random_instance(128, 128, seed=12, dt_factor=0.45)
    T0, co = oracle_inputs(lib, inst, FP32, fp16=True)
    a = GpuGrid(lib, inst, FP32, fp16=True, graph=True)
    b = GpuGrid(lib, inst, FP32, fp16=True, graph=False)
    try:
        _explicit(lib, a)
        _explicit(lib, b)
        ga, gb = a.step(7), b.step(7)
        np.testing.assert_array_equal(ga, gb)
        ref = O.explicit_step(T0, co, 1, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=7)
        assert rel_linf(ga, ref) < 1e-5
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_explicit_ring_minimum_matches_paper(lib, prec):
    """Section 3.1 (caption of the minimum-temperature figure): the unlimited
    explicit method at ncfl = 1 reaches min T = -0.41 on the 512^2 ring; with
    the van Leer limiter T stays within its initial bounds."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ring_explicit_paper_values.json")))
    inst = W.ring_instance(gold["n"], t_hot=gold["T_hot"], t_cold=gold["T_cold"], chi_par=gold["chi_par"],
                           dt_factor=1.0)
    dt = gold["ncfl"] * inst.dx ** 2 / (4 * gold["chi_par"])
    for limiter, check in ((1, "arith"), (0, "vanleer")):
        g = GpuGrid(lib, inst, prec, limiter=limiter)
        try:
            _explicit(lib, g)
            lo = np.inf
            for _ in range(gold["steps_checked"] // 50):
                lib.aniso_step(g.h, g.T, dt, 50)
                lo = min(lo, lib.aniso_total(g.h, g.T)[1])
            if check == "arith":
                assert abs(lo - gold["min_T_without_limiter"]) < gold["min_T_tolerance"]
            else:
                assert lo >= gold["T_cold"] * (1 - 1e-6)
        finally:
            g.close()
