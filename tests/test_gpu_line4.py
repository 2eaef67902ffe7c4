"""The warp-per-line kernel (fast-path option 3) against the FP64 oracle:
line lengths that give uneven segments, one-lane and sub-warp teams,
every limiter, both boundary conditions, FP32 and FP16 fields, batches."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import FP64_TOL_PER_STEP, GpuGrid, fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1
LINE4 = 3

# (nx, ny): 544 -> 34 lanes' worth of chunks on 32 lanes (uneven segments);
# 8 and 12 -> one-lane teams; 96/160 -> sub-warp teams; 2048 -> 16 chunks a lane
SHAPES = [(544, 72), (96, 160), (8, 12), (1024, 1024), (2048, 36), (36, 2048), (64, 64), (200, 136)]


def _inst(nx, ny, bc, seed):
    if bc == 1:
        return W.random_instance(nx, ny, seed=seed, dt_factor=300.0)
    return W.ring_instance(nx, ny=ny, dt_factor=300.0)


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("bc", [0, 1])
def test_line4_steps_fp64(lib, nx, ny, bc):
    inst = _inst(nx, ny, bc, seed=nx + 3 * ny)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, fast=LINE4)
    try:
        got = g.step(3)
        ref = oracle_step(inst, T0, co, 3)
        assert rel_linf(got, ref) < 3 * FP64_TOL_PER_STEP
    finally:
        g.close()


@pytest.mark.parametrize("limiter", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [FP64, FP32])
def test_line4_limiters(lib, limiter, prec):
    inst = W.random_instance(544, 96, seed=5, chi_par=0.5, dt_factor=500.0)
    T0, co = oracle_inputs(lib, inst, prec)
    g = GpuGrid(lib, inst, prec, limiter=limiter, fast=LINE4)
    try:
        got = g.step(4)
        ref = oracle_step(inst, T0, co, 4, limiter=limiter)
        tol = 4 * FP64_TOL_PER_STEP if prec == FP64 else fp32_tol(inst, T0, co, 4, ref)
        assert rel_linf(got, ref) < tol
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (544, 72), (160, 96)])
@pytest.mark.parametrize("fp16", [False, True])
def test_line4_fp32_matches_oracle(lib, nx, ny, fp16):
    inst = W.random_instance(nx, ny, seed=17, chi_par=0.05, dt_factor=100.0)
    T0, co = oracle_inputs(lib, inst, FP32, fp16=fp16)
    g = GpuGrid(lib, inst, FP32, fp16=fp16, fast=LINE4)
    try:
        got = g.step(20)
        ref = oracle_step(inst, T0, co, 20)
        assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 20, ref)
    finally:
        g.close()


@pytest.mark.parametrize("bc", [0, 1])
def test_line4_single_x_sweep_natural_layout(lib, bc):
    """aniso_sweep in x writes T* row-major through the same kernel."""
    inst = _inst(544, 40, bc, seed=2)
    T0, co = oracle_inputs(lib, inst, FP64)
    lamx, _, mu = O.lambdas(inst.dt, inst.dx, inst.dy, inst.chi_par)
    g = GpuGrid(lib, inst, FP64, fast=LINE4)
    try:
        assert rel_linf(g.sweep(lib.ANISO_DIR_X, T0), O.xsweep(T0, co, bc, lamx, mu)) < FP64_TOL_PER_STEP
    finally:
        g.close()


def test_line4_batched_fp64_matches_oracle(lib):
    """A batch of uneven grids on the warp-per-line kernel: every grid against
    the oracle."""
    import torch
    insts = W.batch_instances(6, nsteps=3, size_cap=512)
    grids = [GpuGrid(lib, i, FP64, fast=LINE4) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [3] * len(insts))
        torch.cuda.synchronize()
        for g, inst in zip(grids, insts):
            T0, co = oracle_inputs(lib, inst, FP64)
            assert rel_linf(g.T.cpu().numpy(), oracle_step(inst, T0, co, 3)) < 3 * FP64_TOL_PER_STEP
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_line4_occupancy_split_batch(lib, prec):
    """Line lengths from 64 to 1024 need very different shared memory, so the
    plan splits each sweep into several concurrent launches (one per
    occupancy class).  The kernel count says so, and every grid still matches
    the oracle (FP64) or its own single-grid run bit for bit (FP32).  (The
    shared-memory form: with part of the FP32 line state in tensor memory
    these lines all fit the register-bound class.)"""
    import torch
    shapes = [(1024, 96), (64, 1024), (512, 128), (800, 160), (256, 64), (992, 32), (128, 256)]
    insts = [W.random_instance(nx, ny, seed=31 + k, chi_par=0.05, dt_factor=100.0)
             for k, (nx, ny) in enumerate(shapes)]
    grids = [GpuGrid(lib, i, prec, fast=LINE4) for i in insts]
    singles = [GpuGrid(lib, i, prec, fast=LINE4, graph=False) for i in insts]
    lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_TMEM, 0)
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        assert lib.aniso_batch_kernel_count(b) == 0
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [2] * len(insts))
        torch.cuda.synchronize()
        kernels = lib.aniso_batch_kernel_count(b)
        assert 2 * 2 < kernels <= 2 * 2 * 5  # more than one launch per sweep, at most five
        for g, s, inst in zip(grids, singles, insts):
            got = g.T.double().cpu().numpy()
            if prec == FP64:
                T0, co = oracle_inputs(lib, inst, FP64)
                assert rel_linf(got, oracle_step(inst, T0, co, 2)) < 2 * FP64_TOL_PER_STEP
            else:
                assert np.array_equal(got, s.step(2))
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids + singles:
            g.close()


def test_line4_nonfinite_flag(lib):
    inst = W.random_instance(256, 128, seed=9)
    T0 = inst.T0.copy()
    T0[50, 60] = np.nan
    g = GpuGrid(lib, inst, FP32, fast=LINE4, T0=T0)
    try:
        lib.aniso_step(g.h, g.T, inst.dt, 1)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_sync(g.h)
        assert ei.value.code == lib.ANISO_ERR_NONFINITE
    finally:
        g.close()
