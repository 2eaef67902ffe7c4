"""The long-line kernel (line6): lines of 2048 < n <= 4096 cells in FP32, a
line's team spread over several warps (shuffles inside a warp, shared memory
across warps, PCR of the segment ends in shared memory).  Single grids take
it for the x-then-y fast step whenever a line is above line4's limit and the
cluster kernel does not take it (lines that are not a multiple of 1024 cells,
or ANISO_OPT_CLUSTER_LINES = 1, which these tests set).
Checked against the FP64 oracle, against the general kernels, with FP16
face coefficients, on zero-flux boundaries and inside a batch."""
import numpy as np
import pytest

import workloads as W
from gpu_util import GpuGrid, fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP32 = 1


def _l6(lib, g):
    """Lines of 2049-4096 cells on the long-line kernel."""
    lib.aniso_set_option(g.h, lib.ANISO_OPT_CLUSTER_LINES, 1)
    return g
SAME_KERNELS_TOL = 2e-5  # FP32, different kernels (segment cuts, limiter forms)

SHAPES = [(4096, 256, 1), (256, 4096, 1), (2560, 3072, 1), (4096, 64, 0), (2080, 96, 0), (3000, 200, 1)]


def _inst(nx, ny, bc, seed=11, nsteps=4):
    inst = W.random_instance(nx, ny, seed=seed, chi_par=0.05, dt_factor=60.0, nsteps=nsteps)
    inst.bc = bc
    return inst


@pytest.mark.parametrize("nx,ny,bc", SHAPES)
def test_long_lines_against_the_oracle(lib, nx, ny, bc):
    inst = _inst(nx, ny, bc)
    g = _l6(lib, GpuGrid(lib, inst, FP32, fast=3))
    try:
        got = g.step(4)
    finally:
        g.close()
    T0, co = oracle_inputs(lib, inst, FP32)
    ref = oracle_step(inst, T0, co, 4)
    assert np.isfinite(got).all()
    assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 4, ref)


@pytest.mark.parametrize("nx,ny,bc", SHAPES[:4])
@pytest.mark.parametrize("fp16", [False, True])
def test_long_lines_match_the_general_kernels(lib, nx, ny, bc, fp16):
    inst = _inst(nx, ny, bc, seed=23)
    a = _l6(lib, GpuGrid(lib, inst, FP32, fp16=fp16, fast=3))
    b = GpuGrid(lib, inst, FP32, fp16=fp16, fast=0)
    try:
        assert rel_linf(a.step(3), b.step(3)) < SAME_KERNELS_TOL
    finally:
        a.close()
        b.close()


def test_long_lines_in_a_batch_match_single_grids(lib):
    """A batch mixing long-line grids with line4 grids equals the same grids
    stepped one by one (same kernels, same shapes: bit for bit)."""
    import torch
    insts = [_inst(4096, 128, 1, seed=31), _inst(512, 256, 1, seed=32), _inst(128, 2304, 0, seed=33)]
    grids = [_l6(lib, GpuGrid(lib, i, FP32, fast=3)) for i in insts]
    singles = [_l6(lib, GpuGrid(lib, i, FP32, fast=3)) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        try:
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [3, 3, 3])
            lib.aniso_sync(grids[0].h)
        finally:
            lib.aniso_batch_destroy(b)
        for g, s in zip(grids, singles):
            s.step(3)
            assert torch.equal(g.T, s.T)
    finally:
        for g in grids + singles:
            g.close()
