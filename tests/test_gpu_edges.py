"""Degenerate and boundary requests on the GPU path: zero steps (single grid
and batch) leave T untouched, a batch whose grids have different step counts
advances each grid by its own count, and a uniform T is a fixed point."""
import numpy as np
import pytest

import workloads as W
from gpu_util import GpuGrid

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1


def test_zero_steps_single_and_batch(lib):
    import torch
    insts = [W.random_instance(64, 96, seed=1), W.random_instance(128, 64, seed=2)]
    grids = [GpuGrid(lib, i, FP32, fast=3) for i in insts]
    try:
        before = [g.T.clone() for g in grids]
        lib.aniso_step(grids[0].h, grids[0].T, insts[0].dt, 0)
        lib.aniso_sync(grids[0].h)
        assert torch.equal(before[0], grids[0].T)
        b = lib.aniso_batch_create([g.h for g in grids])
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [0, 0])
        torch.cuda.synchronize()
        for x, g in zip(before, grids):
            assert torch.equal(x, g.T)
        assert lib.aniso_batch_kernel_count(b) == 0
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def test_batch_with_uneven_step_counts_matches_singles(lib):
    import torch
    insts = [W.random_instance(96, 64, seed=3), W.random_instance(64, 128, seed=4),
             W.random_instance(160, 96, seed=5)]
    counts = [3, 0, 5]
    grids = [GpuGrid(lib, i, FP32, fast=3) for i in insts]
    singles = [GpuGrid(lib, i, FP32, fast=3, graph=False) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], counts)
        torch.cuda.synchronize()
        for g, s, k, inst in zip(grids, singles, counts, insts):
            got = g.T.double().cpu().numpy()
            want = s.step(k) if k else inst.T0.astype(np.float32).astype(np.float64)
            assert np.array_equal(got, want)
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids + singles:
            g.close()


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("fast", [3, 0])
def test_uniform_temperature_is_a_fixed_point(lib, prec, fast):
    inst = W.random_instance(96, 80, seed=6, dt_factor=1000.0)
    T0 = np.full((inst.ny, inst.nx), 1.75)
    g = GpuGrid(lib, inst, prec, fast=fast, T0=T0)
    try:
        got = g.step(4)
    finally:
        g.close()
    assert np.array_equal(got, T0)
