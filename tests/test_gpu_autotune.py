"""Block-shape autotuner of the batched fast path (rows per block and PCR
depth chosen by measurement)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import FP64_TOL_PER_STEP, GpuGrid, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP64, FP32 = 0, 1


def _shape_options(lib, g, choice):
    fast, warps, seg = lib.aniso_autotune_candidate(choice)
    lib.aniso_set_option(g.h, lib.ANISO_OPT_FAST_PATH, fast)
    lib.aniso_set_option(g.h, lib.ANISO_OPT_BLOCK_WARPS, warps)
    lib.aniso_set_option(g.h, lib.ANISO_OPT_SEGMENT, seg)


def test_autotune_keeps_inputs_and_batch_matches_singles(lib):
    """The tuner leaves T and the step counters alone; afterwards the batch
    reproduces single-grid steps with the chosen shape bit for bit."""
    import torch
    insts = W.batch_instances(12, nsteps=3, size_cap=1024)
    grids = [GpuGrid(lib, i, FP32) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        before = [g.T.clone() for g in grids]
        choice, ms = lib.aniso_batch_autotune(b, [g.T for g in grids], [i.dt for i in insts], nsteps=2, reps=2)
        torch.cuda.synchronize()
        assert 0 <= choice and ms > 0.0
        for g, t0 in zip(grids, before):
            assert torch.equal(g.T, t0)
            assert lib.aniso_get_state(g.h) == 0
        singles = []
        for inst in insts:
            s = GpuGrid(lib, inst, FP32)
            _shape_options(lib, s, choice)
            singles.append(s)
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [3] * len(insts))
        torch.cuda.synchronize()
        for g, s in zip(grids, singles):
            np.testing.assert_array_equal(g.T.cpu().numpy(), s.step(3).astype(np.float32))
        for s in singles:
            s.close()
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def test_autotuned_fp64_batch_matches_oracle(lib):
    import torch
    insts = W.batch_instances(5, nsteps=2, size_cap=512)
    grids = [GpuGrid(lib, i, FP64) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        choice, _ = lib.aniso_batch_autotune(b, [g.T for g in grids], [i.dt for i in insts], nsteps=1, reps=1)
        assert choice >= 0
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [2] * len(insts))
        torch.cuda.synchronize()
        for g, inst in zip(grids, insts):
            T0, co = oracle_inputs(lib, inst, FP64)
            assert rel_linf(g.T.cpu().numpy(), oracle_step(inst, T0, co, 2)) < 2 * FP64_TOL_PER_STEP
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def test_autotune_without_fast_path_changes_nothing(lib):
    """Grids in the y-then-x order never take the fast path: nothing to tune."""
    insts = W.batch_instances(3, nsteps=2, size_cap=256)
    grids = []
    for inst in insts:
        g = GpuGrid(lib, inst, FP32, fast=1)
        grids.append(g)
    try:
        for g in grids:
            lib.aniso_set_option(g.h, lib.ANISO_OPT_ORDER, lib.ANISO_ORDER_YX)
        b = lib.aniso_batch_create([g.h for g in grids])
        assert lib.aniso_batch_autotune(b, [g.T for g in grids], [i.dt for i in insts]) == (-1, 0.0)
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def test_block_warps_option_rules(lib):
    inst = W.random_instance(64, 64, seed=2)
    g = GpuGrid(lib, inst, FP32)
    try:
        for v in (0, 1, 2, 4, 8):
            lib.aniso_set_option(g.h, lib.ANISO_OPT_BLOCK_WARPS, v)
        for v in (3, 16, -1):
            with pytest.raises(lib.AnisoError) as ei:
                lib.aniso_set_option(g.h, lib.ANISO_OPT_BLOCK_WARPS, v)
            assert ei.value.code == lib.ANISO_ERR_ARG
    finally:
        g.close()


@pytest.mark.parametrize("warps", [1, 2, 4, 8])
@pytest.mark.parametrize("seg", [2, 4, 8])
def test_line4_block_shapes_fp64(lib, warps, seg):
    """Every block shape the tuner may pick computes the same step."""
    inst = W.random_instance(544, 96, seed=11, dt_factor=200.0)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, fast=3)
    try:
        lib.aniso_set_option(g.h, lib.ANISO_OPT_BLOCK_WARPS, warps)
        lib.aniso_set_option(g.h, lib.ANISO_OPT_SEGMENT, seg)
        assert rel_linf(g.step(2), oracle_step(inst, T0, co, 2)) < 2 * FP64_TOL_PER_STEP
    finally:
        g.close()
