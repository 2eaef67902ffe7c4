"""The TMA-staged line kernel (line5) that batched calls use for lines of
768 to 1024 cells: the same line systems as the warp-per-line kernel, with
each block's rows brought into shared memory by tensor-map tile loads.
Checked against the warp-per-line kernel (same segment cuts, same
arithmetic), against the FP64 oracle, on partial tiles and zero-flux
boundaries, and on its failure path (a bounded wait that gives up)."""
import numpy as np
import pytest

import workloads as W
from gpu_util import GpuGrid, fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP32 = 1


def _run_batch(lib, insts, nsteps, tma, limiter=0):
    grids = [GpuGrid(lib, i, FP32, fast=3, limiter=limiter) for i in insts]
    try:
        lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_TMA_LINES, tma)
        b = lib.aniso_batch_create([g.h for g in grids])
        try:
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [nsteps] * len(insts))
            lib.aniso_sync(grids[0].h)
            return [g.T.double().cpu().numpy() for g in grids]
        finally:
            lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def _insts():
    shapes = [(1024, 768), (768, 1024), (992, 96), (1024, 36), (800, 832), (512, 1024)]
    out = []
    for k, (nx, ny) in enumerate(shapes):
        inst = W.random_instance(nx, ny, seed=300 + k, chi_par=0.02, dt_factor=30.0 * (k + 1), nsteps=3)
        if k in (1, 4):
            inst.bc = 0  # zero-flux: mirrored neighbour lines at the grid's edges
        out.append(inst)
    return out


@pytest.mark.parametrize("limiter", [0, 3])
def test_tma_lines_match_the_warp_kernel(lib, limiter):
    insts = _insts()
    a = _run_batch(lib, insts, 3, tma=1, limiter=limiter)
    b = _run_batch(lib, insts, 3, tma=0, limiter=limiter)
    for x, y in zip(a, b):
        assert np.isfinite(x).all()
        assert rel_linf(x, y) < 1e-6


def test_tma_lines_against_the_oracle(lib):
    insts = _insts()
    got = _run_batch(lib, insts, 3, tma=1)
    for inst, g in zip(insts, got):
        T0, co = oracle_inputs(lib, inst, FP32)
        ref = oracle_step(inst, T0, co, 3)
        assert rel_linf(g, ref) < fp32_tol(inst, T0, co, 3, ref)


def test_tma_wait_gives_up_and_reports_timeout(lib):
    """With the testing value 2 the kernel issues no loads: every block's
    bounded wait runs out, the call reports ANISO_ERR_TIMEOUT, and the
    handles work again afterwards."""
    inst = W.random_instance(1024, 64, seed=5, nsteps=1)
    grids = [GpuGrid(lib, inst, FP32, fast=3)]
    try:
        lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_TMA_LINES, 2)
        b = lib.aniso_batch_create([g.h for g in grids])
        try:
            lib.aniso_step_batched(b, [g.T for g in grids], [inst.dt], [1])
            with pytest.raises(lib.AnisoError) as ei:
                lib.aniso_sync(grids[0].h)
            assert ei.value.code == lib.ANISO_ERR_TIMEOUT
            # the flag is cleared; the normal kernel runs again on the same handles
            lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_TMA_LINES, 1)
            T0, co = oracle_inputs(lib, inst, FP32)
            grids[0].T.copy_(__import__("torch").tensor(inst.T0, dtype=grids[0].T.dtype, device="cuda"))
            lib.aniso_step_batched(b, [g.T for g in grids], [inst.dt], [1])
            lib.aniso_sync(grids[0].h)
            got = grids[0].T.double().cpu().numpy()
            assert rel_linf(got, oracle_step(inst, T0, co, 1)) < 1e-5
        finally:
            lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()
