"""The warp-per-line kernel's tensor-memory form (ANISO_OPT_TMEM): each lane's
gamma (the segment-end coupling of its eliminated rows) is kept in the lane's
own TMEM lane instead of shared memory.  The arithmetic is the same, so
batches with and without it must agree bit for bit; and against the oracle."""
import numpy as np
import pytest

import workloads as W
from gpu_util import GpuGrid, fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP32 = 1


def _run(lib, insts, nsteps, tmem, fp16=False, limiter=0):
    import torch
    grids = [GpuGrid(lib, i, FP32, fp16=fp16, fast=3, limiter=limiter) for i in insts]
    try:
        lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_TMEM, tmem)
        b = lib.aniso_batch_create([g.h for g in grids])
        try:
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [nsteps] * len(insts))
            lib.aniso_sync(grids[0].h)
            torch.cuda.synchronize()
            return [g.T.clone() for g in grids]
        finally:
            lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def _insts(seed0=500):
    shapes = [(1024, 96), (64, 1024), (544, 320), (96, 64), (992, 736), (256, 256), (36, 800)]
    out = []
    for k, (nx, ny) in enumerate(shapes):
        inst = W.random_instance(nx, ny, seed=seed0 + k, chi_par=0.03, dt_factor=40.0 * (k + 1), nsteps=3)
        if k % 3 == 2:
            inst.bc = 0
        out.append(inst)
    return out


@pytest.mark.parametrize("fp16,limiter", [(False, 0), (True, 0), (False, 3)])
def test_tmem_form_is_bit_identical(lib, fp16, limiter):
    import torch
    insts = _insts()
    a = _run(lib, insts, 3, 1, fp16, limiter)
    b = _run(lib, insts, 3, 0, fp16, limiter)
    for x, y in zip(a, b):
        assert torch.isfinite(x).all()
        assert torch.equal(x, y)


def test_tmem_form_against_the_oracle(lib):
    insts = _insts(seed0=600)
    got = _run(lib, insts, 3, 1)
    for inst, g in zip(insts, got):
        T0, co = oracle_inputs(lib, inst, FP32)
        ref = oracle_step(inst, T0, co, 3)
        assert rel_linf(g.double().cpu().numpy(), ref) < fp32_tol(inst, T0, co, 3, ref)


def test_lines_too_long_for_tmem_fall_back(lib):
    """2048-cell lines need 16 chunks a lane: their sweep keeps gamma in shared
    memory, with the same results."""
    import torch
    insts = [W.random_instance(2048, 128, seed=41, nsteps=2), W.random_instance(128, 2048, seed=42, nsteps=2)]
    a = _run(lib, insts, 2, 1)
    b = _run(lib, insts, 2, 0)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
