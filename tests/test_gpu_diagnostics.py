"""Per-step diagnostics of batched calls (ANISO_OPT_DIAGNOSTICS): the FP64
sum, minimum and maximum of every grid's T after every step, formed inside
the y-update kernel and read once per call.  Checked against the GPU's own
state (host FP64 reduction of the same values) and against the FP64 oracle
stepped one step at a time."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import GpuGrid, oracle_inputs

pytestmark = pytest.mark.gpu
FP32 = 1


def _batch(lib, insts, diag=True):
    grids = [GpuGrid(lib, i, FP32, fast=3) for i in insts]
    lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_DIAGNOSTICS, int(diag))
    b = lib.aniso_batch_create([g.h for g in grids])
    return grids, b


def _insts():
    shapes = [(64, 96), (256, 128), (1024, 64), (96, 1024), (544, 320), (128, 128)]
    return [W.random_instance(nx, ny, seed=100 + k, chi_par=0.01 * (k + 1), dt_factor=50.0 * (k + 1), nsteps=4)
            for k, (nx, ny) in enumerate(shapes)]


def test_diagnostics_match_the_state_after_every_call(lib):
    """One step per call: the ring equals the FP64 sum / min / max of the
    grid's FP32 state that the call leaves behind."""
    insts = _insts()
    grids, b = _batch(lib, insts)
    try:
        for call in range(3):
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [1] * len(insts))
            ring = lib.aniso_batch_diagnostics(b, len(insts))
            assert ring.shape == (len(insts), 1, 3)
            for k, g in enumerate(grids):
                t = g.T.double().cpu().numpy()
                s, mn, mx = ring[k, 0]
                assert s == pytest.approx(t.sum(), rel=1e-8)
                assert mn == t.min() and mx == t.max()
    finally:
        lib.aniso_batch_destroy(b)
        for g in grids:
            g.close()


def test_diagnostics_follow_the_oracle_step_by_step(lib):
    """A 4-step call: every step's sum, min and max against the FP64 oracle
    on the same FP32-rounded inputs, stepped one step at a time; the sum is
    conserved (periodic grids) to FP32 rounding."""
    insts = _insts()
    grids, b = _batch(lib, insts)
    try:
        nst = [4, 4, 3, 4, 2, 4]  # uneven: missing steps read as NaN
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], nst)
        ring = lib.aniso_batch_diagnostics(b, len(insts))
        assert ring.shape == (len(insts), 4, 3)
        for k, inst in enumerate(insts):
            T, co = oracle_inputs(lib, inst, FP32)
            s0 = T.sum()
            for s in range(4):
                if s >= nst[k]:
                    assert np.isnan(ring[k, s]).all()
                    continue
                T = O.step(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1)
                got_s, got_mn, got_mx = ring[k, s]
                assert got_s == pytest.approx(T.sum(), rel=1e-6)
                assert abs(got_s - s0) / abs(s0) < 1e-6  # conservation of the FP32 state
                scale = np.abs(T).max()
                assert abs(got_mn - T.min()) < 1e-4 * scale
                assert abs(got_mx - T.max()) < 1e-4 * scale
    finally:
        lib.aniso_batch_destroy(b)
        for g in grids:
            g.close()


def test_diagnostics_leave_the_state_unchanged(lib):
    """The recorded call and an unrecorded one give the same T bit for bit."""
    import torch
    insts = _insts()
    ga, ba = _batch(lib, insts, diag=True)
    gb, bb = _batch(lib, insts, diag=False)
    try:
        lib.aniso_step_batched(ba, [g.T for g in ga], [i.dt for i in insts], [3] * len(insts))
        lib.aniso_step_batched(bb, [g.T for g in gb], [i.dt for i in insts], [3] * len(insts))
        torch.cuda.synchronize()
        for a, c in zip(ga, gb):
            assert torch.equal(a.T, c.T)
        with pytest.raises(lib.AnisoError):
            lib.aniso_batch_diagnostics(bb, len(insts))
    finally:
        for b_, gs in ((ba, ga), (bb, gb)):
            lib.aniso_batch_destroy(b_)
            for g in gs:
                g.close()


def test_diagnostics_are_nan_where_the_y_update_is_not_the_warp_per_line_kernel(lib):
    """A grid with columns above 2048 cells (long-line kernel) and one on the
    cluster kernel (rows of 8192) record no diagnostics: their slots are NaN,
    while the warp-per-line grids beside them in the batch record every step."""
    shapes = [(256, 128), (64, 3000), (8192, 64), (96, 1024)]
    insts = [W.random_instance(nx, ny, seed=300 + k, chi_par=0.05, dt_factor=40.0, nsteps=2)
             for k, (nx, ny) in enumerate(shapes)]
    grids, b = _batch(lib, insts)
    try:
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [2] * len(insts))
        ring = lib.aniso_batch_diagnostics(b, len(insts))
        assert ring.shape == (len(insts), 2, 3)
        for k in (0, 3):
            assert np.isfinite(ring[k]).all()
        for k in (1, 2):
            assert np.isnan(ring[k]).all()
    finally:
        lib.aniso_batch_destroy(b)
        for g in grids:
            g.close()
