"""The cluster line kernel (line7): lines of n = CS * np cells (np = 2048 or
1024, CS = 1, 2, 4 or 8 blocks of one thread-block cluster), each block
holding a piece of four lines; the segment-end system is solved per warp
against two interface unknowns, whose cyclic system (2 CS unknowns a line)
every block solves after one exchange through distributed shared memory.
It takes the plain FP32 state on lines of 4096, 8192 and 16384 cells
(ANISO_OPT_CLUSTER_LINES = 2, the default; 1 leaves 4096-cell lines to the
long-line kernel), and the compensated state (hi + lo) in both directions.
Checked against the FP64 oracle (also on the full 4096^2 and 16384^2
configurations in the benchmark's launch configuration), against the
general kernels, for conservation, on zero-flux boundaries, with FP16 face
coefficients and inside a batch."""
import numpy as np
import pytest

import workloads as W
from gpu_util import GpuGrid, fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
FP32 = 1
SAME_KERNELS_TOL = 2e-5  # FP32, different kernels (segment cuts, reduced-system solves)


def _inst(nx, ny, bc, seed=11, chi_par=0.05, dt_factor=60.0):
    inst = W.random_instance(nx, ny, seed=seed, chi_par=chi_par, dt_factor=dt_factor, nsteps=4)
    inst.bc = bc
    return inst


# (nx, ny, bc): x-lines of 16384 (8 blocks a cluster) and 8192 (4), and the
# same as y-lines of the column-major intermediate; zero-flux and periodic
PLAIN = [(16384, 64, 1), (8192, 96, 0), (64, 16384, 0), (96, 8192, 1), (16384, 40, 1)]


@pytest.mark.parametrize("nx,ny,bc", PLAIN)
@pytest.mark.parametrize("fp16", [False, True])
def test_cluster_lines_against_the_oracle(lib, nx, ny, bc, fp16):
    inst = _inst(nx, ny, bc)
    g = GpuGrid(lib, inst, FP32, fp16=fp16, fast=3)
    try:
        got = g.step(3)
    finally:
        g.close()
    T0, co = oracle_inputs(lib, inst, FP32, fp16=fp16)
    ref = oracle_step(inst, T0, co, 3)
    assert np.isfinite(got).all()
    assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 3, ref)


@pytest.mark.parametrize("nx,ny,bc", [(16384, 64, 1), (64, 8192, 0)])
@pytest.mark.parametrize("limiter", [2, 3])
def test_cluster_lines_other_limiters(lib, nx, ny, bc, limiter):
    inst = _inst(nx, ny, bc, seed=5)
    a = GpuGrid(lib, inst, FP32, fast=3, limiter=limiter)
    b = GpuGrid(lib, inst, FP32, fast=0, limiter=limiter)
    try:
        assert rel_linf(a.step(3), b.step(3)) < SAME_KERNELS_TOL
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("nx,ny,bc", [(4096, 128, 1), (128, 4096, 0), (2048, 96, 1)])
def test_cluster_option_takes_4096_lines(lib, nx, ny, bc):
    """ANISO_OPT_CLUSTER_LINES = 2 (the default) puts lines of 4096 cells on
    the cluster kernel (2 blocks a cluster) instead of the long-line kernel."""
    inst = _inst(nx, ny, bc, seed=17)
    g = GpuGrid(lib, inst, FP32, fast=3)
    lib.aniso_set_option(g.h, lib.ANISO_OPT_CLUSTER_LINES, 2)
    ref_g = GpuGrid(lib, inst, FP32, fast=0)
    try:
        got = g.step(3)
        assert rel_linf(got, ref_g.step(3)) < SAME_KERNELS_TOL
    finally:
        g.close()
        ref_g.close()
    T0, co = oracle_inputs(lib, inst, FP32)
    ref = oracle_step(inst, T0, co, 3)
    assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 3, ref)


def _kahan_grid(lib, inst, fp16=False, cluster=1):
    import torch
    h = lib.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, inst.chi_perp, inst.bc)
    lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, FP32)
    lib.aniso_set_option(h, lib.ANISO_OPT_KAHAN, 1)
    if fp16:
        lib.aniso_set_option(h, lib.ANISO_OPT_FIELD_FP16, 1)
    lib.aniso_set_option(h, lib.ANISO_OPT_CLUSTER_LINES, cluster)
    bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
    by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
    lib.aniso_set_field(h, bx, by)
    T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
    return h, T


def _hi_lo(lib, h, T):
    import torch
    lo = torch.empty_like(T)
    lib.aniso_get_state(h, lo)
    lib.aniso_sync(h)
    return T.double().cpu().numpy() + lo.double().cpu().numpy()


# compensated grids: 8 / 1 / 4 / 2 blocks a cluster in x and y
KAHAN = [(16384, 1024, 1, True), (1024, 8192, 0, True), (2048, 4096, 1, False), (4096, 2048, 0, True)]


@pytest.mark.parametrize("nx,ny,bc,fp16", KAHAN)
def test_compensated_cluster_lines_against_the_oracle(lib, nx, ny, bc, fp16):
    inst = _inst(nx, ny, bc, seed=41, chi_par=1.0, dt_factor=1000.0)
    T0, co = oracle_inputs(lib, inst, FP32, fp16=fp16)
    h, T = _kahan_grid(lib, inst, fp16=fp16)
    try:
        lib.aniso_step(h, T, inst.dt, 2)
        got = _hi_lo(lib, h, T)
        ref = oracle_step(inst, T0, co, 2)
        assert np.isfinite(got).all()
        assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 2, ref)
    finally:
        lib.aniso_destroy(h)


@pytest.mark.parametrize("nx,ny,bc", [(16384, 1024, 1), (1024, 8192, 0)])
def test_compensated_cluster_lines_conserve(lib, nx, ny, bc):
    """The FP64 sum of hi + lo stays within 1e-12 of its start (each line's
    rounding residual of delta is removed across the whole cluster)."""
    inst = _inst(nx, ny, bc, seed=7, chi_par=1.0, dt_factor=1000.0)
    h, T = _kahan_grid(lib, inst, fp16=True)
    try:
        s0 = lib.aniso_total(h, T)[0]
        lib.aniso_step(h, T, inst.dt, 10)
        s1 = lib.aniso_total(h, T)[0]
        assert abs(s1 - s0) / abs(s0) < 1e-12
    finally:
        lib.aniso_destroy(h)


def test_compensated_cluster_matches_the_general_kernels(lib):
    """The same compensated grid on the cluster kernel and, with the option
    off, on the general kernels with transposes."""
    inst = _inst(2048, 2048, 1, seed=9, chi_par=1.0, dt_factor=1000.0)
    a, Ta = _kahan_grid(lib, inst, fp16=True, cluster=1)
    b, Tb = _kahan_grid(lib, inst, fp16=True, cluster=0)
    try:
        lib.aniso_step(a, Ta, inst.dt, 5)
        lib.aniso_step(b, Tb, inst.dt, 5)
        assert rel_linf(_hi_lo(lib, a, Ta), _hi_lo(lib, b, Tb)) < SAME_KERNELS_TOL
    finally:
        lib.aniso_destroy(a)
        lib.aniso_destroy(b)


def test_cluster_grids_in_a_batch_match_single_grids(lib):
    """A batch with cluster-kernel grids (plain and compensated need separate
    batches: one precision mode a batch) equals the grids stepped one by one."""
    import torch
    insts = [_inst(8192, 64, 1, seed=31), _inst(512, 256, 1, seed=32), _inst(96, 16384, 0, seed=33)]
    grids = [GpuGrid(lib, i, FP32, fast=3) for i in insts]
    singles = [GpuGrid(lib, i, FP32, fast=3) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        try:
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [3] * len(insts))
            lib.aniso_sync(grids[0].h)
        finally:
            lib.aniso_batch_destroy(b)
        for g, s in zip(grids, singles):
            want = s.step(3)
            assert np.array_equal(g.T.double().cpu().numpy(), want)
    finally:
        for g in grids + singles:
            g.close()


def test_config2_full_grid_against_the_oracle(lib):
    """The 4096^2 random-field FP32 workload in the benchmark's launch
    configuration (aniso_step, default options: both updates on 2-block
    clusters), two steps, every cell against the oracle's full run."""
    inst = W.random_instance(4096, 4096, seed=W.BASE_SEED, chi_par=0.05, dt_factor=100.0, nsteps=2)
    g = GpuGrid(lib, inst, FP32)
    try:
        got = g.step(2)
    finally:
        g.close()
    T0, co = oracle_inputs(lib, inst, FP32)
    ref = oracle_step(inst, T0, co, 2)
    assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 2, ref)


def test_config4_full_grid_against_the_oracle(lib):
    """The 16384^2 compensated workload (FP32 hi+lo state, FP16 face
    coefficients, |k| <= 32, chi_par 1, dt = 1000 x CFL) in the benchmark's
    launch configuration (8-block clusters, the state interleaved between the
    steps of a call): two steps, every cell of hi + lo against the oracle's
    full run on the same FP16-rounded coefficients, and the sum of hi + lo."""
    inst = W.random_instance(16384, 16384, seed=W.BASE_SEED, kmax=32, chi_par=1.0, dt_factor=1000.0, nsteps=2)
    T0, co = oracle_inputs(lib, inst, FP32, fp16=True)
    h, T = _kahan_grid(lib, inst, fp16=True)
    try:
        s0 = lib.aniso_total(h, T)[0]
        lib.aniso_step(h, T, inst.dt, 2)
        s1 = lib.aniso_total(h, T)[0]
        got = _hi_lo(lib, h, T)
    finally:
        lib.aniso_destroy(h)
    assert abs(s1 - s0) / abs(s0) < 1e-12
    ref = oracle_step(inst, T0, co, 2)
    assert np.isfinite(got).all()
    assert rel_linf(got, ref) < 1e-4
