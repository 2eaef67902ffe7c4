"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  FP64 within 1e-12 relative per step.  FP32 within 1e-4
relative L-inf after the stated steps, or within 3x the problem's own FP32
noise floor where that floor is larger (strongly non-square grids, where the
limited scheme amplifies one-ulp changes; see gpu_util.fp32_noise_floor).
FP16 field storage is compared against the oracle run on the same
FP16-rounded coefficients."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import (FP32_TOL, FP64_TOL_PER_STEP, GpuGrid, fp32_tol, oracle_inputs, oracle_step,
                      rel_linf)

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1

# sizes that span several tiles and ragged tails for both kernels
SIZES = [(3, 3), (5, 7), (33, 17), (50, 50), (64, 96), (130, 70), (257, 33), (1024, 40),
         (40, 1024), (96, 1100), (24, 2048)]


def _inst(nx, ny, bc, seed=1):
    if bc == 1:
        return W.random_instance(nx, ny, seed=seed, dt_factor=100.0)
    r = W.ring_instance(nx, ny=ny, dt_factor=100.0)
    return r


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("fast", [1, 3, 0])
def test_single_sweeps_fp64(lib, nx, ny, bc, fast):
    inst = _inst(nx, ny, bc, seed=nx * 7 + ny)
    T0, co = oracle_inputs(lib, inst, FP64)
    lamx, lamy, mu = O.lambdas(inst.dt, inst.dx, inst.dy, inst.chi_par)
    g = GpuGrid(lib, inst, FP64, fast=fast)
    try:
        gx = g.sweep(lib.ANISO_DIR_X, T0)
        ox = O.xsweep(T0, co, bc, lamx, mu)
        assert rel_linf(gx, ox) < FP64_TOL_PER_STEP
        gy = g.sweep(lib.ANISO_DIR_Y, ox)
        oy = O.ysweep(ox, co, bc, lamy, mu)
        assert rel_linf(gy, oy) < FP64_TOL_PER_STEP
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(50, 50), (64, 96), (33, 1030), (8, 6), (256, 2048), (2, 2)])
@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("fast", [1, 3, 0])
def test_steps_fp64_all_orders(lib, nx, ny, order, fast):
    if (nx, ny) == (2, 2):
        nx, ny = 12, 4
    inst = _inst(nx, ny, 1, seed=3)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, order=order, fast=fast)
    try:
        nsteps = 7
        got = g.step(nsteps)
        ref = oracle_step(inst, T0, co, nsteps, order=order)
        assert rel_linf(got, ref) < nsteps * FP64_TOL_PER_STEP
    finally:
        g.close()


def test_ring_config_fp64_and_conservation(lib):
    """Ring test, 50x50, FP64, zero-flux, dt = 10x the explicit limit, 250
    steps to t = 200: per-step parity and exact conservation."""
    inst = W.ring_instance(50)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64)
    try:
        s0 = lib.aniso_total(g.h, g.T)[0]
        T = T0
        for k in range(0, 250, 50):
            got = g.step(50)
            T = oracle_step(inst, T, co, 50)
            assert rel_linf(got, T) < (k + 50) * FP64_TOL_PER_STEP
        s, lo, hi, nf = lib.aniso_total(g.h, g.T)
        assert nf == 0 and abs(s - s0) / s0 < 1e-12
        assert abs(s - T.sum()) / s0 < 1e-12
        assert lo == pytest.approx(T.min(), rel=1e-12) and hi == pytest.approx(T.max(), rel=1e-12)
    finally:
        g.close()


@pytest.mark.parametrize("limiter", [1, 2, 3])
def test_other_limiters_fp64(lib, limiter):
    inst = _inst(48, 40, 1, seed=5)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, limiter=limiter)
    try:
        got = g.step(4)
        ref = oracle_step(inst, T0, co, 4, limiter=limiter)
        assert rel_linf(got, ref) < 4 * FP64_TOL_PER_STEP
    finally:
        g.close()


def test_chi_perp_and_unequal_spacing_fp64(lib):
    inst = W.random_instance(40, 56, seed=8)
    inst.chi_perp = 0.3 * inst.chi_par
    inst.dy = 1.7 * inst.dx
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64)
    try:
        got = g.step(5)
        assert rel_linf(got, oracle_step(inst, T0, co, 5)) < 5 * FP64_TOL_PER_STEP
    finally:
        g.close()


@pytest.mark.parametrize("nx,ny", [(256, 256), (96, 1024), (1024, 64), (100, 1200), (2048, 512)])
def test_random_field_fp32(lib, nx, ny):
    """Random-field workload at reduced size, FP32, dt = 100x the explicit
    limit, 100 steps.  Tolerance: 1e-4, or 3x the FP32 noise floor of the
    problem itself on non-square grids (see gpu_util.fp32_noise_floor)."""
    inst = W.random_instance(nx, ny, seed=20100805, chi_par=0.05, dt_factor=100.0)
    T0, co = oracle_inputs(lib, inst, FP32)
    g = GpuGrid(lib, inst, FP32)
    try:
        got = g.step(100)
        ref = oracle_step(inst, T0, co, 100)
        tol = fp32_tol(inst, T0, co, 100, ref)
        if nx == ny:
            assert tol == FP32_TOL
        assert rel_linf(got, ref) < tol
    finally:
        g.close()


def test_fp16_field_fp32(lib):
    inst = W.random_instance(128, 160, seed=77, chi_par=1.0, dt_factor=1000.0)
    T0, co = oracle_inputs(lib, inst, FP32, fp16=True)
    g = GpuGrid(lib, inst, FP32, fp16=True)
    try:
        got = g.step(20)
        ref = oracle_step(inst, T0, co, 20)
        assert rel_linf(got, ref) < fp32_tol(inst, T0, co, 20, ref)
    finally:
        g.close()


def test_graph_and_direct_launches_agree(lib):
    inst = _inst(72, 88, 1, seed=9)
    a = GpuGrid(lib, inst, FP32, graph=True)
    b = GpuGrid(lib, inst, FP32, graph=False)
    try:
        np.testing.assert_array_equal(a.step(6), b.step(6))
        np.testing.assert_array_equal(a.step(6), b.step(6))  # replay of the cached graph
    finally:
        a.close()
        b.close()


def test_alternating_order_counter_persists(lib):
    inst = _inst(40, 36, 1, seed=4)
    T0, co = oracle_inputs(lib, inst, FP64)
    g = GpuGrid(lib, inst, FP64, order=2)
    try:
        g.step(3)
        got = g.step(2)
        assert lib.aniso_get_state(g.h) == 5
        ref = oracle_step(inst, T0, co, 5, order=2)
        assert rel_linf(got, ref) < 5 * FP64_TOL_PER_STEP
    finally:
        g.close()


def test_fourier_mode_closed_form_on_gpu(lib):
    """Eqs. amp1/amp2 with the arithmetic-mean transverse average, on the GPU
    directly (constant b, periodic)."""
    nx, ny, mx, my, chi = 64, 48, 3, -2, 0.4
    dx, dy = 1.0 / nx, 1.0 / ny
    dt = 300 * W.cfl_dt(dx, dy, chi)
    alpha = 0.7
    bxv, byv = math.cos(alpha), math.sin(alpha)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    T0 = np.cos(2 * math.pi * (mx * x[None, :] + my * y[:, None]))
    inst = W.Instance("mode", nx, ny, dx, dy, 1, chi, 0.0, dt, 1, np.full((ny, nx), bxv),
                      np.full((ny, nx), byv), T0)
    lamx, lamy, mu = O.lambdas(dt, dx, dy, chi)
    tx, ty = 2 * math.pi * mx * dx, 2 * math.pi * my * dy
    num = 1 - mu * bxv * byv * math.sin(tx) * math.sin(ty)
    r = num / (1 + 4 * lamx * bxv ** 2 * math.sin(tx / 2) ** 2) * num / (
        1 + 4 * lamy * byv ** 2 * math.sin(ty / 2) ** 2)
    g = GpuGrid(lib, inst, FP64, limiter=1)
    try:
        np.testing.assert_allclose(g.step(1), r * T0, atol=1e-12)
    finally:
        g.close()


def test_nonfinite_is_reported(lib):
    inst = _inst(32, 32, 1, seed=2)
    T0 = inst.T0.copy()
    T0[5, 7] = np.nan
    g = GpuGrid(lib, inst, FP32, T0=T0, graph=False)
    try:
        lib.aniso_step(g.h, g.T, inst.dt, 1)
        with pytest.raises(lib.AnisoError) as ei:
            lib.aniso_sync(g.h)
        assert ei.value.code == lib.ANISO_ERR_NONFINITE
        lib.aniso_sync(g.h)  # flag cleared
    finally:
        g.close()


def _batch_insts(count, cap=512, nsteps=12):
    return W.batch_instances(count, nsteps=nsteps, size_cap=cap)


def test_batched_matches_oracle_and_single(lib):
    import torch
    insts = _batch_insts(12)
    grids = [GpuGrid(lib, i, FP32) for i in insts]
    singles = [GpuGrid(lib, i, FP32) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        nsteps = [i.nsteps - (k % 3) for k, i in enumerate(insts)]  # uneven step counts
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], nsteps)
        torch.cuda.synchronize()
        for k, (g, s, inst) in enumerate(zip(grids, singles, insts)):
            got = g.T.double().cpu().numpy()
            np.testing.assert_array_equal(got, s.step(nsteps[k]))
            T0, co = oracle_inputs(lib, inst, FP32)
            ref = oracle_step(inst, T0, co, nsteps[k])
            assert rel_linf(got, ref) < fp32_tol(inst, T0, co, nsteps[k], ref)
            assert lib.aniso_get_state(g.h) == nsteps[k]
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids + singles:
            g.close()


def test_batched_fp64_mixed_boundaries(lib):
    import torch
    insts = [W.ring_instance(48, ny=40, dt_factor=50.0), W.random_instance(64, 32, seed=3),
             W.ring_instance(30, ny=66, dt_factor=500.0)]
    grids = [GpuGrid(lib, i, FP64) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        for _ in range(2):  # second call replays the captured graph
            lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [3, 3, 3])
        torch.cuda.synchronize()
        for g, inst in zip(grids, insts):
            T0, co = oracle_inputs(lib, inst, FP64)
            ref = oracle_step(inst, T0, co, 6)
            assert rel_linf(g.T.double().cpu().numpy(), ref) < 6 * FP64_TOL_PER_STEP
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids:
            g.close()


def test_full_size_random_field_sampled_lines(lib):
    """4096^2 random-field workload in FP32, in the launch configuration of the
    benchmark: one x-update and one y-update on the full grid, compared with
    the oracle line by line on sampled rows and columns."""
    inst = W.random_instance(4096, 4096, seed=20100805, chi_par=0.05, dt_factor=100.0)
    T0, co = oracle_inputs(lib, inst, FP32)
    lamx, lamy, mu = O.lambdas(inst.dt, inst.dx, inst.dy, inst.chi_par)
    g = GpuGrid(lib, inst, FP32)
    try:
        Ts = g.sweep(lib.ANISO_DIR_X, T0)
        for j in (0, 1, 777, 2048, 4095):
            ref = O.xsweep_row(T0[j - 1], T0[j], T0[(j + 1) % 4096], co.cxx[j], co.cxy[j], lamx, mu,
                               True)
            assert rel_linf(Ts[j], ref) < 1e-5
        Tn = g.sweep(lib.ANISO_DIR_Y, Ts)
        for i in (0, 5, 1999, 4095):
            ref = O.ysweep_col(Ts[:, i - 1], Ts[:, i], Ts[:, (i + 1) % 4096], co.cyy[:, i],
                               co.cyx[:, i], lamy, mu, True)
            assert rel_linf(Tn[:, i], ref) < 1e-5
    finally:
        g.close()


@pytest.mark.parametrize("kahan", [0, 1])
def test_large_grid_one_dimensional_mode_closed_form(lib, kahan):
    """16384^2 FP32 with FP16 field storage (and the compensated state): a
    y-only mode under constant b decays by exactly
    1/(1 + 4 lamy by^2 sin^2(ky dy/2)) per step (the x-update leaves it
    unchanged), a property that holds at any size."""
    import torch
    n = 16384
    dx = 1.0 / n
    alpha = 0.6
    bxv, byv = math.cos(alpha), math.sin(alpha)
    h = lib.aniso_create(n, n, dx, dx, 1.0, 0.0, 1)
    try:
        lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, FP32)
        lib.aniso_set_option(h, lib.ANISO_OPT_FIELD_FP16, 1)
        lib.aniso_set_option(h, lib.ANISO_OPT_KAHAN, kahan)
        bx = torch.full((n, n), bxv, dtype=torch.float32, device="cuda")
        by = torch.full((n, n), byv, dtype=torch.float32, device="cuda")
        lib.aniso_set_field(h, bx, by)
        del bx, by
        by16 = float(np.float16(np.float64(np.float32(byv)) ** 2))  # stored cyy
        y = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) * dx
        my = 5
        mode = torch.cos(2 * math.pi * my * y)
        T = (2.0 + mode)[:, None].expand(n, n).contiguous().float()
        dt = 1000 * dx * dx / 2
        lib.aniso_step(h, T, dt, 3)
        lib.aniso_sync(h)
        lamy = dt / (dx * dx)
        r = 1.0 / (1.0 + 4 * lamy * by16 * math.sin(math.pi * my * dx) ** 2)
        expect = (2.0 + r ** 3 * mode).float()
        rows = torch.tensor([0, 1, 4097, 9000, n - 1], device="cuda")
        err = (T[rows].double() - expect[rows, None].double()).abs().max().item()
        assert err < 3e-6
        s, lo, hi, nf = lib.aniso_total(h, T)
        assert nf == 0 and abs(s / (n * n) - 2.0) < 1e-6
    finally:
        lib.aniso_destroy(h)


@pytest.mark.parametrize("graph", [True, False])
def test_kernel_timing_events(lib, graph):
    """ANISO_OPT_PROFILE times every sweep launch, inside captured graphs too."""
    inst = _inst(128, 96, 1, seed=6)
    g = GpuGrid(lib, inst, FP32, graph=graph)
    try:
        lib.aniso_set_option(g.h, lib.ANISO_OPT_PROFILE, 1)
        g.step(4)
        g.step(4)
        for kind in (lib.ANISO_KERNEL_XSWEEP, lib.ANISO_KERNEL_YSWEEP):
            ms, n = lib.aniso_kernel_times(h=g.h, kind=kind)
            assert n == 8 and ms > 0.0
        lib.aniso_kernel_times(h=g.h, kind=0, reset=True)
        assert lib.aniso_kernel_times(h=g.h, kind=1) == (0.0, 0)
    finally:
        g.close()


@pytest.mark.parametrize("every", [1, 3])
def test_batch_kernel_timing_every_kth_step(lib, every):
    """In batched calls ANISO_OPT_PROFILE = k times the sweeps of steps 0, k,
    2k, ... of each call (7 steps: 7 or 3 sweeps of each kind a call), and the
    results do not depend on it."""
    insts = [_inst(128, 96, 1, seed=21), _inst(256, 64, 0, seed=22)]
    grids = [GpuGrid(lib, i, FP32) for i in insts]
    plain = [GpuGrid(lib, i, FP32) for i in insts]
    try:
        lib.aniso_set_option(grids[0].h, lib.ANISO_OPT_PROFILE, every)
        b = lib.aniso_batch_create([g.h for g in grids])
        pb = lib.aniso_batch_create([g.h for g in plain])
        try:
            for _ in range(2):
                lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [7, 7])
                lib.aniso_step_batched(pb, [g.T for g in plain], [i.dt for i in insts], [7, 7])
            per_call = 7 if every == 1 else 3
            for kind in (lib.ANISO_KERNEL_XSWEEP, lib.ANISO_KERNEL_YSWEEP):
                ms, n = lib.aniso_kernel_times(batch=b, kind=kind)
                assert n == 2 * per_call and ms > 0.0
            lib.aniso_sync(grids[0].h)
            lib.aniso_sync(plain[0].h)
            for g, p in zip(grids, plain):
                assert np.array_equal(g.T.cpu().numpy(), p.T.cpu().numpy())
        finally:
            lib.aniso_batch_destroy(b)
            lib.aniso_batch_destroy(pb)
    finally:
        for g in grids + plain:
            g.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("nx,ny,bc", [(64, 96, 1), (128, 40, 0), (1024, 1024, 1), (36, 2048, 1),
                                      (512, 96, 1), (1000, 8, 0)])
@pytest.mark.parametrize("fast", [1, 3])
def test_fast_path_matches_general_kernels(lib, prec, nx, ny, bc, fast):
    """The vectorised x-then-y paths (staged and unstaged, transposed
    intermediate) and the general kernels compute the same step: to 1e-12 per
    step in FP64, within FP32 rounding in FP32."""
    inst = _inst(nx, ny, bc, seed=12)
    a = GpuGrid(lib, inst, prec, fast=fast)
    b = GpuGrid(lib, inst, prec, fast=0)
    try:
        ga, gb = a.step(5), b.step(5)
        tol = 5 * FP64_TOL_PER_STEP if prec == FP64 else 2e-5
        assert rel_linf(ga, gb) < tol
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("fast", [1, 3])
def test_fp16_field_fast_and_general_agree(lib, fast):
    inst = W.random_instance(256, 128, seed=31, chi_par=1.0, dt_factor=1000.0)
    a = GpuGrid(lib, inst, FP32, fp16=True, fast=fast)
    b = GpuGrid(lib, inst, FP32, fp16=True, fast=0)
    try:
        assert rel_linf(a.step(3), b.step(3)) < 2e-5
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("fast", [1, 3])
def test_batched_fast_paths_match_single(lib, fast):
    """Batched launches of the staged and unstaged kernels reproduce the
    single-grid steps bit for bit (mixed sizes, one launch per sweep)."""
    import torch
    insts = W.batch_instances(10, nsteps=4, size_cap=1024)
    grids = [GpuGrid(lib, i, FP32, fast=fast) for i in insts]
    singles = [GpuGrid(lib, i, FP32, fast=fast) for i in insts]
    try:
        b = lib.aniso_batch_create([g.h for g in grids])
        lib.aniso_step_batched(b, [g.T for g in grids], [i.dt for i in insts], [4] * len(insts))
        torch.cuda.synchronize()
        for g, s in zip(grids, singles):
            np.testing.assert_array_equal(g.T.double().cpu().numpy(), s.step(4))
        lib.aniso_batch_destroy(b)
    finally:
        for g in grids + singles:
            g.close()
