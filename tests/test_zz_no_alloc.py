"""aniso_step_noalloc, the step entry point for callers that may not allocate
device memory (it works in a fixed scratch array compiled into the library),
must give the same result as aniso_step on consecutive calls: at the scratch
array's size limit, on odd sizes whose scratch regions start off 16-byte
boundaries, and on a stream other than the default one."""
import shutil

import numpy as np
import pytest

import workloads as W
from gpu_util import FP64_TOL_PER_STEP, oracle_inputs, oracle_step, rel_linf

FP32_SAME_KERNELS_TOL = 2e-5  # the FP32 tolerance of the kernel-path comparisons


def _have_nvcc():
    import os
    return bool(shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"))


@pytest.mark.skipif(not _have_nvcc(), reason="building the library needs nvcc")
def test_rejects_grids_above_the_scratch_limit():
    import paper_1008_0861_gb300 as P
    from paper_1008_0861_gb300 import build
    build.build()
    # 2048 x 1024 FP32 cells need 40 MiB of scratch: refused before any GPU work
    with pytest.raises(P.AnisoError) as ei:
        P.aniso_step_noalloc(2048, 1024, 1.0, 1.0, 1.0, 0.0, P.ANISO_BC_PERIODIC, P.ANISO_PREC_FP32,
                             0x1000, 0x1000, 0x1000, 1.0, 1)
    assert ei.value.code == P.ANISO_ERR_ARG and "scratch" in str(ei.value)
    # one FP64 cell over the limit (524,288 cells) is refused too
    with pytest.raises(P.AnisoError) as ei:
        P.aniso_step_noalloc(513, 1024, 1.0, 1.0, 1.0, 0.0, P.ANISO_BC_PERIODIC, P.ANISO_PREC_FP64,
                             0x1000, 0x1000, 0x1000, 1.0, 1)
    assert ei.value.code == P.ANISO_ERR_ARG


def _compare_two_calls(lib, inst, prec, nsteps, stream=None):
    """Two consecutive calls of aniso_step (general kernels) and of
    aniso_step_noalloc from the same T; returns the last noalloc state."""
    import torch
    dtype = torch.float64 if prec == lib.ANISO_PREC_FP64 else torch.float32
    bx = torch.tensor(inst.bx, dtype=dtype, device="cuda")
    by = torch.tensor(inst.by, dtype=dtype, device="cuda")
    T_ref = torch.tensor(inst.T0, dtype=dtype, device="cuda")
    T_na = T_ref.clone()
    torch.cuda.synchronize()
    h = lib.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, prec)
        lib.aniso_set_option(h, lib.ANISO_OPT_FAST_PATH, 0)
        lib.aniso_set_field(h, bx, by)
        for call in range(2):
            lib.aniso_step(h, T_ref, inst.dt, nsteps)
            lib.aniso_sync(h)
            lib.aniso_step_noalloc(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc,
                                   prec, bx, by, T_na, inst.dt, nsteps,
                                   None if stream is None else stream.cuda_stream)
            if stream is None:
                torch.cuda.synchronize()
            else:
                stream.synchronize()
            got = T_na.double().cpu().numpy()
            ref = T_ref.double().cpu().numpy()
            done = nsteps * (call + 1)
            tol = done * FP64_TOL_PER_STEP if prec == lib.ANISO_PREC_FP64 else FP32_SAME_KERNELS_TOL
            assert rel_linf(got, ref) < tol, (call, rel_linf(got, ref))
        return got
    finally:
        lib.aniso_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", ["ring", "random"])
def test_noalloc_matches_aniso_step_on_two_calls(lib, prec, which):
    inst = W.ring_instance(50) if which == "ring" else W.random_instance(96, 64, seed=5)
    _compare_two_calls(lib, inst, prec, nsteps=5)


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,prec", [(1024, 1024, 1), (512, 1024, 0)])
def test_noalloc_at_the_scratch_limit(lib, nx, ny, prec):
    # 5 regions of nx*ny cells fill the 20 MiB exactly: the last byte of the
    # last region (cyx) is the array's last byte
    inst = W.random_instance(nx, ny, seed=11, dt_factor=50.0, nsteps=2)
    _compare_two_calls(lib, inst, prec, nsteps=2)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_odd_size_on_a_side_stream_matches_the_oracle(lib, prec):
    # 51 x 53 cells: every region after the first starts off a 16-byte
    # boundary; the calls go to a non-default stream
    import torch
    inst = W.random_instance(51, 53, seed=3, dt_factor=30.0, nsteps=3)
    inst.bc = 0  # zero-flux on the odd grid
    side = torch.cuda.Stream()
    got = _compare_two_calls(lib, inst, prec, nsteps=3, stream=side)
    # and against the FP64 oracle itself, after both calls (6 steps)
    T0, co = oracle_inputs(lib, inst, prec)
    ref = oracle_step(inst, T0, co, 6)
    tol = 6 * FP64_TOL_PER_STEP if prec == lib.ANISO_PREC_FP64 else 1e-4
    assert rel_linf(got, ref) < tol
    assert np.isfinite(got).all()
