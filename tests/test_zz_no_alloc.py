"""aniso_step_noalloc, the step entry point for callers that may not allocate
device memory (it works in a fixed scratch array compiled into the library),
must give the same result as aniso_step on consecutive calls."""
import pytest

import workloads as W
from gpu_util import FP64_TOL_PER_STEP, rel_linf

FP32_SAME_KERNELS_TOL = 2e-5  # the FP32 tolerance of the kernel-path comparisons


def test_rejects_grids_above_the_scratch_limit():
    import paper_1008_0861_gb300 as P
    from paper_1008_0861_gb300 import build
    build.build()
    # 2048 x 1024 FP32 cells need 40 MiB of scratch: refused before any GPU work
    with pytest.raises(P.AnisoError) as ei:
        P.aniso_step_noalloc(2048, 1024, 1.0, 1.0, 1.0, 0.0, P.ANISO_BC_PERIODIC, P.ANISO_PREC_FP32,
                             0x1000, 0x1000, 0x1000, 1.0, 1)
    assert ei.value.code == P.ANISO_ERR_ARG and "scratch" in str(ei.value)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", ["ring", "random"])
def test_noalloc_matches_aniso_step_on_two_calls(lib, prec, which):
    import torch
    inst = W.ring_instance(50) if which == "ring" else W.random_instance(96, 64, seed=5)
    dtype = torch.float64 if prec == lib.ANISO_PREC_FP64 else torch.float32
    bx = torch.tensor(inst.bx, dtype=dtype, device="cuda")
    by = torch.tensor(inst.by, dtype=dtype, device="cuda")
    T_ref = torch.tensor(inst.T0, dtype=dtype, device="cuda")
    T_na = T_ref.clone()
    h = lib.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, prec)
        lib.aniso_set_option(h, lib.ANISO_OPT_FAST_PATH, 0)
        lib.aniso_set_field(h, bx, by)
        nsteps = 5
        for call in range(2):
            lib.aniso_step(h, T_ref, inst.dt, nsteps)
            lib.aniso_sync(h)
            lib.aniso_step_noalloc(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc,
                                   prec, bx, by, T_na, inst.dt, nsteps)
            torch.cuda.synchronize()
            got = T_na.double().cpu().numpy()
            ref = T_ref.double().cpu().numpy()
            done = nsteps * (call + 1)
            tol = done * FP64_TOL_PER_STEP if prec == lib.ANISO_PREC_FP64 else FP32_SAME_KERNELS_TOL
            assert rel_linf(got, ref) < tol, (call, rel_linf(got, ref))
    finally:
        lib.aniso_destroy(h)
