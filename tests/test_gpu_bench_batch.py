"""The benchmark's own configuration at full size: the 512-instance uneven
FP32 batch, block shape from the autotuner, one 200-step call.  Sampled
instances (the largest, a middle one, the last) against the FP64 oracle, and
every instance finite."""
import importlib.util
import os

import numpy as np
import pytest

import oracle as O
from gpu_util import fp32_tol, oracle_inputs, oracle_step, rel_linf

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_full_bench_batch_sampled_against_oracle(lib):
    import torch
    b = _bench()
    insts = b.make_instances(b.N_INST, 0)
    handles, Ts = [], []
    try:
        for inst in insts:
            h = lib.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
            handles.append(h)
            lib.aniso_set_option(h, lib.ANISO_OPT_PRECISION, lib.ANISO_PREC_FP32)
            bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
            by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
            lib.aniso_set_field(h, bx, by)
            Ts.append(torch.tensor(inst.T0, dtype=torch.float32, device="cuda"))
        batch = lib.aniso_batch_create(handles)
        dts = [i.dt for i in insts]
        choice, _ = lib.aniso_batch_autotune(batch, Ts, dts, nsteps=2, reps=1)
        assert choice >= 0
        lib.aniso_step_batched(batch, Ts, dts, [b.STEPS_PER_CALL] * len(insts))
        torch.cuda.synchronize()
        for k, (inst, T) in enumerate(zip(insts, Ts)):
            got = T.cpu().numpy()
            assert np.all(np.isfinite(got)), k
        big = max(range(len(insts)), key=lambda k: insts[k].cells)
        for k in sorted({big, len(insts) // 2, len(insts) - 1}):
            inst = insts[k]
            T0, co = oracle_inputs(lib, inst, 1)
            ref = oracle_step(inst, T0, co, b.STEPS_PER_CALL)
            got = Ts[k].double().cpu().numpy()
            assert rel_linf(got, ref) < max(1e-4, fp32_tol(inst, T0, co, b.STEPS_PER_CALL, ref)), k
        lib.aniso_batch_destroy(batch)
    finally:
        for h in handles:
            lib.aniso_destroy(h)
