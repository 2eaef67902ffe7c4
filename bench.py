"""Benchmark: batched uneven grids, FP32, all steps of a call in one captured CUDA graph.

Workload (one bench "step" = one aniso_step_batched call): 512 independent
periodic random-field grids, nx and ny drawn from the multiples of 32 in
[64, 1024], chi_par log-uniform in [1e-3, 1e-1], dt log-uniform in
[10, 1000] x the explicit limit, 200 steps each, FP32 state and FP32 face
coefficients.  Metric: Gcell-steps/s = sum(nx*ny*steps) / wall time / 1e9.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-steps/s, FP32 batched vs plain FP64 on one GB300 at L∞ err<=1e-4; % HBM peak"
UNIT = "Gcell-steps/s"
N_INST = 512
STEPS_PER_CALL = 200
PROFILE_EVERY = 8  # batch: sweeps of steps 0, 8, 16, ... of a call are timed by events
BYTES_PER_CELL_SWEEP = 16  # FP32: read T (4) + two face coefficients (8) + write T (4)
WORKLOAD = ("batched 512 uneven periodic random-field grids (nx, ny multiples of 32 in "
            "[64,1024]), FP32, 200 steps per call in a captured CUDA graph, each sweep one launch per "
            "occupancy class of line lengths (run concurrently)")


def parse_args_for_test(argv):
    """parse() on an explicit argument list."""
    old = sys.argv
    try:
        sys.argv = ["bench.py"] + list(argv)
        return parse()
    finally:
        sys.argv = old


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--instances", type=int, default=N_INST)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the block-shape autotuner")
    ap.add_argument("--no-big", action="store_true",
                    help="skip the 16384^2 compensated single-grid leg (and its minute-long oracle run)")
    ap.add_argument("--no-legs", action="store_true",
                    help="only the timed batch: no accuracy, FP64, single-grid or 3-D legs")
    ap.add_argument("--tma-lines", type=int, default=-1,
                    help="ANISO_OPT_TMA_LINES for the batch (-1: library default)")
    ap.add_argument("--tmem", type=int, default=-1,
                    help="ANISO_OPT_TMEM for the batch (-1: library default)")
    ap.add_argument("--segment", type=int, default=0,
                    help="16-byte chunks per thread segment (0: library default)")
    ap.add_argument("--fast", type=int, default=-1,
                    help="ANISO_OPT_FAST_PATH value (-1: library default)")
    ap.add_argument("--workload", default="batch", choices=["batch", "random3d", "random4096", "compensated"],
                    help="batch: the 512-grid 2-D benchmark (default); random3d: one 256^3 "
                         "grid of the three-dimensional split; random4096: one 4096^2 FP32 grid "
                         "(100 steps per call, lines above 2048 cells); compensated: one grid "
                         "(--shape, default 16384x16384) with the FP32 hi+lo state and FP16 "
                         "face coefficients, 50 steps per call")
    ap.add_argument("--cluster-lines", type=int, default=-1,
                    help="ANISO_OPT_CLUSTER_LINES for the random4096 workload (-1: library default; 1 "
                         "puts its 4096-cell lines on the long-line kernel)")
    ap.add_argument("--shape", default="16384x16384",
                    help="NXxNY of the compensated workload (sides of 1024 * 2^k cells, up to 16384)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(value, op, device):
    """MAX or SUM of one number over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(cell_steps_local, ms_local, device):
    """Whole-job Gcell-steps/s: the cell-steps all ranks processed over the
    slowest rank's time.  Returns (value, max ms, total cell-steps)."""
    ms = reduce_over_ranks(ms_local, "max", device)
    units = reduce_over_ranks(cell_steps_local, "sum", device)
    return units / (ms * 1e-3) / 1e9, ms, units


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    # the files that define the profiled kernels (line4 2-D and 3-D, line7) and their job structs
    for f in ("sweep_kernels.cuh", "line2_kernel.cuh", "line4_kernel.cuh", "line7_kernel.cuh",
              "aniso_internal.h", "kernels_line4.cu", "kernels_line7.cu", "kernels_3d.cu"):
        h.update(open(os.path.join(ROOT, "paper_1008_0861_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
        ent = d[kernel]
        if ent.get("source_hash") != kernel_source_hash():
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def make_instances(count, rank):
    import workloads as W
    return W.batch_instances(count, nsteps=STEPS_PER_CALL, first=rank * count)


def cpu_baseline(insts, budget_s=12.0, single_thread_s=0.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    whole instances for their full 200 steps until the time budget is used."""
    import numpy as np
    import oracle as O
    cells = 0
    t0 = time.perf_counter()
    used = []
    for inst in insts:
        w = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
        co = O.face_coeffs(w(inst.bx), w(inst.by), inst.bc, inst.chi_par)
        O.step(w(inst.T0), co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=inst.nsteps)
        cells += inst.cells * inst.nsteps
        used.append(inst.name)
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    out = {"value": cells / el / 1e9, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "%d of %d instances (%s..%s), full %d steps each, FP64, %.1f s" % (
               len(used), len(insts), used[0], used[-1], STEPS_PER_CALL, el)}
    if single_thread_s > 0:
        # the same oracle on one thread, on the largest of the first eight instances
        nt = O.num_threads()
        O.set_num_threads(1)
        try:
            inst = max(insts[:8], key=lambda i: i.cells)
            co = O.face_coeffs(w(inst.bx), w(inst.by), inst.bc, inst.chi_par)
            t1 = time.perf_counter()
            k = 0
            T = w(inst.T0)
            while time.perf_counter() - t1 < single_thread_s:
                T = O.step(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=5)
                k += 5
            el1 = time.perf_counter() - t1
        finally:
            O.set_num_threads(nt)
        out["value_1_thread"] = inst.cells * k / el1 / 1e9
        out["sample_1_thread"] = "%s, %d steps, 1 thread, %.1f s" % (inst.name, k, el1)
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    insts = make_instances(args.instances, 0)
    # each reference step: a bounded sample of the workload (whole instances, full steps)
    per_step_budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(insts[:2], budget_s=0.1)
    vals, samples, step_ms = [], [], []
    for k in range(args.steps):
        start = (k * 3) % len(insts)
        t0 = time.perf_counter()
        b = cpu_baseline(insts[start:] + insts[:start], budget_s=per_step_budget)
        step_ms.append((time.perf_counter() - t0) * 1e3)
        vals.append(b["value"])
        samples.append(b["sample"])
    v = statistics.median(vals)
    import oracle as O
    total_cells = sum(i.cells for i in insts) * STEPS_PER_CALL
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            # measured: the wall time of each step's bounded sample (whole instances, 200 steps each)
            "ms_per_step": statistics.median(step_ms),
            # what one full 512-instance call would take at the sampled rate (not measured)
            "extrapolated_ms_per_full_call": total_cells / (v * 1e9) * 1e3 if v else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "instances": len(insts)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": samples[0]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _w32(a):
    """FP32-rounded copy widened back to FP64: the inputs an FP32 run sees."""
    import numpy as np
    return a.astype(np.float32).astype(np.float64)


def _rel_linf(a, ref):
    import numpy as np
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def _oracle_sample(insts, count=64):
    """Indices of a stratified sample of the batch for the oracle: the most
    non-square half (largest max(nx,ny)/min(nx,ny), where the FP32 state sits
    closest to the scheme's own rounding sensitivity), the other half spread
    evenly over the remaining instances ordered by cell count."""
    order = sorted(range(len(insts)), key=lambda k: -max(insts[k].nx, insts[k].ny) / min(insts[k].nx, insts[k].ny))
    half = min(count // 2, len(insts))
    chosen = order[:half]
    rest = sorted(order[half:], key=lambda k: insts[k].cells)
    m = min(count - half, len(rest))
    if m > 0:
        chosen += [rest[int(round(i * (len(rest) - 1) / max(1, m - 1)))] for i in range(m)]
    return sorted(set(chosen))


def batch_accuracy(P, torch, batch, Ts, insts, dts):
    """The metric's accuracy bar on every instance of the batch.

    The FP32 batch runs one 200-step call from the initial state; the same
    512 grids (FP32-rounded inputs widened exactly) run in FP64 on the GPU as
    one FP64 batch, whose per-step agreement with the FP64 oracle is 1e-12
    (tested).  Reported: rel L-inf of FP32 against FP64 for every instance,
    the FP64 batch's own rate (the plain-FP64 side of the metric on the same
    workload), the oracle itself on a stratified sample of 64 instances, and
    the compensated (hi, lo) FP32 state on the instances where plain FP32 is
    worst."""
    import numpy as np
    import oracle as O
    nst = [STEPS_PER_CALL] * len(insts)
    T0 = [_w32(i.T0) for i in insts]
    for t, a in zip(Ts, T0):
        t.copy_(torch.from_numpy(a.astype(np.float32)))
    P.aniso_step_batched(batch, Ts, dts, nst)
    torch.cuda.synchronize()
    T32 = [t.double().cpu().numpy() for t in Ts]

    # the same batch in FP64
    h64, T64d, keep = [], [], []
    for inst in insts:
        h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP64)
        bx = torch.tensor(_w32(inst.bx), dtype=torch.float64, device="cuda")
        by = torch.tensor(_w32(inst.by), dtype=torch.float64, device="cuda")
        P.aniso_set_field(h, bx, by)
        keep.append((bx, by))
        h64.append(h)
        T64d.append(torch.tensor(_w32(inst.T0), dtype=torch.float64, device="cuda"))
    b64 = P.aniso_batch_create(h64)
    try:
        torch.cuda.synchronize()
        del keep
        P.aniso_step_batched(b64, T64d, dts, nst)  # builds the graph; this call's result is the reference
        torch.cuda.synchronize()
        T64 = [t.cpu().numpy() for t in T64d]
        for t, a in zip(T64d, T0):
            t.copy_(torch.from_numpy(a))
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        P.aniso_step_batched(b64, T64d, dts, nst)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
    finally:
        P.aniso_batch_destroy(b64)
        for h in h64:
            P.aniso_destroy(h)
    cell_steps = sum(i.cells for i in insts) * STEPS_PER_CALL
    rate64 = cell_steps / (ms64 * 1e-3) / 1e9
    peak, note = measured_peak()

    errs = np.array([_rel_linf(a, r) for a, r in zip(T32, T64)])
    drift = max(abs(float(a.sum()) - float(t0.sum())) / abs(float(t0.sum())) for a, t0 in zip(T32, T0))
    worst = int(np.argmax(errs))
    wi = insts[worst]
    above = [k for k in range(len(insts)) if errs[k] > 1e-4]

    def shape(k):
        i = insts[k]
        return {"instance": i.name, "nx": i.nx, "ny": i.ny,
                "lam_x": i.chi_par * i.dt / i.dx ** 2, "lam_y": i.chi_par * i.dt / i.dy ** 2,
                "rel_linf": float(errs[k])}

    # the oracle itself on a stratified sample
    sample = _oracle_sample(insts)
    t0 = time.perf_counter()
    o32, o64 = [], []
    for k in sample:
        inst = insts[k]
        co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par)
        ref = O.step(T0[k], co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=STEPS_PER_CALL)
        o32.append(_rel_linf(T32[k], ref))
        o64.append(_rel_linf(T64[k], ref))
    t_oracle = time.perf_counter() - t0

    # Instances above 1e-4: how far the FP64 oracle itself moves when its
    # initial state changes by rounding alone (relative 1e-15 of seeded
    # noise).  Where that is of the same size as the FP32 error, the bar is
    # beyond what the scheme's own sensitivity allows at this timestep.
    t1 = time.perf_counter()
    sens = []
    rng = np.random.default_rng(7)
    for k in above:
        inst = insts[k]
        co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par)
        ref = O.step(T0[k], co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=STEPS_PER_CALL)
        Tp = T0[k] * (1.0 + 1e-15 * rng.standard_normal(T0[k].shape))
        pert = O.step(Tp, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=STEPS_PER_CALL)
        # the oracle with its state rounded to FP32 after every step: what
        # storing T in FP32 alone costs, whatever the arithmetic
        Tr = T0[k].copy()
        for _ in range(STEPS_PER_CALL):
            Tr = O.step(Tr, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1)
            Tr = Tr.astype(np.float32).astype(np.float64)
        sens.append({"instance": inst.name, "nx": inst.nx, "ny": inst.ny,
                     "fp32_vs_oracle": _rel_linf(T32[k], ref), "fp64_gpu_vs_oracle": _rel_linf(T64[k], ref),
                     "oracle_vs_oracle_perturbed_1e-15": _rel_linf(pert, ref),
                     "oracle_fp32_state_vs_oracle": _rel_linf(Tr, ref)})
        if time.perf_counter() - t1 > 90.0:
            break
    t_sens = time.perf_counter() - t1

    # the compensated (hi, lo) state on the worst plain-FP32 instances
    comp = []
    for k in list(np.argsort(-errs)[:4]):
        inst = insts[int(k)]
        h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
        try:
            P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
            P.aniso_set_option(h, P.ANISO_OPT_KAHAN, 1)
            bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
            by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
            P.aniso_set_field(h, bx, by)
            t = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
            P.aniso_step(h, t, inst.dt, STEPS_PER_CALL)
            P.aniso_sync(h)
            lo = torch.empty_like(t)
            P.aniso_get_state(h, lo)
            torch.cuda.synchronize()
            hilo = t.double().cpu().numpy() + lo.double().cpu().numpy()
        finally:
            P.aniso_destroy(h)
        entry = shape(int(k))
        entry["rel_linf_hi_lo"] = _rel_linf(hilo, T64[int(k)])
        comp.append(entry)

    acc = {
        "sample": "every instance after one 200-step call, FP32 against the same batch in FP64 on the GPU",
        "instances": len(insts),
        "rel_linf_vs_fp64": {"max": float(errs.max()), "median": float(np.median(errs)),
                             "count_above_1e-4": len(above), "worst": shape(worst)},
        "above_1e-4": [shape(k) for k in above][:16],
        "rel_linf_vs_fp64_oracle": max(o32),
        "oracle_sample": {"instances": len(sample), "fp32_max_rel_linf": max(o32),
                          "fp64_gpu_max_rel_linf": max(o64), "seconds": t_oracle,
                          "how": "the 32 most non-square grids and 32 spread by cell count; "
                                 "oracle on the same FP32-rounded inputs, 200 steps"},
        "conservation_drift_fp32": drift,
        "sensitivity_above_1e-4": {
            "how": "for each instance above 1e-4 (up to 90 s of oracle time): the FP32 and FP64 GPU "
                   "results against the oracle, the oracle against itself from an initial state "
                   "perturbed by 1e-15 relative, and the oracle with its state rounded to FP32 after "
                   "every step against the plain oracle",
            "instances": len(sens), "seconds": t_sens,
            "fp32_within_3x_of_oracle_self_sensitivity": sum(
                1 for e in sens if e["fp32_vs_oracle"] <= 3 * max(1e-4, e["oracle_vs_oracle_perturbed_1e-15"])),
            "fp32_within_3x_of_fp32_state_floor": sum(
                1 for e in sens if e["fp32_vs_oracle"] <= 3 * max(1e-4, e["oracle_fp32_state_vs_oracle"])),
            "cases": sens[:12]},
        "compensated_on_worst": comp,
        "worst_shape": "%dx%d" % (wi.nx, wi.ny),
    }
    fp64 = {"workload": "the same 512-instance batch with FP64 state and coefficients, one 200-step call",
            "value": rate64, "unit": UNIT, "ms_per_call": ms64,
            "achieved_GBs": 64 * cell_steps / (ms64 * 1e-3) / 1e9,
            "frac": 64 * cell_steps / (ms64 * 1e-3) / 1e9 / peak, "peak_source": note,
            "bytes_per_cell_step": 64,
            "bound": "FP64 arithmetic (GB300's FP64 rate), not HBM",
            "fp32_speedup": None}
    return acc, fp64


def batch_diagnostics(P, torch, batch, handles, Ts, insts, dts):
    """The fused per-step diagnostics (ANISO_OPT_DIAGNOSTICS) on the bench
    batch: one 200-step call from the initial state with them and one
    without (CUDA events, graphs built beforehand), their cost, and what they
    record: the largest per-step conservation drift of the FP32 sum and the
    paper's relative non-monotonicity (Section 3.1: (min T0 - min T) / min T0
    over the call) of every instance."""
    import numpy as np
    T0 = [_w32(i.T0) for i in insts]
    nst = [STEPS_PER_CALL] * len(insts)
    stream = torch.cuda.current_stream()

    def reset():
        for t, a in zip(Ts, T0):
            t.copy_(torch.from_numpy(a.astype(np.float32)))

    def timed():
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.aniso_step_batched(batch, Ts, dts, nst)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {}
    try:
        P.aniso_set_option(handles[0], P.ANISO_OPT_DIAGNOSTICS, 1)
        reset()
        P.aniso_step_batched(batch, Ts, dts, nst)  # graph with the diagnostics
        ms_on = min(timed(), timed())
        ring = P.aniso_batch_diagnostics(batch, len(insts))
    finally:
        P.aniso_set_option(handles[0], P.ANISO_OPT_DIAGNOSTICS, 0)
    reset()
    P.aniso_step_batched(batch, Ts, dts, nst)
    ms_off = min(timed(), timed())
    s0 = np.array([a.sum() for a in T0])
    m0 = np.array([a.min() for a in T0])
    drift = np.nanmax(np.abs(ring[:, :, 0] - s0[:, None]) / np.abs(s0[:, None]), axis=1)
    nonmono = (m0 - np.nanmin(ring[:, :, 1], axis=1)) / m0
    out.update({
        "ms_per_call_with": ms_on, "ms_per_call_without": ms_off, "cost_frac": ms_on / ms_off - 1.0,
        "steps_recorded": int(np.isfinite(ring[:, :, 0]).sum()),
        "conservation_drift_fp32_max_any_step": float(drift.max()),
        "rel_nonmonotonicity": {"max": float(nonmono.max()), "median": float(np.median(nonmono)),
                                "instances_below_initial_min": int((nonmono > 0).sum())},
        "how": "sum, min and max of T after every step of every instance, formed in the y-update "
               "kernel, one read per call"})
    return out


def fp64_plain_compare(P, torch):
    """Plain FP64 single instance on the GPU: the 50x50 ring workload, 250
    steps, for the FP32-batched vs plain-FP64 comparison."""
    import numpy as np
    import oracle as O
    import workloads as W
    inst = W.ring_instance(50)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        bx = torch.tensor(inst.bx, dtype=torch.float64, device="cuda")
        by = torch.tensor(inst.by, dtype=torch.float64, device="cuda")
        P.aniso_set_field(h, bx, by)
        T = torch.tensor(inst.T0, dtype=torch.float64, device="cuda")
        P.aniso_step(h, T, inst.dt, inst.nsteps)
        P.aniso_sync(h)
        got = T.cpu().numpy()
        ref = O.step(inst.T0, O.face_coeffs(inst.bx, inst.by, 0, inst.chi_par), 0, inst.dt, inst.dx,
                     inst.dy, inst.chi_par, nsteps=inst.nsteps)
        err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        reps = 20
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            P.aniso_step(h, T, inst.dt, inst.nsteps)
        P.aniso_sync(h)
        el = time.perf_counter() - t0
        return {"value": inst.cells * inst.nsteps * reps / el / 1e9, "unit": UNIT,
                "workload": "ring 50x50 FP64 single instance, 250 steps (graph replay)",
                "rel_linf_vs_oracle": err}
    finally:
        P.aniso_destroy(h)


def fp32_single(P, torch):
    """The 4096^2 periodic random-field grid (|k| <= 8, 16 Gaussians, chi_par
    0.05, dt = 100 x the explicit limit), FP32, 100 steps through aniso_step on
    one handle: rate, rel L-inf against the FP64 oracle's full run, and the
    drift of the FP64 sum of T."""
    import numpy as np
    import oracle as O
    import workloads as W
    inst = W.random_instance(4096, 4096, dt_factor=100.0, nsteps=100)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
        by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
        P.aniso_set_field(h, bx, by)
        T0 = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
        T = T0.clone()
        P.aniso_step(h, T, inst.dt, inst.nsteps)  # builds the graph; warm-up
        T.copy_(T0)
        s0 = P.aniso_total(h, T)[0]
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.aniso_step(h, T, inst.dt, inst.nsteps)
        e1.record()
        P.aniso_sync(h)
        ms = e0.elapsed_time(e1)
        s1 = P.aniso_total(h, T)[0]
        got = T.double().cpu().numpy()
    finally:
        P.aniso_destroy(h)
    # the same grid with FP64 state and coefficients (FP32-rounded inputs widened)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP64)
        bx = torch.tensor(_w32(inst.bx), dtype=torch.float64, device="cuda")
        by = torch.tensor(_w32(inst.by), dtype=torch.float64, device="cuda")
        P.aniso_set_field(h, bx, by)
        T0d = torch.tensor(_w32(inst.T0), dtype=torch.float64, device="cuda")
        Td = T0d.clone()
        P.aniso_step(h, Td, inst.dt, inst.nsteps)  # builds the graph
        P.aniso_sync(h)
        got64 = Td.cpu().numpy()
        Td.copy_(T0d)
        torch.cuda.synchronize()
        e0.record()
        P.aniso_step(h, Td, inst.dt, inst.nsteps)
        e1.record()
        P.aniso_sync(h)
        ms64 = e0.elapsed_time(e1)
    finally:
        P.aniso_destroy(h)
    co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par)
    ref = O.step(_w32(inst.T0), co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=inst.nsteps)
    peak, note = measured_peak()
    out = {"workload": "random field 4096^2, FP32, 100 steps, one handle", "unit": UNIT,
           "value": inst.cells * inst.nsteps / (ms * 1e-3) / 1e9,
           "bytes_per_cell_step": 32,
           "frac": 32 * inst.cells * inst.nsteps / (ms * 1e-3) / 1e9 / peak, "peak_source": note,
           "rel_linf_vs_fp64_oracle": _rel_linf(got, ref),
           "conservation_drift_fp32": abs(s1 - s0) / abs(s0)}
    fp64 = {"workload": "random field 4096^2, FP64 state and coefficients, 100 steps, one handle",
            "unit": UNIT, "value": inst.cells * inst.nsteps / (ms64 * 1e-3) / 1e9,
            "rel_linf_vs_fp64_oracle": _rel_linf(got64, ref)}
    return out, fp64


def big_single(P, torch):
    """The largest single grid: 16384^2 periodic random field (|k| <= 32,
    16 Gaussians), chi_par 1, dt = 1000 x the explicit limit, 50 steps, FP32
    state with the compensated (hi, lo) update and FP16 face coefficients,
    through aniso_step on one handle: rate, the fraction of HBM at the
    variant's 40 B per cell-step, and rel L-inf of hi + lo against the FP64
    oracle's full run on the same FP16-rounded coefficients."""
    import numpy as np
    import oracle as O
    import workloads as W
    n, nsteps = 16384, 50
    inst = W.random_instance(n, n, kmax=32, chi_par=1.0, dt_factor=1000.0, nsteps=nsteps)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        P.aniso_set_option(h, P.ANISO_OPT_FIELD_FP16, 1)
        P.aniso_set_option(h, P.ANISO_OPT_KAHAN, 1)
        bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
        by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
        P.aniso_set_field(h, bx, by)
        del bx, by
        T0 = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
        T = T0.clone()
        P.aniso_step(h, T, inst.dt, nsteps)  # builds the graph; its result is the accuracy sample
        P.aniso_sync(h)
        lo = torch.empty_like(T)
        P.aniso_get_state(h, lo)
        torch.cuda.synchronize()
        got = T.double().cpu().numpy() + lo.double().cpu().numpy()
        del lo
        T.copy_(T0)
        P.aniso_set_state(h, 0, None)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.aniso_step(h, T, inst.dt, nsteps)
        e1.record(stream)
        P.aniso_sync(h)
        ms = e0.elapsed_time(e1)
    finally:
        P.aniso_destroy(h)
    del T, T0
    torch.cuda.empty_cache()
    cell_steps = inst.cells * nsteps
    peak, note = measured_peak()
    achieved = 40 * cell_steps / (ms * 1e-3) / 1e9
    t0 = time.perf_counter()
    co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par).rounded(np.float16)
    ref = O.step(_w32(inst.T0), co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=nsteps)
    t_or = time.perf_counter() - t0
    return {"workload": "random field 16384^2 (|k| <= 32), chi_par 1, dt 1000 x CFL, FP32 hi+lo state, "
                        "FP16 face coefficients, 50 steps, one handle", "unit": UNIT,
            "value": cell_steps / (ms * 1e-3) / 1e9, "ms_per_call": ms,
            "bytes_per_cell_step": 40, "achieved_GBs": achieved, "frac": achieved / peak,
            "peak_source": note,
            "rel_linf_vs_fp64_oracle": _rel_linf(got, ref),
            "oracle": "full 50-step FP64 run on the FP16-rounded coefficients, %.0f s" % t_or}


def nonlinear_single(P, torch):
    """The temperature-dependent diffusivity (Section 3.3: chi_par (T/t_ref)^2.5,
    harmonic face average): one 1024^2 periodic random-field grid, FP32, 100
    steps at dt = 10 x the explicit limit of chi_par, with its rel L-inf
    against the FP64 oracle's full run."""
    import numpy as np
    import oracle as O
    import workloads as W
    inst = W.random_instance(1024, 1024, dt_factor=10.0, nsteps=100)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    try:
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        P.aniso_set_nonlinear(h, 2.5, 1.0)
        bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
        by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
        P.aniso_set_field(h, bx, by)
        T0 = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
        T = T0.clone()
        P.aniso_step(h, T, inst.dt, inst.nsteps)  # builds the graph; warm-up
        T.copy_(T0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        P.aniso_step(h, T, inst.dt, inst.nsteps)
        e1.record()
        P.aniso_sync(h)
        ms = e0.elapsed_time(e1)
        got = T.double().cpu().numpy()
    finally:
        P.aniso_destroy(h)
    w = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    co = O.face_coeffs(w(inst.bx), w(inst.by), inst.bc, inst.chi_par)
    ref = O.step_nl(w(inst.T0), co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, 2.5, t_ref=1.0,
                    nsteps=inst.nsteps)
    return {"workload": "random field 1024^2, chi_par (T/1)^2.5, FP32, 100 steps, one handle", "unit": UNIT,
            "value": inst.cells * inst.nsteps / (ms * 1e-3) / 1e9,
            "rel_linf_vs_fp64_oracle": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))}


def explicit_speedup(P, torch):
    """The paper's speed-up claim (Section 3.1: the semi-implicit step at ncfl
    = 1000 against the explicit method at ncfl = 1): time to reach t = 20 on
    the 512^2 ring (T 10 / 0.1), FP32, both through aniso_step on the GPU."""
    import workloads as W
    inst = W.ring_instance(512, t_hot=10.0, t_cold=0.1, chi_par=0.01, dt_factor=1.0)
    t_end = 20.0
    out = {"workload": "ring 512^2, T 10/0.1, chi_par 0.01, zero-flux, FP32, t = 0 -> 20"}
    for name, scheme, ncfl in (("explicit", P.ANISO_SCHEME_EXPLICIT, 1.0),
                               ("semi_implicit", P.ANISO_SCHEME_2STEP, 1000.0)):
        dt = ncfl * inst.dx ** 2 / (4 * inst.chi_par)  # Eq. ncfl
        nsteps = int(round(t_end / dt))
        h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
        try:
            P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
            P.aniso_set_option(h, P.ANISO_OPT_SCHEME, scheme)
            bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
            by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
            P.aniso_set_field(h, bx, by)
            T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
            chunk = min(nsteps, 1000)
            P.aniso_step(h, T.clone(), dt, chunk)  # builds the graph
            T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            done = 0
            e0.record()
            while done < nsteps:
                k = min(chunk, nsteps - done)
                P.aniso_step(h, T, dt, k)
                done += k
            e1.record()
            P.aniso_sync(h)
            ms = e0.elapsed_time(e1)
            _, lo, hi, _ = P.aniso_total(h, T)
            out[name] = {"ncfl": ncfl, "steps": nsteps, "ms": ms, "min_T": lo, "max_T": hi,
                         "Gcell_steps_per_s": inst.cells * nsteps / (ms * 1e-3) / 1e9}
        finally:
            P.aniso_destroy(h)
    out["speedup"] = out["explicit"]["ms"] / out["semi_implicit"]["ms"]
    return out


# ------------------------------------------------------ three-dimensional workload

W3_N = 256
W3_STEPS_PER_CALL = 200
W3_BYTES_PER_CELL_SWEEP = 20  # FP32: read T (4) + three face coefficients (12) + write T (4)
WORKLOAD3 = ("one periodic 256^3 grid of the 3-D split (Section 2.1): b = B/|B|, B = z-hat + curl A "
             "for a random vector potential (1 <= |k| <= 3), T = 1 + 16 Gaussians, FP32, 2-step "
             "x,y,z updates, dt = 10 x min(dx)^2/(2 chi), 200 steps per call")


def make_instance3d(rank=0):
    import workloads as W
    return W.random_instance3d(W3_N, W3_N, W3_N, seed=W.BASE_SEED + rank, dt_factor=10.0,
                               nsteps=W3_STEPS_PER_CALL)


def setup_3d(P, torch, inst):
    h = P.aniso3_create(inst.nx, inst.ny, inst.nz, inst.dx, inst.dy, inst.dz, inst.chi_par,
                        inst.chi_perp, inst.bc)
    P.aniso3_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
    b = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in (inst.bx, inst.by, inst.bz)]
    P.aniso3_set_field(h, *b)
    T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    return h, T


def time_3d(P, torch, h, T, inst, steps, warmup, clocks_gpu=None):
    """Device time of `steps` aniso3_step calls after `warmup` calls.  The
    step is three launches of the same line kernel over the same number of
    cells, so a launch's average duration is the step time / 3."""
    for _ in range(warmup):
        P.aniso3_step(h, T, inst.dt, inst.nsteps)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = Clocks(clocks_gpu) if clocks_gpu is not None else None
    if clk:
        clk.__enter__()
    e0.record(stream)
    for _ in range(steps):
        P.aniso3_step(h, T, inst.dt, inst.nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    ms_call = e0.elapsed_time(e1) / steps
    return ms_call, ms_call / (3 * inst.nsteps), (clk.summary() if clk else None)


def cpu_baseline_3d(inst, budget_s=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the 3-D workload:
    whole steps of the full grid until the time budget is used."""
    import numpy as np
    import oracle as O
    w = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    co = O.face_coeffs3(w(inst.bx), w(inst.by), w(inst.bz), inst.bc, inst.chi_par)
    T = w(inst.T0)
    t0 = time.perf_counter()
    k = 0
    while True:
        T = O.step3(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.dz, inst.chi_par, nsteps=1)
        k += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": inst.cells * k / el / 1e9, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d full steps of the %dx%dx%d grid, FP64, %.1f s" % (k, inst.nx, inst.ny, inst.nz, el)}


def summary_3d(P, torch):
    """Short live measurement of the 3-D workload for the default line."""
    inst = make_instance3d()
    h, T = setup_3d(P, torch, inst)
    try:
        ms_call, launch_ms, _ = time_3d(P, torch, h, T, inst, steps=3, warmup=3)
    finally:
        P.aniso3_destroy(h)
    peak, note = measured_peak()
    achieved = W3_BYTES_PER_CELL_SWEEP * inst.cells / (launch_ms * 1e-3) / 1e9
    return {"workload": WORKLOAD3, "value": inst.cells * inst.nsteps / (ms_call * 1e-3) / 1e9, "unit": UNIT,
            "avg_launch_ms": launch_ms, "achieved_GBs": achieved, "frac": achieved / peak,
            "peak_source": note, "traffic": ncu_traffic("sweep3d"),
            "algorithmic_bytes_per_launch": W3_BYTES_PER_CELL_SWEEP * inst.cells}


def main_3d(args):
    """bench.py --workload random3d: one JSON line for the 3-D workload (one
    bench step = one aniso3_step call of 200 steps)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1008_0861_gb300 as P
    P.load()
    inst = make_instance3d(rank)
    h, T = setup_3d(P, torch, inst)
    T0 = T.clone()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms_call, launch_ms, clocks = time_3d(P, torch, h, T, inst, args.steps, args.warmup, clocks_gpu=local)
    cell_steps = inst.cells * inst.nsteps
    value, ms_step, _ = job_throughput(cell_steps, ms_call, "cuda")

    # end to end: pinned host T in, one call, host T out
    host = torch.empty(T.shape, dtype=torch.float32, pin_memory=True)
    host.copy_(T)
    stream = torch.cuda.current_stream()
    e2e_steps = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        T.copy_(host, non_blocking=True)
        P.aniso3_step(h, T, inst.dt, inst.nsteps)
        host.copy_(T, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, _, _ = job_throughput(cell_steps, e0.elapsed_time(e1) / e2e_steps, "cuda")

    peak, note = measured_peak()
    achieved = W3_BYTES_PER_CELL_SWEEP * inst.cells / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": "Gcell-steps/s, 3-D split step (Section 2.1), FP32; % HBM peak", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD3, "cells_per_gpu": inst.cells, "steps_per_call": inst.nsteps,
                   "l2": "inputs larger than L2: %.2f GB resident per GPU (T, 2 intermediates, 9 "
                         "coefficient arrays)" % (inst.cells * 4 * 12 / 1e9),
                   "parallelism": "one independent grid per GPU (no collective)"},
        "roofline": {"bound": "hbm", "kernel": "sweep3d", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": note, "traffic": ncu_traffic("sweep3d"),
                     "algorithmic_bytes_per_launch": W3_BYTES_PER_CELL_SWEEP * inst.cells,
                     "avg_launch_ms": launch_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": inst.cells * 4,
                "d2h_bytes_per_step": inst.cells * 4},
        "clocks": clocks,
        "gpu_launches": 3 * inst.nsteps * args.steps,
    }
    if rank == 0:
        import oracle as O
        w = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
        t = T0.clone()
        P.aniso3_step(h, t, inst.dt, 1)
        P.aniso3_sync(h)
        co = O.face_coeffs3(w(inst.bx), w(inst.by), w(inst.bz), inst.bc, inst.chi_par)
        ref = O.step3(T0.double().cpu().numpy(), co, inst.bc, inst.dt, inst.dx, inst.dy, inst.dz,
                      inst.chi_par, nsteps=1)
        got = t.double().cpu().numpy()
        line["accuracy"] = {"rel_linf_vs_fp64_oracle": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
                            "sample": "the whole grid after one step"}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_3d(inst)
        print(json.dumps(line), flush=True)
    P.aniso3_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_reference_3d(args):
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    inst = make_instance3d()
    budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline_3d(inst, budget_s=0.1)
    runs = [cpu_baseline_3d(inst, budget_s=budget) for _ in range(args.steps)]
    v = statistics.median(r["value"] for r in runs)
    line = {"impl": "reference", "metric": "Gcell-steps/s, 3-D split step (Section 2.1), FP32; % HBM peak",
            "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": inst.cells * inst.nsteps / (v * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD3},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": runs[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------ one large 2-D grid

WS_N = 4096
WS_STEPS = 100
WORKLOAD_SINGLE = ("one periodic 4096^2 random-field grid (|k| <= 8, 16 Gaussians), chi_par 0.05, dt = 100 x "
                   "the explicit limit, FP32 state and coefficients, 100 steps per call through aniso_step")


def make_single(rank=0):
    import workloads as W
    return W.random_instance(WS_N, WS_N, seed=W.BASE_SEED + rank, dt_factor=100.0, nsteps=WS_STEPS)


def main_single(args):
    """bench.py --workload random4096: one JSON line for the 4096^2 grid (one
    bench step = one aniso_step call of 100 steps; both updates run the
    cluster kernel (2-block clusters), whose launches are timed with CUDA
    events)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1008_0861_gb300 as P
    P.load()
    inst = make_single(rank)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
    if args.cluster_lines >= 0:
        P.aniso_set_option(h, P.ANISO_OPT_CLUSTER_LINES, args.cluster_lines)
    bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
    by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
    P.aniso_set_field(h, bx, by)
    del bx, by
    T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            P.aniso_step(h, T, inst.dt, inst.nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_call = e0.elapsed_time(e1) / args.steps
    # per-launch durations: one more call with CUDA events around every launch
    P.aniso_set_option(h, P.ANISO_OPT_PROFILE, 1)
    P.aniso_step(h, T, inst.dt, inst.nsteps)  # graph with the timing events
    P.aniso_sync(h)
    P.aniso_kernel_times(h=h, kind=0, reset=True)
    P.aniso_kernel_times(h=h, kind=1, reset=True)
    P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    kt = {k: P.aniso_kernel_times(h=h, kind=k) for k in (0, 1)}
    P.aniso_set_option(h, P.ANISO_OPT_PROFILE, 0)
    P.aniso_step(h, T, inst.dt, inst.nsteps)  # the plain graph again, before the e2e region
    P.aniso_sync(h)
    cell_steps = inst.cells * inst.nsteps
    value, ms_step, _ = job_throughput(cell_steps, ms_call, "cuda")
    # e2e: pinned host T in, one call, host T out
    host = torch.empty(T.shape, dtype=torch.float32, pin_memory=True)
    host.copy_(T)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(max(1, min(3, args.steps))):
        T.copy_(host, non_blocking=True)
        P.aniso_step(h, T, inst.dt, inst.nsteps)
        host.copy_(T, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, _, _ = job_throughput(cell_steps, e0.elapsed_time(e1) / max(1, min(3, args.steps)), "cuda")
    peak, note = measured_peak()
    names = {0: "xsweep", 1: "ysweep"}
    dom = max(kt, key=lambda k: kt[k][0])
    launch_ms = kt[dom][0] / max(1, kt[dom][1])
    achieved = BYTES_PER_CELL_SWEEP * inst.cells / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": "Gcell-steps/s, one 4096^2 FP32 grid; % HBM peak", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_SINGLE, "cells_per_gpu": inst.cells, "steps_per_call": inst.nsteps,
                   "l2": "inputs larger than L2: %.2f GB resident (T, T*, 4 coefficient arrays, 2 transposed)"
                         % (inst.cells * 4 * 8 / 1e9),
                   "parallelism": "one independent grid per GPU (no collective)"},
        "roofline": {"bound": "hbm", "kernel": ("line6_" if args.cluster_lines == 1 else "line7_") + names[dom],
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": note,
                     "traffic": ncu_traffic("line6_4096" if args.cluster_lines == 1 else "line7_4096"),
                     "algorithmic_bytes_per_launch": BYTES_PER_CELL_SWEEP * inst.cells, "avg_launch_ms": launch_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": inst.cells * 4,
                "d2h_bytes_per_step": inst.cells * 4},
        "clocks": clk.summary(),
        "gpu_launches": 2 * inst.nsteps * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.aniso_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


WC_STEPS = 50
WC_BYTES_PER_CELL_SWEEP = 20  # read hi + lo (8) + two FP16 face coefficients (4) + write hi + lo (8)


def compensated_shape(args):
    nx, ny = (int(v) for v in args.shape.lower().split("x"))
    return nx, ny


def make_compensated(nx, ny, rank=0):
    import workloads as W
    return W.random_instance(nx, ny, seed=W.BASE_SEED + rank, kmax=32, chi_par=1.0, dt_factor=1000.0,
                             nsteps=WC_STEPS)


def workload_compensated(nx, ny):
    return ("one periodic %dx%d random-field grid (|k| <= 32, 16 Gaussians), chi_par 1, dt = 1000 x the "
            "explicit limit, FP32 hi+lo (compensated) state, FP16 face coefficients, %d steps per call "
            "through aniso_step" % (nx, ny, WC_STEPS))


def main_compensated(args):
    """bench.py --workload compensated: one JSON line for one compensated-state
    grid (the 16384^2 configuration by default).  One bench step = one
    aniso_step call of 50 steps; both updates run the cluster kernel, whose
    launches are timed with CUDA events."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1008_0861_gb300 as P
    P.load()
    nx, ny = compensated_shape(args)
    inst = make_compensated(nx, ny, rank)
    h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
    P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
    P.aniso_set_option(h, P.ANISO_OPT_FIELD_FP16, 1)
    P.aniso_set_option(h, P.ANISO_OPT_KAHAN, 1)
    bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
    by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
    P.aniso_set_field(h, bx, by)
    del bx, by
    T = torch.tensor(inst.T0, dtype=torch.float32, device="cuda")
    s0 = P.aniso_total(h, T)[0]
    for _ in range(args.warmup):
        P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            P.aniso_step(h, T, inst.dt, inst.nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_call = e0.elapsed_time(e1) / args.steps
    s1 = P.aniso_total(h, T)[0]
    # per-launch durations: one more call with CUDA events around every launch
    P.aniso_set_option(h, P.ANISO_OPT_PROFILE, 1)
    P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    P.aniso_kernel_times(h=h, kind=0, reset=True)
    P.aniso_kernel_times(h=h, kind=1, reset=True)
    P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    kt = {k: P.aniso_kernel_times(h=h, kind=k) for k in (0, 1)}
    P.aniso_set_option(h, P.ANISO_OPT_PROFILE, 0)
    P.aniso_step(h, T, inst.dt, inst.nsteps)
    P.aniso_sync(h)
    cell_steps = inst.cells * inst.nsteps
    value, ms_step, _ = job_throughput(cell_steps, ms_call, "cuda")
    # e2e: pinned host T (the hi part) in, one call, host T out; the low parts
    # stay with the handle on the device
    host = torch.empty(T.shape, dtype=torch.float32, pin_memory=True)
    host.copy_(T)
    torch.cuda.synchronize()
    reps = max(1, min(3, args.steps))
    e0.record(stream)
    for _ in range(reps):
        T.copy_(host, non_blocking=True)
        P.aniso_step(h, T, inst.dt, inst.nsteps)
        host.copy_(T, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, _, _ = job_throughput(cell_steps, e0.elapsed_time(e1) / reps, "cuda")
    peak, note = measured_peak()
    names = {0: "xsweep", 1: "ysweep"}
    dom = max(kt, key=lambda k: kt[k][0])
    launch_ms = kt[dom][0] / max(1, kt[dom][1])
    achieved = WC_BYTES_PER_CELL_SWEEP * inst.cells / (launch_ms * 1e-3) / 1e9
    line = {
        "metric": "Gcell-steps/s, one compensated FP32 grid (hi+lo state, FP16 coefficients); % HBM peak",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 hi+lo", "data": "synthetic",
        "config": {"workload": workload_compensated(nx, ny), "cells_per_gpu": inst.cells,
                   "steps_per_call": inst.nsteps,
                   "l2": "inputs larger than L2: %.2f GB resident" % (inst.cells * 4 * 10 / 1e9),
                   "parallelism": "one independent grid per GPU (no collective)"},
        "roofline": {"bound": "hbm", "kernel": "line7k_" + names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": note,
                     "traffic": ncu_traffic("line7k_%dx%d" % (nx, ny)),
                     "algorithmic_bytes_per_launch": WC_BYTES_PER_CELL_SWEEP * inst.cells,
                     "avg_launch_ms": launch_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": inst.cells * 4,
                "d2h_bytes_per_step": inst.cells * 4},
        "conservation_drift": abs(s1 - s0) / abs(s0),
        "clocks": clk.summary(),
        "gpu_launches": 2 * inst.nsteps * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.aniso_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_reference_compensated(args):
    """The FP64 oracle on the compensated workload's grid (the same FP16-rounded
    coefficients): whole steps until the time budget."""
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle as O
    nx, ny = compensated_shape(args)
    inst = make_compensated(nx, ny)
    co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par).rounded(np.float16)
    budget = max(5.0, 120.0 / max(1, args.steps + args.warmup))
    T = _w32(inst.T0)
    vals, ms = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < budget:
            T = O.step(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1)
            n += 1
        el = time.perf_counter() - t0
        if k >= args.warmup:
            vals.append(inst.cells * n / el / 1e9)
            ms.append(el * 1e3)
    v = statistics.median(vals)
    line = {"impl": "reference",
            "metric": "Gcell-steps/s, one compensated FP32 grid (hi+lo state, FP16 coefficients); % HBM peak",
            "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_compensated(nx, ny)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "whole FP64 steps of the grid for %.0f s per bench step" % budget},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_single(args):
    """The FP64 oracle on the 4096^2 grid: whole steps until the time budget."""
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle as O
    inst = make_single()
    co = O.face_coeffs(_w32(inst.bx), _w32(inst.by), inst.bc, inst.chi_par)
    budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    T = _w32(inst.T0)
    vals, ms = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < budget:
            T = O.step(T, co, inst.bc, inst.dt, inst.dx, inst.dy, inst.chi_par, nsteps=1)
            n += 1
        el = time.perf_counter() - t0
        if k >= args.warmup:
            vals.append(inst.cells * n / el / 1e9)
            ms.append(el * 1e3)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "Gcell-steps/s, one 4096^2 FP32 grid; % HBM peak", "value": v,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(ms), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD_SINGLE},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": "whole steps of the 4096^2 grid for %.0f s per bench step" % budget},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        if args.workload == "random3d":
            return run_reference_3d(args)
        if args.workload == "random4096":
            return run_reference_single(args)
        if args.workload == "compensated":
            return run_reference_compensated(args)
        return run_reference(args)
    if args.workload == "random3d":
        return main_3d(args)
    if args.workload == "random4096":
        return main_single(args)
    if args.workload == "compensated":
        return main_compensated(args)
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1008_0861_gb300 as P
    import oracle as O

    P.load()
    insts = make_instances(args.instances, rank)
    handles, Ts, bufs = [], [], []
    for inst in insts:
        h = P.aniso_create(inst.nx, inst.ny, inst.dx, inst.dy, inst.chi_par, 0.0, inst.bc)
        P.aniso_set_option(h, P.ANISO_OPT_PRECISION, P.ANISO_PREC_FP32)
        if args.segment:
            P.aniso_set_option(h, P.ANISO_OPT_SEGMENT, args.segment)
        if args.fast >= 0:
            P.aniso_set_option(h, P.ANISO_OPT_FAST_PATH, args.fast)
        bx = torch.tensor(inst.bx, dtype=torch.float32, device="cuda")
        by = torch.tensor(inst.by, dtype=torch.float32, device="cuda")
        P.aniso_set_field(h, bx, by)
        Ts.append(torch.tensor(inst.T0, dtype=torch.float32, device="cuda"))
        handles.append(h)
        bufs.append((bx, by))
    # the sweeps of every PROFILE_EVERY-th step carry CUDA events (all steps run
    # the same launches; fewer event nodes in the timed graph)
    P.aniso_set_option(handles[0], P.ANISO_OPT_PROFILE, PROFILE_EVERY)
    if args.tma_lines >= 0:
        P.aniso_set_option(handles[0], P.ANISO_OPT_TMA_LINES, args.tma_lines)
    if args.tmem >= 0:
        P.aniso_set_option(handles[0], P.ANISO_OPT_TMEM, args.tmem)
    batch = P.aniso_batch_create(handles)
    P.aniso_set_option(handles[0], P.ANISO_OPT_PROFILE, 0)
    dts = [i.dt for i in insts]
    tuned = None
    if not args.no_tune and args.fast < 0 and not args.segment:
        # block shape (lines per block, PCR depth) by measurement, outside the timed region
        choice, tune_ms = P.aniso_batch_autotune(batch, Ts, dts, nsteps=2, reps=2)
        if choice >= 0:
            f, w, sc = P.aniso_autotune_candidate(choice)
            tuned = {"choice": choice, "fast_path": f, "warps_per_block": w, "chunks_per_lane": sc,
                     "ms_per_2_steps": tune_ms}
    nsteps = [STEPS_PER_CALL] * len(insts)
    cells = sum(i.cells for i in insts)
    cell_steps = cells * STEPS_PER_CALL
    torch.cuda.synchronize()
    del bufs

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        P.aniso_step_batched(batch, Ts, dts, nsteps)
    sync_all()
    P.aniso_kernel_times(batch=batch, kind=0, reset=True)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        sync_all()
        ev0.record(stream)
        for _ in range(args.steps):
            P.aniso_step_batched(batch, Ts, dts, nsteps)
        ev1.record(stream)
        sync_all()
    ms = ev0.elapsed_time(ev1)
    kt = {k: P.aniso_kernel_times(batch=batch, kind=k) for k in (0, 1)}
    value, ms_step, _ = job_throughput(cell_steps, ms / args.steps, "cuda")

    # end to end through the C ABI's host-buffer call: every step copies each
    # grid's T from page-locked host memory to the device, runs the batched
    # call and copies the result back (the call returns when the host arrays
    # hold it)
    host = [torch.empty(t.shape, dtype=torch.float32, pin_memory=True) for t in Ts]
    for hsrc, t in zip(host, Ts):
        hsrc.copy_(t)
    P.aniso_step_batched_host(batch, host, dts, nsteps)  # first call: the batch's device copies, graph
    e2e_steps = max(1, min(3, args.steps))
    sync_all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        P.aniso_step_batched_host(batch, host, dts, nsteps)
    e1.record(stream)
    sync_all()
    e2e_value, e2e_ms, _ = job_throughput(cell_steps, e0.elapsed_time(e1) / e2e_steps, "cuda")
    io_bytes = cells * 4
    del host

    # roofline of the dominant kernel (live CUDA-event durations over the timed region)
    names = {0: "xsweep", 1: "ysweep"}
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms, dom_n = kt[dom]
    achieved = BYTES_PER_CELL_SWEEP * cells / (dom_ms / dom_n * 1e-3) / 1e9 if dom_n else None
    peak, peak_note = measured_peak()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": len(insts), "cells_per_gpu": cells,
                   "steps_per_call": STEPS_PER_CALL,
                   "l2": "inputs larger than L2: %.2f GB resident per GPU (T, T*, 4 coefficient arrays)"
                         % (cells * 4 * 6 / 1e9),
                   "parallelism": "independent instances per GPU (no collective)",
                   "autotuned": tuned},
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak if achieved else None,
                     "peak_source": peak_note, "traffic": ncu_traffic(names[dom]) if args.instances == N_INST else None,
                     "algorithmic_bytes_per_launch": BYTES_PER_CELL_SWEEP * cells,
                     "avg_launch_ms": dom_ms / dom_n if dom_n else None,
                     "launches_timed": "the sweeps of every %dth step of each call (%d of %d steps)"
                                       % (PROFILE_EVERY, -(-STEPS_PER_CALL // PROFILE_EVERY), STEPS_PER_CALL),
                     "per_kernel_ms": {names[k]: kt[k][0] / max(1, kt[k][1]) for k in kt}},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "clocks": clk.summary(),
        "gpu_launches": P.aniso_batch_kernel_count(batch) * args.steps,
    }
    if rank == 0 and args.no_legs:
        print(json.dumps(line), flush=True)
    elif rank == 0:
        # accuracy of this workload on every instance, and its FP64 form
        acc, fp64b = batch_accuracy(P, torch, batch, Ts, insts, dts)
        fp64b["fp32_speedup"] = value / fp64b["value"]
        line["accuracy"] = acc
        line["fp64_batch"] = fp64b
        line["diagnostics"] = batch_diagnostics(P, torch, batch, handles, Ts, insts, dts)
        line["fp64_plain"] = fp64_plain_compare(P, torch)
        line["speedup_vs_explicit"] = explicit_speedup(P, torch)
        line["fp32_single"], line["fp64_single"] = fp32_single(P, torch)
        if not args.no_big:
            line["big_single"] = big_single(P, torch)
        line["nonlinear_chi"] = nonlinear_single(P, torch)
        line["three_d"] = summary_3d(P, torch)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(insts, single_thread_s=4.0)
        print(json.dumps(line), flush=True)
    P.aniso_batch_destroy(batch)
    for h in handles:
        P.aniso_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
