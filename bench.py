"""Benchmark of the GB300 GP-SPCA hot path (one JSON line on rank 0).

Headline workload (the largest single-GPU configuration): A is 20000 x
100000 FP32 (p samples x n variables, 8 GB) = N(0,1) noise + sum_{j<=16}
(100/sqrt j) u_j v_j^T with 1% disjoint Rademacher supports; gamma = 0.05
max||a_i|| (L1) and (0.05 max||a_i||)^2 (L0), scaled on the device.  One step
= four full solves on that A (setup, power iterations to tol 1e-6,
loadings): SL1, SL0, and BL1, BL0 with m = 16 components at mu = 1.  Metric:
power iterations (sweeps) per second over the step.  The line also carries
the 5000 x 20000 step (six solves, block m = 5) under "spikes_5000x20000".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs independent replicas (one process per GPU under torchrun).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# headline: 20000 x 100000 fp32, 16 spikes
P4, N4, M4 = 20000, 100000, 16
CASES4 = [("SL1", None), ("SL0", None), ("BL1", [1.0] * M4), ("BL0", [1.0] * M4)]
# the oracle's bounded sample: noise block 0 of 16 (columns 0..6249, all
# 20000 rows); its time per sweep is scaled by n / 6250 = 16
SAMPLE_BLOCKS = (0, 1)
SAMPLE_COLS = 6250
# secondary: 5000 x 20000 fp32, 5 spikes
P, N, K_SPIKES = 5000, 20000, 5
RHO = 0.05
MU_W = [1.0, 0.9, 0.8, 0.7, 0.6]
CASES = [("SL1", None), ("SL0", None), ("BL1", [1.0] * 5), ("BL0", [1.0] * 5), ("BL1", MU_W), ("BL0", MU_W)]
TOL, MAXIT = 1e-6, 1000
RHO32 = 0.01
# dram bytes (read + write) per launch from ncu captures of the current
# kernels (dram__bytes_read.sum + dram__bytes_write.sum): the fused sweeps on
# the 5000 x 20000 matrix, and on the 20000 x 100000 matrix the tensor-core T
# pass and the whole block and single-unit threshold sweeps (their six
# kernels each); None where the kernels changed since the last capture
TRAFFIC_SL1 = 400.2e6
TRAFFIC_BL1 = 400.6e6
TRAFFIC_T4 = 8115.3e6
TRAFFIC_BLK4 = 9456.1e6
TRAFFIC_SU4 = 8173.1e6
METRIC = "GPower iters/s"
SERVING_SAMPLE = 1000  # requests of the serving mix run by the default benchmark
UNIT = "iters/s"
WORKLOAD4 = ("planted spikes 20000x100000 fp32 (16 spikes, theta_j=100/sqrt(j), 1% supports), SL1+SL0+BL1+BL0 "
             "(block m=16, mu=1), gamma=0.05*max||a_i||, tol 1e-6")
WORKLOAD = ("planted spikes 5000x20000 fp32 (5 spikes, theta_j=40/j, 5% supports), SL1+SL0+BL1+BL0 (m=5, mu=1 and "
            "mu=[1,.9,.8,.7,.6]), gamma=0.05*max||a_i||, tol 1e-6")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(ms, units, device="cpu"):
    """Replicas: the slowest rank's timed region and the units all ranks did.

    One process per GPU runs the whole step on its own copy of the workload
    (the solves share nothing, so nothing is exchanged on the data path); the
    job's time is the maximum over ranks and its work the sum."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t_max = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_sum = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_sum, op=dist.ReduceOp.SUM)
    return float(t_max.item()), float(t_sum.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sms.append(float(f[1]))
                    maxes.append(float(f[2]))
                except ValueError:
                    continue
                for name, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if sms:
            out["sm_mhz"] = statistics.median(sms)
            out["sm_max_mhz"] = max(maxes)
            out["samples"] = len(sms)
        out["reasons"] = sorted(reasons)
        return out


def _run_steps(ctx, stream, dA, hA, cases, p, n, steps, warmup, eager, host=False, label="gpspca_step"):
    """`steps` timed steps of the solves in `cases` (after `warmup` untimed
    ones), issued as one gpspca_solve_batch per step (the solves run
    concurrently on their own streams, ordered on the context's stream).
    host: end to end from the pinned host matrix hA, with the results
    written to pinned host buffers: each step's A is copied in by
    gpspca_upload into one of two device buffers, the copy for step k + 1
    issued before the solves of step k so that it overlaps them (the solves
    of step k + 1 wait for it on the device).
    Returns (ms, sweeps, kernel launches) over the timed steps."""
    import torch

    from paper_1312_6182_gb300 import binding

    outs, counts = [], []
    for form, mu in cases:
        m = 1 if mu is None else len(mu)
        outs.append(binding.alloc_result(m, p, n, "cpu" if host else "cuda", torch.float32, pin=host))
        counts.append(ctx.plan_launches(dA, form, [RHO] * m, mu=mu, gamma_relative=True))
    bufs = [torch.empty_like(dA), torch.empty_like(dA)] if host else None

    def step(k, last):
        if host:
            if k == 0:
                ctx.upload(hA, bufs[0])
            if k + 1 < last:
                ctx.upload(hA, bufs[(k + 1) % 2])
        items = []
        for (form, mu), out in zip(cases, outs):
            m = 1 if mu is None else len(mu)
            items.append(dict(At=bufs[k % 2] if host else dA, form=form, gamma=[RHO] * m, mu=mu, tol=TOL,
                              maxit=MAXIT, gamma_relative=True, out=out, eager=eager))
        results = [ctx.solve(**it) for it in items] if eager else ctx.solve_batch(items)
        # a batch computes the column norms of a matrix that two or more of its
        # single-unit solves share once (one launch), and those solves copy them
        # (one launch each, as their own norm pass would have been)
        sweeps = 0
        launches = 1 if not eager and sum(1 for f, _ in cases if f.startswith("S")) >= 2 else 0
        for res, (pro, per, epi) in zip(results, counts):
            it = int(res.iters.max().item())
            sweeps += it
            launches += pro + it * per + epi
        return sweeps, launches

    torch.cuda.synchronize()
    for k in range(warmup):
        step(k, warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    total_sweeps, total_launches = 0, 0
    # an NVTX range around the timed steps (profilers filter the step's
    # kernels with it, e.g. ncu --nvtx --nvtx-include "gpspca_step/")
    try:
        torch.cuda.nvtx.range_push(label)
        nvtx = True
    except Exception:
        nvtx = False
    ev0.record(stream)
    for k in range(steps):
        sw, la = step(k, steps)
        total_sweeps += sw
        total_launches += la
    ev1.record(stream)
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    del bufs
    return ev0.elapsed_time(ev1), total_sweeps, total_launches


def _roofline(ctx, dA, form, m, bytes_a, peak, peak_kind, kernel, traffic, t_pass=False):
    """The sweep of one iteration (or, with t_pass, the tensor-core sweep's T
    pass) timed alone (CUDA events on the library's stream,
    gpspca_time_sweep); algorithmic bytes = one read of A."""
    mu = [1.0] * m if form.startswith("B") else None
    ms = ctx.time_sweep(dA, form, [RHO] * m, mu=mu, gamma_relative=True, reps=20, t_pass=t_pass)
    ach = bytes_a / (ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
            "frac": round(ach / peak, 4), "peak_source": peak_kind, "traffic": traffic,
            "ms_per_launch": round(ms, 5), "algorithmic_bytes_per_launch": bytes_a}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()
    ctx = binding.Context(local, stream=stream)

    # ---- headline: 20000 x 100000 fp32, four solves per step
    At = synth.workload_spikes_20000x100000(2)
    dA = torch.from_numpy(At).cuda()
    hA = torch.from_numpy(At).pin_memory()
    del At
    if ws > 1:
        torch.distributed.barrier()
    clk = Clocks(local)
    clk.start()
    ms, sweeps, launches = _run_steps(ctx, stream, dA, hA, CASES4, P4, N4, args.steps, args.warmup, args.eager)
    clocks = clk.stop()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms, sweeps_all = reduce_over_ranks(ms, sweeps, "cuda")
    value = sweeps_all / (ms / 1e3)
    # end to end through the C ABI from host (pinned) buffers: every step's
    # A copied in (gpspca_upload, overlapping the previous step's solves)
    # and every result copied out inside the timed region
    e2e_steps = args.steps
    e2e_ms, e2e_sweeps, _ = _run_steps(ctx, stream, dA, hA, CASES4, P4, N4, e2e_steps, args.warmup, False, host=True,
                                       label="gpspca_step_e2e")
    # the host link alone: uploads of the matrix with nothing else running
    # (the copies run on the library's copy stream: timed on the host around
    # a device synchronisation)
    buf = torch.empty_like(dA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        ctx.upload(hA, buf)
    torch.cuda.synchronize()
    h2d_ms = (time.perf_counter() - t0) * 1e3 / 3
    del buf, hA
    h2d = P4 * N4 * 4
    d2h = sum((P4 + N4) * 4 * (1 if mu is None else len(mu)) + ((N4 + 31) // 32) * 4 * (1 if mu is None else len(mu))
              + 24 * (1 if mu is None else len(mu)) for _, mu in CASES4)
    bytes_a = P4 * N4 * 4
    # the kernels of the step: the T pass (T = A^T X on the tensor cores:
    # every sweep of every solve runs one, the block starts' three included;
    # the 20000-row single-unit solves run the tensor-core sweep too), and the
    # threshold sweeps as a whole (T pass, listing of the active columns,
    # rank update over them) of the block and the single-unit solves;
    # algorithmic bytes = one read of A per launch for each.  The T pass, by
    # its share of the step, is the roofline line.
    r_t = _roofline(ctx, dA, "BL1", M4, bytes_a, peak, peak_kind,
                    "tc_t_fused_kernel<48> (+ tc_prep, tc_t_combine): T = A^T X on tcgen05, float A split into exact "
                    "bf16 planes in tensor memory (the MMA's A operand)", TRAFFIC_T4, t_pass=True)
    r_blk = _roofline(ctx, dA, "BL1", M4, bytes_a, peak, peak_kind,
                      "block m=16 threshold sweep: tc_prep + tc_t_fused<48> + tc_t_combine + tc_count + "
                      "tc_compact + tc_y_fused<48> over the active columns", TRAFFIC_BLK4)
    r_su = _roofline(ctx, dA, "SL1", 1, bytes_a, peak, peak_kind,
                     "single-unit threshold sweep on the tensor cores: tc_prep + tc_t_fused<48> + tc_t_combine + "
                     "tc_count + tc_compact + tc_y_fused<48> over the active columns", TRAFFIC_SU4)
    its = _case_iters(ctx, dA, CASES4, P4, N4)
    # block: the start's two power steps and rotation step, and every sweep
    # but the first (its T comes from the rotation step's); single-unit: every sweep
    n_t = sum((2 + it) if f.startswith("B") else it for (f, _), it in zip(CASES4, its))
    step_ms = ms / args.steps
    r_t["launches_per_step"] = n_t
    r_t["share_of_step"] = round(n_t * r_t["ms_per_launch"] / step_ms, 3)
    r_blk["launches_per_step"] = sum(it for (f, _), it in zip(CASES4, its) if f.startswith("B"))
    r_su["launches_per_step"] = sum(it for (f, _), it in zip(CASES4, its) if f.startswith("S"))

    # ---- precision sample (rank 0, after the timed steps): BL1 / BL0 with
    # m = 16 on this matrix in FP32, and on its BF16 and FP8 copies + 3 FP32
    # refinement sweeps
    precision = None
    if rank == 0:
        pres, _, _, psw = _precision(ctx, stream, dA, P4, N4, RHO, 3, 2, 8)
        pbytes = {"f32": P4 * N4 * 4, "bf16": P4 * N4 * 2, "fp8": P4 * N4 + N4 * 4}
        precision = {
            "workload": "planted spikes 20000x100000 (16 spikes, theta_j=100/sqrt(j), 1% supports), BL1/BL0 m=16 "
                        f"mu=1, gamma={RHO:g}*max||a_i||; FP32 vs BF16 and FP8-E4M3 (per-column scales) storage + "
                        "3 FP32 refinement sweeps",
            "results": pres,
            "solves_per_s_vs_f32": {k: round(v["solves_per_s"] / pres[k.split("_")[0] + "_f32"]["solves_per_s"], 3)
                                    for k, v in pres.items() if not k.endswith("f32")},
            "sweeps_m16": {fmt: {"ms_per_sweep": round(v, 4),
                                 "frac": round(pbytes[fmt] / (v / 1e3) / 1e9 / peak, 4)} for fmt, v in psw.items()}}
    del dA
    torch.cuda.empty_cache()

    # ---- secondary: 5000 x 20000 fp32, six solves per step (block m = 5)
    At2 = synth.workload_spikes_5000x20000(0)
    dA2 = torch.from_numpy(At2).cuda()
    ms2, sweeps2, launches2 = _run_steps(ctx, stream, dA2, None, CASES, P, N, args.steps, args.warmup, args.eager,
                                         label="gpspca_step_5000x20000")
    ms2, sweeps2_all = reduce_over_ranks(ms2, sweeps2, "cuda")
    bytes2 = P * N * 4
    secondary = {
        "workload": WORKLOAD, "value": round(sweeps2_all / (ms2 / 1e3), 2), "unit": UNIT,
        "ms_per_step": round(ms2 / args.steps, 4), "sweeps_per_step": round(sweeps2 / args.steps, 2),
        "gpu_launches": launches2,
        "roofline": _roofline(ctx, dA2, "BL1", 5, bytes2, peak, peak_kind,
                              "sweep_kernel<float,5,3,0,6> (block m=5 fused sweep, 6-column tiles)", TRAFFIC_BL1),
        "roofline_single_unit": _roofline(ctx, dA2, "SL1", 1, bytes2, peak, peak_kind,
                                          "sweep_kernel<float,1,2,0,3> (single-unit fused sweep, 3-column tiles)",
                                          TRAFFIC_SL1),
    }
    del dA2
    torch.cuda.empty_cache()

    # ---- sparsity-path sample (rank 0): 64 gammas batched vs separate on a
    # 10000 x 50000 matrix, block L1 with m = 32
    gamma_path = None
    if rank == 0:
        dA3 = torch.from_numpy(synth.workload_spikes_10000x50000(1)).cuda()
        gres, ms_sw, ms_sw32, _ = _gamma_path(ctx, stream, dA3, 10000, 50000, 2, 4)
        gamma_path = {"workload": GAMMA_WORKLOAD, "results": gres, "ms_per_64_gamma_sweep": round(ms_sw, 4),
                      "frac_one_read": round(10000 * 50000 * 4 / (ms_sw / 1e3) / 1e9 / peak, 4),
                      "block_m32_sweep_ms": round(ms_sw32, 4)}
        del dA3
        torch.cuda.empty_cache()
    ctx.close()

    # ---- serving sample (rank 0, after the timed steps): the request mix of
    # the serving workload with SERVING_SAMPLE requests, for p50 / p99 at the
    # offered 200 requests/s beside the throughput
    serving = None
    if rank == 0:
        serving, _, _ = _serving(SERVING_SAMPLE, 3)
        serving = {"workload": f"serving mix: {SERVING_SAMPLE} requests, {SERVING_MIX}", **serving}
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD4, "p": P4, "n": N4, "m_block": M4, "solves_per_step": len(CASES4),
                   "sweeps_per_step": round(sweeps / args.steps, 2), "iters_per_case": its,
                   "l2": "inputs larger than L2 (A is 8 GB)", "parallelism": "replicas" if ws > 1 else "1 gpu"},
        "roofline": r_t,
        "roofline_block_sweep": r_blk,
        "roofline_single_unit_sweep": r_su,
        "e2e": {"value": round(e2e_sweeps / (e2e_ms / 1e3), 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms / e2e_steps, 3),
                "h2d_alone_gbs": round(h2d / (h2d_ms / 1e3) / 1e9, 1)},
        "gpu_launches": launches,
        "clocks": clocks,
        "spikes_5000x20000": secondary,
    }
    for key, val in (("precision_sample", precision), ("gamma_path_sample", gamma_path),
                     ("serving_sample", serving)):
        if val is not None:
            line[key] = val
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(ws)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def _case_iters(ctx, dA, cases, p, n):
    """Iterations of each case of the step (one solve each)."""
    its = []
    for form, mu in cases:
        m = 1 if mu is None else len(mu)
        r = ctx.solve(dA, form, [RHO] * m, mu=mu, tol=TOL, maxit=MAXIT, gamma_relative=True)
        its.append(int(r.iters.max().item()))
    return its


def _oracle_sample(A64, sweeps_per_case):
    """The oracle on a bounded sample of the headline workload (the columns
    of A64): every case of the step, a fixed number of sweeps each (tol = 0),
    gamma relative to the sample's largest column.  Returns (sweeps, seconds)."""
    import numpy as np

    import oracle

    t0 = time.perf_counter()
    done = 0
    for form, mu in CASES4:
        m = 1 if mu is None else len(mu)
        g = oracle.gamma_from_rho(A64, form, [RHO] * m)
        r = oracle.gpower(A64, form, g, mu=mu, tol=0.0, maxit=sweeps_per_case)
        done += int(np.max(r.iters))
    return done, time.perf_counter() - t0


def _sample64():
    import numpy as np

    from paper_1312_6182_gb300 import synth

    At = synth.workload_spikes_20000x100000(2, blocks=SAMPLE_BLOCKS)
    assert At.shape == (SAMPLE_COLS, P4)
    return At.astype(np.float64).T


SAMPLE_NOTE = (f"columns 0..{SAMPLE_COLS - 1} (noise block {SAMPLE_BLOCKS[0]} of 16, all "
               f"{P4} rows) of the 20000x100000 matrix; time per sweep scaled by n/{SAMPLE_COLS} = "
               f"{N4 // SAMPLE_COLS}")


def cpu_baseline(ws):
    if ws > 1 and _dist()[1] != 0:
        return None
    A64 = _sample64()
    sweeps, sec = _oracle_sample(A64, 2)
    scale = N4 / SAMPLE_COLS
    return {"value": round(sweeps / (sec * scale), 3), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{sweeps} sweeps: every case of the step, 2 sweeps each (tol=0), FP64 NumPy on the host, "
                      + SAMPLE_NOTE}


def run_reference(args):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    A64 = _sample64()
    for _ in range(args.warmup):
        _oracle_sample(A64, 1)
    total, sec = 0, 0.0
    for _ in range(args.steps):
        s, t = _oracle_sample(A64, 1)
        total += s
        sec += t
    scale = N4 / SAMPLE_COLS
    value = total / (sec * scale)
    sample = "every case of the step, 1 sweep each (tol=0), FP64 NumPy, " + SAMPLE_NOTE
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(sec * scale / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD4, "p": P4, "n": N4, "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sweep_only(args):
    """The fused sweep alone on one of the benchmark matrices (profiling
    entry): prints the mean time of one sweep and the algorithmic bandwidth."""
    import torch

    from paper_1312_6182_gb300 import binding, synth

    if args.sweep_matrix == "20000x100000":
        At, p, n = synth.workload_spikes_20000x100000(2), P4, N4
    elif args.sweep_matrix == "20000x25000":  # column blocks 0-3 of 16 of the 20000 x 100000 matrix (2 GB)
        At = synth.workload_spikes_20000x100000(2, blocks=(0, 4))
        p, n = At.shape[1], At.shape[0]
    else:
        At, p, n = synth.workload_spikes_5000x20000(0), P, N
    dA = torch.from_numpy(At).cuda()
    del At
    if args.sweep_dtype == "bf16":
        dA = dA.to(torch.bfloat16)
    form = args.sweep_only
    m = args.sweep_m or (1 if form.startswith("S") else 5)
    mu = [1.0] * m if form.startswith("B") else None
    with binding.Context(0) as ctx:
        ms = ctx.time_sweep(dA, form, [RHO] * m, mu=mu, gamma_relative=True, reps=args.reps)
    nbytes = p * n * dA.element_size()
    print(json.dumps({"sweep": form, "m": m, "dtype": args.sweep_dtype, "matrix": f"{p}x{n}", "ms": round(ms, 5),
                      "GB/s": round(nbytes / (ms / 1e3) / 1e9, 1)}), flush=True)


def _event_ms(stream, fn, reps):
    """Mean milliseconds of fn() over reps runs (CUDA events on `stream`)."""
    import torch

    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def _base_line(metric, unit, value, ms_per_step, args, workload, dtype, extra):
    line = {"metric": metric, "value": round(value, 3), "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": workload}}
    line.update(extra)
    return line


def _gamma_path(ctx, stream, dA, p, n, warmup, steps):
    """The sparsity-path measurements on dA (10000 x 50000): the 64 gammas of
    SL1 and SL0 as one batched solve and as 64 separate solves, block L1 with
    m = 32, and the sweeps alone.  Returns (results, ms per 64-gamma sweep,
    ms per m = 32 sweep, clocks)."""
    import torch

    from paper_1312_6182_gb300 import binding, synth

    rho = [float(r) for r in synth.log_spaced_rho(64)]
    res = {}
    clk = Clocks(0)
    clocks = None
    for form in ("SL1", "SL0"):
        out = binding.alloc_result(64, p, n, "cuda", torch.float32)
        one = binding.alloc_result(1, p, n, "cuda", torch.float32)
        for _ in range(warmup):
            ctx.solve(dA, form, rho, gamma_relative=True, out=out)
        if form == "SL1":
            clk.start()
        ms_b, r = _event_ms(stream, lambda: ctx.solve(dA, form, rho, gamma_relative=True, out=out), steps)
        if form == "SL1":
            clocks = clk.stop()
        it_b = int(r.iters.sum().item())
        sweeps_b = int(r.iters.max().item())

        def separate():
            tot = 0
            for g in rho:
                rr = ctx.solve(dA, form, [g], gamma_relative=True, out=one)
                tot += int(rr.iters.item())
            return tot

        separate()
        ms_s, it_s = _event_ms(stream, separate, 1)
        res[form] = {"batched_iters_per_s": round(it_b / (ms_b / 1e3), 1), "batched_ms_per_solve": round(ms_b, 3),
                     "batched_sweeps": sweeps_b, "separate_iters_per_s": round(it_s / (ms_s / 1e3), 1),
                     "separate_ms_for_64": round(ms_s, 3), "iters_sum": it_b,
                     "speedup_batched_vs_separate": round(ms_s / ms_b, 2)}
    # block L1, m = 32, mu = 1 on the same A; gamma = 0.01 max||a_i|| (with
    # only 3 spikes, larger gammas threshold whole noise components away)
    rho32 = [RHO32] * 32
    out32 = binding.alloc_result(32, p, n, "cuda", torch.float32)
    for _ in range(warmup):
        ctx.solve(dA, "BL1", rho32, mu=[1.0] * 32, gamma_relative=True, out=out32)
    ms_32, r32 = _event_ms(stream, lambda: ctx.solve(dA, "BL1", rho32, mu=[1.0] * 32, gamma_relative=True,
                                                    out=out32), max(1, steps // 2))
    res["BL1_m32"] = {"iters_per_s": round(int(r32.iters.max().item()) / (ms_32 / 1e3), 1),
                      "ms_per_solve": round(ms_32, 3), "iters": int(r32.iters.max().item()),
                      "status": sorted(set(int(v) for v in r32.status.tolist())), "rho": RHO32}
    # the sweep of the 64-column batch alone: one read of A is the algorithmic minimum
    ms_sw = ctx.time_sweep(dA, "SL1", rho, gamma_relative=True, reps=10)
    ms_sw32 = ctx.time_sweep(dA, "BL1", rho32, mu=[1.0] * 32, gamma_relative=True, reps=10)
    return res, ms_sw, ms_sw32, clocks


GAMMA_WORKLOAD = ("planted spikes 10000x50000 fp32 (3 spikes, theta_j=40/j, 2% supports), 64 gammas log-spaced "
                  "[0.001,0.5]*max||a_i||, SL1/SL0 batched vs separate; BL1 m=32 gamma=0.01*max||a_i||")


def run_gamma_path(args):
    """Sparsity path: 64 gamma values log-spaced over [0.001, 0.5] max||a_i||,
    single-unit L1 and L0 on a 10000 x 50000 FP32 planted-spike A (3 spikes,
    2% supports), as one batched solve (all 64 columns advance in every
    sweep) against 64 separate solves; plus block L1 with m = 32.  Units:
    solve-iterations (one gamma value, one sweep) per second."""
    import torch

    from paper_1312_6182_gb300 import binding, synth

    p, n = 10000, 50000
    At = synth.workload_spikes_10000x50000(1)
    dA = torch.from_numpy(At).cuda()
    del At
    stream = torch.cuda.Stream()
    ctx = binding.Context(0, stream=stream)
    res, ms_sw, ms_sw32, clocks = _gamma_path(ctx, stream, dA, p, n, args.warmup, args.steps)
    peak, kind = _peaks()
    nbytes = p * n * 4
    flops = 4.0 * p * n * 64
    ctx.close()
    value = res["SL1"]["batched_iters_per_s"]
    line = _base_line("gamma-path solve-iters/s (64 gammas batched)", "iters/s", value,
                      res["SL1"]["batched_ms_per_solve"], args, GAMMA_WORKLOAD, "f32",
                      {"results": res,
                       "roofline": {"bound": "hbm",
                                    "kernel": "tc_t_fused_kernel<192> + tc_y_fused_kernel<192> (tcgen05, float A "
                                              "split into exact bf16 planes in shared memory; two reads of A)",
                                    "frac_of_two_reads": round(2 * nbytes / (ms_sw / 1e3) / 1e9 / peak, 4),
                                    "achieved": round(nbytes / (ms_sw / 1e3) / 1e9, 1), "peak": peak,
                                    "unit": "GB/s", "frac": round(nbytes / (ms_sw / 1e3) / 1e9 / peak, 4),
                                    "peak_source": kind, "traffic": None, "ms_per_sweep": round(ms_sw, 4),
                                    "algorithmic_bytes_per_sweep": nbytes,
                                    "tflops_achieved": round(flops / (ms_sw / 1e3) / 1e12, 2)},
                       "block_m32_sweep_ms": round(ms_sw32, 4), "clocks": clocks})
    print(json.dumps(line), flush=True)


def run_deflation(args):
    """Several single-unit components by projection deflation on the 5000 x
    20000 FP32 planted-spike matrix (five spikes): SL1 and SL0, m = 5
    components, relative gamma 0.05 of each deflated matrix's largest column.
    Units: power iterations (sweeps t = A^T x, all components) per second over
    the whole extraction (working copy, five solves, four deflations).  With
    --oracle, the FP64 oracle's extraction of the same components is timed on
    the host cores and its objectives compared."""
    import time

    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    p, n, m = 5000, 20000, 5
    At = synth.workload_spikes_5000x20000(0)
    dA = torch.from_numpy(At).cuda()
    stream = torch.cuda.Stream()
    ctx = binding.Context(0, stream=stream)
    res = {}
    clk = Clocks(0)
    clocks = None
    for form in ("SL1", "SL0"):
        out = binding.alloc_result(m, p, n, "cuda", torch.float32)
        for _ in range(args.warmup):
            ctx.solve_deflated(dA, form, [0.05] * m, gamma_relative=True, out=out)
        if form == "SL1":
            clk.start()
        ms, r = _event_ms(stream, lambda: ctx.solve_deflated(dA, form, [0.05] * m, gamma_relative=True, out=out),
                          args.steps)
        if form == "SL1":
            clocks = clk.stop()
        iters = [int(v) for v in r.iters.tolist()]
        one = binding.alloc_result(1, p, n, "cuda", torch.float32)
        ms1, r1 = _event_ms(stream, lambda: ctx.solve(dA, form, [0.05], gamma_relative=True, out=one), args.steps)
        # scores of the 5000 samples on the five loadings (gpspca_project):
        # reads the support columns only
        Zc = r.Z.contiguous()
        Sc = torch.empty((m, p), dtype=torch.float32, device="cuda")
        ctx.project(dA, Zc, out=Sc)
        ms_proj, _ = _event_ms(stream, lambda: ctx.project(dA, Zc, out=Sc), args.steps)
        proj_bytes = int((r.Z != 0).sum().item()) * p * 4
        res[form + "_projection"] = {"ms": round(ms_proj, 4), "bytes_read": proj_bytes,
                                     "GB/s": round(proj_bytes / (ms_proj / 1e3) / 1e9, 1)}
        res[form] = {"iters_per_s": round(sum(iters) / (ms / 1e3), 1), "ms_per_extraction": round(ms, 3),
                     "iters": iters, "status": [int(v) for v in r.status.tolist()],
                     "support_sizes": [int(v) for v in (r.Z != 0).sum(dim=1).tolist()],
                     "objective": [float(v) for v in r.objective.tolist()],
                     "first_component_alone_ms": round(ms1, 3)}
        if args.oracle:
            import oracle

            A = At.astype(np.float64).T
            t0 = time.perf_counter()
            ref = oracle.gpower_deflated(A, form, [0.05] * m, tol=1e-6, maxit=1000, relative=True)
            sec = time.perf_counter() - t0
            obj = np.array(res[form]["objective"])
            res[form]["oracle"] = {"seconds": round(sec, 2), "iters": [int(v) for v in ref.iters],
                                   "objective_rel_err_max": float(np.max(np.abs(obj - ref.objective)
                                                                         / np.abs(ref.objective))),
                                   "cores": os.cpu_count()}
    ctx.close()
    value = res["SL1"]["iters_per_s"]
    extra = {"results": res, "clocks": clocks}
    if args.oracle:
        o = res["SL1"]["oracle"]
        extra["cpu_baseline"] = {"value": round(sum(o["iters"]) / o["seconds"], 3), "unit": "iters/s",
                                 "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": "the full SL1 extraction (5 components) once"}
    line = _base_line("deflation power iterations/s (5 single-unit components)", "iters/s", value,
                      res["SL1"]["ms_per_extraction"], args,
                      "planted spikes 5000x20000 fp32 (5 spikes), SL1/SL0, m=5 components by projection deflation, "
                      "gamma=0.05*max||a_i|| of each deflated matrix", "f32", extra)
    print(json.dumps(line), flush=True)


def run_latency(args):
    """The latency-bound case: 200 x 1000 i.i.d. N(0,1) with centred columns,
    FP64, SL1 at gamma = 0.1 max||a_i||, tol 1e-6, maxit 1000 (the matrix is
    1.6 MB, L2-resident).  Reported: microseconds per power iteration through
    the cached CUDA graph (stopping test on the device) and with the same
    kernels launched one by one from the host (one read-back of the active
    count per iteration): their difference is what the graph saves per
    iteration.  With --oracle, the FP64 oracle's time per iteration."""
    import time

    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    At = synth.workload_fp64_200x1000(0)
    dA = torch.from_numpy(At).cuda()
    stream = torch.cuda.Stream()
    ctx = binding.Context(0, stream=stream)
    out = binding.alloc_result(1, 200, 1000, "cuda", torch.float64)
    res = {}
    for eager in (False, True):
        for _ in range(args.warmup):
            ctx.solve(dA, "SL1", [0.1], gamma_relative=True, tol=1e-6, maxit=1000, out=out, eager=eager)
        ms, r = _event_ms(stream, lambda: ctx.solve(dA, "SL1", [0.1], gamma_relative=True, tol=1e-6, maxit=1000,
                                                    out=out, eager=eager), args.steps)
        it = int(r.iters.item())
        res["eager" if eager else "graph"] = {"ms_per_solve": round(ms, 4), "iters": it,
                                              "us_per_iter": round(ms * 1e3 / it, 2)}
    ctx.close()
    res["graph_saves_us_per_iter"] = round(res["eager"]["us_per_iter"] - res["graph"]["us_per_iter"], 2)
    extra = {"results": res}
    if args.oracle:
        import oracle

        A = At.T
        g = oracle.gamma_from_rho(A, "SL1", 0.1)
        t0 = time.perf_counter()
        ref = oracle.gpower(A, "SL1", g, tol=1e-6, maxit=1000)
        sec = time.perf_counter() - t0
        extra["cpu_baseline"] = {"value": round(int(ref.iters[0]) / sec, 1), "unit": "iters/s",
                                 "cores": os.cpu_count(), "kind": "oracle", "sample": "the whole solve once",
                                 "us_per_iter": round(sec * 1e6 / int(ref.iters[0]), 2)}
    value = res["graph"]["iters"] / (res["graph"]["ms_per_solve"] / 1e3)
    line = _base_line("GPower iters/s, latency-bound case", "iters/s", value, res["graph"]["ms_per_solve"], args,
                      "200x1000 N(0,1) centred fp64, SL1 gamma=0.1*max||a_i||, tol 1e-6 (L2-resident)", "f64", extra)
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Many small instances: 256 independent single-unit L1 solves of the
    latency-bound shape (200 x 1000 N(0,1), centred columns, FP64, gamma =
    0.1 max||a_i||, tol 1e-6; each its own seeded matrix) and 256 of 512 x
    4096 FP32 planted spikes (2 spikes, 5% supports, gamma = 0.05
    max||a_i||).  Each set three ways: one gpspca_solve_batch (same-shape
    requests run as groups: one launch per step for all members), the same
    requests queued with gpspca_submit (up to 8 solves in flight on their
    own streams), and one gpspca_solve after another.  Reported: solves/s
    and power iterations/s per way, and that every grouped result equals its
    one-by-one solve bit for bit."""
    import time

    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    count = 256
    sets = []
    mats = [synth.workload_fp64_200x1000(1000 + i) for i in range(count)]
    sets.append(("fp64 200x1000 SL1", [torch.from_numpy(a).cuda() for a in mats], 0.1, torch.float64))
    mats = [synth.planted_spike(512, 4096, 2, [30.0, 15.0], support_frac=0.05, seed=2000 + i, dtype=np.float32)
            for i in range(count)]
    sets.append(("fp32 512x4096 SL1", [torch.from_numpy(a).cuda() for a in mats], 0.05, torch.float32))
    del mats
    ctx = binding.Context(0)
    res = {}
    for name, dAs, rho, tc in sets:
        p, n = int(dAs[0].shape[1]), int(dAs[0].shape[0])
        outs = [binding.alloc_result(1, p, n, "cuda", tc) for _ in dAs]
        items = [dict(At=d, form="SL1", gamma=[rho], gamma_relative=True, out=o) for d, o in zip(dAs, outs)]

        def batch():
            return ctx.solve_batch(items)

        def serial():
            return [ctx.solve(d, "SL1", [rho], gamma_relative=True, out=o) for d, o in zip(dAs, outs)]

        def submitted():
            tickets = [ctx.submit(d, "SL1", [rho], gamma_relative=True, out=o)[0] for d, o in zip(dAs, outs)]
            for t in tickets:
                while ctx.poll(t, 1000) == binding.PENDING:
                    pass
            return outs

        entry = {}
        for way, fn in (("batch_grouped", batch), ("submit_8_in_flight", submitted), ("one_by_one", serial)):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                fn()
            torch.cuda.synchronize()
            sec = (time.perf_counter() - t0) / args.steps
            iters = int(sum(int(o.iters[0]) for o in outs))
            entry[way] = {"ms_per_set": round(sec * 1e3, 3), "solves_per_s": round(count / sec, 1),
                          "iters_per_s": round(iters / sec, 1)}
            if way == "batch_grouped":
                keep = [(o.Z.clone(), o.X.clone(), o.objective.clone()) for o in outs]
        serial()
        torch.cuda.synchronize()
        same = sum(torch.equal(z, o.Z) and torch.equal(x, o.X) and torch.equal(f, o.objective)
                   for (z, x, f), o in zip(keep, outs))
        entry["grouped_equal_one_by_one"] = f"{same}/{count}"
        entry["iters_mean"] = round(float(np.mean([int(o.iters[0]) for o in outs])), 1)
        entry["speedup_grouped_vs_one_by_one"] = round(
            entry["one_by_one"]["ms_per_set"] / entry["batch_grouped"]["ms_per_set"], 2)
        res[name] = entry
    ctx.close()
    value = res["fp64 200x1000 SL1"]["batch_grouped"]["solves_per_s"]
    line = _base_line("grouped small solves/s (256 x 200x1000 fp64 SL1)", "solves/s", value,
                      res["fp64 200x1000 SL1"]["batch_grouped"]["ms_per_set"], args,
                      "256 independent single-unit solves per set: 200x1000 N(0,1) centred fp64 (gamma 0.1) and "
                      "512x4096 fp32 planted spikes (gamma 0.05); grouped batch vs submit/poll vs one by one",
                      "f64|f32", {"results": res})
    print(json.dumps(line), flush=True)


SCALING_FORMS = (("SL0", 0.01), ("BL0", 0.01), ("SL1", 0.05), ("BL1", 0.05))


def run_scaling(args):
    """The paper's efficiency experiment (Section 4.1, Fig. 3) on synthetic
    inputs: A is P x N i.i.d. N(0,1) (the paper's random instances; float32
    here), N from 500 to 32000, P = N / 10, m = 5 components, the four
    formulations at the paper's gamma values (read as relative to the largest
    column norm): SL0 / BL0 at 0.01, SL1 / BL1 at 0.05.  Single-unit forms
    extract their five components by deflation, block forms solve for all
    five at once.  Reported: mean GPU milliseconds per solve (CUDA events,
    A resident), and with --oracle the FP64 oracle's time on the host cores
    for the sizes up to --oracle-max-n (one instance each) and the ratio.
    value = the mean GPU time per solve at the largest N (over forms and
    instances)."""
    import time

    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    sizes = [500, 1000, 2000, 4000, 8000, 16000, 32000]
    stream = torch.cuda.Stream()
    ctx = binding.Context(0, stream=stream)
    table = []
    clk = Clocks(0)
    clk.start()
    for N in sizes:
        P = N // 10
        row = {"N": N, "P": P}
        out = binding.alloc_result(5, P, N, "cuda", torch.float32)
        ms_all = {f: [] for f, _ in SCALING_FORMS}
        iters_all = {f: [] for f, _ in SCALING_FORMS}
        for inst in range(args.instances):
            dA = torch.from_numpy(synth.gaussian(P, N, seed=100000 + 100 * N + inst, dtype=np.float32)).cuda()
            for form, rho in SCALING_FORMS:
                def run():
                    if form.startswith("S"):
                        return ctx.solve_deflated(dA, form, [rho] * 5, gamma_relative=True, out=out)
                    return ctx.solve(dA, form, [rho] * 5, mu=[1.0] * 5, gamma_relative=True, out=out)

                if inst == 0:
                    run()  # warm: graphs and workspace
                ms, r = _event_ms(stream, run, 1)
                ms_all[form].append(ms)
                iters_all[form].append(int(r.iters.sum().item()) if form.startswith("S")
                                       else int(r.iters.max().item()))
            del dA
        for form, rho in SCALING_FORMS:
            cell = {"gpu_ms": round(float(np.mean(ms_all[form])), 3),
                    "iters_mean": round(float(np.mean(iters_all[form])), 1)}
            if args.oracle and N <= args.oracle_max_n:
                import oracle

                A = synth.gaussian(P, N, seed=100000 + 100 * N, dtype=np.float32).astype(np.float64).T
                t0 = time.perf_counter()
                if form.startswith("S"):
                    oracle.gpower_deflated(A, form, [rho] * 5, tol=1e-6, maxit=1000, relative=True)
                else:
                    gam = oracle.gamma_from_rho(A, form, [rho] * 5)
                    oracle.gpower(A, form, gam, tol=1e-6, maxit=1000)
                cell["oracle_ms"] = round((time.perf_counter() - t0) * 1e3, 1)
                cell["oracle_over_gpu"] = round(cell["oracle_ms"] / ms_all[form][0], 1)
            row[form] = cell
        table.append(row)
        print(json.dumps({"scaling_row": row}), file=sys.stderr, flush=True)
    clocks = clk.stop()
    ctx.close()
    last = table[-1]
    value = float(np.mean([last[f]["gpu_ms"] for f, _ in SCALING_FORMS]))
    line = _base_line("GP-SPCA ms per solve, m=5 (Fig. 3 sweep, largest N)", "ms/solve", value, value, args,
                      f"i.i.d. N(0,1) P x N fp32, N in {sizes}, P=N/10, {args.instances} instances, m=5, "
                      "SL0/BL0 gamma=0.01, SL1/BL1 gamma=0.05 (relative), single-unit by deflation", "f32",
                      {"higher_is_better": False, "results": table, "clocks": clocks})
    print(json.dumps(line), flush=True)


def _fp8_columns(dA32):
    """FP8 E4M3 storage with per-column scales s_i = max_r |A_ri| / 448."""
    import torch

    s = dA32.abs().amax(dim=1) / 448.0
    s = torch.where(s > 0, s, torch.ones_like(s))
    q = (dA32 / s[:, None]).to(torch.float8_e4m3fn)
    return q, s.float().contiguous()


def _precision(ctx, stream, d32, p, n, rho, refine_sweeps, warmup, steps):
    """The precision-path measurements on the float matrix d32 (n x p
    column-major storage): BL1 and BL0 with m = 16, solved on the FP32
    matrix, and on its BF16 and FP8 E4M3 (per-column scales) copies followed
    by `refine_sweeps` FP32 sweeps from the converged X; and each storage's sweep
    alone.  Returns (results, kept outputs, clocks, ms per sweep by storage)."""
    import torch

    from paper_1312_6182_gb300 import binding

    m = 16
    dbf = d32.to(torch.bfloat16)
    d8, s8 = _fp8_columns(d32)
    mu = [1.0] * m
    out = binding.alloc_result(m, p, n, "cuda", torch.float32)
    out2 = binding.alloc_result(m, p, n, "cuda", torch.float32)
    res = {}
    keep = {}
    clk = Clocks(0)
    clocks = None
    for form in ("BL1", "BL0"):
        for fmt, dA, cs in (("f32", d32, None), ("bf16", dbf, None), ("fp8", d8, s8)):
            def solve():
                return ctx.solve(dA, form, [rho] * m, mu=mu, gamma_relative=True, out=out, col_scale=cs)

            for _ in range(warmup):
                solve()
            if clocks is None:
                clk.start()
            ms, r = _event_ms(stream, solve, max(1, steps // 4))
            if clocks is None:
                clocks = clk.stop()
            iters = int(r.iters.max().item())
            entry = {"ms_per_solve": round(ms, 3), "iters": iters, "iters_per_s": round(iters / (ms / 1e3), 1),
                     "status": int(r.status.max().item())}
            if fmt != "f32":
                x0 = r.X.contiguous().clone()

                def refine():
                    return ctx.solve(d32, form, [rho] * m, mu=mu, gamma_relative=True, tol=0.0,
                                     maxit=refine_sweeps, x0=x0, out=out2)

                ms_r, rr = _event_ms(stream, refine, max(1, steps // 4))
                entry["refine_ms"] = round(ms_r, 3)
                entry["ms_total"] = round(ms + ms_r, 3)
                keep[(form, fmt)] = {k: getattr(rr, k).clone() for k in ("X", "Z", "objective", "support")}
            else:
                entry["ms_total"] = round(ms, 3)
                keep[(form, fmt)] = {k: getattr(r, k).clone() for k in ("X", "Z", "objective", "support")}
            entry["solves_per_s"] = round(1e3 / entry["ms_total"], 2)
            res[f"{form}_{fmt}"] = entry
    sweep_ms = {fmt: ctx.time_sweep(dA, "BL1", [rho] * m, mu=mu, gamma_relative=True, reps=5, col_scale=cs)
                for fmt, dA, cs in (("f32", d32, None), ("bf16", dbf, None), ("fp8", d8, s8))}
    return res, keep, clocks, sweep_ms


def run_precision(args):
    """Precision path: block L1 and L0, m = 16, on a 20000 x 100000
    planted-spike A (16 spikes, 1% supports, theta_j = 100/sqrt j) stored in
    BF16 and in FP8 E4M3 with per-column scales, each solved to convergence
    and then refined by --refine-sweeps FP32 sweeps (default 3) from the
    converged X on the FP32 copy; against the plain FP32 solve.  --rho sets
    gamma (default 0.05 max||a_i||); a smaller rho or --theta-scale < 1 gives
    a slower-converging instance.  With --oracle, errors of every variant
    against the FP64 oracle on the FP32 matrix (objective, loadings, support)."""
    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    p, n, m = 20000, 100000, 16
    if args.theta_scale == 1.0:
        At = synth.workload_spikes_20000x100000(2)
    else:  # the same draw with weaker spikes (slower convergence)
        At = synth.planted_spike(p, n, 16, [100.0 * args.theta_scale / np.sqrt(j) for j in range(1, 17)],
                                 support_frac=0.01, seed=2, dtype=np.float32, noise_streams=16)
    d32 = torch.from_numpy(At).cuda()
    if not args.oracle:
        del At
    stream = torch.cuda.Stream()
    ctx = binding.Context(0, stream=stream)
    mu = [1.0] * m
    res, keep, clocks, sweep_ms = _precision(ctx, stream, d32, p, n, args.rho, args.refine_sweeps, args.warmup,
                                             args.steps)
    ctx.close()
    if args.oracle:
        import oracle

        A64 = At.astype(np.float64).T
        del At
        for form in ("BL1", "BL0"):
            gam = oracle.gamma_from_rho(A64, form, [args.rho] * m)
            ref = oracle.gpower(A64, form, gam, mu=np.array(mu), tol=1e-6, maxit=1000)
            for fmt in ("f32", "bf16", "fp8"):
                g = keep[(form, fmt)]
                Z = g["Z"].double().cpu().numpy().T
                zerr = [float(np.linalg.norm(Z[:, j] - ref.Z[:, j]) / max(np.linalg.norm(ref.Z[:, j]), 1e-300))
                        for j in range(m)]
                ferr = abs(float(g["objective"].sum().item()) - ref.total) / ref.total
                sup = (Z != 0) != (ref.Z != 0)
                res[f"{form}_{fmt}"]["oracle"] = {"loadings_rel_err_max": max(zerr), "objective_rel_err": ferr,
                                                 "support_mismatches": int(sup.sum()),
                                                 "oracle_iters": int(ref.iters[0]), "oracle_status": int(ref.status[0])}
    peak, kind = _peaks()
    bytes_of = {"f32": p * n * 4, "bf16": p * n * 2, "fp8": p * n + n * 4}
    roof = {fmt: {"ms_per_sweep": round(ms_, 4), "GB/s": round(bytes_of[fmt] / (ms_ / 1e3) / 1e9, 1),
                  "frac": round(bytes_of[fmt] / (ms_ / 1e3) / 1e9 / peak, 4)} for fmt, ms_ in sweep_ms.items()}
    value = res["BL1_bf16"]["solves_per_s"]
    line = _base_line(f"precision-path solves/s (BF16 + {args.refine_sweeps} FP32 refinement sweeps)", "solves/s",
                      value, res["BL1_bf16"]["ms_total"], args,
                      f"planted spikes 20000x100000 (16 spikes, theta_j={100 * args.theta_scale:g}/sqrt(j), 1% "
                      f"supports), BL1/BL0 m=16 mu=1, gamma={args.rho:g}*max||a_i||; BF16 and FP8-E4M3 (per-column "
                      f"scales) storage + {args.refine_sweeps} FP32 sweeps vs FP32",
                      "bf16",
                      {"results": res, "roofline": {"bound": "hbm", "peak": peak, "peak_source": kind, "unit": "GB/s",
                                                    "sweeps_m16": roof}, "clocks": clocks})
    print(json.dumps(line), flush=True)


def _pct(xs, q):
    import numpy as np

    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def _serving(nreq, warmup):
    """The serving mix (Poisson arrivals at 200/s; p, n log-uniform
    over [256, 8192] x [1024, 65536]; FP32 or BF16; the four forms; m in
    1..16; rho ~ U(0.02, 0.2)); each request's planted-spike A is drawn on
    the device (seed 1000 + id, timed as ingest) and submitted to the
    context's continuous-batching scheduler (admission by HBM footprint:
    matrix, outputs and workspace under a 150 GB budget; up to 8 solves
    overlapping).  Measured: served solves/s and p50/p99 latency at the
    offered load, the saturated throughput, and the serial plain per-request
    solves on the same requests (their latency at the same arrivals from a
    single-server FIFO queue).  Returns (summary, clocks, span in seconds)."""
    import numpy as np
    import torch

    from paper_1312_6182_gb300 import binding, synth

    reqs = synth.serving_requests(count=nreq, rate=200.0, seed=3)
    gen_stream = torch.cuda.Stream()
    ctx = binding.Context(0, budget_bytes=150 << 30)

    def make_input(r):
        tdt = torch.float32 if r.dtype == "f32" else torch.bfloat16
        A = torch.empty((r.n, r.p), device="cuda", dtype=tdt)
        binding.synth_spikes(A, max(r.m, 1), r.theta(), 0.05, r.seed, stream=gen_stream)
        gen_stream.synchronize()
        return A

    def mu_of(r):
        return [1.0] * r.m if r.form.startswith("B") else None

    def serve(use_arrivals):
        lat, lat_solve, ingest, results = [], [], [], {}
        pending = {}
        i, t0 = 0, time.perf_counter()
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            if i < len(reqs) and (not use_arrivals or reqs[i].arrival_s <= now) and len(pending) < 64:
                r = reqs[i]
                t_in = time.perf_counter()
                A = make_input(r)
                t_ready = time.perf_counter()
                ingest.append(t_ready - t_in)
                t, out = ctx.submit(A, r.form, r.gammas(), mu=mu_of(r), tol=TOL, maxit=MAXIT, gamma_relative=True)
                pending[t] = (r, A, out, t0 + (r.arrival_s if use_arrivals else 0.0), t_ready)
                i += 1
                continue
            idle = i >= len(reqs) or len(pending) >= 64 or (use_arrivals and reqs[i].arrival_s > now)
            first = True
            for t in list(pending):
                # when there is nothing to submit, wait up to 20 us on the oldest request
                rc = ctx.poll(t, 20 if (idle and first) else 0)
                first = False
                if rc == binding.PENDING:
                    continue
                tc = time.perf_counter()
                r, A, out, t_arr, t_ready = pending.pop(t)
                if rc not in (binding.OK, binding.EDEGENERATE):
                    raise RuntimeError(f"request {r.id} failed: {rc} {binding.last_error()}")
                lat.append(tc - t_arr)
                lat_solve.append(tc - t_ready)
                results[r.id] = out
        return time.perf_counter() - t0, lat, lat_solve, ingest, results

    # warm-up: a few requests through both paths (graph builds for common shapes are per shape)
    for r in reqs[:warmup]:
        A = make_input(r)
        ctx.solve(A, r.form, r.gammas(), mu=mu_of(r), tol=TOL, maxit=MAXIT, gamma_relative=True)
    clk = Clocks(0)
    clk.start()
    span, lat, lat_solve, ingest, served = serve(True)
    clocks = clk.stop()
    span_sat, lat_sat, _, _, _ = serve(False)
    # serial plain per-request solves on the same requests
    svc, serial_out = [], {}
    sample = set(range(0, len(reqs), max(1, len(reqs) // 20)))
    for r in reqs:
        A = make_input(r)
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        res = ctx.solve(A, r.form, r.gammas(), mu=mu_of(r), tol=TOL, maxit=MAXIT, gamma_relative=True)
        svc.append(time.perf_counter() - t_a)
        if r.id in sample:
            serial_out[r.id] = res
    # the same results alone and in the mix
    same = sum(1 for k, v in serial_out.items()
               if torch.equal(v.Z, served[k].Z) and torch.equal(v.objective, served[k].objective))
    # single-server FIFO latency of the serial path at the same arrivals (Lindley)
    free_at, lat_serial = 0.0, []
    for r, sv in zip(reqs, svc):
        start = max(r.arrival_s, free_at)
        free_at = start + sv
        lat_serial.append(free_at - r.arrival_s)
    ctx.close()
    summary = {
        "offered_rate": 200.0, "requests": nreq,
        "served_solves_per_s": round(nreq / span, 2),
        "p50_ms": round(_pct(lat, 50) * 1e3, 3), "p99_ms": round(_pct(lat, 99) * 1e3, 3),
        "p50_solve_ms": round(_pct(lat_solve, 50) * 1e3, 3),
        "p99_solve_ms": round(_pct(lat_solve, 99) * 1e3, 3),
        "ingest_ms_mean": round(float(np.mean(ingest)) * 1e3, 4),
        "saturated_solves_per_s": round(nreq / span_sat, 2),
        "saturated_p50_ms": round(_pct(lat_sat, 50) * 1e3, 3),
        "serial_solves_per_s": round(nreq / sum(svc), 2),
        "serial_p50_ms_at_offered": round(_pct(lat_serial, 50) * 1e3, 3),
        "serial_p99_ms_at_offered": round(_pct(lat_serial, 99) * 1e3, 3),
        "same_alone_and_in_mix": f"{same}/{len(serial_out)}",
        "mean_p_times_n": float(np.mean([r.p * r.n for r in reqs]))}
    return summary, clocks, span


SERVING_MIX = ("p in [256,8192], n in [1024,65536] log-uniform, fp32|bf16, SL1|SL0|BL1|BL0, m 1..16, rho "
               "U(0.02,0.2), device-generated planted spikes (Philox4x32-10, seed 1000+id), Poisson arrivals at 200/s")


def run_serving(args):
    """Serving: the request mix of `_serving` with --requests requests."""
    summary, clocks, span = _serving(args.requests, args.warmup)
    nreq = summary["requests"]
    line = _base_line("served solves/s", "solves/s", nreq / span, span * 1e3 / nreq, args,
                      f"serving mix: {nreq} requests, {SERVING_MIX}", "f32|bf16",
                      {"serving": summary, "clocks": clocks})
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default 100; 4 for the other workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--sweep-only", default=None, choices=["SL1", "SL0", "BL1", "BL0"],
                    help="time the fused sweep alone on the benchmark matrix (profiling)")
    ap.add_argument("--sweep-m", type=int, default=None, help="sweep-only: components or gammas (default 1 / 5)")
    ap.add_argument("--sweep-dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--sweep-matrix", default="5000x20000", choices=["5000x20000", "20000x100000", "20000x25000"],
                    help="sweep-only: the matrix")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--workload", default="step",
                    choices=["step", "gamma-path", "precision", "serving", "deflation", "scaling", "latency", "batch"],
                    help="step: the headline step (20000x100000, with the 5000x20000 step beside it); the others "
                         "measure the sparsity-path batch, the "
                         "BF16/FP8 precision path, the serving mix, deflated multi-component extraction and the "
                         "size sweep of the paper's efficiency experiment (one JSON line each)")
    ap.add_argument("--oracle", action="store_true",
                    help="precision / deflation / scaling workloads: also run (and time) the FP64 oracle")
    ap.add_argument("--instances", type=int, default=4, help="scaling workload: random instances per size")
    ap.add_argument("--oracle-max-n", type=int, default=8000, help="scaling workload: largest N the oracle runs")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: number of requests")
    ap.add_argument("--rho", type=float, default=0.05,
                    help="precision workload: gamma = rho max||a_i|| (L1) / its square (L0)")
    ap.add_argument("--refine-sweeps", type=int, default=3, help="precision workload: FP32 refinement sweeps")
    ap.add_argument("--theta-scale", type=float, default=1.0,
                    help="precision workload: spike strengths theta_j = 100 * scale / sqrt(j) (1 = the workload)")
    ap.add_argument("--eager", action="store_true",
                    help="launch each solve's kernels one by one (profilers cannot follow the CUDA graph's "
                         "conditional node); slower, for launch lists only")
    args = ap.parse_args()
    if args.sweep_only:
        run_sweep_only(args)
        return
    if args.steps is None:
        args.steps = 20 if args.workload == "step" else 4
    if args.workload != "step":
        args.warmup = max(args.warmup, 1)
        {"gamma-path": run_gamma_path, "precision": run_precision, "serving": run_serving,
         "deflation": run_deflation, "scaling": run_scaling, "latency": run_latency,
         "batch": run_batch}[args.workload](args)
        return
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
