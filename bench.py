"""FastTT throughput on one GB300 (nnz/s), one JSON line on stdout.

Headline workload: the banded sparse matrix of the sparse-matrix -> QTT
configuration at 2^12 x 2^12 (5-diagonal band + 5 uniform off-band entries per
row, U(-1,1), row/column bits interleaved into 12 modes of size 4), eps = 1e-6:
the FP64-vs-mixed comparison at relative error <= 1e-6.  The full 2^20 x 2^20
matrix has exact TT ranks near 1e6 and cannot be rounded densely on one GPU; its
grouping (S1-S5) is timed at full size as a secondary line.  A step is one
fasttt_decompose over the whole tensor.  `value` is the FP64 path's
device-resident throughput (the path whose sampled error meets 1e-6); the mixed
path is timed the same way beside it.  `e2e` runs the same call from pinned host
buffers with the host->device copy of the COO input and the device->host copy of
every output core inside the timed region.

Secondary lines (each timed after the headline, guarded): the 5-way 50^5 tensor
(1e5 nnz, eps 1e-8), the Zipf 8-way 100^8 tensor (1e7 nnz, FP32 values, eps 1e-4,
rank cap 64) and the clustered 12-way 64^12 tensor (5e7 nnz, eps 1e-5, rank cap
128), each in FP64 and mixed precision; entry evaluation + adjoint; TT-rounding;
fitting; dynamic truncation; the FDM matrices of Table 2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank decomposes its own tensor (seed + rank, weak scaling,
no collective on the data path); rank 0 prints max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FastTT nnz/s at rel. err <=1e-6 (FP64 vs mixed, 1 GB300); adjoint % HBM roofline"
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2070 MHz
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.070e9 / 1e12  # 128 FFMA/clk/SM x 152 SMs x 2070 MHz
HEADLINE_M = 12                                     # 2^12 x 2^12 banded matrix, 12 modes of size 4
SAMPLE_M = 10                                       # oracle sample: the same recipe at 2^10 x 2^10
OZ_PAIRS_FP64 = 36                                  # slice pairs (s, t), s + t <= 9, of the 8-slice product
ERR_BAR = 1e-6                                      # the metric's relative-error bar
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the headline step's
# kernels, from one ncu capture of the headline decomposition (profiles/ has the summary and
# the command); a kernel changed since the capture has no entry
TRIDIAG64 = "tridiag_panel_kernel<8>+tridiag_kernel<double,8>"
NCU_TRAFFIC = {
    TRIDIAG64: {"bytes": 61.88e9,
                "source": "ncu, 2^12 QTT decomposition, per step: 55 panel launches (61.79 GB read, 0.10 GB "
                          "written) + 1 unblocked launch (3 MB)"},
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return world, rank


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(rank, name="qtt12"):
    from paper_1908_02721_gb300 import workloads as W
    if name == "qtt10":   # small case of the same recipe (profiling captures)
        return W.banded_qtt(SAMPLE_M, seed=3 + 1000 * rank, eps=1e-6)
    return W.banded_qtt(HEADLINE_M, seed=3 + 1000 * rank, eps=1e-6)


def _sample_workload():
    """The oracle's bounded sample: the same recipe at 2^10 x 2^10 (10 modes of size 4)."""
    from paper_1908_02721_gb300 import workloads as W
    return W.banded_qtt(SAMPLE_M, seed=3, eps=1e-6)


def _oracle_step(w):
    from oracle import fasttt as O
    t = time.perf_counter()
    O.fasttt(w.idx, w.vals, w.dims, w.eps)
    return time.perf_counter() - t


def _max_over_ranks(x, device):
    """Max of a per-rank number over all ranks (the slowest replica sets the job's time);
    the number itself when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


HEADLINE_NAME = (f"banded sparse matrix -> QTT: 2^{HEADLINE_M} x 2^{HEADLINE_M}, band5 + 5 off-band per row, "
                 f"U(-1,1), {HEADLINE_M} modes of size 4, eps=1e-6")


def run_reference(args):
    world, rank = _dist()
    if rank != 0:
        return
    w = _sample_workload()
    for _ in range(args.warmup):
        _oracle_step(w)
    ts = [_oracle_step(w) for _ in range(args.steps)]
    total = sum(ts)
    value = w.nnz * args.steps / total
    sample = (f"FP64 oracle, full FastTT per step on the same recipe at 2^{SAMPLE_M} x 2^{SAMPLE_M} "
              f"({SAMPLE_M} modes of size 4, {w.nnz} nnz, eps=1e-6); the 2^{HEADLINE_M} case takes about "
              "10 minutes per run, beyond a bounded step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": HEADLINE_NAME, "sample": sample, "same_config": False},
            "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_steps(F, idx, vals, w, steps, warmup, flush, stream, **kw):
    """Warm-up calls, then `steps` timed decompositions (CUDA events on the launching
    stream, L2 flushed between steps outside the events); the last handle is returned."""
    import torch
    for _ in range(warmup):
        F.fasttt_decompose(idx, vals, w.dims, w.eps, max_rank=w.max_rank, **kw).free()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    tt, stats = None, []
    for i in range(steps):
        if tt is not None:
            tt.free()
        flush.fill_(float(i))
        ev[i][0].record(stream)
        tt = F.fasttt_decompose(idx, vals, w.dims, w.eps, max_rank=w.max_rank, **kw)
        ev[i][1].record(stream)
        stats.append(tt.stats)
    torch.cuda.synchronize()
    return tt, stats, [a.elapsed_time(b) for a, b in ev]


STAGE_KEYS = ("ms_ingest", "ms_group", "ms_depar", "ms_round", "ms_gemm_oz", "ms_gemm", "ms_jacobi", "ms_tsqr",
              "ms_tridiag32", "ms_tridiag", "ms_tdeig", "ms_jacobi32", "ms_sort")
ROUTE_KEYS = ("eig_fast", "eig_tridiag", "eig_fallbacks", "sparse_bonds", "qr_cholqr2", "qr_svd",
              "mixed_fp32_bonds", "mixed_fp64_bonds")


def run_ours(args):
    import torch
    from paper_1908_02721_gb300 import fasttt as F

    world, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = _workload(rank, args.workload)
    idx = torch.from_numpy(w.idx).to(dev)
    vals = torch.from_numpy(w.vals).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def step():
        tt = F.fasttt_decompose(idx, vals, w.dims, w.eps)
        st = tt.stats
        tt.free()
        return st

    for _ in range(args.warmup):
        step()
    # timed region: K steps, L2 flushed between steps outside the per-step events
    stats = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            stats.append(step())
            ev[i][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = _max_over_ranks(sum(step_ms) / args.steps, dev)
    value = w.nnz * world / (ms / 1e3)

    # accuracy of the timed configuration: relative error of B at a fixed sample of nonzeros
    rel_err = _sampled_rel_err(F, idx, w, "fp64")
    mixed_line = None if args.no_mixed else _mixed(args, F, idx, vals, w, flush, stream, ms)

    # e2e through the same C-ABI call from pinned host memory
    e2e_line = None
    if not args.no_e2e:
        e2e_line = _e2e(args, w, F, dev, barrier, world)
    # the other configurations, then the extension timings, each guarded
    configs_line = None if args.no_configs else _configs(args, F, dev, flush, stream, world)
    adjoint_line = None if args.no_adjoint else _adjoint(args, F, dev, stream)
    round_line = None if args.no_tt_round else _tt_round(F, dev, stream)
    next_line = None if args.no_tt_round else _next_rows(F, dev, stream)
    if adjoint_line is not None and "_fit_args" in adjoint_line:
        cores8, aidx, aw, am = adjoint_line.pop("_fit_args")
        adjoint_line["fit_rank8"] = _fit(F, cores8, aidx, aw, dev, stream, am)
        del cores8, aidx, aw
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    st = stats[-1]
    peaks, src = _peaks()
    roofline = _roofline(st, peaks)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sw = _sample_workload()
        t = _oracle_step(sw)
        cpu = {"value": sw.nnz / t, "unit": "nnz/s", "cores": _cores(), "kind": "oracle",
               "sample": (f"FP64 oracle, full FastTT on the same recipe at 2^{SAMPLE_M} x 2^{SAMPLE_M} "
                          f"({sw.nnz} nnz), one run")}
    line = {"metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (HEADLINE_NAME + ", FP64 FastTT" if args.workload == "qtt12"
                                    else f"profiling case {args.workload}"),
                       "nnz": w.nnz, "dims": w.dims, "eps": w.eps, "p": st["p"], "ranks": st["ranks"],
                       "rt": st["rt"], "beta": [st["beta_r"], st["beta_c"]],
                       "l2": "flushed between steps (256 MiB write, outside the step events)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e_line,
            "rel_err_sampled": rel_err,
            "meets_err_bar": rel_err <= ERR_BAR,
            "mixed": mixed_line,
            "configs": configs_line,
            "adjoint": adjoint_line,
            "tt_round": round_line,
            "next_rows": next_line,
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk.summary(),
            "stages_ms": {k: st[k] for k in STAGE_KEYS},
            "routes": {k: st[k] for k in ROUTE_KEYS},
            "jacobi_sweeps": st["jacobi_sweeps"],
            "wall_s": wall, "peaks_source": src}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _roofline(st, peaks):
    """The dominant kernel class of one step by CUDA-event time, its achieved rate against
    its peak.  The tcgen05 GEMM computes an FP64 product from 8 exact bf16 slices per
    operand: 36 slice-pair products, so its tensor-pipe work is 36 x 2MNK bf16 flops,
    measured against the bf16 dense peak -- the sustained one, as the slice GEMM's launches
    are spread over the whole step.  The FP64 tridiagonalisation's work is what its own
    kernels do on the FP64 pipe: per column of a blocked panel 2m^2 (the product with the
    matrix as it was at the panel's start) + 12jm (the panel's sums), per column of the
    unblocked remainder 6m^2; each panel's rank-128 update of the rest is a slice GEMM and
    counts in that class."""
    bf16_peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1921.5))
    classes = {"gemm_f64_kernel": (st["ms_gemm"], st["flop_gemm"], "alu", FP64_PEAK_TFLOPS),
               "jacobi_sweep_kernel<double>": (st["ms_jacobi"], st["flop_jacobi"], "alu", FP64_PEAK_TFLOPS),
               TRIDIAG64: (st["ms_tridiag"], st["flop_tridiag"], "alu", FP64_PEAK_TFLOPS),
               "ozaki_gemm_kernel<8,7,384,64,2>": (st["ms_gemm_oz"], OZ_PAIRS_FP64 * st["flop_gemm_oz"], "tensor",
                                                   bf16_peak),
               "tridiag_kernel<float>": (st["ms_tridiag32"], st["flop_tridiag32"], "alu", FP32_PEAK_TFLOPS),
               "qr_blocks_kernel+qr_apply_kernel": (st["ms_tsqr"], st["flop_tsqr"], "alu", FP64_PEAK_TFLOPS)}
    name, (kms, kwork, bound, peak) = max(classes.items(), key=lambda kv: kv[1][0])
    achieved = kwork / (kms / 1e3) / 1e12 if kms > 0 else 0.0
    out = {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak,
           "unit": "TFLOP/s", "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(name, {}).get("bytes"),
           "traffic_source": NCU_TRAFFIC.get(name, {}).get("source"),
           "peak_source": (("bf16 dense, measured, sustained (MEASURED_PEAKS.json bf16_tflops_sustained: the kernel's "
                            "launches run throughout the step)") if bound == "tensor" else
                           "FP32 FFMA: 128 per clock per SM x 152 SMs x 2070 MHz (derived)" if peak == FP32_PEAK_TFLOPS
                           else "FP64 DFMA: 2 per clock per SM x 152 SMs x 2070 MHz (derived; measured 1.198)"),
           "share_of_step": kms / st["ms_total"] if st["ms_total"] else None,
           "classes_ms": {k: v[0] for k, v in classes.items()}}
    if st["ms_gemm_oz"] > 0:
        out["ozaki_fp64_equivalent_tflops"] = st["flop_gemm_oz"] / (st["ms_gemm_oz"] / 1e3) / 1e12
    return out


def _sampled_rel_err(F, idx, w, precision, tt=None):
    """||B - A|| / ||A|| over 20,000 fixed nonzeros (tt_eval_at on the decomposition)."""
    import numpy as np
    import torch
    own = tt is None
    if own:
        tt = F.fasttt_decompose(idx, torch.from_numpy(w.vals).to(idx.device), w.dims, w.eps, precision=precision)
    rng = np.random.Generator(np.random.Philox(key=99))
    pick = rng.choice(w.nnz, min(20000, w.nnz), replace=False)
    a = F.tt_eval_at(tt.cores(), torch.from_numpy(np.ascontiguousarray(w.idx[:, pick])).to(idx.device))
    ref = w.vals[pick]
    err = float(np.linalg.norm(a.cpu().numpy() - ref) / np.linalg.norm(ref))
    if own:
        tt.free()
    return err


def _mixed(args, F, idx, vals, w, flush, stream, fp64_ms):
    """The headline workload in mixed precision: FP32-level tensor-core contractions
    (3 exact bf16 slices) where a bond's rank decision is resolved at that level, FP64-level
    products where it is not; FP64 Cholesky, rank decisions and error bookkeeping."""
    steps = max(3, args.steps // 4)
    tt, stats, ms_list = _time_steps(F, idx, vals, w, steps, min(args.warmup, 2), flush, stream, precision="mixed")
    ms = sum(ms_list) / steps
    err = _sampled_rel_err(F, idx, w, "mixed", tt)
    st = stats[-1]
    tt.free()
    return {"value": w.nnz / (ms / 1e3), "unit": "nnz/s", "ms_per_step": ms, "steps": steps,
            "speedup_vs_fp64": fp64_ms / ms, "rel_err_sampled": err, "meets_err_bar": err <= ERR_BAR,
            "ranks": st["ranks"], "dtype": "bf16-slice (3 slices, FP32-level) tensor-core contractions + f64",
            "stages_ms": {k: st[k] for k in STAGE_KEYS}, "routes": {k: st[k] for k in ROUTE_KEYS}}


def _configs(args, F, dev, flush, stream, world):
    """The other configurations, each in FP64 and in mixed precision: the 5-way 50^5 tensor
    (1e5 nnz, eps 1e-8; 3 timed steps after 2 warm-ups), the Zipf 100^8 tensor (1e7 nnz,
    FP32 values, eps 1e-4, rank cap 64) and the clustered 64^12 tensor (5e7 nnz, eps 1e-5,
    rank cap 128), one timed call each (they take seconds to minutes)."""
    import torch
    from paper_1908_02721_gb300 import workloads as W
    out = {}
    plan = [("uniform5_50x5", lambda: W.uniform5(seed=2), 3, 2),
            ("zipf8_100x8", lambda: W.zipf_tt(), 1, 0)]
    if world == 1 and not args.no_config5:
        plan.append(("clustered12_64x12", lambda: W.clustered(), 1, 0))
    for name, make, steps, warm in plan:
        entry = {}
        try:
            t = time.perf_counter()
            w = make()
            entry["workload"] = w.name
            entry["generate_s"] = time.perf_counter() - t
            entry["nnz"] = w.nnz
            entry["eps"] = w.eps
            entry["max_rank"] = w.max_rank
            idx = torch.from_numpy(w.idx).to(dev)
            vals = torch.from_numpy(w.vals).to(dev)
            for prec in ("fp64", "mixed"):
                try:
                    tt, stats, ms_list = _time_steps(F, idx, vals, w, steps, warm, flush, stream, precision=prec)
                    st = stats[-1]
                    ms = sorted(ms_list)[len(ms_list) // 2]
                    entry[prec] = {"ms": ms, "nnz_per_s": w.nnz / (ms / 1e3), "p": st["p"], "ranks": st["ranks"],
                                   "rt_max": max(st["rt"]), "rel_err_sampled": _sampled_rel_err(F, idx, w, prec, tt),
                                   "err_bound": math.sqrt(max(st["err2"], 0.0) / st["norm2"]),
                                   "stages_ms": {k: st[k] for k in STAGE_KEYS},
                                   "routes": {k: st[k] for k in ROUTE_KEYS}}
                    if prec == "fp64" and name.startswith("clustered"):
                        entry["adjoint_recompute"] = _adjoint_on(F, tt, idx, w, stream)
                    tt.free()
                except Exception as e:
                    entry[prec] = {"error": str(e)[:300]}
            if "ms" in entry.get("fp64", {}) and "ms" in entry.get("mixed", {}):
                entry["mixed_speedup_vs_fp64"] = entry["fp64"]["ms"] / entry["mixed"]["ms"]
            del idx, vals, w
            torch.cuda.empty_cache()
        except Exception as e:
            entry["error"] = str(e)[:300]
        out[name] = entry
    return out


def _adjoint_on(F, tt, idx, w, stream):
    """Evaluation and adjoint (recomputed left partials, checkpointed every ceil(sqrt(d))
    modes) of the decomposition's TT, cast to FP32, on all of the workload's entries with
    upstream weights = the residuals a - v."""
    import numpy as np
    import torch
    try:
        cores = [c.float().contiguous() for c in tt.cores()]
        vals = torch.from_numpy(np.asarray(w.vals, dtype=np.float32)).to(idx.device)
        F.tt_eval_at(cores, idx)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        a = F.tt_eval_at(cores, idx)
        e[1].record(stream)
        grads = F.tt_eval_backward(cores, idx, a - vals, recompute=True)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        rk = tt.ranks
        flops = w.nnz * 2.0 * 3.0 * sum(rk[k] * rk[k + 1] for k in range(len(rk) - 1))
        out = {"entries": w.nnz, "ranks": rk, "dtype": "f32 cores", "eval_ms": fwd, "backward_ms": bwd,
               "backward_tflops": flops / (bwd / 1e3) / 1e12,
               "backward_fp32_frac": flops / (bwd / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
               "grad_norm": float(sum(float(g.double().norm()) ** 2 for g in grads) ** 0.5)}
        del cores, grads, a
        return out
    except Exception as e:   # reported, never hidden
        return {"error": str(e)[:300]}


def _adjoint(args, F, dev, stream):
    """tt_eval_at + tt_eval_backward on every nonzero of the Zipf(1.2) 100^8 workload (1e7
    entries) for FP32 TTs of rank 8 (the planted rank) and rank 64 (the rank cap)."""
    import math
    import numpy as np
    import torch
    from paper_1908_02721_gb300 import workloads as W
    w = W.zipf_tt(nnz=10_000_000)
    idx = torch.from_numpy(w.idx).to(dev)
    m = w.nnz
    out = {"workload": "Zipf(1.2) 8-way 100^8, 1e7 distinct entries, FP32 cores", "entries": m}
    peaks, _ = _peaks()
    hbm = peaks.get("hbm_gbs", 6686.8)
    for r in (8, 64):
        rng = np.random.Generator(np.random.Philox(key=400 + r))
        ranks = [1] + [r] * 7 + [1]
        cores = [torch.from_numpy((rng.standard_normal((ranks[k], 100, ranks[k + 1])) / math.sqrt(ranks[k]))
                                  .astype(np.float32)).to(dev) for k in range(8)]
        g = torch.from_numpy(rng.standard_normal(m).astype(np.float32)).to(dev)
        grads = [torch.zeros_like(c) for c in cores]
        for _ in range(2):
            F.tt_eval_at(cores, idx)
            F.tt_eval_backward(cores, idx, g, grads)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        F.tt_eval_at(cores, idx)
        e[1].record(stream)
        F.tt_eval_backward(cores, idx, g, grads)
        e[2].record(stream)
        torch.cuda.synchronize()
        fwd, bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        # algorithmic HBM bytes: indices (8 x 4 B) + upstream gradient (4 B) per entry, cores L2-resident
        bytes_bwd = m * (8 * 4 + 4)
        flops_bwd = m * (2 * 2 * sum(ranks[k] * ranks[k + 1] for k in range(8)) + 2 * sum(ranks[k] * ranks[k + 1] for k in range(8)))
        # the binding roof: ranks >= 16 take the index-sorted GEMM path (FP32 FFMA bound);
        # the algorithmic flops are those of the two partial sweeps and the gradient
        flops_sorted = m * 2.0 * 3.0 * sum(ranks[k] * ranks[k + 1] for k in range(8))
        out[f"rank{r}"] = {"eval_ms": fwd, "backward_ms": bwd, "backward_gbs": bytes_bwd / (bwd / 1e3) / 1e9,
                           "backward_hbm_frac": bytes_bwd / (bwd / 1e3) / 1e9 / hbm,
                           "backward_tflops": flops_bwd / (bwd / 1e3) / 1e12,
                           "backward_fp32_frac": flops_sorted / (bwd / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                           "path": "index-sorted GEMM tiles" if r >= 16 else "one thread/warp per entry"}
        if r == 8:   # the fitting runs after every other measurement (see run_ours)
            out["_fit_args"] = (cores, idx, w, m)
    return out


def _fit(F, cores, idx, w, dev, stream, m, steps=3, lr=1e-9):
    """Gradient-descent fitting (tt_fit_gd) of the rank-8 FP32 TT to the workload's 1e7
    values: time per step (evaluation, residual, adjoint, descent).  A small step keeps
    the measurement away from divergence; a failure is reported in the object."""
    import math
    import torch
    try:
        vals = torch.from_numpy(w.vals).to(dev)
        fc = [c.clone() for c in cores]
        F.tt_fit_gd(fc, idx, vals, 1, lr)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        losses = F.tt_fit_gd(fc, idx, vals, steps, lr)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        fin = [float(x) if math.isfinite(x) else None for x in (losses[0], losses[-1])]
        return {"steps": steps, "lr": lr, "ms_per_step": ms, "entries_per_s": m / (ms / 1e3),
                "loss_first": fin[0], "loss_last": fin[1]}
    except Exception as e:   # reported, never hidden
        return {"error": str(e)[:300]}


def _next_rows(F, dev, stream):
    """One timed decomposition for each extension and further workload that runs through
    fasttt_decompose: dynamic truncation (Alg. 8) on the 50^5 workload; the FDM 7-point
    matrices of Table 2 (3-way MPO, p = 2, eps = 1e-14) at n = 20, 30, 40; the banded
    2^20 x 2^20 matrix as a 20-way QTT through the exact grouping (S1-S5, Alg. 9 over all
    20 splits).  Each after one warm-up call; failures are reported in the object."""
    import torch
    from paper_1908_02721_gb300 import workloads as W

    def timed(call):
        call().free()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tt = call()
        e1.record(stream)
        torch.cuda.synchronize()
        return tt, e0.elapsed_time(e1)

    out = {}
    try:
        w = W.uniform5(seed=2)
        idx, vals = torch.from_numpy(w.idx).to(dev), torch.from_numpy(w.vals).to(dev)
        tt, ms = timed(lambda: F.fasttt_decompose(idx, vals, w.dims, w.eps, rounding="dynamic"))
        st = tt.stats
        out["dynamic_alg8"] = {"workload": "5-way 50^5, 1e5 nnz, eps 1e-8, FP64", "ms": ms,
                               "nnz_per_s": w.nnz / (ms / 1e3), "ranks": tt.ranks,
                               "err_bound_used": (st["err2"] / st["norm2"]) ** 0.5}
        tt.free()
    except Exception as e:
        out["dynamic_alg8"] = {"error": str(e)[:300]}
    fdm = {}
    for n in (20, 30, 40):
        for coeffs in ("pattern", "random"):
            key = f"n{n}_{coeffs}"
            try:
                w = W.fdm7(n, coeffs)
                idx, vals = torch.from_numpy(w.idx).to(dev), torch.from_numpy(w.vals).to(dev)
                tt, ms = timed(lambda: F.fasttt_decompose(idx, vals, w.dims, w.eps, p=2))
                fdm[key] = {"nnz": w.nnz, "ms": ms, "R": tt.stats["R"], "rt": tt.stats["rt"], "ranks": tt.ranks}
                tt.free()
            except Exception as e:
                fdm[key] = {"error": str(e)[:300]}
    out["fdm7_table2"] = fdm
    qtt = {}
    try:   # the sparse-matrix -> QTT workload at full size: S1-S5 (exact grouping, Alg. 9 over all 20 splits)
        w = W.banded_qtt(20)
        idx, vals = torch.from_numpy(w.idx).to(dev), torch.from_numpy(w.vals).to(dev)
        tt, ms = timed(lambda: F.fasttt_decompose(idx, vals, w.dims, w.eps, stage="exact"))
        st = tt.stats
        qtt["m20_exact_grouping"] = {"workload": w.name, "nnz": w.nnz, "ms": ms, "nnz_per_s": w.nnz / (ms / 1e3),
                                     "p": st["p"], "R": st["R"], "rt_max": max(st["rt"])}
        tt.free()
    except Exception as e:
        qtt["m20_exact_grouping"] = {"error": str(e)[:300]}
    out["banded_qtt"] = qtt
    return out


def _tt_round(F, dev, stream, reps=3):
    """TT-rounding (Alg. 2) of the Lemma 2 sum S = A + B of two random 8-way 100^8 FP64
    TTs of rank 64 (geometrically decaying bond spectra), ranks 128 in, eps = 1e-6.
    Self-check through the library alone: the rounded R must satisfy
    ||R - S||^2 = err2 (the truncations are orthogonal), with ||R - S|| taken from
    the numerical-rank rounding of the Lemma 2 difference R - S."""
    import math
    import torch
    from paper_1908_02721_gb300 import workloads as W
    dims, ranks = [100] * 8, [1] + [64] * 7 + [1]
    a = [torch.from_numpy(c).to(dev) for c in W.random_tt(dims, ranks, seed=501, decay=0.75)]
    b = [torch.from_numpy(c).to(dev) for c in W.random_tt(dims, ranks, seed=502, decay=0.75)]
    S = F.tt_add(a, b)
    eps = 1e-6
    F.tt_round(S, eps).free()
    times = []
    R = None
    for _ in range(reps):
        if R is not None:
            R.free()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R = F.tt_round(S, eps)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    st = R.stats
    Dlt = F.tt_add(R, S, beta=-1.0)
    dn2 = F.tt_round(Dlt, 0.0).stats["norm2"]
    out = {"workload": "A + B, two random 8-way 100^8 FP64 TTs of rank 64 (Lemma 2 sum, ranks 128), eps 1e-6",
           "ms": sorted(times)[len(times) // 2], "ranks_in": S.ranks, "ranks_out": R.ranks,
           "err2_rel": st["err2"] / st["norm2"], "measured_err_rel": math.sqrt(max(dn2, 0.0) / st["norm2"]),
           "stages_ms": {k: st[k] for k in ("ms_gemm_oz", "ms_gemm", "ms_jacobi", "ms_tsqr", "ms_tridiag32",
                                             "ms_tdeig")},
           "launches": st["launches"]}
    for h in (R, S, Dlt):
        h.free()
    return out


def _e2e(args, w, F, dev, barrier, world):
    """Same call from pinned host buffers: H2D of the COO input and D2H of every core timed."""
    import torch
    idx_h = torch.from_numpy(w.idx).pin_memory()
    vals_h = torch.from_numpy(w.vals).pin_memory()
    e2e_ms, d2h, host = [], 0, None
    for i in range(args.steps + 1):
        barrier()
        t = time.perf_counter()
        di = idx_h.to(dev, non_blocking=True)
        dv = vals_h.to(dev, non_blocking=True)
        tt = F.fasttt_decompose(di, dv, w.dims, w.eps)
        if host is None:
            host = [torch.empty(tt.ranks[k - 1] * w.dims[k - 1] * tt.ranks[k], dtype=torch.float64).pin_memory()
                    for k in range(1, w.d + 1)]
        for k in range(1, w.d + 1):
            F._check(F._lib.fasttt_tt_copy(tt._h, F.ARR["core"], k, host[k - 1].data_ptr(), host[k - 1].numel()))
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        d2h = sum(h.numel() * 8 for h in host)
        tt.free()
        if i > 0:                      # the first pass also pins the host buffers
            e2e_ms.append(el * 1e3)
    e2e = sum(e2e_ms) / len(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e = float(t.item())
    return {"value": w.nnz * world / (e2e / 1e3), "unit": "nnz/s",
            "h2d_bytes_per_step": int(w.idx.nbytes + w.vals.nbytes), "d2h_bytes_per_step": int(d2h)}


PROFILE_CASES = ("grouping-qtt18", "adjoint-zipf1e6-r64", "decompose-qtt12", "decompose-qtt12-mixed",
                 "decompose-uniform5")


def run_profile_case(case):
    """One call of one case, for profiler captures (no timing loop, no other lines):
    grouping-qtt18: the banded 2^18 QTT (2.6e6 nonzeros) through value Depar (S1-S6);
    adjoint-zipf1e6-r64: evaluation + adjoint of a rank-64 FP32 TT on 1e6 Zipf(1.2) entries
    of the 100^8 tensor; decompose-qtt12[-mixed]: the headline decomposition once;
    decompose-uniform5: the 50^5, 1e5-nonzero decomposition once."""
    import math
    import numpy as np
    import torch
    from paper_1908_02721_gb300 import fasttt as F
    from paper_1908_02721_gb300 import workloads as W
    torch.cuda.set_device(0)
    if case == "adjoint-zipf1e6-r64":
        w = W.zipf_tt(nnz=1_000_000)
        idx = torch.from_numpy(w.idx).cuda()
        rng = np.random.Generator(np.random.Philox(key=464))
        ranks = [1] + [64] * 7 + [1]
        cores = [torch.from_numpy((rng.standard_normal((ranks[k], 100, ranks[k + 1])) / math.sqrt(ranks[k]))
                                  .astype(np.float32)).cuda() for k in range(8)]
        g = torch.from_numpy(rng.standard_normal(w.nnz).astype(np.float32)).cuda()
        a = F.tt_eval_at(cores, idx)
        F.tt_eval_backward(cores, idx, g)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": case, "checksum": float(a.abs().sum())}))
        return
    if case == "grouping-qtt18":
        w, kw = W.banded_qtt(18), {"stage": "depar", "keep_intermediates": True}
    elif case == "decompose-uniform5":
        w, kw = W.uniform5(seed=2), {}
    else:
        w, kw = W.banded_qtt(HEADLINE_M), {"precision": "mixed" if case.endswith("mixed") else "fp64"}
    idx = torch.from_numpy(w.idx).cuda()
    vals = torch.from_numpy(w.vals).cuda()
    tt = F.fasttt_decompose(idx, vals, w.dims, w.eps, **kw)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "ranks": tt.ranks, "ms_total": tt.stats["ms_total"]}))
    tt.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision pass")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-tt-round", action="store_true", help="skip the TT-rounding (Alg. 2) measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the other configurations")
    ap.add_argument("--no-config5", action="store_true", help="skip the 5e7-nonzero configuration")
    ap.add_argument("--workload", default="qtt12", choices=["qtt12", "qtt10"],
                    help="qtt10: the same recipe at 2^10 x 2^10, for profiler captures only")
    ap.add_argument("--profile-case", choices=PROFILE_CASES,
                    help="run one case once for a profiler capture and exit")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
