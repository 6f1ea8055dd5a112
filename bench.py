#!/usr/bin/env python3
"""HT truncation throughput on GB300: HT addition + HSVD truncation per step.

One step = ht_add (Lemma "sum of two H-tensors") of seeded HT tensor pairs
followed by the truncation of each sum (orthogonalization, reduced Gramians,
eigendecompositions, rank selection, projection), replayed as one CUDA graph
(ht_graph_add_truncate / ht_graph_launch).  Workloads (--config):

  deep     d=256, n=4096, k=64 -> rank 128, Gaussian leaves,
           sigma_j = 10^(-10j/64), eps = 1e-6 relative (default)
  single   d=64, n=1000, k=32 -> rank 64, orthonormal Gaussian leaves,
           sigma_j = 10^(-8j/32), eps = 1e-8 relative, rank cap 32
  small    256 pairs of d=8, n=32, k=8 -> rank 16, Gaussian leaves,
           sigma_j = 2^-j, truncated to rank 8
  batched  a wave of uneven tensors, d~U{4..32}, n~U{16..512}, k~U{4..48},
           each the sum of 4 tensors (sigma_j = 2^-j) truncated to its own k
  wide     8 pairs of d=16, n=2048, k=128 -> rank 256, orthonormal leaves,
           sigma_j = j^-2, truncated to rank 128

Arms (all on the same workload):
  value              the mixed-precision path (HT_PREC_MIXED: F64 storage,
                     FP64 QR blocks and eigensolves, contractions on the tcgen05
                     tensor cores by exact BF16 slicing), one batched launch
                     per tree level, CUDA-graph replay
  fp32_path          FP32 storage and contractions (HT_PREC_FP32)
  plain_fp64_*       every step in FP64 on the SIMT pipes, one launch per level
                     and one launch per tree node
  errors             each path's results against the CPU FP64 oracle on the
                     workload's first pair (the oracle run is also the
                     cpu_baseline timing)
  --impl reference   the CPU FP64 oracle on the host cores (rank 0 only)

Multi-GPU (torchrun): every rank truncates its own tensors (independent
problems, weak scaling); no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_03340_gb300 import inputs as I  # noqa: E402

METRIC = "HT truncations/s + roofline fraction, mixed vs plain FP64 GPU at stated rel err"
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.070e9  # SMs x FP32 lanes x 2 flop x max clock (80.5 TFLOP/s)


# ---------------------------------------------------------------------------
# workloads: each yields, per rank, a list of pairs (d, n, (ka, xa), (kc, xc), cap)
# ---------------------------------------------------------------------------

def _pairs_single(rank, args):
    (n, ka, xa), (_, kc, xc) = I.single_pair(11 + 1000 * rank)
    return [(64, n, (ka, xa), (kc, xc), 32)]


def _pairs_small(rank, args):
    out = []
    for i in range(args.pairs or 256):
        (n, ka, xa), (_, kc, xc) = I.small_pair(1 + 2 * i + 100000 * rank)
        out.append((8, n, (ka, xa), (kc, xc), 8))
    return out


def _pairs_deep(rank, args):
    (n, ka, xa), (_, kc, xc) = I.deep_pair(21 + 1000 * rank)
    return [(256, n, (ka, xa), (kc, xc), 0)]


def _pairs_wide(rank, args):
    out = []
    for i in range(args.pairs or 8):
        (n, ka, xa), (_, kc, xc) = I.wide_pair(31 + 2 * i + 1000 * rank)
        out.append((16, n, (ka, xa), (kc, xc), 128))
    return out


def _batched_specs(rank, args):
    wave = args.pairs or 64
    specs = I.batched_specs(count=4096, seed=41)
    return [specs[(rank * wave + i) % len(specs)] for i in range(wave)]


WORKLOADS = {
    "single": dict(pairs=_pairs_single, opts=I.SINGLE_OPTS,
                   desc="d=64, n=1000, k=32 -> rank 64 after the addition, orthonormal Gaussian leaves, "
                        "sigma_j=10^(-8j/32), eps=1e-8 relative, rank cap 32"),
    "small": dict(pairs=_pairs_small, opts=dict(mode="rank", rank_cap=8),
                  desc="pairs of d=8, n=32, k=8 -> rank 16, Gaussian leaves, sigma_j=2^-j, truncated to rank 8"),
    "batched": dict(pairs=None, opts=dict(mode="rank"),
                    desc="uneven tensors d~U{4..32}, n~U{16..512}, k~U{4..48}, each the sum of 4 tensors "
                         "(Gaussian leaves, sigma_j=2^-j, rank 4k) truncated to its own k"),
    "deep": dict(pairs=_pairs_deep, opts=I.DEEP_OPTS,
                 desc="d=256, n=4096, k=64 -> rank 128, Gaussian leaves, sigma_j=10^(-10j/64), eps=1e-6 relative"),
    "wide": dict(pairs=_pairs_wide, opts=I.WIDE_OPTS,
                 desc="pairs of d=16, n=2048, k=128 -> rank 256, orthonormal Gaussian leaves, sigma_j=j^-2, "
                      "truncated to rank 128"),
}

# DRAM bytes (read + write) per launch of the dominant kernel family, averaged
# over one step's launches of that family (17 TSQR, 39 contraction launches),
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernels on the same workload; None where not captured.
TRAFFIC_PER_LAUNCH = {("single", "gemm"): 15.56e6, ("single", "qr"): 6.27e6}


def model_flops(d, n, K, r):
    """Algorithmic work of one truncation: 12 K^4 per non-root inner node +
    n K (K + 2r) per leaf; eigen counted separately (9 K^3 per non-root node)."""
    inner = (d - 2) * 12.0 * K ** 4
    leaves = d * n * K * (K + 2 * r)
    eig = (2 * d - 2) * 9.0 * K ** 3
    return inner + leaves, eig


def job_value(local_ms, tensors_per_step, steps, ws, reduce_max):
    """Whole-job throughput of a weak-scaled run: every rank truncates its own
    tensors_per_step tensors per step; the job's time is the slowest rank's
    (reduce_max: max over ranks).  Returns (truncations/s, job ms)."""
    ms = reduce_max(local_ms)
    return ws * tensors_per_step * steps / (ms / 1e3), ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def start_clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL)
    except Exception:
        return None, None
    # the timed region of a short run lasts well under a second: start it only
    # once the sampler writes (at most 3 s of waiting)
    t0 = time.time()
    while time.time() - t0 < 3.0 and proc.poll() is None:
        try:
            if os.path.getsize(path) > 0:
                break
        except OSError:
            break
        time.sleep(0.01)
    return proc, f


def read_clocks(proc, f, path, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except Exception:
        proc.kill()
    f.close()
    mhz, maxm, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9:
            continue
        try:
            if int(p[0]) != gpu_index:
                continue
            mhz.append(float(p[1]))
            maxm.append(float(p[2]))
        except ValueError:
            continue
        for nm, v in zip(names, p[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not mhz:
        return None
    return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": float(max(maxm)), "reasons": sorted(reasons),
            "samples": len(mhz)}


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------

def oracle_sample(config, rank, args, bounded=False):
    """A bounded sample of the workload for the CPU oracle: a list of
    (d, n, (ka, xa), (kc, xc), opts) summand pairs, its description, and the
    number of workload tensors one pass over it stands for.  bounded (the
    reference arm, whose every step must be short): the single-tensor
    workloads whose one truncation takes the oracle tens of seconds are
    sampled by a smaller tensor of the same recipe, its rate rescaled to the
    full tensor by the modelled work (model_flops, eigen included)."""
    from oracle import oracle as O
    wl = WORKLOADS[config]
    items = []
    if bounded and config in ("deep", "wide"):
        # the same tree (the oracle parallelises over a level's nodes, so a
        # smaller d would leave cores idle and understate it) with half the
        # rank; smaller blocks cache better, so if anything this overstates
        # the oracle's rate
        if config == "deep":  # k = 32 instead of 64 (rank 64 after the addition): d, n, decay and eps unchanged
            (n, ka, xa), (_, kc, xc) = I.deep_pair(21, k=32)
            items.append((256, n, (ka, xa), (kc, xc), I.DEEP_OPTS))
            small, full = model_flops(256, 4096, 64, 32), model_flops(256, 4096, 128, 64)
            desc = "1 add + truncate of the deep recipe at k = 32 (d, n, decay and eps unchanged), FP64"
        else:  # k = 64 instead of 128: rank 128 after the addition, truncated to 64
            (n, ka, xa), (_, kc, xc) = I.wide_pair(31, k=64)
            items.append((16, n, (ka, xa), (kc, xc), dict(mode="rank", rank_cap=64)))
            small, full = model_flops(16, 2048, 128, 64), model_flops(16, 2048, 256, 128)
            desc = "1 add + truncate of the wide recipe at k = 64 (rank 128 truncated to 64), FP64"
        ratio = sum(small) / sum(full)
        return items, desc + f", rate rescaled to the full tensor by modelled work (x {ratio:.4f})", ratio
    if config == "batched":
        # tensors of the wave in order, skipping those above twice the mean
        # modelled cost, until about 15 GFLOP; the rate is rescaled to the
        # wave's mean tensor by modelled flops
        wave = _batched_specs(rank, args)
        cost = lambda sp: model_flops(sp[0], sp[1], 4 * sp[2], sp[2])[0]
        mean = float(np.mean([cost(sp) for sp in wave]))
        picked, total = [], 0.0
        for sp in wave:
            if cost(sp) <= 2 * mean:
                picked.append(sp)
                total += cost(sp)
            if total >= 15e9 or len(picked) == 4:
                break
        for (d, n, k, s) in picked:
            terms = I.batched_terms((d, n, k, s))
            nv = terms[0][0]
            a = O.add(d, nv, terms[0][1], terms[0][2], terms[1][1], terms[1][2])
            c = O.add(d, nv, terms[2][1], terms[2][2], terms[3][1], terms[3][2])
            items.append((d, nv, a, c, dict(mode="rank", rank_cap=k)))
        desc = (f"{len(picked)} tensors of the batched wave ((d, n, k) = {[sp[:3] for sp in picked]}, each "
                f"(T1+T2)+(T3+T4), add + truncate, FP64), rate rescaled to the wave's mean tensor by modelled flops")
        return items, desc, total / mean
    for (d, n, (ka, xa), (kc, xc), cap) in wl["pairs"](rank, argparse.Namespace(pairs=1))[:1]:
        items.append((d, n, (ka, xa), (kc, xc), wl["opts"]))
    return items, "1 add + truncate of the workload's first pair, FP64", float(len(items))


def oracle_time(items, reps):
    """Seconds for `reps` passes of add + truncate over the sample."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    for _ in range(reps):
        for (d, n, (ka, xa), (kc, xc), opts) in items:
            k, x = O.add(d, n, ka, xa, kc, xc)
            O.truncate(d, n, k, x, **opts)
    return time.perf_counter() - t0


def run_reference(args):
    from oracle import oracle as O
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = O.set_threads(0)
    items, sample, equiv = oracle_sample(args.config, 0, args, bounded=True)
    for _ in range(args.warmup):
        oracle_time(items, 1)
    secs = oracle_time(items, args.steps)
    value = args.steps * equiv / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "truncations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "shape": WORKLOADS[args.config]["desc"]},
        "cpu_baseline": {"value": value, "unit": "truncations/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step: {sample}"},
        "e2e": {"value": value, "unit": "truncations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arms
# ---------------------------------------------------------------------------

def build_pairs(htgb, config, rank, args, dtype, stream):
    """Device tensors: summands A_i, C_i and outputs X_i (capacity = sum of ranks);
    returns (trees, A, C, X, caps, shapes) with shapes (d, n, K) per output."""
    trees, A, C, X, caps, shapes = {}, [], [], [], [], []
    if config == "batched":
        for (d, n, k, s) in _batched_specs(rank, args):
            tr = trees.setdefault(d, htgb.HTTree(d))
            T = [htgb.HTTensor.from_blob(tr, nv, kv, xv, dtype, stream) for (nv, kv, xv) in I.batched_terms((d, n, k, s))]
            A.append(T[0].add(T[1]))
            C.append(T[2].add(T[3]))
            caps.append(k)
            shapes.append((d, n, 4 * k))
    else:
        for (d, n, (ka, xa), (kc, xc), cap) in WORKLOADS[config]["pairs"](rank, args):
            tr = trees.setdefault(d, htgb.HTTree(d))
            A.append(htgb.HTTensor.from_blob(tr, n, ka, xa, dtype, stream))
            C.append(htgb.HTTensor.from_blob(tr, n, kc, xc, dtype, stream))
            caps.append(cap)
            shapes.append((d, int(np.asarray(n).flat[0]), int(np.max(ka)) + int(np.max(kc))))
    for a, c in zip(A, C):
        k = np.asarray(a.ranks()) + np.asarray(c.ranks())
        k[0] = 1
        X.append(htgb.HTTensor.create(a.tree, a.n, k, dtype, stream))
    return trees, A, C, X, caps, shapes


def make_opts(htgb, config, prec, caps, sched=None, extra=None):
    kw = dict(WORKLOADS[config]["opts"])
    kw.update(extra or {})
    if config == "batched":
        kw["tensor_caps"] = caps
    if sched is not None:
        kw["schedule"] = sched
    return htgb.make_opts(prec=prec, **kw)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="deep", choices=sorted(WORKLOADS))
    ap.add_argument("--pairs", type=int, default=0, help="tensors per step (small: 256, batched: 64, wide: 8)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison arms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-errors", action="store_true", help="skip the error statement against the oracle")
    ap.add_argument("--ncu-step", default=None, choices=["mixed", "fp64", "fp32"],
                    help="for ncu --profile-from-start off: one warm truncation of the workload's first pair, then "
                         "one between cudaProfilerStart and cudaProfilerStop, and exit")
    ap.add_argument("--modes", type=int, default=0, help="deep workload only: number of modes d (default 256)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_step:
        return ncu_step(args)

    import torch
    from paper_1708_03340_gb300 import htgb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2 (129 MB)

    def max_over_ranks(v):
        if ws == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def graph_arm(dtype, prec, steps, warmup, sched=None, extra=None):
        """Timed graph replays: per step, L2 flush then one replay between CUDA events."""
        trees, A, C, X, caps, shapes = build_pairs(htgb, args.config, rank, args, dtype, stream)
        opts = make_opts(htgb, args.config, prec, caps, sched, extra)
        g = htgb.ht_graph_add_truncate([a.handle for a in A], [c.handle for c in C], [x.handle for x in X], opts)
        for _ in range(warmup):
            htgb.ht_graph_launch(g)
        barrier()
        l0 = htgb.ht_launch_count()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            htgb.ht_graph_launch(g)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        launches = htgb.ht_launch_count() - l0
        value, ms = job_value(sum(a.elapsed_time(b) for a, b in evs), len(X), steps, ws, max_over_ranks)
        return dict(ms=ms, value=value, launches=launches, g=g, A=A, C=C, X=X, caps=caps, shapes=shapes, opts=opts,
                    trees=trees)

    def profiled_arm(dtype, prec, steps, sched=None):
        """Direct calls (ht_add_into + ht_truncate_batch) with per-kernel-family CUDA events."""
        trees, A, C, X, caps, shapes = build_pairs(htgb, args.config, rank, args, dtype, stream)
        opts = make_opts(htgb, args.config, prec, caps, sched)

        def step():
            for x, a, c in zip(X, A, C):
                x.add_into(a, c)
            htgb.ht_truncate_batch([x.handle for x in X], opts)

        step()
        barrier()
        mask = (1 << len(htgb.KERNEL_KINDS)) - 1
        htgb.ht_profile_set(mask)
        for kind in range(len(htgb.KERNEL_KINDS)):
            htgb.ht_profile_read(kind, reset=True)
        l0 = htgb.ht_launch_count()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        htgb.ht_profile_set(0)
        prof = {}
        for kind, name in enumerate(htgb.KERNEL_KINDS):
            cnt, tms, fl = htgb.ht_profile_read(kind, reset=True)
            if cnt:
                prof[name] = {"launches": cnt, "ms": tms, "flops": fl}
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs))
        return dict(ms=ms, launches=htgb.ht_launch_count() - l0, prof=prof, X=X)

    # ---- unit peaks of this GPU (roofline denominators the measured peak file lacks)
    peaks = measured_peaks() if rank == 0 else {}

    # ---- headline: graph replays of the mixed-precision path
    clk_path = os.path.join(tempfile.gettempdir(), f"htgb_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path)
    main_arm = graph_arm(htgb.HT_F64, htgb.HT_PREC_MIXED, args.steps, args.warmup)
    clocks = read_clocks(proc, fh, clk_path, local)
    per_step = len(main_arm["X"])
    value = main_arm["value"]
    ms_per_step = main_arm["ms"] / args.steps
    work = 0.0
    for (d, n, K), cap in zip(main_arm["shapes"], main_arm["caps"]):
        w, _ = model_flops(d, n, K, cap or K // 2)
        work += w

    # ---- kernel breakdown and the roofline of the dominant kernel family
    psteps = max(2, min(args.steps, 4))
    prof = profiled_arm(htgb.HT_F64, htgb.HT_PREC_MIXED, psteps)
    roofline = roofline_of(prof["prof"], psteps, peaks)

    line = {
        "metric": METRIC, "value": value, "unit": "truncations/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (contractions: bf16 slices, fp32 accumulate)",
        "data": "synthetic (seeded SplitMix64/Box-Muller HT tensors)",
        "config": {"workload": args.config, "tensors_per_step": per_step, "shape": WORKLOADS[args.config]["desc"],
                   "l2": "flushed between steps (256 MB write)",
                   "path": "mixed: F64 storage, double-float TSQR blocks (FP32 pipe, 2^-47), FP64 QL eigensolves "
                           "(eigenvectors in double-float), "
                           "every contraction on tcgen05 (5 BF16 slices per FP64 operand, exact leading sums), "
                           "one batched launch per level, "
                           "CUDA-graph replay"},
        "gflops": work / (ms_per_step / 1e3) / 1e9,
        "direct_calls_ms_per_step": prof["ms"] / psteps,
        "kernel_ms_per_step": {k: v["ms"] / psteps for k, v in prof["prof"].items()},
        "kernel_launches_per_step": {k: v["launches"] / psteps for k, v in prof["prof"].items()},
        "ranks_first_nodes": [int(v) for v in main_arm["X"][0].ranks()[:8]],
        "gpu_launches": main_arm["launches"],
        "roofline": roofline,
        "unit_peaks": peaks,
        "clocks": clocks,
    }

    # ---- comparison arms on the same workload
    trim_pool()
    if not args.no_plain:
        fs = max(3, args.steps // 2)
        f32 = graph_arm(htgb.HT_F32, htgb.HT_PREC_FP32, fs, 3)
        line["fp32_path"] = {"value": f32["value"], "unit": "truncations/s", "ms_per_step": f32["ms"] / fs}
        htgb.ht_graph_free(f32["g"])
        trim_pool()
        # the mixed path with FP64 Householder QR blocks instead of the double-float ones
        mq = graph_arm(htgb.HT_F64, htgb.HT_PREC_MIXED, fs, 3, extra={"qr_kernel": 3})
        line["mixed_fp64_qr"] = {"value": mq["value"], "unit": "truncations/s", "ms_per_step": mq["ms"] / fs,
                                 "note": "HT_PREC_MIXED with qr_kernel 3: TSQR blocks in FP64 Householder"}
        htgb.ht_graph_free(mq["g"])
        trim_pool()
        ps = 2 if args.config in ("deep", "wide") else 3
        plain = profiled_arm(htgb.HT_F64, htgb.HT_PREC_FP64, ps)
        line["plain_fp64_level"] = {"value": ws * per_step * ps / (plain["ms"] / 1e3), "unit": "truncations/s",
                                    "ms_per_step": plain["ms"] / ps,
                                    "kernel_ms_per_step": {k: v["ms"] / ps for k, v in plain["prof"].items()}}
        trim_pool()
        ns = 1 if args.config in ("deep", "wide") else 3
        node = graph_arm(htgb.HT_F64, htgb.HT_PREC_FP64, ns, 1, sched=htgb.HT_SCHED_NODE)
        line["plain_fp64_per_node"] = {"value": node["value"], "unit": "truncations/s",
                                       "ms_per_step": node["ms"] / ns, "launches_per_step": node["launches"] / ns,
                                       "steps": ns, "warmup": 1}
        htgb.ht_graph_free(node["g"])
        line["speedup_vs_plain_per_node"] = value / line["plain_fp64_per_node"]["value"]
        line["speedup_vs_plain_level"] = value / line["plain_fp64_level"]["value"]
        line["speedup_vs_fp32_path"] = value / line["fp32_path"]["value"]
        line["speedup_vs_mixed_fp64_qr"] = value / line["mixed_fp64_qr"]["value"]

    # ---- end to end through the public API: pinned host blobs in, truncated blobs out, every step
    A, C, X, g = main_arm["A"], main_arm["C"], main_arm["X"], main_arm["g"]
    hA = [torch.from_numpy(a.download()).pin_memory() for a in A]
    hC = [torch.from_numpy(c.download()).pin_memory() for c in C]
    cap_sz = []
    for a, c in zip(A, C):  # room for the largest possible output: the capacity of the sum
        k = np.asarray(a.ranks()) + np.asarray(c.ranks())
        k[0] = 1
        cap_sz.append(int(I.blob_size(a.tree.d, a.n, k)))
    hX = [torch.empty(max(s_, 1), dtype=torch.float64).pin_memory() for s_ in cap_sz]
    e2e_steps = max(3, args.steps // 2)
    h2d = sum(t.numel() * 8 for t in hA + hC)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        for a, c, ha, hc in zip(A, C, hA, hC):
            htgb.ht_tensor_upload(a.handle, ha.numpy())
            htgb.ht_tensor_upload(c.handle, hc.numpy())
        htgb.ht_graph_launch(g)
        d2h = 0
        for x, hx in zip(X, hX):
            sz = htgb.ht_tensor_blob_size(x.handle)
            htgb.ht_tensor_download(x.handle, hx.numpy()[:sz])
            d2h += sz * 8
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    line["e2e"] = {"value": ws * per_step * e2e_steps / e2e_s, "unit": "truncations/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    htgb.ht_graph_free(g)

    # ---- CPU oracle baseline (rank 0, N = 1 only), a bounded sample; its
    # result on the workload's first pair is the reference of the error statement
    if ws == 1 and not args.no_cpu:
        from oracle import oracle as O
        cores = O.set_threads(0)
        items, sample, equiv = oracle_sample(args.config, 0, args)
        t0 = time.perf_counter()
        ref = None
        (d0, n0, (ka0, xa0), (kc0, xc0), opts0) = items[0]
        k0, x0 = O.add(d0, n0, ka0, xa0, kc0, xc0)
        ref = O.truncate(d0, n0, k0, x0, **opts0)
        for it in items[1:]:
            oracle_time([it], 1)
        secs = time.perf_counter() - t0
        reps = 1
        while secs * (reps + 1) / reps < 10.0 and reps < 8:  # about 10 s of CPU work
            secs += oracle_time(items, 1)
            reps += 1
        line["cpu_baseline"] = {"value": reps * equiv / secs, "unit": "truncations/s", "cores": cores,
                                "kind": "oracle", "sample": f"{reps} x {sample}, OpenMP over tree nodes"}
        if args.config != "batched" and not args.no_errors:
            trim_pool()
            try:
                line["errors_vs_oracle"] = errors_vs_oracle(htgb, stream, (d0, n0, ka0, xa0, kc0, xc0, opts0, k0, x0),
                                                            ref)
            except Exception as e:  # the line is printed either way, with the reason
                line["errors_vs_oracle"] = {"unavailable": str(e)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def ncu_step(args):
    """One warm truncation of the workload's first pair, then one bracketed by
    cudaProfilerStart / cudaProfilerStop (direct calls, no graph), so that
    `ncu --profile-from-start off` sees exactly one truncation's launches."""
    import torch
    from paper_1708_03340_gb300 import htgb
    prec = {"mixed": htgb.HT_PREC_MIXED, "fp64": htgb.HT_PREC_FP64, "fp32": htgb.HT_PREC_FP32}[args.ncu_step]
    dtype = htgb.HT_F32 if args.ncu_step == "fp32" else htgb.HT_F64
    if args.config == "deep" and args.modes:
        (n, ka, xa), (_, kc, xc) = I.deep_pair(21, d=args.modes)
        d = args.modes
        opts = I.DEEP_OPTS
    else:
        (d, n, (ka, xa), (kc, xc), _) = WORKLOADS[args.config]["pairs"](0, argparse.Namespace(pairs=1))[0]
        opts = WORKLOADS[args.config]["opts"]
    tree = htgb.HTTree(d)
    A = htgb.HTTensor.from_blob(tree, n, ka, xa, dtype)
    C = htgb.HTTensor.from_blob(tree, n, kc, xc, dtype)
    k = np.asarray(A.ranks()) + np.asarray(C.ranks())
    k[0] = 1
    X = htgb.HTTensor.create(tree, n, k, dtype)
    o = htgb.make_opts(prec=prec, **opts)
    X.add_into(A, C)
    htgb.ht_truncate(X.handle, o)
    X.add_into(A, C)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    htgb.ht_truncate(X.handle, o)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    htgb.ht_device_status()
    print(json.dumps({"ncu_step": args.ncu_step, "config": args.config, "d": d, "seconds": time.perf_counter() - t0}))
    return 0


def trim_pool():
    """Hand the unused memory the library's stream-ordered pool keeps back to
    the device (the library keeps freed workspace for reuse; the arms of this
    benchmark differ in size)."""
    try:
        import ctypes
        import torch
        from paper_1708_03340_gb300 import htgb
        htgb.load()
        rt = ctypes.CDLL("libcudart.so.13")
        pool = ctypes.c_void_p()
        torch.cuda.synchronize()
        if rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0:
            rt.cudaMemPoolTrimTo(pool, ctypes.c_size_t(0))
    except Exception:
        pass


def measured_peaks():
    """Unit throughputs measured on this GPU by peaks/peaks.cu (FP64 and FP32
    FMA chains, tcgen05 BF16 and TF32 MMA issue), next to the measured HBM
    and cuBLAS BF16 figures of the pool's peak file.  {} if unavailable."""
    out = {}
    try:
        from paper_1708_03340_gb300.peaks import peaks as PK
        for k, v in PK.run().items():
            out[k] = v["tflops"]
    except Exception as e:  # the roofline then states the nominal figure it used
        out["error"] = str(e)[:200]
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        out["hbm_gbs"] = mp.get("hbm_gbs")
        out["bf16_cublas"] = mp.get("bf16_tflops")
        out["bf16_cublas_sustained"] = mp.get("bf16_tflops_sustained")
    except Exception:
        pass
    return out


# FP32 instructions per FP64-equivalent flop in the double-float QR blocks:
# per entry and reflector a dot-product term (4 for the product, 6 for the
# two-sum, 2 for the low-order sum) and an update (4 + 6 + 2 + 3 for the
# renormalisation), 27 instructions for 2 multiply-adds = 4 flop
DF_FP32_OPS_PER_FLOP = 27.0 / 4.0


def roofline_of(prof, steps, peaks):
    """Roofline object of the dominant kernel family (by device time) of the
    mixed path, measured live with CUDA events on the launching stream.
    Families and their bound:
      qr     TSQR blocks in double-float arithmetic on the FP32 pipe: ALU,
             4 m n^2 - 4 n^3 / 3 FP64-equivalent flop per block against the FP32
             FMA rate over DF_FP32_OPS_PER_FLOP instructions per such flop
      gemm   tensor-core contractions: tensor pipe, the BF16 work of the slice
             products (S (S + 1) / 2 per FP64-equivalent product, 2 M N K each at the
             plan's maximal dims)
      split  BF16 slicing of the contraction operands: HBM, the FP64 operands read
             and their slices written once
      eig    FP64 QL eigensolves (on the mixed path the eigenvector rotations in
             double-float): FP64 ALU, 9 k^3 flop per Gramian"""
    fams = {}
    for name, rec in prof.items():
        if rec["flops"] <= 0 or name not in ("qr", "gemm", "eig", "split"):
            continue
        per_launch_ms = rec["ms"] / rec["launches"]
        work = rec["flops"] / rec["launches"]
        rate = work / (per_launch_ms / 1e3)
        if name == "gemm":
            bound, unit, ach = "tensor", "TFLOP/s", rate / 1e12
            peak = peaks.get("bf16_cublas") or 1880.0
            src = "cuBLAS BF16 burst (measured peak file)"
        elif name == "split":
            bound, unit, ach = "hbm", "GB/s", rate / 1e9
            peak = peaks.get("hbm_gbs") or 6787.6
            src = "HBM copy (measured peak file)"
        elif name == "qr":
            # FP32 lane instructions per second (the FMA rate in flop/s / 2) over the
            # instructions one FP64-equivalent flop costs in the inner loops
            bound, unit, ach = "alu", "TFLOP/s", rate / 1e12
            f32 = peaks.get("fp32_fma")
            src = (f"FP32 FMA chains measured by peaks.cu / 2 / {DF_FP32_OPS_PER_FLOP} FP32 instructions "
                   "per FP64-equivalent flop (double-float dot and update loops)")
            if not f32:
                f32, src = 80.0, "FP32 nominal / 2 / 6.75 (measurement unavailable)"
            peak = f32 / 2.0 / DF_FP32_OPS_PER_FLOP
        else:
            bound, unit, ach = "alu", "TFLOP/s", rate / 1e12
            peak = peaks.get("fp64_fma")
            src = "FP64 FMA chains, measured by peaks.cu on this GPU"
            if not peak:
                peak, src = 1.25, "FP64 nominal (measurement unavailable)"
        fams[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                      "ms_per_step": rec["ms"] / steps, "launches_per_step": rec["launches"] / steps,
                      "ms_per_launch": per_launch_ms, "work_per_launch": work, "peak_source": src}
    if not fams:
        return None
    name = max(fams, key=lambda k: fams[k]["ms_per_step"])
    kernel = {"qr": "qr_df_kernel (double-float TSQR row blocks)",
              "gemm": "oz_gemm_kernel (tcgen05 BF16 slice products) + split-K reduction",
              "split": "oz_split_kernel (BF16 slicing of FP64 operands)",
              "eig": "eig_ql_kernel<double> (FP64 QL, eigenvectors in double-float)"}[name]
    top = dict(fams[name])
    top["kernel"] = kernel
    top["traffic"] = TRAFFIC_PER_LAUNCH.get(("deep", name))
    top["families"] = fams
    return top


def errors_vs_oracle(htgb, stream, pair, ref):
    """Per-result errors of the mixed, FP64 and FP32 paths against the CPU FP64
    oracle's truncation `ref` of the same sum: sigma per node for sigma >=
    1e-5 sigma_max (normwise |sigma_i - sigma_ref_i| / sigma_max and relative
    |sigma_i - sigma_ref_i| / sigma_ref_i), ||X||, the truncated tensors
    ||T(X) - T_ref(X)|| / ||X||, the truncation errors ||X - T(X)|| / ||X||,
    and the nodes whose rank differs with the oracle's energy between the two
    cuts.  Tensor differences are norms of the orthogonalized sum Y + (-Z)
    (mixed path, FP64 storage), never inner products."""
    d, n, ka, xa, kc, xc, opts, k, x = pair
    tree = htgb.HTTree(d)
    nrm = ref["norm"]

    def tensor(kk, blob):
        return htgb.HTTensor.from_blob(tree, n, kk, blob, htgb.HT_F64, stream)

    def diff_norm(k1, y1, k2, y2):
        """||Y - Z|| = ||B_D||_F of the orthogonalized Y + (-Z) (mixed-path
        orthogonalization: FP64 QR blocks, the products to about 1e-12)."""
        P, Q = tensor(k1, y1), tensor(k2, y2)
        Q.scale(-1.0)
        S = P.add(Q)
        S.orthogonalize(htgb.HT_PREC_MIXED)
        ks = S.ranks()
        root = htgb.ht_tensor_node_ptr(S.handle, 0)[1]
        b = S.download()[:root]
        del S, P, Q
        trim_pool()
        return float(np.linalg.norm(b))

    err_ref = diff_norm(k, x, ref["k"], ref["x"]) / nrm
    out = {"oracle_trunc_err": err_ref, "oracle_ranks_first_nodes": [int(v) for v in ref["k"][:8]]}
    for name, dtype, prec in (("mixed", htgb.HT_F64, htgb.HT_PREC_MIXED), ("fp64", htgb.HT_F64, htgb.HT_PREC_FP64),
                              ("fp32", htgb.HT_F32, htgb.HT_PREC_FP32)):
        A = htgb.HTTensor.from_blob(tree, n, ka, xa, dtype, stream)
        C = htgb.HTTensor.from_blob(tree, n, kc, xc, dtype, stream)
        X = A.add(C)
        rep = X.truncate(prec=prec, **opts)
        kt, xt = X.ranks(), X.download().astype(np.float64)
        worst_nw = worst_rel = 0.0
        o = 0
        for t in range(1, 2 * d - 1):
            a = np.asarray(rep["sigma"][o:o + rep["korth"][t]], np.float64)
            o += int(rep["korth"][t])
            b = np.asarray(ref["sigma"][t], np.float64)
            if len(b) and b[0] > 0:
                sel = b >= 1e-5 * b[0]
                worst_nw = max(worst_nw, float(np.max(np.abs(a[sel] - b[sel])) / b[0]))
                worst_rel = max(worst_rel, float(np.max(np.abs(a[sel] - b[sel]) / b[sel])))
        differ = [t for t in range(1, 2 * d - 1) if int(kt[t]) != int(ref["k"][t])]
        energy = 0.0
        for t in differ:
            lo, hi = sorted((int(kt[t]), int(ref["k"][t])))
            energy += float(np.sqrt(np.sum(np.asarray(ref["sigma"][t][lo:hi], np.float64) ** 2)))
        out[name] = {"sigma_normwise": worst_nw, "sigma_relative": worst_rel,
                     "norm": abs(rep["norm"] - nrm) / nrm,
                     "truncated_tensor": diff_norm(kt, xt, ref["k"], ref["x"]) / nrm,
                     "trunc_err": diff_norm(k, x, kt, xt) / nrm,
                     "rank_diff_nodes": len(differ), "rank_diff_energy": energy / nrm,
                     "ranks_first_nodes": [int(v) for v in kt[:8]]}
    return out


if __name__ == "__main__":
    sys.exit(main())
