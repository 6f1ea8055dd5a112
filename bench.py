#!/usr/bin/env python3
"""HT truncation throughput on GB300: HT addition + HSVD truncation per step.

One step = ht_add (Lemma "sum of two H-tensors") of two seeded HT tensors
followed by ht_truncate (orthogonalization, reduced Gramians, FP64
eigendecompositions, rank selection, projection).  Default workload: d=64,
n=1000, k=32 (rank 64 after the addition), orthonormalised Gaussian leaves,
transfer tensors with mode weights sigma_j = 10^(-8j/32), truncation to
relative eps = 1e-8 with rank cap 32.

Arms:
  default            the GB300 library (FP32 storage/contractions + FP64
                     eigensolves, batched per tree level), with the plain FP64
                     path (per level and one launch per node) timed beside it
  --impl reference   the CPU FP64 oracle on the host cores (rank 0 only)

Multi-GPU (torchrun): every rank truncates its own tensors (independent
problems, weak scaling); no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_03340_gb300 import inputs as I  # noqa: E402

WORKLOADS = {
    "single": dict(d=64, n=1000, k=32, make=I.single_pair, opts=I.SINGLE_OPTS,
                   desc="d=64, n=1000, k=32 -> rank 64 after the addition, orthonormal Gaussian leaves, "
                        "sigma_j=10^(-8j/32), eps=1e-8 relative, rank cap 32"),
    "small": dict(d=8, n=32, k=8, make=I.small_pair, opts=dict(mode="rank", rank_cap=8),
                  desc="d=8, n=32, k=8 -> rank 16, Gaussian leaves, sigma_j=2^-j, truncated to rank 8"),
    "deep": dict(d=256, n=4096, k=64, make=I.deep_pair, opts=I.DEEP_OPTS,
                 desc="d=256, n=4096, k=64 -> rank 128, Gaussian leaves, sigma_j=10^(-10j/64), eps=1e-6 relative"),
}
METRIC = "HT truncations/s + roofline fraction, mixed vs plain FP64 GPU at stated rel err"
FP64_PEAK = 152 * 2 * 2 * 2.070e9   # SMs x FP64 FMA/clk/SM x 2 flop x max clock (recipe: 1.25 TFLOP/s)
FP32_PEAK = 152 * 128 * 2 * 2.070e9  # SMs x FP32 lanes x 2 flop x max clock


def model_flops(d, n, K, r):
    """Algorithmic work of one truncation (SURVEY work model): 12 K^4 per
    non-root inner node + n K (K + 2r) per leaf; eigen counted separately
    (9 K^3 per non-root node)."""
    inner = (d - 2) * 12.0 * K ** 4
    leaves = d * n * K * (K + 2 * r)
    eig = (2 * d - 2) * 9.0 * K ** 3
    return inner + leaves, eig


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
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


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


def oracle_truncations(wl, seed, count, threads=0):
    """Run the CPU oracle on `count` add+truncate steps; returns (seconds, cores)."""
    from oracle import oracle as O
    cores = O.set_threads(threads)
    (n, ka, xa), (_, kc, xc) = wl["make"](seed)
    d = wl["d"]
    t0 = time.perf_counter()
    for _ in range(count):
        k, x = O.add(d, n, ka, xa, kc, xc)
        O.truncate(d, n, k, x, **wl["opts"])
    return time.perf_counter() - t0, cores


def accuracy_vs_fp64(htgb, tree, n, ka, xa, kc, xc, wl, stream):
    """Errors of the FP32-storage path relative to the FP64 GPU path on the same
    (FP32-representable) inputs, all computed by the library on the GPU:
    sigma^2 normwise per node, ||X||, and ||T32(X) - T64(X)|| / ||X|| and the
    truncation errors ||X - T(X)|| / ||X|| of both paths (norms of HT
    differences via orthogonalization, never via inner products)."""
    xa32 = np.asarray(xa, np.float32).astype(np.float64)
    xc32 = np.asarray(xc, np.float32).astype(np.float64)
    out = {}
    res = {}
    for name, dt in (("fp32", htgb.HT_F32), ("fp64", htgb.HT_F64)):
        A = htgb.HTTensor.from_blob(tree, n, ka, xa32, dt, stream)
        C = htgb.HTTensor.from_blob(tree, n, kc, xc32, dt, stream)
        X = A.add(C)
        rep = X.truncate(prec=htgb.HT_PREC_FP32 if dt == htgb.HT_F32 else htgb.HT_PREC_FP64, **wl["opts"])
        res[name] = (rep, X.ranks(), X.download().astype(np.float64))
    X64 = htgb.HTTensor.from_blob(tree, n, ka, xa32, htgb.HT_F64, stream).add(
        htgb.HTTensor.from_blob(tree, n, kc, xc32, htgb.HT_F64, stream))
    nrm = res["fp64"][0]["norm"]

    def diff_norm(ya, ka_, yb, kb_):
        P = htgb.HTTensor.from_blob(tree, n, ka_, ya, htgb.HT_F64, stream) if not isinstance(ya, htgb.HTTensor) else ya
        Q = htgb.HTTensor.from_blob(tree, n, kb_, yb, htgb.HT_F64, stream)
        Q.scale(-1.0)
        return P.add(Q).norm()

    (r32, k32, x32), (r64, k64, x64) = res["fp32"], res["fp64"]
    worst = 0.0
    o32 = o64 = 0
    for t in range(1, len(r64["korth"])):
        a = r32["sigma"][o32:o32 + r32["korth"][t]]
        b = r64["sigma"][o64:o64 + r64["korth"][t]]
        o32 += r32["korth"][t]
        o64 += r64["korth"][t]
        if len(b) and b[0] > 0:
            sel = b >= 1e-5 * b[0]
            worst = max(worst, float(np.max(np.abs(a[sel] ** 2 - b[sel] ** 2)) / b[0] ** 2))
    out["sigma2_normwise"] = worst
    out["norm"] = abs(r32["norm"] - nrm) / nrm
    out["truncated_tensor"] = diff_norm(x32, k32, x64, k64) / nrm
    out["trunc_err_fp32"] = diff_norm(X64, None, x32, k32) / nrm
    out["trunc_err_fp64"] = diff_norm(X64, None, x64, k64) / nrm
    out["ranks_fp32_ge_fp64"] = bool(np.all(np.asarray(k32) >= np.asarray(k64)))
    return out


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_truncations(wl, 11, 1)
    secs, cores = oracle_truncations(wl, 11, args.steps)
    value = args.steps / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "truncations/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "shape": wl["desc"]},
        "cpu_baseline": {"value": value, "unit": "truncations/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} add+truncate steps of the full workload"},
        "e2e": {"value": value, "unit": "truncations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="single", choices=sorted(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison arms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.config]
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    from paper_1708_03340_gb300 import htgb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    d, k = wl["d"], wl["k"]
    seed = 11 + 1000 * rank  # each rank truncates its own tensors
    (n, ka, xa), (_, kc, xc) = wl["make"](seed)
    tree = htgb.HTTree(d)
    ksum = np.asarray(ka) + np.asarray(kc)
    ksum[0] = 1
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def setup(dtype):
        A = htgb.HTTensor.from_blob(tree, n, ka, xa, dtype, stream)
        C = htgb.HTTensor.from_blob(tree, n, kc, xc, dtype, stream)
        X = htgb.HTTensor.create(tree, n, ksum, dtype, stream)
        return A, C, X

    def timed(dtype, prec, sched, steps, warmup, prof_mask=0):
        A, C, X = setup(dtype)
        opts = htgb.make_opts(prec=prec, schedule=sched, **wl["opts"])
        for _ in range(warmup):
            htgb.ht_add_into(A.handle, C.handle, X.handle)
            htgb.ht_truncate(X.handle, opts)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        htgb.ht_profile_set(prof_mask)
        for kind in range(len(htgb.KERNEL_KINDS)):
            htgb.ht_profile_read(kind, reset=True)
        l0 = htgb.ht_launch_count()
        evs = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            htgb.ht_add_into(A.handle, C.handle, X.handle)
            htgb.ht_truncate(X.handle, opts)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        launches = htgb.ht_launch_count() - l0
        htgb.ht_profile_set(0)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        prof = {}
        for kind, name in enumerate(htgb.KERNEL_KINDS):
            cnt, tms, fl = htgb.ht_profile_read(kind, reset=True)
            if cnt:
                prof[name] = {"launches": cnt, "ms": tms, "flops": fl}
        if ws > 1:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        ranks = X.ranks()
        return dict(ms=ms, launches=launches, prof=prof, X=X, ranks=ranks, A=A, C=C)

    # ---- the headline arm: FP32 storage + FP32 SIMT contractions + FP64 eigen, per-level launches
    clk_path = os.path.join(tempfile.gettempdir(), f"htgb_clocks_{os.getpid()}.csv")
    proc, fh = start_clock_sampler(clk_path)
    all_mask = (1 << len(htgb.KERNEL_KINDS)) - 1
    main = timed(htgb.HT_F32, htgb.HT_PREC_FP32, htgb.HT_SCHED_LEVEL, args.steps, args.warmup, all_mask)
    clocks = read_clocks(proc, fh, clk_path, local)
    K = 2 * k
    r_cap = wl["opts"].get("rank_cap", 0) or k
    work, eig_work = model_flops(d, wl["n"], K, r_cap)
    value = ws * args.steps / (main["ms"] / 1e3)
    ms_per_step = main["ms"] / args.steps

    # dominant kernel family by device time, with its roofline: algorithmic
    # flops per launch (counted by the library at plan time) / CUDA-event time
    dom = max(main["prof"].items(), key=lambda kv: kv[1]["ms"]) if main["prof"] else (None, None)
    roofline = None
    if dom[0] is not None:
        name, rec = dom
        per_launch_ms = rec["ms"] / rec["launches"]
        per_launch_flops = rec["flops"] / rec["launches"]
        ach = per_launch_flops / (per_launch_ms / 1e3)
        kernel = {"qr": "qr_reg_kernel / qr_block_kernel (FP32 TSQR blocks)", "gemm": "gemm_kernel (FP32 SIMT)",
                  "eig": "eig_ql_kernel<float> + refine_kernel (FP64)"}.get(name, name)
        peak = FP64_PEAK if name == "eig" else FP32_PEAK
        roofline = {"kernel": kernel, "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "peak_source": ("FP64" if name == "eig" else "FP32") + " unit count x max SM clock (recipe)",
                    "launches_per_step": rec["launches"] / args.steps, "ms_per_launch": per_launch_ms,
                    "flops_per_launch": per_launch_flops}

    line = {
        "metric": METRIC, "value": value, "unit": "truncations/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded SplitMix64/Box-Muller HT tensors)",
        "config": {"workload": args.config, "shape": wl["desc"], "l2": "flushed between steps (256 MB write)",
                   "path": "FP32 storage and contractions, FP64 eigensolves, one batched launch per level"},
        "gflops": work / (ms_per_step / 1e3) / 1e9,
        "kernel_ms_per_step": {kname: v["ms"] / args.steps for kname, v in main["prof"].items()},
        "kernel_tflops": {kname: v["flops"] / max(v["ms"], 1e-9) / 1e9 for kname, v in main["prof"].items()
                          if v["flops"] > 0},
        "ranks_first_nodes": [int(v) for v in main["ranks"][:8]],
        "gpu_launches": main["launches"],
        "roofline": roofline,
        "clocks": clocks,
    }

    # ---- plain FP64 GPU arms (per level, and one launch per node)
    if not args.no_plain:
        ps = max(3, args.steps // 4)
        plain = timed(htgb.HT_F64, htgb.HT_PREC_FP64, htgb.HT_SCHED_LEVEL, ps, 3, all_mask)
        line["plain_fp64_level"] = {"value": ws * ps / (plain["ms"] / 1e3), "unit": "truncations/s",
                                    "ms_per_step": plain["ms"] / ps, "launches_per_step": plain["launches"] / ps,
                                    "kernel_ms_per_step": {kn: v["ms"] / ps for kn, v in plain["prof"].items()}}
        node = timed(htgb.HT_F64, htgb.HT_PREC_FP64, htgb.HT_SCHED_NODE, 3, 3)
        line["plain_fp64_per_node"] = {"value": ws * 3 / (node["ms"] / 1e3), "unit": "truncations/s",
                                       "ms_per_step": node["ms"] / 3, "launches_per_step": node["launches"] / 3}
        line["speedup_vs_plain_per_node"] = value / line["plain_fp64_per_node"]["value"]
        line["speedup_vs_plain_level"] = value / line["plain_fp64_level"]["value"]
        # stated relative error of the mixed path against the plain FP64 GPU path
        # (the FP64 path matches the CPU FP64 oracle to 1e-12 in the parity tests)
        line["rel_err_vs_fp64"] = accuracy_vs_fp64(htgb, tree, n, ka, xa, kc, xc, wl, stream)

    # ---- end to end through the public API with host buffers
    A, C, X = main["A"], main["C"], main["X"]
    blob32 = lambda b: np.ascontiguousarray(b, dtype=np.float32)
    ha = torch.from_numpy(blob32(xa)).pin_memory()
    hc = torch.from_numpy(blob32(xc)).pin_memory()
    X.truncate(report=False, prec=htgb.HT_PREC_FP32, **wl["opts"])
    out_sz = htgb.ht_tensor_blob_size(X.handle)
    hout = torch.empty(4 * max(out_sz, 1), dtype=torch.float32).pin_memory()
    opts = htgb.make_opts(prec=htgb.HT_PREC_FP32, **wl["opts"])
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        htgb.ht_tensor_upload(A.handle, ha.numpy())
        htgb.ht_tensor_upload(C.handle, hc.numpy())
        htgb.ht_add_into(A.handle, C.handle, X.handle)
        htgb.ht_truncate(X.handle, opts)
        sz = htgb.ht_tensor_blob_size(X.handle)
        htgb.ht_tensor_download(X.handle, hout.numpy()[:sz])
        d2h = sz * 4
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = e2e_steps / e2e_s
    if ws > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_val = ws * e2e_steps / float(t.item())
    line["e2e"] = {"value": e2e_val, "unit": "truncations/s", "h2d_bytes_per_step": int(ha.numel() * 4 + hc.numel() * 4),
                   "d2h_bytes_per_step": int(d2h)}

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    if ws == 1 and not args.no_cpu:
        secs, cores = oracle_truncations(wl, 11, 2)
        line["cpu_baseline"] = {"value": 2 / secs, "unit": "truncations/s", "cores": cores, "kind": "oracle",
                                "sample": "2 add+truncate steps of the same workload, FP64, OpenMP over tree nodes"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
