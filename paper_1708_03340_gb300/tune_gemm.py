"""Autotuner of the SIMT contraction kernel's tile-shape table (csrc/gemm_tune.h).

The library picks, per contraction launch, one of three tile shapes (64 x 64,
128 x 64, 128 x 128) from the share of the launch's flops held by "tall"
(M >= tall_m) and "square" (M, N >= tall_m) items.  This script times the
add + truncate step of representative workloads (CUDA-graph replays, FP32
path) for every candidate (tall_m, tall_share, square_share), each in a fresh
process that sets it through ht_set_gemm_tuning, and writes the fastest candidate (geometric mean
of the step times over the workloads) into csrc/gemm_tune.h together with a
results table, gemm_tune_results.md.  The accuracy threshold kTuneCompLen is
not tuned.

    python -m paper_1708_03340_gb300.tune_gemm            # on a GPU
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(HERE, "csrc", "gemm_tune.h")
RESULTS = os.path.join(HERE, "gemm_tune_results.md")

# workload name -> (number of tensors per step, description)
WORKLOADS = {
    "single": "d=64, n=1000, k=32 -> K=64, 1 pair",
    "deep": "d=256, n=4096, k=64 -> K=128, 1 pair",
    "wide": "d=16, n=2048, k=128 -> K=256, 2 pairs",
    "batched": "16 uneven tensors, d 4..32, n 16..512, K=4k with k 4..48",
}
CANDIDATES = list(itertools.product([64, 128, 256], [0.5], [0.3, 0.6, 2.0]))


def _pairs(name):
    """The workload's summand pairs (cached in the temp directory: every
    candidate runs in its own process)."""
    import pickle
    import tempfile
    path = os.path.join(tempfile.gettempdir(), f"htgb_tune_{name}.pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    out = _make_pairs(name)
    with open(path + ".tmp", "wb") as f:
        pickle.dump(out, f)
    os.replace(path + ".tmp", path)
    return out


def _make_pairs(name):
    sys.path.insert(0, ROOT)
    from paper_1708_03340_gb300 import inputs as I
    if name == "single":
        return [(64, *I.single_pair(11))], dict(I.SINGLE_OPTS)
    if name == "deep":
        return [(256, *I.deep_pair(21))], dict(I.DEEP_OPTS)
    if name == "wide":
        return [(16, *I.wide_pair(31 + 2 * i)) for i in range(2)], dict(I.WIDE_OPTS)
    specs = I.batched_specs(count=4096, seed=41)[:16]
    out = []
    for (d, n, k, s) in specs:
        out.append((d, ("sum4", (d, n, k, s)), None))
    return out, dict(mode="rank", tensor_caps=[sp[2] for sp in specs])


def worker(name, steps, warmup):
    """Time `steps` graph replays of the workload; prints ms per step as JSON."""
    sys.path.insert(0, ROOT)
    import torch
    from paper_1708_03340_gb300 import htgb
    from paper_1708_03340_gb300 import inputs as I
    stream = torch.cuda.current_stream()
    pairs, opts = _pairs(name)
    A, C, X, keep = [], [], [], []
    for (d, a, c) in pairs:
        tr = htgb.HTTree(d)
        keep.append(tr)
        if isinstance(a, tuple) and isinstance(a[0], str) and a[0] == "sum4":
            T = [htgb.HTTensor.from_blob(tr, nv, kv, xv, htgb.HT_F32, stream) for (nv, kv, xv) in I.batched_terms(a[1])]
            ta, tc = T[0].add(T[1]), T[2].add(T[3])
        else:
            ta = htgb.HTTensor.from_blob(tr, a[0], a[1], a[2], htgb.HT_F32, stream)
            tc = htgb.HTTensor.from_blob(tr, c[0], c[1], c[2], htgb.HT_F32, stream)
        k = ta.ranks() + tc.ranks()
        k[0] = 1
        A.append(ta), C.append(tc), X.append(htgb.HTTensor.create(tr, ta.n, k, htgb.HT_F32, stream))
    o = htgb.make_opts(prec=htgb.HT_PREC_FP32, **opts)
    g = htgb.ht_graph_add_truncate([a.handle for a in A], [c.handle for c in C], [x.handle for x in X], o)
    for _ in range(warmup):
        htgb.ht_graph_launch(g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        htgb.ht_graph_launch(g)
    e1.record(stream)
    torch.cuda.synchronize()
    htgb.ht_graph_free(g)
    print(json.dumps({"ms": e0.elapsed_time(e1) / steps}))


def run_candidate(name, cand, steps, warmup):
    out = subprocess.run([sys.executable, "-m", "paper_1708_03340_gb300.tune_gemm", "--worker", name,
                          "--steps", str(steps), "--warmup", str(warmup), "--cand", "%d,%g,%g" % cand],
                         cwd=ROOT, capture_output=True, text=True, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(f"worker {name} {cand} failed:\n{out.stderr[-2000:]}")
    return json.loads(out.stdout.strip().splitlines()[-1])["ms"]


def write_header(best, path=HEADER):
    tall_m, tall_share, square_share = best
    src = open(path).read()
    import re
    src = re.sub(r"constexpr int kTuneTallM = \d+;", f"constexpr int kTuneTallM = {tall_m};", src)
    src = re.sub(r"constexpr double kTuneTallShare = [0-9.e+-]+;", f"constexpr double kTuneTallShare = {tall_share};", src)
    src = re.sub(r"constexpr double kTuneSquareShare = [0-9.e+-]+;",
                 f"constexpr double kTuneSquareShare = {square_share};", src)
    open(path, "w").write(src)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--worker", default=None)
    ap.add_argument("--cand", default=None, help="tall_m,tall_share,square_share (worker processes)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--no-write", action="store_true")
    ap.add_argument("--out", default=None, help="write gemm_tune.h and the results table here instead of in place")
    args = ap.parse_args()
    if args.worker:
        if args.cand:
            from paper_1708_03340_gb300 import htgb
            m, a, b = args.cand.split(",")
            htgb.ht_set_gemm_tuning(int(m), float(a), float(b))
        return worker(args.worker, args.steps, args.warmup)
    table = {}
    for cand in CANDIDATES:
        table[cand] = {name: run_candidate(name, cand, args.steps, args.warmup) for name in WORKLOADS}
        print(cand, {k: round(v, 3) for k, v in table[cand].items()}, flush=True)
    ref = table[CANDIDATES[0]]
    score = {c: math.exp(sum(math.log(t[n] / ref[n]) for n in WORKLOADS) / len(WORKLOADS)) for c, t in table.items()}
    best = min(score, key=score.get)
    lines = ["# SIMT contraction tile-shape tuning (GB300)", "",
             f"Written by `python -m paper_1708_03340_gb300.tune_gemm` on {time.strftime('%Y-%m-%d')}.",
             "Step time (ms) of add + truncate, CUDA-graph replays, FP32 path; score = geometric mean of the",
             "step times relative to the first candidate (lower is better).", "",
             "| tall_m | tall_share | square_share | " + " | ".join(WORKLOADS) + " | score |",
             "|---" * (len(WORKLOADS) + 4) + "|"]
    for c in CANDIDATES:
        mark = " **(chosen)**" if c == best else ""
        lines.append(f"| {c[0]} | {c[1]} | {c[2]} | " + " | ".join(f"{table[c][n]:.3f}" for n in WORKLOADS) +
                     f" | {score[c]:.3f}{mark} |")
    lines += ["", "Workloads: " + "; ".join(f"{k}: {v}" for k, v in WORKLOADS.items()) + "."]
    print("\n".join(lines))
    if not args.no_write:
        header, results = HEADER, RESULTS
        if args.out:
            os.makedirs(args.out, exist_ok=True)
            header = os.path.join(args.out, "gemm_tune.h")
            results = os.path.join(args.out, "gemm_tune_results.md")
            with open(header, "w") as f:
                f.write(open(HEADER).read())
        write_header(best, header)
        open(results, "w").write("\n".join(lines) + "\n")


if __name__ == "__main__":
    sys.exit(main())
