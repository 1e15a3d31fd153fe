"""Benchmark: LINE edge-sample updates/s on R-MAT scale 20 (d=128, K=5, FP32).

Workload: R-MAT scale 20 (1,048,576 nodes, edge factor 16, (a,b,c,d) =
(.57,.19,.19,.05), symmetrised, duplicates merged into integer weights),
first- and second-order LINE, d=128, K=5 negatives from deg^0.75, FP32
tables, deterministic minibatch B=4096, lr 0.025 with linear decay over
20 x |E| samples per order.  One step = |E| = 16 * 2^20 samples of each
order (one "epoch" of each), so 20 steps are the full run.  The two orders'
tables are independent and are trained concurrently (line_train_orders, two
streams; the same tables as one order after the other).

Other workloads (``--workload``; not the default line):

* ``rmat20walk`` - the default workload with the positive pairs drawn by the
  walk sampler instead of by arc weight: walks of length 100 from roots drawn
  by arc weight, weighted steps, pairs within a window of 2 (Algorithms 2-3,
  the local walk); the negatives, update and schedule are unchanged.

* ``reuse20`` - the walk-reuse ablation (a single-device form of the paper's
  Reuse-Spill variant): R-MAT 20 with 10% of the edges held out, orders 1
  and 2 trained concurrently on walk pairs (L=100, W=2) for ``--epochs``
  epochs, each walk's pairs serving r = 1, 4 and 16 passes, in the
  minibatch and the Hogwild schedule: updates/s, second-order loss and
  link-prediction AUC of each.
* ``mlp20`` - the warm-start MLP's kernels alone on R-MAT 20 (BF16 tables,
  d=128, hidden 256, BF16 activations): the inputs of every node, the inputs
  of 10% held-out nodes and their predictions, device time of each call.
* ``dchung22`` - weighted directed Chung-Lu graph, 4,194,304 nodes, 2^26 arc
  draws (out-weights power law 2.2, lognormal(0,1) weights); order 2, d=128,
  K=5: the FP32 path at B=4096 against BF16 tables with stochastic rounding
  in the launch configuration the autotuner picks (batch 4K-64K, schedule,
  graph replay), throughput and loss at equal samples.
* ``rmat24`` - R-MAT scale 24 (16,777,216 nodes, 2^28 draws), 10% of the
  edges held out; orders 1 and 2 trained concurrently for ``--epochs``
  epochs with BF16 tables (autotuned launch configuration) and with FP32
  tables (B=4096): updates/s, HBM roofline and link-prediction AUC of each.
* ``warm22`` - R-MAT scale 22 with 10% of the edges (AUC positives) and 10% of
  the nodes held out.  Order-2 LINE trains on the kept nodes (phase 0, FP32
  or BF16); then the held-out nodes arrive and each arm refines on the graph
  without the held-out edges: plain FP32 and plain BF16 from random rows for
  the new nodes, and BF16 with the new rows predicted by the MLP (fit on the
  kept nodes' rows before the arrival).  At every checkpoint: link-prediction
  AUC (inner products of U rows; held-out edges against as many non-edges)
  and device time since the arrival; reports when the BF16 + warm-start arm
  reaches the FP32 arm's final AUC within 0.005.

Output: one JSON line (rank 0).  `value` is device-timed throughput with the
graph and tables resident in HBM; `e2e` is the same metric through the C ABI
from host buffers (graph upload + alias build + training + read-back of the
order-2 U table, every step).  `--impl reference` times the FP64 oracle on
the host cores instead (a bounded prefix of the same workload).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the headline metric as the workload states it; `value` is its first part
# (updates/s), `roofline.frac` the second, and the warm22 workload the third
METRIC = "edge-sample updates/s (d=128,K=5), HBM roofline %, BF16+warm vs FP32 at equal AUC"
UNIT = "updates/s"
DIM, K, B = 128, 5, 4096
ROW_BYTES_F32 = DIM * 4
# algorithmic bytes per edge-sample update: 7 rows read + 7 written, plus
# sampling metadata (edge alias 8 B + arc endpoints 8 B + K neg alias 5 x 8 B)
ALG_BYTES_PATH = 14 * ROW_BYTES_F32 + 8 + 8 + 8 * K
# the update kernels alone move the 14 rows
ALG_BYTES_UPDATE = 14 * ROW_BYTES_F32
META_BYTES = 8 + 8 + 8 * K


def row_bytes(dtype_name: str) -> int:
    return DIM * (2 if dtype_name == "bf16" else 4)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="auto", choices=["auto", "batched", "persistent", "hogwild"],
                   help="hogwild: per-pair immediate updates by lock-free concurrent workers (not deterministic)")
    p.add_argument("--orders", default="concurrent", choices=["concurrent", "sequential"],
                   help="train the two orders' tables concurrently (line_train_orders) or one after the other")
    p.add_argument("--scale", type=int, default=20)
    p.add_argument("--dtype", default="fp32", choices=["fp32", "bf16"],
                   help="table storage of the default and rmat20walk workloads (bf16: stochastic rounding)")
    p.add_argument("--samples-per-step", type=int, default=0, help="0: |E| = 16 * 2^scale")
    p.add_argument("--e2e-steps", type=int, default=6)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-samples", type=int, default=1 << 20)
    p.add_argument("--workload", default="rmat20",
                   choices=["rmat20", "rmat20walk", "reuse20", "mlp20", "dchung22", "warm22", "rmat24"])
    p.add_argument("--walk-length", type=int, default=100, help="rmat20walk: steps per walk")
    p.add_argument("--window", type=int, default=2, help="rmat20walk: pair window")
    p.add_argument("--epochs", type=int, default=10, help="rmat24, reuse20: samples per order = epochs x |E|")
    p.add_argument("--checkpoints", type=int, default=10, help="warm22: refinement epochs (checkpoints)")
    p.add_argument("--fit-nodes", type=int, default=1 << 16, help="warm start: kept nodes the MLP is fit on")
    p.add_argument("--fit-steps", type=int, default=16, help="warm start: Adam steps of the fit")
    p.add_argument("--no-warm", action="store_true", help="default workload: skip the warm-start leg")
    p.add_argument("--no-c3", action="store_true", help="default workload: skip the directed Chung-Lu leg")
    p.add_argument("--no-variants", action="store_true",
                   help="default workload: skip the BF16 and one-order variants")
    return p.parse_args()


def replica_seed(rank: int) -> int:
    """Replicas (one per rank, no collectives on the data path) train with
    different seeds."""
    return 1000 + rank


def max_over_ranks(value: float, world: int) -> float:
    """The job's time is the slowest rank's (max-reduce over the process group)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_traffic():
    """DRAM bytes per batch of the update kernels from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    import hashlib
    import re
    try:
        with open(os.path.join(ROOT, "profiles", "k_gather_k_apply_rmat20_d128_K5_B4096.md")) as f:
            text = f.read()
        with open(os.path.join(ROOT, "paper_2604_09419_gb300", "csrc", "train.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        m = re.search(r"sha256 prefix ([0-9a-f]{16})", text)
        t = re.search(r"traffic_bytes_per_batch: (\d+)", text)
        if m and t and m.group(1) == sha:
            return int(t.group(1))
    except OSError:
        pass
    return None


def metric_of(args):
    return "walk-pair updates/s (d=128,K=5)" if walk_of(args)[0] else METRIC


def walk_of(args):
    """(walk_length, window) of the workload; (0, 0) for arcs drawn by weight."""
    return (args.walk_length, args.window) if args.workload == "rmat20walk" else (0, 0)


def cpu_baseline(g, n_samples: int, walk=(0, 0), pairwise=False):
    """The FP64 oracle, single-threaded, on a prefix of the same workload
    (order 2): the minibatch oracle, or the per-pair one for the Hogwild mode."""
    import numpy as np

    import oracle as O
    T = O.Tables(g)
    U = O.init_uniform(g.n_nodes, DIM, 1)
    C = np.zeros_like(U)
    wk = (O.walk_cumw(g), walk[0], walk[1]) if walk[0] > 0 else None
    fn = O.train_pairwise if pairwise else O.train
    t0 = time.perf_counter()
    fn(T, U, C, order=2, K=K, n_samples=n_samples, seed=11, batch=B, lr_total=20 * 16 * g.n_nodes, walk=wk)
    dt = time.perf_counter() - t0
    kind = "per-pair" if pairwise else "minibatch"
    return {"value": n_samples / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"order-2 FP64 {kind} oracle on the first {n_samples} samples of the workload "
                      f"(single thread, host has {os.cpu_count()} cores); {dt:.1f} s"}


def cpu_hogwild_context(g, n_samples: int):
    """Context, not a reference: multi-threaded FP32 CPU Hogwild LINE (order 2)
    on all host cores, on a prefix of the workload - the kind of CPU LINE the
    paper's multi-threaded baselines are."""
    import numpy as np

    import oracle as O
    T = O.Tables(g)
    U = O.init_uniform(g.n_nodes, DIM, 1).astype(np.float32)
    C = np.zeros_like(U)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    O.train_hogwild_cpu(T, U, C, order=2, K=K, n_samples=n_samples, seed=11, batch=B, lr_total=20 * 16 * g.n_nodes,
                        threads=threads)
    dt = time.perf_counter() - t0
    return {"value": n_samples / dt, "unit": UNIT, "cores": threads, "kind": "multi-threaded FP32 CPU Hogwild (context)",
            "sample": f"order-2 per-pair updates, {n_samples} samples, {threads} threads; {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    from paper_2604_09419_gb300 import inputs as I
    g = I.rmat(args.scale, seed=0)
    n = min(args.cpu_samples, 1 << 19)
    times = []
    for _ in range(args.warmup if args.warmup < 1 else 1):
        cpu_baseline(g, 4096, walk_of(args))
    for _ in range(args.steps):
        r = cpu_baseline(g, n, walk_of(args))
        times.append(n / r["value"])
    value = n / statistics.median(times)
    line = {"impl": "reference", "metric": metric_of(args), "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args, g),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n} samples of order 2 per step (FP64 oracle, single thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args, g):
    wl, ww = walk_of(args)
    sampler = f"_walk{wl}w{ww}" if wl else ""
    tables_gib = 3 * g.n_nodes * row_bytes(args.dtype) / 2 ** 30
    c = {"workload": f"rmat{args.scale}_line_order1+2_d{DIM}_K{K}_B{B}_{args.dtype}{sampler}",
         "graph": f"R-MAT scale {args.scale}, edge factor 16, (.57,.19,.19,.05), symmetrised",
         "n_nodes": g.n_nodes, "n_arcs": g.n_arcs, "dim": DIM, "K": K, "batch": B,
         "samples_per_step": 2 * samples_per_step(args),
         "lr": "0.025 linear decay over 20*|E| samples per order",
         "l2": f"inputs larger than L2 ({args.dtype.upper()} U1, U2, C2 tables: {tables_gib:.2f} GiB; "
               f"alias tables 258 MB)"}
    if wl:
        c["positive_pairs"] = (f"walk sampler: walks of {wl} steps from arcs drawn by weight, weighted steps, "
                               f"pairs within a window of {ww}")
    return c


def samples_per_step(args):
    return args.samples_per_step or 16 * (1 << args.scale)


def c3_compare(steps: int, warmup: int, samples_per_step: int = 0) -> dict:
    """Directed Chung-Lu (4M nodes, 2^26 arc draws), order 2: the FP32 path
    at B = 4096 against BF16 tables with an autotuned batch (4K-64K), gather
    warps, chunk size and schedule; `steps` timed steps of |E| samples (or
    `samples_per_step`) after `warmup` untimed ones, each arm."""
    import torch

    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    g = I.chung_lu_directed()
    stream = torch.cuda.current_stream()
    ctx = L.Context(local, stream.cuda_stream)
    ctx.build_alias(g.n_nodes, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                    torch.from_numpy(g.w).cuda())
    E = g.n_arcs
    total = 10 * E
    S = samples_per_step or E
    peak, peak_kind = peaks()
    res = {}
    for name, dtype in (("fp32", L.DTYPE_F32), ("bf16", L.DTYPE_BF16)):
        ctx.init_embeddings(2, DIM, dtype, seed=2)
        o = L.train_opts_default()
        o.batch = B
        rate_tuned = None
        if dtype == L.DTYPE_BF16:
            o, rate_tuned = ctx.autotune(2, DIM, K, batches=[4096, 8192, 16384, 32768, 65536], try_persistent=True,
                                         total=total, opts=o)
        o.timing = 1
        for i in range(warmup):
            o.sample_offset = i * S
            ctx.train_steps(2, DIM, K, S, 7, total=total, opts=o)
        ctx.reset_stats()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for i in range(steps):
                o.sample_offset = (warmup + i) * S
                ctx.train_steps(2, DIM, K, S, 7, total=total, opts=o)
            ev1.record(stream)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        st = ctx.stats()
        row = DIM * (4 if dtype == L.DTYPE_F32 else 2)
        rate = S * steps / (ms / 1e3)
        upd = st.update_samples * 14 * row / (st.update_ms / 1e3) / 1e9 if st.update_ms > 0 else None
        res[name] = {"value": rate, "ms_per_step": ms / steps, "batch": int(o.batch),
                     "mode": "batched" if o.mode == L.MODE_BATCHED else "persistent",
                     "warps_per_block": int(o.warps_per_block), "chunk_batches": int(o.chunk_batches),
                     "autotuned_rate": rate_tuned,
                     "roofline": {"bound": "hbm", "achieved": upd, "peak": peak, "unit": "GB/s",
                                  "frac": upd / peak if upd else None, "alg_bytes_per_sample": 14 * row,
                                  "peak_kind": peak_kind,
                                  "path_frac": rate * (14 * row + 8 + 8 + 8 * K) / 1e9 / peak},
                     "loss_after": ctx.eval_loss(2, K, 99, 1 << 20),
                     "samples_trained": S * (warmup + steps), "clocks": clk.summary()}
    out = {"workload": "dchung22_line_order2_d128_K5_bf16_vs_fp32",
           "graph": "directed Chung-Lu, 4,194,304 nodes, 2^26 arc draws, out-weight power law 2.2, "
                    "lognormal(0,1) arc weights", "n_nodes": g.n_nodes, "n_arcs": E,
           "samples_per_step": S, "steps": steps, "warmup": warmup, "lr": "0.025 linear decay over 10*|E|",
           "fp32": res["fp32"], "bf16": res["bf16"],
           "bf16_over_fp32": res["bf16"]["value"] / res["fp32"]["value"],
           "loss_rel_diff": (res["bf16"]["loss_after"] - res["fp32"]["loss_after"]) / res["fp32"]["loss_after"]}
    ctx.close()
    return out


def run_dchung22(args):
    """Directed Chung-Lu, order 2: FP32 at B=4096 vs autotuned BF16."""
    r = c3_compare(args.steps, args.warmup, args.samples_per_step)
    line = {"metric": METRIC, "value": r["bf16"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "graph", "n_nodes", "n_arcs", "samples_per_step", "lr")},
            "fp32": r["fp32"], "bf16": r["bf16"], "bf16_over_fp32": r["bf16_over_fp32"],
            "loss_rel_diff": r["loss_rel_diff"]}
    print(json.dumps(line), flush=True)


def warm_compare(scale: int, *, phase0_epochs: int = 10, marks=(0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1, 1.5, 2),
                 fit_nodes: int = 1 << 16, fit_steps: int = 16, fit_batch: int = 16384, curves: bool = True):
    """Warm start of arriving nodes (the C4 comparison) on R-MAT `scale`.

    10% of the edges are held out (link-prediction positives, against as many
    non-edges) and 10% of the nodes arrive after phase 0.  Phase 0 trains
    order-2 LINE on the kept nodes' induced graph for `phase0_epochs` epochs;
    then the new nodes and their edges arrive and each arm refines on the
    graph without the held-out edges:
      fp32       FP32 tables, random rows for the new nodes (the plain path);
      bf16       BF16 tables, random rows;
      bf16_warm  BF16 tables, the new rows predicted by the MLP.  The MLP is
                 fit on a sample of `fit_nodes` kept nodes (their inputs only)
                 for `fit_steps` Adam steps of `fit_batch`, and that fit is
                 charged to the arm: its times count the fit, the new rows'
                 inputs and the prediction.
    Times are wall times of synchronised calls (evaluation and the upload of
    the changed graph, the same for every arm, excluded), counted from the
    arrival and from the start of phase 0, after an untimed warm-up that runs
    each arm's kernels once.  The target is the FP32 arm's
    final AUC - 0.005; samples-to-target-loss is where an arm's loss first
    reaches the loss that random rows of the same precision (bf16) reach at
    their final checkpoint."""
    import numpy as np
    import torch

    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    g = I.rmat(scale, seed=0)
    tr, hs, hd = I.split_edges(g, 0.1, seed=4)
    ans, ad = I.non_edges(g, len(hs), seed=7)
    held, kept = I.hold_out_nodes(tr, 0.1, seed=5)
    inc = held[hs] | held[hd]
    ps, pd = hs[inc], hd[inc]
    cs, cd = I.non_edges(g, 8 * len(ps) + 1000, seed=6)
    m = held[cs] | held[cd]
    ns, nd = cs[m][:len(ps)], cd[m][:len(ps)]
    t_gen = time.perf_counter() - t_gen
    ctx = L.Context(local, stream.cuda_stream)

    def upload(h):
        ctx.build_alias(h.n_nodes, torch.from_numpy(h.src).cuda(), torch.from_numpy(h.dst).cuda(),
                        torch.from_numpy(h.w).cuda())

    def timed(fn):
        torch.cuda.synchronize()
        gc.disable()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        gc.enable()
        return dt

    E = tr.n_arcs
    n0 = phase0_epochs * kept.n_arcs
    total = int(marks[-1] * E) // B * B

    def evaluate():
        return {"auc_all": ctx.eval_auc(2, hs, hd, ans, ad)[0], "auc_new_nodes": ctx.eval_auc(2, ps, pd, ns, nd)[0],
                "loss": ctx.eval_loss(2, K, 99, 1 << 20)}

    def refine(t_start):
        """Refinement on the graph with the new nodes, checkpoint by checkpoint."""
        curve, t_acc, done = [], t_start, 0
        curve.append({"samples": 0, "time_s": t_acc, **evaluate()})
        o = L.train_opts_default()
        o.batch = B
        for x in marks:
            upto = int(x * E) // B * B
            o.sample_offset = done
            n = upto - done
            t_acc += timed(lambda: ctx.train_steps(2, DIM, K, n, 11, total=total, opts=o))
            done = upto
            curve.append({"samples": done, "time_s": t_acc, **evaluate()})
        return curve

    def phase0(dtype):
        upload(kept)
        ctx.init_embeddings(2, DIM, dtype, seed=2)
        t = timed(lambda: ctx.train_steps(2, DIM, K, n0, 3, batch=B, total=n0))
        U = torch.empty((g.n_nodes, DIM), dtype=torch.float32, device="cuda")
        C = torch.empty_like(U)
        ctx.get_embeddings(2, L.WHICH_U, U)
        ctx.get_embeddings(2, L.WHICH_C, C)
        return t, U, C

    def start_tables(dtype, U, C):
        ctx.init_embeddings(2, DIM, dtype, seed=0)
        ctx.set_embeddings(2, L.WHICH_U, U, L.DTYPE_F32)
        ctx.set_embeddings(2, L.WHICH_C, C, L.DTYPE_F32)

    # the new rows, and the sample of kept nodes the MLP is fit on
    rows = np.flatnonzero(held).astype(np.int32)
    deg_kept = np.bincount(kept.src, minlength=g.n_nodes)
    cand = np.flatnonzero(~held & (deg_kept > 0)).astype(np.int32)
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(cand, size=min(fit_nodes, cand.size), replace=False)).astype(np.int32)
    known = (~held).astype(np.uint8)
    known_h, sample_h, rows_h = (torch.from_numpy(known).pin_memory(), torch.from_numpy(sample).pin_memory(),
                                 torch.from_numpy(rows).pin_memory())

    # untimed warm-up: every kernel the arms run, once (module loading,
    # CUDA-graph capture, first allocations): two chunks of training per
    # table type on the kept graph, and the MLP path with BF16 tables
    upload(kept)
    for dt in (L.DTYPE_F32, L.DTYPE_BF16):
        ctx.init_embeddings(2, DIM, dt, seed=2)
        ctx.train_steps(2, DIM, K, 2 * (1 << 18), 3, batch=B, total=n0)
    ctx.mlp_create(2, hidden=256, act_dtype=L.DTYPE_BF16, seed=9)
    ctx.mlp_features_rows(known_h, sample_h)
    ctx.mlp_train(sample_h, steps=2, batch=fit_batch, lr=1e-3, seed=10)
    ctx.mlp_features_rows(known_h, rows_h)
    ctx.mlp_predict(rows_h)
    torch.cuda.synchronize()

    arms = {}
    t0_fp32, U32, C32 = phase0(L.DTYPE_F32)
    upload(tr)  # arrival: the held-out nodes and their edges join (same node count: tables kept)
    arms["fp32"] = {"name": "fp32, random rows for new nodes", "phase0_s": t0_fp32, "curve": refine(0.0)}
    del U32, C32
    t0_bf16, U16, C16 = phase0(L.DTYPE_BF16)
    # the fit, before the arrival (kept graph, phase-0 tables): inputs of a
    # sample of the kept nodes only, then Adam steps on it
    box = {}
    fit = {"mlp_create_s": timed(lambda: ctx.mlp_create(2, hidden=256, act_dtype=L.DTYPE_BF16, seed=9)),
           "features_sample_s": timed(lambda: ctx.mlp_features_rows(known_h, sample_h)),
           "mlp_train_s": timed(lambda: box.update(
               losses=ctx.mlp_train(sample_h, steps=fit_steps, batch=fit_batch, lr=1e-3, seed=10)))}
    upload(tr)  # arrival
    start_tables(L.DTYPE_BF16, U16, C16)
    arms["bf16"] = {"name": "bf16, random rows for new nodes", "phase0_s": t0_bf16, "curve": refine(0.0)}
    start_tables(L.DTYPE_BF16, U16, C16)
    arrival = {"features_new_rows_s": timed(lambda: ctx.mlp_features_rows(known_h, rows_h)),
               "predict_s": timed(lambda: ctx.mlp_predict(rows_h))}
    t_fit, t_arr = sum(fit.values()), sum(arrival.values())
    arms["bf16_warm"] = {"name": "bf16 + MLP warm start of the new rows", "phase0_s": t0_bf16,
                         "fit_before_arrival": fit, "at_arrival": arrival, "fit_nodes": int(sample.size),
                         "fit_steps": fit_steps, "fit_batch": fit_batch,
                         "mlp_first_loss": float(box["losses"][0]),
                         "mlp_last_loss": float(np.mean(box["losses"][-4:])),
                         "curve": refine(t_fit + t_arr)}
    ctx.close()

    fp32_final = arms["fp32"]["curve"][-1]["auc_all"]
    target = fp32_final - 0.005
    loss_ref = arms["bf16"]["curve"][-1]["loss"]
    summary = {}
    for k, a in arms.items():
        hit = next((c for c in a["curve"] if c["auc_all"] >= target), None)
        lhit = next((c for c in a["curve"] if c["loss"] <= loss_ref), None)
        summary[k] = {"from_arrival_s": hit["time_s"] if hit else None,
                      "from_phase0_start_s": a["phase0_s"] + hit["time_s"] if hit else None,
                      "phase0_s": a["phase0_s"], "auc_at_arrival": a["curve"][0]["auc_all"],
                      "auc_new_nodes_at_arrival": a["curve"][0]["auc_new_nodes"],
                      "final_auc": a["curve"][-1]["auc_all"],
                      "samples_to_target_loss": lhit["samples"] if lhit else None}
    w, f = summary["bf16_warm"], summary["fp32"]

    def won(key):
        return bool(w[key] is not None and (f[key] is None or w[key] < f[key]))

    out = {"graph": f"R-MAT scale {scale}", "n_nodes": g.n_nodes, "n_arcs_train": E, "new_nodes": int(len(rows)),
           "phase0_epochs": phase0_epochs, "target_auc": target, "fp32_final_auc": fp32_final,
           "target_loss": loss_ref, "fit_s": t_fit, "arrival_s": t_arr, "fit_parts_s": fit, "arrival_parts_s": arrival,
           "bf16_warm_wins_from_arrival_fit_included": won("from_arrival_s"),
           "bf16_warm_wins_from_phase0_start": won("from_phase0_start_s"),
           "arms": summary, "generation_s": t_gen,
           "time": "wall time of synchronised calls, after an untimed warm-up that runs every arm's kernels once "
                   "(module loading, CUDA-graph capture, first allocations); the warm arm's times include its fit "
                   "(MLP re-created: weights, optimiser state and inputs start over) and its arrival work; "
                   "evaluation and the upload of the changed graph excluded from every arm"}
    if curves:
        out["curves"] = {k: a["curve"] for k, a in arms.items()}
        out["details"] = {k: {kk: vv for kk, vv in a.items() if kk != "curve"} for k, a in arms.items()}
    return out


def run_warm22(args):
    """Warm start of arriving nodes on R-MAT 22: BF16 + MLP vs plain FP32."""
    marks = [x for x in (0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1, 1.5, 2, 3, 5, 10) if x <= args.checkpoints]
    res = warm_compare(22, marks=marks, fit_nodes=args.fit_nodes, fit_steps=args.fit_steps)
    w = res["arms"]["bf16_warm"]
    line = {"metric": "time until BF16 + warm start reaches the FP32 path's link-prediction AUC (within 0.005), "
                      "fit included",
            "value": w["from_arrival_s"], "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "warm22_rmat22_order2_d128_K5_B4096",
                       "graph": "R-MAT scale 22 (4,194,304 nodes), 10% of edges held out for AUC, 10% of nodes "
                                "held out and arriving after phase 0", "checkpoints_epochs": marks,
                       "fit": f"{args.fit_steps} Adam steps of 16384 on {args.fit_nodes} kept nodes"},
            **res}
    print(json.dumps(line), flush=True)


def run_rmat24(args):
    """R-MAT 24, orders 1+2, BF16 (autotuned) vs FP32: throughput and AUC."""
    import torch

    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L
    _, _, local = dist_env()
    # generating the graph peaks near 44 GB of host memory (about 4x R-MAT 22)
    try:
        with open("/proc/meminfo") as f:
            avail_gb = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable")) / 1e6
    except (OSError, StopIteration):
        avail_gb = 0.0
    if avail_gb < 64:
        print(json.dumps({"workload": "rmat24", "unavailable": f"{avail_gb:.0f} GB of host memory available, 64 needed"}))
        return
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    g = I.rmat(24, seed=0)
    tr, hs, hd = I.split_edges(g, 0.1, seed=4)
    ns, nd = I.non_edges(g, len(hs), seed=7)
    del g
    t_gen = time.perf_counter() - t_gen
    ctx = L.Context(local, stream.cuda_stream)
    ctx.build_alias(tr.n_nodes, torch.from_numpy(tr.src).cuda(), torch.from_numpy(tr.dst).cuda(),
                    torch.from_numpy(tr.w).cuda())
    E = tr.n_arcs
    n = args.epochs * E
    peak, peak_kind = peaks()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, dtype in (("bf16", L.DTYPE_BF16), ("fp32", L.DTYPE_F32)):
        ctx.init_embeddings(1, DIM, dtype, seed=1)
        ctx.init_embeddings(2, DIM, dtype, seed=2)
        o = L.train_opts_default()
        o.batch = B
        tuned = None
        if dtype == L.DTYPE_BF16:
            o, tuned = ctx.autotune(2, DIM, K, batches=[4096, 8192, 16384, 32768, 65536], both_orders=True,
                                    total=n, opts=o)
        n_run = n // o.batch * o.batch
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            ctx.train_orders(DIM, K, n_run, 5, total=n_run, opts=o)
            ev1.record(stream)
            torch.cuda.synchronize()
        sec = ev0.elapsed_time(ev1) / 1e3
        row = DIM * (2 if dtype == L.DTYPE_BF16 else 4)
        rate = 2 * n_run / sec
        alg = 14 * row
        res[name] = {"value": rate, "seconds": sec, "samples_per_order": n_run, "batch": int(o.batch),
                     "mode": "batched" if o.mode == L.MODE_BATCHED else "persistent",
                     "warps_per_block": int(o.warps_per_block), "chunk_batches": int(o.chunk_batches),
                     "autotuned_rate_both_orders": tuned,
                     "roofline": {"bound": "hbm", "achieved": rate * alg / 1e9, "peak": peak, "unit": "GB/s",
                                  "frac": rate * alg / 1e9 / peak, "alg_bytes_per_sample": alg, "peak_kind": peak_kind,
                                  "scope": "both orders' update phases over the timed region"},
                     "auc_orders_1_2": ctx.eval_auc(3, hs, hd, ns, nd)[0],
                     "auc_order_2": ctx.eval_auc(2, hs, hd, ns, nd)[0],
                     "loss_order_2": ctx.eval_loss(2, K, 99, 1 << 20), "clocks": clk.summary()}
    line = {"metric": METRIC, "value": res["bf16"]["value"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "rmat24_line_order1+2_d128_K5_bf16_vs_fp32",
                       "graph": "R-MAT scale 24, edge factor 16, (.57,.19,.19,.05), symmetrised; 10% of edges held out",
                       "n_nodes": tr.n_nodes, "n_arcs_train": E, "epochs": args.epochs,
                       "auc_pairs": len(hs), "generation_s": t_gen,
                       "tables": "BF16 U1+U2+C2 = 12.9 GB; FP32 25.8 GB"},
            "bf16": res["bf16"], "fp32": res["fp32"],
            "auc_diff_bf16_minus_fp32": res["bf16"]["auc_orders_1_2"] - res["fp32"]["auc_orders_1_2"]}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_mlp20(args):
    """The MLP input, fit and prediction kernels on R-MAT 20 (two
    repetitions): the inputs of every node, then of the held-out rows; a fit
    of 16 Adam steps of 16,384 rows on 65,536 kept nodes (the warm start's
    default); the held-out rows' predictions written into their table rows."""
    import numpy as np
    import torch

    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    g = I.rmat20()
    ctx = L.Context(local, stream.cuda_stream)
    ctx.build_alias(g.n_nodes, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                    torch.from_numpy(g.w).cuda())
    ctx.init_embeddings(2, DIM, L.DTYPE_BF16, seed=2)
    ctx.mlp_create(2, hidden=256, act_dtype=L.DTYPE_BF16, seed=9)
    held = I.uniform01(1, I.STREAM_NODE_SPLIT, np.arange(g.n_nodes, dtype=np.uint64)) < 0.1
    known = torch.from_numpy((~held).astype(np.uint8)).pin_memory()
    rows = torch.from_numpy(np.flatnonzero(held).astype(np.int32)).pin_memory()
    fit_nodes = torch.from_numpy(np.flatnonzero(~held)[:1 << 16].astype(np.int32)).cuda()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    reps = []
    for _ in range(2):
        reps.append({"inputs_all_ms": timed(lambda: ctx.mlp_features(known)),
                     "inputs_rows_ms": timed(lambda: ctx.mlp_features_rows(known, rows)),
                     "fit_ms": timed(lambda: ctx.mlp_train(fit_nodes, 16, 16384, 1e-3, 3, losses=False)),
                     "predict_ms": timed(lambda: ctx.mlp_predict(rows))})
    line = {"metric": "warm-start MLP kernels, device ms", "unit": "ms", "value": reps[-1]["predict_ms"],
            "higher_is_better": False, "n_gpus": 1, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "mlp20_inputs_and_predictions_d128_h256_bf16", "n_nodes": g.n_nodes,
                       "n_arcs": g.n_arcs, "rows": int(rows.shape[0])},
            "repetitions": reps}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_reuse20(args):
    """Walk reuse r in {1, 4, 16} x {minibatch, Hogwild}: throughput vs quality."""
    import torch

    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    g = I.rmat20()
    tr, hs, hd = I.split_edges(g, 0.1, seed=4)
    ns, nd = I.non_edges(g, len(hs), seed=7)
    ctx = L.Context(local, stream.cuda_stream)
    ctx.build_alias(tr.n_nodes, torch.from_numpy(tr.src).cuda(), torch.from_numpy(tr.dst).cuda(),
                    torch.from_numpy(tr.w).cuda())
    n = args.epochs * tr.n_arcs // B * B
    peak, peak_kind = peaks()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for mode, mname in ((L.MODE_BATCHED, "batched"), (L.MODE_HOGWILD, "hogwild")):
        for r in (1, 4, 16):
            ctx.init_embeddings(1, DIM, L.DTYPE_F32, seed=1)
            ctx.init_embeddings(2, DIM, L.DTYPE_F32, seed=2)
            o = L.train_opts_default()
            o.batch = B
            o.mode = mode
            o.walk_length, o.window, o.walk_reuse = args.walk_length, args.window, r
            torch.cuda.synchronize()
            with ClockSampler(local) as clk:
                ev0.record(stream)
                ctx.train_orders(DIM, K, n, 5, total=n, opts=o)
                ev1.record(stream)
                torch.cuda.synchronize()
            sec = ev0.elapsed_time(ev1) / 1e3
            rate = 2 * n / sec
            rows.append({"mode": mname, "reuse": r, "value": rate, "seconds": sec,
                         "roofline_frac": rate * ALG_BYTES_UPDATE / 1e9 / peak,
                         "auc_orders_1_2": ctx.eval_auc(3, hs, hd, ns, nd)[0],
                         "auc_order_2": ctx.eval_auc(2, hs, hd, ns, nd)[0],
                         "loss_order_2": ctx.eval_loss(2, K, 99, 1 << 20), "clocks": clk.summary()})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    line = {"metric": "walk-pair updates/s (d=128,K=5) and AUC by walk reuse", "unit": UNIT,
            "value": max(x["value"] for x in rows), "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"rmat20_walk{args.walk_length}w{args.window}_reuse_ablation",
                       "graph": "R-MAT scale 20, edge factor 16, (.57,.19,.19,.05), symmetrised; 10% of edges held out",
                       "n_nodes": tr.n_nodes, "n_arcs_train": tr.n_arcs, "epochs": args.epochs,
                       "samples_per_order": n, "auc_pairs": len(hs), "peak_gbs": peak, "peak_kind": peak_kind},
            "runs": rows}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "rmat20walk":
        args.scale = 20
    if args.workload == "dchung22":
        run_dchung22(args)
        return
    if args.workload == "warm22":
        run_warm22(args)
        return
    if args.workload == "rmat24":
        run_rmat24(args)
        return
    if args.workload == "reuse20":
        run_reuse20(args)
        return
    if args.workload == "mlp20":
        run_mlp20(args)
        return
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2604_09419_gb300 import inputs as I
    from paper_2604_09419_gb300 import line as L

    g = I.rmat(args.scale, seed=0)
    S = samples_per_step(args)
    total_per_order = 20 * 16 * (1 << args.scale)
    stream = torch.cuda.current_stream()
    ctx = L.Context(local, stream.cuda_stream)
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    w = torch.from_numpy(g.w).cuda()
    ctx.build_alias(g.n_nodes, src, dst, w)
    mode = {"auto": L.MODE_BATCHED, "batched": L.MODE_BATCHED, "persistent": L.MODE_PERSISTENT,
            "hogwild": L.MODE_HOGWILD}[args.mode]
    seed = replica_seed(rank)

    walk_len, window = walk_of(args)
    tdtype = L.DTYPE_BF16 if args.dtype == "bf16" else L.DTYPE_F32
    rb = row_bytes(args.dtype)
    alg_update = 14 * rb
    alg_path = alg_update + META_BYTES

    def opts(offset):
        o = L.train_opts_default()
        o.batch = B
        o.mode = mode
        o.timing = 1
        o.sample_offset = offset
        o.walk_length = walk_len
        o.window = window
        return o

    ctx.init_embeddings(1, DIM, tdtype, seed=1)
    ctx.init_embeddings(2, DIM, tdtype, seed=2)
    state = {"offset": 0}

    concurrent = args.orders == "concurrent"

    def step():
        off = state["offset"] % total_per_order
        if concurrent:
            ctx.train_orders(DIM, K, S, seed, total=total_per_order, opts=opts(off))
        else:
            for order in (1, 2):
                ctx.train_steps(order, DIM, K, S, seed, total=total_per_order, opts=opts(off))
        state["offset"] += S

    for _ in range(args.warmup):
        step()
    ctx.reset_stats()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    st = ctx.stats()
    ms = max_over_ranks(ms, world)
    updates = 2 * S * args.steps * world
    value = updates / (ms / 1e3)

    peak, peak_kind = peaks()
    update_kernels = {L.MODE_BATCHED: "k_gather + k_apply", L.MODE_PERSISTENT: "k_persistent",
                      L.MODE_HOGWILD: "k_hogwild"}[mode]
    if concurrent:
        # the two orders' update kernels overlap on two streams, so per-launch
        # durations overlap too: their algorithmic bytes over the timed
        # region (CUDA events on the caller's stream) instead
        achieved = 2 * S * args.steps * alg_update / (ms / 1e3) / 1e9
        kernel = f"update phase of both orders ({update_kernels}), concurrent streams, over the timed region"
    else:
        # the update kernels' own CUDA events
        upd_ms = st.update_ms
        achieved = st.update_samples * alg_update / (upd_ms / 1e3) / 1e9 if upd_ms > 0 else None
        kernel = f"update phase ({update_kernels}), its own CUDA events"
    traffic = (measured_traffic() if mode == L.MODE_BATCHED and args.scale == 20 and not walk_len
               and args.dtype == "fp32" else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_unit": "DRAM bytes per 4,096-sample batch (k_gather + k_apply, warm L2)",
                "traffic_source": ("not measured in this run: the ncu summary "
                                   "profiles/k_gather_k_apply_rmat20_d128_K5_B4096.md, taken on the same train.cu "
                                   "(sha256 prefix checked)") if traffic else None,
                "alg_bytes_per_batch": B * alg_update,
                "kernel": kernel,
                "alg_bytes_per_sample": alg_update, "peak_kind": peak_kind,
                "path_achieved_gbs": value / world * alg_path / 1e9,
                "path_frac": value / world * alg_path / 1e9 / peak}
    # kernel launches of the library in the timed region, counted by the
    # library (line_get_stats; a replayed CUDA graph counts its kernels)
    launches = int(st.update_launches + st.prepass_launches)

    # the same workload with BF16 tables, and one order alone (FP32, BF16):
    # a few timed steps each, after the main measurement, on fresh tables
    variants = None
    if (rank == 0 and world == 1 and mode == L.MODE_BATCHED and not walk_len and args.dtype == "fp32"
            and concurrent and not args.no_variants):
        variants = {}
        for name, vdt, both in (("bf16_both_orders", L.DTYPE_BF16, True), ("fp32_one_order", L.DTYPE_F32, False),
                                ("bf16_one_order", L.DTYPE_BF16, False)):
            ctx.init_embeddings(1, DIM, vdt, seed=1)
            ctx.init_embeddings(2, DIM, vdt, seed=2)
            vst = {"offset": 0}

            def vstep():
                off = vst["offset"] % total_per_order
                if both:
                    ctx.train_orders(DIM, K, S, seed, total=total_per_order, opts=opts(off))
                else:
                    ctx.train_steps(2, DIM, K, S, seed, total=total_per_order, opts=opts(off))
                vst["offset"] += S

            vsteps = 5
            for _ in range(2):
                vstep()
            torch.cuda.synchronize()
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(vsteps):
                vstep()
            v1.record(stream)
            torch.cuda.synchronize()
            vrate = (2 if both else 1) * S * vsteps / (v0.elapsed_time(v1) / 1e3)
            vpath = 14 * row_bytes("bf16" if vdt == L.DTYPE_BF16 else "fp32") + META_BYTES
            variants[name] = {"value": vrate, "unit": UNIT, "steps": vsteps, "warmup": 2,
                              "path_bytes_per_update": vpath, "path_frac": vrate * vpath / 1e9 / peak}

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        hs = torch.from_numpy(g.src).pin_memory()
        hd = torch.from_numpy(g.dst).pin_memory()
        hw = torch.from_numpy(g.w).pin_memory()
        tt = torch.bfloat16 if tdtype == L.DTYPE_BF16 else torch.float32
        outs = [torch.empty((g.n_nodes, DIM), dtype=tt).pin_memory() for _ in range(3)]
        ctx2 = L.Context(local, stream.cuda_stream)

        phases = []

        def e2e_step():
            # the step's inputs from pinned host memory, the whole path, and
            # its result (both orders' tables) back to pinned host memory;
            # every call but init_embeddings returns after its work is done,
            # so host stamps between them split the step
            t = [time.perf_counter()]
            ctx2.build_alias(g.n_nodes, hs, hd, hw)
            t.append(time.perf_counter())
            ctx2.init_embeddings(1, DIM, tdtype, seed=1)
            ctx2.init_embeddings(2, DIM, tdtype, seed=2)
            if concurrent:
                ctx2.train_orders(DIM, K, S, seed, total=total_per_order, opts=opts(0))
            else:
                for order in (1, 2):
                    ctx2.train_steps(order, DIM, K, S, seed, total=total_per_order, opts=opts(0))
            t.append(time.perf_counter())
            ctx2.get_embeddings(1, L.WHICH_U, outs[0], tdtype)
            ctx2.get_embeddings(2, L.WHICH_U, outs[1], tdtype)
            ctx2.get_embeddings(2, L.WHICH_C, outs[2], tdtype)
            t.append(time.perf_counter())
            phases.append([1e3 * (b - a) for a, b in zip(t, t[1:])])

        e2e_step()  # untimed warm-up: the context's first-use allocations
        phases.clear()
        barrier()
        gc.collect()
        gc.disable()  # no collector pause inside the host-timed region (as timeit does)
        with ClockSampler(local) as eclk:
            t0 = time.perf_counter()
            for i in range(args.e2e_steps):
                e2e_step()
            barrier()
            dt = time.perf_counter() - t0
        gc.enable()
        ctx2.close()
        med = [sorted(p[k] for p in phases)[len(phases) // 2] for k in range(3)]
        e2e = {"value": 2 * S * args.e2e_steps * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(g.n_arcs * 12), "d2h_bytes_per_step": int(3 * g.n_nodes * rb),
               "includes": "graph upload + alias build + table init + both orders + read-back of U1, U2 and C2",
               "warmup": 1, "steps": args.e2e_steps,
               "phases_ms_median": {"upload_and_alias_build": med[0], "init_and_training": med[1], "read_back": med[2]},
               "step_ms": [sum(p) for p in phases],
               "clocks": eclk.summary()}

    cpu = None
    cpu_mt = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, args.cpu_samples, walk_of(args), pairwise=mode == L.MODE_HOGWILD)
        if not walk_len:
            cpu_mt = cpu_hogwild_context(g, 4 * args.cpu_samples)

    # the third part of the metric: BF16 + warm start against the plain FP32
    # path at equal AUC, on R-MAT 20 (the warm22 workload runs it on R-MAT 22)
    warm = None
    if rank == 0 and world == 1 and not walk_len and not args.no_warm:
        w = warm_compare(20, fit_nodes=args.fit_nodes, fit_steps=args.fit_steps, curves=False)
        warm = {"workload": "warm20_rmat20_order2_d128_K5_B4096", **w}

    # configuration C3 (directed Chung-Lu, order 2, BF16 autotuned against
    # FP32), two timed steps of |E| samples per arm
    c3 = None
    if rank == 0 and world == 1 and not walk_len and not args.no_c3:
        c3 = c3_compare(2, 1)

    if rank == 0:
        line = {"metric": metric_of(args), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if args.dtype == "bf16" else "f32",
                "data": "synthetic",
                "config": workload_config(args, g), "roofline": roofline, "cpu_baseline": cpu,
                "cpu_hogwild_context": cpu_mt,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(), "variants": variants, "warm": warm,
                "c3": c3,
                "mode": {L.MODE_BATCHED: "batched", L.MODE_PERSISTENT: "persistent", L.MODE_HOGWILD: "hogwild"}[mode],
                "orders": args.orders}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
