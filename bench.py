"""Benchmark: Expected Force (EF_2) of every node, clusters/s on one GB300.

Workload (default): the power-law configuration model with n = 4,000,000,
P(d) ~ d^-2.3 on [3, 20000], seed 20230609 -- the ~44M-entry power-law graph
(20.7M undirected edges, 41.3M CSR entries, 1.28e10 clusters).  Other
workloads: --workload ba1m (Barabasi-Albert n=1e6, m=5) or er2000.

One step = one ef_compute_ex call over the whole graph (validation, prep,
wedge pass, triangle pass, finalize), FP32-compensated path, inputs resident
in HBM.  The metric is clusters/s = W / step time with W = sum_v C(D_v, 2),
the number of clusters Algorithm 1 enumerates.

Prints one JSON line.  Beside the headline it carries the other workloads
(`workloads`: ER 2000 and BA 1M in both precisions, the power-law graph in
FP64, its minimum-degree-6 variant with 4.4e7 undirected edges, the 4096-graph
Watts-Strogatz batch with its per-graph time distribution, BA 16M).
`--impl reference` times the CPU oracle instead (the vertex-centric
formulation, OpenMP over the host cores) on bounded random node samples of
the same graph, the same samples the `cpu_baseline` key reports.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    "plcm4m": (3, "power-law configuration model n=4000000 gamma=2.3 degrees in [3,20000] seed=20230609"),
    "ba1m": (2, "Barabasi-Albert n=1000000 m=5 seed=20230608"),
    "er2000": (1, "Erdos-Renyi G(n=2000, p=0.004) seed=20230607"),
    "ws4096": (4, "batch of 4096 Watts-Strogatz graphs, n ~ U[200,20000], k ~ U{4,...,12} even, p=0.1, "
                  "seed=20230610, one ef_compute_batched call (replayed CUDA graph)"),
    "plcm4m_d6": ("3b", "power-law configuration model n=4000000 gamma=2.3 degrees in [6,20000] seed=20230612 "
                        "(4.4e7 undirected edges)"),
    "ba16m": (5, "Barabasi-Albert n=16000000 m=4 seed=20230611"),
}
BATCHED = {"ws4096"}
PASSES = ("prep_ms", "orient_ms", "wedge_small_ms", "wedge_big_ms", "tri_pairs_ms", "finalize_ms")
PASS_KERNEL = {"prep_ms": "k_degrees+k_row_stats+k_row_stats_hub",
               "orient_ms": "k_ftab+layout+scan+k_node_info+k_orient+k_orient_hub+k_hash_rows",
               "wedge_small_ms": "k_wedge_small<4,8,16,32>", "wedge_big_ms": "k_wedge_mid+k_wedge_hub",
               "tri_pairs_ms": "k_tri_pairs", "finalize_ms": "k_finalize"}
PASS_NOTE = {"prep_ms": "bound by random L2 gathers of neighbour degrees",
             "orient_ms": "bound by random L2 gathers of neighbour records; also fills the out-list hash tables",
             "wedge_small_ms": "bound by MUFU lg2 and FP32 adds (one f evaluation per ordered pair)",
             "wedge_big_ms": "bound by MUFU lg2 and FP32 adds over degree classes, and L2 reductions",
             "tri_pairs_ms": "bound by dependent L2 round trips (1.1e8 membership tests), not HBM bandwidth",
             "finalize_ms": "streaming, HBM-bound"}


def algorithmic_bytes(g, st):
    """Bytes each pass must move at least once (inputs read once, outputs
    written once; gathers that hit L2 are not counted)."""
    n, m = g.n, g.nnz
    d = g.degrees.astype(np.int64)
    small = d[(d >= 1) & (d <= 32)]
    big = d[d > 32]
    csr = 4 * (n + 1) + 4 * m
    return {
        # row_ptr + col_idx read; D, sigma1, sigma2, outdeg written
        "prep_ms": csr + 4 * n + 16 * n + 4 * n,
        # CSR + outdeg read; out_ptr, out_col/out_D/out_src/out_pd (20 B per
        # oriented entry), hash tables (2 slots per entry), omega written
        "orient_ms": csr + 4 * n + 4 * (n + 1) + 28 * (m // 2) + 8 * n,
        # rows of the middle nodes read; Ccenter written, one 8-byte credit per row entry
        "wedge_small_ms": 4 * len(small) * 2 + 4 * int(small.sum()) + 8 * len(small) + 8 * int(small.sum()),
        "wedge_big_ms": 4 * len(big) * 2 + 4 * int(big.sum()) + 8 * len(big) + 8 * int(big.sum()),
        # out_ptr, out_col, out_D, out_src, out_pd read; qacc, tcnt written
        "tri_pairs_ms": 4 * (n + 1) + 20 * (m // 2) + 16 * n,
        # D and 7 eight-byte per-node arrays read, EF written
        "finalize_ms": 4 * n + 7 * 8 * n + 8 * n,
    }


PASS_PREFIX = {"prep_ms": ("k_degrees", "k_row_stats", "k_gate"),
               "orient_ms": ("k_ftab", "k_layout", "k_scan", "k_node_info", "k_orient", "k_hash"),
               "wedge_small_ms": ("k_wedge_small",), "wedge_big_ms": ("k_wedge_mid", "k_wedge_hub", "k_wedge_big", "k_big"),
               "tri_pairs_ms": ("k_tri_pairs",), "finalize_ms": ("k_finalize",)}


def committed_kernels(workload):
    """Per-kernel figures of the committed ncu launch list of `workload`
    (profiles/traffic.json: DRAM bytes per launch, L2 hit rate, share of the
    launch time), for the kernels whose source file is unchanged since the
    capture; {} when there is none."""
    import hashlib
    try:
        recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[workload]
    except (OSError, KeyError, ValueError, TypeError):
        return {}
    out, sha = {}, {}
    for k, r in recs.items():
        try:
            if r["source"] not in sha:
                sha[r["source"]] = hashlib.sha256(open(os.path.join(ROOT, r["source"]), "rb").read()).hexdigest()[:16]
            if sha[r["source"]] == r["source_sha256_16"]:
                out[k] = r
        except (OSError, KeyError, TypeError):
            continue
    return out


def passes_ncu(workload):
    """Per pass, from committed_kernels: the kernels, their summed share of the
    launch time and DRAM bytes per launch (the full-size launch list), and,
    time-weighted over the pass's kernels, the L2 hit rate, the share of
    cycles in which a warp scheduler issued (the pass's issue or ALU
    fraction) and the warp slots in use (a smaller case of the same kernels,
    inputs still larger than L2; None for a pass with no fresh record)."""
    recs = committed_kernels(workload)
    res = {}
    for p, pre in PASS_PREFIX.items():
        ks = {k: r for k, r in recs.items() if k.startswith(pre)}
        if not ks:
            res[p] = None
            continue
        t = sum(r["ms_per_launch"] * r["launches"] for r in ks.values())
        def weighted(field):
            # time-weighted over the pass's kernels that have the figure
            hk = {k: r for k, r in ks.items() if r.get(field) is not None}
            th = sum(r["ms_per_launch"] * r["launches"] for r in hk.values())
            return sum(r[field] * r["ms_per_launch"] * r["launches"] for r in hk.values()) / th if th > 0 else None
        res[p] = {"kernels": sorted(ks), "ncu_share": sum(r["share"] for r in ks.values()),
                  "dram_bytes_per_launch": sum(r["dram_bytes_per_launch"] for r in ks.values()),
                  "l2_hit_pct": weighted("l2_hit_pct"),
                  "issue_active_pct": weighted("issue_active_pct"),
                  "warps_active_pct": weighted("warps_active_pct")}
    return res


def committed_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` (name prefix) from the committed ncu
    launch list, or None when there is none for this workload or the
    kernel's source has changed since it was taken."""
    ks = [r for k, r in committed_kernels(workload).items() if k.startswith(kernel)]
    return ks[0]["dram_bytes_per_launch"] if len(ks) == 1 else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=list(WORKLOADS), default="plcm4m")
    p.add_argument("--precision", choices=["fp32c", "fp64"], default="fp32c")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--scale", type=float, default=1.0,
                   help="shrink the workload's node count (small cases for profiling; not a bench line)")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    p.add_argument("--autotune", action="store_true", help="run ef_autotune on the workload before timing")
    p.add_argument("--no-surrogate", action="store_true", help="skip the learned ranking leg")
    p.add_argument("--surrogate-steps", type=int, default=3000)
    p.add_argument("--no-shards", action="store_true", help="skip the sharded-decomposition leg")
    p.add_argument("--no-workloads", action="store_true", help="skip the other workloads' leg")
    p.add_argument("--sir", action="store_true", help="run the SIR validation leg (Figs. 6-8 protocols, BA 1M)")
    p.add_argument("--sir-batch", type=int, default=0, metavar="B",
                   help="only time one ef_sir_run of B simulations from the highest-degree node of BA 1M "
                        "(one call, for profiling)")
    p.add_argument("--rmat-sweep", action="store_true",
                   help="add EF time and clusters/ms on R-MAT graphs of 2^16 nodes, M = 2..32 edges per node")
    return p.parse_args()


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of one number per rank (a MAX all-reduce; the value itself at N = 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def class_evals(g, hub_min: int = 513) -> int:
    """f evaluations of the degree-class wedge kernels: K (K + 1) per middle
    node of degree > 32, K its classes.  Neighbour degrees below 256 (warp
    kernel, degree < hub_min) or 2048 (CTA kernel) merge into one class per
    degree; larger ones are a class each, as the kernels build them."""
    d = g.degrees.astype(np.int64)
    big = np.nonzero(d > 32)[0]
    if big.size == 0:
        return 0
    rp = g.row_ptr.astype(np.int64)
    lens = d[big]
    owner = np.repeat(np.arange(big.size), lens)
    idx = np.arange(owner.size) - np.repeat(np.cumsum(lens) - lens, lens) + np.repeat(rp[big], lens)
    dn = d[g.col_idx[idx]]
    dense = dn < np.where(d[big] < hub_min, 256, 2048)[owner]
    keys = np.unique(owner[dense] * (int(d.max()) + 1) + dn[dense])
    K = np.bincount(keys // (int(d.max()) + 1), minlength=big.size) + np.bincount(owner[~dense], minlength=big.size)
    return int((K * (K + 1)).sum())


def graph_stats(g):
    d = g.degrees.astype(np.int64)
    W = int((d * (d - 1) // 2).sum())
    big = d[d > 32]
    return dict(n=g.n, nnz=g.nnz, W=W, big_evals=int((big * (big - 1)).sum()),
                small_evals=int((d[d <= 32] * (d[d <= 32] - 1)).sum()), maxdeg=int(d.max()) if g.n else 0)


def _closed_credits(g):
    """Credited clusters per node, N_v = D_v (D_v - 2) + sigma1(v) (the oracle's work per node)."""
    d = g.degrees.astype(np.int64)
    src = np.repeat(np.arange(g.n), d)
    return d * (d - 2) + np.bincount(src, weights=d[g.col_idx], minlength=g.n).astype(np.int64)


def oracle_steps(g, steps: int, seconds: float, seed0: int = 0, threads: int = 0):
    """Time the oracle (vertex-centric, OpenMP dynamic over all host cores) on
    `steps` random node samples of about `seconds` each; yields one dict per
    step.  A sample draws uniformly from the nodes whose own work (N_v
    credits) is at most 1/(2 x cores) of the step's, so that no single node
    keeps one core busy after the others finish, sorted largest first.  The
    step size comes from a short calibration run; seeds seed0, seed0 + 1, ...
    make the samples the same in every run."""
    import oracle
    cores = threads if threads > 0 else oracle.num_threads()
    N = _closed_credits(g)
    # calibration: random nodes of at most 50x the median work, doubling
    # until a run takes 0.25 s (or covers the graph)
    rng = np.random.default_rng(12345)
    pool = rng.permutation(np.nonzero(N <= max(int(np.median(N)) * 50, 1))[0]).astype(np.int32)
    k = min(2000, len(pool))
    while True:
        t0 = time.perf_counter()
        oracle.vertex(g, pool[:k], threads=cores)
        dt = time.perf_counter() - t0
        if dt >= 0.25 or k >= len(pool):
            break
        k = min(len(pool), 2 * k)
    rate = max(int(N[pool[:k]].sum()), 1) / max(dt, 1e-4)   # credits/s
    target = rate * seconds
    cap = max(target / (2 * cores), float(np.percentile(N, 50)))
    eligible = np.nonzero(N <= cap)[0]
    for i in range(steps):
        r = np.random.default_rng(seed0 + i)
        perm = r.permutation(eligible)
        k = int(np.searchsorted(np.cumsum(N[perm]), target)) + 1
        nodes = perm[:min(k, len(perm))]
        nodes = nodes[np.argsort(-N[nodes], kind="stable")].astype(np.int32)
        t0 = time.perf_counter()
        res = oracle.vertex(g, nodes, threads=cores)
        dt = time.perf_counter() - t0
        yield {"nodes": len(nodes), "clusters": int(res["N"].sum()) / 4, "s": dt, "cores": cores,
               "eligible": len(eligible), "cap": cap}


def cpu_baseline(g, seconds: float, steps: int = 3, seed0: int = 0):
    """The oracle's clusters/s on `steps` samples of `seconds` / `steps` each
    (oracle_steps; a sample's cluster count is its nodes' credited clusters
    / 4, as every cluster carries 4 credits, so the rate compares with W/t)."""
    rows = list(oracle_steps(g, steps, seconds / steps, seed0))
    clusters = sum(r["clusters"] for r in rows)
    t = sum(r["s"] for r in rows)
    return {"value": clusters / t, "unit": "clusters/s", "cores": rows[0]["cores"], "kind": "oracle",
            "sample": f"{steps} samples (seeds {seed0}..{seed0 + steps - 1}) of {sum(r['nodes'] for r in rows)} "
                      f"uniformly random nodes in all, drawn from the {rows[0]['eligible']} nodes with at most "
                      f"{rows[0]['cap']:.3g} credited clusters; vertex-centric oracle, OpenMP dynamic,2, "
                      f"{clusters:.3g} clusters = credited/4, {t:.1f} s"}


def rmat_sweep(ctx, args, dev) -> list:
    """EF of R-MAT graphs with 2^16 nodes and M = 2..32 edges per node
    (a, b, c = 0.57, 0.19, 0.19; the paper's Figs. 3-4 setting, parameters
    not printed there): ms per graph and clusters per ms on the GPU, and
    the oracle's clusters per ms on the host cores (a node sample of about
    2 s per graph)."""
    import torch
    import paper_2306_00606_gb300 as ef
    rows = []
    stream = torch.cuda.current_stream(dev)
    for M in (2, 4, 8, 16, 32):
        g = synth.rmat(16, M, synth.SEED_BASE + 100 + M)
        rp = torch.from_numpy(g.row_ptr).to(dev)
        ci = torch.from_numpy(g.col_idx).to(dev)
        out = torch.empty(g.n, dtype=torch.float64, device=dev)
        # as the headline step: validation on the device, one replayed CUDA graph per call
        for _ in range(3):
            ef.ef_compute_ex(ctx.handle, rp, ci, precision=args.precision, ef=out, device_check=True, graph=True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            ef.ef_compute_ex(ctx.handle, rp, ci, precision=args.precision, ef=out, device_check=True, graph=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 10
        W = graph_stats(g)["W"]
        cpu = cpu_baseline(g, 2.0, steps=1, seed0=M)
        rows.append({"M": M, "nodes": g.n, "nnz": g.nnz, "avg_degree": g.nnz / g.n, "clusters": W, "ms": ms,
                     "clusters_per_ms": W / ms, "oracle_clusters_per_ms": cpu["value"] / 1e3,
                     "oracle_cores": cpu["cores"], "gpu_over_oracle": (W / ms) / (cpu["value"] / 1e3)})
    return rows


def shard_leg(ctx, rp, ci, args, dev, full_ms: float) -> list:
    """The sharded decomposition on one device: for R shards, the time of
    each shard's ef_compute_shard (CUDA events on the context stream, best of
    3 rounds) and of the finalize from summed partials.  On R devices a job
    would take the slowest shard, the all-reduce of 40 bytes per node and
    the finalize."""
    import torch
    import paper_2306_00606_gb300 as ef
    n = int(rp.shape[0]) - 1
    stream = torch.cuda.current_stream(dev)
    parts = ef.empty_partials(n, dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), r

    rows = []
    for R in (2, 4, 8):
        best = [float("inf")] * R
        for _ in range(3):
            for r in range(R):
                ms, (frac, _) = timed(lambda: ef.ef_compute_shard(ctx.handle, rp, ci, r, R, parts,
                                                                   precision=args.precision))
                best[r] = min(best[r], ms)
        fin = min(timed(lambda: ef.ef_finalize_partials(ctx.handle, parts, frac, precision=args.precision,
                                                         ef=out))[0] for _ in range(3))
        rows.append({"shards": R, "shard_ms_max": max(best), "shard_ms_mean": sum(best) / R,
                     "finalize_ms": fin, "unsharded_ms": full_ms,
                     "projected_speedup_excl_allreduce": full_ms / (max(best) + fin)})
    return rows


def sir_leg(args, dev) -> dict:
    """SIR validation of EF with Section 5.4's protocols on the BA n=1M, m=5
    workload, calibrated as Section 3.1 (gamma = 1/3, beta = 1.3 / (3 <k>)):
    Fig. 7: 10 equally spaced EF values, the node nearest to each as index
    case of 100 simulations: share of global outbreaks (final size >= 25% of
    the nodes), mean final size, length and time to peak; Fig. 6: Pearson's
    r between the spreading power of order 1-4 over global outbreaks (from
    random index cases) and exp(EF), and degree; Fig. 8: 5% of the nodes
    immunized, 10 sets of increasing mean EF, 100 simulations each.  Times
    are CUDA events around ef_sir_run; the oracle runs a few of the same
    simulations on the host for a rate beside it."""
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.workload(2)
    n = g.n
    rp = torch.from_numpy(g.row_ptr).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    ctx = ef.Context(dev.index, torch.cuda.current_stream(dev))
    E = ctx.compute(rp, ci, precision="fp64", outputs=("ef",))["ef"].cpu().numpy()
    deg = np.diff(g.row_ptr).astype(np.float64)
    beta, gamma = 1.3 / (3 * g.nnz / n), 1.0 / 3.0
    glob = int(np.ceil(0.25 * n))
    stream = torch.cuda.current_stream(dev)
    timing = {"sims": 0, "ms": 0.0, "infections": 0}

    def run(index, chunk=500, base=0, **kw):
        outs = []
        for c0 in range(0, len(index), chunk):
            ix = torch.from_numpy(np.ascontiguousarray(index[c0:c0 + chunk], dtype=np.int32)).to(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o = ctx.sir(rp, ci, ix, beta=beta, gamma=gamma, seed=2306, sim_base=base + c0, **kw)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            timing["ms"] += e0.elapsed_time(e1)
            timing["sims"] += len(ix)
            timing["infections"] += int(o["final_size"].sum())
            outs.append({k: v.cpu().numpy() for k, v in o.items()})
        return outs

    # Fig. 7
    levels = np.linspace(E.min(), E.max(), 10)
    idx = np.array([int(np.argmin(np.abs(E - L))) for L in levels])
    outs = run(np.repeat(idx, 100), outputs=("final_size", "length", "peak_step"))
    fs = np.concatenate([o["final_size"] for o in outs]).reshape(10, 100)
    ln = np.concatenate([o["length"] for o in outs]).reshape(10, 100)
    pk = np.concatenate([o["peak_step"] for o in outs]).reshape(10, 100)
    fig7 = [{"ef": float(E[i]), "degree": int(deg[i]), "global_pct": float((fs[j] >= glob).mean() * 100),
             "mean_final_size": float(fs[j].mean()), "mean_length": float(ln[j].mean()),
             "mean_time_to_peak": float(pk[j].mean())} for j, i in enumerate(idx)]
    # Fig. 6
    rng = np.random.default_rng(6)
    rand_idx = rng.integers(0, n, 1000)
    outs = run(rand_idx, base=10000, outputs=("final_size", "spread"), spread_min_size=glob)
    G = int(sum((o["final_size"] >= glob).sum() for o in outs))
    spread = sum(o["spread"].astype(np.float64) for o in outs)
    fig6 = {"global_outbreaks": G, "simulations": len(rand_idx)}
    if G > 0:
        sp = spread / G
        for kk in range(4):
            fig6[f"order{kk + 1}"] = {"r_exp_ef": float(np.corrcoef(sp[kk], np.exp(E))[0, 1]),
                                      "r_degree": float(np.corrcoef(sp[kk], deg)[0, 1])}
    # Fig. 8
    order = np.argsort(E, kind="stable")
    bins = np.array_split(order, 20)   # 5% of the nodes each, by increasing EF
    chosen = [bins[j] for j in np.linspace(0, 19, 10).astype(int)]
    imm = np.zeros((10, n), np.uint8)
    for j, b in enumerate(chosen):
        imm[j, b] = 1
    free = np.nonzero(imm.sum(axis=0) == 0)[0]
    index = rng.choice(free, 1000)
    sets = np.repeat(np.arange(10, dtype=np.int32), 100)
    imm_d = torch.from_numpy(imm).to(dev)
    fsz = []
    for c0 in range(0, 1000, 500):
        o = run(index[c0:c0 + 500], base=20000 + c0, outputs=("final_size",), immune=imm_d,
                immune_set=torch.from_numpy(sets[c0:c0 + 500]).to(dev))
        fsz.append(o[0]["final_size"])
    fsz = np.concatenate(fsz).reshape(10, 100)
    fig8 = [{"mean_ef_immunized": float(E[b].mean()), "global_pct": float((fsz[j] >= glob).mean() * 100)}
            for j, b in enumerate(chosen)]
    # the oracle on a few of the Fig. 7 simulations (top EF level: global outbreaks)
    from oracle import sir as osir
    t0 = time.perf_counter()
    r = osir.simulate(g, np.repeat(idx[-1:], 4), beta, gamma, seed=2306, sim_base=900)
    cpu_s = time.perf_counter() - t0
    del ctx
    return {"workload": "BA n=1e6, m=5", "beta": beta, "gamma": gamma, "global_threshold": glob,
            "gpu": {"simulations": timing["sims"], "ms": timing["ms"],
                    "simulations_per_s": timing["sims"] / (timing["ms"] / 1e3),
                    "infections_per_s": timing["infections"] / (timing["ms"] / 1e3)},
            "oracle": {"simulations": 4, "s": cpu_s, "infections_per_s": float(r["final_size"].sum()) / cpu_s,
                       "kind": "numpy oracle, one host thread"},
            "fig7_index_case_ef": fig7, "fig6_spreading_power": fig6, "fig8_immunization": fig8}


def sir_batch(args) -> int:
    """One ef_sir_run call: B simulations from the highest-degree node of the
    BA n=1M, m=5 workload (Section 3.1's calibration, seed 2), CUDA events."""
    import torch
    import paper_2306_00606_gb300 as ef
    dev = torch.device("cuda", 0)
    g = synth.workload(2)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    ctx = ef.Context(0, torch.cuda.current_stream(dev))
    top = int(np.argmax(np.diff(g.row_ptr)))
    idx = torch.full((args.sir_batch,), top, dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o = ctx.sir(rp, ci, idx, beta=1.3 / (3 * g.nnz / g.n), gamma=1.0 / 3.0, seed=2,
                outputs=("final_size", "length"))
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    inf = int(o["final_size"].sum())
    print(json.dumps({"sir_batch": args.sir_batch, "ms": ms, "simulations_per_s": args.sir_batch / ms * 1e3,
                      "infections_per_s": inf / ms * 1e3, "max_length": int(o["length"].max())}))
    ctx.close()
    return 0


def surrogate_leg(args, dev) -> dict:
    """The learned ranking path on the BA n=16M, m=4 workload: a network
    trained on exact EF of the ER 2000 and BA 1M workloads (features and
    labels from this library) ranks every node; exact EF of the best 2% and
    of a 0.1% audit sample.  Compared with exact EF of all nodes on the
    same GPU: top-1% recall, audit Spearman rho, and the time ratio."""
    import math
    import torch
    import paper_2306_00606_gb300 as ef
    ctx = ef.Context(dev.index)
    xs, ys = [], []
    for idx in (1, 2):
        g = synth.workload(idx)
        rp = torch.from_numpy(g.row_ptr).to(dev)
        ci = torch.from_numpy(g.col_idx).to(dev)
        x = torch.empty((g.n, 16), dtype=torch.float32, device=dev)
        ef.ef_features(ctx.handle, rp, ci, x, mode=0)
        y = torch.empty(g.n, dtype=torch.float64, device=dev)
        ef.ef_compute_ex(ctx.handle, rp, ci, precision=args.precision, ef=y)
        xs.append(x)
        ys.append(y.float())
    x, y = torch.cat(xs), torch.cat(ys)
    model = ef.Model(ctx.handle, seed=1)
    train = model.train(x, y, steps=args.surrogate_steps, batch=8192, lr=2e-3, seed=2)
    del x, y, xs, ys
    g = synth.workload(5)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    n = g.n
    exact = torch.empty(n, dtype=torch.float64, device=dev)
    kt = math.ceil(0.01 * n)
    idx_t = torch.empty(kt, dtype=torch.int32, device=dev)
    ef_t = torch.empty(kt, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    ms_exact = timed(lambda: ef.ef_compute_ex(ctx.handle, rp, ci, precision=args.precision, ef=exact), 3)
    ctx.stats(reset=True)
    ef.ef_compute_ex(ctx.handle, rp, ci, precision=args.precision, ef=exact, profile=True)
    exact_passes = {k: v for k, v in ctx.stats(reset=True).items() if k.endswith("_ms")}
    st = {}

    def rank():
        st.update(model.rank(rp, ci, idx_t, ef_t, top_frac=0.01, cand_frac=0.02, audit_frac=0.001, seed=3,
                             precision=args.precision))
    ms_rank = timed(rank, 3)
    ex = exact.cpu().numpy()
    order = np.lexsort((np.arange(n), -ex))[:kt]
    recall = len(np.intersect1d(order, idx_t.cpu().numpy())) / kt
    ctx.close()
    return {"workload": "Barabasi-Albert n=16000000 m=4 seed=20230611 (trained on the ER 2000 and BA 1M workloads)",
            "top_frac": 0.01, "cand_frac": 0.02, "audit_frac": 0.001, "top1pct_recall": recall,
            "spearman_audit": st.get("spearman_audit"), "max_abs_err_audit": st.get("max_abs_err_audit"),
            "ms_exact_all": ms_exact, "ms_surrogate_rank": ms_rank, "speedup_vs_exact_all": ms_exact / ms_rank,
            "rank_breakdown_ms": {k: st.get(k) for k in ("features_ms", "infer_ms", "select_ms", "exact_ms",
                                                         "exact_tri_ms", "exact_wedge_ms")},
            "exact_all_passes_ms": exact_passes,
            "train": dict(train, steps=args.surrogate_steps, batch=8192, lr=2e-3),
            "network": "16-64-64-1 ReLU, BF16 mma.sync, FP32 accumulate"}


def workload_config(desc, g, st, batched: bool, gpus: int) -> dict:
    """The `config` of a bench line: the workload and its sizes (both arms print the same)."""
    n = g.n
    return {"workload": desc, "nodes": n, "nnz": g.nnz, "edges": g.nnz // 2, "clusters": st["W"],
            "graphs": len(g.graph_off) - 1 if batched else 1, "max_degree": st["maxdeg"],
            "l2": f"inputs larger than L2 (CSR {(4 * (n + 1) + 4 * g.nnz) / 2**20:.0f} MiB), no flush",
            "parallelism": f"replicas x{gpus}"}


def run_reference(args):
    """The oracle as the reference arm: each step times the oracle on one
    bounded random node sample of the workload (oracle_steps: the samples of
    seeds 0, 1, ... are the ones `cpu_baseline` times in the GPU arm), about
    cpu_seconds / 3 per step, shortened so that the steps stay within about
    150 s (warm-up samples take at most 0.5 s each)."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    idx, desc = WORKLOADS[args.workload]
    g = synth.workload(idx)
    st = graph_stats(g)
    batched = args.workload in BATCHED
    per_step = min(args.cpu_seconds / 3, 150.0 / max(args.steps, 1))
    for _ in oracle_steps(g, args.warmup, min(per_step, 0.5), seed0=1000):   # short untimed warm-up samples
        pass
    rows = list(oracle_steps(g, args.steps, per_step, seed0=0))
    clusters = sum(r["clusters"] for r in rows)
    t = sum(r["s"] for r in rows)
    v = clusters / t
    line = {"impl": "reference", "metric": "clusters/s", "value": v, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(desc, g, st, batched, args.gpus),
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": rows[0]["cores"], "kind": "oracle",
                             "sample": f"each step: uniformly random nodes sized for {per_step:.1f} s by a calibration run, "
                                       f"among those with at most {rows[0]['cap']:.3g} credited clusters (seeds "
                                       f"0..{args.steps - 1}; {args.warmup} warm-up samples of seeds 1000.., 0.5 s each), "
                                       f"{sum(r['nodes'] for r in rows)} nodes and {clusters:.3g} clusters in "
                                       f"all, {t:.1f} s measured"},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _time_events(fn, stream, dev, reps: int, warm: int = 3) -> float:
    """Mean ms per call of fn over `reps` calls (CUDA events on `stream`) after `warm` untimed calls."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps


def workloads_leg(args, dev, hbm: float) -> dict:
    """Every workload besides the headline one, one ef_compute_ex (or
    ef_compute_batched) per step as in the headline (validation on the
    device, one replayed CUDA graph), inputs in HBM, 3 warm-up and 10 timed
    calls (CUDA events): ms per graph, clusters/s, the per-pass breakdown
    (a profiled call) and the path's algorithmic bytes (CSR read once, EF
    written once) against HBM; single graphs add the default options' time
    (validation word read back midway).  The batch adds each graph's own time as a
    call of its own (host wall clock around the synchronous call)."""
    import torch
    import paper_2306_00606_gb300 as ef
    stream = torch.cuda.current_stream(dev)
    ctx = ef.Context(dev.index, stream)
    plan = [("er2000", ("fp32c", "fp64")), ("ba1m", ("fp32c", "fp64")), ("plcm4m", ("fp64",)),
            ("plcm4m_d6", ("fp32c", "fp64")), ("ws4096", ("fp32c", "fp64")), ("ba16m", ("fp32c", "fp64"))]
    res = {}
    for name, precs in plan:
        idx, desc = WORKLOADS[name]
        g = synth.workload(idx)
        gs = graph_stats(g)
        batched = name in BATCHED
        G = len(g.graph_off) - 1 if batched else 1
        rp = torch.from_numpy(g.row_ptr).to(dev)
        ci = torch.from_numpy(g.col_idx).to(dev)
        out = torch.empty(g.n, dtype=torch.float64, device=dev)
        path_bytes = 4 * (g.n + 1) + 4 * g.nnz + 8 * g.n
        entry = {"workload": desc, "nodes": g.n, "nnz": g.nnz, "edges": g.nnz // 2, "clusters": gs["W"],
                 "graphs": G, "max_degree": gs["maxdeg"]}
        for prec in precs:
            # as the headline step: validation on the device, one replayed CUDA graph per call
            if batched:
                def call(profile=False):
                    ef.ef_compute_batched(ctx.handle, rp, ci, g.graph_off, precision=prec, ef=out,
                                          graph=not profile, profile=profile, device_check=True)
            else:
                def call(profile=False):
                    ef.ef_compute_ex(ctx.handle, rp, ci, precision=prec, ef=out, profile=profile,
                                     graph=not profile, device_check=True)
            ms = _time_events(call, stream, dev, reps=10)
            ctx.stats(reset=True)
            call(profile=True)
            pst = ctx.stats(reset=True)
            entry[prec] = {"ms_per_step": ms, "ms_per_graph": ms / G, "clusters_per_s": gs["W"] / (ms / 1e3),
                           "passes_ms": {k: pst[k] for k in PASSES},
                           "roofline_path": {"bound": "hbm", "algorithmic_bytes": path_bytes,
                                             "achieved": path_bytes / (ms / 1e3) / 1e9, "peak": hbm,
                                             "unit": "GB/s", "frac": path_bytes / (ms / 1e3) / 1e9 / hbm}}
        if not batched:
            # the default options instead: the validation word read back midway, the passes
            # launched one by one or part B as a replayed graph
            entry["readback_fp32c"] = {}
            for label, kw in (("ms_per_call", {}), ("ms_per_call_graph", {"graph": True})):
                def dcall(kw=kw):
                    ef.ef_compute_ex(ctx.handle, rp, ci, precision="fp32c", ef=out, **kw)
                entry["readback_fp32c"][label] = _time_events(dcall, stream, dev, reps=10)
        if name in ("er2000", "ba1m"):
            # the oracle beside it, on all host cores and on one (bounded samples)
            entry["oracle"] = {}
            for thr, label in ((0, "all_cores"), (1, "one_core")):
                rows = list(oracle_steps(g, 1, 2.0, seed0=0, threads=thr))
                entry["oracle"][label] = {"clusters_per_s": rows[0]["clusters"] / rows[0]["s"],
                                          "cores": rows[0]["cores"], "nodes": rows[0]["nodes"], "s": rows[0]["s"]}
        if batched:
            # each graph alone: its rows relabelled to 0.., one synchronous call each
            off = g.graph_off
            walls, walls_dc, works = [], [], []
            for k in range(G):
                a, b = int(off[k]), int(off[k + 1])
                e0, e1 = int(g.row_ptr[a]), int(g.row_ptr[b])
                srp = (rp[a:b + 1] - e0).contiguous()
                sci = (ci[e0:e1] - a).contiguous()
                sout = out[a:b]
                if k < 8:
                    for _ in range(2):
                        ef.ef_compute_ex(ctx.handle, srp, sci, precision="fp32c", ef=sout)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                ef.ef_compute_ex(ctx.handle, srp, sci, precision="fp32c", ef=sout)
                walls.append((time.perf_counter() - t0) * 1e3)
                t0 = time.perf_counter()
                ef.ef_compute_ex(ctx.handle, srp, sci, precision="fp32c", ef=sout, device_check=True)
                walls_dc.append((time.perf_counter() - t0) * 1e3)
                d = np.diff(g.row_ptr[a:b + 1]).astype(np.int64)
                works.append(int((d * (d - 1) // 2).sum()))
            w = np.array(walls)
            entry["per_graph_alone_fp32c"] = {
                "calls": G, "ms_p10": float(np.percentile(w, 10)), "ms_p50": float(np.percentile(w, 50)),
                "ms_p90": float(np.percentile(w, 90)), "ms_p99": float(np.percentile(w, 99)),
                "ms_max": float(w.max()), "ms_sum": float(w.sum()),
                "clusters_per_graph_p10_p50_p90": [float(np.percentile(works, q)) for q in (10, 50, 90)],
                "note": "each graph as a separate synchronous ef_compute_ex call (host wall clock, validation "
                        "readback included); the batched call above runs all of them in one pass"}
            w = np.array(walls_dc)
            entry["per_graph_alone_fp32c_device_check"] = {
                "ms_p10": float(np.percentile(w, 10)), "ms_p50": float(np.percentile(w, 50)),
                "ms_p90": float(np.percentile(w, 90)), "ms_p99": float(np.percentile(w, 99)),
                "ms_max": float(w.max()), "ms_sum": float(w.sum()),
                "note": "the same calls with device_check (validation on the device, one readback at the end)"}
        res[name] = entry
        del rp, ci, out
        torch.cuda.empty_cache()
    ctx.close()
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2306_00606_gb300 as ef

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    idx, desc = WORKLOADS[args.workload]
    g = synth.workload(idx, args.scale)
    if args.scale != 1.0:
        desc += f" scaled by {args.scale}"
    st = graph_stats(g)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    n = g.n
    stream = torch.cuda.current_stream(dev)
    ctx = ef.Context(local, stream)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    batched = args.workload in BATCHED
    if args.autotune:
        tuned = ef.ef_autotune(ctx.handle, rp, ci, precision=args.precision, reps=2)

    # Every step validates its graph (on the device, no readback midway) and
    # runs as one replayed CUDA graph; profiled steps run the passes one by
    # one with events between them.
    def step(profile=False, io=None, c=None, async_=False):
        kw = dict(precision=args.precision, profile=profile, device_check=True, graph=not profile)
        if io is None:
            kw.update(ef=out)
            a, b = rp, ci
        else:
            kw.update(ef=io[2], host_io=True, async_=async_)
            a, b = io[0], io[1]
        h = (c or ctx).handle
        if batched:
            ef.ef_compute_batched(h, a, b, g.graph_off, **kw)
        else:
            ef.ef_compute_ex(h, a, b, **kw)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    ctx.stats(reset=True)

    # ---- device-resident timing (inputs in HBM; > L2, no flush) ----
    # The timed steps carry no events inside (batches replay the captured
    # CUDA graph); a second region of as many profiled steps, with the
    # library's events between the passes, gives the per-pass breakdown.
    def timed(profile):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(args.steps):
            step(profile=profile)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1), world, dev)

    with ClockSampler(local) as clk:
        ms = timed(profile=False)
    replays = ctx.stats()["graph_replays"]
    ctx.stats(reset=True)
    timed(profile=True)
    passes = ctx.stats(reset=True)
    ms_step = ms / args.steps
    value = st["W"] * args.steps * world / (ms / 1e3)

    # ---- end to end through the C ABI with host buffers (H2D + compute + D2H) ----
    h2d = 4 * (n + 1) + 4 * g.nnz
    d2h = 8 * n
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(g.row_ptr).pin_memory()
        h_ci = torch.from_numpy(g.col_idx).pin_memory()
        h_out = torch.empty(n, dtype=torch.float64).pin_memory()
        io = (h_rp, h_ci, h_out)
        for _ in range(2):
            step(io=io)
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(io=io)
        torch.cuda.synchronize(dev)
        serial_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        # Two steps in flight: two contexts on two streams, each with its own
        # output buffer, calls returning once their copies and kernels are
        # queued (async_), so one step's host-to-device copy runs beside the
        # previous step's kernels.  Every step still copies its inputs in and
        # its EF out inside the timed region.
        s2 = torch.cuda.Stream(dev)
        ctx2 = ef.Context(local, s2)
        ios = (io, (h_rp, h_ci, torch.empty(n, dtype=torch.float64).pin_memory()))
        ctxs = (ctx, ctx2)
        for i in range(2):
            step(io=ios[i], c=ctxs[i])
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(io=ios[i % 2], c=ctxs[i % 2], async_=True)
        for c in ctxs:
            ef.ef_sync(c.handle)
        torch.cuda.synchronize(dev)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        ctx2.close()
        e2e = {"value": st["W"] * args.steps * world / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s / args.steps, "steps_in_flight": 2,
               "serial": {"value": st["W"] * args.steps * world / serial_s,
                          "ms_per_step": 1e3 * serial_s / args.steps,
                          "note": "one synchronous call at a time: copy in, compute, copy out"}}

    # ---- roofline of the dominant pass ----
    per = {k: passes[k] / max(passes["calls"], 1) for k in PASSES + ("total_ms",)}
    clocks = clk.summary()
    dom = max(PASSES, key=lambda k: per[k])
    alg = algorithmic_bytes(g, st)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm, src = float(peaks["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    except (OSError, KeyError, ValueError):
        hbm, src = 6800.0, "fallback"
    achieved = alg[dom] / (per[dom] / 1e3) / 1e9
    roofline = {"kernel": PASS_KERNEL[dom], "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": committed_traffic(PASS_KERNEL[dom], args.workload),
                "algorithmic_bytes": alg[dom], "launch_ms": per[dom], "peak_source": src,
                "note": "bytes = each input read once and each output written once (bench.py "
                        "algorithmic_bytes); " + PASS_NOTE[dom]}
    # the wedge passes against the MUFU issue bound: one lg2 per f evaluation,
    # 16 special-function results per SM per clock
    evals = st["small_evals"] + class_evals(g)
    wedge_ms = per["wedge_small_ms"] + per["wedge_big_ms"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks.get("sm_max_mhz") or 2070.0
    mufu = sms * 16 * mhz * 1e6
    roofline_alu = {"bound": "alu", "kernels": "wedge passes (k_wedge_small, k_wedge_mid, k_wedge_hub)",
                    "f_evaluations": evals, "achieved": evals / (wedge_ms / 1e3) / 1e9 if wedge_ms > 0 else None,
                    "peak": mufu / 1e9, "unit": "Geval/s",
                    "frac": evals / (wedge_ms / 1e3) / mufu if wedge_ms > 0 else None,
                    "peak_source": f"{sms} SMs x 16 MUFU results per clock x {mhz:.0f} MHz"}
    path_bytes = 4 * (n + 1) + 4 * g.nnz + 8 * n
    roofline_path = {"bound": "hbm", "algorithmic_bytes": path_bytes,
                     "achieved": path_bytes / (ms_step / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": path_bytes / (ms_step / 1e3) / 1e9 / hbm}

    line = {
        "metric": "clusters/s", "value": value, "unit": "clusters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32c" else "f64", "data": "synthetic",
        "config": workload_config(desc, g, st, batched, world),
        "precision": args.precision, "tuning": ef.ef_get_tuning(ctx.handle), "autotuned": bool(args.autotune),
        "ef_wall_ms_per_graph": ms_step / (len(g.graph_off) - 1 if batched else 1),
        "graph_replays_in_timed_region": replays,
        "passes_ms": per,
        "roofline": roofline,
        "roofline_path": roofline_path,
        "roofline_alu": roofline_alu,
        "credits_per_s": 4 * value,
        "passes_gbs": {k: alg[k] / (per[k] / 1e3) / 1e9 if per[k] > 0 else None for k in PASSES},
        "passes_ncu": passes_ncu(args.workload),
        "e2e": e2e,
        "gpu_launches": int(passes["kernels"]),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, args.cpu_seconds)
    if rank == 0 and world == 1 and not batched and not args.no_shards:
        line["shards"] = shard_leg(ctx, rp, ci, args, dev, ms_step)
    if rank == 0 and args.sir:
        line["sir"] = sir_leg(args, dev)
    if rank == 0 and args.rmat_sweep:
        line["rmat_sweep"] = rmat_sweep(ctx, args, dev)
    extra = rank == 0 and world == 1 and args.scale == 1.0 and args.workload == "plcm4m"
    if extra and not (args.no_workloads and args.no_surrogate):
        del rp, ci, out
        ctx.close()
        torch.cuda.empty_cache()
        if not args.no_workloads:
            try:
                line["workloads"] = workloads_leg(args, dev, hbm)
            except Exception as e:   # reported, the main line stands
                line["workloads"] = {"error": f"{type(e).__name__}: {e}"}
        if not args.no_surrogate:
            try:
                line["surrogate"] = surrogate_leg(args, dev)
            except Exception as e:   # reported, the main line stands
                line["surrogate"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.sir_batch:
        return sir_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
