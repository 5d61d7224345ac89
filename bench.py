#!/usr/bin/env python
"""Benchmark: FMM evaluations/s (build + evaluate) and P2P Gpair/s at N = 1,048,576.

Workload (the plain FP32 FMM on the GPU): N = 1,048,576 particles uniform in
[0,1)^3 (FP64), charges uniform in [-1,1), Laplace potential + gradient,
ncrit = 64, at P = 8, theta = 0.5: of the configurations P in {3,4,6,8} x
theta in {0.3,0.4,0.5}, the fastest one whose relative L2 error against the
direct sum is below 1e-4 for both potential and gradient (about 1.2e-5 here).  One step = fmm_build (keys, sort, tree,
dual tree traversal, list grouping) + fmm_evaluate (P2M, M2M, M2L, L2L,
P2P + L2P + scatter) with inputs resident in HBM; L2 is flushed (256 MiB
write) before every timed step, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--dist uniform|plummer] [--kahan] [--N ..] [--P ..] [--theta ..] [--ncrit ..]

--dist plummer --kahan --N 4194304 --P 4 --theta 0.4 times the adaptive workload
(Plummer sphere, charges 1/N, compensated P2P accumulation) the same way.

Multi-GPU: the path does not shard (one FMM per GPU), so N GPUs run N
independent replicas; value = all evaluations / max-over-ranks time.
--impl reference times the CPU oracle (FP64 C) on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from math import comb

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM evals/s & P2P Gpair/s at N=1M, rel err 1e-4, vs plain FP32 path"
FLOPS_PER_PAIR = 20          # the paper's count for a potential + force interaction (Table 4)
FP32_LANES_PER_SM = 128
P2P_FP32_OPS_PER_PAIR = 13   # 3 sub, 3 FMA (r^2), 3 mul, 1 add, 3 FMA: the P2P kernel's FP32 work per pair
P2P_MUTUAL_FP32_OPS_PER_PAIR = 9   # mutual: 18 per pair term, which serves both directions (two interactions)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=1048576)
    ap.add_argument("--P", type=int, default=8)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--ncrit", type=int, default=64)
    ap.add_argument("--dist", default="uniform", choices=["uniform", "plummer"])
    ap.add_argument("--kahan", action="store_true", help="compensated P2P accumulation")
    ap.add_argument("--one-sided", action="store_true",
                    help="one-sided near field (every listed leaf pair evaluated for its target only); the default "
                         "is the mutual near field: each unordered leaf pair once, both directions")
    ap.add_argument("--hybrid", type=int, default=None,
                    help="M2L / P2P hybrid at the leaves: MAC-passing leaf pairs with at least this many "
                         "particle pairs go to M2L (default: Algorithm 4 as printed)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variants", default="all",
                    choices=["all", "none", "adaptive", "differentiated", "batched", "systems", "ncrit",
                             "hybrid", "mutual"],
                    help="variant workloads timed after the main line (adaptive: Plummer N=4M with and "
                         "without compensated P2P; differentiated: N=262144 forward + fmm_backward)")
    ap.add_argument("--variants-only", action="store_true", help="time only the variants (no main line)")
    ap.add_argument("--peaks-only", action="store_true", help="measure the FP32 / SFU peaks only and print them")
    ap.add_argument("--batch-n", type=int, default=1048576, help="N of the batched variant (a smaller case for ncu)")
    return ap.parse_args()


def workload(a):
    from paper_1209_3516_gb300 import inputs
    if a.dist == "plummer":
        return inputs.plummer(a.N, inputs.SEED_BASE + 2)
    return inputs.uniform_cube(a.N, inputs.SEED_BASE + 1)


def config(a):
    what = ("uniform cube" if a.dist == "uniform" else
            "Plummer sphere (a=1, r<=100, charges 1/N)")
    return {"workload": "%s N=%d, P=%d, theta=%.2f, ncrit=%d, potential+gradient, one charge vector%s"
                        % (what, a.N, a.P, a.theta, a.ncrit, ", compensated P2P" if a.kahan else ""),
            "N": a.N, "P": a.P, "theta": a.theta, "ncrit": a.ncrit, "dist": a.dist, "kahan": a.kahan,
            "hybrid_min_pairs": a.hybrid,
            "traversal": "Algorithm 4 as printed" if a.hybrid is None else "M2L / P2P hybrid at the leaves",
            "near_field": "one-sided" if a.one_sided else "mutual (each unordered leaf pair once, both directions)",
            "step": "fmm_build + fmm_evaluate",
            "l2": "flushed before every timed step (256 MiB write)"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def error_sample(N):
    """The 4,096-target error sample: every (N // 4096)-th target of the original order."""
    step = max(1, N // 4096)
    return np.arange(0, N, step, dtype=np.int64)[:4096]


def time_oracle(a, x, q, reps=1):
    """Seconds of the FP64 oracle FMM (build + evaluate) on the whole workload, per repetition."""
    import oracle
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        f = oracle.FMM(x.shape[0], a.P, a.theta, a.ncrit).build(x)
        f.evaluate(q)
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_baseline(a, x, q, reps=3):
    """The oracle on the host cores at the full workload (no sampling or scaling):
    the FP64 FMM, median of `reps` build + evaluate runs, and the FP64 direct sum
    on the 4,096-target error sample."""
    import oracle
    q64 = q.astype(np.float32).astype(np.float64)
    ts = time_oracle(a, x, q64, reps)
    tgt = error_sample(a.N)
    t0 = time.perf_counter()
    ref = oracle.direct(x, q64, targets=tgt)
    t_direct = time.perf_counter() - t0
    cpu_baseline.last_direct = (tgt, ref)
    return {"value": 1.0 / statistics.median(ts), "unit": "evals/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": "the whole workload (N=%d): FP64 oracle FMM, build + evaluate, same P/theta/ncrit, "
                      "median of %d runs" % (a.N, reps),
            "seconds_per_eval": statistics.median(ts), "seconds_all": ts,
            "direct_sum_sample": {"targets": int(tgt.shape[0]), "sources": a.N, "seconds": t_direct,
                                  "pairs_per_s": tgt.shape[0] * a.N / t_direct,
                                  "what": "FP64 direct sum (potential + gradient) on the 4,096-target "
                                          "error sample against all N sources"}}


def p2p_traffic(a):
    """DRAM bytes per P2P launch from the committed ncu capture, if it was taken on
    this workload with the current kernel sources (else None)."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_p2p_traffic.json")
    try:
        pj = json.load(open(prof))
        if (pj.get("N"), pj.get("P"), pj.get("theta"), pj.get("ncrit")) != (a.N, a.P, a.theta, a.ncrit):
            return None
        if (pj.get("dist", "uniform"), pj.get("kahan", False), pj.get("hybrid")) != (a.dist, a.kahan, a.hybrid):
            return None
        if pj.get("mutual", False) != (not a.one_sided):
            return None
        h = hashlib.sha256()
        for f in pj["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        return pj["dram_bytes_per_launch"] if h.hexdigest() == pj["sources_sha256"] else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) == len(self.FIELDS):
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_id_for_smi(dev):
    import torch
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis and "," not in vis:
            return vis
        return dev


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_setup(a):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if a.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def job_value(ws, steps, total_ms_max):
    """Whole-job throughput: every rank ran `steps` steps; the slowest rank's
    time (max over ranks, ms) is the job's time."""
    return ws * steps / (total_ms_max / 1e3)


def max_over_ranks(pg, v):
    if pg is None:
        return v
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def run_reference(a):
    """The reference arm: the CPU oracle (FP64 C, OpenMP, all host cores), each
    step one build + evaluate of the FP64 FMM on the whole workload."""
    # under torchrun only rank 0 times the oracle; the other ranks exit without work
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import oracle
    x, q = workload(a)
    q64 = q.astype(np.float32).astype(np.float64)
    time_oracle(a, x, q64, reps=max(0, a.warmup))
    t0 = time.perf_counter()
    ts = time_oracle(a, x, q64, reps=a.steps)
    wall = time.perf_counter() - t0
    per_eval = sum(ts) / len(ts)
    value = 1.0 / per_eval
    sample = ("each step: the whole workload (N=%d), FP64 oracle FMM, build + evaluate, same P/theta/ncrit"
              % a.N)
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "evals/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(a),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return 0


def time_steps(torch, stream, fn, steps, warmup, flush):
    """Mean device time (ms) of fn over `steps` calls, L2 flushed before each."""
    for _ in range(warmup):
        flush.fill_(1)
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return statistics.mean(s.elapsed_time(e) for s, e in ev)


def run_variants(torch, stream, flush, which="all", batch_n=1048576):
    """The adaptive and the differentiated workloads, each against the plain FP32
    path on the same GPU (same inputs, same step, only the variant switched)."""
    from paper_1209_3516_gb300 import fmm, inputs
    out = {}
    if which in ("all", "adaptive"):
        out.update(variant_adaptive(torch, stream, flush))
    if which in ("all", "differentiated"):
        out.update(variant_differentiated(torch, stream, flush))
    if which in ("all", "batched"):
        out.update(variant_batched(torch, stream, flush, batch_n))
    if which in ("all", "systems"):
        out.update(variant_systems(torch, stream, flush))
    if which in ("all", "ncrit"):
        out.update(variant_ncrit(torch))
    if which in ("all", "hybrid"):
        out.update(variant_hybrid(torch, stream, flush))
    if which in ("all", "mutual"):
        out.update(variant_mutual(torch, stream, flush))
    return out


def variant_mutual(torch, stream, flush):
    """The mutual near field (FMM_FLAG_MUTUAL: each unordered leaf pair once, both
    directions) against the one-sided P2P on the N = 1M uniform workload (P = 8,
    theta = 0.5, ncrit = 64), build + evaluate, timed like the main line."""
    from paper_1209_3516_gb300 import fmm, inputs
    N, P, theta, ncrit = 1048576, 8, 0.5, 64
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    phi = torch.empty(N, dtype=torch.float32, device="cuda")
    grad = torch.empty(N, 3, dtype=torch.float32, device="cuda")
    out = {}
    for name, mu in (("one_sided", False), ("mutual", True)):
        h = fmm.FMM(N, P, theta, ncrit, mutual=mu, timing=True)

        def step():
            h.build(xd)
            h.evaluate(qd, phi=phi, grad=grad)
        t = time_steps(torch, stream, step, 20, 3, flush)
        st = h.stats()
        out[name] = {"evals_per_s": 1e3 / t, "ms": t, "p2p_ms": st["ms_phase"]["p2p"],
                     "lists_ms": st["ms_phase"]["lists"], "p2p_pairs": st["p2p_pairs"]}
        h.close()
    return {"mutual_1m": {
        "workload": "uniform cube N=1048576, P=8, theta=0.5, ncrit=64, build + evaluate, L2 flushed: one-sided "
                    "P2P vs the mutual near field (each unordered leaf pair once, both directions)",
        "one_sided": out["one_sided"], "mutual": out["mutual"],
        "mutual_vs_one_sided": out["one_sided"]["ms"] / out["mutual"]["ms"],
        "p2p_phase_ratio": out["one_sided"]["p2p_ms"] / out["mutual"]["p2p_ms"]}}


def variant_hybrid(torch, stream, flush):
    """The M2L / P2P hybrid at the leaves on the N = 1M uniform workload (P = 8,
    theta = 0.5, ncrit = 64): fmm_tune_hybrid over the M2L threshold (-1 is
    Algorithm 4 as printed), then the chosen setting timed like the main line."""
    from paper_1209_3516_gb300 import fmm, inputs
    N, P, theta, ncrit = 1048576, 8, 0.5, 64
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    best, ms = fmm.tune_hybrid(xd, qd, P, theta, ncrit, candidates=(-1, 0, 256, 512, 1024, 2048), reps=3)
    phi = torch.empty(N, dtype=torch.float32, device="cuda")
    grad = torch.empty(N, 3, dtype=torch.float32, device="cuda")
    out = {}
    for name, hyb in (("algorithm_4", None), ("hybrid", best)):
        h = fmm.FMM(N, P, theta, ncrit, hybrid=hyb, timing=True, mutual=True)

        def step():
            h.build(xd)
            h.evaluate(qd, phi=phi, grad=grad)
        t = time_steps(torch, stream, step, 20, 3, flush)
        st = h.stats()
        out[name] = {"evals_per_s": 1e3 / t, "ms": t, "n_m2l": st["n_m2l"], "n_p2p": st["n_p2p"],
                     "p2p_pairs": st["p2p_pairs"], "phases_ms": st["ms_phase"]}
        h.close()
    return {"hybrid_1m": {
        "workload": "uniform cube N=1048576, P=8, theta=0.5, ncrit=64, build + evaluate, L2 flushed, mutual "
                    "near field: Algorithm 4 as printed vs the M2L / P2P hybrid at the leaves (threshold tuned "
                    "with the one-sided near field)",
        "tuned_min_pairs": best, "tune_ms": {str(k): v for k, v in ms.items()},
        "algorithm_4": out["algorithm_4"], "hybrid": out["hybrid"],
        "hybrid_vs_algorithm_4": out["algorithm_4"]["ms"] / out["hybrid"]["ms"]}}


def variant_ncrit(torch):
    """The leaf-size autotuner (fmm_tune_ncrit) on the N = 1M uniform workload,
    P = 8, theta = 0.5: build + evaluate time for each candidate ncrit."""
    from paper_1209_3516_gb300 import fmm, inputs
    N = 1048576
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    best, ms = fmm.tune_ncrit(torch.from_numpy(x).cuda(), torch.from_numpy(q.astype(np.float32)).cuda(), 8, 0.5,
                              candidates=(24, 32, 48, 64, 96, 128), reps=3)
    return {"ncrit_autotune_1m": {
        "workload": "uniform cube N=1048576, P=8, theta=0.5: fmm_tune_ncrit over ncrit candidates "
                    "(median of 3 build + evaluate each)",
        "ms_by_ncrit": {str(k): v for k, v in ms.items()}, "best_ncrit": best,
        "best_vs_ncrit64": ms[64] / ms[best]}}


def variant_systems(torch, stream, flush):
    """64 systems, N lognormal in [1000, 200000] (uniform cube, charges U[-1,1)),
    P = 8, theta = 0.5: the merged evaluation replayed from one CUDA graph against
    64 plain fmm_evaluate calls on per-system handles (trees built once)."""
    from paper_1209_3516_gb300 import fmm, inputs
    P, theta, ncrit = 8, 0.5, 64
    sizes = [int(n) for n in inputs.lognormal_sizes(64)]
    xs, qs = [], []
    for k, n in enumerate(sizes):
        x, q = inputs.uniform_cube(n, inputs.SEED_BASE + 10 + k)
        xs.append(x)
        qs.append(q.astype(np.float32))
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    qd = torch.from_numpy(np.concatenate(qs)).cuda()
    Ntot = sum(sizes)
    phi = torch.empty(Ntot, dtype=torch.float32, device="cuda")
    grad = torch.empty(Ntot, 3, dtype=torch.float32, device="cuda")
    m = fmm.MultiFMM(sizes, P, theta, ncrit)
    m.build(xd)
    ms_m = time_steps(torch, stream, lambda: m.evaluate(qd, phi=phi, grad=grad), 20, 3, flush)
    info = m.info()
    m.close()
    mh = fmm.MultiFMM(sizes, P, theta, ncrit, hybrid=256)   # with the M2L / P2P hybrid at the leaves
    mh.build(xd)
    ms_mh = time_steps(torch, stream, lambda: mh.evaluate(qd, phi=phi, grad=grad), 20, 3, flush)
    mh.close()
    hs, offs, off = [], [], 0
    for n in sizes:
        h = fmm.FMM(n, P, theta, ncrit)
        h.build(xd[off:off + n])
        hs.append(h)
        offs.append(off)
        off += n

    def plain():
        for h, o, n in zip(hs, offs, sizes):
            h.evaluate(qd[o:o + n], phi=phi[o:o + n], grad=grad[o:o + n])
    ms_p = time_steps(torch, stream, plain, 5, 2, flush)
    for h in hs:
        h.close()
    return {"systems_64_lognormal": {
        "workload": "64 systems, N ~ lognormal in [1000, 200000] (total %d), uniform cube, charges U[-1,1), "
                    "P=8, theta=0.5, ncrit=64, trees built once; merged evaluation (one launch per operator) "
                    "replayed from a CUDA graph vs 64 plain fmm_evaluate calls" % Ntot,
        "system_sets_per_s": {"plain_fp32_64_calls": 1e3 / ms_p, "merged_graph": 1e3 / ms_m,
                              "merged_graph_hybrid_256": 1e3 / ms_mh},
        "ms": {"plain_fp32_64_calls": ms_p, "merged_graph": ms_m, "merged_graph_hybrid_256": ms_mh},
        "merged_vs_plain": ms_p / ms_m,
        "graph_nodes": info["graph_nodes"], "p2p_targets_per_item": info["p2p_targets_per_item"],
        "autotune_near_field_ms": {"one_sided_16_targets": info["tune_ms"][0],
                                   "one_sided_8_targets": info["tune_ms"][1],
                                   "mutual_2_per_lane_16_targets": info["tune_ms"][2],
                                   "mutual_2_per_lane_8_targets": info["tune_ms"][3],
                                   "mutual_4_per_lane_16_targets": info["tune_ms"][4],
                                   "mutual_4_per_lane_8_targets": info["tune_ms"][5]},
        "autotune_choice": {"targets_per_item": info["p2p_targets_per_item"],
                            "near_field": ["one-sided", "mutual, 2 sources per lane",
                                           "mutual, 4 sources per lane"][info["mutual"]]},
        "p2p_pairs": info["p2p_pairs"]}}


def variant_batched(torch, stream, flush, N=1048576):
    """32 Gaussian charge vectors on the N = 1M uniform geometry (P = 8, theta = 0.5):
    one fmm_evaluate_batch against 32 plain fmm_evaluate calls, tree built once."""
    from paper_1209_3516_gb300 import fmm, inputs
    P, theta, ncrit, nrhs = 8, 0.5, 64, 32
    x, _ = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    Q = torch.from_numpy(inputs.gaussian_charges(N, nrhs, inputs.SEED_BASE + 3).astype(np.float32)).cuda()
    xd = torch.from_numpy(x).cuda()
    phi = torch.empty(nrhs, N, dtype=torch.float32, device="cuda")
    grad = torch.empty(nrhs, N, 3, dtype=torch.float32, device="cuda")
    h = fmm.FMM(N, P, theta, ncrit, timing=True)
    h.build(xd)
    ms_b = time_steps(torch, stream, lambda: h.evaluate_batch(Q, phi=phi, grad=grad), 5, 2, flush)
    st_b = h.stats()
    phases_b = {k: st_b["ms_phase"][k] for k in ("upward", "m2l", "downward", "p2p")}

    def plain():
        for r in range(nrhs):
            h.evaluate(Q[r], phi=phi[r], grad=grad[r])
    ms_p = time_steps(torch, stream, plain, 3, 1, flush)
    pairs = h.stats()["p2p_pairs"]
    h.close()
    return {"batched_1m_32rhs": {
        "workload": "uniform cube N=%d, 32 charge vectors ~ N(0,1), P=8, theta=0.5, ncrit=64, tree built " % N +
                    "once; fmm_evaluate_batch (FP32 far field, P2P on tensor cores: BF16 hi/lo split, 3 MMAs, "
                    "FP32 accumulate) vs 32 x fmm_evaluate (plain FP32)",
        "vector_evals_per_s": {"plain_fp32": nrhs * 1e3 / ms_p, "batched": nrhs * 1e3 / ms_b},
        "ms": {"plain_fp32_32x": ms_p, "batched": ms_b}, "batched_vs_plain": ms_p / ms_b,
        "batched_phases_ms": phases_b,
        "p2p_pair_vectors_per_s_batched": pairs * nrhs / (phases_b["p2p"] * 1e-3),
        "p2p_pair_vectors_per_s_batched_lower_bound": pairs * nrhs / (ms_b * 1e-3)}}


def variant_adaptive(torch, stream, flush):
    from paper_1209_3516_gb300 import fmm, inputs
    out = {}
    # adaptive: N = 4,194,304 Plummer sphere, charges 1/N, P = 4, theta = 0.4, ncrit = 64
    N, P, theta, ncrit = 4194304, 4, 0.4, 64
    x, q = inputs.plummer(N, inputs.SEED_BASE + 2)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    phi = torch.empty(N, dtype=torch.float32, device="cuda")
    grad = torch.empty(N, 3, dtype=torch.float32, device="cuda")
    res = {}
    for kahan in (False, True):
        h = fmm.FMM(N, P, theta, ncrit, kahan=kahan, timing=True)

        def step():
            h.build(xd)
            h.evaluate(qd, phi=phi, grad=grad)
        ms = time_steps(torch, stream, step, 5, 2, flush)
        st = h.stats()
        res[kahan] = (ms, st["ms_phase"]["p2p"], st["p2p_pairs"], st["ncells"], st["nlevels"])
        h.close()
    ms0, p0, pairs, ncells, nlev = res[False]
    ms1, p1, _, _, _ = res[True]
    out["adaptive_plummer_4m"] = {
        "workload": "Plummer sphere N=4194304 (a=1, r<=100, charges 1/N), P=4, theta=0.4, ncrit=64, "
                    "build + evaluate",
        "evals_per_s": {"plain_fp32": 1e3 / ms0, "compensated_p2p": 1e3 / ms1},
        "p2p_gpair_s": {"plain_fp32": pairs / (p0 * 1e-3) / 1e9, "compensated_p2p": pairs / (p1 * 1e-3) / 1e9},
        "compensated_vs_plain": ms0 / ms1, "p2p_pairs": pairs, "ncells": ncells, "nlevels": nlev}
    return out


def variant_differentiated(torch, stream, flush):
    from paper_1209_3516_gb300 import fmm, inputs
    out = {}
    # differentiated: N = 262,144 uniform cube, P = 6, theta = 0.4: forward + fmm_backward
    N, P, theta, ncrit = 262144, 6, 0.4, 64
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 5)
    g = inputs.rng(inputs.SEED_BASE + 6)
    a = torch.from_numpy(g.standard_normal(N).astype(np.float32)).cuda()
    b = torch.from_numpy(g.standard_normal((N, 3)).astype(np.float32)).cuda()
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    phi = torch.empty(N, dtype=torch.float32, device="cuda")
    grad = torch.empty(N, 3, dtype=torch.float32, device="cuda")
    dq = torch.empty(N, dtype=torch.float32, device="cuda")
    dx = torch.empty(N, 3, dtype=torch.float32, device="cuda")
    h = fmm.FMM(N, P, theta, ncrit)
    h.build(xd)
    ms_f = time_steps(torch, stream, lambda: h.evaluate(qd, phi=phi, grad=grad), 20, 3, flush)

    def fwd_bwd():
        h.evaluate(qd, phi=phi, grad=grad)
        h.backward(a, b, dq=dq, dx=dx)
    ms_fb = time_steps(torch, stream, fwd_bwd, 20, 3, flush)
    h.close()
    out["differentiated_262k"] = {
        "workload": "uniform cube N=262144, P=6, theta=0.4, ncrit=64, tree built once; forward = fmm_evaluate, "
                    "backward = fmm_backward(dphi, dgrad ~ N(0,1)) -> dq, dx",
        "evals_per_s": {"forward": 1e3 / ms_f, "forward_plus_backward": 1e3 / ms_fb},
        "ms": {"forward": ms_f, "backward": ms_fb - ms_f}, "backward_vs_forward": (ms_fb - ms_f) / ms_f}
    return out


def run_ours(a):
    import torch
    from paper_1209_3516_gb300 import fmm

    ws, rank, local, pg = dist_setup(a)
    dev = local if torch.cuda.device_count() > local else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    x, q = workload(a)
    q32 = q.astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q32).cuda()
    phi = torch.empty(a.N, dtype=torch.float32, device="cuda")
    grad = torch.empty(a.N, 3, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    h = fmm.FMM(a.N, a.P, a.theta, a.ncrit, kahan=a.kahan, timing=True, hybrid=a.hybrid, mutual=not a.one_sided)

    def step():
        h.build(xd)
        h.evaluate(qd, phi=phi, grad=grad)

    for _ in range(a.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    launches0 = h.stats()["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    p2p_ms, m2l_ms, phase_acc = [], [], {}
    sampler = ClockSampler(gpu_id_for_smi(dev))
    barrier(pg)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    for k in range(a.steps):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        st = h.stats()
        p2p_ms.append(st["ms_phase"]["p2p"])
        m2l_ms.append(st["ms_phase"]["m2l"])
        for kk, vv in st["ms_phase"].items():
            phase_acc.setdefault(kk, []).append(vv)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms = sum(step_ms)
    st = h.stats()
    launches = st["kernel_launches"] - launches0
    total_ms_max = max_over_ranks(pg, total_ms)
    value = job_value(ws, a.steps, total_ms_max)

    # P2P kernel: algorithmic work per launch = particle pairs of the P2P list
    pairs = st["p2p_pairs"]
    p2p_mean = statistics.mean(p2p_ms)
    gpair_s = pairs / (p2p_mean * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    nominal_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = pairs * FLOPS_PER_PAIR / (p2p_mean * 1e-3) / 1e12
    traffic = p2p_traffic(a)
    # the FP32 FMA and SFU rates of this GPU, measured now (fmm_measure_peaks)
    # with the clocks sampled while they run
    pk_sampler = ClockSampler(gpu_id_for_smi(dev))
    pk_sampler.start()
    time.sleep(0.2)
    peaks = fmm.measure_peaks(stream)
    pk_clocks = pk_sampler.stop()
    peak_tflops = max(peaks["ffma_tflops"], peaks["ffma2_tflops"])
    pair_rate = pairs / (p2p_mean * 1e-3)
    # FP32 operations and SFU rsqrts per interaction of the near field as run
    ops_per_pair = P2P_FP32_OPS_PER_PAIR if a.one_sided else P2P_MUTUAL_FP32_OPS_PER_PAIR
    rsq_per_pair = 1.0 if a.one_sided else 0.5
    # M2L: the truncated contraction's flops per cell pair as the paper writes it
    # (2 C(P+5, 6)), and the multiply-adds the harmonic form executes instead
    # (sum over folded multipole degrees e of (2e + 1) (P - e)^2)
    m2l_mean = statistics.mean(m2l_ms)
    m2l_flops = 2 * comb(a.P + 5, 6) * st["n_m2l"]
    m2l_fma_harmonic = sum((2 * e + 1) * (a.P - e) ** 2 for e in range(a.P))
    m2l_exec_flops = 2 * m2l_fma_harmonic * st["n_m2l"]

    # fmm_evaluate alone on the built tree (the paper's
    # "FMM evals/s": tree construction excluded); reported beside the build +
    # evaluate step of `value`
    ms_eval_only = time_steps(torch, stream, lambda: h.evaluate(qd, phi=phi, grad=grad), 20, 3, flush)

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if a.e2e_steps > 0:
        xh = torch.from_numpy(x).pin_memory()
        qh = torch.from_numpy(q32).pin_memory()
        ph = torch.empty(a.N, dtype=torch.float32).pin_memory()
        gh = torch.empty(a.N, 3, dtype=torch.float32).pin_memory()
        xn, qn, pn, gn = xh.numpy(), qh.numpy(), ph.numpy(), gh.numpy()
        h.evaluate_host(xn, qn, pn, gn)
        e2e_ms = []
        for _ in range(a.e2e_steps):
            flush.fill_(3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.evaluate_host(xn, qn, pn, gn)
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_max = max_over_ranks(pg, sum(e2e_ms))
        e2e = {"value": job_value(ws, a.e2e_steps, e2e_max), "unit": "evals/s",
               "h2d_bytes_per_step": x.nbytes + q32.nbytes, "d2h_bytes_per_step": 4 * a.N * 4}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms_max / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(a),
                "p2p_gpair_s": gpair_s,
                "roofline": {"kernel": "k_p2p" if a.one_sided else "k_p2p_mutual + k_p2p (one-sided entries)",
                             "bound": "alu", "achieved": achieved, "peak": peak_tflops,
                             "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                             "flops_per_pair": FLOPS_PER_PAIR, "pairs_per_launch": pairs,
                             "launch_ms": p2p_mean,
                             "peak_basis": "measured on this GPU in this run: fmm_measure_peaks (register-only "
                                           "FFMA / FFMA2 chains over every SM, fastest of 5 launches, CUDA "
                                           "events), FP32 FMA peak = the faster of the two; nominal %d SMs x 128 "
                                           "lanes x 2 x %.0f MHz = %.1f TFLOP/s" % (sms, sm_max, nominal_tflops),
                             "measured_peaks": dict(peaks, clocks=pk_clocks),
                             "fp32_pipe_frac": pair_rate * ops_per_pair / (peak_tflops * 1e12 / 2),
                             "sfu_frac": pair_rate * rsq_per_pair / peaks["rsqrt_per_s"],
                             "pipe_note": "pairs = target-source particle pairs of the P2P list (each interaction "
                                          "once); fp32_pipe_frac: %d FP32 operations per interaction against the "
                                          "measured FMA operation rate (one-sided: 3 sub, 3 FMA for r^2, 3 mul, 1 "
                                          "add, 3 FMA = 13; mutual: 18 per pair term serving two interactions); "
                                          "sfu_frac: %.1f rsqrt per interaction against the measured SFU rate"
                                          % (ops_per_pair, rsq_per_pair)},
                "m2l_roofline": {"kernel": "k_m2l", "bound": "alu", "unit": "TFLOP/s",
                                 "achieved": m2l_flops / (m2l_mean * 1e-3) / 1e12, "peak": peak_tflops,
                                 "frac": m2l_flops / (m2l_mean * 1e-3) / 1e12 / peak_tflops,
                                 "flops_per_pair": 2 * comb(a.P + 5, 6), "pairs_per_launch": st["n_m2l"],
                                 "launch_ms": m2l_mean,
                                 "executed_flops_per_pair": 2 * m2l_fma_harmonic,
                                 "executed_achieved": m2l_exec_flops / (m2l_mean * 1e-3) / 1e12,
                                 "executed_frac": m2l_exec_flops / (m2l_mean * 1e-3) / 1e12 / peak_tflops,
                                 "flops_note": "flops_per_pair / achieved / frac: the truncated Cartesian "
                                               "contraction |n|+|k|<=P-1 as the paper defines it (2 C(P+5,6) per "
                                               "cell pair); executed_*: the multiply-adds of the harmonic form the "
                                               "kernel runs (multipole folded onto k_z<=1, outputs n_z<=1 "
                                               "contracted, the rest from the trace identity; same result up to "
                                               "rounding); launch_ms: the fold and the contraction; neither count "
                                               "includes the per-pair derivative recurrence"},
                "evaluate_only": {"evals_per_s": 1e3 / ms_eval_only, "ms": ms_eval_only,
                                  "particles_per_s": a.N * 1e3 / ms_eval_only},
                "phases_ms": {k: statistics.mean(v) for k, v in phase_acc.items()},
                "counts": {"ncells": st["ncells"], "nleaves": st["nleaves"], "nlevels": st["nlevels"],
                           "n_m2l": st["n_m2l"], "n_p2p": st["n_p2p"], "p2p_pairs": pairs},
                "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clocks}
        if not a.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(a, x, q)
            # accuracy of this run's result against the FP64 direct sum on the error sample
            tgt, (pr, gr) = cpu_baseline.last_direct
            h.evaluate(qd, phi=phi, grad=grad)
            torch.cuda.synchronize()
            p_gpu = phi.cpu().numpy().astype(np.float64)[tgt]
            gg = grad.cpu().numpy().astype(np.float64)[tgt]
            line["accuracy"] = {"phi_rel_l2_vs_direct": float(np.linalg.norm(p_gpu - pr) / np.linalg.norm(pr)),
                                "grad_rel_l2_vs_direct": float(np.linalg.norm(gg - gr) / np.linalg.norm(gr)),
                                "sample": "%d targets (every %d-th of the original order), FP64 direct sum over "
                                          "all N sources" % (tgt.shape[0], max(1, a.N // 4096)),
                                "bar": 1e-4}
    h.close()
    if line is not None and a.variants != "none" and ws == 1 and a.dist == "uniform":
        try:
            del xd, qd, phi, grad
            line["variants"] = run_variants(torch, stream, flush, a.variants, a.batch_n)
        except Exception as e:   # a variant never hides the main line
            line["variants"] = {"error": repr(e)[:300]}
    if line is not None:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()
    return 0


def run_peaks():
    """The FP32 FMA / FFMA2 and SFU rsqrt rates of GPU 0 with the clocks sampled meanwhile."""
    import torch
    from paper_1209_3516_gb300 import fmm
    torch.cuda.set_device(0)
    smp = ClockSampler(gpu_id_for_smi(0))
    smp.start()
    time.sleep(0.3)
    pk = fmm.measure_peaks()
    clocks = smp.stop()
    props = torch.cuda.get_device_properties(0)
    print(json.dumps(dict(pk, clocks=clocks, gpu=props.name,
                          how="fmm_measure_peaks: register-only FFMA, FFMA2 and rsqrt.approx chains, one full "
                              "wave on every SM, fastest of 5 launches timed with CUDA events")))
    return 0


def main():
    a = parse()
    if a.peaks_only:
        return run_peaks()
    if a.impl == "reference":
        return run_reference(a)
    if a.variants_only:
        import torch
        torch.cuda.set_device(0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        print(json.dumps({"variants": run_variants(torch, torch.cuda.current_stream(), flush, a.variants,
                                                   a.batch_n)}))
        return 0
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
