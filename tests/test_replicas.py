"""The multi-GPU form is replicas only: N processes, one independent FMM each.

bench.py's replica plumbing runs here as two gloo ranks on the CPU (no GPU):
rendezvous on 127.0.0.1, a barrier, the max-over-ranks time and the whole-job
value (all ranks' steps over the slowest rank's time); the reference arm under
a launcher does its work on rank 0 only.
"""
import multiprocessing as mp
import os
import socket
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ws_, rank_, _, pg = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    assert pg is not None and pg.get_backend() == "gloo"
    bench.barrier(pg)
    t = bench.max_over_ranks(pg, 10.0 * (rank + 1))   # rank r "took" 10 (r + 1) ms
    out.put((rank_, ws_, t, bench.job_value(ws_, 5, t)))
    bench.barrier(pg)
    pg.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    # every rank sees the slowest rank's time and the same whole-job value
    assert all(r[2] == 20.0 for r in res)
    assert all(abs(r[3] - 2 * 5 / 0.020) < 1e-9 for r in res)


def test_reference_arm_off_rank_zero_does_no_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    a = types.SimpleNamespace(N=10, P=4, theta=0.4, ncrit=64, steps=1, warmup=0, gpus=2, dist="uniform",
                              kahan=False)
    assert bench.run_reference(a) == 0


def test_reference_arm_prints_one_contract_line():
    """The reference arm (the oracle on the host cores) prints the benchmark's
    JSON line: the same metric and workload keys as the GPU arm, impl, a
    cpu_baseline describing the run and an e2e with no device copies."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "16384",
                        "--P", "4", "--theta", "0.4", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "evals/s"
    assert d["config"]["N"] == 16384 and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0
