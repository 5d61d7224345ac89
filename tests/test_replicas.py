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
