"""The multi-GPU path is replicas: N ranks run independent chains (seeds per
rank, no data-path collective) and the bench reduces only the timing (max
over ranks).  Checked here on CPU with two gloo ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.0 + 0.5 * rank  # rank 1 is the slower replica
        tmax = bench.max_over_ranks(t, world)
        q.put((rank, tmax, bench.whole_job_value(tmax, 2, world), bench.replica_seeds(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_reduce_only_the_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]          # both ranks see the slowest time
    assert res[0][2] == pytest.approx(1.5 / (2 * 2))  # whole job: 4 trajectories in 1.5 s
    s0, s1 = res[0][3], res[1][3]
    assert all(s0[k] != s1[k] for k in s0)            # independent chains


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus, ref_iters = 1, 0, 2, 10
    assert bench.reference_arm(A()) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line(monkeypatch, capsys):
    """`bench.py --impl reference` on rank 0: one JSON line timing the oracle
    on a bounded sample of the workload, with the contract's keys and the
    same metric, unit and config as the library's arm."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")

    class A:
        steps, warmup, gpus, ref_iters = 1, 0, 1, 1000
    assert bench.reference_arm(A()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench._metric()
    assert line["unit"] == "s/trajectory" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["config"] == bench.workload_config()
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)  # every host core
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
