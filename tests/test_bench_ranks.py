"""The multi-GPU path of bench.py is replicas only: each rank runs its own
realisation (sample = rank) and the job time is the slowest rank's. Tested
here with two gloo ranks on the CPU; the realisations themselves are run by
the oracle, so no GPU is needed."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sample = bench.replica_sample(rank)
        st = O.State.flat(128).run(3, 128, 128, 0.9, 0.1, 1, sample)   # this rank's realisation
        seconds = 1.0 + rank                                          # rank 1 is the slower one
        t = bench.max_over_ranks(seconds, dist, device="cpu")
        value = bench.whole_job_value(world, 2, 3, 128, t)
        q.put((rank, sample, st.packed().tobytes(), t, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas_timed_by_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get() for _ in range(world))
    assert [o[1] for o in out] == [0, 1]                    # sample = rank
    assert out[0][2] != out[1][2]                           # independent realisations
    assert all(o[3] == 2.0 for o in out)                    # max over ranks
    assert all(o[4] == pytest.approx(world * 2 * 3 * 128 * 128 / 2.0) for o in out)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(type("A", (), {"gpus": 2, "steps": 1, "warmup": 3, "L": 65536, "mcs": 2000})())
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_complete_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the CPU oracle and prints exactly one
    JSON line with the keys of the benchmark contract."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(type("A", (), {"gpus": 1, "steps": 1, "warmup": 1, "L": 65536, "mcs": 2000})())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["L"] == 65536
