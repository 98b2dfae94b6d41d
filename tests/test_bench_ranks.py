"""The multi-rank logic of bench.py on CPU: two gloo ranks on 127.0.0.1.

A run on N GPUs is N independent replicas (the method has no data-path exchange on one
matrix); the job's step time is the slowest rank's, found by an all-reduce MAX, and the
whole-job throughput is N e^{tau H} per that time.  The reference arm prints from rank 0 only;
the other ranks return without work."""
import os
import socket

import pytest

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [250.0, 400.0][rank]                    # per-rank step times, ms
        ms = bench.max_over_ranks(mine, world)
        rate = bench.whole_job_rate(ms, world)
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{ms} {rate}\n")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, rate = map(float, (tmp_path / f"rank{r}.txt").read_text().split())
        assert ms == 400.0                             # the slowest rank decides the job's step
        assert rate == pytest.approx(2 * 1000.0 / 400.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(123.0, 1) == 123.0
    assert bench.whole_job_rate(500.0, 1) == pytest.approx(2.0)


def test_reference_arm_other_ranks_return_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert rc == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """bench.py --impl reference (rank 0) times the CPU oracle on a bounded sample of the
    workload and prints one JSON line with the keys of the contract."""
    import json
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--sample-m", "12"])
    assert rc == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "expm/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "m=12" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "expm/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "lap2d_m1500"
