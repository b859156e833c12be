"""Host logic of the N>1 bench path on CPU: world-size-2 gloo ranks run
independent replicas, the job time is the slowest rank's, and the value
counts every rank's units.  The reference arm does its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 10.0 * (rank + 1)  # rank 1 is the slow replica
    dist.barrier()
    worst = bench.max_over_ranks(dist, my_ms, "cpu")
    rate = bench.whole_job_rate(1000, 5, world, worst)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"worst": worst, "rate": rate}, f)


def test_two_gloo_replicas_take_slowest_time(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["worst"] == 20.0
        # 1000 units x 5 steps x 2 replicas in 20 ms
        assert r["rate"] == pytest.approx(1000 * 5 * 2 / 0.020)


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.whole_job_rate(10, 4, 1, 2.0) == pytest.approx(20000.0)


def test_reference_arm_other_ranks_do_no_work(capsys):
    class A:
        steps, warmup, gpus = 4, 3, 2
    bench.run_reference(A, rank=1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_shape(capsys, monkeypatch):
    class A:
        steps, warmup, gpus = 2, 3, 1
    # the depth-3 instance on two spawned oracle processes keeps this quick
    monkeypatch.setattr(bench, "ORACLE_CYCLE_S", {5: 1e9, 4: 1e9, 3: 0.13})
    monkeypatch.setattr(bench, "host_cores", lambda: 2)
    bench.run_reference(A, rank=0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"] == bench.workload_config(1)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_headline_line_is_compact_and_complete():
    """The line the run ends with stays a few KB (a driver keeps only the
    tail of stdout) and carries the contract's keys."""
    roof = {"bound": "alu", "achieved": 1.0, "peak": 1.259, "unit": "TFLOP/s", "frac": 0.8, "traffic": None,
            "kernel": "k" * 60, "peak_source": "p" * 80, "sweep_ms": 1.0, "algorithmic_flops_per_launch": 1e9,
            "algorithmic_bytes_per_launch": 7e8, "hbm": {"achieved_gbs": 1.0, "peak_gbs": 6700.0, "frac": 0.1,
                                                         "peak_source": "measured"}, "source_sha256_16": "0" * 16}
    e2e = {"value": 1e9, "unit": bench.UNIT, "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1, "what": "w" * 100}
    cpu = {"value": 1e6, "unit": bench.UNIT, "cores": 72, "kind": "oracle", "sample": "s" * 300,
           "single_core": {"value": 1e5, "cores": 1}}
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 100}
    line = bench.headline_line(3.1e9, 20, 5, 80.0, 1, roof, e2e, 400, clk, cpu)
    txt = json.dumps(line, separators=(",", ":"))
    assert len(txt) < 4096
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
              "cpu_baseline"):
        assert k in line
    assert line["ms_per_step"] == 4.0 and "forms" not in line
