"""Host logic of bench.py that needs no GPU: the reference arm's JSON line
(plain and under torchrun, where only rank 0 reports) and the multi-rank
reduction of the timing over a world_size-2 gloo process group."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _check_reference_line(line):
    d = json.loads(line)
    assert d["impl"] == "reference"
    assert d["metric"] and d["unit"] == "GCUPS" and d["value"] > 0
    assert d["config"]["m"] == 4096 and d["config"]["n"] == 4096
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    return d


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    _check_reference_line(lines[0])


def test_reference_arm_under_torchrun():
    """Two ranks: rank 0 prints the one line, rank 1 exits 0 without work."""
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert _check_reference_line(lines[0])["n_gpus"] == 2


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Rank r took (r + 1) * 10 ms for its steps: the job's time is the slowest rank's.
        t = bench.max_over_ranks((rank + 1) * 0.010, world)
        q.put((rank, t, bench.aggregate_gcups(world, 4096, 4096, 5, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in got:
        assert t == pytest.approx(0.020)
        assert v == pytest.approx(2 * 4096 * 4096 * 5 / 0.020 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.aggregate_gcups(1, 10, 10, 2, 1.0) == pytest.approx(2e-7)


def test_bench_sets_work_queues_without_overriding():
    """bench.py raises the context's hardware work queues for the serving
    measurement, unless the caller chose a value."""
    import subprocess
    import sys
    code = "import os, bench; print(os.environ['CUDA_DEVICE_MAX_CONNECTIONS'])"
    env = dict(os.environ)
    env.pop("CUDA_DEVICE_MAX_CONNECTIONS", None)
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "32", out.stderr
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "12"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "12", out.stderr


def test_roofline_arithmetic():
    """achieved = algorithmic bytes (or ops) per launch / mean launch time,
    frac = achieved / peak, for the kernel with the largest device time; the
    merge's DRAM traffic and DPX pipe figures come from the committed ncu
    summary while merge.cu matches its recorded hash."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"hbm_gbs": 6697.2}
    int_peak = {"derived_gops": 40276.0, "measured_gops": 39000.0}
    prof = {"merge_tile": {"launches": 200, "ms": 20.0, "bytes": 200 * 193.0e6, "ops": 0.0},
            "strip": {"launches": 50, "ms": 9.0, "bytes": 0.0, "ops": 50 * 3.0e12 * 1e-3}}
    r = bench.roofline(prof, peaks, "measured", int_peak)
    assert r["kernel"] == "merge_tile" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["ms_per_launch"] == pytest.approx(0.1)
    assert r["achieved"] == pytest.approx(193.0e6 / 0.1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6697.2)
    assert r["share_of_device_time"] == pytest.approx(20.0 / 29.0)
    assert r["traffic"] == bench.recorded_traffic("paper_2309_09072_gb300/csrc/merge.cu",
                                                  "merge_tile_dpx_pair4096.md")
    # Recorded counters count only while merge.cu matches the summary's hash.
    alu = bench.recorded_counter("paper_2309_09072_gb300/csrc/merge.cu", "merge_tile_dpx_pair4096.md",
                                 "alu_pipe_pct_of_peak_active")
    assert ("measured_bound" in r) == (alu is not None)
    # A strip-dominated profile is counted against the derived INT32 peak.
    prof["strip"]["ms"] = 40.0
    r = bench.roofline(prof, peaks, "measured", int_peak)
    assert r["kernel"] == "strip" and r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(3.0e9 / 0.8e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 40276.0)
    assert bench.roofline({}, peaks, "measured", int_peak) is None


def test_clock_sampler_summary(monkeypatch):
    """Median SM clock under load, the maximum, and every throttle reason seen
    Active during the timed region (a fake nvidia-smi process)."""
    sys.path.insert(0, ROOT)
    import bench
    rows = ("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
            "0, 1980, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active\n"
            "0, 2070, 2070, 1300.2, 0x8, Active, Not Active, Not Active, Not Active\n"
            "garbage line\n")

    class FakeProc:
        def terminate(self):
            pass

        def kill(self):
            pass

        def communicate(self, timeout=None):
            return rows, None

    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: FakeProc())
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]

    def no_smi(*a, **k):
        raise OSError("nvidia-smi not found")

    monkeypatch.setattr(bench.subprocess, "Popen", no_smi)
    assert bench.ClockSampler(0).stop() is None
