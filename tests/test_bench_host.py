"""bench.py's host-side logic, on CPU: the byte model, the DRAM-traffic
lookup, and the reference arm's JSON line (the FP64 oracle on host cores)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_two_pass_bytes_model():
    nbytes, N, M = bench.two_pass_bytes(512, 512, 512)
    assert N == 512 ** 3 and M == 512 * 512 * 257
    assert nbytes == 2 * (4 * N + 24 * M) == 4307550208


def test_traffic_lookup_keys_on_pass_shape_and_sources():
    src = bench.kernel_source_hash()
    lines = [ln for ln in open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) if ln.startswith("pass=")]
    assert lines, "the traffic table must list the captured passes"
    kv = dict(tok.split("=", 1) for tok in lines[0].split() if "=" in tok)
    got = bench.traffic_from_profile(kv["pass"], kv["shape"])
    if kv["src"] == src:
        assert got == float(kv["bytes_per_launch"])
    else:
        assert got is None  # sources changed since the capture: no traffic claimed
    assert bench.traffic_from_profile(kv["pass"], "7x7x7") is None


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=e, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--n", "16", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run(["--impl", "reference", "--n", "16", "--steps", "1"], env={"RANK": "1", "WORLD_SIZE": "2",
                                                                          "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_records_that_void_a_measurement():
    """Slowdown reasons, or clocks far below max with no reason (a leftover
    lock), reject the timed region; the power cap alone does not."""
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 10}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(None)
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1800.0, reasons=["sw_power_cap"]))
    assert bench.clocks_rejected(dict(ok, reasons=["hw_slowdown"]))
    assert bench.clocks_rejected(dict(ok, reasons=["sw_thermal_slowdown", "sw_power_cap"]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1200.0))


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduction_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = bench.max_over_ranks([1.0 + rank, 5.0 - rank], "cpu")
        ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
        bad = bench.clocks_rejected(dict(ok, reasons=["hw_slowdown"]) if rank == 0 else ok, world, "cpu")
        clean = bench.clocks_rejected(ok, world, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"times": times, "bad": bad, "clean": clean}, f)
    finally:
        dist.destroy_process_group()


def test_cross_rank_reductions_on_two_gloo_ranks(tmp_path):
    """The N > 1 bench path on CPU ranks: every rank gets the slowest rank's
    times, and a clock record rejected on one rank makes every rank measure
    again (the ranks never disagree on whether to re-run)."""
    import torch
    torch.multiprocessing.spawn(_reduction_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        r = json.load(open(tmp_path / f"rank{rank}.json"))
        assert r["times"] == [2.0, 5.0]
        assert r["bad"] is True and r["clean"] is False
