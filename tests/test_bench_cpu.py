"""The benchmark's reference arm (the oracle on the host cores) keeps the JSON
line contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["metric"] == "term-point evaluations/s" and d["unit"] == "term-points/s"
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["host"]["model"] and d["cpu_baseline"]["host"]["logical_cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["terms"] == 2000 and d["config"]["T"] == 64
    sys.path.insert(0, ROOT)
    import bench
    # the GPU arm names the workload with the same dict (its own run details go under "plan")
    assert d["config"] == bench.workload_config(bench.make_workload("tiny"), "tiny")


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--gpus", "2", "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_output_ring_never_hands_out_a_live_region():
    """The served benchmark's page-locked output ring, driven with random sizes
    and random completions: live regions never overlap and stay inside the ring
    (a wrapped ring filled exactly to its oldest region must read as full)."""
    import random
    sys.path.insert(0, ROOT)
    import bench
    ring = bench.PinnedRing.__new__(bench.PinnedRing)     # no page-locked buffer needed
    ring.cap, ring.regions = 64 * 256, []
    rnd = random.Random(7)

    def wait_oldest():
        ring.regions.pop(0)

    exact_fills = 0
    for step in range(20000):
        size = rnd.choice([256, 512, 768, 1024, 4096, 256 * rnd.randint(1, 64)])
        start = ring.alloc(size, wait_oldest)
        end = start + (size + 255) // 256 * 256
        assert 0 <= start and end <= ring.cap
        for s0, e0, _ in ring.regions:
            assert end <= s0 or start >= e0, (step, start, end, ring.regions)
        if ring.regions and ring.regions[-1][0] < ring.regions[0][0] and end == ring.regions[0][0]:
            exact_fills += 1
        ring.commit(start, size, step)
        while ring.regions and rnd.random() < 0.3:
            wait_oldest()
    assert exact_fills > 0          # the case that must read as full did occur


def test_served_section_child_and_fallback(monkeypatch):
    # The default line measures the served section in a child process with this
    # run's serving options; a failing child falls back to this process.
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--serve-seconds", "6", "--serve-burst", "1500",
                                      "--serve-streams", "2", "--serve-epoch-jobs", "32", "--serve-rate", "900"])
    args = bench.parse()
    argv = bench.served_child_argv(args)
    assert argv[1] == os.path.join(ROOT, "bench.py")
    monkeypatch.setattr(sys, "argv", argv[1:])
    child = bench.parse()
    assert child.config == "served"
    for k in ("batch_count", "serve_seconds", "serve_rate", "serve_burst", "serve_streams", "serve_epoch_jobs"):
        assert getattr(child, k) == getattr(args, k), k

    class Done:
        def __init__(self, rc, out, err=""):
            self.returncode, self.stdout, self.stderr = rc, out, err

    line = {"metric": "served", "served_over_plain": 3.2, "burst": {"requests": 1500}}
    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: Done(0, "note\n" + json.dumps(line) + "\n"))
    got = bench.served_in_child(args)
    assert got["served_over_plain"] == 3.2 and "metric" not in got and got["process"].startswith("child")
    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: Done(1, "", "Traceback\nRuntimeError: boom"))
    monkeypatch.setattr(bench, "run_served", lambda a, pool=None: {"served_over_plain": 2.0})
    got = bench.served_in_child(args)
    assert got["served_over_plain"] == 2.0 and got["process"].startswith("this process") and "boom" in got["process"]
