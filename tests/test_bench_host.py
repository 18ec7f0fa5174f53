"""Host-side helpers of bench.py (CPU only): the name of the particle kernel a variant launches, and
the rule that the committed ncu traffic figure is reported only while the kernel sources are the
ones it was measured on."""
import hashlib
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kernel_label_names_the_kernel_each_variant_launches():
    b = _bench()
    assert b.kernel_label(4).startswith("k_particles32 ")
    assert b.kernel_label(7).startswith("k_particles32 ")
    for v in (0, 8, 9, 10, 11, 12):
        assert b.kernel_label(v).startswith("k_particles32x2 ")
    assert "variant default" in b.kernel_label(0) and "variant 11" in b.kernel_label(11)
    for v in (17, 18, 21, 22):
        assert b.kernel_label(v).startswith("k_particles32x2 ") and "then variant" in b.kernel_label(v)


def test_traffic_reported_only_for_the_measured_sources(tmp_path):
    b = _bench()
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    rec = {"workload_flag": "pair", "bytes_per_launch": 321564800.0, "variant": 11,
           "dram_bytes_per_launch": 289021184.0, "sources": ["kernel.cu"],
           "source_sha256": hashlib.sha256(b"// kernel v1\n").hexdigest()}
    summary = tmp_path / "traffic.json"
    summary.write_text(json.dumps(rec))
    b.ROOT, b.TRAFFIC_SUMMARY = str(tmp_path), str(summary)
    assert b.measured_traffic("pair", 321564800.0)[0] == 289021184.0
    assert b.measured_traffic("beam", 321564800.0)[0] is None            # another workload
    assert b.measured_traffic("pair", 1.0)[0] is None                    # another size
    assert b.measured_traffic("pair", 321564800.0, 11)[0] == 289021184.0
    assert b.measured_traffic("pair", 321564800.0, 17)[0] is None        # another variant
    src.write_text("// kernel v2\n")
    t, note = b.measured_traffic("pair", 321564800.0)
    assert t is None and "changed" in note
    summary.write_text("{not json")
    assert b.measured_traffic("pair", 321564800.0)[0] is None


def test_committed_traffic_record_is_well_formed():
    with open(os.path.join(ROOT, "profiles", "k_particles32_pair200k_traffic.json")) as f:
        t = json.load(f)
    assert t["dram_bytes_per_launch"] == t["dram_bytes_read"] + t["dram_bytes_write"]
    assert t["bytes_per_launch"] == 8039120 * 40
    assert "--clock-control none" in t["command"] and all(os.path.exists(os.path.join(ROOT, s)) for s in t["sources"])


def test_launcher_command_runs_one_rank_per_gpu():
    b = _bench()
    cmd = b.launcher_argv(["--gpus", "4", "--steps", "10"], 4, 29555)
    assert cmd[1:3] == ["-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "--master-addr=127.0.0.1" in cmd and "--master-port=29555" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "10"] and cmd[-5].endswith("bench.py")


def test_gpus_2_starts_two_gloo_ranks_end_to_end():
    """bench.py --gpus 2 launched without torchrun starts its two ranks itself; in the dry mode
    (no GPU) they split the 64 batched instances over gloo and rank 0 reports n_gpus = 2, every
    instance counted once and the max over ranks."""
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-ranks"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["n_gpus"] == 2 and line["instances"] == 64 and line["max_over_ranks"] == 2.0
