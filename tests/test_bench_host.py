"""Host-side logic of bench.py: the DRAM traffic a bench line reports comes
from an ncu summary under profiles/ only when that summary was taken from
the kernel source being measured."""
import bench


def _write(tmp_path, lines):
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "k.md").write_text("\n".join(lines) + "\n")
    return tmp_path


def test_traffic_is_read_only_for_the_current_kernel_source(tmp_path, monkeypatch):
    root = _write(tmp_path, [
        "# summary",
        "bench-traffic: kernel=link_kernel workload=config2 kernel_sha=aaaa dram_bytes_per_launch=5.2e7",
        "bench-traffic-warm: kernel=link_kernel workload=config2 kernel_sha=aaaa dram_bytes_per_launch=14370000",
        "bench-traffic: kernel=link_kernel workload=config1 kernel_sha=aaaa dram_bytes_per_launch=6000000",
    ])
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "kernel_sha", lambda: "aaaa")
    assert bench._profile_traffic("link_kernel", "config2") == (5.2e7, "profiles/k.md")
    assert bench._profile_traffic("link_kernel", "config2", "bench-traffic-warm")[0] == 14370000.0
    assert bench._profile_traffic("link_kernel", "config1")[0] == 6000000.0
    assert bench._profile_traffic("node_kernel", "config2") == (None, None)
    # another kernel source: no figure at all
    monkeypatch.setattr(bench, "kernel_sha", lambda: "bbbb")
    assert bench._profile_traffic("link_kernel", "config2") == (None, None)


def test_kernel_sha_follows_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    a = bench.kernel_sha()
    assert len(a) == 16 and a == bench.kernel_sha()
    src.write_text("__global__ void k() { }\n")
    assert bench.kernel_sha() != a


def test_reference_arm_prints_one_contract_line_on_the_host():
    # the reference arm is the oracle on the host cores: it needs no GPU
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "config0", "--steps", "1",
                        "--warmup", "1"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "vehicle-updates/s" and d["unit"] == d["metric"]
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    import json
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
                        "--workload", "config0", "--steps", "1", "--warmup", "1"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
