"""Host-side checks of bench.py: the reference arm's JSON line, the profile
hash gate and the algorithmic byte count. No GPU is needed."""
import hashlib
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]


def test_profile_traffic_is_null_when_the_kernel_source_changed(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "p.txt").write_text(f"kernel_source_sha256_16: {h}\ndram_bytes_per_launch: 1.5e9\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.profile_traffic("p.txt", str(src)) == 1.5e9
    src.write_bytes(b"__global__ void k() { }\n")  # any edit of the source
    assert bench.profile_traffic("p.txt", str(src)) is None
    assert bench.profile_traffic("missing.txt", str(src)) is None


def test_committed_profiles_match_their_kernel_sources():
    """Every committed summary that the bench reads names the hash of the source it was taken on."""
    for name, src in (("sart_resident_realistic_fp32.txt", bench.KERNEL_SRC),
                      ("sart_rows_batch_fp32.txt", bench.KERNEL_SRC),
                      ("sart_compact_batch_fp32.txt", bench.STREAM_SRC),
                      ("sart_ring_batch_fp32.txt", bench.RING_SRC),
                      ("sart_multi_tiny64_fp32.txt", bench.MULTI_SRC),
                      ("sart_multi_tiny64_bf16.txt", bench.MULTI_SRC)):
        assert bench.profile_traffic(name, src, algorithmic_bytes=1.0) is not None, name


def test_algorithmic_bytes_grow_by_24_bytes_per_entry_and_iteration():
    S, Mh, Nh = 1000, 50, 80
    one = bench.algorithmic_bytes_per_launch(S, Mh, Nh, 10)
    two = bench.algorithmic_bytes_per_launch(S + 1, Mh, Nh, 10)
    assert two - one == 24 * 10 + 12  # 11 forward passes and 10 back passes of 12 B per entry
    more = bench.algorithmic_bytes_per_launch(S, Mh, Nh, 11)
    assert more - one == bench.algorithmic_bytes_per_launch(S, Mh, Nh, 1) - bench.algorithmic_bytes_per_launch(
        S, Mh, Nh, 0)
