"""The committed profile summaries: every DRAM-traffic record names the
kernel source it was captured on (a hash of the text between the kernel's
begin/end markers) and bench.py reports its traffic only while that source is
unchanged; every summary gives the command that produced it."""
import glob
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_records_match_current_kernels():
    for kind, (path, name) in bench.KERNELS.items():
        rec = os.path.join(ROOT, "profiles", f"traffic_{kind}.txt")
        assert os.path.exists(rec), rec
        vals = dict(line.split(":", 1) for line in open(rec)
                    if ":" in line and not line.startswith("#"))
        assert vals["kernel_source_sha256_16"].strip() == bench.kernel_source_hash(path, name), kind
        assert bench.traffic_per_launch(kind) == float(vals["dram_bytes_per_launch"])


def test_every_summary_states_its_command():
    files = glob.glob(os.path.join(ROOT, "profiles", "*.md")) + \
        glob.glob(os.path.join(ROOT, "profiles", "*.txt"))
    assert files
    for f in files:
        text = open(f).read()
        assert "ommand" in text, f                   # "Command" / "# Command:"
        assert len(text) < 16 * 1024, f              # short summaries, not raw output
