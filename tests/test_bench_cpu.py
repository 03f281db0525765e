"""CPU tests of bench.py's measurement bookkeeping.

The roofline's `traffic` comes from the committed ncu record of the code
sweep and must be reported only while the kernel sources it was captured
from are unchanged: equal to the record for the committed sources, null for
a copy of the tree where one hashed file differs or the record is missing.
"""
import os
import shutil

import bench

FILES = ("sweep.cu", "sweep_block.cuh", "internal.cuh")


def _record_bytes(root):
    path = os.path.join(root, "profiles", "sweep_kernel_stem512_k128_traffic.txt")
    kv = dict(line.split(":", 1) for line in open(path).read().splitlines() if ":" in line)
    return float(kv["dram_bytes_per_launch"])


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2311_15061_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "sweep_kernel_stem512_k128_traffic.txt"), root / "profiles")
    for f in FILES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2311_15061_gb300", "csrc", f), csrc / f)
    return root


def _sources_hash(root):
    import hashlib
    blob = b"".join(open(os.path.join(root, "paper_2311_15061_gb300", "csrc", f), "rb").read() for f in FILES)
    return hashlib.sha256(blob).hexdigest()


def test_traffic_record_follows_the_committed_sources():
    """The record's bytes while its source hash is the sources' own, else null."""
    path = os.path.join(bench.ROOT, "profiles", "sweep_kernel_stem512_k128_traffic.txt")
    kv = dict(line.split(":", 1) for line in open(path).read().splitlines() if ":" in line)
    same = kv["source_sha256"].strip() == _sources_hash(bench.ROOT)
    assert bench._traffic_record(FILES) == (_record_bytes(bench.ROOT) if same else None)


def test_traffic_record_is_null_once_a_kernel_source_changes(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    rec = root / "profiles" / "sweep_kernel_stem512_k128_traffic.txt"
    lines = [l if not l.startswith("source_sha256:") else "source_sha256: " + _sources_hash(str(root))
             for l in rec.read_text().splitlines()]
    rec.write_text("\n".join(lines) + "\n")   # a record taken from exactly these sources
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_record(FILES) == _record_bytes(str(root))
    for f in FILES:
        path = root / "paper_2311_15061_gb300" / "csrc" / f
        original = path.read_bytes()
        path.write_bytes(original + b"\n// edited\n")
        assert bench._traffic_record(FILES) is None, f
        path.write_bytes(original)
    (root / "profiles" / "sweep_kernel_stem512_k128_traffic.txt").unlink()
    assert bench._traffic_record(FILES) is None
