"""The benchmark reads its DRAM traffic and ncu figures from the committed profile summaries only
while their recorded kernel-source hash matches the kernel's source: a changed kernel reports no
traffic rather than a stale one."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KEYS = ("dram_bytes_per_launch", "issue_active_pct", "threads_per_inst", "l2_hit_pct", "l2_to_sm_gbs",
        "global_load_bytes_per_sector")


def _summary(tmp_path, kernel, workload, digest, **figures):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    body = "\n".join(f"{k}: {v}" for k, v in figures.items())
    (d / f"{kernel}_{workload}.md").write_text(f"# {kernel}\n\nkernel_source_sha256_16: {digest}\n{body}\n")


def test_figures_read_when_the_hash_matches(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "00ff00ff00ff00ff")
    figs = {"dram_bytes_per_launch": 305066312, "issue_active_pct": 74.8, "threads_per_inst": 26.9,
            "l2_hit_pct": 97.6, "l2_to_sm_gbs": 2390, "global_load_bytes_per_sector": 12.72}
    _summary(tmp_path, "node_kernel", "large", "00ff00ff00ff00ff", **figs)
    got = bench.profiled("node_kernel", "large")
    assert got == {k: float(v) for k, v in figs.items()}


def test_no_figures_for_another_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda k: "1111111111111111")
    _summary(tmp_path, "node_kernel", "large", "00ff00ff00ff00ff", dram_bytes_per_launch=1)
    assert bench.profiled("node_kernel", "large") is None
    assert bench.profiled("cast_kernel", "large") is None  # no summary at all


def test_source_hash_covers_the_kernel_files():
    src = os.path.join(ROOT, "paper_2609_40297_gb300", "csrc")
    h = bench.kernel_source_hash("node_kernel")
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    # the hash covers every file the node kernel is built from
    for f in bench.KERNEL_SOURCES["node_kernel"]:
        assert os.path.exists(os.path.join(src, f))


def test_committed_figures_parse():
    d = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(d)):
        txt = open(os.path.join(d, name)).read()
        if "kernel_source_sha256_16:" not in txt:
            continue
        # every figure line parses as a number
        for key in KEYS:
            for line in txt.splitlines():
                if line.startswith(key + ":"):
                    float(line.split(":", 1)[1])
