"""bench.py's host-side logic on CPU: the roofline `traffic` figure is taken only from an ncu
summary of the same tiles (capture_config line) captured from the current sweep sources (digest)."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _digest(b):
    h = hashlib.sha256()
    for fn in b.SWEEP_SOURCES:
        h.update(fn.encode())
        with open(os.path.join(ROOT, "paper_2407_13950_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _summary(digest, windows, cb, layout):
    return (f"# k_sweep test summary\n\nKernel sources captured: sources_sha256: {digest} (...)\n\n"
            f"capture_config: windows={windows} col_block={cb} layout={layout}\n\n"
            "traffic_per_launch_bytes: forward=1.5e9 adjoint=2.5e9 (scaled)\n")


def test_traffic_needs_the_same_tiles_and_the_current_sources(tmp_path):
    b = _bench()
    b.PROFILES = str(tmp_path)
    d = _digest(b)
    (tmp_path / "k_sweep_4q_M256_small_full.md").write_text(_summary(d, 256, 9, 1))
    assert b.sweep_traffic("adjoint", 256, 9, 1) == (2.5e9, os.path.relpath(str(tmp_path / "k_sweep_4q_M256_small_full.md"), b.ROOT))
    assert b.sweep_traffic("forward", 256, 9, 1)[0] == 1.5e9
    assert b.sweep_traffic("adjoint", 256, 8, 1) == (None, None)     # other tiles
    assert b.sweep_traffic("adjoint", 64, 9, 1) == (None, None)      # other window count
    assert b.sweep_traffic("adjoint", 256, 9, 2) == (None, None)     # other kernel family
    (tmp_path / "k_sweep_4q_M256_small_full.md").write_text(_summary("0" * 16, 256, 9, 1))
    assert b.sweep_traffic("adjoint", 256, 9, 1) == (None, None)     # stale sources
