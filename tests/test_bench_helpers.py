"""Host logic of bench.py (no GPU): the traffic lookup keyed by the kernel source
hash, the oracle's LOS sample, and the workload string."""
import hashlib
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_traffic_is_read_only_while_the_source_hash_matches(tmp_path, monkeypatch):
    b = _bench()
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1810_06250_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("kernel source v1\n")
    sha = hashlib.sha256(b"kernel source v1\n").hexdigest()[:16]
    (tmp_path / "profiles" / "k.md").write_text("sha256[:16] %s\n\n    traffic_bytes_per_launch: 12345\n" % sha)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.measured_traffic("k.cu", "k.md") == 12345
    (csrc / "k.cu").write_text("kernel source v2\n")             # the kernel changed since the capture
    assert b.measured_traffic("k.cu", "k.md") is None
    assert b.measured_traffic("k.cu", "missing.md") is None


def test_committed_profiles_record_hash_and_traffic():
    # every summary bench.py reads traffic from names the source hash it was taken on
    # and the bytes per launch (bench.py reports null once the source has changed)
    import re
    for name in ("gemm_mwa_bf16x3.md", "gemm_lofar_bf16x3.md", "czt_lofar_ul2.md"):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert re.search(r"sha256\[:16\] [0-9a-f]{16}", text), name
        assert re.search(r"traffic_bytes_per_launch: \d+", text), name


def test_oracle_sample_rows_are_whole_blocks_in_range():
    b = _bench()
    from paper_1810_06250_gb300 import inputs
    import dataclasses
    cfg = dataclasses.replace(inputs.CONFIGS["tiny"], nlos=64 * 40)
    rows, Q, U = b.sample_rows(cfg, 640, np.random.default_rng(1))
    assert len(rows) == 640 and Q.shape == (640, cfg.nchan) and U.shape == Q.shape
    starts = rows[::64]
    assert np.all(starts % 64 == 0) and np.all(np.diff(starts) > 0)
    assert np.all(rows.reshape(-1, 64) == starts[:, None] + np.arange(64)[None, :])
    assert rows.max() < cfg.nlos
    # the sample is the seeded generator's rows, regenerated independently
    Q2, U2 = inputs.make_cube(cfg, int(starts[3]), 64)
    np.testing.assert_array_equal(Q[3 * 64:4 * 64], Q2)
    np.testing.assert_array_equal(U[3 * 64:4 * 64], U2)


def test_workload_string_names_the_shape():
    b = _bench()
    from paper_1810_06250_gb300 import inputs
    s = b.workload_name(inputs.CONFIGS["lofar"], 360, "chan")
    assert s.startswith("lofar: 512x512 LOS x 400 channels (360 active)") and "401 phi" in s
    assert "peak map only" in b.workload_name(inputs.CONFIGS["lofar"], 360, "los", peak_only=True)
