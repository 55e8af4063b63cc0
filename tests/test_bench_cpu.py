"""CPU checks of the bench's roofline arithmetic and traffic bookkeeping (no GPU)."""
import json
import os

import bench


def test_roofline_frac_is_read_on_dram_bytes_with_the_model_beside_it():
    n, nnz, d = 1000, 50_000, 128
    r = bench.roofline_block(n, nnz, d, 2, False, 1e-3, 4e9, 8000.0, "measured", "k")
    assert r["achieved"] == 4e9 / 1e-3 / 1e9 and r["frac"] == r["achieved"] / 8000.0
    mb = 8 * (n + 1) + 4 * nnz + 2 * d * nnz + 2 * d * n
    assert r["model_bytes"] == mb and abs(r["model_frac"] - mb / 1e-3 / 1e9 / 8000.0) < 1e-12
    cb = 8 * (n + 1) + 4 * nnz + 2 * 2 * d * n
    assert r["compulsory_bytes"] == cb
    no_dram = bench.roofline_block(n, nnz, d, 4, True, 1e-3, None, 8000.0, "measured", "k")
    assert no_dram["traffic"] is None and no_dram["frac"] == no_dram["model_frac"]
    assert "model" in no_dram["basis"]


def test_traffic_entries_are_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.source_sha(bench.PROP_SOURCES)
    (prof / "traffic.json").write_text(json.dumps({"entries": {
        "large/bf16": {"source_sha": sha, "dram_bytes": 123},
        "large/f32": {"source_sha": "0" * 16, "dram_bytes": 456}}}))
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # sources are hashed from the real tree
    monkeypatch.setattr(bench, "source_sha", lambda files, _r=real_root: sha)
    assert bench.measured_traffic("large/bf16") == 123
    assert bench.measured_traffic("large/f32") is None  # taken on another kernel build
    assert bench.measured_traffic("mid/bf16") is None
    assert os.path.exists(os.path.join(real_root, "profiles", "traffic.json"))


def test_every_staging_option_has_a_label():
    import paper_2102_02302_gb300 as pkg
    import re
    header = open(os.path.join(bench.ROOT, "include", "cleora.h")).read()
    doc = header[header.index("CLEORA_OPT_STAGING"):header.index("CLEORA_OPT_RING_STAGES")]
    values = {int(v) for v in re.findall(r"(\d) = ", doc)} | {0, 1}
    assert values <= set(bench.STAGING_LABELS)
    assert pkg.cleora.OPTIONS["staging"] == 7
