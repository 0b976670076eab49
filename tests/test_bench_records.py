"""bench.py's recorded ncu figures: a committed profile summary is used only
while its csrc_digest matches the kernel sources it names, and the figures
it carries are the ones bench.py reports (no GPU needed)."""
import os

import pytest

import bench


def test_committed_records_match_the_sources():
    # the summaries under profiles/ name the sources they were taken on; a
    # kernel edited since then has no record until it is captured again
    if bench.recorded_traffic("k_piece_local") is None:
        pytest.skip("the step-1 traffic record predates the current kernel sources")
    vol = bench.recorded_figures("k_vol_512_bernoulli.md", ("ccl_block.cuh", "ccl_internal.h", "ccl_volume.cu"))
    stats = bench.recorded_figures("k_stats_8192_bernoulli.md", ("ccl_block.cuh", "ccl_internal.h", "ccl_stats.cu"))
    if vol is None or stats is None:
        pytest.skip("a volume or statistics record predates the current kernel sources")
    assert set(vol) == {"dram_bytes_per_voxel_p0.3_conn6", "dram_bytes_per_voxel_p0.5_conn26"}
    assert set(stats) == {"dram_bytes_per_pixel_conn8", "dram_bytes_per_pixel_conn4"}
    # DRAM bytes can sit below the algorithmic 5 B per voxel (labels still in
    # L2 at kernel end) but not below the 1 B/voxel read plus the labels
    # that reach DRAM
    assert all(2.0 < v < 20.0 for v in list(vol.values()) + list(stats.values()))


def test_a_digest_mismatch_drops_the_record(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = open(os.path.join(bench.ROOT, "profiles", "k_vol_512_bernoulli.md")).read()
    (prof / "k_vol_512_bernoulli.md").write_text(src)
    (prof / "stale.md").write_text("dram_bytes_per_voxel_x: 1.5\ncsrc_digest: 0000000000000000\n")
    real_digest = bench.csrc_digest(("ccl_block.cuh", "ccl_internal.h", "ccl_volume.cu"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the sources are read from the real tree
    monkeypatch.setattr(bench, "csrc_digest", lambda sources=None: real_digest)
    assert bench.recorded_figures("stale.md", ("ccl_volume.cu",)) is None
    assert bench.recorded_figures("missing.md", ("ccl_volume.cu",)) is None
    assert bench.recorded_figures("k_vol_512_bernoulli.md", ("ccl_volume.cu",))["dram_bytes_per_voxel_p0.3_conn6"] > 0
