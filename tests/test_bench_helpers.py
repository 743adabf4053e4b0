"""bench.py's host-side helpers (CPU only): the source hash that keeps a DRAM-traffic capture
valid ignores comments and blank lines but not code; the per-kernel algorithmic bytes are
positive and scale with the parcel count."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    root = tmp_path / "tree"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2311_03908_gb300", "csrc"), root / "paper_2311_03908_gb300" / "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "include"), root / "include")
    return root


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.source_sha256()
    hdr = root / "include" / "dem.h"
    text = hdr.read_text()
    hdr.write_text("/* a new comment */\n\n" + text.replace("Synchronous.", "Synchronous (reworded).", 1))
    assert bench.source_sha256() == h0
    cu = root / "paper_2311_03908_gb300" / "csrc" / "resort.cu"
    code = cu.read_text()
    assert "constexpr int RZ_SMEM_SORT = 4096;" in code
    cu.write_text(code.replace("constexpr int RZ_SMEM_SORT = 4096;", "constexpr int RZ_SMEM_SORT = 2048;"))
    assert bench.source_sha256() != h0


def test_algorithmic_bytes_scale_with_parcels():
    for k in ("k_key", "k_gas_particle", "k_cells", "k_contact_screen", "k_contact_forces", "k_ranges"):
        a = bench.algorithmic_bytes(k, 1_000_000, 1_572_864, 0.04, 5.8, 4, 3, 0.04, 0.04)
        b = bench.algorithmic_bytes(k, 2_000_000, 1_572_864, 0.04, 5.8, 4, 3, 0.04, 0.04)
        assert 0 < a < b, k
