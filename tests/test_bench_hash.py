"""The bench reports a kernel's DRAM traffic only while the sources it was
measured on are unchanged: the hash ignores comments and blank lines, and
sees every code change."""
import os
import shutil

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1702_02256_gb300", "csrc")


def test_hash_ignores_comments_but_not_code(tmp_path):
    for f in ("spiir_plain.cu", "spiir_api.cu"):
        shutil.copy(os.path.join(CSRC, f), tmp_path / f)
    base = bench._source_hash("spiir_plain.cu", str(tmp_path))
    assert base == bench._source_hash("spiir_plain.cu")
    p = tmp_path / "spiir_plain.cu"
    src = p.read_text()
    p.write_text("// a new comment line\n\n/* and a block\n   comment */\n" +
                 src.replace("\n", "   // trailing\n", 3))
    assert bench._source_hash("spiir_plain.cu", str(tmp_path)) == base
    p.write_text(src.replace("kRowPitch = 33", "kRowPitch = 34", 1))
    assert bench._source_hash("spiir_plain.cu", str(tmp_path)) != base
    p.write_text(src)
    q = tmp_path / "spiir_api.cu"
    q.write_text(q.read_text() + "\nint extra_symbol_for_the_test = 1;\n")
    assert bench._source_hash("spiir_plain.cu", str(tmp_path)) != base
