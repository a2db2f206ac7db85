"""bench.py reports the ncu traffic and pipe figures only while the kernel
sources hash to the value they were taken with (CPU): the hash must ignore
comments and their layout, and follow any change to the code."""
import os
import shutil

import bench


def _copy(tmp_path):
    for name in bench.KERNEL_SOURCES:
        dst = tmp_path / name
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, name), dst)
    return tmp_path


def _hash_at(monkeypatch, root):
    monkeypatch.setattr(bench, "ROOT", str(root))
    return bench.kernel_sha1()


def test_hash_ignores_comments_and_follows_code(tmp_path, monkeypatch):
    root = _copy(tmp_path)
    h0 = _hash_at(monkeypatch, root)
    src = root / "paper_1612_07717_gb300/csrc/mlmc_kernels.cuh"
    text = src.read_text()
    # more comment lines, a block comment, reflowed blank lines: same code
    src.write_text("// one more line\n// and another\n/* a block\n   comment */\n\n" +
                   text.replace("\n\n", "\n\n\n"))
    assert _hash_at(monkeypatch, root) == h0
    # a one-character code change
    src.write_text(text.replace("kBlock / 32", "kBlock / 16", 1))
    assert _hash_at(monkeypatch, root) != h0

