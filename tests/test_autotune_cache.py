"""The autotuner's cache file (host logic only; no GPU needed): malformed lines and
out-of-range launch shapes are skipped, valid keys round-trip, a later line for the same
key replaces the earlier one."""
import os

import pytest

from paper_2202_09733_gb300 import _native as N
from paper_2202_09733_gb300 import api


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(N.LIB_PATH):
        pytest.skip("libfrpmg.so not built")
    return N.load()


def test_cache_roundtrip(lib, tmp_path):
    src = tmp_path / "in.txt"
    src.write_text("\n".join([
        "# comment",
        "GB300_test 3 3 0 15 128 64 256 128 64 128 256 128 2",
        "GB300_test 2 4 1 12 64 64 64 64 64 64 64 64 8",
        "GB300_test 2 4 1 12 96 64 64 64 64 64 64 64 4",      # same key: replaces the line above
        "GB300_test 2 2 0 10 100 64 64 64 64 64 64 64 4",     # 100 is not a multiple of 32: skipped
        "GB300_test 2 2 0 10 64 64 64 64 64 64 64 64 3",      # G = 3: skipped
        "truncated 2 2",
    ]) + "\n")
    api.fr_autotune_load(src)
    out = tmp_path / "out.txt"
    api.fr_autotune_save(out)
    lines = [l for l in out.read_text().splitlines() if l.startswith("GB300_test")]
    assert "GB300_test 3 3 0 15 128 64 256 128 64 128 256 128 2" in lines
    assert "GB300_test 2 4 1 12 96 64 64 64 64 64 64 64 4" in lines
    assert len(lines) == 2


def test_cache_missing_file(lib, tmp_path):
    with pytest.raises(N.FrError):
        api.fr_autotune_load(tmp_path / "nope.txt")
