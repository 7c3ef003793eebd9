"""Launch-shape cache of the tensor-core autotuner: the text format written
and read by the library (host-only calls, no GPU needed)."""
import pytest

import paper_2409_03904_b300 as mrhs
from paper_2409_03904_b300 import MrhsError


def parse(path):
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        n = int(f[0])
        key = tuple(tuple(int(v) for v in f[1 + 6 * i:7 + 6 * i]) for i in range(n))
        rest = f[1 + 6 * n:]
        rows.append((key, tuple(int(v) for v in rest[:3]), float(rest[3])))
    return sorted(rows)


def test_save_load_roundtrip(tmp_path):
    mrhs.autotune_clear()
    src = tmp_path / "a.txt"
    src.write_text("# shapes\n"
                   "1 148 20736 48 81 32 5 2 2 32 7.5\n"
                   "2 148 256 24 9 4 4 148 256 32 81 8 4 8 1 6 0.125\n")
    mrhs.autotune_load(src)
    assert mrhs.autotune_entries() == 2
    out = tmp_path / "b.txt"
    mrhs.autotune_save(out)
    assert parse(out) == parse(src)
    mrhs.autotune_clear()
    assert mrhs.autotune_entries() == 0
    mrhs.autotune_load(out)
    assert mrhs.autotune_entries() == 2
    mrhs.autotune_clear()


@pytest.mark.parametrize("bad", [
    "1 148 20736 48 81 32 5 2 2\n",                 # truncated
    "1 148 20736 48 81 32 5 2 3 32 7.5\n",          # 3 CTAs per SM
    "1 148 20736 48 81 32 5 2 2 1 7.5\n",           # ring depth 1
    "0 2 2 32 1.0\n",                               # empty key
    "x\n",
])
def test_malformed_cache_rejected_whole(tmp_path, bad):
    mrhs.autotune_clear()
    f = tmp_path / "bad.txt"
    f.write_text("1 148 256 24 9 4 4 2 2 32 0.5\n" + bad)
    with pytest.raises(MrhsError):
        mrhs.autotune_load(f)
    assert mrhs.autotune_entries() == 0
    with pytest.raises(MrhsError):
        mrhs.autotune_load(tmp_path / "missing.txt")
