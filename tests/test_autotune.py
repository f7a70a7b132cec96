"""Host logic of the autotuner (no GPU): cache keys and files, the candidate set (mirrors the
library's column-pass rule), the library's default slice-group count, and the selection."""
import json

from paper_1710_01758_gb300 import autotune


def test_cache_round_trip_and_atomic_file(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert autotune.load_cache(path) == {}
    k = autotune.cache_key("NVIDIA GB300", 256, 256, 12, 64, 0)
    assert k == "NVIDIA GB300|256x256|nc12|nb64|prec0"
    assert autotune.cache_key("g", 256, 256, 16, 1, 2, nz=128) == "g|256x256x128|nc16|nb1|prec2"
    autotune.save_cache({k: {"groups": 4, "col_tile": 16, "poll_every": 4, "ms": 1.5}}, path)
    assert autotune.load_cache(path)[k]["col_tile"] == 16
    assert [p.name for p in (tmp_path / "sub").iterdir()] == ["tune.json"]  # no temp file left behind
    (tmp_path / "sub" / "tune.json").write_text("{not json")
    assert autotune.load_cache(path) == {}
    (tmp_path / "sub" / "tune.json").write_text(json.dumps([1, 2]))
    assert autotune.load_cache(path) == {}


def test_col_tile_rule():
    # (ny, nx, ct) -> fits: ct | nx, ct ny / 16 <= 1024 threads, 2 ny ct x 8 B <= 160 KB
    table = {(256, 256, 8): True, (256, 256, 16): True, (256, 256, 32): True,
             (512, 512, 16): True, (512, 512, 32): False, (512, 512, 8): True,
             (320, 320, 32): True, (384, 320, 32): False, (256, 224, 32): True, (256, 40, 16): False,
             (128, 128, 12): False, (64, 32, 32): True}
    for (ny, nx, ct), fits in table.items():
        assert autotune.col_tile_fits(ny, nx, ct) == fits, (ny, nx, ct)


def test_candidates_and_default_groups():
    c = autotune.candidates(256, 256, 64)
    assert len(c) == 4 * 3 * 3 and (4, 16, 4) in c
    assert {g for g, _, _ in autotune.candidates(512, 512, 2)} == {1, 2}
    assert {ct for _, ct, _ in autotune.candidates(512, 512, 8)} == {8, 16}
    assert {ct for _, ct, _ in autotune.candidates(256, 256, 1, nz=128)} == {16}
    # the library's groups = 0: max(1, min(4, nb / 8)), at most nb
    assert [autotune.default_groups(n) for n in (1, 3, 8, 16, 31, 32, 64, 200)] == [1, 1, 1, 2, 3, 4, 4, 4]
    # two q = A p kernels only for 2D FP32 plans with 256 rows
    assert autotune.apply_tiles(256, 256) == [8, 16] and autotune.apply_tiles(128, 256) == [8, 16]
    assert autotune.apply_tiles(256, 128) == [8] and autotune.apply_tiles(256, 256, prec=2) == [8]
    assert autotune.apply_tiles(512, 512) == [8, 16] and autotune.apply_tiles(320, 320) == [8]
    assert autotune.apply_tiles(256, 256, nz=128) == [8]


def test_select_fastest_with_stable_ties():
    t = {(4, 16, 4): 2.0, (2, 8, 4): 1.5, (1, 32, 8): 1.5, (8, 16, 2): 3.0}
    assert autotune.select(t) == (1, 32, 8)


def test_store_and_unwritable_location(tmp_path, monkeypatch):
    path = str(tmp_path / "tune.json")
    assert autotune.store("a", {"groups": 2}, path) and autotune.store("b", {"groups": 4}, path)
    assert autotune.load_cache(path) == {"a": {"groups": 2}, "b": {"groups": 4}}

    def readonly(*a, **k):
        raise OSError("read-only file system")
    monkeypatch.setattr(autotune, "save_cache", readonly)
    assert autotune.store("c", {"groups": 1}, path) is False
    assert "c" not in autotune.load_cache(path)
