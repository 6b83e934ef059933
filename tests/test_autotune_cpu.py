"""Host logic of the launch-shape autotuner, without a GPU: the candidate
list and the cache file (timing the candidates is covered by the GPU tests)."""
import types

import numpy as np

from paper_2111_13667_gb300 import autotune


def stub(n_theta, n_lambda):
    """What candidates() reads of a device problem: the angle and wavelength grids."""
    return types.SimpleNamespace(theta=np.zeros(n_theta), lam=np.zeros(n_lambda))


def shapes(cands):
    return [(c.tile_lambda, c.tile_theta, c.persistent) for c in cands]


def test_the_library_default_comes_first_for_every_shape():
    for nt, nl in ((1, 7), (3, 2), (32, 512), (16, 256), (13, 203), (8, 64)):
        c = shapes(autotune.candidates(stub(nt, nl)))
        assert c[:2] == [(0, 0, 0), (0, 0, 1)]
        assert len(set(c)) == len(c)


def test_a_problem_too_small_for_every_tile_keeps_the_default():
    # 7 wavelengths x 1 angle: every listed tile is wider than twice the
    # wavelength count, so only the default shape remains to be timed
    assert shapes(autotune.candidates(stub(1, 7))) == [(0, 0, 0), (0, 0, 1)]


def test_listed_tiles_fit_one_block():
    c = shapes(autotune.candidates(stub(32, 512)))
    tiles = c[2:]
    assert len(tiles) >= 6
    for tl, tt, _ in tiles:
        assert 64 <= tl * tt <= 512 and 1 <= tt <= 32 and tl >= 4
    assert (16, 32, 0) in tiles and (16, 32, 1) in tiles


def test_persistent_options_are_respected():
    c = shapes(autotune.candidates(stub(8, 64), persistent_options=(1,)))
    assert c[0] == (0, 0, 1) and all(p == 1 for _, _, p in c)


def test_cache_round_trip_and_a_damaged_file(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "cache.json"
    monkeypatch.setattr(autotune, "CACHE_PATH", str(path))
    assert autotune._load_cache() == {}
    e1 = {"cfg": {"tile_lambda": 16, "tile_theta": 32, "persistent": 1, "blocks_per_sm": 0,
                  "max_items_per_block": 0}, "ms": 1.5}
    e2 = {"cfg": {"tile_lambda": 0, "tile_theta": 0, "persistent": 0, "blocks_per_sm": 0,
                  "max_items_per_block": 0}, "ms": 2.0}
    autotune._store("a", e1)
    autotune._store("b", e2)
    assert autotune._load_cache() == {"a": e1, "b": e2}
    assert not list(path.parent.glob("*.tmp*"))  # written through a temporary file, then replaced
    path.write_text("{not json")
    assert autotune._load_cache() == {}  # a damaged cache reads as empty
