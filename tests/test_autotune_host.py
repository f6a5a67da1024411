"""Host logic of the batched-sweep autotuner, without a GPU: the search
(one common z-run length, then each size class halved / doubled) and the
JSON cache, against a synthetic cost whose minimum is known."""
import json
import math

import pytest

from paper_2408_03452_gb300 import autotune


@pytest.fixture
def fake(monkeypatch):
    calls = []

    def cost(grids, zc, coef, coef64, b, tol, maxit, precond, sweep=0, tile=0):
        calls.append((list(zc), sweep, tile))
        # per class a parabola in log2(zc): 48x48x24 is best at 8, 128x128x64 at
        # 32; TMA tile 2 saves a constant, the cp.async sweep costs one
        best = {(48, 48, 24): 3, (128, 128, 64): 5}
        seen = {}
        for g, z in zip(grids, zc):
            seen[tuple(g[:3])] = z
        shape = {(0, 0): 0.0, (0, 1): 0.2, (0, 2): -0.5, (0, 3): 0.1, (1, 0): 1.0}[(sweep, tile)]
        return sum((math.log2(z) - best[k]) ** 2 for k, z in seen.items()) + shape + 2.0

    monkeypatch.setattr(autotune, "_time_batch", cost)
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda *a: "fake-device")
    return calls


GRIDS = [(48, 48, 24), (128, 128, 64), (48, 48, 24)]


def test_search_finds_the_per_class_optimum(fake):
    zc = autotune.tune(GRIDS, None, None, None)
    assert zc == [8, 32, 8]
    # six common candidates, then two trials per class
    assert len(fake) == len(autotune.CANDIDATES) + 2 * 2


def test_cache_roundtrip_and_corrupt_cache(fake, tmp_path):
    cache = str(tmp_path / "zc.json")
    first = autotune.tune(GRIDS, None, None, None, cache=cache)
    n = len(fake)
    again = autotune.tune(GRIDS, None, None, None, cache=cache)
    assert again == first and len(fake) == n  # answered from the cache, nothing timed
    db = json.load(open(cache))
    (key,) = db
    assert json.loads(key)[0] == "fake-device" and db[key]["ms_per_solve"] == 2.0
    # another tolerance is another key; an unreadable cache is ignored and rewritten
    autotune.tune(GRIDS, None, None, None, tol=1e-6, cache=cache)
    assert len(json.load(open(cache))) == 2
    open(cache, "w").write("{not json")
    assert autotune.tune(GRIDS, None, None, None, cache=cache) == first
    assert len(json.load(open(cache))) == 1


def test_batch_search_picks_kernel_tile_and_per_class_runs(fake):
    r = autotune.tune_batch(GRIDS, None, None, None)
    assert r["zc"] == [8, 32, 8] and (r["sweep"], r["tile"]) == (0, 2)
    assert r["ms_per_solve"] == pytest.approx(1.5)
    # six common candidates (TMA tile 0), three other tiles and the cp.async
    # sweep at the best common run, then two trials per class with the best shape
    assert len(fake) == len(autotune.CANDIDATES) + 4 + 2 * 2
    assert all(c[1:] == (0, 2) for c in fake[-4:])
    # the Jacobi variant has one tile: only the cp.async sweep is compared
    fake.clear()
    r = autotune.tune_batch(GRIDS, None, None, None, precond=1)
    assert (r["sweep"], r["tile"]) == (0, 0) and len(fake) == len(autotune.CANDIDATES) + 1 + 4


def test_batch_cache_keeps_kernel_and_tile(fake, tmp_path):
    cache = str(tmp_path / "t.json")
    a = autotune.tune_batch(GRIDS, None, None, None, cache=cache)
    n = len(fake)
    b = autotune.tune_batch(GRIDS, None, None, None, cache=cache)
    assert b == a and len(fake) == n
    # the zc-only search is another key
    autotune.tune(GRIDS, None, None, None, cache=cache)
    assert len(json.load(open(cache))) == 2
