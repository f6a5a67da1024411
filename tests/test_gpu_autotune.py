"""The batched-sweep autotuner returns a valid z-run per instance, caches
it, and its choice solves the batch to tolerance."""
import json

import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def test_autotune_choice_and_cache(tp, tmp_path):
    from paper_2408_03452_gb300 import autotune
    ens = synth.ensemble(seed=3, n_inst=6, sizes=((12, 10, 8), (20, 16, 12)))
    grids = [(w["nx"], w["ny"], w["nz"]) for w in ens]
    K, mask, pD = (torch.from_numpy(np.concatenate([w[k] for w in ens])).cuda()
                   for k in ("K", "mask", "pD"))
    with tp.BatchContext(grids) as bc:
        coef, coef64 = bc.build_trans(K, mask, None, 0.0)
        b = bc.build_rhs(K, mask, None, pD)
    cache = str(tmp_path / "tune.json")
    zc = autotune.tune(grids, coef, coef64, b, tol=1e-8, precond=1, cache=cache)
    assert len(zc) == len(grids) and all(z in (2, 4, 8, 16, 32, 64, 128, 256) for z in zc)
    # one value per size class
    by = {}
    for g, z in zip(grids, zc):
        assert by.setdefault(g, z) == z
    db = json.load(open(cache))
    assert len(db) == 1
    assert autotune.tune(grids, coef, coef64, b, tol=1e-8, precond=1, cache=cache) == zc
    with tp.BatchContext(grids, zc=zc) as bc:
        bc.set_option("precond", 1)
        _, per, tot = bc.cg_solve(coef, coef64, b, tol=1e-8)
        assert tot["code"] == 0 and all(p["status"] == 0 for p in per)
