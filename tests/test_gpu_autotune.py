"""The launch-configuration autotuner picks a valid configuration, applies
it, caches it by signature, and reuses the cache."""
import json

import pytest
import torch

from paper_1904_03618_gb300 import autotune, lbm, workloads as wl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_tune_single_lattice_and_cache(tmp_path):
    d = dict(wall=(0, 0, 1), rho_in_R=3.0, alpha_R=0.9, alpha_B=0.7, A_R=0.01, A_B=0.01)
    p = lbm.make_params(40, 30, 20, **d)
    stream = torch.cuda.Stream(DEV)
    lat = lbm.Lattice(p, device=DEV, stream=stream)
    lat.init_fields(*wl.droplet(40, 30, 20, 6.0, 3.0, 1.0))
    cache = str(tmp_path / "tune.json")
    cands = [(8, 8, 2), (8, 12, 0), (16, 8, 1)]
    ty, zc, hold, ms, src = autotune.tune(lat.ctx, [p], stream, steps=4, cache_path=cache,
                                          candidates=cands)
    assert src == "timed" and (ty, zc, hold) in cands and ms > 0
    assert lbm.lbm_get_fused_config(lat.ctx) == (ty, zc, hold)
    table = json.load(open(cache))
    assert autotune.signature([p], p.storage) in table
    lbm.lbm_set_fused_config(lat.ctx, 8, 4, 0)
    again = autotune.tune(lat.ctx, [p], stream, cache_path=cache)
    assert again[4] == "cache" and lbm.lbm_get_fused_config(lat.ctx) == (ty, zc, hold)
    assert lat.diagnostics()[5] == 0
    lat.close()


def test_tune_batch():
    cases = [lbm.make_params(n, n, n, rho_in_R=2.0, alpha_R=1 - 0.3 / 2, alpha_B=0.7,
                             A_R=0.01, A_B=0.01) for n in (16, 24, 33)]
    stream = torch.cuda.Stream(DEV)
    b = lbm.Batch(cases, device=DEV, stream=stream)
    for k, p in enumerate(cases):
        b.init_fields(k, *wl.droplet(p.nx, p.ny, p.nz, p.nx / 4, 2.0, 1.0))
    ty, zc, hold, ms, src = autotune.tune(b.ctx, cases, stream, steps=3, cache_path=None)
    assert (ty, hold) in autotune.BATCH_SHAPES and src == "timed"
    assert lbm.lbm_get_fused_config(b.ctx) == (ty, zc, hold)
    b.close()
