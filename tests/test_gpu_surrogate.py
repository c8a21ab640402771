"""Droplet-impact surrogate: the footprint counter against the moments, and
a reduced end-to-end run (solver data -> tensor-core training -> held-out
error and speed against the solver)."""
import numpy as np
import pytest
import torch

from paper_1904_03618_gb300 import lbm
from paper_1904_03618_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


def test_footprint_matches_moments():
    setup = S.ImpactSetup(radius=5, box=(24, 20, 16), speed=0.04)
    samples = S.sample_impacts(3, setup, seed=5)
    sizes = [(24, 20, 16), (33, 17, 14), (20, 26, 18)]
    cases = []
    for s, box in zip(samples, sizes):
        setup.box = box
        cases.append(S.impact_case(s, setup))
    b = lbm.Batch([p for p, _ in cases])
    try:
        for k, (_, f) in enumerate(cases):
            b.init_fields(k, *f)
        b.step(150)
        for axis, index in [(2, 0), (2, 3), (0, 7), (1, 2)]:
            got = b.footprint(axis=axis, index=index)
            for k, (p, _) in enumerate(cases):
                rR, rB, _ = b.moments(k)
                rR, rB = rR.cpu().numpy(), rB.cpu().numpy()
                sl = [slice(None)] * 3
                sl[2 - axis] = index          # arrays are (z, y, x)
                a = rR[tuple(sl)] * np.float32(1.0 / p.rho_in_R)
                c = rB[tuple(sl)] * np.float32(1.0 / p.rho_in_B)
                assert got[k] == int(np.count_nonzero(a > c)), (axis, index, k)
        # a drop of radius 5 falling at 0.04 from 2 cells up wets the floor by t = 150
        assert np.all(b.footprint(2, 0) > 0)
        with pytest.raises(lbm.LbmError):
            b.footprint(axis=2, index=14)     # beyond the second case
        with pytest.raises(lbm.LbmError):
            b.footprint(axis=3, index=0)
    finally:
        b.close()


def test_surrogate_reduced_run_beats_baselines():
    setup = S.ImpactSetup(radius=6, box=(40, 40, 24), speed=0.04, t_end=3.0, samples=12)
    samples = S.sample_impacts(320, setup, seed=11)
    runs = S.run_impacts(samples, setup, chunk=320)
    assert runs.valid.mean() > 0.9
    ok = runs.series[runs.valid]
    assert np.all(np.isfinite(ok))
    # spreading: the footprint grows from nothing to more than the drop's diameter
    assert np.median(ok[:, -1]) > 1.0
    rep = S.report(runs, train_steps=2000)
    err, mean_err, lin_err = (rep["held_out_error"]["rmse"], rep["mean_predictor_error"]["rmse"],
                              rep["linear_fit_error"]["rmse"])
    assert err < 0.5 * mean_err, rep
    assert err < lin_err, rep
    assert rep["speedup_vs_solver"] > 100.0, rep
    assert rep["screening"]["recall"] >= 0.8, rep
