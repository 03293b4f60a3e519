"""Pins of the oracle's track finding (orc_find) to the oracle's single-step
functions, which test_oracle.py pins to the paper's geometry: a layer-by-layer
composition of propagate and update, with the argmin over candidates written
out here, must give the same choices and states; one candidate and no gate is
the plain fit; no acceptable candidate leaves the pure propagation."""
import numpy as np
import pytest

import oracle
from paper_2409_09228_gb300 import inputs

GATE = 30.0


def _brute_force(ts, cs, gate):
    nlayer, ncand, _, n = cs.cpos.shape
    out = {"par": np.zeros((6, n)), "cov": np.zeros((21, n)), "chi2": np.zeros(n),
           "chosen": np.full((nlayer, n), -1)}
    for i in range(n):
        p, c, q = ts.par0[:, i].astype(np.float64), ts.cov0[:, i].astype(np.float64), int(ts.q[i])
        chi2 = 0.0
        for l in range(nlayer):
            st, pp, cp = oracle.propagate(ts.mode, ts.B, float(ts.surf[l]), q, p, c)
            if st:
                break
            trial = [oracle.update(ts.mode, q, pp, cp, cs.cpos[l, k, :, i], cs.ccov[l, k, :, i])[4]
                     for k in range(ncand)]
            ok = [k for k in range(ncand) if trial[k] < gate]
            p, c = pp, cp
            if ok:
                best = min(ok, key=lambda k: (trial[k], k))
                out["chosen"][l, i] = best
                _, p, c, q, x = oracle.update(ts.mode, q, pp, cp, cs.cpos[l, best, :, i],
                                              cs.ccov[l, best, :, i])
                chi2 += x
        out["par"][:, i], out["cov"][:, i], out["chi2"][i] = p, c, chi2
    return out


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_find_equals_layerwise_composition(mode):
    ts = inputs.generate(mode, 12, seed=21, nlayer=4)
    cs = inputs.generate_candidates(ts, 3, seed=21, spread=3.0, p_true=0.7)
    got = oracle.find(mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, GATE)
    ref = _brute_force(ts, cs, GATE)
    assert np.array_equal(got["chosen"], ref["chosen"])
    assert (got["chosen"] >= 0).any() and (got["chosen"] != np.maximum(cs.true_slot, -1)).any()
    for k in ("par", "cov", "chi2"):
        assert np.allclose(got[k], ref[k], rtol=1e-13, atol=1e-15), k


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_one_candidate_without_gate_is_the_plain_fit(mode):
    ts = inputs.generate(mode, 200, seed=22)
    cpos, ccov = ts.hpos[:, None], ts.hcov[:, None]
    got = oracle.find(mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cpos, ccov, 1e300)
    ref = oracle.fit_set(ts, want_layers=True)
    for k in ("par", "cov", "q", "chi2", "chi2_layer", "status"):
        assert np.array_equal(got[k], ref[k]), k
    assert (got["chosen"] == 0).all()


def test_no_acceptable_candidate_leaves_the_prediction():
    ts = inputs.generate(inputs.MODE_R, 20, seed=23, nlayer=5)
    cs = inputs.generate_candidates(ts, 2, seed=23, spread=1e4, p_true=0.0)
    got = oracle.find(0, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, GATE)
    assert (got["chosen"] == -1).all() and (got["chi2"] == 0).all()
    assert np.isfinite(got["cand_chi2"]).all() and (got["cand_chi2"] >= GATE).all()
    for i in range(ts.n):
        p, c = ts.par0[:, i].astype(np.float64), ts.cov0[:, i].astype(np.float64)
        for l in range(5):
            _, p, c = oracle.propagate(0, ts.B, float(ts.surf[l]), int(ts.q[i]), p, c)
        assert np.allclose(got["par"][:, i], p, rtol=1e-14) and np.allclose(got["cov"][:, i], c, rtol=1e-14)


def test_well_separated_candidates_find_the_true_hit():
    ts = inputs.generate(inputs.MODE_Z, 500, seed=24)
    cs = inputs.generate_candidates(ts, 4, seed=24, spread=1e3, p_true=1.0)
    got = oracle.find(1, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, GATE)
    assert np.mean(got["chosen"] == cs.true_slot) > 0.999
