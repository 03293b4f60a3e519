"""Track finding on the GPU (fit_find_tracks, fit_find_tracks_f64) against the
oracle's (orc_find).

The choice of candidate is an argmin over chi2 values decided in floating
point.  In double (the paper's default precision) both sides decide alike:
the FP64 kernel must take exactly the oracle's choice on every layer.  In
FP32 a choice is unique where the oracle's best chi2 is further than DELTA
from the runner-up (or from the gate); there the FP32 kernel must agree, and
where it is not unique its choice must be valid, i.e. within DELTA of the
best.  DELTA = 1e-3 chi2 + 0.03 sqrt(chi2) + 1e-3 bounds the FP32 chi2 of one
layer against FP64: a relative 1e-4 from the state (the parity tolerance of
the fit) and the rounding of the residual, 4 x 6.6e-4 sigma, doubled, plus a
margin.  After a differing (valid) choice the two tracks follow different
hits and are no longer compared; tracks whose choices all agree must pass the
fit's parity check.  Except for the covariance of tracks that found no
acceptable hit on more than MAX_SKIPPED layers: each p2r propagation leaves
the covariance without variance along the radius, runs of them without an
update keep it near-singular, and FP32 loses relative accuracy in the
near-null directions (up to ~8e-3 of the entry's scale after 13-16 skipped
layers; the FP64 finder matches the oracle on the same tracks to 1e-11).  Those
tracks are compared on parameters and chi2."""
import numpy as np
import pytest

import oracle
import parity
from paper_2409_09228_gb300 import fit, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA device", allow_module_level=True)

GATE = 30.0
NCAND = 4
MAX_SKIPPED = 3


def _dev(a, ld, dtype):
    pad = [(0, 0)] * (a.ndim - 1) + [(0, ld - a.shape[-1])]
    a = np.pad(a, pad)
    if a.dtype.kind == "f":
        a = a.astype(dtype)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _find(f, ts, cs, dtype, gate=GATE):
    n = ts.n
    ld = (n + 3) // 4 * 4
    d = [_dev(a, ld, dtype) for a in (ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov)]
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    dev = torch.device("cuda")
    out = {"par": torch.empty((6, ld), dtype=tdt, device=dev),
           "cov": torch.empty((21, ld), dtype=tdt, device=dev),
           "q": torch.empty(ld, dtype=torch.int32, device=dev),
           "chi2": torch.empty(ld, dtype=tdt, device=dev),
           "chi2_layer": torch.empty((ts.nlayer, ld), dtype=tdt, device=dev),
           "status": torch.empty(ld, dtype=torch.uint8, device=dev)}
    chosen = torch.empty((ts.nlayer, ld), dtype=torch.int8, device=dev)
    fit.fit_find_tracks(f.h, *d, [n], [ts.mode], gate, chosen, out["par"], out["cov"], out["q"],
                        out["chi2"], chi2_layer=out["chi2_layer"], status=out["status"])
    st = f.sync()
    got = {k: v.cpu().numpy()[..., :n] for k, v in out.items()}
    got["chosen"] = chosen.cpu().numpy()[:, :n].astype(np.int32)
    return got, st


def _setup(mode, n, seed, tol=1e-6):
    ts = inputs.generate(mode, n, seed=seed)
    cs = inputs.generate_candidates(ts, NCAND, seed=seed, spread=20.0, p_true=0.95)
    geom = fit.Geometry(ts.B, ts.surf, tol=tol)
    f = fit.Fitter(geom if mode == 0 else None, geom if mode == 1 else None)
    ref = oracle.find(mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, GATE)
    return ts, cs, f, ref


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_f64_finder_takes_the_oracles_choices(mode):
    ts, cs, f, ref = _setup(mode, 2049, 31 + mode, tol=1e-12)
    try:
        got, st = _find(f, ts, cs, np.float64)
        ok = (got["status"] == 0) & (ref["status"] == 0)
        assert ok.mean() > 0.99
        assert np.array_equal(got["chosen"][:, ok], ref["chosen"][:, ok])
        assert ((ref["chosen"] >= 0) & (ref["chosen"] != cs.true_slot)).any()  # noise was taken
        assert (ref["chosen"] < 0).any()  # and some layers had no acceptable hit
        parity.check({k: v[..., ok] for k, v in got.items()}, {k: v[..., ok] for k, v in ref.items()},
                     "f64 finder", rtol=1e-11, chi2_abs=1e-10)
    finally:
        f.close()


def _delta(x):
    return 1e-3 * np.abs(x) + 0.03 * np.sqrt(np.abs(x)) + 1e-3


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_f32_finder_unique_choices_agree(mode):
    ts, cs, f, ref = _setup(mode, 4097, 41 + mode)
    try:
        got, st = _find(f, ts, cs, np.float32)
        cc = ref["cand_chi2"]  # (nlayer, ncand, n)
        same_path = np.ones(ts.n, bool)
        ambiguous = differing = 0
        for l in range(ts.nlayer):
            g, r = got["chosen"][l], ref["chosen"][l]
            x = np.where(np.isfinite(cc[l]), cc[l], np.inf)
            xs = np.sort(x, axis=0)
            best = np.minimum(xs[0], GATE)
            runner = np.where(xs[0] < GATE, np.minimum(xs[1], GATE), xs[0])
            unique = (runner - best) > _delta(best)
            live = same_path & (ref["status"] == 0) & (got["status"] == 0)
            diff = live & (g != r)
            ambiguous += int((live & ~unique).sum())
            assert not (diff & unique).any(), f"layer {l}: a unique choice differs"
            # a differing choice is valid: its chi2 is within DELTA of the best (or of the gate)
            idx = np.nonzero(diff)[0]
            for i in idx:
                xg = GATE if g[i] < 0 else x[g[i], i]
                assert abs(xg - best[i]) <= _delta(best[i]) or (g[i] < 0 and best[i] >= GATE - _delta(GATE))
            differing += len(idx)
            same_path &= ~diff
        print(f"\nmode {mode}: {ts.n * ts.nlayer} choices, {ambiguous} not unique, {differing} differ")
        keep = same_path & (got["status"] == 0) & (ref["status"] == 0)
        assert keep.mean() > 0.99
        skipped = (ref["chosen"] < 0).sum(axis=0)
        full = keep & (skipped <= MAX_SKIPPED)
        parity.check({k: v[..., full] for k, v in got.items()},
                     {k: v[..., full] for k, v in ref.items()}, "f32 finder")
        rest = keep & ~full
        e = parity.scaled_errors({k: v[..., rest] for k, v in got.items()},
                                 {k: v[..., rest] for k, v in ref.items()})
        assert (e["par"] <= 1).all() and (e["chi2"] <= 1).all()
        print(f"  {int(full.sum())} tracks compared in full, {int(rest.sum())} (more than "
              f"{MAX_SKIPPED} layers without a hit) on parameters and chi2")
    finally:
        f.close()


def test_f64_finder_with_the_most_candidates():
    """ncand = 16, the limit: the FP64 kernel still takes exactly the oracle's
    choices."""
    ts = inputs.generate(inputs.MODE_Z, 257, seed=61)
    cs = inputs.generate_candidates(ts, 16, seed=61, spread=10.0, p_true=0.9)
    f = fit.Fitter(None, fit.Geometry(ts.B, ts.surf, tol=1e-12))
    try:
        ref = oracle.find(1, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, GATE)
        got, _ = _find(f, ts, cs, np.float64)
        ok = (got["status"] == 0) & (ref["status"] == 0)
        assert ok.mean() > 0.99
        assert np.array_equal(got["chosen"][:, ok], ref["chosen"][:, ok])
        assert got["chosen"].max() > 8  # the high slots are used
    finally:
        f.close()


@pytest.mark.parametrize("start", [fit.FIT_START_CROSSING, fit.FIT_START_LINE],
                         ids=["crossing", "line"])
def test_one_candidate_is_the_fit(start):
    ts = inputs.generate(inputs.MODE_R, 1000, seed=51)
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf, start=start), None)
    try:
        cs = inputs.CandidateSet(ts.hpos[:, None], ts.hcov[:, None], np.zeros((20, ts.n), np.int32))
        got, st = _find(f, ts, cs, np.float32, gate=1e30)
        assert (got["chosen"] == 0).all() and st["tracks"] == ts.n
        parity.check(got, oracle.fit_set(ts), f"finder with one candidate, start {start}")
        per = st["iterations"] / (ts.n * ts.nlayer)
        assert per < 1.01 if start == fit.FIT_START_CROSSING else per > 1.5
    finally:
        f.close()


def test_one_candidate_on_strongly_turning_tracks_is_the_fit():
    """Four cylinders 70 cm apart, pT from 1.1 to 2.5 times the reach limit
    of the outermost: between cylinders the tracks turn by up to 1 rad, and
    on many surfaces the p2r crossing start needs its exact form, which the
    FP32 finder runs outside its layer loop.  With one candidate (the track's
    own hit) the finder must give the fused fit's results (which reaches the
    exact form through the one-track path of a packed pair), and the FP64
    finder the oracle's fit (to 1e-9: the 1/pT variance collapses ~170-fold
    per update in this geometry, which amplifies rounding ~2e5-fold)."""
    import gpu_util
    surf = np.array([20.0, 90.0, 160.0, 230.0], np.float32)
    B = float(np.float32(3.8))
    pt_min = inputs.pt_min_p2r(B, 230.0, frac=1.0)
    pt = np.linspace(1.1 * pt_min, 2.5 * pt_min, 1000)
    ts = inputs.generate(inputs.MODE_R, pt.size, seed=32, surf=surf, pt=pt)
    cs = inputs.CandidateSet(ts.hpos[:, None], ts.hcov[:, None],
                             np.zeros((ts.nlayer, ts.n), np.int32))
    ref_fit = gpu_util.run([ts])
    f = fit.Fitter(fit.Geometry(B, surf), None)
    try:
        got, st = _find(f, ts, cs, np.float32, gate=1e30)
    finally:
        f.close()
    assert (got["chosen"] == 0).all() and (got["status"] == 0).all()
    assert st["iterations"] == ref_fit["sync"]["iterations"]
    for k in ("par", "cov", "chi2"):
        a, b = got[k], ref_fit[k][..., :ts.n]
        scale = np.maximum(np.abs(b), 1e-30 if k != "cov" else 0.0)
        if k == "cov":  # relative to the scale of each entry, as in parity.py
            d = np.abs(a - b)
            dia = np.abs(b[parity.DIAG])
            for m, (i, j) in enumerate(parity.PAIRS):
                assert (d[m] <= 1e-6 * np.sqrt(dia[i] * dia[j])).all(), (k, i, j)
        else:
            assert (np.abs(a - b) <= 1e-6 * scale + 1e-6).all(), k
    f = fit.Fitter(fit.Geometry(B, surf, tol=1e-12), None)
    try:
        got64, _ = _find(f, ts, cs, np.float64, gate=1e30)
    finally:
        f.close()
    assert (got64["chosen"] == 0).all()
    parity.check(got64, oracle.fit_set(ts), "FP64 finder, turning tracks", rtol=1e-9,
                 chi2_abs=1e-10)


@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_unreachable_first_surface_returns_the_inputs(dtype):
    """The finder, like the fit, hands back the inputs unchanged for a track
    that cannot reach its first surface (it carries a projection of the input
    covariance); the other tracks match the fit with their own hits."""
    n = 600
    i = np.arange(n)
    pt = np.where(i % 3 == 0, 0.02, np.linspace(0.75, 9.0, n))
    ts = inputs.generate(inputs.MODE_R, n, seed=23, pt=pt)
    cs = inputs.CandidateSet(ts.hpos[:, None], ts.hcov[:, None], np.zeros((ts.nlayer, ts.n), np.int32))
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf, tol=1e-12 if dtype == np.float64 else 1e-6), None)
    try:
        got, _ = _find(f, ts, cs, dtype, gate=1e30)
    finally:
        f.close()
    r = oracle.fit_set(ts)
    first = (r["status"] & 1) != 0
    assert first.sum() == (i % 3 == 0).sum()
    assert np.array_equal(got["status"][first], r["status"][first])
    for k, v in (("par", ts.par0), ("cov", ts.cov0)):
        assert np.array_equal(got[k][:, first], v[:, first].astype(dtype)), k
    assert (got["chi2"][first] == 0).all() and (got["chosen"][:, first] == -1).all()
    ok = ~first
    tol = 1e-9 if dtype == np.float64 else 1e-4
    parity.check({k: (v[..., ok] if isinstance(v, np.ndarray) else v) for k, v in got.items()},
                 {k: v[..., ok] for k, v in r.items() if isinstance(v, np.ndarray)},
                 f"finder, first surface out of reach ({np.dtype(dtype).name})", rtol=tol,
                 **({"chi2_abs": 1e-10} if dtype == np.float64 else {}))


def test_stopped_tracks_and_argument_errors():
    surf = inputs.surfaces(inputs.MODE_R)
    n = 64
    gap = float(surf[1] - surf[0])
    pt = np.where(np.arange(n) % 2 == 0, np.linspace(0.8, 8.0, n),
                  (surf[12].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2)
    ts = inputs.generate(inputs.MODE_R, n, seed=71, pt=pt)
    cs = inputs.generate_candidates(ts, 2, seed=71, spread=20.0, p_true=1.0)
    cs.cpos[np.isnan(cs.cpos)] = 0.0  # hits of unreachable layers: never tried
    cs.ccov[np.isnan(cs.ccov)] = 0.0
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf), None)
    try:
        got, st = _find(f, ts, cs, np.float32)
        stopped = (got["status"] & 1) != 0
        assert stopped.sum() == n // 2 and st["no_intersection"] == n // 2
        assert (got["chosen"][13:, stopped] == -1).all() and (got["chi2_layer"][13:, stopped] == 0).all()
        ld = (n + 3) // 4 * 4
        d = [_dev(a, ld, np.float32) for a in (ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov)]
        chosen = torch.empty((20, ld), dtype=torch.int8, device="cuda")
        o = [torch.empty((6, ld), device="cuda"), torch.empty((21, ld), device="cuda"),
             torch.empty(ld, dtype=torch.int32, device="cuda"), torch.empty(ld, device="cuda")]
        with pytest.raises(fit.FitError):
            fit.fit_find_tracks(f.h, *d, [n], [0], 0.0, chosen, *o)  # gate must be > 0
        big = torch.zeros((20, 17, 3, ld), device="cuda")
        with pytest.raises(fit.FitError):
            fit.fit_find_tracks(f.h, d[0], d[1], d[2], big, torch.zeros((20, 17, 6, ld), device="cuda"),
                                [n], [0], GATE, chosen, *o)  # ncand > 16
    finally:
        f.close()
