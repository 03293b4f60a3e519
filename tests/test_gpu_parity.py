"""Parity of the CUDA fused kernels (through the C ABI) with the FP64 oracle.

Tolerances: tests/parity.py.  Sizes span several 128-thread blocks and ragged
tails; the full-size workload (100 events x 9600 tracks x 20 layers per mode,
in the launch configuration bench.py times) is checked on sampled tracks and
on properties that hold at any size.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2409_09228_gb300 import fit, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA device", allow_module_level=True)

import gpu_util  # noqa: E402

# Lowest accepted fraction of tracks whose chi2 meets the literal 1e-4
# criterion (parity.strict_chi2_rate); the rest are within the FP32
# residual-rounding bound of parity.check.  A regression guard: on a GB300
# the kernels gave 0.969 (p2r) and 0.995 (p2z) at 1024 tracks, 0.971 and
# 0.991 on the full-size sample.
STRICT_CHI2_RATE_MIN = 0.95


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_parity_1x1024x20(mode):
    ts = inputs.generate(mode, 1024, seed=1)
    g = gpu_util.run([ts], layers=True)
    r = oracle.fit_set(ts, want_layers=True)
    s = parity.check(gpu_util.trim(g, 0, ts.n), r, f"mode {mode}")
    assert s["compared"] == ts.n and s["flag_gpu"] == 0
    # chi2 under the specified 1e-4-relative criterion taken literally
    rate = parity.strict_chi2_rate(gpu_util.trim(g, 0, ts.n), r)
    print(f"mode {mode}: strict chi2 pass rate {rate:.4f}")
    assert rate >= STRICT_CHI2_RATE_MIN, rate
    assert g["sync"]["tracks"] == ts.n and g["sync"]["no_intersection"] == 0
    # per-layer chi2 within the same per-track chi2 tolerance, layer by layer
    d = np.abs(g["chi2_layer"][:, :ts.n] - r["chi2_layer"])
    tol = parity.RTOL * r["chi2_layer"] + parity.CHI2_ABS * np.sqrt(r["chi2_layer"] / ts.nlayer)
    assert (d <= tol + 1e-6).all()
    assert np.allclose(g["chi2_layer"][:, :ts.n].sum(0), g["chi2"][:ts.n], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("n", [1, 5, 127, 129, 1000, 4097])
@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_parity_ragged(mode, n):
    ts = inputs.generate(mode, n, seed=100 + n)
    ld = gpu_util.pad_ld(n) + 8
    g = gpu_util.run([ts], ld=ld)
    parity.check(gpu_util.trim(g, 0, n), oracle.fit_set(ts), f"n={n}")
    # nothing written beyond the tracks of the call
    assert np.isnan(g["par"][:, n:]).all() and np.isnan(g["chi2"][n:]).all()


def test_multi_event_mixed_modes():
    sizes = [100, 0, 250, 37, 300, 5, 129]
    modes = [0, 0, 1, 1, 0, 1, 0]
    sets = [inputs.generate(m, k, seed=200 + i) for i, (m, k) in enumerate(zip(modes, sizes))]
    g = gpu_util.run(sets)
    t = 0
    for s in sets:
        if s.n:
            parity.check(gpu_util.trim(g, t, t + s.n), oracle.fit_set(s), f"event at {t}")
        t += s.n
    assert g["sync"]["tracks"] == sum(sizes)


def test_mixed_modes_are_joined_back_to_the_callers_stream():
    """A call with events of both modes runs its p2z launches on the handle's
    second stream and joins them back to the caller's.  With a large p2z
    event between two small p2r events, synchronising the caller's stream
    alone must find every output written (NaN and 0xff before the call) and
    matching the oracle; the counters must hold every track."""
    sets = [inputs.generate(inputs.MODE_R, 64, seed=301),
            inputs.generate(inputs.MODE_Z, 200000, seed=302),
            inputs.generate(inputs.MODE_R, 33, seed=303)]
    f = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf), fit.Geometry(sets[1].B, sets[1].surf))
    try:
        c = gpu_util.concat(sets)
        n = c["par0"].shape[-1]
        ld = gpu_util.pad_ld(n)
        d = [gpu_util.to_dev(c[k], ld) for k in ("par0", "cov0", "q", "hpos", "hcov")]
        out = f.outputs(n, ld=ld)
        for k in ("par", "cov", "chi2"):
            out[k].fill_(float("nan"))
        out["status"].fill_(0xff)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        f.run(*d, [x.n for x in sets], [x.mode for x in sets], out=out, stream=s)
        s.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        st = f.sync(s)
    finally:
        f.close()
    assert (got["status"][:n] != 0xff).all()
    fin = (got["status"][:n] & fit.FIT_ST_NONFINITE) == 0
    assert np.isfinite(got["par"][:, :n][:, fin]).all() and np.isfinite(got["chi2"][:n][fin]).all()
    assert st["tracks"] == n
    t = 0
    for x in sets:
        parity.check(gpu_util.trim(got, t, t + x.n), oracle.fit_set(x), f"event at {t}")
        t += x.n


@pytest.mark.parametrize("start", [fit.FIT_START_CROSSING, fit.FIT_START_LINE],
                         ids=["crossing", "line"])
def test_p2r_starts_reach_the_oracles_crossing(start):
    """Both starts of the path-length iteration end on the oracle's crossing
    (its exact first root).  From the closed-form crossing the first step
    confirms convergence; from the straight line it takes a second one."""
    ts = inputs.generate(inputs.MODE_R, 4097, seed=31)
    g = gpu_util.run([ts], layers=True, start=start)
    parity.check(gpu_util.trim(g, 0, ts.n), oracle.fit_set(ts, want_layers=True), f"start {start}")
    st = g["sync"]
    per = st["iterations"] / (ts.n * ts.nlayer)
    print(f"\nstart {start}: {per:.4f} iterations per track-layer")
    assert st["not_converged"] == 0 and st["no_intersection"] == 0
    if start == fit.FIT_START_CROSSING:
        assert per < 1.01
    else:
        assert 1.5 < per < 3.0


def _path_lengths(start, B, surf, par, q, R):
    """fit_path_lengths with the given start: (h, iterations), h NaN where the
    cylinder is not reached."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    f = fit.Fitter(fit.Geometry(B, surf, start=start), None)
    try:
        h = torch.empty(R.size, device="cuda")
        it = torch.empty(R.size, dtype=torch.int32, device="cuda")
        fit.fit_path_lengths(f.h, dev(par), dev(q), dev(R), h, it)
        return h.cpu().numpy(), it.cpu().numpy()
    finally:
        f.close()


def _h_bound(R, h_ref):
    # the iteration's tolerance 1e-6 R plus a few FP32 roundings of h
    return 1e-6 * R + 8 * 2.0 ** -24 * h_ref


def test_p2r_starts_on_strongly_turning_tracks():
    """Four cylinders 70 cm apart and pT from 1.1 to 2.5 times the reach
    limit of the outermost: between cylinders the tracks turn by up to 1 rad,
    beyond the range of the crossing start's series form (|tan| of half the
    turn <= 1/4), where its exact form takes over.

    (1) The FP32 path-length step alone, from each truth crossing outwards to
    the next cylinder and, reversed, inwards to the previous one.  The
    crossing start reaches every cylinder, as the oracle does, at the
    oracle's root; the straight-line start reaches every outward one but
    gives up on inward starts whose tangent misses the cylinder.  (2) The
    whole fit in FP64 matches the oracle with both starts, to 1e-9: with four
    hits 70 cm apart each update shrinks the 1/pT variance ~170-fold, and the
    update C - K H C amplifies rounding ~2e5-fold (measured in FP32, where it
    leaves ~1e-2 relative with either start), so double keeps ~2e-11 of it,
    not the 1e-11 of the standard workload.  (3) The FP32 fused fit, where a
    packed pair hands a track that needs the exact crossing to the one-track
    path: every track is fitted (status 0), its parameters and chi2 within
    the FP32 tolerances, at one iteration per track-layer from the crossing
    start; the covariance is not compared, for the reason above."""
    surf = np.array([20.0, 90.0, 160.0, 230.0], np.float32)
    B = float(np.float32(3.8))
    pt_min = inputs.pt_min_p2r(B, 230.0, frac=1.0)
    pt = np.linspace(1.1 * pt_min, 2.5 * pt_min, 1000)
    ts = inputs.generate(inputs.MODE_R, pt.size, seed=32, surf=surf, pt=pt, want_truth=True)
    # (1) states: truth at cylinder l -> cylinder l + 1, and reversed -> cylinder l - 1
    par, q, R, inward = [], [], [], []
    for l in range(ts.nlayer):
        if l + 1 < ts.nlayer:
            par.append(ts.truth[l])
            q.append(ts.q)
            R.append(np.full(ts.n, surf[l + 1]))
            inward.append(np.zeros(ts.n, bool))
        if l >= 1:
            rev = ts.truth[l].copy()
            rev[4] += np.pi
            rev[5] = np.pi - rev[5]
            par.append(rev)
            q.append(-ts.q)
            R.append(np.full(ts.n, surf[l - 1]))
            inward.append(np.ones(ts.n, bool))
    par = np.concatenate(par, axis=1).astype(np.float32)
    q = np.concatenate(q).astype(np.int32)
    R = np.concatenate(R).astype(np.float32)
    inward = np.concatenate(inward)
    h_ref, st_ref = oracle.path_lengths(0, B, R.astype(np.float64), q, par.astype(np.float64))
    assert (st_ref == 0).all()
    its = {}
    for start in (fit.FIT_START_CROSSING, fit.FIT_START_LINE):
        h, it = _path_lengths(start, B, surf, par, q, R)
        reached = np.isfinite(h)
        assert reached[~inward].all(), start
        if start == fit.FIT_START_CROSSING:
            assert reached.all()
        assert (np.abs(h - h_ref)[reached] <= _h_bound(R, h_ref)[reached]).all(), start
        its[start] = np.where(reached, it, -1)
    both = (its[fit.FIT_START_LINE] >= 0)
    c, line = its[fit.FIT_START_CROSSING][both], its[fit.FIT_START_LINE][both]
    print(f"\nturning tracks: {c.mean():.3f} (crossing) vs {line.mean():.3f} (line) iterations; "
          f"the line start reaches {both.mean():.3f} of the states")
    assert c.mean() < line.mean()
    # (2) the FP64 fit in this geometry, both starts
    import test_gpu_f64 as f64
    ref = oracle.fit_set(ts)
    for start in (fit.FIT_START_CROSSING, fit.FIT_START_LINE):
        f = fit.Fitter(fit.Geometry(B, surf, tol=f64.TOL_F64, start=start), None)
        try:
            got, st = f64._run64(f, ts, layers=False)
            parity.check(got, ref, f"turning tracks f64, start {start}", rtol=1e-9,
                         chi2_abs=f64.CHI2_ABS_F64)
            assert st["not_converged"] == 0 and (got["status"] == 0).all()
        finally:
            f.close()
    # (3) the FP32 fused fit, both starts
    for start in (fit.FIT_START_CROSSING, fit.FIT_START_LINE):
        g = gpu_util.run([ts], start=start)
        e = parity.scaled_errors(gpu_util.trim(g, 0, ts.n), ref)
        assert (g["status"][:ts.n] == 0).all() and g["sync"]["no_intersection"] == 0, start
        assert e["par"].max() <= 1 and e["chi2"].max() <= 1, start
        if start == fit.FIT_START_CROSSING:
            assert g["sync"]["iterations"] <= 1.01 * ts.n * ts.nlayer


def test_crossing_start_reach_and_roots_on_random_states():
    """200k random p2r states (anywhere within r < 250 cm, any direction,
    pT from 0.5 to 20 GeV, either charge) to random cylinders 5..260 cm: the
    crossing start decides reachability like the oracle (the circle meets the
    cylinder or not), on every state whose track circle passes the cylinder
    by more than 1e-3 R (near-tangent states may go either way in FP32).  Its
    path lengths match the oracle's roots where the problem is resolvable in
    FP32: the crossing not grazing (radial slope > 0.1), a turn below 2 rad,
    R >= 10 cm and |r0 - R| <= 100 cm (so that the tolerance 1e-6 R is above
    the rounding of the coordinates)."""
    rng = np.random.default_rng(7)
    n = 200_000
    r0 = rng.uniform(0, 250, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    par = np.stack([r0 * np.cos(ang), r0 * np.sin(ang), rng.uniform(-50, 50, n),
                    rng.uniform(0.05, 2.0, n), rng.uniform(-np.pi, np.pi, n),
                    rng.uniform(0.5, 2.6, n)]).astype(np.float32)
    q = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int32)
    R = rng.uniform(5, 260, n).astype(np.float32)
    B = float(np.float32(3.8))
    h_ref, st_ref = oracle.path_lengths(0, B, R.astype(np.float64), q, par.astype(np.float64))
    # circle geometry of each state (centre distance cn, radius rho) and, at the
    # oracle's crossing, the turn and the radial slope
    p = par.astype(np.float64)
    kap = -q * inputs.KA * B * p[3]
    cx, cy = p[0] - np.sin(p[4]) / kap, p[1] + np.cos(p[4]) / kap
    cn, rho = np.hypot(cx, cy), 1.0 / np.abs(kap)
    margin = np.minimum(np.abs(R - (cn + rho)), np.abs(R - np.abs(cn - rho)))
    u = 0.5 * kap * h_ref
    chord = 2.0 * np.sin(u) / kap
    xe, ye = p[0] + chord * np.cos(p[4] + u), p[1] + chord * np.sin(p[4] + u)
    slope = np.abs(xe * np.cos(p[4] + 2 * u) + ye * np.sin(p[4] + 2 * u)) / R
    surf = np.array([10.0], np.float32)
    h, it = _path_lengths(fit.FIT_START_CROSSING, B, surf, par, q, R)
    reach, reach_ref = np.isfinite(h), st_ref == 0
    robust = margin > 1e-3 * R
    assert np.array_equal(reach[robust], reach_ref[robust])
    assert (reach != reach_ref).sum() <= 20
    fair = (reach & reach_ref & (slope > 0.1) & (np.abs(kap) * h_ref < 2.0) & (R >= 10)
            & (np.abs(r0 - R) <= 100))
    assert fair.sum() > 50_000
    assert (np.abs(h - h_ref)[fair] <= _h_bound(R, h_ref)[fair]).all()
    assert (it[fair] >= 10).sum() <= 20  # flagged as not converged
    print(f"\nrandom states: {reach_ref.sum()} reachable, {(reach != reach_ref).sum()} "
          f"reach decisions differ; {it[fair].mean():.4f} iterations on {fair.sum()}")


def test_not_converged_tracks_are_flagged_and_counted():
    """The iteration's limit: from the straight-line start with max_iter = 1 most
    p2r track-layers stop one step short of the tolerance.  Those tracks carry
    the NOT_CONVERGED bit, the counter equals the flags, their outputs stay
    finite (the last iterate, with its direction turned by the general
    rotation rather than the converged-step series), and with enough
    iterations the same tracks match the oracle."""
    ts = inputs.generate(inputs.MODE_R, 3000, seed=77)
    g1 = gpu_util.run([ts], max_iter=1, start=fit.FIT_START_LINE)
    st = g1["status"][:ts.n]
    flagged = (st & fit.FIT_ST_NOT_CONVERGED) != 0
    assert flagged.sum() > ts.n // 2
    assert g1["sync"]["not_converged"] == int(flagged.sum())
    assert ((st & ~np.uint8(fit.FIT_ST_NOT_CONVERGED)) == 0).all()
    for k in ("par", "cov", "chi2"):
        assert np.isfinite(g1[k][..., :ts.n]).all(), k
    # one step short of the root moves the state by less than the step itself
    g10 = gpu_util.run([ts], max_iter=10, start=fit.FIT_START_LINE)
    assert (g10["status"][:ts.n] == 0).all()
    assert np.abs(g1["par"][:3, :ts.n] - g10["par"][:3, :ts.n]).max() < 0.05
    parity.check(gpu_util.trim(g10, 0, ts.n), oracle.fit_set(ts), "max_iter 10, line start")


def test_bad_start_is_an_argument_error():
    with pytest.raises(fit.FitError) as e:
        fit.Fitter(fit.Geometry(3.8, inputs.surfaces(0), start=7), None)
    assert e.value.code == fit.FIT_ERR_ARG


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_charge_flip_matches_oracle(mode):
    """Seeds with the wrong charge and a loose 1/pT (sigma_w = 0.1 / GeV
    against w = 0.05 / GeV): the first update drives w through zero, and the
    fit flips q and the sign of w with row and column 3 of C (reading R8).
    Every track flips, on the GPU as in the oracle, and ends where the
    oracle's does."""
    n = 2000
    ts = inputs.generate(mode, n, seed=61 + mode, pt=np.full(n, 20.0))
    ts.q = (-ts.q).astype(np.int32)
    ts.cov0[9] = np.float32(0.1 ** 2)  # (w, w)
    g = gpu_util.run([ts])
    r = oracle.fit_set(ts)
    assert (r["status"] == fit.FIT_ST_CHARGE_FLIP).all()
    assert np.array_equal(g["status"][:n], r["status"])
    assert g["sync"]["charge_flip"] == n
    assert np.array_equal(g["q"][:n], r["q"]) and (r["q"] == -ts.q).all()
    gs = gpu_util.trim(g, 0, n)
    gs["status"] = np.zeros(n, np.uint8)
    rs = dict(r, status=np.zeros(n, np.uint8))
    parity.check(gs, rs, f"charge flip, mode {mode}")


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_nonfinite_track_leaves_its_pair_alone(mode):
    """A NaN hit on layer 5 of every seventh track (both positions of a
    two-track pair): those tracks stop with FIT_ST_NONFINITE, their per-layer
    chi2 from that layer on is 0, and every other track, the partners of the
    bad ones included, fits like the oracle."""
    n = 1000
    ts = inputs.generate(mode, n, seed=71 + mode)
    bad = np.arange(0, n, 7)
    ts.hpos[5, 0, bad] = np.nan
    g = gpu_util.run([ts], layers=True)
    r = oracle.fit_set(ts, want_layers=True)
    good = np.ones(n, bool)
    good[bad] = False
    assert (g["status"][:n][bad] & fit.FIT_ST_NONFINITE).all()
    assert (r["status"][bad] & fit.FIT_ST_NONFINITE).all()
    assert (g["status"][:n][good] == 0).all() and (r["status"][good] == 0).all()
    assert g["sync"]["nonfinite"] == bad.size
    assert (g["chi2_layer"][5:, bad] == 0).all()
    s = parity.check(gpu_util.trim(g, 0, n), r, f"partners of non-finite tracks, mode {mode}")
    assert s["compared"] == good.sum()
    # per-layer chi2 of the good tracks too, the partners' in particular
    partners = np.unique(np.concatenate([bad ^ 1]))
    partners = partners[(partners < n) & good[np.minimum(partners, n - 1)]]
    d = np.abs(g["chi2_layer"][:, partners] - r["chi2_layer"][:, partners])
    tol = parity.RTOL * r["chi2_layer"][:, partners] + parity.CHI2_ABS * np.sqrt(
        r["chi2_layer"][:, partners] / ts.nlayer)
    assert (d <= tol + 1e-6).all()


def test_in_place_equals_out_of_place():
    ts = inputs.generate(inputs.MODE_R, 700, seed=3)
    a = gpu_util.run([ts])
    b = gpu_util.run([ts], in_place=True)
    for k in ("par", "cov", "q", "chi2"):
        assert np.array_equal(a[k][..., :700], b[k][..., :700]), k


def test_max_layers_and_straight_line():
    surf = np.linspace(10.0, 270.0, fit.FIT_MAX_LAYERS).astype(np.float32)
    ts = inputs.generate(inputs.MODE_Z, 300, seed=9, surf=surf)
    parity.check(gpu_util.trim(gpu_util.run([ts]), 0, 300), oracle.fit_set(ts), "64 planes")
    # B = 0: straight lines (the kappa -> 0 limit of every formula)
    for mode in (inputs.MODE_R, inputs.MODE_Z):
        ts = inputs.generate(mode, 300, seed=10 + mode)
        ts.B = 0.0
        parity.check(gpu_util.trim(gpu_util.run([ts]), 0, 300), oracle.fit_set(ts), "B=0")


def test_no_intersection_status_matches_oracle():
    # Half of the p2r tracks have 2 rho half-way between two cylinders, so they
    # stop at the first cylinder they cannot reach (with a margin of ~2.8 cm
    # that the fitted curvature cannot cross).
    surf = inputs.surfaces(inputs.MODE_R)
    n = 400
    gap = np.float64(surf[1] - surf[0])
    layer = 8 + np.arange(n) % 7
    pt = np.where(np.arange(n) % 2 == 0,
                  np.linspace(0.75, 9.0, n),
                  (surf[layer].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2)
    ts = inputs.generate(inputs.MODE_R, n, seed=12, pt=pt)
    g = gpu_util.run([ts])
    r = oracle.fit_set(ts)
    stopped = (r["status"] & 1) != 0
    assert stopped.sum() == n // 2
    assert np.array_equal(g["status"][:n], r["status"])
    assert g["sync"]["no_intersection"] == n // 2
    # the stopped tracks keep their last good state, like the oracle's
    gs = {k: v[..., :n][..., stopped] if isinstance(v, np.ndarray) else v for k, v in g.items()}
    rs = {k: v[..., stopped] for k, v in r.items() if isinstance(v, np.ndarray)}
    gs["status"] = gs["status"] * 0
    rs["status"] = rs["status"] * 0
    parity.check(gs, rs, "stopped tracks")
    parity.check(gpu_util.trim(g, 0, n), r, "all tracks")


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_unreachable_first_surface_returns_the_inputs(mode):
    """A track that cannot reach its first surface has nothing applied: its
    outputs are its inputs bit for bit (the layer loop carries a projection of
    the input covariance, so the kernel reads the inputs back), its status and
    chi2 say so, and the other track of its pair fits as the oracle does.
    p2r: pT = 0.02 GeV (2 rho < 4 cm) on tracks 0, 1, 3 of every 6, so pairs
    with one, the other or both lanes stopped; p2z: eta of either sign (the
    planes of tracks moving to -z are behind them)."""
    n = 1200
    if mode == inputs.MODE_R:
        i = np.arange(n)
        pt = np.where(np.isin(i % 6, [0, 1, 3]), 0.02, np.linspace(0.75, 9.0, n))
        ts = inputs.generate(inputs.MODE_R, n, seed=21, pt=pt)
    else:  # |eta| in [1.5, 2.5] (the p2z workload's range), either sign, in random order
        ts = inputs.generate(inputs.MODE_Z, 3 * n, seed=22, eta_range=(-2.5, 2.5))
        eta = -np.log(np.tan(0.5 * ts.par0[5].astype(np.float64)))
        ts = ts.subset(np.nonzero(np.abs(eta) >= 1.5)[0][:n])
        n = ts.n
    g = gpu_util.run([ts])
    r = oracle.fit_set(ts)
    first = (r["status"] & 1) != 0
    assert 0.2 * n < first.sum() < 0.8 * n
    assert np.array_equal(r["par"][:, first], ts.par0[:, first].astype(np.float64))
    diff = np.nonzero(g["status"][:n] != r["status"])[0]
    assert diff.size == 0, (diff[:10], g["status"][diff[:10]], r["status"][diff[:10]],
                            ts.par0[:, diff[:10]])
    for k, v in (("par", ts.par0), ("cov", ts.cov0)):
        assert np.array_equal(g[k][:, :n][:, first].view(np.uint32), v[:, first].view(np.uint32)), k
    assert (g["chi2"][:n][first] == 0).all() and np.array_equal(g["q"][:n][first], ts.q[first])
    parity.check(gpu_util.trim(g, 0, n), r, "first surface out of reach")


def test_empty_and_zero_tracks():
    f = fit.Fitter(fit.Geometry(3.8, inputs.surfaces(0)), None)
    empty = torch.empty((6, 4), device="cuda")
    fit.fit_propagate_update(f.h, empty, torch.empty((21, 4), device="cuda"),
                             torch.empty(4, dtype=torch.int32, device="cuda"),
                             torch.empty((20, 3, 4), device="cuda"),
                             torch.empty((20, 6, 4), device="cuda"), [], [],
                             chi2=torch.empty(4, device="cuda"))
    fit.fit_propagate_update(f.h, empty, torch.empty((21, 4), device="cuda"),
                             torch.empty(4, dtype=torch.int32, device="cuda"),
                             torch.empty((20, 3, 4), device="cuda"),
                             torch.empty((20, 6, 4), device="cuda"), [0, 0], [0, 0],
                             chi2=torch.empty(4, device="cuda"))
    assert f.sync()["tracks"] == 0
    f.close()


def test_argument_errors():
    f = fit.Fitter(fit.Geometry(3.8, inputs.surfaces(0)), None)
    n, ld = 8, 8
    par = torch.zeros((6, ld), device="cuda")
    cov = torch.zeros((21, ld), device="cuda")
    q = torch.ones(ld, dtype=torch.int32, device="cuda")
    hpos = torch.zeros((20, 3, ld), device="cuda")
    hcov = torch.zeros((20, 6, ld), device="cuda")
    chi2 = torch.zeros(ld, device="cuda")

    def call(**kw):
        args = dict(par_in=par, cov_in=cov, q_in=q, hpos=hpos, hcov=hcov, ntrk=[n], mode=[0],
                    chi2=chi2)
        args.update(kw)
        fit.fit_propagate_update(f.h, **args)

    cases = [dict(mode=[1]),                       # mode not configured
             dict(mode=[7]),                       # no such mode
             dict(ntrk=[ld + 1]),                  # more tracks than ld
             dict(ntrk=[-1]),
             dict(hpos=torch.zeros((19, 3, ld), device="cuda")),  # nlayer mismatch
             dict(par_in=torch.zeros(6 * ld + 1, device="cuda")[1:].view(6, ld)),  # misaligned
             dict(chi2=None)]
    for kw in cases:
        with pytest.raises(fit.FitError) as e:
            call(**kw)
        assert e.value.code == fit.FIT_ERR_ARG, kw
    par6 = torch.zeros((6, 6), device="cuda")
    with pytest.raises(fit.FitError):  # ld not a multiple of 4
        fit.fit_propagate_update(f.h, par6, torch.zeros((21, 6), device="cuda"),
                                 torch.ones(6, dtype=torch.int32, device="cuda"),
                                 torch.zeros((20, 3, 6), device="cuda"),
                                 torch.zeros((20, 6, 6), device="cuda"), [4], [0],
                                 chi2=torch.zeros(6, device="cuda"))
    call()  # and the valid call still works
    f.sync()
    f.close()


def test_sync_timeout_then_complete():
    ts = inputs.generate(inputs.MODE_R, 1_000_000, seed=13)
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf), None)
    ld = gpu_util.pad_ld(ts.n)
    args = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    out = f.outputs(ts.n, ld=ld)
    torch.cuda.synchronize()
    for _ in range(10):
        f.run(*args, [ts.n], [0], out=out)
    with pytest.raises(fit.FitError) as e:
        f.sync(timeout_s=1e-6)  # the queued work takes milliseconds
    assert e.value.code == fit.FIT_ERR_TIMEOUT
    st = f.sync()  # the counters survive a timed-out wait
    assert st["tracks"] == 10 * ts.n and st["no_intersection"] == 0
    f.close()


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_full_size_100x9600x20_sampled(mode):
    """The benchmark workload: oracle on sampled tracks, properties on all."""
    nevt, ntrk = 100, 9600
    ts = inputs.generate(mode, nevt * ntrk, seed=2)
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf) if mode == 0 else None,
                   fit.Geometry(ts.B, ts.surf) if mode == 1 else None)
    ld = ts.n
    args = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    out = f.outputs(ts.n, ld=ld)
    f.run(*args, [ntrk] * nevt, [mode] * nevt, out=out)
    st = f.sync()
    f.close()
    g = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    assert st["tracks"] == ts.n and st["no_intersection"] == 0 and st["nonfinite"] == 0
    assert (g["status"] == 0).all()
    assert np.isfinite(g["par"]).all() and np.isfinite(g["cov"]).all()
    assert ((g["par"][4] > -np.pi - 1e-6) & (g["par"][4] <= np.pi + 1e-6)).all()
    assert (g["cov"][parity.DIAG[[3, 4, 5]]] > 0).all()
    # x and y variances: on a cylinder the variance along the radial direction
    # is zero, so for a track crossing within ~1e-4 rad of the x (y) axis the
    # true x (y) variance is ~1e-12 of the transverse one and FP32 rounding can
    # put it on either side of zero; every such track must still agree with
    # the oracle, and no variance may be negative beyond that rounding
    vx, vy = g["cov"][parity.DIAG[0]], g["cov"][parity.DIAG[1]]
    assert ((vx + vy) > 0).all()
    assert (np.minimum(vx, vy) >= -1e-6 * (vx + vy)).all()
    odd = np.nonzero((vx <= 0) | (vy <= 0))[0]
    if len(odd):
        parity.check(gpu_util.trim({k: v[..., odd] if isinstance(v, np.ndarray) else v
                                    for k, v in g.items()}, 0, len(odd)),
                     oracle.fit_set(ts.subset(odd)), "tracks with a non-positive x or y variance")
    # mean chi2 per layer of a consistent filter is 2 (chi2 with 2 d.o.f.)
    assert abs(g["chi2"].mean() / ts.nlayer - 2.0) < 0.02
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, ntrk - 1, ntrk, ts.n - 1],
                                    rng.choice(ts.n, 3000, replace=False)]))
    sub = ts.subset(idx)
    gs = gpu_util.trim({k: v[..., idx] if isinstance(v, np.ndarray) else v
                        for k, v in g.items()}, 0, len(idx))
    rs = oracle.fit_set(sub)
    parity.check(gs, rs, "full size sample")
    rate = parity.strict_chi2_rate(gs, rs)
    print(f"mode {mode}: full size sample, strict chi2 pass rate {rate:.4f}")
    assert rate >= STRICT_CHI2_RATE_MIN, rate
