"""The batched persistent form (fit_plan_*): uneven events of both modes in one
launch under a CUDA graph, against the FP64 oracle and against the per-segment
path; every launch shape the autotuner can pick; the tuning cache."""
import dataclasses
import os

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


def _events(nevt=60, seed=31):
    """Log-normal event sizes (median 60, clipped 1..400), a few empty events,
    modes p2r/p2z at random."""
    nt = inputs.uneven_event_sizes(nevt, seed, median=60.0, lo=1, hi=400)
    nt[[i for i in (3, 17) if i < nevt]] = 0
    md = inputs.uneven_event_modes(nevt, seed)
    return inputs.generate_events(nt, md, seed=seed)


def _device(ev, ld=None):
    ld = ld or gpu_util.pad_ld(ev.n)
    return ld, [gpu_util.to_dev(a, ld) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]


def _geoms(ev):
    return fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1])


def _outputs(f, ev, ld):
    out = f.outputs(ev.n, ld=ld)
    for k in ("par", "cov", "chi2"):
        out[k].fill_(float("nan"))
    return out


def _fetch(out, n):
    return {k: v.cpu().numpy()[..., :n] for k, v in out.items() if v is not None}


def _check_against_oracle(ev, got, label):
    s = ev.starts()
    for e in range(len(ev.ntrk)):
        if ev.ntrk[e] == 0:
            continue
        sub = {k: v[..., s[e]:s[e + 1]] for k, v in got.items()}
        parity.check(sub, oracle.fit_set(ev.event(e)), f"{label} event {e}")


def test_plan_matches_oracle_and_segments():
    ev = _events()
    ld, dev_in = _device(ev)
    f = fit.Fitter(*_geoms(ev))
    plan = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20)
    try:
        info = fit.fit_plan_get_info(plan)
        assert info["persistent"] and info["tracks"] == ev.n and info["items"] > 0
        out = _outputs(f, ev, ld)
        fit.fit_plan_run(plan, *dev_in, par_out=out["par"], cov_out=out["cov"], q_out=out["q"],
                         chi2=out["chi2"], status=out["status"])
        st = f.sync()
        assert st["tracks"] == ev.n and st["nonfinite"] == 0 and st["no_intersection"] == 0
        got = _fetch(out, ev.n)
        _check_against_oracle(ev, got, "plan")
        # the per-segment path on the same events agrees within the tolerance
        seg = _fetch(f.run(*dev_in, ev.ntrk, ev.mode), ev.n)
        f.sync()
        parity.check(got, seg, "plan vs segments")
        # a second run replays the graph; a new output set is captured anew
        out2 = _outputs(f, ev, ld)
        for _ in range(2):
            fit.fit_plan_run(plan, *dev_in, par_out=out2["par"], cov_out=out2["cov"],
                             q_out=out2["q"], chi2=out2["chi2"], status=out2["status"])
        f.sync()
        got2 = _fetch(out2, ev.n)
        for k in ("par", "cov", "q", "chi2", "status"):
            assert np.array_equal(got2[k], got[k]), k
    finally:
        fit.fit_plan_destroy(plan)
        f.close()



def test_plan_recaptures_for_a_new_hit_covariance_buffer():
    """Two runs with the same hit-position buffer and a different
    hit-covariance buffer: the second must read the new covariances (the
    captured graph is keyed on every buffer it reads), not replay the first
    run's pointer."""
    ev = _events(30, seed=37)
    ld, dev_in = _device(ev)
    f = fit.Fitter(*_geoms(ev))
    plan = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20)
    try:
        hcov2 = dev_in[4] * 4.0  # every hit error doubled
        ev2 = dataclasses.replace(ev, hcov=ev.hcov * np.float32(4.0))
        runs = []
        for hc in (dev_in[4], hcov2):
            out = _outputs(f, ev, ld)
            fit.fit_plan_run(plan, dev_in[0], dev_in[1], dev_in[2], dev_in[3], hc,
                             par_out=out["par"], cov_out=out["cov"], q_out=out["q"],
                             chi2=out["chi2"], status=out["status"])
            f.sync()
            runs.append(_fetch(out, ev.n))
        # the segment path with the same buffers is the reference for each run
        for hc, got, label in ((dev_in[4], runs[0], "first hcov"), (hcov2, runs[1], "second hcov")):
            ref = _fetch(f.run(dev_in[0], dev_in[1], dev_in[2], dev_in[3], hc, ev.ntrk, ev.mode),
                         ev.n)
            f.sync()
            parity.check(got, ref, f"plan, {label}")
        ok = (runs[0]["status"] == 0) & (runs[1]["status"] == 0)
        # larger hit errors, smaller chi2: the second run did read the new buffer
        assert runs[1]["chi2"][ok].mean() < 0.5 * runs[0]["chi2"][ok].mean()
        _check_against_oracle(ev2, runs[1], "plan, second hcov")
    finally:
        fit.fit_plan_destroy(plan)
        f.close()

def _to_layout(dev_in, layout):
    """The (SoA) track and hit arrays converted to `layout` with fit_relayout
    (per-track arrays, q, are the same in both layouts)."""
    if layout == fit.FIT_LAYOUT_SOA:
        return dev_in
    conv = []
    for k, a in enumerate(dev_in):
        if k == 2:
            conv.append(a)
            continue
        b = torch.empty_like(a)
        fit.fit_relayout(a, fit.FIT_LAYOUT_SOA, b, layout)
        conv.append(b)
    return conv


def _from_layout(out, layout):
    if layout == fit.FIT_LAYOUT_SOA:
        return out
    res = dict(out)
    for k in ("par", "cov", "chi2_layer"):
        if out.get(k) is not None:
            b = torch.empty_like(out[k])
            fit.fit_relayout(out[k], layout, b, fit.FIT_LAYOUT_SOA)
            res[k] = b
    return res


@pytest.mark.parametrize("tpb,bps,persistent,tpt,layout",
                         [(64, 1, 1, 2, 0), (64, 6, 1, 2, 0), (128, 1, 1, 2, 0), (128, 3, 1, 2, 0),
                          (32, 12, 1, 2, 0), (32, 1, 1, 2, 0), (128, 0, 0, 2, 0), (64, 0, 1, 1, 0),
                          (128, 2, 1, 1, 0), (256, 0, 1, 2, 0), (256, 1, 1, 1, 0),
                          (256, 0, 1, 1, 0), (128, 0, 1, 2, 1), (32, 5, 1, 2, 1),
                          (256, 0, 1, 2, 1), (64, 0, 1, 1, 1), (256, 2, 1, 1, 1),
                          (128, 0, 0, 2, 1)])
def test_every_launch_shape(tpb, bps, persistent, tpt, layout):
    """Every axis the tuner searches (threads per block, blocks per SM,
    persistent or per segment, tracks per thread, layout) against the oracle."""
    ev = _events(40, seed=41)
    ld, dev_in = _device(ev, ld=(ev.n + 31) // 32 * 32)
    f = fit.Fitter(*_geoms(ev))
    plan = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20, threads_per_block=tpb,
                               blocks_per_sm=bps, persistent=bool(persistent),
                               tracks_per_thread=tpt, layout=layout)
    try:
        info = fit.fit_plan_get_info(plan)
        assert info["tracks_per_thread"] == tpt and info["threads_per_block"] == tpb
        assert info["layout"] == layout
        out = _outputs(f, ev, ld)
        fit.fit_plan_run(plan, *_to_layout(dev_in, layout), par_out=out["par"],
                         cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                         status=out["status"])
        st = f.sync()
        assert st["tracks"] == ev.n
        _check_against_oracle(ev, _fetch(_from_layout(out, layout), ev.n),
                              f"shape {tpb},{bps},{persistent},{tpt},{layout}")
    finally:
        fit.fit_plan_destroy(plan)
        f.close()


def test_relayout_round_trip_and_errors():
    a = torch.arange(7 * 96, dtype=torch.float32, device="cuda").reshape(7, 96)
    b, c = torch.full_like(a, -1.0), torch.full_like(a, -1.0)
    fit.fit_relayout(a, fit.FIT_LAYOUT_SOA, b, fit.FIT_LAYOUT_AOSOA32)
    fit.fit_relayout(b, fit.FIT_LAYOUT_AOSOA32, c, fit.FIT_LAYOUT_SOA)
    assert torch.equal(a, c)
    # component k of track t sits at ((t / 32) * rows + k) * 32 + t % 32
    t, k = 45, 3
    assert b.reshape(-1)[((t // 32) * 7 + k) * 32 + t % 32].item() == a[k, t].item()
    with pytest.raises(fit.FitError):  # AoSoA needs ld % 32 == 0
        fit.fit_relayout(a[:, :90].contiguous(), fit.FIT_LAYOUT_SOA,
                         torch.empty(7, 90, device="cuda"), fit.FIT_LAYOUT_AOSOA32)


def test_tuner_chooses_the_layout():
    """A plan created with FIT_LAYOUT_TUNE has every shape timed in both
    layouts and then runs in the one chosen, which takes buffers in that
    layout; the result matches the oracle."""
    ev = _events(50, seed=53)
    ld, dev_in = _device(ev, ld=(ev.n + 31) // 32 * 32)
    f = fit.Fitter(*_geoms(ev))
    plan = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20, layout=fit.FIT_LAYOUT_TUNE)
    try:
        assert fit.fit_plan_get_info(plan)["layout"] == fit.FIT_LAYOUT_SOA  # until tuned
        out = _outputs(f, ev, ld)
        bufs = dict(par_out=out["par"], cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                    status=out["status"])
        info = fit.fit_plan_tune(plan, *dev_in, **bufs)
        assert info["tuned"] == 1 and info["layout"] in (fit.FIT_LAYOUT_SOA, fit.FIT_LAYOUT_AOSOA32)
        out = _outputs(f, ev, ld)
        fit.fit_plan_run(plan, *_to_layout(dev_in, info["layout"]), par_out=out["par"],
                         cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                         status=out["status"])
        f.sync()
        _check_against_oracle(ev, _fetch(_from_layout(out, info["layout"]), ev.n),
                              f"tuned layout {info['layout']}")
    finally:
        fit.fit_plan_destroy(plan)
        f.close()


def test_tune_and_cache(tmp_path):
    ev = _events(80, seed=51)
    ld, dev_in = _device(ev)
    f = fit.Fitter(*_geoms(ev))
    cache = str(tmp_path / "tune.txt")
    out = _outputs(f, ev, ld)
    bufs = dict(par_out=out["par"], cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                status=out["status"])
    p1 = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20)
    p2 = fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20)
    try:
        f.sync()
        info = fit.fit_plan_tune(p1, *dev_in, cache_path=cache, **bufs)
        assert info["tuned"] == 1 and info["best_ms"] > 0
        assert os.path.exists(cache) and open(cache).read().count("\t") == 1
        assert f.sync()["tracks"] == 0  # the tuning runs are not counted
        info2 = fit.fit_plan_tune(p2, *dev_in, cache_path=cache, **bufs)
        assert info2["tuned"] == 2
        for k in ("threads_per_block", "blocks_per_sm", "persistent", "tracks_per_thread", "layout"):
            assert info2[k] == info[k]
        fit.fit_plan_run(p2, *dev_in, **bufs)
        f.sync()
        _check_against_oracle(ev, _fetch(out, ev.n), "tuned plan")
        # tuning must not overwrite its own inputs
        with pytest.raises(fit.FitError) as e:
            fit.fit_plan_tune(p1, *dev_in, par_out=dev_in[0], cov_out=dev_in[1], q_out=dev_in[2],
                              chi2=out["chi2"])
        assert e.value.code == fit.FIT_ERR_ARG
    finally:
        fit.fit_plan_destroy(p1)
        fit.fit_plan_destroy(p2)
        f.close()


def test_plan_argument_errors():
    ev = _events(10, seed=61)
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), None)  # p2z not configured
    try:
        with pytest.raises(fit.FitError) as e:
            fit.fit_plan_create(f.h, ev.ntrk, ev.mode, 20)
        assert e.value.code == fit.FIT_ERR_ARG
        with pytest.raises(fit.FitError):
            fit.fit_plan_create(f.h, [10], [0], 19)  # nlayer differs
        with pytest.raises(fit.FitError):
            fit.fit_plan_create(f.h, [10], [0], 20, threads_per_block=96)
        with pytest.raises(fit.FitError):
            fit.fit_plan_create(f.h, [10], [0], 20, layout=3)
        with pytest.raises(fit.FitError):  # one track per thread: 64 or 128 threads
            fit.fit_plan_create(f.h, [10], [0], 20, threads_per_block=32, tracks_per_thread=1)
        with pytest.raises(fit.FitError):  # ... and persistent only
            fit.fit_plan_create(f.h, [10], [0], 20, persistent=False, tracks_per_thread=1)
        with pytest.raises(fit.FitError):
            fit.fit_plan_create(f.h, [10], [0], 20, tracks_per_thread=3)
    finally:
        f.close()


def test_full_size_uneven_batch_sampled():
    """The uneven-batch workload at its full size (2000 events, log-normal
    track counts, mixed modes, seed 3: ~6.5M tracks), run by a plan in the
    launch shape the benchmark times: the oracle on sampled tracks of both
    modes, properties on all."""
    nt = inputs.uneven_event_sizes(2000, 3)
    md = inputs.uneven_event_modes(2000, 3)
    ev = inputs.generate_events(nt, md, seed=3)
    n = ev.n
    ld, dev_in = _device(ev)
    f = fit.Fitter(*_geoms(ev))
    plan = fit.fit_plan_create(f.h, nt, md, 20)
    try:
        out = f.outputs(n, ld=ld)
        fit.fit_plan_run(plan, *dev_in, par_out=out["par"], cov_out=out["cov"], q_out=out["q"],
                         chi2=out["chi2"], status=out["status"])
        st = f.sync()
        assert st["tracks"] == n and st["no_intersection"] == 0 and st["nonfinite"] == 0
        got = _fetch(out, n)
        assert (got["status"] == 0).all() and np.isfinite(got["par"]).all()
        assert abs(got["chi2"].mean() / 20 - 2.0) < 0.02
        mode_of_track = np.repeat(md, nt)
        rng = np.random.default_rng(1)
        for m in (0, 1):
            pool = np.nonzero(mode_of_track == m)[0]
            idx = np.sort(rng.choice(pool, 1500, replace=False))
            sub = inputs.TrackSet(m, ev.B, ev.surf[m], ev.par0[:, idx], ev.cov0[:, idx], ev.q[idx],
                                  ev.hpos[:, :, idx], ev.hcov[:, :, idx])
            parity.check({k: v[..., idx] for k, v in got.items()}, oracle.fit_set(sub),
                         f"full-size uneven batch, mode {m}")
    finally:
        fit.fit_plan_destroy(plan)
        f.close()
