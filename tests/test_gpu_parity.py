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


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_parity_1x1024x20(mode):
    ts = inputs.generate(mode, 1024, seed=1)
    g = gpu_util.run([ts], layers=True)
    r = oracle.fit_set(ts, want_layers=True)
    s = parity.check(gpu_util.trim(g, 0, ts.n), r, f"mode {mode}")
    assert s["compared"] == ts.n and s["flag_gpu"] == 0
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
    assert (g["cov"][parity.DIAG[[0, 1, 3, 4, 5]]] > 0).all()
    # mean chi2 per layer of a consistent filter is 2 (chi2 with 2 d.o.f.)
    assert abs(g["chi2"].mean() / ts.nlayer - 2.0) < 0.02
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([[0, ntrk - 1, ntrk, ts.n - 1],
                                    rng.choice(ts.n, 3000, replace=False)]))
    sub = ts.subset(idx)
    parity.check(gpu_util.trim({k: v[..., idx] if isinstance(v, np.ndarray) else v
                                for k, v in g.items()}, 0, len(idx)),
                 oracle.fit_set(sub), "full size sample")
