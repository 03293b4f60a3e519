"""The hand-written adjoint (fit_adjoint_forward / _backward) against the FP64
oracle's dual-number gradient and against central finite differences of the
GPU chi2, and its torch.autograd wrapper.

Tolerance: each gradient component within 1e-3 of its own magnitude plus 2e-3
of the track's gradient scale G (the largest |component| of that track).  The
floor comes from the arithmetic: every layer's residual r is a difference of
~100 cm positions held in FP32 (2^-24 * 110 cm = 6.6e-6 cm, a few roundings
per residual) and the gradient is built from r / sigma^2 with sigma = 0.01 cm,
i.e. ~0.5 / cm of noise per layer term, which is ~1e-3 of a typical G of
~500 / cm.
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

REL, FLOOR = 1e-3, 2e-3
# Lowest accepted pass rates under the plain 1e-3-relative criterion
# (regression guards; on a GB300: tracks 0.997 (p2r) and 1.000 (p2z),
# components 0.919 and 0.952, the rest within the FP32 floor above).
STRICT_TRACK_RATE_MIN = 0.99
STRICT_COMPONENT_RATE_MIN = 0.90


def _setup(mode, n, seed):
    ts = inputs.generate(mode, n, seed=seed)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    geom = fit.Geometry(ts.B, ts.surf)
    f = fit.Fitter(geom if mode == 0 else None, geom if mode == 1 else None)
    return ts, ld, d, f


def _gpu_grad(f, ts, ld, d, weight=None):
    n, mode = ts.n, ts.mode
    tape = torch.empty(fit.fit_tape_bytes(ts.nlayer, ld) // 4, device="cuda")
    out = f.outputs(n, ld=ld)
    fit.fit_adjoint_forward(f.h, *d, [n], [mode], tape, out["par"], out["cov"], out["q"],
                            out["chi2"], status=out["status"])
    w = torch.ones(ld, device="cuda") if weight is None else weight
    gh = torch.empty_like(d[3])
    gp = torch.empty((6, ld), device="cuda")
    gc = torch.empty((21, ld), device="cuda")
    fit.fit_adjoint_backward(f.h, d[3], d[4], [n], [mode], tape, w, gh, gp, gc)
    torch.cuda.synchronize()
    return out, gh.cpu().numpy()[..., :n], gp.cpu().numpy()[:, :n]


def _assert_close(got, ref, scale, label):
    err = np.abs(got - ref) - (REL * np.abs(ref) + FLOOR * scale)
    bad = err > 0
    assert not bad.any(), f"{label}: {int(bad.sum())} components out of tolerance, worst excess {err.max():.3g}"


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_gradient_matches_oracle(mode):
    ts, ld, d, f = _setup(mode, 301, seed=5 + mode)
    out, g_h, g_p = _gpu_grad(f, ts, ld, d)
    ref = oracle.chi2_grad(ts.mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)
    # the forward of the adjoint is the fused fit: same chi2 as the oracle's
    got = {k: v.cpu().numpy()[..., :ts.n] for k, v in out.items() if v is not None}
    assert (got["status"] == 0).all() and (ref["status"] == 0).all()
    c_err = np.abs(got["chi2"] - ref["chi2"]) / (parity.RTOL * ref["chi2"] + parity.CHI2_ABS * np.sqrt(ref["chi2"]))
    assert c_err.max() <= 1
    scale = np.maximum(np.abs(ref["g_hpos"]).max(axis=(0, 1)), np.abs(ref["g_par0"]).max(axis=0))
    _assert_close(g_h, ref["g_hpos"], scale[None, None, :], "hit gradient")
    _assert_close(g_p, ref["g_par0"], scale[None, :], "initial-parameter gradient")
    # the plain 1e-3-relative criterion: the fraction of tracks whose every
    # gradient component is within 1e-3 of the track's gradient scale, and
    # the fraction of components within 1e-3 of their own magnitude
    dev = np.maximum(np.abs(g_h - ref["g_hpos"]).max(axis=(0, 1)),
                     np.abs(g_p - ref["g_par0"]).max(axis=0))
    track_rate = float(np.mean(dev <= 1e-3 * scale))
    comp = np.concatenate([(np.abs(g_h - ref["g_hpos"]) <= 1e-3 * np.abs(ref["g_hpos"])).ravel(),
                           (np.abs(g_p - ref["g_par0"]) <= 1e-3 * np.abs(ref["g_par0"])).ravel()])
    print(f"mode {mode}: 1e-3 relative: tracks {track_rate:.4f}, components {comp.mean():.4f}")
    assert track_rate >= STRICT_TRACK_RATE_MIN and comp.mean() >= STRICT_COMPONENT_RATE_MIN
    if mode == inputs.MODE_Z:
        assert (g_h[:, 2] == 0).all()  # a plane's hit z does not enter the fit
    f.close()


def test_weights_scale_gradients_and_stopped_tracks():
    # weights multiply each track's gradient; a track that stops early
    # (cannot reach an outer cylinder) has no gradient for the layers it missed
    surf = inputs.surfaces(inputs.MODE_R)
    n = 64
    gap = float(surf[1] - surf[0])
    pt = np.where(np.arange(n) % 2 == 0, np.linspace(0.8, 8.0, n),
                  (surf[12].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2)
    ts = inputs.generate(inputs.MODE_R, n, seed=71, pt=pt)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf), None)
    w = torch.zeros(ld, device="cuda")
    w[:n] = torch.linspace(0.5, 2.0, n, device="cuda")
    out, g_h, g_p = _gpu_grad(f, ts, ld, d, weight=w)
    ref = oracle.chi2_grad(ts.mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)
    wn = w[:n].cpu().numpy()
    stopped = (ref["status"] & 1) != 0
    assert stopped.sum() == n // 2
    assert np.array_equal(out["status"].cpu().numpy()[:n] & 1, ref["status"] & 1)
    assert (g_h[13:, :, stopped] == 0).all()
    rh = np.nan_to_num(ref["g_hpos"]) * wn
    rp = ref["g_par0"] * wn
    scale = np.maximum(np.abs(rh).max(axis=(0, 1)), np.abs(rp).max(axis=0))
    _assert_close(g_h, rh, scale[None, None, :], "weighted hit gradient")
    _assert_close(g_p, rp, scale[None, :], "weighted initial-parameter gradient")
    f.close()


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
def test_gradient_against_finite_differences_of_gpu_chi2(mode):
    """Central differences of the GPU's own FP32 chi2.  Its rounding noise
    (~1e-2 for chi2 ~ 40) limits the steps to a fraction of the measurement
    errors; the comparison is to 3 % of the track's gradient scale."""
    ts, ld, d, f = _setup(mode, 8, seed=81 + mode)
    _, g_h, g_p = _gpu_grad(f, ts, ld, d)
    scale = np.maximum(np.abs(g_h).max(axis=(0, 1)), np.abs(g_p).max(axis=0))

    def chi2_of(hpos, par0):
        out = f.outputs(ts.n, ld=ld)
        f.run(par0, d[1], d[2], hpos, d[4], [ts.n], [mode], out=out)
        return out["chi2"].double().cpu().numpy()[:ts.n]

    def close(g, fd, label):
        assert (np.abs(g - fd) <= 0.03 * np.abs(fd) + 0.03 * scale).all(), (label, g, fd)

    checks = [(3, 0, 3e-3), (10, 1, 3e-3), (19, 0, 3e-3)] + ([(5, 2, 3e-2)] if mode == 0 else [])
    for l, k, eps in checks:
        hp, hm = d[3].clone(), d[3].clone()
        hp[l, k] += eps
        hm[l, k] -= eps
        close(g_h[l, k], (chi2_of(hp, d[0]) - chi2_of(hm, d[0])) / (2 * eps), f"hit {l},{k}")
    for k, eps in ((0, 3e-3), (3, 1e-2 * float(ts.par0[3].mean())), (4, 2e-3), (5, 2e-3)):
        pp, pm = d[0].clone(), d[0].clone()
        pp[k] += eps
        pm[k] -= eps
        close(g_p[k], (chi2_of(d[3], pp) - chi2_of(d[3], pm)) / (2 * eps), f"par0 {k}")
    f.close()


def test_autograd_function():
    ts, ld, d, f = _setup(inputs.MODE_R, 100, seed=91)
    hpos = d[3].clone().requires_grad_(True)
    par0 = d[0].clone().requires_grad_(True)
    cov0 = d[1].clone().requires_grad_(True)
    chi2, par, cov = fit.chi2(f, hpos, par0, cov0, d[2], d[4], [ts.n], [0])
    w = torch.rand(ld, device="cuda")
    (chi2 * w).sum().backward()
    _, g_h, g_p = _gpu_grad(f, ts, ld, d, weight=w.detach().clone())
    assert np.allclose(hpos.grad.cpu().numpy()[..., :ts.n], g_h, rtol=1e-6, atol=1e-5)
    assert np.allclose(par0.grad.cpu().numpy()[:, :ts.n], g_p, rtol=1e-6, atol=1e-5)
    assert cov0.grad is not None and torch.isfinite(cov0.grad[:, :ts.n]).all()
    f.close()


def test_full_size_adjoint_sampled():
    """The adjoint's workload at its full size (100k p2r tracks x 20 layers,
    seed 5, ld = n as in the benchmark): gradients against the oracle's on
    sampled tracks."""
    n = 100_000
    ts = inputs.generate(inputs.MODE_R, n, seed=5)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf), None)
    try:
        out, g_h, g_p = _gpu_grad(f, ts, ld, d)
        assert (out["status"].cpu().numpy()[:n] == 0).all()
        idx = np.sort(np.random.default_rng(3).choice(n, 400, replace=False))
        sub = ts.subset(idx)
        ref = oracle.chi2_grad(sub.mode, sub.B, sub.surf, sub.par0, sub.cov0, sub.q, sub.hpos,
                               sub.hcov)
        assert (ref["status"] == 0).all()
        gh, gp = g_h[..., idx], g_p[:, idx]
        scale = np.maximum(np.abs(ref["g_hpos"]).max(axis=(0, 1)), np.abs(ref["g_par0"]).max(axis=0))
        _assert_close(gh, ref["g_hpos"], scale[None, None, :], "full-size hit gradient")
        _assert_close(gp, ref["g_par0"], scale[None, :], "full-size initial-parameter gradient")
    finally:
        f.close()


def test_both_p2r_starts_give_the_same_gradient():
    """The path length is treated as the implicit function of the state that
    the Jacobian holds, so where the iteration starts (the closed-form
    crossing or the straight line) changes nothing beyond its tolerance:
    the two gradients agree component by component within the tolerance
    against the oracle."""
    ts = inputs.generate(inputs.MODE_R, 1000, seed=81)
    ld = gpu_util.pad_ld(ts.n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    grads = {}
    for start in (fit.FIT_START_CROSSING, fit.FIT_START_LINE):
        f = fit.Fitter(fit.Geometry(ts.B, ts.surf, start=start), None)
        try:
            _, gh, gp = _gpu_grad(f, ts, ld, d)
        finally:
            f.close()
        grads[start] = (gh, gp)
    (ha, pa), (hb, pb) = grads[fit.FIT_START_CROSSING], grads[fit.FIT_START_LINE]
    scale = np.maximum(np.abs(ha).reshape(-1, ts.n).max(axis=0), 1e-30)
    _assert_close(ha, hb, scale, "hit gradients, crossing vs line start")
    pscale = np.maximum(np.abs(pa).max(axis=0), 1e-30)
    _assert_close(pa, pb, pscale, "parameter gradients, crossing vs line start")
