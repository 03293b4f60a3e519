"""The learned p2r path-length seed on the GPU: its inputs, forward pass,
gradient and Adam step against the FP64 reference (oracle/mlp.py, BF16
roundings emulated); training on 4M propagations whose path lengths come from
the FP64 oracle; the seeded path-length iteration and the seeded fit against
the oracle; and what the trained network gains over the straight-line seed.

Tolerances.  Inputs: FP32 evaluation of O(1) quantities, 2e-6 absolute.
Targets g = (h - h_line) / (kappa h_line^2 / 2): the FP32 rounding of h and of
h_line, whose x^2 + y^2 - R^2 carries a few units of 2^-24 R^2 (so a few units
of 2^-24 R in h_line), divided by kappa h_line^2 / 2.  Network output:
99 % of the samples within 1e-5, all within one BF16 unit per hidden
activation (see _close_net).  Gradient: 1e-3 relative per parameter block.  Path lengths: the iteration's own tolerance 1e-6 R.
"""
import time

import numpy as np
import pytest

import oracle
import parity
from oracle import mlp as om
from paper_2409_09228_gb300 import fit, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA device", allow_module_level=True)

import gpu_util  # noqa: E402

N_TRAIN = 4_000_000
TOL = 1e-6  # relative path-length tolerance of the iteration (fit_config.tol)


def _dev_samples(ss):
    par = torch.from_numpy(np.ascontiguousarray(ss.par)).cuda()
    q = torch.from_numpy(ss.q).cuda()
    R = torch.from_numpy(ss.R).cuda()
    return par, q, R


def _prepare(ss, h=None):
    par, q, R = _dev_samples(ss)
    x = torch.empty((ss.n, 8), device="cuda")
    t = None
    if h is not None:
        t = torch.empty(ss.n, device="cuda")
        h = torch.from_numpy(np.asarray(h, np.float32)).cuda()
    fit.fit_mlp_prepare(ss.B, par, q, R, x, h_exact=h, target=t)
    return x, t


@pytest.fixture(scope="module")
def trained():
    """A network trained on N_TRAIN p2r propagations labelled by the oracle's
    exact path lengths (200 epochs, batches of 4096, Adam with a cosine decay
    from 2e-3 to 1e-6)."""
    ss = inputs.seed_samples(N_TRAIN, seed=4)
    h, st = oracle.path_lengths(0, ss.B, ss.R.astype(np.float64), ss.q, ss.par.astype(np.float64))
    assert (st == 0).all()
    x, t = _prepare(ss, h)
    m = fit.fit_mlp_create(0, seed=4)
    t0 = time.time()
    curve = fit.fit_mlp_train(m, x, t, epochs=200, batch=4096, lr=2e-3, lr_final=1e-6, seed=4)
    print(f"\ntraining on {N_TRAIN} samples: {time.time() - t0:.2f} s, loss per epoch "
          f"{curve[0]:.3g} ... {curve[-1]:.3g}")
    yield m, curve
    fit.fit_mlp_destroy(m)


def test_inputs_and_targets_match_oracle():
    ss = inputs.seed_samples(100_003, seed=41)
    h, _ = oracle.path_lengths(0, ss.B, ss.R.astype(np.float64), ss.q, ss.par.astype(np.float64))
    x, t = _prepare(ss, h)
    X = om.features(ss.B, ss.par, ss.q, ss.R)
    assert np.abs(x.cpu().numpy() - X).max() <= 2e-6
    g = om.target(ss.B, ss.par, ss.q, ss.R, h)
    hl = om.line_distance(ss.par, ss.R)
    scale = np.abs(0.5 * om.curvature(ss.B, ss.par, ss.q) * hl * hl)
    bound = 16 * 2.0 ** -24 * np.maximum(ss.R, h) / scale + 1e-5 * np.abs(g)
    got = t.cpu().numpy()
    assert (np.abs(got - g) <= bound).all(), np.max(np.abs(got - g) / bound)


def _forward(m, x):
    y = torch.empty(x.shape[0], device="cuda")
    fit.fit_mlp_forward(m, x, y)
    return y.cpu().numpy()


def _close_net(got, P, x, label):
    """GPU output against the reference with the BF16 roundings emulated.  The
    two accumulate in different orders (FP32 tensor cores, FP64), so a hidden
    activation that lands within ~1e-7 of a BF16 rounding boundary can round
    one unit (2^-8 relative) apart.  Every sample must lie within the sum over
    all hidden activations of one such unit times the output's sensitivity to
    it (|W3| for layer 2; |W2|^T |W3| for layer 1), and 99 % of the samples
    within 1e-5 of the output scale."""
    ref, c = om.forward(P, x, emulate=True)
    scale = max(np.sqrt(np.mean(ref ** 2)), 1e-30)
    w3 = np.abs(c["W3r"])
    flips = 2.0 ** -8 * (np.abs(c["a2"]) @ w3 + np.abs(c["a1"]) @ (np.abs(c["W2r"]).T @ w3))
    err = np.abs(got - ref)
    assert (err <= 1e-5 * scale + flips).all(), f"{label}: {np.max(err / (1e-5 * scale + flips)):.3g}"
    close = np.mean(err <= 1e-5 * np.maximum(np.abs(ref), scale))
    assert close >= 0.99, f"{label}: {close:.4f} of the samples within 1e-5"


@pytest.mark.parametrize("n", [1, 31, 4097])
def test_forward_matches_oracle(n):
    ss = inputs.seed_samples(n, seed=43)
    x, _ = _prepare(ss)
    m = fit.fit_mlp_create(0, seed=9)
    try:
        P = fit.fit_mlp_get_params(m).astype(np.float64)
        _close_net(_forward(m, x), P, x.cpu().numpy(), "forward")
    finally:
        fit.fit_mlp_destroy(m)


def test_gradient_matches_oracle():
    n = 4099  # several blocks of 64 and a ragged one
    ss = inputs.seed_samples(n, seed=45)
    h, _ = oracle.path_lengths(0, ss.B, ss.R.astype(np.float64), ss.q, ss.par.astype(np.float64))
    x, t = _prepare(ss, h)
    t[::97] = float("nan")  # samples without a target take no part
    m = fit.fit_mlp_create(0, seed=10)
    try:
        P = fit.fit_mlp_get_params(m).astype(np.float64)
        grad = torch.empty(fit.FIT_MLP_PARAMS, device="cuda")
        loss = torch.empty(1, device="cuda")
        fit.fit_mlp_gradient(m, x, t, grad, loss)
        L, G = om.loss_grad(P, x.cpu().numpy(), t.cpu().numpy(), emulate=True)
        g = grad.cpu().numpy()
        assert abs(float(loss.item()) - L) <= 1e-5 * L
        for name, a, b in (("W1", om.OFF_W1, om.OFF_B1), ("b1", om.OFF_B1, om.OFF_W2),
                           ("W2", om.OFF_W2, om.OFF_B2), ("b2", om.OFF_B2, om.OFF_W3),
                           ("W3", om.OFF_W3, om.OFF_B3), ("b3", om.OFF_B3, om.N_PARAMS)):
            err = np.linalg.norm(g[a:b] - G[a:b]) / np.linalg.norm(G[a:b])
            assert err <= 1e-3, (name, err)
    finally:
        fit.fit_mlp_destroy(m)


def test_adam_steps_match_oracle():
    m = fit.fit_mlp_create(0, seed=11)
    try:
        P0 = fit.fit_mlp_get_params(m).astype(np.float64)
        rng = np.random.default_rng(5)
        P, mo, vo = P0.copy(), np.zeros_like(P0), np.zeros_like(P0)
        for k in range(1, 4):
            g = (rng.standard_normal(fit.FIT_MLP_PARAMS) * 10.0 ** rng.uniform(-4, 0, fit.FIT_MLP_PARAMS))
            g = g.astype(np.float32)
            fit.fit_mlp_adam_step(m, torch.from_numpy(g).cuda(), 1e-3)
            P, mo, vo = om.adam(P, mo, vo, g.astype(np.float64), k, 1e-3)
        got = fit.fit_mlp_get_params(m).astype(np.float64)
        # FP32 parameters: the update to 1e-4 relative plus a few FP32 units of P
        assert (np.abs((got - P0) - (P - P0)) <= 1e-4 * np.abs(P - P0) + 4 * 2.0 ** -24 * np.abs(P0)
                ).all()
        # the forward image follows the parameters
        ss = inputs.seed_samples(257, seed=47)
        x, _ = _prepare(ss)
        _close_net(_forward(m, x), got, x.cpu().numpy(), "forward after Adam")
    finally:
        fit.fit_mlp_destroy(m)


def test_training_learns_the_path_length(trained):
    m, curve = trained
    assert np.all(np.isfinite(curve)) and curve[-1] < 0.05 * curve[0]
    ss = inputs.seed_samples(200_000, seed=400)
    h, _ = oracle.path_lengths(0, ss.B, ss.R.astype(np.float64), ss.q, ss.par.astype(np.float64))
    x, t = _prepare(ss, h)
    y = _forward(m, x)
    # the GPU forward of the trained weights is the reference's
    P = fit.fit_mlp_get_params(m).astype(np.float64)
    _close_net(y, P, x.cpu().numpy(), "trained forward")
    # held-out accuracy: the seed's error in units of the iteration tolerance
    err = np.abs(om.seed(ss.B, ss.par, ss.q, ss.R, y) - h) / (TOL * ss.R)
    line = np.abs(om.line_distance(ss.par, ss.R) - h) / (TOL * ss.R)
    print(f"\nheld-out seed error / tol: median {np.median(err):.3f}, within tol "
          f"{np.mean(err <= 1):.3f} (straight line: median {np.median(line):.1f}, within tol "
          f"{np.mean(line <= 1):.4f})")
    assert np.mean(err <= 1) >= 0.8 and np.median(err) < 0.02 * np.median(line)


def _geom():
    # The network replaces the straight-line start of the iteration, so the
    # plain fits it is compared with start there too.
    return fit.Geometry(inputs.B_FIELD, inputs.surfaces(inputs.MODE_R), tol=TOL,
                        start=fit.FIT_START_LINE)


def test_path_lengths_match_oracle_with_and_without_seed(trained):
    m, _ = trained
    f = fit.Fitter(_geom(), None)
    try:
        fit.fit_mlp_attach(f.h, m)
        ss = inputs.seed_samples(100_001, seed=401)
        par, q, R = _dev_samples(ss)
        h_ref, _ = oracle.path_lengths(0, ss.B, ss.R.astype(np.float64), ss.q,
                                       ss.par.astype(np.float64))
        its = {}
        for seeded in (False, True):
            h = torch.empty(ss.n, device="cuda")
            it = torch.empty(ss.n, dtype=torch.int32, device="cuda")
            fit.fit_path_lengths(f.h, par, q, R, h, it, seeded=seeded)
            hv = h.cpu().numpy()
            assert (np.abs(hv - h_ref) <= TOL * ss.R + 4 * 2.0 ** -24 * h_ref).all()
            its[seeded] = it.cpu().numpy()
        print(f"\nmean iterations: straight-line seed {its[False].mean():.4f}, "
              f"network seed {its[True].mean():.4f}; one iteration: "
              f"{np.mean(its[False] == 1):.4f} vs {np.mean(its[True] == 1):.4f}")
        assert its[True].mean() < its[False].mean() - 0.3
        assert its[True].max() <= its[False].max()
    finally:
        f.close()


@pytest.mark.parametrize("n", [1024, 1000, 4097])
def test_seeded_fit_matches_oracle(trained, n):
    m, _ = trained
    ts = inputs.generate(inputs.MODE_R, n, seed=1)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(_geom(), None)
    try:
        plain = f.run(*d, [n], [0], layers=True)
        st_plain = f.sync()
        fit.fit_mlp_attach(f.h, m)
        seeded = f.run(*d, [n], [0], layers=True)
        st_seed = f.sync()
        ref = oracle.fit_set(ts)
        got = {k: v.cpu().numpy()[..., :n] for k, v in seeded.items() if v is not None}
        parity.check(got, ref, f"seeded fit n={n}")
        assert (got["status"] == 0).all()
        assert st_seed["tracks"] == n and st_seed["not_converged"] == 0
        assert st_seed["iterations"] < st_plain["iterations"]
    finally:
        f.close()


def test_untrained_seed_is_corrected_by_the_iteration():
    """Random weights: the iteration still lands on the oracle's answer, and
    detaching restores the straight-line seed."""
    m = fit.fit_mlp_create(0, seed=12)
    n = 2000
    ts = inputs.generate(inputs.MODE_R, n, seed=13)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(_geom(), None)
    try:
        fit.fit_mlp_attach(f.h, m)
        out = f.run(*d, [n], [0])
        st = f.sync()
        got = {k: v.cpu().numpy()[..., :n] for k, v in out.items() if v is not None}
        parity.check(got, oracle.fit_set(ts), "untrained seed")
        assert st["not_converged"] == 0
        fit.fit_mlp_attach(f.h, None)
        with pytest.raises(fit.FitError):
            fit.fit_path_lengths(f.h, d[0], d[2], torch.full((n,), 50.0, device="cuda"),
                                 torch.empty(n, device="cuda"), seeded=True)
    finally:
        f.close()
        fit.fit_mlp_destroy(m)


def test_stopped_tracks_with_the_seed(trained):
    """Tracks that cannot reach the outer cylinders stop with the same status
    and chi2 bookkeeping as without the seed."""
    m, _ = trained
    surf = inputs.surfaces(inputs.MODE_R)
    n = 96
    gap = float(surf[1] - surf[0])
    pt = np.where(np.arange(n) % 3 == 0, np.linspace(0.8, 8.0, n),
                  (surf[12].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2)
    ts = inputs.generate(inputs.MODE_R, n, seed=71, pt=pt)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(_geom(), None)
    try:
        plain = f.run(*d, [n], [0], layers=True)
        f.sync()
        fit.fit_mlp_attach(f.h, m)
        seeded = f.run(*d, [n], [0], layers=True)
        st = f.sync()
        a = {k: v.cpu().numpy()[..., :n] for k, v in plain.items() if v is not None}
        b = {k: v.cpu().numpy()[..., :n] for k, v in seeded.items() if v is not None}
        assert np.array_equal(a["status"], b["status"])
        assert st["no_intersection"] == int(np.sum(b["status"] & 1))
        stopped = (b["status"] & 1) != 0
        assert (b["chi2_layer"][13:, stopped] == 0).all()
        parity.check(b, oracle.fit_set(ts), "seeded fit with stopped tracks")
    finally:
        f.close()


def test_seed_gain(trained):
    """What the trained network gains: p2r fit of 100k tracks x 20 layers,
    iterations per track-layer and kernel time with the straight-line seed
    (the packed two-tracks-per-thread kernel) and with the network (one track
    per thread, the network on the tensor cores before every layer).  Reports
    both; asserts only that the iterations fall."""
    m, _ = trained
    n = 100_000
    ts = inputs.generate(inputs.MODE_R, n, seed=3)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(_geom(), None)
    res = {}
    try:
        out = f.outputs(n, ld=ld)
        for label, net in (("straight line", None), ("network", m)):
            fit.fit_mlp_attach(f.h, net)
            for _ in range(3):
                f.run(*d, [n], [0], out=out)
            f.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                f.run(*d, [n], [0], out=out)
            e1.record()
            st = f.sync()
            res[label] = (st["iterations"] / (10 * n * 20), e0.elapsed_time(e1) / 10)
        print("\n" + "; ".join(f"{k}: {v[0]:.4f} iterations per track-layer, {v[1]:.3f} ms"
                               for k, v in res.items()))
        assert res["network"][0] < res["straight line"][0]
    finally:
        f.close()


def test_argument_errors():
    m = fit.fit_mlp_create(0, seed=1)
    try:
        x = torch.zeros((100, 8), device="cuda")
        t = torch.zeros(100, device="cuda")
        with pytest.raises(fit.FitError) as e:
            fit.fit_mlp_train(m, x, t, epochs=1, batch=32)
        assert e.value.code == fit.FIT_ERR_ARG
        with pytest.raises(fit.FitError):
            fit.fit_mlp_train(m, x, t, epochs=1, batch=128)  # n < batch
        big = torch.zeros((65537, 8), device="cuda")
        with pytest.raises(fit.FitError):
            fit.fit_mlp_gradient(m, big, torch.zeros(65537, device="cuda"),
                                 torch.empty(fit.FIT_MLP_PARAMS, device="cuda"),
                                 torch.empty(1, device="cuda"))
        with pytest.raises(ValueError):
            fit.fit_mlp_set_params(m, np.zeros(10))
    finally:
        fit.fit_mlp_destroy(m)


def test_full_size_seeded_fit_sampled(trained):
    """The learned seed's workload at its full size (1M p2r tracks x 20
    layers, seed 4): the seeded fit against the oracle on sampled tracks."""
    m, _ = trained
    n = 1_000_000
    ts = inputs.generate(inputs.MODE_R, n, seed=4)
    ld = gpu_util.pad_ld(n)
    d = [gpu_util.to_dev(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(_geom(), None)
    try:
        fit.fit_mlp_attach(f.h, m)
        out = f.run(*d, [n], [0])
        st = f.sync()
        assert st["tracks"] == n and st["no_intersection"] == 0 and st["nonfinite"] == 0
        assert st["not_converged"] == 0 and st["iterations"] < 1.2 * n * 20
        got = {k: v.cpu().numpy()[..., :n] for k, v in out.items() if v is not None}
        assert (got["status"] == 0).all()
        idx = np.unique(np.concatenate([[0, n - 1],
                                        np.random.default_rng(2).choice(n, 3000, replace=False)]))
        parity.check({k: v[..., idx] for k, v in got.items()}, oracle.fit_set(ts.subset(idx)),
                     "full-size seeded fit")
    finally:
        f.close()
