"""Pins of the FP64 reference of the learned path-length seed (oracle/mlp.py)
to things other than itself: torch's own BF16 conversion, central finite
differences, torch autograd, torch.optim.Adam, the circle geometry, and
invariances of the inputs.  Each pin_* takes the reference module, so that
tests/test_oracle_mlp.py can run them on oracle/mlp.py and on copies with
planted mistakes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_09228_gb300 import inputs


def _params(om, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    P = np.zeros(om.N_PARAMS)
    P[om.OFF_W1:om.OFF_B1] = rng.uniform(-1, 1, 512) * np.sqrt(6 / 8)
    P[om.OFF_B1:om.OFF_W2] = rng.uniform(-0.1, 0.1, 64)
    P[om.OFF_W2:om.OFF_B2] = rng.uniform(-1, 1, 4096) * np.sqrt(6 / 64)
    P[om.OFF_B2:om.OFF_W3] = rng.uniform(-0.1, 0.1, 64)
    P[om.OFF_W3:om.OFF_B3] = rng.uniform(-1, 1, 64) * np.sqrt(6 / 64)
    P[om.OFF_B3] = 0.05
    return (P * scale).astype(np.float32).astype(np.float64)


def _inputs(om, n, seed):
    ss = inputs.seed_samples(n, seed)
    return ss, om.features(ss.B, ss.par, ss.q, ss.R).astype(np.float32)


def pin_bf16_matches_torch_and_rounds_ties_to_even(om):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, -2.5, 3.0e38, 1e-40]]).astype(np.float32)
    # exact ties: a BF16 value plus half a BF16 unit in the last place
    base = rng.standard_normal(1000).astype(np.float32)
    bb = base.view(np.uint32) & np.uint32(0xFFFF0000)
    ties = (bb | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(om.bf16(x), ref)
    # a tie goes to the neighbour with an even last bit
    got = om.bf16(ties).astype(np.float32).view(np.uint32)
    assert ((got >> 16) & 1 == 0).all()


def pin_exact_gradient_matches_central_differences(om):
    P = _params(om, 3)
    _, X = _inputs(om, 40, 5)
    t = np.random.default_rng(2).standard_normal(40) * 0.3
    t[7] = np.nan  # a sample without a target takes no part
    L, g = om.loss_grad(P, X, t, emulate=False)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False) for a, b in
                          [(0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4800)]] + [[4800]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(P[i]))
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (om.loss_grad(Pp, X, t, emulate=False)[0] - om.loss_grad(Pm, X, t, emulate=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])


def _torch_net(om, P, X, t, emulate):
    W1, b1, W2, b2, W3, b3 = [torch.tensor(np.array(a), dtype=torch.float64, requires_grad=True)
                              for a in om.unpack(P)]

    def rnd(v):  # BF16 rounding with the gradient passed through
        if not emulate:
            return v
        r = v.detach().to(torch.float32).to(torch.bfloat16).to(torch.float64)
        return v + (r - v).detach()

    x = torch.tensor(X, dtype=torch.float64)
    if emulate:
        hi = x.to(torch.float32).to(torch.bfloat16).to(torch.float64)
        lo = (x.to(torch.float32) - hi.to(torch.float32)).to(torch.bfloat16).to(torch.float64)
        x = hi + lo
    z1 = x @ rnd(W1).T + b1
    a1 = rnd(torch.relu(z1))
    z2 = a1 @ rnd(W2).T + b2
    a2 = rnd(torch.relu(z2))
    y = a2 @ rnd(W3) + b3
    tt = torch.tensor(t, dtype=torch.float64)
    ok = torch.isfinite(tt)
    L = ((y - torch.where(ok, tt, 0.0)) ** 2 * ok).sum() / len(t)
    L.backward()
    g = om.pack(*[a.grad.numpy() for a in (W1, b1, W2, b2, W3, b3)])
    return y.detach().numpy(), float(L.detach()), g


def _forward_and_gradient_match_torch_autograd(om, emulate):
    """torch autograd of the same network; with emulate the BF16 roundings are
    straight-through in torch.  torch does not round the backward error
    signals, so with emulate the gradients of W1, b1 and W2 (downstream of the
    rounded layer-2 signal) agree to that rounding (2^-8 relative each), those
    of b2, W3 and b3 exactly."""
    P = _params(om, 7)
    _, X = _inputs(om, 300, 9)
    t = np.random.default_rng(3).standard_normal(300) * 0.2
    y, c = om.forward(P, X, emulate)
    L, g = om.loss_grad(P, X, t, emulate)
    ty, tL, tg = _torch_net(om, P, X, t, emulate)
    assert np.allclose(y, ty, rtol=1e-12, atol=1e-12)
    assert abs(L - tL) <= 1e-12 * tL
    exact = np.ones(om.N_PARAMS, bool)
    if emulate:
        exact[om.OFF_W1:om.OFF_B2] = False
    assert np.allclose(g[exact], tg[exact], rtol=1e-10, atol=1e-13)
    if emulate:
        for a, b in ((om.OFF_W1, om.OFF_B1), (om.OFF_B1, om.OFF_W2), (om.OFF_W2, om.OFF_B2)):
            assert np.linalg.norm(g[a:b] - tg[a:b]) <= 4e-3 * np.linalg.norm(tg[a:b])
    else:
        assert np.allclose(g, tg, rtol=1e-10, atol=1e-13)


def pin_adam_matches_torch_optim(om):
    P = _params(om, 11)
    rng = np.random.default_rng(12)
    grads = [rng.standard_normal(om.N_PARAMS) * 10.0 ** rng.uniform(-4, 0, om.N_PARAMS)
             for _ in range(4)]
    p = torch.tensor(P, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.8, 0.99), eps=1e-7)
    mine, m, v = P.copy(), np.zeros_like(P), np.zeros_like(P)
    for k, gk in enumerate(grads, start=1):
        opt.zero_grad()
        p.grad = torch.tensor(gk)
        opt.step()
        mine, m, v = om.adam(mine, m, v, gk, k, 3e-3, 0.8, 0.99, 1e-7)
    assert np.allclose(mine, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def pin_inputs_are_rotation_invariant_and_exact_at_special_states(om):
    ss = inputs.seed_samples(500, 21)
    X = om.features(ss.B, ss.par, ss.q, ss.R)
    a = 0.7
    rot = ss.par.astype(np.float64).copy()
    rot[0] = np.cos(a) * ss.par[0] - np.sin(a) * ss.par[1]
    rot[1] = np.sin(a) * ss.par[0] + np.cos(a) * ss.par[1]
    rot[4] = ss.par[4].astype(np.float64) + a
    assert np.allclose(om.features(ss.B, rot, ss.q, ss.R), X, atol=1e-12)
    # a track at (r0, 0) heading along +x: psi = 0, the line reaches R after R - r0
    p = np.array([[30.0], [0.0], [5.0], [0.5], [0.0], [1.0]])
    x = om.features(3.8, p, [1], [50.0])[0]
    assert np.allclose(x, [0.6, 0.1, 0.5 * om.KA * 3.8 * 0.5 * 50.0, 1.0, 0.0, np.cos(1.0), 1.0,
                           0.5])
    assert om.line_distance(p, [50.0])[0] == pytest.approx(20.0, abs=1e-12)
    # heading along +y from (r0, 0): psi = pi/2, the line reaches R after sqrt(R^2 - r0^2)
    p[4] = np.pi / 2
    assert om.features(3.8, p, [1], [50.0])[0][4] == pytest.approx(1.0, abs=1e-15)
    assert om.line_distance(p, [50.0])[0] == pytest.approx(40.0, abs=1e-12)


def pin_target_against_the_circle_through_the_origin(om):
    """From the origin, the exact transverse path to radius R is
    2 rho asin(R / 2 rho) and the straight line's is R, so
    g = (2 rho asin(R / 2 rho) - R) / (kappa R^2 / 2); the oracle's exact path
    length gives the same g, and seed() maps g back to that path length."""
    B, R = 3.8, np.array([10.0, 50.0, 100.0])
    for q in (-1, 1):
        w = np.array([1.0, 0.5, 0.9])
        rho = 1.0 / (om.KA * B * w)
        par = np.stack([np.zeros(3), np.zeros(3), np.zeros(3), w, np.full(3, 0.3), np.full(3, 1.2)])
        h_true = 2 * rho * np.arcsin(R / (2 * rho))
        kappa = -q * om.KA * B * w
        g_true = (h_true - R) / (0.5 * kappa * R * R)
        h_orc, st = oracle.path_lengths(0, B, R, np.full(3, q, np.int32), par)
        assert (st == 0).all()
        g = om.target(B, par, np.full(3, q), R, h_orc)
        assert np.allclose(g, g_true, rtol=1e-9)
        assert np.allclose(om.seed(B, par, np.full(3, q), R, g), h_true, rtol=1e-12)
    # no curvature: no target
    assert np.isnan(om.target(0.0, par, np.full(3, 1), R, R)).all()


def pin_forward_and_gradient_exact(om):
    _forward_and_gradient_match_torch_autograd(om, False)


def pin_forward_and_gradient_bf16(om):
    _forward_and_gradient_match_torch_autograd(om, True)


ALL_PINS = [pin_bf16_matches_torch_and_rounds_ties_to_even,
            pin_exact_gradient_matches_central_differences, pin_forward_and_gradient_exact,
            pin_forward_and_gradient_bf16, pin_adam_matches_torch_optim,
            pin_inputs_are_rotation_invariant_and_exact_at_special_states,
            pin_target_against_the_circle_through_the_origin]
