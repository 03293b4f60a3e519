"""The algebra behind the fused kernel's local covariance form, checked in
FP64 against the oracle (no GPU).

The kernel carries the p2r covariance between cylinders as the 5x5
covariance c of (l, z, w, phi, theta), l the position along the direction
normal to the null vector (bc, bs) of the 6x6 covariance, and transports it
with J_l = A_l + v_l g_l^T (A_l = P' A B, v_l = P' v, g_l = B^T g) instead of
J C J^T; it enters that form through a zero-length propagation to a surface
through the start point.  These tests write that derivation out in numpy
and compare it with the oracle's Jacobian and update: they pin the reading,
not the CUDA code (the GPU parity tests compare the kernel with the oracle).
"""
import numpy as np
import pytest

import oracle as O

KA, B = 0.00299792458, 3.8


def _basis(bc, bs):
    """6x5 B: l along (-bs, bc); z, w, phi, theta unchanged."""
    Bm = np.zeros((6, 5))
    Bm[0, 0], Bm[1, 0] = -bs, bc
    for k in range(1, 5):
        Bm[k + 1, k] = 1.0
    return Bm


def _helix_factors(p, q, h):
    """A (fixed-h derivative), v = dp'/dh and g = grad h of the propagation to
    the cylinder through the point at path length h (the kernel's factors)."""
    x, y, z, w, ph, th = p
    dkdw = -q * KA * B
    kap = dkdw * w
    u = 0.5 * kap * h
    s = np.sin(u) / u
    cu = np.cos(u)
    sp = (cu - s) / u
    cm, sm = np.cos(ph + u), np.sin(ph + u)
    px, py = x + h * s * cm, y + h * s * sm
    c1, s1 = np.cos(ph + 2 * u), np.sin(ph + 2 * u)
    isth = 1 / np.sin(th)
    cot = np.cos(th) * isth
    hh = 0.5 * h * h * dkdw
    Xw, Yw = hh * (sp * cm - s * sm), hh * (sp * sm + s * cm)
    dx, dy = px - x, py - y
    iD = 1 / (px * c1 + py * s1)
    A = np.eye(6)
    A[0, 3], A[0, 4], A[1, 3], A[1, 4], A[2, 5], A[4, 3] = Xw, -dy, Yw, dx, -h * isth**2, h * dkdw
    v = np.array([c1, s1, cot, 0, kap, 0])
    g = np.array([-px * iD, -py * iD, 0, -(px * Xw + py * Yw) * iD, (px * dy - py * dx) * iD, 0])
    return A, v, g, (px, py)


def _rand_state(rng, R1):
    q = int(rng.choice([-1, 1]))
    w = 1 / rng.uniform(0.7, 10)
    Phi = rng.uniform(0, 2 * np.pi)
    bc, bs = np.cos(Phi), np.sin(Phi)
    dl = rng.normal(0, 0.01)  # an update moves the point along the surface
    p = np.array([R1 * bc - bs * dl, R1 * bs + bc * dl, rng.normal(0, 5), w,
                  Phi + rng.uniform(-0.3, 0.3), rng.uniform(0.8, 2.3)])
    M = rng.normal(size=(5, 5))
    sc = np.array([1e-2, 1e-1, 1e-2 * w, 1e-2, 1e-2])
    c = (M @ M.T) * np.outer(sc, sc)
    return q, p, bc, bs, c


def test_local_transport_is_the_projected_J_C_JT():
    rng = np.random.default_rng(11)
    orc = O.default()
    for _ in range(60):
        R1 = rng.uniform(4, 60)
        R2 = R1 + rng.uniform(5, 40)
        q, p, bc, bs, c = _rand_state(rng, R1)
        st, pout, J, h = orc.transport(0, B, R2, q, p)
        assert st == 0
        A, v, g, (px, py) = _helix_factors(p, q, h)
        assert np.allclose(A + np.outer(v, g), J, rtol=0, atol=1e-12 * np.abs(J).max())
        Bm = _basis(bc, bs)
        C6 = Bm @ c @ Bm.T
        ref = J @ C6 @ J.T
        r = np.hypot(px, py)
        c2, s2 = px / r, py / r
        B2 = _basis(c2, s2)
        # J_l = P' (A + v g^T) B with P' = B2^T, in the sparse form the kernel uses
        Al = np.eye(5)
        Al[0, 0] = s2 * bs + c2 * bc
        Al[0, 2] = -s2 * A[0, 3] + c2 * A[1, 3]
        Al[0, 3] = -s2 * A[0, 4] + c2 * A[1, 4]
        Al[1, 4], Al[3, 2] = A[2, 5], A[4, 3]
        vl = np.array([-s2 * v[0] + c2 * v[1], v[2], 0, v[4], 0])
        gl = np.array([-bs * g[0] + bc * g[1], 0, g[3], g[4], 0])
        assert np.allclose(Al + np.outer(vl, gl), B2.T @ J @ Bm, atol=1e-12)
        Jl = Al + np.outer(vl, gl)
        cl = Jl @ c @ Jl.T
        # the 6x6 result has no component along the new normal: B2 cl B2^T is all of it
        err = np.abs(B2 @ cl @ B2.T - ref).max() / np.abs(ref).max()
        assert err < 1e-12, err


def test_local_update_is_the_kalman_update():
    rng = np.random.default_rng(12)
    orc = O.default()
    for _ in range(60):
        R = rng.uniform(4, 110)
        q, p, bc, bs, c = _rand_state(rng, R)
        p = np.array([R * bc, R * bs, *p[2:]])  # on the cylinder, the basis its azimuth
        Bm = _basis(bc, bs)
        C6 = Bm @ c @ Bm.T
        phih = np.arctan2(bs, bc) + rng.normal(0, 0.01 / R)
        m = np.array([R * np.cos(phih), R * np.sin(phih), p[2] + rng.normal(0, 0.1)])
        t = np.array([-np.sin(phih), np.cos(phih), 0.0])
        V = 1e-4 * np.outer(t, t) + 1e-2 * np.outer([0, 0, 1.0], [0, 0, 1.0])
        v6 = np.array([V[0, 0], V[1, 0], V[1, 1], V[2, 0], V[2, 1], V[2, 2]])
        st, po, co, qo, chi = orc.update(0, q, p, O.pack_sym6(C6), m, v6)
        # the update on the local form: H_l = (chp e_l, e_z), chp = t_h . (-bs, bc)
        chp = np.sin(phih) * bs + np.cos(phih) * bc
        Hl = np.zeros((2, 5))
        Hl[0, 0], Hl[1, 1] = chp, 1.0
        S = Hl @ c @ Hl.T + np.array([[t @ V @ t, t @ V[:, 2]], [t @ V[:, 2], V[2, 2]]])
        r = np.array([t[:2] @ (m[:2] - p[:2]), m[2] - p[2]])
        K = c @ Hl.T @ np.linalg.inv(S)
        cl = c - K @ S @ K.T
        dl = K @ r
        pn = p.copy()
        pn[0] -= bs * dl[0]
        pn[1] += bc * dl[0]
        pn[2:] += dl[1:]
        pn[4] = (pn[4] + np.pi) % (2 * np.pi) - np.pi
        C6n = O.unpack_sym6(co)
        assert np.abs(Bm @ cl @ Bm.T - C6n).max() < 1e-10 * np.abs(C6n).max()
        d = pn - po
        d[4] = (d[4] + np.pi) % (2 * np.pi) - np.pi
        assert np.abs(d).max() < 1e-12 * 100
        assert abs(r @ np.linalg.solve(S, r) - chi) < 1e-10 * max(chi, 1.0)


@pytest.mark.parametrize("mode", [0, 1], ids=["p2r-line", "p2z-plane"])
def test_start_projection_leaves_the_first_transport_unchanged(mode):
    """J (J0 C J0^T) J^T = J C J^T, J0 the zero-length propagation to the
    surface through the start point."""
    rng = np.random.default_rng(13 + mode)
    orc = O.default()
    for _ in range(100):
        q = int(rng.choice([-1, 1]))
        w = 1 / rng.uniform(0.7, 10)
        th = rng.uniform(0.8, 2.3) if mode == 0 else rng.uniform(0.16, 0.44)
        p = np.array([rng.normal(0, .01), rng.normal(0, .01), rng.normal(0, .1), w,
                      rng.uniform(-np.pi, np.pi), th])
        M = rng.normal(size=(6, 6))
        C = M @ M.T * 1e-4
        st, pout, J, h = orc.transport(mode, B, 4.0 if mode == 0 else 10.0, q, p)
        assert st == 0
        ref = J @ C @ J.T
        kap = -q * KA * B * w
        cp, sp = np.cos(p[4]), np.sin(p[4])
        cot = np.cos(th) / np.sin(th)
        if mode == 1:  # the plane z = z0: g = -tan(theta) e_z, z row of J0 zero
            g = np.array([0, 0, -np.tan(th), 0, 0, 0])
        else:  # the line (x - x0) cos(phi) + (y - y0) sin(phi) = 0
            g = np.array([-cp, -sp, 0, 0, 0, 0])
        v = np.array([cp, sp, cot, 0, kap, 0])
        J0 = np.eye(6) + np.outer(v, g)
        C0 = J0 @ C @ J0.T
        if mode == 1:
            assert np.abs(J0[2]).max() < 1e-15  # 1 - cot tan = 0
        else:
            assert np.abs(C0 @ np.array([cp, sp, 0, 0, 0, 0])).max() < 1e-15 * np.abs(C0).max() * 10
        err = np.abs(J @ C0 @ J.T - ref).max() / np.abs(ref).max()
        assert err < 1e-13, err


def test_first_order_step_root_near_the_circle():
    """The p2r step takes the first-order root -c2 / (2 b) of
    d^2 + 2 b d + c2 = 0 when |c2| <= 1e-4 b^2: within 2.5e-5 of the exact
    nearer root, which is itself below 5e-5 |b| (reading R4)."""
    rng = np.random.default_rng(14)
    b = rng.uniform(0.1, 120.0, 20000) * rng.choice([-1, 1], 20000)
    c2 = rng.uniform(-1e-4, 1e-4, 20000) * b * b
    exact = -c2 / (b + np.copysign(np.sqrt(b * b - c2), b))
    first = -0.5 * c2 / b
    rel = np.abs(first - exact) / np.maximum(np.abs(exact), 1e-300)
    assert rel.max() <= 2.51e-5
    assert (np.abs(exact) <= 5.0001e-5 * np.abs(b)).all()
