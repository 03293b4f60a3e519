"""Pins of the FP64 oracle to facts outside it.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError
when the oracle disagrees with something the physics or mathematics fixes:

* the Lorentz-force equation of motion, integrated here by RK4 (helix);
* the helix as a rotation about its centre, written here independently;
* straight-line closed forms (B = 0 or w -> 0): line-plane, line-cylinder;
* brute-force scan + bisection of r(h) = R (first crossing of a cylinder),
  and its closed form through the tangent of half the turning angle;
* central finite differences (transport Jacobian, chi2 gradient);
* Kalman limits: infinite hit error changes nothing, zero hit error snaps the
  measured coordinates onto the hit; the information form
  (C^-1 + H^T V^-1 H)^-1; the chi2 split into filtered residual and state
  change; C - C+ positive semi-definite;
* the whole filter on generated tracks: chi2 per layer ~ chi2(2) and pulls
  ~ N(0, 1) (the generator's noise model is the filter's measurement model);
* track finding: the composition of the pinned single steps with the argmin
  over candidates written out here; one candidate without a gate is the plain
  fit; nothing under the gate is pure propagation.

tests/test_oracle.py runs every pin on the oracle; tests/test_oracle_mutants.py
plants mistakes in copies of oracle.cpp and checks that some pin fails.
"""
from __future__ import annotations

import numpy as np

from paper_2409_09228_gb300 import inputs as gen

KA = 0.00299792458  # GeV / (T cm), speed of light / 1e9 in cm/ns units
B = float(np.float32(3.8))
MODE_R, MODE_Z = 0, 1


def _states(rng, n, mode):
    """Random track states inside the tracker, charges, and a target surface."""
    out = []
    for _ in range(n):
        pt = rng.uniform(0.8, 10.0)
        q = int(rng.choice([-1, 1]))
        phi = rng.uniform(-np.pi, np.pi)
        if mode == MODE_R:
            theta = 2 * np.arctan(np.exp(-rng.uniform(-1, 1)))
            r0 = rng.uniform(0, 30)
            a0 = rng.uniform(-np.pi, np.pi)
            p = np.array([r0 * np.cos(a0), r0 * np.sin(a0), rng.uniform(-20, 20), 1 / pt, phi, theta])
            # launch outwards so that the cylinder is reached
            p[4] = a0 + rng.uniform(-0.6, 0.6)
            target = r0 + rng.uniform(5, 60)
        else:
            theta = 2 * np.arctan(np.exp(-rng.uniform(1.5, 2.5)))
            p = np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), rng.uniform(0, 50), 1 / pt,
                          phi, theta])
            target = p[2] + rng.uniform(5, 150)
        out.append((p, q, target))
    return out


def ref_helix(p, q, Bz, h):
    """Helix as a rotation of the transverse position about the track centre.

    The Lorentz force q v x B with B along +z bends a positive track clockwise
    (seen from +z): the centre lies at P + q rho (sin phi, -cos phi) and the
    position rotates by -q h / rho after transverse path h.
    """
    x, y, z, w, phi, theta = p
    if Bz == 0.0 or w == 0.0:
        return np.array([x + h * np.cos(phi), y + h * np.sin(phi), z + h / np.tan(theta), w, phi, theta])
    rho = 1.0 / (KA * Bz * w)
    cx, cy = x + q * rho * np.sin(phi), y - q * rho * np.cos(phi)
    a = -q * h / rho
    dx, dy = x - cx, y - cy
    return np.array([cx + np.cos(a) * dx - np.sin(a) * dy, cy + np.sin(a) * dx + np.cos(a) * dy,
                     z + h / np.tan(theta), w, phi + a, theta])


def _rk4_lorentz(p, q, Bz, s_total, nstep):
    """Integrates dX/ds = T, dT/ds = (q kA B / |p|) T x z_hat over 3-D path s."""
    x, y, z, w, phi, theta = p
    pmag = (1.0 / w) / np.sin(theta)
    k = q * KA * Bz / pmag
    Y = np.array([x, y, z, np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])

    def f(Y):
        T = Y[3:]
        return np.concatenate([T, k * np.array([T[1], -T[0], 0.0])])

    ds = s_total / nstep
    for _ in range(nstep):
        k1 = f(Y)
        k2 = f(Y + 0.5 * ds * k1)
        k3 = f(Y + 0.5 * ds * k2)
        k4 = f(Y + ds * k3)
        Y = Y + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return Y


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def pin_helix_equation_of_motion(orc):
    rng = np.random.default_rng(11)
    for p, q, _ in _states(rng, 12, MODE_R) + _states(rng, 12, MODE_Z):
        h = rng.uniform(1, 80)
        got = orc.helix(B, q, p, h)
        s = h / np.sin(p[5])
        Y = _rk4_lorentz(p, q, B, s, 4000)
        assert np.allclose(got[:3], Y[:3], rtol=0, atol=1e-8), (got[:3], Y[:3])
        phi_dir = np.arctan2(Y[4], Y[3])
        assert abs(_wrap(got[4] - phi_dir)) < 1e-9
        assert got[3] == p[3] and got[5] == p[5]


def pin_helix_geometry(orc):
    rng = np.random.default_rng(12)
    for p, q, _ in _states(rng, 20, MODE_R):
        for h in (0.0, 1e-3, 3.0, 47.0, 260.0):
            got = orc.helix(B, q, p, h)
            ref = ref_helix(p, q, B, h)
            assert np.allclose(got[:3], ref[:3], rtol=0, atol=1e-9), (h, got, ref)
            assert abs(got[4] - ref[4]) < 1e-12
    # straight line limit at B = 0 and at vanishing curvature
    for p, q, _ in _states(rng, 10, MODE_Z):
        for Bz, w in ((0.0, p[3]), (B, 1e-12)):
            pp = p.copy()
            pp[3] = w
            got = orc.helix(Bz, q, pp, 25.0)
            ref = ref_helix(pp, q, 0.0, 25.0)
            assert np.allclose(got[:3], ref[:3], rtol=0, atol=1e-9)


def pin_straight_line_surfaces(orc):
    rng = np.random.default_rng(13)
    for Bz, wscale in ((0.0, 1.0), (B, 1e-11)):
        for p, q, Z in _states(rng, 10, MODE_Z):
            p = p.copy()
            p[3] *= wscale
            st, pout, _, h = orc.transport(MODE_Z, Bz, Z, q, p)
            assert st == 0
            x, y, z, w, phi, th = p
            d = np.array([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
            t = (Z - z) / d[2]  # line-plane intersection, 3-D path t
            exp = np.array([x + t * d[0], y + t * d[1], Z, w, phi, th])
            assert np.allclose(pout, exp, rtol=1e-12, atol=1e-9), (pout, exp)
            assert abs(h - t * np.sin(th)) < 1e-9
        for p, q, R in _states(rng, 10, MODE_R):
            p = p.copy()
            p[3] *= wscale
            st, pout, _, h = orc.transport(MODE_R, Bz, R, q, p)
            assert st == 0
            x, y, z, w, phi, th = p
            d = np.array([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
            # |(x, y) + t d_xy|^2 = R^2, positive root (the start is inside)
            a2 = d[0] ** 2 + d[1] ** 2
            b2 = 2 * (x * d[0] + y * d[1])
            c2 = x * x + y * y - R * R
            t = (-b2 + np.sqrt(b2 * b2 - 4 * a2 * c2)) / (2 * a2)
            exp = np.array([x + t * d[0], y + t * d[1], z + t * d[2], w, phi, th])
            assert np.allclose(pout, exp, rtol=1e-12, atol=1e-9), (pout, exp)


def pin_landing(orc):
    rng = np.random.default_rng(14)
    for p, q, Z in _states(rng, 50, MODE_Z):
        st, pout, _, _ = orc.transport(MODE_Z, B, Z, q, p)
        assert st == 0 and pout[2] == Z
        # and it lies on the track's own helix
        st, h = orc.path_length(MODE_Z, B, Z, q, p)
        assert np.allclose(pout[:2], ref_helix(p, q, B, h)[:2], atol=1e-9)
    for p, q, R in _states(rng, 50, MODE_R):
        st, pout, _, h = orc.transport(MODE_R, B, R, q, p)
        assert st == 0
        assert abs(np.hypot(pout[0], pout[1]) - R) <= 1e-9 * R
        assert np.allclose(pout[:3], ref_helix(p, q, B, h)[:3], atol=1e-9)


def _first_crossing_bruteforce(p, q, R, hmax, nscan=200000):
    hs = np.linspace(0.0, hmax, nscan)
    x, y, z, w, phi, theta = p
    rho = 1.0 / (KA * B * w)
    cx, cy = x + q * rho * np.sin(phi), y - q * rho * np.cos(phi)
    a = -q * hs / rho
    dx, dy = x - cx, y - cy
    px = cx + np.cos(a) * dx - np.sin(a) * dy
    py = cy + np.sin(a) * dx + np.cos(a) * dy
    f = np.hypot(px, py) - R
    idx = np.nonzero((f[:-1] < 0) & (f[1:] >= 0) | (f[:-1] >= 0) & (f[1:] < 0))[0]
    if len(idx) == 0:
        return None
    lo, hi = hs[idx[0]], hs[idx[0] + 1]
    g = lambda h: np.hypot(*ref_helix(p, q, B, h)[:2]) - R  # noqa: E731
    glo = g(lo)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        gm = g(mid)
        if (gm < 0) == (glo < 0):
            lo, glo = mid, gm
        else:
            hi = mid
        if hi - lo < 1e-13:
            break
    return 0.5 * (lo + hi)


def pin_path_r_bruteforce(orc):
    rng = np.random.default_rng(15)
    states = _states(rng, 25, MODE_R)
    # also starts outside the target radius (first crossing on the way in or
    # after a turn) and low-pT tracks that cross after a large turn
    for _ in range(15):
        pt = rng.uniform(0.75, 3)
        a0 = rng.uniform(-np.pi, np.pi)
        r0 = rng.uniform(20, 60)
        p = np.array([r0 * np.cos(a0), r0 * np.sin(a0), 0.0, 1 / pt, rng.uniform(-np.pi, np.pi), 1.2])
        states.append((p, int(rng.choice([-1, 1])), rng.uniform(5, 80)))
    checked = 0
    for p, q, R in states:
        rho = 1.0 / (KA * B * p[3])
        href = _first_crossing_bruteforce(p, q, R, 2 * np.pi * rho * 1.001)
        st, h = orc.path_length(MODE_R, B, R, q, p)
        if href is None:
            assert st != 0, "oracle found a crossing where the scan found none"
            continue
        assert st == 0
        assert abs(h - href) < 1e-7 * max(1.0, href), (h, href)
        checked += 1
    assert checked >= 30


def _first_crossing_half_angle(p, q, R):
    """First forward crossing of r = R in closed form, vectorised over states
    p (6, n): with t = tan(kappa h / 2) the transverse displacement over h is
    the chord 2 sin(kappa h / 2) / kappa at angle phi + kappa h / 2, so
    r(h)^2 = R^2 becomes 2 F t^2 + 2 kappa b0 t + kappa^2 c0 / 2 = 0 with b0,
    t0 the start's components along and across phi, c0 = r0^2 - R^2 and
    F = 1 + kappa (t0 + kappa c0 / 4).  No real root (X = b0^2 - c0 F < 0):
    the circle misses the cylinder (NaN).  Each root gives h = 2 atan(t) /
    kappa modulo a turn; the first crossing is the smaller one in (0, turn]."""
    x, y, w, phi = p[0], p[1], p[3], p[4]
    kap = -q * KA * B * w
    b0 = x * np.cos(phi) + y * np.sin(phi)
    t0 = y * np.cos(phi) - x * np.sin(phi)
    c0 = x * x + y * y - R * R
    F = 1.0 + kap * (t0 + 0.25 * kap * c0)
    X = b0 * b0 - c0 * F
    sq = np.sqrt(np.where(X >= 0, X, 0.0))
    turn = 2 * np.pi / np.abs(kap)
    best = np.full(x.shape, np.inf)
    for sign in (1.0, -1.0):
        hk = 2 * np.arctan2(-0.5 * kap * c0, b0 + sign * sq) / kap
        hk = hk - np.floor(hk / turn) * turn
        hk = np.where(hk > 0, hk, hk + turn)
        best = np.minimum(best, hk)
    return np.where(X >= 0, best, np.nan)


def pin_path_r_half_angle(orc):
    """20k random p2r states (anywhere in r < 250 cm, any direction, pT 0.3-20
    GeV, either charge) to random cylinders: the oracle's path length is the
    half-angle closed form's first crossing, and it reports no intersection
    exactly where the circle misses the cylinder (states whose circle passes
    within 1e-6 R of tangency aside)."""
    rng = np.random.default_rng(23)
    n = 20000
    r0, a0 = rng.uniform(0, 250, n), rng.uniform(-np.pi, np.pi, n)
    p = np.stack([r0 * np.cos(a0), r0 * np.sin(a0), rng.uniform(-50, 50, n),
                  rng.uniform(0.05, 3.3, n), rng.uniform(-np.pi, np.pi, n),
                  rng.uniform(0.5, 2.6, n)])
    q = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int32)
    R = rng.uniform(5, 260, n)
    h_ref, st = orc.path_lengths(MODE_R, B, R, q, p)
    h = _first_crossing_half_angle(p, q, R)
    kap = -q * KA * B * p[3]
    cx, cy = p[0] - np.sin(p[4]) / kap, p[1] + np.cos(p[4]) / kap
    cn, rho = np.hypot(cx, cy), 1 / np.abs(kap)
    clear = np.minimum(np.abs(R - (cn + rho)), np.abs(R - np.abs(cn - rho))) > 1e-6 * R
    reach = st == 0
    assert np.array_equal(reach[clear], np.isfinite(h)[clear])
    both = reach & np.isfinite(h) & clear
    assert both.sum() > 8000 and (~reach & clear).sum() > 4000
    assert (np.abs(h_ref - h)[both] <= 1e-9 * np.maximum(h[both], 1.0)).all()


def _scales(p):
    return np.array([1.0, 1.0, 1.0, p[3], 1.0, 1.0])


def pin_jacobian_fd(orc):
    rng = np.random.default_rng(16)
    for mode in (MODE_R, MODE_Z):
        for p, q, s in _states(rng, 12, mode):
            st, pout, J, _ = orc.transport(mode, B, s, q, p)
            assert st == 0
            sc = _scales(p)
            Jfd = np.zeros((6, 6))
            for j in range(6):
                e = np.zeros(6)
                e[j] = 1e-5 * sc[j]
                s1, pp, _, _ = orc.transport(mode, B, s, q, p + e)
                s2, pm, _, _ = orc.transport(mode, B, s, q, p - e)
                assert s1 == 0 and s2 == 0
                Jfd[:, j] = (pp - pm) / (2 * e[j])
            # compare in the parameters' natural scales
            Jn = J * sc[None, :] / sc[:, None]
            Jfdn = Jfd * sc[None, :] / sc[:, None]
            err = np.abs(Jn - Jfdn).max() / max(1.0, np.abs(Jn).max())
            assert err < 1e-6, (mode, err, J, Jfd)


def _predicted(orc, mode, seed):
    """A propagated state with its covariance, the surface and a nearby hit."""
    ts = gen.generate(mode, 1, seed=seed, nlayer=6)
    p0, c0 = ts.par0[:, 0].astype(np.float64), ts.cov0[:, 0].astype(np.float64)
    q = int(ts.q[0])
    l = 3
    st, pp, cp = orc.propagate(mode, ts.B, float(ts.surf[0]), q, p0, c0)
    assert st == 0
    for k in range(1, l + 1):
        st, pp, cp = orc.propagate(mode, ts.B, float(ts.surf[k]), q, pp, cp)
        assert st == 0
    return pp, cp, q, ts.hpos[l, :, 0].astype(np.float64), ts.hcov[l, :, 0].astype(np.float64), float(ts.surf[l])


def _H(mode, m):
    Hp = np.zeros((2, 3))
    if mode == MODE_Z:
        Hp[0, 0] = Hp[1, 1] = 1.0
    else:
        ph = np.arctan2(m[1], m[0])
        Hp[0, :2] = (-np.sin(ph), np.cos(ph))
        Hp[1, 2] = 1.0
    H = np.zeros((2, 6))
    H[:, :3] = Hp
    return Hp, H


def _sym3(v6):
    return np.array([[v6[0], v6[1], v6[3]], [v6[1], v6[2], v6[4]], [v6[3], v6[4], v6[5]]])


def _sym6(c21):
    M = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            M[i, j] = M[j, i] = c21[k]
            k += 1
    return M


def pin_update_limits(orc):
    for mode in (MODE_R, MODE_Z):
        for seed in (21, 22, 23):
            p, c, q, m, v, s = _predicted(orc, mode, seed)
            # infinite hit error: nothing changes
            st, p1, c1, q1, chi2 = orc.update(mode, q, p, c, m, v * 1e14)
            assert q1 == q
            dp = p1 - p
            dp[4] = _wrap(dp[4])  # the update wraps phi into (-pi, pi]
            assert np.all(np.abs(dp) <= 1e-9 * np.abs(p) + 1e-12), (p1, p)
            C, C1 = _sym6(c), _sym6(c1)
            d = np.sqrt(np.outer(np.diag(C), np.diag(C))) + 1e-300
            assert np.abs((C1 - C) / d).max() < 1e-8
            assert chi2 < 1e-6
            # vanishing hit error: the measured coordinates move onto the hit
            st, p0, c0, _, _ = orc.update(mode, q, p, c, m, v * 1e-14)
            Hp, _ = _H(mode, m)
            assert np.allclose(Hp @ p0[:3], Hp @ m, atol=1e-6), (Hp @ p0[:3], Hp @ m)
            if mode == MODE_Z:
                assert np.allclose(p0[:3], m, atol=1e-6)  # z is already on the plane
            else:
                delta = np.arctan2(m[1], m[0]) - np.arctan2(p[1], p[0])
                bound = s * (1 / np.cos(delta) - 1)
                assert np.linalg.norm(p0[:3] - m) <= bound + 1e-6
            assert -np.pi < p0[4] <= np.pi


def pin_update_information_form(orc):
    rng = np.random.default_rng(24)
    for mode in (MODE_R, MODE_Z):
        for _ in range(10):
            A = rng.normal(size=(6, 6)) * np.array([0.05, 0.05, 0.2, 0.01, 0.003, 0.003])
            C = A @ A.T + np.diag([1e-4, 1e-4, 1e-3, 1e-6, 1e-6, 1e-6])
            ph, th = rng.uniform(-np.pi, np.pi), rng.uniform(0.3, 2.8)
            if mode == MODE_R:
                R = rng.uniform(5, 100)
                p = np.array([R * np.cos(ph), R * np.sin(ph), rng.uniform(-50, 50), 0.5, ph + 0.1, th])
                mh = ph + rng.normal() * 1e-3
                m = np.array([R * np.cos(mh), R * np.sin(mh), p[2] + rng.normal() * 0.1])
                t = np.array([-np.sin(mh), np.cos(mh), 0.0])
                V = 1e-4 * np.outer(t, t) + 1e-2 * np.diag([0, 0, 1.0])
            else:
                p = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), 100.0, 0.5, ph, th])
                m = p[:3] + np.array([rng.normal() * 0.05, rng.normal() * 0.05, 0.0])
                V = np.diag([1e-3, 2e-3, 0.0])
                V[0, 1] = V[1, 0] = 5e-4
            v6 = np.array([V[0, 0], V[1, 0], V[1, 1], V[2, 0], V[2, 1], V[2, 2]])
            c21 = np.array([C[i, j] for i in range(6) for j in range(i + 1)])
            st, p1, c1, q1, chi2 = orc.update(mode, 1, p, c21, m, v6)
            Hp, H = _H(mode, m)
            Vl = Hp @ V @ Hp.T
            Ci = np.linalg.inv(C)
            Cp = np.linalg.inv(Ci + H.T @ np.linalg.inv(Vl) @ H)
            r = Hp @ (m - p[:3])
            pexp = p + Cp @ H.T @ np.linalg.inv(Vl) @ r
            pexp[4] = _wrap(pexp[4])
            C1 = _sym6(c1)
            d = np.sqrt(np.outer(np.diag(Cp), np.diag(Cp)))
            assert np.abs((C1 - Cp) / d).max() < 1e-8
            assert np.allclose(p1, pexp, rtol=1e-9, atol=1e-10), (p1, pexp)
            # predicted chi2 = filtered residual chi2 + state-change chi2
            rf = Hp @ (m - p1[:3])
            dp = p1 - p
            dp[4] = _wrap(dp[4])
            split = rf @ np.linalg.inv(Vl) @ rf + dp @ Ci @ dp
            assert abs(chi2 - split) < 1e-8 * max(1.0, chi2), (chi2, split)
            # the covariance can only shrink
            ev = np.linalg.eigvalsh(C - C1)
            assert ev.min() > -1e-12 * np.abs(ev).max()


def pin_propagated_covariance(orc):
    """J C J^T is symmetric PSD with no variance along the surface normal."""
    for mode in (MODE_R, MODE_Z):
        for seed in (31, 32):
            p, c, q, m, v, s = _predicted(orc, mode, seed)
            C = _sym6(c)
            if mode == MODE_Z:
                n = np.array([0, 0, 1.0, 0, 0, 0])
            else:
                n = np.array([p[0] / s, p[1] / s, 0, 0, 0, 0])
            assert abs(n @ C @ n) < 1e-12 * np.trace(C)
            Q = np.linalg.svd(n.reshape(1, 6))[2][1:]  # orthonormal basis of n-perp
            np.linalg.cholesky(Q @ C @ Q.T)


def pin_no_intersection(orc):
    # a p2r track whose circle never reaches the cylinder
    pt = 0.3
    p = np.array([0, 0, 0, 1 / pt, 0.3, 1.2])
    rho = pt / (KA * B)
    st, _ = orc.path_length(MODE_R, B, 2.2 * rho, 1, p)
    assert st & 1
    # a p2z plane behind the track
    p = np.array([0, 0, 50.0, 0.5, 0.3, 0.4])
    st, _ = orc.path_length(MODE_Z, B, 20.0, 1, p)
    assert st & 1


def _flip_case(rng, mode):
    """A state on the surface whose update drives w = 1/pT through zero: its
    covariance correlates w strongly with the first measured coordinate and
    the hit lies on the side that pushes w past zero."""
    ph, th = rng.uniform(-np.pi, np.pi), rng.uniform(0.5, 2.6)
    w = 0.02
    if mode == MODE_R:
        R = rng.uniform(20, 100)
        p = np.array([R * np.cos(ph), R * np.sin(ph), rng.uniform(-50, 50), w, ph + 0.05, th])
        t = np.array([-np.sin(ph), np.cos(ph), 0.0])  # measured direction at the hit
    else:
        p = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), 120.0, w, ph, th])
        t = np.array([1.0, 0.0, 0.0])
    sig = np.array([0.1, 0.1, 0.2, 0.1, 0.003, 0.003])
    corr = np.eye(6)
    # w correlated (0.9) with the position along t
    for k in range(3):
        corr[3, k] = corr[k, 3] = 0.9 * t[k]
    C = corr * np.outer(sig, sig)
    if mode == MODE_R:  # no variance along the cylinder normal
        n = np.array([np.cos(ph), np.sin(ph), 0, 0, 0, 0])
        P = np.eye(6) - np.outer(n, n)
        C = P @ C @ P
    C += np.diag([1e-8, 1e-8, 1e-8, 1e-8, 1e-8, 1e-8])
    m = p[:3] - 0.25 * t  # the residual along t is -0.25 cm
    if mode == MODE_R:  # keep the hit on the cylinder
        m[:2] *= np.hypot(p[0], p[1]) / np.hypot(m[0], m[1])
    V = 1e-4 * np.outer(t, t) + (1e-2 * np.diag([0, 0, 1.0]) if mode == MODE_R else
                                 1e-4 * np.diag([0, 1.0, 0]))
    return p, C, m, V


def pin_charge_flip(orc):
    """An update that drives w through zero.  The oracle's result must be the
    plain Kalman update (its information form, written here) reparametrised:
    (w, q) -> (-w, -q), which describes the same helix since kappa = -q kA B w
    is unchanged, with the covariance transformed by D = diag(1, 1, 1, -1, 1, 1)
    (row and column 3 negated, C[3][3] kept), and status bit 8 set."""
    rng = np.random.default_rng(27)
    D = np.diag([1.0, 1.0, 1.0, -1.0, 1.0, 1.0])
    for mode in (MODE_R, MODE_Z):
        for q in (1, -1):
            for _ in range(4):
                p, C, m, V = _flip_case(rng, mode)
                v6 = np.array([V[0, 0], V[1, 0], V[1, 1], V[2, 0], V[2, 1], V[2, 2]])
                c21 = np.array([C[i, j] for i in range(6) for j in range(i + 1)])
                st, p1, c1, q1, chi2 = orc.update(mode, q, p, c21, m, v6)
                # the update without normalisation, in information form
                Hp, H = _H(mode, m)
                Vl = Hp @ V @ Hp.T
                Ci = np.linalg.inv(C)
                Cp = np.linalg.inv(Ci + H.T @ np.linalg.inv(Vl) @ H)
                pexp = p + Cp @ H.T @ np.linalg.inv(Vl) @ (Hp @ (m - p[:3]))
                pexp[4] = _wrap(pexp[4])
                assert pexp[3] < -0.05, pexp[3]  # the case really crosses zero
                # (iii) charge negated, status bit set
                assert q1 == -q and (st & 8), (q1, st)
                # w flipped, the other parameters as the plain update
                flip = D @ pexp
                assert np.allclose(p1, flip, rtol=1e-9, atol=1e-11), (p1, flip)
                assert p1[3] > 0
                # (ii) C' = D Cp D, including an unchanged C[3][3]
                C1 = _sym6(c1)
                d = np.sqrt(np.outer(np.diag(Cp), np.diag(Cp)))
                assert np.abs((C1 - D @ Cp @ D) / d).max() < 1e-8
                assert C1[3, 3] > 0 and abs(C1[3, 3] - Cp[3, 3]) < 1e-9 * Cp[3, 3]
                # (i) the flipped state (w > 0, -q) and the plain one (w < 0, q)
                # are the same helix
                for h in (0.5, 7.0, 40.0):
                    a, b = orc.helix(B, q1, p1, h), orc.helix(B, q, pexp, h)
                    assert np.allclose(a[:3], b[:3], rtol=0, atol=1e-9), (h, a, b)
                    assert abs(_wrap(a[4] - b[4])) < 1e-12
                # and reach a surface at the same point
                s_next = (np.hypot(p1[0], p1[1]) + 10.0) if mode == MODE_R else p1[2] + 20.0
                if mode == MODE_Z and np.cos(p1[5]) < 0:
                    s_next = p1[2] - 20.0
                sa, pa, _, ha = orc.transport(mode, B, s_next, q1, p1)
                sb, pb, _, hb = orc.transport(mode, B, s_next, q, pexp)
                assert sa == sb
                if sa == 0:
                    assert abs(ha - hb) < 1e-9 * max(1.0, ha)
                    assert np.allclose(pa[:3], pb[:3], rtol=0, atol=1e-9)
    # and no flip while w stays positive
    p, C, m, V = _flip_case(rng, MODE_Z)
    m = p[:3] + 0.25 * np.array([1.0, 0.0, 0.0])
    v6 = np.array([V[0, 0], V[1, 0], V[1, 1], V[2, 0], V[2, 1], V[2, 2]])
    c21 = np.array([C[i, j] for i in range(6) for j in range(i + 1)])
    st, p1, _, q1, _ = orc.update(MODE_Z, 1, p, c21, m, v6)
    assert q1 == 1 and not (st & 8) and p1[3] > p[3]


def _reverse(p):
    """The same point with the momentum reversed: phi + pi, pi - theta (the
    charge is negated beside it).  kappa changes sign, so the reversed track
    runs back along the same curve."""
    r = p.copy()
    r[4] = _wrap(p[4] + np.pi)
    r[5] = np.pi - p[5]
    return r


def pin_reversibility(orc):
    """Propagating to a surface and then, with the momentum reversed, back to
    the start surface returns the start state (to ~1e-12), and the composed
    surface-to-surface Jacobians are the identity on the start surface's
    tangent space."""
    rng = np.random.default_rng(28)
    Dr = np.diag([1.0, 1.0, 1.0, 1.0, 1.0, -1.0])  # d(reverse)/dp
    for mode in (MODE_R, MODE_Z):
        for p, q, s1 in _states(rng, 15, mode):
            if mode == MODE_R:
                s0 = float(np.hypot(p[0], p[1]))
                if s0 < 1.0:
                    continue
                tang = [np.array([-p[1], p[0], 0, 0, 0, 0]) / s0] + [np.eye(6)[k] for k in (2, 3, 4, 5)]
            else:
                s0 = float(p[2])
                tang = [np.eye(6)[k] for k in (0, 1, 3, 4, 5)]
            st, p1, J1, h1 = orc.transport(mode, B, s1, q, p)
            assert st == 0
            st, p2, J2, h2 = orc.transport(mode, B, s0, -q, _reverse(p1))
            assert st == 0
            back = _reverse(p2)
            d = back - p
            d[4] = _wrap(d[4])
            assert np.all(np.abs(d) <= 1e-12 * np.maximum(np.abs(p), 1.0)), (p, back)
            assert abs(h1 - h2) <= 1e-10 * max(1.0, h1)
            Jt = Dr @ J2 @ Dr @ J1
            for v in tang:
                assert np.allclose(Jt @ v, v, rtol=0, atol=1e-10 * max(1.0, np.abs(J1).max())), (mode, v, Jt @ v)


def _covs_pd_on_surface(mode, par, cov, surf_last):
    for i in range(par.shape[1]):
        C = _sym6(cov[:, i])
        if mode == MODE_Z:
            n = np.array([0, 0, 1.0, 0, 0, 0])
        else:
            n = np.array([par[0, i] / surf_last, par[1, i] / surf_last, 0, 0, 0, 0])
        Q = np.linalg.svd(n.reshape(1, 6))[2][1:]
        np.linalg.cholesky(Q @ C @ Q.T)


def pin_filter_consistency(orc, n=4000):
    for mode in (MODE_R, MODE_Z):
        ts = gen.generate(mode, n, seed=41 + mode, want_truth=True)
        r = orc.fit_set(ts, want_layers=True)
        assert (r["status"] & ~np.uint8(8)).max() == 0
        mean_chi2 = r["chi2_layer"].mean()
        assert abs(mean_chi2 - 2.0) < 0.06, mean_chi2
        tr = ts.truth[-1]
        for k in (3, 4, 5) + ((2,) if mode == MODE_R else (0, 1)):
            var = r["cov"][k * (k + 1) // 2 + k]
            d = r["par"][k] - tr[k]
            if k == 4:
                d = _wrap(d)
            pull = d / np.sqrt(var)
            assert abs(pull.mean()) < 0.08, (mode, k, pull.mean())
            assert abs(pull.std() - 1.0) < 0.06, (mode, k, pull.std())
        assert np.all(r["par"][4] > -np.pi) and np.all(r["par"][4] <= np.pi)
        _covs_pd_on_surface(mode, r["par"][:, :200], r["cov"][:, :200], float(ts.surf[-1]))


def pin_chi2_gradient_fd(orc):
    for mode in (MODE_R, MODE_Z):
        surf = (np.linspace(4, 40, 5) if mode == MODE_R else np.linspace(10, 60, 5)).astype(np.float32)
        ts = gen.generate(mode, 3, seed=51 + mode, surf=surf)
        g = orc.chi2_grad(ts.mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)
        base = orc.fit_set(ts)
        assert np.allclose(g["chi2"], base["chi2"], rtol=1e-12)
        par0 = ts.par0.astype(np.float64)
        hpos = ts.hpos.astype(np.float64)
        sc = np.array([1e-4, 1e-4, 1e-3, 1e-4, 1e-5, 1e-5])
        for k in range(6):
            eps = sc[k] * (par0[3] if k == 3 else 1.0)
            pp, pm = par0.copy(), par0.copy()
            pp[k] += eps
            pm[k] -= eps
            fp = orc.fit(ts.mode, ts.B, ts.surf, pp, ts.cov0, ts.q, hpos, ts.hcov)["chi2"]
            fm = orc.fit(ts.mode, ts.B, ts.surf, pm, ts.cov0, ts.q, hpos, ts.hcov)["chi2"]
            fd = (fp - fm) / (2 * eps)
            assert np.allclose(g["g_par0"][k], fd, rtol=1e-4, atol=1e-4 * np.abs(fd).max() + 1e-6), (k, g["g_par0"][k], fd)
        for l in range(ts.nlayer):
            for k in range(3):
                eps = 1e-5
                hp, hm = hpos.copy(), hpos.copy()
                hp[l, k] += eps
                hm[l, k] -= eps
                fp = orc.fit(ts.mode, ts.B, ts.surf, par0, ts.cov0, ts.q, hp, ts.hcov)["chi2"]
                fm = orc.fit(ts.mode, ts.B, ts.surf, par0, ts.cov0, ts.q, hm, ts.hcov)["chi2"]
                fd = (fp - fm) / (2 * eps)
                assert np.allclose(g["g_hpos"][l, k], fd, rtol=1e-4, atol=1e-3), (l, k, g["g_hpos"][l, k], fd)


# ---- track finding (orc_find) ----------------------------------------------------


def _find_layerwise(orc, ts, cs, gate):
    """Track finding composed here from the single-step propagate and update,
    with the argmin over candidates written out."""
    nlayer, ncand, _, n = cs.cpos.shape
    out = {"par": np.zeros((6, n)), "cov": np.zeros((21, n)), "chi2": np.zeros(n),
           "chosen": np.full((nlayer, n), -1)}
    for i in range(n):
        p, c, q = ts.par0[:, i].astype(np.float64), ts.cov0[:, i].astype(np.float64), int(ts.q[i])
        chi2 = 0.0
        for l in range(nlayer):
            st, pp, cp = orc.propagate(ts.mode, ts.B, float(ts.surf[l]), q, p, c)
            if st:
                break
            trial = [orc.update(ts.mode, q, pp, cp, cs.cpos[l, k, :, i], cs.ccov[l, k, :, i])[4]
                     for k in range(ncand)]
            ok = [k for k in range(ncand) if trial[k] < gate]
            p, c = pp, cp
            if ok:
                best = min(ok, key=lambda k: (trial[k], k))
                out["chosen"][l, i] = best
                _, p, c, q, x = orc.update(ts.mode, q, pp, cp, cs.cpos[l, best, :, i],
                                           cs.ccov[l, best, :, i])
                chi2 += x
        out["par"][:, i], out["cov"][:, i], out["chi2"][i] = p, c, chi2
    return out


def pin_find_layerwise(orc):
    """orc_find equals the composition of the pinned single steps with the
    argmin over candidates, on noisy candidates that make it choose noise,
    nothing and the track's own hit."""
    for mode in (MODE_R, MODE_Z):
        ts = gen.generate(mode, 12, seed=21, nlayer=4)
        cs = gen.generate_candidates(ts, 3, seed=21, spread=3.0, p_true=0.7)
        got = orc.find(mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, 30.0)
        ref = _find_layerwise(orc, ts, cs, 30.0)
        assert np.array_equal(got["chosen"], ref["chosen"])
        assert (got["chosen"] >= 0).any() and (got["chosen"] != cs.true_slot).any()
        for k in ("par", "cov", "chi2"):
            assert np.allclose(got[k], ref[k], rtol=1e-13, atol=1e-15), k


def pin_find_single_candidate(orc):
    """One candidate, the track's own hit, and no gate: the plain fit, bit for
    bit."""
    for mode in (MODE_R, MODE_Z):
        ts = gen.generate(mode, 100, seed=22)
        got = orc.find(mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, ts.hpos[:, None],
                       ts.hcov[:, None], 1e300)
        ref = orc.fit_set(ts, want_layers=True)
        for k in ("par", "cov", "q", "chi2", "chi2_layer", "status"):
            assert np.array_equal(got[k], ref[k]), k
        assert (got["chosen"] == 0).all()


def pin_find_nothing_under_gate(orc):
    """No candidate under the gate: no update, the state is the propagation."""
    ts = gen.generate(MODE_R, 10, seed=23, nlayer=5)
    cs = gen.generate_candidates(ts, 2, seed=23, spread=1e4, p_true=0.0)
    got = orc.find(MODE_R, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, 30.0)
    assert (got["chosen"] == -1).all() and (got["chi2"] == 0).all()
    assert (got["cand_chi2"] >= 30.0).all()
    for i in range(ts.n):
        p, c = ts.par0[:, i].astype(np.float64), ts.cov0[:, i].astype(np.float64)
        for l in range(5):
            _, p, c = orc.propagate(MODE_R, ts.B, float(ts.surf[l]), int(ts.q[i]), p, c)
        assert np.allclose(got["par"][:, i], p, rtol=1e-14) and np.allclose(got["cov"][:, i], c, rtol=1e-14)


def pin_find_separated_candidates(orc):
    """Noise far from the track's hit: the track's hit is found on > 99.9 % of
    layers."""
    ts = gen.generate(MODE_Z, 500, seed=24)
    cs = gen.generate_candidates(ts, 4, seed=24, spread=1e3, p_true=1.0)
    got = orc.find(MODE_Z, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, cs.cpos, cs.ccov, 30.0)
    assert np.mean(got["chosen"] == cs.true_slot) > 0.999


ALL_PINS = [
    pin_helix_equation_of_motion,
    pin_helix_geometry,
    pin_straight_line_surfaces,
    pin_landing,
    pin_path_r_bruteforce,
    pin_path_r_half_angle,
    pin_jacobian_fd,
    pin_update_limits,
    pin_update_information_form,
    pin_propagated_covariance,
    pin_charge_flip,
    pin_reversibility,
    pin_no_intersection,
    pin_filter_consistency,
    pin_chi2_gradient_fd,
    pin_find_layerwise,
    pin_find_single_candidate,
    pin_find_nothing_under_gate,
    pin_find_separated_candidates,
]
