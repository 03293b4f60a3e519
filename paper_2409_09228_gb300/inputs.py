"""Seeded synthetic inputs for the track fit: tracks, hits, detector surfaces.

This module draws the workload only.  It holds none of the fit's arithmetic
(no propagation of a fitted state, no Jacobian, covariance transport or Kalman
update): the truth trajectories are helices through the origin, whose surface
crossings have the simple closed forms below, and the hits are those crossings
smeared by Gaussian noise.  Both the GPU library's tests and the CPU oracle
take their inputs from here.

Workload (paper Sec. 3.1): one seed track smeared per track, one hit per layer
smeared per track.  Distributions are the synthetic stand-ins this library is
measured on:
  * p2r: cylinders at radii uniformly spaced 4..110 cm; |eta| < 1.
  * p2z: planes at z uniformly spaced 10..270 cm; eta in [1.5, 2.5].
  * pT ~ U[0.5, 10] GeV, phi ~ U[0, 2 pi), q = +-1 with probability 1/2,
    theta = 2 atan(exp(-eta)); B = 3.8 T along +z.
  * p2r only: a track whose transverse circle has diameter 2 rho reaches
    radius R only if R <= 2 rho, and crosses it tangentially at R = 2 rho.
    pT is drawn from U[0.5, 10] conditioned on R_max / (2 rho) <= 0.9, i.e.
    U[pT_min, 10] with pT_min = kA B R_max / 1.8 (0.697 GeV at 110 cm, 3.8 T).
  * hits: p2r moves the crossing along the cylinder by N(0, 0.01 cm) in r-phi
    and N(0, 0.1 cm) in z; p2z moves it in the plane by N(0, 0.01 cm) along
    the azimuthal direction and N(0, 0.1 cm) along the radial direction.  The
    hit covariance is the matching rank-2 3x3 matrix.
  * initial state: the truth at the vertex plus N(0, sigma0) with
    sigma0 = (0.01, 0.01, 0.1 cm, 0.05 w, 0.01 rad, 0.01 rad); covariance
    diag(sigma0^2).

Random numbers come from numpy's Philox counter-based generator, one
independent stream per (seed, quantity), drawn in track order, so the inputs
do not depend on thread counts or on how the work is later split.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

KA = 0.00299792458  # GeV / (T cm)
B_FIELD = 3.8
NLAYER = 20
MODE_R = 0
MODE_Z = 1
SIGMA0 = (0.01, 0.01, 0.1, 0.05, 0.01, 0.01)  # w entry is relative
SIGMA_RPHI = 0.01
SIGMA_2 = 0.1  # z for p2r, radial for p2z

_STREAM_PT, _STREAM_ETA, _STREAM_PHI, _STREAM_Q, _STREAM_INIT, _STREAM_HIT = range(6)


def surfaces(mode: int, nlayer: int = NLAYER) -> np.ndarray:
    """Layer positions: radii 4..110 cm (p2r) or z 10..270 cm (p2z), float32."""
    if mode == MODE_R:
        return np.linspace(4.0, 110.0, nlayer).astype(np.float32)
    return np.linspace(10.0, 270.0, nlayer).astype(np.float32)


def pt_min_p2r(B: float, rmax: float, frac: float = 0.9) -> float:
    return KA * B * rmax / (2.0 * frac)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=(int(seed) << 8) | stream))


@dataclass
class TrackSet:
    mode: int
    B: float
    surf: np.ndarray          # (nlayer,) float32
    par0: np.ndarray          # (6, n) float32: x, y, z, w=1/pT, phi, theta
    cov0: np.ndarray          # (21, n) float32, packed lower triangle
    q: np.ndarray             # (n,) int32
    hpos: np.ndarray          # (nlayer, 3, n) float32
    hcov: np.ndarray          # (nlayer, 6, n) float32, (xx, yx, yy, zx, zy, zz)
    truth: Optional[np.ndarray] = field(default=None)  # (nlayer, 6, n) float64

    @property
    def n(self) -> int:
        return self.par0.shape[1]

    @property
    def nlayer(self) -> int:
        return self.hpos.shape[0]

    def subset(self, idx) -> "TrackSet":
        idx = np.asarray(idx)
        return TrackSet(self.mode, self.B, self.surf, np.ascontiguousarray(self.par0[:, idx]),
                        np.ascontiguousarray(self.cov0[:, idx]), np.ascontiguousarray(self.q[idx]),
                        np.ascontiguousarray(self.hpos[:, :, idx]),
                        np.ascontiguousarray(self.hcov[:, :, idx]),
                        None if self.truth is None else np.ascontiguousarray(self.truth[:, :, idx]))


def _p2r_crossing(s, rho, phi0, q, cot):
    """Where a truth helix from the origin crosses the cylinder of radius s: a
    circle through the origin reaches radius s after turning by
    2 asin(s / 2 rho), and the crossing sits on the chord direction.  Returns
    (azimuth of the crossing, its z, momentum azimuth there)."""
    with np.errstate(invalid="ignore"):
        half = np.arcsin(s / (2.0 * rho))
    return phi0 - q * half, 2.0 * rho * half * cot, phi0 - 2.0 * q * half


def generate(mode: int, n: int, seed: int, nlayer: int = NLAYER, B: float = B_FIELD,
             surf: Optional[np.ndarray] = None, pt_range=(0.5, 10.0), eta_range=None,
             want_truth: bool = False, sigma_rphi: float = SIGMA_RPHI,
             sigma_2: float = SIGMA_2, pt: Optional[np.ndarray] = None) -> TrackSet:
    """n independent tracks of one mode with hits on nlayer surfaces.

    pt, if given, replaces the pT draw (and its p2r reach condition): hits on
    cylinders a track cannot reach are NaN.
    """
    surf = surfaces(mode, nlayer) if surf is None else np.asarray(surf, np.float32)
    nlayer = surf.shape[0]
    s64 = surf.astype(np.float64)
    B = float(np.float32(B))
    lo, hi = pt_range
    if mode == MODE_R:
        lo = max(lo, pt_min_p2r(B, float(s64.max())))
        eta_lo, eta_hi = (-1.0, 1.0) if eta_range is None else eta_range
    else:
        eta_lo, eta_hi = (1.5, 2.5) if eta_range is None else eta_range
    pt_draw = _rng(seed, _STREAM_PT).uniform(lo, hi, n)
    pt = pt_draw if pt is None else np.asarray(pt, np.float64)
    eta = _rng(seed, _STREAM_ETA).uniform(eta_lo, eta_hi, n)
    phi0 = _rng(seed, _STREAM_PHI).uniform(0.0, 2.0 * np.pi, n)
    q = np.where(_rng(seed, _STREAM_Q).random(n) < 0.5, -1, 1).astype(np.int32)
    theta = 2.0 * np.arctan(np.exp(-eta))
    w = 1.0 / pt
    cot = 1.0 / np.tan(theta)
    rho = pt / (KA * B)  # transverse radius of curvature [cm]

    noise = _rng(seed, _STREAM_HIT)
    hpos = np.empty((nlayer, 3, n), np.float32)
    hcov = np.zeros((nlayer, 6, n), np.float32)
    truth = np.empty((nlayer, 6, n)) if want_truth else None

    def layer(l, n1, n2):
        s = s64[l]
        if mode == MODE_R:
            chord_phi, z, phi_dir = _p2r_crossing(s, rho, phi0, q, cot)
            phi_hit = chord_phi + n1 * sigma_rphi / s
            c, sn = np.cos(phi_hit), np.sin(phi_hit)
            hpos[l, 0], hpos[l, 1], hpos[l, 2] = s * c, s * sn, z + n2 * sigma_2
            vr = sigma_rphi ** 2
            hcov[l, 0] = vr * sn * sn
            hcov[l, 1] = -vr * sn * c
            hcov[l, 2] = vr * c * c
            hcov[l, 5] = sigma_2 ** 2
            if want_truth:
                truth[l] = (s * np.cos(chord_phi), s * np.sin(chord_phi), z, w, phi_dir, theta)
        else:
            # Transverse path to the plane, then the chord of that arc.
            h = s * np.tan(theta)
            half = -q * h / (2.0 * rho)
            chord = h * np.sinc(half / np.pi)  # numpy: sinc(x) = sin(pi x)/(pi x)
            x = chord * np.cos(phi0 + half)
            y = chord * np.sin(phi0 + half)
            r = np.hypot(x, y)
            ux, uy = x / r, y / r          # radial direction in the plane
            tx, ty = -uy, ux               # azimuthal direction in the plane
            hpos[l, 0] = x + n1 * sigma_rphi * tx + n2 * sigma_2 * ux
            hpos[l, 1] = y + n1 * sigma_rphi * ty + n2 * sigma_2 * uy
            hpos[l, 2] = s
            a, b = sigma_rphi ** 2, sigma_2 ** 2
            hcov[l, 0] = a * tx * tx + b * ux * ux
            hcov[l, 1] = a * ty * tx + b * uy * ux
            hcov[l, 2] = a * ty * ty + b * uy * uy
            if want_truth:
                truth[l] = (x, y, np.full(n, s), w, phi0 + 2.0 * half, theta)

    # The hit noise is drawn layer by layer in this thread (the stream's
    # order), and each layer's arithmetic runs on a worker thread (numpy
    # releases the GIL): the same numbers as a sequential loop, sooner.
    workers = max(1, min(8, (os.cpu_count() or 1)))
    if n < 100000 or workers == 1:
        for l in range(nlayer):
            n1 = noise.standard_normal(n)
            n2 = noise.standard_normal(n)
            layer(l, n1, n2)
    else:
        with ThreadPoolExecutor(workers) as ex:
            futs = []
            for l in range(nlayer):
                if l >= 2 * workers:
                    futs[l - 2 * workers].result()  # bound the noise arrays in flight
                n1 = noise.standard_normal(n)
                n2 = noise.standard_normal(n)
                futs.append(ex.submit(layer, l, n1, n2))
            for f in futs:
                f.result()

    init = _rng(seed, _STREAM_INIT).standard_normal((6, n))
    sig = np.stack([np.full(n, SIGMA0[0]), np.full(n, SIGMA0[1]), np.full(n, SIGMA0[2]),
                    SIGMA0[3] * w, np.full(n, SIGMA0[4]), np.full(n, SIGMA0[5])])
    truth0 = np.stack([np.zeros(n), np.zeros(n), np.zeros(n), w, phi0, theta])
    par0 = (truth0 + sig * init).astype(np.float32)
    cov0 = np.zeros((21, n), np.float32)
    for i in range(6):
        cov0[i * (i + 1) // 2 + i] = (sig[i] ** 2).astype(np.float32)
    return TrackSet(mode, B, surf, par0, cov0, q, hpos, hcov, truth)


# Spread of a filtered state around the truth, used for the learned seed's
# samples: position (x, y, z) in cm, relative w, phi and theta in rad.
SIGMA_STATE = (0.01, 0.01, 0.1, 0.01, 1e-3, 1e-3)


@dataclass
class SeedSamples:
    """Single p2r propagations: state par (6, n) float32 with charge q (n,)
    int32, to the cylinder of radius R (n,) float32, layer index layer (n,)."""
    B: float
    par: np.ndarray
    q: np.ndarray
    R: np.ndarray
    layer: np.ndarray

    @property
    def n(self) -> int:
        return self.par.shape[1]


def seed_samples(n: int, seed: int, nlayer: int = NLAYER, B: float = B_FIELD,
                 surf: Optional[np.ndarray] = None) -> SeedSamples:
    """Samples of the propagations a p2r fit makes: a track drawn as in
    generate(MODE_R, ...), a layer l uniform in [0, nlayer), the cylinder R_l as
    target, and as start the state the fit would hold before layer l -- the
    smeared vertex state for l = 0, else the truth crossing of layer l - 1
    smeared by SIGMA_STATE (the spread of a filtered state)."""
    surf = surfaces(MODE_R, nlayer) if surf is None else np.asarray(surf, np.float32)
    nlayer = surf.shape[0]
    B = float(np.float32(B))
    lo = max(0.5, pt_min_p2r(B, float(surf.astype(np.float64).max())))
    pt = _rng(seed, _STREAM_PT).uniform(lo, 10.0, n)
    eta = _rng(seed, _STREAM_ETA).uniform(-1.0, 1.0, n)
    phi0 = _rng(seed, _STREAM_PHI).uniform(0.0, 2.0 * np.pi, n)
    q = np.where(_rng(seed, _STREAM_Q).random(n) < 0.5, -1, 1).astype(np.int32)
    layer = _rng(seed, 18).integers(0, nlayer, n)
    theta = 2.0 * np.arctan(np.exp(-eta))
    w = 1.0 / pt
    rho = pt / (KA * B)
    s_prev = surf.astype(np.float64)[np.maximum(layer - 1, 0)]
    chord_phi, z, phi_dir = _p2r_crossing(s_prev, rho, phi0, q, 1.0 / np.tan(theta))
    on_layer = np.stack([s_prev * np.cos(chord_phi), s_prev * np.sin(chord_phi), z, w, phi_dir,
                         theta])
    at_vertex = np.stack([np.zeros(n), np.zeros(n), np.zeros(n), w, phi0, theta])
    sig_v = np.array(SIGMA0)[:, None] * np.stack([np.ones(n)] * 3 + [w] + [np.ones(n)] * 2)
    sig_l = np.array(SIGMA_STATE)[:, None] * np.stack([np.ones(n)] * 3 + [w] + [np.ones(n)] * 2)
    noise = _rng(seed, _STREAM_INIT).standard_normal((6, n))
    par = np.where(layer[None, :] == 0, at_vertex + sig_v * noise, on_layer + sig_l * noise)
    return SeedSamples(B, par.astype(np.float32), q, surf[layer], layer.astype(np.int32))


def uneven_event_sizes(nevt: int, seed: int, median: float = 2000.0, sigma_ln: float = 1.0,
                       lo: int = 50, hi: int = 20000) -> np.ndarray:
    """Track counts per event: log-normal (median, sigma_ln) clipped to [lo, hi]."""
    g = _rng(seed, 16)
    ntrk = np.exp(np.log(median) + sigma_ln * g.standard_normal(nevt))
    return np.clip(np.rint(ntrk), lo, hi).astype(np.int64)


def uneven_event_modes(nevt: int, seed: int) -> np.ndarray:
    """Mode per event, p2r or p2z with probability 1/2."""
    return np.where(_rng(seed, 17).random(nevt) < 0.5, MODE_R, MODE_Z).astype(np.int32)


@dataclass
class EventSet:
    """Events stored one after another (event e holds ntrk[e] tracks of mode[e])."""
    ntrk: np.ndarray          # (nevt,) int64
    mode: np.ndarray          # (nevt,) int32
    B: float
    surf: tuple               # (p2r radii, p2z z positions), float32
    par0: np.ndarray          # (6, n)
    cov0: np.ndarray          # (21, n)
    q: np.ndarray             # (n,)
    hpos: np.ndarray          # (nlayer, 3, n)
    hcov: np.ndarray          # (nlayer, 6, n)

    @property
    def n(self) -> int:
        return int(self.ntrk.sum())

    def starts(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.ntrk)]).astype(np.int64)

    def event(self, e: int) -> TrackSet:
        s = self.starts()
        a, b = int(s[e]), int(s[e + 1])
        m = int(self.mode[e])
        return TrackSet(m, self.B, self.surf[m], self.par0[:, a:b], self.cov0[:, a:b],
                        self.q[a:b], self.hpos[:, :, a:b], self.hcov[:, :, a:b])


def generate_events(ntrk, modes, seed: int, nlayer: int = NLAYER, B: float = B_FIELD) -> EventSet:
    """Events of the given sizes and modes; the tracks of each mode come from
    one generate() call (seed, seed + 1), dealt out to that mode's events in
    order."""
    ntrk = np.asarray(ntrk, np.int64)
    modes = np.asarray(modes, np.int32)
    counts = [int(ntrk[modes == m].sum()) for m in (MODE_R, MODE_Z)]
    with ThreadPoolExecutor(2) as ex:  # the two pools draw from independent streams
        pools = list(ex.map(lambda m: generate(m, counts[m], seed=seed + m, nlayer=nlayer, B=B),
                            (MODE_R, MODE_Z)))
    # position in event order of every track of each pool
    dest = [np.empty(c, np.int64) for c in counts]
    next_idx, pos = [0, 0], 0
    for k, m in zip(ntrk, modes):
        dest[m][next_idx[m]:next_idx[m] + k] = np.arange(pos, pos + k)
        next_idx[m] += k
        pos += k
    n = int(ntrk.sum())

    def deal(name):
        a0 = getattr(pools[0], name)
        out = np.empty(a0.shape[:-1] + (n,), a0.dtype)
        for m in (MODE_R, MODE_Z):
            out[..., dest[m]] = getattr(pools[m], name)
        return out

    return EventSet(ntrk, modes, pools[0].B, (pools[0].surf, pools[1].surf), deal("par0"),
                    deal("cov0"), deal("q"), deal("hpos"), deal("hcov"))


@dataclass
class CandidateSet:
    """Candidate hits for track finding: positions (nlayer, ncand, 3, n) and
    covariances (nlayer, ncand, 6, n), float32; true_slot (nlayer, n) is the
    slot holding the track's own hit, or -1 where it is missing."""
    cpos: np.ndarray
    ccov: np.ndarray
    true_slot: np.ndarray


def generate_candidates(ts: TrackSet, ncand: int, seed: int, p_true: float = 0.95,
                        spread: float = 5.0) -> CandidateSet:
    """ncand candidate hits per track and layer: the track's own hit (from ts)
    with probability p_true in a random slot, the other slots noise hits on
    the same surface, displaced from the track's hit by `spread` times the hit
    errors (sigma_rphi along the azimuthal direction, sigma_2 along z for
    cylinders or along the radius for planes), each with the covariance a hit
    at its place would have."""
    nlayer, _, n = ts.hpos.shape
    g = _rng(seed, 19)
    present = g.random((nlayer, n)) < p_true
    slot = g.integers(0, ncand, (nlayer, n))
    true_slot = np.where(present, slot, -1).astype(np.int32)
    cpos = np.empty((nlayer, ncand, 3, n), np.float32)
    ccov = np.zeros((nlayer, ncand, 6, n), np.float32)
    a, b = SIGMA_RPHI ** 2, SIGMA_2 ** 2
    for l in range(nlayer):
        hx, hy, hz = (ts.hpos[l, k].astype(np.float64) for k in range(3))
        r = np.hypot(hx, hy)
        phi = np.arctan2(hy, hx)
        for k in range(ncand):
            n1 = g.standard_normal(n) * spread
            n2 = g.standard_normal(n) * spread
            if ts.mode == MODE_R:
                ph = phi + n1 * SIGMA_RPHI / r
                c, sn = np.cos(ph), np.sin(ph)
                pos = (r * c, r * sn, hz + n2 * SIGMA_2)
                cov = (a * sn * sn, -a * sn * c, a * c * c, 0.0 * c, 0.0 * c, np.full(n, b))
            else:
                ux, uy = hx / r, hy / r
                x = hx + n1 * SIGMA_RPHI * -uy + n2 * SIGMA_2 * ux
                y = hy + n1 * SIGMA_RPHI * ux + n2 * SIGMA_2 * uy
                rr = np.hypot(x, y)
                vx, vy = x / rr, y / rr
                tx, ty = -vy, vx
                pos = (x, y, hz)
                cov = (a * tx * tx + b * vx * vx, a * ty * tx + b * vy * vx,
                       a * ty * ty + b * vy * vy, 0.0 * x, 0.0 * x, 0.0 * x)
            mine = true_slot[l] == k
            for j in range(3):
                cpos[l, k, j] = np.where(mine, ts.hpos[l, j], pos[j])
            for j in range(6):
                ccov[l, k, j] = np.where(mine, ts.hcov[l, j], cov[j])
    return CandidateSet(cpos, ccov, true_slot)


# Layout of the arrays for fit_propagate_update_layout (FIT_LAYOUT_AOSOA32):
# tiles of 32 consecutive tracks, each component of a tile contiguous.


def to_aosoa32(a: np.ndarray, ld: int) -> np.ndarray:
    """(K, n) or (nlayer, k, n) SoA -> flat AoSoA with tiles of 32 tracks over ld slots."""
    a = np.asarray(a)
    K = int(np.prod(a.shape[:-1]))
    s = np.zeros((K, ld), a.dtype)
    s[:, :a.shape[-1]] = a.reshape(K, -1)
    return np.ascontiguousarray(s.reshape(K, ld // 32, 32).transpose(1, 0, 2)).reshape(-1)


def from_aosoa32(a, shape, n: int) -> np.ndarray:
    """Inverse of to_aosoa32 for arrays of `shape` (..., ld): returns (..., n)."""
    a = np.asarray(a)
    K, ld = int(np.prod(shape[:-1])), shape[-1]
    return a.reshape(ld // 32, K, 32).transpose(1, 0, 2).reshape(shape)[..., :n]
