"""FP64 CPU oracle of the fused propagate + Kalman-update track fit.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  The
GPU library (``paper_2409_09228_gb300``) never imports it, and the two share
no code: the oracle is ``oracle/oracle.cpp`` + ``oracle/dual.hpp`` (C++17,
double precision), loaded here through ctypes.

What the oracle computes is stated in the header of ``oracle.cpp``: the
textbook helix in a uniform solenoidal field (paper Sec. 3), the exact
surface intersection (closed form for planes, the exact first root for
cylinders), the transport Jacobian as the derivative of the
propagate-to-surface map, and the Kalman update with the hit's 2-D position
on the surface (paper Sec. 3.2).

Array layouts (track index fastest): par (6, n), cov (21, n) packed lower
triangle, q (n,), hit positions (nlayer, 3, n), hit covariances (nlayer, 6, n).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.cpp"), os.path.join(_HERE, "dual.hpp")]

MODE_R = 0
MODE_Z = 1
ST_NO_INTERSECTION = 1
ST_NOT_CONVERGED = 2
ST_NONFINITE = 4
ST_CHARGE_FLIP = 8


def build_command(out: str = LIB_PATH) -> list:
    # -ffp-contract=off: the same rounding on x86-64 and aarch64 hosts.
    return ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
            "-pthread", os.path.join(_HERE, "oracle.cpp"), "-o", out]


def build(force: bool = False) -> str:
    """Compiles liboracle.so in place (skipped when it is newer than its sources)."""
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in _SRC):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(build_command(tmp), check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t=_D):
    return a.ctypes.data_as(t)


class Oracle:
    """ctypes view of one compiled oracle library (the default one, or a test copy)."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        L.orc_helix.argtypes = [ctypes.c_double, ctypes.c_int, _D, ctypes.c_double, _D]
        L.orc_path_length.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, _D, _D]
        L.orc_transport.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, _D, _D, _D, _D]
        L.orc_propagate.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, _D, _D, _D, _D]
        L.orc_update.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D, _I, _D]
        L.orc_fit.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, ctypes.c_int64,
                              _D, _D, _I, _D, _D, _D, _D, _I, _D, _D, _U8, ctypes.c_int]
        L.orc_find.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, ctypes.c_int64, _D,
                               _D, _I, ctypes.c_int, _D, _D, ctypes.c_double, _D, _D, _I, _D, _D,
                               _I, _D, _U8, ctypes.c_int]
        L.orc_path_lengths.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int64, _D, _I, _D,
                                       _D, _U8, ctypes.c_int]
        L.orc_chi2_grad.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D,
                                    ctypes.c_int64, _D, _D, _I, _D, _D, _D, _D, _D, _U8,
                                    ctypes.c_int]
        self.L = L
        self.path = path

    def helix(self, B: float, q: int, p, h: float) -> np.ndarray:
        """State after transverse path length h along the helix (no surface)."""
        p = _d(p)
        out = np.zeros(6)
        self.L.orc_helix(B, int(q), _p(p), float(h), _p(out))
        return out

    def path_length(self, mode: int, B: float, s: float, q: int, p):
        """(status, h): transverse path length to surface s."""
        p = _d(p)
        h = np.zeros(1)
        st = self.L.orc_path_length(mode, B, s, int(q), _p(p), _p(h))
        return st, float(h[0])

    def path_lengths(self, mode: int, B: float, s, q, p, nthreads: int = 0):
        """(h, status) for n states p (6, n) with charges q (n,) to surfaces s (n,)."""
        s, p = _d(s), _d(p)
        q = np.ascontiguousarray(q, dtype=np.int32)
        n = p.shape[1]
        h, st = np.zeros(n), np.zeros(n, np.uint8)
        self.L.orc_path_lengths(mode, B, n, _p(s), _p(q, _I), _p(p), _p(h), _p(st, _U8), nthreads)
        return h, st

    def transport(self, mode: int, B: float, s: float, q: int, p):
        """(status, p_out, J (6x6), h) of the propagate-to-surface map."""
        p = _d(p)
        pout, J, h = np.zeros(6), np.zeros(36), np.zeros(1)
        st = self.L.orc_transport(mode, B, s, int(q), _p(p), _p(pout), _p(J), _p(h))
        return st, pout, J.reshape(6, 6), float(h[0])

    def propagate(self, mode: int, B: float, s: float, q: int, p, cov21):
        """(status, p_out, cov21_out): one propagation step."""
        p, c = _d(p), _d(cov21)
        pout, cout = np.zeros(6), np.zeros(21)
        st = self.L.orc_propagate(mode, B, s, int(q), _p(p), _p(c), _p(pout), _p(cout))
        return st, pout, cout

    def update(self, mode: int, q: int, p, cov21, m, hcov6):
        """(status, p_out, cov21_out, q_out, chi2): one Kalman update."""
        p, c, m, v = _d(p), _d(cov21), _d(m), _d(hcov6)
        pout, cout, qo, chi2 = np.zeros(6), np.zeros(21), np.zeros(1, np.int32), np.zeros(1)
        st = self.L.orc_update(mode, int(q), _p(p), _p(c), _p(m), _p(v), _p(pout), _p(cout),
                               _p(qo, _I), _p(chi2))
        return st, pout, cout, int(qo[0]), float(chi2[0])

    def fit(self, mode: int, B: float, surf, par0, cov0, q0, hpos, hcov, nthreads: int = 0,
            want_layers: bool = False) -> dict:
        """Full layer-by-layer fit of n tracks (inputs promoted to float64)."""
        surf = _d(surf)
        par0, cov0, hpos, hcov = _d(par0), _d(cov0), _d(hpos), _d(hcov)
        q0 = np.ascontiguousarray(q0, dtype=np.int32)
        nlayer, n = hpos.shape[0], par0.shape[1]
        assert par0.shape == (6, n) and cov0.shape == (21, n) and q0.shape == (n,)
        assert hpos.shape == (nlayer, 3, n) and hcov.shape == (nlayer, 6, n)
        assert surf.shape == (nlayer,)
        par, cov = np.zeros((6, n)), np.zeros((21, n))
        q, chi2 = np.zeros(n, np.int32), np.zeros(n)
        cl = np.zeros((nlayer, n)) if want_layers else None
        status = np.zeros(n, np.uint8)
        self.L.orc_fit(mode, B, nlayer, _p(surf), n, _p(par0), _p(cov0), _p(q0, _I), _p(hpos),
                       _p(hcov), _p(par), _p(cov), _p(q, _I), _p(chi2),
                       _p(cl) if cl is not None else None, _p(status, _U8), nthreads)
        return {"par": par, "cov": cov, "q": q, "chi2": chi2, "chi2_layer": cl,
                "status": status}

    def fit_set(self, ts, nthreads: int = 0, want_layers: bool = False) -> dict:
        """fit() on a TrackSet from paper_2409_09228_gb300.inputs."""
        return self.fit(ts.mode, ts.B, ts.surf, ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov,
                        nthreads=nthreads, want_layers=want_layers)

    def find(self, mode: int, B: float, surf, par0, cov0, q0, cpos, ccov, gate: float,
             nthreads: int = 0) -> dict:
        """Track finding: per layer the candidate (cpos (nlayer, ncand, 3, n), ccov
        (nlayer, ncand, 6, n)) with the smallest chi2 below the gate updates the
        track, or none; returns the fit outputs, chosen (nlayer, n) (-1 = none)
        and the chi2 of every candidate tried (nlayer, ncand, n)."""
        surf = _d(surf)
        par0, cov0, cpos, ccov = _d(par0), _d(cov0), _d(cpos), _d(ccov)
        q0 = np.ascontiguousarray(q0, dtype=np.int32)
        nlayer, ncand, _, n = cpos.shape
        par, cov = np.zeros((6, n)), np.zeros((21, n))
        q, chi2 = np.zeros(n, np.int32), np.zeros(n)
        cl = np.zeros((nlayer, n))
        chosen = np.zeros((nlayer, n), np.int32)
        cc = np.zeros((nlayer, ncand, n))
        status = np.zeros(n, np.uint8)
        self.L.orc_find(mode, B, nlayer, _p(surf), n, _p(par0), _p(cov0), _p(q0, _I), ncand,
                        _p(cpos), _p(ccov), float(gate), _p(par), _p(cov), _p(q, _I), _p(chi2),
                        _p(cl), _p(chosen, _I), _p(cc), _p(status, _U8), nthreads)
        return {"par": par, "cov": cov, "q": q, "chi2": chi2, "chi2_layer": cl,
                "chosen": chosen, "cand_chi2": cc, "status": status}

    def chi2_grad(self, mode: int, B: float, surf, par0, cov0, q0, hpos, hcov,
                  nthreads: int = 0) -> dict:
        """Gradient of each track's summed chi2 w.r.t. its initial parameters and hits."""
        surf = _d(surf)
        par0, cov0, hpos, hcov = _d(par0), _d(cov0), _d(hpos), _d(hcov)
        q0 = np.ascontiguousarray(q0, dtype=np.int32)
        nlayer, n = hpos.shape[0], par0.shape[1]
        chi2, gp, gh = np.zeros(n), np.zeros((6, n)), np.zeros((nlayer, 3, n))
        status = np.zeros(n, np.uint8)
        self.L.orc_chi2_grad(mode, B, nlayer, _p(surf), n, _p(par0), _p(cov0), _p(q0, _I),
                             _p(hpos), _p(hcov), _p(chi2), _p(gp), _p(gh), _p(status, _U8),
                             nthreads)
        return {"chi2": chi2, "g_par0": gp, "g_hpos": gh, "status": status}


_default = None


def default() -> Oracle:
    """The oracle built from oracle.cpp (compiled on first use)."""
    global _default
    if _default is None:
        _default = Oracle(build())
    return _default


def helix(*a, **k):
    return default().helix(*a, **k)


def path_length(*a, **k):
    return default().path_length(*a, **k)


def transport(*a, **k):
    return default().transport(*a, **k)


def path_lengths(*a, **k):
    return default().path_lengths(*a, **k)


def propagate(*a, **k):
    return default().propagate(*a, **k)


def update(*a, **k):
    return default().update(*a, **k)


def fit(*a, **k):
    return default().fit(*a, **k)


def fit_set(*a, **k):
    return default().fit_set(*a, **k)


def chi2_grad(*a, **k):
    return default().chi2_grad(*a, **k)


def find(*a, **k):
    return default().find(*a, **k)


def unpack_sym6(c21) -> np.ndarray:
    """6x6 symmetric matrix from its packed lower triangle (row-major)."""
    M = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            M[i, j] = M[j, i] = c21[k]
            k += 1
    return M


def pack_sym6(M) -> np.ndarray:
    return np.array([M[i, j] for i in range(6) for j in range(i + 1)])
