"""Element-wise comparison of a fit's FP32 outputs with the FP64 oracle.

Tolerances (GPU FP32 vs oracle FP64 on the same FP32-rounded inputs):

* parameters: |d p_k| <= RTOL * max(|p_k|, floor_k), floors (1, 1, 1 cm,
  0.1 1/GeV, 1 rad, 1 rad); phi is compared modulo 2 pi;
* covariance: |d C_ij| <= RTOL * sqrt(s_i s_j) with s_k = C_kk, except
  s_x = s_y = C_xx + C_yy: relative to the scale of the entry, so that
  near-zero correlations are not over-weighted.  On a cylinder the propagated
  covariance is singular along the radial direction, and how that zero splits
  between x and y depends on the azimuth, so x and y share the transverse
  position variance as their scale;
* chi2 (summed over layers): |d chi2| <= RTOL * chi2 + CHI2_ABS * sqrt(chi2).
  chi2 = sum (r / sigma)^2 is a difference of positions of ~100 cm measured
  to sigma = 0.01 cm; FP32 represents such positions to ~2^-24 * 110 cm =
  6.6e-6 cm, so each residual r carries ~e = 6.6e-4 sigma of unavoidable
  rounding and chi2 moves by ~2 |r| e / sigma.  Summed over layers this is
  2 e sqrt(nlayer * chi2) <= CHI2_ABS sqrt(chi2) with CHI2_ABS = 2 * 6.6e-4 *
  sqrt(20) * 4 (a factor 4 for several roundings per residual) = 0.024.

RTOL is 1e-4, the relative tolerance the fit is specified to.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-4
PAR_FLOOR = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
CHI2_ABS = 0.024


def _sym_index(i, j):
    if j > i:
        i, j = j, i
    return i * (i + 1) // 2 + j


DIAG = np.array([_sym_index(i, i) for i in range(6)])
PAIRS = [(i, j) for i in range(6) for j in range(i + 1)]


def wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def scaled_errors(gpu: dict, ref: dict, rtol: float = RTOL, chi2_abs: float = CHI2_ABS) -> dict:
    """Per-track worst error of each output, in units of its tolerance (<= 1 passes)."""
    par_g, par_r = np.asarray(gpu["par"], np.float64), np.asarray(ref["par"], np.float64)
    d = par_g - par_r
    d[4] = wrap(d[4])
    e_par = np.abs(d) / (rtol * np.maximum(np.abs(par_r), PAR_FLOOR[:, None]))
    cov_g, cov_r = np.asarray(gpu["cov"], np.float64), np.asarray(ref["cov"], np.float64)
    dia = np.abs(cov_r[DIAG])
    dia[0] = dia[1] = dia[0] + dia[1]
    e_cov = np.empty_like(cov_r)
    for k, (i, j) in enumerate(PAIRS):
        scale = np.sqrt(dia[i] * dia[j])
        e_cov[k] = np.abs(cov_g[k] - cov_r[k]) / (rtol * np.maximum(scale, 1e-30))
    c_g, c_r = np.asarray(gpu["chi2"], np.float64), np.asarray(ref["chi2"], np.float64)
    e_chi2 = np.abs(c_g - c_r) / (rtol * np.abs(c_r) + chi2_abs * np.sqrt(np.abs(c_r)) + 1e-30)
    return {"par": e_par.max(axis=0), "cov": e_cov.max(axis=0), "chi2": e_chi2,
            "par_each": e_par, "cov_each": e_cov}


def strict_chi2_rate(gpu: dict, ref: dict) -> float:
    """Fraction of the tracks neither side flagged whose summed chi2 agrees
    to 1e-4 relative with a floor of 1e-3 on the tolerance,
    |d chi2| <= max(1e-4 chi2, 1e-3): the fit's specified chi2 criterion
    taken literally, without the FP32 residual-rounding term of CHI2_ABS.
    Reported beside check() so that a loss of chi2 accuracy shows even where
    it stays within the looser bound."""
    ok = (np.asarray(gpu["status"]) == 0) & (np.asarray(ref["status"]) == 0)
    c_g = np.asarray(gpu["chi2"], np.float64)[ok]
    c_r = np.asarray(ref["chi2"], np.float64)[ok]
    if not ok.any():
        return 1.0
    return float(np.mean(np.abs(c_g - c_r) <= np.maximum(RTOL * np.abs(c_r), 1e-3)))


def check(gpu: dict, ref: dict, label: str = "", rtol: float = RTOL,
          chi2_abs: float = CHI2_ABS) -> dict:
    """Asserts parity on every track that neither side flagged; returns a summary."""
    st_g = np.asarray(gpu["status"]).astype(np.uint8)
    st_r = np.asarray(ref["status"]).astype(np.uint8)
    ok = (st_g == 0) & (st_r == 0)
    e = scaled_errors(gpu, ref, rtol, chi2_abs)
    worst = {k: float(e[k][ok].max()) if ok.any() else 0.0 for k in ("par", "cov", "chi2")}
    bad = ok & ((e["par"] > 1) | (e["cov"] > 1) | (e["chi2"] > 1))
    assert not bad.any(), (
        f"{label}: {int(bad.sum())} of {int(ok.sum())} tracks out of tolerance; worst "
        f"(in tolerance units) {worst}; first bad track {int(np.nonzero(bad)[0][0])}")
    assert np.array_equal(np.asarray(gpu["q"]), np.asarray(ref["q"])) or not ok.all(), \
        f"{label}: charges differ"
    return {"tracks": int(len(ok)), "compared": int(ok.sum()), "flag_gpu": int((st_g != 0).sum()),
            "flag_ref": int((st_r != 0).sum()), "worst": worst}
