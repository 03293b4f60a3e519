"""The FP64 variant (fit_propagate_update_f64) against the FP64 oracle on the
same inputs: with every operation in double the two differ only by rounding
and by where the p2r iteration stops, so the tolerance is RTOL_F64 = 1e-11
instead of the FP32 path's 1e-4.

The p2r iteration runs with tol = 1e-12 R here (TOL_F64), the setting for a
double fit: the iteration stops once its step d is below tol R, and the
Jacobian is taken from the helix quantities of the last iterate, one step d
short of the root, which costs ~kappa d relative (kappa <= 0.017 / cm).  At
the FP32 path's default 1e-6 R that is ~1e-6, far below FP32's tolerance but
the whole error of a double fit; at 1e-12 R it is ~2e-12.

RTOL_F64 = 1e-11: what is left is rounding, a few
units of 2^-53 per operation through ~20 layers of ~1e3 operations (~1e-13
relative on parameters and covariance, measured 7e-13 worst on an emulation of
the same code), and for chi2 the rounding of ~100 cm positions
(2^-53 * 110 cm = 1.2e-14 cm) against sigma = 0.01 cm hits, summed over 20
layers as for the FP32 path's CHI2_ABS, ~5e-11 sqrt(chi2) at most (CHI2_ABS_F64 = 1e-10, a factor 2).
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

RTOL_F64 = 1e-11
CHI2_ABS_F64 = 1e-10
TOL_F64 = 1e-12


def _dev64(a, ld):
    pad = [(0, 0)] * (a.ndim - 1) + [(0, ld - a.shape[-1])]
    a = np.pad(a, pad)
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.float64) if a.dtype.kind == "f" else a)).cuda()


def _run64(f, ts, layers=True):
    n = ts.n
    ld = n + 3
    d = [_dev64(a, ld) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    dev = torch.device("cuda")
    out = {"par": torch.empty((6, ld), dtype=torch.float64, device=dev),
           "cov": torch.empty((21, ld), dtype=torch.float64, device=dev),
           "q": torch.empty(ld, dtype=torch.int32, device=dev),
           "chi2": torch.empty(ld, dtype=torch.float64, device=dev),
           "chi2_layer": torch.empty((ts.nlayer, ld), dtype=torch.float64, device=dev) if layers else None,
           "status": torch.empty(ld, dtype=torch.uint8, device=dev)}
    fit.fit_propagate_update_f64(f.h, *d, [n], [ts.mode], out["par"], out["cov"], out["q"],
                                 out["chi2"], chi2_layer=out["chi2_layer"], status=out["status"])
    st = f.sync()
    return {k: v.cpu().numpy()[..., :n] for k, v in out.items() if v is not None}, st


@pytest.mark.parametrize("mode", [inputs.MODE_R, inputs.MODE_Z], ids=["p2r", "p2z"])
@pytest.mark.parametrize("n", [1024, 4097])
def test_f64_matches_oracle_to_1e11(mode, n):
    ts = inputs.generate(mode, n, seed=1)
    geom = fit.Geometry(ts.B, ts.surf, tol=TOL_F64)
    f = fit.Fitter(geom if mode == 0 else None, geom if mode == 1 else None)
    try:
        got, st = _run64(f, ts)
        ref = oracle.fit_set(ts)
        res = parity.check(got, ref, f"f64 {mode} {n}", rtol=RTOL_F64, chi2_abs=CHI2_ABS_F64)
        print(f"\nf64 mode {mode} n {n}: worst in units of the 1e-11 tolerance {res['worst']}")
        assert (got["status"] == 0).all() and st["tracks"] == n
        assert np.allclose(got["chi2_layer"].sum(axis=0), got["chi2"], rtol=1e-12)
        # and it is far tighter than the FP32 path on the same tracks
        e = parity.scaled_errors(got, ref)
        assert e["par"].max() < 1e-3 and e["cov"].max() < 1e-3
    finally:
        f.close()


def test_f64_stopped_tracks_and_errors():
    surf = inputs.surfaces(inputs.MODE_R)
    n = 64
    gap = float(surf[1] - surf[0])
    pt = np.where(np.arange(n) % 2 == 0, np.linspace(0.8, 8.0, n),
                  (surf[12].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2)
    ts = inputs.generate(inputs.MODE_R, n, seed=71, pt=pt)
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf, tol=TOL_F64), None)
    try:
        got, st = _run64(f, ts)
        ref = oracle.fit_set(ts)
        assert np.array_equal(got["status"] & 1, ref["status"] & 1)
        assert st["no_intersection"] == n // 2
        stopped = (got["status"] & 1) != 0
        assert (got["chi2_layer"][13:, stopped] == 0).all()
        # the stopped tracks hold their state at the last reached layer, as the oracle's
        e = parity.scaled_errors(got, ref, RTOL_F64, CHI2_ABS_F64)
        assert e["par"].max() <= 1 and e["chi2"].max() <= 1
        with pytest.raises(ValueError):  # float32 buffers are refused by the binding
            d = [gpu_util.to_dev(a, gpu_util.pad_ld(n)) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
            fit.fit_propagate_update_f64(f.h, *d, [n], [0], d[0], d[1], d[2],
                                         torch.empty(gpu_util.pad_ld(n), device="cuda"))
    finally:
        f.close()
