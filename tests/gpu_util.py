"""Helpers for the GPU tests: upload a TrackSet, run libfit, fetch the outputs."""
from __future__ import annotations

import numpy as np
import torch

from paper_2409_09228_gb300 import fit, inputs


def pad_ld(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


def to_dev(a: np.ndarray, ld: int, fill=0) -> torch.Tensor:
    pad = [(0, 0)] * (a.ndim - 1) + [(0, ld - a.shape[-1])]
    return torch.from_numpy(np.ascontiguousarray(np.pad(a, pad, constant_values=fill))).cuda()


def concat(sets):
    """Concatenates TrackSets (events) along the track axis."""
    cat = lambda name: np.concatenate([getattr(s, name) for s in sets], axis=-1)  # noqa: E731
    return {k: cat(k) for k in ("par0", "cov0", "q", "hpos", "hcov")}


def run(sets, geom_r=None, geom_z=None, ld=None, layers=False, in_place=False, max_iter=10,
        tol=1e-6, start=fit.FIT_START_CROSSING):
    """Fits the events `sets` (one TrackSet per event) in one fit_propagate_update call."""
    B = sets[0].B
    if geom_r is None and any(s.mode == inputs.MODE_R for s in sets):
        geom_r = fit.Geometry(B, next(s.surf for s in sets if s.mode == inputs.MODE_R), max_iter, tol,
                              start)
    if geom_z is None and any(s.mode == inputs.MODE_Z for s in sets):
        geom_z = fit.Geometry(B, next(s.surf for s in sets if s.mode == inputs.MODE_Z), max_iter, tol,
                              start)
    f = fit.Fitter(geom_r, geom_z)
    c = concat(sets)
    n = c["par0"].shape[-1]
    ld = ld or pad_ld(n)
    par, cov, q = to_dev(c["par0"], ld), to_dev(c["cov0"], ld), to_dev(c["q"], ld)
    hpos, hcov = to_dev(c["hpos"], ld), to_dev(c["hcov"], ld)
    if in_place:
        out = {"par": par, "cov": cov, "q": q, "chi2": torch.empty(ld, device="cuda"),
               "status": torch.empty(ld, dtype=torch.uint8, device="cuda"),
               "chi2_layer": torch.empty((hpos.shape[0], ld), device="cuda") if layers else None}
    else:
        out = f.outputs(n, ld=ld, layers=layers)
        for k in ("par", "cov", "chi2"):
            out[k].fill_(float("nan"))
    f.run(par, cov, q, hpos, hcov, [s.n for s in sets], [s.mode for s in sets], out=out)
    st = f.sync()
    f.close()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["sync"] = st
    res["n"] = n
    return res


def trim(res, lo, hi):
    return {k: (v[..., lo:hi] if isinstance(v, np.ndarray) else v) for k, v in res.items()}
