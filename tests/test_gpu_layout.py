"""fit_propagate_update_layout with the AoSoA layout (tiles of 32 tracks, the
paper's Matriplex-style blocks): the same arithmetic on the same tracks, so
the results must be bit-identical to the structure-of-arrays path."""
import numpy as np
import pytest

from paper_2409_09228_gb300 import fit, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA device", allow_module_level=True)

import gpu_util  # noqa: E402


@pytest.mark.parametrize("nevt,median", [(12, 2000.0), (5, 37.0)])
def test_aosoa_is_bit_identical_to_soa(nevt, median):
    nt = inputs.uneven_event_sizes(nevt, 5 + nevt, median=median, lo=1, hi=6000)
    md = inputs.uneven_event_modes(nevt, 5 + nevt)
    ev = inputs.generate_events(nt, md, seed=5 + nevt)
    n = ev.n
    ld = (n + 31) // 32 * 32
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1]))
    try:
        d = [gpu_util.to_dev(a, ld) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]
        soa = f.run(*d, ev.ntrk, ev.mode, layers=True)
        st_soa = f.sync()
        up = lambda a: torch.from_numpy(inputs.to_aosoa32(a, ld)).cuda()  # noqa: E731
        ai = [up(a) for a in (ev.par0, ev.cov0)] + [gpu_util.to_dev(ev.q, ld)] + \
             [up(a) for a in (ev.hpos, ev.hcov)]
        out = {"par": torch.empty(6 * ld, device="cuda"), "cov": torch.empty(21 * ld, device="cuda"),
               "q": torch.empty(ld, dtype=torch.int32, device="cuda"),
               "chi2": torch.empty(ld, device="cuda"),
               "chi2_layer": torch.empty(20 * ld, device="cuda"),
               "status": torch.empty(ld, dtype=torch.uint8, device="cuda")}
        fit.fit_propagate_update_layout(f.h, *ai, ev.ntrk, ev.mode, fit.FIT_LAYOUT_AOSOA32, ld,
                                        out["par"], out["cov"], out["q"], out["chi2"],
                                        chi2_layer=out["chi2_layer"], status=out["status"])
        st = f.sync()
        back = {"par": inputs.from_aosoa32(out["par"].cpu().numpy(), (6, ld), n),
                "cov": inputs.from_aosoa32(out["cov"].cpu().numpy(), (21, ld), n),
                "chi2_layer": inputs.from_aosoa32(out["chi2_layer"].cpu().numpy(), (20, ld), n),
                "q": out["q"].cpu().numpy()[:n], "chi2": out["chi2"].cpu().numpy()[:n],
                "status": out["status"].cpu().numpy()[:n]}
        for k, v in back.items():
            ref = soa[k].cpu().numpy()[..., :n]
            assert np.array_equal(v.view(np.uint8), ref.view(np.uint8)), k
        assert st == st_soa
        with pytest.raises(fit.FitError):  # slots not a multiple of 32
            fit.fit_propagate_update_layout(f.h, *ai, ev.ntrk, ev.mode, fit.FIT_LAYOUT_AOSOA32,
                                            ld + 4, out["par"], out["cov"], out["q"], out["chi2"])
    finally:
        f.close()
