"""fit_propagate_update_noalloc against fit_propagate_update (GPU, through the C ABI).

The no-allocation entry point serves callers that must not allocate device
memory while they run (an online trigger process that reserves its GPU memory
at start-up, a plug-in inside a framework that owns the device memory).  It
keeps its scratch (per-event counters, event offsets) in a fixed array inside
the library, so it must give the same fit as the handle-based entry point on
every call, and clear its counters between calls; the fit is also checked
against the FP64 oracle, and the free device memory is checked to be
unchanged by a call once the library's kernels are loaded.  This file is
collected last so that a run stopping at the first failure has run every
other test.
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


def _events():
    """Mixed-mode events of uneven size, some with tracks that stop early."""
    surf_r = inputs.surfaces(inputs.MODE_R)
    gap = float(surf_r[1] - surf_r[0])
    loop_pt = (surf_r[9].astype(np.float64) + 0.5 * gap) * inputs.KA * float(np.float32(3.8)) / 2
    n_loop = 200
    pt = np.where(np.arange(n_loop) % 2 == 0, np.linspace(0.8, 8.0, n_loop), loop_pt)
    return [inputs.generate(inputs.MODE_R, 300, seed=501),
            inputs.generate(inputs.MODE_R, n_loop, seed=502, pt=pt),
            inputs.generate(inputs.MODE_Z, 250, seed=503),
            inputs.generate(inputs.MODE_R, 0, seed=504),
            inputs.generate(inputs.MODE_R, 129, seed=505),
            inputs.generate(inputs.MODE_Z, 5, seed=506),
            inputs.generate(inputs.MODE_R, 1000, seed=507)]


def test_noalloc_matches_handle_path_on_two_calls():
    sets = _events()
    ntrk = [s.n for s in sets]
    modes = [s.mode for s in sets]
    geom_r = fit.Geometry(sets[0].B, inputs.surfaces(inputs.MODE_R))
    geom_z = fit.Geometry(sets[0].B, inputs.surfaces(inputs.MODE_Z))
    c = gpu_util.concat(sets)
    n = c["par0"].shape[-1]
    ld = gpu_util.pad_ld(n)
    dev_in = [gpu_util.to_dev(c[k], ld) for k in ("par0", "cov0", "q", "hpos", "hcov")]

    # reference: the handle-based entry point
    f = fit.Fitter(geom_r, geom_z)
    ref = f.run(*dev_in, ntrk, modes)
    ref_sync = f.sync()
    f.close()
    ref_np = {k: v.cpu().numpy()[..., :n] for k, v in ref.items() if v is not None}
    starts = np.concatenate([[0], np.cumsum(ntrk)])

    # every output buffer exists before the first call, so that the free
    # device memory measured around the second call sees only the library
    outs = [{"par": torch.full((6, ld), float("nan"), device="cuda"),
             "cov": torch.full((21, ld), float("nan"), device="cuda"),
             "q": torch.zeros(ld, dtype=torch.int32, device="cuda"),
             "chi2": torch.full((ld,), float("nan"), device="cuda"),
             "status": torch.full((ld,), 255, dtype=torch.uint8, device="cuda")}
            for _ in range(2)]
    oracle_events = [oracle.fit_set(s) if s.n else None for s in sets]
    for call in range(2):
        out = outs[call]
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        per_event = fit.fit_propagate_update_noalloc(
            geom_r, geom_z, *dev_in, ntrk, modes, par_out=out["par"], cov_out=out["cov"],
            q_out=out["q"], chi2=out["chi2"], status=out["status"])
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the library's kernels; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        got = {k: v.cpu().numpy()[..., :n] for k, v in out.items()}
        # same outputs as the handle path, within the parity tolerance
        s = parity.check(got, ref_np, f"no-alloc call {call}")
        assert s["compared"] == int((ref_np["status"] == 0).sum())
        # and the same fit as the FP64 oracle, event by event
        for e, ref_e in enumerate(oracle_events):
            if ref_e is not None:
                sub = {k: v[..., starts[e]:starts[e + 1]] for k, v in got.items()}
                parity.check(sub, ref_e, f"no-alloc call {call} event {e} vs oracle")
        assert np.array_equal(got["status"], ref_np["status"])
        assert np.array_equal(got["q"], ref_np["q"])
        # per-event counters: fresh on each call and consistent with the statuses
        assert len(per_event) == len(sets)
        for e in range(len(sets)):
            st = ref_np["status"][starts[e]:starts[e + 1]]
            assert per_event[e]["tracks"] == ntrk[e]
            assert per_event[e]["no_intersection"] == int(((st & 1) != 0).sum())
            assert per_event[e]["not_converged"] == int(((st & 2) != 0).sum())
            assert per_event[e]["nonfinite"] == int(((st & 4) != 0).sum())
            if modes[e] == inputs.MODE_Z or ntrk[e] == 0:
                assert per_event[e]["iterations"] == 0
        assert per_event[1]["no_intersection"] == 100
        assert sum(p["iterations"] for p in per_event) == ref_sync["iterations"]
        assert sum(p["no_intersection"] for p in per_event) == ref_sync["no_intersection"]


def test_noalloc_rejects_too_many_events():
    geom_r = fit.Geometry(3.8, inputs.surfaces(inputs.MODE_R))
    nevt = fit.FIT_NOALLOC_MAX_EVENTS + 1
    ld = 4
    t = lambda *shape: torch.zeros(shape, device="cuda")  # noqa: E731
    with pytest.raises(fit.FitError) as e:
        fit.fit_propagate_update_noalloc(geom_r, None, t(6, ld), t(21, ld),
                                         torch.ones(ld, dtype=torch.int32, device="cuda"),
                                         t(20, 3, ld), t(20, 6, ld), [0] * nevt, [0] * nevt,
                                         chi2=t(ld))
    assert e.value.code == fit.FIT_ERR_ARG
    assert "FIT_NOALLOC_MAX_EVENTS" in str(e.value)


def test_noalloc_at_the_event_limit():
    """FIT_NOALLOC_MAX_EVENTS events (the limit) of one track each, modes
    alternating in runs: every event's counters are its own track's."""
    nevt = fit.FIT_NOALLOC_MAX_EVENTS
    modes = (np.arange(nevt) // 7) % 2
    sets = [inputs.generate(inputs.MODE_R, int((modes == 0).sum()), seed=511),
            inputs.generate(inputs.MODE_Z, int((modes == 1).sum()), seed=512)]
    order = np.argsort(np.argsort(modes, kind="stable"), kind="stable")  # rank within the sorted pools
    pools = gpu_util.concat(sets)
    c = {k: v[..., order] for k, v in pools.items()}
    ld = gpu_util.pad_ld(nevt)
    dev_in = [gpu_util.to_dev(c[k], ld) for k in ("par0", "cov0", "q", "hpos", "hcov")]
    geom_r = fit.Geometry(sets[0].B, inputs.surfaces(inputs.MODE_R))
    geom_z = fit.Geometry(sets[0].B, inputs.surfaces(inputs.MODE_Z))
    out = {"par": torch.empty((6, ld), device="cuda"), "cov": torch.empty((21, ld), device="cuda"),
           "q": torch.empty(ld, dtype=torch.int32, device="cuda"),
           "chi2": torch.empty(ld, device="cuda"),
           "status": torch.empty(ld, dtype=torch.uint8, device="cuda")}
    per_event = fit.fit_propagate_update_noalloc(
        geom_r, geom_z, *dev_in, [1] * nevt, modes.tolist(), par_out=out["par"],
        cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"], status=out["status"])
    assert len(per_event) == nevt
    assert all(p["tracks"] == 1 for p in per_event)
    st = out["status"].cpu().numpy()[:nevt]
    assert (st == 0).all() and all(p["no_intersection"] == 0 for p in per_event)
    it = np.array([p["iterations"] for p in per_event])
    assert (it[modes == 1] == 0).all() and (it[modes == 0] >= 20).all()
    # and the fit agrees with the handle path on the same tracks
    f = fit.Fitter(geom_r, geom_z)
    ref = f.run(*dev_in, [1] * nevt, modes.tolist())
    f.close()
    got = {k: v.cpu().numpy()[..., :nevt] for k, v in out.items()}
    parity.check(got, {k: v.cpu().numpy()[..., :nevt] for k, v in ref.items() if v is not None},
                 "no-alloc at the event limit")
