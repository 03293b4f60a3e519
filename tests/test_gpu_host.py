"""fit_propagate_update_host: the fused fit on host buffers, copied through
the library's three staging sets in chunks of FIT_HOST_CHUNK tracks.  Its results must
be bit-identical to fit_propagate_update on the same data in device memory:
chunks start at even track indices, so every track meets the same kernel with
the same pairing."""
import numpy as np
import pytest

from paper_2409_09228_gb300 import fit, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA device", allow_module_level=True)

import gpu_util  # noqa: E402


def _events(nevt, seed, median):
    nt = inputs.uneven_event_sizes(nevt, seed, median=median, lo=1, hi=40000)
    nt[[i for i in (2, 5) if i < nevt]] = 0
    md = inputs.uneven_event_modes(nevt, seed)
    return inputs.generate_events(nt, md, seed=seed)


def _host(ev, ld, pinned):
    def h(a):
        a = np.ascontiguousarray(np.pad(a, [(0, 0)] * (a.ndim - 1) + [(0, ld - a.shape[-1])]))
        return torch.from_numpy(a).pin_memory() if pinned else a
    return [h(a) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]


def _host_out(n, ld, nlayer, pinned):
    def e(shape, dtype):
        t = torch.full(shape, 7, dtype=dtype)
        return t.pin_memory() if pinned else t.numpy()
    return {"par": e((6, ld), torch.float32), "cov": e((21, ld), torch.float32),
            "q": e((ld,), torch.int32), "chi2": e((ld,), torch.float32),
            "chi2_layer": e((nlayer, ld), torch.float32), "status": e((ld,), torch.uint8)}


def _np(x, n):
    return (x.numpy() if hasattr(x, "numpy") else np.asarray(x))[..., :n]


@pytest.mark.parametrize("nevt,median,pinned", [(60, 9000.0, True), (7, 100.0, False)])
def test_host_path_is_bit_identical_to_device_path(nevt, median, pinned):
    ev = _events(nevt, 91 + nevt, median)
    n = ev.n
    ld = gpu_util.pad_ld(n) + 4
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1]))
    try:
        d = [gpu_util.to_dev(a, ld) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]
        dev = f.run(*d, ev.ntrk, ev.mode, layers=True)
        st_dev = f.sync()
        hin = _host(ev, ld, pinned)
        hout = _host_out(n, ld, 20, pinned)
        fit.fit_propagate_update_host(f.h, *hin, ev.ntrk, ev.mode, par_out=hout["par"],
                                      cov_out=hout["cov"], q_out=hout["q"], chi2=hout["chi2"],
                                      chi2_layer=hout["chi2_layer"], status=hout["status"])
        st_host = f.sync()
        for k in ("par", "cov", "q", "chi2", "chi2_layer", "status"):
            a, b = dev[k].cpu().numpy()[..., :n], _np(hout[k], n)
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k
        assert st_host == st_dev
        if pinned:
            assert n > 2 * fit.FIT_HOST_CHUNK  # several chunks, events straddling their edges
    finally:
        f.close()


def test_host_path_in_place_and_seeded():
    ev = _events(12, 17, 3000.0)
    n = ev.n
    ld = gpu_util.pad_ld(n)
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1]))
    m = fit.fit_mlp_create(0, seed=3)
    try:
        fit.fit_mlp_attach(f.h, m)
        d = [gpu_util.to_dev(a, ld) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]
        dev = f.run(*d, ev.ntrk, ev.mode)
        f.sync()
        hin = _host(ev, ld, True)
        chi2 = torch.empty(ld).pin_memory()
        fit.fit_propagate_update_host(f.h, *hin, ev.ntrk, ev.mode, chi2=chi2)  # in place
        f.sync()
        assert np.array_equal(dev["par"].cpu().numpy()[:, :n], hin[0].numpy()[:, :n])
        assert np.array_equal(dev["cov"].cpu().numpy()[:, :n], hin[1].numpy()[:, :n])
        assert np.array_equal(dev["chi2"].cpu().numpy()[:n], chi2.numpy()[:n])
    finally:
        f.close()
        fit.fit_mlp_destroy(m)


def test_host_path_argument_errors():
    ev = _events(3, 5, 50.0)
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), None)
    try:
        hin = _host(ev, gpu_util.pad_ld(ev.n), False)
        with pytest.raises(fit.FitError):  # p2z events, p2z not configured
            fit.fit_propagate_update_host(f.h, *hin, ev.ntrk, np.ones(3, np.int32),
                                          chi2=np.zeros(gpu_util.pad_ld(ev.n), np.float32))
        with pytest.raises(ValueError):
            d = gpu_util.to_dev(ev.par0, gpu_util.pad_ld(ev.n))
            fit.fit_propagate_update_host(f.h, d, *hin[1:], ev.ntrk, ev.mode)
    finally:
        f.close()


def test_mapped_path_is_bit_identical_and_checks_its_pointers():
    """fit_propagate_update_mapped: the fused kernels read the tracks and hits
    from page-locked host memory and write the outputs there, with no staging
    copy.  Same kernels on the same values: bit-identical to the device path.
    Pageable or device buffers are refused before anything runs."""
    ev = _events(9, 29, 4000.0)
    n = ev.n
    ld = gpu_util.pad_ld(n) + 4
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1]))
    try:
        d = [gpu_util.to_dev(a, ld) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]
        dev = f.run(*d, ev.ntrk, ev.mode, layers=True)
        st_dev = f.sync()
        hin = _host(ev, ld, True)
        hout = _host_out(n, ld, 20, True)
        outs = dict(par_out=hout["par"], cov_out=hout["cov"], q_out=hout["q"], chi2=hout["chi2"],
                    chi2_layer=hout["chi2_layer"], status=hout["status"])
        fit.fit_propagate_update_mapped(f.h, *hin, ev.ntrk, ev.mode, **outs)
        st_map = f.sync()
        for k in ("par", "cov", "q", "chi2", "chi2_layer", "status"):
            a, b = dev[k].cpu().numpy()[..., :n], _np(hout[k], n)
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k
        assert st_map == st_dev
        # refused: a pageable input, a pageable output; the outputs stay untouched
        before = hout["chi2"].clone()
        pageable = [np.array(t.numpy()) for t in hin]
        with pytest.raises(fit.FitError) as e:
            fit.fit_propagate_update_mapped(f.h, pageable[0], *hin[1:], ev.ntrk, ev.mode, **outs)
        assert e.value.code == fit.FIT_ERR_ARG and "page-locked" in str(e.value)
        with pytest.raises(fit.FitError) as e:
            fit.fit_propagate_update_mapped(f.h, *hin, ev.ntrk, ev.mode,
                                            **{**outs, "chi2": torch.empty(ld).numpy()})
        assert e.value.code == fit.FIT_ERR_ARG
        torch.cuda.synchronize()
        assert torch.equal(before, hout["chi2"])
    finally:
        f.close()
