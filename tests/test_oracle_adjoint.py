"""Pins of the oracle's discrete-adjoint gradient (CPU only): it equals central
finite differences of the FP64 misfit along random smooth directions."""
import numpy as np
import pytest

import workloads as wl


def setup(ndim, seed=0):
    if ndim == 2:
        shape = (30, 36)
        src, rec = (18, 0, 6), np.array([(x, 0, 4) for x in range(4, 32, 3)], np.int32)
    else:
        shape = (14, 16, 18)
        src, rec = (9, 8, 5), np.array([(x, y, 3) for y in (5, 10) for x in range(3, 16, 3)], np.int32)
    v = wl.grf_velocity(shape, corr_cells=3.0, vmin=1800.0, vmax=3000.0, seed=seed).astype(np.float64)
    h = 10.0
    dt = 0.35 * h / 3000.0
    nt = 70
    wav = wl.ricker(nt, dt, 35.0)
    vt = v * (1.0 + 0.04 * np.exp(-sum((np.indices(shape)[i] - shape[i] / 2) ** 2 for i in range(ndim)) / 8.0))
    return dict(ndim=ndim, shape=shape, h=h, dt=dt, v=v, vt=vt, src=src, rec=rec, wav=wav, nt=nt)


@pytest.mark.parametrize("ndim,width", [(2, 0), (2, 5), (3, 3)])
def test_gradient_equals_finite_differences(oracle, ndim, width):
    c = setup(ndim)
    kw = dict(sponge_width=width, src=c["src"], wavelet=c["wav"], receivers=c["rec"], nsteps=c["nt"],
              sponge_vmax=3200.0)
    _, _, dobs = oracle.run(ndim, c["shape"], c["h"], c["dt"], c["vt"], sponge_width=width, src=c["src"],
                            wavelet=c["wav"], receivers=c["rec"], nsteps=c["nt"], sponge_vmax=3200.0)
    J, grad, _ = oracle.misfit_gradient(ndim, c["shape"], c["h"], c["dt"], c["v"], observed=dobs, **kw)
    assert J > 0
    m = 1.0 / c["v"] ** 2
    rng = np.random.default_rng(5)
    for trial in range(2):
        dm = wl.random_field(c["shape"], 2.0, 100 + trial) * m * 0.02
        eps = 1e-3
        Jp, _, _ = oracle.misfit_gradient(ndim, c["shape"], c["h"], c["dt"], 1.0 / np.sqrt(m + eps * dm),
                                          observed=dobs, **kw)
        Jm, _, _ = oracle.misfit_gradient(ndim, c["shape"], c["h"], c["dt"], 1.0 / np.sqrt(m - eps * dm),
                                          observed=dobs, **kw)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * dm))
        assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
    del rng


def test_gradient_sign_mistake_is_caught(oracle):
    """A flipped gradient (a plausible adjoint bug) disagrees with the differences."""
    c = setup(2, seed=1)
    kw = dict(sponge_width=0, src=c["src"], wavelet=c["wav"], receivers=c["rec"], nsteps=c["nt"])
    _, _, dobs = oracle.run(2, c["shape"], c["h"], c["dt"], c["vt"], src=c["src"], wavelet=c["wav"],
                            receivers=c["rec"], nsteps=c["nt"])
    _, grad, _ = oracle.misfit_gradient(2, c["shape"], c["h"], c["dt"], c["v"], observed=dobs, **kw)
    m = 1.0 / c["v"] ** 2
    dm = wl.random_field(c["shape"], 2.0, 7) * m * 0.02
    Jp, _, _ = oracle.misfit_gradient(2, c["shape"], c["h"], c["dt"], 1.0 / np.sqrt(m + 1e-3 * dm),
                                      observed=dobs, **kw)
    Jm, _, _ = oracle.misfit_gradient(2, c["shape"], c["h"], c["dt"], 1.0 / np.sqrt(m - 1e-3 * dm),
                                      observed=dobs, **kw)
    fd = (Jp - Jm) / 2e-3
    assert abs(fd - float(np.sum(-grad * dm))) > 0.5 * abs(fd)
