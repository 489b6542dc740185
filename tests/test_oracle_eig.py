"""Pins of the oracle's eigenmodes (CPU only).

- the whole spectrum of D^dag D and of the even-odd Mhat^dag Mhat at U = 1
  against the closed forms derived in oracle/eig.py (periodic, anti-periodic
  and twisted boundaries);
- the dense eigenpairs are eigenpairs (residuals) and orthonormal;
- the Lanczos route agrees with the dense one on a random gauge field.
"""
import numpy as np
import pytest

import oracle
import oracle.eig as oeig
import synth

BC_AP = (1.0, 1.0, 1.0, -1.0)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (4, 2, 2, 2)])
def test_free_field_spectra(dims):
    kappa = 0.11
    u1 = synth.unit_gauge(dims)
    shape = dims[::-1] + (4, 3)
    w, _ = oeig.lowest_dense(lambda v: oracle.mdagm_full(u1, v, kappa, BC_AP), shape, 12 * int(np.prod(dims)))
    assert np.allclose(w, oeig.free_field_full_spectrum(dims, kappa), rtol=0, atol=1e-13)
    e = oracle.even_mask(dims)[..., None, None]
    we, _ = oeig.lowest_dense(lambda v: oracle.mdagm_eo(u1, v * e, kappa, BC_AP) * e, shape,
                              6 * int(np.prod(dims)), mask=e)
    assert np.allclose(we, oeig.free_field_eo_spectrum(dims, kappa), rtol=0, atol=1e-13)


def test_free_field_eo_spectrum_twisted():
    dims = (2, 2, 2, 4)
    kappa = 0.13
    theta = (0.7, 0.0, 0.0, np.pi)
    bc = (np.exp(0.7j), 1.0, 1.0, -1.0)
    u1 = synth.unit_gauge(dims)
    shape = dims[::-1] + (4, 3)
    e = oracle.even_mask(dims)[..., None, None]
    we, _ = oeig.lowest_dense(lambda v: oracle.mdagm_eo(u1, v * e, kappa, bc) * e, shape, 6 * int(np.prod(dims)),
                              mask=e)
    assert np.allclose(we, oeig.free_field_eo_spectrum(dims, kappa, theta), rtol=0, atol=1e-13)


def test_dense_eigenpairs_and_lanczos():
    dims = (2, 2, 2, 4)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.4, synth.seed_for(99, 0))
    shape = dims[::-1] + (4, 3)
    e = oracle.even_mask(dims)[..., None, None]
    op = lambda v: oracle.mdagm_eo(u, v * e, kappa, BC_AP) * e  # noqa: E731
    w, vecs = oeig.lowest_dense(op, shape, 8, mask=e)
    assert np.all(np.diff(w) >= 0) and w[0] > 0
    assert np.max(oeig.residuals(op, w, vecs)) < 1e-12
    flat = vecs.reshape(8, -1)
    gram = flat.conj() @ flat.T
    assert np.allclose(gram, np.eye(8), atol=1e-13)
    assert np.max(np.abs(vecs * (1 - e))) == 0
    wl = oeig.lowest_lanczos(op, shape, 8, mask=e)
    assert np.allclose(wl, w, rtol=1e-10, atol=0)
