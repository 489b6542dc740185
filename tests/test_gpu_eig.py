"""GPU eigensolver (Kalkreuter-Simma) against the oracle's eigenpairs.

The lowest eigenvalues must equal the oracle's (dense decomposition of the
same operator, whose free-field spectra are pinned in closed form), the
eigenvectors must be orthonormal eigenvectors whose residuals the oracle's
operator confirms, and a non-degenerate eigenvector must span the same line
as the oracle's.  Degenerate levels (the free field) are compared through
eigenvalues and residuals only, since any basis of such a level is correct.
"""
import numpy as np
import pytest

import oracle
import oracle.eig as oeig
import synth
from helpers import BC_AP, to_dev

pytestmark = pytest.mark.gpu

KAPPA = 0.124


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def start(dims, nev, seed):
    return to_dev(synth.gaussian_spinor(dims, synth.seed_for(100, seed), nrhs=nev))


def op_of(u, dims, op, kappa=KAPPA, bc=BC_AP):
    if op == "eo":
        e = oracle.even_mask(dims)[..., None, None]
        return (lambda v: oracle.mdagm_eo(u, v * e, kappa, bc) * e), e
    return (lambda v: oracle.mdagm_full(u, v, kappa, bc)), None


def check_vectors(apply_a, vals, vecs, mask, tol):
    n = len(vals)
    flat = vecs.reshape(n, -1)
    gram = flat.conj() @ flat.T
    assert np.max(np.abs(gram - np.eye(n))) < 1e-12
    res = oeig.residuals(apply_a, vals, vecs)
    assert np.all(res <= tol * np.abs(vals)), res / vals
    if mask is not None:
        assert np.max(np.abs(vecs * (1 - mask))) == 0.0


@pytest.mark.parametrize("op", ["eo", "full"])
def test_random_field_matches_dense(cola, op):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(100, 0))
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    nev = 8
    vals, vecs, info = cola.eig_lowest(g, start(dims, nev, 1), op=op, tol=1e-9)
    vals, vecs = vals.numpy(), vecs.cpu().numpy()
    apply_a, mask = op_of(u, dims, op)
    want, wvecs = oeig.lowest_dense(apply_a, dims[::-1] + (4, 3), nev, mask=mask)
    assert info.status == 0 and info.max_rel_resid <= 1e-9
    assert np.max(np.abs(vals - want) / want) < 1e-10, (vals, want)
    check_vectors(apply_a, vals, vecs, mask, 1e-9)
    # the lowest level is non-degenerate here: same line as the oracle's vector
    assert want[1] - want[0] > 1e-3 * want[0]
    ov = abs(np.vdot(wvecs[0].reshape(-1), vecs[0].reshape(-1)))
    assert abs(ov - 1.0) < 1e-8


def test_free_field_closed_form(cola):
    dims = (4, 4, 4, 4)
    u1 = synth.unit_gauge(dims)
    g = cola.Gauge(to_dev(u1), dims, 0.11, BC_AP, precisions=("f64",))
    nev = 12
    vals, vecs, info = cola.eig_lowest(g, start(dims, nev, 2), op="eo", tol=1e-10, max_cg=60)
    want = oeig.free_field_eo_spectrum(dims, 0.11)[:nev]
    assert info.status == 0
    assert np.max(np.abs(vals.numpy() - want) / want) < 1e-10, (vals, want)
    apply_a, mask = op_of(u1, dims, "eo", kappa=0.11)
    check_vectors(apply_a, vals.numpy(), vecs.cpu().numpy(), mask, 1e-10)


def test_near_degenerate_pair_on_ragged_lattice(cola):
    """The two lowest levels here are 4e-4 apart (relative): resolved by Rayleigh-Ritz (3 wanted + 2 guards)."""
    dims = (6, 4, 2, 8)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(100, 3))
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    vals, vecs, info = cola.eig_lowest(g, start(dims, 5, 4), nev=3, op="eo", tol=1e-10)
    apply_a, mask = op_of(u, dims, "eo")
    want, _ = oeig.lowest_dense(apply_a, dims[::-1] + (4, 3), 3, mask=mask)
    assert (want[1] - want[0]) / want[0] < 1e-3
    assert info.status == 0
    assert np.max(np.abs(vals.numpy() - want) / want) < 1e-10
    check_vectors(apply_a, vals.numpy(), vecs.cpu().numpy(), mask, 1e-10)


def test_single_vector(cola):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(100, 0))
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    vals, vecs, info = cola.eig_lowest(g, start(dims, 1, 9), op="eo", tol=1e-10)
    apply_a, mask = op_of(u, dims, "eo")
    want, _ = oeig.lowest_dense(apply_a, dims[::-1] + (4, 3), 1, mask=mask)
    assert info.status == 0
    assert abs(vals.numpy()[0] - want[0]) < 1e-10 * want[0]
    check_vectors(apply_a, vals.numpy(), vecs.cpu().numpy(), mask, 1e-10)


def test_eig_errors(cola):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(100, 5))
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    with pytest.raises(cola.ColaError, match="nev"):
        cola.eig_lowest(g, start(dims, 65, 6))
    # two identical starting vectors cannot be made independent
    v = start(dims, 2, 7)
    v[1] = v[0]
    with pytest.raises(cola.ColaError, match="vanished"):
        cola.eig_lowest(g, v)
    vals, vecs, info = cola.eig_lowest(g, start(dims, 4, 8), tol=1e-14, max_sweeps=1, max_cg=2,
                                       raise_on_error=False)
    assert info.status == -4 and info.sweeps == 1
