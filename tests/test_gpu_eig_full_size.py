"""Eigensolver at the 16^3x32 workload size (GPU; slow test).

kappa 0.125, links exp(0.3 i H) (the 16^3x32 configuration): the twelve
lowest eigenpairs of Mhat^dag Mhat with four guard vectors, in the
configuration bench.py times.  At
this size the oracle checks properties that hold at any size: for sampled
eigenpairs the residual |A v - lambda v| by the oracle's whole-lattice
operator and the oracle's Rayleigh quotient; orthonormality of all vectors;
and the ordering of the eigenvalues.
"""
import numpy as np
import pytest

import oracle
import oracle.eig as oeig
import synth
from helpers import BC_AP, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def test_lowest_twelve_16x16x16x32(cola):
    dims = (16, 16, 16, 32)
    kappa = 0.125
    u = synth.gauge_field(dims, 0.3, synth.seed_for(1, 0))
    v0 = to_dev(synth.gaussian_spinor(dims, synth.seed_for(1, 5), nrhs=16))
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64",), recon={"f64": 18})
    vals, vecs, info = cola.eig_lowest(g, v0, nev=12, op="eo", tol=1e-8)
    vals, vecs = vals.numpy(), vecs.cpu().numpy()
    assert info.status == 0 and info.max_rel_resid <= 1e-8
    assert np.all(np.diff(vals) >= -1e-12 * vals[-1]) and vals[0] > 0
    flat = vecs.reshape(12, -1)
    assert np.max(np.abs(flat.conj() @ flat.T - np.eye(12))) < 1e-12
    e = oracle.even_mask(dims)[..., None, None]
    op = lambda v: oracle.mdagm_eo(u, v * e, kappa, BC_AP) * e  # noqa: E731
    for j in (0, 11):
        av = op(vecs[j])
        rq = np.vdot(vecs[j].reshape(-1), av.reshape(-1)).real
        assert abs(rq - vals[j]) < 1e-10 * vals[j]
        res = oeig.residuals(op, [vals[j]], [vecs[j]])[0]
        assert res <= 1e-8 * vals[j], res / vals[j]
