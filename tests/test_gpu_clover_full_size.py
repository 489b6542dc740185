"""Clover term at the benchmark's full size, checked against the FP64 oracle.

32^3x64, kappa 0.1245, links exp(0.25 i H), c_sw = 1 (tree level):
* the clover Dirac operator D = A - kappa H in FP64 and FP16 storage on
  sampled sites, with A(x) and (H psi)(x) evaluated by the oracle site by
  site;
* the mixed FP16 even-odd solve of the Dirac system D x = b in the
  graph-driven configuration the benchmark times: the residual b - D x is
  recomputed by the oracle on sampled sites, whose root-mean-square must
  match a 1e-10 true relative residual.
"""
import numpy as np
import pytest

import oracle
import oracle.clover as ocl
import synth
from helpers import BC_AP, to_dev

pytestmark = pytest.mark.gpu

DIMS = (32, 32, 32, 64)
KAPPA = 0.1245
CSW = 1.0


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


@pytest.fixture(scope="module")
def inputs():
    u = synth.gauge_field(DIMS, 0.25, synth.seed_for(2, 0))
    b = synth.gaussian_spinor(DIMS, synth.seed_for(2, 1))
    rng = np.random.default_rng(7)
    vol = int(np.prod(DIMS))
    # both parities, the lattice corners and random interior sites
    sites = np.unique(np.concatenate([[0, 1, vol - 1, vol - 2], rng.integers(0, vol, 1500)]))
    return u, b, sites


def dirac_at_sites(u, psi, sites):
    a = ocl.clover_sites(u, KAPPA, CSW, sites)
    flat = psi.reshape(-1, 4, 3)
    return np.einsum("nsatb,ntb->nsa", a, flat[sites]) - KAPPA * oracle.hop_sites(u, psi, BC_AP, sites)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_clover_dirac_full_size_sampled_sites(cola, inputs, prec):
    u, b, sites = inputs
    g = cola.Gauge(to_dev(u), DIMS, KAPPA, BC_AP, precisions=("f64", prec), recon={"f64": 18, prec: 12})
    g.attach_clover(CSW)
    got = cola.apply_dirac(g, to_dev(b), prec=prec).cpu().numpy().reshape(-1, 4, 3)[sites]
    want = dirac_at_sites(u, b, sites)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < (1e-13 if prec == "f64" else 2e-3), err


def test_clover_mixed_fp16_dirac_solve_full_size(cola, inputs):
    u, b, sites = inputs
    g = cola.Gauge(to_dev(u), DIMS, KAPPA, BC_AP, precisions=("f64", "f16"), recon={"f64": 18, "f16": 12})
    g.attach_clover(CSW)
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op="eo", system="dirac", inner="f16", delta=0.1,
                            use_graph=True)
    assert info[0].status == 0 and info[0].reliable_updates >= 2
    assert info[0].true_rel_resid <= 1e-10
    xr = x.cpu().numpy()
    r = b.reshape(-1, 4, 3)[sites] - dirac_at_sites(u, xr, sites)
    rms_r = np.sqrt(np.mean(np.abs(r) ** 2))
    rms_b = np.sqrt(np.mean(np.abs(b.reshape(-1, 4, 3)[sites]) ** 2))
    # the sampled mean square estimates the whole-lattice one
    assert rms_r / rms_b < 5 * max(info[0].true_rel_resid, 1e-12), (rms_r / rms_b, info[0].true_rel_resid)
