"""HMC at the benchmark's 24^3x48 size (GPU; slow test).

kappa 0.124, beta 5.6, links exp(0.3 i H): the plaquette against the oracle
on the whole lattice; the gauge force and the link exponential on sampled
links against the oracle evaluated link by link; and the trajectory the
benchmark times (tau = 0.5, 5 Omelyan steps, FP32-inner force solves), run
forward and back to its start (reversibility at full size).
"""
import numpy as np
import pytest

import oracle
import oracle.hmc as ohmc
import synth
from helpers import BC_AP, to_dev

pytestmark = pytest.mark.gpu

DIMS = (24, 24, 24, 48)
KAPPA = 0.124
BETA = 5.6


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
    u = synth.gauge_field(DIMS, 0.3, synth.seed_for(5, 0))
    p = synth.su3_direction(DIMS, synth.seed_for(5, 1))
    eta = synth.gaussian_spinor(DIMS, synth.seed_for(5, 2))
    return u, p, eta


def test_gauge_kernels_full_size(cola, inputs):
    u, p, _ = inputs
    ud = to_dev(u)
    g = cola.Gauge(ud, DIMS, KAPPA, BC_AP, precisions=("f64",), recon={"f64": 18})
    assert abs(cola.plaquette(g) - ohmc.mean_plaquette(u)) < 1e-13
    rng = np.random.default_rng(11)
    vol = int(np.prod(DIMS))
    links = [(int(m), int(i)) for m, i in zip(rng.integers(0, 4, 1500), rng.integers(0, vol, 1500))]
    links += [(0, 0), (3, vol - 1)]
    f = cola.gauge_force(g, BETA).cpu().numpy().reshape(4, -1, 8)
    got = np.array([f[m, i] for m, i in links])
    want = ohmc.gauge_force_links(u, BETA, links)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    cola.link_update(g, ud, to_dev(p), 0.1)
    un = ud.cpu().numpy().reshape(4, -1, 3, 3)
    uf, pf = u.reshape(4, -1, 3, 3), p.reshape(4, -1, 8)
    sub_u = np.array([uf[m, i] for m, i in links])
    sub_p = np.array([pf[m, i] for m, i in links])
    want = oracle.link_variation(sub_u, sub_p, 0.1)
    assert np.max(np.abs(np.array([un[m, i] for m, i in links]) - want)) < 1e-13


def test_benchmark_trajectory_is_reversible(cola, inputs):
    u, p, eta = inputs
    ud, pd = to_dev(u), to_dev(p)
    g = cola.Gauge(ud, DIMS, KAPPA, BC_AP, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
    kw = dict(uniform=0.0, md_tol=1e-12, md_inner="f32", action_tol=1e-12)
    i1 = cola.hmc_trajectory(g, ud, pd, to_dev(eta), BETA, 0.5, 5, "omelyan", **kw)
    assert i1.accepted and i1.force_evals == 11
    # backward: -p and the same phi, i.e. eta1 with D^dag(U1) eta1 = D^dag(U0) eta
    g0 = cola.Gauge(to_dev(u), DIMS, KAPPA, BC_AP, precisions=("f64",), recon={"f64": 18})
    phi = cola.apply_dirac(g0, to_dev(eta), dagger=True)
    del g0
    x, info = cola.cg_solve(g, phi, tol=1e-13, op="full", system="normal", inner="f32")
    eta1 = cola.apply_dirac(g, x)
    pd.neg_()
    i2 = cola.hmc_trajectory(g, ud, pd, eta1, BETA, 0.5, 5, "omelyan", **kw)
    assert np.max(np.abs(ud.cpu().numpy() - u)) < 1e-8
    assert np.max(np.abs(-pd.cpu().numpy() - p)) < 1e-6
    assert abs(i1.dH + i2.dH) < 1e-4 * max(1.0, abs(i1.dH))
