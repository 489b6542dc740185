"""GPU Hybrid Monte Carlo against the FP64 oracle.

The gauge-field kernels element by element: the plaquette, the Wilson gauge
force and the link exponential on several lattices and reconstructions.
Whole trajectories: final links, momenta and dH against the oracle's own
trajectory with the same momenta and pseudofermion source, for leapfrog and
Omelyan, with and without fermions.  Then the properties the oracle is
pinned by, re-checked on the device: reversibility, second-order scaling of
dH, and the Metropolis rejection restoring the links bitwise.
"""
import numpy as np
import pytest

import oracle
import oracle.hmc as ohmc
import synth
from helpers import BC_AP, rel_err, to_dev

pytestmark = pytest.mark.gpu

KAPPA = 0.12
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


def momenta(dims, seed):
    return synth.su3_direction(dims, synth.seed_for(98, seed))


def gauge(cola, u_dev, dims, recon=18, precisions=("f64",)):
    return cola.Gauge(u_dev, dims, KAPPA, BC_AP, precisions=precisions, recon={"f64": recon, "f32": 12})


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 8, 10)])
@pytest.mark.parametrize("recon", [12, 18])
def test_plaquette_and_gauge_force(cola, dims, recon):
    u = synth.gauge_field(dims, 0.5, synth.seed_for(98, 0))
    g = gauge(cola, to_dev(u), dims, recon)
    assert abs(cola.plaquette(g) - ohmc.mean_plaquette(u)) < 1e-14
    f = cola.gauge_force(g, BETA).cpu().numpy()
    assert rel_err(f, ohmc.gauge_force(u, BETA)) < 1e-13


@pytest.mark.parametrize("eps", [0.05, 0.7, 3.0])
def test_link_update(cola, eps):
    dims = (4, 6, 2, 8)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(98, 1))
    p = momenta(dims, 2)
    ud = to_dev(u)
    g = gauge(cola, ud, dims)
    cola.link_update(g, ud, to_dev(p), eps)
    want = ohmc.update_links(u, p, eps)
    assert np.max(np.abs(ud.cpu().numpy() - want)) < 1e-13
    # the handle was re-packed from the new links
    psi = synth.gaussian_spinor(dims, synth.seed_for(98, 3))
    got = cola.apply_dirac(g, to_dev(psi)).cpu().numpy()
    assert rel_err(got, oracle.dirac(want, psi, KAPPA, BC_AP)) < 1e-13


@pytest.mark.parametrize("integrator,fermions,md_op", [("leapfrog", False, "full"), ("omelyan", False, "full"),
                                                        ("leapfrog", True, "full"), ("omelyan", True, "full"),
                                                        ("omelyan", True, "eo")])
def test_trajectory_matches_oracle(cola, integrator, fermions, md_op):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(98, 4))
    p = momenta(dims, 5)
    eta = synth.gaussian_spinor(dims, synth.seed_for(98, 6)) if fermions else None
    tau, n = 0.5, 4
    u1, p1 = ohmc.integrate(u, p, None if eta is None else oracle.dirac_dag(u, eta, KAPPA, BC_AP), BETA, KAPPA,
                            BC_AP, tau, n, integrator, tol=1e-13)
    _, dh_want, _ = ohmc.trajectory(u, p, eta, BETA, KAPPA, BC_AP, tau, n, integrator, uniform=0.0, tol=1e-13)
    ud, pd = to_dev(u), to_dev(p)
    g = gauge(cola, ud, dims)
    info = cola.hmc_trajectory(g, ud, pd, None if eta is None else to_dev(eta), BETA, tau, n, integrator,
                               uniform=0.0, md_tol=1e-13, action_tol=1e-13, md_op=md_op)
    assert info.accepted
    assert info.force_evals == (n + 1 if integrator == "leapfrog" else 2 * n + 1)
    assert np.max(np.abs(ud.cpu().numpy() - u1)) < 1e-10
    assert np.max(np.abs(pd.cpu().numpy() - p1)) < 1e-9
    assert abs(info.dH - dh_want) < 1e-8, (info.dH, dh_want)
    assert abs(info.plaquette - ohmc.mean_plaquette(u1)) < 1e-13
    assert abs(info.H0 - (ohmc.kinetic(p) + ohmc.gauge_action(u, BETA)
                          + (0.0 if eta is None else float(np.sum(np.abs(eta) ** 2))))) < 1e-9 * abs(info.H0)


def test_reversibility_on_device(cola):
    import torch

    dims = (4, 4, 4, 8)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(98, 7))
    p = momenta(dims, 8)
    eta = to_dev(synth.gaussian_spinor(dims, synth.seed_for(98, 9)))
    ud, pd = to_dev(u), to_dev(p)
    g = gauge(cola, ud, dims, precisions=("f64", "f32"))
    i1 = cola.hmc_trajectory(g, ud, pd, eta, BETA, 0.6, 6, "omelyan", uniform=0.0, md_tol=1e-13, md_inner="f32",
                             action_tol=1e-13)
    assert np.max(np.abs(ud.cpu().numpy() - u)) > 1e-2
    pd.neg_()
    # phi is redrawn from eta on the new links; flip it back by using the same phi:
    # D^dag(U1) eta1 = D^dag(U0) eta  =>  solve for eta1 on the device through D^-dag
    phi = cola.apply_dirac(gauge(cola, to_dev(u), dims), eta, dagger=True)
    x, _ = cola.cg_solve(g, phi, tol=1e-14, op="full", system="normal", inner="f64")
    eta1 = cola.apply_dirac(g, x)  # D X with X = (D^dag D)^-1 phi  =>  D^dag eta1 = phi
    i2 = cola.hmc_trajectory(g, ud, pd, eta1, BETA, 0.6, 6, "omelyan", uniform=0.0, md_tol=1e-13, md_inner="f32",
                             action_tol=1e-13)
    assert np.max(np.abs(ud.cpu().numpy() - u)) < 1e-9
    assert np.max(np.abs(-pd.cpu().numpy() - p)) < 1e-8
    assert abs(i1.dH + i2.dH) < 1e-7
    torch.cuda.synchronize()


def test_dh_is_second_order(cola):
    dims = (4, 4, 4, 8)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(98, 10))
    p = momenta(dims, 11)
    eta = to_dev(synth.gaussian_spinor(dims, synth.seed_for(98, 12)))
    dh = {}
    for integrator in ("leapfrog", "omelyan"):
        for n in (5, 10):
            ud, pd = to_dev(u), to_dev(p)
            g = gauge(cola, ud, dims)
            dh[integrator, n] = cola.hmc_trajectory(g, ud, pd, eta, BETA, 1.0, n, integrator, uniform=0.0,
                                                    md_tol=1e-12, action_tol=1e-13).dH
        r = dh[integrator, 5] / dh[integrator, 10]
        assert 3.0 < r < 5.0, (integrator, dh)
    assert abs(dh["omelyan", 5]) < abs(dh["leapfrog", 5])


def test_rejection_restores_links_bitwise(cola):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(98, 13))
    p = momenta(dims, 14)
    ud, pd = to_dev(u), to_dev(p)
    g = gauge(cola, ud, dims)
    # one long leapfrog step: dH is large and positive for this seed
    info = cola.hmc_trajectory(g, ud, pd, None, BETA, 1.5, 1, "leapfrog", uniform=0.999999)
    assert info.dH > 1.0 and not info.accepted
    assert np.array_equal(ud.cpu().numpy(), u)
    assert abs(info.plaquette - ohmc.mean_plaquette(u)) < 1e-14
    psi = synth.gaussian_spinor(dims, synth.seed_for(98, 15))
    assert rel_err(cola.apply_dirac(g, to_dev(psi)).cpu().numpy(), oracle.dirac(u, psi, KAPPA, BC_AP)) < 1e-14


def test_hmc_argument_errors(cola):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(98, 16))
    ud, pd = to_dev(u), to_dev(momenta(dims, 17))
    g = gauge(cola, ud, dims)
    with pytest.raises(cola.ColaError, match="nsteps"):
        cola.hmc_trajectory(g, ud, pd, None, BETA, 1.0, 0)
    with pytest.raises(cola.ColaError, match="uniform"):
        cola.hmc_trajectory(g, ud, pd, None, BETA, 1.0, 2, uniform=1.0)
    g32 = cola.Gauge(ud, dims, KAPPA, BC_AP, precisions=("f32",))
    with pytest.raises(cola.ColaError, match="FP64"):
        cola.plaquette(g32)
