"""GPU clover force and HMC with the clover term, against the FP64 oracle.

The fermion force of a handle with a clover term (hopping part plus clover
part) element by element against the oracle on lattices with extents of 2
(links met twice by one plaquette), anisotropic extents and both link
reconstructions; the same force at 24^3x48 on sampled links against the
oracle's per-link form; the raw link gradient of the clover operator
against the oracle; whole clover HMC trajectories (links, momenta, dH)
against the oracle's trajectory; and on the device the second-order scaling
of dH that only the correct clover force gives.
"""
import numpy as np
import pytest

import oracle
import oracle.clover as ocl
import oracle.hmc as ohmc
import synth
from helpers import BC_AP, rel_err, to_dev

pytestmark = pytest.mark.gpu

KAPPA = 0.12
BETA = 5.6
CSW = 1.2


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
    return synth.su3_direction(dims, synth.seed_for(99, seed))


@pytest.mark.parametrize("dims,recon", [((2, 2, 2, 2), 18), ((4, 6, 2, 8), 12), ((6, 4, 4, 10), 18)])
def test_clover_force_matches_oracle(cola, dims, recon):
    bc = (1.0, np.exp(0.5j), 1.0, -1.0)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(99, 0))
    x = synth.gaussian_spinor(dims, synth.seed_for(99, 1))
    y = synth.gaussian_spinor(dims, synth.seed_for(99, 2))
    g = cola.Gauge(to_dev(u), dims, KAPPA, bc, precisions=("f64",), recon={"f64": recon})
    g.attach_clover(CSW)
    f = cola.fermion_force(g, to_dev(x), to_dev(y)).cpu().numpy()
    want = oracle.force_coeffs(u, x, y, KAPPA, bc) + ocl.clover_force_coeffs(u, x, y, KAPPA, CSW)
    assert rel_err(f, want) < 1e-13
    # the clover part alone: the same handle without the term gives the hopping part
    g.attach_clover(0.0)
    f0 = cola.fermion_force(g, to_dev(x), to_dev(y)).cpu().numpy()
    assert rel_err(f - f0, ocl.clover_force_coeffs(u, x, y, KAPPA, CSW)) < 1e-12


@pytest.mark.parametrize("dims,recon", [((2, 2, 2, 2), 18), ((4, 6, 2, 8), 12)])
def test_clover_link_grad_matches_oracle(cola, dims, recon):
    """Raw complex link gradient (PyTorch's convention) of Re <gy, D_sw psi>: hopping plus clover parts."""
    bc = (1.0, np.exp(0.5j), 1.0, -1.0)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(99, 13))
    psi = synth.gaussian_spinor(dims, synth.seed_for(99, 14))
    gy = synth.gaussian_spinor(dims, synth.seed_for(99, 15))
    g = cola.Gauge(to_dev(u), dims, KAPPA, bc, precisions=("f64",), recon={"f64": recon})
    g.attach_clover(CSW)
    got = cola.dirac_link_grad(g, to_dev(psi), to_dev(gy)).cpu().numpy()
    want = oracle.dirac_link_grad(u, psi, gy, KAPPA, bc) + ocl.dirac_link_grad_clover(u, psi, gy, KAPPA, CSW)
    assert rel_err(got, want) < 1e-13


def test_clover_autograd_action_gradient_is_the_force(cola):
    """dS/dU from PseudofermionAction.backward with the clover term (the link-gradient kernel)
    projects onto the clover fermion force (the force kernel), F^a = Re<G, i T^a U>; and the
    link gradient of Re <w, X> through SolveNormal against the oracle's solves and gradients."""
    import torch

    dims = (4, 4, 2, 4)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(99, 16))
    phi = synth.gaussian_spinor(dims, synth.seed_for(99, 17))
    links = to_dev(u).requires_grad_(True)
    S = cola.PseudofermionAction.apply(links, to_dev(phi), dims, kappa, BC_AP, 1e-13, "f32", CSW)
    S.backward()
    G = links.grad.cpu().numpy()
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64",))
    g.attach_clover(CSW)
    X, _ = cola.cg_solve(g, to_dev(phi), tol=1e-13, op="full", inner="f64")
    F = cola.fermion_force(g, X, cola.apply_dirac(g, X)).cpu().numpy()
    tu = np.einsum("kab,...bc->...kac", oracle.T_GEN, u)
    proj = np.real(np.einsum("...ab,...kab->...k", G.conj(), 1j * tu))
    assert rel_err(proj, F) < 1e-9
    w = synth.gaussian_spinor(dims, synth.seed_for(99, 18))
    links = to_dev(u).requires_grad_(True)
    Xs = cola.SolveNormal.apply(links, to_dev(phi), dims, kappa, BC_AP, 1e-13, "f64", CSW)
    torch.real(torch.vdot(to_dev(w).reshape(-1), Xs.reshape(-1))).backward()
    x = ocl.solve_normal_full_clover(u, phi, kappa, BC_AP, CSW, tol=1e-13)[0]
    z = ocl.solve_normal_full_clover(u, w, kappa, BC_AP, CSW, tol=1e-13)[0]
    y, wz = ocl.dirac_clover(u, x, kappa, BC_AP, CSW), ocl.dirac_clover(u, z, kappa, BC_AP, CSW)

    def grad(psi, gy):
        return oracle.dirac_link_grad(u, psi, gy, kappa, BC_AP) + ocl.dirac_link_grad_clover(u, psi, gy, kappa, CSW)

    assert rel_err(links.grad.cpu().numpy(), -(grad(z, y) + grad(x, wz))) < 1e-9


def test_clover_force_full_size_sampled(cola):
    """24^3x48 (the HMC benchmark's lattice), 1500 sampled links and the corners."""
    dims = (24, 24, 24, 48)
    u_dev = synth.gauge_field_device(dims, 0.3, synth.seed_for(99, 3))
    x_dev = synth.gaussian_spinor_device(dims, synth.seed_for(99, 4))
    y_dev = synth.gaussian_spinor_device(dims, synth.seed_for(99, 5))
    g = cola.Gauge(u_dev, dims, 0.124, BC_AP, precisions=("f64",), recon={"f64": 18})
    g.attach_clover(1.0)
    g0 = cola.Gauge(u_dev, dims, 0.124, BC_AP, precisions=("f64",), recon={"f64": 18})
    fc = (cola.fermion_force(g, x_dev, y_dev) - cola.fermion_force(g0, x_dev, y_dev)).cpu().numpy().reshape(4, -1, 8)
    u, x, y = u_dev.cpu().numpy(), x_dev.cpu().numpy(), y_dev.cpu().numpy()
    rng = np.random.default_rng(13)
    vol = int(np.prod(dims))
    links = [(0, 0), (3, vol - 1), (1, vol // 2)]
    links += [(int(m), int(i)) for m, i in zip(rng.integers(0, 4, 1500), rng.integers(0, vol, 1500))]
    want = ocl.clover_force_links(u, x, y, 0.124, 1.0, links)
    got = np.array([fc[m, i] for m, i in links])
    assert np.max(np.abs(got - want)) < 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("integrator,md_op", [("leapfrog", "full"), ("omelyan", "eo")])
def test_clover_trajectory_matches_oracle(cola, integrator, md_op):
    dims = (4, 4, 2, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(99, 6))
    p = momenta(dims, 7)
    eta = synth.gaussian_spinor(dims, synth.seed_for(99, 8))
    tau, n = 0.5, 3
    phi = ocl.dirac_clover_dag(u, eta, KAPPA, BC_AP, CSW)
    u1, p1 = ohmc.integrate(u, p, phi, BETA, KAPPA, BC_AP, tau, n, integrator, tol=1e-13, csw=CSW)
    _, dh_want, _ = ohmc.trajectory(u, p, eta, BETA, KAPPA, BC_AP, tau, n, integrator, uniform=0.0, tol=1e-13,
                                    csw=CSW)
    ud, pd = to_dev(u), to_dev(p)
    g = cola.Gauge(ud, dims, KAPPA, BC_AP, precisions=("f64",), recon={"f64": 18})
    g.attach_clover(CSW)
    info = cola.hmc_trajectory(g, ud, pd, to_dev(eta), BETA, tau, n, integrator, uniform=0.0, md_tol=1e-13,
                               action_tol=1e-13, md_op=md_op)
    assert info.accepted
    assert np.max(np.abs(ud.cpu().numpy() - u1)) < 1e-10
    assert np.max(np.abs(pd.cpu().numpy() - p1)) < 1e-9
    assert abs(info.dH - dh_want) < 1e-8, (info.dH, dh_want)
    # the handle's clover term follows the new links
    psi = synth.gaussian_spinor(dims, synth.seed_for(99, 9))
    assert rel_err(cola.apply_dirac(g, to_dev(psi)).cpu().numpy(),
                   ocl.dirac_clover(ud.cpu().numpy(), psi, KAPPA, BC_AP, CSW)) < 1e-13


def test_clover_dh_is_second_order(cola):
    dims = (4, 4, 4, 8)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(99, 10))
    p = momenta(dims, 11)
    eta = to_dev(synth.gaussian_spinor(dims, synth.seed_for(99, 12)))
    dh = {}
    for n in (5, 10):
        ud, pd = to_dev(u), to_dev(p)
        g = cola.Gauge(ud, dims, KAPPA, BC_AP, precisions=("f64",))
        g.attach_clover(CSW)
        dh[n] = cola.hmc_trajectory(g, ud, pd, eta, BETA, 1.0, n, "leapfrog", uniform=0.0, md_tol=1e-12,
                                    action_tol=1e-13).dH
    assert 3.0 < dh[5] / dh[10] < 5.0, dh
