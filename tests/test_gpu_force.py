"""GPU fermion force, link gradient and autograd wrappers against the oracle.

The force from the same X, Y must match the oracle's to 1e-13; end to end it
is checked by central finite differences of the action along a random su(3)
direction, with the action evaluated by the variational estimator
S~ = 2 Re<phi, X~> - |D X~|^2, whose error is quadratic in the solve residual.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP, rel_err, to_dev

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


@pytest.mark.parametrize("dims,recon", [((2, 2, 2, 2), 18), ((4, 6, 4, 8), 12), ((6, 4, 2, 4), 18)])
def test_force_matches_oracle_same_xy(cola, dims, recon):
    kappa = 0.124
    bc = (1.0, np.exp(0.5j), 1.0, -1.0)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(6, 0))
    X = synth.gaussian_spinor(dims, synth.seed_for(6, 1))
    Y = synth.gaussian_spinor(dims, synth.seed_for(6, 2))
    g = cola.Gauge(to_dev(u), dims, kappa, bc, precisions=("f64",), recon={"f64": recon})
    f = cola.fermion_force(g, to_dev(X), to_dev(Y)).cpu().numpy()
    assert rel_err(f, oracle.force_coeffs(u, X, Y, kappa, bc)) < 1e-13


def test_link_grad_matches_oracle(cola):
    dims = (4, 6, 4, 8)
    kappa = 0.13
    bc = (np.exp(0.3j), 1.0, 1.0, -1.0)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(7, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(7, 1))
    gy = synth.gaussian_spinor(dims, synth.seed_for(7, 2))
    g = cola.Gauge(to_dev(u), dims, kappa, bc, precisions=("f64",))
    got = cola.dirac_link_grad(g, to_dev(psi), to_dev(gy)).cpu().numpy()
    assert rel_err(got, oracle.dirac_link_grad(u, psi, gy, kappa, bc)) < 1e-13


def test_dirac_op_gradcheck(cola):
    import torch

    dims = (2, 2, 2, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(8, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(8, 1))
    links = to_dev(u).requires_grad_(True)
    p = to_dev(psi).requires_grad_(True)
    fn = lambda lk, ps: cola.DiracOp.apply(lk, ps, dims, 0.13, (1, 1, 1, -1))  # noqa: E731
    assert torch.autograd.gradcheck(fn, (links, p), eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)


def _variational_action(cola, g, phi, tol=1e-13):
    import torch

    x, _ = cola.cg_solve(g, phi, tol=tol, op="full", inner="f64")
    dx = cola.apply_dirac(g, x)
    return (2 * torch.vdot(phi.reshape(-1), x.reshape(-1)).real - torch.vdot(dx.reshape(-1), dx.reshape(-1)).real).item()


def test_force_end_to_end_finite_differences(cola):
    """phi = D^dag eta at 4^4; F from a GPU solve vs central differences (eps 1e-6)."""
    import torch

    dims = (4, 4, 4, 4)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(4, 0))
    eta = synth.gaussian_spinor(dims, synth.seed_for(4, 1))
    phi = oracle.dirac_dag(u, eta, kappa, BC_AP)
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64",))
    X, info = cola.cg_solve(g, to_dev(phi), tol=1e-13, op="full", inner="f64")
    Y = cola.apply_dirac(g, X)
    F = cola.fermion_force(g, X, Y).cpu().numpy()
    # closed form at the base point: S = |eta|^2
    s0 = _variational_action(cola, g, to_dev(phi))
    assert abs(s0 - np.sum(np.abs(eta) ** 2)) < 1e-10 * s0
    # force of the same X, Y by the oracle
    assert rel_err(F, oracle.force_coeffs(u, X.cpu().numpy(), Y.cpu().numpy(), kappa, BC_AP)) < 1e-13
    omega = synth.su3_direction(dims, synth.seed_for(4, 2))
    eps = 1e-6
    s = []
    for sgn in (+1, -1):
        gp = cola.Gauge(to_dev(oracle.link_variation(u, omega, sgn * eps)), dims, kappa, BC_AP, precisions=("f64",))
        s.append(_variational_action(cola, gp, to_dev(phi)))
    fd = (s[0] - s[1]) / (2 * eps)
    an = float(np.sum(F * omega))
    assert abs(fd - an) < 1e-5 * abs(an)


def test_autograd_action_gradient_is_the_force(cola):
    """dS/dU from PseudofermionAction.backward projects onto F^a = Re<G, i T^a U>."""
    import torch

    dims = (4, 4, 2, 4)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(9, 0))
    phi = synth.gaussian_spinor(dims, synth.seed_for(9, 1))
    links = to_dev(u).requires_grad_(True)
    S = cola.PseudofermionAction.apply(links, to_dev(phi), dims, kappa, BC_AP, 1e-13, "f32")
    S.backward()
    G = links.grad.cpu().numpy()
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64",))
    X, _ = cola.cg_solve(g, to_dev(phi), tol=1e-13, op="full", inner="f64")
    F = cola.fermion_force(g, X, cola.apply_dirac(g, X)).cpu().numpy()
    tu = np.einsum("kab,...bc->...kac", oracle.T_GEN, u)          # T^a U
    proj = np.real(np.einsum("...ab,...kab->...k", G.conj(), 1j * tu))
    assert rel_err(proj, F) < 1e-9
    # the solve's backward: gradient of |X|^2 w.r.t. phi is 2 A^-1 X
    p = to_dev(phi).requires_grad_(True)
    Xs = cola.SolveNormal.apply(to_dev(u), p, dims, kappa, BC_AP, 1e-13, "f64")
    (Xs.abs() ** 2).sum().backward()
    z = oracle.solve_normal_full(u, 2 * Xs.detach().cpu().numpy(), kappa, BC_AP, tol=1e-13)[0]
    assert rel_err(p.grad.cpu().numpy(), z) < 1e-9
