"""Pins of the oracle's CG solves and force (CPU only).

Solves are checked against dense LU solves of the same operator (brute force
on 2^4-sized lattices); the even-odd solve against the unpreconditioned one;
the force against central finite differences of an exactly computed action,
against the closed form S = |eta|^2 at phi = D^dag eta, and the raw link
gradient against finite differences in the real and imaginary directions.
"""
import numpy as np
import pytest

import oracle
import synth

BC_AP = (1.0, 1.0, 1.0, -1.0)


def norm(a):
    return np.sqrt(np.sum(np.abs(a) ** 2))


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(94, 0))
    b = synth.gaussian_spinor(dims, synth.seed_for(94, 1))
    return dims, u, b


def test_cg_full_against_dense_solve(small):
    dims, u, b = small
    kappa = 0.124
    shape = b.shape
    a = oracle.dense_matrix(lambda v: oracle.mdagm_full(u, v, kappa, BC_AP), shape)
    x_dense = np.linalg.solve(a, b.reshape(-1)).reshape(shape)
    x, it, res = oracle.solve_normal_full(u, b, kappa, BC_AP, tol=1e-12)
    assert res <= 1e-12 and it > 0
    cond = np.linalg.cond(a)
    assert norm(x - x_dense) / norm(x_dense) < cond * 1e-12


def test_cg_eo_normal_against_dense_schur(small):
    dims, u, b = small
    kappa = 0.124
    shape = b.shape
    par = np.repeat(oracle.parity_of_sites(dims).reshape(-1), 12)
    ev = np.where(par == 0)[0]
    a = oracle.dense_matrix(lambda v: oracle.mdagm_eo(u, v, kappa, BC_AP), shape)[np.ix_(ev, ev)]
    xe_dense = np.linalg.solve(a, b.reshape(-1)[ev])
    x, it, res = oracle.solve_normal_eo(u, b, kappa, BC_AP, tol=1e-12)
    assert res <= 1e-12
    flat = x.reshape(-1)
    assert np.all(flat[par == 1] == 0)
    assert norm(flat[ev] - xe_dense) / norm(xe_dense) < np.linalg.cond(a) * 1e-12


def test_eo_dirac_solve_equals_full_solve(small):
    dims, u, b = small
    kappa = 0.124
    shape = b.shape
    d = oracle.dense_matrix(lambda v: oracle.dirac(u, v, kappa, BC_AP), shape)
    x_dense = np.linalg.solve(d, b.reshape(-1)).reshape(shape)
    x, it, res = oracle.solve_dirac_eo(u, b, kappa, BC_AP, tol=1e-12)
    assert res <= 1e-11
    assert norm(x - x_dense) / norm(x_dense) < np.linalg.cond(d) * 1e-12


def test_cg_restarts_from_true_residual():
    """A loose max_iter leaves a residual above tol; the reported one is the true one."""
    dims = (2, 2, 2, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(95, 0))
    b = synth.gaussian_spinor(dims, synth.seed_for(95, 1))
    x, it, res = oracle.solve_normal_full(u, b, 0.124, BC_AP, tol=1e-10, max_iter=3)
    r = b - oracle.mdagm_full(u, x, 0.124, BC_AP)
    assert it == 3 and abs(res - norm(r) / norm(b)) < 1e-14


def _action_dense(u, phi, kappa, bc):
    shape = phi.shape
    a = oracle.dense_matrix(lambda v: oracle.mdagm_full(u, v, kappa, bc), shape)
    x = np.linalg.solve(a, phi.reshape(-1))
    return float(np.real(np.vdot(phi.reshape(-1), x)))


def test_force_closed_form_and_finite_differences():
    dims = (2, 2, 2, 2)
    kappa = 0.124
    bc = (1.0, np.exp(0.7j), 1.0, -1.0)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(96, 0))
    eta = synth.gaussian_spinor(dims, synth.seed_for(96, 1))
    phi = oracle.dirac_dag(u, eta, kappa, bc)
    s0 = _action_dense(u, phi, kappa, bc)
    assert abs(s0 - norm(eta) ** 2) < 1e-12 * s0
    x, _, res = oracle.solve_normal_full(u, phi, kappa, bc, tol=1e-13)
    y = oracle.dirac(u, x, kappa, bc)
    f = oracle.force_coeffs(u, x, y, kappa, bc)
    # directional derivative along a random su(3) field
    omega = synth.su3_direction(dims, synth.seed_for(96, 2))
    eps = 1e-5
    sp = _action_dense(oracle.link_variation(u, omega, eps), phi, kappa, bc)
    sm = _action_dense(oracle.link_variation(u, omega, -eps), phi, kappa, bc)
    fd = (sp - sm) / (2 * eps)
    an = float(np.sum(f * omega))
    assert abs(fd - an) < 1e-6 * abs(an)
    # single links, single generators (catches a swapped index or generator)
    for mu, site, a in [(0, (0, 0, 0, 0), 0), (3, (1, 1, 0, 1), 7), (1, (1, 0, 1, 0), 4), (2, (0, 1, 1, 1), 2)]:
        om = np.zeros_like(omega)
        om[(mu,) + site + (a,)] = 1.0
        sp = _action_dense(oracle.link_variation(u, om, eps), phi, kappa, bc)
        sm = _action_dense(oracle.link_variation(u, om, -eps), phi, kappa, bc)
        fd = (sp - sm) / (2 * eps)
        assert abs(fd - f[(mu,) + site + (a,)]) < 1e-6 * np.max(np.abs(f))


def test_link_gradient_against_finite_differences():
    """grad_U of L = Re<w, D psi> in PyTorch's convention, dL/dRe + i dL/dIm."""
    dims = (2, 2, 2, 4)
    kappa = 0.13
    bc = (np.exp(0.3j), 1.0, 1.0, -1.0)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(97, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(97, 1))
    w = synth.gaussian_spinor(dims, synth.seed_for(97, 2))

    def loss(uu):
        return float(np.real(np.sum(np.conj(w) * oracle.dirac(uu, psi, kappa, bc))))

    g = oracle.dirac_link_grad(u, psi, w, kappa, bc)
    h = 1e-6
    for idx in [(0, 3, 1, 1, 1, 0, 2), (3, 3, 0, 0, 0, 1, 1), (2, 0, 1, 0, 1, 2, 0), (1, 2, 1, 1, 0, 0, 0)]:
        for direction, part in ((1.0, "re"), (1j, "im")):
            up = u.copy()
            um = u.copy()
            up[idx] += h * direction
            um[idx] -= h * direction
            d = (loss(up) - loss(um)) / (2 * h)
            want = g[idx].real if part == "re" else g[idx].imag
            assert abs(d - want) < 1e-8 * max(1.0, abs(want))


def test_shifted_solves_against_dense(small):
    dims, u, b = small
    kappa = 0.124
    e = oracle.even_mask(dims)[..., None, None]
    be = b * e
    shifts = [0.0, 0.01, 0.3, 2.5]
    op = lambda v: oracle.mdagm_eo(u, v * e, kappa, BC_AP) * e  # noqa: E731
    xs, res = oracle.solve_shifted(op, be, shifts, tol=1e-12)
    par = np.repeat(oracle.parity_of_sites(dims).reshape(-1), 12)
    ev = np.where(par == 0)[0]
    a = oracle.dense_matrix(op, b.shape)[np.ix_(ev, ev)]
    for sigma, x, r in zip(shifts, xs, res):
        m = a + sigma * np.eye(len(ev))
        want = np.linalg.solve(m, be.reshape(-1)[ev])
        assert r <= 1e-12
        assert norm(x.reshape(-1)[ev] - want) / norm(want) < np.linalg.cond(m) * 1e-12
    # larger shifts give smaller solutions (A + sigma is positive definite, growing with sigma)
    norms = [norm(x) for x in xs]
    assert all(n1 > n2 for n1, n2 in zip(norms, norms[1:]))
