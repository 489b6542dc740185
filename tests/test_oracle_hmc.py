"""Pins of the oracle's HMC (CPU only).

- the gauge action: zero at U = 1, gauge invariant, and a hand-built constant
  abelian field in closed form (beta V (1 - mean cos B_c) in the flux plane);
- the gauge force against central finite differences of the action, along a
  random su(3) direction and along single (link, generator) pairs;
- free motion (beta = 0, no fermions) is U(tau) = exp(i tau P) U exactly;
- the link exponential itself against scipy's Pade expm at large steps,
  unitarity, unit determinant and the one-parameter group law;
- reversibility: integrating back with -p returns the start (leapfrog and
  Omelyan, with and without fermions);
- energy conservation: dH falls by about 4 when the step halves (both
  integrators are second order), and Omelyan's dH is below leapfrog's;
- the start of a trajectory: S_F = |eta|^2 at phi = D^dag eta;
- the same reversibility, second order and start with the clover term (a
  missing or wrong clover force leaves dH first order in the step).
"""
import numpy as np
import pytest

import oracle
import oracle.clover as clover
import oracle.hmc as hmc
import synth
from test_oracle_clover import _abelian_field

BC_AP = (1.0, 1.0, 1.0, -1.0)


def momenta(dims, seed):
    return synth.su3_direction(dims, synth.seed_for(97, seed))


def test_gauge_action_zero_at_unit_and_gauge_invariant():
    dims = (4, 2, 4, 2)
    assert hmc.gauge_action(synth.unit_gauge(dims), 5.5) == 0.0
    u = synth.gauge_field(dims, 0.5, synth.seed_for(97, 0))
    om = synth.random_su3_field(dims, synth.seed_for(97, 1), eps=1.0)
    ug = np.empty_like(u)
    for mu in range(4):
        ug[mu] = np.einsum("...ab,...bc,...dc->...ad", om, u[mu], np.roll(om, -1, axis=3 - mu).conj())
    assert abs(hmc.gauge_action(ug, 5.5) - hmc.gauge_action(u, 5.5)) < 1e-12 * hmc.gauge_action(u, 5.5)


@pytest.mark.parametrize("plane", [(0, 1), (2, 3)])
def test_gauge_action_constant_abelian_field(plane):
    dims = (4, 6, 2, 4)
    u, B = _abelian_field(dims, plane[0], plane[1], (1, 2, -3))
    vol = int(np.prod(dims))
    want = 5.5 * vol * (1.0 - np.mean(np.cos(B)))
    assert abs(hmc.gauge_action(u, 5.5) - want) < 1e-12 * want


def test_gauge_force_finite_differences():
    dims = (2, 4, 2, 4)
    beta = 5.7
    u = synth.gauge_field(dims, 0.4, synth.seed_for(97, 2))
    f = hmc.gauge_force(u, beta)
    omega = momenta(dims, 3)
    h = 1e-5
    fd = (hmc.gauge_action(oracle.link_variation(u, omega, h), beta)
          - hmc.gauge_action(oracle.link_variation(u, omega, -h), beta)) / (2 * h)
    assert abs(fd - np.sum(f * omega)) < 1e-7 * np.sum(np.abs(f * omega))
    for (mu, site, a) in [(0, (0, 0, 0, 0), 0), (3, (3, 1, 2, 1), 7), (1, (1, 0, 3, 1), 4)]:
        e = np.zeros_like(omega)
        e[(mu,) + site + (a,)] = 1.0
        fd = (hmc.gauge_action(oracle.link_variation(u, e, h), beta)
              - hmc.gauge_action(oracle.link_variation(u, e, -h), beta)) / (2 * h)
        assert abs(fd - f[(mu,) + site + (a,)]) < 1e-8


def test_free_motion_is_exact():
    dims = (2, 2, 2, 4)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(97, 4))
    p = momenta(dims, 5)
    u1, p1 = hmc.integrate(u, p, None, 0.0, 0.0, BC_AP, 0.7, 5, "leapfrog")
    assert np.array_equal(p1, p)
    assert np.max(np.abs(u1 - oracle.link_variation(u, p, 0.7))) < 1e-13


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
@pytest.mark.parametrize("fermions", [False, True])
def test_reversibility(integrator, fermions):
    dims = (2, 2, 2, 4)
    kappa, beta = 0.12, 5.6
    u = synth.gauge_field(dims, 0.3, synth.seed_for(97, 6))
    p = momenta(dims, 7)
    phi = synth.gaussian_spinor(dims, synth.seed_for(97, 8)) if fermions else None
    u1, p1 = hmc.integrate(u, p, phi, beta, kappa, BC_AP, 0.4, 4, integrator, tol=1e-13)
    u0, p0 = hmc.integrate(u1, -p1, phi, beta, kappa, BC_AP, 0.4, 4, integrator, tol=1e-13)
    assert np.max(np.abs(u0 - u)) < 1e-10
    assert np.max(np.abs(-p0 - p)) < 1e-9
    assert np.max(np.abs(u1 - u)) > 1e-2


def test_energy_conservation_is_second_order():
    dims = (2, 2, 2, 4)
    kappa, beta = 0.12, 5.6
    u = synth.gauge_field(dims, 0.3, synth.seed_for(97, 9))
    p = momenta(dims, 10)
    eta = synth.gaussian_spinor(dims, synth.seed_for(97, 11))
    dh = {}
    for integrator in ("leapfrog", "omelyan"):
        for n in (4, 8):
            _, dh[integrator, n], _ = hmc.trajectory(u, p, eta, beta, kappa, BC_AP, 0.5, n, integrator,
                                                     tol=1e-13)
        r = dh[integrator, 4] / dh[integrator, 8]
        assert 3.0 < r < 5.0, (integrator, r, dh)
    assert abs(dh["omelyan", 4]) < abs(dh["leapfrog", 4])


def test_trajectory_start_and_metropolis():
    dims = (2, 2, 2, 2)
    kappa, beta = 0.12, 5.6
    u = synth.gauge_field(dims, 0.3, synth.seed_for(97, 12))
    eta = synth.gaussian_spinor(dims, synth.seed_for(97, 13))
    phi = oracle.dirac_dag(u, eta, kappa, BC_AP)
    assert abs(hmc.fermion_action(u, phi, kappa, BC_AP) - np.sum(np.abs(eta) ** 2)) < 1e-10 * np.sum(np.abs(eta) ** 2)
    p = momenta(dims, 14)
    u_acc, dh, acc = hmc.trajectory(u, p, eta, beta, kappa, BC_AP, 0.3, 3, uniform=0.0)
    assert acc and not np.array_equal(u_acc, u)
    u_rej, dh2, acc2 = hmc.trajectory(u, p, eta, beta, kappa, BC_AP, 0.3, 3, uniform=1.0 - 1e-300)
    assert dh2 == dh
    assert acc2 == (dh <= 0) and (acc2 or np.array_equal(u_rej, u))


def test_gauge_force_links_matches_whole_lattice():
    dims = (4, 6, 2, 4)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(97, 15))
    full = hmc.gauge_force(u, 5.7).reshape(4, -1, 8)
    links = [(mu, i) for mu in range(4) for i in range(0, full.shape[1], 7)]
    got = hmc.gauge_force_links(u, 5.7, links)
    want = np.array([full[mu, i] for mu, i in links])
    assert np.max(np.abs(got - want)) < 1e-13


def test_clover_trajectory_reversible_and_second_order():
    """HMC with the clover term: the integrator is reversible, dH shrinks four-fold
    when the step halves (the forces are the derivatives of H), and phi = D_sw^dag eta
    gives S_F = |eta|^2 at the start."""
    dims = (2, 2, 2, 4)
    kappa, beta, csw = 0.12, 5.6, 1.2
    u = synth.gauge_field(dims, 0.3, synth.seed_for(97, 20))
    p = momenta(dims, 21)
    eta = synth.gaussian_spinor(dims, synth.seed_for(97, 22))
    phi = clover.dirac_clover_dag(u, eta, kappa, BC_AP, csw)
    e2 = np.sum(np.abs(eta) ** 2)
    assert abs(hmc.fermion_action(u, phi, kappa, BC_AP, csw=csw) - e2) < 1e-10 * e2
    u1, p1 = hmc.integrate(u, p, phi, beta, kappa, BC_AP, 0.4, 3, "omelyan", tol=1e-13, csw=csw)
    u0, p0 = hmc.integrate(u1, -p1, phi, beta, kappa, BC_AP, 0.4, 3, "omelyan", tol=1e-13, csw=csw)
    assert np.max(np.abs(u0 - u)) < 1e-10 and np.max(np.abs(-p0 - p)) < 1e-9
    dh = {n: hmc.trajectory(u, p, eta, beta, kappa, BC_AP, 0.5, n, "leapfrog", tol=1e-13, csw=csw)[1] for n in (4, 8)}
    assert 3.0 < dh[4] / dh[8] < 5.0, dh


def test_link_variation_is_the_group_exponential():
    """exp(i eps P) U with P = sum_a p^a T^a, at large eps: equal to scipy's Pade
    expm (a different algorithm from the oracle's eigendecomposition), unitary with
    unit determinant, and a one-parameter group (exp(i a P) exp(i b P) = exp(i (a+b) P))."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    dims = (2, 2, 2, 2)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(97, 30))
    p = momenta(dims, 31)
    for eps in (0.05, 0.7, 3.0):
        got = oracle.link_variation(u, p, eps)
        for idx in [(0, 0, 0, 0, 0), (3, 1, 1, 0, 1), (1, 0, 1, 1, 0), (2, 1, 0, 1, 1)]:
            gen = np.einsum("k,kab->ab", p[idx], oracle.T_GEN)
            want = scipy_linalg.expm(1j * eps * gen) @ u[idx]
            assert np.max(np.abs(got[idx] - want)) < 1e-13, (eps, idx)
        eye = np.einsum("...ab,...cb->...ac", got, got.conj())
        assert np.max(np.abs(eye - np.eye(3))) < 1e-13
        assert np.max(np.abs(np.linalg.det(got) - 1.0)) < 1e-13
    two = oracle.link_variation(oracle.link_variation(u, p, 0.4), p, 0.9)
    assert np.max(np.abs(two - oracle.link_variation(u, p, 1.3))) < 1e-13
