"""Pins of the FP64 oracle's operator against closed forms and invariants (CPU only).

Each test fixes something a plausible slip in the oracle would break:
a sign of gamma_mu (free field, sin term), a wrong link or a missing dagger on
the backward hop (gauge covariance, adjoint identity), a roll in the wrong
direction (free field at non-cubic extents), a lost boundary phase (free field
with twisted phases), a wrong parity mask (Schur identity).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

BC_AP = (1.0, 1.0, 1.0, -1.0)


def rnd_spinor(dims, seed):
    return synth.gaussian_spinor(dims, seed)


def inner(a, b):
    return np.sum(np.conj(a) * b)


def test_gamma_algebra():
    g = oracle.GAMMA
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=0)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4), atol=0)
        assert np.allclose(oracle.GAMMA5 @ g[mu] + g[mu] @ oracle.GAMMA5, 0, atol=0)
    assert np.allclose(oracle.GAMMA5, np.diag([1, 1, -1, -1]), atol=0)


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (2, 4, 6, 4), (6, 2, 2, 8)])
def test_free_field_plane_waves(dims):
    """U = 1: D e^{ipx} u = [(1 - 2k sum cos p) + 2ik sum gamma_mu sin p_mu] e^{ipx} u."""
    kappa = 0.137
    theta = np.array([0.3, -1.1, 2.0, np.pi])            # twisted phases, anti-periodic t
    bc = np.exp(1j * theta)
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    coords = [x, y, z, t]
    u1 = synth.unit_gauge(dims)
    rng = np.random.default_rng(7)
    for n in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (1, 1, 2, 3), (-1, 2, 0, -2)]:
        p = [(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)]
        phase = np.exp(1j * sum(p[m] * coords[m] for m in range(4)))
        u0 = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi = phase[..., None, None] * u0
        got = oracle.dirac(u1, psi, kappa, bc)
        dp = (1 - 2 * kappa * sum(np.cos(pm) for pm in p)) * np.eye(4) + 2j * kappa * sum(
            oracle.GAMMA[m] * np.sin(p[m]) for m in range(4))
        want = phase[..., None, None] * (dp @ u0)
        assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_free_field_spectrum_dense(dims):
    """Spectrum of D^dag D at U = 1: (1 - 2k sum cos p)^2 + 4k^2 sum sin^2 p, 12-fold."""
    kappa = 0.12
    u1 = synth.unit_gauge(dims)
    lx, ly, lz, lt = dims
    shape = (lt, lz, ly, lx, 4, 3)
    m = oracle.dense_matrix(lambda v: oracle.mdagm_full(u1, v, kappa, BC_AP), shape)
    assert np.allclose(m, m.conj().T, atol=1e-14)
    ev = np.sort(np.linalg.eigvalsh(m))
    theta = [0, 0, 0, np.pi]
    want = []
    for n in itertools.product(*[range(d) for d in dims]):
        p = [(2 * np.pi * n[k] + theta[k]) / dims[k] for k in range(4)]
        a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        want += [a * a + 4 * kappa * kappa * sum(np.sin(q) ** 2 for q in p)] * 12
    assert np.allclose(ev, np.sort(want), rtol=0, atol=1e-13)


def test_gamma5_hermiticity_and_adjoint():
    dims = (4, 4, 2, 6)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(90, 0))
    chi = rnd_spinor(dims, 11)
    psi = rnd_spinor(dims, 12)
    kappa = 0.124
    lhs = inner(chi, oracle.dirac(u, psi, kappa, BC_AP))
    g5 = oracle.gamma5_apply
    rhs = inner(g5(oracle.dirac(u, g5(chi), kappa, BC_AP)), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # dagger flag is the true adjoint: <chi, H psi> = <H^dag chi, psi>
    a = inner(chi, oracle.hop(u, psi, BC_AP))
    b = inner(oracle.hop(u, chi, BC_AP, dagger=True), psi)
    assert abs(a - b) < 1e-13 * abs(a)
    # and equals gamma5 H gamma5
    h_dag = oracle.hop(u, psi, BC_AP, dagger=True)
    assert np.max(np.abs(h_dag - g5(oracle.hop(u, g5(psi), BC_AP)))) < 1e-13
    # Schur operator: Mhat^dag is the adjoint of Mhat
    e = oracle.even_mask(dims)[..., None, None]
    ce, pe = chi * e, psi * e
    a = inner(ce, oracle.mhat(u, pe, kappa, BC_AP))
    b = inner(oracle.mhat_dag(u, ce, kappa, BC_AP), pe)
    assert abs(a - b) < 1e-13 * abs(a)


def test_gauge_covariance():
    """D[U^Omega] Omega psi = Omega D[U] psi with U^Omega_mu(x) = Omega(x) U_mu(x) Omega(x+mu)^dag."""
    dims = (4, 2, 4, 6)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(91, 0))
    om = synth.random_su3_field(dims, synth.seed_for(91, 3), eps=1.0)
    psi = rnd_spinor(dims, 13)
    ug = np.empty_like(u)
    for mu in range(4):
        om_fwd = np.roll(om, -1, axis=3 - mu)
        ug[mu] = np.einsum("...ab,...bc,...dc->...ad", om, u[mu], om_fwd.conj())
    psig = np.einsum("...ab,...sb->...sa", om, psi)
    got = oracle.dirac(ug, psig, kappa, BC_AP)
    want = np.einsum("...ab,...sb->...sa", om, oracle.dirac(u, psi, kappa, BC_AP))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def test_hop_sites_matches_whole_lattice():
    dims = (6, 4, 2, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(92, 0))
    psi = rnd_spinor(dims, 14)
    bc = (np.exp(0.4j), 1.0, -1.0, -1.0)
    for dag in (False, True):
        full = oracle.hop(u, psi, bc, dagger=dag).reshape(-1, 4, 3)
        sites = np.arange(0, full.shape[0], 3)
        got = oracle.hop_sites(u, psi, bc, sites, dagger=dag)
        assert np.max(np.abs(got - full[sites])) < 1e-14 * np.max(np.abs(full))


def _dense_wilson_by_index(u, kappa, bc):
    """D assembled entry by entry from the definition with explicit site arithmetic."""
    _, lt, lz, ly, lx = u.shape[:5]
    dims = (lx, ly, lz, lt)
    vol = lx * ly * lz * lt
    n = 12 * vol
    d = np.eye(n, dtype=np.complex128)

    def site(c):
        return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))

    for i in range(vol):
        c = [i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)]
        for mu in range(4):
            f = list(c)
            f[mu] = (c[mu] + 1) % dims[mu]
            b = list(c)
            b[mu] = (c[mu] - 1) % dims[mu]
            j, k = site(f), site(b)
            uf = u[mu, c[3], c[2], c[1], c[0]] * (bc[mu] if c[mu] == dims[mu] - 1 else 1.0)
            ub = u[mu, b[3], b[2], b[1], b[0]] * (bc[mu] if b[mu] == dims[mu] - 1 else 1.0)
            blk_f = np.kron(np.eye(4) - oracle.GAMMA[mu], uf)
            blk_b = np.kron(np.eye(4) + oracle.GAMMA[mu], ub.conj().T)
            d[12 * i:12 * i + 12, 12 * j:12 * j + 12] -= kappa * blk_f
            d[12 * i:12 * i + 12, 12 * k:12 * k + 12] -= kappa * blk_b
    return d


def test_dense_matrix_and_schur_on_2x2x2x2():
    dims = (2, 2, 2, 2)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(93, 0))
    shape = (2, 2, 2, 2, 4, 3)
    d = oracle.dense_matrix(lambda v: oracle.dirac(u, v, kappa, BC_AP), shape)
    d_idx = _dense_wilson_by_index(u, kappa, BC_AP)
    assert np.max(np.abs(d - d_idx)) < 1e-14
    # even/odd blocks and the Schur complement of the odd-odd block
    par = oracle.parity_of_sites(dims).reshape(-1)
    comp = np.repeat(par, 12)
    ev, od = np.where(comp == 0)[0], np.where(comp == 1)[0]
    assert np.allclose(d[np.ix_(od, od)], np.eye(len(od)), atol=0)
    schur = d[np.ix_(ev, ev)] - d[np.ix_(ev, od)] @ np.linalg.solve(d[np.ix_(od, od)], d[np.ix_(od, ev)])
    m = oracle.dense_matrix(lambda v: oracle.mhat(u, v, kappa, BC_AP), shape)
    assert np.max(np.abs(m[np.ix_(ev, ev)] - schur)) < 1e-14
    sd, ld = np.linalg.slogdet(d)
    sm, lm = np.linalg.slogdet(schur)
    assert abs(ld - lm) < 1e-12 and abs(sd - sm) < 1e-12
