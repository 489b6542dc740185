"""Pins of the oracle's clover term (CPU only).

Checked against what the definitions fix without re-typing them:
- sigma_mn algebra (Hermitian, squares to 1, antisymmetric, commutes with gamma5);
- the unit gauge, where the clover term vanishes and D_sw is the Wilson D;
- a constant abelian field built by hand, whose clover matrix has the closed
  form 1 -/+ kappa c_sw (sin B_c - mean) per colour;
- the weak-field limit, where F_mn is eps times the lattice curl of the
  generators averaged over the four leaves (computed here by explicit site
  arithmetic), with an O(eps^2) remainder;
- Q_nm = Q_mn^dag for a random non-abelian field (leaf orientation);
- gauge covariance of A(x) and of D_sw;
- gamma5 hermiticity of D_sw and Mhat;
- the even-odd Schur complement and determinant identity on dense 2^4
  matrices, and a CG solve of the even-odd normal system against dense LU;
- the clover force: central finite differences of -2 Re <Y, D_sw(U) X> (all
  links at once and single (link, generator) pairs) and of the action
  phi^dag (D_sw^dag D_sw)^-1 phi, zero at c_sw = 0, gauge covariance, and the
  per-link form against the whole-lattice form;
- the raw link gradient of Re <w, D_sw psi> against finite differences in the
  real and imaginary directions of single link entries.
"""
import numpy as np
import pytest

import oracle
import oracle.clover as clv
import synth

BC_AP = (1.0, 1.0, 1.0, -1.0)


def rnd_spinor(dims, seed):
    return synth.gaussian_spinor(dims, synth.seed_for(96, seed))


def inner(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def test_sigma_algebra():
    for m in range(4):
        for n in range(4):
            s = clv.SIGMA[m, n]
            assert np.allclose(s, s.conj().T, atol=0)
            assert np.allclose(s, -clv.SIGMA[n, m], atol=0)
            assert np.allclose(oracle.GAMMA5 @ s, s @ oracle.GAMMA5, atol=0)
            if m != n:
                assert np.allclose(s @ s, np.eye(4), atol=1e-15)
            else:
                assert np.all(s == 0)


def test_unit_gauge_reduces_to_wilson():
    dims = (4, 2, 2, 4)
    u = synth.unit_gauge(dims)
    f = clv.field_strength(u)
    assert all(np.max(np.abs(v)) == 0 for v in f.values())
    psi = rnd_spinor(dims, 1)
    got = clv.dirac_clover(u, psi, 0.13, BC_AP, 1.7)
    want = oracle.dirac(u, psi, 0.13, BC_AP)
    assert np.max(np.abs(got - want)) < 1e-14


def _abelian_field(dims, mu, nu, n_c):
    """Constant flux B_c = 2 pi n_c / (L_mu L_nu) through every (mu, nu) plaquette, colour by colour."""
    lx, ly, lz, lt = dims
    L = dims
    u = np.zeros((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    B = 2 * np.pi * np.asarray(n_c, dtype=np.float64) / (L[mu] * L[nu])
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = (x, y, z, t)
                    u[nu, t, z, y, x] = np.diag(np.exp(1j * B * c[mu]))
                    if c[mu] == L[mu] - 1:
                        u[mu, t, z, y, x] = np.diag(np.exp(-1j * B * L[mu] * c[nu]))
    return u, B


@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 3)])
def test_constant_abelian_field_closed_form(plane):
    mu, nu = plane
    dims = (4, 6, 2, 4)
    n_c = (1, 2, -3)
    u, B = _abelian_field(dims, mu, nu, n_c)
    # the links are SU(3): unit determinant
    assert np.max(np.abs(np.linalg.det(u) - 1)) < 1e-13
    f = clv.field_strength(u)
    fc = np.sin(B) - np.mean(np.sin(B))
    for key, v in f.items():
        want = np.diag(fc) if key == plane else np.zeros((3, 3))
        assert np.max(np.abs(v - want)) < 1e-14, key
    kappa, csw = 0.125, 1.9
    a = clv.clover_matrix(u, kappa, csw).reshape(dims[3], dims[2], dims[1], dims[0], 12, 12)
    ev = np.linalg.eigvalsh(a.reshape(-1, 12, 12))
    want = np.sort(np.concatenate([1 + kappa * csw * fc, 1 - kappa * csw * fc] * 2))
    assert np.max(np.abs(ev - want[None, :])) < 1e-14


def _weak_field(dims, eps, seed):
    """u_mu(x) = exp(i eps X_mu(x)) with X = sum_a c_a T^a Hermitian traceless."""
    c = synth.su3_direction(dims, seed)
    x = np.einsum("...a,aij->...ij", c, oracle.T_GEN)
    w, v = np.linalg.eigh(x)
    u = np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), v.conj())
    return u, x


def _curl_average(x, dims, mu, nu):
    """(1/4) sum over the four leaves at each site of X_mu + X_nu(+mu) - X_mu(+nu) - X_nu, by site arithmetic."""
    lx, ly, lz, lt = dims
    out = np.zeros(x.shape[1:], dtype=np.complex128)

    def at(d, c):
        return x[d, c[3] % lt, c[2] % lz, c[1] % ly, c[0] % lx]

    def step(c, d, s):
        c = list(c)
        c[d] += s
        return c

    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for xx in range(lx):
                    c = [xx, y, z, t]
                    acc = np.zeros((3, 3), dtype=np.complex128)
                    # corner of each leaf: x, x - mu, x - mu - nu, x - nu
                    for corner in (c, step(c, mu, -1), step(step(c, mu, -1), nu, -1), step(c, nu, -1)):
                        acc += at(mu, corner) + at(nu, step(corner, mu, 1)) - at(mu, step(corner, nu, 1)) - at(nu, corner)
                    out[t, z, y, xx] = acc / 4
    return out


def test_weak_field_limit_is_lattice_curl():
    dims = (4, 2, 4, 4)   # no plane with both extents 2, where the four leaves cancel to first order
    errs = []
    for eps in (2e-3, 1e-3):
        u, x = _weak_field(dims, eps, synth.seed_for(96, 20))
        f = clv.field_strength(u)
        err = 0.0
        for (mu, nu), v in f.items():
            want = eps * _curl_average(x, dims, mu, nu)
            assert np.max(np.abs(want)) > 0.1 * eps
            err = max(err, np.max(np.abs(v - want)))
        errs.append(err)
    assert errs[1] < 10 * 1e-3 ** 2   # |X| is O(1): the remainder is O(eps^2)
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_leaf_orientation_symmetry():
    dims = (4, 2, 4, 2)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(96, 2))
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            q = clv.clover_leaves(u, mu, nu)
            qt = clv.clover_leaves(u, nu, mu)
            assert np.max(np.abs(qt - np.conj(np.swapaxes(q, -1, -2)))) < 1e-14


def test_clover_hermitian_block_diagonal_and_traceless_field():
    dims = (4, 2, 2, 4)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(96, 3))
    for v in clv.field_strength(u).values():
        assert np.max(np.abs(v - np.conj(np.swapaxes(v, -1, -2)))) < 1e-15
        assert np.max(np.abs(np.trace(v, axis1=-2, axis2=-1))) < 1e-15
    a = clv.clover_matrix(u, 0.12, 1.3)
    m = a.reshape(a.shape[:4] + (12, 12))
    assert np.max(np.abs(m - np.conj(np.swapaxes(m, -1, -2)))) < 1e-15
    assert clv.gamma5_commutator(a) == 0.0
    # spins (0,1) and (2,3) do not mix
    assert np.max(np.abs(a[..., 0:2, :, 2:4, :])) == 0.0
    assert np.max(np.abs(a[..., 2:4, :, 0:2, :])) == 0.0


def test_gauge_covariance():
    dims = (4, 2, 4, 2)
    kappa, csw = 0.124, 1.5
    u = synth.gauge_field(dims, 0.4, synth.seed_for(96, 4))
    om = synth.random_su3_field(dims, synth.seed_for(96, 5), eps=1.0)
    ug = np.empty_like(u)
    for mu in range(4):
        om_fwd = np.roll(om, -1, axis=3 - mu)
        ug[mu] = np.einsum("...ab,...bc,...dc->...ad", om, u[mu], om_fwd.conj())
    a = clv.clover_matrix(u, kappa, csw)
    ag = clv.clover_matrix(ug, kappa, csw)
    want = np.einsum("...ab,...sbtc,...dc->...satd", om, a, om.conj())
    assert np.max(np.abs(ag - want)) < 1e-13
    psi = rnd_spinor(dims, 6)
    psig = np.einsum("...ab,...sb->...sa", om, psi)
    got = clv.dirac_clover(ug, psig, kappa, BC_AP, csw)
    want = np.einsum("...ab,...sb->...sa", om, clv.dirac_clover(u, psi, kappa, BC_AP, csw))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def test_gamma5_hermiticity():
    dims = (4, 4, 2, 2)
    kappa, csw = 0.13, 1.8
    u = synth.gauge_field(dims, 0.4, synth.seed_for(96, 7))
    chi, psi = rnd_spinor(dims, 8), rnd_spinor(dims, 9)
    a = inner(chi, clv.dirac_clover(u, psi, kappa, BC_AP, csw))
    b = inner(clv.dirac_clover_dag(u, chi, kappa, BC_AP, csw), psi)
    c = inner(oracle.gamma5_apply(clv.dirac_clover(u, oracle.gamma5_apply(chi), kappa, BC_AP, csw)), psi)
    assert abs(a - b) < 1e-13 * abs(a) and abs(a - c) < 1e-13 * abs(a)
    e = oracle.even_mask(dims)[..., None, None]
    ce, pe = chi * e, psi * e
    a = inner(ce, clv.mhat_clover(u, pe, kappa, BC_AP, csw))
    b = inner(clv.mhat_clover(u, ce, kappa, BC_AP, csw, dagger=True), pe)
    assert abs(a - b) < 1e-13 * abs(a)


def test_dense_schur_complement_and_determinant():
    dims = (2, 2, 2, 2)
    kappa, csw = 0.124, 1.6
    u = synth.gauge_field(dims, 0.4, synth.seed_for(96, 10))
    shape = (2, 2, 2, 2, 4, 3)
    d = oracle.dense_matrix(lambda v: clv.dirac_clover(u, v, kappa, BC_AP, csw), shape)
    dw = oracle.dense_matrix(lambda v: oracle.dirac(u, v, kappa, BC_AP), shape)
    a = clv.clover_matrix(u, kappa, csw).reshape(-1, 12, 12)
    blk = np.zeros_like(d)
    for i in range(a.shape[0]):
        blk[12 * i:12 * i + 12, 12 * i:12 * i + 12] = a[i] - np.eye(12)
    assert np.max(np.abs(d - (dw + blk))) < 1e-14
    par = np.repeat(oracle.parity_of_sites(dims).reshape(-1), 12)
    ev, od = np.where(par == 0)[0], np.where(par == 1)[0]
    schur = d[np.ix_(ev, ev)] - d[np.ix_(ev, od)] @ np.linalg.solve(d[np.ix_(od, od)], d[np.ix_(od, ev)])
    m = oracle.dense_matrix(lambda v: clv.mhat_clover(u, v, kappa, BC_AP, csw), shape)
    assert np.max(np.abs(m[np.ix_(ev, ev)] - schur)) < 1e-13
    assert np.max(np.abs(m[:, od])) == 0 and np.max(np.abs(m[od, :])) == 0
    sd, ld = np.linalg.slogdet(d)
    so, lo = np.linalg.slogdet(d[np.ix_(od, od)])
    sm, lm = np.linalg.slogdet(schur)
    assert abs(ld - (lo + lm)) < 1e-12 and abs(sd - so * sm) < 1e-12
    # normal operators
    mm = oracle.dense_matrix(lambda v: clv.mdagm_eo_clover(u, v, kappa, BC_AP, csw), shape)
    assert np.max(np.abs(mm[np.ix_(ev, ev)] - schur.conj().T @ schur)) < 1e-13
    mf = oracle.dense_matrix(lambda v: clv.mdagm_full_clover(u, v, kappa, BC_AP, csw), shape)
    assert np.max(np.abs(mf - d.conj().T @ d)) < 1e-13


def test_cg_on_clover_normal_system_matches_dense_solve():
    dims = (2, 2, 2, 4)
    kappa, csw = 0.124, 1.6
    u = synth.gauge_field(dims, 0.3, synth.seed_for(96, 11))
    b = rnd_spinor(dims, 12) * oracle.even_mask(dims)[..., None, None]
    shape = b.shape
    op = lambda v: clv.mdagm_eo_clover(u, v, kappa, BC_AP, csw)  # noqa: E731
    x, it, res = oracle.cg(op, b, tol=1e-12)
    par = np.repeat(oracle.parity_of_sites(dims).reshape(-1), 12)
    ev = np.where(par == 0)[0]
    a = oracle.dense_matrix(op, shape)[np.ix_(ev, ev)]
    x_dense = np.linalg.solve(a, b.reshape(-1)[ev])
    assert it > 0 and res <= 1e-12
    err = np.linalg.norm(x.reshape(-1)[ev] - x_dense) / np.linalg.norm(x_dense)
    assert err < np.linalg.cond(a) * 1e-12


def test_tree_level_clover_cancels_the_wilson_shift_of_landau_zero_modes():
    """Sign of the clover term, fixed by O(a) improvement.

    In a constant abelian field the massless continuum Dirac operator has
    exact zero modes (the lowest Landau level, one per flux quantum and
    two-dimensional spinor).  The Wilson term lifts them by about
    kappa |B| (in D = 1 - kappa H at kappa = 1/8); the tree-level clover term
    (c_sw = 1) exists to cancel that O(a) lift, so with the correct sign the
    modes return to O(B^2), while the opposite sign doubles the lift.
    """
    dims = (6, 6, 1, 1)
    kappa = 0.125
    u, B = _abelian_field(dims, 0, 1, (1, 1, -2))
    shape = (1, 1, 6, 6, 4, 3)
    bc = (1.0, 1.0, 1.0, 1.0)
    low = {}
    for csw in (0.0, 1.0):
        d = oracle.dense_matrix(lambda v: clv.dirac_clover(u, v, kappa, bc, csw), shape)
        ev = np.linalg.eigvals(d)
        low[csw] = ev[np.argsort(np.abs(ev))][:8]
        assert np.max(np.abs(low[csw].imag)) < 1e-10      # real modes
    lift = np.sort(np.abs(low[0.0].real))
    want = kappa * np.abs(np.array([B[0]] * 4 + [B[2]] * 4))
    assert np.max(np.abs(lift - want) / want) < 0.1
    assert np.max(np.abs(low[1.0])) < 0.05 * np.min(lift)


def test_clover_sites_matches_whole_lattice():
    dims = (4, 6, 2, 4)
    kappa, csw = 0.13, 1.4
    u = synth.gauge_field(dims, 0.5, synth.seed_for(96, 13))
    full = clv.clover_matrix(u, kappa, csw).reshape(-1, 4, 3, 4, 3)
    sites = np.arange(0, full.shape[0], 5)
    got = clv.clover_sites(u, kappa, csw, sites)
    assert np.max(np.abs(got - full[sites])) < 1e-14


def test_clover_force_matches_bilinear_finite_difference():
    """dS = -2 Re Y^dag dD_sw X: the hopping plus clover forces are the derivative of
    -2 Re <Y, D_sw(U) X> at fixed X, Y, along a random direction on every link and
    generator by generator on single links (a link hit twice by the 2-extents is
    counted through both of its appearances)."""
    dims = (4, 2, 2, 4)
    kappa, csw = 0.12, 1.3
    u = synth.gauge_field(dims, 0.5, synth.seed_for(98, 0))
    x = synth.gaussian_spinor(dims, synth.seed_for(98, 1))
    y = synth.gaussian_spinor(dims, synth.seed_for(98, 2))
    f = oracle.force_coeffs(u, x, y, kappa, BC_AP) + clv.clover_force_coeffs(u, x, y, kappa, csw)

    def bilinear(omega, e):
        ue = oracle.link_variation(u, omega, e)
        return -2.0 * inner(y, clv.dirac_clover(ue, x, kappa, BC_AP, csw)).real

    rng = np.random.default_rng(3)
    omega = rng.standard_normal(f.shape)
    h = 1e-4
    fd = (bilinear(omega, h) - bilinear(omega, -h)) / (2 * h)
    an = float(np.sum(omega * f))
    assert abs(fd - an) < 1e-7 * abs(an)
    for _ in range(6):
        idx = (int(rng.integers(4)),) + tuple(int(rng.integers(n)) for n in f.shape[1:5]) + (int(rng.integers(8)),)
        e = np.zeros_like(omega)
        e[idx] = 1.0
        fd = (bilinear(e, h) - bilinear(e, -h)) / (2 * h)
        assert abs(fd - f[idx]) < 1e-7 * max(1.0, abs(f[idx])), (idx, fd, f[idx])


def test_clover_force_is_the_derivative_of_the_action():
    """S = phi^dag (D_sw^dag D_sw)^-1 phi, differentiated by central differences of
    converged solves, against the force from X and Y = D_sw X."""
    dims = (2, 2, 2, 4)
    kappa, csw = 0.124, 1.0
    u = synth.gauge_field(dims, 0.4, synth.seed_for(98, 3))
    phi = synth.gaussian_spinor(dims, synth.seed_for(98, 4))

    def action(uu):
        xx, _, res = clv.solve_normal_full_clover(uu, phi, kappa, BC_AP, csw, tol=1e-14)
        assert res < 1e-13
        return inner(phi, xx).real

    x, _, _ = clv.solve_normal_full_clover(u, phi, kappa, BC_AP, csw, tol=1e-14)
    y = clv.dirac_clover(u, x, kappa, BC_AP, csw)
    f = oracle.force_coeffs(u, x, y, kappa, BC_AP) + clv.clover_force_coeffs(u, x, y, kappa, csw)
    omega = np.random.default_rng(4).standard_normal(f.shape)
    h = 1e-4
    fd = (action(oracle.link_variation(u, omega, h)) - action(oracle.link_variation(u, omega, -h))) / (2 * h)
    an = float(np.sum(omega * f))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_clover_force_vanishes_without_the_term_and_is_gauge_covariant():
    dims = (4, 2, 2, 4)
    kappa = 0.12
    u = synth.gauge_field(dims, 0.5, synth.seed_for(98, 5))
    x = synth.gaussian_spinor(dims, synth.seed_for(98, 6))
    y = synth.gaussian_spinor(dims, synth.seed_for(98, 7))
    assert np.all(clv.clover_force_coeffs(u, x, y, kappa, 0.0) == 0.0)
    f = clv.clover_force_coeffs(u, x, y, kappa, 1.5)
    # gauge transformation: U_mu(x) -> W(x) U_mu(x) W(x + mu)^dag, psi(x) -> W(x) psi(x);
    # the force matrix sum_a F^a T^a at each link rotates to W(x) F W(x)^dag
    w = synth.gauge_field(dims, 2.0, synth.seed_for(98, 8))[0]
    ug = np.stack([np.einsum("...ab,...bc,...dc->...ad", w, u[m], np.conj(clv._shift(w, m, 1))) for m in range(4)])
    xg = np.einsum("...ab,...sb->...sa", w, x)
    yg = np.einsum("...ab,...sb->...sa", w, y)
    fg = clv.clover_force_coeffs(ug, xg, yg, kappa, 1.5)
    tg = oracle.force.T_GEN
    m = np.einsum("...k,kab->...ab", f, tg)
    mg = np.einsum("...k,kab->...ab", fg, tg)
    assert np.max(np.abs(mg - np.einsum("...ab,m...bc,...dc->m...ad", w, m, np.conj(w)))) < 1e-12 * np.max(np.abs(m))


def test_clover_force_links_matches_whole_lattice():
    dims = (4, 6, 2, 4)
    u = synth.gauge_field(dims, 0.5, synth.seed_for(98, 9))
    x = synth.gaussian_spinor(dims, synth.seed_for(98, 10))
    y = synth.gaussian_spinor(dims, synth.seed_for(98, 11))
    f = clv.clover_force_coeffs(u, x, y, 0.13, 1.1).reshape(4, -1, 8)
    rng = np.random.default_rng(12)
    vol = int(np.prod(dims))
    links = [(0, 0), (3, vol - 1)] + [(int(m), int(i)) for m, i in zip(rng.integers(0, 4, 40), rng.integers(0, vol, 40))]
    got = clv.clover_force_links(u, x, y, 0.13, 1.1, links)
    want = np.array([f[m, i] for m, i in links])
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def test_clover_link_gradient_against_finite_differences():
    """grad_U of L = Re<w, D_sw psi> in PyTorch's convention (dL/dRe + i dL/dIm of each
    link entry, U a general complex matrix): hopping plus clover parts."""
    dims = (4, 2, 2, 4)
    kappa, csw = 0.13, 1.4
    bc = (np.exp(0.3j), 1.0, 1.0, -1.0)
    u = synth.gauge_field(dims, 0.4, synth.seed_for(98, 12))
    psi = synth.gaussian_spinor(dims, synth.seed_for(98, 13))
    w = synth.gaussian_spinor(dims, synth.seed_for(98, 14))

    def loss(uu):
        return float(np.real(np.sum(np.conj(w) * clv.dirac_clover(uu, psi, kappa, bc, csw))))

    g = oracle.dirac_link_grad(u, psi, w, kappa, bc) + clv.dirac_link_grad_clover(u, psi, w, kappa, csw)
    h = 1e-6
    rng = np.random.default_rng(15)
    idxs = [(0, 3, 1, 1, 3, 0, 2), (3, 0, 0, 0, 0, 1, 1)]
    idxs += [tuple(int(rng.integers(n)) for n in u.shape) for _ in range(6)]
    for idx in idxs:
        for direction, part in ((1.0, "re"), (1j, "im")):
            up = u.copy()
            um = u.copy()
            up[idx] += h * direction
            um[idx] -= h * direction
            d = (loss(up) - loss(um)) / (2 * h)
            want = g[idx].real if part == "re" else g[idx].imag
            assert abs(d - want) < 1e-8 * max(1.0, abs(want)), (idx, part, d, want)
    assert np.all(clv.dirac_link_grad_clover(u, psi, w, kappa, 0.0) == 0)
