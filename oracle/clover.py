"""Clover (Sheikholeslami-Wohlert) term, FP64 (test infrastructure only).

The paper's overview of COLA's physics features cites the clover-improved
Wilson actions (FLIC fermions among them) that the library runs but writes no
formula for them.  The definitions here are the standard Sheikholeslami-
Wohlert term in the kappa normalisation of wilson.py (Luscher et al. 1996
sign and clover-leaf field strength, with the traceless projection of F):

  sigma_mn = (i/2) [gamma_m, gamma_n]                      (Hermitian)
  Q_mn(x)  = sum of the four plaquettes in the (m, n) plane that touch x,
             each oriented m -> n (the "clover" of leaves)
  F_mn(x)  = (Q_mn - Q_mn^dag) / (8 i), minus its trace / 3  (Hermitian, traceless)
  A(x)     = 1 - kappa c_sw sum_{m<n} sigma_mn F_mn(x)      (a 12x12 Hermitian matrix per site)
  D_sw     = A - kappa H

sigma_mn commutes with gamma5 = diag(1, 1, -1, -1), so A is block diagonal:
one 6x6 block on spins (0, 1) and one on spins (2, 3).  The plaquettes use
the gauge links without the fermion boundary phase (a closed loop carries
the phase and its conjugate).

Even-odd: D_sw = [[A_ee, -kappa H_eo], [-kappa H_oe, A_oo]], Schur operator on
even sites Mhat = A_ee - kappa^2 H_eo A_oo^-1 H_oe, det D_sw = det A_oo det Mhat,
Mhat^dag = A_ee - kappa^2 H^dag_eo A_oo^-1 H^dag_oe = gamma5 Mhat gamma5.

Clover force.  For S = phi^dag (D_sw^dag D_sw)^-1 phi, X = (D_sw^dag D_sw)^-1 phi
and Y = D_sw X, dS = -2 Re Y^dag dD_sw X (force.py); the clover part is
dA = -kappa c_sw sum sigma_mn dF_mn, so with
  Lam_mn(x)_ba = sum_st (sigma_mn)_st X(x)_tb conj(Y(x)_sa),
  Gam_mn(x)    = L + L^dag,  L = Lam_mn(x) - tr Lam_mn(x) / 3   (Hermitian, traceless),
the traceless projection moves onto Lam, Re Tr[dF Lam] = Im Tr[dQ Gam] / 8, and
  dS_clover = (kappa c_sw / 4) sum_x sum_{m<n} Im Tr[dQ_mn(x) Gam_mn(x)].
Under U_r(y) -> (1 + i eps T^a) U_r(y), a leaf B U A (U = U_r(y)) changes by
i eps B T U A and a leaf B U^dag A by -i eps B U^dag T A, so each factor of
each leaf adds (kappa c_sw / 4) Re Tr[T^a U A Gam B] or
-(kappa c_sw / 4) Re Tr[T^a A Gam B U^dag] to the link it stands for.
clover_force_coeffs writes exactly that sum over leaves and factors.
"""
from __future__ import annotations

import numpy as np

from .force import T_GEN
from .solve import cg
from .wilson import GAMMA, GAMMA5, hop, hop_block, parity_of_sites

SIGMA = np.zeros((4, 4, 4, 4), dtype=np.complex128)
for _m in range(4):
    for _n in range(4):
        SIGMA[_m, _n] = 0.5j * (GAMMA[_m] @ GAMMA[_n] - GAMMA[_n] @ GAMMA[_m])


def _shift(f, mu, step):
    """f(x + step * mu) for a field laid out [Lt, Lz, Ly, Lx, ...]."""
    return np.roll(f, -step, axis=3 - mu)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("...ab,...bc->...ac", out, m)
    return out


def clover_leaves(u, mu, nu):
    """Q_mn(x): the four plaquettes of the (mu, nu) plane touching x, oriented mu -> nu."""
    um, un = u[mu], u[nu]
    p1 = _mm(um, _shift(un, mu, 1), _dag(_shift(um, nu, 1)), _dag(un))
    p2 = _mm(un, _dag(_shift(_shift(um, mu, -1), nu, 1)), _dag(_shift(un, mu, -1)), _shift(um, mu, -1))
    p3 = _mm(_dag(_shift(um, mu, -1)), _dag(_shift(_shift(un, mu, -1), nu, -1)), _shift(_shift(um, mu, -1), nu, -1),
             _shift(un, nu, -1))
    p4 = _mm(_dag(_shift(un, nu, -1)), _shift(um, nu, -1), _shift(_shift(un, mu, 1), nu, -1), _dag(um))
    return p1 + p2 + p3 + p4


def field_strength(u):
    """F[(mu, nu)] for mu < nu: Hermitian traceless [Lt, Lz, Ly, Lx, 3, 3] arrays."""
    out = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            q = clover_leaves(u, mu, nu)
            f = (q - _dag(q)) / 8j
            tr = np.trace(f, axis1=-2, axis2=-1) / 3.0
            out[(mu, nu)] = f - tr[..., None, None] * np.eye(3)
    return out


def clover_matrix(u, kappa, csw):
    """A(x) as [Lt, Lz, Ly, Lx, 4, 3, 4, 3] (spin, colour; spin, colour)."""
    f = field_strength(u)
    lt, lz, ly, lx = u.shape[1:5]
    a = np.zeros((lt, lz, ly, lx, 4, 3, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            a[..., s, c, s, c] = 1.0
    for (mu, nu), fmn in f.items():
        a -= kappa * csw * np.einsum("st,...ab->...satb", SIGMA[mu, nu], fmn)
    return a


def apply_site_matrix(a, psi):
    return np.einsum("...satb,...tb->...sa", a, psi)


def invert_site_matrix(a):
    shp = a.shape
    m = a.reshape(shp[:4] + (12, 12))
    return np.linalg.inv(m).reshape(shp)


def dirac_clover(u, psi, kappa, bc, csw):
    """D_sw psi = A psi - kappa H psi."""
    return apply_site_matrix(clover_matrix(u, kappa, csw), psi) - kappa * hop(u, psi, bc)


def dirac_clover_dag(u, psi, kappa, bc, csw):
    """D_sw^dag psi = A psi - kappa H^dag psi (A is Hermitian)."""
    return apply_site_matrix(clover_matrix(u, kappa, csw), psi) - kappa * hop(u, psi, bc, dagger=True)


def mhat_clover(u, psi_e, kappa, bc, csw, dagger=False):
    """Mhat psi_e = A_ee psi_e - kappa^2 H_eo A_oo^-1 H_oe psi_e (dagger: H -> H^dag)."""
    dims = (psi_e.shape[3], psi_e.shape[2], psi_e.shape[1], psi_e.shape[0])
    par = parity_of_sites(dims)
    pe = psi_e * (par == 0)[..., None, None]
    a = clover_matrix(u, kappa, csw)
    ainv = invert_site_matrix(a)
    t = hop_block(u, pe, bc, 1, dagger)
    t = apply_site_matrix(ainv, t) * (par == 1)[..., None, None]
    return (apply_site_matrix(a, pe) - kappa * kappa * hop_block(u, t, bc, 0, dagger)) * (par == 0)[..., None, None]


def mdagm_eo_clover(u, psi_e, kappa, bc, csw):
    return mhat_clover(u, mhat_clover(u, psi_e, kappa, bc, csw), kappa, bc, csw, dagger=True)


def mdagm_full_clover(u, psi, kappa, bc, csw):
    return dirac_clover_dag(u, dirac_clover(u, psi, kappa, bc, csw), kappa, bc, csw)


def gamma5_commutator(a):
    """Largest entry of |gamma5 A(x) - A(x) gamma5| over the lattice."""
    g5a = np.einsum("su,...uatb->...satb", GAMMA5, a)
    ag5 = np.einsum("...satb,tu->...saub", a, GAMMA5)
    return float(np.max(np.abs(g5a - ag5)))


def clover_sites(u, kappa, csw, sites):
    """A(x) at the listed lexicographic sites i = x + Lx (y + Ly (z + Lz t)), [n, 4, 3, 4, 3].

    Per-site restatement of clover_matrix with explicit coordinate arithmetic
    (no whole-lattice shifts), for sampled checks on lattices too large for
    the whole-lattice form.
    """
    _, lt, lz, ly, lx = u.shape[:5]
    dims = (lx, ly, lz, lt)

    def link(c, mu, step):
        p = [(c[k] + step[k]) % dims[k] for k in range(4)]
        return u[mu, p[3], p[2], p[1], p[0]]

    out = np.zeros((len(sites), 4, 3, 4, 3), dtype=np.complex128)
    for n, i in enumerate(sites):
        i = int(i)
        c = [i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)]
        a = np.eye(12, dtype=np.complex128)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                def at(dm, dn, d):
                    step = [0, 0, 0, 0]
                    step[mu] += dm
                    step[nu] += dn
                    return link(c, mu if d == 0 else nu, step)
                dg = lambda m: m.conj().T  # noqa: E731
                q = (at(0, 0, 0) @ at(1, 0, 1) @ dg(at(0, 1, 0)) @ dg(at(0, 0, 1))
                     + at(0, 0, 1) @ dg(at(-1, 1, 0)) @ dg(at(-1, 0, 1)) @ at(-1, 0, 0)
                     + dg(at(-1, 0, 0)) @ dg(at(-1, -1, 1)) @ at(-1, -1, 0) @ at(0, -1, 1)
                     + dg(at(0, -1, 1)) @ at(0, -1, 0) @ at(1, -1, 1) @ dg(at(0, 0, 0)))
                f = (q - dg(q)) / 8j
                f = f - np.trace(f) / 3.0 * np.eye(3)
                a -= kappa * csw * np.kron(SIGMA[mu, nu], f)
        out[n] = a.reshape(4, 3, 4, 3)
    return out


# The four leaves of Q_mn(x) as paths of factors (d, om, on, adj): the link of
# direction mu (d = 0) or nu (d = 1) at x + om mu + on nu, adjoint or not, in
# the order of the products in clover_leaves.
LEAF_PATHS = (
    ((0, 0, 0, False), (1, 1, 0, False), (0, 0, 1, True), (1, 0, 0, True)),
    ((1, 0, 0, False), (0, -1, 1, True), (1, -1, 0, True), (0, -1, 0, False)),
    ((0, -1, 0, True), (1, -1, -1, True), (0, -1, -1, False), (1, 0, -1, False)),
    ((1, 0, -1, True), (0, 0, -1, False), (1, 1, -1, False), (0, 0, 0, True)),
)


def _shift2(f, mu, om, nu, on):
    """f(x + om mu + on nu)."""
    return _shift(_shift(f, mu, om), nu, on)


def clover_force_gamma(x_field, y_field):
    """Gam_mn(x) for m < n: {(m, n): [Lt, Lz, Ly, Lx, 3, 3]} (Hermitian, traceless)."""
    out = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            lam = np.einsum("st,...tb,...sa->...ba", SIGMA[mu, nu], x_field, y_field.conj())
            lam = lam - (np.trace(lam, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
            out[(mu, nu)] = lam + _dag(lam)
    return out


def clover_force_coeffs(u, x_field, y_field, kappa, csw):
    """Clover part of dS/deps^a for S = phi^dag (D_sw^dag D_sw)^-1 phi: [4, Lt, Lz, Ly, Lx, 8].

    X = (D_sw^dag D_sw)^-1 phi and Y = D_sw X; the hopping part is
    force.force_coeffs.  Links without the fermion boundary phase.
    """
    out = np.zeros((4,) + x_field.shape[:4] + (8,), dtype=np.float64)
    gam = clover_force_gamma(x_field, y_field)
    for (mu, nu), g in gam.items():
        for path in LEAF_PATHS:
            mats = []
            for d, om, on, adj in path:
                m = _shift2(u[mu if d == 0 else nu], mu, om, nu, on)
                mats.append(_dag(m) if adj else m)
            for k, (d, om, on, adj) in enumerate(path):
                after = _mm(*mats[k + 1:]) if k < 3 else None
                before = _mm(*mats[:k]) if k > 0 else None
                chain = [m for m in (after, g, before) if m is not None]
                if adj:
                    w = _mm(*chain, mats[k])
                    sign = -1.0
                else:
                    w = _mm(mats[k], *chain)
                    sign = 1.0
                tr = np.einsum("kab,...ba->...k", T_GEN, w).real
                # the factor is the link at x + om mu + on nu: move the term there
                out[mu if d == 0 else nu] += sign * 0.25 * kappa * csw * _shift2(tr, mu, -om, nu, -on)
    return out


def solve_normal_full_clover(u, b, kappa, bc, csw, tol=1e-10, x0=None, max_iter=100000):
    """D_sw^dag D_sw x = b on the whole lattice by CG (A(x) built once, then
    D_sw v = A v - kappa H v and D_sw^dag t = A t - kappa H^dag t)."""
    a = clover_matrix(u, kappa, csw)

    def op(v):
        t = apply_site_matrix(a, v) - kappa * hop(u, v, bc)
        return apply_site_matrix(a, t) - kappa * hop(u, t, bc, dagger=True)

    return cg(op, b, x0, tol, max_iter)


def clover_force_links(u, x_field, y_field, kappa, csw, links):
    """clover_force_coeffs at a list of (mu, lexicographic site) links: [n, 8].

    Per-link restatement with explicit coordinate arithmetic, for sampled
    checks on lattices too large for the whole-lattice form: every factor of
    every leaf of every plane through the link that stands for it.
    """
    _, lt, lz, ly, lx = u.shape[:5]
    dims = (lx, ly, lz, lt)

    def coords(i):
        return [i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)]

    def at(field, c):
        return field[c[3], c[2], c[1], c[0]]

    def moved(c, steps):
        return [(c[k] + steps[k]) % dims[k] for k in range(4)]

    out = np.zeros((len(links), 8))
    for n, (rho, i) in enumerate(links):
        y = coords(int(i))
        for mu in range(4):
            for nu in range(mu + 1, 4):
                if rho not in (mu, nu):
                    continue
                for path in LEAF_PATHS:
                    for k, (d, om, on, adj) in enumerate(path):
                        if (mu if d == 0 else nu) != rho:
                            continue
                        step = [0, 0, 0, 0]
                        step[mu] -= om
                        step[nu] -= on
                        xs = moved(y, step)  # the leaf's base site: the factor sits at x + om mu + on nu = y
                        mats = []
                        for dd, omm, onn, aa in path:
                            s2 = [0, 0, 0, 0]
                            s2[mu] += omm
                            s2[nu] += onn
                            m = at(u[mu if dd == 0 else nu], moved(xs, s2))
                            mats.append(m.conj().T if aa else m)
                        xv, yv = at(x_field, xs), at(y_field, xs)
                        lam = np.einsum("st,tb,sa->ba", SIGMA[mu, nu], xv, yv.conj())
                        lam = lam - np.trace(lam) / 3.0 * np.eye(3)
                        g = lam + lam.conj().T
                        after = np.eye(3, dtype=np.complex128)
                        for m in mats[k + 1:]:
                            after = after @ m
                        before = np.eye(3, dtype=np.complex128)
                        for m in mats[:k]:
                            before = before @ m
                        if adj:
                            w = after @ g @ before @ mats[k]
                            sign = -1.0
                        else:
                            w = mats[k] @ after @ g @ before
                            sign = 1.0
                        out[n] += sign * 0.25 * kappa * csw * np.einsum("kab,ba->k", T_GEN, w).real
    return out


def dirac_link_grad_clover(u, psi, g, kappa, csw):
    """Clover part of the raw complex link gradient of a real loss through
    y = D_sw psi, in PyTorch's convention (grad = 2 dL/d conj(U), U a general
    complex matrix), given g = dL/dy in that convention: [4, Lt, Lz, Ly, Lx, 3, 3].

    dL = Re g^dag dA psi = -(kappa c_sw / 8) sum_x sum_{m<n} Im Tr[dQ_mn Gam_mn]
    with Gam from (X, Y) = (psi, g) as in clover_force_gamma.  A factor U of a
    leaf B U C gives Im Tr[dU M], M = C Gam B, whose gradient is -i c M^dag;
    a factor U^dag gives Im Tr[dU^dag M], gradient +i c M; c = kappa c_sw / 8.
    The hopping part is force.dirac_link_grad.
    """
    out = np.zeros(u.shape, dtype=np.complex128)
    gam = clover_force_gamma(psi, g)
    c = kappa * csw / 8.0
    for (mu, nu), gm in gam.items():
        for path in LEAF_PATHS:
            mats = []
            for d, om, on, adj in path:
                m = _shift2(u[mu if d == 0 else nu], mu, om, nu, on)
                mats.append(_dag(m) if adj else m)
            for k, (d, om, on, adj) in enumerate(path):
                after = _mm(*mats[k + 1:]) if k < 3 else None
                before = _mm(*mats[:k]) if k > 0 else None
                m = _mm(*[x for x in (after, gm, before) if x is not None])
                term = 1j * c * m if adj else -1j * c * _dag(m)
                out[mu if d == 0 else nu] += _shift2(term, mu, -om, nu, -on)
    return out
