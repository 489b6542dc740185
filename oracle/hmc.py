"""Hybrid Monte Carlo around the fermion force, FP64 (test infrastructure only).

Hybrid Monte Carlo (Duane, Kennedy, Pendleton and Roweth 1987) is one of
COLA's key algorithms (the paper's overview of the library); the paper
writes no formula.  The definitions here, in the link-variation convention of
force.py (U_mu(x) -> (1 + i eps T^a) U_mu(x), T^a = lambda^a / 2):

Wilson gauge action, with the links WITHOUT fermion boundary phases,
  S_G = beta sum_x sum_{mu<nu} (1 - Re tr U_munu(x) / 3),
  U_munu(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag,
and its force
  dS_G/deps^a = (beta / 3) Im Tr[T^a U_mu(x) V_mu(x)],
  V_mu(x) = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                         + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
(U_mu(x) V_mu(x) is the sum of the six plaquettes through the link, each
starting at x along mu).

Momenta: real p^a_mu(x), P = sum_a p^a T^a, kinetic energy K = sum p^2 / 2
(Gaussian p of unit variance sample exp(-K)).  Pseudofermion phi = D^dag eta
with Gaussian eta, S_F = phi^dag (D^dag D)^-1 phi, equal to |eta|^2 at the
links phi was drawn on.  H = K + S_G + S_F.  With a clover term (csw != 0)
D is D_sw of clover.py throughout and the force adds its clover part.  Equations of motion
dU/dt = i P U, dp^a/dt = -dS/deps^a.  Integrators over n steps of size
eps = tau / n:
  leapfrog:  p -= eps/2 F;  n x [U <- exp(i eps P) U;  p -= eps F] with the
             last momentum step eps/2;
  Omelyan 2MN (Omelyan, Mryglod and Folk 2003), per step:
             p -= lam eps F; U <- exp(i eps/2 P) U; p -= (1 - 2 lam) eps F;
             U <- exp(i eps/2 P) U; p -= lam eps F,  lam = 0.1931833275037836.
Metropolis: accept when the uniform number u <= exp(-dH) (probability
min(1, exp(-dH)) for u uniform on [0, 1); u = 0 always accepts).
"""
from __future__ import annotations

import numpy as np

from . import clover
from .force import T_GEN, force_coeffs, link_variation
from .solve import solve_normal_full
from .wilson import dirac, dirac_dag

OMELYAN_LAMBDA = 0.1931833275037836


def _shift(f, mu, step):
    """f(x + step * mu) on [Lt, Lz, Ly, Lx, ...] arrays."""
    return np.roll(f, -step, axis=3 - mu)


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.einsum("...ab,...bc->...ac", out, m)
    return out


def plaquettes(u):
    """Re tr U_munu(x) / 3 for the six planes mu < nu: [6, Lt, Lz, Ly, Lx]."""
    out = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = _mm(u[mu], _shift(u[nu], mu, 1), _dag(_shift(u[mu], nu, 1)), _dag(u[nu]))
            out.append(np.trace(p, axis1=-2, axis2=-1).real / 3.0)
    return np.array(out)


def mean_plaquette(u):
    return float(np.mean(plaquettes(u)))


def gauge_action(u, beta):
    return float(beta * np.sum(1.0 - plaquettes(u)))


def staples(u, mu):
    """V_mu(x), so that U_mu(x) V_mu(x) is the sum of the six plaquettes through the link."""
    v = np.zeros_like(u[mu])
    for nu in range(4):
        if nu == mu:
            continue
        v += _mm(_shift(u[nu], mu, 1), _dag(_shift(u[mu], nu, 1)), _dag(u[nu]))
        back = lambda f: _shift(f, nu, -1)  # noqa: E731
        v += _mm(_dag(back(_shift(u[nu], mu, 1))), _dag(back(u[mu])), back(u[nu]))
    return v


def gauge_force(u, beta):
    """dS_G/deps^a as a real array [4, Lt, Lz, Ly, Lx, 8]."""
    out = np.zeros((4,) + u.shape[1:5] + (8,), dtype=np.float64)
    for mu in range(4):
        w = _mm(u[mu], staples(u, mu))
        tr = np.einsum("kab,...ba->...k", T_GEN, w)
        out[mu] = beta / 3.0 * tr.imag
    return out


def kinetic(p):
    return float(0.5 * np.sum(p * p))


def _solve(u, phi, kappa, bc, tol, csw):
    if csw == 0.0:
        return solve_normal_full(u, phi, kappa, bc, tol=tol)[0]
    return clover.solve_normal_full_clover(u, phi, kappa, bc, csw, tol=tol)[0]


def fermion_action(u, phi, kappa, bc, tol=1e-12, csw=0.0):
    x = _solve(u, phi, kappa, bc, tol, csw)
    return float(np.vdot(phi.reshape(-1), x.reshape(-1)).real)


def total_force(u, phi, beta, kappa, bc, tol=1e-12, csw=0.0):
    f = gauge_force(u, beta)
    if phi is not None:
        x = _solve(u, phi, kappa, bc, tol, csw)
        if csw == 0.0:
            f = f + force_coeffs(u, x, dirac(u, x, kappa, bc), kappa, bc)
        else:
            y = clover.dirac_clover(u, x, kappa, bc, csw)
            f = f + force_coeffs(u, x, y, kappa, bc) + clover.clover_force_coeffs(u, x, y, kappa, csw)
    return f


def update_links(u, p, eps):
    """U_mu(x) <- exp(i eps P_mu(x)) U_mu(x)."""
    return link_variation(u, p, eps)


def integrate(u, p, phi, beta, kappa, bc, tau, nsteps, integrator="leapfrog", tol=1e-12, csw=0.0):
    """Molecular-dynamics trajectory of length tau; returns (U, p)."""
    eps = tau / nsteps
    force = lambda uu: total_force(uu, phi, beta, kappa, bc, tol, csw)  # noqa: E731
    u = np.array(u, copy=True)
    p = np.array(p, copy=True)
    if integrator == "leapfrog":
        p = p - 0.5 * eps * force(u)
        for k in range(nsteps):
            u = update_links(u, p, eps)
            p = p - (eps if k + 1 < nsteps else 0.5 * eps) * force(u)
    elif integrator == "omelyan":
        lam = OMELYAN_LAMBDA
        for _ in range(nsteps):
            p = p - lam * eps * force(u)
            u = update_links(u, p, 0.5 * eps)
            p = p - (1.0 - 2.0 * lam) * eps * force(u)
            u = update_links(u, p, 0.5 * eps)
            p = p - lam * eps * force(u)
    else:
        raise ValueError(integrator)
    return u, p


def hamiltonian(u, p, phi, beta, kappa, bc, tol=1e-12, csw=0.0):
    h = kinetic(p) + gauge_action(u, beta)
    if phi is not None:
        h += fermion_action(u, phi, kappa, bc, tol, csw)
    return h


def trajectory(u, p, eta, beta, kappa, bc, tau, nsteps, integrator="leapfrog", uniform=0.5, tol=1e-12, csw=0.0):
    """One HMC update: phi = D^dag eta, integrate, Metropolis.

    eta is None for the pure gauge theory.  Returns (U after the accept or
    reject, dH, accepted).
    """
    if eta is None:
        phi = None
    elif csw == 0.0:
        phi = dirac_dag(u, eta, kappa, bc)
    else:
        phi = clover.dirac_clover_dag(u, eta, kappa, bc, csw)
    h0 = kinetic(p) + gauge_action(u, beta) + (0.0 if eta is None else float(np.sum(np.abs(eta) ** 2)))
    u1, p1 = integrate(u, p, phi, beta, kappa, bc, tau, nsteps, integrator, tol, csw)
    dh = hamiltonian(u1, p1, phi, beta, kappa, bc, tol, csw) - h0
    accept = bool(uniform <= np.exp(-dh))
    return (u1 if accept else np.array(u, copy=True)), dh, accept


def gauge_force_links(u, beta, links):
    """dS_G/deps^a for a list of (mu, lexicographic site) links, by explicit site arithmetic: [n, 8]."""
    _, lt, lz, ly, lx = u.shape[:5]
    dims = (lx, ly, lz, lt)

    def at(c, mu, step):
        p = [(c[k] + step[k]) % dims[k] for k in range(4)]
        return u[mu, p[3], p[2], p[1], p[0]]

    out = np.zeros((len(links), 8))
    for n, (mu, i) in enumerate(links):
        i = int(i)
        c = [i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)]
        v = np.zeros((3, 3), dtype=np.complex128)
        for nu in range(4):
            if nu == mu:
                continue
            e_mu = [int(k == mu) for k in range(4)]
            e_nu = [int(k == nu) for k in range(4)]
            m_nu = [-x for x in e_nu]
            v += at(c, nu, e_mu) @ at(c, mu, e_nu).conj().T @ at(c, nu, [0, 0, 0, 0]).conj().T
            v += (at(c, nu, [a + b for a, b in zip(e_mu, m_nu)]).conj().T @ at(c, mu, m_nu).conj().T
                  @ at(c, nu, m_nu))
        w = at(c, mu, [0, 0, 0, 0]) @ v
        out[n] = beta / 3.0 * np.einsum("kab,ba->k", T_GEN, w).imag
    return out
