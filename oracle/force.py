"""Fermion force and the link gradient of D, FP64 (test infrastructure only).

Hybrid Monte Carlo is one of COLA's key algorithms (the paper's overview of
the library); the paper does not write its force.  The definitions here:

Action S(U) = phi^dag (D^dag D)^-1 phi, with X = (D^dag D)^-1 phi, Y = D X.
Varying one link by left multiplication, U_mu(x) -> (1 + i eps T^a) U_mu(x),
T^a = lambda^a / 2 (Gell-Mann), gives

  dS/deps^a = -2 kappa Im Tr[T^a W_mu(x)],   W_mu(x) = Ut_mu(x) (P + Q^dag),
  P_ba = sum_s [(1 - gamma_mu) X(x + mu)]_sb conj(Y(x)_sa)
  Q_ba = sum_s [(1 + gamma_mu) X(x)]_sb     conj(Y(x + mu)_sa)

(from dS = -X^dag d(D^dag D) X = -2 Re Y^dag dD X and dD = -kappa dH).

The raw complex gradient of a real loss through y = D psi, in PyTorch's
convention (grad = 2 dL/d conj(z)), with g = dL/dy in that convention:

  grad_U_mu(x)_ab = -kappa conj(ph) [ sum_s g(x)_sa conj([(1 - gamma_mu) psi(x + mu)]_sb)
                                     + sum_s [(1 + gamma_mu) psi(x)]_sa conj(g(x + mu)_sb) ]

where ph is the boundary phase carried by that link (1 off the boundary).
"""
from __future__ import annotations

import numpy as np

from .wilson import GAMMA, IDENTITY4, phased_links

GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1], GELL_MANN[1][1, 0] = -1j, 1j
GELL_MANN[2][0, 0], GELL_MANN[2][1, 1] = 1, -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2], GELL_MANN[4][2, 0] = -1j, 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2], GELL_MANN[6][2, 1] = -1j, 1j
GELL_MANN[7][0, 0] = GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
GELL_MANN[7][2, 2] = -2 / np.sqrt(3)
T_GEN = GELL_MANN / 2


def _bc_slice_phase(dims, mu, bc):
    """Phase carried by Ut_mu(x) at each site: bc[mu] on x_mu = L_mu - 1."""
    lx, ly, lz, lt = dims
    ph = np.ones((lt, lz, ly, lx), dtype=np.complex128)
    sl = [slice(None)] * 4
    sl[3 - mu] = -1
    ph[tuple(sl)] = complex(bc[mu])
    return ph


def force_coeffs(u, x_field, y_field, kappa, bc):
    """F^a_mu(x) = dS/deps^a as a real array [4, Lt, Lz, Ly, Lx, 8]."""
    ut = phased_links(u, bc)
    out = np.zeros((4,) + x_field.shape[:4] + (8,), dtype=np.float64)
    for mu in range(4):
        ax = 3 - mu
        x_fwd = np.roll(x_field, -1, axis=ax)
        y_fwd = np.roll(y_field, -1, axis=ax)
        h_p = np.einsum("st,...tb->...sb", IDENTITY4 - GAMMA[mu], x_fwd)
        h_q = np.einsum("st,...tb->...sb", IDENTITY4 + GAMMA[mu], x_field)
        p = np.einsum("...sb,...sa->...ba", h_p, y_field.conj())
        q = np.einsum("...sb,...sa->...ba", h_q, y_fwd.conj())
        w = np.einsum("...ab,...bc->...ac", ut[mu], p + np.swapaxes(q.conj(), -1, -2))
        tr = np.einsum("kab,...ba->...k", T_GEN, w)
        out[mu] = -2.0 * kappa * tr.imag
    return out


def dirac_link_grad(u, psi, g, kappa, bc):
    """Raw complex gradient on U of a real loss through y = D psi (PyTorch convention)."""
    dims = (psi.shape[3], psi.shape[2], psi.shape[1], psi.shape[0])
    grad = np.zeros_like(u)
    for mu in range(4):
        ax = 3 - mu
        ph = _bc_slice_phase(dims, mu, bc)
        h_f = np.einsum("st,...tb->...sb", IDENTITY4 - GAMMA[mu], np.roll(psi, -1, axis=ax))
        h_b = np.einsum("st,...tb->...sb", IDENTITY4 + GAMMA[mu], psi)
        g_fwd = np.roll(g, -1, axis=ax)
        a_term = np.einsum("...sa,...sb->...ab", g, h_f.conj())
        b_term = np.einsum("...sa,...sb->...ab", h_b, g_fwd.conj())
        grad[mu] = -kappa * np.conj(ph)[..., None, None] * (a_term + b_term)
    return grad


def link_variation(u, omega, eps):
    """U_mu(x) -> exp(i eps sum_a omega^a T^a) U_mu(x), per link."""
    gen = np.einsum("...k,kab->...ab", omega, T_GEN)
    w, v = np.linalg.eigh(gen)
    rot = np.einsum("...ab,...b,...cb->...ac", v, np.exp(1j * eps * w), v.conj())
    return np.einsum("...ab,...bc->...ac", rot, u)
