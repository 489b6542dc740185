"""Wilson-Dirac operator, FP64, canonical layout (test infrastructure only).

Definitions (the paper names the fermion matrix but does not write it; this
is the kappa-normalised Wilson form used by the mixed-precision work it
cites, Clark et al. 2010):

  (H psi)(x) = sum_mu [ (1 - gamma_mu) Ut_mu(x) psi(x + mu)
                      + (1 + gamma_mu) Ut_mu(x - mu)^dag psi(x - mu) ]
  D = 1 - kappa H

Ut_mu(x) = U_mu(x) * phase_mu when x_mu = L_mu - 1, else U_mu(x): the
boundary phase rides on the link that crosses the boundary, so the backward
hop across it carries the conjugate phase.  Anti-periodic time is
phase (1, 1, 1, -1).

H^dag swaps the two projectors:  H^dag = gamma5 H gamma5.

Gamma matrices: Euclidean, Hermitian, chiral (DeGrand-Rossi) basis,
gamma5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1).

Arrays: spinor [Lt, Lz, Ly, Lx, 4, 3], gauge [4, Lt, Lz, Ly, Lx, 3, 3];
direction mu (x, y, z, t) lives on spinor axis 3 - mu.
"""
from __future__ import annotations

import numpy as np

I_ = 1j
GAMMA = np.array(
    [
        [[0, 0, 0, I_], [0, 0, I_, 0], [0, -I_, 0, 0], [-I_, 0, 0, 0]],  # gamma_x
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],      # gamma_y
        [[0, 0, I_, 0], [0, 0, 0, -I_], [-I_, 0, 0, 0], [0, I_, 0, 0]],  # gamma_z
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],        # gamma_t
    ],
    dtype=np.complex128,
)
IDENTITY4 = np.eye(4, dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def _dims_of(psi):
    lt, lz, ly, lx = psi.shape[:4]
    return (lx, ly, lz, lt)


def _axis(mu):
    return 3 - mu


def parity_of_sites(dims):
    """(x + y + z + t) mod 2 as an [Lt, Lz, Ly, Lx] int array."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2


def even_mask(dims):
    return parity_of_sites(dims) == 0


def phased_links(u, bc):
    """Ut_mu(x): U_mu(x) times bc[mu] on the slice x_mu = L_mu - 1."""
    ut = np.array(u, dtype=np.complex128, copy=True)
    for mu in range(4):
        ax = _axis(mu)
        sl = [slice(None)] * 4
        sl[ax] = -1
        ut[(mu,) + tuple(sl)] *= complex(bc[mu])
    return ut


def hop(u, psi, bc, dagger=False):
    """H psi (dagger=False) or H^dag psi (dagger=True) on the whole lattice."""
    ut = phased_links(u, bc)
    sign = -1.0 if dagger else 1.0
    out = np.zeros_like(psi)
    for mu in range(4):
        ax = _axis(mu)
        p_fwd = IDENTITY4 - sign * GAMMA[mu]   # (1 - gamma_mu), or (1 + gamma_mu) for H^dag
        p_bwd = IDENTITY4 + sign * GAMMA[mu]
        psi_fwd = np.roll(psi, -1, axis=ax)                   # psi(x + mu)
        u_psi = np.einsum("...ab,...sb->...sa", ut[mu], psi_fwd)
        out += np.einsum("st,...ta->...sa", p_fwd, u_psi)
        u_back = np.roll(ut[mu], 1, axis=ax)                  # Ut_mu(x - mu)
        psi_bwd = np.roll(psi, 1, axis=ax)                    # psi(x - mu)
        ud_psi = np.einsum("...ba,...sb->...sa", u_back.conj(), psi_bwd)
        out += np.einsum("st,...ta->...sa", p_bwd, ud_psi)
    return out


def dirac(u, psi, kappa, bc):
    """D psi = psi - kappa H psi."""
    return psi - kappa * hop(u, psi, bc)


def dirac_dag(u, psi, kappa, bc):
    """D^dag psi = psi - kappa H^dag psi."""
    return psi - kappa * hop(u, psi, bc, dagger=True)


def gamma5_apply(psi):
    return np.einsum("st,...ta->...sa", GAMMA5, psi)


def hop_block(u, psi, bc, out_parity, dagger=False):
    """H_{p, 1-p}: hop from the opposite-parity part of psi onto parity `out_parity`.

    Fields are whole-lattice arrays; the result is zero off parity `out_parity`.
    """
    par = parity_of_sites(_dims_of(psi))
    src = psi * (par != out_parity)[..., None, None]
    return hop(u, src, bc, dagger) * (par == out_parity)[..., None, None]


def mhat(u, psi_e, kappa, bc):
    """Schur operator on even sites: Mhat = 1 - kappa^2 H_eo H_oe.

    With D = [[1, -kappa H_eo], [-kappa H_oe, 1]] in (even, odd) blocks, the
    Schur complement of the odd-odd identity block is Mhat; det D = det Mhat.
    """
    par = parity_of_sites(_dims_of(psi_e))
    pe = psi_e * (par == 0)[..., None, None]
    t = hop_block(u, pe, bc, 1)
    return pe - kappa * kappa * hop_block(u, t, bc, 0)


def mhat_dag(u, psi_e, kappa, bc):
    """Mhat^dag = 1 - kappa^2 (H^dag)_eo (H^dag)_oe = gamma5 Mhat gamma5."""
    par = parity_of_sites(_dims_of(psi_e))
    pe = psi_e * (par == 0)[..., None, None]
    t = hop_block(u, pe, bc, 1, dagger=True)
    return pe - kappa * kappa * hop_block(u, t, bc, 0, dagger=True)


def mdagm_full(u, psi, kappa, bc):
    """D^dag D psi on the whole lattice."""
    return dirac_dag(u, dirac(u, psi, kappa, bc), kappa, bc)


def mdagm_eo(u, psi_e, kappa, bc):
    """Mhat^dag Mhat psi_e on the even sites."""
    return mhat_dag(u, mhat(u, psi_e, kappa, bc), kappa, bc)


def hop_sites(u, psi, bc, sites, dagger=False):
    """(H psi) at a list of sites only, by explicit neighbour arithmetic.

    `sites` is an int array of canonical site indices i = x + Lx(y + Ly(z + Lz t)).
    Returns [len(sites), 4, 3].  Used to check outputs of lattices too large
    for a whole-lattice oracle apply in a test's time budget.
    """
    lx, ly, lz, lt = _dims_of(psi)
    dims = (lx, ly, lz, lt)
    flat_psi = psi.reshape(-1, 4, 3)
    flat_u = u.reshape(4, -1, 3, 3)
    sites = np.asarray(sites, dtype=np.int64)
    x = sites % lx
    y = (sites // lx) % ly
    z = (sites // (lx * ly)) % lz
    t = sites // (lx * ly * lz)
    coord = [x, y, z, t]
    sign = -1.0 if dagger else 1.0
    out = np.zeros((len(sites), 4, 3), dtype=np.complex128)

    def index(c):
        return c[0] + lx * (c[1] + ly * (c[2] + lz * c[3]))

    for mu in range(4):
        fwd = list(coord)
        fwd[mu] = (coord[mu] + 1) % dims[mu]
        bwd = list(coord)
        bwd[mu] = (coord[mu] - 1) % dims[mu]
        ph = complex(bc[mu])
        ph_f = np.where(coord[mu] == dims[mu] - 1, ph, 1.0)       # link x -> x+mu crosses
        ph_b = np.where(coord[mu] == 0, np.conj(ph), 1.0)          # link x-mu -> x crosses
        u_f = flat_u[mu, sites] * ph_f[:, None, None]
        u_b = flat_u[mu, index(bwd)].conj().transpose(0, 2, 1) * ph_b[:, None, None]
        term_f = np.einsum("nab,nsb->nsa", u_f, flat_psi[index(fwd)])
        term_b = np.einsum("nab,nsb->nsa", u_b, flat_psi[index(bwd)])
        out += np.einsum("st,nta->nsa", IDENTITY4 - sign * GAMMA[mu], term_f)
        out += np.einsum("st,nta->nsa", IDENTITY4 + sign * GAMMA[mu], term_b)
    return out
