"""Low-lying eigenmodes of the normal operators, FP64 (test infrastructure only).

The paper names eigenmode solvers among COLA's key algorithms, citing
Kalkreuter and Simma (1996), who find the lowest eigenpairs of a Hermitian
positive operator by minimising the Ritz functional.  The eigenpairs
A v = lambda v have a plain definition, so the oracle is that definition:

  lowest_dense    the lowest n eigenpairs of the dense matrix of A (on the
                  even sites for the even-odd operator), by a Hermitian
                  eigendecomposition (small lattices)
  lowest_lanczos  the same through scipy's Lanczos routine on the operator
                  (a library step, for lattices too large for a dense matrix)
  free_field_*    closed forms of the whole spectrum at U = 1, derived below

At U = 1, H on a plane wave e^{ipx} u is h(p) = sum_mu 2 cos p_mu
- 2 i sum_mu gamma_mu sin p_mu, with eigenvalues a +- 2 i |s| (a = sum 2 cos p,
|s|^2 = sum sin^2 p).  D^dag D then has |1 - kappa (a +- 2 i |s|)|^2, twelve
states per momentum.  For the even-odd operator: with the parity sign
e(x) = (-1)^{sum x} = e^{i pi x}, the even projection P_e e^{ipx} is mapped
by H to h(p) P_o e^{ipx} because h(p + pi) = -h(p), so
Mhat P_e e^{ipx} u = P_e (1 - kappa^2 h(p)^2) e^{ipx} u: Mhat^dag Mhat has
|1 - kappa^2 (a + 2 i |s|)^2|^2 (the sign of |s| does not change it), six
states per momentum over all V momenta (p and p + pi give the same state).
Twisted boundaries shift the momenta: p_mu = (2 pi n + theta_mu) / L_mu.
"""
from __future__ import annotations

import itertools

import numpy as np

from .solve import dense_matrix


def _momenta(dims, theta):
    for n in itertools.product(*[range(d) for d in dims]):
        yield [(2 * np.pi * n[k] + theta[k]) / dims[k] for k in range(4)]


def free_field_full_spectrum(dims, kappa, theta=(0.0, 0.0, 0.0, np.pi)):
    """Every eigenvalue of D^dag D at U = 1, sorted (12 V values)."""
    out = []
    for p in _momenta(dims, theta):
        a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
        out += [a * a + 4 * kappa * kappa * sum(np.sin(q) ** 2 for q in p)] * 12
    return np.sort(np.array(out))


def free_field_eo_spectrum(dims, kappa, theta=(0.0, 0.0, 0.0, np.pi)):
    """Every eigenvalue of Mhat^dag Mhat at U = 1 on the even sites, sorted (6 V values)."""
    out = []
    for p in _momenta(dims, theta):
        a = 2 * sum(np.cos(q) for q in p)
        s = np.sqrt(sum(np.sin(q) ** 2 for q in p))
        z = a + 2j * s
        out += [abs(1 - kappa * kappa * z * z) ** 2] * 6
    return np.sort(np.array(out))


def lowest_dense(apply_a, shape, n, mask=None):
    """Lowest n eigenpairs of A on the sites where mask is true (all sites if None).

    Returns (values [n], vectors [n, *shape]) with the vectors zero off the mask.
    """
    m = dense_matrix(apply_a, shape)
    idx = np.arange(m.shape[0]) if mask is None else np.where(np.broadcast_to(mask, shape).reshape(-1))[0]
    sub = m[np.ix_(idx, idx)]
    w, v = np.linalg.eigh(sub)
    vecs = np.zeros((n,) + tuple(shape), dtype=np.complex128)
    for k in range(n):
        full = np.zeros(m.shape[0], dtype=np.complex128)
        full[idx] = v[:, k]
        vecs[k] = full.reshape(shape)
    return w[:n], vecs


def lowest_lanczos(apply_a, shape, n, mask=None, tol=1e-12):
    """Lowest n eigenvalues of A on the mask through scipy's Lanczos routine (eigsh)."""
    from scipy.sparse.linalg import LinearOperator, eigsh

    full = int(np.prod(shape))
    idx = np.arange(full) if mask is None else np.where(np.broadcast_to(mask, shape).reshape(-1))[0]

    def mv(v):
        x = np.zeros(full, dtype=np.complex128)
        x[idx] = np.asarray(v).reshape(-1)
        return apply_a(x.reshape(shape)).reshape(-1)[idx]

    op = LinearOperator((len(idx), len(idx)), matvec=mv, dtype=np.complex128)
    w = eigsh(op, k=n, which="SA", tol=tol, return_eigenvectors=False)
    return np.sort(w)


def residuals(apply_a, values, vectors):
    """|A v - lambda v| / |v| for each pair."""
    return np.array([np.linalg.norm((apply_a(v) - lam * v).ravel()) / np.linalg.norm(v.ravel())
                     for lam, v in zip(values, vectors)])
