"""Conjugate-gradient solves, FP64 (test infrastructure only).

The paper's inverter is a conjugate-gradient solver (Fig. 2 discussion); it
does not print the recurrence, so this is the textbook Hestenes-Stiefel CG
for a Hermitian positive-definite A:

  r = b - A x0, p = r, rho = <r, r>
  repeat:  q = A p;  alpha = rho / <p, q>;  x += alpha p;  r -= alpha q
           rho' = <r, r>;  if sqrt(rho') <= tol |b|: confirm with the true
           residual b - A x (stop if it also meets tol, else restart from it)
           p = r + (rho' / rho) p;  rho = rho'

Norms are Euclidean over every site, spin, colour and re/im part; sums are
numpy's pairwise float64 sums in canonical order, so results are repeatable.
"""
from __future__ import annotations

import numpy as np

from . import wilson


def vdot(a, b):
    """<a, b> = sum conj(a) b, as a pairwise float64 sum."""
    return np.sum(np.conj(a) * b)


def norm2(a):
    return float(np.sum(a.real * a.real + a.imag * a.imag))


def cg(apply_a, b, x0=None, tol=1e-10, max_iter=100000):
    """Solve A x = b.  Returns (x, iterations, true relative residual)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, copy=True)
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - apply_a(x)
    p = r.copy()
    rho = norm2(r)
    it = 0
    while it < max_iter:
        if np.sqrt(rho) <= tol * bnorm:
            r_true = b - apply_a(x)
            rho_true = norm2(r_true)
            if np.sqrt(rho_true) <= tol * bnorm:
                return x, it, np.sqrt(rho_true) / bnorm
            r = r_true
            p = r.copy()
            rho = rho_true
        q = apply_a(p)
        pq = vdot(p, q).real
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rho_new = norm2(r)
        p = r + (rho_new / rho) * p
        rho = rho_new
        it += 1
    r_true = b - apply_a(x)
    return x, it, np.sqrt(norm2(r_true)) / bnorm


def solve_normal_full(u, b, kappa, bc, tol=1e-10, x0=None, max_iter=100000):
    """D^dag D x = b on the whole lattice (unpreconditioned)."""
    return cg(lambda v: wilson.mdagm_full(u, v, kappa, bc), b, x0, tol, max_iter)


def solve_normal_eo(u, b, kappa, bc, tol=1e-10, x0=None, max_iter=100000):
    """Mhat^dag Mhat x_e = b_e on the even sites (b's odd sites are ignored)."""
    par = wilson.parity_of_sites(b.shape[3::-1])
    be = b * (par == 0)[..., None, None]
    return cg(lambda v: wilson.mdagm_eo(u, v, kappa, bc), be, x0, tol, max_iter)


def solve_dirac_eo(u, b, kappa, bc, tol=1e-10, max_iter=100000):
    """D x = b through the even-odd Schur complement and its normal equations.

    bhat_e = b_e + kappa H_eo b_o;  Mhat^dag Mhat x_e = Mhat^dag bhat_e;
    x_o = b_o + kappa H_oe x_e.  Returns (x, iterations, |b - D x| / |b|).
    """
    par = wilson.parity_of_sites(b.shape[3::-1])
    be = b * (par == 0)[..., None, None]
    bo = b * (par == 1)[..., None, None]
    bhat = be + kappa * wilson.hop_block(u, bo, bc, 0)
    rhs = wilson.mhat_dag(u, bhat, kappa, bc)
    xe, it, _ = cg(lambda v: wilson.mdagm_eo(u, v, kappa, bc), rhs, None, tol, max_iter)
    x = xe + bo + kappa * wilson.hop_block(u, xe, bc, 1)
    res = b - wilson.dirac(u, x, kappa, bc)
    return x, it, np.sqrt(norm2(res) / norm2(b))


def dense_matrix(apply_op, shape):
    """Dense matrix of a linear map on complex arrays of `shape`, column by column."""
    n = int(np.prod(shape))
    m = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        m[:, j] = apply_op(e.reshape(shape)).reshape(-1)
        e[j] = 0.0
    return m


def solve_shifted(apply_a, b, shifts, tol=1e-10, max_iter=100000):
    """x_i = (A + sigma_i)^-1 b for every shift, each by its own CG (the definition
    a multi-shift solver must reproduce).  Returns ([x_i], [true relative residual])."""
    xs, res = [], []
    for sigma in shifts:
        x, _, r = cg(lambda v, s=sigma: apply_a(v) + s * v, b, None, tol, max_iter)
        xs.append(x)
        res.append(r)
    return xs, res
