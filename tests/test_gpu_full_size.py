"""Full-size workloads checked against the FP64 oracle (GPU; slow tests).

* 32^3x64, kappa 0.1245, links exp(0.25 i H): the mixed FP16/FP32 even-odd CG
  with FP64 reliable updates, in the graph-driven configuration the benchmark
  times; its true relative residual is recomputed by the oracle's own
  whole-lattice operator.
* 24^3x48, kappa 0.124, links exp(0.3 i H), phi = D^dag eta: the fermion force
  from a GPU solve, compared with the oracle's force of the same X, Y on
  sampled links (the oracle formula evaluated link by link).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def test_mixed_fp16_solve_32x32x32x64_true_residual_by_oracle(cola):
    import torch

    dims = (32, 32, 32, 64)
    kappa = 0.1245
    u_dev = synth.gauge_field(dims, 0.25, synth.seed_for(2, 0), device="cuda", as_numpy=False)
    b = synth.gaussian_spinor(dims, synth.seed_for(2, 1))
    g = cola.Gauge(u_dev, dims, kappa, BC_AP, precisions=("f64", "f16"), recon={"f64": 18, "f16": 12})
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op="eo", inner="f16", delta=0.1, use_graph=True)
    assert info[0].status == 0 and info[0].reliable_updates >= 2
    u = u_dev.cpu().numpy()
    del u_dev, g
    torch.cuda.empty_cache()
    e = oracle.even_mask(dims)[..., None, None]
    xr = x.cpu().numpy()
    res = rel_err(oracle.mdagm_eo(u, xr * e, kappa, BC_AP) * e, b * e)
    assert res <= 1e-10, res
    assert abs(res - info[0].true_rel_resid) < 1e-12


def _force_at_links(u, X, Y, kappa, bc, links):
    """Oracle force formula evaluated on a list of (mu, site) links only."""
    lt, lz, ly, lx = X.shape[:4]
    dims = (lx, ly, lz, lt)
    flatX, flatY = X.reshape(-1, 4, 3), Y.reshape(-1, 4, 3)
    flatU = u.reshape(4, -1, 3, 3)
    out = []
    for mu, i in links:
        c = [i % lx, (i // lx) % ly, (i // (lx * ly)) % lz, i // (lx * ly * lz)]
        f = list(c)
        f[mu] = (c[mu] + 1) % dims[mu]
        j = f[0] + lx * (f[1] + ly * (f[2] + lz * f[3]))
        hp = (np.eye(4) - oracle.GAMMA[mu]) @ flatX[j]
        hq = (np.eye(4) + oracle.GAMMA[mu]) @ flatX[i]
        p = np.einsum("sb,sa->ba", hp, flatY[i].conj())
        q = np.einsum("sb,sa->ba", hq, flatY[j].conj())
        ut = flatU[mu, i] * (bc[mu] if c[mu] == dims[mu] - 1 else 1.0)
        w = ut @ (p + q.conj().T)
        out.append([-2 * kappa * np.trace(t @ w).imag for t in oracle.T_GEN])
    return np.array(out)


def test_force_24x24x24x48_sampled_links(cola):
    dims = (24, 24, 24, 48)
    kappa = 0.124
    u_dev = synth.gauge_field(dims, 0.3, synth.seed_for(4, 0), device="cuda", as_numpy=False)
    eta = synth.gaussian_spinor(dims, synth.seed_for(4, 1))
    g = cola.Gauge(u_dev, dims, kappa, BC_AP, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
    phi = cola.apply_dirac(g, to_dev(eta), dagger=True)
    X, info = cola.cg_solve(g, phi, tol=1e-10, op="full", inner="f32", delta=0.1, use_graph=True)
    assert info[0].status == 0
    Y = cola.apply_dirac(g, X)
    F = cola.fermion_force(g, X, Y).cpu().numpy().reshape(4, -1, 8)
    u = u_dev.cpu().numpy()
    Xn, Yn = X.cpu().numpy(), Y.cpu().numpy()
    v = 24 ** 3 * 48
    rng = np.random.default_rng(11)
    links = [(3, v - 1), (3, 0), (0, 23), (1, 24 * 23)] + [(int(m), int(s)) for m, s in
                                                            zip(rng.integers(0, 4, 300), rng.integers(0, v, 300))]
    want = _force_at_links(u, Xn, Yn, kappa, BC_AP, links)
    got = np.array([F[m, s] for m, s in links])
    assert rel_err(got, want) < 1e-13
    # Y = D X and the phi = D^dag eta structure: X is the solution of D^dag D X = D^dag eta, so D X = eta
    assert rel_err(Yn, eta) < 1e-8


def _eo_resid(u, x, b, kappa, dims):
    e = oracle.even_mask(dims)[..., None, None]
    return rel_err(oracle.mdagm_eo(u, x * e, kappa, BC_AP) * e, b * e)


def test_point_sources_and_batch_full_size(cola):
    """12 point sources on 24^3x48 in one graph-captured FP32/FP64 solve, then the batch
    8^4 + 12^3x24 + 16^3x32 + 24^3x48 with 4 Gaussian sources each; residuals by the oracle."""
    import torch

    kappa = 0.124
    d24 = (24, 24, 24, 48)
    u24d = synth.gauge_field(d24, 0.3, synth.seed_for(3, 0), device="cuda", as_numpy=False)
    g24 = cola.Gauge(u24d, d24, kappa, BC_AP, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
    pts = synth.point_sources(d24)
    x, infos = cola.cg_solve(g24, to_dev(pts), tol=1e-10, op="eo", inner="f32", delta=0.1, use_graph=True)
    assert all(i.status == 0 for i in infos)
    u24 = u24d.cpu().numpy()
    xs = x.cpu().numpy()
    del x
    for r in (0, 7, 11):
        assert _eo_resid(u24, xs[r], pts[r], kappa, d24) <= 1e-10
    del xs
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), d24]
    gauges, bs, us = [], [], []
    for k, d in enumerate(dims_list):
        if d == d24:
            u, g = u24, g24
        else:
            u = synth.gauge_field(d, 0.3, synth.seed_for(3, 4 + k))
            g = cola.Gauge(to_dev(u), d, kappa, BC_AP, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
        us.append(u)
        gauges.append(g)
        bs.append(synth.gaussian_spinor(d, synth.seed_for(3, 8 + k), nrhs=4))
    xb, ib = cola.cg_solve_batched(gauges, [to_dev(b) for b in bs], tol=1e-10, op="eo", inner="f32", delta=0.1,
                                   use_graph=True)
    for k, d in enumerate(dims_list):
        assert all(i.status == 0 for i in ib[k])
        rows = range(4) if d != d24 else (2,)
        xk = xb[k].cpu().numpy()
        for r in rows:
            assert _eo_resid(us[k], xk[r], bs[k][r], kappa, d) <= 1e-10
    torch.cuda.empty_cache()
