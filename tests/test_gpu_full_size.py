"""Full-size workloads checked against the FP64 oracle (GPU; slow tests).

* 32^3x64, kappa 0.1245, links exp(0.25 i H): the mixed FP16/FP32 even-odd CG
  with FP64 reliable updates, in the graph-driven configuration the benchmark
  times; its true relative residual is recomputed by the oracle's own
  whole-lattice operator.
* 24^3x48, kappa 0.124, links exp(0.3 i H), phi = D^dag eta: the fermion force
  through the autograd backward, checked by central finite differences of the
  action and by the closed form S = |eta|^2; the force kernel on seeded X, Y
  against the oracle's formula evaluated link by link.
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


def test_force_24x24x24x48_autograd_fd_and_oracle(cola):
    """The HMC force workload as configured: 24^3x48, kappa 0.124, links
    exp(0.3 i H), phi = D^dag eta with eta standard complex Gaussian.

    * The link gradient comes from PseudofermionAction.backward (the autograd
      path), FP64 force accumulation, projected onto the generators T^a.
    * Central finite differences of the action along a random su(3) field
      omega (U -> exp(+-i eps omega.T) U, eps = 1e-6, perturbed links by the
      oracle's exponential) must match sum F.omega to 1e-5 relative.  The
      action is the variational estimator S~ = 2 Re<phi, X~> - |D X~|^2 from
      FP64 GPU solves to 1e-12, whose error is quadratic in the residual.
    * At the base point S = |eta|^2 exactly.
    * The force kernel, on seeded X and Y (inputs independent of the GPU
      path), matches the oracle's force formula on sampled links to 1e-13;
      the projected autograd gradient equals that kernel on the solve's own
      X and Y = D X.
    """
    import torch

    dims = (24, 24, 24, 48)
    kappa = 0.124
    u_dev = synth.gauge_field(dims, 0.3, synth.seed_for(4, 0), device="cuda", as_numpy=False)
    u = u_dev.cpu().numpy()
    eta = synth.gaussian_spinor(dims, synth.seed_for(4, 1))
    phi_np = oracle.dirac_dag(u, eta, kappa, BC_AP)
    phi = to_dev(phi_np)

    # autograd: dS/dU from PseudofermionAction.backward
    links = u_dev.clone().requires_grad_(True)
    S = cola.PseudofermionAction.apply(links, phi, dims, kappa, BC_AP, 1e-12, "f32")
    S.backward()
    G = links.grad
    T = torch.from_numpy(oracle.T_GEN).to("cuda")
    F_auto = torch.stack([torch.real(torch.sum(G.conj() * (1j * torch.einsum("ab,...bc->...ac", T[a], u_dev)),
                                               dim=(-2, -1))) for a in range(8)], dim=-1)
    F_auto = F_auto.cpu().numpy()  # [4, Lt, Lz, Ly, Lx, 8]
    del G, links
    eta2 = float(np.sum(np.abs(eta) ** 2))
    assert abs(S.item() - eta2) < 1e-8 * eta2

    # the force kernel on the solve's own X, Y = D X equals the projected gradient
    g = cola.Gauge(u_dev, dims, kappa, BC_AP, precisions=("f64",), recon={"f64": 18})

    def s_var(gg):
        x, info = cola.cg_solve(gg, phi, tol=1e-12, op="full", inner="f64", use_graph=True)
        assert info[0].status == 0 and info[0].true_rel_resid <= 1e-12
        dx = cola.apply_dirac(gg, x)
        return (2 * torch.vdot(phi.reshape(-1), x.reshape(-1)).real
                - torch.vdot(dx.reshape(-1), dx.reshape(-1)).real).item(), x, dx

    s0, X, Y = s_var(g)
    assert abs(s0 - eta2) < 1e-10 * eta2  # closed form at phi = D^dag eta
    F = cola.fermion_force(g, X, Y).cpu().numpy()
    assert rel_err(F_auto, F) < 1e-9
    del X, Y

    # central finite differences along omega
    omega = synth.su3_direction(dims, synth.seed_for(4, 2))
    eps = 1e-6
    s = []
    for sgn in (+1, -1):
        gp = cola.Gauge(to_dev(oracle.link_variation(u, omega, sgn * eps)), dims, kappa, BC_AP,
                        precisions=("f64",), recon={"f64": 18})
        s.append(s_var(gp)[0])
        del gp
    fd = (s[0] - s[1]) / (2 * eps)
    an = float(np.sum(F_auto * omega))
    assert abs(fd - an) < 1e-5 * abs(an), (fd, an)

    # the force kernel against the oracle formula on seeded X, Y at sampled links
    Xs = synth.gaussian_spinor(dims, synth.seed_for(4, 3))
    Ys = synth.gaussian_spinor(dims, synth.seed_for(4, 4))
    Fs = cola.fermion_force(g, to_dev(Xs), to_dev(Ys)).cpu().numpy().reshape(4, -1, 8)
    v = 24 ** 3 * 48
    rng = np.random.default_rng(11)
    sampled = [(3, v - 1), (3, 0), (0, 23), (1, 24 * 23)] + [(int(m), int(i)) for m, i in
                                                              zip(rng.integers(0, 4, 300), rng.integers(0, v, 300))]
    want = _force_at_links(u, Xs, Ys, kappa, BC_AP, sampled)
    got = np.array([Fs[m, i] for m, i in sampled])
    assert rel_err(got, want) < 1e-13
    torch.cuda.empty_cache()


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
