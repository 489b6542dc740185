"""Degenerate and edge cases of the GPU path (GPU).

kappa = 0 (D = 1), the free field (U = 1) against its closed form through the
packed kernels, many right-hand sides in one launch, batches that mix a 2^4
lattice with larger ones and the Dirac system in a batch.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP, TOL, rel_err, to_dev

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


@pytest.mark.parametrize("inner", ["f64", "f16"])
def test_kappa_zero_solve_returns_source(cola, inner):
    dims = (4, 4, 4, 4)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(80, 0))
    b = synth.gaussian_spinor(dims, synth.seed_for(80, 1))
    g = cola.Gauge(to_dev(u), dims, 0.0, BC_AP, precisions=("f64", "f16"))
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op="full", inner=inner)
    # FP64: one step is exact; FP16 storage: each reliable update removes a factor ~1e-3
    assert info[0].status == 0 and info[0].iters <= (1 if inner == "f64" else 6)
    assert rel_err(x.cpu().numpy(), b) < 1e-10


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_free_field_plane_wave_through_the_kernels(cola, prec):
    """U = 1 with twisted phases: D e^{ipx} u = [(1 - 2k sum cos p) + 2ik sum gamma sin p] e^{ipx} u."""
    dims = (4, 6, 2, 8)
    kappa = 0.137
    theta = np.array([0.3, -1.1, 2.0, np.pi])
    bc = tuple(np.exp(1j * theta))
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    n = (1, 1, 0, 3)
    p = [(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)]
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u0 = np.random.default_rng(5).normal(size=(4, 3)) + 1j * np.random.default_rng(6).normal(size=(4, 3))
    psi = phase[..., None, None] * u0
    g = cola.Gauge(to_dev(synth.unit_gauge(dims)), dims, kappa, bc, precisions=("f64", "f32", "f16"))
    got = cola.apply_dirac(g, to_dev(psi), prec=prec).cpu().numpy()
    dp = (1 - 2 * kappa * sum(np.cos(q) for q in p)) * np.eye(4) + 2j * kappa * sum(
        oracle.GAMMA[m] * np.sin(p[m]) for m in range(4))
    assert rel_err(got, phase[..., None, None] * (dp @ u0)) < TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_many_rhs_in_one_launch(cola, prec):
    dims = (4, 4, 2, 8)
    nrhs = 37
    u = synth.gauge_field(dims, 0.3, synth.seed_for(81, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(81, 1), nrhs=nrhs)
    g = cola.Gauge(to_dev(u), dims, 0.124, BC_AP, precisions=(prec,))
    pin = cola.pack(g, to_dev(psi), prec)
    pout = g.empty_packed(prec, nrhs)
    cola.dslash(g, pout, pin, parity=2, dagger=True, prec=prec, nrhs=nrhs)
    got = cola.unpack(g, pout, prec, nrhs=nrhs).cpu().numpy()
    for r in (0, 17, 36):
        assert rel_err(got[r], oracle.hop(u, psi[r], BC_AP, dagger=True)) < TOL[prec]


def test_batch_with_2x2x2x2_and_dirac_system(cola):
    kappa = 0.124
    dims_list = [(2, 2, 2, 2), (4, 6, 4, 8)]
    gs, bs, us = [], [], []
    for k, d in enumerate(dims_list):
        u = synth.gauge_field(d, 0.3, synth.seed_for(82 + k, 0))
        us.append(u)
        gs.append(cola.Gauge(to_dev(u), d, kappa, BC_AP, precisions=("f64", "f32")))
        bs.append(synth.gaussian_spinor(d, synth.seed_for(82 + k, 1), nrhs=2))
    for op in ("eo", "full"):
        xs, infos = cola.cg_solve_batched(gs, [to_dev(b) for b in bs], tol=1e-11, op=op, system="dirac",
                                          inner="f32", use_graph=True)
        for k in range(2):
            for r in range(2):
                x = xs[k][r].cpu().numpy()
                res = rel_err(oracle.dirac(us[k], x, kappa, BC_AP), bs[k][r])
                assert res <= 1e-11 and abs(res - infos[k][r].true_rel_resid) < 1e-13
