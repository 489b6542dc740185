"""The largest lattice the tests run: 64^3x128, 33.5 M sites (GPU; slow test).

At this size one FP64 parity field is 3.2 GB and the FP64 links 12.9 GB, so
every byte offset into a field, a batch of right-hand sides or the links is
past 2^31: an index computed in 32 bits anywhere in packing, the hopping
kernels, the vector kernels or the solver would show here.  Checked against
the oracle on sampled sites (both parities, the lattice corners, random
interior sites): D psi in FP64 and FP16 storage, and the mixed FP16 even-odd
solve of the Dirac system, whose residual b - D x the oracle recomputes on
the samples.  About 110 GB of device memory.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP

pytestmark = pytest.mark.gpu

DIMS = (64, 64, 64, 128)
KAPPA = 0.124


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def test_max_size_dirac_and_solve(cola):
    import torch

    vol = int(np.prod(DIMS))
    # inputs drawn on the device (the host recipe would take minutes at this size)
    u_dev = synth.gauge_field_device(DIMS, 0.25, synth.seed_for(6, 0))
    b_dev = synth.gaussian_spinor_device(DIMS, synth.seed_for(6, 1))
    b_np = b_dev.cpu().numpy()
    g = cola.Gauge(u_dev, DIMS, KAPPA, BC_AP, precisions=("f64", "f16"), recon={"f64": 12, "f16": 12})
    rng = np.random.default_rng(17)
    sites = np.unique(np.concatenate([[0, 1, vol // 2, vol - 2, vol - 1], rng.integers(0, vol, 600)]))
    idx = torch.from_numpy(sites).cuda()
    got = {}
    for prec in ("f64", "f16"):
        out = cola.apply_dirac(g, b_dev, prec=prec)
        got[prec] = out.reshape(-1, 4, 3).index_select(0, idx).cpu().numpy()
        del out
    x, info = cola.cg_solve(g, b_dev, tol=1e-10, op="eo", system="dirac", inner="f16", delta=0.1, use_graph=True)
    assert info[0].status == 0 and info[0].true_rel_resid <= 1e-10
    x_s = x.reshape(-1, 4, 3).index_select(0, idx).cpu().numpy()
    del g
    u = u_dev.cpu().numpy()
    del u_dev
    torch.cuda.empty_cache()
    want = b_np.reshape(-1, 4, 3)[sites] - KAPPA * oracle.hop_sites(u, b_np, BC_AP, sites)
    for prec, tol in (("f64", 1e-13), ("f16", 2e-3)):
        err = np.linalg.norm(got[prec] - want) / np.linalg.norm(want)
        assert err < tol, (prec, err)
    # residual of the solve on the samples: b - (x - kappa H x)
    xf = x.cpu().numpy()
    del x
    r = b_np.reshape(-1, 4, 3)[sites] - (x_s - KAPPA * oracle.hop_sites(u, xf, BC_AP, sites))
    rms_r = np.sqrt(np.mean(np.abs(r) ** 2))
    rms_b = np.sqrt(np.mean(np.abs(b_np.reshape(-1, 4, 3)[sites]) ** 2))
    assert rms_r / rms_b < 5 * max(info[0].true_rel_resid, 1e-12)


def test_device_inputs_equal_host_inputs(cola):
    dims = (4, 4, 4, 8)
    s = synth.gaussian_spinor_device(dims, synth.seed_for(6, 1), chunk=1000).cpu().numpy()
    assert np.max(np.abs(s - synth.gaussian_spinor(dims, synth.seed_for(6, 1)))) < 1e-15
    u = synth.gauge_field_device(dims, 0.25, synth.seed_for(6, 0), chunk=333).cpu().numpy()
    assert np.max(np.abs(u - synth.gauge_field(dims, 0.25, synth.seed_for(6, 0)))) < 1e-14
