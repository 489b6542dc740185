"""GPU hopping term, packing and normal operators against the FP64 oracle.

Element-by-element comparisons on seeded inputs, relative-norm tolerances
1e-13 (FP64), 1e-6 (FP32 storage), 2e-3 (FP16 storage), over several lattice
shapes (2^4 where x + mu and x - mu coincide, non-cubic extents, sizes that
span several thread blocks with a ragged last block).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP, TOL, lattice_inputs, rel_err, to_dev

pytestmark = pytest.mark.gpu

DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 8, 10)]


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def make_gauge(cola, u, dims, kappa=0.124, bc=BC_AP, recon=None):
    return cola.Gauge(to_dev(u), dims, kappa, bc, precisions=("f64", "f32", "f16"), recon=recon or {})


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_pack_roundtrip(cola, prec):
    dims = (4, 6, 2, 8)
    u, psi = lattice_inputs(dims, nrhs=3)
    g = make_gauge(cola, u, dims)
    back = cola.unpack(g, cola.pack(g, to_dev(psi), prec), prec, nrhs=3).cpu().numpy()
    # The packed spinor is S psi (S = (gamma_t + gamma5) / sqrt(2), unitary):
    # a stored component is (u +- d) / sqrt(2), at most sqrt(2) max|psi| at the
    # site, and unpacking combines two stored components again.  So a
    # canonical component carries at most 2 units of the storage rounding
    # relative to the site's max|psi|: 2^-23 for FP32, 2^-10 for FP16 (half an
    # FP16 ulp of the per-site scale), and a few FP64 roundings.
    per_site = np.max(np.abs(back - psi), axis=(-1, -2)) / np.max(np.abs(psi), axis=(-1, -2))
    bound = {"f64": 1e-15, "f32": 2.0 ** -23, "f16": 2.0 ** -10}[prec]
    assert per_site.max() < bound * 1.0001, (prec, per_site.max())


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f32", 12), ("f32", 18), ("f16", 12), ("f16", 18)])
def test_hop_both_parities(cola, dims, prec, recon):
    bc = (np.exp(0.4j), 1.0, 1.0, -1.0)
    u, psi = lattice_inputs(dims, config=51)
    g = make_gauge(cola, u, dims, bc=bc, recon={prec: recon})
    pin = cola.pack(g, to_dev(psi), prec)
    for dag in (False, True):
        pout = g.empty_packed(prec)
        cola.dslash(g, pout, pin, parity=2, dagger=dag, prec=prec)
        got = cola.unpack(g, pout, prec).cpu().numpy()
        want = oracle.hop(u, psi, bc, dagger=dag)
        assert rel_err(got, want) < TOL[prec], (dims, prec, recon, dag)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_hop_single_parity_and_xpay(cola, prec):
    dims = (4, 6, 2, 8)
    kappa = 0.124
    u, psi = lattice_inputs(dims, config=52)
    xs = synth.gaussian_spinor(dims, synth.seed_for(52, 2))
    g = make_gauge(cola, u, dims, kappa)
    pin = cola.pack(g, to_dev(psi), prec)
    pxs = cola.pack(g, to_dev(xs), prec)
    par = oracle.parity_of_sites(dims)
    for parity in (0, 1):
        for dag in (False, True):
            out = cola.pack(g, to_dev(np.zeros_like(psi)), prec)
            cola.dslash(g, out, pin, pxs, a=0.7, b=-kappa, parity=parity, dagger=dag, prec=prec)
            got = cola.unpack(g, out, prec).cpu().numpy()
            mask = (par == parity)[..., None, None]
            want = (0.7 * xs - kappa * oracle.hop(u, psi, BC_AP, dagger=dag)) * mask
            assert rel_err(got, want) < TOL[prec]
            assert np.all(got[~np.broadcast_to(mask, got.shape)] == 0)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_dirac_full(cola, prec):
    dims = (6, 4, 8, 10)
    kappa = 0.124
    u, psi = lattice_inputs(dims, config=53)
    g = make_gauge(cola, u, dims, kappa)
    for dag in (False, True):
        got = cola.apply_dirac(g, to_dev(psi), dagger=dag, prec=prec).cpu().numpy()
        want = (oracle.dirac_dag if dag else oracle.dirac)(u, psi, kappa, BC_AP)
        assert rel_err(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("op", ["eo", "full"])
def test_mdagm(cola, prec, op):
    dims = (4, 6, 2, 8)
    kappa = 0.124
    u, psi = lattice_inputs(dims, config=54)
    g = make_gauge(cola, u, dims, kappa)
    pin = cola.pack(g, to_dev(psi), prec)
    pout = cola.pack(g, to_dev(np.zeros_like(psi)), prec)
    cola.mdagm(g, pout, pin, op=op, prec=prec)
    got = cola.unpack(g, pout, prec).cpu().numpy()
    if op == "eo":
        e = oracle.even_mask(dims)[..., None, None]
        want = oracle.mdagm_eo(u, psi * e, kappa, BC_AP)
        got = got * e
    else:
        want = oracle.mdagm_full(u, psi, kappa, BC_AP)
    tol = {"f64": 1e-13, "f32": 2e-6, "f16": 6e-3}[prec]  # four chained applies
    assert rel_err(got, want) < tol


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [2, 5, 12])
def test_multi_rhs_equals_single(cola, prec, nrhs):
    dims = (4, 4, 6, 8)
    u, psi = lattice_inputs(dims, config=55, nrhs=nrhs)
    g = make_gauge(cola, u, dims)
    pin = cola.pack(g, to_dev(psi), prec)
    pout = g.empty_packed(prec, nrhs)
    cola.dslash(g, pout, pin, pin, a=1.0, b=-0.124, parity=2, dagger=False, prec=prec, nrhs=nrhs)
    got = cola.unpack(g, pout, prec, nrhs=nrhs).cpu().numpy()
    for r in range(nrhs):
        single_in = cola.pack(g, to_dev(psi[r]), prec)
        single_out = g.empty_packed(prec, 1)
        cola.dslash(g, single_out, single_in, single_in, a=1.0, b=-0.124, parity=2, prec=prec)
        one = cola.unpack(g, single_out, prec).cpu().numpy()
        assert np.array_equal(got[r], one)
        assert rel_err(got[r], oracle.dirac(u, psi[r], 0.124, BC_AP)) < TOL[prec]


def test_errors(cola):
    dims = (4, 4, 4, 4)
    u, psi = lattice_inputs(dims)
    g = cola.Gauge(to_dev(u), dims, 0.12, BC_AP, precisions=("f64",))
    pin = cola.pack(g, to_dev(psi), "f64")
    with pytest.raises(cola.ColaError, match="UNSUPPORTED"):
        cola.dslash(g, g.empty_packed("f32"), pin, prec="f32")
    with pytest.raises(cola.ColaError, match="alias"):
        cola.dslash(g, pin, pin, prec="f64")


@pytest.fixture(scope="module")
def big(cola):
    dims = (32, 32, 32, 64)
    u_dev = synth.gauge_field(dims, 0.25, synth.seed_for(2, 0), device="cuda", as_numpy=False)
    psi = synth.gaussian_spinor(dims, synth.seed_for(2, 1))
    g = cola.Gauge(u_dev, dims, 0.1245, BC_AP, precisions=("f64", "f32", "f16"), recon={"f64": 12})
    u = u_dev.cpu().numpy()
    del u_dev
    return dims, g, u, psi


@pytest.mark.parametrize("prec", ["f16", "f32", "f64"])
def test_full_size_sampled_sites(cola, big, prec):
    """32^3x64 (the mixed-precision workload), links exp(0.25 i H): sampled sites vs the oracle."""
    dims, g, u, psi = big
    pin = cola.pack(g, to_dev(psi), prec)
    pout = g.empty_packed(prec)
    cola.dslash(g, pout, pin, parity=2, prec=prec)
    got = cola.unpack(g, pout, prec).cpu().numpy().reshape(-1, 4, 3)
    rng = np.random.default_rng(3)
    v = 32 * 32 * 32 * 64
    # corners and faces (boundary phases) plus random sites
    sites = np.concatenate([np.array([0, 31, v - 1, v - 32, 32 * 32 * 32 * 63, 32 * 31]),
                            rng.integers(0, v, 4000)])
    want = oracle.hop_sites(u, psi, BC_AP, sites)
    assert rel_err(got[sites], want) < TOL[prec]


def test_gauge_update_repacks_links(cola):
    dims = (4, 6, 2, 8)
    u1, psi = lattice_inputs(dims, config=56)
    u2 = synth.gauge_field(dims, 0.3, synth.seed_for(57, 0))
    g = make_gauge(cola, u1, dims)
    g.update(to_dev(u2))
    for prec in ("f64", "f32", "f16"):
        got = cola.apply_dirac(g, to_dev(psi), prec=prec).cpu().numpy()
        assert rel_err(got, oracle.dirac(u2, psi, 0.124, BC_AP)) < TOL[prec]
