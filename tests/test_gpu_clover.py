"""GPU clover term against the FP64 oracle.

Element-by-element comparisons on seeded inputs: the construction of A and
A^-1 (through their application to random spinors, every parity and
precision), the clover Dirac operator D = A - kappa H and its adjoint, the
even-odd and whole-lattice normal operators, solves whose true residual the
oracle recomputes, multi-RHS and batched solves, gauge updates, detaching,
autograd through the clover operator, and the FP64 links the term needs.  Tolerances as for the Wilson
operator: 1e-13 (FP64), 1e-6 (FP32 storage), 2e-3 (FP16 storage).
"""
import numpy as np
import pytest

import oracle
import oracle.clover as ocl
import synth
from helpers import BC_AP, TOL, lattice_inputs, rel_err, to_dev

pytestmark = pytest.mark.gpu

DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 8, 10)]
KAPPA = 0.124
CSW = 1.3


@pytest.fixture(scope="module")
def cola():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_00850_gb300 as cola
    from paper_2302_00850_gb300 import build

    build.build()
    return cola


def clover_gauge(cola, u, dims, kappa=KAPPA, csw=CSW, bc=BC_AP, recon=None, precisions=("f64", "f32", "f16")):
    g = cola.Gauge(to_dev(u), dims, kappa, bc, precisions=precisions, recon=recon or {})
    g.attach_clover(csw)
    return g


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_clover_and_inverse_apply(cola, dims, prec):
    u, psi = lattice_inputs(dims, eps=0.5, config=60)
    g = clover_gauge(cola, u, dims)
    assert g.csw == CSW
    a = ocl.clover_matrix(u, KAPPA, CSW)
    want = ocl.apply_site_matrix(a, psi)
    want_inv = ocl.apply_site_matrix(ocl.invert_site_matrix(a), psi)
    got = cola.apply_clover(g, to_dev(psi), prec=prec).cpu().numpy()
    got_inv = cola.apply_clover(g, to_dev(psi), inverse=True, prec=prec).cpu().numpy()
    assert rel_err(got, want) < TOL[prec], (dims, prec)
    assert rel_err(got_inv, want_inv) < TOL[prec], (dims, prec)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_clover_single_parity_leaves_the_other(cola, prec):
    dims = (4, 6, 2, 8)
    u, psi = lattice_inputs(dims, eps=0.5, config=61)
    g = clover_gauge(cola, u, dims)
    par = oracle.parity_of_sites(dims)
    ainv = ocl.invert_site_matrix(ocl.clover_matrix(u, KAPPA, CSW))
    keep = synth.gaussian_spinor(dims, synth.seed_for(61, 5))
    pin = cola.pack(g, to_dev(psi), prec)
    for parity in (0, 1):
        out = cola.pack(g, to_dev(keep), prec)
        cola.clover(g, out, pin, parity=parity, inverse=True, prec=prec)
        got = cola.unpack(g, out, prec).cpu().numpy()
        m = (par == parity)[..., None, None]
        want = np.where(m, ocl.apply_site_matrix(ainv, psi), keep)
        assert rel_err(got, want) < TOL[prec]
    # in place
    cola.clover(g, pin, pin, parity=2, inverse=False, prec=prec)
    got = cola.unpack(g, pin, prec).cpu().numpy()
    assert rel_err(got, ocl.apply_site_matrix(ocl.clover_matrix(u, KAPPA, CSW), psi)) < TOL[prec]


def test_unit_gauge_clover_is_identity(cola):
    dims = (4, 4, 2, 4)
    u = synth.unit_gauge(dims)
    psi = synth.gaussian_spinor(dims, synth.seed_for(62, 1))
    g = clover_gauge(cola, u, dims)
    # A = 1 at U = 1; the packed spin basis's rotations in and out of the
    # chirality blocks leave only FP64 rounding
    got = cola.apply_clover(g, to_dev(psi)).cpu().numpy()
    assert rel_err(got, psi) < 1e-15
    got = cola.apply_clover(g, to_dev(psi), inverse=True).cpu().numpy()
    assert rel_err(got, psi) < 1e-15
    got = cola.apply_dirac(g, to_dev(psi)).cpu().numpy()
    assert rel_err(got, oracle.dirac(u, psi, KAPPA, BC_AP)) < 1e-15


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f32", 12), ("f16", 12), ("f16", 18)])
def test_clover_dirac_operator(cola, dims, prec, recon):
    bc = (np.exp(0.4j), 1.0, 1.0, -1.0)
    u, psi = lattice_inputs(dims, eps=0.4, config=63)
    g = clover_gauge(cola, u, dims, bc=bc, recon={prec: recon, "f64": 18 if prec != "f64" else recon})
    for dag in (False, True):
        got = cola.apply_dirac(g, to_dev(psi), dagger=dag, prec=prec).cpu().numpy()
        want = (ocl.dirac_clover_dag if dag else ocl.dirac_clover)(u, psi, KAPPA, bc, CSW)
        assert rel_err(got, want) < TOL[prec], (dims, prec, recon, dag)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_clover_normal_operators(cola, prec):
    dims = (4, 6, 2, 8)
    u, psi = lattice_inputs(dims, eps=0.4, config=64)
    g = clover_gauge(cola, u, dims)
    e = oracle.even_mask(dims)[..., None, None]
    pin = cola.pack(g, to_dev(psi), prec)
    out = g.empty_packed(prec).zero_()   # the odd half is left as it was
    cola.mdagm(g, out, pin, op="eo", prec=prec)
    got = cola.unpack(g, out, prec).cpu().numpy() * e
    want = ocl.mdagm_eo_clover(u, psi * e, KAPPA, BC_AP, CSW)
    assert rel_err(got, want) < TOL[prec]
    cola.mdagm(g, out, pin, op="full", prec=prec)
    got = cola.unpack(g, out, prec).cpu().numpy()
    assert rel_err(got, ocl.mdagm_full_clover(u, psi, KAPPA, BC_AP, CSW)) < TOL[prec]


def test_noalloc_normal_operator_with_clover(cola):
    import torch

    dims = (4, 4, 4, 8)
    u, psi = lattice_inputs(dims, eps=0.4, config=65)
    g = clover_gauge(cola, u, dims)
    for prec in ("f64", "f16"):
        pin = cola.pack(g, to_dev(psi), prec)
        for op in (0, 1):
            a = g.empty_packed(prec)
            b = g.empty_packed(prec)
            a.zero_()
            b.zero_()
            cola.mdagm(g, a, pin, op=("full", "eo")[op], prec=prec)
            from paper_2302_00850_gb300._lib import check

            check(g.lib.cola_mdagm_apply_noalloc(g.handle, b.data_ptr(), pin.data_ptr(), op, cola.api.PREC[prec], 1,
                                                 torch.cuda.current_stream().cuda_stream))
            torch.cuda.synchronize()
            assert torch.equal(a, b)


def resid_eo(u, x, b, dims):
    e = oracle.even_mask(dims)[..., None, None]
    return rel_err(ocl.mdagm_eo_clover(u, x * e, KAPPA, BC_AP, CSW) * e, b * e)


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
@pytest.mark.parametrize("use_graph", [False, True])
def test_clover_eo_normal_solve(cola, inner, use_graph):
    dims = (4, 6, 4, 8)
    u, b = lattice_inputs(dims, eps=0.3, config=66)
    g = clover_gauge(cola, u, dims)
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op="eo", inner=inner, use_graph=use_graph)
    assert info[0].status == 0
    assert resid_eo(u, x.cpu().numpy(), b, dims) <= 1e-10
    if inner != "f64":
        assert info[0].reliable_updates >= 2


@pytest.mark.parametrize("inner", ["f64", "f16"])
@pytest.mark.parametrize("op", ["eo", "full"])
def test_clover_dirac_system(cola, inner, op):
    dims = (4, 4, 4, 8)
    u, b = lattice_inputs(dims, eps=0.3, config=67)
    g = clover_gauge(cola, u, dims)
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op=op, system="dirac", inner=inner, use_graph=True)
    x = x.cpu().numpy()
    res = rel_err(ocl.dirac_clover(u, x, KAPPA, BC_AP, CSW), b)
    assert info[0].status == 0
    assert res <= 1e-10
    assert abs(info[0].true_rel_resid - res) < 1e-12
    # the Wilson solution differs: the clover term is really in the operator
    xw = oracle.solve_dirac_eo(u, b, KAPPA, BC_AP, tol=1e-8)[0]
    assert rel_err(x, xw) > 1e-3


def test_clover_multi_rhs_matches_single(cola):
    dims = (4, 4, 4, 8)
    u = synth.gauge_field(dims, 0.3, synth.seed_for(68, 0))
    b = synth.gaussian_spinor(dims, synth.seed_for(68, 1), nrhs=3)
    g = clover_gauge(cola, u, dims)
    x, info = cola.cg_solve(g, to_dev(b), tol=1e-10, op="eo", inner="f32", use_graph=True)
    x = x.cpu().numpy()
    for r in range(3):
        assert info[r].status == 0
        assert resid_eo(u, x[r], b[r], dims) <= 1e-10
        x1, _ = cola.cg_solve(g, to_dev(b[r]), tol=1e-10, op="eo", inner="f32", use_graph=True)
        assert rel_err(x[r], x1.cpu().numpy()) < 1e-8


def test_clover_batched_uneven_lattices(cola):
    shapes = [(4, 4, 4, 8), (2, 4, 6, 4), (6, 2, 2, 2)]
    csws = [1.3, 0.9, 1.7]
    gs, bs, us = [], [], []
    for k, (dims, csw) in enumerate(zip(shapes, csws)):
        u = synth.gauge_field(dims, 0.3, synth.seed_for(69, 2 * k))
        b = synth.gaussian_spinor(dims, synth.seed_for(69, 2 * k + 1), nrhs=2)
        gs.append(clover_gauge(cola, u, dims, csw=csw))
        us.append(u)
        bs.append(to_dev(b))
    xs, infos = cola.cg_solve_batched(gs, bs, tol=1e-10, op="eo", system="dirac", inner="f16", use_graph=True)
    for k, (dims, csw) in enumerate(zip(shapes, csws)):
        for r in range(2):
            b = bs[k][r].cpu().numpy()
            res = rel_err(ocl.dirac_clover(us[k], xs[k][r].cpu().numpy(), KAPPA, BC_AP, csw), b)
            assert infos[k][r].status == 0 and res <= 1e-10, (k, r, res)


def test_batch_must_agree_on_clover(cola):
    dims = (4, 4, 4, 4)
    u, b = lattice_inputs(dims, config=70)
    g1 = clover_gauge(cola, u, dims)
    g2 = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP)
    with pytest.raises(cola.ColaError, match="clover"):
        cola.cg_solve_batched([g1, g2], [to_dev(b), to_dev(b)], tol=1e-10, op="eo", inner="f64")


def test_gauge_update_rebuilds_and_detach_restores(cola):
    dims = (4, 6, 2, 8)
    u1, psi = lattice_inputs(dims, eps=0.4, config=71)
    u2 = synth.gauge_field(dims, 0.4, synth.seed_for(71, 7))
    g = clover_gauge(cola, u1, dims)
    g.update(to_dev(u2))
    got = cola.apply_dirac(g, to_dev(psi)).cpu().numpy()
    assert rel_err(got, ocl.dirac_clover(u2, psi, KAPPA, BC_AP, CSW)) < TOL["f64"]
    g.attach_clover(0.0)
    assert g.csw == 0.0
    got = cola.apply_dirac(g, to_dev(psi)).cpu().numpy()
    assert rel_err(got, oracle.dirac(u2, psi, KAPPA, BC_AP)) < TOL["f64"]
    with pytest.raises(cola.ColaError):
        cola.apply_clover(g, to_dev(psi))


def test_clover_needs_fp64_links(cola):
    dims = (4, 4, 4, 4)
    u, psi = lattice_inputs(dims, config=72)
    g32 = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f32",))
    with pytest.raises(cola.ColaError, match="FP64"):
        g32.attach_clover(CSW)
    assert g32.csw == 0.0


def test_dirac_op_autograd_gradients_with_clover(cola):
    import torch

    dims = (4, 4, 2, 4)
    u, psi = lattice_inputs(dims, eps=0.4, config=73)
    gy = synth.gaussian_spinor(dims, synth.seed_for(73, 4))
    p = to_dev(psi).requires_grad_(True)
    y = cola.DiracOp.apply(to_dev(u), p, dims, KAPPA, BC_AP, CSW)
    assert rel_err(y.detach().cpu().numpy(), ocl.dirac_clover(u, psi, KAPPA, BC_AP, CSW)) < 1e-13
    (gp,) = torch.autograd.grad(y, p, to_dev(gy))
    assert rel_err(gp.cpu().numpy(), ocl.dirac_clover_dag(u, gy, KAPPA, BC_AP, CSW)) < 1e-13
    lk = to_dev(u).requires_grad_(True)
    y = cola.DiracOp.apply(lk, to_dev(psi), dims, KAPPA, BC_AP, CSW)
    (gl,) = torch.autograd.grad(y, lk, to_dev(gy))
    want = oracle.dirac_link_grad(u, psi, gy, KAPPA, BC_AP) + ocl.dirac_link_grad_clover(u, psi, gy, KAPPA, CSW)
    assert rel_err(gl.cpu().numpy(), want) < 1e-13


def test_multishift_and_eigensolver_on_a_clover_handle(cola):
    """Both drive the handle's operator, so with a clover term they solve / diagonalise the clover
    normal operator: checked against the oracle's Mhat^dag Mhat with A."""
    import oracle.eig as oeig

    dims = (4, 4, 4, 4)
    u, b = lattice_inputs(dims, eps=0.3, config=74)
    g = clover_gauge(cola, u, dims)
    e = oracle.even_mask(dims)[..., None, None]
    op = lambda v: ocl.mdagm_eo_clover(u, v * e, KAPPA, BC_AP, CSW) * e  # noqa: E731
    shifts = [0.0, 0.2]
    x, infos = cola.multishift_solve(g, to_dev(b), shifts, tol=1e-10, op="eo", inner="f16")
    for k, sg in enumerate(shifts):
        xk = x[k].cpu().numpy() * e
        assert infos[k].status == 0
        assert rel_err(op(xk) + sg * xk, b * e) <= 1e-10
    v0 = to_dev(synth.gaussian_spinor(dims, synth.seed_for(74, 3), nrhs=6))
    vals, vecs, info = cola.eig_lowest(g, v0, nev=4, op="eo", tol=1e-9)
    want, _ = oeig.lowest_dense(op, dims[::-1] + (4, 3), 4, mask=e)
    assert info.status == 0
    assert np.max(np.abs(vals.numpy() - want) / want) < 1e-9
    res = oeig.residuals(op, vals.numpy(), vecs.cpu().numpy())
    assert np.all(res <= 1e-9 * vals.numpy())
