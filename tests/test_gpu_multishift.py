"""GPU multi-shift CG against the oracle's definition (one CG per shift).

Every x_i must solve (A + sigma_i) x_i = b to the requested true relative
residual as recomputed by the oracle's operator, and agree with the oracle's
own per-shift solve; covered: the even-odd and whole-lattice operators, FP64,
FP32 and FP16 storage in phase 1, shift sets with and without zero, unsorted
and repeated shifts, a single shift (equal to the shifted single solve), the
zero source, and the argument errors.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import BC_AP, lattice_inputs, rel_err, to_dev

pytestmark = pytest.mark.gpu

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


def operator(u, dims, op):
    if op == "eo":
        e = oracle.even_mask(dims)[..., None, None]
        return (lambda v: oracle.mdagm_eo(u, v * e, KAPPA, BC_AP) * e), e
    return (lambda v: oracle.mdagm_full(u, v, KAPPA, BC_AP)), np.ones(dims[::-1] + (1, 1))


def check_against_oracle(u, b, dims, op, shifts, x, infos, tol, sol_tol):
    apply_a, mask = operator(u, dims, op)
    bm = b * mask
    xo, _ = oracle.solve_shifted(apply_a, bm, shifts, tol=1e-12)
    for i, sigma in enumerate(shifts):
        xi = x[i] * mask
        res = rel_err(apply_a(xi) + sigma * xi, bm)
        assert infos[i].status == 0, (i, sigma)
        assert res <= tol, (i, sigma, res)
        assert abs(infos[i].true_rel_resid - res) < 1e-12
        assert rel_err(xi, xo[i]) < sol_tol, (i, sigma)
        if op == "eo":
            assert np.max(np.abs(x[i] * (1 - mask))) == 0.0


@pytest.mark.parametrize("op", ["eo", "full"])
@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_multishift_matches_oracle(cola, op, inner):
    dims = (4, 4, 4, 8)
    u, b = lattice_inputs(dims, eps=0.3, config=80)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64", "f32", "f16"))
    shifts = [0.0, 0.02, 0.3, 1.5]
    x, infos = cola.multishift_solve(g, to_dev(b), shifts, tol=1e-10, op=op, inner=inner)
    check_against_oracle(u, b, dims, op, shifts, x.cpu().numpy(), infos, 1e-10, 1e-7)
    # larger shifts converge in fewer iterations
    its = [i.iters for i in infos]
    assert its[-1] <= its[0]


def test_unsorted_repeated_shifts_without_zero(cola):
    dims = (4, 6, 2, 8)
    u, b = lattice_inputs(dims, eps=0.3, config=81)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64", "f32"))
    shifts = [0.4, 0.05, 2.0, 0.05, 0.11]
    x, infos = cola.multishift_solve(g, to_dev(b), shifts, tol=1e-10, op="eo", inner="f32")
    xn = x.cpu().numpy()
    check_against_oracle(u, b, dims, "eo", shifts, xn, infos, 1e-10, 1e-7)
    assert rel_err(xn[1], xn[3]) < 1e-9


def test_fp64_phase_one_needs_no_refinement(cola):
    dims = (4, 4, 4, 4)
    u, b = lattice_inputs(dims, eps=0.3, config=82)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    shifts = [0.01, 0.1, 1.0]
    x, infos = cola.multishift_solve(g, to_dev(b), shifts, tol=1e-11, op="eo", inner="f64")
    check_against_oracle(u, b, dims, "eo", shifts, x.cpu().numpy(), infos, 1e-11, 1e-8)
    # phase 2 found the FP64 phase-1 solutions converged, or nearly: its first
    # FP64 residual, at most one more
    assert all(i.reliable_updates <= 2 for i in infos)


def test_single_shift_equals_shifted_solve(cola):
    dims = (4, 4, 4, 8)
    u, b = lattice_inputs(dims, eps=0.3, config=83)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64", "f32", "f16"))
    x, infos = cola.multishift_solve(g, to_dev(b), [0.25], tol=1e-10, op="eo", inner="f16")
    check_against_oracle(u, b, dims, "eo", [0.25], x.cpu().numpy(), infos, 1e-10, 1e-7)


def test_zero_source(cola):
    dims = (4, 4, 4, 4)
    u, _ = lattice_inputs(dims, config=84)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64", "f32"))
    b = np.zeros(dims[::-1] + (4, 3), dtype=np.complex128)
    x, infos = cola.multishift_solve(g, to_dev(b), [0.0, 0.5], tol=1e-10, op="full", inner="f32")
    assert np.max(np.abs(x.cpu().numpy())) == 0.0
    assert all(i.status == 0 for i in infos)


def test_multishift_argument_errors(cola):
    dims = (4, 4, 4, 4)
    u, b = lattice_inputs(dims, config=85)
    g = cola.Gauge(to_dev(u), dims, KAPPA, BC_AP, precisions=("f64",))
    with pytest.raises(cola.ColaError, match="shifts"):
        cola.multishift_solve(g, to_dev(b), [0.1, -0.2])
    with pytest.raises(cola.ColaError, match="nshift"):
        cola.multishift_solve(g, to_dev(b), [0.1] * 65)
    with pytest.raises(cola.ColaError, match="inner precision"):
        cola.multishift_solve(g, to_dev(b), [0.1], inner="f32")
