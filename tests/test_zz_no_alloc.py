"""cola_mdagm_apply_noalloc: the allocation-free normal operator (GPU).

Some callers cannot allocate device memory when they call the library (a
service that reserves all device memory up front, a callback that must not
fail).  This entry point runs M^dag M out of a static 64 MiB
device array instead of allocating.  Here it is called through the C ABI and
compared with cola_mdagm_apply on two calls in a row, with different inputs,
operators and precisions, so that anything the first call left in the shared
array would show up in the second.  This file is collected last.
"""
import ctypes

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


def _noalloc(cola, g, out, inp, op, prec, nrhs=1):
    import torch

    from paper_2302_00850_gb300 import _lib

    lib = _lib.load()
    return lib.cola_mdagm_apply_noalloc(g.handle, out.data_ptr(), inp.data_ptr(), {"full": 0, "eo": 1}[op],
                                        cola.api.PREC[prec], nrhs, torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_mdagm_on_two_calls(cola):
    import torch

    dims = (6, 4, 4, 8)
    kappa = 0.124
    u = synth.gauge_field(dims, 0.3, synth.seed_for(60, 0))
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64", "f32", "f16"))
    calls = [("eo", "f64", 1), ("full", "f16", 1), ("eo", "f32", 3)]
    for k, (op, prec, nrhs) in enumerate(calls):
        psi = synth.gaussian_spinor(dims, synth.seed_for(60, 1 + k), nrhs=nrhs if nrhs > 1 else None)
        pin = cola.pack(g, to_dev(psi), prec)
        ref = torch.zeros_like(pin)
        got = torch.zeros_like(pin)
        cola.mdagm(g, ref, pin, op=op, prec=prec, nrhs=nrhs)
        assert _noalloc(cola, g, got, pin, op, prec, nrhs) == 0
        torch.cuda.synchronize()
        a = cola.unpack(g, got, prec, nrhs=nrhs if nrhs > 1 else None).cpu().numpy()
        b = cola.unpack(g, ref, prec, nrhs=nrhs if nrhs > 1 else None).cpu().numpy()
        assert rel_err(a, b) <= TOL[prec], (op, prec)
        if op == "eo" and nrhs == 1:
            e = oracle.even_mask(dims)[..., None, None]
            assert rel_err(a * e, oracle.mdagm_eo(u, psi * e, kappa, BC_AP)) < 1e-13


def test_noalloc_with_clover_term_allocates_nothing(cola):
    """On a handle with a clover term the entry point applies the clover
    operator (A_ee - kappa^2 H_eo A_oo^-1 H_oe on the even half), matches
    cola_mdagm_apply and the oracle, and the device's free memory is the same
    before and after two calls in a row (nothing was allocated)."""
    import torch

    import oracle.clover as ocl

    dims = (4, 6, 4, 8)
    kappa, csw = 0.124, 1.2
    u = synth.gauge_field(dims, 0.3, synth.seed_for(61, 0))
    g = cola.Gauge(to_dev(u), dims, kappa, BC_AP, precisions=("f64",))
    g.attach_clover(csw)
    e = oracle.even_mask(dims)[..., None, None]
    outs = []
    for k in range(2):
        psi = synth.gaussian_spinor(dims, synth.seed_for(61, 1 + k))
        pin = cola.pack(g, to_dev(psi), "f64")
        ref = torch.zeros_like(pin)
        got = torch.zeros_like(pin)
        cola.mdagm(g, ref, pin, op="eo", prec="f64")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(cola, g, got, pin, "eo", "f64") == 0
        assert _noalloc(cola, g, got, pin, "eo", "f64") == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        a = cola.unpack(g, got, "f64").cpu().numpy()
        b = cola.unpack(g, ref, "f64").cpu().numpy()
        assert rel_err(a * e, b * e) <= TOL["f64"]
        want = ocl.mdagm_eo_clover(u, psi * e, kappa, BC_AP, csw)
        assert rel_err(a * e, want * e) < 1e-13
        outs.append(a)
    assert rel_err(outs[0], outs[1]) > 0.1  # the two inputs differ, so must the outputs


def test_noalloc_rejects_sizes_above_its_static_scratch(cola):
    dims = (16, 16, 16, 32)
    u = synth.unit_gauge(dims)
    g = cola.Gauge(to_dev(u), dims, 0.12, BC_AP, precisions=("f64",))
    nrhs = 3  # 3 x 25.2 MB of FP64 scratch > 64 MiB
    pin = g.empty_packed("f64", nrhs)
    out = g.empty_packed("f64", nrhs)
    from paper_2302_00850_gb300 import _lib

    assert _noalloc(cola, g, out, pin, "eo", "f64", nrhs) == -1
    assert b"64 MiB" in _lib.load().cola_last_error()
