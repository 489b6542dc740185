"""The multi-right-hand-side hopping kernel with 2 and 4 right-hand sides per
thread (GPU).

The autotuner picks how many right-hand sides each thread carries; here a
child process forces each choice (COLA_DSLASH_NR) so that both variants of
the FP32 kernel run, on a lattice with a partial last site block and a
right-hand-side count that leaves the last group partly empty.  Each
right-hand side must equal the oracle's hopping term (FP32 tolerance), the
xpay epilogue must match single-right-hand-side launches, the clover
epilogue the oracle's clover operator, and multi-RHS mixed solves (Wilson,
and clover with the inverse epilogue) must reach the 1e-10 true residual by
the oracle.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json
import numpy as np
import torch
import oracle
import oracle.clover as ocl
import synth
import paper_2302_00850_gb300 as cola

bc = (1.0, 1.0, 1.0, -1.0)
kappa = 0.124
dims = (6, 4, 6, 10)
nrhs = 5
res = {}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


u = synth.gauge_field(dims, 0.3, synth.seed_for(90, 0))
psi = synth.gaussian_spinor(dims, synth.seed_for(90, 1), nrhs=nrhs)
g = cola.Gauge(torch.from_numpy(u).cuda(), dims, kappa, bc, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
pin = cola.pack(g, torch.from_numpy(psi).cuda(), "f32")
out = g.empty_packed("f32", nrhs)
cola.dslash(g, out, pin, parity=2, prec="f32", nrhs=nrhs)
got = cola.unpack(g, out, "f32", nrhs=nrhs).cpu().numpy()
res["hop"] = max(rel(got[r], oracle.hop(u, psi[r], bc)) for r in range(nrhs))
# xpay on one parity: each right-hand side against its own single launch
xo = g.empty_packed("f32", nrhs)
cola.dslash(g, xo, pin, in_self=pin, a=1.0, b=-kappa, parity=0, prec="f32", nrhs=nrhs)
worst = 0.0
for r in range(nrhs):
    p1 = cola.pack(g, torch.from_numpy(psi[r]).cuda(), "f32")
    o1 = g.empty_packed("f32")
    cola.dslash(g, o1, p1, in_self=p1, a=1.0, b=-kappa, parity=0, prec="f32")
    half = o1.numel() // 2
    a = xo.reshape(nrhs, -1)[r][:half].double()
    b = o1.reshape(-1)[:half].double()
    worst = max(worst, float((a - b).norm() / b.norm()))
res["xpay_vs_single"] = worst
# multi-RHS mixed solve (FP32 inner), residuals by the oracle
x, infos = cola.cg_solve(g, torch.from_numpy(psi).cuda(), tol=1e-10, op="eo", inner="f32", use_graph=True)
e = oracle.even_mask(dims)[..., None, None]
xs = x.cpu().numpy()
res["solve"] = max(rel(oracle.mdagm_eo(u, xs[r] * e, kappa, bc) * e, psi[r] * e) for r in range(nrhs))
res["status"] = max(abs(i.status) for i in infos)
# the clover epilogues (Dirac operator with a clover term)
gc = cola.Gauge(torch.from_numpy(u).cuda(), dims, kappa, bc, precisions=("f64", "f32"), recon={"f64": 18, "f32": 12})
gc.attach_clover(1.1)
pc = cola.pack(gc, torch.from_numpy(psi).cuda(), "f32")
oc = gc.empty_packed("f32", nrhs)
cola.dirac(gc, oc, pc, prec="f32", nrhs=nrhs)
gotc = cola.unpack(gc, oc, "f32", nrhs=nrhs).cpu().numpy()
res["clover_dirac"] = max(rel(gotc[r], ocl.dirac_clover(u, psi[r], kappa, bc, 1.1)) for r in range(nrhs))
# the clover inverse epilogue: a multi-RHS clover solve of Mhat^dag Mhat
xc, ic = cola.cg_solve(gc, torch.from_numpy(psi).cuda(), tol=1e-10, op="eo", inner="f32", use_graph=True)
xcs = xc.cpu().numpy()
res["clover_solve"] = max(rel(ocl.mdagm_eo_clover(u, xcs[r] * e, kappa, bc, 1.1) * e, psi[r] * e)
                          for r in range(nrhs))
res["status"] = max(res["status"], max(abs(i.status) for i in ic))
print("RESULT " + json.dumps(res))
'''


@pytest.fixture(scope="module")
def built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_00850_gb300 import build

    build.build()


@pytest.mark.parametrize("nr", [2, 4])
def test_forced_rhs_per_thread(built, nr):
    env = dict(os.environ, COLA_DSLASH_NR=str(nr), PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["hop"] < 1e-6, res
    assert res["xpay_vs_single"] < 1e-6, res
    assert res["status"] == 0 and res["solve"] <= 1e-10, res
    assert res["clover_dirac"] < 1e-6, res
    assert res["clover_solve"] <= 1e-10, res
