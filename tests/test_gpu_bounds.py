"""The bounds-checking debug build on the GPU (slow test: builds a second library).

libcola built with -DCOLA_BOUNDS checks every neighbour, link and site index
its kernels compute; an index out of range is counted and redirected to 0.
A child process loads that build (COLA_LIB) and runs the operators, solves
and forces on small lattices with extents of 2, 4, 6 and 8 (both link
reconstructions, every storage precision, a batch of two lattices, the
clover term, an HMC trajectory), checks a few results against the oracle,
and reads the violation count, which must be zero.
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
from paper_2302_00850_gb300 import _lib

assert _lib.LIB_PATH.endswith("_build_bounds/libcola.so"), _lib.LIB_PATH
bc = (1.0, 1.0, 1.0, -1.0)
kappa = 0.12
res = {}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a):
    return torch.from_numpy(a).cuda()


for dims in ((2, 2, 2, 2), (4, 6, 2, 8)):
    u = synth.gauge_field(dims, 0.3, synth.seed_for(7, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(7, 1))
    ud, pd = dev(u), dev(psi)
    want = oracle.dirac(u, psi, kappa, bc)
    for recon in (12, 18):
        g = cola.Gauge(ud, dims, kappa, bc, precisions=("f64", "f32", "f16"),
                       recon={"f64": recon, "f32": recon, "f16": recon})
        for prec in ("f64", "f32", "f16"):
            res[f"dirac {dims} r{recon} {prec}"] = rel(cola.apply_dirac(g, pd, prec=prec).cpu().numpy(), want)
        x, info = cola.cg_solve(g, pd, tol=1e-10, op="eo", inner="f16", use_graph=True)
        res[f"solve {dims} r{recon}"] = info[0].true_rel_resid
        cola.fermion_force(g, pd, pd)
        cola.dirac_link_grad(g, pd, pd)
        cola.gauge_force(g, 5.6)
        cola.plaquette(g)
        g.attach_clover(1.0)
        res[f"clover {dims} r{recon}"] = rel(cola.apply_dirac(g, pd).cpu().numpy(),
                                             ocl.dirac_clover(u, psi, kappa, bc, 1.0))
        cola.fermion_force(g, pd, pd)
        cola.dirac_link_grad(g, pd, pd)
        if dims != (2, 2, 2, 2):
            xs, infos = cola.multishift_solve(g, pd, [0.0, 0.5], tol=1e-10, op="eo", inner="f16")
            res[f"multishift {dims} r{recon}"] = max(i.true_rel_resid for i in infos)
        del g
dims_b = [(4, 4, 4, 4), (4, 6, 2, 8)]
gs, bs = [], []
for k, d in enumerate(dims_b):
    gs.append(cola.Gauge(dev(synth.gauge_field(d, 0.3, synth.seed_for(8, k))), d, kappa, bc, precisions=("f64", "f32")))
    bs.append(dev(synth.gaussian_spinor(d, synth.seed_for(8, 10 + k), nrhs=3)))
xs, infos = cola.cg_solve_batched(gs, bs, tol=1e-10, op="eo", inner="f32", use_graph=True)
res["batched"] = max(i.true_rel_resid for row in infos for i in row)
d = (4, 4, 4, 4)
u = synth.gauge_field(d, 0.3, synth.seed_for(9, 0))
ud = dev(u)
mom = dev(synth.su3_direction(d, synth.seed_for(9, 1)))
eta = dev(synth.gaussian_spinor(d, synth.seed_for(9, 2)))
g = cola.Gauge(ud, d, kappa, bc, precisions=("f64", "f32"))
info = cola.hmc_trajectory(g, ud, mom, eta, 5.6, 0.2, 2, "omelyan", uniform=0.0, md_tol=1e-10, md_inner="f32")
res["hmc dH"] = info.dH
torch.cuda.synchronize()
count, line = cola.debug_bounds()
res["violations"], res["first_line"] = count, line
print(json.dumps(res))
'''


def test_bounds_build_reports_no_violation():
    from paper_2302_00850_gb300 import build

    path = build.build_bounds()
    env = dict(os.environ, COLA_LIB=path)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["violations"] == 0, res
    for k, v in res.items():
        if k.startswith("dirac") and k.endswith("f64") or k.startswith("clover"):
            assert v < 1e-13, (k, v)
        elif k.startswith("dirac"):
            assert v < (1e-6 if k.endswith("f32") else 2e-3), (k, v)
        elif k.startswith(("solve", "multishift", "batched")):
            assert v <= 1e-10, (k, v)
    assert res["hmc dH"] == res["hmc dH"], res  # a number, not NaN
