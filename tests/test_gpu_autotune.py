"""Autotuned launch shapes change no result (GPU).

The hopping kernel computes each output site independently, so any block
shape gives bit-identical output; the tuner's cache file must hold the
configurations it tuned.  Environment switches are read once per process, so
each setting runs in a child process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_2302_00850_gb300 as cola, synth
dims = (6, 4, 8, 8)
u = synth.gauge_field(dims, 0.3, synth.seed_for(70, 0))
psi = synth.gaussian_spinor(dims, synth.seed_for(70, 1), nrhs=5)
g = cola.Gauge(torch.from_numpy(u).cuda(), dims, 0.124, (1, 1, 1, -1), precisions=("f64", "f32", "f16"))
out = {{}}
for prec in ("f64", "f32", "f16"):
    p = cola.pack(g, torch.from_numpy(psi).cuda(), prec)
    o = g.empty_packed(prec, 5)
    cola.dslash(g, o, p, p, a=1.0, b=-0.124, parity=2, dagger=True, prec=prec, nrhs=5)
    out[prec] = cola.unpack(g, o, prec, nrhs=5).cpu().numpy()
np.savez(sys.argv[1], **out)
"""


def _run(tmp_path, name, env_extra):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_00850_gb300 import build

    build.build()
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT))
    env = dict(os.environ)
    env.update(env_extra)
    res = tmp_path / f"{name}.npz"
    subprocess.run([sys.executable, str(script), str(res)], env=env, check=True, timeout=600)
    return np.load(res)


def test_tuned_shapes_give_identical_results(tmp_path):
    cache = tmp_path / "tune.txt"
    a = _run(tmp_path, "untuned", {"COLA_TUNE": "0"})
    b = _run(tmp_path, "tuned", {"COLA_TUNE": "1", "COLA_TUNE_CACHE": str(cache)})
    for prec in ("f64", "f32", "f16"):
        assert np.array_equal(a[prec], b[prec])
    lines = cache.read_text().splitlines()
    assert len(lines) >= 3 and all("|" in ln for ln in lines)
    c = _run(tmp_path, "cached", {"COLA_TUNE": "1", "COLA_TUNE_CACHE": str(cache)})
    for prec in ("f64", "f32", "f16"):
        assert np.array_equal(a[prec], c[prec])
    assert cache.read_text().splitlines() == lines  # nothing re-tuned
