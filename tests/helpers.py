"""Shared helpers of the GPU tests: seeded inputs and error measures."""
import numpy as np

import synth

BC_AP = (1.0, 1.0, 1.0, -1.0)
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3}


def rel_err(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def lattice_inputs(dims, eps=0.3, config=50, nrhs=None):
    u = synth.gauge_field(dims, eps, synth.seed_for(config, 0))
    psi = synth.gaussian_spinor(dims, synth.seed_for(config, 1), nrhs=nrhs)
    return u, psi


def to_dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
