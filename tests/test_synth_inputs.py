"""Checks of the seeded input generator (CPU only)."""
import numpy as np

import synth


def test_splitmix_is_counter_based():
    a = synth.splitmix64(12345, 0, 100)
    b = synth.splitmix64(12345, 40, 60)
    assert np.array_equal(a[40:], b)
    assert len(set(a.tolist())) == 100


def test_normals_moments():
    g = synth.normals(synth.seed_for(0, 1), 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    z = synth.complex_normals(synth.seed_for(0, 1), (50000,))
    assert abs(np.mean(np.abs(z) ** 2) - 1) < 0.02


def test_gauge_links_are_su3():
    u = synth.gauge_field((4, 4, 2, 6), 0.3, synth.seed_for(0, 0))
    eye = np.eye(3)
    assert np.max(np.abs(np.einsum("...ab,...cb->...ac", u, u.conj()) - eye)) < 1e-14
    assert np.max(np.abs(np.linalg.det(u) - 1)) < 1e-14
    # third row is the conjugate cross product of the first two
    r2 = np.cross(u[..., 0, :], u[..., 1, :]).conj()
    assert np.max(np.abs(u[..., 2, :] - r2)) < 1e-15
    # links near the identity: mean Re tr U / 3 close to 1 - eps^2 <H^2> / 2
    plaq = np.mean(np.trace(u, axis1=-2, axis2=-1).real) / 3
    assert 0.9 < plaq < 0.98


def test_point_sources():
    s = synth.point_sources((4, 4, 4, 4))
    assert s.shape == (12, 4, 4, 4, 4, 4, 3)
    assert np.all(np.sum(np.abs(s), axis=(1, 2, 3, 4, 5, 6)) == 1)
    assert s[5, 0, 0, 0, 0, 1, 2] == 1


def test_device_generators_follow_the_host_recipe():
    """The chunked torch path (run here on the CPU device) draws the same stream."""
    import torch  # noqa: F401

    seed = synth.seed_for(6, 1)
    assert np.array_equal(synth.uniforms(seed, 10, 1000), synth._device_uniforms(seed, 10, 1000, "cpu").numpy())
    dims = (4, 4, 2, 4)
    s_host = synth.gaussian_spinor(dims, seed)
    s_dev = synth.gaussian_spinor_device(dims, seed, device="cpu", chunk=100).numpy()
    assert np.max(np.abs(s_host - s_dev)) < 1e-15
    u_host = synth.gauge_field(dims, 0.3, seed)
    u_dev = synth.gauge_field_device(dims, 0.3, seed, device="cpu", chunk=7).numpy()
    assert np.max(np.abs(u_host - u_dev)) < 1e-15
