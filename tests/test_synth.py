"""Pins of the seeded input generators (analytic SDFs and samplers)."""
import numpy as np

from paper_2505_21319_gb300 import synth


def test_sphere_sdf_closed_form():
    s = synth.sphere(0.5)
    q = np.array([[0, 0, 0], [0.5, 0, 0], [1, 0, 0], [0, -0.2, 0]], float)
    np.testing.assert_allclose(s.sdf(q), [-0.5, 0.0, 0.5, -0.3], atol=1e-15)


def test_box_and_torus_sdf_closed_form():
    box = synth.Shape(np.array([synth.BOX]), np.array([[0.1, 0.0, 0.0]]), np.array([[0.2, 0.3, 0.4]]))
    q = np.array([[0.1, 0, 0], [0.3, 0, 0], [0.6, 0, 0], [0.6, 0.7, 0], [0.1, 0.25, 0.0]], float)
    np.testing.assert_allclose(box.sdf(q), [-0.2, 0.0, 0.3, np.hypot(0.3, 0.4), -0.05], atol=1e-15)
    tor = synth.Shape(np.array([synth.TORUS]), np.zeros((1, 3)), np.array([[0.3, 0.1, 0.0]]))
    q = np.array([[0.3, 0, 0], [0, 0.4, 0], [0, 0, 0], [0.3, 0, 0.25]], float)
    np.testing.assert_allclose(tor.sdf(q), [-0.1, 0.0, 0.2, 0.15], atol=1e-15)


def test_union_is_min():
    u = synth.random_union(3)
    q = synth.rng(0).uniform(-1, 1, (100, 3))
    parts = [synth.Shape(u.kind[i:i + 1], u.centre[i:i + 1], u.size[i:i + 1]).sdf(q) for i in range(len(u.kind))]
    np.testing.assert_array_equal(u.sdf(q), np.min(parts, axis=0))


def test_surface_points_lie_on_union_boundary():
    u = synth.random_union(5)
    pts = synth.surface_points(u, 2000, synth.rng(1))
    d = u.sdf(pts)
    assert np.all(d >= -1e-6) and np.all(np.abs(d) < 1e-9)


def test_sample_batch_is_seeded_and_split():
    u = synth.random_union(2)
    a = synth.sample_batch(u, 4096, seed=7)
    b = synth.sample_batch(u, 4096, seed=7)
    np.testing.assert_array_equal(a, b)
    assert a.dtype == np.float32 and a.shape == (4096, 4)
    near = np.abs(a[:, 3]) < 0.05
    assert 0.45 < near.mean() < 0.7
    np.testing.assert_allclose(a[:, 3], u.sdf(a[:, :3].astype(np.float64)), atol=1e-7)
    assert not np.array_equal(a, synth.sample_batch(u, 4096, seed=8))


def test_device_sampler_matches_the_host_distribution():
    """sample_batch_torch draws sample_batch's distribution (another random
    stream): half the rows uniform in the cube, half within a few sigma of
    the surface, targets equal to the union SDF at the stored point."""
    import torch
    shape = synth.random_union(3)
    J = 100000
    a = synth.sample_batch(shape, J, seed=5)
    b = synth.sample_batch_torch(shape, J, seed=5, device="cpu").numpy()
    assert b.shape == (J, 4) and b.dtype == np.float32
    np.testing.assert_allclose(b[:, 3], shape.sdf(b[:, :3].astype(np.float64)), atol=1e-7)
    for x in (a, b):
        assert abs((np.abs(x[:, 3]) < 0.05).mean() - 0.54) < 0.01
        assert np.all(np.abs(x[:, :3]) <= 1.2)
    assert abs(np.abs(a[:, 3]).mean() - np.abs(b[:, 3]).mean()) < 2e-3
    g = synth.sdf_grid_torch(shape, 8, "cpu").numpy()
    c = -1 + (np.arange(8) + 0.5) * 0.25
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    np.testing.assert_allclose(g.reshape(-1), shape.sdf(np.stack([X, Y, Z], -1).reshape(-1, 3)), atol=1e-7)
    assert torch.equal(synth.sample_batch_torch(shape, 1000, seed=9, device="cpu"),
                       synth.sample_batch_torch(shape, 1000, seed=9, device="cpu"))
