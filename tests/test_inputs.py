"""The seeded generator: determinism, distribution, recipe shapes."""
import numpy as np

from paper_2206_15397_gb300 import inputs


def test_philox_deterministic_and_counter_sensitive():
    a = inputs.standard_normal(7, 1000, stream=3)
    b = inputs.standard_normal(7, 1000, stream=3)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, inputs.standard_normal(8, 1000, stream=3))
    assert not np.array_equal(a, inputs.standard_normal(7, 1000, stream=4))
    # prefix property: element i does not depend on how many are drawn
    np.testing.assert_array_equal(inputs.standard_normal(7, 10, stream=3), a[:10])


def test_philox_avalanche():
    """Flipping one counter bit flips about half of the 128 output bits."""
    ctr = np.zeros((64, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(64, dtype=np.uint32)
    key = np.zeros((64, 2), dtype=np.uint32)
    base = inputs.philox4x32_10(ctr, key)
    ctr2 = ctr.copy()
    ctr2[:, 2] ^= np.uint32(1)
    diff = inputs.philox4x32_10(ctr2, key) ^ base
    bits = np.unpackbits(diff.view(np.uint8)).reshape(64, -1).sum(axis=1)
    assert 40 < bits.mean() < 88


def test_normal_moments():
    z = inputs.standard_normal(1, 400_000)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    # tail mass beyond 2 sigma: 0.0455
    assert abs((np.abs(z) > 2).mean() - 0.0455) < 0.002


def test_haar_orthogonal():
    v = inputs.haar(3, 50)
    np.testing.assert_allclose(v.T @ v, np.eye(50), atol=1e-13)


def test_activation_recipe():
    xs = inputs.activation_batches(0, 20, 16, 3, alpha=1.0, bias=True)
    assert len(xs) == 3 and xs[0].shape == (21, 16) and xs[0].dtype == np.float32
    np.testing.assert_array_equal(xs[1][-1], np.ones(16, dtype=np.float32))
    om = inputs.omega(0, 20, 5)
    assert om.shape == (20, 5) and om.dtype == np.float32
