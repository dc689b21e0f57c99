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


def test_philox_known_answers():
    """The block function against the published known-answer vectors."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = inputs.philox4x32_10(np.array([v[0:4]], dtype=np.uint32), np.array([v[4:6]], dtype=np.uint32))[0]
        assert [int(x) for x in out] == v[6:10], r


def test_seeded_omega_definition():
    """The seed path's test matrix: element (i, j) is value i*k + j of the
    stream, values 4b..4b+3 from Philox block b (counter (b, 0, 1)) through two
    Box-Muller pairs; checked element by element on a ragged shape."""
    d, k, seed = 7, 5, (3 << 32) + 11
    om = inputs.seeded_omega(seed, d, k)
    assert om.shape == (d, k) and om.dtype == np.float32
    for e in range(d * k):
        b, t = divmod(e, 4)
        w = inputs.philox4x32_10(np.array([[b, 0, 0, 1]], dtype=np.uint32),
                                 np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint32))[0]
        u = [(int(x) // 512 + 0.5) / 2.0 ** 23 for x in w]
        a = 0 if t < 2 else 2
        rho = np.sqrt(-2.0 * np.log(u[a]))
        z = rho * (np.cos(2 * np.pi * u[a + 1]) if t % 2 == 0 else np.sin(2 * np.pi * u[a + 1]))
        assert om[e // k, e % k] == np.float32(z), e
    # the key's high half matters; the stream itself does not depend on the shape
    assert not np.array_equal(om, inputs.seeded_omega(11, d, k))
    np.testing.assert_array_equal(inputs.seeded_omega(seed, 2, 10).reshape(-1)[:10], om.reshape(-1)[:10])


def test_seeded_omega_moments():
    z = inputs.seeded_omega(5, 1000, 400).astype(np.float64).reshape(-1)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert abs((np.abs(z) > 2).mean() - 0.0455) < 0.002
    # columns of a sketch are uncorrelated
    c = np.corrcoef(inputs.seeded_omega(6, 4000, 8).T.astype(np.float64))
    assert np.abs(c - np.eye(8)).max() < 0.06


def test_training_layer_omega_seeds_are_distinct():
    """The training layer keys every factor's test matrix by (optimiser seed,
    inversion count, factor position): no two inversions or factors of one
    optimiser share a seed, and two optimisers with different seeds differ."""
    from paper_2206_15397_gb300.optim import omega_seed
    seeds = {omega_seed(5, inv, f) for inv in range(200) for f in range(64)}
    assert len(seeds) == 200 * 64
    assert omega_seed(5, 0, 0) != omega_seed(6, 0, 0)
    assert all(0 <= s < 2 ** 64 for s in seeds)
