"""The seeded candidate generators shared by the tests, the benchmark and the
oracle checks: reproducible, in range, and with the stated mixture."""
import numpy as np

from paper_1407_7737_gb300 import inputs


def test_uniform_is_seeded_and_in_the_box():
    a = inputs.uniform(1000, 7, 3)
    assert np.array_equal(a, inputs.uniform(1000, 7, 3))
    assert not np.array_equal(a, inputs.uniform(1000, 7, 4))
    assert a.shape == (1000, 7) and a.dtype == np.float64
    assert a.min() >= -100.0 and a.max() <= 100.0
    assert abs(a.mean()) < 3.0 and abs(a.std() - 200.0 / np.sqrt(12.0)) < 3.0


def test_near_and_mixed():
    c = np.linspace(-50.0, 50.0, 5)
    x = inputs.near(c, 20000, 0.5, 1)
    assert np.allclose(x.mean(axis=0), c, atol=0.03)
    assert np.allclose(x.std(axis=0), 0.5, rtol=0.03)
    m = inputs.mixed(100, 5, 2, center=c, frac_near=0.1, sigma=1e-3)
    assert np.all(np.abs(m[:10] - c) < 1e-2)           # the first 10 % near c
    assert np.array_equal(m[10:], inputs.uniform(100, 5, 2)[10:])
    assert np.array_equal(inputs.mixed(100, 5, 2), inputs.uniform(100, 5, 2))


def test_shuffled_mixture_is_a_permutation_of_the_mixture():
    c = np.zeros(4)
    s = inputs.shuffled_mixture(1000, 4, 9, c, frac_near=0.3, sigma=10.0)
    m = inputs.mixed(1000, 4, 9, c, 0.3, 10.0)
    assert np.array_equal(np.sort(s, axis=0), np.sort(m, axis=0))
    assert not np.array_equal(s, m)


def test_ragged_instances_ranges():
    items = inputs.ragged_instances(500, 7)
    assert items == inputs.ragged_instances(500, 7)
    fids, Ds, Ns = zip(*items)
    assert min(fids) >= 0 and max(fids) <= 36
    assert set(Ds) <= {10, 30, 50, 100, 500, 1000}
    assert min(Ns) >= 32 and max(Ns) <= 8192
    assert len(set(fids)) > 30 and len(set(Ds)) == 6
