"""The seeded input generators of the batched and serving workloads: sizes, parameter
ranges, determinism, and the arrival process."""
import numpy as np

import workloads as wl


def test_serving_parameters_cover_the_stated_ranges():
    ps = [wl.serving_params(np.random.default_rng([7, i])) for i in range(3000)]
    n = np.array([p[0] for p in ps])
    rho = np.array([p[1] for p in ps])
    lik = np.array([p[2] for p in ps])
    assert n.min() >= 1000 and n.max() <= 200_000
    # log-uniform: the log of n is uniform, mean (log 1e3 + log 2e5) / 2
    assert abs(np.log(n).mean() - 0.5 * (np.log(1e3) + np.log(2e5))) < 0.1
    assert rho.min() >= 0.02 and rho.max() <= 0.2
    assert 0.45 < (lik == wl.LIK_POISSON_LOG).mean() < 0.55


def test_batched_parameters_cover_the_stated_ranges():
    ps = [wl.batched_params(np.random.default_rng([5, i])) for i in range(2000)]
    n = np.array([p[0] for p in ps])
    assert n.min() >= 5000 and n.max() <= 50_000
    assert {p[1] for p in ps} == {10, 20, 30}
    # the stated total for 256 problems is about 5e6 points
    assert 3.5e6 < sum(wl.batched_params(np.random.default_rng([5, i]))[0] for i in range(256)) < 6.5e6


def test_generators_are_deterministic_and_consistent():
    a, b = wl.serving_problem(3, n=2000), wl.serving_problem(3, n=2000)
    assert np.array_equal(a.locs, b.locs) and np.array_equal(a.y, b.y) and np.array_equal(a.order, b.order)
    assert a.m == 20 and a.cov == wl.COV_MATERN15 and a.test_locs.shape == (1000, 2)
    assert sorted(a.order.tolist()) == list(range(2000))
    c = wl.batched_problem(4, n=3000)
    assert c.cov == wl.COV_EXPONENTIAL and c.lik == wl.LIK_BERNOULLI_LOGIT and c.test_locs is None
    assert set(np.unique(c.y)) <= {0.0, 1.0}
    # the full-size draw uses the parameters drawn first from the same generator
    assert wl.serving_problem(11).n == wl.serving_params(np.random.default_rng([7, 11]))[0]


def test_poisson_arrivals_rate():
    t = wl.poisson_arrivals(50.0, 60.0, seed=11)
    assert np.all(np.diff(t) > 0) and t.max() < 60.0
    assert abs(len(t) - 3000) < 5 * np.sqrt(3000)
