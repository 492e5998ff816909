"""Host-side parts of the parameter fit (Sec. 4.3): the Hooke-Jeeves pattern
search, the super-parameters and the region assignment."""
import numpy as np

from paper_1502_02908_gb300 import fitting as F
from paper_1502_02908_gb300 import workloads as W


def test_hooke_jeeves_finds_quadratic_minimum_from_1_6_times():
    c = np.array([8.8e-3 * 28, 3.2e-3 * 25, 1e-3 * 22])
    wts = np.array([1.0, 3.0, 0.5])
    f = lambda x: float(np.sum(wts * (x - c) ** 2) / np.sum(c ** 2))
    r = F.hooke_jeeves(f, 1.6 * c, 0.5 * c, iterations=60, min_step=1e-9)
    assert np.all(np.abs(r.x - c) <= 1e-6 * c)
    fs = [h[2] for h in r.history]
    assert all(b <= a for a, b in zip(fs, fs[1:]))        # never increases
    assert r.evaluations < 600


def test_hooke_jeeves_makes_pattern_moves_on_a_valley():
    # Rosenbrock's valley: the pattern moves must carry the search far along it
    f = lambda x: float((1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2)
    r = F.hooke_jeeves(f, np.array([-1.2, 1.0]), np.array([0.5, 0.5]), iterations=400, min_step=1e-10)
    assert r.f < 1e-6 and np.allclose(r.x, [1, 1], atol=1e-2)


def test_hooke_jeeves_respects_iteration_budget():
    calls = []
    f = lambda x: calls.append(1) or float(np.sum(x ** 2))
    r = F.hooke_jeeves(f, np.array([3.0, -2.0, 1.0]), 1.0, iterations=20)
    assert r.iterations == 20 and r.evaluations == len(calls)


def test_superparameters_and_regions():
    k = F.superparameters([8.8e-3, 3.2e-3, 1e-3], [1 / 28, 1 / 25, 1 / 22])
    assert np.allclose(k, [8.8e-3 * 28, 3.2e-3 * 25, 1e-3 * 22])
    reg = F.county_regions(37_000)
    assert reg.dtype == np.int32 and reg.min() == 0 and reg.max() == 20
    assert np.array_equal(reg, F.county_regions(37_000))
    assert np.bincount(reg).min() > 1500
    p = W.Params.broadcast(4, [1e-3, 2e-3, 3e-3], [0.1, 0.2, 0.3], 1.0, 0.01, 1e-6)
    q = F.with_upsilon(p, [5e-3, 6e-3, 7e-3])
    assert np.allclose(q.upsilon, [[5e-3, 6e-3, 7e-3]] * 4) and np.allclose(q.gamma, p.gamma)
    assert F.relative_residual(3.0, 2.0) == 0.5
