"""GPU: region statistics and the goal function of the parameter fit (Sec. 4.3),
parameter replacement, and a short pattern search."""
import numpy as np
import pytest

import oracle
from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import fitting as F
from paper_1502_02908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load_library()


def _oracle_region_moments(w, regions, J, days):
    # the oracle stepped one day at a time; region totals of every replicate
    counts = np.repeat(w.u0[None], w.R, 0)
    phi = np.repeat(w.phi0[None], w.R, 0)
    s1 = np.zeros((days, J, w.nc), np.int64)
    s2 = np.zeros((days, J, w.nc), np.int64)
    for d in range(days):
        r = oracle.run(w, ndays=1, d0=d, counts=counts, phi=phi)
        counts, phi = r.counts, r.phi
        for rep in range(w.R):
            tot = np.zeros((J, w.nc), np.int64)
            for c in range(w.nc):
                tot[:, c] = np.bincount(regions, weights=counts[rep, c], minlength=J).astype(np.int64)
            s1[d] += tot
            s2[d] += tot * tot
    return s1, s2


@pytest.mark.parametrize("launch", ["stream", "graph"])
def test_region_moments_equal_oracle(launch):
    w = W.sise3_national(N=500, T=12, n_events=8_000, R=3)
    J = 5
    regions = F.county_regions(w.N, J, seed=3)
    s = B.Sim.from_workload(w)
    s.set_launch(launch)
    s.set_regions(regions, J)
    s.run(7)
    s.run(w.T - 7)
    g1, g2 = s.region_moments()
    ref1, ref2 = _oracle_region_moments(w, regions, J, w.T)
    assert np.array_equal(g1.astype(np.int64), ref1) and np.array_equal(g2.astype(np.int64), ref2)
    # the goal against an arbitrary reference, vs the formulas on the exact sums
    ref = ref1[:, :, :] // 3 + 7
    G2, VG2 = s.goal(ref[4:10], 4, 6)
    R = 3
    a, b = ref1[4:10].astype(np.float64), ref2[4:10].astype(np.float64)
    np.testing.assert_allclose(G2, np.sum((a / R - ref[4:10]) ** 2), rtol=1e-12)
    np.testing.assert_allclose(VG2, np.sum((R * b - a * a) / (R * (R - 1))), rtol=1e-12)
    s.close()


def test_set_state_and_reset_clear_region_rows():
    w = W.sise3_national(N=300, T=10, n_events=4_000, R=2)
    regions = F.county_regions(w.N, 4, seed=1)
    s = B.Sim.from_workload(w)
    s.set_regions(regions, 4)
    s.run(w.T)
    full1, full2 = s.region_moments()
    s.set_state(np.repeat(w.u0[None], 2, 0), np.repeat(w.phi0[None], 2, 0), 0)
    z1, _ = s.region_moments()
    assert not z1.any()
    s.run(w.T)
    again1, again2 = s.region_moments()
    assert np.array_equal(again1, full1) and np.array_equal(again2, full2)
    s.close()


def test_set_params_equals_fresh_handle():
    w = W.sise3_national(N=800, T=30, n_events=12_000, R=2)
    alt = F.with_upsilon(w.params, [2e-2, 1e-2, 4e-3])
    s = B.Sim.from_workload(w)
    s.set_params(alt)
    s.run(w.T)
    c1, p1, _ = s.state()
    s.close()
    w2 = W.Workload(w.name, w.model, w.N, w.T, w.R, w.u0, w.phi0, alt, w.events, w.seed)
    s2 = B.Sim.from_workload(w2)
    s2.run(w.T)
    c2, p2, _ = s2.state()
    s2.close()
    assert np.array_equal(c1, c2) and np.array_equal(p1, p2)
    with pytest.raises(B.SimError):
        bad = F.with_upsilon(w.params, [-1.0, 0.0, 0.0])
        s3 = B.Sim.from_workload(w)
        try:
            s3.set_params(bad)
        finally:
            s3.close()


def test_pattern_search_reduces_goal_from_1_6_k_star():
    w = W.sise3_national(N=1500, T=60, n_events=25_000)
    J = 6
    regions = F.county_regions(w.N, J, seed=2)
    ups_star = np.array([8.8e-3, 3.2e-3, 1e-3])
    gam = w.params.gamma[0]
    k_star = F.superparameters(ups_star, gam)
    ref = F.reference_totals(w, regions, J, ups_star)
    goal = F.Goal(w, regions, J, ref, trajectories=8)
    try:
        g_star, vg_star = goal(k_star)
        g0, _ = goal(1.6 * k_star)
        assert g0 > g_star > 0 and vg_star > 0
        res = F.hooke_jeeves(lambda k: goal(k)[0], 1.6 * k_star, 0.3 * k_star, iterations=4)
        assert res.f < g0
        assert goal.evaluations >= res.evaluations
    finally:
        goal.close()


def test_gradient_fit_recovers_scales():
    # prevalence goal with the score-function gradient: from (1.5 upsilon*, 0.7 gamma*)
    # back to (upsilon*, gamma*); the target curve comes from independent streams
    w = W.sise_plain(N=400, T=60, n_events=2000, R=256)
    days = np.arange(2, 60, 3)
    target = F.prevalence_curve(w, days, seed_offset=101)
    goal = F.PrevalenceGoal(w, days, target)
    x0 = np.log([1.5, 0.7])
    g0, grad0, se0 = goal(x0)
    assert np.all(np.abs(grad0) > 3 * se0)             # the estimate resolves the gradient here
    r = F.gradient_descent(goal, x0, step=0.2, iterations=25)
    assert r.f < 0.01 * g0
    assert np.all(np.abs(r.x) < 0.08), r.x
