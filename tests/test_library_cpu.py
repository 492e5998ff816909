"""CPU tests of the C-ABI library (no GPU): it loads, exports every function
include/episim.h declares, validates events, and its host-side event schedule
(per-day dependency levels) reproduces sequential input order."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import workloads as W


def test_library_exports_every_header_symbol():
    L = B.load_library()
    names = B.header_symbols()
    assert "sim_create" in names and "sim_run_days" in names and "sim_schedule_events" in names
    for n in names:
        assert hasattr(L, n), n


def _random_events(rng, N, T, n, model, hub=True):
    na = 3 if model == W.SISE3 else 1
    kinds = [W.EXIT, W.ENTER, W.EXTERNAL] + ([W.INTERNAL] if na > 1 else [])
    kind = rng.choice(kinds, size=n)
    # a few hub nodes make deep dependency chains
    node = np.where(rng.random(n) < (0.3 if hub else 0.0), rng.integers(0, 3, size=n), rng.integers(0, N, size=n))
    dest = (node + rng.integers(1, N, size=n)) % N
    cls = np.where(kind == W.INTERNAL, rng.integers(0, max(na - 1, 1), size=n),
                   np.where(kind == W.ENTER, rng.integers(-1, na, size=n), rng.integers(-1, na, size=n)))
    return W.Events(rng.integers(0, T, size=n).astype(np.int32), kind.astype(np.int32), node.astype(np.int32),
                    np.where(kind == W.EXTERNAL, dest, -1).astype(np.int32),
                    rng.integers(0, 7, size=n).astype(np.int32), cls.astype(np.int32))


@pytest.mark.parametrize("model", [W.SISE, W.SISE3])
def test_schedule_levels_reproduce_input_order(model):
    rng = np.random.default_rng(3)
    N, T = 40, 12
    ev = _random_events(rng, N, T, 4000, model)
    order, level = B.schedule_events(ev, N, model, T)
    assert order.size == len(ev)
    stable = np.argsort(ev.day, kind="stable")              # input index of each position
    day_of = ev.day[stable]
    # execution order is by (day, level, position)
    key = np.stack([day_of[order], level, order])
    assert (np.diff(day_of[order]) >= 0).all()
    same_day = np.diff(day_of[order]) == 0
    assert ((np.diff(level)[same_day] > 0) | ((np.diff(level)[same_day] == 0) & (np.diff(order)[same_day] > 0))).all()
    # the dependency rules hold within every level
    for d in range(T):
        sel = day_of[order] == d
        for L in np.unique(level[sel]):
            idx = stable[order[sel][level[sel] == L]]
            sampled = ev.node[idx][ev.kind[idx] != W.ENTER]
            added = np.concatenate([ev.node[idx][ev.kind[idx] == W.ENTER], ev.dest[idx][ev.kind[idx] == W.EXTERNAL]])
            assert len(np.unique(sampled)) == len(sampled)
            assert not set(sampled.tolist()) & set(added.tolist())
    # applying the schedule equals applying the input order (oracle event processor)
    nc = 6 if model == W.SISE3 else 2
    u0 = rng.integers(0, 30, size=(nc, N)).astype(np.int32)
    w = W.tiny_node(model=model, herd=1, infected=0, copies=N, T=T,
                    params=dict(upsilon=0.0, gamma=0.0, alpha=0.0, beta=0.0, epsilon=0.0), seed=9)
    w.u0 = u0
    seq = oracle.run(w, events=ev)
    c = u0.copy()
    ctr = oracle.apply_events(w, c, order, ev.select(stable[order]))
    assert np.array_equal(c, seq.counts[0])
    assert ctr[1] == seq.counters[0, 1] and ctr[2] == seq.counters[0, 2]
    # a shuffled order inside each level gives the same result too
    perm = np.arange(order.size)
    for d in range(T):
        for L in np.unique(level):
            m = np.nonzero((day_of[order] == d) & (level == L))[0]
            perm[m] = rng.permutation(m)
    c2 = u0.copy()
    oracle.apply_events(w, c2, order[perm], ev.select(stable[order[perm]]))
    assert np.array_equal(c2, seq.counts[0])


# a long list over many days; all of it on the last of three days (empty day
# ranges); on two days of fifty; all of it on one day
@pytest.mark.parametrize("T,days", [(40, None), (3, [2]), (50, [7, 31]), (1, [0])])
def test_schedule_of_a_long_list_equals_its_days_scheduled_alone(T, days):
    # days are scheduled independently (a long list in ranges of days on several
    # threads, then joined): the whole list's schedule restricted to a day equals
    # that day's events scheduled on their own, shifted to the day's first position
    rng = np.random.default_rng(11)
    N, n = 500, 300_000
    ev = _random_events(rng, N, T, n, W.SISE3)
    if days is not None:
        ev.day[:] = rng.choice(days, size=n)
    order, level = B.schedule_events(ev, N, W.SISE3, T)
    stable = np.argsort(ev.day, kind="stable")
    first = np.searchsorted(ev.day[stable], np.arange(T + 1))
    assert order.size == n
    for d in range(T):
        if first[d + 1] == first[d]:
            continue
        one = ev.select(stable[first[d]:first[d + 1]])
        one.day[:] = 0
        o1, l1 = B.schedule_events(one, N, W.SISE3, 1)
        assert np.array_equal(order[first[d]:first[d + 1]], o1 + first[d])
        assert np.array_equal(level[first[d]:first[d + 1]], l1)


def test_schedule_level_depth_of_a_hub_chain():
    # five exits on one node in one day form a chain of five levels; enters on
    # another node share one level
    z = np.zeros(10, np.int32)
    kind = np.array([W.EXIT] * 5 + [W.ENTER] * 5, np.int32)
    node = np.array([0] * 5 + [1] * 5, np.int32)
    ev = W.Events(z, kind, node, z - 1, z + 1, z - 1)
    order, level = B.schedule_events(ev, 4, W.SISE, 1)
    assert sorted(level.tolist()) == [1, 1, 1, 1, 1, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("bad,field,msg", [
    (-1, "day", "day < 0"), (7, "kind", "unknown kind"), (99, "node", "out of range"),
    (-2, "count", "out of range"), (5, "cls", "out of range"),
])
def test_schedule_rejects_bad_events(bad, field, msg):
    one = dict(day=0, kind=W.EXIT, node=0, dest=-1, count=1, cls=-1)
    one[field] = bad
    ev = W.Events(*(np.array([one[k]], np.int32) for k in ("day", "kind", "node", "dest", "count", "cls")))
    with pytest.raises(B.SimError) as ei:
        B.schedule_events(ev, 4, W.SISE, 5)
    assert ei.value.status == B.SIM_E_INVALID_ARG and msg in str(ei.value)


def test_schedule_rejects_self_transfer_and_bad_aging():
    ev = W.Events(*(np.array([x], np.int32) for x in (0, W.EXTERNAL, 1, 1, 1, -1)))
    with pytest.raises(B.SimError):
        B.schedule_events(ev, 4, W.SISE, 5)
    ev = W.Events(*(np.array([x], np.int32) for x in (0, W.INTERNAL, 1, -1, 1, 2)))
    with pytest.raises(B.SimError):
        B.schedule_events(ev, 4, W.SISE3, 5)       # class 3 has no next class


def test_schedule_drops_days_past_horizon():
    ev = W.Events(*(np.array(x, np.int32) for x in ([0, 5, 9], [W.ENTER] * 3, [0, 0, 0], [-1] * 3, [1] * 3, [0] * 3)))
    order, level = B.schedule_events(ev, 2, W.SISE, 6)
    assert order.tolist() == [0, 1]


def test_integer_pipe_division_matches_ieee_on_host():
    rng = np.random.default_rng(5)
    n = 400_000
    ex = rng.integers(1023 - 60, 1023 + 60, size=n, dtype=np.uint64)
    ey = rng.integers(1023 - 60, 1023 + 60, size=n, dtype=np.uint64)
    mx = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    my = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    my[::5] &= np.uint64(0xF)                 # divisors at and near powers of two
    mx[::7] = np.uint64((1 << 52) - 1) - (mx[::7] & np.uint64(0xF))
    x = ((ex << np.uint64(52)) | mx).view(np.float64).copy()
    y = ((ey << np.uint64(52)) | my).view(np.float64).copy()
    x[:4] = [1.0, 3.0, np.nextafter(2.0, 0), 1e-300]
    y[:4] = [3.0, 3.0, np.nextafter(1.0, 2), 1e300]      # last: subnormal quotient path
    out = np.empty(n); ref = np.empty(n)
    B.debug_div(x.ctypes.data, y.ctypes.data, out.ctypes.data, ref.ctypes.data, n, device=False)
    assert np.array_equal(out.view(np.uint64), (x / y).view(np.uint64))


@pytest.mark.parametrize("change,msg", [
    (lambda w: setattr(w, "u0", np.where(np.arange(w.u0.size).reshape(w.u0.shape) == 7, -2, w.u0)), "u0["),
    (lambda w: setattr(w, "u0", np.where(np.arange(w.u0.size).reshape(w.u0.shape) == 1, (1 << 30) + 5, w.u0)),
     "2^30"),
    (lambda w: setattr(w, "phi0", np.where(np.arange(w.N) == 3, np.inf, w.phi0)), "phi0["),
    (lambda w: w.params.beta.__setitem__((0, 2), 1.5), "parameters"),
    (lambda w: w.params.gamma.__setitem__((0, 0), -0.1), "parameters"),
    (lambda w: setattr(w, "model", 2), "model"),
])
def test_create_rejects_bad_arguments(change, msg):
    # sim_create validates every argument before it touches a device
    w = W.sise_plain(N=30, T=5, n_events=0)
    change(w)
    with pytest.raises(B.SimError) as ei:
        B.Sim.from_workload(w)
    assert ei.value.status == B.SIM_E_INVALID_ARG and msg in str(ei.value)


def test_create_rejects_unknown_flags_and_reserved():
    import ctypes
    L = B.load_library()
    w = W.sise_plain(N=10, T=5, n_events=0)
    keep = [np.ascontiguousarray(x, np.float64) for x in (w.params.upsilon, w.params.gamma, w.params.alpha,
                                                          w.params.beta, w.params.epsilon)]
    sp = B.SimParams(*[x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in keep])
    u0 = np.ascontiguousarray(w.u0, np.int32); phi0 = np.ascontiguousarray(w.phi0, np.float64)
    for flags, reserved in ((1 << 7, 0), (0, 3)):
        cfg = B.SimConfig(W.SISE, w.N, 1, w.T, 0, flags, 1, 0, reserved)
        h = ctypes.c_void_p()
        st = L.sim_create(ctypes.byref(cfg), u0.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          phi0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(sp), ctypes.byref(h))
        assert st == B.SIM_E_INVALID_ARG and not h.value


def test_gradient_estimate_is_the_sample_covariance_of_f_and_the_score():
    """sim_gradient_estimate, from chunked moment sums, against numpy's sample
    covariance of the raw per-replicate values and the standard error of the mean
    of the centred product (f - mean f) * s."""
    rng = np.random.default_rng(11)
    R, F = 300, 3
    f = rng.random((R, F))
    s = rng.normal(size=(R, 8)) + 0.3 * f[:, :1]
    chunks = []
    for r0, r1 in ((0, 100), (100, 250), (250, 300)):
        m = np.zeros((F, B.N_MOMENTS))
        fc, sc = f[r0:r1], s[r0:r1]
        m[:, 0] = fc.sum(0); m[:, 1] = (fc ** 2).sum(0)
        for k in range(8):
            m[:, 2 + 4 * k] = sc[:, k].sum(); m[:, 3 + 4 * k] = (sc[:, k] ** 2).sum()
            m[:, 4 + 4 * k] = (fc * sc[:, k:k + 1]).sum(0)
            m[:, 5 + 4 * k] = ((fc * sc[:, k:k + 1]) ** 2).sum(0)
            m[:, 34 + k] = (fc * sc[:, k:k + 1] ** 2).sum(0)
        chunks.append(m)
    J = rng.random((8, 4))
    mean_f, grad, se = B.gradient_estimate(np.stack(chunks), R, J)
    np.testing.assert_allclose(mean_f, f.mean(0), rtol=1e-13)
    cov = np.array([[np.cov(f[:, i], s[:, k])[0, 1] for k in range(8)] for i in range(F)])
    np.testing.assert_allclose(grad, cov @ J, rtol=1e-10)
    # the standard error of the mean of the centred product (f - mean f) s
    fs = (f - f.mean(0))[:, :, None] * s[:, None, :]              # [R, F, 8]
    se8 = fs.std(0) / np.sqrt(R)
    np.testing.assert_allclose(se, np.sqrt((se8 ** 2) @ (J ** 2)), rtol=1e-10)
    with pytest.raises(B.SimError):
        B.gradient_estimate(np.stack(chunks), 1, J)


def test_batch_shape_accepts_the_listed_shapes_only():
    # host-side argument check only: no kernel runs until sim_run_batch
    for shape in B.BATCH_SHAPES:
        B.batch_shape(*shape)
    for bad in ((384, 1), (256, 3), (512, 1), (0, 1), (-1, 2)):
        with pytest.raises(B.SimError, match="batch shape"):
            B.batch_shape(*bad)
    B.batch_shape(*B.BATCH_SHAPES[0])


def test_autotune_candidates_time_every_batch_shape_for_the_persistent_mode_only():
    from paper_1502_02908_gb300 import autotune
    shapes = B.BATCH_SHAPES
    got = list(autotune._candidates((1 << 30, 200), (1 << 30, 100, 300), ("graph", "persistent"), shapes))
    # a group threshold at or above the warp threshold is skipped (300 >= 200), except the first
    pairs = {(t, g) for t, g, _, _ in got}
    assert pairs == {(1 << 30, 1 << 30), (1 << 30, 100), (1 << 30, 300), (200, 1 << 30), (200, 100)}
    for t, g, mode, shape in got:
        assert (shape is None) == (mode != "persistent")
    assert len(got) == len(pairs) * (1 + len(shapes))
    per = [s for t, g, m, s in got if (t, g) == (200, 100) and m == "persistent"]
    assert per == list(shapes)
