"""CPU tests of the general model's host logic in the C-ABI library (no GPU):
model validation and the dependency graph of Sec. 3.3 (which rates a firing
can change), checked against graphs written out by hand."""
import numpy as np
import pytest

from paper_1502_02908_gb300 import binding as B
from paper_1502_02908_gb300 import workloads as W


def _bits(*sets):
    return [sum(1 << j for j in s) for s in sets]


def test_dependency_graph_sir():
    # inf = S+I -> 2I reads S, I (and N, unchanged by both); rec = I -> R reads I
    assert B.gen_dependency(W.sir_general(N=2, n_events=0).model).tolist() == _bits({0, 1}, {0, 1})


def test_dependency_graph_seirs():
    # 0 S->E (y0 S), 1 S->E (S I / N), 2 E->I, 3 I->R, 4 R->S, 5 S->E (y1 S)
    m = W.seirs_env(N=2, n_events=0).model
    want = _bits({0, 1, 2, 5}, {0, 1, 2, 5}, {1, 2, 3}, {1, 3, 4}, {0, 1, 4, 5}, {0, 1, 2, 5})
    assert B.gen_dependency(m).tolist() == want


def test_dependency_graph_population_change():
    # a birth (S + 1) or an arrival in R changes N, so the frequency-dependent
    # infection rate (transition 2) depends on them; the constant rates depend on nothing
    m = W.general_model(("S", "I", "R"),
                        [dict(change={"S": 1}),
                         dict(change={"I": -1, "R": 1}, a="I"),
                         dict(change={"S": -1, "I": 1}, a="S", b="I", pop=("S", "I", "R")),
                         dict(change={"R": 1})])
    dep = B.gen_dependency(m).tolist()
    assert dep == _bits({2}, {1, 2}, {1, 2}, {2})


def test_dependency_graph_erlang_chain():
    m = W.erlang_sis(N=2, n_events=0).model
    dep = B.gen_dependency(m).tolist()
    assert dep[0] == dep[1] == _bits({0, 1, 2})[0]
    assert dep[2] == _bits({1, 2, 3})[0]             # I1 -> I2 also changes S I1 / N
    for k in range(3, 10):                           # I_(k-1) -> I_k, and I8 -> R
        assert dep[k] == _bits({k, k + 1})[0]
    assert dep[10] == _bits({0, 1, 10})[0]


def _sir_model(**over):
    m = W.sir_general(N=2, n_events=0).model
    for k, v in over.items():
        setattr(m, k, v)
    return m


@pytest.mark.parametrize("change,msg", [
    (dict(stoich=np.array([[-1, 0], [1, -1], [0, -1]], np.int32)), "not a factor"),
    (dict(stoich=np.array([[-2, 0], [1, -1], [0, 1]], np.int32)), "outside"),
    (dict(factor_a=np.array([3, 1], np.int32)), "factor_a"),
    (dict(cont=np.array([0, -1], np.int32)), "cont"),
    (dict(pop_mask=np.array([8, 0], np.uint32)), "pop_mask"),
    (dict(select=np.array([7, 0], np.uint32)), "select"),
    (dict(shift=np.array([[3, 0, 0]], np.int32)), "shift"),
    (dict(y_source=5), "y_source"),
])
def test_model_check_rejects(change, msg):
    with pytest.raises(B.SimError) as e:
        B.gen_dependency(_sir_model(**change))
    assert e.value.status == B.SIM_E_INVALID_ARG and msg in str(e.value)


def test_model_limits():
    big = W.general_model(tuple(f"C{i}" for i in range(17)), [])
    with pytest.raises(B.SimError):
        B.gen_dependency(big)
    ok = W.general_model(tuple(f"C{i}" for i in range(16)),
                         [dict(change={f"C{i}": -1, f"C{(i + 1) % 16}": 1}, a=f"C{i}") for i in range(32) if i < 16] * 2)
    assert B.gen_dependency(ok).size == 32
    too_many = W.general_model(("A", "B"), [dict(change={"A": -1, "B": 1}, a="A")] * 33)
    with pytest.raises(B.SimError):
        B.gen_dependency(too_many)


def _create(w, **over):
    """gen_create with one argument replaced; its validation runs before any device call."""
    kw = dict(u0=w.u0, y0=w.y0, rates=w.rates, var_params=w.var_params)
    kw.update(over)
    return B.GenSim(w.model, kw["u0"], kw["y0"], kw["rates"], kw["var_params"], w.T, seed=w.seed)


@pytest.mark.parametrize("field,value,msg", [
    ("u0", lambda w: np.where(np.arange(w.u0.size).reshape(w.u0.shape) == 5, -1, w.u0), "u0["),
    ("u0", lambda w: np.where(np.arange(w.u0.size).reshape(w.u0.shape) == 0, (1 << 30) + 1, w.u0), "2^30"),
    ("y0", lambda w: np.where(np.arange(w.y0.size).reshape(w.y0.shape) == 3, -0.5, w.y0), "y0["),
    ("rates", lambda w: w.rates * np.array([1.0, 1.0, -1.0, 1.0, 1.0, 1.0]), "rate["),
    ("var_params", lambda w: np.concatenate([w.var_params[..., :1], np.full(w.var_params[..., 1:5].shape, 1.5),
                                             w.var_params[..., 5:]], -1), "beta"),
    ("var_params", lambda w: np.concatenate([np.full(w.var_params[..., :1].shape, np.nan), w.var_params[..., 1:]], -1),
     "alpha"),
])
def test_create_rejects_bad_arguments(field, value, msg):
    w = W.seirs_env(N=40, T=5, n_events=0, R=1)
    with pytest.raises(B.SimError) as e:
        _create(w, **{field: value(w)})
    assert e.value.status == B.SIM_E_INVALID_ARG and msg in str(e.value)
