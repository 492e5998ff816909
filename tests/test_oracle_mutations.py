"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks that
at least one pin fails for each, so the pins constrain every part of the
arithmetic: rates, the time step, the stopping rule, transition selection, the
phi recursion and its season index, event routing and sampling, and the score
terms."""
import pathlib

import pytest

import oracle
from tests import test_oracle_model as M
from tests import test_oracle_score as S

SRC = (pathlib.Path(oracle.__file__).parent / "oracle.c").read_text()

MUTATIONS = [
    ("selection threshold drops P_{j-1}",
     "double thr = (cls == 0) ? ainf[0] : P[cls - 1] + ainf[cls];",
     "double thr = ainf[cls];", [M.test_frozen_phi_two_state_law_sise3_per_class]),
    ("tau multiplies instead of divides",
     "double tau = E / a0;", "double tau = E * a0;", [M.test_pure_death_binomial]),
    ("recovery rate uses S",
     "arec[cls] = c->gamma[cls] * (double)X(2 * cls + 1, v);",
     "arec[cls] = c->gamma[cls] * (double)X(2 * cls, v);", [M.test_pure_death_binomial]),
    ("stopping rule ignores elapsed time",
     "if (tn >= 1.0) break;", "if (tau >= 1.0) break;", [M.test_frozen_phi_two_state_law_sise]),
    ("phi update drops epsilon",
     "return ((phi * omb) + q) + c->epsilon;", "return ((phi * omb) + q);",
     [M.test_phi_closed_form_constant_beta]),
    ("season index off by one day",
     "double omb = 1.0 - c->beta[season(day)];", "double omb = 1.0 - c->beta[season(day + 1)];",
     [M.test_phi_closed_form_seasonal_beta_and_empty_node]),
    ("aging keeps the class",
     "if (kind == EV_INTERNAL) X(got + 2, node) += 1;", "if (kind == EV_INTERNAL) X(got, node) += 1;",
     [M.test_events_bookkeeping_without_clamping]),
    ("sampling slot off by one",
     "if (slot < have) { X(comp[q], v) -= 1; return comp[q]; }",
     "if (slot <= have) { X(comp[q], v) -= 1; return comp[q]; }",
     [M.test_exit_sample_is_hypergeometric]),
    ("upsilon score drops phi",
     "- phi[v] * T->int_s[j];", "- T->int_s[j];", [S.test_score_identity_independent_animals]),
    ("beta tangent sign",
     "dphi_b[v] = dphi_b[v] * omb - phi[v];", "dphi_b[v] = dphi_b[v] * omb + phi[v];",
     [S.test_score_identity_independent_animals]),
    ("end-of-day integral uses the whole day",
     "double dt = 1.0 - tlast[j];", "double dt = 1.0;", [S.test_score_identity_independent_animals]),
    ("alpha tangent drops I/N",
     "dphi_a[v] = dphi_a[v] * omb + q_tmp[v];", "dphi_a[v] = dphi_a[v] * omb;",
     [S.test_score_identity_path_dependent_phi]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, pins, tmp_path, monkeypatch):
    assert SRC.count(old) == 1, name
    L = oracle.compile_variant(SRC.replace(old, new), tmp_path / "libmut.so")
    monkeypatch.setattr(oracle, "_LIB", L)
    for pin in pins:
        with pytest.raises(AssertionError):
            pin()
