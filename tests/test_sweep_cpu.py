"""Host bookkeeping of the parameter study (no GPU): the variant grid of
Sec. 4.2 and the error measure E = relerr - e_min with its rankings."""
import pytest

from paper_1805_06604_gb300 import sweep


def test_grid_is_the_papers():
    vs = sweep.variants()
    # 3 hp x 3 beta0 x 3 eta x 4 (gamma, gamma_bar) pairs, plus A-HALS.
    assert len(vs) == 1 + 3 * 3 * 3 * 4
    assert len({name for name, _, _ in vs}) == len(vs)
    assert vs[0][0] == sweep.AHALS and vs[0][2] == {"beta0": 0.0}
    for _, h, ov in vs[1:]:
        assert ov["hp"] == h and 1 < ov["gamma_bar"] < ov["gamma"] < ov["eta"]


def test_summarize_hand_computed():
    # Two data sets x two initialisations; E-A-HALS variants a, b (hp 1), c (hp 3).
    rel = {(0, 0): {"A-HALS": 0.50, "a": 0.40, "b": 0.45, "c": 0.41},
           (0, 1): {"A-HALS": 0.52, "a": 0.39, "b": 0.44, "c": 0.40},
           (1, 0): {"A-HALS": 0.31, "a": 0.30, "b": 0.32, "c": 0.29},
           (1, 1): {"A-HALS": 0.33, "a": 0.30, "b": 0.31, "c": 0.30}}
    hp_of = {"A-HALS": 0, "a": 1, "b": 1, "c": 3}
    s = sweep.summarize(rel, hp_of, exact_low_rank=False)
    assert s["e_min"] == {"0": 0.39, "1": 0.29}
    # E(a) over the runs: 0.01, 0.00, 0.01, 0.01
    assert s["per_variant"]["a"]["mean_E"] == pytest.approx(0.0075)
    assert s["per_variant"]["A-HALS"]["mean_E"] == pytest.approx((0.11 + 0.13 + 0.02 + 0.04) / 4)
    assert s["best"] == {"1": "a", "3": "c"} and s["worst"] == {"1": "b", "3": "c"}
    # ranking among A-HALS, a, b, c per run (ties share the better rank)
    assert s["ranking"]["a"] == [3, 1, 0, 0]
    assert s["ranking"]["c"] == [2, 2, 0, 0]
    assert s["ranking"]["A-HALS"] == [0, 0, 1, 3]
    assert all(sum(v) == 4 for v in s["ranking"].values())


def test_summarize_low_rank_uses_zero_e_min():
    rel = {(0, 0): {"A-HALS": 1e-3, "a": 1e-6}}
    s = sweep.summarize(rel, {"A-HALS": 0, "a": 1}, exact_low_rank=True)
    assert s["e_min"] == {"0": 0.0}
    assert s["per_variant"]["a"]["mean_E"] == pytest.approx(1e-6)
