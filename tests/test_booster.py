"""Merge booster (Algorithms 6-7) pins: the paper's worked example counts and
the Divider's splits, plus exactness of boosted plans against the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S
from plan_interp import interpret

pytestmark = pytest.mark.usefixtures("built_lib")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def example_circuit(rng):
    """The 8-qubit, 40-gate circuit of the illustrative example, rebuilt from
    its printed counts: 6, 6, 7, 7 gates inside the 2-qubit groups, 7 and 4
    inside the 4-qubit halves, then 3 gates across the halves.  Only
    non-diagonal gates, so every gate updates its whole (sub-)state."""
    g = []
    def two(a, b):
        return C.Gate("cx", (a, b)) if rng.random() < 0.5 else C.Gate("u1q", (a,), matrix=C.haar_u2(rng))
    for (a, b), cnt in zip([(0, 1), (2, 3), (4, 5), (6, 7)], [6, 6, 7, 7]):
        g += [C.Gate("cx", (a, b))] + [two(a, b) for _ in range(cnt - 1)]
    for lo, cnt in [(0, 7), (4, 4)]:
        # two crossing gates first: every qubit of the half waits for level 1
        g += [C.Gate("cx", (lo, lo + 2)), C.Gate("cx", (lo + 1, lo + 3))]
        g += [C.Gate("ry", (lo + int(rng.integers(4)),), (0.3 + 0.1 * i,)) for i in range(cnt - 2)]
    g += [C.Gate("cx", (3, 4)), C.Gate("cx", (0, 7)), C.Gate("h", (4,))]
    return C.Circuit(8, g)


def test_booster_worked_example_1336():
    gold = _gold("booster_example.json")
    c = example_circuit(np.random.default_rng(0))
    assert len(c.gates) == gold["gates_total"]
    opt = S.default_options(flags=S.SIM_F_BOOST, booster_div=4)      # divSize = (8+4-1)/4 = 2
    p = S.plan_json(8, c.gates, S.SIM_C128, 0, opt)
    assert p["booster_queue"] == gold["divider_queue_n8_div2"]
    assert p["stats"]["state_updates"] == gold["boosted_state_updates"]
    plain = S.plan_json(8, c.gates, S.SIM_C128, 0, S.default_options(flags=0))
    assert plain["stats"]["state_updates"] == gold["naive_state_updates"]
    np.testing.assert_allclose(interpret(p), oracle.run(c), atol=1e-13)


def test_divider_top_level_is_two_halves():
    gold = _gold("divider_top_level.json")
    c = C.Circuit(32, [C.Gate("h", (q,)) for q in range(32)])
    p = S.plan_json(32, c.gates, S.SIM_C64, 0)
    q = p["booster_queue"]
    assert sum(q) == 32 and max(q) <= 12
    tens = [op for op in p["ops"] if op["op"] == "tensor"]
    assert [tens[-1]["n_lo"], tens[-1]["n_hi"]] == gold["top_level_merge"]
    assert tens[-1]["buf"] == 0


@pytest.mark.parametrize("n,div", [(5, 2), (9, 3), (13, 2), (17, 5), (28, 12), (30, 4)])
def test_divider_properties(n, div):
    c = C.Circuit(n, [C.Gate("h", (q,)) for q in range(n)])
    opt = S.default_options(flags=S.SIM_F_BOOST, booster_div=div)
    q = S.plan_json(n, c.gates, S.SIM_C64, 0, opt)["booster_queue"]
    ds = (n + div - 1) // div
    if n <= ds:
        assert q == []
    else:
        assert sum(q) == n and all(1 <= x <= ds for x in q)


@pytest.mark.parametrize("maker", [lambda: C.layered(12, 5, 3), lambda: C.qft(13, 4), lambda: C.diag_heavy(14, 120, 5),
                                   lambda: C.random_mixed(13, 150, 6, max_k=3), lambda: C.qaoa(14, 2, 7)])
@pytest.mark.parametrize("div", [2, 3, 5])
def test_boosted_plans_are_exact(maker, div):
    c = maker()
    opt = S.default_options(flags=S.SIM_F_ALL & ~S.SIM_F_TC, booster_div=div)
    p = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, opt)
    assert p["booster_queue"]
    np.testing.assert_allclose(interpret(p, basis=c.basis), oracle.run(c), atol=1e-12)


def test_no_booster_for_unknown_state():
    c = C.layered(12, 3, 1)
    p = S.plan_json(12, c.gates, S.SIM_C64, None, S.default_options(booster_div=3))
    assert p["booster_queue"] == []
    assert not any(op["op"] == "tensor" for op in p["ops"])
