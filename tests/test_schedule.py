"""Host-side task schedule of batched launches (corr_plan_schedule): the
longest-processing-time-first rule, checked against its definition, its
classical bound (makespan <= (4/3 - 1/(3m)) x optimum, Graham 1969) and the
brute-force optimum on small cases.  No GPU is needed."""
import itertools

import numpy as np
import pytest

from paper_1904_07778_gb300 import build

build.build()
from paper_1904_07778_gb300 import xengine as xe  # noqa: E402


def _loads(cost, order, first):
    return [sum(cost[order[j]] for j in range(first[c], first[c + 1])) for c in range(len(first) - 1)]


def _optimum(cost, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(cost)):
        loads = [0.0] * m
        for c, a in zip(cost, assign):
            loads[a] += c
        best = min(best, max(loads))
    return best


@pytest.mark.parametrize("seed", range(12))
def test_lpt_bound_and_structure(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 9)), int(rng.integers(1, 4))
    cost = rng.integers(1, 20, size=n).astype(float)
    order, first = xe.corr_plan_schedule(cost, m)
    assert first[0] == 0 and first[-1] == n and np.all(np.diff(first) >= 0)
    assert sorted(order.tolist()) == list(range(n))          # every task exactly once
    for c in range(m):                                       # each list longest first
        cs = [cost[order[j]] for j in range(first[c], first[c + 1])]
        assert cs == sorted(cs, reverse=True)
    opt = _optimum(cost, m)
    assert max(_loads(cost, order, first)) <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9


def test_lpt_rule_step_by_step():
    """Each task, taken in decreasing cost, goes to the least loaded CTA."""
    cost = [7, 7, 6, 6, 5, 4, 4, 2]
    order, first = xe.corr_plan_schedule(cost, 3)
    cta_of = {}
    for c in range(3):
        for j in range(first[c], first[c + 1]):
            cta_of[int(order[j])] = c
    loads = [0.0] * 3
    for t in sorted(range(len(cost)), key=lambda t: -cost[t]):   # stable: ties by index
        c = min(range(3), key=lambda k: (loads[k], k))
        assert cta_of[t] == c
        loads[c] += cost[t]


def test_equal_tasks_spread_evenly():
    order, first = xe.corr_plan_schedule([1.0] * 300, 152)
    counts = np.diff(first)
    assert counts.max() - counts.min() <= 1


def test_bad_arguments():
    with pytest.raises(xe.CorrError):
        xe.corr_plan_schedule([1.0, -2.0], 2)
    with pytest.raises(xe.CorrError):
        xe.corr_plan_schedule([1.0], 0)
