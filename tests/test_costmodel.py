"""The cost model of Sec. "Model Analysis" (host arithmetic, no GPU): the collected polynomial of
Eq. operations equals the sum of the sorting and polish phases as the section derives them term by
term; closed forms of the degenerate cases; and the element counts its terms are built from equal
the oracle's measured counts when sigma_i and e_i are taken from the same run."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
import workloads as W

cm = pytest.importorskip("paper_1907_08817_gb300.costmodel")


def _phases(n, sigma, e, theta, feed):
    """s(n) + p(n), each term as the section states it in words."""
    t = len(sigma)
    P = lambda k: float(np.prod(sigma[:k])) if k else 1.0  # noqa: E731  share entering iteration k+1
    left = P(t) * n
    s = (left * math.log2(left) if left > 0 else 0.0)  # traditional sort of the last conflict array
    for i in range(t):
        s += theta * (sum(sigma[:i + 1]) if feed == "printed" else P(i)) * n
    p = 0.0
    for i in range(t):
        ooo = e[i] * (1 - sigma[i]) * P(i) * n          # out-of-order elements of o_i
        p += ooo * (P(i) * n / 2)                        # each inserted at half the output
        p += (1 - e[i]) * (1 - sigma[i]) * P(i) * n      # ordered elements of o_i appended
        p += P(i + 1) * n                                # elements of w appended
    return s + p


@pytest.mark.parametrize("feed", ["printed", "entering"])
def test_collected_polynomial_equals_phase_sum(feed):
    rs = np.random.RandomState(3)
    for _ in range(200):
        t = rs.randint(1, 6)
        sigma = list(rs.uniform(0.01, 0.99, t))
        e = list(rs.uniform(0, 1, t))
        theta = float(rs.choice([1, 8, 32, 8448]))
        n = int(rs.choice([2, 17, 1000, 10 ** 6, 3 * 10 ** 8]))
        got = cm.operations(n, sigma, e, theta, feed)
        want = _phases(n, sigma, e, theta, feed)
        assert abs(got - want) <= 1e-9 * abs(want), (got, want)


def test_degenerate_cases():
    n, theta = 10 ** 6, 32.0
    assert cm.operations(1, [0.5], [0.5], theta) == 1.0
    # a perfect model: no conflicts, nothing out of order -> one pass and one append per element
    assert cm.operations(n, [0.0], [0.0], theta, "entering") == pytest.approx(theta * n + n)
    assert cm.operations(n, [0.0], [0.0], theta, "printed") == pytest.approx(n)
    # everything conflicts every iteration -> the conflict array is the input: n log n + passes
    t = 3
    c1, c2, c3 = cm.coefficients([1.0] * t, [0.3] * t, theta, "entering")
    assert c1 == 0.0 and c2 == 1.0 and c3 == pytest.approx(t * theta + t)
    # no conflicts but every element out of order: inserts dominate, n^2 / 2
    c1, c2, _ = cm.coefficients([0.0], [1.0], theta)
    assert c1 == 0.5 and c2 == 0.0
    assert cm.quicksort_operations(1024) == 1024 * 10


def test_terms_count_what_the_oracle_counts():
    n = 20_000
    keys = W.lognormal_dup_f32(n, 2, sigma=2.0)
    om, _, _ = orc.train(keys, 1, 8, 0, orc.ORDBITS, sample_n=500, steps=40, seed=1)
    L, _, _ = orc.nm_split(n)
    slots, _ = orc.predict_slots(keys, om)
    _, _, st, _ = orc.nnsort(keys, slots, L, 4, 0)
    assert st["t"] >= 2
    t = st["t"]
    w = st["w_size"]
    sigma = [w[i + 1] / w[i] for i in range(t)]
    e = [st["out_of_order"][i] / st["placed"][i] if st["placed"][i] else 0.0 for i in range(t)]
    pc = cm.predicted_counts(n, sigma, e)
    np.testing.assert_allclose(pc["entering"], w[:t], rtol=1e-12)
    assert pc["leftover"] == pytest.approx(w[t], rel=1e-12)
    np.testing.assert_allclose(pc["out_of_order"], st["out_of_order"], rtol=1e-9, atol=1e-9)
