"""Operation count of NN-sort (Sec. "Model Analysis"): T(n, e, sigma, t, theta).

n elements; per completed iteration i = 1..t the conflict rate sigma_i (|c_i| over the elements
entering iteration i) and the out-of-order rate e_i of o_i; theta operations per element and pass
through the model f. Sec. "Model Analysis" splits T into the sorting phase s(n) (model passes plus
the traditional sort of the last conflict array) and the polish phase p(n) (appends of ordered
elements, inserts of out-of-order ones at half the current output on average), then collects the
terms as C1 n^2 + C2 n log n + C3 n (Eq. operations, derived in the equation that follows it).

Readings where the printed equations are garbled: the alpha_i in C3 is sigma_i, and the inner sum
printed over n runs over j. The logarithm's base is not stated; base 2 is used (comparison sorts).
The model-pass term is taken as printed, theta * sum_{j<=i} sigma_j * n in iteration i
(feed="printed"); feed="entering" instead charges theta per element entering iteration i,
theta * prod_{j<i} sigma_j * n, which is what the text's description of the iterations implies.

This is the paper's analytic model, used beside the measured counts of an eps sweep; it plays no
part in a sort.
"""
from __future__ import annotations

import math
from typing import Sequence


def _prod(xs: Sequence[float]) -> float:
    p = 1.0
    for x in xs:
        p *= x
    return p


def coefficients(sigma: Sequence[float], e: Sequence[float], theta: float,
                 feed: str = "printed") -> tuple[float, float, float]:
    """(C1, C2, C3) of Eq. operations for t = len(sigma) completed iterations."""
    t = len(sigma)
    if len(e) != t or t < 1:
        raise ValueError("sigma and e need one entry per completed iteration (t >= 1)")
    if feed not in ("printed", "entering"):
        raise ValueError("feed is 'printed' or 'entering'")
    c1 = 0.5 * sum(e[i] * (1.0 - sigma[i]) * _prod(sigma[:i]) ** 2 for i in range(t))
    pt = _prod(sigma)
    c2 = pt
    c3 = 0.0
    for i in range(t):
        before = _prod(sigma[:i])          # share of n entering iteration i+1
        model = sum(sigma[:i + 1]) if feed == "printed" else before
        c3 += theta * model + (1.0 - e[i]) * (1.0 - sigma[i]) * before + _prod(sigma[:i + 1])
    c3 += 0.0 if pt <= 0.0 else pt * math.log2(pt)
    return c1, c2, c3


def operations(n: int, sigma: Sequence[float], e: Sequence[float], theta: float,
               feed: str = "printed") -> float:
    """T(n, e, sigma, t, theta): 1 for n = 1, else C1 n^2 + C2 n log2 n + C3 n."""
    if n <= 1:
        return 1.0
    c1, c2, c3 = coefficients(sigma, e, theta, feed)
    return c1 * n * n + c2 * n * math.log2(n) + c3 * n


def predicted_counts(n: int, sigma: Sequence[float], e: Sequence[float]) -> dict:
    """The element counts the model's terms are built from: elements entering each iteration,
    the final conflict array (sorted traditionally) and the out-of-order elements of each o_i."""
    t = len(sigma)
    entering = [_prod(sigma[:i]) * n for i in range(t)]
    return {"entering": entering,
            "leftover": _prod(sigma) * n,
            "out_of_order": [e[i] * (1.0 - sigma[i]) * entering[i] for i in range(t)]}


def quicksort_operations(n: int) -> float:
    """The n log2 n baseline the paper compares T against."""
    return n * math.log2(n) if n > 1 else 1.0
