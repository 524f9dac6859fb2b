"""Oversampling parameters of the single-pass method (Sections 6.3 and 6.6).

For a sketch budget T = 2k + l_1 + l_2 (k the target rank, the paper's p; a
real matrix with T >= 2k + 6), the baseline single pass (Alg. 7 with
l_c = l_1) takes (l_1, l_2) from one of three schemes meant for a flat, a
moderately decaying or a rapidly decaying spectrum.  With l_1 ~= l_2 the
truncation parameter l_c of Alg. 7 is chosen instead, as a fixed ratio of
l_1 or by the minimum-variance rule (lr_single_pass with l_c = MINVAR).
These are host-side parameter rules; no array is touched here.
"""
from __future__ import annotations

import math

__all__ = ["flat", "decay", "rapid", "equal_split", "fixed_ratio", "MINVAR"]

#: l_c value asking lr_single_pass to pick l_c by the minimum-variance rule.
MINVAR = -2


def _check(T: int, k: int) -> None:
    if k < 1 or T < 2 * k + 6:
        raise ValueError("need k >= 1 and a budget T >= 2k + 6")


def flat(T: int, k: int) -> tuple[int, int]:
    """(l_1, l_2) for a relatively flat spectrum."""
    _check(T, k)
    r = (T - 1) * (math.sqrt(k * (T - k - 2) * (1.0 - 2.0 / (T - 1))) - (k - 1)) / (T - 2 * k - 1)
    l1 = max(2, math.floor(r) - k)
    return l1, T - 2 * k - l1


def decay(T: int, k: int) -> tuple[int, int]:
    """(l_1, l_2) for a moderately decaying spectrum (the all-round choice)."""
    _check(T, k)
    l1 = max(2, (T - 1) // 3 - k)
    return l1, T - 2 * k - l1


def rapid(T: int, k: int) -> tuple[int, int]:
    """(l_1, l_2) for a rapidly decaying spectrum."""
    _check(T, k)
    l1 = (T - 2) // 2 - k
    return l1, T - 2 * k - l1


def equal_split(T: int, k: int) -> tuple[int, int]:
    """l_1 ~= l_2: l_1 = floor(T / 2) - k, l_2 = T - 2k - l_1 (used with l_c)."""
    _check(T, k)
    l1 = T // 2 - k
    return l1, T - 2 * k - l1


def fixed_ratio(l1: int, alpha: float) -> int:
    """l_c = floor(alpha l_1), 0 <= alpha <= 1."""
    if not 0.0 <= alpha <= 1.0 or l1 < 0:
        raise ValueError("need 0 <= alpha <= 1 and l_1 >= 0")
    return int(math.floor(alpha * l1))
