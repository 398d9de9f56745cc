"""Mesh-size rules of Section 2.3.1 (Eq. mesh_target and the three strategies).

Readings:
* ``paper`` target: N = ceil(2*|a_alpha|/Delta + 1), exactly as Eq. mesh_target prints it
  (the factor 2 makes the realised spacing about Delta/2).
* ``spacing`` target: N = ceil(|a_alpha|/Delta), the plain spacing rule used for the
  uneven batched workload.
Strategies map a target to an FFT size: ``pow2`` (next power of two), ``smooth`` (the
smallest integer >= target with prime factors in {2, 3, 5}; the paper's default) and
``ceil`` (the target itself).

Parity: pinned by brute-force enumeration in tests/test_oracle_meshdims.py.
"""
from __future__ import annotations

import math

import numpy as np


def is_smooth(n: int) -> bool:
    for f in (2, 3, 5):
        while n % f == 0 and n > 1:
            n //= f
    return n == 1


def next_smooth(n: int) -> int:
    n = max(1, int(n))
    while not is_smooth(n):
        n += 1
    return n


def next_pow2(n: int) -> int:
    n = max(1, int(n))
    return 1 << (n - 1).bit_length()


def target(box: np.ndarray, spacing: float, rule: str = "paper") -> list[int]:
    lens = np.linalg.norm(np.asarray(box, dtype=np.float64), axis=1)
    if rule == "paper":
        return [int(math.ceil(2.0 * L / spacing + 1.0)) for L in lens]
    if rule == "spacing":
        return [int(math.ceil(L / spacing)) for L in lens]
    raise ValueError(rule)


def mesh_dims(box, spacing: float, strategy: str = "smooth", rule: str = "paper",
              clamp: tuple[int, int] | None = None) -> list[int]:
    out = []
    for t in target(box, spacing, rule):
        if strategy == "pow2":
            n = next_pow2(t)
        elif strategy == "smooth":
            n = next_smooth(t)
        elif strategy == "ceil":
            n = t
        else:
            raise ValueError(strategy)
        if clamp is not None:
            n = min(max(n, clamp[0]), clamp[1])
        out.append(int(n))
    return out
