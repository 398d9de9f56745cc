"""Pins for the mesh-size rules of Section 2.3.1 (brute-force enumeration)."""
import math

import numpy as np

from oracle import meshdims


def _brute_smooth(t):
    n = t
    while True:
        m = n
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1:
            return n
        n += 1


def test_strategies_against_enumeration():
    for t in range(1, 400):
        assert meshdims.next_smooth(t) == _brute_smooth(t)
        p2 = meshdims.next_pow2(t)
        assert p2 >= t and p2 & (p2 - 1) == 0 and (p2 // 2 < t or p2 == 1)


def test_paper_target_rule():
    box = np.diag([22.56, 30.0, 51.0])
    got = meshdims.target(box, 0.7, "paper")
    assert got == [math.ceil(2 * L / 0.7 + 1) for L in (22.56, 30.0, 51.0)]
    assert meshdims.mesh_dims(box, 0.7, "smooth") == [_brute_smooth(t) for t in got]
    assert meshdims.mesh_dims(box, 0.7, "ceil") == got


def test_spacing_rule_with_clamp():
    for L in (12.7, 18.0, 25.3, 32.1, 45.0):
        n = meshdims.mesh_dims(np.eye(3) * L, 0.8, "smooth", rule="spacing", clamp=(16, 48))
        assert all(16 <= x <= 48 and meshdims.is_smooth(x) for x in n)


def test_mesh_dims_follow_the_lattice_vectors():
    # the sizes depend on the lattice vectors (rows) only through their lengths: rotating the
    # cell leaves them unchanged, reordering the vectors reorders them
    box = np.array([[18.3, 0.0, 0.0], [6.0, 21.0, 0.0], [-4.0, 3.5, 26.0]])   # no target near an integer
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    for strategy in ("smooth", "pow2", "ceil"):
        for rule in ("paper", "spacing"):
            n0 = meshdims.mesh_dims(box, 0.9, strategy, rule)
            assert meshdims.mesh_dims(box @ Q.T, 0.9, strategy, rule) == n0
            assert meshdims.mesh_dims(box[[2, 0, 1]], 0.9, strategy, rule) == [n0[2], n0[0], n0[1]]
    # not vacuous: the columns of this box have other lengths than its rows
    assert meshdims.target(box.T, 0.9) != meshdims.target(box, 0.9)
