"""Host-side arithmetic of the benchmark, on CPU: the pair count behind the pair term's flop
figure (the roofline's numerator) against brute force over the periodic images."""
import itertools

import numpy as np
import pytest

pytest.importorskip("scipy")

import workloads as W


def _brute_ordered_pairs(pos, L, rcut):
    # ordered (i, j), i != j, and every image n with |r_j - r_i + n L| < rcut
    d0 = pos[None, :, :] - pos[:, None, :]
    count = 0
    for n in itertools.product((-1, 0, 1), repeat=3):
        d = d0 + np.asarray(n, np.float64) * L
        r2 = (d * d).sum(-1)
        count += int(((r2 < rcut * rcut) & (r2 > 0.0)).sum())
    return count


@pytest.mark.parametrize("n,L,rcut", [(128, (16.0, 16.0, 16.0), 7.0), (96, (14.0, 17.5, 15.2), 6.5),
                                      (200, (18.6, 18.6, 18.6), 9.0)])
def test_pair_hits_matches_brute_force(n, L, rcut):
    import bench
    fr = W.molten_nacl(n, seed=n)
    L = np.asarray(L)
    pos = fr.pos / fr.box[0, 0] * L              # spread the frame over the orthorhombic box
    pos[:5] += L * np.array([1.0, -2.0, 0.0])    # some positions outside the cell
    box = np.diag(L)
    got = bench.pair_hits(pos, box, rcut)
    assert got == _brute_ordered_pairs(np.mod(pos, L), L, rcut)
    assert got > 10 * n                           # not vacuous


def test_pair_hits_refuses_a_cutoff_beyond_half_the_box():
    import bench
    fr = W.molten_nacl(64, seed=1)               # L = 12.7 A
    with pytest.raises(ValueError):
        bench.pair_hits(fr.pos, fr.box, 6.5)
