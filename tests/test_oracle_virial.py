"""Virial of the plain PME (O2): W_ab = -dE/d(eps_ab) for the homogeneous strain of positions
and lattice vectors r -> (I + eps) r with the dipoles held fixed.

Pins: the definition (central differences of the energy under strain) against the term-by-term
evaluation, in a cubic and a triclinic cell, with and without dipoles, and with a net charge
(the background term); and the scaling
identity of the exact Ewald sum (O1): under r -> (1 + l) r the charge-charge, charge-dipole
and dipole-dipole energies scale as 1/L, 1/L^2 and 1/L^3, so
tr W = E_qq + 2 E_qmu + 3 E_mumu for a neutral frame, which O2 meets once its mesh and
real-space cutoff are converged.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ewald as O1
from oracle import pme as O2


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("dipoles", [False, True])
def test_virial_definition_matches_terms_cubic(dipoles):
    fr = W.molten_nacl(192, seed=11)
    mu = fr.mu * 3 if dipoles else None
    o = O2.PMEOracle(fr.box, (24, 24, 24), 6, 0.35, 8.0)
    Wd = o.virial(fr.pos, fr.q, mu)
    Wt = o.virial_terms(fr.pos, fr.q, mu)
    assert _rel(Wd, Wt) < 1e-8
    if dipoles:
        # fixed dipoles make the energy depend on the cell's orientation: W is not symmetric
        assert np.abs(Wd - Wd.T).max() > 1e-3 * np.abs(Wd).max()
    else:
        assert np.abs(Wd - Wd.T).max() < 1e-8 * np.abs(Wd).max()


def test_virial_definition_matches_terms_charged():
    # a frame with net charge Q: the neutralising background -pi Q^2 / (2 V alpha^2) scales as
    # 1/V and adds E_bg I to the virial (zero on the neutral frames above)
    fr = W.molten_nacl(96, seed=17)
    q = fr.q.copy()
    q[:3] += 0.4
    o = O2.PMEOracle(fr.box, (20, 20, 20), 6, 0.35, 7.0)
    Wd = o.virial(fr.pos, q, fr.mu)
    assert _rel(Wd, o.virial_terms(fr.pos, q, fr.mu)) < 1e-8
    e_bg = np.pi * q.sum() ** 2 / (2 * o.V * 0.35 ** 2)
    assert e_bg > 1e-3 * np.abs(Wd).max()     # the check is not vacuous


def test_virial_definition_matches_terms_triclinic():
    box = np.array([[18.0, 0.0, 0.0], [3.0, 17.0, 0.0], [-2.0, 1.5, 19.0]])
    rng = np.random.default_rng(13)
    fr = W.molten_nacl(160, seed=13)
    pos = rng.uniform(size=(160, 3)) @ box
    o = O2.PMEOracle(box, (24, 24, 25), 6, 0.35, 7.0)
    assert _rel(o.virial(pos, fr.q, fr.mu * 2), o.virial_terms(pos, fr.q, fr.mu * 2)) < 1e-8


def test_virial_trace_is_the_ewald_scaling_identity():
    fr = W.molten_nacl(128, seed=8)
    q, mu = fr.q, fr.mu * 4
    E = O1.ewald(fr.pos, q, mu, fr.box, 0.35)["energy"]
    Eqq = O1.ewald(fr.pos, q, 0 * mu, fr.box, 0.35)["energy"]
    Emm = O1.ewald(fr.pos, 0 * q, mu, fr.box, 0.35)["energy"]
    target = Eqq + 2 * (E - Eqq - Emm) + 3 * Emm
    o = O2.PMEOracle(fr.box, (48, 48, 48), 7, 0.50, 9.5)     # mesh and cutoff converged
    assert abs(np.trace(o.virial_terms(fr.pos, q, mu)) - target) < 1e-6 * abs(target)
    # a truncated real-space sum misses it by the truncation error
    o_short = O2.PMEOracle(fr.box, (48, 48, 48), 7, 0.35, 8.0)
    assert abs(np.trace(o_short.virial_terms(fr.pos, q, mu)) - target) > 1e-4 * abs(target)
