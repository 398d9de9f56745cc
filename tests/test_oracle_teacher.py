"""Pins of the polarisable teacher O3 (oracle/teacher.py): the self-consistency residual, the
stationarity of the polarisation energy in the dipoles, the Hellmann-Feynman forces against
central differences of the energy with the dipoles re-solved at each geometry, the a -> 0
limit (plain fixed-charge PME), and an isolated polarisable ion pair against its closed form."""
import numpy as np
import pytest

import workloads as W
from oracle import pme as O2
from oracle import teacher as T

KW = dict(mesh=(12, 12, 12), order=4, alpha=0.4, rcut=4.5)


@pytest.fixture(scope="module")
def small():
    return W.molten_nacl(32, seed=13)


def test_self_consistency_and_stationarity(small):
    fr = small
    q, a = T.species_arrays(fr.species)
    o = O2.PMEOracle(fr.box, KW["mesh"], KW["order"], KW["alpha"], KW["rcut"])
    mu, out, iters = T.solve_dipoles(o, fr.pos, q, a)
    assert iters > 3
    assert np.abs(a[:, None] * out["field"] - mu).max() < 1e-10
    assert np.abs(mu).max() > 1e-2                      # the dipoles are not negligible

    def U(m):
        return o.evaluate(fr.pos, q, m, field_grad=False)["energy"] + T.polarisation_energy(m, a)

    d = np.random.default_rng(1).normal(size=mu.shape)
    u0 = U(mu)
    g1 = U(mu + 1e-3 * d) - u0
    g2 = U(mu + 2e-3 * d) - u0
    # quadratic in the step: no linear term at the self-consistent dipoles
    assert g1 > 0 and abs(g2 / g1 - 4.0) < 1e-4


def test_hellmann_feynman_forces(small):
    fr = small
    lab = T.label(fr, **KW)

    def U(pos):
        g = W.Frame(pos=pos, q=fr.q, mu=fr.mu, box=fr.box, species=fr.species)
        return T.label(g, mu0=lab["mu"], **KW)["energy"]

    h = 1e-5
    for i, c in [(0, 0), (7, 2), (20, 1)]:
        d = np.zeros_like(fr.pos)
        d[i, c] = h
        fd = (U(fr.pos + d) - U(fr.pos - d)) / (2 * h)
        assert abs(fd + lab["force"][i, c]) < 1e-6 * max(1.0, abs(fd))


def test_zero_polarisability_is_fixed_charge_pme(small):
    fr = small
    lab = T.label(fr, polarisability=(0.0, 0.0), **KW)
    q = np.where(fr.species == 0, 1.0, -1.0)
    ref = O2.PMEOracle(fr.box, KW["mesh"], KW["order"], KW["alpha"], KW["rcut"]).evaluate(
        fr.pos, q, np.zeros_like(fr.pos), field_grad=False)
    assert abs(lab["energy"] - ref["energy"]) < 1e-12 * abs(ref["energy"])
    assert np.abs(lab["force"] - ref["force"]).max() < 1e-12


def test_isolated_pair_closed_form():
    # Na+ and Cl- 3 A apart along x in a 60 A box: in vacuum the induced dipoles along the
    # axis solve mu1 = a1 (q2/R^2 + 2 mu2/R^3) and mu2 = a2 (q1/R^2 + 2 mu1/R^3) in the
    # coordinate along the unit vector from ion 2 to ion 1 (for ion 2 the field direction is
    # reversed, hence the sign of q1); the periodic images change the field by ~1e-3 relative
    R, L = 3.0, 60.0
    pos = np.array([[30.0, 30, 30], [30.0 - R, 30, 30]])   # ion 1 (Na) at +x of ion 2 (Cl)
    fr = W.Frame(pos=pos, q=np.zeros(2), mu=np.zeros((2, 3)), box=np.eye(3) * L,
                 species=np.array([0, 1]))
    lab = T.label(fr, mesh=(64, 64, 64), order=6, alpha=0.25, rcut=12.0)
    a1, a2 = T.POLARISABILITY
    q1, q2 = T.CHARGE
    # unknowns along +x: mu1 = a1 (q2/R^2 + 2 mu2/R^3); field at 2 along +x = -q1/R^2 + 2 mu1/R^3
    M = np.array([[1.0, -2 * a1 / R ** 3], [-2 * a2 / R ** 3, 1.0]])
    rhs = np.array([a1 * q2 / R ** 2, -a2 * q1 / R ** 2])
    mu1, mu2 = np.linalg.solve(M, rhs)
    got = lab["mu"][:, 0]
    assert abs(got[0] - mu1) < 1e-2 * abs(mu1) and abs(got[1] - mu2) < 1e-2 * abs(mu2)
    assert np.abs(lab["mu"][:, 1:]).max() < 1e-6
