"""Pins for O1, the explicit Ewald oracle."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import ewald, pme


def _golden(root):
    vals = {}
    with open(os.path.join(root, "tests", "golden", "madelung_rocksalt.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_rocksalt_madelung(root):
    g = _golden(root)
    fr = W.rocksalt(int(g["ncell"]), g["a"])
    ref = -fr.n * g["M"] / (2 * g["r0"])
    r = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, 0.45)
    assert abs(r["energy"] - ref) / abs(ref) < 1e-9
    # zero forces and equal potentials magnitude on a perfect lattice
    assert np.abs(r["force"]).max() < 1e-10
    assert np.allclose(np.abs(r["phi"]), np.abs(r["phi"][0]), rtol=1e-10)


def _golden_file(root, name):
    vals = {}
    with open(os.path.join(root, "tests", "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


_FCC = [(0, 0, 0), (0.5, 0.5, 0), (0.5, 0, 0.5), (0, 0.5, 0.5)]
CRYSTALS = {
    # golden file, fractional basis of the cubic cell, charges, nearest-neighbour distance / a
    "cscl": ("madelung_cscl.txt", [(0, 0, 0), (0.5, 0.5, 0.5)], [1, -1], np.sqrt(3) / 2),
    "zincblende": ("madelung_zincblende.txt", _FCC + [(x + 0.25, y + 0.25, z + 0.25) for x, y, z in _FCC],
                   [1] * 4 + [-1] * 4, np.sqrt(3) / 4),
}


@pytest.mark.parametrize("name", list(CRYSTALS))
def test_other_crystal_madelung_constants(root, name):
    # two more structures with tabulated Madelung constants: body-centred (CsCl) and
    # tetrahedral (zinc blende) coordination; O1 is exact, O2 carries its mesh error
    fname, basis, charges, r0a = CRYSTALS[name]
    g = _golden_file(root, fname)
    fr = W.cubic_crystal(basis, charges, int(g["ncell"]), g["a"])
    ref = -fr.n * g["M"] / (2 * r0a * g["a"])
    r = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, 0.5)
    assert abs(r["energy"] - ref) / abs(ref) < 1e-8
    assert np.abs(r["force"]).max() < 1e-10
    o2 = pme.PMEOracle(fr.box, (48, 48, 48), 6, 0.7, 0.49 * fr.box[0, 0]).evaluate(
        fr.pos, fr.q, fr.mu, field_grad=False)
    assert abs(o2["energy"] - ref) / abs(ref) < 1e-5


def test_alpha_independence_charges_and_dipoles():
    fr = W.rocksalt(2, 5.64, jitter=0.15, mu_sigma=0.1, seed=5)
    Es = [ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, a)["energy"] for a in (0.25, 0.4, 0.6)]
    assert max(Es) - min(Es) < 1e-10 * abs(Es[0])
    rs = [ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, a) for a in (0.3, 0.55)]
    for key in ("force", "phi", "field", "field_grad"):
        assert np.allclose(rs[0][key], rs[1][key], atol=1e-10 * np.abs(rs[0][key]).max())


def test_surface_term_against_brute_force_images():
    fr = W.charged_dimer(sep=6.0, L=20.0)
    r = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, 0.35, surface_eps=1.0)
    errs = [abs(ewald.coulomb_images(fr.pos, fr.q, fr.mu, fr.box, n) - r["energy"])
            for n in (8, 16, 24)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-8 * abs(r["energy"]) + 3e-9


def test_translation_invariance_and_zero_net_force():
    fr = W.rocksalt(2, 5.64, jitter=0.2, mu_sigma=0.1, seed=7)
    r0 = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, 0.4)
    r1 = ewald.ewald(fr.pos + np.array([0.37, -1.9, 2.3]), fr.q, fr.mu, fr.box, 0.4)
    assert abs(r0["energy"] - r1["energy"]) < 1e-11 * abs(r0["energy"])
    assert np.allclose(r0["force"], r1["force"], atol=1e-11)
    assert np.abs(r0["force"].sum(0)).max() < 1e-11


def test_background_term_for_charged_system():
    fr = W.rocksalt(2, 5.64, jitter=0.2, seed=8)
    q = fr.q.copy()
    q[0] += 0.3  # net charge 0.3
    Es = [ewald.ewald(fr.pos, q, fr.mu, fr.box, a)["energy"] for a in (0.3, 0.5)]
    # with the neutralising background the total stays alpha-independent
    assert abs(Es[0] - Es[1]) < 1e-10 * abs(Es[0])


def _fd_check(fn, x, grad, idx, h):
    for i in idx:
        xp = x.copy()
        xm = x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        fd = (fn(xp) - fn(xm)) / (2 * h)
        assert abs(fd - grad.flat[i]) < 1e-7 * max(1.0, abs(grad.flat[i])), (i, fd, grad.flat[i])


def test_derivatives_central_differences():
    fr = W.rocksalt(2, 5.64, jitter=0.2, mu_sigma=0.1, seed=9)
    a = 0.4
    r = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, a)
    idx = [0, 5, 17, 40]
    _fd_check(lambda x: ewald.ewald(x, fr.q, fr.mu, fr.box, a)["energy"], fr.pos, -r["force"], idx, 1e-5)
    _fd_check(lambda x: ewald.ewald(fr.pos, x, fr.mu, fr.box, a)["energy"], fr.q, r["phi"], [0, 3, 9], 1e-5)
    _fd_check(lambda x: ewald.ewald(fr.pos, fr.q, x, fr.box, a)["energy"], fr.mu, -r["field"], idx, 1e-5)


def test_field_gradient_is_derivative_of_spatial_field():
    # field_grad is the gradient of the field of all other sources at the ion: it is
    # symmetric, traceless (Laplace: no other source sits at r_i) and gives
    # F = q E + (mu . grad) E
    fr = W.rocksalt(2, 5.64, jitter=0.2, mu_sigma=0.1, seed=11)
    a = 0.4
    r = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, a)
    F = fr.q[:, None] * r["field"] + np.einsum("iab,ib->ia", r["field_grad"], fr.mu)
    assert np.allclose(F, r["force"], atol=1e-12)
    assert np.allclose(r["field_grad"], np.transpose(r["field_grad"], (0, 2, 1)), atol=1e-12)
    tr = np.trace(r["field_grad"], axis1=1, axis2=2)
    assert np.abs(tr).max() < 1e-10 * np.abs(r["field_grad"]).max()


def test_dipole_is_limit_of_charge_pair():
    # mu = q d: replace each dipole by +-q at r +- d/2; removing the bare intra-pair
    # Coulomb energy -q^2/d, the Ewald energy converges to the dipole energy as O(d^2)
    fr = W.rocksalt(1, 5.64, jitter=0.2, mu_sigma=0.1, seed=13)
    a = 0.45
    Ed = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, a)["energy"]
    errs = []
    mnorm = np.linalg.norm(fr.mu, axis=1)
    u = fr.mu / mnorm[:, None]
    for sep in (0.02, 0.01):
        qd = mnorm / sep
        pos = np.concatenate([fr.pos, fr.pos + 0.5 * sep * u, fr.pos - 0.5 * sep * u])
        q = np.concatenate([fr.q, qd, -qd])
        Ec = ewald.ewald(pos, q, np.zeros_like(pos), fr.box, a)["energy"]
        Ec += np.sum(qd * qd / sep)
        errs.append(abs(Ec - Ed))
    assert errs[1] < errs[0] / 3.0
    assert errs[1] < 1e-6 * abs(Ed)
