"""Each test plants one plausible mistake in the oracle (on the CPU, through monkeypatch) and
checks that at least one of the oracle's pins then fails. This shows the pins are sensitive
to dropped terms, wrong signs, transposed operands and wrong factors."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import bspline, ewald
from oracle import pme as O2

import test_oracle_ewald as TE
import test_oracle_pme as TP


@pytest.fixture
def small():
    return W.rocksalt(1, 5.64, jitter=0.25, mu_sigma=0.1, seed=21)


@pytest.fixture
def salt():
    return W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000)


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_dipole_sign_in_mesh_is_caught(monkeypatch, small):
    orig = O2.PMEOracle.mesh_density
    monkeypatch.setattr(O2.PMEOracle, "mesh_density",
                        lambda self, pos, q, mu: orig(self, pos, q, -mu))
    _fails(TP.test_dipole_is_limit_of_charge_pair_on_mesh, small)


def test_dropped_dipole_density_is_caught(monkeypatch, small):
    orig = O2.PMEOracle.mesh_density
    monkeypatch.setattr(O2.PMEOracle, "mesh_density",
                        lambda self, pos, q, mu: orig(self, pos, q, mu * 0))
    _fails(TP.test_dipole_is_limit_of_charge_pair_on_mesh, small)


def test_transposed_inverse_cell_is_caught(monkeypatch, small):
    # dipole projected on the rows of C^{-1} instead of its columns: invisible for a cubic
    # cell, wrong for a triclinic one. mu' = mu C^{-T} C makes the oracle's mu' C^{-1} equal
    # to mu C^{-T}.
    orig = O2.PMEOracle.mesh_density

    def bad(self, pos, q, mu):
        t = torch.as_tensor(self.Cinv.T @ self.C)
        return orig(self, pos, q, mu @ t)
    monkeypatch.setattr(O2.PMEOracle, "mesh_density", bad)
    _fails(TP.test_triclinic_cell, small)


def test_missing_deconvolution_is_caught(monkeypatch, salt):
    ref = ewald.ewald(salt.pos, salt.q, salt.mu, salt.box, 0.3, rcut=10.0)
    orig = O2.PMEOracle.__init__

    def init(self, *a, **k):
        k["deconvolution"] = False
        orig(self, *a, **k)
    monkeypatch.setattr(O2.PMEOracle, "__init__", init)
    _fails(TP.test_converges_to_ewald_with_mesh, salt, ref, 6)


def test_wrong_energy_normalisation_is_caught(monkeypatch, salt):
    orig = O2.PMEOracle.recip_energy
    monkeypatch.setattr(O2.PMEOracle, "recip_energy", lambda self, r: 2.0 * orig(self, r))
    _fails(TP.test_recip_energy_matches_ksum, salt)


def test_wrong_dipole_self_term_is_caught(monkeypatch):
    orig = ewald.ewald

    def bad(pos, q, mu, box, alpha, **k):
        r = orig(pos, q, mu, box, alpha, **k)
        mu = np.zeros_like(pos) if mu is None else np.asarray(mu)
        r["energy"] = r["energy"] + (alpha ** 3 / (3 * math.sqrt(math.pi))) * np.sum(mu * mu)
        return r
    monkeypatch.setattr(ewald, "ewald", bad)
    _fails(TE.test_alpha_independence_charges_and_dipoles)


def test_wrong_b2_coefficient_is_caught(monkeypatch, small):
    orig = O2.PMEOracle._bfuncs

    def bad(r2, alpha, lmax):
        B = orig(r2, alpha, lmax)
        if lmax >= 2:
            B[2] = B[2] * 1.01
        return B
    monkeypatch.setattr(O2.PMEOracle, "_bfuncs", staticmethod(bad))
    _fails(TP.test_pair_term_matches_o1_real_space, small)


def test_spline_derivative_sign_is_caught(monkeypatch):
    import test_oracle_bspline as TB
    orig = bspline.W
    monkeypatch.setattr(bspline, "W", lambda p, t, deriv=0: (-1) ** deriv * orig(p, t, deriv))
    _fails(TB.test_derivatives_central_differences, 4, 1)


def test_wrong_real_space_field_sign_is_caught(monkeypatch):
    orig = ewald.real_space

    def bad(*a, **k):
        E, phi, field, fg = orig(*a, **k)
        return E, phi, -field, fg
    monkeypatch.setattr(ewald, "real_space", bad)
    _fails(TE.test_derivatives_central_differences)


# ---- the quadrupole extension (O1Q and O2 with theta) ---------------------------------

import test_oracle_quadrupole as TQ  # noqa: E402
from oracle import quadrupole as O1Q  # noqa: E402


@pytest.fixture
def small_quad():
    fr = W.rocksalt(1, 5.64, jitter=0.25, mu_sigma=0.1, seed=21)
    return fr, W.quadrupoles(fr.n, 0.1, seed=22)


def test_quadrupole_self_factor_is_caught(monkeypatch, small_quad):
    # Theta:Theta with weight 1 instead of 2 in the Gaussian-cloud self energy
    orig = O1Q.self_energy

    def bad(q, mu, theta, alpha):
        E, dq, dmu, dT = orig(q, mu, theta, alpha)
        c = alpha / math.sqrt(math.pi) * (4 * alpha ** 4 / 5)
        return E + c * np.sum(theta * theta), dq, dmu, dT + 2 * c * theta
    monkeypatch.setattr(O1Q, "self_energy", bad)
    _fails(TQ.test_alpha_independence_with_quadrupoles, small_quad)


def test_quadrupole_sign_in_structure_factor_is_caught(monkeypatch):
    # +Theta:kk instead of -Theta:kk in S(k)
    orig = O1Q.reciprocal
    monkeypatch.setattr(O1Q, "reciprocal",
                        lambda pos, q, mu, th, *a, **k: orig(pos, q, mu, -th, *a, **k))
    _fails(TQ.test_quadrupole_is_limit_of_charge_cluster)


def test_quadrupole_mesh_factor_is_caught(monkeypatch):
    # the mesh sees 2 Theta (a missing 1/2 in the second-moment convention)
    orig = O2.PMEOracle.mesh_density

    def bad(self, pos, q, mu, theta=None):
        return orig(self, pos, q, mu, None if theta is None else 2 * theta)
    monkeypatch.setattr(O2.PMEOracle, "mesh_density", bad)
    _fails(TQ.test_o2_converges_to_o1q_with_mesh_refinement)


def test_quadrupole_pair_cross_sign_is_caught(monkeypatch, small_quad):
    # mu_j - Theta_i cross term with the wrong sign: the pair energy then sees -mu for
    # sources j in the Theta_i contraction only
    orig = O2.PMEOracle.pair_energy

    def bad(self, pos, q, mu, pairs=None, theta=None):
        if theta is None:
            return orig(self, pos, q, mu, pairs)
        e_full = orig(self, pos, q, mu, pairs, theta)
        e_mu0 = orig(self, pos, q, mu * 0, pairs, theta)
        e_th0 = orig(self, pos, q, mu, pairs, None)
        e_both0 = orig(self, pos, q, mu * 0, pairs, None)
        # flip the whole mu-theta coupling
        return e_full - 2 * (e_full - e_mu0 - e_th0 + e_both0)
    monkeypatch.setattr(O2.PMEOracle, "pair_energy", bad)
    _fails(TQ.test_o2_pair_term_matches_o1q_real_space, small_quad)
