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


# ---- the learned network O4 and the polarisable teacher O3 -----------------------------

import test_oracle_net as TN  # noqa: E402
import test_oracle_teacher as TT  # noqa: E402
from oracle import net as N  # noqa: E402
from oracle import teacher as T  # noqa: E402


def _net_params():
    # as the network pins' fixture: seeded weights with non-zero biases
    p = W.net_params(seed=11)
    rng = np.random.default_rng(3)
    for k in ("bh", "bq", "bE"):
        p[k] = rng.normal(0, 0.3, size=p[k].shape)
    return p


@pytest.fixture
def net_frame():
    return W.molten_nacl(64, seed=21)


def test_dropped_charge_neutralisation_is_caught(monkeypatch, net_frame):
    # the charge head without its per-frame mean subtraction
    def bad(hs, hv, params):
        H = hs @ params["Wh"] + params["bh"]
        qt = N.silu(H[:, :N.S]) @ params["wq"] + params["bq"][0]
        _, mu, Ei = orig(hs, hv, params)
        return qt, mu, Ei
    orig = N.readout
    monkeypatch.setattr(N, "readout", bad)
    _fails(TN.test_neutral_charges, net_frame, _net_params())


def test_dipole_head_bias_is_caught(monkeypatch, net_frame):
    # a constant vector added to every dipole: not equivariant
    orig = N.readout

    def bad(hs, hv, params):
        q, mu, Ei = orig(hs, hv, params)
        return q, mu + torch.tensor([0.01, 0.0, 0.0], dtype=torch.float64), Ei
    monkeypatch.setattr(N, "readout", bad)
    _fails(TN.test_rotation_equivariance, net_frame, _net_params())


def test_dropped_periodic_images_is_caught(monkeypatch, net_frame):
    # the edge list without the neighbours that are periodic images
    orig = N.edges

    def bad(pos, box, rc=N.RC):
        i, j, sh = orig(pos, box, rc)
        keep = ~np.abs(sh).max(axis=1).astype(bool) if len(sh) else np.zeros(0, bool)
        return i[keep], j[keep], sh[keep]
    monkeypatch.setattr(N, "edges", bad)
    _fails(TN.test_supercell_replica_is_extensive, net_frame, _net_params())


def test_wrong_envelope_coefficient_is_caught(monkeypatch):
    monkeypatch.setattr(N, "envelope", lambda x: 1.0 - 21.0 * x ** 5 + 34.0 * x ** 6 - 15.0 * x ** 7)
    _fails(TN.test_bessel_basis_orthonormal_and_envelope)


def test_wrong_bessel_normalisation_is_caught(monkeypatch):
    orig = N.radial_basis
    monkeypatch.setattr(N, "radial_basis", lambda r: orig(r) / math.sqrt(2.0))
    _fails(TN.test_bessel_basis_orthonormal_and_envelope)


def test_model_force_sign_is_caught(monkeypatch):
    orig = N.Model.forces

    def bad(self, pos, species, params):
        r = orig(self, pos, species, params)
        r["force"] = -r["force"]
        return r
    monkeypatch.setattr(N.Model, "forces", bad)
    _fails(TN.test_forces_central_differences, _net_params())


def test_polarisation_energy_factor_is_caught(monkeypatch):
    # |mu|^2 / a instead of |mu|^2 / (2a): the energy is no longer stationary at mu = a E
    orig = T.polarisation_energy
    monkeypatch.setattr(T, "polarisation_energy", lambda mu, a: 2.0 * orig(mu, a))
    _fails(TT.test_self_consistency_and_stationarity, W.molten_nacl(32, seed=13))


def test_loose_dipole_convergence_is_caught(monkeypatch):
    # mixing stopped at a residual of 1e-4
    orig = T.solve_dipoles

    def bad(oracle, pos, q, a, **kw):
        kw["tol"] = 1e-4
        return orig(oracle, pos, q, a, **kw)
    monkeypatch.setattr(T, "solve_dipoles", bad)
    _fails(TT.test_self_consistency_and_stationarity, W.molten_nacl(32, seed=13))


def test_teacher_forces_without_dipoles_are_caught(monkeypatch):
    # forces taken from the charges alone, the induced dipoles left out
    orig = T.label

    def bad(frame, mesh=(32, 32, 32), order=4, alpha=0.30, rcut=9.0, **kw):
        lab = orig(frame, mesh=mesh, order=order, alpha=alpha, rcut=rcut, **kw)
        o = O2.PMEOracle(frame.box, mesh, order, alpha, rcut)
        lab["force"] = o.evaluate(frame.pos, lab["q"], np.zeros_like(frame.pos), field_grad=False)["force"]
        return lab
    monkeypatch.setattr(T, "label", bad)
    _fails(TT.test_hellmann_feynman_forces, W.molten_nacl(32, seed=13))


# ---- the virial (O2) -------------------------------------------------------------------

import test_oracle_virial as TV  # noqa: E402


def test_virial_without_background_is_caught(monkeypatch):
    # the term-by-term virial missing E_bg I (invisible on a neutral frame)
    orig = O2.PMEOracle.virial_terms

    def bad(self, pos, q, mu):
        Q = float(np.sum(q))
        return orig(self, pos, q, mu) + self.k * math.pi * Q * Q / (2 * self.V * self.alpha ** 2) * np.eye(3)
    monkeypatch.setattr(O2.PMEOracle, "virial_terms", bad)
    _fails(TV.test_virial_definition_matches_terms_charged)


def test_transposed_strain_is_caught(monkeypatch):
    # the cell strained by (I + eps^T): W comes out transposed, which fixed dipoles make visible
    orig = O2.PMEOracle.strained
    monkeypatch.setattr(O2.PMEOracle, "strained", lambda self, eps: orig(self, np.asarray(eps).T))
    _fails(TV.test_virial_definition_matches_terms_cubic, True)


def test_background_sign_in_pme_is_caught(monkeypatch):
    # O2's neutralising background with the wrong sign (invisible on a neutral frame)
    orig = O2.PMEOracle.energy

    def bad(self, pos, q, mu, pairs=None, parts=False, theta=None):
        E, P = orig(self, pos, q, mu, pairs, parts=True, theta=theta)
        E = E - 2.0 * P["e_bg"]
        if parts:
            P = dict(P, e_bg=-P["e_bg"])
            return E, P
        return E
    monkeypatch.setattr(O2.PMEOracle, "energy", bad)
    _fails(TP.test_charged_frame_matches_ewald_with_background)


# ---- the mesh-size rules ---------------------------------------------------------------

import test_oracle_meshdims as TM  # noqa: E402
from oracle import meshdims  # noqa: E402


def test_mesh_target_from_box_columns_is_caught(monkeypatch):
    # the lengths of the box's columns taken for those of its lattice vectors
    orig = meshdims.target
    monkeypatch.setattr(meshdims, "target",
                        lambda box, spacing, rule="paper": orig(np.asarray(box).T, spacing, rule))
    _fails(TM.test_mesh_dims_follow_the_lattice_vectors)


def test_smooth_size_below_target_is_caught(monkeypatch):
    # the largest smooth size <= target instead of the smallest >= target
    def bad(n):
        n = max(1, int(n))
        while not meshdims.is_smooth(n):
            n -= 1
        return n
    monkeypatch.setattr(meshdims, "next_smooth", bad)
    _fails(TM.test_strategies_against_enumeration)
