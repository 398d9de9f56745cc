"""Pins for O2, the plain CPU particle-mesh Ewald oracle (Section 2.3)."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ewald, pme


@pytest.fixture(scope="module")
def salt():
    return W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000)


@pytest.fixture(scope="module")
def small():
    return W.rocksalt(1, 5.64, jitter=0.25, mu_sigma=0.1, seed=21)


@pytest.fixture(scope="module")
def ewald_ref(salt):
    # converged reciprocal space, real space truncated at the same 10 A as the PME pair term
    return ewald.ewald(salt.pos, salt.q, salt.mu, salt.box, 0.3, rcut=10.0)


def _frmse(F, Fref):
    return np.sqrt(((F - Fref) ** 2).mean()) / np.sqrt((Fref ** 2).mean())


def test_energy_forms_agree(salt):
    # Eq. energy_recip printed as (1/2V) sum rho phi equals the spectral sum (Parseval)
    o = pme.PMEOracle(salt.box, (20, 24, 18), 5, 0.3, 10.0)
    rho = o.mesh_density(*(torch.as_tensor(x) for x in (salt.pos, salt.q, salt.mu)))
    a = float(o.recip_energy(rho))
    b = float(o.recip_energy_realspace(rho))
    assert abs(a - b) < 1e-12 * abs(a)


def test_total_charge_on_mesh(salt):
    # the mesh carries the total charge (partition of unity) and dipoles add none
    o = pme.PMEOracle(salt.box, (24, 24, 24), 6, 0.3, 10.0)
    rho = o.stage_mesh(salt.pos, salt.q + 0.01, salt.mu)
    assert abs(rho.sum() - (salt.q + 0.01).sum()) < 1e-11
    # and the first moment of the dipole density is the total dipole (in mesh units)
    rho_mu = o.stage_mesh(salt.pos, np.zeros(salt.n), salt.mu)
    assert abs(rho_mu.sum()) < 1e-12


@pytest.mark.parametrize("p", [4, 6])
def test_converges_to_ewald_with_mesh(salt, ewald_ref, p):
    Fref = ewald_ref["force"]
    errs = []
    meshes = (16, 24, 32) if p == 4 else (16, 20, 24)
    for m in meshes:
        o = pme.PMEOracle(salt.box, (m, m, m), p, 0.3, 10.0)
        r = o.evaluate(salt.pos, salt.q, salt.mu, field_grad=False)
        errs.append(_frmse(r["force"], Fref))
    # error falls at least like h^(p-1) between the two finest meshes
    h = [salt.box[0, 0] / m for m in meshes]
    slope = math.log(errs[-2] / errs[-1]) / math.log(h[-2] / h[-1])
    assert errs[0] > errs[1] > errs[2]
    assert slope >= p - 1 - 0.3, (errs, slope)


def test_order_and_deconvolution(salt, ewald_ref):
    Eref = ewald_ref["energy"]
    out = {}
    for p, dec in [(4, True), (5, True), (6, True), (7, True), (4, False)]:
        o = pme.PMEOracle(salt.box, (32, 32, 32), p, 0.3, 10.0, deconvolution=dec)
        r = o.evaluate(salt.pos, salt.q, salt.mu, field_grad=False)
        out[(p, dec)] = (abs(r["energy"] - Eref), _frmse(r["force"], ewald_ref["force"]))
    f = [out[(p, True)][1] for p in (4, 5, 6, 7)]
    assert f[0] > f[1] > f[2] > f[3]
    # without the deconvolution of Eq. influence the error is far larger (Fig. ablation)
    assert out[(4, False)][0] > 100 * out[(4, True)][0]
    assert out[(4, False)][1] > 50 * out[(4, True)][1]
    assert out[(7, True)][1] < 1e-6


def test_recip_energy_matches_ksum(salt):
    # the mesh energy alone against the converged k-sum at the same alpha
    o = pme.PMEOracle(salt.box, (48, 48, 48), 6, 0.3, 10.0, include_pair=False,
                      include_self=False, include_background=False)
    r = o.evaluate(salt.pos, salt.q, salt.mu, field_grad=False)
    Ek, *_ = ewald.reciprocal(salt.pos, salt.q, salt.mu, salt.box, 0.3, ewald.kmax_for(0.3, 1e-16))
    assert abs(r["energy"] - Ek) < 3e-7 * abs(Ek)


def test_pair_term_matches_o1_real_space(small):
    o = pme.PMEOracle(small.box, (16, 16, 16), 4, 0.35, 7.0)
    E, phi, g, H = o.stage_pair(small.pos, small.q, small.mu)
    Er, phr, fr, gr = ewald.real_space(small.pos, small.q, small.mu, small.box, 0.35, 7.0)
    assert abs(E - Er) < 1e-12 * abs(Er)
    assert np.allclose(phi, phr, atol=1e-12)
    assert np.allclose(-g, fr, atol=1e-12)
    assert np.allclose(-H, gr, atol=1e-11)


def test_kdtree_pairs_match_bruteforce():
    fr = W.molten_nacl(512, seed=31)
    a = pme.pair_list(fr.pos, fr.box, 5.0)
    b = pme.pair_list_kdtree(fr.pos, np.diag(fr.box), 5.0)
    ka = sorted(zip(a[0], a[1], *np.round(a[2], 6).T))
    kb = sorted(zip(b[0], b[1], *np.round(b[2], 6).T))
    assert ka == kb


def test_translation_by_whole_mesh_cells(small):
    o = pme.PMEOracle(small.box, (12, 15, 16), 5, 0.35, 6.0)
    r0 = o.evaluate(small.pos, small.q, small.mu, field_grad=False)
    h = np.diag(small.box) / np.array([12, 15, 16])
    r1 = o.evaluate(small.pos + h * np.array([3, -2, 7]), small.q, small.mu, field_grad=False)
    assert abs(r0["energy"] - r1["energy"]) < 1e-12 * abs(r0["energy"])
    assert np.allclose(r0["force"], r1["force"], atol=1e-12)


def test_dipole_is_limit_of_charge_pair_on_mesh(small):
    o = pme.PMEOracle(small.box, (16, 16, 16), 6, 0.4, 5.0)
    Ed = o.evaluate(small.pos, small.q, small.mu, field_grad=False)["energy"]
    mnorm = np.linalg.norm(small.mu, axis=1)
    u = small.mu / mnorm[:, None]
    errs = []
    for sep in (0.02, 0.01):
        qd = mnorm / sep
        pos = np.concatenate([small.pos, small.pos + 0.5 * sep * u, small.pos - 0.5 * sep * u])
        q = np.concatenate([small.q, qd, -qd])
        Ec = o.evaluate(pos, q, np.zeros_like(pos), field_grad=False)["energy"] + np.sum(qd * qd / sep)
        errs.append(abs(Ec - Ed))
    assert errs[1] < errs[0] / 3.0
    assert errs[1] < 1e-6 * abs(Ed)


def test_autograd_gradients_central_differences(small):
    o = pme.PMEOracle(small.box, (16, 16, 16), 6, 0.35, 6.0)
    r = o.evaluate(small.pos, small.q, small.mu, field_grad=False)

    def E(pos=small.pos, q=small.q, mu=small.mu):
        return o.evaluate(pos, q, mu, field_grad=False)["energy"]

    h = 1e-5
    for i, c in [(0, 0), (3, 2), (6, 1)]:
        d = np.zeros_like(small.pos)
        d[i, c] = h
        assert abs((E(pos=small.pos + d) - E(pos=small.pos - d)) / (2 * h) + r["force"][i, c]) < 1e-8
        assert abs((E(mu=small.mu + d) - E(mu=small.mu - d)) / (2 * h) + r["field"][i, c]) < 1e-8
        dq = np.zeros(small.n)
        dq[i] = h
        assert abs((E(q=small.q + dq) - E(q=small.q - dq)) / (2 * h) - r["phi"][i]) < 1e-8


def test_field_gradient_consistency(salt):
    o = pme.PMEOracle(salt.box, (24, 24, 24), 6, 0.3, 10.0)
    r = o.evaluate(salt.pos, salt.q, salt.mu)
    F = salt.q[:, None] * r["field"] + np.einsum("iab,ib->ia", r["field_grad"], salt.mu)
    assert np.allclose(F, r["force"], atol=1e-12)


def test_hvp_central_differences(small):
    o = pme.PMEOracle(small.box, (16, 16, 16), 6, 0.35, 6.0)
    gF, gphi, gfield = W.tangent(small.n, seed=5)
    gE = 0.7
    a, b, c = o.hvp(small.pos, small.q, small.mu, gE, gF, gphi, gfield)

    def L(pos=small.pos, q=small.q, mu=small.mu):
        r = o.evaluate(pos, q, mu, field_grad=False)
        return (gE * r["energy"] + (gF * r["force"]).sum() + (gphi * r["phi"]).sum()
                + (gfield * r["field"]).sum())

    h = 1e-5
    for i, cc in [(1, 0), (4, 2), (7, 1)]:
        d = np.zeros_like(small.pos)
        d[i, cc] = h
        assert abs((L(pos=small.pos + d) - L(pos=small.pos - d)) / (2 * h) - a[i, cc]) < 1e-7
        assert abs((L(mu=small.mu + d) - L(mu=small.mu - d)) / (2 * h) - c[i, cc]) < 1e-7
        dq = np.zeros(small.n)
        dq[i] = h
        assert abs((L(q=small.q + dq) - L(q=small.q - dq)) / (2 * h) - b[i]) < 1e-7


def test_hvp_with_only_energy_cotangent_is_gradient(small):
    o = pme.PMEOracle(small.box, (16, 16, 16), 4, 0.35, 6.0)
    z = np.zeros_like(small.pos)
    a, b, c = o.hvp(small.pos, small.q, small.mu, 2.0, z, np.zeros(small.n), z)
    r = o.evaluate(small.pos, small.q, small.mu, field_grad=False)
    assert np.allclose(a, -2.0 * r["force"], atol=1e-13)
    assert np.allclose(b, 2.0 * r["phi"], atol=1e-13)
    assert np.allclose(c, -2.0 * r["field"], atol=1e-13)


def test_triclinic_cell(small):
    # the mesh path takes a general cell: compare a sheared cell against O1
    box = np.array([[11.0, 0.0, 0.0], [2.5, 10.5, 0.0], [-1.5, 1.0, 12.0]])
    rng = np.random.default_rng(4)
    frac = rng.uniform(size=(12, 3))
    pos = frac @ box
    q = rng.normal(size=12)
    q -= q.mean()
    mu = rng.normal(0, 0.1, size=(12, 3))
    ref = ewald.ewald(pos, q, mu, box, 0.45, rcut=8.0)
    o = pme.PMEOracle(box, (36, 36, 40), 7, 0.45, 8.0)
    r = o.evaluate(pos, q, mu, field_grad=False)
    assert abs(r["energy"] - ref["energy"]) < 1e-5 * abs(ref["energy"])
    assert _frmse(r["force"], ref["force"]) < 1e-4


def test_charged_frame_matches_ewald_with_background():
    # a frame with net charge 0.3: O2's neutralising background (energy -pi Q^2 / (2 V alpha^2),
    # potential -pi Q / (V alpha^2)) against the exact Ewald sum O1 with its own; at these
    # settings the two agree to 1e-7 of |E|, and the background is 5.6e-5 of |E| and 1.3e-3 in
    # the potential
    fr = W.molten_nacl(64, seed=5)
    q = fr.q.copy()
    q[0] += 0.3
    ref = ewald.ewald(fr.pos, q, fr.mu, fr.box, 0.6)
    r = pme.PMEOracle(fr.box, (32, 32, 32), 6, 0.6, 6.0).evaluate(fr.pos, q, fr.mu, field_grad=False)
    assert abs(r["energy"] - ref["energy"]) < 1e-6 * abs(ref["energy"])
    assert np.abs(r["phi"] - ref["phi"]).max() < 1e-5
    assert np.abs(r["force"] - ref["force"]).max() < 1e-5
    assert abs(ref["e_bg"]) > 3e-5 * abs(ref["energy"])      # the check is not vacuous


def test_parallel_dipole_lattice_closed_form():
    # identical parallel dipoles on a simple cubic lattice: the spherical vacuum sum over the
    # other dipoles vanishes by cubic symmetry (Lorentz), so with conducting boundaries (the
    # Ewald form) each site feels the field (4 pi / 3) M / V and E = -2 pi |M|^2 / (3 V), M the
    # total dipole; the forces and field gradients vanish. O1 is exact; O2's error falls with
    # the mesh at about the order of the spline
    fr = W.cubic_crystal([(0, 0, 0)], [0.0], 6, 3.0)
    mu = np.tile(np.array([0.1, 0.2, -0.05]), (fr.n, 1))
    V = abs(np.linalg.det(fr.box))
    M = mu.sum(0)
    e_ref = -2 * math.pi * (M @ M) / (3 * V)
    f_ref = (4 * math.pi / 3) * M / V
    r = ewald.ewald(fr.pos, fr.q, mu, fr.box, 0.5)
    assert abs(r["energy"] - e_ref) < 1e-12 * abs(e_ref)
    assert np.abs(r["field"] - f_ref).max() < 1e-12 * np.abs(f_ref).max()
    assert np.abs(r["force"]).max() < 1e-14 and np.abs(r["field_grad"]).max() < 1e-12
    errs = []
    for mesh in ((36, 36, 36), (48, 48, 48)):
        o = pme.PMEOracle(fr.box, mesh, 6, 0.5, 8.9).evaluate(fr.pos, fr.q, mu, field_grad=False)
        errs.append(abs(o["energy"] - e_ref) / abs(e_ref))
        assert np.abs(o["field"] - f_ref).max() < 2 * errs[-1] * np.abs(f_ref).max() + 1e-12
    assert errs[1] < 2e-5 and errs[0] / errs[1] > (48 / 36) ** 5


def test_stage_helpers_compose_to_the_evaluation():
    # the stage helpers the per-kernel GPU tests compare against (mesh density, solve, gather,
    # pair) reassemble, with the self and background terms of the Ewald split, the potential,
    # field and energy that evaluate() takes from autograd of the total energy
    fr = W.with_net_charge(W.molten_nacl(64, seed=31), 0.2, 4)
    a = 0.35
    o = pme.PMEOracle(fr.box, (20, 18, 16), 5, a, 6.0)
    rho = o.stage_mesh(fr.pos, fr.q, fr.mu)
    Phi, e_rec = o.stage_solve(rho)
    phi_m, g_m, _ = o.stage_gather(fr.pos, Phi)
    e_pair, phi_p, g_p, _ = o.stage_pair(fr.pos, fr.q, fr.mu)
    ev = o.evaluate(fr.pos, fr.q, fr.mu, field_grad=False)
    Q = fr.q.sum()
    V = abs(np.linalg.det(fr.box))
    phi = phi_m + phi_p - 2 * a / math.sqrt(math.pi) * fr.q - math.pi * Q / (V * a * a)
    field = -(g_m + g_p) + 4 * a ** 3 / (3 * math.sqrt(math.pi)) * fr.mu
    e_self = -a / math.sqrt(math.pi) * (fr.q ** 2).sum() - 2 * a ** 3 / (3 * math.sqrt(math.pi)) * (fr.mu ** 2).sum()
    e_bg = -math.pi * Q * Q / (2 * V * a * a)
    assert np.abs(phi - ev["phi"]).max() < 1e-12 * np.abs(ev["phi"]).max()
    assert np.abs(field - ev["field"]).max() < 1e-12 * np.abs(ev["field"]).max()
    assert abs(e_rec + e_pair + e_self + e_bg - ev["energy"]) < 1e-12 * abs(ev["energy"])
