"""Pins for O1Q, the explicit Ewald oracle with point quadrupoles (the rank-2 channel the
paper's closing discussion names as future work; the readings are in oracle/quadrupole.py)."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import ewald, quadrupole as Q


@pytest.fixture(scope="module")
def small():
    fr = W.rocksalt(1, 5.64, jitter=0.25, mu_sigma=0.1, seed=21)
    return fr, W.quadrupoles(fr.n, 0.1, seed=22)


def _autograd_tensors(rv, alpha, nmax):
    r = torch.tensor(rv, dtype=torch.float64, requires_grad=True)
    rn = torch.sqrt((r * r).sum(-1))
    f = torch.special.erfc(alpha * rn) / rn
    outs = [f.detach().numpy()]
    cur = [f]               # flattened list of the current-order components
    shape = ()
    for n in range(1, nmax + 1):
        nxt = []
        for c in cur:
            (g,) = torch.autograd.grad(c.sum(), r, create_graph=True)
            nxt.extend([g[:, k] for k in range(3)])
        cur = nxt
        shape = shape + (3,)
        outs.append(torch.stack(cur, -1).reshape((len(rv),) + shape).detach().numpy())
    return outs


def test_psi_derivative_tensors_match_autograd():
    rng = np.random.default_rng(3)
    rv = rng.normal(0, 2.0, size=(7, 3)) + np.array([0.5, 0.0, 0.0])
    D = Q.psi_derivatives(rv, 0.37, 5)
    A = _autograd_tensors(rv, 0.37, 5)
    for n in range(6):
        scale = np.abs(A[n]).max()
        assert np.allclose(D[n], A[n], atol=1e-12 * scale, rtol=0), n


def test_reduces_to_o1_without_quadrupoles(small):
    fr, _ = small
    a = Q.ewald(fr.pos, fr.q, fr.mu, None, fr.box, 0.45)
    b = ewald.ewald(fr.pos, fr.q, fr.mu, fr.box, 0.45)
    assert abs(a["energy"] - b["energy"]) < 1e-12 * abs(b["energy"])
    for key in ("phi", "field", "field_grad", "force"):
        assert np.allclose(a[key], b[key], atol=1e-11 * np.abs(b[key]).max()), key


def test_alpha_independence_with_quadrupoles(small):
    fr, T = small
    rs = [Q.ewald(fr.pos, fr.q, fr.mu, T, fr.box, a) for a in (0.35, 0.5, 0.65)]
    Es = [r["energy"] for r in rs]
    assert max(Es) - min(Es) < 1e-10 * abs(Es[0])
    for key in ("phi", "field", "field_grad", "force"):
        for r in rs[1:]:
            assert np.allclose(r[key], rs[0][key], atol=1e-10 * np.abs(rs[0][key]).max()), key


def _cluster(center, T, d):
    """Charges at center + {0, +-d e_k} along the eigenvectors e_k of T, with zero net charge
    and dipole and second moment 1/2 sum q d d = T (third moment zero)."""
    lam, E = np.linalg.eigh(T)
    pos, q = [center], [0.0]
    for k in range(3):
        s = lam[k] / (d * d)
        for sgn in (1.0, -1.0):
            pos.append(center + sgn * d * E[:, k])
            q.append(s)
        q[0] -= 2 * s
    return np.array(pos), np.array(q)


def _internal(pos, q):
    E = 0.0
    for a in range(len(q)):
        for b in range(a + 1, len(q)):
            E += q[a] * q[b] / np.linalg.norm(pos[a] - pos[b])
    return E


def test_quadrupole_is_limit_of_charge_cluster():
    fr = W.rocksalt(1, 5.64, jitter=0.25, seed=23)
    T = W.quadrupoles(fr.n, 0.3, seed=24)
    Eq = Q.ewald(fr.pos, fr.q, None, T, fr.box, 0.45)["energy"]
    errs = []
    # the error falls as d^2 until rounding of the ~1/d^5 intra-cluster energies takes over
    # (below d ~ 0.03 here)
    for d in (0.08, 0.04):
        P, C, Ein = [], [], 0.0
        for i in range(fr.n):
            p, c = _cluster(fr.pos[i], T[i], d)
            c = c.copy()
            c[0] += fr.q[i]
            # bare energy of every pair inside the cluster (the ion's own charge included):
            # the point-multipole sum leaves out i = j, n = 0
            Ein += _internal(p, c)
            P.append(p)
            C.append(c)
        P = np.concatenate(P)
        C = np.concatenate(C)
        Ec = ewald.ewald(P, C, None, fr.box, 0.45)["energy"] - Ein
        errs.append(Ec - Eq)
    assert abs(errs[1]) < abs(errs[0]) / 3.0, errs
    # Richardson: E(d) = Eq + c d^2 + O(d^4)
    assert abs((4 * errs[1] - errs[0]) / 3) < 1e-6 * abs(Eq), errs


def test_translation_invariance_and_zero_net_force(small):
    fr, T = small
    r0 = Q.ewald(fr.pos, fr.q, fr.mu, T, fr.box, 0.45)
    r1 = Q.ewald(fr.pos + np.array([0.37, -1.9, 2.3]), fr.q, fr.mu, T, fr.box, 0.45)
    assert abs(r0["energy"] - r1["energy"]) < 1e-11 * abs(r0["energy"])
    assert np.allclose(r0["force"], r1["force"], atol=1e-10)
    assert np.abs(r0["force"].sum(0)).max() < 1e-10


def test_derivatives_central_differences(small):
    fr, T = small
    r = Q.ewald(fr.pos, fr.q, fr.mu, T, fr.box, 0.45)

    def E(pos=fr.pos, q=fr.q, mu=fr.mu, th=T):
        return Q.ewald(pos, q, mu, th, fr.box, 0.45, rcut=r["rcut"], kmax=r["kmax"])["energy"]

    h = 1e-5
    tol = 1e-7
    for i, c in [(0, 0), (3, 2), (6, 1)]:
        d = np.zeros_like(fr.pos)
        d[i, c] = h
        assert abs((E(pos=fr.pos + d) - E(pos=fr.pos - d)) / (2 * h) + r["force"][i, c]) < tol
        assert abs((E(mu=fr.mu + d) - E(mu=fr.mu - d)) / (2 * h) + r["field"][i, c]) < tol
        dq = np.zeros(fr.n)
        dq[i] = h
        assert abs((E(q=fr.q + dq) - E(q=fr.q - dq)) / (2 * h) - r["phi"][i]) < tol
    for i, a, b in [(1, 0, 0), (2, 1, 2), (5, 2, 2), (7, 0, 1)]:
        dT = np.zeros_like(T)
        dT[i, a, b] += h
        if a != b:
            dT[i, b, a] += h
        fd = (E(th=T + dT) - E(th=T - dT)) / (2 * h)
        mult = 1.0 if a == b else 2.0
        assert abs(fd + mult * r["field_grad"][i, a, b]) < tol, (i, a, b)
    assert np.allclose(r["field_grad"], np.transpose(r["field_grad"], (0, 2, 1)), atol=1e-12)


# ---- O2 with quadrupoles --------------------------------------------------------------

from oracle import pme  # noqa: E402


def _frmse(F, Fref):
    return np.sqrt(((F - Fref) ** 2).mean()) / np.sqrt((Fref ** 2).mean())


def test_o2_pair_term_matches_o1q_real_space(small):
    fr, T = small
    o = pme.PMEOracle(fr.box, (16, 16, 16), 4, 0.45, 6.0)
    pairs = o._pairs(fr.pos)
    Ep = float(o.pair_energy(*(torch.as_tensor(x) for x in (fr.pos, fr.q, fr.mu)), pairs,
                             theta=torch.as_tensor(T)))
    Er, _ = Q.real_space(fr.pos, fr.q, fr.mu, T, fr.box, 0.45, 6.0)
    assert abs(Ep - Er) < 1e-12 * abs(Er)


def test_o2_reduces_without_quadrupoles(small):
    fr, _ = small
    o = pme.PMEOracle(fr.box, (16, 16, 16), 6, 0.45, 5.0)
    a = o.evaluate_quad(fr.pos, fr.q, fr.mu, np.zeros((fr.n, 3, 3)))
    b = o.evaluate(fr.pos, fr.q, fr.mu)
    assert abs(a["energy"] - b["energy"]) < 1e-13 * abs(b["energy"])
    for key in ("force", "phi", "field", "field_grad"):
        assert np.allclose(a[key], b[key], atol=1e-12 * np.abs(b[key]).max()), key


def test_o2_converges_to_o1q_with_mesh_refinement():
    fr = W.rocksalt(2, 5.64, jitter=0.2, mu_sigma=0.1, seed=25)
    T = W.quadrupoles(fr.n, 0.1, seed=26)
    ref = Q.ewald(fr.pos, fr.q, fr.mu, T, fr.box, 0.4, rcut=8.0)
    errE, errF, errG = [], [], []
    for N in (16, 24, 36):
        r = pme.PMEOracle(fr.box, (N, N, N), 6, 0.4, 8.0).evaluate_quad(fr.pos, fr.q, fr.mu, T)
        errE.append(abs(r["energy"] - ref["energy"]) / abs(ref["energy"]))
        errF.append(_frmse(r["force"], ref["force"]))
        errG.append(_frmse(r["field_grad"], ref["field_grad"]))
    assert errF[0] > errF[1] > errF[2], errF
    assert errG[0] > errG[1] > errG[2], errG
    assert errE[2] < 1e-6 and errF[2] < 1e-4 and errG[2] < 1e-4, (errE, errF, errG)


def test_o2_quadrupole_is_limit_of_charge_cluster_on_mesh():
    fr = W.rocksalt(1, 5.64, jitter=0.25, seed=27)
    T = W.quadrupoles(fr.n, 0.3, seed=28)
    # a cutoff where erfc(alpha rcut) ~ 1e-16: a cluster cut by the cutoff sphere would
    # otherwise leave a truncation error that grows with its ~1/d^2 charges
    o = pme.PMEOracle(fr.box, (16, 16, 16), 6, 0.45, 13.5)
    Eq = o.evaluate_quad(fr.pos, fr.q, np.zeros_like(fr.pos), T)["energy"]
    errs = []
    for d in (0.08, 0.04):
        P, C, Ein = [], [], 0.0
        for i in range(fr.n):
            p, c = _cluster(fr.pos[i], T[i], d)
            c = c.copy()
            c[0] += fr.q[i]
            Ein += _internal(p, c)
            P.append(p)
            C.append(c)
        P = np.concatenate(P)
        C = np.concatenate(C)
        Ec = o.evaluate(P, C, np.zeros_like(P), field_grad=False)["energy"] - Ein
        errs.append(Ec - Eq)
    assert abs(errs[1]) < abs(errs[0]) / 3.0, errs
    assert abs((4 * errs[1] - errs[0]) / 3) < 1e-6 * abs(Eq), errs


def test_o2_translation_by_whole_mesh_cells(small):
    fr, T = small
    o = pme.PMEOracle(fr.box, (12, 15, 16), 5, 0.45, 5.0)
    r0 = o.evaluate_quad(fr.pos, fr.q, fr.mu, T)
    h = np.diag(fr.box) / np.array([12, 15, 16])
    r1 = o.evaluate_quad(fr.pos + h * np.array([3, -2, 7]), fr.q, fr.mu, T)
    assert abs(r0["energy"] - r1["energy"]) < 1e-12 * abs(r0["energy"])
    assert np.allclose(r0["force"], r1["force"], atol=1e-11)
    assert np.allclose(r0["field_grad"], r1["field_grad"], atol=1e-11)


def test_o2_quad_hvp_central_differences(small):
    # the force-matching backward with quadrupoles (the VJP a later GPU backward is checked
    # against): central differences of L = gE E - gF.F + gphi.phi - gfield.field
    fr, T = small
    o = pme.PMEOracle(fr.box, (16, 16, 16), 6, 0.45, 5.0)
    gF, gphi, gfield = W.tangent(fr.n, seed=47)
    gE = 0.7
    a, b, c, d = o.hvp_quad(fr.pos, fr.q, fr.mu, T, gE, gF, gphi, gfield)

    def L(pos=fr.pos, q=fr.q, mu=fr.mu, th=T):
        r = o.evaluate_quad(pos, q, mu, th)
        return (gE * r["energy"] + (gF * r["force"]).sum() + (gphi * r["phi"]).sum()
                + (gfield * r["field"]).sum())

    h = 1e-5
    for i, cc in [(1, 0), (4, 2), (7, 1)]:
        dd = np.zeros_like(fr.pos)
        dd[i, cc] = h
        assert abs((L(pos=fr.pos + dd) - L(pos=fr.pos - dd)) / (2 * h) - a[i, cc]) < 1e-7
        assert abs((L(mu=fr.mu + dd) - L(mu=fr.mu - dd)) / (2 * h) - c[i, cc]) < 1e-7
        dq = np.zeros(fr.n)
        dq[i] = h
        assert abs((L(q=fr.q + dq) - L(q=fr.q - dq)) / (2 * h) - b[i]) < 1e-7
    for i, p_, q_ in [(2, 0, 0), (5, 1, 2)]:
        dT = np.zeros_like(T)
        dT[i, p_, q_] += h
        if p_ != q_:
            dT[i, q_, p_] += h
        fd = (L(th=T + dT) - L(th=T - dT)) / (2 * h)
        assert abs(fd - (1.0 if p_ == q_ else 2.0) * d[i, p_, q_]) < 1e-7
    # with only the energy cotangent it is the gradient
    z = np.zeros_like(fr.pos)
    a0, b0, c0, d0 = o.hvp_quad(fr.pos, fr.q, fr.mu, T, 2.0, z, np.zeros(fr.n), z)
    r = o.evaluate_quad(fr.pos, fr.q, fr.mu, T)
    assert np.allclose(a0, -2.0 * r["force"], atol=1e-12)
    assert np.allclose(d0, -2.0 * r["field_grad"], atol=1e-12)


def test_o2_quad_forces_are_energy_gradient_at_order4(small):
    # at p = 4 the quadrupole density uses the second spline derivative, which is continuous:
    # the mesh energy is then continuous with kinks only where an ion crosses a spline knot,
    # and away from them the force (with Theta : grad^3 phi) is -dE/dr; central differences
    # with a step far below any ion's distance to a knot check it
    fr, T = small
    o = pme.PMEOracle(fr.box, (16, 16, 16), 4, 0.45, 5.0)
    r = o.evaluate_quad(fr.pos, fr.q, fr.mu, T)
    h = 1e-6
    x = fr.pos @ np.linalg.inv(fr.box) * 16.0          # mesh coordinates
    for i, c in [(0, 0), (2, 1), (5, 2), (7, 0)]:
        # knots of the order-4 stencil are at integer mesh coordinates
        assert np.abs(x[i] - np.round(x[i])).min() > 1e-3
        d = np.zeros_like(fr.pos)
        d[i, c] = h
        ep = o.evaluate_quad(fr.pos + d, fr.q, fr.mu, T)["energy"]
        em = o.evaluate_quad(fr.pos - d, fr.q, fr.mu, T)["energy"]
        assert abs((ep - em) / (2 * h) + r["force"][i, c]) < 1e-6 * max(1.0, abs(r["force"][i, c]))
