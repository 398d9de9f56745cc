"""Pins of the network oracle O4 (oracle/net.py) against what symmetry and calculus fix:
rotation equivariance, translation / permutation invariance, extensivity under a supercell
replica (periodic images), locality of a 2-layer net with a 5 A cutoff, neutral charges, a vanishing dipole in a symmetric environment, the Bessel basis'
orthonormality and the envelope's closed form, forces and the force-matching gradient against
central differences."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import net as N


@pytest.fixture(scope="module")
def params():
    p = W.net_params(seed=11)
    # non-zero biases so that they are exercised
    rng = np.random.default_rng(3)
    for k in ("bh", "bq", "bE"):
        p[k] = rng.normal(0, 0.3, size=p[k].shape)
    return p


@pytest.fixture(scope="module")
def frame():
    return W.molten_nacl(64, seed=21)   # L = 12.7 A: several periodic images within 5 A


def _pred(pos, species, box, params):
    q, mu, e = N.predict(N._t(pos), species, box, N.to_torch(params))
    return q.numpy(), mu.numpy(), float(e)


def _rotation(seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q * np.sign(np.linalg.det(Q))


def test_rotation_equivariance(frame, params):
    q0, mu0, e0 = _pred(frame.pos, frame.species, frame.box, params)
    R = _rotation(5)
    # rotating positions and lattice vectors (rows) together: q and E invariant, mu rotates
    q1, mu1, e1 = _pred(frame.pos @ R.T, frame.species, frame.box @ R.T, params)
    assert np.allclose(q1, q0, atol=1e-12)
    assert abs(e1 - e0) < 1e-10 * max(1.0, abs(e0))
    assert np.allclose(mu1, mu0 @ R.T, atol=1e-12)
    assert np.abs(mu0).max() > 1e-3        # the check is not vacuous


def test_translation_and_permutation(frame, params):
    q0, mu0, e0 = _pred(frame.pos, frame.species, frame.box, params)
    q1, mu1, e1 = _pred(frame.pos + np.array([1.3, -7.1, 0.4]), frame.species, frame.box, params)
    assert np.allclose(q1, q0, atol=1e-12) and np.allclose(mu1, mu0, atol=1e-12)
    assert abs(e1 - e0) < 1e-10 * abs(e0)
    perm = np.random.default_rng(2).permutation(frame.n)
    q2, mu2, e2 = _pred(frame.pos[perm], frame.species[perm], frame.box, params)
    assert np.allclose(q2, q0[perm], atol=1e-12) and np.allclose(mu2, mu0[perm], atol=1e-12)
    assert abs(e2 - e0) < 1e-10 * abs(e0)


def test_supercell_replica_is_extensive(frame, params):
    # a periodic frame and its 2 x 1 x 1 replica are the same material: the replica's charges
    # and dipoles are the frame's, twice over, and its short-range energy is twice the frame's;
    # in the 12.7 A cell many 5 A neighbours are periodic images, so a lost image shows
    box2 = frame.box.copy()
    box2[0] = 2.0 * frame.box[0]
    pos2 = np.vstack([frame.pos, frame.pos + frame.box[0]])
    sp2 = np.concatenate([frame.species, frame.species])
    q0, mu0, e0 = _pred(frame.pos, frame.species, frame.box, params)
    q1, mu1, e1 = _pred(pos2, sp2, box2, params)
    assert np.allclose(q1, np.concatenate([q0, q0]), atol=1e-12)
    assert np.allclose(mu1, np.vstack([mu0, mu0]), atol=1e-12)
    assert abs(e1 - 2.0 * e0) < 1e-10 * abs(e0)
    _, _, sh = N.edges(frame.pos, frame.box)
    assert np.abs(sh).max(axis=1).astype(bool).mean() > 0.2   # the check is not vacuous


def test_neutral_charges(frame, params):
    q, _, _ = _pred(frame.pos, frame.species, frame.box, params)
    assert abs(q.sum()) < 1e-12 and np.abs(q).max() > 1e-3


def test_locality_of_two_layers(params):
    # in a large box, moving an ion farther than 2 r_c from ion 0 changes nothing at ion 0;
    # moving one within r_c of a neighbour of ion 0 does
    box = np.eye(3) * 40.0
    pos = np.array([[20.0, 20, 20], [23.0, 20, 20], [20.0, 23.5, 20], [26.0, 20, 20], [32.0, 20, 20]])
    sp = np.array([0, 1, 1, 0, 1])
    _, mu0, _ = _pred(pos, sp, box, params)
    far = pos.copy()
    far[4] += [0.0, 0.0, 1.5]                 # ion 4 stays > 10 A from ion 0
    _, mu1, _ = _pred(far, sp, box, params)
    assert np.allclose(mu1[0], mu0[0], atol=1e-14)
    near = pos.copy()
    near[3] += [0.0, 0.7, 0.0]                # ion 3 is 3 A from ion 1, 6 A from ion 0
    _, mu2, _ = _pred(near, sp, box, params)
    assert np.abs(mu2[0] - mu0[0]).max() > 1e-8


def test_symmetric_environment_has_no_dipole(params):
    # an ion at the centre of a regular octahedron of identical ions: by symmetry its dipole
    # vanishes; an ion with a single neighbour has its dipole along the bond
    box = np.eye(3) * 40.0
    c = np.array([20.0, 20, 20])
    octa = c + 2.8 * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    pos = np.vstack([c, octa])
    sp = np.array([0, 1, 1, 1, 1, 1, 1])
    _, mu, _ = _pred(pos, sp, box, params)
    assert np.abs(mu[0]).max() < 1e-13 and np.abs(mu[1]).max() > 1e-4
    pair = np.array([[20.0, 20, 20], [21.5, 22.0, 19.0]])
    _, mu2, _ = _pred(pair, np.array([0, 1]), box, params)
    d = pair[1] - pair[0]
    assert np.linalg.norm(np.cross(mu2[0], d)) < 1e-13 * max(1.0, np.linalg.norm(mu2[0]))


def test_bessel_basis_orthonormal_and_envelope():
    # without the envelope, sqrt(2/rc) sin(k pi r/rc)/r are orthonormal with weight r^2 on
    # [0, rc]; the order-5 envelope is 1 at 0 and vanishes with two derivatives at rc
    r = torch.linspace(1e-6, N.RC, 200001, dtype=torch.float64)[:-1]   # the integrand is 0 at rc
    e = N.radial_basis(r) / N.envelope(r / N.RC)[:, None]
    w = (r * r)[:, None]
    G = torch.trapezoid(e[:, :, None] * e[:, None, :] * w[:, :, None], r, dim=0).numpy()
    assert np.abs(G - np.eye(N.NRAD)).max() < 1e-6
    x = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    u = N.envelope(x)
    (d1,) = torch.autograd.grad(u, x, create_graph=True)
    (d2,) = torch.autograd.grad(d1, x)
    assert abs(float(u)) < 1e-14 and abs(float(d1)) < 1e-12 and abs(float(d2)) < 1e-12
    assert float(N.envelope(torch.tensor(0.0, dtype=torch.float64))) == 1.0


def test_forces_central_differences(params):
    fr = W.molten_nacl(32, seed=9)
    m = N.Model(fr.box, mesh=(12, 12, 12), order=4, alpha=0.4, rcut=4.5)
    r = m.forces(fr.pos, fr.species, params)
    P = N.to_torch(params)

    def E(pos):
        return float(m.energy(N._t(pos), fr.species, P)[0])

    h = 1e-5
    for i, c in [(0, 0), (5, 1), (17, 2)]:
        d = np.zeros_like(fr.pos)
        d[i, c] = h
        fd = (E(fr.pos + d) - E(fr.pos - d)) / (2 * h)
        assert abs(fd + r["force"][i, c]) < 1e-7 * max(1.0, abs(fd))


def test_loss_gradient_central_differences(params):
    # the gradient of Eq. loss (energies and forces) with respect to the parameters, through
    # the double backward, against central differences of the loss itself
    frames = [W.molten_nacl(32, seed=s) for s in (31, 32)]
    rng = np.random.default_rng(4)
    e_ref = [float(rng.normal()) for _ in frames]
    f_ref = [rng.normal(0, 0.2, size=(fr.n, 3)) for fr in frames]
    kw = dict(mesh=(12, 12, 12), order=4, alpha=0.4, rcut=4.5, lambda_e=0.7, lambda_f=1.3)
    args = ([fr.pos for fr in frames], [fr.species for fr in frames], [fr.box for fr in frames],
            e_ref, f_ref)
    L, LE, LF, g = N.loss_and_grad(*args, params, **kw)
    assert LE > 0 and LF > 0
    h = 1e-6
    for name, idx in [("WA1", (3, 40)), ("WR0", (2, 50)), ("WU1", (40, 35)), ("WY0", (20, 7)),
                      ("Wh", (5, 10)), ("wmu", (4,)), ("emb", (1, 3)), ("bq", (0,))]:
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[name][idx] += h
        pm[name][idx] -= h
        fd = (N.loss_and_grad(*args, pp, **kw)[0] - N.loss_and_grad(*args, pm, **kw)[0]) / (2 * h)
        assert abs(fd - g[name][idx]) < 1e-6 * max(1e-3, abs(fd)), (name, fd, g[name][idx])
