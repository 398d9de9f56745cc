"""O4: the learned charge/dipole network, float64 PyTorch on the CPU (test infrastructure:
only tests, the smoke check and the benchmark's CPU leg use it).

The paper predicts latent charges from the scalar (rank-0) features and dipoles from the
vector (rank-1) features of a HotPP Cartesian-tensor message-passing backbone (Sections 2.1
and 2.2, Eqs. charge_pred, dipole_pred, site_energy), with a Bessel radial basis of 8
functions, a polynomial cutoff envelope of order 5 and a 5 A cutoff (Section 3.1). The
backbone itself is external code; the network here is the project's own small E(3)-
equivariant Cartesian-tensor net of that family, written plainly:

* Inputs: positions r_i, species s_i in {0 (Na), 1 (Cl)}, periodic box per frame.
* Edges: every ordered pair (i, j) of one frame and every periodic image with
  0 < |d| < r_c, d = r_j - r_i + n C (n integer, rows of C the lattice vectors), r = |d|,
  d^ = d / r. Radial basis e_k(r) = sqrt(2/r_c) sin(k pi r / r_c) / r * u(r / r_c),
  k = 1..8, with the envelope u(x) = 1 - 21 x^5 + 35 x^6 - 15 x^7 (order 5: u and its first
  two derivatives vanish at the cutoff).
* Features: S = 32 scalar channels h^s_i, V = 16 vector channels h^v_i (3 x 16); h^s starts as
  a learned embedding of the species, h^v at zero.
* Each of the 2 layers:
    A = h^s WA (32 -> 48), B = h^v WB (16 -> 32, the same matrix on each Cartesian component);
    radial weights R = e(r) WR (8 -> 80) per edge, split R_ss (32), R_sv (16), R_vs (16),
    R_vv (16); messages summed over the edges of i and divided by 16 (the mean neighbour
    count at the task's density):
      m^s_c      = sum_j R_ss,c A_j,c                  c < 32
      m^s_(32+c) = sum_j R_sv,c (d^ . B_j,c)           c < 16
      m^v_c      = sum_j R_vs,c d^ A_j,(32+c)          c < 16
      m^v_(16+c) = sum_j R_vv,c B_j,(16+c)             c < 16
    U = m^s WU (48 -> 48), Y = m^v WY (32 -> 16);
    h^s <- h^s + SiLU(U_(:32)),  h^v <- h^v + sigmoid(U_(32:48)) * Y (one gate per vector
    channel, the same on its three components).
  Vector features are only mixed linearly across channels and scaled by invariant scalars,
  so they rotate with the frame; scalars are invariant.
* Readouts: H = h^s Wh + bh (32 -> 64); charges q~_i = wq . SiLU(H_(:32)) + bq (Eq.
  charge_pred, a two-layer perceptron with SiLU), made neutral per frame, q = q~ - mean(q~);
  dipoles mu_i = sum_c wmu_c h^v_i,c (Eq. dipole_pred: a bias-free channel mix keeps it
  equivariant); site energies E_i = wE . SiLU(H_(32:)) + bE (Eq. site_energy).

The weights of the five channel-mixing products (WA, WB, WU, WY, Wh) are given as bfloat16
values; the oracle uses them as exact float64 numbers. The total energy of a frame is
E = sum_i E_i + E_PME(r, q, mu) (Section 2.4, Eq. E_total) with E_PME the plain PME of O2.

Pins (tests/test_oracle_net.py): rotation equivariance (q, E invariant; mu rotates),
translation and permutation invariance, a two-ion system against a hand-expanded numpy
evaluation of the same definitions, the envelope's vanishing value and derivatives at r_c,
forces against central differences, and the force-matching gradient of Eq. loss against
central differences of the loss. Parity: pinned.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import pme as O2

S, V, NRAD, LAYERS = 32, 16, 8, 2
RC = 5.0
NAVG = 16.0


def _t(x):
    return torch.as_tensor(np.asarray(x, np.float64))


def edges(pos, box, rc: float = RC):
    """(i, j, shift) of every ordered pair and periodic image with 0 < |r_j - r_i + shift| < rc
    (shift = n C, all integer n that can reach)."""
    pos = np.asarray(pos, np.float64)
    C = np.asarray(box, np.float64).reshape(3, 3)
    # image range from the perpendicular widths of the cell
    vol = abs(np.linalg.det(C))
    widths = [vol / np.linalg.norm(np.cross(C[(a + 1) % 3], C[(a + 2) % 3])) for a in range(3)]
    nmax = [int(math.ceil(rc / w)) + 1 for w in widths]
    I, J, SH = [], [], []
    n = len(pos)
    for a in range(-nmax[0], nmax[0] + 1):
        for b in range(-nmax[1], nmax[1] + 1):
            for c in range(-nmax[2], nmax[2] + 1):
                sh = a * C[0] + b * C[1] + c * C[2]
                d = pos[None, :, :] - pos[:, None, :] + sh          # [i, j] : r_j - r_i + sh
                r2 = (d * d).sum(-1)
                ok = (r2 < rc * rc) & (r2 > 0.0)
                ii, jj = np.nonzero(ok)
                I.append(ii)
                J.append(jj)
                SH.append(np.repeat(sh[None], len(ii), 0))
    if n == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros((0, 3))
    return np.concatenate(I), np.concatenate(J), np.concatenate(SH)


def envelope(x):
    return 1.0 - 21.0 * x ** 5 + 35.0 * x ** 6 - 15.0 * x ** 7


def radial_basis(r):
    """e_k(r), k = 1..8, as [E, 8]."""
    k = torch.arange(1, NRAD + 1, dtype=torch.float64)
    return (math.sqrt(2.0 / RC) * torch.sin(k[None, :] * math.pi * r[:, None] / RC) / r[:, None]
            * envelope(r / RC)[:, None])


def silu(x):
    return x * torch.sigmoid(x)


def features(pos, species, params, edge_list):
    """Final scalar and vector features (h^s [n, 32], h^v [n, 3, 16]) of one frame."""
    i, j, sh = edge_list
    i = torch.as_tensor(i)
    j = torch.as_tensor(j)
    n = pos.shape[0]
    d = pos[j] - pos[i] + _t(sh)
    r = torch.sqrt((d * d).sum(-1))
    dh = d / r[:, None]
    e = radial_basis(r)
    hs = params["emb"][torch.as_tensor(np.asarray(species, np.int64))]
    hv = torch.zeros((n, 3, V), dtype=torch.float64)
    for t in range(LAYERS):
        A = hs @ params[f"WA{t}"]                        # [n, 48]
        B = hv @ params[f"WB{t}"]                        # [n, 3, 32]
        R = e @ params[f"WR{t}"]                         # [E, 80]
        Rss, Rsv, Rvs, Rvv = R[:, :S], R[:, S:S + V], R[:, S + V:S + 2 * V], R[:, S + 2 * V:]
        ms = torch.zeros((n, S + V), dtype=torch.float64)
        mv = torch.zeros((n, 3, 2 * V), dtype=torch.float64)
        ms = ms.index_add(0, i, torch.cat([Rss * A[j, :S],
                                           Rsv * torch.einsum("ea,eac->ec", dh, B[j][:, :, :V])], 1))
        mv = mv.index_add(0, i, torch.cat([Rvs[:, None, :] * dh[:, :, None] * A[j, None, S:],
                                           Rvv[:, None, :] * B[j][:, :, V:]], 2))
        ms = ms / NAVG
        mv = mv / NAVG
        U = ms @ params[f"WU{t}"]                        # [n, 48]
        Y = mv @ params[f"WY{t}"]                        # [n, 3, 16]
        hs = hs + silu(U[:, :S])
        hv = hv + torch.sigmoid(U[:, S:])[:, None, :] * Y
    return hs, hv


def readout(hs, hv, params):
    """(q, mu, site energies) of one frame from its final features."""
    H = hs @ params["Wh"] + params["bh"]
    qt = silu(H[:, :S]) @ params["wq"] + params["bq"][0]
    q = qt - qt.mean() if len(qt) else qt
    mu = hv @ params["wmu"]
    Ei = silu(H[:, S:]) @ params["wE"] + params["bE"][0]
    return q, mu, Ei


def to_torch(params, requires_grad=False):
    return {k: _t(v).clone().requires_grad_(requires_grad) for k, v in params.items()}


def predict(pos, species, box, params, edge_list=None):
    """q [n], mu [n, 3], E_sr = sum of site energies, for one frame (torch tensors; pos and
    params may require grad)."""
    if edge_list is None:
        edge_list = edges(pos.detach().numpy() if torch.is_tensor(pos) else pos, box)
    pos = pos if torch.is_tensor(pos) else _t(pos)
    hs, hv = features(pos, species, params, edge_list)
    q, mu, Ei = readout(hs, hv, params)
    return q, mu, Ei.sum()


class Model:
    """The learned model of Eq. E_total on one frame: network + plain PME (O2) on the given
    mesh, energy E = E_sr + E_PME(r, q(r), mu(r))."""

    def __init__(self, box, mesh=(32, 32, 32), order: int = 4, alpha: float = 0.30,
                 rcut: float = 9.0):
        self.box = np.asarray(box, np.float64)
        self.pme = O2.PMEOracle(self.box, mesh, order, alpha, rcut)

    def energy(self, pos, species, params, edge_list=None, pairs=None):
        if pairs is None:
            pairs = self.pme._pairs(pos.detach().numpy())
        q, mu, esr = predict(pos, species, self.box, params, edge_list)
        return esr + self.pme.energy(pos, q, mu, pairs), (q, mu, esr)

    def forces(self, pos, species, params):
        """Energy, forces -dE/dr (through q(r) and mu(r) too), q, mu, E_sr (numpy)."""
        pos_t = _t(pos).requires_grad_(True)
        E, (q, mu, esr) = self.energy(pos_t, species, to_torch(params))
        (g,) = torch.autograd.grad(E, pos_t)
        return dict(energy=float(E), force=(-g).numpy(), q=q.detach().numpy(),
                    mu=mu.detach().numpy(), e_sr=float(esr))


def loss_and_grad(frames, species, boxes, e_ref, f_ref, params, lambda_e=1.0, lambda_f=1.0,
                  mesh=(32, 32, 32), order: int = 4, alpha: float = 0.30, rcut: float = 9.0):
    """Force-matching loss of Eq. loss over a batch of frames,
        L = lambda_e mean_b ((E_b - E_ref,b) / N_b)^2 + lambda_f / (3 sum_b N_b) sum (F - F_ref)^2,
    and its gradient with respect to every parameter (by double backward through the forces).
    Returns (L, L_E, L_F, grads dict of numpy arrays)."""
    P = to_torch(params, requires_grad=True)
    LE = torch.zeros((), dtype=torch.float64)
    LF = torch.zeros((), dtype=torch.float64)
    ntot = sum(len(s) for s in species)
    for pos, sp, box, er, fr_ in zip(frames, species, boxes, e_ref, f_ref):
        m = Model(box, mesh, order, alpha, rcut)
        pos_t = _t(pos).requires_grad_(True)
        E, _ = m.energy(pos_t, sp, P)
        (g,) = torch.autograd.grad(E, pos_t, create_graph=True)
        F = -g
        nb = len(sp)
        LE = LE + ((E - float(er)) / nb) ** 2 / len(frames)
        LF = LF + ((F - _t(fr_)) ** 2).sum() / (3 * ntot)
    L = lambda_e * LE + lambda_f * LF
    grads = torch.autograd.grad(L, list(P.values()))
    return float(L), float(LE), float(LF), {k: gr.numpy() for k, gr in zip(P.keys(), grads)}
