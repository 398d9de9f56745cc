"""O1Q: explicit Ewald summation for point charges, dipoles and quadrupoles, float64 numpy.

The paper's closing discussion names quadrupolar (rank-2) channels as the next multipole
order for its PME layer but gives no formulas; this module is the definition the
quadrupole channel is checked against. Everything below is a reading, stated here:

* A quadrupole is a symmetric Cartesian tensor Theta (not made traceless) entering the
  interaction operator L_i = q_i + mu_i . grad_i + Theta_i : grad_i grad_i, so that the
  energy of ion i in an external potential phi is q phi + mu . grad phi + Theta : grad grad phi
  and a cluster of charges q_c at r + d_c with zero net charge and dipole tends to
  Theta = 1/2 sum_c q_c d_c (x) d_c. The total energy is
      E = 1/2 sum'_{i,j,n} L_i L_j 1/|r_i - r_j + n|     (tin-foil boundary).
* The Ewald split with psi(r) = erfc(alpha r)/r gives, with r = r_i - r_j + n and grad
  acting on r (grad_j = -grad):
      real space   1/2 sum' (q_i + mu_i.grad + Theta_i:grad grad)(q_j - mu_j.grad + Theta_j:grad grad) psi
      reciprocal   (2 pi / V) sum_{k != 0} exp(-k^2/4 alpha^2)/k^2 |S(k)|^2,
                   S(k) = sum_j (q_j + i mu_j.k - Theta_j:k k) exp(i k.r_j)
      self         -1/2 sum_i [L_i L_i' erf(alpha r)/r]_{r -> 0}, which with
                   erf(x)/x = (2/sqrt(pi))(1 - x^2/3 + x^4/10 - ...) is
                   -(alpha/sqrt(pi)) sum_i [q^2 + (2 alpha^2/3)|mu|^2 - (4 alpha^2/3) q tr Theta
                                            + (4 alpha^4/5)((tr Theta)^2 + 2 Theta:Theta)]
                   (the q and mu parts are the paper's Eqs. self_q and self_mu)
      background   -pi Q^2 / (2 V alpha^2), charges only (k = 0 is dropped for every order).
* The derivative tensors of the radial psi follow from d/dr_a B_l = -r_a B_{l+1}, with
  B_0 = psi and B_l = [(2l - 1) B_{l-1} + (2 alpha^2)^l exp(-alpha^2 r^2)/(alpha sqrt(pi))]/r^2:
  grad^n psi is the sum over the ways of pairing k of the n indices into Kronecker deltas
  (the other n - 2k carry a factor r) of (-1)^(n-k) B_(n-k) times that product.

Per-ion outputs: phi = dE/dq, field = -dE/dmu, field_grad = -dE/dTheta (the symmetric 3x3
G with dE = -G : dTheta for symmetric dTheta; it reduces to the field gradient of O1 when all
Theta vanish), force = -dE/dr = -(q grad phi + (grad grad phi) mu + Theta : grad^3 phi) with
phi the potential of all sources (real space of the others plus the reciprocal sum).

Pins (tests/test_oracle_quadrupole.py): the derivative tensors against automatic
differentiation, alpha-independence of the total energy, the quadrupole as the limit of a
charge cluster (error O(d^2)), reduction to O1 when Theta = 0, translation invariance and
zero net force, and central finite differences of the energy for every per-ion output.
Parity: pinned (the paper prints no quadrupole numbers; the pins are mathematical).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from scipy.special import erfc

from .ewald import image_shifts, kmax_for, kvectors, real_cutoff_for

SQRT_PI = math.sqrt(math.pi)


def radial_B(r2: np.ndarray, alpha: float, lmax: int):
    """B_0 .. B_lmax of the screened Coulomb psi = erfc(alpha r)/r at squared distances r2."""
    r = np.sqrt(r2)
    ex = np.exp(-alpha * alpha * r2)
    B = [erfc(alpha * r) / r]
    for l in range(1, lmax + 1):
        B.append(((2 * l - 1) * B[-1] + (2 * alpha * alpha) ** l * ex / (alpha * SQRT_PI)) / r2)
    return B


def _pairings(idx):
    """Every way to split the index tuple idx into disjoint pairs and singletons:
    yields (pairs, singles)."""
    idx = tuple(idx)
    if not idx:
        yield (), ()
        return
    first, rest = idx[0], idx[1:]
    for pairs, singles in _pairings(rest):            # first stays single
        yield pairs, (first,) + singles
    for k, partner in enumerate(rest):                # first pairs with partner
        others = rest[:k] + rest[k + 1:]
        for pairs, singles in _pairings(others):
            yield ((first, partner),) + pairs, singles


def psi_derivatives(rv: np.ndarray, alpha: float, nmax: int):
    """Full derivative tensors grad^n psi(r), n = 0..nmax, at displacements rv [P, 3]:
    a list of arrays of shapes [P], [P,3], [P,3,3], ..."""
    r2 = np.einsum("pk,pk->p", rv, rv)
    B = radial_B(r2, alpha, nmax)
    out = [B[0]]
    eye = np.eye(3)
    for n in range(1, nmax + 1):
        T = np.zeros((len(rv),) + (3,) * n)
        terms = list(_pairings(range(n)))
        for comp in itertools.product(range(3), repeat=n):
            v = np.zeros(len(rv))
            for pairs, singles in terms:
                k = len(pairs)
                d = 1.0
                for a, b in pairs:
                    d *= eye[comp[a], comp[b]]
                if d == 0.0:
                    continue
                f = (-1.0) ** (n - k) * B[n - k]
                for s in singles:
                    f = f * rv[:, comp[s]]
                v = v + f
            T[(slice(None),) + comp] = v
        out.append(T)
    return out


def _contract_sources(D, qj, mj, Tj, order):
    """Potential derivative of order `order` at the field point from sources (q, mu, Theta)
    at displacement r: grad^order (q psi - mu . grad psi + Theta : grad grad psi)."""
    n = order
    val = qj.reshape((-1,) + (1,) * n) * D[n]
    val = val - np.einsum("p...k,pk->p...", D[n + 1], mj)
    val = val + np.einsum("p...kl,pkl->p...", D[n + 2], Tj)
    return val


def real_space(pos, q, mu, theta, box, alpha, rcut):
    """Real-space erfc sum over every image inside rcut. Returns (E_real, [phi, grad phi,
    grad^2 phi, grad^3 phi]) of the potential of the other ions' images at each ion."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    shifts = image_shifts(box, rcut)
    zero = np.where(np.all(np.abs(shifts) < 1e-12, axis=1))[0][0]
    P = [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3, 3))]
    for i in range(n):
        d = pos[i][None, None, :] - pos[None, :, :] + shifts[:, None, :]
        r2 = np.einsum("snk,snk->sn", d, d)
        mask = r2 < rcut * rcut
        mask[zero, i] = False
        rv = d[mask]
        jj = np.broadcast_to(np.arange(n)[None, :], mask.shape)[mask]
        D = psi_derivatives(rv, alpha, 5)
        for o in range(4):
            P[o][i] = _contract_sources(D, q[jj], mu[jj], theta[jj], o).sum(0)
    E = 0.5 * np.sum(q * P[0] + np.einsum("ik,ik->i", mu, P[1]) + np.einsum("ikl,ikl->i", theta, P[2]))
    return E, P


def reciprocal(pos, q, mu, theta, box, alpha, kmax, chunk: int = 2048):
    """Reciprocal k-sum. Returns (E_recip, [phi, grad phi, grad^2 phi, grad^3 phi]) of the
    Gaussian-screened potential of every source (the ion's own cloud included)."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    V = abs(np.linalg.det(box))
    K = kvectors(box, kmax)
    P = [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3, 3))]
    E = 0.0
    for s in range(0, len(K), chunk):
        k = K[s:s + chunk]
        k2 = np.einsum("kc,kc->k", k, k)
        A = np.exp(-k2 / (4 * alpha * alpha)) / k2
        ph = np.exp(1j * (pos @ k.T))                                     # [n, K]
        src = q[:, None] + 1j * (mu @ k.T) - np.einsum("iab,ka,kb->ik", theta, k, k)
        S = np.sum(src * ph, axis=0)
        E += (4 * math.pi / V) * np.sum(A * np.abs(S) ** 2)              # half space: x2
        # potential of all sources at r: (8 pi / V) sum_half A Re(e^{ik.r} S*)
        t = ph * np.conj(S)[None, :] * A[None, :]
        c = 8 * math.pi / V
        P[0] += c * np.real(t).sum(1)
        P[1] += c * np.einsum("ik,ka->ia", -np.imag(t), k)               # Re(i k t)
        P[2] += c * np.einsum("ik,ka,kb->iab", -np.real(t), k, k)         # Re(-k k t)
        P[3] += c * np.einsum("ik,ka,kb,kc->iabc", np.imag(t), k, k, k)  # Re(-i k k k t)
    return E, P


def self_energy(q, mu, theta, alpha):
    """Self energy of the Gaussian clouds (see the module docstring) and its derivatives
    with respect to q, mu and Theta (a symmetric matrix, as field_grad)."""
    a = alpha
    trT = np.einsum("iaa->i", theta)
    TT = np.einsum("iab,iab->i", theta, theta)
    c = a / SQRT_PI
    E = -c * np.sum(q * q + (2 * a * a / 3) * np.einsum("ik,ik->i", mu, mu)
                    - (4 * a * a / 3) * q * trT + (4 * a ** 4 / 5) * (trT * trT + 2 * TT))
    dq = -c * (2 * q - (4 * a * a / 3) * trT)
    dmu = -c * (4 * a * a / 3) * mu
    eye = np.eye(3)[None]
    dT = -c * (-(4 * a * a / 3) * q[:, None, None] * eye
               + (4 * a ** 4 / 5) * (2 * trT[:, None, None] * eye + 4 * theta))
    return E, dq, dmu, dT


def ewald(pos, q, mu, theta, box, alpha, *, rcut=None, kmax=None, tol=1e-16, coulomb_k=1.0):
    """Full explicit Ewald sum with quadrupoles (tin-foil). theta: [n, 3, 3] symmetric."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    mu = np.zeros_like(pos) if mu is None else np.asarray(mu, np.float64)
    theta = np.zeros((len(pos), 3, 3)) if theta is None else np.asarray(theta, np.float64)
    box = np.asarray(box, np.float64)
    V = abs(np.linalg.det(box))
    if rcut is None:
        rcut = real_cutoff_for(alpha, tol)
    if kmax is None:
        kmax = kmax_for(alpha, tol)
    Er, Pr = real_space(pos, q, mu, theta, box, alpha, rcut)
    Ek, Pk = reciprocal(pos, q, mu, theta, box, alpha, kmax)
    Es, dq, dmu, dT = self_energy(q, mu, theta, alpha)
    Q = q.sum()
    E_bg = -math.pi * Q * Q / (2 * V * alpha * alpha)
    P = [Pr[o] + Pk[o] for o in range(4)]
    phi = P[0] + dq - math.pi * Q / (V * alpha * alpha)
    field = -P[1] - dmu
    field_grad = -P[2] - dT
    force = -(q[:, None] * P[1] + np.einsum("iab,ib->ia", P[2], mu)
              + np.einsum("iab,iabc->ic", theta, P[3]))
    E = Er + Ek + Es + E_bg
    k = coulomb_k
    return dict(energy=k * E, e_real=k * Er, e_recip=k * Ek, e_self=k * Es, e_bg=k * E_bg,
                phi=k * phi, field=k * field, field_grad=k * field_grad, force=k * force,
                rcut=rcut, kmax=kmax)


def sym_from6(t6: np.ndarray) -> np.ndarray:
    """[n, 6] (xx, yy, zz, xy, xz, yz) -> [n, 3, 3] symmetric."""
    t6 = np.asarray(t6, np.float64)
    T = np.empty((len(t6), 3, 3))
    T[:, 0, 0], T[:, 1, 1], T[:, 2, 2] = t6[:, 0], t6[:, 1], t6[:, 2]
    T[:, 0, 1] = T[:, 1, 0] = t6[:, 3]
    T[:, 0, 2] = T[:, 2, 0] = t6[:, 4]
    T[:, 1, 2] = T[:, 2, 1] = t6[:, 5]
    return T


def to6(T: np.ndarray) -> np.ndarray:
    """[n, 3, 3] -> [n, 6] (xx, yy, zz, xy, xz, yz)."""
    T = np.asarray(T)
    return np.stack([T[:, 0, 0], T[:, 1, 1], T[:, 2, 2], T[:, 0, 1], T[:, 0, 2], T[:, 1, 2]], 1)
