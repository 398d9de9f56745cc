"""O1: explicit Ewald summation for point charges and point dipoles, float64 numpy.

This is the conventional Ewald reference the paper validates its PME against
(Section 2.3, introduction of the PME module; Results, Example 1 and Example 2).
The interaction operator is E = 1/2 sum'_{i,j,n} (q_i + mu_i.grad_i)(q_j + mu_j.grad_j)
1/|r_i - r_j + n|; the Ewald split with psi(r) = erfc(alpha r)/r gives

* real space:  1/2 sum' [q_i q_j B0 + (q_i mu_j - q_j mu_i).r B1 + mu_i.mu_j B1
                          - (mu_i.r)(mu_j.r) B2],  r = r_i - r_j + n,
  B0 = erfc(alpha r)/r,  B_l = [(2l-1) B_{l-1} + (2 alpha^2)^l exp(-alpha^2 r^2)/(alpha sqrt(pi))]/r^2;
* reciprocal:  (2 pi / V) sum_{k != 0} exp(-k^2/4 alpha^2)/k^2 |S(k)|^2,
  S(k) = sum_j (q_j + i mu_j.k) exp(i k.r_j)  (the Fourier transform of erf(alpha r)/r
  is the Green's function of Eq. green);
* self terms of Eqs. self_q and self_mu;
* neutralising background -pi Q^2 / (2 V alpha^2) (zero for neutral systems, the case
  the paper treats when it drops k = 0 under Eq. energy_recip);
* surface term 2 pi |M|^2 / ((2 eps' + 1) V), M = sum q r + sum mu; tin-foil (eps' = inf,
  zero) by default, which matches dropping k = 0.

Per-ion outputs: phi_i = dE/dq_i, field_i = -dE/dmu_i (the field of every other source,
including the dipole self term +4 alpha^3 mu_i/(3 sqrt(pi)) that cancels the ion's own
screening cloud), field_grad_i = gradient of that field at r_i (3x3; the reciprocal sum's
own-cloud part (4 alpha^3/(3 sqrt(pi))) q_i I is removed the same way, so both are
independent of alpha), force_i = -dE/dr_i = q_i field_i + field_grad_i mu_i.
Everything is analytic; nothing is differentiated numerically.

Pins (tests/test_oracle_ewald.py): rock-salt Madelung constant, alpha-independence of
the total energy, brute-force spherical image sums with the vacuum surface term, the
dipole as the limit of a charge pair, translation invariance, zero net force, and
central finite differences of the energy for forces, phi and field.  Parity: pinned.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

SQRT_PI = math.sqrt(math.pi)


def real_cutoff_for(alpha: float, tol: float) -> float:
    """Smallest R with erfc(alpha R) <= tol (bisection)."""
    lo, hi = 0.0, 100.0 / alpha
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if erfc(alpha * mid) > tol:
            lo = mid
        else:
            hi = mid
    return hi


def kmax_for(alpha: float, tol: float) -> float:
    """|k| beyond which exp(-k^2 / 4 alpha^2) <= tol."""
    return 2.0 * alpha * math.sqrt(-math.log(tol))


def perpendicular_widths(box: np.ndarray) -> np.ndarray:
    a = np.asarray(box, dtype=np.float64)
    V = abs(np.linalg.det(a))
    return np.array([V / np.linalg.norm(np.cross(a[(i + 1) % 3], a[(i + 2) % 3]))
                     for i in range(3)])


def image_shifts(box: np.ndarray, rcut: float) -> np.ndarray:
    """All lattice translations n.C that can bring a pair inside rcut (both signs)."""
    w = perpendicular_widths(box)
    K = [int(math.ceil(rcut / wi)) + 1 for wi in w]
    ns = np.array([[i, j, k] for i in range(-K[0], K[0] + 1)
                   for j in range(-K[1], K[1] + 1) for k in range(-K[2], K[2] + 1)],
                  dtype=np.float64)
    return ns @ np.asarray(box, dtype=np.float64)


def _bfuncs(r2: np.ndarray, alpha: float, lmax: int):
    r = np.sqrt(r2)
    ex = np.exp(-alpha * alpha * r2)
    B = [erfc(alpha * r) / r]
    for l in range(1, lmax + 1):
        B.append(((2 * l - 1) * B[-1] + (2 * alpha * alpha) ** l * ex / (alpha * SQRT_PI)) / r2)
    return B


def real_space(pos, q, mu, box, alpha, rcut):
    """Real-space erfc sum: returns (E_real, phi [n], field [n,3], field_grad [n,3,3])."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    shifts = image_shifts(box, rcut)
    zero = np.where(np.all(np.abs(shifts) < 1e-12, axis=1))[0][0]
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    fgrad = np.zeros((n, 3, 3))
    eye = np.eye(3)
    for i in range(n):
        d = pos[i][None, None, :] - pos[None, :, :] + shifts[:, None, :]  # [S, n, 3]
        r2 = np.einsum("snk,snk->sn", d, d)
        mask = r2 < rcut * rcut
        mask[zero, i] = False
        rv = d[mask]
        r2m = r2[mask]
        jj = np.broadcast_to(np.arange(n)[None, :], mask.shape)[mask]
        qj = q[jj]
        mj = mu[jj]
        B0, B1, B2, B3 = _bfuncs(r2m, alpha, 3)
        mr = np.einsum("pk,pk->p", mj, rv)
        phi[i] = np.sum(qj * B0 + mr * B1)
        field[i] = np.sum(qj[:, None] * rv * B1[:, None] - mj * B1[:, None]
                          + (mr * B2)[:, None] * rv, axis=0)
        rr = rv[:, :, None] * rv[:, None, :]
        g = (qj[:, None, None] * (eye[None] * B1[:, None, None] - rr * B2[:, None, None])
             + (mj[:, :, None] * rv[:, None, :] + rv[:, :, None] * mj[:, None, :]) * B2[:, None, None]
             + eye[None] * (mr * B2)[:, None, None]
             - rr * (mr * B3)[:, None, None])
        fgrad[i] = g.sum(axis=0)
    E = 0.5 * np.sum(q * phi - np.einsum("ik,ik->i", mu, field))
    return E, phi, field, fgrad


def kvectors(box: np.ndarray, kmax: float) -> np.ndarray:
    """Half-space set of reciprocal vectors 0 < |k| <= kmax (k and -k counted once)."""
    a = np.asarray(box, dtype=np.float64)
    b = 2.0 * math.pi * np.linalg.inv(a).T  # rows are b_alpha, a_alpha . b_beta = 2 pi delta
    nmax = [int(math.ceil(kmax * np.linalg.norm(a[i]) / (2 * math.pi))) + 1 for i in range(3)]
    nx = np.arange(-nmax[0], nmax[0] + 1)
    ny = np.arange(-nmax[1], nmax[1] + 1)
    nz = np.arange(-nmax[2], nmax[2] + 1)
    N = np.stack(np.meshgrid(nx, ny, nz, indexing="ij"), -1).reshape(-1, 3)
    half = (N[:, 0] > 0) | ((N[:, 0] == 0) & (N[:, 1] > 0)) | \
           ((N[:, 0] == 0) & (N[:, 1] == 0) & (N[:, 2] > 0))
    N = N[half]
    K = N @ b
    k2 = np.einsum("kc,kc->k", K, K)
    return K[k2 <= kmax * kmax]


def reciprocal(pos, q, mu, box, alpha, kmax, chunk: int = 2048):
    """Reciprocal k-sum: returns (E_recip, phi, field, field_grad)."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    V = abs(np.linalg.det(box))
    K = kvectors(box, kmax)
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    fgrad = np.zeros((n, 3, 3))
    E = 0.0
    for s in range(0, len(K), chunk):
        k = K[s:s + chunk]
        k2 = np.einsum("kc,kc->k", k, k)
        A = np.exp(-k2 / (4 * alpha * alpha)) / k2
        ph = np.exp(1j * (pos @ k.T))                     # [n, K]
        src = q[:, None] + 1j * (mu @ k.T)                # q_j + i mu_j.k
        S = np.sum(src * ph, axis=0)                      # [K]
        E += (4 * math.pi / V) * np.sum(A * np.abs(S) ** 2)   # half space: x2
        t = ph * np.conj(S)[None, :] * A[None, :]         # A e^{ik r_i} S*
        phi += (8 * math.pi / V) * np.real(t).sum(1)
        field += (8 * math.pi / V) * (np.imag(t) @ k)
        fgrad += (8 * math.pi / V) * np.einsum("ik,ka,kb->iab", np.real(t), k, k)
    return E, phi, field, fgrad


def ewald(pos, q, mu, box, alpha, *, rcut=None, kmax=None, tol=1e-16,
          surface_eps=math.inf, coulomb_k=1.0):
    """Full explicit Ewald sum. Returns a dict of energies and per-ion derivatives."""
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    mu = np.zeros_like(pos) if mu is None else np.asarray(mu, np.float64)
    box = np.asarray(box, np.float64)
    V = abs(np.linalg.det(box))
    if rcut is None:
        rcut = real_cutoff_for(alpha, tol)
    if kmax is None:
        kmax = kmax_for(alpha, tol)
    Er, phr, fr, gr = real_space(pos, q, mu, box, alpha, rcut)
    Ek, phk, fk, gk = reciprocal(pos, q, mu, box, alpha, kmax)
    Q = q.sum()
    E_self = -(alpha / SQRT_PI) * np.sum(q * q) - (2 * alpha ** 3 / (3 * SQRT_PI)) * np.sum(mu * mu)
    E_bg = -math.pi * Q * Q / (2 * V * alpha * alpha)
    phi = phr + phk - 2 * alpha / SQRT_PI * q - math.pi * Q / (V * alpha * alpha)
    c_self = 4 * alpha ** 3 / (3 * SQRT_PI)
    field = fr + fk + c_self * mu
    fgrad = gr + gk - c_self * q[:, None, None] * np.eye(3)[None]
    if math.isinf(surface_eps):
        E_surf = 0.0
    else:
        c = 4 * math.pi / ((2 * surface_eps + 1) * V)
        M = (q[:, None] * pos).sum(0) + mu.sum(0)
        E_surf = 0.5 * c * float(M @ M)
        phi = phi + c * (pos @ M)
        field = field - c * M
    force = q[:, None] * field + np.einsum("iab,ib->ia", fgrad, mu)
    E = Er + Ek + E_self + E_bg + E_surf
    k = coulomb_k
    return dict(energy=k * E, e_real=k * Er, e_recip=k * Ek, e_self=k * E_self, e_bg=k * E_bg,
                e_surf=k * E_surf, phi=k * phi, field=k * field, field_grad=k * fgrad,
                force=k * force, rcut=rcut, kmax=kmax)


def coulomb_images(pos, q, mu, box, nmax: int):
    """Brute-force Coulomb energy summed over image cells n with |n| <= nmax (integer
    triples inside a sphere): the vacuum (eps' = 1) lattice sum in the limit nmax -> inf.
    Only for tiny systems."""
    pos = np.asarray(pos, np.float64)
    n = len(pos)
    rng = np.arange(-nmax, nmax + 1)
    N = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    N = N[np.einsum("kc,kc->k", N, N) <= nmax * nmax]
    shifts = N @ np.asarray(box, np.float64)
    E = 0.0
    for i in range(n):
        for j in range(n):
            d = pos[i] - pos[j] + shifts
            r2 = np.einsum("kc,kc->k", d, d)
            if i == j:
                d = d[r2 > 0]
                r2 = r2[r2 > 0]
            r = np.sqrt(r2)
            mi = mu[i] @ d.T
            mj = mu[j] @ d.T
            E += 0.5 * np.sum(q[i] * q[j] / r + (q[i] * mj - q[j] * mi) / r ** 3
                              + (mu[i] @ mu[j]) / r ** 3 - 3 * mi * mj / r ** 5)
    return E
