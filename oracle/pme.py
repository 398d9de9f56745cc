"""O2: plain particle-mesh Ewald for charges and dipoles, float64 PyTorch on the CPU.

The reciprocal part follows Section 2.3 step by step, in the paper's order and notation:

1. Mesh construction (Section 2.3.1): rows of C are the lattice vectors, the reciprocal
   basis b_alpha are the rows of 2 pi C^{-T}, V = |det C|.
2. Spline assignment (Section 2.3.2, Eqs. w3d and charge_dipole_assign): s = r C^{-1},
   x = N o s; the charge q_i and the dipole terms N_alpha (mu_i . C^{-1}_{:alpha}) times
   the derivative of the weight along mesh direction alpha are scattered onto the p^3
   stencil with periodic wrap (index_put with accumulate, as the paper does).
3. FFT of the mesh density (Eq. fft), unnormalised forward transform.
4. Green's function G(k) = 4 pi exp(-k^2/4 alpha^2)/k^2, G(0) = 0 (Eq. green), with
   k = n_x b_x + n_y b_y + n_z b_z over the signed FFT indices, times the deconvolution
   C(n) = 1/|B(n)|^(2 gamma), B(n) = prod_alpha sinc^p(n_alpha/N_alpha) (Eqs. Bk, influence).
5. Reciprocal energy (Eq. energy_recip). Reading: with phi the *unnormalised* inverse
   transform of G C rho_hat, (1/2V) sum_m rho(m) phi(m) = (1/2V) sum_{n != 0} G C |rho_hat|^2;
   the k = 0 term is excluded. The spectral form is what is evaluated here, over the full
   (not half) spectrum; tests check the two forms agree.
6. Self terms (Eqs. self_q, self_mu), and the neutralising background -pi Q^2/(2 V alpha^2)
   which the paper drops for neutral systems (reading: kept so learned charges that are
   neutral only to rounding still give a consistent energy).

Alongside the mesh runs the real-space erfc pair term of conventional Ewald (charge-charge,
charge-dipole, dipole-dipole, with B0..B2 radial functions) over an explicit pair list that
includes every periodic image inside the cutoff. It is written independently of O1.

Derivatives come from torch autograd, exactly as the paper obtains them: forces
F = -dE/dr (Eq. forces), dE/dq, dE/dmu, and, by double backward, the Hessian-vector
product that the force-matching loss (Eq. loss) needs. Field gradients at the ions are
obtained by autograd of the interpolated potential at a probe point with the sources held
fixed.

The virial W_ab = -dE/d(eps_ab) under the homogeneous strain r -> (I + eps) r of positions
and lattice vectors, with the dipoles held fixed (an extension: stress is not among the
paper's outputs), is evaluated from its definition by central differences of the energy,
and pinned against a term-by-term evaluation and the scaling identity
tr W = E_qq + 2 E_qmu + 3 E_mumu of the exact (O1) Ewald sum.

Point quadrupoles (an extension: the paper names the rank-2 channel as future work) enter
the spread as Theta : grad grad W, the pair term through the quadrupole contractions of
grad^2..grad^4 psi, and the self energy through the quadrupole parts of the Gaussian-cloud
self interaction (readings stated in oracle/quadrupole.py); their pins are in
tests/test_oracle_quadrupole.py (against O1Q, the charge-cluster limit on the mesh, and
mesh refinement).

Pins (tests/test_oracle_pme.py): agreement with O1 within the mesh error, which falls with
mesh refinement and with order and is larger without deconvolution; the two forms of Eq.
energy_recip; the dipole as the limit of a charge pair; exact invariance under whole-mesh-
cell translations; autograd gradients and Hessian-vector products against central
differences; the pair term against O1's real-space sum; F = q E + (mu.grad) E.
Parity: pinned.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import bspline

SQRT_PI = math.sqrt(math.pi)
f64 = torch.float64


def _t(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


# --------------------------------------------------------------------------------------
# pair list (numpy, float64)
# --------------------------------------------------------------------------------------

def pair_list(pos: np.ndarray, box: np.ndarray, rcut: float, chunk: int = 64):
    """Full ordered pair list (i, j, shift) with |r_i - r_j + shift| < rcut over all images,
    excluding (i, i, 0). Brute force over image translations; shift rows are n.C."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    n = len(pos)
    V = abs(np.linalg.det(box))
    w = [V / np.linalg.norm(np.cross(box[(a + 1) % 3], box[(a + 2) % 3])) for a in range(3)]
    K = [int(math.ceil(rcut / wa)) + 1 for a, wa in enumerate(w)]
    ns = np.array([[a, b, c] for a in range(-K[0], K[0] + 1) for b in range(-K[1], K[1] + 1)
                   for c in range(-K[2], K[2] + 1)], dtype=np.float64)
    shifts = ns @ box
    I, J, S = [], [], []
    rc2 = rcut * rcut
    for s0 in range(0, n, chunk):
        idx = np.arange(s0, min(n, s0 + chunk))
        d = pos[idx][:, None, None, :] - pos[None, :, None, :] + shifts[None, None, :, :]
        r2 = np.einsum("ijsk,ijsk->ijs", d, d)
        m = r2 < rc2
        ii, jj, ss = np.nonzero(m)
        ii = idx[ii]
        keep = ~((ii == jj) & (np.abs(shifts[ss]).sum(1) < 1e-12))
        I.append(ii[keep])
        J.append(jj[keep])
        S.append(shifts[ss[keep]])
    return np.concatenate(I), np.concatenate(J), np.concatenate(S)


def pair_list_kdtree(pos: np.ndarray, L: np.ndarray, rcut: float):
    """Same list for an orthorhombic box with rcut < L/2, via scipy's periodic k-d tree
    (minimum image is then unique). Returns (i, j, shift) in the same convention."""
    from scipy.spatial import cKDTree
    L = np.asarray(L, np.float64)
    if np.any(rcut >= L / 2):
        raise ValueError("k-d tree path needs rcut < L/2")
    w = np.mod(pos, L)
    tree = cKDTree(w, boxsize=L)
    pairs = tree.query_pairs(rcut, output_type="ndarray")
    i = np.concatenate([pairs[:, 0], pairs[:, 1]])
    j = np.concatenate([pairs[:, 1], pairs[:, 0]])
    # shift such that r_i - r_j + shift is the minimum image (for the caller's positions)
    d = pos[i] - pos[j]
    shift = -L * np.round(d / L)
    return i, j, shift


# --------------------------------------------------------------------------------------
# the oracle
# --------------------------------------------------------------------------------------

class PMEOracle:
    """Plain PME on one periodic frame; all inputs float64, all arithmetic float64."""

    def __init__(self, box, mesh, order: int, alpha: float, rcut: float, *,
                 influence_power: float = 1.0, deconvolution: bool = True,
                 coulomb_k: float = 1.0, include_pair: bool = True,
                 include_self: bool = True, include_background: bool = True,
                 influence_kind: str = "deconvolution", alias_range: int = 2):
        self.C = np.asarray(box, np.float64).reshape(3, 3)
        self.influence_kind = influence_kind
        self.alias_range = int(alias_range)
        self.Cinv = np.linalg.inv(self.C)
        self.b = 2.0 * math.pi * self.Cinv.T            # rows b_alpha
        self.V = abs(np.linalg.det(self.C))
        self.N = tuple(int(x) for x in mesh)
        self.p = int(order)
        self.alpha = float(alpha)
        self.rcut = float(rcut)
        self.gamma = float(influence_power)
        self.deconv = bool(deconvolution)
        self.k = float(coulomb_k)
        self.include_pair = include_pair
        self.include_self = include_self
        self.include_bg = include_background
        self.GC = _t(self.influence())

    # -- Section 2.3.3 / 2.3.4: influence function on the full signed spectrum ----------
    def influence(self) -> np.ndarray:
        if self.influence_kind == "p3m":
            return self.influence_p3m(self.alias_range)
        Nx, Ny, Nz = self.N
        n = [np.fft.fftfreq(Na) * Na for Na in self.N]
        nx, ny, nz = np.meshgrid(*n, indexing="ij")
        kvec = (nx[..., None] * self.b[0] + ny[..., None] * self.b[1] + nz[..., None] * self.b[2])
        k2 = np.einsum("...c,...c->...", kvec, kvec)
        G = np.zeros_like(k2)
        nz0 = k2 > 0
        G[nz0] = 4 * math.pi * np.exp(-k2[nz0] / (4 * self.alpha ** 2)) / k2[nz0]
        if self.deconv:
            B = (bspline.sinc_response(self.p, nx, Nx) * bspline.sinc_response(self.p, ny, Ny)
                 * bspline.sinc_response(self.p, nz, Nz))
            Cn = 1.0 / np.abs(B) ** (2 * self.gamma)
        else:
            Cn = np.ones_like(G)
        return G * Cn

    # -- alternative (not the paper's): the P3M influence function ------------------------
    def influence_p3m(self, mrange: int) -> np.ndarray:
        """Influence function that minimises the mean-square error of the forces obtained by
        differentiating the interpolated potential (analytical differentiation), for this
        assignment function, in the least-squares sense of Hockney and Eastwood: with the
        aliases k_m = sum_a (n_a + m_a N_a) b_a of the signed frequency n and
        U(k_m) = prod_a sinc^(2p)(n_a / N_a + m_a),
            G(n) = sum_m k_m^2 U(k_m) phi(k_m) / [(sum_m U(k_m)) (sum_m k_m^2 U(k_m))],
        phi(k) = 4 pi e^{-k^2/4 alpha^2}/k^2, G(0) = 0, sums over |m_a| <= mrange. Keeping only
        m = 0 gives phi / U, the sinc deconvolution with gamma = 1."""
        n = [np.fft.fftfreq(Na) * Na for Na in self.N]
        nx, ny, nz = np.meshgrid(*n, indexing="ij")
        num = np.zeros(nx.shape)
        s1 = np.zeros(nx.shape)
        s2 = np.zeros(nx.shape)
        for mx in range(-mrange, mrange + 1):
            ux = np.sinc(nx / self.N[0] + mx) ** (2 * self.p)
            for my in range(-mrange, mrange + 1):
                uy = np.sinc(ny / self.N[1] + my) ** (2 * self.p)
                for mz in range(-mrange, mrange + 1):
                    uz = np.sinc(nz / self.N[2] + mz) ** (2 * self.p)
                    kv = ((nx + mx * self.N[0])[..., None] * self.b[0] + (ny + my * self.N[1])[..., None] * self.b[1]
                          + (nz + mz * self.N[2])[..., None] * self.b[2])
                    k2 = np.einsum("...c,...c->...", kv, kv)
                    with np.errstate(divide="ignore", invalid="ignore"):
                        ph = np.where(k2 > 0, 4 * math.pi * np.exp(-k2 / (4 * self.alpha ** 2)) / k2, 0.0)
                    U = ux * uy * uz
                    num += k2 * U * ph
                    s1 += U
                    s2 += k2 * U
        with np.errstate(divide="ignore", invalid="ignore"):
            G = np.where(s2 > 0, num / (s1 * s2), 0.0)
        G[0, 0, 0] = 0.0
        return G

    # -- Section 2.3.2: spline assignment of charges and dipoles ------------------------
    def _stencils(self, pos):
        s = pos @ _t(self.Cinv)
        x = s * _t(np.array(self.N, np.float64))
        out = []
        for a in range(3):
            m0, w = bspline.stencil_weights(self.p, x[:, a], 0)
            _, dw = bspline.stencil_weights(self.p, x[:, a], 1)
            idx = torch.remainder(m0[:, None] + torch.arange(self.p), self.N[a])
            out.append((idx, w, dw))
        return out

    def mesh_density(self, pos, q, mu, theta=None):
        """rho_mesh of Eq. charge_dipole_assign as a flat torch tensor [Nx*Ny*Nz].

        With theta ([n,3,3] symmetric point quadrupoles, the rank-2 extension) each ion also
        adds Theta : grad grad W, the second derivative of its weights with respect to its
        position: sum_ab Theta'_ab d_a d_b W in mesh coordinates, with
        Theta'_ab = N_a N_b (C^-T Theta C^-1)_ab."""
        Nx, Ny, Nz = self.N
        (ix, wx, dx), (iy, wy, dy), (iz, wz, dz) = self._stencils(pos)
        dmu = (mu @ _t(self.Cinv)) * _t(np.array(self.N, np.float64))   # N_a (mu . C^-1_{:a})
        val = (q[:, None, None, None] * wx[:, :, None, None] * wy[:, None, :, None] * wz[:, None, None, :]
               + dmu[:, 0, None, None, None] * dx[:, :, None, None] * wy[:, None, :, None] * wz[:, None, None, :]
               + dmu[:, 1, None, None, None] * wx[:, :, None, None] * dy[:, None, :, None] * wz[:, None, None, :]
               + dmu[:, 2, None, None, None] * wx[:, :, None, None] * wy[:, None, :, None] * dz[:, None, None, :])
        if theta is not None:
            s = pos @ _t(self.Cinv)
            x = s * _t(np.array(self.N, np.float64))
            d2 = [bspline.stencil_weights(self.p, x[:, a], 2)[1] for a in range(3)]
            G = _t(self.Cinv * np.array(self.N, np.float64)[None, :])   # G[alpha, a] = N_a C^-1[alpha, a]
            Tp = torch.einsum("ka,ikl,lb->iab", G, theta, G)
            one = [wx, wy, wz]
            der1 = [dx, dy, dz]
            for a in range(3):
                for b in range(3):
                    f = []
                    for c in range(3):
                        order = (a == c) + (b == c)
                        f.append(one[c] if order == 0 else (der1[c] if order == 1 else d2[c]))
                    val = val + Tp[:, a, b, None, None, None] * (
                        f[0][:, :, None, None] * f[1][:, None, :, None] * f[2][:, None, None, :])
        flat = (ix[:, :, None, None] * Ny + iy[:, None, :, None]) * Nz + iz[:, None, None, :]
        rho = torch.zeros(Nx * Ny * Nz, dtype=f64)
        return rho.index_put((flat.reshape(-1),), val.reshape(-1), accumulate=True)

    # -- Section 2.3.4: FFT, Green x deconvolution, energy ------------------------------
    def recip_energy(self, rho_flat):
        rho_hat = torch.fft.fftn(rho_flat.reshape(self.N))
        return (0.5 / self.V) * torch.sum(self.GC * (rho_hat.real ** 2 + rho_hat.imag ** 2))

    def potential_mesh(self, rho_flat) -> torch.Tensor:
        """Phi(m) = (1/V) * unnormalised inverse FFT of G C rho_hat, so that
        E_recip = 1/2 sum_m rho(m) Phi(m)."""
        rho_hat = torch.fft.fftn(rho_flat.reshape(self.N))
        M = float(np.prod(self.N))
        return (torch.fft.ifftn(self.GC * rho_hat).real * (M / self.V))

    def recip_energy_realspace(self, rho_flat):
        """Eq. energy_recip as printed: (1/2V) sum_m rho(m) phi(m), phi the unnormalised
        inverse transform (used only to pin the spectral form)."""
        Phi = self.potential_mesh(rho_flat)
        return 0.5 * torch.sum(rho_flat.reshape(self.N) * Phi)

    # -- real-space pair term -----------------------------------------------------------
    def _pairs(self, pos_np):
        L = np.diag(self.C)
        ortho = np.allclose(self.C, np.diag(L))
        if ortho and np.all(self.rcut < L / 2) and len(pos_np) > 2048:
            return pair_list_kdtree(pos_np, L, self.rcut)
        return pair_list(pos_np, self.C, self.rcut)

    @staticmethod
    def _bfuncs(r2, alpha, lmax):
        r = torch.sqrt(r2)
        ex = torch.exp(-alpha * alpha * r2)
        B = [torch.special.erfc(alpha * r) / r]
        for l in range(1, lmax + 1):
            B.append(((2 * l - 1) * B[-1] + (2 * alpha * alpha) ** l * ex / (alpha * SQRT_PI)) / r2)
        return B

    def pair_energy(self, pos, q, mu, pairs=None, theta=None):
        if pairs is None:
            pairs = self._pairs(pos.detach().numpy())
        i, j, sh = pairs
        i = torch.as_tensor(i)
        j = torch.as_tensor(j)
        r = pos[i] - pos[j] + _t(sh)
        r2 = (r * r).sum(-1)
        B = self._bfuncs(r2, self.alpha, 2 if theta is None else 4)
        B0, B1, B2 = B[:3]
        mir = (mu[i] * r).sum(-1)
        mjr = (mu[j] * r).sum(-1)
        u = (q[i] * q[j] * B0 + (q[i] * mjr - q[j] * mir) * B1
             + (mu[i] * mu[j]).sum(-1) * B1 - mir * mjr * B2)
        if theta is not None:
            # quadrupole terms of (q_i + mu_i.grad + Th_i:grad grad)(q_j - mu_j.grad + Th_j:grad grad)
            # psi, each a contraction of grad^n psi written out with the B_l:
            #   A : grad^2 psi         = -tr A B1 + (r.A.r) B2
            #   m . grad^3 psi : A     = (tr A (m.r) + 2 m.A.r) B2 - (r.A.r)(m.r) B3
            #   A : grad^4 psi : C     = (tr A tr C + 2 A:C) B2
            #                            - (tr A (r.C.r) + tr C (r.A.r) + 4 (A r).(C r)) B3
            #                            + (r.A.r)(r.C.r) B4
            B3, B4 = B[3], B[4]
            Ti, Tj = theta[i], theta[j]
            tri = torch.einsum("paa->p", Ti)
            trj = torch.einsum("paa->p", Tj)
            Tir = torch.einsum("pab,pb->pa", Ti, r)
            Tjr = torch.einsum("pab,pb->pa", Tj, r)
            rTir = (Tir * r).sum(-1)
            rTjr = (Tjr * r).sum(-1)
            u = u + (q[i] * (-trj * B1 + rTjr * B2) + q[j] * (-tri * B1 + rTir * B2))
            u = u + ((trj * mir + 2 * (mu[i] * Tjr).sum(-1)) * B2 - rTjr * mir * B3)
            u = u - ((tri * mjr + 2 * (mu[j] * Tir).sum(-1)) * B2 - rTir * mjr * B3)
            u = u + ((tri * trj + 2 * (Ti * Tj).sum((-1, -2))) * B2
                     - (tri * rTjr + trj * rTir + 4 * (Tir * Tjr).sum(-1)) * B3 + rTir * rTjr * B4)
        return 0.5 * u.sum()

    # -- total energy -------------------------------------------------------------------
    def energy(self, pos, q, mu, pairs=None, parts=False, theta=None):
        quad = {} if theta is None else dict(theta=theta)
        rho = self.mesh_density(pos, q, mu, **quad)
        E_rec = self.recip_energy(rho)
        E_pair = self.pair_energy(pos, q, mu, pairs, **quad) if self.include_pair else pos.sum() * 0.0
        a = self.alpha
        E_self = (-(a / SQRT_PI) * (q * q).sum() - (2 * a ** 3 / (3 * SQRT_PI)) * (mu * mu).sum()) \
            if self.include_self else q.sum() * 0.0
        if theta is not None and self.include_self:
            # quadrupole parts of -1/2 sum_i [L_i L_i' erf(alpha r)/r] at r -> 0, from
            # erf(x)/x = (2/sqrt(pi))(1 - x^2/3 + x^4/10 - ...)
            tr = torch.einsum("iaa->i", theta)
            E_self = E_self - (a / SQRT_PI) * (-(4 * a * a / 3) * (q * tr).sum()
                                                + (4 * a ** 4 / 5) * ((tr * tr).sum() + 2 * (theta * theta).sum()))
        Q = q.sum()
        E_bg = (-math.pi * Q * Q / (2 * self.V * a * a)) if self.include_bg else Q * 0.0
        E = self.k * (E_rec + E_pair + E_self + E_bg)
        if parts:
            return E, dict(e_recip=self.k * E_rec, e_pair=self.k * E_pair,
                           e_self=self.k * E_self, e_bg=self.k * E_bg)
        return E

    # -- virial (stress), an extension beyond the paper's outputs ------------------------
    def strained(self, eps):
        """The same PME on the homogeneously strained cell, lattice rows a_i -> (I + eps) a_i."""
        F = np.eye(3) + np.asarray(eps, np.float64)
        return PMEOracle(self.C @ F.T, self.N, self.p, self.alpha, self.rcut,
                         influence_power=self.gamma, deconvolution=self.deconv, coulomb_k=self.k,
                         include_pair=self.include_pair, include_self=self.include_self,
                         include_background=self.include_bg, influence_kind=self.influence_kind,
                         alias_range=self.alias_range)

    def virial(self, pos, q, mu, h: float = 1e-5):
        """W_ab = -dE/d(eps_ab) for the homogeneous strain r -> (I + eps) r, a_i -> (I + eps) a_i
        with the dipoles held fixed: the definition, by central differences of the energy.
        The pair list (with its image shifts, which strain as lattice vectors) is held fixed,
        so no pair crosses the cutoff inside the difference stencil."""
        pos = np.asarray(pos, np.float64)
        q = np.asarray(q, np.float64)
        mu = np.zeros_like(pos) if mu is None else np.asarray(mu, np.float64)
        pairs = self._pairs(pos) if self.include_pair else None
        W = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                E = []
                for sgn in (1.0, -1.0):
                    eps = np.zeros((3, 3))
                    eps[a, b] = sgn * h
                    F = np.eye(3) + eps
                    pr = None if pairs is None else (pairs[0], pairs[1], pairs[2] @ F.T)
                    E.append(float(self.strained(eps).energy(_t(pos @ F.T), _t(q), _t(mu), pairs=pr)))
                W[a, b] = -(E[0] - E[1]) / (2 * h)
        return W

    def virial_terms(self, pos, q, mu):
        """The same virial assembled term by term (a second evaluation that pins virial()):
        reciprocal  E_rec I - (1/V) sum_n G C |rho_hat|^2 (1/k^2 + 1/(4 alpha^2)) k (x) k
                    + sum_i (dE_rec/dmu_i) (x) mu_i        (the mesh sees mu through C^-1),
        pair        -1/2 sum_(i,j) (du_ij/dr_ij) (x) r_ij  (each ordered pair),
        background  E_bg I; the self terms do not depend on the cell. Times coulomb_k."""
        pos_t = _t(pos)
        q_t = _t(q)
        mu_t = _t(np.zeros_like(pos) if mu is None else mu).requires_grad_(True)
        rho = self.mesh_density(pos_t, q_t, mu_t)
        E_rec = self.recip_energy(rho)
        (gmu,) = torch.autograd.grad(E_rec, (mu_t,))
        rho_hat = torch.fft.fftn(rho.detach().reshape(self.N)).numpy()
        n = [np.fft.fftfreq(Na) * Na for Na in self.N]
        nx, ny, nz = np.meshgrid(*n, indexing="ij")
        kvec = (nx[..., None] * self.b[0] + ny[..., None] * self.b[1] + nz[..., None] * self.b[2])
        k2 = np.einsum("...c,...c->...", kvec, kvec)
        with np.errstate(divide="ignore", invalid="ignore"):
            wgt = np.where(k2 > 0, self.GC.numpy() * np.abs(rho_hat) ** 2
                           * (1.0 / k2 + 1.0 / (4 * self.alpha ** 2)), 0.0)
        S = np.einsum("xyz,xyza,xyzb->ab", wgt, kvec, kvec)
        W = float(E_rec.detach()) * np.eye(3) - S / self.V + gmu.numpy().T @ mu_t.detach().numpy()
        if self.include_pair:
            i, j, sh = self._pairs(np.asarray(pos, np.float64))
            i, j = torch.as_tensor(i), torch.as_tensor(j)
            r = (pos_t[i] - pos_t[j] + _t(sh)).requires_grad_(True)
            r2 = (r * r).sum(-1)
            B0, B1, B2 = self._bfuncs(r2, self.alpha, 2)
            m = mu_t.detach()
            mir = (m[i] * r).sum(-1)
            mjr = (m[j] * r).sum(-1)
            u = (q_t[i] * q_t[j] * B0 + (q_t[i] * mjr - q_t[j] * mir) * B1
                 + (m[i] * m[j]).sum(-1) * B1 - mir * mjr * B2)
            (du,) = torch.autograd.grad(u.sum(), (r,))
            W = W - 0.5 * (du.T @ r.detach()).numpy()
        if self.include_bg:
            Q = float(q_t.sum())
            W = W - math.pi * Q * Q / (2 * self.V * self.alpha ** 2) * np.eye(3)
        return self.k * W

    # -- public evaluation --------------------------------------------------------------
    def evaluate(self, pos, q, mu, *, field_grad: bool = True, pairs=None):
        """Energy and per-ion derivatives (numpy float64):
        force = -dE/dr, phi = dE/dq, field = -dE/dmu, field_grad = gradient of the field of
        all other sources at each ion (3x3), so that force = q field + field_grad mu."""
        pos_t = _t(pos).requires_grad_(True)
        q_t = _t(q).requires_grad_(True)
        mu_t = _t(np.zeros_like(pos) if mu is None else mu).requires_grad_(True)
        if pairs is None and self.include_pair:
            pairs = self._pairs(np.asarray(pos, np.float64))
        E, parts = self.energy(pos_t, q_t, mu_t, pairs, parts=True)
        gr, gq, gm = torch.autograd.grad(E, (pos_t, q_t, mu_t))
        out = dict(energy=float(E.detach()), force=(-gr).numpy(), phi=gq.numpy(), field=(-gm).numpy())
        out.update({k: float(v.detach()) if torch.is_tensor(v) else float(v) for k, v in parts.items()})
        if field_grad:
            out["field_grad"] = self.field_gradient(np.asarray(pos, np.float64), np.asarray(q, np.float64),
                                                    np.asarray(mu_t.detach().numpy()), pairs)
        return out

    def evaluate_quad(self, pos, q, mu, theta, *, pairs=None):
        """Energy and per-ion derivatives with point quadrupoles theta [n,3,3] (numpy float64):
        force = -dE/dr, phi = dE/dq, field = -dE/dmu, field_grad = -dE/dTheta, the symmetric
        matrix G with dE = -G : dTheta for every symmetric dTheta (it reduces to the field
        gradient of all other sources when theta = 0)."""
        pos_t = _t(pos).requires_grad_(True)
        q_t = _t(q).requires_grad_(True)
        mu_t = _t(np.zeros_like(pos) if mu is None else mu).requires_grad_(True)
        th_t = _t(theta).requires_grad_(True)
        if pairs is None and self.include_pair:
            pairs = self._pairs(np.asarray(pos, np.float64))
        E, parts = self.energy(pos_t, q_t, mu_t, pairs, parts=True, theta=th_t)
        gr, gq, gm, gt = torch.autograd.grad(E, (pos_t, q_t, mu_t, th_t))
        out = dict(energy=float(E.detach()), force=(-gr).numpy(), phi=gq.numpy(),
                   field=(-gm).numpy(), field_grad=(-0.5 * (gt + gt.transpose(1, 2))).numpy())
        out.update({k: float(v.detach()) for k, v in parts.items()})
        return out

    def hvp(self, pos, q, mu, g_energy, g_force, g_phi, g_field, pairs=None):
        """Vector-Jacobian product of (pos, q, mu) -> (E, force, phi, field) with the given
        cotangents, by double backward. Returns (grad_pos, grad_q, grad_mu) as numpy."""
        pos_t = _t(pos).requires_grad_(True)
        q_t = _t(q).requires_grad_(True)
        mu_t = _t(mu).requires_grad_(True)
        if pairs is None and self.include_pair:
            pairs = self._pairs(np.asarray(pos, np.float64))
        E = self.energy(pos_t, q_t, mu_t, pairs)
        gr, gq, gm = torch.autograd.grad(E, (pos_t, q_t, mu_t), create_graph=True)
        L = (float(g_energy) * E - (gr * _t(g_force)).sum() + (gq * _t(g_phi)).sum()
             - (gm * _t(g_field)).sum())
        a, b, c = torch.autograd.grad(L, (pos_t, q_t, mu_t))
        return a.numpy(), b.numpy(), c.numpy()

    def hvp_quad(self, pos, q, mu, theta, g_energy, g_force, g_phi, g_field, pairs=None):
        """The same vector-Jacobian product with point quadrupoles theta [n,3,3] (cotangents on
        E, force, phi and field; none on -dE/dTheta), by double backward. Returns (grad_pos,
        grad_q, grad_mu, grad_theta) as numpy; grad_theta is the symmetric matrix G with
        dL = G : dTheta for symmetric dTheta."""
        pos_t = _t(pos).requires_grad_(True)
        q_t = _t(q).requires_grad_(True)
        mu_t = _t(mu).requires_grad_(True)
        th_t = _t(theta).requires_grad_(True)
        if pairs is None and self.include_pair:
            pairs = self._pairs(np.asarray(pos, np.float64))
        E = self.energy(pos_t, q_t, mu_t, pairs, theta=th_t)
        gr, gq, gm = torch.autograd.grad(E, (pos_t, q_t, mu_t), create_graph=True)
        L = (float(g_energy) * E - (gr * _t(g_force)).sum() + (gq * _t(g_phi)).sum()
             - (gm * _t(g_field)).sum())
        a, b, c, d = torch.autograd.grad(L, (pos_t, q_t, mu_t, th_t))
        return a.numpy(), b.numpy(), c.numpy(), (0.5 * (d + d.transpose(1, 2))).numpy()

    # -- stage-level helpers (per-kernel parity) ------------------------------------------
    def stage_mesh(self, pos, q, mu, theta=None) -> np.ndarray:
        with torch.no_grad():
            th = None if theta is None else _t(theta)
            return self.mesh_density(_t(pos), _t(q), _t(mu), th).reshape(self.N).numpy()

    def stage_solve(self, rho: np.ndarray):
        """Returns (Phi mesh, E_recip) for a given mesh density (no coulomb_k factor)."""
        with torch.no_grad():
            r = _t(rho).reshape(-1)
            return self.potential_mesh(r).numpy(), float(self.recip_energy(r))

    def interpolated_potential(self, probe, Phi):
        """phi(r) = sum_m W(x(r) - m) Phi(m) at probe points (torch, differentiable)."""
        Nx, Ny, Nz = self.N
        (ix, wx, _), (iy, wy, _), (iz, wz, _) = self._stencils(probe)
        flat = (ix[:, :, None, None] * Ny + iy[:, None, :, None]) * Nz + iz[:, None, None, :]
        vals = Phi.reshape(-1)[flat]
        return (vals * wx[:, :, None, None] * wy[:, None, :, None] * wz[:, None, None, :]).sum((1, 2, 3))

    def pair_potential(self, probe, pos, q, mu, pairs):
        """Pair-term potential at probe_i from every (j, shift) partner of i (sources fixed)."""
        i, j, sh = pairs
        i = torch.as_tensor(i)
        j = torch.as_tensor(j)
        r = probe[i] - _t(pos)[j] + _t(sh)
        r2 = (r * r).sum(-1)
        B0, B1 = self._bfuncs(r2, self.alpha, 1)
        contrib = _t(q)[j] * B0 + (_t(mu)[j] * r).sum(-1) * B1
        return torch.zeros(len(pos), dtype=f64).index_add(0, i, contrib)

    def _derivs(self, fn, pos):
        """Per-ion value, gradient and Hessian of a separable probe potential sum."""
        P = _t(pos).requires_grad_(True)
        phi = fn(P)
        g = torch.autograd.grad(phi.sum(), P, create_graph=True)[0]
        H = torch.stack([torch.autograd.grad(g[:, a].sum(), P, retain_graph=True)[0]
                         for a in range(3)], 1)
        return phi.detach().numpy(), g.detach().numpy(), H.detach().numpy()

    def stage_gather(self, pos, Phi):
        """Mesh-interpolated potential, its gradient and Hessian at each ion."""
        Phi_t = _t(Phi)
        return self._derivs(lambda P: self.interpolated_potential(P, Phi_t), pos)

    def stage_pair(self, pos, q, mu, pairs=None):
        """Pair-term energy and potential / gradient / Hessian at each ion (no k factor)."""
        pos = np.asarray(pos, np.float64)
        if pairs is None:
            pairs = self._pairs(pos)
        with torch.no_grad():
            E = float(self.pair_energy(_t(pos), _t(q), _t(mu), pairs))
        phi, g, H = self._derivs(lambda P: self.pair_potential(P, pos, q, mu, pairs), pos)
        return E, phi, g, H

    def field_gradient(self, pos, q, mu, pairs=None):
        """Gradient of the electric field of all other sources at each ion: -Hess(phi) of
        mesh + pair, minus the ion's own screening-cloud term (4 alpha^3/(3 sqrt(pi))) q_i I
        (the counterpart, for the field gradient, of the dipole self term in the field)."""
        with torch.no_grad():
            rho = self.mesh_density(_t(pos), _t(q), _t(mu))
            Phi = self.potential_mesh(rho)
        _, _, H = self.stage_gather(pos, Phi.numpy())
        if self.include_pair:
            _, _, _, Hp = self.stage_pair(pos, q, mu, pairs)
            H = H + Hp
        c_self = 4 * self.alpha ** 3 / (3 * SQRT_PI) if self.include_self else 0.0
        return -self.k * (H + c_self * np.asarray(q)[:, None, None] * np.eye(3)[None])
