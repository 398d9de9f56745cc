"""O3: the fixed analytic teacher that labels the learned-charge training frames (test
infrastructure: only tests, the smoke check and the benchmark's CPU leg use it).

The paper trains its charge and dipole heads without direct supervision, from energies and
forces only (Section 2.2), on DFT data that is not available here. The stand-in labels come
from a polarisable point-ion model evaluated with the plain PME oracle O2 (charges, dipoles,
pair term, self and background terms on the same mesh):

* species charges q_i = +1 (Na, species 0) and -1 (Cl, species 1);
* induced dipoles mu_i = a_i E_i with polarisabilities a_Na = 0.15 and a_Cl = 3.0 A^3, where
  E_i = -dE_elec/dmu_i is the field at ion i of all other sources (O2's `field`, which includes
  the dipole self-field term of the Ewald split), solved self-consistently by linear mixing
  mu <- (1 - w) mu + w a E(mu), w = 0.5, until max |a E(mu) - mu| < 1e-10 (float64);
* energy U = E_elec(q, mu*) + sum_i |mu*_i|^2 / (2 a_i), the usual polarisation energy, which
  is stationary in mu at mu* (dU/dmu = -E + mu/a = 0);
* forces F = -dE_elec/dr at fixed mu* (Hellmann-Feynman: stationarity removes the dmu/dr
  terms).

Pins (tests/test_oracle_teacher.py): the self-consistency residual; stationarity of U in mu
(U(mu* + t d) - U(mu*) is quadratic in t); the Hellmann-Feynman forces against central
differences of U with mu re-solved at each displaced geometry; the a -> 0 limit equals plain
fixed-charge PME; and an isolated polarisable pair in a large box against its closed form.
Parity: pinned.
"""
from __future__ import annotations

import numpy as np

from . import pme as O2

POLARISABILITY = (0.15, 3.0)   # A^3: Na (species 0), Cl (species 1)
CHARGE = (1.0, -1.0)


def species_arrays(species, polarisability=POLARISABILITY, charge=CHARGE):
    s = np.asarray(species, np.int64)
    q = np.where(s == 0, charge[0], charge[1]).astype(np.float64)
    a = np.where(s == 0, polarisability[0], polarisability[1]).astype(np.float64)
    return q, a


def solve_dipoles(oracle: O2.PMEOracle, pos, q, a, *, omega: float = 0.5, tol: float = 1e-10,
                  max_iter: int = 2000, pairs=None, mu0=None):
    """Self-consistent induced dipoles mu = a E(mu) by linear mixing. Returns (mu, out, iters)
    with out the oracle's evaluation at the converged dipoles."""
    pos = np.asarray(pos, np.float64)
    if pairs is None and oracle.include_pair:
        pairs = oracle._pairs(pos)
    mu = np.zeros_like(pos) if mu0 is None else np.array(mu0, np.float64)
    a3 = np.asarray(a, np.float64)[:, None]
    for it in range(1, max_iter + 1):
        out = oracle.evaluate(pos, q, mu, field_grad=False, pairs=pairs)
        target = a3 * out["field"]
        res = float(np.abs(target - mu).max()) if len(mu) else 0.0
        if res < tol:
            return mu, out, it
        mu = (1.0 - omega) * mu + omega * target
    raise RuntimeError(f"induced dipoles did not converge (residual {res:.3e})")


def polarisation_energy(mu, a):
    """sum_i |mu_i|^2 / (2 a_i); an ion with a_i = 0 carries no induced dipole and no term."""
    a = np.asarray(a, np.float64)
    m2 = np.sum(np.asarray(mu) ** 2, axis=1)
    pol = a > 0
    return float(np.sum(m2[pol] / (2.0 * a[pol])))


def label(frame, mesh=(32, 32, 32), order: int = 4, alpha: float = 0.30, rcut: float = 9.0,
          polarisability=POLARISABILITY, charge=CHARGE, **solve):
    """Teacher energy, forces and converged dipoles of one frame (float64 numpy):
    dict(energy, force, mu, q, iters)."""
    q, a = species_arrays(frame.species, polarisability, charge)
    o = O2.PMEOracle(frame.box, mesh, order, alpha, rcut)
    mu, out, iters = solve_dipoles(o, frame.pos, q, a, **solve)
    U = out["energy"] + polarisation_energy(mu, a)
    return dict(energy=U, force=out["force"], mu=mu, q=q, iters=iters)
