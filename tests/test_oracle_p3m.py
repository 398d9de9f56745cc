"""P3M influence function (an alternative to the paper's sinc deconvolution, which the paper
does not use): the least-squares force-optimal influence function for analytical
differentiation, with alias sums.

Pins: restricted to the m = 0 alias it is the sinc deconvolution exactly; the alias sums have
converged at |m| <= 2; its forces are at least as close to the exact Ewald sum as the
deconvolution's on coarse meshes (it is the optimum of that error over influence functions, in
the mean over positions), and the two differ by little (the deconvolution is close to optimal
for analytical differentiation)."""
import numpy as np
import pytest

import workloads as W
from oracle import ewald as O1
from oracle import pme as O2


def test_p3m_reduces_to_deconvolution_without_aliases():
    fr = W.molten_nacl(64, seed=3)
    a = O2.PMEOracle(fr.box, (16, 18, 20), 4, 0.35, 6.0).GC.numpy()
    b = O2.PMEOracle(fr.box, (16, 18, 20), 4, 0.35, 6.0, influence_kind="p3m", alias_range=0).GC.numpy()
    assert np.abs(a - b).max() < 1e-14 * np.abs(a).max()


@pytest.mark.parametrize("p,tol", [(3, 5e-6), (4, 1e-8), (6, 1e-12)])
def test_p3m_alias_sums_converged(p, tol):
    # |m| <= 2 against |m| <= 4: the tail falls like 1/m^(2p)
    fr = W.molten_nacl(64, seed=3)
    a = O2.PMEOracle(fr.box, (12, 12, 12), p, 0.35, 6.0, influence_kind="p3m", alias_range=2).GC.numpy()
    b = O2.PMEOracle(fr.box, (12, 12, 12), p, 0.35, 6.0, influence_kind="p3m", alias_range=4).GC.numpy()
    assert np.abs(a - b).max() < tol * np.abs(b).max()


@pytest.mark.parametrize("mesh,p", [((12, 12, 12), 3), ((16, 16, 16), 4)])
def test_p3m_forces_no_worse_than_deconvolution(mesh, p):
    errs = {"deconvolution": [], "p3m": []}
    for seed in (21, 22, 23):
        fr = W.molten_nacl(256, seed=seed)
        ref = O1.ewald(fr.pos, fr.q, 0 * fr.mu, fr.box, 0.35, rcut=8.0)
        for kind in errs:
            r = O2.PMEOracle(fr.box, mesh, p, 0.35, 8.0, influence_kind=kind).evaluate(
                fr.pos, fr.q, 0 * fr.mu, field_grad=False)
            errs[kind].append(np.mean((r["force"] - ref["force"]) ** 2))
    e_d, e_p = np.mean(errs["deconvolution"]), np.mean(errs["p3m"])
    assert e_p <= e_d
    assert e_p > 0.95 * e_d
