"""Stage-level parity of the CUDA path (through the C ABI) against the FP64 oracle O2:
spread mesh elementwise, solve (potential mesh and reciprocal energy), gather per ion and the
real-space pair term per ion. Ragged brick tails, every spline order, meshes as small as
the order, ions exactly on mesh points and on the box faces."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_E, TOL_MESH, check, check_energy, prepared, relmax, sym6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _frame(n=512, seed=41):
    fr = W.molten_nacl(n, seed=seed)
    pos, q, mu = prepared(fr)
    # edge positions: on a mesh point, on the box faces, just below L
    L = fr.box[0, 0]
    pos[0] = [0.0, 0.0, 0.0]
    pos[1] = [L * (1 - 1e-7), L / 2, L / 3]
    pos[2] = [L * 0.263, L / 5 + 0.01, L / 9 + 0.02]
    return fr.box, np.asarray(np.float32(pos), np.float64), q, mu


def _cuda(*arrs):
    return [torch.tensor(np.asarray(a, np.float32), device="cuda") for a in arrs]


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("mesh", [(30, 27, 45), (16, 16, 16)])
def test_spread_matches_oracle(gb, order, mesh):
    box, pos, q, mu = _frame()
    plan = gb.Plan(box, mesh, order, 0.3, 9.0, max_ions=4096)
    rho = plan.spread(*_cuda(pos, q, mu)).cpu().numpy()
    ref = O2.PMEOracle(box, mesh, order, 0.3, 9.0).stage_mesh(pos, q, mu)
    assert relmax(rho, ref) < TOL_MESH
    # charges alone: the mesh carries the total charge
    rq = plan.spread(*_cuda(pos, q, 0 * mu)).double().sum().item()
    assert abs(rq - q.sum()) < 1e-4


def test_spread_mesh_equal_to_order(gb):
    box, pos, q, mu = _frame(64, seed=3)
    for order, mesh in [(6, (6, 7, 6)), (4, (4, 9, 5))]:
        plan = gb.Plan(box, mesh, order, 0.3, 9.0, max_ions=256)
        rho = plan.spread(*_cuda(pos, q, mu)).cpu().numpy()
        ref = O2.PMEOracle(box, mesh, order, 0.3, 9.0).stage_mesh(pos, q, mu)
        assert relmax(rho, ref) < TOL_MESH


def test_spread_is_bitwise_deterministic_and_permutation_invariant(gb):
    box, pos, q, mu = _frame(4096, seed=8)
    plan = gb.Plan(box, (48, 48, 48), 6, 0.3, 9.0, max_ions=4096)
    a = plan.spread(*_cuda(pos, q, mu))
    b = plan.spread(*_cuda(pos, q, mu))
    assert torch.equal(a, b)
    perm = np.random.default_rng(0).permutation(len(q))
    c = plan.spread(*_cuda(pos[perm], q[perm], mu[perm]))
    assert relmax(c.cpu().numpy(), a.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("order,mesh", [(4, (32, 32, 32)), (6, (30, 27, 45)), (5, (20, 24, 18))])
def test_solve_matches_oracle(gb, order, mesh):
    box, pos, q, mu = _frame()
    o = O2.PMEOracle(box, mesh, order, 0.3, 9.0)
    rho = o.stage_mesh(pos, q, mu)
    Phi_ref, E_ref = o.stage_solve(np.asarray(np.float32(rho), np.float64))
    plan = gb.Plan(box, mesh, order, 0.3, 9.0, max_ions=1024)
    Phi, E = plan.solve(torch.tensor(np.float32(rho), device="cuda"))
    assert relmax(Phi.cpu().numpy(), Phi_ref) < TOL_MESH
    check_energy(E.item(), E_ref, "E_recip")


def test_solve_without_deconvolution(gb):
    box, pos, q, mu = _frame()
    mesh = (24, 24, 24)
    o = O2.PMEOracle(box, mesh, 4, 0.35, 9.0, deconvolution=False)
    rho = np.asarray(np.float32(o.stage_mesh(pos, q, mu)), np.float64)
    Phi_ref, E_ref = o.stage_solve(rho)
    plan = gb.Plan(box, mesh, 4, 0.35, 9.0, deconvolution=False, max_ions=1024)
    Phi, E = plan.solve(torch.tensor(np.float32(rho), device="cuda"))
    assert relmax(Phi.cpu().numpy(), Phi_ref) < TOL_MESH
    check_energy(E.item(), E_ref, "E_recip")


@pytest.mark.parametrize("order", [2, 3, 4, 5, 6, 7])
def test_gather_matches_oracle(gb, order):
    box, pos, q, mu = _frame()
    mesh = (30, 27, 45)
    o = O2.PMEOracle(box, mesh, order, 0.3, 9.0)
    rng = np.random.default_rng(order)
    Phi = np.asarray(np.float32(rng.normal(size=mesh)), np.float64)
    phi, g, H = o.stage_gather(pos, Phi)
    plan = gb.Plan(box, mesh, order, 0.3, 9.0, max_ions=1024)
    out = plan.gather(torch.tensor(np.float32(pos), device="cuda"),
                      torch.tensor(np.float32(Phi), device="cuda")).cpu().numpy()
    assert relmax(out[:, 0], phi) < TOL_MESH
    assert relmax(out[:, 1:4], g) < TOL_MESH
    if order >= 3:   # the Hessian of W is continuous from order 3 on
        assert relmax(out[:, 4:], sym6(H)) < TOL_MESH


@pytest.mark.parametrize("name", ["cells", "images", "triclinic"])
def test_pair_matches_oracle(gb, name):
    if name == "cells":
        fr = W.molten_nacl(1024, seed=5)
        box, rc = fr.box, 9.0
        pos, q, mu = prepared(fr)
    elif name == "images":       # box shorter than 2 rcut: every image inside the cutoff
        fr = W.molten_nacl(64, seed=6)
        box, rc = fr.box, 9.0
        pos, q, mu = prepared(fr)
    else:
        box = np.array([[26.0, 0.0, 0.0], [3.0, 25.0, 0.0], [-2.0, 1.5, 27.0]])
        rng = np.random.default_rng(2)
        fr = W.molten_nacl(512, seed=7)
        pos = np.asarray(np.float32(rng.uniform(size=(512, 3)) @ box), np.float64)
        _, q, mu = prepared(fr)
        rc = 5.0
    o = O2.PMEOracle(box, (16, 16, 16), 4, 0.3, rc)
    E_ref, phi, g, H = o.stage_pair(pos, q, mu)
    plan = gb.Plan(box, (16, 16, 16), 4, 0.3, rc, max_ions=2048)
    out, E = plan.pair(*_cuda(pos, q, mu))
    out = out.cpu().numpy()
    # the pair energy alone (no self term to cancel against) is a sum of per-ion energies of
    # both signs; each is formed from float32 pair terms, so the bar is on their magnitudes,
    # 1/2 sum |q phi| + |mu . grad phi|
    scale = 0.5 * np.sum(np.abs(q * phi) + np.abs(np.einsum("ik,ik->i", mu, g)))
    check("E_pair (err/(1/2 sum |q phi| + |mu.grad phi|))", abs(E.item() - E_ref) / scale, TOL_E)
    assert relmax(out[:, 0], phi) < TOL_MESH
    assert relmax(out[:, 1:4], g) < TOL_MESH
    assert relmax(out[:, 4:], sym6(H)) < TOL_MESH
