"""Virial (W_ab = -dE/d eps_ab under the homogeneous strain of positions and lattice vectors,
dipoles held fixed) through pme_forward_virial / pme_batch_forward_virial against the float64
plain PME's virial (tests/test_oracle_virial.py pins that one to the strain derivative of its
energy and to the Ewald scaling identity).

Bar: float32 sums, 2e-5 of the largest component (the force bar is 1e-5 RMSE; the virial
adds N pair terms and the k-space sums)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import f32, prepared

pytestmark = pytest.mark.gpu
TOL_W = 2e-5


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


@pytest.mark.parametrize("dipoles", [True, False])
def test_virial_molten_cubic(gb, dipoles):
    fr = W.molten_nacl(512, seed=51)
    pos, q, mu = prepared(fr)
    mu = mu * 3 if dipoles else None
    plan = gb.Plan(fr.box, (32, 32, 32), 6, 0.30, 9.0, max_ions=1024)
    out = plan.forward(_c(pos), _c(q), None if mu is None else _c(mu), virial=True)
    ref = O2.PMEOracle(fr.box, (32, 32, 32), 6, 0.30, 9.0).virial_terms(pos, q, mu)
    assert _rel(out["virial"].cpu().numpy(), ref) < TOL_W
    plain = plan.forward(_c(pos), _c(q), None if mu is None else _c(mu))
    for k in ("energy", "force", "phi", "field"):
        assert torch.equal(out[k], plain[k]), k
    plan.close()


def test_virial_triclinic_and_host_pointers(gb):
    box = np.array([[24.0, 0.0, 0.0], [4.0, 23.0, 0.0], [-3.0, 2.0, 25.0]])
    rng = np.random.default_rng(53)
    fr = W.molten_nacl(400, seed=53)
    pos = f32(rng.uniform(size=(400, 3)) @ box)
    _, q, mu = prepared(fr)
    plan = gb.Plan(box, (30, 30, 32), 6, 0.35, 6.0, max_ions=1024)
    out = plan.forward(torch.tensor(np.float32(pos)), torch.tensor(np.float32(q)),
                       torch.tensor(np.float32(mu)), virial=True)          # host tensors
    ref = O2.PMEOracle(box, (30, 30, 32), 6, 0.35, 6.0).virial_terms(pos, q, mu)
    assert out["virial"].device.type == "cpu"
    assert _rel(out["virial"].numpy(), ref) < TOL_W
    plan.close()


def test_virial_batch_frames(gb):
    specs = W.uneven_frames(n_frames=12, seed=1002)
    frames = [s.frame for s in specs]
    meshes = [gb.mesh_dims(fr.box, s.spacing, rule=1, strategy=1, clamp=(16, 48)) for fr, s in zip(frames, specs)]
    orders = [s.order for s in specs]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    bp = gb.BatchPlan([fr.box for fr in frames], meshes, orders, offsets, 0.30, 9.0)
    out = bp.forward(_c(pos), _c(q), _c(mu), virial=True)
    for f in (0, 5, 11):
        lo, hi = offsets[f], offsets[f + 1]
        ref = O2.PMEOracle(frames[f].box, meshes[f], orders[f], 0.30, 9.0).virial_terms(pos[lo:hi], q[lo:hi], mu[lo:hi])
        assert _rel(out["virial"][f].cpu().numpy(), ref) < TOL_W, f
    bp.close()


def test_virial_needs_pair_lists(gb):
    fr = W.molten_nacl(256, seed=55)
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, (24, 24, 24), 6, 0.30, 9.0, max_ions=1 << 18)   # lists > 1 GiB: none
    with pytest.raises(gb.PMEError) as e:
        plan.forward(_c(pos), _c(q), _c(mu), virial=True)
    assert e.value.status == 5
    plan.close()
