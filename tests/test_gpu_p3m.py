"""P3M influence function (influence='p3m', a table per frame built on the device) against
the float64 plain PME with the same influence function, forward and backward, single frame
and batched; and its forces against the exact Ewald sum next to the deconvolution's."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ewald as O1
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, TOL_HVP, check_energy, f32, prepared, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


@pytest.mark.parametrize("mesh,p", [((24, 24, 24), 4), ((20, 27, 24), 6)])
def test_p3m_matches_oracle(gb, mesh, p):
    fr = W.molten_nacl(512, seed=61)
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, 0.35, 8.0, max_ions=1024, influence="p3m")
    out = plan.forward(_c(pos), _c(q), _c(mu))
    o = O2.PMEOracle(fr.box, mesh, p, 0.35, 8.0, influence_kind="p3m")
    ref = o.evaluate(pos, q, mu, field_grad=False)
    check_energy(out["energy"].item(), ref)
    for k in ("force", "phi", "field"):
        assert relrmse(out[k].cpu().numpy(), ref[k]) < TOL_F, k
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=63))
    got = plan.backward(_c(pos), _c(q), _c(mu), torch.tensor([0.5], dtype=torch.float64, device="cuda"),
                        _c(gF), _c(gphi), _c(gfield))
    hv = o.hvp(pos, q, mu, 0.5, gF, gphi, gfield)
    for g_, r_ in zip(got, hv):
        assert relrmse(g_.cpu().numpy(), r_) < TOL_HVP
    with pytest.raises(gb.PMEError):
        plan.forward(_c(pos), _c(q), _c(mu), virial=True)
    plan.close()


def test_p3m_batch_and_set_box(gb):
    specs = W.uneven_frames(n_frames=6, seed=1002)
    frames = [s.frame for s in specs]
    meshes = [gb.mesh_dims(fr.box, s.spacing, rule=1, strategy=1, clamp=(16, 48)) for fr, s in zip(frames, specs)]
    orders = [s.order for s in specs]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    bp = gb.BatchPlan([fr.box for fr in frames], meshes, orders, offsets, 0.30, 9.0, influence="p3m")
    out = bp.forward(_c(pos), _c(q), _c(mu))
    for f in (0, 3, 5):
        lo, hi = offsets[f], offsets[f + 1]
        ref = O2.PMEOracle(frames[f].box, meshes[f], orders[f], 0.30, 9.0, influence_kind="p3m").evaluate(
            pos[lo:hi], q[lo:hi], mu[lo:hi], field_grad=False)
        assert relrmse(out["force"][lo:hi].cpu().numpy(), ref["force"]) < TOL_F, f
    bp.close()
    # a new box rebuilds the table
    fr = frames[2]
    plan = gb.Plan(fr.box * 1.0, meshes[2], orders[2], 0.30, 9.0, max_ions=1024, influence="p3m")
    box2 = fr.box * 1.05
    plan.set_box(box2)
    lo, hi = offsets[2], offsets[3]
    p2 = pos[lo:hi] * 1.05
    out = plan.forward(_c(p2), _c(q[lo:hi]), _c(mu[lo:hi]))
    ref = O2.PMEOracle(box2, meshes[2], orders[2], 0.30, 9.0, influence_kind="p3m").evaluate(
        p2, q[lo:hi], mu[lo:hi], field_grad=False)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    plan.close()


def test_p3m_force_error_against_ewald(gb):
    # the GPU's P3M and deconvolution forces against the exact Ewald sum (charges, coarse mesh)
    errs = {"deconvolution": [], "p3m": []}
    for seed in (71, 72, 73):
        fr = W.molten_nacl(256, seed=seed)
        pos, q, _ = prepared(fr)
        ref = O1.ewald(pos, q, None, fr.box, 0.35, rcut=8.0)
        for kind in errs:
            plan = gb.Plan(fr.box, (16, 16, 16), 4, 0.35, 8.0, max_ions=1024, influence=kind)
            f = plan.forward(_c(pos), _c(q), None)["force"].cpu().numpy()
            errs[kind].append(np.mean((f - ref["force"]) ** 2))
            plan.close()
    assert np.mean(errs["p3m"]) <= np.mean(errs["deconvolution"])
