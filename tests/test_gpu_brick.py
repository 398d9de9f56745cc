"""Every built brick shape of the spread against the float64 oracle O2, and the brick
autotuner. The brick only changes how the spread's work is cut into CTAs: every shape must
give the oracle's mesh density, energy, forces and backward within the usual bars (spline
orders 4-6, a ragged mesh with an odd order, a triclinic cell, batched frames, the quadrupole
forward). The tuner returns one of the shapes, never slower than the default by its own
timing, and the automatic choice of pme_plan_create is that shape."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_F, TOL_HVP, TOL_MESH, check, check_energy, f32, prepared, relmax, relrmse

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 16), (8, 8, 32), (16, 8, 16), (16, 16, 16), (4, 8, 16)]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


CASES = {
    "nacl4096_p6": lambda: (W.molten_nacl(4096, L=51.0, seed=1001), (64, 64, 64), 6, 0.30, 9.0),
    "ragged_p5": lambda: (W.molten_nacl(1000, seed=77), (27, 30, 25), 5, 0.35, 8.0),
    "rocksalt_p4": lambda: (W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000), (32, 32, 32), 4, 0.30, 10.0),
}


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", list(CASES))
def test_brick_shapes_match_oracle(gb, shape, name):
    fr, mesh, p, a, rc = CASES[name]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max(1024, fr.n), brick=shape)
    o = O2.PMEOracle(fr.box, mesh, p, a, rc)
    check(f"rho {shape} (rel max)", relmax(plan.spread(_c(pos), _c(q), _c(mu)).cpu().numpy(),
                                           o.stage_mesh(pos, q, mu)), TOL_MESH)
    out = plan.forward(_c(pos), _c(q), _c(mu))
    ref = o.evaluate(pos, q, mu, field_grad=False)
    check_energy(out["energy"].item(), ref)
    check(f"force {shape} (rel RMSE)", relrmse(out["force"].cpu().numpy(), ref["force"]), TOL_F)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=5))
    got = plan.backward(_c(pos), _c(q), _c(mu), torch.tensor([0.4], dtype=torch.float64, device="cuda"),
                        _c(gF), _c(gphi), _c(gfield))
    hv = o.hvp(pos, q, mu, 0.4, gF, gphi, gfield)
    for g_, r_ in zip(got, hv):
        check(f"hvp {shape} (rel RMSE)", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
    plan.close()


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_brick_shapes_triclinic_batch_and_quadrupoles(gb, shape):
    # triclinic single frame
    box = np.array([[26.0, 0.0, 0.0], [3.0, 25.0, 0.0], [-2.0, 1.5, 27.0]])
    rng = np.random.default_rng(3)
    fr = W.molten_nacl(512, seed=8)
    pos = f32(rng.uniform(size=(512, 3)) @ box)
    _, q, mu = prepared(fr)
    plan = gb.Plan(box, (24, 24, 25), 6, 0.35, 6.0, max_ions=1024, brick=shape)
    out = plan.forward(_c(pos), _c(q), _c(mu))
    ref = O2.PMEOracle(box, (24, 24, 25), 6, 0.35, 6.0).evaluate(pos, q, mu, field_grad=False)
    check_energy(out["energy"].item(), ref)
    check(f"triclinic force {shape}", relrmse(out["force"].cpu().numpy(), ref["force"]), TOL_F)
    # batched frames with this brick against single-frame plans with the default brick
    specs = W.uneven_frames(n_frames=6, seed=1005)
    frames = [s.frame for s in specs]
    meshes = [gb.mesh_dims(f_.box, s.spacing, rule=1, strategy=1, clamp=(16, 48)) for f_, s in zip(frames, specs)]
    orders = [s.order for s in specs]
    offsets = np.concatenate([[0], np.cumsum([f_.n for f_ in frames])]).astype(np.int64)
    P = np.concatenate([f32(f_.pos) for f_ in frames])
    Q = np.concatenate([f32(f_.q) for f_ in frames])
    MU = np.concatenate([f32(f_.mu) for f_ in frames])
    bp = gb.BatchPlan([f_.box for f_ in frames], meshes, orders, offsets, 0.30, 9.0, brick=shape)
    e_b = bp.forward(_c(P), _c(Q), _c(MU))["energy"].cpu().numpy()
    for f, f_ in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        sp = gb.Plan(f_.box, meshes[f], orders[f], 0.30, 9.0, max_ions=max(f_.n, 64), fft=bp.fft_kind,
                     brick=(8, 8, 16))
        e = sp.forward(_c(P[lo:hi]), _c(Q[lo:hi]), _c(MU[lo:hi]))["energy"].item()
        check(f"batch frame {f} {shape} vs default brick (rel)", abs(e_b[f] - e) / abs(e), 1e-6)
        sp.close()
    bp.close()
    # quadrupole forward
    th = f32(W.quadrupoles(512, 0.1, seed=9))
    th6 = np.stack([th[:, 0, 0], th[:, 1, 1], th[:, 2, 2], th[:, 0, 1], th[:, 0, 2], th[:, 1, 2]], 1)
    fr2 = W.molten_nacl(512, seed=10)
    p2, q2, m2 = prepared(fr2)
    qp = gb.Plan(fr2.box, (24, 24, 24), 6, 0.35, 8.0, max_ions=1024, brick=shape)
    got = qp.forward_quad(_c(p2), _c(q2), _c(m2), _c(th6))
    refq = O2.PMEOracle(fr2.box, (24, 24, 24), 6, 0.35, 8.0).evaluate_quad(p2, q2, m2, th)
    check_energy(got["energy"].item(), refq)
    check(f"quad force {shape}", relrmse(got["force"].cpu().numpy(), refq["force"]), TOL_F)
    qp.close()


def test_unsupported_brick_is_refused(gb):
    fr = W.molten_nacl(512, seed=3)
    with pytest.raises(gb.PMEError) as e:
        gb.Plan(fr.box, (24, 24, 24), 4, 0.3, 9.0, max_ions=1024, brick=(8, 8, 8))
    assert e.value.status == 5


def test_autotuner_on_the_benchmark_frame(gb):
    fr, cfg = W.workload("nacl32k")
    shape, times = gb.autotune_brick(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], fr.n)
    print("[tune]", shape, {k: (None if v is None else round(v, 4)) for k, v in times.items()})
    assert shape in SHAPES
    assert times[(8, 8, 16)] is not None and times[shape] is not None
    assert times[shape] <= times[(8, 8, 16)]
    # the automatic choice of a plan is the tuner's (cached) choice
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    pos, q, mu = prepared(fr)
    r_auto = plan.spread(_c(pos), _c(q), _c(mu))
    fixed = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n, brick=shape)
    assert torch.equal(r_auto, fixed.spread(_c(pos), _c(q), _c(mu)))
    plan.close()
    fixed.close()
