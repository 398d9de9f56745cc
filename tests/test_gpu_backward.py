"""Parity of pme_backward (the vector-Jacobian product of (pos, q, mu) -> (E, F, phi, field),
i.e. the gradient plus the Hessian-vector product) against O2's double backward, and of the
autograd wrapper (double backward through forces) against the same loss on the oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, TOL_HVP, check_energy, f32, prepared, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


CASES = {
    "nacl512_p6": lambda: (W.molten_nacl(512, seed=201), (32, 32, 32), 6, 0.30, 9.0),
    "nacl64_images_p5": lambda: (W.molten_nacl(64, seed=202), (16, 16, 16), 5, 0.30, 9.0),
    "nacl1000_ragged_p7": lambda: (W.molten_nacl(1000, seed=203), (27, 30, 25), 7, 0.35, 8.0),
    # net charge +1: the background enters the gradient (-pi Q / (V alpha^2) in dE/dq) as well
    # as the Hessian-vector product
    "nacl512_charged_p6": lambda: (W.with_net_charge(W.molten_nacl(512, seed=204), 1.0, 8), (32, 32, 32), 6,
                                   0.30, 9.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("gE", [0.0, 0.7])
def test_backward_matches_double_backward(gb, name, gE):
    fr, mesh, p, a, rc = CASES[name]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, scale=1.0, seed=9))
    o = O2.PMEOracle(fr.box, mesh, p, a, rc)
    ref = o.hvp(pos, q, mu, gE, gF, gphi, gfield)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max(1024, fr.n))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    got = plan.backward(c(pos), c(q), c(mu), torch.tensor([gE], dtype=torch.float64, device="cuda"),
                        c(gF), c(gphi), c(gfield))
    for g, r, what in zip(got, ref, ("grad_pos", "grad_q", "grad_mu")):
        err = relrmse(g.cpu().numpy(), r)
        assert err < TOL_HVP, (what, err)


def test_backward_single_cotangents(gb):
    # each cotangent alone (force, phi, field), so no term hides behind another
    fr, mesh, p, a, rc = CASES["nacl512_p6"]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=11))
    z3, z1 = np.zeros_like(gF), np.zeros_like(gphi)
    o = O2.PMEOracle(fr.box, mesh, p, a, rc)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    for args in ((gF, z1, z3), (z3, gphi, z3), (z3, z1, gfield)):
        ref = o.hvp(pos, q, mu, 0.0, *args)
        got = plan.backward(c(pos), c(q), c(mu), None, *(c(x) for x in args))
        for g, r in zip(got, ref):
            assert relrmse(g.cpu().numpy(), r) < TOL_HVP


def test_backward_energy_only_is_gradient(gb):
    fr, mesh, p, a, rc = CASES["nacl512_p6"]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    fw = plan.forward(c(pos), c(q), c(mu))
    gp, gq, gm = plan.backward(c(pos), c(q), c(mu), torch.tensor([2.0], dtype=torch.float64, device="cuda"))
    assert relrmse(gp.cpu().numpy(), -2 * fw["force"].cpu().numpy()) < 1e-6
    assert relrmse(gq.cpu().numpy(), 2 * fw["phi"].cpu().numpy()) < 1e-6
    assert relrmse(gm.cpu().numpy(), -2 * fw["field"].cpu().numpy()) < 1e-6


def test_autograd_force_matching_double_backward(gb):
    fr, mesh, p, a, rc = CASES["nacl512_p6"]()
    pos, q, mu = prepared(fr)
    Fref = f32(np.random.default_rng(4).normal(0, 0.05, size=(fr.n, 3)))
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)

    def loss_of(pos_t, q_t, mu_t, energy_fn):
        E = energy_fn(pos_t, q_t, mu_t)
        F = -torch.autograd.grad(E, pos_t, create_graph=True)[0]
        return E, ((F - torch.as_tensor(Fref, dtype=F.dtype, device=F.device)) ** 2).sum()

    dev = [torch.tensor(np.float32(x), device="cuda", requires_grad=True) for x in (pos, q, mu)]
    E, L = loss_of(*dev, lambda a_, b_, c_: gb.pme_energy(plan, a_, b_, c_))
    L.backward()
    o = O2.PMEOracle(fr.box, mesh, p, a, rc)
    cpu = [torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (pos, q, mu)]
    pairs = o._pairs(pos)
    E2, L2 = loss_of(*cpu, lambda a_, b_, c_: o.energy(a_, b_, c_, pairs))
    L2.backward()
    assert abs(L.item() - L2.item()) < 1e-4 * abs(L2.item())
    for t_gpu, t_cpu in zip(dev, cpu):
        assert relrmse(t_gpu.grad.cpu().numpy(), t_cpu.grad.numpy()) < TOL_HVP


def test_backward_host_pointer_path(gb):
    fr, mesh, p, a, rc = CASES["nacl64_images_p5"]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=3))
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=256)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    gE = torch.tensor([0.3], dtype=torch.float64)
    d = plan.backward(c(pos), c(q), c(mu), gE.cuda(), c(gF), c(gphi), c(gfield))
    # pinned and pageable host arrays, both staged through the plan's buffers
    h = plan.backward(*(c(x).cpu().pin_memory() for x in (pos, q, mu)), gE.pin_memory(),
                      *(c(x).cpu().pin_memory() for x in (gF, gphi, gfield)))
    for x, y in zip(d, h):
        assert torch.equal(x.cpu(), y)
    pg = plan.backward(*(c(x).cpu() for x in (pos, q, mu)), gE,
                       *(c(x).cpu() for x in (gF, gphi, gfield)))
    for x, y in zip(d, pg):
        assert torch.equal(x.cpu(), y)
    # and the forward the same way
    fd = plan.forward(c(pos), c(q), c(mu))
    for hx in ((c(x).cpu().pin_memory() for x in (pos, q, mu)), (c(x).cpu() for x in (pos, q, mu))):
        fh = plan.forward(*hx)
        for k in fd:
            assert torch.equal(fd[k].cpu(), fh[k]), k


@pytest.mark.parametrize("name", list(CASES))
def test_backward_after_forward_reuses_pair_lists_bitwise(gb, name):
    # a backward on the positions of the plan's last forward evaluates the pair term from the
    # hit lists that forward recorded; it must equal the full cell-list pass bit for bit, and
    # any change of the positions (here one coordinate by one ulp) must fall back to that pass
    fr, mesh, p, a, rc = CASES[name]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, scale=1.0, seed=19))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    gE = torch.tensor([0.4], dtype=torch.float64, device="cuda")
    args = (c(pos), c(q), c(mu), gE, c(gF), c(gphi), c(gfield))
    warm = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    warm.forward(*args[:3])
    listed = warm.backward(*args)
    fresh = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024).backward(*args)
    for x, y in zip(listed, fresh):
        assert torch.equal(x, y)
    pos2 = np.float32(pos).copy()
    pos2[3, 0] = np.nextafter(pos2[3, 0], np.float32(np.inf))
    args2 = (torch.tensor(pos2, device="cuda"),) + args[1:]
    warm.forward(*args[:3])          # lists recorded for the original positions
    moved = warm.backward(*args2)
    fresh2 = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024).backward(*args2)
    for x, y in zip(moved, fresh2):
        assert torch.equal(x, y)
    warm.close()


def test_pair_lists_disabled_and_overflowing_paths(gb):
    # a plan whose lists would need more than 1 GiB has none (fused pass only); a clustered
    # frame overflows the lists sized from the plan's mean density (fused fallback); both give
    # the same forward and backward as the list path, bit for bit, and match the oracle
    fr, mesh, p, a, rc = CASES["nacl512_p6"]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, scale=1.0, seed=29))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    gE = torch.tensor([0.3], dtype=torch.float64, device="cuda")
    args = (c(pos), c(q), c(mu), gE, c(gF), c(gphi), c(gfield))
    outs = []
    for max_ions in (1024, 1 << 18):
        # one brick for both (the automatic choice is tuned per capacity)
        plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max_ions, brick=(8, 8, 16))
        f = plan.forward(*args[:3], field_grad=True)
        b = plan.backward(*args)
        outs.append((f, b))
        plan.close()
    for k in outs[0][0]:
        assert torch.equal(outs[0][0][k], outs[1][0][k]), k
    for x, y in zip(outs[0][1], outs[1][1]):
        assert torch.equal(x, y)
    # 200 ions (at least 1 A apart) inside a 7 A ball in a 40 A box: each has 199 partners
    # against lists sized for the mean density of 1024 ions in that box (160 entries)
    rng = np.random.default_rng(31)
    box = np.diag([40.0, 40.0, 40.0])
    pts = []
    while len(pts) < 200:
        x = rng.uniform(-7.0, 7.0, 3)
        if np.linalg.norm(x) < 7.0 and all(np.linalg.norm(x - y) > 1.0 for y in pts):
            pts.append(x)
    pts = 20.0 + np.array(pts)
    qc = np.where(np.arange(200) % 2 == 0, 0.5, -0.5)
    muc = rng.normal(0, 0.05, (200, 3))
    pc, qc, muc = f32(pts), f32(qc), f32(muc)
    plan = gb.Plan(box, (40, 40, 40), 6, 0.30, 9.0, max_ions=1024)
    out = plan.forward(c(pc), c(qc), c(muc))
    ref = O2.PMEOracle(box, (40, 40, 40), 6, 0.30, 9.0).evaluate(pc, qc, muc, field_grad=False)
    # alternating +-0.5 charges packed in a ball: E is a small remainder of E_recip and E_self
    # (float64 on both sides), so the bar is on the float32 parts
    check_energy(out["energy"].item(), ref, cancel=True)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    gFc, gphic, gfieldc = (f32(x) for x in W.tangent(200, seed=37))
    got = plan.backward(c(pc), c(qc), c(muc), gE, c(gFc), c(gphic), c(gfieldc))
    hv = O2.PMEOracle(box, (40, 40, 40), 6, 0.30, 9.0).hvp(pc, qc, muc, 0.3, gFc, gphic, gfieldc)
    for g_, r_ in zip(got, hv):
        assert relrmse(g_.cpu().numpy(), r_) < TOL_HVP
    plan.close()


def test_backward_reuse_is_invalidated_when_it_must_be(gb):
    # the forward's sort, records and pair lists serve only the first backward on exactly the
    # forward's inputs; every other sequence must give what a fresh plan gives, bit for bit
    fr, mesh, p, a, rc = CASES["nacl1000_ragged_p7"]()
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, scale=1.0, seed=41))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    gE = torch.tensor([0.6], dtype=torch.float64, device="cuda")
    P, Q, MU = c(pos), c(q), c(mu)
    tang = (gE, c(gF), c(gphi), c(gfield))
    fresh = lambda *x: gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024).backward(*x)
    ref = fresh(P, Q, MU, *tang)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    # a second backward after one forward
    plan.forward(P, Q, MU)
    for _ in range(2):
        for x, y in zip(plan.backward(P, Q, MU, *tang), ref):
            assert torch.equal(x, y)
    # the charges changed between forward and backward
    Q2 = Q.clone()
    Q2[7] += 0.125
    plan.forward(P, Q, MU)
    for x, y in zip(plan.backward(P, Q2, MU, *tang), fresh(P, Q2, MU, *tang)):
        assert torch.equal(x, y)
    # a stage call on other positions between forward and backward
    plan.forward(P, Q, MU)
    plan.spread(P.flip(0), Q, MU)
    for x, y in zip(plan.backward(P, Q, MU, *tang), ref):
        assert torch.equal(x, y)
    # dipoles given to the forward, none to the backward
    plan.forward(P, Q, MU)
    for x, y in zip(plan.backward(P, Q, None, *tang), fresh(P, Q, None, *tang)):
        assert torch.equal(x, y)
    plan.close()
