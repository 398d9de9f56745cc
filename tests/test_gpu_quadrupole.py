"""Parity of pme_forward_quad (charges, dipoles and point quadrupoles: the rank-2 channel)
against the FP64 oracle O2 with quadrupoles on the same mesh, and of the total against the
explicit Ewald sum with quadrupoles (O1Q) within the mesh error the oracle itself shows."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2
from oracle import quadrupole as O1Q

from gpu_util import TOL_E, TOL_F, TOL_HVP, check, check_energy, f32, prepared, relrmse, sym6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


CASES = {
    # rock-salt 4x4x4, 512 ions, 32^3, p = 4, rcut 10: the pair term loops over images
    "rocksalt512": lambda: (W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000),
                            (32, 32, 32), 4, 0.30, 10.0),
    # molten NaCl 4096 ions, 64^3, p = 6, rcut 9: several pair cells per axis
    "nacl4096": lambda: (W.molten_nacl(4096, L=51.0, seed=1001), (64, 64, 64), 6, 0.30, 9.0),
    # 64 ions in a 12.7 A box: one pair cell per axis, every image inside rcut
    "nacl64": lambda: (W.molten_nacl(64, seed=1002), (16, 16, 16), 4, 0.30, 9.0),
    # ragged mesh, odd order
    "nacl1000_ragged": lambda: (W.molten_nacl(1000, seed=77), (27, 30, 25), 5, 0.35, 8.0),
}


def _inputs(name, sigma=0.1):
    fr, mesh, p, a, rc = CASES[name]()
    pos, q, mu = prepared(fr)
    th = f32(W.quadrupoles(fr.n, sigma, seed=300))
    return fr, mesh, p, a, rc, pos, q, mu, th


def _gpu(gb, fr, mesh, p, a, rc, pos, q, mu, th, **kw):
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max(1024, len(q)), **kw)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu, th)]
    out = plan.forward_quad(*t)
    return plan, {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


@pytest.mark.parametrize("name", list(CASES))
def test_quad_forward_matches_plain_pme(gb, name):
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs(name)
    _, got = _gpu(gb, fr, mesh, p, a, rc, pos, q, mu, th)
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate_quad(pos, q, mu, th)
    check_energy(got["energy"][0], ref)
    assert relrmse(got["force"], ref["force"]) < TOL_F
    assert relrmse(got["phi"], ref["phi"]) < TOL_F
    assert relrmse(got["field"], ref["field"]) < TOL_F
    assert relrmse(got["field_grad"], sym6(ref["field_grad"])) < TOL_F


def test_quad_options(gb):
    # no pair term, no self/background, eV units: each toggles the same way as O2
    base = _inputs("nacl1000_ragged")
    fr, mesh, p, a, rc, pos, q, mu, th = base
    for kw in (dict(include_pair=False), dict(include_self=False, include_background=False),
               dict(coulomb_k=14.3996454784), dict(deconvolution=False)):
        _, got = _gpu(gb, *base, **kw)
        ref = O2.PMEOracle(fr.box, mesh, p, a, rc, **kw).evaluate_quad(pos, q, mu, th)
        check_energy(got["energy"][0], ref, f"energy {kw}")
        assert relrmse(got["force"], ref["force"]) < TOL_F, kw
        assert relrmse(got["field_grad"], sym6(ref["field_grad"])) < TOL_F, kw


def test_quad_vs_explicit_ewald(gb):
    # the GPU's discretisation error against O1Q equals the oracle's own to within float32
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl64")
    _, got = _gpu(gb, fr, (24, 24, 24), 6, a, rc, pos, q, mu, th)
    ref = O2.PMEOracle(fr.box, (24, 24, 24), 6, a, rc).evaluate_quad(pos, q, mu, th)
    ew = O1Q.ewald(pos, q, mu, th, fr.box, a, rcut=rc)
    e_pme = abs(ref["energy"] - ew["energy"])
    assert abs(got["energy"][0] - ew["energy"]) <= 1.1 * e_pme + TOL_E * abs(ew["energy"])
    f_pme = relrmse(ref["force"], ew["force"])
    assert relrmse(got["force"], ew["force"]) <= 1.1 * f_pme + TOL_F
    g_pme = relrmse(sym6(ref["field_grad"]), O1Q.to6(ew["field_grad"]))
    assert relrmse(got["field_grad"], O1Q.to6(ew["field_grad"])) <= 1.1 * g_pme + TOL_F


def test_quad_zero_theta_equals_plain_forward(gb):
    fr, mesh, p, a, rc, pos, q, mu, _ = _inputs("nacl4096")
    plan, got = _gpu(gb, fr, mesh, p, a, rc, pos, q, mu, np.zeros((fr.n, 6)))
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)]
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in plan.forward(*t, field_grad=True).items()}
    assert abs(got["energy"][0] - out["energy"][0]) < 1e-6 * abs(out["energy"][0])
    for k in ("force", "phi", "field", "field_grad"):
        assert relrmse(got[k], out[k]) < 1e-6, k


def test_quad_deterministic_and_host_pointers(gb):
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu, th)]
    o1 = plan.forward_quad(*t)
    o2 = plan.forward_quad(*t)
    for k in o1:
        assert torch.equal(o1[k], o2[k]), k
    o3 = plan.forward_quad(*[x.cpu() for x in t])
    for k in o1:
        assert torch.equal(o1[k].cpu(), o3[k]), k
    # a plain forward and backward after a quadrupole forward recompute from their inputs
    f = plan.forward(*t[:3])
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate(pos, q, mu, field_grad=False)
    assert relrmse(f["force"].cpu().numpy(), ref["force"]) < TOL_F
    gp, gq, gm = plan.backward(*t[:3], g_energy=1.0)
    assert relrmse(-gp.cpu().numpy(), ref["force"]) < TOL_F


def test_quad_refusals(gb):
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl64")
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu, th)]
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024, recip_method="ewald")
    with pytest.raises(gb.PMEError) as e:
        plan.forward_quad(*t)
    assert e.value.status == 5   # PME_ERR_UNSUPPORTED
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    with pytest.raises(gb.PMEError) as e:
        plan.forward_quad(*t[:3], None)
    assert e.value.status == 1   # PME_ERR_ARG


def test_quad_triclinic_cell(gb):
    # a sheared cell: the mesh sees Theta through D^T Theta D, which a transposed D would
    # leave unchanged in a cubic box
    box = np.array([[14.0, 0.0, 0.0], [3.0, 13.5, 0.0], [-2.0, 1.5, 15.0]])
    rng = np.random.default_rng(41)
    n = 96
    pos = f32(rng.uniform(size=(n, 3)) @ box)
    q = rng.normal(size=n)
    q = f32(q - q.mean())
    mu = f32(rng.normal(0, 0.05, size=(n, 3)))
    th = f32(W.quadrupoles(n, 0.1, seed=42))
    mesh, p, a, rc = (28, 27, 30), 6, 0.35, 6.5
    plan = gb.Plan(box, mesh, p, a, rc, max_ions=1024)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu, th)]
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in plan.forward_quad(*t).items()}
    ref = O2.PMEOracle(box, mesh, p, a, rc).evaluate_quad(pos, q, mu, th)
    check_energy(got["energy"][0], ref)
    assert relrmse(got["force"], ref["force"]) < TOL_F
    assert relrmse(got["field_grad"], sym6(ref["field_grad"])) < TOL_F


@pytest.mark.parametrize("order", [1, 2, 3])
def test_quad_low_orders_refused(gb, order):
    # the second spline derivative is discontinuous for p <= 3, so the quadrupole mesh energy
    # is not smooth in r there and the library refuses those orders (PME_ERR_UNSUPPORTED = 5)
    fr, mesh, _, a, rc, pos, q, mu, th = _inputs("nacl64")
    with pytest.raises(gb.PMEError) as e:
        _gpu(gb, fr, mesh, order, a, rc, pos, q, mu, th)
    assert e.value.status == 5


@pytest.mark.parametrize("order", [4, 6])
def test_quad_force_is_energy_gradient(gb, order):
    # the force of pme_forward_quad (with Theta : grad^3 phi) is -dE/dr of its mesh energy: a
    # central difference of the GPU energy along the force direction (the largest change of
    # E per step, far above its float32 rounding), taken between the float32-rounded displaced
    # positions, matches -F . dr. The pair term is off: its cutoff makes the energy jump
    # where a pair crosses rcut, which the oracle's float64 central differences show as well;
    # at p = 4 the force is the gradient away from spline knots (crossings give kinks only)
    fr, mesh, _, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    plan = gb.Plan(fr.box, mesh, order, a, rc, max_ions=1024, include_pair=False)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    F = plan.forward_quad(c(pos), c(q), c(mu), c(th))["force"].double().cpu().numpy()
    d = F / np.sqrt((F ** 2).mean())
    h = 2e-3
    pp, pm = f32(pos + h * d), f32(pos - h * d)
    ep = plan.forward_quad(c(pp), c(q), c(mu), c(th))["energy"].item()
    em = plan.forward_quad(c(pm), c(q), c(mu), c(th))["energy"].item()
    fd = ep - em
    an = -float(np.sum(F * (pp - pm)))
    check(f"FD of E vs -F.dr, p = {order} (rel)", abs(fd - an) / abs(an), 1e-4)


@pytest.mark.parametrize("order", [4, 5, 7])
def test_quad_spline_orders(gb, order):
    fr, mesh, _, a, rc, pos, q, mu, th = _inputs("nacl64")
    _, got = _gpu(gb, fr, mesh, order, a, rc, pos, q, mu, th)
    ref = O2.PMEOracle(fr.box, mesh, order, a, rc).evaluate_quad(pos, q, mu, th)
    check_energy(got["energy"][0], ref)
    assert relrmse(got["force"], ref["force"]) < TOL_F
    assert relrmse(got["field_grad"], sym6(ref["field_grad"])) < TOL_F


def test_quad_energy_autograd(gb):
    # first derivatives of pme_quad_energy are the forward's outputs; the energy is quadratic
    # in (q, mu, Theta), so a central difference along Theta is exact up to rounding
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    th6 = sym6(th)
    t = [torch.tensor(np.float32(x), device="cuda", requires_grad=True) for x in (pos, q, mu, th6)]
    E = gb.pme_quad_energy(plan, *t)
    gpos, gq, gmu, gth = torch.autograd.grad(E, t)
    out = plan.forward_quad(*[x.detach() for x in t])
    assert torch.equal(gpos, -out["force"])
    assert torch.equal(gq, out["phi"])
    rng = np.random.default_rng(43)
    d = torch.tensor(np.float32(rng.normal(size=th6.shape)), device="cuda")
    h = 0.05
    ep = plan.forward_quad(t[0].detach(), t[1].detach(), t[2].detach(), t[3].detach() + h * d)["energy"].item()
    em = plan.forward_quad(t[0].detach(), t[1].detach(), t[2].detach(), t[3].detach() - h * d)["energy"].item()
    fd = (ep - em) / (2 * h)
    ad = float((gth.double() * d.double()).sum())
    assert abs(fd - ad) < 1e-3 * abs(ad) + 2e-5 * abs(E.item()) / h
    # twice differentiable through the forces: a force-matching loss L = sum (F - F0) . w
    # differentiated by autograd equals the oracle's double backward
    F0 = np.float32(np.random.default_rng(3).normal(size=(len(pos), 3)))
    E = gb.pme_quad_energy(plan, *t)
    (gp1,) = torch.autograd.grad(E, t[0], create_graph=True)
    L = ((-gp1 - torch.tensor(F0, device="cuda")) ** 2).sum()
    gg = torch.autograd.grad(L, t)
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).hvp_quad(pos, q, mu, th, 0.0,
                                                        2 * ((-gp1).detach().double().cpu().numpy() - F0),
                                                        np.zeros(len(pos)), np.zeros((len(pos), 3)))
    w6 = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    for g_, r_, nm in zip(gg, (ref[0], ref[1], ref[2], sym6(ref[3]) * w6), ("pos", "q", "mu", "theta")):
        check(f"double backward {nm} (rel RMSE)", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
    # a loss on -dE/dTheta has no second derivative here
    with pytest.raises(RuntimeError):
        gt1 = torch.autograd.grad(gb.pme_quad_energy(plan, *t), t[3], create_graph=True)[0]
        torch.autograd.grad((gt1 ** 2).sum(), t[0])


QB_CASES = ["rocksalt512", "nacl4096", "nacl64", "nacl1000_ragged"]


@pytest.mark.parametrize("name", QB_CASES)
def test_quad_backward_matches_oracle(gb, name):
    # pme_backward_quad: g_E dE + H v in (r, q, mu, Theta) against the oracle's double backward
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs(name)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max(1024, len(q)))
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=17))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    got = plan.backward_quad(c(pos), c(q), c(mu), c(sym6(th)), torch.tensor([0.6], dtype=torch.float64, device="cuda"),
                             c(gF), c(gphi), c(gfield))
    plan.sync_status()
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).hvp_quad(pos, q, mu, th, 0.6, gF, gphi, gfield)
    for g_, r_, nm in zip(got, (ref[0], ref[1], ref[2], sym6(ref[3])), ("pos", "q", "mu", "theta")):
        check(f"hvp_quad {nm} (rel RMSE)", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
    plan.close()


def test_quad_backward_options_triclinic_and_batch(gb):
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    # options: no pair term, eV units, no self / background
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=19))
    for kw in (dict(include_pair=False), dict(coulomb_k=14.3996454784),
               dict(include_self=False, include_background=False)):
        plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024, **kw)
        got = plan.backward_quad(c(pos), c(q), c(mu), c(sym6(th)), torch.tensor([0.3], dtype=torch.float64,
                                                                              device="cuda"),
                                 c(gF), c(gphi), c(gfield))
        ref = O2.PMEOracle(fr.box, mesh, p, a, rc, **kw).hvp_quad(pos, q, mu, th, 0.3, gF, gphi, gfield)
        for g_, r_, nm in zip(got, (ref[0], ref[1], ref[2], sym6(ref[3])), ("pos", "q", "mu", "theta")):
            check(f"hvp_quad {kw} {nm}", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
        plan.close()
    # triclinic cell
    box = np.array([[26.0, 0.0, 0.0], [3.0, 25.0, 0.0], [-2.0, 1.5, 27.0]])
    rng = np.random.default_rng(4)
    f2 = W.molten_nacl(512, seed=9)
    p2 = f32(rng.uniform(size=(512, 3)) @ box)
    _, q2, m2 = prepared(f2)
    t2 = f32(W.quadrupoles(512, 0.1, seed=31))
    g2 = [f32(x) for x in W.tangent(512, seed=21)]
    plan = gb.Plan(box, (24, 24, 25), 6, 0.35, 6.0, max_ions=1024)
    got = plan.backward_quad(c(p2), c(q2), c(m2), c(sym6(t2)), torch.tensor([0.2], dtype=torch.float64, device="cuda"),
                             *[c(x) for x in g2])
    ref = O2.PMEOracle(box, (24, 24, 25), 6, 0.35, 6.0).hvp_quad(p2, q2, m2, t2, 0.2, *g2)
    for g_, r_, nm in zip(got, (ref[0], ref[1], ref[2], sym6(ref[3])), ("pos", "q", "mu", "theta")):
        check(f"hvp_quad triclinic {nm}", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
    plan.close()
    # an uneven batch (orders 4 and 6) against single-frame plans and the oracle
    specs = W.uneven_frames(n_frames=5, seed=1007)
    frames = [sp.frame for sp in specs]
    meshes = [gb.mesh_dims(f_.box, sp.spacing, rule=1, strategy=1, clamp=(16, 48)) for f_, sp in zip(frames, specs)]
    orders = [sp.order for sp in specs]
    offsets = np.concatenate([[0], np.cumsum([f_.n for f_ in frames])]).astype(np.int64)
    P = np.concatenate([f32(f_.pos) for f_ in frames])
    Qv = np.concatenate([f32(f_.q) for f_ in frames])
    MU = np.concatenate([f32(f_.mu) for f_ in frames])
    TH = f32(W.quadrupoles(len(Qv), 0.1, seed=45))
    gFb, gpb, gfb = (f32(x) for x in W.tangent(len(Qv), seed=23))
    gE = np.linspace(0.1, 0.5, len(frames))
    bp = gb.BatchPlan([f_.box for f_ in frames], meshes, orders, offsets, 0.30, 9.0)
    got = bp.backward_quad(c(P), c(Qv), c(MU), c(sym6(TH)), torch.tensor(gE, device="cuda"), c(gFb), c(gpb), c(gfb))
    bp.sync_status()
    for f, f_ in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        ref = O2.PMEOracle(f_.box, meshes[f], orders[f], 0.30, 9.0).hvp_quad(
            P[lo:hi], Qv[lo:hi], MU[lo:hi], TH[lo:hi], gE[f], gFb[lo:hi], gpb[lo:hi], gfb[lo:hi])
        for g_, r_, nm in zip(got, (ref[0], ref[1], ref[2], sym6(ref[3])), ("pos", "q", "mu", "theta")):
            check(f"hvp_quad batch frame {f} {nm}", relrmse(g_[lo:hi].cpu().numpy(), r_), TOL_HVP)
    bp.close()


def test_quad_backward_refusals(gb):
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl64")
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    plan = gb.Plan(fr.box, mesh, 3, a, rc, max_ions=1024)
    with pytest.raises(gb.PMEError) as e:
        plan.backward_quad(c(pos), c(q), c(mu), c(sym6(th)), None, c(pos), c(q), c(mu))
    assert e.value.status == 5
    plan.close()


def test_quad_batch_matches_single_frames(gb):
    specs = W.uneven_frames(n_frames=8, seed=1003)
    frames = [sp.frame for sp in specs]
    meshes = [gb.mesh_dims(fr.box, sp.spacing, rule=1, strategy=1, clamp=(16, 48)) for fr, sp in zip(frames, specs)]
    orders = [sp.order for sp in specs]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    th = sym6(f32(W.quadrupoles(len(q), 0.1, seed=44)))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    bp = gb.BatchPlan([fr.box for fr in frames], meshes, orders, offsets, 0.30, 9.0)
    out = bp.forward_quad(c(pos), c(q), c(mu), c(th))
    for f, fr in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        sp = gb.Plan(fr.box, meshes[f], orders[f], 0.30, 9.0, max_ions=max(fr.n, 64), fft=bp.fft_kind)
        ref = sp.forward_quad(c(pos[lo:hi]), c(q[lo:hi]), c(mu[lo:hi]), c(th[lo:hi]))
        e = ref["energy"].item()
        assert abs(out["energy"][f].item() - e) < 1e-6 * abs(e), f
        for k in ("force", "phi", "field", "field_grad"):
            assert relrmse(out[k][lo:hi].cpu().numpy(), ref[k].cpu().numpy()) < 1e-6, (f, k)
        sp.close()
    # one frame against the oracle
    f = 3
    lo, hi = offsets[f], offsets[f + 1]
    o = O2.PMEOracle(frames[f].box, meshes[f], orders[f], 0.30, 9.0).evaluate_quad(
        pos[lo:hi], q[lo:hi], mu[lo:hi], O1Q.sym_from6(th[lo:hi]))
    # this 310-ion frame has E = 1.6 from E_recip = 31.9 and E_self = -33.8: bar on the
    # float32 parts
    check_energy(out["energy"][f].item(), o, f"energy frame {f}", cancel=True)
    assert relrmse(out["force"][lo:hi].cpu().numpy(), o["force"]) < TOL_F
    assert relrmse(out["field_grad"][lo:hi].cpu().numpy(), sym6(o["field_grad"])) < TOL_F


def test_quad_pair_lists_disabled_and_overflowing(gb):
    # without hit lists (a plan whose lists would exceed 1 GiB) the cell-walking kernel does the
    # pair term; with lists the list-driven one does; a clustered frame overflows the lists and
    # falls back to the cell walk. All agree with each other and with the oracle.
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    outs = []
    for max_ions in (1024, 1 << 18):
        plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max_ions)
        outs.append({k: v.cpu().numpy() for k, v in plan.forward_quad(c(pos), c(q), c(mu), c(th)).items()})
        plan.close()
    assert abs(outs[0]["energy"][0] - outs[1]["energy"][0]) < 1e-6 * abs(outs[1]["energy"][0])
    for k in ("force", "phi", "field", "field_grad"):
        assert relrmse(outs[0][k], outs[1][k]) < 1e-6, k
    rng = np.random.default_rng(45)
    box = np.diag([40.0, 40.0, 40.0])
    pts = []
    while len(pts) < 200:
        x = rng.uniform(-7.0, 7.0, 3)
        if np.linalg.norm(x) < 7.0 and all(np.linalg.norm(x - y) > 1.0 for y in pts):
            pts.append(x)
    pc = f32(20.0 + np.array(pts))
    qc = f32(np.where(np.arange(200) % 2 == 0, 0.5, -0.5))
    muc = f32(rng.normal(0, 0.05, (200, 3)))
    thc = f32(W.quadrupoles(200, 0.1, seed=46))
    plan = gb.Plan(box, (40, 40, 40), 6, 0.30, 9.0, max_ions=1024)
    out = plan.forward_quad(c(pc), c(qc), c(muc), c(thc))
    ref = O2.PMEOracle(box, (40, 40, 40), 6, 0.30, 9.0).evaluate_quad(pc, qc, muc, thc)
    check_energy(out["energy"].item(), ref)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    assert relrmse(out["field_grad"].cpu().numpy(), sym6(ref["field_grad"])) < TOL_F
    plan.close()


def test_quad_empty_and_single_ion(gb):
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl64")
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    e = torch.zeros((0, 3), device="cuda")
    out = plan.forward_quad(e, torch.zeros(0, device="cuda"), e, torch.zeros((0, 6), device="cuda"))
    assert out["energy"].item() == 0.0 and out["force"].shape == (0, 3)
    # one neutral ion carrying only a quadrupole: its energy is the interaction with its own
    # periodic images (mesh + pair) plus the cloud self term
    p1 = np.array([[3.1, 4.7, 5.9]])
    t1 = np.array([[[0.3, 0.05, -0.1], [0.05, -0.2, 0.07], [-0.1, 0.07, 0.15]]])
    z = np.zeros((1, 3))
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    got = plan.forward_quad(c(p1), c(np.zeros(1)), c(z), c(f32(t1)))
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate_quad(f32(p1), np.zeros(1), z, f32(t1))
    # a lone ion: its mesh self-interaction and the cloud self term cancel (see check_energy)
    check_energy(got["energy"].item(), ref, cancel=True)
    assert np.allclose(got["field_grad"].cpu().numpy(), sym6(ref["field_grad"]), rtol=1e-4, atol=1e-6)


def test_quad_nonfinite_theta_is_flagged(gb):
    # a NaN quadrupole is reported as PME_ERR_NONFINITE (4) by the next status check (the
    # kernels index nothing by Theta, so nothing faults); the plan then keeps working
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    bad = np.array(th)
    bad[11, 1, 2] = np.nan
    plan.forward_quad(c(pos), c(q), c(mu), c(bad))
    with pytest.raises(gb.PMEError) as e:
        plan.sync_status()
    assert e.value.status == 4
    out = plan.forward_quad(c(pos), c(q), c(mu), c(th))
    plan.sync_status()
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate_quad(pos, q, mu, th)
    check_energy(out["energy"].item(), ref)


def test_quad_without_dipoles(gb):
    # mu = NULL is the same as zero dipoles, bit for bit
    fr, mesh, p, a, rc, pos, q, mu, th = _inputs("nacl1000_ragged")
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    o1 = plan.forward_quad(c(pos), c(q), None, c(th))
    o2 = plan.forward_quad(c(pos), c(q), c(np.zeros_like(mu)), c(th))
    for k in o1:
        assert torch.equal(o1[k], o2[k]), k
