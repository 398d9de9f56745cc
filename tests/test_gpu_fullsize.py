"""Full-size parity in the launch configurations the benchmark times, and at 262144 ions.

* The 32768-ion molten-NaCl frame (L = 102 A, 128^3 mesh, order 6, alpha 0.30 / A,
  rcut 9 A) through a default plan (pair term on the plan's second stream), forward and
  backward against the float64 plain PME on the same mesh.
* The 256-frame uneven batch built exactly as the benchmark builds it (64-1024 ions per
  frame, spacing 0.8 A rounded to 2,3,5-smooth meshes in [16, 48], orders 4 and 6), with
  sampled frames against the same oracle, and every frame's energy against a single-frame
  plan.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, TOL_HVP, TOL_MESH, check, check_energy, check_rmse, f32, prepared, relmax, relrmse, sym6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


@pytest.fixture(scope="module")
def frame32k():
    fr, cfg = W.workload("nacl32k")
    return fr, cfg


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


def test_32k_forward_matches_plain_pme(gb, frame32k):
    fr, cfg = frame32k
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    out = plan.forward(_c(pos), _c(q), _c(mu), field_grad=True)
    o = O2.PMEOracle(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"])
    ref = o.evaluate(pos, q, mu)
    # E = -367 is what is left of E_recip = 3194 (float32 mesh work, accurate to ~2e-7 of
    # itself) and E_self = -3567 (float64 on both sides): 1e-6 |E| is below the float32
    # rounding of E_recip alone, so the bar is on the float32 parts E_recip + E_pair
    check_energy(out["energy"].item(), ref, cancel=True)
    for k in ("force", "phi", "field"):
        assert relrmse(out[k].cpu().numpy(), ref[k]) < TOL_F, k
    assert relrmse(out["field_grad"].cpu().numpy(), sym6(ref["field_grad"])) < TOL_F
    plan.close()


def test_32k_backward_matches_double_backward(gb, frame32k):
    fr, cfg = frame32k
    pos, q, mu = prepared(fr)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=99))
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    got = plan.backward(_c(pos), _c(q), _c(mu), torch.tensor([0.5], dtype=torch.float64, device="cuda"),
                        _c(gF), _c(gphi), _c(gfield))
    o = O2.PMEOracle(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"])
    ref = o.hvp(pos, q, mu, 0.5, gF, gphi, gfield)
    for g_, r_ in zip(got, ref):
        assert relrmse(g_.cpu().numpy(), r_) < TOL_HVP
    plan.close()


def test_32k_quad_backward_matches_double_backward(gb, frame32k):
    # the quadrupole backward (pme_backward_quad) at the benchmark configuration, point
    # quadrupoles sigma 0.1 e A^2, against the oracle's double backward with quadrupoles
    fr, cfg = frame32k
    pos, q, mu = prepared(fr)
    th = f32(W.quadrupoles(fr.n, 0.1, seed=300))
    th6 = sym6(th)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=99))
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    got = plan.backward_quad(_c(pos), _c(q), _c(mu), _c(th6), torch.tensor([0.5], dtype=torch.float64, device="cuda"),
                             _c(gF), _c(gphi), _c(gfield))
    plan.sync_status()
    ref = O2.PMEOracle(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"]).hvp_quad(
        pos, q, mu, th, 0.5, gF, gphi, gfield)
    for g_, r_, nm in zip(got, (ref[0], ref[1], ref[2], sym6(ref[3])), ("pos", "q", "mu", "theta")):
        check(f"32k hvp_quad {nm} (rel RMSE)", relrmse(g_.cpu().numpy(), r_), TOL_HVP)
    plan.close()


@pytest.fixture(scope="module")
def batch256(gb):
    specs = W.uneven_frames(n_frames=256, seed=1002)
    frames = [s.frame for s in specs]
    meshes = [gb.mesh_dims(fr.box, s.spacing, rule=1, strategy=1, clamp=(16, 48)) for fr, s in zip(frames, specs)]
    orders = [s.order for s in specs]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    return dict(frames=frames, meshes=meshes, orders=orders, offsets=offsets, pos=pos, q=q, mu=mu)


def test_batch256_sampled_frames_match_oracle(gb, batch256):
    B = batch256
    bp = gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    out = bp.forward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]))
    n = int(B["offsets"][-1])
    gF, gphi, gfield = (f32(x) for x in W.tangent(n, seed=7))
    gE = np.full(len(B["frames"]), 0.3)
    got = bp.backward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]), torch.tensor(gE, device="cuda"),
                      _c(gF), _c(gphi), _c(gfield))
    # the smallest and the largest frame of each order, and two in between
    sizes = np.array([fr.n for fr in B["frames"]])
    picks = set()
    for order in (4, 6):
        idx = [f for f in range(len(B["frames"])) if B["orders"][f] == order]
        idx.sort(key=lambda f: sizes[f])
        picks.update([idx[0], idx[-1], idx[len(idx) // 2]])
    for f in sorted(picks):
        fr = B["frames"][f]
        lo, hi = B["offsets"][f], B["offsets"][f + 1]
        o = O2.PMEOracle(fr.box, B["meshes"][f], B["orders"][f], 0.30, 9.0)
        ref = o.evaluate(B["pos"][lo:hi], B["q"][lo:hi], B["mu"][lo:hi], field_grad=False)
        check_energy(out["energy"][f].item(), ref, f"energy frame {f}")
        assert relrmse(out["force"][lo:hi].cpu().numpy(), ref["force"]) < TOL_F, f
        assert relrmse(out["phi"][lo:hi].cpu().numpy(), ref["phi"]) < TOL_F, f
        hv = o.hvp(B["pos"][lo:hi], B["q"][lo:hi], B["mu"][lo:hi], 0.3, gF[lo:hi], gphi[lo:hi], gfield[lo:hi])
        for g_, r_ in zip(got, hv):
            assert relrmse(g_[lo:hi].cpu().numpy(), r_) < TOL_HVP, f
    bp.close()


def test_batch256_energies_match_single_frame_plans(gb, batch256):
    B = batch256
    bp = gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    e_b = bp.forward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]))["energy"].cpu().numpy()
    for f, fr in enumerate(B["frames"]):
        lo, hi = B["offsets"][f], B["offsets"][f + 1]
        sp = gb.Plan(fr.box, B["meshes"][f], B["orders"][f], 0.30, 9.0, max_ions=max(fr.n, 64),
                     fft=bp.fft_kind)   # the batch's transforms: like for like
        e = sp.forward(_c(B["pos"][lo:hi]), _c(B["q"][lo:hi]), _c(B["mu"][lo:hi]))["energy"].item()
        assert abs(e_b[f] - e) < 1e-6 * abs(e), f
        sp.close()
    bp.close()


# ---- the 262144-ion frame (L = 204 A, 256^3, p = 6): the mesh stages over the whole mesh,
# the gather and the pair term at sampled ions, and the backward through properties that
# hold at any size (a Hessian is symmetric; the energy-only cotangent gives the gradient) ----

@pytest.fixture(scope="module")
def frame262k():
    fr, cfg = W.workload("nacl262k")
    pos, q, mu = prepared(fr)
    return fr, cfg, pos, q, mu


def _sampled_pairs(pos, L, rcut, sample):
    """(i, j, shift) of every partner j within rcut of each sampled ion i (minimum image:
    rcut < L / 2), in the oracle's pair convention r_ij = pos_i - pos_j + shift."""
    I, J, S = [], [], []
    for i in sample:
        d = pos[i] - pos
        sh = -L * np.round(d / L)
        r2 = ((d + sh) ** 2).sum(1)
        js = np.nonzero((r2 < rcut * rcut) & (np.arange(len(pos)) != i))[0]
        I.append(np.full(len(js), i))
        J.append(js)
        S.append(sh[js])
    return np.concatenate(I), np.concatenate(J), np.concatenate(S)


def test_262k_mesh_stages_match_oracle(gb, frame262k):
    fr, cfg, pos, q, mu = frame262k
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    o = O2.PMEOracle(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"])
    # spread over the whole mesh
    rho = plan.spread(_c(pos), _c(q), _c(mu)).cpu().numpy()
    rho_ref = o.stage_mesh(pos, q, mu)
    assert relmax(rho, rho_ref) < TOL_MESH
    # solve over the whole mesh, from the same (float32) density
    rho32 = np.asarray(np.float32(rho_ref), np.float64)
    Phi_ref, E_ref = o.stage_solve(rho32)
    Phi, E = plan.solve(torch.tensor(np.float32(rho_ref), device="cuda"))
    assert relmax(Phi.cpu().numpy(), Phi_ref) < TOL_MESH
    check_energy(E.item(), E_ref, "E_recip")
    # gather of that potential at sampled ions
    sample = np.random.default_rng(7).choice(fr.n, 64, replace=False)
    out = plan.gather(_c(pos), torch.tensor(np.float32(Phi_ref), device="cuda")).cpu().numpy()[sample]
    phi, g, H = o.stage_gather(pos[sample], np.asarray(np.float32(Phi_ref), np.float64))
    assert relmax(out[:, 0], phi) < TOL_MESH
    assert relmax(out[:, 1:4], g) < TOL_MESH
    # second-derivative spline weights are differences of three B-spline values, so their
    # float32 rounding, relative to the Hessian of a smooth potential, is about twice that of
    # the potential and gradient: the mesh Hessian is held to twice the mesh bar
    check("262k gathered Hessian (rel max)", relmax(out[:, 4:10], sym6(H)), 2 * TOL_MESH)
    plan.close()


def test_262k_pair_term_at_sampled_ions(gb, frame262k):
    fr, cfg, pos, q, mu = frame262k
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=fr.n)
    out, _ = plan.pair(_c(pos), _c(q), _c(mu))
    sample = np.random.default_rng(8).choice(fr.n, 48, replace=False)
    o = O2.PMEOracle(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"])
    pairs = _sampled_pairs(pos, fr.box[0, 0], cfg["rcut"], sample)
    phi, g, H = o._derivs(lambda P: o.pair_potential(P, pos, q, mu, pairs), pos)
    got = out.cpu().numpy()[sample]
    assert relmax(got[:, 0], phi[sample]) < TOL_MESH
    assert relmax(got[:, 1:4], g[sample]) < TOL_MESH
    assert relmax(got[:, 4:10], sym6(H[sample])) < TOL_MESH
    plan.close()


def test_262k_backward_properties(gb, frame262k):
    fr, cfg, pos, q, mu = frame262k
    n = fr.n
    plan = gb.Plan(fr.box, cfg["mesh"], cfg["order"], cfg["alpha"], cfg["rcut"], max_ions=n)
    P, Q, MU = _c(pos), _c(q), _c(mu)
    zero3, zero1 = torch.zeros((n, 3), device="cuda"), torch.zeros(n, device="cuda")
    f64 = lambda x: torch.tensor([x], dtype=torch.float64, device="cuda")
    # energy-only cotangent: the gradient of E, i.e. (-force, phi, -field) of the forward
    fw = plan.forward(P, Q, MU)
    gp, gq, gm = plan.backward(P, Q, MU, f64(1.0), zero3, zero1, zero3)
    assert relrmse(gp.cpu().numpy(), -fw["force"].cpu().numpy()) < 1e-6
    assert relrmse(gq.cpu().numpy(), fw["phi"].cpu().numpy()) < 1e-6
    assert relrmse(gm.cpu().numpy(), -fw["field"].cpu().numpy()) < 1e-6
    # force cotangents v and w: grad_pos = -H v; the Hessian of E is symmetric, so
    # w . (H v) = v . (H w)
    rng = np.random.default_rng(9)
    v = torch.tensor(np.float32(rng.normal(size=(n, 3))), device="cuda")
    w = torch.tensor(np.float32(rng.normal(size=(n, 3))), device="cuda")
    Hv = plan.backward(P, Q, MU, f64(0.0), v, zero1, zero3)[0].double()
    Hw = plan.backward(P, Q, MU, f64(0.0), w, zero1, zero3)[0].double()
    a = float((w.double() * Hv).sum())
    b = float((v.double() * Hw).sum())
    scale = float(w.double().norm() * Hv.norm())
    assert abs(a - b) < 1e-5 * scale
    plan.close()
