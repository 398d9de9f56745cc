"""The power-of-two kernels of the mesh convolution (every axis 64 or 128 points: compile-time
four-step transforms) against the float64 oracle, against the general own transforms and
against cuFFT: the solve on cubic and mixed meshes, forward and backward (with the tangent
spectrum, with and without rho kept from the forward), the virial sums, the P3M table, and a
batch of mixed power-of-two shapes against single-frame plans."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_F, TOL_HVP, TOL_MESH, check, check_energy, f32, prepared, relmax, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


def _frame(n=2048, seed=41, L=None):
    fr = W.molten_nacl(n, seed=seed) if L is None else W.molten_nacl(n, L=L, seed=seed)
    pos, q, mu = prepared(fr)
    return fr, pos, q, mu


@pytest.mark.parametrize("mesh,order", [((128, 128, 128), 6), ((64, 64, 64), 4), ((64, 128, 64), 5),
                                        ((128, 64, 128), 6), ((64, 64, 128), 7)])
def test_p2_solve_matches_oracle_and_general_kernels(gb, mesh, order):
    fr, pos, q, mu = _frame(1024, seed=3)
    o = O2.PMEOracle(fr.box, mesh, order, 0.3, 9.0)
    rho = np.asarray(np.float32(o.stage_mesh(pos, q, mu)), np.float64)
    Phi_ref, E_ref = o.stage_solve(rho)
    res = {}
    for fft, kernels in (("auto", "power-of-two"), ("own-general", "general")):
        plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=1024, fft=fft)
        assert plan.fft_kernels == kernels
        Phi, E = plan.solve(torch.tensor(np.float32(rho), device="cuda"))
        res[fft] = (Phi.cpu().numpy().astype(np.float64), E.item())
        plan.close()
    Phi, E = res["auto"]
    check(f"p2 solve Phi vs oracle {mesh} (rel max)", relmax(Phi, Phi_ref), TOL_MESH)
    check_energy(E, E_ref, "E_recip")
    # the two kernel sets round differently but agree far inside the mesh tolerance
    check(f"p2 vs general Phi {mesh} (rel max)", relmax(Phi, res["own-general"][0]), 2e-6)
    assert abs(E - res["own-general"][1]) < 1e-6 * abs(E)


@pytest.mark.parametrize("mesh,order", [((64, 64, 64), 6), ((128, 64, 128), 5)])
def test_p2_forward_backward_match_cufft_and_oracle(gb, mesh, order):
    fr, pos, q, mu = _frame(2048, seed=5)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=3))
    gE = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    outs = {}
    for fft in ("auto", "cufft"):
        plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft)
        assert plan.fft_kernels == ("power-of-two" if fft == "auto" else "cufft")
        args = (_c(pos), _c(q), _c(mu))
        f = plan.forward(*args, field_grad=True)
        # the backward on the forward's inputs (rho and Phi kept, only the tangent mesh
        # transformed) and on a fresh plan (both meshes transformed) give the same bits
        b = plan.backward(*args, gE, _c(gF), _c(gphi), _c(gfield))
        fresh = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft)
        b2 = fresh.backward(*args, gE, _c(gF), _c(gphi), _c(gfield))
        for x, y in zip(b, b2):
            assert torch.equal(x, y)
        outs[fft] = ({k: v.double().cpu().numpy() for k, v in f.items()}, [x.double().cpu().numpy() for x in b])
        plan.close()
        fresh.close()
    fa, ba = outs["auto"]
    fc, bc = outs["cufft"]
    assert abs(fa["energy"].item() - fc["energy"].item()) < 1e-6 * abs(fc["energy"].item())
    for k in ("force", "phi", "field"):
        check(f"p2 vs cufft {k} {mesh} (rel RMSE)", relrmse(fa[k], fc[k]), 2e-6)
    # the field gradient and the backward carry second and third spline derivatives, whose
    # float32 rounding differs between any two transforms by more: both against the oracle,
    # the power-of-two kernels no less accurate than cuFFT
    o = O2.PMEOracle(fr.box, mesh, order, 0.3, 9.0)
    ref = o.evaluate(pos, q, mu, field_grad=True)
    fg_ref = np.asarray(ref["field_grad"]).reshape(-1, 9)[:, [0, 4, 8, 1, 2, 5]]   # xx yy zz xy xz yz
    e_p2, e_cu = relrmse(fa["field_grad"], fg_ref), relrmse(fc["field_grad"], fg_ref)
    check(f"p2 field_grad vs oracle {mesh} (rel RMSE; cuFFT {e_cu:.2e})", e_p2, min(TOL_F, 1.5 * e_cu + 2e-7))
    check_energy(fa["energy"].item(), ref)
    check(f"p2 force vs oracle {mesh} (rel RMSE)", relrmse(fa["force"], ref["force"]), TOL_F)
    hv = o.hvp(pos, q, mu, 0.7, gF, gphi, gfield)
    for x, y, r in zip(ba, bc, hv):
        e_p2, e_cu = relrmse(x, r), relrmse(y, r)
        check(f"p2 backward vs oracle {mesh} (rel RMSE; cuFFT {e_cu:.2e})", e_p2, min(TOL_HVP, 1.5 * e_cu + 2e-7))


@pytest.mark.parametrize("influence", ["deconvolution", "p3m"])
def test_p2_virial_and_p3m(gb, influence):
    fr, pos, q, mu = _frame(1024, seed=17)
    mesh, order = (64, 64, 64), 5
    res = {}
    for fft in ("auto", "cufft"):
        plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft, influence=influence)
        if influence == "deconvolution":
            out = plan.forward(_c(pos), _c(q), _c(mu), virial=True)
            res[fft] = (out["energy"].item(), out["virial"].double().cpu().numpy())
        else:
            out = plan.forward(_c(pos), _c(q), _c(mu))
            res[fft] = (out["energy"].item(), out["force"].double().cpu().numpy())
        plan.close()
    (ea, va), (ec, vc) = res["auto"], res["cufft"]
    assert abs(ea - ec) < 1e-6 * abs(ec)
    assert relrmse(va, vc) < 2e-6


def test_p2_batch_of_mixed_shapes_matches_single_frames(gb):
    meshes = [(64, 64, 64), (128, 64, 128), (64, 128, 64), (128, 128, 128)]
    orders = [4, 6, 5, 6]
    sizes = [300, 512, 256, 700]
    frames = [W.molten_nacl(n, seed=60 + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    bp = gb.BatchPlan([fr.box for fr in frames], meshes, orders, offsets, 0.3, 9.0)
    assert bp.fft_kernels == "power-of-two"
    out = bp.forward(_c(pos), _c(q), _c(mu))
    n = int(offsets[-1])
    gF, gphi, gfield = (f32(x) for x in W.tangent(n, seed=7))
    gE = torch.tensor(np.full(len(frames), 0.4), device="cuda")
    back = bp.backward(_c(pos), _c(q), _c(mu), gE, _c(gF), _c(gphi), _c(gfield))
    for f in range(len(frames)):
        lo, hi = int(offsets[f]), int(offsets[f + 1])
        sp = gb.Plan(frames[f].box, meshes[f], orders[f], 0.3, 9.0, max_ions=hi - lo)
        assert sp.fft_kernels == "power-of-two"
        so = sp.forward(_c(pos[lo:hi]), _c(q[lo:hi]), _c(mu[lo:hi]))
        sb = sp.backward(_c(pos[lo:hi]), _c(q[lo:hi]), _c(mu[lo:hi]), gE[f:f + 1], _c(gF[lo:hi]),
                         _c(gphi[lo:hi]), _c(gfield[lo:hi]))
        assert abs(out["energy"][f].item() - so["energy"].item()) < 1e-6 * abs(so["energy"].item())
        check(f"p2 batch frame {f} force (rel RMSE)",
              relrmse(out["force"][lo:hi].cpu().numpy(), so["force"].cpu().numpy()), 1e-6)
        for x, y in zip(back, sb):
            check(f"p2 batch frame {f} backward (rel RMSE)",
                  relrmse(x[lo:hi].cpu().numpy(), y.cpu().numpy()), 1e-6)
        sp.close()
    bp.close()
