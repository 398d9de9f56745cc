"""The mesh convolution on the library's own transforms (shared-memory Stockham FFTs, the x
transform fused with the influence multiply) against the float64 oracle and against the
cuFFT path of the same plan: 2,3,5-smooth axes from 3 to 256 points, odd lengths, the
largest plane that fits in shared memory, meshes that fall back to cuFFT, batches of mixed
shapes, the backward's tangent spectra, the virial sums and the P3M table lookup."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, TOL_HVP, TOL_MESH, check_energy, f32, prepared, relmax, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


def _frame(n=512, seed=41):
    fr = W.molten_nacl(n, seed=seed)
    pos, q, mu = prepared(fr)
    return fr, pos, q, mu


@pytest.mark.parametrize("mesh,order,kind", [
    ((8, 8, 8), 4, "own"),
    ((12, 5, 3), 3, "own"),          # odd y and z: an unpaired last row, N_z / 2 + 1 = 2
    ((25, 27, 45), 6, "own"),        # radix 5 and 3 only
    ((16, 18, 20), 5, "own"),
    ((30, 36, 40), 4, "own"),
    ((256, 12, 10), 4, "own"),       # longest x (pass-B tile of 256 rows)
    ((10, 256, 16), 4, "own"),       # longest y
    ((16, 16, 256), 4, "own"),       # longest z
    ((160, 160, 160), 6, "own"),     # the largest cube whose plane fits in shared memory
    ((192, 192, 192), 6, "cufft"),   # plane too large: cuFFT
    ((7, 8, 9), 4, "cufft"),         # 7 is not 2,3,5-smooth
])
def test_solve_matches_oracle(gb, mesh, order, kind):
    fr, pos, q, mu = _frame()
    o = O2.PMEOracle(fr.box, mesh, order, 0.3, 9.0)
    rho = np.asarray(np.float32(o.stage_mesh(pos, q, mu)), np.float64)
    Phi_ref, E_ref = o.stage_solve(rho)
    plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=1024, fft="own" if kind == "own" else "auto")
    assert plan.fft_kind == kind
    Phi, E = plan.solve(torch.tensor(np.float32(rho), device="cuda"))
    assert relmax(Phi.cpu().numpy(), Phi_ref) < TOL_MESH
    check_energy(E.item(), E_ref, "E_recip")
    plan.close()


def test_own_transforms_refused_where_they_do_not_apply(gb):
    fr, pos, q, mu = _frame()
    with pytest.raises(gb.PMEError) as e:
        gb.Plan(fr.box, (7, 8, 9), 4, 0.3, 9.0, max_ions=1024, fft="own")
    assert e.value.status == 5   # PME_ERR_UNSUPPORTED


@pytest.mark.parametrize("mesh,order", [((30, 27, 45), 6), ((48, 40, 36), 4), ((32, 32, 32), 5)])
def test_own_transforms_match_cufft_forward_and_backward(gb, mesh, order):
    fr, pos, q, mu = _frame(2048, seed=5)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=3))
    gE = torch.tensor([0.7], dtype=torch.float64, device="cuda")
    outs = {}
    for fft in ("own", "cufft"):
        plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft)
        assert plan.fft_kind == fft
        f = plan.forward(_c(pos), _c(q), _c(mu), field_grad=True)
        b = plan.backward(_c(pos), _c(q), _c(mu), gE, _c(gF), _c(gphi), _c(gfield))
        outs[fft] = ({k: v.double().cpu().numpy() for k, v in f.items()}, [x.double().cpu().numpy() for x in b])
        plan.close()
    fa, ba = outs["own"]
    fc, bc = outs["cufft"]
    # both paths round in float32; they agree far inside the oracle tolerances
    assert abs(fa["energy"].item() - fc["energy"].item()) < 1e-6 * abs(fc["energy"].item())
    for k in ("force", "phi", "field", "field_grad"):
        assert relrmse(fa[k], fc[k]) < 2e-6, k
    for x, y in zip(ba, bc):
        assert relrmse(x, y) < 2e-6
    # and the own path against the oracle
    o = O2.PMEOracle(fr.box, mesh, order, 0.3, 9.0)
    ref = o.evaluate(pos, q, mu, field_grad=False)
    check_energy(fa["energy"].item(), ref)
    assert relrmse(fa["force"], ref["force"]) < TOL_F
    hv = o.hvp(pos, q, mu, 0.7, gF, gphi, gfield)
    for x, r in zip(ba, hv):
        assert relrmse(x, r) < TOL_HVP


def test_forward_is_bitwise_deterministic(gb):
    fr, pos, q, mu = _frame(4096, seed=8)
    plan = gb.Plan(fr.box, (48, 48, 48), 6, 0.3, 9.0, max_ions=fr.n, fft="own")
    a = plan.forward(_c(pos), _c(q), _c(mu))
    b = plan.forward(_c(pos), _c(q), _c(mu))
    for k in a:
        assert torch.equal(a[k], b[k]), k
    plan.close()


def _batch(gb, meshes, orders, seed=11, fft="auto"):
    sizes = [200, 334, 512, 150][:len(meshes)]
    frames = [W.molten_nacl(n, seed=seed + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    bp = gb.BatchPlan([fr.box for fr in frames], meshes, orders, offsets, 0.3, 9.0, fft=fft)
    return frames, offsets, pos, q, mu, bp


def test_batch_of_mixed_shapes_matches_cufft_and_oracle(gb):
    meshes = [(20, 24, 18), (25, 27, 30), (32, 32, 32), (16, 20, 15)]
    orders = [4, 6, 5, 4]
    res = {}
    for fft in ("own", "cufft"):
        frames, offsets, pos, q, mu, bp = _batch(gb, meshes, orders, fft=fft)
        assert bp.fft_kind == fft
        out = bp.forward(_c(pos), _c(q), _c(mu))
        n = int(offsets[-1])
        gF, gphi, gfield = (f32(x) for x in W.tangent(n, seed=7))
        gE = torch.tensor(np.full(len(frames), 0.4), device="cuda")
        back = bp.backward(_c(pos), _c(q), _c(mu), gE, _c(gF), _c(gphi), _c(gfield))
        res[fft] = (out["energy"].cpu().numpy(), out["force"].cpu().numpy(), [x.cpu().numpy() for x in back])
        bp.close()
    ea, Fa, ba = res["own"]
    ec, Fc, bc = res["cufft"]
    assert np.all(np.abs(ea - ec) < 1e-6 * np.abs(ec))
    assert relrmse(Fa, Fc) < 2e-6
    for x, y in zip(ba, bc):
        assert relrmse(x, y) < 2e-6
    for f in range(len(meshes)):
        lo, hi = offsets[f], offsets[f + 1]
        o = O2.PMEOracle(frames[f].box, meshes[f], orders[f], 0.3, 9.0)
        ref = o.evaluate(pos[lo:hi], q[lo:hi], mu[lo:hi], field_grad=False)
        check_energy(ea[f], ref, f"energy frame {f}")
        assert relrmse(Fa[lo:hi], ref["force"]) < TOL_F, f


def test_batch_with_one_unsupported_mesh_uses_cufft(gb):
    frames, offsets, pos, q, mu, bp = _batch(gb, [(20, 24, 18), (21, 22, 14)], [4, 4])
    assert bp.fft_kind == "cufft"   # 21 = 3 x 7 and 22 = 2 x 11
    out = bp.forward(_c(pos), _c(q), _c(mu))
    o = O2.PMEOracle(frames[1].box, (21, 22, 14), 4, 0.3, 9.0)
    lo, hi = offsets[1], offsets[2]
    ref = o.evaluate(pos[lo:hi], q[lo:hi], mu[lo:hi], field_grad=False)
    check_energy(out["energy"][1].item(), ref)
    bp.close()


@pytest.mark.parametrize("influence", ["deconvolution", "p3m"])
def test_virial_and_p3m_on_own_transforms(gb, influence):
    fr, pos, q, mu = _frame(1024, seed=17)
    mesh, order = (30, 32, 27), 5
    res = {}
    for fft in ("own", "cufft"):
        plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft, influence=influence)
        if influence == "deconvolution":
            out = plan.forward(_c(pos), _c(q), _c(mu), virial=True)
            res[fft] = (out["energy"].item(), out["virial"].double().cpu().numpy())
        else:
            out = plan.forward(_c(pos), _c(q), _c(mu))
            res[fft] = (out["energy"].item(), out["force"].double().cpu().numpy())
        plan.close()
    (ea, va), (ec, vc) = res["own"], res["cufft"]
    assert abs(ea - ec) < 1e-6 * abs(ec)
    assert relrmse(va, vc) < 2e-6


@pytest.mark.parametrize("fft", ["own", "cufft"])
def test_solve_between_forward_and_backward(gb, fft):
    # pme_solve replaces the plan's mesh: a later backward on the forward's inputs must not take
    # the forward's rho (or, on the own transforms, its Phi) as still in place
    fr, pos, q, mu = _frame(1024, seed=29)
    gF, gphi, gfield = (f32(x) for x in W.tangent(fr.n, seed=31))
    gE = torch.tensor([0.6], dtype=torch.float64, device="cuda")
    mesh, order = (32, 30, 36), 5
    args = (_c(pos), _c(q), _c(mu), gE, _c(gF), _c(gphi), _c(gfield))
    fresh = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft)
    ref = fresh.backward(*args)
    plan = gb.Plan(fr.box, mesh, order, 0.3, 9.0, max_ions=fr.n, fft=fft)
    plan.forward(*args[:3])
    rng = np.random.default_rng(2)
    plan.solve(torch.tensor(np.float32(rng.normal(size=mesh)), device="cuda"))
    got = plan.backward(*args)
    for g_, r_ in zip(got, ref):
        assert torch.equal(g_, r_)
    # and the reuse path proper (forward, then backward) gives the same bits
    plan.forward(*args[:3])
    again = plan.backward(*args)
    for g_, r_ in zip(again, ref):
        assert torch.equal(g_, r_)
    plan.close()
    fresh.close()
