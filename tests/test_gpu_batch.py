"""Batched uneven frames (one launch per stage for the whole batch) against the same frames
run one by one through single-frame plans, and spot checks of two frames against the FP64
oracle. Frames follow the uneven-batch recipe: 64-1024 ions at the molten-NaCl density,
mesh spacing 0.8 A rounded to 2,3,5-smooth sizes in [16, 48], orders 4 and 6 alternating."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, TOL_HVP, check_energy, f32, relrmse, sym6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


@pytest.fixture(scope="module")
def batch(gb):
    specs = W.uneven_frames(n_frames=24, seed=1002)
    frames = [s.frame for s in specs]
    meshes = [gb.mesh_dims(fr.box, s.spacing, rule=1, strategy=1, clamp=(16, 48)) for fr, s in zip(frames, specs)]
    orders = [s.order for s in specs]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])]).astype(np.int64)
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    q = np.concatenate([f32(fr.q) for fr in frames])
    mu = np.concatenate([f32(fr.mu) for fr in frames])
    return dict(frames=frames, meshes=meshes, orders=orders, offsets=offsets, pos=pos, q=q, mu=mu)


def _c(x):
    return torch.tensor(np.float32(x), device="cuda")


@pytest.mark.parametrize("fft", ["auto", "cufft"])
def test_batch_forward_matches_single_frames(gb, batch, fft):
    B = batch
    bp = gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0,
                      fft=fft)
    out = bp.forward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]), field_grad=True)
    for f, fr in enumerate(B["frames"]):
        lo, hi = B["offsets"][f], B["offsets"][f + 1]
        sp = gb.Plan(fr.box, B["meshes"][f], B["orders"][f], 0.30, 9.0, max_ions=max(fr.n, 64),
                     fft=bp.fft_kind)   # the batch's transforms: like for like
        ref = sp.forward(_c(B["pos"][lo:hi]), _c(B["q"][lo:hi]), _c(B["mu"][lo:hi]), field_grad=True)
        e = ref["energy"].item()
        assert abs(out["energy"][f].item() - e) < 1e-6 * abs(e), f
        for k in ("force", "phi", "field", "field_grad"):
            assert relrmse(out[k][lo:hi].cpu().numpy(), ref[k].cpu().numpy()) < 1e-6, (f, k)
        sp.close()


def test_batch_backward_matches_single_frames(gb, batch):
    B = batch
    n = int(B["offsets"][-1])
    gF, gphi, gfield = (f32(x) for x in W.tangent(n, seed=21))
    gE = np.linspace(0.1, 0.9, len(B["frames"]))
    bp = gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    got = bp.backward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]), torch.tensor(gE, device="cuda"),
                      _c(gF), _c(gphi), _c(gfield))
    for f, fr in enumerate(B["frames"]):
        lo, hi = B["offsets"][f], B["offsets"][f + 1]
        sp = gb.Plan(fr.box, B["meshes"][f], B["orders"][f], 0.30, 9.0, max_ions=max(fr.n, 64),
                     fft=bp.fft_kind)   # the batch's transforms: like for like
        ref = sp.backward(_c(B["pos"][lo:hi]), _c(B["q"][lo:hi]), _c(B["mu"][lo:hi]),
                          torch.tensor([gE[f]], dtype=torch.float64, device="cuda"),
                          _c(gF[lo:hi]), _c(gphi[lo:hi]), _c(gfield[lo:hi]))
        for g_, r_ in zip(got, ref):
            assert relrmse(g_[lo:hi].cpu().numpy(), r_.cpu().numpy()) < 1e-6, f
        sp.close()


@pytest.mark.parametrize("pick", [0, 1])
def test_batch_frames_match_oracle(gb, batch, pick):
    # one frame of each order against the float64 plain PME
    B = batch
    f = next(i for i, o in enumerate(B["orders"]) if o == (4 if pick == 0 else 6))
    fr = B["frames"][f]
    lo, hi = B["offsets"][f], B["offsets"][f + 1]
    bp = gb.BatchPlan([x.box for x in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    out = bp.forward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]), field_grad=True)
    o = O2.PMEOracle(fr.box, B["meshes"][f], B["orders"][f], 0.30, 9.0)
    ref = o.evaluate(B["pos"][lo:hi], B["q"][lo:hi], B["mu"][lo:hi])
    check_energy(out["energy"][f].item(), ref, f"energy frame {f}")
    assert relrmse(out["force"][lo:hi].cpu().numpy(), ref["force"]) < TOL_F
    assert relrmse(out["field_grad"][lo:hi].cpu().numpy(), sym6(ref["field_grad"])) < TOL_F
    n = hi - lo
    gF, gphi, gfield = (f32(x) for x in W.tangent(int(B["offsets"][-1]), seed=5))
    gE = np.zeros(len(B["frames"]))
    gE[f] = 0.4
    got = bp.backward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]), torch.tensor(gE, device="cuda"),
                      _c(gF), _c(gphi), _c(gfield))
    hv = o.hvp(B["pos"][lo:hi], B["q"][lo:hi], B["mu"][lo:hi], 0.4, gF[lo:hi], gphi[lo:hi], gfield[lo:hi])
    for g_, r_ in zip(got, hv):
        assert relrmse(g_[lo:hi].cpu().numpy(), r_) < TOL_HVP
    assert n > 0


def test_batch_host_pointers_and_rejections(gb, batch):
    B = batch
    bp = gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    d = bp.forward(_c(B["pos"]), _c(B["q"]), _c(B["mu"]))
    h = bp.forward(*(_c(x).cpu().pin_memory() for x in (B["pos"], B["q"], B["mu"])))
    for k in d:
        assert torch.equal(d[k].cpu(), h[k]), k
    # single-frame calls reject a batched plan and vice versa (PME_ERR_ARG = 1)
    pos, q = _c(B["pos"]), _c(B["q"])
    p_ = lambda t: ctypes.c_void_p(t.data_ptr())
    assert bp.lib.pme_forward(bp.handle, None, 10, p_(pos), p_(q), *([None] * 6)) == 1
    sp = gb.Plan(B["frames"][0].box, B["meshes"][0], B["orders"][0], 0.30, 9.0, max_ions=2048)
    assert sp.lib.pme_batch_forward(sp.handle, None, p_(pos), p_(q), *([None] * 6)) == 1
    assert bp.lib.pme_batch_frames(bp.handle) == len(B["frames"])


def test_batch_backward_after_forward_is_bitwise_the_same(gb, batch):
    B = batch
    n = int(B["offsets"][-1])
    gF, gphi, gfield = (f32(x) for x in W.tangent(n, seed=23))
    gE = torch.tensor(np.linspace(0.2, 0.6, len(B["frames"])), device="cuda")
    args = (_c(B["pos"]), _c(B["q"]), _c(B["mu"]), gE, _c(gF), _c(gphi), _c(gfield))
    mk = lambda: gb.BatchPlan([fr.box for fr in B["frames"]], B["meshes"], B["orders"], B["offsets"], 0.30, 9.0)
    bp = mk()
    bp.forward(*args[:3])
    listed = bp.backward(*args)
    fresh = mk().backward(*args)
    for x, y in zip(listed, fresh):
        assert torch.equal(x, y)
