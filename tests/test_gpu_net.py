"""Parity of the learned charge/dipole network on the GPU (include/gbnet.h) with its float64
oracle O4 (oracle/net.py): the tensor-core channel mixing against a float64 product, the
forward (q, mu, E_sr), the backward (position and parameter gradients), and the gradient of
the force-matching loss of Eq. loss through the model E_sr + E_PME, which the library forms
by forward-over-reverse differentiation with the PME's Hessian-vector product.

Bars. The tensor cores see the activations split into two bfloat16 parts: each element keeps
its value to 2^-18 relative, and the float32 accumulation adds ~K 2^-24; through two layers
and the readouts the outputs are expected within ~1e-5 relative of the float64 oracle that
uses the same bfloat16 weights, and TOL_NET = 5e-5 is held (relative RMSE, max norm for the
mixing). Gradients of the loss involve the PME's second derivatives (float32, ~1e-6) and
the same products: TOL_NET as well."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import net as N

from gpu_util import check, f32, relmax, relrmse

pytestmark = pytest.mark.gpu

TOL_NET = 5e-5


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _bf16_bits(x):
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


@pytest.mark.parametrize("k,nout", [(32, 48), (16, 32), (48, 48), (32, 16), (32, 64), (48, 32), (64, 32)])
def test_mix_matches_float64_product(gb, k, nout):
    from paper_2606_01598_gb300 import net as gnet
    rng = np.random.default_rng(k * 100 + nout)
    M = 1000 + k          # ragged last tile
    X = rng.normal(size=(M, k)).astype(np.float32)
    Wb = _bf16_bits(rng.normal(size=(k, nout)) / np.sqrt(k))
    Wv = (Wb.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    Xt = torch.tensor(X, device="cuda")
    wt = torch.tensor(np.ascontiguousarray(Wb.T).view(np.int16), device="cuda")
    Y, err = gnet.mix(Xt, wt)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = X.astype(np.float64) @ Wv
    check(f"mix {k}x{nout} (rel max)", relmax(Y.cpu().numpy(), ref), 2e-5)
    # accumulate into an existing Y
    Y0 = torch.tensor(rng.normal(size=(M, nout)).astype(np.float32), device="cuda")
    Y1, _ = gnet.mix(Xt, wt, Y0.clone(), accumulate=True)
    check("mix accumulate (rel max)", relmax(Y1.cpu().numpy(), ref + Y0.cpu().numpy()), 2e-5)


def _frames(n_frames, n, seed):
    frames = [W.molten_nacl(n, seed=seed + f) for f in range(n_frames)]
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])])
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    species = np.concatenate([fr.species for fr in frames])
    boxes = np.stack([fr.box for fr in frames])
    return frames, offsets, pos, species, boxes


def _params(seed=5):
    p = W.net_params(seed=seed)
    rng = np.random.default_rng(seed)
    for k in ("bh", "bq", "bE"):
        p[k] = np.asarray(np.float32(rng.normal(0, 0.3, size=p[k].shape)), np.float64)
    return p


@pytest.mark.parametrize("n_frames,n", [(3, 64), (2, 512)])
def test_forward_matches_oracle(gb, n_frames, n):
    frames, offsets, pos, species, boxes = _frames(n_frames, n, 40)
    params = _params()
    net = gb.Net(len(pos), n_frames)
    net.set_frames(offsets, boxes, species)
    net.set_params(params)
    out = net.forward(torch.tensor(np.float32(pos), device="cuda"))
    net.sync_status()
    P = N.to_torch(params)
    q_ref, mu_ref, e_ref = [], [], []
    for f, fr in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        q, mu, e = N.predict(N._t(pos[lo:hi]), fr.species, fr.box, P)
        q_ref.append(q.numpy())
        mu_ref.append(mu.numpy())
        e_ref.append(float(e))
    check("q (rel RMSE)", relrmse(out["q"].cpu().numpy(), np.concatenate(q_ref)), TOL_NET)
    check("mu (rel RMSE)", relrmse(out["mu"].cpu().numpy(), np.concatenate(mu_ref)), TOL_NET)
    check("E_sr (rel max)", relmax(out["e_sr"].cpu().numpy(), np.array(e_ref)), TOL_NET)
    # neutral frames
    qg = out["q"].double().cpu().numpy()
    for f in range(n_frames):
        assert abs(qg[offsets[f]:offsets[f + 1]].sum()) < 1e-4
    net.close()


def test_backward_matches_oracle(gb):
    frames, offsets, pos, species, boxes = _frames(3, 64, 50)
    params = _params(7)
    net = gb.Net(len(pos), 3)
    net.set_frames(offsets, boxes, species)
    net.set_params(params)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    net.forward(c(pos))
    rng = np.random.default_rng(3)
    gq = f32(rng.normal(size=len(pos)))
    gmu = f32(rng.normal(size=(len(pos), 3)))
    gesr = rng.normal(size=3)
    gp, gpar = net.backward(c(gq), c(gmu), torch.tensor(gesr, device="cuda"))
    net.sync_status()
    P = N.to_torch(params, requires_grad=True)
    pos_t = N._t(pos).requires_grad_(True)
    L = 0.0
    for f, fr in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        q, mu, e = N.predict(pos_t[lo:hi], fr.species, fr.box, P)
        L = L + (q * N._t(gq[lo:hi])).sum() + (mu * N._t(gmu[lo:hi])).sum() + gesr[f] * e
    grads = torch.autograd.grad(L, [pos_t] + list(P.values()))
    check("g_pos (rel RMSE)", relrmse(gp.cpu().numpy(), grads[0].numpy()), TOL_NET)
    got = gb.unpack_params(gpar.cpu().numpy())
    for (name, _), g in zip(P.items(), grads[1:]):
        if name == "bq":      # the neutralisation removes bq: its gradient is exactly zero
            assert abs(got[name][0]) < 1e-5
            continue
        check(f"g_{name} (rel RMSE)", relrmse(got[name], g.numpy()), TOL_NET)
    net.close()


def _loss_case(gb, n_frames, n, mesh, order, alpha, rcut, seed):
    frames, offsets, pos, species, boxes = _frames(n_frames, n, seed)
    params = _params(seed)
    rng = np.random.default_rng(seed)
    e_ref = rng.normal(-50.0, 5.0, size=n_frames)
    f_ref = f32(rng.normal(0, 0.3, size=pos.shape))
    net = gb.Net(len(pos), n_frames)
    net.set_frames(offsets, boxes, species)
    net.set_params(params)
    bp = gb.BatchPlan(list(boxes), [mesh] * n_frames, [order] * n_frames, offsets, alpha, rcut)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    loss, force, grad = net.loss_grad(bp, c(pos), torch.tensor(e_ref, device="cuda"), c(f_ref),
                                      lambda_e=0.5, lambda_f=2.0)
    net.sync_status()
    bp.sync_status()
    L, LE, LF, g = N.loss_and_grad([pos[offsets[f]:offsets[f + 1]] for f in range(n_frames)],
                                   [fr.species for fr in frames], list(boxes), list(e_ref),
                                   [f_ref[offsets[f]:offsets[f + 1]] for f in range(n_frames)], params,
                                   lambda_e=0.5, lambda_f=2.0, mesh=mesh, order=order, alpha=alpha, rcut=rcut)
    lg = loss.cpu().numpy()
    # the library reports the weighted parts (they add up to L)
    check("loss (rel)", abs(lg[0] - L) / L, TOL_NET)
    check("loss_E (rel)", abs(lg[1] - 0.5 * LE) / (0.5 * LE), TOL_NET)
    check("loss_F (rel)", abs(lg[2] - 2.0 * LF) / (2.0 * LF), TOL_NET)
    got = gb.unpack_params(grad.cpu().numpy())
    flat_got = np.concatenate([got[k].ravel() for k in g if k != "bq"])
    flat_ref = np.concatenate([g[k].ravel() for k in g if k != "bq"])
    check("dL/dtheta all (rel RMSE)", relrmse(flat_got, flat_ref), TOL_NET)
    for k in g:
        if k != "bq":
            check(f"dL/d{k} (rel RMSE)", relrmse(got[k], g[k]), TOL_NET)
    return net, bp


def test_loss_gradient_matches_oracle_small(gb):
    # three 64-ion frames (12.7 A boxes: the PME pair term loops over images)
    _loss_case(gb, 3, 64, (16, 16, 16), 4, 0.35, 6.0, 60)


def test_loss_gradient_matches_oracle_training_config(gb):
    # the training configuration: 512-ion frames (25.5 A), 32^3 mesh, order 4, alpha 0.30,
    # rcut 9 A; two frames of the batch layout
    _loss_case(gb, 2, 512, (32, 32, 32), 4, 0.30, 9.0, 70)
