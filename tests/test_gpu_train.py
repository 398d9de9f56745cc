"""Training the learned charge/dipole network through the differentiable PME on the GPU, on
energies and forces of the polarisable teacher O3 (oracle/teacher.py): species charges +-1 and
self-consistent induced dipoles mu = a E, labelled by the plain float64 PME.

* The batched gradient (one launch per stage for all frames) equals the sum of per-frame
  gradients (the plain per-frame form), so both train identically.
* Training lowers the loss.
* What the trained network gains: on held-out teacher frames its forces are closer to the
  teacher's than those of plain fixed-charge PME (species charges +-1, no dipoles), the
  method without the learned part. The numbers are printed and, when GBPME_TRAIN_LOG names a
  file, written there as one JSON line."""
import json
import multiprocessing as mp
import os
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest
import torch

import workloads as W

from gpu_util import f32, relrmse

pytestmark = pytest.mark.gpu

PME = dict(mesh=(32, 32, 32), order=4, alpha=0.30, rcut=9.0)   # the training configuration


def _label(args):
    n, seed = args
    torch.set_num_threads(1)
    from oracle import teacher as T
    fr = W.molten_nacl(n, seed=seed)
    lab = T.label(fr, **PME)
    return seed, lab["energy"], lab["force"]


@pytest.fixture(scope="module")
def labelled():
    """Teacher labels of 512-ion molten-NaCl frames: 16 for training, 4 held out. Labelled in
    a spawned process pool (the oracle is float64 CPU work)."""
    seeds = [1003000 + f for f in range(20)]
    with ProcessPoolExecutor(max_workers=min(20, os.cpu_count() or 4),
                             mp_context=mp.get_context("spawn")) as ex:
        out = list(ex.map(_label, [(512, s) for s in seeds]))
    frames = [W.molten_nacl(512, seed=s) for s in seeds]
    return frames, [o[1] for o in out], [o[2] for o in out]


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _batch(gb, frames):
    offsets = np.concatenate([[0], np.cumsum([fr.n for fr in frames])])
    pos = np.concatenate([f32(fr.pos) for fr in frames])
    species = np.concatenate([fr.species for fr in frames])
    boxes = np.stack([fr.box for fr in frames])
    return offsets, pos, species, boxes


def _setup(gb, frames, params):
    offsets, pos, species, boxes = _batch(gb, frames)
    net = gb.Net(len(pos), len(frames))
    net.set_frames(offsets, boxes, species)
    net.set_params(params)
    bp = gb.BatchPlan(list(boxes), [PME["mesh"]] * len(frames), [PME["order"]] * len(frames), offsets,
                      PME["alpha"], PME["rcut"])
    return net, bp, offsets, pos


def test_batched_gradient_equals_per_frame_sum(gb):
    frames = [W.molten_nacl(512, seed=900 + f) for f in range(4)]
    params = W.net_params(seed=3)
    rng = np.random.default_rng(1)
    e_ref = rng.normal(-80, 5, size=4)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    net, bp, offsets, pos = _setup(gb, frames, params)
    f_ref = f32(rng.normal(0, 0.2, size=pos.shape))
    _, _, g_batch = net.loss_grad(bp, c(pos), torch.tensor(e_ref, device="cuda"), c(f_ref), 0.3, 1.0)
    # per frame: lambda_e / F and lambda_f N_b / sum N reproduce the batch normalisation
    ntot = len(pos)
    g_sum = torch.zeros_like(g_batch)
    for f, fr in enumerate(frames):
        lo, hi = offsets[f], offsets[f + 1]
        n1, b1, _, p1 = _setup(gb, [fr], params)
        n1.loss_grad(b1, c(pos[lo:hi]), torch.tensor(e_ref[f:f + 1], device="cuda"), c(f_ref[lo:hi]),
                     0.3 / len(frames), 1.0 * fr.n / ntot, grad=g_sum, accumulate=True)
        n1.close()
        b1.close()
    err = relrmse(g_sum.cpu().numpy(), g_batch.cpu().numpy())
    assert err < 1e-5, err
    net.close()
    bp.close()


def _force_rmse(pred, ref):
    return float(np.sqrt(np.mean((np.asarray(pred) - np.asarray(ref)) ** 2)))


def test_training_beats_fixed_charge_pme(gb, labelled):
    frames, energies, forces = labelled
    train, val = frames[:16], frames[16:]
    e_tr, f_tr = np.array(energies[:16]), np.concatenate(forces[:16])
    e_va, f_va = np.array(energies[16:]), np.concatenate(forces[16:])
    params = W.net_params(seed=2024)
    net, bp, offsets, pos = _setup(gb, train, params)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    P, E_r, F_r = c(pos), torch.tensor(e_tr, device="cuda"), c(f_tr)
    steps, lr0 = 1500, 3e-3
    losses = []
    t0 = time.time()
    for k in range(steps):
        lr = lr0 * (0.02 ** (k / steps))
        loss = net.train_step(bp, P, E_r, F_r, lambda_e=1.0, lambda_f=1.0, lr=lr)
        if k % 50 == 0 or k == steps - 1:
            losses.append(loss.cpu().numpy().tolist())
    torch.cuda.synchronize()
    t_train = time.time() - t0
    net.sync_status()
    assert losses[-1][0] < 0.2 * losses[0][0], losses
    # held-out frames: the trained network's forces (through q(r), mu(r), E_sr) ...
    vnet, vbp, voff, vpos = _setup(gb, val, net.get_params().cpu().numpy())
    zero_e = torch.zeros(len(val), dtype=torch.float64, device="cuda")
    _, f_learn, _ = vnet.loss_grad(vbp, c(vpos), zero_e, c(f_va), 1.0, 1.0)
    rmse_learn = _force_rmse(f_learn.cpu().numpy(), f_va)
    # ... against plain fixed-charge PME with the teacher's species charges and no dipoles
    species = np.concatenate([fr.species for fr in val])
    q_fix = np.where(species == 0, 1.0, -1.0)
    out = vbp.forward(c(vpos), c(q_fix), torch.zeros((len(vpos), 3), device="cuda"))
    rmse_fixed = _force_rmse(out["force"].cpu().numpy(), f_va)
    rms_teacher = float(np.sqrt(np.mean(f_va ** 2)))
    res = dict(frames_train=len(train), frames_val=len(val), ions_per_frame=512, steps=steps,
               train_seconds=t_train, loss_first=losses[0], loss_last=losses[-1],
               force_rmse_learned=rmse_learn, force_rmse_fixed_charge=rmse_fixed,
               teacher_force_rms=rms_teacher)
    print("[train]", json.dumps(res))
    path = os.environ.get("GBPME_TRAIN_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(res) + "\n")
    assert rmse_learn < rmse_fixed, res
