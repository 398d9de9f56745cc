"""Parity of the GPU explicit Ewald k-sum (recip_method 'ewald') against the FP64 explicit
Ewald oracle O1 with the same alpha, real-space cutoff and k cutoff."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ewald as O1

from gpu_util import TOL_E, TOL_F, check, check_energy, prepared, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _run(gb, box, pos, q, mu, alpha, rcut, kmax):
    plan = gb.Plan(box, (8, 8, 8), 4, alpha, rcut, recip_method="ewald", ewald_kmax=kmax,
                   max_ions=max(1024, len(q)))
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)]
    out = plan.forward(*t, field_grad=True)
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    ref = O1.ewald(pos, q, mu, box, alpha, rcut=rcut, kmax=kmax)
    return plan, got, ref


def _fg6(H):
    return np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]], 1)


@pytest.mark.parametrize("case", ["rocksalt512", "nacl1000", "triclinic"])
def test_ewald_ksum_matches_oracle(gb, case):
    if case == "rocksalt512":
        fr = W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000)
        box, (pos, q, mu), a, rc, km = fr.box, prepared(fr), 0.30, 10.0, 2.4
    elif case == "nacl1000":
        fr = W.molten_nacl(1000, seed=301)
        box, (pos, q, mu), a, rc, km = fr.box, prepared(fr), 0.35, 8.0, 2.8
    else:
        box = np.array([[21.0, 0.0, 0.0], [3.0, 20.0, 0.0], [-2.0, 1.5, 22.0]])
        rng = np.random.default_rng(5)
        fr = W.molten_nacl(300, seed=302)
        _, q, mu = prepared(fr)
        pos = np.asarray(np.float32(rng.uniform(size=(300, 3)) @ box), np.float64)
        a, rc, km = 0.40, 6.0, 3.0
    plan, got, ref = _run(gb, box, pos, q, mu, a, rc, km)
    check_energy(got["energy"][0], ref)
    assert relrmse(got["force"], ref["force"]) < TOL_F
    assert relrmse(got["phi"], ref["phi"]) < TOL_F
    assert relrmse(got["field"], ref["field"]) < TOL_F
    assert relrmse(got["field_grad"], _fg6(ref["field_grad"])) < TOL_F


def test_ewald_plan_has_no_backward(gb):
    fr = W.molten_nacl(64, seed=303)
    pos, q, mu = (torch.tensor(np.float32(x), device="cuda") for x in prepared(fr))
    plan = gb.Plan(fr.box, (8, 8, 8), 4, 0.3, 6.0, recip_method="ewald", max_ions=256)
    with pytest.raises(gb.PMEError) as e:
        plan.backward(pos, q, mu, None, torch.zeros_like(pos), None, None)
    assert e.value.status == 5


def test_mesh_and_ksum_agree(gb):
    # the same frame through the mesh and the explicit sum: the GPU's mesh-vs-k-sum gap equals
    # the oracle's own O2-vs-O1 gap (the discretisation error) to within float32 rounding
    from oracle import pme as O2
    fr = W.molten_nacl(1024, seed=304)
    pos, q, mu = prepared(fr)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)]
    mesh = gb.Plan(fr.box, (40, 40, 40), 7, 0.30, 9.0, max_ions=1024).forward(*t)
    ks = gb.Plan(fr.box, (8, 8, 8), 4, 0.30, 9.0, recip_method="ewald", ewald_kmax=3.5,
                 max_ions=1024).forward(*t)
    o2 = O2.PMEOracle(fr.box, (40, 40, 40), 7, 0.30, 9.0).evaluate(pos, q, mu, field_grad=False)
    o1 = O1.ewald(pos, q, mu, fr.box, 0.30, rcut=9.0, kmax=3.5)
    # |E| ~ 38 is the remainder of |E_recip| ~ 150 and |E_self| ~ 110 (float64 on both sides):
    # the mesh energy's bar is on the float32 parts E_recip + E_pair
    check_energy(mesh["energy"].item(), o2, "mesh vs plain PME", cancel=True)
    check_energy(ks["energy"].item(), o1, "k-sum vs explicit Ewald")
    gap_gpu = mesh["energy"].item() - ks["energy"].item()
    gap_ref = o2["energy"] - o1["energy"]
    check("gap vs oracle gap (err/(|E_rec|+|E_pair|))",
          abs(gap_gpu - gap_ref) / (abs(o2["e_recip"]) + abs(o2["e_pair"])), 2 * TOL_E)
    fg = relrmse(mesh["force"].cpu().numpy(), ks["force"].cpu().numpy())
    fr_ = relrmse(o2["force"], o1["force"])
    assert abs(fg - fr_) < 0.1 * fr_ + TOL_F
