"""Parity of pme_forward (energy, forces, dE/dq, field, field gradient) against the FP64
oracle O2 on the same mesh, and of the total against explicit Ewald (O1) within the mesh
error the oracle itself shows at that mesh and order."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ewald as O1
from oracle import pme as O2

from gpu_util import TOL_E, TOL_F, check_energy, f32, prepared, relrmse, sym6

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


CASES = {
    # rock-salt 4x4x4, 512 ions, 32^3, p = 4, alpha 0.30, rcut 10: box < 2 rcut + 5 cells,
    # so the pair term loops over periodic images
    "rocksalt512": lambda: (W.rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000),
                            (32, 32, 32), 4, 0.30, 10.0),
    # molten NaCl 4096 ions, 64^3, p = 6, rcut 9: cell-list path
    "nacl4096": lambda: (W.molten_nacl(4096, L=51.0, seed=1001), (64, 64, 64), 6, 0.30, 9.0),
    # small uneven-batch frame: 64 ions, L = 12.7 A, 16^3, p = 4 (every image within rcut)
    "nacl64": lambda: (W.molten_nacl(64, seed=1002), (16, 16, 16), 4, 0.30, 9.0),
    # ragged mesh, odd order, 1000 ions
    "nacl1000_ragged": lambda: (W.molten_nacl(1000, seed=77), (27, 30, 25), 5, 0.35, 8.0),
    # net charge +1 (on the first eight ions): the neutralising background acts
    "nacl512_charged": lambda: (W.with_net_charge(W.molten_nacl(512, seed=1003), 1.0, 8), (32, 32, 32), 6, 0.30, 9.0),
}


def _run(gb, name, **kw):
    fr, mesh, p, a, rc = CASES[name]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=max(1024, len(q)), **kw)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)]
    out = plan.forward(*t, field_grad=True)
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc, **kw).evaluate(pos, q, mu)
    return fr, got, ref, (pos, q, mu)


@pytest.mark.parametrize("name", list(CASES))
def test_forward_matches_plain_pme(gb, name):
    fr, got, ref, _ = _run(gb, name)
    check_energy(got["energy"][0], ref)
    assert relrmse(got["force"], ref["force"]) < TOL_F
    assert relrmse(got["phi"], ref["phi"]) < TOL_F
    assert relrmse(got["field"], ref["field"]) < TOL_F
    assert relrmse(got["field_grad"], sym6(ref["field_grad"])) < TOL_F


def test_forward_options(gb):
    # deconvolution off, gamma = 0.5, no pair term, eV units: each toggles the same way as O2
    for kw in (dict(deconvolution=False), dict(influence_power=0.5), dict(include_pair=False),
               dict(coulomb_k=14.3996454784), dict(include_self=False, include_background=False)):
        fr, got, ref, _ = _run(gb, "nacl1000_ragged", **kw)
        check_energy(got["energy"][0], ref, f"energy {kw}")
        assert relrmse(got["force"], ref["force"]) < TOL_F, kw
        assert relrmse(got["phi"], ref["phi"]) < TOL_F, kw


def test_forward_vs_explicit_ewald(gb):
    # the discretisation error of the GPU against O1 equals the oracle's own to within float32
    fr, got, ref, (pos, q, mu) = _run(gb, "rocksalt512")
    ew = O1.ewald(pos, q, mu, fr.box, 0.30, rcut=10.0)
    e_pme = abs(ref["energy"] - ew["energy"])
    e_gpu = abs(got["energy"][0] - ew["energy"])
    assert e_gpu <= 1.1 * e_pme + TOL_E * abs(ew["energy"])
    f_pme = relrmse(ref["force"], ew["force"])
    f_gpu = relrmse(got["force"], ew["force"])
    assert f_gpu <= 1.1 * f_pme + TOL_F


def test_rocksalt_madelung_on_gpu(gb):
    fr = W.rocksalt(4, 5.64)
    plan = gb.Plan(fr.box, (48, 48, 48), 6, 0.35, 11.0, max_ions=1024)
    out = plan.forward(*[torch.tensor(np.float32(x), device="cuda") for x in (fr.pos, fr.q, fr.mu)])
    ref = -fr.n * 1.74756459463 / (2 * 2.82)
    assert abs(out["energy"].item() - ref) < 2e-5 * abs(ref)
    assert out["force"].abs().max().item() < 1e-4


def test_forward_deterministic_and_host_pointer_path(gb):
    fr, mesh, p, a, rc = CASES["nacl4096"]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=4096)
    t = [torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)]
    o1 = plan.forward(*t, field_grad=True)
    o2 = plan.forward(*t, field_grad=True)
    for k in o1:
        assert torch.equal(o1[k], o2[k]), k
    # host (pinned) buffers through the same C ABI call
    h = [x.cpu().pin_memory() for x in t]
    o3 = plan.forward(*h, field_grad=True)
    for k in o1:
        assert torch.equal(o1[k].cpu(), o3[k]), k
    # pageable host buffers
    o4 = plan.forward(*[x.cpu() for x in t], field_grad=True)
    for k in o1:
        assert torch.equal(o1[k].cpu(), o4[k]), k
    # the caller's pinned output buffers, the forward not synchronised: its outputs are complete
    # once the backward that follows on the same stream has synchronised
    n = len(q)
    fo = {k: torch.empty_like(v.cpu()).pin_memory() for k, v in o1.items()}
    bo = tuple(torch.empty(s, dtype=torch.float32).pin_memory() for s in [(n, 3), (n,), (n, 3)])
    rng = np.random.default_rng(3)
    cot = [torch.tensor(np.float32(rng.normal(size=sh))) for sh in [(n, 3), (n,), (n, 3)]]
    gE = torch.tensor([0.4], dtype=torch.float64)
    ref_b = plan.backward(*t, gE.cuda(), *[c.cuda() for c in cot])
    for _ in range(2):   # the second pair of calls replays the recorded pass graphs
        o5 = plan.forward(*h, field_grad=True, out=fo, sync=False)
        b5 = plan.backward(*h, gE.pin_memory(), *[c.pin_memory() for c in cot], out=bo, sync=True)
        assert all(o5[k] is fo[k] for k in fo) and all(x is y for x, y in zip(b5, bo))
        for k in o1:
            assert torch.equal(o1[k].cpu(), fo[k]), k
        for x, y in zip(ref_b, bo):
            assert torch.equal(x.cpu(), y)
    with pytest.raises(ValueError):
        plan.forward(*h, out={"force": torch.empty((n, 2)).pin_memory()})


def test_charges_only_and_empty(gb):
    fr, mesh, p, a, rc = CASES["nacl1000_ragged"]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    out = plan.forward(torch.tensor(np.float32(pos), device="cuda"),
                       torch.tensor(np.float32(q), device="cuda"), None)
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate(pos, q, 0 * mu)
    check_energy(out["energy"].item(), ref)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    e = plan.forward(torch.zeros((0, 3), device="cuda"), torch.zeros(0, device="cuda"), None)
    assert e["energy"].item() == 0.0


def test_triclinic_cell(gb):
    box = np.array([[24.0, 0.0, 0.0], [4.0, 23.0, 0.0], [-3.0, 2.0, 25.0]])
    rng = np.random.default_rng(12)
    fr = W.molten_nacl(400, seed=12)
    pos = np.asarray(np.float32(rng.uniform(size=(400, 3)) @ box), np.float64)
    _, q, mu = prepared(fr)
    plan = gb.Plan(box, (30, 30, 32), 6, 0.35, 6.0, max_ions=1024)
    out = plan.forward(*[torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)],
                       field_grad=True)
    ref = O2.PMEOracle(box, (30, 30, 32), 6, 0.35, 6.0).evaluate(pos, q, mu)
    check_energy(out["energy"].item(), ref)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    assert relrmse(out["field_grad"].cpu().numpy(), sym6(ref["field_grad"])) < TOL_F


def test_nonfinite_inputs_are_flagged(gb):
    # a NaN position and an infinite charge are wrapped / zeroed on the device (no fault) and
    # reported as PME_ERR_NONFINITE (4) by the next status check; the plan then keeps working
    fr, mesh, p, a, rc = CASES["nacl1000_ragged"]()
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, mesh, p, a, rc, max_ions=1024)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    for bad_pos, bad_q in ((True, False), (False, True)):
        P, Q = np.array(pos), np.array(q)
        if bad_pos:
            P[17, 1] = np.nan
        if bad_q:
            Q[5] = np.inf
        plan.forward(c(P), c(Q), c(mu))
        with pytest.raises(gb.PMEError) as e:
            plan.sync_status()
        assert e.value.status == 4
    out = plan.forward(c(pos), c(q), c(mu))
    plan.sync_status()
    ref = O2.PMEOracle(fr.box, mesh, p, a, rc).evaluate(pos, q, mu, field_grad=False)
    check_energy(out["energy"].item(), ref)


def test_single_ion(gb):
    # one charged dipole in a 12 A box: only its own mesh images and self terms act
    box = np.diag([12.0, 12.0, 12.0])
    pos = np.array([[3.1, 7.7, 5.2]])
    q = np.array([0.8])
    mu = np.array([[0.05, -0.02, 0.04]])
    pos, q, mu = f32(pos), f32(q), f32(mu)
    plan = gb.Plan(box, (16, 16, 16), 6, 0.35, 9.0, max_ions=64)
    out = plan.forward(*[torch.tensor(np.float32(x), device="cuda") for x in (pos, q, mu)])
    ref = O2.PMEOracle(box, (16, 16, 16), 6, 0.35, 9.0).evaluate(pos, q, mu, field_grad=False)
    # a lone ion: the self term removes the mesh self-interaction of its own cloud, so E is
    # what is left of two float64-exact cancelling parts; the bar is on the float32 parts
    check_energy(out["energy"].item(), ref, cancel=True)
    assert relrmse(out["phi"].cpu().numpy(), ref["phi"]) < TOL_F
    # the field of the ion's own images is what remains of its mesh field after the own-cloud
    # term is removed; the float32 rounding that is left comes from the ion's own cloud field
    # at the stencil points the gather sums, 4 alpha^3 / (3 sqrt(pi)) (|mu| + |q| h) within one
    # mesh spacing h, which cancels in the exact result: the bar scales with that
    h = 12.0 / 16
    own = 4 * 0.35 ** 3 / (3 * np.sqrt(np.pi)) * (np.linalg.norm(mu) + abs(q[0]) * h)
    err = np.linalg.norm(out["field"].cpu().numpy() - ref["field"])
    assert err < TOL_F * max(np.linalg.norm(ref["field"]), own)
