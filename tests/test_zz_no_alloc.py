"""GPU test of pme_spread_noalloc, the allocation-free spread for callers that cannot call
cudaMalloc (a host framework that has reserved the whole device for its own pool, or a loop
that must not allocate because allocation can synchronise the device).

It is called through the C ABI several times in a row -- on different inputs, so later calls
also show that the shared static scratch carries nothing over -- and each result must equal
pme_spread of a plan with the same box, mesh, order and brick (8 x 8 x 16) bit for bit (the
header promises the same kernels in the same order), and match the float64 oracle's mesh
density within the mesh tolerance of the other parity tests. The largest case fills the fixed scratch: 32768 ions on a
128^3 mesh (the largest candidate-brick table). A NaN input is reported through the optional
device status word. Sizes beyond the fixed scratch must be rejected. The file name makes pytest
collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_MESH, check, prepared, relmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _noalloc(lib, box, mesh, order, pos, q, mu, rho, status=None):
    b = (ctypes.c_double * 9)(*np.asarray(box, np.float64).reshape(9))
    m = (ctypes.c_int * 3)(*mesh)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return lib.pme_spread_noalloc(stream, b, m, order, int(pos.shape[0]), ptr(pos), ptr(q),
                                  ptr(mu), ptr(rho), ptr(status))


def test_noalloc_spread_equals_plan_spread_in_a_row(gb):
    lib = gb.load_library()
    fr32k, cfg = W.workload("nacl32k")
    cases = [
        (W.molten_nacl(4096, L=51.0, seed=1001), (64, 64, 64), 6),
        (W.molten_nacl(1000, seed=77), (27, 30, 25), 5),
        (fr32k, tuple(cfg["mesh"]), cfg["order"]),   # the scratch's limits: 32768 ions, 128^3
    ]
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for fr, mesh, order in cases:   # calls in a row on the shared scratch
        pos64, q64, mu64 = prepared(fr)
        pos, q, mu = (torch.tensor(np.float32(x), device="cuda") for x in (pos64, q64, mu64))
        plan = gb.Plan(fr.box, mesh, order, 0.30, 9.0, max_ions=max(4096, fr.n), brick=(8, 8, 16))
        ref = plan.spread(pos, q, mu)
        rho = torch.full(mesh, float("nan"), dtype=torch.float32, device="cuda")
        st = _noalloc(lib, fr.box, mesh, order, pos, q, mu, rho, status)
        torch.cuda.synchronize()
        assert st == 0
        assert status.item() == 0
        assert torch.equal(rho, ref), (fr.n, mesh)
        rho_ref = O2.PMEOracle(fr.box, mesh, order, 0.30, 9.0).stage_mesh(pos64, q64, mu64)
        check(f"noalloc rho vs oracle n={fr.n} mesh={mesh} (rel max)",
              relmax(rho.cpu().numpy(), rho_ref), TOL_MESH)
        plan.close()


def test_noalloc_reports_nonfinite_input(gb):
    lib = gb.load_library()
    fr = W.molten_nacl(512, seed=5)
    pos, q, mu = (torch.tensor(np.float32(x), device="cuda") for x in prepared(fr))
    rho = torch.zeros((24, 24, 24), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    bad = pos.clone()
    bad[17, 1] = float("nan")
    assert _noalloc(lib, fr.box, (24, 24, 24), 4, bad, q, mu, rho, status) == 0
    torch.cuda.synchronize()
    assert status.item() == 4   # PME_ERR_NONFINITE
    # the next call on finite inputs reports a clean status and the plan spread's result
    assert _noalloc(lib, fr.box, (24, 24, 24), 4, pos, q, mu, rho, status) == 0
    torch.cuda.synchronize()
    assert status.item() == 0
    plan = gb.Plan(fr.box, (24, 24, 24), 4, 0.30, 9.0, max_ions=1024, brick=(8, 8, 16))
    assert torch.equal(rho, plan.spread(pos, q, mu))
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(gb):
    lib = gb.load_library()
    fr = W.rocksalt(2, 5.64)
    pos, q, mu = (torch.tensor(np.float32(x), device="cuda") for x in (fr.pos, fr.q, fr.mu))
    rho = torch.zeros((16, 16, 16), device="cuda")
    big = torch.zeros((32769, 3), device="cuda")
    assert _noalloc(lib, fr.box, (16, 16, 16), 4, big, big[:, 0].contiguous(), None, rho) == 1
    big_mesh = torch.zeros((136, 16, 16), device="cuda")
    assert _noalloc(lib, fr.box, (136, 16, 16), 4, pos, q, mu, big_mesh) == 1
    assert _noalloc(lib, fr.box, (16, 16, 16), 8, pos, q, mu, rho) == 1
    # and a valid call still works afterwards
    assert _noalloc(lib, fr.box, (16, 16, 16), 4, pos, q, mu, rho) == 0
    torch.cuda.synchronize()
    assert abs(rho.double().sum().item() - float(np.float32(fr.q).astype(np.float64).sum())) < 1e-4
