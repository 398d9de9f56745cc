"""GPU test of pme_spread_noalloc, the allocation-free spread for callers that cannot call
cudaMalloc (a host framework that has reserved the whole device for its own pool, or a loop
that must not allocate because allocation can synchronise the device).

It is called through the C ABI twice in a row -- on different inputs, so the second call also
shows that the shared static scratch does not carry anything over -- and each result is
compared with pme_spread of a plan with the same box, mesh and order, within the mesh
tolerance the other parity tests use. Sizes beyond the fixed scratch must be rejected. The
file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

from gpu_util import TOL_MESH, prepared, relmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def _noalloc(lib, box, mesh, order, pos, q, mu, rho):
    b = (ctypes.c_double * 9)(*np.asarray(box, np.float64).reshape(9))
    m = (ctypes.c_int * 3)(*mesh)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return lib.pme_spread_noalloc(stream, b, m, order, int(pos.shape[0]), ptr(pos), ptr(q),
                                  ptr(mu), ptr(rho))


def test_noalloc_spread_matches_plan_spread_twice(gb):
    lib = gb.load_library()
    cases = [
        (W.molten_nacl(4096, L=51.0, seed=1001), (64, 64, 64), 6),
        (W.molten_nacl(1000, seed=77), (27, 30, 25), 5),
    ]
    for fr, mesh, order in cases:   # two calls in a row on the shared scratch
        pos, q, mu = (torch.tensor(np.float32(x), device="cuda") for x in prepared(fr))
        plan = gb.Plan(fr.box, mesh, order, 0.30, 9.0, max_ions=4096)
        ref = plan.spread(pos, q, mu)
        rho = torch.full(mesh, float("nan"), dtype=torch.float32, device="cuda")
        st = _noalloc(lib, fr.box, mesh, order, pos, q, mu, rho)
        torch.cuda.synchronize()
        assert st == 0
        assert torch.isfinite(rho).all()
        assert relmax(rho.cpu().numpy(), ref.cpu().numpy()) < TOL_MESH


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
