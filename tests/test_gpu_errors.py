"""Allocation failure on the real path: a batched plan whose meshes need far more memory than
the device has (64 frames of 1000^3 points: 512 GB for the densities alone, so the first
device allocation fails at once, before any memory is touched) is refused with
PME_ERR_NOMEM, frees what it had, and leaves the device usable for the next plan."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pme as O2

from gpu_util import TOL_F, prepared, relrmse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2606_01598_gb300 as g
    return g


def test_plan_larger_than_the_device_is_refused_and_recovers(gb):
    F = 64
    box = np.diag([400.0, 400.0, 400.0])
    offsets = np.arange(F + 1, dtype=np.int64) * 2
    with pytest.raises(gb.PMEError) as e:
        gb.BatchPlan([box] * F, [(1000, 1000, 1000)] * F, [4] * F, offsets, 0.3, 9.0, include_pair=False)
    assert e.value.status == 7   # PME_ERR_NOMEM
    # the failure left nothing behind: a normal plan works and agrees with the oracle
    fr = W.molten_nacl(512, seed=61)
    pos, q, mu = prepared(fr)
    plan = gb.Plan(fr.box, (32, 32, 32), 5, 0.3, 9.0, max_ions=512)
    c = lambda x: torch.tensor(np.float32(x), device="cuda")
    out = plan.forward(c(pos), c(q), c(mu))
    plan.sync_status()
    ref = O2.PMEOracle(fr.box, (32, 32, 32), 5, 0.3, 9.0).evaluate(pos, q, mu, field_grad=False)
    assert relrmse(out["force"].cpu().numpy(), ref["force"]) < TOL_F
    plan.close()
