"""The index-checking build (GBPME_BOUNDS): the forward, backward, batch, stage and quadrupole
parity tests run again, in a child process, against libgbpme_bounds.so, whose sort, spread,
gather, pair-list and combine kernels test every derived index before the access and record a
flag instead of touching memory out of range. The child must pass those tests and finish with
no index check failed (pme_bounds_flags() == 0) under the checking build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

FILES = ["tests/test_gpu_forward.py", "tests/test_gpu_backward.py", "tests/test_gpu_batch.py",
         "tests/test_gpu_stages.py", "tests/test_gpu_quadrupole.py"]


def test_parity_cases_under_index_checks(root, tmp_path):
    report = tmp_path / "bounds.json"
    env = dict(os.environ, GBPME_BOUNDS="1", GBPME_BOUNDS_REPORT=str(report))
    env.pop("GBPME_PARITY_LOG", None)
    r = subprocess.run([sys.executable, "-c", "import __graft_entry__ as g; g.build()"], cwd=root, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    # tests that assert bitwise equality between two different kernels (hit-list vs cell-walk
    # pair term) are left out: the index checks change the code the compiler generates for one
    # of them, so their rounding may differ in the last bit under this build
    r = subprocess.run([sys.executable, "-m", "pytest", *FILES, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider",
                        "-k", "not bitwise"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    print(tail)
    assert r.returncode == 0, tail
    rep = json.loads(report.read_text())
    assert rep.get("checking") == 1, rep
    assert rep.get("flags") == 0, rep
