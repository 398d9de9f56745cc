"""Host-side parts of the benchmark, on CPU: the pair count behind the pair term's flop figure
(the roofline's numerator) against brute force over the periodic images, and the reference
arm's JSON line (the oracle timed on the host cores) with the contract's keys and the same
config as the CUDA arm."""
import itertools

import numpy as np
import pytest

pytest.importorskip("scipy")

import workloads as W


def _brute_ordered_pairs(pos, L, rcut):
    # ordered (i, j), i != j, and every image n with |r_j - r_i + n L| < rcut
    d0 = pos[None, :, :] - pos[:, None, :]
    count = 0
    for n in itertools.product((-1, 0, 1), repeat=3):
        d = d0 + np.asarray(n, np.float64) * L
        r2 = (d * d).sum(-1)
        count += int(((r2 < rcut * rcut) & (r2 > 0.0)).sum())
    return count


@pytest.mark.parametrize("n,L,rcut", [(128, (16.0, 16.0, 16.0), 7.0), (96, (14.0, 17.5, 15.2), 6.5),
                                      (200, (18.6, 18.6, 18.6), 9.0)])
def test_pair_hits_matches_brute_force(n, L, rcut):
    import bench
    fr = W.molten_nacl(n, seed=n)
    L = np.asarray(L)
    pos = fr.pos / fr.box[0, 0] * L              # spread the frame over the orthorhombic box
    pos[:5] += L * np.array([1.0, -2.0, 0.0])    # some positions outside the cell
    box = np.diag(L)
    got = bench.pair_hits(pos, box, rcut)
    assert got == _brute_ordered_pairs(np.mod(pos, L), L, rcut)
    assert got > 10 * n                           # not vacuous


def test_pair_hits_refuses_a_cutoff_beyond_half_the_box():
    import bench
    fr = W.molten_nacl(64, seed=1)               # L = 12.7 A
    with pytest.raises(ValueError):
        bench.pair_hits(fr.pos, fr.box, 6.5)


def test_reference_arm_line_on_cpu(monkeypatch, capsys):
    # the reference arm times the float64 oracle on the host cores: one step of the small
    # rock-salt workload, and the JSON line carries the keys of the benchmark contract
    import json

    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class Args:
        workload = "rocksalt512"
        steps = 1
        warmup = 0
    assert bench.run_reference(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["value"] > 0
    assert line["config"]["workload"].startswith("rock-salt NaCl 512 ions")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    fr, cfg = bench.build_frame("rocksalt512")
    assert line["config"] == bench.config_dict(cfg, fr, 1)   # the same config as the CUDA arm's
