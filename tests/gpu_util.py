"""Helpers shared by the GPU parity tests (comparison metrics, bars and frame preparation).

Inputs are rounded to float32 once, and the oracle receives exactly those float32 values
(converted to float64), so oracle and CUDA path see the same input.

Every parity check goes through ``check``: it asserts the bar and records the achieved error
(printed, and appended as one JSON line to the file named by the environment variable
GBPME_PARITY_LOG when that is set), so a run shows how far inside its bar each case is."""
import json
import os

import numpy as np


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def relmax(a, b):
    """max |a - b| / max |b| (recorded: the caller asserts its bar)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    e = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    record("rel max", e, None)
    return e


def relrmse(a, b):
    """RMS(a - b) / RMS(b) (recorded: the caller asserts its bar)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    e = float(np.sqrt(np.mean((a - b) ** 2)) / max(np.sqrt(np.mean(b ** 2)), 1e-300))
    record("rel RMSE", e, None)
    return e


def sym6(H):
    """[n,3,3] -> [n,6] in the order xx, yy, zz, xy, xz, yz."""
    return np.stack([H[:, 0, 0], H[:, 1, 1], H[:, 2, 2], H[:, 0, 1], H[:, 0, 2], H[:, 1, 2]], 1)


def prepared(frame):
    """(pos, q, mu) rounded to float32 and returned as float64 arrays."""
    return f32(frame.pos), f32(frame.q), f32(frame.mu)


# Tolerances. The energy and force bars are the ones stated for float32 mesh work against
# the float64 plain PME on the same mesh: relative energy error 1e-6 of |E| and relative force
# RMSE 1e-5. phi, field and field gradient share the force bar. Intermediate mesh quantities
# are held to a max-norm bar of the same order. The backward (a Hessian-vector product) is
# held to the force bar as well: measured errors are a few 1e-7 (512-32768 ions, p = 4-7).
TOL_E = 1e-6
TOL_F = 1e-5
TOL_MESH = 2e-5
TOL_HVP = 1e-5


def record(what, err, bar):
    """Print the achieved error of one check and log it (GBPME_PARITY_LOG)."""
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    print(f"[parity] {test} {what}: {err:.3e}" + ("" if bar is None else f" (bar {bar:.1e})"))
    path = os.environ.get("GBPME_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": test, "what": what, "err": err, "bar": bar}) + "\n")


def check(what, err, bar):
    record(what, float(err), float(bar))
    assert err < bar, (what, err, bar)


def check_energy(got, ref, what="energy", cancel=None):
    """|got - E| < TOL_E |E| with E = ref["energy"] (or ref itself when it is a number).

    cancel=True is for the cases where the parts of the Ewald split cancel (a lone ion, whose
    mesh self-interaction is removed by the self term; a dense neutral frame whose float64
    self energy removes most of E_recip): the float32 parts E_recip and E_pair then carry
    rounding above 1e-6 |E|, and the bar becomes TOL_E (|E_recip| + |E_pair|). cancel=None
    decides from the oracle's parts: the float64 terms cancel more than half of the float32
    parts, |E| < (|E_recip| + |E_pair|) / 2. The float64 parts E_self and E_bg never enter a
    bar."""
    E = ref["energy"] if isinstance(ref, dict) else ref
    if cancel is None:
        cancel = (isinstance(ref, dict) and "e_recip" in ref and "e_pair" in ref
                  and abs(float(E)) < 0.5 * (abs(float(ref["e_recip"])) + abs(float(ref["e_pair"]))))
    err = abs(float(got) - float(E))
    if cancel:
        scale = abs(ref["e_recip"]) + abs(ref["e_pair"])
        record(what + " (err/|E|)", err / max(abs(E), 1e-300), float("inf"))
        check(what + " (err/(|E_rec|+|E_pair|))", err / scale, TOL_E)
    else:
        check(what + " (err/|E|)", err / max(abs(E), 1e-300), TOL_E)


def check_rmse(what, got, ref, bar=TOL_F):
    check(what + " (rel RMSE)", relrmse(got, ref), bar)
