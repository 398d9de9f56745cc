"""Host-side checks of the C ABI that need no GPU: the library loads, exports every function
the public header declares, every ctypes signature has the prototype's number of parameters,
the ctypes mirror of pme_opts has the C compiler's layout of the header's struct, and the
host-only mesh-size rule agrees with the oracle's."""
import ctypes

import numpy as np
import pytest

from oracle import meshdims


@pytest.fixture(scope="module")
def lib():
    import paper_2606_01598_gb300 as g
    from paper_2606_01598_gb300 import build as b
    b.build()
    return g.load_library()


def test_every_header_symbol_is_exported(lib):
    import paper_2606_01598_gb300 as g
    names = g.header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(9):
        assert lib.pme_status_string(s)
    assert lib.pme_bounds_checking() == 0 and lib.pme_bounds_flags() == 0
    assert lib.pme_last_error(None) == b"null plan"


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("strategy", [0, 1, 2])
def test_mesh_dims_matches_oracle(lib, rule, strategy):
    import paper_2606_01598_gb300 as g
    names = {0: "pow2", 1: "smooth", 2: "ceil"}
    rules = {0: "paper", 1: "spacing"}
    rng = np.random.default_rng(rule * 3 + strategy)
    for _ in range(50):
        box = np.diag(rng.uniform(5, 120, size=3))
        box[1, 0] = rng.uniform(-3, 3)
        sp = rng.uniform(0.2, 1.5)
        got = g.mesh_dims(box, sp, rule, strategy)
        ref = meshdims.mesh_dims(box, sp, names[strategy], rules[rule])
        assert got == ref


def test_mesh_dims_rejects_bad_arguments(lib):
    m = (ctypes.c_int * 3)()
    b = (ctypes.c_double * 9)(*np.eye(3).reshape(9))
    assert lib.pme_mesh_dims(b, 0.0, 0, 1, 0, 0, m) == 1
    assert lib.pme_mesh_dims(b, 0.5, 2, 1, 0, 0, m) == 1
    assert lib.pme_mesh_dims(b, 0.5, 0, 3, 0, 0, m) == 1


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.pme_plan_destroy(None) == 1
    assert lib.pme_forward(None, None, 0, *([None] * 8)) == 1
    assert lib.pme_backward(None, None, 0, *([None] * 10)) == 1


def _prototypes():
    """name -> number of parameters, from every prototype the public headers declare."""
    import re

    import paper_2606_01598_gb300._abi as A
    out = {}
    for h in A.HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
        for name, args in re.findall(r"\b((?:pme|gbnet)_[a-z_0-9]+)\s*\(([^()]*)\)\s*;", src, flags=re.S):
            args = " ".join(args.split())
            out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_ctypes_signatures_match_the_header_prototypes():
    # a ctypes signature with a parameter more or fewer than the C prototype would pass
    # shifted arguments to the library
    import paper_2606_01598_gb300._abi as A
    protos = _prototypes()
    assert set(protos) == set(A.header_functions())
    wrong = {n: (len(A._SIGS[n][1]), k) for n, k in protos.items() if len(A._SIGS[n][1]) != k}
    assert not wrong, wrong


def test_opts_struct_layout_matches_the_header(tmp_path):
    # the ctypes mirror of pme_opts against the C compiler's layout of the header's struct
    import shutil
    import subprocess

    import paper_2606_01598_gb300._abi as A
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in A.PMEOpts._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gbpme.h"\nint main(void) {\n'
                    '  printf("%zu\\n", sizeof(pme_opts));\n'
                    + "".join(f'  printf("%zu\\n", offsetof(pme_opts, {n}));\n' for n in names)
                    + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    inc = __import__("os").path.dirname(A.HEADER)
    subprocess.run([cc, "-std=c99", "-I", inc, str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(A.PMEOpts)
    assert got[1:] == [getattr(A.PMEOpts, n).offset for n in names]


def _c_kind(decl):
    d = " ".join(decl.split())
    if "*" in d or "[" in d or d.endswith("_t") or " pme_plan_t" in d or d.startswith("pme_plan_t") \
            or d.startswith("gbnet_t"):
        return "ptr"
    if "double" in d:
        return "f64"
    if "float" in d:
        return "f32"
    if "long long" in d:
        return "i64"
    if "int" in d or "size_t" in d:
        return "i32" if "size_t" not in d else "i64"
    return "?" + d


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    return {ctypes.c_double: "f64", ctypes.c_float: "f32", ctypes.c_int: "i32", ctypes.c_longlong: "i64",
            ctypes.c_size_t: "i64"}.get(t, "?" + repr(t))


def test_ctypes_parameter_kinds_match_the_header():
    # pointer / float64 / float32 / integer class of each parameter (a double passed where the
    # prototype has an int, or the reverse, lands in the wrong register)
    import re

    import paper_2606_01598_gb300._abi as A
    bad = {}
    for h in A.HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        src = re.sub(r"^\s*#.*$", "", src, flags=re.M)
        for name, args in re.findall(r"\b((?:pme|gbnet)_[a-z_0-9]+)\s*\(([^()]*)\)\s*;", src, flags=re.S):
            args = " ".join(args.split())
            c = [] if args in ("", "void") else [_c_kind(a) for a in args.split(",")]
            py = [_ctypes_kind(t) for t in A._SIGS[name][1]]
            if c != py:
                bad[name] = (c, py)
    assert not bad, bad
