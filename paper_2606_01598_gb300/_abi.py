"""ctypes declarations of the libgbpme C ABI (include/gbpme.h). Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import re

from .build import ROOT, lib_path

c_int = ctypes.c_int
c_double = ctypes.c_double
c_void_p = ctypes.c_void_p
c_float_p = ctypes.POINTER(ctypes.c_float)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_int_p = ctypes.POINTER(ctypes.c_int)

HEADER = os.path.join(ROOT, "include", "gbpme.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "gbnet.h")]

STATUS = {0: "PME_OK", 1: "PME_ERR_ARG", 2: "PME_ERR_CUDA", 3: "PME_ERR_CUFFT",
          4: "PME_ERR_NONFINITE", 5: "PME_ERR_UNSUPPORTED", 6: "PME_ERR_TIMEOUT",
          7: "PME_ERR_NOMEM", 8: "PME_ERR_BOUNDS"}


class PMEOpts(ctypes.Structure):
    _fields_ = [("influence_power", c_double), ("deconvolution", c_int), ("coulomb_k", c_double),
                ("include_pair", c_int), ("include_self", c_int), ("include_background", c_int),
                ("max_ions", c_int), ("brick", c_int * 3), ("overlap_pair", c_int),
                ("recip_method", c_int), ("ewald_kmax", c_double), ("influence_kind", c_int),
                ("fft", c_int), ("autotune", c_int), ("reserved", c_int * 3)]


_SIGS = {
    "pme_opts_default": (None, [ctypes.POINTER(PMEOpts)]),
    "pme_mesh_dims": (c_int, [c_double_p, c_double, c_int, c_int, c_int, c_int, c_int_p]),
    "pme_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_double_p, c_int_p, c_int, c_double,
                                c_double, ctypes.POINTER(PMEOpts)]),
    "pme_plan_set_box": (c_int, [c_void_p, c_double_p]),
    "pme_plan_destroy": (c_int, [c_void_p]),
    "pme_plan_fft_kind": (c_int, [c_void_p, c_int_p]),
    "pme_plan_brick": (c_int, [c_void_p, c_int_p]),
    "pme_last_error": (ctypes.c_char_p, [c_void_p]),
    "pme_status_string": (ctypes.c_char_p, [c_int]),
    "pme_sync_status": (c_int, [c_void_p, c_void_p]),
    "pme_forward": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 8),
    "pme_forward_virial": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 9),
    "pme_forward_quad": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 9),
    "pme_backward": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 10),
    "pme_backward_quad": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 12),
    "pme_batch_backward_quad": (c_int, [c_void_p, c_void_p] + [c_void_p] * 12),
    "pme_spread": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 4),
    "pme_solve": (c_int, [c_void_p, c_void_p] + [c_void_p] * 3),
    "pme_gather": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 3),
    "pme_pair": (c_int, [c_void_p, c_void_p, c_int] + [c_void_p] * 5),
    "pme_launch_count": (ctypes.c_longlong, []),
    "pme_bounds_flags": (c_int, []),
    "pme_bounds_checking": (c_int, []),
    "pme_autotune_brick": (c_int, [c_double_p, c_int_p, c_int, c_double, c_double, c_int,
                                   ctypes.POINTER(PMEOpts), c_int_p, c_double_p]),
    "pme_profile_enable": (c_int, [c_void_p, c_int]),
    "pme_profile_read": (c_int, [c_void_p, c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
    "pme_spread_noalloc": (c_int, [c_void_p, c_double_p, c_int_p, c_int, c_int] + [c_void_p] * 5),
    "pme_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int_p, c_double_p, c_int_p, c_int_p,
                                 c_double, c_double, ctypes.POINTER(PMEOpts)]),
    "pme_batch_frames": (c_int, [c_void_p]),
    "pme_batch_forward": (c_int, [c_void_p, c_void_p] + [c_void_p] * 8),
    "pme_batch_forward_virial": (c_int, [c_void_p, c_void_p] + [c_void_p] * 9),
    "pme_batch_forward_quad": (c_int, [c_void_p, c_void_p] + [c_void_p] * 9),
    "pme_batch_backward": (c_int, [c_void_p, c_void_p] + [c_void_p] * 10),
    # the learned charge/dipole network (include/gbnet.h)
    "gbnet_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int]),
    "gbnet_destroy": (c_int, [c_void_p]),
    "gbnet_last_error": (ctypes.c_char_p, [c_void_p]),
    "gbnet_set_frames": (c_int, [c_void_p, c_void_p, c_int, c_int_p, c_double_p, c_void_p]),
    "gbnet_set_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "gbnet_get_params": (c_int, [c_void_p, c_void_p, c_void_p]),
    "gbnet_forward": (c_int, [c_void_p, c_void_p] + [c_void_p] * 4),
    "gbnet_backward": (c_int, [c_void_p, c_void_p] + [c_void_p] * 5),
    "gbnet_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double,
                                c_void_p, c_void_p, c_void_p, c_int]),
    "gbnet_adam": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_double, c_double, c_double]),
    "gbnet_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double,
                                 c_double, c_void_p]),
    "gbnet_mix": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "gbnet_sync_status": (c_int, [c_void_p, c_void_p]),
    "gbnet_last_launches": (ctypes.c_longlong, [c_void_p]),
}

NOALLOC_MAX_IONS = 32768
NOALLOC_MAX_MESH = 128

NUM_STAGES = 18
STAGE_NAMES = ["sort", "spread", "fft_r2c", "influence", "fft_c2r", "gather", "pair",
               "combine", "pair_eval"]

_LIB = None


def header_functions() -> list[str]:
    """Names of every function the public headers declare."""
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b((?:pme|gbnet)_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def load():
    """Load libgbpme.so (built in-tree), or with GBPME_BOUNDS=1 in the environment the
    index-checking libgbpme_bounds.so. Raises if it is missing: there is no fallback."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path(os.environ.get("GBPME_BOUNDS") == "1")
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class PMEError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))
