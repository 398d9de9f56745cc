"""Python binding of the learned charge/dipole network (include/gbnet.h): argument marshalling
only. Every arithmetic step runs in libgbpme.so; torch provides device memory and streams."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import PMEError
from .pme import _ptr, _stream_handle

S, V, NR, LAYERS = 32, 16, 8, 2
NUM_PARAMS = 13266
MAX_NEIGHBOURS = 64
CUTOFF = 5.0

# the parameter vector of gbnet.h: (name, shape) in order, row-major blocks
PARAM_LAYOUT = ([("emb", (2, S))]
                + [item for t in range(LAYERS) for item in (
                    (f"WA{t}", (S, S + V)), (f"WB{t}", (V, 2 * V)), (f"WR{t}", (NR, S + 3 * V)),
                    (f"WU{t}", (S + V, S + V)), (f"WY{t}", (2 * V, V)))]
                + [("Wh", (S, 2 * S)), ("bh", (2 * S,)), ("wq", (S,)), ("bq", (1,)), ("wE", (S,)),
                   ("bE", (1,)), ("wmu", (V,))])


def pack_params(params: dict) -> np.ndarray:
    """Named parameter arrays -> the flat float32 vector of gbnet.h."""
    out = np.concatenate([np.asarray(params[k], np.float64).reshape(-1) for k, _ in PARAM_LAYOUT])
    assert out.size == NUM_PARAMS
    return out.astype(np.float32)


def unpack_params(flat) -> dict:
    """The flat parameter vector -> named float64 arrays."""
    flat = np.asarray(flat, np.float64).reshape(-1)
    out, o = {}, 0
    for k, shape in PARAM_LAYOUT:
        size = int(np.prod(shape))
        out[k] = flat[o:o + size].reshape(shape)
        o += size
    return out


def mix(X: torch.Tensor, wt_bits: torch.Tensor, Y: torch.Tensor | None = None, accumulate=False):
    """gbnet_mix: Y = X W (+ Y) on the tensor cores, W given as W^T bfloat16 bits [nout][k]
    (int16 tensor). Returns (Y, error word)."""
    lib = _abi.load()
    M, k = X.shape
    nout = wt_bits.shape[0]
    if Y is None:
        Y = torch.empty((M, nout), dtype=torch.float32, device=X.device)
    err = torch.zeros(1, dtype=torch.int32, device=X.device)
    with torch.cuda.device(X.device):
        st = lib.gbnet_mix(_stream_handle(X.device), M, k, nout, _ptr(X), _ptr(wt_bits), _ptr(Y),
                           int(bool(accumulate)), _ptr(err))
    if st:
        raise PMEError(st, "gbnet_mix")
    return Y, err


class Net:
    """Handle of the network: frames, parameters, optimiser state and scratch on one device."""

    def __init__(self, max_ions: int, max_frames: int, device="cuda"):
        self.lib = _abi.load()
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.gbnet_create(ctypes.byref(h), int(max_ions), int(max_frames))
        if st:
            raise PMEError(st, "gbnet_create")
        self.handle = h
        self.n = 0
        self.nframes = 0

    def _check(self, st, where):
        if st:
            raise PMEError(st, where, self.lib.gbnet_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gbnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _s(self):
        return _stream_handle(self.device)

    def set_frames(self, offsets, boxes, species):
        offsets = np.asarray(offsets, np.int64)
        F = len(offsets) - 1
        o = (ctypes.c_int * (F + 1))(*[int(x) for x in offsets])
        b = (ctypes.c_double * (9 * F))(*np.asarray(boxes, np.float64).reshape(-1))
        sp = torch.as_tensor(np.asarray(species), dtype=torch.int32, device=self.device).contiguous()
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_set_frames(self.handle, self._s(), F, o, b, _ptr(sp)), "gbnet_set_frames")
        self.n = int(offsets[-1])
        self.nframes = F

    def set_params(self, params):
        flat = pack_params(params) if isinstance(params, dict) else np.asarray(params, np.float32)
        t = torch.as_tensor(flat, dtype=torch.float32, device=self.device).contiguous()
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_set_params(self.handle, self._s(), _ptr(t)), "gbnet_set_params")
            torch.cuda.current_stream(self.device).synchronize()

    def set_params_device(self, t: torch.Tensor):
        """Copy parameters from a float32 device tensor on the call's stream (no host sync)."""
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_set_params(self.handle, self._s(), _ptr(t)), "gbnet_set_params")

    def get_params(self) -> torch.Tensor:
        t = torch.empty(NUM_PARAMS, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_get_params(self.handle, self._s(), _ptr(t)), "gbnet_get_params")
        return t

    def forward(self, pos):
        q = torch.empty(self.n, dtype=torch.float32, device=self.device)
        mu = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        e = torch.empty(self.nframes, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_forward(self.handle, self._s(), _ptr(pos.contiguous()), _ptr(q), _ptr(mu),
                                               _ptr(e)), "gbnet_forward")
        return dict(q=q, mu=mu, e_sr=e)

    def backward(self, g_q=None, g_mu=None, g_esr=None):
        gp = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        gpar = torch.empty(NUM_PARAMS, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_backward(self.handle, self._s(), _ptr(g_q), _ptr(g_mu), _ptr(g_esr),
                                                _ptr(gp), _ptr(gpar)), "gbnet_backward")
        return gp, gpar

    def loss_grad(self, pme, pos, e_ref, f_ref, lambda_e=1.0, lambda_f=1.0, grad=None, accumulate=False):
        loss = torch.empty(3, dtype=torch.float64, device=self.device)
        force = torch.empty((self.n, 3), dtype=torch.float32, device=self.device)
        if grad is None:
            grad = torch.zeros(NUM_PARAMS, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_loss_grad(self.handle, pme.handle, self._s(), _ptr(pos), _ptr(e_ref),
                                                 _ptr(f_ref), float(lambda_e), float(lambda_f), _ptr(loss),
                                                 _ptr(force), _ptr(grad), int(bool(accumulate))),
                        "gbnet_loss_grad")
        return loss, force, grad

    def adam(self, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_adam(self.handle, self._s(), _ptr(grad), float(lr), float(beta1),
                                            float(beta2), float(eps)), "gbnet_adam")

    def train_step(self, pme, pos, e_ref, f_ref, lambda_e=1.0, lambda_f=1.0, lr=1e-3, loss=None):
        if loss is None:
            loss = torch.empty(3, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_train_step(self.handle, pme.handle, self._s(), _ptr(pos), _ptr(e_ref),
                                                  _ptr(f_ref), float(lambda_e), float(lambda_f), float(lr),
                                                  _ptr(loss)), "gbnet_train_step")
        return loss

    def sync_status(self):
        with torch.cuda.device(self.device):
            self._check(self.lib.gbnet_sync_status(self.handle, self._s()), "gbnet_sync_status")

    def last_launches(self) -> int:
        return int(self.lib.gbnet_last_launches(self.handle))
