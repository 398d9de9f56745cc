"""Python face of libgbpme: a plan object over the C ABI and a differentiable energy.

Every step of the computation runs in the library's CUDA kernels (the 3D transforms in the
library's own kernels or in cuFFT, see Plan(fft=...)); this module only allocates output
tensors, passes pointers and the current CUDA stream, and wires the adjoint into
torch.autograd:

  E = PMEEnergy.apply(plan, pos, q, mu)
  F = -torch.autograd.grad(E, pos, create_graph=True)[0]      # Eq. forces
  loss = ((F - F_ref) ** 2).mean(); loss.backward()           # Eq. loss: double backward

The first derivatives come from pme_forward; the derivative of those derivatives (the
Hessian-vector product the force-matching loss needs) from pme_backward, which reuses what
the plan kept from the forward when its inputs are the forward's (checked on the device) and
recomputes everything otherwise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import PMEError, PMEOpts


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(device):
    if device.type != "cuda":
        return None
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _f32(t, device):
    if t is None:
        return None
    if (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.device == device
            and t.is_contiguous()):
        return t   # the common case, without the conversion calls
    t = torch.as_tensor(t)
    if device.type == "cuda":
        t = t.to(device=device)
    return t.to(torch.float32).contiguous()


class _on_device:
    """torch.cuda.device(device), skipped when that device is already current."""

    def __init__(self, device):
        self.device = device
        self.ctx = None

    def __enter__(self):
        if torch.cuda.current_device() != self.device.index:
            self.ctx = torch.cuda.device(self.device)
            self.ctx.__enter__()

    def __exit__(self, *exc):
        if self.ctx is not None:
            self.ctx.__exit__(*exc)


def mesh_dims(box, spacing: float, rule: int = 0, strategy: int = 1, clamp=(0, 0)):
    """Mesh-size rules of Section 2.3.1 (see pme_mesh_dims in include/gbpme.h)."""
    lib = _abi.load()
    b = (ctypes.c_double * 9)(*np.asarray(box, np.float64).reshape(9))
    m = (ctypes.c_int * 3)()
    st = lib.pme_mesh_dims(b, float(spacing), int(rule), int(strategy), int(clamp[0]), int(clamp[1]), m)
    if st:
        raise PMEError(st, "pme_mesh_dims")
    return [m[0], m[1], m[2]]


def spread_noalloc(box, mesh, order: int, pos, q, mu=None, status=None):
    """pme_spread_noalloc: the mesh density without a plan and without any device allocation
    (for callers that cannot allocate; see include/gbpme.h). Device tensors in; rho is
    allocated here by torch only because this helper returns a new tensor -- callers that
    cannot allocate pass their own output through the C ABI. status: optional int32 device
    tensor of one element, set on the stream to 4 (PME_ERR_NONFINITE) when an input held a NaN
    or Inf, else 0."""
    lib = _abi.load()
    dev = pos.device
    pos, q, mu = (_f32(t, dev) for t in (pos, q, mu))
    if pos.shape[0] > _abi.NOALLOC_MAX_IONS or max(mesh) > _abi.NOALLOC_MAX_MESH:
        raise ValueError(f"pme_spread_noalloc takes at most {_abi.NOALLOC_MAX_IONS} ions and "
                         f"mesh dimensions up to {_abi.NOALLOC_MAX_MESH}")
    rho = torch.empty(tuple(int(m) for m in mesh), dtype=torch.float32, device=dev)
    b = (ctypes.c_double * 9)(*np.asarray(box, np.float64).reshape(9))
    m = (ctypes.c_int * 3)(*[int(x) for x in mesh])
    with torch.cuda.device(dev):
        st = lib.pme_spread_noalloc(_stream_handle(dev), b, m, int(order), int(pos.shape[0]),
                                    _ptr(pos), _ptr(q), _ptr(mu), _ptr(rho),
                                    None if status is None else _ptr(status))
    if st:
        raise PMEError(st, "pme_spread_noalloc")
    return rho


def _set_brick(opts, brick, autotune):
    if brick is not None:
        b = [int(x) for x in brick]
        if len(b) != 3:
            raise ValueError("brick is three edges (x, y, z)")
        opts.brick[0], opts.brick[1], opts.brick[2] = b
    opts.autotune = int(bool(autotune))


SPREAD_SHAPES = [(8, 8, 16), (8, 8, 32), (16, 8, 16), (16, 16, 16), (4, 8, 16)]


def autotune_brick(box, mesh, order: int, alpha: float, rcut: float, n_ions: int, device=None):
    """pme_autotune_brick: the fastest brick shape for this mesh, order and ion count, and the
    median forward + backward milliseconds of every built shape (None where it does not apply)."""
    lib = _abi.load()
    dev = torch.device("cuda") if device is None else torch.device(device)
    b = (ctypes.c_double * 9)(*np.asarray(box, np.float64).reshape(9))
    m = (ctypes.c_int * 3)(*[int(x) for x in mesh])
    out = (ctypes.c_int * 3)()
    ms = (ctypes.c_double * len(SPREAD_SHAPES))()
    with torch.cuda.device(dev):
        st = lib.pme_autotune_brick(b, m, int(order), float(alpha), float(rcut), int(n_ions), None, out, ms)
    if st:
        raise PMEError(st, "pme_autotune_brick")
    times = {sh: (ms[k] if ms[k] >= 0 else None) for k, sh in enumerate(SPREAD_SHAPES)}
    return (out[0], out[1], out[2]), times


def _outputs(want, given, alloc, dev):
    # the output tensors of a call: fresh ones, or the caller's, checked against what the call
    # writes (a wrong buffer would be overwritten past its end by the library)
    out = {}
    for k, spec in want.items():
        if spec is None:
            continue
        shape, dtype = spec
        t = None if given is None else given.get(k)
        if t is None:
            t = torch.empty(shape, dtype=dtype, **alloc)
        elif (tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous()
              or t.device.type != dev.type):
            raise ValueError(f"output '{k}': expected a contiguous {dtype} tensor of shape {shape} on {dev}")
        out[k] = t
    return out


def launch_count() -> int:
    return int(_abi.load().pme_launch_count())


_FFT_KINDS = {"auto": 0, "cufft": 1, "own": 2, "own-general": 3}


class Plan:
    """One box, mesh, spline order, alpha and cutoff; owns all device scratch."""

    def __init__(self, box, mesh, order: int, alpha: float, rcut: float, *,
                 influence_power: float = 1.0, deconvolution: bool = True,
                 coulomb_k: float = 1.0, include_pair: bool = True, include_self: bool = True,
                 include_background: bool = True, max_ions: int = 1 << 18,
                 overlap_pair: bool = True, recip_method: str = "mesh", ewald_kmax: float = 0.0,
                 influence: str = "deconvolution", fft: str = "auto", brick=None, autotune: bool = True,
                 device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("gbpme needs a CUDA device; there is no CPU fallback")
        self.lib = _abi.load()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("a plan lives on a CUDA device")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        torch.cuda.init()
        opts = PMEOpts()
        self.lib.pme_opts_default(ctypes.byref(opts))
        opts.influence_power = float(influence_power)
        opts.deconvolution = int(bool(deconvolution))
        opts.coulomb_k = float(coulomb_k)
        opts.include_pair = int(bool(include_pair))
        opts.include_self = int(bool(include_self))
        opts.include_background = int(bool(include_background))
        opts.max_ions = int(max_ions)
        opts.overlap_pair = int(bool(overlap_pair))
        if recip_method not in ("mesh", "ewald"):
            raise ValueError("recip_method is 'mesh' or 'ewald'")
        if influence not in ("deconvolution", "p3m"):
            raise ValueError("influence is 'deconvolution' or 'p3m'")
        opts.influence_kind = 0 if influence == "deconvolution" else 1
        if fft not in _FFT_KINDS:
            raise ValueError("fft is 'auto', 'cufft', 'own' or 'own-general'")
        opts.fft = _FFT_KINDS[fft]
        opts.recip_method = 0 if recip_method == "mesh" else 1
        opts.ewald_kmax = float(ewald_kmax)
        _set_brick(opts, brick, autotune)
        self.box = np.asarray(box, np.float64).reshape(3, 3).copy()
        self.mesh = tuple(int(x) for x in mesh)
        self.order = int(order)
        self.alpha = float(alpha)
        self.rcut = float(rcut)
        self.coulomb_k = float(coulomb_k)
        self.max_ions = int(max_ions)
        b = (ctypes.c_double * 9)(*self.box.reshape(9))
        m = (ctypes.c_int * 3)(*self.mesh)
        h = ctypes.c_void_p()
        with _on_device(self.device):
            st = self.lib.pme_plan_create(ctypes.byref(h), b, m, self.order, self.alpha, self.rcut,
                                          ctypes.byref(opts))
        if st:
            raise PMEError(st, "pme_plan_create")
        self.handle = h
        self.brick = self._brick()

    # -- helpers ---------------------------------------------------------------------------
    def _brick(self):
        b = (ctypes.c_int * 3)()
        self._check(self.lib.pme_plan_brick(self.handle, b), "pme_plan_brick")
        return (b[0], b[1], b[2])

    def _check(self, st, where):
        if st:
            raise PMEError(st, where, self.lib.pme_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pme_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_box(self, box):
        self.box = np.asarray(box, np.float64).reshape(3, 3).copy()
        b = (ctypes.c_double * 9)(*self.box.reshape(9))
        self._check(self.lib.pme_plan_set_box(self.handle, b), "pme_plan_set_box")

    @property
    def fft_kind(self) -> str:
        """'own' (the library's transforms, general or power-of-two kernels) or 'cufft'
        (pme_plan_fft_kind)."""
        k = ctypes.c_int(-1)
        self._check(self.lib.pme_plan_fft_kind(self.handle, ctypes.byref(k)), "pme_plan_fft_kind")
        return "cufft" if k.value == 1 else "own"

    @property
    def fft_kernels(self) -> str:
        """'general', 'power-of-two' (the library's own) or 'cufft' (pme_plan_fft_kind)."""
        k = ctypes.c_int()
        self._check(self.lib.pme_plan_fft_kind(self.handle, ctypes.byref(k)), "pme_plan_fft_kind")
        return {0: "general", 1: "cufft", 2: "power-of-two"}[k.value]

    def sync_status(self):
        with _on_device(self.device):
            self._check(self.lib.pme_sync_status(self.handle, _stream_handle(self.device)),
                        "pme_sync_status")

    def profile(self, enable: bool = True):
        """Turn the per-stage CUDA-event timers on or off (see pme_profile_enable)."""
        self._check(self.lib.pme_profile_enable(self.handle, int(bool(enable))), "pme_profile_enable")

    def profile_read(self):
        """{'fwd.spread': (ms_total, calls), ...} since the last read; resets the timers."""
        ms = (ctypes.c_double * _abi.NUM_STAGES)()
        calls = (ctypes.c_longlong * _abi.NUM_STAGES)()
        with _on_device(self.device):
            self._check(self.lib.pme_profile_read(self.handle, ms, calls), "pme_profile_read")
        out = {}
        for k in range(_abi.NUM_STAGES):
            name = ("fwd." if k < 9 else "bwd.") + _abi.STAGE_NAMES[k % 9]
            if calls[k]:
                out[name] = (float(ms[k]), int(calls[k]))
        return out

    @property
    def M(self):
        return int(np.prod(self.mesh))

    # -- full passes -----------------------------------------------------------------------
    def forward(self, pos, q, mu=None, *, energy=True, force=True, phi=True, field=True,
                field_grad=False, virial=False, out=None, sync=True):
        """Energy and derivatives (and, with virial=True, the 3x3 virial -dE/d strain; see
        pme_forward_virial). Device tensors stay on the device; CPU tensors are passed as
        host pointers (the library stages them). Returns a dict of tensors.

        out: optional dict of preallocated output tensors (the keys asked for, with the shapes
        and dtypes this method would allocate, on the inputs' device; pinned host memory for
        host calls), written instead of fresh ones. sync=False skips the stream synchronisation
        after a host call: host outputs are then complete only once the current stream has been
        synchronised (by a later call with sync=True, for instance)."""
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        pos = _f32(pos, dev)
        q = _f32(q, dev)
        mu = _f32(mu, dev)
        n = int(pos.shape[0])
        pin = (not on_dev)
        alloc = dict(device=dev, pin_memory=pin) if pin else dict(device=dev)
        want = {"energy": ((1,), torch.float64) if (energy or virial) else None,
                "force": ((n, 3), torch.float32) if force else None,
                "phi": ((n,), torch.float32) if phi else None,
                "field": ((n, 3), torch.float32) if field else None,
                "field_grad": ((n, 6), torch.float32) if field_grad else None,
                "virial": ((3, 3), torch.float64) if virial else None}
        out = _outputs(want, out, alloc, dev)
        with _on_device(self.device):
            args = (self.handle, _stream_handle(self.device), n, _ptr(pos), _ptr(q),
                    _ptr(mu), _ptr(out.get("energy")), _ptr(out.get("force")),
                    _ptr(out.get("phi")), _ptr(out.get("field")), _ptr(out.get("field_grad")))
            if virial:
                st = self.lib.pme_forward_virial(*args, _ptr(out["virial"]))
                self._check(st, "pme_forward_virial")
            else:
                st = self.lib.pme_forward(*args)
                self._check(st, "pme_forward")
            if not on_dev and sync:
                torch.cuda.current_stream(self.device).synchronize()
        return out

    def forward_quad(self, pos, q, mu, theta, *, energy=True, force=True, phi=True, field=True,
                     field_grad=True):
        """Forward with point quadrupoles theta [n, 6] (xx, yy, zz, xy, xz, yz) or [n, 3, 3]
        (pme_forward_quad): field_grad is then -dE/dTheta. Returns a dict of tensors."""
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        if theta is not None and tuple(theta.shape[-2:]) == (3, 3):
            t = torch.as_tensor(theta)
            theta = torch.stack([t[:, 0, 0], t[:, 1, 1], t[:, 2, 2], t[:, 0, 1], t[:, 0, 2], t[:, 1, 2]], 1)
        pos = _f32(pos, dev)
        q = _f32(q, dev)
        mu = _f32(mu, dev)
        theta = _f32(theta, dev)
        n = int(pos.shape[0])
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        out = {}
        if energy:
            out["energy"] = torch.empty(1, dtype=torch.float64, **alloc)
        if force:
            out["force"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if phi:
            out["phi"] = torch.empty(n, dtype=torch.float32, **alloc)
        if field:
            out["field"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if field_grad:
            out["field_grad"] = torch.empty((n, 6), dtype=torch.float32, **alloc)
        with _on_device(self.device):
            st = self.lib.pme_forward_quad(self.handle, _stream_handle(self.device), n, _ptr(pos), _ptr(q),
                                           _ptr(mu), _ptr(theta), _ptr(out.get("energy")),
                                           _ptr(out.get("force")), _ptr(out.get("phi")),
                                           _ptr(out.get("field")), _ptr(out.get("field_grad")))
            self._check(st, "pme_forward_quad")
            if not on_dev:
                torch.cuda.current_stream(self.device).synchronize()
        return out

    def backward(self, pos, q, mu=None, g_energy=None, g_force=None, g_phi=None, g_field=None, *,
                 out=None, sync=True):
        """Vector-Jacobian product of (pos, q, mu) -> (E, force, phi, field). out: optional
        preallocated (grad_pos [n, 3], grad_q [n], grad_mu [n, 3]) float32 tensors; sync as for
        forward."""
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        pos = _f32(pos, dev)
        q = _f32(q, dev)
        mu = _f32(mu, dev)
        g_force = _f32(g_force, dev)
        g_phi = _f32(g_phi, dev)
        g_field = _f32(g_field, dev)
        if g_energy is not None:
            g_energy = torch.as_tensor(g_energy, dtype=torch.float64).reshape(1)
            g_energy = g_energy.to(dev).contiguous()
        n = int(pos.shape[0])
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        want = {"gp": ((n, 3), torch.float32), "gq": ((n,), torch.float32), "gm": ((n, 3), torch.float32)}
        o = _outputs(want, None if out is None else dict(zip(("gp", "gq", "gm"), out)), alloc, dev)
        gp, gq, gm = o["gp"], o["gq"], o["gm"]
        with _on_device(self.device):
            st = self.lib.pme_backward(self.handle, _stream_handle(self.device), n, _ptr(pos), _ptr(q),
                                       _ptr(mu), _ptr(g_energy), _ptr(g_force), _ptr(g_phi),
                                       _ptr(g_field), _ptr(gp), _ptr(gq), _ptr(gm))
            self._check(st, "pme_backward")
            if not on_dev and sync:
                torch.cuda.current_stream(self.device).synchronize()
        return gp, gq, gm

    def backward_quad(self, pos, q, mu, theta, g_energy=None, g_force=None, g_phi=None, g_field=None):
        """pme_backward_quad: vector-Jacobian product of (pos, q, mu, theta) -> (E, force, phi,
        field) of the quadrupole forward. Returns (grad_pos, grad_q, grad_mu, grad_theta [n, 6],
        the symmetric matrix with dL = G : dTheta)."""
        return self._backward_quad(pos, q, mu, theta, g_energy, g_force, g_phi, g_field, 1,
                                   self.lib.pme_backward_quad, True)

    def _backward_quad(self, pos, q, mu, theta, g_energy, g_force, g_phi, g_field, nE, fn, single):
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        if theta is not None and tuple(theta.shape[-2:]) == (3, 3):
            t = torch.as_tensor(theta)
            theta = torch.stack([t[:, 0, 0], t[:, 1, 1], t[:, 2, 2], t[:, 0, 1], t[:, 0, 2], t[:, 1, 2]], 1)
        pos, q, mu, theta, g_force, g_phi, g_field = (_f32(t, dev) for t in (pos, q, mu, theta, g_force, g_phi,
                                                                             g_field))
        if g_energy is not None:
            g_energy = torch.as_tensor(g_energy, dtype=torch.float64).reshape(nE).to(dev).contiguous()
        n = int(pos.shape[0])
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        gp = torch.empty((n, 3), dtype=torch.float32, **alloc)
        gq = torch.empty(n, dtype=torch.float32, **alloc)
        gm = torch.empty((n, 3), dtype=torch.float32, **alloc)
        gt = torch.empty((n, 6), dtype=torch.float32, **alloc)
        args = (_ptr(pos), _ptr(q), _ptr(mu), _ptr(theta), _ptr(g_energy), _ptr(g_force), _ptr(g_phi),
                _ptr(g_field), _ptr(gp), _ptr(gq), _ptr(gm), _ptr(gt))
        with _on_device(self.device):
            if single:
                st = fn(self.handle, _stream_handle(self.device), n, *args)
            else:
                st = fn(self.handle, _stream_handle(self.device), *args)
            self._check(st, "pme_backward_quad" if single else "pme_batch_backward_quad")
            if not on_dev:
                torch.cuda.current_stream(self.device).synchronize()
        return gp, gq, gm, gt

    # -- stage-level entry points (device tensors) -------------------------------------------
    def spread(self, pos, q, mu=None):
        pos, q, mu = (_f32(t, self.device) for t in (pos, q, mu))
        rho = torch.empty(self.mesh, dtype=torch.float32, device=self.device)
        with _on_device(self.device):
            self._check(self.lib.pme_spread(self.handle, _stream_handle(self.device), int(pos.shape[0]),
                                            _ptr(pos), _ptr(q), _ptr(mu), _ptr(rho)), "pme_spread")
        return rho

    def solve(self, rho):
        rho = _f32(rho, self.device)
        phi = torch.empty(self.mesh, dtype=torch.float32, device=self.device)
        e = torch.empty(1, dtype=torch.float64, device=self.device)
        with _on_device(self.device):
            self._check(self.lib.pme_solve(self.handle, _stream_handle(self.device), _ptr(rho), _ptr(phi),
                                           _ptr(e)), "pme_solve")
        return phi, e

    def gather(self, pos, phi_mesh):
        pos = _f32(pos, self.device)
        phi_mesh = _f32(phi_mesh, self.device)
        out = torch.empty((pos.shape[0], 10), dtype=torch.float32, device=self.device)
        with _on_device(self.device):
            self._check(self.lib.pme_gather(self.handle, _stream_handle(self.device), int(pos.shape[0]),
                                            _ptr(pos), _ptr(phi_mesh), _ptr(out)), "pme_gather")
        return out

    def pair(self, pos, q, mu=None):
        pos, q, mu = (_f32(t, self.device) for t in (pos, q, mu))
        out = torch.empty((pos.shape[0], 10), dtype=torch.float32, device=self.device)
        e = torch.empty(1, dtype=torch.float64, device=self.device)
        with _on_device(self.device):
            self._check(self.lib.pme_pair(self.handle, _stream_handle(self.device), int(pos.shape[0]),
                                          _ptr(pos), _ptr(q), _ptr(mu), _ptr(out), _ptr(e)), "pme_pair")
        return out, e


class BatchPlan(Plan):
    """Many frames of uneven sizes in one plan (pme_batch_create): every stage is one launch
    over the whole batch. Frame f owns ions [offsets[f], offsets[f+1]) of the batch arrays."""

    def __init__(self, boxes, meshes, orders, offsets, alpha: float, rcut: float, *,
                 influence_power: float = 1.0, deconvolution: bool = True,
                 coulomb_k: float = 1.0, include_pair: bool = True, include_self: bool = True,
                 include_background: bool = True, overlap_pair: bool = True,
                 influence: str = "deconvolution", fft: str = "auto", brick=None, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("gbpme needs a CUDA device; there is no CPU fallback")
        self.lib = _abi.load()
        dev = torch.device("cuda") if device is None else torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        torch.cuda.init()
        opts = PMEOpts()
        self.lib.pme_opts_default(ctypes.byref(opts))
        opts.influence_power = float(influence_power)
        opts.deconvolution = int(bool(deconvolution))
        opts.coulomb_k = float(coulomb_k)
        opts.include_pair = int(bool(include_pair))
        if influence not in ("deconvolution", "p3m"):
            raise ValueError("influence is 'deconvolution' or 'p3m'")
        opts.influence_kind = 0 if influence == "deconvolution" else 1
        if fft not in _FFT_KINDS:
            raise ValueError("fft is 'auto', 'cufft', 'own' or 'own-general'")
        opts.fft = _FFT_KINDS[fft]
        opts.include_self = int(bool(include_self))
        opts.include_background = int(bool(include_background))
        opts.overlap_pair = int(bool(overlap_pair))
        _set_brick(opts, brick, False)
        boxes = np.asarray(boxes, np.float64).reshape(-1, 9)
        meshes = np.asarray(meshes, np.int32).reshape(-1, 3)
        orders = np.asarray(orders, np.int32).reshape(-1)
        offsets = np.asarray(offsets, np.int32).reshape(-1)
        F = len(orders)
        if not (len(boxes) == len(meshes) == F and len(offsets) == F + 1):
            raise ValueError("boxes, meshes, orders need one entry per frame and offsets F + 1")
        self.nframes = F
        self.offsets = offsets.copy()
        self.n = int(offsets[-1])
        self.coulomb_k = float(coulomb_k)
        b = (ctypes.c_double * (9 * F))(*boxes.reshape(-1))
        m = (ctypes.c_int * (3 * F))(*meshes.reshape(-1).tolist())
        o = (ctypes.c_int * F)(*orders.tolist())
        off = (ctypes.c_int * (F + 1))(*offsets.tolist())
        h = ctypes.c_void_p()
        with _on_device(self.device):
            st = self.lib.pme_batch_create(ctypes.byref(h), F, off, b, m, o, float(alpha), float(rcut),
                                           ctypes.byref(opts))
        if st:
            raise PMEError(st, "pme_batch_create")
        self.handle = h
        self.brick = self._brick()

    def forward(self, pos, q, mu=None, *, energy=True, force=True, phi=True, field=True,
                field_grad=False, virial=False):
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        pos, q, mu = (_f32(t, dev) for t in (pos, q, mu))
        n = self.n
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        out = {}
        if energy:
            out["energy"] = torch.empty(self.nframes, dtype=torch.float64, **alloc)
        if force:
            out["force"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if phi:
            out["phi"] = torch.empty(n, dtype=torch.float32, **alloc)
        if field:
            out["field"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if field_grad:
            out["field_grad"] = torch.empty((n, 6), dtype=torch.float32, **alloc)
        if virial:
            out.setdefault("energy", torch.empty(self.nframes, dtype=torch.float64, **alloc))
            out["virial"] = torch.empty((self.nframes, 3, 3), dtype=torch.float64, **alloc)
        with _on_device(self.device):
            args = (self.handle, _stream_handle(self.device), _ptr(pos), _ptr(q),
                    _ptr(mu), _ptr(out.get("energy")), _ptr(out.get("force")),
                    _ptr(out.get("phi")), _ptr(out.get("field")), _ptr(out.get("field_grad")))
            if virial:
                st = self.lib.pme_batch_forward_virial(*args, _ptr(out["virial"]))
                self._check(st, "pme_batch_forward_virial")
            else:
                st = self.lib.pme_batch_forward(*args)
                self._check(st, "pme_batch_forward")
            if not on_dev:
                torch.cuda.current_stream(self.device).synchronize()
        return out

    def forward_quad(self, pos, q, mu, theta, *, energy=True, force=True, phi=True, field=True,
                     field_grad=True):
        """pme_batch_forward_quad: every frame with point quadrupoles theta [n, 6] (xx, yy, zz,
        xy, xz, yz) or [n, 3, 3]; energy [F]; field_grad = -dE/dTheta."""
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        if theta is not None and tuple(theta.shape[-2:]) == (3, 3):
            t = torch.as_tensor(theta)
            theta = torch.stack([t[:, 0, 0], t[:, 1, 1], t[:, 2, 2], t[:, 0, 1], t[:, 0, 2], t[:, 1, 2]], 1)
        pos, q, mu, theta = (_f32(t, dev) for t in (pos, q, mu, theta))
        n = self.n
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        out = {}
        if energy:
            out["energy"] = torch.empty(self.nframes, dtype=torch.float64, **alloc)
        if force:
            out["force"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if phi:
            out["phi"] = torch.empty(n, dtype=torch.float32, **alloc)
        if field:
            out["field"] = torch.empty((n, 3), dtype=torch.float32, **alloc)
        if field_grad:
            out["field_grad"] = torch.empty((n, 6), dtype=torch.float32, **alloc)
        with _on_device(self.device):
            st = self.lib.pme_batch_forward_quad(self.handle, _stream_handle(self.device), _ptr(pos), _ptr(q),
                                                 _ptr(mu), _ptr(theta), _ptr(out.get("energy")),
                                                 _ptr(out.get("force")), _ptr(out.get("phi")),
                                                 _ptr(out.get("field")), _ptr(out.get("field_grad")))
            self._check(st, "pme_batch_forward_quad")
            if not on_dev:
                torch.cuda.current_stream(self.device).synchronize()
        return out

    def backward(self, pos, q, mu=None, g_energy=None, g_force=None, g_phi=None, g_field=None):
        dev = pos.device if isinstance(pos, torch.Tensor) else torch.device("cpu")
        on_dev = dev.type == "cuda"
        pos, q, mu, g_force, g_phi, g_field = (_f32(t, dev) for t in (pos, q, mu, g_force, g_phi, g_field))
        if g_energy is not None:
            g_energy = torch.as_tensor(g_energy, dtype=torch.float64).reshape(self.nframes).to(dev).contiguous()
        n = self.n
        alloc = dict(device=dev, pin_memory=True) if not on_dev else dict(device=dev)
        gp = torch.empty((n, 3), dtype=torch.float32, **alloc)
        gq = torch.empty(n, dtype=torch.float32, **alloc)
        gm = torch.empty((n, 3), dtype=torch.float32, **alloc)
        with _on_device(self.device):
            st = self.lib.pme_batch_backward(self.handle, _stream_handle(self.device), _ptr(pos), _ptr(q),
                                             _ptr(mu), _ptr(g_energy), _ptr(g_force), _ptr(g_phi),
                                             _ptr(g_field), _ptr(gp), _ptr(gq), _ptr(gm))
            self._check(st, "pme_batch_backward")
            if not on_dev:
                torch.cuda.current_stream(self.device).synchronize()
        return gp, gq, gm

    def backward_quad(self, pos, q, mu, theta, g_energy=None, g_force=None, g_phi=None, g_field=None):
        """pme_batch_backward_quad: as Plan.backward_quad for every frame (g_energy [F])."""
        return self._backward_quad(pos, q, mu, theta, g_energy, g_force, g_phi, g_field, self.nframes,
                                   self.lib.pme_batch_backward_quad, False)


# ------------------------------------------------------------------------------------------
# autograd
# ------------------------------------------------------------------------------------------

class _PMEGrad(torch.autograd.Function):
    """(pos, q, mu) -> (dE/dr, dE/dq, dE/dmu); its VJP is the Hessian-vector product."""

    @staticmethod
    def forward(ctx, plan, pos, q, mu, dEdr, dEdq, dEdmu):
        ctx.plan = plan
        ctx.save_for_backward(pos, q, mu)
        return dEdr.clone(), dEdq.clone(), dEdmu.clone()

    @staticmethod
    def backward(ctx, v_r, v_q, v_mu):
        pos, q, mu = ctx.saved_tensors
        z = lambda t, like: torch.zeros_like(like) if t is None else t
        v_r, v_q, v_mu = z(v_r, pos), z(v_q, q), z(v_mu, mu)
        gp, gq, gm = ctx.plan.backward(pos.detach(), q.detach(), mu.detach(), None,
                                       -v_r.detach(), v_q.detach(), -v_mu.detach())
        return None, gp, gq, gm, None, None, None


class PMEEnergy(torch.autograd.Function):
    """Differentiable total energy of Eq. (1) of include/gbpme.h, twice differentiable."""

    @staticmethod
    def forward(ctx, plan, pos, q, mu):
        out = plan.forward(pos.detach(), q.detach(), mu.detach(), energy=True, force=True,
                           phi=True, field=True)
        ctx.plan = plan
        ctx.save_for_backward(pos, q, mu, out["force"], out["phi"], out["field"])
        return out["energy"].reshape(())

    @staticmethod
    def backward(ctx, gE):
        pos, q, mu, F, phi, field = ctx.saved_tensors
        dEdr, dEdq, dEdmu = _PMEGrad.apply(ctx.plan, pos, q, mu, -F, phi, -field)
        g = gE.to(torch.float32)
        return None, g * dEdr, g * dEdq, g * dEdmu


_W6 = (1.0, 1.0, 1.0, 2.0, 2.0, 2.0)   # independent entries of a symmetric 3x3: off-diagonals twice


class _PMEQuadGrad(torch.autograd.Function):
    """(pos, q, mu, theta6) -> (dE/dr, dE/dq, dE/dmu, dE/dtheta6); its VJP along cotangents on the
    first three is the quadrupole Hessian-vector product (pme_backward_quad). A cotangent on
    dE/dtheta6 (a loss on -dE/dTheta) is not supported and raises."""

    @staticmethod
    def forward(ctx, plan, pos, q, mu, theta, dEdr, dEdq, dEdmu, dEdt):
        ctx.plan = plan
        ctx.save_for_backward(pos, q, mu, theta)
        return dEdr.clone(), dEdq.clone(), dEdmu.clone(), dEdt.clone()

    @staticmethod
    def backward(ctx, v_r, v_q, v_mu, v_t):
        pos, q, mu, theta = ctx.saved_tensors
        if v_t is not None and bool((v_t != 0).any()):
            raise RuntimeError("no second derivative through dE/dTheta (pme_backward_quad takes no "
                               "cotangent on -dE/dTheta)")
        z = lambda t, like: torch.zeros_like(like) if t is None else t
        v_r, v_q, v_mu = z(v_r, pos), z(v_q, q), z(v_mu, mu)
        gp, gq, gm, gt = ctx.plan.backward_quad(pos.detach(), q.detach(), mu.detach(), theta.detach(), None,
                                                -v_r.detach(), v_q.detach(), -v_mu.detach())
        w = torch.tensor(_W6, dtype=gt.dtype, device=gt.device)
        return None, gp, gq, gm, gt * w, None, None, None, None


class PMEQuadEnergy(torch.autograd.Function):
    """Total energy with point quadrupoles theta [n, 6] (xx, yy, zz, xy, xz, yz), through
    pme_forward_quad. The gradients are -force, phi, -field and, for the six independent
    entries of theta, -field_grad with the off-diagonal entries doubled (each appears twice in
    the symmetric tensor). Twice differentiable through the force, phi and field gradients
    (pme_backward_quad): a force-matching loss trains the quadrupole channel."""

    @staticmethod
    def forward(ctx, plan, pos, q, mu, theta):
        out = plan.forward_quad(pos.detach(), q.detach(), mu.detach(), theta.detach())
        ctx.plan = plan
        ctx.save_for_backward(pos, q, mu, theta, out["force"], out["phi"], out["field"], out["field_grad"])
        return out["energy"].reshape(())

    @staticmethod
    def backward(ctx, gE):
        pos, q, mu, theta, F, phi, field, fg = ctx.saved_tensors
        w = torch.tensor(_W6, dtype=fg.dtype, device=fg.device)
        dEdr, dEdq, dEdmu, dEdt = _PMEQuadGrad.apply(ctx.plan, pos, q, mu, theta, -F, phi, -field, -fg * w)
        g = gE.to(torch.float32)
        return None, g * dEdr, g * dEdq, g * dEdmu, g * dEdt


def pme_quad_energy(plan: Plan, pos, q, mu, theta):
    """Energy with point quadrupoles (theta [n, 6]); twice differentiable through the forces."""
    if mu is None:
        mu = torch.zeros_like(pos)
    return PMEQuadEnergy.apply(plan, pos, q, mu, theta)


def pme_energy(plan: Plan, pos, q, mu=None):
    if mu is None:
        mu = torch.zeros_like(pos)
    return PMEEnergy.apply(plan, pos, q, mu)
