"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws random numbers and lays out geometry: it holds none of the
particle-mesh Ewald arithmetic (no weights, no Green's function, no energies). Both
the CPU oracle (``oracle/``) and the CUDA path consume what it returns.

The paper's own datasets (a charged molecular dimer and a liquid-NaCl trajectory) are
not available, so these generators stand in for them with the same sizes, densities
and value distributions:

* ``rocksalt``    -- NaCl rock-salt supercell (q = +-1), optional Gaussian jitter and
                     Gaussian point dipoles.
* ``molten_nacl`` -- random sequential addition of Na/Cl ions with a minimum image
                     separation at ~1.5 g/cm^3 (32.35 A^3 per ion), charges +-0.8 with
                     Gaussian jitter shifted to zero net charge, Gaussian dipoles.
* ``uneven_frames`` -- a batch of molten-NaCl frames whose ion counts are uniform in
                     [64, 1024], each box scaled so the density stays fixed.
* ``quadrupoles`` -- Gaussian symmetric point quadrupoles for the rank-2 channel.

Units: Angstrom for lengths, elementary charges for q, e*Angstrom for dipoles.
All arrays are float64 numpy arrays; callers cast as they need.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

VOLUME_PER_ION = 32.35  # A^3 per ion, ~1.5 g/cm^3 molten NaCl


@dataclass
class Frame:
    """One periodic configuration: rows of ``box`` are the lattice vectors."""

    pos: np.ndarray          # [n, 3]
    q: np.ndarray            # [n]
    mu: np.ndarray           # [n, 3]
    box: np.ndarray          # [3, 3]
    species: np.ndarray = field(default=None)  # [n] int, 0 = Na, 1 = Cl

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def rocksalt(ncell: int = 4, a: float = 5.64, jitter: float = 0.0,
             mu_sigma: float = 0.0, seed: int = 1000) -> Frame:
    """Rock-salt NaCl: ``ncell``^3 conventional cubic cells of edge ``a`` (8 ions each).

    With jitter = mu_sigma = 0 this is the perfect crystal whose Coulomb energy per ion
    pair is fixed by the Madelung constant.
    """
    rng = np.random.default_rng(seed)
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    cl = base + np.array([0.5, 0.0, 0.0])
    cells = np.array([[i, j, k] for i in range(ncell) for j in range(ncell) for k in range(ncell)],
                     dtype=np.float64)
    na_pos = (cells[:, None, :] + base[None]).reshape(-1, 3) * a
    cl_pos = (cells[:, None, :] + cl[None]).reshape(-1, 3) * a
    pos = np.concatenate([na_pos, cl_pos])
    q = np.concatenate([np.ones(len(na_pos)), -np.ones(len(cl_pos))])
    species = np.concatenate([np.zeros(len(na_pos), np.int64), np.ones(len(cl_pos), np.int64)])
    L = ncell * a
    if jitter > 0:
        pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    pos = np.mod(pos, L)
    mu = rng.normal(0.0, mu_sigma, size=pos.shape) if mu_sigma > 0 else np.zeros_like(pos)
    return Frame(pos=pos, q=q, mu=mu, box=np.eye(3) * L, species=species)


def _rsa_positions(n: int, L: float, min_sep: float, rng: np.random.Generator,
                   max_tries: int = 200) -> np.ndarray:
    """Random sequential addition in a cubic periodic box with a minimum image separation."""
    nc = max(1, int(L // min_sep))
    cell = L / nc
    grid: dict[tuple[int, int, int], list[int]] = {}
    out = np.empty((n, 3), dtype=np.float64)
    s2 = min_sep * min_sep
    accepted = 0
    tries = 0
    batch = rng.uniform(0.0, L, size=(4096, 3))
    bi = 0
    while accepted < n:
        if bi == len(batch):
            batch = rng.uniform(0.0, L, size=(4096, 3))
            bi = 0
        x, y, z = batch[bi]
        bi += 1
        cx, cy, cz = int(x / cell) % nc, int(y / cell) % nc, int(z / cell) % nc
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    lst = grid.get(((cx + dx) % nc, (cy + dy) % nc, (cz + dz) % nc))
                    if not lst:
                        continue
                    for j in lst:
                        px, py, pz = out[j]
                        ex = x - px
                        ey = y - py
                        ez = z - pz
                        ex -= L * round(ex / L)
                        ey -= L * round(ey / L)
                        ez -= L * round(ez / L)
                        if ex * ex + ey * ey + ez * ez < s2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[accepted] = (x, y, z)
            grid.setdefault((cx, cy, cz), []).append(accepted)
            accepted += 1
            tries = 0
        else:
            tries += 1
            if tries > max_tries * n:
                raise RuntimeError("random sequential addition jammed")
    return out


def molten_nacl(n: int, L: float | None = None, min_sep: float = 2.2, q0: float = 0.8,
                q_sigma: float = 0.05, mu_sigma: float = 0.05, seed: int = 1001) -> Frame:
    """Molten-NaCl-like frame: n/2 Na and n/2 Cl at random positions (random species order).

    ``L`` defaults to (32.35 * n)^(1/3), i.e. the ~1.5 g/cm^3 density. Charges are
    +-q0 plus N(0, q_sigma^2), then shifted so that the sum is exactly zero in float64;
    dipoles are N(0, mu_sigma^2) per component.
    """
    if n % 2:
        raise ValueError("n must be even")
    rng = np.random.default_rng(seed)
    if L is None:
        L = (VOLUME_PER_ION * n) ** (1.0 / 3.0)
    pos = _rsa_positions(n, L, min_sep, rng)
    species = np.concatenate([np.zeros(n // 2, np.int64), np.ones(n // 2, np.int64)])
    rng.shuffle(species)
    q = np.where(species == 0, q0, -q0) + rng.normal(0.0, q_sigma, size=n)
    q = q - q.mean()
    mu = rng.normal(0.0, mu_sigma, size=(n, 3))
    return Frame(pos=pos, q=q, mu=mu, box=np.eye(3) * L, species=species)


def cubic_crystal(basis, charges, ncell: int, a: float) -> Frame:
    """ncell^3 cubic cells of edge a, each holding ions of the given charges at the fractional
    positions ``basis`` (a perfect crystal; no dipoles)."""
    cells = np.array([(i, j, k) for i in range(ncell) for j in range(ncell) for k in range(ncell)], np.float64)
    b = np.asarray(basis, np.float64)
    pos = ((cells[:, None, :] + b[None, :, :]) * a).reshape(-1, 3)
    q = np.tile(np.asarray(charges, np.float64), len(cells))
    species = (q < 0).astype(np.int64)
    return Frame(pos=pos, q=q, mu=np.zeros_like(pos), box=np.eye(3) * (ncell * a), species=species)


def with_net_charge(fr: Frame, Q: float, k: int) -> Frame:
    """The frame with Q / k added to the charges of its first k ions (net charge Q)."""
    q = np.array(fr.q, np.float64)
    q[:k] += Q / k
    return Frame(pos=fr.pos, q=q, mu=fr.mu, box=fr.box, species=fr.species)


def charged_dimer(sep: float = 8.0, L: float = 30.0, mu_sigma: float = 0.05,
                  seed: int = 1005) -> Frame:
    """Two small ion clusters of opposite total charge in a cubic box (a stand-in for the
    paper's charged molecular dimer, whose geometry is not given)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, 0.8, size=(4, 3)) + np.array([L / 2 - sep / 2, L / 2, L / 2])
    b = rng.normal(0.0, 0.8, size=(4, 3)) + np.array([L / 2 + sep / 2, L / 2, L / 2])
    pos = np.concatenate([a, b])
    qa = rng.normal(0.25, 0.1, size=4)
    qb = rng.normal(-0.25, 0.1, size=4)
    qa += (1.0 - qa.sum()) / 4
    qb += (-1.0 - qb.sum()) / 4
    q = np.concatenate([qa, qb])
    mu = rng.normal(0.0, mu_sigma, size=(8, 3))
    return Frame(pos=pos, q=q, mu=mu, box=np.eye(3) * L,
                 species=np.array([0, 0, 0, 0, 1, 1, 1, 1]))


@dataclass
class FrameSpec:
    """Per-frame settings of the uneven batch: mesh spacing target and spline order."""

    frame: Frame
    spacing: float
    order: int


def uneven_frames(n_frames: int = 256, n_min: int = 64, n_max: int = 1024,
                  spacing: float = 0.8, orders=(4, 6), seed: int = 1002) -> list[FrameSpec]:
    """Batch of molten-NaCl frames with ion counts uniform in [n_min, n_max] (even),
    box edge (32.35 n)^(1/3), orders alternating by frame index."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n_frames):
        n = int(rng.integers(n_min // 2, n_max // 2 + 1)) * 2
        fr = molten_nacl(n, seed=seed * 1000 + f)
        out.append(FrameSpec(frame=fr, spacing=spacing, order=orders[f % len(orders)]))
    return out


def quadrupoles(n: int, sigma: float = 0.05, seed: int = 55) -> np.ndarray:
    """Random symmetric point quadrupoles [n, 3, 3] (e*Angstrom^2): each independent entry
    of the upper triangle drawn from N(0, sigma^2), mirrored below the diagonal."""
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, sigma, size=(n, 3, 3))
    return np.triu(A) + np.transpose(np.triu(A, 1), (0, 2, 1))


def tangent(n: int, scale: float = 1.0, seed: int = 77):
    """Random cotangents (g_force [n,3], g_phi [n], g_field [n,3]) for backward tests."""
    rng = np.random.default_rng(seed)
    return (rng.normal(0, scale, size=(n, 3)), rng.normal(0, scale, size=n),
            rng.normal(0, scale, size=(n, 3)))


# Named workloads: mesh/order/alpha/rcut settings that go with each generator.
WORKLOADS = {
    "rocksalt512": dict(gen=lambda: rocksalt(4, 5.64, jitter=0.1, mu_sigma=0.05, seed=1000),
                        mesh=(32, 32, 32), order=4, alpha=0.30, rcut=10.0, desc="rock-salt NaCl"),
    "nacl4096": dict(gen=lambda: molten_nacl(4096, L=51.0, seed=1001),
                     mesh=(64, 64, 64), order=6, alpha=0.30, rcut=9.0, desc="molten-NaCl"),
    "nacl32k": dict(gen=lambda: molten_nacl(32768, L=102.0, seed=1004),
                    mesh=(128, 128, 128), order=6, alpha=0.30, rcut=9.0, desc="molten-NaCl"),
    "nacl262k": dict(gen=lambda: molten_nacl(262144, L=204.0, seed=1014),
                     mesh=(256, 256, 256), order=6, alpha=0.30, rcut=9.0, desc="molten-NaCl"),
}


def workload(name: str):
    """Return (Frame, settings dict) for a named workload."""
    w = WORKLOADS[name]
    fr = w["gen"]()
    cfg = {k: v for k, v in w.items() if k != "gen"}
    return fr, cfg



# ---- the learned charge/dipole network: seeded parameters and training frames ---------

NET_SCALARS, NET_VECTORS, NET_RADIAL, NET_LAYERS = 32, 16, 8, 2
# (name, shape, stored as bfloat16?) in the order of the flat parameter vector; the shapes
# are (fan_in, fan_out) for the channel-mixing matrices
NET_LAYOUT = (
    [("emb", (2, NET_SCALARS), False)]
    + [item for t in range(NET_LAYERS) for item in (
        (f"WA{t}", (NET_SCALARS, NET_SCALARS + NET_VECTORS), True),
        (f"WB{t}", (NET_VECTORS, 2 * NET_VECTORS), True),
        (f"WR{t}", (NET_RADIAL, NET_SCALARS + 3 * NET_VECTORS), False),
        (f"WU{t}", (NET_SCALARS + NET_VECTORS, NET_SCALARS + NET_VECTORS), True),
        (f"WY{t}", (2 * NET_VECTORS, NET_VECTORS), True))]
    + [("Wh", (NET_SCALARS, 2 * NET_SCALARS), True), ("bh", (2 * NET_SCALARS,), False),
       ("wq", (NET_SCALARS,), False), ("bq", (1,), False),
       ("wE", (NET_SCALARS,), False), ("bE", (1,), False),
       ("wmu", (NET_VECTORS,), False)]
)


def to_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def net_params(seed: int = 2024) -> dict:
    """Gaussian initial parameters of the network, sigma = 1/sqrt(fan_in) for every weight
    matrix (the embedding table and the radial weights included), biases zero. The
    channel-mixing matrices are rounded to bfloat16 (the precision they are stored in);
    everything else is float32. Returns float64 arrays by name."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shape, bf16 in NET_LAYOUT:
        if name.startswith("b"):
            v = np.zeros(shape)
        else:
            v = rng.normal(0.0, 1.0 / math.sqrt(shape[0]), size=shape)
        out[name] = to_bf16(v) if bf16 else np.asarray(np.float32(v), np.float64)
    return out


def training_frames(n_frames: int = 32, n: int = 512, seed: int = 1003) -> list[Frame]:
    """Molten-NaCl frames of the learned-charge task: n ions each at ~1.5 g/cm^3
    (L = 25.5 A for 512 ions), species set; charges and dipoles are not used (the teacher
    assigns them)."""
    return [molten_nacl(n, seed=seed * 1000 + f) for f in range(n_frames)]
