"""Seeded synthetic inputs for the pore / water-vapour MD: wall lattices, vapour placements, velocities.

This module is the one place both sides of the parity checks take their inputs from: the CUDA path
(through the C-ABI) and the FP64 CPU oracle read the identical arrays it returns. It draws random
numbers and builds geometry; it holds none of the simulation's arithmetic (no pair potential, no
integrator, no thermostat, no observables).

Reduced Lennard-Jones units throughout (sigma = epsilon = m = k_B = 1). The box is centred at the
origin: x, y in [-L/2, L/2) (periodic), z in [-Lz/2, Lz/2] (specular walls).

Geometry conventions
--------------------
* Wall: a simple-cubic lattice of spacing ``a`` with sites at ``-L/2 + (i + 1/2) a`` on every axis,
  kept where ``|z| < slab_half`` and removed where a pore's carve predicate holds (strict ``<``).
* Pore kinds and their carve predicates, with (dx, dy) the minimum-image offset from the pore axis
  (cx, cy) and h the slab half-thickness:
    - CYLINDER:  dx^2 + dy^2 < r0^2
    - CONE:      sqrt(dx^2 + dy^2) < r0 + (r1 - r0) (z + h) / (2 h)   (narrow end r0 at z = -h)
    - SLIT:      |dy| < width / 2                                       (spans the whole x extent)
    - INKBOTTLE: dx^2 + dy^2 < r0^2  or  dx^2 + dy^2 + z^2 < r_cavity^2 (neck through the slab,
                 spherical cavity at the slab centre)
    - PRISM:     |dx| < r0 and |dy| < r1 and z > h - width   (rectangular pore open at the slab's top
                 face; a floor at z = h - width when 0 < width < 2h, else through the slab)
* Wall models: 0 = fixed LJ wall atoms (the lattice above); 1 = hard walls -- no atoms, the slab
  minus the pores is a solid that reflects molecules specularly (the paper's reflecting pore walls).
* Planar systems (dims = 2): every molecule at y = 0 with vy = 0, moving in the x-z plane.
* Vapour: random sequential addition, uniform in ``slab_half < |z| < Lz/2``, at least ``min_sep``
  from every wall atom and from every other vapour molecule (periodic in x, y). Pores start empty.
* Velocities: each component drawn from N(0, T0/m), then the mean (centre-of-mass) velocity removed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

PORE_NONE, PORE_CYLINDER, PORE_CONE, PORE_SLIT, PORE_INKBOTTLE, PORE_PRISM = 0, 1, 2, 3, 4, 5
PORE_KIND_NAMES = {PORE_CYLINDER: "cylinder", PORE_CONE: "cone", PORE_SLIT: "slit",
                   PORE_INKBOTTLE: "inkbottle", PORE_PRISM: "prism"}


@dataclasses.dataclass
class Pore:
    kind: int
    cx: float = 0.0
    cy: float = 0.0
    r0: float = 0.0        # cylinder radius / cone radius at z=-h / ink-bottle neck / prism half-side x
    r1: float = 0.0        # cone radius at z=+h / prism half-side y
    r_cavity: float = 0.0  # ink-bottle cavity radius
    width: float = 0.0     # slit width / prism depth from the top face (<= 0 or >= 2h: through)


@dataclasses.dataclass
class Potential:
    """Lennard-Jones 12-6 parameters with cutoff (reduced units)."""
    eps: float = 1.0
    sigma: float = 1.0
    mass: float = 1.0
    rc: float = 2.5
    eps_w: float = 1.5
    sigma_w: float = 1.0
    rc_w: float = 2.5
    skin: float = 0.3
    shift_energy: int = 1
    r_ads: float = 1.5       # a vapour molecule counts as adsorbed when a wall atom is closer than this
    bin_width: float = 0.5   # axial (z) density-profile bin width
    cell_size: float = 0.0   # minimum cell side of the GPU path (0: max(rc, rc_w) + skin); no physics


@dataclasses.dataclass
class System:
    name: str
    Lx: float
    Ly: float
    Lz: float
    slab_half: float
    lattice_a: float
    pores: List[Pore]
    x0: np.ndarray           # (n, 3) float64
    v0: np.ndarray           # (n, 3) float64
    wall: np.ndarray         # (nw, 3) float64
    T0: float
    dt: float = 0.005
    tau_B: float = 0.0       # 0 -> thermostat_every * dt (plain velocity rescaling)
    thermostat_every: int = 10
    seed: int = 0
    dims: int = 3            # 2: planar system in x-z (y = 0, vy = 0)
    wall_model: int = 0      # 0 LJ wall atoms, 1 hard reflecting walls (no atoms)

    @property
    def n_vapor(self) -> int:
        return int(self.x0.shape[0])

    @property
    def n_wall(self) -> int:
        return int(self.wall.shape[0])


# ----------------------------------------------------------------------------------------------
# geometry


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    d = d.copy()
    d[d >= 0.5 * L] -= L
    d[d < -0.5 * L] += L
    return d


def carve_mask(points: np.ndarray, pore: Pore, Lx: float, Ly: float, slab_half: float) -> np.ndarray:
    """True where ``points`` (n,3) fall inside the carved-out region of ``pore``."""
    dx = _min_image(points[:, 0] - pore.cx, Lx)
    dy = _min_image(points[:, 1] - pore.cy, Ly)
    z = points[:, 2]
    rxy2 = dx * dx + dy * dy
    if pore.kind == PORE_CYLINDER:
        return rxy2 < pore.r0 * pore.r0
    if pore.kind == PORE_CONE:
        h = slab_half
        R = pore.r0 + (pore.r1 - pore.r0) * (z + h) / (2.0 * h)
        return np.sqrt(rxy2) < R
    if pore.kind == PORE_SLIT:
        return np.abs(dy) < 0.5 * pore.width
    if pore.kind == PORE_INKBOTTLE:
        return (rxy2 < pore.r0 * pore.r0) | (rxy2 + z * z < pore.r_cavity * pore.r_cavity)
    if pore.kind == PORE_PRISM:
        h = slab_half
        floor = h - pore.width if 0.0 < pore.width < 2.0 * h else -2.0 * h
        return (np.abs(dx) < pore.r0) & (np.abs(dy) < pore.r1) & (z > floor)
    raise ValueError(f"unknown pore kind {pore.kind}")


def sc_wall(Lx: float, Ly: float, Lz: float, slab_half: float, a: float,
            pores: Sequence[Pore]) -> np.ndarray:
    """Simple-cubic wall sites (half-offset lattice) in ``|z| < slab_half`` minus every pore."""
    nx, ny, nz = int(round(Lx / a)), int(round(Ly / a)), int(round(Lz / a))
    xs = -0.5 * Lx + (np.arange(nx) + 0.5) * a
    ys = -0.5 * Ly + (np.arange(ny) + 0.5) * a
    zs = -0.5 * Lz + (np.arange(nz) + 0.5) * a
    zs = zs[np.abs(zs) < slab_half]
    if zs.size == 0:
        return np.zeros((0, 3))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    keep = np.ones(len(pts), dtype=bool)
    for p in pores:
        keep &= ~carve_mask(pts, p, Lx, Ly, slab_half)
    return np.ascontiguousarray(pts[keep])


# ----------------------------------------------------------------------------------------------
# random placement


def _periodic_tree(points: np.ndarray, Lx: float, Ly: float, Lz: float):
    from scipy.spatial import cKDTree
    shifted = points + np.array([0.5 * Lx, 0.5 * Ly, 0.5 * Lz])
    # wrap x, y into [0, L) for the periodic tree; z is not periodic (a box far larger than Lz)
    shifted[:, 0] = np.mod(shifted[:, 0], Lx)
    shifted[:, 1] = np.mod(shifted[:, 1], Ly)
    box = np.array([Lx, Ly, 64.0 * Lz + 64.0])
    shifted[:, 2] += 16.0 * Lz
    return cKDTree(shifted, boxsize=box), (lambda q: _shift_query(q, Lx, Ly, Lz))


def _shift_query(q: np.ndarray, Lx: float, Ly: float, Lz: float) -> np.ndarray:
    s = q + np.array([0.5 * Lx, 0.5 * Ly, 0.5 * Lz])
    s[:, 0] = np.mod(s[:, 0], Lx)
    s[:, 1] = np.mod(s[:, 1], Ly)
    s[:, 2] += 16.0 * Lz
    return s


def rsa_vapor(rng: np.random.Generator, n: int, Lx: float, Ly: float, Lz: float, z_lo: float,
              z_hi: float, wall: np.ndarray, min_sep: float = 0.9,
              max_attempt_factor: int = 1000, planar: bool = False,
              upper_only: bool = False) -> np.ndarray:
    """Random sequential addition of ``n`` points uniform in ``z_lo < |z| < z_hi`` (x, y periodic),
    each at least ``min_sep`` from the wall points and from each other.

    Candidates are drawn in batches; a candidate is rejected if it is too close to a wall point, to
    an accepted point, or to an earlier surviving candidate of its own batch.
    """
    from scipy.spatial import cKDTree
    if n == 0:
        return np.zeros((0, 3))
    wall_tree, wq = (None, None)
    if len(wall):
        wall_tree, wq = _periodic_tree(wall, Lx, Ly, Lz)
    accepted = np.zeros((0, 3))
    attempts = 0
    while len(accepted) < n:
        need = n - len(accepted)
        k = max(256, int(need * 1.25) + 16)
        attempts += k
        if attempts > max_attempt_factor * n:
            raise RuntimeError("random sequential addition did not converge")
        x = rng.uniform(-0.5 * Lx, 0.5 * Lx, k)
        y = rng.uniform(-0.5 * Ly, 0.5 * Ly, k)
        az = rng.uniform(z_lo, z_hi, k)
        sgn = np.where(rng.uniform(0.0, 1.0, k) < 0.5, -1.0, 1.0)
        if upper_only:
            sgn[:] = 1.0
        cand = np.stack([x, 0.0 * y if planar else y, sgn * az], axis=1)
        ok = np.ones(k, dtype=bool)
        if wall_tree is not None:
            d, _ = wall_tree.query(wq(cand), k=1, distance_upper_bound=min_sep)
            ok &= ~(d < min_sep)
        if len(accepted):
            acc_tree, aq = _periodic_tree(accepted, Lx, Ly, Lz)
            d, _ = acc_tree.query(aq(cand), k=1, distance_upper_bound=min_sep)
            ok &= ~(d < min_sep)
        idx = np.flatnonzero(ok)
        if len(idx) > 1:
            btree, bq = _periodic_tree(cand[idx], Lx, Ly, Lz)
            pairs = btree.query_pairs(min_sep, output_type="ndarray")
            if len(pairs):
                drop = np.unique(pairs.max(axis=1))
                keep = np.ones(len(idx), dtype=bool)
                keep[drop] = False
                idx = idx[keep]
        accepted = np.concatenate([accepted, cand[idx[:need]]], axis=0)
    return np.ascontiguousarray(accepted)


def rsa_in_pores(rng: np.random.Generator, n: int, pores: Sequence[Pore], Lx: float, Ly: float,
                 Lz: float, slab_half: float, obstacles: np.ndarray, min_sep: float = 0.9,
                 max_attempt_factor: int = 1000, planar: bool = False,
              upper_only: bool = False) -> np.ndarray:
    """Random sequential addition of ``n`` points uniform in the carved regions of ``pores`` within
    the slab ``|z| < slab_half``, each at least ``min_sep`` from the obstacle points (wall atoms)
    and from each other. Candidates are drawn uniform in the slab and kept where a pore's
    predicate holds (rejection), in batches as in ``rsa_vapor``."""
    from scipy.spatial import cKDTree
    if n == 0:
        return np.zeros((0, 3))
    obs_tree, oq = (None, None)
    if len(obstacles):
        obs_tree, oq = _periodic_tree(obstacles, Lx, Ly, Lz)
    accepted = np.zeros((0, 3))
    attempts = 0
    while len(accepted) < n:
        need = n - len(accepted)
        k = max(4096, 16 * need)
        attempts += k
        if attempts > max_attempt_factor * 16 * n:
            raise RuntimeError("random sequential addition in the pores did not converge")
        cand = np.stack([rng.uniform(-0.5 * Lx, 0.5 * Lx, k), rng.uniform(-0.5 * Ly, 0.5 * Ly, k),
                         rng.uniform(-slab_half, slab_half, k)], axis=1)
        if planar:
            cand[:, 1] = 0.0
        inside = np.zeros(k, dtype=bool)
        for p in pores:
            inside |= carve_mask(cand, p, Lx, Ly, slab_half)
        cand = cand[inside]
        ok = np.ones(len(cand), dtype=bool)
        if obs_tree is not None and len(cand):
            d, _ = obs_tree.query(oq(cand), k=1, distance_upper_bound=min_sep)
            ok &= ~(d < min_sep)
        if len(accepted) and len(cand):
            acc_tree, aq = _periodic_tree(accepted, Lx, Ly, Lz)
            d, _ = acc_tree.query(aq(cand), k=1, distance_upper_bound=min_sep)
            ok &= ~(d < min_sep)
        idx = np.flatnonzero(ok)
        if len(idx) > 1:
            btree, _ = _periodic_tree(cand[idx], Lx, Ly, Lz)
            pairs = btree.query_pairs(min_sep, output_type="ndarray")
            if len(pairs):
                keep = np.ones(len(idx), dtype=bool)
                keep[np.unique(pairs.max(axis=1))] = False
                idx = idx[keep]
        accepted = np.concatenate([accepted, cand[idx[:need]]], axis=0)
    return np.ascontiguousarray(accepted)


def maxwell_velocities(rng: np.random.Generator, n: int, T0: float, mass: float = 1.0,
                       planar: bool = False) -> np.ndarray:
    if n == 0:
        return np.zeros((0, 3))
    v = rng.normal(0.0, math.sqrt(T0 / mass), size=(n, 3))
    if planar:
        v[:, 1] = 0.0
    v -= v.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(v)


def make_system(name: str, Lx: float, Ly: float, Lz: float, slab_half: float, pores: List[Pore],
                n_vapor: int, T0: float, seed: int, lattice_a: float = 1.0, min_sep: float = 0.9,
                z_lo: Optional[float] = None, z_hi: Optional[float] = None, dt: float = 0.005,
                thermostat_every: int = 10, tau_B: float = 0.0, mass: float = 1.0) -> System:
    rng = np.random.default_rng(seed)
    wall = sc_wall(Lx, Ly, Lz, slab_half, lattice_a, pores) if slab_half > 0 else np.zeros((0, 3))
    zl = slab_half if z_lo is None else z_lo
    zh = 0.5 * Lz if z_hi is None else z_hi
    x0 = rsa_vapor(rng, n_vapor, Lx, Ly, Lz, zl, zh, wall, min_sep)
    v0 = maxwell_velocities(rng, n_vapor, T0, mass)
    return System(name=name, Lx=Lx, Ly=Ly, Lz=Lz, slab_half=slab_half, lattice_a=lattice_a,
                  pores=list(pores), x0=x0, v0=v0, wall=wall, T0=T0, dt=dt, tau_B=tau_B,
                  thermostat_every=thermostat_every, seed=seed)


# ----------------------------------------------------------------------------------------------
# the named workloads (reduced LJ units; rc = 2.5, dt = 0.005, wall eps_w = 1.5, sigma_w = 1)


def cylinder_pore_1k(seed: int = 1) -> System:
    """20x20x40 box, slab |z|<5 (3,480 SC wall sites, a=1), cylinder of radius 4 on the z axis,
    1,000 vapour molecules in 5<|z|<20 at T*=1.0, rescaling every 10 steps."""
    return make_system("cylinder_pore_1k", 20.0, 20.0, 40.0, 5.0, [Pore(PORE_CYLINDER, r0=4.0)],
                       1000, 1.0, seed)


def pore_shape_systems_20k(seeds=(21, 22, 23, 24), n_vapor: int = 20000) -> List[System]:
    """Four 40x40x80 boxes with slab |z|<10 and 20,000 vapour molecules each at T*=1.0:
    cylinder r=5, cone r 3->8 across the slab, slit of width 6 spanning x, ink-bottle
    (neck r=3 through the slab, cavity r=8 at its centre)."""
    pores = [Pore(PORE_CYLINDER, r0=5.0), Pore(PORE_CONE, r0=3.0, r1=8.0),
             Pore(PORE_SLIT, width=6.0), Pore(PORE_INKBOTTLE, r0=3.0, r_cavity=8.0)]
    out = []
    for p, s in zip(pores, seeds):
        out.append(make_system(f"{PORE_KIND_NAMES[p.kind]}_pore_{n_vapor // 1000}k", 40.0, 40.0,
                               80.0, 10.0, [p], n_vapor, 1.0, s))
    return out


def cylinder_pore_200k(seed: int = 3, n_vapor: int = 200000) -> System:
    """150x150x300 box, slab |z|<30 (~1.33 M wall sites), cylinder r=10, 200,000 vapour at T*=0.9."""
    return make_system("cylinder_pore_200k", 150.0, 150.0, 300.0, 30.0,
                       [Pore(PORE_CYLINDER, r0=10.0)], n_vapor, 0.9, seed)


def _replica_box(n: int, rho: float, h: float) -> float:
    """Side L of a box with Lz = 2L holding n molecules at density rho outside a slab |z|<h:
    L^2 (2L - 2h) rho = n, solved by bisection."""
    lo, hi = h + 1e-9, 1e4
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid * mid * (2.0 * mid - 2.0 * h) * rho < n:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def single_parameter_pore(kind: int, R: float, L: float, h: float, r_list: float = 2.8) -> Pore:
    """A pore of ``kind`` described by one size R (radius or width)."""
    if kind == PORE_CYLINDER:
        return Pore(kind, r0=R)
    if kind == PORE_CONE:
        return Pore(kind, r0=R, r1=min(R + 5.0, 0.5 * L - r_list))
    if kind == PORE_SLIT:
        return Pore(kind, width=R)
    if kind == PORE_INKBOTTLE:
        return Pore(kind, r0=R, r_cavity=min(8.0 * R / 3.0, h - 1.0))
    raise ValueError(kind)


def replica_batch_specs(n_replicas: int = 256, seed: int = 4, n_min: int = 1000,
                        n_max: int = 50000, rho: float = 0.02, h: float = 8.0):
    """Draw (kind, R, n, T0, L) for each replica of an uneven batch: kind uniform over the four
    shapes, R ~ U[2, 10], n log-uniform in [n_min, n_max], T0 ~ U[0.8, 1.2]; box L x L x 2L with
    vapour density rho outside the slab |z| < h."""
    rng = np.random.default_rng(seed)
    kinds = rng.integers(1, 5, n_replicas)
    Rs = rng.uniform(2.0, 10.0, n_replicas)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_replicas)).astype(np.int64)
    Ts = rng.uniform(0.8, 1.2, n_replicas)
    specs = []
    for i in range(n_replicas):
        L = _replica_box(int(ns[i]), rho, h)
        specs.append(dict(kind=int(kinds[i]), R=float(Rs[i]), n=int(ns[i]), T0=float(Ts[i]), L=L, h=h))
    return specs


def replica_batch(n_replicas: int = 256, seed: int = 4, n_min: int = 1000, n_max: int = 50000,
                  rho: float = 0.02, h: float = 8.0, init_seed_base: int = 4000) -> List[System]:
    """An uneven batch of independent pore systems (see ``replica_batch_specs``); replica i is
    initialised with seed ``init_seed_base + i``."""
    out = []
    for i, s in enumerate(replica_batch_specs(n_replicas, seed, n_min, n_max, rho, h)):
        L = s["L"]
        pore = single_parameter_pore(s["kind"], s["R"], L, h)
        out.append(make_system(f"replica{i}_{PORE_KIND_NAMES[s['kind']]}", L, L, 2.0 * L, h, [pore],
                               s["n"], s["T0"], init_seed_base + i))
    return out


def pore_array_2m(seed: int = 5, n_vapor: int = 2_000_000, pitch: float = 100.0) -> System:
    """400x400x200 box, slab |z|<20, a 4x4 array of pores on a 100 pitch (kinds uniform over
    cylinder/cone/ink-bottle, R ~ U[4, 10]), 2,000,000 vapour molecules at T*=0.85."""
    rng = np.random.default_rng(seed)
    L, Lz, h = 400.0, 200.0, 20.0
    centres = [-1.5 * pitch, -0.5 * pitch, 0.5 * pitch, 1.5 * pitch]
    kinds = rng.choice([PORE_CYLINDER, PORE_CONE, PORE_INKBOTTLE], size=16)
    Rs = rng.uniform(4.0, 10.0, 16)
    pores = []
    k = 0
    for cy in centres:
        for cx in centres:
            p = single_parameter_pore(int(kinds[k]), float(Rs[k]), L, h)
            p.cx, p.cy = cx, cy
            pores.append(p)
            k += 1
    return make_system("pore_array_2m", L, L, Lz, h, pores, n_vapor, 0.85, seed + 1)


def drying_cylinder_pore(seed: int = 7, n_in: int = 1000, n_out: int = 4800, R: float = 8.0,
                         T0: float = 1.0, tau_B: float = 0.5) -> System:
    """Drying of a pore (the paper's 3D scenario, Sec. 5: a pore filled with saturated vapour
    empties into surroundings at 20 % saturation), in reduced units: a 40x40x80 box, wall slab
    |z|<10 with a cylinder of radius R on the axis; n_in molecules start inside the pore
    (density ~0.25) and n_out outside the slab (~0.05, a fifth of it); T*=1.0, Berendsen
    coupling with tau_B = 0.5 applied every 10 steps. Seed ``seed`` draws the outer molecules,
    ``seed + 1`` the pore filling, ``seed + 2`` the velocities."""
    L, Lz, h = 40.0, 80.0, 10.0
    pore = Pore(PORE_CYLINDER, r0=R)
    wall = sc_wall(L, L, Lz, h, 1.0, [pore])
    inner = rsa_in_pores(np.random.default_rng(seed + 1), n_in, [pore], L, L, Lz, h, wall)
    outer = rsa_vapor(np.random.default_rng(seed), n_out, L, L, Lz, h, 0.5 * Lz,
                      np.concatenate([wall, inner], axis=0))
    x0 = np.ascontiguousarray(np.concatenate([inner, outer], axis=0))
    v0 = maxwell_velocities(np.random.default_rng(seed + 2), len(x0), T0)
    return System(name="drying_cylinder_pore", Lx=L, Ly=L, Lz=Lz, slab_half=h, lattice_a=1.0,
                  pores=[pore], x0=x0, v0=v0, wall=wall, T0=T0, dt=0.005, tau_B=tau_B,
                  thermostat_every=10, seed=seed)


def paper_prism_pore(seed: int = 11, n_in: int = 250, n_out: int = 450, side: float = 5.0,
                     depth: float = 50.0, T0: float = 1.0, tau_B: float = 0.5) -> System:
    """The paper's 3D drying geometry (Sec. 5) in reduced units, with its reflecting walls: a
    rectangular prism pore of cross-section side x side and depth ``depth`` (the paper's 10:1:1
    prism), closed on five faces, its top face open into an outer space nine times the pore volume
    (3 side x 3 side x depth above the slab; periodic in x, y, reflecting at the box top); hard walls,
    no wall atoms. n_in molecules start in the pore and n_out outside, at a fifth of the pore
    density (the paper's saturated pore and 20 % saturated surroundings), T*=1.0, Berendsen
    tau_B = 0.5. Seeds: ``seed`` outer placement, ``seed + 1`` pore filling, ``seed + 2``
    velocities."""
    L = 3.0 * side
    h = 0.5 * depth + 1.0                  # floor at z = h - depth = 1 - depth / 2
    Lz = 2.0 * (h + depth)
    pore = Pore(PORE_PRISM, r0=0.5 * side, r1=0.5 * side, width=depth)
    none = np.zeros((0, 3))
    inner = rsa_in_pores(np.random.default_rng(seed + 1), n_in, [pore], L, L, Lz, h, none)
    outer = rsa_vapor(np.random.default_rng(seed), n_out, L, L, Lz, h, 0.5 * Lz, inner,
                      upper_only=True)
    x0 = np.ascontiguousarray(np.concatenate([inner, outer], axis=0))
    v0 = maxwell_velocities(np.random.default_rng(seed + 2), len(x0), T0)
    return System(name="paper_prism_pore", Lx=L, Ly=L, Lz=Lz, slab_half=h, lattice_a=1.0,
                  pores=[pore], x0=x0, v0=v0, wall=none, T0=T0, dt=0.005, tau_B=tau_B,
                  thermostat_every=10, seed=seed, dims=3, wall_model=1)


def paper_pore_2d(seed: int = 13, n_in: int = 84, n_out: int = 352, lx: float = 20.0,
                  ly: float = 20.0, k: int = 3, T0: float = 1.0, tau_B: float = 0.5) -> System:
    """The paper's 2D geometry (Sec. 4, Fig. 5) in reduced units: a planar system (dims = 2, the x-z
    plane at y = 0) with a pore lx deep and ly wide, reflecting walls on three sides, open into an
    outer space k lx high and (2k + 1) ly wide (21 times the pore for k = 3; periodic in x,
    reflecting at the box top). n_in molecules start in the pore and n_out outside, at a fifth of
    the pore density, T*=1.0, Berendsen tau_B = 0.5. Ly = 9 only spaces the (empty) periodic
    images in y. Seeds: ``seed`` outer, ``seed + 1`` pore, ``seed + 2`` velocities."""
    Lx, Ly = (2 * k + 1) * ly, 9.0
    h = 0.5 * lx + 1.0
    Lz = 2.0 * (h + k * lx)
    pore = Pore(PORE_PRISM, r0=0.5 * ly, r1=1.0e6, width=lx)
    none = np.zeros((0, 3))
    inner = rsa_in_pores(np.random.default_rng(seed + 1), n_in, [pore], Lx, Ly, Lz, h, none,
                         planar=True)
    outer = rsa_vapor(np.random.default_rng(seed), n_out, Lx, Ly, Lz, h, 0.5 * Lz, inner,
                      planar=True, upper_only=True)
    x0 = np.ascontiguousarray(np.concatenate([inner, outer], axis=0))
    v0 = maxwell_velocities(np.random.default_rng(seed + 2), len(x0), T0, planar=True)
    return System(name="paper_pore_2d", Lx=Lx, Ly=Ly, Lz=Lz, slab_half=h, lattice_a=1.0,
                  pores=[pore], x0=x0, v0=v0, wall=none, T0=T0, dt=0.005, tau_B=tau_B,
                  thermostat_every=10, seed=seed, dims=2, wall_model=1)


def vapor_only_box(n: int, L: float, Lz: float, T0: float, seed: int, min_sep: float = 0.9) -> System:
    """A wall-free box (periodic x, y; reflecting z) filled uniformly: used for invariance checks."""
    return make_system(f"vapor_box_{n}", L, L, Lz, 0.0, [], n, T0, seed, min_sep=min_sep,
                       z_lo=0.0, z_hi=0.5 * Lz)
