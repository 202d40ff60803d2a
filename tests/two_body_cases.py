"""Two-body systems for the pair-force sweep, and their exact forces.

Each case is one replica holding a single vapour pair, or one molecule and one wall atom, at a
separation drawn in [0.8, 2.499] sigma along a random direction; some pairs straddle the periodic
edge in x or y. Coordinates sit on a 2^-20 grid, which makes every coordinate difference exact in
FP64: what is left to test is the pair term's own arithmetic (r^2, 1/r^2, the powers, the force
factor). The exact force is the Lennard-Jones pair force of Eq. 2 (Sec. 2) evaluated in
rational arithmetic (``fractions.Fraction``) on the very doubles the code under test reads -- the
positions, and the constants 48 eps sigma^12 and 24 eps sigma^6 -- so the only error left in a
result is that of its own floating-point evaluation.

Error scale: S = |F_rep| + |F_att| = (48 eps sigma^12 r^-13 + 24 eps sigma^6 r^-7), the sum of the
magnitudes of the two terms, since the force itself passes through zero at r = 2^(1/6) sigma.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from paper_1812_07993_gb300 import workloads as W

BOX = 9.0          # at least 3 list cells of rc + skin = 2.8 across x and y
R_MIN, R_MAX = 0.8, 2.499
GRID = 2.0 ** 20   # coordinates are multiples of 1 / GRID


def cases(n_vapour_pairs: int = 192, n_wall_pairs: int = 96, seed: int = 2024):
    """Systems (one replica each) and, per system, the pair's (i, j-or-wall) positions."""
    rng = np.random.default_rng(seed)
    systems = []
    for k in range(n_vapour_pairs + n_wall_pairs):
        wall = k >= n_vapour_pairs
        r = rng.uniform(R_MIN, R_MAX)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        # the pair's midpoint: near the periodic edge in x or y for a quarter of the cases
        c = rng.uniform(-1.0, 1.0, size=3)
        if k % 4 == 1:
            c[0] = 0.5 * BOX - 0.2 * r
        elif k % 4 == 2:
            c[1] = -0.5 * BOX + 0.3 * r
        a = c + 0.5 * r * u
        b = c - 0.5 * r * u
        for p in (a, b):
            # on a 2^-20 grid, so that every coordinate difference (with or without the periodic
            # shift) is exact in FP64 and the only rounding left is the pair term's own; then x, y
            # wrapped into [-L/2, L/2) (the box side is a multiple of the grid)
            p[:] = np.round(p * GRID) / GRID
            p[:2] -= BOX * np.floor((p[:2] + 0.5 * BOX) / BOX)
        x0 = a.reshape(1, 3) if wall else np.stack([a, b])
        v0 = np.zeros_like(x0)
        wxyz = b.reshape(1, 3) if wall else np.zeros((0, 3))
        systems.append(W.System(name=f"two_body_{k}", Lx=BOX, Ly=BOX, Lz=BOX, slab_half=0.0,
                                lattice_a=1.0, pores=[], x0=x0, v0=v0, wall=wxyz, T0=1.0,
                                thermostat_every=0))
    return systems


def _image(d: Fraction, L: Fraction) -> Fraction:
    if d >= L / 2:
        return d - L
    if d < -L / 2:
        return d + L
    return d


def exact_force(xi, xj, eps: float, sigma: float):
    """Exact force on i from j (a list of three Fractions) and the error scale S (a float)."""
    s6 = Fraction(sigma) ** 6
    a12 = Fraction(48.0 * eps * float(s6 * s6))   # the doubles the codes hold
    b6 = Fraction(24.0 * eps * float(s6))
    L = Fraction(BOX)
    d = [Fraction(float(xi[0])) - Fraction(float(xj[0])),
         Fraction(float(xi[1])) - Fraction(float(xj[1])),
         Fraction(float(xi[2])) - Fraction(float(xj[2]))]
    d[0], d[1] = _image(d[0], L), _image(d[1], L)
    r2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
    inv2 = 1 / r2
    inv6 = inv2 ** 3
    fr = inv2 * inv6 * (a12 * inv6 - b6)
    scale = float(inv2 * inv6 * (a12 * inv6 + b6)) * float(r2) ** 0.5
    return [fr * c for c in d], scale


def errors(systems, forces_per_system, potential=None):
    """Per case, |F_got - F_exact| / S for the force on the first molecule (and, for a vapour
    pair, the second)."""
    pot = potential or W.Potential()
    out = []
    for s, f in zip(systems, forces_per_system):
        wall = s.n_wall == 1
        xj = s.wall[0] if wall else s.x0[1]
        eps, sig = (pot.eps_w, pot.sigma_w) if wall else (pot.eps, pot.sigma)
        fe, scale = exact_force(s.x0[0], xj, eps, sig)
        targets = [(0, fe)] if wall else [(0, fe), (1, [-c for c in fe])]
        for row, ex in targets:
            dev = [float(Fraction(float(f[row][k])) - ex[k]) for k in range(3)]
            out.append(float(np.sqrt(sum(e * e for e in dev))) / scale)
    return np.array(out)
