"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics (not to itself).

Each test names the passage of arXiv:1812.07993 whose arithmetic it pins. A plausible mistake in
the oracle -- a dropped term, a wrong sign, a transposed operand, a wrong integrator order -- fails
at least one of them:
  * LJ closed forms (Sec. 2): zero force at 2^(1/6) sigma, energy -eps there, U(sigma) = 0,
    F(sigma) = 24 eps / sigma, the truncation values at rc.
  * force = -grad E by central finite differences (Eq. 2).
  * Newton's third law: zero net force and conserved x/y momentum without walls.
  * all pairs == cell list == an independent brute-force pair enumeration.
  * integrator (Figs. 2, 3): exact ballistic flight with specular reflection, time reversibility,
    second-order energy error of a bound dimer.
  * thermostat (Fig. 4): rescaling reaches T0 exactly; the Berendsen relation for general tau_B.
  * observables: hand-placed molecules inside/outside each pore shape, adsorption threshold,
    bin edges, ideal-gas occupancy.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1812_07993_gb300 import workloads as W


def P(**kw):
    return oracle.make_params(**kw)


# ---------------------------------------------------------------- Sec. 2: the LJ 12-6 pair


def exact_lj(r2: Fraction, eps: Fraction, sigma: Fraction):
    """U and F(r)/r from the textbook 12-6 form, in exact rational arithmetic."""
    s6 = (sigma * sigma / r2) ** 3
    u = 4 * eps * (s6 * s6 - s6)
    f_over_r = 24 * eps * (2 * s6 * s6 - s6) / r2
    return f_over_r, u


@pytest.mark.parametrize("r2", [Fraction(1), Fraction(81, 100), Fraction(5, 4), Fraction(9, 4),
                                Fraction(625, 100), Fraction(3, 2)])
@pytest.mark.parametrize("eps,sigma", [(Fraction(1), Fraction(1)), (Fraction(3, 2), Fraction(1)),
                                       (Fraction(1), Fraction(11, 10))])
def test_lj_matches_exact_rational(r2, eps, sigma):
    fr, u = oracle.lj(float(r2), float(eps), float(sigma))
    efr, eu = exact_lj(r2, eps, sigma)
    assert fr == pytest.approx(float(efr), rel=1e-14, abs=1e-14)
    assert u == pytest.approx(float(eu), rel=1e-14, abs=1e-14)


def test_lj_special_points():
    rmin2 = 2.0 ** (1.0 / 3.0)               # r = 2^(1/6) sigma
    fr, u = oracle.lj(rmin2)
    assert abs(fr) < 1e-13 and u == pytest.approx(-1.0, abs=1e-14)
    fr, u = oracle.lj(rmin2, eps=1.5)       # wall pair minimum is -eps_w
    assert abs(fr) < 1e-13 and u == pytest.approx(-1.5, abs=1e-14)
    fr, u = oracle.lj(1.0)                  # U(sigma) = 0, F(sigma) = 24 eps / sigma (repulsive)
    assert u == 0.0 and fr == pytest.approx(24.0, rel=1e-15)
    fr, u = oracle.lj(2.5 ** 2)             # cutoff values: U(2.5) = -0.0163169, |F| = 0.0389994
    assert u == pytest.approx(4 * (2.5 ** -12 - 2.5 ** -6), rel=1e-14)
    assert u == pytest.approx(-0.016316891136, abs=1e-11)
    assert fr * 2.5 == pytest.approx(-0.0389994775, abs=1e-9)


def two_body(r, direction, eps_w=None):
    """Two molecules (or molecule + wall atom) at separation r along ``direction``."""
    d = np.asarray(direction, float) / np.linalg.norm(direction)
    xi = np.array([0.3, -0.2, 0.1])
    xj = xi - r * d
    p = P(Lx=20.0, Ly=20.0, Lz=20.0)
    if eps_w is None:
        f, _, st = oracle.forces(p, np.stack([xi, xj]), None, method=0)
        return f, st, d
    p.eps_w = eps_w
    f, d2, st = oracle.forces(p, xi[None, :], xj[None, :], method=0)
    return f, st, d


@pytest.mark.parametrize("r", [0.95, 1.05, 1.12, 1.3, 2.0, 2.49])
def test_two_body_force_vector_and_third_law(r):
    f, st, d = two_body(r, [0.3, -0.7, 0.65])
    F = 24.0 / r * (2 * r ** -12 - r ** -6)        # -dU/dr, positive = repulsive
    np.testing.assert_allclose(f[0], F * d, rtol=1e-13, atol=1e-15)   # on i, along r_i - r_j
    np.testing.assert_allclose(f[1], -F * d, rtol=1e-13, atol=1e-15)
    assert st["pairs_vv"] == 1 and st["pairs_vw"] == 0
    U = 4 * (r ** -12 - r ** -6) - 4 * (2.5 ** -12 - 2.5 ** -6)
    assert st["pe_vv"] == pytest.approx(U, rel=1e-13, abs=1e-15)
    assert st["vir_vv"] == pytest.approx(F * r, rel=1e-13, abs=1e-15)


def test_cutoff_is_strict_and_excludes_far_pairs():
    for r, pairs in [(2.5, 0), (2.5 - 1e-9, 1), (2.6, 0)]:
        _, st, _ = two_body(r, [1.0, 0.0, 0.0])
        assert st["pairs_vv"] == pairs


def test_wall_pair_uses_wall_parameters_and_acts_on_vapor_only():
    r = 1.3
    f, st, d = two_body(r, [0.2, 0.9, -0.4], eps_w=1.5)
    F = 1.5 * 24.0 / r * (2 * r ** -12 - r ** -6)
    np.testing.assert_allclose(f[0], F * d, rtol=1e-13)
    assert st["pairs_vw"] == 1 and st["pairs_vv"] == 0
    U = 1.5 * 4 * ((r ** -12 - r ** -6) - (2.5 ** -12 - 2.5 ** -6))
    assert st["pe_vw"] == pytest.approx(U, rel=1e-13)


# ---------------------------------------------------------------- Eq. 2: f = -dU/dr


def random_cluster(n, L, seed, min_sep=0.95, nwall=0, Lz=None):
    rng = np.random.default_rng(seed)
    Lz = L if Lz is None else Lz
    pts = []
    while len(pts) < n + nwall:
        c = np.array([rng.uniform(-L / 2, L / 2), rng.uniform(-L / 2, L / 2),
                      rng.uniform(-Lz / 2 + 0.5, Lz / 2 - 0.5)])
        ok = True
        for q in pts:
            d = c - q
            d[:2] -= L * np.round(d[:2] / L)
            if d @ d < min_sep ** 2:
                ok = False
                break
        if ok:
            pts.append(c)
    pts = np.array(pts)
    return pts[:n].copy(), pts[n:].copy()


def total_pe(p, x, w):
    _, _, st = oracle.forces(p, x, w, method=0)
    return st["pe_vv"] + st["pe_vw"]


def pair_distances(x, w, L):
    allp = np.concatenate([x, w]) if len(w) else x
    d = x[:, None, :] - allp[None, :, :]
    d[..., :2] -= L * np.round(d[..., :2] / L)
    return np.sqrt((d ** 2).sum(-1))


def test_force_is_minus_gradient_of_energy():
    L = 9.0
    x, w = random_cluster(40, L, seed=7, nwall=25)
    p = P(Lx=L, Ly=L, Lz=L, eps_w=1.5)
    f, _, _ = oracle.forces(p, x, w, method=0)
    h = 1e-5
    r = pair_distances(x, w, L)
    checked = 0
    for i in range(len(x)):
        near_cut = np.any(np.abs(r[i] - 2.5) < 10 * h)
        if near_cut:
            continue
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            g = (total_pe(p, xp, w) - total_pe(p, xm, w)) / (2 * h)
            assert f[i, c] == pytest.approx(-g, rel=2e-6, abs=2e-6 * max(1.0, abs(f[i]).max()))
        checked += 1
    assert checked > 30


# ---------------------------------------------------------------- Newton's third law


def test_net_force_vanishes_without_walls():
    s = W.vapor_only_box(300, 10.0, 12.0, 1.0, seed=11)
    p = P(Lx=s.Lx, Ly=s.Ly, Lz=s.Lz)
    f, _, _ = oracle.forces(p, s.x0, None, method=1)
    assert np.abs(f.sum(0)).max() < 1e-12 * np.abs(f).sum()


def test_xy_momentum_conserved_over_1000_steps():
    s = W.vapor_only_box(200, 9.0, 10.0, 1.0, seed=12)
    p = P(Lx=s.Lx, Ly=s.Ly, Lz=s.Lz, thermostat_every=0)
    st = oracle.State(p, s.x0, s.v0 + np.array([0.3, -0.2, 0.0]), None)
    p0 = st.v.sum(0)
    st.run(1000)
    p1 = st.v.sum(0)
    assert abs(p1[0] - p0[0]) < 1e-10 and abs(p1[1] - p0[1]) < 1e-10


def test_vapor_wall_path_equals_vapor_vapor_path_for_equal_parameters():
    """With eps_w = eps and sigma_w = sigma a wall atom acts like a (frozen) vapour molecule."""
    L = 9.0
    x, w = random_cluster(30, L, seed=3, nwall=30)
    p = P(Lx=L, Ly=L, Lz=L, eps_w=1.0, sigma_w=1.0)
    f_wall, _, st_w = oracle.forces(p, x, w, method=0)
    f_all, _, st_all = oracle.forces(p, np.concatenate([x, w]), None, method=0)
    np.testing.assert_allclose(f_wall, f_all[: len(x)], rtol=1e-12, atol=1e-12)
    r_ww = pair_distances(w, np.zeros((0, 3)), L)
    ww_pairs = int(np.triu(r_ww < 2.5, k=1).sum())
    assert st_w["pairs_vv"] + st_w["pairs_vw"] + ww_pairs == st_all["pairs_vv"]


# ---------------------------------------------------------------- cell list == all pairs == brute force


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cell_list_equals_all_pairs_and_brute_force(seed):
    rng = np.random.default_rng(seed)
    L, Lz = 10.4, 15.6                                   # 4 x 4 x 6 cells of side 2.6
    n, nw = 150, 60
    x = np.stack([rng.uniform(-L / 2, L / 2, n), rng.uniform(-L / 2, L / 2, n),
                  rng.uniform(-Lz / 2, Lz / 2, n)], 1)
    w = np.stack([rng.uniform(-L / 2, L / 2, nw), rng.uniform(-L / 2, L / 2, nw),
                  rng.uniform(-2, 2, nw)], 1)
    # molecules exactly on cell faces and on the periodic boundary
    x[:10, 0] = -L / 2 + 2.6 * rng.integers(0, 4, 10)
    x[10:20, 1] = -L / 2 + 2.6 * rng.integers(0, 4, 10)
    x[20:25, 2] = -Lz / 2 + 2.6 * rng.integers(0, 6, 5)
    x[25, 2] = Lz / 2
    p = P(Lx=L, Ly=L, Lz=Lz, rc=2.5, rc_w=2.5, eps_w=1.5)
    # keep pairs away from r = 0 (huge forces are fine, but not infinities)
    r = pair_distances(x, w, L)
    np.fill_diagonal(r[:, :n], 10.0)
    assert r.min() > 1e-3
    f0, d0, s0 = oracle.forces(p, x, w, method=0)
    f1, d1, s1 = oracle.forces(p, x, w, method=1)
    assert s0["pairs_vv"] == s1["pairs_vv"] and s0["pairs_vw"] == s1["pairs_vw"]
    scale = np.sqrt((f0 ** 2).sum(1).mean())
    assert np.abs(f0 - f1).max() <= 1e-13 * scale
    np.testing.assert_array_equal(d0, d1)
    # independent brute-force enumeration of the pair sets
    rv = r[:, :n]
    assert int(np.triu(rv < 2.5, k=1).sum()) == s0["pairs_vv"]
    assert int((r[:, n:] < 2.5).sum()) == s0["pairs_vw"]
    d2min = np.where(r[:, n:] < 2.5, r[:, n:] ** 2, np.inf).min(1)
    np.testing.assert_allclose(d0, d2min, rtol=1e-12)


def test_threads_do_not_change_results():
    s = W.cylinder_pore_1k()
    p = oracle.make_params(s, W.Potential())
    f1, d1, s1 = oracle.forces(p, s.x0, s.wall, method=1, nthreads=1)
    f4, d4, s4 = oracle.forces(p, s.x0, s.wall, method=1, nthreads=4)
    np.testing.assert_array_equal(f1, f4)
    assert s1 == s4


# ---------------------------------------------------------------- Figs. 2-3: velocity Verlet


def fold(z, Lz):
    """Position of a free particle after specular reflections off z = +-Lz/2 (closed form)."""
    u = np.mod(z + Lz / 2, 2 * Lz)
    return np.where(u <= Lz, u, 2 * Lz - u) - Lz / 2


def test_ballistic_flight_with_specular_reflection():
    Lx, Ly, Lz, dt = 12.0, 14.0, 16.0, 0.005
    x0 = np.array([[1.0, -2.0, 3.0]])
    v0 = np.array([[3.7, -5.3, 11.9]])
    p = P(Lx=Lx, Ly=Ly, Lz=Lz, dt=dt)
    st = oracle.State(p, x0, v0, None)
    n = 700
    st.run(n)
    t = n * dt
    ex = np.mod(x0[0, 0] + v0[0, 0] * t + Lx / 2, Lx) - Lx / 2
    ey = np.mod(x0[0, 1] + v0[0, 1] * t + Ly / 2, Ly) - Ly / 2
    ez = fold(x0[0, 2] + v0[0, 2] * t, Lz)
    np.testing.assert_allclose(st.x[0], [ex, ey, ez], atol=1e-11)
    nref = int(np.floor((x0[0, 2] + v0[0, 2] * t + Lz / 2) / Lz))
    assert st.v[0, 2] == pytest.approx(v0[0, 2] * (-1) ** nref)
    np.testing.assert_allclose(st.v[0, :2], v0[0, :2])


def test_time_reversibility():
    s = W.make_system("rev", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_CYLINDER, r0=3.0)], 150, 1.0, 5)
    p = oracle.make_params(s, W.Potential(), thermostat_every=0)
    st = oracle.State(p, s.x0, s.v0, s.wall)
    st.run(200)
    st.v = -st.v
    st.run(200)
    d = st.x - s.x0
    d[:, :2] -= np.array([s.Lx, s.Ly]) * np.round(d[:, :2] / np.array([s.Lx, s.Ly]))
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-st.v, s.v0, atol=1e-9)


def dimer_energy_error(dt, t_total=2.0):
    p = P(Lx=20.0, Ly=20.0, Lz=20.0, dt=dt)
    x = np.array([[0.0, 0.0, 0.0], [1.05, 0.3, -0.2]])
    v = np.array([[0.2, -0.1, 0.3], [-0.2, 0.1, -0.3]])
    st = oracle.State(p, x, v, None)
    e0 = oracle.kinetic(p, st.v) + st.stats["pe_vv"]
    ke, pe = st.run(int(round(t_total / dt)))
    return np.abs(ke + pe - e0).max()


def test_velocity_verlet_energy_error_is_second_order():
    e1 = dimer_energy_error(0.004)
    e2 = dimer_energy_error(0.002)
    assert 3.6 < e1 / e2 < 4.4
    assert e1 < 1e-3


# ---------------------------------------------------------------- Fig. 4: thermostat


def test_rescaling_reaches_T0_exactly():
    s = W.make_system("th", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_SLIT, width=4.0)], 200, 1.7, 9)
    p = oracle.make_params(s, W.Potential(), thermostat_every=10, T0=1.0, tau_B=0.0)
    st = oracle.State(p, s.x0, s.v0, s.wall)
    st.run(10)
    T = (st.v ** 2).sum() / (3 * len(st.v))
    assert T == pytest.approx(1.0, rel=1e-13)


def test_berendsen_relation_for_general_tau():
    s = W.make_system("th2", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_CONE, r0=2.0, r1=4.0)], 200,
                      1.4, 10)
    n_th, dt, tau = 10, 0.005, 0.4
    p = oracle.make_params(s, W.Potential(), thermostat_every=n_th, T0=0.8, tau_B=tau)
    st = oracle.State(p, s.x0, s.v0, s.wall)
    ke, _ = st.run(n_th)
    T_before = 2 * ke[-1] / (3 * len(st.v))
    T_after = (st.v ** 2).sum() / (3 * len(st.v))
    assert T_after == pytest.approx(T_before + (n_th * dt / tau) * (0.8 - T_before), rel=1e-12)
    # no rescaling on the other steps
    ke2, _ = st.run(5)
    assert abs(2 * ke2[-1] / (3 * len(st.v)) - T_after) < 0.2


# ---------------------------------------------------------------- observables


def obs_for(points, pores, Lx=40.0, Ly=40.0, Lz=40.0, slab_half=10.0, d2wall=None, **kw):
    p = P(Lx=Lx, Ly=Ly, Lz=Lz, slab_half=slab_half, **kw)
    x = np.asarray(points, float)
    d2 = np.full(len(x), np.inf) if d2wall is None else np.asarray(d2wall, float)
    return oracle.observables(p, pores, x, d2)


@pytest.mark.parametrize("pore,inside,outside", [
    (W.Pore(W.PORE_CYLINDER, r0=4.0), [[0, 0, 0], [3.9, 0, 9.9], [0, -3.9, -9.9], [2.8, 2.8, 1]],
     [[4.1, 0, 0], [0, 0, 10.1], [2.9, 2.9, 0]]),
    (W.Pore(W.PORE_CONE, r0=3.0, r1=8.0), [[2.9, 0, -9.9], [5.4, 0, 0], [0, 7.9, 9.95]],
     [[3.2, 0, -9.9], [5.6, 0, 0], [0, 8.1, 9.95]]),
    (W.Pore(W.PORE_SLIT, width=6.0), [[15, 2.9, 0], [-19, -2.9, 5], [0, 0, -9.9]],
     [[0, 3.1, 0], [5, -3.1, 0], [0, 0, 10.5]]),
    (W.Pore(W.PORE_INKBOTTLE, r0=3.0, r_cavity=8.0), [[7.9, 0, 0], [2.9, 0, 9.9], [0, 4.5, 6.5]],
     [[4, 0, 7.5], [8.1, 0, 0], [3.1, 0, 9.9]]),
])
def test_occupancy_hand_placed(pore, inside, outside):
    for pt in inside:
        occ, _, prof = obs_for([pt], [pore])
        assert occ[0] == 1, pt
    for pt in outside:
        occ, _, prof = obs_for([pt], [pore])
        assert occ[0] == 0, pt
    occ, _, prof = obs_for(inside + outside, [pore])
    assert occ[0] == len(inside)
    assert prof.sum() == len(inside) + len(outside)


def test_pore_offset_axis_and_periodic_image():
    pore = W.Pore(W.PORE_CYLINDER, cx=18.0, cy=-18.0, r0=4.0)
    # (-19.5, 19.5) is (1.5, -2.5) from the axis across both periodic boundaries (L = 40)
    occ, _, _ = obs_for([[-19.5, 19.5, 0.0], [10.0, -10.0, 0.0]], [pore])
    assert occ[0] == 1


def test_adsorbed_threshold_and_group_assignment():
    wall = np.array([[0.0, 0.0, 0.0], [20.0 - 0.5, 0.0, 0.0]])
    # molecules 2 and 3 see the second wall atom across the periodic boundary in x (L = 40)
    x = np.array([[1.4, 0.0, 0.0], [0.0, 1.6, 0.0], [-19.0, 0.0, 0.0], [-19.0, 0.0, 1.0]])
    p = P(Lx=40.0, Ly=40.0, Lz=40.0, slab_half=10.0, eps_w=1.5)
    _, d2, _ = oracle.forces(p, x, wall, method=0)
    np.testing.assert_allclose(d2, [1.96, 2.56, 2.25, 3.25], rtol=1e-12)
    pores = [W.Pore(W.PORE_CYLINDER, cx=0.0, cy=0.0, r0=3.0),
             W.Pore(W.PORE_CYLINDER, cx=-18.0, cy=0.0, r0=3.0)]
    occ, ads, prof = oracle.observables(p, pores, x, d2)
    # molecules 0, 1 belong to pore 0; 2, 3 to pore 1 (nearest axis). d < 1.5: molecules 0 only
    # in group 0; molecule 2 at distance 1.5 exactly is not adsorbed (strict), 3 is not either
    assert list(ads) == [1, 0]
    assert list(prof.sum(1)) == [2, 2]
    assert list(occ) == [2, 2]


def test_profile_bin_edges():
    Lz = 40.0
    x = np.array([[0, 0, -20.0], [0, 0, 20.0], [0, 0, 0.0], [0, 0, -0.25], [1, 1, 19.75]])
    _, _, prof = obs_for(x, [], Lz=Lz, slab_half=0.0)
    assert prof.shape == (1, 80)
    assert prof[0, 0] == 1 and prof[0, 79] == 2 and prof[0, 40] == 1 and prof[0, 39] == 1


def test_ideal_gas_occupancy_and_flat_profile():
    rng = np.random.default_rng(1)
    n, L, Lz, h, R = 200000, 20.0, 40.0, 5.0, 4.0
    x = np.stack([rng.uniform(-L / 2, L / 2, n), rng.uniform(-L / 2, L / 2, n),
                  rng.uniform(-Lz / 2, Lz / 2, n)], 1)
    occ, _, prof = obs_for(x, [W.Pore(W.PORE_CYLINDER, r0=R)], Lx=L, Ly=L, Lz=Lz, slab_half=h)
    p_in = math.pi * R * R * 2 * h / (L * L * Lz)
    mean, sd = n * p_in, math.sqrt(n * p_in * (1 - p_in))
    assert abs(occ[0] - mean) < 5 * sd
    expected = n / prof.shape[1]
    chi2 = ((prof[0] - expected) ** 2 / expected).sum()
    assert chi2 < prof.shape[1] + 6 * math.sqrt(2 * prof.shape[1])


# ---------------------------------------------------------------- Sec. 2: virial pressure per pore


def test_pore_volume_closed_forms_and_monte_carlo():
    p = P(Lx=40.0, Ly=40.0, Lz=60.0, slab_half=10.0)
    cyl = W.Pore(W.PORE_CYLINDER, r0=5.0)
    cone = W.Pore(W.PORE_CONE, r0=3.0, r1=8.0)
    slit = W.Pore(W.PORE_SLIT, width=6.0)
    ink = W.Pore(W.PORE_INKBOTTLE, r0=3.0, r_cavity=8.0)
    assert oracle.pore_volume(p, cyl) == pytest.approx(math.pi * 25 * 20, rel=1e-12)
    assert oracle.pore_volume(p, cone) == pytest.approx(math.pi / 3 * 20 * (9 + 24 + 64), rel=1e-12)
    assert oracle.pore_volume(p, slit) == pytest.approx(6.0 * 40.0 * 20.0, rel=1e-12)
    # ink-bottle: neck cylinder plus the part of the sphere outside it (Monte Carlo, independent)
    rng = np.random.default_rng(5)
    n = 2_000_000
    pts = np.stack([rng.uniform(-9, 9, n), rng.uniform(-9, 9, n), rng.uniform(-10, 10, n)], 1)
    inside = W.carve_mask(pts, ink, 40.0, 40.0, 10.0)
    mc = inside.mean() * 18 * 18 * 20
    assert oracle.pore_volume(p, ink) == pytest.approx(mc, rel=5e-3)


def test_pore_pressure_kinetic_and_pair_terms():
    L, h = 20.0, 5.0
    pore = W.Pore(W.PORE_CYLINDER, r0=4.0)
    p = P(Lx=L, Ly=L, Lz=40.0, slab_half=h)
    V = math.pi * 16 * 2 * h
    # one molecule moving inside the pore, nothing to interact with: P = m v^2 / (3 V)
    x = np.array([[0.5, 0.0, 1.0]])
    v = np.array([[0.3, -1.2, 0.7]])
    wv = oracle.molecule_virials(p, x, None)
    assert oracle.pore_pressure(p, [pore], x, v, wv)[0] == pytest.approx(
        (0.09 + 1.44 + 0.49) / (3 * V), rel=1e-13)
    # two molecules at rest, both in the pore: P = r F(r) / (3 V); one outside: its half is dropped
    r = 1.1
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    wv = oracle.molecule_virials(p, x, None)
    rF = 24.0 * (2 * r ** -12 - r ** -6)
    assert wv.sum() == pytest.approx(rF, rel=1e-13)
    assert oracle.pore_pressure(p, [pore], x, np.zeros_like(x), wv)[0] == pytest.approx(
        rF / (3 * V), rel=1e-13)
    x2 = np.array([[0.0, 0.0, 4.6], [0.0, 0.0, 4.6 + r]])   # second molecule above the slab
    wv2 = oracle.molecule_virials(p, x2, None)
    assert oracle.pore_pressure(p, [pore], x2, np.zeros_like(x2), wv2)[0] == pytest.approx(
        0.5 * rF / (3 * V), rel=1e-13)
    # a wall atom acts on the molecule only, fully counted
    wall = np.array([[1.3, 0.0, 0.0]])
    x3 = np.array([[0.0, 0.0, 0.0]])
    wv3 = oracle.molecule_virials(p, x3, wall)
    assert wv3[0] == pytest.approx(1.5 * 24.0 * (2 * 1.3 ** -12 - 1.3 ** -6), rel=1e-13)


# ------------------------------------------------ hard walls, prism pores, planar systems
# The paper's reflecting pore walls (Sec. 4 and Sec. 5): the slab minus the pores is a solid that
# reflects molecules specularly. Pinned by free flight between parallel mirrors (closed form),
# by never entering the solid, by energy conservation, and by the planar system's invariants.

def unfold(x0, v, t, a, b):
    """Free flight between specular walls at a and b: position and the sign of the velocity."""
    L = b - a
    u = np.mod(x0 - a + v * t, 2.0 * L)
    return (a + u, 1.0) if u <= L else (a + 2.0 * L - u, -1.0)


PRISM = W.Pore(W.PORE_PRISM, cx=1.0, cy=-2.0, r0=3.0, r1=2.0, width=12.0)


def test_prism_pore_ballistic_reflections_off_sides_and_floor():
    """One molecule in a blind prism pore (slab |z| < 8, floor at z = -4), no forces: x and y fold
    between the side walls, z between the floor and (not reached) the top."""
    dt, n = 0.005, 400
    p = P(Lx=30.0, Ly=30.0, Lz=40.0, dt=dt, slab_half=8.0, hard_walls=1)
    x0 = np.array([[1.5, -1.2, 0.0]])
    v0 = np.array([[7.3, -5.1, -3.3]])
    st = oracle.State(p, x0, v0, None, pores=[PRISM])
    st.run(n)
    t = n * dt
    ex, sx = unfold(1.5, 7.3, t, -2.0, 4.0)
    ey, sy = unfold(-1.2, -5.1, t, -4.0, 0.0)
    ez, sz = unfold(0.0, -3.3, t, -4.0, 1e6)
    np.testing.assert_allclose(st.x[0], [ex, ey, ez], atol=1e-10)
    np.testing.assert_allclose(st.v[0], [7.3 * sx, -5.1 * sy, -3.3 * sz], rtol=1e-14)


def test_molecule_above_the_slab_reflects_off_its_top_face():
    dt, n = 0.005, 600
    p = P(Lx=30.0, Ly=30.0, Lz=40.0, dt=dt, slab_half=8.0, hard_walls=1)
    x0 = np.array([[-10.0, 5.0, 12.0]])
    v0 = np.array([[0.5, 0.2, -6.1]])
    st = oracle.State(p, x0, v0, None, pores=[PRISM])
    st.run(n)
    t = n * dt
    ez, sz = unfold(12.0, -6.1, t, 8.0, 20.0)       # slab top face and the box wall
    np.testing.assert_allclose(st.x[0], [-10.0 + 0.5 * t, 5.0 + 0.2 * t, ez], atol=1e-10)
    assert st.v[0, 2] == pytest.approx(-6.1 * sz, rel=1e-14)


def hard_wall_gas(dims, seed, n_in=60, n_out=90):
    s = (W.paper_pore_2d(seed=seed, n_in=n_in, n_out=n_out) if dims == 2 else
         W.paper_prism_pore(seed=seed, n_in=n_in, n_out=n_out))
    return s, oracle.make_params(s, W.Potential(), thermostat_every=0)


@pytest.mark.parametrize("dims", [3, 2])
def test_hard_walls_keep_molecules_out_of_the_solid_and_conserve_energy(dims):
    s, p = hard_wall_gas(dims, 31)
    assert oracle.in_solid(p, s.pores, s.x0).sum() == 0
    st = oracle.State(p, s.x0, s.v0, None, pores=s.pores)
    e0 = oracle.kinetic(p, st.v) + st.stats["pe_vv"]
    emax = 0.0
    for _ in range(20):
        ke, pe = st.run(100)
        assert oracle.in_solid(p, s.pores, st.x).sum() == 0
        emax = max(emax, np.abs(ke + pe - e0).max() / len(st.x))
    assert emax < 2e-3                                 # reflections conserve kinetic energy
    if dims == 2:
        assert (st.x[:, 1] == 0.0).all() and (st.v[:, 1] == 0.0).all() and (st.f[:, 1] == 0.0).all()


def test_planar_thermostat_uses_2n_degrees_of_freedom():
    s, _ = hard_wall_gas(2, 33)
    p = oracle.make_params(s, W.Potential(), thermostat_every=10, T0=0.7, tau_B=0.0)
    assert p.dims == 2
    st = oracle.State(p, s.x0, s.v0, None, pores=s.pores)
    st.run(10)
    assert (st.v ** 2).sum() / (2 * len(st.v)) == pytest.approx(0.7, rel=1e-13)


def test_prism_volume_area_and_occupancy():
    p3 = P(Lx=30.0, Ly=30.0, Lz=40.0, slab_half=8.0)
    assert oracle.pore_volume(p3, PRISM) == pytest.approx(6.0 * 4.0 * 12.0, rel=1e-12)
    through = W.Pore(W.PORE_PRISM, r0=3.0, r1=2.0, width=0.0)
    assert oracle.pore_volume(p3, through) == pytest.approx(6.0 * 4.0 * 16.0, rel=1e-12)
    p2 = P(Lx=30.0, Ly=9.0, Lz=40.0, slab_half=8.0, dims=2)
    assert oracle.pore_volume(p2, PRISM) == pytest.approx(6.0 * 12.0, rel=1e-12)
    inside = [[1.0, -2.0, 0.0], [3.9, -0.1, -3.9], [-1.9, -3.9, 7.9]]
    outside = [[1.0, -2.0, -4.1], [4.1, -2.0, 0.0], [1.0, 0.1, 0.0], [1.0, -2.0, 8.1]]
    occ, _, _ = obs_for(inside + outside, [PRISM], Lx=30.0, Ly=30.0, Lz=40.0, slab_half=8.0)
    assert occ[0] == len(inside)


def test_planar_pore_pressure_divides_by_2_area():
    """A free planar gas inside a 2D pore: P = sum m v^2 / (2 A)."""
    p = P(Lx=30.0, Ly=9.0, Lz=40.0, slab_half=8.0, dims=2)
    x = np.array([[0.5, 0.0, 0.0], [2.0, 0.0, -3.0], [20.0, 0.0, 12.0]])
    v = np.array([[1.0, 0.0, 2.0], [-0.5, 0.0, 0.3], [3.0, 0.0, 3.0]])
    planar = W.Pore(W.PORE_PRISM, cx=1.0, cy=0.0, r0=3.0, r1=1e6, width=12.0)
    press = oracle.pore_pressure(p, [planar], x, v, np.zeros(3))
    assert press[0] == pytest.approx((5.0 + 0.34) / (2.0 * 6.0 * 12.0), rel=1e-12)


def test_two_body_sweep_against_exact_rational_forces():
    """480 pair forces (vapour pairs from both ends and vapour-wall pairs, separations 0.8-2.499,
    random directions, some across the periodic edge) against Eq. 2 evaluated exactly in rational
    arithmetic on the same doubles: every deviation within 1e-15 of the pair's error scale S (the
    sum of the repulsive and attractive magnitudes, about 9 ulps), 3e-16 in the RMS -- FP64
    evaluation to a few ulps, not merely close."""
    import two_body_cases as T
    systems = T.cases()
    pot = W.Potential()
    got = []
    for s in systems:
        g, _, _ = oracle.forces(oracle.make_params(s, pot), s.x0, s.wall, method=0)
        got.append(g)
    e = T.errors(systems, got, pot)
    assert e.max() <= 1e-15
    assert np.sqrt((e ** 2).mean()) <= 3e-16
