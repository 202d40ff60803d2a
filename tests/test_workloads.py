"""The seeded input generator: geometry counts, placement constraints, reproducibility."""
import numpy as np
import pytest

from paper_1812_07993_gb300 import workloads as W


def min_periodic_distance(a, b, Lx, Ly, same=False):
    d = a[:, None, :] - b[None, :, :]
    d[..., 0] -= Lx * np.round(d[..., 0] / Lx)
    d[..., 1] -= Ly * np.round(d[..., 1] / Ly)
    r = np.sqrt((d ** 2).sum(-1))
    if same:
        np.fill_diagonal(r, np.inf)
    return r.min()


def test_small_cylinder_system():
    s = W.cylinder_pore_1k()
    assert s.n_wall == 3480 and s.n_vapor == 1000       # 10 layers x 348 sites
    z = np.abs(s.x0[:, 2])
    assert (z > 5).all() and (z < 20).all()
    assert min_periodic_distance(s.x0, s.x0, 20, 20, same=True) >= 0.9
    assert min_periodic_distance(s.x0, s.wall, 20, 20) >= 0.9
    assert np.abs(s.v0.mean(0)).max() < 1e-12
    assert abs((s.v0 ** 2).mean() - 1.0) < 0.1
    rxy = np.hypot(s.wall[:, 0], s.wall[:, 1])
    assert rxy.min() >= 4.0 and (np.abs(s.wall[:, 2]) < 5).all()


def test_maxwell_velocities_statistics():
    """Per component N(0, T0/m) minus the sample mean: zero mean exactly, each component's
    variance within 4 standard errors of T0/m (standard error T0/m sqrt(2/n)), a Gaussian's
    kurtosis 3 (standard error sqrt(24/n)), uncorrelated components; planar draws have vy = 0."""
    n, T0, m = 200_000, 0.85, 1.0
    v = W.maxwell_velocities(np.random.default_rng(11), n, T0, mass=m)
    assert np.abs(v.mean(0)).max() < 1e-12
    var = v.var(0)
    assert np.all(np.abs(var - T0 / m) < 4 * (T0 / m) * np.sqrt(2.0 / n))
    kurt = (v ** 4).mean(0) / var ** 2
    assert np.all(np.abs(kurt - 3.0) < 4 * np.sqrt(24.0 / n))
    c = np.corrcoef(v.T)
    assert np.abs(c[np.triu_indices(3, 1)]).max() < 4 / np.sqrt(n)
    vp = W.maxwell_velocities(np.random.default_rng(12), 1000, T0, planar=True)
    assert (vp[:, 1] == 0.0).all() and np.abs(vp.mean(0)).max() < 1e-12


def test_reproducible_by_seed():
    a, b = W.cylinder_pore_1k(), W.cylinder_pore_1k()
    np.testing.assert_array_equal(a.x0, b.x0)
    np.testing.assert_array_equal(a.v0, b.v0)
    c = W.cylinder_pore_1k(seed=2)
    assert not np.array_equal(a.x0, c.x0)


def test_pore_shape_wall_counts():
    counts = [W.sc_wall(40, 40, 80, 10, 1.0, [p]).shape[0] for p in [
        W.Pore(W.PORE_CYLINDER, r0=5.0), W.Pore(W.PORE_CONE, r0=3.0, r1=8.0),
        W.Pore(W.PORE_SLIT, width=6.0), W.Pore(W.PORE_INKBOTTLE, r0=3.0, r_cavity=8.0)]]
    assert counts == [30400, 29976, 27200, 29680]


def test_replica_specs_ranges():
    specs = W.replica_batch_specs(256, seed=4)
    assert len(specs) == 256
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 1000 and ns.max() <= 50000
    for s in specs:
        L = s["L"]
        assert s["n"] / (L * L * (2 * L - 16)) == pytest.approx(0.02, rel=1e-6)
        assert 2 <= s["R"] <= 10 and 0.8 <= s["T0"] <= 1.2 and s["kind"] in (1, 2, 3, 4)
    assert specs == W.replica_batch_specs(256, seed=4)


def test_drying_pore_filled_inside_dilute_outside():
    s = W.drying_cylinder_pore()
    assert s.n_vapor == 5800 and s.tau_B == 0.5 and s.thermostat_every == 10
    inside = W.carve_mask(s.x0, s.pores[0], s.Lx, s.Ly, s.slab_half) & (np.abs(s.x0[:, 2]) < 10)
    outside = np.abs(s.x0[:, 2]) > 10
    assert inside.sum() == 1000 and outside.sum() == 4800
    assert min_periodic_distance(s.x0, s.x0, 40, 40, same=True) >= 0.9
    assert min_periodic_distance(s.x0[inside], s.wall, 40, 40) >= 0.9
    rho_in = 1000 / (np.pi * 8.0 ** 2 * 20.0)
    rho_out = 4800 / (40.0 * 40.0 * 60.0)
    assert rho_out / rho_in == pytest.approx(0.2, abs=0.02)
    b = W.drying_cylinder_pore()
    np.testing.assert_array_equal(s.x0, b.x0)


def test_bench_workload_names_build_their_own_systems():
    """Every workload name the bench accepts builds that workload (the 4x20k pore shapes are the
    fallback, so a name the builder missed would silently time them instead); the two largest
    are checked by name only, their generation taking tens of seconds."""
    import bench
    for name in sorted(bench.WORKLOADS):
        if name in ("pore_array_2m", "replica_batch_256"):
            continue
        systems, label = bench.make_workload(name)
        assert label == name
        if name == "replica_batch_32":
            assert len(systems) == 32
            assert sum(s.n_vapor for s in systems) == 461031
            assert sum(len(s.wall) for s in systems) == 2392655
    import inspect
    src = inspect.getsource(bench.make_workload)
    for name in ("pore_array_2m", "replica_batch_256"):
        assert f'name == "{name}"' in src
