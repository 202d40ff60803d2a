"""Host logic of the skin autotuner (autotune.choose_skin) with a stand-in context: which
candidates it keeps, how it ranks them, and what it records. No GPU: the stand-in replaces the
library's Simulation, and the clock is the stand-in's."""
import pytest

import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import autotune
from paper_1812_07993_gb300 import workloads as W

# per skin: seconds per timed step and rebuilds per timed step, or an error the context raises
PLAN = {
    0.2: dict(sec=2.0e-3, reb=0.25),
    0.3: dict(sec=1.5e-3, reb=0.17),
    0.4: dict(sec=1.1e-3, reb=0.13),
    0.5: dict(error="create"),          # refused at creation (cells do not fit)
    0.6: dict(sec=1.2e-3, reb=0.10),
    0.8: dict(error="step"),            # list overflow found while stepping
}


# per cell scale (cell side / (rc + skin)): a factor on the seconds per step, or a refusal
CELL_PLAN = {1.0: 1.0, 1.25: 0.8, 1.5: 0.9, 2.0: "create"}


class FakeSim:
    clock = 0.0

    def __init__(self, systems, potential, precision=0, stream=None):
        self.plan = dict(PLAN[potential.skin])
        scale = 1.0
        if potential.cell_size:
            scale = round(potential.cell_size / (max(potential.rc, potential.rc_w) + potential.skin), 6)
        factor = CELL_PLAN[scale]
        if self.plan.get("error") == "create" or factor == "create":
            raise md.MDError(md.MD_EINVAL, "box x/y must hold at least 3 cells")
        if "sec" in self.plan:
            self.plan["sec"] *= factor
        self.steps = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def autotune(self, trials):
        return {}, 1.0

    def step(self, n):
        if self.plan.get("error") == "step":
            raise md.MDError(md.MD_EOVERFLOW, "neighbour list overflow")
        self.steps += n
        FakeSim.clock += n * self.plan["sec"]

    def sync(self):
        pass

    def observables(self, r):
        return ({"n_rebuilds": round(self.steps * self.plan["reb"])},)


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(autotune, "Simulation", FakeSim)
    monkeypatch.setattr(autotune.time, "perf_counter", lambda: FakeSim.clock)


def test_choose_skin_keeps_the_fastest_and_records_the_refused(fake):
    got = autotune.choose_skin([W.cylinder_pore_1k()], steps=100, warmup=20)
    assert got["skin"] == 0.4
    rows = {r["skin"]: r for r in got["table"]}
    assert set(rows) == set(PLAN)
    assert rows[0.4]["steps_per_s"] == pytest.approx(1 / 1.1e-3)
    # rebuilds over the timed steps only: 120 steps less the 20 of the warm-up
    assert rows[0.2]["rebuilds"] == 30 - 5 and rows[0.6]["rebuilds"] == 12 - 2
    assert "error" in rows[0.5] and "cells" in rows[0.5]["error"]
    assert "error" in rows[0.8] and "overflow" in rows[0.8]["error"]


def test_choose_skin_with_no_usable_candidate(fake):
    got = autotune.choose_skin([W.cylinder_pore_1k()], skins=(0.5, 0.8))
    assert got["skin"] is None and len(got["table"]) == 2


def test_choose_geometry_picks_skin_then_cell_side_and_caches(fake, tmp_path):
    cache = str(tmp_path / "tune.json")
    got = autotune.choose_geometry([W.cylinder_pore_1k()], steps=100, warmup=20,
                                   cache_path=cache)
    assert got["skin"] == 0.4 and not got["cached"]
    assert got["cell_size"] == pytest.approx(1.25 * 2.9)
    rows = {r["scale"]: r for r in got["cell_table"]}
    assert set(rows) == {1.25, 1.5, 2.0} and "error" in rows[2.0]
    assert rows[1.25]["steps_per_s"] == pytest.approx(1 / (0.8 * 1.1e-3))
    again = autotune.choose_geometry([W.cylinder_pore_1k()], cache_path=cache)
    assert again["cached"] and again["skin"] == 0.4 and again["cell_size"] == got["cell_size"]
