"""The C-ABI library: builds, loads, exports every entry point declared in include/md.h, and the
Python binding's struct layouts match the C compiler's. CPU only (no kernel is launched)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1812_07993_gb300 as md
from paper_1812_07993_gb300 import build as mdbuild
from paper_1812_07993_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


@pytest.fixture(scope="module")
def lib():
    mdbuild.build()
    return md.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", md.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(md_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)
    assert set(md._SIGNATURES) == set(names)


def test_struct_layout_matches_c(tmp_path):
    structs = {"md_pore": md.md_pore, "md_system": md.md_system, "md_potential": md.md_potential,
               "md_tuning": md.md_tuning, "md_obs": md.md_obs}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "md.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_status_strings(lib):
    for s in range(8):
        assert lib.md_status_string(s) and lib.md_status_string(s) != b"unknown status"
    assert lib.md_status_string(99) == b"unknown status"


def test_checked_build_exports_every_declared_function():
    """The MD_CHECKED variant (index checks reporting MD_EBOUNDS) builds and exports the same
    entry points."""
    path = mdbuild.build(checked=True)
    assert path.endswith("libmd_checked.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(md_\w+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def small_system(**kw):
    s = W.make_system("t", 12.0, 12.0, 20.0, 3.0, [W.Pore(W.PORE_CYLINDER, r0=3.0)], 20, 1.0, 1)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("change,fragment", [
    (dict(Lx=7.0), "3 cells"),
    (dict(dt=0.0), "dt"),
    (dict(thermostat_every=10, tau_B=0.01), "tau_B"),
    (dict(x0=np.array([[100.0, 0.0, 0.0]] * 20)), "outside the box"),
    (dict(dt=float("inf")), "finite"),
    (dict(T0=float("nan")), "finite"),
    (dict(tau_B=float("nan")), "finite"),
    (dict(pores=[W.Pore(W.PORE_CYLINDER, r0=float("nan"))]), "pore parameters must be finite"),
])
def test_invalid_systems_rejected_before_any_gpu_work(lib, change, fragment):
    s = small_system(**change)
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s)
    assert ei.value.status == md.MD_EINVAL
    assert fragment in str(ei.value)


def test_invalid_potential_rejected(lib):
    s = small_system()
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s, W.Potential(r_ads=3.0))
    assert ei.value.status == md.MD_EINVAL and "r_ads" in str(ei.value)
    with pytest.raises(md.MDError):
        md.Simulation(s, W.Potential(sigma=0.0))
    for bad in (dict(eps=float("inf")), dict(skin=float("nan")), dict(rc=float("inf"))):
        with pytest.raises(md.MDError) as ei:
            md.Simulation(s, W.Potential(**bad))
        assert ei.value.status == md.MD_EINVAL and "not finite" in str(ei.value)


def test_unknown_pore_kind_rejected(lib):
    s = small_system(pores=[W.Pore(9, r0=1.0)])
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s, generate_wall=True)
    assert ei.value.status == md.MD_EINVAL


def planar_system(**kw):
    s = W.paper_pore_2d(n_in=10, n_out=20)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("make,fragment", [
    (lambda: planar_system(wall_model=0), "planar system needs hard walls"),
    (lambda: planar_system(pores=[W.Pore(W.PORE_SLIT, width=4.0)]), "planar system needs prism"),
    (lambda: planar_system(x0=np.where(np.arange(30)[:, None] == 3, [0.0, 0.5, 0.0],
                                       planar_system().x0)), "y = 0"),
    (lambda: planar_system(dims=4), "dims"),
    (lambda: small_system(wall_model=1), "prism or slit"),
    (lambda: small_system(wall_model=7), "unknown wall model"),
    (lambda: small_system(pores=[W.Pore(W.PORE_PRISM, r0=0.0, r1=2.0, width=3.0)]), "half-sides"),
])
def test_invalid_geometry_rejected_before_any_gpu_work(lib, make, fragment):
    """Planar systems, hard walls and prism pores: the argument checks run before any CUDA call."""
    s = make()
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s)
    assert ei.value.status == md.MD_EINVAL
    assert fragment in str(ei.value)


def test_hard_walls_take_no_wall_atoms(lib):
    s = W.paper_prism_pore(n_in=10, n_out=20)
    s.wall = np.array([[0.0, 0.0, 0.0]])
    with pytest.raises(md.MDError) as ei:
        md.Simulation(s)
    assert ei.value.status == md.MD_EINVAL and "no wall atoms" in str(ei.value)
