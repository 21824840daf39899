"""The seeded input recipe: every workload has the shapes, sizes and parameter ranges its
documentation states, the same seed gives the same instances, and sharding partitions a
workload over ranks.  (Parameters only: nothing here runs the lattice Boltzmann method.)"""
import math

import numpy as np
import pytest

from paper_2509_22308_gb300 import workloads as W


def _check_instance(i):
    """What every instance must satisfy to be run by both sides."""
    assert i["period"] >= 4 and i["period"] % 3 == 0, i          # T = 3 lambda, lambda an integer
    assert i["ramp"] == i["period"]
    cx, cy = (i["nx"] - 1) / 2.0, (i["ny"] - 1) / 2.0
    # the contour encloses the cylinder and lies strictly inside the lattice
    assert i["a"] < i["R"]
    assert 1.0 <= cx - i["R"] and cx + i["R"] <= i["nx"] - 2
    assert 1.0 <= cy - i["R"] and cy + i["R"] <= i["ny"] - 2
    assert i["eps1"] >= 1.0 and (i["pec2"] or i["eps2"] >= 1.0)


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_every_instance_is_runnable(name):
    for i in W.WORKLOADS[name]():
        _check_instance(i)


def test_benchmark_workload_md_janus_512():
    ins = W.md_janus_512()
    assert len(ins) == 7
    assert [round(math.degrees(i["phi0"])) for i in ins] == list(range(0, 181, 30))
    for i in ins:
        assert (i["nx"], i["ny"], i["a"], i["period"], i["periods"], i["R"]) == (512, 512, 32.0, 96, 30, 64.0)
        assert i["pec2"] and 2.0 <= i["eps1"] <= 10.0
    # a / lambda = 1, as in the paper's metallo-dielectric maps
    assert ins[0]["a"] == ins[0]["period"] / 3
    # seeded: the same seed gives the same instances, another rank's seed others
    assert W.md_janus_512() == ins
    assert W.rank_workload("md_janus_512", 0) == ins
    other = W.rank_workload("md_janus_512", 1)
    assert [i["eps1"] for i in other] != [i["eps1"] for i in ins]


def test_dielectric_janus_2048_size_parameters_and_settled_runs():
    ins = W.dielectric_janus_2048()
    assert len(ins) == 15
    lams = sorted({i["period"] // 3 for i in ins})
    assert lams == [40, 80, 161]
    for i in ins:
        k0a = 2 * math.pi * i["a"] / (i["period"] / 3)
        assert min(abs(k0a - k) / k for k in (5.0, 10.0, 20.0)) < 0.01
        assert i["eps1"] == 2.0 and not i["pec2"] and i["eps2"] in (2.0, 4.5, 7.0, 9.5, 12.0)
        assert i["R"] == pytest.approx(1.6 * 128)
    # 20 periods after the incident front (speed 1/3) has crossed the contour
    assert sorted({i["periods"] for i in ins}) == [28, 36, 51]
    for i in ins:
        front = 3.0 * ((i["nx"] - 1) / 2.0 + i["R"])
        assert (i["periods"] - 20 - 1) * i["period"] < front <= (i["periods"] - 20) * i["period"]


def test_design_map_256_ranges_and_uneven_sizes():
    ins = W.design_map_256()
    assert len(ins) == 256
    sizes = {i["nx"] for i in ins}
    assert sizes == {256, 512, 1024}                      # uneven grids, all three present
    for i in ins:
        assert i["nx"] == i["ny"] == 16 * i["a"] and i["a"] in (16.0, 32.0, 64.0)
        assert i["period"] == 3 * i["a"] and i["periods"] == 20
        assert 2.0 <= i["eps2"] <= 12.0 and i["eps1"] == 2.0 and not i["pec2"]
        assert 0.0 <= i["phi0"] <= math.pi
    assert W.design_map_256() == ins
    assert W.design_map_256(n=10) == ins[:10]


def test_md_janus_8192_size_parameter():
    (i,) = W.md_janus_8192()
    assert (i["nx"], i["a"], i["period"]) == (8192, 512.0, 240)
    assert 2 * math.pi * i["a"] / 80 == pytest.approx(40.2, abs=0.05)   # k0 a ~ 40
    assert 2.0 <= i["eps1"] <= 12.0 and i["pec2"]
    s = W.settled(i)
    assert s["periods"] == W.transit_periods(8192, 8192, 240, i["R"]) + 20 > i["periods"]


def test_small_cases_are_ragged():
    ins = W.small_cases()
    assert any(i["nx"] % 32 for i in ins) and any(i["ny"] % 8 for i in ins)
    assert any(i["nx"] != i["ny"] for i in ins)
    assert {i["pec2"] for i in ins} == {True, False}


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_shard_partitions_a_workload(world):
    ins = W.design_map_256(n=37)
    parts = [W.shard(ins, r, world) for r in range(world)]
    assert sum(len(p) for p in parts) == len(ins)
    got = sorted((id(x) for p in parts for x in p))
    assert got == sorted(id(x) for x in ins)                # every instance exactly once
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_workloads_module_is_independent_of_both_sides():
    """The module that serves the CUDA path and the oracle imports neither of them (only the
    standard library and numpy), and its instances hold plain parameters."""
    import ast
    tree = ast.parse(open(W.__file__).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {n.name.split(".")[0] for n in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add((node.module or "").split(".")[0])
    assert mods <= {"__future__", "math", "numpy"}, mods
    assert all(isinstance(v, (int, float, bool)) for i in W.small_cases() for v in i.values())
    assert np.isfinite([i["eps2"] for i in W.design_map_256()]).all()
