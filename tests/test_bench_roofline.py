"""The bench line's roofline object for every scheme the bl_pair workloads can run (4th / 6th
order, centred / lopsided advection, with and without the cubic term), on the CPU: each builds,
the fractions recompute from the line's own fields, and the per-kernel capture constants are used
only for the kernel they were taken from."""
import importlib.util
import os

import pytest

import grf_inputs as gi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("decoupled", [0, 1])
@pytest.mark.parametrize("ng", [3, 4])
@pytest.mark.parametrize("advection", [0, 1])
@pytest.mark.parametrize("g3", [0.0, 0.1])
def test_roofline_record_builds_for_every_scheme(bench, ng, advection, g3, decoupled):
    params = gi.Params(lam=0.05, g2=0.01, advection=advection, g3=g3, decoupled=decoupled)
    npts = 256 ** 3
    launch_ms = 126.0
    clk = {"sm_mhz": 2070.0}
    roof, scheme, default = bench.roofline_record(ng, params, npts, launch_ms, 3.3e7, clk, None)
    assert scheme == {"order": 2 * ng - 2, "advection": "lopsided" if advection else "centred"}
    assert default == (ng == 3 and advection == 0 and g3 == 0.0 and not decoupled)
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(bench.FLOP_ALG_PER_POINT_STAGE * npts / (launch_ms * 1e-3) / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    if decoupled:
        assert "overstate" in roof["note"]
    elif not default:
        assert "lower bounds" in roof["note"]
    # capture constants only for the kernel they were taken from (none of the decoupled kernels)
    key = (2 * ng - 2, "lopsided" if advection else "centred", g3 != 0.0)
    instr, want = (None, None) if decoupled else bench.STAGE_CAPTURES.get(key, (None, None))
    assert roof["traffic"] == (want * npts if want else None)
    assert (roof.get("fp64_issue") or {}).get("instr_per_point_stage") == instr
    if "fp64_issue" in roof:
        f = roof["fp64_issue"]
        assert roof["fp64_issue_frac"] == pytest.approx(f["instr_per_s"] / f["ceiling"])
        assert f["ceiling"] == pytest.approx(2 * 152 * 2070e6)
