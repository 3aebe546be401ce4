"""The pipe workload's derived parameters against the values the paper
prints (Table 1; Sec. 2.1): friction velocity u_tau = Re_tau nu / R, wall
unit ratio dx / y_tau = u_tau / nu, and the bulk Reynolds number 2 U R / nu
of about 5300 for the bulk velocity U = 14.7 u_tau used by the workload."""
import json
import os

import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_pipe.json")


def rows():
    return json.load(open(GOLDEN))["rows"]


@pytest.mark.parametrize("row", rows(), ids=lambda r: r["case"])
def test_friction_velocity_and_wall_unit(row):
    p = workloads.pipe_parameters(row["R"], row["nu"], row["re_tau"])
    # printed to three significant figures
    assert p["u_tau"] == pytest.approx(row["u_tau"], abs=5e-6)
    assert p["u_tau"] / row["nu"] == pytest.approx(row["dx_over_y_tau"], abs=5e-3)
    assert p["tau"] == pytest.approx(3 * row["nu"] + 0.5)


def test_bulk_reynolds_number():
    d = json.load(open(GOLDEN))
    for row in d["rows"]:
        p = workloads.pipe_parameters(row["R"], row["nu"], row["re_tau"])
        re_bulk = 2 * p["u_bulk"] * row["R"] / row["nu"]
        assert re_bulk == pytest.approx(d["re_bulk"], rel=0.01)
