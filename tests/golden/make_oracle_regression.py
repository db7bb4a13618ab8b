"""Writes tests/golden/oracle_regression.json: oracle outputs on seeded inputs, a regression
snapshot (not a pin: the pins are tests/test_oracle_pins.py and closed_forms.json). It calls only
the oracle and the seeded input generators. Run from the repository root:
    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import grf_inputs as gi  # noqa: E402
import oracle  # noqa: E402


def generic_point(seed):
    rng = np.random.default_rng(seed)
    v = rng.uniform(-0.2, 0.2, 27)
    v[0] = rng.uniform(0.3, 1.0)
    for m, d in zip(range(1, 7), [1, 0, 0, 1, 0, 1]):
        v[m] = d + rng.uniform(-0.15, 0.15)
    v[18] = rng.uniform(0.4, 1.0)
    return v, rng.normal(size=(27, 3)) * 0.3, rng.normal(size=(27, 6)) * 0.3


def snapshot():
    p = gi.Params(lam=0.3, g2=0.2, beta_kind=1)
    v, d1, d2 = generic_point(2024)
    rhs, diag, st = oracle.point_rhs(p, v, d1, d2)
    out = {
        "_about": "Oracle outputs on seeded inputs (regression snapshot, written by make_oracle_regression.py).",
        "params": p.to_dict(),
        "point_seed": 2024,
        "point_rhs": rhs.tolist(),
        "point_rho8_S8_LGB": diag[:11].tolist(),
        "point_constraints": oracle.point_constraints(p, v, d1, d2).tolist(),
        "point_energy": oracle.point_energy(p, v, d1, d2).tolist(),
    }
    psi = oracle.point_psi4(p, v, d1, d2, np.array([0.7, -0.4, 1.1]))
    out["point_psi4_xyz"] = [0.7, -0.4, 1.1]
    out["point_psi4"] = [psi.real, psi.imag]
    box = gi.Box(12, 11, 10, 0.3, -1.65, -1.5, -1.35, bc=gi.BC_PERIODIC)
    s = gi.random_perturbed_state(box, 5, base=gi.single_puncture(box, amp=0.05), eps=2e-2)
    oracle.fill_ghosts(box, s)
    a = oracle.extract_modes(box, s[25], None, 0, 1.2, (0.05, -0.05, 0.1), 8, 16, 3)
    out["modes_phi_l3"] = {"box": [12, 11, 10, 0.3, -1.65, -1.5, -1.35], "state_seed": 5, "radius": 1.2,
                           "centre": [0.05, -0.05, 0.1], "ntheta": 8, "nphi": 16,
                           "re": a.real.tolist(), "im": a.imag.tolist()}
    r = oracle.rhs(box, p, s)
    out["box_rhs_interior_sum_abs_per_field"] = np.sum(np.abs(box.interior(r)), axis=(1, 2, 3)).tolist()
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as fh:
        json.dump(snapshot(), fh, indent=1)
    print("wrote", path)
