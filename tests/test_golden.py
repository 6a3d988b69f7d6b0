"""Values the paper prints, stored with their citations under tests/golden/,
checked against the oracle."""
import os

import numpy as np
import pytest

from paper_1709_06350_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """key value pairs of a fixture; lines starting with # are its citation."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, value = line.split()
                out[key] = float(value)
    return out


def test_update_derivative(O):
    """At random cells of a smooth field, moving theta_c changes s = lap + 3
    by the printed -6/h^2 per unit and leaves p and q unchanged (up to the
    rounding of forming the traceless part as H - tr/3, where theta_c cancels
    only in exact arithmetic)."""
    g = read_golden("update_derivative.txt")
    N, h = 12, 1.5
    t = synth.smooth_field(N, 5, 0.6, kmax=3)
    zero = np.zeros_like(t)
    rng = np.random.default_rng(9)
    for _ in range(5):
        i, j, k = rng.integers(0, N, 3)
        eps = 1e-4
        tp, tm = t.copy(), t.copy()
        tp[i, j, k] += eps
        tm[i, j, k] -= eps
        sp, pp, qp = O.cubic_grid(tp, zero, 0.0, h)
        sm, pm, qm = O.cubic_grid(tm, zero, 0.0, h)
        ds = (sp[i, j, k] - sm[i, j, k]) / (2 * eps)
        dp = (pp[i, j, k] - pm[i, j, k]) / (2 * eps)
        dq = (qp[i, j, k] - qm[i, j, k]) / (2 * eps)
        assert ds * h * h == pytest.approx(g["dL_dtheta_times_h2"], rel=1e-9)
        assert abs(dp) < 1e-9 * abs(ds) and abs(dq) < 1e-9 * abs(ds)


def test_cubic_test_closed_form(O):
    """The paper's cubic test at a quarter of its size in every dimension
    (the printed cube/box ratio kept, 32^3 particles and mesh): inside the
    cube the oracle's Laplacian equals 3 (b_in^(1/3) - 1), which is the
    printed configuration's 3 (box/cube - 1) when no mass is lost to the
    floor (the closed form is checked for the paper's numbers too)."""
    g = read_golden("cubic_test.txt")
    ratio = g["box_side_mpc_h"] / g["cube_side_mpc_h"]
    assert 3.0 * (ratio - 1.0) == pytest.approx(35.4)
    N = int(g["particles_per_side"]) // 4
    L = float(N)
    l = L / ratio
    b = O.smooth_and_floor(O.cic_deposit(synth.cube_positions(N, L, l), N, L), L, 0.0)
    c = N // 2
    assert b[c, c, c] ** (1.0 / 3.0) == pytest.approx(ratio, rel=0.05)   # the floor takes a little
    t, info = O.solve(b, L, tol=1e-3, max_cycles=80)
    assert info["status"] == 0
    lap = sum(np.roll(t, -1, a) + np.roll(t, 1, a) - 2 * t for a in range(3))
    expect = 3.0 * (b[c, c, c] ** (1.0 / 3.0) - 1.0)
    assert np.all(np.abs(lap[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] / expect - 1.0) < 1e-3)
