"""The schedule autotuner's coordinate descent (host logic, no GPU): it finds
the optimum of a separable cost over the discrete space, never returns a
config slower than its start, and never keeps one that did not converge."""
import pytest

from paper_1709_06350_gb300 import autotune

SPACE = {"nu1": (1, 2, 3), "nu2": (1, 2, 3), "mixed_switch_rtol": (1e-3, 1e-4, 3e-5),
         "mixed_linear_vcycles": (1, 2, 3, 4), "fused_chunk": (0, 16, 32)}
OPT = {"nu1": 2, "nu2": 3, "mixed_switch_rtol": 1e-4, "mixed_linear_vcycles": 3, "fused_chunk": 16}


def cost(cfg):
    """separable bowl with its minimum at OPT"""
    t = 1.0
    for k, vals in SPACE.items():
        t += 0.1 * abs(vals.index(cfg[k]) - vals.index(OPT[k]))
    return t


def test_descent_finds_the_separable_optimum():
    start = {"nu1": 1, "nu2": 1, "mixed_switch_rtol": 1e-3, "mixed_linear_vcycles": 1, "fused_chunk": 0}
    best, t, n = autotune.descend(lambda c: (cost(c), True), start, SPACE)
    assert best == OPT and t == pytest.approx(1.0)
    assert n > 1


def test_descent_never_worse_than_its_start_and_skips_unconverged():
    start = dict(OPT, nu1=3)
    seen = []

    def measure(c):
        seen.append(dict(c))
        if c["fused_chunk"] == 32:
            return None                 # rejected (e.g. an invalid config)
        if c["nu1"] == 2:
            return 0.5, False           # faster but did not reach the tolerance
        return cost(c), True

    best, t, _ = autotune.descend(measure, start, SPACE)
    assert t <= cost(start)
    assert best["nu1"] != 2 and best["fused_chunk"] != 32
    assert any(c["nu1"] == 2 for c in seen)


def test_descent_rejects_an_unconverged_start():
    with pytest.raises(ValueError):
        autotune.descend(lambda c: (1.0, False), dict(OPT), SPACE)
