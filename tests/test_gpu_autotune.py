"""The schedule autotuner finds a config that converges no slower than the
default and caches it."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_autotune_small_grid(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import autotune, build, recon
    build.build()
    path = str(tmp_path / "tune.json")
    res = autotune.tune(64, 64.0, reps=1, rounds=1, path=path)
    assert res["seconds"] <= res["default_seconds"] * 1.05
    cfg = autotune.cached_config(64, path=path)
    assert cfg == res["config"]
    s = recon.Solver(64, 64.0, recon.RECON_MIXED)
    assert autotune.apply(s, path=path)
    assert all(s.config()[k] == v for k, v in cfg.items())
    b = autotune._field(64, 64.0, 1, torch.device("cuda", 0))
    _, st = s.solve(b, tol=1e-8)
    assert st["rel_residual"] < 1e-8
    s.close()
