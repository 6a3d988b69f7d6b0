"""Autotuner of the solve schedule: sweeps per level (nu1, nu2), the FP32 ->
defect-correction switch point, linear V-cycles per correction and the plane
chunk of the fused smoother sweeps, chosen per (N, dtype, GPU) by timing
time-to-tolerance on a seeded synthetic field, cached in a JSON file.

It only times librecon calls (recon_solve through the binding); it computes
nothing itself.
"""
from __future__ import annotations

import json
import os
import time

from . import recon, synth

# tuned schedules, keyed by GPU name, grid size and dtype (written by tune())
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

# candidate values; the search is a coordinate descent from the cached
# config for the same GPU, N and dtype, else from the defaults
SPACE = {
    "nu1": (1, 2, 3),
    "nu2": (1, 2, 3),
    "mixed_switch_rtol": (1e-3, 3e-4, 2e-4, 1.5e-4, 1e-4, 3e-5),
    "mixed_linear_vcycles": (1, 2, 3, 4),
    "fused_chunk": (0, 16, 32, 64),
}


def _key(N: int, dtype: int) -> str:
    import torch
    name = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"
    return f"{name}|N={N}|dtype={dtype}"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cached_config(N: int, dtype: int = recon.RECON_MIXED, path: str = CACHE):
    return load_cache(path).get(_key(N, dtype), {}).get("config")


def _field(N, L, seed, device):
    import torch
    _, dh = synth.linear_field(N, L, 1.0, seed, backend="torch", device=device)
    pos = synth.zeldovich_positions(dh, N, L).contiguous()
    s = recon.Solver(N, L, recon.RECON_F64)
    b = s.smooth_density(s.deposit_cic(pos), 2.0 * L / N)
    s.close()
    return b


def _time(solver, b, tol, reps):
    import torch
    phi = torch.zeros_like(b)
    solver.solve(b, phi=phi, tol=tol, max_cycles=40)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        _, st = solver.solve(b, phi=phi, tol=tol, max_cycles=40)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best, st


def descend(measure, start: dict, space: dict = SPACE, rounds: int = 2, verbose: bool = False):
    """Coordinate descent over `space` from `start`.  measure(cfg) returns
    (seconds, converged) or None when the config is rejected; a candidate is
    kept only if it converged and is faster than the best so far, so the
    result is never slower than `start`.  Returns (best_cfg, best_seconds,
    number of configs measured)."""
    best_cfg = dict(start)
    m = measure(best_cfg)
    if m is None or not m[1]:
        raise ValueError("the starting config does not converge")
    best_t, n = m[0], 1
    for _ in range(rounds):
        improved = False
        for k, values in space.items():
            for v in values:
                if v == best_cfg[k]:
                    continue
                cand = dict(best_cfg, **{k: v})
                if cand.get("nu1", 1) + cand.get("nu2", 1) < 1:
                    continue
                m = measure(cand)
                if m is None:
                    continue
                n += 1
                if verbose:
                    print(f"  {cand} -> {m[0] * 1e3:.2f} ms")
                if m[1] and m[0] < best_t:
                    best_t, best_cfg, improved = m[0], cand, True
        if not improved:
            break
    return best_cfg, best_t, n


def tune(N: int, L: float | None = None, dtype: int = recon.RECON_MIXED, tol: float = 1e-8,
         reps: int = 2, path: str = CACHE, rounds: int = 2, verbose: bool = False) -> dict:
    """Coordinate descent over SPACE, started from the cached config for this
    (GPU, N, dtype) when there is one (else from the defaults), so a re-tune
    never replaces a schedule with a slower one; returns and caches the best."""
    import torch
    L = float(L if L is not None else N)
    b = _field(N, L, 9000 + N, torch.device("cuda", 0))
    solver = recon.Solver(N, L, dtype)
    base = solver.config()
    defaults = {k: base[k] for k in SPACE}

    def measure(cfg):
        solver.configure(**cfg)
        try:
            t, st = _time(solver, b, tol, reps)
        except recon.ReconError:
            return None
        return t, st["rel_residual"] < tol

    m = measure(defaults)
    default_t = m[0] if m is not None and m[1] else float("inf")
    # start from the cached schedule or the defaults, whichever is faster now
    # (kernels change: a schedule tuned for older ones can fall behind)
    start = cached_config(N, dtype, path) or defaults
    if start != defaults:
        mc = measure(start)
        if mc is None or not mc[1] or mc[0] > default_t:
            start = defaults
    try:
        best_cfg, best_t, n = descend(measure, start, SPACE, rounds, verbose)
    except ValueError:   # a cached schedule that no longer converges
        best_cfg, best_t, n = descend(measure, defaults, SPACE, rounds, verbose)
    solver.close()
    cache = load_cache(path)
    cache[_key(N, dtype)] = {"config": best_cfg, "seconds": best_t, "trials": n + 1,
                             "default_seconds": default_t}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(cache, f, indent=1)
    return cache[_key(N, dtype)]


def apply(solver_or_batch, N: int | None = None, dtype: int = recon.RECON_MIXED,
          path: str = CACHE) -> bool:
    """Apply a cached config (if any) to a Solver or Batch; True if applied."""
    if isinstance(solver_or_batch, recon.Batch):
        ok = False
        for i, n in enumerate(solver_or_batch.sizes):
            cfg = cached_config(n, dtype, path)
            if cfg:
                h = solver_or_batch.handle(i)
                c = recon.recon_get_config(h)
                for k, v in cfg.items():
                    setattr(c, k, v)
                recon.recon_set_config(h, c)
                ok = True
        return ok
    cfg = cached_config(N or solver_or_batch.N, dtype, path)
    if cfg:
        solver_or_batch.configure(**cfg)
        return True
    return False
