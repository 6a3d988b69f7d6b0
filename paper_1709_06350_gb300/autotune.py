"""Autotuner of the solve schedule: sweeps per level (nu1, nu2), the FP32 ->
defect-correction switch point, linear V-cycles per correction and the plane
chunk of the fused smoother sweeps, chosen per (N, dtype, GPU) by timing
time-to-tolerance on a seeded synthetic field, cached in a JSON file.

It only times librecon calls (recon_solve through the binding); it computes
nothing itself.
"""
from __future__ import annotations

import itertools
import json
import os
import time

from . import recon, synth

# tuned schedules, keyed by GPU name, grid size and dtype (written by tune())
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")

# candidate values; the search is a coordinate descent from the defaults
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
    b = synth.smooth_and_floor(s.deposit_cic(pos), L, 2.0 * L / N, fft_dtype=torch.float32)
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


def tune(N: int, L: float | None = None, dtype: int = recon.RECON_MIXED, tol: float = 1e-8,
         reps: int = 2, path: str = CACHE, rounds: int = 2, verbose: bool = False) -> dict:
    """Coordinate descent over SPACE; returns and caches the best config."""
    import torch
    L = float(L if L is not None else N)
    b = _field(N, L, 9000 + N, torch.device("cuda", 0))
    solver = recon.Solver(N, L, dtype)
    base = solver.config()
    best_cfg = {k: base[k] for k in SPACE}
    best_t, _ = _time(solver, b, tol, reps)
    trials = [(dict(best_cfg), best_t)]
    for _ in range(rounds):
        improved = False
        for k, values in SPACE.items():
            for v in values:
                if v == best_cfg[k]:
                    continue
                cand = dict(best_cfg, **{k: v})
                if cand["nu1"] + cand["nu2"] < 1:
                    continue
                solver.configure(**cand)
                try:
                    t, st = _time(solver, b, tol, reps)
                except recon.ReconError:
                    continue
                trials.append((cand, t))
                if verbose:
                    print(f"  {cand} -> {t * 1e3:.2f} ms")
                if st["rel_residual"] < tol and t < best_t:
                    best_t, best_cfg, improved = t, cand, True
            solver.configure(**best_cfg)
        if not improved:
            break
    solver.close()
    cache = load_cache(path)
    cache[_key(N, dtype)] = {"config": best_cfg, "seconds": best_t, "trials": len(trials),
                             "default_seconds": trials[0][1]}
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
