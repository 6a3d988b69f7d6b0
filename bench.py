#!/usr/bin/env python
"""Benchmark of the GB300 multigrid Monge-Ampere reconstruction.

One step = one whole reconstruction of a seeded 512^3 Zel'dovich field
(L = 512 Mpc/h, sigma_lin = 1, smoothing R = 2 Mpc/h) with particles already
resident in HBM:
    CIC deposit -> density preparation (Gaussian window, floor, mean 1:
    recon_smooth_density) -> mixed-precision FAS solve to ||r|| / ||b - 1||
    < 1e-8 -> displacement.
All reconstruction steps run in librecon's hand-written sm_103a kernels.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (on a bounded sample of the same recipe, extrapolated).
Multi-GPU runs (torchrun) are independent replicas: every rank reconstructs
its own realisation (weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("512³ time-to-‖r‖/‖δ‖<1e-8 (mixed vs FP64 GPU); "
          "GS cell-updates/s; HBM %")
UNIT = "512^3 reconstructions/s"


def parse_cpulist(spec: str) -> set:
    """CPU numbers of a kernel CPU list such as "0-3,8,10-11"."""
    cpus = set()
    for part in spec.strip().split(","):
        if part:
            first, _, last = part.partition("-")
            cpus.update(range(int(first), int(last or first) + 1))
    return cpus


def pin_to_local_cpus(dev_index, sysfs="/sys/bus/pci/devices"):
    """Restrict this process to the CPUs attached to the GPU (its PCI
    device's local_cpulist), so that page-locked buffers allocated afterwards
    are placed on that CPU's memory node.  Returns the list, or None when the
    platform does not report one (nothing is changed then)."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        bdf = "%04x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        with open(os.path.join(sysfs, bdf, "local_cpulist")) as f:
            spec = f.read().strip()
        cpus = parse_cpulist(spec) & os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception:   # best effort: any failure leaves the affinity as it was
        return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="mixed-512")
    p.add_argument("--dtype", default="mixed", choices=["mixed", "f64"])
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-assignment", action="store_true")
    p.add_argument("--no-cubic", action="store_true")
    p.add_argument("--no-1024", action="store_true", help="skip the 1024^3 time-to-tolerance section")
    p.add_argument("--batch-count", type=int, default=64)
    p.add_argument("--adjoint-n", type=int, default=256)
    p.add_argument("--fd-directions", type=int, default=32)
    p.add_argument("--kernel-only", type=int, default=0, metavar="N",
                   help="only time the roofline kernel at N^3 (small case for profilers)")
    p.add_argument("--profile-solve", type=int, default=0, metavar="N",
                   help="only run two whole mixed reconstructions of an N^3 field of the "
                        "workload's recipe (a small case for profilers); prints their times")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- CPU side
def workload_config(W):
    """The config dict both arms report for workload W (same keys, same values)."""
    return {"workload": (f"{W.name}: {W.N}^3 seeded Zel'dovich field, L = {W.L:g} Mpc/h, "
                         f"sigma_lin = {W.sigma_lin}, R = {W.R:g} Mpc/h, CIC + density preparation "
                         f"+ solve to ||r||/||b-1|| < {W.tol:g} + displacement"),
            "l2": "inputs larger than L2 (particle positions "
                  f"{3 * 8 * W.N ** 3 / 1e9:.1f} GB, fields {W.N ** 3 * 8 / 1e9:.2f} GB)"}


def oracle_calibration(W, n: int = 64):
    """The oracle's whole reconstruction of one n^3 realisation of W's recipe
    (same h, sigma_lin and R in cells) against one oracle sweep of its density:
    both cost O(n^3), so their ratio carries over to W's grid.  Returns
    (seconds of the reconstruction, seconds of one sweep, FAS cycles)."""
    import numpy as np
    from oracle import oracle as O
    from paper_1709_06350_gb300 import synth
    h = W.L / W.N
    L = n * h
    _, dh = synth.linear_field(n, L, W.sigma_lin, W.seed + 17)
    pos = synth.zeldovich_positions(dh, n, L)
    t0 = time.perf_counter()
    rho = O.cic_deposit(pos, n, L)
    b = O.smooth_and_floor(rho, L, W.R)
    theta, info = O.solve(b, L, tol=W.tol, max_cycles=40)
    O.displace(theta, b, L)
    t_rec = time.perf_counter() - t0
    t_sw = min(_oracle_sweep_seconds(b, h) for _ in range(3))
    return t_rec, t_sw, info["cycles"]


def _oracle_sweep_seconds(b, h):
    """One oracle Gauss-Seidel sweep (red-black, snapshot order, Newton rule)
    of the density b from theta = 0."""
    import numpy as np
    from oracle import oracle as O
    th = np.zeros_like(b)
    t0 = time.perf_counter()
    O.sweep(th, b, 0.0, h)
    return time.perf_counter() - t0


def oracle_workload_density(W):
    """W's density built by the oracle (CIC and density preparation) from the
    generator's seeded particles; for the reference arm, which has no GPU."""
    from oracle import oracle as O
    from paper_1709_06350_gb300 import synth
    _, dh = synth.linear_field(W.N, W.L, W.sigma_lin, W.seed)
    pos = synth.zeldovich_positions(dh, W.N, W.L)
    del dh
    rho = O.cic_deposit(pos, W.N, W.L)
    del pos
    return O.smooth_and_floor(rho, W.L, W.R)


def oracle_sample_line(b_host, W, t_sweeps, cal):
    """cpu_baseline of one oracle sweep of W's full density, scaled to whole
    reconstructions by the calibration ratio (oracle_calibration)."""
    t_rec, t_sw, cycles = cal
    t_sweep = statistics.median(t_sweeps)
    ratio = t_rec / t_sw
    return {"value": 1.0 / (t_sweep * ratio), "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(),
            "sample": (f"one oracle Gauss-Seidel sweep (single-threaded FP64 C, red-black snapshot order, "
                       f"Newton rule, from theta = 0) over the {W.N}^3 workload density: "
                       f"{t_sweep:.2f} s; scaled to a whole reconstruction by the oracle's own ratio "
                       f"reconstruction / sweep = {t_rec:.2f} s / {t_sw:.3f} s = {ratio:.1f}, measured on "
                       f"a 64^3 realisation of the same recipe ({cycles} FAS cycles; CIC, density "
                       f"preparation, solve to {W.tol:g} and displacement)"),
            "sweep_s": t_sweep}


def reference_arm(args):
    """The oracle on this workload: every step is one oracle sweep of the
    full-size density (bounded: ~15 s), scaled to reconstructions/s by the
    calibration ratio; ms_per_step is the measured time of a step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1709_06350_gb300 import synth
    W = synth.WORKLOADS[args.workload]
    b = oracle_workload_density(W)
    cal = oracle_calibration(W)
    h = W.L / W.N
    for _ in range(args.warmup):
        _oracle_sweep_seconds(b, h)
    times = [_oracle_sweep_seconds(b, h) for _ in range(args.steps)]
    cpu = oracle_sample_line(b, W, times, cal)
    v = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(W), "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU side
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    from paper_1709_06350_gb300 import build as pbuild
    from paper_1709_06350_gb300 import recon, synth

    if args.kernel_only:
        pbuild.build()
        torch.cuda.set_device(0)
        n = args.kernel_only
        roof = kernel_roofline(recon, torch, n, float(n), torch.device("cuda", 0),
                               torch.cuda.current_stream())
        print(json.dumps({"kernel_only": n, "kernels": roof}), flush=True)
        return 0

    if args.profile_solve:
        pbuild.build()
        torch.cuda.set_device(0)
        return profile_solve(recon, synth, torch, args.profile_solve, synth.WORKLOADS[args.workload])

    from paper_1709_06350_gb300 import replicas
    world, rank, local = replicas.world()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # all work on created streams: the legacy default stream would serialise
    # with the end-to-end leg's copy stream
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()
    recon.load()

    def barrier():
        replicas.barrier(dist if world > 1 else None)

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, dist if world > 1 else None, dev)

    W = synth.WORKLOADS[args.workload]
    N, L, R, tol = W.N, W.L, W.R, W.tol
    delta_lin, dh = synth.linear_field(N, L, W.sigma_lin, replicas.replica_seed(W.seed, rank),
                                       backend="torch", device=dev)
    pos = synth.zeldovich_positions(dh, N, L).contiguous()
    del dh
    torch.cuda.empty_cache()
    # page-locked host buffers of the end-to-end leg, made before any timed
    # work, on the memory node of the CPUs attached to this GPU
    host = None
    host_cpus = None
    if not args.no_e2e:
        host_cpus = pin_to_local_cpus(local)
        host = {"pos": pos.cpu().pin_memory(),
                "dl": [torch.empty((N, N, N), dtype=torch.float64).pin_memory() for _ in range(2)]}

    dtype = recon.RECON_MIXED if args.dtype == "mixed" else recon.RECON_F64
    solver = recon.Solver(N, L, dtype)
    from paper_1709_06350_gb300 import autotune
    tuned = autotune.apply(solver, N, dtype)
    stream = torch.cuda.current_stream()
    rho = torch.zeros((N, N, N), dtype=torch.float64, device=dev)
    phi = torch.zeros_like(rho)
    bbuf = torch.empty_like(rho)
    last = {}

    def step(pos_dev):
        rho.zero_()
        solver.deposit_cic(pos_dev, rho=rho)
        b = solver.smooth_density(rho, R, out=bbuf)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = solver.solve(b, phi=phi, tol=tol, max_cycles=40)
        e1.record(stream)
        psi, dl = solver.displace(phi, b)
        last.update(st=st, b=b, dl=dl, ev=(e0, e1))
        return dl

    for _ in range(max(args.warmup, 3)):
        step(pos)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    launches0 = recon.recon_kernel_launches()
    with ClockSampler(uuid) as clk:
        barrier()
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        solve_ms = []
        for _ in range(args.steps):
            step(pos)
            solve_ms.append(last["ev"])
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = recon.recon_kernel_launches() - launches0
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end))
    solve_in_step_ms = statistics.median([a.elapsed_time(b) for a, b in solve_ms])
    st = last["st"]
    # the solve alone, nothing else on the GPU (time to tolerance)
    ref_b, ref_dl = last["b"].clone(), last["dl"]
    # the paper's own convergence measure of the same solve (untimed: one FP64
    # pass with the cubic's largest root per cell)
    solver.configure(report_paper_eps=1)
    _, st_eps = solver.solve(ref_b, phi=phi, tol=tol, max_cycles=40)
    solver.configure(report_paper_eps=0)
    solve_times = []
    torch.cuda.synchronize()
    for _ in range(3):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        solver.solve(ref_b, phi=phi, tol=tol, max_cycles=40)
        a1.record(stream)
        torch.cuda.synchronize()
        solve_times.append(a0.elapsed_time(a1))

    # ---- end to end through the public API from pinned host buffers.  The
    # copy engines move the positions of step k+1 in (double-buffered) and
    # delta_r of step k out on a copy stream while step k computes; the
    # kernels' SMs are not used for the transfers.
    e2e = None
    if not args.no_e2e:
        dl_dev = ref_dl.view(N, N, N).cpu()
        pos_host, dl_host = host["pos"], host["dl"]
        posbuf = [torch.empty_like(pos) for _ in range(2)]
        dlbuf = [torch.empty((N, N, N), dtype=torch.float64, device=dev) for _ in range(2)]
        psibuf = torch.empty((3, N, N, N), dtype=torch.float64, device=dev)
        copy = torch.cuda.Stream(device=dev)       # positions in
        copy_out = torch.cuda.Stream(device=dev)   # delta_r out (the other direction)

        def run_host(K):
            h2d = [torch.cuda.Event() for _ in range(2)]
            used = [torch.cuda.Event() for _ in range(2)]
            d2h = [None, None]
            with torch.cuda.stream(copy):
                posbuf[0].copy_(pos_host, non_blocking=True)
                h2d[0].record(copy)
            for k in range(K):
                cur, nxt = k % 2, (k + 1) % 2
                stream.wait_event(h2d[cur])
                if k + 1 < K:
                    with torch.cuda.stream(copy):
                        if k >= 1:
                            copy.wait_event(used[nxt])   # deposit(k-1) has read posbuf[nxt]
                        posbuf[nxt].copy_(pos_host, non_blocking=True)
                        h2d[nxt].record(copy)
                rho.zero_()
                solver.deposit_cic(posbuf[cur], rho=rho)
                used[cur].record(stream)
                b = solver.smooth_density(rho, R, out=bbuf)
                solver.solve(b, phi=phi, tol=tol, max_cycles=40)
                if d2h[cur] is not None:
                    stream.wait_event(d2h[cur])   # delta_r of step k-2 has left dlbuf[cur]
                solver.displace(phi, b, psi=psibuf, dl=dlbuf[cur])
                done = torch.cuda.Event()
                done.record(stream)
                with torch.cuda.stream(copy_out):
                    copy_out.wait_event(done)
                    dl_host[cur].copy_(dlbuf[cur], non_blocking=True)
                    d2h[cur] = torch.cuda.Event()
                    d2h[cur].record(copy_out)
            stream.wait_stream(copy)
            stream.wait_stream(copy_out)
            return dl_host[(K - 1) % 2]

        ke = max(1, args.steps)
        run_host(1)  # warm
        barrier()
        torch.cuda.synchronize()
        a, bev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = run_host(ke)
        bev.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(bev)) / ke
        check = float((out - dl_dev).abs().max())
        e2e = {"value": world * 1e3 / e2e_ms, "unit": UNIT,
               "h2d_bytes_per_step": pos.numel() * 8, "d2h_bytes_per_step": N ** 3 * 8,
               "ms_per_step": e2e_ms,
               "transfer": "positions of step k+1 copied in and delta_r of step k copied out by "
                           "the copy engines, one stream per direction, overlapping step k",
               "host_buffers_cpus": host_cpus,
               "max_abs_diff_vs_device_step": check}
        del pos_host, dl_host, posbuf, dlbuf, psibuf, host

    # ---- FP64 GPU path on the same density (the comparison the metric names)
    fp64 = None
    if not args.no_fp64_compare and dtype == recon.RECON_MIXED:
        s64 = recon.Solver(N, L, recon.RECON_F64)
        b = ref_b
        p64 = torch.zeros_like(b)
        s64.solve(b, phi=p64, tol=tol, max_cycles=40)
        torch.cuda.synchronize()
        a, bev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st64 = s64.solve(b, phi=p64, tol=tol, max_cycles=40)
        bev.record(stream)
        torch.cuda.synchronize()
        diff = float(torch.linalg.norm(p64 - phi) / torch.linalg.norm(p64))
        fp64 = {"time_to_tol_s": a.elapsed_time(bev) / 1e3, "cycles": st64["cycles"],
                "rel_residual": st64["rel_residual"], "mixed_vs_fp64_rel_l2": diff}
        s64.close()
        # the mixed path with its fine-grid residual in plain FP64 (the literal
        # form) beside the double-float default: same schedule, same density
        solver.configure(mixed_df_residual=0)
        pr = torch.zeros_like(b)
        solver.solve(b, phi=pr, tol=tol, max_cycles=40)
        torch.cuda.synchronize()
        a.record(stream)
        _, str64 = solver.solve(b, phi=pr, tol=tol, max_cycles=40)
        bev.record(stream)
        torch.cuda.synchronize()
        fp64["mixed_fp64_residual"] = {
            "time_to_tol_s": a.elapsed_time(bev) / 1e3, "fas_cycles": str64["cycles"],
            "outer_iterations": str64["outer_iterations"], "rel_residual": str64["rel_residual"],
            "vs_fp64_rel_l2": float(torch.linalg.norm(pr - p64) / torch.linalg.norm(p64)),
            "vs_double_float_rel_l2": float(torch.linalg.norm(pr - phi) / torch.linalg.norm(phi))}
        solver.configure(mixed_df_residual=1)
        del p64, pr

    # ---- rooflines of the two FP32 smoothers, timed in isolation at N^3
    kern = kernel_roofline(recon, torch, N, L, dev, stream)
    roof = dict(kern[0])
    kern64 = fp64_rooflines(recon, torch, N, L, dev, stream)

    # ---- reconstruction quality: r(k) of delta_r against the seeded linear field
    from paper_1709_06350_gb300 import analysis
    kk, rr, _ = analysis.correlation(ref_dl.view(N, N, N), delta_lin, L)
    rk = analysis.r_at(kk, rr, (0.05, 0.1, 0.2, 0.3, 0.5))
    # 1-point Gaussianisation of delta_r (Sec. III): time and its r(k)
    gauss = None
    if rank == 0:
        gfield = solver.gaussianise(ref_dl.view(N, N, N))
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            solver.gaussianise(ref_dl.view(N, N, N))
        a1.record(stream)
        torch.cuda.synchronize()
        kg, rg, _ = analysis.correlation(gfield, delta_lin, L)
        gauss = {"ms": a0.elapsed_time(a1) / 3,
                 "r_k": list(analysis.r_at(kg, rg, (0.05, 0.1, 0.2, 0.3, 0.5)).values())}
        del gfield
    del delta_lin

    batch = None
    if not args.no_batch and rank == 0:
        solver.close()
        torch.cuda.empty_cache()
        batch = bench_batch(recon, synth, torch, dev, args.batch_count)
        solver = recon.Solver(N, L, dtype)
        autotune.apply(solver, N, dtype)

    assign = None
    if not args.no_assignment and rank == 0:
        torch.cuda.empty_cache()
        assign = bench_assignment(recon, synth, torch, dev, pos, W, autotune)

    cubic = None
    if not args.no_cubic and rank == 0:
        torch.cuda.empty_cache()
        cubic = bench_cubic(recon, synth, torch, dev)

    big = None
    if not args.no_1024 and rank == 0 and args.workload == "mixed-512":
        torch.cuda.empty_cache()
        try:
            big = bench_1024(recon, synth, torch, dev, stream, autotune)
        except Exception as ex:   # reported, never fatal to the bench line
            big = {"error": f"{type(ex).__name__}: {ex}"}
        torch.cuda.empty_cache()

    adj = None
    if not args.no_adjoint and rank == 0:
        torch.cuda.empty_cache()
        adj = bench_adjoint(recon, synth, torch, dev, args.adjoint_n, args.fd_directions)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        b_host = ref_b.cpu().numpy()
        cal = oracle_calibration(W)
        cpu = oracle_sample_line(b_host, W, [_oracle_sweep_seconds(b_host, L / N)], cal)
        del b_host

    if rank == 0:
        ms = elapsed_ms / args.steps
        line = {
            "metric": METRIC, "value": replicas.job_throughput(args.steps, world, elapsed_ms / 1e3),
            "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64" if dtype == recon.RECON_MIXED else "f64",
            "data": "synthetic",
            "config": workload_config(W),
            "solver_config": {"solver": solver.config(),
                              "schedule": "autotuned (paper_1709_06350_gb300/autotune_cache.json)"
                                          if tuned else "defaults"},
            "time_to_tol_s": {"mixed": statistics.median(solve_times) / 1e3,
                              "fp64": fp64["time_to_tol_s"] if fp64 else None,
                              "mixed_inside_step": solve_in_step_ms / 1e3},
            "solve": {"fas_cycles": st["cycles"], "outer_iterations": st["outer_iterations"],
                      "rel_residual": st["rel_residual"], "compat_c": st["compat_c"],
                      "paper_eps": st_eps["paper_eps"], "history": st["history"]},
            "fp64_path": fp64,
            "r_k": {"k_h_per_Mpc": list(rk.keys()), "r": list(rk.values()),
                    "fields": "delta_r (displacement output, Lagrangian grid) vs the seeded "
                              "linear field"},
            "gaussianised": gauss,
            "batched": batch,
            "assignment": assign,
            "cubic_test": cubic,
            "adjoint": adj,
            "mixed_1024": big,
            "gs_cell_updates_per_s": {"fas_newton": kern[1]["cell_updates_per_s"],
                                      "linear": roof.pop("cell_updates_per_s", None)},
            "roofline": roof,
            "other_kernels": kern[1:] + kern64,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def bench_assignment(recon, synth, torch, dev, pos, W, autotune):
    """NGP / CIC / TSC deposits of the workload's particles (timed), and the
    convergence of mixed solves with the three schemes and three tracer /
    mesh ratios (Sec. I: N^3 on N^3, 8N^3 on N^3, N^3 on 8N^3)."""
    N, L, R, tol = W.N, W.L, W.R, W.tol
    out = {"deposit_ms": {}, "convergence": []}
    cases = [(f"{N}^3 particles", N, pos), (f"{N}^3 particles", N // 2, pos)]
    _, dh = synth.linear_field(N // 2, L, W.sigma_lin, W.seed + 1, backend="torch", device=dev)
    cases.append((f"{N // 2}^3 particles", N, synth.zeldovich_positions(dh, N // 2, L).contiguous()))
    del dh
    for label, mesh, P in cases:
        s = recon.Solver(mesh, L, recon.RECON_MIXED)
        autotune.apply(s, mesh, recon.RECON_MIXED)
        for scheme in ("ngp", "cic", "tsc"):
            rho = torch.zeros((mesh,) * 3, dtype=torch.float64, device=dev)
            s.deposit(P, scheme, rho=rho)
            if mesh == N and P is pos:
                torch.cuda.synchronize()
                a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(3):
                    rho.zero_()
                    s.deposit(P, scheme, rho=rho)
                b_.record()
                torch.cuda.synchronize()
                out["deposit_ms"][scheme] = a.elapsed_time(b_) / 3
            b = s.smooth_density(rho, R)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = s.solve(b, tol=tol, max_cycles=40)
            torch.cuda.synchronize()
            out["convergence"].append({"particles": label, "mesh": f"{mesh}^3", "scheme": scheme,
                                       "fas_cycles": st["cycles"], "outer": st["outer_iterations"],
                                       "rel_residual": st["rel_residual"],
                                       "solve_s": time.perf_counter() - t0})
            del rho, b
        s.close()
    out["deposit_workload"] = f"{N}^3 particles on the {N}^3 mesh (mean 1)"
    return out


def bench_1024(recon, synth, torch, dev, stream, autotune):
    """The 1024^3 workload (L = 1024 Mpc/h, sigma_lin = 1, R = 2 Mpc/h): the
    mixed solve's time to ||r|| / ||b - 1|| < 1e-8 (median of three, b on the
    device), the FP64 GPU path on the same density, their difference, and
    the two FP32 smoothers' rooflines at 1024^3."""
    W = synth.WORKLOADS["mixed-1024"]
    N, L = W.N, W.L
    _, dh = synth.linear_field(N, L, W.sigma_lin, W.seed, backend="torch", device=dev)
    pos = synth.zeldovich_positions(dh, N, L).contiguous()
    del dh
    s = recon.Solver(N, L, recon.RECON_MIXED)
    autotune.apply(s, N, recon.RECON_MIXED)
    b = s.smooth_density(s.deposit_cic(pos), W.R)
    del pos
    torch.cuda.empty_cache()
    phi = torch.zeros_like(b)
    _, st = s.solve(b, phi=phi, tol=W.tol, max_cycles=40)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        _, st = s.solve(b, phi=phi, tol=W.tol, max_cycles=40)
        a1.record(stream)
        torch.cuda.synchronize()
        times.append(a0.elapsed_time(a1) / 1e3)
    s.close()
    s64 = recon.Solver(N, L, recon.RECON_F64)
    p64 = torch.zeros_like(b)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    _, st64 = s64.solve(b, phi=p64, tol=W.tol, max_cycles=40)
    a1.record(stream)
    torch.cuda.synchronize()
    diff = float(torch.linalg.norm(p64 - phi) / torch.linalg.norm(p64))
    s64.close()
    del b, phi, p64
    torch.cuda.empty_cache()
    kern = kernel_roofline(recon, torch, N, L, dev, stream)
    return {"workload": f"{W.name}: {N}^3, L = {L:g} Mpc/h, sigma_lin = {W.sigma_lin}, R = {W.R:g} Mpc/h",
            "time_to_tol_s": {"mixed": statistics.median(times), "fp64": a0.elapsed_time(a1) / 1e3},
            "mixed": {"fas_cycles": st["cycles"], "outer_iterations": st["outer_iterations"],
                      "rel_residual": st["rel_residual"]},
            "fp64": {"cycles": st64["cycles"], "rel_residual": st64["rel_residual"]},
            "mixed_vs_fp64_rel_l2": diff,
            "smoothers": [{k: v for k, v in x.items() if k in ("kernel", "avg_launch_ms", "achieved", "frac")}
                          for x in kern]}


def bench_cubic(recon, synth, torch, dev, tol=1e-3):
    """Sec. III.A cubic test at the paper's sizes: 128^3 particles filling a
    cube of side 10 Mpc/h at the centre of a 128 Mpc/h box, CIC on 128^3,
    floor 0.05, no smoothing; FP64 and mixed solves to `tol`, and the
    interior closed form lap(theta) = 3 (b_in^(1/3) - 1), Hbar = 0."""
    N, L, l = 128, 128.0, 10.0
    pos = torch.from_numpy(synth.cube_positions(N, L, l)).to(dev)
    out = {"workload": f"{N}^3 particles in a {l:g} Mpc/h cube, box {L:g} Mpc/h, mesh {N}^3, "
                       f"CIC, floor 0.05, tol {tol:g}"}
    for name, dtype in (("fp64", recon.RECON_F64), ("mixed", recon.RECON_MIXED)):
        s = recon.Solver(N, L, dtype)
        b = s.smooth_density(s.deposit_cic(pos), 0.0)
        phi = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = s.solve(b, phi=phi, tol=tol, max_cycles=200, raise_on_noconv=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c = N // 2
        t = phi[c - 2:c + 2, c - 2:c + 2, c - 2:c + 2]
        H = [(t.roll(-1, a) + t.roll(1, a) - 2 * t)[1:3, 1:3, 1:3] for a in range(3)]
        lap = H[0] + H[1] + H[2]
        expect = 3.0 * (float(b[c, c, c]) ** (1.0 / 3.0) - 1.0)
        out[name] = {"seconds": dt, "cycles": st["cycles"], "outer": st["outer_iterations"],
                     "rel_residual": st["rel_residual"], "lap_centre": float(lap.mean()),
                     "lap_expected": expect,
                     "hbar_max_rel": max(float((H[a] - lap / 3).abs().max()) for a in range(3)) / expect}
        if dtype == recon.RECON_F64:
            # the scaled-defect factor of every coarse level, cycle by cycle
            # (the nested-iteration start and one cycle, then resumed cycles)
            trace, rel = [], []
            phi.zero_()
            s.configure(start=0)
            for k in range(12):
                _, stk = s.solve(b, phi=phi, tol=1e-30, max_cycles=1, raise_on_noconv=False)
                trace.append(s.level_scales())
                rel.append(stk["rel_residual"])
                s.configure(start=1)
            out[name]["level_scale_trace"] = {"levels": [N >> (l + 1) for l in range(len(trace[0]))],
                                              "s_per_cycle": trace, "rel_residual_per_cycle": rel}
        s.close()
    return out


def bench_batch(recon, synth, torch, dev, count):
    """Config 4: `count` realisations, N cycling through 64..256 (h = 2 Mpc/h),
    solved to 1e-8 by one recon_batch (CUDA graphs), against the same solves
    run one after another on single handles."""
    Ws = synth.batched_workloads(count)
    sizes = [w.N for w in Ws]
    boxes = [w.L for w in Ws]
    deposit = {}
    bs = []
    for w in Ws:
        if w.N not in deposit:
            deposit[w.N] = recon.Solver(w.N, w.L, recon.RECON_F64)
        _, dh = synth.linear_field(w.N, w.L, w.sigma_lin, w.seed, backend="torch", device=dev)
        pos = synth.zeldovich_positions(dh, w.N, w.L).contiguous()
        rho = deposit[w.N].deposit_cic(pos)
        bs.append(deposit[w.N].smooth_density(rho, w.R))
        del dh, pos, rho
    for s in deposit.values():
        s.close()
    B = recon.Batch(sizes, boxes)
    from paper_1709_06350_gb300 import autotune
    autotune.apply(B)
    phis = [torch.zeros_like(b) for b in bs]
    B.solve(bs, phis=phis, tol=1e-8, max_cycles=40)          # captures the graphs
    torch.cuda.synchronize()
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        _, stats = B.solve(bs, phis=phis, tol=1e-8, max_cycles=40)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) / reps
    B.close()
    single = {}
    for n, L in sorted(set(zip(sizes, boxes))):
        single[n] = recon.Solver(n, L, recon.RECON_MIXED)
        autotune.apply(single[n], n, recon.RECON_MIXED)   # the same schedules as the batch
    for b, n in zip(bs[:5], sizes[:5]):
        single[n].solve(b, tol=1e-8, max_cycles=40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b, n in zip(bs, sizes):
        single[n].solve(b, tol=1e-8, max_cycles=40)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    for s in single.values():
        s.close()
    cells = sum(n ** 3 for n in sizes)
    worst = max(s["rel_residual"] for s in stats)
    del bs, phis
    return {"workload": f"{count} realisations, N cycling 64/96/128/192/256, L = 2N Mpc/h, "
                        "sigma_lin = 0.8, R = 4 Mpc/h, mixed solve to 1e-8",
            "seconds_per_batch": t_batch, "realisations_per_s": count / t_batch,
            "cells_per_s": cells / t_batch, "sequential_seconds": t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "worst_rel_residual": worst,
            "cycles": stats[0]["cycles"],
            "outer_iterations_max": max(s["outer_iterations"] for s in stats)}


def bench_adjoint(recon, synth, torch, dev, n, directions):
    """Config 5: FP64 solve of a 256^3 field (L = 512 Mpc/h, sigma_lin = 0.8,
    R = 4 Mpc/h), then the adjoint of loss = <w, phi(b)>; checked against
    central finite differences along random directions."""
    L = 2.0 * n
    w = synth.WORKLOADS.get("adjoint-256")
    delta_lin, dh = synth.linear_field(n, L, 0.8, w.seed if w else 5000, backend="torch", device=dev)
    pos = synth.zeldovich_positions(dh, n, L).contiguous()
    s = recon.Solver(n, L, recon.RECON_F64)
    b = s.smooth_density(s.deposit_cic(pos), 4.0)
    del dh, pos
    gen = torch.Generator(device=dev).manual_seed(11)
    wv = torch.randn((n, n, n), dtype=torch.float64, device=dev, generator=gen)
    t0 = time.perf_counter()
    phi, st = s.solve(b, tol=1e-12, max_cycles=60)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    modes = {}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]   # before any adjoint workspace exists
    res0 = torch.cuda.memory_reserved(dev)
    for store in (1, 0):
        # the adjoint's device workspace: the drop in free device memory since
        # before any adjoint call, less what torch's allocator took meanwhile
        # (switching modes frees the other mode's workspace)
        s.configure(adjoint_store_cofactors=store)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = s.adjoint(wv)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        ws = (free0 - torch.cuda.mem_get_info(dev)[0]) - (torch.cuda.memory_reserved(dev) - res0)
        t0 = time.perf_counter()
        g = s.adjoint(wv)                      # null vector (and stored cofactors) reused
        torch.cuda.synchronize()
        modes["stored" if store else "formed"] = {
            "adjoint_seconds_first": t_adj, "adjoint_seconds_repeat": time.perf_counter() - t0,
            "workspace_gb": ws / 1e9, "gradient": g}
    g = modes["formed"].pop("gradient")
    g_st = modes["stored"].pop("gradient")
    modes["formed_vs_stored_rel_l2"] = float(torch.linalg.norm(g - g_st) / torch.linalg.norm(g_st))
    del g_st
    t_adj = modes["formed"]["adjoint_seconds_first"]
    t_adj2 = modes["formed"]["adjoint_seconds_repeat"]
    eps = 1e-4
    errs = []
    aux = recon.Solver(n, L, recon.RECON_F64)
    for _ in range(directions):
        d = torch.randn((n, n, n), dtype=torch.float64, device=dev, generator=gen)
        pp, _ = aux.solve(b + eps * d, tol=1e-12, max_cycles=60)
        lp = float((wv * pp).sum())
        pm, _ = aux.solve(b - eps * d, tol=1e-12, max_cycles=60)
        lm = float((wv * pm).sum())
        fd = (lp - lm) / (2 * eps)
        errs.append(abs(float((g * d).sum()) - fd) / abs(fd))
    out = {"workload": f"{n}^3, L = {L:g} Mpc/h, sigma_lin = 0.8, R = 4 Mpc/h, FP64",
           "solve_seconds": t_solve, "adjoint_seconds_first": t_adj,
           "adjoint_seconds_repeat": t_adj2, "finest_level_cofactors": modes, "fd_directions": directions,
           "fd_max_rel_error": max(errs) if errs else None, "fd_step": eps}
    try:
        out["delta_r_loss"] = _adjoint_delta_r_loss(recon, torch, s, aux, b, phi, delta_lin, n, L, gen)
    except Exception as ex:   # reported, never fatal to the bench line
        out["delta_r_loss"] = {"error": f"{type(ex).__name__}: {ex}"}
    aux.close()
    s.close()
    return out


def _adjoint_delta_r_loss(recon, torch, s, aux, b, phi, delta_lin, n, L, gen, directions=32):
    """The loss of the adjoint workload on the reconstructed density:
    sum over |k| < 0.5 h/Mpc of |FFT(delta_r) - FFT(delta_L, seed)|^2, delta_r
    the FP64 output at phi(b).  Its gradient with respect to b is the output's
    adjoint (direct b term) plus the solve's adjoint of its phi term.

    Checked by central differences along `directions` random directions in
    the loss's band (|k| < 0.5 h/Mpc, unit rms), each with a step that moves
    no q across a CIC cell face: the CIC weights are piecewise linear, so a
    step that crosses a face measures a kink, not the gradient.  Per
    direction d the largest such step follows from the map: with u the CIC
    coordinate of every q and du/deps its response to b + eps d (from two
    solves 1e-7 apart), eps_safe = min over cells and axes of (distance of u
    to its nearest face) / |du/deps|; the check uses eps = eps_safe / 2 and
    verifies that no cell changed.  The perturbed solves start from phi(b)
    (FP64, resumed V-cycles to the FP64 floor), so the difference of two
    solves carries the O(eps) response and not the solves' own iteration
    error."""
    import math
    h = L / n
    kf = 2 * math.pi / L
    f = torch.fft.fftfreq(n, d=1.0 / n, device=b.device) * kf
    fz = torch.fft.rfftfreq(n, d=1.0 / n, device=b.device) * kf
    kk = torch.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2)
    mask = (kk < 0.5).to(torch.float64)
    ref = torch.fft.rfftn(delta_lin.to(torch.float64))

    def loss_of(dl):
        return float((mask * (torch.fft.rfftn(dl) - ref).abs() ** 2).sum())

    def ucoords(p):
        # u = q N / L - 1/2 per axis, q = x + central gradient of phi (mod L)
        out = []
        idx = torch.arange(n, device=b.device, dtype=torch.float64)
        for ax in range(3):
            g = (torch.roll(p, -1, ax) - torch.roll(p, 1, ax)) / (2 * h)
            shape = [1, 1, 1]
            shape[ax] = n
            q = torch.remainder(((idx + 0.5) * h).view(shape) + g, L)
            out.append(q / h - 0.5)
        return out

    aux.configure(start=recon.START_GUESS)

    def solve(bb):
        p = phi.clone()
        _, st = aux.solve(bb, phi=p, tol=1e-15, max_cycles=12, raise_on_noconv=False)
        return p, st["rel_residual"]

    _, dl = s.displace_fp64(phi, b)
    dlr = dl.detach().clone().requires_grad_(True)
    (mask * (torch.fft.rfftn(dlr) - ref).abs() ** 2).sum().backward()
    gdl = dlr.grad.contiguous()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gphi, gb_direct = s.displace_adjoint(phi, b, None, gdl)
    gb = gb_direct + s.adjoint(gphi)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    u0 = ucoords(phi)
    dist = [torch.minimum(u - torch.floor(u), torch.ceil(u) - u) for u in u0]
    errs, steps, crossings, resid = [], [], [], []
    for _ in range(directions):
        d = torch.randn((n, n, n), dtype=torch.float64, device=b.device, generator=gen)
        d = torch.fft.irfftn(torch.fft.rfftn(d) * mask, s=(n, n, n))
        d = d / d.pow(2).mean().sqrt()
        e0 = 1e-7
        pp, _ = solve(b + e0 * d)
        pm, _ = solve(b - e0 * d)
        dphi = (pp - pm) / (2 * e0)
        du = [(torch.roll(dphi, -1, ax) - torch.roll(dphi, 1, ax)) / (2 * h * h) for ax in range(3)]
        eps = 0.5 * min(float((dist[ax] / du[ax].abs().clamp_min(1e-300)).min()) for ax in range(3))
        vals, cross = [], 0
        for sg in (1.0, -1.0):
            bp = b + sg * eps * d
            p2, rr = solve(bp)
            resid.append(rr)
            vals.append(loss_of(aux.displace_fp64(p2, bp)[1]))
            cross += sum(int((torch.floor(a) != torch.floor(c)).sum()) for a, c in zip(u0, ucoords(p2)))
        fd = (vals[0] - vals[1]) / (2 * eps)
        errs.append(abs(float((gb * d).sum()) - fd) / abs(fd))
        steps.append(eps)
        crossings.append(cross)
    return {"loss": "sum_{|k|<0.5 h/Mpc} |FFT(delta_r) - FFT(delta_L seed)|^2, delta_r FP64",
            "gradient_seconds": t_grad, "fd_directions": directions,
            "fd_step": "per direction eps_safe / 2 (no q crosses a CIC cell face)",
            "fd_steps_min_median_max": [min(steps), statistics.median(steps), max(steps)],
            "min_face_distance_cells": min(float(x.min()) for x in dist),
            "face_crossings": sum(crossings), "fd_solve_rel_residual_max": max(resid),
            "fd_max_rel_error": max(errs), "fd_median_rel_error": statistics.median(errs),
            "fd_fraction_below_1e-5": sum(e < 1e-5 for e in errs) / len(errs),
            "fd_errors": sorted(errs)}


def _time_launches(torch, stream, fn, reps):
    """Mean time of one launch: (time of fn(reps + 1) - time of fn(1)) / reps,
    so per-call set-up drops out (both counts are odd: an odd number of
    ping-pong sweeps ends with the same copy back into the caller's array)."""
    def timed(k):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(k)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3
    fn(2)
    t1 = min(timed(1) for _ in range(3))
    tr = timed(reps + 1)
    return (tr - t1) / reps


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each register-blocked fused smoother, from an ncu capture of the 384^3 case
# (python bench.py --kernel-only 384; ncu -k regex:k_sweep_reg, -s 2 -c 1 for
# the FAS smoother, -s 18 -c 1 for the linear one); a launch at N^3
# moves (N/384)^3 times as much.  Valid for the kernels as they were
# captured: re-measure after a change to either kernel.
# DRAM bytes (read + write) of one 384^3 launch from the last ncu capture of
# each smoother; both kernels changed after that capture (a device scalar is
# now folded into each update), so the roofline reports traffic as null and
# these figures only as the earlier capture's context.
NCU_TRAFFIC_384 = {"LIN": 689.353472e6 + 208.309248e6, "FAS": 472.232960e6 + 210.356992e6}


def profile_solve(recon, synth, torch, N, W):
    """Two whole mixed reconstructions (CIC, density preparation, solve,
    displacement) of an N^3 field of W's recipe at W's cell size (L = W.L N /
    W.N), with the autotuned schedule of W's grid: a small case that runs
    every kernel of the step, for a profiler.  Prints the two solve times."""
    from paper_1709_06350_gb300 import autotune
    dev = torch.device("cuda", 0)
    L = W.L * N / W.N
    _, dh = synth.linear_field(N, L, W.sigma_lin, W.seed, backend="torch", device=dev)
    pos = synth.zeldovich_positions(dh, N, L).contiguous()
    del dh
    solver = recon.Solver(N, L, recon.RECON_MIXED)
    autotune.apply(solver, W.N, recon.RECON_MIXED)
    phi = torch.zeros((N, N, N), dtype=torch.float64, device=dev)
    out = []
    for _ in range(2):
        rho = solver.deposit_cic(pos)
        b = solver.smooth_density(rho, W.R)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = solver.solve(b, phi=phi, tol=W.tol, max_cycles=40)
        torch.cuda.synchronize()
        out.append(time.perf_counter() - t0)
        solver.displace(phi, b)
    torch.cuda.synchronize()
    solver.close()
    print(json.dumps({"profile_solve": N, "L": L, "solve_seconds": out, "fas_cycles": st["cycles"],
                      "outer_iterations": st["outer_iterations"], "rel_residual": st["rel_residual"]}),
          flush=True)
    return 0


def kernel_roofline(recon, torch, N, L, dev, stream):
    """The two FP32 smoothers at N^3, each timed in isolation with CUDA events
    on its stream (one launch = one fused red+black sweep for N >= 128).
    The linear smoother comes first: it is the larger share of the step.

    Algorithmic bytes per sweep: linear smoother 16 B/cell (read theta, e,
    f; write e); FAS smoother 12 B/cell (read theta and b, write theta)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    src = "measured (MEASURED_PEAKS.json hbm_gbs, burst)" if hbm else "fallback 6800 GB/s"
    hbm = hbm or 6800.0
    from paper_1709_06350_gb300 import synth
    h = L / N
    th = torch.from_numpy(synth.smooth_field(N, 1, 0.3 * h * h, kmax=4)).to(dev, torch.float32)
    g = torch.from_numpy(1.0 + synth.smooth_field(N, 2, 0.4, kmax=4)).to(dev, torch.float32)
    work = torch.empty_like(th)
    reps = 10
    t_fas = _time_launches(torch, stream, lambda k: recon.recon_step_sweep(
        th, g, 0.0, h, sweeps=k, work=work, stream=stream), reps)
    e = torch.zeros_like(th)
    work7 = torch.empty(7 * N ** 3, dtype=torch.float32, device=dev)
    t_lin = _time_launches(torch, stream, lambda k: recon.recon_step_linear_sweep(
        e, g, th, h, sweeps=k, work=work7, stream=stream), reps)
    del th, g, work, e, work7
    out = []
    for key, name, t, bpc in (
            ("LIN", "k_sweep_reg<LIN> (FP32 red-black smoother of J e = f, one fused sweep, 2x2 register blocks)",
             t_lin, 16.0),
            ("FAS", "k_sweep_reg<FAS> (FP32 red-black Newton smoother, one fused sweep, 2x2 register blocks)",
             t_fas, 12.0)):
        alg = bpc * N ** 3
        ach = alg / t / 1e9
        out.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": None,
                    "traffic_source": "null: the kernel changed after its last ncu capture (a device "
                                      "scalar folded into the update); that capture's DRAM bytes, "
                                      "scaled from 384^3 by cells, are in traffic_last_capture",
                    "traffic_last_capture": NCU_TRAFFIC_384[key] * (N / 384.0) ** 3,
                    "peak_source": src, "algorithmic_bytes_per_launch": alg,
                    "avg_launch_ms": t * 1e3, "cell_updates_per_s": N ** 3 / t})
    return out


def fp64_peak_tflops(recon, torch, dev, stream):
    """Measured FP64 FMA rate of this GPU (recon_measure_fp64_fma: 8
    independent FMA chains per thread, 16 CTAs of 256 threads per SM), best of
    five launches timed with events on the stream."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 16 * sms, 20000
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    recon.recon_measure_fp64_fma(blocks, 100, out, stream)
    best = None
    for _ in range(5):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        recon.recon_measure_fp64_fma(blocks, iters, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        best = t if best is None else min(best, t)
    return 4096.0 * blocks * iters / best / 1e12


# Algorithmic FP64 work of one cell update of the nonlinear smoother (eq.
# update: the Hessian stencils, the cubic's coefficients, one Newton step and
# its acceptance test), counting a fused multiply-add as two flops.
FP64_FLOPS_PER_CELL_UPDATE = 70.0


def fp64_rooflines(recon, torch, N, L, dev, stream):
    """The FP64 path's smoother at N^3 against the measured FP64 FMA rate:
    the fused sweep (both colours, one launch) and the two-pass kernels (an
    array not aligned to an element pair runs them: two launches a sweep)."""
    from paper_1709_06350_gb300 import synth
    peak = fp64_peak_tflops(recon, torch, dev, stream)
    h = L / N
    th = torch.from_numpy(synth.smooth_field(N, 1, 0.3 * h * h, kmax=4)).to(dev, torch.float64)
    g = torch.from_numpy(1.0 + synth.smooth_field(N, 2, 0.4, kmax=4)).to(dev, torch.float64)
    work = torch.empty_like(th)
    t_fused = _time_launches(torch, stream, lambda k: recon.recon_step_sweep(
        th, g, 0.0, h, sweeps=k, work=work, stream=stream), 3)
    buf = torch.empty(th.numel() + 1, dtype=torch.float64, device=dev)
    tu = buf[1:].view(th.shape)
    tu.copy_(th)
    t_two = _time_launches(torch, stream, lambda k: recon.recon_step_sweep(
        tu, g, 0.0, h, sweeps=k, work=work, stream=stream), 3)
    del th, g, work, buf, tu
    out = []
    for name, t, launches in (("k_sweep_fused<double, FAS> (FP64 red-black Newton smoother, one fused sweep)",
                               t_fused, 1),
                              ("k_rb_pass<double> (FP64 red-black Newton smoother, one colour pass)", t_two, 2)):
        flops = FP64_FLOPS_PER_CELL_UPDATE * N ** 3 / launches
        ach = flops / (t / launches) / 1e12
        out.append({"kernel": name, "bound": "fp64", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "peak_source": "measured: recon_measure_fp64_fma (FP64 FMA chains)",
                    "algorithmic_flops_per_launch": flops, "avg_launch_ms": t / launches * 1e3})
    return out


if __name__ == "__main__":
    sys.exit(main())
