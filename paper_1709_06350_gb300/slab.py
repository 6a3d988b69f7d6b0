"""Slab decomposition of the FP64 FAS solve over several processes.

One field too large (or too slow) for one GPU is split across P processes,
one GPU each.  Every level of the multigrid hierarchy (Sec. II.A.3) is cut
along i into P equal slabs of whole planes; rank r owns planes
[r n, (r + 1) n), n = N_l / P, and holds two more planes on each side (its
halo), copied from its neighbours (periodic: rank 0's lower neighbour is
rank P - 1).

What crosses process boundaries, per V-cycle:

* Halo exchange of theta before every step that reads neighbours.  The
  colour passes of a sweep read only values from before the pass (the
  red-black snapshot ordering), so a sweep can run on a two-plane halo: the
  first colour pass is also applied to the first halo plane on each side
  (the same arithmetic its owner does), and the second pass then finds every
  value it reads up to date.  One exchange of two planes per sweep replaces
  one exchange of one plane per colour pass.
* Sums over a level (the mean of the restricted residual, the compatibility
  scalar c, the gauge mean of theta, the residual norms of the stopping
  rule): every rank forms the partial sum of each of its planes, the plane
  partials of all ranks are gathered and added in plane order.  A sum is
  then the same number whatever P is (bitwise), and equals a single
  process's sum taken the same way.
* The scaled-defect factor of the coarse equation is a minimum over cells:
  the ranks' minima are combined by a min.
* Agglomeration: a level whose planes cannot be split evenly into slabs of
  at least ``min_planes`` planes (default 64: below 64^3 a level is cheap and
  latency-bound) is held whole by rank 0.  Restriction onto such a level
  gathers the ranks' restricted planes on rank 0; rank 0 runs the rest of the
  V-cycle there (down to the coarsest grid's solve) and scatters back each
  rank's coarse planes, with one halo plane on each side, for the
  prolongation.

The cell arithmetic is done by a backend with one method per step of the
V-cycle, each applied to the planes a rank owns (``SlabBackend``).  The
driver calls the steps in the order of the single-process FAS solve
(nested-iteration start, V-cycles, compatibility scalar and gauge after each
cycle, the stopping rule on the mean-free residual), so with a backend that
performs the single-process arithmetic the decomposed solve reproduces the
single-process result bit for bit.  ``GpuSlabBackend`` runs the steps as
CUDA kernels of ``librecon.so`` (``recon_slab_*``), on the rank's own GPU.

Communication goes through ``torch.distributed`` (NCCL between GPUs, gloo
between CPU processes): point-to-point send/recv for halos, all_gather for
plane partials, gather/scatter for agglomeration.  Nothing here uses
multicast or remote loads; every buffer lives in the rank's own memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


# ---------------------------------------------------------------- layout
@dataclass(frozen=True)
class Layout:
    """The planes of one level that one array holds.

    N      -- the level's side (the level has N^3 cells)
    first  -- global index of the array's plane 0 (may be negative: halo
              planes are taken mod N)
    planes -- planes the array holds (own planes plus halos)
    lo, hi -- the array's own planes are [lo, hi) (local indices)
    """
    N: int
    first: int
    planes: int
    lo: int
    hi: int

    @property
    def own(self) -> int:
        return self.hi - self.lo

    @property
    def own_first(self) -> int:
        """Global index of the first own plane."""
        return self.first + self.lo

    @property
    def whole(self) -> bool:
        """The array is the whole periodic grid (no halos)."""
        return self.planes == self.N and self.lo == 0 and self.hi == self.N and self.first == 0


HALO = 2


def num_levels(N: int) -> int:
    """Levels of the hierarchy: halve N while the half is even and >= 4
    (Sec. II.A.3; grids that are not powers of two stop at the last even
    size, 96 -> 48 -> 24 -> 12 -> 6)."""
    L = 1
    while N % 2 == 0 and N // 2 >= 4 and (N // 2) % 2 == 0:
        N //= 2
        L += 1
    return L


def split_levels(N: int, P: int, min_planes: int = 64) -> list[bool]:
    """Per level: True when it is split into P slabs, False when rank 0 holds
    it whole.  A level is split when its planes divide evenly into P slabs of
    at least max(min_planes, HALO) planes, an even number of them (so that
    restriction maps whole own planes onto whole coarse own planes), and the
    slab with its halos still fits in the grid; every finer level is split
    too, and the coarsest level is never split (its solve is one process's
    Gauss-Seidel)."""
    L = num_levels(N)
    out = []
    ok = P > 1
    for l in range(L):
        Nl = N >> l
        n = Nl // P if P > 0 else 0
        split = (ok and l < L - 1 and Nl % P == 0 and n >= max(min_planes, HALO) and n % 2 == 0
                 and n + 2 * HALO <= Nl)
        ok = split
        out.append(split)
    return out


def slab_layout(N: int, P: int, rank: int, split: bool, halo: int = HALO) -> Layout | None:
    """Layout of rank ``rank``'s array on a level of side N; None when the
    level is whole on rank 0 and this is another rank."""
    if not split:
        return Layout(N, 0, N, 0, N) if rank == 0 else None
    n = N // P
    return Layout(N, rank * n - halo, n + 2 * halo, halo, halo + n)


# ---------------------------------------------------------------- communication
class Comm:
    """Process-group operations the slab solve needs, over torch.distributed.

    Tensors passed in live where the process group's backend wants them
    (CUDA for NCCL, CPU for gloo)."""

    def __init__(self, dist=None, group=None):
        if dist is None:
            import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.size = dist.get_world_size(group) if dist.is_initialized() else 1

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        """Send send_lo to the lower neighbour and send_hi to the upper one;
        receive the lower neighbour's send_hi into recv_lo and the upper
        neighbour's send_lo into recv_hi."""
        P = self.size
        if P == 1:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
            return
        d = self.dist
        lo, hi = (self.rank - 1) % P, (self.rank + 1) % P
        # with two ranks both neighbours are the same process: the tags (and,
        # for backends that ignore tags, the order of the operations, which is
        # the same on every rank) tell the two messages apart
        ops = [d.P2POp(d.isend, send_lo, lo, self.group, tag=1),
               d.P2POp(d.isend, send_hi, hi, self.group, tag=2),
               d.P2POp(d.irecv, recv_hi, hi, self.group, tag=1),
               d.P2POp(d.irecv, recv_lo, lo, self.group, tag=2)]
        for w in d.batch_isend_irecv(ops):
            w.wait()

    def all_gather(self, t):
        """List of every rank's tensor t (same shape on every rank)."""
        if self.size == 1:
            return [t]
        out = [t.new_empty(t.shape) for _ in range(self.size)]
        self.dist.all_gather(out, t, group=self.group)
        return out

    def gather0(self, t):
        """Rank 0 gets the list of every rank's t; the others get None."""
        if self.size == 1:
            return [t]
        out = [t.new_empty(t.shape) for _ in range(self.size)] if self.rank == 0 else None
        self.dist.gather(t, out, dst=0, group=self.group)
        return out

    def scatter0(self, chunks, out):
        """Rank 0's chunks[r] lands in rank r's out."""
        if self.size == 1:
            out.copy_(chunks[0])
            return
        self.dist.scatter(out, chunks if self.rank == 0 else None, src=0, group=self.group)

    def broadcast0(self, t):
        if self.size > 1:
            self.dist.broadcast(t, src=0, group=self.group)
        return t

    def min(self, t):
        if self.size > 1:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return t


# ---------------------------------------------------------------- backend
class SlabBackend:
    """The cell arithmetic of one rank.  Arrays are (planes, N, N) float64
    tensors described by a Layout; every method writes only the own planes
    of its output and reads the halos it needs (at most two planes).

    sweep(t, g, c, h, lay, rule)      one Gauss-Seidel sweep of eq. update
                                      (both colours, snapshot ordering; rule
                                      0 Newton step, 1 largest root) on the
                                      own planes; t needs its two-plane halo
                                      (or is whole), g one plane
    residual(t, g, c, h, lay, r)      r = g + c - det(I + H theta)  (one-plane halo)
    det(t, h, lay, out)               out = det(I + H theta)        (one-plane halo)
    restrict(f, lay_f, out, lay_c)    out's own planes = mean of 8 sons of f's own planes
    prolong_add(cn, co, lay_c, s, f, lay_f)
                                      f += s P(cn - co) (one-plane halo on cn, co)
    plane_sums(a, lay, m, sq)         per own plane: sum (a - m) or (a - m)^2
                                      (float64 tensor, on the comm device)
    eps_planes(t, g, c, h, lay)       per own plane: sum of L_h^2
    defect_min(dH, rr, lay, floor)    the scaled-defect factor over own planes
                                      (0 below 1e-3, as a whole-grid factor)
    form_rhs(dH, rr, s, lay, g)       g = dH + s rr    (own planes)
    sub(a, m, lay)                    a -= m            (own planes)
    coarse_solve(t, g, c, h, max_sweeps, rtol, rule)
                                      whole-grid solve of the coarsest level
                                      (Gauss-Seidel until the mean-free rms
                                      residual drops by rtol, stops falling,
                                      or max_sweeps)
    zeros(lay) / fill(a, v) / copy(dst, src)
                                      storage
    comm_device                       where the communication's small
                                      tensors live ("cpu" for gloo, the
                                      rank's CUDA device for NCCL)
    """


# ---------------------------------------------------------------- the solve
@dataclass
class SlabParams:
    nu1: int = 2
    nu2: int = 2
    coarse_max_sweeps: int = 200
    coarse_rtol: float = 1e-3
    rule: int = 0
    scale_floor: float = 0.5
    min_planes: int = 64


class SlabSolver:
    """FAS solve of det(I + H theta) = b + c on a grid split into slabs.

    Every rank calls ``solve`` with its own planes of b (level 0, the planes
    ``split_levels`` / ``slab_layout`` give it; when level 0 is not split,
    rank 0 passes the whole grid and the others None) and gets back its own
    planes of theta and the solve's statistics (the same on every rank)."""

    def __init__(self, N: int, L: float, backend, comm: Comm | None = None,
                 params: SlabParams | None = None):
        self.N, self.Lbox = int(N), float(L)
        self.be = backend
        self.comm = comm or Comm()
        self.P, self.rank = self.comm.size, self.comm.rank
        self.par = params or SlabParams()
        self.nlev = num_levels(self.N)
        self.split = split_levels(self.N, self.P, self.par.min_planes)
        self.lays = [slab_layout(self.N >> l, self.P, self.rank, self.split[l]) for l in range(self.nlev)]
        self.h = [self.Lbox / self.N * (1 << l) for l in range(self.nlev)]
        Z = self.be.zeros
        self.t = [Z(ly) if ly else None for ly in self.lays]
        self.g = [Z(ly) if ly else None for ly in self.lays]
        self.told = [Z(ly) if ly else None for ly in self.lays]
        self.r = [Z(ly) if ly else None for ly in self.lays]
        self.exchanges = 0

    # ---- communication helpers
    def _halo(self, l, a):
        """Fill a's halo planes from the neighbours (split levels only)."""
        if not self.split[l]:
            return
        ly = self.lays[l]
        w = ly.lo
        self.comm.exchange(a[ly.lo:ly.lo + w], a[ly.hi - w:ly.hi], a[0:w], a[ly.hi:ly.hi + w])
        self.exchanges += 1

    def _sum(self, l, a, m=0.0, sq=False, everywhere=False):
        """Sum over level l of (a - m) or (a - m)^2 from the plane partials,
        added in plane order.  On a split level every rank takes part and
        gets the sum; on a level held whole by rank 0 rank 0 sums alone, and
        with everywhere=True every rank calls and rank 0 broadcasts it."""
        ly = self.lays[l]
        if self.split[l]:
            return _ordered_sum(self.comm.all_gather(self.be.plane_sums(a, ly, m, sq)))
        s = _ordered_sum([self.be.plane_sums(a, ly, m, sq)]) if self.rank == 0 else 0.0
        return self._bcast_scalar(s) if everywhere else s

    def _bcast_scalar(self, x):
        import torch
        if self.P == 1:
            return x
        t = torch.tensor([x if self.rank == 0 else 0.0], dtype=torch.float64, device=self.be.comm_device)
        return float(self.comm.broadcast0(t).item())

    def _mean(self, l, a, everywhere=False):
        Nl = self.N >> l
        return self._sum(l, a, everywhere=everywhere) / float(Nl * Nl * Nl)

    def _restrict_to(self, l, fine, coarse):
        """Restriction of level l's own planes onto level l+1 (own planes, or
        gathered whole on rank 0 when level l+1 is not split)."""
        lf, lc = self.lays[l], self.lays[l + 1]
        if self.split[l + 1] or not self.split[l]:
            if lc is not None:
                self.be.restrict(fine, lf, coarse, lc)
            return
        # split -> whole: restrict into a slab-shaped buffer, gather on rank 0
        Nc = self.N >> (l + 1)
        nc = lf.own // 2
        tmp_ly = Layout(Nc, lf.own_first // 2, nc, 0, nc)
        tmp = self.be.zeros(tmp_ly)
        self.be.restrict(fine, lf, tmp, tmp_ly)
        parts = self.comm.gather0(tmp)
        if self.rank == 0:
            for r, p in enumerate(parts):
                self.be.copy(coarse[r * nc:(r + 1) * nc], p)

    def _coarse_for_prolong(self, l, a):
        """Level l+1's array a as the prolongation onto level l's own planes
        reads it: a itself (halo filled) when level l+1 is split or level l is
        whole; else each rank's coarse planes with one halo plane on each side,
        scattered from rank 0's whole grid.  Returns (array, layout)."""
        if self.split[l + 1]:
            self._halo(l + 1, a)
            return a, self.lays[l + 1]
        if not self.split[l]:
            return a, self.lays[l + 1]
        Nc = self.N >> (l + 1)
        nc = self.lays[l].own // 2
        ly = Layout(Nc, self.rank * nc - 1, nc + 2, 1, nc + 1)
        out = self.be.zeros(ly)
        chunks = None
        if self.rank == 0:
            import torch
            idx = [[(r * nc - 1 + p) % Nc for p in range(nc + 2)] for r in range(self.P)]
            chunks = [a[torch.tensor(ix, device=a.device)].contiguous() for ix in idx]
        self.comm.scatter0(chunks, out)
        return out, ly

    # ---- one level of the V-cycle (the single-process solve's steps, in order)
    def _sweeps(self, l, c, count):
        for _ in range(count):
            self._halo(l, self.t[l])
            self.be.sweep(self.t[l], self.g[l], c, self.h[l], self.lays[l], self.par.rule)

    def _vcycle(self, l, c):
        ly = self.lays[l]
        if ly is None:
            return self._vcycle_idle(l)
        par = self.par
        if l == self.nlev - 1:
            # the coarsest level is whole on rank 0
            self.be.coarse_solve(self.t[l], self.g[l], c, self.h[l], par.coarse_max_sweeps,
                                 par.coarse_rtol, par.rule)
            return
        self._sweeps(l, c, par.nu1)
        self._halo(l, self.t[l])
        self.be.residual(self.t[l], self.g[l], c, self.h[l], ly, self.r[l])
        self._restrict_to(l, self.t[l], self.t[l + 1])
        lc = self.lays[l + 1]
        sc = 0.0
        if lc is not None:
            self.be.copy(self.told[l + 1], self.t[l + 1])
            rr, dH = self.be.zeros(lc), self.be.zeros(lc)
        self._restrict_to(l, self.r[l], rr if lc is not None else None)
        if lc is not None:
            m = self._mean(l + 1, rr)
            self.be.sub(rr, m, lc)
            self._halo(l + 1, self.t[l + 1])
            self.be.det(self.t[l + 1], self.h[l + 1], lc, dH)
            sc = self.be.defect_min(dH, rr, lc, par.scale_floor)
        if self.split[l + 1]:
            sc = self._min_scalar(sc)
        elif self.split[l]:
            sc = self._bcast_scalar(sc)
        if sc > 0.0:
            if lc is not None:
                self.be.form_rhs(dH, rr, sc, lc, self.g[l + 1])
                self._halo(l + 1, self.g[l + 1])
            self._vcycle(l + 1, 0.0)
            cn, lyc = self._coarse_for_prolong(l, self.t[l + 1])
            co, _ = self._coarse_for_prolong(l, self.told[l + 1])
            self.be.prolong_add(cn, co, lyc, 1.0 / sc, self.t[l], ly)
        self._sweeps(l, c, par.nu2)

    def _vcycle_idle(self, l):
        """A rank without planes on level l (held whole by rank 0) waits."""
        return

    def _min_scalar(self, x):
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.be.comm_device)
        return float(self.comm.min(t).item())

    def _compat_and_gauge(self, l, c):
        """r = g + c - det(theta); c -= mean r; theta -= mean theta (every
        rank calls; c is known on every rank)."""
        ly = self.lays[l]
        if ly is not None:
            self._halo(l, self.t[l])
            self.be.residual(self.t[l], self.g[l], c, self.h[l], ly, self.r[l])
        c = c - self._mean(l, self.r[l], everywhere=True)
        mt = self._mean(l, self.t[l])
        if ly is not None:
            self.be.sub(self.t[l], mt, ly)
        return c

    def _prolong_start(self, l):
        """Nested iteration: theta_l = P theta_{l+1} (from zero)."""
        ly = self.lays[l]
        zc = None
        cn, lyc = self._coarse_for_prolong(l, self.t[l + 1])
        if ly is not None:
            self.be.fill(self.t[l], 0.0)
            zc = self.be.zeros(lyc)
            self.be.prolong_add(cn, zc, lyc, 1.0, self.t[l], ly)

    # ---- the solve
    def solve(self, b_own, tol: float = 1e-10, max_cycles: int = 50):
        """FAS solve from nested iteration (theta = 0 on the coarsest grid).

        b_own: this rank's even share of the planes of b, planes
        [rank N/P, (rank + 1) N/P) as an (N/P, N, N) float64 tensor on the
        backend's device (N must be a multiple of P).  Returns (theta_own,
        info): theta on the same planes, and info =
        dict(status, cycles, rel_residual, c, paper_eps, history); status 0 =
        converged, 3 = max_cycles reached, 4 = non-finite residual."""
        ly0 = self.lays[0]
        if self.N % self.P:
            raise ValueError("the grid's side must be a multiple of the number of ranks")
        if self.split[0] or self.P == 1:
            self.be.copy(self.g[0][ly0.lo:ly0.hi], b_own)
            self._halo(0, self.g[0])
        else:
            parts = self.comm.gather0(b_own.contiguous())
            if self.rank == 0:
                n = self.N // self.P
                for r, p in enumerate(parts):
                    self.be.copy(self.g[0][r * n:(r + 1) * n], p)
        # b down the hierarchy
        for l in range(1, self.nlev):
            self._restrict_to(l - 1, self.g[l - 1], self.g[l])
            self._halo(l, self.g[l])
        lc = self.nlev - 1
        c = 0.0
        if self.lays[lc] is not None:
            self.be.fill(self.t[lc], 0.0)
        self._vcycle(lc, c)
        c = self._compat_and_gauge(lc, c)
        for l in range(lc - 1, -1, -1):
            self._prolong_start(l)
            if l == 0:
                break
            self._vcycle(l, c)
            c = self._compat_and_gauge(l, c)
        Nn = float(self.N) ** 3
        denom = math.sqrt(self._sum(0, self.g[0], 1.0, True, everywhere=True))
        if denom == 0.0:
            denom = 1.0
        hist, rel, status, cyc = [], 0.0, 3, 0
        for cyc in range(1, max_cycles + 1):
            self._vcycle(0, c)
            if ly0 is not None:
                self._halo(0, self.t[0])
                self.be.residual(self.t[0], self.g[0], c, self.h[0], ly0, self.r[0])
            m = self._sum(0, self.r[0], everywhere=True) / Nn
            c -= m
            mt = self._sum(0, self.t[0]) / Nn
            if ly0 is not None:
                self.be.sub(self.t[0], mt, ly0)
            rel = math.sqrt(self._sum(0, self.r[0], m, True, everywhere=True)) / denom
            hist.append(rel)
            if not math.isfinite(rel):
                status = 4
                break
            if rel < tol:
                status = 0
                break
        if ly0 is not None:
            self._halo(0, self.t[0])
            eps_parts = self.be.eps_planes(self.t[0], self.g[0], c, self.h[0], ly0)
        if self.split[0]:
            eps_sum = _ordered_sum(self.comm.all_gather(eps_parts))
        else:
            eps_sum = self._bcast_scalar(_ordered_sum([eps_parts]) if self.rank == 0 else 0.0)
        info = dict(status=status, cycles=cyc, rel_residual=rel, c=c,
                    paper_eps=math.sqrt(eps_sum / Nn), history=hist)
        theta = self.t[0][ly0.lo:ly0.hi] if ly0 is not None else None
        if not self.split[0] and self.P > 1:
            theta = self._scatter_level0(theta)
        return theta, info

    def _scatter_level0(self, whole):
        """Level 0 whole on rank 0: hand every rank its even share of planes."""
        n = self.N // self.P
        out = self.be.zeros(Layout(self.N, self.rank * n, n, 0, n))
        chunks = [whole[r * n:(r + 1) * n].contiguous() for r in range(self.P)] if self.rank == 0 else None
        self.comm.scatter0(chunks, out)
        return out


class GpuSlabBackend:
    """The per-rank steps as the recon_slab_* kernels of librecon.so, on this
    process's current CUDA device and stream (FP64)."""

    def __init__(self, device=None):
        import torch
        from . import recon
        recon.load()
        self.R = recon
        self.torch = torch
        self.comm_device = torch.device(device) if device is not None else torch.device("cuda")
        self._work = {}

    def zeros(self, lay):
        return self.torch.zeros((lay.planes, lay.N, lay.N), dtype=self.torch.float64, device=self.comm_device)

    def fill(self, a, v):
        a.fill_(v)

    def copy(self, dst, src):
        dst.copy_(src)

    def _scratch(self, lay):
        key = (lay.N, lay.planes)
        if key not in self._work:
            self._work[key] = self.zeros(lay)
        return self._work[key]

    def sweep(self, t, g, c, h, lay, rule):
        self.R.recon_slab_sweep(lay, h, rule, t, g, c, self._scratch(lay))

    def residual(self, t, g, c, h, lay, r):
        self.R.recon_slab_residual(lay, h, t, g, c, r)

    def det(self, t, h, lay, out):
        self.R.recon_slab_det(lay, h, t, out)

    def restrict(self, f, lay_f, out, lay_c):
        self.R.recon_slab_restrict(lay_f, f, lay_c, out)

    def prolong_add(self, cn, co, lay_c, scale, f, lay_f):
        self.R.recon_slab_prolong_add(lay_c, cn, co, scale, lay_f, f)

    def _per_plane(self, lay):
        return self.torch.empty(lay.own, dtype=self.torch.float64, device=self.comm_device)

    def plane_sums(self, a, lay, m, sq):
        out = self._per_plane(lay)
        self.R.recon_slab_plane_sums(lay, a, m, sq, out)
        return out

    def eps_planes(self, t, g, c, h, lay):
        out = self._per_plane(lay)
        self.R.recon_slab_eps_planes(lay, h, t, g, c, out)
        return out

    def defect_min(self, dH, rr, lay, floor):
        if floor <= 0.0:
            return 1.0
        out = self._per_plane(lay)
        self.R.recon_slab_defect_min(lay, dH, rr, floor, out)
        s = min(out.tolist())
        return 0.0 if s < 1e-3 else s

    def form_rhs(self, dH, rr, s, lay, g):
        self.R.recon_slab_form_rhs(lay, dH, rr, s, g)

    def sub(self, a, m, lay):
        self.R.recon_slab_sub(lay, a, m)

    def coarse_solve(self, t, g, c, h, max_sweeps, rtol, rule):
        self.R.recon_step_coarse_solve(t, g, c, h, max_sweeps, rtol, rule)


def _ordered_sum(parts) -> float:
    """Add the plane partials of all ranks in plane order (rank order, then
    plane order within a rank), one IEEE addition at a time."""
    s = 0.0
    for p in parts:
        for x in p.tolist():
            s += x
    return s
