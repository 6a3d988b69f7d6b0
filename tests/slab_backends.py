"""A slab backend whose cell arithmetic is the oracle's (test infrastructure).

Each step embeds the rank's planes (own planes and halos) at their global
positions in a whole N^3 grid filled with NaN, runs the oracle's whole-grid
routine on it and keeps the own planes of the result.  A value a rank does
not hold is NaN, so a step that read outside the planes the decomposition
provides would leave NaN in the rank's own planes."""
import numpy as np
import torch


class OracleSlabBackend:
    comm_device = "cpu"

    def __init__(self, O):
        self.O = O

    # storage
    def zeros(self, lay):
        return torch.zeros((lay.planes, lay.N, lay.N), dtype=torch.float64)

    def fill(self, a, v):
        a.fill_(v)

    def copy(self, dst, src):
        dst.copy_(src)

    # whole-grid embedding
    def _embed(self, a, lay):
        full = np.full((lay.N,) * 3, np.nan)
        full[(lay.first + np.arange(lay.planes)) % lay.N] = a.numpy()
        return full

    def _own(self, full, lay):
        return torch.from_numpy(np.ascontiguousarray(full[(lay.own_first + np.arange(lay.own)) % lay.N]))

    def _ownv(self, a, lay):
        return a[lay.lo:lay.hi].numpy()

    # steps
    def sweep(self, t, g, c, h, lay, rule):
        out = self.O.sweep(self._embed(t, lay), self._embed(g, lay), c, h, "rb-snapshot",
                           "newton1" if rule == 0 else "exact")
        t[lay.lo:lay.hi] = self._own(out, lay)

    def residual(self, t, g, c, h, lay, r):
        r[lay.lo:lay.hi] = self._own(self.O.residual(self._embed(t, lay), self._embed(g, lay), c, h), lay)

    def det(self, t, h, lay, out):
        out[lay.lo:lay.hi] = self._own(self.O.det_grid(self._embed(t, lay), h), lay)

    def restrict(self, f, lay_f, out, lay_c):
        out[lay_c.lo:lay_c.hi] = self._own(self.O.restrict(self._embed(f, lay_f)), lay_c)

    def prolong_add(self, cn, co, lay_c, scale, f, lay_f):
        res = self.O.prolong_add(self._embed(cn, lay_c), self._embed(co, lay_c), self._embed(f, lay_f), scale)
        f[lay_f.lo:lay_f.hi] = self._own(res, lay_f)

    def plane_sums(self, a, lay, m, sq):
        return torch.from_numpy(self.O.plane_sums(self._ownv(a, lay), m, sq))

    def eps_planes(self, t, g, c, h, lay):
        parts = self.O.paper_eps_planes(self._embed(t, lay), self._embed(g, lay), c, h)
        return torch.from_numpy(np.ascontiguousarray(parts[(lay.own_first + np.arange(lay.own)) % lay.N]))

    def defect_min(self, dH, rr, lay, floor):
        return self.O.defect_scale(self._ownv(dH, lay), self._ownv(rr, lay), floor)

    def form_rhs(self, dH, rr, s, lay, g):
        g[lay.lo:lay.hi] = dH[lay.lo:lay.hi] + rr[lay.lo:lay.hi] * s

    def sub(self, a, m, lay):
        a[lay.lo:lay.hi] -= m

    def coarse_solve(self, t, g, c, h, max_sweeps, rtol, rule):
        out, _ = self.O.coarse_solve(t.numpy(), g.numpy(), c, h, max_sweeps, rtol, "rb-snapshot",
                                     "newton1" if rule == 0 else "exact")
        t.copy_(torch.from_numpy(out))


class ThreadGroup:
    """P ranks as threads of one process: the collectives of slab.Comm done
    through shared slots and a barrier (with a timeout, so a rank that
    diverges fails the test instead of waiting forever).  Tensors are cloned
    when posted, so on a GPU every copy is ordered on the shared stream after
    the kernels that wrote its source."""

    def __init__(self, P, timeout=120.0):
        import threading
        self.P = P
        self.slots = [None] * P
        self.barrier = threading.Barrier(P, timeout=timeout)


class ThreadComm:
    def __init__(self, group, rank):
        self.g, self.rank, self.size = group, rank, group.P

    def _post(self, obj):
        self.g.slots[self.rank] = obj
        self.g.barrier.wait()
        vals = list(self.g.slots)
        self.g.barrier.wait()
        return vals

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        vals = self._post((send_lo.clone(), send_hi.clone()))
        P = self.size
        recv_lo.copy_(vals[(self.rank - 1) % P][1])
        recv_hi.copy_(vals[(self.rank + 1) % P][0])

    def all_gather(self, t):
        return self._post(t.clone())

    def gather0(self, t):
        vals = self._post(t.clone())
        return vals if self.rank == 0 else None

    def scatter0(self, chunks, out):
        vals = self._post([c.clone() for c in chunks] if self.rank == 0 else None)
        out.copy_(vals[0][self.rank])

    def broadcast0(self, t):
        vals = self._post(t.clone() if self.rank == 0 else None)
        t.copy_(vals[0])
        return t

    def min(self, t):
        vals = self._post(t.clone())
        t.copy_(torch.stack(vals).min(0).values)
        return t


def run_threads(P, fn):
    """fn(rank, comm) on P threads; returns the results in rank order (an
    exception in any rank is raised here)."""
    import threading
    grp = ThreadGroup(P)
    out, err = [None] * P, []

    def body(r):
        try:
            out[r] = fn(r, ThreadComm(grp, r))
        except BaseException as e:          # noqa: BLE001 - reported below
            err.append(e)
            grp.barrier.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(P)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out
