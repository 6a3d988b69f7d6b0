"""The slab-decomposed FAS solve (several processes, one slab of planes each)
on CPU: gloo ranks with the oracle's cell arithmetic reproduce the
single-process oracle solve bit for bit, at world sizes 1, 2 and 4, with
levels split across ranks, levels agglomerated on rank 0, and the coarsest
solve on rank 0 (Sec. II.A.3 hierarchy; the halo, sum and agglomeration
rules are the decomposition's own)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1709_06350_gb300 import slab

L_BOX = 64.0
KW = dict(nu1=2, nu2=2, coarse_max_sweeps=200, coarse_rtol=1e-3, rule=0, scale_floor=0.5)


def _density(O, N, seed):
    from tests.workloads import zeldovich_density
    b, _, _ = zeldovich_density(O, N, L_BOX, 0.8, 2.5 * L_BOX / N, seed)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


# ---------------------------------------------------------------- host logic
def test_levels_and_layouts():
    assert slab.num_levels(512) == 8 and slab.num_levels(96) == 5 and slab.num_levels(6) == 1
    # 512^3 on 8 ranks: only the finest level has 64 planes per rank
    assert slab.split_levels(512, 8) == [True] + [False] * 7
    assert slab.split_levels(1024, 8) == [True, True] + [False] * 7
    assert slab.split_levels(512, 1) == [False] * 8
    # small slabs for the tests: 32^3 on 4 ranks, 2 planes per rank allowed
    assert slab.split_levels(32, 4, min_planes=2) == [True, True, True, False]
    # an odd number of own planes cannot restrict onto whole coarse planes:
    # 24^3 on 4 ranks splits 6 planes each, whose 3 restricted planes go to
    # rank 0; 12^3 (3 planes each) is not split at all
    assert slab.split_levels(24, 4, min_planes=2) == [True, False, False]
    assert slab.split_levels(12, 4, min_planes=2) == [False, False]
    # the slab plus its halos must fit in the grid
    assert slab.split_levels(8, 2, min_planes=2) == [True, False]
    assert slab.split_levels(4 * 2, 2, min_planes=2)[0] is True
    lay = slab.slab_layout(32, 4, 0, True)
    assert (lay.first, lay.planes, lay.lo, lay.hi, lay.own_first) == (-2, 12, 2, 10, 0)
    lay = slab.slab_layout(32, 4, 3, True)
    assert (lay.first, lay.own_first, lay.own) == (22, 24, 8)
    assert slab.slab_layout(32, 4, 2, False) is None
    assert slab.slab_layout(32, 4, 0, False).whole


def test_plane_sums_pin(O):
    """The oracle's grid sums are per-plane running sums added in plane
    order: checked against explicit loops, bit for bit."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, 4, 4)) * 10.0 ** rng.integers(-8, 8, size=(3, 4, 4))
    want, want2 = [], []
    for i in range(3):
        s = s2 = 0.0
        for x in a[i].ravel().tolist():
            s += x - 0.25
            s2 += (x - 0.25) * (x - 0.25)
        want.append(s)
        want2.append(s2)
    assert O.plane_sums(a, 0.25).tolist() == want
    assert O.plane_sums(a, 0.25, squared=True).tolist() == want2


def _solve_ranks(O, b, P, min_planes, tol, max_cycles, rank=0, comm=None):
    be = __import__("tests.slab_backends", fromlist=["x"]).OracleSlabBackend(O)
    N = b.shape[0]
    sv = slab.SlabSolver(N, L_BOX, be, comm or slab.Comm(),
                         slab.SlabParams(**KW, min_planes=min_planes))
    n = N // sv.P
    th, info = sv.solve(torch.from_numpy(np.ascontiguousarray(b[rank * n:(rank + 1) * n])), tol, max_cycles)
    return th.numpy().copy(), info, sv.split, sv.exchanges


def _same_as_oracle(O, b, theta, info, tol, max_cycles):
    kw = dict(KW, rule="newton1" if KW["rule"] == 0 else "exact")
    t_or, i_or = O.solve(b, L_BOX, tol=tol, max_cycles=max_cycles, ordering="rb-snapshot", **kw)
    assert info["status"] == i_or["status"] and info["cycles"] == i_or["cycles"]
    assert np.array_equal(theta, t_or)
    assert info["c"] == i_or["c"]
    assert info["history"] == i_or["history"]
    assert info["rel_residual"] == i_or["rel_residual"]
    assert info["paper_eps"] == i_or["paper_eps"]


def test_one_rank_equals_oracle(O):
    b = _density(O, 16, 41)
    th, info, split, _ = _solve_ranks(O, b, 1, 2, 1e-9, 12)
    assert split == [False] * 3
    _same_as_oracle(O, b, th, info, 1e-9, 12)


def _rank_main(rank, world, port, N, seed, min_planes, tol, max_cycles, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    torch.set_num_threads(1)
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _density(O, N, seed)
        th, info, split, ex = _solve_ranks(O, b, world, min_planes, tol, max_cycles, rank, slab.Comm(dist))
        out[rank] = (th, info, split, ex)
    finally:
        dist.destroy_process_group()


def _run_world(world, N, seed, min_planes, tol, max_cycles):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, N, seed, min_planes, tol, max_cycles, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    for p in procs:
        if p.exitcode is None:
            p.kill()
        assert p.exitcode == 0
    return [out[r] for r in range(world)]


@pytest.mark.parametrize("world,N,min_planes,want_split", [
    (2, 16, 2, [True, True, False]),           # split down to the coarsest solve
    (4, 32, 2, [True, True, True, False]),
    (2, 32, 8, [True, True, False, False]),    # 8^3 agglomerated on rank 0 above the coarsest
])
def test_gloo_ranks_equal_oracle(O, world, N, min_planes, want_split):
    tol, max_cycles = 1e-9, 12
    res = _run_world(world, N, 43 + world, min_planes, tol, max_cycles)
    theta = np.concatenate([r[0] for r in res])
    for th, info, split, ex in res:
        assert split == want_split and ex > 0
        assert info == res[0][1]                  # the same statistics on every rank
    b = _density(O, N, 43 + world)
    _same_as_oracle(O, b, theta, res[0][1], tol, max_cycles)
    assert res[0][1]["status"] == 0


def test_gloo_whole_grid_on_rank0(O):
    """A grid too small to split: every level on rank 0, theta scattered back."""
    res = _run_world(2, 8, 7, 64, 1e-9, 10)
    assert all(r[2] == [False, False] for r in res)
    b = _density(O, 8, 7)
    _same_as_oracle(O, b, np.concatenate([r[0] for r in res]), res[0][1], 1e-9, 10)


def test_thread_ranks_equal_oracle(O):
    """The same decomposition with ranks as threads of one process (the form
    the GPU test uses on one GPU) also reproduces the oracle bit for bit."""
    from tests.slab_backends import OracleSlabBackend, run_threads
    N, tol, max_cycles = 32, 1e-9, 12
    b = _density(O, N, 47)

    def rank_fn(r, comm):
        sv = slab.SlabSolver(N, L_BOX, OracleSlabBackend(O), comm, slab.SlabParams(**KW, min_planes=2))
        n = N // 4
        th, info = sv.solve(torch.from_numpy(np.ascontiguousarray(b[r * n:(r + 1) * n])), tol, max_cycles)
        return th.numpy().copy(), info, sv.split

    res = run_threads(4, rank_fn)
    assert res[0][2] == [True, True, True, False]
    _same_as_oracle(O, b, np.concatenate([r[0] for r in res]), res[0][1], tol, max_cycles)
