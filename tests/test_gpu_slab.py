"""The slab-decomposed FP64 solve on the GPU: the recon_slab_* kernels as
each rank's arithmetic.  One rank (whole grids) is checked against the
oracle's solve; 2 and 4 ranks, run as threads of one process on the one GPU
(halos and sums exchanged on the host between launches; no kernel waits on
another), reproduce the one-rank GPU result bit for bit, and the library's
own FP64 solve to its parity tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L_BOX = 64.0
PAR = dict(nu1=2, nu2=2, coarse_max_sweeps=200, coarse_rtol=1e-3, rule=0, scale_floor=0.5)


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    recon.load()
    return recon


def _density(O, N, seed):
    from tests.workloads import zeldovich_density
    b, _, _ = zeldovich_density(O, N, L_BOX, 0.8, 2.5 * L_BOX / N, seed)
    return b


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_solve(b, P, min_planes, tol, max_cycles):
    from paper_1709_06350_gb300 import slab
    from tests.slab_backends import run_threads
    N = b.shape[0]
    n = N // P
    bd = torch.from_numpy(b).cuda()

    def rank_fn(r, comm):
        sv = slab.SlabSolver(N, L_BOX, slab.GpuSlabBackend(), comm, slab.SlabParams(**PAR, min_planes=min_planes))
        th, info = sv.solve(bd[r * n:(r + 1) * n].contiguous(), tol, max_cycles)
        torch.cuda.synchronize()
        return th.cpu().numpy(), info, sv.split

    if P == 1:
        from paper_1709_06350_gb300 import slab as S
        sv = S.SlabSolver(N, L_BOX, S.GpuSlabBackend(), S.Comm(), S.SlabParams(**PAR, min_planes=min_planes))
        th, info = sv.solve(bd, tol, max_cycles)
        return th.cpu().numpy(), info, sv.split
    res = run_threads(P, rank_fn)
    for r in res[1:]:
        assert r[1] == res[0][1]
    return np.concatenate([r[0] for r in res]), res[0][1], res[0][2]


def test_one_rank_matches_oracle(R, O):
    N, tol = 32, 1e-10
    b = _density(O, N, 61)
    th, info, split = _gpu_solve(b, 1, 2, tol, 30)
    ref, i_or = O.solve(b, L_BOX, tol=tol, max_cycles=30, ordering="rb-snapshot",
                        **dict(PAR, rule="newton1"))
    assert info["status"] == 0 and i_or["status"] == 0
    assert rel_l2(th, ref) < 1e-10
    assert abs(info["cycles"] - i_or["cycles"]) <= 1
    assert info["c"] == pytest.approx(i_or["c"], rel=1e-6, abs=1e-13)
    np.testing.assert_allclose(info["history"][:3], i_or["history"][:3], rtol=1e-6)
    assert info["paper_eps"] == pytest.approx(i_or["paper_eps"], rel=1e-4, abs=1e-12)


@pytest.mark.parametrize("P,N,min_planes,want", [
    (2, 32, 8, [True, True, False, False]),     # 8^3 agglomerated on rank 0 above the coarsest
    (4, 32, 2, [True, True, True, False]),
    (4, 128, 8, [True, True, True, False, False, False]),
])
def test_ranks_equal_one_rank_bitwise(R, O, P, N, min_planes, want):
    tol = 1e-10
    b = _density(O, N, 62 + P)
    th1, i1, _ = _gpu_solve(b, 1, min_planes, tol, 30)
    thP, iP, split = _gpu_solve(b, P, min_planes, tol, 30)
    assert split == want
    assert i1["status"] == 0
    assert np.array_equal(thP, th1)
    assert iP == i1


def test_matches_library_fp64_solve(R, O):
    """The decomposed solve and the single-GPU FP64 solver agree."""
    N, tol = 128, 1e-10
    b = _density(O, N, 70)
    th, info, _ = _gpu_solve(b, 4, 8, tol, 30)
    s = R.Solver(N, L_BOX, R.RECON_F64, start=0, **PAR)
    phi, st = s.solve(torch.from_numpy(b).cuda(), tol=tol, max_cycles=30)
    got = phi.cpu().numpy()
    s.close()
    assert info["status"] == 0 and st["rel_residual"] < tol
    assert rel_l2(th, got) < 1e-8
