"""Batched solves of uneven N (recon_batch_*) against single solves and the oracle."""
import numpy as np
import pytest

from tests.workloads import zeldovich_density

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    return recon


def test_batch_matches_single_solves_and_oracle(R, O):
    sizes = [16, 24, 32, 48, 64, 96, 128, 32]
    boxes = [2.0 * n for n in sizes]
    bs_np = [zeldovich_density(O, n, L, 0.8, 4.0, 4000 + i)[0]
             for i, (n, L) in enumerate(zip(sizes, boxes))]
    bs = [torch.from_numpy(b).cuda() for b in bs_np]
    B = R.Batch(sizes, boxes)
    phis, stats = B.solve(bs, tol=1e-10, max_cycles=30)
    for i, (n, L) in enumerate(zip(sizes, boxes)):
        assert stats[i]["rel_residual"] < 1e-10
        s = R.Solver(n, L, R.RECON_MIXED)
        ref, _ = s.solve(bs[i], tol=1e-10, max_cycles=30)
        got = phis[i].cpu().numpy()
        assert np.linalg.norm(got - ref.cpu().numpy()) < 1e-7 * np.linalg.norm(ref.cpu().numpy())
        s.close()
        if n <= 48:
            o, _ = O.solve(bs_np[i], L, tol=1e-10, max_cycles=40)
            assert np.linalg.norm(got - o) < 1e-6 * np.linalg.norm(o)
    # second call reuses the captured graphs and gives the same answers
    again = [torch.zeros_like(p) for p in phis]
    phis2, _ = B.solve(bs, phis=again, tol=1e-10, max_cycles=30)
    phis3, _ = B.solve(bs, phis=again, tol=1e-10, max_cycles=30)
    for p2, p3 in zip(phis2, phis3):
        assert torch.equal(p2, p3)
    B.close()


def test_batch_rejects_bad_density(R):
    B = R.Batch([16, 16], [16.0, 16.0])
    bs = [torch.ones((16,) * 3, dtype=torch.float64, device="cuda") for _ in range(2)]
    bs[1][0, 0, 0] = -1.0
    with pytest.raises(R.ReconError) as e:
        B.solve(bs)
    assert e.value.status == 2 and "realisation 1" in str(e.value)
    B.close()
