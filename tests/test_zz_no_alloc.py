"""The coarsest-grid solve that allocates no device memory.

recon_step_coarse_solve_noalloc serves callers that cannot call cudaMalloc
when they run this step (a host that reserves all device memory for its own
pool, a loop that forbids allocation after start-up, code inside a library
that does not own the device).  It must give the same answer as
recon_step_coarse_solve, whose scratch the caller allocates, call after call:
the fixed scratch keeps the previous call's contents, which must not leak
into the next result.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _density(N, seed):
    from paper_1709_06350_gb300 import synth
    b = 1.0 + synth.smooth_field(N, seed, 0.6, kmax=2)
    return b / b.mean()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_allocating_coarse_solve_twice(dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    cases = [(16, 40.0, 11, 200, 1e-3), (6, 12.0, 12, 9, 0.0)]   # two calls in a row
    for N, L, seed, sweeps, rtol in cases:
        h = L / N
        g = torch.from_numpy(_density(N, seed)).to(device="cuda", dtype=dtype)
        ref = torch.zeros((N,) * 3, dtype=dtype, device="cuda")
        n_ref = recon.recon_step_coarse_solve(ref, g, 0.01, h, max_sweeps=sweeps, rtol=rtol)
        got = torch.zeros_like(ref)
        done = torch.zeros(1, dtype=torch.int32, device="cuda")
        recon.recon_step_coarse_solve_noalloc(got, g, 0.01, h, max_sweeps=sweeps, rtol=rtol,
                                              sweeps_done=done)
        torch.cuda.synchronize()
        a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert int(done.item()) == n_ref
        assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-300)


def test_noalloc_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    t = torch.zeros((18,) * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(recon.ReconError) as e:
        recon.recon_step_coarse_solve_noalloc(t, torch.ones_like(t), 0.0, 1.0)
    assert e.value.status == 1 and "4096" in str(e.value)
