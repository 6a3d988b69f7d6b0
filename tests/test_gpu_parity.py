"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 steps agree to 1e-12 relative (only the order of rounding
differs); index work (restriction sums, CIC cells) is bit-exact; a full FP64
solve agrees to 1e-10 relative L2 and a MIXED solve to 1e-6 (both converge to
the same discrete solution; the bound is the stated target of each path).
"""
import numpy as np
import pytest

from tests.workloads import smooth_density, zeldovich_density

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    recon.load()
    return recon


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ steps
@pytest.mark.parametrize("N", [4, 6, 10, 48, 128, 160])
@pytest.mark.parametrize("rule", ["newton1", "exact"])
def test_sweep_parity(R, O, N, rule):
    """N >= 128 runs the fused shared-memory sweep (160: a ragged k-tile)."""
    L = 1.5 * N
    h = L / N
    from paper_1709_06350_gb300 import synth
    t0 = synth.smooth_field(N, 3, 0.4 * h * h, kmax=2)
    g = smooth_density(N, 4, 0.8)
    c = 0.013
    ref = O.sweep(t0, g, c, h, rule=rule, sweeps=3)
    th = dev(t0)
    R.recon_step_sweep(th, dev(g), c, h, sweeps=3, rule=R.RULE_EXACT if rule == "exact" else R.RULE_NEWTON1)
    assert rel_max(host(th), ref) < 1e-12


@pytest.mark.parametrize("N", [32, 128])
def test_sweep_fp32_tracks_fp64(R, O, N):
    L = float(N)
    h = L / N
    from paper_1709_06350_gb300 import synth
    t0 = synth.smooth_field(N, 5, 0.3, kmax=2)
    g = smooth_density(N, 6, 0.8)
    ref = O.sweep(t0, g, 0.0, h, sweeps=2)
    th = dev(t0, torch.float32)
    R.recon_step_sweep(th, dev(g, torch.float32), 0.0, h, sweeps=2)
    assert rel_max(host(th), ref) < 1e-4


@pytest.mark.parametrize("N", [6, 48, 128, 144])
def test_linear_sweep_vs_oracle_jacobian(R, O, N):
    """Red-black Gauss-Seidel on J e = f against the same sweep written with
    the oracle's sparse Jacobian (N >= 128 runs the fused kernel, which forms
    the cofactors from theta; 144: a ragged k-tile)."""
    L = 2.0 * N
    h = L / N
    from paper_1709_06350_gb300 import synth
    t = synth.smooth_field(N, 21, 0.4 * h * h, kmax=3).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(22)
    f = rng.standard_normal((N,) * 3).astype(np.float32).astype(np.float64)
    e0 = (0.1 * rng.standard_normal((N,) * 3)).astype(np.float32).astype(np.float64)
    J = O.jacobian_matrix(t, h)
    d = J.diagonal()
    i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    red = ((i + j + k) % 2 == 0).ravel()
    e = e0.ravel().copy()
    for _ in range(2):
        for col in (red, ~red):
            upd = e + (f.ravel() - J @ e) / d
            e = np.where(col, upd, e)
    ev = dev(e0, torch.float32)
    R.recon_step_linear_sweep(ev, dev(f, torch.float32), dev(t, torch.float32), h, sweeps=2)
    assert rel_max(host(ev).ravel(), e) < 2e-5


def _offset_view(x):
    """the same values in a contiguous tensor whose storage starts one element
    past an allocation boundary (not aligned to an element pair)"""
    buf = torch.empty(x.numel() + 1, dtype=x.dtype, device=x.device)
    v = buf[1:].view(x.shape)
    v.copy_(x)
    return v


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_fused_and_two_pass_sweeps_agree(R, dtype):
    """An unaligned theta runs the two-pass kernels; an aligned one the fused
    kernel: same sweeps, same results up to rounding order."""
    N, h = 128, 1.0
    from paper_1709_06350_gb300 import synth
    t0 = dev(synth.smooth_field(N, 31, 0.3, kmax=3), dtype)
    g = dev(smooth_density(N, 32, 0.8), dtype)
    a = t0.clone()
    R.recon_step_sweep(a, g, 0.01, h, sweeps=2)
    b = _offset_view(t0)
    assert b.data_ptr() % (2 * b.element_size()) != 0
    R.recon_step_sweep(b, g, 0.01, h, sweeps=2)
    tol = 1e-5 if dtype == torch.float32 else 1e-13
    assert rel_max(host(b), host(a)) < tol
    # linear smoother
    th = dev(synth.smooth_field(N, 33, 0.3, kmax=3), torch.float32)
    f = dev(np.random.default_rng(34).standard_normal((N,) * 3), torch.float32)
    e0 = torch.zeros_like(f)
    ea = e0.clone()
    R.recon_step_linear_sweep(ea, f, th, h, sweeps=2)
    eb = _offset_view(e0)
    R.recon_step_linear_sweep(eb, f, th, h, sweeps=2)
    assert rel_max(host(eb), host(ea)) < 1e-5


@pytest.mark.parametrize("N", [4, 12, 48])
def test_residual_det_jacobian_parity(R, O, N):
    L = 2.0 * N
    h = L / N
    from paper_1709_06350_gb300 import synth
    t = synth.smooth_field(N, 7, 0.5 * h * h, kmax=3)
    g = smooth_density(N, 8)
    v = np.random.default_rng(9).standard_normal((N,) * 3)
    out = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    R.recon_step_residual(dev(t), dev(g), 0.02, h, out)
    assert np.max(np.abs(host(out) - O.residual(t, g, 0.02, h))) < 1e-13
    R.recon_step_det(dev(t), h, out)
    assert np.max(np.abs(host(out) - O.det_grid(t, h))) < 1e-13
    R.recon_step_jacobian_apply(dev(t), dev(v), h, out)
    assert rel_max(host(out), O.jacobian_apply(t, v, h)) < 1e-12


@pytest.mark.parametrize("Nf", [4, 10, 48])
def test_restriction_bit_exact(R, O, Nf):
    f = np.random.default_rng(Nf).standard_normal((Nf,) * 3)
    out = torch.empty((Nf // 2,) * 3, dtype=torch.float64, device="cuda")
    R.recon_step_restrict(dev(f), out)
    assert np.array_equal(host(out), O.restrict(f))


@pytest.mark.parametrize("Nc", [2, 5, 24])
def test_prolongation_parity(R, O, Nc):
    rng = np.random.default_rng(Nc)
    cn, co, fi = rng.standard_normal((Nc,) * 3), rng.standard_normal((Nc,) * 3), rng.standard_normal((2 * Nc,) * 3)
    ref = O.prolong_add(cn, co, fi, scale=1.7)
    out = dev(fi)
    R.recon_step_prolong_add(dev(cn), dev(co), out, scale=1.7)
    assert np.max(np.abs(host(out) - ref)) < 1e-14


@pytest.mark.parametrize("N", [4, 6, 16])
def test_coarse_solve_parity(R, O, N):
    L = 3.0 * N
    h = L / N
    g = smooth_density(N, 10 + N, 0.7)
    ref, n_ref = O.coarse_solve(np.zeros((N,) * 3), g, 0.0, h, max_sweeps=9, rtol=0.0, rule="newton1")
    th = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    n = R.recon_step_coarse_solve(th, dev(g), 0.0, h, max_sweeps=9, rtol=0.0)
    assert n == n_ref == 9
    assert rel_max(host(th), ref) < 1e-12
    # to-tolerance mode: same decision on when to stop (allow one sweep)
    ref2, n2 = O.coarse_solve(np.zeros((N,) * 3), g, 0.0, h, max_sweeps=200, rtol=1e-3)
    th2 = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    m2 = R.recon_step_coarse_solve(th2, dev(g), 0.0, h, max_sweeps=200, rtol=1e-3)
    assert abs(m2 - n2) <= 1


def test_cic_cells_bit_exact(R, O):
    from paper_1709_06350_gb300 import synth
    N, L = 32, 100.0
    _, dh = synth.linear_field(N, L, 0.8, 77)
    pos = synth.zeldovich_positions(dh, N, L)
    edge = np.array([[0.0, L - 1e-13, 50.0], [L / N * 3, L / N * 0.5, 99.999999999]])
    pos = np.concatenate([pos, edge])
    cells_ref, frac_ref = O.cic_cells(pos, N, L)
    cells = torch.empty(pos.shape, dtype=torch.int32, device="cuda")
    frac = torch.empty(pos.shape, dtype=torch.float64, device="cuda")
    R.recon_step_cic_cells(dev(pos), N, L, cells, frac)
    torch.cuda.synchronize()
    assert np.array_equal(cells.cpu().numpy(), cells_ref)
    assert np.array_equal(frac.cpu().numpy(), frac_ref)


@pytest.mark.parametrize("N,L", [(32, 100.0), (48, 96.0), (32, 32.0), (64, 128.0), (32, 8.0)])
def test_cic_deposit_parity(R, O, N, L):
    from paper_1709_06350_gb300 import synth
    _, dh = synth.linear_field(N, L, 1.0, 78)
    pos = synth.zeldovich_positions(dh, N, L)
    ref = O.cic_deposit(pos, N, L)
    s = R.Solver(N, L)
    rho = s.deposit_cic(dev(pos))
    got = host(rho)
    assert np.max(np.abs(got - ref)) < 1e-12 * ref.max()
    assert abs(got.sum() - N ** 3) < 1e-8
    # particles at the edges of the box and of cells (N/L a power of two takes
    # the fixed-point coordinate): x = 0, tiny, half a cell, just below a
    # cell centre, L - ulp, L, and slightly negative (the FP64 form)
    h = L / N
    edge = np.array([0.0, 1e-300, 1e-17, 0.5 * h, 0.5 * h - 1e-13, h, 3.5 * h,
                     np.nextafter(L, 0.0), L, -1e-12, -0.3 * h])
    pe = np.stack(np.meshgrid(edge, edge[:4], edge[4:8], indexing="ij"), -1).reshape(-1, 3)
    ref_e = O.cic_deposit(pe, N, L, mass=1.0)
    got_e = host(s.deposit_cic(dev(pe), mass=1.0))
    assert np.max(np.abs(got_e - ref_e)) < 1e-12 * max(ref_e.max(), 1.0)
    # empty input deposits nothing
    empty = s.deposit_cic(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert host(empty).sum() == 0.0
    s.close()


# ------------------------------------------------------------------ solves
def test_solve_delta_zero_is_exactly_zero(R):
    N, L = 16, 64.0
    s = R.Solver(N, L)
    phi, st = s.solve(torch.ones((N,) * 3, dtype=torch.float64, device="cuda"), tol=1e-10)
    assert torch.count_nonzero(phi).item() == 0 and st["compat_c"] == 0.0
    s.close()


@pytest.mark.parametrize("N,L,sig,Rs", [(32, 100.0, 0.5, 5.0), (48, 48.0, 1.0, 2.0),
                                        (128, 256.0, 0.8, 4.0)])
def test_solve_f64_parity(R, O, N, L, sig, Rs):
    b, _, _ = zeldovich_density(O, N, L, sig, Rs, 1000 + N)
    ref, info = O.solve(b, L, tol=1e-10, max_cycles=40)
    assert info["status"] == 0
    s = R.Solver(N, L)
    phi, st = s.solve(dev(b), tol=1e-10, max_cycles=40)
    got = host(phi)
    assert rel_l2(got, ref) < 1e-10
    assert abs(st["cycles"] - info["cycles"]) <= 1
    assert st["compat_c"] == pytest.approx(info["c"], rel=1e-6, abs=1e-13)
    np.testing.assert_allclose(st["history"][:3], info["history"][:3], rtol=1e-6)
    s.close()


@pytest.mark.parametrize("N,L,sig,Rs,dfres", [(32, 100.0, 0.5, 5.0, 1), (64, 64.0, 1.0, 2.0, 1),
                                              (128, 256.0, 0.8, 4.0, 1), (64, 64.0, 1.0, 2.0, 0)])
def test_solve_mixed_parity(R, O, N, L, sig, Rs, dfres):
    """N = 128 runs the fused FP32 FAS and linear smoothers; dfres selects the
    double-float (1) or FP64 (0) fine-grid residual."""
    b, _, _ = zeldovich_density(O, N, L, sig, Rs, 2000 + N)
    ref, info = O.solve(b, L, tol=1e-10, max_cycles=40)
    s = R.Solver(N, L, R.RECON_MIXED, mixed_df_residual=dfres)
    phi, st = s.solve(dev(b), tol=1e-10, max_cycles=30)
    assert st["rel_residual"] < 1e-10
    assert rel_l2(host(phi), ref) < 1e-6
    s.close()


def test_solve_exact_rule_and_resume(R, O):
    N, L = 32, 64.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 31)
    ref, _ = O.solve(b, L, tol=1e-11, rule="exact")
    s = R.Solver(N, L, rule=R.RULE_EXACT)
    phi, st = s.solve(dev(b), tol=1e-11)
    assert rel_l2(host(phi), ref) < 1e-9
    # resume from the answer: one cycle suffices
    s.configure(start=R.START_GUESS)
    phi2, st2 = s.solve(dev(b), phi=phi.clone(), tol=1e-10)
    assert st2["cycles"] == 1
    s.close()


def test_solve_domain_and_limits(R):
    N, L = 16, 16.0
    s = R.Solver(N, L)
    b = torch.ones((N,) * 3, dtype=torch.float64, device="cuda")
    b[3, 4, 5] = 0.0
    with pytest.raises(R.ReconError) as e:
        s.solve(b)
    assert e.value.status == 2
    b[3, 4, 5] = float("nan")
    with pytest.raises(R.ReconError) as e:
        s.solve(b)
    assert e.value.status == 2
    b[3, 4, 5] = 1.5
    status, st = R.recon_solve(s.h, N, b, torch.zeros_like(b), 1e-14, 1, raise_on_noconv=False)
    assert status == 3 and st["cycles"] == 1
    s.close()


# ------------------------------------------------------------------ output
@pytest.mark.parametrize("N,L,sig,Rs,seed", [(32, 64.0, 0.8, 4.0, 41), (64, 64.0, 1.0, 2.0, 3000),
                                              (32, 100.0, 0.8, 5.0, 42)])
def test_displace_parity(R, O, N, L, sig, Rs, seed):
    """64^3 at sigma 1, R = 2 h^-1 Mpc: the bench recipe's resolution, with
    cells down to b ~ 0.14 where v = 3 - tr((I+H)^-1) is most sensitive.
    h = 2 and 1 scale psi by moving the exponent; h = 100/32 multiplies."""
    b, _, _ = zeldovich_density(O, N, L, sig, Rs, seed)
    t, _ = O.solve(b, L, tol=1e-11, max_cycles=40)
    psi_ref, dl_ref = O.displace(t, b, L)
    s = R.Solver(N, L)
    psi, dl = s.displace(dev(t), dev(b))
    assert np.max(np.abs(host(psi) - psi_ref)) < 1e-13 * np.abs(psi_ref).max()
    # v = 3 - tr((I+H)^-1) and the (b v, b) accumulation are FP32 on the GPU:
    # |delta_r| < 3 with ~8 contributions per cell gives ~1e-6 absolute
    assert np.max(np.abs(host(dl) - dl_ref)) < 1e-5
    assert host(dl).max() < 3.0
    s.close()


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("N,L", [(6, 12.0), (4, 8.0), (96, 192.0)])
def test_solve_single_level_and_odd_hierarchies(R, O, N, L):
    """N = 4, 6: one level (the coarsest solve is the whole solve); 96: ends at 6^3."""
    b, _, _ = zeldovich_density(O, N, L, 0.5, 2.0 * L / N, 60 + N)
    ref, info = O.solve(b, L, tol=1e-10, max_cycles=60)
    for dt in (R.RECON_F64, R.RECON_MIXED):
        s = R.Solver(N, L, dt)
        phi, st = s.solve(dev(b), tol=1e-10, max_cycles=60)
        assert rel_l2(host(phi), ref) < (1e-10 if dt == R.RECON_F64 else 1e-6)
        s.close()


def test_mixed_resume_and_noconv(R, O):
    N, L = 32, 64.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 71)
    s = R.Solver(N, L, R.RECON_MIXED)
    phi, st = s.solve(dev(b), tol=1e-10)
    s.configure(start=R.START_GUESS, mixed_fas_max_cycles=0)
    phi2, st2 = s.solve(dev(b), phi=phi.clone(), tol=1e-9)
    assert st2["outer_iterations"] == 1 and st2["rel_residual"] < 1e-9
    status, st3 = R.recon_solve(s.h, N, dev(b), torch.zeros_like(phi), 1e-15, 1,
                                raise_on_noconv=False)
    assert status == 3 and st3["outer_iterations"] == 1
    s.close()


def test_launch_counter_counts_our_kernels(R):
    before = R.recon_kernel_launches()
    s = R.Solver(16, 16.0)
    s.solve(torch.ones((16,) * 3, dtype=torch.float64, device="cuda") * 1.0, tol=1e-8)
    assert R.recon_kernel_launches() > before
    s.close()


def test_page_locked_host_buffers(R, O):
    """Positions read from page-locked host memory and delta_r written into it
    give the device results; pageable host memory is refused, not read."""
    import ctypes
    from paper_1709_06350_gb300 import synth
    N, L = 32, 64.0
    _, dh = synth.linear_field(N, L, 0.8, 91)
    pos = synth.zeldovich_positions(dh, N, L)
    s = R.Solver(N, L)
    rho_dev = s.deposit_cic(dev(pos))
    pos_pinned = torch.from_numpy(pos).pin_memory()
    rho_host_read = s.deposit_cic(pos_pinned)
    assert np.max(np.abs(host(rho_host_read) - host(rho_dev))) < 1e-12 * host(rho_dev).max()
    with pytest.raises(TypeError):
        s.deposit_cic(torch.from_numpy(pos))            # pageable: refused by the binding
    rho = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    st = R.load().recon_deposit_cic(s.h, ctypes.c_void_p(pos.ctypes.data), pos.shape[0], 1.0,
                                    ctypes.c_void_p(rho.data_ptr()))
    assert st == 1                                        # RECON_E_INVALID from the C ABI
    assert host(rho).sum() == 0.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 92)
    t, _ = O.solve(b, L, tol=1e-10)
    psi_d, dl_d = s.displace(dev(t), dev(b))
    dl_h = torch.empty((N,) * 3, dtype=torch.float64).pin_memory()
    psi_h = torch.empty((3,) + (N,) * 3, dtype=torch.float64).pin_memory()
    s.displace(dev(t), dev(b), psi=psi_h, dl=dl_h)
    torch.cuda.synchronize()
    assert np.max(np.abs(psi_h.numpy() - host(psi_d))) == 0.0
    assert np.max(np.abs(dl_h.numpy() - host(dl_d))) < 1e-6
    s.close()


# ------------------------------------------------------------------ NGP / TSC
@pytest.mark.parametrize("scheme", ["ngp", "cic", "tsc"])
def test_assignment_parity(R, O, scheme):
    """NGP cells (and so the NGP density, a sum of equal masses) are
    bit-exact; CIC and TSC densities agree with the oracle to 1e-12.
    Includes particles on the seam, just below 0 and far outside [0, L)."""
    from paper_1709_06350_gb300 import synth
    N, L = 32, 100.0
    _, dh = synth.linear_field(N, L, 1.0, 81)
    pos = synth.zeldovich_positions(dh, N, L)
    edge = np.array([[0.0, L - 1e-13, 50.0], [L / N * 3, L / N * 0.5, 99.999999999],
                     [-1e-13, -0.4, L + 0.3], [-2.5 * L, 3.7 * L, 1e9]])
    pos = np.concatenate([pos, edge])
    ref = O.assign_deposit(pos, N, L, scheme)
    s = R.Solver(N, L)
    got = host(s.deposit(dev(pos), scheme))
    if scheme == "ngp":
        assert np.array_equal(got, ref)
    else:
        assert np.max(np.abs(got - ref)) < 1e-12 * ref.max()
    assert abs(got.sum() - N ** 3) < 1e-8
    s.close()


def test_convergence_with_tracer_and_mesh_ratios(R):
    """Sec. I: 8 N^3 particles on an N^3 mesh, or N^3 particles on an (2N)^3
    mesh, converge at a rate similar to N^3 on N^3, for NGP, CIC and TSC
    (mixed solves to 1e-8: FP32 cycles plus corrections within two)."""
    from paper_1709_06350_gb300 import synth
    N, L, Rs = 64, 128.0, 4.0
    counts = {}
    for label, n_lat, n_mesh in (("N3 on N3", N, N), ("8N3 on N3", 2 * N, N), ("N3 on 8N3", N, 2 * N)):
        _, dh = synth.linear_field(n_lat, L, 0.8, 32)
        pos = torch.from_numpy(synth.zeldovich_positions(dh, n_lat, L)).cuda()
        s = R.Solver(n_mesh, L, R.RECON_MIXED)
        for scheme in ("ngp", "cic", "tsc"):
            b = s.smooth_density(s.deposit(pos, scheme), Rs)
            _, st = s.solve(b, tol=1e-8, max_cycles=40)
            assert st["rel_residual"] < 1e-8
            counts[(label, scheme)] = st["cycles"] + st["outer_iterations"]
        s.close()
    assert max(counts.values()) - min(counts.values()) <= 2, counts


# ------------------------------------------------------------------ density preparation
@pytest.mark.parametrize("N,L,Rs,seed", [(32, 100.0, 5.0, 1000), (64, 64.0, 2.0, 3000), (48, 96.0, 4.0, 2001),
                                         (8, 8.0, 3.0, 7)])
def test_smooth_density_parity(R, O, N, L, Rs, seed):
    """recon_smooth_density against the oracle's FFT definition on a seeded
    Zel'dovich density (oracle CIC).  The GPU applies the window as three
    FP32 circular convolutions of half-width T <= 13 here; with positive taps
    summing to 1, each pass adds at most (2T + 1) 2^-24 relative rounding and
    the truncation at 1e-9 of the centre tap is negligible, so three passes
    stay within 3 x 27 x 6e-8 ~ 5e-6 of max(b).  (8, 8.0, 3.0): a window
    wider than the box, where the kernel covers the whole periodic line."""
    from paper_1709_06350_gb300 import synth
    _, dh = synth.linear_field(N, L, 0.8, seed)
    rho = O.cic_deposit(synth.zeldovich_positions(dh, N, L), N, L)
    ref = O.smooth_and_floor(rho, L, Rs)
    s = R.Solver(N, L)
    got = s.smooth_density(dev(rho), Rs)
    assert np.max(np.abs(host(got) - ref)) < 5e-6 * ref.max()
    assert host(got).mean() == pytest.approx(1.0, abs=1e-12)
    # in place, and no smoothing (floor and mean only)
    x = dev(rho)
    s.smooth_density(x, 0.0, out=x)
    ref0 = O.smooth_and_floor(rho, L, 0.0)
    assert np.max(np.abs(host(x) - ref0)) < 1e-7 * ref0.max()
    s.close()


def test_smooth_density_narrow_window_and_bad_arguments(R, O):
    """R = 1 cell: the window is 7e-3 at the Nyquist frequency, so the exact
    periodic kernel spans the whole line (129 taps at N = 128, FP32 sums:
    tolerance 129 x 2^-24 x 3 passes ~ 3e-5); bad arguments are refused."""
    from paper_1709_06350_gb300 import synth
    N, L = 128, 256.0
    _, dh = synth.linear_field(N, L, 0.8, 2002)
    rho = O.cic_deposit(synth.zeldovich_positions(dh, N, L), N, L)
    ref = O.smooth_and_floor(rho, L, 2.0)
    s = R.Solver(N, L)
    got = host(s.smooth_density(dev(rho), 2.0))
    assert np.max(np.abs(got - ref)) < 3e-5 * ref.max()
    x = dev(rho)
    with pytest.raises(R.ReconError, match="RECON_E_INVALID"):
        s.smooth_density(x, -1.0)
    with pytest.raises(R.ReconError, match="RECON_E_INVALID"):
        s.smooth_density(x, 2.0, floor=0.0)
    s.close()


# ------------------------------------------------------------------ cubic test
def test_cubic_test(R, O):
    """Sec. III.A cubic test at 64^3 (a cube of side 5 in a box of 64, the
    paper's 10/128): after exactly 12 FAS cycles the FP64 GPU iterate equals
    the oracle's; the mixed solve to 1e-3 has the interior closed form
    lap(theta) = 3 (b_in^(1/3) - 1), Hbar = 0."""
    from paper_1709_06350_gb300 import synth
    N, L, l = 64, 64.0, 5.0
    b = O.smooth_and_floor(O.cic_deposit(synth.cube_positions(N, L, l), N, L), L, 0.0)
    ref, info = O.solve(b, L, tol=1e-14, max_cycles=12)
    s = R.Solver(N, L)
    phi, st = s.solve(dev(b), tol=1e-14, max_cycles=12, raise_on_noconv=False)
    assert st["cycles"] == info["cycles"] == 12
    assert rel_l2(host(phi), ref) < 1e-9
    s.close()
    m = R.Solver(N, L, R.RECON_MIXED)
    phim, stm = m.solve(dev(b), tol=1e-3, max_cycles=80)
    assert stm["rel_residual"] < 1e-3
    t = host(phim)
    c = N // 2
    H = [np.roll(t, -1, a) + np.roll(t, 1, a) - 2 * t for a in range(3)]
    lap = sum(H)[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1]
    expect = 3.0 * (b[c, c, c] ** (1.0 / 3.0) - 1.0)
    assert np.all(np.abs(lap / expect - 1.0) < 1e-3)
    for a in range(3):
        assert np.max(np.abs(H[a][c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] - lap / 3.0)) < 1e-3 * expect
    m.close()


# ------------------------------------------------------------------ Gaussianisation
@pytest.mark.parametrize("N", [16, 48, 64])
def test_gaussianise_parity(R, O, N):
    """The GPU radix sort's ranks equal a stable sort's (ties and both zero
    signs included): the output orders exactly like the oracle's; values
    agree to FP64 quantile rounding (CUDA's normcdfinv against scipy's ndtri,
    both near FP64 precision); a second call gives the same result."""
    rng = np.random.default_rng(N)
    v = np.round(rng.gamma(2.0, 1.0, (N,) * 3) * 64) / 64 - 2.0
    v.ravel()[:3] = [0.0, -0.0, 0.0]
    g_ref, _ = O.gaussianise(v)
    s = R.Solver(N, float(N))
    g = host(s.gaussianise(dev(v)))
    assert np.max(np.abs(g - g_ref)) < 1e-11 * v.std()
    assert np.array_equal(np.argsort(g, axis=None, kind="stable"),
                          np.argsort(g_ref, axis=None, kind="stable"))
    assert np.array_equal(host(s.gaussianise(dev(v))), g)
    s.close()


def test_gaussianise_keeps_strict_order_above_2_24_cells(R, O):
    """320^3 = 32.8 M cells > 2^24: adjacent ranks' probabilities differ by
    less than an FP32 spacing near 1/2, so only an FP64 probability keeps
    distinct inputs distinct; the output is strictly increasing along the
    input's order and equals the oracle's to FP64 rounding."""
    N = 320
    v = np.random.default_rng(320).standard_normal((N,) * 3)
    s = R.Solver(N, float(N))
    g = host(s.gaussianise(dev(v)))
    s.close()
    order = np.argsort(v, axis=None, kind="stable")
    assert np.all(np.diff(g.ravel()[order]) > 0)
    g_ref, _ = O.gaussianise(v)
    # the extreme ranks sit at |g| ~ 5.6 (p ~ 1.5e-8), where CUDA's
    # normcdfinv and scipy's ndtri differ by a few 1e-10
    assert np.max(np.abs(g - g_ref)) < 1e-9 * v.std()


@pytest.mark.parametrize("dtype", ["f64", "mixed"])
def test_paper_eps_matches_oracle(R, O, dtype):
    """recon_stats.paper_eps (Sec. II.A.2's convergence measure, on request)
    equals the oracle's epsilon of the same phi, b and c; NaN when not asked."""
    N, L = 32, 100.0
    b, _, _ = zeldovich_density(O, N, L, 0.5, 5.0, 1032)
    s = R.Solver(N, L, R.RECON_F64 if dtype == "f64" else R.RECON_MIXED)
    _, st0 = s.solve(dev(b), tol=1e-10, max_cycles=40)
    assert np.isnan(st0["paper_eps"])
    s.configure(report_paper_eps=1)
    phi, st = s.solve(dev(b), tol=1e-10, max_cycles=40)
    want = O.paper_eps(host(phi), b, st["compat_c"], L / N)
    # L_h = (s - 3) - (root - 3) is a difference of O(1) numbers: rounding
    # moves each cell's value by ~1e-15, against epsilon ~1e-11 here
    assert st["paper_eps"] == pytest.approx(want, rel=1e-3, abs=1e-14)
    assert 0.0 < st["paper_eps"] < 1e-8
    s.close()


def test_level_scales(R, O):
    """recon_level_scales: one factor per coarse level; a mild field never
    scales the coarse right side (s = 1), the cubic test's first cycle does
    (the oracle's V-cycle on the same 64^3 problem gives s ~ 0.5-0.9 on the
    finest coarse level in its first cycles)."""
    from paper_1709_06350_gb300 import synth
    N, L = 32, 64.0
    b = smooth_density(N, 90, 0.3)
    s = R.Solver(N, L)
    s.solve(dev(b), tol=1e-10, max_cycles=30)
    sc = s.level_scales()
    assert len(sc) == O.num_levels(N) - 1 and all(x == 1.0 for x in sc)
    s.close()
    N, Lb = 64, 64.0
    s = R.Solver(N, Lb)
    rho = s.deposit_cic(dev(synth.cube_positions(N, Lb, Lb * 10 / 128)))
    bc = s.smooth_density(rho, 0.0)
    s.solve(bc, tol=1e-30, max_cycles=1, raise_on_noconv=False)
    sc = s.level_scales()
    assert len(sc) == O.num_levels(N) - 1
    assert 0.0 <= min(sc) < 1.0 and max(sc) <= 1.0
    s.close()
