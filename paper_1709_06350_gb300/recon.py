"""Thin Python binding of librecon (include/recon.h, include/recon_steps.h).

Argument marshalling only: every function forwards device pointers of torch
CUDA tensors to the C ABI and raises ``ReconError`` on a non-OK status.  No
computation happens here, and there is no CPU fallback: without a built
``librecon.so`` (``paper_1709_06350_gb300.build.build()``) every call raises.

The function names follow the C ABI (``recon_create`` ...); ``Solver`` wraps a
handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librecon.so")

RECON_F64, RECON_MIXED = 0, 1
RULE_NEWTON1, RULE_EXACT = 0, 1
START_FMG, START_GUESS = 0, 1
STATUS = {0: "RECON_OK", 1: "RECON_E_INVALID", 2: "RECON_E_DOMAIN", 3: "RECON_E_NOCONV",
          4: "RECON_E_DIVERGED", 5: "RECON_E_CUDA", 6: "RECON_E_OOM", 7: "RECON_E_TIMEOUT",
          8: "RECON_E_UNIMPLEMENTED"}
HISTORY_MAX = 64

_lock = threading.Lock()
_lib = None


class ReconError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class recon_config(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("coarse_max_sweeps", ctypes.c_int), ("coarse_rtol", ctypes.c_double),
                ("rule", ctypes.c_int), ("start", ctypes.c_int),
                ("scale_floor", ctypes.c_double), ("mixed_switch_rtol", ctypes.c_double),
                ("mixed_fas_max_cycles", ctypes.c_int), ("mixed_linear_vcycles", ctypes.c_int),
                ("mixed_df_residual", ctypes.c_int), ("fused_chunk", ctypes.c_int),
                ("adjoint_store_cofactors", ctypes.c_int), ("report_paper_eps", ctypes.c_int)]


class recon_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("compat_c", ctypes.c_double),
                ("paper_eps", ctypes.c_double),
                ("seconds", ctypes.c_double), ("n_history", ctypes.c_int),
                ("history", ctypes.c_double * HISTORY_MAX)]

    def as_dict(self):
        return dict(cycles=self.cycles, outer_iterations=self.outer_iterations,
                    rel_residual=self.rel_residual, compat_c=self.compat_c, paper_eps=self.paper_eps,
                    seconds=self.seconds, history=list(self.history[:self.n_history]))


class recon_slab(ctypes.Structure):
    """A slab of planes of a periodic N^3 grid (include/recon_slab.h)."""
    _fields_ = [("N", ctypes.c_int), ("planes", ctypes.c_int), ("first", ctypes.c_int),
                ("lo", ctypes.c_int), ("hi", ctypes.c_int)]


_P, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_SP = ctypes.POINTER(recon_slab)
_SIGS = {
    "recon_create": (_I, [_I, _D, _I, ctypes.POINTER(_P)]),
    "recon_destroy": (None, [_P]),
    "recon_workspace_bytes": (ctypes.c_size_t, [_I, _I]),
    "recon_set_stream": (_I, [_P, _P]),
    "recon_get_config": (_I, [_P, ctypes.POINTER(recon_config)]),
    "recon_set_config": (_I, [_P, ctypes.POINTER(recon_config)]),
    "recon_deposit_cic": (_I, [_P, _P, _LL, _D, _P]),
    "recon_deposit": (_I, [_P, _I, _P, _LL, _D, _P]),
    "recon_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(recon_stats)]),
    "recon_displace": (_I, [_P, _P, _P, _P, _P]),
    "recon_adjoint": (_I, [_P, _P, _P]),
    "recon_displace_fp64": (_I, [_P, _P, _P, _P, _P]),
    "recon_displace_adjoint": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "recon_gaussianise": (_I, [_P, _P, _P]),
    "recon_level_scales": (_I, [_P, _P, _I, ctypes.POINTER(_I)]),
    "recon_smooth_density": (_I, [_P, _P, _D, _D, _P]),
    "recon_last_error": (ctypes.c_char_p, [_P]),
    "recon_status_string": (ctypes.c_char_p, [_I]),
    "recon_kernel_launches": (ctypes.c_ulonglong, []),
    "recon_batch_create": (_I, [_I, _P, _P, ctypes.POINTER(_P)]),
    "recon_batch_destroy": (None, [_P]),
    "recon_batch_set_stream": (_I, [_P, _P]),
    "recon_batch_handle": (_P, [_P, _I]),
    "recon_batch_solve": (_I, [_P, _P, _P, _D, _I, _P]),
    "recon_batch_last_error": (ctypes.c_char_p, [_P]),
    "recon_step_sweep": (_I, [_I, _D, _I, _I, _P, _P, _D, _I, _P, _P]),
    "recon_step_residual": (_I, [_I, _D, _P, _P, _D, _P, _P]),
    "recon_step_det": (_I, [_I, _D, _P, _P, _P]),
    "recon_step_restrict": (_I, [_I, _I, _P, _P, _P]),
    "recon_step_prolong_add": (_I, [_I, _I, _P, _P, _D, _P, _P]),
    "recon_step_coarse_solve": (_I, [_I, _D, _I, _I, _P, _P, _D, _I, _D, _P, _P, _P]),
    "recon_step_coarse_solve_noalloc": (_I, [_I, _D, _I, _I, _P, _P, _D, _I, _D, _P, _P]),
    "recon_step_cic_cells": (_I, [_P, _LL, _I, _D, _P, _P, _P]),
    "recon_step_jacobian_apply": (_I, [_I, _D, _P, _P, _P, _P]),
    "recon_step_linear_sweep": (_I, [_I, _D, _P, _P, _P, _I, _P, _P]),
    "recon_measure_fp64_fma": (_I, [_I, _I, _P, _P]),
    "recon_slab_sweep": (_I, [_SP, _D, _I, _P, _P, _D, _P, _P]),
    "recon_slab_residual": (_I, [_SP, _D, _P, _P, _D, _P, _P]),
    "recon_slab_det": (_I, [_SP, _D, _P, _P, _P]),
    "recon_slab_restrict": (_I, [_SP, _P, _SP, _P, _P]),
    "recon_slab_prolong_add": (_I, [_SP, _P, _P, _D, _SP, _P, _P]),
    "recon_slab_plane_sums": (_I, [_SP, _P, _D, _I, _P, _P]),
    "recon_slab_eps_planes": (_I, [_SP, _D, _P, _P, _D, _P, _P]),
    "recon_slab_defect_min": (_I, [_SP, _P, _P, _D, _P, _P]),
    "recon_slab_form_rhs": (_I, [_SP, _P, _P, _D, _P, _P]),
    "recon_slab_sub": (_I, [_SP, _P, _D, _P]),
}
EXPORTS = tuple(_SIGS)


def load():
    """Load librecon.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1709_06350_gb300.build.build() (no CPU fallback exists)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ---------------------------------------------------------------- marshalling
def _dev_ptr(t, dtype=None, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _reachable_ptr(t, dtype=None, numel=None):
    """A CUDA tensor, or a CPU tensor in page-locked memory (kernels read or
    write it over the host link); pageable CPU tensors are refused."""
    import torch
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned():
            raise TypeError("expected a CUDA tensor or a pinned (page-locked) CPU tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"expected {numel} elements, got {t.numel()}")
        return ctypes.c_void_p(t.data_ptr())
    return _dev_ptr(t, dtype, numel)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, handle=None):
    if status != 0:
        msg = load().recon_last_error(handle)
        raise ReconError(status, (msg or b"").decode())


# ---------------------------------------------------------------- C ABI, 1:1
def recon_create(N: int, L: float, dtype: int = RECON_F64):
    h = ctypes.c_void_p()
    _check(load().recon_create(int(N), float(L), int(dtype), ctypes.byref(h)), None)
    return h


def recon_destroy(h) -> None:
    load().recon_destroy(h)


def recon_workspace_bytes(N: int, dtype: int = RECON_F64) -> int:
    return int(load().recon_workspace_bytes(int(N), int(dtype)))


def recon_set_stream(h, stream=None) -> None:
    _check(load().recon_set_stream(h, _stream(stream)), h)


def recon_get_config(h) -> recon_config:
    c = recon_config()
    _check(load().recon_get_config(h, ctypes.byref(c)), h)
    return c


def recon_set_config(h, cfg: recon_config) -> None:
    _check(load().recon_set_config(h, ctypes.byref(cfg)), h)


def recon_deposit_cic(h, N: int, pos, mass: float, rho) -> None:
    import torch
    n = pos.numel() // 3
    _check(load().recon_deposit_cic(h, _reachable_ptr(pos, torch.float64) if n else None, n,
                                    float(mass), _dev_ptr(rho, torch.float64, N ** 3)), h)


ASSIGN = {"ngp": 0, "cic": 1, "tsc": 2}


def recon_deposit(h, N: int, scheme, pos, mass: float, rho) -> None:
    import torch
    n = pos.numel() // 3
    sc = ASSIGN[scheme] if isinstance(scheme, str) else int(scheme)
    _check(load().recon_deposit(h, sc, _reachable_ptr(pos, torch.float64) if n else None, n,
                                float(mass), _dev_ptr(rho, torch.float64, N ** 3)), h)


def recon_solve(h, N: int, b, phi, tol: float, max_cycles: int, raise_on_noconv=True):
    import torch
    st = recon_stats()
    status = load().recon_solve(h, _dev_ptr(b, torch.float64, N ** 3),
                                _dev_ptr(phi, torch.float64, N ** 3), float(tol),
                                int(max_cycles), ctypes.byref(st))
    if status == 3 and not raise_on_noconv:
        return status, st.as_dict()
    _check(status, h)
    return status, st.as_dict()


def recon_displace(h, N: int, phi, b, psi, deltaL) -> None:
    import torch
    _check(load().recon_displace(h, _dev_ptr(phi, torch.float64, N ** 3),
                                 _dev_ptr(b, torch.float64, N ** 3),
                                 _reachable_ptr(psi, torch.float64, 3 * N ** 3),
                                 _reachable_ptr(deltaL, torch.float64, N ** 3)), h)


def recon_displace_fp64(h, N: int, phi, b, psi, deltaL) -> None:
    import torch
    _check(load().recon_displace_fp64(h, _dev_ptr(phi, torch.float64, N ** 3),
                                      _dev_ptr(b, torch.float64, N ** 3),
                                      _reachable_ptr(psi, torch.float64, 3 * N ** 3),
                                      _reachable_ptr(deltaL, torch.float64, N ** 3)), h)


def recon_displace_adjoint(h, N: int, phi, b, gbar_psi, gbar_deltaL, gbar_phi, gbar_b) -> None:
    """gbar_psi / gbar_deltaL: CUDA tensors or None (zero)."""
    import torch
    gp = None if gbar_psi is None else _dev_ptr(gbar_psi, torch.float64, 3 * N ** 3)
    gd = None if gbar_deltaL is None else _dev_ptr(gbar_deltaL, torch.float64, N ** 3)
    _check(load().recon_displace_adjoint(h, _dev_ptr(phi, torch.float64, N ** 3),
                                         _dev_ptr(b, torch.float64, N ** 3), gp, gd,
                                         _dev_ptr(gbar_phi, torch.float64, N ** 3),
                                         _dev_ptr(gbar_b, torch.float64, N ** 3)), h)


def recon_smooth_density(h, N: int, rho, R: float, floor: float, b) -> None:
    import torch
    _check(load().recon_smooth_density(h, _dev_ptr(rho, torch.float64, N ** 3), float(R), float(floor),
                                       _dev_ptr(b, torch.float64, N ** 3)), h)


def recon_level_scales(h, n: int = 16) -> list:
    """The scaled-defect factor of each coarse level in the handle's last FAS
    V-cycle (level 1 first)."""
    out = (ctypes.c_double * max(n, 1))()
    levels = ctypes.c_int(0)
    _check(load().recon_level_scales(h, out, int(n), ctypes.byref(levels)), h)
    return [out[i] for i in range(min(n, levels.value))]


def recon_gaussianise(h, N: int, field, out) -> None:
    import torch
    _check(load().recon_gaussianise(h, _dev_ptr(field, torch.float64, N ** 3),
                                    _dev_ptr(out, torch.float64, N ** 3)), h)


def recon_adjoint(h, N: int, gbar_phi, gbar_b) -> None:
    import torch
    _check(load().recon_adjoint(h, _dev_ptr(gbar_phi, torch.float64, N ** 3),
                                _dev_ptr(gbar_b, torch.float64, N ** 3)), h)


def recon_kernel_launches() -> int:
    return int(load().recon_kernel_launches())


# ---------------------------------------------------------------- steps
def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return 0
    if t.dtype == torch.float32:
        return 1
    raise TypeError("grids must be float64 or float32")


def recon_step_sweep(theta, g, c, h, sweeps=1, rule=RULE_NEWTON1, work=None, stream=None):
    import torch
    N = theta.shape[0]
    work = torch.empty_like(theta) if work is None else work
    _check(load().recon_step_sweep(N, float(h), _prec(theta), int(rule), _dev_ptr(theta, theta.dtype),
                                   _dev_ptr(g, theta.dtype, theta.numel()), float(c), int(sweeps),
                                   _dev_ptr(work, theta.dtype, theta.numel()), _stream(stream)))


def recon_step_residual(theta, g, c, h, r, stream=None):
    import torch
    N = theta.shape[0]
    _check(load().recon_step_residual(N, float(h), _dev_ptr(theta, torch.float64),
                                      _dev_ptr(g, torch.float64, N ** 3), float(c),
                                      _dev_ptr(r, torch.float64, N ** 3), _stream(stream)))


def recon_step_det(theta, h, out, stream=None):
    import torch
    N = theta.shape[0]
    _check(load().recon_step_det(N, float(h), _dev_ptr(theta, torch.float64),
                                 _dev_ptr(out, torch.float64, N ** 3), _stream(stream)))


def recon_step_restrict(fine, coarse, stream=None):
    Nf = fine.shape[0]
    _check(load().recon_step_restrict(Nf, _prec(fine), _dev_ptr(fine, fine.dtype),
                                      _dev_ptr(coarse, fine.dtype, (Nf // 2) ** 3), _stream(stream)))


def recon_step_prolong_add(cnew, cold, fine, scale=1.0, stream=None):
    Nc = cnew.shape[0]
    _check(load().recon_step_prolong_add(
        Nc, _prec(cnew), _dev_ptr(cnew, cnew.dtype),
        _dev_ptr(cold, cnew.dtype, Nc ** 3) if cold is not None else None, float(scale),
        _dev_ptr(fine, cnew.dtype, 8 * Nc ** 3), _stream(stream)))


def recon_step_coarse_solve(theta, g, c, h, max_sweeps=200, rtol=1e-3, rule=RULE_NEWTON1,
                            stream=None):
    """Returns the number of sweeps done (synchronises to read it)."""
    import torch
    N = theta.shape[0]
    work = torch.empty_like(theta)
    done = torch.zeros(1, dtype=torch.int32, device=theta.device)
    _check(load().recon_step_coarse_solve(N, float(h), _prec(theta), int(rule),
                                          _dev_ptr(theta, theta.dtype),
                                          _dev_ptr(g, theta.dtype, N ** 3), float(c),
                                          int(max_sweeps), float(rtol),
                                          _dev_ptr(work, theta.dtype, N ** 3),
                                          _dev_ptr(done, torch.int32), _stream(stream)))
    return int(done.item())


def recon_step_coarse_solve_noalloc(theta, g, c, h, max_sweeps=200, rtol=1e-3,
                                    rule=RULE_NEWTON1, sweeps_done=None, stream=None):
    """Coarsest-grid solve without any device allocation by the library.

    For callers that cannot allocate device memory when they run this step;
    the scratch is a fixed 32 KiB array inside librecon (N^3 <= 4096).
    ``sweeps_done`` is an optional caller-owned device int32 tensor.
    """
    import torch
    N = theta.shape[0]
    _check(load().recon_step_coarse_solve_noalloc(
        N, float(h), _prec(theta), int(rule), _dev_ptr(theta, theta.dtype),
        _dev_ptr(g, theta.dtype, N ** 3), float(c), int(max_sweeps), float(rtol),
        _dev_ptr(sweeps_done, torch.int32) if sweeps_done is not None else None,
        _stream(stream)))


def recon_step_cic_cells(pos, N, L, cells, frac, stream=None):
    import torch
    n = pos.numel() // 3
    _check(load().recon_step_cic_cells(_dev_ptr(pos, torch.float64), n, int(N), float(L),
                                       _dev_ptr(cells, torch.int32, 3 * n),
                                       _dev_ptr(frac, torch.float64, 3 * n), _stream(stream)))


def recon_step_linear_sweep(e, f, theta, h, sweeps=1, work=None, stream=None):
    """work: 7 N^3 floats (ping-pong grid + six cofactor arrays)."""
    import torch
    N = e.shape[0]
    work = torch.empty(7 * N ** 3, dtype=torch.float32, device=e.device) if work is None else work
    _check(load().recon_step_linear_sweep(N, float(h), _dev_ptr(e, torch.float32),
                                          _dev_ptr(f, torch.float32, N ** 3),
                                          _dev_ptr(theta, torch.float32, N ** 3), int(sweeps),
                                          _dev_ptr(work, torch.float32, 7 * N ** 3), _stream(stream)))


def recon_measure_fp64_fma(blocks: int, iters: int, out, stream=None) -> None:
    """FP64 FMA rate probe: 4096 * blocks * iters flops (time it with events)."""
    import torch
    _check(load().recon_measure_fp64_fma(int(blocks), int(iters), _dev_ptr(out, torch.float64),
                                         _stream(stream)))


def recon_step_jacobian_apply(theta, v, h, out, stream=None):
    import torch
    N = theta.shape[0]
    _check(load().recon_step_jacobian_apply(N, float(h), _dev_ptr(theta, torch.float64),
                                            _dev_ptr(v, torch.float64, N ** 3),
                                            _dev_ptr(out, torch.float64, N ** 3),
                                            _stream(stream)))


# ---------------------------------------------------------------- convenience
class Solver:
    """One librecon handle (N^3 grid of side L, FP64 or MIXED)."""

    def __init__(self, N: int, L: float, dtype: int = RECON_F64, stream=None, **config):
        self.N, self.L, self.dtype = int(N), float(L), int(dtype)
        self.h = recon_create(self.N, self.L, self.dtype)
        recon_set_stream(self.h, stream)
        if config:
            self.configure(**config)

    def configure(self, **kw):
        c = recon_get_config(self.h)
        for k, v in kw.items():
            if not hasattr(c, k):
                raise KeyError(k)
            setattr(c, k, v)
        recon_set_config(self.h, c)
        return self

    def config(self) -> dict:
        c = recon_get_config(self.h)
        return {name: getattr(c, name) for name, _ in c._fields_}

    def deposit_cic(self, pos, mass=None, rho=None):
        """pos: CUDA tensor or pinned CPU tensor (read by the kernel over the
        host link); rho: CUDA tensor, accumulated into."""
        import torch
        n = pos.numel() // 3
        if rho is None:
            rho = torch.zeros((self.N,) * 3, dtype=torch.float64,
                              device=pos.device if pos.is_cuda else torch.device("cuda"))
        m = float(self.N) ** 3 / max(n, 1) if mass is None else float(mass)
        recon_deposit_cic(self.h, self.N, pos, m, rho)
        return rho

    def deposit(self, pos, scheme="cic", mass=None, rho=None):
        """NGP / CIC / TSC density of pos (CUDA or pinned CPU tensor), mean 1
        by default; accumulated into rho when given."""
        import torch
        n = pos.numel() // 3
        if rho is None:
            rho = torch.zeros((self.N,) * 3, dtype=torch.float64,
                              device=pos.device if pos.is_cuda else torch.device("cuda"))
        m = float(self.N) ** 3 / max(n, 1) if mass is None else float(mass)
        recon_deposit(self.h, self.N, scheme, pos, m, rho)
        return rho

    def solve(self, b, phi=None, tol=1e-8, max_cycles=50, raise_on_noconv=True):
        import torch
        if phi is None:
            phi = torch.zeros_like(b)
        _, stats = recon_solve(self.h, self.N, b, phi, tol, max_cycles, raise_on_noconv)
        return phi, stats

    def level_scales(self):
        """Scaled-defect factor of each coarse level in the last FAS V-cycle."""
        return recon_level_scales(self.h)

    def displace(self, phi, b, psi=None, dl=None):
        """psi, dl: optional outputs (CUDA tensors or pinned CPU tensors)."""
        import torch
        if psi is None:
            psi = torch.empty((3,) + tuple(phi.shape), dtype=torch.float64, device=phi.device)
        if dl is None:
            dl = torch.empty_like(phi)
        recon_displace(self.h, self.N, phi, b, psi, dl)
        return psi, dl

    def displace_fp64(self, phi, b, psi=None, dl=None):
        """The same output as displace() in plain FP64 (the map whose gradient
        displace_adjoint returns)."""
        import torch
        if psi is None:
            psi = torch.empty((3,) + tuple(phi.shape), dtype=torch.float64, device=phi.device)
        if dl is None:
            dl = torch.empty_like(phi)
        recon_displace_fp64(self.h, self.N, phi, b, psi, dl)
        return psi, dl

    def displace_adjoint(self, phi, b, gbar_psi=None, gbar_dl=None):
        """(dLoss/dphi, dLoss/db) from dLoss/dpsi and dLoss/ddelta_r (None: zero)."""
        import torch
        gphi = torch.empty_like(phi)
        gb = torch.empty_like(b)
        recon_displace_adjoint(self.h, self.N, phi, b, gbar_psi, gbar_dl, gphi, gb)
        return gphi, gb

    def smooth_density(self, rho, R, floor=0.05, out=None):
        """Gaussian window of width R, floor, mean 1 (rho may be out)."""
        import torch
        if out is None:
            out = torch.empty_like(rho)
        recon_smooth_density(self.h, self.N, rho, R, floor, out)
        return out

    def gaussianise(self, field):
        """1-point Gaussianisation (rank mapping onto Gaussian quantiles)."""
        import torch
        out = torch.empty_like(field)
        recon_gaussianise(self.h, self.N, field, out)
        return out

    def adjoint(self, gbar_phi):
        import torch
        out = torch.empty_like(gbar_phi)
        recon_adjoint(self.h, self.N, gbar_phi, out)
        return out

    def close(self):
        if self.h is not None:
            recon_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent MIXED solves (uneven N) advanced together through
    CUDA-graph launches (recon_batch_* of include/recon.h)."""

    def __init__(self, sizes, boxes, stream=None):
        n = len(sizes)
        Ns = (ctypes.c_int * n)(*[int(v) for v in sizes])
        Ls = (ctypes.c_double * n)(*[float(v) for v in boxes])
        self.b = ctypes.c_void_p()
        st = load().recon_batch_create(n, Ns, Ls, ctypes.byref(self.b))
        if st != 0:
            raise ReconError(st, (load().recon_last_error(None) or b"").decode())
        self.sizes, self.boxes = list(sizes), list(boxes)
        if stream is not None:
            load().recon_batch_set_stream(self.b, _stream(stream))

    def handle(self, i):
        return ctypes.c_void_p(load().recon_batch_handle(self.b, int(i)))

    def configure(self, **kw):
        for i in range(len(self.sizes)):
            h = self.handle(i)
            c = recon_get_config(h)
            for k, v in kw.items():
                setattr(c, k, v)
            recon_set_config(h, c)
        return self

    def solve(self, bs, phis=None, tol=1e-8, max_cycles=50, raise_on_noconv=True):
        import torch
        n = len(self.sizes)
        if phis is None:
            phis = [torch.zeros_like(x) for x in bs]
        for x, N in zip(list(bs) + list(phis), self.sizes + self.sizes):
            _dev_ptr(x, torch.float64, N ** 3)
        bp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in bs])
        pp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in phis])
        stats = (recon_stats * n)()
        st = load().recon_batch_solve(self.b, bp, pp, float(tol), int(max_cycles), stats)
        if st != 0 and not (st == 3 and not raise_on_noconv):
            raise ReconError(st, (load().recon_batch_last_error(self.b) or b"").decode())
        return phis, [s.as_dict() for s in stats]

    def close(self):
        if self.b is not None:
            load().recon_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- slab steps
def _slab(lay):
    """recon_slab from any object with N, planes, first, lo, hi."""
    return ctypes.byref(recon_slab(int(lay.N), int(lay.planes), int(lay.first), int(lay.lo), int(lay.hi)))


def _slab_ptr(t, lay):
    import torch
    return _dev_ptr(t, torch.float64, lay.planes * lay.N * lay.N)


def recon_slab_sweep(lay, h, rule, theta, g, c, work, stream=None):
    _check(load().recon_slab_sweep(_slab(lay), float(h), int(rule), _slab_ptr(theta, lay), _slab_ptr(g, lay),
                                   float(c), _slab_ptr(work, lay), _stream(stream)))


def recon_slab_residual(lay, h, theta, g, c, r, stream=None):
    _check(load().recon_slab_residual(_slab(lay), float(h), _slab_ptr(theta, lay), _slab_ptr(g, lay), float(c),
                                      _slab_ptr(r, lay), _stream(stream)))


def recon_slab_det(lay, h, theta, out, stream=None):
    _check(load().recon_slab_det(_slab(lay), float(h), _slab_ptr(theta, lay), _slab_ptr(out, lay),
                                 _stream(stream)))


def recon_slab_restrict(lay_f, fine, lay_c, coarse, stream=None):
    _check(load().recon_slab_restrict(_slab(lay_f), _slab_ptr(fine, lay_f), _slab(lay_c),
                                      _slab_ptr(coarse, lay_c), _stream(stream)))


def recon_slab_prolong_add(lay_c, cnew, cold, scale, lay_f, fine, stream=None):
    _check(load().recon_slab_prolong_add(_slab(lay_c), _slab_ptr(cnew, lay_c),
                                         _slab_ptr(cold, lay_c) if cold is not None else None, float(scale),
                                         _slab(lay_f), _slab_ptr(fine, lay_f), _stream(stream)))


def recon_slab_plane_sums(lay, a, m, squared, out, stream=None):
    import torch
    _check(load().recon_slab_plane_sums(_slab(lay), _slab_ptr(a, lay), float(m), int(bool(squared)),
                                        _dev_ptr(out, torch.float64, lay.hi - lay.lo), _stream(stream)))


def recon_slab_eps_planes(lay, h, theta, g, c, out, stream=None):
    import torch
    _check(load().recon_slab_eps_planes(_slab(lay), float(h), _slab_ptr(theta, lay), _slab_ptr(g, lay), float(c),
                                        _dev_ptr(out, torch.float64, lay.hi - lay.lo), _stream(stream)))


def recon_slab_defect_min(lay, dH, rr, floor, out, stream=None):
    import torch
    _check(load().recon_slab_defect_min(_slab(lay), _slab_ptr(dH, lay), _slab_ptr(rr, lay), float(floor),
                                        _dev_ptr(out, torch.float64, lay.hi - lay.lo), _stream(stream)))


def recon_slab_form_rhs(lay, dH, rr, scale, g, stream=None):
    _check(load().recon_slab_form_rhs(_slab(lay), _slab_ptr(dH, lay), _slab_ptr(rr, lay), float(scale),
                                      _slab_ptr(g, lay), _stream(stream)))


def recon_slab_sub(lay, a, m, stream=None):
    _check(load().recon_slab_sub(_slab(lay), _slab_ptr(a, lay), float(m), _stream(stream)))
