"""Python face of the FP64 CPU oracle (test infrastructure only).

The arithmetic lives in ``recon_oracle.c`` (plain C, single-threaded, built
with ``-ffp-contract=off``); this module compiles it with gcc, loads it with
ctypes and marshals numpy arrays.  Two oracle steps are written here because
their clearest statement is a library primitive:

* ``adjoint`` -- the gradient of a loss on theta with respect to b, from the
  implicit-function theorem on the augmented system
  ``det(I + H theta) - c = b, mean(theta) = 0``, solved on the transposed
  Jacobian with a sparse LU (scipy) up to 16^3 and GMRES with an
  incomplete-LU preconditioner (to a 1e-14 relative residual) beyond.
* ``jacobian_matrix`` -- the sparse matrix of J v = sum adj(I+H)_ab D_ab v
  assembled from the C rows.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recon_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librecon_oracle.so")
_lock = threading.Lock()
_lib = None

ORDERINGS = {"rb-snapshot": 0, "rb-lex": 1, "4-colour": 2}
RULES = {"newton1": 0, "exact": 1}

_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_largest_root": (_D, [_D, _D]),
            "or_point_update": (_D, [_D, _D, _D, _D, _D, _I]),
            "or_sweep": (None, [_P, _P, _D, _I, _D, _I, _I]),
            "or_residual": (None, [_P, _P, _D, _I, _D, _P]),
            "or_paper_eps": (_D, [_P, _P, _D, _I, _D]),
            "or_paper_eps_planes": (None, [_P, _P, _D, _I, _D, _P]),
            "or_plane_sums": (None, [_P, _I, _I, _D, _I, _P]),
            "or_restrict": (None, [_P, _I, _P]),
            "or_prolong_add": (None, [_P, _P, _I, _D, _P]),
            "or_defect_scale": (_D, [_P, _P, _L, _D]),
            "or_coarse_solve": (_I, [_P, _P, _D, _I, _D, _P]),
            "or_num_levels": (_I, [_I]),
            "or_solve": (_I, [_P, _I, _D, _P, _P, _D, _I, _P, _I, _P]),
            "or_vcycle": (None, [_P, _I, _D, _P, _D, _P]),
            "or_cic_deposit": (None, [_P, _L, _I, _D, _D, _P]),
            "or_assign_deposit": (None, [_P, _L, _I, _D, _D, _I, _P]),
            "or_cic_cells": (None, [_P, _L, _I, _D, _P, _P]),
            "or_displace": (None, [_P, _P, _I, _D, _P, _P]),
            "or_cofactors": (None, [_P, _I, _D, _P]),
            "or_jacobian_apply": (None, [_P, _P, _I, _D, _P]),
            "or_jacobian_coo": (None, [_P, _I, _D, _P, _P, _P]),
            "or_det_grid": (None, [_P, _I, _D, _P]),
            "or_det_cells": (None, [_P, _I, _D, _L, _P, _P]),
            "or_cubic_grid": (None, [_P, _P, _D, _I, _D, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class _Params(ctypes.Structure):
    """Mirror of the oracle's or_params struct."""
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("coarse_max_sweeps", ctypes.c_int), ("coarse_rtol", ctypes.c_double),
                ("ordering", ctypes.c_int), ("rule", ctypes.c_int),
                ("scale_floor", ctypes.c_double)]


def _params(nu1=2, nu2=2, coarse_max_sweeps=200, coarse_rtol=1e-3,
            ordering="rb-snapshot", rule="newton1", scale_floor=0.5):
    return _Params(int(nu1), int(nu2), int(coarse_max_sweeps), float(coarse_rtol),
                   ORDERINGS[ordering], RULES[rule], float(scale_floor))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _grid_n(a: np.ndarray) -> int:
    if a.ndim != 3 or not (a.shape[0] == a.shape[1] == a.shape[2]):
        raise ValueError("expected an N^3 grid")
    return a.shape[0]


# ---------------------------------------------------------------- pointwise
def largest_root(p: float, q: float) -> float:
    """Largest real root of s^3 + p s + q (eq. root, read as the largest root)."""
    return _load().or_largest_root(float(p), float(q))


def point_update(theta_c, h, s, p, q, rule="newton1") -> float:
    """Eq. update: theta_c - (h^2/6)(s_new - s)."""
    return _load().or_point_update(float(theta_c), float(h), float(s), float(p),
                                   float(q), RULES[rule])


# ---------------------------------------------------------------- grids
def det_grid(theta, h) -> np.ndarray:
    """det(I + H_h theta) per cell (eq. basic_eqs with eq. discrete_examples)."""
    t = _f64(theta)
    out = np.empty_like(t)
    _load().or_det_grid(_ptr(t), _grid_n(t), float(h), _ptr(out))
    return out


def det_cells(theta, h, ijk) -> np.ndarray:
    """det(I + H_h theta) at the cells listed in ijk ([m, 3] ints)."""
    t = _f64(theta)
    idx = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    out = np.empty(idx.shape[0])
    _load().or_det_cells(_ptr(t), _grid_n(t), float(h), idx.shape[0], _ptr(idx), _ptr(out))
    return out


def cubic_grid(theta, g, c, h):
    """Per-cell (s, p, q) of the cubic of eq. final_PDE with rhs = g + c."""
    t, gg = _f64(theta), _f64(g)
    s, p, q = (np.empty_like(t) for _ in range(3))
    _load().or_cubic_grid(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h),
                          _ptr(s), _ptr(p), _ptr(q))
    return s, p, q


def sweep(theta, g, c, h, ordering="rb-snapshot", rule="newton1", sweeps=1):
    """``sweeps`` Gauss-Seidel sweeps (Sec. II.A.2); returns a new array."""
    t = _f64(theta).copy()
    gg = _f64(g)
    lib = _load()
    for _ in range(sweeps):
        lib.or_sweep(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h),
                     ORDERINGS[ordering], RULES[rule])
    return t


def residual(theta, g, c, h) -> np.ndarray:
    """r = g + c - det(I + H theta)."""
    t, gg = _f64(theta), _f64(g)
    r = np.empty_like(t)
    _load().or_residual(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h), _ptr(r))
    return r


def paper_eps(theta, g, c, h) -> float:
    """The paper's epsilon = rms(lap theta - Sigma) (Sec. II.A.2)."""
    t, gg = _f64(theta), _f64(g)
    return _load().or_paper_eps(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h))


def paper_eps_planes(theta, g, c, h) -> np.ndarray:
    """Per-plane partial sums of L_h^2 (the terms of the paper's epsilon)."""
    t, gg = _f64(theta), _f64(g)
    out = np.empty(t.shape[0])
    _load().or_paper_eps_planes(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h), _ptr(out))
    return out


def plane_sums(a, m=0.0, squared=False) -> np.ndarray:
    """Per-plane sums of (a - m) or (a - m)^2 over a (planes, N, N) array, each
    a running sum in memory order: the partial sums every grid sum of the
    oracle is built from (added in plane order)."""
    x = _f64(a)
    if x.ndim != 3 or x.shape[1] != x.shape[2]:
        raise ValueError("expected a (planes, N, N) array")
    out = np.empty(x.shape[0])
    _load().or_plane_sums(_ptr(x), x.shape[0], x.shape[1], float(m), int(bool(squared)), _ptr(out))
    return out


def restrict(fine) -> np.ndarray:
    """R: mean of the 8 son cells (Sec. II.A.3)."""
    f = _f64(fine)
    n = _grid_n(f)
    out = np.empty((n // 2,) * 3)
    _load().or_restrict(_ptr(f), n, _ptr(out))
    return out


def prolong_add(coarse_new, coarse_old, fine, scale=1.0) -> np.ndarray:
    """fine + scale P(coarse_new - coarse_old), P cell-centred trilinear (eq. corrections)."""
    cn, co = _f64(coarse_new), _f64(coarse_old)
    f = _f64(fine).copy()
    _load().or_prolong_add(_ptr(cn), _ptr(co), _grid_n(cn), float(scale), _ptr(f))
    return f


def defect_scale(det_coarse, restricted_residual, floor=0.5) -> float:
    """Scaled-defect factor s of the coarse equation (0 = skip the coarse grid)."""
    d, r = _f64(det_coarse), _f64(restricted_residual)
    return _load().or_defect_scale(_ptr(d), _ptr(r), d.size, float(floor))


def coarse_solve(theta, g, c, h, max_sweeps=200, rtol=1e-3,
                 ordering="rb-snapshot", rule="newton1"):
    """Coarsest-grid Gauss-Seidel to a relative residual drop; returns (theta, sweeps)."""
    t = _f64(theta).copy()
    gg = _f64(g)
    P = _params(0, 0, max_sweeps, rtol, ordering, rule)
    n = _load().or_coarse_solve(_ptr(t), _ptr(gg), float(c), _grid_n(t), float(h),
                                ctypes.byref(P))
    return t, n


def num_levels(N: int) -> int:
    return _load().or_num_levels(int(N))


def solve(b, L, theta0=None, c0=0.0, tol=1e-10, max_cycles=50, nu1=2, nu2=2,
          coarse_max_sweeps=200, coarse_rtol=1e-3, ordering="rb-snapshot",
          rule="newton1", scale_floor=0.5, fmg=None):
    """Full FAS solve (Sec. II.A.2-3).

    ``fmg`` (default: on when no ``theta0`` is given) starts with nested
    iteration from theta = 0 on the coarsest grid.  Returns ``(theta, info)``
    with info = dict(status, cycles, rel_residual, c, paper_eps, history);
    status 0 = converged, 3 = max_cycles reached, 4 = non-finite residual.
    """
    bb = _f64(b)
    N = _grid_n(bb)
    if fmg is None:
        fmg = theta0 is None
    t = np.zeros_like(bb) if theta0 is None else _f64(theta0).copy()
    c = ctypes.c_double(float(c0))
    stats = np.zeros(4 + max_cycles)
    P = _params(nu1, nu2, coarse_max_sweeps, coarse_rtol, ordering, rule, scale_floor)
    st = _load().or_solve(_ptr(bb), N, float(L), _ptr(t), ctypes.byref(c),
                          float(tol), int(max_cycles), ctypes.byref(P), int(bool(fmg)),
                          _ptr(stats))
    cyc = int(stats[0])
    info = dict(status=st, cycles=cyc, rel_residual=float(stats[1]),
                c=float(stats[2]), paper_eps=float(stats[3]),
                history=stats[4:4 + cyc].tolist())
    return t, info


def vcycle(b, L, theta, c=0.0, nu1=2, nu2=2, coarse_max_sweeps=200,
           coarse_rtol=1e-3, ordering="rb-snapshot", rule="newton1", scale_floor=0.5):
    """One FAS V-cycle on the finest level (no c / gauge update); returns theta."""
    bb = _f64(b)
    t = _f64(theta).copy()
    P = _params(nu1, nu2, coarse_max_sweeps, coarse_rtol, ordering, rule, scale_floor)
    _load().or_vcycle(_ptr(bb), _grid_n(bb), float(L), _ptr(t), float(c), ctypes.byref(P))
    return t


# ---------------------------------------------------------------- CIC
def cic_cells(pos, N, L):
    """Per particle and axis: CIC base cell index and fraction (footnote on CIC)."""
    p = _f64(pos).reshape(-1, 3)
    cells = np.empty(p.shape, dtype=np.int32)
    frac = np.empty(p.shape)
    _load().or_cic_cells(_ptr(p), p.shape[0], int(N), float(L), _ptr(cells), _ptr(frac))
    return cells, frac


def cic_deposit(pos, N, L, mass=None) -> np.ndarray:
    """CIC density; default mass N^3 / n_particles gives a mean-1 field."""
    p = _f64(pos).reshape(-1, 3)
    n = p.shape[0]
    m = (float(N) ** 3 / n) if mass is None else float(mass)
    rho = np.zeros((N, N, N))
    _load().or_cic_deposit(_ptr(p), n, int(N), float(L), m, _ptr(rho))
    return rho


ASSIGN = {"ngp": 0, "cic": 1, "tsc": 2}


def assign_deposit(pos, N, L, scheme="cic", mass=None) -> np.ndarray:
    """NGP / CIC / TSC density (Sec. I footnote); default mass N^3 / n."""
    p = _f64(pos).reshape(-1, 3)
    n = p.shape[0]
    m = (float(N) ** 3 / n) if mass is None else float(mass)
    rho = np.zeros((N, N, N))
    _load().or_assign_deposit(_ptr(p), n, int(N), float(L), m, ASSIGN[scheme], _ptr(rho))
    return rho


# ---------------------------------------------------------------- output
def displace(theta, b, L):
    """Sec. II.B restated: psi = -grad theta [3,N,N,N] and delta_r on the q-grid."""
    t, bb = _f64(theta), _f64(b)
    N = _grid_n(t)
    psi = np.empty((3, N, N, N))
    dl = np.empty_like(t)
    _load().or_displace(_ptr(t), _ptr(bb), N, float(L), _ptr(psi), _ptr(dl))
    return psi, dl


def displace_adjoint(theta, b, L, gbar_psi=None, gbar_dl=None):
    """Adjoint of ``displace`` (Sec. II.B as restated there): given the
    gradients of a loss with respect to psi [3,N,N,N] and delta_r [N,N,N]
    (None = zero), return its gradients with respect to theta and b.

    The forward map, cell c at x_c = (i + 1/2) h:
      g_c = central-difference gradient of theta,  psi_c = -g_c,
      q_c = x_c + g_c (mod L),  A_c = I + H_c theta,  v_c = 3 - tr(A_c^-1),
      num = CIC(q, b v),  den = CIC(q, b),  delta_r = num / max(den, 1e-12).
    Chain rule, in reverse order (plain FP64 numpy; the CIC cells and
    fractions come from ``cic_cells``, the same formula as the forward):
      gN = gbar_dl / max(den, eps),  gD = -gbar_dl num / den^2 (den > eps),
      per cell: gwv = sum_corners gN W,  gwb = sum_corners gD W,
                gq_d = sum_corners (b v gN + b gD) dW/dq_d  (dW/dq_d = +-W_other / h),
      gbar_b = gwv v + gwb,  gv = gwv b,  dv/dA = A^-2 (A symmetric),
      gbar_theta = sum_ab D_ab(gv (A^-2)_ab) - sum_d D_d(gq_d - gbar_psi_d),
    with D_ab the (self-adjoint) second-difference stencils of eq.
    discrete_examples and D_d the (anti-self-adjoint) central differences.
    """
    t, bb = _f64(theta), _f64(b)
    N = _grid_n(t)
    h = L / N
    gps = np.zeros((3, N, N, N)) if gbar_psi is None else _f64(gbar_psi).reshape(3, N, N, N)
    gdl = np.zeros((N, N, N)) if gbar_dl is None else _f64(gbar_dl).reshape(N, N, N)

    def sh(a, s, ax):            # sh(a, 1, ax)[i] = a[i + 1] (periodic)
        return np.roll(a, -s, axis=ax)

    def d1(a, ax):               # central difference
        return (sh(a, 1, ax) - sh(a, -1, ax)) / (2.0 * h)

    def d2(a, ax, bx):           # second-difference stencils D_ab
        if ax == bx:
            return (sh(a, 1, ax) + sh(a, -1, ax) - 2.0 * a) / (h * h)
        return (sh(sh(a, 1, ax), 1, bx) + sh(sh(a, -1, ax), -1, bx)
                - sh(sh(a, -1, ax), 1, bx) - sh(sh(a, 1, ax), -1, bx)) / (4.0 * h * h)

    # forward intermediates
    g = [d1(t, a) for a in range(3)]
    A = np.empty((N, N, N, 3, 3))
    for a in range(3):
        for c in range(3):
            A[..., a, c] = d2(t, a, c) + (1.0 if a == c else 0.0)
    Ainv = np.linalg.inv(A)
    v = 3.0 - np.trace(Ainv, axis1=-2, axis2=-1)
    x = (np.arange(N) + 0.5) * h
    X = np.meshgrid(x, x, x, indexing="ij")
    q = np.empty((N, N, N, 3))
    for a in range(3):
        qa = np.fmod(X[a] + g[a], L)
        q[..., a] = np.where(qa < 0.0, qa + L, qa)
    cells, frac = cic_cells(q.reshape(-1, 3), N, L)
    wv, wb = (bb * v).ravel(), bb.ravel()
    corners = []
    for ca in (0, 1):
        for cb in (0, 1):
            for cc in (0, 1):
                off = np.array([ca, cb, cc])
                idx = (cells + off) % N
                flat = (idx[:, 0] * N + idx[:, 1]) * N + idx[:, 2]
                w1 = np.where(off == 1, frac, 1.0 - frac)          # per-axis weights
                sgn = np.where(off == 1, 1.0, -1.0) / h             # d w1 / d q
                W = w1[:, 0] * w1[:, 1] * w1[:, 2]
                dW = np.stack([sgn[0] * w1[:, 1] * w1[:, 2],
                               w1[:, 0] * sgn[1] * w1[:, 2],
                               w1[:, 0] * w1[:, 1] * sgn[2]], axis=1)
                corners.append((flat, W, dW))
    num = np.zeros(N ** 3)
    den = np.zeros(N ** 3)
    for flat, W, _ in corners:
        np.add.at(num, flat, wv * W)
        np.add.at(den, flat, wb * W)
    gd = gdl.ravel()
    gN = gd / np.maximum(den, 1e-12)
    gD = np.where(den > 1e-12, -gd * num / np.where(den > 1e-12, den, 1.0) ** 2, 0.0)
    gwv = np.zeros(N ** 3)
    gwb = np.zeros(N ** 3)
    gq = np.zeros((N ** 3, 3))
    for flat, W, dW in corners:
        gwv += gN[flat] * W
        gwb += gD[flat] * W
        gq += (wv * gN[flat] + wb * gD[flat])[:, None] * dW
    gb = (gwv * v.ravel() + gwb).reshape(N, N, N)
    gv = (gwv * bb.ravel()).reshape(N, N, N)
    G = gv[..., None, None] * (Ainv @ Ainv)
    gt = np.zeros((N, N, N))
    for a in range(3):
        for c in range(3):
            gt += d2(G[..., a, c], a, c)
    for a in range(3):
        gt -= d1(gq[:, a].reshape(N, N, N) - gps[a], a)
    return gt, gb


def cofactors(theta, h) -> np.ndarray:
    """adj(I + H theta) entries (xx, yy, zz, xy, yz, xz) as [6,N,N,N]."""
    t = _f64(theta)
    N = _grid_n(t)
    out = np.empty((6, N, N, N))
    _load().or_cofactors(_ptr(t), N, float(h), _ptr(out))
    return out


def jacobian_apply(theta, v, h) -> np.ndarray:
    """J v = sum adj(I+H)_ab D_ab v, the linearisation of det(I + H theta)."""
    t, vv = _f64(theta), _f64(v)
    out = np.empty_like(t)
    _load().or_jacobian_apply(_ptr(t), _ptr(vv), _grid_n(t), float(h), _ptr(out))
    return out


def jacobian_matrix(theta, h):
    """Sparse J (scipy CSR, n x n) assembled from the oracle's stencil rows."""
    import scipy.sparse as sp
    t = _f64(theta)
    N = _grid_n(t)
    n = N ** 3
    rows = np.empty(19 * n, dtype=np.int64)
    cols = np.empty(19 * n, dtype=np.int64)
    vals = np.empty(19 * n)
    _load().or_jacobian_coo(_ptr(t), N, float(h), _ptr(rows), _ptr(cols), _ptr(vals))
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def adjoint(theta, gbar_theta, h):
    """Gradient of a loss on theta with respect to b (implicit-function theorem).

    The solve defines theta(b) through F(theta, c; b) = det(I+H theta) - c - b = 0
    with mean(theta) = 0.  With A = [[J, -1], [1^T/n, 0]] the forward
    sensitivity is A [dtheta; dc] = [db; 0], so the adjoint solves
    A^T [lam; mu] = [gbar; 0] and returns lam (= dLoss/db).  lam has zero sum.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    t = _f64(theta)
    N = _grid_n(t)
    n = N ** 3
    J = jacobian_matrix(t, h)
    ones = np.ones((n, 1))
    A = sp.bmat([[J, sp.csr_matrix(-ones)],
                 [sp.csr_matrix(ones.T / n), None]], format="csc")
    rhs = np.concatenate([_f64(gbar_theta).ravel(), [0.0]])
    AT = A.T.tocsc()
    if n <= 5000:
        sol = spl.spsolve(AT, rhs)
    else:
        # the direct factorisation's fill grows too fast beyond ~16^3; GMRES
        # with an incomplete-LU preconditioner solves the same system to a
        # relative residual of 1e-14
        ilu = spl.spilu(AT, drop_tol=1e-5, fill_factor=20)
        M = spl.LinearOperator(AT.shape, ilu.solve)
        sol, info = spl.gmres(AT, rhs, M=M, rtol=1e-14, atol=0, restart=200, maxiter=2000)
        res = np.linalg.norm(AT @ sol - rhs) / np.linalg.norm(rhs)
        if info != 0 or res > 1e-12:
            raise RuntimeError(f"oracle adjoint: GMRES did not converge (residual {res:.2e})")
    return sol[:n].reshape(N, N, N)


# ---------------------------------------------------------------- density preparation
def smooth_and_floor(rho, L, R, floor=0.05):
    """Density preparation before the solve, in FP64:
        1. Gaussian window of width R (Sec. III smooths its density fields
           with one): multiply the DFT of rho by exp(-k^2 R^2 / 2), k the
           box's wave vector 2 pi m / L (m the signed DFT index per axis);
        2. floor: 1 + delta >= floor, so every cell's right side is positive;
        3. divide by the mean, restoring mean 1.
    numpy's FFT is the library step for 1."""
    r = _f64(rho)
    N = _grid_n(r)
    if R > 0:
        m = np.fft.fftfreq(N, d=1.0 / N)
        k = 2.0 * np.pi * m / L
        k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
        r = np.fft.ifftn(np.fft.fftn(r) * np.exp(-0.5 * k2 * R * R)).real
    b = np.maximum(r, floor)
    return b / b.mean()


# ---------------------------------------------------------------- post-processing
def gaussianise(field):
    """1-point Gaussianisation of a field (Sec. III, after Weinberg 1992 and
    Neyrinck 2009), read as the rank mapping
        g_i = mean + std * Phi^-1((rank_i + 1/2) / n),
    rank_i the position of value i in ascending order with ties broken by
    position (a stable sort), mean and std the input's (population std).
    A library sort and scipy's ndtri are the steps.  Returns (g, rank)."""
    from scipy.special import ndtri
    f = _f64(field)
    v = f.ravel()
    order = np.argsort(v, kind="stable")
    rank = np.empty(v.size, dtype=np.int64)
    rank[order] = np.arange(v.size)
    g = v.mean() + v.std() * ndtri((rank + 0.5) / v.size)
    return g.reshape(f.shape), rank.reshape(f.shape)
