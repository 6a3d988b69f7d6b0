"""Statistics of reconstructed fields: the shell-averaged cross-correlation
coefficient r(k) of two fields (Sec. III.C of the paper defines r per mode as
Re(d1 d2*) / (|d1| |d2|); averaged over spherical shells of width 2 pi / L:
r(k) = sum Re(d1 d2*) / sqrt(sum |d1|^2 sum |d2|^2)).

Measurement code: it is not part of the reconstruction path.  Works on numpy
arrays or torch tensors (on any device)."""
from __future__ import annotations

import numpy as np


def correlation(d1, d2, L: float, kmax: float | None = None):
    """Return (k_centres, r, modes) of two N^3 fields of box side L."""
    N = d1.shape[0]
    kf = 2.0 * np.pi / L
    try:
        import torch
        is_t = isinstance(d1, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        import torch
        f1 = torch.fft.rfftn(d1.double())
        f2 = torch.fft.rfftn(d2.double())
        k1 = torch.fft.fftfreq(N, d=1.0 / N, device=d1.device, dtype=torch.float64)
        kz = torch.fft.rfftfreq(N, d=1.0 / N, device=d1.device, dtype=torch.float64)
        kk = torch.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
        shell = torch.round(kk).long().ravel()
        # rfft half-plane weights: modes with 0 < kz < N/2 stand for two modes
        w = torch.full(kz.shape, 2.0, dtype=torch.float64, device=d1.device)
        w[0] = 1.0
        if N % 2 == 0:
            w[-1] = 1.0
        w = w[None, None, :].expand(N, N, kz.numel()).reshape(-1)
        nb = int(N // 2) + 1
        cr = torch.zeros(nb, dtype=torch.float64, device=d1.device)
        a1 = torch.zeros_like(cr)
        a2 = torch.zeros_like(cr)
        m = torch.zeros_like(cr)
        sel = shell < nb
        s = shell[sel]
        cr.index_add_(0, s, (w * (f1 * f2.conj()).real.ravel())[sel])
        a1.index_add_(0, s, (w * (f1.abs() ** 2).ravel())[sel])
        a2.index_add_(0, s, (w * (f2.abs() ** 2).ravel())[sel])
        m.index_add_(0, s, w[sel])
        cr, a1, a2, m = (x.cpu().numpy() for x in (cr, a1, a2, m))
    else:
        f1 = np.fft.rfftn(d1)
        f2 = np.fft.rfftn(d2)
        k1 = np.fft.fftfreq(N, d=1.0 / N)
        kz = np.fft.rfftfreq(N, d=1.0 / N)
        kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
        shell = np.rint(kk).astype(np.int64)
        w = np.full(kz.shape, 2.0)
        w[0] = 1.0
        if N % 2 == 0:
            w[-1] = 1.0
        w = np.broadcast_to(w[None, None, :], kk.shape)
        nb = N // 2 + 1
        sel = shell < nb
        cr = np.bincount(shell[sel], (w * (f1 * np.conj(f2)).real)[sel], nb)
        a1 = np.bincount(shell[sel], (w * np.abs(f1) ** 2)[sel], nb)
        a2 = np.bincount(shell[sel], (w * np.abs(f2) ** 2)[sel], nb)
        m = np.bincount(shell[sel], w[sel], nb)
    ok = (m > 0) & (a1 > 0) & (a2 > 0)
    ok[0] = False
    k = np.arange(nb) * kf
    r = np.where(ok, cr / np.sqrt(np.where(ok, a1 * a2, 1.0)), np.nan)
    if kmax is not None:
        keep = k <= kmax
        return k[keep], r[keep], m[keep]
    return k, r, m


def r_at(k, r, targets):
    """r(k) interpolated at the target wavenumbers (nan where undefined)."""
    good = np.isfinite(r)
    return {float(t): float(np.interp(t, k[good], r[good])) for t in targets}
