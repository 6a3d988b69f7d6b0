// recon_slab.cu -- the FP64 steps of the FAS V-cycle (Sec. II.A.2-3) on a
// slab of planes of a periodic N^3 grid, for the decomposition of one field
// over several processes (each process one slab of every level, with halo
// planes from its neighbours).
//
// An array holds `planes` planes of N x N values (C order); its plane p is
// the grid's plane (first + p) mod N, and its own planes (the ones a step
// writes) are [lo, hi).  A whole grid is planes = N, first = 0, lo = 0,
// hi = N: neighbours then wrap periodically along i.  For a slab the host
// checks that every plane a step reads is held, so the stencils never wrap
// along i inside the array.  Along j and k every array is the whole periodic
// line.
//
// The cell arithmetic is cellmath.cuh's (the single-grid solver's); the sums
// are per plane (one CTA per plane, a fixed reduction order) so that the
// caller adds them in plane order.  One thread per cell: these steps serve a
// decomposition whose cost is the exchange between processes, not the
// smoother's throughput.
#include "cellmath.cuh"
#include "internal.cuh"
#include "recon_slab.h"

namespace recon {
namespace {

struct Slab {
    int N, planes, first, lo, hi;
};

__device__ __forceinline__ int pmod(int a, int n)
{
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// 19-point neighbourhood of local plane i (neighbour planes i +- 1 wrap
// modulo the array's planes: only a whole grid ever wraps)
__device__ __forceinline__ Nb19<double> load19s(const double *__restrict__ a, const Slab &S, int i, int j, int k)
{
    const unsigned n = (unsigned)S.N, nn = n * n;
    const int P = S.planes, N = S.N;
    const unsigned ri = (unsigned)i * nn, rip = (unsigned)(i + 1 == P ? 0 : i + 1) * nn,
                   rim = (unsigned)(i == 0 ? P - 1 : i - 1) * nn;
    const unsigned cj = (unsigned)j * n, cjp = (unsigned)wp(j, N) * n, cjm = (unsigned)wm(j, N) * n;
    const unsigned kk = (unsigned)k, kp = (unsigned)wp(k, N), km = (unsigned)wm(k, N);
    Nb19<double> v;
    v.c = a[ri + cj + kk];
    v.xp = a[rip + cj + kk];
    v.xm = a[rim + cj + kk];
    v.yp = a[ri + cjp + kk];
    v.ym = a[ri + cjm + kk];
    v.zp = a[ri + cj + kp];
    v.zm = a[ri + cj + km];
    v.xpyp = a[rip + cjp + kk];
    v.xmym = a[rim + cjm + kk];
    v.xmyp = a[rim + cjp + kk];
    v.xpym = a[rip + cjm + kk];
    v.ypzp = a[ri + cjp + kp];
    v.ymzm = a[ri + cjm + km];
    v.ymzp = a[ri + cjm + kp];
    v.ypzm = a[ri + cjp + km];
    v.xpzp = a[rip + cj + kp];
    v.xmzm = a[rim + cj + km];
    v.xmzp = a[rim + cj + kp];
    v.xpzm = a[rip + cj + km];
    return v;
}

// one colour pass over local planes [pa, pb): cells of colour col get eq.
// update from src's values, the others are copied (so dst = src with one
// colour relaxed)
__global__ void __launch_bounds__(kThreads)
k_slab_pass(const double *__restrict__ src, double *__restrict__ dst, const double *__restrict__ g, double c,
            double ih2, double h2_6, Slab S, int pa, int pb, int col, int rule)
{
    const unsigned nn = (unsigned)S.N * (unsigned)S.N;
    const size_t cells = (size_t)(pb - pa) * nn;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (size_t)gridDim.x * blockDim.x) {
        const int i = pa + (int)(x / nn);
        const unsigned r = (unsigned)(x % nn);
        const int j = (int)(r / (unsigned)S.N), k = (int)(r % (unsigned)S.N);
        const unsigned id = (unsigned)i * nn + r;
        if (((S.first + i + j + k) & 1) != col) {
            dst[id] = src[id];
            continue;
        }
        const Nb19<double> n = load19s(src, S, i, j, k);
        double s, p, q;
        cubic_coeffs(n, ih2, g[id] + c, s, p, q);
        dst[id] = point_update(n.c, h2_6, s, p, q, rule);
    }
}

// MODE 0: r = g + c - det(I + H theta);  MODE 1: out = det(I + H theta)
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_slab_det(const double *__restrict__ t, const double *__restrict__ g, double c, double ih2, Slab S,
           double *__restrict__ out)
{
    const unsigned nn = (unsigned)S.N * (unsigned)S.N;
    const size_t cells = (size_t)(S.hi - S.lo) * nn;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (size_t)gridDim.x * blockDim.x) {
        const int i = S.lo + (int)(x / nn);
        const unsigned r = (unsigned)(x % nn);
        const int j = (int)(r / (unsigned)S.N), k = (int)(r % (unsigned)S.N);
        const unsigned id = (unsigned)i * nn + r;
        const double d = det_IH(load19s(t, S, i, j, k), ih2);
        out[id] = MODE == 0 ? g[id] + c - d : d;
    }
}

// coarse own planes = mean of the 8 sons (Sec. II.A.3)
__global__ void __launch_bounds__(kThreads)
k_slab_restrict(const double *__restrict__ f, Slab F, double *__restrict__ cr, Slab C)
{
    const int Nc = C.N, Nf = F.N;
    const unsigned nnc = (unsigned)Nc * (unsigned)Nc, nnf = (unsigned)Nf * (unsigned)Nf;
    const size_t cells = (size_t)(C.hi - C.lo) * nnc;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (size_t)gridDim.x * blockDim.x) {
        const int I = C.lo + (int)(x / nnc);
        const unsigned r = (unsigned)(x % nnc);
        const int J = (int)(r / (unsigned)Nc), K = (int)(r % (unsigned)Nc);
        const int gI = pmod(C.first + I, Nc);
        double acc = 0.0;
        for (int a = 0; a < 2; ++a) {
            const unsigned fi = (unsigned)pmod(2 * gI + a - F.first, Nf);
            for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc)
                    acc += f[fi * nnf + (unsigned)(2 * J + b) * (unsigned)Nf + (unsigned)(2 * K + cc)];
        }
        cr[(unsigned)I * nnc + r] = acc / 8.0;
    }
}

// fine own planes += scale P(cn - co), P the cell-centred trilinear
// interpolation of eq. corrections (weights 3/4, 1/4 per axis)
__global__ void __launch_bounds__(kThreads)
k_slab_prolong(const double *__restrict__ cn, const double *__restrict__ co, Slab C, double scale,
               double *__restrict__ f, Slab F)
{
    const int Nc = C.N, Nf = F.N;
    const unsigned nnc = (unsigned)Nc * (unsigned)Nc, nnf = (unsigned)Nf * (unsigned)Nf;
    const size_t cells = (size_t)(F.hi - F.lo) * nnf;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < cells; x += (size_t)gridDim.x * blockDim.x) {
        const int i = F.lo + (int)(x / nnf);
        const unsigned r = (unsigned)(x % nnf);
        const int j = (int)(r / (unsigned)Nf), k = (int)(r % (unsigned)Nf);
        const int gi = pmod(F.first + i, Nf);
        const int I = gi >> 1, J = j >> 1, K = k >> 1;
        const int di = (gi & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1, dk = (k & 1) ? 1 : -1;
        double acc = 0.0;
        for (int a = 0; a < 2; ++a) {
            const unsigned ci = (unsigned)pmod(I + a * di - C.first, Nc);
            for (int b = 0; b < 2; ++b) {
                const unsigned cj = (unsigned)pmod(J + b * dj, Nc);
                for (int cc = 0; cc < 2; ++cc) {
                    const unsigned ck = (unsigned)pmod(K + cc * dk, Nc);
                    const double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (cc ? 0.25 : 0.75);
                    const unsigned id = ci * nnc + cj * (unsigned)Nc + ck;
                    acc += w * (cn[id] - (co ? co[id] : 0.0));
                }
            }
        }
        f[(unsigned)i * nnf + r] += scale * acc;
    }
}

// per own plane (one CTA each): MODE 0 sum (a - m), 1 sum (a - m)^2,
// 2 sum of L_h^2 (the paper's epsilon; a = theta, b = g),
// 3 min over cells with rr < 0 of floor max(dH, 0) / (-rr), from 1 (a = dH, b = rr)
constexpr int kPlaneThreads = 512;
template <int MODE>
__global__ void __launch_bounds__(kPlaneThreads)
k_slab_planes(const double *__restrict__ a, const double *__restrict__ b, double m, double ih2, Slab S,
              double *__restrict__ out)
{
    __shared__ double sh[kPlaneThreads / 32];
    const int i = S.lo + blockIdx.x;
    const unsigned nn = (unsigned)S.N * (unsigned)S.N;
    double v = MODE == 3 ? 1.0 : 0.0;
    for (unsigned r = threadIdx.x; r < nn; r += blockDim.x) {
        const unsigned id = (unsigned)i * nn + r;
        if (MODE == 0) {
            v += a[id] - m;
        } else if (MODE == 1) {
            const double d = a[id] - m;
            v += d * d;
        } else if (MODE == 2) {
            const int j = (int)(r / (unsigned)S.N), k = (int)(r % (unsigned)S.N);
            double s, p, q;
            cubic_coeffs(load19s(a, S, i, j, k), ih2, b[id] + m, s, p, q);
            const double L = (s - 3.0) - (largest_root(p, q) - 3.0);
            v += L * L;
        } else {
            const double rr = b[id];
            if (rr < 0.0) {
                const double d = a[id] > 0.0 ? a[id] : 0.0;
                v = fmin(v, m * d / (-rr));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = MODE == 3 ? fmin(v, w) : v + w;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kPlaneThreads / 32 ? sh[threadIdx.x] : (MODE == 3 ? 1.0 : 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = MODE == 3 ? fmin(v, w) : v + w;
        }
        if (threadIdx.x == 0) out[blockIdx.x] = v;
    }
}

// own planes (contiguous): MODE 0 g = dH + s rr;  MODE 1 a -= m
template <int MODE>
__global__ void __launch_bounds__(kThreads)
k_slab_axpy(const double *__restrict__ dH, const double *__restrict__ rr, double s, double *__restrict__ out,
            size_t n)
{
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
        out[x] = MODE == 0 ? dH[x] + s * rr[x] : out[x] - s;
}

bool whole(const Slab &S) { return S.planes == S.N && S.first == 0 && S.lo == 0 && S.hi == S.N; }

// the layout is a slab of an even N^3 grid within the 32-bit offset range;
// `halo` planes on each side of the own planes are held (or the grid is whole)
bool valid(const recon_slab *s, int halo)
{
    if (!s) return false;
    const Slab S{s->N, s->planes, s->first, s->lo, s->hi};
    if (S.N < 4 || S.N > kMaxN || S.N % 2 != 0) return false;
    if (S.planes < 1 || S.planes > S.N + 8 || S.lo < 0 || S.hi > S.planes || S.lo >= S.hi) return false;
    if (whole(S)) return true;
    if (S.planes > S.N) return false;   // a slab never holds a plane twice
    return S.lo >= halo && S.hi + halo <= S.planes;
}

Slab dev(const recon_slab *s) { return Slab{s->N, s->planes, s->first, s->lo, s->hi}; }

size_t own_cells(const Slab &S) { return (size_t)(S.hi - S.lo) * S.N * S.N; }

// the global planes [g0, g1] (inclusive, unwrapped) are held by S
bool holds(const Slab &S, int g0, int g1)
{
    if (whole(S)) return true;
    for (int g = g0; g <= g1; ++g) {
        const int p = ((g - S.first) % S.N + S.N) % S.N;
        if (p >= S.planes) return false;
    }
    return true;
}

recon_status finish(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error((std::string(what) + ": " + cudaGetErrorString(e)).c_str());
        return RECON_E_CUDA;
    }
    return RECON_OK;
}

recon_status bad(const char *what)
{
    set_thread_error((std::string(what) + ": bad slab layout or argument").c_str());
    return RECON_E_INVALID;
}

}  // namespace

cudaError_t paper_eps_planes(int N, double h, const double *theta, const double *g, double c, double *out,
                             cudaStream_t s)
{
    const Slab S{N, N, 0, 0, N};
    note_launch(1);
    k_slab_planes<2><<<N, kPlaneThreads, 0, s>>>(theta, g, c, 1.0 / (h * h), S, out);
    return cudaGetLastError();
}

}  // namespace recon

using namespace recon;

extern "C" recon_status recon_slab_sweep(const recon_slab *s, double h, int rule, double *theta, const double *g,
                                         double c, double *work, void *stream)
{
    if (!valid(s, 2) || !(h > 0) || !theta || !g || !work || (rule != 0 && rule != 1))
        return bad("recon_slab_sweep");
    const Slab S = dev(s);
    const cudaStream_t st = (cudaStream_t)stream;
    const double ih2 = 1.0 / (h * h), h2_6 = h * h / 6.0;
    const int a0 = whole(S) ? 0 : S.lo - 1, b0 = whole(S) ? S.N : S.hi + 1;
    const size_t nn = (size_t)S.N * S.N;
    note_launch(2);
    k_slab_pass<<<stride_blocks((size_t)(b0 - a0) * nn), kThreads, 0, st>>>(theta, work, g, c, ih2, h2_6, S, a0, b0,
                                                                            0, rule);
    k_slab_pass<<<stride_blocks(own_cells(S)), kThreads, 0, st>>>(work, theta, g, c, ih2, h2_6, S, S.lo, S.hi, 1,
                                                                  rule);
    return finish("recon_slab_sweep");
}

extern "C" recon_status recon_slab_residual(const recon_slab *s, double h, const double *theta, const double *g,
                                            double c, double *r, void *stream)
{
    if (!valid(s, 1) || !(h > 0) || !theta || !g || !r) return bad("recon_slab_residual");
    const Slab S = dev(s);
    note_launch(1);
    k_slab_det<0><<<stride_blocks(own_cells(S)), kThreads, 0, (cudaStream_t)stream>>>(theta, g, c, 1.0 / (h * h),
                                                                                     S, r);
    return finish("recon_slab_residual");
}

extern "C" recon_status recon_slab_det(const recon_slab *s, double h, const double *theta, double *out,
                                       void *stream)
{
    if (!valid(s, 1) || !(h > 0) || !theta || !out) return bad("recon_slab_det");
    const Slab S = dev(s);
    note_launch(1);
    k_slab_det<1><<<stride_blocks(own_cells(S)), kThreads, 0, (cudaStream_t)stream>>>(theta, nullptr, 0.0,
                                                                                     1.0 / (h * h), S, out);
    return finish("recon_slab_det");
}

extern "C" recon_status recon_slab_restrict(const recon_slab *fs, const double *fine, const recon_slab *cs,
                                            double *coarse, void *stream)
{
    if (!valid(fs, 0) || !valid(cs, 0) || !fine || !coarse || fs->N != 2 * cs->N) return bad("recon_slab_restrict");
    const Slab F = dev(fs), C = dev(cs);
    const int g0 = C.first + C.lo, g1 = C.first + C.hi - 1;
    if (!whole(C) && (g0 < 0 || g1 >= C.N)) return bad("recon_slab_restrict");
    if (!holds(F, 2 * g0, 2 * g1 + 1)) return bad("recon_slab_restrict");
    note_launch(1);
    k_slab_restrict<<<stride_blocks(own_cells(C)), kThreads, 0, (cudaStream_t)stream>>>(fine, F, coarse, C);
    return finish("recon_slab_restrict");
}

extern "C" recon_status recon_slab_prolong_add(const recon_slab *cs, const double *cnew, const double *cold,
                                               double scale, const recon_slab *fs, double *fine, void *stream)
{
    if (!valid(cs, 0) || !valid(fs, 0) || !cnew || !fine || fs->N != 2 * cs->N) return bad("recon_slab_prolong_add");
    const Slab C = dev(cs), F = dev(fs);
    const int g0 = F.first + F.lo, g1 = F.first + F.hi - 1;
    if (!whole(F) && (g0 < 0 || g1 >= F.N)) return bad("recon_slab_prolong_add");
    if (!holds(C, g0 / 2 - 1, g1 / 2 + 1)) return bad("recon_slab_prolong_add");
    note_launch(1);
    k_slab_prolong<<<stride_blocks(own_cells(F)), kThreads, 0, (cudaStream_t)stream>>>(cnew, cold, C, scale, fine,
                                                                                       F);
    return finish("recon_slab_prolong_add");
}

extern "C" recon_status recon_slab_plane_sums(const recon_slab *s, const double *a, double m, int squared,
                                              double *out, void *stream)
{
    if (!valid(s, 0) || !a || !out || (squared != 0 && squared != 1)) return bad("recon_slab_plane_sums");
    const Slab S = dev(s);
    note_launch(1);
    if (squared)
        k_slab_planes<1><<<S.hi - S.lo, kPlaneThreads, 0, (cudaStream_t)stream>>>(a, nullptr, m, 0.0, S, out);
    else
        k_slab_planes<0><<<S.hi - S.lo, kPlaneThreads, 0, (cudaStream_t)stream>>>(a, nullptr, m, 0.0, S, out);
    return finish("recon_slab_plane_sums");
}

extern "C" recon_status recon_slab_eps_planes(const recon_slab *s, double h, const double *theta, const double *g,
                                              double c, double *out, void *stream)
{
    if (!valid(s, 1) || !(h > 0) || !theta || !g || !out) return bad("recon_slab_eps_planes");
    const Slab S = dev(s);
    note_launch(1);
    k_slab_planes<2><<<S.hi - S.lo, kPlaneThreads, 0, (cudaStream_t)stream>>>(theta, g, c, 1.0 / (h * h), S, out);
    return finish("recon_slab_eps_planes");
}

extern "C" recon_status recon_slab_defect_min(const recon_slab *s, const double *dH, const double *rr,
                                              double floor_, double *out, void *stream)
{
    if (!valid(s, 0) || !dH || !rr || !out || !(floor_ > 0)) return bad("recon_slab_defect_min");
    const Slab S = dev(s);
    note_launch(1);
    k_slab_planes<3><<<S.hi - S.lo, kPlaneThreads, 0, (cudaStream_t)stream>>>(dH, rr, floor_, 0.0, S, out);
    return finish("recon_slab_defect_min");
}

extern "C" recon_status recon_slab_form_rhs(const recon_slab *s, const double *dH, const double *rr, double scale,
                                            double *g, void *stream)
{
    if (!valid(s, 0) || !dH || !rr || !g) return bad("recon_slab_form_rhs");
    const Slab S = dev(s);
    const size_t off = (size_t)S.lo * S.N * S.N, n = own_cells(S);
    note_launch(1);
    k_slab_axpy<0><<<stride_blocks(n), kThreads, 0, (cudaStream_t)stream>>>(dH + off, rr + off, scale, g + off, n);
    return finish("recon_slab_form_rhs");
}

extern "C" recon_status recon_slab_sub(const recon_slab *s, double *a, double m, void *stream)
{
    if (!valid(s, 0) || !a) return bad("recon_slab_sub");
    const Slab S = dev(s);
    const size_t off = (size_t)S.lo * S.N * S.N, n = own_cells(S);
    note_launch(1);
    k_slab_axpy<1><<<stride_blocks(n), kThreads, 0, (cudaStream_t)stream>>>(nullptr, nullptr, m, a + off, n);
    return finish("recon_slab_sub");
}
