// recon_adjoint.cu -- adjoint of the solve (implicit-function theorem).
//
// The solve defines phi(b) through F(phi, c; b) = det(I + H phi) - c - b = 0
// with mean(phi) = 0.  With J = dF/dphi = sum_ab adj(I+H)_ab D_ab (stencils
// of eq. discrete_examples) the gradient of a loss with respect to b is the
// lam of
//     J^T lam + mu 1 = gbar,   sum(lam) = 0,
// with J^T lam = sum_ab D_ab (adj_ab * lam) (the D_ab are symmetric).  J 1 = 0
// makes range(J^T) the mean-free fields, so mu = mean(gbar); J^T has one null
// vector n = 1 + w (J^T w = -J^T 1), and lam = lam0 - (sum lam0 / sum n) n for
// any solution lam0 of J^T lam0 = gbar - mean(gbar).
//
// Both linear solves use FP64 red-black Gauss-Seidel multigrid on J^T.  The
// coarse levels' cofactors are computed once per call from the restricted
// potential and kept; the finest level's are formed again from phi in every
// application of J^T (k_jt_fine) unless adjoint_store_cofactors keeps them
// too (48 N^3 bytes).
#include <cmath>
#include <string>

#include "cellmath.cuh"
#include "internal.cuh"

namespace recon {

namespace {

constexpr int kRT = kRowX * kRowY;

struct CofPtr {
    const double *xx, *yy, *zz, *xy, *yz, *xz;
};
__host__ __device__ inline CofPtr cof_of(const double *base, size_t n)
{
    return {base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n};
}

__global__ void __launch_bounds__(kRT)
k_cof6(const double *__restrict__ th, int N, double ih2, double *__restrict__ cof)
{
    const size_t n = (size_t)N * N * N;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const Cof<double> a = cofactors(load19<double>(th, N, i, j, k), ih2);
        const unsigned id = offs(N, i, j, k);
        cof[id] = a.xx;
        cof[n + id] = a.yy;
        cof[2 * n + id] = a.zz;
        cof[3 * n + id] = a.xy;
        cof[4 * n + id] = a.yz;
        cof[5 * n + id] = a.xz;
    }
}

// (J^T lam) at (i, j, k) and the diagonal of J^T there.
__device__ __forceinline__ double jt_at(const CofPtr C, const double *lam, int N, int i, int j,
                                        int k, double ih2, double *diag)
{
    const int ip = wp(i, N), im = wm(i, N), jp = wp(j, N), jm = wm(j, N), kp = wp(k, N), km = wm(k, N);
    auto L = [&](int a, int b, int c) { return lam[offs(N, a, b, c)]; };
    auto X = [&](const double *cc, int a, int b, int c) {
        const unsigned o = offs(N, a, b, c);
        return cc[o] * lam[o];
    };
    const unsigned o = offs(N, i, j, k);
    const double dxx = X(C.xx, ip, j, k) + X(C.xx, im, j, k) - 2.0 * C.xx[o] * L(i, j, k);
    const double dyy = X(C.yy, i, jp, k) + X(C.yy, i, jm, k) - 2.0 * C.yy[o] * L(i, j, k);
    const double dzz = X(C.zz, i, j, kp) + X(C.zz, i, j, km) - 2.0 * C.zz[o] * L(i, j, k);
    const double dxy = (X(C.xy, ip, jp, k) + X(C.xy, im, jm, k)) - (X(C.xy, im, jp, k) + X(C.xy, ip, jm, k));
    const double dyz = (X(C.yz, i, jp, kp) + X(C.yz, i, jm, km)) - (X(C.yz, i, jm, kp) + X(C.yz, i, jp, km));
    const double dxz = (X(C.xz, ip, j, kp) + X(C.xz, im, j, km)) - (X(C.xz, im, j, kp) + X(C.xz, ip, j, km));
    if (diag) *diag = -2.0 * (C.xx[o] + C.yy[o] + C.zz[o]) * ih2;
    return (dxx + dyy + dzz) * ih2 + (dxy + dyz + dxz) * (0.5 * ih2);
}

// one colour pass of Gauss-Seidel on J^T lam = f (snapshot semantics)
__global__ void __launch_bounds__(kRT)
k_jt_pass(const double *__restrict__ src, double *__restrict__ dst, const double *__restrict__ f,
          const double *__restrict__ cof, int N, double ih2, int colour)
{
    const CofPtr C = cof_of(cof, (size_t)N * N * N);
    const int half = N >> 1;
    FOR_ROWS(N, i, j)
    {
        const int par = (colour + i + j) & 1;
        const unsigned base = offs(N, i, j, 0);
        for (int m = threadIdx.x; m < half; m += kRowX) {
            const int ka = 2 * m + par, kb = 2 * m + 1 - par;
            double d;
            const double jt = jt_at(C, src, N, i, j, ka, ih2, &d);
            dst[base + ka] = src[base + ka] + (f[base + ka] - jt) / d;
            dst[base + kb] = src[base + kb];
        }
    }
}

// fH = R(f - J^T lam) (8-son mean) and block partial sums of it
__global__ void __launch_bounds__(kRT)
k_jt_restrict_residual(const double *__restrict__ lam, const double *__restrict__ f,
                       const double *__restrict__ cof, int Nf, double ih2, double *__restrict__ fH,
                       double *__restrict__ partials)
{
    __shared__ double sh[32];
    const CofPtr C = cof_of(cof, (size_t)Nf * Nf * Nf);
    const int Nc = Nf >> 1;
    double s = 0.0;
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        double acc = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc) {
                    const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + cc;
                    acc += f[offs(Nf, i, j, k)] - jt_at(C, lam, Nf, i, j, k, ih2, nullptr);
                }
        const double v = acc * 0.125;
        fH[offs(Nc, I, J, K)] = v;
        s += v;
    }
    const double v = block_sum<kRT>(s, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
}

// out = sign * J^T v (v == nullptr: v = 1); partial sums of out^2 (col 1)
// and of (f - out)^2 when f is given (col 1 then holds the residual norm)
__global__ void __launch_bounds__(kRT)
k_jt_apply(const double *__restrict__ v, const double *__restrict__ f, const double *__restrict__ cof,
           int N, double ih2, double sign, double *__restrict__ out, double *__restrict__ partials)
{
    __shared__ double sh[32];
    const CofPtr C = cof_of(cof, (size_t)N * N * N);
    double s2 = 0.0;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        double r;
        if (v) {
            r = sign * jt_at(C, v, N, i, j, k, ih2, nullptr);
        } else {
            // J^T 1 = sum_ab D_ab adj_ab
            const int ip = wp(i, N), im = wm(i, N), jp = wp(j, N), jm = wm(j, N), kp = wp(k, N), km = wm(k, N);
            auto c = [&](const double *a, int x, int y, int z) { return a[offs(N, x, y, z)]; };
            const unsigned o = offs(N, i, j, k);
            const double d = (c(C.xx, ip, j, k) + c(C.xx, im, j, k) - 2.0 * C.xx[o]) +
                             (c(C.yy, i, jp, k) + c(C.yy, i, jm, k) - 2.0 * C.yy[o]) +
                             (c(C.zz, i, j, kp) + c(C.zz, i, j, km) - 2.0 * C.zz[o]);
            const double m = ((c(C.xy, ip, jp, k) + c(C.xy, im, jm, k)) - (c(C.xy, im, jp, k) + c(C.xy, ip, jm, k))) +
                             ((c(C.yz, i, jp, kp) + c(C.yz, i, jm, km)) - (c(C.yz, i, jm, kp) + c(C.yz, i, jp, km))) +
                             ((c(C.xz, ip, j, kp) + c(C.xz, im, j, km)) - (c(C.xz, im, j, kp) + c(C.xz, ip, j, km)));
            r = sign * (d * ih2 + m * (0.5 * ih2));
        }
        const unsigned id = offs(N, i, j, k);
        if (f) {
            const double e = f[id] - r;
            s2 += e * e;
        } else {
            out[id] = r;
            s2 += r * r;
        }
    }
    const double t = block_sum<kRT>(s2, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 1] = t;
}

// ---- the finest level without stored cofactors ----------------------------
// J^T applied with the cofactors of I + H phi formed in shared memory: a CTA
// streams chunks of 64 planes of the i columns of 8 x 32 (j, k) tiles (work
// items taken in turn by the CTAs of a grid of at most kMaxRedBlocks); per
// plane p it stages phi
// (tile + 2-cell halo) and lam (tile + 1), forms the six cofactors of plane
// p + 1 on the tile + 1 ring, and applies J^T at plane p.  Three barriers per
// plane; no N^3 cofactor arrays.
//   MODE 0: one colour pass of Gauss-Seidel on J^T lam = f (snapshot: out is
//           the destination array, cells of the other colour copied)
//   MODE 1: r = f - J^T lam (written to out unless out is null) and per-CTA
//           sums of r^2 (partials column 1)
//   MODE 2: out = sign * J^T 1 and per-CTA sums of out^2 (column 1)
constexpr int kFJ = 8, kFK = 32, kFT = kFJ * kFK, kFChunk = 64;
constexpr int kFPK = kFK + 4, kFPP = (kFJ + 4) * kFPK;   // phi planes
constexpr int kFCK = kFK + 2, kFCP = (kFJ + 2) * kFCK;   // cofactor / lam planes
constexpr size_t kFineSmem = sizeof(double) * (5 * kFPP + 3 * 6 * kFCP + 3 * kFCP);

template <int MODE>
__global__ void __launch_bounds__(kFT)
k_jt_fine(const double *__restrict__ phi, const double *__restrict__ lam, const double *__restrict__ f,
          double *__restrict__ out, int N, double ih2, int colour, double sign, double *__restrict__ partials)
{
    extern __shared__ double smd[];
    double *sphi = smd;                       // [5][kFPP]
    double *scof = sphi + 5 * kFPP;           // [3][6][kFCP]
    double *slam = scof + 3 * 6 * kFCP;       // [3][kFCP]
    __shared__ double sh[32];
    const int tid = threadIdx.x, tj = tid / kFK, tk = tid % kFK;
    const unsigned NN = (unsigned)N * (unsigned)N;
    const int ncols = (N / kFK) * (N / kFJ), CI = N < kFChunk ? N : kFChunk, nchunks = N / CI;
    auto wr = [&](int x) { return x < 0 ? x + N : (x >= N ? x - N : x); };
    double s2 = 0.0;
    for (int item = blockIdx.x; item < ncols * nchunks; item += gridDim.x) {
        const int col = item % ncols, i0 = (item / ncols) * CI, i1 = i0 + CI;
        const int k0 = (col % (N / kFK)) * kFK, j0 = (col / (N / kFK)) * kFJ;
        auto load_phi = [&](int p) {
            double *d = sphi + ((p + 10) % 5) * kFPP;
            const unsigned pb = (unsigned)wr(p) * NN;
            for (int e = tid; e < kFPP; e += kFT) {
                const int r = e / kFPK, c = e - r * kFPK;
                d[e] = phi[pb + (unsigned)wr(j0 - 2 + r) * (unsigned)N + (unsigned)wr(k0 - 2 + c)];
            }
        };
        auto load_lam = [&](int p) {
            if (MODE == 2) return;
            double *d = slam + ((p + 9) % 3) * kFCP;
            const unsigned pb = (unsigned)wr(p) * NN;
            for (int e = tid; e < kFCP; e += kFT) {
                const int r = e / kFCK, c = e - r * kFCK;
                d[e] = lam[pb + (unsigned)wr(j0 - 1 + r) * (unsigned)N + (unsigned)wr(k0 - 1 + c)];
            }
        };
        auto cof_plane = [&](int p) {   // cofactors of plane p on the tile + 1 ring (phi planes p-1..p+1 staged)
            const double *pm = sphi + ((p + 9) % 5) * kFPP, *pc = sphi + ((p + 10) % 5) * kFPP,
                         *pp = sphi + ((p + 11) % 5) * kFPP;
            double *d = scof + ((p + 9) % 3) * 6 * kFCP;
            for (int e = tid; e < kFCP; e += kFT) {
                const int r = e / kFCK, c = e - r * kFCK;
                const int o = (r + 1) * kFPK + (c + 1);
                Nb19<double> v;
                v.c = pc[o];
                v.xp = pp[o];
                v.xm = pm[o];
                v.yp = pc[o + kFPK];
                v.ym = pc[o - kFPK];
                v.zp = pc[o + 1];
                v.zm = pc[o - 1];
                v.xpyp = pp[o + kFPK];
                v.xmym = pm[o - kFPK];
                v.xmyp = pm[o + kFPK];
                v.xpym = pp[o - kFPK];
                v.ypzp = pc[o + kFPK + 1];
                v.ymzm = pc[o - kFPK - 1];
                v.ymzp = pc[o - kFPK + 1];
                v.ypzm = pc[o + kFPK - 1];
                v.xpzp = pp[o + 1];
                v.xmzm = pm[o - 1];
                v.xmzp = pm[o + 1];
                v.xpzm = pp[o - 1];
                const Cof<double> a = cofactors(v, ih2);
                d[e] = a.xx;
                d[kFCP + e] = a.yy;
                d[2 * kFCP + e] = a.zz;
                d[3 * kFCP + e] = a.xy;
                d[4 * kFCP + e] = a.yz;
                d[5 * kFCP + e] = a.xz;
            }
        };
        // prologue: phi planes i0-2..i0+1, lam planes i0-1, i0, cofactors of planes i0-1, i0
        for (int p = i0 - 2; p <= i0 + 1; ++p) load_phi(p);
        load_lam(i0 - 1);
        load_lam(i0);
        __syncthreads();
        cof_plane(i0 - 1);
        cof_plane(i0);
        for (int p = i0; p < i1; ++p) {
            __syncthreads();   // every read of the slots refilled below is done
            load_phi(p + 2);
            load_lam(p + 1);
            __syncthreads();
            cof_plane(p + 1);
            __syncthreads();
            // J^T lam at tile cell (tj, tk) of plane p
            const double *cm = scof + ((p + 8) % 3) * 6 * kFCP, *cc = scof + ((p + 9) % 3) * 6 * kFCP,
                         *cp = scof + ((p + 10) % 3) * 6 * kFCP;
            const double *lm = slam + ((p + 8) % 3) * kFCP, *lc = slam + ((p + 9) % 3) * kFCP,
                         *lp = slam + ((p + 10) % 3) * kFCP;
            const int o = (tj + 1) * kFCK + (tk + 1);
            auto X = [&](const double *cpl, const double *lpl, int comp, int off) {
                return MODE == 2 ? cpl[comp * kFCP + o + off] : cpl[comp * kFCP + o + off] * lpl[o + off];
            };
            auto jt_here = [&]() {
                const double dxx = X(cp, lp, 0, 0) + X(cm, lm, 0, 0) - 2.0 * X(cc, lc, 0, 0);
                const double dyy = X(cc, lc, 1, kFCK) + X(cc, lc, 1, -kFCK) - 2.0 * X(cc, lc, 1, 0);
                const double dzz = X(cc, lc, 2, 1) + X(cc, lc, 2, -1) - 2.0 * X(cc, lc, 2, 0);
                const double dxy =
                    (X(cp, lp, 3, kFCK) + X(cm, lm, 3, -kFCK)) - (X(cm, lm, 3, kFCK) + X(cp, lp, 3, -kFCK));
                const double dyz = (X(cc, lc, 4, kFCK + 1) + X(cc, lc, 4, -kFCK - 1)) -
                                   (X(cc, lc, 4, -kFCK + 1) + X(cc, lc, 4, kFCK - 1));
                const double dxz = (X(cp, lp, 5, 1) + X(cm, lm, 5, -1)) - (X(cm, lm, 5, 1) + X(cp, lp, 5, -1));
                return (dxx + dyy + dzz) * ih2 + (dxy + dyz + dxz) * (0.5 * ih2);
            };
            const int j = j0 + tj, k = k0 + tk;
            const unsigned id = (unsigned)p * NN + (unsigned)j * (unsigned)N + (unsigned)k;
            if (MODE == 0) {
                const double l0 = lc[o];
                if (((p + j + k) & 1) == colour) {
                    const double diag = -2.0 * (cc[o] + cc[kFCP + o] + cc[2 * kFCP + o]) * ih2;
                    out[id] = l0 + (f[id] - jt_here()) / diag;
                } else {
                    out[id] = l0;
                }
            } else if (MODE == 1) {
                const double jt = jt_here();
                const double r = f[id] - jt;
                if (out) out[id] = r;
                s2 += r * r;
            } else {
                const double v = sign * jt_here();
                out[id] = v;
                s2 += v * v;
            }
        }
        __syncthreads();   // the next column refills every slot
    }
    if (MODE != 0) {
        const double t = block_sum<kFT>(s2, sh);
        if (ltid() == 0) partials[4 * blockIdx.x + 1] = t;
    }
}

// Single-CTA Gauss-Seidel on the coarsest level (N^3 <= 4096).
__global__ void __launch_bounds__(kCoarseThreads)
k_jt_coarse(double *lam, double *work, const double *f, const double *cof, int N, double ih2,
            int max_sweeps, double rtol)
{
    __shared__ double sh[32];
    __shared__ double sval;
    const CofPtr C = cof_of(cof, (size_t)N * N * N);
    const int n = N * N * N, half = N >> 1, npairs = N * N * half;
    auto rms = [&]() -> double {
        double s2 = 0.0;
        for (int id = threadIdx.x; id < n; id += blockDim.x) {
            const int k = id % N, j = (id / N) % N, i = id / (N * N);
            const double r = f[id] - jt_at(C, lam, N, i, j, k, ih2, nullptr);
            s2 += r * r;
        }
        const double tot = block_sum<kCoarseThreads>(s2, sh);
        if (ltid() == 0) sval = sqrt(tot / n);
        __syncthreads();
        const double v = sval;
        __syncthreads();
        return v;
    };
    const double r0 = rms();
    double prev = r0;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        for (int colour = 0; colour < 2; ++colour) {
            const double *src = colour == 0 ? lam : work;
            double *dst = colour == 0 ? work : lam;
            for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
                const int m = pi % half, r = pi / half;
                const int j = r % N, i = r / N;
                const int par = (colour + i + j) & 1;
                const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                double d;
                const double jt = jt_at(C, src, N, i, j, ka, ih2, &d);
                const double vnew = src[offs(N, i, j, ka)] + (f[offs(N, i, j, ka)] - jt) / d;
                const double vcopy = src[offs(N, i, j, kb)];
                dst[offs(N, i, j, ka)] = vnew;
                dst[offs(N, i, j, kb)] = vcopy;
            }
            __syncthreads();
        }
        const double cur = rms();
        if (cur <= rtol * r0) break;
        if (rtol > 0.0 && cur >= prev) break;
        prev = cur;
    }
}

__global__ void __launch_bounds__(kThreads)
k_sub_mean(double *__restrict__ a, size_t n, const double *__restrict__ mean)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) a[id] -= *mean;
}

__global__ void __launch_bounds__(kThreads)
k_add_one(double *__restrict__ a, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) a[id] += 1.0;
}

// lam -= (s_lam / s_n) * nvec
__global__ void __launch_bounds__(kThreads)
k_null_fix(double *__restrict__ lam, const double *__restrict__ nvec, size_t n,
           const double *__restrict__ s_lam, const double *__restrict__ s_n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) lam[id] -= (*s_lam / *s_n) * nvec[id];
}

__global__ void __launch_bounds__(kThreads)
k_sum(const double *__restrict__ a, size_t n, double *__restrict__ partials)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x)
        s += a[id];
    const double v = block_sum<kThreads>(s, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
}

__global__ void __launch_bounds__(kReduceThreads)
k_reduce_col(const double *__restrict__ partials, int nb, int col, double scale, double *out)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[4 * b + col];
    v = block_sum<kReduceThreads>(v, sh);
    if (ltid() == 0) *out = v * scale;
}

inline unsigned nred(size_t n)
{
    const size_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < (size_t)kMaxRedBlocks ? (b ? b : 1) : kMaxRedBlocks);
}

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return e_;                                          \
    } while (0)

// grid of the cofactor-forming kernel: its (column, 64-plane chunk) items,
// at most kMaxRedBlocks CTAs
inline unsigned fine_grid(int N)
{
    const unsigned items = (unsigned)(N / kFK) * (unsigned)(N / kFJ) * (unsigned)(N < kFChunk ? 1 : N / kFChunk);
    return items < (unsigned)kMaxRedBlocks ? items : (unsigned)kMaxRedBlocks;
}

// level l applies J^T with cofactors formed from phi (no stored arrays)
inline bool formed(const recon_handle *H, int l) { return l == 0 && !H->adj.stored0; }

cudaError_t jt_sweep(recon_handle *H, int l, double *lam, const double *f, int sweeps)
{
    AdjWork &A = H->adj;
    const int N = H->Nl[l];
    const double ih2 = 1.0 / (H->hl[l] * H->hl[l]);
    if (formed(H, l)) {
        for (int it = 0; it < sweeps; ++it) {
            note_launch(2);
            k_jt_fine<0><<<fine_grid(N), kFT, kFineSmem, H->stream>>>(A.th[0], lam, f, H->work64, N, ih2, 0, 1.0,
                                                                     nullptr);
            k_jt_fine<0><<<fine_grid(N), kFT, kFineSmem, H->stream>>>(A.th[0], H->work64, f, lam, N, ih2, 1, 1.0,
                                                                     nullptr);
        }
        return cudaGetLastError();
    }
    for (int it = 0; it < sweeps; ++it) {
        note_launch(2);
        k_jt_pass<<<row_grid(N), row_block(), 0, H->stream>>>(lam, H->work64, f, A.cof[l], N, ih2, 0);
        k_jt_pass<<<row_grid(N), row_block(), 0, H->stream>>>(H->work64, lam, f, A.cof[l], N, ih2, 1);
    }
    return cudaGetLastError();
}

// linear V-cycle on J^T lam = f at level l (lam[l], f[l] in the workspace,
// level 0 uses the caller's arrays)
cudaError_t jt_vcycle(recon_handle *H, int l, double *lam, const double *f)
{
    AdjWork &A = H->adj;
    cudaStream_t s = H->stream;
    const recon_config &cf = H->cfg;
    const int N = H->Nl[l];
    const double ih2 = 1.0 / (H->hl[l] * H->hl[l]);
    if (l == H->nlev - 1) {
        note_launch();
        k_jt_coarse<<<1, kCoarseThreads, 0, s>>>(lam, H->work64, f, A.cof[l], N, ih2,
                                                 cf.coarse_max_sweeps, cf.coarse_rtol);
        return cudaGetLastError();
    }
    CK(jt_sweep(H, l, lam, f, cf.nu1));
    const int Nc = H->Nl[l + 1];
    const size_t nc = (size_t)Nc * Nc * Nc;
    if (formed(H, l)) {
        // r = f - J^T lam (cofactors formed from phi), then its 8-son mean
        note_launch(3);
        k_jt_fine<1><<<fine_grid(N), kFT, kFineSmem, s>>>(A.th[0], lam, f, H->work64b, N, ih2, 0, 1.0,
                                                          H->partials);
        CK(restrict_plain<double>(N, H->work64b, A.f[l + 1], s));
        k_sum<<<nred(nc), kThreads, 0, s>>>(A.f[l + 1], nc, H->partials);
        k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nred(nc), 0, 1.0 / (double)nc,
                                                  H->scal + S_ADJ_MEAN);
    } else {
        const unsigned nb = row_grid(Nc, kMaxRedBlocks);
        note_launch(2);
        k_jt_restrict_residual<<<nb, row_block(), 0, s>>>(lam, f, A.cof[l], N, ih2, A.f[l + 1], H->partials);
        k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nb, 0, 1.0 / (double)nc, H->scal + S_ADJ_MEAN);
    }
    note_launch();
    k_sub_mean<<<blocks_for(nc), kThreads, 0, s>>>(A.f[l + 1], nc, H->scal + S_ADJ_MEAN);
    CK(cudaMemsetAsync(A.lam[l + 1], 0, sizeof(double) * nc, s));
    CK(jt_vcycle(H, l + 1, A.lam[l + 1], A.f[l + 1]));
    CK(prolong_add<double>(Nc, A.lam[l + 1], (const double *)nullptr, nullptr, 1.0, lam, s));
    return jt_sweep(H, l, lam, f, cf.nu2);
}

// V-cycles on J^T lam = f (level 0) from lam = 0 until the residual drops
// below tol * ||f|| (or max_cycles).  Returns the cycle count, -1 on error.
int jt_solve(recon_handle *H, double *lam, const double *f, double tol, int max_cycles,
             double *rel_out)
{
    cudaStream_t s = H->stream;
    const int N = H->N;
    const size_t n = (size_t)N * N * N;
    const double ih2 = 1.0 / (H->h * H->h);
    const bool fm = formed(H, 0);
    const unsigned nb = fm ? fine_grid(N) : row_grid(N, kMaxRedBlocks);
    // partial sums of ||f - J^T lam||^2 (column 1)
    auto resid_norm = [&]() {
        note_launch();
        if (fm)
            k_jt_fine<1><<<nb, kFT, kFineSmem, s>>>(H->adj.th[0], lam, f, nullptr, N, ih2, 0, 1.0, H->partials);
        else
            k_jt_apply<<<nb, row_block(), 0, s>>>(lam, f, H->adj.cof[0], N, ih2, 1.0, nullptr, H->partials);
    };
    if (cudaMemsetAsync(lam, 0, sizeof(double) * n, s) != cudaSuccess) return -1;
    double fnorm2 = 0.0;
    {
        // ||f||^2 as the residual norm at lam = 0
        resid_norm();
        note_launch();
        k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nb, 1, 1.0, H->scal + S_ADJ_NORM);
        if (cudaMemcpyAsync(&H->hscal[S_ADJ_NORM], H->scal + S_ADJ_NORM, sizeof(double),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return -1;
        fnorm2 = H->hscal[S_ADJ_NORM];
    }
    const double fnorm = sqrt(fnorm2);
    if (fnorm == 0.0) {
        if (rel_out) *rel_out = 0.0;
        return 0;
    }
    int cyc = 0;
    double rel = 1.0;
    for (cyc = 1; cyc <= max_cycles; ++cyc) {
        if (jt_vcycle(H, 0, lam, f) != cudaSuccess) return -1;
        resid_norm();
        note_launch();
        k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nb, 1, 1.0, H->scal + S_ADJ_NORM);
        if (cudaMemcpyAsync(&H->hscal[S_ADJ_NORM], H->scal + S_ADJ_NORM, sizeof(double),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return -1;
        rel = sqrt(H->hscal[S_ADJ_NORM]) / fnorm;
        if (!std::isfinite(rel)) return -1;
        if (rel < tol) break;
    }
    if (rel_out) *rel_out = rel;
    return cyc > max_cycles ? max_cycles : cyc;
}

// the finest level's cofactors are formed on the fly when configured so and
// the grid tiles into the kernel's 8 x 32 columns
inline bool store0(const recon_handle *H)
{
    return H->cfg.adjoint_store_cofactors != 0 || H->N % kFK != 0 || H->N % kFJ != 0 ||
           (H->N > kFChunk && H->N % kFChunk != 0);
}

cudaError_t adj_alloc(recon_handle *H)
{
    AdjWork &A = H->adj;
    if (A.ready) return cudaSuccess;
    A.stored0 = store0(H);
    if (!A.stored0) {
        static bool attr = false;
        if (!attr) {
            CK(cudaFuncSetAttribute(k_jt_fine<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFineSmem));
            CK(cudaFuncSetAttribute(k_jt_fine<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFineSmem));
            CK(cudaFuncSetAttribute(k_jt_fine<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFineSmem));
            attr = true;
        }
    }
    for (int l = 0; l < H->nlev; ++l) {
        const size_t n = (size_t)H->Nl[l] * H->Nl[l] * H->Nl[l];
        if (l > 0) {
            CK(cudaMalloc(&A.th[l], sizeof(double) * n));
            CK(cudaMalloc(&A.lam[l], sizeof(double) * n));
            CK(cudaMalloc(&A.f[l], sizeof(double) * n));
        }
        if (l > 0 || A.stored0) CK(cudaMalloc(&A.cof[l], sizeof(double) * 6 * n));
    }
    const size_t n0 = (size_t)H->N * H->N * H->N;
    CK(cudaMalloc(&A.nvec, sizeof(double) * n0));
    CK(cudaMalloc(&A.f[0], sizeof(double) * n0));
    A.ready = true;
    return cudaSuccess;
}

}  // namespace

void adj_free(recon_handle *H)
{
    AdjWork &A = H->adj;
    for (int l = 0; l < kMaxLevels; ++l) {
        if (l > 0) {
            if (A.th[l]) cudaFree(A.th[l]);
            if (A.lam[l]) cudaFree(A.lam[l]);
        }
        if (A.f[l]) cudaFree(A.f[l]);
        if (A.cof[l]) cudaFree(A.cof[l]);
    }
    if (A.nvec) cudaFree(A.nvec);
    A = AdjWork{};
}

recon_status adjoint(recon_handle *H, const double *gbar, double *lam)
{
    cudaStream_t s = H->stream;
    AdjWork &A = H->adj;
    cudaError_t e = adj_alloc(H);
    if (e != cudaSuccess) {
        adj_free(H);
        cudaGetLastError();
        H->err = "adjoint workspace allocation failed";
        return RECON_E_OOM;
    }
    const int N = H->N;
    const size_t n = (size_t)N * N * N;
    const double tol = 1e-12;
    const int maxc = 100;
    if (A.ready && A.stored0 != store0(H)) {
        // the cofactor option changed since the workspace was made
        adj_free(H);
        if ((e = adj_alloc(H)) != cudaSuccess) {
            adj_free(H);
            cudaGetLastError();
            H->err = "adjoint workspace allocation failed";
            return RECON_E_OOM;
        }
    }
    if (!A.null_ready) {
        // cofactors of every level, from phi and its restrictions
        A.th[0] = const_cast<double *>(H->last_phi);
        for (int l = 1; l < H->nlev; ++l)
            if ((e = restrict_plain<double>(H->Nl[l - 1], A.th[l - 1], A.th[l], s)) != cudaSuccess)
                return RECON_E_CUDA;
        for (int l = A.stored0 ? 0 : 1; l < H->nlev; ++l) {
            note_launch();
            k_cof6<<<row_grid(H->Nl[l]), row_block(), 0, s>>>(A.th[l], H->Nl[l],
                                                              1.0 / (H->hl[l] * H->hl[l]), A.cof[l]);
        }
        // null vector of J^T: n = 1 + w, J^T w = -J^T 1
        note_launch();
        if (A.stored0)
            k_jt_apply<<<row_grid(N, kMaxRedBlocks), row_block(), 0, s>>>(nullptr, nullptr, A.cof[0], N,
                                                                        1.0 / (H->h * H->h), -1.0, A.f[0],
                                                                        H->partials);
        else
            k_jt_fine<2><<<fine_grid(N), kFT, kFineSmem, s>>>(A.th[0], nullptr, nullptr, A.f[0], N,
                                                              1.0 / (H->h * H->h), 0, -1.0, H->partials);
        double rel = 0.0;
        const int c1 = jt_solve(H, A.nvec, A.f[0], tol, maxc, &rel);
        if (c1 < 0) {
            H->err = "adjoint null-vector solve failed";
            return RECON_E_CUDA;
        }
        note_launch();
        k_add_one<<<blocks_for(n), kThreads, 0, s>>>(A.nvec, n);
        A.null_ready = true;
        A.null_rel = rel;
    }
    // f = gbar - mean(gbar)
    note_launch(3);
    k_sum<<<nred(n), kThreads, 0, s>>>(gbar, n, H->partials);
    k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nred(n), 0, 1.0 / (double)n, H->scal + S_ADJ_MEAN);
    if ((e = cudaMemcpyAsync(A.f[0], gbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return RECON_E_CUDA;
    k_sub_mean<<<blocks_for(n), kThreads, 0, s>>>(A.f[0], n, H->scal + S_ADJ_MEAN);
    double rel = 0.0;
    const int c2 = jt_solve(H, lam, A.f[0], tol, maxc, &rel);
    if (c2 < 0) {
        H->err = "adjoint solve failed";
        return RECON_E_CUDA;
    }
    // lam -= (sum lam / sum n) n
    note_launch(5);
    k_sum<<<nred(n), kThreads, 0, s>>>(lam, n, H->partials);
    k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nred(n), 0, 1.0, H->scal + S_ADJ_SLAM);
    k_sum<<<nred(n), kThreads, 0, s>>>(A.nvec, n, H->partials);
    k_reduce_col<<<1, kReduceThreads, 0, s>>>(H->partials, nred(n), 0, 1.0, H->scal + S_ADJ_SN);
    k_null_fix<<<blocks_for(n), kThreads, 0, s>>>(lam, A.nvec, n, H->scal + S_ADJ_SLAM, H->scal + S_ADJ_SN);
    if ((e = cudaGetLastError()) != cudaSuccess) return RECON_E_CUDA;
    if (rel >= 1e-8 || A.null_rel >= 1e-8) {
        H->err = "adjoint linear solve stalled at relative residual " + std::to_string(rel);
        return RECON_E_NOCONV;
    }
    H->adj_cycles = c2;
    H->adj_rel = rel;
    return RECON_OK;
}

}  // namespace recon
