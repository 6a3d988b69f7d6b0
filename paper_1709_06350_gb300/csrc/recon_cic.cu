// recon_cic.cu -- cloud-in-cell assignment and the reconstruction output.
//
// CIC (Sec. I footnote): along each axis u = x (N/L) - 1/2, i0 = floor(u)
// mod N, f = u - floor(u); a particle gives (1 - f, f) to cells (i0, i0+1).
// The index arithmetic uses explicitly rounded operations (no fused
// multiply-add), so cell indices and fractions are bit-identical to a plain
// IEEE evaluation of the same formula on any host.
//
// Atomics: neighbouring threads handle neighbouring particles (or cells),
// which often land in the same target cells; lanes of a warp that target
// the same cell first combine their contributions (__match_any_sync +
// shuffles) and one lane issues the atomicAdd.
#include <cmath>

#include "cellmath.cuh"
#include "internal.cuh"

namespace recon {

__device__ __forceinline__ void cic_axis(double x, int N, double inv_h, int &i0, double &f)
{
    const double u = __dsub_rn(__dmul_rn(x, inv_h), 0.5);
    const double fl = floor(u);
    f = __dsub_rn(u, fl);
    long long ii = (long long)fl % (long long)N;
    if (ii < 0) ii += N;
    i0 = (int)ii;
}

// Sum `v` over the lanes of the warp that share `key`; the lowest such lane
// gets the total and true, the others false.  Every lane must call this.
__device__ __forceinline__ bool warp_aggregate(unsigned key, double &v)
{
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    double tot = 0.0;
    for (unsigned m = peers; m; m &= m - 1) tot += __shfl_sync(peers, v, __ffs(m) - 1);
    v = tot;
    return lane == __ffs(peers) - 1;
}

// Deposit `val` (per thread) with CIC weights at position (x, y, z).
__device__ __forceinline__ void cic_scatter(bool active, const double xyz[3], double val, int N,
                                            double inv_h, double *__restrict__ rho)
{
    int i0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    if (active)
        for (int d = 0; d < 3; ++d) cic_axis(xyz[d], N, inv_h, i0[d], f[d]);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
                const int i = a ? (i0[0] + 1 == N ? 0 : i0[0] + 1) : i0[0];
                const int j = b ? (i0[1] + 1 == N ? 0 : i0[1] + 1) : i0[1];
                const int k = cc ? (i0[2] + 1 == N ? 0 : i0[2] + 1) : i0[2];
                const double w = __dmul_rn(__dmul_rn(a ? f[0] : 1.0 - f[0], b ? f[1] : 1.0 - f[1]),
                                           cc ? f[2] : 1.0 - f[2]);
                double v = active ? __dmul_rn(val, w) : 0.0;
                const unsigned key = active ? offs(N, i, j, k) : 0xffffffffu;
                if (warp_aggregate(key, v) && active) atomicAdd(rho + offs(N, i, j, k), v);
            }
}

__global__ void __launch_bounds__(kThreads)
k_cic_deposit(const double *__restrict__ pos, long long n, int N, double inv_h, double mass,
              double *__restrict__ rho)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < n;
    double xyz[3] = {0.0, 0.0, 0.0};
    if (active)
        for (int d = 0; d < 3; ++d) xyz[d] = pos[3 * p + d];
    cic_scatter(active, xyz, mass, N, inv_h, rho);
}

__global__ void __launch_bounds__(kThreads)
k_cic_cells(const double *__restrict__ pos, long long n, int N, double inv_h,
            int *__restrict__ cells, double *__restrict__ frac)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int d = 0; d < 3; ++d) cic_axis(pos[3 * p + d], N, inv_h, cells[3 * p + d], frac[3 * p + d]);
}

cudaError_t cic_cells(const double *pos, long long n, int N, double L, int *cells,
                      double *frac, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    note_launch();
    k_cic_cells<<<blocks_for((size_t)n), kThreads, 0, s>>>(pos, n, N, (double)N / L, cells, frac);
    return cudaGetLastError();
}

cudaError_t cic_deposit(const double *pos, long long n, int N, double L, double mass,
                        double *rho, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    note_launch();
    k_cic_deposit<<<blocks_for((size_t)n), kThreads, 0, s>>>(pos, n, N, (double)N / L, mass, rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- displace
// Per Eulerian cell x_c: psi = -grad phi (central differences), the mapped
// Lagrangian position q = x + grad phi (mod L), v = 3 - tr((I + H)^-1), and
// CIC deposits of b v (numerator) and b (denominator) at q.
__global__ void __launch_bounds__(kRowX * kRowY)
k_displace_cells(const double *__restrict__ t, const double *__restrict__ b, int N, double L,
                 double h, double ih2, double *__restrict__ psi, double *__restrict__ num,
                 double *__restrict__ den)
{
    const unsigned n = (unsigned)N * N * N;
    const double inv_h = (double)N / L;
    FOR_ROWS(N, i, j)
    for (int k0 = 0; k0 < N; k0 += kRowX) {   // uniform trip count: every lane
        const int k = k0 + threadIdx.x;        // takes part in the aggregation
        const bool active = k < N;
        double q[3] = {0.0, 0.0, 0.0};
        double wv = 0.0, wb = 0.0;
        if (active) {
            const unsigned id = offs(N, i, j, k);
            const Nb19<double> nb = load19<double>(t, N, i, j, k);
            const double g[3] = {(nb.xp - nb.xm) / (2.0 * h), (nb.yp - nb.ym) / (2.0 * h),
                                 (nb.zp - nb.zm) / (2.0 * h)};
            // explicitly rounded so that q (and hence its CIC cell) does not
            // depend on multiply-add contraction
            const double x[3] = {__dmul_rn(i + 0.5, h), __dmul_rn(j + 0.5, h), __dmul_rn(k + 0.5, h)};
            for (int d = 0; d < 3; ++d) {
                psi[(size_t)d * n + id] = -g[d];
                // q mod L: for q in (-L, 2L) the conditional form gives exactly
                // fmod's result (q - L is exact there); fmod handles the rest
                double qq = __dadd_rn(x[d], g[d]);
                if (qq >= L) qq = qq < 2.0 * L ? __dsub_rn(qq, L) : fmod(qq, L);
                else if (qq < 0.0 && qq <= -L) qq = fmod(qq, L);
                if (qq < 0.0) qq = __dadd_rn(qq, L);
                q[d] = qq;
            }
            const Cof<double> a = cofactors(nb, ih2);
            const double D = det_IH(nb, ih2);
            const double v = 3.0 - (a.xx + a.yy + a.zz) / D;
            wb = b[id];
            wv = wb * v;
        }
        cic_scatter(active, q, wv, N, inv_h, num);
        cic_scatter(active, q, wb, N, inv_h, den);
    }
}

__global__ void __launch_bounds__(kThreads)
k_displace_finish(const double *__restrict__ num, const double *__restrict__ den, size_t n,
                  double *__restrict__ out)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) out[id] = num[id] / (den[id] > 1e-12 ? den[id] : 1e-12);
}

cudaError_t displace(int N, double L, const double *phi, const double *b, double *psi,
                     double *deltaL, double *num, double *den, cudaStream_t s)
{
    const size_t n = (size_t)N * N * N;
    const double h = L / N;
    cudaError_t e = cudaMemsetAsync(num, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(den, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) return e;
    note_launch();
    k_displace_cells<<<row_grid(N), row_block(), 0, s>>>(phi, b, N, L, h, 1.0 / (h * h), psi, num, den);
    note_launch();
    k_displace_finish<<<blocks_for(n), kThreads, 0, s>>>(num, den, n, deltaL);
    return cudaGetLastError();
}

}  // namespace recon
