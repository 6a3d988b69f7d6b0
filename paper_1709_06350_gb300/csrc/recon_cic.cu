// recon_cic.cu -- cloud-in-cell assignment and the reconstruction output.
//
// CIC (Sec. I footnote): along each axis u = x (N/L) - 1/2, i0 = floor(u)
// mod N, f = u - floor(u); a particle gives (1 - f, f) to cells (i0, i0+1).
// The index arithmetic uses explicitly rounded operations (no fused
// multiply-add), so cell indices and fractions are bit-identical to a plain
// IEEE evaluation of the same formula on any host.
//
// Atomics: plain FP64 atomicAdd for the density.  Warp aggregation of lanes
// that hit the same cell (__match_any_sync + shuffles) was measured slower on
// GB300 (512^3 deposit 17.5 ms aggregated vs 9.9 ms plain).  The displacement
// step accumulates its (b v, b) pair with one float2 vector atomic per corner.
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

// Deposit `val` (per thread) with CIC weights at position (x, y, z).
__device__ __forceinline__ void cic_scatter(bool active, const double xyz[3], double val, int N,
                                            double inv_h, double *__restrict__ rho)
{
    if (!active) return;
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) cic_axis(xyz[d], N, inv_h, i0[d], f[d]);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
                const int i = a ? (i0[0] + 1 == N ? 0 : i0[0] + 1) : i0[0];
                const int j = b ? (i0[1] + 1 == N ? 0 : i0[1] + 1) : i0[1];
                const int k = cc ? (i0[2] + 1 == N ? 0 : i0[2] + 1) : i0[2];
                const double w = __dmul_rn(__dmul_rn(a ? f[0] : 1.0 - f[0], b ? f[1] : 1.0 - f[1]),
                                           cc ? f[2] : 1.0 - f[2]);
                atomicAdd(rho + offs(N, i, j, k), __dmul_rn(val, w));
            }
}

// CIC of a value pair (vector atomic): acc[cell] += (v0, v1) * w.
__device__ __forceinline__ void cic_scatter2(const double xyz[3], float v0, float v1, int N,
                                             double inv_h, float2 *__restrict__ acc)
{
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) cic_axis(xyz[d], N, inv_h, i0[d], f[d]);
    const float fx = (float)f[0], fy = (float)f[1], fz = (float)f[2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int cc = 0; cc < 2; ++cc) {
                const int i = a ? (i0[0] + 1 == N ? 0 : i0[0] + 1) : i0[0];
                const int j = b ? (i0[1] + 1 == N ? 0 : i0[1] + 1) : i0[1];
                const int k = cc ? (i0[2] + 1 == N ? 0 : i0[2] + 1) : i0[2];
                const float w = (a ? fx : 1.0f - fx) * (b ? fy : 1.0f - fy) * (cc ? fz : 1.0f - fz);
                atomicAdd(acc + offs(N, i, j, k), make_float2(v0 * w, v1 * w));
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
    cic_scatter(active, xyz, mass, N, inv_h, rho);   // inactive lanes return at once
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
// Per Eulerian cell x_c: psi = -grad phi (central differences, FP64), the
// mapped Lagrangian position q = x + grad phi (mod L, FP64), and
// v = 3 - tr((I + H)^-1) computed in FP32 from the FP64 Hessian; the pair
// (b v, b) is accumulated at q with FP32 CIC weights (vector atomics).
// delta_r = sum(b v) / max(sum(b), 1e-12) then carries FP32 rounding
// (~1e-6 absolute for |delta_r| < 3).
__global__ void __launch_bounds__(kRowX * kRowY)
k_displace_cells(const double *__restrict__ t, const double *__restrict__ b, int N, double L,
                 double h, double ih2, double *__restrict__ psi, float2 *__restrict__ acc)
{
    const unsigned n = (unsigned)N * N * N;
    const double inv_h = (double)N / L, inv_2h = 0.5 / h;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const unsigned id = offs(N, i, j, k);
        const Nb19<double> nb = load19<double>(t, N, i, j, k);
        // central gradient; a multiply by 1/(2h) (within 1 ulp of the quotient)
        const double g[3] = {(nb.xp - nb.xm) * inv_2h, (nb.yp - nb.ym) * inv_2h,
                             (nb.zp - nb.zm) * inv_2h};
        const double x[3] = {__dmul_rn(i + 0.5, h), __dmul_rn(j + 0.5, h), __dmul_rn(k + 0.5, h)};
        double q[3];
        for (int d = 0; d < 3; ++d) {
            psi[(size_t)d * n + id] = -g[d];
            // q mod L: for q in (-L, 2L) the conditional form gives exactly
            // fmod's result (q - L is exact there); fmod handles the rest
            double qq = __dadd_rn(x[d], g[d]);
            if (qq >= L) qq = qq < 2.0 * L ? __dsub_rn(qq, L) : fmod(qq, L);
            else if (qq <= -L) qq = fmod(qq, L);
            if (qq < 0.0) qq = __dadd_rn(qq, L);
            q[d] = qq;
        }
        // Hessian in FP64 (differences of phi), the rest in FP32
        const float axx = (float)(1.0 + ((nb.xp + nb.xm) - 2.0 * nb.c) * ih2);
        const float ayy = (float)(1.0 + ((nb.yp + nb.ym) - 2.0 * nb.c) * ih2);
        const float azz = (float)(1.0 + ((nb.zp + nb.zm) - 2.0 * nb.c) * ih2);
        const float hxy = (float)(((nb.xpyp + nb.xmym) - (nb.xmyp + nb.xpym)) * (0.25 * ih2));
        const float hyz = (float)(((nb.ypzp + nb.ymzm) - (nb.ymzp + nb.ypzm)) * (0.25 * ih2));
        const float hxz = (float)(((nb.xpzp + nb.xmzm) - (nb.xmzp + nb.xpzm)) * (0.25 * ih2));
        const float cxx = ayy * azz - hyz * hyz, cyy = axx * azz - hxz * hxz, czz = axx * ayy - hxy * hxy;
        const float D = axx * cxx - hxy * (hxy * azz - hyz * hxz) + hxz * (hxy * hyz - ayy * hxz);
        const float v = 3.0f - (cxx + cyy + czz) / D;
        const float bb = (float)b[id];
        cic_scatter2(q, bb * v, bb, N, inv_h, acc);
    }
}

__global__ void __launch_bounds__(kThreads)
k_displace_finish(const float2 *__restrict__ acc, size_t n, double *__restrict__ out)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) {
        const float2 a = acc[id];
        const double den = (double)a.y;
        out[id] = (double)a.x / (den > 1e-12 ? den : 1e-12);
    }
}

cudaError_t displace(int N, double L, const double *phi, const double *b, double *psi,
                     double *deltaL, double *scratch, cudaStream_t s)
{
    const size_t n = (size_t)N * N * N;
    const double h = L / N;
    float2 *acc = reinterpret_cast<float2 *>(scratch);   // N^3 float2 = N^3 doubles of room
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float2) * n, s);
    if (e != cudaSuccess) return e;
    note_launch(2);
    k_displace_cells<<<row_grid(N), row_block(), 0, s>>>(phi, b, N, L, h, 1.0 / (h * h), psi, acc);
    k_displace_finish<<<blocks_for(n), kThreads, 0, s>>>(acc, n, deltaL);
    return cudaGetLastError();
}

}  // namespace recon
