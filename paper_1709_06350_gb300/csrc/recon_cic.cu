// recon_cic.cu -- cloud-in-cell assignment and the reconstruction output.
//
// CIC (Sec. I footnote): along each axis u = x (N/L) - 1/2, i0 = floor(u)
// mod N, f = u - floor(u); a particle gives (1 - f, f) to cells (i0, i0+1).
// The index arithmetic uses explicitly rounded operations (no fused
// multiply-add), so cell indices and fractions are bit-identical to a plain
// IEEE evaluation of the same formula on any host.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, so both kernels keep FP64
// arithmetic to what an FP64 result needs: the deposit forms u in FP64 and
// does the rest (floor, fraction, corner weights) in 64-bit fixed point on
// the integer pipes; the displacement forms psi in FP64 and the rest from
// FP32 parts of phi.  Atomics: FP64 for the density, one float2 vector
// atomic per corner for the displacement's (b v, b) pair; lanes that hold
// consecutive particles (cells) merge shared z corners first.
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

// Cell and fraction of u = x N/L - 1/2 in 64-bit fixed point, from the bits
// of u (integer pipes only): i0 = floor(u) (mod N), f = (u - floor(u)) 2^64.
// Exact for u in (-1, 2^31); returns false outside (the caller then uses
// the FP64 form).
__device__ __forceinline__ bool cic_fixed(double u, int N, int &i0, unsigned long long &f)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
    const int e = (int)((bits >> 52) & 0x7ff);
    const unsigned long long m = (bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    const int sh = 1075 - e;   // fractional bits of the 53-bit integer m
    if (e == 0) {              // +-0 or subnormal: cell 0, fraction ~0
        i0 = 0;
        f = 0;
        return true;
    }
    if (sh <= 22) return false;   // |u| >= 2^31
    unsigned long long ip, fr;
    if (sh < 64) {
        ip = m >> sh;
        fr = (m & ((1ull << sh) - 1)) << (64 - sh);
    } else {
        ip = 0;
        fr = sh - 64 < 64 ? m >> (sh - 64) : 0;
    }
    if (bits >> 63) {   // u < 0: floor = -1 and fraction 1 - |u| for |u| < 1
        if (ip != 0 || fr == 0) return false;
        i0 = N - 1;
        f = 0ull - fr;
        return true;
    }
    i0 = (int)(ip < (unsigned long long)N ? ip : ip % (unsigned long long)N);
    f = fr;
    return true;
}

// Cell and fraction of u = x 2^k - 1/2 when N/L = 2^k (k = pow2): x 2^k is
// exact, so floor(u) and u - floor(u) follow from the bits of x in 64-bit
// fixed point with no FP64 instruction.  The FP64 evaluation of u rounds
// x 2^k - 1/2 only when it is not representable, i.e. for 0 < x 2^k < 1/4 by
// less than 2^-53: the same cell, a fraction within 2^-53.  Returns false for
// x < 0 and x 2^k >= 2^31 (the caller then uses the FP64 form).
constexpr int kNoPow2 = -100000;
__device__ __forceinline__ bool cic_fixed_pow2(double x, int k, int N, int &i0, unsigned long long &f)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    if (bits >> 63) return false;
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0) {              // +0 or subnormal: u = -1/2 (+ a subnormal)
        i0 = N - 1;
        f = 1ull << 63;
        return true;
    }
    const int sh = 1075 - (e + k);   // fractional bits of the 53-bit m at the exponent of x 2^k
    if (sh <= 22) return false;      // x 2^k >= 2^31
    const unsigned long long m = (bits & 0xfffffffffffffull) | (1ull << 52);
    unsigned long long ip, fr;
    if (sh < 64) {
        ip = m >> sh;
        fr = (m & ((1ull << sh) - 1)) << (64 - sh);
    } else {
        ip = 0;
        fr = sh - 64 < 64 ? m >> (sh - 64) : 0;
    }
    if (fr >= (1ull << 63)) {        // u = X - 1/2 keeps the integer part
        f = fr - (1ull << 63);
        i0 = (int)(ip < (unsigned long long)N ? ip : ip % (unsigned long long)N);
    } else {                         // borrows one
        f = fr + (1ull << 63);
        const unsigned long long im = ip == 0 ? (unsigned long long)N - 1 : ip - 1;
        i0 = (int)(im < (unsigned long long)N ? im : im % (unsigned long long)N);
    }
    return true;
}

// (a b) / 2^63 for 63-bit fixed-point weights a, b in [0, 2^63]
__device__ __forceinline__ unsigned long long mul63(unsigned long long a, unsigned long long b)
{
    return (__umul64hi(a, b) << 1) | ((a * b) >> 63);
}

// a 63-bit fixed-point weight w (w / 2^63 in [0, 1]) as a double (truncated
// to 53 bits), assembled on the integer pipes
__device__ __forceinline__ double fixed63_to_double(unsigned long long w)
{
    if (w == 0) return 0.0;
    const int lz = __clzll((long long)w);
    const unsigned long long mant = (w << lz) >> 11;   // 53 bits, leading one at bit 52
    return __longlong_as_double((long long)(((unsigned long long)(1023 - lz) << 52) |
                                            (mant & 0xfffffffffffffull)));
}

// a 62-bit fixed-point value w (w / 2^62 in [0, 2]) as a double (truncated
// to 53 bits)
__device__ __forceinline__ double fixed62_to_double(unsigned long long w)
{
    if (w == 0) return 0.0;
    const int lz = __clzll((long long)w);
    const unsigned long long mant = (w << lz) >> 11;
    return __longlong_as_double((long long)(((unsigned long long)(1024 - lz) << 52) |
                                            (mant & 0xfffffffffffffull)));
}

// Warp-neighbour merge of a CIC z pair.  Lanes hold consecutive particles
// (or cells) whose z targets are usually consecutive too: when lane L's
// upper target t1 is lane L+1's lower target t0 (same (x, y) corner row),
// lane L+1 adds lane L's value to its own and one atomic serves both.  All
// 32 lanes must call this (inactive lanes pass the kNoCell targets).
constexpr unsigned kNoCell = 0xffffffffu, kNoCell0 = 0xfffffffeu;
__device__ __forceinline__ double shfl_up_v(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float2 shfl_up_v(float2 v)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ double add_v(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add_v(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

template <typename V>
__device__ __forceinline__ void zpair_add(V *__restrict__ acc, unsigned t0, unsigned t1, V v0, V v1,
                                          bool active)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned up_t1 = __shfl_up_sync(0xffffffffu, t1, 1);
    const unsigned dn_t0 = __shfl_down_sync(0xffffffffu, t0, 1);
    const V up_v1 = shfl_up_v(v1);
    const bool take = lane > 0 && up_t1 == t0;
    const bool give = lane < 31 && dn_t0 == t1;
    if (active) {
        atomicAdd(acc + t0, take ? add_v(v0, up_v1) : v0);
        if (!give) atomicAdd(acc + t1, v1);
    }
}

// The merge for unit mass on 63-bit fixed-point corner weights: the two
// weights of a shared corner are added as integers (halved to 62 bits, so the
// sum cannot overflow) and converted to double once.
__device__ __forceinline__ void zpair_add_fixed(double *__restrict__ acc, unsigned t0, unsigned t1,
                                                unsigned long long w0, unsigned long long w1, bool active)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned up_t1 = __shfl_up_sync(0xffffffffu, t1, 1);
    const unsigned dn_t0 = __shfl_down_sync(0xffffffffu, t0, 1);
    const unsigned long long a0 = w0 >> 1, a1 = w1 >> 1;
    const unsigned long long up_a1 = __shfl_up_sync(0xffffffffu, a1, 1);
    const bool take = lane > 0 && up_t1 == t0;
    const bool give = lane < 31 && dn_t0 == t1;
    if (active) {
        atomicAdd(acc + t0, fixed62_to_double(take ? a0 + up_a1 : a0));
        if (!give) atomicAdd(acc + t1, fixed62_to_double(a1));
    }
}

// Deposit `val` with CIC weights at position (x, y, z) (inactive lanes take
// part in the merge with no targets).  u is formed in FP64 with the two
// roundings of the definition; the fraction, the corner weights
// (w_x w_y) w_z and their conversion to double are 64-bit fixed point,
// within ~1e-16 of the FP64 products.  val == 1 needs no multiply.
__device__ __forceinline__ void cic_scatter(bool active, const double xyz[3], double val, int N,
                                            double inv_h, int pow2, bool unit, double *__restrict__ rho)
{
    int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0};
    unsigned long long w[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (active)
        for (int d = 0; d < 3; ++d) {
            unsigned long long f;
            if (pow2 != kNoPow2 && cic_fixed_pow2(xyz[d], pow2, N, i0[d], f)) {
                // N/L = 2^pow2: no FP64 instruction
            } else if (!cic_fixed(__dsub_rn(__dmul_rn(xyz[d], inv_h), 0.5), N, i0[d], f)) {
                // far outside [0, L): the FP64 form
                double ff;
                cic_axis(xyz[d], N, inv_h, i0[d], ff);
                f = ff >= 1.0 ? ~0ull : (unsigned long long)ldexp(ff, 64);
            }
            i1[d] = i0[d] + 1 == N ? 0 : i0[d] + 1;
            w[d][1] = f >> 1;
            w[d][0] = (1ull << 63) - w[d][1];
        }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const unsigned long long wab = mul63(w[0][a], w[1][b]);
            const unsigned row = offs(N, a ? i1[0] : i0[0], b ? i1[1] : i0[1], 0);
            if (unit) {
                zpair_add_fixed(rho, active ? row + i0[2] : kNoCell0, active ? row + i1[2] : kNoCell,
                                mul63(wab, w[2][0]), mul63(wab, w[2][1]), active);
                continue;
            }
            const double c0 = fixed63_to_double(mul63(wab, w[2][0]));
            const double c1 = fixed63_to_double(mul63(wab, w[2][1]));
            zpair_add<double>(rho, active ? row + i0[2] : kNoCell0, active ? row + i1[2] : kNoCell,
                              __dmul_rn(val, c0), __dmul_rn(val, c1), active);
        }
}

__global__ void __launch_bounds__(kThreads)
k_cic_deposit(const double *__restrict__ pos, long long n, int N, double inv_h, int pow2, int unit,
              double mass, double *__restrict__ rho)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = p < n;
    double xyz[3] = {0.0, 0.0, 0.0};
    if (active)
        for (int d = 0; d < 3; ++d) xyz[d] = pos[3 * p + d];
    cic_scatter(active, xyz, mass, N, inv_h, pow2, unit != 0, rho);
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
    // N/L a power of two (h = 1 in the benchmark's boxes): the cell
    // coordinate in fixed point; unit mass: the corner merge in fixed point
    const double inv_h = (double)N / L;
    int e2 = 0;
    const double m2 = std::frexp(inv_h, &e2);
    const int pow2 = (m2 == 0.5 && e2 - 1 >= -60 && e2 - 1 <= 60) ? e2 - 1 : kNoPow2;
    k_cic_deposit<<<blocks_for((size_t)n), kThreads, 0, s>>>(pos, n, N, inv_h, pow2, mass == 1.0 ? 1 : 0, mass,
                                                            rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- NGP / TSC
// Density assignment by nearest grid point or triangular-shaped cloud
// (Sec. I footnote: the method works with NGP, CIC or TSC).  Along each
// axis u = x N/L (FP64, one rounding), i = floor(u), t = u - i from the bits
// of u; NGP puts the mass on cell i, TSC the quadratic B-spline weights
//   (1 - t)^2 / 2,  3/4 - (t - 1/2)^2,  t^2 / 2   on cells i-1, i, i+1,
// in 63-bit fixed point (the middle weight is one minus the other two,
// exactly), corner weights (w_x w_y) w_z, converted to double by bit assembly.
__device__ __forceinline__ void nearest_fixed(double x, int N, double inv_h, int &i, unsigned long long &t)
{
    const double u = __dmul_rn(x, inv_h);
    if (!cic_fixed(u, N, i, t)) {   // far outside [0, L): the FP64 form
        const double fl = floor(u);
        const double tf = u - fl;
        long long ii = (long long)fl % (long long)N;
        if (ii < 0) ii += N;
        i = (int)ii;
        t = tf >= 1.0 ? ~0ull : (unsigned long long)ldexp(tf, 64);
    }
}

__global__ void __launch_bounds__(kThreads)
k_ngp_deposit(const double *__restrict__ pos, long long n, int N, double inv_h, double mass,
              double *__restrict__ rho)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int i[3];
    for (int d = 0; d < 3; ++d) {
        unsigned long long t;
        nearest_fixed(pos[3 * p + d], N, inv_h, i[d], t);
    }
    atomicAdd(rho + offs(N, i[0], i[1], i[2]), mass);
}

__global__ void __launch_bounds__(kThreads)
k_tsc_deposit(const double *__restrict__ pos, long long n, int N, double inv_h, double mass,
              double *__restrict__ rho)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c[3][3];
    unsigned long long w[3][3];
    for (int d = 0; d < 3; ++d) {
        int i;
        unsigned long long t;
        nearest_fixed(pos[3 * p + d], N, inv_h, i, t);
        const unsigned long long t63 = t >> 1, s63 = (1ull << 63) - t63;
        w[d][0] = mul63(s63, s63) >> 1;
        w[d][2] = mul63(t63, t63) >> 1;
        w[d][1] = (1ull << 63) - w[d][0] - w[d][2];
        c[d][0] = i == 0 ? N - 1 : i - 1;
        c[d][1] = i;
        c[d][2] = i + 1 == N ? 0 : i + 1;
    }
    const bool unit = mass == 1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const unsigned long long wab = mul63(w[0][a], w[1][b]);
            const unsigned row = offs(N, c[0][a], c[1][b], 0);
            for (int cc = 0; cc < 3; ++cc) {
                const double v = fixed63_to_double(mul63(wab, w[2][cc]));
                atomicAdd(rho + row + c[2][cc], unit ? v : __dmul_rn(mass, v));
            }
        }
}

cudaError_t assign_deposit(int scheme, const double *pos, long long n, int N, double L, double mass,
                           double *rho, cudaStream_t s)
{
    if (scheme == 1) return cic_deposit(pos, n, N, L, mass, rho, s);
    if (n == 0) return cudaSuccess;
    note_launch();
    if (scheme == 0)
        k_ngp_deposit<<<blocks_for((size_t)n), kThreads, 0, s>>>(pos, n, N, (double)N / L, mass, rho);
    else
        k_tsc_deposit<<<blocks_for((size_t)n), kThreads, 0, s>>>(pos, n, N, (double)N / L, mass, rho);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- displace
// Per Eulerian cell x_c: psi = -grad phi (central differences, FP64), the
// mapped Lagrangian position q = x + grad phi (mod L), and
// v = 3 - tr((I + H)^-1); the pair (b v, b) is accumulated at q with CIC
// weights (FP32 vector atomics) and delta_r = sum(b v) / max(sum(b), 1e-12).
//
// Only psi (an FP64 output) is formed in FP64.  Everything else comes from
// phi split into FP32 parts, phi = hi + lo (|lo| <= ulp(hi)/2): the
// differences hi_n - hi_c of neighbouring values are exact in FP32
// (Sterbenz) wherever they matter, so the second differences of H and the
// CIC coordinate u = i + g/h carry one FP32 rounding of the result, not of
// phi.  The CIC cell is floor(u) = i + floor(g/h) (mod N) with fraction
// g/h - floor(g/h), the same numbers as x + g mapped through u = q/h - 1/2.
// delta_r carries FP32 rounding (~1e-6 absolute for |delta_r| < 3).
__global__ void __launch_bounds__(kRowX * kRowY)
k_displace_cells(const double *__restrict__ t, const float *__restrict__ hi,
                 const float *__restrict__ lo, const double *__restrict__ b, int N, double h,
                 float ih2, double *__restrict__ psi, float2 *__restrict__ acc)
{
    const unsigned n = (unsigned)N * N * N;
    const double inv_2h = 0.5 / h;
    FOR_ROWS(N, i, j)
    for (int kb = 0; kb < N; kb += kRowX) {   // uniform trip count: the warp merges z pairs
        const int k = kb + (int)threadIdx.x;
        const bool active = k < N;
        unsigned t0[4] = {kNoCell0, kNoCell0, kNoCell0, kNoCell0};
        unsigned t1[4] = {kNoCell, kNoCell, kNoCell, kNoCell};
        float2 v0[4], v1[4];
        if (active) {
            const unsigned id = offs(N, i, j, k);
            // psi in FP64 from the face neighbours of phi (multiply by
            // 1/(2h): within 1 ulp of the quotient)
            psi[id] = (t[offs(N, wm(i, N), j, k)] - t[offs(N, wp(i, N), j, k)]) * inv_2h;
            psi[(size_t)n + id] = (t[offs(N, i, wm(j, N), k)] - t[offs(N, i, wp(j, N), k)]) * inv_2h;
            psi[2 * (size_t)n + id] = (t[offs(N, i, j, wm(k, N))] - t[offs(N, i, j, wp(k, N))]) * inv_2h;
            // differences to the centre: exact for hi, tiny for lo
            const Nb19<float> H = load19<float>(hi, N, i, j, k);
            const Nb19<float> Lo = load19<float>(lo, N, i, j, k);
            auto d = [&](float hn, float ln) { return (hn - H.c) + (ln - Lo.c); };
            auto dd = [&](float h1, float l1, float h2, float l2) {
                return ((h1 - H.c) + (h2 - H.c)) + ((l1 + l2) - 2.0f * Lo.c);
            };
            const float q4 = 0.25f * ih2;
            const float axx = 1.0f + dd(H.xp, Lo.xp, H.xm, Lo.xm) * ih2;
            const float ayy = 1.0f + dd(H.yp, Lo.yp, H.ym, Lo.ym) * ih2;
            const float azz = 1.0f + dd(H.zp, Lo.zp, H.zm, Lo.zm) * ih2;
            const float hxy = (dd(H.xpyp, Lo.xpyp, H.xmym, Lo.xmym) - dd(H.xmyp, Lo.xmyp, H.xpym, Lo.xpym)) * q4;
            const float hyz = (dd(H.ypzp, Lo.ypzp, H.ymzm, Lo.ymzm) - dd(H.ymzp, Lo.ymzp, H.ypzm, Lo.ypzm)) * q4;
            const float hxz = (dd(H.xpzp, Lo.xpzp, H.xmzm, Lo.xmzm) - dd(H.xmzp, Lo.xmzp, H.xpzm, Lo.xpzm)) * q4;
            const float cxx = ayy * azz - hyz * hyz, cyy = axx * azz - hxz * hxz, czz = axx * ayy - hxy * hxy;
            const float D = axx * cxx - hxy * (hxy * azz - hyz * hxz) + hxz * (hxy * hyz - ayy * hxz);
            const float v = 3.0f - (cxx + cyy + czz) / D;
            // CIC coordinate along each axis: u = i + g/h, g/h = (phi_+ - phi_-) / (2 h^2)
            const float half_ih2 = 0.5f * ih2;
            const float u[3] = {(d(H.xp, Lo.xp) - d(H.xm, Lo.xm)) * half_ih2,
                                (d(H.yp, Lo.yp) - d(H.ym, Lo.ym)) * half_ih2,
                                (d(H.zp, Lo.zp) - d(H.zm, Lo.zm)) * half_ih2};
            const int own[3] = {i, j, k};
            int c0[3], c1[3];
            float f[3];
            for (int a = 0; a < 3; ++a) {
                const float fl = floorf(u[a]);
                f[a] = u[a] - fl;
                int c = own[a] + (int)fl;
                if (c < 0 || c >= N) c = ((c % N) + N) % N;
                c0[a] = c;
                c1[a] = c + 1 == N ? 0 : c + 1;
            }
            const float bb = (float)b[id];
            const float w0 = bb * v, w1 = bb;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int bq = 0; bq < 2; ++bq) {
                    const float wab = (a ? f[0] : 1.0f - f[0]) * (bq ? f[1] : 1.0f - f[1]);
                    const float wz0 = wab * (1.0f - f[2]), wz1 = wab * f[2];
                    const unsigned row = offs(N, a ? c1[0] : c0[0], bq ? c1[1] : c0[1], 0);
                    t0[2 * a + bq] = row + c0[2];
                    t1[2 * a + bq] = row + c1[2];
                    v0[2 * a + bq] = make_float2(w0 * wz0, w1 * wz0);
                    v1[2 * a + bq] = make_float2(w0 * wz1, w1 * wz1);
                }
        } else {
            for (int q = 0; q < 4; ++q) v0[q] = v1[q] = make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) zpair_add<float2>(acc, t0[q], t1[q], v0[q], v1[q], active);
    }
}

// delta_r = sum(b v) / max(sum(b), 1e-12): FP32 quotient (the sums are FP32)
__global__ void __launch_bounds__(kThreads)
k_displace_finish(const float2 *__restrict__ acc, size_t n, double *__restrict__ out)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) {
        const float2 a = acc[id];
        out[id] = (double)(a.x / fmaxf(a.y, 1e-12f));
    }
}

// ---- the reconstruction output in plain FP64, and its adjoint ----------
// Per cell c at x_c = (i + 1/2) h.  The CIC coordinate (the gradient, q and
// u below) is evaluated with explicit IEEE roundings and no fused
// multiply-add, so that the CIC cells of q match any host's bit for bit; the
// rest (A, v, the weights) is ordinary FP64 arithmetic that the compiler may
// contract into fused multiply-adds:
//   g = central-difference gradient of phi,  psi = -g,
//   q = x + g (mod L),  per axis u = q N/L - 1/2 (CIC cell and fraction),
//   A = I + H phi (stencils of eq. discrete_examples),  v = 3 - tr(A^-1),
// and delta_r = CIC(q, b v) / max(CIC(q, b), 1e-12).  This is the map whose
// gradient recon_displace_adjoint computes; recon_displace evaluates the same
// map from FP32 parts of phi (about 1e-6 of rounding in delta_r).
struct CellFwd {
    int c0[3], c1[3];   // CIC cells along each axis
    double f[3];        // CIC fractions
    double g[3];        // central-difference gradient of phi
    double ai[6];       // A^-1: xx, yy, zz, xy, yz, xz
    double v;           // 3 - tr(A^-1)
};

__device__ __forceinline__ void cell_forward64(const double *__restrict__ t, int N, double L, double h,
                                               double nl, int i, int j, int k, CellFwd &o)
{
    const double two_h = 2.0 * h;
    const int own[3] = {i, j, k};
    const double tp[3] = {t[offs(N, wp(i, N), j, k)], t[offs(N, i, wp(j, N), k)], t[offs(N, i, j, wp(k, N))]};
    const double tm[3] = {t[offs(N, wm(i, N), j, k)], t[offs(N, i, wm(j, N), k)], t[offs(N, i, j, wm(k, N))]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.g[a] = __ddiv_rn(__dsub_rn(tp[a], tm[a]), two_h);
        const double x = __dmul_rn(__dadd_rn((double)own[a], 0.5), h);
        double q = fmod(__dadd_rn(x, o.g[a]), L);
        if (q < 0.0) q = __dadd_rn(q, L);
        cic_axis(q, N, nl, o.c0[a], o.f[a]);
        o.c1[a] = o.c0[a] + 1 == N ? 0 : o.c0[a] + 1;
    }
    const Nb19<double> n = load19<double>(t, N, i, j, k);
    const double h2 = h * h, q4 = 4.0 * h2;
    const double axx = 1.0 + ((n.xp + n.xm) - 2.0 * n.c) / h2;
    const double ayy = 1.0 + ((n.yp + n.ym) - 2.0 * n.c) / h2;
    const double azz = 1.0 + ((n.zp + n.zm) - 2.0 * n.c) / h2;
    const double axy = (((n.xpyp + n.xmym) - n.xmyp) - n.xpym) / q4;
    const double ayz = (((n.ypzp + n.ymzm) - n.ymzp) - n.ypzm) / q4;
    const double axz = (((n.xpzp + n.xmzm) - n.xmzp) - n.xpzm) / q4;
    // adj(A) and det(A) (first-row expansion)
    const double cxx = ayy * azz - ayz * ayz, cyy = axx * azz - axz * axz, czz = axx * ayy - axy * axy;
    const double cxy = axz * ayz - axy * azz, cyz = axy * axz - axx * ayz, cxz = axy * ayz - axz * ayy;
    const double det = axx * cxx + axy * cxy + axz * cxz;
    o.v = 3.0 - (cxx + cyy + czz) / det;
    const double id = 1.0 / det;
    o.ai[0] = cxx * id;
    o.ai[1] = cyy * id;
    o.ai[2] = czz * id;
    o.ai[3] = cxy * id;
    o.ai[4] = cyz * id;
    o.ai[5] = cxz * id;
}

// CIC weight of corner (a, bq, cz) and its derivative along each axis of q
// (d f / d q = 1 / h, the lower corner weighs 1 - f)
__device__ __forceinline__ double corner_w(const double f[3], int a, int bq, int cz)
{
    return ((a ? f[0] : 1.0 - f[0]) * (bq ? f[1] : 1.0 - f[1])) * (cz ? f[2] : 1.0 - f[2]);
}

// psi (if non-null) and the CIC sums num = sum b v W, den = sum b W (FP64
// atomics; num and den start at zero)
__global__ void __launch_bounds__(kRowX * kRowY)
k_disp64_deposit(const double *__restrict__ t, const double *__restrict__ b, int N, double L,
                 double h, double nl, double *__restrict__ psi, double *__restrict__ num,
                 double *__restrict__ den)
{
    const size_t n = (size_t)N * N * N;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        CellFwd o;
        cell_forward64(t, N, L, h, nl, i, j, k, o);
        const unsigned id = offs(N, i, j, k);
        if (psi) {
            psi[id] = -o.g[0];
            psi[n + id] = -o.g[1];
            psi[2 * n + id] = -o.g[2];
        }
        const double wb = b[id], wv = wb * o.v;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int bq = 0; bq < 2; ++bq)
#pragma unroll
                for (int cz = 0; cz < 2; ++cz) {
                    const double W = corner_w(o.f, a, bq, cz);
                    const unsigned c = offs(N, a ? o.c1[0] : o.c0[0], bq ? o.c1[1] : o.c0[1], cz ? o.c1[2] : o.c0[2]);
                    atomicAdd(num + c, wv * W);
                    atomicAdd(den + c, wb * W);
                }
    }
}

__global__ void __launch_bounds__(kThreads)
k_disp64_finish(const double *__restrict__ num, const double *__restrict__ den, size_t n,
                double *__restrict__ out)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) out[id] = num[id] / (den[id] > 1e-12 ? den[id] : 1e-12);
}

// adjoint of the quotient, in place: num <- gbar / max(den, eps),
// den <- -gbar num / den^2 where den > eps (else 0)
__global__ void __launch_bounds__(kThreads)
k_dadj_quot(double *__restrict__ num, double *__restrict__ den, const double *__restrict__ gdl, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) {
        const double d = den[id], nm = num[id], gd = gdl[id];
        num[id] = gd / (d > 1e-12 ? d : 1e-12);
        den[id] = d > 1e-12 ? (-gd * nm) / (d * d) : 0.0;
    }
}

// per cell: gbar_b, and the nine fields the potential's gradient is built
// from -- gv (A^-2)_ab (xx, yy, zz, xy, yz, xz) and gq_d - gbar_psi_d -- in
// G9 = [9][N^3].  gN, gD: the quotient adjoint on the q-grid (null: no
// delta_r term); gpsi: [3][N^3] or null.
__global__ void __launch_bounds__(kRowX * kRowY)
k_dadj_cells(const double *__restrict__ t, const double *__restrict__ b, const double *__restrict__ gN,
             const double *__restrict__ gD, const double *__restrict__ gpsi, int N, double L, double h,
             double nl, double *__restrict__ gb_out, double *__restrict__ G9)
{
    const size_t n = (size_t)N * N * N;
    const double ih = 1.0 / h;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        CellFwd o;
        cell_forward64(t, N, L, h, nl, i, j, k, o);
        const unsigned id = offs(N, i, j, k);
        const double wb = b[id], wv = wb * o.v;
        double gwv = 0.0, gwb = 0.0, gq[3] = {0.0, 0.0, 0.0};
        if (gN) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int bq = 0; bq < 2; ++bq)
#pragma unroll
                    for (int cz = 0; cz < 2; ++cz) {
                        const double w0 = a ? o.f[0] : 1.0 - o.f[0];
                        const double w1 = bq ? o.f[1] : 1.0 - o.f[1];
                        const double w2 = cz ? o.f[2] : 1.0 - o.f[2];
                        const double s0 = a ? ih : -ih, s1 = bq ? ih : -ih, s2 = cz ? ih : -ih;
                        const unsigned c = offs(N, a ? o.c1[0] : o.c0[0], bq ? o.c1[1] : o.c0[1], cz ? o.c1[2] : o.c0[2]);
                        const double n_c = gN[c], d_c = gD[c];
                        const double W = (w0 * w1) * w2;
                        gwv += n_c * W;
                        gwb += d_c * W;
                        const double e = wv * n_c + wb * d_c;
                        gq[0] += e * (s0 * w1 * w2);
                        gq[1] += e * (w0 * s1 * w2);
                        gq[2] += e * (w0 * w1 * s2);
                    }
        }
        gb_out[id] = gwv * o.v + gwb;
        const double gv = gwv * wb;
        // (A^-1)^2, symmetric
        const double *m = o.ai;   // xx, yy, zz, xy, yz, xz
        const double sxx = m[0] * m[0] + m[3] * m[3] + m[5] * m[5];
        const double syy = m[3] * m[3] + m[1] * m[1] + m[4] * m[4];
        const double szz = m[5] * m[5] + m[4] * m[4] + m[2] * m[2];
        const double sxy = m[0] * m[3] + m[3] * m[1] + m[5] * m[4];
        const double syz = m[3] * m[5] + m[1] * m[4] + m[4] * m[2];
        const double sxz = m[0] * m[5] + m[3] * m[4] + m[5] * m[2];
        G9[id] = gv * sxx;
        G9[n + id] = gv * syy;
        G9[2 * n + id] = gv * szz;
        G9[3 * n + id] = gv * sxy;
        G9[4 * n + id] = gv * syz;
        G9[5 * n + id] = gv * sxz;
#pragma unroll
        for (int a = 0; a < 3; ++a) G9[(6 + a) * n + id] = gq[a] - (gpsi ? gpsi[a * n + id] : 0.0);
    }
}

// gbar_phi = sum_a D_aa(G_aa) + 2 sum_{a<b} D_ab(G_ab) - sum_d D_d(Y_d): the
// second-difference stencils are self-adjoint, the central difference is
// anti-self-adjoint (periodic grid)
__global__ void __launch_bounds__(kRowX * kRowY)
k_dadj_theta(const double *__restrict__ G9, int N, double h, double *__restrict__ out)
{
    const size_t n = (size_t)N * N * N;
    const double ih2 = 1.0 / (h * h), iq4 = 1.0 / (4.0 * h * h), i2h = 1.0 / (2.0 * h);
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const int ip = wp(i, N), im = wm(i, N), jp = wp(j, N), jm = wm(j, N), kp = wp(k, N), km = wm(k, N);
        const double *Gxx = G9, *Gyy = G9 + n, *Gzz = G9 + 2 * n;
        const double *Gxy = G9 + 3 * n, *Gyz = G9 + 4 * n, *Gxz = G9 + 5 * n;
        const double *Yx = G9 + 6 * n, *Yy = G9 + 7 * n, *Yz = G9 + 8 * n;
        const unsigned c = offs(N, i, j, k);
        double r = ((Gxx[offs(N, ip, j, k)] + Gxx[offs(N, im, j, k)]) - 2.0 * Gxx[c]) * ih2;
        r += ((Gyy[offs(N, i, jp, k)] + Gyy[offs(N, i, jm, k)]) - 2.0 * Gyy[c]) * ih2;
        r += ((Gzz[offs(N, i, j, kp)] + Gzz[offs(N, i, j, km)]) - 2.0 * Gzz[c]) * ih2;
        r += 2.0 * (((Gxy[offs(N, ip, jp, k)] + Gxy[offs(N, im, jm, k)]) - Gxy[offs(N, im, jp, k)]) - Gxy[offs(N, ip, jm, k)]) * iq4;
        r += 2.0 * (((Gyz[offs(N, i, jp, kp)] + Gyz[offs(N, i, jm, km)]) - Gyz[offs(N, i, jm, kp)]) - Gyz[offs(N, i, jp, km)]) * iq4;
        r += 2.0 * (((Gxz[offs(N, ip, j, kp)] + Gxz[offs(N, im, j, km)]) - Gxz[offs(N, im, j, kp)]) - Gxz[offs(N, ip, j, km)]) * iq4;
        r -= (Yx[offs(N, ip, j, k)] - Yx[offs(N, im, j, k)]) * i2h;
        r -= (Yy[offs(N, i, jp, k)] - Yy[offs(N, i, jm, k)]) * i2h;
        r -= (Yz[offs(N, i, j, kp)] - Yz[offs(N, i, j, km)]) * i2h;
        out[c] = r;
    }
}

// FP64 output: num, den: N^3 doubles of scratch each
cudaError_t displace_fp64(int N, double L, const double *phi, const double *b, double *psi,
                          double *deltaL, double *num, double *den, cudaStream_t s)
{
    const size_t n = (size_t)N * N * N;
    cudaError_t e = cudaMemsetAsync(num, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(den, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) return e;
    note_launch(2);
    k_disp64_deposit<<<row_grid(N), row_block(), 0, s>>>(phi, b, N, L, L / N, (double)N / L, psi, num, den);
    k_disp64_finish<<<blocks_for(n), kThreads, 0, s>>>(num, den, n, deltaL);
    return cudaGetLastError();
}

// adjoint: num, den: N^3 doubles of scratch each; G9: 9 N^3 doubles
cudaError_t displace_adjoint(int N, double L, const double *phi, const double *b, const double *gpsi,
                             const double *gdl, double *gphi, double *gb, double *num, double *den,
                             double *G9, cudaStream_t s)
{
    const size_t n = (size_t)N * N * N;
    const double h = L / N, nl = (double)N / L;
    if (gdl) {
        cudaError_t e = cudaMemsetAsync(num, 0, sizeof(double) * n, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(den, 0, sizeof(double) * n, s);
        if (e != cudaSuccess) return e;
        note_launch(2);
        k_disp64_deposit<<<row_grid(N), row_block(), 0, s>>>(phi, b, N, L, h, nl, nullptr, num, den);
        k_dadj_quot<<<blocks_for(n), kThreads, 0, s>>>(num, den, gdl, n);
    }
    note_launch(2);
    k_dadj_cells<<<row_grid(N), row_block(), 0, s>>>(phi, b, gdl ? num : nullptr, gdl ? den : nullptr, gpsi,
                                                    N, L, h, nl, gb, G9);
    k_dadj_theta<<<row_grid(N), row_block(), 0, s>>>(G9, N, h, gphi);
    return cudaGetLastError();
}

// scratch: N^3 doubles of room (the float2 sums); split: N^3 doubles of
// room for the FP32 parts of phi
cudaError_t displace(int N, double L, const double *phi, const double *b, double *psi,
                     double *deltaL, double *scratch, double *split, cudaStream_t s)
{
    const size_t n = (size_t)N * N * N;
    const double h = L / N;
    float2 *acc = reinterpret_cast<float2 *>(scratch);
    float *hi = reinterpret_cast<float *>(split), *lo = hi + n;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float2) * n, s);
    if (e != cudaSuccess) return e;
    note_launch(3);
    k_split_df<<<blocks_for(n), kThreads, 0, s>>>(phi, hi, lo, n);
    k_displace_cells<<<row_grid(N), row_block(), 0, s>>>(phi, hi, lo, b, N, h, (float)(1.0 / (h * h)),
                                                        psi, acc);
    k_displace_finish<<<blocks_for(n), kThreads, 0, s>>>(acc, n, deltaL);
    return cudaGetLastError();
}

}  // namespace recon
