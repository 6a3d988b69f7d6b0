// recon_smooth.cu -- density preparation before the solve: Gaussian
// smoothing of the assigned density, a floor on 1 + delta and a
// renormalisation to mean 1.
//
// The window is exp(-k^2 R^2 / 2) on the periodic box's wave vectors (the
// Gaussian window of Sec. III, width R), the floor 1 + delta >= floor keeps
// the right side of the cell cubic positive (empty CIC cells), and the mean is
// restored to 1 after the floor.  The window factorises over the axes, so the
// filter is three circular convolutions along k, j and i with the 1-D kernel
//     g[n] = (1/N) sum_m exp(-k_m^2 R^2 / 2) cos(2 pi m n / N),
//     k_m = 2 pi min(m, N - m) / L,
// the inverse DFT of the sampled window: the same operator as multiplying the
// 3-D DFT by the window, truncated where |g[n]| < 1e-9 g[0].  For R of a few
// cells the kernel decays within ~6.4 R / h cells; for R below ~1.5 h the
// window is still sizeable at the grid's Nyquist frequency and the kernel
// spans the whole periodic line (up to N taps: exact, and slower).  Taps and
// sums are FP32 (the output carries ~(taps) 2^-24 relative rounding), input
// and output FP64; the two intermediate fields are FP32 in the caller's
// scratch.
#include <cmath>

#include "internal.cuh"

namespace recon {
namespace {

constexpr int kMaxTaps = kMaxN / 2;  // largest half-width T: the whole periodic line
struct Taps {
    int T;                           // g[-T .. T], g symmetric
    float w[kMaxTaps + 1];           // w[n] = g[n], n = 0 .. T
};

// ---- pass along k (contiguous): a CTA per row, the row and its wrapped
// halo staged in shared memory
template <typename TIn>
__global__ void __launch_bounds__(256)
k_smooth_k(const TIn *__restrict__ in, float *__restrict__ out, int N, Taps tp)
{
    extern __shared__ float srow[];
    const unsigned row = blockIdx.x;
    const unsigned base = row * (unsigned)N;
    const int T = tp.T;
    for (int x = threadIdx.x; x < N + 2 * T; x += blockDim.x) {
        int k = x - T;
        k = k < 0 ? k + N : (k >= N ? k - N : k);
        srow[x] = (float)in[base + (unsigned)k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float acc = tp.w[0] * srow[k + T];
        for (int n = 1; n <= T; ++n) acc = fmaf(tp.w[n], srow[k + T - n] + srow[k + T + n], acc);
        out[base + (unsigned)k] = acc;
    }
}

// ---- pass along j (AX = 1) or i (AX = 0): a CTA per (other index, 32
// columns of k, 64 outputs along the axis); the tile of 64 + 2T rows of 32
// columns is staged in shared memory (coalesced along k).  FINAL: the i pass,
// which floors, writes FP64 and sums the floored values per CTA (partials,
// one double per CTA).
constexpr int kSX = 32, kSY = 8, kSOut = 64;
template <int AX, bool FINAL>
__global__ void __launch_bounds__(kSX *kSY)
k_smooth_axis(const float *__restrict__ in, float *__restrict__ out32, double *__restrict__ out64, int N,
              Taps tp, float floor_, double *__restrict__ partials)
{
    extern __shared__ float stile[];   // [kSOut + 2T][kSX]
    const int T = tp.T;
    const int k0 = blockIdx.x * kSX, a0 = blockIdx.y * kSOut, other = blockIdx.z;
    const unsigned NN = (unsigned)N * (unsigned)N;
    // element (axis index a, column k): AX = 1 -> (i = other, j = a), AX = 0 -> (i = a, j = other)
    auto at = [&](int a, int k) -> unsigned {
        return AX == 1 ? (unsigned)other * NN + (unsigned)a * (unsigned)N + (unsigned)k
                       : (unsigned)a * NN + (unsigned)other * (unsigned)N + (unsigned)k;
    };
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int rows = kSOut + 2 * T;
    for (int r = ty; r < rows; r += kSY) {
        int a = a0 + r - T;
        a = a < 0 ? a + N : (a >= N ? a - N : a);
        const int k = k0 + lane;
        stile[r * kSX + lane] = k < N ? in[at(a, k)] : 0.0f;
    }
    __syncthreads();
    double sum = 0.0;
    const int k = k0 + lane;
    for (int o = ty; o < kSOut; o += kSY) {
        const int a = a0 + o;
        if (a >= N || k >= N) continue;
        float acc = tp.w[0] * stile[(o + T) * kSX + lane];
        for (int n = 1; n <= T; ++n)
            acc = fmaf(tp.w[n], stile[(o + T - n) * kSX + lane] + stile[(o + T + n) * kSX + lane], acc);
        if constexpr (FINAL) {
            const double v = fmax((double)acc, (double)floor_);
            out64[at(a, k)] = v;
            sum += v;
        } else {
            out32[at(a, k)] = acc;
        }
    }
    if constexpr (FINAL) {
        __shared__ double sh[32];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) sh[ty] = sum;
        __syncthreads();
        if (ty == 0) {
            double v = lane < kSY ? sh[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            const unsigned b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
            if (lane == 0) partials[b] = v;
        }
    }
}

// mean of the floored field from nb CTA partials (fixed order), then b /= mean
__global__ void __launch_bounds__(1024)
k_smooth_mean(const double *__restrict__ partials, int nb, double n, double *__restrict__ mean)
{
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *mean = v / n;
    }
}

__global__ void __launch_bounds__(kThreads)
k_smooth_scale(double *__restrict__ b, size_t n, const double *__restrict__ mean)
{
    const double s = 1.0 / *mean;
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        b[id] *= s;
}

}  // namespace

// Taps of the kernel, truncated where it stays below 1e-9 of its centre.
static void smooth_taps(int N, double L, double R, Taps &tp)
{
    const int half = N / 2;
    double W[kMaxN], g[kMaxTaps + 1];
    for (int m = 0; m < N; ++m) {
        const double km = 2.0 * M_PI * (double)(m <= half ? m : N - m) / L;
        W[m] = std::exp(-0.5 * km * km * R * R);
    }
    for (int n = 0; n <= half; ++n) {
        double acc = 0.0;
        for (int m = 0; m < N; ++m) acc += W[m] * std::cos(2.0 * M_PI * (double)(((long)m * n) % N) / (double)N);
        g[n] = acc / (double)N;
    }
    int T = 0;
    for (int n = 1; n <= half; ++n)
        if (std::fabs(g[n]) >= 1e-9 * g[0]) T = n;
    if (2 * T + 1 > N) {
        // the kernel spans the whole periodic line: g[-N/2] and g[N/2] are the
        // same cell, counted once
        T = half;
        tp.T = T;
        for (int n = 0; n <= T; ++n) tp.w[n] = (float)g[n];
        if (2 * T == N) tp.w[T] = (float)(0.5 * g[T]);
        return;
    }
    tp.T = T;
    for (int n = 0; n <= T; ++n) tp.w[n] = (float)g[n];
}

static bool g_smooth_ready = false;

// rho -> b; w32: 2 N^3 floats of scratch (8-byte aligned; the first field
// holds the i pass's per-CTA sums once the j pass has read it); mean: one
// device double.
cudaError_t smooth_density(int N, double L, double R, double floor_, const double *rho, double *b, float *w32,
                           double *mean, cudaStream_t s)
{
    if (N > kMaxN) return cudaErrorInvalidValue;
    if (!g_smooth_ready) {
        // the staging tile of the widest kernel: (64 + N) rows of 32 floats
        const int most = (int)sizeof(float) * (kSOut + 2 * kMaxTaps) * kSX;
        cudaError_t e = cudaFuncSetAttribute(k_smooth_axis<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_smooth_axis<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e != cudaSuccess) return e;
        g_smooth_ready = true;
    }
    // the taps of the last (N, L, R) on this host thread are reused
    static thread_local int cN = 0;
    static thread_local double cL = 0.0, cR = -1.0;
    static thread_local Taps tp;
    if (N != cN || L != cL || R != cR) {
        if (R <= 0.0) {
            tp.T = 0;
            tp.w[0] = 1.0f;
        } else {
            smooth_taps(N, L, R, tp);
        }
        cN = N;
        cL = L;
        cR = R;
    }
    const size_t n = (size_t)N * N * N;
    float *w1 = w32, *w2 = w32 + n;
    const dim3 blk(kSX, kSY);
    const dim3 grid((N + kSX - 1) / kSX, (N + kSOut - 1) / kSOut, N);
    const unsigned nb = grid.x * grid.y * grid.z;
    double *partials = reinterpret_cast<double *>(w1);
    if ((size_t)nb * 2 > n) return cudaErrorInvalidValue;
    const size_t tile = sizeof(float) * (size_t)(kSOut + 2 * tp.T) * kSX;
    note_launch(5);
    k_smooth_k<double><<<(unsigned)N * (unsigned)N, 256, sizeof(float) * (size_t)(N + 2 * tp.T), s>>>(rho, w1, N, tp);
    k_smooth_axis<1, false><<<grid, blk, tile, s>>>(w1, w2, nullptr, N, tp, (float)floor_, nullptr);
    k_smooth_axis<0, true><<<grid, blk, tile, s>>>(w2, nullptr, b, N, tp, (float)floor_, partials);
    k_smooth_mean<<<1, 1024, 0, s>>>(partials, (int)nb, (double)n, mean);
    k_smooth_scale<<<stride_blocks(n), kThreads, 0, s>>>(b, n, mean);
    return cudaGetLastError();
}

}  // namespace recon
