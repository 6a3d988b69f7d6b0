// common.cuh -- shared host/device helpers of librecon (grid addressing,
// launch shapes, block reductions, device scalar slots).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "recon.h"
#include "recon_steps.h"

namespace recon {

// ---------------------------------------------------------------- grid
// C order [i][j][k], k fastest.  N <= 1024, so every offset fits 32 bits.
constexpr int kMaxN = 1024;
__host__ __device__ __forceinline__ unsigned offs(int N, int i, int j, int k)
{
    return ((unsigned)i * (unsigned)N + (unsigned)j) * (unsigned)N + (unsigned)k;
}
__device__ __forceinline__ int wp(int a, int N) { return a + 1 == N ? 0 : a + 1; }
__device__ __forceinline__ int wm(int a, int N) { return a == 0 ? N - 1 : a - 1; }

constexpr int kThreads = 256;      // block size of the elementwise kernels
constexpr int kReduceThreads = 1024;
constexpr int kCoarseThreads = 512;
constexpr int kMaxCoarseCells = 4096;  // 16^3: the single-CTA coarsest solve

inline unsigned blocks_for(size_t work, int threads = kThreads)
{
    return (unsigned)((work + threads - 1) / threads);
}

// Grid of the grid-stride elementwise kernels: enough blocks to fill the
// GPU, few enough that per-thread set-up (an FP64 scalar read and converted
// once) is amortised over many elements.
constexpr unsigned kMaxStrideBlocks = 4096;
inline unsigned stride_blocks(size_t work)
{
    const unsigned b = blocks_for(work);
    return b == 0 ? 1u : (b < kMaxStrideBlocks ? b : kMaxStrideBlocks);
}

// Per-thread sum of values of type T, returned as double.  For float the
// sum is compensated (Kahan): GB300 runs FP64 at 1/64 of the FP32 rate, so
// FP32 kernels accumulate in FP32 and widen once per thread.
template <typename T>
struct ThreadSum;
template <>
struct ThreadSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct ThreadSum<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Row-based launch shape of the grid kernels: 32 threads along k (or along
// k-pairs), 8 rows (i, j) per block, a grid-stride loop over the N^2 rows.
// Index arithmetic is a single 32-bit division per row.
constexpr int kRowX = 32, kRowY = 8;
constexpr unsigned kMaxRowBlocks = 8192;
inline dim3 row_block() { return dim3(kRowX, kRowY, 1); }
inline unsigned row_grid(int N, unsigned cap = kMaxRowBlocks)
{
    const unsigned rows = (unsigned)N * (unsigned)N;
    const unsigned b = (rows + kRowY - 1) / kRowY;
    return b < cap ? b : cap;
}
#define FOR_ROWS(N, i, j)                                                              \
    for (unsigned row_ = blockIdx.x * blockDim.y + threadIdx.y;                        \
         row_ < (unsigned)(N) * (unsigned)(N); row_ += gridDim.x * blockDim.y)          \
        if (const int i = (int)(row_ / (unsigned)(N)), j = (int)(row_ % (unsigned)(N)); true)

// ---------------------------------------------------------------- scalars
// Device-resident scalars of one handle (doubles), so that a cycle needs no
// host round trip except the convergence read.
enum Slot {
    S_C = 0,          // compatibility scalar c of the finest level
    S_ZERO = 1,       // always 0 (c of the coarse levels)
    S_REL = 2,        // ||r - mean r|| / ||b - 1|| after the last cycle
    S_MEAN_R = 3,     // mean residual of the last cycle
    S_MEAN_T = 4,     // mean of theta (gauge shift)
    S_DENOM = 5,      // ||b - 1||_2 (1 when b == 1)
    S_BMIN = 6,       // min(b)   (domain check)
    S_BBAD = 7,       // count of non-finite b
    S_LEVEL = 8,      // per-level slots start here: 4 per level
    S_ADJ_MEAN = S_LEVEL + 4 * 16,   // adjoint: means, norms, null-space sums
    S_ADJ_NORM,
    S_ADJ_SLAM,
    S_ADJ_SN,
    S_SMOOTH_MEAN,    // recon_smooth_density: mean of the floored field
    S_COUNT
};
// per-level slots (level l >= 1): restricted-residual mean, defect scale s,
// prolongation factor 1/s (0 = skip), spare
__host__ __device__ __forceinline__ int slot_rmean(int l) { return S_LEVEL + 4 * l + 0; }
__host__ __device__ __forceinline__ int slot_scale(int l) { return S_LEVEL + 4 * l + 1; }
__host__ __device__ __forceinline__ int slot_pscale(int l) { return S_LEVEL + 4 * l + 2; }

// ---------------------------------------------------------------- reductions
// Linear thread index (blocks may be 2-D); reductions return in ltid() == 0.
__device__ __forceinline__ int ltid() { return threadIdx.x + threadIdx.y * blockDim.x; }

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = ltid(), lane = t & 31, warp = t >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;   // valid in ltid() == 0
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    const int t = ltid(), lane = t & 31, warp = t >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = INFINITY;
    if (warp == 0) {
        r = lane < NT / 32 ? sh[lane] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) r = fmin(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    return r;
}

}  // namespace recon
