// common.cuh -- shared host/device helpers of librecon (grid addressing,
// launch shapes, block reductions, device scalar slots).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "recon.h"
#include "recon_steps.h"

namespace recon {

// ---------------------------------------------------------------- grid
// C order [i][j][k], k fastest; 64-bit offsets so N^3 may exceed 2^31.
__host__ __device__ __forceinline__ size_t offs(int N, int i, int j, int k)
{
    return ((size_t)i * (size_t)N + (size_t)j) * (size_t)N + (size_t)k;
}
__device__ __forceinline__ int wp(int a, int N) { return a + 1 == N ? 0 : a + 1; }
__device__ __forceinline__ int wm(int a, int N) { return a == 0 ? N - 1 : a - 1; }

constexpr int kThreads = 256;      // default block size of the grid kernels
constexpr int kReduceThreads = 1024;
constexpr int kCoarseThreads = 512;
constexpr int kMaxCoarseCells = 4096;  // 16^3: the single-CTA coarsest solve

inline unsigned blocks_for(size_t work, int threads = kThreads)
{
    return (unsigned)((work + threads - 1) / threads);
}

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
    S_COUNT = S_LEVEL + 4 * 16
};
// per-level slots (level l >= 1): restricted-residual mean, defect scale s,
// prolongation factor 1/s (0 = skip), spare
__host__ __device__ __forceinline__ int slot_rmean(int l) { return S_LEVEL + 4 * l + 0; }
__host__ __device__ __forceinline__ int slot_scale(int l) { return S_LEVEL + 4 * l + 1; }
__host__ __device__ __forceinline__ int slot_pscale(int l) { return S_LEVEL + 4 * l + 2; }

// ---------------------------------------------------------------- reductions
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < NT / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
