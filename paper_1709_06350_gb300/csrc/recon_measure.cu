// recon_measure.cu -- measurement helpers (not part of the method): the FP64
// fused multiply-add rate, the roof of the FP64 path's smoother.
#include "internal.cuh"

namespace recon {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int iters)
{
    double a[kChains];
#pragma unroll
    for (int u = 0; u < kChains; ++u) a[u] = 1.0 + 1e-3 * (double)(threadIdx.x + u);
    const double m = 0.9999999999, c = 1e-10;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kChains; ++u) s += a[u];
    if (s == -1.0) *out = s;   // never: the chains stay live
}

}  // namespace
}  // namespace recon

extern "C" recon_status recon_measure_fp64_fma(int blocks, int iters, double *out, void *stream)
{
    if (blocks < 1 || iters < 1 || !out) return RECON_E_INVALID;
    recon::note_launch();
    recon::k_fp64_fma<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, iters);
    return cudaGetLastError() == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}
