// recon_noalloc.cu -- a coarsest-grid solve that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this step: a
// host that pre-reserves all device memory for its own pool, a real-time
// loop that forbids allocation after start-up, or code running inside a
// library that does not own the device.  recon_step_coarse_solve needs an
// N^3 scratch buffer from its caller; this variant keeps that scratch in a
// fixed array compiled into the library instead.
#include <mutex>

#include "internal.cuh"

namespace {

// Scratch of recon_step_coarse_solve_noalloc: room for the largest coarsest
// grid, 16^3 = 4096 cells (4096 doubles or 8192 floats, 32 KiB).  Every GPU
// that loads the library holds this array until the process exits.
constexpr int kNoAllocCells = recon::kMaxCoarseCells;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocCells];

// Device address of the array, looked up once per device.  In host code the
// name g_noalloc_scratch is only a host-side stand-in: passing it to a kernel
// would fault (or, where the GPU can reach host memory, silently use the
// wrong memory), so kernels get the address from cudaGetSymbolAddress.
// The cached address belongs to the device's current context: after
// cudaDeviceReset the module is loaded again at a new address, and calls made
// after a reset are not supported (the cache is not invalidated; the
// allocating recon_step_coarse_solve has no such limit).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

recon_status scratch_for_current_device(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        recon::set_thread_error("no usable current CUDA device");
        return RECON_E_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            recon::set_thread_error(cudaGetErrorString(e));
            return RECON_E_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RECON_OK;
}

}  // namespace

extern "C" recon_status recon_step_coarse_solve_noalloc(int N, double h, int prec, int rule,
                                                        void *theta, const void *g, double c,
                                                        int max_sweeps, double rtol,
                                                        int *sweeps_done, void *stream)
{
    if (N < 4 || N % 2 != 0 || (long)N * N * N > kNoAllocCells) {
        recon::set_thread_error("recon_step_coarse_solve_noalloc: N must be even, >= 4 and "
                                "N^3 <= 4096 (the fixed scratch holds one 16^3 grid)");
        return RECON_E_INVALID;
    }
    if (!(h > 0) || max_sweeps < 1 || !(rtol >= 0) || !theta || !g ||
        (rule != 0 && rule != 1) || (prec != 0 && prec != 1)) {
        recon::set_thread_error("recon_step_coarse_solve_noalloc: bad argument");
        return RECON_E_INVALID;
    }
    void *scratch = nullptr;
    const recon_status st = scratch_for_current_device(&scratch);
    if (st != RECON_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = prec == 0
        ? recon::coarse_solve<double>(N, h, rule, (double *)theta, (const double *)g, nullptr, c,
                                      max_sweeps, rtol, (double *)scratch, sweeps_done, s)
        : recon::coarse_solve<float>(N, h, rule, (float *)theta, (const float *)g, nullptr, c,
                                     max_sweeps, rtol, (float *)scratch, sweeps_done, s);
    if (e != cudaSuccess) {
        recon::set_thread_error(cudaGetErrorString(e));
        return RECON_E_CUDA;
    }
    return RECON_OK;
}
