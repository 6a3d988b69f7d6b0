// recon_gauss.cu -- 1-point Gaussianisation of a field (Sec. III: the paper
// tried it on delta_r), read as the rank mapping
//     g_i = mean + std * Phi^-1((rank_i + 1/2) / n),
// rank_i the position of value i in ascending order, ties broken by
// position; mean and std (population) of the input.
//
// Ranks come from a least-significant-digit radix sort of (key, index)
// pairs: key = the value's bits made order-preserving as an unsigned 64-bit
// integer (-0 taken as +0), 8 passes of 8-bit digits.  Each pass: a digit
// histogram per tile of 4096 elements, an exclusive scan of the
// (digit-major, tile-minor) counts, and a stable scatter in which each tile
// ranks its elements in order (warp match on the digit, per-warp counts
// prefix-summed across warps).  The quantile is FP32 (normcdfinvf of the
// smaller tail probability, so the tails keep their precision): g carries
// ~1e-6 relative rounding, like delta_r itself.
#include <climits>

#include "internal.cuh"

namespace recon {

#define CK(expr)                                \
    do {                                        \
        const cudaError_t ck_e = (expr);        \
        if (ck_e != cudaSuccess) return ck_e;   \
    } while (0)

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;                        // items per thread per tile
constexpr int kTile = kRadixThreads * kRadixItems;     // 4096
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanSeg = kScanThreads * kScanItems;    // 4096 counts per scan block

__device__ __forceinline__ unsigned long long order_key(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v == 0.0 ? 0.0 : v);
    return (b >> 63) ? ~b : (b | (1ull << 63));
}

// keys, identity indices, and per-block sums of v and v^2
__global__ void __launch_bounds__(kThreads)
k_gauss_keys(const double *__restrict__ v, size_t n, unsigned long long *__restrict__ key,
             unsigned *__restrict__ idx, double *__restrict__ partials)
{
    __shared__ double sh[32];
    ThreadSum<double> s1, s2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double x = v[i];
        key[i] = order_key(x);
        idx[i] = (unsigned)i;
        s1.add(x);
        s2.add(x * x);
    }
    double t = block_sum<kThreads>(s1.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = t;
    t = block_sum<kThreads>(s2.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 1] = t;
}

// scal[0] = mean, scal[1] = population std
__global__ void __launch_bounds__(kReduceThreads)
k_gauss_moments(const double *__restrict__ partials, int nb, double n, double *__restrict__ scal)
{
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += partials[4 * i + 0];
        b += partials[4 * i + 1];
    }
    a = block_sum<kReduceThreads>(a, sh);
    b = block_sum<kReduceThreads>(b, sh);
    if (ltid() == 0) {
        const double m = a / n, var = b / n - m * m;
        scal[0] = m;
        scal[1] = var > 0.0 ? sqrt(var) : 0.0;
    }
}

// counts[d * ntile + tile] = occurrences of digit d in the tile
__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const unsigned long long *__restrict__ key, size_t n, int shift, int ntile,
             unsigned *__restrict__ counts)
{
    __shared__ unsigned hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kTile;
    for (int r = 0; r < kRadixItems; ++r) {
        const size_t e = base + (size_t)r * kRadixThreads + threadIdx.x;
        if (e < n) atomicAdd(&hist[(unsigned)(key[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * ntile + blockIdx.x] = hist[threadIdx.x];
}

// block-wide exclusive scan of one value per thread (total in *total)
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *sh, unsigned *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;   // inclusive prefix over warps
    }
    __syncthreads();
    const unsigned before = warp ? sh[warp - 1] : 0u;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// exclusive scan of each kScanSeg-long segment in place; segsum = its total
__global__ void __launch_bounds__(kScanThreads)
k_scan_seg(unsigned *__restrict__ a, size_t m, unsigned *__restrict__ segsum)
{
    __shared__ unsigned sh[32];
    const size_t base = (size_t)blockIdx.x * kScanSeg + (size_t)threadIdx.x * kScanItems;
    unsigned v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < m ? a[base + k] : 0u;
        s += v[k];
    }
    unsigned total;
    unsigned run = block_excl_scan(s, sh, &total);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < m) a[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) segsum[blockIdx.x] = total;
}

// exclusive scan of the segment totals (one block, any count)
__global__ void __launch_bounds__(kScanThreads)
k_scan_top(unsigned *__restrict__ segsum, int nseg)
{
    __shared__ unsigned sh[32];
    unsigned carry = 0;
    for (int base = 0; base < nseg; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const unsigned v = i < nseg ? segsum[i] : 0u;
        unsigned total;
        const unsigned ex = block_excl_scan(v, sh, &total);
        if (i < nseg) segsum[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_add(unsigned *__restrict__ a, size_t m, const unsigned *__restrict__ segsum)
{
    const size_t base = (size_t)blockIdx.x * kScanSeg + (size_t)threadIdx.x * kScanItems;
    const unsigned add = segsum[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < m) a[base + k] += add;
}

// stable scatter of one tile by the digit at `shift`; offs[d * ntile + tile]
// is where the tile's first element of digit d goes
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const unsigned long long *__restrict__ kin, const unsigned *__restrict__ iin, size_t n,
                int shift, int ntile, const unsigned *__restrict__ offs,
                unsigned long long *__restrict__ kout, unsigned *__restrict__ iout)
{
    constexpr int kW = kRadixThreads / 32;
    __shared__ unsigned base[256], total[256];
    __shared__ unsigned wcnt[kW][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(size_t)tid * ntile + blockIdx.x];
    const size_t tile = (size_t)blockIdx.x * kTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kRadixItems; ++r) {
        for (int w = 0; w < kW; ++w) wcnt[w][tid] = 0;
        const size_t e = tile + (size_t)r * kRadixThreads + tid;
        const bool valid = e < n;
        const unsigned long long k = valid ? kin[e] : 0ull;
        const unsigned d = valid ? ((unsigned)(k >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt);
        __syncthreads();   // base / wcnt ready
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over the warps of this round
            unsigned run = 0;
            for (int w = 0; w < kW; ++w) {
                const unsigned c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            total[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const unsigned pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = k;
            iout[pos] = iin[e];
        }
        __syncthreads();
        base[tid] += total[tid];
    }
}

// g[idx[r]] = mean + std * Phi^-1((r + 1/2) / n).  The probability and the
// quantile are FP64: above 2^24 cells adjacent ranks would round to the same
// FP32 probability and distinct inputs would get equal outputs.  The quantile
// is taken of the smaller tail probability and mirrored, so the two halves
// are exactly antisymmetric.
__global__ void __launch_bounds__(kThreads)
k_gauss_out(const unsigned *__restrict__ idx, size_t n, const double *__restrict__ scal,
            double *__restrict__ g)
{
    const double m = scal[0], sd = scal[1];
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (size_t)gridDim.x * blockDim.x) {
        const size_t lo = r < n - 1 - r ? r : n - 1 - r;
        const double q = ((double)lo + 0.5) / (double)n;   // smaller tail probability
        const double z = normcdfinv(q);
        g[idx[r]] = m + sd * (r == lo ? z : -z);
    }
}

cudaError_t gauss_alloc(recon_handle *H, size_t n)
{
    GaussWork &G = H->gauss;
    if (G.cap >= n) return cudaSuccess;
    gauss_free(H);
    const size_t ntile = (n + kTile - 1) / kTile, m = 256 * ntile;
    const size_t nseg = (m + kScanSeg - 1) / kScanSeg;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMalloc(&G.key[b], sizeof(unsigned long long) * n);
        if (e == cudaSuccess) e = cudaMalloc(&G.idx[b], sizeof(unsigned) * n);
    }
    if (e == cudaSuccess) e = cudaMalloc(&G.counts, sizeof(unsigned) * m);
    if (e == cudaSuccess) e = cudaMalloc(&G.segsum, sizeof(unsigned) * nseg);
    if (e == cudaSuccess) e = cudaMalloc(&G.moments, sizeof(double) * 2);
    if (e != cudaSuccess) {
        gauss_free(H);
        return e;
    }
    G.cap = n;
    return cudaSuccess;
}

void gauss_free(recon_handle *H)
{
    GaussWork &G = H->gauss;
    for (int b = 0; b < 2; ++b) {
        if (G.key[b]) cudaFree(G.key[b]);
        if (G.idx[b]) cudaFree(G.idx[b]);
    }
    if (G.counts) cudaFree(G.counts);
    if (G.segsum) cudaFree(G.segsum);
    if (G.moments) cudaFree(G.moments);
    G = GaussWork{};
}

cudaError_t gaussianise(recon_handle *H, const double *v, size_t n, double *g)
{
    cudaStream_t s = H->stream;
    CK(gauss_alloc(H, n));
    GaussWork &G = H->gauss;
    const int ntile = (int)((n + kTile - 1) / kTile);
    const size_t m = 256 * (size_t)ntile;
    const int nseg = (int)((m + kScanSeg - 1) / kScanSeg);
    const unsigned nb = stride_blocks(n) < (unsigned)kMaxRedBlocks ? stride_blocks(n) : (unsigned)kMaxRedBlocks;
    note_launch(2);
    k_gauss_keys<<<nb, kThreads, 0, s>>>(v, n, G.key[0], G.idx[0], H->partials);
    k_gauss_moments<<<1, kReduceThreads, 0, s>>>(H->partials, (int)nb, (double)n, G.moments);
    int cur = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        note_launch(5);
        k_radix_hist<<<ntile, kRadixThreads, 0, s>>>(G.key[cur], n, shift, ntile, G.counts);
        k_scan_seg<<<nseg, kScanThreads, 0, s>>>(G.counts, m, G.segsum);
        k_scan_top<<<1, kScanThreads, 0, s>>>(G.segsum, nseg);
        k_scan_add<<<nseg, kScanThreads, 0, s>>>(G.counts, m, G.segsum);
        k_radix_scatter<<<ntile, kRadixThreads, 0, s>>>(G.key[cur], G.idx[cur], n, shift, ntile, G.counts,
                                                        G.key[cur ^ 1], G.idx[cur ^ 1]);
        cur ^= 1;
    }
    note_launch();
    k_gauss_out<<<stride_blocks(n), kThreads, 0, s>>>(G.idx[cur], n, G.moments, g);
    return cudaGetLastError();
}

}  // namespace recon
