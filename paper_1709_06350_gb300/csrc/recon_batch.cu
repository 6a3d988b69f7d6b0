// recon_batch.cu -- many independent solves (uneven N) advanced together.
//
// Each realisation keeps its own handle (workspace, device scalars) and its
// own stream.  Every phase of the mixed solve (start, one FP32 FAS cycle,
// switch, one defect-correction iteration, finish) is captured once into a
// CUDA graph whose branches are the realisations, so one graph launch runs
// that phase for all of them concurrently; the graph ends with a gather of
// every realisation's relative residual, which the host reads in one copy.
// Graphs are rebuilt only when the pointers or options change.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

struct recon_batch {
    int count = 0;
    std::vector<recon_handle *> h;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t origin = nullptr;     // caller's stream (default: own stream)
    cudaStream_t own = nullptr;
    const double **rel_src = nullptr;  // device: &scal[S_REL] of each handle
    double *rel_dev = nullptr, *rel_host = nullptr;
    cudaGraphExec_t g[5] = {};
    unsigned long long g_kernels[5] = {};
    std::vector<const double *> key_b;
    std::vector<double *> key_phi;
    std::vector<recon_config> key_cfg;
    std::string err;
};

namespace {

enum { G_START = 0, G_FAS, G_SWITCH, G_OUTER, G_FINISH };

__global__ void k_gather(const double *const *src, double *dst, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = *src[i];
}

void destroy_graphs(recon_batch *B)
{
    for (auto &g : B->g)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Capture `body(i)` for every realisation as parallel branches of one graph.
template <class F>
cudaError_t capture(recon_batch *B, F body, int which)
{
    cudaStream_t o = B->origin;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t inner = cudaEventRecord(B->fork, o);
    const unsigned long long counted = recon::launch_count();   // capture runs nothing
    for (int i = 0; i < B->count && inner == cudaSuccess; ++i) {
        inner = cudaStreamWaitEvent(B->streams[i], B->fork, 0);
        if (inner == cudaSuccess) inner = body(i);
        if (inner == cudaSuccess) inner = cudaEventRecord(B->join[i], B->streams[i]);
        if (inner == cudaSuccess) inner = cudaStreamWaitEvent(o, B->join[i], 0);
    }
    if (inner == cudaSuccess) {
        k_gather<<<(B->count + 127) / 128, 128, 0, o>>>(B->rel_src, B->rel_dev, B->count);
        inner = cudaGetLastError();
    }
    e = cudaStreamEndCapture(o, &graph);
    recon::unnote_launch(recon::launch_count() - counted);
    if (inner != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return inner;
    }
    if (e != cudaSuccess) return e;
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    unsigned long long kern = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
    }
    B->g_kernels[which] = kern;
    e = cudaGraphInstantiate(&B->g[which], graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

cudaError_t launch(recon_batch *B, int which)
{
    recon::note_launch(B->g_kernels[which]);
    return cudaGraphLaunch(B->g[which], B->origin);
}

cudaError_t read_rel(recon_batch *B)
{
    cudaError_t e = cudaMemcpyAsync(B->rel_host, B->rel_dev, sizeof(double) * B->count,
                                    cudaMemcpyDeviceToHost, B->origin);
    return e == cudaSuccess ? cudaStreamSynchronize(B->origin) : e;
}

recon_status berr(recon_batch *B, recon_status s, const std::string &m)
{
    B->err = m;
    return s;
}

}  // namespace

extern "C" {

recon_status recon_batch_create(int count, const int *N, const double *L, recon_batch **out)
{
    if (!out || count < 1 || count > 4096 || !N || !L) return RECON_E_INVALID;
    *out = nullptr;
    recon_batch *B = new (std::nothrow) recon_batch();
    if (!B) return RECON_E_OOM;
    B->count = count;
    recon_status st = RECON_OK;
    for (int i = 0; i < count && st == RECON_OK; ++i) {
        recon_handle *h = nullptr;
        st = recon_create(N[i], L[i], RECON_MIXED, &h);
        if (st == RECON_OK) B->h.push_back(h);
    }
    cudaError_t e = cudaSuccess;
    if (st == RECON_OK) {
        B->streams.resize(count);
        B->join.resize(count);
        for (int i = 0; i < count && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&B->streams[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming);
            if (e == cudaSuccess) B->h[i]->stream = B->streams[i];
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->own, cudaStreamNonBlocking);
        B->origin = B->own;
        if (e == cudaSuccess) e = cudaMalloc(&B->rel_src, sizeof(double *) * count);
        if (e == cudaSuccess) e = cudaMalloc(&B->rel_dev, sizeof(double) * count);
        if (e == cudaSuccess) e = cudaMallocHost(&B->rel_host, sizeof(double) * count);
        if (e == cudaSuccess) {
            std::vector<const double *> src(count);
            for (int i = 0; i < count; ++i) src[i] = B->h[i]->scal + recon::S_REL;
            e = cudaMemcpy(B->rel_src, src.data(), sizeof(double *) * count, cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) st = RECON_E_CUDA;
    }
    if (st != RECON_OK) {
        recon_batch_destroy(B);
        return st;
    }
    *out = B;
    return RECON_OK;
}

void recon_batch_destroy(recon_batch *B)
{
    if (!B) return;
    if (B->origin) cudaStreamSynchronize(B->origin);
    destroy_graphs(B);
    for (auto h : B->h) recon_destroy(h);
    for (auto s : B->streams)
        if (s) cudaStreamDestroy(s);
    for (auto ev : B->join)
        if (ev) cudaEventDestroy(ev);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->own) cudaStreamDestroy(B->own);
    if (B->rel_src) cudaFree(B->rel_src);
    if (B->rel_dev) cudaFree(B->rel_dev);
    if (B->rel_host) cudaFreeHost(B->rel_host);
    delete B;
}

recon_status recon_batch_set_stream(recon_batch *B, void *stream)
{
    if (!B) return RECON_E_INVALID;
    cudaStream_t s = stream ? (cudaStream_t)stream : B->own;
    if (s != B->origin) destroy_graphs(B);
    B->origin = s;
    return RECON_OK;
}

recon_handle *recon_batch_handle(recon_batch *B, int i)
{
    return (B && i >= 0 && i < B->count) ? B->h[i] : nullptr;
}

const char *recon_batch_last_error(const recon_batch *B) { return B ? B->err.c_str() : ""; }

recon_status recon_batch_solve(recon_batch *B, const double *const *b, double *const *phi,
                               double tol, int max_cycles, recon_stats *stats)
{
    if (!B) return RECON_E_INVALID;
    if (!b || !phi || !(tol > 0.0) || max_cycles < 1)
        return berr(B, RECON_E_INVALID, "bad arguments");
    B->err.clear();
    const int n = B->count;
    for (int i = 0; i < n; ++i) {
        if (!b[i] || !phi[i]) return berr(B, RECON_E_INVALID, "NULL field pointer");
        if (stats) std::memset(&stats[i], 0, sizeof(recon_stats));
        B->h[i]->have_solve = false;
        B->h[i]->adj.null_ready = false;
        const recon_status s = recon::check_domain(B->h[i], b[i]);   // also ||b - 1||
        if (s != RECON_OK) return berr(B, s, "realisation " + std::to_string(i) + ": " + B->h[i]->err);
    }
    // (re)build the graphs when the fields or the options changed
    std::vector<recon_config> cfg(n);
    for (int i = 0; i < n; ++i) cfg[i] = B->h[i]->cfg;
    const bool same = B->g[0] && B->key_b == std::vector<const double *>(b, b + n) &&
                      B->key_phi == std::vector<double *>(phi, phi + n) &&
                      std::memcmp(B->key_cfg.data(), cfg.data(), sizeof(recon_config) * n) == 0;
    if (!same) {
        destroy_graphs(B);
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess)
            e = capture(B, [&](int i) { return recon::mixed_start(B->h[i], b[i], phi[i]); }, G_START);
        if (e == cudaSuccess)
            e = capture(B, [&](int i) { return recon::mixed_fas_cycle(B->h[i]); }, G_FAS);
        if (e == cudaSuccess)
            e = capture(B, [&](int i) { return recon::mixed_switch(B->h[i], b[i], phi[i], false); }, G_SWITCH);
        if (e == cudaSuccess)
            e = capture(B, [&](int i) {
                cudaError_t r = recon::mixed_residual(B->h[i], b[i], phi[i]);
                return r == cudaSuccess ? recon::mixed_correct(B->h[i], phi[i]) : r;
            }, G_OUTER);
        if (e == cudaSuccess)
            e = capture(B, [&](int i) { return recon::mixed_finish(B->h[i], phi[i], true); }, G_FINISH);
        if (e != cudaSuccess) {
            destroy_graphs(B);
            return berr(B, RECON_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        B->key_b.assign(b, b + n);
        B->key_phi.assign(phi, phi + n);
        B->key_cfg = cfg;
    }
    auto fail = [&](cudaError_t e, const char *w) {
        return berr(B, RECON_E_CUDA, std::string(w) + ": " + cudaGetErrorString(e));
    };
    auto push = [&](int i, double v) {
        if (stats && stats[i].n_history < RECON_HISTORY_MAX) stats[i].history[stats[i].n_history++] = v;
    };
    // the caller's stream orders the batch after earlier work on it
    cudaError_t e = launch(B, G_START);
    if (e != cudaSuccess) return fail(e, "start");
    // FP32 FAS: until every realisation reached the switch level or stalled
    std::vector<double> prev(n, INFINITY);
    std::vector<char> done(n, 0);
    int fas = 0;
    const recon_config &c0 = B->h[0]->cfg;
    for (fas = 1; fas <= c0.mixed_fas_max_cycles; ++fas) {
        if ((e = launch(B, G_FAS)) != cudaSuccess || (e = read_rel(B)) != cudaSuccess)
            return fail(e, "FAS cycle");
        bool all = true;
        for (int i = 0; i < n; ++i) {
            const double r = B->rel_host[i];
            if (!std::isfinite(r)) return berr(B, RECON_E_DIVERGED, "realisation " + std::to_string(i) + " diverged");
            if (!done[i]) push(i, r);
            if (r < B->h[i]->cfg.mixed_switch_rtol || r > 0.7 * prev[i]) done[i] = 1;
            prev[i] = r;
            all = all && done[i];
        }
        if (all) break;
    }
    if (fas > c0.mixed_fas_max_cycles) fas = c0.mixed_fas_max_cycles;
    if ((e = launch(B, G_SWITCH)) != cudaSuccess) return fail(e, "switch");
    // defect correction: until every realisation meets tol
    recon_status status = RECON_E_NOCONV;
    std::vector<char> conv(n, 0);
    std::vector<int> outer(n, 0);
    int o = 0;
    for (o = 1; o <= max_cycles; ++o) {
        if ((e = launch(B, G_OUTER)) != cudaSuccess || (e = read_rel(B)) != cudaSuccess)
            return fail(e, "defect correction");
        bool all = true;
        for (int i = 0; i < n; ++i) {
            const double r = B->rel_host[i];
            if (!std::isfinite(r)) return berr(B, RECON_E_DIVERGED, "realisation " + std::to_string(i) + " diverged");
            if (!conv[i]) {
                push(i, r);
                outer[i] = o;
                if (r < tol) conv[i] = 1;
            }
            all = all && conv[i];
        }
        if (all) {
            status = RECON_OK;
            break;
        }
    }
    if ((e = launch(B, G_FINISH)) != cudaSuccess || (e = cudaStreamSynchronize(B->origin)) != cudaSuccess)
        return fail(e, "finish");
    for (int i = 0; i < n; ++i) {
        recon_handle *h = B->h[i];
        cudaMemcpy(h->hscal, h->scal, sizeof(double) * recon::S_COUNT, cudaMemcpyDeviceToHost);
        if (stats) {
            stats[i].cycles = fas;
            stats[i].outer_iterations = outer[i];
            stats[i].rel_residual = stats[i].n_history ? stats[i].history[stats[i].n_history - 1] : 0.0;
            stats[i].compat_c = h->hscal[recon::S_C];
            stats[i].paper_eps = std::nan("");   // not evaluated by batched solves
        }
        if (conv[i]) {
            h->last_phi = phi[i];
            h->last_b = b[i];
            h->have_solve = true;
        }
    }
    if (status == RECON_E_NOCONV) B->err = "max_cycles reached before every realisation met tol";
    return status;
}

}  // extern "C"
