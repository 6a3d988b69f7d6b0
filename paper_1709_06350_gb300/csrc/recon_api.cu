// recon_api.cu -- the C ABI of librecon (include/recon.h, include/recon_steps.h):
// argument checks, workspace ownership, status codes and messages.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace recon;

namespace {

thread_local std::string g_create_err;

// Hierarchy of Sec. II.A.3: halve while the half is even and >= 4.
int level_sizes(int N, int *Nl)
{
    int L = 0;
    Nl[L++] = N;
    while (N % 2 == 0 && N / 2 >= 4 && (N / 2) % 2 == 0 && L < kMaxLevels) {
        N /= 2;
        Nl[L++] = N;
    }
    return L;
}

const char *check_size(int N, int *Nl, int *nlev)
{
    if (N < 4 || N % 2 != 0) return "N must be even and >= 4";
    if (N > kMaxN) return "N must be <= 1024";
    *nlev = level_sizes(N, Nl);
    const int Nc = Nl[*nlev - 1];
    if ((long)Nc * Nc * Nc > kMaxCoarseCells)
        return "the coarsest grid (halving N while the half is even and >= 4) must be <= 16^3";
    return nullptr;
}

recon_config default_config()
{
    recon_config c;
    std::memset(&c, 0, sizeof(c));   // padding too: batches compare configs bytewise
    c.nu1 = 2;
    c.nu2 = 2;
    c.coarse_max_sweeps = 200;
    c.coarse_rtol = 1e-3;
    c.rule = RECON_RULE_NEWTON1;
    c.start = RECON_START_FMG;
    c.scale_floor = 0.5;
    c.mixed_switch_rtol = 1e-4;
    c.mixed_fas_max_cycles = 12;
    c.mixed_linear_vcycles = 2;
    c.mixed_df_residual = 1;
    c.fused_chunk = 0;
    c.adjoint_store_cofactors = 0;
    c.report_paper_eps = 0;
    return c;
}

// Byte plan of the workspace; alloc = false only sums the sizes.
struct Planner {
    bool alloc;
    size_t total = 0;
    bool failed = false;
    template <typename T>
    void take(T **p, size_t count)
    {
        const size_t bytes = ((sizeof(T) * count + 255) / 256) * 256;
        total += bytes;
        if (!alloc || failed) return;
        if (cudaMalloc((void **)p, bytes) != cudaSuccess) {
            failed = true;
            *p = nullptr;
        }
    }
};

void plan(recon_handle *H, Planner &P)
{
    const size_t n0 = (size_t)H->N * H->N * H->N;
    P.take(&H->work64, n0);
    P.take(&H->work64b, n0);
    for (int l = 1; l < H->nlev; ++l) {
        const size_t n = (size_t)H->Nl[l] * H->Nl[l] * H->Nl[l];
        if (H->dtype == RECON_F64) {
            P.take(&H->t64[l], n);
            P.take(&H->g64[l], n);
            P.take(&H->told64[l], n);
            P.take(&H->aux64[l], n);
        }
    }
    if (H->dtype == RECON_MIXED) {
        for (int l = 0; l < H->nlev; ++l) {
            const size_t n = (size_t)H->Nl[l] * H->Nl[l] * H->Nl[l];
            P.take(&H->t32[l], n);
            P.take(&H->g32[l], n);
            P.take(&H->e32[l], n);
            P.take(&H->f32[l], n);
            // the fused linear sweeps form the cofactors from theta32
            if (H->Nl[l] < kFusedMinN) P.take(&H->cof32[l], 6 * n);
            if (l > 0) {
                P.take(&H->told32[l], n);
                P.take(&H->aux32[l], n);
            }
        }
        P.take(&H->work32, n0);
        P.take(&H->lo32, n0);
        P.take(&H->blo32, n0);
    }
    P.take(&H->scal, (size_t)S_COUNT);
    P.take(&H->partials, (size_t)4 * kMaxRedBlocks);
    P.take(&H->iscratch, (size_t)64);
}

void free_all(recon_handle *H)
{
    auto f = [](void *p) {
        if (p) cudaFree(p);
    };
    f(H->work64);
    f(H->work64b);
    f(H->work32);
    f(H->lo32);
    f(H->blo32);
    for (int l = 0; l < kMaxLevels; ++l) {
        if (l > 0) {
            f(H->t64[l]);
            f(H->g64[l]);
        }
        f(H->told64[l]);
        f(H->aux64[l]);
        f(H->t32[l]);
        f(H->g32[l]);
        f(H->told32[l]);
        f(H->aux32[l]);
        f(H->e32[l]);
        f(H->f32[l]);
        f(H->cof32[l]);
    }
    f(H->scal);
    f(H->partials);
    f(H->iscratch);
    if (H->hscal) cudaFreeHost(H->hscal);
}

recon_status set_err(recon_handle *H, recon_status s, const std::string &msg)
{
    if (H) H->err = msg;
    return s;
}

recon_status cuda_status(recon_handle *H, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return RECON_OK;
    return set_err(H, RECON_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

const char *recon_status_string(recon_status s)
{
    switch (s) {
    case RECON_OK: return "RECON_OK";
    case RECON_E_INVALID: return "RECON_E_INVALID";
    case RECON_E_DOMAIN: return "RECON_E_DOMAIN";
    case RECON_E_NOCONV: return "RECON_E_NOCONV";
    case RECON_E_DIVERGED: return "RECON_E_DIVERGED";
    case RECON_E_CUDA: return "RECON_E_CUDA";
    case RECON_E_OOM: return "RECON_E_OOM";
    case RECON_E_TIMEOUT: return "RECON_E_TIMEOUT";
    case RECON_E_UNIMPLEMENTED: return "RECON_E_UNIMPLEMENTED";
    }
    return "RECON_E_UNKNOWN";
}

size_t recon_workspace_bytes(int N, recon_dtype dtype)
{
    recon_handle H;
    if (check_size(N, H.Nl, &H.nlev)) return 0;
    if (dtype != RECON_F64 && dtype != RECON_MIXED) return 0;
    H.N = N;
    H.dtype = dtype;
    Planner P{false};
    plan(&H, P);
    return P.total;
}

recon_status recon_create(int N, double L, recon_dtype dtype, recon_handle **out)
{
    g_create_err.clear();
    if (!out) {
        g_create_err = "out is NULL";
        return RECON_E_INVALID;
    }
    *out = nullptr;
    recon_handle *H = new (std::nothrow) recon_handle();
    if (!H) {
        g_create_err = "host allocation failed";
        return RECON_E_OOM;
    }
    const char *why = check_size(N, H->Nl, &H->nlev);
    if (!why && !(L > 0.0 && std::isfinite(L))) why = "L must be finite and > 0";
    if (!why && dtype != RECON_F64 && dtype != RECON_MIXED) why = "unknown dtype";
    if (why) {
        g_create_err = why;
        delete H;
        return RECON_E_INVALID;
    }
    H->N = N;
    H->L = L;
    H->h = L / N;
    for (int l = 0; l < H->nlev; ++l) H->hl[l] = H->h * (double)(1 << l);
    H->dtype = dtype;
    H->cfg = default_config();
    Planner P{true};
    plan(H, P);
    if (P.failed) {
        g_create_err = "cudaMalloc of " + std::to_string(P.total) + " bytes of workspace failed";
        free_all(H);
        delete H;
        cudaGetLastError();
        return RECON_E_OOM;
    }
    if (cudaMallocHost((void **)&H->hscal, sizeof(double) * S_COUNT) != cudaSuccess) {
        H->hscal = nullptr;
        g_create_err = "cudaMallocHost failed";
        free_all(H);
        delete H;
        cudaGetLastError();
        return RECON_E_OOM;
    }
    cudaError_t e = prepare_kernels();
    if (e == cudaSuccess) e = cudaMemset(H->scal, 0, sizeof(double) * S_COUNT);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_create_err = std::string("initialising the workspace: ") + cudaGetErrorString(e);
        free_all(H);
        delete H;
        return RECON_E_CUDA;
    }
    *out = H;
    return RECON_OK;
}

void recon_destroy(recon_handle *H)
{
    if (!H) return;
    if (H->stream) cudaStreamSynchronize(H->stream);
    else cudaDeviceSynchronize();
    adj_free(H);
    gauss_free(H);
    if (H->dadj) cudaFree(H->dadj);
    free_all(H);
    delete H;
}

recon_status recon_set_stream(recon_handle *H, void *stream)
{
    if (!H) return RECON_E_INVALID;
    H->stream = (cudaStream_t)stream;
    return RECON_OK;
}

recon_status recon_get_config(const recon_handle *H, recon_config *cfg)
{
    if (!H || !cfg) return RECON_E_INVALID;
    *cfg = H->cfg;
    return RECON_OK;
}

recon_status recon_set_config(recon_handle *H, const recon_config *c)
{
    if (!H || !c) return RECON_E_INVALID;
    if (c->nu1 < 0 || c->nu2 < 0 || c->nu1 + c->nu2 < 1 || c->nu1 > 64 || c->nu2 > 64)
        return set_err(H, RECON_E_INVALID, "nu1, nu2 must be in [0, 64] with nu1 + nu2 >= 1");
    if (c->coarse_max_sweeps < 1 || c->coarse_max_sweeps > 100000)
        return set_err(H, RECON_E_INVALID, "coarse_max_sweeps must be in [1, 100000]");
    if (!(c->coarse_rtol >= 0.0 && c->coarse_rtol < 1.0))
        return set_err(H, RECON_E_INVALID, "coarse_rtol must be in [0, 1)");
    if (c->rule != RECON_RULE_NEWTON1 && c->rule != RECON_RULE_EXACT)
        return set_err(H, RECON_E_INVALID, "unknown rule");
    if (c->start != RECON_START_FMG && c->start != RECON_START_GUESS)
        return set_err(H, RECON_E_INVALID, "unknown start");
    if (!(c->scale_floor < 1.0) || !std::isfinite(c->scale_floor))
        return set_err(H, RECON_E_INVALID, "scale_floor must be < 1");
    if (!(c->mixed_switch_rtol > 0.0) || c->mixed_fas_max_cycles < 0 || c->mixed_linear_vcycles < 1 ||
        (c->mixed_df_residual != 0 && c->mixed_df_residual != 1) ||
        (c->fused_chunk != 0 && (c->fused_chunk < 4 || c->fused_chunk > 128)) ||
        (c->adjoint_store_cofactors != 0 && c->adjoint_store_cofactors != 1) ||
        (c->report_paper_eps != 0 && c->report_paper_eps != 1))
        return set_err(H, RECON_E_INVALID, "bad mixed-precision options");
    H->cfg = *c;
    return RECON_OK;
}

// Device memory, managed memory or page-locked host memory (which kernels
// reach directly); anything else (pageable host memory) is refused.
static bool gpu_reachable(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
           (a.type == cudaMemoryTypeHost && a.devicePointer == p);
}

recon_status recon_deposit_cic(recon_handle *H, const double *pos, long long n_part, double mass,
                               double *rho)
{
    if (!H) return RECON_E_INVALID;
    if (n_part < 0 || (n_part > 0 && !pos) || !rho)
        return set_err(H, RECON_E_INVALID, "bad particle count or NULL pointer");
    if (n_part > 0 && !gpu_reachable(pos))
        return set_err(H, RECON_E_INVALID, "pos must be device or page-locked host memory");
    return cuda_status(H, cic_deposit(pos, n_part, H->N, H->L, mass, rho, H->stream), "cic");
}

recon_status recon_deposit(recon_handle *H, recon_assign scheme, const double *pos, long long n_part,
                           double mass, double *rho)
{
    if (!H) return RECON_E_INVALID;
    if (scheme != RECON_ASSIGN_NGP && scheme != RECON_ASSIGN_CIC && scheme != RECON_ASSIGN_TSC)
        return set_err(H, RECON_E_INVALID, "unknown assignment scheme");
    if (n_part < 0 || (n_part > 0 && !pos) || !rho)
        return set_err(H, RECON_E_INVALID, "bad particle count or NULL pointer");
    if (n_part > 0 && !gpu_reachable(pos))
        return set_err(H, RECON_E_INVALID, "pos must be device or page-locked host memory");
    return cuda_status(H, assign_deposit((int)scheme, pos, n_part, H->N, H->L, mass, rho, H->stream),
                       "deposit");
}

recon_status recon_solve(recon_handle *H, const double *b, double *phi, double tol, int max_cycles,
                         recon_stats *stats)
{
    if (!H) return RECON_E_INVALID;
    if (!b || !phi) return set_err(H, RECON_E_INVALID, "b and phi must be device pointers");
    if (!(tol > 0.0) || max_cycles < 1 || max_cycles > 100000)
        return set_err(H, RECON_E_INVALID, "tol must be > 0 and max_cycles in [1, 100000]");
    H->err.clear();
    H->have_solve = false;
    H->adj.null_ready = false;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    recon_status s = check_domain(H, b);
    if (s != RECON_OK) return s;
    s = H->dtype == RECON_F64 ? solve_f64(H, b, phi, tol, max_cycles, stats)
                              : solve_mixed(H, b, phi, tol, max_cycles, stats);
    if (stats) stats->paper_eps = std::nan("");
    if (stats && H->cfg.report_paper_eps && (s == RECON_OK || s == RECON_E_NOCONV)) {
        // per-plane sums of L_h^2 on the device, added here in plane order
        const int N = H->N;
        cudaError_t e = paper_eps_planes(N, H->L / N, phi, b, stats->compat_c, H->partials, H->stream);
        std::vector<double> planes((size_t)N);
        if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy(planes.data(), H->partials, sizeof(double) * N, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(H, e, "paper_eps");
        double acc = 0.0;
        for (int i = 0; i < N; ++i) acc += planes[i];
        stats->paper_eps = std::sqrt(acc / ((double)N * N * N));
    }
    if (s == RECON_OK) {
        H->last_phi = phi;
        H->last_b = b;
        H->have_solve = true;
    }
    return s;
}

recon_status recon_displace(recon_handle *H, const double *phi, const double *b, double *psi,
                            double *deltaL)
{
    if (!H) return RECON_E_INVALID;
    if (!phi || !b || !psi || !deltaL) return set_err(H, RECON_E_INVALID, "NULL pointer");
    if (!gpu_reachable(psi) || !gpu_reachable(deltaL))
        return set_err(H, RECON_E_INVALID, "psi and deltaL must be device or page-locked host memory");
    return cuda_status(H, displace(H->N, H->L, phi, b, psi, deltaL, H->work64, H->work64b, H->stream),
                       "displace");
}

recon_status recon_smooth_density(recon_handle *H, const double *rho, double R, double floor_, double *b)
{
    if (!H) return RECON_E_INVALID;
    if (!rho || !b) return set_err(H, RECON_E_INVALID, "NULL pointer");
    if (!(R >= 0.0) || !std::isfinite(R) || !(floor_ > 0.0) || !std::isfinite(floor_))
        return set_err(H, RECON_E_INVALID, "R must be >= 0 and floor > 0, both finite");
    return cuda_status(H, smooth_density(H->N, H->L, R, floor_, rho, b, reinterpret_cast<float *>(H->work64),
                                         H->scal + S_SMOOTH_MEAN, H->stream),
                       "smooth_density");
}

recon_status recon_level_scales(recon_handle *H, double *out, int n, int *levels)
{
    if (!H) return RECON_E_INVALID;
    if (n > 0 && !out) return set_err(H, RECON_E_INVALID, "NULL pointer");
    const int coarse = H->nlev - 1;
    if (levels) *levels = coarse;
    if (n <= 0 || coarse <= 0) return RECON_OK;
    std::vector<double> scal(recon::S_COUNT);
    cudaError_t e = cudaStreamSynchronize(H->stream);
    if (e == cudaSuccess) e = cudaMemcpy(scal.data(), H->scal, sizeof(double) * recon::S_COUNT, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(H, e, "recon_level_scales");
    for (int l = 1; l <= coarse && l <= n; ++l) out[l - 1] = scal[recon::slot_scale(l)];
    return RECON_OK;
}

recon_status recon_gaussianise(recon_handle *H, const double *field, double *out)
{
    if (!H) return RECON_E_INVALID;
    if (!field || !out) return set_err(H, RECON_E_INVALID, "NULL pointer");
    if (field == out) return set_err(H, RECON_E_INVALID, "field and out must not alias");
    return cuda_status(H, gaussianise(H, field, (size_t)H->N * H->N * H->N, out), "gaussianise");
}

recon_status recon_displace_fp64(recon_handle *H, const double *phi, const double *b, double *psi,
                                 double *deltaL)
{
    if (!H) return RECON_E_INVALID;
    if (!phi || !b || !psi || !deltaL) return set_err(H, RECON_E_INVALID, "NULL pointer");
    if (!gpu_reachable(psi) || !gpu_reachable(deltaL))
        return set_err(H, RECON_E_INVALID, "psi and deltaL must be device or page-locked host memory");
    return cuda_status(H, displace_fp64(H->N, H->L, phi, b, psi, deltaL, H->work64, H->work64b, H->stream),
                       "displace_fp64");
}

recon_status recon_displace_adjoint(recon_handle *H, const double *phi, const double *b,
                                    const double *gbar_psi, const double *gbar_deltaL,
                                    double *gbar_phi, double *gbar_b)
{
    if (!H) return RECON_E_INVALID;
    if (!phi || !b || !gbar_phi || !gbar_b) return set_err(H, RECON_E_INVALID, "NULL pointer");
    const size_t n = (size_t)H->N * H->N * H->N;
    // byte ranges: gbar_psi holds 3 N^3 doubles, every other array N^3; an
    // output may not overlap any input or the other output
    auto overlap = [](const void *a, size_t na, const void *b, size_t nb) {
        if (!a || !b) return false;
        const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
        return x < y + nb * sizeof(double) && y < x + na * sizeof(double);
    };
    const void *ins[4] = {phi, b, gbar_psi, gbar_deltaL};
    const size_t nin[4] = {n, n, 3 * n, n};
    for (int a = 0; a < 4; ++a)
        if (overlap(ins[a], nin[a], gbar_phi, n) || overlap(ins[a], nin[a], gbar_b, n))
            return set_err(H, RECON_E_INVALID, "gbar_phi and gbar_b must not overlap an input");
    if (overlap(gbar_phi, n, gbar_b, n)) return set_err(H, RECON_E_INVALID, "gbar_phi and gbar_b must not overlap");
    H->err.clear();
    if (!H->dadj && cudaMalloc(&H->dadj, sizeof(double) * 9 * n) != cudaSuccess) {
        cudaGetLastError();
        H->dadj = nullptr;
        return set_err(H, RECON_E_OOM, "recon_displace_adjoint: cannot allocate its 9 N^3 doubles");
    }
    return cuda_status(H, displace_adjoint(H->N, H->L, phi, b, gbar_psi, gbar_deltaL, gbar_phi, gbar_b,
                                           H->work64, H->work64b, H->dadj, H->stream),
                       "displace_adjoint");
}

recon_status recon_adjoint(recon_handle *H, const double *gbar_phi, double *gbar_b)
{
    if (!H) return RECON_E_INVALID;
    if (!gbar_phi || !gbar_b) return set_err(H, RECON_E_INVALID, "NULL pointer");
    if (!H->have_solve) return set_err(H, RECON_E_INVALID, "no successful recon_solve on this handle");
    H->err.clear();
    return adjoint(H, gbar_phi, gbar_b);
}

const char *recon_last_error(const recon_handle *H)
{
    return H ? H->err.c_str() : g_create_err.c_str();
}

// ---------------------------------------------------------------- steps
static bool step_size_ok(int N) { return N >= 4 && N % 2 == 0 && N <= kMaxN; }

recon_status recon_step_sweep(int N, double h, int prec, int rule, void *theta, const void *g,
                              double c, int sweeps, void *work, void *stream)
{
    if (!step_size_ok(N) || !(h > 0) || sweeps < 0 || !theta || !g || !work || (rule != 0 && rule != 1))
        return RECON_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    set_fused_chunk(0);
    cudaError_t e = prec == 0
        ? sweep<double>(N, h, rule, (double *)theta, (const double *)g, nullptr, c, sweeps, (double *)work, s)
        : prec == 1 ? sweep<float>(N, h, rule, (float *)theta, (const float *)g, nullptr, c, sweeps, (float *)work, s)
                    : cudaErrorInvalidValue;
    if (prec != 0 && prec != 1) return RECON_E_INVALID;
    return e == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_residual(int N, double h, const double *theta, const double *g, double c,
                                 double *r, void *stream)
{
    if (!step_size_ok(N) || !(h > 0) || !theta || !g || !r) return RECON_E_INVALID;
    return residual_write(N, h, theta, g, nullptr, c, r, (cudaStream_t)stream) == cudaSuccess
               ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_det(int N, double h, const double *theta, double *det, void *stream)
{
    if (!step_size_ok(N) || !(h > 0) || !theta || !det) return RECON_E_INVALID;
    return det_write(N, h, theta, det, (cudaStream_t)stream) == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_restrict(int Nf, int prec, const void *fine, void *coarse, void *stream)
{
    if (Nf < 2 || Nf % 2 != 0 || Nf > kMaxN || !fine || !coarse || (prec != 0 && prec != 1))
        return RECON_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = prec == 0 ? restrict_plain<double>(Nf, (const double *)fine, (double *)coarse, s)
                              : restrict_plain<float>(Nf, (const float *)fine, (float *)coarse, s);
    return e == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_prolong_add(int Nc, int prec, const void *cnew, const void *cold,
                                    double scale, void *fine, void *stream)
{
    if (Nc < 1 || 2 * Nc > kMaxN || !cnew || !fine || (prec != 0 && prec != 1)) return RECON_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = prec == 0
        ? prolong_add<double>(Nc, (const double *)cnew, (const double *)cold, nullptr, scale, (double *)fine, s)
        : prolong_add<float>(Nc, (const float *)cnew, (const float *)cold, nullptr, scale, (float *)fine, s);
    return e == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_coarse_solve(int N, double h, int prec, int rule, void *theta,
                                     const void *g, double c, int max_sweeps, double rtol,
                                     void *work, int *sweeps_done, void *stream)
{
    if (!step_size_ok(N) || (long)N * N * N > kMaxCoarseCells || !(h > 0) || max_sweeps < 1 ||
        !(rtol >= 0) || !theta || !g || !work || (rule != 0 && rule != 1) || (prec != 0 && prec != 1))
        return RECON_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = prec == 0
        ? coarse_solve<double>(N, h, rule, (double *)theta, (const double *)g, nullptr, c, max_sweeps,
                               rtol, (double *)work, sweeps_done, s)
        : coarse_solve<float>(N, h, rule, (float *)theta, (const float *)g, nullptr, c, max_sweeps,
                              rtol, (float *)work, sweeps_done, s);
    return e == cudaSuccess ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_cic_cells(const double *pos, long long n, int N, double L, int *cells,
                                  double *frac, void *stream)
{
    if (n < 0 || N < 1 || N > kMaxN || !(L > 0) || (n > 0 && (!pos || !cells || !frac))) return RECON_E_INVALID;
    return cic_cells(pos, n, N, L, cells, frac, (cudaStream_t)stream) == cudaSuccess ? RECON_OK
                                                                                     : RECON_E_CUDA;
}

recon_status recon_step_linear_sweep(int N, double h, float *e, const float *f, const float *theta,
                                     int sweeps, float *work, void *stream)
{
    if (!step_size_ok(N) || !(h > 0) || sweeps < 0 || !e || !f || !theta || !work)
        return RECON_E_INVALID;
    set_fused_chunk(0);
    return linear_sweep(N, h, e, f, theta, sweeps, work, (cudaStream_t)stream) == cudaSuccess
               ? RECON_OK : RECON_E_CUDA;
}

recon_status recon_step_jacobian_apply(int N, double h, const double *theta, const double *v,
                                       double *out, void *stream)
{
    if (!step_size_ok(N) || !(h > 0) || !theta || !v || !out) return RECON_E_INVALID;
    return jacobian_apply(N, h, theta, v, out, (cudaStream_t)stream) == cudaSuccess ? RECON_OK
                                                                                    : RECON_E_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------- diagnostics
#include <atomic>
static std::atomic<unsigned long long> g_launches{0};
void recon::note_launch(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void recon::set_thread_error(const char *msg) { g_create_err = msg ? msg : ""; }
void recon::unnote_launch(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
unsigned long long recon::launch_count() { return g_launches.load(); }
extern "C" unsigned long long recon_kernel_launches(void) { return g_launches.load(); }
