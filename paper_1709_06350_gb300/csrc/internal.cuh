// internal.cuh -- the handle and the launchers shared by librecon's
// translation units (not part of the public ABI).
#pragma once

#include <string>

#include "common.cuh"

constexpr int kMaxLevels = 16;
constexpr int kMaxRedBlocks = 2048;   // grid cap of every reducing kernel
constexpr int kFusedMinN = 128;       // grids of at least this size use the fused sweeps

// Workspace of the adjoint (allocated at its first call): the potential of
// every coarse level, the six cofactor arrays of every level, the iterate and
// right side of every coarse level, the null vector of J^T.
// workspace of recon_gaussianise (allocated at its first call)
struct GaussWork {
    size_t cap = 0;
    unsigned long long *key[2] = {};
    unsigned *idx[2] = {};
    unsigned *counts = nullptr, *segsum = nullptr;
    double *moments = nullptr;
};

struct AdjWork {
    bool ready = false;
    bool stored0 = true;       // the finest level's cofactors are kept (else formed in every J^T)
    bool null_ready = false;   // cofactors and null vector match the last solve
    double null_rel = 0.0;
    double *th[kMaxLevels] = {}, *cof[kMaxLevels] = {}, *lam[kMaxLevels] = {}, *f[kMaxLevels] = {};
    double *nvec = nullptr;
};

struct recon_handle {
    int N = 0;
    double L = 0.0, h = 0.0;
    recon_dtype dtype = RECON_F64;
    recon_config cfg{};
    cudaStream_t stream = nullptr;

    int nlev = 0;
    int Nl[kMaxLevels] = {};
    double hl[kMaxLevels] = {};

    // FP64 hierarchy: level 0 theta / g are the caller's phi / b.
    double *t64[kMaxLevels] = {}, *g64[kMaxLevels] = {}, *told64[kMaxLevels] = {},
           *aux64[kMaxLevels] = {};
    double *work64 = nullptr;    // N^3: smoother ping-pong, displace numerator
    double *work64b = nullptr;   // N^3: displace denominator, adjoint scratch

    // FP32 hierarchy (MIXED): FAS theta / g / saved theta / aux, linear e / f.
    float *t32[kMaxLevels] = {}, *g32[kMaxLevels] = {}, *told32[kMaxLevels] = {},
          *aux32[kMaxLevels] = {};
    float *e32[kMaxLevels] = {}, *f32[kMaxLevels] = {};
    float *work32 = nullptr;
    float *lo32 = nullptr, *blo32 = nullptr;   // low halves of phi and b (double-float)
    float *cof32[kMaxLevels] = {};             // cofactors of I + H theta32, [6][n_l] (levels below kFusedMinN)

    double *scal = nullptr;      // device scalars (recon::Slot)
    double *partials = nullptr;  // kMaxRedBlocks x 4 doubles
    int *iscratch = nullptr;     // small device ints
    double *hscal = nullptr;     // pinned host mirror of scal

    const double *last_phi = nullptr;
    const double *last_b = nullptr;
    bool have_solve = false;

    AdjWork adj;
    GaussWork gauss;
    double *dadj = nullptr;   // 9 N^3: recon_displace_adjoint (allocated at its first call)
    int adj_cycles = 0;
    double adj_rel = 0.0;

    std::string err;
};

namespace recon {

// Kernels launched by this library in this process (diagnostics).
void note_launch(unsigned long long n = 1);

void unnote_launch(unsigned long long n);
unsigned long long launch_count();

// Dynamic shared-memory limits of the fused kernels (set before any capture).
cudaError_t prepare_kernels();
// Register-blocked fused FP32 sweeps (recon_sweep.cu): sides a multiple of 64.
cudaError_t prepare_reg_sweeps();
bool reg_sweep_ok(int N, const float *src, const float *dst, const float *g, const float *th);
int reg_sweep_chunk(int N, int want);
// one sweep src -> dst; lin: J e = f with theta th (else the FAS cubic with
// right side g + c, c from cptr or cval); chunk: planes per CTA (0 = by size)
// gshift (nullable): a device scalar.  FAS: subtracted from every value the
// sweep stores (a gauge shift folded into the sweep: the update depends only
// on differences of theta).  LIN: subtracted from the right side f.
cudaError_t reg_sweep_launch(bool lin, int N, const float *src, float *dst, const float *g, const float *th,
                             const double *cptr, double cval, float ih2, float h2_6, int rule, int chunk,
                             cudaStream_t s, const double *gshift = nullptr);
// Planes per CTA of the fused sweeps enqueued next on this host thread (0 = auto).
void set_fused_chunk(int c);

// Message returned by recon_last_error(NULL) on this thread.
void set_thread_error(const char *msg);
// per-plane sums of L_h^2 (the paper's epsilon) over a whole N^3 grid, N
// doubles into out (recon_slab.cu)
cudaError_t paper_eps_planes(int N, double h, const double *theta, const double *g, double c, double *out,
                             cudaStream_t s);

// ---- multigrid launchers (recon_mg.cu); all asynchronous on `s`.
// gshift (nullable): a device scalar subtracted from theta before the first
// sweep (folded into it where the register-blocked kernel runs)
template <typename T>
cudaError_t sweep(int N, double h, int rule, T *t, const T *g, const double *cptr,
                  double cval, int sweeps, T *work, cudaStream_t s, const double *gshift = nullptr);
cudaError_t residual_write(int N, double h, const double *t, const double *g,
                           const double *cptr, double cval, double *r, cudaStream_t s);
cudaError_t det_write(int N, double h, const double *t, double *out, cudaStream_t s);
template <typename T>
cudaError_t restrict_plain(int Nf, const T *fine, T *coarse, cudaStream_t s);
template <typename T>
cudaError_t prolong_add(int Nc, const T *cnew, const T *cold, const double *pscale,
                        double scale, T *fine, cudaStream_t s);
template <typename T>
cudaError_t coarse_solve(int N, double h, int rule, T *t, const T *g, const double *cptr,
                         double cval, int max_sweeps, double rtol, T *work, int *sweeps_out,
                         cudaStream_t s);
cudaError_t jacobian_apply(int N, double h, const double *t, const double *v, double *out,
                           cudaStream_t s);
cudaError_t linear_sweep(int N, double h, float *e, const float *f, const float *th, int sweeps,
                         float *work, cudaStream_t s);

// ---- the solvers (recon_mg.cu)
recon_status solve_f64(recon_handle *H, const double *b, double *phi, double tol,
                       int max_cycles, recon_stats *st);
recon_status solve_mixed(recon_handle *H, const double *b, double *phi, double tol,
                         int max_cycles, recon_stats *st);
recon_status check_domain(recon_handle *H, const double *b);

// capture-safe phases of the mixed solve (recon_mg.cu): enqueue work on
// H->stream and never synchronise
cudaError_t mixed_start(recon_handle *H, const double *b, const double *phi);
cudaError_t mixed_fas_cycle(recon_handle *H);
cudaError_t mixed_switch(recon_handle *H, const double *b, double *phi, bool from_phi);
cudaError_t mixed_residual(recon_handle *H, const double *b, const double *phi);
cudaError_t mixed_correct(recon_handle *H, double *phi);
cudaError_t mixed_finish(recon_handle *H, double *phi, bool converged);

// ---- CIC and displacement (recon_cic.cu)
cudaError_t cic_cells(const double *pos, long long n, int N, double L, int *cells,
                      double *frac, cudaStream_t s);
cudaError_t cic_deposit(const double *pos, long long n, int N, double L, double mass,
                        double *rho, cudaStream_t s);
// scheme: 0 NGP, 1 CIC, 2 TSC
cudaError_t assign_deposit(int scheme, const double *pos, long long n, int N, double L, double mass,
                           double *rho, cudaStream_t s);
// FP64 form of the reconstruction output, and its adjoint (recon_cic.cu);
// num, den: N^3 doubles of scratch each, G9: 9 N^3 doubles
cudaError_t displace_fp64(int N, double L, const double *phi, const double *b, double *psi,
                          double *deltaL, double *num, double *den, cudaStream_t s);
cudaError_t displace_adjoint(int N, double L, const double *phi, const double *b, const double *gpsi,
                             const double *gdl, double *gphi, double *gb, double *num, double *den,
                             double *G9, cudaStream_t s);
// ---- adjoint (recon_adjoint.cu)
recon_status adjoint(recon_handle *H, const double *gbar, double *lam);
void adj_free(recon_handle *H);
cudaError_t gauss_alloc(recon_handle *H, size_t n);
void gauss_free(recon_handle *H);
cudaError_t gaussianise(recon_handle *H, const double *v, size_t n, double *g);

// ---- density preparation (recon_smooth.cu): Gaussian window of radius R,
// floor, mean 1; w32: 2 N^3 floats of scratch; mean: one device double
cudaError_t smooth_density(int N, double L, double R, double floor_, const double *rho, double *b, float *w32,
                           double *mean, cudaStream_t s);

// phi -> (hi, lo) FP32 parts (recon_mg.cu)
__global__ void k_split_df(const double *__restrict__ a, float *__restrict__ hi, float *__restrict__ lo,
                           size_t n);
cudaError_t displace(int N, double L, const double *phi, const double *b, double *psi,
                     double *deltaL, double *scratch, double *split, cudaStream_t s);

}  // namespace recon
