/*
 * recon.h -- C ABI of librecon: GB300 (sm_103a) multigrid solve of the
 * mass-conservation (Monge-Ampere) equation of Shi, Cautun & Li,
 * "New method for initial density reconstruction" (arXiv:1709.06350).
 *
 * The library finds the displacement potential phi (the paper's theta,
 * Sec. II eq. theta0: Theta = x^2/2 + theta) on a periodic N^3 grid with
 *
 *     det(I + H_h phi) = b + c,      mean(phi) = 0,                     (*)
 *
 * where b = 1 + delta is the normalised final density (eq. basic_eqs),
 * H_h the second-order Hessian stencils of eq. discrete_examples and c one
 * scalar that makes the discrete problem solvable (the discrete determinant
 * is not exactly mass-conserving; c is O(h^2) and is reported).
 *
 * Conventions for every call
 *   - grids are N^3 doubles in C order [i][j][k] (k fastest, i = x axis),
 *     cell centres at (i + 1/2) h, h = L / N, periodic;
 *   - every array pointer is a DEVICE pointer owned by the caller unless the
 *     argument says "host"; the handle owns only its workspace;
 *   - work is enqueued on the handle's stream (recon_set_stream; default the
 *     legacy default stream).  recon_solve synchronises the stream once per
 *     V-cycle to read the convergence scalar; the other calls return without
 *     synchronising;
 *   - no call throws; each returns a recon_status and, on failure, stores a
 *     message retrievable with recon_last_error (per handle);
 *   - a handle is not thread-safe: use one handle per host thread / stream.
 */
#ifndef RECON_H
#define RECON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RECON_OK = 0,
    RECON_E_INVALID = 1,        /* bad argument (size, pointer, option)            */
    RECON_E_DOMAIN = 2,         /* b <= 0 or non-finite somewhere                  */
    RECON_E_NOCONV = 3,         /* max_cycles reached before the tolerance         */
    RECON_E_DIVERGED = 4,       /* residual became non-finite or grew 1e3-fold     */
    RECON_E_CUDA = 5,           /* a CUDA runtime call or kernel launch failed     */
    RECON_E_OOM = 6,            /* device allocation failed                        */
    RECON_E_TIMEOUT = 7,        /* a bounded device wait ran out                   */
    RECON_E_UNIMPLEMENTED = 8
} recon_status;

typedef enum {
    RECON_F64 = 0,              /* every step in FP64                              */
    RECON_MIXED = 1             /* FP32 multigrid inside a defect correction whose
                                   fine-grid residual and phi keep (near-)FP64
                                   precision; phi is returned in FP64            */
} recon_dtype;

typedef enum {
    RECON_RULE_NEWTON1 = 0,     /* one safeguarded Newton step on the cell cubic   */
    RECON_RULE_EXACT = 1        /* the paper's update: largest root of the cubic   */
} recon_rule;

typedef enum {
    RECON_START_FMG = 0,        /* nested iteration from phi = 0 on the coarsest
                                   grid; the contents of phi on entry are ignored  */
    RECON_START_GUESS = 1       /* V-cycles start from phi as passed in (resume)   */
} recon_start;

/* Solver options.  Defaults (recon_create): nu1 = nu2 = 2,
 * coarse_max_sweeps = 200, coarse_rtol = 1e-3, rule = NEWTON1, start = FMG,
 * scale_floor = 0.5, mixed_switch_rtol = 1e-4, mixed_fas_max_cycles = 12,
 * mixed_linear_vcycles = 2, mixed_df_residual = 1, fused_chunk = 0,
 * adjoint_store_cofactors = 0, report_paper_eps = 0. */
typedef struct {
    int nu1, nu2;               /* pre- / post-smoothing sweeps per level          */
    int coarse_max_sweeps;      /* coarsest grid: sweep cap                        */
    double coarse_rtol;         /* coarsest grid: stop when the mean-free rms
                                   residual falls by this factor                   */
    int rule;                   /* recon_rule                                      */
    int start;                  /* recon_start                                     */
    double scale_floor;         /* scaled-defect safeguard: the coarse right side
                                   is det_H(R phi) + s R r with the largest s <= 1
                                   keeping it >= (1 - scale_floor) det_H(R phi);
                                   the correction is divided by s (<= 0: s = 1)   */
    double mixed_switch_rtol;   /* MIXED: FP32 FAS cycles until this relative
                                   residual, then FP64 defect correction           */
    int mixed_fas_max_cycles;   /* MIXED: cap on the FP32 FAS cycles               */
    int mixed_linear_vcycles;   /* MIXED: FP32 linear V-cycles per correction      */
    int mixed_df_residual;      /* MIXED: 1 = the fine-grid residual and phi are
                                   double-float pairs (hi + lo floats, 48-bit
                                   significand, FP32 pipes) while iterating;
                                   0 = plain FP64 arithmetic for both          */
    int fused_chunk;            /* planes per thread block of the fused smoother
                                   sweeps (grids >= 128^3): 4..128, 0 = by size;
                                   on grids of side a multiple of 64 it is taken
                                   down to a multiple of 4 that divides N       */
    int adjoint_store_cofactors; /* recon_adjoint: 0 = the finest grid's six
                                   cofactor fields of I + H phi are formed
                                   again from phi in every application of J^T
                                   (grids of side a multiple of 32; saves 48 N^3
                                   bytes); 1 = kept in memory (faster)          */
    int report_paper_eps;       /* recon_solve: 1 = fill recon_stats.paper_eps
                                   (one FP64 pass with the cubic's largest root
                                   per cell: ~0.3 s at 512^3); 0 = NaN         */
} recon_config;

#define RECON_HISTORY_MAX 64

typedef struct {
    int cycles;                 /* F64: finest-grid FAS V-cycles.
                                   MIXED: FP32 FAS V-cycles                        */
    int outer_iterations;       /* MIXED: FP64 defect-correction iterations        */
    double rel_residual;        /* ||r - mean r||_2 / ||b - 1||_2 at exit, r the
                                   FP64 residual b + c - det(I + H phi)            */
    double compat_c;            /* the scalar c of (*)                             */
    double paper_eps;           /* the paper's convergence measure (Sec. II.A.2):
                                   rms over cells of L_h = lap_h phi - Sigma with
                                   Sigma = largest root of the cell cubic (eq.
                                   root) - 3, rhs = b + c; FP64, at exit; NaN
                                   unless report_paper_eps = 1                  */
    double seconds;             /* wall time of the call                           */
    int n_history;              /* entries of history[] that are set               */
    double history[RECON_HISTORY_MAX]; /* relative residual after each cycle /
                                   outer iteration, in order                       */
} recon_stats;

typedef struct recon_handle recon_handle;

/* Create a solver for an N^3 grid of side L (Mpc/h or any length unit;
 * phi comes out in that unit squared).  N must be even, 4 <= N <= 1024, and the
 * multigrid hierarchy (halve N while the half is even and >= 4) must end at
 * a coarsest grid of at most 16^3; L > 0.  Allocates the whole workspace
 * (recon_workspace_bytes) with cudaMalloc on the current device.
 * Errors: RECON_E_INVALID, RECON_E_OOM, RECON_E_CUDA. */
recon_status recon_create(int N, double L, recon_dtype dtype, recon_handle **out);

/* Free the workspace and the handle (NULL is ignored). */
void recon_destroy(recon_handle *h);

/* Bytes of device workspace a handle of this size holds (0 if invalid). */
size_t recon_workspace_bytes(int N, recon_dtype dtype);

/* Enqueue all later work of this handle on `stream` (a cudaStream_t). */
recon_status recon_set_stream(recon_handle *h, void *stream);

/* Read / replace the solver options (host structs). */
recon_status recon_get_config(const recon_handle *h, recon_config *cfg);
recon_status recon_set_config(recon_handle *h, const recon_config *cfg);

/* Cloud-in-cell density assignment (Sec. I footnote).
 * pos: n_part x 3 doubles (x, y, z) in [0, L) (wrapped if not), in device
 *      memory or in page-locked host memory (cudaHostAlloc / cudaHostRegister,
 *      or a pinned framework tensor): the kernel then reads the positions
 *      over the host link itself, with no staging copy.
 * rho: device N^3, ACCUMULATED into (zero it first for a fresh density);
 * each particle adds mass * prod_axis w, w = (1 - f, f) on cells
 * (i0, i0 + 1), u = x * (N / L) - 1/2, i0 = floor(u) mod N, f = u - floor(u).
 * Use mass = N^3 / n_part for a density normalised to mean 1.
 * Errors: RECON_E_INVALID (n_part < 0, null pointers, pos in pageable host
 * memory), RECON_E_CUDA. */
recon_status recon_deposit_cic(recon_handle *h, const double *pos, long long n_part,
                               double mass, double *rho);

/* Density assignment by nearest grid point, cloud in cell or triangular-
 * shaped cloud (Sec. I footnote: the method works with any of the three).
 * Cell i covers [i h, (i+1) h); along each axis u = x (N / L), i = floor(u)
 * mod N, t = u - floor(u):
 *   RECON_ASSIGN_NGP: mass on cell i;
 *   RECON_ASSIGN_CIC: as recon_deposit_cic;
 *   RECON_ASSIGN_TSC: the quadratic B-spline, weights (1 - t)^2 / 2,
 *                     3/4 - (t - 1/2)^2, t^2 / 2 on cells i-1, i, i+1,
 * times the product over the three axes.  pos, rho, mass and the errors as
 * for recon_deposit_cic (rho is accumulated into). */
typedef enum { RECON_ASSIGN_NGP = 0, RECON_ASSIGN_CIC = 1, RECON_ASSIGN_TSC = 2 } recon_assign;
recon_status recon_deposit(recon_handle *h, recon_assign scheme, const double *pos, long long n_part,
                           double mass, double *rho);

/* Solve (*) (Sec. II.A: Gauss-Seidel relaxation of eq. update inside the
 * FAS V-cycles of eqs. PDE_H and corrections).
 * b:   device N^3, 1 + delta, every entry finite and > 0 (else RECON_E_DOMAIN).
 * phi: device N^3; on entry the initial guess when start = GUESS (ignored
 *      for FMG); on exit the mean-free solution.
 * tol: stop when ||r - mean r||_2 / ||b - 1||_2 < tol (r the FP64 residual).
 * max_cycles: cap on finest-grid cycles (F64) / outer iterations (MIXED).
 * stats: host, nullable.
 * Returns RECON_OK, RECON_E_NOCONV (phi holds the last iterate),
 * RECON_E_DIVERGED, RECON_E_DOMAIN, RECON_E_INVALID, RECON_E_CUDA.
 * The handle keeps a pointer to phi's values for recon_adjoint (it copies
 * nothing; do not change phi between recon_solve and recon_adjoint). */
recon_status recon_solve(recon_handle *h, const double *b, double *phi, double tol,
                         int max_cycles, recon_stats *stats);

/* Reconstruction output (Sec. II.B steps B2-B3, eq. reconstructed_density,
 * and x - q = -grad theta of Sec. III.B), restated on the grid:
 *   psi  (3 x N^3, component-major) = -(central gradient of phi);
 *   q_c = x_c + grad phi (mod L) for every Eulerian cell centre x_c;
 *   v_c = 3 - tr((I + H phi)^-1)   (div_q chi, chi = q - x);
 *   deltaL (N^3, on the Lagrangian grid) =
 *       CIC(q_c, b_c v_c) / max(CIC(q_c, b_c), 1e-12).
 * phi, b: device N^3.  psi and deltaL: device memory or page-locked host
 * memory (written by the kernels over the host link).  psi is FP64
 * differencing; v, the CIC weights and the two sums are FP32 (deltaL to
 * ~1e-6 absolute).  Uses 2 N^3 doubles of handle workspace.
 * Errors: RECON_E_INVALID (null pointers, an output in pageable host
 * memory), RECON_E_CUDA. */
recon_status recon_displace(recon_handle *h, const double *phi, const double *b,
                            double *psi, double *deltaL);

/* The same output as recon_displace (Sec. II.B restated above), evaluated in
 * plain FP64: per cell q = x + g (mod L) with x = (i + 1/2) h and g the
 * central-difference gradient, the CIC cell and fraction of u = q N/L - 1/2
 * per axis, v and both CIC sums in FP64 (FP64 atomics).  This is the map
 * whose gradient recon_displace_adjoint returns; use it where a gradient is
 * checked against finite differences.  Same arguments, workspace and errors
 * as recon_displace. */
recon_status recon_displace_fp64(recon_handle *h, const double *phi, const double *b,
                                 double *psi, double *deltaL);

/* Adjoint of the reconstruction output (the map of recon_displace_fp64;
 * Sec. II.B, carried by the chain rule, no counterpart printed in the
 * paper): given gbar_psi = dLoss/dpsi (device 3 N^3, component-major, or
 * NULL for zero) and gbar_deltaL = dLoss/ddeltaL (device N^3 or NULL),
 * writes gbar_phi = dLoss/dphi and gbar_b = dLoss/db (device N^3 each,
 * overwritten) at the given phi and b (device N^3):
 *   gN = gbar_deltaL / max(den, 1e-12),  gD = -gbar_deltaL num / den^2,
 *   per cell: gbar_b = v sum W gN + sum W gD,  gv = b sum W gN,
 *             gq = sum (b v gN + b gD) dW/dq  over the 8 CIC corners W,
 *   gbar_phi = sum_ab D_ab(gv (A^-2)_ab) - sum_d D_d(gq_d - gbar_psi_d),
 * with A = I + H phi, D_ab the stencils of eq. discrete_examples and D_d
 * central differences.  The CIC weights are piecewise linear, so the map is
 * differentiable except where some q lies on a cell face.  For a loss on
 * the output of a solve, pass gbar_phi on to recon_adjoint and add its
 * gbar_b to this one.  The first call allocates 9 N^3 doubles of workspace,
 * held by the handle until recon_destroy; also uses 2 N^3 doubles of the
 * handle workspace.  Outputs must not overlap an input or each other
 * (byte ranges: gbar_psi 3 N^3 doubles, every other array N^3).
 * Errors: RECON_E_INVALID, RECON_E_OOM, RECON_E_CUDA. */
recon_status recon_displace_adjoint(recon_handle *h, const double *phi, const double *b,
                                    const double *gbar_psi, const double *gbar_deltaL,
                                    double *gbar_phi, double *gbar_b);

/* Density preparation before the solve: Gaussian smoothing, floor, mean 1.
 *   b = max(IDFT(DFT(rho) exp(-k^2 R^2 / 2)), floor) / mean(...)
 * with k the box's wave vectors (2 pi m / L per axis, |m| <= N/2): the
 * Gaussian window of width R (length units of L) that Sec. III applies to
 * its density fields; the floor keeps every cell's right side positive
 * (empty assignment cells) and the final division restores mean 1.  The
 * window is applied as three circular convolutions (k, j, i) with the
 * inverse DFT of the 1-D window, truncated where it falls below 1e-9 of its
 * centre, in FP32 taps and sums: b carries ~1e-7 relative rounding for R of
 * a few cells; below ~1.5 cells the window is not small at the grid's
 * Nyquist frequency, the kernel spans the whole periodic line (up to N taps:
 * exact, slower, rounding growing with the tap count).
 * rho, b: device N^3 (they may be the same array).  R >= 0 (0: no
 * smoothing), floor > 0.  Uses the handle's N^3-double workspace.
 * Errors: RECON_E_INVALID (null pointers, R < 0, floor <= 0 or non-finite),
 * RECON_E_CUDA. */
recon_status recon_smooth_density(recon_handle *h, const double *rho, double R, double floor, double *b);

/* The scaled-defect factor s of each coarse level in the last FAS V-cycle
 * the handle ran (Sec. II.A.3, the coarse right side det_H(R phi) + s R r
 * with the correction divided by s): out[l - 1] for level l = 1 .. L - 1
 * (level 0 the finest grid, L the number of levels), at most n values; 1 =
 * no scaling, 0 = the coarse correction was skipped.  For RECON_MIXED the
 * factors of the last FP32 FAS cycle.  Synchronizes the handle's stream.
 * *levels (nullable) receives L - 1.
 * Errors: RECON_E_INVALID (null handle or out with n > 0), RECON_E_CUDA. */
recon_status recon_level_scales(recon_handle *h, double *out, int n, int *levels);

/* 1-point Gaussianisation of an N^3 field (Sec. III: tried on delta_r),
 * read as the rank mapping
 *     out_i = mean + std * Phi^-1((rank_i + 1/2) / N^3),
 * rank_i the position of field_i in ascending order with ties broken by
 * position (-0 equals +0), mean and std (population) of field.  field, out:
 * device N^3, distinct; field must be finite.  The probability and the
 * quantile are FP64 (distinct ranks give distinct outputs at any size up to
 * 1024^3).  The first call allocates
 * 24 N^3 bytes of workspace, held by the handle until recon_destroy.
 * Errors: RECON_E_INVALID, RECON_E_OOM, RECON_E_CUDA. */
recon_status recon_gaussianise(recon_handle *h, const double *field, double *out);

/* Adjoint of the last recon_solve on this handle (implicit-function theorem
 * on (*)): given gbar_phi = dLoss/dphi (device N^3), writes
 * gbar_b = dLoss/db (device N^3, zero-sum), i.e. lam with
 *   J^T lam + mu 1 = gbar_phi,  sum(lam) = 0,  J = d det(I + H phi)/d phi.
 * Errors: RECON_E_INVALID (no previous solve), RECON_E_NOCONV,
 * RECON_E_CUDA, RECON_E_UNIMPLEMENTED (not available in this build). */
recon_status recon_adjoint(recon_handle *h, const double *gbar_phi, double *gbar_b);

/* ---------------------------------------------------------------------------
 * Batches: many independent MIXED solves (uneven N allowed) advanced together.
 * Each realisation has its own handle and stream; every phase of the solve
 * for all realisations is one CUDA-graph launch (graphs are captured at the
 * first solve and reused while the field pointers and options stay the
 * same).  All realisations run the same number of FP32 FAS cycles (until each
 * reached mixed_switch_rtol or stalled) and correction iterations (until each
 * met tol; the ones that met it earlier keep refining). */
typedef struct recon_batch recon_batch;

/* count realisations of sizes N[i] (rules of recon_create) and boxes L[i]. */
recon_status recon_batch_create(int count, const int *N, const double *L, recon_batch **out);
void recon_batch_destroy(recon_batch *batch);

/* The graphs are launched on `stream` (NULL: the batch's own stream). */
recon_status recon_batch_set_stream(recon_batch *batch, void *stream);

/* Handle of realisation i (for recon_set_config / recon_get_config and
 * recon_adjoint after a batch solve); owned by the batch. */
recon_handle *recon_batch_handle(recon_batch *batch, int i);

/* Solve realisation i for b[i] into phi[i] (host arrays of device pointers,
 * each field as in recon_solve).  stats: host array of count (nullable).
 * Returns RECON_OK when every realisation met tol, else RECON_E_NOCONV /
 * RECON_E_DIVERGED / RECON_E_DOMAIN / RECON_E_CUDA (message:
 * recon_batch_last_error). */
recon_status recon_batch_solve(recon_batch *batch, const double *const *b, double *const *phi,
                               double tol, int max_cycles, recon_stats *stats);
const char *recon_batch_last_error(const recon_batch *batch);

/* Message of the last failing call on this handle ("" if none); a handle
 * of NULL gives the last message of recon_create or
 * recon_step_coarse_solve_noalloc on this thread. */
const char *recon_last_error(const recon_handle *h);

/* Name of a status code. */
const char *recon_status_string(recon_status s);

/* Number of CUDA kernels this library has launched in this process so far
 * (all handles and step calls; diagnostics for launch accounting). */
unsigned long long recon_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* RECON_H */
