/*
 * recon_steps.h -- single steps of the librecon solve, exposed one kernel
 * (or one short kernel sequence) per call so that each step can be checked
 * against an independent implementation on the same inputs.
 *
 * Every pointer is a DEVICE pointer owned by the caller; `prec` selects the
 * element type of the grid arrays (0 = double, 1 = float); every call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream);
 * grids are N^3 in C order [i][j][k], periodic, spacing h.  The returned
 * status is RECON_E_INVALID for a bad size / option, RECON_E_CUDA when a
 * launch fails, else RECON_OK.  Scalars that the full solver keeps on the
 * device (c, scale factors) are passed here as host values.
 */
#ifndef RECON_STEPS_H
#define RECON_STEPS_H

#include "recon.h"

#ifdef __cplusplus
extern "C" {
#endif

/* `sweeps` red-black Gauss-Seidel sweeps of eq. update (Sec. II.A.2) on
 * det(I + H theta) = g + c.  Red = (i+j+k) even, then black; within one
 * colour every update reads the values held at the start of that colour
 * pass.  rule: recon_rule.  work: N^3 scratch of the same type.  N even. */
recon_status recon_step_sweep(int N, double h, int prec, int rule, void *theta,
                              const void *g, double c, int sweeps, void *work,
                              void *stream);

/* r = g + c - det(I + H theta) (FP64). */
recon_status recon_step_residual(int N, double h, const double *theta,
                                 const double *g, double c, double *r, void *stream);

/* det(I + H theta) per cell (FP64). */
recon_status recon_step_det(int N, double h, const double *theta, double *det,
                            void *stream);

/* coarse = 8-son mean of fine (Sec. II.A.3), coarse is (Nf/2)^3. */
recon_status recon_step_restrict(int Nf, int prec, const void *fine, void *coarse,
                                 void *stream);

/* fine += scale * P(cnew - cold), P the cell-centred trilinear prolongation
 * (eq. corrections); cnew, cold are Nc^3, fine (2 Nc)^3; cold may be NULL
 * (taken as zero). */
recon_status recon_step_prolong_add(int Nc, int prec, const void *cnew,
                                    const void *cold, double scale, void *fine,
                                    void *stream);

/* Coarsest-grid solve: sweeps of recon_step_sweep until the mean-free rms
 * residual falls below rtol times its start, or (when rtol > 0) a sweep no
 * longer lowers it, or max_sweeps sweeps ran; one thread block,
 * N^3 <= 4096, relaxed in the block's shared memory (work is reserved: the
 * current kernel does not touch it).  sweeps_done: device int (nullable). */
recon_status recon_step_coarse_solve(int N, double h, int prec, int rule, void *theta,
                                     const void *g, double c, int max_sweeps,
                                     double rtol, void *work, int *sweeps_done,
                                     void *stream);

/* The coarsest-grid solve of recon_step_coarse_solve for callers that cannot
 * allocate device memory (a host that reserves all device memory for its own
 * pool, a loop that forbids allocation after start-up, code inside a library
 * that does not own the device).  The paper has no counterpart: this is an
 * interface variant, not a step of the method.
 * Same arguments and result as recon_step_coarse_solve, without `work`: the
 * N^3 scratch lives in a fixed device array of 4096 doubles (32 KiB) compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  N must be even, >= 4, with N^3 <= 4096; larger N returns
 * RECON_E_INVALID and recon_last_error(NULL) says why.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call uses the same array, which keeps
 * the last call's contents; the solve writes every scratch entry before
 * reading it, so nothing has to start at zero.  Calls whose executions
 * overlap on the GPU (different streams, or several host threads) race on
 * the array: serialise them. */
recon_status recon_step_coarse_solve_noalloc(int N, double h, int prec, int rule,
                                             void *theta, const void *g, double c,
                                             int max_sweeps, double rtol, int *sweeps_done,
                                             void *stream);

/* CIC cell of every particle and axis: cells (n x 3 int32) = floor(u) mod N,
 * frac (n x 3 double) = u - floor(u), u = x * (N/L) - 1/2. */
recon_status recon_step_cic_cells(const double *pos, long long n, int N, double L,
                                  int *cells, double *frac, void *stream);

/* `sweeps` red-black Gauss-Seidel sweeps on the linear system J(theta) e = f
 * (FP32 grids), the smoother of the mixed-precision defect correction:
 * e_c += (f - J e)_c / J_cc with J_cc = -2 (adj_xx + adj_yy + adj_zz) / h^2,
 * red then black, each colour reading the values held at the start of its
 * pass.  theta: the FP32 potential whose cofactors define J.  work: 7 N^3
 * floats of scratch (a ping-pong grid and the six cofactor arrays, computed
 * once per call).  N even. */
recon_status recon_step_linear_sweep(int N, double h, float *e, const float *f,
                                     const float *theta, int sweeps, float *work,
                                     void *stream);

/* J v = sum_ab adj(I + H theta)_ab D_ab v, the linearisation of
 * det(I + H theta) in theta (FP64). */
recon_status recon_step_jacobian_apply(int N, double h, const double *theta,
                                       const double *v, double *out, void *stream);

/* Measurement helper, no counterpart in the paper: the FP64 FMA rate of this
 * GPU, against which the FP64 path's smoother is reported.  Launches
 * `blocks` CTAs of 256 threads, each thread running 8 independent chains of
 * `iters` dependent FP64 fused multiply-adds (2 flops each): 4096 * blocks *
 * iters flops in all.  out: device, 1 double (written only in a case that
 * never occurs; it keeps the chains from being optimised away).  Time the
 * launch with events on `stream`.  Errors: RECON_E_INVALID (blocks < 1,
 * iters < 1, out NULL), RECON_E_CUDA. */
recon_status recon_measure_fp64_fma(int blocks, int iters, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RECON_STEPS_H */
