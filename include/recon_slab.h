/*
 * recon_slab.h -- the FP64 steps of the FAS V-cycle (Sec. II.A.2-3: the
 * point update of eq. update, the residual of eq. basic_eqs with the
 * stencils of eq. discrete_examples, the 8-son restriction and the
 * trilinear prolongation of eq. corrections) on a slab of whole planes of a
 * periodic N^3 grid, for solving one field with several processes, one slab
 * of every multigrid level each.  The process-level logic (which planes a
 * process owns, halo exchange, sums, agglomeration of coarse levels) is the
 * Python module paper_1709_06350_gb300.slab; these calls are its per-process
 * arithmetic on the process's own GPU.
 *
 * Layout (recon_slab): an array holds `planes` planes of N x N doubles in C
 * order; its plane p is the grid's plane (first + p) mod N (first may be
 * negative); the planes a call writes ("own planes") are [lo, hi).  A whole
 * grid is planes = N, first = 0, lo = 0, hi = N, and its stencils wrap
 * periodically along i; a slab (planes <= N, each plane held once) must hold
 * every plane a call reads: `halo` planes on each side of [lo, hi), with halo
 * 2 for recon_slab_sweep, 1 for residual, det and eps, 0 otherwise.  N is
 * even, 4 <= N <= 1024.
 *
 * Every pointer is a DEVICE pointer owned by the caller; every call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 * Errors: RECON_E_INVALID for a bad layout or argument (nothing launched;
 * recon_last_error(NULL) says which call), RECON_E_CUDA when a launch fails.
 */
#ifndef RECON_SLAB_H
#define RECON_SLAB_H

#include "recon.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct recon_slab {
    int N;       /* side of the grid (level) */
    int planes;  /* planes the array holds */
    int first;   /* grid plane of the array's plane 0 (mod N) */
    int lo, hi;  /* own planes [lo, hi) */
} recon_slab;

/* One red-black Gauss-Seidel sweep of eq. update on det(I + H theta) = g + c
 * over the own planes (rule: recon_rule).  Red ((i+j+k) even, i the grid's
 * plane index) then black; each colour pass reads only values from before
 * the pass.  On a slab the red pass is also applied to the first halo plane
 * on each side, so the black pass reads up-to-date red values there: theta
 * and g need two halo planes each side (g only one is read).  Only own
 * planes of theta change.  work: an array of theta's layout (scratch). */
recon_status recon_slab_sweep(const recon_slab *s, double h, int rule, double *theta, const double *g,
                              double c, double *work, void *stream);

/* r = g + c - det(I + H theta) on the own planes (one halo plane). */
recon_status recon_slab_residual(const recon_slab *s, double h, const double *theta, const double *g,
                                 double c, double *r, void *stream);

/* out = det(I + H theta) on the own planes (one halo plane). */
recon_status recon_slab_det(const recon_slab *s, double h, const double *theta, double *out, void *stream);

/* Own planes of the coarse array (level N/2) = mean of the 8 son cells of
 * the fine array (level N; Sec. II.A.3).  The fine array must hold both son
 * planes of every own coarse plane. */
recon_status recon_slab_restrict(const recon_slab *fine_layout, const double *fine,
                                 const recon_slab *coarse_layout, double *coarse, void *stream);

/* Own planes of fine += scale * P(cnew - cold) (eq. corrections; P the
 * cell-centred trilinear interpolation, weights 3/4 and 1/4 per axis); the
 * coarse arrays must hold every coarse plane within one of the own fine
 * planes' parents.  cold may be NULL (zero). */
recon_status recon_slab_prolong_add(const recon_slab *coarse_layout, const double *cnew, const double *cold,
                                    double scale, const recon_slab *fine_layout, double *fine, void *stream);

/* out[p] (hi - lo doubles) = sum over own plane lo + p of (a - m), or of
 * (a - m)^2 when squared = 1; each plane's sum in a fixed order. */
recon_status recon_slab_plane_sums(const recon_slab *s, const double *a, double m, int squared, double *out,
                                   void *stream);

/* out[p] = sum over own plane lo + p of L_h^2, L_h = lap_h theta - Sigma
 * (Sigma = largest root of the cell cubic with rhs g + c, minus 3): the
 * terms of the paper's convergence measure epsilon (Sec. II.A.2). */
recon_status recon_slab_eps_planes(const recon_slab *s, double h, const double *theta, const double *g,
                                   double c, double *out, void *stream);

/* out[p] = min(1, min over cells of own plane lo + p with rr < 0 of
 * floor * max(dH, 0) / (-rr)): per plane, the scaled-defect factor of the
 * coarse equation (the caller takes the minimum over planes and processes,
 * and skips the coarse grid below 1e-3).  floor > 0. */
recon_status recon_slab_defect_min(const recon_slab *s, const double *dH, const double *rr, double floor_,
                                   double *out, void *stream);

/* Own planes: g = dH + scale * rr (the coarse right side of eq. PDE_H). */
recon_status recon_slab_form_rhs(const recon_slab *s, const double *dH, const double *rr, double scale,
                                 double *g, void *stream);

/* Own planes: a -= m. */
recon_status recon_slab_sub(const recon_slab *s, double *a, double m, void *stream);

#ifdef __cplusplus
}
#endif

#endif
