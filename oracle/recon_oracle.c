/*
 * recon_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * multigrid Monge-Ampere reconstruction solve of Shi, Cautun & Li,
 * "New method for initial density reconstruction" (arXiv:1709.06350).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check
 * and the benchmark's CPU-baseline leg may load this code.  It shares no
 * source, header, table or helper with the CUDA implementation, and the
 * product never calls it.
 *
 * Every routine restates one passage of the paper (section / equation named
 * in its comment) as directly as possible: loops over cells in index order,
 * no blocking, no fusion.  Where the paper is silent or garbled the reading
 * taken is stated at the routine.
 *
 * Conventions
 *   grid      N^3 cells, C order [i][j][k] (k fastest), periodic, spacing h;
 *             axis 0 = x = i, axis 1 = y = j, axis 2 = z = k.
 *   theta     the paper's theta = Theta - x^2/2 (Sec. II, eq. theta0).
 *   rhs       the normalised final density 1+delta (eq. basic_eqs), plus the
 *             scalar compatibility constant c (reading: the discrete
 *             determinant is not a null Lagrangian, so the discrete equation
 *             det_h(I + H_h theta) = b + c carries one free scalar c).
 *
 * Build (done by oracle/oracle.py):  gcc -O2 -ffp-contract=off -fPIC -shared
 *   -ffp-contract=off keeps every product and sum rounded separately, so the
 *   result does not depend on whether the host compiler fuses a*b+c.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* grid addressing                                                      */
/* ------------------------------------------------------------------ */

static int wrap(int a, int N) { a %= N; return a < 0 ? a + N : a; }

static long at(int N, int i, int j, int k)
{
    return ((long)wrap(i, N) * N + wrap(j, N)) * N + wrap(k, N);
}

/* ------------------------------------------------------------------ */
/* Sec. II.A.1, eq. discrete_examples: second-order stencils            */
/*   d2/dx2     (t[i+1]+t[i-1]-2t)/h^2                                  */
/*   d2/dxdy    (t[i+1,j+1]+t[i-1,j-1]-t[i-1,j+1]-t[i+1,j-1])/(4h^2)    */
/* H[a][b] is the discrete Hessian of theta at cell (i,j,k).            */
/* ------------------------------------------------------------------ */
void or_hessian(const double *t, int N, double h, int i, int j, int k,
                double H[3][3])
{
    double c = t[at(N, i, j, k)];
    double h2 = h * h;
    double q4 = 4.0 * h2;
    H[0][0] = (t[at(N, i + 1, j, k)] + t[at(N, i - 1, j, k)] - 2.0 * c) / h2;
    H[1][1] = (t[at(N, i, j + 1, k)] + t[at(N, i, j - 1, k)] - 2.0 * c) / h2;
    H[2][2] = (t[at(N, i, j, k + 1)] + t[at(N, i, j, k - 1)] - 2.0 * c) / h2;
    H[0][1] = (t[at(N, i + 1, j + 1, k)] + t[at(N, i - 1, j - 1, k)]
             - t[at(N, i - 1, j + 1, k)] - t[at(N, i + 1, j - 1, k)]) / q4;
    H[1][2] = (t[at(N, i, j + 1, k + 1)] + t[at(N, i, j - 1, k - 1)]
             - t[at(N, i, j - 1, k + 1)] - t[at(N, i, j + 1, k - 1)]) / q4;
    H[0][2] = (t[at(N, i + 1, j, k + 1)] + t[at(N, i - 1, j, k - 1)]
             - t[at(N, i - 1, j, k + 1)] - t[at(N, i + 1, j, k - 1)]) / q4;
    H[1][0] = H[0][1];
    H[2][1] = H[1][2];
    H[2][0] = H[0][2];
}

/* determinant of a 3x3 matrix, expansion along the first row */
static double det3(double A[3][3])
{
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* det(I + H) at one cell: the left side of eq. basic_eqs with
 * Theta = x^2/2 + theta (eq. theta0), i.e. grad grad Theta = I + H. */
double or_det_cell(const double *t, int N, double h, int i, int j, int k)
{
    double H[3][3], A[3][3];
    or_hessian(t, N, h, i, j, k, H);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            A[a][b] = H[a][b] + (a == b ? 1.0 : 0.0);
    return det3(A);
}

/* ------------------------------------------------------------------ */
/* Sec. II, eqs. transformation_derivatives, final_PDE: the cubic       */
/*   s^3 + p s + q = 0,  s = 3 + lap theta,                             */
/*   p = -(9/2) tr(Hbar^2),  q = 9 tr(Hbar^3) - 27 rhs,                  */
/* with Hbar = H - (tr H / 3) I the traceless part.  For a traceless     */
/* symmetric matrix tr(Hbar^3) = 3 det(Hbar), so q = 27 det Hbar - 27rhs.*/
/* ------------------------------------------------------------------ */
void or_cell_cubic(const double *t, int N, double h, int i, int j, int k,
                   double rhs, double *s, double *p, double *q)
{
    double H[3][3], Hb[3][3];
    or_hessian(t, N, h, i, j, k, H);
    double tr = H[0][0] + H[1][1] + H[2][2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            Hb[a][b] = H[a][b] - (a == b ? tr / 3.0 : 0.0);
    double tr2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            tr2 += Hb[a][b] * Hb[b][a];
    *s = 3.0 + tr;
    *p = -4.5 * tr2;
    *q = 27.0 * det3(Hb) - 27.0 * rhs;
}

/* ------------------------------------------------------------------ */
/* Sec. II, eq. root: the physical branch of the cubic.                 */
/* Reading (the printed Delta<0 formula is garbled): the physical root  */
/* is the LARGEST real root.  It is the one continuous with s = 3 at    */
/* delta = 0 and the only one with I + H positive definite.             */
/*   Delta = q^2/4 + p^3/27                                             */
/*   Delta >= 0: one real root, Cardano's formula in the cancellation-  */
/*               free form u = cbrt(-q/2 + sgn(-q/2) sqrt(Delta)),      */
/*               s = u - p/(3u)                                         */
/*   Delta <  0: three real roots 2 sqrt(-p/3) cos((sigma - 2 pi m)/3), */
/*               cos sigma = (3q/2p) sqrt(-3/p), sigma in [0, pi];      */
/*               the largest is m = 0.                                  */
/* ------------------------------------------------------------------ */
double or_largest_root(double p, double q)
{
    double D = q * q / 4.0 + p * p * p / 27.0;
    if (D >= 0.0) {
        double a = -q / 2.0;
        double sg = (a >= 0.0) ? 1.0 : -1.0;
        double u = cbrt(a + sg * sqrt(D));
        if (u == 0.0)
            return 0.0;
        return u - p / (3.0 * u);
    }
    double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
    if (arg > 1.0) arg = 1.0;
    if (arg < -1.0) arg = -1.0;
    double sigma = acos(arg);
    return 2.0 * sqrt(-p / 3.0) * cos(sigma / 3.0);
}

/* ------------------------------------------------------------------ */
/* Sec. II.A.2, eq. update: one Gauss-Seidel point update.              */
/* dL/dtheta_c = -6/h^2, so theta_c <- theta_c - (h^2/6)(s_new - s).     */
/* rule 1 ("exact", the paper's update): s_new = largest root of the     */
/*         cubic (eq. root as read above), then one Newton polish where  */
/*         f' > 0.                                                       */
/* rule 0 ("newton1"): one Newton step on f(s) = s^3 + p s + q from the   */
/*         current s, which is Newton on det(I+H) - rhs in theta_c.      */
/*         Safeguard (reading; a bare Newton step diverges on strongly   */
/*         anisotropic cells, where f' is small): the step is taken only */
/*         from the right of the local minimum of f (s > sqrt(-p/3)) and */
/*         kept only if it does not increase |f|; otherwise rule 1.      */
/* Returns the new theta_c.                                             */
/* ------------------------------------------------------------------ */
static double exact_root_polished(double p, double q)
{
    double sn = or_largest_root(p, q);
    double fp = 3.0 * sn * sn + p;
    if (fp > 0.0)
        sn = sn - (sn * sn * sn + p * sn + q) / fp;
    return sn;
}

double or_point_update(double theta_c, double h, double s, double p, double q,
                       int rule)
{
    double sn;
    double smin = sqrt(p < 0.0 ? -p / 3.0 : 0.0);
    if (rule == 0 && s > smin) {
        double f = s * s * s + p * s + q;
        double fp = 3.0 * s * s + p;
        sn = s - f / fp;
        double fn = sn * sn * sn + p * sn + q;
        if (!(fabs(fn) <= fabs(f)))
            sn = exact_root_polished(p, q);
    } else {
        sn = exact_root_polished(p, q);
    }
    return theta_c - (h * h / 6.0) * (sn - s);
}

/* ------------------------------------------------------------------ */
/* Sec. II.A.2: a full sweep.  Orderings (the paper's text near the      */
/* red-black description):                                               */
/*   0 "rb-snapshot": red ((i+j+k) even) then black; within one colour   */
/*     pass every update reads the values held at the start of the pass */
/*     (same-colour edge neighbours are not yet updated).                */
/*   1 "rb-lex": red then black, each colour in lexicographic order,     */
/*     in place (updated same-colour neighbours are used at once).       */
/*   2 "4-colour": the paper's suggested 4-way split: colour =           */
/*     2*((i+k)&1) + ((j+k)&1); no two cells of one colour are face or   */
/*     edge neighbours, so in-place order within a colour is irrelevant. */
/* rhs per cell = g[cell] + c.                                           */
/* ------------------------------------------------------------------ */
static int colour_of(int ordering, int i, int j, int k)
{
    if (ordering == 2)
        return 2 * ((i + k) & 1) + ((j + k) & 1);
    return (i + j + k) & 1;
}

void or_sweep(double *t, const double *g, double c, int N, double h,
              int ordering, int rule)
{
    long n = (long)N * N * N;
    int ncol = (ordering == 2) ? 4 : 2;
    double *snap = NULL;
    if (ordering == 0)
        snap = (double *)malloc(sizeof(double) * n);
    for (int col = 0; col < ncol; ++col) {
        const double *src = t;
        if (ordering == 0) {
            memcpy(snap, t, sizeof(double) * n);
            src = snap;
        }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j)
                for (int k = 0; k < N; ++k) {
                    if (colour_of(ordering, i, j, k) != col)
                        continue;
                    long id = at(N, i, j, k);
                    double s, p, q;
                    or_cell_cubic(src, N, h, i, j, k, g[id] + c, &s, &p, &q);
                    t[id] = or_point_update(src[id], h, s, p, q, rule);
                }
    }
    free(snap);
}

/* ------------------------------------------------------------------ */
/* Residual of the mass-conservation equation (eq. basic_eqs with the    */
/* compatibility scalar):  r = g + c - det(I + H theta).                 */
/* ------------------------------------------------------------------ */
void or_residual(const double *t, const double *g, double c, int N, double h,
                 double *r)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                r[id] = g[id] + c - or_det_cell(t, N, h, i, j, k);
            }
}

/* The paper's own convergence measure (Sec. II.A.2, residual epsilon):  */
/* eps = rms over cells of L_h = lap_h theta - Sigma, Sigma = root - 3   */
/* (eq. discretisition), with rhs = g + c.  L_h is dimensionless, so its */
/* value is the same in the paper's code units.                          */
/* per-plane partial sums of L_h^2 (out[i] for plane i, N values) */
void or_paper_eps_planes(const double *t, const double *g, double c, int N, double h,
                         double *out)
{
    for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                double s, p, q;
                or_cell_cubic(t, N, h, i, j, k, g[at(N, i, j, k)] + c, &s, &p, &q);
                double L = (s - 3.0) - (or_largest_root(p, q) - 3.0);
                acc += L * L;
            }
        out[i] = acc;
    }
}

double or_paper_eps(const double *t, const double *g, double c, int N, double h)
{
    double *ps = (double *)malloc(sizeof(double) * N);
    or_paper_eps_planes(t, g, c, N, h, ps);
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += ps[i];
    free(ps);
    return sqrt(acc / ((double)N * N * N));
}

/* ------------------------------------------------------------------ */
/* Sec. II.A.3: restriction R = mean of the 8 son cells.                 */
/* coarse cell (I,J,K) has sons (2I+a, 2J+b, 2K+c), a,b,c in {0,1}.      */
/* ------------------------------------------------------------------ */
void or_restrict(const double *f, int Nf, double *cr)
{
    int Nc = Nf / 2;
    for (int I = 0; I < Nc; ++I)
        for (int J = 0; J < Nc; ++J)
            for (int K = 0; K < Nc; ++K) {
                double acc = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int cc = 0; cc < 2; ++cc)
                            acc += f[at(Nf, 2 * I + a, 2 * J + b, 2 * K + cc)];
                cr[at(Nc, I, J, K)] = acc / 8.0;
            }
}

/* ------------------------------------------------------------------ */
/* Sec. II.A.3, eq. corrections: theta_h += scale P(theta_H_new - theta_H_old)*/
/* (scale = 1 in the paper; 1/s for the scaled-defect variant below).    */
/* Reading (P is not specified): cell-centred trilinear interpolation.   */
/* A fine cell centre sits a quarter coarse spacing from its parent's    */
/* centre along each axis, so per axis the parent weighs 3/4 and the     */
/* coarse neighbour on the fine cell's side 1/4.                         */
/* ------------------------------------------------------------------ */
void or_prolong_add(const double *cnew, const double *cold, int Nc, double scale,
                    double *f)
{
    int Nf = 2 * Nc;
    for (int i = 0; i < Nf; ++i)
        for (int j = 0; j < Nf; ++j)
            for (int k = 0; k < Nf; ++k) {
                int I = i / 2, J = j / 2, K = k / 2;
                int di = (i % 2) ? 1 : -1;
                int dj = (j % 2) ? 1 : -1;
                int dk = (k % 2) ? 1 : -1;
                double acc = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int cc = 0; cc < 2; ++cc) {
                            double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75)
                                     * (cc ? 0.25 : 0.75);
                            long id = at(Nc, I + a * di, J + b * dj, K + cc * dk);
                            acc += w * (cnew[id] - cold[id]);
                        }
                f[at(Nf, i, j, k)] += scale * acc;
            }
}

/* ------------------------------------------------------------------ */
/* Sums over a grid.  The paper fixes no summation order; here a sum over */
/* an N^3 grid is the sum, in plane order, of per-plane partial sums      */
/* (each a running sum over the N^2 values of plane i in memory order).  */
/* A grid split into slabs of whole planes (several processes, one slab  */
/* each) then gives the same sums from its slabs' plane partials.        */
/* ------------------------------------------------------------------ */
/* partial sums of the planes of a (nplanes x N x N) array:               */
/*   out[i] = sum over plane i of (a - m)       (sq = 0)                 */
/*   out[i] = sum over plane i of (a - m)^2     (sq = 1)                 */
void or_plane_sums(const double *a, int nplanes, int N, double m, int sq, double *out)
{
    long pl = (long)N * N;
    for (int i = 0; i < nplanes; ++i) {
        double s = 0.0;
        for (long x = 0; x < pl; ++x) {
            double d = a[i * pl + x] - m;
            s += sq ? d * d : d;
        }
        out[i] = s;
    }
}

static double grid_sum(const double *a, int N, double m, int sq)
{
    double *ps = (double *)malloc(sizeof(double) * N);
    or_plane_sums(a, N, N, m, sq, ps);
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += ps[i];
    free(ps);
    return s;
}

static double mean_of(const double *a, int N)
{
    return grid_sum(a, N, 0.0, 0) / ((double)N * N * N);
}

static double norm2_centered(const double *a, int N, double m)
{
    return sqrt(grid_sum(a, N, m, 1));
}

void or_det_grid(const double *t, int N, double h, double *out);

/* ------------------------------------------------------------------ */
/* Scaled-defect safeguard for the coarse equation (reading; the paper   */
/* is silent).  eq. PDE_H asks det_H(theta_H) = det_H(R theta) + R d.    */
/* Far from the solution that right side can turn negative, and a        */
/* negative "density" has no convex solution.  Following the nonlinear  */
/* multigrid method of Hackbusch (scaled defect), the coarse right side */
/* is det_H(R theta) + s R d and the correction is divided by s, with    */
/*   s = min(1, floor * det_H(R theta) / (-R d))  over cells with R d<0, */
/* which keeps every coarse right side >= (1 - floor) det_H(R theta).    */
/* Returns 0 (skip the coarse correction) when s < 1e-3.                 */
/* ------------------------------------------------------------------ */
double or_defect_scale(const double *dH, const double *rr, long nc, double floor_)
{
    if (floor_ <= 0.0)
        return 1.0;
    double s = 1.0;
    for (long x = 0; x < nc; ++x) {
        if (rr[x] < 0.0) {
            double d = dH[x] > 0.0 ? dH[x] : 0.0;
            double cand = floor_ * d / (-rr[x]);
            if (cand < s) s = cand;
        }
    }
    return s < 1e-3 ? 0.0 : s;
}

/* ------------------------------------------------------------------ */
/* Multigrid hierarchy (Sec. II.A.3): halve N while the result is even   */
/* and at least 4; the paper's power-of-two grids end at 4^3.  Reading   */
/* for other N (the paper is silent): stop at the first size whose half  */
/* would be odd or below 4 (96 -> 48 -> 24 -> 12 -> 6).                  */
/* ------------------------------------------------------------------ */
int or_num_levels(int N)
{
    int L = 1;
    while (N % 2 == 0 && N / 2 >= 4 && (N / 2) % 2 == 0) {
        N /= 2;
        ++L;
    }
    return L;
}

typedef struct {
    int nu1, nu2;            /* pre / post sweeps per level            */
    int coarse_max_sweeps;   /* coarsest grid: sweep cap               */
    double coarse_rtol;      /* coarsest grid: stop at this reduction  */
    int ordering, rule;      /* see or_sweep / or_point_update         */
    double scale_floor;      /* scaled-defect safeguard; <= 0: off     */
} or_params;

/* rms of (r - mean r) on one level */
static double proj_rms(const double *r, int N)
{
    double m = mean_of(r, N);
    return norm2_centered(r, N, m) / sqrt((double)N * N * N);
}

/* Coarsest-grid solve (Sec. II.A.3: the hierarchy ends at 4^3; the      */
/* method there is not given).  Reading: Gauss-Seidel sweeps with the    */
/* same point update until the mean-free rms residual falls below        */
/* coarse_rtol times its starting value, or a sweep no longer lowers it  */
/* (round-off floor; only when coarse_rtol > 0), or coarse_max_sweeps.   */
/* Returns the number of sweeps done.                                    */
int or_coarse_solve(double *t, const double *g, double c, int N, double h,
                    const or_params *P)
{
    long n = (long)N * N * N;
    double *r = (double *)malloc(sizeof(double) * n);
    or_residual(t, g, c, N, h, r);
    double r0 = proj_rms(r, N);
    double prev = r0;
    int sw = 0;
    while (sw < P->coarse_max_sweeps) {
        or_sweep(t, g, c, N, h, P->ordering, P->rule);
        ++sw;
        or_residual(t, g, c, N, h, r);
        double cur = proj_rms(r, N);
        if (cur <= P->coarse_rtol * r0)
            break;
        if (P->coarse_rtol > 0.0 && cur >= prev)
            break;              /* no progress: round-off floor reached */
        prev = cur;
    }
    free(r);
    return sw;
}

/* ------------------------------------------------------------------ */
/* FAS V-cycle, Sec. II.A.3 (eqs. PDE_h_w_error, PDE_H, corrections).    */
/* Level l holds theta_l, right side g_l, scalar c_l (c_l = 0 below the  */
/* finest level).  Going down:                                           */
/*   d  = g + c - det_h(theta)          (residual, eq. PDE_h_w_error)    */
/*   thetaH = R theta,  saved copy thetaH_old                            */
/*   gH = det_H(R theta) + R d - mean(R d)   (eq. PDE_H, read with L^H   */
/*        on the first term; the mean of the restricted residual is      */
/*        removed because a periodic problem only constrains mean-free   */
/*        right sides)                                                   */
/* Coming up: theta += P(thetaH - thetaH_old)  (eq. corrections).        */
/* ------------------------------------------------------------------ */
typedef struct {
    int L;
    int *N;
    double *h;
    double **t, **g, **told, **r;
} or_hier;

static void hier_init(or_hier *Hh, int N, double h)
{
    Hh->L = or_num_levels(N);
    Hh->N = (int *)malloc(sizeof(int) * Hh->L);
    Hh->h = (double *)malloc(sizeof(double) * Hh->L);
    Hh->t = (double **)calloc(Hh->L, sizeof(double *));
    Hh->g = (double **)calloc(Hh->L, sizeof(double *));
    Hh->told = (double **)calloc(Hh->L, sizeof(double *));
    Hh->r = (double **)calloc(Hh->L, sizeof(double *));
    for (int l = 0; l < Hh->L; ++l) {
        Hh->N[l] = N >> l;
        Hh->h[l] = h * (double)(1 << l);
        long n = (long)Hh->N[l] * Hh->N[l] * Hh->N[l];
        Hh->r[l] = (double *)calloc(n, sizeof(double));
        if (l > 0) {
            Hh->t[l] = (double *)calloc(n, sizeof(double));
            Hh->g[l] = (double *)calloc(n, sizeof(double));
            Hh->told[l] = (double *)calloc(n, sizeof(double));
        }
    }
}

static void hier_free(or_hier *Hh)
{
    for (int l = 0; l < Hh->L; ++l) {
        free(Hh->r[l]);
        if (l > 0) {
            free(Hh->t[l]);
            free(Hh->g[l]);
            free(Hh->told[l]);
        }
    }
    free(Hh->N); free(Hh->h); free(Hh->t); free(Hh->g); free(Hh->told); free(Hh->r);
}

static void vcycle(or_hier *Hh, int l, double c, const or_params *P)
{
    int N = Hh->N[l];
    double h = Hh->h[l];
    if (l == Hh->L - 1) {
        or_coarse_solve(Hh->t[l], Hh->g[l], c, N, h, P);
        return;
    }
    for (int s = 0; s < P->nu1; ++s)
        or_sweep(Hh->t[l], Hh->g[l], c, N, h, P->ordering, P->rule);

    or_residual(Hh->t[l], Hh->g[l], c, N, h, Hh->r[l]);
    int Nc = Hh->N[l + 1];
    double hc = Hh->h[l + 1];
    long nc = (long)Nc * Nc * Nc;
    or_restrict(Hh->t[l], N, Hh->t[l + 1]);
    memcpy(Hh->told[l + 1], Hh->t[l + 1], sizeof(double) * nc);
    double *rr = (double *)malloc(sizeof(double) * nc);
    double *dH = (double *)malloc(sizeof(double) * nc);
    or_restrict(Hh->r[l], N, rr);
    double m = mean_of(rr, Nc);
    for (long x = 0; x < nc; ++x) rr[x] -= m;
    or_det_grid(Hh->t[l + 1], Nc, hc, dH);
    double sc = or_defect_scale(dH, rr, nc, P->scale_floor);
    if (sc > 0.0) {
        for (long x = 0; x < nc; ++x)
            Hh->g[l + 1][x] = dH[x] + sc * rr[x];
        vcycle(Hh, l + 1, 0.0, P);
        or_prolong_add(Hh->t[l + 1], Hh->told[l + 1], Nc, 1.0 / sc, Hh->t[l]);
    }
    free(rr);
    free(dH);
    for (int s = 0; s < P->nu2; ++s)
        or_sweep(Hh->t[l], Hh->g[l], c, N, h, P->ordering, P->rule);
}

/* ------------------------------------------------------------------ */
/* Solve driver (Sec. II.A.2-3).                                         */
/* Start (reading; the paper starts from theta = 0 on the mesh):          */
/*   fmg = 1: nested iteration.  b is restricted down the hierarchy, the  */
/*            coarsest grid is solved from theta = 0, and on every finer  */
/*            grid the prolonged coarse answer starts one V-cycle (with   */
/*            its compatibility / gauge update); theta_in is ignored.     */
/*   fmg = 0: V-cycles start from the caller's theta (0 in the paper;     */
/*            any earlier answer to resume); c and the gauge are first    */
/*            re-derived from it as after a cycle.                        */
/* After every cycle on a grid (reading; the paper is silent):            */
/*   r = b + c - det(theta);  c <- c - mean(r);  theta <- theta - mean.   */
/* Stop rule: ||r - mean r||_2 / ||b - 1||_2 < tol (denominator 1 when    */
/* b == 1 exactly).  At least one finest-grid cycle is always run.        */
/* stats (nullable, length >= 4 + max_cycles):                            */
/*   [0] cycles, [1] final relative residual, [2] c, [3] paper epsilon,   */
/*   [4 + m] relative residual after cycle m+1.                           */
/* Returns 0 on convergence, 3 when max_cycles ran out, 4 on a non-finite */
/* residual.                                                              */
/* ------------------------------------------------------------------ */
static void compat_and_gauge(or_hier *Hh, int l, double *c)
{
    int N = Hh->N[l];
    long n = (long)N * N * N;
    or_residual(Hh->t[l], Hh->g[l], *c, N, Hh->h[l], Hh->r[l]);
    *c -= mean_of(Hh->r[l], N);
    double mt = mean_of(Hh->t[l], N);
    for (long x = 0; x < n; ++x) Hh->t[l][x] -= mt;
}

int or_solve(const double *b, int N, double L, double *theta, double *c_io,
             double tol, int max_cycles, const or_params *P, int fmg,
             double *stats)
{
    double h = L / (double)N;
    long n = (long)N * N * N;
    or_hier Hh;
    hier_init(&Hh, N, h);
    Hh.t[0] = theta;
    Hh.g[0] = (double *)b;

    double c = c_io ? *c_io : 0.0;
    if (fmg) {
        for (int l = 1; l < Hh.L; ++l)
            or_restrict(Hh.g[l - 1], Hh.N[l - 1], Hh.g[l]);
        int lc = Hh.L - 1;
        long ncst = (long)Hh.N[lc] * Hh.N[lc] * Hh.N[lc];
        memset(Hh.t[lc] ? Hh.t[lc] : theta, 0, sizeof(double) * ncst);
        c = 0.0;
        vcycle(&Hh, lc, c, P);
        compat_and_gauge(&Hh, lc, &c);
        for (int l = lc - 1; l >= 0; --l) {
            long nl = (long)Hh.N[l] * Hh.N[l] * Hh.N[l];
            long nu = (long)Hh.N[l + 1] * Hh.N[l + 1] * Hh.N[l + 1];
            double *zero = (double *)calloc(nu, sizeof(double));
            memset(Hh.t[l], 0, sizeof(double) * nl);
            or_prolong_add(Hh.t[l + 1], zero, Hh.N[l + 1], 1.0, Hh.t[l]);
            free(zero);
            if (l == 0)
                break;              /* the finest grid's cycles follow below */
            vcycle(&Hh, l, c, P);
            compat_and_gauge(&Hh, l, &c);
        }
    } else {
        /* resuming from the caller's theta: c follows from it the same way it
         * is updated after every cycle (c <- c - mean r) */
        compat_and_gauge(&Hh, 0, &c);
    }

    double denom = norm2_centered(b, N, 1.0);
    if (denom == 0.0) denom = 1.0;
    double rel = 0.0;
    int cyc = 0, status = 3;
    for (cyc = 1; cyc <= max_cycles; ++cyc) {
        vcycle(&Hh, 0, c, P);
        or_residual(theta, b, c, N, h, Hh.r[0]);
        double m = mean_of(Hh.r[0], N);
        c -= m;
        double mt = mean_of(theta, N);
        for (long x = 0; x < n; ++x) theta[x] -= mt;
        rel = norm2_centered(Hh.r[0], N, m) / denom;
        if (stats) stats[4 + cyc - 1] = rel;
        if (!isfinite(rel)) { status = 4; break; }
        if (rel < tol) { status = 0; break; }
    }
    if (cyc > max_cycles) cyc = max_cycles;
    if (stats) {
        stats[0] = (double)cyc;
        stats[1] = rel;
        stats[2] = c;
        stats[3] = or_paper_eps(theta, b, c, N, h);
    }
    if (c_io) *c_io = c;
    hier_free(&Hh);
    return status;
}

/* One V-cycle on the finest level only (no c / gauge update): used to   */
/* compare single cycles and to time the CPU baseline on a bounded       */
/* sample.                                                               */
void or_vcycle(const double *b, int N, double L, double *theta, double c,
               const or_params *P)
{
    or_hier Hh;
    hier_init(&Hh, N, L / (double)N);
    Hh.t[0] = theta;
    Hh.g[0] = (double *)b;
    vcycle(&Hh, 0, c, P);
    hier_free(&Hh);
}

/* ------------------------------------------------------------------ */
/* Cloud-in-cell assignment (Sec. I, footnote on NGP/CIC/TSC).           */
/* Along each axis: u = x * (N/L) - 1/2, i0 = floor(u), f = u - i0;      */
/* the particle gives (1-f) to cell i0 and f to cell i0+1 (periodic).    */
/* mass: the amount each particle deposits (N^3 / n for a density       */
/* normalised to mean 1).  Particles are taken in input order.          */
/* ------------------------------------------------------------------ */
void or_cic_cell(double x, int N, double L, int *i0, double *f)
{
    double u = x * ((double)N / L) - 0.5;
    double fl = floor(u);
    *f = u - fl;
    long ii = (long)fl;
    ii %= N;
    if (ii < 0) ii += N;
    *i0 = (int)ii;
}

void or_cic_deposit(const double *pos, long npart, int N, double L,
                    double mass, double *rho)
{
    for (long p = 0; p < npart; ++p) {
        int i0[3];
        double f[3];
        for (int d = 0; d < 3; ++d)
            or_cic_cell(pos[3 * p + d], N, L, &i0[d], &f[d]);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc) {
                    double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1])
                             * (cc ? f[2] : 1.0 - f[2]);
                    rho[at(N, i0[0] + a, i0[1] + b, i0[2] + cc)] += mass * w;
                }
    }
}

/* ------------------------------------------------------------------ */
/* Nearest-grid-point and triangular-shaped-cloud assignment (Sec. I,    */
/* footnote: the method works with any density assignment, NGP, CIC or  */
/* TSC).  Cell i covers [i h, (i+1) h), centre (i + 1/2) h.  Along each  */
/* axis, with u = x (N/L), i = floor(u), d = u - i - 1/2 in [-1/2, 1/2): */
/*   NGP: weight 1 on cell i;                                            */
/*   TSC: the quadratic B-spline of width 3h centred on the particle,    */
/*        sampled at the cell centres:                                   */
/*        W(i-1) = (1/2 - d)^2 / 2,  W(i) = 3/4 - d^2,                   */
/*        W(i+1) = (1/2 + d)^2 / 2.                                      */
/* The 3-D weight is the product over the axes (periodic cells).         */
/* scheme: 0 NGP, 1 CIC (or_cic_deposit above), 2 TSC.                   */
/* ------------------------------------------------------------------ */
static void nearest_cell(double x, int N, double L, int *i, double *d)
{
    double u = x * ((double)N / L);
    double fl = floor(u);
    *d = (u - fl) - 0.5;
    long ii = (long)fl;
    ii %= N;
    if (ii < 0) ii += N;
    *i = (int)ii;
}

void or_assign_deposit(const double *pos, long npart, int N, double L, double mass,
                       int scheme, double *rho)
{
    if (scheme == 1) {
        or_cic_deposit(pos, npart, N, L, mass, rho);
        return;
    }
    for (long p = 0; p < npart; ++p) {
        int i[3];
        double d[3], w[3][3];
        for (int a = 0; a < 3; ++a) {
            nearest_cell(pos[3 * p + a], N, L, &i[a], &d[a]);
            w[a][0] = 0.5 * (0.5 - d[a]) * (0.5 - d[a]);
            w[a][1] = 0.75 - d[a] * d[a];
            w[a][2] = 0.5 * (0.5 + d[a]) * (0.5 + d[a]);
        }
        if (scheme == 0) {
            rho[at(N, i[0], i[1], i[2])] += mass;
            continue;
        }
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
                for (int c = -1; c <= 1; ++c)
                    rho[at(N, i[0] + a, i[1] + b, i[2] + c)] +=
                        mass * (w[0][a + 1] * w[1][b + 1] * w[2][c + 1]);
    }
}

/* CIC with a per-particle value: rho[cell] += value[p] * w.  Used by the */
/* displacement step below.                                              */
static void cic_weighted(const double *pos, long npart, int N, double L,
                         const double *val, double *rho)
{
    for (long p = 0; p < npart; ++p) {
        int i0[3];
        double f[3];
        for (int d = 0; d < 3; ++d)
            or_cic_cell(pos[3 * p + d], N, L, &i0[d], &f[d]);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc) {
                    double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1])
                             * (cc ? f[2] : 1.0 - f[2]);
                    rho[at(N, i0[0] + a, i0[1] + b, i0[2] + cc)] += val[p] * w;
                }
    }
}

/* ------------------------------------------------------------------ */
/* Reconstruction output, Sec. II.B (steps B2, B3; eq.                   */
/* reconstructed_density) and Sec. III.B (x - q = -grad theta).          */
/* Reading (the paper uses iso-q contours and an external Delaunay       */
/* estimator): for every Eulerian cell centre x_c                        */
/*   psi_c = x - q = -(central-difference gradient of theta)             */
/*   q_c   = x_c + grad theta (mod L)                                    */
/*   v_c   = div_q chi = 3 - tr((I + H)^-1)  (chi = q - x)               */
/* and the Lagrangian-grid field is the mass-weighted CIC average        */
/*   delta_r(q) = CIC(q_c, b_c v_c) / max(CIC(q_c, b_c), 1e-12).         */
/* psi layout: [3][N^3] (component-major).                               */
/* ------------------------------------------------------------------ */
void or_displace(const double *t, const double *b, int N, double L,
                 double *psi, double *deltaL)
{
    double h = L / (double)N;
    long n = (long)N * N * N;
    double *qpos = (double *)malloc(sizeof(double) * 3 * n);
    double *wv = (double *)malloc(sizeof(double) * n);
    double *wb = (double *)malloc(sizeof(double) * n);
    double *num = (double *)calloc(n, sizeof(double));
    double *den = (double *)calloc(n, sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                double g[3];
                g[0] = (t[at(N, i + 1, j, k)] - t[at(N, i - 1, j, k)]) / (2.0 * h);
                g[1] = (t[at(N, i, j + 1, k)] - t[at(N, i, j - 1, k)]) / (2.0 * h);
                g[2] = (t[at(N, i, j, k + 1)] - t[at(N, i, j, k - 1)]) / (2.0 * h);
                double x[3] = {(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h};
                for (int d = 0; d < 3; ++d) {
                    psi[d * n + id] = -g[d];
                    double qq = fmod(x[d] + g[d], L);
                    if (qq < 0.0) qq += L;
                    qpos[3 * id + d] = qq;
                }
                double H[3][3], A[3][3];
                or_hessian(t, N, h, i, j, k, H);
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb)
                        A[a][bb] = H[a][bb] + (a == bb ? 1.0 : 0.0);
                double D = det3(A);
                /* diagonal of the inverse = diagonal cofactors / det */
                double inv_tr = ((A[1][1] * A[2][2] - A[1][2] * A[2][1])
                               + (A[0][0] * A[2][2] - A[0][2] * A[2][0])
                               + (A[0][0] * A[1][1] - A[0][1] * A[1][0])) / D;
                double v = 3.0 - inv_tr;
                wv[id] = b[id] * v;
                wb[id] = b[id];
            }
    cic_weighted(qpos, n, N, L, wv, num);
    cic_weighted(qpos, n, N, L, wb, den);
    for (long x = 0; x < n; ++x)
        deltaL[x] = num[x] / (den[x] > 1e-12 ? den[x] : 1e-12);
    free(qpos); free(wv); free(wb); free(num); free(den);
}

/* ------------------------------------------------------------------ */
/* Linearisation of det(I + H theta) (for the adjoint and the defect-    */
/* correction reading).  d det(A) = tr(adj(A) dA), dA = H(v), so         */
/*   J v = sum_ab adj(I+H)_ab (D_ab v)                                   */
/* with D_ab the stencils of eq. discrete_examples.  cof layout:         */
/* [6][N^3] = (xx, yy, zz, xy, yz, xz) entries of adj(I + H theta).      */
/* ------------------------------------------------------------------ */
void or_cofactors(const double *t, int N, double h, double *cof)
{
    long n = (long)N * N * N;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                double H[3][3], A[3][3];
                or_hessian(t, N, h, i, j, k, H);
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb)
                        A[a][bb] = H[a][bb] + (a == bb ? 1.0 : 0.0);
                cof[0 * n + id] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
                cof[1 * n + id] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
                cof[2 * n + id] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
                cof[3 * n + id] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
                cof[4 * n + id] = A[0][1] * A[0][2] - A[0][0] * A[1][2];
                cof[5 * n + id] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
            }
}

void or_jacobian_apply(const double *t, const double *v, int N, double h,
                       double *out)
{
    long n = (long)N * N * N;
    double *cof = (double *)malloc(sizeof(double) * 6 * n);
    or_cofactors(t, N, h, cof);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                double D[3][3];
                or_hessian(v, N, h, i, j, k, D);
                out[id] = cof[0 * n + id] * D[0][0] + cof[1 * n + id] * D[1][1]
                        + cof[2 * n + id] * D[2][2]
                        + 2.0 * (cof[3 * n + id] * D[0][1] + cof[4 * n + id] * D[1][2]
                               + cof[5 * n + id] * D[0][2]);
            }
    free(cof);
}

/* One row of J at cell (i,j,k): the 19 (column, value) pairs of           */
/*   J v = sum_ab adj(I+H)_ab (D_ab v)                                     */
/* written out stencil by stencil (centre, 6 faces, 12 edges; duplicate    */
/* columns are possible only for N < 4 and are summed by the caller).      */
void or_jacobian_row(const double *t, int N, double h, int i, int j, int k,
                     long *cols, double *vals)
{
    double H[3][3], A[3][3];
    or_hessian(t, N, h, i, j, k, H);
    for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 3; ++bb)
            A[a][bb] = H[a][bb] + (a == bb ? 1.0 : 0.0);
    double cxx = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double cyy = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    double czz = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    double cxy = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    double cyz = A[0][1] * A[0][2] - A[0][0] * A[1][2];
    double cxz = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    double h2 = h * h;
    int m = 0;
    /* centre: -2/h^2 from each of the three diagonal second differences */
    cols[m] = at(N, i, j, k); vals[m++] = -2.0 * (cxx + cyy + czz) / h2;
    cols[m] = at(N, i + 1, j, k); vals[m++] = cxx / h2;
    cols[m] = at(N, i - 1, j, k); vals[m++] = cxx / h2;
    cols[m] = at(N, i, j + 1, k); vals[m++] = cyy / h2;
    cols[m] = at(N, i, j - 1, k); vals[m++] = cyy / h2;
    cols[m] = at(N, i, j, k + 1); vals[m++] = czz / h2;
    cols[m] = at(N, i, j, k - 1); vals[m++] = czz / h2;
    /* mixed terms: adj is symmetric, so each off-diagonal pair counts twice */
    double wxy = 2.0 * cxy / (4.0 * h2);
    double wyz = 2.0 * cyz / (4.0 * h2);
    double wxz = 2.0 * cxz / (4.0 * h2);
    cols[m] = at(N, i + 1, j + 1, k); vals[m++] = wxy;
    cols[m] = at(N, i - 1, j - 1, k); vals[m++] = wxy;
    cols[m] = at(N, i - 1, j + 1, k); vals[m++] = -wxy;
    cols[m] = at(N, i + 1, j - 1, k); vals[m++] = -wxy;
    cols[m] = at(N, i, j + 1, k + 1); vals[m++] = wyz;
    cols[m] = at(N, i, j - 1, k - 1); vals[m++] = wyz;
    cols[m] = at(N, i, j - 1, k + 1); vals[m++] = -wyz;
    cols[m] = at(N, i, j + 1, k - 1); vals[m++] = -wyz;
    cols[m] = at(N, i + 1, j, k + 1); vals[m++] = wxz;
    cols[m] = at(N, i - 1, j, k - 1); vals[m++] = wxz;
    cols[m] = at(N, i - 1, j, k + 1); vals[m++] = -wxz;
    cols[m] = at(N, i + 1, j, k - 1); vals[m++] = -wxz;
}

/* Whole-grid helpers used by the Python wrapper (loops over cells only). */
void or_det_grid(const double *t, int N, double h, double *out)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k)
                out[at(N, i, j, k)] = or_det_cell(t, N, h, i, j, k);
}

void or_cubic_grid(const double *t, const double *g, double c, int N, double h,
                   double *s, double *p, double *q)
{
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                or_cell_cubic(t, N, h, i, j, k, g[id] + c, &s[id], &p[id], &q[id]);
            }
}

void or_jacobian_coo(const double *t, int N, double h, long *rows, long *cols,
                     double *vals)
{
    long m = 0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                long id = at(N, i, j, k);
                or_jacobian_row(t, N, h, i, j, k, cols + m, vals + m);
                for (int e = 0; e < 19; ++e) rows[m + e] = id;
                m += 19;
            }
}

void or_cic_cells(const double *pos, long npart, int N, double L, int *cells,
                  double *frac)
{
    for (long p = 0; p < npart; ++p)
        for (int d = 0; d < 3; ++d)
            or_cic_cell(pos[3 * p + d], N, L, &cells[3 * p + d], &frac[3 * p + d]);
}

/* det(I + H theta) at a list of cells (ijk: ncells x 3 ints); used to check
 * a large solution on sampled cells. */
void or_det_cells(const double *t, int N, double h, long ncells, const int *ijk, double *out)
{
    for (long m = 0; m < ncells; ++m)
        out[m] = or_det_cell(t, N, h, ijk[3 * m], ijk[3 * m + 1], ijk[3 * m + 2]);
}
