// cellmath.cuh -- per-cell arithmetic of the reconstruction equation, for
// T = double or float.  Every kernel that touches the discrete operator goes
// through these functions.
//
//   Hessian stencils          Sec. II.A.1, eq. discrete_examples
//   cubic s^3 + p s + q = 0   Sec. II, eqs. final_PDE / final_PDE2, with the
//                             traceless part Hbar of eq. transformation_derivatives
//   physical root             eq. root, read as the LARGEST real root
//   point update              eq. update, dL/dtheta_c = -6/h^2
#pragma once

#include "common.cuh"

namespace recon {

__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float m_cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double m_acos(double x) { return acos(x); }
__device__ __forceinline__ float m_acos(float x) { return acosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }

// The 19-point neighbourhood of a cell: centre, 6 faces, 12 edges (no corners).
template <typename T>
struct Nb19 {
    T c;
    T xp, xm, yp, ym, zp, zm;
    T xpyp, xmym, xmyp, xpym;  // (i+-1, j+-1, k)
    T ypzp, ymzm, ymzp, ypzm;  // (i, j+-1, k+-1)
    T xpzp, xmzm, xmzp, xpzm;  // (i+-1, j, k+-1)
};

// 32-bit offsets: grids are limited to N <= 1024 (N^3 < 2^32).
template <typename T, typename P>
__device__ __forceinline__ Nb19<T> load19(P a, int N, int i, int j, int k)
{
    const unsigned n = (unsigned)N, nn = n * n;
    const unsigned ri = (unsigned)i * nn, rip = (unsigned)wp(i, N) * nn, rim = (unsigned)wm(i, N) * nn;
    const unsigned cj = (unsigned)j * n, cjp = (unsigned)wp(j, N) * n, cjm = (unsigned)wm(j, N) * n;
    const unsigned kk = (unsigned)k, kp = (unsigned)wp(k, N), km = (unsigned)wm(k, N);
    Nb19<T> v;
    v.c = a[ri + cj + kk];
    v.xp = a[rip + cj + kk];
    v.xm = a[rim + cj + kk];
    v.yp = a[ri + cjp + kk];
    v.ym = a[ri + cjm + kk];
    v.zp = a[ri + cj + kp];
    v.zm = a[ri + cj + km];
    v.xpyp = a[rip + cjp + kk];
    v.xmym = a[rim + cjm + kk];
    v.xmyp = a[rim + cjp + kk];
    v.xpym = a[rip + cjm + kk];
    v.ypzp = a[ri + cjp + kp];
    v.ymzm = a[ri + cjm + km];
    v.ymzp = a[ri + cjm + kp];
    v.ypzm = a[ri + cjp + km];
    v.xpzp = a[rip + cj + kp];
    v.xmzm = a[rim + cj + km];
    v.xmzp = a[rim + cj + kp];
    v.xpzm = a[rip + cj + km];
    return v;
}

// Off-diagonal Hessian entries (4-point edge stencils / (4 h^2)).
template <typename T>
__device__ __forceinline__ void mixed(const Nb19<T> &n, T q4, T &hxy, T &hyz, T &hxz)
{
    hxy = ((n.xpyp + n.xmym) - (n.xmyp + n.xpym)) * q4;
    hyz = ((n.ypzp + n.ymzm) - (n.ymzp + n.ypzm)) * q4;
    hxz = ((n.xpzp + n.xmzm) - (n.xmzp + n.xpzm)) * q4;
}

// Coefficients of the cell cubic s^3 + p s + q = 0 with s = 3 + lap theta:
//   Hbar_aa = (2 S_a - S_b - S_c) / (3 h^2)  (S_a = sum of the two face
//   neighbours along a; the centre cancels, as the paper notes),
//   p = -(9/2) tr(Hbar^2),  q = 27 det(Hbar) - 27 rhs.
template <typename T>
__device__ __forceinline__ void cubic_coeffs(const Nb19<T> &n, T ih2, T rhs, T &s, T &p, T &q)
{
    const T X = n.xp + n.xm, Y = n.yp + n.ym, Z = n.zp + n.zm;
    const T third = ih2 * T(1.0 / 3.0);
    const T bxx = (T(2) * X - Y - Z) * third;
    const T byy = (T(2) * Y - Z - X) * third;
    const T bzz = (T(2) * Z - X - Y) * third;
    T hxy, hyz, hxz;
    mixed(n, ih2 * T(0.25), hxy, hyz, hxz);
    s = T(3) + ((X + Y + Z) - T(6) * n.c) * ih2;
    const T tr2 = bxx * bxx + byy * byy + bzz * bzz + T(2) * (hxy * hxy + hyz * hyz + hxz * hxz);
    const T detb = bxx * (byy * bzz - hyz * hyz) - hxy * (hxy * bzz - hyz * hxz)
                 + hxz * (hxy * hyz - byy * hxz);
    p = T(-4.5) * tr2;
    q = T(27) * detb - T(27) * rhs;
}

// det(I + H) at the cell (first-row expansion).
template <typename T>
__device__ __forceinline__ T det_IH(const Nb19<T> &n, T ih2)
{
    const T axx = T(1) + ((n.xp + n.xm) - T(2) * n.c) * ih2;
    const T ayy = T(1) + ((n.yp + n.ym) - T(2) * n.c) * ih2;
    const T azz = T(1) + ((n.zp + n.zm) - T(2) * n.c) * ih2;
    T hxy, hyz, hxz;
    mixed(n, ih2 * T(0.25), hxy, hyz, hxz);
    return axx * (ayy * azz - hyz * hyz) - hxy * (hxy * azz - hyz * hxz)
         + hxz * (hxy * hyz - ayy * hxz);
}

// adj(I + H): (xx, yy, zz, xy, yz, xz); J v = sum adj_ab D_ab v.
template <typename T>
struct Cof {
    T xx, yy, zz, xy, yz, xz;
};
template <typename T>
__device__ __forceinline__ Cof<T> cofactors(const Nb19<T> &n, T ih2)
{
    const T axx = T(1) + ((n.xp + n.xm) - T(2) * n.c) * ih2;
    const T ayy = T(1) + ((n.yp + n.ym) - T(2) * n.c) * ih2;
    const T azz = T(1) + ((n.zp + n.zm) - T(2) * n.c) * ih2;
    T hxy, hyz, hxz;
    mixed(n, ih2 * T(0.25), hxy, hyz, hxz);
    Cof<T> a;
    a.xx = ayy * azz - hyz * hyz;
    a.yy = axx * azz - hxz * hxz;
    a.zz = axx * ayy - hxy * hxy;
    a.xy = hxz * hyz - hxy * azz;
    a.yz = hxy * hxz - axx * hyz;
    a.xz = hxy * hyz - hxz * ayy;
    return a;
}

// sum_ab adj_ab D_ab v at a cell, from v's 19-point neighbourhood.
template <typename T>
__device__ __forceinline__ T jac_apply(const Cof<T> &a, const Nb19<T> &v, T ih2)
{
    const T dxx = ((v.xp + v.xm) - T(2) * v.c) * ih2;
    const T dyy = ((v.yp + v.ym) - T(2) * v.c) * ih2;
    const T dzz = ((v.zp + v.zm) - T(2) * v.c) * ih2;
    T dxy, dyz, dxz;
    mixed(v, ih2 * T(0.25), dxy, dyz, dxz);
    return a.xx * dxx + a.yy * dyy + a.zz * dzz + T(2) * (a.xy * dxy + a.yz * dyz + a.xz * dxz);
}

// Largest real root of s^3 + p s + q (p <= 0 for a symmetric Hbar).
//   Delta >= 0: u = cbrt(-q/2 + sgn(-q/2) sqrt(Delta)), s = u - p/(3u)
//   Delta <  0: s = 2 sqrt(-p/3) cos(sigma/3), cos sigma = (3q/2p) sqrt(-3/p)
template <typename T>
__device__ __forceinline__ T largest_root(T p, T q)
{
    const T D = q * q * T(0.25) + p * p * p * T(1.0 / 27.0);
    if (D >= T(0)) {
        const T a = -q * T(0.5);
        const T u = m_cbrt(a + (a >= T(0) ? m_sqrt(D) : -m_sqrt(D)));
        return u == T(0) ? T(0) : u - p / (T(3) * u);
    }
    T arg = (T(3) * q / (T(2) * p)) * m_sqrt(T(-3) / p);
    arg = arg > T(1) ? T(1) : (arg < T(-1) ? T(-1) : arg);
    return T(2) * m_sqrt(-p * T(1.0 / 3.0)) * m_cos(m_acos(arg) * T(1.0 / 3.0));
}

template <typename T>
__device__ __forceinline__ T root_polished(T p, T q)
{
    T sn = largest_root(p, q);
    const T fp = T(3) * sn * sn + p;
    if (fp > T(0)) sn = sn - (sn * sn * sn + p * sn + q) / fp;
    return sn;
}

// right of the cubic's local minimum: s > sqrt(-p/3).  FP32 tests the
// equivalent s > 0 and 3 s^2 > -p (no square root); FP64 keeps the
// square root of the definition.
__device__ __forceinline__ bool right_of_min(double s, double p)
{
    return s > m_sqrt(p < 0.0 ? -p * (1.0 / 3.0) : 0.0);
}
__device__ __forceinline__ bool right_of_min(float s, float p) { return s > 0.0f && 3.0f * s * s > -p; }

// the Newton quotient f / f': IEEE in FP64, the fast reciprocal form
// (2 ulp) in the FP32 smoother, whose result the defect correction refines
__device__ __forceinline__ double newton_quot(double f, double fp) { return f / fp; }
__device__ __forceinline__ float newton_quot(float f, float fp) { return __fdividef(f, fp); }

// keep the Newton step s_new = s - quot (quot = f / f') if |f(s_new)| <= |f(s)|.
// FP64 evaluates f(s_new).  FP32 uses the same test in the cancellation-free
// form: f(s + d) = f + f' d + 3 s d^2 + d^3 = d^2 (3 s + d) for d = -quot, so
// the test is |d| |3 s + d| <= f'; recomputing f(s_new) in FP32 near
// convergence gives rounding noise, which rejected good steps at random.
__device__ __forceinline__ bool newton_keep(double s, double p, double q, double f, double, double sn,
                                            double)
{
    const double fn = sn * sn * sn + p * sn + q;
    return fabs(fn) <= fabs(f);
}
__device__ __forceinline__ bool newton_keep(float s, float, float, float, float fp, float, float quot)
{
    return fabsf(quot * (3.0f * s - quot)) <= fp;
}

// Eq. update: theta_c - (h^2/6)(s_new - s).
//   rule 1: s_new = largest root (the paper's update), Newton-polished;
//   rule 0: one Newton step on the cubic from s, taken only right of the
//           local minimum of f and kept only if |f| does not grow; else rule 1.
template <typename T>
__device__ __forceinline__ T point_update(T theta_c, T h2_6, T s, T p, T q, int rule)
{
    T sn;
    bool done = false;
    if (rule == 0 && right_of_min(s, p)) {
        const T f = s * s * s + p * s + q;
        const T fp = T(3) * s * s + p;
        const T quot = newton_quot(f, fp);
        sn = s - quot;
        done = newton_keep(s, p, q, f, fp, sn, quot);
    }
    if (!done) sn = root_polished(p, q);
    return theta_c - h2_6 * (sn - s);
}

}  // namespace recon
