// dfresid.cuh -- the mixed path's fine-grid residual of one cell,
//     r = b + c - det(I + H phi)      (Sec. II, eq. nonlinear_PDE with
//                                      Theta = |x|^2/2 + phi, eq. theta0;
//                                      stencils of eq. discrete_examples)
// with phi = phi_hi + phi_lo and b = b_hi + b_lo double-float pairs, on the
// FP32 pipes.  The absolute error is a few units of 2^-48 times the largest
// of |phi|/h^2 and the determinant's products, the same order as generic
// double-float arithmetic (dfloat.cuh) at about two thirds of its operations:
//
//  * each second difference of phi sums the hi parts by TwoSum (exact) and
//    the lo parts and TwoSum errors in plain float (their rounding is 2^-24 of
//    terms already 2^-24 of phi); a power-of-two 1/h^2 scales the pair
//    exactly; one FastTwoSum leaves each entry of A = I + H phi as a
//    normalised pair, |A_lo| <= ulp(A_hi)/2;
//  * det(A) = det(A_hi) + sum_ij adj(A_hi)_ij A_lo_ij + O(A_lo^2): det(A_hi)
//    is expanded along the first row from cofactors held as exact TwoProd
//    differences, the first-order term from A_lo is evaluated in plain float,
//    and the neglected second-order terms are below 2^-46 of |A|^3.
#pragma once

#include "dfloat.cuh"

namespace recon {

// (s + e) * q for an unnormalised pair (s, e); exact when q is a power of two
template <bool POW2>
__host__ __device__ __forceinline__ df dfr_scale(float s, float e, df q)
{
    if constexpr (POW2)
        return {s * q.hi, e * q.hi};
    else
        return df_mul(df_make(s, e), q);
}

// ((p + m) - 2 c) * q for double-float p, m, c: an unnormalised pair
template <bool POW2>
__host__ __device__ __forceinline__ df dfr_second(float ph, float pl, float mh, float ml, float ch, float cl, df q)
{
    float s1, e1, s2, e2;
    two_sum(ph, mh, s1, e1);
    two_sum(s1, -2.0f * ch, s2, e2);
    return dfr_scale<POW2>(s2, fmaf(-2.0f, cl, (e1 + e2) + (pl + ml)), q);
}

// 1 + d, normalised
__host__ __device__ __forceinline__ df dfr_one_plus(df d)
{
    float s, e;
    two_sum(1.0f, d.hi, s, e);
    df r;
    fast_two_sum(s, e + d.lo, r.hi, r.lo);
    return r;
}

// ((a + b) - (c + d)) * q for double-float a, b, c, d, normalised
template <bool POW2>
__host__ __device__ __forceinline__ df dfr_cross(float ah, float al, float bh, float bl, float ch, float cl,
                                                 float dh, float dl, df q)
{
    float s1, e1, s2, e2, s, e;
    two_sum(ah, bh, s1, e1);
    two_sum(ch, dh, s2, e2);
    two_sum(s1, -s2, s, e);
    const df u = dfr_scale<POW2>(s, (e + (e1 - e2)) + ((al + bl) - (cl + dl)), q);
    df r;
    fast_two_sum(u.hi, u.lo, r.hi, r.lo);
    return r;
}

// x1 y1 - x2 y2 as an unnormalised pair (s, t), exact up to the float sum t
__host__ __device__ __forceinline__ void dfr_cofactor(float x1, float y1, float x2, float y2, float &s, float &t)
{
    float p1, q1, p2, q2, u;
    two_prod(x1, y1, p1, q1);
    two_prod(x2, y2, p2, q2);
    two_sum(p1, -p2, s, u);
    t = u + (q1 - q2);
}

// det of the symmetric matrix [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]] of
// normalised pairs, as an unnormalised pair
__host__ __device__ __forceinline__ df dfr_det3(df xx, df yy, df zz, df xy, df yz, df xz)
{
    const float a = xx.hi, b = yy.hi, c = zz.hi, d = xy.hi, e = yz.hi, f = xz.hi;
    // first-row cofactors: C1 = bc - e^2, C2 = dc - ef, C3 = de - bf
    float C1, t1, C2, t2, C3, t3;
    dfr_cofactor(b, c, e, e, C1, t1);
    dfr_cofactor(d, c, e, f, C2, t2);
    dfr_cofactor(d, e, b, f, C3, t3);
    // det(A_hi) = a C1 - d C2 + f C3
    float P1, Q1, P2, Q2, P3, Q3;
    two_prod(a, C1, P1, Q1);
    two_prod(d, C2, P2, Q2);
    two_prod(f, C3, P3, Q3);
    Q1 = fmaf(a, t1, Q1);
    Q2 = fmaf(d, t2, Q2);
    Q3 = fmaf(f, t3, Q3);
    float S1, T1, S, T;
    two_sum(P1, -P2, S1, T1);
    two_sum(S1, P3, S, T);
    // sum_ij adj(A_hi)_ij A_lo_ij; adj_xx = C1, adj_xy = -C2, adj_xz = C3,
    // and the off-diagonal entries count twice
    const float adj_yy = fmaf(a, c, -f * f), adj_zz = fmaf(a, b, -d * d), adj_yz = fmaf(d, f, -a * e);
    float corr = fmaf(adj_yy, yy.lo, C1 * xx.lo);
    corr = fmaf(adj_zz, zz.lo, corr);
    corr = fmaf(2.0f, fmaf(-C2, xy.lo, fmaf(C3, xz.lo, adj_yz * yz.lo)), corr);
    return df_make(S, ((T + T1) + ((Q1 - Q2) + Q3)) + corr);
}

// r = (b_hi + b_lo) + c - det(I + H phi) rounded to float; ph/pl: the 19-point
// neighbourhoods of phi_hi and phi_lo, ih2 = 1/h^2 (POW2: a power of two, lo 0)
template <bool POW2, typename NB>
__host__ __device__ __forceinline__ float dfr_residual(const NB &H, const NB &L, float bh, float bl, df c, df ih2)
{
    const df q4 = df_scale2(ih2, 0.25f);
    const df axx = dfr_one_plus(dfr_second<POW2>(H.xp, L.xp, H.xm, L.xm, H.c, L.c, ih2));
    const df ayy = dfr_one_plus(dfr_second<POW2>(H.yp, L.yp, H.ym, L.ym, H.c, L.c, ih2));
    const df azz = dfr_one_plus(dfr_second<POW2>(H.zp, L.zp, H.zm, L.zm, H.c, L.c, ih2));
    const df hxy = dfr_cross<POW2>(H.xpyp, L.xpyp, H.xmym, L.xmym, H.xmyp, L.xmyp, H.xpym, L.xpym, q4);
    const df hyz = dfr_cross<POW2>(H.ypzp, L.ypzp, H.ymzm, L.ymzm, H.ymzp, L.ymzp, H.ypzm, L.ypzm, q4);
    const df hxz = dfr_cross<POW2>(H.xpzp, L.xpzp, H.xmzm, L.xmzm, H.xmzp, L.xmzp, H.xpzm, L.xpzm, q4);
    const df det = dfr_det3(axx, ayy, azz, hxy, hyz, hxz);
    float s1, e1, s2, e2;
    two_sum(bh, c.hi, s1, e1);
    two_sum(s1, -det.hi, s2, e2);
    return s2 + (((e1 + e2) + (bl + c.lo)) - det.lo);
}

}  // namespace recon
