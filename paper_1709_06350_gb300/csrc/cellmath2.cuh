// cellmath2.cuh -- the FP32 cell arithmetic of cellmath.cuh for two cells
// at once, on Blackwell's paired FP32 instructions (f32x2 add / mul / fma:
// one instruction updates both halves of a float2).
//
// Same equations as the scalar forms (eqs. discrete_examples, final_PDE2,
// update; the linear smoother's J e = f with J = sum_ab adj(I+H)_ab D_ab),
// rearranged so that every step is a paired add, multiply or fma:
//
//   Hbar_aa = S_a ih2 - (S_x + S_y + S_z) ih2 / 3        (S_a = face sum)
//   theta_new = theta_c + (h^2/6) f / f'                  (Newton step)
//   e_new = e_c + (J'e / 2 - h^2 f / 2) / (adj_xx + adj_yy + adj_zz)
//     with J'e = J e h^2 (the 1/h^2 of the stencils of e taken out)
//
// The Newton step of the FP32 smoother is kept when it does not increase
// |f|.  For a cubic, f(s + d) = f + f' d + 3 s d^2 + d^3, so with the
// Newton step d = -f / f' the new value is d^2 (3 s + d) and the test
// |f(s + d)| <= |f(s)| is |d| |3 s + d| <= f' -- the same decision,
// evaluated without the cancellation of recomputing f(s + d), which in
// FP32 near convergence is rounding noise and rejected good steps at random.
#pragma once

#include "cellmath.cuh"

namespace recon {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// approximate reciprocal (PTX rcp.approx, ~1 ulp), per half
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }

// the largest root of s^3 + p s + q (eq. root), Newton-polished: the
// fallback of the paired update, kept out of line so that the common path
// stays small in the instruction cache
static __device__ __noinline__ float root_polished_ool(float p, float q) { return root_polished(p, q); }

// Two cells' neighbourhoods as one Nb19<float2>: cell 0 in .x, cell 1 in .y.
__device__ __forceinline__ Nb19<float2> pack19(const Nb19<float> &a, const Nb19<float> &b)
{
    Nb19<float2> v;
    v.c = make_float2(a.c, b.c);
    v.xp = make_float2(a.xp, b.xp);
    v.xm = make_float2(a.xm, b.xm);
    v.yp = make_float2(a.yp, b.yp);
    v.ym = make_float2(a.ym, b.ym);
    v.zp = make_float2(a.zp, b.zp);
    v.zm = make_float2(a.zm, b.zm);
    v.xpyp = make_float2(a.xpyp, b.xpyp);
    v.xmym = make_float2(a.xmym, b.xmym);
    v.xmyp = make_float2(a.xmyp, b.xmyp);
    v.xpym = make_float2(a.xpym, b.xpym);
    v.ypzp = make_float2(a.ypzp, b.ypzp);
    v.ymzm = make_float2(a.ymzm, b.ymzm);
    v.ymzp = make_float2(a.ymzp, b.ymzp);
    v.ypzm = make_float2(a.ypzm, b.ypzm);
    v.xpzp = make_float2(a.xpzp, b.xpzp);
    v.xmzm = make_float2(a.xmzm, b.xmzm);
    v.xmzp = make_float2(a.xmzp, b.xmzp);
    v.xpzm = make_float2(a.xpzm, b.xpzm);
    return v;
}

// (a + b) - (c + d): the unscaled 4-point edge combination of D_ab
__device__ __forceinline__ float2 edge2(float2 a, float2 b, float2 c, float2 d)
{
    return sub2(add2(a, b), add2(c, d));
}

// Eq. update for two cells (FAS smoother).  rhs = b + c per cell.
__device__ __forceinline__ float2 fas_update2(const Nb19<float2> &n, float2 rhs, float ih2, float h2_6,
                                              int rule)
{
    const float2 X = add2(n.xp, n.xm), Y = add2(n.yp, n.ym), Z = add2(n.zp, n.zm);
    const float2 Sg = add2(add2(X, Y), Z);
    const float2 nSt = mul2(Sg, f2(-ih2 * (1.0f / 3.0f)));
    const float2 bxx = fma2(X, f2(ih2), nSt);
    const float2 byy = fma2(Y, f2(ih2), nSt);
    const float2 bzz = fma2(Z, f2(ih2), nSt);
    const float2 q4 = f2(0.25f * ih2);
    const float2 hxy = mul2(edge2(n.xpyp, n.xmym, n.xmyp, n.xpym), q4);
    const float2 hyz = mul2(edge2(n.ypzp, n.ymzm, n.ymzp, n.ypzm), q4);
    const float2 hxz = mul2(edge2(n.xpzp, n.xmzm, n.xmzp, n.xpzm), q4);
    const float2 s = fma2(fma2(n.c, f2(-6.0f), Sg), f2(ih2), f2(3.0f));
    const float2 off = fma2(hxz, hxz, fma2(hyz, hyz, mul2(hxy, hxy)));
    const float2 dia = fma2(bzz, bzz, fma2(byy, byy, mul2(bxx, bxx)));
    const float2 p = mul2(fma2(off, f2(2.0f), dia), f2(-4.5f));
    // det(Hbar), first-row expansion
    const float2 A = fma2(hyz, neg2(hyz), mul2(byy, bzz));
    const float2 B = fma2(hxy, bzz, neg2(mul2(hyz, hxz)));
    const float2 C = fma2(hxy, hyz, neg2(mul2(byy, hxz)));
    const float2 det = fma2(hxz, C, fma2(neg2(hxy), B, mul2(bxx, A)));
    const float2 q = fma2(det, f2(27.0f), mul2(rhs, f2(-27.0f)));
    // Newton step from the right of the cubic's local minimum (f' > 0, s > 0)
    const float2 s2 = mul2(s, s);
    const float2 f = fma2(s, add2(s2, p), q);
    const float2 fp = fma2(s2, f2(3.0f), p);
    const float2 quot = mul2(f, rcp2(fp));                  // -d
    const float2 t = fma2(s, f2(3.0f), neg2(quot));         // 3 s + d
    const float2 u = mul2(quot, t);
    float2 out = fma2(quot, f2(h2_6), n.c);                 // theta_c - (h^2/6) d
    const bool okx = rule == 0 && s.x > 0.0f && fp.x > 0.0f && fabsf(u.x) <= fp.x;
    const bool oky = rule == 0 && s.y > 0.0f && fp.y > 0.0f && fabsf(u.y) <= fp.y;
    if (!okx) out.x = n.c.x - h2_6 * (root_polished_ool(p.x, q.x) - s.x);
    if (!oky) out.y = n.c.y - h2_6 * (root_polished_ool(p.y, q.y) - s.y);
    return out;
}

// Gauss-Seidel on J e = f for two cells (linear smoother); h2 = h^2.
__device__ __forceinline__ float2 lin_update2(const Nb19<float2> &t, const Nb19<float2> &e, float2 rhs,
                                              float ih2, float h2)
{
    // I + H theta
    const float2 axx = fma2(fma2(t.c, f2(-2.0f), add2(t.xp, t.xm)), f2(ih2), f2(1.0f));
    const float2 ayy = fma2(fma2(t.c, f2(-2.0f), add2(t.yp, t.ym)), f2(ih2), f2(1.0f));
    const float2 azz = fma2(fma2(t.c, f2(-2.0f), add2(t.zp, t.zm)), f2(ih2), f2(1.0f));
    const float2 q4 = f2(0.25f * ih2);
    const float2 hxy = mul2(edge2(t.xpyp, t.xmym, t.xmyp, t.xpym), q4);
    const float2 hyz = mul2(edge2(t.ypzp, t.ymzm, t.ymzp, t.ypzm), q4);
    const float2 hxz = mul2(edge2(t.xpzp, t.xmzm, t.xmzp, t.xpzm), q4);
    // adj(I + H theta)
    const float2 cxx = fma2(hyz, neg2(hyz), mul2(ayy, azz));
    const float2 cyy = fma2(hxz, neg2(hxz), mul2(axx, azz));
    const float2 czz = fma2(hxy, neg2(hxy), mul2(axx, ayy));
    const float2 cxy = fma2(hxz, hyz, neg2(mul2(hxy, azz)));
    const float2 cyz = fma2(hxy, hxz, neg2(mul2(axx, hyz)));
    const float2 cxz = fma2(hxy, hyz, neg2(mul2(hxz, ayy)));
    // h^2 D_ab e: diagonal second differences and edge combinations / 4
    const float2 dxx = fma2(e.c, f2(-2.0f), add2(e.xp, e.xm));
    const float2 dyy = fma2(e.c, f2(-2.0f), add2(e.yp, e.ym));
    const float2 dzz = fma2(e.c, f2(-2.0f), add2(e.zp, e.zm));
    const float2 dxy = edge2(e.xpyp, e.xmym, e.xmyp, e.xpym);
    const float2 dyz = edge2(e.ypzp, e.ymzm, e.ymzp, e.ypzm);
    const float2 dxz = edge2(e.xpzp, e.xmzm, e.xmzp, e.xpzm);
    const float2 offd = fma2(cxz, dxz, fma2(cyz, dyz, mul2(cxy, dxy)));
    const float2 diag = fma2(czz, dzz, fma2(cyy, dyy, mul2(cxx, dxx)));
    const float2 Je = fma2(offd, f2(0.5f), diag);            // h^2 J e
    const float2 tr = add2(add2(cxx, cyy), czz);             // -h^2 J_cc / 2
    const float2 num = fma2(Je, f2(0.5f), mul2(rhs, f2(-0.5f * h2)));
    return fma2(num, rcp2(tr), e.c);
}

}  // namespace recon
