// recon_sweep.cu -- register-blocked fused smoother sweep: both colour passes
// of one Gauss-Seidel sweep in a single pass over memory, for grids whose side
// is a multiple of 64 (the fine levels of every benchmark workload).
//
// Semantics are those of two snapshot colour passes (Sec. II.A.2, eq. update;
// colour = (i + j + k) % 2): every red cell reads old values only, every black
// cell reads the new values of its six red faces and the old values of its
// twelve edges and its centre.  The nonlinear variant (FAS) relaxes the cell
// equation det(I + H theta) = rhs; the linear variant (LIN) relaxes J e = f,
// J = sum_ab adj(I+H theta)_ab D_ab, forming the cofactors from the staged
// theta at every update.
//
// Work split.  A CTA of 8 warps owns a 16 x 64 (j, k) tile and a chunk of CI
// planes along i (CI a multiple of 4 dividing N).  Warp w owns tile rows 2w
// and 2w + 1, and its lane m owns columns 2m and 2m + 1: every thread holds a
// 2 x 2 block of cells per plane, two red and two black, and streams along i.
// At step s it relaxes its red cells of plane s + 1 and its black cells of
// plane s, both pairs at once on the paired FP32 instructions (cellmath2.cuh).
// The block's old values of planes s-1 .. s+2 and its new red values of planes
// s-1 .. s+1 stay in registers, so a black cell's x faces (the same column's
// red cells one plane up and down) and every neighbour inside the block cost
// no load; the remaining neighbours come from shared memory:
//
//   OLD  ring of 6 planes of the source (tile + 2-cell halo), each row stored
//        k-parity split (even k, then odd k) so that the 32 lanes of a warp
//        reading one neighbour of their same-colour cells read 32 consecutive
//        positions; LIN keeps e and theta as two such planes, so that every
//        load lands in the half of a register pair that the paired
//        instructions use.  Planes arrive by cp.async two steps ahead,
//        together with the right side of the tile and of its ring.
//   RED  two planes of new red values on the tile + 1 ring.
//
// The black cells on the tile's edge read the red cells of the ring around
// it (rows -1 and 16, columns -1 and 64), which are relaxed here as well:
// warp 0 takes the two ring rows (one paired update per lane), warp 7 the two
// ring columns.  (A ninth warp dedicated to the ring measured slower: nine-warp
// CTAs leave five warps on some schedulers, which caps registers at 96.)  One
// barrier per plane.  DRAM traffic: source, right side (and theta) read once,
// destination written once.
#include "cellmath2.cuh"
#include "internal.cuh"

namespace recon {
namespace {

constexpr int kBK = 64;                          // tile columns (k)
constexpr int kBJ = 16;                          // tile rows (j)
constexpr int kCW = kBJ / 2;                     // warps
constexpr int kBT = 32 * kCW;                    // threads
constexpr int kHOH = (kBK + 4) / 2;              // 34 positions of one k parity per OLD row
constexpr int kHOW = 2 * kHOH;                   // 68 staged positions per OLD row
constexpr int kHOR = kHOW + 1;                   // OLD row stride: odd, so that the ring columns'
                                                 // cells (rows 2 apart) hit distinct banks
constexpr int kHOJ = kBJ + 4;                    // 20 OLD rows
constexpr int kHOP = kHOJ * kHOR;                // OLD plane stride (floats)
constexpr int kHOS = kHOJ * kHOW;                // 1360 staged positions per OLD plane
constexpr int kHRH = kBK / 2 + 1;                // 33 red cells per RED row
constexpr int kHRJ = kBJ + 2;                    // 18 RED rows
constexpr int kHRP = kHRJ * kHRH;                // 594 per RED plane
constexpr int kGT = kBJ * kBK;                   // right-side values of the tile per plane
constexpr int kGP = kGT + 2 * kBK + 2 * kBJ;     // ... and of the ring (rows -1, kBJ; columns -1, kBK)
constexpr int kSlots = 6;                        // planes s-1 .. s+2 in use, s+3 and s+4 in flight
constexpr int kStage = (kHOS + kBT - 1) / kBT;   // OLD positions staged per thread per plane
constexpr unsigned kNoStage = 0xFFFu;            // packed staging position: none
static_assert(kBK / 2 == 32 && kGT / 4 == kBT && kBK / 4 == 16 && kBJ == 16,
              "lane m owns columns 2m, 2m+1; one 16-byte copy of the tile's right side per thread; "
              "warp 7 copies the ring's right side in two instructions");
static_assert((kStage - 1) * kBT <= kHOS, "only the last staging round can run past the plane");
static_assert(kHOP < (int)kNoStage && kMaxN * kMaxN <= (1 << 20), "staging offsets are packed into 12 + 20 bits");

// A slot holds one OLD plane (LIN: the e plane, then the theta plane)
// followed by the same plane's right side (floats).
template <bool LIN>
__host__ __device__ constexpr int slot_floats() { return (LIN ? 2 : 1) * kHOP + kGP; }
template <bool LIN>
__host__ __device__ constexpr int g_off() { return (LIN ? 2 : 1) * kHOP; }
template <bool LIN>
__host__ __device__ constexpr size_t reg_smem_bytes() { return 4u * ((size_t)kSlots * slot_floats<LIN>() + 2u * kHRP); }
static_assert(slot_floats<false>() % 4 == 0 && slot_floats<true>() % 4 == 0 && g_off<false>() % 4 == 0 &&
                  g_off<true>() % 4 == 0,
              "16-byte copies of the right side need 16-byte aligned slots");

// the sweep's dynamic shared memory, addressed by float index
extern __shared__ __align__(16) float rsm[];

__device__ __forceinline__ int wrapn(int x, int N) { return x < 0 ? x + N : (x >= N ? x - N : x); }

// cp.async to the shared-window address sa
__device__ __forceinline__ void cpa4(unsigned sa, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cpa16(unsigned sa, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// ---- neighbourhoods -------------------------------------------------------
// Block position (A, B): row 2w + A, column 2m + B of the tile (A, B may be
// -1 or 2: outside the thread's block).  pb = (OLD plane) + (2w + 2) kHOR + m
// is the thread's base in an OLD plane, rb = (RED plane) + (2w + 1) kHRH + m
// in a RED plane.

// Old value at block position (A, B) of the plane in register slot Q, or of
// the shared OLD plane whose thread base is pb when outside the block.
template <int Q, int A, int B>
__device__ __forceinline__ float old_at(const float (&v)[4][4], int pb)
{
    if constexpr (A >= 0 && A <= 1 && B >= 0 && B <= 1)
        return v[Q][2 * A + B];
    else
        return rsm[pb + A * kHOR + (B & 1) * kHOH + ((B + 2) >> 1)];
}

// New red value at block position (A, B) of the plane in register slot Q, or
// of the shared RED plane whose thread base is rb.
template <int Q, int A, int B>
__device__ __forceinline__ float red_at(const float (&r)[4][4], int rb)
{
    if constexpr (A >= 0 && A <= 1 && B >= 0 && B <= 1)
        return r[Q][2 * A + B];
    else
        return rsm[rb + A * kHRH + ((B + 1) >> 1)];
}

// Old 19-point neighbourhood of block cell (A, B) of the plane in register
// slot Q0; QM, QP: the slots of the planes below and above; pm, pc, pp: the
// thread bases in the same three planes of the OLD ring.
template <int QM, int Q0, int QP, int A, int B>
__device__ __forceinline__ Nb19<float> old19(const float (&v)[4][4], int pm, int pc, int pp)
{
    Nb19<float> n;
    n.c = old_at<Q0, A, B>(v, pc);
    n.xp = old_at<QP, A, B>(v, pp);
    n.xm = old_at<QM, A, B>(v, pm);
    n.yp = old_at<Q0, A + 1, B>(v, pc);
    n.ym = old_at<Q0, A - 1, B>(v, pc);
    n.zp = old_at<Q0, A, B + 1>(v, pc);
    n.zm = old_at<Q0, A, B - 1>(v, pc);
    n.xpyp = old_at<QP, A + 1, B>(v, pp);
    n.xmym = old_at<QM, A - 1, B>(v, pm);
    n.xmyp = old_at<QM, A + 1, B>(v, pm);
    n.xpym = old_at<QP, A - 1, B>(v, pp);
    n.ypzp = old_at<Q0, A + 1, B + 1>(v, pc);
    n.ymzm = old_at<Q0, A - 1, B - 1>(v, pc);
    n.ymzp = old_at<Q0, A - 1, B + 1>(v, pc);
    n.ypzm = old_at<Q0, A + 1, B - 1>(v, pc);
    n.xpzp = old_at<QP, A, B + 1>(v, pp);
    n.xmzm = old_at<QM, A, B - 1>(v, pm);
    n.xmzp = old_at<QM, A, B + 1>(v, pm);
    n.xpzm = old_at<QP, A, B - 1>(v, pp);
    return n;
}

// The six faces of black cell (A, B) from the new red values: x faces are the
// same column one plane down / up (registers), the in-plane faces come from
// the block or the RED plane (thread base rb).
template <int QM, int Q0, int QP, int A, int B>
__device__ __forceinline__ void red_faces(Nb19<float> &n, const float (&r)[4][4], int rb)
{
    n.xp = r[QP][2 * A + B];
    n.xm = r[QM][2 * A + B];
    n.yp = red_at<Q0, A + 1, B>(r, rb);
    n.ym = red_at<Q0, A - 1, B>(r, rb);
    n.zp = red_at<Q0, A, B + 1>(r, rb);
    n.zm = red_at<Q0, A, B - 1>(r, rb);
}

// 19-point old neighbourhood of a ring cell at plane offset S (its own
// k-parity half) with its k-1 neighbour at O (k+1 at O + 1), from three OLD
// planes at offsets pm, pc, pp.
__device__ __forceinline__ Nb19<float> gather_at(int pm, int pc, int pp, int S, int O)
{
    Nb19<float> v;
    v.c = rsm[pc + S];
    v.xp = rsm[pp + S];
    v.xm = rsm[pm + S];
    v.yp = rsm[pc + S + kHOR];
    v.ym = rsm[pc + S - kHOR];
    v.zp = rsm[pc + O + 1];
    v.zm = rsm[pc + O];
    v.xpyp = rsm[pp + S + kHOR];
    v.xmym = rsm[pm + S - kHOR];
    v.xmyp = rsm[pm + S + kHOR];
    v.xpym = rsm[pp + S - kHOR];
    v.ypzp = rsm[pc + O + kHOR + 1];
    v.ymzm = rsm[pc + O - kHOR];
    v.ymzp = rsm[pc + O - kHOR + 1];
    v.ypzm = rsm[pc + O + kHOR];
    v.xpzp = rsm[pp + O + 1];
    v.xmzm = rsm[pm + O];
    v.xmzp = rsm[pm + O + 1];
    v.xpzm = rsm[pp + O];
    return v;
}

// Eq. update for two cells, written on A = I + H theta directly.  With
// s = tr A and the diagonal cofactors' sum S = tr adj A, the cell cubic is
// f(s) = 27 (det A - rhs) with f'(s) = 9 S, so Newton's step on the cubic
// (eq. update's root by one Newton step) is
//     tau = (det A - rhs) / S,   theta_c += (h^2 / 2) tau
// (every diagonal entry of A moves by -tau).  It is kept from the right of
// the cubic's local minimum (s > 0, S > 0) when |f| does not grow, which for
// the cubic is |tau| |s - tau| <= S (f(s + d) = d^2 (3 s + d) at the Newton
// step d = -3 tau), evaluated without cancellation.  Otherwise the paper's
// update (the largest root, Newton-polished) with p = 9 S - 3 s^2 and
// q = 27 det A - 9 s S + 2 s^3 - 27 rhs; that rare fallback runs behind one
// warp vote, so the common path has no divergent branch.  Call with all lanes.
__device__ __forceinline__ float2 fas_update2_det(const Nb19<float2> &n, float2 rhs, float ih2, float h2_2,
                                                  float h2_6, int rule)
{
    const float2 axx = fma2(fma2(n.c, f2(-2.0f), add2(n.xp, n.xm)), f2(ih2), f2(1.0f));
    const float2 ayy = fma2(fma2(n.c, f2(-2.0f), add2(n.yp, n.ym)), f2(ih2), f2(1.0f));
    const float2 azz = fma2(fma2(n.c, f2(-2.0f), add2(n.zp, n.zm)), f2(ih2), f2(1.0f));
    const float2 q4 = f2(0.25f * ih2);
    const float2 hxy = mul2(edge2(n.xpyp, n.xmym, n.xmyp, n.xpym), q4);
    const float2 hyz = mul2(edge2(n.ypzp, n.ymzm, n.ymzp, n.ypzm), q4);
    const float2 hxz = mul2(edge2(n.xpzp, n.xmzm, n.xmzp, n.xpzm), q4);
    const float2 cxx = fma2(hyz, neg2(hyz), mul2(ayy, azz));
    const float2 cyy = fma2(hxz, neg2(hxz), mul2(axx, azz));
    const float2 czz = fma2(hxy, neg2(hxy), mul2(axx, ayy));
    const float2 cxy = fma2(hxz, hyz, neg2(mul2(hxy, azz)));
    const float2 cxz = fma2(hxy, hyz, neg2(mul2(hxz, ayy)));
    const float2 det = fma2(axx, cxx, fma2(hxy, cxy, mul2(hxz, cxz)));
    const float2 S = add2(add2(cxx, cyy), czz);
    const float2 s = add2(add2(axx, ayy), azz);
    const float2 F = sub2(det, rhs);
    const float2 tau = mul2(F, rcp2(S));
    const float2 u = mul2(tau, sub2(s, tau));
    float2 out = fma2(tau, f2(h2_2), n.c);
    const bool okx = rule == 0 && s.x > 0.0f && S.x > 0.0f && fabsf(u.x) <= S.x;
    const bool oky = rule == 0 && s.y > 0.0f && S.y > 0.0f && fabsf(u.y) <= S.y;
    if (!__all_sync(0xffffffffu, okx && oky)) {
        if (!okx) {
            const float p = 9.0f * S.x - 3.0f * s.x * s.x;
            const float q = 27.0f * (det.x - rhs.x) + s.x * (2.0f * s.x * s.x - 9.0f * S.x);
            out.x = n.c.x - h2_6 * (root_polished_ool(p, q) - s.x);
        }
        if (!oky) {
            const float p = 9.0f * S.y - 3.0f * s.y * s.y;
            const float q = 27.0f * (det.y - rhs.y) + s.y * (2.0f * s.y * s.y - 9.0f * S.y);
            out.y = n.c.y - h2_6 * (root_polished_ool(p, q) - s.y);
        }
    }
    return out;
}

// OLD-plane offset of the tile cell (jl, kl), jl in [-2, kBJ + 1], kl in [-2, kBK + 1]
__device__ __forceinline__ int opos(int jl, int kl) { return (jl + 2) * kHOR + (kl & 1) * kHOH + ((kl + 2) >> 1); }

// ---- the sweep ------------------------------------------------------------
template <bool LIN>
struct RegSweep {
    const float *src, *th, *g;
    float *dst;
    int N;
    unsigned NN;
    int j0, k0, i0, i1;
    float ih2, h2_6, c;
    float gsh;                   // subtracted from the stored values (FAS: a folded gauge shift)
    int rule, w, lane;
    bool hrow, hcol;             // this warp relaxes the ring's rows / columns (warp-uniform)
    int tb, rb;                  // thread bases within an OLD / RED plane
    unsigned gown;               // in-plane offset of cell (j0 + 2w, k0 + 2m)
    unsigned smem;               // shared-window address of rsm
    unsigned stg[kStage];        // staging: in-plane global offset (low 20 bits, N <= 1024) and
                                 // OLD-plane position (high 12 bits; all ones: none)
    int sl[kSlots];              // float offsets of the slots of planes s-1 .. s+4
    float v[4][4];               // old values (FAS theta, LIN e) of the block, [plane & 3][2a + b]
    float t[4][4];               // LIN: old theta of the block
    float r[4][4];               // new red values of the block, [plane & 3][2a + b]
    float gb[2][2];              // right side of the black cells of planes s, s+1, [plane & 1][a]

    // copy OLD plane q (needed: i0-2 .. i1+1) and its right side (i0-1 .. i1,
    // tile and ring) into the slot at float offset so; always commits a group
    __device__ __forceinline__ void issue(int q, int so)
    {
        if (q <= i1 + 1) {
            const unsigned pb = (unsigned)wrapn(q, N) * NN;
            const unsigned sb = smem + 4u * (unsigned)so;
#pragma unroll
            for (int x = 0; x < kStage; ++x)
                if (x < kStage - 1 || (stg[x] >> 20) != kNoStage) {
                    const unsigned so4 = sb + 4u * (stg[x] >> 20), go = pb + (stg[x] & 0xFFFFFu);
                    cpa4(so4, src + go);
                    if constexpr (LIN) cpa4(so4 + 4u * kHOP, th + go);
                }
            if (q <= i1 && q >= i0 - 1) {
                const unsigned gs = sb + 4u * (unsigned)g_off<LIN>();
                const int tid = 32 * w + lane, row = tid >> 4, col = (tid & 15) * 4;
                cpa16(gs + 4u * (unsigned)(row * kBK + col),
                      g + pb + (unsigned)(j0 + row) * (unsigned)N + (unsigned)(k0 + col));
                if (hcol) {
                    // ring rows -1 and kBJ (16 copies of 16 bytes each), then columns -1 and kBK
                    const int hi = lane >> 4, c4 = (lane & 15) * 4;
                    const unsigned jr = (unsigned)wrapn(hi ? j0 + kBJ : j0 - 1, N);
                    cpa16(gs + 4u * (unsigned)(kGT + hi * kBK + c4), g + pb + jr * (unsigned)N + (unsigned)(k0 + c4));
                    const unsigned kc = (unsigned)wrapn(hi ? k0 + kBK : k0 - 1, N);
                    cpa4(gs + 4u * (unsigned)(kGT + 2 * kBK + hi * kBJ + (lane & 15)),
                         g + pb + (unsigned)(j0 + (lane & 15)) * (unsigned)N + kc);
                }
            }
        }
        cpa_commit();
    }

    template <int Q>
    __device__ __forceinline__ void load_own(int so)
    {
        const int b = so + tb;
        v[Q][0] = rsm[b + 1];
        v[Q][1] = rsm[b + kHOH + 1];
        v[Q][2] = rsm[b + kHOR + 1];
        v[Q][3] = rsm[b + kHOR + kHOH + 1];
        if constexpr (LIN) {
            t[Q][0] = rsm[b + kHOP + 1];
            t[Q][1] = rsm[b + kHOP + kHOH + 1];
            t[Q][2] = rsm[b + kHOP + kHOR + 1];
            t[Q][3] = rsm[b + kHOP + kHOR + kHOH + 1];
        }
    }

    // red cells of plane q (parity P = q % 2: chunks start at a multiple of 4,
    // tiles at an even row) of the block: (0, P) and (1, 1 - P).  Register
    // slots QM, Q0, QP of planes q-1, q, q+1; OLD slots som, soc, sop; right
    // side from the slot soc.  New values go to r[Q0] and to the RED plane
    // P; the black cells' right sides are kept for step q.  Register arrays
    // are indexed by compile-time constants only, so they stay in registers.
    template <int P, int QM, int Q0, int QP>
    __device__ __forceinline__ void red_own(int som, int soc, int sop)
    {
        constexpr int B0 = P, B1 = 1 - P;
        const int gp = soc + g_off<LIN>() + 2 * w * kBK + 2 * lane;
        const float2 g0 = *reinterpret_cast<const float2 *>(&rsm[gp]);
        const float2 g1 = *reinterpret_cast<const float2 *>(&rsm[gp + kBK]);
        const float2 rhs = make_float2(B0 ? g0.y : g0.x, B1 ? g1.y : g1.x);
        gb[P][0] = B0 ? g0.x : g0.y;
        gb[P][1] = B1 ? g1.x : g1.y;
        const int pm = som + tb, pc = soc + tb, pp = sop + tb;
        const Nb19<float> n0 = old19<QM, Q0, QP, 0, B0>(v, pm, pc, pp);
        const Nb19<float> n1 = old19<QM, Q0, QP, 1, B1>(v, pm, pc, pp);
        float2 out;
        if constexpr (LIN) {
            const Nb19<float> t0 = old19<QM, Q0, QP, 0, B0>(t, pm + kHOP, pc + kHOP, pp + kHOP);
            const Nb19<float> t1 = old19<QM, Q0, QP, 1, B1>(t, pm + kHOP, pc + kHOP, pp + kHOP);
            out = lin_update2(pack19(t0, t1), pack19(n0, n1), add2(rhs, f2(c)), ih2, 6.0f * h2_6);
        } else {
            out = fas_update2_det(pack19(n0, n1), add2(rhs, f2(c)), ih2, 3.0f * h2_6, h2_6, rule);
        }
        r[Q0][B0] = out.x;
        r[Q0][2 + B1] = out.y;
        const int rp = P * kHRP + rb;
        rsm[rp + ((B0 + 1) >> 1)] = out.x;
        rsm[rp + kHRH + ((B1 + 1) >> 1)] = out.y;
    }

    // black cells of plane s (parity P) of the block: (0, 1 - P) and (1, P);
    // stores the block's four cells of plane s (red values from r[Q0]).
    template <int P, int QM, int Q0, int QP>
    __device__ __forceinline__ void black_own(int s, int som, int soc, int sop)
    {
        constexpr int B0 = 1 - P, B1 = P;
        const int pm = som + tb, pc = soc + tb, pp = sop + tb;
        const int rp = P * kHRP + rb;
        const Nb19<float> n0 = old19<QM, Q0, QP, 0, B0>(v, pm, pc, pp);
        const Nb19<float> n1 = old19<QM, Q0, QP, 1, B1>(v, pm, pc, pp);
        const float2 rhs = make_float2(gb[P][0], gb[P][1]);
        Nb19<float> a0 = n0, a1 = n1;
        red_faces<QM, Q0, QP, 0, B0>(a0, r, rp);
        red_faces<QM, Q0, QP, 1, B1>(a1, r, rp);
        float2 out;
        if constexpr (LIN) {
            const Nb19<float> t0 = old19<QM, Q0, QP, 0, B0>(t, pm + kHOP, pc + kHOP, pp + kHOP);
            const Nb19<float> t1 = old19<QM, Q0, QP, 1, B1>(t, pm + kHOP, pc + kHOP, pp + kHOP);
            out = lin_update2(pack19(t0, t1), pack19(a0, a1), add2(rhs, f2(c)), ih2, 6.0f * h2_6);
        } else {
            out = fas_update2_det(pack19(a0, a1), add2(rhs, f2(c)), ih2, 3.0f * h2_6, h2_6, rule);
        }
        const unsigned base = (unsigned)s * NN + gown;
        float2 row0 = B0 ? make_float2(r[Q0][0], out.x) : make_float2(out.x, r[Q0][1]);
        float2 row1 = B1 ? make_float2(r[Q0][2], out.y) : make_float2(out.y, r[Q0][3]);
        if constexpr (!LIN) {
            row0 = sub2(row0, f2(gsh));
            row1 = sub2(row1, f2(gsh));
        }
        *reinterpret_cast<float2 *>(dst + base) = row0;
        *reinterpret_cast<float2 *>(dst + base + (unsigned)N) = row1;
    }

    // Ring cells of plane q (parity P).  PAIR 0 (warp 0): lane m relaxes the
    // red cell of column pair m in rows -1 and kBJ; PAIR 1 (warp 7): lanes
    // below kBJ / 2 relax the red cell of row pair m in columns -1 and kBK
    // (the other lanes repeat theirs and store nothing).
    template <int P, int PAIR>
    __device__ __forceinline__ void red_ring(int som, int soc, int sop)
    {
        int ja, ka, jb, kb, ga, gbi;
        if constexpr (PAIR == 0) {
            ja = -1;
            ka = 2 * lane + ((P + 1) & 1);
            jb = kBJ;
            kb = 2 * lane + (P & 1);
            ga = kGT + ka;
            gbi = kGT + kBK + kb;
        } else {
            const int rr = lane & (kBJ / 2 - 1);
            ja = 2 * rr + ((P + 1) & 1);
            ka = -1;
            jb = 2 * rr + (P & 1);
            kb = kBK;
            ga = kGT + 2 * kBK + ja;
            gbi = kGT + 2 * kBK + kBJ + jb;
        }
        const int Sa = opos(ja, ka), Oa = opos(ja, ka - 1);
        const int Sb = opos(jb, kb), Ob = opos(jb, kb - 1);
        const Nb19<float> na = gather_at(som, soc, sop, Sa, Oa);
        const Nb19<float> nb = gather_at(som, soc, sop, Sb, Ob);
        const int gs = soc + g_off<LIN>();
        const float2 rhs = make_float2(rsm[gs + ga], rsm[gs + gbi]);
        float2 out;
        if constexpr (LIN) {
            const Nb19<float> ta = gather_at(som + kHOP, soc + kHOP, sop + kHOP, Sa, Oa);
            const Nb19<float> tb_ = gather_at(som + kHOP, soc + kHOP, sop + kHOP, Sb, Ob);
            out = lin_update2(pack19(ta, tb_), pack19(na, nb), add2(rhs, f2(c)), ih2, 6.0f * h2_6);
        } else {
            out = fas_update2_det(pack19(na, nb), add2(rhs, f2(c)), ih2, 3.0f * h2_6, h2_6, rule);
        }
        if (PAIR == 0 || lane < kBJ / 2) {
            const int rbase = kSlots * slot_floats<LIN>() + P * kHRP;
            rsm[rbase + (ja + 1) * kHRH + ((ka + 1) >> 1)] = out.x;
            rsm[rbase + (jb + 1) * kHRH + ((kb + 1) >> 1)] = out.y;
        }
    }

    // one step: red cells of plane s + 1, black cells of plane s.  U = s & 3
    // (the chunk starts at a multiple of 4 and the tile at an even row, so a
    // plane's colour pattern and register slot follow from U).
    template <int U>
    __device__ __forceinline__ void step(int s)
    {
        constexpr int PR = (U + 1) & 1, PB = U & 1;
        constexpr int QSM = (U + 3) & 3, QS = U, QS1 = (U + 1) & 3, QS2 = (U + 2) & 3;
        issue(s + 4, sl[5]);
        load_own<QS2>(sl[3]);
        red_own<PR, QS, QS1, QS2>(sl[1], sl[2], sl[3]);
        if (hrow) red_ring<PR, 0>(sl[1], sl[2], sl[3]);
        if (hcol) red_ring<PR, 1>(sl[1], sl[2], sl[3]);
        black_own<PB, QSM, QS, QS1>(s, sl[0], sl[1], sl[2]);
        cpa_wait<1>();
        __syncthreads();
        const int t0 = sl[0];
#pragma unroll
        for (int x = 0; x < kSlots - 1; ++x) sl[x] = sl[x + 1];
        sl[kSlots - 1] = t0;
    }

    __device__ __forceinline__ void run()
    {
        // prologue: OLD planes i0-2 .. i0+2 (and right sides i0-1 .. i0+2) in
        // slots 0..4, plane i0+3 in flight into slot 5
#pragma unroll
        for (int d = 0; d < kSlots; ++d) sl[d] = d * slot_floats<LIN>();
#pragma unroll
        for (int d = 0; d < kSlots; ++d) issue(i0 - 2 + d, sl[d]);
        cpa_wait<1>();
        __syncthreads();
        // i0 % 4 == 0: plane i0 + d sits in register slot d & 3
        load_own<2>(sl[0]);
        load_own<3>(sl[1]);
        load_own<0>(sl[2]);
        load_own<1>(sl[3]);
        red_own<1, 2, 3, 0>(sl[0], sl[1], sl[2]);   // own column x faces of black(i0)
        red_own<0, 3, 0, 1>(sl[1], sl[2], sl[3]);
        if (hrow) red_ring<0, 0>(sl[1], sl[2], sl[3]);
        if (hcol) red_ring<0, 1>(sl[1], sl[2], sl[3]);
        __syncthreads();
        // planes s-1 .. s+4 for s = i0: slots 1..5, then slot 0 (plane i0-2, free)
        const int t0 = sl[0];
#pragma unroll
        for (int x = 0; x < kSlots - 1; ++x) sl[x] = sl[x + 1];
        sl[kSlots - 1] = t0;
        for (int s = i0; s < i1; s += 4) {
            step<0>(s);
            step<1>(s + 1);
            step<2>(s + 2);
            step<3>(s + 3);
        }
        cpa_wait<0>();
    }
};

// CTAs per SM: FAS 2 (four warps per scheduler, 128 registers); LIN 1 (its
// e and theta neighbourhoods need ~180 registers, and spilling cost more than
// the lower occupancy: 512^3 sweep 1.13 ms at two CTAs, 0.88 ms at one)
#ifndef RECON_REG_CTAS_FAS
#define RECON_REG_CTAS_FAS 2
#endif
#ifndef RECON_REG_CTAS_LIN
#define RECON_REG_CTAS_LIN 1
#endif
template <bool LIN>
__global__ void __launch_bounds__(kBT, LIN ? RECON_REG_CTAS_LIN : RECON_REG_CTAS_FAS)
k_sweep_reg(const float *__restrict__ src, float *__restrict__ dst, const float *__restrict__ g,
            const float *__restrict__ th, const double *__restrict__ cptr, double cval, int N, int CI,
            float ih2, float h2_6, int rule, const double *__restrict__ gshift)
{
    RegSweep<LIN> S;
    S.src = src;
    S.th = th;
    S.g = g;
    S.dst = dst;
    S.N = N;
    S.NN = (unsigned)N * (unsigned)N;
    S.k0 = blockIdx.x * kBK;
    S.j0 = blockIdx.y * kBJ;
    S.i0 = blockIdx.z * CI;
    S.i1 = S.i0 + CI;
    S.ih2 = ih2;
    S.h2_6 = h2_6;
    // FAS: the compatibility scalar c added to the right side; LIN: minus the
    // shift subtracted from f (its mean, folded in: f + (-m) rounds as f - m)
    S.c = LIN ? (gshift ? -(float)*gshift : 0.0f) : (float)(cptr ? *cptr : cval);
    S.gsh = (!LIN && gshift) ? (float)*gshift : 0.0f;
    S.rule = rule;
    const int tid = threadIdx.x;
    // the warp index through a shuffle from lane 0: the compiler sees it as
    // warp-uniform, so the ring-warp branches need no divergence handling
    S.w = __shfl_sync(0xffffffffu, tid >> 5, 0);
    S.lane = tid & 31;
    S.hrow = S.w == 0;
    S.hcol = S.w == kCW - 1;
    S.tb = (2 * S.w + 2) * kHOR + S.lane;
    S.rb = (2 * S.w + 1) * kHRH + S.lane + kSlots * slot_floats<LIN>();
    S.gown = (unsigned)(S.j0 + 2 * S.w) * (unsigned)N + (unsigned)(S.k0 + 2 * S.lane);
    S.smem = (unsigned)__cvta_generic_to_shared(rsm);
#pragma unroll
    for (int t = 0; t < kStage; ++t) {
        const int e = tid + t * kBT;   // staged position: row rr, column k0 - 2 + q
        const int rr = e / kHOW, q = e - rr * kHOW;
        const unsigned so = e < kHOS ? (unsigned)(rr * kHOR + (q & 1) * kHOH + (q >> 1)) : kNoStage;
        const unsigned go = (unsigned)wrapn(S.j0 - 2 + (e < kHOS ? rr : 0), N) * (unsigned)N +
                            (unsigned)wrapn(S.k0 - 2 + q, N);
        S.stg[t] = (so << 20) | go;
    }
    S.run();
}

bool g_reg_ready = false;

}  // namespace

cudaError_t prepare_reg_sweeps()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep_reg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)reg_smem_bytes<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_reg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)reg_smem_bytes<true>());
    if (e == cudaSuccess) g_reg_ready = true;
    return e;
}

// The register-blocked sweep takes grids of side a multiple of 64 (>= 128)
// and arrays aligned to 16 bytes (right side: 16-byte copies; destination:
// 8-byte pair stores).
bool reg_sweep_ok(int N, const float *src, const float *dst, const float *g, const float *th)
{
    auto al = [](const void *p, uintptr_t a) { return p == nullptr || ((uintptr_t)p % a) == 0; };
    return N >= kFusedMinN && N % kBK == 0 && N % kBJ == 0 && al(src, 4) && al(dst, 8) && al(g, 16) &&
           al(th, 4);
}

// planes per CTA: the request rounded down to a multiple of 4 dividing N
int reg_sweep_chunk(int N, int want)
{
    int ci = want > 0 ? want : (N >= 512 ? 64 : (N >= 256 ? 32 : 16));
    ci &= ~3;
    while (ci > 4 && N % ci != 0) ci -= 4;
    return ci < 4 ? 4 : ci;
}

cudaError_t reg_sweep_launch(bool lin, int N, const float *src, float *dst, const float *g, const float *th,
                             const double *cptr, double cval, float ih2, float h2_6, int rule, int chunk,
                             cudaStream_t s, const double *gshift)
{
    if (!g_reg_ready) {
        const cudaError_t e = prepare_reg_sweeps();
        if (e != cudaSuccess) return e;
    }
    const int CI = reg_sweep_chunk(N, chunk);
    const dim3 grid(N / kBK, N / kBJ, N / CI);
    note_launch();
    if (lin)
        k_sweep_reg<true><<<grid, kBT, reg_smem_bytes<true>(), s>>>(src, dst, g, th, cptr, cval, N, CI, ih2,
                                                                    h2_6, rule, gshift);
    else
        k_sweep_reg<false><<<grid, kBT, reg_smem_bytes<false>(), s>>>(src, dst, g, th, cptr, cval, N, CI, ih2,
                                                                      h2_6, rule, gshift);
    return cudaGetLastError();
}

}  // namespace recon
