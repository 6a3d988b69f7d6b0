// recon_sweep.cu -- register-blocked fused smoother sweep: both colour passes
// of one Gauss-Seidel sweep in a single pass over memory, for grids whose side
// is a multiple of 64 (the fine levels of every benchmark workload).
//
// Semantics are those of two snapshot colour passes (Sec. II.A.2, eq. update;
// colour = (i + j + k) % 2): every red cell reads old values only, every black
// cell reads the new values of its six red faces and the old values of its
// twelve edges and its centre.  The nonlinear variant (FAS) relaxes the cell
// cubic; the linear variant (LIN) relaxes J e = f, J = sum_ab adj(I+H theta)_ab
// D_ab, forming the cofactors from the staged theta at every update.
//
// Work split.  A CTA owns a 16 x 64 (j, k) tile and a chunk of CI planes along
// i (CI a multiple of 4 dividing N).  Compute warp w (0..7) owns tile rows 2w
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
// Warp 8, the halo warp, relaxes the red cells of that ring (rows -1 and 16,
// columns -1 and 64 of the tile), which the black cells on the tile's edge
// read; it is sized to cost about what a compute warp does per step.  One
// barrier per plane.  DRAM traffic: source, right side (and theta) read once,
// destination written once.
#include "cellmath2.cuh"
#include "internal.cuh"

namespace recon {
namespace {

constexpr int kBK = 64;                          // tile columns (k)
constexpr int kBJ = 16;                          // tile rows (j)
constexpr int kCW = kBJ / 2;                     // compute warps
// RECON_REG_HALO_WARP 1: a ninth warp relaxes the ring's red cells; 0: compute
// warps 0 and kCW - 1 take its two jobs (rows, columns) besides their own
#ifndef RECON_REG_HALO_WARP
#define RECON_REG_HALO_WARP 0
#endif
constexpr bool kHaloWarp = RECON_REG_HALO_WARP != 0;
constexpr int kBT = 32 * (kCW + (kHaloWarp ? 1 : 0));   // threads
constexpr int kHOH = (kBK + 4) / 2;              // 34 positions of one k parity per OLD row
constexpr int kHOW = 2 * kHOH;                   // 68 staged positions per OLD row
constexpr int kHOR = kHOW + 1;                   // OLD row stride: odd, so that the halo warp's
                                                 // column cells (rows 2 apart) hit distinct banks
constexpr int kHOJ = kBJ + 4;                    // 20 OLD rows
constexpr int kHOP = kHOJ * kHOR;                // plane stride (positions)
constexpr int kHOS = kHOJ * kHOW;                // 1360 staged positions per OLD plane
constexpr int kHRH = kBK / 2 + 1;                // 33 red cells per RED row
constexpr int kHRJ = kBJ + 2;                    // 18 RED rows
constexpr int kHRP = kHRJ * kHRH;                // 594 per RED plane
constexpr int kGT = kBJ * kBK;                   // right-side values of the tile per plane
constexpr int kGP = kGT + 2 * kBK + 2 * kBJ;     // ... and of the red ring (rows -1, kBJ; columns -1, kBK)
constexpr int kSlots = 6;                        // planes s-1 .. s+2 in use, s+3 and s+4 in flight
constexpr int kStage = (kHOS + kBT - 1) / kBT;   // OLD positions staged per thread per plane
static_assert(kBK / 2 == 32 && kGT / 4 == 32 * kCW && kBK / 4 == 16 && kBJ == 16,
              "lane m owns columns 2m, 2m+1; one 16-byte copy of the tile's right side per compute thread; "
              "the halo warp copies the ring's right side in two instructions");
static_assert((kStage - 1) * kBT <= kHOS, "only the last staging round can run past the plane");

// A slot holds one OLD plane (LIN: the e plane, then the theta plane)
// followed by the same plane's right side.
template <bool LIN>
__host__ __device__ constexpr int slot_bytes() { return 4 * ((LIN ? 2 : 1) * kHOP + kGP); }
template <bool LIN>
__host__ __device__ constexpr int g_off() { return 4 * (LIN ? 2 : 1) * kHOP; }
template <bool LIN>
__host__ __device__ constexpr size_t reg_smem_bytes() { return (size_t)kSlots * slot_bytes<LIN>() + 2u * kHRP * sizeof(float); }
static_assert(slot_bytes<false>() % 16 == 0 && slot_bytes<true>() % 16 == 0 && g_off<false>() % 16 == 0 &&
                  g_off<true>() % 16 == 0,
              "16-byte copies of the right side need 16-byte aligned slots");

__device__ __forceinline__ int wrapn(int x, int N) { return x < 0 ? x + N : (x >= N ? x - N : x); }

__device__ __forceinline__ void cpa4(void *sdst, const void *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cpa16(void *sdst, const void *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// ---- neighbourhoods -------------------------------------------------------
// Block position (A, B): row 2w + A, column 2m + B of the tile (A, B may be
// -1 or 2: outside the thread's block).  tb = (2w + 2) kHOR + m is the
// thread's base in an OLD plane, rb = (2w + 1) kHRH + m in a RED plane.

// Old value at block position (A, B) of the plane in register slot Q, or of
// the shared OLD plane sp when outside the block.
template <int Q, int A, int B, typename V>
__device__ __forceinline__ V old_at(const V (&v)[4][4], const V *sp, int tb)
{
    if constexpr (A >= 0 && A <= 1 && B >= 0 && B <= 1)
        return v[Q][2 * A + B];
    else
        return sp[tb + A * kHOR + (B & 1) * kHOH + ((B + 2) >> 1)];
}

// New red value at block position (A, B) of the plane in register slot Q, or
// of the shared RED plane rp.
template <int Q, int A, int B>
__device__ __forceinline__ float red_at(const float (&r)[4][4], const float *rp, int rb)
{
    if constexpr (A >= 0 && A <= 1 && B >= 0 && B <= 1)
        return r[Q][2 * A + B];
    else
        return rp[rb + A * kHRH + ((B + 1) >> 1)];
}

// Old 19-point neighbourhood of block cell (A, B) of the plane in register
// slot Q0; QM, QP: the slots of the planes below and above; pm, pc, pp: the
// same three planes in the OLD ring.
template <int QM, int Q0, int QP, int A, int B, typename V>
__device__ __forceinline__ Nb19<V> old19(const V (&v)[4][4], const V *pm, const V *pc, const V *pp, int tb)
{
    Nb19<V> n;
    n.c = old_at<Q0, A, B>(v, pc, tb);
    n.xp = old_at<QP, A, B>(v, pp, tb);
    n.xm = old_at<QM, A, B>(v, pm, tb);
    n.yp = old_at<Q0, A + 1, B>(v, pc, tb);
    n.ym = old_at<Q0, A - 1, B>(v, pc, tb);
    n.zp = old_at<Q0, A, B + 1>(v, pc, tb);
    n.zm = old_at<Q0, A, B - 1>(v, pc, tb);
    n.xpyp = old_at<QP, A + 1, B>(v, pp, tb);
    n.xmym = old_at<QM, A - 1, B>(v, pm, tb);
    n.xmyp = old_at<QM, A + 1, B>(v, pm, tb);
    n.xpym = old_at<QP, A - 1, B>(v, pp, tb);
    n.ypzp = old_at<Q0, A + 1, B + 1>(v, pc, tb);
    n.ymzm = old_at<Q0, A - 1, B - 1>(v, pc, tb);
    n.ymzp = old_at<Q0, A - 1, B + 1>(v, pc, tb);
    n.ypzm = old_at<Q0, A + 1, B - 1>(v, pc, tb);
    n.xpzp = old_at<QP, A, B + 1>(v, pp, tb);
    n.xmzm = old_at<QM, A, B - 1>(v, pm, tb);
    n.xmzp = old_at<QM, A, B + 1>(v, pm, tb);
    n.xpzm = old_at<QP, A, B - 1>(v, pp, tb);
    return n;
}

// The six faces of black cell (A, B) from the new red values: x faces are the
// same column one plane down / up (registers), the in-plane faces come from
// the block or the RED plane rp.
template <int QM, int Q0, int QP, int A, int B>
__device__ __forceinline__ void red_faces(Nb19<float> &n, const float (&r)[4][4], const float *rp, int rb)
{
    n.xp = r[QP][2 * A + B];
    n.xm = r[QM][2 * A + B];
    n.yp = red_at<Q0, A + 1, B>(r, rp, rb);
    n.ym = red_at<Q0, A - 1, B>(r, rp, rb);
    n.zp = red_at<Q0, A, B + 1>(r, rp, rb);
    n.zm = red_at<Q0, A, B - 1>(r, rp, rb);
}

// 19-point old neighbourhood of a cell at plane offset S (its own k-parity
// half) with its k-1 neighbour at O (k+1 at O + 1), from three OLD planes:
// the halo warp's gather, whose cells sit outside any thread block.
template <typename V>
__device__ __forceinline__ Nb19<V> gather_at(const V *pm, const V *pc, const V *pp, int S, int O)
{
    Nb19<V> v;
    v.c = pc[S];
    v.xp = pp[S];
    v.xm = pm[S];
    v.yp = pc[S + kHOR];
    v.ym = pc[S - kHOR];
    v.zp = pc[O + 1];
    v.zm = pc[O];
    v.xpyp = pp[S + kHOR];
    v.xmym = pm[S - kHOR];
    v.xmyp = pm[S + kHOR];
    v.xpym = pp[S - kHOR];
    v.ypzp = pc[O + kHOR + 1];
    v.ymzm = pc[O - kHOR];
    v.ymzp = pc[O - kHOR + 1];
    v.ypzm = pc[O + kHOR];
    v.xpzp = pp[O + 1];
    v.xmzm = pm[O];
    v.xmzp = pm[O + 1];
    v.xpzm = pp[O];
    return v;
}

// The nonlinear update of two cells (eq. update), as fas_update2, with the
// rare fallback to the largest root taken behind one warp vote: the common
// path has no divergent branch.  Call with all 32 lanes.
__device__ __forceinline__ float2 fas_update2_voted(const Nb19<float2> &n, float2 rhs, float ih2, float h2_6,
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
    const float2 A = fma2(hyz, neg2(hyz), mul2(byy, bzz));
    const float2 B = fma2(hxy, bzz, neg2(mul2(hyz, hxz)));
    const float2 C = fma2(hxy, hyz, neg2(mul2(byy, hxz)));
    const float2 det = fma2(hxz, C, fma2(neg2(hxy), B, mul2(bxx, A)));
    const float2 q = fma2(det, f2(27.0f), mul2(rhs, f2(-27.0f)));
    const float2 s2 = mul2(s, s);
    const float2 f = fma2(s, add2(s2, p), q);
    const float2 fp = fma2(s2, f2(3.0f), p);
    const float2 quot = mul2(f, rcp2(fp));                  // -d
    const float2 t = fma2(s, f2(3.0f), neg2(quot));         // 3 s + d
    const float2 u = mul2(quot, t);
    float2 out = fma2(quot, f2(h2_6), n.c);
    const bool okx = rule == 0 && s.x > 0.0f && fp.x > 0.0f && fabsf(u.x) <= fp.x;
    const bool oky = rule == 0 && s.y > 0.0f && fp.y > 0.0f && fabsf(u.y) <= fp.y;
    if (!__all_sync(0xffffffffu, okx && oky)) {
        if (!okx) out.x = n.c.x - h2_6 * (root_polished_ool(p.x, q.x) - s.x);
        if (!oky) out.y = n.c.y - h2_6 * (root_polished_ool(p.y, q.y) - s.y);
    }
    return out;
}

// OLD-plane offsets of the tile cell (jl, kl), jl in [-2, kBJ + 1], kl in [-2, kBK + 1]
__device__ __forceinline__ int opos(int jl, int kl) { return (jl + 2) * kHOR + (kl & 1) * kHOH + ((kl + 2) >> 1); }

// ---- the sweep ------------------------------------------------------------
template <bool LIN>
struct RegSweep {
    using V = float;
    const float *src, *th, *g;
    float *dst;
    int N;
    unsigned NN;
    int j0, k0, i0, i1;
    float ih2, h2_6, c;
    int rule, tid, w, lane;
    bool halo;                   // the dedicated halo warp
    bool hrow, hcol;             // this warp relaxes the ring's rows / columns
    int tb, rb;
    unsigned gown;               // in-plane offset of cell (j0 + 2w, k0 + 2m)
    unsigned goff[kStage];       // staging: in-plane global offset ...
    int soff[kStage];            // ... and OLD-plane position (-1: none)
    unsigned char *sm;
    float *red;
    int sl[kSlots];              // byte offsets of the slots of planes s-1 .. s+4
    float v[4][4];               // old values (FAS theta, LIN e) of the block, [plane & 3][2a + b]
    float t[4][4];               // LIN: old theta of the block
    float r[4][4];               // new red values of the block, [plane & 3][2a + b]
    float gb[2][2];              // right side of the black cells of planes s, s+1, [plane & 1][a]

    __device__ __forceinline__ V *oplane(int so) const { return reinterpret_cast<V *>(sm + so); }
    // LIN: the theta plane of a slot
    __device__ __forceinline__ V *tplane(int so) const { return reinterpret_cast<V *>(sm + so) + kHOP; }
    __device__ __forceinline__ const float *gplane(int so) const
    {
        return reinterpret_cast<const float *>(sm + so + g_off<LIN>());
    }

    // copy OLD plane q (needed: i0-2 .. i1+1) and its right side (i0-1 .. i1;
    // the halo warp copies the ring's) into the slot at byte offset so;
    // always commits a group
    __device__ __forceinline__ void issue(int q, int so)
    {
        if (q <= i1 + 1) {
            const unsigned pb = (unsigned)wrapn(q, N) * NN;
            V *op = oplane(so);
#pragma unroll
            for (int x = 0; x < kStage; ++x)
                if (x < kStage - 1 || soff[x] >= 0) {
                    cpa4(op + soff[x], src + pb + goff[x]);
                    if constexpr (LIN) cpa4(op + kHOP + soff[x], th + pb + goff[x]);
                }
            if (q <= i1 && q >= i0 - 1) {
                unsigned char *gs = sm + so + g_off<LIN>();
                if (!halo) {
                    const int row = tid >> 4, col = (tid & 15) * 4;
                    cpa16(gs + 4 * (row * kBK + col), g + pb + (unsigned)(j0 + row) * (unsigned)N + (unsigned)(k0 + col));
                }
                if (hcol) {
                    // rows -1 and kBJ (16 copies of 16 bytes each), then columns -1 and kBK
                    const int hi = lane >> 4, c4 = (lane & 15) * 4;
                    const unsigned jr = (unsigned)wrapn(hi ? j0 + kBJ : j0 - 1, N);
                    cpa16(gs + 4 * (kGT + hi * kBK + c4), g + pb + jr * (unsigned)N + (unsigned)(k0 + c4));
                    const unsigned kc = (unsigned)wrapn(hi ? k0 + kBK : k0 - 1, N);
                    cpa4(gs + 4 * (kGT + 2 * kBK + hi * kBJ + (lane & 15)),
                         g + pb + (unsigned)(j0 + (lane & 15)) * (unsigned)N + kc);
                }
            }
        }
        cpa_commit();
    }

    template <int Q>
    __device__ __forceinline__ void load_own(int so)
    {
        const V *op = oplane(so);
        v[Q][0] = op[tb + 1];
        v[Q][1] = op[tb + kHOH + 1];
        v[Q][2] = op[tb + kHOR + 1];
        v[Q][3] = op[tb + kHOR + kHOH + 1];
        if constexpr (LIN) {
            const V *tp = tplane(so);
            t[Q][0] = tp[tb + 1];
            t[Q][1] = tp[tb + kHOH + 1];
            t[Q][2] = tp[tb + kHOR + 1];
            t[Q][3] = tp[tb + kHOR + kHOH + 1];
        }
    }

    // red cells of plane q (parity P) of the block: (0, P) and (1, 1 - P).
    // Register slots QM, Q0, QP of planes q-1, q, q+1; OLD slots sm_, sc, sp_;
    // right side from the G plane of slot sc.  New values go to r[Q0] and to
    // the RED plane of q; the black cells' right sides are kept for step q.
    // Register arrays are indexed by P (= q % 2: chunks start at a multiple
    // of 4), never by q, so they stay in registers.
    template <int P, int QM, int Q0, int QP>
    __device__ __forceinline__ void red_own(int q, int som, int soc, int sop)
    {
        constexpr int B0 = P, B1 = 1 - P;
        const V *pm = oplane(som), *pc = oplane(soc), *pp = oplane(sop);
        const float *gp = gplane(soc);
        const float2 g0 = *reinterpret_cast<const float2 *>(gp + (2 * w) * kBK + 2 * lane);
        const float2 g1 = *reinterpret_cast<const float2 *>(gp + (2 * w + 1) * kBK + 2 * lane);
        const float2 rhs = make_float2(B0 ? g0.y : g0.x, B1 ? g1.y : g1.x);
        gb[P][0] = B0 ? g0.x : g0.y;
        gb[P][1] = B1 ? g1.x : g1.y;
        const Nb19<V> n0 = old19<QM, Q0, QP, 0, B0>(v, pm, pc, pp, tb);
        const Nb19<V> n1 = old19<QM, Q0, QP, 1, B1>(v, pm, pc, pp, tb);
        float2 out;
        if constexpr (LIN) {
            const Nb19<V> t0 = old19<QM, Q0, QP, 0, B0>(t, pm + kHOP, pc + kHOP, pp + kHOP, tb);
            const Nb19<V> t1 = old19<QM, Q0, QP, 1, B1>(t, pm + kHOP, pc + kHOP, pp + kHOP, tb);
            out = lin_update2(pack19(t0, t1), pack19(n0, n1), rhs, ih2, 6.0f * h2_6);
        } else {
            out = fas_update2_voted(pack19(n0, n1), add2(rhs, f2(c)), ih2, h2_6, rule);
        }
        r[Q0][B0] = out.x;
        r[Q0][2 + B1] = out.y;
        float *rp = red + P * kHRP;
        rp[rb + ((B0 + 1) >> 1)] = out.x;
        rp[rb + kHRH + ((B1 + 1) >> 1)] = out.y;
    }

    // black cells of plane s (parity P) of the block: (0, 1 - P) and (1, P);
    // stores the block's four cells of plane s (red values from r[Q0]).
    template <int P, int QM, int Q0, int QP>
    __device__ __forceinline__ void black_own(int s, int som, int soc, int sop)
    {
        constexpr int B0 = 1 - P, B1 = P;
        const V *pm = oplane(som), *pc = oplane(soc), *pp = oplane(sop);
        const float *rp = red + P * kHRP;
        const Nb19<V> n0 = old19<QM, Q0, QP, 0, B0>(v, pm, pc, pp, tb);
        const Nb19<V> n1 = old19<QM, Q0, QP, 1, B1>(v, pm, pc, pp, tb);
        const float2 rhs = make_float2(gb[P][0], gb[P][1]);
        Nb19<float> a0 = n0, a1 = n1;
        red_faces<QM, Q0, QP, 0, B0>(a0, r, rp, rb);
        red_faces<QM, Q0, QP, 1, B1>(a1, r, rp, rb);
        float2 out;
        if constexpr (LIN) {
            const Nb19<V> t0 = old19<QM, Q0, QP, 0, B0>(t, pm + kHOP, pc + kHOP, pp + kHOP, tb);
            const Nb19<V> t1 = old19<QM, Q0, QP, 1, B1>(t, pm + kHOP, pc + kHOP, pp + kHOP, tb);
            out = lin_update2(pack19(t0, t1), pack19(a0, a1), rhs, ih2, 6.0f * h2_6);
        } else {
            out = fas_update2_voted(pack19(a0, a1), add2(rhs, f2(c)), ih2, h2_6, rule);
        }
        const unsigned base = (unsigned)s * NN + gown;
        const float2 row0 = B0 ? make_float2(r[Q0][0], out.x) : make_float2(out.x, r[Q0][1]);
        const float2 row1 = B1 ? make_float2(r[Q0][2], out.y) : make_float2(out.y, r[Q0][3]);
        *reinterpret_cast<float2 *>(dst + base) = row0;
        *reinterpret_cast<float2 *>(dst + base + (unsigned)N) = row1;
    }

    // halo cells of plane q (parity P): lane m takes the red cell of column
    // pair m in rows -1 and kBJ (one paired update) and, for lanes below
    // kBJ / 2, the red cell of row pair m in columns -1 and kBK (another).
    __device__ __forceinline__ void halo_cells(int P, int hj[4], int hk[4]) const
    {
        const int rr = lane & (kBJ / 2 - 1);
        hj[0] = -1;
        hk[0] = 2 * lane + ((P + 1) & 1);
        hj[1] = kBJ;
        hk[1] = 2 * lane + (P & 1);
        hj[2] = 2 * rr + ((P + 1) & 1);
        hk[2] = -1;
        hj[3] = 2 * rr + (P & 1);
        hk[3] = kBK;
    }

    // the right side of the ring cell (jl, kl) in the G plane gp
    __device__ __forceinline__ static int gring(int jl, int kl)
    {
        return jl < 0 ? kGT + kl : jl >= kBJ ? kGT + kBK + kl : kGT + 2 * kBK + (kl < 0 ? 0 : kBJ) + jl;
    }

    // PAIR 0: the ring's rows, 1: its columns
    template <int P, int PAIR>
    __device__ __forceinline__ void red_halo(int q, int som, int soc, int sop)
    {
        const V *pm = oplane(som), *pc = oplane(soc), *pp = oplane(sop);
        const float *gp = gplane(soc);
        int hj[4], hk[4];
        halo_cells(P, hj, hk);
        float *rp = red + P * kHRP;
        {
            constexpr int pair = PAIR;
            const int a = 2 * pair, b = a + 1;
            const int Sa = opos(hj[a], hk[a]), Oa = opos(hj[a], hk[a] - 1);
            const int Sb = opos(hj[b], hk[b]), Ob = opos(hj[b], hk[b] - 1);
            const Nb19<V> na = gather_at<V>(pm, pc, pp, Sa, Oa);
            const Nb19<V> nb = gather_at<V>(pm, pc, pp, Sb, Ob);
            const float2 rhs = make_float2(gp[gring(hj[a], hk[a])], gp[gring(hj[b], hk[b])]);
            float2 out;
            if constexpr (LIN) {
                const Nb19<V> ta = gather_at<V>(pm + kHOP, pc + kHOP, pp + kHOP, Sa, Oa);
                const Nb19<V> tb_ = gather_at<V>(pm + kHOP, pc + kHOP, pp + kHOP, Sb, Ob);
                out = lin_update2(pack19(ta, tb_), pack19(na, nb), rhs, ih2, 6.0f * h2_6);
            } else {
                out = fas_update2_voted(pack19(na, nb), add2(rhs, f2(c)), ih2, h2_6, rule);
            }
            if (pair == 0 || lane < kBJ / 2) {
                rp[(hj[a] + 1) * kHRH + ((hk[a] + 1) >> 1)] = out.x;
                rp[(hj[b] + 1) * kHRH + ((hk[b] + 1) >> 1)] = out.y;
            }
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
        if (!halo) {
            load_own<QS2>(sl[3]);
            red_own<PR, QS, QS1, QS2>(s + 1, sl[1], sl[2], sl[3]);
            black_own<PB, QSM, QS, QS1>(s, sl[0], sl[1], sl[2]);
        }
        if (hrow) red_halo<PR, 0>(s + 1, sl[1], sl[2], sl[3]);
        if (hcol) red_halo<PR, 1>(s + 1, sl[1], sl[2], sl[3]);
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
        for (int d = 0; d < kSlots; ++d) sl[d] = d * slot_bytes<LIN>();
#pragma unroll
        for (int d = 0; d < kSlots; ++d) issue(i0 - 2 + d, sl[d]);
        cpa_wait<1>();
        __syncthreads();
        // i0 % 4 == 0: plane i0 + d sits in register slot d & 3
        if (!halo) {
            load_own<2>(sl[0]);
            load_own<3>(sl[1]);
            load_own<0>(sl[2]);
            load_own<1>(sl[3]);
            red_own<1, 2, 3, 0>(i0 - 1, sl[0], sl[1], sl[2]);   // own column x faces of black(i0)
            red_own<0, 3, 0, 1>(i0, sl[1], sl[2], sl[3]);
        }
        if (hrow) red_halo<0, 0>(i0, sl[1], sl[2], sl[3]);
        if (hcol) red_halo<0, 1>(i0, sl[1], sl[2], sl[3]);
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

// CTAs per SM: 2 (8 warps each: four warps per scheduler, 128 registers)
#ifndef RECON_REG_CTAS_FAS
#define RECON_REG_CTAS_FAS 2
#endif
#ifndef RECON_REG_CTAS_LIN
#define RECON_REG_CTAS_LIN 2
#endif
template <bool LIN>
__global__ void __launch_bounds__(kBT, LIN ? RECON_REG_CTAS_LIN : RECON_REG_CTAS_FAS)
k_sweep_reg(const float *__restrict__ src, float *__restrict__ dst, const float *__restrict__ g,
            const float *__restrict__ th, const double *__restrict__ cptr, double cval, int N, int CI,
            float ih2, float h2_6, int rule)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
    S.c = LIN ? 0.0f : (float)(cptr ? *cptr : cval);
    S.rule = rule;
    S.tid = threadIdx.x;
    S.w = S.tid >> 5;
    S.lane = S.tid & 31;
    S.halo = kHaloWarp && S.w == kCW;
    S.hrow = kHaloWarp ? S.halo : S.w == 0;
    S.hcol = kHaloWarp ? S.halo : S.w == kCW - 1;
    const int wc = S.halo ? 0 : S.w;
    S.tb = (2 * wc + 2) * kHOR + S.lane;
    S.rb = (2 * wc + 1) * kHRH + S.lane;
    S.gown = (unsigned)(S.j0 + 2 * wc) * (unsigned)N + (unsigned)(S.k0 + 2 * S.lane);
#pragma unroll
    for (int t = 0; t < kStage; ++t) {
        const int e = S.tid + t * kBT;   // staged position: row rr, column k0 - 2 + q
        const int rr = e / kHOW, q = e - rr * kHOW;
        S.soff[t] = e < kHOS ? rr * kHOR + (q & 1) * kHOH + (q >> 1) : -1;
        S.goff[t] = (unsigned)wrapn(S.j0 - 2 + (e < kHOS ? rr : 0), N) * (unsigned)N +
                    (unsigned)wrapn(S.k0 - 2 + q, N);
    }
    S.sm = smem_raw;
    S.red = reinterpret_cast<float *>(smem_raw + (size_t)kSlots * slot_bytes<LIN>());
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
                             cudaStream_t s)
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
                                                                    h2_6, rule);
    else
        k_sweep_reg<false><<<grid, kBT, reg_smem_bytes<false>(), s>>>(src, dst, g, th, cptr, cval, N, CI, ih2,
                                                                      h2_6, rule);
    return cudaGetLastError();
}

}  // namespace recon
