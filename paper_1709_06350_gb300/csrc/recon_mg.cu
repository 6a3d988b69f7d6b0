// recon_mg.cu -- multigrid kernels and the two solve drivers of librecon.
//
// Method (Shi, Cautun & Li, Sec. II.A): Gauss-Seidel relaxation of the cell
// cubic (eq. update) inside FAS V-cycles (eqs. PDE_h_w_error, PDE_H,
// corrections) down to a coarsest grid of at most 16^3.
//
// Layout: every level is a dense N_l^3 array in C order; the finest level
// uses the caller's phi and b directly.  Red-black passes use a ping-pong
// buffer so that every update of one colour reads the values held at the
// start of the pass (the same-colour edge neighbours enter the cubic's
// coefficients, so an in-place parallel pass would race).
//
// Launch shape of the grid kernels: blocks of 32 x 8 threads, 32 along k
// (coalesced), 8 rows (i, j), grid-stride over the N^2 rows (FOR_ROWS).
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>

#include <type_traits>

#include "cellmath.cuh"
#include "cellmath2.cuh"
#include "dfloat.cuh"
#include "dfresid.cuh"
#include "internal.cuh"

namespace recon {

constexpr int kRowThreads = kRowX * kRowY;

static inline unsigned red_blocks(size_t work, int threads = kThreads)
{
    size_t b = (work + threads - 1) / threads;
    return (unsigned)(b < (size_t)kMaxRedBlocks ? (b == 0 ? 1 : b) : kMaxRedBlocks);
}

// ======================================================================
// smoother: one colour pass; a thread handles the cell pair (2m, 2m+1) of
// its row, of which exactly one has the pass's colour
// ======================================================================
// a -= *m (a gauge shift)
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gauge_by(T *__restrict__ a, size_t n, const double *__restrict__ m)
{
    const T v = (T)(*m);
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n; id += (size_t)gridDim.x * blockDim.x)
        a[id] -= v;
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads)
k_rb_pass(const T *__restrict__ src, T *__restrict__ dst, const T *__restrict__ g,
          const double *__restrict__ cptr, double cval, int N, T ih2, T h2_6, int colour,
          int rule)
{
    const T c = (T)(cptr ? *cptr : cval);
    const int half = N >> 1;
    FOR_ROWS(N, i, j)
    {
        const int par = (colour + i + j) & 1;   // (i + j + k) % 2 == colour
        const unsigned base = offs(N, i, j, 0);
        for (int m = threadIdx.x; m < half; m += kRowX) {
            const int ka = 2 * m + par, kb = 2 * m + 1 - par;
            const Nb19<T> nb = load19<T>(src, N, i, j, ka);
            T s, p, q;
            cubic_coeffs(nb, ih2, g[base + ka] + c, s, p, q);
            dst[base + ka] = point_update(nb.c, h2_6, s, p, q, rule);
            dst[base + kb] = src[base + kb];
        }
    }
}

// ----------------------------------------------------------------------
// Fused sweep: both colour passes in one kernel, src -> dst, with the same
// snapshot semantics as two k_rb_pass launches.  A CTA owns a TJ x TK tile
// of (j, k) and streams a chunk of planes along i through shared memory:
//
//   OLD  ring of 6 planes of src, tile + 2-cell halo.  Each row is stored
//        colour-split: the cells of even k first, then those of odd k, so
//        that a warp reading one neighbour of 32 same-colour cells reads 32
//        consecutive words (no bank conflicts).  The linear variant (LIN)
//        stores an (e, theta) pair per position instead (e at float 2x,
//        theta at 2x + 1): one 64-bit load brings both operands of a
//        neighbour.
//   RED  ring of 4 planes holding only the new red values, tile + 1 halo.
//
// Step s (one barrier): the red cells of plane s+2 (they read only OLD) and
// the black cells of plane s (faces from RED planes s-1..s+1, edges and
// centre from OLD); plane s+4 arrives by cp.async meanwhile.  The red cells
// are computed on the tile + 1 halo, so a CTA needs nothing from another.
// DRAM traffic: src and g read once, dst written once (linear variant:
// theta read once more).  The linear variant (LIN) relaxes J e = f: the
// staged unknown is e, g is f, and the cofactors of I + H theta at each
// updated cell are formed from the staged theta.
//
// Work split: warp w relaxes tile rows w and w+8 (black) and RED rows w,
// w+8 (and w+16 for w < 2) at red index = lane; the last red cell of each
// of the 18 RED rows goes to lanes 0..17 of warp 7.  Rows 8 apart share
// their colour, so one set of shared-memory offsets serves all of a
// thread's rows (the others are immediates), and the ring slots rotate in
// registers.  Requires N >= kFusedMinN (one wrap suffices for every halo
// index).
// ----------------------------------------------------------------------
constexpr int kTJ = 16, kTK = 64;
constexpr int kOJ = kTJ + 4;                 // OLD rows
constexpr int kOH = (kTK + 4) / 2;           // 34 cells of one k parity per OLD row
constexpr int kOR = 2 * kOH;                 // OLD row stride
constexpr int kRJ = kTJ + 2;                 // RED rows
constexpr int kRH = (kTK + 2) / 2;           // 33 red cells per RED row
constexpr int kFT = 256;                     // threads per CTA
constexpr int kWarps = kFT / 32;
constexpr int kOPlane = kOJ * kOR;           // 1360 elements per OLD / TH plane
constexpr int kRPlane = kRJ * kRH;           // 594 elements per RED plane
constexpr int kLoadsPerThread = (kOPlane + kFT - 1) / kFT;   // 6
constexpr int kOSlots = 6, kRSlots = 4;
// The OLD ring holds one value per position (FAS) or an (e, theta) pair per
// position (LIN: e at float 2x, theta at 2x + 1, so one 64-bit load brings
// both operands of a neighbour); the RED ring follows it.
template <bool LIN>
__host__ __device__ constexpr int red_base() { return (LIN ? 2 : 1) * kOSlots * kOPlane; }
static_assert(kTK / 2 == 32 && kRH == 33 && kWarps == 8 && kTJ == 2 * kWarps,
              "warp w owns tile rows w and w + 8 and red index = lane");
static_assert(kRJ - 2 * kWarps == 2, "RED rows 16 and 17 go to warps 0 and 1");

template <typename T, bool LIN>
constexpr size_t fused_smem_bytes()
{
    return sizeof(T) * (size_t)(red_base<LIN>() + kRSlots * kRPlane);
}

__device__ __forceinline__ int wrap1(int x, int N) { return x < 0 ? x + N : (x >= N ? x - N : x); }

// Colour-split position of cell (i, j, k) in a per-cell operand array of the
// linear smoother on the two-pass (unfused) path: within each row (i, j) the
// N/2 cells of colour (i+j+k) % 2 == 0 come first, then the N/2 others, each
// in k order, so the cells one colour pass updates are contiguous.
__host__ __device__ __forceinline__ unsigned cof_slot(int N, int i, int j, int k)
{
    return ((unsigned)i * (unsigned)N + (unsigned)j) * (unsigned)N +
           (((i + j + k) & 1) ? (unsigned)(N >> 1) : 0u) + (unsigned)(k >> 1);
}

__device__ __forceinline__ void cp_async_elem(float *sdst, const float *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_elem(double *sdst, const double *gsrc)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }

// 19-point neighbourhood of a cell from three colour-split planes at
// element offsets pm, pc, pp of the shared buffer sm.  S: the cell's offset
// within a plane (its own parity half); O: the offset of its k-1 neighbour
// (other half), k+1 being O + 1.
template <typename T>
__device__ __forceinline__ Nb19<T> gather19(const T *sm, int pm, int pc, int pp, int S, int O)
{
    Nb19<T> v;
    v.c = sm[pc + S];
    v.xp = sm[pp + S];
    v.xm = sm[pm + S];
    v.yp = sm[pc + S + kOR];
    v.ym = sm[pc + S - kOR];
    v.zp = sm[pc + O + 1];
    v.zm = sm[pc + O];
    v.xpyp = sm[pp + S + kOR];
    v.xmym = sm[pm + S - kOR];
    v.xmyp = sm[pm + S + kOR];
    v.xpym = sm[pp + S - kOR];
    v.ypzp = sm[pc + O + kOR + 1];
    v.ymzm = sm[pc + O - kOR];
    v.ymzp = sm[pc + O - kOR + 1];
    v.ypzm = sm[pc + O + kOR];
    v.xpzp = sm[pp + O + 1];
    v.xmzm = sm[pm + O];
    v.xmzp = sm[pm + O + 1];
    v.xpzm = sm[pp + O];
    return v;
}

// (e, theta) of the 19-point neighbourhood from the linear smoother's
// interleaved OLD ring (position x: e at float 2x, theta at 2x + 1); same
// positions as gather19.
__device__ __forceinline__ void gather19_il(const float *sm, int pm, int pc, int pp, int S, int O,
                                            Nb19<float> &e, Nb19<float> &t)
{
    const float2 *s2 = reinterpret_cast<const float2 *>(sm);
    auto ld = [&](int x, float &ev, float &tv) {
        const float2 v = s2[x];
        ev = v.x;
        tv = v.y;
    };
    ld(pc + S, e.c, t.c);
    ld(pp + S, e.xp, t.xp);
    ld(pm + S, e.xm, t.xm);
    ld(pc + S + kOR, e.yp, t.yp);
    ld(pc + S - kOR, e.ym, t.ym);
    ld(pc + O + 1, e.zp, t.zp);
    ld(pc + O, e.zm, t.zm);
    ld(pp + S + kOR, e.xpyp, t.xpyp);
    ld(pm + S - kOR, e.xmym, t.xmym);
    ld(pm + S + kOR, e.xmyp, t.xmyp);
    ld(pp + S - kOR, e.xpym, t.xpym);
    ld(pc + O + kOR + 1, e.ypzp, t.ypzp);
    ld(pc + O - kOR, e.ymzm, t.ymzm);
    ld(pc + O - kOR + 1, e.ymzp, t.ymzp);
    ld(pc + O + kOR, e.ypzm, t.ypzm);
    ld(pp + O + 1, e.xpzp, t.xpzp);
    ld(pm + O, e.xmzm, t.xmzm);
    ld(pm + O + 1, e.xmzp, t.xmzp);
    ld(pp + O, e.xpzm, t.xpzm);
}

// The nonlinear cell update (eq. update).
template <typename T>
__device__ __forceinline__ T fas_update(const Nb19<T> &nb, T rhs, T ih2, T h2_6, int rule)
{
    T s, p, q;
    cubic_coeffs(nb, ih2, rhs, s, p, q);
    return point_update(nb.c, h2_6, s, p, q, rule);
}

// Gauss-Seidel on J e = f at a cell: J = sum_ab adj(I + H theta)_ab D_ab,
// J_cc = -2 (adj_xx + adj_yy + adj_zz) / h^2.
template <typename T>
__device__ __forceinline__ T lin_update(const Nb19<T> &nt, const Nb19<T> &ne, T rhs, T ih2)
{
    const Cof<T> a = cofactors(nt, ih2);
    const T Je = jac_apply(a, ne, ih2);
    const T diag = T(-2) * (a.xx + a.yy + a.zz) * ih2;
    return ne.c + (rhs - Je) / diag;
}

template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

template <typename T, bool LIN>
// CTAs per SM: FP64 2 (registers), linear 3 (shared memory), FP32 FAS 4
// (64 registers for the paired updates without spills)
__global__ void __launch_bounds__(kFT, sizeof(T) == 8 ? 2 : (LIN ? 3 : 4))
k_sweep_fused(const T *__restrict__ src, T *__restrict__ dst, const T *__restrict__ g,
              const T *__restrict__ th, const double *__restrict__ cptr, double cval, int N,
              int CI, T ih2, T h2_6, int rule)
{
    // FP32: a thread's two rows 8 apart are relaxed together with paired
    // FP32 instructions (cellmath2.cuh); FP64 relaxes them one by one
    constexpr bool kPaired = std::is_same<T, float>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const T c = LIN ? T(0) : (T)(cptr ? *cptr : cval);
    const int k0 = blockIdx.x * kTK, j0 = blockIdx.y * kTJ, i0 = blockIdx.z * CI;
    const int i1 = min(i0 + CI, N);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned NN = (unsigned)N * (unsigned)N;

    // this thread's share of a plane copy: in-plane global offset and
    // colour-split offset within the plane (the same for every plane)
    unsigned goff[kLoadsPerThread];
    int soff[kLoadsPerThread];
#pragma unroll
    for (int t = 0; t < kLoadsPerThread; ++t) {
        const int e = tid + t * kFT;
        const int r = e / kOR, q = e - r * kOR;
        soff[t] = e < kOPlane ? r * kOR + (q & 1) * kOH + (q >> 1) : -1;
        goff[t] = (unsigned)wrap1(j0 - 2 + (r < kOJ ? r : 0), N) * (unsigned)N +
                  (unsigned)wrap1(k0 - 2 + q, N);
    }
    auto issue_plane = [&](int slot, int p) {   // slot: position offset of an OLD plane
        const unsigned pb = (unsigned)wrap1(p, N) * NN;
        if constexpr (LIN) {
#pragma unroll
            for (int t = 0; t < kLoadsPerThread; ++t)
                if (soff[t] >= 0) {
                    T *d = sm + 2 * (slot + soff[t]);
                    cp_async_elem(d, src + pb + goff[t]);
                    cp_async_elem(d + 1, th + pb + goff[t]);
                }
        } else {
#pragma unroll
            for (int t = 0; t < kLoadsPerThread; ++t)
                if (soff[t] >= 0) cp_async_elem(sm + slot + soff[t], src + pb + goff[t]);
        }
        cp_async_commit();
    };

    // global offsets of this thread's red cells within a plane: RED rows
    // w + 8i (row j0 - 1 + w + 8i), red index lane (column k0 - 1 + 2 lane + pr)
    unsigned grow[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) grow[i] = (unsigned)wrap1(j0 - 1 + w + 8 * i, N) * (unsigned)N;
    const unsigned gcol0 = (unsigned)wrap1(k0 - 1 + 2 * lane, N);
    const unsigned gcol1 = (unsigned)wrap1(k0 + 2 * lane, N);
    // the last red cell (index 32) of RED row `lane`, for lanes 0..17 of warp 7
    const bool colw = w == kWarps - 1 && lane < kRJ;
    const unsigned crow = (unsigned)wrap1(j0 - 1 + (colw ? lane : 0), N) * (unsigned)N;
    const unsigned ccol0 = (unsigned)wrap1(k0 + kTK - 1, N), ccol1 = (unsigned)wrap1(k0 + kTK, N);

    // red cells of plane p on the tile + 1 halo into the RED plane at rs;
    // om, oc, op: OLD planes p-1, p, p+1.  A red cell at RED row r, index h
    // sits at RED column 2h + pr: OLD row r+1, parity pr ^ 1, same-parity
    // index h + pr, k-1 neighbour at other-parity index h.
    auto red_plane = [&](int p, int om, int oc, int op, int rs) {
        const unsigned pb = (unsigned)wrap1(p, N) * NN;
        const int pr = (p + j0 + w) & 1;   // rows w + 8i share it
        const int S0 = (w + 1) * kOR + (pr ^ 1) * kOH + lane + pr;
        const int O0 = (w + 1) * kOR + pr * kOH + lane;
        const unsigned gc = pb + (pr ? gcol1 : gcol0);
        if constexpr (kPaired) {
            // RED rows w and w + 8 as one pair of paired-FP32 updates
            constexpr int D = 8 * kOR;
            const float2 rhs = make_float2(g[gc + grow[0]], g[gc + grow[1]]);
            float2 v;
            if constexpr (LIN) {
                Nb19<T> ea, ta, eb, tb;
                gather19_il(sm, om, oc, op, S0, O0, ea, ta);
                gather19_il(sm, om, oc, op, S0 + D, O0 + D, eb, tb);
                v = lin_update2(pack19(ta, tb), pack19(ea, eb), rhs, ih2, T(6) * h2_6);
            } else {
                const Nb19<float2> nb = pack19(gather19<T>(sm, om, oc, op, S0, O0),
                                               gather19<T>(sm, om, oc, op, S0 + D, O0 + D));
                v = fas_update2(nb, add2(rhs, f2(c)), ih2, h2_6, rule);
            }
            sm[rs + w * kRH + lane] = v.x;
            sm[rs + (w + 8) * kRH + lane] = v.y;
        }
#pragma unroll
        for (int i = kPaired ? 2 : 0; i < 3; ++i) {
            if (i == 2 && w >= kRJ - 2 * kWarps) break;
            const int S = S0 + 8 * i * kOR, O = O0 + 8 * i * kOR;
            const T rhs = g[gc + grow[i]];
            T v;
            if constexpr (LIN) {
                Nb19<T> e, t;
                gather19_il(sm, om, oc, op, S, O, e, t);
                v = lin_update<T>(t, e, rhs, ih2);
            } else {
                v = fas_update<T>(gather19<T>(sm, om, oc, op, S, O), rhs + c, ih2, h2_6, rule);
            }
            sm[rs + (w + 8 * i) * kRH + lane] = v;
        }
        if (colw) {
            const int r = lane, prc = (p + j0 + r) & 1, h = kRH - 1;
            const int S = (r + 1) * kOR + (prc ^ 1) * kOH + h + prc;
            const int O = (r + 1) * kOR + prc * kOH + h;
            const T rhs = g[pb + crow + (prc ? ccol1 : ccol0)];
            T v;
            if constexpr (LIN) {
                Nb19<T> e, t;
                gather19_il(sm, om, oc, op, S, O, e, t);
                v = lin_update<T>(t, e, rhs, ih2);
            } else {
                v = fas_update<T>(gather19<T>(sm, om, oc, op, S, O), rhs + c, ih2, h2_6, rule);
            }
            sm[rs + r * kRH + h] = v;
        }
    };
    // black cells of plane s on the tile rows w, w + 8, written with their red
    // partners as (even k, odd k) pairs; pair m = lane.  The black cell is at
    // tile column 2m + pb: OLD row r+2, parity pb, index m+1, k-1 neighbour at
    // other-parity index m + pb; its red faces at RED row r+1, index m + pb
    // (x, y) and m, m+1 (z).  rm, rc, rp: RED planes s-1, s, s+1.
    auto black_plane = [&](int s, int om, int oc, int op, int rm, int rc, int rp) {
        const int pb = (s + j0 + w + 1) & 1;
        const int S0 = (w + 2) * kOR + pb * kOH + lane + 1;
        const int O0 = (w + 2) * kOR + (pb ^ 1) * kOH + lane + pb;
        const int Q0 = (w + 1) * kRH + lane;
        const unsigned sb = (unsigned)s * NN;
        const int gk0 = k0 + 2 * lane;
        if constexpr (kPaired) {
            // tile rows w and w + 8 as one pair of paired-FP32 updates; a
            // row or column outside the grid (ragged tile) is computed from
            // the wrapped halo values but neither read from g nor stored
            constexpr int D = 8 * kOR, DR = 8 * kRH;
            const int gj = j0 + w;
            const bool in0 = gk0 < N && gj < N, in1 = gk0 < N && gj + 8 < N;
            Nb19<T> a, b, ta, tb;   // ta, tb: theta (linear smoother)
            if constexpr (LIN) {
                gather19_il(sm, om, oc, op, S0, O0, a, ta);
                gather19_il(sm, om, oc, op, S0 + D, O0 + D, b, tb);
            } else {
                a = gather19<T>(sm, om, oc, op, S0, O0);
                b = gather19<T>(sm, om, oc, op, S0 + D, O0 + D);
            }
            a.xp = sm[rp + Q0 + pb];
            a.xm = sm[rm + Q0 + pb];
            a.yp = sm[rc + Q0 + kRH + pb];
            a.ym = sm[rc + Q0 - kRH + pb];
            a.zp = sm[rc + Q0 + 1];
            a.zm = sm[rc + Q0];
            b.xp = sm[rp + Q0 + DR + pb];
            b.xm = sm[rm + Q0 + DR + pb];
            b.yp = sm[rc + Q0 + DR + kRH + pb];
            b.ym = sm[rc + Q0 + DR - kRH + pb];
            b.zp = sm[rc + Q0 + DR + 1];
            b.zm = sm[rc + Q0 + DR];
            const unsigned gb0 = sb + (unsigned)gj * (unsigned)N + (unsigned)gk0;
            const unsigned gb1 = gb0 + 8u * (unsigned)N;
            const float2 rhs = make_float2(in0 ? g[gb0 + pb] : T(1), in1 ? g[gb1 + pb] : T(1));
            float2 vb;
            if constexpr (LIN) {
                vb = lin_update2(pack19(ta, tb), pack19(a, b), rhs, ih2, T(6) * h2_6);
            } else {
                vb = fas_update2(pack19(a, b), add2(rhs, f2(c)), ih2, h2_6, rule);
            }
            const T vr0 = sm[rc + Q0 + 1 - pb], vr1 = sm[rc + Q0 + DR + 1 - pb];
            if (in0) *reinterpret_cast<float2 *>(dst + gb0) = pb ? make_float2(vr0, vb.x) : make_float2(vb.x, vr0);
            if (in1) *reinterpret_cast<float2 *>(dst + gb1) = pb ? make_float2(vr1, vb.y) : make_float2(vb.y, vr1);
        } else {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int gj = j0 + w + 8 * i;
                if (gj >= N || gk0 >= N) continue;
                const int S = S0 + 8 * i * kOR, O = O0 + 8 * i * kOR, Q = Q0 + 8 * i * kRH;
                Nb19<T> nb, nt;   // nt: theta (linear smoother)
                if constexpr (LIN) {
                    gather19_il(sm, om, oc, op, S, O, nb, nt);
                } else {
                    nb = gather19<T>(sm, om, oc, op, S, O);
                }
                nb.xp = sm[rp + Q + pb];
                nb.xm = sm[rm + Q + pb];
                nb.yp = sm[rc + Q + kRH + pb];
                nb.ym = sm[rc + Q - kRH + pb];
                nb.zp = sm[rc + Q + 1];
                nb.zm = sm[rc + Q];
                const unsigned gb = sb + (unsigned)gj * (unsigned)N + (unsigned)gk0;
                T vb;
                if constexpr (LIN) {
                    vb = lin_update<T>(nt, nb, g[gb + pb], ih2);
                } else {
                    vb = fas_update<T>(nb, g[gb + pb] + c, ih2, h2_6, rule);
                }
                const T vr = sm[rc + Q + 1 - pb];
                typename Pair<T>::type v;
                v.x = pb ? vr : vb;
                v.y = pb ? vb : vr;
                *reinterpret_cast<typename Pair<T>::type *>(dst + gb) = v;
            }
        }
    };

    // prologue: OLD planes i0-2 .. i0+2 into slots 0..4, then RED planes
    // i0-1 .. i0+1 into RED slots 0..2 while plane i0+3 arrives in slot 5.
    // The chunk needs OLD planes i0-2 .. i1+1 and RED planes i0-1 .. i1.
    for (int d = 0; d < 5; ++d) issue_plane(d * kOPlane, i0 - 2 + d);
    cp_async_wait<0>();
    __syncthreads();
    if (i0 + 3 <= i1 + 1) issue_plane(5 * kOPlane, i0 + 3);
    constexpr int kRB = red_base<LIN>();
    red_plane(i0 - 1, 0 * kOPlane, 1 * kOPlane, 2 * kOPlane, kRB + 0 * kRPlane);
    red_plane(i0, 1 * kOPlane, 2 * kOPlane, 3 * kOPlane, kRB + 1 * kRPlane);
    red_plane(i0 + 1, 2 * kOPlane, 3 * kOPlane, 4 * kOPlane, kRB + 2 * kRPlane);
    // ring slots of OLD planes s-1 .. s+4 and RED planes s-1 .. s+2
    int o0 = 1 * kOPlane, o1 = 2 * kOPlane, o2 = 3 * kOPlane, o3 = 4 * kOPlane, o4 = 5 * kOPlane, o5 = 0;
    int q0 = kRB, q1 = kRB + kRPlane, q2 = kRB + 2 * kRPlane, q3 = kRB + 3 * kRPlane;
    for (int s = i0; s < i1; ++s) {
        cp_async_wait<0>();   // this thread's copies of plane s+3 have landed
        __syncthreads();      // everyone's; RED s+1 written; slots of planes s-2 free
        if (s + 4 <= i1 + 1) issue_plane(o5, s + 4);
        if (s + 2 <= i1) red_plane(s + 2, o2, o3, o4, q3);
        black_plane(s, o0, o1, o2, q0, q1, q2);
        const int to = o0;
        o0 = o1;
        o1 = o2;
        o2 = o3;
        o3 = o4;
        o4 = o5;
        o5 = to;
        const int tq = q0;
        q0 = q1;
        q1 = q2;
        q2 = q3;
        q3 = tq;
    }
    cp_async_wait<0>();
}

template <typename T, bool LIN>
static cudaError_t fused_attr()
{
    return cudaFuncSetAttribute(k_sweep_fused<T, LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fused_smem_bytes<T, LIN>());
}

static bool g_kernels_ready = false;
static cudaError_t coarse_attrs();   // shared-memory limits of the coarsest solves
static cudaError_t tail_attrs();     // and of the single-block V-cycle tails
// planes per CTA of the fused sweeps for the solve being enqueued on this
// host thread (recon_config.fused_chunk; 0 = by grid size)
static thread_local int g_fused_chunk = 0;
void set_fused_chunk(int c) { g_fused_chunk = c; }

cudaError_t prepare_kernels()
{
    cudaError_t e = fused_attr<float, false>();
    if (e == cudaSuccess) e = fused_attr<double, false>();
    if (e == cudaSuccess) e = fused_attr<float, true>();
    if (e == cudaSuccess) e = prepare_reg_sweeps();
    if (e == cudaSuccess) e = coarse_attrs();
    if (e == cudaSuccess) e = tail_attrs();
    if (e == cudaSuccess) g_kernels_ready = true;
    return e;
}

// The fused sweeps store (even k, odd k) pairs as one vector: the arrays they
// write must be aligned to two elements (true of every allocation; a caller's
// offset view may not be, and then the two-pass kernels run instead).
template <typename T>
static inline bool pair_aligned(const T *p)
{
    return ((uintptr_t)p % (2 * sizeof(T))) == 0;
}

// th: the theta of the linear variant (nullptr for the nonlinear one)
template <typename T, bool LIN>
static cudaError_t fused_sweep_launch(int N, const T *src, T *dst, const T *g, const T *th,
                                      const double *cptr, double cval, T ih2, T h2_6, int rule,
                                      cudaStream_t s)
{
    // set once per process (recon_create does it before any graph capture;
    // step entry points may run without a handle)
    const size_t smem = fused_smem_bytes<T, LIN>();
    if (!g_kernels_ready) {
        const cudaError_t e = prepare_kernels();
        if (e != cudaSuccess) return e;
    }
    const int CI = g_fused_chunk > 0 ? g_fused_chunk : (N >= 512 ? 64 : (N >= 256 ? 32 : 16));
    const dim3 grid((N + kTK - 1) / kTK, (N + kTJ - 1) / kTJ, (N + CI - 1) / CI);
    note_launch();
    k_sweep_fused<T, LIN><<<grid, kFT, smem, s>>>(src, dst, g, th, cptr, cval, N, CI, ih2, h2_6, rule);
    return cudaGetLastError();
}

template <typename T>
cudaError_t sweep(int N, double h, int rule, T *t, const T *g, const double *cptr,
                  double cval, int sweeps, T *work, cudaStream_t s, const double *gshift)
{
    const T ih2 = (T)(1.0 / (h * h)), h2_6 = (T)(h * h / 6.0);
    if constexpr (std::is_same<T, float>::value) {
        if (sweeps > 0 && reg_sweep_ok(N, t, work, g, nullptr) && reg_sweep_ok(N, work, t, g, nullptr)) {
            T *a = t, *b = work;
            for (int it = 0; it < sweeps; ++it) {
                const cudaError_t e = reg_sweep_launch(false, N, a, b, g, nullptr, cptr, cval, ih2, h2_6, rule,
                                                       g_fused_chunk, s, it == 0 ? gshift : nullptr);
                if (e != cudaSuccess) return e;
                T *tmp = a;
                a = b;
                b = tmp;
            }
            if (a != t) return cudaMemcpyAsync(t, a, sizeof(T) * (size_t)N * N * N, cudaMemcpyDeviceToDevice, s);
            return cudaSuccess;
        }
    }
    if (gshift) {   // no kernel here folds it: subtract first
        note_launch();
        k_gauge_by<T><<<stride_blocks((size_t)N * N * N), kThreads, 0, s>>>(t, (size_t)N * N * N, gshift);
    }
    if (N >= kFusedMinN && pair_aligned(t) && pair_aligned(work)) {
        T *a = t, *b = work;
        for (int it = 0; it < sweeps; ++it) {
            const cudaError_t e = fused_sweep_launch<T, false>(N, a, b, g, (const T *)nullptr, cptr, cval, ih2, h2_6, rule, s);
            if (e != cudaSuccess) return e;
            T *tmp = a;
            a = b;
            b = tmp;
        }
        if (a != t) return cudaMemcpyAsync(t, a, sizeof(T) * (size_t)N * N * N, cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    for (int it = 0; it < sweeps; ++it) {
        note_launch(2);
        k_rb_pass<T><<<row_grid(N), row_block(), 0, s>>>(t, work, g, cptr, cval, N, ih2, h2_6, 0, rule);
        k_rb_pass<T><<<row_grid(N), row_block(), 0, s>>>(work, t, g, cptr, cval, N, ih2, h2_6, 1, rule);
    }
    return cudaGetLastError();
}
template cudaError_t sweep<double>(int, double, int, double *, const double *, const double *, double, int, double *, cudaStream_t, const double *);
template cudaError_t sweep<float>(int, double, int, float *, const float *, const double *, double, int, float *, cudaStream_t, const double *);

// ======================================================================
// residuals
// ======================================================================
__global__ void __launch_bounds__(kRowThreads)
k_residual_write(const double *__restrict__ t, const double *__restrict__ g,
                 const double *__restrict__ cptr, double cval, int N, double ih2,
                 double *__restrict__ r)
{
    const double c = cptr ? *cptr : cval;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const unsigned id = offs(N, i, j, k);
        r[id] = (g[id] + c) - det_IH(load19<double>(t, N, i, j, k), ih2);
    }
}

__global__ void __launch_bounds__(kRowThreads)
k_det_write(const double *__restrict__ t, int N, double ih2, double *__restrict__ out)
{
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX)
        out[offs(N, i, j, k)] = det_IH(load19<double>(t, N, i, j, k), ih2);
}

// partials[4 b + 0..2] = sum r, sum r^2, sum theta over this block's cells,
// r = g + c - det(I + H theta).  When f32out is set (mixed path, T = double)
// the residual is also stored as float and theta as float in t32out.
template <typename T>
__global__ void __launch_bounds__(kRowThreads)
k_residual_norms(const T *__restrict__ t, const T *__restrict__ g,
                 const double *__restrict__ cptr, int N, T ih2, double *__restrict__ partials,
                 float *__restrict__ f32out, float *__restrict__ t32out)
{
    __shared__ double sh[32];
    const T c = (T)(*cptr);
    ThreadSum<T> sr, sr2, st;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const unsigned id = offs(N, i, j, k);
        const Nb19<T> nb = load19<T>(t, N, i, j, k);
        const T res = (g[id] + c) - det_IH(nb, ih2);
        sr.add(res);
        sr2.add(res * res);
        st.add(nb.c);
        if (f32out) {
            f32out[id] = (float)res;
            t32out[id] = (float)nb.c;
        }
    }
    double v = block_sum<kRowThreads>(sr.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
    v = block_sum<kRowThreads>(sr2.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 1] = v;
    v = block_sum<kRowThreads>(st.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 2] = v;
}

// Single block: total of column `col` of the partials, in a fixed order.
__device__ double sum_partials(const double *partials, int nb, int col, double *sh)
{
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[4 * b + col];
    return block_sum<kReduceThreads>(v, sh);
}

// After a cycle on a level with n cells: m = mean r; c -= m;
// rel = sqrt(sum (r - m)^2) / denom; mean theta for the gauge.
__global__ void __launch_bounds__(kReduceThreads)
k_finalize_cycle(const double *__restrict__ partials, int nb, double n, double *scal)
{
    __shared__ double sh[32];
    const double sr = sum_partials(partials, nb, 0, sh);
    const double sr2 = sum_partials(partials, nb, 1, sh);
    const double st = sum_partials(partials, nb, 2, sh);
    if (ltid() == 0) {
        const double m = sr / n;
        const double var = sr2 - n * m * m;
        scal[S_MEAN_R] = m;
        scal[S_C] -= m;
        scal[S_REL] = sqrt(var > 0.0 ? var : 0.0) / scal[S_DENOM];
        scal[S_MEAN_T] = st / n;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_gauge(T *__restrict__ t, size_t n, const double *__restrict__ scal)
{
    const T m = (T)scal[S_MEAN_T];
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x)
        t[id] -= m;
}

// ======================================================================
// transfers
// ======================================================================
// Fused residual + restriction: per coarse cell, the 8 sons' residuals
// r = g + c - det(I + H theta) and values are averaged (Sec. II.A.3: coarse
// value = mean of the 8 son cells); the fine residual is never stored.
// Fine windows of the restrictions.  Every 19-point stencil of the eight
// children (2I+a, 2J+b, 2K+c) of coarse cell (I, J, K) lies in the fine block
// i, j, k in 2I-1 .. 2I+2 (etc.) without the corners of its two outer
// planes: 56 loads instead of 8 x 19.  Window index 1 + a is child a.
// CTAs per SM the windowed kernels are compiled for (their 56-value windows
// need ~120 registers at 2; the FP32 residual/restriction and norm kernels
// also fit at 3)
#ifndef RECON_WIN_CTAS
#define RECON_WIN_CTAS 2
#endif
#ifndef RECON_RR_CTAS_F
#define RECON_RR_CTAS_F 2
#endif
#ifndef RECON_NW_CTAS_F
#define RECON_NW_CTAS_F 2
#endif
struct Win {
    unsigned pl[4], row[4], col[4];
    __device__ __forceinline__ Win(int Nf, int I, int J, int K)
    {
        const unsigned nn = (unsigned)Nf * (unsigned)Nf;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            pl[d] = (unsigned)wrap1(2 * I - 1 + d, Nf) * nn;
            row[d] = (unsigned)wrap1(2 * J - 1 + d, Nf) * (unsigned)Nf;
            col[d] = (unsigned)wrap1(2 * K - 1 + d, Nf);
        }
    }
    __device__ __forceinline__ unsigned at(int d, int b, int c) const { return pl[d] + row[b] + col[c]; }
};

// window plane d of array a; the corners are loaded only for inner planes
template <typename T, bool INNER>
__device__ __forceinline__ void win_plane(const T *__restrict__ a, const Win &w, int d, T (&P)[4][4])
{
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            P[b][c] = (!INNER && (b == 0 || b == 3) && (c == 0 || c == 3)) ? T(0) : a[w.at(d, b, c)];
}

// 19-point neighbourhood of the child at window (b, c) of the middle plane
template <typename T>
__device__ __forceinline__ Nb19<T> win_nb(const T (&Pm)[4][4], const T (&Pc)[4][4], const T (&Pp)[4][4],
                                          int b, int c)
{
    Nb19<T> v;
    v.c = Pc[b][c];
    v.xp = Pp[b][c];
    v.xm = Pm[b][c];
    v.yp = Pc[b + 1][c];
    v.ym = Pc[b - 1][c];
    v.zp = Pc[b][c + 1];
    v.zm = Pc[b][c - 1];
    v.xpyp = Pp[b + 1][c];
    v.xmym = Pm[b - 1][c];
    v.xmyp = Pm[b + 1][c];
    v.xpym = Pp[b - 1][c];
    v.ypzp = Pc[b + 1][c + 1];
    v.ymzm = Pc[b - 1][c - 1];
    v.ymzp = Pc[b - 1][c + 1];
    v.ypzm = Pc[b + 1][c - 1];
    v.xpzp = Pp[b][c + 1];
    v.xmzm = Pm[b][c - 1];
    v.xmzp = Pm[b][c + 1];
    v.xpzm = Pp[b][c - 1];
    return v;
}

// Residual norms of an even grid from the fine windows of its 2 x 2 x 2
// blocks (7 loads per cell instead of 19); same outputs as k_residual_norms.
template <typename T>
__global__ void __launch_bounds__(kRowThreads, sizeof(T) == 4 ? RECON_NW_CTAS_F : RECON_WIN_CTAS)
k_residual_norms_win(const T *__restrict__ t, const T *__restrict__ g,
                     const double *__restrict__ cptr, int N, T ih2, double *__restrict__ partials,
                     float *__restrict__ f32out, float *__restrict__ t32out)
{
    __shared__ double sh[32];
    const T c = (T)(*cptr);
    const int Nc = N >> 1;
    ThreadSum<T> sr, sr2, st;
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        const Win w(N, I, J, K);
        T P0[4][4], P1[4][4], P2[4][4];
        win_plane<T, false>(t, w, 0, P0);
        win_plane<T, true>(t, w, 1, P1);
        win_plane<T, true>(t, w, 2, P2);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a == 1) win_plane<T, false>(t, w, 3, P0);
#pragma unroll
            for (int b = 1; b <= 2; ++b)
#pragma unroll
                for (int cc = 1; cc <= 2; ++cc) {
                    const Nb19<T> nb = a == 0 ? win_nb<T>(P0, P1, P2, b, cc) : win_nb<T>(P1, P2, P0, b, cc);
                    const unsigned id = w.at(1 + a, b, cc);
                    const T res = (g[id] + c) - det_IH(nb, ih2);
                    sr.add(res);
                    sr2.add(res * res);
                    st.add(nb.c);
                    if (f32out) {
                        f32out[id] = (float)res;
                        t32out[id] = (float)nb.c;
                    }
                }
        }
    }
    double v = block_sum<kRowThreads>(sr.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
    v = block_sum<kRowThreads>(sr2.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 1] = v;
    v = block_sum<kRowThreads>(st.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 2] = v;
}

// Residual norms on any grid: the windowed kernel for even N >= 32
template <typename T>
static unsigned launch_residual_norms(const T *t, const T *g, const double *cptr, int N, T ih2,
                                      double *partials, float *f32out, float *t32out, cudaStream_t s)
{
    note_launch();
    if (N % 2 == 0 && N >= 32) {
        const unsigned nbr = row_grid(N / 2, kMaxRedBlocks);
        k_residual_norms_win<T><<<nbr, row_block(), 0, s>>>(t, g, cptr, N, ih2, partials, f32out, t32out);
        return nbr;
    }
    const unsigned nbr = row_grid(N, kMaxRedBlocks);
    k_residual_norms<T><<<nbr, row_block(), 0, s>>>(t, g, cptr, N, ih2, partials, f32out, t32out);
    return nbr;
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads, sizeof(T) == 4 ? RECON_RR_CTAS_F : RECON_WIN_CTAS)
k_restrict_residual(const T *__restrict__ t, const T *__restrict__ g,
                    const double *__restrict__ cptr, int Nf, T ih2, T *__restrict__ tH,
                    T *__restrict__ toldH, T *__restrict__ rrH, double *__restrict__ partials)
{
    __shared__ double sh[32];
    const int Nc = Nf >> 1;
    const T c = (T)(*cptr);
    ThreadSum<T> srr;
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        const Win w(Nf, I, J, K);
        T P0[4][4], P1[4][4], P2[4][4];
        win_plane<T, false>(t, w, 0, P0);
        win_plane<T, true>(t, w, 1, P1);
        win_plane<T, true>(t, w, 2, P2);
        T at = T(0), ar = T(0);
#pragma unroll
        for (int b = 1; b <= 2; ++b)
#pragma unroll
            for (int cc = 1; cc <= 2; ++cc) {   // children in fine plane 2I: window planes 0..2
                const Nb19<T> nb = win_nb<T>(P0, P1, P2, b, cc);
                at += nb.c;
                ar += (g[w.at(1, b, cc)] + c) - det_IH(nb, ih2);
            }
        win_plane<T, false>(t, w, 3, P0);   // children in fine plane 2I+1: planes 1..3
#pragma unroll
        for (int b = 1; b <= 2; ++b)
#pragma unroll
            for (int cc = 1; cc <= 2; ++cc) {
                const Nb19<T> nb = win_nb<T>(P1, P2, P0, b, cc);
                at += nb.c;
                ar += (g[w.at(2, b, cc)] + c) - det_IH(nb, ih2);
            }
        const T vt = at * T(0.125), vr = ar * T(0.125);
        const unsigned id = offs(Nc, I, J, K);
        tH[id] = vt;
        toldH[id] = vt;
        rrH[id] = vr;
        srr.add(vr);
    }
    const double v = block_sum<kRowThreads>(srr.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
}

__global__ void __launch_bounds__(kReduceThreads)
k_finalize_mean(const double *__restrict__ partials, int nb, double n, double *out)
{
    __shared__ double sh[32];
    const double s = sum_partials(partials, nb, 0, sh);
    if (ltid() == 0) *out = s / n;
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads)
k_restrict_plain(const T *__restrict__ f, int Nf, T *__restrict__ cr)
{
    const int Nc = Nf >> 1;
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        T acc = T(0);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int cc = 0; cc < 2; ++cc) acc += f[offs(Nf, 2 * I + a, 2 * J + b, 2 * K + cc)];
        cr[offs(Nc, I, J, K)] = acc * T(0.125);
    }
}

template <typename T>
cudaError_t restrict_plain(int Nf, const T *fine, T *coarse, cudaStream_t s)
{
    note_launch();
    k_restrict_plain<T><<<row_grid(Nf / 2), row_block(), 0, s>>>(fine, Nf, coarse);
    return cudaGetLastError();
}
template cudaError_t restrict_plain<double>(int, const double *, double *, cudaStream_t);
template cudaError_t restrict_plain<float>(int, const float *, float *, cudaStream_t);

// Coarse right side, first half: rr = R r - mean(R r) (stored back in gH),
// dH = det_H(I + H theta_H) (stored in aux), and the block minimum of the
// scaled-defect ratio floor * max(dH, 0) / (-rr) over cells with rr < 0.
template <typename T>
__global__ void __launch_bounds__(kRowThreads)
k_coarse_rhs(const T *__restrict__ tH, T *__restrict__ gH, T *__restrict__ dH,
             const double *__restrict__ mean_ptr, int Nc, T ih2, double floor_,
             double *__restrict__ partials)
{
    __shared__ double sh[32];
    const T m = (T)(*mean_ptr);
    const T fl = (T)floor_;
    T mn = T(INFINITY);
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        const unsigned id = offs(Nc, I, J, K);
        const T rr = gH[id] - m;
        const T d = det_IH(load19<T>(tH, Nc, I, J, K), ih2);
        gH[id] = rr;
        dH[id] = d;
        if (rr < T(0)) {
            const T cand = fl * (d > T(0) ? d : T(0)) / (-rr);
            mn = cand < mn ? cand : mn;
        }
    }
    const double v = block_min<kRowThreads>((double)mn, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 3] = v;
}

// s = min(1, min ratio) (1 when the safeguard is off); s < 1e-3 -> 0 (skip).
__global__ void __launch_bounds__(kReduceThreads)
k_finalize_scale(const double *__restrict__ partials, int nb, double floor_, double *sslot,
                 double *pslot)
{
    __shared__ double sh[32];
    double v = INFINITY;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v = fmin(v, partials[4 * b + 3]);
    v = block_min<kReduceThreads>(v, sh);
    if (ltid() == 0) {
        double s = floor_ <= 0.0 ? 1.0 : fmin(1.0, v);
        if (s < 1e-3) s = 0.0;
        *sslot = s;
        *pslot = s > 0.0 ? 1.0 / s : 0.0;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_form_rhs(T *__restrict__ gH, const T *__restrict__ dH, size_t nc,
           const double *__restrict__ sslot)
{
    const T sc = (T)(*sslot);
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < nc;
         id += (size_t)gridDim.x * blockDim.x)
        gH[id] = dH[id] + sc * gH[id];
}

// fine += scale * P(cnew - cold), P cell-centred trilinear: per axis the
// parent weighs 3/4 and the coarse neighbour on the fine cell's side 1/4.
// scale = *pscale when pscale is given (0 = no correction), else `scale`.
// A thread takes one coarse cell (threads along K, rows (I, J) grid-stride)
// and its 2 x 2 x 2 children: the 27 coarse differences d = cnew - cold
// around the parent are formed once and interpolated axis by axis (i, then
// j, then k; the product weights of the trilinear form factorise), and each
// child pair along k is read and written as one vector when `fine` is
// aligned to a pair.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
__global__ void __launch_bounds__(kRowThreads)
k_prolong_add(const T *__restrict__ cnew, const T *__restrict__ cold, int Nc,
              const double *__restrict__ pscale, double scale, T *__restrict__ fine, int pairs)
{
    using V2 = typename Vec2<T>::type;
    const double sc = pscale ? *pscale : scale;
    if (sc == 0.0) return;
    const T s = (T)sc, w0 = T(0.75), w1 = T(0.25);
    const int Nf = 2 * Nc;
    FOR_ROWS(Nc, I, J)
    {
        const int Ip[3] = {I == 0 ? Nc - 1 : I - 1, I, I + 1 == Nc ? 0 : I + 1};
        const int Jp[3] = {J == 0 ? Nc - 1 : J - 1, J, J + 1 == Nc ? 0 : J + 1};
        for (int K = threadIdx.x; K < Nc; K += kRowX) {
            const int Kp[3] = {K == 0 ? Nc - 1 : K - 1, K, K + 1 == Nc ? 0 : K + 1};
            // the four fine pairs first: their DRAM reads overlap the coarse loads
            unsigned fo[2][2];
            V2 fv[2][2];
#pragma unroll
            for (int ei = 0; ei < 2; ++ei)
#pragma unroll
                for (int ej = 0; ej < 2; ++ej) {
                    fo[ei][ej] = offs(Nf, 2 * I + ei, 2 * J + ej, 2 * K);
                    if (pairs) {
                        fv[ei][ej] = *reinterpret_cast<const V2 *>(fine + fo[ei][ej]);
                    } else {
                        fv[ei][ej].x = fine[fo[ei][ej]];
                        fv[ei][ej].y = fine[fo[ei][ej] + 1];
                    }
                }
            T d[3][3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const unsigned o = offs(Nc, Ip[a], Jp[b], Kp[c]);
                        d[a][b][c] = cold ? cnew[o] - cold[o] : cnew[o];
                    }
#pragma unroll
            for (int ei = 0; ei < 2; ++ei) {
                T u[3][3];   // along i: child ei takes the neighbour 2 (ei = 1) or 0
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) u[b][c] = w0 * d[1][b][c] + w1 * d[ei ? 2 : 0][b][c];
#pragma unroll
                for (int ej = 0; ej < 2; ++ej) {
                    T v[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[c] = w0 * u[1][c] + w1 * u[ej ? 2 : 0][c];
                    V2 x = fv[ei][ej];
                    x.x += s * (w0 * v[1] + w1 * v[0]);
                    x.y += s * (w0 * v[1] + w1 * v[2]);
                    if (pairs) {
                        *reinterpret_cast<V2 *>(fine + fo[ei][ej]) = x;
                    } else {
                        fine[fo[ei][ej]] = x.x;
                        fine[fo[ei][ej] + 1] = x.y;
                    }
                }
            }
        }
    }
}

template <typename T>
cudaError_t prolong_add(int Nc, const T *cnew, const T *cold, const double *pscale,
                        double scale, T *fine, cudaStream_t s)
{
    note_launch();
    const int pairs = ((uintptr_t)fine % (2 * sizeof(T))) == 0;
    k_prolong_add<T><<<row_grid(Nc), row_block(), 0, s>>>(cnew, cold, Nc, pscale, scale, fine, pairs);
    return cudaGetLastError();
}
template cudaError_t prolong_add<double>(int, const double *, const double *, const double *, double, double *, cudaStream_t);
template cudaError_t prolong_add<float>(int, const float *, const float *, const double *, double, float *, cudaStream_t);

// ======================================================================
// coarsest grid: one thread block, N^3 <= 4096, sweeps until the mean-free
// rms residual drops by rtol, or a sweep no longer lowers it (round-off
// floor, only when rtol > 0), or max_sweeps ran (at least one sweep).
// t and work are read and written by different threads of the block across
// __syncthreads(), so they are plain (not read-only) pointers.
// ======================================================================
template <typename T, int NT>
__device__ double coarse_proj_rms(const T *t, T *work, const T *g, T c, int N, T ih2,
                                  double *sh, double *sval)
{
    const int n = N * N * N;
    double sr = 0.0;
    for (int id = threadIdx.x; id < n; id += blockDim.x) {
        const int k = id % N, j = (id / N) % N, i = id / (N * N);
        const T r = (g[id] + c) - det_IH(load19<T>(t, N, i, j, k), ih2);
        work[id] = r;
        sr += (double)r;
    }
    double tot = block_sum<NT>(sr, sh);
    if (ltid() == 0) *sval = tot / n;
    __syncthreads();
    const double m = *sval;
    double s2 = 0.0;
    for (int id = threadIdx.x; id < n; id += blockDim.x) {
        const double d = (double)work[id] - m;
        s2 += d * d;
    }
    tot = block_sum<NT>(s2, sh);
    if (ltid() == 0) *sval = sqrt(tot / n);
    __syncthreads();
    const double v = *sval;
    __syncthreads();
    return v;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_coarse_solve(T *t, T *work, const T *g, const double *cptr, double cval, int N, T ih2, T h2_6,
               int rule, int max_sweeps, double rtol, int *sweeps_out)
{
    // the grid (<= 16^3) is relaxed in shared memory: theta, the colour
    // pass's scratch and g are staged once and theta is written back at the
    // end (the global scratch `work` is not touched)
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    __shared__ double sh[32];
    __shared__ double sval;
    const int n = N * N * N;
    T *ts = reinterpret_cast<T *>(coarse_smem), *ws = ts + n, *gs = ws + n;
    for (int id = threadIdx.x; id < n; id += blockDim.x) {
        ts[id] = t[id];
        gs[id] = g[id];
    }
    __syncthreads();
    const T c = (T)(cptr ? *cptr : cval);
    const int half = N >> 1;
    const int npairs = N * N * half;
    const double r0 = coarse_proj_rms<T, NT>(ts, ws, gs, c, N, ih2, sh, &sval);
    double prev = r0;
    int sw = 0;
    while (sw < max_sweeps) {
        for (int colour = 0; colour < 2; ++colour) {
            const T *src = colour == 0 ? ts : ws;
            T *dst = colour == 0 ? ws : ts;
            for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
                const int m = pi % half, r = pi / half;
                const int j = r % N, i = r / N;
                const int par = (colour + i + j) & 1;
                const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                const Nb19<T> nb = load19<T>(src, N, i, j, ka);
                T s, p, q;
                cubic_coeffs(nb, ih2, gs[offs(N, i, j, ka)] + c, s, p, q);
                const T vnew = point_update(nb.c, h2_6, s, p, q, rule);
                const T vcopy = src[offs(N, i, j, kb)];
                dst[offs(N, i, j, ka)] = vnew;
                dst[offs(N, i, j, kb)] = vcopy;
            }
            __syncthreads();
        }
        ++sw;
        const double cur = coarse_proj_rms<T, NT>(ts, ws, gs, c, N, ih2, sh, &sval);
        if (cur <= rtol * r0) break;
        if (rtol > 0.0 && cur >= prev) break;   // no progress: round-off floor
        prev = cur;
    }
    for (int id = threadIdx.x; id < n; id += blockDim.x) t[id] = ts[id];
    if (ltid() == 0 && sweeps_out) *sweeps_out = sw;
}

template <typename T>
cudaError_t coarse_solve(int N, double h, int rule, T *t, const T *g, const double *cptr,
                         double cval, int max_sweeps, double rtol, T *work, int *sweeps_out,
                         cudaStream_t s)
{
    const T ih2 = (T)(1.0 / (h * h)), h2_6 = (T)(h * h / 6.0);
    if ((long)N * N * N > kMaxCoarseCells) return cudaErrorInvalidValue;
    if (!g_kernels_ready) {
        const cudaError_t e = prepare_kernels();
        if (e != cudaSuccess) return e;
    }
    note_launch();
    // one thread per cell pair up to 128 pairs (the block-wide sums and
    // barriers of every sweep are cheaper with fewer warps), 512 beyond
    const size_t smem = 3 * sizeof(T) * (size_t)N * N * N;
    const int pairs = N * N * N / 2;
    if (pairs <= 64)
        k_coarse_solve<T, 64><<<1, 64, smem, s>>>(t, work, g, cptr, cval, N, ih2, h2_6, rule, max_sweeps, rtol,
                                                  sweeps_out);
    else if (pairs <= 128)
        k_coarse_solve<T, 128><<<1, 128, smem, s>>>(t, work, g, cptr, cval, N, ih2, h2_6, rule, max_sweeps,
                                                    rtol, sweeps_out);
    else
        k_coarse_solve<T, kCoarseThreads><<<1, kCoarseThreads, smem, s>>>(t, work, g, cptr, cval, N, ih2, h2_6,
                                                                          rule, max_sweeps, rtol, sweeps_out);
    return cudaGetLastError();
}
template cudaError_t coarse_solve<double>(int, double, int, double *, const double *, const double *, double, int, double, double *, int *, cudaStream_t);
template cudaError_t coarse_solve<float>(int, double, int, float *, const float *, const double *, double, int, double, float *, int *, cudaStream_t);

// ======================================================================
// Jacobian (linearisation of det(I + H theta))
// ======================================================================
__global__ void __launch_bounds__(kRowThreads)
k_jacobian_apply(const double *__restrict__ t, const double *__restrict__ v, int N, double ih2,
                 double *__restrict__ out)
{
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const Cof<double> a = cofactors(load19<double>(t, N, i, j, k), ih2);
        out[offs(N, i, j, k)] = jac_apply(a, load19<double>(v, N, i, j, k), ih2);
    }
}

cudaError_t jacobian_apply(int N, double h, const double *t, const double *v, double *out,
                           cudaStream_t s)
{
    note_launch();
    k_jacobian_apply<<<row_grid(N), row_block(), 0, s>>>(t, v, N, 1.0 / (h * h), out);
    return cudaGetLastError();
}

cudaError_t residual_write(int N, double h, const double *t, const double *g,
                           const double *cptr, double cval, double *r, cudaStream_t s)
{
    note_launch();
    k_residual_write<<<row_grid(N), row_block(), 0, s>>>(t, g, cptr, cval, N, 1.0 / (h * h), r);
    return cudaGetLastError();
}

cudaError_t det_write(int N, double h, const double *t, double *out, cudaStream_t s)
{
    note_launch();
    k_det_write<<<row_grid(N), row_block(), 0, s>>>(t, N, 1.0 / (h * h), out);
    return cudaGetLastError();
}

// ======================================================================
// domain check of b and the stop-rule denominator ||b - 1||_2
// ======================================================================
__global__ void __launch_bounds__(kThreads)
k_b_stats(const double *__restrict__ b, size_t n, double *__restrict__ partials)
{
    // finiteness and the minimum on the bit patterns (integer pipes); the
    // norm from the FP64 difference b - 1 widened once per thread.
    __shared__ double sh[32];
    ThreadSum<float> s2;
    long long kmin = LLONG_MAX;   // order-preserving key of the smallest finite b
    unsigned bad = 0;
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x) {
        const double v = b[id];
        const long long bits = __double_as_longlong(v);
        if (((bits >> 52) & 0x7ff) == 0x7ff) {
            ++bad;
        } else {
            const long long key = bits < 0 ? (bits ^ LLONG_MAX) : bits;
            kmin = key < kmin ? key : kmin;
            const float d = (float)(v - 1.0);
            s2.add(d * d);
        }
    }
    double v = block_sum<kThreads>(s2.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
    v = block_sum<kThreads>((double)bad, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 1] = v;
    const double mn = kmin == LLONG_MAX ? INFINITY
                                        : __longlong_as_double(kmin < 0 ? (kmin ^ LLONG_MAX) : kmin);
    v = block_min<kThreads>(mn, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 3] = v;
}

__global__ void __launch_bounds__(kReduceThreads)
k_finalize_b(const double *__restrict__ partials, int nb, double *scal)
{
    __shared__ double sh[32];
    const double s2 = sum_partials(partials, nb, 0, sh);
    const double bad = sum_partials(partials, nb, 1, sh);
    double mn = INFINITY;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) mn = fmin(mn, partials[4 * b + 3]);
    mn = block_min<kReduceThreads>(mn, sh);
    if (ltid() == 0) {
        scal[S_DENOM] = s2 > 0.0 ? sqrt(s2) : 1.0;
        scal[S_BBAD] = bad;
        scal[S_BMIN] = mn;
    }
}

// ======================================================================
// mixed-precision helpers
// ======================================================================
__global__ void __launch_bounds__(kThreads)
k_to_float(const double *__restrict__ a, float *__restrict__ out, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) out[id] = df_from_double_bits(a[id]).hi;   // RN(a), rounded with integer operations
}

__global__ void __launch_bounds__(kThreads)
k_to_double(const float *__restrict__ a, double *__restrict__ out, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) out[id] = (double)a[id];
}

// theta64 += e - mean(theta64) (defect-correction update with the gauge)
__global__ void __launch_bounds__(kThreads)
k_update_theta(double *__restrict__ t, const float *__restrict__ e, size_t n,
               const double *__restrict__ scal)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) t[id] = (t[id] - scal[S_MEAN_T]) + (double)e[id];
}

__global__ void __launch_bounds__(kThreads)
k_sub_scalar(float *__restrict__ a, size_t n, const double *__restrict__ v)
{
    const float m = (float)(*v);
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x)
        a[id] -= m;
}

// ---- double-float fine-grid residual of the mixed path
// r = b + c - det(I + H phi) with phi = phi_hi + phi_lo and b = b_hi + b_lo
// evaluated in double-float arithmetic (dfresid.cuh; POW2: 1/h^2 is a power
// of two); writes float(r) for the linear solve and the block partials
// sum r, sum r^2 (float per thread, double per block).
template <bool POW2>
__global__ void __launch_bounds__(kRowThreads)
k_residual_df(const float *__restrict__ phi_hi, const float *__restrict__ phi_lo,
              const float *__restrict__ b_hi, const float *__restrict__ b_lo,
              const double *__restrict__ cptr, int N, float ih2_hi, float ih2_lo,
              float *__restrict__ fout, double *__restrict__ partials)
{
    __shared__ double sh[32];
    const df c = df_from_double(*cptr);
    const df ih2 = df_make(ih2_hi, ih2_lo);
    float sr = 0.0f, sr2 = 0.0f;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const Nb19<float> H = load19<float>(phi_hi, N, i, j, k);
        const Nb19<float> Lo = load19<float>(phi_lo, N, i, j, k);
        const unsigned id = offs(N, i, j, k);
        const float rf = dfr_residual<POW2>(H, Lo, b_hi[id], b_lo[id], c, ih2);
        fout[id] = rf;
        sr += rf;
        sr2 = fmaf(rf, rf, sr2);
    }
    double v = block_sum<kRowThreads>((double)sr, sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
    v = block_sum<kRowThreads>((double)sr2, sh);
    if (ltid() == 0) {
        partials[4 * blockIdx.x + 1] = v;
        partials[4 * blockIdx.x + 2] = 0.0;   // no gauge shift while iterating
    }
}

// b -> (b_hi, b_lo)
__global__ void __launch_bounds__(kThreads)
k_split_df(const double *__restrict__ a, float *__restrict__ hi, float *__restrict__ lo, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) {
        const df v = df_from_double_bits(a[id]);
        hi[id] = v.hi;
        lo[id] = v.lo;
    }
}

// (phi_hi, phi_lo) += e
__global__ void __launch_bounds__(kThreads)
k_update_df(float *__restrict__ hi, float *__restrict__ lo, const float *__restrict__ e, size_t n)
{
    const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id < n) {
        const df v = df_add(df_make(hi[id], lo[id]), df_make(e[id], 0.0f));
        hi[id] = v.hi;
        lo[id] = v.lo;
    }
}

// block partial sums of phi_hi + phi_lo (double-float sums per thread)
__global__ void __launch_bounds__(kThreads)
k_df_sum(const float *__restrict__ hi, const float *__restrict__ lo, size_t n, double *__restrict__ partials)
{
    __shared__ double sh[32];
    df s = df_make(0.0f, 0.0f);
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x)
        s = df_add(s, df_make(hi[id], lo[id]));
    const double v = block_sum<kThreads>(df_to_double_bits(s), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
}

// phi = (phi_hi + phi_lo) - mean in FP64: the difference in double-float,
// then both parts widened exactly and added (one FP64 instruction per cell)
__global__ void __launch_bounds__(kThreads)
k_df_to_double_gauged(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ phi,
                      size_t n, const double *__restrict__ mean)
{
    const df m = df_from_double(*mean);
    for (size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x; id < n;
         id += (size_t)gridDim.x * blockDim.x)
        phi[id] = df_to_double_bits(df_sub(df_make(hi[id], lo[id]), m));
}

// ---- linear multigrid for J e = f in FP32.  J = sum adj(I + H theta)_ab D_ab
// with the FP32 theta of the level.  Grids of at least kFusedMinN form the
// cofactors from theta inside each kernel; the coarser grids read six
// cofactor arrays ([6][N^3]) computed once per correction (k_cof6f), stored
// colour-split within each row (cof_slot).
__global__ void __launch_bounds__(kRowThreads)
k_cof6f(const float *__restrict__ th, int N, float ih2, float *__restrict__ cof)
{
    const size_t n = (size_t)N * N * N;
    FOR_ROWS(N, i, j)
    for (int k = threadIdx.x; k < N; k += kRowX) {
        const Cof<float> a = cofactors(load19<float>(th, N, i, j, k), ih2);
        const unsigned id = cof_slot(N, i, j, k);
        cof[id] = a.xx;
        cof[n + id] = a.yy;
        cof[2 * n + id] = a.zz;
        cof[3 * n + id] = a.xy;
        cof[4 * n + id] = a.yz;
        cof[5 * n + id] = a.xz;
    }
}

__device__ __forceinline__ Cof<float> cof_at(const float *cof, size_t n, unsigned o)
{
    Cof<float> a;
    a.xx = cof[o];
    a.yy = cof[n + o];
    a.zz = cof[2 * n + o];
    a.xy = cof[3 * n + o];
    a.yz = cof[4 * n + o];
    a.xz = cof[5 * n + o];
    return a;
}

// One colour pass of Gauss-Seidel on J: e_c += (f - J e)_c / J_cc,
// J_cc = -2 (adj_xx + adj_yy + adj_zz) / h^2.
__global__ void __launch_bounds__(kRowThreads)
k_lin_pass(const float *__restrict__ src, float *__restrict__ dst, const float *__restrict__ f,
           const float *__restrict__ cof, int N, float ih2, int colour)
{
    const size_t n = (size_t)N * N * N;
    const int half = N >> 1;
    FOR_ROWS(N, i, j)
    {
        const int par = (colour + i + j) & 1;
        const unsigned base = offs(N, i, j, 0);
        for (int m = threadIdx.x; m < half; m += kRowX) {
            const int ka = 2 * m + par, kb = 2 * m + 1 - par;
            const Cof<float> a = cof_at(cof, n, cof_slot(N, i, j, ka));
            const Nb19<float> ev = load19<float>(src, N, i, j, ka);
            const float Je = jac_apply(a, ev, ih2);
            const float diag = -2.0f * (a.xx + a.yy + a.zz) * ih2;
            dst[base + ka] = ev.c + (f[base + ka] - Je) / diag;
            dst[base + kb] = src[base + kb];
        }
    }
}

static inline bool lin_fused(int N, const float *e, const float *work)
{
    return N >= kFusedMinN && pair_aligned(e) && pair_aligned(work);
}

// cof: the level's cofactor arrays (read by the two-pass kernels); th: its
// theta (read by the fused kernel)
// fshift (nullable): a device scalar subtracted from f on the fly; only the
// register-blocked kernel takes it (the caller checks lin_fold_ok)
static cudaError_t lin_sweep(int N, double h, float *e, const float *f, const float *cof,
                             const float *th, int sweeps, float *work, cudaStream_t s,
                             const double *fshift = nullptr)
{
    const float ih2 = (float)(1.0 / (h * h));
    if (reg_sweep_ok(N, e, work, f, th) && reg_sweep_ok(N, work, e, f, th)) {
        float *a = e, *b = work;
        for (int it = 0; it < sweeps; ++it) {
            const cudaError_t err = reg_sweep_launch(true, N, a, b, f, th, nullptr, 0.0, ih2, (float)(h * h / 6.0),
                                                     0, g_fused_chunk, s, fshift);
            if (err != cudaSuccess) return err;
            float *tmp = a;
            a = b;
            b = tmp;
        }
        if (a != e) return cudaMemcpyAsync(e, a, sizeof(float) * (size_t)N * N * N, cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    if (lin_fused(N, e, work)) {
        float *a = e, *b = work;
        for (int it = 0; it < sweeps; ++it) {
            const cudaError_t err = fused_sweep_launch<float, true>(N, a, b, f, th, nullptr, 0.0, ih2,
                                                                   (float)(h * h / 6.0), 0, s);
            if (err != cudaSuccess) return err;
            float *tmp = a;
            a = b;
            b = tmp;
        }
        if (a != e) return cudaMemcpyAsync(e, a, sizeof(float) * (size_t)N * N * N, cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    for (int it = 0; it < sweeps; ++it) {
        note_launch(2);
        k_lin_pass<<<row_grid(N), row_block(), 0, s>>>(e, work, f, cof, N, ih2, 0);
        k_lin_pass<<<row_grid(N), row_block(), 0, s>>>(work, e, f, cof, N, ih2, 1);
    }
    return cudaGetLastError();
}

cudaError_t linear_sweep(int N, double h, float *e, const float *f, const float *th, int sweeps,
                         float *work, cudaStream_t s)
{
    // work: N^3 ping-pong followed by room for the 6 N^3 cofactor arrays
    // (used by the two-pass kernels only)
    const size_t n = (size_t)N * N * N;
    float *cof = work + n;
    if (!lin_fused(N, e, work)) {
        note_launch();
        k_cof6f<<<row_grid(N), row_block(), 0, s>>>(th, N, (float)(1.0 / (h * h)), cof);
    }
    return lin_sweep(N, h, e, f, cof, th, sweeps, work, s);
}

// fH = R (f - J e), block partial sums for the mean projection, from the
// fine windows of e and (FROM_TH) theta; otherwise the cofactors come from
// the colour-split arrays cof.
template <bool FROM_TH>
__global__ void __launch_bounds__(kRowThreads, RECON_WIN_CTAS)
k_lin_restrict_residual(const float *__restrict__ e, const float *__restrict__ f,
                        const float *__restrict__ cof, const float *__restrict__ th, int Nf,
                        float ih2, float *__restrict__ fH, double *__restrict__ partials,
                        const double *__restrict__ fshift)
{
    __shared__ double sh[32];
    const size_t nf = (size_t)Nf * Nf * Nf;
    const int Nc = Nf >> 1;
    const float fs = fshift ? (float)*fshift : 0.0f;   // subtracted from f (its mean, folded in)
    ThreadSum<float> sacc;
    FOR_ROWS(Nc, I, J)
    for (int K = threadIdx.x; K < Nc; K += kRowX) {
        const Win w(Nf, I, J, K);
        float E0[4][4], E1[4][4], E2[4][4], T0[4][4], T1[4][4], T2[4][4];
        win_plane<float, false>(e, w, 0, E0);
        win_plane<float, true>(e, w, 1, E1);
        win_plane<float, true>(e, w, 2, E2);
        if constexpr (FROM_TH) {
            win_plane<float, false>(th, w, 0, T0);
            win_plane<float, true>(th, w, 1, T1);
            win_plane<float, true>(th, w, 2, T2);
        }
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a == 1) {   // slide the window: fine plane 2I+1 needs window planes 1..3
                win_plane<float, false>(e, w, 3, E0);
                if constexpr (FROM_TH) win_plane<float, false>(th, w, 3, T0);
            }
#pragma unroll
            for (int b = 1; b <= 2; ++b)
#pragma unroll
                for (int cc = 1; cc <= 2; ++cc) {
                    const Nb19<float> ne = a == 0 ? win_nb<float>(E0, E1, E2, b, cc) : win_nb<float>(E1, E2, E0, b, cc);
                    Cof<float> A;
                    if constexpr (FROM_TH) {
                        A = cofactors(a == 0 ? win_nb<float>(T0, T1, T2, b, cc) : win_nb<float>(T1, T2, T0, b, cc), ih2);
                    } else {
                        A = cof_at(cof, nf, cof_slot(Nf, 2 * I + a, 2 * J + b - 1, 2 * K + cc - 1));
                    }
                    acc += (f[w.at(1 + a, b, cc)] - fs) - jac_apply(A, ne, ih2);
                }
        }
        const float v = acc * 0.125f;
        fH[offs(Nc, I, J, K)] = v;
        sacc.add(v);
    }
    const double v = block_sum<kRowThreads>(sacc.get(), sh);
    if (ltid() == 0) partials[4 * blockIdx.x + 0] = v;
}

template <int NT>
__global__ void __launch_bounds__(NT)
k_lin_coarse(float *e, float *work, const float *f, const float *cof, int N, float ih2,
             int max_sweeps, double rtol)
{
    // relaxed in shared memory: e, the colour pass's scratch, f and the six
    // cofactor arrays are staged once, e is written back at the end
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    const size_t ncof = (size_t)N * N * N;
    __shared__ double sh[32];
    __shared__ double sval;
    const int n = N * N * N, half = N >> 1, npairs = N * N * half;
    float *es = reinterpret_cast<float *>(coarse_smem), *ws = es + n, *fs = ws + n, *cs = fs + n;
    for (int id = threadIdx.x; id < n; id += blockDim.x) {
        es[id] = e[id];
        fs[id] = f[id];
    }
    for (int id = threadIdx.x; id < 6 * n; id += blockDim.x) cs[id] = cof[id];
    __syncthreads();
    auto proj_rms = [&]() -> double {
        double sr = 0.0;
        for (int id = threadIdx.x; id < n; id += blockDim.x) {
            const int k = id % N, j = (id / N) % N, i = id / (N * N);
            const float r = fs[id] - jac_apply(cof_at(cs, ncof, cof_slot(N, i, j, k)), load19<float>(es, N, i, j, k), ih2);
            ws[id] = r;
            sr += (double)r;
        }
        double tot = block_sum<NT>(sr, sh);
        if (ltid() == 0) sval = tot / n;
        __syncthreads();
        const double m = sval;
        double s2 = 0.0;
        for (int id = threadIdx.x; id < n; id += blockDim.x) {
            const double d = (double)ws[id] - m;
            s2 += d * d;
        }
        tot = block_sum<NT>(s2, sh);
        if (ltid() == 0) sval = sqrt(tot / n);
        __syncthreads();
        const double v = sval;
        __syncthreads();
        return v;
    };
    const double r0 = proj_rms();
    double prev = r0;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        for (int colour = 0; colour < 2; ++colour) {
            const float *src = colour == 0 ? es : ws;
            float *dst = colour == 0 ? ws : es;
            for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
                const int m = pi % half, r = pi / half;
                const int j = r % N, i = r / N;
                const int par = (colour + i + j) & 1;
                const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                const Cof<float> a = cof_at(cs, ncof, cof_slot(N, i, j, ka));
                const Nb19<float> ev = load19<float>(src, N, i, j, ka);
                const float Je = jac_apply(a, ev, ih2);
                const float diag = -2.0f * (a.xx + a.yy + a.zz) * ih2;
                const float vnew = ev.c + (fs[offs(N, i, j, ka)] - Je) / diag;
                const float vcopy = src[offs(N, i, j, kb)];
                dst[offs(N, i, j, ka)] = vnew;
                dst[offs(N, i, j, kb)] = vcopy;
            }
            __syncthreads();
        }
        const double cur = proj_rms();
        if (cur <= rtol * r0) break;
        if (rtol > 0.0 && cur >= prev) break;   // no progress: round-off floor
        prev = cur;
    }
    for (int id = threadIdx.x; id < n; id += blockDim.x) e[id] = es[id];
}

template <typename T, int NT>
static cudaError_t coarse_attr()
{
    return cudaFuncSetAttribute(k_coarse_solve<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(3 * sizeof(T) * kMaxCoarseCells));
}
template <int NT>
static cudaError_t lin_coarse_attr()
{
    return cudaFuncSetAttribute(k_lin_coarse<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(9 * sizeof(float) * kMaxCoarseCells));
}
static cudaError_t coarse_attrs()
{
    cudaError_t e = coarse_attr<double, 64>();
    if (e == cudaSuccess) e = coarse_attr<double, 128>();
    if (e == cudaSuccess) e = coarse_attr<double, kCoarseThreads>();
    if (e == cudaSuccess) e = coarse_attr<float, 64>();
    if (e == cudaSuccess) e = coarse_attr<float, 128>();
    if (e == cudaSuccess) e = coarse_attr<float, kCoarseThreads>();
    if (e == cudaSuccess) e = lin_coarse_attr<64>();
    if (e == cudaSuccess) e = lin_coarse_attr<128>();
    if (e == cudaSuccess) e = lin_coarse_attr<kCoarseThreads>();
    return e;
}


// ======================================================================
// The V-cycle below 16^3 in one thread block.  On a hierarchy level whose
// grid has at most kMaxCoarseCells cells, the rest of the FAS V-cycle (and
// of the linear one) runs in one CTA on shared memory: every level's arrays
// are staged once, each step of the multi-kernel cycle is one block-wide
// loop separated by barriers, and only the top level's solution goes back
// to global memory.  The steps and their arithmetic are those of the grid
// kernels (k_rb_pass / k_lin_pass, k_restrict_residual, k_coarse_rhs with
// k_finalize_scale, k_form_rhs, k_prolong_add, the coarsest solves); the sums
// of the means and the minimum of the scale factor are taken in another
// order.  One launch replaces about a dozen per level, which on small grids
// are each a few microseconds of launch latency.
// ======================================================================
constexpr int kTailMaxLevels = 8;

template <typename T>
struct TailFas {
    int nl;                          // levels in the tail (>= 2)
    int N[kTailMaxLevels];
    T ih2[kTailMaxLevels], h2_6[kTailMaxLevels];
    T *t;                            // top level: theta (in/out) and g (global)
    const T *g;
    const double *cptr;              // c of the top level (coarser levels: 0)
    double *scal;                    // the handle's device scalars: the per-level
    int l0;                          // slots of levels l0 + 1 .. are written
    int nu1, nu2, rule, cmax;
    double floor_, crtol;
};

struct TailLin {
    int nl;
    int N[kTailMaxLevels];
    float ih2[kTailMaxLevels];
    float *e;                        // top level: e (in/out) and f (global)
    const float *f;
    const float *cof[kTailMaxLevels];  // every level's six colour-split cofactor arrays
    int nu1, nu2, cmax;
    double crtol;
};

// snapshot red-black sweeps of eq. update on a shared-memory grid (t -> w -> t)
template <typename T, int NT>
__device__ void tail_sweeps(T *t, T *w, const T *g, T c, int N, T ih2, T h2_6, int rule, int sweeps)
{
    const int half = N >> 1, npairs = N * N * half;
    for (int it = 0; it < sweeps; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            const T *src = colour == 0 ? t : w;
            T *dst = colour == 0 ? w : t;
            for (int pi = threadIdx.x; pi < npairs; pi += NT) {
                const int m = pi % half, r = pi / half;
                const int j = r % N, i = r / N;
                const int par = (colour + i + j) & 1;
                const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                const Nb19<T> nb = load19<T>(src, N, i, j, ka);
                T s, p, q;
                cubic_coeffs(nb, ih2, g[offs(N, i, j, ka)] + c, s, p, q);
                dst[offs(N, i, j, ka)] = point_update(nb.c, h2_6, s, p, q, rule);
                dst[offs(N, i, j, kb)] = src[offs(N, i, j, kb)];
            }
            __syncthreads();
        }
}

// fine += scale P(cn - co) on shared-memory grids (co may be null), the
// separable form of k_prolong_add
template <typename T, int NT>
__device__ void tail_prolong(const T *cn, const T *co, int Nc, T s, T *fine)
{
    const int Nf = 2 * Nc, ncc = Nc * Nc * Nc;
    const T w0 = T(0.75), w1 = T(0.25);
    for (int id = threadIdx.x; id < ncc; id += NT) {
        const int K = id % Nc, J = (id / Nc) % Nc, I = id / (Nc * Nc);
        const int Ip[3] = {I == 0 ? Nc - 1 : I - 1, I, I + 1 == Nc ? 0 : I + 1};
        const int Jp[3] = {J == 0 ? Nc - 1 : J - 1, J, J + 1 == Nc ? 0 : J + 1};
        const int Kp[3] = {K == 0 ? Nc - 1 : K - 1, K, K + 1 == Nc ? 0 : K + 1};
        T d[3][3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) {
                    const unsigned o = offs(Nc, Ip[a], Jp[b], Kp[c]);
                    d[a][b][c] = co ? cn[o] - co[o] : cn[o];
                }
        for (int ei = 0; ei < 2; ++ei) {
            T u[3][3];
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c) u[b][c] = w0 * d[1][b][c] + w1 * d[ei ? 2 : 0][b][c];
            for (int ej = 0; ej < 2; ++ej) {
                T v[3];
                for (int c = 0; c < 3; ++c) v[c] = w0 * u[1][c] + w1 * u[ej ? 2 : 0][c];
                const unsigned f = offs(Nf, 2 * I + ei, 2 * J + ej, 2 * K);
                fine[f] += s * (w0 * v[1] + w1 * v[0]);
                fine[f + 1] += s * (w0 * v[1] + w1 * v[2]);
            }
        }
    }
    __syncthreads();
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_fas_tail(TailFas<T> A)
{
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ double sh[32];
    __shared__ double sval;
    __shared__ double spscale[kTailMaxLevels];
    T *tl[kTailMaxLevels], *gl[kTailMaxLevels], *ol[kTailMaxLevels], *wl[kTailMaxLevels];
    {
        T *p = reinterpret_cast<T *>(tail_smem);
        for (int l = 0; l < A.nl; ++l) {
            const int n = A.N[l] * A.N[l] * A.N[l];
            tl[l] = p;
            gl[l] = p + n;
            ol[l] = p + 2 * n;
            wl[l] = p + 3 * n;
            p += 4 * n;
        }
    }
    const int n0 = A.N[0] * A.N[0] * A.N[0];
    for (int id = threadIdx.x; id < n0; id += NT) {
        tl[0][id] = A.t[id];
        gl[0][id] = A.g[id];
    }
    __syncthreads();
    const T c0 = (T)(*A.cptr);
    // down: pre-smoothing, residual + restriction, the coarse right side
    for (int l = 0; l + 1 < A.nl; ++l) {
        const T c = l == 0 ? c0 : T(0);
        const int N = A.N[l], Nc = A.N[l + 1], nc = Nc * Nc * Nc;
        tail_sweeps<T, NT>(tl[l], wl[l], gl[l], c, N, A.ih2[l], A.h2_6[l], A.rule, A.nu1);
        double sr = 0.0;
        for (int id = threadIdx.x; id < nc; id += NT) {
            const int K = id % Nc, J = (id / Nc) % Nc, I = id / (Nc * Nc);
            T at = T(0), ar = T(0);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int cc = 0; cc < 2; ++cc) {
                        const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + cc;
                        const Nb19<T> nb = load19<T>(tl[l], N, i, j, k);
                        at += nb.c;
                        ar += (gl[l][offs(N, i, j, k)] + c) - det_IH(nb, A.ih2[l]);
                    }
            const T vt = at * T(0.125), vr = ar * T(0.125);
            tl[l + 1][id] = vt;
            ol[l + 1][id] = vt;
            gl[l + 1][id] = vr;
            sr += (double)vr;
        }
        double tot = block_sum<NT>(sr, sh);
        if (ltid() == 0) {
            sval = tot / nc;
            A.scal[slot_rmean(A.l0 + l + 1)] = sval;
        }
        __syncthreads();
        const T m = (T)sval;
        const T fl = (T)A.floor_;
        T mn = T(INFINITY);
        for (int id = threadIdx.x; id < nc; id += NT) {
            const int K = id % Nc, J = (id / Nc) % Nc, I = id / (Nc * Nc);
            const T rr = gl[l + 1][id] - m;
            const T d = det_IH(load19<T>(tl[l + 1], Nc, I, J, K), A.ih2[l + 1]);
            gl[l + 1][id] = rr;
            wl[l + 1][id] = d;
            if (rr < T(0)) {
                const T cand = fl * (d > T(0) ? d : T(0)) / (-rr);
                mn = cand < mn ? cand : mn;
            }
        }
        const double v = block_min<NT>((double)mn, sh);
        if (ltid() == 0) {
            double sc = A.floor_ <= 0.0 ? 1.0 : fmin(1.0, v);
            if (sc < 1e-3) sc = 0.0;
            sval = sc;
            spscale[l + 1] = sc > 0.0 ? 1.0 / sc : 0.0;
            A.scal[slot_scale(A.l0 + l + 1)] = sc;
            A.scal[slot_pscale(A.l0 + l + 1)] = spscale[l + 1];
        }
        __syncthreads();
        const T sc = (T)sval;
        for (int id = threadIdx.x; id < nc; id += NT) gl[l + 1][id] = wl[l + 1][id] + sc * gl[l + 1][id];
        __syncthreads();
    }
    // bottom: the coarsest-grid solve (c = 0 below the top level)
    {
        const int lc = A.nl - 1, N = A.N[lc], half = N >> 1, npairs = N * N * half;
        T *ts = tl[lc], *ws = wl[lc];
        const T *gs = gl[lc];
        const double r0 = coarse_proj_rms<T, NT>(ts, ws, gs, T(0), N, A.ih2[lc], sh, &sval);
        double prev = r0;
        for (int sw = 0; sw < A.cmax; ++sw) {
            for (int colour = 0; colour < 2; ++colour) {
                const T *src = colour == 0 ? ts : ws;
                T *dst = colour == 0 ? ws : ts;
                for (int pi = threadIdx.x; pi < npairs; pi += NT) {
                    const int m = pi % half, r = pi / half;
                    const int j = r % N, i = r / N;
                    const int par = (colour + i + j) & 1;
                    const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                    const Nb19<T> nb = load19<T>(src, N, i, j, ka);
                    T s, p, q;
                    cubic_coeffs(nb, A.ih2[lc], gs[offs(N, i, j, ka)], s, p, q);
                    dst[offs(N, i, j, ka)] = point_update(nb.c, A.h2_6[lc], s, p, q, A.rule);
                    dst[offs(N, i, j, kb)] = src[offs(N, i, j, kb)];
                }
                __syncthreads();
            }
            const double cur = coarse_proj_rms<T, NT>(ts, ws, gs, T(0), N, A.ih2[lc], sh, &sval);
            if (cur <= A.crtol * r0) break;
            if (A.crtol > 0.0 && cur >= prev) break;
            prev = cur;
        }
    }
    // up: the corrections and post-smoothing
    for (int l = A.nl - 2; l >= 0; --l) {
        const double ps = spscale[l + 1];
        if (ps != 0.0) tail_prolong<T, NT>(tl[l + 1], ol[l + 1], A.N[l + 1], (T)ps, tl[l]);
        tail_sweeps<T, NT>(tl[l], wl[l], gl[l], l == 0 ? c0 : T(0), A.N[l], A.ih2[l], A.h2_6[l], A.rule,
                           A.nu2);
    }
    for (int id = threadIdx.x; id < n0; id += NT) A.t[id] = tl[0][id];
}

template <int NT>
__global__ void __launch_bounds__(NT) k_lin_tail(TailLin A)
{
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ double sh[32];
    __shared__ double sval;
    float *el[kTailMaxLevels], *fl[kTailMaxLevels], *cl[kTailMaxLevels], *wl[kTailMaxLevels];
    int nl_[kTailMaxLevels];
    {
        float *p = reinterpret_cast<float *>(tail_smem);
        for (int l = 0; l < A.nl; ++l) {
            const int n = A.N[l] * A.N[l] * A.N[l];
            nl_[l] = n;
            el[l] = p;
            fl[l] = p + n;
            wl[l] = p + 2 * n;
            cl[l] = p + 3 * n;
            p += 9 * n;
        }
    }
    for (int l = 0; l < A.nl; ++l)
        for (int id = threadIdx.x; id < 6 * nl_[l]; id += NT) cl[l][id] = A.cof[l][id];
    for (int id = threadIdx.x; id < nl_[0]; id += NT) {
        el[0][id] = A.e[id];
        fl[0][id] = A.f[id];
    }
    __syncthreads();
    auto sweeps = [&](int l, int count) {
        const int N = A.N[l], half = N >> 1, npairs = N * N * half;
        const size_t n = (size_t)nl_[l];
        for (int it = 0; it < count; ++it)
            for (int colour = 0; colour < 2; ++colour) {
                const float *src = colour == 0 ? el[l] : wl[l];
                float *dst = colour == 0 ? wl[l] : el[l];
                for (int pi = threadIdx.x; pi < npairs; pi += NT) {
                    const int m = pi % half, r = pi / half;
                    const int j = r % N, i = r / N;
                    const int par = (colour + i + j) & 1;
                    const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                    const Cof<float> a = cof_at(cl[l], n, cof_slot(N, i, j, ka));
                    const Nb19<float> ev = load19<float>(src, N, i, j, ka);
                    const float Je = jac_apply(a, ev, A.ih2[l]);
                    const float diag = -2.0f * (a.xx + a.yy + a.zz) * A.ih2[l];
                    dst[offs(N, i, j, ka)] = ev.c + (fl[l][offs(N, i, j, ka)] - Je) / diag;
                    dst[offs(N, i, j, kb)] = src[offs(N, i, j, kb)];
                }
                __syncthreads();
            }
    };
    for (int l = 0; l + 1 < A.nl; ++l) {
        const int N = A.N[l], Nc = A.N[l + 1], nc = Nc * Nc * Nc;
        const size_t nf = (size_t)nl_[l];
        sweeps(l, A.nu1);
        double sr = 0.0;
        for (int id = threadIdx.x; id < nc; id += NT) {
            const int K = id % Nc, J = (id / Nc) % Nc, I = id / (Nc * Nc);
            float acc = 0.0f;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int cc = 0; cc < 2; ++cc) {
                        const int i = 2 * I + a, j = 2 * J + b, k = 2 * K + cc;
                        const Cof<float> C = cof_at(cl[l], nf, cof_slot(N, i, j, k));
                        acc += fl[l][offs(N, i, j, k)] - jac_apply(C, load19<float>(el[l], N, i, j, k), A.ih2[l]);
                    }
            const float v = acc * 0.125f;
            fl[l + 1][id] = v;
            el[l + 1][id] = 0.0f;
            sr += (double)v;
        }
        const double tot = block_sum<NT>(sr, sh);
        if (ltid() == 0) sval = tot / nc;
        __syncthreads();
        const float m = (float)sval;
        for (int id = threadIdx.x; id < nc; id += NT) fl[l + 1][id] -= m;
        __syncthreads();
    }
    {   // the coarsest grid
        const int lc = A.nl - 1, N = A.N[lc], n = nl_[lc], half = N >> 1, npairs = N * N * half;
        const size_t ncof = (size_t)n;
        float *es = el[lc], *ws = wl[lc], *fs = fl[lc], *cs = cl[lc];
        auto proj_rms = [&]() -> double {
            double sr = 0.0;
            for (int id = threadIdx.x; id < n; id += NT) {
                const int k = id % N, j = (id / N) % N, i = id / (N * N);
                const float r = fs[id] - jac_apply(cof_at(cs, ncof, cof_slot(N, i, j, k)),
                                                   load19<float>(es, N, i, j, k), A.ih2[lc]);
                ws[id] = r;
                sr += (double)r;
            }
            double tt = block_sum<NT>(sr, sh);
            if (ltid() == 0) sval = tt / n;
            __syncthreads();
            const double mm = sval;
            double s2 = 0.0;
            for (int id = threadIdx.x; id < n; id += NT) {
                const double d = (double)ws[id] - mm;
                s2 += d * d;
            }
            tt = block_sum<NT>(s2, sh);
            if (ltid() == 0) sval = sqrt(tt / n);
            __syncthreads();
            const double vv = sval;
            __syncthreads();
            return vv;
        };
        const double r0 = proj_rms();
        double prev = r0;
        for (int sw = 0; sw < A.cmax; ++sw) {
            for (int colour = 0; colour < 2; ++colour) {
                const float *src = colour == 0 ? es : ws;
                float *dst = colour == 0 ? ws : es;
                for (int pi = threadIdx.x; pi < npairs; pi += NT) {
                    const int m = pi % half, r = pi / half;
                    const int j = r % N, i = r / N;
                    const int par = (colour + i + j) & 1;
                    const int ka = 2 * m + par, kb = 2 * m + 1 - par;
                    const Cof<float> a = cof_at(cs, ncof, cof_slot(N, i, j, ka));
                    const Nb19<float> ev = load19<float>(src, N, i, j, ka);
                    const float Je = jac_apply(a, ev, A.ih2[lc]);
                    const float diag = -2.0f * (a.xx + a.yy + a.zz) * A.ih2[lc];
                    dst[offs(N, i, j, ka)] = ev.c + (fs[offs(N, i, j, ka)] - Je) / diag;
                    dst[offs(N, i, j, kb)] = src[offs(N, i, j, kb)];
                }
                __syncthreads();
            }
            const double cur = proj_rms();
            if (cur <= A.crtol * r0) break;
            if (A.crtol > 0.0 && cur >= prev) break;
            prev = cur;
        }
    }
    for (int l = A.nl - 2; l >= 0; --l) {
        tail_prolong<float, NT>(el[l + 1], nullptr, A.N[l + 1], 1.0f, el[l]);
        sweeps(l, A.nu2);
    }
    for (int id = threadIdx.x; id < nl_[0]; id += NT) A.e[id] = el[0][id];
}

// shared memory of the tails: FAS 4 arrays per level, linear 9
template <typename T>
static size_t tail_fas_smem(const int *Nl, int nl)
{
    size_t c = 0;
    for (int l = 0; l < nl; ++l) c += 4 * (size_t)Nl[l] * Nl[l] * Nl[l];
    return c * sizeof(T);
}
static size_t tail_lin_smem(const int *Nl, int nl)
{
    size_t c = 0;
    for (int l = 0; l < nl; ++l) c += 9 * (size_t)Nl[l] * Nl[l] * Nl[l];
    return c * sizeof(float);
}
// the most any tail can need: a top level of kMaxCoarseCells cells, each
// level below an eighth of the one above
constexpr size_t kTailCells = kMaxCoarseCells + kMaxCoarseCells / 7 + 1;

static cudaError_t tail_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_fas_tail<float, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(4 * kTailCells * sizeof(float)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fas_tail<float, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * kTailCells * sizeof(float)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fas_tail<double, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * kTailCells * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fas_tail<double, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(4 * kTailCells * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lin_tail<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(9 * kTailCells * sizeof(float)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_lin_tail<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(9 * kTailCells * sizeof(float)));
    return e;
}

// ======================================================================
// drivers
// ======================================================================
namespace {

template <typename T>
struct Hier {
    T **t, **g, **told, **aux;
    T *work;
};

Hier<double> hier64(recon_handle *H)
{
    return {H->t64, H->g64, H->told64, H->aux64, H->work64};
}
Hier<float> hier32(recon_handle *H)
{
    return {H->t32, H->g32, H->told32, H->aux32, H->work32};
}

inline size_t ncell(int N) { return (size_t)N * N * N; }

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return e_;                                          \
    } while (0)

// The rest of the FAS V-cycle from level l (at most kMaxCoarseCells cells)
// in one thread block.
template <typename T>
cudaError_t fas_tail(recon_handle *H, const Hier<T> &Y, int l, const double *cptr)
{
    const recon_config &cf = H->cfg;
    TailFas<T> A{};
    A.nl = H->nlev - l;
    for (int q = 0; q < A.nl; ++q) {
        A.N[q] = H->Nl[l + q];
        const double h = H->hl[l + q];
        A.ih2[q] = (T)(1.0 / (h * h));
        A.h2_6[q] = (T)(h * h / 6.0);
    }
    A.t = Y.t[l];
    A.g = Y.g[l];
    A.cptr = cptr;
    A.scal = H->scal;
    A.l0 = l;
    A.nu1 = cf.nu1;
    A.nu2 = cf.nu2;
    A.rule = cf.rule;
    A.cmax = cf.coarse_max_sweeps;
    A.floor_ = cf.scale_floor;
    A.crtol = cf.coarse_rtol;
    if (!g_kernels_ready) {
        const cudaError_t e = prepare_kernels();
        if (e != cudaSuccess) return e;
    }
    const size_t smem = tail_fas_smem<T>(A.N, A.nl);
    note_launch();
    if (ncell(A.N[0]) / 2 <= 1024)
        k_fas_tail<T, 256><<<1, 256, smem, H->stream>>>(A);
    else
        k_fas_tail<T, 512><<<1, 512, smem, H->stream>>>(A);
    return cudaGetLastError();
}

// FAS V-cycle from level l (Sec. II.A.3).  gshift (nullable): a device
// scalar subtracted from level l's theta first (a deferred gauge shift;
// folded into the first sweep where it can be).
template <typename T>
cudaError_t vcycle(recon_handle *H, const Hier<T> &Y, int l, const double *cptr, const double *gshift = nullptr)
{
    cudaStream_t s = H->stream;
    const recon_config &cf = H->cfg;
    set_fused_chunk(cf.fused_chunk);
    const int N = H->Nl[l];
    const double h = H->hl[l];
    if (gshift && (l == H->nlev - 1 || ncell(N) <= (size_t)kMaxCoarseCells)) {
        note_launch();
        k_gauge_by<T><<<stride_blocks(ncell(N)), kThreads, 0, s>>>(Y.t[l], ncell(N), gshift);
        gshift = nullptr;
    }
    if (l < H->nlev - 1 && ncell(N) <= (size_t)kMaxCoarseCells && H->nlev - l <= kTailMaxLevels)
        return fas_tail<T>(H, Y, l, cptr);
    if (l == H->nlev - 1)
        return coarse_solve<T>(N, h, cf.rule, Y.t[l], Y.g[l], cptr, 0.0, cf.coarse_max_sweeps,
                               cf.coarse_rtol, Y.work, nullptr, s);
    CK(sweep<T>(N, h, cf.rule, Y.t[l], Y.g[l], cptr, 0.0, cf.nu1, Y.work, s, gshift));

    const int Nc = H->Nl[l + 1];
    const size_t nc = ncell(Nc);
    const unsigned nbr = row_grid(Nc, kMaxRedBlocks);
    note_launch();
    k_restrict_residual<T><<<nbr, row_block(), 0, s>>>(Y.t[l], Y.g[l], cptr, N, (T)(1.0 / (h * h)),
                                                    Y.t[l + 1], Y.told[l + 1], Y.g[l + 1],
                                                    H->partials);
    note_launch();
    k_finalize_mean<<<1, kReduceThreads, 0, s>>>(H->partials, nbr, (double)nc,
                                                 H->scal + slot_rmean(l + 1));
    const double hc = H->hl[l + 1];
    note_launch();
    k_coarse_rhs<T><<<nbr, row_block(), 0, s>>>(Y.t[l + 1], Y.g[l + 1], Y.aux[l + 1],
                                             H->scal + slot_rmean(l + 1), Nc,
                                             (T)(1.0 / (hc * hc)), cf.scale_floor, H->partials);
    note_launch();
    k_finalize_scale<<<1, kReduceThreads, 0, s>>>(H->partials, nbr, cf.scale_floor,
                                                  H->scal + slot_scale(l + 1),
                                                  H->scal + slot_pscale(l + 1));
    note_launch();
    k_form_rhs<T><<<stride_blocks(nc), kThreads, 0, s>>>(Y.g[l + 1], Y.aux[l + 1], nc,
                                                      H->scal + slot_scale(l + 1));
    CK(cudaGetLastError());
    CK(vcycle<T>(H, Y, l + 1, H->scal + S_ZERO));
    CK(prolong_add<T>(Nc, Y.t[l + 1], Y.told[l + 1], H->scal + slot_pscale(l + 1), 1.0,
                      Y.t[l], s));
    return sweep<T>(N, h, cf.rule, Y.t[l], Y.g[l], cptr, 0.0, cf.nu2, Y.work, s);
}

// residual norms of level l, then c -= mean r, rel, and theta -= mean theta
// (apply = false: the mean is left in scal[S_MEAN_T] for the next cycle to
// subtract)
template <typename T>
cudaError_t compat_gauge(recon_handle *H, const Hier<T> &Y, int l, bool apply = true)
{
    cudaStream_t s = H->stream;
    const int N = H->Nl[l];
    const size_t n = ncell(N);
    const double h = H->hl[l];
    const unsigned nbr = launch_residual_norms<T>(Y.t[l], Y.g[l], H->scal + S_C, N, (T)(1.0 / (h * h)),
                                                  H->partials, nullptr, nullptr, s);
    note_launch();
    k_finalize_cycle<<<1, kReduceThreads, 0, s>>>(H->partials, nbr, (double)n, H->scal);
    if (apply) {
        note_launch();
        k_gauge<T><<<stride_blocks(n), kThreads, 0, s>>>(Y.t[l], n, H->scal);
    }
    return cudaGetLastError();
}

// Nested iteration: restrict b to every level, solve the coarsest from 0,
// prolong up with one V-cycle per level; leaves the prolonged start on level 0.
template <typename T>
cudaError_t fmg_start(recon_handle *H, const Hier<T> &Y)
{
    cudaStream_t s = H->stream;
    const int lc = H->nlev - 1;
    for (int l = 1; l <= lc; ++l) CK(restrict_plain<T>(H->Nl[l - 1], Y.g[l - 1], Y.g[l], s));
    CK(cudaMemsetAsync(Y.t[lc], 0, sizeof(T) * ncell(H->Nl[lc]), s));
    CK(cudaMemsetAsync(H->scal + S_C, 0, sizeof(double), s));
    CK(vcycle<T>(H, Y, lc, H->scal + S_C));
    CK(compat_gauge<T>(H, Y, lc));
    for (int l = lc - 1; l >= 0; --l) {
        CK(cudaMemsetAsync(Y.t[l], 0, sizeof(T) * ncell(H->Nl[l]), s));
        CK(prolong_add<T>(H->Nl[l + 1], Y.t[l + 1], (const T *)nullptr, nullptr, 1.0, Y.t[l], s));
        if (l == 0) break;
        CK(vcycle<T>(H, Y, l, H->scal + S_C));
        CK(compat_gauge<T>(H, Y, l));
    }
    return cudaSuccess;
}

cudaError_t read_scalars(recon_handle *H)
{
    CK(cudaMemcpyAsync(H->hscal, H->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost,
                       H->stream));
    return cudaStreamSynchronize(H->stream);
}

recon_status fail_cuda(recon_handle *H, cudaError_t e, const char *where)
{
    H->err = std::string(where) + ": " + cudaGetErrorString(e);
    return RECON_E_CUDA;
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void hist_push(recon_stats *st, double v)
{
    if (st && st->n_history < RECON_HISTORY_MAX) st->history[st->n_history++] = v;
}

}  // namespace

recon_status check_domain(recon_handle *H, const double *b)
{
    const size_t n = ncell(H->N);
    const unsigned nbr = red_blocks(n);
    note_launch();
    k_b_stats<<<nbr, kThreads, 0, H->stream>>>(b, n, H->partials);
    note_launch();
    k_finalize_b<<<1, kReduceThreads, 0, H->stream>>>(H->partials, nbr, H->scal);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = read_scalars(H);
    if (e != cudaSuccess) return fail_cuda(H, e, "domain check");
    if (H->hscal[S_BBAD] > 0.0) {
        H->err = "b has non-finite entries";
        return RECON_E_DOMAIN;
    }
    if (!(H->hscal[S_BMIN] > 0.0)) {
        H->err = "b must be > 0 everywhere (min(b) = " + std::to_string(H->hscal[S_BMIN]) + ")";
        return RECON_E_DOMAIN;
    }
    return RECON_OK;
}

// ---------------------------------------------------------------- FP64
recon_status solve_f64(recon_handle *H, const double *b, double *phi, double tol,
                       int max_cycles, recon_stats *st)
{
    const double t0 = now_s();
    H->t64[0] = phi;
    H->g64[0] = const_cast<double *>(b);
    const Hier<double> Y = hier64(H);
    cudaError_t e = cudaSuccess;
    if (H->cfg.start == RECON_START_FMG) {
        e = fmg_start<double>(H, Y);
    } else {
        // resume: c (and the gauge) follow from the initial guess, as after a cycle
        e = cudaMemsetAsync(H->scal + S_C, 0, sizeof(double), H->stream);
        if (e == cudaSuccess) e = compat_gauge<double>(H, Y, 0);
    }
    if (e != cudaSuccess) return fail_cuda(H, e, "fmg start");

    const size_t n = ncell(H->N);
    recon_status status = RECON_E_NOCONV;
    double best = INFINITY;
    int cyc = 0;
    for (cyc = 1; cyc <= max_cycles; ++cyc) {
        e = vcycle<double>(H, Y, 0, H->scal + S_C);
        if (e == cudaSuccess) e = compat_gauge<double>(H, Y, 0);
        if (e == cudaSuccess) e = read_scalars(H);
        if (e != cudaSuccess) return fail_cuda(H, e, "V-cycle");
        const double rel = H->hscal[S_REL];
        hist_push(st, rel);
        (void)n;
        if (!std::isfinite(rel) || rel > 1e3 * best) {
            H->err = "residual diverged";
            status = RECON_E_DIVERGED;
            break;
        }
        best = rel < best ? rel : best;
        if (rel < tol) {
            status = RECON_OK;
            break;
        }
    }
    if (cyc > max_cycles) cyc = max_cycles;
    if (status == RECON_E_NOCONV) H->err = "max_cycles reached before the tolerance";
    if (st) {
        st->cycles = cyc;
        st->outer_iterations = 0;
        st->rel_residual = H->hscal[S_REL];
        st->compat_c = H->hscal[S_C];
        st->seconds = now_s() - t0;
    }
    return status;
}

// ---------------------------------------------------------------- MIXED
// (i) FP32 FAS (same cycle as above) until the FP32 residual reaches
//     mixed_switch_rtol, stagnates, or mixed_fas_max_cycles ran;
// (ii) defect correction: r64 = b + c - det(I + H phi) in FP64, then
//     mixed_linear_vcycles FP32 linear V-cycles on J(phi) e = r64 - mean,
//     phi += e, until ||r64 - mean|| / ||b - 1|| < tol.
namespace {

// Level l's f can carry its mean unsubtracted into a linear V-cycle when
// every kernel that reads it there folds the shift in: the register-blocked
// sweep (both directions of its ping-pong) and the restriction (a level above
// the single-block tail and the coarsest solve).
static bool lin_fold_ok(recon_handle *H, int l)
{
    const int N = H->Nl[l];
    return l < H->nlev - 1 && ncell(N) > (size_t)kMaxCoarseCells &&
           reg_sweep_ok(N, H->e32[l], H->work32, H->f32[l], H->t32[l]) &&
           reg_sweep_ok(N, H->work32, H->e32[l], H->f32[l], H->t32[l]);
}

// fshift (nullable, level l only): a device scalar subtracted from f on the
// fly by the register-blocked sweep and the restriction (lin_fold_ok)
cudaError_t lin_vcycle(recon_handle *H, int l, const double *fshift = nullptr)
{
    cudaStream_t s = H->stream;
    const recon_config &cf = H->cfg;
    set_fused_chunk(cf.fused_chunk);
    const int N = H->Nl[l];
    const double h = H->hl[l];
    const float ih2 = (float)(1.0 / (h * h));
    if (l < H->nlev - 1 && ncell(N) <= (size_t)kMaxCoarseCells && H->nlev - l <= kTailMaxLevels &&
        H->cof32[l]) {
        // the rest of the linear V-cycle in one thread block
        TailLin A{};
        A.nl = H->nlev - l;
        for (int q = 0; q < A.nl; ++q) {
            A.N[q] = H->Nl[l + q];
            const double hq = H->hl[l + q];
            A.ih2[q] = (float)(1.0 / (hq * hq));
            A.cof[q] = H->cof32[l + q];
        }
        A.e = H->e32[l];
        A.f = H->f32[l];
        A.nu1 = cf.nu1;
        A.nu2 = cf.nu2;
        A.cmax = cf.coarse_max_sweeps;
        A.crtol = cf.coarse_rtol;
        if (!g_kernels_ready) {
            const cudaError_t e = prepare_kernels();
            if (e != cudaSuccess) return e;
        }
        const size_t smem = tail_lin_smem(A.N, A.nl);
        note_launch();
        if (ncell(A.N[0]) / 2 <= 1024)
            k_lin_tail<256><<<1, 256, smem, s>>>(A);
        else
            k_lin_tail<512><<<1, 512, smem, s>>>(A);
        return cudaGetLastError();
    }
    if (l == H->nlev - 1) {
        note_launch();
        const size_t smem = 9 * sizeof(float) * ncell(N);
        const int pairs = (int)(ncell(N) / 2);
        if (pairs <= 64)
            k_lin_coarse<64><<<1, 64, smem, s>>>(H->e32[l], H->work32, H->f32[l], H->cof32[l], N, ih2,
                                                 cf.coarse_max_sweeps, cf.coarse_rtol);
        else if (pairs <= 128)
            k_lin_coarse<128><<<1, 128, smem, s>>>(H->e32[l], H->work32, H->f32[l], H->cof32[l], N, ih2,
                                                   cf.coarse_max_sweeps, cf.coarse_rtol);
        else
            k_lin_coarse<kCoarseThreads><<<1, kCoarseThreads, smem, s>>>(H->e32[l], H->work32, H->f32[l],
                                                                         H->cof32[l], N, ih2, cf.coarse_max_sweeps,
                                                                         cf.coarse_rtol);
        return cudaGetLastError();
    }
    CK(lin_sweep(N, h, H->e32[l], H->f32[l], H->cof32[l], H->t32[l], cf.nu1, H->work32, s, fshift));
    const int Nc = H->Nl[l + 1];
    const size_t nc = ncell(Nc);
    const unsigned nbr = row_grid(Nc, kMaxRedBlocks);
    note_launch();
    if (H->cof32[l])
        k_lin_restrict_residual<false><<<nbr, row_block(), 0, s>>>(H->e32[l], H->f32[l], H->cof32[l], nullptr,
                                                                    N, ih2, H->f32[l + 1], H->partials, fshift);
    else
        k_lin_restrict_residual<true><<<nbr, row_block(), 0, s>>>(H->e32[l], H->f32[l], nullptr, H->t32[l],
                                                                   N, ih2, H->f32[l + 1], H->partials, fshift);
    note_launch();
    k_finalize_mean<<<1, kReduceThreads, 0, s>>>(H->partials, nbr, (double)nc,
                                                 H->scal + slot_rmean(l + 1));
    // f - mean f on the coarse level: folded into its kernels where they can
    const bool fold = lin_fold_ok(H, l + 1);
    if (!fold) {
        note_launch();
        k_sub_scalar<<<stride_blocks(nc), kThreads, 0, s>>>(H->f32[l + 1], nc, H->scal + slot_rmean(l + 1));
    }
    CK(cudaMemsetAsync(H->e32[l + 1], 0, sizeof(float) * nc, s));
    CK(lin_vcycle(H, l + 1, fold ? H->scal + slot_rmean(l + 1) : nullptr));
    CK(prolong_add<float>(Nc, H->e32[l + 1], (const float *)nullptr, nullptr, 1.0, H->e32[l], s));
    return lin_sweep(N, h, H->e32[l], H->f32[l], H->cof32[l], H->t32[l], cf.nu2, H->work32, s, fshift);
}


}  // namespace

// ---- capture-safe phases of the mixed solve (no host synchronisation)
cudaError_t mixed_start(recon_handle *H, const double *b, const double *phi)
{
    cudaStream_t s = H->stream;
    const size_t n = ncell(H->N);
    const Hier<float> Y = hier32(H);
    note_launch();
    k_to_float<<<blocks_for(n), kThreads, 0, s>>>(b, H->g32[0], n);
    if (H->cfg.start == RECON_START_FMG) {
        CK(fmg_start<float>(H, Y));
    } else {
        note_launch();
        k_to_float<<<blocks_for(n), kThreads, 0, s>>>(phi, H->t32[0], n);
        CK(cudaMemsetAsync(H->scal + S_C, 0, sizeof(double), s));
        CK(compat_gauge<float>(H, Y, 0));
    }
    // no gauge shift pending for the first FP32 cycle
    return cudaMemsetAsync(H->scal + S_MEAN_T, 0, sizeof(double), s);
}

// One FP32 FAS cycle on the finest grid.  The gauge (theta -= mean theta)
// of the previous cycle is applied by this cycle's first sweep (the update
// depends only on differences of theta), and this cycle's is left pending:
// one pass over theta per cycle fewer.
cudaError_t mixed_fas_cycle(recon_handle *H)
{
    const Hier<float> Y = hier32(H);
    CK(vcycle<float>(H, Y, 0, H->scal + S_C, H->scal + S_MEAN_T));
    return compat_gauge<float>(H, Y, 0, false);
}

// from_phi: no FP32 cycle ran after a START_GUESS start, so the caller's FP64
// phi (not its FP32 copy) is the iterate to continue from.
cudaError_t mixed_switch(recon_handle *H, const double *b, double *phi, bool from_phi)
{
    cudaStream_t s = H->stream;
    const size_t n = ncell(H->N);
    if (!from_phi) {   // the last FP32 cycle's gauge, still pending
        note_launch();
        k_gauge_by<float><<<stride_blocks(n), kThreads, 0, s>>>(H->t32[0], n, H->scal + S_MEAN_T);
    }
    if (H->cfg.mixed_df_residual) {
        // phi as a double-float pair (theta32 + 0, or the split of phi); b split too
        note_launch(from_phi ? 2 : 1);
        k_split_df<<<blocks_for(n), kThreads, 0, s>>>(b, H->g32[0], H->blo32, n);
        if (from_phi) {
            k_split_df<<<blocks_for(n), kThreads, 0, s>>>(phi, H->t32[0], H->lo32, n);
            return cudaGetLastError();
        }
        return cudaMemsetAsync(H->lo32, 0, sizeof(float) * n, s);
    }
    if (from_phi) return cudaSuccess;
    note_launch();
    k_to_double<<<blocks_for(n), kThreads, 0, s>>>(H->t32[0], phi, n);
    return cudaGetLastError();
}

// r = b + c - det(I + H phi) (double-float or FP64), c -= mean r, rel
cudaError_t mixed_residual(recon_handle *H, const double *b, const double *phi)
{
    cudaStream_t s = H->stream;
    const size_t n = ncell(H->N);
    unsigned nbr = row_grid(H->N, kMaxRedBlocks);
    const double ih2 = 1.0 / (H->h * H->h);
    if (H->cfg.mixed_df_residual) {
        const df ih2df = df_from_double(ih2);
        int ex;
        const bool pow2 = ih2df.lo == 0.0f && std::frexp(ih2, &ex) == 0.5;
        note_launch();
        if (pow2)
            k_residual_df<true><<<nbr, row_block(), 0, s>>>(H->t32[0], H->lo32, H->g32[0], H->blo32,
                                                            H->scal + S_C, H->N, ih2df.hi, ih2df.lo,
                                                            H->f32[0], H->partials);
        else
            k_residual_df<false><<<nbr, row_block(), 0, s>>>(H->t32[0], H->lo32, H->g32[0], H->blo32,
                                                             H->scal + S_C, H->N, ih2df.hi, ih2df.lo,
                                                             H->f32[0], H->partials);
    } else {
        nbr = launch_residual_norms<double>(phi, b, H->scal + S_C, H->N, ih2, H->partials, H->f32[0],
                                            H->t32[0], s);
    }
    note_launch();
    k_finalize_cycle<<<1, kReduceThreads, 0, s>>>(H->partials, nbr, (double)n, H->scal);
    return cudaGetLastError();
}

// J(phi) e = r - mean r by FP32 linear multigrid, then phi += e
cudaError_t mixed_correct(recon_handle *H, double *phi)
{
    cudaStream_t s = H->stream;
    const size_t n = ncell(H->N);
    // r - mean r: subtracted on the fly by the finest level's kernels where
    // they can, else in a pass of its own
    const bool fold = lin_fold_ok(H, 0);
    if (!fold) {
        note_launch();
        k_sub_scalar<<<stride_blocks(n), kThreads, 0, s>>>(H->f32[0], n, H->scal + S_MEAN_R);
    }
    for (int l = 1; l < H->nlev; ++l) CK(restrict_plain<float>(H->Nl[l - 1], H->t32[l - 1], H->t32[l], s));
    for (int l = 0; l < H->nlev; ++l) {
        if (H->Nl[l] >= kFusedMinN) continue;   // formed from theta32 in the kernels
        note_launch();
        k_cof6f<<<row_grid(H->Nl[l]), row_block(), 0, s>>>(H->t32[l], H->Nl[l],
                                                           (float)(1.0 / (H->hl[l] * H->hl[l])), H->cof32[l]);
    }
    CK(cudaMemsetAsync(H->e32[0], 0, sizeof(float) * n, s));
    for (int v = 0; v < H->cfg.mixed_linear_vcycles; ++v)
        CK(lin_vcycle(H, 0, fold ? H->scal + S_MEAN_R : nullptr));
    note_launch();
    if (H->cfg.mixed_df_residual)
        k_update_df<<<blocks_for(n), kThreads, 0, s>>>(H->t32[0], H->lo32, H->e32[0], n);
    else
        k_update_theta<<<blocks_for(n), kThreads, 0, s>>>(phi, H->e32[0], n, H->scal);
    return cudaGetLastError();
}

// phi out: FP64, mean-free
cudaError_t mixed_finish(recon_handle *H, double *phi, bool converged)
{
    cudaStream_t s = H->stream;
    const size_t n = ncell(H->N);
    if (H->cfg.mixed_df_residual) {
        const unsigned nb2 = red_blocks(n);
        note_launch(3);
        k_df_sum<<<nb2, kThreads, 0, s>>>(H->t32[0], H->lo32, n, H->partials);
        k_finalize_mean<<<1, kReduceThreads, 0, s>>>(H->partials, nb2, (double)n, H->scal + S_MEAN_T);
        k_df_to_double_gauged<<<stride_blocks(n), kThreads, 0, s>>>(H->t32[0], H->lo32, phi, n,
                                                                   H->scal + S_MEAN_T);
    } else if (converged) {
        note_launch();
        k_gauge<double><<<stride_blocks(n), kThreads, 0, s>>>(phi, n, H->scal);
    }
    return cudaGetLastError();
}

// (i) FP32 FAS until the FP32 residual reaches mixed_switch_rtol, stalls, or
// mixed_fas_max_cycles ran; (ii) defect correction: the fine-grid residual in
// double-float (or FP64), mixed_linear_vcycles FP32 linear V-cycles on
// J(phi) e = r - mean r, phi += e, until ||r - mean r|| / ||b - 1|| < tol.
recon_status solve_mixed(recon_handle *H, const double *b, double *phi, double tol,
                         int max_cycles, recon_stats *st)
{
    const double t0 = now_s();
    const recon_config &cf = H->cfg;
    cudaError_t e = mixed_start(H, b, phi);
    if (e != cudaSuccess) return fail_cuda(H, e, "mixed start");
    int fas = 0;
    double prev = INFINITY;
    for (fas = 1; fas <= cf.mixed_fas_max_cycles; ++fas) {
        e = mixed_fas_cycle(H);
        if (e == cudaSuccess) e = read_scalars(H);
        if (e != cudaSuccess) return fail_cuda(H, e, "FP32 V-cycle");
        const double rel = H->hscal[S_REL];
        hist_push(st, rel);
        if (!std::isfinite(rel)) {
            H->err = "FP32 residual diverged";
            return RECON_E_DIVERGED;
        }
        if (rel < cf.mixed_switch_rtol || rel > 0.7 * prev) break;
        prev = rel;
    }
    if (fas > cf.mixed_fas_max_cycles) fas = cf.mixed_fas_max_cycles;
    const bool from_phi = cf.start == RECON_START_GUESS && fas == 0;
    if ((e = mixed_switch(H, b, phi, from_phi)) != cudaSuccess) return fail_cuda(H, e, "mixed switch");

    recon_status status = RECON_E_NOCONV;
    double best = INFINITY;
    int o = 0;
    for (o = 1; o <= max_cycles; ++o) {
        e = mixed_residual(H, b, phi);
        if (e == cudaSuccess) e = read_scalars(H);
        if (e != cudaSuccess) return fail_cuda(H, e, "fine-grid residual");
        const double rel = H->hscal[S_REL];
        hist_push(st, rel);
        if (!std::isfinite(rel) || rel > 1e3 * best) {
            H->err = "residual diverged";
            status = RECON_E_DIVERGED;
            break;
        }
        best = rel < best ? rel : best;
        if (rel < tol) {
            status = RECON_OK;
            break;
        }
        if ((e = mixed_correct(H, phi)) != cudaSuccess) return fail_cuda(H, e, "linear correction");
    }
    if (o > max_cycles) o = max_cycles;
    if (status == RECON_E_NOCONV) H->err = "max_cycles reached before the tolerance";
    e = mixed_finish(H, phi, status == RECON_OK);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);
    if (e != cudaSuccess) return fail_cuda(H, e, "mixed solve");
    if (st) {
        st->cycles = fas;
        st->outer_iterations = o;
        st->rel_residual = H->hscal[S_REL];
        st->compat_c = H->hscal[S_C];
        st->seconds = now_s() - t0;
    }
    return status;
}

}  // namespace recon
