// Stage 0 (pack) and stage 1 (compatibility graph, Eq. 1).
//
// pack:   [N][3] x, y (float32, any 4-byte alignment) -> points in two device
//         layouts with zero padding: structure of arrays pts[6][n_pad] and
//         32-byte records pts8[n_pad] = (x0,x1,x2,y0 | y1,y2,w,0), w = 1 when
//         a coordinate lies beyond 2^24 in magnitude (else 0); flags NaN/Inf;
//         clears the per-call accumulators.
// compat: G_ij = [ | ||x_i - x_j|| - ||y_i - y_j|| | <= tau ], i != j, G_ii = 0
//         (Eq. 1; zero diagonal because App. B equates G^_ij with the number
//         of triangles on edge (i,j)).  Written as a row bitset (operand of the
//         clique search), as FP8 E4M3 0/1 bytes (operand of the SC^2 GEMM) and
//         as node degrees.
//
// Work decomposition: 128 x 128 tiles (I, J) with I <= J only.  A block
// computes its tile once and writes it twice (rows i of tile (I, J) and,
// transposed, rows j of tile (J, I)): G is symmetric bit for bit because
// x_j - x_i = -(x_i - x_j) exactly in IEEE arithmetic.  The 128 row points
// of a tile are staged in shared memory with one 1-D TMA bulk copy; every
// thread keeps 4 column points in registers.
//
// Exactness: the decision is taken in FP32 without square roots and retaken
// in FP64 with the fixed operation order ((dx*dx + dy*dy) + dz*dz) and
// correctly rounded sqrt for the few pairs inside a guard band.  With the
// squared distances s_X, s_Y, D = s_X - s_Y, Q = s_X + s_Y and
// delta = |d_X - d_Y|: (d_X + d_Y)^2 = 2Q - delta^2 (parallelogram law), so
// D^2 = f(delta^2) with f(x) = x (2Q - x), increasing on [0, Q] and
// delta^2 <= Q.  Hence, for Q >= tau^2, delta <= tau iff
// D^2 <= f(tau^2) = 2 tau^2 Q - tau^4; for Q < tau^2 the pair is compatible
// (delta^2 <= Q) and D^2 <= Q^2 < tau^4.  One expression covers both cases:
//     Phi = D^2 - 2 tau^2 max(Q, tau^2) + tau^4,    G_ij = [Phi <= 0].
// FP32 error (u = 2^-24; coordinates |c| <= 2^24, 2^-20 <= tau <= 2^20, so
// nothing overflows and every quantity the bound scales by is normal): the
// squared distances carry relative error <= 5.01u; with Qc = max(Q, tau^2)
// and a = |D~|, |D~ - D| <= 5.02u Qc + 1.01u a, |Qc~ - Qc| <= 6.05u Qc, and
// |Phi~ - Phi| <= 12.22u a Qc + 25.3u^2 Qc^2 + 18.4u tau^2 Qc + u |Phi~|.
// The band g = Qc~ (16u a + 32u^2 Qc~ + 24u tau^2) exceeds that bound by
// more than a quarter after its own rounding, so every pair with |Phi~| > g
// has the sign of the exact Phi, which also decides like the FP64
// evaluation (FP64 moves delta by ~1e-16 (d_X + d_Y), far inside the band).
// In delta the band is about 4u (d_X + d_Y) wide; on the indoor N = 5000
// workload it holds a handful of the 12.5 M pairs.  Tiles with a coordinate
// beyond 2^24 (flagged by pack) and tau outside [2^-20, 2^20] send every
// pair to FP64.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kT = 128;          // tile edge
constexpr int kThreads = 128;    // 4 warps x 32 rows; each lane 4 columns
constexpr int kR = 32;           // rows per warp
constexpr float kRangeMax = 16777216.0f;   // 2^24: larger coordinates take the FP64 decision
constexpr float kTauMin = 9.5367431640625e-07f, kTauMax = 1048576.0f;   // 2^-20, 2^20

// One block per 256 points of one problem; src/dst are the (concatenated)
// inputs, the problem's matches start at v.in_off.
__global__ void __launch_bounds__(256) pack_kernel(ManyViews vs, const float* __restrict__ src_cat,
                                                   const float* __restrict__ dst_cat)
{
    pdl_release();   // the compatibility blocks may take their places (they wait for this grid)
    int lb;
    const ProbView v = vs.get(ST_PACK, blockIdx.x, lb);
    const float* src = src_cat + 3 * v.in_off;
    const float* dst = dst_cat + 3 * v.in_off;
    bool bad = false, wide = false;
    const int k = lb * 256 + threadIdx.x;
    if (k < v.n_pad) {
        float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (k < v.n) {
            a[0] = src[3 * k + 0]; a[1] = src[3 * k + 1]; a[2] = src[3 * k + 2];
            a[3] = dst[3 * k + 0]; a[4] = dst[3 * k + 1]; a[5] = dst[3 * k + 2];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                bad |= !isfinite(a[c]);
                wide |= !(fabsf(a[c]) <= kRangeMax);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) v.pts[(size_t)c * v.n_pad + k] = a[c];
        float4* p8 = reinterpret_cast<float4*>(v.pts8 + (size_t)k * 8);
        p8[0] = make_float4(a[0], a[1], a[2], a[3]);
        p8[1] = make_float4(a[4], a[5], wide ? 1.f : 0.f, 0.f);
        v.rowscore[k] = 0;
        v.deg[k] = 0;
        if (v.rowmax) v.rowmax[k] = 0;
        v.hist[k] = 0;
    }
    if (k == 0) v.hist[v.n_pad] = 0;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&v.ctl->err, TR_ERR_NONFINITE);
}

// Constants of the FP32 decision, each in both halves where it enters a
// packed instruction: c1 = -2 tau^2, c0 = tau^4, cq = 32u^2, ct = 24u tau^2;
// t2 = tau^2; ca = 16u, or +inf when every pair must take the FP64 decision
// (the band then becomes +inf or NaN, and both read as "inside").
struct Decide {
    f2 c1, c0, cq, ct;
    float t2, ca;
};

__device__ __forceinline__ Decide decide_consts(float tau, bool all64)
{
    // FP32 only (the FP64 pipe is narrow): t2 = fl(tau^2); e = tau^2 - t2
    // exactly (fma); tau^4 = t2^2 + 2 t2 e + e^2, rounded once up to e^2
    Decide k;
    k.t2 = tau * tau;
    const float e = fmaf(tau, tau, -k.t2);
    const float c1 = -2.0f * k.t2;
    const float c0 = fmaf(k.t2, k.t2, 2.0f * k.t2 * e);
    const float cq = 1.1368683772161603e-13f;           // 32 u^2 = 2^-43
    const float ct = 1.430511474609375e-06f * k.t2;     // 24u tau^2 (24u = 1.5 * 2^-20, exact)
    k.c1 = pk(c1, c1);
    k.c0 = pk(c0, c0);
    k.cq = pk(cq, cq);
    k.ct = pk(ct, ct);
    k.ca = all64 ? __int_as_float(0x7f800000) : 9.5367431640625e-07f;   // 16u = 2^-20
    return k;
}

__device__ __noinline__ bool compat_fp64(float xi0, float xi1, float xi2, float yi0, float yi1, float yi2,
                                         float xj0, float xj1, float xj2, float yj0, float yj1, float yj2,
                                         float tau)
{
    const double dx = __dsub_rn((double)xi0, (double)xj0);
    const double dy = __dsub_rn((double)xi1, (double)xj1);
    const double dz = __dsub_rn((double)xi2, (double)xj2);
    const double ex = __dsub_rn((double)yi0, (double)yj0);
    const double ey = __dsub_rn((double)yi1, (double)yj1);
    const double ez = __dsub_rn((double)yi2, (double)yj2);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    double t = __dmul_rn(ex, ex);
    t = __dadd_rn(t, __dmul_rn(ey, ey));
    t = __dadd_rn(t, __dmul_rn(ez, ez));
    return fabs(__dsub_rn(__dsqrt_rn(s), __dsqrt_rn(t))) <= (double)tau;
}

// FP32 decision for two columns at once (Phi <= 0, see the file header); n0/n1
// are set when |Phi| is inside the guard band (or the arithmetic produced
// NaN/Inf) and the FP64 evaluation must decide.  s = (ax^2 + ay^2) + az^2 by
// mul then two fma; everything that can is a packed pair (add/sub/mul/fma
// .rn.f32x2 round each half exactly like the scalar instructions).
__device__ __forceinline__ void compat_fast2(const f2 (&XI)[6], const f2 (&XJ)[6], const Decide& k, bool& a0,
                                             bool& a1, bool& n0, bool& n1)
{
    const f2 ax = sub2(XI[0], XJ[0]), ay = sub2(XI[1], XJ[1]), az = sub2(XI[2], XJ[2]);
    const f2 bx = sub2(XI[3], XJ[3]), by = sub2(XI[4], XJ[4]), bz = sub2(XI[5], XJ[5]);
    const f2 sX = fma2(az, az, fma2(ay, ay, mul2(ax, ax)));
    const f2 sY = fma2(bz, bz, fma2(by, by, mul2(bx, bx)));
    const f2 D = sub2(sX, sY);
    float Q0, Q1;
    upk(add2(sX, sY), Q0, Q1);
    const f2 Qc = pk(fmaxf(Q0, k.t2), fmaxf(Q1, k.t2));
    float P0, P1, D0, D1, w0, w1, g0, g1;
    upk(fma2(D, D, fma2(Qc, k.c1, k.c0)), P0, P1);        // Phi
    upk(D, D0, D1);
    upk(fma2(Qc, k.cq, k.ct), w0, w1);                     // 32u^2 Qc + 24u tau^2
    w0 = fmaf(fabsf(D0), k.ca, w0);
    w1 = fmaf(fabsf(D1), k.ca, w1);
    upk(mul2(Qc, pk(w0, w1)), g0, g1);                     // the band
    n0 = !(fabsf(P0) > g0);
    n1 = !(fabsf(P1) > g1);
    a0 = P0 <= 0.f;
    a1 = P1 <= 0.f;
}

// 4 bits -> 4 bytes of FP8 E4M3 (0x38 = 1.0 for a set bit, 0x00 otherwise)
__device__ __forceinline__ uint32_t nibble_to_fp8(uint32_t nib)
{
    return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
}

__device__ __forceinline__ uint4 bits16_to_fp8(uint32_t b16)
{
    return make_uint4(nibble_to_fp8(b16 & 0xF), nibble_to_fp8((b16 >> 4) & 0xF), nibble_to_fp8((b16 >> 8) & 0xF),
                      nibble_to_fp8((b16 >> 12) & 0xF));
}

// kAuto: the SC^2 path is chosen on the device (one problem): no FP8 matrix,
// and the degree sum 2 |E| is added up in the control block
template <bool kAuto>
__global__ void __launch_bounds__(kThreads, 8) compat_kernel(ManyViews vs)
{
    // the block's problem from the launch's descriptors (static for the launch):
    // read while the predecessor still runs
    int t;
    const ProbView v = vs.get(ST_COMPAT, blockIdx.x, t);
    pdl_wait();
    pdl_release();
    __shared__ __align__(128) float4 srow[kT][2];        // row points as copied (x0,x1,x2,y0 | y1,y2,w,0)
    __shared__ __align__(16) ulonglong2 srow2[kT][3];    // the same six values, each in both halves of a pair
    __shared__ __align__(16) uint4 srbits[kT];           // row r's four bitset words (ballots of its warp)
    __shared__ __align__(16) uint32_t colpart[kT][4];    // column c: the 32-row masks of the 4 warps
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_wide;

    // triangular tile index -> (I, J), I <= J
    int J = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (J * (J + 1) / 2 > t) --J;
    while ((J + 1) * (J + 2) / 2 <= t) ++J;
    const int I = t - J * (J + 1) / 2;
    const int i0 = I * kT, j0 = J * kT;
    const bool diag = (I == J);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_wide = 0;
    }
    __syncthreads();
    // failure injection (tests only): the row copy is never issued, so the
    // wait below can only expire (after the short kStallWaitNs)
    const bool stall = (v.dbg & TR_DBG_STALL_COMPAT) != 0u;
    if (threadIdx.x == 0 && !stall) {
        mbar_arrive_expect_tx(&bar, kT * 32);
        bulk_g2s(&srow[0][0], v.pts8 + (size_t)i0 * 8, kT * 32, &bar);
    }
    // this thread's 4 column points j = j0 + lane + 32 q, as packed pairs (q 0,1) and (q 2,3)
    f2 XJ[2][6];
    bool jok[4];
    bool wide = false;
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const int j = j0 + lane + 64 * pr;
        const float4* p = reinterpret_cast<const float4*>(v.pts8 + (size_t)j * 8);
        const float4* p2 = reinterpret_cast<const float4*>(v.pts8 + (size_t)(j + 32) * 8);
        const float4 a = p[0], b = p[1], a2 = p2[0], b2 = p2[1];
        XJ[pr][0] = pk(a.x, a2.x); XJ[pr][1] = pk(a.y, a2.y); XJ[pr][2] = pk(a.z, a2.z);
        XJ[pr][3] = pk(a.w, a2.w); XJ[pr][4] = pk(b.x, b2.x); XJ[pr][5] = pk(b.y, b2.y);
        wide |= (b.z != 0.f) | (b2.z != 0.f);
        jok[2 * pr] = j < v.n;
        jok[2 * pr + 1] = j + 32 < v.n;
    }
    // row points: thread t duplicates row t into pairs
    const bool ok = mbar_wait(&bar, 0, stall ? kStallWaitNs : kWaitNs);
    if (ok) {
        const int r = threadIdx.x;
        const float4 p = srow[r][0], p2 = srow[r][1];
        srow2[r][0] = make_ulonglong2(pk(p.x, p.x).v, pk(p.y, p.y).v);
        srow2[r][1] = make_ulonglong2(pk(p.z, p.z).v, pk(p.w, p.w).v);
        srow2[r][2] = make_ulonglong2(pk(p2.x, p2.x).v, pk(p2.y, p2.y).v);
        wide |= p2.z != 0.f;
    }
    if (wide) s_wide = 1;
    // a wait that gave up (in any thread) leaves the tile empty: the later
    // stages then see no edge here, and the registration reports the timeout
    const bool got = __syncthreads_and(ok) != 0;
    if (!got && threadIdx.x == 0) atomicOr(&v.ctl->err, TR_ERR_TIMEOUT);
    const float tau = v.tau;
    const Decide K = decide_consts(tau, s_wide != 0 || !(tau >= kTauMin && tau <= kTauMax));
    // bit r of cmask[q]: G(i0 + 32 warp + r, j_q), before the validity masks;
    // bit r of nflag: row r has a pair inside the guard band
    uint32_t cmask[4] = {0u, 0u, 0u, 0u};
    uint32_t nflag = 0u;
    if (got) {
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int rr = warp * kR + r;
            const ulonglong2 p0 = srow2[rr][0], p1 = srow2[rr][1], p2 = srow2[rr][2];
            const f2 XI[6] = {{p0.x}, {p0.y}, {p1.x}, {p1.y}, {p2.x}, {p2.y}};
            bool a[4], nq[4];
            compat_fast2(XI, XJ[0], K, a[0], a[1], nq[0], nq[1]);
            compat_fast2(XI, XJ[1], K, a[2], a[3], nq[2], nq[3]);
            if (nq[0] | nq[1] | nq[2] | nq[3]) nflag |= 1u << r;
            uint32_t word[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (a[q]) cmask[q] |= 1u << r;
                word[q] = __ballot_sync(0xffffffffu, a[q]);
            }
            if (lane == 0) srbits[rr] = make_uint4(word[0], word[1], word[2], word[3]);
        }
        __syncwarp();
        // rare: the pairs inside the band are decided again in FP64 with the
        // reference operation order, and their bits patched
        if (__any_sync(0xffffffffu, nflag != 0u)) {
#pragma unroll 1
            for (uint32_t f = nflag; f != 0u; f &= f - 1u) {
                const int r = __ffs(f) - 1;
                const int rr = warp * kR + r;
                const ulonglong2 p0 = srow2[rr][0], p1 = srow2[rr][1], p2 = srow2[rr][2];
                const f2 XI[6] = {{p0.x}, {p0.y}, {p1.x}, {p1.y}, {p2.x}, {p2.y}};
                bool a[4], nq[4];
                compat_fast2(XI, XJ[0], K, a[0], a[1], nq[0], nq[1]);
                compat_fast2(XI, XJ[1], K, a[2], a[3], nq[2], nq[3]);
                const float4 ra = srow[rr][0], rb = srow[rr][1];
                uint32_t* wr = reinterpret_cast<uint32_t*>(&srbits[rr]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!nq[q]) continue;
                    // the column point again from memory: keeping it in registers costs more than this rare load
                    const float4* pj = reinterpret_cast<const float4*>(v.pts8 + (size_t)(j0 + lane + 32 * q) * 8);
                    const float4 ca = pj[0], cb = pj[1];
                    const bool e = compat_fp64(ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, ca.x, ca.y, ca.z, ca.w, cb.x, cb.y,
                                               tau);
                    if (e) {
                        cmask[q] |= 1u << r;
                        atomicOr(wr + q, 1u << lane);
                    } else {
                        cmask[q] &= ~(1u << r);
                        atomicAnd(wr + q, ~(1u << lane));
                    }
                }
            }
        }
    }
    // validity: columns j < n, rows i < n, no diagonal entry
    uint32_t colv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) colv[q] = __ballot_sync(0xffffffffu, jok[q]);
    const int nrow = min(max(v.n - (i0 + warp * kR), 0), kR);
    const uint32_t rowv = nrow >= 32 ? 0xFFFFFFFFu : (1u << nrow) - 1u;
#pragma unroll
    for (int q = 0; q < 4; ++q) cmask[q] &= jok[q] ? rowv : 0u;
    __syncwarp();
    // direct rows i0 + 32 warp + r (r = 0..31): lane r stores row r's bitset words (16 B)
    uint32_t wrow_bits[4] = {0u, 0u, 0u, 0u};
    {
        const int i = i0 + warp * kR + lane;
        if (got && i < v.n) {
            const uint4 w = srbits[warp * kR + lane];
            wrow_bits[0] = w.x & colv[0]; wrow_bits[1] = w.y & colv[1];
            wrow_bits[2] = w.z & colv[2]; wrow_bits[3] = w.w & colv[3];
            if (diag) {   // column i - j0 = 32 warp + lane of this row: word warp, bit lane
                const uint32_t off = ~(1u << lane);
                const int qc = warp;
                wrow_bits[0] &= qc == 0 ? off : 0xFFFFFFFFu;
                wrow_bits[1] &= qc == 1 ? off : 0xFFFFFFFFu;
                wrow_bits[2] &= qc == 2 ? off : 0xFFFFFFFFu;
                wrow_bits[3] &= qc == 3 ? off : 0xFFFFFFFFu;
            }
        }
        *reinterpret_cast<uint4*>(v.bits + (size_t)i * v.ldb + (j0 >> 5)) =
            make_uint4(wrow_bits[0], wrow_bits[1], wrow_bits[2], wrow_bits[3]);
        const int d = __popc(wrow_bits[0]) + __popc(wrow_bits[1]) + __popc(wrow_bits[2]) + __popc(wrow_bits[3]);
        if (d) atomicAdd(&v.deg[i], d);
        if (kAuto && diag) {   // the diagonal tile's rows (off the diagonal: twice the columns, below)
            const unsigned ds = __reduce_add_sync(0xFFFFFFFFu, static_cast<unsigned>(d));
            if (lane == 0 && ds) atomicAdd(&v.ctl->deg_sum, ds);
        }
    }
    // FP8 rows (only for the tensor-core SC^2), 128 contiguous bytes per row:
    // pass k writes rows 4k .. 4k + 3 of the warp's 32, lane l the 16-byte
    // segment l % 8 of row 4k + l / 8
    const bool fp8 = !kAuto && v.a8 != nullptr;
#pragma unroll
    for (int k = 0; k < kR / 4 && fp8; ++k) {
        const int r = 4 * k + (lane >> 3);
        const int seg = lane & 7;
        const uint32_t w0 = __shfl_sync(0xffffffffu, wrow_bits[0], r);
        const uint32_t w1 = __shfl_sync(0xffffffffu, wrow_bits[1], r);
        const uint32_t w2 = __shfl_sync(0xffffffffu, wrow_bits[2], r);
        const uint32_t w3 = __shfl_sync(0xffffffffu, wrow_bits[3], r);
        const uint32_t w = (seg >> 1) == 0 ? w0 : (seg >> 1) == 1 ? w1 : (seg >> 1) == 2 ? w2 : w3;
        const int i = i0 + warp * kR + r;
        *reinterpret_cast<uint4*>(v.a8 + (size_t)i * v.n_pad + j0 + seg * 16) =
            bits16_to_fp8((w >> ((seg & 1) * 16)) & 0xFFFFu);
    }
    if (diag) return;
    // mirrored tile: row j gets bits of rows i0 .. i0+127; column c's word w
    // holds rows 32w .. 32w+31
#pragma unroll
    for (int q = 0; q < 4; ++q) colpart[lane + 32 * q][warp] = cmask[q];
    __syncthreads();
    {
        const int c = threadIdx.x;
        const uint4 cw = *reinterpret_cast<const uint4*>(colpart[c]);
        const int j = j0 + c;
        *reinterpret_cast<uint4*>(v.bits + (size_t)j * v.ldb + (i0 >> 5)) = cw;
        const int d = __popc(cw.x) + __popc(cw.y) + __popc(cw.z) + __popc(cw.w);
        if (d) atomicAdd(&v.deg[j], d);
        if (kAuto) {
            const unsigned ds = __reduce_add_sync(0xffffffffu, static_cast<unsigned>(d));
            if (lane == 0 && ds) atomicAdd(&v.ctl->deg_sum, 2u * ds);
        }
    }
    // FP8 rows: pass k writes rows j0 + 16k .. +15, eight threads per 128-byte row
#pragma unroll
    for (int k = 0; k < 8 && fp8; ++k) {
        const int c = 16 * k + (threadIdx.x >> 3);
        const int seg = threadIdx.x & 7;
        const uint32_t w = reinterpret_cast<const uint32_t*>(colpart[c])[seg >> 1];
        *reinterpret_cast<uint4*>(v.a8 + (size_t)(j0 + c) * v.n_pad + i0 + seg * 16) =
            bits16_to_fp8((w >> ((seg & 1) * 16)) & 0xFFFFu);
    }
}

}  // namespace

const void* pack_kernel_func() { return reinterpret_cast<const void*>(&pack_kernel); }

void launch_pack(const Batch& b, int total, const float* src, const float* dst, cudaStream_t s)
{
    pack_kernel<<<total, 256, 0, s>>>(ManyViews{b}, src, dst);
}

void launch_compat(const Batch& b, int total, cudaStream_t s, bool auto_sc2)
{
    if (auto_sc2) launch_pdl(compat_kernel<true>, total, kThreads, 0, s, ManyViews{b});
    else launch_pdl(compat_kernel<false>, total, kThreads, 0, s, ManyViews{b});
}

}  // namespace tr
