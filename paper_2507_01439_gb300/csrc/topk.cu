// Stage 3: pivot selection (Eq. 4) on the O2Graph.
//
// P = the min(K1, |E+|) edges (i < j, W_ij > 0) of largest weight, ties at
// the threshold weight alpha broken by the lowest (i, j) (row-major linear
// index), listed in (W desc, i asc, j asc) order.  With the learned
// proposal the competing weight is floor(W_ij p_i p_j) (pivot_weight).
//
// Exact radix-style selection; the selected set, and so the pivots, do not
// depend on the order in which blocks run:
//   hist    histogram of edge weights (built by the SC^2 GEMM epilogue, or
//           by hist_kernel for the CUDA-core SC^2 path and for callers)
//   select  alpha = K1-th largest weight, c_gt = #{W > alpha}, m = K1' - c_gt
//           ties still needed (K1' = min(K1, |E+|)): every count block for
//           one problem whose histogram the GEMM completed, else one block
//           per problem of the select launch
//   count   blocks of eight row pairs (i, n-1-i): #{j : W_ij > alpha} and
//           #{j : W_ij == alpha}; rows with such edges join the active list
//           (rows whose largest weight, recorded by the SC^2 pass, is below
//           alpha are skipped without reading W)
//   emit    blocks over the active rows: W > alpha edges take slots from one
//           atomic per row (the rank pass orders them); ties get global tie
//           ranks (tie prefix over the active rows above) + rank-in-row
//           (column order) and ranks < m are kept
//   rank    candidate keys (W << 32 | ~(i*n+j)) are unique; each pivot's
//           position is the number of larger keys.  In the registration
//           pipeline the clique search computes these ranks itself (one warp
//           per selected edge); rank_kernel serves the allocation-free
//           selection entry point.
#include "tr_common.cuh"
#include "tr_problem.h"
#include "tr_select.cuh"

namespace tr {

namespace {

constexpr int kHistSmemMaxBins = 24576;   // 96 KB of shared bins; larger N uses global atomics
constexpr int kHistRowsPerBlock = 64;     // 8 warps x 8 rows
constexpr int kCountThreads = 256;
constexpr int kCountPairs = 8;            // row pairs per count block

__device__ __forceinline__ uint64_t edge_key(int w, int i, int j, int n)
{
    const uint32_t lin = static_cast<uint32_t>(i) * static_cast<uint32_t>(n) + static_cast<uint32_t>(j);
    return (static_cast<uint64_t>(w) << 32) | static_cast<uint64_t>(0xFFFFFFFFu - lin);
}

// Largest learned pivot weight a row can hold, before truncation: every entry
// of row i has floor(W_ij p_i p_j) with W_ij <= rowmax_i and p_j <= max p, and
// correctly rounded products of non-negative factors are monotonic, so
// fl(fl(W_ij p_i) p_j) <= fl(fl(rowmax_i p_i) pmax).  Infinite when no bound
// is available (plain weights, or no row maxima).
__device__ __forceinline__ float learned_row_bound(const ProbView& v, int i)
{
    if (v.prob == nullptr || v.rowmax == nullptr) return __int_as_float(0x7f800000);
    const float pmax = __uint_as_float(__ldcg(&v.ctl->pmax_bits));
    return __fmul_rn(__fmul_rn(static_cast<float>(__ldcg(v.rowmax + i)), __ldcg(v.prob + i)), pmax);
}

// Iterate row i's upper-triangle entries j in (i, n) in chunks of 8 uint16
// (16-byte loads); lane l takes chunks c0 + l, c0 + l + 32, ..., two loads in
// flight per lane.  Chunks whose 8 weights are all zero are skipped.
template <typename F>
__device__ __forceinline__ void for_row_chunks(const ProbView& v, int i, int lane, F&& f)
{
    if (i + 1 >= v.n) return;
    const uint16_t* wrow = v.w + (size_t)i * v.n_pad;
    const int c0 = (i + 1) >> 3, c1 = (v.n - 1) >> 3;
    for (int c = c0 + lane; c <= c1; c += 64) {
        const int cb = c + 32;
        const uint4 qa = *reinterpret_cast<const uint4*>(wrow + c * 8);
        const uint4 qb = cb <= c1 ? *reinterpret_cast<const uint4*>(wrow + cb * 8) : make_uint4(0, 0, 0, 0);
        const uint32_t u[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int j = (e < 8 ? c : cb) * 8 + (e & 7);
            const int w = (u[e >> 1] >> ((e & 1) * 16)) & 0xFFFF;
            if (u[e >> 1] == 0u) continue;
            f(j, (j > i && j < v.n) ? pivot_weight(v, i, j, w) : 0);
        }
    }
}

// Histogram of edge weights (used when SC^2 comes from the CUDA-core path or
// from a caller): 64 rows per block, shared-memory bins when they fit.  A
// caller's weight above n - 2 (no SC^2 count can be larger; the bins end at
// n) is not counted: it sets TR_ERR_BAD_WEIGHT, and the select kernel then
// selects nothing.
template <class VS, bool kSmem>
__global__ void __launch_bounds__(256) hist_kernel(VS vs)
{
    int lb;
    const ProbView v = vs.get(ST_HIST, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    extern __shared__ uint32_t sh[];
    const int nb = v.n + 1;
    if (kSmem) {
        for (int q = threadIdx.x; q < nb; q += blockDim.x) sh[q] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = 0; r < kHistRowsPerBlock / 8; ++r) {
        const int i = lb * kHistRowsPerBlock + warp * (kHistRowsPerBlock / 8) + r;
        if (i >= v.n) break;
        // learned weights: a row whose bound is below 1 holds only zeros (not counted)
        if (!(learned_row_bound(v, i) >= 1.f)) continue;
        for_row_chunks(v, i, lane, [&](int, int w) {
            if (VS::kCallerWeights && w > v.n - 2) {
                atomicOr(&v.ctl->err, TR_ERR_BAD_WEIGHT);
            } else if (w > 0) {
                if (kSmem) atomicAdd(&sh[w], 1u);
                else atomicAdd(&v.hist[w], 1u);
            }
        });
    }
    if (kSmem) {
        __syncthreads();
        for (int q = threadIdx.x; q < nb; q += blockDim.x)
            if (sh[q]) atomicAdd(&v.hist[q], sh[q]);
    }
}

template <class VS>
__global__ void __launch_bounds__(1024) select_kernel(VS vs)
{
    int lb;
    const ProbView v = vs.get(ST_SELECT, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    __shared__ int sbuf[33];
    if (VS::kCallerWeights && (v.ctl->err & TR_ERR_BAD_WEIGHT) != 0u) {
        // out-of-range weights: select nothing, so that the count, emit and
        // rank passes write no candidate (rank reports the error)
        if (threadIdx.x == 0) {
            v.ctl->n_edges = 0;
            v.ctl->n_sel = 0;
            v.ctl->alpha = 0x7FFFFFFF;
            v.ctl->c_gt = 0;
            v.ctl->m_ties = 0;
        }
        return;
    }
    select_alpha(v, sbuf);
}

// Zero the weights of a 16-byte chunk (8 entries, columns 8c .. 8c+7) outside
// the row's upper part (row, n): only a row's first and last chunks have any.
__device__ __forceinline__ uint4 mask_chunk(uint4 q, int c, int row, int n)
{
    const int lo = row + 1 - c * 8, hi = n - c * 8;   // keep entries e with lo <= e < hi
    if (lo <= 0 && hi >= 8) return q;
    uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 8; ++e)
        if (e < lo || e >= hi) wd[e >> 1] &= (e & 1) ? 0x0000FFFFu : 0xFFFF0000u;
    return make_uint4(wd[0], wd[1], wd[2], wd[3]);
}

// #{entries > alpha} and #{entries == alpha} of a chunk, as packed 16-bit
// SIMD compares (weights and alpha < 2^16; a zeroed entry never counts, alpha >= 1).
__device__ __forceinline__ void count_chunk(uint4 q, uint32_t a2, int& g, int& e)
{
    g += (__popc(__vcmpgtu2(q.x, a2)) + __popc(__vcmpgtu2(q.y, a2)) + __popc(__vcmpgtu2(q.z, a2)) +
          __popc(__vcmpgtu2(q.w, a2))) >> 4;
    e += (__popc(__vcmpeq2(q.x, a2)) + __popc(__vcmpeq2(q.y, a2)) + __popc(__vcmpeq2(q.z, a2)) +
          __popc(__vcmpeq2(q.w, a2))) >> 4;
}

// Per-row counts of the weight > alpha and weight == alpha edges.  A block
// owns eight row pairs (w, n-1-w), whose upper-triangle parts hold about n/8
// 16-byte chunks per pair, so every block has about the same span of rows.
// Rows whose largest weight (recorded by the SC^2 pass) is below alpha hold
// no such edge and are skipped without reading W (the learned pivot weight
// floor(W p_i p_j) never exceeds W).  The chunks of the remaining rows are
// spread over all the block's threads, eight 16-byte loads in flight each,
// so a block with one or two such rows reads them in one round.  Rows
// holding such edges are appended to the active list as (row, #gt, #eq), in
// any order.
// select_here (one problem whose histogram the SC^2 GEMM completed): every
// block chooses the threshold itself from the histogram, staged in dynamic
// shared memory while its row maxima load, and block 0 records it for the
// later passes; otherwise it comes from the select launch.
template <class VS>
__global__ void __launch_bounds__(kCountThreads, 3) count_kernel(VS vs, int select_here)
{
    int lb;
    const ProbView v = vs.get(ST_COUNT, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    extern __shared__ __align__(16) uint32_t shist_stage[];   // select_here: n + 4 words
    __shared__ int srow[16], sc0[16], soff[17], sg[16], se[16];
    __shared__ int ssel[40];
    const int n = v.n;
    const int t = threadIdx.x;
    // entry k = t (< 16): pair p = 8 lb + k / 2, side k % 2
    const int p = lb * kCountPairs + (t >> 1);
    const int row = (t & 1) ? n - 1 - p : p;
    bool act = t < 16 && p < (n + 1) / 2 && !((t & 1) && row == p) && row + 1 < n;
    const int rmax = (act && v.rowmax != nullptr) ? __ldg(v.rowmax + row) : 0;
    int n_sel, alpha;
    if (select_here) {
        select_alpha(v, ssel, shist_stage, ssel + 33);
        __syncthreads();
        n_sel = ssel[34];
        alpha = ssel[35];
        if (lb == 0 && t == 0) {
            v.ctl->n_edges = ssel[33];
            v.ctl->n_sel = n_sel;
            v.ctl->alpha = alpha;
            v.ctl->c_gt = ssel[36];
            v.ctl->m_ties = ssel[37];
        }
    } else {
        n_sel = v.ctl->n_sel;
        alpha = v.ctl->alpha;
    }
    if (n_sel == 0) return;                   // uniform over the block
    if (t < 32) {
        if (act && v.rowmax != nullptr) act = rmax >= alpha;
        if (act && v.prob != nullptr) act = learned_row_bound(v, row) >= static_cast<float>(alpha);
        const int c0 = (row + 1) >> 3;
        const int len = act ? ((n - 1) >> 3) - c0 + 1 : 0;
        int incl = len;
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (t >= off) incl += y;
        }
        if (t < 16) {
            srow[t] = row;
            sc0[t] = c0;
            soff[t] = incl - len;
            sg[t] = 0;
            se[t] = 0;
        }
        if (t == 15) soff[16] = incl;
    }
    __syncthreads();
    const int tot = soff[16];
    if (tot == 0) return;                     // uniform over the block
    const uint32_t a2 = static_cast<uint32_t>(alpha) * 0x10001u;
    const bool learned = v.prob != nullptr;
    int kcur = -1, g = 0, e = 0;              // running counts of entry kcur
    for (int base = t; base < tot; base += 8 * kCountThreads) {
        uint4 q[8];
        int kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int x = base + u * kCountThreads;
            int k = 0;
#pragma unroll
            for (int m = 1; m < 16; ++m) k += soff[m] <= x ? 1 : 0;
            kk[u] = k;
            q[u] = x < tot ? *reinterpret_cast<const uint4*>(v.w + (size_t)srow[k] * v.n_pad +
                                                             (size_t)(sc0[k] + x - soff[k]) * 8)
                           : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int x = base + u * kCountThreads;
            if (x >= tot) break;
            const int k = kk[u];
            const int row = srow[k], c = sc0[k] + x - soff[k];
            if (k != kcur) {
                if (kcur >= 0) {
                    if (g) atomicAdd(&sg[kcur], g);
                    if (e) atomicAdd(&se[kcur], e);
                }
                kcur = k;
                g = e = 0;
            }
            const uint4 qm = mask_chunk(q[u], c, row, n);
            if (!learned) {
                count_chunk(qm, a2, g, e);
            } else if ((qm.x | qm.y | qm.z | qm.w) != 0u) {
#pragma unroll
                for (int el = 0; el < 8; ++el) {
                    const uint32_t word = el < 2 ? qm.x : el < 4 ? qm.y : el < 6 ? qm.z : qm.w;
                    const int pw = pivot_weight(v, row, c * 8 + el, static_cast<int>((word >> ((el & 1) * 16)) & 0xFFFFu));
                    g += pw > alpha;
                    e += pw == alpha;
                }
            }
        }
    }
    if (kcur >= 0) {
        if (g) atomicAdd(&sg[kcur], g);
        if (e) atomicAdd(&se[kcur], e);
    }
    __syncthreads();
    if (t < 16 && (sg[t] | se[t]))
        v.active[atomicAdd(&v.ctl->n_active, 1u)] = make_int4(srow[t], sg[t], se[t], 0);
}

// Blocks take the active rows in any order.  W > alpha edges take slots
// base + rank-in-row from one atomic per row (any slots in [0, c_gt) will
// do: the rank pass orders the keys).  Ties must be the m lowest (i, j):
// a row with ties sums the tie counts of the active rows above it (its tie
// prefix) and keeps tie ranks prefix + rank-in-row < m.  Thread t reads
// chunks 4t .. 4t+3 of each 1024-chunk sweep (thread order = column order).
// The block's first active row is read speculatively in the same round as
// the counters, and the row's first sweep, its tie prefix and its slot
// atomic go out together in the next.
template <class VS>
__global__ void __launch_bounds__(256) emit_kernel(VS vs)
{
    int lb;
    const ProbView v = vs.get(ST_EMIT, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    __shared__ int sg[8], se[8];
    __shared__ int s_base;
    // the counters through L1: every warp of every block reads them
    const int n_sel = v.ctl->n_sel;
    const int nact = static_cast<int>(v.ctl->n_active);
    const int m = v.ctl->m_ties, alpha = v.ctl->alpha;
    const int4 ar0 = v.active[lb];                  // lb < n_pad: inside the list's capacity
    if (n_sel == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c1 = (v.n - 1) >> 3;
    const int eb = emit_blocks(v.n);
    for (int a = lb; a < nact; a += eb) {
        const int4 ar = a == lb ? ar0 : v.active[a];
        const int i = ar.x, ng = ar.y, ne = ar.z;
        const uint16_t* wrow = v.w + (size_t)i * v.n_pad;
        // first sweep of the row
        const int cb0 = (i + 1) >> 3;
        uint4 q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int cc = cb0 + threadIdx.x * 4 + k;
            q[k] = cc <= c1 ? *reinterpret_cast<const uint4*>(wrow + cc * 8) : make_uint4(0u, 0u, 0u, 0u);
        }
        // slots of the W > alpha edges
        if (threadIdx.x == 0)
            s_base = ng > 0 ? static_cast<int>(atomicAdd(&v.ctl->gt_slot, static_cast<uint32_t>(ng))) : 0;
        // tie prefix: ties in active rows above i
        int pe = 0;
        if (ne > 0) {
            int part = 0;
            for (int b = threadIdx.x; b < nact; b += blockDim.x) {
                const int4 o = v.active[b];
                part += o.x < i ? o.z : 0;
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) se[warp] = part;
            __syncthreads();
            for (int w8 = 0; w8 < 8; ++w8) pe += se[w8];
        }
        __syncthreads();
        const bool want_eq = ne > 0 && pe < m;
        if (ng == 0 && !want_eq) continue;   // uniform over the block
        const int pg = s_base;
        const int c_gt = v.ctl->c_gt;
        int base_g = pg, base_e = pe;
        for (int cb = cb0; cb <= c1; cb += blockDim.x * 4) {
            uint32_t gm = 0, em = 0;   // bit 8*k + e: chunk k, element e
            const int cfirst = cb + threadIdx.x * 4;
            if (cb != cb0) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    q[k] = cfirst + k <= c1 ? *reinterpret_cast<const uint4*>(wrow + (cfirst + k) * 8)
                                            : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if ((q[k].x | q[k].y | q[k].z | q[k].w) == 0u) continue;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t word = e < 2 ? q[k].x : e < 4 ? q[k].y : e < 6 ? q[k].z : q[k].w;
                    const int j = (cfirst + k) * 8 + e;
                    const bool in = j > i && j < v.n;
                    const int w = in ? pivot_weight(v, i, j, (word >> ((e & 1) * 16)) & 0xFFFF) : 0;
                    gm |= static_cast<uint32_t>(in && w > alpha) << (8 * k + e);
                    em |= static_cast<uint32_t>(in && w == alpha) << (8 * k + e);
                }
            }
            // block exclusive scans of the two counts (thread order = column order)
            const int g = __popc(gm), eN = __popc(em);
            int gi = g, ei = eN;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, gi, off);
                const int y = __shfl_up_sync(0xffffffffu, ei, off);
                if (lane >= off) { gi += x; ei += y; }
            }
            if (lane == 31) { sg[warp] = gi; se[warp] = ei; }
            __syncthreads();
            int wg = 0, we = 0, tg = 0, te = 0;
            for (int w8 = 0; w8 < 8; ++w8) {
                if (w8 < warp) { wg += sg[w8]; we += se[w8]; }
                tg += sg[w8];
                te += se[w8];
            }
            __syncthreads();
            int rg = base_g + wg + gi - g, re = base_e + we + ei - eN;
            while (gm) {
                const int b = __ffs(gm) - 1;
                gm &= gm - 1;
                const int j = (cfirst + (b >> 3)) * 8 + (b & 7);
                v.cand[rg++] = edge_key(pivot_weight(v, i, j, wrow[j]), i, j, v.n);
            }
            while (em) {
                const int b = __ffs(em) - 1;
                em &= em - 1;
                if (re < m) v.cand[c_gt + re] = edge_key(alpha, i, (cfirst + (b >> 3)) * 8 + (b & 7), v.n);
                ++re;
            }
            base_g += tg;
            base_e += te;
            if (base_g - pg >= ng && (!want_eq || base_e >= m || base_e - pe >= ne)) break;
        }
    }
}

// 32 candidates per block (one per lane); the 8 warps split the comparison
// range; all n_sel keys of the problem are staged in shared memory.
template <class VS>
__global__ void __launch_bounds__(256) rank_kernel(VS vs)
{
    int lb;
    const ProbView v = vs.get(ST_RANK, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    extern __shared__ uint64_t sk[];
    __shared__ int part[8][32];
    const int n_sel = v.ctl->n_sel;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lb == 0 && threadIdx.x == 0)
        v.ctl->n_pivots = (VS::kCallerWeights && (v.ctl->err & TR_ERR_BAD_WEIGHT) != 0u) ? -TURBOREG_ERR_INVALID_ARG
                                                                                         : n_sel;
    if (lb * 32 >= n_sel) return;
    for (int q = threadIdx.x; q < n_sel; q += blockDim.x) sk[q] = v.cand[q];
    __syncthreads();
    const int e = lb * 32 + lane;
    const uint64_t key = (e < n_sel) ? sk[e] : ~0ull;
    const int chunk = (n_sel + 7) / 8;
    const int f0 = warp * chunk, f1 = min(n_sel, f0 + chunk);
    int cnt = 0;
#pragma unroll 8
    for (int f = f0; f < f1; ++f) cnt += sk[f] > key;
    part[warp][lane] = cnt;
    __syncthreads();
    if (warp == 0 && e < n_sel) {
        int rank = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) rank += part[w][lane];
        const uint32_t lin = 0xFFFFFFFFu - static_cast<uint32_t>(key & 0xFFFFFFFFull);
        const int i = static_cast<int>(lin / static_cast<uint32_t>(v.n));
        const int j = static_cast<int>(lin % static_cast<uint32_t>(v.n));
        v.piv[rank] = make_int4(i, j, static_cast<int>(key >> 32), 0);
    }
}

int g_num_sms = 0;

template <class VS>
cudaError_t set_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(rank_kernel<VS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TURBOREG_K1_MAX * 8);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(hist_kernel<VS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kHistSmemMaxBins * 4);
}

template <class VS>
void launch_hist_vs(const VS& vs, int total, int max_n, cudaStream_t s)
{
    if (max_n + 1 <= kHistSmemMaxBins)
        launch_pdl(hist_kernel<VS, true>, total, 256, (max_n + 1) * 4, s, vs);
    else
        launch_pdl(hist_kernel<VS, false>, total, 256, 0, s, vs);
}

}  // namespace

cudaError_t topk_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = set_attrs<ManyViews>();
    if (e != cudaSuccess) return e;
    return set_attrs<OneView>();
}

void launch_hist(const Batch& b, int total, int max_n, cudaStream_t s)
{
    launch_hist_vs(ManyViews{b}, total, max_n, s);
}

void launch_select(const Batch& b, cudaStream_t s) { launch_pdl(select_kernel<ManyViews>, b.num, 1024, 0, s, ManyViews{b}); }

void launch_count_emit(const Batch& b, const int32_t tot[kNumBatchStages], bool select_here, int max_n,
                       cudaStream_t s)
{
    const ManyViews vs{b};
    const size_t stage = select_here ? static_cast<size_t>((max_n + 4) / 4 * 4) * 4 : 0;
    launch_pdl(count_kernel<ManyViews>, tot[ST_COUNT], kCountThreads, stage, s, vs, select_here ? 1 : 0);
    launch_pdl(emit_kernel<ManyViews>, tot[ST_EMIT], 256, 0, s, vs);
}

// One problem passed by value (no device-side problem table).
void launch_topk_single(const ProbView& v, cudaStream_t s)
{
    const OneView vs{v};
    launch_hist_vs(vs, (v.n + kHistRowsPerBlock - 1) / kHistRowsPerBlock, v.n, s);
    launch_pdl(select_kernel<OneView>, 1, 1024, 0, s, vs);
    launch_pdl(count_kernel<OneView>, count_blocks(v.n), kCountThreads, 0, s, vs, 0);
    launch_pdl(emit_kernel<OneView>, emit_blocks(v.n), 256, 0, s, vs);
    launch_pdl(rank_kernel<OneView>, (v.k1 + 31) / 32, 256, v.k1 * 8, s, vs);
}

}  // namespace tr
