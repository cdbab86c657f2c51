// Stage 3: pivot selection (Eq. 4) on the O2Graph.
//
// P = the min(K1, |E+|) edges (i < j, W_ij > 0) of largest weight, ties at
// the threshold weight alpha broken by the lowest (i, j) (row-major linear
// index), listed in (W desc, i asc, j asc) order.
//
// Exact radix-style selection in five passes over the upper triangle of W
// (uint16, L2/HBM bound):
//   hist    histogram of edge weights (shared-memory bins per block)
//   select  one block: alpha = K1-th largest weight, c_gt = #{W > alpha},
//           m = K1' - c_gt ties still needed (K1' = min(K1, |E+|))
//   collect warp per row: every W > alpha edge into a candidate slot (order
//           free), and the number of W == alpha edges of the row
//   scan    one block: exclusive prefix of the per-row tie counts
//   emit    warp per row: the row's ties in column order get global tie
//           ranks prefix[i] + rank-in-row; ranks < m are kept
//   rank    candidate keys (W << 32 | ~(i*n+j)) are unique; each pivot's
//           position is the number of larger keys.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kHistSmemMaxBins = 24576;   // 96 KB of shared bins; larger N uses global atomics

__device__ __forceinline__ uint64_t edge_key(int w, int i, int j, int n)
{
    const uint32_t lin = static_cast<uint32_t>(i) * static_cast<uint32_t>(n) + static_cast<uint32_t>(j);
    return (static_cast<uint64_t>(w) << 32) | static_cast<uint64_t>(0xFFFFFFFFu - lin);
}

// Iterate row i's upper-triangle entries j in (i, n) in chunks of 8 uint16
// (16-byte loads); lane l takes chunks c0 + l, c0 + l + 32, ..., two loads in
// flight per lane.
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
            f(j, (j > i && j < v.n) ? w : 0);
        }
    }
}

template <bool kSmem>
__global__ void __launch_bounds__(256) hist_kernel(ProbView v)
{
    extern __shared__ uint32_t sh[];
    const int nb = v.n + 1;
    if (kSmem) {
        for (int q = threadIdx.x; q < nb; q += blockDim.x) sh[q] = 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = wid; i < v.n; i += nw) {
        for_row_chunks(v, i, lane, [&](int, int w) {
            if (w > 0) {
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

// block-wide inclusive scan of one int per thread (blockDim.x = 1024)
__device__ __forceinline__ int block_incl_scan(int x, int* sbuf)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) sbuf[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? sbuf[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        sbuf[lane] = s;
    }
    __syncthreads();
    const int r = x + (warp > 0 ? sbuf[warp - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) select_kernel(ProbView v)
{
    __shared__ int sbuf[32];
    const int nb = v.n;                       // weights 1..n (W <= n - 2)
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    // thread t owns weights (hi - per, hi], hi = n - t*per, scanned from the top
    const int hi = nb - static_cast<int>(threadIdx.x) * per;
    int mine = 0;
    for (int q = 0; q < per; ++q) {
        const int wv = hi - q;
        if (wv >= 1) mine += static_cast<int>(v.hist[wv]);
    }
    const int incl = block_incl_scan(mine, sbuf);
    __shared__ int total;
    if (threadIdx.x == blockDim.x - 1) total = incl;
    __syncthreads();
    const int n_edges = total;
    const int n_sel = n_edges < v.k1 ? n_edges : v.k1;
    if (threadIdx.x == 0) {
        v.ctl->n_edges = n_edges;
        v.ctl->n_sel = n_sel;
        v.ctl->gt_slot = 0;
        if (n_sel == 0) { v.ctl->alpha = 0x7FFFFFFF; v.ctl->c_gt = 0; v.ctl->m_ties = 0; }
    }
    if (n_sel == 0) return;
    const int excl = incl - mine;
    if (excl < n_sel && n_sel <= incl) {
        int run = excl;
        for (int q = 0; q < per; ++q) {
            const int wv = hi - q;
            if (wv < 1) break;
            const int h = static_cast<int>(v.hist[wv]);
            if (run + h >= n_sel) {
                v.ctl->alpha = wv;
                v.ctl->c_gt = run;
                v.ctl->m_ties = n_sel - run;
                break;
            }
            run += h;
        }
    }
}

__global__ void __launch_bounds__(256) collect_kernel(ProbView v)
{
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (v.ctl->n_sel == 0) return;
    const int alpha = v.ctl->alpha;
    for (int i = wid; i < v.n; i += nw) {
        int ties = 0;
        for_row_chunks(v, i, lane, [&](int j, int w) {
            if (w > alpha) {
                const uint32_t slot = atomicAdd(&v.ctl->gt_slot, 1u);
                if (slot < static_cast<uint32_t>(v.k1)) v.cand[slot] = edge_key(w, i, j, v.n);
                else atomicOr(&v.ctl->err, TR_ERR_OVERFLOW);
            } else if (w == alpha) {
                ++ties;
            }
        });
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) ties += __shfl_xor_sync(0xffffffffu, ties, off);
        if (lane == 0) v.rowcnt[i] = ties;
    }
}

__global__ void __launch_bounds__(1024) scan_rows_kernel(ProbView v)
{
    __shared__ int sbuf[32];
    if (v.ctl->n_sel == 0) return;
    const int per = (v.n + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    int mine = 0;
    for (int q = 0; q < per; ++q)
        if (lo + q < v.n) mine += v.rowcnt[lo + q];
    const int incl = block_incl_scan(mine, sbuf);
    int run = incl - mine;
    for (int q = 0; q < per; ++q)
        if (lo + q < v.n) { v.rowpref[lo + q] = run; run += v.rowcnt[lo + q]; }
}

__global__ void __launch_bounds__(256) emit_ties_kernel(ProbView v)
{
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    if (v.ctl->n_sel == 0) return;
    const int alpha = v.ctl->alpha, m = v.ctl->m_ties, c_gt = v.ctl->c_gt;
    for (int i = wid; i < v.n; i += nw) {
        if (v.rowcnt[i] == 0 || v.rowpref[i] >= m) continue;
        int base = v.rowpref[i];
        const uint16_t* wrow = v.w + (size_t)i * v.n_pad;
        const int c0 = (i + 1) >> 3, c1 = (v.n - 1) >> 3;
        // chunk-major sweep in column order: the warp covers 32 chunks (256 columns) per step
        for (int cb = c0; cb <= c1 && base < m; cb += 32) {
            const int c = cb + lane;
            uint32_t tmask = 0;
            if (c <= c1) {
                const uint4 q = *reinterpret_cast<const uint4*>(wrow + c * 8);
                const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int j = c * 8 + e;
                    const int w = (u[e >> 1] >> ((e & 1) * 16)) & 0xFFFF;
                    if (j > i && j < v.n && w == alpha) tmask |= 1u << e;
                }
            }
            const int cnt = __popc(tmask);
            int pre = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, off);
                if (lane >= off) pre += y;
            }
            const int tot = __shfl_sync(0xffffffffu, pre, 31);
            int r = base + pre - cnt;
            while (tmask) {
                const int e = __ffs(tmask) - 1;
                tmask &= tmask - 1;
                if (r < m) v.cand[c_gt + r] = edge_key(alpha, i, c * 8 + e, v.n);
                ++r;
            }
            base += tot;
        }
    }
}

// 32 candidates per block (one per lane); the 8 warps split the comparison
// range; all n_sel keys are staged in shared memory.
__global__ void __launch_bounds__(256) rank_kernel(ProbView v)
{
    extern __shared__ uint64_t sk[];
    __shared__ int part[8][32];
    const int n_sel = v.ctl->n_sel;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) v.ctl->n_pivots = n_sel;
    if (static_cast<int>(blockIdx.x * 32) >= n_sel) return;
    for (int q = threadIdx.x; q < n_sel; q += blockDim.x) sk[q] = v.cand[q];
    __syncthreads();
    const int e = blockIdx.x * 32 + lane;
    const uint64_t key = (e < n_sel) ? sk[e] : ~0ull;
    const int chunk = (n_sel + 7) / 8;
    const int f0 = warp * chunk, f1 = min(n_sel, f0 + chunk);
    int cnt = 0;
#pragma unroll 4
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

}  // namespace

cudaError_t topk_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TURBOREG_K1_MAX * 8);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(hist_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kHistSmemMaxBins * 4);
}

void launch_topk_after_hist(const ProbView& v, cudaStream_t s)
{
    const int row_blocks = (v.n + 7) / 8;   // one row per warp
    select_kernel<<<1, 1024, 0, s>>>(v);
    collect_kernel<<<row_blocks, 256, 0, s>>>(v);
    scan_rows_kernel<<<1, 1024, 0, s>>>(v);
    emit_ties_kernel<<<row_blocks, 256, 0, s>>>(v);
    rank_kernel<<<(v.k1 + 31) / 32, 256, v.k1 * 8, s>>>(v);
}

void launch_topk(const ProbView& v, cudaStream_t s)
{
    const int sms = g_num_sms > 0 ? g_num_sms : 148;
    const int hist_blocks = min((v.n + 7) / 8, 4 * sms);
    if (v.n + 1 <= kHistSmemMaxBins)
        hist_kernel<true><<<hist_blocks, 256, (v.n + 1) * 4, s>>>(v);
    else
        hist_kernel<false><<<hist_blocks, 256, 0, s>>>(v);
    launch_topk_after_hist(v, s);
}

}  // namespace tr
