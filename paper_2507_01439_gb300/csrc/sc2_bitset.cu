// Stage 2 on CUDA cores: the SC^2 weights of the O2Graph (Eq. 2, Def. 2)
// from the adjacency bitset by AND + population count,
//
//   W_ij = G_ij * popc(row_i & row_j)   for i < j,
//
// the same integers as the tensor-core GEMM (App. B: the number of triangles
// on edge (i, j)), but with work only on the edges: |E+| N_pad/32 word
// operations instead of the dense N_pad^3 multiply-adds.  Its floor is the
// population count itself (16 per clock per SM): 81.6 M words at N = 5000 and
// 4 % density, about 16 us on 152 SMs.
//
// Work tiles: row blocks of 128 rows i by column chunks of 256 columns j of
// the upper triangle (j > i).  Two forms (the pipelined one for N_pad <= 5120):
//   pipelined  halves of the tiles (128 x 128) as units; a CTA's rows i are
//              one bulk copy into shared memory, every warp streams its rows j
//              through a private queue of bulk copies; edges by warp-wide AND +
//              popc with one redux.sync each (below);
//   general    64-row halves; rows j loaded by the warps from global memory,
//              rows i staged in shared memory when they fit.
// Both write the W block staged in shared memory as full row segments (zeros
// included, so W needs no clearing), and accumulate row sums, row maxima and
// the edge-weight histogram in shared memory, with the same results as the
// GEMM's epilogue.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kBT = 128;      // rows of a work tile (row block)
constexpr int kBC = 256;      // columns of a work tile (column chunk)

// Work tiles: row blocks of kBT rows by column chunks of kBC columns that hold
// some j > i; row block bi has the chunks bi/2 .. ncb-1.  prefix(bi) = tiles
// of the row blocks before bi.
__host__ __device__ inline int bitset_tile_prefix(int bi, int ncb)
{
    const int a = bi >> 1, r = bi & 1;
    return bi * ncb - a * (a - 1) - r * a;
}

__device__ __forceinline__ void bitset_tile_of(int t, int n_pad, int& bi, int& bj)
{
    const int ncb = n_pad / kBC, nrb = n_pad / kBT;
    int lo = 0, hi = nrb;   // largest bi with prefix(bi) <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bitset_tile_prefix(mid, ncb) <= t) lo = mid;
        else hi = mid;
    }
    bi = lo;
    bj = (lo >> 1) + (t - bitset_tile_prefix(lo, ncb));
}

// Add this CTA's histogram bins of problem v to its global histogram and clear them.
__device__ __forceinline__ void flush_hist(const ProbView& v, uint32_t* sh, int tid, int nthreads)
{
    for (int b = tid + 1; b <= v.n; b += nthreads) {
        const uint32_t h = sh[b];
        if (h) {
            atomicAdd(v.hist + b, h);
            sh[b] = 0u;
        }
    }
}

// One edge (row ri of the staged block, column j): W = popc(row_i & row_j)
// by the warp (lane l holds words l + 32 q of row j in r[q]), recorded in the
// shared tile, row sums and maxima and the histogram by lane 0.  Returns W.
template <int WPL>
__device__ __forceinline__ int edge_weight(const uint32_t* si, const uint32_t (&r)[WPL], int ldb, int lane)
{
    uint32_t c = 0u;
#pragma unroll
    for (int q = 0; q < WPL; ++q)
        if (lane + 32 * q < ldb) c += __popc(si[lane + 32 * q] & r[q]);
    return static_cast<int>(__reduce_add_sync(0xffffffffu, c));
}

__device__ __forceinline__ void record_edge(uint16_t* tile, int* rsum, int* rmax, uint32_t* shist, uint32_t* ghist,
                                            int ri, int col, int c)
{
    tile[ri * kBC + col] = static_cast<uint16_t>(c);
    if (c) {
        atomicAdd(&rsum[ri], c);
        atomicMax(&rmax[ri], c);
        if (shist) atomicAdd(&shist[c], 1u);
        else atomicAdd(&ghist[c], 1u);
    }
}

// ---------------------------------------------------------------------------
// Pipelined form (N_pad <= 5120).  Work units are halves of the tiles: 128
// rows i by 128 columns j; a CTA takes a contiguous run of units in row-block-
// major order, so its 128 bitset rows i (one bulk copy into shared memory)
// change about once per CTA.  Each of the 24 warps takes the columns
// j = jlo + warp + 24 k of a unit and streams their bitset rows through a
// private three-slot queue in shared memory: lane 0 issues the 1-D bulk copy
// of a row three rows ahead, completion counted on the slot's mbarrier, so no
// warp waits for another.  For its row j a warp reads the four words over
// columns i0 .. i0+127 (the adjacent rows i < j) and computes each edge's
// popc(row_i & row_j) with kW words of AND + popc per lane and one
// redux.sync, two edges interleaved.  Row sums, row maxima and the histogram
// come from one pass over the finished unit in shared memory.
// ---------------------------------------------------------------------------
constexpr int kUC = 128;                          // columns of a work unit
constexpr int kPWarps = 24;
constexpr int kQ = 3;                             // queue slots per warp
constexpr int kPipeThreads = 32 * kPWarps;

__host__ __device__ inline size_t pipe_smem_bytes(int ldb_max, int hist_bins)
{
    return static_cast<size_t>(kBT) * ldb_max * 4 + static_cast<size_t>(kPWarps) * kQ * ldb_max * 4 +
           static_cast<size_t>(kBT) * kUC * 2 + (kPWarps * kQ + 2) * 8 + static_cast<size_t>(hist_bins) * 4;
}

// popc(row_i & row_j) summed over the warp for two rows i at once (si0, si1);
// r: this lane's words of row j (word lane + 32 q); kExact: ldb == 32 WPL
template <int WPL, bool kExact>
__device__ __forceinline__ void edge_pair(const uint32_t* si0, const uint32_t* si1, const uint32_t (&r)[WPL], int ldb,
                                          int lane, int& c0, int& c1)
{
    uint32_t a = 0u, b = 0u;
#pragma unroll
    for (int q = 0; q < WPL; ++q) {
        if (kExact || lane + 32 * q < ldb) {
            a += __popc(si0[lane + 32 * q] & r[q]);
            b += __popc(si1[lane + 32 * q] & r[q]);
        }
    }
    c0 = static_cast<int>(__reduce_add_sync(0xffffffffu, a));
    c1 = static_cast<int>(__reduce_add_sync(0xffffffffu, b));
}

template <int WPL, bool kExact>
__global__ void __launch_bounds__(kPipeThreads, 1) sc2_bitset_pipe_kernel(Batch bt, int total, int ldb_max, int hist_bins)
{
    extern __shared__ __align__(16) uint8_t ps_raw[];
    uint8_t* q8 = ps_raw;
    uint32_t* srows = reinterpret_cast<uint32_t*>(q8);   q8 += static_cast<size_t>(kBT) * ldb_max * 4;
    uint32_t* squeue = reinterpret_cast<uint32_t*>(q8);  q8 += static_cast<size_t>(kPWarps) * kQ * ldb_max * 4;
    uint16_t* stile = reinterpret_cast<uint16_t*>(q8);   q8 += static_cast<size_t>(kBT) * kUC * 2;
    uint64_t* qbar = reinterpret_cast<uint64_t*>(q8);    q8 += kPWarps * kQ * 8;
    uint64_t* rows_bar = reinterpret_cast<uint64_t*>(q8); q8 += 16;
    uint32_t* shist = reinterpret_cast<uint32_t*>(q8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kPWarps * kQ + 1) mbar_init(threadIdx.x < kPWarps * kQ ? &qbar[threadIdx.x] : rows_bar, 1);
    if (threadIdx.x == 0) fence_mbar_init();
    for (int b = threadIdx.x; b < hist_bins; b += kPipeThreads) shist[b] = 0u;
    for (int q = threadIdx.x; q < kBT * kUC / 8; q += kPipeThreads) reinterpret_cast<uint4*>(stile)[q] = make_uint4(0, 0, 0, 0);
    const int units = 2 * total;
    const int u0 = static_cast<int>((static_cast<long long>(units) * blockIdx.x) / gridDim.x);
    const int u1 = static_cast<int>((static_cast<long long>(units) * (blockIdx.x + 1)) / gridDim.x);
    __syncthreads();
    pdl_wait();
    pdl_release();
    bool ok = true;
    int cur_p = -1, cur_bi = -1;
    uint32_t rows_uses = 0, qn = 0;     // row-block loads (all threads); this warp's queue uses
    uint32_t* myq = squeue + static_cast<size_t>(warp) * kQ * ldb_max;
    uint64_t* mybar = qbar + warp * kQ;
    for (int u = u0; u < u1; ++u) {
        int lt;
        const int p = locate(bt, ST_BITSET, u >> 1, lt);
        const ProbView v = bt.views[p];
        int bi, bj;
        bitset_tile_of(lt, v.n_pad, bi, bj);
        const int i0 = bi * kBT, j0 = bj * kBC + (u & 1) * kUC;
        const int n = v.n, ldb = v.ldb, n_pad = v.n_pad;
        const int jlo = j0 > i0 + 1 ? j0 : i0 + 1;
        const int jhi = j0 + kUC < n ? j0 + kUC : n;
        if (p != cur_p && cur_p >= 0 && hist_bins > 0) {
            flush_hist(bt.views[cur_p], shist, threadIdx.x, kPipeThreads);
            __syncthreads();
        }
        const bool new_rows = p != cur_p || bi != cur_bi;
        cur_p = p;
        cur_bi = bi;
        if (new_rows && threadIdx.x == 0) {
            fence_proxy_async();   // the previous rows were read through the generic proxy
            mbar_arrive_expect_tx(rows_bar, kBT * ldb * 4);
            bulk_g2s(srows, v.bits + (size_t)i0 * ldb, kBT * ldb * 4, rows_bar);
        }
        // this warp's rows j, kQ in flight
        const int nj = jhi > jlo + warp ? (jhi - jlo - warp + kPWarps - 1) / kPWarps : 0;
        if (lane == 0) {
            for (int k = 0; k < kQ && k < nj; ++k) {
                const uint32_t sl = (qn + k) % kQ;
                mbar_arrive_expect_tx(&mybar[sl], ldb * 4);
                bulk_g2s(myq + sl * ldb_max, v.bits + (size_t)(jlo + warp + k * kPWarps) * ldb, ldb * 4, &mybar[sl]);
            }
        }
        if (new_rows) ok &= mbar_wait(rows_bar, rows_uses & 1u);
        const int wi = i0 >> 5;   // first word of the block's rows (multiple of 4)
        for (int k = 0; k < nj; ++k) {
            const uint32_t sl = (qn + k) % kQ, ph = ((qn + k) / kQ) & 1u;
            const bool got = mbar_wait(&mybar[sl], ph);
            ok &= got;
            const int j = jlo + warp + k * kPWarps;
            const uint32_t* rj = myq + sl * ldb_max;
            uint32_t r[WPL];
#pragma unroll
            for (int q = 0; q < WPL; ++q) r[q] = (kExact || lane + 32 * q < ldb) ? rj[lane + 32 * q] : 0u;
            const uint4 mw = *reinterpret_cast<const uint4*>(rj + wi);   // adjacency of j to rows i0 .. i0+127
            __syncwarp();
            if (lane == 0 && k + kQ < nj) {   // the slot is read: refill it with the row kQ ahead
                fence_proxy_async();
                mbar_arrive_expect_tx(&mybar[sl], ldb * 4);
                bulk_g2s(myq + sl * ldb_max, v.bits + (size_t)(j + kQ * kPWarps) * ldb, ldb * 4, &mybar[sl]);
            }
            if (!got) continue;
            uint32_t m[4] = {mw.x, mw.y, mw.z, mw.w};
            const int lim = j - i0;            // rows i < j
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int lh = lim - 32 * h;
                if (lh <= 0) m[h] = 0u;
                else if (lh < 32) m[h] &= (1u << lh) - 1u;
            }
            int colsum = 0;
            uint16_t* tcol = stile + (j - j0);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t mask = m[h];
                while (mask) {
                    const int ra = 32 * h + __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int rb = mask ? 32 * h + __ffs(mask) - 1 : ra;   // second edge (or a repeat)
                    mask &= mask - 1u;
                    int ca, cb;
                    edge_pair<WPL, kExact>(srows + ra * ldb, srows + rb * ldb, r, ldb, lane, ca, cb);
                    if (rb == ra) cb = 0;
                    colsum += ca + cb;
                    if (lane == 0) tcol[ra * kUC] = static_cast<uint16_t>(ca);
                    if (lane == 1 && rb != ra) tcol[rb * kUC] = static_cast<uint16_t>(cb);
                }
            }
            if (lane == 0 && colsum) atomicAdd(&v.rowscore[j], colsum);
        }
        qn += static_cast<uint32_t>(nj);
        rows_uses += new_rows ? 1u : 0u;
        __syncthreads();   // the unit is complete in shared memory
        // W rows i0 .. i0+127 (256-byte segments), row sums, row maxima, histogram
        for (int q = threadIdx.x; q < kBT * kUC / 8; q += kPipeThreads) {
            const int rr = q >> 4, c8 = (q & 15) * 8;
            *reinterpret_cast<uint4*>(v.w + (size_t)(i0 + rr) * n_pad + j0 + c8) = reinterpret_cast<const uint4*>(stile)[q];
        }
        if (threadIdx.x < 4 * kBT) {
            const int rr = threadIdx.x >> 2, qt = threadIdx.x & 3;
            const uint4* src = reinterpret_cast<const uint4*>(stile + rr * kUC + qt * 32);
            int sum = 0, mx = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint4 w4 = src[c];
                const uint32_t wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (wv[e] == 0u) continue;
                    const int lo = static_cast<int>(wv[e] & 0xFFFFu), hi = static_cast<int>(wv[e] >> 16);
                    sum += lo + hi;
                    mx = max(mx, max(lo, hi));
                    uint32_t* hh = hist_bins > 0 ? shist : v.hist;
                    if (lo) atomicAdd(&hh[lo], 1u);
                    if (hi) atomicAdd(&hh[hi], 1u);
                }
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
            if (qt == 0) {
                if (sum) atomicAdd(&v.rowscore[i0 + rr], sum);
                if (mx && v.rowmax) atomicMax(&v.rowmax[i0 + rr], mx);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kBT * kUC / 8; q += kPipeThreads) reinterpret_cast<uint4*>(stile)[q] = make_uint4(0, 0, 0, 0);
        __syncthreads();   // cleared for the next unit; the row block may be replaced
    }
    if (!ok && lane == 0) atomicOr(&bt.views[0].ctl->err, TR_ERR_TIMEOUT);
    if (cur_p >= 0 && hist_bins > 0) flush_hist(bt.views[cur_p], shist, threadIdx.x, kPipeThreads);
}

// ---------------------------------------------------------------------------
// General form (any N): persistent CTAs of 8 warps take the same tiles as two
// halves of 64 rows; a warp loads row j straight from global memory (the next
// one in flight while it works on the current).  The 64 rows i are staged in
// shared memory when they fit, else read from global memory (largest N).
// ---------------------------------------------------------------------------
constexpr int kBR = 64;
constexpr int kBsThreads = 256;
constexpr int kBsWarps = kBsThreads / 32;

// rows_ldb: words per staged row (0: rows i from global memory); hist_bins: 0
// when the bins do not fit and are added to the global histogram directly
template <int WPL>
__global__ void __launch_bounds__(kBsThreads, 2) sc2_bitset_kernel(Batch bt, int total, int rows_ldb, int hist_bins)
{
    extern __shared__ __align__(16) uint8_t bs_raw[];
    uint16_t* stile = reinterpret_cast<uint16_t*>(bs_raw);
    uint32_t* srows = reinterpret_cast<uint32_t*>(bs_raw + kBR * kBC * 2);
    int* srsum = reinterpret_cast<int*>(srows + kBR * rows_ldb);
    int* srmax = srsum + kBR;
    uint32_t* shist = reinterpret_cast<uint32_t*>(srmax + kBR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < hist_bins; b += kBsThreads) shist[b] = 0u;
    const int t0 = static_cast<int>((static_cast<long long>(total) * blockIdx.x) / gridDim.x);
    const int t1 = static_cast<int>((static_cast<long long>(total) * (blockIdx.x + 1)) / gridDim.x);
    pdl_wait();
    pdl_release();
    int cur_p = -1;
    for (int t = t0; t < t1; ++t) {
        int lt;
        const int p = locate(bt, ST_BITSET, t, lt);
        const ProbView v = bt.views[p];
        int bi, bj;
        bitset_tile_of(lt, v.n_pad, bi, bj);
        const int n = v.n, ldb = v.ldb;
        if (p != cur_p && cur_p >= 0 && hist_bins > 0) {
            __syncthreads();
            flush_hist(bt.views[cur_p], shist, threadIdx.x, kBsThreads);
        }
        cur_p = p;
        for (int half = 0; half < 2; ++half) {
            const int i0 = bi * kBT + half * kBR, j0 = bj * kBC;
            __syncthreads();   // the previous half's shared data is consumed
            if (rows_ldb > 0) {
                const uint4* src = reinterpret_cast<const uint4*>(v.bits + (size_t)i0 * ldb);
                for (int q = threadIdx.x; q < kBR * ldb / 4; q += kBsThreads) reinterpret_cast<uint4*>(srows)[q] = src[q];
            }
            for (int q = threadIdx.x; q < kBR * kBC / 8; q += kBsThreads)
                reinterpret_cast<uint4*>(stile)[q] = make_uint4(0, 0, 0, 0);
            if (threadIdx.x < kBR) {
                srsum[threadIdx.x] = 0;
                srmax[threadIdx.x] = 0;
            }
            __syncthreads();
            const int wi = i0 >> 5;
            const int jlo = j0 > i0 + 1 ? j0 : i0 + 1;
            const int jhi = j0 + kBC < n ? j0 + kBC : n;
            int j = jlo + warp;
            uint32_t r[WPL];
#pragma unroll
            for (int q = 0; q < WPL; ++q)
                r[q] = (j < jhi && lane + 32 * q < ldb) ? __ldg(v.bits + (size_t)j * ldb + lane + 32 * q) : 0u;
            for (; j < jhi; j += kBsWarps) {
                uint32_t rn[WPL];
                const int jn = j + kBsWarps;
#pragma unroll
                for (int q = 0; q < WPL; ++q)
                    rn[q] = (jn < jhi && lane + 32 * q < ldb) ? __ldg(v.bits + (size_t)jn * ldb + lane + 32 * q) : 0u;
                // adjacency of j to rows i0 .. i0+63 (words wi, wi+1 of row j, an L1 hit;
                // selecting them from the lanes' registers would index the array)
                const uint2 wm = __ldg(reinterpret_cast<const uint2*>(v.bits + (size_t)j * ldb + wi));
                uint64_t mask = static_cast<uint64_t>(wm.x) | (static_cast<uint64_t>(wm.y) << 32);
                const int lim = j - i0;
                if (lim < 64) mask &= (1ull << lim) - 1ull;
                int colsum = 0;
                while (mask) {
                    const int ri = __ffsll(static_cast<long long>(mask)) - 1;
                    mask &= mask - 1ull;
                    const uint32_t* si = rows_ldb > 0 ? srows + ri * ldb : v.bits + (size_t)(i0 + ri) * ldb;
                    const int c = edge_weight<WPL>(si, r, ldb, lane);
                    colsum += c;
                    if (lane == 0)
                        record_edge(stile, srsum, srmax, hist_bins > 0 ? shist : nullptr, v.hist, ri, j - j0, c);
                }
                if (lane == 0 && colsum) atomicAdd(&v.rowscore[j], colsum);
#pragma unroll
                for (int q = 0; q < WPL; ++q) r[q] = rn[q];
            }
            __syncthreads();
            for (int q = threadIdx.x; q < kBR * kBC / 8; q += kBsThreads) {
                const int rr = q >> 5, c8 = (q & 31) * 8;
                *reinterpret_cast<uint4*>(v.w + (size_t)(i0 + rr) * v.n_pad + j0 + c8) =
                    reinterpret_cast<const uint4*>(stile)[q];
            }
            if (threadIdx.x < kBR) {
                const int s = srsum[threadIdx.x], m = srmax[threadIdx.x];
                if (s) atomicAdd(&v.rowscore[i0 + threadIdx.x], s);
                if (m && v.rowmax) atomicMax(&v.rowmax[i0 + threadIdx.x], m);
            }
        }
    }
    if (cur_p >= 0 && hist_bins > 0) {
        __syncthreads();
        flush_hist(bt.views[cur_p], shist, threadIdx.x, kBsThreads);
    }
}

int g_bs_sms = 0;

size_t bitset_smem(int rows_ldb, int hist_bins)
{
    return static_cast<size_t>(kBR) * kBC * 2 + static_cast<size_t>(kBR) * rows_ldb * 4 + 2 * kBR * 4 +
           static_cast<size_t>(hist_bins) * 4;
}

constexpr int kBsSmemMax = 232448;
constexpr int kPipeMaxLdb = 160;   // the pipelined form: N_pad <= 5120

template <int WPL>
cudaError_t bs_attr()
{
    return cudaFuncSetAttribute(sc2_bitset_kernel<WPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBsSmemMax);
}

template <int WPL, bool kExact>
cudaError_t pipe_attr()
{
    return cudaFuncSetAttribute(sc2_bitset_pipe_kernel<WPL, kExact>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBsSmemMax);
}

}  // namespace

int bitset_tiles(int n_pad) { return bitset_tile_prefix(n_pad / kBT, n_pad / kBC); }

cudaError_t sc2_bitset_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_bs_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = bs_attr<8>();
    if (e == cudaSuccess) e = bs_attr<16>();
    if (e == cudaSuccess) e = bs_attr<32>();
    if (e == cudaSuccess) e = pipe_attr<2, false>();
    if (e == cudaSuccess) e = pipe_attr<5, false>();
    if (e == cudaSuccess) e = pipe_attr<5, true>();
    return e;
}

bool launch_sc2_bitset(const Batch& b, int total_tiles, int max_n, int min_n, cudaStream_t s)
{
    const int max_npad = (max_n + kSc2BN - 1) / kSc2BN * kSc2BN;
    const int max_ldb = max_npad / 32;
    const int sms = g_bs_sms > 0 ? g_bs_sms : 148;
    if (max_ldb <= kPipeMaxLdb) {
        int hist_bins = max_n + 1;
        if (pipe_smem_bytes(max_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
        const size_t smem = pipe_smem_bytes(max_ldb, hist_bins);
        const int grid = sms < 2 * total_tiles ? sms : 2 * total_tiles;
        // kExact (no per-lane word guard) when every problem's rows are 5 x 32 words
        const int min_ldb = (min_n + kSc2BN - 1) / kSc2BN * kSc2BN / 32;
        const int exact_ldb = min_ldb == max_ldb ? max_ldb : 0;
        if (max_ldb <= 64)
            launch_pdl(sc2_bitset_pipe_kernel<2, false>, grid, kPipeThreads, smem, s, b, total_tiles, max_ldb, hist_bins);
        else if (exact_ldb == 160)
            launch_pdl(sc2_bitset_pipe_kernel<5, true>, grid, kPipeThreads, smem, s, b, total_tiles, max_ldb, hist_bins);
        else
            launch_pdl(sc2_bitset_pipe_kernel<5, false>, grid, kPipeThreads, smem, s, b, total_tiles, max_ldb, hist_bins);
        return true;
    }
    // shared memory for the row block and the histogram bins, as far as they fit
    int rows_ldb = max_ldb, hist_bins = max_n + 1;
    if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
    if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) {
        rows_ldb = 0;
        hist_bins = max_n + 1;
        if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
    }
    const size_t smem = bitset_smem(rows_ldb, hist_bins);
    const int per_sm = smem <= static_cast<size_t>(kBsSmemMax / 2 - 1024) ? 2 : 1;
    int grid = sms * per_sm;
    if (grid > total_tiles) grid = total_tiles;
    const int wpl = (max_ldb + 31) / 32;
    if (wpl <= 8) launch_pdl(sc2_bitset_kernel<8>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    else if (wpl <= 16) launch_pdl(sc2_bitset_kernel<16>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    else launch_pdl(sc2_bitset_kernel<32>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    return true;
}

}  // namespace tr
