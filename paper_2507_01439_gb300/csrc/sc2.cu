// Stage 2: SC^2 graph (Eq. 2) restricted to the O2Graph (Def. 2).
//
//   W_ij = G_ij * sum_k G_ik G_jk  for i < j,   i.e.  W = triu(G .* (G G), 1)
//
// Main path: a binary GEMM on the 5th-generation tensor cores.  G is stored
// as FP8 E4M3 0/1 bytes; since G is symmetric, G G = G G^T, so both MMA
// operands are K-major row blocks of the same matrix.  Products of 0/1 are
// exact and the FP32 accumulator holds integers <= N-2 < 2^24 exactly, so the
// result is the integer SC^2 count.  Only output tiles that contain some
// i < j are computed (the upper triangle, about half the square).
//
// Kernel anatomy (one 128 x 256 output tile per CTA, 128 threads):
//   warp 0 lane 0  TMA producer: 128-byte-swizzled K-major tiles A[i-block,k],
//                  A[j-block,k] into a 4-stage shared-memory ring (mbarriers)
//   warp 1 lane 0  MMA issuer: tcgen05.mma kind::f8f6f4, M=128 N=256 K=32,
//                  4 per stage, accumulating in 256 TMEM columns
//   warps 0-3      epilogue: tcgen05.ld the accumulator (warp w owns TMEM
//                  lanes 32w..32w+31 = tile rows), mask with the adjacency
//                  bitset and i < j, store uint16 W, and add the row and
//                  column sums into the SC^2 row scores.
//
// Alternative (sc2_bitset.cu): the same integers from the adjacency bitset
// with AND + popcount on CUDA cores, work only on the edges.
#include "tr_common.cuh"
#include "tr_problem.h"
#include "tr_select.cuh"

namespace tr {

namespace {

constexpr int kStages = 4;
constexpr int kABytes = kSc2BM * kSc2BK;   // 16 KB
constexpr int kBBytes = kSc2BN * kSc2BK;   // 32 KB
constexpr int kEpiWarps = 16;              // 4 per TMEM lane quarter, each a quarter of the columns
constexpr int kEpiCols = 4 * kSc2BN / kEpiWarps;   // 64 columns per epilogue warp
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kPipeBytes = kStages * (kABytes + kBBytes);
constexpr int kBarBytes = 512;            // mbarriers, TMEM slot, select scratch
constexpr int kSmemMax = 232448;           // 227 KB opt-in limit per block
constexpr uint32_t kTmemCols = 512;        // two 256-column FP32 accumulators
// E4M3 x E4M3 -> F32, M = 128, N = 256, both K-major
constexpr uint32_t kIdesc = idesc_f32acc(0u, 0u, kSc2BM, kSc2BN);

__device__ __forceinline__ void tile_of(int t, int& bm, int& bn)
{
    // tiles of column block bn are row blocks 0 .. 2bn+1; column block bn starts at t = bn(bn+1)
    int b = static_cast<int>((sqrtf(4.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (b * (b + 1) > t) --b;
    while ((b + 1) * (b + 2) <= t) ++b;
    bn = b;
    bm = t - b * (b + 1);
}

// Epilogue of one 128 x 256 output tile whose FP32 accumulator is at TMEM
// column tacc: warp (quarter, part) reads TMEM lanes 32 quarter .. +31 (tile
// rows) and the kEpiCols columns of its part, masks with the adjacency bitset
// and i < j, stores uint16 W, adds the row and column sums to the SC^2 row
// scores and counts the edge weights (shared or global histogram).  The
// bitset words of the warp's columns are fetched before the accumulator is
// waited for (epi_words), so their latency overlaps the MMAs.
__device__ __forceinline__ uint2 epi_words(const ProbView& v, int bm, int bn, int quarter, int part, int lane)
{
    static_assert(kEpiCols == 64, "one 8-byte bitset load per warp row");
    const int row = bm * kSc2BM + quarter * 32 + lane;
    return *reinterpret_cast<const uint2*>(v.bits + (size_t)row * v.ldb + ((bn * kSc2BN + part * kEpiCols) >> 5));
}

template <bool kSingle>
__device__ __forceinline__ void sc2_epilogue_tile(const ProbView& v, uint32_t tacc, int bm, int bn, int quarter,
                                                  int part, int lane, uint2 words, uint32_t* shist)
{
    const int row = bm * kSc2BM + quarter * 32 + lane;
    uint16_t* wrow = v.w + (size_t)row * v.n_pad;
    int rsum = 0, rmax = 0;
#pragma unroll 1
    for (int c = 0; c < kEpiCols / 32; ++c) {
        const int cc = part * kEpiCols + c * 32;
        uint32_t acc[32];
        tmem_ld32(tacc + static_cast<uint32_t>(cc) + (static_cast<uint32_t>(quarter * 32) << 16),
                  acc);
        tmem_ld_wait();
        const int col0 = bn * kSc2BN + cc;
        uint32_t word = c == 0 ? words.x : words.y;
        if (col0 + 31 <= row) word = 0u;                       // keep only j > row
        else if (col0 <= row) word &= ~0u << (row - col0 + 1);
        int val[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            val[q] = ((word >> q) & 1u) ? static_cast<int>(__uint_as_float(acc[q])) : 0;
            rsum += val[q];
            rmax = max(rmax, val[q]);
        }
        if (word) {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (val[q] > 0) {
                    if (kSingle) atomicAdd(&shist[val[q]], 1u);
                    else atomicAdd(&v.hist[val[q]], 1u);
                }
        }
        uint4* dst = reinterpret_cast<uint4*>(wrow + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 pk;
            pk.x = static_cast<uint32_t>(val[8 * q + 0]) | (static_cast<uint32_t>(val[8 * q + 1]) << 16);
            pk.y = static_cast<uint32_t>(val[8 * q + 2]) | (static_cast<uint32_t>(val[8 * q + 3]) << 16);
            pk.z = static_cast<uint32_t>(val[8 * q + 4]) | (static_cast<uint32_t>(val[8 * q + 5]) << 16);
            pk.w = static_cast<uint32_t>(val[8 * q + 6]) | (static_cast<uint32_t>(val[8 * q + 7]) << 16);
            dst[q] = pk;
        }
        // column sums over this warp's 32 rows (butterfly transpose-reduce):
        // afterwards lane l holds the sum of column col0 + l
        if (__any_sync(0xffffffffu, word != 0u)) {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const bool upper = (lane & off) != 0;
#pragma unroll
                for (int q = 0; q < off; ++q) {
                    const int send = upper ? val[q] : val[q + off];
                    const int keepv = upper ? val[q + off] : val[q];
                    val[q] = keepv + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            if (val[0] != 0) atomicAdd(&v.rowscore[col0 + lane], val[0]);
        }
    }
    if (rsum != 0) atomicAdd(&v.rowscore[row], rsum);
    if (rmax != 0 && v.rowmax) atomicMax(&v.rowmax[row], rmax);
}

// The same epilogue through the warp's 2 KB of shared memory `stg`, which
// holds the warp's 32 x 32 block of W (row r as four 16-byte chunks, chunk q
// at slot q ^ ((r >> 1) & 3), so that row-wise and column-wise accesses are
// both free of bank conflicts).  From there:
//   W store       pass k writes rows 8k .. 8k + 7, lane l chunk l % 4 of row
//                 8k + l / 4: each instruction covers 8 x 64 contiguous bytes
//   column sums   lane l reads 8 bytes (4 columns) of rows 4k + l / 8; the
//                 four row groups are added with two shuffles per column
//   histogram     each lane visits only the set bits of its adjacency word
// These replace per-lane row stores (a half-filled sector per lane), the
// 31-shuffle butterfly and 32 predicated atomics per chunk.
__device__ __forceinline__ uint32_t stg_slot(int r, int q) { return static_cast<uint32_t>(r * 4 + (q ^ ((r >> 1) & 3))); }

template <bool kSingle>
__device__ __forceinline__ void sc2_epilogue_tile_staged(const ProbView& v, uint32_t tacc, int bm, int bn, int quarter,
                                                         int part, int lane, uint2 words, uint32_t* shist, uint4* stg)
{
    const int row0 = bm * kSc2BM + quarter * 32;
    const int row = row0 + lane;
    int rsum = 0, rmax = 0;
#pragma unroll 1
    for (int c = 0; c < kEpiCols / 32; ++c) {
        const int cc = part * kEpiCols + c * 32;
        uint32_t acc[32];
        tmem_ld32(tacc + static_cast<uint32_t>(cc) + (static_cast<uint32_t>(quarter * 32) << 16),
                  acc);
        tmem_ld_wait();
        const int col0 = bn * kSc2BN + cc;
        uint32_t word = c == 0 ? words.x : words.y;
        if (col0 + 31 <= row) word = 0u;                       // keep only j > row
        else if (col0 <= row) word &= ~0u << (row - col0 + 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int a = 8 * q + 2 * e;
                const int lo = ((word >> a) & 1u) ? static_cast<int>(__uint_as_float(acc[a])) : 0;
                const int hi = ((word >> (a + 1)) & 1u) ? static_cast<int>(__uint_as_float(acc[a + 1])) : 0;
                rsum += lo + hi;
                rmax = max(rmax, max(lo, hi));
                h[e] = static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
            }
            stg[stg_slot(lane, q)] = make_uint4(h[0], h[1], h[2], h[3]);
        }
        __syncwarp();
        // W rows, as full 64-byte segments
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + (lane >> 2), q = lane & 3;
            *reinterpret_cast<uint4*>(v.w + (size_t)(row0 + r) * v.n_pad + col0 + q * 8) = stg[stg_slot(r, q)];
        }
        // column sums: lane l adds columns 4 (l % 8) .. +3 over rows l / 8 + 4k
        if (__any_sync(0xffffffffu, word != 0u)) {
            static_assert(2 * (TURBOREG_MAX_N - 2) < 65536, "two weights add without a carry out of 16 bits");
            const int m = lane & 7;
            int cs[4] = {0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const uint2 d0 = reinterpret_cast<const uint2*>(stg + stg_slot(4 * k + (lane >> 3), m >> 1))[m & 1];
                const uint2 d1 = reinterpret_cast<const uint2*>(stg + stg_slot(4 * k + 4 + (lane >> 3), m >> 1))[m & 1];
                const uint32_t x = d0.x + d1.x, y = d0.y + d1.y;   // two rows per 16-bit lane
                cs[0] += static_cast<int>(x & 0xFFFFu);
                cs[1] += static_cast<int>(x >> 16);
                cs[2] += static_cast<int>(y & 0xFFFFu);
                cs[3] += static_cast<int>(y >> 16);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cs[e] += __shfl_xor_sync(0xffffffffu, cs[e], 8);
                cs[e] += __shfl_xor_sync(0xffffffffu, cs[e], 16);
            }
            // lane l reports column 4 (l % 8) + l / 8
            const int e = lane >> 3;
            const int sum = e == 0 ? cs[0] : e == 1 ? cs[1] : e == 2 ? cs[2] : cs[3];
            if (sum != 0) atomicAdd(&v.rowscore[col0 + 4 * m + e], sum);
        }
        // histogram of the edge weights: only this lane's edges
        for (uint32_t bits = word; bits != 0u; bits &= bits - 1u) {
            const int q = __ffs(bits) - 1;
            const int w = reinterpret_cast<const uint16_t*>(stg + stg_slot(lane, q >> 3))[q & 7];
            if (w > 0) {
                if (kSingle) atomicAdd(&shist[w], 1u);
                else atomicAdd(&v.hist[w], 1u);
            }
        }
        __syncwarp();   // the next chunk overwrites the staging area
    }
    if (rsum != 0) atomicAdd(&v.rowscore[row], rsum);
    if (rmax != 0 && v.rowmax) atomicMax(&v.rowmax[row], rmax);
}

// Persistent, warp-specialised: CTA b handles global tiles b, b + grid, ...
// of all problems of the batch (problem p's tiles are [pre[p], pre[p+1]) of
// stage ST_GEMM; tensor maps of problem p at maps[2p], maps[2p+1]).
//   warp 0 lane 0   TMA producer over all (tile, k) of this CTA
//   warp 1 lane 0   MMA issuer; accumulator buffer (tile count & 1)
//   warps 2..17     epilogue of the previous tile while the next one runs
// kSingle: one problem: the edge-weight histogram is kept in shared memory
// and added to the global one at the end (the count pass then chooses the
// pivot threshold from it).
template <bool kSingle>
__global__ void __launch_bounds__(kThreads, 1) sc2_tcgen05_kernel(Batch bt, int total)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPipeBytes);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;      // [2] accumulator ready
    uint64_t* tempty = tfull + 2;           // [2] accumulator drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + kPipeBytes + kBarBytes);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbins = kSingle ? bt.views[0].n + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        fence_mbar_init();
    }
    if (kSingle)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) shist[b] = 0u;
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    const int u0 = static_cast<int>(blockIdx.x);
    const int us = static_cast<int>(gridDim.x);
    const int nu = total;
    // the set-up above (barriers, tensor memory, shared histogram) overlaps the
    // previous stage; its outputs are read only from here on
    pdl_wait();
    pdl_release();

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int it = 0;
            for (int u = u0; u < nu && ok; u += us) {
                int lt;
                const int p = locate(bt, ST_GEMM, u, lt);
                const int KT = bt.views[p].n_pad / kSc2BK;
                const CUtensorMap* mA = bt.maps + 2 * p;
                const CUtensorMap* mB = mA + 1;
                int bm, bn;
                tile_of(lt, bm, bn);
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int s = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
                    mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
                    tma_load_2d(sA + s * kABytes, mA, kb * kSc2BK, bm * kSc2BM, &full[s]);
                    tma_load_2d(sB + s * kBBytes, mB, kb * kSc2BK, bn * kSc2BN, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int it = 0, tc = 0;
            for (int u = u0; u < nu && ok; u += us, ++tc) {
                int lt;
                const int p = locate(bt, ST_GEMM, u, lt);
                const int KT = bt.views[p].n_pad / kSc2BK;
                const int buf = tc & 1;
                const uint32_t use = static_cast<uint32_t>(tc >> 1);
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * kSc2BN);
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int s = it % kStages;
                    const uint32_t ph = (it / kStages) & 1u;
                    if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kABytes);
                    const uint32_t b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
                    for (int k = 0; k < kSc2BK / 32; ++k)   // K = 32 FP8 per MMA, 32-byte steps in the swizzle row
                        mma_f8f6f4(d, sdesc_k_sw128(a0 + k * 32), sdesc_k_sw128(b0 + k * 32), kIdesc,
                                   (kb | k) != 0 ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[buf]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        const int quarter = warp & 3;              // TMEM lanes this warp may access
        const int part = (warp - 2) >> 2;          // column part of the tile
        int tc = 0;
        for (int u = u0; u < nu; u += us, ++tc) {
            int lt;
            const int p = locate(bt, ST_GEMM, u, lt);
            const ProbView v = bt.views[p];
            int bm, bn;
            tile_of(lt, bm, bn);
            const int buf = tc & 1;
            const uint32_t use = static_cast<uint32_t>(tc >> 1);
            const uint2 words = epi_words(v, bm, bn, quarter, part, lane);
            const bool got = mbar_wait(&tfull[buf], use & 1u);
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            tc_fence_after();
            sc2_epilogue_tile<kSingle>(v, tmem + static_cast<uint32_t>(buf * kSc2BN), bm, bn, quarter, part, lane, words,
                                       shist);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    if (!ok && lane == 0) atomicOr(&bt.views[0].ctl->err, TR_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
    if (!kSingle) return;
    // this CTA's histogram into the global one, from which the count pass
    // chooses the pivot threshold
    const ProbView v0 = bt.views[0];
    for (int b = threadIdx.x + 1; b < nbins; b += blockDim.x)
        if (shist[b]) atomicAdd(&v0.hist[b], shist[b]);
}

// 2-SM form (cta_group::2): the two CTAs of a cluster compute one 256 x 256
// output block with pair MMAs (M = 256: 128 rows of A per CTA; N = 256: 128
// columns of B per CTA).  Each CTA's shared memory holds only its own halves
// (32 KB per 128-deep K stage instead of 48 KB), so five stages fit beside a
// 32 KB staging area through which the epilogue writes W as full 64-byte row
// segments (the direct per-row stores of the other forms half-fill a sector
// per lane and slow the concurrent MMAs).
//   both CTAs  warp 0 lane 0: TMA loads of this CTA's A and B halves, counted
//              on the leader's `full` barrier; the leader announces 64 KB
//   leader     warp 1 lane 0: pair MMAs; their commits release the stage in
//              both CTAs (`empty`) and hand each CTA its accumulator (`tfull`)
//   both CTAs  warps 2..17: epilogue of this CTA's 128 x 256 rows; the
//              accumulator is free again when the epilogue warps of both CTAs
//              have arrived on the leader's `tempty`
// Every wait is bounded; before exit each producer waits for the last stage
// releases and the cluster synchronises, so no arrival targets a finished CTA.
constexpr int kStages2 = 5;
constexpr int kPipeBytes2 = kStages2 * 2 * kABytes;   // 160 KB
constexpr int kStageBytes2 = kEpiWarps * 2048;       // W staging: 32 x 32 uint16 per epilogue warp
constexpr int kBase2 = kPipeBytes2 + kBarBytes + kStageBytes2 + 1024;   // before the shared histogram

// auto_mode: one problem whose SC^2 path the CUDA-core kernel before this one
// chose; when it chose itself, every CTA returns at once (before any set-up).
template <bool kHist>
__global__ void __launch_bounds__(kThreads, 1) sc2_pair_mma_kernel(Batch bt, int total, int hist_bins, int auto_mode)
{
    if (auto_mode) {
        const Ctl* ctl = bt.views[0].ctl;   // the descriptor before the wait, the flag after it
        pdl_wait();
        if (__ldcg(&ctl->sc2_path) != 2u) {
            pdl_release();
            return;
        }
    }
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                                  // [stage] 128 rows x 128 B
    uint8_t* sB = smem + kStages2 * kABytes;             // [stage] 128 rows x 128 B (this CTA's B half)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPipeBytes2);
    uint64_t* empty = full + kStages2;
    uint64_t* tfull = empty + kStages2;      // [2] accumulator ready
    uint64_t* tempty = tfull + 2;            // [2] accumulator drained (leader's counts both CTAs)
    uint64_t* hsync = tempty + 2;            // epilogue warps: a problem's bins complete / flushed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 3);
    uint4* stg = reinterpret_cast<uint4*>(smem + kPipeBytes2 + kBarBytes);
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + kPipeBytes2 + kBarBytes + kStageBytes2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbins = kHist ? hist_bins : 0;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages2; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * kEpiWarps);
        }
        mbar_init(hsync, kEpiWarps);
        fence_mbar_init();
    }
    if (kHist)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) shist[b] = 0u;
    if (warp == 0) tmem_alloc_pair(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // both CTAs' barriers and tensor memory are ready
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    const int u0 = static_cast<int>(blockIdx.x >> 1);
    const int us = static_cast<int>(gridDim.x >> 1);
    const int nu = total >> 1;
    const uint32_t full_l = mapa_shared(&full[0], 0);      // leader's barriers, cluster addresses
    const uint32_t tempty_l = mapa_shared(&tempty[0], 0);
    pdl_wait();
    pdl_release();

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            int it = 0;
            for (int u = u0; u < nu && ok; u += us) {
                const int t = 2 * u + static_cast<int>(rank);
                int lt;
                const int p = locate(bt, ST_GEMM, t, lt);
                const int KT = bt.views[p].n_pad / kSc2BK;
                const CUtensorMap* mA = bt.maps + 2 * p;   // 128-row boxes
                int bm, bn;
                tile_of(lt, bm, bn);
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int s = it % kStages2;
                    const uint32_t ph = (it / kStages2) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
                    if (leader) mbar_arrive_expect_tx(&full[s], 4 * kABytes);   // both CTAs' A and B halves
                    const uint32_t bar = full_l + static_cast<uint32_t>(s * sizeof(uint64_t));
                    tma_load_2d_pair(sA + s * kABytes, mA, kb * kSc2BK, bm * kSc2BM, bar);
                    tma_load_2d_pair(sB + s * kABytes, mA, kb * kSc2BK, bn * kSc2BN + static_cast<int>(rank) * kSc2BM, bar);
                }
            }
            // tail: the leader's last releases of every stage have arrived here
            for (int q = 0; q < kStages2; ++q, ++it) {
                const int s = it % kStages2;
                const uint32_t ph = (it / kStages2) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- pair MMA issuer (leader) ----------------
            constexpr uint32_t kIdesc2 = idesc_f32acc(0u, 0u, 2 * kSc2BM, kSc2BN);   // M = 256, N = 256
            int it = 0, tc = 0;
            for (int u = u0; u < nu && ok; u += us, ++tc) {
                const int t = 2 * u;
                int lt;
                const int p = locate(bt, ST_GEMM, t, lt);
                const int KT = bt.views[p].n_pad / kSc2BK;
                const int buf = tc & 1;
                const uint32_t use = static_cast<uint32_t>(tc >> 1);
                if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(buf * kSc2BN);
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int s = it % kStages2;
                    const uint32_t ph = (it / kStages2) & 1u;
                    if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kABytes);
                    const uint32_t b0 = smem_u32(sB + s * kABytes);
#pragma unroll
                    for (int k = 0; k < kSc2BK / 32; ++k)
                        mma_f8f6f4_pair(d, sdesc_k_sw128(a0 + k * 32), sdesc_k_sw128(b0 + k * 32), kIdesc2,
                                        (kb | k) != 0 ? 1u : 0u);
                    mma_commit_pair_mc(&empty[s], 0x3);
                }
                if (!ok) break;
                mma_commit_pair_mc(&tfull[buf], 0x3);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps (both CTAs) ----------------
        const int quarter = warp & 3;
        const int part = (warp - 2) >> 2;
        int tc = 0;
        for (int u = u0; u < nu; u += us, ++tc) {
            const int t = 2 * u + static_cast<int>(rank);
            int lt;
            const int p = locate(bt, ST_GEMM, t, lt);
            const ProbView v = bt.views[p];
            int bm, bn;
            tile_of(lt, bm, bn);
            const int buf = tc & 1;
            const uint32_t use = static_cast<uint32_t>(tc >> 1);
            const uint2 words = epi_words(v, bm, bn, quarter, part, lane);
            // a batch: whether this CTA's next block belongs to another problem
            bool flush_after = false;
            if (kHist && u + us < nu) {
                int ltn;
                flush_after = locate(bt, ST_GEMM, 2 * (u + us) + static_cast<int>(rank), ltn) != p;
            }
            const bool got = mbar_wait(&tfull[buf], use & 1u);
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            tc_fence_after();
            sc2_epilogue_tile_staged<kHist>(v, tmem + static_cast<uint32_t>(buf * kSc2BN), bm, bn, quarter, part,
                                            lane, words, shist, stg + (warp - 2) * 128);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(tempty_l + static_cast<uint32_t>(buf * sizeof(uint64_t)));
            if (flush_after) {
                // the epilogue warps add this problem's bins to its global
                // histogram and clear them (a rendezvous before and after)
                const ProbView* vf = bt.views + p;
                const int nf = vf->n;
                uint32_t* hf = vf->hist;
                if (lane == 0) mbar_arrive(hsync);
                if (!__all_sync(0xffffffffu, mbar_wait(hsync, 0u))) { ok = false; break; }
                for (int b = (warp - 2) * 32 + lane + 1; b <= nf; b += 32 * kEpiWarps) {
                    const uint32_t h = shist[b];
                    if (h) {
                        atomicAdd(hf + b, h);
                        shist[b] = 0u;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(hsync);
                if (!__all_sync(0xffffffffu, mbar_wait(hsync, 1u))) { ok = false; break; }
            }
        }
    }
    if (!ok && lane == 0) atomicOr(&bt.views[0].ctl->err, TR_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    // the problem of this cluster's last block (both CTAs of a cluster take the
    // same blocks): its bins are still in shared memory
    int p_last = -1;
    if (u0 < nu) {
        int lt;
        p_last = locate(bt, ST_GEMM, 2 * (u0 + ((nu - 1 - u0) / us) * us), lt);
    }
    if (kHist && !leader && p_last >= 0) {
        // the peer's histogram into the leader's (distributed shared memory), so
        // that one CTA per cluster adds to the global bins
        const uint32_t lead_hist = mapa_shared(shist, 0);
        for (int b = threadIdx.x + 1; b < nbins; b += blockDim.x) {
            const uint32_t h = shist[b];
            if (h) red_add_cluster(lead_hist + 4u * static_cast<uint32_t>(b), h);
        }
    }
    cluster_sync_all();   // neither CTA exits or frees tensor memory while the other may still use it;
                          // orders the peer's additions before the leader's flush
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
    if (!kHist || !leader || p_last < 0) return;
    // the cluster's histogram into the global one, from which the count pass
    // (one problem) or the select launch (a batch) chooses the pivot threshold
    const ProbView vl = bt.views[p_last];
    for (int b = threadIdx.x + 1; b <= vl.n; b += blockDim.x)
        if (shist[b]) atomicAdd(&vl.hist[b], shist[b]);
}

int g_sc2_sms = 0;
int g_sc2_pair_clusters = 0;   // co-resident 2-CTA clusters of the pair kernels (0: use single CTAs)

// kHist: the blocks keep the edge-weight histogram in shared memory
// (hist_bins bins)
template <bool kHist>
cudaError_t launch_pair(const Batch& b, int total_tiles, size_t smem, int hist_bins, cudaStream_t s, int auto_mode)
{
    int grid = 2 * g_sc2_pair_clusters;
    if (grid > total_tiles) grid = total_tiles;   // total_tiles is even
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, sc2_pair_mma_kernel<kHist>, b, total_tiles, hist_bins, auto_mode);
}

}  // namespace

int device_sms() { return g_sc2_sms > 0 ? g_sc2_sms : 148; }

int sc2_pair_clusters() { return g_sc2_pair_clusters; }

cudaError_t sc2_tcgen05_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sc2_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sc2_tcgen05_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sc2_tcgen05_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPipeBytes + kBarBytes + 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sc2_pair_mma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sc2_pair_mma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBase2);
    if (e == cudaSuccess) {
        // how many 2-CTA clusters fit at once with the largest shared-memory request
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * 256);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmemMax;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, sc2_pair_mma_kernel<true>, &cfg) == cudaSuccess)
            g_sc2_pair_clusters = nc;
        else
            cudaGetLastError();   // no cluster support: the single-CTA kernel is used
    }
    return e;
}

// A single problem keeps its histogram in shared memory when it fits; a
// batch (or a very large problem) uses global atomics.
bool launch_sc2_tcgen05(const Batch& b, int total_tiles, int max_n, bool pair_mma, cudaStream_t s, bool auto_mode)
{
    const bool pair = pair_mma && g_sc2_pair_clusters > 0;
    const int sms = g_sc2_sms > 0 ? g_sc2_sms : 148;
    const int grid = total_tiles < sms ? total_tiles : sms;
    const size_t base = pair ? static_cast<size_t>(kBase2) : static_cast<size_t>(kPipeBytes + kBarBytes + 1024);
    const size_t hist = static_cast<size_t>(max_n + 1) * 4;
    const bool fits = base + hist <= static_cast<size_t>(kSmemMax);
    const bool single = b.num == 1 && fits;
    if (pair) {
        if (fits)
            launch_pair<true>(b, total_tiles, base + hist, max_n + 1, s, auto_mode ? 1 : 0);
        else
            launch_pair<false>(b, total_tiles, base, 0, s, auto_mode ? 1 : 0);
    } else if (single) {
        launch_pdl(sc2_tcgen05_kernel<true>, grid, kThreads, base + hist, s, b, total_tiles);
    } else {
        launch_pdl(sc2_tcgen05_kernel<false>, grid, kThreads, base, s, b, total_tiles);
    }
    return single;
}


}  // namespace tr
