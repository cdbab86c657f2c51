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
// Alternative (TURBOREG_FLAG_SC2_BITSET): the same integers from the
// adjacency bitset with AND + popcount on CUDA cores, one block per row.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kStages = 4;
constexpr int kABytes = kSc2BM * kSc2BK;   // 16 KB
constexpr int kBBytes = kSc2BN * kSc2BK;   // 32 KB
constexpr int kSmemBytes = kStages * (kABytes + kBBytes) + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t kTmemCols = 256;
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

__global__ void __launch_bounds__(128, 1)
sc2_tcgen05_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ProbView v)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int bm, bn;
    tile_of(blockIdx.x, bm, bn);
    const int m0 = bm * kSc2BM, n0 = bn * kSc2BN;
    const int KT = v.n_pad / kSc2BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        for (int it = 0; it < KT; ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u)) { ok = false; break; }
            mbar_arrive_expect_tx(&full[s], kABytes + kBBytes);
            tma_load_2d(sA + s * kABytes, &tmA, it * kSc2BK, m0, &full[s]);
            tma_load_2d(sB + s * kBBytes, &tmB, it * kSc2BK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        for (int it = 0; it < KT; ++it) {
            const int s = it % kStages;
            const uint32_t ph = (it / kStages) & 1u;
            if (!mbar_wait(&full[s], ph)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + s * kABytes);
            const uint32_t b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
            for (int k = 0; k < kSc2BK / 32; ++k) {
                // advance 32 bytes (K = 32 FP8 elements) inside the 128-byte swizzle row
                mma_f8f6f4(tmem, sdesc_k_sw128(a0 + k * 32), sdesc_k_sw128(b0 + k * 32), kIdesc,
                           (it | k) != 0 ? 1u : 0u);
            }
            mma_commit(&empty[s]);   // frees this stage when its MMAs are done
        }
        mma_commit(accf);            // accumulator complete
    }
    __syncwarp();

    // ---------------- epilogue (all 4 warps) ----------------
    if (!mbar_wait(accf, 0)) ok = false;
    if (!ok) {
        if (lane == 0) atomicOr(&v.ctl->err, TR_ERR_TIMEOUT);
    } else {
        tc_fence_after();
        const int row = m0 + warp * 32 + lane;
        const uint32_t* brow = v.bits + (size_t)row * v.ldb;
        uint16_t* wrow = v.w + (size_t)row * v.n_pad;
        int rsum = 0;
#pragma unroll 1
        for (int c = 0; c < kSc2BN / 32; ++c) {
            uint32_t acc[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c * 32, acc);
            tmem_ld_wait();
            const int col0 = n0 + c * 32;
            const uint32_t word = brow[col0 >> 5];
            int val[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int j = col0 + q;
                const bool keep = ((word >> q) & 1u) && (row < j);
                val[q] = keep ? static_cast<int>(__uint_as_float(acc[q])) : 0;
                rsum += val[q];
            }
            uint4* dst = reinterpret_cast<uint4*>(wrow + col0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 p;
                p.x = static_cast<uint32_t>(val[8 * q + 0]) | (static_cast<uint32_t>(val[8 * q + 1]) << 16);
                p.y = static_cast<uint32_t>(val[8 * q + 2]) | (static_cast<uint32_t>(val[8 * q + 3]) << 16);
                p.z = static_cast<uint32_t>(val[8 * q + 4]) | (static_cast<uint32_t>(val[8 * q + 5]) << 16);
                p.w = static_cast<uint32_t>(val[8 * q + 6]) | (static_cast<uint32_t>(val[8 * q + 7]) << 16);
                dst[q] = p;
            }
            // column sums over this warp's 32 rows: butterfly transpose-reduce,
            // afterwards lane l holds the sum of column col0 + l
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
        if (rsum != 0) atomicAdd(&v.rowscore[row], rsum);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// CUDA-core alternative: block per row i; W_ij = popc(row_i & row_j) for j > i with G_ij.
__global__ void __launch_bounds__(256) sc2_bitset_kernel(ProbView v)
{
    extern __shared__ uint32_t srow[];
    const int i = blockIdx.x;
    const uint32_t* bi = v.bits + (size_t)i * v.ldb;
    for (int q = threadIdx.x; q < v.ldb; q += blockDim.x) srow[q] = bi[q];
    __syncthreads();
    uint16_t* wrow = v.w + (size_t)i * v.n_pad;
    int rsum = 0;
    for (int j = threadIdx.x; j < v.n_pad; j += blockDim.x) {
        int c = 0;
        if (j > i && ((srow[j >> 5] >> (j & 31)) & 1u)) {
            const uint4* bj = reinterpret_cast<const uint4*>(v.bits + (size_t)j * v.ldb);
            const uint4* si = reinterpret_cast<const uint4*>(srow);
            for (int q = 0; q < v.ldb / 4; ++q) {
                const uint4 a = si[q], b = bj[q];
                c += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
            }
            if (c) atomicAdd(&v.rowscore[j], c);
        }
        wrow[j] = static_cast<uint16_t>(c);
        rsum += c;
    }
    // block reduce of the row sum
    __shared__ int red[32];
    for (int off = 16; off >= 1; off >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t) atomicAdd(&v.rowscore[i], t);
    }
}

}  // namespace

cudaError_t sc2_tcgen05_setup()
{
    return cudaFuncSetAttribute(sc2_tcgen05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

void launch_sc2_tcgen05(const ProbView& v, const CUtensorMap& tmA, const CUtensorMap& tmB, cudaStream_t s)
{
    const int nb = v.n_pad / kSc2BN;
    const int tiles = nb * (nb + 1);
    sc2_tcgen05_kernel<<<tiles, 128, kSmemBytes, s>>>(tmA, tmB, v);
}

void launch_sc2_bitset(const ProbView& v, cudaStream_t s)
{
    sc2_bitset_kernel<<<v.n_pad, 256, v.ldb * sizeof(uint32_t), s>>>(v);
}

}  // namespace tr
