// Learned pivot proposal: a per-correspondence inlier-scoring MLP.
//
//   features f_i (8): (x_i - mean x) / rms_x (3), (y_i - mean y) / rms_y (3),
//                     degree_i / N, SC^2 row score_i / max_j row score_j
//   MLP 8 -> 64 -> 128 -> 64 -> 1, ReLU between layers, p_i = sigmoid(z4)
//   weights and activations in BF16, FP32 accumulation
//
// Parameter vector (FP32 master copy, 17217 values, row-major [out][in]):
//   W1[64][8] b1[64] W2[128][64] b2[128] W3[64][128] b3[64] W4[64] b4[1]
//
// Forward (inference and training): one CTA of 128 threads per 128 rows.
// Layer 1 (K = 8) and layer 4 (N = 1) run on CUDA cores; layers 2 and 3 run
// on the tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32 TMEM
// accumulators) with operands written to shared memory in the 128-byte
// swizzled K-major layout by the threads themselves.
// Backward: the activation gradients of layers 3 and 2 and the weight
// gradients of layers 2 and 3 on the tensor cores (BF16 operands, FP32
// accumulation, the weight gradients accumulated in tensor memory over a
// CTA's sample tiles); layers 1 and 4 and the biases on CUDA cores.  Adam on
// CUDA cores.
#include <cuda_bf16.h>

#include "tr_common.cuh"
#include "tr_problem.h"
#include "tr_mlp.h"

namespace tr {

namespace {

constexpr int kRows = 128;
// shared-memory layout of the forward kernel (offsets from a 1024-aligned base)
constexpr int kOffH1 = 0;                       // A of layer 2: 128 rows x 64 bf16
constexpr int kOffW2 = kOffH1 + 128 * 128;      // B of layer 2: 128 rows (out) x 64 bf16 (in)
constexpr int kOffH2 = kOffW2 + 128 * 128;      // A of layer 3: 2 K-blocks x 128 rows x 64 bf16
constexpr int kOffW3 = kOffH2 + 2 * 128 * 128;  // B of layer 3: 2 K-blocks x 64 rows x 64 bf16
constexpr int kOffSmall = kOffW3 + 2 * 64 * 128;
constexpr int kSmallFloats = 512 + 64 + 128 + 64 + 64 + 1;   // W1 b1 b2 b3 W4 b4
constexpr int kOffBar = kOffSmall + ((kSmallFloats * 4 + 127) / 128) * 128;
constexpr int kFwdSmem = kOffBar + 128 + 1024;
constexpr uint32_t kIdescL2 = idesc_f32acc(1u, 1u, 128, 128);   // BF16 x BF16 -> F32, M 128, N 128
constexpr uint32_t kIdescL3 = idesc_f32acc(1u, 1u, 128, 64);    // M 128, N 64

// byte offset of 16-byte chunk c of row r in a K-major 128-byte-swizzled tile
__device__ __forceinline__ int sw128(int r, int c) { return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float bf16r(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// act (optional, training): per row h1[64] h2[128] h3[64] (bf16) and z4 (f32)
struct FwdOut {
    float* prob;               // [m] sigmoid(z4) (may be null)
    float* z4;                 // [m] (may be null)
    __nv_bfloat16* h1;         // [m][64]  (may be null)
    __nv_bfloat16* h2;         // [m][128]
    __nv_bfloat16* h3;         // [m][64]
};

// Set-up of a forward CTA: the weights into shared memory (B operands in the
// swizzled layout), the mbarrier and 256 tensor-memory columns; returns the
// tensor-memory address.  All threads of the CTA call it.
__device__ uint32_t mlp_setup_cta(const float* __restrict__ wbf, uint8_t* smem)
{
    uint8_t* sW2 = smem + kOffW2;
    uint8_t* sW3 = smem + kOffW3;
    float* sW1 = reinterpret_cast<float*>(smem + kOffSmall);
    float* sb1 = sW1 + 512;
    float* sb2 = sb1 + 64;
    float* sb3 = sb2 + 128;
    float* sW4 = sb3 + 64;
    float* sb4 = sW4 + 64;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kOffBar + 16);
    const int t = threadIdx.x, warp = t >> 5;

    // weights (already BF16-rounded values stored as FP32) -> shared memory
    for (int q = t; q < 512; q += kRows) sW1[q] = wbf[kW1 + q];
    for (int q = t; q < 64; q += kRows) { sb1[q] = wbf[kB1 + q]; sb3[q] = wbf[kB3 + q]; sW4[q] = wbf[kW4 + q]; }
    for (int q = t; q < 128; q += kRows) sb2[q] = wbf[kB2 + q];
    if (t == 0) sb4[0] = wbf[kB4];
    {   // W2 row t (64 inputs) as B operand row t of layer 2
        const float* w = wbf + kW2 + t * 64;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            *reinterpret_cast<uint4*>(sW2 + sw128(t, c)) =
                make_uint4(pack_bf16(w[8 * c + 0], w[8 * c + 1]), pack_bf16(w[8 * c + 2], w[8 * c + 3]),
                           pack_bf16(w[8 * c + 4], w[8 * c + 5]), pack_bf16(w[8 * c + 6], w[8 * c + 7]));
    }
    if (t < 64) {   // W3 row t (128 inputs) as B operand row t of layer 3 (two K-blocks)
        const float* w = wbf + kW3 + t * 128;
#pragma unroll
        for (int c = 0; c < 16; ++c)
            *reinterpret_cast<uint4*>(sW3 + (c >> 3) * 8192 + sw128(t, c & 7)) =
                make_uint4(pack_bf16(w[8 * c + 0], w[8 * c + 1]), pack_bf16(w[8 * c + 2], w[8 * c + 3]),
                           pack_bf16(w[8 * c + 4], w[8 * c + 5]), pack_bf16(w[8 * c + 6], w[8 * c + 7]));
    }
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *tslot;
}

// One tile of 128 rows (row0 ..) after mlp_setup_cta: completes two phases of
// the CTA's mbarrier (parities 0 then 1), so tiles can follow one another.
// Returns this thread's probability (0 for rows past m).
__device__ float mlp_tile(const float* __restrict__ feat, int m, int row0, FwdOut out, uint8_t* smem, uint32_t tmem,
                          uint32_t* err)
{
    uint8_t* sH1 = smem + kOffH1;
    uint8_t* sW2 = smem + kOffW2;
    uint8_t* sH2 = smem + kOffH2;
    uint8_t* sW3 = smem + kOffW3;
    float* sW1 = reinterpret_cast<float*>(smem + kOffSmall);
    float* sb1 = sW1 + 512;
    float* sb2 = sb1 + 64;
    float* sb3 = sb2 + 128;
    float* sW4 = sb3 + 64;
    float* sb4 = sW4 + 64;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
    const int t = threadIdx.x, warp = t >> 5;

    // layer 1 on CUDA cores: row = t
    const int row = row0 + t;
    float f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = row < m ? bf16r(feat[(size_t)row * 8 + k]) : 0.f;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {   // 8 outputs of layer 1 per 16-byte chunk of the A operand
        float h8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int o = 8 * c + q;
            float z = sb1[o];
#pragma unroll
            for (int k = 0; k < 8; ++k) z = fmaf(sW1[o * 8 + k], f[k], z);
            h8[q] = fmaxf(z, 0.f);
        }
        *reinterpret_cast<uint4*>(sH1 + sw128(t, c)) =
            make_uint4(pack_bf16(h8[0], h8[1]), pack_bf16(h8[2], h8[3]), pack_bf16(h8[4], h8[5]),
                       pack_bf16(h8[6], h8[7]));
    }
    if (out.h1 && row < m) {
        uint4* d = reinterpret_cast<uint4*>(out.h1 + (size_t)row * 64);
#pragma unroll
        for (int c = 0; c < 8; ++c) d[c] = *reinterpret_cast<const uint4*>(sH1 + sw128(t, c));
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // layer 2 on the tensor cores: D[128 x 128] = H1[128 x 64] * W2^T
    if (t == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sH1), b0 = smem_u32(sW2);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)   // K = 16 BF16 (32 bytes) per MMA
            mma_f16(tmem, sdesc_k_sw128(a0 + ks * 32), sdesc_k_sw128(b0 + ks * 32), kIdescL2, ks > 0 ? 1u : 0u);
        mma_commit(bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, 0)) atomicOr(err, TR_ERR_TIMEOUT);
    tc_fence_after();
    // bias + ReLU, BF16, into the A operand of layer 3 (two K-blocks of 64)
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
        uint32_t acc[32];
        tmem_ld32(tmem + lane_base + cb * 32, acc);
        tmem_ld_wait();
        float hv[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) hv[q] = bf16r(fmaxf(__uint_as_float(acc[q]) + sb2[cb * 32 + q], 0.f));
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            const int k8 = cb * 4 + c4;   // 16-byte chunk index over the 128 inputs of layer 3
            *reinterpret_cast<uint4*>(sH2 + (k8 >> 3) * 16384 + sw128(t, k8 & 7)) =
                make_uint4(pack_bf16(hv[8 * c4 + 0], hv[8 * c4 + 1]), pack_bf16(hv[8 * c4 + 2], hv[8 * c4 + 3]),
                           pack_bf16(hv[8 * c4 + 4], hv[8 * c4 + 5]), pack_bf16(hv[8 * c4 + 6], hv[8 * c4 + 7]));
        }
        if (out.h2 && row < m) {
            uint4* d = reinterpret_cast<uint4*>(out.h2 + (size_t)row * 128 + cb * 32);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const int k8 = cb * 4 + c4;
                d[c4] = *reinterpret_cast<const uint4*>(sH2 + (k8 >> 3) * 16384 + sw128(t, k8 & 7));
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    // layer 3 on the tensor cores: D[128 x 64] = H2[128 x 128] * W3^T, TMEM columns 128..191
    if (t == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sH2), b0 = smem_u32(sW3);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_f16(tmem + 128, sdesc_k_sw128(a0 + kb * 16384 + ks * 32), sdesc_k_sw128(b0 + kb * 8192 + ks * 32),
                        kIdescL3, (kb | ks) != 0 ? 1u : 0u);
        mma_commit(bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, 1)) atomicOr(err, TR_ERR_TIMEOUT);
    tc_fence_after();
    float z4 = sb4[0];
#pragma unroll 1
    for (int cb = 0; cb < 2; ++cb) {
        uint32_t acc[32];
        tmem_ld32(tmem + lane_base + 128 + cb * 32, acc);
        tmem_ld_wait();
        float hv[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            hv[q] = bf16r(fmaxf(__uint_as_float(acc[q]) + sb3[cb * 32 + q], 0.f));
            z4 = fmaf(sW4[cb * 32 + q], hv[q], z4);
        }
        if (out.h3 && row < m) {
            uint4* d = reinterpret_cast<uint4*>(out.h3 + (size_t)row * 64 + cb * 32);
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4)
                d[c4] = make_uint4(pack_bf16(hv[8 * c4 + 0], hv[8 * c4 + 1]), pack_bf16(hv[8 * c4 + 2], hv[8 * c4 + 3]),
                                   pack_bf16(hv[8 * c4 + 4], hv[8 * c4 + 5]), pack_bf16(hv[8 * c4 + 6], hv[8 * c4 + 7]));
        }
    }
    float pr = 0.f;
    if (row < m) {
        pr = 1.f / (1.f + __expf(-z4));
        if (out.z4) out.z4[row] = z4;
        if (out.prob) out.prob[row] = pr;
    }
    // the tile's tensor-memory reads are complete before the next tile's MMAs
    tc_fence_before();
    __syncthreads();
    return pr;
}

__device__ void mlp_teardown_cta(uint32_t tmem)
{
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

__device__ void mlp_forward_tile(const float* __restrict__ feat, int m, int row0, const float* __restrict__ wbf,
                                 FwdOut out, uint8_t* smem, uint32_t* err)
{
    const uint32_t tmem = mlp_setup_cta(wbf, smem);
    mlp_tile(feat, m, row0, out, smem, tmem, err);
    mlp_teardown_cta(tmem);
}

__device__ __forceinline__ uint8_t* aligned_smem(uint8_t* raw)
{
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
}

// Standalone forward over an arbitrary feature array (training and tests).
__global__ void __launch_bounds__(kRows, 1) mlp_fwd_kernel(const float* feat, int m, const float* wbf, FwdOut out,
                                                           uint32_t* err)
{
    extern __shared__ uint8_t smem_raw[];
    mlp_forward_tile(feat, m, blockIdx.x * kRows, wbf, out, aligned_smem(smem_raw), err);
}

// Registration path: persistent CTAs (weights, mbarrier and tensor memory set
// up once, before the wait for the features) take the 128-row tiles of all
// problems in turn: rows of a problem's feature buffer -> its prob buffer,
// and the problem's largest probability into its control block (bounds of
// the learned pivot weights for the selection passes).
__global__ void __launch_bounds__(kRows, 2) mlp_proposal_kernel(Batch bt, int total, const float* wbf)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    const uint32_t tmem = mlp_setup_cta(wbf, smem);
    pdl_wait();
    pdl_release();
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        int lb;
        const ProbView v = bt.views[locate(bt, ST_MLP, tile, lb)];
        FwdOut out = {v.prob, nullptr, nullptr, nullptr, nullptr};
        float pm = mlp_tile(v.feat, v.n, lb * kRows, out, smem, tmem, &v.ctl->err);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, off));
        if ((threadIdx.x & 31) == 0 && pm > 0.f) atomicMax(&v.ctl->pmax_bits, __float_as_uint(pm));
    }
    mlp_teardown_cta(tmem);
}

// Features of one problem (one block of 1024 threads per problem).
__global__ void __launch_bounds__(1024) features_kernel(ManyViews vs)
{
    pdl_wait();
    pdl_release();
    __shared__ float red[32][8];
    __shared__ float tot[8];
    int lb;
    const ProbView v = vs.get(ST_FEAT, blockIdx.x, lb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // pass 1: sums of x, y and the largest row score
    float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = threadIdx.x; k < v.n; k += blockDim.x) {
        const float4* r = reinterpret_cast<const float4*>(v.pts8 + (size_t)k * 8);
        const float4 a = r[0], b = r[1];
        s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w; s[4] += b.x; s[5] += b.y;
        s[6] = fmaxf(s[6], static_cast<float>(v.rowscore[k]));
    }
    for (int q = 0; q < 7; ++q)
        for (int off = 16; off >= 1; off >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, s[q], off);
            s[q] = q == 6 ? fmaxf(s[q], o) : s[q] + o;
        }
    if (lane == 0)
        for (int q = 0; q < 7; ++q) red[warp][q] = s[q];
    __syncthreads();
    if (threadIdx.x < 7) {
        float a = threadIdx.x == 6 ? 0.f : 0.f;
        for (int w = 0; w < 32; ++w) a = threadIdx.x == 6 ? fmaxf(a, red[w][6]) : a + red[w][threadIdx.x];
        tot[threadIdx.x] = threadIdx.x == 6 ? a : a / static_cast<float>(v.n);
    }
    __syncthreads();
    // pass 2: mean squared distances to the centroids
    float d[2] = {0.f, 0.f};
    for (int k = threadIdx.x; k < v.n; k += blockDim.x) {
        const float4* r = reinterpret_cast<const float4*>(v.pts8 + (size_t)k * 8);
        const float4 a = r[0], b = r[1];
        const float ex = a.x - tot[0], ey = a.y - tot[1], ez = a.z - tot[2];
        const float fx = a.w - tot[3], fy = b.x - tot[4], fz = b.y - tot[5];
        d[0] += ex * ex + ey * ey + ez * ez;
        d[1] += fx * fx + fy * fy + fz * fz;
    }
    for (int q = 0; q < 2; ++q)
        for (int off = 16; off >= 1; off >>= 1) d[q] += __shfl_xor_sync(0xffffffffu, d[q], off);
    __syncthreads();
    if (lane == 0) { red[warp][0] = d[0]; red[warp][1] = d[1]; }
    __syncthreads();
    __shared__ float inv[2];
    if (threadIdx.x < 2) {
        float a = 0.f;
        for (int w = 0; w < 32; ++w) a += red[w][threadIdx.x];
        const float rms = sqrtf(a / static_cast<float>(v.n));
        inv[threadIdx.x] = rms > 0.f ? 1.f / rms : 0.f;
    }
    __syncthreads();
    const float invn = 1.f / static_cast<float>(v.n);
    const float invr = tot[6] > 0.f ? 1.f / tot[6] : 0.f;
    for (int k = threadIdx.x; k < v.n; k += blockDim.x) {
        const float4* r = reinterpret_cast<const float4*>(v.pts8 + (size_t)k * 8);
        const float4 a = r[0], b = r[1];
        float4* o = reinterpret_cast<float4*>(v.feat + (size_t)k * 8);
        o[0] = make_float4((a.x - tot[0]) * inv[0], (a.y - tot[1]) * inv[0], (a.z - tot[2]) * inv[0],
                           (a.w - tot[3]) * inv[1]);
        o[1] = make_float4((b.x - tot[4]) * inv[1], (b.y - tot[5]) * inv[1], static_cast<float>(v.deg[k]) * invn,
                           static_cast<float>(v.rowscore[k]) * invr);
    }
}

// ---------------- training: backward on the tensor cores ----------------
//
// Persistent CTAs of 128 threads take 128-sample tiles (thread t: sample
// row0 + t).  Per sample:
//   dz4 = (sigmoid(z4) - y) / m                  (mean binary cross-entropy)
//   dz3 = W4 dz4 * [h3 > 0]                      (CUDA cores)
//   dz2 = (dz3 W3) * [h2 > 0]                    MMA1: D1[128 x 128] = DZ3[128 x 64] W3
//   dz1 = (dz2 W2) * [h1 > 0]                    MMA2: D2[128 x 64] = DZ2[128 x 128] W2
// and the weight gradients, summed over the samples and kept in tensor memory
// over all tiles of the CTA:
//   dW3^T[128 in x 64 out] += H2^T[128 x 128 s] DZ3[128 s x 64]     MMA3 (G3)
//   dW2[128 out x 64 in]    += DZ2^T[128 x 128 s] H1[128 s x 64]     MMA4 (G2)
// dW1 = dz1^T x, dW4 = h3^T dz4 and the biases (sums of dz over the samples)
// on CUDA cores, in registers over the tiles.  The MMAs take BF16 operands (dz
// rounded to BF16; weights and activations are the forward's BF16 values) and
// accumulate in FP32; every operand is written by the threads into shared
// memory in the 128-byte swizzled K-major layout of the forward (transposed
// operands element by element), and every MMA has a shape of the forward's
// layers 2 and 3 (M 128, N 128 or 64, K 64 or 128).
constexpr int kBOffDz3 = 0;                      // A  MMA1: 128 samples x 64 (dz3)
constexpr int kBOffW3t = kBOffDz3 + 16384;       // B  MMA1: 128 (in3) x 64 (out3)
constexpr int kBOffDz2 = kBOffW3t + 16384;       // A  MMA2: 2 K-blocks x 128 samples x 64 (dz2)
constexpr int kBOffW2t = kBOffDz2 + 32768;       // B  MMA2: 2 K-blocks x 64 (in2) x 64 (out2)
constexpr int kBOffH2t = kBOffW2t + 16384;       // A  MMA3: 2 K-blocks x 128 (in3) x 64 samples
constexpr int kBOffDz3t = kBOffH2t + 32768;      // B  MMA3: 2 K-blocks x 64 (out3) x 64 samples
constexpr int kBOffDz2t = kBOffDz3t + 16384;     // A  MMA4: 2 K-blocks x 128 (out2) x 64 samples
constexpr int kBOffH1t = kBOffDz2t + 32768;      // B  MMA4: 2 K-blocks x 64 (in2) x 64 samples
constexpr int kBRedLd = 129;                     // FP32 [64][129] scratch (column sums over samples)
constexpr int kBOffRed = kBOffH1t + 16384;
constexpr int kBOffX = kBOffRed + 64 * kBRedLd * 4;   // FP32 [8][128] features of the tile
constexpr int kBOffG4 = kBOffX + 8 * 128 * 4;         // FP32 [128] dz4 of the tile
constexpr int kBOffW4 = kBOffG4 + 128 * 4;            // FP32 [64] W4
constexpr int kBOffLoss = kBOffW4 + 64 * 4;           // FP32 [4] per-warp loss
constexpr int kBOffBar = (kBOffLoss + 16 + 127) / 128 * 128;
constexpr int kBwdTcSmem = kBOffBar + 128 + 1024;
constexpr uint32_t kBwdTmemCols = 512;   // D1 0..127, D2 128..191, G3 192..255, G2 256..319

// element (row r, column k) of a K-major 128-byte-swizzled BF16 operand made
// of K-blocks of 64 columns, each `blk` bytes: byte offset
__device__ __forceinline__ int sw128_elem(int r, int k, int blk)
{
    return (k >> 6) * blk + sw128(r, (k & 63) >> 3) + (k & 7) * 2;
}

__device__ __forceinline__ void st_bf16(uint8_t* base, int off, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// sum over the 128 samples of row r of a transposed operand (2 K-blocks of blk bytes)
__device__ __forceinline__ float sum_row_bf16(const uint8_t* base, int r, int blk)
{
    float s = 0.f;
#pragma unroll
    for (int c16 = 0; c16 < 16; ++c16) {
        const uint4 q = *reinterpret_cast<const uint4*>(base + (c16 >> 3) * blk + sw128(r, c16 & 7));
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            s += __uint_as_float(w[e] << 16);
            s += __uint_as_float(w[e] & 0xFFFF0000u);
        }
    }
    return s;
}

__global__ void __launch_bounds__(kRows, 1)
    mlp_bwd_kernel(const float* feat, const float* label, int m, const float* wbf, const float* z4,
                   const __nv_bfloat16* h1, const __nv_bfloat16* h2, const __nv_bfloat16* h3, float* grad,
                   float* loss, uint32_t* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = aligned_smem(smem_raw);
    uint8_t* sDz3 = smem + kBOffDz3;
    uint8_t* sW3t = smem + kBOffW3t;
    uint8_t* sDz2 = smem + kBOffDz2;
    uint8_t* sW2t = smem + kBOffW2t;
    uint8_t* sH2t = smem + kBOffH2t;
    uint8_t* sDz3t = smem + kBOffDz3t;
    uint8_t* sDz2t = smem + kBOffDz2t;
    uint8_t* sH1t = smem + kBOffH1t;
    float* sRed = reinterpret_cast<float*>(smem + kBOffRed);
    float* sX = reinterpret_cast<float*>(smem + kBOffX);
    float* sG4 = reinterpret_cast<float*>(smem + kBOffG4);
    float* sW4 = reinterpret_cast<float*>(smem + kBOffW4);
    float* sLoss = reinterpret_cast<float*>(smem + kBOffLoss);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kBOffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kBOffBar + 16);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ntiles = (m + kRows - 1) / kRows;
    if (static_cast<int>(blockIdx.x) >= ntiles) return;

    // weights: W3^T (B of MMA1: row n = input of layer 3, K = its 64 outputs) and
    // W2^T (B of MMA2: row n = input of layer 2, K = its 128 outputs), W4
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float w8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w8[q] = wbf[kW3 + (8 * c + q) * 128 + t];
        *reinterpret_cast<uint4*>(sW3t + sw128(t, c)) =
            make_uint4(pack_bf16(w8[0], w8[1]), pack_bf16(w8[2], w8[3]), pack_bf16(w8[4], w8[5]),
                       pack_bf16(w8[6], w8[7]));
    }
    if (t < 64) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float w8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) w8[q] = wbf[kW2 + (8 * c + q) * 64 + t];
            *reinterpret_cast<uint4*>(sW2t + (c >> 3) * 8192 + sw128(t, c & 7)) =
                make_uint4(pack_bf16(w8[0], w8[1]), pack_bf16(w8[2], w8[3]), pack_bf16(w8[4], w8[5]),
                           pack_bf16(w8[6], w8[7]));
        }
        sW4[t] = wbf[kW4 + t];
    }
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, kBwdTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
    const float inv_m = 1.f / static_cast<float>(m);

    // per-thread gradient sums over the tiles: dW1 row o = t & 63, inputs
    // 4 (t >> 6) .. +3 and (t < 64) b1[o]; b2[t]; t < 64: b3[t]; t >= 64: W4[t - 64], b4
    const int o1 = t & 63, k1 = 4 * (t >> 6);
    float gW1[4] = {0.f, 0.f, 0.f, 0.f};
    float gb1 = 0.f, gb2 = 0.f, gb3w4 = 0.f, gb4 = 0.f, lsum = 0.f;
    bool first = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int s = tile * kRows + t;
        const bool valid = s < m;
        // ---- sample t: dz4, dz3, masks; operands of MMA1 and MMA3 ----
#pragma unroll
        for (int k = 0; k < 8; ++k) sX[k * 128 + t] = valid ? bf16r(feat[(size_t)s * 8 + k]) : 0.f;
        float g4 = 0.f;
        if (valid) {
            const float z = z4[s], y = label[s];
            const float p = 1.f / (1.f + __expf(-z));
            lsum += log1pf(__expf(-fabsf(z))) + fmaxf(z, 0.f) - y * z;
            g4 = (p - y) * inv_m;
        }
        sG4[t] = g4;
        const uint4* h3r = reinterpret_cast<const uint4*>(h3 + (size_t)(valid ? s : 0) * 64);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint4 q = valid ? h3r[c] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
            float d8[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float hv = __uint_as_float(e & 1 ? (w[e >> 1] & 0xFFFF0000u) : (w[e >> 1] << 16));
                const int col = 8 * c + e;
                d8[e] = bf16r(hv > 0.f ? sW4[col] * g4 : 0.f);
                sRed[col * kBRedLd + t] = g4 * hv;                       // for dW4
                st_bf16(sDz3t, sw128_elem(col, t, 8192), d8[e]);         // B of MMA3: row out3, column sample
            }
            *reinterpret_cast<uint4*>(sDz3 + sw128(t, c)) =
                make_uint4(pack_bf16(d8[0], d8[1]), pack_bf16(d8[2], d8[3]), pack_bf16(d8[4], d8[5]),
                           pack_bf16(d8[6], d8[7]));
        }
        uint32_t mask2[4] = {0u, 0u, 0u, 0u}, mask1[2] = {0u, 0u};
        const uint4* h2r = reinterpret_cast<const uint4*>(h2 + (size_t)(valid ? s : 0) * 128);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const uint4 q = valid ? h2r[c] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint16_t hb = static_cast<uint16_t>(e & 1 ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xFFFFu));
                const int col = 8 * c + e;
                mask2[col >> 5] |= (hb != 0 && !(hb & 0x8000u) ? 1u : 0u) << (col & 31);   // h2 > 0
                *reinterpret_cast<uint16_t*>(sH2t + sw128_elem(col, t, 16384)) = hb;     // A of MMA3
            }
        }
        const uint4* h1r = reinterpret_cast<const uint4*>(h1 + (size_t)(valid ? s : 0) * 64);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint4 q = valid ? h1r[c] : make_uint4(0u, 0u, 0u, 0u);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint16_t hb = static_cast<uint16_t>(e & 1 ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xFFFFu));
                const int col = 8 * c + e;
                mask1[col >> 5] |= (hb != 0 && !(hb & 0x8000u) ? 1u : 0u) << (col & 31);   // h1 > 0
                *reinterpret_cast<uint16_t*>(sH1t + sw128_elem(col, t, 8192)) = hb;      // B of MMA4
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // MMA1 (D1 = DZ3 W3) and MMA3 (G3 += H2^T DZ3)
        if (t == 0) {
            tc_fence_after();
            const uint32_t a1 = smem_u32(sDz3), b1 = smem_u32(sW3t);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_f16(tmem, sdesc_k_sw128(a1 + ks * 32), sdesc_k_sw128(b1 + ks * 32), kIdescL2, ks > 0 ? 1u : 0u);
            const uint32_t a3 = smem_u32(sH2t), b3 = smem_u32(sDz3t);
#pragma unroll
            for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_f16(tmem + 192, sdesc_k_sw128(a3 + kb * 16384 + ks * 32),
                            sdesc_k_sw128(b3 + kb * 8192 + ks * 32), kIdescL3, (first && kb == 0 && ks == 0) ? 0u : 1u);
            mma_commit(bar);
        }
        __syncwarp();
        // meanwhile: dW4, b4, b3 column sums of this tile
        if (t < 64) {
            gb3w4 += sum_row_bf16(sDz3t, t, 8192);
        } else {
            const float* r = sRed + (t - 64) * kBRedLd;
            float a = 0.f;
            for (int u = 0; u < 128; ++u) a += r[u];
            gb3w4 += a;
            if (t == 64)
                for (int u = 0; u < 128; ++u) gb4 += sG4[u];
        }
        if (!mbar_wait(bar, 0)) atomicOr(err, TR_ERR_TIMEOUT);
        tc_fence_after();
        // ---- dz2 = D1 * [h2 > 0]: A of MMA2 (row = sample) and A of MMA4 (row = output of layer 2) ----
#pragma unroll 1
        for (int cb = 0; cb < 4; ++cb) {
            uint32_t acc[32];
            tmem_ld32(tmem + lane_base + cb * 32, acc);
            tmem_ld_wait();
            const uint32_t mk = cb == 0 ? mask2[0] : cb == 1 ? mask2[1] : cb == 2 ? mask2[2] : mask2[3];
            float dv[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = cb * 32 + q;
                dv[q] = bf16r((mk >> q) & 1u ? __uint_as_float(acc[q]) : 0.f);
                st_bf16(sDz2t, sw128_elem(col, t, 16384), dv[q]);
            }
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const int k8 = cb * 4 + c4;   // 16-byte chunk over the 128 outputs of layer 2
                *reinterpret_cast<uint4*>(sDz2 + (k8 >> 3) * 16384 + sw128(t, k8 & 7)) =
                    make_uint4(pack_bf16(dv[8 * c4 + 0], dv[8 * c4 + 1]), pack_bf16(dv[8 * c4 + 2], dv[8 * c4 + 3]),
                               pack_bf16(dv[8 * c4 + 4], dv[8 * c4 + 5]), pack_bf16(dv[8 * c4 + 6], dv[8 * c4 + 7]));
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        // MMA2 (D2 = DZ2 W2) and MMA4 (G2 += DZ2^T H1)
        if (t == 0) {
            tc_fence_after();
            const uint32_t a2 = smem_u32(sDz2), b2 = smem_u32(sW2t);
            const uint32_t a4 = smem_u32(sDz2t), b4 = smem_u32(sH1t);
#pragma unroll
            for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_f16(tmem + 128, sdesc_k_sw128(a2 + kb * 16384 + ks * 32),
                            sdesc_k_sw128(b2 + kb * 8192 + ks * 32), kIdescL3, (kb | ks) != 0 ? 1u : 0u);
#pragma unroll
            for (int kb = 0; kb < 2; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    mma_f16(tmem + 256, sdesc_k_sw128(a4 + kb * 16384 + ks * 32),
                            sdesc_k_sw128(b4 + kb * 8192 + ks * 32), kIdescL3, (first && kb == 0 && ks == 0) ? 0u : 1u);
            mma_commit(bar);
        }
        __syncwarp();
        gb2 += sum_row_bf16(sDz2t, t, 16384);   // b2: the 128 samples of output t of layer 2
        if (!mbar_wait(bar, 1)) atomicOr(err, TR_ERR_TIMEOUT);
        tc_fence_after();
        // ---- dz1 = D2 * [h1 > 0] (FP32) -> dW1, b1 on CUDA cores ----
#pragma unroll 1
        for (int cb = 0; cb < 2; ++cb) {
            uint32_t acc[32];
            tmem_ld32(tmem + lane_base + 128 + cb * 32, acc);
            tmem_ld_wait();
            const uint32_t mk = cb == 0 ? mask1[0] : mask1[1];
#pragma unroll
            for (int q = 0; q < 32; ++q)
                sRed[(cb * 32 + q) * kBRedLd + t] = (mk >> q) & 1u ? __uint_as_float(acc[q]) : 0.f;
        }
        tc_fence_before();
        __syncthreads();   // sRed holds dz1 (rows: outputs of layer 1); tensor memory D1, D2 read
        {
            const float* r = sRed + o1 * kBRedLd;
            for (int u = 0; u < 128; ++u) {
                const float a = r[u];
                if (t < 64) gb1 += a;
#pragma unroll
                for (int k = 0; k < 4; ++k) gW1[k] = fmaf(a, sX[(k1 + k) * 128 + u], gW1[k]);
            }
        }
        __syncthreads();   // the tile's shared operands and scratch are consumed
        first = false;
    }
    // ---- the CTA's sums into the global gradient ----
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&grad[kW1 + o1 * 8 + k1 + k], gW1[k]);
    if (t < 64) {
        atomicAdd(&grad[kB1 + t], gb1);
        atomicAdd(&grad[kB3 + t], gb3w4);
    } else {
        atomicAdd(&grad[kW4 + t - 64], gb3w4);
        if (t == 64) atomicAdd(&grad[kB4], gb4);
    }
    atomicAdd(&grad[kB2 + t], gb2);
    tc_fence_after();
#pragma unroll 1
    for (int cb = 0; cb < 2; ++cb) {
        uint32_t g3[32], g2[32];
        tmem_ld32(tmem + lane_base + 192 + cb * 32, g3);   // dW3[out = column][in = t]
        tmem_ld32(tmem + lane_base + 256 + cb * 32, g2);   // dW2[out = t][in = column]
        tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            atomicAdd(&grad[kW3 + (cb * 32 + q) * 128 + t], __uint_as_float(g3[q]));
            atomicAdd(&grad[kW2 + t * 64 + cb * 32 + q], __uint_as_float(g2[q]));
        }
    }
    for (int off = 16; off >= 1; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if (lane == 0) sLoss[warp] = lsum;
    tc_fence_before();
    __syncthreads();
    if (t == 0) atomicAdd(loss, (sLoss[0] + sLoss[1] + sLoss[2] + sLoss[3]) * inv_m);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kBwdTmemCols);
    }
}

// ---------------- training: Adam (CUDA cores) ----------------

// Adam (bias-corrected), FP32 master weights; the forward's BF16-rounded copy
// is refreshed from them.
__global__ void __launch_bounds__(256) mlp_adam_kernel(float* w, float* mom, float* vel, const float* g, float* wbf,
                                                       int step, float lr, float b1, float b2, float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpParams) return;
    const float gk = g[k];
    const float m1 = b1 * mom[k] + (1.f - b1) * gk;
    const float v1 = b2 * vel[k] + (1.f - b2) * gk * gk;
    mom[k] = m1;
    vel[k] = v1;
    const float mh = m1 / (1.f - powf(b1, static_cast<float>(step)));
    const float vh = v1 / (1.f - powf(b2, static_cast<float>(step)));
    const float nw = w[k] - lr * mh / (sqrtf(vh) + eps);
    w[k] = nw;
    wbf[k] = bf16r(nw);
}

__global__ void __launch_bounds__(256) mlp_round_kernel(const float* w, float* wbf)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kMlpParams) wbf[k] = bf16r(w[k]);
}

}  // namespace

cudaError_t mlp_setup()
{
    cudaError_t e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_proposal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdTcSmem);
    return e;
}

void launch_mlp_round(const float* w, float* wbf, cudaStream_t s)
{
    mlp_round_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, wbf);
}

void launch_features(const Batch& b, cudaStream_t s) { launch_pdl(features_kernel, b.num, 1024, 0, s, ManyViews{b}); }

void launch_mlp_proposal(const Batch& b, int total, const float* wbf, cudaStream_t s)
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = total < 2 * sms ? total : 2 * sms;
    launch_pdl(mlp_proposal_kernel, grid, kRows, kFwdSmem, s, b, total, wbf);
}

void launch_mlp_forward(const float* feat, int m, const float* wbf, float* prob, float* z4, __nv_bfloat16* h1,
                        __nv_bfloat16* h2, __nv_bfloat16* h3, uint32_t* err, cudaStream_t s)
{
    FwdOut out = {prob, z4, h1, h2, h3};
    mlp_fwd_kernel<<<(m + kRows - 1) / kRows, kRows, kFwdSmem, s>>>(feat, m, wbf, out, err);
}

void launch_mlp_backward(const float* feat, const float* label, int m, const float* wbf, const float* z4,
                         const __nv_bfloat16* h1, const __nv_bfloat16* h2, const __nv_bfloat16* h3, float* grad,
                         float* loss, uint32_t* err, cudaStream_t s)
{
    const int ntiles = (m + kRows - 1) / kRows;
    const int sms = device_sms();
    const int grid = ntiles < sms ? ntiles : sms;   // one CTA per SM (shared memory and tensor memory)
    mlp_bwd_kernel<<<grid, kRows, kBwdTcSmem, s>>>(feat, label, m, wbf, z4, h1, h2, h3, grad, loss, err);
}

void launch_mlp_adam(float* w, float* mom, float* vel, const float* g, float* wbf, int step, float lr,
                     cudaStream_t s)
{
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, mom, vel, g, wbf, step, lr, 0.9f, 0.999f, 1e-8f);
}

}  // namespace tr
