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
// Backward and Adam run on CUDA cores (FP32 arithmetic on the BF16 weights
// and activations the forward used).
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

// ---------------- training: backward and Adam (CUDA cores) ----------------

// Per sample: dz4 = (sigmoid(z4) - y) / m (mean binary cross-entropy), then
// dz3 = W4 dz4 * [h3 > 0], dz2 = W3^T dz3 * [h2 > 0], dz1 = W2^T dz2 * [h1 > 0].
constexpr int kBwdSmem = (64 * 128 * 2 + 64) * 4;

__global__ void __launch_bounds__(128) mlp_bwd_act_kernel(const float* z4, const float* label, int m,
                                                          const float* wbf, const __nv_bfloat16* h1,
                                                          const __nv_bfloat16* h2, const __nv_bfloat16* h3,
                                                          float* dz1, float* dz2, float* dz3, float* dz4,
                                                          float* loss)
{
    extern __shared__ float bsm[];
    float* sW3 = bsm;                  // [64][128]
    float* sW2t = bsm + 64 * 128;      // W2 transposed: [in 64][out 128]
    float* sW4 = bsm + 2 * 64 * 128;   // [64]
    __shared__ float sl[4];
    for (int q = threadIdx.x; q < 64 * 128; q += blockDim.x) {
        sW3[q] = wbf[kW3 + q];
        const int o = q / 64, i = q % 64;   // W2[o][i]
        sW2t[i * 128 + o] = wbf[kW2 + q];
    }
    for (int q = threadIdx.x; q < 64; q += blockDim.x) sW4[q] = wbf[kW4 + q];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (s < m) {
        const float z = z4[s], y = label[s];
        const float p = 1.f / (1.f + __expf(-z));
        // log(1 + e^-|z|) + max(z, 0) - y z
        l = log1pf(__expf(-fabsf(z))) + fmaxf(z, 0.f) - y * z;
        const float g4 = (p - y) / static_cast<float>(m);
        dz4[s] = g4;
        float d3[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
            d3[c] = __bfloat162float(h3[(size_t)s * 64 + c]) > 0.f ? sW4[c] * g4 : 0.f;
            dz3[(size_t)s * 64 + c] = d3[c];
        }
        for (int i = 0; i < 128; ++i) {
            float a = 0.f;
#pragma unroll
            for (int c = 0; c < 64; ++c) a = fmaf(sW3[c * 128 + i], d3[c], a);
            dz2[(size_t)s * 128 + i] = __bfloat162float(h2[(size_t)s * 128 + i]) > 0.f ? a : 0.f;
        }
        for (int i = 0; i < 64; ++i) {
            float a = 0.f;
            for (int o = 0; o < 128; ++o) a = fmaf(sW2t[i * 128 + o], dz2[(size_t)s * 128 + o], a);
            dz1[(size_t)s * 64 + i] = __bfloat162float(h1[(size_t)s * 64 + i]) > 0.f ? a : 0.f;
        }
    }
    for (int off = 16; off >= 1; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(loss, (sl[0] + sl[1] + sl[2] + sl[3]) / static_cast<float>(m));
}

// dW[o][i] += sum over a sample chunk of dz[s][o] * a[s][i]; db[o] += sum dz[s][o].
// Block: 16 x 16 output tile; grid.z splits the samples.
template <typename TA>
__global__ void __launch_bounds__(256) mlp_wgrad_kernel(const float* dz, int O, const TA* a, int I, int m,
                                                        int chunk, float* dW, float* db)
{
    __shared__ float sdz[64][17];
    __shared__ float sa[64][17];
    const int o0 = blockIdx.y * 16, i0 = blockIdx.x * 16;
    const int to = threadIdx.x / 16, ti = threadIdx.x % 16;
    const int s0 = blockIdx.z * chunk, s1 = min(m, s0 + chunk);
    float acc = 0.f, accb = 0.f;
    for (int sb = s0; sb < s1; sb += 64) {
        for (int q = threadIdx.x; q < 64 * 16; q += blockDim.x) {
            const int r = q / 16, c = q % 16, s = sb + r;
            sdz[r][c] = (s < s1 && o0 + c < O) ? dz[(size_t)s * O + o0 + c] : 0.f;
            float av = 0.f;
            if (s < s1 && i0 + c < I) {
                if constexpr (sizeof(TA) == 2) av = __bfloat162float(a[(size_t)s * I + i0 + c]);
                else av = __bfloat162float(__float2bfloat16_rn(static_cast<float>(a[(size_t)s * I + i0 + c])));
            }
            sa[r][c] = av;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 64; ++r) {
            acc = fmaf(sdz[r][to], sa[r][ti], acc);
            accb += sdz[r][to];
        }
        __syncthreads();
    }
    if (o0 + to < O && i0 + ti < I) atomicAdd(&dW[(o0 + to) * I + i0 + ti], acc);
    if (blockIdx.x == 0 && ti == 0 && o0 + to < O) atomicAdd(&db[o0 + to], accb);
}

// dW4[c] += sum dz4 h3[c]; db4 += sum dz4 (one block per 1024-sample chunk)
__global__ void __launch_bounds__(256) mlp_wgrad4_kernel(const float* dz4, const __nv_bfloat16* h3, int m,
                                                         float* g)
{
    __shared__ float acc[65];
    if (threadIdx.x < 65) acc[threadIdx.x] = 0.f;
    __syncthreads();
    const int s0 = blockIdx.x * 1024;
    for (int q = threadIdx.x; q < 1024 * 65; q += blockDim.x) {
        const int r = q / 65, c = q % 65, s = s0 + r;
        if (s >= m) continue;
        const float d = dz4[s];
        atomicAdd(&acc[c], c < 64 ? d * __bfloat162float(h3[(size_t)s * 64 + c]) : d);
    }
    __syncthreads();
    if (threadIdx.x < 64) atomicAdd(&g[kW4 + threadIdx.x], acc[threadIdx.x]);
    if (threadIdx.x == 64) atomicAdd(&g[kB4], acc[64]);
}

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
        e = cudaFuncSetAttribute(mlp_bwd_act_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
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
                         const __nv_bfloat16* h1, const __nv_bfloat16* h2, const __nv_bfloat16* h3, float* dz1,
                         float* dz2, float* dz3, float* dz4, float* grad, float* loss, cudaStream_t s)
{
    mlp_bwd_act_kernel<<<(m + 127) / 128, 128, kBwdSmem, s>>>(z4, label, m, wbf, h1, h2, h3, dz1, dz2, dz3, dz4,
                                                               loss);
    const int chunk = 4096;
    const int zc = (m + chunk - 1) / chunk;
    // layer 1: dW1 [64][8] from dz1 and the (BF16-rounded) features
    mlp_wgrad_kernel<float><<<dim3(1, 4, zc), 256, 0, s>>>(dz1, 64, feat, 8, m, chunk, grad + kW1, grad + kB1);
    mlp_wgrad_kernel<__nv_bfloat16><<<dim3(4, 8, zc), 256, 0, s>>>(dz2, 128, h1, 64, m, chunk, grad + kW2, grad + kB2);
    mlp_wgrad_kernel<__nv_bfloat16><<<dim3(8, 4, zc), 256, 0, s>>>(dz3, 64, h2, 128, m, chunk, grad + kW3, grad + kB3);
    mlp_wgrad4_kernel<<<(m + 1023) / 1024, 256, 0, s>>>(dz4, h3, m, grad);
}

void launch_mlp_adam(float* w, float* mom, float* vel, const float* g, float* wbf, int step, float lr,
                     cudaStream_t s)
{
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, mom, vel, g, wbf, step, lr, 0.9f, 0.999f, 1e-8f);
}

}  // namespace tr
