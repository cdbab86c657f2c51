// Stages 5-7: model estimation (Sec. 3.5, Eq. 9).
//
// kabsch:   per TurboClique h, the proper rotation R and translation t that
//           minimise sum_a ||R x_a + t - y_a||^2 over its 3 matches.
// verify:   IN(h) = #{k : ||R_h x_k + t_h - y_k||^2 <= theta^2}.
// finalize: h* = argmax IN (lowest h on ties) -> turboreg_result.
//
// The closed-form 3-point Kabsch itself is in tr_kabsch.cuh.
//
#include "tr_common.cuh"
#include "tr_kabsch.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

// Closed form for every hypothesis (used by the clique-Kabsch entry point; the
// registration path solves cliques inside the clique search).
__global__ void __launch_bounds__(128) kabsch_kernel(ManyViews vs)
{
    int lb;
    const ProbView v = vs.get(ST_KABSCH, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    const int h = lb * blockDim.x + threadIdx.x;
    const int nh = v.ctl->n_pivots * v.k2;
    if (h >= nh) return;
    kabsch_hypothesis(v, h, v.cliques[h]);
}

// Verification.  A block holds 128 hypotheses (R, t staged in shared memory)
// and 256 correspondences (as packed pairs (v, v), so a point feeds the
// packed arithmetic straight from shared memory); each of its 4 warps takes 64 of
// the correspondences for all 128 hypotheses, 4 per lane, evaluated as two
// packed pairs: e = R x + (t - y), d2 = |e|^2 with fma.rn.f32x2 (the same
// rounding as the scalar expression, two hypotheses per instruction).  The
// warps' counts are summed in shared memory; one atomic per hypothesis.
// Hypotheses whose Kabsch is valid (flags bit 1) are evaluated.
//
// Capped-error scores (MAE, MSE of the ranking study, Table 6): each match
// adds min(e, theta) or min(e^2, theta^2), rounded to an integer number of
// units of 2^-22 theta (theta^2).  Integer sums are independent of the order
// in which blocks add them, so a problem's scores do not depend on how the
// work was split (one problem or a batch).
// The points per warp of a block (PW, 32/64/128; the block then holds
// 4 PW points) are a tile-shape choice of the caller (TURBOREG_FLAG_VERIFY_*).
constexpr int kVWarps = 4;
constexpr int kVHyp = 128;
constexpr int kCapPerSm = 4;    // blocks per SM of the balanced single-problem tile
int g_cap_dyn[3] = {0, 0, 0};   // dynamic shared-memory padding for that cap (32, 64, 128 points per warp)
constexpr int kHypWords = TURBOREG_K1_MAX * TURBOREG_K2_MAX / 32;   // words of one flag-bit array
constexpr float kScoreUnits = 4194304.f;   // 2^22 units per theta (MAE) or theta^2 (MSE)

template <int PW>
struct VerifyShared {
    ulonglong2 sp[kVWarps * PW][3];   // points as packed pairs (v, v): x0 x1 | x2 y0 | y1 y2
    float srt[kVHyp][17];   // R, t of each hypothesis; 17 floats apart: lanes hit distinct banks
    int scnt[kVWarps][kVHyp];
    uint32_t ssc[kVWarps][kVHyp];
    int sok[kVHyp];
};

// Stages this block's matches as packed (v, v) pairs.  They were written by
// the first stage of the registration, so this runs before the wait for the
// clique search (whose hypotheses are staged after it).
template <int PW>
__device__ __forceinline__ void stage_matches(const ProbView& v, int lb, VerifyShared<PW>& sh)
{
    const int vppb = v.vppb;
    const int npb = (v.n + vppb - 1) / vppb;
    const int k0 = (lb % npb) * vppb;
    const int kn = min(vppb, v.n - k0);
    const float4* src = reinterpret_cast<const float4*>(v.pts8 + (size_t)k0 * 8);
    for (int q = threadIdx.x; q < kn; q += blockDim.x) {
        const float4 a = __ldcg(src + 2 * q), b = __ldcg(src + 2 * q + 1);   // from L2, past any stale L1 line
        auto dup = [](float f) {
            const unsigned long long u = __float_as_uint(f);
            return (u << 32) | u;
        };
        sh.sp[q][0] = make_ulonglong2(dup(a.x), dup(a.y));
        sh.sp[q][1] = make_ulonglong2(dup(a.z), dup(a.w));
        sh.sp[q][2] = make_ulonglong2(dup(b.x), dup(b.y));
    }
}

template <int kScore, int PW>
__device__ __forceinline__ void verify_body(const ProbView& v, int lb, VerifyShared<PW>& sh)
{
    const int vppb = v.vppb;                            // matches per block, <= kVWarps * PW
    const int npb = (v.n + vppb - 1) / vppb;            // match blocks of this problem
    const int h0 = (lb / npb) * kVHyp;
    const int slot = h0 + threadIdx.x;
    // this thread's hypothesis record, read in the same round as the pivot
    // count (slots up to K1 K2 are inside the buffer; those past the count
    // are ignored)
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
    if (slot < v.k1 * v.k2) {
        const float4* rt = reinterpret_cast<const float4*>(v.rt + (size_t)slot * 16);
        r0 = __ldcg(rt); r1 = __ldcg(rt + 1); r2 = __ldcg(rt + 2); r3 = __ldcg(rt + 3);
    }
    const int nh = v.ctl->n_pivots * v.k2;   // through L1: every warp of every block reads it
    if (h0 >= nh) return;
    const int k0 = (lb % npb) * vppb;
    const int kn = min(vppb, v.n - k0);                 // matches of this block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        bool ok = false;
        uint32_t flags = 0u;
        if (slot < nh) {
            flags = __float_as_uint(r3.y);
            ok = (flags & 1u) != 0u;
            if (!ok) r2.y = r2.z = r2.w = __int_as_float(0x7fc00000);   // NaN t: never an inlier
        } else {
            r2.y = r2.z = r2.w = __int_as_float(0x7fc00000);
        }
        float* d = sh.srt[threadIdx.x];
        d[0] = r0.x; d[1] = r0.y; d[2] = r0.z; d[3] = r0.w;
        d[4] = r1.x; d[5] = r1.y; d[6] = r1.z; d[7] = r1.w;
        d[8] = r2.x; d[9] = r2.y; d[10] = r2.z; d[11] = r2.w;
        sh.sok[threadIdx.x] = ok ? 1 : 0;
        // the tile's first match block records, one bit per hypothesis, which
        // are valid and which took the FP64 normals (read by the model selection)
        if (k0 == 0) {
            const uint32_t bv = __ballot_sync(0xffffffffu, ok);
            const uint32_t bf = __ballot_sync(0xffffffffu, (flags & 2u) != 0u);
            if (lane == 0) {
                v.hbits[(h0 >> 5) + warp] = bv;
                v.hbits[kHypWords + (h0 >> 5) + warp] = bf;
            }
        }
    }
    __syncthreads();
    // this lane's hypotheses: slots lane + 32 a, a = 0..3, as packed pairs (0,1), (2,3)
    f2 R[2][9], T[2][3];
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const float* A = sh.srt[lane + 64 * pr];
        const float* B = sh.srt[lane + 64 * pr + 32];
#pragma unroll
        for (int c = 0; c < 9; ++c) R[pr][c] = pk(A[c], B[c]);
#pragma unroll
        for (int c = 0; c < 3; ++c) T[pr][c] = pk(A[9 + c], B[9 + c]);
    }
    const float th = v.theta;
    const float th2 = th * th;
    // d2 <= th2 compared on the bit patterns: both are non-negative (a sum of
    // squares, a square), so the order is the integer order; NaN (an invalid
    // hypothesis) is above every finite threshold
    const uint32_t th2b = __float_as_uint(th2);
    const float qs = kScore == TURBOREG_SCORE_MAE ? kScoreUnits / th : kScoreUnits / th2;
    const int ppw = (vppb + kVWarps - 1) / kVWarps;     // matches per warp
    const int kb = warp * ppw;
    const int cnt = max(0, min(ppw, kn - kb));
    int in[4] = {0, 0, 0, 0};
    uint32_t sc[4] = {0u, 0u, 0u, 0u};
#pragma unroll 2
    for (int k = 0; k < cnt; ++k) {
        const ulonglong2 q0 = sh.sp[kb + k][0], q1 = sh.sp[kb + k][1], q2 = sh.sp[kb + k][2];
        const f2 X0{q0.x}, X1{q0.y}, X2{q1.x}, Y0{q1.y}, Y1{q2.x}, Y2{q2.y};
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const f2 e0 = fma2(R[pr][0], X0, fma2(R[pr][1], X1, fma2(R[pr][2], X2, sub2(T[pr][0], Y0))));
            const f2 e1 = fma2(R[pr][3], X0, fma2(R[pr][4], X1, fma2(R[pr][5], X2, sub2(T[pr][1], Y1))));
            const f2 e2 = fma2(R[pr][6], X0, fma2(R[pr][7], X1, fma2(R[pr][8], X2, sub2(T[pr][2], Y2))));
            const f2 d2 = fma2(e0, e0, fma2(e1, e1, mul2(e2, e2)));
            float lo, hi;
            upk(d2, lo, hi);
            in[2 * pr] += static_cast<int>((__float_as_uint(lo) - th2b - 1u) >> 31);
            in[2 * pr + 1] += static_cast<int>((__float_as_uint(hi) - th2b - 1u) >> 31);
            if (kScore == TURBOREG_SCORE_MAE) {
                // fminf(NaN, theta) = theta: an invalid hypothesis is never selected anyway
                sc[2 * pr] += __float2uint_rn(fminf(sqrtf(lo), th) * qs);
                sc[2 * pr + 1] += __float2uint_rn(fminf(sqrtf(hi), th) * qs);
            } else if (kScore == TURBOREG_SCORE_MSE) {
                sc[2 * pr] += __float2uint_rn(fminf(lo, th2) * qs);
                sc[2 * pr + 1] += __float2uint_rn(fminf(hi, th2) * qs);
            }
        }
    }
    sh.scnt[warp][lane] = in[0];
    sh.scnt[warp][lane + 32] = in[1];
    sh.scnt[warp][lane + 64] = in[2];
    sh.scnt[warp][lane + 96] = in[3];
    if (kScore != TURBOREG_SCORE_IN) {
        sh.ssc[warp][lane] = sc[0];
        sh.ssc[warp][lane + 32] = sc[1];
        sh.ssc[warp][lane + 64] = sc[2];
        sh.ssc[warp][lane + 96] = sc[3];
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (slot >= nh) return;
    const int hh = slot;
    const int tot = sh.scnt[0][t] + sh.scnt[1][t] + sh.scnt[2][t] + sh.scnt[3][t];
    if (tot) atomicAdd(&v.inl[hh], tot);
    if (kScore != TURBOREG_SCORE_IN && sh.sok[t]) {
        // per block at most 256 terms of <= 2^22 + 1 units: fits 32 bits
        const uint32_t s = sh.ssc[0][t] + sh.ssc[1][t] + sh.ssc[2][t] + sh.ssc[3][t];
        atomicAdd(&v.score[hh], static_cast<unsigned long long>(s));
    }
}

template <int PW>
__global__ void __launch_bounds__(128) verify_kernel(ManyViews vs)
{
    __shared__ __align__(16) VerifyShared<PW> sh;
    int lb;
    const ProbView v = vs.get(ST_VERIFY, blockIdx.x, lb);   // descriptors: uploaded before the first stage
    stage_matches(v, lb, sh);
    pdl_wait();
    pdl_release();
    switch (v.scoring) {      // uniform over the block: a block serves one problem
        case TURBOREG_SCORE_MAE: verify_body<TURBOREG_SCORE_MAE, PW>(v, lb, sh); break;
        case TURBOREG_SCORE_MSE: verify_body<TURBOREG_SCORE_MSE, PW>(v, lb, sh); break;
        default: verify_body<TURBOREG_SCORE_IN, PW>(v, lb, sh); break;
    }
}

// Selection key of hypothesis h (larger wins; distinct h give distinct keys,
// and ties of the score go to the lower h).  Inlier number: (IN + 1) << 32 |
// ~h.  Capped error: (2^40 - 1 - units) << 20 | (2^20 - 1 - h); the unit sum
// is at most N (2^22 + 1) < 2^38 and h < K1_MAX * K2_MAX = 2^17.
__device__ __forceinline__ unsigned long long select_key(int scoring, int inl, unsigned long long score, int h)
{
    if (scoring == TURBOREG_SCORE_IN)
        return (static_cast<unsigned long long>(static_cast<uint32_t>(inl) + 1u) << 32) |
               (0xFFFFFFFFull - static_cast<unsigned long long>(h));
    return ((0xFFFFFFFFFFull - score) << 20) | (0xFFFFFull - static_cast<unsigned long long>(h));
}

__device__ __forceinline__ int key_hypothesis(const ProbView& v, unsigned long long key)
{
    if (v.scoring == TURBOREG_SCORE_IN) return static_cast<int>(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
    return static_cast<int>(0xFFFFFull - (key & 0xFFFFFull));
}

// Model selection (Eq. 9), one block of 1024 threads per problem: h* = the
// largest selection key over the valid hypotheses, counts, and the result.
// One round of loads: the inlier numbers (and scores) of every slot up to
// K1 K2 and the verification's flag words, masked by the pivot count after.
// (Folding it into the last verification block was measured slower: the
// completion counter of ~1300 blocks on one address serialises in L2.)
__global__ void __launch_bounds__(1024) finalize_kernel(ManyViews vs, turboreg_result* out)
{
    int lb;
    const ProbView v = vs.get(ST_FINAL, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();
    __shared__ unsigned long long sbest[32];
    __shared__ int scnt[32], sfp[32];
    __shared__ float srec[16];
    __shared__ int4 scl;
    __shared__ int sinl;
    __shared__ unsigned long long sscore;
    const int hmax = v.k1 * v.k2;
    const int np = __ldcg(&v.ctl->n_pivots);
    unsigned long long best = 0ull;
    int nvalid = 0, nfp = 0;
    for (int h0 = threadIdx.x; h0 < hmax; h0 += 4 * blockDim.x) {
        uint32_t bv[4], bf[4];
        int in4[4];
        unsigned long long sc4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int h = h0 + u * blockDim.x;
            bv[u] = h < hmax ? __ldcg(v.hbits + (h >> 5)) : 0u;
            bf[u] = h < hmax ? __ldcg(v.hbits + kHypWords + (h >> 5)) : 0u;
            in4[u] = h < hmax ? __ldcg(v.inl + h) : 0;
            sc4[u] = (h < hmax && v.scoring != TURBOREG_SCORE_IN) ? __ldcg(v.score + h) : 0ull;
        }
        const int nh = np * v.k2;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int h = h0 + u * blockDim.x;
            const bool valid = h < nh && ((bv[u] >> (h & 31)) & 1u);
            const unsigned long long key = valid ? select_key(v.scoring, in4[u], sc4[u], h) : 0ull;
            nfp += (h < nh && ((bf[u] >> (h & 31)) & 1u)) ? 1 : 0;
            nvalid += valid ? 1 : 0;
            best = key > best ? key : best;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o > best ? o : best;
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, off);
        nfp += __shfl_xor_sync(0xffffffffu, nfp, off);
    }
    if (lane == 0) { sbest[warp] = best; scnt[warp] = nvalid; sfp[warp] = nfp; }
    __syncthreads();
    if (warp == 0) {
        const int nw = static_cast<int>(blockDim.x >> 5);
        best = lane < nw ? sbest[lane] : 0ull;
        nvalid = lane < nw ? scnt[lane] : 0;
        nfp = lane < nw ? sfp[lane] : 0;
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
            best = o > best ? o : best;
            nvalid += __shfl_xor_sync(0xffffffffu, nvalid, off);
            nfp += __shfl_xor_sync(0xffffffffu, nfp, off);
        }
        // second round: the winner's record, one load per lane
        if (best != 0ull) {
            const int h = key_hypothesis(v, best);
            if (lane < 16) srec[lane] = __ldcg(v.rt + (size_t)h * 16 + lane);
            else if (lane == 16) scl = v.cliques[h];
            else if (lane == 17) sinl = __ldcg(v.inl + h);
            else if (lane == 18 && v.scoring != TURBOREG_SCORE_IN) sscore = __ldcg(v.score + h);
        }
        if (lane == 0) { sbest[0] = best; scnt[0] = nvalid; sfp[0] = nfp; }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    best = sbest[0];
    nvalid = scnt[0];
    nfp = sfp[0];
    v.ctl->n_valid = nvalid;
    v.ctl->n_fp64 = nfp;
    turboreg_result r;
    for (int q = 0; q < 9; ++q) r.R[q] = (q % 4 == 0) ? 1.f : 0.f;
    r.t[0] = r.t[1] = r.t[2] = 0.f;
    r.clique[0] = r.clique[1] = r.clique[2] = -1;
    r.inlier_count = 0;
    r.score = 0.f;
    r.hypothesis = -1;
    r.n_pivots = np;
    r.n_valid = nvalid;
    r.used_fp64 = 0;
    r.used_fallback = 0;
    const uint32_t err = __ldcg(&v.ctl->err);
    if (err & TR_ERR_NONFINITE) {
        r.status = TURBOREG_ERR_NONFINITE;
    } else if (err & TR_ERR_TIMEOUT) {
        r.status = TURBOREG_ERR_TIMEOUT;
    } else if (err & TR_ERR_OVERFLOW) {
        r.status = TURBOREG_ERR_CUDA;
    } else if (best == 0ull) {
        r.status = TURBOREG_ERR_NO_HYPOTHESIS;
    } else {
        const int h = key_hypothesis(v, best);
        for (int q = 0; q < 9; ++q) r.R[q] = srec[q];
        for (int q = 0; q < 3; ++q) r.t[q] = srec[9 + q];
        r.clique[0] = scl.x; r.clique[1] = scl.y; r.clique[2] = scl.z;
        r.inlier_count = sinl;
        if (v.scoring == TURBOREG_SCORE_IN) {
            r.score = static_cast<float>(r.inlier_count);
        } else {
            const double unit = v.scoring == TURBOREG_SCORE_MAE ? (double)v.theta : (double)v.theta * v.theta;
            r.score = static_cast<float>((double)sscore * unit / (4194304.0 * v.n));
        }
        r.hypothesis = h;
        r.used_fp64 = (__float_as_uint(srec[13]) & 2u) ? 1 : 0;
        r.status = TURBOREG_OK;
    }
    // the caller's result array (page-locked host or device memory, one entry
    // per problem of the launch), or the workspace's
    if (out != nullptr) out[blockIdx.x] = r;
    else *v.res = r;
    // the next registration of this slot starts from cleared error bits and
    // counters (every other control field is written before it is read; the
    // pivot count stays readable for inspection)
    v.ctl->err = 0u;
    v.ctl->n_active = 0u;
    v.ctl->gt_slot = 0u;
    v.ctl->done_blocks = 0u;
    v.ctl->pmax_bits = 0u;
    v.ctl->deg_sum = 0u;
}

}  // namespace

void launch_finalize(const Batch& b, turboreg_result* out, cudaStream_t s)
{
    launch_pdl(finalize_kernel, b.num, 1024, 0, s, ManyViews{b}, out);
}

const void* finalize_kernel_func() { return reinterpret_cast<const void*>(&finalize_kernel); }

void launch_kabsch(const Batch& b, int total, cudaStream_t s)
{
    launch_pdl(kabsch_kernel, total, 128, 0, s, ManyViews{b});
}

cudaError_t verify_setup()
{
    cudaError_t e = cudaFuncSetAttribute(verify_kernel<32>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(verify_kernel<64>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(verify_kernel<128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // padding that leaves room for kCapPerSm blocks per SM and no more: the
    // balanced single-problem tile launches exactly kCapPerSm blocks per SM, and
    // its blocks become resident while the clique search still runs (early
    // launch); without the cap the first SMs to free up would take more than
    // their share
    int dev = 0, smem_sm = 0, reserved = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    const void* fns[3] = {reinterpret_cast<const void*>(&verify_kernel<32>),
                          reinterpret_cast<const void*>(&verify_kernel<64>),
                          reinterpret_cast<const void*>(&verify_kernel<128>)};
    for (int k = 0; k < 3; ++k) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, fns[k])) != cudaSuccess) return e;
        const int per_block = smem_sm / (kCapPerSm + 1) + 1;       // kCapPerSm + 1 blocks no longer fit
        int dyn = per_block - reserved - static_cast<int>(fa.sharedSizeBytes);
        dyn = dyn <= 0 ? 0 : (dyn + 1023) / 1024 * 1024;
        if (kCapPerSm * (static_cast<int>(fa.sharedSizeBytes) + dyn + reserved) > smem_sm) dyn = 0;
        if ((e = cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess)
            return e;
        g_cap_dyn[k] = dyn;
    }
    return cudaSuccess;
}

void launch_verify(const Batch& b, int total, int pw, bool capped, cudaStream_t s)
{
    const int k = pw == 32 ? 0 : pw == 128 ? 2 : 1;
    const size_t dyn = capped ? static_cast<size_t>(g_cap_dyn[k]) : 0;
    if (pw == 32) launch_pdl(verify_kernel<32>, total, 128, dyn, s, ManyViews{b});
    else if (pw == 128) launch_pdl(verify_kernel<128>, total, 128, dyn, s, ManyViews{b});
    else launch_pdl(verify_kernel<64>, total, 128, dyn, s, ManyViews{b});
}

// Per-problem block counts of every stage.
int32_t balanced_vppb(int32_t n, int32_t nh, int32_t num_sms)
{
    const int32_t nhb = (nh + kVHyp - 1) / kVHyp;
    const int32_t npb_min = (n + 4 * 128 - 1) / (4 * 128);             // capacity of the widest tile
    int32_t npb = nhb > 0 ? (kCapPerSm * num_sms) / nhb : npb_min;
    if (npb < npb_min) npb = npb_min;
    int32_t vppb = (n + npb - 1) / npb;
    vppb = (vppb + kVWarps - 1) / kVWarps * kVWarps;
    return vppb < 64 ? 64 : vppb;                                      // at least 16 matches per warp
}

void stage_blocks(int32_t n, int32_t k1, int32_t k2, int32_t vppb, int32_t blocks[kNumBatchStages])
{
    const int32_t vpts = vppb;
    const int32_t n_pad = (n + kSc2BN - 1) / kSc2BN * kSc2BN;
    const int32_t T = n_pad / 128;
    const int32_t nb = n_pad / kSc2BN;
    const int32_t nh = k1 * k2;
    blocks[ST_PACK] = n_pad / 256;
    blocks[ST_COMPAT] = T * (T + 1) / 2;
    blocks[ST_SELECT] = 1;
    blocks[ST_COUNT] = count_blocks(n);
    blocks[ST_SCAN] = 0;   // no separate row-scan pass
    blocks[ST_EMIT] = emit_blocks(n);
    blocks[ST_RANK] = (k1 + 31) / 32;
    blocks[ST_PGS] = (k1 + 7) / 8;
    blocks[ST_KABSCH] = (nh + 127) / 128;
    blocks[ST_VERIFY] = ((nh + kVHyp - 1) / kVHyp) * ((n + vpts - 1) / vpts);
    blocks[ST_FINAL] = 1;
    blocks[ST_HIST] = (n + 63) / 64;
    blocks[ST_BITSET] = bitset_tiles(n_pad);
    blocks[ST_GEMM] = nb * (nb + 1);
    blocks[ST_FEAT] = 1;
    blocks[ST_MLP] = (n + 127) / 128;
}

}  // namespace tr
