// Device view of one registration problem's workspace, passed by value to
// every stage kernel, and the host-side launchers of the stages.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "turboreg.h"

namespace tr {

struct Ctl;

// Points are kept structure-of-arrays: pts[c * n_pad + k] for c in
// {x0, x1, x2, y0, y1, y2}; padding entries are zero.
struct ProbView {
    int64_t in_off;      // first match of this problem in the (concatenated) input arrays
    int32_t n;           // correspondences
    int32_t n_pad;       // n rounded up to 256 (GEMM tile multiple); leading dimension of a8 and w
    int32_t ldb;         // words per bitset row = n_pad / 32
    int32_t k1, k2;      // Eq. 4 / Eq. 7
    float tau;           // Eq. 1 threshold
    float theta;         // inlier threshold
    float kappa_fp64;    // FP64 Kabsch above this sigma1/sigma2
    int32_t graph_mode;  // TURBOREG_GRAPH_O2 / _SC2: the graph the clique search runs on
    int32_t scoring;     // TURBOREG_SCORE_IN / _MAE / _MSE
    int32_t vppb;        // verification tile: matches per block (<= 4 x the kernel's points per warp)
    uint32_t dbg;        // failure injection for tests (TR_DBG_*), 0 in normal use
    uint8_t* a8_auto;    // non-null: the SC^2 path is chosen on the device from the degrees (one
                         // problem, n_pad <= 5120); a8 is then null, so the compatibility kernel
                         // writes the bitset only, and the FP8 matrix is expanded into a8_auto
                         // if the tensor-core GEMM is chosen
    float* pts;          // [6][n_pad]
    float* pts8;         // [n_pad][8] = (x0, x1, x2, y0, y1, y2, 0, 0)
    uint8_t* a8;         // [n_pad][n_pad] FP8 E4M3 0/1 adjacency
    uint32_t* bits;      // [n_pad][ldb] adjacency bitset
    uint16_t* w;         // [n_pad][n_pad] O2Graph weights (i < j only)
    int32_t* rowscore;   // [n_pad] SC^2 row sums
    int32_t* deg;        // [n_pad] degrees
    int32_t* rowmax;     // [n_pad] largest O2Graph weight of each row (j > i), or null: rows
                         // below the pivot threshold are skipped by the selection passes
    uint32_t* hist;      // [n_pad + 1] histogram of O2Graph edge weights
    int4* active;        // [n_pad] (row, #weight > alpha, #weight == alpha, 0) of the rows
                         // holding such edges, in any order
    uint64_t* cand;      // [K1_MAX] selected edge keys (weight << 32 | ~(i*n+j))
    int4* piv;           // [K1_MAX] pivots (i, j, w, 0) in Eq. 4 order
    int4* cliques;       // [K1_MAX*K2_MAX] (i, j, z, valid) in Alg. 2 order
    float* rt;           // [K1_MAX*K2_MAX][16] R, t, kappa, flags
    int32_t* inl;        // [K1_MAX*K2_MAX] inlier numbers
    uint32_t* hbits;     // [2][K1_MAX*K2_MAX/32] bit h of word h/32: hypothesis h valid, and
                         // (second half) solved with FP64 normals; written by verification
    unsigned long long* score;  // [K1_MAX*K2_MAX] capped error sums in units of 2^-22 theta (^2)
    float* feat;         // [n_pad][8] proposal features (learned proposal only)
    float* prob;         // [n_pad] inlier probabilities; non-null selects the learned pivot weight
    Ctl* ctl;            // device scalars
    turboreg_result* res;  // device result
};

// A group of problems processed by one launch per stage.  Stage k's blocks
// are numbered consecutively over the problems: problem p owns blocks
// [pre[k*(num+1) + p], pre[k*(num+1) + p + 1]).
enum Stage {
    ST_PACK = 0, ST_COMPAT, ST_SELECT, ST_COUNT, ST_SCAN, ST_EMIT, ST_RANK, ST_PGS, ST_KABSCH,
    ST_VERIFY, ST_FINAL, ST_HIST, ST_BITSET, ST_GEMM, ST_FEAT, ST_MLP, kNumBatchStages
};

// Blocks of the per-row count pass (eight row pairs per block) and of the
// emit pass (active rows strided over the blocks).
__host__ __device__ inline int count_blocks(int n) { return ((n + 1) / 2 + 7) / 8; }
__host__ __device__ inline int emit_blocks(int n) { return (n + 7) / 8; }

struct Batch {
    const ProbView* views;   // [num] device
    const int32_t* pre;      // [kNumBatchStages][num + 1] device
    const CUtensorMap* maps; // [num][2] device (A box 128 rows, B box 256 rows)
    int32_t num;
};

#ifdef __CUDACC__
// Problem owning block b of stage st, and the block's index within it.
__device__ __forceinline__ int locate(const Batch& bt, int st, int b, int& local)
{
    const int32_t* pr = bt.pre + st * (bt.num + 1);
    int lo = 0, hi = bt.num;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pr + mid) <= b) lo = mid;
        else hi = mid;
    }
    local = b - __ldg(pr + lo);
    return lo;
}

// Weight an edge competes with for a pivot slot (Eq. 4): the O2Graph weight,
// or with the learned proposal floor(W_ij p_i p_j) (the same integer range,
// so the exact integer top-K applies unchanged).
__device__ __forceinline__ int pivot_weight(const ProbView& v, int i, int j, int w)
{
    if (v.prob == nullptr || w == 0) return w;
    return static_cast<int>(__fmul_rn(__fmul_rn(static_cast<float>(w), v.prob[i]), v.prob[j]));
}

// Where a kernel finds its problem: one problem passed by value (the
// allocation-free selection on a caller's weight matrix, whose weights are
// checked against the range 0..n-2 of an SC^2 count) ...
struct OneView {
    static constexpr bool kCallerWeights = true;
    ProbView v;
    __device__ __forceinline__ ProbView get(int, int b, int& local) const
    {
        local = b;
        return v;
    }
};
// ... or a group of problems, located per block.
struct ManyViews {
    static constexpr bool kCallerWeights = false;   // weights come from the library's own SC^2 pass
    Batch bt;
    __device__ __forceinline__ ProbView get(int st, int b, int& local) const
    {
        return bt.views[locate(bt, st, b, local)];
    }
};
#endif

// per-problem block counts of each stage (host side, from n, k1, k2)
// vppb: matches per verification block (ProbView::vppb)
void stage_blocks(int32_t n, int32_t k1, int32_t k2, int32_t vppb, int32_t blocks[kNumBatchStages]);
// Matches per verification block for a single problem: the block count
// (hypothesis blocks x match blocks) close to 4 blocks per SM, so that one
// wave covers the problem with every SM holding the same number of blocks.
int32_t balanced_vppb(int32_t n, int32_t nh, int32_t num_sms);

// stage launchers (all asynchronous on `s`); total = sum of the stage's blocks
void launch_pack(const Batch& b, int total, const float* src, const float* dst, cudaStream_t s);
const void* pack_kernel_func();   // identifies the pack node inside a captured graph
void launch_compat(const Batch& b, int total, cudaStream_t s, bool auto_sc2 = false);
// pair_mma: 2-CTA clusters with pair MMAs (cta_group::2); otherwise
// independent CTAs.  Returns true when the GEMM completed one problem's
// weight histogram from shared memory, so that the count pass may choose the
// pivot threshold; otherwise the caller launches the select.
bool launch_sc2_tcgen05(const Batch& b, int total_tiles, int max_n, bool pair_mma, cudaStream_t s,
                        bool auto_mode = false);
// co-resident 2-CTA clusters of the pair-MMA GEMM (0: none)
int sc2_pair_clusters();
// SC^2 by AND + popcount over the bitset (sc2_bitset.cu); total = the batch's
// tiles (bitset_tiles per problem).  Returns true when every problem's
// edge-weight histogram is complete in global memory at its end (always).
bool launch_sc2_bitset(const Batch& b, int total_tiles, int max_n, int min_n, int auto_clusters, cudaStream_t s);
int bitset_tiles(int n_pad);
cudaError_t sc2_bitset_setup();
void launch_hist(const Batch& b, int total, int max_n, cudaStream_t s);
void launch_select(const Batch& b, cudaStream_t s);
// count and emit passes of the selection (the clique search ranks the pivots)
// select_here: the count blocks choose the threshold from the histogram the
// SC^2 GEMM completed (one problem of at most max_n matches)
void launch_count_emit(const Batch& b, const int32_t tot[kNumBatchStages], bool select_here, int max_n,
                       cudaStream_t s);
// The clique search also orders the pivots (each warp ranks its selected edge)
void launch_pgs(const Batch& b, int total, int k2_max, int max_k1, cudaStream_t s);
void launch_kabsch(const Batch& b, int total, cudaStream_t s);
// out: results of the launch's problems in order (page-locked host or device
// memory), or null for the workspace's result array
void launch_finalize(const Batch& b, turboreg_result* out, cudaStream_t s);
const void* finalize_kernel_func();
// Kabsch of caller-given k-cliques (k >= 4) into v.rt; idx [m][k] on the device.
void launch_kabsch_n(const ProbView& v, const int32_t* idx, int k, int m, cudaStream_t s);
// pw: the kernel's points per warp (32, 64, 128); every problem's vppb <= 4 pw
// capped: at most four blocks per SM (the balanced single-problem tile)
void launch_verify(const Batch& b, int total, int pw, bool capped, cudaStream_t s);

// set kernel attributes (dynamic shared memory limits) once per device
cudaError_t sc2_tcgen05_setup();
// SM count of the device (after sc2_tcgen05_setup)
int device_sms();
cudaError_t topk_setup();
// Shared-memory carveout of the verification and clique-search kernels: the
// largest shared part, so that every block of a launch is resident at once
cudaError_t verify_pgs_setup();

// single-problem pivot selection used by the allocation-free entry point
void launch_topk_single(const ProbView& v, cudaStream_t s);

constexpr int kSc2BM = 128;   // GEMM tile rows  (TMEM lanes)
constexpr int kSc2BN = 256;   // GEMM tile cols  (TMEM columns)
constexpr int kSc2BK = 128;   // K bytes per pipeline stage (one 128-byte swizzle row)
constexpr int kSc2AutoMaxNpad = 5120;   // the device-side choice of the SC^2 path: n_pad <= 5120
constexpr int kSc2BitsetAlwaysNpad = 2048;   // ... below which the CUDA-core path is taken directly

}  // namespace tr
