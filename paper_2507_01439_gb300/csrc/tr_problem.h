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
    int32_t n;           // correspondences
    int32_t n_pad;       // n rounded up to 256 (GEMM tile multiple); leading dimension of a8 and w
    int32_t ldb;         // words per bitset row = n_pad / 32
    int32_t k1, k2;      // Eq. 4 / Eq. 7
    float tau;           // Eq. 1 threshold
    float theta;         // inlier threshold
    float kappa_fp64;    // FP64 Kabsch above this sigma1/sigma2
    float* pts;          // [6][n_pad]
    float* pts8;         // [n_pad][8] = (x0, x1, x2, y0, y1, y2, 0, 0)
    uint8_t* a8;         // [n_pad][n_pad] FP8 E4M3 0/1 adjacency
    uint32_t* bits;      // [n_pad][ldb] adjacency bitset
    uint16_t* w;         // [n_pad][n_pad] O2Graph weights (i < j only)
    int32_t* rowscore;   // [n_pad] SC^2 row sums
    int32_t* deg;        // [n_pad] degrees
    uint32_t* hist;      // [n_pad + 1] histogram of O2Graph edge weights
    int32_t* rowcnt;     // [n_pad] per-row count of edges with weight == alpha
    int32_t* rowpref;    // [n_pad] exclusive prefix of rowcnt
    int32_t* rowcnt_gt;  // [n_pad] per-row count of edges with weight > alpha
    int32_t* rowpref_gt; // [n_pad] exclusive prefix of rowcnt_gt
    uint64_t* cand;      // [K1_MAX] selected edge keys (weight << 32 | ~(i*n+j))
    int4* piv;           // [K1_MAX] pivots (i, j, w, 0) in Eq. 4 order
    int4* cliques;       // [K1_MAX*K2_MAX] (i, j, z, valid) in Alg. 2 order
    float* rt;           // [K1_MAX*K2_MAX][16] R, t, kappa, flags
    int32_t* inl;        // [K1_MAX*K2_MAX] inlier numbers
    int32_t* fp64_list;  // [K1_MAX*K2_MAX] hypotheses whose Kabsch needs FP64
    Ctl* ctl;            // device scalars
    turboreg_result* res;  // device result
};

// stage launchers (all asynchronous on `s`)
void launch_pack(const ProbView& v, const float* src, const float* dst, cudaStream_t s);
const void* pack_kernel_func();   // identifies the pack node inside a captured graph
void launch_compat(const ProbView& v, cudaStream_t s);
void launch_sc2_tcgen05(const ProbView& v, const CUtensorMap& tmA, const CUtensorMap& tmB, cudaStream_t s);
void launch_sc2_bitset(const ProbView& v, cudaStream_t s);
void launch_topk(const ProbView& v, cudaStream_t s);             // histogram pass + selection
void launch_topk_after_hist(const ProbView& v, cudaStream_t s);  // selection (histogram already built)
void launch_topk_after_select(const ProbView& v, cudaStream_t s);  // selection (alpha already chosen)
void launch_pgs(const ProbView& v, cudaStream_t s);
void launch_kabsch(const ProbView& v, cudaStream_t s);             // FP32 closed form, FP64 list
void launch_verify(const ProbView& v, cudaStream_t s);             // hypotheses with a valid FP32 Kabsch
void launch_kabsch_fp64_verify(const ProbView& v, cudaStream_t s); // FP64 list: Kabsch + verification
void launch_finalize(const ProbView& v, cudaStream_t s);

// set kernel attributes (dynamic shared memory limits) once per device
cudaError_t sc2_tcgen05_setup();
cudaError_t topk_setup();

constexpr int kSc2BM = 128;   // GEMM tile rows  (TMEM lanes)
constexpr int kSc2BN = 256;   // GEMM tile cols  (TMEM columns)
constexpr int kSc2BK = 128;   // K bytes per pipeline stage (one 128-byte swizzle row)

}  // namespace tr
