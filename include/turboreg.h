/*
 * turboreg.h -- C ABI of the GB300 (sm_103a) TurboReg registration library.
 *
 * Robust point-cloud registration from putative correspondences, following
 * TurboReg (ICCV 2025): compatibility graph (Eq. 1), SC^2 graph (Eq. 2),
 * O2Graph (Def. 2), Pivot-Guided Search for TurboCliques (Eq. 4-7, Alg. 1,
 * Alg. 2), a Kabsch transform per TurboClique and selection of the
 * transform with the largest inlier number (Sec. 3.5, Eq. 9).
 *
 * Problem (Sec. 3.1, App. A.1): N matches m_i = (x_i, y_i), x_i, y_i in R^3,
 * with y_i = R x_i + t + r_i for inliers.  The library returns (R, t) in SE(3).
 *
 * Conventions shared by every entry point
 *  - Points are float32, row-major [N][3] (x, y, z of match i at 3*i).
 *  - Input pointers may be host or device memory; the kind is detected with
 *    cudaPointerGetAttributes.  Device pointers must be readable from the
 *    context's device and stay valid until the call returns.  Page-locked
 *    host inputs mapped into the device's address space are read in place by
 *    the first kernel (over the CPU-GPU link); other host inputs are copied to
 *    the device inside the call.
 *  - The caller owns every input and output buffer.  The library never keeps
 *    a pointer to caller memory after a call returns.
 *  - Every call is synchronous with respect to the host: it enqueues its work
 *    on the context's stream and waits for it before returning.
 *  - A context is not thread-safe.  Use one context per host thread / stream.
 *  - Return values are turboreg_status codes.  Invalid arguments are rejected
 *    before any device work is enqueued; the context is then unchanged.
 */
#ifndef TURBOREG_H
#define TURBOREG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TURBOREG_ABI_VERSION 1

/* Limits of one context (compile-time). */
#define TURBOREG_MAX_N 32768   /* correspondences per problem */
#define TURBOREG_K1_MAX 8192   /* pivots, Eq. 4 */
#define TURBOREG_K2_MAX 16     /* TurboCliques per pivot, Eq. 7 */

typedef struct turboreg_ctx turboreg_ctx;   /* opaque; owns the device workspace */

typedef enum {
    TURBOREG_OK = 0,
    TURBOREG_ERR_INVALID_ARG = 1,   /* null pointer, N > max_n, K out of range, tau < 0, theta <= 0 */
    TURBOREG_ERR_TOO_FEW = 2,       /* N < 3: no TurboClique can exist */
    TURBOREG_ERR_NONFINITE = 3,     /* a NaN or Inf coordinate */
    TURBOREG_ERR_OOM = 4,           /* device or pinned-host allocation failed */
    TURBOREG_ERR_CUDA = 5,          /* a CUDA runtime error (the context should be destroyed) */
    TURBOREG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    TURBOREG_ERR_NO_HYPOTHESIS = 7  /* no edge, no TurboClique or no non-degenerate Kabsch */
} turboreg_status;

/* graph_mode: the graph G- that Pivot-Guided Search runs on (Alg. 1 accepts either) */
#define TURBOREG_GRAPH_O2 0          /* O2Graph (Def. 2), the paper's default: the third match z of
                                        pivot (i, j) ranges over z > j, so every TurboClique is
                                        found by at most one pivot (App. C) */
#define TURBOREG_GRAPH_SC2 1         /* undirected SC^2 graph (Eq. 2): z ranges over every common
                                        neighbour of i and j, so a 3-clique can be found from up
                                        to three pivots (the ablation of Table 5) */
/* scoring: how the winning hypothesis is chosen (Eq. 9 and the ranking study of Table 6).
   e_k = ||R x_k + t - y_k|| over all N matches, theta = inlier_thresh. */
#define TURBOREG_SCORE_IN 0          /* largest inlier number #{k : e_k <= theta} (Eq. 9) */
#define TURBOREG_SCORE_MAE 1         /* smallest (1/N) sum_k min(e_k, theta) */
#define TURBOREG_SCORE_MSE 2         /* smallest (1/N) sum_k min(e_k^2, theta^2) */
/* proposal */
#define TURBOREG_PROPOSAL_PLAIN 0    /* pivots = top-K1 SC^2 edges (Eq. 4) */
#define TURBOREG_PROPOSAL_LEARNED 1  /* pivots ranked by floor(W_ij p_i p_j), p = inlier probability
                                        of the proposal MLP (set with turboreg_set_proposal_model) */
/* flags */
#define TURBOREG_FLAG_SC2_BITSET 0x1u  /* SC^2 by bitset AND+popcount on CUDA cores
                                          instead of the tcgen05 FP8 GEMM (same integers) */
#define TURBOREG_FLAG_SC2_GEMM 0x40u   /* SC^2 by the tcgen05 FP8 GEMM.  Without either flag a single
                                          problem with N <= 5120 (and pair MMAs available) gets the
                                          path chosen on the device after the compatibility graph,
                                          from N and the edge count (the CUDA-core path up to about
                                          5 % density at N = 5000); batches and larger problems use
                                          the GEMM.  Same integers on every path */
#define TURBOREG_FLAG_STAGE_TIMES 0x2u /* record per-stage CUDA-event times (turboreg_stage_times) */
#define TURBOREG_FLAG_NO_GRAPH 0x4u    /* launch the stages one by one instead of replaying the
                                          captured CUDA graph of this problem shape */
#define TURBOREG_FLAG_SC2_SINGLE_CTA 0x8u /* SC^2 GEMM on independent CTAs (128 x 256 tiles); by default
                                             2-CTA clusters compute 256 x 256 blocks with pair MMAs
                                             (cta_group::2), each CTA holding half of A and of B
                                             (same integers either way) */
#define TURBOREG_FLAG_VERIFY_PTS32 0x10u   /* verification tile of 128 hypotheses x 128 matches per block */
#define TURBOREG_FLAG_VERIFY_PTS128 0x20u  /* ... x 512 matches per block (default: 256); tile shapes are
                                              chosen by the autotuner (same results either way); in a
                                              batch the first problem's tile flags apply to all */

typedef struct {
    float tau;            /* compatibility threshold of Eq. 1, metres, >= 0 */
    int32_t k1;           /* pivot count K1 of Eq. 4, 1..TURBOREG_K1_MAX */
    int32_t k2;           /* TurboCliques per pivot K2 of Eq. 7, 1..TURBOREG_K2_MAX (paper: 2) */
    float inlier_thresh;  /* theta: a match is an inlier of (R,t) iff ||R x + t - y|| <= theta, > 0 */
    int32_t graph_mode;   /* TURBOREG_GRAPH_O2 or TURBOREG_GRAPH_SC2 */
    int32_t proposal;     /* TURBOREG_PROPOSAL_PLAIN or _LEARNED */
    float kappa_fp64;     /* when sigma1/sigma2 of a clique's 3x3 cross-covariance exceeds this
                             bound (0 selects the default 100), its closed-form Kabsch is redone
                             with the triangle normals computed in FP64 (the ill-conditioned
                             step; the rest stays FP32) */
    uint32_t flags;       /* TURBOREG_FLAG_* */
    int32_t learned_min_inliers; /* learned proposal: if its best inlier number is below this (or it
                                    finds no hypothesis) the plain proposal decides the result;
                                    0 selects max(10, N / 200) */
    int32_t scoring;      /* TURBOREG_SCORE_IN, _MAE or _MSE; ties go to the lowest h */
} turboreg_params;

typedef struct {
    float R[9];             /* row-major rotation, y = R x + t */
    float t[3];             /* translation, metres */
    int32_t clique[3];      /* winning TurboClique: pivot (i < j) then z (z > j on the O2Graph), or -1 */
    int32_t inlier_count;   /* inlier number of the winner (Eq. 9) */
    int32_t hypothesis;     /* h* in Alg. 2 order h = r*|P| + p, lowest h on ties; -1 if none */
    int32_t n_pivots;       /* |P| = min(K1, number of O2Graph edges) */
    int32_t n_valid;        /* hypotheses with a TurboClique and a non-degenerate Kabsch */
    int32_t used_fp64;      /* 1 if the winner's Kabsch used the FP64 normals (see kappa_fp64) */
    int32_t used_fallback;  /* learned proposal: 1 if the plain path decided the result */
    int32_t status;         /* turboreg_status of this problem */
    float score;            /* the winner's selection score: the inlier number (SCORE_IN), or its
                               capped mean error in metres (MAE) or square metres (MSE), computed
                               in FP32 with each term rounded to 2^-22 theta (theta^2) */
} turboreg_result;

/* Fill p with the paper's defaults (K2 = 2, O2Graph, plain proposal,
 * inlier-number scoring, kappa bound 100) and the given tau, K1 and inlier
 * threshold. */
void turboreg_default_params(turboreg_params* p, float tau, int32_t k1, float inlier_thresh);

/* Create a context on CUDA device `device` sized for problems of up to
 * max_n correspondences and batches of up to max_batch problems whose total
 * correspondence count is at most max_n * max_batch.  `cuda_stream` is a
 * cudaStream_t to run on, or NULL to let the context create its own.  The
 * device workspace (about 3.1 * max_n^2 bytes plus 2.3 * max_n^2 bytes per
 * batched problem slot) is allocated here, never inside register calls.
 * On success *out receives the context.
 * Errors: INVALID_ARG (out NULL, max_n < 3 or > TURBOREG_MAX_N, max_batch < 1),
 *         OOM, CUDA. */
int turboreg_create(int device, int32_t max_n, int32_t max_batch, void* cuda_stream,
                    turboreg_ctx** out);

/* Register one problem: src, dst = x, y as float32 [n][3]; writes the result
 * to the host struct *out (out->status equals the return value).
 * Errors: INVALID_ARG, TOO_FEW, NONFINITE, CUDA, TIMEOUT, NO_HYPOTHESIS
 * (then R = I, t = 0, inlier_count = 0). */
int turboreg_register(turboreg_ctx* ctx, const float* src, const float* dst, int32_t n,
                      const turboreg_params* params, turboreg_result* out);

/* The same registration enqueued on the context's stream without waiting for
 * it, so that consecutive registrations run back to back on the GPU while
 * the host prepares the next ones (the paper has no counterpart: it is the
 * stream form of turboreg_register).  src, dst: device memory or page-locked
 * host memory (read in place by the first kernel when mapped, else copied on
 * the stream); out: device memory or page-locked host memory, written by the
 * last kernel.  Inputs and out must
 * stay valid and unchanged until turboreg_synchronize returns.  The learned
 * proposal is not accepted (its plain fallback needs the result on the host)
 * and stage times are not recorded.  Argument, size and host-side finiteness
 * errors are returned at once and nothing is enqueued (out is not written);
 * device-side outcomes (NO_HYPOTHESIS, TIMEOUT, NONFINITE of device inputs)
 * arrive in out->status.
 * Errors: INVALID_ARG (also: pageable host src, dst or out, or the learned
 *         proposal), TOO_FEW, NONFINITE, CUDA. */
int turboreg_register_async(turboreg_ctx* ctx, const float* src, const float* dst, int32_t n,
                            const turboreg_params* params, turboreg_result* out);

/* Wait for everything enqueued on the context's stream.  Errors: CUDA. */
int turboreg_synchronize(turboreg_ctx* ctx);

/* Register `num` independent problems in one batched pass.  Problem b uses
 * matches [offsets[b], offsets[b+1]) of src_cat / dst_cat (float32 [total][3]);
 * offsets is a HOST array of num+1 non-decreasing int64 with offsets[0] = 0.
 * params points to 1 struct (shared) or num structs (one per problem): pass
 * params_count = 1 or num.  out is a HOST array of num results; each carries
 * its own status.  Return value: OK if every problem was processed (per-problem
 * failures such as NO_HYPOTHESIS are reported in out[b].status only), else the
 * first argument / CUDA error.
 * Errors: INVALID_ARG (num < 1 or > max_batch, a problem with n > max_n,
 *         total > max_n * max_batch, bad offsets), NONFINITE is per problem,
 *         CUDA, TIMEOUT. */
int turboreg_register_batched(turboreg_ctx* ctx, const float* src_cat, const float* dst_cat,
                              const int64_t* offsets, int32_t num,
                              const turboreg_params* params, int32_t params_count,
                              turboreg_result* out);

/* Release the context and its device workspace.  NULL-safe. */
void turboreg_destroy(turboreg_ctx* ctx);

/* Human-readable name of a status code (static storage). */
const char* turboreg_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TURBOREG_H */
