/*
 * turboreg_internal.h -- inspection and training entry points of the GB300
 * TurboReg library.  Not part of the four-call registration contract in
 * turboreg.h; used by the test-suite (stage-by-stage parity), the benchmark
 * (per-stage times) and the learned-proposal trainer.
 *
 * Same conventions as turboreg.h: plain C types, caller-owned buffers,
 * synchronous calls, status-code returns.
 */
#ifndef TURBOREG_INTERNAL_H
#define TURBOREG_INTERNAL_H

#include <stdint.h>
#include "turboreg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Device buffers that hold one stage's output of the most recent
 * turboreg_register call on a context (n_pad = N rounded up to 256). */
typedef enum {
    TURBOREG_BUF_ADJ_BITS = 1,  /* uint32 [n_pad][n_pad/32]: bit (j%32) of word [i][j/32] = G_ij (Eq. 1) */
    TURBOREG_BUF_ADJ_FP8 = 2,   /* uint8  [n_pad][n_pad]: G_ij as FP8 E4M3 (0x38 = 1.0, 0x00 = 0) */
    TURBOREG_BUF_SC2 = 3,       /* uint16 [n_pad][n_pad]: O2Graph weights G~_ij (Eq. 2, Def. 2);
                                   only i < j is defined */
    TURBOREG_BUF_PIVOTS = 4,    /* int32 [n_pivots][4]: (i, j, G~_ij, 0) in Eq. 4 order */
    TURBOREG_BUF_CLIQUES = 5,   /* int32 [k2*n_pivots][4]: (i, j, z, valid) in Alg. 2 order */
    TURBOREG_BUF_RT = 6,        /* float [k2*n_pivots][16]: R (9, row-major), t (3), kappa,
                                   flags (as int32 bits: 1 valid, 2 fp64), 2 unused */
    TURBOREG_BUF_INLIERS = 7,   /* int32 [k2*n_pivots]: inlier number per hypothesis */
    TURBOREG_BUF_ROWSCORE = 8,  /* int32 [n]: sum_j G^_ij (SC^2 row score) */
    TURBOREG_BUF_DEGREE = 9,    /* int32 [n]: sum_j G_ij (degree in the compatibility graph) */
    TURBOREG_BUF_FEATURES = 10, /* float [n][8]: proposal features (learned proposal) */
    TURBOREG_BUF_PROB = 11,     /* float [n]: proposal inlier probabilities (learned proposal) */
    TURBOREG_BUF_SCORES = 12    /* uint64 [k2*n_pivots]: capped error sum per hypothesis in units of
                                   2^-22 theta (MAE) or 2^-22 theta^2 (MSE); zero in SCORE_IN mode */
} turboreg_buffer;

/* Failure injection for tests (a turboreg_params flag; no counterpart in the
 * paper).  Every compatibility-graph block of the registration skips the copy
 * of its row points, so its bounded wait for that copy can only expire: after
 * 20 ms (instead of the normal 2 s bound) the block records a timeout and
 * leaves its tile of the graph empty, the later stages run on the empty graph,
 * and the result's status is TURBOREG_ERR_TIMEOUT.  No device fault and no
 * hang: the context stays usable and the next registration is unaffected. */
#define TURBOREG_FLAG_DEBUG_STALL_COMPAT 0x10000u

/* Allocation-failure injection for tests: when the environment variable
 * TURBOREG_DEBUG_FAIL_ALLOC holds k >= 1, the k-th memory allocation made by
 * turboreg_create (device, page-locked and plain host memory, counted per call
 * and thread) fails; turboreg_create then frees what it had allocated and
 * returns TURBOREG_ERR_OOM.  Unset or 0: no effect. */

/* Shape of the most recent turboreg_register call: n, n_pad, |P| and the
 * number of hypotheses k2*|P|.  Any pointer may be NULL. */
int turboreg_debug_shape(turboreg_ctx* ctx, int32_t* n, int32_t* n_pad, int32_t* n_pivots,
                         int32_t* n_hyp);

/* SC^2 path of the most recent registration call: 1 the CUDA-core bitset
 * form, 2 the tensor-core GEMM (chosen on the device for one problem without
 * an SC^2 flag, from N and the edge count).  Returns a turboreg_status. */
int turboreg_debug_sc2_path(turboreg_ctx* ctx, int32_t* path);

/* Copy stage buffer `which` of the most recent call to host memory `dst`
 * (at most max_bytes).  Returns the byte count copied (>= 0) or -status. */
int64_t turboreg_debug_copy(turboreg_ctx* ctx, int which, void* dst, int64_t max_bytes);

/* Per-stage device times (ms) of the most recent call made with
 * TURBOREG_FLAG_STAGE_TIMES (a single registration or a batch): pack, compat,
 * sc2, proposal (the threshold's select launch when the SC^2 stage did not
 * choose it, and the learned proposal's features, network, weight histogram
 * and select), topk (count and emit), pgs (with the pivot ranks and the
 * cliques' Kabsch), verify, finalize.  Writes up to `max` floats; returns the
 * number of stages. */
int turboreg_stage_times(turboreg_ctx* ctx, float* ms, int32_t max);

/* Names of the stages reported by turboreg_stage_times. */
const char* turboreg_stage_name(int32_t stage);

/* Score caller-given rigid transforms on one problem with the library's
 * verification kernel (the inlier number of Eq. 9 and the capped errors of
 * the ranking study, Table 6), e.g. to compare the selected hypothesis with
 * a reference transform.  src, dst: float32 [n][3], host or device.
 * rt: HOST float32 [m][12], transform k = R (row-major 3x3) then t; 1 <= m <=
 * TURBOREG_K1_MAX.  params: tau, K1, K2, graph_mode and proposal are
 * ignored; inlier_thresh and scoring are used.  Outputs (HOST): out_in[m] the
 * inlier numbers; out_units[m] (may be NULL) the capped-error sums in the
 * units of TURBOREG_BUF_SCORES (all zero under TURBOREG_SCORE_IN).  The call
 * reuses problem slot 0, so the inspection buffers of the previous register
 * call are overwritten.
 * Errors: INVALID_ARG (null pointer, m out of range, bad params, non-finite
 * rt), TOO_FEW, NONFINITE, CUDA. */
int turboreg_score_transforms(turboreg_ctx* ctx, const float* src, const float* dst, int32_t n,
                              const turboreg_params* params, const float* rt, int32_t m,
                              int32_t* out_in, uint64_t* out_units);

/* Kabsch of caller-given cliques (Sec. 3.5; the 3-clique vs 10-clique
 * comparison of App. A.2): for each of m tuples of k match indices, the
 * proper rotation R and translation t minimising sum ||R x + t - y||^2 over
 * the tuple's matches.  k = 3 runs the registration path's closed form (FP32,
 * FP64 normals above params->kappa_fp64); 4 <= k <= 32 runs Horn's
 * quaternion method with Jacobi eigen-decomposition in FP64.
 * src, dst: float32 [n][3], host or device.  idx: HOST int32 [m][k], every
 * index in [0, n).  m >= 1 and m * k <= 4 * TURBOREG_K1_MAX * TURBOREG_K2_MAX.
 * Outputs (HOST): out_rt[m][12] = R (row-major) then t; out_valid[m] = 1 for
 * a valid transform, 0 for a degenerate tuple (collinear or repeated points,
 * s2 <= 1e-12 s1), in which case out_rt is unspecified.  Reuses problem slot 0
 * (overwrites the inspection buffers of the previous register call).
 * Errors: INVALID_ARG (null pointer, k or m out of range, index out of range,
 * bad params), TOO_FEW, NONFINITE, CUDA. */
int turboreg_kabsch_cliques(turboreg_ctx* ctx, const float* src, const float* dst, int32_t n,
                            const turboreg_params* params, const int32_t* idx, int32_t k, int32_t m,
                            float* out_rt, int32_t* out_valid);

/* ---- learned proposal (project extension; the paper ranks pivots by SC^2 alone) ----
 * A per-correspondence inlier-scoring MLP 8 -> 64 -> 128 -> 64 -> 1 (ReLU,
 * sigmoid output), BF16 weights and activations, FP32 accumulation.  Its
 * parameters are one FP32 vector of TURBOREG_MLP_PARAMS values, row-major
 * [out][in]: W1[64][8] b1[64] W2[128][64] b2[128] W3[64][128] b3[64] W4[64] b4[1].
 * Features of correspondence i (8 floats): (x_i - mean x)/rms_x (3),
 * (y_i - mean y)/rms_y (3), degree_i / N, SC^2 row score_i / max row score. */
#define TURBOREG_MLP_PARAMS 17217

/* Set the proposal model of a context (host FP32 parameter vector, copied). */
int turboreg_set_proposal_model(turboreg_ctx* ctx, const float* params);

/* Features of one problem: runs the compatibility graph and SC^2 and writes
 * feat[n][8] (float32; host or device pointer). */
int turboreg_features(turboreg_ctx* ctx, const float* src, const float* dst, int32_t n,
                      const turboreg_params* params, float* feat);

typedef struct turboreg_mlp turboreg_mlp;   /* trainer: FP32 master weights, Adam moments, scratch */

/* Create a trainer on `device` for mini-batches of up to max_samples rows;
 * weights are He-initialised from `seed`.  cuda_stream: cudaStream_t or NULL. */
int turboreg_mlp_create(int device, int32_t max_samples, uint64_t seed, void* cuda_stream, turboreg_mlp** out);
void turboreg_mlp_destroy(turboreg_mlp* t);   /* NULL-safe */
/* Parameters (host FP32 [TURBOREG_MLP_PARAMS]). */
int turboreg_mlp_get_params(turboreg_mlp* t, float* params);
int turboreg_mlp_set_params(turboreg_mlp* t, const float* params);
/* Adam state (host FP32 [TURBOREG_MLP_PARAMS] each, and the step count). */
int turboreg_mlp_get_state(turboreg_mlp* t, float* m, float* v, int32_t* step);
int turboreg_mlp_set_state(turboreg_mlp* t, const float* m, const float* v, int32_t step);
/* Inference: prob[k] = p(inlier) for feat[k][8], k < m (device pointers). */
int turboreg_mlp_forward(turboreg_mlp* t, const float* feat, int32_t m, float* prob);
/* Gradient of the mean binary cross-entropy over (feat, label) (device
 * pointers, labels 0/1 as float) w.r.t. the parameters: grad (host
 * [TURBOREG_MLP_PARAMS]) and loss (host). */
int turboreg_mlp_grad(turboreg_mlp* t, const float* feat, const float* label, int32_t m, float* grad,
                      float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean BCE of the
 * mini-batch; loss (host, may be NULL) receives the loss before the step. */
int turboreg_mlp_train_step(turboreg_mlp* t, const float* feat, const float* label, int32_t m, float lr,
                            float* loss);

/* Largest n accepted by turboreg_select_pivots_noalloc. */
#define TURBOREG_NOALLOC_MAX_N 8192

/* Pivot selection (top-K1 O2Graph edges, ties to the lowest (i, j)) on a
 * caller-provided weight matrix, allocating nothing.  The paper has no
 * counterpart to this entry point: it exists for callers that cannot call
 * cudaMalloc, such as a plugin inside a host framework that owns all device
 * memory through its own pool, or a real-time loop that forbids allocation
 * after start-up (cudaMalloc may synchronise the device and take unbounded
 * time).  Its scratch (histogram, active-row list with per-row counts,
 * candidate keys, control block: about 225 KB) is one fixed array in the library's device memory,
 * loaded with the module and held by every GPU that loads the library until
 * the process exits; nothing is allocated or freed by this call.
 *
 *  w_dev       device, uint16 [n][ldw] row-major, 16-byte aligned; entry (i, j)
 *              for i < j < n is the O2Graph weight (an SC^2 count, 0..n-2).
 *              Entries with j <= i or j >= n are ignored.  ldw % 8 == 0 and
 *              ldw >= n rounded up to 8.  If any entry (i < j < n) exceeds
 *              n - 2, the call selects nothing and *n_pivots_dev receives
 *              -TURBOREG_ERR_INVALID_ARG (the values are only seen on the GPU,
 *              so the error arrives with the results, not as the return code).
 *  n           nodes, 1 .. TURBOREG_NOALLOC_MAX_N
 *  k1          pivots wanted, 1 .. TURBOREG_K1_MAX
 *  pivots_dev  device, int32 [k1][4] out: (i, j, weight, 0) in (weight desc,
 *              i asc, j asc) order; rows past *n_pivots_dev are untouched
 *  n_pivots_dev device, int32 out: min(k1, number of edges with weight > 0),
 *              or -TURBOREG_ERR_INVALID_ARG for weights above n - 2
 *  cuda_stream cudaStream_t to run on (NULL = legacy default stream)
 *
 * Asynchronous on cuda_stream; results are ready when the stream reaches
 * them.  Returns INVALID_ARG (clear message on stderr for sizes beyond the
 * fixed limits) or CUDA; OK otherwise.  Every call shares the one scratch
 * array, which keeps the last call's contents (the call clears what must
 * start at zero), so calls that overlap on the GPU race: serialise calls per
 * device.  The first call on a device looks up the array's device address
 * with that device current; make that first call before any stream capture.
 * Later calls outside a capture look the address up again and redo the
 * set-up when it changed (a device reset, a context re-created by the host
 * framework); a call under capture uses the address recorded last, so the
 * context must not be replaced between the last uncaptured call and a
 * captured one. */
int turboreg_select_pivots_noalloc(const uint16_t* w_dev, int32_t n, int32_t ldw, int32_t k1,
                                   int32_t* pivots_dev, int32_t* n_pivots_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TURBOREG_INTERNAL_H */
