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
    TURBOREG_BUF_DEGREE = 9     /* int32 [n]: sum_j G_ij (degree in the compatibility graph) */
} turboreg_buffer;

/* Shape of the most recent turboreg_register call: n, n_pad, |P| and the
 * number of hypotheses k2*|P|.  Any pointer may be NULL. */
int turboreg_debug_shape(turboreg_ctx* ctx, int32_t* n, int32_t* n_pad, int32_t* n_pivots,
                         int32_t* n_hyp);

/* Copy stage buffer `which` of the most recent call to host memory `dst`
 * (at most max_bytes).  Returns the byte count copied (>= 0) or -status. */
int64_t turboreg_debug_copy(turboreg_ctx* ctx, int which, void* dst, int64_t max_bytes);

/* Per-stage device times (ms) of the most recent call made with
 * TURBOREG_FLAG_STAGE_TIMES: pack, compat, sc2, topk, pgs, kabsch, verify,
 * finalize.  Writes up to `max` floats; returns the number of stages. */
int turboreg_stage_times(turboreg_ctx* ctx, float* ms, int32_t max);

/* Names of the stages reported by turboreg_stage_times. */
const char* turboreg_stage_name(int32_t stage);

#ifdef __cplusplus
}
#endif
#endif /* TURBOREG_INTERNAL_H */
