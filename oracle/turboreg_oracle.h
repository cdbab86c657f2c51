/*
 * FP64 CPU oracle for the TurboReg registration hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this code: only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table
 * or constant with the CUDA implementation.
 *
 * Each function is a plain, slow, step-by-step statement of one part of the
 * method (TurboReg, ICCV 2025):
 *   orc_compat   Eq. 1  compatibility graph G (0/1, zero diagonal)
 *   orc_sc2      Eq. 2  SC^2 graph  G^_ij = G_ij * sum_k G_ik G_jk
 *   orc_pivots   Eq. 4 + Def. 2  top-K1 edges of the O2Graph
 *   orc_cliques  Eq. 5-7, Alg. 1  per-pivot top-K2 TurboCliques, Alg. 2 layout,
 *                on the O2Graph (Def. 2) or the undirected SC^2 graph
 *   orc_kabsch   Sec. 3.5  least-squares rigid transform from 3 matches (SVD)
 *   orc_kabsch_n the same over m matches (App. A.2 compares 3- and 10-cliques)
 *   orc_inliers  Sec. 3.5 / Eq. 9  inlier number of one hypothesis
 *   orc_score    App. (ranking study, Table 6)  IN, MAE or MSE of one hypothesis
 *   orc_register the whole path, Eq. 1 -> Eq. 9
 *
 * Inputs are float32 and are promoted exactly to double.  Everything after
 * that is double precision, compiled with -ffp-contract=off so the operation
 * order written here is the order evaluated.
 *
 * Parity status: every function is pinned by tests under tests/ (brute
 * force, closed forms, invariants, a hand-worked graph); see the pin list in
 * the design notes.  None is "parity unpinned".
 */
#ifndef TURBOREG_ORACLE_H
#define TURBOREG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float tau;          /* compatibility threshold, Eq. 1 */
    int32_t k1;         /* pivot count, Eq. 4 */
    int32_t k2;         /* TurboCliques per pivot, Eq. 7 */
    float theta;        /* inlier threshold of the inlier number, Eq. 9 */
    double near_band;   /* report residuals with | ||r|| - theta | <= near_band */
    int32_t graph_mode; /* 0: O2Graph (Def. 2), 1: undirected SC^2 graph (Eq. 2) */
    int32_t scoring;    /* hypothesis selection: 0 IN (Eq. 9), 1 MAE, 2 MSE (see orc_score) */
} orc_params;

typedef struct {
    double R[9];        /* row-major, y = R x + t */
    double t[3];
    int32_t clique[3];
    int32_t inlier_count;
    int32_t hypothesis; /* h* in Alg. 2 order h = r*|P| + p, or -1 */
    int32_t n_pivots;   /* |P| */
    int32_t n_valid;    /* hypotheses with a clique and a non-degenerate Kabsch */
    int32_t status;     /* 0 ok, 7 no hypothesis */
    double kappa;       /* sigma1/sigma2 of the winning clique */
    double score;       /* the winner's selection score (IN as a number, or MAE / MSE) */
} orc_result;

/* Eq. 1.  A[i*n+j] = 1 iff | ||x_i-x_j|| - ||y_i-y_j|| | <= tau, i != j; A_ii = 0. */
void orc_compat(const float* x, const float* y, int32_t n, float tau, uint8_t* A);

/* Eq. 2.  S[i*n+j] = A_ij * sum_k A_ik A_jk (full symmetric n x n). */
void orc_sc2(const uint8_t* A, int32_t n, int32_t* S);

/* Eq. 4 on the O2Graph (Def. 2): edges (i<j, S_ij>0) sorted by
 * (S desc, i asc, j asc); the first min(k1, |E+|) are written to pi/pj/pw.
 * Returns |P|. */
int32_t orc_pivots(const int32_t* S, int32_t n, int32_t k1,
                   int32_t* pi, int32_t* pj, int32_t* pw);

/* Eq. 5-7 / Alg. 1 on the graph G- chosen by graph_mode: 0 the O2Graph
 * (G-_ab = S_ab for a < b, else 0), 1 the undirected SC^2 graph (G-_ab =
 * S_ab).  cliques[(r*np+p)*3 + {0,1,2}] = (i,j,z) of the rank-r TurboClique
 * of pivot p (Alg. 2 layout), valid[h] = 1 if it exists.  Ties of the
 * aggregated weight go to the lower z. */
void orc_cliques(const int32_t* S, int32_t n, const int32_t* pi, const int32_t* pj,
                 int32_t np, int32_t k2, int32_t graph_mode, int32_t* cliques, uint8_t* valid);

/* Kabsch on 3 matches: R,t minimise sum_a ||R xa + t - ya||^2 over proper
 * rotations.  xs, ys: 3 points each, row-major [3][3].  kappa = s1/s2 of the
 * centred cross-covariance.  Returns 1 if valid (s2 > 1e-12 s1), else 0. */
int32_t orc_kabsch(const double* xs, const double* ys, double* R, double* t,
                   double* kappa);

/* Kabsch on m >= 3 matches (the same least-squares problem over a larger
 * clique, as in the 3-clique vs 10-clique comparison of the appendix):
 * xs, ys row-major [m][3].  Valid if s2 > 1e-12 s1 (not collinear). */
int32_t orc_kabsch_n(const double* xs, const double* ys, int32_t m, double* R, double* t,
                     double* kappa);

/* Jacobi SVD of a 3x3 matrix H = U diag(s) V^T, s descending. */
void orc_svd3(const double* H, double* U, double* s, double* V);

/* Inlier number: #{k : ||R x_k + t - y_k||^2 <= theta^2}.  n_near (optional)
 * receives #{k : | ||r_k|| - theta | <= band}. */
int32_t orc_inliers(const float* x, const float* y, int32_t n, const double* R,
                    const double* t, float theta, double band, int32_t* n_near);

/* Selection score of one hypothesis over all n matches, e_k = ||R x_k + t - y_k||:
 *   mode 0 (IN):  #{k : e_k^2 <= theta^2}                 (larger is better)
 *   mode 1 (MAE): (1/n) sum_k min(e_k, theta)             (smaller is better)
 *   mode 2 (MSE): (1/n) sum_k min(e_k^2, theta^2)         (smaller is better)
 * MAE and MSE are the mean absolute / squared residuals with every residual
 * capped at theta, so an outlier costs theta (or theta^2) whatever its size. */
double orc_score(const float* x, const float* y, int32_t n, const double* R, const double* t,
                 float theta, int32_t mode);

/* Whole path.  Optional outputs (may be NULL): per-hypothesis inlier counts
 * in_counts[k1*k2], near counts near_counts[k1*k2], per-hypothesis R,t
 * (rt[h*12 .. +12] = R row-major then t), valid flags hyp_valid[k1*k2],
 * selection scores scores[k1*k2] (orc_score with prm->scoring; NaN where no
 * valid hypothesis).  The winner is the largest IN (scoring 0) or the
 * smallest MAE / MSE (scoring 1, 2); ties go to the lowest h.
 * Returns 0 on success, 7 if no valid hypothesis, 1 on bad arguments,
 * 4 on allocation failure. */
int32_t orc_register(const float* x, const float* y, int32_t n, const orc_params* prm,
                     orc_result* res, int32_t* in_counts, int32_t* near_counts,
                     double* rt, uint8_t* hyp_valid, double* scores);

#ifdef __cplusplus
}
#endif
#endif
