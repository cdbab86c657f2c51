/*
 * FP64 CPU oracle for the TurboReg registration hot path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * CPU baseline of the benchmark; never by the product path.  It shares no
 * code with the CUDA implementation.  Build with -ffp-contract=off so that
 * the double-precision operation order written below is the one evaluated.
 *
 * Section / equation references are to the TurboReg paper (ICCV 2025).
 */
#include "turboreg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Eq. 1: compatibility graph                                          */
/* ------------------------------------------------------------------ */

static double dist3(const float* p, const float* q)
{
    /* fixed order: ((dx*dx + dy*dy) + dz*dz), each product rounded */
    double dx = (double)p[0] - (double)q[0];
    double dy = (double)p[1] - (double)q[1];
    double dz = (double)p[2] - (double)q[2];
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    return sqrt(s);
}

void orc_compat(const float* x, const float* y, int32_t n, float tau, uint8_t* A)
{
    /* Eq. 1 with the diagonal set to 0: the appendix identifies G^_ij with the
     * number of triangles on edge (i,j), which needs k outside {i,j}. */
    const double t = (double)tau;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = 0; j < n; ++j) {
            uint8_t g = 0;
            if (i != j) {
                double dX = dist3(x + 3 * (size_t)i, x + 3 * (size_t)j);
                double dY = dist3(y + 3 * (size_t)i, y + 3 * (size_t)j);
                g = (fabs(dX - dY) <= t) ? 1 : 0;
            }
            A[(size_t)i * n + j] = g;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Eq. 2: SC^2 graph                                                   */
/* ------------------------------------------------------------------ */

void orc_sc2(const uint8_t* A, int32_t n, int32_t* S)
{
    /* G^_ij = G_ij * sum_k G_ik G_jk.  The sum is evaluated as the popcount
     * of the AND of rows i and j packed 64 entries per word: the same
     * integer as the term-by-term sum. */
    const int32_t nw = (n + 63) / 64;
    uint64_t* rows = (uint64_t*)calloc((size_t)n * nw, sizeof(uint64_t));
    memset(S, 0, sizeof(int32_t) * (size_t)n * n);
    if (!rows) return;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = 0; k < n; ++k)
            if (A[(size_t)i * n + k])
                rows[(size_t)i * nw + k / 64] |= (uint64_t)1 << (k % 64);
    for (int32_t i = 0; i < n; ++i) {
        const uint64_t* ri = rows + (size_t)i * nw;
        for (int32_t j = i + 1; j < n; ++j) {
            if (!A[(size_t)i * n + j]) continue;
            const uint64_t* rj = rows + (size_t)j * nw;
            int32_t c = 0;
            for (int32_t w = 0; w < nw; ++w) c += __builtin_popcountll(ri[w] & rj[w]);
            S[(size_t)i * n + j] = c;
            S[(size_t)j * n + i] = c;
        }
    }
    free(rows);
}

/* ------------------------------------------------------------------ */
/* Eq. 4 on the O2Graph (Def. 2): pivot selection                      */
/* ------------------------------------------------------------------ */

typedef struct { int32_t w, i, j; } edge_t;

static int edge_cmp(const void* a, const void* b)
{
    const edge_t* p = (const edge_t*)a;
    const edge_t* q = (const edge_t*)b;
    if (p->w != q->w) return (p->w > q->w) ? -1 : 1;   /* weight descending */
    if (p->i != q->i) return (p->i < q->i) ? -1 : 1;   /* then lowest (i, j) */
    if (p->j != q->j) return (p->j < q->j) ? -1 : 1;
    return 0;
}

int32_t orc_pivots(const int32_t* S, int32_t n, int32_t k1,
                   int32_t* pi, int32_t* pj, int32_t* pw)
{
    /* O2Graph: G~_ij = G^_ij for i < j, else 0.  Edges are the positive
     * entries; a zero entry is not an edge and never a pivot. */
    size_t ne = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j)
            if (S[(size_t)i * n + j] > 0) ++ne;
    edge_t* e = (edge_t*)malloc(sizeof(edge_t) * (ne ? ne : 1));
    if (!e) return -1;
    size_t m = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) {
            int32_t w = S[(size_t)i * n + j];
            if (w > 0) { e[m].w = w; e[m].i = i; e[m].j = j; ++m; }
        }
    qsort(e, ne, sizeof(edge_t), edge_cmp);
    int32_t np = (ne < (size_t)k1) ? (int32_t)ne : k1;
    for (int32_t p = 0; p < np; ++p) { pi[p] = e[p].i; pj[p] = e[p].j; pw[p] = e[p].w; }
    free(e);
    return np;
}

/* ------------------------------------------------------------------ */
/* Eq. 5-7 / Alg. 1: TurboClique search and per-pivot selection         */
/* ------------------------------------------------------------------ */

static int32_t o2(const int32_t* S, int32_t n, int32_t a, int32_t b)
{
    return (a < b) ? S[(size_t)a * n + b] : 0;   /* Def. 2 */
}

/* The graph G- that Alg. 1 searches: the O2Graph or the undirected SC^2 graph. */
static int32_t gbar(const int32_t* S, int32_t n, int32_t mode, int32_t a, int32_t b)
{
    return (mode == 1) ? S[(size_t)a * n + b] : o2(S, n, a, b);
}

void orc_cliques(const int32_t* S, int32_t n, const int32_t* pi, const int32_t* pj,
                 int32_t np, int32_t k2, int32_t graph_mode, int32_t* cliques, uint8_t* valid)
{
    int32_t* topz = (int32_t*)malloc(sizeof(int32_t) * (size_t)k2);
    int32_t* tops = (int32_t*)malloc(sizeof(int32_t) * (size_t)k2);
    for (int32_t p = 0; p < np; ++p) {
        const int32_t i = pi[p], j = pj[p];
        const int32_t gij = gbar(S, n, graph_mode, i, j);
        int32_t cnt = 0;
        for (int32_t z = 0; z < n; ++z) {
            if (z == i || z == j) continue;
            const int32_t giz = gbar(S, n, graph_mode, i, z), gjz = gbar(S, n, graph_mode, j, z);
            if (!(giz > 0 && gjz > 0)) continue;            /* Eq. 5 */
            const int32_t s = gij + giz + gjz;              /* Eq. 6 */
            /* Eq. 7: keep the K2 largest; z ascends, so a later z only
             * displaces on a strictly larger weight (ties keep lower z). */
            int32_t pos = cnt;
            while (pos > 0 && tops[pos - 1] < s) --pos;
            if (pos >= k2) continue;
            int32_t last = (cnt < k2) ? cnt : k2 - 1;
            for (int32_t q = last; q > pos; --q) { tops[q] = tops[q - 1]; topz[q] = topz[q - 1]; }
            tops[pos] = s; topz[pos] = z;
            if (cnt < k2) ++cnt;
        }
        for (int32_t r = 0; r < k2; ++r) {
            const size_t h = (size_t)r * np + p;            /* Alg. 2 layout */
            if (r < cnt) {
                cliques[h * 3 + 0] = i; cliques[h * 3 + 1] = j; cliques[h * 3 + 2] = topz[r];
                valid[h] = 1;
            } else {
                cliques[h * 3 + 0] = i; cliques[h * 3 + 1] = j; cliques[h * 3 + 2] = -1;
                valid[h] = 0;
            }
        }
    }
    free(topz); free(tops);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.5: Kabsch                                                    */
/* ------------------------------------------------------------------ */

void orc_svd3(const double* H, double* U, double* s, double* V)
{
    /* One-sided (Hestenes) Jacobi: rotate column pairs of W = H V until the
     * columns are mutually orthogonal; then s_c = ||w_c||, U = W diag(1/s). */
    double W[3][3], Vm[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int r = 0; r < 3; ++r) for (int c = 0; c < 3; ++c) W[r][c] = H[r * 3 + c];
    static const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int k = 0; k < 3; ++k) {
            const int p = pr[k][0], q = pr[k][1];
            double al = 0, be = 0, ga = 0;
            for (int r = 0; r < 3; ++r) {
                al += W[r][p] * W[r][p];
                be += W[r][q] * W[r][q];
                ga += W[r][p] * W[r][q];
            }
            if (ga == 0.0) continue;
            double rel = fabs(ga) / sqrt(al * be);
            if (!(rel > 1e-16)) continue;
            if (rel > off) off = rel;
            double zeta = (be - al) / (2.0 * ga);
            double tt = ((zeta >= 0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
            for (int r = 0; r < 3; ++r) {
                double wp = W[r][p], wq = W[r][q];
                W[r][p] = c * wp - sn * wq;
                W[r][q] = sn * wp + c * wq;
                double vp = Vm[r][p], vq = Vm[r][q];
                Vm[r][p] = c * vp - sn * vq;
                Vm[r][q] = sn * vp + c * vq;
            }
        }
        if (off <= 1e-15) break;
    }
    double sv[3];
    int idx[3] = {0, 1, 2};
    for (int r = 0; r < 9; ++r) U[r] = (r % 4 == 0) ? 1.0 : 0.0;
    for (int c = 0; c < 3; ++c)
        sv[c] = sqrt(W[0][c] * W[0][c] + W[1][c] * W[1][c] + W[2][c] * W[2][c]);
    for (int a = 0; a < 3; ++a)            /* order columns by s descending */
        for (int b = a + 1; b < 3; ++b)
            if (sv[idx[b]] > sv[idx[a]]) { int tmp = idx[a]; idx[a] = idx[b]; idx[b] = tmp; }
    for (int c = 0; c < 3; ++c) {
        s[c] = sv[idx[c]];
        for (int r = 0; r < 3; ++r) V[r * 3 + c] = Vm[r][idx[c]];
    }
    /* left singular vectors; complete with cross products where a singular
     * value is zero to working precision (rank-deficient H) */
    for (int c = 0; c < 3; ++c) {
        if (s[c] > 1e-10 * s[0] && s[c] > 0) {
            for (int r = 0; r < 3; ++r) U[r * 3 + c] = W[r][idx[c]] / s[c];
        } else if (c == 2) {
            U[0 * 3 + 2] = U[1 * 3 + 0] * U[2 * 3 + 1] - U[2 * 3 + 0] * U[1 * 3 + 1];
            U[1 * 3 + 2] = U[2 * 3 + 0] * U[0 * 3 + 1] - U[0 * 3 + 0] * U[2 * 3 + 1];
            U[2 * 3 + 2] = U[0 * 3 + 0] * U[1 * 3 + 1] - U[1 * 3 + 0] * U[0 * 3 + 1];
        } else {
            /* second column degenerate too: any unit vector orthogonal to u0 */
            double a0 = U[0], a1 = U[3], a2 = U[6];
            double e[3] = {0, 0, 0};
            int m = (fabs(a0) <= fabs(a1) && fabs(a0) <= fabs(a2)) ? 0 : (fabs(a1) <= fabs(a2) ? 1 : 2);
            e[m] = 1.0;
            double v0 = a1 * e[2] - a2 * e[1], v1 = a2 * e[0] - a0 * e[2], v2 = a0 * e[1] - a1 * e[0];
            double nv = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
            U[0 * 3 + 1] = v0 / nv; U[1 * 3 + 1] = v1 / nv; U[2 * 3 + 1] = v2 / nv;
        }
    }
}

static double det3(const double* M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7])
         - M[1] * (M[3] * M[8] - M[5] * M[6])
         + M[2] * (M[3] * M[7] - M[4] * M[6]);
}

int32_t orc_kabsch_n(const double* xs, const double* ys, int32_t m, double* R, double* t, double* kappa)
{
    double cx[3] = {0, 0, 0}, cy[3] = {0, 0, 0};
    for (int32_t a = 0; a < m; ++a)
        for (int d = 0; d < 3; ++d) {
            cx[d] += xs[a * 3 + d];
            cy[d] += ys[a * 3 + d];
        }
    for (int d = 0; d < 3; ++d) {
        cx[d] /= (double)m;
        cy[d] /= (double)m;
    }
    /* cross-covariance H = sum_a (x_a - cx)(y_a - cy)^T */
    double H[9] = {0};
    for (int32_t a = 0; a < m; ++a)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                H[r * 3 + c] += (xs[a * 3 + r] - cx[r]) * (ys[a * 3 + c] - cy[c]);
    double U[9], s[3], V[9];
    orc_svd3(H, U, s, V);
    *kappa = (s[1] > 0) ? s[0] / s[1] : INFINITY;
    /* R = V diag(1, 1, d) U^T with d = sign(det(V U^T)): the proper rotation
     * maximising tr(R H) */
    double d = (det3(V) * det3(U) < 0) ? -1.0 : 1.0;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            R[r * 3 + c] = V[r * 3 + 0] * U[c * 3 + 0] + V[r * 3 + 1] * U[c * 3 + 1]
                         + d * V[r * 3 + 2] * U[c * 3 + 2];
    for (int r = 0; r < 3; ++r)
        t[r] = cy[r] - (R[r * 3 + 0] * cx[0] + R[r * 3 + 1] * cx[1] + R[r * 3 + 2] * cx[2]);
    return (m >= 3 && s[0] > 0 && s[1] > 1e-12 * s[0]) ? 1 : 0;
}

int32_t orc_kabsch(const double* xs, const double* ys, double* R, double* t, double* kappa)
{
    return orc_kabsch_n(xs, ys, 3, R, t, kappa);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.5: inlier number                                             */
/* ------------------------------------------------------------------ */

int32_t orc_inliers(const float* x, const float* y, int32_t n, const double* R,
                    const double* t, float theta, double band, int32_t* n_near)
{
    const double th = (double)theta;
    int32_t cnt = 0, near = 0;
    for (int32_t k = 0; k < n; ++k) {
        const float* xk = x + 3 * (size_t)k;
        const float* yk = y + 3 * (size_t)k;
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double ra = R[a * 3 + 0] * (double)xk[0] + R[a * 3 + 1] * (double)xk[1]
                      + R[a * 3 + 2] * (double)xk[2] + t[a] - (double)yk[a];
            r2 += ra * ra;
        }
        if (r2 <= th * th) ++cnt;
        if (fabs(sqrt(r2) - th) <= band) ++near;
    }
    if (n_near) *n_near = near;
    return cnt;
}

double orc_score(const float* x, const float* y, int32_t n, const double* R, const double* t,
                 float theta, int32_t mode)
{
    const double th = (double)theta;
    double acc = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        const float* xk = x + 3 * (size_t)k;
        const float* yk = y + 3 * (size_t)k;
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double ra = R[a * 3 + 0] * (double)xk[0] + R[a * 3 + 1] * (double)xk[1]
                      + R[a * 3 + 2] * (double)xk[2] + t[a] - (double)yk[a];
            r2 += ra * ra;
        }
        if (mode == 0) acc += (r2 <= th * th) ? 1.0 : 0.0;
        else if (mode == 1) acc += fmin(sqrt(r2), th);
        else acc += fmin(r2, th * th);
    }
    return (mode == 0) ? acc : acc / (double)n;
}

/* ------------------------------------------------------------------ */
/* Whole path                                                          */
/* ------------------------------------------------------------------ */

int32_t orc_register(const float* x, const float* y, int32_t n, const orc_params* prm,
                     orc_result* res, int32_t* in_counts, int32_t* near_counts,
                     double* rt, uint8_t* hyp_valid, double* scores)
{
    memset(res, 0, sizeof(*res));
    res->R[0] = res->R[4] = res->R[8] = 1.0;
    res->hypothesis = -1;
    res->clique[0] = res->clique[1] = res->clique[2] = -1;
    if (n < 3) { res->status = 2; return 2; }
    if (prm->k1 < 1 || prm->k2 < 1 || !(prm->tau >= 0) || !(prm->theta > 0) ||
        prm->graph_mode < 0 || prm->graph_mode > 1 || prm->scoring < 0 || prm->scoring > 2) {
        res->status = 1; return 1;
    }
    const int32_t k1 = prm->k1, k2 = prm->k2;
    uint8_t* A = (uint8_t*)malloc((size_t)n * n);
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * n);
    int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * (size_t)k1);
    int32_t* pj = (int32_t*)malloc(sizeof(int32_t) * (size_t)k1);
    int32_t* pw = (int32_t*)malloc(sizeof(int32_t) * (size_t)k1);
    if (!A || !S || !pi || !pj || !pw) {
        free(A); free(S); free(pi); free(pj); free(pw);
        res->status = 4; return 4;
    }
    orc_compat(x, y, n, prm->tau, A);                      /* Eq. 1 */
    orc_sc2(A, n, S);                                      /* Eq. 2 */
    int32_t np = orc_pivots(S, n, k1, pi, pj, pw);         /* Eq. 4, Def. 2 */
    res->n_pivots = np;
    const int32_t nh = np * k2;
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nh ? nh : 1));
    uint8_t* va = (uint8_t*)malloc((size_t)(nh ? nh : 1));
    orc_cliques(S, n, pi, pj, np, k2, prm->graph_mode, cl, va);   /* Eq. 5-7 */
    int32_t best = -1, best_in = -1, nvalid = 0;
    double bestR[9], bestt[3], bestk = 0, best_sc = 0;
    for (int32_t h = 0; h < k1 * k2; ++h) {
        if (in_counts) in_counts[h] = -1;
        if (near_counts) near_counts[h] = 0;
        if (hyp_valid) hyp_valid[h] = 0;
        if (scores) scores[h] = NAN;
    }
    for (int32_t h = 0; h < nh; ++h) {
        if (!va[h]) continue;
        double xs[9], ys[9], R[9], t[3], kap;
        for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) {
                xs[a * 3 + d] = (double)x[3 * (size_t)cl[h * 3 + a] + d];
                ys[a * 3 + d] = (double)y[3 * (size_t)cl[h * 3 + a] + d];
            }
        if (!orc_kabsch(xs, ys, R, t, &kap)) continue;
        ++nvalid;
        int32_t near = 0;
        int32_t in = orc_inliers(x, y, n, R, t, prm->theta, prm->near_band, &near);
        if (in_counts) in_counts[h] = in;
        if (near_counts) near_counts[h] = near;
        if (hyp_valid) hyp_valid[h] = 1;
        if (rt) { memcpy(rt + (size_t)h * 12, R, sizeof(R)); memcpy(rt + (size_t)h * 12 + 9, t, sizeof(t)); }
        const double sc = (prm->scoring == 0) ? (double)in
                                              : orc_score(x, y, n, R, t, prm->theta, prm->scoring);
        if (scores) scores[h] = sc;
        /* Eq. 9 (largest IN) or the smallest capped error; lowest h on ties */
        const int better = (best < 0) || (prm->scoring == 0 ? sc > best_sc : sc < best_sc);
        if (better) {
            best_in = in; best = h; best_sc = sc;
            memcpy(bestR, R, sizeof(R)); memcpy(bestt, t, sizeof(t)); bestk = kap;
        }
    }
    res->n_valid = nvalid;
    if (best >= 0) {
        memcpy(res->R, bestR, sizeof(bestR));
        memcpy(res->t, bestt, sizeof(bestt));
        res->clique[0] = cl[best * 3 + 0];
        res->clique[1] = cl[best * 3 + 1];
        res->clique[2] = cl[best * 3 + 2];
        res->inlier_count = best_in;
        res->hypothesis = best;
        res->kappa = bestk;
        res->score = best_sc;
        res->status = 0;
    } else {
        res->status = 7;
    }
    free(A); free(S); free(pi); free(pj); free(pw); free(cl); free(va);
    return res->status;
}
