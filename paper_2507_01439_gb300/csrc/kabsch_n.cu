// Kabsch over cliques of k >= 4 matches (the 3-clique vs 10-clique study of
// the appendix, App. A.2): the proper rotation R and translation t that
// minimise sum_a ||R x_a + t - y_a||^2 over the clique's matches.
//
// One thread per clique, FP64.  With a_a = x_a - mean(x), b_a = y_a - mean(y)
// and S = sum_a a_a b_a^T, the optimal unit quaternion is the eigenvector of
// the largest eigenvalue of Horn's symmetric 4x4 matrix
//   N = [[Sxx+Syy+Szz, Syz-Szy,      Szx-Sxz,      Sxy-Syx     ],
//        [Syz-Szy,     Sxx-Syy-Szz,  Sxy+Syx,      Szx+Sxz     ],
//        [Szx-Sxz,     Sxy+Syx,     -Sxx+Syy-Szz,  Syz+Szy     ],
//        [Sxy-Syx,     Szx+Sxz,      Syz+Szy,     -Sxx-Syy+Szz ]]
// (Horn, JOSA A 1987), found here by cyclic Jacobi rotations.  Sorted
// descending, N's eigenvalues are s1+s2+s3', s1-s2-s3', -s1+s2-s3',
// -s1-s2+s3' (s_i the singular values of S, s3' = sign(det S) s3), so
// s1 = (l1 + l2) / 2 and s2 = (l1 + l3) / 2 give kappa = s1/s2 without a
// separate SVD.  A clique with s2 <= 1e-12 s1 (collinear) is invalid.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

// Cyclic Jacobi eigen-decomposition of a symmetric 4x4 matrix: A becomes
// (numerically) diagonal, V holds the eigenvectors as columns.  Each
// rotation in plane (p, q) uses t = tan(phi) from
// theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
// which zeroes a_pq; at most 24 sweeps (quadratic convergence needs a few).
__device__ void jacobi4(double A[4][4], double V[4][4])
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) V[r][c] = r == c ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 24; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
                tot += A[r][c] * A[r][c];
                if (r < c) off += A[r][c] * A[r][c];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < 3; ++p) {
            for (int q = p + 1; q < 4; ++q) {
                const double apq = A[p][q];
                if (apq == 0.0) continue;
                const double th = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0);
                const double s = t * c;
                for (int r = 0; r < 4; ++r) {
                    const double arp = A[r][p], arq = A[r][q];
                    A[r][p] = c * arp - s * arq;
                    A[r][q] = s * arp + c * arq;
                }
                for (int r = 0; r < 4; ++r) {
                    const double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = c * apr - s * aqr;
                    A[q][r] = s * apr + c * aqr;
                }
                for (int r = 0; r < 4; ++r) {
                    const double vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = c * vrp - s * vrq;
                    V[r][q] = s * vrp + c * vrq;
                }
            }
        }
    }
}

// idx: [m][k] match indices (checked on the host to lie in [0, n)).
// out: rt rows of the verification layout: R (9), t (3), kappa, flags (1 = valid).
__global__ void __launch_bounds__(128) kabsch_n_kernel(const float* __restrict__ pts8,
                                                       const int32_t* __restrict__ idx, int k, int m,
                                                       float* __restrict__ out_rt)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= m) return;
    const int32_t* id = idx + (size_t)h * k;
    double cx[3] = {0, 0, 0}, cy[3] = {0, 0, 0};
    for (int a = 0; a < k; ++a) {
        const float4* r = reinterpret_cast<const float4*>(pts8 + (size_t)id[a] * 8);
        const float4 u = r[0], w = r[1];
        cx[0] += u.x; cx[1] += u.y; cx[2] += u.z;
        cy[0] += u.w; cy[1] += w.x; cy[2] += w.y;
    }
    for (int d = 0; d < 3; ++d) {
        cx[d] /= k;
        cy[d] /= k;
    }
    double S[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < k; ++a) {
        const float4* r = reinterpret_cast<const float4*>(pts8 + (size_t)id[a] * 8);
        const float4 u = r[0], w = r[1];
        const double p[3] = {u.x - cx[0], u.y - cx[1], u.z - cx[2]};
        const double q[3] = {u.w - cy[0], w.x - cy[1], w.y - cy[2]};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) S[i][j] += p[i] * q[j];
    }
    double N[4][4] = {
        {S[0][0] + S[1][1] + S[2][2], S[1][2] - S[2][1], S[2][0] - S[0][2], S[0][1] - S[1][0]},
        {S[1][2] - S[2][1], S[0][0] - S[1][1] - S[2][2], S[0][1] + S[1][0], S[2][0] + S[0][2]},
        {S[2][0] - S[0][2], S[0][1] + S[1][0], -S[0][0] + S[1][1] - S[2][2], S[1][2] + S[2][1]},
        {S[0][1] - S[1][0], S[2][0] + S[0][2], S[1][2] + S[2][1], -S[0][0] - S[1][1] + S[2][2]}};
    double V[4][4];
    jacobi4(N, V);
    // eigenvalues descending: track the order of the four diagonal entries
    int o[4] = {0, 1, 2, 3};
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (N[o[j]][o[j]] > N[o[i]][o[i]]) {
                const int t = o[i];
                o[i] = o[j];
                o[j] = t;
            }
    const double l1 = N[o[0]][o[0]], l2 = N[o[1]][o[1]], l3 = N[o[2]][o[2]];
    const double s1 = 0.5 * (l1 + l2), s2 = 0.5 * (l1 + l3);
    double qw = V[0][o[0]], qx = V[1][o[0]], qy = V[2][o[0]], qz = V[3][o[0]];
    const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= qn; qx /= qn; qy /= qn; qz /= qn;
    const double R[9] = {qw * qw + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                         2 * (qx * qy + qw * qz), qw * qw - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - qw * qx),
                         2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), qw * qw - qx * qx - qy * qy + qz * qz};
    float* out = out_rt + (size_t)h * 16;
    const bool valid = s1 > 0.0 && s2 > 1e-12 * s1;
    for (int r = 0; r < 9; ++r) out[r] = static_cast<float>(R[r]);
    for (int r = 0; r < 3; ++r)
        out[9 + r] = static_cast<float>(cy[r] - (R[3 * r] * cx[0] + R[3 * r + 1] * cx[1] + R[3 * r + 2] * cx[2]));
    out[12] = static_cast<float>(s2 > 0.0 ? s1 / s2 : INFINITY);
    out[13] = __int_as_float(valid ? 1 : 0);
    out[14] = out[15] = 0.f;
}

}  // namespace

void launch_kabsch_n(const ProbView& v, const int32_t* idx, int k, int m, cudaStream_t s)
{
    kabsch_n_kernel<<<(m + 127) / 128, 128, 0, s>>>(v.pts8, idx, k, m, v.rt);
}

}  // namespace tr
