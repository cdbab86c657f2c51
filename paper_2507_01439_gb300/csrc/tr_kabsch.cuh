// Closed-form 3-point Kabsch (Sec. 3.5), shared by the clique search (which
// solves each pivot's cliques as soon as it has chosen them) and by the
// clique-Kabsch entry point.
//
// Closed-form 3-point Kabsch.  With a_k = x_k - mean(x), b_k = y_k - mean(y)
// the cross-covariance H = sum_k a_k b_k^T has rank <= 2 (three points are
// coplanar).  Write a_k = E P_k, b_k = F Q_k with E = [e1 e2], F = [f1 f2]
// orthonormal in-plane frames and n_x = e1 x e2, n_y = f1 x f2.  Then
// H = E M F^T with the 2x2 M = sum_k P_k Q_k^T, and every proper rotation
// maximising tr(R H) has the form R = F X E^T + det(X) n_y n_x^T with X in
// O(2) maximising tr(X M):
//   rotation   X = [[c,-s],[s,c]] : tr = c(m11+m22) + s(m12-m21)
//   reflection X = [[c,s],[s,-c]] : tr = c(m11-m22) + s(m12+m21)
// The larger of the two vector norms is sigma1 + sigma2, the smaller
// |sigma1 - sigma2| (singular values of M, hence of H), and (c, s) is the
// normalised winning vector.  No iteration, no atan2.
//
// Precision: FP32.  For a thin triangle (kappa = sigma1/sigma2 large) all of
// the closed form's rounding error enters through the triangle normal, a
// cross product of two nearly parallel edges (relative error ~ u kappa); the
// frames, projections and the 2x2 step are well conditioned.  So when kappa
// exceeds the bound (default 100) or the FP32 frames are undefined, the two
// normals are recomputed in FP64 from exact FP64 differences of the FP32
// inputs, rounded to FP32, and the rest is redone in FP32: checked against the
// FP64 SVD, the rotation then stays within ~4e-7 of it up to kappa ~ 1e5,
// where the all-FP32 form is off by ~4e-3.  The clique search computes these
// FP64 components with six lanes per clique (one per triangle and component),
// so a warp issues a dozen FP64 instructions instead of a hundred.  A clique
// with sigma2 <= 1e-12 sigma1 (collinear or repeated points) is invalid.
#pragma once

#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

template <typename T>
__device__ __forceinline__ T inv_sqrt(T x);
template <>
__device__ __forceinline__ float inv_sqrt<float>(float x) { return 1.0f / sqrtf(x); }
template <typename T>
struct KabschOut {
    T R[9];
    T t[3];
    T kappa;
    bool ok;    // frames defined and sigma1 > 0
    T s1, s2;
};

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
__device__ __forceinline__ T dot3(const T a[3], const T b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Component c of the normal (p1 - p0) x (p2 - p0) in FP64 from exact FP64
// differences of the FP32 coordinates, rounded to FP32.
__device__ __forceinline__ float exact_normal_comp(const float (&p)[3][3], int c)
{
    const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
    const double a1 = static_cast<double>(p[1][c1]) - static_cast<double>(p[0][c1]);
    const double a2 = static_cast<double>(p[1][c2]) - static_cast<double>(p[0][c2]);
    const double b1 = static_cast<double>(p[2][c1]) - static_cast<double>(p[0][c1]);
    const double b2 = static_cast<double>(p[2][c2]) - static_cast<double>(p[0][c2]);
    return static_cast<float>(__fma_rn(a1, b2, -__dmul_rn(a2, b1)));
}

// In-plane orthonormal frame of a triangle: e1 along its longest edge,
// n = unit normal of (p1 - p0) x (p2 - p0), e2 = n x e1.  ng: the normal's
// components given by the caller (FP64 cross product rounded to FP32), and
// then *nlen receives their length |(p1 - p0) x (p2 - p0)| (twice the area).
template <typename T, bool kGiven>
__device__ __forceinline__ bool frame3(const T p[3][3], T e1[3], T e2[3], T nrm[3], const T* ng, T* nlen)
{
    T d01[3], d02[3], d12[3];
    for (int c = 0; c < 3; ++c) {
        d01[c] = p[1][c] - p[0][c];
        d02[c] = p[2][c] - p[0][c];
        d12[c] = p[2][c] - p[1][c];
    }
    if (kGiven) {
        nrm[0] = ng[0]; nrm[1] = ng[1]; nrm[2] = ng[2];
    } else {
        cross3(d01, d02, nrm);
    }
    const T nn = dot3(nrm, nrm);
    if (kGiven) *nlen = sqrt(nn);
    const T l01 = dot3(d01, d01), l02 = dot3(d02, d02), l12 = dot3(d12, d12);
    int sel = 0;   // longest edge, selected by value (no pointer into local arrays)
    T le = l01;
    if (l02 > le) { sel = 1; le = l02; }
    if (l12 > le) { sel = 2; le = l12; }
    if (!(nn > T(0)) || !(le > T(0))) return false;
    const T in = inv_sqrt(nn), ie = inv_sqrt(le);
    for (int c = 0; c < 3; ++c) {
        nrm[c] *= in;
        e1[c] = (sel == 0 ? d01[c] : sel == 1 ? d02[c] : d12[c]) * ie;
    }
    cross3(nrm, e1, e2);
    return true;
}

// kGiven: the two triangles' normals nxg, nyg are given by the caller (the
// FP64 path); otherwise they are the FP32 cross products.
template <typename T, bool kGiven = false>
__device__ __forceinline__ void kabsch3(const T p[3][3], const T q[3][3], KabschOut<T>& o, const T* nxg = nullptr,
                                        const T* nyg = nullptr)
{
    T cx[3], cy[3];
    for (int c = 0; c < 3; ++c) {
        cx[c] = (p[0][c] + p[1][c] + p[2][c]) * T(1.0 / 3.0);
        cy[c] = (q[0][c] + q[1][c] + q[2][c]) * T(1.0 / 3.0);
    }
    T e1[3], e2[3], nx[3], f1[3], f2[3], ny[3];
    T lx = T(0), ly = T(0);
    o.ok = frame3<T, kGiven>(p, e1, e2, nx, nxg, &lx) && frame3<T, kGiven>(q, f1, f2, ny, nyg, &ly);
    if (!o.ok) {
        o.kappa = T(INFINITY);
        o.s1 = o.s2 = T(0);
        return;
    }
    T m11 = 0, m12 = 0, m21 = 0, m22 = 0;
    for (int k = 0; k < 3; ++k) {
        T a[3], b[3];
        for (int c = 0; c < 3; ++c) {
            a[c] = p[k][c] - cx[c];
            b[c] = q[k][c] - cy[c];
        }
        const T P1 = dot3(a, e1), P2 = dot3(a, e2);
        const T Q1 = dot3(b, f1), Q2 = dot3(b, f2);
        m11 += P1 * Q1; m12 += P1 * Q2;
        m21 += P2 * Q1; m22 += P2 * Q2;
    }
    const T rx = m11 + m22, ry = m12 - m21;   // rotation candidate
    const T fx = m11 - m22, fy = m12 + m21;   // reflection candidate
    const T r2 = rx * rx + ry * ry, q2 = fx * fx + fy * fy;
    if (!(r2 > T(0) || q2 > T(0))) {
        o.ok = false;
        o.kappa = T(INFINITY);
        o.s1 = o.s2 = T(0);
        return;
    }
    const bool rot = r2 >= q2;
    const T ih = inv_sqrt(rot ? r2 : q2);               // 1 / (sigma1 + sigma2)
    const T hi = (rot ? r2 : q2) * ih;
    const T lo2 = rot ? q2 : r2;
    const T lo = lo2 > T(0) ? lo2 * inv_sqrt(lo2) : T(0);
    o.s1 = (hi + lo) * T(0.5);
    o.s2 = (hi - lo) * T(0.5);
    if (kGiven && o.s1 > T(0)) {
        // sigma2 of a thin clique from sigma1 sigma2 = |det M| = |n_x| |n_y| / 3
        // (Cauchy-Binet over three centred points), with the lengths of the
        // accurate normals, instead of the cancelling difference (hi - lo) / 2
        o.s2 = lx * ly / (T(3) * o.s1);
    }
    o.kappa = o.s2 > T(0) ? static_cast<T>(static_cast<float>(o.s1) / static_cast<float>(o.s2)) : T(INFINITY);
    T X00, X01, X10, X11, sg;
    if (rot) {
        const T c = rx * ih, s = ry * ih;
        X00 = c; X01 = -s; X10 = s; X11 = c; sg = T(1);
    } else {
        const T c = fx * ih, s = fy * ih;
        X00 = c; X01 = s; X10 = s; X11 = -c; sg = T(-1);
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            o.R[r * 3 + c] = X00 * f1[r] * e1[c] + X01 * f1[r] * e2[c] + X10 * f2[r] * e1[c] +
                             X11 * f2[r] * e2[c] + sg * ny[r] * nx[c];
    for (int r = 0; r < 3; ++r)
        o.t[r] = cy[r] - (o.R[r * 3 + 0] * cx[0] + o.R[r * 3 + 1] * cx[1] + o.R[r * 3 + 2] * cx[2]);
}

__device__ __forceinline__ void load_clique(const ProbView& v, const int4 cl, float p[3][3], float q[3][3])
{
    const int idx[3] = {cl.x, cl.y, cl.z};
    for (int a = 0; a < 3; ++a) {
        const float4* r = reinterpret_cast<const float4*>(v.pts8 + (size_t)idx[a] * 8);
        const float4 u = r[0], w = r[1];
        p[a][0] = u.x; p[a][1] = u.y; p[a][2] = u.z;
        q[a][0] = u.w; q[a][1] = w.x; q[a][2] = w.y;
    }
}

// Writes hypothesis h: R, t and kappa of a solved clique (flags: 1 valid,
// 2 the FP64 normals were used), zero for an empty slot; the inlier count
// and score are cleared.
__device__ __forceinline__ void store_hypothesis(const ProbView& v, int h, bool present, const KabschOut<float>& o,
                                                 uint32_t flags)
{
    v.inl[h] = 0;
    v.score[h] = 0ull;
    float o16[13];
#pragma unroll
    for (int r = 0; r < 13; ++r) o16[r] = 0.f;
    if (present) {
        if (o.ok && o.s1 > 0.f && o.s2 > 1e-12f * o.s1) {
#pragma unroll
            for (int r = 0; r < 9; ++r) o16[r] = o.R[r];
#pragma unroll
            for (int r = 0; r < 3; ++r) o16[9 + r] = o.t[r];
            flags |= 1u;
        }
        o16[12] = o.kappa;
    } else {
        flags = 0u;
    }
    float4* o4 = reinterpret_cast<float4*>(v.rt + (size_t)h * 16);
    o4[0] = make_float4(o16[0], o16[1], o16[2], o16[3]);
    o4[1] = make_float4(o16[4], o16[5], o16[6], o16[7]);
    o4[2] = make_float4(o16[8], o16[9], o16[10], o16[11]);
    o4[3] = make_float4(o16[12], __int_as_float(static_cast<int>(flags)), 0.f, 0.f);
}

// Closed form of hypothesis h with clique cl by one thread (the FP64 normals,
// when needed, computed by the same thread).
__device__ __forceinline__ void kabsch_hypothesis(const ProbView& v, int h, int4 cl)
{
    KabschOut<float> o;
    uint32_t flags = 0;
    if (cl.w) {
        float p[3][3], q[3][3];
        load_clique(v, cl, p, q);
        kabsch3<float>(p, q, o);
        if (!(o.ok && o.kappa <= v.kappa_fp64)) {   // ill-conditioned: FP64 normals
            float nx[3], ny[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nx[c] = exact_normal_comp(p, c);
                ny[c] = exact_normal_comp(q, c);
            }
            kabsch3<float, true>(p, q, o, nx, ny);
            flags = 2u;
        }
    }
    store_hypothesis(v, h, cl.w != 0, o, flags);
}

}  // namespace

}  // namespace tr
