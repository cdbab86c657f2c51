// Stage 0 (pack) and stage 1 (compatibility graph, Eq. 1).
//
// pack:   [N][3] x, y (host-order float32, any 4-byte alignment) -> structure
//         of arrays pts[6][n_pad] with zero padding; flags NaN/Inf; clears the
//         per-call accumulators.
// compat: G_ij = [ | ||x_i - x_j|| - ||y_i - y_j|| | <= tau ], i != j, G_ii = 0
//         (Eq. 1; zero diagonal because App. B equates G^_ij with the number
//         of triangles on edge (i,j)).  Written twice: as FP8 E4M3 0/1 bytes
//         (the operand of the SC^2 tensor-core GEMM) and as a row bitset
//         (the operand of clique search), plus the degree of every node.
//
// Exactness: the decision is taken in FP32 and, for the few pairs whose FP32
// |dX - dY| lies within a rounding guard band g of tau, retaken in FP64 with
// the fixed operation order ((dx*dx + dy*dy) + dz*dz), correctly rounded
// sqrt.  FP32 error analysis (u = 2^-24): each distance carries relative
// error <= 3.5u, so |diff32 - diff_exact| <= 4.5u (dX + dY); the FP64
// evaluation is within 4.5 * 2^-53 (dX + dY) of exact.  With
// g = 2^-21 (dX + dY) + 1e-18 (absolute slack for underflowed squares) any
// pair outside the band is decided identically in FP32 and FP64, so the
// whole matrix equals the FP64 evaluation bit for bit.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kRows = 64;    // rows (i) per block, staged in shared memory by TMA
constexpr int kCols = 256;   // columns (j) per block, one per thread

__global__ void __launch_bounds__(256) pack_kernel(ProbView v, const float* __restrict__ src,
                                                   const float* __restrict__ dst)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    bool bad = false;
    for (int k = tid; k < v.n_pad; k += stride) {
        float a[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (k < v.n) {
            a[0] = src[3 * k + 0]; a[1] = src[3 * k + 1]; a[2] = src[3 * k + 2];
            a[3] = dst[3 * k + 0]; a[4] = dst[3 * k + 1]; a[5] = dst[3 * k + 2];
#pragma unroll
            for (int c = 0; c < 6; ++c) bad |= !isfinite(a[c]);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) v.pts[(size_t)c * v.n_pad + k] = a[c];
        v.rowscore[k] = 0;
        v.deg[k] = 0;
        v.rowcnt[k] = 0;
    }
    for (int k = tid; k <= v.n_pad; k += stride) v.hist[k] = 0;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&v.ctl->err, TR_ERR_NONFINITE);
}

__device__ __forceinline__ bool compat_pair(const float xi[6], const float xj[6], float tau)
{
    // FP32 evaluation, no contraction (explicit round-to-nearest intrinsics)
    const float ax = __fsub_rn(xi[0], xj[0]), ay = __fsub_rn(xi[1], xj[1]), az = __fsub_rn(xi[2], xj[2]);
    const float bx = __fsub_rn(xi[3], xj[3]), by = __fsub_rn(xi[4], xj[4]), bz = __fsub_rn(xi[5], xj[5]);
    const float sX = __fadd_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)), __fmul_rn(az, az));
    const float sY = __fadd_rn(__fadd_rn(__fmul_rn(bx, bx), __fmul_rn(by, by)), __fmul_rn(bz, bz));
    const float dX = __fsqrt_rn(sX), dY = __fsqrt_rn(sY);
    const float diff = fabsf(__fsub_rn(dX, dY));
    const float g = __fmaf_rn(__fadd_rn(dX, dY), 4.76837158203125e-07f, 1e-18f);  // 2^-21 (dX+dY) + slack
    if (fabsf(__fsub_rn(diff, tau)) > g) return diff <= tau;   // false for NaN/Inf -> FP64 path
    // FP64 re-evaluation in the reference operation order
    const double dx = __dsub_rn((double)xi[0], (double)xj[0]);
    const double dy = __dsub_rn((double)xi[1], (double)xj[1]);
    const double dz = __dsub_rn((double)xi[2], (double)xj[2]);
    const double ex = __dsub_rn((double)xi[3], (double)xj[3]);
    const double ey = __dsub_rn((double)xi[4], (double)xj[4]);
    const double ez = __dsub_rn((double)xi[5], (double)xj[5]);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    double t = __dmul_rn(ex, ex);
    t = __dadd_rn(t, __dmul_rn(ey, ey));
    t = __dadd_rn(t, __dmul_rn(ez, ez));
    const double DX = __dsqrt_rn(s), DY = __dsqrt_rn(t);
    return fabs(__dsub_rn(DX, DY)) <= (double)tau;
}

// Block = 256 threads = 8 warps; covers rows [i0, i0+64) x cols [j0, j0+256).
// The 64 row points are staged in shared memory with 1-D TMA bulk copies;
// each thread keeps its column point in registers.
__global__ void __launch_bounds__(256) compat_kernel(ProbView v)
{
    __shared__ __align__(128) float sx[6][kRows];
    __shared__ __align__(16) uint8_t tile[kRows][kCols];
    __shared__ int sdeg[kRows];
    __shared__ __align__(8) uint64_t bar;

    const int j0 = blockIdx.x * kCols;
    const int i0 = blockIdx.y * kRows;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < kRows) sdeg[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, 6 * kRows * sizeof(float));
#pragma unroll
        for (int c = 0; c < 6; ++c)
            bulk_g2s(&sx[c][0], v.pts + (size_t)c * v.n_pad + i0, kRows * sizeof(float), &bar);
    }
    const int j = j0 + threadIdx.x;
    float xj[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xj[c] = v.pts[(size_t)c * v.n_pad + j];
    const bool jok = j < v.n;
    if (!mbar_wait(&bar, 0)) {
        if (threadIdx.x == 0) atomicOr(&v.ctl->err, TR_ERR_TIMEOUT);
        return;
    }
    const float tau = v.tau;
    for (int r = 0; r < kRows; ++r) {
        const int i = i0 + r;
        bool a = false;
        if (jok && i < v.n && i != j) {
            float xi[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) xi[c] = sx[c][r];
            a = compat_pair(xi, xj, tau);
        }
        tile[r][threadIdx.x] = a ? 0x38 : 0x00;   // FP8 E4M3: 0x38 = 1.0
        const unsigned bal = __ballot_sync(0xffffffffu, a);
        if (lane == 0) {
            v.bits[(size_t)i * v.ldb + (j0 >> 5) + warp] = bal;
            if (bal) atomicAdd(&sdeg[r], __popc(bal));
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kRows * kCols / 16; q += blockDim.x) {
        const int r = q / (kCols / 16), c16 = q % (kCols / 16);
        *reinterpret_cast<uint4*>(v.a8 + (size_t)(i0 + r) * v.n_pad + j0 + c16 * 16) =
            *reinterpret_cast<const uint4*>(&tile[r][c16 * 16]);
    }
    if (threadIdx.x < kRows && sdeg[threadIdx.x]) atomicAdd(&v.deg[i0 + threadIdx.x], sdeg[threadIdx.x]);
}

}  // namespace

void launch_pack(const ProbView& v, const float* src, const float* dst, cudaStream_t s)
{
    const int blocks = (v.n_pad + 255) / 256;
    pack_kernel<<<blocks, 256, 0, s>>>(v, src, dst);
}

void launch_compat(const ProbView& v, cudaStream_t s)
{
    dim3 grid(v.n_pad / kCols, v.n_pad / kRows);
    compat_kernel<<<grid, 256, 0, s>>>(v);
}

}  // namespace tr
