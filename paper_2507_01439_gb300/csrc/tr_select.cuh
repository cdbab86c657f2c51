// Threshold step of the exact top-K1 pivot selection (Eq. 4), shared by the
// standalone select kernel and the count kernel's blocks.
#pragma once

#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

// Block-wide inclusive scan of one int per thread (blockDim.x a multiple of
// 32, at most 1024); sbuf holds 33 ints of shared memory.
__device__ __forceinline__ int block_incl_scan(int x, int* sbuf)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = static_cast<int>(blockDim.x >> 5);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) sbuf[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nwarps ? sbuf[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += y;
        }
        sbuf[lane] = t;
    }
    __syncthreads();
    const int r = x + (warp > 0 ? sbuf[warp - 1] : 0);
    __syncthreads();
    return r;
}

// From the weight histogram: |E+|, n_sel = min(K1, |E+|), alpha = the K1-th
// largest weight, c_gt = #{W > alpha}, m = n_sel - c_gt ties still needed.
// Every thread of the block must call it.  stage: optional shared memory of
// n + 4 words (16-byte aligned); the histogram is then copied there in one
// coalesced round (16-byte loads when the histogram is 16-byte aligned) and
// both passes below read it from there.  res: optional shared memory of five
// words that receives (|E+|, n_sel, alpha, c_gt, m) instead of the problem's
// control block; the caller synchronises the block before reading it.
__device__ __forceinline__ void select_alpha(const ProbView& v, int* sbuf, uint32_t* stage = nullptr,
                                             int* res = nullptr)
{
    const int nb = v.n;                       // weights 1..n (W <= n - 2)
    const uint32_t* H = v.hist;
    if (stage != nullptr && (reinterpret_cast<uintptr_t>(v.hist) & 15u) == 0u) {
        const int nq = (nb + 4) >> 2;         // 16-byte words covering bins 0..n
        const uint4* H4 = reinterpret_cast<const uint4*>(v.hist);
        for (int q0 = threadIdx.x; q0 < nq; q0 += 8 * blockDim.x) {
            uint4 h4[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * static_cast<int>(blockDim.x);
                h4[u] = q < nq ? __ldcg(H4 + q) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * static_cast<int>(blockDim.x);
                if (q < nq) reinterpret_cast<uint4*>(stage)[q] = h4[u];
            }
        }
        __syncthreads();
        H = stage;
    } else if (stage != nullptr) {
        for (int q0 = threadIdx.x + 1; q0 <= nb; q0 += 8 * blockDim.x) {
            uint32_t h8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int b = q0 + q * static_cast<int>(blockDim.x);
                h8[q] = b <= nb ? __ldcg(v.hist + b) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int b = q0 + q * static_cast<int>(blockDim.x);
                if (b <= nb) stage[b] = h8[q];
            }
        }
        __syncthreads();
        H = stage;
    }
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    // thread t owns weights (hi - per, hi], hi = n - t*per, scanned from the top
    const int hi = nb - static_cast<int>(threadIdx.x) * per;
    int mine = 0;
    for (int q0 = 0; q0 < per; q0 += 8) {       // 8 loads in flight per step
        uint32_t h8[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int wv = hi - q0 - q;
            h8[q] = (q0 + q < per && wv >= 1) ? H[wv] : 0u;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) mine += static_cast<int>(h8[q]);
    }
    const int incl = block_incl_scan(mine, sbuf);
    if (threadIdx.x == blockDim.x - 1) sbuf[32] = incl;
    __syncthreads();
    const int n_edges = sbuf[32];
    const int n_sel = n_edges < v.k1 ? n_edges : v.k1;
    // result k of (n_edges, n_sel, alpha, c_gt, m_ties)
    auto put = [&](int k, int val) {
        if (res != nullptr) {
            res[k] = val;
            return;
        }
        switch (k) {
            case 0: v.ctl->n_edges = val; break;
            case 1: v.ctl->n_sel = val; break;
            case 2: v.ctl->alpha = val; break;
            case 3: v.ctl->c_gt = val; break;
            default: v.ctl->m_ties = val; break;
        }
    };
    if (threadIdx.x == 0) {
        put(0, n_edges);
        put(1, n_sel);
        if (n_sel == 0) {
            put(2, 0x7FFFFFFF);
            put(3, 0);
            put(4, 0);
        }
    }
    if (n_sel == 0) return;
    const int excl = incl - mine;
    if (excl < n_sel && n_sel <= incl) {
        // the thread holding the K1-th edge walks its bins from the top, eight
        // loads in flight per step
        int run = excl;
        bool done = false;
        for (int q0 = 0; q0 < per && !done; q0 += 8) {
            uint32_t h8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int wv = hi - q0 - q;
                h8[q] = (q0 + q < per && wv >= 1) ? H[wv] : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int wv = hi - q0 - q;
                if (done || q0 + q >= per || wv < 1) continue;
                const int h = static_cast<int>(h8[q]);
                if (run + h >= n_sel) {
                    put(2, wv);
                    put(3, run);
                    put(4, n_sel - run);
                    done = true;
                } else {
                    run += h;
                }
            }
        }
    }
}

}  // namespace tr
