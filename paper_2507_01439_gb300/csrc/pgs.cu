// Stage 4: Pivot-Guided Search (Eq. 5-7, Alg. 1) on the O2Graph or on the
// undirected SC^2 graph.
//
// O2Graph (Def. 2), pivot p = (i, j) (i < j):
//   N(i,j) = { z : G~_iz > 0 and G~_jz > 0 }            (Eq. 5)
// On the O2Graph G~_iz > 0 needs i < z, so z > j; and for a pivot edge,
// G~_iz > 0 <=> G_iz = 1 (j is then a common neighbour of i and z).  So
//   N(i,j) = { z > j : G_iz = G_jz = 1 } = bits of (row_i AND row_j) above j.
//   S(z)   = W_ij + W_iz + W_jz                          (Eq. 6)
// and the K2 largest S (ties: lower z) form the pivot's TurboCliques (Eq. 7),
// written in the Alg. 2 layout h = r * |P| + p.  Empty slots are invalid.
// Undirected SC^2 graph: the same with z over every common neighbour
// (z != i, j follows from the zero diagonal) and W read symmetrically,
// W_ab = W_min(a,b),max(a,b) (only the upper triangle is stored).
//
// One warp per pivot: lane l ANDs bitset words l, l+32, ... of the two rows
// (four words of each row in flight per sweep), looks up the weights of its
// candidates eight at a time, keeps a private top-K2 list, and the warp
// merges the 32 lists with K2 rounds of a 64-bit max-reduction over keys
// (S << 32 | ~z).
#include "tr_common.cuh"
#include "tr_kabsch.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

template <int K2C>
__global__ void __launch_bounds__(256) pgs_kernel(ManyViews vs)
{
    pdl_wait();
    int lb;
    const ProbView v = vs.get(ST_PGS, blockIdx.x, lb);
    const int lane = threadIdx.x & 31;
    // pivots are in weight order and heavier pivots have more common neighbours:
    // warp w of block b takes pivot w * blocks + b, spreading them over the SMs
    const int p = (threadIdx.x >> 5) * ((v.k1 + 7) / 8) + lb;
    const int np = v.ctl->n_pivots;
    if (p >= np) return;
    const int k2 = K2C > 0 ? K2C : v.k2;
    const int4 pv = v.piv[p];
    const int i = pv.x, j = pv.y, wij = pv.z;
    const uint32_t* bi = v.bits + (size_t)i * v.ldb;
    const uint32_t* bj = v.bits + (size_t)j * v.ldb;
    const uint16_t* wi = v.w + (size_t)i * v.n_pad;
    const uint16_t* wj = v.w + (size_t)j * v.n_pad;
    const bool undirected = v.graph_mode == TURBOREG_GRAPH_SC2;

    constexpr int L = K2C > 0 ? K2C : TURBOREG_K2_MAX;
    uint64_t top[L];
#pragma unroll
    for (int r = 0; r < L; ++r) top[r] = 0ull;

    // candidate z are gathered 8 at a time so their 16 weight loads are in flight together
    int zb[8];
    int nz = 0;
    auto flush = [&]() {
        int wa[8], wb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int z = zb[q];
            if (q < nz) {
                // z > j > i on the O2Graph; the undirected search also meets z < j
                wa[q] = static_cast<int>(z > i ? wi[z] : v.w[(size_t)z * v.n_pad + i]);
                wb[q] = static_cast<int>(z > j ? wj[z] : v.w[(size_t)z * v.n_pad + j]);
            } else {
                wa[q] = wb[q] = 0;
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q >= nz) break;
            const int sz = wij + wa[q] + wb[q];
            const uint64_t key = (static_cast<uint64_t>(sz) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(zb[q]));
            if (key > top[L - 1]) {          // insertion into the descending list (keys are unique)
                uint64_t cur = key;
#pragma unroll
                for (int r = 0; r < L; ++r) {
                    if (cur > top[r]) {
                        const uint64_t t = top[r];
                        top[r] = cur;
                        cur = t;
                    }
                }
            }
        }
        nz = 0;
    };
    const int zs = undirected ? 0 : j + 1;
    const int w0 = zs >> 5;
    // lane l takes words w0 + l + 32 t; the 2 x 4 word loads of a sweep are in flight together
    for (int wb = w0 + lane; wb < v.ldb; wb += 32 * 4) {
        uint32_t mw[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int wd = wb + 32 * t;
            mw[t] = wd < v.ldb ? (bi[wd] & bj[wd]) : 0u;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int wd = wb + 32 * t;
            uint32_t m = mw[t];
            if (wd == w0) m &= ~0u << (zs & 31);
            while (m) {
                zb[nz++] = wd * 32 + __ffs(m) - 1;
                m &= m - 1;
                if (nz == 8) flush();
            }
        }
    }
    if (nz) flush();
    // warp merge: k2 rounds of argmax over the lanes' list heads; lane r keeps
    // round r's clique and solves its Kabsch afterwards
    int head = 0;
    int4 mine_cl = make_int4(i, j, -1, 0);
    for (int r = 0; r < k2; ++r) {
        uint64_t mine = 0ull;
#pragma unroll
        for (int q = 0; q < L; ++q)
            if (q == head) mine = top[q];
        uint64_t best = mine;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const uint64_t o = __shfl_xor_sync(0xffffffffu, best, off);
            best = o > best ? o : best;
        }
        if (best == mine && mine != 0ull) ++head;
        const int4 cl = best != 0ull
            ? make_int4(i, j, static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(best & 0xFFFFFFFFull)), 1)
            : make_int4(i, j, -1, 0);
        if (lane == 0) v.cliques[static_cast<size_t>(r) * np + p] = cl;
        if (lane == r) mine_cl = cl;
    }
    // Kabsch of this pivot's cliques (Sec. 3.5), one lane each
    if (lane < k2) kabsch_hypothesis(v, lane * np + p, mine_cl);
}

}  // namespace

// k2 is the common K2 of the batch, or 0 when problems differ (generic list)
void launch_pgs(const Batch& b, int total, int k2, cudaStream_t s)
{
    const ManyViews vs{b};
    switch (k2) {
        case 1: launch_pdl(pgs_kernel<1>, total, 256, 0, s, vs); break;
        case 2: launch_pdl(pgs_kernel<2>, total, 256, 0, s, vs); break;
        case 3: launch_pdl(pgs_kernel<3>, total, 256, 0, s, vs); break;
        case 4: launch_pdl(pgs_kernel<4>, total, 256, 0, s, vs); break;
        default: launch_pdl(pgs_kernel<0>, total, 256, 0, s, vs); break;
    }
}

}  // namespace tr
