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
// One warp per selected edge (Eq. 4, in the order the selection wrote
// them): the warp first finds the edge's pivot index, its rank among the
// selected keys (staged once per block in shared memory), and writes the
// pivot list entry; all outputs go to that index.  Candidates: every lane
// loads its share of both rows'
// bitset words at once (eight words of each per lane in flight), and the
// warp compacts the set bits of their AND into a per-warp list in shared
// memory (popcount prefix sums).  Scoring: lanes take list entries
// l, l + 32, ..., eight at a time so that their 16 weight loads are in
// flight together (sixteen at a time measured slower), and keep private top-K2 lists of keys (S << 32 | ~z); the warp
// merges the 32 lists with K2 rounds of a 64-bit max-reduction.  A list that
// would overflow is scored and emptied first, so any graph density works.
//
// Kabsch (Sec. 3.5): lane r solves clique r in FP32; for ill-conditioned
// cliques the warp computes the FP64 triangle normals with six lanes per
// clique (triangle x or y, component 0..2) and lane r redoes the closed form
// with them.
#include "tr_common.cuh"
#include "tr_kabsch.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kCand = 1024;   // per-warp candidate list (z indices)
constexpr int kListBytes = 8 * kCand * 4;   // the 8 warps' lists
constexpr int kWords = 8;     // bitset words per lane per load round
constexpr int kBatch = 8;     // list entries per lane per scoring round (16 weight loads in flight)

// kDense: registers bounded for three blocks per SM (a batch: many waves of
// blocks, latency hidden by occupancy); otherwise two, with more registers
// per warp (one problem: a single wave)
template <int K2C, bool kDense = false>
__global__ void __launch_bounds__(256, kDense ? 3 : 2) pgs_kernel(ManyViews vs)
{
    // dynamic shared memory: per-warp candidate lists, then the selected edge keys
    extern __shared__ __align__(16) uint8_t pgs_smem[];
    int (*scand)[kCand] = reinterpret_cast<int (*)[kCand]>(pgs_smem);
    uint64_t* skey = reinterpret_cast<uint64_t*>(pgs_smem + kListBytes);
    int lb;
    const ProbView v = vs.get(ST_PGS, blockIdx.x, lb);   // launch descriptors: before the wait
    pdl_wait();
    pdl_release();   // the balanced verification tile caps itself at four blocks per SM, so
                     // blocks placed beside these still end up evenly spread
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the selected edges (Eq. 4) in the order the selection wrote them; a
    // pivot's index is its rank: the number of larger keys (W << 32 | ~(i n + j)
    // are unique, larger = heavier, then lower (i, j)).  All K1 key slots are
    // staged in the same round of loads as the number of selected edges (the
    // selection fills the first n_sel; the rest are ignored).
    const int np = v.ctl->n_sel;   // through L1: every warp of every block reads it
    const int kcap = v.k1;
    // warp w of block b takes selected edge w * blocks + b
    const int c = warp * ((kcap + 7) / 8) + lb;
    const uint64_t mykey = c < kcap ? __ldcg(v.cand + c) : 0ull;
    for (int q0 = threadIdx.x; q0 < kcap; q0 += 8 * static_cast<int>(blockDim.x)) {
        uint64_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * static_cast<int>(blockDim.x);
            kk[u] = q < kcap ? __ldcg(v.cand + q) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + u * static_cast<int>(blockDim.x);
            if (q < kcap) skey[q] = kk[u];
        }
    }
    if (lb == 0 && threadIdx.x == 0) v.ctl->n_pivots = np;
    const uint32_t lin = 0xFFFFFFFFu - static_cast<uint32_t>(mykey & 0xFFFFFFFFull);
    const int i = c < np ? static_cast<int>(lin / static_cast<uint32_t>(v.n)) : 0;
    const int j = c < np ? static_cast<int>(lin % static_cast<uint32_t>(v.n)) : 0;
    const int wij = static_cast<int>(mykey >> 32);
    const bool undirected = v.graph_mode == TURBOREG_GRAPH_SC2;
    const uint32_t* bi = v.bits + (size_t)i * v.ldb;
    const uint32_t* bj = v.bits + (size_t)j * v.ldb;
    // the first round of this pivot's bitset words, in flight across the
    // block barrier and the rank count
    const int zs = undirected ? 0 : j + 1;
    const int w0 = zs >> 5;
    uint32_t mw0[kWords];
#pragma unroll
    for (int t = 0; t < kWords; ++t) {
        const int wd = w0 + lane + 32 * t;
        mw0[t] = (c < np && wd < v.ldb) ? (__ldg(bi + wd) & __ldg(bj + wd)) : 0u;
    }
    __syncthreads();
    if (c >= np) return;
    int p = 0;
    for (int q = lane; q < np; q += 32) p += skey[q] > mykey ? 1 : 0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) p += __shfl_xor_sync(0xffffffffu, p, off);
    if (lane == 0) v.piv[p] = make_int4(i, j, wij, 0);
    int* cand = scand[warp];
    const int k2 = K2C > 0 ? K2C : v.k2;
    const uint16_t* wi = v.w + (size_t)i * v.n_pad;
    const uint16_t* wj = v.w + (size_t)j * v.n_pad;

    constexpr int L = K2C > 0 ? K2C : TURBOREG_K2_MAX;
    uint64_t top[L];
#pragma unroll
    for (int r = 0; r < L; ++r) top[r] = 0ull;

    // score list entries [0, cnt): W_iz and W_jz (z > j > i on the O2Graph; the
    // undirected search also meets z < j and reads W symmetrically)
    auto score = [&](int cnt) {
        for (int c0 = 0; c0 < cnt; c0 += 32 * kBatch) {
            int zq[kBatch], wa[kBatch], wb[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int c = c0 + lane + 32 * b;
                zq[b] = c < cnt ? cand[c] : -1;
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int z = zq[b];
                wa[b] = z < 0 ? 0 : static_cast<int>(z > i ? wi[z] : v.w[(size_t)z * v.n_pad + i]);
                wb[b] = z < 0 ? 0 : static_cast<int>(z > j ? wj[z] : v.w[(size_t)z * v.n_pad + j]);
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                if (zq[b] < 0) continue;
                const int sz = wij + wa[b] + wb[b];
                const uint64_t key = (static_cast<uint64_t>(sz) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(zq[b]));
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
        }
    };

    int nlist = 0;
    for (int wb = w0; wb < v.ldb; wb += 32 * kWords) {
        uint32_t mw[kWords];
#pragma unroll
        for (int t = 0; t < kWords; ++t) {
            const int wd = wb + lane + 32 * t;
            mw[t] = wb == w0 ? mw0[t] : wd < v.ldb ? (__ldg(bi + wd) & __ldg(bj + wd)) : 0u;
            if (wd == w0) mw[t] &= ~0u << (zs & 31);
        }
        // one prefix sum per round: lane l writes its candidates (all its words)
        // after those of lanes < l; the list order does not matter
        int cnt = 0;
#pragma unroll
        for (int t = 0; t < kWords; ++t) cnt += __popc(mw[t]);
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (nlist + total <= kCand) {
            int pos = nlist + incl - cnt;
#pragma unroll
            for (int t = 0; t < kWords; ++t) {
                const int zb = (wb + lane + 32 * t) * 32;
                for (uint32_t m = mw[t]; m != 0u; m &= m - 1u) cand[pos++] = zb + __ffs(m) - 1;
            }
            nlist += total;
        } else {
            // dense rows: word by word, scoring the list whenever it would overflow
#pragma unroll 1
            for (int t = 0; t < kWords; ++t) {
                const int c1 = __popc(mw[t]);
                int in1 = c1;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, in1, off);
                    if (lane >= off) in1 += y;
                }
                const int tot1 = __shfl_sync(0xffffffffu, in1, 31);
                if (nlist + tot1 > kCand) {   // warp-uniform
                    __syncwarp();
                    score(nlist);
                    nlist = 0;
                    __syncwarp();
                }
                int pos = nlist + in1 - c1;
                const int zb = (wb + lane + 32 * t) * 32;
                for (uint32_t m = mw[t]; m != 0u; m &= m - 1u) cand[pos++] = zb + __ffs(m) - 1;
                nlist += tot1;
            }
        }
    }
    __syncwarp();
    score(nlist);

    // warp merge: k2 rounds of argmax over the lanes' list heads; lane r keeps
    // round r's clique
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

    // Kabsch of this pivot's cliques (Sec. 3.5): lane r < k2 solves clique r in FP32
    float P[3][3], Q[3][3];
    KabschOut<float> o;
    o.ok = false;
    bool need = false;
    const bool present = lane < k2 && mine_cl.w != 0;
    if (present) {
        load_clique(v, mine_cl, P, Q);
        kabsch3<float>(P, Q, o);
        need = !(o.ok && o.kappa <= v.kappa_fp64);
    }
    const uint32_t needm = __ballot_sync(0xffffffffu, need);
    if (needm != 0u) {
        // FP64 normals, five cliques per round: lane L works for clique
        // base + L / 6, triangle (L / 3) & 1 (x, y), component L % 3
        float nx[3] = {0.f, 0.f, 0.f}, ny[3] = {0.f, 0.f, 0.f};
        for (int base = 0; base < k2 && (needm >> base) != 0u; base += 5) {
            const int r = base + lane / 6;
            const int src = r < 32 ? r : 31;
            const int cz = __shfl_sync(0xffffffffu, mine_cl.z, src);
            const bool act = lane < 30 && r < k2 && ((needm >> src) & 1u);
            float val = 0.f;
            if (act) {
                const int tri = (lane / 3) & 1, comp = lane % 3;
                const int idx[3] = {i, j, cz};
                float T3[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float* pt = v.pts8 + (size_t)idx[a] * 8 + 3 * tri;
                    T3[a][0] = pt[0]; T3[a][1] = pt[1]; T3[a][2] = pt[2];
                }
                val = exact_normal_comp(T3, comp);
            }
            // lane r of this round collects its six components from lanes 6 (r - base) ..
            const int mine0 = 6 * (lane - base);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int from = (lane >= base && lane < base + 5) ? mine0 + k : 0;
                const float g = __shfl_sync(0xffffffffu, val, from);
                if (lane >= base && lane < base + 5) {
                    if (k < 3) nx[k] = g;
                    else ny[k - 3] = g;
                }
            }
        }
        if (need) kabsch3<float, true>(P, Q, o, nx, ny);
    }
    if (lane < k2) store_hypothesis(v, lane * np + p, present, o, need ? 2u : 0u);
}

}  // namespace

cudaError_t pgs_setup()
{
    cudaError_t e = cudaSuccess;
    const void* fns[] = {reinterpret_cast<const void*>(pgs_kernel<0>), reinterpret_cast<const void*>(pgs_kernel<1>),
                         reinterpret_cast<const void*>(pgs_kernel<2>), reinterpret_cast<const void*>(pgs_kernel<3>),
                         reinterpret_cast<const void*>(pgs_kernel<4>), reinterpret_cast<const void*>(pgs_kernel<2, true>)};
    for (const void* f : fns) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kListBytes + TURBOREG_K1_MAX * static_cast<int>(sizeof(uint64_t)));
    }
    return e;
}

// k2 is the common K2 of the batch, or 0 when problems differ (generic list);
// max_k1 sizes the shared copy of the selected keys
void launch_pgs(const Batch& b, int total, int k2, int max_k1, cudaStream_t s)
{
    const ManyViews vs{b};
    const size_t smem = kListBytes + static_cast<size_t>(max_k1) * sizeof(uint64_t);
    switch (k2) {
        case 1: launch_pdl(pgs_kernel<1>, total, 256, smem, s, vs); break;
        case 2:
            if (b.num > 1) launch_pdl(pgs_kernel<2, true>, total, 256, smem, s, vs);
            else launch_pdl(pgs_kernel<2>, total, 256, smem, s, vs);
            break;
        case 3: launch_pdl(pgs_kernel<3>, total, 256, smem, s, vs); break;
        case 4: launch_pdl(pgs_kernel<4>, total, 256, smem, s, vs); break;
        default: launch_pdl(pgs_kernel<0>, total, 256, smem, s, vs); break;
    }
}

cudaError_t verify_setup();

cudaError_t verify_pgs_setup()
{
    const cudaError_t e = verify_setup();
    return e == cudaSuccess ? pgs_setup() : e;
}

}  // namespace tr
