// Stage 2 on CUDA cores: the SC^2 weights of the O2Graph (Eq. 2, Def. 2)
// from the adjacency bitset by AND + population count,
//
//   W_ij = G_ij * popc(row_i & row_j)   for i < j,
//
// the same integers as the tensor-core GEMM (App. B: the number of triangles
// on edge (i, j)), but with work only on the edges: |E+| N_pad/32 word
// operations instead of the dense N_pad^3 multiply-adds.  Its floor is the
// population count itself (16 per clock per SM): 81.6 M words at N = 5000 and
// 4 % density, about 16 us on 152 SMs.
//
// Work tiles: row blocks of 128 rows i by column chunks of 256 columns j of
// the upper triangle (j > i).  Two forms:
//   lane     (N_pad <= 5120) quarters of the tiles (128 x 64) as units, both
//            row sets in shared memory, one edge per group of 8 lanes (below);
//   general  64-row halves; rows j loaded by the warps from global memory,
//            rows i staged in shared memory when they fit, one edge per warp.
// Both write every W entry of their tiles (zeros included, so W needs no
// clearing), and accumulate row sums, row maxima and the edge-weight
// histogram in shared memory, with the same results as the GEMM's epilogue.
#include "tr_common.cuh"
#include "tr_problem.h"

namespace tr {

namespace {

constexpr int kBT = 128;      // rows of a work tile (row block)
constexpr int kBC = 256;      // columns of a work tile (column chunk)

// Work tiles: row blocks of kBT rows by column chunks of kBC columns that hold
// some j > i; row block bi has the chunks bi/2 .. ncb-1.  prefix(bi) = tiles
// of the row blocks before bi.
__host__ __device__ inline int bitset_tile_prefix(int bi, int ncb)
{
    const int a = bi >> 1, r = bi & 1;
    return bi * ncb - a * (a - 1) - r * a;
}

__device__ __forceinline__ void bitset_tile_of(int t, int n_pad, int& bi, int& bj)
{
    const int ncb = n_pad / kBC, nrb = n_pad / kBT;
    int lo = 0, hi = nrb;   // largest bi with prefix(bi) <= t
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bitset_tile_prefix(mid, ncb) <= t) lo = mid;
        else hi = mid;
    }
    bi = lo;
    bj = (lo >> 1) + (t - bitset_tile_prefix(lo, ncb));
}

// Add this CTA's histogram bins of problem v to its global histogram and clear them.
__device__ __forceinline__ void flush_hist(const ProbView& v, uint32_t* sh, int tid, int nthreads)
{
    for (int b = tid + 1; b <= v.n; b += nthreads) {
        const uint32_t h = sh[b];
        if (h) {
            atomicAdd(v.hist + b, h);
            sh[b] = 0u;
        }
    }
}

// One edge (row ri of the staged block, column j): W = popc(row_i & row_j)
// by the warp (lane l holds words l + 32 q of row j in r[q]), recorded in the
// shared tile, row sums and maxima and the histogram by lane 0.  Returns W.
template <int WPL>
__device__ __forceinline__ int edge_weight(const uint32_t* si, const uint32_t (&r)[WPL], int ldb, int lane)
{
    uint32_t c = 0u;
#pragma unroll
    for (int q = 0; q < WPL; ++q)
        if (lane + 32 * q < ldb) c += __popc(si[lane + 32 * q] & r[q]);
    return static_cast<int>(__reduce_add_sync(0xffffffffu, c));
}

__device__ __forceinline__ void record_edge(uint16_t* tile, int* rsum, int* rmax, uint32_t* shist, uint32_t* ghist,
                                            int ri, int col, int c)
{
    tile[ri * kBC + col] = static_cast<uint16_t>(c);
    if (c) {
        atomicAdd(&rsum[ri], c);
        atomicMax(&rmax[ri], c);
        if (shist) atomicAdd(&shist[c], 1u);
        else atomicAdd(&ghist[c], 1u);
    }
}

// ---------------------------------------------------------------------------
// Lane form (N_pad <= 5120).  Work units are quarters of the tiles: 128 rows
// i by 64 columns j, an equal contiguous run of them per CTA of 16 warps.  A
// unit costs a half about 2 us plus 12 ns per edge (2.6 us more where a row
// block begins), so CTAs end unevenly; a contiguous split weighted by that
// cost gains only ~2 us, because a unit is coarse against the halves'
// alternation, which is less than the split itself costs at the start of
// every CTA.  The CTA's 128 bitset rows i (one bulk copy, about
// once per CTA) are in shared memory.  The CTA works as two halves of 8
// warps that take alternate units, each with its own buffer of 64 rows j (one
// bulk copy per unit) and its own edge list, synchronised by its own named
// barrier, so that one half's preparation of a unit (the copy, zeros over the
// unit's W block, the list) overlaps the other half's edge work; the halves
// meet only where a new row block begins, to exchange the rows i.  A unit's
// edges (i < j, ordered by column, then row) are listed from the adjacency
// words of its columns, the list cut into 32 equal runs, one per group of 8
// lanes of the half.  A group computes popc(row_i & row_j) for one edge at a
// time with 20 words per lane (8 lanes x 5 uint4 = 160 words; lane l of the
// group reads uint4 l + 8k, so the 8 lanes of a shared-memory phase hit
// distinct banks), keeps row j in registers while consecutive edges share
// it, and adds the lanes' counts with three shuffles; lane 0 of the group
// stores the weight into W and adds it to the row and column sums, the row
// maximum and the histogram in shared memory.  kCsa: a lane's 20 words are
// first added bit-sliced through a carry-save adder tree (full adders, 28
// logic operations), leaving six words of weights 1, 2, 4 and 8 for the
// population count.
// ---------------------------------------------------------------------------
constexpr int kLUC = 64;                    // columns of a unit
constexpr int kLWarps = 16;
constexpr int kLThreads = 32 * kLWarps;
constexpr int kLGroups = kLThreads / 8;     // groups of 8 lanes, one edge at a time each
constexpr int kLMaxLdb = 160;
constexpr int kLList = kBT * kLUC;          // list capacity of a unit (every pair an edge)

__host__ __device__ inline size_t lane_smem_bytes(int ldb_max, int hist_bins)
{
    return static_cast<size_t>(kBT) * ldb_max * 4 + static_cast<size_t>(2 * kLUC) * ldb_max * 4 +
           static_cast<size_t>(2 * kLList) * 2 + (2 * kBT + 2 * kLUC) * 4 + 32 + 128 + 256 +
           static_cast<size_t>(hist_bins) * 4;
}

struct LaneUnit {
    int p, i0, j0;
};

__device__ __forceinline__ LaneUnit lane_unit(const Batch& bt, int u)
{
    int lt;
    const int p = locate(bt, ST_BITSET, u >> 2, lt);
    int bi, bj;
    bitset_tile_of(lt, bt.views[p].n_pad, bi, bj);
    return {p, bi * kBT, bj * kBC + (u & 3) * kLUC};
}

// The fields of a problem the lane form reads, kept in shared memory (a ring
// of four slots by problem index: the units k-1 .. k+2 a CTA has in hand
// belong to at most four consecutive problems), so that no descriptor read
// from global memory sits on a unit's critical path.
struct LaneView {
    uint32_t* bits;
    uint16_t* w;
    int32_t* rowscore;
    int32_t* rowmax;
    uint32_t* hist;
    int32_t n, n_pad, ldb, pad;
};
static_assert(sizeof(LaneView) <= 64, "four views in 256 bytes of shared memory");

__device__ __forceinline__ void lane_view_load(LaneView& d, const ProbView& v)
{
    d.bits = v.bits;
    d.w = v.w;
    d.rowscore = v.rowscore;
    d.rowmax = v.rowmax;
    d.hist = v.hist;
    d.n = v.n;
    d.n_pad = v.n_pad;
    d.ldb = v.ldb;
}

// Adds a CTA's histogram bins of a problem to its global histogram and clears them.
__device__ __forceinline__ void lane_flush_hist(const LaneView& v, uint32_t* sh, int tid)
{
    for (int b = tid + 1; b <= v.n; b += blockDim.x) {
        const uint32_t h = sh[b];
        if (h) {
            atomicAdd(v.hist + b, h);
            sh[b] = 0u;
        }
    }
}

// The unit after `un` in unit order (row blocks in turn, each from its first
// tile to the last column; then the next problem's first unit); n_pad: un's problem.
__device__ __forceinline__ LaneUnit lane_next(LaneUnit un, int n_pad)
{
    un.j0 += kLUC;
    if (un.j0 < n_pad) return un;
    un.i0 += kBT;
    if (un.i0 < n_pad) {
        un.j0 = (un.i0 / kBT >> 1) * kBC;
        return un;
    }
    return {un.p + 1, 0, 0};
}

// full adder on every bit position: a + b + d = s + 2 c, one three-input
// logic operation each (truth tables 0x96: a ^ b ^ d, 0xE8: majority)
__device__ __forceinline__ void full_add(uint32_t& c, uint32_t& s, uint32_t a, uint32_t b, uint32_t d)
{
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(s) : "r"(a), "r"(b), "r"(d));
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(c) : "r"(a), "r"(b), "r"(d));
}

// sum over this lane's words of popc(row_i word & row_j word)
template <int NQ, bool kCsa>
__device__ __forceinline__ uint32_t and_popc(const uint4 (&a)[NQ], const uint4 (&b)[NQ])
{
    uint32_t w[4 * NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        w[4 * k + 0] = a[k].x & b[k].x;
        w[4 * k + 1] = a[k].y & b[k].y;
        w[4 * k + 2] = a[k].z & b[k].z;
        w[4 * k + 3] = a[k].w & b[k].w;
    }
    if constexpr (!kCsa || NQ != 5) {
        uint32_t s = 0u;
#pragma unroll
        for (int k = 0; k < 4 * NQ; ++k) s += __popc(w[k]);
        return s;
    } else {
        // 20 words of weight 1 -> o8, w19 (1), u3 (2), g0, f3 (4), e0 (8)
        uint32_t t0, o0, t1, o1, t2, o2, t3, o3, t4, o4, t5, o5;
        full_add(t0, o0, w[0], w[1], w[2]);
        full_add(t1, o1, w[3], w[4], w[5]);
        full_add(t2, o2, w[6], w[7], w[8]);
        full_add(t3, o3, w[9], w[10], w[11]);
        full_add(t4, o4, w[12], w[13], w[14]);
        full_add(t5, o5, w[15], w[16], w[17]);
        uint32_t t6, o6, t7, o7, t8, o8;
        full_add(t6, o6, o0, o1, o2);
        full_add(t7, o7, o3, o4, o5);
        full_add(t8, o8, o6, o7, w[18]);
        uint32_t f0, u0, f1, u1, f2, u2, f3, u3, e0, g0;
        full_add(f0, u0, t0, t1, t2);
        full_add(f1, u1, t3, t4, t5);
        full_add(f2, u2, t6, t7, t8);
        full_add(f3, u3, u0, u1, u2);
        full_add(e0, g0, f0, f1, f2);
        return __popc(o8) + __popc(w[19]) + 2u * __popc(u3) + 4u * (__popc(g0) + __popc(f3)) + 8u * __popc(e0);
    }
}

// The SC^2 path for one problem, chosen on the device after the compatibility
// graph: predicted times (us) fitted to measurements on GB300 at N = 1000 ..
// 5000 and 1.7 .. 14 % density.  This CUDA-core form: a + b |E+| / 1e6, with
// (a, b) = (21.5, 49) at n_pad = 5120 and (13.9, 70.8) at 3072, linear in
// between (fewer units per CTA for smaller N), and always the faster one up
// to n_pad = 2048; the tensor-core GEMM: 12.5 + waves x K-stages x 0.368 (its
// 2-CTA clusters over the 256 x 256 upper-triangle tiles, 0.368 us per
// 128-deep stage) plus 4 (n_pad / 5120)^2 for the FP8 matrix it then needs.
__device__ __forceinline__ bool sc2_bitset_faster(int n_pad, unsigned long long deg_sum, int clusters)
{
    if (n_pad <= 2048) return true;
    const float d = static_cast<float>(5120 - n_pad) / 2048.f;
    const float edges_m = static_cast<float>(deg_sum) * 0.5e-6f;
    const float t_bitset = (21.5f - 7.6f * d) + (49.f + 21.8f * d) * edges_m;
    const int nb = n_pad / 256;
    const int tiles = nb * (nb + 1) / 2;
    const int waves = (tiles + clusters - 1) / clusters;
    const float r = static_cast<float>(n_pad) / 5120.f;
    const float t_gemm = 12.5f + static_cast<float>(waves * (n_pad / 128)) * 0.368f + 4.f * r * r;
    return t_bitset <= t_gemm;
}

// 4 adjacency bits -> 4 bytes of FP8 E4M3 (0x38 = 1.0 for a set bit, 0 otherwise)
__device__ __forceinline__ uint32_t nib_fp8(uint32_t nib) { return ((nib * 0x00204081u) & 0x01010101u) * 0x38u; }

__device__ __forceinline__ uint4 half_word_fp8(uint32_t b16)
{
    return make_uint4(nib_fp8(b16 & 0xFu), nib_fp8((b16 >> 4) & 0xFu), nib_fp8((b16 >> 8) & 0xFu),
                      nib_fp8((b16 >> 12) & 0xFu));
}

// auto_clusters > 0: one problem whose SC^2 path is chosen here (the GEMM's
// co-resident 2-CTA clusters); if the GEMM is the faster path, the CTAs expand
// the bitset into its FP8 operand and leave the rest to it.
template <int NQ, bool kExact, bool kCsa>
__global__ void __launch_bounds__(kLThreads, 1)
    sc2_bitset_lane_kernel(Batch bt, int total, int ldb_max, int hist_bins, int auto_clusters)
{
    extern __shared__ __align__(16) uint8_t ls_raw[];
    uint8_t* q8 = ls_raw;
    uint32_t* srows = reinterpret_cast<uint32_t*>(q8);  q8 += static_cast<size_t>(kBT) * ldb_max * 4;
    uint32_t* scols = reinterpret_cast<uint32_t*>(q8);  q8 += static_cast<size_t>(2 * kLUC) * ldb_max * 4;
    uint16_t* slist = reinterpret_cast<uint16_t*>(q8);  q8 += static_cast<size_t>(2 * kLList) * 2;
    int* srsum = reinterpret_cast<int*>(q8);            q8 += kBT * 4;
    int* srmax = reinterpret_cast<int*>(q8);            q8 += kBT * 4;
    int* scsum = reinterpret_cast<int*>(q8);            q8 += 2 * kLUC * 4;   // [half][column]
    uint64_t* bars = reinterpret_cast<uint64_t*>(q8);   q8 += 32;            // rows i, rows j [half]
    int* sw = reinterpret_cast<int*>(q8);               q8 += 128;           // list scans: [half][warp of half]
    LaneView* lv = reinterpret_cast<LaneView*>(q8);     q8 += 256;           // [problem & 3]
    uint32_t* shist = reinterpret_cast<uint32_t*>(q8);
    uint64_t* rows_full = bars;
    uint64_t* cols_full = bars + 1;
    const int tid = threadIdx.x, lane = tid & 31;
    const int half = tid >> 8, ht = tid & 255, hwarp = ht >> 5;   // two halves of 8 warps
    const int grp = ht >> 3, gl = tid & 7;                          // groups of 8 lanes within the half
    if (tid < 3) mbar_init(&bars[tid], 1);
    if (tid == 0) fence_mbar_init();
    for (int b = tid; b < hist_bins; b += kLThreads) shist[b] = 0u;
    if (tid < kBT) {
        srsum[tid] = 0;
        srmax[tid] = 0;
    }
    if (tid < 2 * kLUC) scsum[tid] = 0;
    // this CTA's units: an equal contiguous run
    const int units = 4 * total;
    const int u0 = static_cast<int>((static_cast<long long>(units) * blockIdx.x) / gridDim.x);
    const int u1 = static_cast<int>((static_cast<long long>(units) * (blockIdx.x + 1)) / gridDim.x);
    const int K = u1 - u0;
    bool ok = true;

    auto half_sync = [&]() { asm volatile("bar.sync %0, 256;" ::"r"(1 + half) : "memory"); };
    auto issue_cols = [&](const LaneUnit& un, int slot) {
        const LaneView& v = lv[un.p & 3];
        const uint32_t bytes = static_cast<uint32_t>(kLUC * v.ldb * 4);
        mbar_arrive_expect_tx(&cols_full[slot], bytes);
        bulk_g2s(scols + static_cast<size_t>(slot) * kLUC * ldb_max, v.bits + static_cast<size_t>(un.j0) * v.ldb,
                 bytes, &cols_full[slot]);
    };
    auto issue_rows = [&](const LaneUnit& un) {
        const LaneView& v = lv[un.p & 3];
        const uint32_t bytes = static_cast<uint32_t>(kBT * v.ldb * 4);
        mbar_arrive_expect_tx(rows_full, bytes);
        bulk_g2s(srows, v.bits + static_cast<size_t>(un.i0) * v.ldb, bytes, rows_full);
    };
    auto flush_rows = [&](const LaneUnit& un, bool hist) {   // a finished row block (and problem)
        const LaneView& pv = lv[un.p & 3];
        if (tid < kBT) {
            const int x = srsum[tid], mx = srmax[tid];
            if (x) atomicAdd(&pv.rowscore[un.i0 + tid], x);
            if (mx && pv.rowmax) atomicMax(&pv.rowmax[un.i0 + tid], mx);
            srsum[tid] = 0;
            srmax[tid] = 0;
        }
        if (hist && hist_bins > 0) lane_flush_hist(pv, shist, tid);
    };
    // The first unit and its problem's fields come from the launch's
    // descriptors only, so they are read before the dependency wait; the
    // first row block and each half's first unit are then copied at once
    // after it (the degree-sum read of the path choice overlaps the copies).
    LaneUnit cur = {0, 0, 0};
    if (K > 0) {
        cur = lane_unit(bt, u0);
        if (tid == 0) lane_view_load(lv[cur.p & 3], bt.views[cur.p]);
    }
    __syncthreads();   // barriers initialised, the first problem's fields in place
    LaneUnit prev = cur;
    // this half's first unit (unit `half` of the run) when it is copied early
    const LaneUnit first1 = K > 1 ? lane_next(cur, lv[cur.p & 3].n_pad) : cur;
    const bool early_cols = K > half && (half == 0 || first1.p == cur.p);
    pdl_wait();
    pdl_release();
    if (K > 0) {
        if (tid == 0) issue_rows(cur);
        if (ht == 0 && early_cols) issue_cols(half == 0 ? cur : first1, half);
    }
    if (auto_clusters > 0) {
        // the degree sum 2 |E| of the problem (added up by the compatibility blocks)
        const ProbView& v0 = bt.views[0];
        const unsigned long long deg_sum = __ldcg(&v0.ctl->deg_sum);
        const bool bitset = sc2_bitset_faster(v0.n_pad, deg_sum, auto_clusters);
        if (blockIdx.x == 0 && tid == 0) v0.ctl->sc2_path = bitset ? 1u : 2u;
        if (!bitset) {
            // no copy may still be landing in shared memory when the CTA leaves
            if (K > 0) {
                bool landed = mbar_wait(rows_full, 0u);
                if (early_cols) landed &= mbar_wait(&cols_full[half], 0u);
                if (!landed) atomicOr(&v0.ctl->err, TR_ERR_TIMEOUT);
            }
            // the GEMM's FP8 operand from the bitset: word q of the matrix -> 32 bytes
            const size_t words = static_cast<size_t>(v0.n_pad) * v0.ldb;
            for (size_t q = static_cast<size_t>(blockIdx.x) * kLThreads + tid; q < words;
                 q += static_cast<size_t>(gridDim.x) * kLThreads) {
                const uint32_t w = __ldcg(v0.bits + q);
                const size_t row = q / static_cast<size_t>(v0.ldb), col = (q % static_cast<size_t>(v0.ldb)) * 32;
                uint4* dst = reinterpret_cast<uint4*>(v0.a8_auto + row * v0.n_pad + col);
                dst[0] = half_word_fp8(w & 0xFFFFu);
                dst[1] = half_word_fp8(w >> 16);
            }
            return;
        }
    }
    if (K <= 0) return;
    uint32_t rows_uses = 0, cols_uses = 0;   // this half's uses of its rows-j buffer
    uint32_t pref = 0u;                       // this thread's adjacency word of the half's next unit,
    bool have_pref = false;                   // loaded during the current unit's edge loop
    // Every thread walks all units in order; half h takes the units k with
    // k % 2 == h.  The halves meet only where a new row block begins (both
    // have finished every earlier unit there), to exchange the rows i.
    for (int k = 0; k < K; ++k) {
        if (k > 0) cur = lane_next(prev, lv[prev.p & 3].n_pad);
        const bool new_rows = k > 0 && (cur.p != prev.p || cur.i0 != prev.i0);
        if (new_rows) {
            __syncthreads();   // both halves are past every unit of the old row block
            flush_rows(prev, cur.p != prev.p);
            if (tid == 0) {
                if (cur.p != prev.p) lane_view_load(lv[cur.p & 3], bt.views[cur.p]);
                fence_proxy_async();
                issue_rows(cur);
            }
            __syncthreads();   // the old block's sums are taken; the new problem's fields are in place
        }
        if (k == 0 || new_rows) {
            ok &= mbar_wait(rows_full, rows_uses & 1u);
            ++rows_uses;
        }
        prev = cur;
        if ((k & 1) != half) continue;
        // ---------------- unit k, by this half ----------------
        const LaneView& v = lv[cur.p & 3];
        const int slot = half;
        if (ht == 0 && !(k == half && early_cols)) {
            fence_proxy_async();   // the buffer's previous rows were read by this half's threads
            issue_cols(cur, slot);
        }
        // zeros over the unit's W block (the weights are stored over them after the next barrier)
        for (int q = ht; q < kBT * kLUC / 8; q += 256)
            *reinterpret_cast<uint4*>(v.w + static_cast<size_t>(cur.i0 + (q >> 3)) * v.n_pad + cur.j0 + (q & 7) * 8) =
                make_uint4(0u, 0u, 0u, 0u);
        // the unit's edges: thread ht takes column j0 + ht / 4, rows 32 (ht % 4) .. +31
        uint32_t m;
        {
            const int jl = ht >> 2, h = ht & 3;
            const int j = cur.j0 + jl;
            const uint32_t w = have_pref ? pref : __ldg(v.bits + static_cast<size_t>(j) * v.ldb + (cur.i0 >> 5) + h);
            const int lh = (j < v.n ? j - cur.i0 : 0) - 32 * h;   // rows 32 h + r, r < lh
            m = lh <= 0 ? 0u : lh < 32 ? w & ((1u << lh) - 1u) : w;
        }
        int inc = __popc(m);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        if (lane == 31) sw[half * 8 + hwarp] = inc;
        half_sync();
        int E = 0, base = inc - __popc(m);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const int x = sw[half * 8 + w];
            if (w < hwarp) base += x;
            E += x;
        }
        uint16_t* lst = slist + slot * kLList;
        {
            const int jl = ht >> 2, h = ht & 3;
            for (; m; m &= m - 1u) lst[base++] = static_cast<uint16_t>((jl << 7) | (32 * h + __ffs(m) - 1));
        }
        half_sync();   // the list and the zeros are complete
        {   // the half's next unit (two ahead): its adjacency word, in flight during the edge loop
            const LaneUnit n1 = lane_next(cur, v.n_pad);
            const LaneUnit n2 = n1.p == cur.p ? lane_next(n1, v.n_pad) : n1;
            have_pref = k + 2 < K && n2.p == cur.p;
            if (have_pref)
                pref = __ldg(v.bits + static_cast<size_t>(n2.j0 + (ht >> 2)) * v.ldb + (n2.i0 >> 5) + (ht & 3));
        }
        ok &= mbar_wait(&cols_full[slot], cols_uses & 1u);
        ++cols_uses;
        {
            const int ldb = v.ldb;
            const int l4 = ldb >> 2;
            const int lo = (grp * E) / (kLGroups / 2), hi = ((grp + 1) * E) / (kLGroups / 2);
            const int cnt = hi - lo;
            const int T = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(cnt)));
            const uint32_t* cols = scols + static_cast<size_t>(slot) * kLUC * ldb_max;
            int* csum = scsum + half * kLUC;
            uint32_t* hh = hist_bins > 0 ? shist : v.hist;
            uint16_t* wblk = v.w + static_cast<size_t>(cur.i0) * v.n_pad + cur.j0;
            const int e_last = cnt > 0 ? hi - 1 : 0;
            int cj = -1;
            uint4 jr[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) jr[q] = make_uint4(0u, 0u, 0u, 0u);
            int ent = T > 0 ? lst[cnt > 0 ? lo : 0] : 0;
            for (int t = 0; t < T; ++t) {
                const bool valid = t < cnt;
                const int il = ent & 127, jl = ent >> 7;
                ent = lst[t + 1 < cnt ? lo + t + 1 : e_last];   // the next entry, ahead of its use
                if (jl != cj) {
                    cj = jl;
                    const uint4* r4 = reinterpret_cast<const uint4*>(cols + static_cast<size_t>(jl) * ldb);
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        jr[q] = (kExact || gl + 8 * q < l4) ? r4[gl + 8 * q] : make_uint4(0u, 0u, 0u, 0u);
                }
                const uint4* a4 = reinterpret_cast<const uint4*>(srows + static_cast<size_t>(il) * ldb);
                uint4 a[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    a[q] = (kExact || gl + 8 * q < l4) ? a4[gl + 8 * q] : make_uint4(0u, 0u, 0u, 0u);
                uint32_t s = and_popc<NQ, kCsa>(a, jr);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                if (gl == 0 && valid && s) {
                    wblk[static_cast<size_t>(il) * v.n_pad + jl] = static_cast<uint16_t>(s);
                    atomicAdd(&srsum[il], static_cast<int>(s));
                    atomicMax(&srmax[il], static_cast<int>(s));
                    atomicAdd(&csum[jl], static_cast<int>(s));
                    atomicAdd(&hh[s], 1u);
                }
            }
        }
        half_sync();   // the unit's items are done: its buffers are free, its column sums complete
        if (ht < kLUC) {
            int* cs = scsum + half * kLUC;
            const int x = cs[ht];
            if (x) atomicAdd(&v.rowscore[cur.j0 + ht], x);
            cs[ht] = 0;
        }
    }
    __syncthreads();
    flush_rows(prev, true);   // the last row block and problem
    if (!ok && lane == 0) atomicOr(&bt.views[0].ctl->err, TR_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// General form (any N): persistent CTAs of 8 warps take the same tiles as two
// halves of 64 rows; a warp loads row j straight from global memory (the next
// one in flight while it works on the current).  The 64 rows i are staged in
// shared memory when they fit, else read from global memory (largest N).
// ---------------------------------------------------------------------------
constexpr int kBR = 64;
constexpr int kBsThreads = 256;
constexpr int kBsWarps = kBsThreads / 32;

// rows_ldb: words per staged row (0: rows i from global memory); hist_bins: 0
// when the bins do not fit and are added to the global histogram directly
template <int WPL>
__global__ void __launch_bounds__(kBsThreads, 2) sc2_bitset_kernel(Batch bt, int total, int rows_ldb, int hist_bins)
{
    extern __shared__ __align__(16) uint8_t bs_raw[];
    uint16_t* stile = reinterpret_cast<uint16_t*>(bs_raw);
    uint32_t* srows = reinterpret_cast<uint32_t*>(bs_raw + kBR * kBC * 2);
    int* srsum = reinterpret_cast<int*>(srows + kBR * rows_ldb);
    int* srmax = srsum + kBR;
    uint32_t* shist = reinterpret_cast<uint32_t*>(srmax + kBR);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < hist_bins; b += kBsThreads) shist[b] = 0u;
    const int t0 = static_cast<int>((static_cast<long long>(total) * blockIdx.x) / gridDim.x);
    const int t1 = static_cast<int>((static_cast<long long>(total) * (blockIdx.x + 1)) / gridDim.x);
    pdl_wait();
    pdl_release();
    int cur_p = -1;
    for (int t = t0; t < t1; ++t) {
        int lt;
        const int p = locate(bt, ST_BITSET, t, lt);
        const ProbView v = bt.views[p];
        int bi, bj;
        bitset_tile_of(lt, v.n_pad, bi, bj);
        const int n = v.n, ldb = v.ldb;
        if (p != cur_p && cur_p >= 0 && hist_bins > 0) {
            __syncthreads();
            flush_hist(bt.views[cur_p], shist, threadIdx.x, kBsThreads);
        }
        cur_p = p;
        for (int half = 0; half < 2; ++half) {
            const int i0 = bi * kBT + half * kBR, j0 = bj * kBC;
            __syncthreads();   // the previous half's shared data is consumed
            if (rows_ldb > 0) {
                const uint4* src = reinterpret_cast<const uint4*>(v.bits + (size_t)i0 * ldb);
                for (int q = threadIdx.x; q < kBR * ldb / 4; q += kBsThreads) reinterpret_cast<uint4*>(srows)[q] = src[q];
            }
            for (int q = threadIdx.x; q < kBR * kBC / 8; q += kBsThreads)
                reinterpret_cast<uint4*>(stile)[q] = make_uint4(0, 0, 0, 0);
            if (threadIdx.x < kBR) {
                srsum[threadIdx.x] = 0;
                srmax[threadIdx.x] = 0;
            }
            __syncthreads();
            const int wi = i0 >> 5;
            const int jlo = j0 > i0 + 1 ? j0 : i0 + 1;
            const int jhi = j0 + kBC < n ? j0 + kBC : n;
            int j = jlo + warp;
            uint32_t r[WPL];
#pragma unroll
            for (int q = 0; q < WPL; ++q)
                r[q] = (j < jhi && lane + 32 * q < ldb) ? __ldg(v.bits + (size_t)j * ldb + lane + 32 * q) : 0u;
            for (; j < jhi; j += kBsWarps) {
                uint32_t rn[WPL];
                const int jn = j + kBsWarps;
#pragma unroll
                for (int q = 0; q < WPL; ++q)
                    rn[q] = (jn < jhi && lane + 32 * q < ldb) ? __ldg(v.bits + (size_t)jn * ldb + lane + 32 * q) : 0u;
                // adjacency of j to rows i0 .. i0+63 (words wi, wi+1 of row j, an L1 hit;
                // selecting them from the lanes' registers would index the array)
                const uint2 wm = __ldg(reinterpret_cast<const uint2*>(v.bits + (size_t)j * ldb + wi));
                uint64_t mask = static_cast<uint64_t>(wm.x) | (static_cast<uint64_t>(wm.y) << 32);
                const int lim = j - i0;
                if (lim < 64) mask &= (1ull << lim) - 1ull;
                int colsum = 0;
                while (mask) {
                    const int ri = __ffsll(static_cast<long long>(mask)) - 1;
                    mask &= mask - 1ull;
                    const uint32_t* si = rows_ldb > 0 ? srows + ri * ldb : v.bits + (size_t)(i0 + ri) * ldb;
                    const int c = edge_weight<WPL>(si, r, ldb, lane);
                    colsum += c;
                    if (lane == 0)
                        record_edge(stile, srsum, srmax, hist_bins > 0 ? shist : nullptr, v.hist, ri, j - j0, c);
                }
                if (lane == 0 && colsum) atomicAdd(&v.rowscore[j], colsum);
#pragma unroll
                for (int q = 0; q < WPL; ++q) r[q] = rn[q];
            }
            __syncthreads();
            for (int q = threadIdx.x; q < kBR * kBC / 8; q += kBsThreads) {
                const int rr = q >> 5, c8 = (q & 31) * 8;
                *reinterpret_cast<uint4*>(v.w + (size_t)(i0 + rr) * v.n_pad + j0 + c8) =
                    reinterpret_cast<const uint4*>(stile)[q];
            }
            if (threadIdx.x < kBR) {
                const int s = srsum[threadIdx.x], m = srmax[threadIdx.x];
                if (s) atomicAdd(&v.rowscore[i0 + threadIdx.x], s);
                if (m && v.rowmax) atomicMax(&v.rowmax[i0 + threadIdx.x], m);
            }
        }
    }
    if (cur_p >= 0 && hist_bins > 0) {
        __syncthreads();
        flush_hist(bt.views[cur_p], shist, threadIdx.x, kBsThreads);
    }
}

int g_bs_sms = 0;

size_t bitset_smem(int rows_ldb, int hist_bins)
{
    return static_cast<size_t>(kBR) * kBC * 2 + static_cast<size_t>(kBR) * rows_ldb * 4 + 2 * kBR * 4 +
           static_cast<size_t>(hist_bins) * 4;
}

constexpr int kBsSmemMax = 232448;

template <int WPL>
cudaError_t bs_attr()
{
    return cudaFuncSetAttribute(sc2_bitset_kernel<WPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBsSmemMax);
}

template <int NQ, bool kExact, bool kCsa>
cudaError_t lane_attr()
{
    return cudaFuncSetAttribute(sc2_bitset_lane_kernel<NQ, kExact, kCsa>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBsSmemMax);
}



}  // namespace

int bitset_tiles(int n_pad) { return bitset_tile_prefix(n_pad / kBT, n_pad / kBC); }

cudaError_t sc2_bitset_setup()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_bs_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = bs_attr<8>();
    if (e == cudaSuccess) e = bs_attr<16>();
    if (e == cudaSuccess) e = bs_attr<32>();
    if (e == cudaSuccess) e = lane_attr<2, false, false>();
    if (e == cudaSuccess) e = lane_attr<5, false, true>();
    if (e == cudaSuccess) e = lane_attr<5, true, true>();
    return e;
}

bool launch_sc2_bitset(const Batch& b, int total_tiles, int max_n, int min_n, int auto_clusters, cudaStream_t s)
{
    const int max_npad = (max_n + kSc2BN - 1) / kSc2BN * kSc2BN;
    const int max_ldb = max_npad / 32;
    const int sms = g_bs_sms > 0 ? g_bs_sms : 148;
    if (max_ldb <= kLMaxLdb) {
        int hist_bins = max_n + 1;
        if (lane_smem_bytes(max_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
        const size_t smem = lane_smem_bytes(max_ldb, hist_bins);
        const int grid = sms < 4 * total_tiles ? sms : 4 * total_tiles;
        // kExact (no per-lane word guard) when every problem's rows are 5 x 32 words
        const int min_ldb = (min_n + kSc2BN - 1) / kSc2BN * kSc2BN / 32;
        const bool exact = min_ldb == max_ldb && max_ldb == kLMaxLdb;
        if (max_ldb <= 64)
            launch_pdl(sc2_bitset_lane_kernel<2, false, false>, grid, kLThreads, smem, s, b, total_tiles, max_ldb, hist_bins, auto_clusters);
        else if (exact)
            launch_pdl(sc2_bitset_lane_kernel<5, true, true>, grid, kLThreads, smem, s, b, total_tiles, max_ldb, hist_bins, auto_clusters);
        else
            launch_pdl(sc2_bitset_lane_kernel<5, false, true>, grid, kLThreads, smem, s, b, total_tiles, max_ldb, hist_bins, auto_clusters);
        return true;
    }
    // shared memory for the row block and the histogram bins, as far as they fit
    int rows_ldb = max_ldb, hist_bins = max_n + 1;
    if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
    if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) {
        rows_ldb = 0;
        hist_bins = max_n + 1;
        if (bitset_smem(rows_ldb, hist_bins) > static_cast<size_t>(kBsSmemMax)) hist_bins = 0;
    }
    const size_t smem = bitset_smem(rows_ldb, hist_bins);
    const int per_sm = smem <= static_cast<size_t>(kBsSmemMax / 2 - 1024) ? 2 : 1;
    int grid = sms * per_sm;
    if (grid > total_tiles) grid = total_tiles;
    const int wpl = (max_ldb + 31) / 32;
    if (wpl <= 8) launch_pdl(sc2_bitset_kernel<8>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    else if (wpl <= 16) launch_pdl(sc2_bitset_kernel<16>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    else launch_pdl(sc2_bitset_kernel<32>, grid, kBsThreads, smem, s, b, total_tiles, rows_ldb, hist_bins);
    return true;
}

}  // namespace tr
