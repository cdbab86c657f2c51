// Host runtime and C ABI of the GB300 TurboReg library (see include/turboreg.h).
//
// A context owns a device workspace sized at creation: max_batch problem
// slots, each sized for max_n.  A register call builds a plan (per-problem
// views, per-stage block prefixes, tensor maps), enqueues one launch per
// stage for all of its problems on the context's stream, copies the 92-byte
// results back and synchronises.  The enqueued pipeline is captured once per
// plan shape as a CUDA graph and replayed; the pack node's input pointers are
// patched per call.  No host round trip happens between stages: pivot
// counts, thresholds and validity stay on the device (Ctl block).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tr_common.cuh"
#include "tr_mlp.h"
#include "tr_problem.h"
#include "turboreg.h"
#include "turboreg_internal.h"

using namespace tr;

namespace {

constexpr int kNumStages = 8;
// "proposal": the threshold's select launch when the SC^2 stage did not fuse
// it, and the learned proposal's features, network, histogram and select
const char* kStageNames[kNumStages] = {"pack", "compat", "sc2", "proposal", "topk", "pgs", "verify", "finalize"};
constexpr int kGraphSlots = 8;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline int32_t round_up(int32_t a, int32_t b) { return (a + b - 1) / b * b; }

// Per-slot workspace: slot s of every buffer starts at s * (per-slot size).
struct Workspace {
    int32_t slots = 0;
    int32_t np = 0;          // n_pad of max_n
    size_t nh = 0;           // K1_MAX * K2_MAX
    float* pts = nullptr;            // [slots][6 np]
    float* pts8 = nullptr;           // [slots][8 np]
    uint8_t* a8 = nullptr;           // [slots][np^2]
    uint32_t* bits = nullptr;        // [slots][np^2 / 32]
    uint16_t* w = nullptr;           // [slots][np^2]
    int32_t* rows = nullptr;         // [slots][7][np]: rowscore, deg, active (int4 per row), rowmax
    uint32_t* hist = nullptr;        // [slots][np + 1]
    uint64_t* cand = nullptr;        // [slots][K1_MAX]
    int4* piv = nullptr;             // [slots][K1_MAX]
    int4* cliques = nullptr;         // [slots][nh]
    float* rt = nullptr;             // [slots][nh * 16]
    int32_t* inl = nullptr;          // [slots][nh]
    uint32_t* hbits = nullptr;       // [slots][2][nh / 32]
    unsigned long long* score = nullptr;  // [slots][nh]
    float* feat = nullptr;           // [slots][np][8] proposal features
    float* prob = nullptr;           // [slots][np] proposal probabilities
    Ctl* ctl = nullptr;              // [slots]
    turboreg_result* res = nullptr;  // [slots]
    float* in_src = nullptr;         // staging for host inputs [max_n * slots * 3]
    float* in_dst = nullptr;
    // descriptors for direct (non-graph) launches, and pinned host mirrors
    uint8_t* desc = nullptr;
    ProbView* h_views = nullptr;
    int32_t* h_pre = nullptr;
    CUtensorMap* h_maps = nullptr;
    int32_t* map_npad = nullptr;     // host: n_pad each slot's maps were encoded for
    CUtensorMap* map_cache = nullptr;  // host: encoded maps per slot
};

// A plan: the problems of one call (in slots 0..num-1) and per-stage block totals.
struct Plan {
    int32_t num = 0;
    int32_t max_n = 0, min_n = 0, max_k1 = 0, k2_common = 0;
    int32_t bitset = 0, timed = 0, learned = 0;
    int32_t sc2_auto = 0;    // one problem: the SC^2 path is chosen on the device (CUDA-core or GEMM)
    int32_t pair_mma = 1;    // SC^2 GEMM: 1 pair MMAs on 2-CTA clusters, 0 independent CTAs
    int32_t vpw = 64;        // verification tile: points per warp
    int32_t vcap = 0;        // balanced tile: verification launched with at most four blocks per SM
    int32_t tot[kNumBatchStages] = {};
};

size_t desc_bytes(int32_t num)
{
    const size_t v = sizeof(ProbView) * num;
    const size_t p = sizeof(int32_t) * kNumBatchStages * (num + 1);
    return (v + 127) / 128 * 128 + (p + 127) / 128 * 128 + sizeof(CUtensorMap) * 2 * num;
}

}  // namespace

struct turboreg_ctx {
    int device = 0;
    int32_t max_n = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Workspace ws;
    turboreg_result* host_res = nullptr;   // pinned [max_batch]
    float* mlp_wbf = nullptr;              // proposal model (BF16-rounded FP32 values), device
    bool has_model = false;
    // the control blocks may hold nonzero counters or error bits (before the
    // first registration, after an entry point that runs part of the path)
    bool ctl_dirty = true;
    EncodeTiledFn encode = nullptr;
    cudaEvent_t ev[kNumStages + 1] = {};
    // the descriptor uploads read the page-locked staging (ws.h_views, h_pre,
    // h_maps) when the stream reaches them; it is rewritten only after this
    // event (recorded behind each upload) has completed
    cudaEvent_t desc_done = nullptr;
    bool desc_pending = false;
    float stage_ms[kNumStages] = {};
    int32_t last_n = 0, last_npad = 0, last_k1 = 0, last_k2 = 0;
    bool last_fp8 = false;   // the last plan materialised the FP8 adjacency (tensor-core SC^2)
    bool last_auto = false;  // ... or left the choice to the device (the FP8 matrix exists if the GEMM ran)
    bool have_times = false;
    // Captured pipelines.  Each slot owns a private copy of its descriptors in
    // device memory, so replays of different shapes never see each other's.
    struct GraphSlot {
        bool used = false;
        std::vector<uint8_t> key;          // plan signature
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t pack_node = nullptr;
        cudaKernelNodeParams pack_params = {};
        tr::Batch batch = {};
        const float* src = nullptr;
        const float* dst = nullptr;
        void* args[3] = {};
        cudaGraphNode_t fin_node = nullptr;   // finalize: its result pointer is patched per call
        cudaKernelNodeParams fin_params = {};
        turboreg_result* out = nullptr;
        void* fin_args[2] = {};
        void* desc = nullptr;
        uint64_t stamp = 0;
    };
    GraphSlot gslot[kGraphSlots];
    uint64_t gclock = 0;
};

namespace {

#define TR_CHECK(expr)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            std::fprintf(stderr, "turboreg: %s failed: %s\n", #expr, cudaGetErrorString(e_));  \
            return TURBOREG_ERR_CUDA;                                                          \
        }                                                                                      \
    } while (0)

// Failure injection for tests: with TURBOREG_DEBUG_FAIL_ALLOC=k in the
// environment, the k-th allocation (1-based, counted per turboreg_create call
// and thread) fails as if the device or host memory were exhausted.
thread_local int t_alloc_seq = 0;
thread_local int t_alloc_fail = 0;

bool injected_alloc_failure() { return ++t_alloc_seq == t_alloc_fail; }

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 256);
}

template <typename T>
cudaError_t halloc(T** p, size_t count)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(reinterpret_cast<void**>(p), count * sizeof(T) + 64);
}

void free_ws(Workspace& ws)
{
    void* dptrs[] = {ws.pts, ws.pts8, ws.a8, ws.bits, ws.w, ws.rows, ws.hist, ws.cand, ws.piv, ws.cliques,
                     ws.rt, ws.inl, ws.hbits, ws.score, ws.feat, ws.prob, ws.ctl, ws.res, ws.in_src, ws.in_dst,
                     ws.desc};
    for (void* p : dptrs)
        if (p) cudaFree(p);
    void* hptrs[] = {ws.h_views, ws.h_pre, ws.h_maps};
    for (void* p : hptrs)
        if (p) cudaFreeHost(p);
    std::free(ws.map_npad);
    std::free(ws.map_cache);
    ws = Workspace();
}

int alloc_ws(Workspace& ws, int32_t max_n, int32_t slots)
{
    const int32_t np = round_up(max_n, kSc2BN);
    const size_t n2 = static_cast<size_t>(np) * np;
    const size_t nh = static_cast<size_t>(TURBOREG_K1_MAX) * TURBOREG_K2_MAX;
    const size_t S = static_cast<size_t>(slots);
    ws.slots = slots;
    ws.np = np;
    ws.nh = nh;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&ws.pts, S * 6 * np);
    if (e == cudaSuccess) e = dalloc(&ws.pts8, S * 8 * np);
    if (e == cudaSuccess) e = dalloc(&ws.a8, S * n2);
    if (e == cudaSuccess) e = dalloc(&ws.bits, S * n2 / 32);
    if (e == cudaSuccess) e = dalloc(&ws.w, S * n2);
    if (e == cudaSuccess) e = dalloc(&ws.rows, S * 7 * np);
    if (e == cudaSuccess) e = dalloc(&ws.hist, S * (np + 1));
    if (e == cudaSuccess) e = dalloc(&ws.cand, S * TURBOREG_K1_MAX);
    if (e == cudaSuccess) e = dalloc(&ws.piv, S * TURBOREG_K1_MAX);
    if (e == cudaSuccess) e = dalloc(&ws.cliques, S * nh);
    if (e == cudaSuccess) e = dalloc(&ws.rt, S * nh * 16);
    if (e == cudaSuccess) e = dalloc(&ws.inl, S * nh);
    if (e == cudaSuccess) e = dalloc(&ws.hbits, S * nh / 16);
    if (e == cudaSuccess) e = dalloc(&ws.score, S * nh);
    if (e == cudaSuccess) e = dalloc(&ws.feat, S * np * 8);
    if (e == cudaSuccess) e = dalloc(&ws.prob, S * np);
    if (e == cudaSuccess) e = dalloc(&ws.ctl, S);
    if (e == cudaSuccess) e = dalloc(&ws.res, S);
    if (e == cudaSuccess) e = dalloc(&ws.in_src, S * max_n * 3);
    if (e == cudaSuccess) e = dalloc(&ws.in_dst, S * max_n * 3);
    if (e == cudaSuccess) e = dalloc(&ws.desc, desc_bytes(slots));
    if (e == cudaSuccess) e = halloc(&ws.h_views, S);
    if (e == cudaSuccess) e = halloc(&ws.h_pre, static_cast<size_t>(kNumBatchStages) * (S + 1));
    if (e == cudaSuccess) e = halloc(&ws.h_maps, 2 * S);
    if (e == cudaSuccess) {
        ws.map_npad = injected_alloc_failure() ? nullptr : static_cast<int32_t*>(std::calloc(S, sizeof(int32_t)));
        ws.map_cache = injected_alloc_failure() ? nullptr
                                                : static_cast<CUtensorMap*>(std::calloc(2 * S, sizeof(CUtensorMap)));
        if (!ws.map_npad || !ws.map_cache) e = cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ws(ws);
        return e == cudaErrorMemoryAllocation ? TURBOREG_ERR_OOM : TURBOREG_ERR_CUDA;
    }
    return TURBOREG_OK;
}

int check_params(const turboreg_ctx* c, int32_t n, const turboreg_params* p)
{
    if (!p) return TURBOREG_ERR_INVALID_ARG;
    if (n < 3) return TURBOREG_ERR_TOO_FEW;
    if (n > c->max_n) return TURBOREG_ERR_INVALID_ARG;
    if (p->k1 < 1 || p->k1 > TURBOREG_K1_MAX || p->k2 < 1 || p->k2 > TURBOREG_K2_MAX)
        return TURBOREG_ERR_INVALID_ARG;
    if (!(p->tau >= 0.f) || !std::isfinite(p->tau) || !(p->inlier_thresh > 0.f) || !std::isfinite(p->inlier_thresh))
        return TURBOREG_ERR_INVALID_ARG;
    if (p->graph_mode != TURBOREG_GRAPH_O2 && p->graph_mode != TURBOREG_GRAPH_SC2) return TURBOREG_ERR_INVALID_ARG;
    if (p->scoring < TURBOREG_SCORE_IN || p->scoring > TURBOREG_SCORE_MSE) return TURBOREG_ERR_INVALID_ARG;
    if (p->proposal != TURBOREG_PROPOSAL_PLAIN &&
        !(p->proposal == TURBOREG_PROPOSAL_LEARNED && c->has_model))
        return TURBOREG_ERR_INVALID_ARG;
    if (p->learned_min_inliers < 0) return TURBOREG_ERR_INVALID_ARG;
    if (p->kappa_fp64 < 0.f || std::isnan(p->kappa_fp64)) return TURBOREG_ERR_INVALID_ARG;
    return TURBOREG_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// No NaN or Inf among cnt floats: the exponent field of each is checked
// without an early exit, so the compiler vectorises the loop (about 3x
// faster than a branch per element on 15 000 floats).
bool host_finite(const float* p, size_t cnt)
{
    uint32_t bad = 0u;
    for (size_t k = 0; k < cnt; ++k) {
        uint32_t u;
        std::memcpy(&u, p + k, sizeof(u));
        bad |= static_cast<uint32_t>((u & 0x7F800000u) == 0x7F800000u);
    }
    return bad == 0u;
}

void fail_result(turboreg_result* out, int rc)
{
    std::memset(out, 0, sizeof(*out));
    out->R[0] = out->R[4] = out->R[8] = 1.f;
    out->hypothesis = -1;
    out->clique[0] = out->clique[1] = out->clique[2] = -1;
    out->status = rc;
}

ProbView make_view(turboreg_ctx* c, int slot, int64_t in_off, int32_t n, const turboreg_params* p)
{
    Workspace& ws = c->ws;
    const size_t np = ws.np, n2 = np * np, s = static_cast<size_t>(slot);
    ProbView v = {};
    v.in_off = in_off;
    v.n = n;
    v.n_pad = round_up(n, kSc2BN);
    v.ldb = v.n_pad / 32;
    v.k1 = p->k1;
    v.k2 = p->k2;
    v.tau = p->tau;
    v.theta = p->inlier_thresh;
    v.kappa_fp64 = p->kappa_fp64 > 0.f ? p->kappa_fp64 : 100.f;
    v.graph_mode = p->graph_mode;
    v.scoring = p->scoring;
    v.dbg = (p->flags & TURBOREG_FLAG_DEBUG_STALL_COMPAT) ? TR_DBG_STALL_COMPAT : 0u;
    v.pts = ws.pts + s * 6 * np;
    v.pts8 = ws.pts8 + s * 8 * np;
    v.a8 = ws.a8 + s * n2;
    v.bits = ws.bits + s * n2 / 32;
    v.w = ws.w + s * n2;
    int32_t* rows = ws.rows + s * 7 * np;
    v.rowscore = rows;
    v.deg = rows + np;
    v.active = reinterpret_cast<int4*>(rows + 2 * np);   // np is a multiple of 256: 16-byte aligned
    v.rowmax = rows + 6 * np;
    v.hist = ws.hist + s * (np + 1);
    v.cand = ws.cand + s * TURBOREG_K1_MAX;
    v.piv = ws.piv + s * TURBOREG_K1_MAX;
    v.cliques = ws.cliques + s * ws.nh;
    v.rt = ws.rt + s * ws.nh * 16;
    v.inl = ws.inl + s * ws.nh;
    v.hbits = ws.hbits + s * ws.nh / 16;
    v.score = ws.score + s * ws.nh;
    v.feat = ws.feat + s * np * 8;
    v.prob = p->proposal == TURBOREG_PROPOSAL_LEARNED ? ws.prob + s * np : nullptr;
    v.ctl = ws.ctl + s;
    v.res = ws.res + s;
    return v;
}

// TMA descriptors of slot `slot` for the operand tiles of its FP8 adjacency.
int encode_maps(turboreg_ctx* c, int slot, int32_t n_pad, CUtensorMap* out2)
{
    Workspace& ws = c->ws;
    if (ws.map_npad[slot] != n_pad) {
        void* base = ws.a8 + static_cast<size_t>(slot) * ws.np * ws.np;
        const cuuint64_t dims[2] = {static_cast<cuuint64_t>(n_pad), static_cast<cuuint64_t>(n_pad)};
        const cuuint64_t strides[1] = {static_cast<cuuint64_t>(n_pad)};   // bytes between rows
        const cuuint32_t boxA[2] = {static_cast<cuuint32_t>(kSc2BK), static_cast<cuuint32_t>(kSc2BM)};
        const cuuint32_t boxB[2] = {static_cast<cuuint32_t>(kSc2BK), static_cast<cuuint32_t>(kSc2BN)};
        const cuuint32_t estr[2] = {1, 1};
        CUtensorMap* m = ws.map_cache + 2 * slot;
        CUresult r1 = c->encode(&m[0], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, boxA, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r2 = c->encode(&m[1], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, boxB, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
            std::fprintf(stderr, "turboreg: cuTensorMapEncodeTiled failed (%d, %d)\n", (int)r1, (int)r2);
            ws.map_npad[slot] = 0;
            return TURBOREG_ERR_CUDA;
        }
        ws.map_npad[slot] = n_pad;
    }
    out2[0] = ws.map_cache[2 * slot];
    out2[1] = ws.map_cache[2 * slot + 1];
    return TURBOREG_OK;
}

// Fill the host mirrors (h_views, h_pre, h_maps) for problems in slots
// [0, num) and compute the plan's block totals.
int build_plan(turboreg_ctx* c, int32_t num, const int64_t* in_off, const int32_t* n,
               const turboreg_params* const* prm, Plan& plan)
{
    Workspace& ws = c->ws;
    if (c->desc_pending) {   // a queued upload may still read the staging rewritten below
        TR_CHECK(cudaEventSynchronize(c->desc_done));
        c->desc_pending = false;
    }
    plan = Plan();
    plan.num = num;
    plan.bitset = (prm[0]->flags & TURBOREG_FLAG_SC2_BITSET) != 0;
    plan.timed = (prm[0]->flags & TURBOREG_FLAG_STAGE_TIMES) != 0;
    plan.learned = prm[0]->proposal == TURBOREG_PROPOSAL_LEARNED;
    plan.pair_mma = (prm[0]->flags & TURBOREG_FLAG_SC2_SINGLE_CTA) ? 0 : 1;
    plan.sc2_auto = num == 1 && !plan.bitset &&
                    !(prm[0]->flags & (TURBOREG_FLAG_SC2_SINGLE_CTA | TURBOREG_FLAG_SC2_GEMM)) &&
                    round_up(n[0], kSc2BN) <= kSc2AutoMaxNpad && sc2_pair_clusters() > 0;
    if (plan.sc2_auto && round_up(n[0], kSc2BN) <= kSc2BitsetAlwaysNpad) {
        plan.sc2_auto = 0;   // the CUDA-core path is the faster one at any density: no choice to make
        plan.bitset = 1;
    }
    // verification tile: the flags' width for every problem, or for a single
    // problem without tile flags the balanced width (one even wave); the
    // kernel's points per warp (plan.vpw) is the narrowest that holds them all
    const bool vflag = (prm[0]->flags & (TURBOREG_FLAG_VERIFY_PTS32 | TURBOREG_FLAG_VERIFY_PTS128)) != 0;
    const int32_t vpw_flag = (prm[0]->flags & TURBOREG_FLAG_VERIFY_PTS32) ? 32
                             : (prm[0]->flags & TURBOREG_FLAG_VERIFY_PTS128) ? 128 : 64;
    int32_t vppb_max = 0;
    plan.k2_common = prm[0]->k2;
    for (int st = 0; st < kNumBatchStages; ++st) ws.h_pre[st * (num + 1)] = 0;
    for (int32_t b = 0; b < num; ++b) {
        ws.h_views[b] = make_view(c, b, in_off[b], n[b], prm[b]);
        if (plan.bitset) ws.h_views[b].a8 = nullptr;   // the CUDA-core SC^2 reads the bitset only
        if (plan.sc2_auto) {   // the FP8 operand only if the device chooses the GEMM
            ws.h_views[b].a8_auto = ws.h_views[b].a8;
            ws.h_views[b].a8 = nullptr;
        }
        const int32_t vppb = (num == 1 && !vflag) ? balanced_vppb(n[b], prm[b]->k1 * prm[b]->k2, device_sms())
                                                  : 4 * vpw_flag;
        ws.h_views[b].vppb = vppb;
        if (vppb > vppb_max) vppb_max = vppb;
        int32_t blocks[kNumBatchStages];
        stage_blocks(n[b], prm[b]->k1, prm[b]->k2, vppb, blocks);
        for (int st = 0; st < kNumBatchStages; ++st) {
            plan.tot[st] += blocks[st];
            ws.h_pre[st * (num + 1) + b + 1] = plan.tot[st];
        }
        if (n[b] > plan.max_n) plan.max_n = n[b];
        if (b == 0 || n[b] < plan.min_n) plan.min_n = n[b];
        if (prm[b]->k1 > plan.max_k1) plan.max_k1 = prm[b]->k1;
        if (prm[b]->k2 != plan.k2_common) plan.k2_common = 0;
        if (!plan.bitset) {
            const int rc = encode_maps(c, b, ws.h_views[b].n_pad, ws.h_maps + 2 * b);
            if (rc != TURBOREG_OK) return rc;
        }
    }
    plan.vpw = vppb_max <= 4 * 32 ? 32 : vppb_max <= 4 * 64 ? 64 : 128;
    c->last_fp8 = !plan.bitset && !plan.sc2_auto;
    c->last_auto = plan.sc2_auto != 0;
    plan.vcap = num == 1 && !vflag;
    return TURBOREG_OK;
}

// Copy the plan's descriptors to `dev` (views | pre | maps, 128-byte aligned parts).
int upload_desc(turboreg_ctx* c, int32_t num, void* dev, Batch& bt, cudaStream_t s)
{
    Workspace& ws = c->ws;
    uint8_t* d = static_cast<uint8_t*>(dev);
    const size_t v = sizeof(ProbView) * num;
    const size_t p = sizeof(int32_t) * kNumBatchStages * (num + 1);
    const size_t po = (v + 127) / 128 * 128, mo = po + (p + 127) / 128 * 128;
    TR_CHECK(cudaMemcpyAsync(d, ws.h_views, v, cudaMemcpyHostToDevice, s));
    TR_CHECK(cudaMemcpyAsync(d + po, ws.h_pre, p, cudaMemcpyHostToDevice, s));
    TR_CHECK(cudaMemcpyAsync(d + mo, ws.h_maps, sizeof(CUtensorMap) * 2 * num, cudaMemcpyHostToDevice, s));
    TR_CHECK(cudaEventRecord(c->desc_done, s));
    c->desc_pending = true;
    bt.views = reinterpret_cast<const ProbView*>(d);
    bt.pre = reinterpret_cast<const int32_t*>(d + po);
    bt.maps = reinterpret_cast<const CUtensorMap*>(d + mo);
    bt.num = num;
    return TURBOREG_OK;
}

// Enqueue the whole path for the plan's problems (inputs on the device).
int enqueue_plan(turboreg_ctx* c, const Plan& pl, const Batch& bt, const float* dsrc, const float* ddst,
                 turboreg_result* out)
{
    cudaStream_t s = c->stream;
    const bool timed = pl.timed != 0;
#define TR_EV(k) \
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[k], s, cudaEventRecordExternal))
    TR_EV(0);
    // the control blocks start cleared: the finalize kernel of the previous
    // registration resets the fields that must start at zero (run_plan clears
    // them when another entry point may have left them set)
    launch_pack(bt, pl.tot[ST_PACK], dsrc, ddst, s);
    TR_EV(1);
    launch_compat(bt, pl.tot[ST_COMPAT], s, pl.sc2_auto != 0);
    TR_EV(2);
    bool fused = false;
    if (pl.sc2_auto) {
        // one problem: the CUDA-core kernel chooses the path from the degrees and
        // either computes SC^2 or expands the FP8 operand; the GEMM then runs or
        // returns at once.  Both keep the histogram for the count blocks.
        launch_sc2_bitset(bt, pl.tot[ST_BITSET], pl.max_n, pl.min_n, sc2_pair_clusters(), s);
        launch_sc2_tcgen05(bt, pl.tot[ST_GEMM], pl.max_n, true, s, true);
        fused = true;
    } else if (pl.bitset) {
        // the histogram is complete in global memory at the end of the kernel;
        // one problem: the count blocks choose the threshold from it
        fused = launch_sc2_bitset(bt, pl.tot[ST_BITSET], pl.max_n, pl.min_n, 0, s) && pl.num == 1;
    } else {
        // one problem whose histogram fits in the GEMM's shared memory: the
        // count blocks choose the threshold; a batch or a larger problem adds
        // a select launch
        fused = launch_sc2_tcgen05(bt, pl.tot[ST_GEMM], pl.max_n, pl.pair_mma != 0, s);
    }
    TR_EV(3);
    if (!fused && !pl.learned) launch_select(bt, s);
    if (pl.learned) {
        // learned proposal: features -> MLP -> histogram of floor(W p_i p_j) -> threshold
        TR_CHECK(cudaMemsetAsync(c->ws.hist, 0, sizeof(uint32_t) * (c->ws.np + 1) * pl.num, s));
        launch_features(bt, s);
        launch_mlp_proposal(bt, pl.tot[ST_MLP], c->mlp_wbf, s);
        launch_hist(bt, pl.tot[ST_HIST], pl.max_n, s);
        launch_select(bt, s);
    }
    TR_EV(4);
    // the count blocks stage the histogram in (at most 48 KB of) shared memory
    bool sel_in_count = fused && !pl.learned;
    if (sel_in_count && static_cast<size_t>(pl.max_n + 4) * 4 > 48 * 1024) {
        launch_select(bt, s);
        sel_in_count = false;
    }
    launch_count_emit(bt, pl.tot, sel_in_count, pl.max_n, s);
    TR_EV(5);
    launch_pgs(bt, pl.tot[ST_PGS], pl.k2_common, pl.max_k1, s);   // also ranks the pivots and solves the cliques' Kabsch
    TR_EV(6);
    launch_verify(bt, pl.tot[ST_VERIFY], pl.vpw, pl.vcap != 0, s);
    TR_EV(7);
    launch_finalize(bt, out, s);
    TR_EV(8);
#undef TR_EV
    TR_CHECK(cudaGetLastError());
    return TURBOREG_OK;
}

void drop_slot(turboreg_ctx::GraphSlot& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    if (g.desc) cudaFree(g.desc);
    g = turboreg_ctx::GraphSlot();
}

// Signature of a plan: everything the captured graph bakes in.
std::vector<uint8_t> plan_key(turboreg_ctx* c, const Plan& pl)
{
    std::vector<uint8_t> k;
    auto put = [&](const void* p, size_t b) {
        const uint8_t* q = static_cast<const uint8_t*>(p);
        k.insert(k.end(), q, q + b);
    };
    put(&pl, sizeof(pl));
    for (int32_t b = 0; b < pl.num; ++b) {
        const ProbView& v = c->ws.h_views[b];
        put(&v.in_off, sizeof(v.in_off));
        put(&v.n, sizeof(v.n));
        put(&v.k1, sizeof(v.k1));
        put(&v.k2, sizeof(v.k2));
        put(&v.tau, sizeof(v.tau));
        put(&v.theta, sizeof(v.theta));
        put(&v.kappa_fp64, sizeof(v.kappa_fp64));
        put(&v.graph_mode, sizeof(v.graph_mode));
        put(&v.scoring, sizeof(v.scoring));
        put(&v.dbg, sizeof(v.dbg));
    }
    return k;
}

// Run a plan: replay its captured graph (capturing it on first use) with the
// given input pointers; TURBOREG_FLAG_NO_GRAPH launches the stages directly.
int run_plan(turboreg_ctx* c, const Plan& pl, bool no_graph, const float* dsrc, const float* ddst,
             turboreg_result* out)
{
    if (c->ctl_dirty)   // outside any capture: not part of the replayed graph
        TR_CHECK(cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl) * static_cast<size_t>(c->ws.slots), c->stream));
    // clean again only once this registration, finalize included, is enqueued
    c->ctl_dirty = true;
    if (no_graph) {
        Batch bt;
        int rc = upload_desc(c, pl.num, c->ws.desc, bt, c->stream);
        if (rc != TURBOREG_OK) return rc;
        rc = enqueue_plan(c, pl, bt, dsrc, ddst, out);
        if (rc == TURBOREG_OK) c->ctl_dirty = false;
        return rc;
    }
    const std::vector<uint8_t> key = plan_key(c, pl);
    turboreg_ctx::GraphSlot* g = nullptr;
    bool fresh = false;   // captured by this call: the graph holds this call's pointers already
    for (auto& sl : c->gslot)
        if (sl.used && sl.key == key) g = &sl;
    if (!g) {
        g = &c->gslot[0];
        for (auto& sl : c->gslot) {
            if (!sl.used) { g = &sl; break; }
            if (sl.stamp < g->stamp) g = &sl;
        }
        // an evicted graph may still have launches queued (asynchronous calls)
        if (g->used) TR_CHECK(cudaStreamSynchronize(c->stream));
        drop_slot(*g);
        TR_CHECK(cudaMalloc(&g->desc, desc_bytes(pl.num)));
        int rc = upload_desc(c, pl.num, g->desc, g->batch, c->stream);
        if (rc != TURBOREG_OK) return rc;
        TR_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_plan(c, pl, g->batch, dsrc, ddst, out);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (rc != TURBOREG_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            drop_slot(*g);
            std::fprintf(stderr, "turboreg: graph capture failed: %s\n", cudaGetErrorString(e));
            return rc != TURBOREG_OK ? rc : TURBOREG_ERR_CUDA;
        }
        g->graph = graph;
        size_t cnt = 0;
        TR_CHECK(cudaGraphGetNodes(graph, nullptr, &cnt));
        std::vector<cudaGraphNode_t> nodes(cnt);
        TR_CHECK(cudaGraphGetNodes(graph, nodes.data(), &cnt));
        for (size_t k = 0; k < cnt; ++k) {
            cudaGraphNodeType ty;
            TR_CHECK(cudaGraphNodeGetType(nodes[k], &ty));
            if (ty != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            TR_CHECK(cudaGraphKernelNodeGetParams(nodes[k], &kp));
            if (kp.func == pack_kernel_func()) {
                g->pack_node = nodes[k];
                g->pack_params = kp;
            } else if (kp.func == finalize_kernel_func()) {
                g->fin_node = nodes[k];
                g->fin_params = kp;
            }
        }
        if (!g->pack_node || !g->fin_node || cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            drop_slot(*g);
            return TURBOREG_ERR_CUDA;
        }
        g->used = true;
        g->key = key;
        g->src = dsrc;
        g->dst = ddst;
        g->out = out;
        fresh = true;
    }
    g->stamp = ++c->gclock;
    // the input and result pointers are patched only when they differ from
    // the ones the executable graph holds (a caller reusing its buffers, or
    // the synchronous call's staged inputs and result slot, skips both updates)
    if (!fresh && (dsrc != g->src || ddst != g->dst)) {
        g->src = dsrc;
        g->dst = ddst;
        g->args[0] = &g->batch;
        g->args[1] = &g->src;
        g->args[2] = &g->dst;
        cudaKernelNodeParams kp = g->pack_params;
        kp.kernelParams = g->args;
        kp.extra = nullptr;
        const cudaError_t e = cudaGraphExecKernelNodeSetParams(g->exec, g->pack_node, &kp);
        if (e != cudaSuccess) {
            g->src = g->dst = nullptr;   // unknown now: patched again on the next call
            std::fprintf(stderr, "turboreg: graph input update failed: %s\n", cudaGetErrorString(e));
            return TURBOREG_ERR_CUDA;
        }
    }
    if (!fresh && out != g->out) {
        g->out = out;
        g->fin_args[0] = &g->batch;
        g->fin_args[1] = &g->out;
        cudaKernelNodeParams fp = g->fin_params;
        fp.kernelParams = g->fin_args;
        fp.extra = nullptr;
        const cudaError_t e = cudaGraphExecKernelNodeSetParams(g->exec, g->fin_node, &fp);
        if (e != cudaSuccess) {
            g->out = nullptr;
            std::fprintf(stderr, "turboreg: graph result update failed: %s\n", cudaGetErrorString(e));
            return TURBOREG_ERR_CUDA;
        }
    }
    TR_CHECK(cudaGraphLaunch(g->exec, c->stream));
    c->ctl_dirty = false;
    return TURBOREG_OK;
}

int collect_times(turboreg_ctx* c)
{
    if (!c->have_times) return TURBOREG_OK;
    for (int k = 0; k < kNumStages; ++k) {
        if (cudaEventElapsedTime(&c->stage_ms[k], c->ev[k], c->ev[k + 1]) != cudaSuccess) {
            cudaGetLastError();   // not fatal: report the stage as unmeasured
            c->stage_ms[k] = -1.f;
        }
    }
    return TURBOREG_OK;
}

// Learned proposal fallback rule: the plain proposal decides when the learned
// run found no hypothesis or its best inlier number is below the floor.
bool needs_fallback(const turboreg_result& r, int32_t n, const turboreg_params* p)
{
    if (p->proposal != TURBOREG_PROPOSAL_LEARNED) return false;
    if (r.status == TURBOREG_ERR_NO_HYPOTHESIS) return true;
    if (r.status != TURBOREG_OK) return false;
    const int32_t floor_in = p->learned_min_inliers > 0 ? p->learned_min_inliers : (n / 200 > 10 ? n / 200 : 10);
    return r.inlier_count < floor_in;
}

enum PtrKind { kPtrDevice, kPtrPinned, kPtrPageable };

// mapped: for page-locked host memory mapped into the device's address space,
// the address kernels read it at (else null)
PtrKind pointer_kind(const void* p, const void** mapped = nullptr)
{
    if (mapped) *mapped = nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kPtrPageable;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return kPtrDevice;
    if (a.type != cudaMemoryTypeHost) return kPtrPageable;
    if (mapped) *mapped = a.devicePointer;
    return kPtrPinned;
}

// Checks, input copies and the launch of one registration (graph replay or
// direct launches); finalize writes the result to `out` (page-locked host or
// device memory).  async: host inputs must be page-locked.  *s_in, *d_in
// receive the device inputs used.
int enqueue_single(turboreg_ctx* c, const float* src, const float* dst, int32_t n, const turboreg_params* p,
                   bool async, const float** s_in, const float** d_in, bool* timed, turboreg_result* out)
{
    int rc = check_params(c, n, p);
    if (rc != TURBOREG_OK) return rc;
    TR_CHECK(cudaSetDevice(c->device));
    const void *ms = nullptr, *md = nullptr;
    const PtrKind ks = pointer_kind(src, &ms), kd = pointer_kind(dst, &md);
    if (async && (ks == kPtrPageable || kd == kPtrPageable)) return TURBOREG_ERR_INVALID_ARG;
    const size_t bytes = static_cast<size_t>(n) * 3 * sizeof(float);
    // page-locked inputs mapped into the device's address space are read in
    // place by the first kernel (over the CPU-GPU link, no copy-engine
    // operation); other host inputs are copied to the workspace first
    if (ks != kPtrDevice) {
        if (!host_finite(src, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        if (ms != nullptr) {
            *s_in = static_cast<const float*>(ms);
        } else {
            TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src, bytes, cudaMemcpyHostToDevice, c->stream));
            *s_in = c->ws.in_src;
        }
    }
    if (kd != kPtrDevice) {
        if (!host_finite(dst, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        if (md != nullptr) {
            *d_in = static_cast<const float*>(md);
        } else {
            TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst, bytes, cudaMemcpyHostToDevice, c->stream));
            *d_in = c->ws.in_dst;
        }
    }
    Plan pl;
    const int64_t off0 = 0;
    rc = build_plan(c, 1, &off0, &n, &p, pl);
    if (rc != TURBOREG_OK) return rc;
    const bool no_graph = (p->flags & TURBOREG_FLAG_NO_GRAPH) != 0;
    rc = run_plan(c, pl, no_graph, *s_in, *d_in, out);
    if (rc != TURBOREG_OK) return rc;
    c->last_n = n;
    c->last_npad = round_up(n, kSc2BN);
    c->last_k1 = p->k1;
    c->last_k2 = p->k2;
    *timed = !async && pl.timed != 0;
    return TURBOREG_OK;
}

}  // namespace

extern "C" {

void turboreg_default_params(turboreg_params* p, float tau, int32_t k1, float inlier_thresh)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tau = tau;
    p->k1 = k1;
    p->k2 = 2;
    p->inlier_thresh = inlier_thresh;
    p->graph_mode = TURBOREG_GRAPH_O2;
    p->proposal = TURBOREG_PROPOSAL_PLAIN;
    p->kappa_fp64 = 100.f;
    p->flags = 0;
}

const char* turboreg_status_string(int status)
{
    switch (status) {
        case TURBOREG_OK: return "ok";
        case TURBOREG_ERR_INVALID_ARG: return "invalid argument";
        case TURBOREG_ERR_TOO_FEW: return "fewer than 3 correspondences";
        case TURBOREG_ERR_NONFINITE: return "non-finite coordinate";
        case TURBOREG_ERR_OOM: return "out of memory";
        case TURBOREG_ERR_CUDA: return "CUDA error";
        case TURBOREG_ERR_TIMEOUT: return "device wait timed out";
        case TURBOREG_ERR_NO_HYPOTHESIS: return "no valid hypothesis";
        default: return "unknown status";
    }
}

int turboreg_create(int device, int32_t max_n, int32_t max_batch, void* cuda_stream, turboreg_ctx** out)
{
    if (!out) return TURBOREG_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_n < 3 || max_n > TURBOREG_MAX_N || max_batch < 1) return TURBOREG_ERR_INVALID_ARG;
    if (static_cast<int64_t>(max_n) * max_batch > (int64_t)1 << 28) return TURBOREG_ERR_INVALID_ARG;
    int ndev = 0;
    TR_CHECK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return TURBOREG_ERR_INVALID_ARG;
    TR_CHECK(cudaSetDevice(device));
    int major = 0;
    TR_CHECK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
    if (major < 10) {
        std::fprintf(stderr, "turboreg: device %d is not an sm_100-family GPU\n", device);
        return TURBOREG_ERR_CUDA;
    }
    t_alloc_seq = 0;
    const char* fail_env = std::getenv("TURBOREG_DEBUG_FAIL_ALLOC");
    t_alloc_fail = fail_env ? std::atoi(fail_env) : 0;
    turboreg_ctx* c = injected_alloc_failure() ? nullptr : new (std::nothrow) turboreg_ctx();
    if (!c) return TURBOREG_ERR_OOM;
    c->device = device;
    c->max_n = max_n;
    c->max_batch = max_batch;
    int rc = alloc_ws(c->ws, max_n, max_batch);
    if (rc != TURBOREG_OK) {
        delete c;
        return rc;
    }
    if (halloc(&c->host_res, static_cast<size_t>(max_batch)) != cudaSuccess) {
        free_ws(c->ws);
        delete c;
        return TURBOREG_ERR_OOM;
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            turboreg_destroy(c);
            return TURBOREG_ERR_CUDA;
        }
        c->own_stream = true;
    }
    for (int k = 0; k <= kNumStages; ++k) {
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
            turboreg_destroy(c);
            return TURBOREG_ERR_CUDA;
        }
    }
    if (cudaEventCreateWithFlags(&c->desc_done, cudaEventDisableTiming) != cudaSuccess) {
        turboreg_destroy(c);
        return TURBOREG_ERR_CUDA;
    }
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        std::fprintf(stderr, "turboreg: cuTensorMapEncodeTiled not available\n");
        turboreg_destroy(c);
        return TURBOREG_ERR_CUDA;
    }
    c->encode = reinterpret_cast<EncodeTiledFn>(fn);
    cudaError_t se = sc2_tcgen05_setup();
    if (se == cudaSuccess) se = sc2_bitset_setup();
    if (se == cudaSuccess) se = topk_setup();
    if (se == cudaSuccess) se = verify_pgs_setup();
    if (se == cudaSuccess) se = mlp_setup();
    if (se != cudaSuccess) {
        std::fprintf(stderr, "turboreg: kernel set-up failed: %s\n", cudaGetErrorString(se));
        cudaGetLastError();
        turboreg_destroy(c);
        return TURBOREG_ERR_CUDA;
    }
    *out = c;
    return TURBOREG_OK;
}

void turboreg_destroy(turboreg_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& sl : c->gslot) drop_slot(sl);
    for (int k = 0; k <= kNumStages; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->desc_done) cudaEventDestroy(c->desc_done);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    free_ws(c->ws);
    if (c->host_res) cudaFreeHost(c->host_res);
    if (c->mlp_wbf) cudaFree(c->mlp_wbf);
    delete c;
}

int turboreg_register(turboreg_ctx* c, const float* src, const float* dst, int32_t n, const turboreg_params* p,
                      turboreg_result* out)
{
    if (!c || !src || !dst || !out) return TURBOREG_ERR_INVALID_ARG;
    const float* s_in = src;
    const float* d_in = dst;
    bool timed = false;
    int rc = enqueue_single(c, src, dst, n, p, false, &s_in, &d_in, &timed, c->host_res);
    if (rc == TURBOREG_ERR_NONFINITE) {   // host inputs rejected before any device work
        TR_CHECK(cudaStreamSynchronize(c->stream));
        fail_result(out, rc);
        return rc;
    }
    if (rc != TURBOREG_OK) {
        if (rc == TURBOREG_ERR_INVALID_ARG || rc == TURBOREG_ERR_TOO_FEW) fail_result(out, rc);
        return rc;
    }
    TR_CHECK(cudaStreamSynchronize(c->stream));   // finalize wrote c->host_res
    c->have_times = timed;
    rc = collect_times(c);
    if (rc != TURBOREG_OK) return rc;
    *out = c->host_res[0];
    if (needs_fallback(*out, n, p)) {
        turboreg_params q = *p;
        q.proposal = TURBOREG_PROPOSAL_PLAIN;
        q.flags &= ~TURBOREG_FLAG_STAGE_TIMES;
        const int rc2 = turboreg_register(c, s_in, d_in, n, &q, out);
        out->used_fallback = 1;
        return rc2;
    }
    return out->status;
}

int turboreg_register_async(turboreg_ctx* c, const float* src, const float* dst, int32_t n,
                            const turboreg_params* p, turboreg_result* out)
{
    if (!c || !src || !dst || !out || !p) return TURBOREG_ERR_INVALID_ARG;
    if (p->proposal == TURBOREG_PROPOSAL_LEARNED) return TURBOREG_ERR_INVALID_ARG;
    if (pointer_kind(out) == kPtrPageable) return TURBOREG_ERR_INVALID_ARG;
    const float* s_in = src;
    const float* d_in = dst;
    bool timed = false;
    const int rc = enqueue_single(c, src, dst, n, p, true, &s_in, &d_in, &timed, out);
    if (rc != TURBOREG_OK) return rc;
    c->have_times = false;
    return TURBOREG_OK;
}

int turboreg_synchronize(turboreg_ctx* c)
{
    if (!c) return TURBOREG_ERR_INVALID_ARG;
    TR_CHECK(cudaSetDevice(c->device));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    return TURBOREG_OK;
}

int turboreg_register_batched(turboreg_ctx* c, const float* src_cat, const float* dst_cat, const int64_t* offsets,
                              int32_t num, const turboreg_params* params, int32_t params_count,
                              turboreg_result* out)
{
    if (!c || !src_cat || !dst_cat || !offsets || !params || !out) return TURBOREG_ERR_INVALID_ARG;
    if (num < 1 || num > c->max_batch) return TURBOREG_ERR_INVALID_ARG;
    if (params_count != 1 && params_count != num) return TURBOREG_ERR_INVALID_ARG;
    if (offsets[0] != 0) return TURBOREG_ERR_INVALID_ARG;
    for (int32_t b = 0; b < num; ++b) {
        if (offsets[b + 1] < offsets[b]) return TURBOREG_ERR_INVALID_ARG;
        if (offsets[b + 1] - offsets[b] > c->max_n) return TURBOREG_ERR_INVALID_ARG;
    }
    const int64_t total = offsets[num];
    if (total > static_cast<int64_t>(c->max_n) * c->max_batch) return TURBOREG_ERR_INVALID_ARG;
    const uint32_t mode = params->flags & (TURBOREG_FLAG_SC2_BITSET | TURBOREG_FLAG_NO_GRAPH);
    for (int32_t b = 0; b < params_count; ++b)
        if ((params[b].flags & (TURBOREG_FLAG_SC2_BITSET | TURBOREG_FLAG_NO_GRAPH)) != mode ||
            params[b].proposal != params->proposal)
            return TURBOREG_ERR_INVALID_ARG;   // one SC^2 path, launch mode and proposal per batch
    TR_CHECK(cudaSetDevice(c->device));
    const bool dsrc = is_device_ptr(src_cat), ddst = is_device_ptr(dst_cat);
    const size_t bytes = static_cast<size_t>(total) * 3 * sizeof(float);
    const float* s_in = src_cat;
    const float* d_in = dst_cat;
    if (!dsrc && total > 0) {
        TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src_cat, bytes, cudaMemcpyHostToDevice, c->stream));
        s_in = c->ws.in_src;
    }
    if (!ddst && total > 0) {
        TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst_cat, bytes, cudaMemcpyHostToDevice, c->stream));
        d_in = c->ws.in_dst;
    }
    // problems that fail host-side checks are reported without device work
    std::vector<int> pre(num);
    std::vector<int32_t> nn;
    std::vector<int64_t> off;
    std::vector<const turboreg_params*> pp;
    for (int32_t b = 0; b < num; ++b) {
        const turboreg_params* p = params_count == 1 ? params : params + b;
        const int32_t n = static_cast<int32_t>(offsets[b + 1] - offsets[b]);
        int rc = check_params(c, n, p);
        if (rc == TURBOREG_OK && !dsrc && !host_finite(src_cat + 3 * offsets[b], static_cast<size_t>(n) * 3))
            rc = TURBOREG_ERR_NONFINITE;
        if (rc == TURBOREG_OK && !ddst && !host_finite(dst_cat + 3 * offsets[b], static_cast<size_t>(n) * 3))
            rc = TURBOREG_ERR_NONFINITE;
        pre[b] = rc;
        if (rc != TURBOREG_OK) continue;
        nn.push_back(n);
        off.push_back(offsets[b]);
        pp.push_back(p);
    }
    const int32_t m = static_cast<int32_t>(nn.size());
    bool timed = false;
    if (m > 0) {
        Plan pl;
        int rc = build_plan(c, m, off.data(), nn.data(), pp.data(), pl);
        if (rc == TURBOREG_OK)
            rc = run_plan(c, pl, (mode & TURBOREG_FLAG_NO_GRAPH) != 0, s_in, d_in, c->host_res);
        if (rc != TURBOREG_OK) return rc;
        timed = pl.timed != 0;
    }
    TR_CHECK(cudaStreamSynchronize(c->stream));
    c->have_times = timed;   // stage times of the batch's pipeline (the fallback's are not kept)
    if (timed) collect_times(c);
    int32_t q = 0;
    std::vector<int32_t> fb;   // problems the plain proposal must decide (learned fallback)
    for (int32_t b = 0; b < num; ++b) {
        if (pre[b] != TURBOREG_OK) fail_result(&out[b], pre[b]);
        else {
            out[b] = c->host_res[q++];
            const turboreg_params* p = params_count == 1 ? params : params + b;
            if (needs_fallback(out[b], static_cast<int32_t>(offsets[b + 1] - offsets[b]), p)) fb.push_back(b);
        }
    }
    if (!fb.empty()) {
        std::vector<int32_t> fn;
        std::vector<int64_t> fo;
        std::vector<turboreg_params> fq;
        for (int32_t b : fb) {
            turboreg_params pq = params_count == 1 ? params[0] : params[b];
            pq.proposal = TURBOREG_PROPOSAL_PLAIN;
            fq.push_back(pq);
            fn.push_back(static_cast<int32_t>(offsets[b + 1] - offsets[b]));
            fo.push_back(offsets[b]);
        }
        std::vector<const turboreg_params*> fp(fq.size());
        for (size_t k = 0; k < fq.size(); ++k) fp[k] = &fq[k];
        Plan pl;
        int rc = build_plan(c, static_cast<int32_t>(fb.size()), fo.data(), fn.data(), fp.data(), pl);
        if (rc == TURBOREG_OK)
            rc = run_plan(c, pl, (mode & TURBOREG_FLAG_NO_GRAPH) != 0, s_in, d_in, c->host_res);
        if (rc != TURBOREG_OK) return rc;
        TR_CHECK(cudaStreamSynchronize(c->stream));
        for (size_t k = 0; k < fb.size(); ++k) {
            out[fb[k]] = c->host_res[k];
            out[fb[k]].used_fallback = 1;
        }
    }
    if (m > 0) {   // inspection buffers refer to the first processed problem (slot 0)
        c->last_n = nn[0];
        c->last_npad = round_up(nn[0], kSc2BN);
        c->last_k1 = pp[0]->k1;
        c->last_k2 = pp[0]->k2;
    }
    return TURBOREG_OK;
}

int turboreg_debug_sc2_path(turboreg_ctx* c, int32_t* path)
{
    if (!c || !path) return TURBOREG_ERR_INVALID_ARG;
    TR_CHECK(cudaSetDevice(c->device));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    if (c->last_auto) {
        Ctl h;
        TR_CHECK(cudaMemcpy(&h, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
        *path = static_cast<int32_t>(h.sc2_path);
    } else {
        *path = c->last_fp8 ? 2 : 1;
    }
    return TURBOREG_OK;
}

int turboreg_debug_shape(turboreg_ctx* c, int32_t* n, int32_t* n_pad, int32_t* n_pivots, int32_t* n_hyp)
{
    if (!c) return TURBOREG_ERR_INVALID_ARG;
    Ctl h;
    TR_CHECK(cudaSetDevice(c->device));
    TR_CHECK(cudaMemcpy(&h, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (n) *n = c->last_n;
    if (n_pad) *n_pad = c->last_npad;
    if (n_pivots) *n_pivots = h.n_pivots;
    if (n_hyp) *n_hyp = h.n_pivots * c->last_k2;
    return TURBOREG_OK;
}

int64_t turboreg_debug_copy(turboreg_ctx* c, int which, void* dst, int64_t max_bytes)
{
    if (!c || !dst || max_bytes < 0) return -TURBOREG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return -TURBOREG_ERR_CUDA;
    // asynchronous registrations may still be running on the context's stream
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -TURBOREG_ERR_CUDA;
    Ctl h;
    if (cudaMemcpy(&h, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return -TURBOREG_ERR_CUDA;
    turboreg_params p0;
    turboreg_default_params(&p0, 0.f, c->last_k1 > 0 ? c->last_k1 : 1, 1.f);
    p0.k2 = c->last_k2 > 0 ? c->last_k2 : 1;
    const ProbView v = make_view(c, 0, 0, c->last_n, &p0);   // slot 0
    const size_t np = static_cast<size_t>(c->last_npad);
    const size_t nh = static_cast<size_t>(h.n_pivots) * c->last_k2;
    const void* src = nullptr;
    size_t bytes = 0;
    switch (which) {
        case TURBOREG_BUF_ADJ_BITS: src = v.bits; bytes = np * np / 8; break;
        case TURBOREG_BUF_ADJ_FP8:
            if (!c->last_fp8 && !(c->last_auto && h.sc2_path == 2u))
                return -TURBOREG_ERR_INVALID_ARG;   // not materialised by that plan (or that choice)
            src = v.a8;
            bytes = np * np;
            break;
        case TURBOREG_BUF_SC2: src = v.w; bytes = np * np * 2; break;
        case TURBOREG_BUF_PIVOTS: src = v.piv; bytes = static_cast<size_t>(h.n_pivots) * 16; break;
        case TURBOREG_BUF_CLIQUES: src = v.cliques; bytes = nh * 16; break;
        case TURBOREG_BUF_RT: src = v.rt; bytes = nh * 64; break;
        case TURBOREG_BUF_INLIERS: src = v.inl; bytes = nh * 4; break;
        case TURBOREG_BUF_SCORES: src = v.score; bytes = nh * 8; break;
        case TURBOREG_BUF_ROWSCORE: src = v.rowscore; bytes = static_cast<size_t>(c->last_n) * 4; break;
        case TURBOREG_BUF_DEGREE: src = v.deg; bytes = static_cast<size_t>(c->last_n) * 4; break;
        case TURBOREG_BUF_FEATURES: src = v.feat; bytes = static_cast<size_t>(c->last_n) * 32; break;
        case TURBOREG_BUF_PROB: src = c->ws.prob; bytes = static_cast<size_t>(c->last_n) * 4; break;
        default: return -TURBOREG_ERR_INVALID_ARG;
    }
    if (bytes > static_cast<size_t>(max_bytes)) bytes = static_cast<size_t>(max_bytes);
    if (bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return -TURBOREG_ERR_CUDA;
    return static_cast<int64_t>(bytes);
}

int turboreg_stage_times(turboreg_ctx* c, float* ms, int32_t max)
{
    if (!c || !ms) return -TURBOREG_ERR_INVALID_ARG;
    const int k = max < kNumStages ? max : kNumStages;
    for (int q = 0; q < k; ++q) ms[q] = c->have_times ? c->stage_ms[q] : -1.f;
    return kNumStages;
}

const char* turboreg_stage_name(int32_t stage)
{
    return (stage >= 0 && stage < kNumStages) ? kStageNames[stage] : "";
}

int turboreg_set_proposal_model(turboreg_ctx* c, const float* params)
{
    if (!c || !params) return TURBOREG_ERR_INVALID_ARG;
    for (int k = 0; k < kMlpParams; ++k)
        if (!std::isfinite(params[k])) return TURBOREG_ERR_NONFINITE;
    TR_CHECK(cudaSetDevice(c->device));
    if (!c->mlp_wbf) TR_CHECK(cudaMalloc(&c->mlp_wbf, sizeof(float) * kMlpParams));
    float* tmp = nullptr;
    TR_CHECK(cudaMalloc(&tmp, sizeof(float) * kMlpParams));
    cudaError_t e = cudaMemcpyAsync(tmp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        launch_mlp_round(tmp, c->mlp_wbf, c->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "turboreg: setting the proposal model failed: %s\n", cudaGetErrorString(e));
        return TURBOREG_ERR_CUDA;
    }
    c->has_model = true;
    for (auto& sl : c->gslot) drop_slot(sl);   // captured graphs bake the model pointer in: recapture
    return TURBOREG_OK;
}

int turboreg_score_transforms(turboreg_ctx* c, const float* src, const float* dst, int32_t n,
                              const turboreg_params* p, const float* rt, int32_t m, int32_t* out_in,
                              uint64_t* out_units)
{
    if (!c || !src || !dst || !p || !rt || !out_in) return TURBOREG_ERR_INVALID_ARG;
    if (m < 1 || m > TURBOREG_K1_MAX) return TURBOREG_ERR_INVALID_ARG;
    if (!host_finite(rt, static_cast<size_t>(m) * 12)) return TURBOREG_ERR_INVALID_ARG;
    turboreg_params q = *p;
    q.proposal = TURBOREG_PROPOSAL_PLAIN;
    q.flags = 0;
    q.k1 = m;
    q.k2 = 1;
    q.graph_mode = TURBOREG_GRAPH_O2;
    if (!(q.tau >= 0.f) || !std::isfinite(q.tau)) q.tau = 0.f;
    int rc = check_params(c, n, &q);
    if (rc != TURBOREG_OK) return rc;
    TR_CHECK(cudaSetDevice(c->device));
    const size_t bytes = static_cast<size_t>(n) * 3 * sizeof(float);
    const float* s_in = src;
    const float* d_in = dst;
    if (!is_device_ptr(src)) {
        if (!host_finite(src, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s_in = c->ws.in_src;
    }
    if (!is_device_ptr(dst)) {
        if (!host_finite(dst, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst, bytes, cudaMemcpyHostToDevice, c->stream));
        d_in = c->ws.in_dst;
    }
    Plan pl;
    const int64_t off0 = 0;
    const turboreg_params* pq = &q;
    rc = build_plan(c, 1, &off0, &n, &pq, pl);
    if (rc != TURBOREG_OK) return rc;
    Batch bt;
    rc = upload_desc(c, 1, c->ws.desc, bt, c->stream);
    if (rc != TURBOREG_OK) return rc;
    const ProbView& v = c->ws.h_views[0];
    // hypotheses in the verification layout: R (9), t (3), kappa, flags = 1 (valid)
    std::vector<float> h(static_cast<size_t>(m) * 16, 0.f);
    const int32_t valid = 1;
    for (int32_t k = 0; k < m; ++k) {
        std::memcpy(&h[static_cast<size_t>(k) * 16], rt + static_cast<size_t>(k) * 12, 12 * sizeof(float));
        std::memcpy(&h[static_cast<size_t>(k) * 16 + 13], &valid, sizeof(valid));
    }
    c->ctl_dirty = true;   // this entry point runs part of the path: no reset at its end
    TR_CHECK(cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl), c->stream));
    launch_pack(bt, pl.tot[ST_PACK], s_in, d_in, c->stream);
    TR_CHECK(cudaMemcpyAsync(v.rt, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    TR_CHECK(cudaMemcpyAsync(&v.ctl->n_pivots, &m, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    TR_CHECK(cudaMemsetAsync(v.inl, 0, sizeof(int32_t) * m, c->stream));
    TR_CHECK(cudaMemsetAsync(v.score, 0, sizeof(unsigned long long) * m, c->stream));
    launch_verify(bt, pl.tot[ST_VERIFY], pl.vpw, pl.vcap != 0, c->stream);
    TR_CHECK(cudaGetLastError());
    TR_CHECK(cudaMemcpyAsync(out_in, v.inl, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, c->stream));
    if (out_units)
        TR_CHECK(cudaMemcpyAsync(out_units, v.score, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost,
                                 c->stream));
    Ctl hc;
    TR_CHECK(cudaMemcpyAsync(&hc, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    if (hc.err & TR_ERR_NONFINITE) return TURBOREG_ERR_NONFINITE;
    if (hc.err) return TURBOREG_ERR_TIMEOUT;
    return TURBOREG_OK;
}

int turboreg_kabsch_cliques(turboreg_ctx* c, const float* src, const float* dst, int32_t n,
                            const turboreg_params* p, const int32_t* idx, int32_t k, int32_t m, float* out_rt,
                            int32_t* out_valid)
{
    if (!c || !src || !dst || !p || !idx || !out_rt || !out_valid) return TURBOREG_ERR_INVALID_ARG;
    const int64_t cap = 4ll * TURBOREG_K1_MAX * TURBOREG_K2_MAX;
    if (k < 3 || k > 32 || m < 1 || static_cast<int64_t>(m) * k > cap) return TURBOREG_ERR_INVALID_ARG;
    if (k == 3 && static_cast<int64_t>(m) > static_cast<int64_t>(TURBOREG_K1_MAX) * TURBOREG_K2_MAX)
        return TURBOREG_ERR_INVALID_ARG;
    if (n < 3) return TURBOREG_ERR_TOO_FEW;
    for (int64_t q = 0; q < static_cast<int64_t>(m) * k; ++q)
        if (idx[q] < 0 || idx[q] >= n) return TURBOREG_ERR_INVALID_ARG;
    turboreg_params q = *p;
    q.proposal = TURBOREG_PROPOSAL_PLAIN;
    q.flags = 0;
    q.graph_mode = TURBOREG_GRAPH_O2;
    q.scoring = TURBOREG_SCORE_IN;
    // k = 3 uses the path's hypothesis layout: m cliques as m pivots with K2 = 1
    q.k1 = k == 3 ? (m < TURBOREG_K1_MAX ? m : TURBOREG_K1_MAX) : 1;
    q.k2 = k == 3 ? (m + q.k1 - 1) / q.k1 : 1;
    if (!(q.tau >= 0.f) || !std::isfinite(q.tau)) q.tau = 0.f;
    if (!(q.inlier_thresh > 0.f) || !std::isfinite(q.inlier_thresh)) q.inlier_thresh = 1.f;
    int rc = check_params(c, n, &q);
    if (rc != TURBOREG_OK) return rc;
    TR_CHECK(cudaSetDevice(c->device));
    const size_t bytes = static_cast<size_t>(n) * 3 * sizeof(float);
    const float* s_in = src;
    const float* d_in = dst;
    if (!is_device_ptr(src)) {
        if (!host_finite(src, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s_in = c->ws.in_src;
    }
    if (!is_device_ptr(dst)) {
        if (!host_finite(dst, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst, bytes, cudaMemcpyHostToDevice, c->stream));
        d_in = c->ws.in_dst;
    }
    Plan pl;
    const int64_t off0 = 0;
    const turboreg_params* pq = &q;
    rc = build_plan(c, 1, &off0, &n, &pq, pl);
    if (rc != TURBOREG_OK) return rc;
    Batch bt;
    rc = upload_desc(c, 1, c->ws.desc, bt, c->stream);
    if (rc != TURBOREG_OK) return rc;
    const ProbView& v = c->ws.h_views[0];
    c->ctl_dirty = true;   // this entry point runs part of the path: no reset at its end
    TR_CHECK(cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl), c->stream));
    launch_pack(bt, pl.tot[ST_PACK], s_in, d_in, c->stream);
    if (k == 3) {
        // cliques (i, j, z, valid) in slots 0..m-1; slots up to k1*k2 are empty
        const int32_t slots = q.k1 * q.k2;
        std::vector<int32_t> cl(static_cast<size_t>(slots) * 4, 0);
        for (int32_t h = 0; h < m; ++h) {
            cl[4 * h + 0] = idx[3 * h + 0];
            cl[4 * h + 1] = idx[3 * h + 1];
            cl[4 * h + 2] = idx[3 * h + 2];
            cl[4 * h + 3] = 1;
        }
        TR_CHECK(cudaMemcpyAsync(v.cliques, cl.data(), cl.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 c->stream));
        TR_CHECK(cudaMemcpyAsync(&v.ctl->n_pivots, &q.k1, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        launch_kabsch(bt, pl.tot[ST_KABSCH], c->stream);
    } else {
        // the tuples go to the (otherwise unused here) clique buffer, as int32 [m][k]
        int32_t* didx = reinterpret_cast<int32_t*>(v.cliques);
        TR_CHECK(cudaMemcpyAsync(didx, idx, sizeof(int32_t) * m * k, cudaMemcpyHostToDevice, c->stream));
        launch_kabsch_n(v, didx, k, m, c->stream);
    }
    TR_CHECK(cudaGetLastError());
    std::vector<float> rt(static_cast<size_t>(m) * 16);
    TR_CHECK(cudaMemcpyAsync(rt.data(), v.rt, rt.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    Ctl hc;
    TR_CHECK(cudaMemcpyAsync(&hc, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    if (hc.err & TR_ERR_NONFINITE) return TURBOREG_ERR_NONFINITE;
    if (hc.err) return TURBOREG_ERR_TIMEOUT;
    for (int32_t h = 0; h < m; ++h) {
        int32_t flags;
        std::memcpy(&flags, &rt[static_cast<size_t>(h) * 16 + 13], sizeof(flags));
        out_valid[h] = (flags & 1) ? 1 : 0;
        std::memcpy(out_rt + static_cast<size_t>(h) * 12, &rt[static_cast<size_t>(h) * 16], 12 * sizeof(float));
    }
    return TURBOREG_OK;
}

int turboreg_features(turboreg_ctx* c, const float* src, const float* dst, int32_t n, const turboreg_params* p,
                      float* feat)
{
    if (!c || !src || !dst || !p || !feat) return TURBOREG_ERR_INVALID_ARG;
    turboreg_params q = *p;
    q.proposal = TURBOREG_PROPOSAL_PLAIN;
    q.flags &= ~(TURBOREG_FLAG_SC2_BITSET | TURBOREG_FLAG_STAGE_TIMES);
    q.flags |= TURBOREG_FLAG_SC2_GEMM;   // this entry point launches the GEMM directly
    int rc = check_params(c, n, &q);
    if (rc != TURBOREG_OK) return rc;
    TR_CHECK(cudaSetDevice(c->device));
    const size_t bytes = static_cast<size_t>(n) * 3 * sizeof(float);
    const float* s_in = src;
    const float* d_in = dst;
    if (!is_device_ptr(src)) {
        if (!host_finite(src, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src, bytes, cudaMemcpyHostToDevice, c->stream));
        s_in = c->ws.in_src;
    }
    if (!is_device_ptr(dst)) {
        if (!host_finite(dst, static_cast<size_t>(n) * 3)) return TURBOREG_ERR_NONFINITE;
        TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst, bytes, cudaMemcpyHostToDevice, c->stream));
        d_in = c->ws.in_dst;
    }
    Plan pl;
    const int64_t off0 = 0;
    const turboreg_params* pq = &q;
    rc = build_plan(c, 1, &off0, &n, &pq, pl);
    if (rc != TURBOREG_OK) return rc;
    Batch bt;
    rc = upload_desc(c, 1, c->ws.desc, bt, c->stream);
    if (rc != TURBOREG_OK) return rc;
    c->ctl_dirty = true;   // this entry point runs part of the path: no reset at its end
    TR_CHECK(cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl), c->stream));
    launch_pack(bt, pl.tot[ST_PACK], s_in, d_in, c->stream);
    launch_compat(bt, pl.tot[ST_COMPAT], c->stream);
    launch_sc2_tcgen05(bt, pl.tot[ST_GEMM], pl.max_n, 2, c->stream);
    launch_features(bt, c->stream);
    TR_CHECK(cudaGetLastError());
    TR_CHECK(cudaMemcpyAsync(feat, c->ws.feat, static_cast<size_t>(n) * 8 * sizeof(float), cudaMemcpyDefault,
                             c->stream));
    Ctl h;
    TR_CHECK(cudaMemcpyAsync(&h, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    if (h.err & TR_ERR_NONFINITE) return TURBOREG_ERR_NONFINITE;
    if (h.err) return TURBOREG_ERR_TIMEOUT;
    return TURBOREG_OK;
}

}  // extern "C"
