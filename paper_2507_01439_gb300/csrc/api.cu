// Host runtime and C ABI of the GB300 TurboReg library (see include/turboreg.h).
//
// A context owns one device workspace sized for max_n at creation; register
// calls only enqueue kernels on the context's stream, copy the 88-byte result
// back and synchronise.  No host round trip happens between stages: pivot
// counts, thresholds and validity stay on the device (Ctl block).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "tr_common.cuh"
#include "tr_problem.h"
#include "turboreg.h"
#include "turboreg_internal.h"

using namespace tr;

namespace {

constexpr int kNumStages = 8;
const char* kStageNames[kNumStages] = {"pack", "compat", "sc2", "topk", "pgs", "kabsch", "verify", "finalize"};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline int32_t round_up(int32_t a, int32_t b) { return (a + b - 1) / b * b; }

struct Workspace {
    int32_t n_pad_max = 0;
    float* pts = nullptr;
    float* pts8 = nullptr;
    int32_t* fp64_list = nullptr;
    uint8_t* a8 = nullptr;
    uint32_t* bits = nullptr;
    uint16_t* w = nullptr;
    int32_t* rowscore = nullptr;
    int32_t* deg = nullptr;
    uint32_t* hist = nullptr;
    int32_t* rowcnt = nullptr;
    int32_t* rowpref = nullptr;
    int32_t* rowcnt_gt = nullptr;
    int32_t* rowpref_gt = nullptr;
    uint64_t* cand = nullptr;
    int4* piv = nullptr;
    int4* cliques = nullptr;
    float* rt = nullptr;
    int32_t* inl = nullptr;
    Ctl* ctl = nullptr;
    turboreg_result* res = nullptr;   // [max_batch]
    float* in_src = nullptr;          // staging for host inputs [max_n*max_batch*3]
    float* in_dst = nullptr;
};

}  // namespace

struct turboreg_ctx {
    int device = 0;
    int32_t max_n = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;               // FP64 Kabsch + its verification run here,
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;  // concurrently with the main verification
    Workspace ws;
    turboreg_result* host_res = nullptr;   // pinned [max_batch]
    EncodeTiledFn encode = nullptr;
    CUtensorMap tmA, tmB;
    int32_t tm_npad = 0;
    cudaEvent_t ev[kNumStages + 1] = {};
    float stage_ms[kNumStages] = {};
    int32_t last_n = 0, last_npad = 0, last_k1 = 0, last_k2 = 0;
    bool have_times = false;
    // captured per-problem pipelines, replayed with cudaGraphLaunch; only the
    // pack node's input pointers change between calls
    struct GraphSlot {
        bool used = false;
        int32_t n = 0, k1 = 0, k2 = 0;
        float tau = 0.f, theta = 0.f, kappa = 0.f;
        uint32_t flags = 0;
        turboreg_result* res = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t pack_node = nullptr;
        cudaKernelNodeParams pack_params = {};
        tr::ProbView pv = {};
        const float* src = nullptr;
        const float* dst = nullptr;
        void* args[3] = {};
        uint64_t stamp = 0;
    };
    static constexpr int kGraphSlots = 8;
    GraphSlot gslot[kGraphSlots];
    uint64_t gclock = 0;
};

namespace {

#define TR_CHECK(expr)                                      \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) {                            \
            std::fprintf(stderr, "turboreg: %s failed: %s\n", #expr, cudaGetErrorString(e_)); \
            return TURBOREG_ERR_CUDA;                       \
        }                                                   \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 256);
}

void free_ws(Workspace& ws)
{
    void* ptrs[] = {ws.pts, ws.pts8, ws.fp64_list, ws.a8, ws.bits, ws.w, ws.rowscore, ws.deg, ws.hist, ws.rowcnt, ws.rowpref, ws.rowcnt_gt, ws.rowpref_gt,
                    ws.cand, ws.piv, ws.cliques, ws.rt, ws.inl, ws.ctl, ws.res, ws.in_src, ws.in_dst};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ws = Workspace();
}

int alloc_ws(Workspace& ws, int32_t max_n, int32_t max_batch)
{
    const int32_t np = round_up(max_n, kSc2BN);
    const size_t n2 = static_cast<size_t>(np) * np;
    const size_t nh = static_cast<size_t>(TURBOREG_K1_MAX) * TURBOREG_K2_MAX;
    const size_t tot = static_cast<size_t>(max_n) * max_batch;
    ws.n_pad_max = np;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&ws.pts, 6 * static_cast<size_t>(np));
    if (e == cudaSuccess) e = dalloc(&ws.pts8, 8 * static_cast<size_t>(np));
    if (e == cudaSuccess) e = dalloc(&ws.fp64_list, nh);
    if (e == cudaSuccess) e = dalloc(&ws.a8, n2);
    if (e == cudaSuccess) e = dalloc(&ws.bits, n2 / 32);
    if (e == cudaSuccess) e = dalloc(&ws.w, n2);
    if (e == cudaSuccess) e = dalloc(&ws.rowscore, np);
    if (e == cudaSuccess) e = dalloc(&ws.deg, np);
    if (e == cudaSuccess) e = dalloc(&ws.hist, np + 1);
    if (e == cudaSuccess) e = dalloc(&ws.rowcnt, np);
    if (e == cudaSuccess) e = dalloc(&ws.rowpref, np);
    if (e == cudaSuccess) e = dalloc(&ws.rowcnt_gt, np);
    if (e == cudaSuccess) e = dalloc(&ws.rowpref_gt, np);
    if (e == cudaSuccess) e = dalloc(&ws.cand, TURBOREG_K1_MAX);
    if (e == cudaSuccess) e = dalloc(&ws.piv, TURBOREG_K1_MAX);
    if (e == cudaSuccess) e = dalloc(&ws.cliques, nh);
    if (e == cudaSuccess) e = dalloc(&ws.rt, nh * 16);
    if (e == cudaSuccess) e = dalloc(&ws.inl, nh);
    if (e == cudaSuccess) e = dalloc(&ws.ctl, 1);
    if (e == cudaSuccess) e = dalloc(&ws.res, max_batch);
    if (e == cudaSuccess) e = dalloc(&ws.in_src, tot * 3);
    if (e == cudaSuccess) e = dalloc(&ws.in_dst, tot * 3);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_ws(ws);
        return e == cudaErrorMemoryAllocation ? TURBOREG_ERR_OOM : TURBOREG_ERR_CUDA;
    }
    // zero the FP8 adjacency and W once so padding is defined even before the first call
    if (cudaMemset(ws.a8, 0, n2) != cudaSuccess || cudaMemset(ws.w, 0, n2 * 2) != cudaSuccess) {
        free_ws(ws);
        return TURBOREG_ERR_CUDA;
    }
    return TURBOREG_OK;
}

int encode_maps(turboreg_ctx* c, int32_t n_pad)
{
    if (c->tm_npad == n_pad) return TURBOREG_OK;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(n_pad), static_cast<cuuint64_t>(n_pad)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(n_pad)};   // bytes between rows
    const cuuint32_t boxA[2] = {static_cast<cuuint32_t>(kSc2BK), static_cast<cuuint32_t>(kSc2BM)};
    const cuuint32_t boxB[2] = {static_cast<cuuint32_t>(kSc2BK), static_cast<cuuint32_t>(kSc2BN)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r1 = c->encode(&c->tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, c->ws.a8, dims, strides, boxA, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = c->encode(&c->tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, c->ws.a8, dims, strides, boxB, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
        std::fprintf(stderr, "turboreg: cuTensorMapEncodeTiled failed (%d, %d)\n", (int)r1, (int)r2);
        c->tm_npad = 0;
        return TURBOREG_ERR_CUDA;
    }
    c->tm_npad = n_pad;
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
    if (p->graph_mode != TURBOREG_GRAPH_O2) return TURBOREG_ERR_INVALID_ARG;
    if (p->proposal != TURBOREG_PROPOSAL_PLAIN) return TURBOREG_ERR_INVALID_ARG;
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

bool host_finite(const float* p, size_t cnt)
{
    for (size_t k = 0; k < cnt; ++k)
        if (!std::isfinite(p[k])) return false;
    return true;
}

ProbView make_view(turboreg_ctx* c, int32_t n, const turboreg_params* p, turboreg_result* res_dev)
{
    Workspace& ws = c->ws;
    ProbView v;
    v.n = n;
    v.n_pad = round_up(n, kSc2BN);
    v.ldb = v.n_pad / 32;
    v.k1 = p->k1;
    v.k2 = p->k2;
    v.tau = p->tau;
    v.theta = p->inlier_thresh;
    v.kappa_fp64 = p->kappa_fp64 > 0.f ? p->kappa_fp64 : 100.f;
    v.pts = ws.pts;
    v.pts8 = ws.pts8;
    v.fp64_list = ws.fp64_list;
    v.a8 = ws.a8;
    v.bits = ws.bits;
    v.w = ws.w;
    v.rowscore = ws.rowscore;
    v.deg = ws.deg;
    v.hist = ws.hist;
    v.rowcnt = ws.rowcnt;
    v.rowpref = ws.rowpref;
    v.rowcnt_gt = ws.rowcnt_gt;
    v.rowpref_gt = ws.rowpref_gt;
    v.cand = ws.cand;
    v.piv = ws.piv;
    v.cliques = ws.cliques;
    v.rt = ws.rt;
    v.inl = ws.inl;
    v.ctl = ws.ctl;
    v.res = res_dev;
    return v;
}

// Enqueue the whole path for one problem whose points are already on the device.
int enqueue_problem(turboreg_ctx* c, const float* dsrc, const float* ddst, int32_t n, const turboreg_params* p,
                    turboreg_result* res_dev)
{
    ProbView v = make_view(c, n, p, res_dev);
    const bool timed = (p->flags & TURBOREG_FLAG_STAGE_TIMES) != 0;
    const bool bitset = (p->flags & TURBOREG_FLAG_SC2_BITSET) != 0;
    if (!bitset) {
        int rc = encode_maps(c, v.n_pad);
        if (rc != TURBOREG_OK) return rc;
    }
    cudaStream_t s = c->stream;
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal));
    TR_CHECK(cudaMemsetAsync(c->ws.ctl, 0, sizeof(Ctl), s));
    launch_pack(v, dsrc, ddst, s);
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal));
    launch_compat(v, s);
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal));
    if (bitset) launch_sc2_bitset(v, s);
    else launch_sc2_tcgen05(v, c->tmA, c->tmB, s);   // also builds the weight histogram
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal));
    if (bitset) launch_topk(v, s);
    else launch_topk_after_select(v, s);   // the GEMM's last CTA chose alpha
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[4], s, cudaEventRecordExternal));
    launch_pgs(v, s);
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[5], s, cudaEventRecordExternal));
    launch_kabsch(v, s);
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[6], s, cudaEventRecordExternal));
    // fork: ill-conditioned cliques (FP64 list) on the side stream, the rest here
    TR_CHECK(cudaEventRecord(c->fork_ev, s));
    TR_CHECK(cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    launch_kabsch_fp64_verify(v, c->side);
    TR_CHECK(cudaEventRecord(c->join_ev, c->side));
    launch_verify(v, s);
    TR_CHECK(cudaStreamWaitEvent(s, c->join_ev, 0));
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[7], s, cudaEventRecordExternal));
    launch_finalize(v, s);
    if (timed) TR_CHECK(cudaEventRecordWithFlags(c->ev[8], s, cudaEventRecordExternal));
    TR_CHECK(cudaGetLastError());
    c->last_n = n;
    c->last_npad = v.n_pad;
    c->last_k1 = p->k1;
    c->last_k2 = p->k2;
    c->have_times = timed;
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

void drop_slot(turboreg_ctx::GraphSlot& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = turboreg_ctx::GraphSlot();
}

bool slot_matches(const turboreg_ctx::GraphSlot& g, int32_t n, const turboreg_params* p, turboreg_result* res)
{
    return g.used && g.n == n && g.k1 == p->k1 && g.k2 == p->k2 && g.tau == p->tau && g.theta == p->inlier_thresh &&
           g.kappa == p->kappa_fp64 && g.flags == p->flags && g.res == res;
}

// Capture the pipeline for this shape once, then replay it; the pack node's
// (src, dst) arguments are patched in the instantiated graph on every call.
int run_problem(turboreg_ctx* c, const float* dsrc, const float* ddst, int32_t n, const turboreg_params* p,
                turboreg_result* res_dev)
{
    if (p->flags & TURBOREG_FLAG_NO_GRAPH) return enqueue_problem(c, dsrc, ddst, n, p, res_dev);
    turboreg_ctx::GraphSlot* g = nullptr;
    for (auto& sl : c->gslot)
        if (slot_matches(sl, n, p, res_dev)) g = &sl;
    if (!g) {
        g = &c->gslot[0];
        for (auto& sl : c->gslot) {
            if (!sl.used) { g = &sl; break; }
            if (sl.stamp < g->stamp) g = &sl;
        }
        drop_slot(*g);
        TR_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_problem(c, dsrc, ddst, n, p, res_dev);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (rc != TURBOREG_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            std::fprintf(stderr, "turboreg: graph capture failed: %s\n", cudaGetErrorString(e));
            return rc != TURBOREG_OK ? rc : TURBOREG_ERR_CUDA;
        }
        size_t cnt = 0;
        TR_CHECK(cudaGraphGetNodes(graph, nullptr, &cnt));
        cudaGraphNode_t nodes[64];
        if (cnt > 64) {
            cudaGraphDestroy(graph);
            return TURBOREG_ERR_CUDA;
        }
        TR_CHECK(cudaGraphGetNodes(graph, nodes, &cnt));
        for (size_t k = 0; k < cnt; ++k) {
            cudaGraphNodeType ty;
            TR_CHECK(cudaGraphNodeGetType(nodes[k], &ty));
            if (ty != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            TR_CHECK(cudaGraphKernelNodeGetParams(nodes[k], &kp));
            if (kp.func == pack_kernel_func()) {
                g->pack_node = nodes[k];
                g->pack_params = kp;
            }
        }
        if (!g->pack_node) {
            cudaGraphDestroy(graph);
            return TURBOREG_ERR_CUDA;
        }
        g->graph = graph;
        if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
            cudaGetLastError();
            drop_slot(*g);
            return TURBOREG_ERR_CUDA;
        }
        g->used = true;
        g->n = n; g->k1 = p->k1; g->k2 = p->k2;
        g->tau = p->tau; g->theta = p->inlier_thresh; g->kappa = p->kappa_fp64;
        g->flags = p->flags;
        g->res = res_dev;
        g->pv = make_view(c, n, p, res_dev);
    }
    g->stamp = ++c->gclock;
    g->src = dsrc;
    g->dst = ddst;
    g->args[0] = &g->pv;
    g->args[1] = &g->src;
    g->args[2] = &g->dst;
    cudaKernelNodeParams kp = g->pack_params;
    kp.kernelParams = g->args;
    kp.extra = nullptr;
    TR_CHECK(cudaGraphExecKernelNodeSetParams(g->exec, g->pack_node, &kp));
    TR_CHECK(cudaGraphLaunch(g->exec, c->stream));
    c->last_n = n;
    c->last_npad = g->pv.n_pad;
    c->last_k1 = p->k1;
    c->last_k2 = p->k2;
    c->have_times = (p->flags & TURBOREG_FLAG_STAGE_TIMES) != 0;
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
    turboreg_ctx* c = new (std::nothrow) turboreg_ctx();
    if (!c) return TURBOREG_ERR_OOM;
    c->device = device;
    c->max_n = max_n;
    c->max_batch = max_batch;
    int rc = alloc_ws(c->ws, max_n, max_batch);
    if (rc != TURBOREG_OK) {
        delete c;
        return rc;
    }
    if (cudaMallocHost(reinterpret_cast<void**>(&c->host_res), sizeof(turboreg_result) * max_batch) != cudaSuccess) {
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
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
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
    if (se == cudaSuccess) se = topk_setup();
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
    if (c->side) cudaStreamSynchronize(c->side);
    for (auto& sl : c->gslot) drop_slot(sl);
    for (int k = 0; k <= kNumStages; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    free_ws(c->ws);
    if (c->host_res) cudaFreeHost(c->host_res);
    delete c;
}

int turboreg_register(turboreg_ctx* c, const float* src, const float* dst, int32_t n, const turboreg_params* p,
                      turboreg_result* out)
{
    if (!c || !src || !dst || !out) return TURBOREG_ERR_INVALID_ARG;
    int rc = check_params(c, n, p);
    if (rc != TURBOREG_OK) {
        std::memset(out, 0, sizeof(*out));
        out->R[0] = out->R[4] = out->R[8] = 1.f;
        out->hypothesis = -1;
        out->clique[0] = out->clique[1] = out->clique[2] = -1;
        out->status = rc;
        return rc;
    }
    TR_CHECK(cudaSetDevice(c->device));
    const bool dsrc = is_device_ptr(src), ddst = is_device_ptr(dst);
    const float* s_in = src;
    const float* d_in = dst;
    const size_t bytes = static_cast<size_t>(n) * 3 * sizeof(float);
    if (!dsrc) {
        if (!host_finite(src, static_cast<size_t>(n) * 3)) rc = TURBOREG_ERR_NONFINITE;
        else {
            TR_CHECK(cudaMemcpyAsync(c->ws.in_src, src, bytes, cudaMemcpyHostToDevice, c->stream));
            s_in = c->ws.in_src;
        }
    }
    if (!ddst && rc == TURBOREG_OK) {
        if (!host_finite(dst, static_cast<size_t>(n) * 3)) rc = TURBOREG_ERR_NONFINITE;
        else {
            TR_CHECK(cudaMemcpyAsync(c->ws.in_dst, dst, bytes, cudaMemcpyHostToDevice, c->stream));
            d_in = c->ws.in_dst;
        }
    }
    if (rc != TURBOREG_OK) {
        TR_CHECK(cudaStreamSynchronize(c->stream));
        std::memset(out, 0, sizeof(*out));
        out->R[0] = out->R[4] = out->R[8] = 1.f;
        out->hypothesis = -1;
        out->clique[0] = out->clique[1] = out->clique[2] = -1;
        out->status = rc;
        return rc;
    }
    rc = run_problem(c, s_in, d_in, n, p, c->ws.res);
    if (rc != TURBOREG_OK) return rc;
    TR_CHECK(cudaMemcpyAsync(c->host_res, c->ws.res, sizeof(turboreg_result), cudaMemcpyDeviceToHost, c->stream));
    TR_CHECK(cudaStreamSynchronize(c->stream));
    rc = collect_times(c);
    if (rc != TURBOREG_OK) return rc;
    *out = c->host_res[0];
    return out->status;
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
    int32_t* pre = static_cast<int32_t*>(std::calloc(num, sizeof(int32_t)));
    if (!pre) return TURBOREG_ERR_OOM;
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
        rc = enqueue_problem(c, s_in + 3 * offsets[b], d_in + 3 * offsets[b], n, p, c->ws.res + b);
        if (rc != TURBOREG_OK) {
            std::free(pre);
            return rc;
        }
    }
    cudaError_t e = cudaMemcpyAsync(c->host_res, c->ws.res, sizeof(turboreg_result) * num, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        std::free(pre);
        std::fprintf(stderr, "turboreg: batched copy-back failed: %s\n", cudaGetErrorString(e));
        return TURBOREG_ERR_CUDA;
    }
    for (int32_t b = 0; b < num; ++b) {
        if (pre[b] != TURBOREG_OK) {
            std::memset(&out[b], 0, sizeof(out[b]));
            out[b].R[0] = out[b].R[4] = out[b].R[8] = 1.f;
            out[b].hypothesis = -1;
            out[b].clique[0] = out[b].clique[1] = out[b].clique[2] = -1;
            out[b].status = pre[b];
        } else {
            out[b] = c->host_res[b];
        }
    }
    std::free(pre);
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
    Ctl h;
    if (cudaMemcpy(&h, c->ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return -TURBOREG_ERR_CUDA;
    const size_t np = static_cast<size_t>(c->last_npad);
    const size_t nh = static_cast<size_t>(h.n_pivots) * c->last_k2;
    const void* src = nullptr;
    size_t bytes = 0;
    switch (which) {
        case TURBOREG_BUF_ADJ_BITS: src = c->ws.bits; bytes = np * np / 8; break;
        case TURBOREG_BUF_ADJ_FP8: src = c->ws.a8; bytes = np * np; break;
        case TURBOREG_BUF_SC2: src = c->ws.w; bytes = np * np * 2; break;
        case TURBOREG_BUF_PIVOTS: src = c->ws.piv; bytes = static_cast<size_t>(h.n_pivots) * 16; break;
        case TURBOREG_BUF_CLIQUES: src = c->ws.cliques; bytes = nh * 16; break;
        case TURBOREG_BUF_RT: src = c->ws.rt; bytes = nh * 64; break;
        case TURBOREG_BUF_INLIERS: src = c->ws.inl; bytes = nh * 4; break;
        case TURBOREG_BUF_ROWSCORE: src = c->ws.rowscore; bytes = static_cast<size_t>(c->last_n) * 4; break;
        case TURBOREG_BUF_DEGREE: src = c->ws.deg; bytes = static_cast<size_t>(c->last_n) * 4; break;
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

}  // extern "C"
