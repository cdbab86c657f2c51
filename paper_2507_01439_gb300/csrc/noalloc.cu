// Pivot selection without any device allocation.
//
// Some callers cannot call cudaMalloc: a plugin that runs inside a host
// framework which owns all device memory through its own pool (a stray
// cudaMalloc breaks its accounting or fails outright), or a real-time loop
// that forbids allocation after start-up because cudaMalloc may synchronise
// the device and take unbounded time.  turboreg_select_pivots_noalloc gives
// them the pivot-selection stage with every scratch buffer it needs placed in
// one fixed array in the library's own device memory (kScratchBytes, about
// 225 KB, loaded with the module and held by every GPU that loads the library
// until the process exits).  The caller passes the weight matrix and the output buffers;
// nothing is allocated or freed, by this code or by any library it calls.
//
// The scratch is shared by every call: the histogram and the control block
// (which holds the active-row and slot counters) are cleared with
// cudaMemsetAsync at the start of each call, and two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it.  Serialise calls per device.
//
// In host code the name g_pivot_scratch only stands in for the array; its
// device address comes from cudaGetSymbolAddress, taken with the device
// current on the first call made on that device.  That first call should
// therefore be made before any stream capture begins.  Every later call made
// outside a stream capture looks the address up again and, if it changed (the
// device was reset, or the host framework tore the context down and made a
// new one), repeats the set-up, since the kernels' shared-memory attributes
// went with the old context; a call made while its stream is being captured
// uses the address recorded last, so the context must not be replaced between
// the last uncaptured call and the end of a capture.
//
// A weight above n - 2 (no SC^2 count is larger) in the caller's matrix is
// not counted: the call then selects nothing and writes -TURBOREG_ERR_INVALID_ARG
// to *n_pivots_dev.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "tr_common.cuh"
#include "tr_problem.h"
#include "turboreg_internal.h"

namespace tr {

namespace {

constexpr int32_t kMaxN = TURBOREG_NOALLOC_MAX_N;
constexpr int32_t kMaxK1 = TURBOREG_K1_MAX;

// layout of the scratch array (each part 256-byte aligned)
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffHist = align256(sizeof(Ctl));
constexpr size_t kOffActive = kOffHist + align256(sizeof(uint32_t) * (kMaxN + 1));
constexpr size_t kOffCand = kOffActive + align256(sizeof(int4) * kMaxN);
constexpr size_t kScratchBytes = kOffCand + align256(sizeof(uint64_t) * kMaxK1);

static __device__ __align__(256) uint8_t g_pivot_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_dev_scratch[kMaxDevices] = {};
bool g_dev_ready[kMaxDevices] = {};

// Device address of the scratch array on `device` (current); set up on first
// use, and again when a call outside stream capture finds the address changed.
int scratch_for(int device, cudaStream_t s, uint8_t** out)
{
    if (device < 0 || device >= kMaxDevices) return TURBOREG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    bool recheck = !g_dev_ready[device];
    if (!recheck) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
            cudaGetLastError();   // e.g. the legacy stream while another stream captures: keep the record
            cs = cudaStreamCaptureStatusActive;
        }
        recheck = cs == cudaStreamCaptureStatusNone;
    }
    if (recheck) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pivot_scratch);
        if (e != cudaSuccess || p == nullptr) {
            std::fprintf(stderr, "turboreg: cudaGetSymbolAddress of the pivot scratch failed: %s\n",
                         cudaGetErrorString(e));
            return TURBOREG_ERR_CUDA;
        }
        if (g_dev_ready[device] && g_dev_scratch[device] == static_cast<uint8_t*>(p)) {
            *out = g_dev_scratch[device];
            return TURBOREG_OK;
        }
        e = topk_setup();
        if (e != cudaSuccess) {
            std::fprintf(stderr, "turboreg: pivot-selection set-up failed: %s\n", cudaGetErrorString(e));
            return TURBOREG_ERR_CUDA;
        }
        g_dev_scratch[device] = static_cast<uint8_t*>(p);
        g_dev_ready[device] = true;
    }
    *out = g_dev_scratch[device];
    return TURBOREG_OK;
}

}  // namespace

}  // namespace tr

extern "C" int turboreg_select_pivots_noalloc(const uint16_t* w_dev, int32_t n, int32_t ldw, int32_t k1,
                                              int32_t* pivots_dev, int32_t* n_pivots_dev, void* cuda_stream)
{
    using namespace tr;
    if (!w_dev || !pivots_dev || !n_pivots_dev) return TURBOREG_ERR_INVALID_ARG;
    if (n < 1 || k1 < 1) return TURBOREG_ERR_INVALID_ARG;
    if (n > kMaxN || k1 > kMaxK1) {
        std::fprintf(stderr,
                     "turboreg_select_pivots_noalloc: n = %d or k1 = %d exceeds the fixed scratch limits "
                     "(n <= %d, k1 <= %d)\n", n, k1, kMaxN, kMaxK1);
        return TURBOREG_ERR_INVALID_ARG;
    }
    // rows are read with 16-byte loads of 8 weights: ldw covers n rounded up to 8
    if (ldw < ((n + 7) / 8) * 8 || ldw % 8 != 0 || (reinterpret_cast<uintptr_t>(w_dev) & 15u) != 0)
        return TURBOREG_ERR_INVALID_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return TURBOREG_ERR_CUDA;
    uint8_t* scr = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = scratch_for(device, s, &scr);
    if (rc != TURBOREG_OK) return rc;

    ProbView v = {};
    v.n = n;
    v.n_pad = ldw;
    v.k1 = k1;
    v.w = const_cast<uint16_t*>(w_dev);
    v.ctl = reinterpret_cast<Ctl*>(scr + kOffCtl);
    v.hist = reinterpret_cast<uint32_t*>(scr + kOffHist);
    v.active = reinterpret_cast<int4*>(scr + kOffActive);
    v.cand = reinterpret_cast<uint64_t*>(scr + kOffCand);
    v.piv = reinterpret_cast<int4*>(pivots_dev);

    // the previous call's contents stay in the array: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(scr + kOffCtl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.hist, 0, sizeof(uint32_t) * (n + 1), s);
    if (e != cudaSuccess) return TURBOREG_ERR_CUDA;
    launch_topk_single(v, s);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n_pivots_dev, &v.ctl->n_pivots, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "turboreg_select_pivots_noalloc: %s\n", cudaGetErrorString(e));
        return TURBOREG_ERR_CUDA;
    }
    return TURBOREG_OK;
}
