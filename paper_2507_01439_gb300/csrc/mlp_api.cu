// C ABI of the proposal-MLP trainer (include/turboreg_internal.h): FP32
// master weights, Adam moments and activation scratch on the device; the
// forward, backward and update run in the kernels of mlp.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "tr_common.cuh"
#include "tr_mlp.h"
#include "turboreg_internal.h"

using namespace tr;

struct turboreg_mlp {
    int device = 0;
    int32_t max_samples = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t step = 0;
    float* w = nullptr;      // FP32 master [P]
    float* wbf = nullptr;    // BF16-rounded copy used by the forward [P]
    float* mom = nullptr;    // Adam first moment [P]
    float* vel = nullptr;    // Adam second moment [P]
    float* grad = nullptr;   // [P]
    float* loss = nullptr;   // [1]
    uint32_t* err = nullptr;
    float* z4 = nullptr;     // [max_samples]
    __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
};

namespace {

#define TM_CHECK(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            std::fprintf(stderr, "turboreg mlp: %s failed: %s\n", #expr, cudaGetErrorString(e_)); \
            return TURBOREG_ERR_CUDA;                                                            \
        }                                                                                        \
    } while (0)

void free_all(turboreg_mlp* t)
{
    void* ptrs[] = {t->w, t->wbf, t->mom, t->vel, t->grad, t->loss, t->err, t->z4, t->h1, t->h2, t->h3};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// Backward pass of the last forward: grad (device) = d(mean BCE)/d params.
int backward(turboreg_mlp* t, const float* feat, const float* label, int32_t m)
{
    TM_CHECK(cudaMemsetAsync(t->grad, 0, sizeof(float) * kMlpParams, t->stream));
    TM_CHECK(cudaMemsetAsync(t->loss, 0, sizeof(float), t->stream));
    launch_mlp_forward(feat, m, t->wbf, nullptr, t->z4, t->h1, t->h2, t->h3, t->err, t->stream);
    launch_mlp_backward(feat, label, m, t->wbf, t->z4, t->h1, t->h2, t->h3, t->grad, t->loss, t->err, t->stream);
    TM_CHECK(cudaGetLastError());
    return TURBOREG_OK;
}

}  // namespace

extern "C" {

int turboreg_mlp_create(int device, int32_t max_samples, uint64_t seed, void* cuda_stream, turboreg_mlp** out)
{
    if (!out || max_samples < 1) return TURBOREG_ERR_INVALID_ARG;
    *out = nullptr;
    TM_CHECK(cudaSetDevice(device));
    turboreg_mlp* t = new (std::nothrow) turboreg_mlp();
    if (!t) return TURBOREG_ERR_OOM;
    t->device = device;
    t->max_samples = max_samples;
    const size_t M = static_cast<size_t>(max_samples);
    cudaError_t e = cudaSuccess;
    auto al = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = cudaMalloc(p, b);
    };
    al(reinterpret_cast<void**>(&t->w), sizeof(float) * kMlpParams);
    al(reinterpret_cast<void**>(&t->wbf), sizeof(float) * kMlpParams);
    al(reinterpret_cast<void**>(&t->mom), sizeof(float) * kMlpParams);
    al(reinterpret_cast<void**>(&t->vel), sizeof(float) * kMlpParams);
    al(reinterpret_cast<void**>(&t->grad), sizeof(float) * kMlpParams);
    al(reinterpret_cast<void**>(&t->loss), sizeof(float));
    al(reinterpret_cast<void**>(&t->err), sizeof(uint32_t));
    al(reinterpret_cast<void**>(&t->z4), sizeof(float) * M);
    al(reinterpret_cast<void**>(&t->h1), sizeof(__nv_bfloat16) * M * 64);
    al(reinterpret_cast<void**>(&t->h2), sizeof(__nv_bfloat16) * M * 128);
    al(reinterpret_cast<void**>(&t->h3), sizeof(__nv_bfloat16) * M * 64);
    if (e == cudaSuccess) e = mlp_setup();
    if (e == cudaSuccess) {
        if (cuda_stream) t->stream = static_cast<cudaStream_t>(cuda_stream);
        else {
            e = cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking);
            t->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_all(t);
        delete t;
        return e == cudaErrorMemoryAllocation ? TURBOREG_ERR_OOM : TURBOREG_ERR_CUDA;
    }
    // He-normal initialisation (std = sqrt(2 / fan_in)), zero biases
    std::vector<float> w(kMlpParams, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int out_dim, int in_dim) {
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / static_cast<float>(in_dim)));
        for (int k = 0; k < out_dim * in_dim; ++k) w[off + k] = nd(rng);
    };
    fill(kW1, 64, 8);
    fill(kW2, 128, 64);
    fill(kW3, 64, 128);
    fill(kW4, 1, 64);
    int rc = turboreg_mlp_set_params(t, w.data());
    if (rc == TURBOREG_OK) {
        std::vector<float> z(kMlpParams, 0.f);
        rc = turboreg_mlp_set_state(t, z.data(), z.data(), 0);
    }
    if (rc != TURBOREG_OK) {
        turboreg_mlp_destroy(t);
        return rc;
    }
    *out = t;
    return TURBOREG_OK;
}

void turboreg_mlp_destroy(turboreg_mlp* t)
{
    if (!t) return;
    cudaSetDevice(t->device);
    if (t->stream) cudaStreamSynchronize(t->stream);
    free_all(t);
    if (t->own_stream && t->stream) cudaStreamDestroy(t->stream);
    delete t;
}

int turboreg_mlp_get_params(turboreg_mlp* t, float* params)
{
    if (!t || !params) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemcpyAsync(params, t->w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaStreamSynchronize(t->stream));
    return TURBOREG_OK;
}

int turboreg_mlp_set_params(turboreg_mlp* t, const float* params)
{
    if (!t || !params) return TURBOREG_ERR_INVALID_ARG;
    for (int k = 0; k < kMlpParams; ++k)
        if (!std::isfinite(params[k])) return TURBOREG_ERR_NONFINITE;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemcpyAsync(t->w, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, t->stream));
    launch_mlp_round(t->w, t->wbf, t->stream);
    TM_CHECK(cudaGetLastError());
    TM_CHECK(cudaStreamSynchronize(t->stream));
    return TURBOREG_OK;
}

int turboreg_mlp_get_state(turboreg_mlp* t, float* m, float* v, int32_t* step)
{
    if (!t || !m || !v || !step) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemcpyAsync(m, t->mom, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaMemcpyAsync(v, t->vel, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaStreamSynchronize(t->stream));
    *step = t->step;
    return TURBOREG_OK;
}

int turboreg_mlp_set_state(turboreg_mlp* t, const float* m, const float* v, int32_t step)
{
    if (!t || !m || !v || step < 0) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemcpyAsync(t->mom, m, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, t->stream));
    TM_CHECK(cudaMemcpyAsync(t->vel, v, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, t->stream));
    TM_CHECK(cudaStreamSynchronize(t->stream));
    t->step = step;
    return TURBOREG_OK;
}

int turboreg_mlp_forward(turboreg_mlp* t, const float* feat, int32_t m, float* prob)
{
    if (!t || !feat || !prob || m < 1) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemsetAsync(t->err, 0, sizeof(uint32_t), t->stream));
    launch_mlp_forward(feat, m, t->wbf, prob, nullptr, nullptr, nullptr, nullptr, t->err, t->stream);
    TM_CHECK(cudaGetLastError());
    uint32_t err = 0;
    TM_CHECK(cudaMemcpyAsync(&err, t->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaStreamSynchronize(t->stream));
    return err ? TURBOREG_ERR_TIMEOUT : TURBOREG_OK;
}

int turboreg_mlp_grad(turboreg_mlp* t, const float* feat, const float* label, int32_t m, float* grad, float* loss)
{
    if (!t || !feat || !label || !grad || m < 1 || m > t->max_samples) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    TM_CHECK(cudaMemsetAsync(t->err, 0, sizeof(uint32_t), t->stream));
    const int rc = backward(t, feat, label, m);
    if (rc != TURBOREG_OK) return rc;
    TM_CHECK(cudaMemcpyAsync(grad, t->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, t->stream));
    float l = 0.f;
    uint32_t err = 0;
    TM_CHECK(cudaMemcpyAsync(&l, t->loss, sizeof(float), cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaMemcpyAsync(&err, t->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, t->stream));
    TM_CHECK(cudaStreamSynchronize(t->stream));
    if (loss) *loss = l;
    return err ? TURBOREG_ERR_TIMEOUT : TURBOREG_OK;
}

int turboreg_mlp_train_step(turboreg_mlp* t, const float* feat, const float* label, int32_t m, float lr,
                            float* loss)
{
    if (!t || !feat || !label || m < 1 || m > t->max_samples || !(lr > 0.f)) return TURBOREG_ERR_INVALID_ARG;
    TM_CHECK(cudaSetDevice(t->device));
    int rc = backward(t, feat, label, m);
    if (rc != TURBOREG_OK) return rc;
    t->step += 1;
    launch_mlp_adam(t->w, t->mom, t->vel, t->grad, t->wbf, t->step, lr, t->stream);
    TM_CHECK(cudaGetLastError());
    if (loss) {
        TM_CHECK(cudaMemcpyAsync(loss, t->loss, sizeof(float), cudaMemcpyDeviceToHost, t->stream));
        TM_CHECK(cudaStreamSynchronize(t->stream));
    }
    return TURBOREG_OK;
}

}  // extern "C"
