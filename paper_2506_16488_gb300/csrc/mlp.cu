// Learned stepping increment: a 12 -> 64 -> 64 -> 1 MLP with bf16 weights and
// fp32 accumulation, hand-written inference and training kernels.
//
// The paper chooses Delta of Delta*-stepping by doubling it until the running
// time stops improving (Sec. 6.1); Delta only reorders work (Theorems 3.3/3.4
// hold for any stepping schedule), so a prediction can never change an answer.
// The network predicts y = log2(Delta_best / Delta_default) from cheap per-group
// features; Delta = Delta_default * 2^y, clamped.
//
// Parameter vector (fp32 master copy, 5,081 floats):
//   mean[12] std[12] W1[64x12] b1[64] W2[64x64] b2[64] W3[64] b3[1]
// Inference and the training forward pass use W rounded to bf16 (round to
// nearest even); mean, std and biases stay fp32.  Sums run in fp32 in a fixed
// order (k ascending).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "graph_impl.h"
#include "mlp_internal.h"

namespace ppsp {

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One CTA of 64 threads per sample; thread j owns hidden unit j.
__device__ __forceinline__ float mlp_forward_sample(const float* P, const __nv_bfloat16* Wb, const float* feat,
                                                    float* s_x, float* s_h1, float* s_h2, float* s_red,
                                                    bool keep, float* z1_out, float* z2_out) {
    const int j = threadIdx.x;
    if (j < MLP_NF) s_x[j] = (feat[j] - P[MLP_OFF_MEAN + j]) / P[MLP_OFF_STD + j];
    __syncthreads();
    float z1 = P[MLP_OFF_B1 + j];
    for (int k = 0; k < MLP_NF; ++k) z1 += __bfloat162float(Wb[MLP_OFF_W1 + j * MLP_NF + k]) * s_x[k];
    s_h1[j] = z1 > 0.f ? z1 : 0.f;
    __syncthreads();
    float z2 = P[MLP_OFF_B2 + j];
    for (int k = 0; k < MLP_H; ++k) z2 += __bfloat162float(Wb[MLP_OFF_W2 + j * MLP_H + k]) * s_h1[k];
    const float h2 = z2 > 0.f ? z2 : 0.f;
    s_h2[j] = h2;
    __syncthreads();
    // y = b3 + sum_j W3[j] h2[j], summed in j order by thread 0
    float y = 0.f;
    if (j == 0) {
        y = P[MLP_OFF_B3];
        for (int k = 0; k < MLP_H; ++k) y += __bfloat162float(Wb[MLP_OFF_W3 + k]) * s_h2[k];
        s_red[0] = y;
    }
    if (keep) {
        *z1_out = z1;
        *z2_out = z2;
    }
    __syncthreads();
    return s_red[0];
}

// Refresh the bf16 copy of W1, W2, W3 from the fp32 masters.
__global__ void mlp_round_kernel(const float* P, __nv_bfloat16* Wb) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAMS; k += gridDim.x * blockDim.x) {
        const bool w = (k >= MLP_OFF_W1 && k < MLP_OFF_B1) || (k >= MLP_OFF_W2 && k < MLP_OFF_B2) ||
                       (k >= MLP_OFF_W3 && k < MLP_OFF_B3);
        Wb[k] = __float2bfloat16_rn(w ? P[k] : 0.f);
    }
}

// y[s] for every sample; with groups != null also writes each group's Delta.
__global__ void __launch_bounds__(MLP_H) mlp_infer_kernel(const float* P, const __nv_bfloat16* Wb,
                                                          const float* feats, u64 count, float* y_out,
                                                          GroupDev* groups, u64 delta_default, float ymin,
                                                          float ymax) {
    __shared__ float s_x[MLP_NF], s_h1[MLP_H], s_h2[MLP_H], s_red[1];
    for (u64 s = blockIdx.x; s < count; s += gridDim.x) {
        float z1, z2;
        const float y = mlp_forward_sample(P, Wb, feats + s * MLP_NF, s_x, s_h1, s_h2, s_red, false, &z1, &z2);
        if (threadIdx.x == 0) {
            if (y_out) y_out[s] = y;
            if (groups && groups[s].mode != GM_SSSP) {  // SSSP groups keep the default
                float yc = fminf(fmaxf(y, ymin), ymax);
                const double base = (double)delta_default;
                double dd = floor(base * exp2((double)yc) + 0.5);
                if (!(dd >= 1.0)) dd = 1.0;
                if (dd > 4.0e18) dd = 4.0e18;
                groups[s].delta = (u64)dd;
            }
        }
        __syncthreads();
    }
}

// Gradient of the mean squared error over all samples and the summed squared
// error.  Thread j owns hidden unit j and accumulates the gradient of its rows
// in registers over the CTA's samples; one atomicAdd per parameter per CTA at
// the end (the caller zeroes grad).
__global__ void __launch_bounds__(MLP_H) mlp_grad_kernel(const float* P, const __nv_bfloat16* Wb,
                                                         const float* feats, const float* labels, u64 count,
                                                         float* grad, float* sse) {
    __shared__ float s_x[MLP_NF], s_h1[MLP_H], s_h2[MLP_H], s_red[1], s_g2[MLP_H];
    const int j = threadIdx.x;
    const float inv_n = 1.0f / (float)count;
    float gW1[MLP_NF], gW2[MLP_H];
#pragma unroll
    for (int k = 0; k < MLP_NF; ++k) gW1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) gW2[k] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, e2 = 0.f;
    for (u64 s = blockIdx.x; s < count; s += gridDim.x) {
        float z1, z2;
        const float y = mlp_forward_sample(P, Wb, feats + s * MLP_NF, s_x, s_h1, s_h2, s_red, true, &z1, &z2);
        const float r = y - labels[s];
        const float gy = 2.0f * r * inv_n;
        e2 += r * r;
        gb3 += gy;
        gW3 += gy * s_h2[j];
        const float gz2 = (z2 > 0.f) ? gy * __bfloat162float(Wb[MLP_OFF_W3 + j]) : 0.f;
        s_g2[j] = gz2;
        gb2 += gz2;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) gW2[k] += gz2 * s_h1[k];
        __syncthreads();
        float gh1 = 0.f;
        for (int i = 0; i < MLP_H; ++i) gh1 += __bfloat162float(Wb[MLP_OFF_W2 + i * MLP_H + j]) * s_g2[i];
        const float gz1 = (z1 > 0.f) ? gh1 : 0.f;
        gb1 += gz1;
#pragma unroll
        for (int k = 0; k < MLP_NF; ++k) gW1[k] += gz1 * s_x[k];
        __syncthreads();
    }
    if (blockIdx.x < count) {
#pragma unroll
        for (int k = 0; k < MLP_NF; ++k) atomicAdd(grad + MLP_OFF_W1 + j * MLP_NF + k, gW1[k]);
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) atomicAdd(grad + MLP_OFF_W2 + j * MLP_H + k, gW2[k]);
        atomicAdd(grad + MLP_OFF_B1 + j, gb1);
        atomicAdd(grad + MLP_OFF_B2 + j, gb2);
        atomicAdd(grad + MLP_OFF_W3 + j, gW3);
        if (j == 0) {
            atomicAdd(grad + MLP_OFF_B3, gb3);
            atomicAdd(sse, e2);
        }
    }
}

// Adam on every trained parameter (mean and std are inputs, not trained).
__global__ void mlp_adam_kernel(float* P, float* m, float* v, const float* grad, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAMS; k += gridDim.x * blockDim.x) {
        if (k < MLP_OFF_W1) continue;
        const float g = grad[k];
        const float mk = b1 * m[k] + (1.f - b1) * g;
        const float vk = b2 * v[k] + (1.f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

ppsp_status mlp_launch_infer(const DeltaModel* m, const float* d_feats, u64 count, float* d_y, GroupDev* d_groups,
                             u64 delta_default, cudaStream_t stream) {
    if (count == 0) return PPSP_OK;
    const u32 blocks = (u32)std::min<u64>(count, 4096);
    mlp_infer_kernel<<<blocks, MLP_H, 0, stream>>>(m->d_P, m->d_Wb, d_feats, count, d_y, d_groups, delta_default,
                                                  MLP_YMIN, MLP_YMAX);
    PPSP_CUDA_TRY(cudaGetLastError());
    return PPSP_OK;
}

static ppsp_status ensure_scratch(DeltaModel* m, u64 count) {
    if (count <= m->cap) return PPSP_OK;
    cudaFree(m->d_feats);
    cudaFree(m->d_labels);
    cudaFree(m->d_y);
    m->d_feats = m->d_labels = m->d_y = nullptr;
    m->cap = 0;
    PPSP_CUDA_TRY(cudaMalloc(&m->d_feats, count * MLP_NF * 4));
    PPSP_CUDA_TRY(cudaMalloc(&m->d_labels, count * 4));
    PPSP_CUDA_TRY(cudaMalloc(&m->d_y, count * 4));
    m->cap = count;
    return PPSP_OK;
}

static ppsp_status grad_pass(DeltaModel* m, u64 count, float* sse_host) {
    PPSP_CUDA_TRY(cudaMemset(m->d_grad, 0, (MLP_NPARAMS + 1) * 4));
    const u32 blocks = (u32)std::min<u64>(count, 256);
    mlp_grad_kernel<<<blocks, MLP_H>>>(m->d_P, m->d_Wb, m->d_feats, m->d_labels, count, m->d_grad,
                                      m->d_grad + MLP_NPARAMS);
    PPSP_CUDA_TRY(cudaGetLastError());
    if (sse_host) PPSP_CUDA_TRY(cudaMemcpy(sse_host, m->d_grad + MLP_NPARAMS, 4, cudaMemcpyDeviceToHost));
    return PPSP_OK;
}

}  // namespace ppsp

using namespace ppsp;

ppsp_status ppsp_delta_model::upload() {
    PPSP_CUDA_TRY(cudaMemcpy(d_P, h_P.data(), MLP_NPARAMS * 4, cudaMemcpyHostToDevice));
    mlp_round_kernel<<<8, 256>>>(d_P, d_Wb);
    PPSP_CUDA_TRY(cudaGetLastError());
    return PPSP_OK;
}

extern "C" {

ppsp_status ppsp_delta_model_create(const float* params, ppsp_delta_model** out) {
    if (!params || !out) return PPSP_ERR_INVALID_ARG;
    *out = nullptr;
    for (int k = 0; k < MLP_NF; ++k)
        if (!(params[MLP_OFF_STD + k] > 0.f)) return PPSP_ERR_INVALID_ARG;
    auto m = new (std::nothrow) DeltaModel();
    if (!m) return PPSP_ERR_OOM;
    m->h_P.assign(params, params + MLP_NPARAMS);
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_P, MLP_NPARAMS * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_Wb, MLP_NPARAMS * 2)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_m, MLP_NPARAMS * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_v, MLP_NPARAMS * 4)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_grad, (MLP_NPARAMS + 1) * 4)) != cudaSuccess) {
        set_last_cuda_error(e, "cudaMalloc(model)", __FILE__, __LINE__);
        cudaGetLastError();
        delete m;
        return e == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
    }
    cudaMemset(m->d_m, 0, MLP_NPARAMS * 4);
    cudaMemset(m->d_v, 0, MLP_NPARAMS * 4);
    ppsp_status st = m->upload();
    if (st != PPSP_OK) {
        delete m;
        return st;
    }
    *out = m;
    return PPSP_OK;
}

void ppsp_delta_model_destroy(ppsp_delta_model* m) { delete m; }

ppsp_status ppsp_delta_model_get_params(const ppsp_delta_model* m, float* out) {
    if (!m || !out) return PPSP_ERR_INVALID_ARG;
    memcpy(out, m->h_P.data(), MLP_NPARAMS * 4);
    return PPSP_OK;
}

ppsp_status ppsp_delta_model_predict(ppsp_delta_model* m, const float* feats, uint64_t count, float* out) {
    if (!m || (count && (!feats || !out))) return PPSP_ERR_INVALID_ARG;
    if (count == 0) return PPSP_OK;
    ppsp_status st = ensure_scratch(m, count);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(m->d_feats, feats, count * MLP_NF * 4, cudaMemcpyHostToDevice));
    st = mlp_launch_infer(m, m->d_feats, count, m->d_y, nullptr, 1, 0);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(out, m->d_y, count * 4, cudaMemcpyDeviceToHost));
    return PPSP_OK;
}

ppsp_status ppsp_delta_model_grad(ppsp_delta_model* m, const float* feats, const float* labels, uint64_t count,
                                  float* grad_out, float* loss_out) {
    if (!m || !count || !feats || !labels || !grad_out) return PPSP_ERR_INVALID_ARG;
    ppsp_status st = ensure_scratch(m, count);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(m->d_feats, feats, count * MLP_NF * 4, cudaMemcpyHostToDevice));
    PPSP_CUDA_TRY(cudaMemcpy(m->d_labels, labels, count * 4, cudaMemcpyHostToDevice));
    float sse = 0.f;
    st = grad_pass(m, count, &sse);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(grad_out, m->d_grad, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost));
    if (loss_out) *loss_out = sse / (float)count;
    return PPSP_OK;
}

ppsp_status ppsp_delta_model_train(ppsp_delta_model* m, const float* feats, const float* labels, uint64_t count,
                                   uint32_t epochs, float lr, float* loss_out) {
    if (!m || !count || !feats || !labels || !(lr > 0.f)) return PPSP_ERR_INVALID_ARG;
    ppsp_status st = ensure_scratch(m, count);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(m->d_feats, feats, count * MLP_NF * 4, cudaMemcpyHostToDevice));
    PPSP_CUDA_TRY(cudaMemcpy(m->d_labels, labels, count * 4, cudaMemcpyHostToDevice));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float sse = 0.f;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        st = grad_pass(m, count, (ep + 1 == epochs) ? &sse : nullptr);
        if (st != PPSP_OK) return st;
        m->step += 1;
        const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
        mlp_adam_kernel<<<8, 256>>>(m->d_P, m->d_m, m->d_v, m->d_grad, lr, b1, b2, eps, c1, c2);
        mlp_round_kernel<<<8, 256>>>(m->d_P, m->d_Wb);
        PPSP_CUDA_TRY(cudaGetLastError());
    }
    PPSP_CUDA_TRY(cudaMemcpy(m->h_P.data(), m->d_P, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost));
    if (loss_out) *loss_out = sse / (float)count;  // loss before the last update
    return PPSP_OK;
}

ppsp_status ppsp_graph_set_delta_model(ppsp_graph* g, int32_t mode, ppsp_delta_model* m) {
    if (!g || mode < PPSP_BIDS || mode > PPSP_ASTAR) return PPSP_ERR_INVALID_ARG;
    g->delta_model[mode] = m;
    return PPSP_OK;
}

}  // extern "C"
