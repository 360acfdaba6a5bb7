// Learned stepping increment: model object and parameter layout.
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "ppsp_internal.h"

namespace ppsp {

constexpr int MLP_NF = 12;
constexpr int MLP_H = 64;
constexpr int MLP_OFF_MEAN = 0;
constexpr int MLP_OFF_STD = MLP_OFF_MEAN + MLP_NF;
constexpr int MLP_OFF_W1 = MLP_OFF_STD + MLP_NF;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_H * MLP_NF;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_H * MLP_H;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;
constexpr int MLP_NPARAMS = MLP_OFF_B3 + 1;  // 5081
constexpr float MLP_YMIN = -8.0f;             // Delta >= Delta_default / 256
constexpr float MLP_YMAX = 6.0f;              // Delta <= Delta_default * 64

}  // namespace ppsp

struct ppsp_delta_model {
    std::vector<float> h_P;          // fp32 master parameters (host copy)
    float* d_P = nullptr;            // fp32 master parameters
    __nv_bfloat16* d_Wb = nullptr;   // bf16 copy used by every forward pass
    float* d_m = nullptr;            // Adam moments
    float* d_v = nullptr;
    float* d_grad = nullptr;         // gradient + 1 float of summed squared error
    float* d_feats = nullptr;        // scratch for predict / train
    float* d_labels = nullptr;
    float* d_y = nullptr;
    uint64_t cap = 0;
    uint64_t step = 0;
    ppsp_status upload();
    ~ppsp_delta_model() {
        cudaFree(d_P);
        cudaFree(d_Wb);
        cudaFree(d_m);
        cudaFree(d_v);
        cudaFree(d_grad);
        cudaFree(d_feats);
        cudaFree(d_labels);
        cudaFree(d_y);
        cudaGetLastError();
    }
};

namespace ppsp {
typedef ppsp_delta_model DeltaModel;

// groups[s].delta = clamp(delta_default * 2^y(s)) for s < count (stream-ordered).
ppsp_status mlp_launch_infer(const DeltaModel* m, const float* d_feats, u64 count, float* d_y,
                             GroupDev* d_groups, u64 delta_default, cudaStream_t stream);
}  // namespace ppsp
