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

// Refresh the bf16 copy of W1, W2, W3 from the fp32 masters.
__global__ void mlp_round_kernel(const float* P, __nv_bfloat16* Wb) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_NPARAMS; k += gridDim.x * blockDim.x) {
        const bool w = (k >= MLP_OFF_W1 && k < MLP_OFF_B1) || (k >= MLP_OFF_W2 && k < MLP_OFF_B2) ||
                       (k >= MLP_OFF_W3 && k < MLP_OFF_B3);
        Wb[k] = __float2bfloat16_rn(w ? P[k] : 0.f);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core inference: one warp evaluates 16 samples with warp-level
// mma.sync m16n8k16 (bf16 operands, fp32 accumulation).  The weights are bf16
// by definition; an fp32 activation a is split into three bf16 terms
// a = hi + mid + lo (8 significant bits each, so the split holds a's 24-bit
// significand up to a last-place rounding), and every layer sums the three
// products with W, each exact in fp32: the result is fp32 arithmetic in
// another summation order.  The accumulator layout of one m16n8 tile is the
// operand layout of the next layer's k-chunk, so activations stay in
// registers between layers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 pack_bf2(float lo_k, float hi_k) {
    // two bf16 values, the lower k index in the low half
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
    return *reinterpret_cast<const u32*>(&v);
}

// a = hi + mid + lo in bf16
__device__ __forceinline__ void split3(float a, float& hi, float& mid, float& lo) {
    hi = __bfloat162float(__float2bfloat16_rn(a));
    const float r1 = a - hi;  // exact
    mid = __bfloat162float(__float2bfloat16_rn(r1));
    lo = r1 - mid;            // exact; rounded to bf16 when packed
}

__device__ __forceinline__ void mma_bf16(float c[4], const u32 a[4], const u32 b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B operand of the k-chunk kc and n-tile nt for z[n] = sum_k W[n][k] x[k]
// (W row-major [rows][kdim], rows beyond `rows` or k beyond kdim are 0):
// this thread holds W[n][k], W[n][k+1] and W[n][k+8], W[n][k+9] with
// n = 8 nt + lane / 4 and k = 16 kc + 2 (lane % 4).
__device__ __forceinline__ void load_b(const __nv_bfloat16* W, int rows, int kdim, int kc, int nt, u32 b[2]) {
    const int lane = threadIdx.x & 31, n = 8 * nt + (lane >> 2), k = 16 * kc + 2 * (lane & 3);
    const unsigned short* w = reinterpret_cast<const unsigned short*>(W);
    u32 r[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kk = k + 8 * h;
        const u32 x0 = (n < rows && kk < kdim) ? w[n * kdim + kk] : 0u;
        const u32 x1 = (n < rows && kk + 1 < kdim) ? w[n * kdim + kk + 1] : 0u;
        r[h] = x0 | (x1 << 16);
    }
    b[0] = r[0];
    b[1] = r[1];
}

// acc[nt][.] += A(16 x 16 chunk, three bf16 terms in a3[t][.]) * B(chunk kc, tile nt)
template <int NT>
__device__ __forceinline__ void mma_chunk3(float acc[][4], const u32 a3[3][4], const __nv_bfloat16* W, int rows,
                                           int kdim, int kc) {
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        u32 b[2];
        load_b(W, rows, kdim, kc, nt, b);
#pragma unroll
        for (int t = 0; t < 3; ++t) mma_bf16(acc[nt], a3[t], b);
    }
}

// The A operand of one 16-wide k-chunk from fp32 values v[r][c] held in the
// accumulator layout (rows g and g + 8, columns 2 (lane % 4) and + 1 of two
// adjacent n-tiles), split into three bf16 terms.
__device__ __forceinline__ void a_from_acc(const float t0[4], const float t1[4], u32 a3[3][4]) {
    float h[8], m[8], l[8];
    const float v[8] = {t0[0], t0[1], t0[2], t0[3], t1[0], t1[1], t1[2], t1[3]};
#pragma unroll
    for (int q = 0; q < 8; ++q) split3(v[q], h[q], m[q], l[q]);
    // a0,a1: (g, 2t..) = t0[0..1]; a2,a3: (g+8, 2t..) = t0[2..3];
    // a4,a5: (g, 8+2t..) = t1[0..1]; a6,a7: (g+8, 8+2t..) = t1[2..3]
    const float* parts[3] = {h, m, l};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        a3[t][0] = pack_bf2(parts[t][0], parts[t][1]);
        a3[t][1] = pack_bf2(parts[t][2], parts[t][3]);
        a3[t][2] = pack_bf2(parts[t][4], parts[t][5]);
        a3[t][3] = pack_bf2(parts[t][6], parts[t][7]);
    }
}

// y[s] for every sample, 16 samples per warp on the tensor cores; with
// groups != null also writes each group's Delta.
__global__ void __launch_bounds__(128) mlp_infer_mma_kernel(const float* P, const __nv_bfloat16* Wb,
                                                            const float* feats, u64 count, float* y_out,
                                                            GroupDev* groups, u64 delta_default, float ymin,
                                                            float ymax) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const u64 warps = (u64)gridDim.x * (blockDim.x >> 5);
    for (u64 tile = (u64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < count; tile += warps) {
        const u64 s0 = tile * 16;
        // layer 1 operand: standardised features x[s][k], k < 12 (k 12..15
        // zero), in the operand layout (see a_from_acc)
        u32 a3[3][4];
        {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int row = g + ((q >> 1) & 1) * 8, k = 2 * tq + (q & 1) + ((q >> 2) & 1) * 8;
                const u64 s = s0 + row;
                float xv = 0.f;
                if (s < count && k < MLP_NF) xv = (feats[s * MLP_NF + k] - P[MLP_OFF_MEAN + k]) / P[MLP_OFF_STD + k];
                v[q] = xv;
            }
            const float t0[4] = {v[0], v[1], v[2], v[3]}, t1[4] = {v[4], v[5], v[6], v[7]};
            a_from_acc(t0, t1, a3);
        }
        // z1 = W1 x + b1, 8 n-tiles of 8 hidden units
        float z1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float b0 = P[MLP_OFF_B1 + 8 * nt + 2 * tq], b1 = P[MLP_OFF_B1 + 8 * nt + 2 * tq + 1];
            z1[nt][0] = b0;
            z1[nt][1] = b1;
            z1[nt][2] = b0;
            z1[nt][3] = b1;
        }
        mma_chunk3<8>(z1, a3, Wb + MLP_OFF_W1, MLP_H, MLP_NF, 0);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) z1[nt][q] = z1[nt][q] > 0.f ? z1[nt][q] : 0.f;
        // z2 = W2 h1 + b2: k-chunk kc takes hidden units 16 kc .. 16 kc + 15,
        // i.e. the n-tiles 2 kc and 2 kc + 1 of layer 1
        float z2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float b0 = P[MLP_OFF_B2 + 8 * nt + 2 * tq], b1 = P[MLP_OFF_B2 + 8 * nt + 2 * tq + 1];
            z2[nt][0] = b0;
            z2[nt][1] = b1;
            z2[nt][2] = b0;
            z2[nt][3] = b1;
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            a_from_acc(z1[2 * kc], z1[2 * kc + 1], a3);
            mma_chunk3<8>(z2, a3, Wb + MLP_OFF_W2, MLP_H, MLP_H, kc);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) z2[nt][q] = z2[nt][q] > 0.f ? z2[nt][q] : 0.f;
        // y = W3 h2 + b3: one output row (the other seven columns of the tile are 0)
        float y3[1][4] = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            a_from_acc(z2[2 * kc], z2[2 * kc + 1], a3);
            mma_chunk3<1>(y3, a3, Wb + MLP_OFF_W3, 1, MLP_H, kc);
        }
        // column 0 of the output tile: lanes with lane % 4 == 0 hold rows g
        // (y3[0][0]) and g + 8 (y3[0][2])
        if (tq == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const u64 s = s0 + g + 8 * h;
                if (s >= count) continue;
                const float y = y3[0][2 * h] + P[MLP_OFF_B3];
                if (y_out) y_out[s] = y;
                if (groups && groups[s].mode != GM_SSSP) {  // SSSP groups keep the default
                    const float yc = fminf(fmaxf(y, ymin), ymax);
                    const double base = (double)delta_default;
                    double dd = floor(base * exp2((double)yc) + 0.5);
                    if (!(dd >= 1.0)) dd = 1.0;
                    if (dd > 4.0e18) dd = 4.0e18;
                    groups[s].delta = (u64)dd;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core gradient: one warp takes 16 samples at a time, runs the forward
// pass as in inference, then the backward pass as four small GEMMs:
//   gW3 = gy^T h2, gz2 = (z2 > 0) gy W3, gW2 = gz2^T h1 (K = the 16 samples),
//   gh1 = gz2 W2, gz1 = (z1 > 0) gh1, gW1 = gz1^T x.
// Products of two fp32 quantities split both operands into three bf16 terms
// and sum the six partial products of order at most 2^-16 (the dropped ones
// are below 2^-24 of the product); products with a weight use the exact bf16
// weight.  Per-tile sums go to the gradient with atomicAdd (the caller zeroes
// it).
// ---------------------------------------------------------------------------
// the three-term A operand of the 16 x 16 tile A[m][k] = S[k][m0 + m] (S: 16
// rows of stride ld in shared memory, read transposed)
__device__ __forceinline__ void a_frag_T3(const float* S, int ld, int m0, u32 a[3][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ks[8] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9, 2 * t + 8, 2 * t + 9};
    const int ms[8] = {g, g, g + 8, g + 8, g, g, g + 8, g + 8};
    float p[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split3(S[ks[q] * ld + m0 + ms[q]], p[0][q], p[1][q], p[2][q]);
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int r = 0; r < 4; ++r) a[u][r] = pack_bf2(p[u][2 * r], p[u][2 * r + 1]);
}

// the three-term B operand of the 16 x 8 tile B[k][n] = S[k][n0 + n], columns
// at or beyond ncols read as 0
__device__ __forceinline__ void b_frag3(const float* S, int ld, int n0, int ncols, u32 b[3][2]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const bool ok = n0 + g < ncols;
    const int ks[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
    float p[3][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split3(ok ? S[ks[q] * ld + n0 + g] : 0.f, p[0][q], p[1][q], p[2][q]);
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        b[u][0] = pack_bf2(p[u][0], p[u][1]);
        b[u][1] = pack_bf2(p[u][2], p[u][3]);
    }
}

// c += A B for three-term operands: the six partial products hi.hi, hi.mid,
// mid.hi, hi.lo, lo.hi, mid.mid
__device__ __forceinline__ void mma_split6(float c[4], const u32 a[3][4], const u32 b[3][2]) {
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v + u < 3; ++v) mma_bf16(c, a[u], b[v]);
}

// B operand of z[n] = sum_k W[k][n] x[k] (W row-major [kdim][ncols], read
// down its columns): W[k][n], W[k+1][n] and W[k+8][n], W[k+9][n] with
// n = 8 nt + lane / 4 and k = 16 kc + 2 (lane % 4)
__device__ __forceinline__ void load_bT(const __nv_bfloat16* W, int ncols, int kc, int nt, u32 b[2]) {
    const int lane = threadIdx.x & 31, n = 8 * nt + (lane >> 2), k = 16 * kc + 2 * (lane & 3);
    const unsigned short* w = reinterpret_cast<const unsigned short*>(W);
    b[0] = (u32)w[k * ncols + n] | ((u32)w[(k + 1) * ncols + n] << 16);
    b[1] = (u32)w[(k + 8) * ncols + n] | ((u32)w[(k + 9) * ncols + n] << 16);
}

constexpr int MLP_GW = 4;            // warps per CTA of the gradient kernel
constexpr int MLP_SLD = MLP_H + 1;   // shared-memory row stride (floats)

__global__ void __launch_bounds__(32 * MLP_GW) mlp_grad_mma_kernel(const float* P, const __nv_bfloat16* Wb,
                                                                   const float* feats, const float* labels,
                                                                   u64 count, float* grad, float* sse) {
    __shared__ float s_a[MLP_GW][16 * MLP_SLD];  // gz2, then gz1 (rows = samples)
    __shared__ float s_b[MLP_GW][16 * MLP_SLD];  // h1, then x
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3, w = threadIdx.x >> 5;
    float* SA = s_a[w];
    float* SB = s_b[w];
    const float inv_n = 1.0f / (float)count;
    const u64 warps = (u64)gridDim.x * MLP_GW;
    float acc_b1[8][2] = {}, acc_b2[8][2] = {}, acc_w3[8][2] = {};  // per-thread partial sums over rows
    float acc_b3 = 0.f, acc_e2 = 0.f;
    for (u64 tile = (u64)blockIdx.x * MLP_GW + w; tile * 16 < count; tile += warps) {
        const u64 s0 = tile * 16;
        // ---- forward (as the inference kernel), keeping z1, z2 and x ----
        float xv[8];
        u32 a3[3][4];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int row = g + ((q >> 1) & 1) * 8, k = 2 * tq + (q & 1) + ((q >> 2) & 1) * 8;
            const u64 s = s0 + row;
            xv[q] = (s < count && k < MLP_NF) ? (feats[s * MLP_NF + k] - P[MLP_OFF_MEAN + k]) / P[MLP_OFF_STD + k]
                                              : 0.f;
        }
        {
            const float t0[4] = {xv[0], xv[1], xv[2], xv[3]}, t1[4] = {xv[4], xv[5], xv[6], xv[7]};
            a_from_acc(t0, t1, a3);
        }
        float z1[8][4], z2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float b0 = P[MLP_OFF_B1 + 8 * nt + 2 * tq], b1 = P[MLP_OFF_B1 + 8 * nt + 2 * tq + 1];
            z1[nt][0] = b0;
            z1[nt][1] = b1;
            z1[nt][2] = b0;
            z1[nt][3] = b1;
            const float c0 = P[MLP_OFF_B2 + 8 * nt + 2 * tq], c1 = P[MLP_OFF_B2 + 8 * nt + 2 * tq + 1];
            z2[nt][0] = c0;
            z2[nt][1] = c1;
            z2[nt][2] = c0;
            z2[nt][3] = c1;
        }
        mma_chunk3<8>(z1, a3, Wb + MLP_OFF_W1, MLP_H, MLP_NF, 0);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            float h0[4], h1t[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h0[q] = fmaxf(z1[2 * kc][q], 0.f);
                h1t[q] = fmaxf(z1[2 * kc + 1][q], 0.f);
            }
            a_from_acc(h0, h1t, a3);
            mma_chunk3<8>(z2, a3, Wb + MLP_OFF_W2, MLP_H, MLP_H, kc);
        }
        float y3[1][4] = {{0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            float h0[4], h1t[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h0[q] = fmaxf(z2[2 * kc][q], 0.f);
                h1t[q] = fmaxf(z2[2 * kc + 1][q], 0.f);
            }
            a_from_acc(h0, h1t, a3);
            mma_chunk3<1>(y3, a3, Wb + MLP_OFF_W3, 1, MLP_H, kc);
        }
        // ---- output error: rows g and g + 8, y held by the quad's lane 0 ----
        float gy[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float yv = __shfl_sync(0xffffffffu, y3[0][2 * h], lane & ~3) + P[MLP_OFF_B3];
            const u64 s = s0 + g + 8 * h;
            const float r = (s < count) ? yv - labels[s] : 0.f;
            gy[h] = 2.0f * r * inv_n;
            if (tq == 0) {
                acc_e2 += r * r;
                acc_b3 += gy[h];
            }
        }
        // ---- gW3, gb2, gz2 (accumulator layout) ----
        float gz2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 8 * nt + 2 * tq + (q & 1);
                const float gyr = gy[q >> 1];
                const float h2 = fmaxf(z2[nt][q], 0.f);
                acc_w3[nt][q & 1] += gyr * h2;
                const float v = (z2[nt][q] > 0.f) ? gyr * __bfloat162float(Wb[MLP_OFF_W3 + j]) : 0.f;
                gz2[nt][q] = v;
                acc_b2[nt][q & 1] += v;
            }
        // stage gz2 and h1 (rows = samples) for gW2 = gz2^T h1
        __syncwarp();
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q >> 1), col = 8 * nt + 2 * tq + (q & 1);
                SA[row * MLP_SLD + col] = gz2[nt][q];
                SB[row * MLP_SLD + col] = fmaxf(z1[nt][q], 0.f);
            }
        __syncwarp();
#pragma unroll 1
        for (int mt = 0; mt < 4; ++mt) {
            u32 at[3][4];
            a_frag_T3(SA, MLP_SLD, 16 * mt, at);
#pragma unroll 1
            for (int nt = 0; nt < 8; ++nt) {
                u32 bt[3][2];
                b_frag3(SB, MLP_SLD, 8 * nt, MLP_H, bt);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_split6(c, at, bt);
                const int j = 16 * mt + g, k = 8 * nt + 2 * tq;
                atomicAdd(grad + MLP_OFF_W2 + j * MLP_H + k, c[0]);
                atomicAdd(grad + MLP_OFF_W2 + j * MLP_H + k + 1, c[1]);
                atomicAdd(grad + MLP_OFF_W2 + (j + 8) * MLP_H + k, c[2]);
                atomicAdd(grad + MLP_OFF_W2 + (j + 8) * MLP_H + k + 1, c[3]);
            }
        }
        // ---- gh1 = gz2 W2, gz1, gb1 ----
        float gh1[8][4] = {};
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            a_from_acc(gz2[2 * kc], gz2[2 * kc + 1], a3);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                u32 b[2];
                load_bT(Wb + MLP_OFF_W2, MLP_H, kc, nt, b);
#pragma unroll
                for (int u = 0; u < 3; ++u) mma_bf16(gh1[nt], a3[u], b);
            }
        }
        __syncwarp();
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q >> 1), col = 8 * nt + 2 * tq + (q & 1);
                const float v = (z1[nt][q] > 0.f) ? gh1[nt][q] : 0.f;
                acc_b1[nt][q & 1] += v;
                SA[row * MLP_SLD + col] = v;  // gz1
            }
        // x (rows = samples, 12 columns) for gW1 = gz1^T x
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int row = g + ((q >> 1) & 1) * 8, k = 2 * tq + (q & 1) + ((q >> 2) & 1) * 8;
            SB[row * MLP_SLD + k] = xv[q];
        }
        __syncwarp();
#pragma unroll 1
        for (int mt = 0; mt < 4; ++mt) {
            u32 at[3][4];
            a_frag_T3(SA, MLP_SLD, 16 * mt, at);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                u32 bt[3][2];
                b_frag3(SB, MLP_SLD, 8 * nt, MLP_NF, bt);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_split6(c, at, bt);
                const int j = 16 * mt + g, k = 8 * nt + 2 * tq;
                if (k < MLP_NF) {
                    atomicAdd(grad + MLP_OFF_W1 + j * MLP_NF + k, c[0]);
                    atomicAdd(grad + MLP_OFF_W1 + (j + 8) * MLP_NF + k, c[2]);
                }
                if (k + 1 < MLP_NF) {
                    atomicAdd(grad + MLP_OFF_W1 + j * MLP_NF + k + 1, c[1]);
                    atomicAdd(grad + MLP_OFF_W1 + (j + 8) * MLP_NF + k + 1, c[3]);
                }
            }
        }
        __syncwarp();
    }
    // per-column sums over the warp's rows: lanes with the same lane % 4 hold
    // the same columns
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float b1v = acc_b1[nt][c], b2v = acc_b2[nt][c], w3v = acc_w3[nt][c];
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                b1v += __shfl_xor_sync(0xffffffffu, b1v, o);
                b2v += __shfl_xor_sync(0xffffffffu, b2v, o);
                w3v += __shfl_xor_sync(0xffffffffu, w3v, o);
            }
            if (g == 0) {
                const int j = 8 * nt + 2 * tq + c;
                atomicAdd(grad + MLP_OFF_B1 + j, b1v);
                atomicAdd(grad + MLP_OFF_B2 + j, b2v);
                atomicAdd(grad + MLP_OFF_W3 + j, w3v);
            }
        }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        acc_b3 += __shfl_xor_sync(0xffffffffu, acc_b3, o);
        acc_e2 += __shfl_xor_sync(0xffffffffu, acc_e2, o);
    }
    if (lane == 0) {
        atomicAdd(grad + MLP_OFF_B3, acc_b3);
        atomicAdd(sse, acc_e2);
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
    // four warps of 16 samples per CTA on the tensor cores
    const u32 blocks = (u32)std::min<u64>((count + 63) / 64, 4096);
    mlp_infer_mma_kernel<<<blocks, 128, 0, stream>>>(m->d_P, m->d_Wb, d_feats, count, d_y, d_groups, delta_default,
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
    const u32 blocks = (u32)std::min<u64>((count + 16 * MLP_GW - 1) / (16 * MLP_GW), 1024);
    mlp_grad_mma_kernel<<<blocks, 32 * MLP_GW>>>(m->d_P, m->d_Wb, m->d_feats, m->d_labels, count, m->d_grad,
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
