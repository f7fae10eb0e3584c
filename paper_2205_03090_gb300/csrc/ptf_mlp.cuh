// ptf_mlp.cuh -- the two networks of the learned form (Sec. 4): BF16
// weights and activations, FP32 accumulation, SiLU hidden layers.
//
// Inputs u = bf16((v - mean) * rstd), v = (z_1..z_nc, P, T) (the scaling
// layer, Sec. 4.1.1).  Two architectures:
//  - arch 0: three hidden layers a_l = bf16(silu(W_l a_{l-1} + b_l)) and a
//    linear output (the classifier of Sec. 4.1.1 has 3 x 32 units; widths 64
//    and 128 are the larger variants used elsewhere);
//  - arch 1 (the initializer of Sec. 4.2.1): h_0 = bf16(silu(W_0 u + b_0)),
//    three residual blocks h_k = bf16(h_{k-1} + silu(W_{2k} silu(W_{2k-1}
//    h_{k-1} + b) + b)) (every activation bf16), and a linear output on the
//    concatenation [u; h_3] (the wide shortcut).
// Layers: arch 0 has 4 (din->H, H->H, H->H, H->dout); arch 1 has 8
// (din->H, six H->H, din+H->dout).
//
// Parameter storage:
//  - theta: FP32 master vector, W_0, b_0, W_1, b_1, ... (each W row-major
//    [out, in]);
//  - wt: BF16 compute copy of the weights, each layer transposed [in][out]
//    and padded to a multiple of 8 outputs, so one 16-byte load fetches 8
//    consecutive outputs of one input.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace ptf {

constexpr int kMlpMaxIn = 18;  // nc + 2 with nc <= 16

struct MLP {
    int din, hid, dout;
    const float* theta;          // FP32 master (natural layout)
    const __nv_bfloat16* wt;     // BF16 transposed, padded
    const float* mean;           // [din] feature means
    const float* rstd;           // [din] 1 / feature standard deviations
    int arch = 0;                // 0: three hidden layers; 1: residual blocks + wide output
};

__host__ __device__ inline int pad8(int x) { return (x + 7) & ~7; }
__host__ __device__ inline int n_layers(const MLP& a) { return a.arch ? 8 : 4; }
__host__ __device__ inline int layer_in(const MLP& a, int l) {
    return l == 0 ? a.din : (a.arch && l == 7 ? a.din + a.hid : a.hid);
}
__host__ __device__ inline int layer_out(const MLP& a, int l) { return l == n_layers(a) - 1 ? a.dout : a.hid; }
// offsets of W_l and b_l in theta
__host__ __device__ inline int64_t theta_W(const MLP& a, int l) {
    int64_t o = 0;
    for (int k = 0; k < l; k++) o += (int64_t)layer_out(a, k) * layer_in(a, k) + layer_out(a, k);
    return o;
}
__host__ __device__ inline int64_t theta_b(const MLP& a, int l) {
    return theta_W(a, l) + (int64_t)layer_out(a, l) * layer_in(a, l);
}
__host__ __device__ inline int64_t theta_size(const MLP& a) { return theta_W(a, n_layers(a)); }
// offset of layer l in wt ([in][pad8(out)])
__host__ __device__ inline int64_t wt_off(const MLP& a, int l) {
    int64_t o = 0;
    for (int k = 0; k < l; k++) o += (int64_t)layer_in(a, k) * pad8(layer_out(a, k));
    return o;
}
__host__ __device__ inline int64_t wt_size(const MLP& a) { return wt_off(a, n_layers(a)); }

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigmoidf_(float x) { return 1.0f / (1.0f + __expf(-x)); }

// Load 8 consecutive BF16 weights (16 bytes) as floats.
__device__ __forceinline__ void ld8(const __nv_bfloat16* p, float* w) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float2 f = __bfloat1622float2(h[j]);
        w[2 * j] = f.x;
        w[2 * j + 1] = f.y;
    }
}

// One linear layer for one sample: pre[o] = b[o] + sum_k W[o][k] in[k];
// in / out are this sample's columns (element stride `st`).  If HIDDEN, the
// output column gets bf16(silu(pre)) and dsl (optional) gets silu'(pre);
// otherwise the raw pre-activation.
template <bool HIDDEN>
__device__ __forceinline__ void layer_sample(const MLP& a, int l, const float* in, int64_t in_st, float* out,
                                             int64_t out_st, float* dsl, int64_t dsl_st) {
    const int nin = layer_in(a, l), nout = layer_out(a, l), po = pad8(nout);
    const __nv_bfloat16* W = a.wt + wt_off(a, l);
    const float* bias = a.theta + theta_b(a, l);
    for (int o0 = 0; o0 < nout; o0 += 8) {
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] = (o0 + j < nout) ? __ldg(bias + o0 + j) : 0.0f;
        for (int k = 0; k < nin; k++) {
            const float x = in[k * in_st];
            float w[8];
            ld8(W + (int64_t)k * po + o0, w);
#pragma unroll
            for (int j = 0; j < 8; j++) acc[j] = fmaf(w[j], x, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (o0 + j >= nout) break;
            if (HIDDEN) {
                const float s = sigmoidf_(acc[j]);
                out[(o0 + j) * out_st] = bf16_round(acc[j] * s);
                if (dsl) dsl[(o0 + j) * dsl_st] = s * (1.0f + acc[j] * (1.0f - s));
            } else {
                out[(o0 + j) * out_st] = acc[j];
            }
        }
    }
}

// Standardised, bf16-rounded features of one mixture into `u` (stride st).
__device__ __forceinline__ void features(const MLP& a, int nc, int64_t ld, const double* P, const double* T,
                                         const double* z, int64_t m, float* u, int64_t st) {
    for (int i = 0; i < a.din; i++) {
        const double v = i < nc ? z[i * ld + m] : (i == nc ? P[m] : T[m]);
        u[i * st] = bf16_round(((float)v - __ldg(a.mean + i)) * __ldg(a.rstd + i));
    }
}

// Forward pass of one sample, activations in a column of stride st with
// rows [u (din)][h (hid)][t1 (hid)][t2 (hid)]; u filled by the caller (arch 1
// reads [u; h] as the output layer's input).  Output to out (stride out_st).
__device__ __forceinline__ void forward_sample(const MLP& a, float* col, int64_t st, float* out, int64_t out_st) {
    float* u = col;
    float* h = col + a.din * st;
    float* t1 = h + a.hid * st;
    float* t2 = t1 + a.hid * st;
    if (a.arch == 0) {
        layer_sample<true>(a, 0, u, st, h, st, nullptr, 0);
        layer_sample<true>(a, 1, h, st, t1, st, nullptr, 0);
        layer_sample<true>(a, 2, t1, st, h, st, nullptr, 0);
        layer_sample<false>(a, 3, h, st, out, out_st, nullptr, 0);
        return;
    }
    layer_sample<true>(a, 0, u, st, h, st, nullptr, 0);
    for (int k = 1; k <= 3; k++) {
        layer_sample<true>(a, 2 * k - 1, h, st, t1, st, nullptr, 0);
        layer_sample<true>(a, 2 * k, t1, st, t2, st, nullptr, 0);
        for (int j = 0; j < a.hid; j++) h[j * st] = bf16_round(h[j * st] + t2[j * st]);
    }
    layer_sample<false>(a, 7, u, st, out, out_st, nullptr, 0);
}

// Network inference over n mixtures (defined in ptf_nn.cu): out[o * out_ld + m].
cudaError_t nn_infer_launch(const MLP& a, int nc, int64_t n, int64_t ld, const double* P, const double* T,
                            const double* z, float* out, int64_t out_ld, int sms, cudaStream_t s);

}  // namespace ptf
