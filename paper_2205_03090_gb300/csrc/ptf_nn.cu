// ptf_nn.cu -- the learned form (Sec. 4): network inference, features,
// training (forward, backward, Adam) and the C ABI of the networks.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ptflash.h"
#include "ptf_ctx.cuh"

using namespace ptf;

namespace {

thread_local char g_err[256] = "";
int fail(cudaError_t e) {
    std::snprintf(g_err, sizeof(g_err), "%s", cudaGetErrorString(e));
    cudaGetLastError();
    return PTF_ERR_CUDA;
}
#define NN_CUDA(call)                            \
    do {                                         \
        cudaError_t _e = (call);                 \
        if (_e != cudaSuccess) return fail(_e);  \
    } while (0)

constexpr int kTile = 128;  // samples per block (one per thread)

size_t infer_smem(const MLP& a) { return (size_t)(kMlpMaxIn + 2 * a.hid) * kTile * sizeof(float); }

// Inference: each thread runs its sample through the network, keeping the
// activations in its own shared-memory column (no cross-thread traffic).
__global__ void __launch_bounds__(kTile) k_nn_infer(MLP a, int nc, int64_t n, int64_t ld, const double* P,
                                                    const double* T, const double* z, float* out, int64_t out_ld) {
    extern __shared__ float sm[];
    const int s = threadIdx.x;
    float* u = sm + s;
    float* h0 = sm + kMlpMaxIn * kTile + s;
    float* h1 = h0 + a.hid * kTile;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int64_t m = base + s;
        if (m >= n) continue;
        features(a, nc, ld, P, T, z, m, u, kTile);
        layer_sample<true>(a, 0, u, kTile, h0, kTile, nullptr, 0);
        layer_sample<true>(a, 1, h0, kTile, h1, kTile, nullptr, 0);
        layer_sample<true>(a, 2, h1, kTile, h0, kTile, nullptr, 0);
        layer_sample<false>(a, 3, h0, kTile, out + m, out_ld, nullptr, 0);
    }
}

// Standardised bf16 features X[i][m] (row stride n).
__global__ void k_nn_features(MLP a, int nc, int64_t n, int64_t ld, const double* P, const double* T,
                              const double* z, float* X) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
        features(a, nc, ld, P, T, z, m, X + m, n);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

size_t train_block_floats(const MLP& a) { return (size_t)(kMlpMaxIn + 8 * a.hid) * kTile; }

// One training step on a batch (kTile samples per block): forward with the
// activations and silu' kept in the block's scratch, loss (kind 0: binary
// cross-entropy on the logit, Sec. 4.1.1; kind 1: absolute error of ln K
// summed over components, Sec. 4.2.1; both averaged over the batch),
// backward, and the weight / bias gradients summed over the block's samples
// and added to `grad`.
__global__ void __launch_bounds__(kTile) k_nn_train_step(MLP a, int kind, int64_t ld, const float* X, const float* Y,
                                                         const int32_t* perm, int batch, float* grad,
                                                         float* scratch, float* loss_acc) {
    const int s = threadIdx.x, lane = s & 31, warp = s >> 5, H = a.hid;
    float* base = scratch + (size_t)blockIdx.x * ((size_t)(kMlpMaxIn + 8 * H) * kTile);
    float* u = base;                           // [din][kTile]
    float* act = u + kMlpMaxIn * kTile;        // [3][H][kTile]
    float* dsl = act + 3 * H * kTile;          // [3][H][kTile]
    float* bufA = dsl + 3 * H * kTile;         // [H][kTile]
    float* bufB = bufA + H * kTile;            // [H][kTile]
    const int64_t idx = perm[(int64_t)blockIdx.x * kTile + s];
    for (int i = 0; i < a.din; i++) u[i * kTile + s] = X[i * ld + idx];
    layer_sample<true>(a, 0, u + s, kTile, act + s, kTile, dsl + s, kTile);
    layer_sample<true>(a, 1, act + s, kTile, act + H * kTile + s, kTile, dsl + H * kTile + s, kTile);
    layer_sample<true>(a, 2, act + H * kTile + s, kTile, act + 2 * H * kTile + s, kTile, dsl + 2 * H * kTile + s,
                       kTile);
    float outv[16];
    layer_sample<false>(a, 3, act + 2 * H * kTile + s, kTile, outv, 1, nullptr, 0);
    const float inv_b = 1.0f / (float)batch;
    float l = 0.0f;
    if (kind == 0) {
        const float zz = outv[0], y = Y[idx];
        l = fmaxf(zz, 0.0f) + log1pf(__expf(-fabsf(zz))) - y * zz;  // softplus(z) - y z
        bufA[s] = (sigmoidf_(zz) - y) * inv_b;
    } else {
        for (int o = 0; o < a.dout; o++) {
            const float d = outv[o] - Y[o * ld + idx];
            l += fabsf(d);
            bufA[o * kTile + s] = (d > 0.0f ? inv_b : (d < 0.0f ? -inv_b : 0.0f));
        }
    }
    l = warp_sum(l);
    if (lane == 0) atomicAdd(loss_acc, l * inv_b);
    __syncthreads();
    float* cur = bufA;
    float* nxt = bufB;
    for (int L = 3; L >= 0; L--) {
        const float* ain = (L == 0) ? u : act + (L - 1) * H * kTile;
        const int nin = layer_in(a, L), nout = layer_out(a, L);
        // dW[o][k] = sum_s cur[o][s] ain[k][s]; db[o] = sum_s cur[o][s]
        float* gW = grad + theta_W(a, L);
        float* gb = grad + theta_b(a, L);
        for (int p = warp; p < nout * nin; p += kTile / 32) {
            const int o = p / nin, k = p - o * nin;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < kTile / 32; j++) acc = fmaf(cur[o * kTile + lane + 32 * j], ain[k * kTile + lane + 32 * j], acc);
            acc = warp_sum(acc);
            if (lane == 0) atomicAdd(gW + p, acc);
        }
        for (int o = warp; o < nout; o += kTile / 32) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < kTile / 32; j++) acc += cur[o * kTile + lane + 32 * j];
            acc = warp_sum(acc);
            if (lane == 0) atomicAdd(gb + o, acc);
        }
        if (L > 0) {
            // d pre_{L-1}[k] = silu'(pre_{L-1}[k]) sum_o W_L[o][k] cur[o]; W_L[o][k] = wt_L[k][o]
            const __nv_bfloat16* W = a.wt + wt_off(a, L);
            const int po = pad8(nout);
            const float* ds = dsl + (L - 1) * H * kTile;
            for (int k = 0; k < nin; k++) {
                float acc = 0.0f;
                for (int o0 = 0; o0 < nout; o0 += 8) {
                    float w[8];
                    ld8(W + (int64_t)k * po + o0, w);
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (o0 + j < nout) acc = fmaf(w[j], cur[(o0 + j) * kTile + s], acc);
                }
                nxt[k * kTile + s] = acc * ds[k * kTile + s];
            }
            float* t = cur;
            cur = nxt;
            nxt = t;
        }
        __syncthreads();
    }
}

// Adam (Kingma & Ba) on the FP32 master; refreshes the BF16 transposed copy
// and clears the gradient accumulator.
__global__ void k_nn_adam(MLP a, int64_t np, float* theta, __nv_bfloat16* wt, float* grad, float* m, float* v,
                          float lr, float b1, float b2, float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = grad[i];
        grad[i] = 0.0f;
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        theta[i] = th;
        for (int L = 0; L < 4; L++) {
            const int64_t w0 = theta_W(a, L), b0 = theta_b(a, L);
            if (i >= w0 && i < b0) {
                const int nin = layer_in(a, L);
                const int64_t o = (i - w0) / nin, k = (i - w0) - o * nin;
                wt[wt_off(a, L) + k * pad8(layer_out(a, L)) + o] = __float2bfloat16_rn(th);
            }
        }
    }
}

// Mean loss and (classifier) number of correct labels at p = 1/2 over X.
__global__ void __launch_bounds__(kTile) k_nn_eval(MLP a, int kind, int64_t n, const float* X, const float* Y,
                                                   double* acc) {
    extern __shared__ float sm[];
    const int s = threadIdx.x;
    float* u = sm + s;
    float* h0 = sm + kMlpMaxIn * kTile + s;
    float* h1 = h0 + a.hid * kTile;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int64_t m = base + s;
        if (m >= n) continue;
        for (int i = 0; i < a.din; i++) u[i * kTile] = X[i * n + m];
        layer_sample<true>(a, 0, u, kTile, h0, kTile, nullptr, 0);
        layer_sample<true>(a, 1, h0, kTile, h1, kTile, nullptr, 0);
        layer_sample<true>(a, 2, h1, kTile, h0, kTile, nullptr, 0);
        float outv[16];
        layer_sample<false>(a, 3, h0, kTile, outv, 1, nullptr, 0);
        double l = 0.0, ok = 0.0;
        if (kind == 0) {
            const float zz = outv[0], y = Y[m];
            l = fmaxf(zz, 0.0f) + log1pf(__expf(-fabsf(zz))) - y * zz;
            ok = ((zz >= 0.0f) == (y >= 0.5f)) ? 1.0 : 0.0;
        } else {
            for (int o = 0; o < a.dout; o++) l += fabsf(outv[o] - Y[o * n + m]);
        }
        atomicAdd(acc, l);
        atomicAdd(acc + 1, ok);
    }
}

// float -> bfloat16, round to nearest even (host)
uint16_t to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

int nn_check(ptflash_ctx* c, int which) {
    if (!c || which < 0 || which > 1) return PTF_ERR_INVALID_ARG;
    if (!c->nn[which].ready) return PTF_ERR_NOT_READY;
    return PTF_OK;
}

}  // namespace

namespace ptf {
// Launch network inference for the flash pipeline (declared in ptf_mlp.cuh).
cudaError_t nn_infer_launch(const MLP& a, int nc, int64_t n, int64_t ld, const double* P, const double* T,
                            const double* z, float* out, int64_t out_ld, int sms, cudaStream_t s) {
    const size_t sm = infer_smem(a);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_nn_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < (int64_t)sms * 8 ? tiles : (int64_t)sms * 8);
    k_nn_infer<<<grid > 0 ? grid : 1, kTile, sm, s>>>(a, nc, n, ld, P, T, z, out, out_ld);
    return cudaGetLastError();
}
}  // namespace ptf

extern "C" {

int ptflash_nn_set(ptflash_ctx* c, int which, int hidden, const float* theta, const float* mean, const float* std) {
    if (!c || which < 0 || which > 1 || !theta || !mean || !std) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (hidden != 64 && hidden != 128) return PTF_ERR_INVALID_ARG;
    const int nc = c->comp.nc, din = nc + 2, dout = which == 0 ? 1 : nc;
    for (int i = 0; i < din; i++)
        if (!(std[i] > 0.0f) || !std::isfinite(mean[i])) return PTF_ERR_INVALID_ARG;
    NNState& N = c->nn[which];
    const int64_t np = theta_size(din, hidden, dout), nw = wt_size(din, hidden, dout);
    if (N.ready && (N.din != din || N.hid != hidden || N.dout != dout)) {
        cudaFree(N.theta);
        cudaFree(N.wt);
        cudaFree(N.mean);
        cudaFree(N.rstd);
        cudaFree(N.grad);
        cudaFree(N.adam_m);
        cudaFree(N.adam_v);
        N = NNState();
    }
    if (!N.theta) {
        if (cudaMalloc(&N.theta, np * 4) != cudaSuccess || cudaMalloc(&N.wt, nw * 2) != cudaSuccess ||
            cudaMalloc(&N.mean, din * 4) != cudaSuccess || cudaMalloc(&N.rstd, din * 4) != cudaSuccess ||
            cudaMalloc(&N.grad, np * 4) != cudaSuccess || cudaMalloc(&N.adam_m, np * 4) != cudaSuccess ||
            cudaMalloc(&N.adam_v, np * 4) != cudaSuccess) {
            cudaGetLastError();
            return PTF_ERR_NO_MEMORY;
        }
    }
    N.din = din;
    N.hid = hidden;
    N.dout = dout;
    // BF16 transposed, padded copy built on the host
    MLP meta{din, hidden, dout, nullptr, nullptr, nullptr, nullptr};
    std::vector<uint16_t> w(nw, 0);
    for (int L = 0; L < 4; L++) {
        const int nin = layer_in(meta, L), nout = layer_out(meta, L);
        const float* W = theta + theta_W(meta, L);
        for (int o = 0; o < nout; o++)
            for (int k = 0; k < nin; k++) w[wt_off(meta, L) + (int64_t)k * pad8(nout) + o] = to_bf16(W[o * nin + k]);
    }
    std::vector<float> rs(din);
    for (int i = 0; i < din; i++) rs[i] = 1.0f / std[i];
    NN_CUDA(cudaMemcpy(N.theta, theta, np * 4, cudaMemcpyHostToDevice));
    NN_CUDA(cudaMemcpy(N.wt, w.data(), nw * 2, cudaMemcpyHostToDevice));
    NN_CUDA(cudaMemcpy(N.mean, mean, din * 4, cudaMemcpyHostToDevice));
    NN_CUDA(cudaMemcpy(N.rstd, rs.data(), din * 4, cudaMemcpyHostToDevice));
    NN_CUDA(cudaMemset(N.grad, 0, np * 4));
    NN_CUDA(cudaMemset(N.adam_m, 0, np * 4));
    NN_CUDA(cudaMemset(N.adam_v, 0, np * 4));
    N.t = 0;
    N.ready = true;
    if (!c->nnbuf) {
        if (cudaMalloc(&c->nnbuf, (size_t)(1 + c->nc_max) * c->n_max * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return PTF_ERR_NO_MEMORY;
        }
    }
    return PTF_OK;
}

int ptflash_nn_get(ptflash_ctx* c, int which, float* theta) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (!theta) return PTF_ERR_INVALID_ARG;
    const NNState& N = c->nn[which];
    NN_CUDA(cudaDeviceSynchronize());
    NN_CUDA(cudaMemcpy(theta, N.theta, theta_size(N.din, N.hid, N.dout) * 4, cudaMemcpyDeviceToHost));
    return PTF_OK;
}

int64_t ptflash_nn_param_count(int din, int hidden, int dout) {
    if (din < 1 || din > kMlpMaxIn || hidden < 1 || dout < 1 || dout > 16) return 0;
    return theta_size(din, hidden, dout);
}

int ptflash_nn_features(ptflash_ctx* c, int which, int64_t n, const double* P, const double* T, const double* z,
                        float* X, void* stream) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!P || !T || !z || !X))) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    k_nn_features<<<c->sm_count * 4, 256, 0, (cudaStream_t)stream>>>(c->nn[which].view(), c->comp.nc, n, n, P, T,
                                                                     z, X);
    NN_CUDA(cudaGetLastError());
    return PTF_OK;
}

int ptflash_nn_infer(ptflash_ctx* c, int which, int64_t n, const double* P, const double* T, const double* z,
                     float* out, void* stream) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!P || !T || !z || !out))) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    NN_CUDA(nn_infer_launch(c->nn[which].view(), c->comp.nc, n, n, P, T, z, out, n, c->sm_count,
                            (cudaStream_t)stream));
    return PTF_OK;
}

int ptflash_nn_train_steps(ptflash_ctx* c, int which, int64_t n, const float* X, const float* Y, const int32_t* perm,
                           int64_t steps, int batch, const float* lr, float beta1, float beta2, float eps,
                           float* loss, void* stream) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (n < 1 || !X || !Y || !perm || !lr || steps < 0 || batch < kTile || batch % kTile) return PTF_ERR_INVALID_ARG;
    NNState& N = c->nn[which];
    cudaStream_t s = (cudaStream_t)stream;
    const MLP a = N.view();
    const size_t need = train_block_floats(a) * (batch / kTile) * sizeof(float);
    if (c->train_scratch_bytes < need) {
        cudaFree(c->train_scratch);
        c->train_scratch = nullptr;
        c->train_scratch_bytes = 0;
        if (cudaMalloc(&c->train_scratch, need) != cudaSuccess) {
            cudaGetLastError();
            return PTF_ERR_NO_MEMORY;
        }
        c->train_scratch_bytes = need;
    }
    const int64_t np = theta_size(N.din, N.hid, N.dout);
    float* dummy_loss = nullptr;
    if (!loss) {
        NN_CUDA(cudaMalloc(&dummy_loss, sizeof(float)));
    }
    for (int64_t k = 0; k < steps; k++) {
        float* lk = loss ? loss + k : dummy_loss;
        if (!loss) NN_CUDA(cudaMemsetAsync(dummy_loss, 0, sizeof(float), s));
        k_nn_train_step<<<batch / kTile, kTile, 0, s>>>(a, which, n, X, Y, perm + k * batch, batch, N.grad,
                                                        c->train_scratch, lk);
        N.t++;
        const float bc1 = 1.0f - std::pow(beta1, (float)N.t), bc2 = 1.0f - std::pow(beta2, (float)N.t);
        k_nn_adam<<<64, 256, 0, s>>>(a, np, N.theta, N.wt, N.grad, N.adam_m, N.adam_v, lr[k], beta1, beta2, eps,
                                     bc1, bc2);
    }
    cudaError_t e = cudaGetLastError();
    if (dummy_loss) {
        cudaStreamSynchronize(s);
        cudaFree(dummy_loss);
    }
    if (e != cudaSuccess) return fail(e);
    return PTF_OK;
}

int ptflash_nn_eval(ptflash_ctx* c, int which, int64_t n, const float* X, const float* Y, double* loss,
                    double* accuracy, void* stream) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (n < 1 || !X || !Y || !loss) return PTF_ERR_INVALID_ARG;
    const MLP a = c->nn[which].view();
    cudaStream_t s = (cudaStream_t)stream;
    double* d = nullptr;
    NN_CUDA(cudaMalloc(&d, 2 * sizeof(double)));
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(double), s);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_nn_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    if (e == cudaSuccess) {
        const int64_t tiles = (n + kTile - 1) / kTile;
        const int grid = (int)(tiles < (int64_t)c->sm_count * 8 ? tiles : (int64_t)c->sm_count * 8);
        k_nn_eval<<<grid, kTile, infer_smem(a), s>>>(a, which, n, X, Y, d);
        e = cudaGetLastError();
    }
    double h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return fail(e);
    *loss = h[0] / (double)n;
    if (accuracy) *accuracy = h[1] / (double)n;
    return PTF_OK;
}

}  // extern "C"
