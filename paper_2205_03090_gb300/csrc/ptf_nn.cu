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

int infer_rows(const MLP& a) { return a.din + (a.arch ? 3 : 2) * a.hid; }
size_t infer_smem(const MLP& a) { return (size_t)infer_rows(a) * kTile * sizeof(float); }

// Inference: each thread runs its sample through the network, keeping the
// activations in its own shared-memory column (no cross-thread traffic).
__global__ void __launch_bounds__(kTile) k_nn_infer(MLP a, int nc, int64_t n, int64_t ld, const double* P,
                                                    const double* T, const double* z, float* out, int64_t out_ld) {
    extern __shared__ float sm[];
    const int s = threadIdx.x;
    float* col = sm + s;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int64_t m = base + s;
        if (m >= n) continue;
        features(a, nc, ld, P, T, z, m, col, kTile);
        forward_sample(a, col, kTile, out + m, out_ld);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core inference: each layer is a [samples x in] x [in x out] product,
// run with the warp-level bf16 MMA (m16n8k16, FP32 accumulators).  A block of
// 256 threads takes 128 samples per round; each warp owns 16 of them (one
// M tile), so the layers need only warp-level ordering.  All weights live in
// shared memory as bf16 [out][in] rows (rounded from the FP32 master like the
// compute copy), padded by 8 elements so that the fragment loads hit 32
// different banks; activations are bf16 rows padded the same way.  Epilogues
// apply bias, SiLU and the bf16 rounding of the scalar path (FP32 sums run in
// another order).  arch 1 keeps [u | h] in one row: the output layer reads the
// concatenation directly and each residual block updates h in place.
// ---------------------------------------------------------------------------
constexpr int kMmaTile = 128;    // samples per block round
constexpr int kMmaThreads = 256;  // 8 warps x 16 samples
constexpr int kUPad = 32;         // input features padded to two k-steps

struct MmaGeom {
    int nl;                // layers
    int K[8], N[8];        // padded inner / output sizes per layer
    int woff[8];           // bf16 element offset of each layer's weights
    int boff[8];           // float offset of each layer's bias
    int wtotal, btotal;
    int rs, ts;            // row strides (bf16 elements) of the activation tiles
    int act0, act1, act2;  // bf16 element offsets of the tiles
    size_t bytes;
};

__host__ __device__ inline MmaGeom mma_geom(const MLP& a) {
    MmaGeom g{};
    const int H = a.hid, L = n_layers(a);
    g.nl = L;
    int w = 0, b = 0;
    for (int l = 0; l < L; l++) {
        const int nout = layer_out(a, l);
        g.K[l] = l == 0 ? kUPad : (a.arch == 1 && l == 7 ? kUPad + H : H);
        g.N[l] = (nout + 7) & ~7;
        g.woff[l] = w;
        g.boff[l] = b;
        w += g.N[l] * (g.K[l] + 8);
        b += g.N[l];
    }
    g.wtotal = w;
    g.btotal = b;
    if (a.arch == 1) {
        g.rs = kUPad + H + 8;  // [u | h]
        g.ts = H + 8;          // a_k
        g.act0 = w;
        g.act1 = w + kMmaTile * g.rs;
        g.act2 = g.act1 + kMmaTile * g.ts;
    } else {
        g.rs = kUPad + 8;      // u
        g.ts = H + 8;          // two hidden tiles
        g.act0 = w;
        g.act1 = w + kMmaTile * g.rs;
        g.act2 = g.act1 + kMmaTile * g.ts;
    }
    const int elems = g.act2 + (a.arch == 1 ? 0 : kMmaTile * g.ts);
    g.bytes = (size_t)elems * 2 + (size_t)g.btotal * 4 + 16;
    return g;
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One layer for this warp's 16 rows: in (row stride sin, first column cin,
// K columns) times W^T (N x K rows of stride K + 8) plus bias.  mode 0:
// out = bf16(silu(.)) into tile (stride sout, column cout); mode 1: residual,
// out = bf16(out + bf16(silu(.))); mode 2: FP32 to global y[o * ld + m].
__device__ __forceinline__ void mma_layer(const __nv_bfloat16* in, int sin, int cin, int K, const __nv_bfloat16* W,
                                          const float* bias, int N, int nreal, __nv_bfloat16* out, int sout,
                                          int cout, int mode, float* y, int64_t ld, int64_t m0, int64_t n) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int ws = K + 8;
    for (int n0 = 0; n0 < N; n0 += 32) {
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
        for (int k0 = 0; k0 < K; k0 += 16) {
            uint32_t af[4];
            const __nv_bfloat16* ar = in + g * sin + cin + k0 + 2 * t;
            af[0] = ld_u32(ar);
            af[1] = ld_u32(ar + 8 * sin);
            af[2] = ld_u32(ar + 8);
            af[3] = ld_u32(ar + 8 * sin + 8);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int nb = n0 + 8 * j;
                if (nb < N) {
                    const __nv_bfloat16* br = W + (nb + g) * ws + k0 + 2 * t;
                    mma_bf16(acc[j], af, ld_u32(br), ld_u32(br + 8));
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int nb = n0 + 8 * j;
            if (nb >= N) continue;
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int row = g + (v >> 1) * 8, col = nb + 2 * t + (v & 1);
                if (col >= nreal) continue;
                const float pre = acc[j][v] + bias[col];
                if (mode == 2) {
                    const int64_t m = m0 + row;
                    if (m < n) y[col * ld + m] = pre;
                } else {
                    float h = bf16_round(pre * sigmoidf_(pre));
                    __nv_bfloat16* o = out + row * sout + cout + col;
                    if (mode == 1) h = bf16_round(__bfloat162float(*o) + h);
                    *o = __float2bfloat16_rn(h);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kMmaThreads, 1) k_nn_infer_mma(MLP a, int nc, int64_t n, int64_t ld, const double* P,
                                                                const double* T, const double* z, float* out,
                                                                int64_t out_ld) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
    const MmaGeom G = mma_geom(a);
    float* sb = reinterpret_cast<float*>(smraw + (size_t)(G.act2 + (a.arch == 1 ? 0 : kMmaTile * G.ts)) * 2);
    // weights: bf16 [N][K + 8] from the FP32 master, zero padding; biases
    for (int l = 0; l < G.nl; l++) {
        const int nin = layer_in(a, l), nout = layer_out(a, l), ws = G.K[l] + 8;
        const float* Wl = a.theta + theta_W(a, l);
        const float* bl = a.theta + theta_b(a, l);
        for (int e = threadIdx.x; e < G.N[l] * ws; e += blockDim.x) {
            const int o = e / ws, kk = e - o * ws;
            int k = -1;  // source column
            if (a.arch == 1 && l == 7) k = kk < a.din ? kk : (kk >= kUPad && kk < kUPad + a.hid ? a.din + kk - kUPad : -1);
            else if (kk < nin) k = kk;
            const float v = (o < nout && k >= 0) ? Wl[o * nin + k] : 0.0f;
            sm[G.woff[l] + e] = __float2bfloat16_rn(v);
        }
        for (int e = threadIdx.x; e < G.N[l]; e += blockDim.x) sb[G.boff[l] + e] = e < nout ? bl[e] : 0.0f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __nv_bfloat16* R = sm + G.act0;     // u (arch 0) or [u | h] (arch 1)
    __nv_bfloat16* A1 = sm + G.act1;
    __nv_bfloat16* A2 = sm + G.act2;
    const int r0 = warp * 16;
    for (int64_t base = (int64_t)blockIdx.x * kMmaTile; base < n; base += (int64_t)gridDim.x * kMmaTile) {
        // features of this warp's 16 samples: two lanes per sample
        for (int e = lane; e < 16 * kUPad; e += 32) {
            const int row = e / kUPad, i = e - row * kUPad;
            const int64_t m = base + r0 + row;
            float v = 0.0f;
            if (m < n && i < a.din) {
                const double x = i < nc ? z[i * ld + m] : (i == nc ? P[m] : T[m]);
                v = ((float)x - __ldg(a.mean + i)) * __ldg(a.rstd + i);
            }
            R[(r0 + row) * G.rs + i] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        const int64_t m0 = base + r0;
        if (a.arch == 0) {
            mma_layer(R + r0 * G.rs, G.rs, 0, G.K[0], sm + G.woff[0], sb + G.boff[0], G.N[0], a.hid,
                      A1 + r0 * G.ts, G.ts, 0, 0, nullptr, 0, 0, 0);
            __syncwarp();
            mma_layer(A1 + r0 * G.ts, G.ts, 0, G.K[1], sm + G.woff[1], sb + G.boff[1], G.N[1], a.hid,
                      A2 + r0 * G.ts, G.ts, 0, 0, nullptr, 0, 0, 0);
            __syncwarp();
            mma_layer(A2 + r0 * G.ts, G.ts, 0, G.K[2], sm + G.woff[2], sb + G.boff[2], G.N[2], a.hid,
                      A1 + r0 * G.ts, G.ts, 0, 0, nullptr, 0, 0, 0);
            __syncwarp();
            mma_layer(A1 + r0 * G.ts, G.ts, 0, G.K[3], sm + G.woff[3], sb + G.boff[3], G.N[3], a.dout,
                      nullptr, 0, 0, 2, out, out_ld, m0, n);
        } else {
            mma_layer(R + r0 * G.rs, G.rs, 0, G.K[0], sm + G.woff[0], sb + G.boff[0], G.N[0], a.hid,
                      R + r0 * G.rs, G.rs, kUPad, 0, nullptr, 0, 0, 0);
            __syncwarp();
            for (int k = 1; k <= 3; k++) {
                mma_layer(R + r0 * G.rs, G.rs, kUPad, G.K[2 * k - 1], sm + G.woff[2 * k - 1], sb + G.boff[2 * k - 1],
                          G.N[2 * k - 1], a.hid, A1 + r0 * G.ts, G.ts, 0, 0, nullptr, 0, 0, 0);
                __syncwarp();
                mma_layer(A1 + r0 * G.ts, G.ts, 0, G.K[2 * k], sm + G.woff[2 * k], sb + G.boff[2 * k], G.N[2 * k],
                          a.hid, R + r0 * G.rs, G.rs, kUPad, 1, nullptr, 0, 0, 0);
                __syncwarp();
            }
            mma_layer(R + r0 * G.rs, G.rs, 0, G.K[7], sm + G.woff[7], sb + G.boff[7], G.N[7], a.dout, nullptr, 0, 0,
                      2, out, out_ld, m0, n);
        }
        __syncwarp();
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

// Vapour fraction of z with K by Rachford-Rice (Eq. RR) on the
// Leibovici-Neoschil window (Appendix C), bisection with Newton steps inside
// the bracket, FP64; and its implicit-function-theorem derivative
// d theta / d ln K_i = K_i z_i / t_i^2 / sum_j z_j (K_j - 1)^2 / t_j^2,
// t_i = 1 + (K_i - 1) theta (Sec. 4.2.2).  False if K does not bracket 1.
__device__ bool rr_theta(int nc, const double* z, const double* K, double& th, double* dth) {
    double kmax = K[0], kmin = K[0];
    for (int i = 1; i < nc; i++) {
        kmax = fmax(kmax, K[i]);
        kmin = fmin(kmin, K[i]);
    }
    if (!(kmax > 1.0 && kmin < 1.0)) return false;
    double lo = 1.0 / (1.0 - kmax), hi = 1.0 / (1.0 - kmin);
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 100; it++) {
        double f = 0.0, fp = 0.0;
        for (int i = 0; i < nc; i++) {
            const double km = K[i] - 1.0, ti = 1.0 / fma(km, t, 1.0);
            f = fma(z[i] * km, ti, f);
            fp = fma(-z[i] * km * km, ti * ti, fp);
        }
        if (f > 0.0) lo = t; else hi = t;
        double tn = t - f / fp;
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const bool done = fabs(tn - t) <= 1e-14 * fmax(1.0, fabs(t));
        t = tn;
        if (done || !(hi > lo)) break;
    }
    double den = 0.0;
    for (int i = 0; i < nc; i++) {
        const double km = K[i] - 1.0, ti = 1.0 / fma(km, t, 1.0);
        den = fma(z[i] * km * km, ti * ti, den);
    }
    for (int i = 0; i < nc; i++) {
        const double ti = 1.0 / fma(K[i] - 1.0, t, 1.0);
        dth[i] = K[i] * z[i] * ti * ti / den;
    }
    th = t;
    return true;
}

// Loss kinds: 0 binary cross-entropy on the logit (classifier, Sec. 4.1.1);
// 1 absolute error of ln K summed over components (initializer, Sec. 4.2.1);
// 2 kind 1 plus wth |theta - theta_hat|, theta_hat the Rachford-Rice root
// for the predicted K (Sec. 4.2.2, second stage).  Kind 2 targets Y carry
// 2 nc + 1 rows: ln K, theta, then the raw z.
// Per-sample loss and, with g != null, d loss / d output into g[o * gst].
__device__ float sample_loss(int kind, int dout, float wth, const float* outv, const float* Y, int64_t ld, int64_t idx,
                             float scale, float* g, int gst, float* th_err) {
    float l = 0.0f;
    if (th_err) *th_err = 0.0f;
    if (kind == 0) {
        const float zz = outv[0], y = Y[idx];
        l = fmaxf(zz, 0.0f) + log1pf(__expf(-fabsf(zz))) - y * zz;  // softplus(z) - y z
        if (g) g[0] = (sigmoidf_(zz) - y) * scale;
        return l;
    }
    for (int o = 0; o < dout; o++) {
        const float d = outv[o] - Y[o * ld + idx];
        l += fabsf(d);
        if (g) g[o * gst] = (d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f));
    }
    if (kind == 2) {
        double z[16], K[16], dth[16], th;
        for (int i = 0; i < dout; i++) {
            z[i] = (double)Y[(dout + 1 + i) * ld + idx];
            K[i] = exp((double)outv[i]);
        }
        if (rr_theta(dout, z, K, th, dth)) {
            const double e = th - (double)Y[dout * ld + idx];
            l += wth * (float)fabs(e);
            if (th_err) *th_err = (float)fabs(e);
            if (g) {
                const float sg = e > 0.0 ? scale * wth : (e < 0.0 ? -scale * wth : 0.0f);
                for (int i = 0; i < dout; i++) g[i * gst] += sg * (float)dth[i];
            }
        }
    }
    return l;
}

// Block-level gradient of one dense layer: dW[o][k] += sum_s cur[o][s] in[k][s],
// db[o] += sum_s cur[o][s] over the block's kTile samples (columns).
__device__ void accum_grads(const MLP& a, int L, const float* cur, const float* ain, float* grad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nin = layer_in(a, L), nout = layer_out(a, L);
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
}

// Per-sample input gradient of one dense layer for inputs k0 .. k0 + nk - 1:
// dx[k - k0] = (add ? dx : 0) + sum_o W_L[o][k] cur[o] (W_L[o][k] = wt_L[k][o]),
// times silu'(pre) of that input when ds is given.
__device__ void back_input(const MLP& a, int L, const float* cur, float* dx, int k0, int nk, const float* ds,
                           bool add) {
    const int s = threadIdx.x, nout = layer_out(a, L), po = pad8(nout);
    const __nv_bfloat16* W = a.wt + wt_off(a, L);
    for (int k = k0; k < k0 + nk; k++) {
        float acc = 0.0f;
        for (int o0 = 0; o0 < nout; o0 += 8) {
            float w[8];
            ld8(W + (int64_t)k * po + o0, w);
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (o0 + j < nout) acc = fmaf(w[j], cur[(o0 + j) * kTile + s], acc);
        }
        float v = add ? dx[(k - k0) * kTile + s] + acc : acc;
        if (ds) v *= ds[(k - k0) * kTile + s];
        dx[(k - k0) * kTile + s] = v;
    }
}

__host__ __device__ size_t train_block_floats(const MLP& a) {
    return (size_t)(a.arch ? a.din + 17 * a.hid : kMlpMaxIn + 8 * a.hid) * kTile;
}

// One training step on a batch (kTile samples per block): forward with the
// activations and silu' kept in the block's scratch, loss (sample_loss,
// averaged over the batch), backward, and the weight / bias gradients summed
// over the block's samples and added to `grad`.  The bf16 rounding of the
// forward pass is passed through unchanged by the backward pass.
__global__ void __launch_bounds__(kTile) k_nn_train_step(MLP a, int kind, float wth, int64_t ld, const float* X,
                                                         const float* Y, const int32_t* perm, int batch, float* grad,
                                                         float* scratch, float* loss_acc) {
    const int s = threadIdx.x, lane = s & 31, H = a.hid;
    float* base = scratch + (size_t)blockIdx.x * train_block_floats(a);
    const int64_t idx = perm[(int64_t)blockIdx.x * kTile + s];
    const float inv_b = 1.0f / (float)batch;
    float outv[16];
    float l;
    if (a.arch == 0) {
        float* u = base;                           // [din][kTile]
        float* act = u + kMlpMaxIn * kTile;        // [3][H][kTile]
        float* dsl = act + 3 * H * kTile;          // [3][H][kTile]
        float* bufA = dsl + 3 * H * kTile;         // [H][kTile]
        float* bufB = bufA + H * kTile;            // [H][kTile]
        for (int i = 0; i < a.din; i++) u[i * kTile + s] = X[i * ld + idx];
        for (int L = 0; L < 3; L++)
            layer_sample<true>(a, L, (L == 0 ? u : act + (L - 1) * H * kTile) + s, kTile, act + L * H * kTile + s,
                               kTile, dsl + L * H * kTile + s, kTile);
        layer_sample<false>(a, 3, act + 2 * H * kTile + s, kTile, outv, 1, nullptr, 0);
        l = sample_loss(kind, a.dout, wth, outv, Y, ld, idx, inv_b, bufA + s, kTile, nullptr);
        __syncthreads();
        float* cur = bufA;
        float* nxt = bufB;
        for (int L = 3; L >= 0; L--) {
            const float* ain = (L == 0) ? u : act + (L - 1) * H * kTile;
            accum_grads(a, L, cur, ain, grad);
            if (L > 0) {
                back_input(a, L, cur, nxt, 0, H, dsl + (L - 1) * H * kTile, false);
                float* t = cur;
                cur = nxt;
                nxt = t;
            }
            __syncthreads();
        }
    } else {
        // rows: [u (din)][h3 (H)] contiguous (the output layer's input), h0, h1,
        // h2, a1, a2, a3, silu' of the 7 hidden pre-activations, three buffers
        float* u = base;
        float* h3 = u + a.din * kTile;
        float* hk = h3 + H * kTile;                // h0, h1, h2
        float* ak = hk + 3 * H * kTile;            // a1, a2, a3
        float* dsl = ak + 3 * H * kTile;           // layer 0, then (a_k, c_k) for k = 1..3
        float* bufA = dsl + 7 * H * kTile;
        float* bufB = bufA + H * kTile;
        float* bufC = bufB + H * kTile;
        auto hp = [&](int k) { return k == 3 ? h3 : hk + k * H * kTile; };
        for (int i = 0; i < a.din; i++) u[i * kTile + s] = X[i * ld + idx];
        layer_sample<true>(a, 0, u + s, kTile, hp(0) + s, kTile, dsl + s, kTile);
        for (int k = 1; k <= 3; k++) {
            float* ah = ak + (k - 1) * H * kTile;
            layer_sample<true>(a, 2 * k - 1, hp(k - 1) + s, kTile, ah + s, kTile, dsl + (2 * k - 1) * H * kTile + s,
                               kTile);
            layer_sample<true>(a, 2 * k, ah + s, kTile, bufC + s, kTile, dsl + 2 * k * H * kTile + s, kTile);
            float* hn = hp(k);
            const float* hpv = hp(k - 1);
            for (int j = 0; j < H; j++) hn[j * kTile + s] = bf16_round(hpv[j * kTile + s] + bufC[j * kTile + s]);
        }
        layer_sample<false>(a, 7, u + s, kTile, outv, 1, nullptr, 0);
        l = sample_loss(kind, a.dout, wth, outv, Y, ld, idx, inv_b, bufA + s, kTile, nullptr);
        __syncthreads();
        accum_grads(a, 7, bufA, u, grad);              // input [u; h3]
        back_input(a, 7, bufA, bufB, a.din, H, nullptr, false);  // bufB = d h3
        __syncthreads();
        for (int k = 3; k >= 1; k--) {
            // c_k = silu(W_2k a_k + b): d pre = d h_k * silu'
            for (int j = 0; j < H; j++) bufC[j * kTile + s] = bufB[j * kTile + s] * dsl[(2 * k * H + j) * kTile + s];
            __syncthreads();
            accum_grads(a, 2 * k, bufC, ak + (k - 1) * H * kTile, grad);
            back_input(a, 2 * k, bufC, bufA, 0, H, dsl + (2 * k - 1) * H * kTile, false);  // d pre of a_k
            __syncthreads();
            accum_grads(a, 2 * k - 1, bufA, hp(k - 1), grad);
            back_input(a, 2 * k - 1, bufA, bufB, 0, H, nullptr, true);  // d h_{k-1} = d h_k + W^T d pre
            __syncthreads();
        }
        for (int j = 0; j < H; j++) bufB[j * kTile + s] *= dsl[j * kTile + s];
        __syncthreads();
        accum_grads(a, 0, bufB, u, grad);
        __syncthreads();
    }
    l = warp_sum(l);
    if (lane == 0) atomicAdd(loss_acc, l * inv_b);
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
        for (int L = 0; L < n_layers(a); L++) {
            const int64_t w0 = theta_W(a, L), b0 = theta_b(a, L);
            if (i >= w0 && i < b0) {
                const int nin = layer_in(a, L);
                const int64_t o = (i - w0) / nin, k = (i - w0) - o * nin;
                wt[wt_off(a, L) + k * pad8(layer_out(a, L)) + o] = __float2bfloat16_rn(th);
            }
        }
    }
}

// Mean loss over X and a second statistic: the number of correct labels at
// p = 1/2 (kind 0) or the summed |theta - theta_hat| (kind 2).
__global__ void __launch_bounds__(kTile) k_nn_eval(MLP a, int kind, float wth, int64_t n, const float* X,
                                                   const float* Y, double* acc) {
    extern __shared__ float sm[];
    const int s = threadIdx.x;
    float* col = sm + s;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int64_t m = base + s;
        if (m >= n) continue;
        for (int i = 0; i < a.din; i++) col[i * kTile] = X[i * n + m];
        float outv[16];
        forward_sample(a, col, kTile, outv, 1);
        float the = 0.0f;
        const double l = sample_loss(kind, a.dout, wth, outv, Y, n, m, 1.0f, nullptr, 0, &the);
        double ok = 0.0;
        if (kind == 0) ok = ((outv[0] >= 0.0f) == (Y[m] >= 0.5f)) ? 1.0 : 0.0;
        if (kind == 2) ok = the;
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
    const MmaGeom G = mma_geom(a);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_nn_infer_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    if (G.bytes > 220 * 1024) return cudaErrorInvalidValue;
    const int64_t tiles = (n + kMmaTile - 1) / kMmaTile;
    const int grid = (int)(tiles < (int64_t)sms ? tiles : (int64_t)sms);
    k_nn_infer_mma<<<grid > 0 ? grid : 1, kMmaThreads, G.bytes, s>>>(a, nc, n, ld, P, T, z, out, out_ld);
    return cudaGetLastError();
}

// The scalar forward pass (one thread per sample, FP32 sums in input order),
// kept beside the tensor-core one for the comparison test.
cudaError_t nn_infer_scalar_launch(const MLP& a, int nc, int64_t n, int64_t ld, const double* P, const double* T,
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

int ptflash_nn_set_arch(ptflash_ctx* c, int which, int arch, int hidden, const float* theta, const float* mean,
                        const float* std) {
    if (!c || which < 0 || which > 1 || !theta || !mean || !std) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (arch == 0 && hidden != 32 && hidden != 64 && hidden != 128) return PTF_ERR_INVALID_ARG;
    if (arch == 1 && hidden != 32 && hidden != 64) return PTF_ERR_INVALID_ARG;
    if (arch != 0 && arch != 1) return PTF_ERR_INVALID_ARG;
    const int nc = c->comp.nc, din = nc + 2, dout = which == 0 ? 1 : nc;
    for (int i = 0; i < din; i++)
        if (!(std[i] > 0.0f) || !std::isfinite(mean[i])) return PTF_ERR_INVALID_ARG;
    NNState& N = c->nn[which];
    MLP meta{din, hidden, dout, nullptr, nullptr, nullptr, nullptr, arch};
    const int64_t np = theta_size(meta), nw = wt_size(meta);
    if (N.ready && (N.din != din || N.hid != hidden || N.dout != dout || N.arch != arch)) {
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
    N.arch = arch;
    // BF16 transposed, padded copy built on the host
    std::vector<uint16_t> w(nw, 0);
    for (int L = 0; L < n_layers(meta); L++) {
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

int ptflash_nn_set(ptflash_ctx* c, int which, int hidden, const float* theta, const float* mean, const float* std) {
    return ptflash_nn_set_arch(c, which, 0, hidden, theta, mean, std);
}

int ptflash_nn_set_theta_loss(ptflash_ctx* c, int which, float weight) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (which != 1 || !(weight >= 0.0f) || !std::isfinite(weight)) return PTF_ERR_INVALID_ARG;
    c->nn[which].theta_w = weight;
    return PTF_OK;
}

int ptflash_nn_get(ptflash_ctx* c, int which, float* theta) {
    int rc = nn_check(c, which);
    if (rc) return rc;
    if (!theta) return PTF_ERR_INVALID_ARG;
    const NNState& N = c->nn[which];
    NN_CUDA(cudaDeviceSynchronize());
    NN_CUDA(cudaMemcpy(theta, N.theta, theta_size(N.view()) * 4, cudaMemcpyDeviceToHost));
    return PTF_OK;
}

int64_t ptflash_nn_param_count_arch(int arch, int din, int hidden, int dout) {
    if (din < 1 || din > kMlpMaxIn || hidden < 1 || dout < 1 || dout > 16 || (arch != 0 && arch != 1)) return 0;
    return theta_size(MLP{din, hidden, dout, nullptr, nullptr, nullptr, nullptr, arch});
}

int64_t ptflash_nn_param_count(int din, int hidden, int dout) { return ptflash_nn_param_count_arch(0, din, hidden, dout); }

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
    const int64_t np = theta_size(a);
    const int kind = which == 0 ? 0 : (N.theta_w > 0.0f ? 2 : 1);
    float* dummy_loss = nullptr;
    if (!loss) {
        NN_CUDA(cudaMalloc(&dummy_loss, sizeof(float)));
    }
    for (int64_t k = 0; k < steps; k++) {
        float* lk = loss ? loss + k : dummy_loss;
        if (!loss) NN_CUDA(cudaMemsetAsync(dummy_loss, 0, sizeof(float), s));
        k_nn_train_step<<<batch / kTile, kTile, 0, s>>>(a, kind, N.theta_w, n, X, Y, perm + k * batch, batch, N.grad,
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
    const int kind = which == 0 ? 0 : (c->nn[which].theta_w > 0.0f ? 2 : 1);
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
        k_nn_eval<<<grid, kTile, infer_smem(a), s>>>(a, kind, c->nn[which].theta_w, n, X, Y, d);
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
