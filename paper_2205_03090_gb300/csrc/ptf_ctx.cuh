// ptf_ctx.cuh -- the context behind the opaque ptflash_ctx handle.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ptf_launch.cuh"
#include "ptf_mlp.cuh"

namespace ptf {
// One network of the learned form: parameters, Adam state, feature scaler.
struct NNState {
    int din = 0, hid = 0, dout = 0;
    float* theta = nullptr;          // FP32 master, natural layout
    __nv_bfloat16* wt = nullptr;     // BF16 transposed compute copy
    float* mean = nullptr;           // [din]
    float* rstd = nullptr;           // [din]
    float* grad = nullptr;           // FP32 gradient accumulator (zeroed by the Adam step)
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long t = 0;                 // Adam step count
    bool ready = false;
    int arch = 0;                    // 0: three hidden layers; 1: residual blocks + wide output
    float theta_w = 0.0f;            // initializer: weight of |theta - theta_hat| in the loss (0: off)

    MLP view() const { return MLP{din, hid, dout, theta, wt, mean, rstd, arch}; }
};
}  // namespace ptf

using namespace ptf;

struct ptflash_ctx {
    int device = 0;
    int nc_max = 0;
    int64_t n_max = 0;
    int sm_count = 0;
    CompHost comp{};
    bool have_comp = false;
    // device scratch
    double* wsd = nullptr;    // (8 nc_max + 3) n_max doubles
    int32_t* wsi = nullptr;   // 9 n_max + 64 int32
    // staging for the host-pointer entry point
    double* hd = nullptr;     // (4 nc_max + 3) n_max doubles: P, T, z, beta, x, y, K
    int32_t* hi = nullptr;    // 3 n_max: nphase, status, iters
    unsigned long long* acc = nullptr;  // device: queue sizes summed over the chunks of a call
    // learned form (Sec. 4): 0 classifier, 1 initializer
    NNState nn[2];
    float* nnbuf = nullptr;       // (1 + nc_max) n_max floats: classifier logit, initializer ln K
    float* train_scratch = nullptr;
    size_t train_scratch_bytes = 0;
    bool profiling = false;
    Conc conc;  // streams and events of the concurrent split SS (flash calls without profiling)
    cudaEvent_t ev[kStages + 1] = {};
    double stage_ms[kStages] = {};
};

// Device scratch of one chunk of n mixtures, carved from the context's buffers.
inline ptf::WS make_ws(ptflash_ctx* c, int64_t n) {
    const int nc = c->comp.nc;
    ptf::WS w;
    w.n = n;
    double* p = c->wsd;
    w.sA = p; p += (int64_t)nc * n;
    w.B = p; p += (int64_t)nc * n;
    w.lnz = p; p += (int64_t)nc * n;
    w.d = p; p += (int64_t)nc * n;
    w.lnK = p; p += (int64_t)nc * n;
    w.nV = p; p += (int64_t)nc * n;
    w.lnW = p; p += 2 * (int64_t)nc * n;
    w.theta = p; p += n;
    w.tm = p; p += 2 * n;
    int32_t* q = c->wsi;
    w.cnt = q; q += 64;
    w.tflag = q; q += 2 * n;
    w.q_stab = q; q += n;
    w.q_split = q; q += n;
    w.q_stab_tr = q; q += 2 * n;
    w.q_split_tr = q; q += n;
    w.q_redo = q; q += n;
    w.q_sort = q; q += n;
    w.acc = c->acc;
    w.nnp = c->nnbuf;
    w.nnk = c->nnbuf ? c->nnbuf + n : nullptr;
    return w;
}
