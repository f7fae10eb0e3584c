// ptf_launch.cuh -- host-side launch sequences, one instantiation per NC.
#pragma once
#include <cmath>
#include "ptf_kernels.cuh"
#include "ptf_comp.cuh"
#include "ptf_mlp.cuh"

namespace ptf {

// Stage order of the timing events: prep(+precheck), stability SS,
// stability TR, decide (or stability output), split SS, split TR.
constexpr int kStages = 6;

// Blocks of 128 threads for a persistent (refill) kernel: as many as fit on
// the device at once.
template <class Kernel>
int persistent_grid(Kernel k, int sms) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, 128, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return sms * b;
}

// mode 0: plain flash; mode 1: stability only.  ev (optional, kStages + 1
// events) is recorded before each stage and after the last one.  `grid` is
// the grid of the one-pass kernels; the persistent kernels are sized to the
// device (sms = grid / 8).
// mode 2: learned form; nn = {classifier, initializer}, p_l / p_r its thresholds.
template <int NC>
cudaError_t launch_plain(const CompHost& h, const WS& ws, const IO& io, int grid, int mode, cudaStream_t s,
                         cudaEvent_t* ev, const MLP* nn = nullptr, float p_l = 0.02f, float p_r = 0.98f) {
    const Comp<NC> cp = make_comp<NC>(h);
    const int sms = grid / 8 > 0 ? grid / 8 : 1;
    static const int g_pre = persistent_grid(k_precheck<NC>, sms);
    static const int g_sss = persistent_grid(k_stab_ss<NC>, sms);
    static const int g_sps = persistent_grid(k_split_ss<NC>, sms);
    static const int g_str = persistent_grid(k_stab_tr<NC>, sms);
    static const int g_spt = persistent_grid(k_split_tr<NC>, sms);
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], s);
    };
    mark(0);
    if (mode == 0) {
        k_prep<NC, true><<<grid, 128, 0, s>>>(cp, ws, io);
        k_precheck<NC><<<g_pre, 128, 0, s>>>(cp, ws, io);
    } else if (mode == 2) {
        k_prep<NC, true><<<grid, 128, 0, s>>>(cp, ws, io);
        cudaError_t e = nn_infer_launch(nn[0], NC, ws.n, io.ld, io.P, io.T, io.z, ws.nnp, ws.n, sms, s);
        if (e == cudaSuccess) e = nn_infer_launch(nn[1], NC, ws.n, io.ld, io.P, io.T, io.z, ws.nnk, ws.n, sms, s);
        if (e != cudaSuccess) return e;
        k_nn_route<NC><<<grid, 128, 0, s>>>(cp, ws, io, p_l, p_r);
    } else {
        k_prep<NC, false><<<grid, 128, 0, s>>>(cp, ws, io);
    }
    mark(1);
    k_stab_ss<NC><<<g_sss, 128, 0, s>>>(cp, ws, io);
    mark(2);
    k_stab_tr<NC><<<g_str, 128, 0, s>>>(cp, ws, io);
    mark(3);
    if (mode != 1) k_stab_decide<NC><<<grid, 128, 0, s>>>(cp, ws, io);
    else k_stab_out<NC><<<grid, 128, 0, s>>>(cp, ws, io);
    mark(4);
    if (mode != 1) {
        k_split_ss<NC><<<g_sps, 128, 0, s>>>(cp, ws, io);
        mark(5);
        k_split_tr<NC><<<g_spt, 128, 0, s>>>(cp, ws, io);
        mark(6);
    } else {
        mark(5);
        mark(6);
    }
    return cudaGetLastError();
}

// explicit instantiations live in ptf_inst_*.cu
#define PTF_DECLARE_NC(NC) \
    extern template cudaError_t launch_plain<NC>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, \
                                                 cudaEvent_t*, const MLP*, float, float);
PTF_DECLARE_NC(2) PTF_DECLARE_NC(3) PTF_DECLARE_NC(4) PTF_DECLARE_NC(5) PTF_DECLARE_NC(6) PTF_DECLARE_NC(7)
PTF_DECLARE_NC(8) PTF_DECLARE_NC(9) PTF_DECLARE_NC(10) PTF_DECLARE_NC(11) PTF_DECLARE_NC(12) PTF_DECLARE_NC(13)
PTF_DECLARE_NC(14) PTF_DECLARE_NC(15) PTF_DECLARE_NC(16)
#undef PTF_DECLARE_NC

}  // namespace ptf
