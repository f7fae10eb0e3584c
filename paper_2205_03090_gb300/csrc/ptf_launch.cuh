// ptf_launch.cuh -- host-side launch sequences, one instantiation per NC.
#pragma once
#include <cmath>
#include "ptf_kernels.cuh"
#include "ptf_comp.cuh"
#include "ptf_mlp.cuh"
#include "ptf_adjoint.cuh"
#include "ptf_grid.h"

namespace ptf {

// Stage order of the timing events: prep(+precheck), stability SS,
// stability TR, decide (or stability output), split SS, split TR.
constexpr int kStages = 6;

// Blocks of 128 threads for a persistent (refill) kernel K on the current
// device with `sms` SMs: as many as fit on the device at once.
template <auto K>
int persistent_grid(int sms) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = -1;
    }
    const int per_sm = BlocksPerSM<K>::get(dev, [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, 128, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 1;
        }
        return b;
    });
    return persistent_blocks(sms, per_sm);
}

// Streams and events (owned by the caller) that let the split SS of the
// mixtures the precheck (or the classifier gate) sends to the split run beside
// the stability stages: those do not depend on stability analysis.  The
// stability chain runs on the high-priority stream; the independent split SS
// runs on the low-priority one in short blocks, which take the SMs the chain's
// kernels leave idle as they drain.
struct Conc {
    cudaStream_t hi = nullptr, lo = nullptr;
    cudaEvent_t fork = nullptr, pre = nullptr, lo_done = nullptr, hi_done = nullptr;
};
// Items per block of the low-priority split SS (2 per thread; 512 and more
// measured slower).
constexpr int kFillerQuota = 256;

// The flash pipeline over one workspace.  mode 0: plain flash; mode 1:
// stability only; mode 2: learned form (nn = {classifier, initializer}, p_l /
// p_r its thresholds; the plain method judges the networks' routes, and a
// second pass of the plain stages redoes the rejected mixtures, the split
// trust-region stage's events then covering both).  ev (optional, kStages + 1 events) is recorded before
// each stage and after the last one.  `grid` is the grid of the one-pass
// kernels; the persistent kernels are sized to the device (sms = grid / 8),
// or to `pgrid` blocks when it is positive.  CS is the component source
// (OneSys or ManySys).  cc (optional, flash modes without stage events): run
// the stages on cc's streams as described at Conc; the work is ordered after
// what s holds and s waits for all of it.
template <int NC, class CS>
cudaError_t launch_pipeline(const CS& cs, const WS& ws, const IO& io, int grid, int mode, cudaStream_t s,
                            cudaEvent_t* ev, const MLP* nn = nullptr, float p_l = 0.02f, float p_r = 0.98f,
                            int pgrid = 0, const Conc* cc = nullptr) {
    const int sms = grid / 8 > 0 ? grid / 8 : 1;
    const int g_pre = persistent_grid<k_precheck<NC, CS>>(sms);
    const int g_p32 = persistent_grid<k_precheck32<NC, CS>>(sms);
    const int g_sss = persistent_grid<k_stab_ss<NC, CS>>(sms);
    const int g_s32 = persistent_grid<k_stab_ss32<NC, CS>>(sms);
    const int g_sps = persistent_grid<k_split_ss<NC, CS>>(sms);
    const int g_s3s = persistent_grid<k_split_ss32<NC, CS>>(sms);
    const int g_str = persistent_grid<k_stab_tr<NC, CS>>(sms);
    const int g_spt = persistent_grid<k_split_tr<NC, CS>>(sms);
    auto pg = [&](int g) { return pgrid > 0 ? pgrid : g; };
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], s);
    };
    const bool conc = cc && !ev && mode != 1;
    const cudaStream_t s0 = s;
    if (conc) {
        cudaEventRecord(cc->fork, s0);
        cudaStreamWaitEvent(cc->hi, cc->fork, 0);
        s = cc->hi;
    }
    mark(0);
    if (mode == 0) {
        k_prep<NC, true, CS><<<grid, 128, 0, s>>>(cs, ws, io);
        k_precheck32<NC, CS><<<pg(g_p32), 128, 0, s>>>(cs, ws, io);
        k_precheck<NC, CS><<<pg(g_pre), 128, 0, s>>>(cs, ws, io);
    } else if (mode == 2) {
        k_prep<NC, true, CS><<<grid, 128, 0, s>>>(cs, ws, io);
        cudaError_t e = nn_infer_launch(nn[0], NC, ws.n, io.ld, io.P, io.T, io.z, ws.nnp, ws.n, sms, s);
        if (e == cudaSuccess) e = nn_infer_launch(nn[1], NC, ws.n, io.ld, io.P, io.T, io.z, ws.nnk, ws.n, sms, s);
        if (e != cudaSuccess) return e;
        k_nn_route<NC, CS><<<grid, 128, 0, s>>>(cs, ws, io, p_l, p_r);
        // the mixtures the networks leave to the plain method (status 0)
        k_precheck32<NC, CS><<<pg(g_p32), 128, 0, s>>>(cs, ws, io);
        k_precheck<NC, CS><<<pg(g_pre), 128, 0, s>>>(cs, ws, io);
    } else {
        k_prep<NC, false, CS><<<grid, 128, 0, s>>>(cs, ws, io);
    }
    mark(1);
    if (conc) {
        cudaEventRecord(cc->pre, s);
        cudaStreamWaitEvent(cc->lo, cc->pre, 0);
        const int fg = (int)((ws.n + kFillerQuota - 1) / kFillerQuota);
        k_split_ss32<NC, CS><<<fg > 0 ? fg : 1, 128, 0, cc->lo>>>(cs, ws, io, 0, kFillerQuota);
        k_split_ss<NC, CS><<<fg > 0 ? fg : 1, 128, 0, cc->lo>>>(cs, ws, io, 0, kFillerQuota);
        cudaEventRecord(cc->lo_done, cc->lo);
    }
    k_stab_ss32<NC, CS><<<pg(g_s32), 128, 0, s>>>(cs, ws, io);
    k_stab_ss<NC, CS><<<pg(g_sss), 128, 0, s>>>(cs, ws, io);
    mark(2);
    k_stab_tr<NC, CS><<<pg(g_str), 128, 0, s>>>(cs, ws, io);
    mark(3);
    if (mode != 1) k_stab_decide<NC, CS><<<grid, 128, 0, s>>>(cs, ws, io);
    else k_stab_out<NC, CS><<<grid, 128, 0, s>>>(cs, ws, io);
    mark(4);
    if (mode != 1) {
        k_split_ss32<NC, CS><<<pg(g_s3s), 128, 0, s>>>(cs, ws, io, conc ? 1 : 2, 0);
        k_split_ss<NC, CS><<<pg(g_sps), 128, 0, s>>>(cs, ws, io, conc ? 1 : 2, 0);
        if (conc) cudaStreamWaitEvent(s, cc->lo_done, 0);
        mark(5);
        k_tr_order<<<grid, 128, 0, s>>>(ws);
        k_split_tr<NC, CS><<<pg(g_spt), 128, 0, s>>>(cs, ws, io);
        if (mode == 2) {
            // judge the network-started splits, then the plain method's second
            // pass over the rejected mixtures (one after another, on s)
            k_nn_judge<NC, CS><<<grid, 128, 0, s>>>(cs, ws, io);
            if (ws.acc) k_fold_counts<<<1, 32, 0, s>>>(ws.cnt, ws.acc);
            cudaMemsetAsync(ws.cnt, 0, Q_REDO * sizeof(int32_t), s);
            cudaMemsetAsync(ws.cnt + Q_REDO + 1, 0, (kCntSlots - Q_REDO - 1) * sizeof(int32_t), s);
            WS w2 = ws;
            w2.q_pre = ws.q_redo;
            k_precheck32<NC, CS><<<pg(g_p32), 128, 0, s>>>(cs, w2, io);
            k_precheck<NC, CS><<<pg(g_pre), 128, 0, s>>>(cs, w2, io);
            k_stab_ss32<NC, CS><<<pg(g_s32), 128, 0, s>>>(cs, w2, io);
            k_stab_ss<NC, CS><<<pg(g_sss), 128, 0, s>>>(cs, w2, io);
            k_stab_tr<NC, CS><<<pg(g_str), 128, 0, s>>>(cs, w2, io);
            k_stab_decide<NC, CS><<<grid, 128, 0, s>>>(cs, w2, io);
            k_split_ss32<NC, CS><<<pg(g_s3s), 128, 0, s>>>(cs, w2, io, 2, 0);
            k_split_ss<NC, CS><<<pg(g_sps), 128, 0, s>>>(cs, w2, io, 2, 0);
            k_tr_order<<<grid, 128, 0, s>>>(w2);
            k_split_tr<NC, CS><<<pg(g_spt), 128, 0, s>>>(cs, w2, io);
        }
        mark(6);
    } else {
        mark(5);
        mark(6);
    }
    if (conc) {
        cudaEventRecord(cc->hi_done, s);
        cudaStreamWaitEvent(s0, cc->hi_done, 0);
    }
    return cudaGetLastError();
}

// One fluid system (the component table as a kernel parameter).
template <int NC>
cudaError_t launch_plain(const CompHost& h, const WS& ws, const IO& io, int grid, int mode, cudaStream_t s,
                         cudaEvent_t* ev, const MLP* nn = nullptr, float p_l = 0.02f, float p_r = 0.98f,
                         const Conc* cc = nullptr) {
    const OneSys<NC> cs{make_comp<NC>(h)};
    return launch_pipeline<NC>(cs, ws, io, grid, mode, s, ev, nn, p_l, p_r, 0, cc);
}

// Several systems of one nc over one workspace (a group of a batch): mode 0
// or 1, `pgrid` blocks for the persistent kernels (0: device-filling).
template <int NC>
cudaError_t launch_many(const Comp<NC>* tab, const int32_t* sys, const WS& ws, const IO& io, int grid, int mode,
                        int pgrid, cudaStream_t s) {
    const ManySys<NC> cs{tab, sys};
    return launch_pipeline<NC>(cs, ws, io, grid, mode, s, nullptr, nullptr, 0.02f, 0.98f, pgrid);
}

// Phase EOS at given compositions (k_phase_eos).
template <int NC>
cudaError_t launch_eos(const CompHost& h, int64_t n, const double* P, const double* T, const double* c, double* Z,
                       double* lnphi, int grid, cudaStream_t s) {
    const Comp<NC> cp = make_comp<NC>(h);
    k_phase_eos<NC><<<grid, 128, 0, s>>>(cp, n, P, T, c, Z, lnphi);
    return cudaGetLastError();
}

// explicit instantiations live in ptf_inst_*.cu
#define PTF_DECLARE_NC(NC)                                                                                      \
    extern template cudaError_t launch_plain<NC>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, \
                                                 cudaEvent_t*, const MLP*, float, float, const Conc*);           \
    extern template cudaError_t launch_many<NC>(const Comp<NC>*, const int32_t*, const WS&, const IO&, int, int, \
                                                int, cudaStream_t);                                              \
    extern template cudaError_t launch_adjoint<NC>(const CompHost&, const AdjIO&, int, cudaStream_t);            \
    extern template cudaError_t launch_eos<NC>(const CompHost&, int64_t, const double*, const double*,          \
                                               const double*, double*, double*, int, cudaStream_t);
PTF_DECLARE_NC(2) PTF_DECLARE_NC(3) PTF_DECLARE_NC(4) PTF_DECLARE_NC(5) PTF_DECLARE_NC(6) PTF_DECLARE_NC(7)
PTF_DECLARE_NC(8) PTF_DECLARE_NC(9) PTF_DECLARE_NC(10) PTF_DECLARE_NC(11) PTF_DECLARE_NC(12) PTF_DECLARE_NC(13)
PTF_DECLARE_NC(14) PTF_DECLARE_NC(15) PTF_DECLARE_NC(16)
#undef PTF_DECLARE_NC

// Used once per NC by the instantiation units.
#define PTF_INSTANTIATE_NC(NC)                                                                                    \
    template cudaError_t launch_plain<NC>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, \
                                          const MLP*, float, float, const Conc*);                                  \
    template cudaError_t launch_many<NC>(const Comp<NC>*, const int32_t*, const WS&, const IO&, int, int, int,     \
                                         cudaStream_t);                                                            \
    template cudaError_t launch_adjoint<NC>(const CompHost&, const AdjIO&, int, cudaStream_t);                     \
    template cudaError_t launch_eos<NC>(const CompHost&, int64_t, const double*, const double*, const double*,      \
                                        double*, double*, int, cudaStream_t);

}  // namespace ptf
