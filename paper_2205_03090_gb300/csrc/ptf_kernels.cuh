// ptf_kernels.cuh -- stage kernels of the plain flash (Sec. 2.2.3 flowchart).
//
// Stages communicate through device-resident index queues (the GPU form of
// the paper's synchronizer and barriers, Sec. 3 and Alg. 1): every kernel
// reads its queue length from device memory, so a whole flash is a fixed
// sequence of launches on one stream with no host synchronisation.
//
//   prep_precheck : per-mixture constants, ln z, d = ln z + ln phi(z), Wilson
//                   K, 3 split-SS iterations (two in FP32, the last and the
//                   tpd tests in FP64) -> STAB or SPLIT queue
//   stab_ss       : one item per (mixture, trial); SS with DEM (Eq.
//                   ss_analyser), FP32 pre-iteration then FP64 -> done or
//                   STAB_TR queue
//   stab_tr       : trust region in beta = 2 sqrt(W) (Appendix B.1)
//   stab_decide   : label, K re-estimate (Sec. 2.2.1) -> SPLIT queue or done
//   split_ss      : SS with DEM and Rachford-Rice (Sec. 2.2.2), FP32
//                   pre-iteration then FP64 -> done or SPLIT_TR queue
//   split_tr      : trust region on G in n^V (Appendix B.2) + Newton polish
//
// The FP32 stages only move the point the FP64 iteration starts from; every
// decision and every stored result is FP64.
//
// All arrays are SoA with the mixture index fastest ([i * n + m]), so a warp
// of consecutive mixtures reads and writes coalesced 256-byte rows.
#pragma once
#include "ptf_device.cuh"
#include "ptf_group.cuh"

namespace ptf {

struct WS {
    int64_t n;  // mixtures in this chunk (stride of every SoA array)
    double *sA, *B, *lnz, *d, *lnK, *theta, *nV;  // [NC n] (theta: [n])
    double* lnW;       // [2 NC n]: trial t, component i at ((t NC + i) n + m)
    double* tm;        // [2 n]
    int32_t* tflag;    // [2 n]: ss iters | tr iters << 8 | used_tr << 16 | maxiter << 17 | nonfinite << 18
    int32_t *q_stab, *q_split, *q_stab_tr, *q_split_tr;
    int32_t* q_sort;   // [n]: the split trust-region queue laid out longest expected runs first
    int32_t* cnt;      // queue counters and read heads (enums below)
    float* nnp = nullptr;  // learned form: classifier logits [n]
    float* nnk = nullptr;  // learned form: initializer ln K [NC n]
    Ctl ctl;               // tolerances and iteration caps of the call
    // learned form: mixtures whose network route the plain method rejected
    // (q_redo, count in cnt[Q_REDO]); q_pre != nullptr makes the precheck
    // take its mixtures from that list instead of 0 .. n-1
    int32_t* q_redo = nullptr;
    const int32_t* q_pre = nullptr;
    unsigned long long* acc = nullptr;  // queue sizes summed over the passes of a call
};

struct IO {
    int64_t ld;  // leading dimension (stride between components) of z, x, y, K
    const double *P, *T, *z;
    int32_t* nphase;
    double *beta, *x, *y, *K;
    int32_t* status;
    int32_t* iters;  // packed: split SS | split TR << 8 | stab SS << 16 | stab TR << 24 (may be null)
};

// ws.cnt slots: append counters of the queues, and read heads of the
// persistent (refill) kernels
// The split queue q_split is filled from both ends: from the front by the
// precheck (or the classifier gate), counter Q_SPLIT; from the back by the
// stability decision, counter Q_SPLIT_B (entry k at n - 1 - k).  The two parts
// do not depend on each other, so their split SS can run concurrently.
enum { Q_STAB = 0, Q_SPLIT = 1, Q_STAB_TR = 2, Q_SPLIT_TR = 3, Q_SPLIT_B = 6 };
// Split trust-region queue order.  A trust-region run is a chain of dependent
// evaluations, each about as long on an otherwise idle SM as on a busy one (an
// FP64 warp instruction occupies the SM's narrow FP64 pipe as long whatever
// the number of active lanes), so a long run that starts late sets the
// kernel's length.  The split SS rates each hand-off by the residual it leaves
// and its last contraction ratio -- runs that leave SS far from convergence,
// or contracting slowly, take the most trust-region steps -- into kTRBuckets
// buckets, and k_tr_order lays the queue out longest expected runs first.
// Only the order of the work changes.  (The same order for the stability
// trust region measured slower: 7.0 -> 7.4 ms at nc = 8, 1e6.)
constexpr int kTRBuckets = 8;
constexpr int QB_SPLIT = 32;  // cnt slots: split items per bucket, then the scatter cursors
__device__ __forceinline__ int tr_bucket(double log10_res, bool slow, double slow_bonus) {
    const double score = log10_res + (slow ? slow_bonus : 0.0);
    return (int)fmin(fmax(floor(-score), 0.0), (double)(kTRBuckets - 1));
}
// Split SS hand-off: contraction ratio above which SS counts as slow.
constexpr double kSlowSS = 0.3;
// ws.tflag bit: a stability item the FP32 pre-iteration handed to the FP64 SS
constexpr int kSSFinish = 1 << 20;
enum { H_PRE = 8, H_STAB = 9, H_STAB_TR = 10, H_SPLIT = 11, H_SPLIT_TR = 12, H_SPLIT_B = 13, H_STAB_FIN = 14,
       H_PRE32 = 15, H_SPLIT32 = 16, H_SPLIT32_B = 17 };
// Every slot but Q_REDO holds one pass's queue counters and read heads; the
// learned form's second pass (over the rejected mixtures) starts them at zero
// again.  Q_REDO counts the rejected mixtures.
constexpr int Q_REDO = 4;
constexpr int kCntSlots = 64;  // the counter block of a workspace

// Fold one pass's four queue counters into the call's accumulator (the split
// queue is counted from both of its ends).
static __global__ void k_fold_counts(const int32_t* cnt, unsigned long long* acc) {
    if (threadIdx.x < 4)
        acc[threadIdx.x] += (unsigned long long)cnt[threadIdx.x] + (threadIdx.x == Q_SPLIT ? cnt[Q_SPLIT_B] : 0);
}

// Component data of a launch.  OneSys: one fluid system, a kernel parameter
// read through the constant bank.  ManySys: several systems of the same nc (a
// batch of uneven systems is grouped by nc), a table in global memory and the
// system of each mixture.
template <int NC>
struct OneSys {
    Comp<NC> c;
    __device__ __forceinline__ const Comp<NC>& of(int64_t) const { return c; }
};
template <int NC>
struct ManySys {
    const Comp<NC>* tab;  // [number of systems]
    const int32_t* sys;   // [n]: system of each mixture
    __device__ __forceinline__ const Comp<NC>& of(int64_t m) const { return tab[__ldg(sys + m)]; }
};

// Warp-aggregated append: every lane of the warp must call it (full mask).
__device__ __forceinline__ void warp_append(int32_t* cnt, int32_t* queue, bool pred, int32_t value) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pred) queue[base + __popc(m & ((1u << lane) - 1u))] = value;
}

// Warp-aggregated append at the back of a queue of capacity cap (entry k at
// cap - 1 - k).  Every lane of the warp must call it.
__device__ __forceinline__ void warp_append_back(int32_t* cnt, int32_t* queue, int64_t cap, bool pred, int32_t value) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pred) queue[cap - 1 - (base + __popc(m & ((1u << lane) - 1u)))] = value;
}

// Refill for persistent kernels: the lanes that need work (need = true) take
// the next positions of a queue whose read head is *head; returns this lane's
// position, or -1 if it needs none or the queue is exhausted.  Every lane of
// the warp must call it.  `drained` (warp-uniform) stops further atomics.
__device__ __forceinline__ int64_t warp_fetch(int32_t* head, bool need, int64_t len, bool& drained,
                                              int* blk_taken = nullptr, int quota = 0) {
    const unsigned m = __ballot_sync(0xffffffffu, need);
    const int lane = threadIdx.x & 31;
    int64_t base = len;
    if (m && !drained) {
        int b = 0;
        if (lane == 0) {
            // a block with a quota stops fetching once its warps took that many items
            if (quota > 0 && atomicAdd(blk_taken, __popc(m)) >= quota) b = -1;
            else b = atomicAdd(head, __popc(m));
        }
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b < 0) {
            drained = true;
        } else {
            base = b;
            if (base + __popc(m) >= len) drained = true;  // this fetch reached the end
        }
    }
    const int64_t pos = base + __popc(m & ((1u << lane) - 1u));
    return (need && pos < len) ? pos : -1;
}

// Loop over items in whole-warp rounds so that queue appends see a converged
// warp: item = round_base + lane, valid = item < len.
#define PTF_WARP_ROUNDS(len, item, valid)                                                              \
    for (int64_t _rb = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)); _rb < (len);          \
         _rb += (int64_t)gridDim.x * blockDim.x)                                                       \
        for (int64_t item = _rb + (threadIdx.x & 31), _once = 1; _once; _once = 0)                     \
            for (bool valid = item < (len); _once; _once = 0)

template <int NC>
__device__ __forceinline__ void load_mix(const WS& ws, int64_t m, Mix<NC>& mx) {
#pragma unroll
    for (int i = 0; i < NC; i++) {
        mx.sA[i] = ws.sA[i * ws.n + m];
        mx.B[i] = ws.B[i * ws.n + m];
    }
}

template <int NC>
__device__ __forceinline__ void write_single(const IO& io, int64_t m, const double* z) {
    const int64_t n = io.ld;
    io.nphase[m] = 1;
    io.beta[m] = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        io.x[i * n + m] = z[i];
        io.y[i * n + m] = z[i];
        io.K[i * n + m] = 1.0;
    }
}

// Two-phase result with canonical labels: y is the lower-density phase.
template <int NC>
__device__ __forceinline__ void write_two(const IO& io, int64_t m, double th, const double* x, const double* y,
                                          double ZL, double ZV) {
    const int64_t n = io.ld;
    const bool swap = ZV < ZL;
    io.nphase[m] = 2;
    io.beta[m] = swap ? 1.0 - th : th;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        double xi = swap ? y[i] : x[i], yi = swap ? x[i] : y[i];
        io.x[i * n + m] = xi;
        io.y[i * n + m] = yi;
        io.K[i * n + m] = yi / xi;
    }
}

// ---------------------------------------------------------------------------
// prep (Appendix A): per-mixture constants, ln z, d = ln z + ln phi(z).
// Uniform work, one thread per mixture.  Non-finite inputs get their final
// outputs here; the stability-only pipeline enqueues every other mixture.
// ---------------------------------------------------------------------------
// Returns 0 done (non-finite), 1 to the stability queue, 2 to the precheck.
template <int NC, bool PRECHECK, class CS>
__device__ __forceinline__ int prep_item(const CS& cs, const WS& ws, const IO& io, int64_t m) {
    const Comp<NC>& cp = cs.of(m);
    const int64_t n = ws.n;
    const double P = io.P[m], T = io.T[m];
    double z[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) z[i] = io.z[i * io.ld + m];
    Mix<NC> mx;
    mix_init<NC>(cp, P, T, mx);
    Phase<NC> pz;
    eos<NC>(cp, mx, z, pz);
    bool finite = true;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double lz = log_fast(z[i]);
        const double d = lz + pz.lnphi[i];
        finite = finite && isfinite(d);
        ws.sA[i * n + m] = mx.sA[i];
        ws.B[i * n + m] = mx.B[i];
        ws.lnz[i * n + m] = lz;
        ws.d[i * n + m] = d;
    }
    if (io.iters) io.iters[m] = 0;
    if (!finite || !(P > 0.0 && T > 0.0)) {
        io.status[m] = ST_NONFINITE;
        if (PRECHECK) {
            write_single<NC>(io, m, z);
        } else {  // stability-only outputs: stable, tm = NaN, K = 1
            io.nphase[m] = 1;
            io.beta[m] = NAN;
#pragma unroll
            for (int i = 0; i < NC; i++) io.K[i * io.ld + m] = 1.0;
        }
        return 0;
    }
    if (!PRECHECK) {
        io.status[m] = ST_STAB_RUN;
        return 1;
    }
    io.status[m] = 0;
    return 2;
}

template <int NC, bool PRECHECK, class CS>
__global__ void __launch_bounds__(128) k_prep(const __grid_constant__ CS cs, WS ws, IO io) {
    PTF_WARP_ROUNDS(ws.n, m, valid) {
        const int route = valid ? prep_item<NC, PRECHECK>(cs, ws, io, m) : 0;
        warp_append(ws.cnt + Q_STAB, ws.q_stab, route == 1, (int32_t)m);
    }
}

// ---------------------------------------------------------------------------
// precheck (Sec. 2.2.3): three split-SS evaluations from Wilson K, then the
// tpd(x), tpd(y), Delta G tests.  One step = one evaluation of one mixture.
//
// The first two evaluations run in FP32 (PrecheckSS32).  Their iterate differs
// from an all-FP64 run's by about 1e-6 in ln K, so every route decision taken
// on it carries a margin that bounds that difference with room to spare (a
// relative 1e-4); a mixture whose decision falls inside the margin redoes all
// three evaluations in FP64 from Wilson K.  The routes are therefore those of
// an all-FP64 precheck.
//
// Rachford-Rice route: the root lies in (0, 1) iff f(0) = sum z_i (K_i - 1) > 0
// and f(1) = sum z_i (1 - 1/K_i) < 0 (f decreases on its window, Appendix C);
// otherwise (theta outside (0, 1), or K not bracketing 1) the mixture goes to
// stability analysis.  Returns +1 root in (0, 1), -1 stability analysis, 0
// within the relative margin `rel` of either sign test.
// ---------------------------------------------------------------------------
// The precheck sends a mixture to stability analysis: the plain route from
// there on (a mixture the classifier called unstable loses its network bits;
// the reject bit of a second-pass mixture stays).
__device__ __forceinline__ void route_to_stability(const IO& io, int64_t m) {
    io.status[m] = (io.status[m] & ST_NN_REJECT) | ST_STAB_RUN;
}

template <int NC, class F>
__device__ __forceinline__ int rr_route(const F* z, const F* K, F rel) {
    F f0 = 0, f1 = 0, s0 = 0, s1 = 0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const F ik = F(1) / K[i];
        f0 += z[i] * (K[i] - F(1));
        f1 += z[i] * (F(1) - ik);
        s0 += z[i] * K[i];
        s1 += z[i] * ik;
    }
    if (f0 < -rel * s0 || f1 > rel * s1) return -1;
    if (f0 > rel * s0 && f1 < -rel * s1) return 1;
    return 0;
}
constexpr float kRouteMargin = 1e-4f;

template <int NC>
struct PrecheckSS {
    int64_t m;
    Mix<NC> mx;
    double z[NC], lnK[NC], th;
    int it;
    bool from32;  // started from the FP32 evaluations

    // Start after the FP32 evaluations (PrecheckSS32, which starts from Wilson
    // K): ln K and theta from the workspace, the last evaluation to go.  A NaN
    // theta marks an FP32 evaluation that was not finite: then all the
    // evaluations run here, from Wilson K, as without the FP32 stage.
    template <class CS>
    __device__ __forceinline__ void begin_finish(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        m = mm;
        load_mix<NC>(ws, m, mx);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            z[i] = io.z[i * io.ld + m];
            lnK[i] = ws.lnK[i * n + m];
        }
        th = ws.theta[m];
        it = kPrecheck - 1;
        from32 = true;
        if (!(th == th)) restart(cs, io);
    }

    // all evaluations in FP64 from Wilson K
    template <class CS>
    __device__ __forceinline__ void restart(const CS& cs, const IO& io) {
        wilson<NC>(cs.of(m), io.P[m], io.T[m], lnK);
        th = 0.5;
        it = 0;
        from32 = false;
    }

    // 0 continue, 1 to the stability queue, 2 to the split queue
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        const int64_t n = ws.n;
        double K[NC], t[NC], x[NC], y[NC];
        Phase<NC> pl, pv;
#pragma unroll
        for (int i = 0; i < NC; i++) K[i] = exp_fast(lnK[i]);
        if (from32 && rr_route<NC, double>(z, K, kRouteMargin) == 0) {  // too close to call on this iterate
            restart(cs, io);
            return 0;
        }
        if (!rachford_rice<NC>(z, K, th, t) || !(th > 0.0 && th < 1.0)) {
            route_to_stability(io, m);
            return 1;
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
            x[i] = z[i] * t[i];
            y[i] = K[i] * x[i];
        }
        eos<NC>(cp, mx, x, pl);
        eos<NC>(cp, mx, y, pv);
        if (++it < kPrecheck) {
#pragma unroll
            for (int i = 0; i < NC; i++) lnK[i] -= lnK[i] + pv.lnphi[i] - pl.lnphi[i];
            return 0;
        }
        // Eq. tpd for the current phases; Delta G = (1-theta) tpd(x) + theta tpd(y).
        // sx, sy: sum c_i |ln c_i + ln phi_i(c) - d_i|, the first-order size of a
        // change of tpd per relative change of the phase compositions.  y = K x,
        // so ln y = ln K + ln x with the ln K these phases came from (one
        // logarithm per component instead of two).
        double tx = 0.0, ty = 0.0, sx = 0.0, sy = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            const double d = ws.d[i * n + m];
            const double lx = log_fast(x[i]);
            const double gx = lx + pl.lnphi[i] - d, gy = (lx + lnK[i]) + pv.lnphi[i] - d;
            tx = fma(x[i], gx, tx);
            ty = fma(y[i], gy, ty);
            sx = fma(x[i], fabs(gx), sx);
            sy = fma(y[i], fabs(gy), sy);
            lnK[i] -= lnK[i] + pv.lnphi[i] - pl.lnphi[i];  // the next K (the split starts from it)
        }
        const double dG = (1.0 - th) * tx + th * ty;
        if (from32) {
            // the tests on an FP32-started iterate must hold with a margin
            const double mx_ = kRouteMargin * (1e-6 + sx), my_ = kRouteMargin * (1e-6 + sy);
            const double mg = (1.0 - th) * mx_ + th * my_;
            const bool neg = tx < -kEpsNeg - mx_ || ty < -kEpsNeg - my_ || dG < -kEpsNeg - mg;
            const bool pos = tx > -kEpsNeg + mx_ && ty > -kEpsNeg + my_ && dG > -kEpsNeg + mg;
            if (!neg && !pos) {
                restart(cs, io);
                return 0;
            }
        }
        if (!(tx < -kEpsNeg || ty < -kEpsNeg || dG < -kEpsNeg)) {
            route_to_stability(io, m);
            return 1;
        }
        io.status[m] |= ST_PRECHECK_UNSTABLE;
        // the split starts from the precheck's K, or from the initializer's
        // (learned form) for a mixture the classifier called unstable
        const bool net = (io.status[m] & ST_NN_INIT) != 0;
#pragma unroll
        for (int i = 0; i < NC; i++)
            ws.lnK[i * n + m] = net ? fmin(fmax((double)ws.nnk[i * n + m], -15.0), 15.0) : lnK[i];
        return 2;
    }
};

// FP32 precheck evaluations (mixed-precision refinement, as the FP32
// stability pre-iteration): all but the last of the kPrecheck evaluations
// from Wilson K, by rachford_rice_f and eos_f.  A Rachford-Rice route that is
// clear by the margin of rr_route sends the mixture to stability analysis
// (theta outside (0, 1) or no root) or on; one inside the margin, or a
// non-finite evaluation, hands the mixture to k_precheck to redo every
// evaluation in FP64.  Otherwise ln K and theta wait in the workspace for
// the last, FP64 evaluation and the tests, which k_precheck takes.
template <int NC>
struct PrecheckSS32 {
    int64_t m;
    float sA[NC], B[NC], z[NC], lnK[NC], th;
    int it;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        m = mm;
        const Comp<NC>& cp = cs.of(m);
        double lk[NC];
        wilson<NC>(cp, io.P[m], io.T[m], lk);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            sA[i] = (float)ws.sA[i * n + m];
            B[i] = (float)ws.B[i * n + m];
            z[i] = (float)io.z[i * io.ld + m];
            lnK[i] = (float)lk[i];
        }
        th = 0.5f;
        it = 0;
    }

    // 0 continue, 1 to the stability queue, 3 waits for the FP64 evaluation
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        const int64_t n = ws.n;
        float K[NC], t[NC], x[NC], y[NC], pl[NC], pv[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) K[i] = __expf(lnK[i]);
        const int route = rr_route<NC, float>(z, K, kRouteMargin);
        if (route == 0) {  // too close to call in FP32: every evaluation in FP64
            ws.theta[m] = NAN;
            return 3;
        }
        if (route < 0) {
            route_to_stability(io, m);
            return 1;
        }
        if (!rachford_rice_f<NC>(z, K, th, t) || !(th > 0.0f && th < 1.0f)) {  // rounding at a clear margin
            ws.theta[m] = NAN;
            return 3;
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
            x[i] = z[i] * t[i];
            y[i] = K[i] * x[i];
        }
        const bool ok = eos_f<NC>(cp, sA, B, x, pl) && eos_f<NC>(cp, sA, B, y, pv);
#pragma unroll
        for (int i = 0; i < NC; i++) lnK[i] = pl[i] - pv[i];
        if (!ok) {  // the FP64 stage redoes every evaluation from Wilson K
            ws.theta[m] = NAN;
            return 3;
        }
        if (++it >= kPrecheck - 1) {  // hand on to the last, FP64 evaluation
#pragma unroll
            for (int i = 0; i < NC; i++) ws.lnK[i * n + m] = (double)lnK[i];
            ws.theta[m] = (double)th;
            return 3;
        }
        return 0;
    }
};

// Mixtures the precheck takes: 0 .. n-1, or the list ws.q_pre (learned form,
// second pass).  Only those not yet routed run it (status 0, or only the
// learned form's bits: unstable by the classifier, or rejected by the judge):
// the others are final (non-finite, stable by the classifier) or routed.
constexpr int kPrecheckBits = ST_NN_REJECT | ST_NN_UNSTABLE | ST_NN_INIT;
__device__ __forceinline__ int64_t precheck_len(const WS& ws) {
    return ws.q_pre ? (int64_t)(*(volatile int32_t*)(ws.cnt + Q_REDO)) : ws.n;
}
__device__ __forceinline__ int64_t precheck_item(const WS& ws, const IO& io, int64_t pos) {
    if (pos < 0) return -1;
    const int64_t m = ws.q_pre ? (int64_t)ws.q_pre[pos] : pos;
    return (io.status[m] & ~kPrecheckBits) == 0 ? m : -1;
}

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_precheck32(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = precheck_len(ws);
    PrecheckSS32<NC> s;
    bool have = false, drained = false;
    for (;;) {
        const int64_t m = precheck_item(ws, io, warp_fetch(ws.cnt + H_PRE32, !have, len, drained));
        if (m >= 0) {
            s.begin(cs, ws, io, m);
            have = true;
        }
        if (!__any_sync(0xffffffffu, have) && drained) break;
        const int r = have ? s.step(cs, ws, io) : 0;
        warp_append(ws.cnt + Q_STAB, ws.q_stab, r == 1, (int32_t)s.m);
        if (r) have = false;
    }
}

// FP64 precheck: the last evaluation and the tests for the mixtures the FP32
// evaluations handed on (status still 0).  Persistent kernel: lanes whose
// mixture finished take the next one.  Three resident blocks per SM (168
// registers, the rest spilled): the extra warps hide more FP64 latency than
// the spills cost (also for split SS and split TR; the stability TR kernel is
// no faster that way).
template <int NC, class CS>
__global__ void __launch_bounds__(128, 3) k_precheck(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = precheck_len(ws);
    PrecheckSS<NC> s;
    bool have = false, drained = false;
    for (;;) {
        // a mixture that is final or routed already is skipped: the lane fetches again next round
        const int64_t m = precheck_item(ws, io, warp_fetch(ws.cnt + H_PRE, !have, len, drained));
        if (m >= 0) {
            s.begin_finish(cs, ws, io, m);
            have = true;
        }
        if (!__any_sync(0xffffffffu, have) && drained) break;
        const int r = have ? s.step(cs, ws, io) : 0;
        warp_append(ws.cnt + Q_STAB, ws.q_stab, r == 1, (int32_t)s.m);
        warp_append(ws.cnt + Q_SPLIT, ws.q_split, r == 2, (int32_t)s.m);
        if (r) have = false;
    }
}

// ---------------------------------------------------------------------------
// Stability trial evaluation (reading R2 of tm): W = exp(lnW), c = W / sum W,
// gt = ln W + ln phi(c) - d, tm = 1 + sum W (gt - 1).
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ bool stab_eval(const Comp<NC>& cp, const Mix<NC>& mx, const double* d, const double* lnW,
                                          double* W, double& Wt, double* c, Phase<NC>& ph, double* gt, double& tm) {
    Wt = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        W[i] = exp_fast(lnW[i]);
        Wt += W[i];
    }
    double inv = 1.0 / Wt;
#pragma unroll
    for (int i = 0; i < NC; i++) c[i] = W[i] * inv;
    eos<NC>(cp, mx, c, ph);
    double t = 1.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        gt[i] = lnW[i] + ph.lnphi[i] - d[i];
        t = fma(W[i], gt[i] - 1.0, t);
    }
    tm = t;
    return isfinite(t);
}

// ---------------------------------------------------------------------------
// Stability SS (Sec. 2.2.1, Eq. ss_analyser) with DEM; item = 2 q + trial.
// One step = one evaluation of one trial.
// ---------------------------------------------------------------------------
template <int NC>
struct StabSS {
    int64_t m, item;
    Mix<NC> mx;
    double d[NC], lnW[NC], dp[NC], dem_f, res_prev, tm;
    int t, it, iters;
    bool dem_pending;

    // Start from the iterate the FP32 pre-iteration (StabSS32, which starts
    // from the trial K) left (flag kSSFinish): the same evaluation count, so
    // the cap counts both.  Returns false if the item is not waiting for FP64.
    template <class CS>
    __device__ __forceinline__ bool begin_finish(const CS& cs, const WS& ws, const IO& io, int64_t it_) {
        const int64_t n = ws.n;
        item = it_;
        m = ws.q_stab[item >> 1];
        t = (int)(item & 1);
        const int32_t f = ws.tflag[t * n + m];
        if (!(f & kSSFinish)) return false;
        load_mix<NC>(ws, m, mx);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            d[i] = ws.d[i * n + m];
            lnW[i] = ws.lnW[(t * NC + i) * n + m];
            dp[i] = 0.0;
        }
        res_prev = INFINITY;
        dem_f = 0.0;
        tm = 0.0;
        iters = f & 0xff;
        it = (f >> 8) & 0xff;
        dem_pending = false;
        return true;
    }

    __device__ __forceinline__ void store(const WS& ws, int flags) {
        const int64_t n = ws.n;
#pragma unroll
        for (int i = 0; i < NC; i++) ws.lnW[(t * NC + i) * n + m] = lnW[i];
        ws.tm[t * n + m] = tm;
        ws.tflag[t * n + m] = iters | flags;
    }

    // 0 continue, 1 done, 2 needs the trust region
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        double W[NC], c[NC], gt[NC], Wt;
        Phase<NC> ph;
        const bool bad = !stab_eval<NC>(cp, mx, d, lnW, W, Wt, c, ph, gt, tm);
        const double res = bad ? INFINITY : maxabs<NC>(gt);
        const int this_it = it++;
        if (dem_pending && (bad || !(res < res_prev))) {  // undo the accelerated update
            dem_pending = false;
#pragma unroll
            for (int i = 0; i < NC; i++) lnW[i] -= dp[i] * dem_f;
            return 0;  // the next step re-evaluates the plain update
        }
        dem_pending = false;
        if (bad) {
            tm = NAN;
            store(ws, 1 << 18);
            return 1;
        }
        if (tm < -kEpsNeg || res < ws.ctl.tol_stab) {
            store(ws, 0);
            return 1;
        }
        if (this_it >= ws.ctl.ss_stab) {
            store(ws, 1 << 16);
            return 2;
        }
        double dk[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dk[i] = -gt[i];
            lnW[i] += dk[i];
        }
        const int s = iters + 1;
        if (s % kDemPeriod == 0) {
            const double f = dem_factor<NC>(dk, dp);
            if (f > 0.0) {
#pragma unroll
                for (int i = 0; i < NC; i++) lnW[i] += dk[i] * f;
                dem_f = f;
                dem_pending = true;
                res_prev = res;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dp[i] = dk[i];
        }
        iters = s;
        return 0;
    }
};

// ---------------------------------------------------------------------------
// FP32 pre-iteration of stability SS (mixed-precision refinement): the same
// SS with DEM from the same start, evaluated by eos_f, until the update falls
// below kSSFinishRes, or tm comes within kSSFinishTm of zero (FP32 rounding
// of tm is about 1e-6), or the iteration cap.  The item then waits for the
// FP64 iteration (kSSFinish), which evaluates the point again and takes every
// decision: convergence, the first negative tm (so the run stops where an
// FP64 run would), the cap.  At the cap the item goes to the trust region as
// in the FP64 iteration.  FP32 operations cost a small fraction of an FP64 one
// here; the FP64 iteration is left a third of the evaluations.
// ---------------------------------------------------------------------------
constexpr float kSSFinishRes = 3e-5f;
constexpr float kSSFinishTm = 3e-6f;

template <int NC>
struct StabSS32 {
    int64_t m, item;
    int t, it, iters;
    bool dem_pending;
    float sA[NC], B[NC], d[NC], lnW[NC], dp[NC], dem_f, res_prev;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t it_) {
        const int64_t n = ws.n;
        item = it_;
        m = ws.q_stab[item >> 1];
        const Comp<NC>& cp = cs.of(m);
        t = (int)(item & 1);
        double lnKw[NC];
        wilson<NC>(cp, io.P[m], io.T[m], lnKw);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            sA[i] = (float)ws.sA[i * n + m];
            B[i] = (float)ws.B[i * n + m];
            d[i] = (float)ws.d[i * n + m];
            const double lz = ws.lnz[i * n + m];
            lnW[i] = (float)(t == 0 ? lz + lnKw[i] : lz - lnKw[i]);
            dp[i] = 0.0f;
        }
        res_prev = INFINITY;
        dem_f = 0.0f;
        it = iters = 0;
        dem_pending = false;
    }

    // hand the current point on: to the FP64 iteration (finish) or the trust region
    __device__ __forceinline__ void store(const WS& ws, int this_it, bool finish) {
        const int64_t n = ws.n;
#pragma unroll
        for (int i = 0; i < NC; i++) ws.lnW[(t * NC + i) * n + m] = (double)lnW[i];
        ws.tm[t * n + m] = 0.0;
        ws.tflag[t * n + m] = finish ? (iters | (this_it << 8) | kSSFinish) : (iters | (1 << 16));
    }

    // 0 continue, 2 needs the trust region, 3 waits for the FP64 iteration
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        float W[NC], c[NC], lnphi[NC], gt[NC], Wt = 0.0f;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            W[i] = __expf(lnW[i]);
            Wt += W[i];
        }
        const float inv = 1.0f / Wt;
#pragma unroll
        for (int i = 0; i < NC; i++) c[i] = W[i] * inv;
        bool ok = eos_f<NC>(cp, sA, B, c, lnphi);
        float tm = 1.0f, res = 0.0f;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            gt[i] = lnW[i] + lnphi[i] - d[i];
            tm = fmaf(W[i], gt[i] - 1.0f, tm);
            res = fmaxf(res, fabsf(gt[i]));
        }
        ok = ok && isfinite(tm) && isfinite(res);
        const int this_it = it++;
        if (dem_pending && (!ok || !(res < res_prev))) {  // undo the accelerated update
            dem_pending = false;
#pragma unroll
            for (int i = 0; i < NC; i++) lnW[i] -= dp[i] * dem_f;
            return 0;
        }
        dem_pending = false;
        if (!ok || res < kSSFinishRes || tm < kSSFinishTm) {
            store(ws, this_it, true);
            return 3;
        }
        if (this_it >= ws.ctl.ss_stab) {
            store(ws, this_it, false);
            return 2;
        }
        float dk[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dk[i] = -gt[i];
            lnW[i] += dk[i];
        }
        const int s = iters + 1;
        if (s % kDemPeriod == 0) {
            const float f = dem_factor_f<NC>(dk, dp);
            if (f > 0.0f) {
#pragma unroll
                for (int i = 0; i < NC; i++) lnW[i] += dk[i] * f;
                dem_f = f;
                dem_pending = true;
                res_prev = res;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) dp[i] = dk[i];
        iters = s;
        return 0;
    }
};

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_stab_ss32(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = 2 * (int64_t)(*(volatile int32_t*)(ws.cnt + Q_STAB));
    StabSS32<NC> s;
    bool have = false, drained = false;
    for (;;) {
        const int64_t pos = warp_fetch(ws.cnt + H_STAB, !have, len, drained);
        if (pos >= 0) {
            s.begin(cs, ws, io, pos);
            have = true;
        }
        if (!__any_sync(0xffffffffu, have)) break;
        const int r = have ? s.step(cs, ws, io) : 0;
        warp_append(ws.cnt + Q_STAB_TR, ws.q_stab_tr, r == 2, (int32_t)s.item);
        if (r) have = false;
    }
}

// FP64 stability SS: finishes the items the FP32 pre-iteration handed on
// (kSSFinish); the others are done or wait for the trust region.
template <int NC, class CS>
__global__ void __launch_bounds__(128) k_stab_ss(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = 2 * (int64_t)(*(volatile int32_t*)(ws.cnt + Q_STAB));
    StabSS<NC> s;
    bool have = false, drained = false;
    for (;;) {
        const int64_t pos = warp_fetch(ws.cnt + H_STAB_FIN, !have, len, drained);
        if (pos >= 0) have = s.begin_finish(cs, ws, io, pos);
        if (!__any_sync(0xffffffffu, have) && drained) break;
        const int r = have ? s.step(cs, ws, io) : 0;
        warp_append(ws.cnt + Q_STAB_TR, ws.q_stab_tr, r == 2, (int32_t)s.item);
        if (r) have = false;
    }
}

// ---------------------------------------------------------------------------
// Stability trust region (Appendix B.1, Eqs. tr_sa, analysis_grad/hess).
// ---------------------------------------------------------------------------
template <int NC>
struct StabPt {
    double lnW[NC], gt[NC], g[NC], tm;
    double H[NC * (NC + 1) / 2];
};

// One entry of the stability Hessian, H_ij = (sqrt(W_i) / sum W) sqrt(W_j)
// J_ij, plus 1 + gt_i / 2 on the diagonal; explicit, so that the one-lane
// and the several-lanes-per-run evaluations round alike.
__device__ __forceinline__ double stab_hs(bool diag, double ri, double sWj, double Jij, double gti) {
    const double rj = mul_rn<double>(ri, sWj);
    return diag ? fma(rj, Jij, fma(0.5, gti, 1.0)) : mul_rn<double>(rj, Jij);
}

// sWin (optional): sqrt(W_i) of the point, when the caller has it (a trust-
// region trial point beta + u gives it without an exponential); else from
// ln W.  W = sqrt(W)^2, so no square root is taken either way.
template <int NC>
__device__ __forceinline__ bool stab_point(const Comp<NC>& cp, const Mix<NC>& mx, const double* d, StabPt<NC>& p,
                                           const double* sWin = nullptr) {
    double sW[NC], W[NC], c[NC], Wt = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        sW[i] = sWin ? sWin[i] : exp_fast(0.5 * p.lnW[i]);
        W[i] = mul_rn<double>(sW[i], sW[i]);
        Wt = add_rn<double>(Wt, W[i]);
    }
    const double inv = 1.0 / Wt;
#pragma unroll
    for (int i = 0; i < NC; i++) c[i] = W[i] * inv;
    Phase<NC> ph;
    eos<NC>(cp, mx, c, ph);
    double t = 1.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        p.gt[i] = p.lnW[i] + ph.lnphi[i] - d[i];
        t = fma(W[i], p.gt[i] - 1.0, t);
    }
    p.tm = t;
    if (!isfinite(t)) return false;
    // H_ij = sqrt(W_i W_j) J_ij / sum W + delta_ij (1 + gt_i / 2)
    double J[NC * (NC + 1) / 2];
    dlnphi_dn_r<NC, double>(cp, mx, ph, J);
#pragma unroll
    for (int i = 0; i < NC; i++) p.g[i] = sW[i] * p.gt[i];
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double ri = sW[i] * inv;
#pragma unroll
        for (int j = 0; j <= i; j++) p.H[tri(i, j)] = stab_hs(i == j, ri, sW[j], J[tri(i, j)], p.gt[i]);
    }
    return true;
}

// One step = one factorisation of the subproblem and, once its step is known,
// one evaluation (EOS and d ln phi / dn) of the trial point; the start point
// is evaluated on the first step.  The tests that end a run follow the
// evaluation, so a lane that finishes takes a new item on the next trip.
template <int NC>
struct StabTR {
    int64_t m, item;
    int t, it, iters, phase, idle;  // phase 0: evaluate the start point; 1: iterate; idle: trips without evaluation
    int32_t fl;
    Mix<NC> mx;
    double d[NC], beta[NC], radius, eta_lo;
    TRShift sh;
    StabPt<NC> cur;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t it_) {
        const int64_t n = ws.n;
        item = it_;
        m = ws.q_stab[item >> 1];
        const Comp<NC>& cp = cs.of(m);
        t = (int)(item & 1);
        load_mix<NC>(ws, m, mx);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            d[i] = ws.d[i * n + m];
            cur.lnW[i] = ws.lnW[(t * NC + i) * n + m];
        }
        fl = ws.tflag[t * n + m];
        it = iters = phase = idle = 0;
        radius = -1.0;
        eta_lo = 0.0;
        sh.active = 0;
        sh.warm = 0.0;
    }

    __device__ __forceinline__ void store(const WS& ws, int maxiter, int nonfinite) {
        const int64_t n = ws.n;
#pragma unroll
        for (int i = 0; i < NC; i++) ws.lnW[(t * NC + i) * n + m] = cur.lnW[i];
        ws.tm[t * n + m] = nonfinite ? NAN : cur.tm;
        ws.tflag[t * n + m] = (fl & 0xff) | (iters << 8) | (1 << 16) | (maxiter << 17) | (nonfinite << 18);
    }

    // 0 continue, 1 done.  tail: the queue is exhausted, so the lane runs the
    // whole shift iteration in this trip (the same iterates either way).
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io, bool tail) {
        const Comp<NC>& cp = cs.of(m);
        StabPt<NC> nxt;
        double u[NC], sWn[NC], pred = 0.0;
        if (phase == 0) {
#pragma unroll
            for (int i = 0; i < NC; i++) nxt.lnW[i] = cur.lnW[i];
        } else {
            double Lf[NC * (NC + 1) / 2];
            // one shift per trip while the queue lasts: few stability solves
            // need more than one, and those lanes skip this trip's evaluation
            // instead of holding the warp.  Once it is exhausted the slowest
            // runs set the kernel's length, and a lane takes all its shifts.
            int r = 0;
#pragma unroll 1
            for (int k = 0; k < (tail ? kTRShiftCap + 2 : 1) && r == 0; k++)
                r = tr_shift_step<NC, double>(cur.H, cur.g, radius, eta_lo, false, sh, Lf, u);
            if (r == 0) {
                // a solve takes at most kTRShiftCap + 3 calls; the budget bounds a run whatever happens
                if (++idle > (ws.ctl.tr_stab + 2) * (kTRShiftCap + 3)) {
                    store(ws, 1, 0);
                    return 1;
                }
                return 0;
            }
            if (r < 0) {  // the solve failed (a model that is not finite): stop at the current point
                store(ws, 1, 0);
                return 1;
            }
            for (int i = 0; i < NC; i++) {
                double hd = 0.0;
                for (int j = 0; j < NC; j++) hd = fma(cur.H[i >= j ? tri(i, j) : tri(j, i)], u[j], hd);
                pred = fma(cur.g[i], u[i], fma(0.5 * u[i], hd, pred));
            }
#pragma unroll
            for (int i = 0; i < NC; i++) {
                sWn[i] = 0.5 * fabs(beta[i] + u[i]);
                nxt.lnW[i] = 2.0 * log_fast(sWn[i]);
            }
        }
        const bool ok = stab_point<NC>(cp, mx, d, nxt, phase == 0 ? nullptr : sWn);
        if (phase == 0) {
            if (!ok) {
                store(ws, 0, 1);
                return 1;
            }
            cur = nxt;
#pragma unroll
            for (int i = 0; i < NC; i++) beta[i] = 2.0 * exp_fast(0.5 * cur.lnW[i]);
            phase = 1;
        } else {
            const bool trusted = fabs(pred) > kPredTrust * (1.0 + fabs(cur.tm));
            const double rho = !ok ? -1.0 : (trusted ? (nxt.tm - cur.tm) / pred : 0.5);
            if (rho > 0.0) {
#pragma unroll
                for (int i = 0; i < NC; i++) beta[i] = fabs(beta[i] + u[i]);
                cur = nxt;
                eta_lo = 0.0;
            } else {
                eta_lo = sh.eta;  // same H, smaller radius: the shift can only grow
            }
            if (rho <= 0.25) radius *= 0.5;
            else if (rho >= 0.75) radius *= 2.0;
            iters = ++it;
        }
        if (cur.tm < -kEpsNeg || maxabs<NC>(cur.g) < ws.ctl.tol_stab) {
            store(ws, 0, 0);
            return 1;
        }
        if (it >= ws.ctl.tr_stab) {
            store(ws, 1, 0);
            return 1;
        }
        return 0;
    }
};

// ---------------------------------------------------------------------------
// The stability trust region with G lanes per run (lane r: component r):
// StabTR::step operation for operation (the whole shift iteration in one
// trip, as StabTR does once its queue has drained).
// ---------------------------------------------------------------------------
template <int NC, int G>
struct StabTRG {
    static constexpr int kHead = H_STAB_TR;
    int64_t m, item;
    int t, it, iters, phase, idle;
    int32_t fl;
    double kkr[NC];                 // row r of 1 - k_ij
    double sA, Bi, d, beta;         // component r
    double radius, eta_lo;
    TRShift sh;
    double lnW, gt, g, tm;          // current point: component r, and tm
    double H[NC];                   // row r of the Hessian

    template <class CS>
    __device__ __forceinline__ void load_kk(const Grp& gr, const CS& cs) {
        const Comp<NC>& cp = cs.of(m);
        const int rr = gr.r < NC ? gr.r : 0;
#pragma unroll
        for (int j = 0; j < NC; j++) kkr[j] = cp.kk[rr * NC + j];
    }

    // a fresh run: queue position pos (as StabTR::begin)
    template <class CS>
    __device__ __forceinline__ void begin_pos(const Grp& gr, const CS& cs, const WS& ws, const IO&, int64_t pos) {
        const int64_t n = ws.n;
        const int rr = gr.r < NC ? gr.r : 0;
        item = ws.q_stab_tr[pos];
        m = ws.q_stab[item >> 1];
        t = (int)(item & 1);
        load_kk(gr, cs);
        sA = ws.sA[rr * n + m];
        Bi = ws.B[rr * n + m];
        d = ws.d[rr * n + m];
        lnW = ws.lnW[(t * NC + rr) * n + m];
        fl = ws.tflag[t * n + m];
        it = iters = phase = idle = 0;
        radius = -1.0;
        eta_lo = 0.0;
        sh.active = 0;
        sh.warm = 0.0;
    }

    // the run that lane src of the warp holds in its one-lane state s
    // (every lane of the warp calls this: full-warp shuffles)
    __device__ __forceinline__ void take_state(const Grp& gr, const StabTR<NC>& s, int src) {
        constexpr unsigned F = 0xffffffffu;
        const int rr = gr.r < NC ? gr.r : 0;
        m = __shfl_sync(F, s.m, src);
        item = __shfl_sync(F, s.item, src);
        t = __shfl_sync(F, s.t, src);
        it = __shfl_sync(F, s.it, src);
        iters = __shfl_sync(F, s.iters, src);
        phase = __shfl_sync(F, s.phase, src);
        idle = __shfl_sync(F, s.idle, src);
        fl = __shfl_sync(F, s.fl, src);
        radius = __shfl_sync(F, s.radius, src);
        eta_lo = __shfl_sync(F, s.eta_lo, src);
        sh.eta = __shfl_sync(F, s.sh.eta, src);
        sh.elo = __shfl_sync(F, s.sh.elo, src);
        sh.ehi = __shfl_sync(F, s.sh.ehi, src);
        sh.active = __shfl_sync(F, s.sh.active, src);
        sh.it = __shfl_sync(F, s.sh.it, src);
        sh.warm = __shfl_sync(F, s.sh.warm, src);
        sh.zero = __shfl_sync(F, s.sh.zero, src);
        tm = __shfl_sync(F, s.cur.tm, src);
#pragma unroll
        for (int k = 0; k < NC; k++) {
            const double a1 = __shfl_sync(F, s.mx.sA[k], src), a2 = __shfl_sync(F, s.mx.B[k], src);
            const double a3 = __shfl_sync(F, s.d[k], src), a4 = __shfl_sync(F, s.beta[k], src);
            const double a5 = __shfl_sync(F, s.cur.lnW[k], src), a6 = __shfl_sync(F, s.cur.gt[k], src);
            const double a7 = __shfl_sync(F, s.cur.g[k], src);
            if (rr == k) {
                sA = a1;
                Bi = a2;
                d = a3;
                beta = a4;
                lnW = a5;
                gt = a6;
                g = a7;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
#pragma unroll
            for (int j = 0; j <= i; j++) {
                const double v = __shfl_sync(F, s.cur.H[tri(i, j)], src);
                if (rr == i) H[j] = v;
                if (rr == j) H[i] = v;
            }
        }
    }

    // as StabTR::store
    __device__ __forceinline__ void store(const Grp& gr, const WS& ws, int maxiter, int nonfinite) {
        const int64_t n = ws.n;
        if (gr.r < NC) ws.lnW[(t * NC + gr.r) * n + m] = lnW;
        if (gr.r == 0) {
            ws.tm[t * n + m] = nonfinite ? NAN : tm;
            ws.tflag[t * n + m] = (fl & 0xff) | (iters << 8) | (1 << 16) | (maxiter << 17) | (nonfinite << 18);
        }
    }

    // as stab_point at component r's ln W_r (sWin: sqrt(W_r) when the caller has it)
    struct Pt {
        double lnW, gt, g, tm;
        double H[NC];
    };
    __device__ __forceinline__ bool point(const Grp& gr, Pt& p, bool have_sW, double sWin) const {
        const double sW = have_sW ? sWin : exp_fast(0.5 * p.lnW);
        const double W = mul_rn<double>(sW, sW);
        double Wt = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++) Wt = add_rn<double>(Wt, gat<G>(gr, W, i));
        const double inv = 1.0 / Wt;
        const double c = W * inv;
        PhaseG ph;
        eos_g<NC, G>(gr, kkr, sA, Bi, c, ph);
        p.gt = p.lnW + ph.lnphi - d;
        double tt = 1.0;
#pragma unroll
        for (int i = 0; i < NC; i++) tt = fma(gat<G>(gr, W, i), gat<G>(gr, p.gt, i) - 1.0, tt);
        p.tm = tt;
        if (!isfinite(tt)) return false;
        double J[NC];
        dlnphi_dn_g<NC, G>(gr, kkr, sA, Bi, ph, J);
        p.g = sW * p.gt;
        const double ri = sW * inv;
#pragma unroll
        for (int j = 0; j < NC; j++) {
            const double sWj = gat<G>(gr, sW, j);
            if (j <= gr.r) p.H[j] = stab_hs(j == gr.r, ri, sWj, J[j], p.gt);
        }
        sym_fill<NC, G>(gr, p.H);
        return true;
    }

    // as StabTR::step with tail = true
    template <class CS>
    __device__ __forceinline__ int step(const Grp& gr, const CS&, const WS& ws, const IO&) {
        Pt nxt;
        double u = 0.0, sWn = 0.0, pred = 0.0;
        if (phase == 0) {
            nxt.lnW = lnW;
        } else {
            double a[NC];
            int r = 0;
#pragma unroll 1
            for (int k = 0; k < kTRShiftCap + 2 && r == 0; k++)
                r = tr_shift_step_g<NC, G>(gr, H, g, radius, eta_lo, false, sh, a, u);
            if (r == 0) {
                if (++idle > (ws.ctl.tr_stab + 2) * (kTRShiftCap + 3)) {
                    store(gr, ws, 1, 0);
                    return 1;
                }
                return 0;
            }
            if (r < 0) {
                store(gr, ws, 1, 0);
                return 1;
            }
            double hd = 0.0;
#pragma unroll
            for (int j = 0; j < NC; j++) hd = fma(H[j], gat<G>(gr, u, j), hd);
#pragma unroll
            for (int i = 0; i < NC; i++) {
                const double ui = gat<G>(gr, u, i);
                pred = fma(gat<G>(gr, g, i), ui, fma(0.5 * ui, gat<G>(gr, hd, i), pred));
            }
            sWn = 0.5 * fabs(beta + u);
            nxt.lnW = 2.0 * log_fast(sWn);
        }
        const bool ok = point(gr, nxt, phase != 0, sWn);
        if (phase == 0) {
            if (!ok) {
                store(gr, ws, 0, 1);
                return 1;
            }
            lnW = nxt.lnW;
            gt = nxt.gt;
            g = nxt.g;
            tm = nxt.tm;
#pragma unroll
            for (int j = 0; j < NC; j++) H[j] = nxt.H[j];
            beta = 2.0 * exp_fast(0.5 * lnW);
            phase = 1;
        } else {
            const bool trusted = fabs(pred) > kPredTrust * (1.0 + fabs(tm));
            const double rho = !ok ? -1.0 : (trusted ? (nxt.tm - tm) / pred : 0.5);
            if (rho > 0.0) {
                beta = fabs(beta + u);
                lnW = nxt.lnW;
                gt = nxt.gt;
                g = nxt.g;
                tm = nxt.tm;
#pragma unroll
                for (int j = 0; j < NC; j++) H[j] = nxt.H[j];
                eta_lo = 0.0;
            } else {
                eta_lo = sh.eta;
            }
            if (rho <= 0.25) radius *= 0.5;
            else if (rho >= 0.75) radius *= 2.0;
            iters = ++it;
        }
        if (tm < -kEpsNeg || gmaxabs<NC, G>(gr, g) < ws.ctl.tol_stab) {
            store(gr, ws, 0, 0);
            return 1;
        }
        if (it >= ws.ctl.tr_stab) {
            store(gr, ws, 1, 0);
            return 1;
        }
        return 0;
    }
};

// Trust-region runs with G lanes each (RunG: SplitTRG or StabTRG; Run: the
// one-lane state of the same kind).  `pending` lists the warp's lanes whose
// runs are still to be taken: each group that has no run takes the next of
// them (lowest lane first), the rest stay parked in their lanes until a
// group is free.  With refill, a free group takes the next run of the queue
// instead.  Every lane of the warp calls this.
template <class RunG, int G, class Run, class CS>
__device__ __noinline__ void tr_groups(const CS& cs, const WS& ws, const IO& io, const Run& s, unsigned pending,
                                          bool refill, int64_t len) {
    constexpr unsigned F = 0xffffffffu;
    const Grp g = make_grp<G>();
    const int lane = threadIdx.x & 31, q = lane / G;
    RunG t;
    bool ghave = false, gdrained = !refill;
    for (;;) {
        const unsigned idle = __ballot_sync(F, !ghave && g.r == 0);  // leader lanes of the free groups
        if (pending && idle) {
            // the k-th free group (by lane) takes the k-th lowest pending lane's run
            const bool free = (idle >> (q * G)) & 1u;
            const int k = __popc(idle & ((1u << (q * G)) - 1u));
            unsigned pm = pending;
            for (int i = 0; i < k && pm; i++) pm &= pm - 1;
            const bool gets = free && pm != 0;
            const int src = gets ? __ffs(pm) - 1 : lane;
            RunG tk;
            tk.take_state(g, s, src);  // full-warp shuffles
            if (gets) {
                t = tk;
                t.load_kk(g, cs);
                ghave = true;
            }
            const int taken = min(__popc(idle), __popc(pending));
            for (int i = 0; i < taken; i++) pending &= pending - 1;
        }
        if (!ghave && !gdrained) {
            int pos = 0;
            if (g.r == 0) pos = atomicAdd(ws.cnt + RunG::kHead, 1);
            pos = __shfl_sync(g.mask, pos, 0, G);
            if (pos < len) {
                t.begin_pos(g, cs, ws, io, pos);
                ghave = true;
            } else {
                gdrained = true;
            }
        }
        if (!__any_sync(F, ghave) && !pending) break;
        if (ghave && t.step(g, cs, ws, io)) ghave = false;
    }
}

// One lane per run while the queue lasts; once this warp's fetch has found
// it drained and at most kGroupSwitch runs are left, G lanes per run, 32 / G
// runs at a time (same results, shorter trips: see ptf_group.cuh).
// ws.ctl.tr_coop 1: one lane throughout; 2: G lanes throughout.  A group trip
// takes about half as long as a one-lane trip but costs 1.6x its FP64 work
// per run, so groups pay only once the queue has drained; switching at 8 runs
// left measured best (4 and 16 within 0.3 ms of it, 32 slower).
constexpr int kGroupSwitch = 8;

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_stab_tr(const __grid_constant__ CS cs, WS ws, IO io) {
    constexpr int G = GroupLanes<NC>::G;
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_STAB_TR);
    StabTR<NC> s;
    bool have = false, drained = false;
    if constexpr (GroupLanes<NC>::ok) {
        if (ws.ctl.tr_coop == 2) {
            tr_groups<StabTRG<NC, G>, G>(cs, ws, io, s, 0u, true, len);
            return;
        }
    }
    for (;;) {
        const int64_t pos = warp_fetch(ws.cnt + H_STAB_TR, !have, len, drained);
        if (pos >= 0) {
            s.begin(cs, ws, io, ws.q_stab_tr[pos]);
            have = true;
        }
        const unsigned live = __ballot_sync(0xffffffffu, have);
        if (!live) break;
        if constexpr (GroupLanes<NC>::ok) {
            if (drained && ws.ctl.tr_coop == 0 && __popc(live) <= kGroupSwitch) {
                tr_groups<StabTRG<NC, G>, G>(cs, ws, io, s, live, false, len);
                break;
            }
        }
        if (have && s.step(cs, ws, io, drained)) have = false;
    }
}

// K from the stability trial t with the lower tm (Sec. 2.2.1, last sentence;
// reading R16), w = W / sum W the trial composition: ln K = ln w - ln z for
// the vapour-like trial (t = 0), ln z - ln w for the liquid-like one.
template <int NC>
__device__ __forceinline__ void stab_lnK(const WS& ws, int64_t m, int t, double* lnK) {
    const int64_t n = ws.n;
    double lw[NC], sw = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        lw[i] = ws.lnW[(t * NC + i) * n + m];
        sw += exp_fast(lw[i]);
    }
    const double ls = log(sw);
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double lz = ws.lnz[i * n + m];
        lnK[i] = t == 1 ? lz - (lw[i] - ls) : (lw[i] - ls) - lz;
    }
}

// ---------------------------------------------------------------------------
// Stability decision and K re-estimate (Sec. 2.2.1, last sentence).
// ---------------------------------------------------------------------------
// Returns true if the mixture goes to the split queue.
template <int NC, class CS>
__device__ __forceinline__ bool stab_decide_item(const CS& cs, const WS& ws, const IO& io, int64_t m) {
    const Comp<NC>& cp = cs.of(m);
    const int64_t n = ws.n;
    bool to_split = false;
    {
        {
            const double tv = ws.tm[m], tl = ws.tm[n + m];
            const int32_t fv = ws.tflag[m], fl = ws.tflag[n + m];
            int32_t st = io.status[m];
            if ((fv | fl) & (1 << 16)) st |= ST_STAB_TR;
            if ((fv | fl) & (1 << 17)) st |= ST_MAXITER;
            if (io.iters)
                io.iters[m] = ((((fv & 0xff) + (fl & 0xff)) & 0xff) << 16) |
                              (((((fv >> 8) & 0xff) + ((fl >> 8) & 0xff)) & 0xff) << 24);
            double z[NC];
#pragma unroll
            for (int i = 0; i < NC; i++) z[i] = io.z[i * io.ld + m];
            if ((fv | fl) & (1 << 18)) {
                st |= ST_NONFINITE;
                write_single<NC>(io, m, z);
            } else {
                double tmin = tv < tl ? tv : tl;
                if (!(tmin < -kEpsNeg)) {
                    write_single<NC>(io, m, z);
                } else {
                    double lnK[NC];
                    stab_lnK<NC>(ws, m, tl < tv ? 1 : 0, lnK);
#pragma unroll
                    for (int i = 0; i < NC; i++) ws.lnK[i * n + m] = lnK[i];
                    to_split = true;
                }
            }
            io.status[m] = st;
        }
    }
    return to_split;
}

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_stab_decide(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_STAB);
    PTF_WARP_ROUNDS(len, qi, valid) {
        const int64_t m = valid ? ws.q_stab[qi] : 0;
        const bool to_split = valid ? stab_decide_item<NC>(cs, ws, io, m) : false;
        warp_append_back(ws.cnt + Q_SPLIT_B, ws.q_split, ws.n, to_split, (int32_t)m);
    }
}

// ---------------------------------------------------------------------------
// Phase-split SS (Sec. 2.2.2) with DEM, convergence at the fugacity residual.
// One step = one evaluation (Rachford-Rice, both phases) of one mixture.
// ---------------------------------------------------------------------------
template <int NC>
struct SplitSS {
    int64_t m;
    Mix<NC> mx;
    double z[NC], lnK[NC], dp[NC], dem_f, res_prev, th;
    int it, iters, bucket;
    bool dem_pending, slow_hint;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        m = mm;
        const Comp<NC>& cp = cs.of(m);
        load_mix<NC>(ws, m, mx);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            z[i] = io.z[i * io.ld + m];
            lnK[i] = ws.lnK[i * n + m];
            dp[i] = 0.0;
        }
        slow_hint = false;
        th = 0.5;
        res_prev = INFINITY;
        dem_f = 0.0;
        it = iters = 0;
        dem_pending = false;
    }

    // Continue from the point the FP32 pre-iteration (SplitSS32) left: ln K,
    // theta and the counts from the workspace; that point is evaluated again.
    template <class CS>
    __device__ __forceinline__ void begin_finish(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        begin(cs, ws, io, mm);
        th = ws.theta[m];
        const int32_t f = ws.tflag[m];
        iters = f & 0xff;
        it = (f >> 8) & 0xff;
        slow_hint = (f >> 16) & 1;
#pragma unroll
        for (int i = 0; i < NC; i++) dp[i] = ws.nV[i * ws.n + m];
    }

    __device__ __forceinline__ void finish(const IO& io, int32_t add_status) {
        io.status[m] |= add_status;
        if (io.iters) io.iters[m] = (io.iters[m] & ~0xff) | (iters & 0xff);
    }

    // 0 continue, 1 done, 2 needs the trust region (order bucket in `bucket`)
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        const int64_t n = ws.n;
        double K[NC], t[NC], x[NC], y[NC], gt[NC];
        Phase<NC> pl, pv;
        int fail = 0;  // 1 collapse (trivial K / no Rachford-Rice root), 2 non-finite
        double res = INFINITY;
        if (maxabs<NC>(lnK) < kTrivialLnK) fail = 1;
        if (!fail) {
#pragma unroll
            for (int i = 0; i < NC; i++) K[i] = exp_fast(lnK[i]);
            if (!rachford_rice<NC>(z, K, th, t)) fail = 1;
        }
        if (!fail) {
#pragma unroll
            for (int i = 0; i < NC; i++) {
                x[i] = z[i] * t[i];
                y[i] = K[i] * x[i];
            }
            eos<NC>(cp, mx, x, pl);
            eos<NC>(cp, mx, y, pv);
#pragma unroll
            for (int i = 0; i < NC; i++) gt[i] = lnK[i] + pv.lnphi[i] - pl.lnphi[i];
            res = maxabs<NC>(gt);
            if (!(res < INFINITY)) fail = 2;
        }
        const int this_it = it++;
        if (dem_pending && (fail || !(res < res_prev))) {  // undo the accelerated update
            dem_pending = false;
#pragma unroll
            for (int i = 0; i < NC; i++) lnK[i] -= dp[i] * dem_f;
            return 0;  // the next step re-evaluates the plain update
        }
        dem_pending = false;
        if (fail == 1) {
            finish(io, ST_COLLAPSE);
            write_single<NC>(io, m, z);
            return 1;
        }
        if (fail == 2) {
            finish(io, ST_NONFINITE);
            write_single<NC>(io, m, z);
            return 1;
        }
        if (fail == 0 && res <= ws.ctl.tol_fug) {
            if (th > 0.0 && th < 1.0) {
                finish(io, 0);
                write_two<NC>(io, m, th, x, y, pl.Z, pv.Z);
            } else {
                finish(io, ST_COLLAPSE);
                write_single<NC>(io, m, z);
            }
            return 1;
        }
        if (this_it >= ws.ctl.ss_split) {
            // trust-region start: the last evaluated SS point, or the
            // material-balance point at theta = 1/2 for a negative flash
            const bool inside = th > 0.0 && th < 1.0;
#pragma unroll
            for (int i = 0; i < NC; i++)
                ws.nV[i * n + m] = inside ? th * y[i] : 0.5 * K[i] * z[i] / (1.0 + 0.5 * (K[i] - 1.0));
            finish(io, ST_SPLIT_TR);
            const double dpm = maxabs<NC>(dp);  // 0 when this iteration took no update yet
            const bool slow = dpm > 0.0 ? res > kSlowSS * dpm : slow_hint;
            // expected length: about one more trust-region step per decade of
            // residual, and several more when SS contracted slowly
            bucket = tr_bucket(log_fast(res) * 0.4342944819032518, slow, 3.0);
            return 2;
        }
        double dk[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dk[i] = -gt[i];
            lnK[i] += dk[i];
        }
        const int s = iters + 1;
        if (s % kDemPeriod == 0) {
            const double f = dem_factor<NC>(dk, dp);
            if (f > 0.0) {
#pragma unroll
                for (int i = 0; i < NC; i++) lnK[i] += dk[i] * f;
                dem_f = f;
                dem_pending = true;
                res_prev = res;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dp[i] = dk[i];
        }
        iters = s;
        return 0;
    }
};

// ---------------------------------------------------------------------------
// FP32 pre-iteration of the phase-split SS (mixed-precision refinement, as
// for stability analysis): the same SS with DEM from the same K, evaluated by
// rachford_rice_f and eos_f, until the update falls below kSplitFinishRes or
// the cap; then, and for every case that needs a decision (no Rachford-Rice
// root, K near 1, a non-finite point), the FP64 iteration evaluates the point
// again and continues: convergence to the fugacity residual, collapse, the
// trust-region hand-off and every output are FP64.
// ---------------------------------------------------------------------------
constexpr float kSplitFinishRes = 1e-5f;

template <int NC>
struct SplitSS32 {
    int64_t m;
    float sA[NC], B[NC], z[NC], lnK[NC], dp[NC], dem_f, res_prev, th;
    int it, iters;
    bool dem_pending;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        m = mm;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            sA[i] = (float)ws.sA[i * n + m];
            B[i] = (float)ws.B[i * n + m];
            z[i] = (float)io.z[i * io.ld + m];
            lnK[i] = (float)ws.lnK[i * n + m];
            dp[i] = 0.0f;
        }
        th = 0.5f;
        res_prev = INFINITY;
        dem_f = 0.0f;
        it = iters = 0;
        dem_pending = false;
    }

    // hand the current point to the FP64 iteration, with the last update (in
    // ws.nV, free until the trust-region hand-off; DEM continues from it) and
    // the split TR queue order hint (kSlowSS) in case the FP64 iteration takes
    // no update before the trust region
    __device__ __forceinline__ int hand_on(const WS& ws, int this_it, bool slow) {
        const int64_t n = ws.n;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            ws.lnK[i * n + m] = (double)lnK[i];
            ws.nV[i * n + m] = (double)dp[i];
        }
        ws.theta[m] = (double)th;
        ws.tflag[m] = iters | (this_it << 8) | (slow ? 1 << 16 : 0);
        return 3;
    }

    // 0 continue, 3 waits for the FP64 iteration
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        float K[NC], t[NC], x[NC], y[NC], pl[NC], pv[NC], gt[NC];
        float kmx = 0.0f;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            K[i] = __expf(lnK[i]);
            kmx = fmaxf(kmx, fabsf(lnK[i]));
        }
        const int this_it = it++;
        const float th0 = th;
        bool ok = kmx > 1e-4f && rachford_rice_f<NC>(z, K, th, t);
        float res = INFINITY;
        if (ok) {
#pragma unroll
            for (int i = 0; i < NC; i++) {
                x[i] = z[i] * t[i];
                y[i] = K[i] * x[i];
            }
            ok = eos_f<NC>(cp, sA, B, x, pl) && eos_f<NC>(cp, sA, B, y, pv);
            res = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; i++) {
                gt[i] = lnK[i] + pv[i] - pl[i];
                res = fmaxf(res, fabsf(gt[i]));
            }
            ok = ok && res < INFINITY;
        }
        if (dem_pending && (!ok || !(res < res_prev))) {  // undo the accelerated update
            dem_pending = false;
#pragma unroll
            for (int i = 0; i < NC; i++) lnK[i] -= dp[i] * dem_f;
            return 0;
        }
        dem_pending = false;
        if (!ok) {
            th = th0;
            return hand_on(ws, this_it, false);
        }
        if (res < kSplitFinishRes || this_it >= ws.ctl.ss_split) {
            float dpm = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; i++) dpm = fmaxf(dpm, fabsf(dp[i]));
            return hand_on(ws, this_it, res > (float)kSlowSS * dpm);
        }
        float dk[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) {
            dk[i] = -gt[i];
            lnK[i] += dk[i];
        }
        const int s = iters + 1;
        if (s % kDemPeriod == 0) {
            const float f = dem_factor_f<NC>(dk, dp);
            if (f > 0.0f) {
#pragma unroll
                for (int i = 0; i < NC; i++) lnK[i] += dk[i] * f;
                dem_f = f;
                dem_pending = true;
                res_prev = res;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) dp[i] = dk[i];
        iters = s;
        return 0;
    }
};

// part and quota as in k_split_ss
template <int NC, class CS>
__global__ void __launch_bounds__(128) k_split_ss32(const __grid_constant__ CS cs, WS ws, IO io, int part, int quota) {
    const int64_t na = *(volatile int32_t*)(ws.cnt + Q_SPLIT), nb = *(volatile int32_t*)(ws.cnt + Q_SPLIT_B);
    const int64_t len = part == 0 ? na : (part == 1 ? nb : na + nb);
    const int64_t front = part == 1 ? 0 : na;
    int32_t* head = ws.cnt + (part == 1 ? H_SPLIT32_B : H_SPLIT32);
    __shared__ int blk_taken;
    if (threadIdx.x == 0) blk_taken = 0;
    __syncthreads();
    SplitSS32<NC> s;
    bool have = false, drained = false;
    for (;;) {
        const int64_t pos = warp_fetch(head, !have, len, drained, &blk_taken, quota);
        if (pos >= 0) {
            s.begin(cs, ws, io, ws.q_split[pos < front ? pos : ws.n - 1 - (pos - front)]);
            have = true;
        }
        if (!__any_sync(0xffffffffu, have)) break;
        if (have && s.step(cs, ws, io)) have = false;
    }
}

// part 0: the front of the split queue; 1: its back; 2: both.  quota > 0:
// each block takes at most about `quota` items and exits (short blocks, so
// that a concurrent higher-priority kernel gets SMs as they free up);
// otherwise the kernel is persistent.
template <int NC, class CS>
__global__ void __launch_bounds__(128, 3) k_split_ss(const __grid_constant__ CS cs, WS ws, IO io, int part, int quota) {
    const int64_t na = *(volatile int32_t*)(ws.cnt + Q_SPLIT), nb = *(volatile int32_t*)(ws.cnt + Q_SPLIT_B);
    const int64_t len = part == 0 ? na : (part == 1 ? nb : na + nb);
    const int64_t front = part == 1 ? 0 : na;  // positions below `front` read the front part
    int32_t* head = ws.cnt + (part == 1 ? H_SPLIT_B : H_SPLIT);
    __shared__ int blk_taken;
    if (threadIdx.x == 0) blk_taken = 0;
    __syncthreads();
    SplitSS<NC> s;
    bool have = false, drained = false;
    for (;;) {
        const int64_t pos = warp_fetch(head, !have, len, drained, &blk_taken, quota);
        if (pos >= 0) {
            s.begin_finish(cs, ws, io, ws.q_split[pos < front ? pos : ws.n - 1 - (pos - front)]);
            have = true;
        }
        if (!__any_sync(0xffffffffu, have)) break;
        const int r = have ? s.step(cs, ws, io) : 0;
        warp_append(ws.cnt + Q_SPLIT_TR, ws.q_split_tr, r == 2, (int32_t)s.m);
        if (r == 2) {
            ws.tflag[s.m] = s.bucket;
            atomicAdd(ws.cnt + QB_SPLIT + s.bucket, 1);
        }
        if (r) have = false;
    }
}

// ---------------------------------------------------------------------------
// Phase-split trust region (Appendix B.2, Eqs. newton_splitter, split_grad,
// split_hess) in the scaled variable u = D^{1/2} dn^V, D = diag(z / (x y)).
// ---------------------------------------------------------------------------
template <int NC>
struct SplitPt {
    double th, x[NC], y[NC], gt[NC], gs[NC], S[NC], G, ZL, ZV;
    double Hs[NC * (NC + 1) / 2];  // S H S
};

// Evaluation of a split point in FP64 (every decision rests on it): the
// phases, their EOS, the gradient gt = mu^V - mu^L (Eq. split_grad), G
// (Eq. gibbs) and the scaling S_i = (z_i / (x_i y_i))^(-1/2) of
// u = D^(1/2) dn^V.  w = 1 / (theta (1 - theta)), pl and pv feed split_model.
template <int NC>
__device__ __forceinline__ bool split_eval(const Comp<NC>& cp, const Mix<NC>& mx, const double* z, const double* iz,
                                           const double* nV, SplitPt<NC>& p, Phase<NC>& pl, Phase<NC>& pv,
                                           double& w) {
    double th = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) th += nV[i];
    p.th = th;
    // one division: w, then 1 / theta = w (1 - theta), 1 / (1 - theta) = w theta
    w = 1.0 / (th * (1.0 - th));
    const double iv = w * (1.0 - th), il = w * th;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        p.y[i] = nV[i] * iv;
        p.x[i] = (z[i] - nV[i]) * il;
    }
    eos<NC>(cp, mx, p.x, pl);
    eos<NC>(cp, mx, p.y, pv);
    p.ZL = pl.Z;
    p.ZV = pv.Z;
    double G = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        double mul = log_fast(p.x[i]) + pl.lnphi[i], muv = log_fast(p.y[i]) + pv.lnphi[i];
        p.gt[i] = muv - mul;
        G = fma(z[i] - nV[i], mul, fma(nV[i], muv, G));
        p.S[i] = sqrt(p.x[i] * p.y[i] * iz[i]);
        p.gs[i] = p.S[i] * p.gt[i];
    }
    p.G = G;
    return isfinite(G);
}

// One entry of S H S: h = theta J^L_ij + (1 - theta) J^V_ij - 1, then
// w S_i S_j h, plus w on the diagonal (shared by the one-lane and the
// several-lanes-per-run models, so both round alike).
template <class R>
__device__ __forceinline__ R split_h(R th, R th1, R jl, R jv) {
    return sub_rn<R>(fma(th, jl, mul_rn<R>(th1, jv)), R(1));  // explicit: no context contracts it otherwise
}
template <class R>
__device__ __forceinline__ double split_hs(bool diag, R wSi, R Si, R Sj, R h, double w) {
    return diag ? fma((double)mul_rn<R>(wSi, Si), (double)h, w) : (double)mul_rn<R>(mul_rn<R>(wSi, Sj), h);
}

// The trust region's model at an evaluated point: the scaled Hessian
// S H S (Eq. split_hess, reading R5) from both phases' n_T d ln phi / dn,
// formed in R.  The diagonal term z_i / (x_i y_i) of H scales to exactly 1.
template <int NC, class R>
__device__ __forceinline__ void split_model(const Comp<NC>& cp, const Mix<NC>& mx, const Phase<NC>& pl,
                                            const Phase<NC>& pv, double w, SplitPt<NC>& p) {
    R JL[NC * (NC + 1) / 2], JV[NC * (NC + 1) / 2];
    dlnphi_dn_r<NC, R>(cp, mx, pl, JL);
    dlnphi_dn_r<NC, R>(cp, mx, pv, JV);
    const R th = (R)p.th, th1 = (R)(1.0 - p.th);
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const R wSi = (R)mul_rn<double>(w, p.S[i]);
#pragma unroll
        for (int j = 0; j <= i; j++) {
            const R h = split_h<R>(th, th1, JL[tri(i, j)], JV[tri(i, j)]);
            p.Hs[tri(i, j)] = split_hs<R>(i == j, wSi, (R)p.S[i], (R)p.S[j], h, w);
        }
    }
}

// 0.99 fraction-to-boundary cut keeping 0 < n^V_i + d_i < z_i: the smallest
// ratio is found by cross-multiplication, with one division at the end
template <int NC>
__device__ __forceinline__ double boundary_cut(const double* z, const double* nV, const double* d) {
    double num = 1.0, den = 1.0;  // tau = num / den, starting at 1
#pragma unroll
    for (int i = 0; i < NC; i++) {
        const double a = d[i] < 0.0 ? 0.99 * nV[i] : 0.99 * (z[i] - nV[i]);
        const double b = fabs(d[i]);
        if (b > 0.0 && a * den < num * b) {
            num = a;
            den = b;
        }
    }
    return num == den ? 1.0 : num / den;
}

// One step = one factorisation of the subproblem and, once its step is known,
// one evaluation of both phases with their derivatives at the trial point
// (trust-region or Newton polish; the start point on the first step).  Both
// kinds of step share the one factorisation site, and the tests that end a
// run follow the evaluation.
template <int NC>
struct SplitTR {
    int64_t m;
    int it, iters, newton_steps, phase, trips;  // phase 0: start point; 1: trust region; 2: Newton polish
    int32_t st;
    Mix<NC> mx;
    double z[NC], iz[NC], nV[NC], radius, eta_lo;  // iz = 1 / z
    TRShift sh;
    SplitPt<NC> cur;

    template <class CS>
    __device__ __forceinline__ void begin(const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        m = mm;
        const Comp<NC>& cp = cs.of(m);
        load_mix<NC>(ws, m, mx);
#pragma unroll
        for (int i = 0; i < NC; i++) {
            z[i] = io.z[i * io.ld + m];
            iz[i] = 1.0 / z[i];
            nV[i] = ws.nV[i * n + m];
        }
        st = io.status[m];
        it = iters = newton_steps = phase = trips = 0;
        radius = -1.0;
        eta_lo = 0.0;
        sh.active = 0;
        sh.warm = 0.0;
    }

    // kind 0 result, 1 non-finite, 2 collapsed onto one phase without converging
    __device__ __forceinline__ int finish(const IO& io, int kind) {
        if (kind == 1) {
            st |= ST_NONFINITE;
            write_single<NC>(io, m, z);
        } else if (kind == 2) {
            st |= ST_COLLAPSE | ST_MAXITER;
            write_single<NC>(io, m, z);
        } else if (!(cur.th > 0.0 && cur.th < 1.0)) {
            st |= ST_COLLAPSE;
            write_single<NC>(io, m, z);
        } else {
            write_two<NC>(io, m, cur.th, cur.x, cur.y, cur.ZL, cur.ZV);
        }
        io.status[m] = st;
        if (io.iters) io.iters[m] = (io.iters[m] & ~0xff00) | ((iters & 0xff) << 8);
        return 1;
    }

    // 0 continue, 1 done.  The model stays FP64 here: the Newton polish must
    // land well inside the 1e-10 residual for the outputs to agree with
    // another FP64 implementation to 1e-8 (an FP32 model's polish step stops
    // at ~1e-11, which ill-conditioned splits turn into 1e-7 in beta).  Every
    // trip evaluates a point or ends the run but for a solve that needs more
    // than a trip; a budget of trips bounds the run whatever happens.
    template <class CS>
    __device__ __forceinline__ int step(const CS& cs, const WS& ws, const IO& io) {
        const Comp<NC>& cp = cs.of(m);
        if (++trips > ws.ctl.tr_split + ws.ctl.polish + 8) {
            st |= ST_MAXITER;
            return finish(io, 0);
        }
        double u[NC], dstep[NC], trial[NC], pred = 0.0;
        if (phase == 0) {
#pragma unroll
            for (int i = 0; i < NC; i++) trial[i] = nV[i];
        } else {
            double Lf[NC * (NC + 1) / 2];
            // split solves need several shifts where they need any, so they
            // finish within the trip (one factorisation site all the same)
            int r = 0;
#pragma unroll 1
            for (int k = 0; k < kTRShiftCap + 2 && r == 0; k++)
                r = tr_shift_step<NC, double>(cur.Hs, cur.gs, radius, eta_lo, phase == 2, sh, Lf, u);
            if (r == 0) return 0;
            if (r < 0) {  // Newton polish on an indefinite Hessian, or a failed solve: stop here
                if (phase == 1 || maxabs<NC>(cur.gt) > ws.ctl.tol_fug) st |= ST_MAXITER;
                return finish(io, 0);
            }
#pragma unroll
            for (int i = 0; i < NC; i++) dstep[i] = cur.S[i] * u[i];
            const double tau = boundary_cut<NC>(z, nV, dstep);
            if (tau < 1.0) {
#pragma unroll
                for (int i = 0; i < NC; i++) {
                    u[i] *= tau;
                    dstep[i] *= tau;
                }
            }
            if (phase == 1) {
                for (int i = 0; i < NC; i++) {
                    double hd = 0.0;
                    for (int j = 0; j < NC; j++) hd = fma(cur.Hs[i >= j ? tri(i, j) : tri(j, i)], u[j], hd);
                    pred = fma(cur.gs[i], u[i], fma(0.5 * u[i], hd, pred));
                }
            }
#pragma unroll
            for (int i = 0; i < NC; i++) trial[i] = nV[i] + dstep[i];
        }
        SplitPt<NC> nxt;
        bool ok;
        {
            Phase<NC> pl, pv;
            double w;
            ok = split_eval<NC>(cp, mx, z, iz, trial, nxt, pl, pv, w);
            if (ok) split_model<NC, double>(cp, mx, pl, pv, w, nxt);
        }
        if (phase == 0) {
            if (!ok) return finish(io, 1);
            cur = nxt;
            phase = 1;
        } else if (phase == 2) {  // Newton polish steps are taken unconditionally
            if (!ok) return finish(io, 1);
#pragma unroll
            for (int i = 0; i < NC; i++) nV[i] = trial[i];
            cur = nxt;
            newton_steps++;
            iters++;
        } else {
            const bool trusted = fabs(pred) > kPredTrust * (1.0 + fabs(cur.G));
            const double rho = !ok ? -1.0 : (trusted ? (nxt.G - cur.G) / pred : 0.5);
            if (rho > 0.0) {
#pragma unroll
                for (int i = 0; i < NC; i++) nV[i] = trial[i];
                cur = nxt;
                eta_lo = 0.0;
            } else {
                eta_lo = sh.eta;  // same H, smaller radius: the shift can only grow
            }
            if (rho <= 0.25) radius *= 0.5;
            else if (rho >= 0.75) radius *= 2.0;
            iters = ++it;
        }
        if (!(cur.th > kCollapseTheta && cur.th < 1.0 - kCollapseTheta)) return finish(io, 2);
        const double res = maxabs<NC>(cur.gt);
        if (phase == 1 && res < ws.ctl.tol_split_tr) phase = 2;
        if (phase == 2) {
            if (res <= ws.ctl.tol_fug && newton_steps >= 1) return finish(io, 0);
            if (newton_steps >= ws.ctl.polish) {
                st |= ST_MAXITER;
                return finish(io, 0);
            }
        } else if (it >= ((st & ST_NN_INIT) ? min(ws.ctl.tr_split, kTRStab) : ws.ctl.tr_split)) {
            // a network-started run gets the paper's stability cap K_tr (Alg. 2):
            // one that has not converged by then is redone by the plain method
            st |= ST_MAXITER;
            return finish(io, 0);
        }
        return 0;
    }
};

// ---------------------------------------------------------------------------
// The split trust region with G lanes per run (lane r: component r), used
// once the queue has drained: SplitTR::step operation for operation, so the
// results are the same bit for bit (see ptf_group.cuh).
// ---------------------------------------------------------------------------
template <int NC>
struct PtG {
    double th, G, ZL, ZV;   // scalars (the same on every lane of the group)
    double x, y, gt, gs, S;  // component r
    double H[NC];            // row r of S H S
};

template <int NC, int G>
struct SplitTRG {
    static constexpr int kHead = H_SPLIT_TR;
    int64_t m;
    int it, iters, newton_steps, phase, trips;
    int32_t st;
    double kkr[NC];                // row r of 1 - k_ij
    double sA, Bi, z, iz, nV;      // component r
    double radius, eta_lo;
    TRShift sh;
    PtG<NC> cur;

    template <class CS>
    __device__ __forceinline__ void load_kk(const Grp& g, const CS& cs) {
        const Comp<NC>& cp = cs.of(m);
        const int rr = g.r < NC ? g.r : 0;  // padding lanes copy component 0
#pragma unroll
        for (int j = 0; j < NC; j++) kkr[j] = cp.kk[rr * NC + j];
    }

    // a fresh run from the queue (as SplitTR::begin)
    template <class CS>
    __device__ __forceinline__ void begin(const Grp& g, const CS& cs, const WS& ws, const IO& io, int64_t mm) {
        const int64_t n = ws.n;
        const int rr = g.r < NC ? g.r : 0;
        m = mm;
        load_kk(g, cs);
        sA = ws.sA[rr * n + m];
        Bi = ws.B[rr * n + m];
        z = io.z[rr * io.ld + m];
        iz = 1.0 / z;
        nV = ws.nV[rr * n + m];
        st = io.status[m];
        it = iters = newton_steps = phase = trips = 0;
        radius = -1.0;
        eta_lo = 0.0;
        sh.active = 0;
        sh.warm = 0.0;
    }

    // a fresh run: queue position pos (in the order k_tr_order laid out)
    template <class CS>
    __device__ __forceinline__ void begin_pos(const Grp& g, const CS& cs, const WS& ws, const IO& io, int64_t pos) {
        begin(g, cs, ws, io, ws.q_sort[pos]);
    }

    // the run that lane src of the warp holds in its one-lane state s
    // (every lane of the warp calls this: full-warp shuffles)
    __device__ __forceinline__ void take_state(const Grp& g, const SplitTR<NC>& s, int src) {
        constexpr unsigned F = 0xffffffffu;
        const int rr = g.r < NC ? g.r : 0;
        m = __shfl_sync(F, s.m, src);
        it = __shfl_sync(F, s.it, src);
        iters = __shfl_sync(F, s.iters, src);
        newton_steps = __shfl_sync(F, s.newton_steps, src);
        phase = __shfl_sync(F, s.phase, src);
        trips = __shfl_sync(F, s.trips, src);
        st = __shfl_sync(F, s.st, src);
        radius = __shfl_sync(F, s.radius, src);
        eta_lo = __shfl_sync(F, s.eta_lo, src);
        sh.eta = __shfl_sync(F, s.sh.eta, src);
        sh.elo = __shfl_sync(F, s.sh.elo, src);
        sh.ehi = __shfl_sync(F, s.sh.ehi, src);
        sh.active = __shfl_sync(F, s.sh.active, src);
        sh.it = __shfl_sync(F, s.sh.it, src);
        sh.warm = __shfl_sync(F, s.sh.warm, src);
        sh.zero = __shfl_sync(F, s.sh.zero, src);
        cur.th = __shfl_sync(F, s.cur.th, src);
        cur.G = __shfl_sync(F, s.cur.G, src);
        cur.ZL = __shfl_sync(F, s.cur.ZL, src);
        cur.ZV = __shfl_sync(F, s.cur.ZV, src);
#pragma unroll
        for (int k = 0; k < NC; k++) {
            const double a1 = __shfl_sync(F, s.mx.sA[k], src), a2 = __shfl_sync(F, s.mx.B[k], src);
            const double a3 = __shfl_sync(F, s.z[k], src), a4 = __shfl_sync(F, s.iz[k], src);
            const double a5 = __shfl_sync(F, s.nV[k], src), a6 = __shfl_sync(F, s.cur.x[k], src);
            const double a7 = __shfl_sync(F, s.cur.y[k], src), a8 = __shfl_sync(F, s.cur.gt[k], src);
            const double a9 = __shfl_sync(F, s.cur.gs[k], src), a10 = __shfl_sync(F, s.cur.S[k], src);
            if (rr == k) {
                sA = a1;
                Bi = a2;
                z = a3;
                iz = a4;
                nV = a5;
                cur.x = a6;
                cur.y = a7;
                cur.gt = a8;
                cur.gs = a9;
                cur.S = a10;
            }
        }
#pragma unroll
        for (int i = 0; i < NC; i++) {
#pragma unroll
            for (int j = 0; j <= i; j++) {
                const double v = __shfl_sync(F, s.cur.Hs[tri(i, j)], src);
                if (rr == i) cur.H[j] = v;
                if (rr == j) cur.H[i] = v;
            }
        }
    }

    __device__ __forceinline__ void write_single_g(const Grp& g, const IO& io) {
        const int64_t n = io.ld;
        if (g.r == 0) {
            io.nphase[m] = 1;
            io.beta[m] = 0.0;
        }
        if (g.r < NC) {
            io.x[g.r * n + m] = z;
            io.y[g.r * n + m] = z;
            io.K[g.r * n + m] = 1.0;
        }
    }

    // as SplitTR::finish
    __device__ __forceinline__ int finish(const Grp& g, const IO& io, int kind) {
        if (kind == 1) {
            st |= ST_NONFINITE;
            write_single_g(g, io);
        } else if (kind == 2) {
            st |= ST_COLLAPSE | ST_MAXITER;
            write_single_g(g, io);
        } else if (!(cur.th > 0.0 && cur.th < 1.0)) {
            st |= ST_COLLAPSE;
            write_single_g(g, io);
        } else {
            const int64_t n = io.ld;
            const bool swap = cur.ZV < cur.ZL;
            if (g.r == 0) {
                io.nphase[m] = 2;
                io.beta[m] = swap ? 1.0 - cur.th : cur.th;
            }
            if (g.r < NC) {
                const double xi = swap ? cur.y : cur.x, yi = swap ? cur.x : cur.y;
                io.x[g.r * n + m] = xi;
                io.y[g.r * n + m] = yi;
                io.K[g.r * n + m] = yi / xi;
            }
        }
        if (g.r == 0) {
            io.status[m] = st;
            if (io.iters) io.iters[m] = (io.iters[m] & ~0xff00) | ((iters & 0xff) << 8);
        }
        return 1;
    }

    // as split_eval, component r's vapour moles nv
    __device__ __forceinline__ bool eval(const Grp& g, double nv, PtG<NC>& p, PhaseG& pl, PhaseG& pv, double& w) {
        double th = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++) th += gat<G>(g, nv, i);
        p.th = th;
        w = 1.0 / (th * (1.0 - th));
        const double iv = w * (1.0 - th), il = w * th;
        p.y = nv * iv;
        p.x = (z - nv) * il;
        eos_g<NC, G>(g, kkr, sA, Bi, p.x, pl);
        eos_g<NC, G>(g, kkr, sA, Bi, p.y, pv);
        p.ZL = pl.Z;
        p.ZV = pv.Z;
        const double mul = log_fast(p.x) + pl.lnphi, muv = log_fast(p.y) + pv.lnphi;
        p.gt = muv - mul;
        const double zn = z - nv;
        double Gs = 0.0;
#pragma unroll
        for (int i = 0; i < NC; i++)
            Gs = fma(gat<G>(g, zn, i), gat<G>(g, mul, i), fma(gat<G>(g, nv, i), gat<G>(g, muv, i), Gs));
        p.G = Gs;
        p.S = sqrt(p.x * p.y * iz);
        p.gs = p.S * p.gt;
        return isfinite(Gs);
    }

    // as split_model (FP64)
    __device__ __forceinline__ void model(const Grp& g, const PhaseG& pl, const PhaseG& pv, double w, PtG<NC>& p) {
        double JL[NC], JV[NC];
        dlnphi_dn_g<NC, G>(g, kkr, sA, Bi, pl, JL);
        dlnphi_dn_g<NC, G>(g, kkr, sA, Bi, pv, JV);
        const double th = p.th, th1 = 1.0 - p.th;
        const double wSi = mul_rn<double>(w, p.S);
#pragma unroll
        for (int j = 0; j < NC; j++) {
            const double Sj = gat<G>(g, p.S, j);
            if (j <= g.r) {
                const double h = split_h<double>(th, th1, JL[j], JV[j]);
                p.H[j] = split_hs<double>(j == g.r, wSi, p.S, Sj, h, w);
            }
        }
        sym_fill<NC, G>(g, p.H);
    }

    // as boundary_cut, component r's step d
    __device__ __forceinline__ double boundary_cut_g(const Grp& g, double d) const {
        const double a = d < 0.0 ? 0.99 * nV : 0.99 * (z - nV);
        const double b = fabs(d);
        double num = 1.0, den = 1.0;
#pragma unroll
        for (int i = 0; i < NC; i++) {
            const double ai = gat<G>(g, a, i), bi = gat<G>(g, b, i);
            if (bi > 0.0 && ai * den < num * bi) {
                num = ai;
                den = bi;
            }
        }
        return num == den ? 1.0 : num / den;
    }

    // as SplitTR::step
    template <class CS>
    __device__ __forceinline__ int step(const Grp& g, const CS& cs, const WS& ws, const IO& io) {
        if (++trips > ws.ctl.tr_split + ws.ctl.polish + 8) {
            st |= ST_MAXITER;
            return finish(g, io, 0);
        }
        double u = 0.0, trial, pred = 0.0;
        if (phase == 0) {
            trial = nV;
        } else {
            double a[NC];
            int r = 0;
#pragma unroll 1
            for (int k = 0; k < kTRShiftCap + 2 && r == 0; k++)
                r = tr_shift_step_g<NC, G>(g, cur.H, cur.gs, radius, eta_lo, phase == 2, sh, a, u);
            if (r == 0) return 0;
            if (r < 0) {
                if (phase == 1 || gmaxabs<NC, G>(g, cur.gt) > ws.ctl.tol_fug) st |= ST_MAXITER;
                return finish(g, io, 0);
            }
            double dstep = cur.S * u;
            const double tau = boundary_cut_g(g, dstep);
            if (tau < 1.0) {
                u *= tau;
                dstep *= tau;
            }
            if (phase == 1) {
                double hd = 0.0;
#pragma unroll
                for (int j = 0; j < NC; j++) hd = fma(cur.H[j], gat<G>(g, u, j), hd);
#pragma unroll
                for (int i = 0; i < NC; i++) {
                    const double ui = gat<G>(g, u, i);
                    pred = fma(gat<G>(g, cur.gs, i), ui, fma(0.5 * ui, gat<G>(g, hd, i), pred));
                }
            }
            trial = nV + dstep;
        }
        PtG<NC> nxt;
        bool ok;
        {
            PhaseG pl, pv;
            double w;
            ok = eval(g, trial, nxt, pl, pv, w);
            if (ok) model(g, pl, pv, w, nxt);
        }
        if (phase == 0) {
            if (!ok) return finish(g, io, 1);
            cur = nxt;
            phase = 1;
        } else if (phase == 2) {
            if (!ok) return finish(g, io, 1);
            nV = trial;
            cur = nxt;
            newton_steps++;
            iters++;
        } else {
            const bool trusted = fabs(pred) > kPredTrust * (1.0 + fabs(cur.G));
            const double rho = !ok ? -1.0 : (trusted ? (nxt.G - cur.G) / pred : 0.5);
            if (rho > 0.0) {
                nV = trial;
                cur = nxt;
                eta_lo = 0.0;
            } else {
                eta_lo = sh.eta;
            }
            if (rho <= 0.25) radius *= 0.5;
            else if (rho >= 0.75) radius *= 2.0;
            iters = ++it;
        }
        if (!(cur.th > kCollapseTheta && cur.th < 1.0 - kCollapseTheta)) return finish(g, io, 2);
        const double res = gmaxabs<NC, G>(g, cur.gt);
        if (phase == 1 && res < ws.ctl.tol_split_tr) phase = 2;
        if (phase == 2) {
            if (res <= ws.ctl.tol_fug && newton_steps >= 1) return finish(g, io, 0);
            if (newton_steps >= ws.ctl.polish) {
                st |= ST_MAXITER;
                return finish(g, io, 0);
            }
        } else if (it >= ((st & ST_NN_INIT) ? min(ws.ctl.tr_split, kTRStab) : ws.ctl.tr_split)) {
            st |= ST_MAXITER;
            return finish(g, io, 0);
        }
        return 0;
    }
};

// Lay the split trust-region queue out by bucket (longest expected runs
// first) into ws.q_sort: each block forms the bucket offsets from the counts,
// and the items of a bucket take consecutive positions from its cursor.
static __global__ void __launch_bounds__(128) k_tr_order(WS ws) {
    __shared__ int base[kTRBuckets];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < kTRBuckets; b++) {
            base[b] = acc;
            acc += *(volatile int32_t*)(ws.cnt + QB_SPLIT + b);
        }
    }
    __syncthreads();
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_SPLIT_TR);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t m = ws.q_split_tr[k];
        const int b = ws.tflag[m];
        ws.q_sort[base[b] + atomicAdd(ws.cnt + QB_SPLIT + kTRBuckets + b, 1)] = m;
    }
}

// As k_stab_tr: one lane per run while the queue lasts, then G lanes per run.
template <int NC, class CS>
__global__ void __launch_bounds__(128, 3) k_split_tr(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_SPLIT_TR);
    SplitTR<NC> s;
    bool have = false, drained = false;
    if constexpr (GroupLanes<NC>::ok) {
        if (ws.ctl.tr_coop == 2) {
            tr_groups<SplitTRG<NC, GroupLanes<NC>::G>, GroupLanes<NC>::G>(cs, ws, io, s, 0u, true, len);
            return;
        }
    }
    for (;;) {
        const int64_t pos = warp_fetch(ws.cnt + H_SPLIT_TR, !have, len, drained);
        if (pos >= 0) {
            s.begin(cs, ws, io, ws.q_sort[pos]);  // in the order k_tr_order laid out
            have = true;
        }
        const unsigned live = __ballot_sync(0xffffffffu, have);
        if (!live) break;
        if constexpr (GroupLanes<NC>::ok) {
            if (drained && ws.ctl.tr_coop == 0 && __popc(live) <= kGroupSwitch) {
                tr_groups<SplitTRG<NC, GroupLanes<NC>::G>, GroupLanes<NC>::G>(cs, ws, io, s, live, false, len);
                break;
            }
        }
        if (have && s.step(cs, ws, io)) have = false;
    }
}

// ---------------------------------------------------------------------------
// Stability-only outputs (ptflash_stability): io.nphase = stable flag,
// io.beta = min tm, io.K = K re-estimate.
// ---------------------------------------------------------------------------
template <int NC, class CS>
__device__ __forceinline__ void stab_out_item(const CS& cs, const WS& ws, const IO& io, int64_t m) {
    const Comp<NC>& cp = cs.of(m);
    const int64_t n = ws.n;
    {
        {
            const double tv = ws.tm[m], tl = ws.tm[n + m];
            const int32_t fv = ws.tflag[m], fl = ws.tflag[n + m];
            int32_t st = io.status[m];
            if ((fv | fl) & (1 << 16)) st |= ST_STAB_TR;
            if ((fv | fl) & (1 << 17)) st |= ST_MAXITER;
            if ((fv | fl) & (1 << 18)) st |= ST_NONFINITE;
            const double tmin = tv < tl ? tv : tl;
            io.nphase[m] = (tmin < -kEpsNeg) ? 0 : 1;
            io.beta[m] = tmin;
            double lnK[NC];
            stab_lnK<NC>(ws, m, tl < tv ? 1 : 0, lnK);
#pragma unroll
            for (int i = 0; i < NC; i++) io.K[i * io.ld + m] = exp_fast(lnK[i]);
            io.status[m] = st;
        }
    }
}

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_stab_out(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_STAB);
    PTF_WARP_ROUNDS(len, qi, valid) {
        if (valid) stab_out_item<NC>(cs, ws, io, ws.q_stab[qi]);
    }
}

// ---------------------------------------------------------------------------
// Phase EOS at given compositions (Appendix A: Eqs. a_i, b_i, mixing_rule,
// cubic_Z with the lower-gbar root of reading R6, lnphi), one thread per
// point: the A2 primitive of every stage, evaluated alone.
// ---------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(128) k_phase_eos(const __grid_constant__ Comp<NC> cp, int64_t n, const double* P,
                                                   const double* T, const double* c, double* Z, double* lnphi) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        double cc[NC];
#pragma unroll
        for (int i = 0; i < NC; i++) cc[i] = c[i * n + m];
        Mix<NC> mx;
        mix_init<NC>(cp, P[m], T[m], mx);
        Phase<NC> ph;
        eos<NC>(cp, mx, cc, ph);
        Z[m] = ph.Z;
#pragma unroll
        for (int i = 0; i < NC; i++) lnphi[i * n + m] = ph.lnphi[i];
    }
}

// ---------------------------------------------------------------------------
// Learned form (Sec. 4.3), with the plain method as judge of what the networks
// decide.  The classifier gives the probability p that the mixture is stable:
//  - p >= p_r: single phase (NN_STABLE), unless tpd (Eq. tpd) is negative at
//    one of four trial phases, w proportional to z K and to z / K for the
//    initializer's K and for Wilson K (the trials of Sec. 2.2.1, before any
//    iteration).  A negative tpd proves instability: such a mixture takes the
//    plain route instead.
//  - p <= p_l with the initializer's ln K finite and bracketing K = 1
//    (NN_UNSTABLE | NN_INIT): the plain precheck still runs, and only if it
//    proves instability does the split start from the initializer's K (else
//    the mixture takes the plain route from stability analysis on: where the
//    precheck cannot prove instability, the plain method's split starts from
//    a stability trial, and near three-phase conditions the initializer's K
//    can lead to another stationary point of G).  k_nn_judge checks the split.
//  - otherwise the plain route (status 0): the precheck, stability analysis
//    from Wilson K and the split, exactly as in the plain flash.
// The initializer's ln K are clamped to [-15, 15].
// ---------------------------------------------------------------------------
template <int NC>
__device__ __forceinline__ double trial_tpd(const Comp<NC>& cp, const Mix<NC>& mx, const double* z, const double* d,
                                            const double* lnK, bool vapour_like) {
    double w[NC], sw = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) {
        w[i] = z[i] * exp_fast(vapour_like ? lnK[i] : -lnK[i]);
        sw += w[i];
    }
    const double inv = 1.0 / sw;
#pragma unroll
    for (int i = 0; i < NC; i++) w[i] *= inv;
    Phase<NC> ph;
    eos<NC>(cp, mx, w, ph);
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < NC; i++) t = fma(w[i], log_fast(w[i]) + ph.lnphi[i] - d[i], t);
    return t;  // NaN when not finite: no proof either way
}

template <int NC, class CS>
__global__ void __launch_bounds__(128) k_nn_route(const __grid_constant__ CS cs, WS ws, IO io, float p_l,
                                                  float p_r) {
    const int64_t n = ws.n;
    PTF_WARP_ROUNDS(n, m, valid) {
        if (valid && !(io.status[m] & ST_NONFINITE)) {
            const Comp<NC>& cp = cs.of(m);
            const float p = 1.0f / (1.0f + __expf(-ws.nnp[m]));
            double lnK[NC], kmax = -1e300, kmin = 1e300;
            bool fin = true;
#pragma unroll
            for (int i = 0; i < NC; i++) {
                double v = (double)ws.nnk[i * n + m];
                fin = fin && isfinite(v);
                v = fmin(fmax(v, -15.0), 15.0);
                lnK[i] = v;
                kmax = fmax(kmax, v);
                kmin = fmin(kmin, v);
            }
            if (p >= p_r) {
                double z[NC], d[NC], lw[NC];
                Mix<NC> mx;
                load_mix<NC>(ws, m, mx);
                wilson<NC>(cp, io.P[m], io.T[m], lw);
#pragma unroll
                for (int i = 0; i < NC; i++) {
                    z[i] = io.z[i * io.ld + m];
                    d[i] = ws.d[i * n + m];
                    lw[i] = fmin(fmax(lw[i], -30.0), 30.0);
                }
                bool unstable = false;
#pragma unroll 1
                for (int t = fin ? 0 : 2; t < 4 && !unstable; t++)
                    unstable = trial_tpd<NC>(cp, mx, z, d, t < 2 ? lnK : lw, (t & 1) == 0) < -kEpsNeg;
                if (unstable) {
                    io.status[m] = 0;  // the plain route
                } else {
                    io.status[m] = ST_NN_STABLE;
                    write_single<NC>(io, m, z);
                }
            } else if (p <= p_l && fin && kmax > 0.0 && kmin < 0.0) {
                io.status[m] = ST_NN_UNSTABLE | ST_NN_INIT;  // the precheck decides the split's start
            } else {
                io.status[m] = 0;  // the plain route
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Judge of the network-started splits (learned form, Sec. 4.3): a mixture the
// classifier and the precheck sent to the split from the initializer's K keeps
// that result only if the split proves instability where the initializer
// pointed: two phases, converged
// (no cap, no collapse, finite), Delta G = sum z_i (mu_i - d_i) < -1e-10 at
// the converged phases (mu_i = ln x_i + ln phi_i(x), the same in both phases;
// d_i = ln z_i + ln phi_i(z)), and every converged ln K_i within
// ctl.nn_lnk_dev of the network's.  Any other outcome -- one phase, a cap, a
// non-finite state, or a stationary point of G far from the prediction (where
// several exist the plain method can reach another) -- is redone by the plain
// method: status NN_REJECT, appended to q_redo for the second pass.
// ---------------------------------------------------------------------------
template <int NC, class CS>
__global__ void __launch_bounds__(128) k_nn_judge(const __grid_constant__ CS cs, WS ws, IO io) {
    const int64_t len = *(volatile int32_t*)(ws.cnt + Q_SPLIT);  // the front part of the split queue
    const int64_t n = ws.n;
    PTF_WARP_ROUNDS(len, qi, valid) {
        const int64_t m = valid ? ws.q_split[qi] : 0;
        bool redo = false;
        if (valid && (io.status[m] & ST_NN_UNSTABLE)) {
            const int32_t st = io.status[m];
            redo = io.nphase[m] != 2 || (st & (ST_MAXITER | ST_COLLAPSE | ST_NONFINITE)) != 0;
            if (!redo) {
                const Comp<NC>& cp = cs.of(m);
                double x[NC], z[NC], dev = 0.0;
                Mix<NC> mx;
                load_mix<NC>(ws, m, mx);
#pragma unroll
                for (int i = 0; i < NC; i++) {
                    x[i] = io.x[i * io.ld + m];
                    z[i] = io.z[i * io.ld + m];
                    const double net = fmin(fmax((double)ws.nnk[i * n + m], -15.0), 15.0);
                    dev = fmax(dev, fabs(log_fast(io.K[i * io.ld + m]) - net));
                }
                Phase<NC> px;
                eos<NC>(cp, mx, x, px);
                double dG = 0.0;
#pragma unroll
                for (int i = 0; i < NC; i++) dG = fma(z[i], log_fast(x[i]) + px.lnphi[i] - ws.d[i * n + m], dG);
                redo = !(dG < -kEpsNeg) || !(dev <= ws.ctl.nn_lnk_dev);
            }
            if (redo) {
                io.status[m] = ST_NN_REJECT;
                if (io.iters) io.iters[m] = 0;
            }
        }
        warp_append(ws.cnt + Q_REDO, ws.q_redo, redo, (int32_t)m);
    }
}

}  // namespace ptf
