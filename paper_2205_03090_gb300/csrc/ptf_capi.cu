// ptf_capi.cu -- the C ABI declared in include/ptflash.h.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/ptflash.h"
#include "ptf_launch.cuh"
#include "ptf_ctx.cuh"

using namespace ptf;

namespace {
thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return PTF_ERR_CUDA;
}
#define PTF_CUDA(call)                              \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)
}  // namespace

static cudaError_t dispatch(ptflash_ctx* c, const WS& ws, const IO& io, int mode, cudaStream_t s, float p_l = 0.02f,
                           float p_r = 0.98f) {
    const int grid = c->sm_count * 8;
    cudaEvent_t* ev = c->profiling ? c->ev : nullptr;
    MLP nn[2];
    if (mode == 2) {
        nn[0] = c->nn[0].view();
        nn[1] = c->nn[1].view();
    }
    switch (c->comp.nc) {
#define PTF_CASE(NC) \
    case NC: return launch_plain<NC>(c->comp, ws, io, grid, mode, s, ev, nn, p_l, p_r, c->conc.hi ? &c->conc : nullptr);
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Self-check of the library's own elementary functions against the CUDA math
// library.  log: n inputs spread log-uniformly over [1e-300, 1e300] plus n
// inputs in [0.5, 2].  exp: n inputs uniform over [-700, 700] plus n in
// [-40, 10].  The largest error in units of the last place of the library
// result is folded into err[0] (log) and err[1] (exp) (positive doubles
// order like their bit patterns).
__device__ __forceinline__ double ulp_of(double ref) {
    if (ref == 0.0) return 4.9e-324;
    int ex;
    frexp(ref, &ex);
    return ldexp(1.0, ex - 53);
}

__global__ void k_check_math(int64_t n, unsigned long long* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 2 * n; k += (int64_t)gridDim.x * blockDim.x) {
        const double u = (double)(k % n) / (double)n;
        const double x = (k < n) ? exp2(-996.0 + 1992.0 * u) * (1.0 + 0.61803398874989 * u) : 0.5 + 1.5 * u;
        const double ref = log(x), got = log_fast(x);
        atomicMax(err, (unsigned long long)__double_as_longlong(fabs(got - ref) / ulp_of(ref)));
        const double y = (k < n) ? -700.0 + 1400.0 * u : -40.0 + 50.0 * u;
        const double re = exp(y), ge = exp_fast(y);
        atomicMax(err + 1, (unsigned long long)__double_as_longlong(fabs(ge - re) / ulp_of(re)));
    }
}

// FP64 throughput probe: 8 independent FMA chains per thread, so that the
// FP64 pipes (not the chain latency) bound the rate.  The final test can never
// hold for these inputs; it keeps the chains live.
__global__ void __launch_bounds__(256) k_fp64_fma(int64_t iters, double b, double cst, double* sink) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = 1.0 + 1e-3 * threadIdx.x + k;
#pragma unroll 1
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int k = 0; k < 8; k++) a[k] = fma(a[k], b, cst);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) t += a[k];
    if (t == -1.0) sink[0] = t;
}

extern "C" {

int ptflash_fp64_fma_rate(int64_t iters, double* tflops, double* ms) {
    if (iters < 1 || iters > ((int64_t)1 << 32) || !tflops || !ms) return PTF_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    PTF_CUDA(cudaGetDevice(&dev));
    PTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 4, threads = 256;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PTF_CUDA(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    float t = 0.0f;
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, threads>>>(iters / 8 + 1, 0.999999999, 1e-9, nullptr);  // warm-up
        e = cudaEventRecord(e0);
    }
    if (e == cudaSuccess) {
        k_fp64_fma<<<blocks, threads>>>(iters, 0.999999999, 1e-9, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e);
    *ms = t;
    *tflops = 2.0 * 32.0 * (double)iters * blocks * threads / (t * 1e-3) / 1e12;
    return PTF_OK;
}

int ptflash_phase_eos(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* comp, double* Z,
                      double* lnphi, void* stream) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (n < 0) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !comp || !Z || !lnphi) return PTF_ERR_INVALID_ARG;
    const int grid = c->sm_count * 8;
    cudaStream_t s = (cudaStream_t)stream;
    switch (c->comp.nc) {
#define PTF_CASE(NC) \
    case NC: PTF_CUDA(launch_eos<NC>(c->comp, n, P, T, comp, Z, lnphi, grid, s)); return PTF_OK;
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
    }
    return PTF_ERR_UNSUPPORTED;
}

int ptflash_check_math(int64_t n, double* max_ulp_log, double* max_ulp_exp) {
    if (n < 1 || n > (int64_t)1 << 28 || !max_ulp_log || !max_ulp_exp) return PTF_ERR_INVALID_ARG;
    unsigned long long* d = nullptr;
    PTF_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
        k_check_math<<<1024, 256>>>(n, d);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e);
    *max_ulp_log = __builtin_bit_cast(double, h[0]);
    *max_ulp_exp = __builtin_bit_cast(double, h[1]);
    return PTF_OK;
}

const char* ptflash_strerror(int code) {
    switch (code) {
        case PTF_OK: return "ok";
        case PTF_ERR_INVALID_ARG: return "invalid argument";
        case PTF_ERR_CUDA: return "CUDA error";
        case PTF_ERR_NOT_READY: return "components not set";
        case PTF_ERR_NO_MEMORY: return "device allocation failed";
        case PTF_ERR_UNSUPPORTED: return "unsupported number of components";
        default: return "unknown error";
    }
}

const char* ptflash_last_cuda_error(void) { return g_cuda_err; }

int ptflash_create(ptflash_ctx** out, int nc_max, int64_t n_max) {
    if (!out) return PTF_ERR_INVALID_ARG;
    *out = nullptr;
    if (nc_max < 2 || nc_max > 16) return PTF_ERR_UNSUPPORTED;
    if (n_max < 1 || n_max > (int64_t)1 << 30) return PTF_ERR_INVALID_ARG;
    ptflash_ctx* c = new (std::nothrow) ptflash_ctx();
    if (!c) return PTF_ERR_NO_MEMORY;
    c->nc_max = nc_max;
    c->n_max = n_max;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e);
    }
    size_t nd = (size_t)(8 * nc_max + 3) * (size_t)n_max, ni = 9 * (size_t)n_max + 64;
    if (cudaMalloc(&c->wsd, nd * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->wsi, ni * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&c->acc, 8 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->wsd);
        cudaFree(c->wsi);
        cudaFree(c->acc);
        delete c;
        return PTF_ERR_NO_MEMORY;
    }
    // streams of the concurrent split SS: the stability chain at the highest
    // priority, the independent split SS at the lowest
    int lo = 0, hi = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&c->conc.hi, cudaStreamNonBlocking, hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&c->conc.lo, cudaStreamNonBlocking, lo) == cudaSuccess;
    for (cudaEvent_t* e : {&c->conc.fork, &c->conc.pre, &c->conc.lo_done, &c->conc.hi_done})
        ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ptflash_destroy(c);
        return PTF_ERR_CUDA;
    }
    *out = c;
    return PTF_OK;
}

int ptflash_destroy(ptflash_ctx* c) {
    if (!c) return PTF_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    if (c->conc.hi) cudaStreamDestroy(c->conc.hi);
    if (c->conc.lo) cudaStreamDestroy(c->conc.lo);
    for (cudaEvent_t e : {c->conc.fork, c->conc.pre, c->conc.lo_done, c->conc.hi_done})
        if (e) cudaEventDestroy(e);
    cudaFree(c->wsd);
    cudaFree(c->wsi);
    cudaFree(c->hd);
    cudaFree(c->hi);
    cudaFree(c->acc);
    for (int k = 0; k <= kStages; k++)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    delete c;
    return PTF_OK;
}

int ptflash_set_components(ptflash_ctx* c, int nc, const double* Tc, const double* Pc, const double* omega,
                           const double* kij) {
    if (!c || !Tc || !Pc || !omega || !kij) return PTF_ERR_INVALID_ARG;
    if (nc < 2 || nc > 16 || nc > c->nc_max) return PTF_ERR_UNSUPPORTED;
    for (int i = 0; i < nc; i++) {
        if (!(Tc[i] > 0.0) || !(Pc[i] > 0.0) || !std::isfinite(Tc[i]) || !std::isfinite(Pc[i]) ||
            !std::isfinite(omega[i]))
            return PTF_ERR_INVALID_ARG;
        for (int j = 0; j < nc; j++) {
            double k = kij[i * nc + j];
            if (!std::isfinite(k) || k != kij[j * nc + i] || (i == j && k != 0.0)) return PTF_ERR_INVALID_ARG;
        }
    }
    CompHost h{};
    h.nc = nc;
    for (int i = 0; i < nc; i++) {
        h.Tc[i] = Tc[i];
        h.Pc[i] = Pc[i];
        h.om[i] = omega[i];
    }
    for (int i = 0; i < nc * nc; i++) h.kij[i] = kij[i];
    c->comp = h;
    c->have_comp = true;
    return PTF_OK;
}

// The options of one call: learned-form thresholds, tolerances and caps.
struct CallOpts {
    int mode = 0;  // 0 plain, 2 learned form
    float p_l = 0.02f, p_r = 0.98f;
    Ctl ctl;
};

// Validate *opt (NULL = defaults) into o.  The learned form needs both networks.
static int parse_options(const ptflash_ctx* c, const ptflash_options* opt, CallOpts& o) {
    o = CallOpts();
    if (!opt) return PTF_OK;
    auto cap = [](int32_t v, int& dst) {
        if (v == 0) return true;
        if (v < 1 || v > 200) return false;
        dst = v;
        return true;
    };
    auto tol = [](double v, double& dst) {
        if (v == 0.0) return true;
        if (!(v > 0.0) || !std::isfinite(v)) return false;
        dst = v;
        return true;
    };
    if (!cap(opt->max_ss_stab, o.ctl.ss_stab) || !cap(opt->max_tr_stab, o.ctl.tr_stab) ||
        !cap(opt->max_ss_split, o.ctl.ss_split) || !cap(opt->max_tr_split, o.ctl.tr_split) ||
        !cap(opt->max_polish, o.ctl.polish) || !tol(opt->tol_stab, o.ctl.tol_stab) ||
        !tol(opt->tol_split_tr, o.ctl.tol_split_tr) || !tol(opt->tol_fug, o.ctl.tol_fug) ||
        !tol(opt->nn_lnk_dev, o.ctl.nn_lnk_dev) || opt->tr_lanes < 0 || opt->tr_lanes > 2)
        return PTF_ERR_INVALID_ARG;
    o.ctl.tr_coop = opt->tr_lanes;
    if (opt->use_nn) {
        if (!(opt->p_l >= 0.0 && opt->p_l <= opt->p_r && opt->p_r <= 1.0)) return PTF_ERR_INVALID_ARG;
        if (!c->nn[0].ready || !c->nn[1].ready) return PTF_ERR_NOT_READY;
        o.mode = 2;
        o.p_l = (float)opt->p_l;
        o.p_r = (float)opt->p_r;
    }
    return PTF_OK;
}

static int run(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z, int32_t* o_i,
               double* o_d, double* x, double* y, double* K, int32_t* status, int32_t* iters, int mode,
               bool zero_counts, cudaStream_t s, float p_l = 0.02f, float p_r = 0.98f, const Ctl& ctl = Ctl()) {
    if (zero_counts) {
        PTF_CUDA(cudaMemsetAsync(c->acc, 0, 8 * sizeof(unsigned long long), s));
        for (int k = 0; k < kStages; k++) c->stage_ms[k] = 0.0;
    }
    for (int64_t m0 = 0; m0 < n; m0 += c->n_max) {
        const int64_t cn = (n - m0 < c->n_max) ? n - m0 : c->n_max;
        WS ws = make_ws(c, cn);
        ws.ctl = ctl;
        IO io;
        io.ld = n;
        io.P = P + m0;
        io.T = T + m0;
        io.z = z + m0;
        io.nphase = o_i + m0;
        io.beta = o_d + m0;
        io.x = x ? x + m0 : nullptr;
        io.y = y ? y + m0 : nullptr;
        io.K = K + m0;
        io.status = status + m0;
        io.iters = iters ? iters + m0 : nullptr;
        PTF_CUDA(cudaMemsetAsync(ws.cnt, 0, 64 * sizeof(int32_t), s));
        PTF_CUDA(dispatch(c, ws, io, mode, s, p_l, p_r));
        k_fold_counts<<<1, 32, 0, s>>>(ws.cnt, c->acc);
        PTF_CUDA(cudaGetLastError());
        if (c->profiling) {  // profiling mode waits for each chunk to read its stage times
            PTF_CUDA(cudaEventSynchronize(c->ev[kStages]));
            for (int k = 0; k < kStages; k++) {
                float ms = 0.0f;
                PTF_CUDA(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
                c->stage_ms[k] += ms;
            }
        }
    }
    return PTF_OK;
}

int ptflash_flash(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z, int32_t* nphase,
                  double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                  const ptflash_options* opt, void* stream) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (n < 0) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !z || !nphase || !beta || !x || !y || !K || !status) return PTF_ERR_INVALID_ARG;
    CallOpts o;
    if (int rc = parse_options(c, opt, o)) return rc;
    return run(c, n, P, T, z, nphase, beta, x, y, K, status, iters, o.mode, true, (cudaStream_t)stream, o.p_l,
               o.p_r, o.ctl);
}

int ptflash_default_options(ptflash_options* opt) {
    if (!opt) return PTF_ERR_INVALID_ARG;
    std::memset(opt, 0, sizeof(*opt));
    const Ctl d;
    opt->p_l = 0.02;
    opt->p_r = 0.98;
    opt->max_ss_stab = d.ss_stab;
    opt->max_tr_stab = d.tr_stab;
    opt->max_ss_split = d.ss_split;
    opt->max_tr_split = d.tr_split;
    opt->max_polish = d.polish;
    opt->tol_stab = d.tol_stab;
    opt->tol_split_tr = d.tol_split_tr;
    opt->tol_fug = d.tol_fug;
    opt->nn_lnk_dev = d.nn_lnk_dev;
    return PTF_OK;
}

int ptflash_flash_adjoint(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z,
                          const int32_t* nphase, const double* beta, const double* x, const double* y,
                          const double* gbeta, const double* gx, const double* gy, double* gP, double* gT,
                          double* gz, int32_t* astatus, void* stream) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (n < 0) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !z || !nphase || !beta || !x || !y || !gP || !gT || !gz) return PTF_ERR_INVALID_ARG;
    AdjIO a{n, P, T, z, nphase, beta, x, y, gbeta, gx, gy, gP, gT, gz, astatus};
    const int grid = c->sm_count * 8;
    cudaStream_t s = (cudaStream_t)stream;
    switch (c->comp.nc) {
#define PTF_CASE(NC) \
    case NC: PTF_CUDA(launch_adjoint<NC>(c->comp, a, grid, s)); return PTF_OK;
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
    }
    return PTF_ERR_UNSUPPORTED;
}

int ptflash_stability(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z,
                      int32_t* stable, double* tm_min, double* K, int32_t* status, void* stream) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (n < 0) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !z || !stable || !tm_min || !K || !status) return PTF_ERR_INVALID_ARG;
    return run(c, n, P, T, z, stable, tm_min, nullptr, nullptr, K, status, nullptr, 1, true, (cudaStream_t)stream);
}

int ptflash_flash_host(ptflash_ctx* c, int64_t n, const double* P, const double* T, const double* z,
                       int32_t* nphase, double* beta, double* x, double* y, double* K, int32_t* status,
                       int32_t* iters, const ptflash_options* opt, void* stream) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (!c->have_comp) return PTF_ERR_NOT_READY;
    if (n < 0) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !z || !nphase || !beta || !x || !y || !K || !status) return PTF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nm = c->n_max;
    const int nc = c->comp.nc;
    if (!c->hd) {
        if (cudaMalloc(&c->hd, (size_t)(4 * c->nc_max + 3) * nm * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&c->hi, (size_t)3 * nm * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(c->hd);
            c->hd = nullptr;
            return PTF_ERR_NO_MEMORY;
        }
    }
    CallOpts o;
    if (int rc = parse_options(c, opt, o)) return rc;
    PTF_CUDA(cudaMemsetAsync(c->acc, 0, 8 * sizeof(unsigned long long), s));
    for (int64_t m0 = 0; m0 < n; m0 += nm) {
        const int64_t cn = (n - m0 < nm) ? n - m0 : nm;
        double* dP = c->hd;
        double* dT = dP + cn;
        double* dz = dT + cn;
        double* dbeta = dz + (int64_t)nc * cn;
        double* dx = dbeta + cn;
        double* dy = dx + (int64_t)nc * cn;
        double* dK = dy + (int64_t)nc * cn;
        int32_t* dnp = c->hi;
        int32_t* dst = dnp + cn;
        int32_t* dit = dst + cn;
        const size_t rowb = (size_t)cn * sizeof(double), pitch = (size_t)n * sizeof(double);
        PTF_CUDA(cudaMemcpyAsync(dP, P + m0, rowb, cudaMemcpyHostToDevice, s));
        PTF_CUDA(cudaMemcpyAsync(dT, T + m0, rowb, cudaMemcpyHostToDevice, s));
        PTF_CUDA(cudaMemcpy2DAsync(dz, rowb, z + m0, pitch, rowb, nc, cudaMemcpyHostToDevice, s));
        int rc = run(c, cn, dP, dT, dz, dnp, dbeta, dx, dy, dK, dst, iters ? dit : nullptr, o.mode, false, s, o.p_l,
                     o.p_r, o.ctl);
        if (rc) return rc;
        PTF_CUDA(cudaMemcpyAsync(nphase + m0, dnp, cn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaMemcpyAsync(status + m0, dst, cn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (iters) PTF_CUDA(cudaMemcpyAsync(iters + m0, dit, cn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaMemcpyAsync(beta + m0, dbeta, rowb, cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaMemcpy2DAsync(x + m0, pitch, dx, rowb, rowb, nc, cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaMemcpy2DAsync(y + m0, pitch, dy, rowb, rowb, nc, cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaMemcpy2DAsync(K + m0, pitch, dK, rowb, rowb, nc, cudaMemcpyDeviceToHost, s));
        PTF_CUDA(cudaStreamSynchronize(s));
    }
    return PTF_OK;
}

int ptflash_set_profiling(ptflash_ctx* c, int enable) {
    if (!c) return PTF_ERR_INVALID_ARG;
    if (enable && !c->ev[0]) {
        for (int k = 0; k <= kStages; k++) PTF_CUDA(cudaEventCreate(&c->ev[k]));
    }
    c->profiling = enable != 0;
    return PTF_OK;
}

int ptflash_last_stage_ms(ptflash_ctx* c, double* ms, int count) {
    if (!c || !ms || count < 0) return PTF_ERR_INVALID_ARG;
    for (int k = 0; k < count && k < kStages; k++) ms[k] = c->stage_ms[k];
    return PTF_OK;
}

int ptflash_last_counts(ptflash_ctx* c, int64_t* counts) {
    if (!c || !counts) return PTF_ERR_INVALID_ARG;
    unsigned long long a[4];
    PTF_CUDA(cudaDeviceSynchronize());
    PTF_CUDA(cudaMemcpy(a, c->acc, sizeof(a), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; k++) counts[k] = (int64_t)a[k];
    return PTF_OK;
}

}  // extern "C"
