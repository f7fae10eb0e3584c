// ptf_noalloc.cu -- ptflash_flash_noalloc: the plain flash without any
// device allocation.
//
// Some callers cannot allocate device memory once they are running: a
// simulator time-step loop that budgeted all GPU memory at start-up, a host
// application whose own allocator owns the device heap, or code that cannot
// afford the device-wide synchronisation cudaMalloc / cudaFree may imply.
// For them this entry point keeps its scratch (per-mixture stage state and
// the stage queues) in one file-scope __device__ array of fixed size, which
// every GPU that loads this library holds until the process exits.  The
// caller still passes the input and output arrays.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/ptflash.h"
#include "ptf_launch.cuh"

using namespace ptf;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code `g_scratch` is only a host-side stand-in
// for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Per-device set-up, done on the first call made with that device current.
int setup(int dev, void** ptr, int* sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PTF_ERR_CUDA;
        }
        int s = 0;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) {
            cudaGetLastError();
            return PTF_ERR_CUDA;
        }
        g_dev_ptr[dev] = p;
        g_sms[dev] = s;
    }
    *ptr = g_dev_ptr[dev];
    *sms = g_sms[dev];
    return PTF_OK;
}

// Bytes of scratch one mixture needs: (8 nc + 3) doubles of stage state and
// 8 int32 of queue entries; 256 bytes of queue counters per call.
size_t bytes_per_mixture(int nc) { return (size_t)(8 * nc + 3) * sizeof(double) + 8 * sizeof(int32_t); }

WS carve(unsigned char* base, int nc, int64_t n) {
    WS w;
    w.n = n;
    int32_t* cnt = reinterpret_cast<int32_t*>(base);
    double* p = reinterpret_cast<double*>(base + 256);
    w.sA = p; p += (int64_t)nc * n;
    w.B = p; p += (int64_t)nc * n;
    w.lnz = p; p += (int64_t)nc * n;
    w.d = p; p += (int64_t)nc * n;
    w.lnK = p; p += (int64_t)nc * n;
    w.nV = p; p += (int64_t)nc * n;
    w.lnW = p; p += 2 * (int64_t)nc * n;
    w.theta = p; p += n;
    w.tm = p; p += 2 * n;
    int32_t* q = reinterpret_cast<int32_t*>(p);
    w.cnt = cnt;
    w.tflag = q; q += 2 * n;
    w.q_stab = q; q += n;
    w.q_split = q; q += n;
    w.q_stab_tr = q; q += 2 * n;
    w.q_split_tr = q; q += n;
    w.q_sort = q; q += n;
    return w;
}

}  // namespace

extern "C" int64_t ptflash_noalloc_max_mixtures(int nc) {
    if (nc < 2 || nc > 16) return 0;
    return (int64_t)((kScratchBytes - 256) / bytes_per_mixture(nc));
}

extern "C" int ptflash_flash_noalloc(int nc, const double* Tc, const double* Pc, const double* omega,
                                     const double* kij, int64_t n, const double* P, const double* T,
                                     const double* z, int32_t* nphase, double* beta, double* x, double* y,
                                     double* K, int32_t* status, int32_t* iters, void* stream) {
    if (!Tc || !Pc || !omega || !kij) return PTF_ERR_INVALID_ARG;
    if (nc < 2 || nc > 16) return PTF_ERR_UNSUPPORTED;
    for (int i = 0; i < nc; i++) {
        if (!(Tc[i] > 0.0) || !(Pc[i] > 0.0) || !std::isfinite(Tc[i]) || !std::isfinite(Pc[i]) ||
            !std::isfinite(omega[i]))
            return PTF_ERR_INVALID_ARG;
        for (int j = 0; j < nc; j++) {
            double k = kij[i * nc + j];
            if (!std::isfinite(k) || k != kij[j * nc + i] || (i == j && k != 0.0)) return PTF_ERR_INVALID_ARG;
        }
    }
    if (n < 0 || n > ptflash_noalloc_max_mixtures(nc)) return PTF_ERR_INVALID_ARG;
    if (n == 0) return PTF_OK;
    if (!P || !T || !z || !nphase || !beta || !x || !y || !K || !status) return PTF_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return PTF_ERR_CUDA;
    }
    void* base = nullptr;
    int sms = 0;
    int rc = setup(dev, &base, &sms);
    if (rc) return rc;
    CompHost h{};
    h.nc = nc;
    for (int i = 0; i < nc; i++) {
        h.Tc[i] = Tc[i];
        h.Pc[i] = Pc[i];
        h.om[i] = omega[i];
    }
    for (int i = 0; i < nc * nc; i++) h.kij[i] = kij[i];
    cudaStream_t s = (cudaStream_t)stream;
    WS ws = carve(static_cast<unsigned char*>(base), nc, n);
    IO io;
    io.ld = n;
    io.P = P;
    io.T = T;
    io.z = z;
    io.nphase = nphase;
    io.beta = beta;
    io.x = x;
    io.y = y;
    io.K = K;
    io.status = status;
    io.iters = iters;
    // the queue counters must start at zero on every call
    if (cudaMemsetAsync(ws.cnt, 0, 256, s) != cudaSuccess) {
        cudaGetLastError();
        return PTF_ERR_CUDA;
    }
    const int grid = sms * 8;
    cudaError_t e = cudaErrorInvalidValue;
    switch (nc) {
#define PTF_CASE(NC) \
    case NC: e = launch_plain<NC>(h, ws, io, grid, 0, s, nullptr); break;
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTF_ERR_CUDA;
    }
    return PTF_OK;
}
