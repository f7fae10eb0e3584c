// ptf_batch.cu -- uneven batches: many fluid systems, each with its own
// number of components and component data, flashed by one CUDA graph launch.
//
// The systems are grouped by nc.  Each group owns a component table (one
// Comp<nc> per system), a map from its mixtures to their systems, a workspace
// and staging buffers, and a stream.  One flash of the batch is, per group:
// zero the queue counters, gather the group's mixtures from the packed inputs
// into a contiguous component-major slice, run the flash pipeline with the
// ManySys component source, scatter the results to the packed outputs.  The
// groups are parallel branches of one captured graph, so the persistent
// kernels of different groups fill the GPU together and overlap their tails.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ptflash.h"
#include "ptf_launch.cuh"

using namespace ptf;

namespace {

struct SysDesc {
    int64_t off;     // first mixture of the system in P, T, nphase, beta, status, iters
    int64_t zoff;    // first element of the system's [nc][n] block in z, x, y, K
    int64_t n;       // mixtures of the system
    int64_t gstart;  // first mixture of the system in its group's slice
};

__global__ void k_fill_sys(int32_t* sys_of, int64_t gstart, int64_t n, int32_t j) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        sys_of[gstart + k] = j;
}

__global__ void k_gather(int nc, int64_t N, const int32_t* __restrict__ sys_of, const SysDesc* __restrict__ d,
                         const double* __restrict__ P, const double* __restrict__ T, const double* __restrict__ z,
                         double* gP, double* gT, double* gz) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        const SysDesc s = d[sys_of[g]];
        const int64_t m = g - s.gstart;
        gP[g] = P[s.off + m];
        gT[g] = T[s.off + m];
        for (int i = 0; i < nc; i++) gz[i * N + g] = z[s.zoff + i * s.n + m];
    }
}

__global__ void k_scatter(int nc, int64_t N, const int32_t* __restrict__ sys_of, const SysDesc* __restrict__ d,
                          const int32_t* gnp, const double* gb, const double* gx, const double* gy, const double* gK,
                          const int32_t* gst, const int32_t* git, int32_t* nphase, double* beta, double* x, double* y,
                          double* K, int32_t* status, int32_t* iters) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        const SysDesc s = d[sys_of[g]];
        const int64_t m = g - s.gstart, o = s.off + m;
        nphase[o] = gnp[g];
        beta[o] = gb[g];
        status[o] = gst[g];
        if (iters) iters[o] = git[g];
        for (int i = 0; i < nc; i++) {
            const int64_t zo = s.zoff + i * s.n + m;
            x[zo] = gx[i * N + g];
            y[zo] = gy[i * N + g];
            K[zo] = gK[i * N + g];
        }
    }
}

struct Group {
    int nc = 0;
    int64_t N = 0;                // mixtures of the group
    std::vector<int> sys;         // systems of the batch in this group
    void* tab = nullptr;          // device Comp<nc>[sys.size()]
    SysDesc* desc = nullptr;      // device [sys.size()]
    int32_t* sys_of = nullptr;    // device [N]
    double* wsd = nullptr;        // workspace doubles, (8 nc + 3) N
    int32_t* wsi = nullptr;       // workspace ints, 8 N + 64
    double* sd = nullptr;         // staging doubles: P, T [N]; z, x, y, K [nc N]; beta [N]
    int32_t* si = nullptr;        // staging ints: nphase, status, iters [N]
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    int pgrid = 0;                // persistent-kernel blocks (0: device-filling default)
    int bps = 0;                  // the tuned blocks per SM behind pgrid (0: default)

    WS ws() const {
        WS w;
        w.n = N;
        double* p = wsd;
        w.sA = p; p += (int64_t)nc * N;
        w.B = p; p += (int64_t)nc * N;
        w.lnz = p; p += (int64_t)nc * N;
        w.d = p; p += (int64_t)nc * N;
        w.lnK = p; p += (int64_t)nc * N;
        w.nV = p; p += (int64_t)nc * N;
        w.lnW = p; p += 2 * (int64_t)nc * N;
        w.theta = p; p += N;
        w.tm = p; p += 2 * N;
        int32_t* q = wsi;
        w.cnt = q; q += 64;
        w.tflag = q; q += 2 * N;
        w.q_stab = q; q += N;
        w.q_split = q; q += N;
        w.q_stab_tr = q; q += 2 * N;
        w.q_split_tr = q; q += N;
        w.q_sort = q; q += N;
        return w;
    }
    IO io() const {
        IO o;
        o.ld = N;
        double* p = sd;
        o.P = p; p += N;
        o.T = p; p += N;
        o.z = p; p += (int64_t)nc * N;
        o.x = p; p += (int64_t)nc * N;
        o.y = p; p += (int64_t)nc * N;
        o.K = p; p += (int64_t)nc * N;
        o.beta = p;
        o.nphase = si;
        o.status = si + N;
        o.iters = si + 2 * N;
        return o;
    }
};

int validate(int nc, const double* Tc, const double* Pc, const double* om, const double* kij) {
    if (nc < 2 || nc > 16) return PTF_ERR_UNSUPPORTED;
    for (int i = 0; i < nc; i++) {
        if (!(Tc[i] > 0.0) || !(Pc[i] > 0.0) || !std::isfinite(Tc[i]) || !std::isfinite(Pc[i]) ||
            !std::isfinite(om[i]))
            return PTF_ERR_INVALID_ARG;
        for (int j = 0; j < nc; j++) {
            const double k = kij[i * nc + j];
            if (!std::isfinite(k) || k != kij[j * nc + i] || (i == j && k != 0.0)) return PTF_ERR_INVALID_ARG;
        }
    }
    return PTF_OK;
}

// Host image of a group's component table.
template <int NC>
std::vector<unsigned char> table(const std::vector<CompHost>& hs) {
    std::vector<unsigned char> b(hs.size() * sizeof(Comp<NC>));
    for (size_t k = 0; k < hs.size(); k++) {
        const Comp<NC> c = make_comp<NC>(hs[k]);
        std::memcpy(b.data() + k * sizeof(Comp<NC>), &c, sizeof(Comp<NC>));
    }
    return b;
}

std::vector<unsigned char> table_for(int nc, const std::vector<CompHost>& hs) {
    switch (nc) {
#define PTF_CASE(NC) \
    case NC: return table<NC>(hs);
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
    }
    return {};
}

cudaError_t pipeline(const Group& g, int grid, cudaStream_t s) {
    const WS ws = g.ws();
    const IO io = g.io();
    switch (g.nc) {
#define PTF_CASE(NC) \
    case NC: return launch_many<NC>(static_cast<const Comp<NC>*>(g.tab), g.sys_of, ws, io, grid, 0, g.pgrid, s);
        PTF_CASE(2) PTF_CASE(3) PTF_CASE(4) PTF_CASE(5) PTF_CASE(6) PTF_CASE(7) PTF_CASE(8) PTF_CASE(9)
        PTF_CASE(10) PTF_CASE(11) PTF_CASE(12) PTF_CASE(13) PTF_CASE(14) PTF_CASE(15) PTF_CASE(16)
#undef PTF_CASE
    }
    return cudaErrorInvalidValue;
}

struct Args {
    const double *P, *T, *z;
    int32_t* nphase;
    double *beta, *x, *y, *K;
    int32_t *status, *iters;
    bool operator==(const Args& o) const { return std::memcmp(this, &o, sizeof(Args)) == 0; }
};

}  // namespace

struct ptflash_batch {
    int device = 0, sm_count = 0, nsys = 0;
    int64_t N = 0;
    std::vector<Group> groups;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
    Args key{};

    // One group's flash on stream s: counters, gather, pipeline, scatter.
    cudaError_t enqueue(const Group& g, const Args& a, cudaStream_t s) const {
        const int grid = sm_count * 8;
        const IO io = g.io();
        cudaError_t e = cudaMemsetAsync(g.wsi, 0, 64 * sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
        k_gather<<<grid, 256, 0, s>>>(g.nc, g.N, g.sys_of, g.desc, a.P, a.T, a.z, const_cast<double*>(io.P),
                                      const_cast<double*>(io.T), const_cast<double*>(io.z));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = pipeline(g, grid, s)) != cudaSuccess) return e;
        k_scatter<<<grid, 256, 0, s>>>(g.nc, g.N, g.sys_of, g.desc, io.nphase, io.beta, io.x, io.y, io.K, io.status,
                                       io.iters, a.nphase, a.beta, a.x, a.y, a.K, a.status, a.iters);
        return cudaGetLastError();
    }

    cudaError_t capture(const Args& a) {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        cudaError_t q = cudaEventRecord(fork, cap);
        for (const Group& g : groups) {
            if (q != cudaSuccess) break;
            if ((q = cudaStreamWaitEvent(g.st, fork, 0)) != cudaSuccess) break;
            if ((q = enqueue(g, a, g.st)) != cudaSuccess) break;
            if ((q = cudaEventRecord(g.done, g.st)) != cudaSuccess) break;
            q = cudaStreamWaitEvent(cap, g.done, 0);
        }
        e = cudaStreamEndCapture(cap, &graph);
        if (q != cudaSuccess) e = q;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nullptr, &nodes);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess && exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        key = a;
        return e;
    }
};

namespace {
void release(ptflash_batch* b) {
    for (Group& g : b->groups) {
        cudaFree(g.tab);
        cudaFree(g.desc);
        cudaFree(g.sys_of);
        cudaFree(g.wsd);
        cudaFree(g.wsi);
        cudaFree(g.sd);
        cudaFree(g.si);
        if (g.st) cudaStreamDestroy(g.st);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

int check_args(const ptflash_batch* b, const Args& a) {
    if (!b) return PTF_ERR_INVALID_ARG;
    if (b->N == 0) return PTF_OK;
    if (!a.P || !a.T || !a.z || !a.nphase || !a.beta || !a.x || !a.y || !a.K || !a.status) return PTF_ERR_INVALID_ARG;
    return PTF_OK;
}
}  // namespace

extern "C" {

int ptflash_batch_create(ptflash_batch** out, int nsys, const int32_t* nc, const int64_t* n, const double* Tc,
                         const double* Pc, const double* omega, const double* kij) {
    if (!out) return PTF_ERR_INVALID_ARG;
    *out = nullptr;
    if (nsys < 1 || nsys > (1 << 20) || !nc || !n || !Tc || !Pc || !omega || !kij) return PTF_ERR_INVALID_ARG;
    std::vector<CompHost> hs(nsys);
    std::vector<int64_t> off(nsys), zoff(nsys);
    int64_t N = 0, Z = 0, ci = 0, ki = 0;
    for (int s = 0; s < nsys; s++) {
        int rc = validate(nc[s], Tc + ci, Pc + ci, omega + ci, kij + ki);
        if (rc) return rc;
        if (n[s] < 0 || n[s] > ((int64_t)1 << 30)) return PTF_ERR_INVALID_ARG;
        CompHost& h = hs[s];
        h = CompHost{};
        h.nc = nc[s];
        for (int i = 0; i < nc[s]; i++) {
            h.Tc[i] = Tc[ci + i];
            h.Pc[i] = Pc[ci + i];
            h.om[i] = omega[ci + i];
        }
        for (int i = 0; i < nc[s] * nc[s]; i++) h.kij[i] = kij[ki + i];
        ci += nc[s];
        ki += (int64_t)nc[s] * nc[s];
        off[s] = N;
        zoff[s] = Z;
        N += n[s];
        Z += (int64_t)nc[s] * n[s];
    }
    ptflash_batch* b = new (std::nothrow) ptflash_batch();
    if (!b) return PTF_ERR_NO_MEMORY;
    b->nsys = nsys;
    b->N = N;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    // one group per nc present with at least one mixture, in decreasing nc
    // (the slowest groups start first)
    for (int k = 16; k >= 2 && e == cudaSuccess; k--) {
        Group g;
        g.nc = k;
        for (int s = 0; s < nsys; s++)
            if (nc[s] == k && n[s] > 0) {
                g.sys.push_back(s);
                g.N += n[s];
            }
        if (g.sys.empty()) continue;
        if (g.N > ((int64_t)1 << 30)) {
            release(b);
            return PTF_ERR_INVALID_ARG;
        }
        b->groups.push_back(g);
        Group& G = b->groups.back();
        std::vector<CompHost> gh;
        std::vector<SysDesc> d;
        int64_t gs = 0;
        for (int s : G.sys) {
            gh.push_back(hs[s]);
            d.push_back(SysDesc{off[s], zoff[s], n[s], gs});
            gs += n[s];
        }
        const std::vector<unsigned char> tab = table_for(k, gh);
        const int64_t N_ = G.N;
        if ((e = cudaMalloc(&G.tab, tab.size())) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.desc, d.size() * sizeof(SysDesc))) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.sys_of, N_ * sizeof(int32_t))) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.wsd, (size_t)(8 * k + 3) * N_ * sizeof(double))) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.wsi, (size_t)(8 * N_ + 64) * sizeof(int32_t))) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.sd, (size_t)(4 * k + 3) * N_ * sizeof(double))) != cudaSuccess) break;
        if ((e = cudaMalloc(&G.si, (size_t)3 * N_ * sizeof(int32_t))) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaMemcpy(G.tab, tab.data(), tab.size(), cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMemcpy(G.desc, d.data(), d.size() * sizeof(SysDesc), cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        for (size_t j = 0; j < d.size() && e == cudaSuccess; j++) {
            k_fill_sys<<<b->sm_count * 4, 256, 0, G.st>>>(G.sys_of, d[j].gstart, d[j].n, (int32_t)j);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(G.st);
    }
    if (e != cudaSuccess) {
        const int rc = (e == cudaErrorMemoryAllocation) ? PTF_ERR_NO_MEMORY : PTF_ERR_CUDA;
        cudaGetLastError();
        release(b);
        return rc;
    }
    *out = b;
    return PTF_OK;
}

int ptflash_batch_destroy(ptflash_batch* b) {
    if (!b) return PTF_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    release(b);
    return PTF_OK;
}

int ptflash_batch_flash(ptflash_batch* b, const double* P, const double* T, const double* z, int32_t* nphase,
                        double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                        void* stream) {
    const Args a{P, T, z, nphase, beta, x, y, K, status, iters};
    int rc = check_args(b, a);
    if (rc || b->N == 0) return rc;
    if (!b->exec || !(b->key == a)) {
        if (b->capture(a) != cudaSuccess) {
            cudaGetLastError();
            return PTF_ERR_CUDA;
        }
    }
    if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return PTF_ERR_CUDA;
    }
    return PTF_OK;
}

int ptflash_batch_tune(ptflash_batch* b, const double* P, const double* T, const double* z, int32_t* nphase,
                       double* beta, double* x, double* y, double* K, int32_t* status, int32_t* iters,
                       int32_t* blocks_per_sm, float* group_ms) {
    const Args a{P, T, z, nphase, beta, x, y, K, status, iters};
    int rc = check_args(b, a);
    if (rc) return rc;
    if (blocks_per_sm)
        for (int k = 0; k < 17; k++) blocks_per_sm[k] = 0;
    if (group_ms)
        for (int k = 0; k < 17; k++) group_ms[k] = 0.0f;
    if (b->N == 0) return PTF_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return PTF_ERR_CUDA;
    }
    // candidates: the default (each persistent kernel as many blocks as fit),
    // and 1, 2, 3 or 4 resident 128-thread blocks per SM for all of them
    const int cand[5] = {0, 1, 2, 3, 4};
    cudaError_t e = cudaSuccess;
    for (Group& g : b->groups) {
        float best = 1e30f;
        int best_b = 0;
        for (int c = 0; c < 5 && e == cudaSuccess; c++) {
            g.pgrid = cand[c] * b->sm_count;
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
                e = cudaEventRecord(e0, g.st);
                if (e == cudaSuccess) e = b->enqueue(g, a, g.st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, g.st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float t = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                if (e == cudaSuccess && t < ms) ms = t;
            }
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_b = cand[c];
            }
        }
        g.bps = best_b;
        g.pgrid = best_b * b->sm_count;
        if (blocks_per_sm) blocks_per_sm[g.nc] = best_b;
        if (group_ms) group_ms[g.nc] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->exec) {  // the captured graph holds the old grids
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PTF_ERR_CUDA;
    }
    return PTF_OK;
}

int ptflash_batch_info(const ptflash_batch* b, int32_t* ngroups, int64_t* graph_nodes, int64_t* mixtures) {
    if (!b) return PTF_ERR_INVALID_ARG;
    if (ngroups) *ngroups = (int32_t)b->groups.size();
    if (graph_nodes) *graph_nodes = (int64_t)b->nodes;
    if (mixtures) *mixtures = b->N;
    return PTF_OK;
}

}  // extern "C"
