// Set-up kernels: the node coefficient w = omega^2 m^2 of Eq. 2 from the
// slowness, its injection onto coarser levels, and the launch counter.
#include <atomic>
#include <cstring>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "helm_internal.cuh"

namespace helm {

namespace {
std::atomic<uint64_t> g_launches{0};

struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
    double bytes, flops;
};
struct Prof {
    std::mutex mu;
    bool on = false;
    bool capturing = false;             // records go to `captured` (event nodes in a graph)
    std::vector<ProfRec> recs;
    std::vector<ProfRec> captured;
    std::map<std::string, double[3]> graph_agg;   // name -> ms, bytes, flops of replays
    std::map<std::string, uint64_t> graph_cnt;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t pending = nullptr;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
} g_prof;

__global__ void k_make_w(const double *__restrict__ m, size_t n, double om2,
                         double *__restrict__ w64, float *__restrict__ w32, int *__restrict__ flag) {
    int bad = 0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (size_t)gridDim.x * blockDim.x) {
        const double v = m[p];
        bad |= !(isfinite(v) && v > 0.0);
        const double w = om2 * v * v;
        w64[p] = w;
        if (w32) w32[p] = __double2float_rn(w);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void k_make_rho(const double *__restrict__ rho, size_t n, float *__restrict__ rho32,
                           int *__restrict__ flag) {
    int bad = 0;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (size_t)gridDim.x * blockDim.x) {
        const double v = rho[p];
        bad |= !(isfinite(v) && v > 0.0);
        rho32[p] = __double2float_rn(v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0 && flag) atomicOr(flag, 1);
}

template <typename T>
__global__ void k_inject(const T *__restrict__ fine, int fnx, int fny, T *__restrict__ coarse,
                         int cnx, int cny, int cnz) {
    const size_t n = (size_t)cnx * cny * cnz;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const int I = (int)(q % cnx);
        const int J = (int)((q / cnx) % cny);
        const int K = (int)(q / ((size_t)cnx * cny));
        coarse[q] = fine[((size_t)(2 * K) * fny + 2 * J) * fnx + 2 * I];
    }
}
}  // namespace

int device_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 152;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

void count_launch(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
void uncount_launch(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

bool prof_on() { return g_prof.on; }

void prof_begin(cudaStream_t st) {
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.pending = g_prof.get();
    if (g_prof.capturing)
        cudaEventRecordWithFlags(g_prof.pending, st, cudaEventRecordExternal);
    else
        cudaEventRecord(g_prof.pending, st);
}

void prof_end(const char *name, cudaStream_t st, double bytes, double flops64) {
    if (!g_prof.on || !g_prof.pending) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e1 = g_prof.get();
    if (g_prof.capturing) {
        cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal);
        g_prof.captured.push_back({name, g_prof.pending, e1, bytes, flops64});
    } else {
        cudaEventRecord(e1, st);
        g_prof.recs.push_back({name, g_prof.pending, e1, bytes, flops64});
    }
    g_prof.pending = nullptr;
}

void prof_capture_begin() {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.capturing = true;
    g_prof.captured.clear();
}

std::vector<ProfRecPublic> prof_capture_end() {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.capturing = false;
    std::vector<ProfRecPublic> out;
    for (auto &r : g_prof.captured) out.push_back({r.name, r.e0, r.e1, r.bytes, r.flops});
    g_prof.captured.clear();
    return out;
}

void prof_graph_replayed(const std::vector<ProfRecPublic> &recs) {
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto &r : recs) {
        if (cudaEventSynchronize(r.e1) != cudaSuccess) return;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        auto &a = g_prof.graph_agg[r.name];
        a[0] += ms;
        a[1] += r.bytes;
        a[2] += r.flops;
        g_prof.graph_cnt[r.name] += 1;
    }
}

void launch_make_w(const double *m, size_t n, double omega, double *w64, float *w32, int *flag,
                   cudaStream_t st) {
    size_t b = (n + 255) / 256;
    int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_make_w<<<nb, 256, 0, st>>>(m, n, omega * omega, w64, w32, flag);
    count_launch();
}

void launch_make_rho(const double *rho64, size_t n, float *rho32, int *flag, cudaStream_t st) {
    size_t b = (n + 255) / 256;
    int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_make_rho<<<nb, 256, 0, st>>>(rho64, n, rho32, flag);
    count_launch();
}

template <typename T>
void launch_inject(const T *fine, int fnx, int fny, T *coarse, int cnx, int cny, int cnz,
                   cudaStream_t st) {
    size_t n = (size_t)cnx * cny * cnz;
    size_t b = (n + 255) / 256;
    int nb = (int)(b < 4096 ? (b ? b : 1) : 4096);
    k_inject<T><<<nb, 256, 0, st>>>(fine, fnx, fny, coarse, cnx, cny, cnz);
    count_launch();
}

template void launch_inject<float>(const float *, int, int, float *, int, int, int, cudaStream_t);
template void launch_inject<double>(const double *, int, int, double *, int, int, int,
                                    cudaStream_t);

}  // namespace helm

extern "C" {

helm_status helm_profile_start(void) {
    std::lock_guard<std::mutex> lk(helm::g_prof.mu);
    for (auto &r : helm::g_prof.recs) {
        helm::g_prof.pool.push_back(r.e0);
        helm::g_prof.pool.push_back(r.e1);
    }
    helm::g_prof.recs.clear();
    helm::g_prof.graph_agg.clear();
    helm::g_prof.graph_cnt.clear();
    helm::g_prof.on = true;
    return HELM_OK;
}

helm_status helm_profile_stop(char *json, size_t cap) {
    std::lock_guard<std::mutex> lk(helm::g_prof.mu);
    helm::g_prof.on = false;
    struct Agg { uint64_t n = 0; double ms = 0, bytes = 0, flops = 0; };
    std::map<std::string, Agg> agg;
    for (auto &r : helm::g_prof.recs) {
        if (cudaEventSynchronize(r.e1) != cudaSuccess) return HELM_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        Agg &a = agg[r.name];
        a.n += 1;
        a.ms += ms;
        a.bytes += r.bytes;
        a.flops += r.flops;
    }
    for (auto &kv : helm::g_prof.graph_agg) {
        Agg &a = agg[kv.first];
        a.n += helm::g_prof.graph_cnt[kv.first];
        a.ms += kv.second[0];
        a.bytes += kv.second[1];
        a.flops += kv.second[2];
    }
    std::string out = "{";
    bool first = true;
    for (auto &kv : agg) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s\"%s\": {\"launches\": %llu, \"ms\": %.6f, \"bytes\": %.6e, "
                 "\"flops64\": %.6e}", first ? "" : ", ", kv.first.c_str(),
                 (unsigned long long)kv.second.n, kv.second.ms, kv.second.bytes, kv.second.flops);
        out += buf;
        first = false;
    }
    out += "}";
    if (!json || cap < out.size() + 1) return HELM_ERR_ARG;
    memcpy(json, out.c_str(), out.size() + 1);
    return HELM_OK;
}

}  // extern "C"
