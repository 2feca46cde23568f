// Per-kernel launch accounting (CUDA-event timing on the launching stream) and the
// FP64 DMMA peak probe.
#include <cstring>
#include <vector>

#include "../../include/dmrg_profile.h"
#include "handle.h"

namespace dmrg {

int Profiler::kernel_id(const char* name) {
    for (size_t i = 0; i < names.size(); ++i)
        if (names[i] == name) return int(i);
    names.emplace_back(name);
    launches.push_back(0); flops.push_back(0); bytes.push_back(0); ms.push_back(0);
    return int(names.size() - 1);
}

cudaEvent_t Profiler::take_event() {
    if (pool_used < pool.size()) return pool[pool_used++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
    ++pool_used;
    return e;
}

void Profiler::begin(int id, cudaStream_t st, double f, double b, Pending* p) {
    p->id = id; p->start = p->stop = nullptr;
    if (!counting) {   // capturing a graph: remember the launch, count it at replay
        cap_kids.push_back(id); cap_flops.push_back(f); cap_bytes.push_back(b);
        return;
    }
    launches[id] += 1; flops[id] += f; bytes[id] += b;
    if (!timing) return;
    p->start = take_event();
    if (p->start) cudaEventRecord(p->start, st);
}

void Profiler::end(const Pending& p, cudaStream_t st) {
    if (!timing || !p.start) return;
    cudaEvent_t e = take_event();
    if (!e) return;
    cudaEventRecord(e, st);
    recs.push_back({p.id, p.start, e});
}

void Profiler::reset() {
    for (auto& v : launches) v = 0;
    for (auto& v : flops) v = 0;
    for (auto& v : bytes) v = 0;
    for (auto& v : ms) v = 0;
    recs.clear();
    pool_used = 0;
}

int Profiler::collect() {
    for (const Rec& r : recs) {
        if (cudaEventSynchronize(r.stop) != cudaSuccess) return DMRG_ERR_CUDA;
        float t = 0;
        if (cudaEventElapsedTime(&t, r.start, r.stop) == cudaSuccess) ms[r.id] += t;
    }
    recs.clear();
    pool_used = 0;
    return DMRG_OK;
}

Profiler::~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

namespace {

__global__ void k_dmma_peak(double* out, int iters) {
    double a[8], b[4];
    for (int i = 0; i < 8; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int i = 0; i < 4; ++i) b[i] = 1.0 - 1e-3 * (threadIdx.x + i);
    double c[2][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
                "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
                : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                  "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = c[0][0] + c[0][1] + c[0][2] + c[0][3] + c[1][0] +
                                                 c[1][1] + c[1][2] + c[1][3];
}

}  // namespace
}  // namespace dmrg

using dmrg::Handle;

extern "C" {

int dmrg_heff_profile(dmrg_heff_t hh, int32_t enable) {
    if (!hh) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null handle");
    Handle* h = static_cast<Handle*>(hh);
    h->prof.collect();
    h->prof.reset();
    h->prof.timing = enable != 0;
    return DMRG_OK;
}

int dmrg_heff_profile_read(dmrg_heff_t hh, dmrg_kernel_stat* stats, int32_t* n) {
    if (!hh || !n) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    Handle* h = static_cast<Handle*>(hh);
    if (h->prof.collect() != DMRG_OK) return dmrg::fail(DMRG_ERR_CUDA, "event synchronize");
    const int32_t k = int32_t(h->prof.names.size());
    if (stats) {
        if (*n < k) return dmrg::fail(DMRG_ERR_INVALID_ARG, "stats buffer too small");
        for (int32_t i = 0; i < k; ++i) {
            std::memset(stats[i].name, 0, sizeof(stats[i].name));
            std::strncpy(stats[i].name, h->prof.names[i].c_str(), sizeof(stats[i].name) - 1);
            stats[i].launches = h->prof.launches[i];
            stats[i].ms_total = h->prof.ms[i];
            stats[i].flops_total = h->prof.flops[i];
            stats[i].bytes_total = h->prof.bytes[i];
        }
    }
    *n = k;
    return DMRG_OK;
}

int dmrg_probe_fp64_peak(double* tflops) {
    if (!tflops) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "device query");
    const int threads = 256, blocks = sms * 4, iters = 2048;
    double* out = nullptr;
    e = cudaMalloc(&out, sizeof(double) * threads * blocks);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "probe buffer");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dmrg::k_dmma_peak<<<blocks, threads>>>(out, iters);  // warm-up
    cudaEventRecord(e0);
    const int reps = 3;
    for (int r = 0; r < reps; ++r) dmrg::k_dmma_peak<<<blocks, threads>>>(out, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "probe");
    // 2 MMAs of 2*16*8*16 flops per warp per iteration
    const double flops = double(reps) * blocks * (threads / 32) * iters * 2.0 * 4096.0;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return DMRG_OK;
}

}  // extern "C"
