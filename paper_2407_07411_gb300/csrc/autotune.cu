// Schedule of the grouped GEMMs and its autotuner.
//
// A schedule fixes how the planned GEMMs are cut into work items (the K extent of a
// stage-2 item, per shape class of contraction length, and the output tile of the FP64
// kernel), how many CTAs of the FP64 tile kernel share an SM, and whether each grouped
// GEMM runs as one persistent launch of its stage or as a launch of its own.  The autotuner measures candidate schedules
// on the handle's own plan with CUDA events (coordinate descent: one parameter at a
// time, every candidate of it, the fastest kept) and leaves the best one in place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "split.h"

namespace dmrg {
namespace {

// Deterministic test vectors for timing (values of unit magnitude, no zeros).
__global__ void k_fill_probe(double* x, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t h = uint32_t(i) * 2654435761u ^ uint32_t(i >> 32) * 40503u;
        x[i] = (double(h >> 8) + 0.5) * (1.0 / 16777216.0) - 0.5;
    }
}

Schedule from_abi(const dmrg_schedule& a) {
    Schedule s;
    for (int c = 0; c < N_KCLASS; ++c) {
        s.fp64_kchunk[c] = a.fp64_kchunk[c];
        s.split_kchunk[c] = a.split_kchunk[c];
    }
    s.fp64_ctas_per_sm = a.fp64_ctas_per_sm;
    s.per_gemm = a.per_gemm;
    s.fp64_tile = a.fp64_tile;
    return s;
}

dmrg_schedule to_abi(const Schedule& s) {
    dmrg_schedule a;
    std::memset(&a, 0, sizeof(a));
    for (int c = 0; c < N_KCLASS; ++c) {
        a.fp64_kchunk[c] = s.fp64_kchunk[c];
        a.split_kchunk[c] = s.split_kchunk[c];
    }
    a.fp64_ctas_per_sm = s.fp64_ctas_per_sm;
    a.per_gemm = s.per_gemm;
    a.fp64_tile = s.fp64_tile;
    return a;
}

}  // namespace

// Shape classes of stage 2 that hold at least one GEMM (for the vectors of plan nv).
static std::vector<int> present_classes(const Handle& h, int nv) {
    std::vector<char> has(N_KCLASS, 0);
    if (h.precision == DMRG_PREC_FP64) {
        for (int32_t g : h.plan.s2gemms) has[size_t(kclass(h.plan.gemms[size_t(g)].K))] = 1;
    } else if (h.split_plan_host(nv)) {
        for (const SGemm& m : h.split_plan_host(nv)->gemms)
            if (m.kind == 1) has[size_t(kclass(int64_t(m.kt) * SPL_TK))] = 1;
    }
    std::vector<int> out;
    for (int c = 0; c < N_KCLASS; ++c)
        if (has[size_t(c)]) out.push_back(c);
    return out;
}

int Handle::autotune(int32_t nvec, int32_t reps, dmrg_tune_report* rep) {
    if (plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    if (nvec < 1 || nvec > max_nvec) return fail(DMRG_ERR_INVALID_ARG, "nvec outside [1, max_nvec]");
    if (reps < 1 || reps > 100) return fail(DMRG_ERR_INVALID_ARG, "reps outside [1, 100]");
    std::memset(rep, 0, sizeof(*rep));
    rep->nvec = nvec;
    if (plan.dim == 0) {
        rep->best = to_abi(sched);
        rep->tile_m = precision == DMRG_PREC_FP64 ? FP64_TILE_M[sched.fp64_tile] : SPL_TM;
        rep->tile_n = precision == DMRG_PREC_FP64 ? FP64_TILE_N[sched.fp64_tile] : SPL_TN;
        return DMRG_OK;
    }
    double* x = nullptr;
    double* y = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t n = size_t(plan.dim) * size_t(nvec);
    cudaError_t e = cudaMalloc(&x, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fill_probe<<<unsigned(std::min<int64_t>(int64_t(n_sm) * 8, (int64_t(n) + 255) / 256)), 256, 0, st>>>(
            x, int64_t(n));
        e = cudaGetLastError();
    }
    int rc = e == cudaSuccess ? int(DMRG_OK) : cuda_fail(e, "autotune set-up");
    const Schedule start = sched;
    // median time of `reps` applies under schedule s (after one untimed apply)
    auto measure = [&](const Schedule& s, double* ms) {
        int r = set_schedule(s);
        if (r != DMRG_OK) return r;
        if ((r = apply_direct(x, y, nvec, st)) != DMRG_OK) return r;
        std::vector<float> t(static_cast<size_t>(reps));
        for (int i = 0; i < reps; ++i) {
            cudaEventRecord(e0, st);
            if ((r = apply_direct(x, y, nvec, st)) != DMRG_OK) return r;
            cudaEventRecord(e1, st);
            cudaError_t ee = cudaEventSynchronize(e1);
            if (ee != cudaSuccess) return cuda_fail(ee, "autotune timing");
            cudaEventElapsedTime(&t[size_t(i)], e0, e1);
        }
        if ((r = check_status()) != DMRG_OK) return r;
        std::sort(t.begin(), t.end());
        *ms = double(t[t.size() / 2]);
        rep->trials += 1;
        return int(DMRG_OK);
    };
    Schedule best = start;
    double best_ms = 0.0;
    if (rc == DMRG_OK) rc = measure(best, &best_ms);
    rep->default_ms = best_ms;
    // one parameter at a time: its candidates with the others at their best so far
    auto tune = [&](int32_t* field, const std::vector<int32_t>& cands) {
        const int32_t keep = *field;
        int32_t choice = keep;
        for (int32_t v : cands) {
            if (rc != DMRG_OK) return;
            if (v == keep) continue;
            *field = v;
            double ms = 0.0;
            rc = measure(best, &ms);
            if (rc == DMRG_OK && ms < best_ms) {
                best_ms = ms;
                choice = v;
            }
        }
        *field = choice;
    };
    const std::vector<int> classes = present_classes(*this, nvec);
    if (precision == DMRG_PREC_FP64) {
        tune(&best.fp64_tile, {0, 1, 2});
        for (int c : classes) tune(&best.fp64_kchunk[c], {256, 512, 1024, 2048, 4096, 0});
        std::vector<int32_t> ctas;
        for (int32_t v : {2, 4, 8, 16})
            if (v < tiles_per_sm[best.fp64_tile]) ctas.push_back(v);
        ctas.push_back(0);
        tune(&best.fp64_ctas_per_sm, ctas);
    } else {
        for (int c : classes) tune(&best.split_kchunk[c], {0, 16, 32, 64, 128, 256});
    }
    // leave the best schedule in place (or the starting one after an error)
    const int rc2 = set_schedule(rc == DMRG_OK ? best : start);
    if (rc == DMRG_OK) rc = rc2;
    rep->best_ms = best_ms;
    rep->best = to_abi(sched);
    rep->tile_m = precision == DMRG_PREC_FP64 ? FP64_TILE_M[sched.fp64_tile] : SPL_TM;
    rep->tile_n = precision == DMRG_PREC_FP64 ? FP64_TILE_N[sched.fp64_tile] : SPL_TN;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    return rc;
}

}  // namespace dmrg

using dmrg::Handle;

extern "C" {

int dmrg_heff_schedule_get(dmrg_heff_t h, dmrg_schedule* s) {
    if (!h || !s) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    *s = dmrg::to_abi(static_cast<Handle*>(h)->sched);
    return DMRG_OK;
}

int dmrg_heff_schedule_set(dmrg_heff_t h, const dmrg_schedule* s) {
    if (!h || !s) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    return static_cast<Handle*>(h)->set_schedule(dmrg::from_abi(*s));
}

int dmrg_heff_gemm_count(dmrg_heff_t h, int32_t nvec, int64_t counts[2]) {
    if (!h || !counts) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    const Handle* H = static_cast<Handle*>(h);
    if (nvec < 1 || nvec > H->max_nvec) return dmrg::fail(DMRG_ERR_INVALID_ARG, "nvec outside [1, max_nvec]");
    counts[0] = counts[1] = 0;
    const dmrg::SplitHost* sp = H->split_plan_host(nvec);
    if (H->precision == DMRG_PREC_SPLIT_BF16 && sp) {
        for (const dmrg::SGemm& m : sp->gemms) counts[m.kind == 0 ? 0 : 1] += 1;
    } else {
        counts[0] = int64_t(H->plan.s1gemms.size());
        counts[1] = int64_t(H->plan.s2gemms.size());
    }
    return DMRG_OK;
}

int dmrg_heff_autotune(dmrg_heff_t h, int32_t nvec, int32_t reps, dmrg_tune_report* report) {
    if (!h || !report) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    return static_cast<Handle*>(h)->autotune(nvec, reps, report);
}

}  // extern "C"
