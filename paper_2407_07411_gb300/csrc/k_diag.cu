// Diagonal of H_eff, the Davidson preconditioner's input: only groups whose output
// block is their input block (Delta = 0 in U(1); Delta n = 0 and unchanged spins in
// SU(2)) have diagonal entries, diag[(l, r)] = sum_t (scaled A_t)[l, l] B_t[r, r].
#include <cstdint>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"

namespace dmrg {
namespace {

// One CTA per block; the block's jobs are accumulated in job order by that CTA.  ops
// holds the layout entries from ops_lo on; only blocks whose first job's A stack lies
// in [lo, hi) are formed (a block's stacks lie in one window of the layout).
__global__ void k_diag(const DiagJob* __restrict__ jobs, const int32_t* __restrict__ first,
                       const double* __restrict__ ops, int64_t ops_lo, int64_t lo, int64_t hi,
                       double* __restrict__ diag) {
    const int32_t j0 = first[blockIdx.x], j1 = first[blockIdx.x + 1];
    if (j0 == j1) return;
    const DiagJob J0 = jobs[j0];
    if (J0.a_stack < lo || J0.a_stack >= hi) return;
    for (int64_t e = threadIdx.x; e < int64_t(J0.rows) * J0.cols; e += blockDim.x) {
        const int i = int(e / J0.cols), j = int(e % J0.cols);
        double s = 0.0;
        for (int32_t q = j0; q < j1; ++q) {
            const DiagJob J = jobs[q];
            double g = 0.0;
            for (int t = 0; t < J.n; ++t)
                g += ops[J.a_stack - ops_lo + int64_t(t) * J.rows * J.rows + int64_t(i) * J.rows + i] *
                     ops[J.b_stack - ops_lo + int64_t(t) * J.cols * J.cols + int64_t(j) * J.cols + j];
            s += J.sign * g;
        }
        diag[J0.off + e] = s;
    }
}

}  // namespace

cudaError_t Handle::launch_diag(const double* ops, int64_t ops_lo, int64_t lo, int64_t hi, double* diag,
                                cudaStream_t st) {
    if (plan.blocks.empty()) return cudaSuccess;
    const int32_t* first = reinterpret_cast<const int32_t*>(
        reinterpret_cast<const char*>(d_diag_jobs) + sizeof(DiagJob) * n_diag_jobs);
    k_diag<<<int(plan.blocks.size()), 256, 0, st>>>(d_diag_jobs, first, ops, ops_lo, lo, hi, diag);
    return cudaGetLastError();
}

int Handle::init_diag() {
    std::vector<DiagJob> jobs;
    std::vector<int32_t> first(1, 0);
    std::vector<std::vector<int32_t>> per_block(plan.blocks.size());
    for (int32_t g = 0; g < int32_t(plan.groups.size()); ++g) {
        const Group& G = plan.groups[g];
        if (G.in_block == G.out_block) per_block[G.in_block].push_back(g);   // U(1): Delta = 0
    }
    for (size_t k = 0; k < plan.blocks.size(); ++k) {
        for (int32_t g : per_block[k]) {
            const Group& G = plan.groups[g];
            jobs.push_back({G.a_stack, G.b_stack, plan.blocks[k].off, int32_t(G.terms.size()), G.a, G.c, 0,
                            G.sign});
        }
        first.push_back(int32_t(jobs.size()));
    }
    n_diag_jobs = int32_t(jobs.size());
    const size_t bytes = sizeof(DiagJob) * jobs.size() + sizeof(int32_t) * first.size();
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d_diag_jobs), bytes + 16);
    if (e != cudaSuccess) return cuda_fail(e, "diag jobs");
    e = cudaMemcpy(d_diag_jobs, jobs.data(), sizeof(DiagJob) * jobs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(reinterpret_cast<char*>(d_diag_jobs) + sizeof(DiagJob) * jobs.size(), first.data(),
                       sizeof(int32_t) * first.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "diag jobs");
    return DMRG_OK;
}

int Handle::diagonal(double* diag, cudaStream_t st) {
    if (plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    if (plan.dim == 0) return DMRG_OK;
    if (!diag) return fail(DMRG_ERR_INVALID_ARG, "null diag");
    cudaError_t e;
    if (d_diag) {   // split handles: formed while the operators were streamed in
        e = cudaMemcpyAsync(diag, d_diag, sizeof(double) * plan.dim, cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? DMRG_OK : cuda_fail(e, "copy diag");
    }
    e = cudaMemsetAsync(diag, 0, sizeof(double) * plan.dim, st);
    if (e != cudaSuccess) return cuda_fail(e, "zero diag");
    e = launch_diag(d_ops, 0, 0, INT64_MAX, diag, st);
    if (e != cudaSuccess) return cuda_fail(e, "diag kernel");
    return DMRG_OK;
}

}  // namespace dmrg
