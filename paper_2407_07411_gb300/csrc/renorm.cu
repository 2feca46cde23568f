// Operator renormalisation: O'[p <- q] = U_p^T O[p <- q] U_q for a list of operator
// blocks, with per-sector bases U_q (d_q x d'_q, orthonormal columns in the DMRG use:
// the truncated basis of the enlarged block).  Two stages of the FP64 grouped tile
// kernel, one persistent launch each over every block:
//   stage 1  X_b = O_b U_q        (d_p x d'_q, K = d_q)
//   stage 2  O'_b = U_p^T X_b     (d'_p x d'_q, K = d_p; U^T copied once per sector)
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "kernels.h"
#include "plan.h"

namespace dmrg {
namespace {

// UT (per sector d'_q x d_q, row-major) from U (d_q x d'_q); one block per sector
__global__ void k_transpose_bases(const double* __restrict__ U, double* __restrict__ UT, const int64_t* __restrict__ off,
                                  const int32_t* __restrict__ d, const int32_t* __restrict__ dn) {
    const int q = blockIdx.x;
    const int64_t o = off[q];
    const int rows = d[q], cols = dn[q];
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
        const int i = e / cols, j = e % cols;
        UT[o + int64_t(j) * rows + i] = U[o + e];
    }
}

struct Bufs {
    std::vector<void*> p;
    ~Bufs() {
        for (void* q : p)
            if (q) cudaFree(q);
    }
    template <class T>
    int alloc(T** out, size_t n, const char* what) {
        *out = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(out), sizeof(T) * (n > 0 ? n : 1));
        if (e != cudaSuccess) return cuda_fail(e, what);
        p.push_back(*out);
        return DMRG_OK;
    }
    template <class T>
    int upload(T** out, const std::vector<T>& v, const char* what) {
        int rc = alloc(out, v.size(), what);
        if (rc || v.empty()) return rc;
        cudaError_t e = cudaMemcpy(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? int(DMRG_OK) : cuda_fail(e, what);
    }
};

}  // namespace
}  // namespace dmrg

namespace dmrg {

// A renormalisation plan: the GEMM lists of one block list and the device buffers its
// launches need, built once and run any number of times.
struct RenormPlan {
    Plan P;
    int32_t nsec = 0;
    int64_t nu = 0, op_len = 0, out_len = 0;
    int n_sm = 152;
    Bufs B;
    double *uu = nullptr, *X = nullptr, *part = nullptr;
    Tile *t1 = nullptr, *t2 = nullptr;
    Gemm* gm = nullptr;
    Seg* sg = nullptr;
    Reduce* red = nullptr;
    int32_t* counters = nullptr;
    int64_t* d_uoff = nullptr;
    int32_t *d_d = nullptr, *d_dn = nullptr;
};

}  // namespace dmrg

extern "C" int dmrg_renorm_create(int32_t nsec, const int32_t* dims, const int32_t* dims_new, const int64_t* blocks,
                                  int64_t n_blocks, int64_t op_len, int64_t out_len, int64_t* out_off,
                                  dmrg_renorm_t* plan) {
    using namespace dmrg;
    // ---- validation (host only, before any device work)
    if (!plan) return fail(DMRG_ERR_INVALID_ARG, "null plan");
    *plan = nullptr;
    if (nsec < 1 || n_blocks < 0 || op_len < 0 || out_len < 0) return fail(DMRG_ERR_INVALID_ARG, "negative size");
    if (!dims || !dims_new || (n_blocks > 0 && (!blocks || !out_off)))
        return fail(DMRG_ERR_INVALID_ARG, "null argument");
    std::vector<int64_t> u_off(size_t(nsec) + 1, 0);
    for (int32_t q = 0; q < nsec; ++q) {
        if (dims[q] < 1 || dims_new[q] < 1 || dims_new[q] > dims[q] || dims[q] > (1 << 20))
            return fail(DMRG_ERR_INVALID_ARG, "sector dims: 1 <= new dim <= dim");
        u_off[size_t(q) + 1] = u_off[size_t(q)] + int64_t(dims[q]) * dims_new[q];
    }
    int64_t pos = 0;
    for (int64_t b = 0; b < n_blocks; ++b) {
        const int64_t q = blocks[3 * b], p = blocks[3 * b + 1], off = blocks[3 * b + 2];
        if (q < 0 || q >= nsec || p < 0 || p >= nsec) return fail(DMRG_ERR_INVALID_ARG, "block sector out of range");
        if (off < 0 || off + int64_t(dims[p]) * dims[q] > op_len) return fail(DMRG_ERR_INVALID_ARG, "block outside op");
        out_off[b] = pos;
        pos += int64_t(dims_new[p]) * dims_new[q];
    }
    if (pos > out_len) return fail(DMRG_ERR_INVALID_ARG, "out too small");

    // ---- the two-stage GEMM lists
    RenormPlan* R = new (std::nothrow) RenormPlan();
    if (!R) return fail(DMRG_ERR_OOM, "host allocation");
    R->nsec = nsec;
    R->op_len = op_len;
    R->out_len = out_len;
    R->nu = u_off[size_t(nsec)];
    Plan& P = R->P;
    int64_t scr = 0;
    for (int64_t b = 0; b < n_blocks; ++b) {
        const int32_t q = int32_t(blocks[3 * b]), p = int32_t(blocks[3 * b + 1]);
        const int64_t off = blocks[3 * b + 2];
        const int32_t dq = dims[q], dp = dims[p], nq = dims_new[q], np_ = dims_new[p];
        Seg s1{};
        s1.l_space = SP_OPS; s1.l_off = off; s1.l_ld = dq; s1.l_ts = 0;
        s1.r_space = SP_X; s1.r_off = u_off[size_t(q)]; s1.r_ld = nq; s1.r_ts = 0; s1.r_trans = 0;
        s1.kc = dq; s1.nt = 1;
        Gemm g1{};
        g1.d_space = SP_SCR; g1.d_off = scr; g1.ldd = nq; g1.M = dp; g1.N = nq; g1.K = dq;
        g1.seg0 = int32_t(P.segs.size()); g1.nseg = 1; g1.alpha = 1.0;
        P.segs.push_back(s1);
        P.s1gemms.push_back(int32_t(P.gemms.size()));
        P.gemms.push_back(g1);
        Seg s2{};   // L = U_p^T (the transposed copies follow the bases in the x space)
        s2.l_space = SP_X; s2.l_off = u_off[size_t(nsec)] + u_off[size_t(p)]; s2.l_ld = dp; s2.l_ts = 0;
        s2.r_space = SP_SCR; s2.r_off = scr; s2.r_ld = nq; s2.r_ts = 0; s2.r_trans = 0;
        s2.kc = dp; s2.nt = 1;
        Gemm g2{};
        g2.d_space = SP_Y; g2.d_off = out_off[b]; g2.ldd = nq; g2.M = np_; g2.N = nq; g2.K = dp;
        g2.seg0 = int32_t(P.segs.size()); g2.nseg = 1; g2.alpha = 1.0;
        P.segs.push_back(s2);
        P.s2gemms.push_back(int32_t(P.gemms.size()));
        P.gemms.push_back(g2);
        scr += int64_t(dp) * nq;
    }
    std::string err;
    int rc = build_fp64_work(P, Schedule{}, &err);
    if (rc != DMRG_OK) {
        delete R;
        return fail(rc, err);
    }

    if (P.gemms.empty()) {   // no blocks: nothing on the device
        *plan = reinterpret_cast<dmrg_renorm_t>(R);
        return DMRG_OK;
    }
    // ---- device buffers and tables, once
    Bufs& B = R->B;
    if ((rc = B.alloc(&R->uu, size_t(2 * R->nu), "bases")) ||
        (rc = B.alloc(&R->X, size_t(scr), "renormalisation scratch")) ||
        (rc = B.alloc(&R->part, size_t(P.n_slots) * FP64_BM * FP64_BN, "partials")) ||
        (rc = B.upload(&R->t1, P.tiles1, "tiles")) || (rc = B.upload(&R->t2, P.tiles2, "tiles")) ||
        (rc = B.upload(&R->gm, P.gemms, "gemms")) || (rc = B.upload(&R->sg, P.segs, "segments")) ||
        (rc = B.upload(&R->red, P.reduces, "reduce jobs")) || (rc = B.alloc(&R->counters, 2, "counters")) ||
        (rc = B.upload(&R->d_uoff, u_off, "basis offsets")) ||
        (rc = B.upload(&R->d_d, std::vector<int32_t>(dims, dims + nsec), "dims")) ||
        (rc = B.upload(&R->d_dn, std::vector<int32_t>(dims_new, dims_new + nsec), "dims"))) {
        delete R;
        return rc;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&R->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete R;
        return cuda_fail(e, "device attributes");
    }
    *plan = reinterpret_cast<dmrg_renorm_t>(R);
    return DMRG_OK;
}

extern "C" int dmrg_renorm_run(dmrg_renorm_t plan, const double* U, const double* op, double* out, void* stream) {
    using namespace dmrg;
    if (!plan) return fail(DMRG_ERR_INVALID_ARG, "null plan");
    RenormPlan* R = reinterpret_cast<RenormPlan*>(plan);
    const Plan& P = R->P;
    if (P.gemms.empty()) return DMRG_OK;
    if (!U || !op || !out) return fail(DMRG_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(R->uu, U, sizeof(double) * size_t(R->nu), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        k_transpose_bases<<<unsigned(R->nsec), 256, 0, st>>>(R->uu, R->uu + R->nu, R->d_uoff, R->d_d, R->d_dn);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(R->counters, 0, sizeof(int32_t) * 2, st);
    Spaces sp{};
    sp.ops = op; sp.x = R->uu; sp.scr = R->X; sp.y = out; sp.part = R->part;
    const int64_t cap = int64_t(R->n_sm) * fp64_tiles_per_sm();
    auto grid = [&](size_t n) { return int32_t(std::min<int64_t>(int64_t(n), cap)); };
    if (e == cudaSuccess && !P.tiles1.empty())
        e = launch_fp64_tiles(R->t1, int32_t(P.tiles1.size()), R->gm, R->sg, sp, 1, R->counters, grid(P.tiles1.size()),
                              st);
    if (e == cudaSuccess && !P.tiles2.empty())
        e = launch_fp64_tiles(R->t2, int32_t(P.tiles2.size()), R->gm, R->sg, sp, 1, R->counters + 1,
                              grid(P.tiles2.size()), st);
    if (e == cudaSuccess && !P.reduces.empty()) e = launch_fp64_reduce(R->red, int32_t(P.reduces.size()), R->gm, sp, 1, st);
    return e == cudaSuccess ? DMRG_OK : cuda_fail(e, "renormalisation");
}

extern "C" void dmrg_renorm_destroy(dmrg_renorm_t plan) { delete reinterpret_cast<dmrg::RenormPlan*>(plan); }

extern "C" int dmrg_renormalise(int32_t nsec, const int32_t* dims, const int32_t* dims_new, const double* U,
                                const int64_t* blocks, int64_t n_blocks, const double* op, int64_t op_len,
                                double* out, int64_t out_len, int64_t* out_off, void* stream) {
    using namespace dmrg;
    if (n_blocks > 0 && (!U || !op || !out)) return fail(DMRG_ERR_INVALID_ARG, "null argument");
    dmrg_renorm_t plan = nullptr;
    int rc = dmrg_renorm_create(nsec, dims, dims_new, blocks, n_blocks, op_len, out_len, out_off, &plan);
    if (rc != DMRG_OK) return rc;
    rc = dmrg_renorm_run(plan, U, op, out, stream);
    // the plan's buffers are released only after its launches have run
    const cudaError_t es = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    dmrg_renorm_destroy(plan);
    if (rc != DMRG_OK) return rc;
    if (es != cudaSuccess) return cuda_fail(es, "renormalisation");
    return DMRG_OK;
}
