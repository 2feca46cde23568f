// Two-site decomposition and truncation: per left sector of the wave function the matrix
// M_q = [psi_b ...] of its blocks side by side (rows = dim of the left sector; one block
// per left sector in U(1), one per coupled right spin in SU(2)), its singular values and
// left vectors by one-sided (Hestenes) Jacobi in FP64, one CTA per matrix (one cluster of
// 8 CTAs for a matrix above 200 KB): column pairs in the round-robin order, fixed-order
// sums, a sweep without rotation above 1e-15 of the pair's norms ends it.  The columns then hold
// sigma_j u_j.  The host keeps the D largest singular values over all matrices and the
// kernel k_svd_emit writes the kept left vectors.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <tuple>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "jacobi_rot.cuh"

namespace dmrg {
namespace {

constexpr int SVD_NT = 512;
constexpr int64_t SVD_SMEM_MAX = 200 * 1024;   // shared-memory limit of the one-CTA kernel
constexpr int64_t SVD_CLUSTER_MIN = 64 * 1024;  // matrices above this size go to the cluster kernel
constexpr int SVD_WARPS = SVD_NT / 32;
constexpr int SVD_LPP = 8;                               // lanes per column pair
constexpr int SVD_BATCH = SVD_WARPS * (32 / SVD_LPP);    // pairs in flight (64)
constexpr int SVD_MAX_SWEEPS = 40;
constexpr double SVD_ZERO = 1e-13;   // singular values below this fraction of the largest are zero

struct SvdJob {
    int64_t off;      // of the matrix's first block in psi and of the matrix in the scratch
    int64_t sv_off;   // of its cols singular values / column order
    int32_t rows, cols;
    int32_t b0, nb;   // its blocks: consecutive in psi, cols bcols[b0 .. b0 + nb)
};

// Sum over the warp, the same value in every lane: lane 0's result is broadcast (the
// butterfly leaves each lane with its own rounding order), so a rotation decision and
// its (c, s) agree across the lanes that apply it.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// SMEM: the matrix is rotated in dynamic shared memory (rows * cols doubles) and copied to
// the scratch A at the end; otherwise it is rotated in A.  The arithmetic is the same.
// (Larger matrices go to k_svd_cluster below.)
template <bool SMEM>
__global__ void __launch_bounds__(SVD_NT) k_svd_jacobi(const double* __restrict__ psi, double* __restrict__ A,
                                                       const SvdJob* __restrict__ jobs,
                                                       const int32_t* __restrict__ bcols, double* __restrict__ raw,
                                                       double* __restrict__ sv, int32_t* __restrict__ order) {
    extern __shared__ __align__(16) double s_mat[];
    const SvdJob J = jobs[blockIdx.x];
    const int rows = J.rows, cols = J.cols, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double* a = SMEM ? s_mat : A + J.off;   // column j at a + j * rows
    int cbase = 0;
    int64_t boff = J.off;
    for (int bi = 0; bi < J.nb; ++bi) {   // block bi: row-major rows x cb, columns [cbase, cbase + cb)
        const int cb = bcols[J.b0 + bi];
        for (int64_t e = tid; e < int64_t(rows) * cb; e += SVD_NT) {
            const int r = int(e / cb), c = int(e % cb);
            a[int64_t(cbase + c) * rows + r] = psi[boff + e];
        }
        cbase += cb;
        boff += int64_t(rows) * cb;
    }
    __syncthreads();
    // Each round's disjoint pairs go in batches of SVD_BATCH: (1) 8 lanes per pair form
    // partial dot products over a stride-8 row stripe, (2) one thread per pair sums them
    // in lane order and computes the rotation, (3) the 8 lanes apply it.  The rotation's
    // divisions and square roots are then paid once per pair, not once per lane (FP64
    // issue slots are the limit of this kernel).
    __shared__ double s_part[SVD_BATCH][3][SVD_LPP];
    __shared__ double s_cs[SVD_BATCH][2];
    __shared__ int s_rot;
    const int M = (cols + 1) & ~1, half = M / 2;
    const int sub = lane % SVD_LPP, slot = warp * (32 / SVD_LPP) + lane / SVD_LPP;   // pair slot in a batch
    for (int sweep = 0; sweep < SVD_MAX_SWEEPS && cols >= 2; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < M - 1; ++r) {
            for (int kb = 0; kb < half; kb += SVD_BATCH) {
                // round-robin pair k of round r: columns p < q (q == cols is the padding column)
                const int k = kb + slot;
                int p = 0, q = cols;
                if (k < half) {
                    const int x = k == 0 ? 0 : ((k - 1 + r) % (M - 1)) + 1;
                    const int y = ((M - 2 - k + r) % (M - 1)) + 1;
                    p = min(x, y);
                    q = max(x, y);
                }
                const bool act = k < half && q < cols;
                double* ap = a + int64_t(p) * rows;
                double* aq = a + int64_t(q) * rows;
                if (act) {
                    double al = 0.0, be = 0.0, ga = 0.0;
                    for (int i = sub; i < rows; i += SVD_LPP) {
                        const double u = ap[i], w = aq[i];
                        al += u * u; be += w * w; ga += u * w;
                    }
                    s_part[slot][0][sub] = al;
                    s_part[slot][1][sub] = be;
                    s_part[slot][2][sub] = ga;
                }
                __syncthreads();
                if (tid < SVD_BATCH) {
                    const int kk = kb + tid;
                    double c = 1.0, sn = 0.0;
                    if (kk < half) {
                        const int x = kk == 0 ? 0 : ((kk - 1 + r) % (M - 1)) + 1;
                        const int y = ((M - 2 - kk + r) % (M - 1)) + 1;
                        if (max(x, y) < cols) {
                            double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
                            for (int l = 0; l < SVD_LPP; ++l) {
                                al += s_part[tid][0][l];
                                be += s_part[tid][1][l];
                                ga += s_part[tid][2][l];
                            }
                            if (jacobi_rotate_needed(ga, al, be)) {
                                jacobi_rotation(be - al, ga, &c, &sn);
                                s_rot = 1;
                            }
                        }
                    }
                    s_cs[tid][0] = c;
                    s_cs[tid][1] = sn;
                }
                __syncthreads();
                if (act) {
                    const double c = s_cs[slot][0], sn = s_cs[slot][1];
                    if (sn != 0.0)
                        for (int i = sub; i < rows; i += SVD_LPP) {
                            const double u = ap[i], w = aq[i];
                            ap[i] = c * u - sn * w;
                            aq[i] = sn * u + c * w;
                        }
                }
            }
            __syncthreads();   // the next round's pairs read these columns
        }
        const int rot = s_rot;   // every thread reads it before the barrier below
        __syncthreads();
        if (rot == 0) break;
    }
    // column norms (sigma_j, any order), then ranks: descending, ties to the lower index
    for (int j = warp; j < cols; j += SVD_WARPS) {
        const double* aj = a + int64_t(j) * rows;
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s += aj[i] * aj[i];
        s = warp_sum(s);
        if (lane == 0) raw[J.sv_off + j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < cols; j += SVD_NT) {
        const double sj = raw[J.sv_off + j];
        int rank = 0;
        for (int k = 0; k < cols; ++k) {
            const double sk = raw[J.sv_off + k];
            rank += (sk > sj || (sk == sj && k < j)) ? 1 : 0;
        }
        sv[J.sv_off + rank] = sj;
        order[J.sv_off + rank] = j;
    }
    if (SMEM)   // the emit kernel reads the rotated columns from A
        for (int64_t e = tid; e < int64_t(rows) * cols; e += SVD_NT) A[J.off + e] = s_mat[e];
}

// Matrices above the shared-memory size: one cluster of SVD_CL CTAs per matrix, the
// columns in the scratch A (L2-resident; read and written past L1, whose lines are not
// coherent between SMs), the round's disjoint pairs dealt to the CTAs (pair k to rank
// k % SVD_CL), one warp per pair: 32-lane dot products summed in a fixed butterfly and
// broadcast, so every lane forms the same rotation (angle in single precision made
// exactly orthonormal in double, jacobi_rotation), then applied by the warp.  A cluster
// barrier ends each round.  Whether a sweep rotated is gathered in flag[2 job + sweep
// parity] (rank 0 clears the other parity once every CTA has read it, after this
// sweep's first barrier), and every CTA reads it after the sweep's last barrier, so all
// CTAs of a cluster leave the sweep loop together.  FP64 issue is this kernel's limit: the cluster divides each
// round's work by SVD_CL.
constexpr int SVD_CL = 8;
__global__ void __launch_bounds__(SVD_NT) k_svd_cluster(const double* __restrict__ psi, double* __restrict__ A,
                                                        const SvdJob* __restrict__ jobs,
                                                        const int32_t* __restrict__ bcols, double* __restrict__ raw,
                                                        double* __restrict__ sv, int32_t* __restrict__ order,
                                                        int* __restrict__ flag) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int job = blockIdx.x / SVD_CL, rank = int(cluster.block_rank());
    const SvdJob J = jobs[job];
    const int rows = J.rows, cols = J.cols, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double* a = A + J.off;   // column j at a + j * rows
    {   // the blocks into column-major A, dealt over the cluster's threads
        int cbase = 0;
        int64_t boff = J.off;
        for (int bi = 0; bi < J.nb; ++bi) {
            const int cb = bcols[J.b0 + bi];
            for (int64_t e = int64_t(rank) * SVD_NT + tid; e < int64_t(rows) * cb; e += int64_t(SVD_CL) * SVD_NT) {
                const int r = int(e / cb), c = int(e % cb);
                __stcg(a + int64_t(cbase + c) * rows + r, psi[boff + e]);
            }
            cbase += cb;
            boff += int64_t(rows) * cb;
        }
    }
    if (rank == 0 && tid == 0) {
        flag[2 * job] = 0;
        flag[2 * job + 1] = 0;
    }
    __shared__ int s_rot;
    cluster.sync();
    const int M = (cols + 1) & ~1, half = M / 2;
    for (int sweep = 0; sweep < SVD_MAX_SWEEPS && cols >= 2; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < M - 1; ++r) {
            for (int k = rank + SVD_CL * warp; k < half; k += SVD_CL * SVD_WARPS) {
                const int x = k == 0 ? 0 : ((k - 1 + r) % (M - 1)) + 1;
                const int y = ((M - 2 - k + r) % (M - 1)) + 1;
                const int p = min(x, y), q = max(x, y);
                if (q >= cols) continue;   // the padding column (warp-uniform)
                double* ap = a + int64_t(p) * rows;
                double* aq = a + int64_t(q) * rows;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < rows; i += 32) {
                    const double u = __ldcg(ap + i), w = __ldcg(aq + i);
                    al += u * u; be += w * w; ga += u * w;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (jacobi_rotate_needed(ga, al, be)) {
                    double c, sn;
                    jacobi_rotation(be - al, ga, &c, &sn);
                    if (lane == 0) s_rot = 1;
                    for (int i = lane; i < rows; i += 32) {
                        const double u = __ldcg(ap + i), w = __ldcg(aq + i);
                        __stcg(ap + i, c * u - sn * w);
                        __stcg(aq + i, sn * u + c * w);
                    }
                }
            }
            cluster.sync();   // the next round's pairs read these columns
        }
        // the other parity was read at the end of the previous sweep, before this sweep's
        // first barrier; it is written again only after the barrier below
        if (rank == 0 && tid == 0) flag[2 * job + ((sweep + 1) & 1)] = 0;
        __syncthreads();
        if (tid == 0 && s_rot) atomicOr(flag + 2 * job + (sweep & 1), 1);
        cluster.sync();
        if (__ldcg(flag + 2 * job + (sweep & 1)) == 0) break;   // the same value in every CTA
    }
    if (rank != 0) return;
    // column norms (sigma_j, any order), then ranks: descending, ties to the lower index
    for (int j = warp; j < cols; j += SVD_WARPS) {
        const double* aj = a + int64_t(j) * rows;
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) {
            const double v = __ldcg(aj + i);
            s += v * v;
        }
        s = warp_sum(s);
        if (lane == 0) raw[J.sv_off + j] = sqrt(s);
    }
    __syncthreads();
    for (int j = tid; j < cols; j += SVD_NT) {
        const double sj = raw[J.sv_off + j];
        int rank_j = 0;
        for (int k = 0; k < cols; ++k) {
            const double sk = raw[J.sv_off + k];
            rank_j += (sk > sj || (sk == sj && k < j)) ? 1 : 0;
        }
        sv[J.sv_off + rank_j] = sj;
        order[J.sv_off + rank_j] = j;
    }
}

// U_q (rows x kept_q, row-major at u_off[q]) = kept columns / their singular values
__global__ void k_svd_emit(const double* __restrict__ A, const SvdJob* __restrict__ jobs, const double* __restrict__ sv,
                           const int32_t* __restrict__ order, const int32_t* __restrict__ kept,
                           const int64_t* __restrict__ u_off, double* __restrict__ U) {
    const SvdJob J = jobs[blockIdx.x];
    const int k = kept[blockIdx.x];
    for (int64_t e = threadIdx.x; e < int64_t(J.rows) * k; e += blockDim.x) {
        const int i = int(e / k), r = int(e % k);
        const int col = order[J.sv_off + r];
        U[u_off[blockIdx.x] + e] = A[J.off + int64_t(col) * J.rows + i] / sv[J.sv_off + r];
    }
}

}  // namespace
}  // namespace dmrg

using dmrg::Handle;

extern "C" int dmrg_heff_psi_blocks(dmrg_heff_t hh, int64_t* buf, int64_t* n_blocks) {
    using namespace dmrg;
    if (!hh || !n_blocks) return fail(DMRG_ERR_INVALID_ARG, "null argument");
    const Handle* h = static_cast<Handle*>(hh);
    const int64_t n = int64_t(h->plan.blocks.size());
    if (buf) {
        if (*n_blocks < n) return fail(DMRG_ERR_INVALID_ARG, "block buffer too small");
        for (int64_t b = 0; b < n; ++b) {
            const PsiBlock& B = h->plan.blocks[size_t(b)];
            buf[5 * b] = B.iL; buf[5 * b + 1] = B.iR; buf[5 * b + 2] = B.rows; buf[5 * b + 3] = B.cols;
            buf[5 * b + 4] = B.off;
        }
    }
    *n_blocks = n;
    return DMRG_OK;
}

extern "C" int dmrg_svd_truncate(dmrg_heff_t hh, const double* psi, int32_t D, double* sv_out, int32_t* kept_out,
                                 double* U, int64_t u_len, int64_t* u_off, double* discarded) {
    using namespace dmrg;
    if (!hh) return fail(DMRG_ERR_INVALID_ARG, "null handle");
    Handle* h = static_cast<Handle*>(hh);
    if (h->plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    const auto& pblocks = h->plan.blocks;
    // one matrix per left sector: its blocks are consecutive in the layout
    struct Mat { int64_t off; int32_t rows, cols, b0, nb; };
    std::vector<Mat> blocks;
    std::vector<int32_t> bcols(pblocks.size());
    for (size_t b = 0; b < pblocks.size(); ++b) {
        const PsiBlock& B = pblocks[b];
        bcols[b] = B.cols;
        if (!blocks.empty() && pblocks[b - 1].iL == B.iL) {
            blocks.back().cols += B.cols;
            blocks.back().nb += 1;
        } else {
            blocks.push_back({B.off, B.rows, B.cols, int32_t(b), 1});
        }
    }
    const int64_t nb = int64_t(blocks.size());
    if (D < 1 || u_len < 0) return fail(DMRG_ERR_INVALID_ARG, "D >= 1, u_len >= 0");
    if (nb == 0) {
        if (discarded) *discarded = 0.0;
        return DMRG_OK;
    }
    if (!psi || !sv_out || !kept_out || !u_off || !discarded) return fail(DMRG_ERR_INVALID_ARG, "null argument");
    std::vector<SvdJob> jobs(static_cast<size_t>(nb));
    int64_t nsv = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const Mat& B = blocks[size_t(b)];
        if (B.cols > 8192) return fail(DMRG_ERR_UNSUPPORTED, "a left sector with more than 8192 columns");
        jobs[size_t(b)] = {B.off, nsv, B.rows, B.cols, B.b0, B.nb};
        nsv += B.cols;
    }
    const int64_t dim = h->plan.dim;
    double *A = nullptr, *raw = nullptr, *sv = nullptr;
    int32_t *order = nullptr, *d_kept = nullptr, *d_bcols = nullptr;
    int64_t* d_uoff = nullptr;
    SvdJob* d_jobs = nullptr;
    std::vector<void*> owned;
    auto al = [&](void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 8);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    };
    auto release = [&]() {
        for (void* p : owned) cudaFree(p);
    };
    cudaError_t e = al(reinterpret_cast<void**>(&A), sizeof(double) * size_t(dim));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&raw), sizeof(double) * size_t(nsv));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&sv), sizeof(double) * size_t(nsv));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&order), sizeof(int32_t) * size_t(nsv));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&d_jobs), sizeof(SvdJob) * size_t(nb));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&d_kept), sizeof(int32_t) * size_t(nb));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&d_uoff), sizeof(int64_t) * size_t(nb));
    if (e == cudaSuccess) e = al(reinterpret_cast<void**>(&d_bcols), sizeof(int32_t) * bcols.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_jobs, jobs.data(), sizeof(SvdJob) * size_t(nb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_bcols, bcols.data(), sizeof(int32_t) * bcols.size(), cudaMemcpyHostToDevice);
    // matrices up to SVD_CLUSTER_MIN on one CTA each (rotated in shared memory), the
    // larger ones on a cluster each, the two launches side by side on two streams
    std::vector<SvdJob> small, large;
    int64_t smem = 0;
    for (const SvdJob& J : jobs) {
        const int64_t bytes = int64_t(J.rows) * J.cols * int64_t(sizeof(double));
        if (bytes <= SVD_CLUSTER_MIN) {
            small.push_back(J);
            smem = std::max(smem, bytes);
        } else {
            large.push_back(J);
        }
    }
    static_assert(SVD_CLUSTER_MIN <= SVD_SMEM_MAX, "one-CTA matrices must fit in shared memory");
    cudaStream_t side = nullptr;
    if (e == cudaSuccess && !large.empty()) e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    SvdJob *d_small = nullptr, *d_large = nullptr;
    if (e == cudaSuccess && !small.empty()) e = al(reinterpret_cast<void**>(&d_small), sizeof(SvdJob) * small.size());
    if (e == cudaSuccess && !large.empty()) e = al(reinterpret_cast<void**>(&d_large), sizeof(SvdJob) * large.size());
    if (e == cudaSuccess && !small.empty())
        e = cudaMemcpy(d_small, small.data(), sizeof(SvdJob) * small.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !large.empty())
        e = cudaMemcpy(d_large, large.data(), sizeof(SvdJob) * large.size(), cudaMemcpyHostToDevice);
    int* d_flag = nullptr;
    if (e == cudaSuccess && !large.empty()) e = al(reinterpret_cast<void**>(&d_flag), sizeof(int) * 2 * large.size());
    // the side stream does not order itself after the default stream: the copies above
    // (and the caller's work on psi) finish before either kernel starts
    if (e == cudaSuccess && side) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && !small.empty())
        e = cudaFuncSetAttribute(k_svd_jacobi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess && !small.empty()) {
        k_svd_jacobi<true><<<unsigned(small.size()), SVD_NT, size_t(smem)>>>(psi, A, d_small, d_bcols, raw, sv, order);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !large.empty()) {   // one cluster of SVD_CL CTAs per large matrix
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(large.size() * SVD_CL));
        cfg.blockDim = dim3(SVD_NT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = side;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = SVD_CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_svd_cluster, static_cast<const double*>(psi), A,
                               static_cast<const SvdJob*>(d_large), static_cast<const int32_t*>(d_bcols), raw, sv,
                               order, d_flag);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (side) {
        const cudaError_t es = cudaStreamSynchronize(side);
        if (e == cudaSuccess) e = es;
        cudaStreamDestroy(side);
    }
    std::vector<double> hsv(static_cast<size_t>(nsv));
    if (e == cudaSuccess) e = cudaMemcpy(hsv.data(), sv, sizeof(double) * size_t(nsv), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "svd");
    }
    // the D largest over all matrices (ties: earlier matrix, then earlier position)
    double smax = 0.0, total = 0.0;
    for (double s : hsv) {
        smax = std::max(smax, s);
        total += s * s;
    }
    std::vector<std::tuple<double, int64_t, int32_t>> cand;
    for (int64_t b = 0; b < nb; ++b) {
        const int k = std::min(blocks[size_t(b)].rows, blocks[size_t(b)].cols);
        for (int i = 0; i < k; ++i) {
            const double s = hsv[size_t(jobs[size_t(b)].sv_off + i)];
            if (s > SVD_ZERO * smax) cand.emplace_back(-s, b, i);
        }
    }
    std::sort(cand.begin(), cand.end());
    if (int64_t(cand.size()) > D) cand.resize(size_t(D));
    std::vector<int32_t> kept(static_cast<size_t>(nb), 0);
    double kept_w = 0.0;
    for (const auto& c : cand) {
        kept[size_t(std::get<1>(c))] += 1;
        kept_w += std::get<0>(c) * std::get<0>(c);
    }
    int64_t pos = 0, ns = 0;
    std::vector<int64_t> uo(static_cast<size_t>(nb));
    for (int64_t b = 0; b < nb; ++b) {
        uo[size_t(b)] = pos;
        pos += int64_t(blocks[size_t(b)].rows) * kept[size_t(b)];
        const int k = std::min(blocks[size_t(b)].rows, blocks[size_t(b)].cols);
        for (int i = 0; i < k; ++i) sv_out[ns + i] = hsv[size_t(jobs[size_t(b)].sv_off + i)];
        ns += k;
        kept_out[b] = kept[size_t(b)];
        u_off[b] = uo[size_t(b)];
    }
    *discarded = total - kept_w;
    if (pos > 0 && (!U || pos > u_len)) {
        release();
        return fail(DMRG_ERR_INVALID_ARG, "U too small for the kept vectors");
    }
    e = cudaMemcpy(d_kept, kept.data(), sizeof(int32_t) * size_t(nb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_uoff, uo.data(), sizeof(int64_t) * size_t(nb), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && pos > 0) {
        k_svd_emit<<<unsigned(nb), SVD_NT>>>(A, d_jobs, sv, order, d_kept, d_uoff, U);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    release();
    return e == cudaSuccess ? int(DMRG_OK) : cuda_fail(e, "svd emit");
}
