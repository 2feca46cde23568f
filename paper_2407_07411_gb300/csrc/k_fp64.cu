// FP64 path: grouped GEMM tiles on the FP64 tensor cores (DMMA, mma.sync
// m16n8k16 .f64), one output tile per CTA iteration (32x32 with 4 warps, or 64x32 /
// 32x64 with 8, by the schedule), K staged through shared memory 16 columns at a time;
// every warp owns a 16x16 quarter-tile.
//
// On GB300 the FP64 tensor pipe sustains about 1.1 TFLOP/s (m16n8k16, measured by
// the library's probe; m8n8k4 and plain DFMA about 1.0-1.05), three orders of
// magnitude below the BF16 pipe, so this kernel is bound by DMMA issue alone: the design goals are no padded MMA
// work beyond the 16x8x16 granularity (warps skip strips that lie outside the
// GEMM), enough resident warps to keep the pipe busy, and balanced work
// (dynamic tile queue, largest K range first).  Operand staging is plain loads;
// at ~7 flop/clk/SM of FP64 they are never on the critical path.
#include <cstdint>

#include "kernels.h"

namespace dmrg {
namespace {

constexpr int BK = FP64_BK;
template <int BM, int BN>
constexpr int fp64_threads() { return (BM / 16) * (BN / 16) * 32; }

__device__ __forceinline__ const double* space_ptr(const Spaces& sp, int32_t s, int v) {
    switch (s) {
        case SP_OPS: return sp.ops;
        case SP_X: return sp.x + int64_t(v) * sp.x_vs;
        case SP_SCR: return sp.scr + int64_t(v) * sp.scr_vs;
        case SP_Y: return sp.y + int64_t(v) * sp.y_vs;
        default: return sp.part + int64_t(v) * sp.part_vs;
    }
}

__device__ __forceinline__ void dmma16816(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
        "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
          "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

template <int BM, int BN>
__global__ void __launch_bounds__(fp64_threads<BM, BN>()) k_fp64_tiles(const Tile* __restrict__ tiles, int32_t n_tiles,
                                                   const Gemm* __restrict__ gemms,
                                                   const Seg* __restrict__ segs, Spaces sp,
                                                   int32_t nvec, int32_t* counter) {
    constexpr int NT = fp64_threads<BM, BN>();
    __shared__ double sL[BM][BK + 1];
    __shared__ double sR[BK][BN + 1];
    __shared__ const double* s_lp[BK];
    __shared__ const double* s_rp[BK];
    __shared__ int32_t s_lld[BK], s_rsn[BK];
    __shared__ int32_t s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int wm = (warp / (BN / 16)) * 16, wn = (warp % (BN / 16)) * 16;
    const int64_t n_items = int64_t(n_tiles) * nvec;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const Tile tl = tiles[item / nvec];
        const int v = int(item % nvec);
        const Gemm gm = gemms[tl.gemm];
        const int rows = min(BM, gm.M - tl.m0), cols = min(BN, gm.N - tl.n0);
        const bool warp_rows = wm < rows;
        double acc[2][4] = {};

        for (int64_t kb = tl.k0; kb < tl.k1; kb += BK) {
            if (tid < BK) {   // decode column kb + tid into operand pointers
                const int64_t K = kb + tid;
                const double* lp = nullptr;
                const double* rp = nullptr;
                int32_t lld = 0, rsn = 0;
                if (K < tl.k1) {
                    int64_t base = 0;
                    for (int s = gm.seg0; s < gm.seg0 + gm.nseg; ++s) {
                        const Seg sg = segs[s];
                        const int64_t ext = int64_t(sg.kc) * sg.nt;
                        if (K < base + ext) {
                            const int64_t t = (K - base) / sg.kc, k = (K - base) % sg.kc;
                            lp = space_ptr(sp, sg.l_space, v) + sg.l_off + t * sg.l_ts + k +
                                 int64_t(tl.m0) * sg.l_ld;
                            lld = sg.l_ld;
                            if (sg.r_trans) {
                                rp = space_ptr(sp, sg.r_space, v) + sg.r_off + t * sg.r_ts + k +
                                     int64_t(tl.n0) * sg.r_ld;
                                rsn = sg.r_ld;
                            } else {
                                rp = space_ptr(sp, sg.r_space, v) + sg.r_off + t * sg.r_ts +
                                     k * sg.r_ld + tl.n0;
                                rsn = 1;
                            }
                            break;
                        }
                        base += ext;
                    }
                }
                s_lp[tid] = lp; s_rp[tid] = rp; s_lld[tid] = lld; s_rsn[tid] = rsn;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < BM * BK / NT; ++j) {
                const int e = tid + j * NT, r = e / BK, kk = e % BK;
                const double* p = s_lp[kk];
                sL[r][kk] = (p != nullptr && r < rows) ? p[int64_t(r) * s_lld[kk]] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < BN * BK / NT; ++j) {
                const int e = tid + j * NT, n = e / BK, kk = e % BK;
                const double* p = s_rp[kk];
                sR[kk][n] = (p != nullptr && n < cols) ? p[int64_t(n) * s_rsn[kk]] : 0.0;
            }
            __syncthreads();
            if (warp_rows) {
                double a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = sL[wm + g + 8 * (i & 1)][tg + 4 * (i >> 1)];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    if (wn + 8 * j < cols) {
                        double b[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) b[i] = sR[tg + 4 * i][wn + 8 * j + g];
                        dmma16816(acc[j], a, b);
                    }
                }
            }
            __syncthreads();
        }

        // Epilogue: c0 (g, 2tg), c1 (g, 2tg+1), c2 (g+8, 2tg), c3 (g+8, 2tg+1).
        if (tl.slot < 0) {
            double* D = const_cast<double*>(space_ptr(sp, gm.d_space, v)) + gm.d_off;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = wm + g + 8 * (e >> 1), c = wn + 8 * j + 2 * tg + (e & 1);
                    if (r < rows && c < cols)
                        D[int64_t(tl.m0 + r) * gm.ldd + tl.n0 + c] = gm.alpha * acc[j][e];
                }
        } else {
            double* Pt = sp.part + int64_t(v) * sp.part_vs + int64_t(tl.slot) * (BM * BN);
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = wm + g + 8 * (e >> 1), c = wn + 8 * j + 2 * tg + (e & 1);
                    Pt[r * BN + c] = acc[j][e];
                }
        }
    }
}

template <int BM, int BN>
__global__ void __launch_bounds__(128) k_fp64_reduce(const Reduce* __restrict__ red,
                                                    const Gemm* __restrict__ gemms, Spaces sp) {
    constexpr int NT = 128;
    const Reduce rj = red[blockIdx.x];
    const int v = blockIdx.y;
    const Gemm gm = gemms[rj.gemm];
    const int rows = min(BM, gm.M - rj.m0), cols = min(BN, gm.N - rj.n0);
    const double* Pt = sp.part + int64_t(v) * sp.part_vs + int64_t(rj.p0) * (BM * BN);
    double* D = const_cast<double*>(space_ptr(sp, gm.d_space, v)) + gm.d_off;
    for (int e = threadIdx.x; e < BM * BN; e += NT) {
        const int r = e / BN, c = e % BN;
        if (r >= rows || c >= cols) continue;
        double s = 0.0;
        for (int p = 0; p < rj.np; ++p) s += Pt[int64_t(p) * (BM * BN) + e];
        D[int64_t(rj.m0 + r) * gm.ldd + rj.n0 + c] = gm.alpha * s;
    }
}

}  // namespace

cudaError_t launch_fp64_tiles(const Tile* tiles, int32_t n_tiles, const Gemm* gemms,
                              const Seg* segs, const Spaces& sp, int32_t nvec, int32_t* counter,
                              int32_t grid, cudaStream_t st, int shape) {
    if (n_tiles <= 0) return cudaSuccess;
    if (shape == 1)
        k_fp64_tiles<64, 32><<<grid, fp64_threads<64, 32>(), 0, st>>>(tiles, n_tiles, gemms, segs, sp, nvec, counter);
    else if (shape == 2)
        k_fp64_tiles<32, 64><<<grid, fp64_threads<32, 64>(), 0, st>>>(tiles, n_tiles, gemms, segs, sp, nvec, counter);
    else
        k_fp64_tiles<32, 32><<<grid, fp64_threads<32, 32>(), 0, st>>>(tiles, n_tiles, gemms, segs, sp, nvec, counter);
    return cudaGetLastError();
}

cudaError_t launch_fp64_reduce(const Reduce* red, int32_t n_red, const Gemm* gemms,
                               const Spaces& sp, int32_t nvec, cudaStream_t st, int shape) {
    if (n_red <= 0) return cudaSuccess;
    if (shape == 1)
        k_fp64_reduce<64, 32><<<dim3(n_red, nvec), 128, 0, st>>>(red, gemms, sp);
    else if (shape == 2)
        k_fp64_reduce<32, 64><<<dim3(n_red, nvec), 128, 0, st>>>(red, gemms, sp);
    else
        k_fp64_reduce<32, 32><<<dim3(n_red, nvec), 128, 0, st>>>(red, gemms, sp);
    return cudaGetLastError();
}

int fp64_tiles_per_sm(int shape) {
    int n = 0;
    cudaError_t e;
    if (shape == 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fp64_tiles<64, 32>, fp64_threads<64, 32>(), 0);
    else if (shape == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fp64_tiles<32, 64>, fp64_threads<32, 64>(), 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fp64_tiles<32, 32>, fp64_threads<32, 32>(), 0);
    if (e != cudaSuccess) return 8;
    return n > 0 ? n : 1;
}

}  // namespace dmrg
