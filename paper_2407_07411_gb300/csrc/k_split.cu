// Split-precision (Ozaki) H_eff*psi on the tcgen05 tensor cores (the arithmetic, the
// exponent bounds and the layouts are described in split.h).  Kernels:
//   k_slice_max, k_slice_digits
//             operator vectors -> their exponents (and the row-norm bounds of the
//             stage-1 operators) and 6 BF16 digit slices in the UMMA canonical K-major
//             layout; run once when the handle is created.
//   k_xprep   per apply: every psi operand of stage 1 -> exponents, digit slices and
//             the sums the bound needs; also clears the stage-2 sums and bounds.
//   k_uest    per apply: the estimate pass, one slice pair over the stage-1 GEMMs, that
//             fixes the exponent bound of every stage-2 intermediate vector.
//   k_umma    warp-specialised slice GEMM: one producer thread streams 42 KB stages with
//             cp.async.bulk (the row groups that hold GEMM rows), one thread issues the
//             21 tcgen05.mma of each 16-K tile into five TMEM accumulators, twelve
//             epilogue warps drain the exact FP32 sums into int64 every 256 K.  Stage 1
//             turns its results into the stage-2 digit slices in the epilogue; stage 2
//             adds its int64 results atomically (exact, so order-independent).
//   k_finalize  stage-2 int64 sums -> FP64 wave-function blocks.
// Every mbarrier wait is bounded; on timeout the CTA records DMRG_ERR_DEVICE_TIMEOUT in
// the handle's status word, drains its own copies and MMAs and releases TMEM.
#include <algorithm>
#include <array>
#include <climits>
#include <map>
#include <type_traits>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "split.h"

namespace dmrg {

constexpr int UM_STAGES = 5;
constexpr int UM_EPI_WARPS = 12;      // 4 TMEM lane quarters x 3 column thirds of 32
constexpr int UM_THREADS = 64 + 32 * UM_EPI_WARPS;   // warp 0 producer, warp 1 MMA, the rest epilogue
constexpr int UM_EPI_COLS = 32;
constexpr int UM_TMEM_COLS = 512;     // five accumulators of SPL_TN columns
static_assert(SPL_ACCS * SPL_TN <= UM_TMEM_COLS && SPL_TN % 32 == 0, "TMEM accumulators");
static_assert(SPL_TN == 3 * UM_EPI_COLS, "three epilogue column thirds");
constexpr uint32_t UM_L_BYTES = SPL_S * SPL_LT * 2;   // 24 KB
constexpr uint32_t UM_R_BYTES = SPL_S * SPL_RT * 2;   // 18 KB
constexpr long long UM_WAIT_CYCLES = 4000000000ll;     // ~2 s at 2 GHz

struct UmmaSmem {
    uint16_t L[UM_STAGES][SPL_S * SPL_LT];
    uint16_t R[UM_STAGES][SPL_S * SPL_RT];
    uint64_t full[UM_STAGES], empty[UM_STAGES], tfull[SPL_ACCS], tempty[SPL_ACCS], done;
    uint32_t tmem_base;
    volatile int abort;
};

static_assert(sizeof(UmmaSmem) <= 232448, "slice GEMM shared memory exceeds the opt-in limit");
static_assert(SPL_S2_KCHUNK / SPL_DRAIN_KT <= SPL_MAX_DRAINS, "stage-2 items span too many drains");

// Device descriptors of the split plan for one number of stacked vectors.
struct SplitDevPlan {
    SGemm* gemms = nullptr;
    SWork* work1 = nullptr;
    SWork* work2 = nullptr;
    SSeg* segs = nullptr;
    SJob* jobs = nullptr;
    SXJob* xjobs = nullptr;
    SSlab* slabs = nullptr;
    SItem* items = nullptr;
    STile* tiles = nullptr;
    SBlock* blocks = nullptr;
    SPart* parts = nullptr;
    int64_t n_work1 = 0, n_work2 = 0, n_blocks = 0, n_xjobs = 0, n_items = 0, n_tiles = 0;
    std::vector<std::pair<int32_t, int32_t>> r1, r2;   // per-GEMM work ranges (per_gemm)
    int32_t xchunks = 1, fin_chunks = 1;               // CTAs per psi job / per output block
    int n_chunks = 1;                                  // output chunks and their work ranges
    std::vector<int32_t> cw1, cw2, cr1, cr2;
    int64_t s2_len = 0, mid0 = 0, mid1 = 0;
    double x_bytes = 0;                                // algorithmic DRAM bytes of the psi pass
    // per output chunk: algorithmic DRAM bytes of stage 1, stage 2 and the estimate pass,
    // and FP64-equivalent flops per vector of the two stages
    std::vector<double> s1_bytes, s2_bytes, e_bytes, s1_flops, s2_flops;
    void release() {
        void* p[] = {gemms, work1, work2, segs, jobs, xjobs, slabs, items, tiles, blocks, parts};
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

struct SplitState {
    uint16_t* op_sl = nullptr;   // operator slices (shared by every plan)
    int32_t* op_ex = nullptr;
    int32_t* srow = nullptr;     // stage-1 operator rows: sum of |top digit|
    uint16_t* ap_sl = nullptr;   // per-apply buffers, sized for the largest plan
    int32_t* ap_ex = nullptr;
    float* xs = nullptr;         // psi vectors: the bound's scaled sum of |x|
    int64_t* s2 = nullptr;
    int32_t* status = nullptr;
    std::vector<SplitDevPlan> plans;   // plans[nv - 1]
    std::vector<SplitHost> hosts;      // their host copies (work lists rebuilt per schedule)
    std::vector<size_t> cap_w1, cap_w2;
    int kid_x = -1, kid_e = -1, kid_s1 = -1, kid_s2 = -1, kid_fin = -1;
    ~SplitState() {
        for (SplitDevPlan& d : plans) d.release();
        void* p[] = {op_sl, op_ex, srow, ap_sl, ap_ex, xs, s2, status};
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

namespace {

// ----------------------------------------------------------------------------------
// digits

// Smallest E with |a| < 2^E (INT_MIN for zero).  Subnormals count: |a| = m 2^-1074 with
// m < 2^52, so |a| < 2^(msb(m) + 1 - 1074).
__device__ __forceinline__ int exp_f64(double a) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(a));
    const int ex = int((b >> 52) & 0x7FF);
    if (ex != 0) return ex - 1022;          // |a| < 2^(ex-1022)
    const unsigned long long m = b & ((1ull << 52) - 1);
    return m == 0 ? INT_MIN : (64 - __clzll(m)) - 1074;
}

// Balanced base-256 digits (each in [-127, 128]) of the non-negative integer R <= 2^47,
// most significant first, with the sign applied.  The digit set is a complete residue
// system mod 256, so the representation is unique; digit k is byte (5 - k) of
// R + 0x7F7F7F7F7F7F minus 127 (the added 127s produce exactly the carries), and
// R <= 2^47 needs no seventh digit.
__device__ __forceinline__ void balanced_digits(unsigned long long R, bool neg, int (&d)[SPL_S]) {
    const unsigned long long Rb = R + 0x7F7F7F7F7F7Full;
    const uint32_t lo = uint32_t(Rb), hi = uint32_t(Rb >> 32);
#pragma unroll
    for (int k = 0; k < SPL_S; ++k) {
        const int byte = SPL_S - 1 - k;
        const int b = int(((byte < 4 ? lo >> (8 * byte) : hi >> (8 * (byte - 4)))) & 255u);
        d[k] = neg ? 127 - b : b - 127;
    }
}

// R = round(|a| 2^(47 - E)) from the FP64 bit pattern (integer ops only).  |a| =
// m 2^(ex - 1075) for normal numbers (m with its leading bit) and m 2^-1074 for
// subnormals, i.e. the normal formula with ex = 1 and no leading bit.
__device__ __forceinline__ void digits_f64(double a, int E, int (&d)[SPL_S]) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(a));
    const int ex = int((b >> 52) & 0x7FF);
    const unsigned long long m = (b & ((1ull << 52) - 1)) | (ex != 0 ? (1ull << 52) : 0ull);
    unsigned long long R = 0;
    if (m != 0) {
        // >= 6 for normal a because |a| < 2^E; a subnormal a in a vector of subnormals
        // can need a left shift (R < 2^47 either way)
        const int sh = 1028 + E - (ex != 0 ? ex : 1);
        R = sh > 0 ? (sh >= 64 ? 0ull : (m + (1ull << (sh - 1))) >> sh) : m << (-sh);
    }
    balanced_digits(R, (b >> 63) != 0, d);
}

// BF16 bit pattern of d 2^(-8k) for a digit |d| <= 128 (exact: 8 significant bits).
// float(d) is formed as (2^23 + (d + 128)) - (2^23 + 128): both lie in [2^23, 2^24)
// where FP32 holds every integer, so the difference is exact, with full-rate FP32
// operations instead of an int->float conversion.
__device__ __forceinline__ uint16_t digit_bf16(int d, int k) {
    const float x = __uint_as_float(0x4B000000u + uint32_t(d + 128));   // 2^23 + d + 128
    const float f = (x - 8388736.0f) * __int_as_float((127 - 8 * k) << 23);   // d * 2^(-8k)
    return uint16_t(__float_as_uint(f) >> 16);
}

// Slice k of R (<= 2^47; the sign is applied by the caller) as the FP32 bit pattern of
// d_k 2^(-8k), given Rb = R + 0x7F7F7F7F7F7F: d_k is byte (5 - k) of Rb minus 127, one
// byte permute places that byte b under the exponent of 2^23, and one fused
// multiply-add forms (2^23 + b) 2^(-8k) - (2^23 + 127) 2^(-8k), exact because the result
// has at most 8 significant bits.  Only the upper 16 bits (the BF16 value) are used.
template <int k>
__device__ __forceinline__ uint32_t digit_float(unsigned long long Rb) {
    constexpr int byte = SPL_S - 1 - k;
    const uint32_t src = byte < 4 ? uint32_t(Rb) : uint32_t(Rb >> 32);
    const uint32_t u = __byte_perm(src, 0x4B000000u, 0x7540u | uint32_t(byte & 3));   // 2^23 + b
    const float s = __int_as_float((127 - 8 * k) << 23);
    return __float_as_uint(fmaf(__uint_as_float(u), s, -8388735.0f * s));
}

// ----------------------------------------------------------------------------------
// operator slicing (once per handle)

struct SliceArgs {
    const SItem* items;
    int64_t n_items;
    const SSlab* slabs;
    const SJob* jobs;
    const SSeg* segs;
    const double* ops;   // operator layout entries [ops_lo, ...) (a window of it)
    int64_t ops_lo;
    int32_t* op_ex;
};

// Exponent pass: every source row (term t, vector v) raises its vector's exponent with
// an integer atomicMax (exact, so the result does not depend on order).
__global__ void __launch_bounds__(256) k_slice_max(SliceArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const SItem I = a.items[item];
        const SSlab S = a.slabs[I.slab];
        const SJob J = a.jobs[S.job];
        const SSeg g = a.segs[S.seg];
        for (int rr = warp; rr < I.nrows; rr += 8) {
            const int64_t r = I.r0 + rr;
            const int t = int(r / J.nvalid), vec = int(r - int64_t(t) * J.nvalid);
            const int vg = vec / g.vper, vr = vec - vg * g.vper;
            const int64_t base = g.off + t * g.ts + vg * g.vgs + int64_t(vr) * g.vs - a.ops_lo;
            int E = INT_MIN;
            for (int k = lane; k < g.kc; k += 32) E = max(E, exp_f64(a.ops[base + k * g.ks]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
            if (lane == 0 && E != INT_MIN) atomicMax(a.op_ex + J.out_exp + vec, E);
        }
    }
}

struct TileArgs {
    const STile* tiles;
    int64_t n_tiles;
    const SJob* jobs;
    const SSeg* segs;
    const double* ops;   // operator layout entries [ops_lo, ...)
    int64_t ops_lo;
    uint16_t* op_sl;
    const int32_t* op_ex;
    int32_t* srow;
};

constexpr int DIG_WARPS = 8;

// Writes the digits held in sd[q][vv][0..32) (8 vectors x 32 K of slice q) as the
// 16-byte chunks of the two 16-K tiles they belong to: lanes 0-15 the first tile, lanes
// 16-31 the second (skipped beyond the job's last tile).
__device__ __forceinline__ void store_digit_block(uint16_t (*sd)[8][32], uint16_t* out, const SJob& J, int vt, int rg,
                                                  int kt0, int lane) {
    const int64_t te = int64_t(J.rows_tile) * SPL_TK;
    const int h = lane >> 4, kg = (lane >> 3) & 1, vv = lane & 7;
    const int kt = kt0 + h;
    if (kt >= J.kt) return;
#pragma unroll
    for (int q = 0; q < SPL_S; ++q) {
        const int64_t dst = J.out_tiles + ((int64_t(vt) * J.kt + kt) * SPL_S + q) * te + (rg * 2 + kg) * 64 + vv * 8;
        *reinterpret_cast<uint4*>(out + dst) = *reinterpret_cast<const uint4*>(&sd[q][vv][h * 16 + kg * 8]);
    }
}

// Digit pass: 8 vectors x 256 K of one operator job, one warp per item.  For each
// 32-K sub-block every lane decodes one K index (segment, term, entry; the padding of
// a term's run up to kcp is zero) and forms the digits of its 8 entries.
__global__ void __launch_bounds__(32 * DIG_WARPS) k_slice_digits(TileArgs a) {
    __shared__ __align__(16) uint16_t sd_all[DIG_WARPS][SPL_S][8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint16_t (*sd)[8][32] = sd_all[warp];
    for (int64_t item = int64_t(blockIdx.x) * DIG_WARPS + warp; item < a.n_tiles;
         item += int64_t(gridDim.x) * DIG_WARPS) {
        const STile T = a.tiles[item];
        const SJob J = a.jobs[T.job];
        const int nv = min(8, J.nvalid - 8 * T.vg);
        int E[8];
#pragma unroll
        for (int vv = 0; vv < 8; ++vv) E[vv] = vv < nv ? a.op_ex[J.out_exp + 8 * T.vg + vv] : 0;
        const int vt = (8 * T.vg) / J.rows_tile, rg = ((8 * T.vg) % J.rows_tile) >> 3;
        const int nsub = min(SPL_TILE_K / 32, (J.kt * SPL_TK - T.k0 + 31) / 32);
        for (int sb = 0; sb < nsub; ++sb) {
            const int K = T.k0 + sb * 32 + lane;
            int d[8][SPL_S];
#pragma unroll
            for (int vv = 0; vv < 8; ++vv)
#pragma unroll
                for (int q = 0; q < SPL_S; ++q) d[vv][q] = 0;
            if (K < J.K) {
                int sg = T.seg;   // holds the item's first K; later runs follow in order
                while (sg < J.seg0 + J.nseg - 1 && K >= a.segs[sg + 1].kbase) ++sg;
                const SSeg g = a.segs[sg];
                const int t = (K - g.kbase) / g.kcp, k = (K - g.kbase) - t * g.kcp;
                if (k < g.kc) {
                    const int64_t base = g.off + t * g.ts + k * g.ks - a.ops_lo;
                    int vg = (8 * T.vg) / g.vper, vr = 8 * T.vg - vg * g.vper;
                    double xv[8];
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv) {
                        xv[vv] = vv < nv ? a.ops[base + vg * g.vgs + int64_t(vr) * g.vs] : 0.0;
                        if (++vr == g.vper) {
                            vr = 0;
                            ++vg;
                        }
                    }
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv)
                        if (vv < nv) digits_f64(xv[vv], E[vv], d[vv]);
                }
            }
#pragma unroll
            for (int vv = 0; vv < 8; ++vv)
#pragma unroll
                for (int q = 0; q < SPL_S; ++q) sd[q][vv][lane] = digit_bf16(d[vv][q], q);
            if (J.top_sums) {   // sum |d_0| per row for the estimate pass (exact integers)
#pragma unroll
                for (int vv = 0; vv < 8; ++vv) {
                    int t0 = abs(d[vv][0]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t0 += __shfl_xor_sync(0xffffffffu, t0, o);
                    if (lane == 0 && vv < nv && t0 != 0) atomicAdd(a.srow + J.out_exp + 8 * T.vg + vv, t0);
                }
            }
            __syncwarp();
            store_digit_block(sd, a.op_sl, J, vt, rg, T.k0 / SPL_TK + sb * 2, lane);
            __syncwarp();
        }
    }
}

// ----------------------------------------------------------------------------------
// psi operands (per apply)

struct XArgs {
    const SXJob* xjobs;
    const SJob* jobs;
    const double* x;
    int64_t dim;
    uint16_t* ap_sl;
    int32_t* ap_ex;
    float* xs;
    int64_t* s2;
    int64_t s2_len;
    int64_t mid0, mid1;   // exponents of the stage-2 intermediate vectors (reset to none)
    int32_t vchunks;      // CTAs per psi job (XP_VCH vectors each)
};
constexpr int XP_VCH = 64;   // psi vectors per CTA of the psi pass (a multiple of 8)

// One CTA per (psi job, run of XP_VCH of its vectors, Davidson vector): pass 1, one warp
// per vector (a column or a row of the block), the exact exponent E and the estimate
// pass's term 1.005 2^-8
// sum |x| 2^-E (rounded up); pass 2, the digits of 8 vectors x 32 K per warp item,
// written as the 16-byte chunks of two 16-K tiles.  The grid also clears the stage-2
// sums and resets the stage-2 vector bounds to "none".
__global__ void __launch_bounds__(256) k_xprep(XArgs a) {
    __shared__ __align__(16) uint16_t sd_all[8][SPL_S][8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const int64_t nthr = int64_t(gridDim.x) * gridDim.y * blockDim.x;
        const int64_t t0 = (int64_t(blockIdx.y) * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
        for (int64_t i = t0; i < a.s2_len; i += nthr) a.s2[i] = 0;
        for (int64_t i = a.mid0 + t0; i < a.mid1; i += nthr) a.ap_ex[i] = SPL_EXP_NONE;
    }
    const SXJob X = a.xjobs[blockIdx.x / a.vchunks];
    const int k0 = int(blockIdx.x % a.vchunks) * XP_VCH, k1 = min(X.cp, k0 + XP_VCH);
    if (k0 >= X.cp) return;
    const SJob J = a.jobs[X.job];
    const int v = blockIdx.y;
    const double* src = a.x + int64_t(v) * a.dim + X.off;
    int32_t* ex = a.ap_ex + J.out_exp + int64_t(v) * X.cp;
    float* xs = a.xs + J.out_exp + int64_t(v) * X.cp;
    for (int k = k0 + warp; k < k1; k += 8) {
        int E = INT_MIN;
        if (k < X.nk)
            for (int K = lane; K < X.K; K += 32) E = max(E, exp_f64(src[int64_t(K) * X.ks + int64_t(k) * X.vs]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
        double s1 = 0.0;
        if (E != INT_MIN) {
            for (int K = lane; K < X.K; K += 32) s1 += fabs(scalbn(src[int64_t(K) * X.ks + int64_t(k) * X.vs], -E));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (lane == 0) {
            ex[k] = E == INT_MIN ? SPL_EXP_NONE : E;
            // the sum's rounding (relative 2^-40 at most) is covered by the 1.005 factor
            xs[k] = __double2float_ru(s1 * (1.005 / 256.0));
        }
    }
    __syncthreads();   // the exponents written above are visible to the whole CTA
    uint16_t (*sd)[8][32] = sd_all[warp];
    const int g0 = k0 / 8, ngrp = (k1 - k0) / 8, nsub = (X.K + 31) / 32;
    for (int it = warp; it < ngrp * nsub; it += 8) {
        const int g8 = g0 + it / nsub, sb = it - (it / nsub) * nsub;
        const int K = sb * 32 + lane;
#pragma unroll
        for (int vv = 0; vv < 8; ++vv) {
            const int k = 8 * g8 + vv;
            int d[SPL_S] = {0, 0, 0, 0, 0, 0};
            if (K < X.K && k < X.nk) {
                const int E = ex[k];
                if (E != SPL_EXP_NONE) digits_f64(src[int64_t(K) * X.ks + int64_t(k) * X.vs], E, d);
            }
#pragma unroll
            for (int q = 0; q < SPL_S; ++q) sd[q][vv][lane] = digit_bf16(d[q], q);
        }
        __syncwarp();
        const int n0 = v * X.cp + 8 * g8;   // job vector of this group's first vector
        store_digit_block(sd, a.ap_sl, J, n0 / J.rows_tile, (n0 % J.rows_tile) >> 3, sb * 2, lane);
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------------
// tcgen05 slice GEMM

__device__ __forceinline__ uint32_t su32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor, K-major without swizzle: 8x8 core matrices of 128
// contiguous bytes, LBO = 128 B between the two K-adjacent cores of a 16-K tile, SBO =
// 256 B between 8-row groups.  The low word holds the start address (bits 0-13, address
// / 16) and LBO / 16 (bits 16-29); the high word SBO / 16 (bits 32-45) and the fixed
// version bit 46.  Every operand of a stage sits below 256 KB of shared memory, so
// operand offsets are added to the low word without a carry out of the address field.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr) { return ((addr >> 4) & 0x3FFF) | ((128u >> 4) << 16); }
constexpr uint32_t UM_DESC_HI = (256u >> 4) | (1u << (46 - 32));

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major, M=128, N=n
// (a multiple of 16 up to SPL_TN).
__host__ __device__ constexpr uint32_t um_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(SPL_TM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t ph) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(ph)
        : "memory");
    return ok != 0;
}

// Bounded wait; false on timeout (recorded in *abort and the status word) or when
// another role of the CTA has aborted.
// The abort flag and the clock are looked at only every 16th poll: the flag lives in
// shared memory, whose bandwidth the tensor cores' operand reads need, and twelve
// epilogue warps wait at once.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* b, uint32_t ph, long long limit, volatile int* abort,
                                                int* status) {
    if (mbar_try(b, ph)) return true;
    const long long t0 = clock64();
    for (unsigned n = 1;; ++n) {
        if (mbar_try(b, ph)) return true;
        if ((n & 15u) == 0) {
            if (*abort) return false;
            if (clock64() - t0 > limit) {
                *abort = 1;
                atomicExch(status, DMRG_ERR_DEVICE_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ bool mbar_wait(UmmaSmem& sm, uint64_t* b, uint32_t ph, int* status) {
    return mbar_wait_limit(b, ph, UM_WAIT_CYCLES, &sm.abort, status);
}

__device__ __forceinline__ bool mbar_wait_final(uint64_t* b, uint32_t ph) {
    const long long t0 = clock64();
    while (!mbar_try(b, ph))
        if (clock64() - t0 > UM_WAIT_CYCLES) return false;
    return true;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void umma(uint32_t d, uint32_t a_lo, uint32_t b_lo, uint32_t accumulate, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\n.reg .b64 da, db;\nsetp.ne.b32 p, %3, 0;\nmov.b64 da, {%1, %4};\nmov.b64 db, {%2, %4};\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(d),
        "r"(a_lo), "r"(b_lo), "r"(accumulate), "r"(UM_DESC_HI), "r"(idesc));
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
}

// Work list of one slice-GEMM launch (the Davidson vectors of an apply are stacked
// inside its GEMMs).
struct UmmaArgs {
    const SWork* work;
    int64_t n_work;
    const SGemm* gemms;
    const uint16_t* op_sl;
    uint16_t* ap_sl;
    int64_t* s2;
    const int32_t* op_ex;
    int32_t* ap_ex;
    int* status;
};

// Issue order of the 21 slice pairs (i, j) of a 16-K tile: accumulator c (pair level c
// for c < 4, levels 4 and 5 for c = 4) alternates with the others, so that consecutive
// MMAs never feed the same accumulator (a run into one accumulator stalls on its own
// sum).  The first tile of a chunk ("open" tile) uses a second order in which the first
// uses of the accumulators come as late as the alternation allows, in the order 4, 3,
// 2, 1, 0 in which the epilogue empties them (accumulator 0 at the 20th MMA), so the
// issuer waits as little as possible for the drains; both orders take the pairs of
// accumulator 4 in the same sequence (its inexact FP32 sums do not depend on which
// order a tile uses).
#define UM_ORDER_C {4, 3, 4, 2, 4, 3, 4, 1, 4, 2, 4, 3, 4, 0, 4, 1, 4, 2, 4, 3, 4}
#define UM_ORDER_I {0, 0, 1, 0, 2, 1, 3, 0, 4, 1, 0, 2, 1, 0, 2, 1, 3, 2, 4, 3, 5}
#define UM_ORDER_J {4, 3, 3, 2, 2, 2, 1, 1, 0, 1, 5, 1, 4, 0, 3, 0, 2, 0, 1, 0, 0}
#define UM_OPEN_C {4, 3, 4, 3, 4, 3, 4, 3, 4, 2, 4, 2, 4, 2, 4, 1, 4, 1, 4, 0, 4}
#define UM_OPEN_I {0, 0, 1, 1, 2, 2, 3, 3, 4, 0, 0, 1, 1, 2, 2, 0, 3, 1, 4, 0, 5}
#define UM_OPEN_J {4, 3, 3, 2, 2, 1, 1, 0, 0, 2, 5, 1, 4, 0, 3, 1, 2, 0, 1, 0, 0}

// Drain schedule: after item-relative K tile kt, when the tile closes a chunk d = kt / 16
// of 16 tiles (256 K) or the work item, the accumulators of mask um_drain_mask are
// emptied.  Accumulators 2, 3 (exact up to 341 and 256 K) and 4 are emptied after every
// chunk; accumulator 1 (exact up to 512 K: |sum| <= 2 * 512 * 2^14 = 2^24 units) after
// every second, accumulator 0 (up to 1024 K) after every fourth, and all of them at the
// item's end.  Exact sums do not depend on where they are cut, and accumulator 4's
// rounding points are the chunk ends; stage-2 items start at multiples of 16 tiles, so
// the result does not depend on how a stage-2 GEMM is cut into items.  (Staggering the
// chunk ends of the five accumulators was measured slower: the MMAs of the accumulator
// whose chunk starts had to run back to back.)
__host__ __device__ __forceinline__ bool um_drains(int kt, int len) {
    return kt == len - 1 || kt % SPL_DRAIN_KT == SPL_DRAIN_KT - 1;
}
__host__ __device__ __forceinline__ int um_drain_mask(int kt, int len) {
    if (kt == len - 1) return 0x1F;
    const int d = kt / SPL_DRAIN_KT;
    return 0x1C | ((d & 1) ? 0x2 : 0) | ((d & 3) == 3 ? 0x1 : 0);
}

// The 21 MMAs of one 16-K tile, fully unrolled.  OPEN = false: every accumulator keeps
// accumulating.  OPEN = true: the tile starts a chunk; each accumulator of open_mask
// (the ones emptied at the end of the previous chunk, or all at an item's start) waits
// for its own drain (tempty) before its first pair, which overwrites it; the others keep
// accumulating.  nd[c] counts the drains of accumulator c so far in this CTA.
template <bool OPEN>
__device__ __forceinline__ bool issue_tile(UmmaSmem& sm, uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t idesc,
                                           const int (&nd)[SPL_ACCS], int open_mask, int* status) {
    constexpr int sc[SPL_PAIRS] = UM_ORDER_C, si[SPL_PAIRS] = UM_ORDER_I, sj[SPL_PAIRS] = UM_ORDER_J;
    constexpr int pc[SPL_PAIRS] = UM_OPEN_C, pi[SPL_PAIRS] = UM_OPEN_I, pj[SPL_PAIRS] = UM_OPEN_J;
#pragma unroll
    for (int p = 0; p < SPL_PAIRS; ++p) {
        const int c = OPEN ? pc[p] : sc[p];
        const int i = OPEN ? pi[p] : si[p], j = OPEN ? pj[p] : sj[p];
        bool first = OPEN;
#pragma unroll
        for (int p2 = 0; p2 < p; ++p2)
            if ((OPEN ? pc[p2] : sc[p2]) == c) first = false;
        first = first && ((open_mask >> c) & 1);
        if (first && nd[c] > 0) {
            if (!mbar_wait(sm, &sm.tempty[c], uint32_t((nd[c] - 1) & 1), status)) return false;
            tc_fence_after();
        }
        umma(tmem + uint32_t(c * SPL_TN), a0 + uint32_t(i * (SPL_LT * 2)) / 16, b0 + uint32_t(j * (SPL_RT * 2)) / 16,
             first ? 0u : 1u, idesc);
    }
    return true;
}

// Drain of accumulator c into the int64 sums acc (units of 2^-31 of the digit-product
// unit).  32-bit conversions only (the 64-bit one is an FP64-rate operation): acc c holds
// the exact level sum in units of 2^(-8c) for c < 4 (|sum| <= 2^24 in those units, acc 0
// over up to four chunks and acc 1 over two), acc 4 the rest, rounded to units of 2^-31
// (< 2^24 of them); each is added in units of 2^-31, and the running sum of a work item
// (at most 8192 K, a partial sum of its digit products) stays below 2^58.01.  The
// accumulator is handed back to the MMA issuer as soon as it is in registers.  n: the
// drains of accumulator c before this one.
template <int c>
__device__ __forceinline__ bool drain_acc(UmmaSmem& sm, uint32_t tmem_row, int col0, int n,
                                          long long (&acc)[UM_EPI_COLS], int* status) {
    // warp-uniform outcome: the TMEM loads below are .sync.aligned
    if (!__all_sync(0xffffffffu, mbar_wait(sm, &sm.tfull[c], uint32_t(n & 1), status))) return false;
    tc_fence_after();
    uint32_t rv[UM_EPI_COLS];
    tmem_ld32(tmem_row + uint32_t(c * SPL_TN + col0), rv);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_fence_before();
    mbar_arrive(&sm.tempty[c]);
    constexpr float scale = c == 0 ? 1.0f : c == 1 ? 256.0f : c == 2 ? 65536.0f : c == 3 ? 16777216.0f : 2147483648.0f;
#pragma unroll
    for (int j = 0; j < UM_EPI_COLS; ++j) {
        const int iv = __float2int_rn(__uint_as_float(rv[j]) * scale);
        if constexpr (c < SPL_ACCS - 1)
            acc[j] += static_cast<long long>(iv) * (1ll << (31 - 8 * c));
        else
            acc[j] += iv;
    }
    return true;
}

// The exponents the stage-1 epilogue needs, loaded before the drain so that no global
// load sits between the drain and the stores: the psi vector exponents of the warp's 32
// columns (lane l holds column cbase + l), the row's operator exponent and the bound of
// the stage-2 vector of each group of 8 columns.
struct S1Pre { int ec_lane, erow, E[UM_EPI_COLS / 8]; };

__device__ __forceinline__ S1Pre stage1_prefetch(const UmmaArgs& a, const SGemm& G, int r, int cbase, int lane) {
    S1Pre p;
    p.ec_lane = cbase + lane < G.N ? a.ap_ex[G.ec_off + cbase + lane] : 0;
    p.erow = 0;
#pragma unroll
    for (int g = 0; g < UM_EPI_COLS / 8; ++g) p.E[g] = SPL_EXP_NONE;
    if (r < G.M) {
        p.erow = a.op_ex[G.er_off + r];
        const int i = r % G.per;
#pragma unroll
        for (int g = 0; g < UM_EPI_COLS / 8; ++g) {
            const int col = cbase + 8 * g;
            if (col < G.N) p.E[g] = a.ap_ex[G.dst_exp + (col / G.cp) * G.per + i];
        }
    }
    return p;
}

// Stage-1 epilogue: this thread's row of the tile and its 32 columns (4 groups of 8; a
// group lies inside one Davidson vector because cp is a multiple of 8) -> 6 digits per
// entry relative to the stage-2 vector bound, stored as 16-byte chunks (8 K of one
// slice) straight into the stage-2 job's tiles.
__device__ __forceinline__ void stage1_store(const UmmaArgs& a, const SGemm& G, int r, int cbase, const S1Pre& pre,
                                             const long long (&acc)[UM_EPI_COLS]) {
    const bool rv = r < G.M;
    const int t = rv ? r / G.per : 0, i = rv ? r - t * G.per : 0;
    const int erow = pre.erow;
    const int ec_lane = pre.ec_lane;
    int vprev = -1, E = SPL_EXP_NONE;
    int64_t tile_base = 0;
    int vr = 0;
    const int64_t tile_elems = int64_t(SPL_S) * G.dst_rows_tile * SPL_TK;
#pragma unroll
    for (int g = 0; g < UM_EPI_COLS / 8; ++g) {
        const int col = cbase + 8 * g;   // the same for every lane
        int ec[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) ec[e] = __shfl_sync(0xffffffffu, ec_lane, 8 * g + e);
        if (!rv || col >= G.N) continue;
        const int v = col / G.cp, k0 = col - v * G.cp;
        E = pre.E[g];   // bound from the estimate pass
        if (v != vprev) {
            vprev = v;
            const int V = v * G.per + i;
            const int vt = V / G.dst_rows_tile;
            vr = V - vt * G.dst_rows_tile;
            tile_base = G.d_off + int64_t(vt) * G.dst_kt * tile_elems;
        }
        const int K0 = G.kbase + t * G.cp + k0;
        unsigned long long Rb[8];
        uint32_t sgn[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const long long F = G.sign > 0 ? acc[8 * g + e] : -acc[8 * g + e];
            unsigned long long R = 0;
            if (F != 0) {
                const unsigned long long u =
                    F < 0 ? static_cast<unsigned long long>(-F) : static_cast<unsigned long long>(F);
                // value = F 2^(erow + ec - 45) < 2^E; R = round(|value| 2^(47 - E)) = round(|F| 2^-sh)
                // (the bound keeps sh > -47; the clamp only keeps shifts defined)
                const int sh = E - erow - ec[e] - 2;
                R = sh > 0 ? (sh >= 64 ? 0ull : (u + (1ull << (sh - 1))) >> sh) : (sh > -64 ? u << (-sh) : 0ull);
            }
            Rb[e] = R + 0x7F7F7F7F7F7Full;
            sgn[e] = F < 0 ? 0x80000000u : 0u;
        }
        const int kt = K0 >> 4, kh = (K0 >> 3) & 1;
        uint4* dst = reinterpret_cast<uint4*>(a.ap_sl + tile_base + int64_t(kt) * tile_elems +
                                              ((vr >> 3) * 2 + kh) * 64 + (vr & 7) * 8);
        const int64_t qstride = int64_t(G.dst_rows_tile) * SPL_TK / 8;   // one slice, in 16-byte units
        auto put = [&](auto kc) {
            constexpr int q = decltype(kc)::value;
            uint32_t w[4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
                w[p] = __byte_perm(digit_float<q>(Rb[2 * p]) ^ sgn[2 * p], digit_float<q>(Rb[2 * p + 1]) ^ sgn[2 * p + 1],
                                   0x7632);
            dst[q * qstride] = make_uint4(w[0], w[1], w[2], w[3]);
        };
        put(std::integral_constant<int, 0>{});
        put(std::integral_constant<int, 1>{});
        put(std::integral_constant<int, 2>{});
        put(std::integral_constant<int, 3>{});
        put(std::integral_constant<int, 4>{});
        put(std::integral_constant<int, 5>{});
    }
}

__global__ void __launch_bounds__(UM_THREADS, 1) k_umma(UmmaArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    UmmaSmem& sm = *reinterpret_cast<UmmaSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem_base)),
                     "r"(UM_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // zero the operand stages once: rows that are never copied then hold valid digits
    {
        uint4* z = reinterpret_cast<uint4*>(&sm.L[0][0]);
        constexpr int n16 = int((sizeof(sm.L) + sizeof(sm.R)) / 16);
        static_assert(offsetof(UmmaSmem, R) == sizeof(UmmaSmem::L), "stages are contiguous");
        for (int i = threadIdx.x; i < n16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < UM_STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int c = 0; c < SPL_ACCS; ++c) {
            mbar_init(&sm.tfull[c], 1);
            mbar_init(&sm.tempty[c], 32 * UM_EPI_WARPS);
        }
        mbar_init(&sm.done, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const int64_t total = a.n_work;
    const int64_t step = gridDim.x;

    if (warp == 0 && lane == 0) {
        // ---- producer
        int64_t kidx = 0;
        bool ok = true;
        // descriptors are loaded ahead (the work item two items ahead, its GEMM one
        // item ahead), so no dependent global load sits at an item boundary
        SWork W1{}, W2{};
        SGemm G1{};
        if (blockIdx.x < total) {
            W1 = a.work[blockIdx.x];
            G1 = a.gemms[W1.gemm];
        }
        if (blockIdx.x + step < total) W2 = a.work[blockIdx.x + step];
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = W1;
            const SGemm G = G1;
            W1 = W2;
            if (it + step < total) G1 = a.gemms[W1.gemm];
            if (it + 2 * step < total) W2 = a.work[it + 2 * step];
            const uint16_t* Lb = (G.l_buf ? a.ap_sl : a.op_sl) + G.l_tiles;
            const uint16_t* Rb = (G.r_buf ? a.ap_sl : a.op_sl) + G.r_tiles;
            // only the 8-row groups that hold rows of the GEMM are copied: the first lg (rg)
            // 256-byte groups of every slice; the rest of the stage keeps digits of an
            // earlier tile (or the zeros of set-up), whose products land in accumulator
            // rows / columns that the epilogue never reads
            const int lg = (min(SPL_TM, G.M - W.mtile * SPL_TM) + 7) >> 3;
            const int rg = (min(SPL_TN, G.N - W.ntile * SPL_TN) + 7) >> 3;
            const uint32_t lbytes = uint32_t(lg) * 256u, rbytes = uint32_t(rg) * 256u;
            for (int kt = W.k0; kt < W.k1; ++kt, ++kidx) {
                const int s = int(kidx % UM_STAGES);
                const int64_t n = kidx / UM_STAGES;
                if (n > 0 && !(ok = mbar_wait(sm, &sm.empty[s], uint32_t((n - 1) & 1), a.status))) break;
                mbar_expect_tx(&sm.full[s], uint32_t(SPL_S) * (lbytes + rbytes));
                const uint16_t* lt = Lb + (int64_t(W.mtile) * G.kt + kt) * (SPL_S * SPL_LT);
                const uint16_t* rt = Rb + (int64_t(W.ntile) * G.kt + kt) * (SPL_S * SPL_RT);
                if (lbytes == UM_L_BYTES / SPL_S) {
                    bulk_g2s(sm.L[s], lt, UM_L_BYTES, &sm.full[s]);
                } else {
                    for (int q = 0; q < SPL_S; ++q) bulk_g2s(sm.L[s] + q * SPL_LT, lt + q * SPL_LT, lbytes, &sm.full[s]);
                }
                if (rbytes == UM_R_BYTES / SPL_S) {
                    bulk_g2s(sm.R[s], rt, UM_R_BYTES, &sm.full[s]);
                } else {
                    for (int q = 0; q < SPL_S; ++q) bulk_g2s(sm.R[s] + q * SPL_RT, rt + q * SPL_RT, rbytes, &sm.full[s]);
                }
            }
        }
        // every issued stage must land before the CTA may exit
        for (int64_t q = kidx - UM_STAGES; q < kidx; ++q)
            if (q >= 0) mbar_wait_final(&sm.full[q % UM_STAGES], uint32_t((q / UM_STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        int64_t kidx = 0;
        int nd[SPL_ACCS] = {0, 0, 0, 0, 0};
        bool ok = true;
        SWork Wn{};
        SGemm Gn{};
        if (blockIdx.x < total) {
            Wn = a.work[blockIdx.x];
            Gn = a.gemms[Wn.gemm];
        }
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = Wn;
            // the MMA's N: the tile's valid columns rounded up to 16
            const int ncols = min(SPL_TN, Gn.N - W.ntile * SPL_TN);
            const uint32_t idesc = um_idesc((ncols + 15) & ~15);
            if (it + step < total) {
                Wn = a.work[it + step];
                Gn = a.gemms[Wn.gemm];
            }
            const int len = W.k1 - W.k0;
            for (int kt = 0; kt < len; ++kt, ++kidx) {
                const int s = int(kidx % UM_STAGES);
                if (!(ok = mbar_wait(sm, &sm.full[s], uint32_t((kidx / UM_STAGES) & 1), a.status))) break;
                tc_fence_after();
                const uint32_t a0 = sdesc_lo(su32(sm.L[s])), b0 = sdesc_lo(su32(sm.R[s]));
                // a chunk's first tile: the accumulators emptied at the end of the previous
                // chunk (all at an item's start) start over
                if (kt == 0 || um_drains(kt - 1, len))
                    ok = issue_tile<true>(sm, tmem, a0, b0, idesc, nd, kt == 0 ? 0x1F : um_drain_mask(kt - 1, len),
                                          a.status);
                else
                    ok = issue_tile<false>(sm, tmem, a0, b0, idesc, nd, 0, a.status);
                if (!ok) break;
                umma_commit(&sm.empty[s]);
                if (um_drains(kt, len)) {
                    const int m = um_drain_mask(kt, len);
#pragma unroll
                    for (int c = SPL_ACCS - 1; c >= 0; --c)
                        if ((m >> c) & 1) {
                            umma_commit(&sm.tfull[c]);
                            ++nd[c];
                        }
                }
            }
        }
        umma_commit(&sm.done);   // completes when every MMA issued above has finished
        mbar_wait_final(&sm.done, 0);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (tile rows) and the column
        // third (w-2)/4 of every accumulator
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = 32 * q + lane, col0 = h * UM_EPI_COLS;
        const uint32_t tmem_row = tmem + (uint32_t(32 * q) << 16);
        int nd[SPL_ACCS] = {0, 0, 0, 0, 0};
        bool ok = true;
        // the next work item is loaded ahead; its GEMM descriptor is read at the item's
        // start, while the first drain waits for the MMAs
        SWork W1{};
        if (blockIdx.x < total) W1 = a.work[blockIdx.x];
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = W1;
            if (it + step < total) W1 = a.work[it + step];
            const int r = W.mtile * SPL_TM + row;
            const int cbase = W.ntile * SPL_TN + col0;
            // stage 1: the exponents of the epilogue, loaded before the drain (the GEMM
            // descriptor is read again after it, from L1)
            S1Pre pre{};
            {
                const SGemm G0 = a.gemms[W.gemm];
                if (G0.kind == 0) pre = stage1_prefetch(a, G0, r, cbase, lane);
            }
            long long acc[UM_EPI_COLS];
#pragma unroll
            for (int j = 0; j < UM_EPI_COLS; ++j) acc[j] = 0;
            const int len = W.k1 - W.k0;
            for (int kt = 0; kt < len && ok; ++kt) {
                if (!um_drains(kt, len)) continue;
                const int m = um_drain_mask(kt, len);
                ok = drain_acc<4>(sm, tmem_row, col0, nd[4], acc, a.status) &&
                     drain_acc<3>(sm, tmem_row, col0, nd[3], acc, a.status) &&
                     drain_acc<2>(sm, tmem_row, col0, nd[2], acc, a.status) &&
                     (!(m & 2) || drain_acc<1>(sm, tmem_row, col0, nd[1], acc, a.status)) &&
                     (!(m & 1) || drain_acc<0>(sm, tmem_row, col0, nd[0], acc, a.status));
#pragma unroll
                for (int c = 0; c < SPL_ACCS; ++c) nd[c] += (m >> c) & 1;
            }
            if (!ok) break;
            const SGemm G = a.gemms[W.gemm];
            if (G.kind == 0) {
                stage1_store(a, G, r, cbase, pre, acc);
            } else if (r < G.M) {
                // F = round(2^fs * sum): exact for fs >= 31 (up to 32 drains of 2^53.01 stay
                // below 2^58.01; the GEMM's shift keeps F below 2^62); for fs < 31 only the
                // part below 2^-fs, i.e. of acc 4, is rounded
                const int fs = G.fshift;
                unsigned long long* D = reinterpret_cast<unsigned long long*>(a.s2 + G.d_off + int64_t(r) * G.ldd);
#pragma unroll
                for (int j = 0; j < UM_EPI_COLS; ++j) {
                    const long long F = fs >= 31
                                            ? static_cast<long long>(static_cast<unsigned long long>(acc[j]) << (fs - 31))
                                            : (acc[j] + (1ll << (30 - fs))) >> (31 - fs);
                    const int c = cbase + j;
                    if (c < G.N && F != 0) atomicAdd(D + c, static_cast<unsigned long long>(F));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UM_TMEM_COLS));
    }
}

// ----------------------------------------------------------------------------------
// estimate pass: the stage-2 vector bounds

constexpr int EST_KT = 4;          // K tiles per stage (slice 0 of each)
constexpr int EST_STAGES = 6;
constexpr int EST_DRAIN_KT = 64;   // level-0 sums stay exact integers below 2^24 for 1024 K
constexpr int EST_TMEM_COLS = 256; // two accumulator slots of SPL_TN columns
struct EstSmem {
    uint16_t L[EST_STAGES][EST_KT * SPL_LT];
    uint16_t R[EST_STAGES][EST_KT * SPL_RT];
    uint64_t full[EST_STAGES], empty[EST_STAGES], tfull[2], tempty[2], done;
    uint32_t tmem_base;
    volatile int abort;
};
static_assert(sizeof(EstSmem) <= 232448, "estimate pass shared memory");
static_assert(2 * SPL_TN <= EST_TMEM_COLS, "estimate accumulators");

struct EstArgs {
    const SWork* work;
    int64_t n_work;
    const SGemm* gemms;
    const uint16_t* op_sl;
    const uint16_t* ap_sl;
    const int32_t* op_ex;
    int32_t* ap_ex;
    const int32_t* srow;
    const float* xs;
    int* status;
};

__device__ __forceinline__ bool est_wait(EstSmem& sm, uint64_t* b, uint32_t ph, int* status) {
    return mbar_wait_limit(b, ph, UM_WAIT_CYCLES, &sm.abort, status);
}

// Over the stage-1 work list: the top-digit product X~ = sum a~ x~ (slice pair (0, 0),
// one MMA per 16-K tile, exact integer sums drained every 1024 K into two alternating
// TMEM slots), then per entry the bound
//     |X| < 2^(E_a + E_x) f,  f = |X~| 2^-(E_a+E_x) + 1.005 2^-8 (sum|x| 2^-E_x + sum|a~| 2^-E_a)
// (enlarged by 2^-20 relative and 2^-30 absolute for the rounding of f and of the
// stage-1 result), and each stage-2 vector's bound exponent is raised to the largest
// E_a + E_x + ceil(log2 f) of its entries with an integer atomicMax.
__global__ void __launch_bounds__(UM_THREADS, 1) k_uest(EstArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    EstSmem& sm = *reinterpret_cast<EstSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem_base)),
                     "r"(EST_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    {
        uint4* z = reinterpret_cast<uint4*>(&sm.L[0][0]);
        constexpr int n16 = int((sizeof(sm.L) + sizeof(sm.R)) / 16);
        static_assert(offsetof(EstSmem, R) == sizeof(EstSmem::L), "stages are contiguous");
        for (int i = threadIdx.x; i < n16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < EST_STAGES; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], 1);
        }
        for (int c = 0; c < 2; ++c) {
            mbar_init(&sm.tfull[c], 1);
            mbar_init(&sm.tempty[c], 32 * UM_EPI_WARPS);
        }
        mbar_init(&sm.done, 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const int64_t total = a.n_work;
    const int64_t step = gridDim.x;

    if (warp == 0 && lane == 0) {
        // ---- producer: slice 0 of EST_KT K tiles of L and R per stage
        int64_t sidx = 0;
        bool ok = true;
        // descriptors loaded ahead, as in the slice GEMM: no dependent global load at an
        // item boundary (the items of this pass are short)
        SWork W1{}, W2{};
        SGemm G1{};
        if (blockIdx.x < total) {
            W1 = a.work[blockIdx.x];
            G1 = a.gemms[W1.gemm];
        }
        if (blockIdx.x + step < total) W2 = a.work[blockIdx.x + step];
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = W1;
            const SGemm G = G1;
            W1 = W2;
            if (it + step < total) G1 = a.gemms[W1.gemm];
            if (it + 2 * step < total) W2 = a.work[it + 2 * step];
            const uint16_t* Lb = (G.l_buf ? a.ap_sl : a.op_sl) + G.l_tiles;
            const uint16_t* Rb = (G.r_buf ? a.ap_sl : a.op_sl) + G.r_tiles;
            const int lg = (min(SPL_TM, G.M - W.mtile * SPL_TM) + 7) >> 3;
            const int rg = (min(SPL_TN, G.N - W.ntile * SPL_TN) + 7) >> 3;
            for (int kt0 = W.k0; kt0 < W.k1; kt0 += EST_KT, ++sidx) {
                const int s = int(sidx % EST_STAGES);
                const int64_t n = sidx / EST_STAGES;
                if (n > 0 && !(ok = est_wait(sm, &sm.empty[s], uint32_t((n - 1) & 1), a.status))) break;
                const int nk = min(EST_KT, W.k1 - kt0);
                mbar_expect_tx(&sm.full[s], uint32_t(nk) * uint32_t(lg + rg) * 256u);
                for (int j = 0; j < nk; ++j) {
                    bulk_g2s(sm.L[s] + j * SPL_LT, Lb + (int64_t(W.mtile) * G.kt + kt0 + j) * (SPL_S * SPL_LT),
                             uint32_t(lg) * 256u, &sm.full[s]);
                    bulk_g2s(sm.R[s] + j * SPL_RT, Rb + (int64_t(W.ntile) * G.kt + kt0 + j) * (SPL_S * SPL_RT),
                             uint32_t(rg) * 256u, &sm.full[s]);
                }
            }
        }
        for (int64_t q = sidx - EST_STAGES; q < sidx; ++q)
            if (q >= 0) mbar_wait_final(&sm.full[q % EST_STAGES], uint32_t((q / EST_STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: one MMA per K tile into the slot of the current drain chunk
        int64_t sidx = 0, chunk = 0;
        bool ok = true;
        SWork Wn{};
        int Nn = 0;
        if (blockIdx.x < total) {
            Wn = a.work[blockIdx.x];
            Nn = a.gemms[Wn.gemm].N;
        }
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = Wn;
            const int ncols = min(SPL_TN, Nn - W.ntile * SPL_TN);
            if (it + step < total) {
                Wn = a.work[it + step];
                Nn = a.gemms[Wn.gemm].N;
            }
            const uint32_t idesc = um_idesc((ncols + 15) & ~15);
            for (int kc0 = W.k0; kc0 < W.k1 && ok; kc0 += EST_DRAIN_KT, ++chunk) {
                const int kc1 = min(kc0 + EST_DRAIN_KT, W.k1);
                const int slot = int(chunk & 1);
                if (chunk >= 2) {   // the slot's previous chunk has been read
                    if (!(ok = est_wait(sm, &sm.tempty[slot], uint32_t(((chunk >> 1) - 1) & 1), a.status))) break;
                    tc_fence_after();
                }
                for (int kt0 = kc0; kt0 < kc1; kt0 += EST_KT, ++sidx) {
                    const int s = int(sidx % EST_STAGES);
                    if (!(ok = est_wait(sm, &sm.full[s], uint32_t((sidx / EST_STAGES) & 1), a.status))) break;
                    tc_fence_after();
                    const int nk = min(EST_KT, kc1 - kt0);
                    const uint32_t a0 = sdesc_lo(su32(sm.L[s])), b0 = sdesc_lo(su32(sm.R[s]));
                    for (int j = 0; j < nk; ++j)
                        umma(tmem + uint32_t(slot * SPL_TN), a0 + uint32_t(j * SPL_LT * 2) / 16,
                             b0 + uint32_t(j * SPL_RT * 2) / 16, (kt0 == kc0 && j == 0) ? 0u : 1u, idesc);
                    umma_commit(&sm.empty[s]);
                }
                if (ok) umma_commit(&sm.tfull[slot]);
            }
        }
        umma_commit(&sm.done);
        mbar_wait_final(&sm.done, 0);
    } else if (warp >= 2) {
        // ---- epilogue
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = 32 * q + lane, col0 = h * UM_EPI_COLS;
        const uint32_t tmem_row = tmem + (uint32_t(32 * q) << 16);
        int64_t chunk = 0;
        bool ok = true;
        SWork W1{}, W2{};
        SGemm G1{};
        if (blockIdx.x < total) {
            W1 = a.work[blockIdx.x];
            G1 = a.gemms[W1.gemm];
        }
        if (blockIdx.x + step < total) W2 = a.work[blockIdx.x + step];
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = W1;
            const SGemm G = G1;
            W1 = W2;
            if (it + step < total) G1 = a.gemms[W1.gemm];
            if (it + 2 * step < total) W2 = a.work[it + 2 * step];
            const int r = W.mtile * SPL_TM + row;
            const int cbase = W.ntile * SPL_TN + col0;
            // every load of the bound is issued before the drain wait
            int ex_lane = SPL_EXP_NONE;
            float xs_lane = 0.0f;
            if (cbase + lane < G.N) {
                ex_lane = a.ap_ex[G.ec_off + cbase + lane];
                xs_lane = a.xs[G.ec_off + cbase + lane];
            }
            const bool rv_ok = r < G.M;
            const int ea = rv_ok ? a.op_ex[G.er_off + r] : SPL_EXP_NONE;
            const int sa_i = rv_ok ? a.srow[G.er_off + r] : 0;
            // the level-0 sums: an item of one chunk (every stage-1 item up to 1024 K)
            // keeps the exact FP32 sum itself (bits in acc); longer ones add chunks in int
            const bool one_chunk = W.k1 - W.k0 <= EST_DRAIN_KT;
            int acc[UM_EPI_COLS];
#pragma unroll
            for (int j = 0; j < UM_EPI_COLS; ++j) acc[j] = 0;
            for (int kc0 = W.k0; kc0 < W.k1 && ok; kc0 += EST_DRAIN_KT, ++chunk) {
                const int slot = int(chunk & 1);
                ok = __all_sync(0xffffffffu, est_wait(sm, &sm.tfull[slot], uint32_t((chunk >> 1) & 1), a.status));
                if (!ok) break;
                tc_fence_after();
                uint32_t rv[UM_EPI_COLS];
                tmem_ld32(tmem_row + uint32_t(slot * SPL_TN + col0), rv);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&sm.tempty[slot]);
                if (one_chunk) {
#pragma unroll
                    for (int j = 0; j < UM_EPI_COLS; ++j) acc[j] = int(rv[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < UM_EPI_COLS; ++j) acc[j] += __float2int_rn(__uint_as_float(rv[j]));
                }
            }
            if (!ok) break;
            const int i = rv_ok ? r % G.per : 0;
            const float sa = float(sa_i) * (1.005f / 32768.0f);
            // the Davidson vector of the columns changes at multiples of cp (>= 8), the
            // same for every lane: no division per column
            int v = cbase / G.cp, vend = (v + 1) * G.cp, Emax = SPL_EXP_NONE;
            const bool row_ok = rv_ok && ea > -(1 << 28);
            int32_t* dst = a.ap_ex + G.dst_exp + i;
#pragma unroll
            for (int j = 0; j < UM_EPI_COLS; ++j) {
                const int ex = __shfl_sync(0xffffffffu, ex_lane, j);
                const float xsj = __shfl_sync(0xffffffffu, xs_lane, j);
                const int col = cbase + j;
                if (col >= vend) {
                    if (row_ok && Emax > SPL_EXP_NONE) atomicMax(dst + v * G.per, Emax);
                    ++v;
                    vend += G.cp;
                    Emax = SPL_EXP_NONE;
                }
                const float aj = one_chunk ? fabsf(__int_as_float(acc[j])) : float(abs(acc[j]));   // exact either way
                const float f = (aj * (1.0f / 16384.0f) + xsj + sa) * (1.0f + 1.0f / 1048576.0f) +
                                (1.0f / 1073741824.0f);
                // f is a positive normal float: f < 2^(biased exponent - 126)
                const int e = int((__float_as_uint(f) >> 23) & 255u) - 126;
                if (col < G.N && ex > SPL_EXP_NONE / 2) Emax = max(Emax, ea + ex + e);
            }
            if (row_ok && Emax > SPL_EXP_NONE) atomicMax(dst + v * G.per, Emax);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(EST_TMEM_COLS));
    }
}

// Self-test of the timeout path: one thread waits on an mbarrier that nothing arrives
// at, with the bounded wait of the slice GEMM.
__global__ void k_wait_selftest(int* status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (mbar_wait_limit(&bar, 0, limit, &abort, status)) atomicExch(status, 1);
    }
}

// ----------------------------------------------------------------------------------
// stage-2 sums -> FP64 wave function

constexpr int FIN_CHUNK = 2048;   // output entries per CTA of the finalize pass
__global__ void k_finalize(const SBlock* __restrict__ blocks, const SPart* __restrict__ parts,
                           const int64_t* __restrict__ s2, const int32_t* __restrict__ op_ex,
                           const int32_t* __restrict__ ap_ex, double* __restrict__ y, int64_t dim) {
    const SBlock B = blocks[blockIdx.x];
    const int v = blockIdx.y;
    const int e1 = min(B.rows * B.cols, int(blockIdx.z + 1) * FIN_CHUNK);
    for (int e = int(blockIdx.z) * FIN_CHUNK + threadIdx.x; e < e1; e += blockDim.x) {
        const int i = e / B.cols, j = e % B.cols;
        double sum = 0.0;
        for (int p = B.p0; p < B.p0 + B.np; ++p) {
            const SPart P = parts[p];
            const int ri = v * P.rstack + i, cj = v * P.cstack + j;
            const long long F = s2[P.acc_off + int64_t(ri) * P.ld + cj];
            if (F == 0) continue;
            const int er = (P.er_buf ? ap_ex : op_ex)[P.er_off + ri];
            const int ec = (P.ec_buf ? ap_ex : op_ex)[P.ec_off + cj];
            sum += scalbn(static_cast<double>(F), er + ec - P.e_off);
        }
        y[int64_t(v) * dim + B.y_off + e] = sum;
    }
}

}  // namespace

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// s = 47 - ceil(log2 K): |F| <= K 2^14 2^s (1 + 2^-6) < 2^62 for any contraction length
// (s >= 24 because K <= 2^23, so the shifts s - 8, s - 16, s - 24 of the epilogue are valid).
int32_t fshift_for(int64_t K) {
    int c = 0;
    while ((int64_t(1) << c) < K) ++c;
    return 47 - c;
}

// ----------------------------------------------------------------------------------
// host side

namespace {
int64_t job_tile_elems(int rows_tile) { return int64_t(SPL_S) * rows_tile * SPL_TK; }
}  // namespace

// Host-side bounds proof of a split plan: every slicer read and write, bulk-copy source
// range, exponent and bound-table access, stage-1 epilogue store, stage-2 sum and
// finalize read lies inside its buffer.
int validate_split_plan(const Plan& P, const SplitHost& H, std::string* err) {
    auto bad = [&](const char* what) {
        *err = std::string("split plan out of bounds: ") + what;
        return DMRG_ERR_BOUNDS;
    };
    const int64_t n_jobs = int64_t(H.jobs.size());
    auto job_ok = [&](int64_t j) { return j >= 0 && j < n_jobs; };
    for (const SJob& J : H.jobs) {
        if (J.rows_tile != SPL_TM && J.rows_tile != SPL_TN) return bad("job tile height");
        const int64_t tiles = int64_t(J.npad / J.rows_tile) * J.kt * job_tile_elems(J.rows_tile);
        const int64_t sl = J.out_buf ? H.ap_sl_vs : H.op_sl;
        const int64_t ex = J.out_buf ? H.ap_ex_vs : H.op_ex;
        if (J.npad % J.rows_tile || J.npad < J.nvalid || J.nvalid < 0 || int64_t(J.kt) * SPL_TK < J.K || J.K < 0)
            return bad("job shape");
        if (J.out_tiles < 0 || J.out_tiles % 8 || J.out_tiles + tiles > sl) return bad("slice tiles");
        if (J.out_exp < 0 || J.out_exp + J.npad > ex) return bad("exponents");
        if (J.top_sums && (J.out_buf || J.nseg != 1)) return bad("row sums");
        if (J.out_buf) continue;
        int64_t K = 0;
        for (int s = J.seg0; s < J.seg0 + J.nseg; ++s) {
            if (s < 0 || s >= int32_t(H.segs.size())) return bad("segment index");
            const SSeg& g = H.segs[s];
            if (g.kbase != K || g.kc < 1 || g.kcp < g.kc || g.nt < 1 || g.vper < 1) return bad("segment shape");
            if (J.top_sums && g.nt != 1) return bad("row-sum segment");
            K += int64_t(g.kcp) * g.nt;
            if (J.nvalid == 0) continue;
            const int ngrp = (J.nvalid - 1) / g.vper, rmax = std::min(J.nvalid, g.vper) - 1;
            const int64_t last = g.off + (g.nt - 1) * g.ts + ngrp * g.vgs + int64_t(rmax) * g.vs + int64_t(g.kc - 1) * g.ks;
            if (g.off < 0 || g.ts < 0 || g.vgs < 0 || g.vs < 0 || g.ks < 0 || last >= P.ops_len)
                return bad("slice source");
        }
        if (K != J.K) return bad("job K");
    }
    for (const SXJob& X : H.xjobs) {
        if (!job_ok(X.job)) return bad("psi job index");
        const SJob& J = H.jobs[size_t(X.job)];
        if (!J.out_buf || J.rows_tile != SPL_TN || X.cp % SPL_KPAD || X.cp < X.nk || X.nk < 1 ||
            J.nvalid != H.nv * X.cp || J.K != X.K || X.K < 1)
            return bad("psi job shape");
        const int64_t last = int64_t(H.nv - 1) * P.dim + X.off + int64_t(X.K - 1) * X.ks + int64_t(X.nk - 1) * X.vs;
        if (X.off < 0 || X.ks < 0 || X.vs < 0 || last >= P.dim * H.nv) return bad("psi source");
    }
    if (H.ap_ex_mid0 < 0 || H.ap_ex_mid0 > H.ap_ex_mid1 || H.ap_ex_mid1 > H.ap_ex_vs) return bad("bound range");
    // per-apply jobs by (first slice entry, output chunk); within a chunk no two share one
    std::map<std::pair<int64_t, int32_t>, int32_t> mid_jobs;
    for (int32_t j = 0; j < int32_t(H.jobs.size()); ++j) {
        const SJob& J = H.jobs[size_t(j)];
        if (J.out_buf && J.npad > 0 && !mid_jobs.emplace(std::make_pair(J.out_tiles, J.chunk), j).second)
            return bad("two per-apply jobs share their slices");
    }
    auto check_work = [&](const std::vector<SWork>& w) -> const char* {
        for (const SWork& x : w) {
            if (x.gemm < 0 || x.gemm >= int32_t(H.gemms.size())) return "work gemm index";
            const SGemm& G = H.gemms[size_t(x.gemm)];
            if (x.k0 < 0 || x.k1 > G.kt || x.k0 >= x.k1) return "work K range";
            if (cdiv(x.k1 - x.k0, SPL_DRAIN_KT) > SPL_MAX_DRAINS) return "work drains";   // epilogue sum bound
            const int64_t lsz = G.l_buf ? H.ap_sl_vs : H.op_sl, rsz = G.r_buf ? H.ap_sl_vs : H.op_sl;
            const int64_t lend = G.l_tiles + (int64_t(x.mtile) * G.kt + x.k1) * (SPL_S * SPL_LT);
            const int64_t rend = G.r_tiles + (int64_t(x.ntile) * G.kt + x.k1) * (SPL_S * SPL_RT);
            if (G.l_tiles < 0 || G.r_tiles < 0 || G.l_tiles % 8 || G.r_tiles % 8 || lend > lsz || rend > rsz)
                return "work operand tiles";
            if (x.mtile < 0 || x.ntile < 0 || int64_t(x.mtile) * SPL_TM >= G.M || int64_t(x.ntile) * SPL_TN >= G.N)
                return "work output tile";
            if (G.kind == 1) {
                const int64_t dend = G.d_off + int64_t(G.M - 1) * G.ldd + G.N;
                if (G.d_off < 0 || G.ldd < G.N || dend > H.s2_vs) return "stage-2 sums";
                // its intermediate operand: a job of the GEMM's own output chunk
                if (G.l_buf + G.r_buf != 1) return "stage-2 operands";
                const int64_t mid = G.l_buf ? G.l_tiles : G.r_tiles;
                if (mid < H.ap_sl_mid0 || !mid_jobs.count({mid, G.chunk})) return "stage-2 intermediate";
                continue;
            }
            // stage-1 epilogue: row r = t*per + i, column v*cp + k -> vector v*per + i,
            // K = kbase + t*cp + k of the destination job (written in groups of 8 K)
            if (G.per < 1 || G.cp < 1 || G.cp % SPL_KPAD || G.kbase % SPL_KPAD || G.M % G.per || G.N % G.cp)
                return "stage-1 shape";
            const int64_t nt = G.M / G.per, nvv = G.N / G.cp;
            if (nvv != H.nv) return "stage-1 vectors";
            if (G.r_buf != 1 || G.l_buf != 0 || G.r_tiles >= H.ap_sl_mid0) return "stage-1 operands";
            bool dst_ok = false;
            const auto it = mid_jobs.find({G.d_off, G.chunk});
            if (it != mid_jobs.end()) {
                const SJob& J = H.jobs[size_t(it->second)];
                dst_ok = J.out_exp == G.dst_exp && J.rows_tile == G.dst_rows_tile && J.kt == G.dst_kt &&
                         int64_t(H.nv) * G.per <= J.nvalid && G.kbase + nt * G.cp <= J.K;
            }
            if (!dst_ok) return "stage-1 destination";
            if (G.er_off < 0 || G.er_off + G.M > H.op_ex || G.ec_off < 0 || G.ec_off + G.N > H.ap_ex_vs) return "stage-1 exponents";
            // the bounds the stage-1 epilogue reads and the estimate pass raises
            if (G.dst_exp < H.ap_ex_mid0 || G.dst_exp + int64_t(H.nv) * G.per > H.ap_ex_mid1) return "stage-1 bounds";
        }
        return nullptr;
    };
    // output chunks: intermediates of one chunk are disjoint and above the psi slices
    // (which no chunk reuses); every work range holds the items of its chunk only
    if (H.n_chunks < 1 || H.ap_sl_mid0 < 0 || H.ap_sl_mid0 > H.ap_sl_vs) return bad("output chunks");
    for (const SGemm& G : H.gemms)
        if (G.chunk < 0 || G.chunk >= H.n_chunks) return bad("gemm chunk");
    {
        std::vector<std::array<int64_t, 3>> mids;
        for (const SJob& J : H.jobs) {
            if (!J.out_buf) continue;
            const int64_t end = J.out_tiles + int64_t(J.npad / J.rows_tile) * J.kt * job_tile_elems(J.rows_tile);
            if (J.out_tiles < H.ap_sl_mid0) {
                if (end > H.ap_sl_mid0) return bad("psi slices reach the intermediates");
                continue;
            }
            if (J.chunk < 0 || J.chunk >= H.n_chunks) return bad("job chunk");
            mids.push_back({J.chunk, J.out_tiles, end});
        }
        std::sort(mids.begin(), mids.end());
        for (size_t i = 1; i < mids.size(); ++i)
            if (mids[i][0] == mids[i - 1][0] && mids[i][1] < mids[i - 1][2]) return bad("intermediates of a chunk overlap");
    }
    auto check_ranges = [&](const std::vector<SWork>& w, const std::vector<int32_t>& cw,
                            const std::vector<std::pair<int32_t, int32_t>>& R, const std::vector<int32_t>& cr) {
        if (cw.size() != size_t(H.n_chunks) + 1 || cr.size() != cw.size() || cw[0] != 0 || cr[0] != 0 ||
            cw.back() != int32_t(w.size()) || cr.back() != int32_t(R.size()))
            return false;
        for (int c = 0; c < H.n_chunks; ++c) {
            if (cw[size_t(c)] > cw[size_t(c) + 1] || cr[size_t(c)] > cr[size_t(c) + 1]) return false;
            for (int32_t i = cw[size_t(c)]; i < cw[size_t(c) + 1]; ++i) {
                const int32_t g = w[size_t(i)].gemm;
                if (g < 0 || g >= int32_t(H.gemms.size()) || H.gemms[size_t(g)].chunk != c) return false;
            }
            for (int32_t r = cr[size_t(c)]; r < cr[size_t(c) + 1]; ++r)
                if (R[size_t(r)].first < cw[size_t(c)] || R[size_t(r)].second > cw[size_t(c) + 1] ||
                    R[size_t(r)].first >= R[size_t(r)].second)
                    return false;
        }
        return true;
    };
    if (!check_ranges(H.w1, H.cw1, H.r1, H.cr1) || !check_ranges(H.w2, H.cw2, H.r2, H.cr2)) return bad("chunk work ranges");
    if (const char* why = check_work(H.w1)) return bad(why);
    if (const char* why = check_work(H.w2)) return bad(why);
    for (const STile& T : H.tiles) {   // the digit pass starts its segment search at T.seg
        if (!job_ok(T.job)) return bad("slice tile job");
        const SJob& J = H.jobs[size_t(T.job)];
        if (J.out_buf || T.vg < 0 || 8 * T.vg >= J.nvalid || 8 * T.vg + 8 > J.npad) return bad("slice tile rows");
        if (T.k0 < 0 || T.k0 >= J.K || T.k0 % SPL_TILE_K) return bad("slice tile K");
        if (T.seg < J.seg0 || T.seg >= J.seg0 + J.nseg || H.segs[size_t(T.seg)].kbase > T.k0) return bad("tile segment");
    }
    for (const SItem& I : H.items) {
        if (I.slab < 0 || I.slab >= int32_t(H.slabs.size())) return bad("slice item");
        const SSlab& Sl = H.slabs[size_t(I.slab)];
        if (I.r0 < 0 || I.nrows <= 0 || I.r0 + I.nrows > Sl.rows) return bad("slice item rows");
        if (!job_ok(Sl.job)) return bad("slice slab job");
        const SJob& J = H.jobs[size_t(Sl.job)];
        if (J.out_buf || Sl.seg < J.seg0 || Sl.seg >= J.seg0 + J.nseg ||
            Sl.rows != int64_t(H.segs[size_t(Sl.seg)].nt) * J.nvalid)
            return bad("slice slab");
    }
    for (const SBlock& B : H.blocks)
        for (int p = B.p0; p < B.p0 + B.np; ++p) {
            if (p < 0 || p >= int32_t(H.parts.size())) return bad("finalize part");
            const SPart& Q = H.parts[size_t(p)];
            const int64_t rmax = int64_t(H.nv - 1) * Q.rstack + B.rows, cmax = int64_t(H.nv - 1) * Q.cstack + B.cols;
            if (Q.ld < cmax || Q.acc_off < 0 || Q.acc_off + (rmax - 1) * Q.ld + cmax > H.s2_vs) return bad("finalize sums");
            if (Q.er_off < 0 || Q.er_off + rmax > (Q.er_buf ? H.ap_ex_vs : H.op_ex)) return bad("finalize row exps");
            if (Q.ec_off < 0 || Q.ec_off + cmax > (Q.ec_buf ? H.ap_ex_vs : H.op_ex)) return bad("finalize col exps");
        }
    return DMRG_OK;
}

void build_split_work(SplitHost& H, const Schedule& S) {
    std::vector<SWork>& w1 = H.w1;
    std::vector<SWork>& w2 = H.w2;
    w1.clear(); w2.clear(); H.r1.clear(); H.r2.clear();
    // stage 1: every output tile over the whole contraction (at most 8192 K)
    for (size_t gi = 0; gi < H.gemms.size(); ++gi) {
        const SGemm& m = H.gemms[gi];
        if (m.kind != 0) continue;
        for (int mt = 0; mt < cdiv(m.M, SPL_TM); ++mt)
            for (int nt = 0; nt < cdiv(m.N, SPL_TN); ++nt) w1.push_back({int32_t(gi), mt, nt, 0, m.kt, 0});
    }
    // stage 2: output tiles x K chunks.  A shape class with no scheduled chunk takes the
    // adaptive one: the longest multiple of the drain length up to SPL_S2_KCHUNK K tiles
    // that leaves >= 4 items per SM.  Scheduled chunks are given in units of 32 K.
    int64_t tile_kt = 0;
    for (const SGemm& m : H.gemms)
        if (m.kind == 1) tile_kt += cdiv(m.M, SPL_TM) * cdiv(m.N, SPL_TN) * int64_t(m.kt);
    int adaptive = SPL_S2_KCHUNK;
    while (adaptive > SPL_DRAIN_KT && tile_kt / adaptive < 4 * 152) adaptive /= 2;
    // K chunk outermost: CTAs that run at the same time share the L tile of an M row
    // across its N tiles and the R tile of an N column across its M tiles (L2 reuse)
    for (size_t gi = 0; gi < H.gemms.size(); ++gi) {
        const SGemm& m = H.gemms[gi];
        if (m.kind != 1) continue;
        const int sc = S.split_kchunk[kclass(int64_t(m.kt) * SPL_TK)];
        const int chunk = sc > 0 ? sc * (32 / SPL_TK) : adaptive;
        for (int k0 = 0; k0 < m.kt; k0 += chunk)
            for (int mt = 0; mt < cdiv(m.M, SPL_TM); ++mt)
                for (int nt = 0; nt < cdiv(m.N, SPL_TN); ++nt)
                    w2.push_back({int32_t(gi), mt, nt, k0, std::min(m.kt, k0 + chunk), 0});
    }
    // output chunk first; then longest items first, or (one launch per GEMM) each GEMM's
    // items contiguous
    auto ck = [&](const SWork& x) { return H.gemms[size_t(x.gemm)].chunk; };
    auto by_cost = [&](const SWork& x, const SWork& y) {
        return ck(x) != ck(y) ? ck(x) < ck(y) : (x.k1 - x.k0) > (y.k1 - y.k0);
    };
    auto by_gemm = [&](const SWork& x, const SWork& y) {
        if (ck(x) != ck(y)) return ck(x) < ck(y);
        return x.gemm != y.gemm ? x.gemm < y.gemm : (x.k1 - x.k0) > (y.k1 - y.k0);
    };
    for (int st = 0; st < 2; ++st) {
        std::vector<SWork>& w = st == 0 ? w1 : w2;
        std::vector<int32_t>& cw = st == 0 ? H.cw1 : H.cw2;
        std::vector<int32_t>& cr = st == 0 ? H.cr1 : H.cr2;
        auto& R = st == 0 ? H.r1 : H.r2;
        std::stable_sort(w.begin(), w.end(), [&](const SWork& x, const SWork& y) {
            return S.per_gemm ? by_gemm(x, y) : by_cost(x, y);
        });
        if (S.per_gemm)
            for (int32_t i = 0; i < int32_t(w.size());) {
                int32_t j = i;
                while (j < int32_t(w.size()) && w[j].gemm == w[i].gemm) ++j;
                R.push_back({i, j});
                i = j;
            }
        cw.assign(size_t(H.n_chunks) + 1, 0);
        cr.assign(size_t(H.n_chunks) + 1, 0);
        size_t i = 0, r = 0;
        for (int c = 0; c < H.n_chunks; ++c) {
            while (i < w.size() && ck(w[i]) == c) ++i;
            while (r < R.size() && ck(w[size_t(R[r].first)]) == c) ++r;
            cw[size_t(c) + 1] = int32_t(i);
            cr[size_t(c) + 1] = int32_t(r);
        }
    }
}

int build_split_plan(const Plan& P, int nv, SplitHost& H, std::string* err, const Schedule& S, int64_t mid_cap) {
    H = SplitHost{};
    H.nv = nv;
    if (mid_cap <= 0) mid_cap = SPL_MID_CAP;
    if (nv < 1 || nv > 64) {
        *err = "nvec out of range";
        return DMRG_ERR_INVALID_ARG;
    }
    if (int64_t(P.groups.size()) > (int64_t(1) << 28) || P.dim * nv > (int64_t(1) << 40)) {
        *err = "too many groups";
        return DMRG_ERR_INVALID_ARG;
    }
    std::vector<SJob>& jobs = H.jobs;
    std::vector<SSeg>& segs = H.segs;
    std::vector<int32_t> op_jobs;
    int64_t op_sl = 0, op_ex = 0, ap_sl = 0, ap_ex = 0, s2 = 0;
    auto add_job = [&](int out_buf, int rows_tile, int64_t nvalid, int64_t K, const std::vector<SSeg>& js) {
        SJob J{};
        J.out_buf = out_buf;
        J.rows_tile = rows_tile;
        J.nvalid = int32_t(nvalid);
        J.npad = int32_t(cdiv(nvalid, rows_tile) * rows_tile);
        J.K = int32_t(K);
        J.kt = int32_t(cdiv(K, SPL_TK));
        J.seg0 = int32_t(segs.size());
        J.nseg = int32_t(js.size());
        int32_t kb = 0;
        for (SSeg g : js) {
            g.kbase = kb;
            kb += g.kcp * g.nt;
            segs.push_back(g);
        }
        int64_t& sl = out_buf ? ap_sl : op_sl;
        int64_t& ex = out_buf ? ap_ex : op_ex;
        J.out_tiles = sl;
        J.out_exp = ex;
        sl += int64_t(J.npad / rows_tile) * J.kt * job_tile_elems(rows_tile);
        ex += J.npad;
        jobs.push_back(J);
        if (!out_buf) op_jobs.push_back(int32_t(jobs.size() - 1));
        return int32_t(jobs.size() - 1);
    };
    // operator run: nt sub-blocks (terms) of kc entries padded to kcp
    auto seg = [](int64_t off, int64_t ts, int64_t vs, int kc, int kcp, int nt) {
        SSeg s{};
        s.off = off; s.ts = ts; s.vs = vs; s.ks = 1; s.kc = kc; s.kcp = kcp; s.nt = nt;
        s.vper = 1 << 30;
        return s;
    };
    for (const Group& G : P.groups) {
        const int64_t kmax = int64_t(std::max({G.a, G.b, G.c, G.d}));
        if (kmax > SPL_MAX_DRAINS * SPL_DRAIN_KT * SPL_TK) {   // one stage-1 item spans the whole contraction
            *err = "split path: a sector dimension above 8192";
            return DMRG_ERR_INVALID_ARG;
        }
    }

    // psi jobs: one per (input block, contraction side), shared by the groups that use it
    std::vector<int32_t> xjob_of(P.blocks.size() * 2, -1);
    auto xjob = [&](int32_t q, int side) {
        int32_t& x = xjob_of[size_t(q) * 2 + size_t(side)];
        if (x >= 0) return x;
        const PsiBlock& B = P.blocks[size_t(q)];
        SXJob X{};
        X.off = B.off;
        if (side == 0) {   // vectors = columns (K over the block's rows)
            X.K = B.rows; X.nk = B.cols; X.ks = B.cols; X.vs = 1;
        } else {           // vectors = rows (K over the block's columns)
            X.K = B.cols; X.nk = B.rows; X.ks = 1; X.vs = B.cols;
        }
        X.cp = kpad(X.nk);
        X.job = add_job(1, SPL_TN, int64_t(nv) * X.cp, X.K, {});
        H.xjobs.push_back(X);
        x = int32_t(H.xjobs.size() - 1);
        return x;
    };

    // every psi job first, so that the exponents of the stage-2 intermediate vectors
    // (reset per apply) form one range after them
    for (const Group& G : P.groups) xjob(G.in_block, G.order);
    H.ap_ex_mid0 = ap_ex;
    H.ap_sl_mid0 = ap_sl;
    // stage 2 next (the stage-1 epilogues need their destination jobs): per output block
    // one GEMM over its A-first groups and one over its B-first groups
    std::vector<int32_t> dst_of(P.groups.size(), -1);
    std::vector<int32_t> kbase_of(P.groups.size(), 0);
    std::vector<std::vector<int32_t>> by_out(P.blocks.size());
    for (int32_t g = 0; g < int32_t(P.groups.size()); ++g) by_out[size_t(P.groups[size_t(g)].out_block)].push_back(g);
    std::vector<SGemm> s2g;
    H.blocks.assign(P.blocks.size(), SBlock{});
    // output chunks: the intermediates of the blocks of one chunk take the apply space
    // from ap_sl_mid0 on; a block that would take a chunk beyond mid_cap bytes opens the
    // next chunk (whose intermediates reuse the space)
    std::vector<int32_t> chunk_of(P.blocks.size(), 0);
    int32_t chunk = 0;
    int64_t mid_end = ap_sl;
    for (size_t o = 0; o < P.blocks.size(); ++o) {
        const PsiBlock& O = P.blocks[o];
        H.blocks[o] = {O.off, O.rows, O.cols, int32_t(H.parts.size()), 0};
        int64_t need = 0;   // this block's intermediate slice entries
        for (int order = 0; order < 2; ++order) {
            int64_t K = 0;
            for (int32_t g : by_out[o]) {
                const Group& G = P.groups[size_t(g)];
                if (G.order == order) K += int64_t(kpad(order == 0 ? G.c : G.b)) * int64_t(G.terms.size());
            }
            if (K == 0) continue;
            const int rt = order == 0 ? SPL_TM : SPL_TN;
            need += cdiv(int64_t(nv) * (order == 0 ? O.rows : O.cols), rt) * cdiv(K, SPL_TK) * job_tile_elems(rt);
        }
        if (ap_sl > H.ap_sl_mid0 && 2 * (ap_sl - H.ap_sl_mid0 + need) > mid_cap) {
            ++chunk;
            ap_sl = H.ap_sl_mid0;
        }
        chunk_of[o] = chunk;
        for (int order = 0; order < 2; ++order) {
            std::vector<SSeg> opseg;
            std::vector<int32_t> gs;
            int64_t K = 0;
            for (int32_t g : by_out[o]) {
                const Group& G = P.groups[size_t(g)];
                if (G.order != order) continue;
                const int n = int(G.terms.size());
                kbase_of[size_t(g)] = int32_t(K);
                if (order == 0) {   // K = (t, k < c): R = B_t rows (output columns)
                    opseg.push_back(seg(G.b_stack, int64_t(G.d) * G.c, G.c, G.c, kpad(G.c), n));
                    K += int64_t(kpad(G.c)) * n;
                } else {            // K = (t, k < b): L = c_t A_t rows (output rows)
                    opseg.push_back(seg(G.a_stack, int64_t(G.a) * G.b, G.b, G.b, kpad(G.b), n));
                    K += int64_t(kpad(G.b)) * n;
                }
                gs.push_back(g);
            }
            if (gs.empty()) continue;
            if (K > SPL_MAX_K || K > INT32_MAX / 2) {
                *err = "stage-2 contraction longer than 2^23";
                return DMRG_ERR_INVALID_ARG;
            }
            // the intermediate side: vectors v*rows + i (A-first, L) or v*cols + j (B-first, R)
            const int32_t ij = order == 0 ? add_job(1, SPL_TM, int64_t(nv) * O.rows, K, {})
                                          : add_job(1, SPL_TN, int64_t(nv) * O.cols, K, {});
            jobs[size_t(ij)].chunk = chunk;
            const int32_t oj = order == 0 ? add_job(0, SPL_TN, O.cols, K, opseg) : add_job(0, SPL_TM, O.rows, K, opseg);
            for (int32_t g : gs) dst_of[size_t(g)] = ij;
            const SJob IJ = jobs[size_t(ij)];
            const SJob OJ = jobs[size_t(oj)];
            SGemm m{};
            m.kind = 1; m.sign = 1; m.chunk = chunk;
            m.M = order == 0 ? nv * O.rows : O.rows;
            m.N = order == 0 ? O.cols : nv * O.cols;
            m.kt = int32_t(cdiv(K, SPL_TK));
            m.l_buf = order == 0 ? 1 : 0; m.r_buf = order == 0 ? 0 : 1;
            m.l_tiles = order == 0 ? IJ.out_tiles : OJ.out_tiles;
            m.r_tiles = order == 0 ? OJ.out_tiles : IJ.out_tiles;
            m.d_off = s2; m.ldd = m.N;
            m.fshift = fshift_for(K);
            SPart part{};
            part.acc_off = s2;
            part.er_off = order == 0 ? IJ.out_exp : OJ.out_exp;
            part.ec_off = order == 0 ? OJ.out_exp : IJ.out_exp;
            part.er_buf = order == 0 ? 1 : 0;
            part.ec_buf = order == 0 ? 0 : 1;
            part.e_off = 14 + m.fshift; part.ld = m.N;
            part.rstack = order == 0 ? O.rows : 0;
            part.cstack = order == 0 ? 0 : O.cols;
            H.parts.push_back(part);
            H.blocks[o].np += 1;
            s2 += int64_t(m.M) * m.N;
            s2g.push_back(m);
        }
        mid_end = std::max(mid_end, ap_sl);
    }
    ap_sl = mid_end;
    H.n_chunks = chunk + 1;
    H.block_chunk = chunk_of;
    H.ap_ex_mid1 = ap_ex;
    // stage 1: one GEMM per group; L = stacked operator rows (c_t A_t or B_t), R = psi
    for (size_t g = 0; g < P.groups.size(); ++g) {
        const Group& G = P.groups[g];
        const int n = int(G.terms.size());
        const int32_t xi = xjob(G.in_block, G.order);
        const SXJob X = H.xjobs[size_t(xi)];
        const SJob XJ = jobs[size_t(X.job)];   // copies: add_job below may reallocate
        const int per = G.order == 0 ? G.a : G.d;
        int32_t lj;
        if (G.order == 0)   // X_g = A_stack (n a x b) * [x_q^(v)] (b x nv c)
            lj = add_job(0, SPL_TM, int64_t(n) * G.a, G.b, {seg(G.a_stack, 0, G.b, G.b, G.b, 1)});
        else                // Z_g^T = B_stack (n d x c) * [x_q^(v)T] (c x nv b)
            lj = add_job(0, SPL_TM, int64_t(n) * G.d, G.c, {seg(G.b_stack, 0, G.c, G.c, G.c, 1)});
        jobs[size_t(lj)].top_sums = 1;
        const SJob LJ = jobs[size_t(lj)];
        if (dst_of[g] < 0) {
            *err = "split plan: a group without its output block";
            return DMRG_ERR_INVALID_ARG;
        }
        const SJob DJ = jobs[size_t(dst_of[g])];
        SGemm m{};
        m.kind = 0;
        m.chunk = chunk_of[size_t(G.out_block)];
        m.M = n * per; m.N = nv * X.cp; m.kt = LJ.kt;
        m.l_buf = 0; m.r_buf = 1; m.l_tiles = LJ.out_tiles; m.r_tiles = XJ.out_tiles;
        m.sign = G.sign < 0 ? -1 : 1;
        m.fshift = fshift_for(X.K);
        m.per = per; m.cp = X.cp; m.kbase = kbase_of[g];
        m.d_off = DJ.out_tiles; m.dst_rows_tile = DJ.rows_tile; m.dst_kt = DJ.kt; m.dst_exp = int32_t(DJ.out_exp);
        m.er_off = int32_t(LJ.out_exp); m.ec_off = int32_t(XJ.out_exp);
        H.gemms.push_back(m);
    }
    for (const SGemm& m : s2g) H.gemms.push_back(m);
    if (op_ex > INT32_MAX || ap_ex > INT32_MAX) {
        *err = "split plan: exponent tables beyond 2^31 entries";
        return DMRG_ERR_INVALID_ARG;
    }
    build_split_work(H, S);
    // operator slicing work: exponent items (rows of every segment) and digit tiles
    for (int32_t j : op_jobs) {
        const SJob& J = jobs[size_t(j)];
        for (int sg = J.seg0; sg < J.seg0 + J.nseg; ++sg) {
            const int64_t rows = int64_t(segs[size_t(sg)].nt) * J.nvalid;
            if (rows == 0) continue;
            const int32_t sl = int32_t(H.slabs.size());
            H.slabs.push_back({rows, j, sg, segs[size_t(sg)].kbase, 0});
            for (int64_t r0 = 0; r0 < rows; r0 += SPL_ROWS_PER_ITEM)
                H.items.push_back({r0, sl, int32_t(std::min<int64_t>(SPL_ROWS_PER_ITEM, rows - r0))});
        }
        for (int vg = 0; 8 * vg < J.nvalid; ++vg) {
            int32_t sg = J.seg0;
            for (int k0 = 0; k0 < J.K; k0 += SPL_TILE_K) {
                while (sg < J.seg0 + J.nseg - 1 && k0 >= segs[size_t(sg)].kbase + segs[size_t(sg)].kcp * segs[size_t(sg)].nt)
                    ++sg;
                H.tiles.push_back({j, vg, k0, sg});
            }
        }
    }
    H.op_sl = op_sl;
    H.op_ex = op_ex + 1;
    H.ap_sl_vs = cdiv(ap_sl, 64) * 64;
    H.ap_ex_vs = cdiv(ap_ex, 4) * 4 + 4;
    H.s2_vs = s2;
    return validate_split_plan(P, H, err);
}

int Handle::init_split(const double* op_data) {
    const Plan& P = plan;
    SplitState* S = new SplitState();
    split = S;
    std::string err;
    // one plan per number of stacked vectors; operator slices are identical in all of them
    std::vector<SplitHost> hosts;
    std::vector<SWindow> win;
    int rc0 = build_split_hosts(P, max_nvec, split_mid_cap, hosts, win, &mem, &err);
    if (rc0 != DMRG_OK) return fail(rc0, err);
    int64_t ap_sl = 0, ap_ex = 0, s2 = 0;
    for (const SplitHost& H : hosts) {
        ap_sl = std::max(ap_sl, H.ap_sl_vs);
        ap_ex = std::max(ap_ex, H.ap_ex_vs);
        s2 = std::max(s2, H.s2_vs);
    }
    const int64_t op_sl = hosts[0].op_sl, op_ex = hosts[0].op_ex;
    auto al = [&](void** p, size_t bytes, const char* w) {
        *p = nullptr;
        if (bytes == 0) return DMRG_OK;
        cudaError_t e = cudaMalloc(p, bytes);
        return e == cudaSuccess ? DMRG_OK : cuda_fail(e, w);
    };
    auto up = [&](void** p, const void* src, size_t bytes, const char* w) {
        int rc = al(p, bytes, w);
        if (rc || bytes == 0) return rc;
        cudaError_t e = cudaMemcpy(*p, src, bytes, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? DMRG_OK : cuda_fail(e, w);
    };
    int rc;
    if ((rc = al((void**)&S->op_sl, sizeof(uint16_t) * op_sl, "operator slices")) ||
        (rc = al((void**)&S->op_ex, sizeof(int32_t) * op_ex, "operator exponents")) ||
        (rc = al((void**)&S->srow, sizeof(int32_t) * op_ex, "operator top-digit sums")) ||
        (rc = al((void**)&S->ap_sl, sizeof(uint16_t) * ap_sl, "apply slices")) ||
        (rc = al((void**)&S->ap_ex, sizeof(int32_t) * ap_ex, "apply exponents")) ||
        (rc = al((void**)&S->xs, sizeof(float) * ap_ex, "psi sums")) ||
        (rc = al((void**)&S->s2, sizeof(int64_t) * s2, "stage-2 int64 sums")) ||
        (rc = al((void**)&S->status, sizeof(int32_t), "status")))
        return rc;
    S->plans.resize(size_t(max_nvec));
    for (int nv = 1; nv <= max_nvec; ++nv) {
        const SplitHost& H = hosts[size_t(nv - 1)];
        SplitDevPlan& D = S->plans[size_t(nv - 1)];
        if ((rc = up((void**)&D.gemms, H.gemms.data(), sizeof(SGemm) * H.gemms.size(), "split gemms")) ||
            (rc = up((void**)&D.work1, H.w1.data(), sizeof(SWork) * H.w1.size(), "split work")) ||
            (rc = up((void**)&D.work2, H.w2.data(), sizeof(SWork) * H.w2.size(), "split work")) ||
            (rc = up((void**)&D.segs, H.segs.data(), sizeof(SSeg) * H.segs.size(), "slice segments")) ||
            (rc = up((void**)&D.jobs, H.jobs.data(), sizeof(SJob) * H.jobs.size(), "slice jobs")) ||
            (rc = up((void**)&D.xjobs, H.xjobs.data(), sizeof(SXJob) * H.xjobs.size(), "psi jobs")) ||
            (rc = up((void**)&D.slabs, H.slabs.data(), sizeof(SSlab) * H.slabs.size(), "slice slabs")) ||
            (rc = up((void**)&D.items, H.items.data(), sizeof(SItem) * H.items.size(), "slice items")) ||
            (rc = up((void**)&D.tiles, H.tiles.data(), sizeof(STile) * H.tiles.size(), "slice tiles")) ||
            (rc = up((void**)&D.blocks, H.blocks.data(), sizeof(SBlock) * H.blocks.size(), "output blocks")) ||
            (rc = up((void**)&D.parts, H.parts.data(), sizeof(SPart) * H.parts.size(), "output parts")))
            return rc;
        D.n_work1 = int64_t(H.w1.size());
        D.n_work2 = int64_t(H.w2.size());
        D.r1 = H.r1;
        D.r2 = H.r2;
        D.n_chunks = H.n_chunks;
        D.cw1 = H.cw1; D.cw2 = H.cw2; D.cr1 = H.cr1; D.cr2 = H.cr2;
        D.n_blocks = int64_t(H.blocks.size());
        D.n_xjobs = int64_t(H.xjobs.size());
        D.n_items = int64_t(H.items.size());
        D.n_tiles = int64_t(H.tiles.size());
        D.s2_len = H.s2_vs;
        D.mid0 = H.ap_ex_mid0;
        D.mid1 = H.ap_ex_mid1;
        // algorithmic DRAM bytes: slice tiles read once (12 B per entry), stage-1 digit
        // slices written (12 B per entry), stage-2 int64 sums added (8 B per entry); the
        // psi pass reads psi and writes its slices
        const size_t nc = size_t(H.n_chunks);
        D.s1_bytes.assign(nc, 0.0); D.s2_bytes.assign(nc, 0.0); D.e_bytes.assign(nc, 0.0);
        D.s1_flops.assign(nc, 0.0); D.s2_flops.assign(nc, 0.0);
        for (const SGemm& m : H.gemms) {
            const double rd = 12.0 * (double(m.M) + m.N) * m.kt * SPL_TK;
            const size_t c = size_t(m.chunk);
            if (m.kind == 0) {
                D.s1_bytes[c] += rd + 12.0 * double(m.M) * m.N;
                D.e_bytes[c] += rd / SPL_S;   // the estimate pass reads slice 0 only
            } else {
                D.s2_bytes[c] += rd + 8.0 * double(m.M) * m.N;
            }
        }
        for (const Group& G : P.groups) {   // the planned order's flops, as for the handle totals
            const size_t c = size_t(H.block_chunk[size_t(G.out_block)]);
            const double n = double(G.terms.size()), a = G.a, b = G.b, cc = G.c, d = G.d;
            D.s1_flops[c] += G.order == 0 ? n * 2 * a * b * cc : n * 2 * b * cc * d;
            D.s2_flops[c] += G.order == 0 ? n * 2 * a * cc * d : n * 2 * a * b * d;
        }
        for (const SXJob& X : H.xjobs) {
            D.x_bytes += double(nv) * (8.0 * X.K * X.nk + 12.0 * X.K * X.cp);
            D.xchunks = std::max<int32_t>(D.xchunks, int32_t(cdiv(X.cp, XP_VCH)));
        }
        for (const SBlock& B : H.blocks)
            D.fin_chunks = std::max<int32_t>(D.fin_chunks, int32_t(cdiv(int64_t(B.rows) * B.cols, FIN_CHUNK)));
    }
    for (const SplitHost& H : hosts) {
        S->cap_w1.push_back(H.w1.size());
        S->cap_w2.push_back(H.w2.size());
    }
    S->hosts = std::move(hosts);
    cudaError_t e = cudaMemset(S->status, 0, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "status");
    e = cudaFuncSetAttribute(k_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(UmmaSmem)));
    if (e != cudaSuccess) return cuda_fail(e, "umma shared memory");
    e = cudaFuncSetAttribute(k_uest, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(EstSmem)));
    if (e != cudaSuccess) return cuda_fail(e, "estimate shared memory");
    S->kid_x = prof.kernel_id("split_xprep");
    S->kid_e = prof.kernel_id("split_estimate");
    S->kid_s1 = prof.kernel_id("umma_slices/stage1");
    S->kid_s2 = prof.kernel_id("umma_slices/stage2");
    S->kid_fin = prof.kernel_id("split_finalize");
    // slice buffers start at zero (padding is never written again), exponents at "none"
    if (op_sl > 0 && (e = cudaMemset(S->op_sl, 0, sizeof(uint16_t) * op_sl)) != cudaSuccess) return cuda_fail(e, "zero slices");
    if (ap_sl > 0 && (e = cudaMemset(S->ap_sl, 0, sizeof(uint16_t) * ap_sl)) != cudaSuccess) return cuda_fail(e, "zero slices");
    if ((e = cudaMemset(S->op_ex, 0xC0, sizeof(int32_t) * op_ex)) != cudaSuccess) return cuda_fail(e, "exponents");
    if ((e = cudaMemset(S->srow, 0, sizeof(int32_t) * op_ex)) != cudaSuccess) return cuda_fail(e, "top-digit sums");
    if (ap_ex > 0 && (e = cudaMemset(S->ap_ex, 0xE0, sizeof(int32_t) * ap_ex)) != cudaSuccess) return cuda_fail(e, "exponents");
    // operator slices and the diagonal, once (from the first plan; every plan has the same
    // operator jobs): the FP64 layout is scaled on the host through a bounded buffer and
    // staged on the device one window at a time
    if ((e = cudaMalloc(reinterpret_cast<void**>(&d_diag), sizeof(double) * std::max<int64_t>(P.dim, 1))) !=
        cudaSuccess)
        return cuda_fail(e, "diagonal");
    if (P.dim > 0 && (e = cudaMemset(d_diag, 0, sizeof(double) * P.dim)) != cudaSuccess) return cuda_fail(e, "zero diagonal");
    if (win.empty()) return DMRG_OK;
    const SplitDevPlan& D0 = S->plans[0];
    int64_t wmax = 0;
    for (const SWindow& w : win) wmax = std::max(wmax, w.hi - w.lo);
    double* d_stage = nullptr;
    if ((rc = al((void**)&d_stage, sizeof(double) * wmax, "operator staging")) != DMRG_OK) return rc;
    const size_t cap = size_t(std::min<int64_t>(wmax, int64_t(1) << 25));   // 256 MB host buffer
    std::vector<double> hbuf(cap);
    size_t wi = 0, fill = 0;
    int64_t pos = 0, fill_lo = 0;   // layout position of the next entry, of hbuf[0]
    cudaError_t ce = cudaSuccess;
    auto flush = [&]() {
        if (fill > 0 && ce == cudaSuccess)
            ce = cudaMemcpy(d_stage + (fill_lo - win[wi].lo), hbuf.data(), sizeof(double) * fill,
                            cudaMemcpyHostToDevice);
        fill_lo += int64_t(fill);
        fill = 0;
    };
    auto slice_window = [&]() {
        const SWindow& w = win[wi];
        if (ce != cudaSuccess) return;
        if (w.item1 > w.item0) {
            SliceArgs sa{D0.items + w.item0, w.item1 - w.item0, D0.slabs, D0.jobs, D0.segs, d_stage, w.lo, S->op_ex};
            k_slice_max<<<unsigned(std::min<int64_t>(w.item1 - w.item0, int64_t(n_sm) * 16)), 256>>>(sa);
        }
        if (w.tile1 > w.tile0) {
            TileArgs ta{D0.tiles + w.tile0, w.tile1 - w.tile0, D0.jobs, D0.segs, d_stage, w.lo,
                        S->op_sl, S->op_ex, S->srow};
            k_slice_digits<<<unsigned(std::min<int64_t>(cdiv(w.tile1 - w.tile0, DIG_WARPS), int64_t(n_sm) * 16)),
                             32 * DIG_WARPS>>>(ta);
        }
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = launch_diag(d_stage, w.lo, w.lo, w.hi, d_diag, nullptr);
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();   // the staging buffer is reused
    };
    stream_ops(P, op_data, [&](const double* src, int64_t n, double scale) {
        while (n > 0 && wi < win.size()) {
            const int64_t k = std::min({n, int64_t(cap - fill), win[wi].hi - pos});
            for (int64_t i = 0; i < k; ++i) hbuf[fill + size_t(i)] = scale * src[i];
            fill += size_t(k);
            pos += k;
            src += k;
            n -= k;
            if (fill == cap) flush();
            if (pos == win[wi].hi) {
                flush();
                slice_window();
                ++wi;
            }
        }
    });
    cudaFree(d_stage);
    if (ce != cudaSuccess) return cuda_fail(ce, "operator slicing");
    if (wi != win.size() || pos != P.ops_len) return fail(DMRG_ERR_BOUNDS, "operator layout size");
    return DMRG_OK;
}

// One split H_eff*psi for nvec stacked vectors: psi pass (exponents, bounds, slices;
// stage-2 sums cleared); per output chunk the estimate pass, the stage-1 slice GEMM (its
// epilogue writes the chunk's stage-2 slices) and the stage-2 slice GEMM (int64 sums);
// finalize.
int Handle::apply_split(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    SplitState* S = split;
    const SplitDevPlan& D = S->plans[size_t(nvec - 1)];
    Profiler::Pending pe;
    cudaError_t e;
    // one stage of one chunk: a single persistent launch over the chunk's work items
    // [w0, w1), or (per_gemm) one launch per GEMM over its ranges rg[r0, r1)
    auto gemm = [&](const SWork* w, int32_t w0, int32_t w1, const std::vector<std::pair<int32_t, int32_t>>& rg,
                    int32_t r0, int32_t r1, int kid, double flops, double bytes) {
        if (w1 <= w0) return cudaSuccess;
        auto launch = [&](const SWork* wp, int64_t n) {
            UmmaArgs ua{wp, n, D.gemms, S->op_sl, S->ap_sl, S->s2, S->op_ex, S->ap_ex, S->status};
            k_umma<<<unsigned(std::min<int64_t>(n, n_sm)), UM_THREADS, sizeof(UmmaSmem), st>>>(ua);
            return cudaGetLastError();
        };
        prof.begin(kid, st, flops, bytes, &pe);
        cudaError_t le = cudaSuccess;
        if (!sched.per_gemm)
            le = launch(w + w0, w1 - w0);
        else
            for (int32_t r = r0; r < r1 && le == cudaSuccess; ++r)
                le = launch(w + rg[size_t(r)].first, rg[size_t(r)].second - rg[size_t(r)].first);
        prof.end(pe, st);
        return le;
    };
    if (D.n_xjobs > 0) {
        XArgs xa{D.xjobs, D.jobs, x, plan.dim, S->ap_sl, S->ap_ex, S->xs, S->s2, D.s2_len, D.mid0, D.mid1, D.xchunks};
        prof.begin(S->kid_x, st, 0.0, D.x_bytes, &pe);
        k_xprep<<<dim3(unsigned(D.n_xjobs * D.xchunks), unsigned(nvec)), 256, 0, st>>>(xa);
        prof.end(pe, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "psi slices");
    }
    for (int c = 0; c < D.n_chunks; ++c) {
        const int32_t a0 = D.cw1[size_t(c)], a1 = D.cw1[size_t(c) + 1];
        if (a1 > a0) {   // the stage-2 vector bounds of the chunk, over its stage-1 work
            EstArgs ea{D.work1 + a0, a1 - a0, D.gemms, S->op_sl, S->ap_sl, S->op_ex, S->ap_ex, S->srow, S->xs,
                       S->status};
            prof.begin(S->kid_e, st, 0.0, D.e_bytes[size_t(c)], &pe);
            k_uest<<<unsigned(std::min<int64_t>(a1 - a0, n_sm)), UM_THREADS, sizeof(EstSmem), st>>>(ea);
            prof.end(pe, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "estimate pass");
        }
        if ((e = gemm(D.work1, a0, a1, D.r1, D.cr1[size_t(c)], D.cr1[size_t(c) + 1], S->kid_s1,
                      D.s1_flops[size_t(c)] * nvec, D.s1_bytes[size_t(c)])) != cudaSuccess)
            return cuda_fail(e, "stage-1 slice gemm");
        if ((e = gemm(D.work2, D.cw2[size_t(c)], D.cw2[size_t(c) + 1], D.r2, D.cr2[size_t(c)], D.cr2[size_t(c) + 1],
                      S->kid_s2, D.s2_flops[size_t(c)] * nvec, D.s2_bytes[size_t(c)])) != cudaSuccess)
            return cuda_fail(e, "stage-2 slice gemm");
    }
    if (D.n_blocks > 0) {
        prof.begin(S->kid_fin, st, 0.0, 0.0, &pe);
        k_finalize<<<dim3(unsigned(D.n_blocks), unsigned(nvec), unsigned(D.fin_chunks)), 256, 0, st>>>(D.blocks, D.parts, S->s2, S->op_ex,
                                                                              S->ap_ex, y, plan.dim);
        prof.end(pe, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "finalize");
    }
    return DMRG_OK;
}

int Handle::check_status() {
    if (!split) return DMRG_OK;
    int32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, split->status, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read status");
    if (v != 0) {
        cudaMemset(split->status, 0, sizeof(int32_t));
        return fail(v, "a bounded device wait in the slice GEMM timed out");
    }
    return DMRG_OK;
}

}  // namespace dmrg

extern "C" int dmrg_selftest_wait_timeout(int64_t wait_cycles) {
    using namespace dmrg;
    if (wait_cycles < 1 || wait_cycles > (int64_t(1) << 34)) return fail(DMRG_ERR_INVALID_ARG, "wait_cycles range");
    int* st = nullptr;
    cudaError_t e = cudaMalloc(&st, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "self-test status");
    int v = 0;
    e = cudaMemset(st, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(st, static_cast<long long>(wait_cycles));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(st);
    if (e != cudaSuccess) return cuda_fail(e, "self-test");
    if (v == DMRG_ERR_DEVICE_TIMEOUT) return fail(DMRG_ERR_DEVICE_TIMEOUT, "bounded wait ran out (self-test)");
    return v == 1 ? DMRG_OK : fail(DMRG_ERR_CUDA, "self-test status not written");
}

namespace dmrg {

// New work lists for schedule s in every stacked-vector plan, validated like the
// originals, then uploaded (plan-only handles: built and validated on the host).
int Handle::split_set_schedule(const Schedule& s) {
    std::string err;
    if (!split) {
        for (int nv = 1; nv <= max_nvec; ++nv) {
            SplitHost H;
            const int rc = build_split_plan(plan, nv, H, &err, s, split_mid_cap);
            if (rc != DMRG_OK) return fail(rc, err);
        }
        return DMRG_OK;
    }
    SplitState* S = split;
    for (int nv = 1; nv <= max_nvec; ++nv) {
        SplitHost& H = S->hosts[size_t(nv - 1)];
        SplitDevPlan& D = S->plans[size_t(nv - 1)];
        build_split_work(H, s);
        int rc = validate_split_plan(plan, H, &err);
        if (rc != DMRG_OK) return fail(rc, err);
        auto put = [&](const std::vector<SWork>& w, SWork** d, size_t* cap) {
            if (w.size() > *cap) {
                if (*d) cudaFree(*d);
                *d = nullptr;
                *cap = 0;
                cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), sizeof(SWork) * w.size());
                if (e != cudaSuccess) return cuda_fail(e, "split work");
                *cap = w.size();
            }
            if (w.empty()) return int(DMRG_OK);
            cudaError_t e = cudaMemcpy(*d, w.data(), sizeof(SWork) * w.size(), cudaMemcpyHostToDevice);
            return e == cudaSuccess ? int(DMRG_OK) : cuda_fail(e, "split work");
        };
        if ((rc = put(H.w1, &D.work1, &S->cap_w1[size_t(nv - 1)])) != DMRG_OK) return rc;
        if ((rc = put(H.w2, &D.work2, &S->cap_w2[size_t(nv - 1)])) != DMRG_OK) return rc;
        D.n_work1 = int64_t(H.w1.size());
        D.n_work2 = int64_t(H.w2.size());
        D.r1 = H.r1;
        D.r2 = H.r2;
        D.cw1 = H.cw1; D.cw2 = H.cw2; D.cr1 = H.cr1; D.cr2 = H.cr2;
    }
    return DMRG_OK;
}

const SplitHost* Handle::split_plan_host(int nv) const {
    if (!split || nv < 1 || nv > int(split->hosts.size())) return nullptr;
    return &split->hosts[size_t(nv - 1)];
}

void Handle::release_split() {
    delete split;
    split = nullptr;
}

}  // namespace dmrg
