// Split-precision (Ozaki) H_eff*psi on the tcgen05 tensor cores (the arithmetic is
// described in split.h).  Kernels:
//   k_slice_max, k_slice_digits
//             FP64 or int64 operand vectors -> 6 BF16 digit slices in the UMMA
//             canonical K-major layout, plus the vectors' exponents (integer ops only
//             for int64 sources).  The nvec vectors of an apply are stacked inside
//             every GEMM (along N in stage 1, along M or N in stage 2).
//   k_umma    warp-specialised slice GEMM: one producer thread streams up to 72 KB
//             stages with cp.async.bulk (the row groups that hold GEMM rows), one
//             thread issues the 42 tcgen05.mma of each K tile into five accumulators
//             (8 TMEM slots: accumulators 2-4 alternate between two), eight epilogue
//             warps drain the exact FP32 sums into int64 every 256 K and store /
//             atomically add.
//   k_finalize  stage-2 int64 sums -> FP64 wave-function blocks.
// Every mbarrier wait is bounded; on timeout the CTA records DMRG_ERR_DEVICE_TIMEOUT in
// the handle's status word, drains its own copies and MMAs and releases TMEM.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "split.h"

namespace dmrg {

constexpr int UM_STAGES = 3;
constexpr int UM_EPI_WARPS = 8;       // two per TMEM lane quarter, each drains 32 of the 64 columns
constexpr int UM_THREADS = 64 + 32 * UM_EPI_WARPS;   // warp 0 producer, warp 1 MMA, the rest epilogue
constexpr int UM_EPI_COLS = SPL_TN / (UM_EPI_WARPS / 4);
constexpr int UM_TMEM_COLS = 512;     // 8 accumulator slots x 64 columns
// TMEM slots: accumulators 0 and 1 have one slot each, 2-4 two each (alternating drain
// chunks), so the epilogue drains a chunk while the MMAs of the next one run; the
// epilogue reads accumulators 0 and 1 first, the only ones the next chunk waits for.
constexpr int UM_SLOTS = 8;
constexpr int UM_SINGLE = 2;          // accumulators 0 .. UM_SINGLE-1 have one slot
__host__ __device__ constexpr int um_slot(int c, int64_t chunk) {
    return c < UM_SINGLE ? c : UM_SINGLE + 2 * (c - UM_SINGLE) + int(chunk & 1);
}
// completions of a slot's barriers before the one of this chunk
__host__ __device__ constexpr uint32_t um_use(int c, int64_t chunk) {
    return uint32_t(c < UM_SINGLE ? chunk : chunk >> 1);
}
static_assert(UM_SINGLE + 2 * (SPL_ACCS - UM_SINGLE) <= UM_SLOTS && UM_SLOTS * SPL_TN <= UM_TMEM_COLS, "TMEM slots");
constexpr uint32_t UM_L_BYTES = SPL_S * SPL_LT * 2;   // 48 KB
constexpr uint32_t UM_R_BYTES = SPL_S * SPL_RT * 2;   // 24 KB
constexpr long long UM_WAIT_CYCLES = 4000000000ll;     // ~2 s at 2 GHz

constexpr int UM_TR_LD = 5;           // row pitch (int64) of an epilogue warp's transpose patch
struct UmmaSmem {
    uint16_t L[UM_STAGES][SPL_S * SPL_LT];
    uint16_t R[UM_STAGES][SPL_S * SPL_RT];
    long long tr[UM_EPI_WARPS][32 * UM_TR_LD];   // 32 rows x 4 columns per pass of the stage-1 store
    uint64_t full[UM_STAGES], empty[UM_STAGES], tfull[UM_SLOTS], tempty[UM_SLOTS], done;
    uint32_t tmem_base;
    volatile int abort;
};

static_assert(sizeof(UmmaSmem) <= 232448, "slice GEMM shared memory exceeds the opt-in limit");
static_assert(UM_EPI_COLS % 4 == 0, "the stage-1 store moves 4 columns per pass");
static_assert(SPL_S2_KCHUNK / SPL_DRAIN_KT <= SPL_MAX_DRAINS, "stage-2 items span too many drains");

// Device descriptors of the split plan for one number of stacked vectors.
struct SplitDevPlan {
    SGemm* gemms = nullptr;
    SWork* work1 = nullptr;
    SWork* work2 = nullptr;
    SSeg* segs = nullptr;
    SJob* jobs = nullptr;
    SSlab* slabs = nullptr;
    SItem* items = nullptr;     // [operator items | x items | intermediate items]
    STile* tiles = nullptr;     // [operator tiles | x tiles | intermediate tiles]
    SBlock* blocks = nullptr;
    SPart* parts = nullptr;
    int64_t n_work1 = 0, n_work2 = 0, n_blocks = 0;
    std::vector<std::pair<int32_t, int32_t>> r1, r2;   // per-GEMM work ranges (per_gemm)
    int64_t it_op0 = 0, it_x0 = 0, it_mid0 = 0, it_end = 0;      // item ranges
    int64_t tl_op0 = 0, tl_x0 = 0, tl_mid0 = 0, tl_end = 0;      // tile ranges
    int64_t ap_ex_len = 0, s2_len = 0;
    double s1_bytes = 0, s2_bytes = 0;                           // algorithmic DRAM bytes
    void release() {
        void* p[] = {gemms, work1, work2, segs, jobs, slabs, items, tiles, blocks, parts};
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

struct SplitState {
    uint16_t* op_sl = nullptr;   // operator slices (shared by every plan)
    int32_t* op_ex = nullptr;
    uint16_t* ap_sl = nullptr;   // per-apply buffers, sized for the largest plan
    int32_t* ap_ex = nullptr;
    int64_t* s1 = nullptr;
    int64_t* s2 = nullptr;
    int32_t* status = nullptr;
    std::vector<SplitDevPlan> plans;   // plans[nv - 1]
    std::vector<SplitHost> hosts;      // their host copies (work lists rebuilt per schedule)
    std::vector<size_t> cap_w1, cap_w2;
    int kid_x = -1, kid_s1 = -1, kid_mid = -1, kid_s2 = -1, kid_fin = -1;
    ~SplitState() {
        for (SplitDevPlan& d : plans) d.release();
        void* p[] = {op_sl, op_ex, ap_sl, ap_ex, s1, s2, status};
        for (void* q : p)
            if (q) cudaFree(q);
    }
};

namespace {

// ----------------------------------------------------------------------------------
// slicing

// Smallest E with |a| < 2^E (INT_MIN for zero).  Subnormals count: |a| = m 2^-1074 with
// m < 2^52, so |a| < 2^(msb(m) + 1 - 1074).
__device__ __forceinline__ int exp_f64(double a) {
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(a));
    const int ex = int((b >> 52) & 0x7FF);
    if (ex != 0) return ex - 1022;          // |a| < 2^(ex-1022)
    const unsigned long long m = b & ((1ull << 52) - 1);
    return m == 0 ? INT_MIN : (64 - __clzll(m)) - 1074;
}

__device__ __forceinline__ int exp_i64(long long F, int eF) {
    if (F == 0) return INT_MIN;
    const unsigned long long u = F < 0 ? static_cast<unsigned long long>(-F) : static_cast<unsigned long long>(F);
    return (64 - __clzll(u)) + eF;          // |F 2^eF| < 2^(msb+1+eF)
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

// value = F 2^eF; R = round(|F| 2^(eF + 47 - E)).
__device__ __forceinline__ void digits_i64(long long F, int eF, int E, int (&d)[SPL_S]) {
    unsigned long long u = F < 0 ? static_cast<unsigned long long>(-F) : static_cast<unsigned long long>(F);
    const int sh = E - eF - 47;
    unsigned long long R;
    if (sh > 0) R = sh >= 63 ? 0ull : (u + (1ull << (sh - 1))) >> sh;
    else R = u << (-sh);
    balanced_digits(R, F < 0, d);
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

// Position of (vector v, K index K) inside a job's tile array (bf16 elements), slice s.
__device__ __forceinline__ int64_t tile_pos(const SJob& J, int v, int K, int s) {
    const int sh = J.rows_tile == SPL_TM ? 7 : 6;   // rows_tile is 128 (L) or 64 (R)
    const int vt = v >> sh, vr = v & (J.rows_tile - 1), kt = K / SPL_TK, kr = K % SPL_TK;
    const int64_t tile = (int64_t(vt) * J.kt + kt) * SPL_S + s;
    return J.out_tiles + tile * (int64_t(J.rows_tile) * SPL_TK) + ((vr >> 3) * 4 + (kr >> 3)) * 64 + (vr & 7) * 8 +
           (kr & 7);
}

struct SliceArgs {
    const SItem* items;
    int64_t n_items;
    const SSlab* slabs;
    const SJob* jobs;
    const SSeg* segs;
    const double* ops;
    const double* x;
    int64_t x_vs;
    const int64_t* s1;
    int64_t s1_vs;
    uint16_t* op_sl;
    uint16_t* ap_sl;
    int64_t ap_sl_vs;
    int32_t* op_ex;
    int32_t* ap_ex;
    int64_t ap_ex_vs;
    int nvec;
};

// Pass 1 (FP64 sources): every source row (term t, vector v) raises its vector's
// exponent with an integer atomicMax (exact, so the result does not depend on order).
// Exponents of int64 intermediates are raised by the stage-1 epilogue instead.
__global__ void __launch_bounds__(256) k_slice_max(SliceArgs a) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t item = blockIdx.x; item < a.n_items * a.nvec; item += gridDim.x) {
        const SItem I = a.items[item / a.nvec];
        const int v = int(item % a.nvec);
        const SSlab S = a.slabs[I.slab];
        const SJob J = a.jobs[S.job];
        const SSeg g = a.segs[S.seg];
        const double* src = g.space == SP_OPS ? a.ops : a.x + int64_t(v) * a.x_vs;
        int32_t* oex = J.out_buf ? a.ap_ex + int64_t(v) * a.ap_ex_vs : a.op_ex;
        for (int rr = warp; rr < I.nrows; rr += 8) {
            const int64_t r = I.r0 + rr;
            const int t = int(r / J.nvalid), vec = int(r - int64_t(t) * J.nvalid);
            const int vg = vec / g.vper, vr = vec - vg * g.vper;
            const int64_t base = g.off + t * g.ts + vg * g.vgs + int64_t(vr) * g.vs;
            int E = INT_MIN;
            for (int k = lane; k < g.kc; k += 32) E = max(E, exp_f64(src[base + k * g.ks]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
            if (lane == 0 && E != INT_MIN) atomicMax(oex + J.out_exp + vec, E);
        }
    }
}

struct TileArgs {
    const STile* tiles;
    int64_t n_tiles;
    const SJob* jobs;
    const SSeg* segs;
    const double* ops;
    const double* x;
    int64_t x_vs;
    const int64_t* s1;
    int64_t s1_vs;
    uint16_t* op_sl;
    uint16_t* ap_sl;
    int64_t ap_sl_vs;
    const int32_t* op_ex;
    const int32_t* ap_ex;
    int64_t ap_ex_vs;
    int nvec;
};

// Pass 2: digits of 8 vectors x 256 K of one job relative to the vectors' exponents,
// one warp per such item.  For each 32-K sub-tile every lane decodes one K column
// (segment, term, entry) and forms the digits of its 8 entries; the warp assembles the
// 8x8 core matrices of every slice in its own shared-memory patch and writes them as
// 16-byte chunks (512 contiguous bytes per slice and sub-tile).  Positions outside the
// valid vectors and K stay zero from set-up.
constexpr int DIG_WARPS = 8;

__global__ void __launch_bounds__(32 * DIG_WARPS) k_slice_digits(TileArgs a) {
    __shared__ __align__(16) uint16_t sd_all[DIG_WARPS][SPL_S][8][SPL_TK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint16_t (*sd)[8][SPL_TK] = sd_all[warp];
    const int64_t n_items = a.n_tiles * a.nvec;
    for (int64_t item = int64_t(blockIdx.x) * DIG_WARPS + warp; item < n_items;
         item += int64_t(gridDim.x) * DIG_WARPS) {
        const STile T = a.tiles[item / a.nvec];
        const int v = int(item % a.nvec);
        const SJob J = a.jobs[T.job];
        const int32_t* oex = J.out_buf ? a.ap_ex + int64_t(v) * a.ap_ex_vs : a.op_ex;
        const int nv = min(8, J.nvalid - 8 * T.vg);
        int E[8];
#pragma unroll
        for (int vv = 0; vv < 8; ++vv) E[vv] = vv < nv ? oex[J.out_exp + 8 * T.vg + vv] : 0;
        uint16_t* out = J.out_buf ? a.ap_sl + int64_t(v) * a.ap_sl_vs : a.op_sl;
        const int64_t tile_elems = int64_t(J.rows_tile) * SPL_TK;
        const int vt = (8 * T.vg) / J.rows_tile, rg = ((8 * T.vg) % J.rows_tile) >> 3;
        const int kt0 = T.k0 / SPL_TK;
        const int nkt = min(SPL_TILE_K / SPL_TK, J.kt - kt0);
        for (int kt = 0; kt < nkt; ++kt) {
            const int K = T.k0 + kt * SPL_TK + lane;
            int d[8][SPL_S];
#pragma unroll
            for (int vv = 0; vv < 8; ++vv)
#pragma unroll
                for (int q = 0; q < SPL_S; ++q) d[vv][q] = 0;
            if (K < J.K) {
                int sg = T.seg;   // holds the tile's first K; later runs follow in order
                while (sg < J.seg0 + J.nseg - 1 && K >= a.segs[sg + 1].kbase) ++sg;
                const SSeg g = a.segs[sg];
                const int kb = g.kbase;
                const int t = (K - kb) / g.kc, k = (K - kb) - t * g.kc;
                const int64_t base = g.off + t * g.ts + k * g.ks;
                int vg = (8 * T.vg) / g.vper, vr = 8 * T.vg - vg * g.vper;
                if (g.is_i64) {   // loads first, then the integer digit arithmetic
                    const int64_t* s1 = a.s1 + int64_t(v) * a.s1_vs;
                    const int32_t* cex = a.ap_ex + int64_t(v) * a.ap_ex_vs + g.ec_off + k;
                    const int32_t* er = a.op_ex + g.er_off + int64_t(t) * g.er_ts;
                    long long F[8];
                    int e[8];
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv) {
                        F[vv] = vv < nv ? s1[base + vg * g.vgs + int64_t(vr) * g.vs] : 0;
                        e[vv] = vv < nv ? er[vr] + cex[int64_t(vg) * g.ec_vgs] - g.e_off : 0;
                        if (++vr == g.vper) {
                            vr = 0;
                            ++vg;
                        }
                    }
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv)
                        if (F[vv] != 0) digits_i64(F[vv], e[vv], E[vv], d[vv]);
                } else {
                    const double* src = g.space == SP_OPS ? a.ops : a.x + int64_t(v) * a.x_vs;
                    double xv[8];
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv) {
                        xv[vv] = vv < nv ? src[base + vg * g.vgs + int64_t(vr) * g.vs] : 0.0;
                        if (++vr == g.vper) {
                            vr = 0;
                            ++vg;
                        }
                    }
#pragma unroll
                    for (int vv = 0; vv < 8; ++vv) digits_f64(xv[vv], E[vv], d[vv]);
                }
            }
#pragma unroll
            for (int vv = 0; vv < 8; ++vv)
#pragma unroll
                for (int q = 0; q < SPL_S; ++q) sd[q][vv][lane] = digit_bf16(d[vv][q], q);
            __syncwarp();
            // lane -> core matrix kg = lane / 8 (K [8 kg, +8)), row vv = lane % 8
            const int kg = lane >> 3, vv = lane & 7;
#pragma unroll
            for (int q = 0; q < SPL_S; ++q) {
                const int64_t dst = J.out_tiles + ((int64_t(vt) * J.kt + kt0 + kt) * SPL_S + q) * tile_elems +
                                    (rg * 4 + kg) * 64 + vv * 8;
                *reinterpret_cast<uint4*>(out + dst) = *reinterpret_cast<const uint4*>(&sd[q][vv][kg * 8]);
            }
            __syncwarp();
        }
    }
}

// ----------------------------------------------------------------------------------
// tcgen05 slice GEMM

__device__ __forceinline__ uint32_t su32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor, K-major without swizzle: 8x8 core matrices of 128
// contiguous bytes, LBO = 128 B between K-adjacent cores, SBO = 512 B between 8-row groups.
// The low word holds the start address (bits 0-13, address / 16) and LBO / 16 (bits
// 16-29); the high word SBO / 16 (bits 32-45) and the fixed version bit 46.  Every
// operand of a stage sits below 256 KB of shared memory, so operand offsets are added to
// the low word without a carry out of the address field.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr) { return ((addr >> 4) & 0x3FFF) | ((128u >> 4) << 16); }
constexpr uint32_t UM_DESC_HI = (512u >> 4) | (1u << (46 - 32));

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major, M=128, N=64.
constexpr uint32_t UM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(SPL_TN >> 3) << 17) |
                              (uint32_t(SPL_TM >> 4) << 24);

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
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* b, uint32_t ph, long long limit, volatile int* abort,
                                                int* status) {
    const long long t0 = clock64();
    while (!mbar_try(b, ph)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            atomicExch(status, DMRG_ERR_DEVICE_TIMEOUT);
            return false;
        }
    }
    return true;
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
__device__ __forceinline__ void umma(uint32_t d, uint32_t a_lo, uint32_t b_lo, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\n.reg .b64 da, db;\nsetp.ne.b32 p, %3, 0;\nmov.b64 da, {%1, %4};\nmov.b64 db, {%2, %4};\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(d),
        "r"(a_lo), "r"(b_lo), "r"(accumulate), "r"(UM_DESC_HI), "r"(UM_IDESC));
}
__device__ __forceinline__ void umma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}

// Work list of one slice-GEMM launch (the Davidson vectors of an apply are stacked
// inside its GEMMs).
struct UmmaArgs {
    const SWork* work;
    int64_t n_work;
    const SGemm* gemms;
    const uint16_t* op_sl;
    const uint16_t* ap_sl;
    int64_t* s1;
    int64_t* s2;
    const int32_t* op_ex;
    int32_t* ap_ex;
    int* status;
};

// The 42 MMAs of one K tile (two K=16 steps x 21 slice pairs), fully unrolled so that
// each costs two 32-bit adds besides the MMA itself.  Order: K step, then level
// l = i + j, then i (consecutive MMAs mostly feed different accumulators; a run into one
// accumulator stalls on its own sum).  Level l feeds accumulator c = min(l, 4) in the
// chunk's TMEM slot.  first: the tile opens drain chunk `chunk`, so the first pair of
// every accumulator overwrites it, once the epilogue has emptied the slot (tempty).
// last: the tile closes the chunk and hands its accumulators to the epilogue (tfull);
// the next chunk waits only for accumulators 0 and 1 to be read.
__device__ __forceinline__ bool umma_ktile(UmmaSmem& sm, uint32_t tmem, uint32_t la, uint32_t ra, bool first,
                                           bool last, int64_t chunk, int* status) {
    const uint32_t a0 = sdesc_lo(la), b0 = sdesc_lo(ra);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int l = 0; l < SPL_S; ++l) {
            const int c = l < SPL_ACCS - 1 ? l : SPL_ACCS - 1;
            const int slot = um_slot(c, chunk);
            if (first && ks == 0 && l == c) {   // previous use of the slot: chunk - 1 or chunk - 2
                const uint32_t use = um_use(c, chunk);
                if (use > 0) {
                    if (!mbar_wait(sm, &sm.tempty[slot], (use - 1) & 1, status)) return false;
                    tc_fence_after();
                }
            }
#pragma unroll
            for (int i = 0; i <= l; ++i) {
                const int j = l - i;
                const uint32_t accumulate = (first && ks == 0 && i == 0 && l == c) ? 0u : 1u;
                umma(tmem + uint32_t(slot) * SPL_TN, a0 + uint32_t(i * (SPL_LT * 2) + ks * 256) / 16,
                     b0 + uint32_t(j * (SPL_RT * 2) + ks * 256) / 16, accumulate);
            }
        }
    if (last)
#pragma unroll
        for (int c = 0; c < SPL_ACCS; ++c) umma_commit(&sm.tfull[um_slot(c, chunk)]);
    return true;
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
        for (int c = 0; c < UM_SLOTS; ++c) {
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
            // 512-byte groups of every slice; the rest of the stage keeps digits of an
            // earlier tile (or the zeros of set-up), whose products land in accumulator
            // rows / columns that the epilogue never reads
            const int lg = (min(SPL_TM, G.M - W.mtile * SPL_TM) + 7) >> 3;
            const int rg = (min(SPL_TN, G.N - W.ntile * SPL_TN) + 7) >> 3;
            const uint32_t lbytes = uint32_t(lg) * 512u, rbytes = uint32_t(rg) * 512u;
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
        int64_t kidx = 0, dchunk = 0;
        bool ok = true;
        SWork Wn{};
        if (blockIdx.x < total) Wn = a.work[blockIdx.x];
        for (int64_t it = blockIdx.x; it < total && ok; it += step) {
            const SWork W = Wn;
            if (it + step < total) Wn = a.work[it + step];
            for (int kc0 = W.k0; kc0 < W.k1 && ok; kc0 += SPL_DRAIN_KT, ++dchunk) {
                const int kc1 = min(kc0 + SPL_DRAIN_KT, W.k1);
                for (int kt = kc0; kt < kc1; ++kt, ++kidx) {
                    const int s = int(kidx % UM_STAGES);
                    if (!(ok = mbar_wait(sm, &sm.full[s], uint32_t((kidx / UM_STAGES) & 1), a.status))) break;
                    tc_fence_after();
                    if (!(ok = umma_ktile(sm, tmem, su32(sm.L[s]), su32(sm.R[s]), kt == kc0, kt == kc1 - 1, dchunk,
                                          a.status)))
                        break;
                    umma_commit(&sm.empty[s]);
                }
            }
        }
        umma_commit(&sm.done);   // completes when every MMA issued above has finished
        mbar_wait_final(&sm.done, 0);
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (tile rows) and the column
        // half (w-2)/4 of every accumulator
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = 32 * q + lane, col0 = h * UM_EPI_COLS;
        const uint32_t lane_addr = uint32_t(32 * q) << 16;
        int64_t dchunk = 0;
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
            const int fs = G.fshift;
            const int r = W.mtile * SPL_TM + row;
            const int cbase = W.ntile * SPL_TN + col0;
            // stage 1: the exponents its epilogue needs, loaded before the drain (both
            // arrays are read-only while stage 1 runs): column cbase + lane, this row
            const bool rv = r < G.M;
            int cex_l = 0, erow = 0;
            if (G.kind == 0) {
                if (cbase + lane < G.N) cex_l = a.ap_ex[G.ec_off + cbase + lane];
                if (rv) erow = a.op_ex[G.er_off + r];
            }
            long long acc[UM_EPI_COLS];   // slice sums of the item in units of 2^-31
#pragma unroll
            for (int j = 0; j < UM_EPI_COLS; ++j) acc[j] = 0;
            for (int kc0 = W.k0; kc0 < W.k1 && ok; kc0 += SPL_DRAIN_KT, ++dchunk) {
                // 32-bit conversions only (the 64-bit one is an FP64-rate operation): acc c
                // holds the exact level sum in units of 2^(-8c) for c < 4 (|sum| <=
                // (c+1) 2^22 in those units), acc 4 the rest, rounded to units of 2^-31
                // (< 2^24 of them); each is added in units of 2^-31, the chunk's total
                // staying below 2^53.01.  An accumulator is handed back to the MMA issuer
                // as soon as it is in registers.
#pragma unroll
                for (int c = 0; c < SPL_ACCS; ++c) {
                    // warp-uniform outcome: the TMEM loads below are .sync.aligned
                    const int slot = um_slot(c, dchunk);
                    ok = __all_sync(0xffffffffu, mbar_wait(sm, &sm.tfull[slot], um_use(c, dchunk) & 1, a.status));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t base = tmem + lane_addr + uint32_t(slot) * SPL_TN + col0;
                    uint32_t rv[UM_EPI_COLS];
#pragma unroll
                    for (int c0 = 0; c0 < UM_EPI_COLS; c0 += 8)
                        tmem_ld8(base + c0, *reinterpret_cast<uint32_t(*)[8]>(rv + c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    tc_fence_before();
                    mbar_arrive(&sm.tempty[slot]);
                    const float scale = c == 0 ? 1.0f : c == 1 ? 256.0f : c == 2 ? 65536.0f : c == 3 ? 16777216.0f : 2147483648.0f;
#pragma unroll
                    for (int j = 0; j < UM_EPI_COLS; ++j) {
                        const int iv = __float2int_rn(__uint_as_float(rv[j]) * scale);
                        if (c == 0)
                            acc[j] += static_cast<long long>(iv) * (1ll << 31);
                        else if (c < SPL_ACCS - 1)
                            acc[j] += static_cast<long long>(iv) * (1 << (31 - 8 * c));
                        else
                            acc[j] += iv;
                    }
                }
            }
            if (!ok) break;
            // F = round(2^fs * sum): exact for fs >= 31 (up to 32 drains of 2^53.01 stay
            // below 2^58.01; the GEMM's shift keeps F below 2^62); for fs < 31 only the
            // part below 2^-fs, i.e. of i4, is rounded
#pragma unroll
            for (int j = 0; j < UM_EPI_COLS; ++j)
                acc[j] = fs >= 31 ? static_cast<long long>(static_cast<unsigned long long>(acc[j]) << (fs - 31))
                                  : (acc[j] + (1ll << (30 - fs))) >> (31 - fs);
            if (G.kind == 0) {
                // exponents of the stage-2 vectors fed by this row: the column exponents
                // come with one load per warp (lane l holds column cbase + l) and a
                // broadcast per column, so no global load sits between the atomics
                const int rs = rv ? r : 0;
                // stage-2 vector of entry (r, c): (c / colgroup) * period + r % period
                int32_t* x2 = a.ap_ex + G.x2_exp + rs % G.x2_period;
                const int eoff = erow - (14 + G.fshift);
                int emax = INT_MIN, grp = cbase / G.x2_colgroup;
                int next = (grp + 1) * G.x2_colgroup;   // first column of the next group
#pragma unroll
                for (int j = 0; j < UM_EPI_COLS; ++j) {
                    const int c = cbase + j;   // the same for every lane
                    const int ce = __shfl_sync(0xffffffffu, cex_l, j);
                    if (c < G.N) {
                        if (c >= next) {
                            if (rv && emax != INT_MIN) atomicMax(x2 + grp * G.x2_period, emax + eoff);
                            emax = INT_MIN;
                            ++grp;
                            next += G.x2_colgroup;
                        }
                        if (acc[j] != 0) {
                            const unsigned long long u = acc[j] < 0 ? static_cast<unsigned long long>(-acc[j])
                                                                    : static_cast<unsigned long long>(acc[j]);
                            emax = max(emax, (64 - __clzll(u)) + ce);
                        }
                    }
                }
                if (rv && emax != INT_MIN) atomicMax(x2 + grp * G.x2_period, emax + eoff);
                // row-major store through the warp's shared-memory patch: each pass moves
                // 4 columns of the warp's 32 rows, written as 8 rows x 32 contiguous bytes
                // per instruction instead of 32 rows x 8 bytes
                long long* tp = sm.tr[warp - 2];
                int64_t* D = a.s1 + G.d_off;
                const int rbase = W.mtile * SPL_TM + 32 * q;
#pragma unroll
                for (int c4 = 0; c4 < UM_EPI_COLS; c4 += 4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) tp[lane * UM_TR_LD + j] = G.sign > 0 ? acc[c4 + j] : -acc[c4 + j];
                    __syncwarp();
                    const int cc = lane & 3, c = cbase + c4 + cc;
#pragma unroll
                    for (int rep = 0; rep < 4; ++rep) {
                        const int rr = 8 * rep + (lane >> 2), gr = rbase + rr;
                        if (gr < G.M && c < G.N) D[int64_t(gr) * G.ldd + c] = tp[rr * UM_TR_LD + cc];
                    }
                    __syncwarp();
                }
            } else if (r < G.M) {
                unsigned long long* D = reinterpret_cast<unsigned long long*>(a.s2 +
                                                                              G.d_off + int64_t(r) * G.ldd);
#pragma unroll
                for (int j = 0; j < UM_EPI_COLS; ++j) {
                    const int c = cbase + j;
                    if (c < G.N && acc[j] != 0) atomicAdd(D + c, static_cast<unsigned long long>(acc[j]));
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

__global__ void k_finalize(const SBlock* __restrict__ blocks, const SPart* __restrict__ parts,
                           const int64_t* __restrict__ s2, int64_t s2_vs, const int32_t* __restrict__ op_ex,
                           const int32_t* __restrict__ ap_ex, int64_t ap_ex_vs, double* __restrict__ y, int64_t dim) {
    const SBlock B = blocks[blockIdx.x];
    const int v = blockIdx.y;
    const int32_t* aex = ap_ex + int64_t(v) * ap_ex_vs;
    const int64_t* S2 = s2 + int64_t(v) * s2_vs;
    for (int e = threadIdx.x; e < B.rows * B.cols; e += blockDim.x) {
        const int i = e / B.cols, j = e % B.cols;
        double sum = 0.0;
        for (int p = B.p0; p < B.p0 + B.np; ++p) {
            const SPart P = parts[p];
            const int ri = v * P.rstack + i, cj = v * P.cstack + j;
            const long long F = S2[P.acc_off + int64_t(ri) * P.ld + cj];
            if (F == 0) continue;
            const int er = (P.er_buf ? aex : op_ex)[P.er_off + ri];
            const int ec = (P.ec_buf ? aex : op_ex)[P.ec_off + cj];
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

// Host-side bounds proof of a split plan: every bulk-copy source range, slicer write,
// exponent read/write, stage-1 store and stage-2 sum lies inside its buffer.
int validate_split_plan(const Plan& P, const SplitHost& H, std::string* err) {
    auto bad = [&](const char* what) {
        *err = std::string("split plan out of bounds: ") + what;
        return DMRG_ERR_BOUNDS;
    };
    for (const SJob& J : H.jobs) {
        const int64_t tiles = int64_t(J.npad / J.rows_tile) * J.kt * SPL_S * J.rows_tile * SPL_TK;
        const int64_t sl = J.out_buf ? H.ap_sl_vs : H.op_sl;
        const int64_t ex = J.out_buf ? H.ap_ex_vs : H.op_ex;
        if (J.npad % J.rows_tile || J.npad < J.nvalid || J.kt * SPL_TK < J.K) return bad("job shape");
        if (J.out_tiles < 0 || J.out_tiles % 8 || J.out_tiles + tiles > sl) return bad("slice tiles");
        if (J.out_exp < 0 || J.out_exp + J.npad > ex) return bad("exponents");
        int64_t K = 0;
        for (int s = J.seg0; s < J.seg0 + J.nseg; ++s) {
            const SSeg& g = H.segs[s];
            if (g.kbase != K) return bad("segment K base");
            K += int64_t(g.kc) * g.nt;
            if (J.nvalid == 0 || g.kc <= 0 || g.nt <= 0) continue;
            if (g.vper < 1) return bad("vector grouping");
            const int ngrp = (J.nvalid - 1) / g.vper, rmax = std::min(J.nvalid, g.vper) - 1;
            const int64_t last = g.off + (g.nt - 1) * g.ts + ngrp * g.vgs + int64_t(rmax) * g.vs + int64_t(g.kc - 1) * g.ks;
            const int64_t lim = g.space == SP_OPS ? P.ops_len
                                                  : (g.space == SP_X ? P.dim * H.nv : P.scratch_len * H.nv);
            if (g.off < 0 || last >= lim) return bad("slice source");
            if (g.is_i64) {
                if (g.space != SP_SCR) return bad("int64 source space");
                if (g.er_off < 0 || g.er_off + int64_t(g.nt - 1) * g.er_ts + rmax + 1 > H.op_ex) return bad("row exps");
                if (g.ec_off < 0 || g.ec_off + int64_t(ngrp) * g.ec_vgs + g.kc > H.ap_ex_vs) return bad("col exps");
            }
        }
        if (K != J.K) return bad("job K");
    }
    for (const STile& T : H.tiles) {   // the digit pass starts its segment search at T.seg
        if (T.job < 0 || T.job >= int32_t(H.jobs.size())) return bad("tile job");
        const SJob& J = H.jobs[size_t(T.job)];
        if (T.seg < J.seg0 || T.seg >= J.seg0 + J.nseg || T.k0 < 0 || T.k0 >= J.K || 8 * T.vg >= J.nvalid ||
            H.segs[size_t(T.seg)].kbase > T.k0)
            return bad("tile segment");
    }
    auto check_work = [&](const std::vector<SWork>& w) {
        for (const SWork& x : w) {
            const SGemm& G = H.gemms[x.gemm];
            if (x.k0 < 0 || x.k1 > G.kt || x.k0 >= x.k1) return false;
            if (cdiv(x.k1 - x.k0, SPL_DRAIN_KT) > SPL_MAX_DRAINS) return false;   // epilogue sum bound
            const int64_t lsz = G.l_buf ? H.ap_sl_vs : H.op_sl, rsz = G.r_buf ? H.ap_sl_vs : H.op_sl;
            const int64_t lend = G.l_tiles + (int64_t(x.mtile) * G.kt + x.k1) * (SPL_S * SPL_LT);
            const int64_t rend = G.r_tiles + (int64_t(x.ntile) * G.kt + x.k1) * (SPL_S * SPL_RT);
            if (G.l_tiles % 8 || G.r_tiles % 8 || lend > lsz || rend > rsz) return false;
            if (int64_t(x.mtile) * SPL_TM >= G.M || int64_t(x.ntile) * SPL_TN >= G.N) return false;
            const int64_t dend = G.d_off + int64_t(G.M - 1) * G.ldd + G.N;
            if (G.ldd < G.N || dend > (G.kind == 0 ? H.s1_vs : H.s2_vs)) return false;
            if (G.kind == 0) {   // stage-1 epilogue exponent reads and raises
                const int64_t ngrp = G.x2_colgroup > 0 ? (G.N - 1) / G.x2_colgroup : -1;
                if (G.x2_exp < 0 || G.x2_period <= 0 || ngrp < 0 ||
                    G.x2_exp + (ngrp + 1) * G.x2_period > H.ap_ex_vs)
                    return false;
                if (G.er_off < 0 || G.er_off + G.M > H.op_ex || G.ec_off < 0 || G.ec_off + G.N > H.ap_ex_vs)
                    return false;
            }
        }
        return true;
    };
    if (!check_work(H.w1) || !check_work(H.w2)) return bad("gemm work");
    for (const STile& T : H.tiles) {
        if (T.job < 0 || T.job >= int32_t(H.jobs.size())) return bad("slice tile job");
        const SJob& J = H.jobs[T.job];
        if (T.vg < 0 || 8 * T.vg >= J.nvalid || 8 * T.vg + 8 > J.npad || J.rows_tile % 8) return bad("slice tile rows");
        if (T.k0 < 0 || T.k0 >= J.K || T.k0 % SPL_TILE_K) return bad("slice tile K");
    }
    for (const SItem& I : H.items) {
        if (I.slab < 0 || I.slab >= int32_t(H.slabs.size())) return bad("slice item");
        const SSlab& Sl = H.slabs[I.slab];
        if (I.r0 < 0 || I.nrows <= 0 || I.r0 + I.nrows > Sl.rows) return bad("slice item rows");
        const SJob& J = H.jobs[Sl.job];
        if (Sl.seg < J.seg0 || Sl.seg >= J.seg0 + J.nseg || Sl.rows != int64_t(H.segs[Sl.seg].nt) * J.nvalid)
            return bad("slice slab");
    }
    for (const SBlock& B : H.blocks)
        for (int p = B.p0; p < B.p0 + B.np; ++p) {
            const SPart& Q = H.parts[p];
            const int64_t rmax = int64_t(H.nv - 1) * Q.rstack + B.rows, cmax = int64_t(H.nv - 1) * Q.cstack + B.cols;
            if (Q.ld < cmax || Q.acc_off + (rmax - 1) * Q.ld + cmax > H.s2_vs) return bad("finalize sums");
            if (Q.er_off + rmax > (Q.er_buf ? H.ap_ex_vs : H.op_ex)) return bad("finalize row exps");
            if (Q.ec_off + cmax > (Q.ec_buf ? H.ap_ex_vs : H.op_ex)) return bad("finalize col exps");
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
    // that leaves >= 4 items per SM.
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
        const int chunk = sc > 0 ? sc : adaptive;
        for (int k0 = 0; k0 < m.kt; k0 += chunk)
            for (int mt = 0; mt < cdiv(m.M, SPL_TM); ++mt)
                for (int nt = 0; nt < cdiv(m.N, SPL_TN); ++nt)
                    w2.push_back({int32_t(gi), mt, nt, k0, std::min(m.kt, k0 + chunk), 0});
    }
    // longest items first; one launch per GEMM keeps each GEMM's items contiguous
    auto by_cost = [](const SWork& x, const SWork& y) { return (x.k1 - x.k0) > (y.k1 - y.k0); };
    auto by_gemm = [](const SWork& x, const SWork& y) {
        return x.gemm != y.gemm ? x.gemm < y.gemm : (x.k1 - x.k0) > (y.k1 - y.k0);
    };
    for (int st = 0; st < 2; ++st) {
        std::vector<SWork>& w = st == 0 ? w1 : w2;
        if (!S.per_gemm) {
            std::stable_sort(w.begin(), w.end(), by_cost);
            continue;
        }
        std::stable_sort(w.begin(), w.end(), by_gemm);
        auto& R = st == 0 ? H.r1 : H.r2;
        for (int32_t i = 0; i < int32_t(w.size());) {
            int32_t j = i;
            while (j < int32_t(w.size()) && w[j].gemm == w[i].gemm) ++j;
            R.push_back({i, j});
            i = j;
        }
    }
}

int build_split_plan(const Plan& P, int nv, SplitHost& H, std::string* err, const Schedule& S) {
    std::vector<SGemm>& gemms = H.gemms;
    std::vector<SSeg>& segs = H.segs;
    std::vector<SJob>& jobs = H.jobs;
    std::vector<int32_t> op_jobs, x_jobs, mid_jobs;
    std::vector<SBlock>& blocks = H.blocks;
    blocks.assign(P.blocks.size(), SBlock{});
    std::vector<SPart>& parts = H.parts;
    int64_t op_sl = 0, op_ex = 0, ap_sl = 0, ap_ex = 0, s2 = 0;

    auto add_job = [&](int out_buf, int rows_tile, int nvalid, int64_t K, const std::vector<SSeg>& js,
                       int64_t* tiles_off, int64_t* exp_off) {
        SJob J{};
        J.out_buf = out_buf;
        J.rows_tile = rows_tile;
        J.nvalid = nvalid;
        J.npad = int32_t(cdiv(nvalid, rows_tile) * rows_tile);
        J.K = int32_t(K);
        J.kt = int32_t(cdiv(K, SPL_TK));
        J.seg0 = int32_t(segs.size());
        J.nseg = int32_t(js.size());
        int32_t kb = 0;
        for (SSeg g : js) {
            g.kbase = kb;
            kb += g.kc * g.nt;
            segs.push_back(g);
        }
        int64_t& sl = out_buf ? ap_sl : op_sl;
        int64_t& ex = out_buf ? ap_ex : op_ex;
        J.out_tiles = sl;
        J.out_exp = ex;
        sl += int64_t(J.npad) * J.kt * SPL_TK * SPL_S;
        ex += J.npad;
        *tiles_off = J.out_tiles;
        *exp_off = J.out_exp;
        jobs.push_back(J);
        return int32_t(jobs.size() - 1);
    };
    auto seg = [](int space, int64_t off, int64_t ts, int64_t vs, int64_t ks, int kc, int nt) {
        SSeg s{};
        s.space = space; s.off = off; s.ts = ts; s.vs = vs; s.ks = ks; s.kc = kc; s.nt = nt;
        s.vper = 1 << 30;   // one vector group unless stacked
        return s;
    };
    // the same entries for nv stacked Davidson vectors: vector v*per + r of vector v
    auto stacked = [](SSeg s, int per, int64_t vgs, int32_t ec_vgs) {
        s.vper = per; s.vgs = vgs; s.ec_vgs = ec_vgs;
        return s;
    };
    if (nv < 1 || nv > 64) {
        *err = "nvec out of range";
        return DMRG_ERR_INVALID_ARG;
    }
    if (int64_t(P.groups.size()) > (int64_t(1) << 30)) {
        *err = "too many groups";
        return DMRG_ERR_INVALID_ARG;
    }

    // stage 1: one GEMM per group; L = stacked operator (operator slices), R = x block
    std::vector<int64_t> s1_lexp(P.groups.size()), s1_rexp(P.groups.size());
    std::vector<int32_t> s1_eoff(P.groups.size());
    for (size_t g = 0; g < P.groups.size(); ++g) {
        const Group& G = P.groups[g];
        const PsiBlock& B = P.blocks[G.in_block];
        const int n = int(G.terms.size());
        SGemm m{};
        int64_t lt, le, rt, re;
        // the nv Davidson vectors stack along N: column v*c + j is column j of vector v
        if (G.order == 0) {   // X_g = A_stack (n a x b) * [x_q^(v)] (b x nv c)
            m.M = n * G.a; m.N = nv * G.c;
            op_jobs.push_back(add_job(0, SPL_TM, m.M, G.b, {seg(SP_OPS, G.a_stack, 0, G.b, 1, G.b, 1)}, &lt, &le));
            x_jobs.push_back(add_job(1, SPL_TN, m.N, G.b,
                                     {stacked(seg(SP_X, B.off, 0, 1, G.c, G.b, 1), G.c, P.dim, 0)}, &rt, &re));
        } else {              // Z_g^T = B_stack (n d x c) * [x_q^(v)T] (c x nv b)
            m.M = n * G.d; m.N = nv * G.b;
            op_jobs.push_back(add_job(0, SPL_TM, m.M, G.c, {seg(SP_OPS, G.b_stack, 0, G.c, 1, G.c, 1)}, &lt, &le));
            x_jobs.push_back(add_job(1, SPL_TN, m.N, G.c,
                                     {stacked(seg(SP_X, B.off, 0, G.c, 1, G.c, 1), G.b, P.dim, 0)}, &rt, &re));
        }
        m.l_tiles = lt; m.r_tiles = rt; m.l_buf = 0; m.r_buf = 1;
        m.kt = int32_t(cdiv(G.order == 0 ? G.b : G.c, SPL_TK));
        if (m.kt > SPL_MAX_DRAINS * SPL_DRAIN_KT) {   // one stage-1 item spans the whole contraction
            *err = "split path: a sector dimension above 8192";
            return DMRG_ERR_INVALID_ARG;
        }
        m.d_off = int64_t(nv) * G.scratch; m.ldd = m.N; m.kind = 0; m.sign = G.sign < 0 ? -1 : 1;
        m.fshift = fshift_for(G.order == 0 ? G.b : G.c);
        m.er_off = le; m.ec_off = re; m.x2_exp = -1;
        m.x2_period = G.order == 0 ? G.a : G.d;
        m.x2_colgroup = G.order == 0 ? G.c : G.b;
        s1_lexp[g] = le; s1_rexp[g] = re; s1_eoff[g] = 14 + m.fshift;
        gemms.push_back(m);
    }
    // stage 2: per output block, one GEMM over its A-first groups and one over its B-first groups
    std::vector<std::vector<int32_t>> by_out(P.blocks.size());
    for (int32_t g = 0; g < int32_t(P.groups.size()); ++g) by_out[P.groups[g].out_block].push_back(g);
    for (size_t o = 0; o < P.blocks.size(); ++o) {
        const PsiBlock& O = P.blocks[o];
        blocks[o] = {O.off, O.rows, O.cols, int32_t(parts.size()), 0};
        for (int order = 0; order < 2; ++order) {
            std::vector<SSeg> lseg, rseg;
            int64_t K = 0;
            for (int32_t g : by_out[o]) {
                const Group& G = P.groups[g];
                if (G.order != order) continue;
                const int n = int(G.terms.size());
                const int64_t sc = int64_t(nv) * G.scratch;
                if (order == 0) {  // L = X_g rows (int64), vectors stacked along M; R = B_t rows
                    // vector v*a + i, entry (t, k) = X_g[t a + i][v c + k]  (X_g is n a x nv c)
                    SSeg s = stacked(seg(SP_SCR, sc, int64_t(G.a) * nv * G.c, int64_t(nv) * G.c, 1, G.c, n),
                                     G.a, G.c, G.c);
                    s.is_i64 = 1; s.er_off = s1_lexp[g]; s.er_ts = G.a; s.ec_off = s1_rexp[g]; s.e_off = s1_eoff[g];
                    lseg.push_back(s);
                    rseg.push_back(seg(SP_OPS, G.b_stack, int64_t(G.d) * G.c, G.c, 1, G.c, n));
                    K += int64_t(G.c) * n;
                } else {           // L = c_t A_t rows; R = Z_g^T rows (int64), vectors stacked along N
                    // vector v*d + j, entry (t, k) = Z_g^T[t d + j][v b + k]  (Z_g^T is n d x nv b)
                    lseg.push_back(seg(SP_OPS, G.a_stack, int64_t(G.a) * G.b, G.b, 1, G.b, n));
                    SSeg s = stacked(seg(SP_SCR, sc, int64_t(G.d) * nv * G.b, int64_t(nv) * G.b, 1, G.b, n),
                                     G.d, G.b, G.b);
                    s.is_i64 = 1; s.er_off = s1_lexp[g]; s.er_ts = G.d; s.ec_off = s1_rexp[g]; s.e_off = s1_eoff[g];
                    rseg.push_back(s);
                    K += int64_t(G.b) * n;
                }
            }
            if (lseg.empty()) continue;
            if (K > SPL_MAX_K) {
                *err = "stage-2 contraction longer than 2^23";
                return DMRG_ERR_INVALID_ARG;
            }
            SGemm m{};
            m.M = order == 0 ? nv * O.rows : O.rows;
            m.N = order == 0 ? O.cols : nv * O.cols;
            m.kt = int32_t(cdiv(K, SPL_TK));
            int64_t lt, le, rt, re;
            const int lbuf = order == 0 ? 1 : 0, rbuf = order == 0 ? 0 : 1;
            int32_t lj = add_job(lbuf, SPL_TM, m.M, K, lseg, &lt, &le);
            int32_t rj = add_job(rbuf, SPL_TN, m.N, K, rseg, &rt, &re);
            for (int32_t g : by_out[o])   // stage-1 GEMMs whose rows feed this job's vectors
                if (P.groups[g].order == order) gemms[g].x2_exp = order == 0 ? le : re;
            (lbuf ? mid_jobs : op_jobs).push_back(lj);
            (rbuf ? mid_jobs : op_jobs).push_back(rj);
            m.l_tiles = lt; m.r_tiles = rt; m.l_buf = lbuf; m.r_buf = rbuf;
            m.d_off = s2; m.ldd = m.N; m.kind = 1; m.sign = 1;
            m.fshift = fshift_for(K);
            SPart part{};
            part.acc_off = s2; part.er_off = le; part.ec_off = re; part.er_buf = lbuf; part.ec_buf = rbuf;
            part.e_off = 14 + m.fshift; part.ld = m.N;
            part.rstack = order == 0 ? O.rows : 0;
            part.cstack = order == 0 ? 0 : O.cols;
            parts.push_back(part);
            blocks[o].np += 1;
            s2 += int64_t(m.M) * m.N;
            gemms.push_back(m);
        }
    }
    build_split_work(H, S);
    std::vector<SSlab>& slabs = H.slabs;
    std::vector<SItem>& items = H.items;
    auto add_items = [&](const std::vector<int32_t>& js) {
        for (int32_t j : js) {
            int32_t kb = 0;
            for (int sg = jobs[j].seg0; sg < jobs[j].seg0 + jobs[j].nseg; ++sg) {
                const int64_t n = int64_t(segs[sg].nt) * jobs[j].nvalid;
                if (n > 0) {
                    const int32_t sl = int32_t(slabs.size());
                    slabs.push_back({n, j, sg, kb, 0});
                    for (int64_t r0 = 0; r0 < n; r0 += SPL_ROWS_PER_ITEM)
                        items.push_back({r0, sl, int32_t(std::min<int64_t>(SPL_ROWS_PER_ITEM, n - r0))});
                }
                kb += segs[sg].kc * segs[sg].nt;
            }
        }
    };
    H.it_op0 = 0;
    add_items(op_jobs);
    H.it_x0 = int64_t(items.size());
    add_items(x_jobs);
    H.it_mid0 = int64_t(items.size());
    add_items(mid_jobs);
    H.it_end = int64_t(items.size());
    std::vector<STile>& tiles = H.tiles;
    auto add_tiles = [&](const std::vector<int32_t>& js) {
        for (int32_t j : js)
            for (int vg = 0; 8 * vg < jobs[j].nvalid; ++vg) {
                int32_t sg = jobs[j].seg0;
                for (int k0 = 0; k0 < jobs[j].K; k0 += SPL_TILE_K) {
                    while (sg < jobs[j].seg0 + jobs[j].nseg - 1 && k0 >= segs[sg].kbase + segs[sg].kc * segs[sg].nt)
                        ++sg;
                    tiles.push_back({j, vg, k0, sg});
                }
            }
    };
    H.tl_op0 = 0;
    add_tiles(op_jobs);
    H.tl_x0 = int64_t(tiles.size());
    add_tiles(x_jobs);
    H.tl_mid0 = int64_t(tiles.size());
    add_tiles(mid_jobs);
    H.tl_end = int64_t(tiles.size());
    H.op_sl = op_sl;
    H.op_ex = op_ex + 1;
    H.ap_sl_vs = cdiv(ap_sl, 64) * 64;
    H.ap_ex_vs = cdiv(ap_ex, 4) * 4 + 4;
    H.s1_vs = P.scratch_len * nv;
    H.s2_vs = s2;
    H.nv = nv;
    return validate_split_plan(P, H, err);
}

int Handle::init_split() {
    const Plan& P = plan;
    SplitState* S = new SplitState();
    split = S;
    std::string err;
    // one plan per number of stacked vectors; operator slices are identical in all of them
    std::vector<SplitHost> hosts(static_cast<size_t>(max_nvec));
    int64_t ap_sl = 0, ap_ex = 0, s1 = 0, s2 = 0;
    for (int nv = 1; nv <= max_nvec; ++nv) {
        SplitHost& H = hosts[size_t(nv - 1)];
        const int rc0 = build_split_plan(P, nv, H, &err);
        if (rc0 != DMRG_OK) return fail(rc0, err);
        if (H.op_sl != hosts[0].op_sl || H.op_ex != hosts[0].op_ex)
            return fail(DMRG_ERR_BOUNDS, "operator slice layout differs between plans");
        ap_sl = std::max(ap_sl, H.ap_sl_vs);
        ap_ex = std::max(ap_ex, H.ap_ex_vs);
        s1 = std::max(s1, H.s1_vs);
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
        (rc = al((void**)&S->ap_sl, sizeof(uint16_t) * ap_sl, "apply slices")) ||
        (rc = al((void**)&S->ap_ex, sizeof(int32_t) * ap_ex, "apply exponents")) ||
        (rc = al((void**)&S->s1, sizeof(int64_t) * s1, "stage-1 int64 results")) ||
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
        D.n_blocks = int64_t(H.blocks.size());
        D.it_op0 = H.it_op0; D.it_x0 = H.it_x0; D.it_mid0 = H.it_mid0; D.it_end = H.it_end;
        D.tl_op0 = H.tl_op0; D.tl_x0 = H.tl_x0; D.tl_mid0 = H.tl_mid0; D.tl_end = H.tl_end;
        D.ap_ex_len = H.ap_ex_vs;
        D.s2_len = H.s2_vs;
        // algorithmic DRAM bytes of the two slice-GEMM launches: slice tiles read once
        // (12 B per entry) plus the int64 results written (stage 1) or added (stage 2)
        for (size_t gi = 0; gi < H.gemms.size(); ++gi) {
            const SGemm& m = H.gemms[gi];
            const double bytes = 12.0 * (double(m.M) + m.N) * m.kt * SPL_TK + 8.0 * double(m.M) * m.N;
            (m.kind == 0 ? D.s1_bytes : D.s2_bytes) += bytes;
        }
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
    S->kid_x = prof.kernel_id("split_slice/x");
    S->kid_s1 = prof.kernel_id("umma_slices/stage1");
    S->kid_mid = prof.kernel_id("split_slice/intermediate");
    S->kid_s2 = prof.kernel_id("umma_slices/stage2");
    S->kid_fin = prof.kernel_id("split_finalize");
    // slice buffers start at zero (padding is never written again), exponents at "none"
    if (op_sl > 0 && (e = cudaMemset(S->op_sl, 0, sizeof(uint16_t) * op_sl)) != cudaSuccess) return cuda_fail(e, "zero slices");
    if (ap_sl > 0 && (e = cudaMemset(S->ap_sl, 0, sizeof(uint16_t) * ap_sl)) != cudaSuccess) return cuda_fail(e, "zero slices");
    if ((e = cudaMemset(S->op_ex, 0xC0, sizeof(int32_t) * op_ex)) != cudaSuccess) return cuda_fail(e, "exponents");
    // operator slices, once (from the first plan; every plan has the same operator jobs)
    const SplitDevPlan& D0 = S->plans[0];
    if (D0.it_x0 > D0.it_op0) {
        SliceArgs sa{D0.items + D0.it_op0, D0.it_x0 - D0.it_op0, D0.slabs, D0.jobs, D0.segs, d_ops, nullptr, 0,
                     nullptr, 0, S->op_sl, S->ap_sl, 0, S->op_ex, S->ap_ex, 0, 1};
        TileArgs ta{D0.tiles + D0.tl_op0, D0.tl_x0 - D0.tl_op0, D0.jobs, D0.segs, d_ops, nullptr, 0, nullptr, 0,
                    S->op_sl, S->ap_sl, 0, S->op_ex, S->ap_ex, 0, 1};
        k_slice_max<<<unsigned(std::min<int64_t>(D0.it_x0 - D0.it_op0, int64_t(n_sm) * 16)), 256>>>(sa);
        k_slice_digits<<<unsigned(std::min<int64_t>(cdiv(D0.tl_x0 - D0.tl_op0, DIG_WARPS), int64_t(n_sm) * 16)),
                         32 * DIG_WARPS>>>(ta);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "operator slicing");
    }
    return DMRG_OK;
}

// One split H_eff*psi for nvec stacked vectors: slice x, stage-1 slice GEMM (int64 results,
// stage-2 exponents raised), slice intermediates, stage-2 slice GEMM (int64 sums), finalize.
int Handle::apply_split(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    SplitState* S = split;
    const SplitDevPlan& D = S->plans[size_t(nvec - 1)];
    Profiler::Pending pe;
    cudaError_t e;
    const int64_t slice_grid_cap = int64_t(n_sm) * 16;
    auto slice = [&](int64_t i0, int64_t i1, int64_t t0, int64_t t1, bool with_max, int kid) {
        if (t1 == t0) return cudaSuccess;
        SliceArgs sa{D.items + i0, i1 - i0, D.slabs, D.jobs, D.segs, d_ops, x, 0, S->s1, 0,
                     S->op_sl, S->ap_sl, 0, S->op_ex, S->ap_ex, 0, 1};
        TileArgs ta{D.tiles + t0, t1 - t0, D.jobs, D.segs, d_ops, x, 0, S->s1, 0, S->op_sl,
                    S->ap_sl, 0, S->op_ex, S->ap_ex, 0, 1};
        prof.begin(kid, st, 0.0, 0.0, &pe);
        if (with_max && i1 > i0)
            k_slice_max<<<unsigned(std::min<int64_t>(i1 - i0, slice_grid_cap)), 256, 0, st>>>(sa);
        k_slice_digits<<<unsigned(std::min<int64_t>(cdiv(t1 - t0, DIG_WARPS), slice_grid_cap)), 32 * DIG_WARPS, 0,
                         st>>>(ta);
        prof.end(pe, st);
        return cudaGetLastError();
    };
    // one stage: a single persistent launch over its work list, or (per_gemm) one launch
    // per GEMM over that GEMM's contiguous range
    auto gemm = [&](const SWork* w, int64_t nw, const std::vector<std::pair<int32_t, int32_t>>& rg, int kid,
                    double flops, double bytes) {
        if (nw == 0) return cudaSuccess;
        auto launch = [&](const SWork* w0, int64_t n) {
            UmmaArgs ua{w0, n, D.gemms, S->op_sl, S->ap_sl, S->s1, S->s2, S->op_ex, S->ap_ex, S->status};
            k_umma<<<unsigned(std::min<int64_t>(n, n_sm)), UM_THREADS, sizeof(UmmaSmem), st>>>(ua);
            return cudaGetLastError();
        };
        prof.begin(kid, st, flops, bytes, &pe);
        cudaError_t le = cudaSuccess;
        if (!sched.per_gemm)
            le = launch(w, nw);
        else
            for (size_t r = 0; r < rg.size() && le == cudaSuccess; ++r)
                le = launch(w + rg[r].first, rg[r].second - rg[r].first);
        prof.end(pe, st);
        return le;
    };
    if ((e = cudaMemsetAsync(S->ap_ex, 0xC0, sizeof(int32_t) * D.ap_ex_len, st)) != cudaSuccess)
        return cuda_fail(e, "reset exponents");
    if ((e = slice(D.it_x0, D.it_mid0, D.tl_x0, D.tl_mid0, true, S->kid_x)) != cudaSuccess)
        return cuda_fail(e, "slice x");
    if ((e = gemm(D.work1, D.n_work1, D.r1, S->kid_s1, s1_flops * nvec, D.s1_bytes)) != cudaSuccess)
        return cuda_fail(e, "stage-1 slice gemm");
    if ((e = slice(D.it_mid0, D.it_end, D.tl_mid0, D.tl_end, false, S->kid_mid)) != cudaSuccess)
        return cuda_fail(e, "slice intermediates");
    if (D.s2_len > 0 && (e = cudaMemsetAsync(S->s2, 0, sizeof(int64_t) * D.s2_len, st)) != cudaSuccess)
        return cuda_fail(e, "zero stage-2 sums");
    if ((e = gemm(D.work2, D.n_work2, D.r2, S->kid_s2, s2_flops * nvec, D.s2_bytes)) != cudaSuccess)
        return cuda_fail(e, "stage-2 slice gemm");
    if (D.n_blocks > 0) {
        prof.begin(S->kid_fin, st, 0.0, 0.0, &pe);
        k_finalize<<<dim3(unsigned(D.n_blocks), unsigned(nvec)), 256, 0, st>>>(D.blocks, D.parts, S->s2, 0, S->op_ex,
                                                                              S->ap_ex, 0, y, plan.dim);
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
            const int rc = build_split_plan(plan, nv, H, &err, s);
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
