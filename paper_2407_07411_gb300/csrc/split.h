// Split-precision (Ozaki) path: descriptors shared by the host planner and the kernels.
//
// Arithmetic.  An FP64 operand is cut, per row of the left factor and per column of
// the right factor (a "vector" along the contraction index K), into S = 6 balanced
// base-256 digits relative to the vector's exponent E (|a| < 2^E for every entry):
//     a = 2^(E-7) * sum_k d_k 2^(-8k),   d_0 in [-128, 128], d_k in [-127, 128],
// rounded after the sixth digit (relative error <= 2^-48 of the vector's maximum).
// Slice k stores the exact BF16 value d_k 2^(-8k).  A product L*R is the sum of the
// slice-pair products with i + j <= 5 (21 pairs; the dropped pairs weigh <= 2^-48),
// accumulated on the tensor cores in five FP32 accumulators, one per pair level
// l = i + j up to 3 and one for the rest:
//     acc0 = L_0 R_0                        (integers, exact while K <= 1024)
//     acc1 = L_0 R_1 + L_1 R_0              (multiples of 2^-8, exact while K <= 512)
//     acc2 = the 3 pairs with i + j = 2     (multiples of 2^-16, exact while K <= 341)
//     acc3 = the 4 pairs with i + j = 3     (multiples of 2^-24, exact while K <= 256)
//     acc4 = the 11 pairs with i + j = 4, 5 (magnitude ~2^-32 of acc0)
// The tensor cores add with truncation, so an inexact accumulator drifts by ~2^-23 of
// its own magnitude per addition; keeping every level up to 3 exact confines that drift
// to acc4, ~2^-47 of the result.  The accumulators are drained every 256 K with 32-bit
// conversions only: acc0..acc3 exactly, acc4 rounded to a multiple of 2^-31, summed in
// int64 in units of 2^-31 over the (at most 32) drains of a work item, and then
//     F = round(2^s (acc0 + ... + acc4)),
// with a per-GEMM shift s = 47 - ceil(log2 K) that keeps |F| < 2^62 for K <= 2^23 while
// short contractions keep a resolution far below 2^-46 of the result (for s < 31 only
// the acc4 part is rounded); then
//     L*R = 2^(E_row + E_col - 14 - s) * F.
// Stage-1 results are kept as int64 F (their exponents implied by the operand vectors),
// sliced again for stage 2 with integer shifts only, and stage-2 results are summed as
// int64 with atomics (exact, hence independent of order) before one conversion to
// FP64 per output entry.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "plan.h"

namespace dmrg {

constexpr int SPL_S = 6;          // digit slices per operand
constexpr int SPL_PAIRS = 21;     // slice pairs (i, j) with i + j <= 5
constexpr int SPL_TM = 128;       // MMA tile rows (M)
constexpr int SPL_TN = 64;        // MMA tile columns (N)
constexpr int SPL_TK = 32;        // K per tile (two K=16 MMAs)
constexpr int SPL_LT = SPL_TM * SPL_TK;   // bf16 elements per L slice tile
constexpr int SPL_RT = SPL_TN * SPL_TK;   // bf16 elements per R slice tile
constexpr int SPL_DRAIN_KT = 8;           // K tiles per exact drain (256 K)
constexpr int SPL_ACCS = 5;               // TMEM accumulators (pair levels 0-3 exact, rest)
constexpr int64_t SPL_MAX_K = int64_t(1) << 23;   // longest contraction (s >= 24)
constexpr int SPL_S2_KCHUNK = 256;        // K tiles per stage-2 work item (8192 K)
constexpr int SPL_MAX_DRAINS = 32;        // drains per work item (int64 sums of the epilogue)

// One split GEMM: D (M x N) = L (M x K) * R (K x N) over kt K tiles.  L and R are
// sliced tile arrays (buffer 0 = operator slices, 1 = per-apply slices); tile (mt, kt)
// of L holds the 5 slices of rows [128 mt, +128) x K [32 kt, +32) contiguously.
struct SGemm {
    int64_t l_tiles, r_tiles;   // bf16 element offsets of tile (0, 0)
    int64_t d_off;              // int64 element offset of D (stage-1 scratch or stage-2 sums)
    int32_t l_buf, r_buf;
    int32_t M, N, ldd, kt;
    int32_t kind;               // 0: store sign*F (stage 1), 1: atomic add (stage 2)
    int32_t sign;
    int32_t fshift;             // s: F = round(2^s * accumulated slice sums)
    int32_t x2_period;          // stage 1: entry (r, col) feeds stage-2 vector
    int32_t x2_colgroup;        //   (col / x2_colgroup) * x2_period + r % x2_period
    int32_t pad;
    // stage 1: the epilogue raises the exponents of the stage-2 vectors its entries feed,
    //   ap_exp[x2_exp + vector] = max(..., msb(F)+1 + op_exp[er_off + r]
    //                                 + ap_exp[ec_off + col] - (14 + s))
    int64_t x2_exp, er_off, ec_off;
};

struct SWork { int32_t gemm, mtile, ntile, k0, k1, pad; };

// A contraction run of a sliced operand: nt sub-blocks of kc entries.  Vector v of the
// operand splits into (vg, vr) = (v / vper, v % vper) -- the stacked Davidson vector
// and the row or column inside it -- and entry k of sub-block t is at
//     off + t*ts + vg*vgs + vr*vs + k*ks
// in its source space.  For int64 sources (stage-1 results F) the entry is F * 2^e with
//     e = op_exp[er_off + t*er_ts + vr] + ap_exp[ec_off + vg*ec_vgs + k] - e_off.
struct SSeg {
    int64_t off, ts, vs, ks, vgs;
    int64_t er_off, ec_off;
    int32_t space, kc, nt, er_ts;
    int32_t is_i64, e_off, vper, ec_vgs;
    int32_t kbase, pad;   // first K index of the run inside its job
};

// Slice one operand: vectors [0, npad) (valid below nvalid) along K [0, kt*32) (valid
// below K), rows_tile vectors per tile (128 for L, 64 for R).
struct SJob {
    int64_t out_tiles;   // bf16 element offset in the output slice buffer
    int64_t out_exp;     // int32 offset in the output exponent buffer
    int32_t out_buf, rows_tile;
    int32_t nvalid, npad, K, kt;
    int32_t seg0, nseg;
};

// Rows (term t, vector v) of one segment of one job.
struct SSlab { int64_t rows; int32_t job, seg, kbase, pad; };
// A run of up to SPL_ROWS_PER_ITEM rows of one slab, the unit of work of the slicer.
struct SItem { int64_t r0; int32_t slab, nrows; };
constexpr int SPL_ROWS_PER_ITEM = 64;
// Output tile of the digit pass: vectors [8 vg, 8 vg + 8) x K [k0, k0 + SPL_TILE_K) of one
// job; seg is the job's segment that holds K index k0.
struct STile { int32_t job, vg, k0, seg; };
constexpr int SPL_TILE_K = 256;

// Output block of the wave function and the stage-2 sums that land on it.  Entry (i, j)
// of Davidson vector v is F[(v*rstack + i)*ld + v*cstack + j] with row exponent
// [er_off + v*rstack + i] and column exponent [ec_off + v*cstack + j] (vectors stack
// along the rows of A-first sums and along the columns of B-first sums).
struct SBlock { int64_t y_off; int32_t rows, cols, p0, np; };
struct SPart {
    int64_t acc_off, er_off, ec_off;
    int32_t er_buf, ec_buf, e_off, ld, rstack, cstack;
};

// Host-side split plan.
struct SplitHost {
    std::vector<SGemm> gemms;
    std::vector<SSeg> segs;
    std::vector<SJob> jobs;
    std::vector<SWork> w1, w2;
    std::vector<std::pair<int32_t, int32_t>> r1, r2;   // per-GEMM ranges of w1 / w2 (per_gemm)
    std::vector<SBlock> blocks;
    std::vector<SPart> parts;
    std::vector<SSlab> slabs;
    std::vector<SItem> items;   // [operator items | x items | intermediate items] (exponent pass)
    int64_t it_op0 = 0, it_x0 = 0, it_mid0 = 0, it_end = 0;
    std::vector<STile> tiles;   // [operator tiles | x tiles | intermediate tiles] (digit pass)
    int64_t tl_op0 = 0, tl_x0 = 0, tl_mid0 = 0, tl_end = 0;
    int64_t op_sl = 0, op_ex = 0, ap_sl_vs = 0, ap_ex_vs = 0, s1_vs = 0, s2_vs = 0;
    int nv = 1;   // Davidson vectors stacked in this plan
};

int64_t cdiv(int64_t a, int64_t b);
int32_t fshift_for(int64_t K);
int build_split_plan(const Plan& P, int nv, SplitHost& H, std::string* err, const Schedule& S = Schedule{});
// (Re)builds the work lists w1, w2 (and their per-GEMM ranges) of H from its GEMMs.
void build_split_work(SplitHost& H, const Schedule& S);
int validate_split_plan(const Plan& P, const SplitHost& H, std::string* err);

}  // namespace dmrg
