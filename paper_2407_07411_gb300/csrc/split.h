// Split-precision (Ozaki) path: descriptors shared by the host planner and the kernels.
//
// Arithmetic.  An FP64 operand is cut, per row of the left factor and per column of
// the right factor (a "vector" along the contraction index K), into S = 6 balanced
// base-256 digits relative to an exponent E of the vector (|a| < 2^E for every entry):
//     a = 2^(E-7) * sum_k d_k 2^(-8k),   d_0 in [-128, 128], d_k in [-127, 128],
// rounded after the sixth digit (error <= 2^(E-48)).  Slice k stores the exact BF16
// value d_k 2^(-8k).  A product L*R is the sum of the slice-pair products with
// i + j <= 5 (21 pairs; the dropped pairs weigh <= 2^-48), accumulated on the tensor
// cores in five FP32 accumulators, one per pair level l = i + j up to 3 and one for
// the rest:
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
//
// Exponents.  Operator vectors and the vectors of psi use the exact maximum of their
// entries.  A stage-2 vector of the intermediates (a row of X = A psi_q over all the
// terms and blocks that feed one output block, or a row of Z^T = B psi_q^T) is sliced
// by the epilogue of the stage-1 GEMM that produces it, before the other producers of
// the same vector have run, so its exponent E_V is a bound fixed by an estimate pass
// over the stage-1 GEMMs beforehand.  With a~ = 2^(E_a - 7) d_0(a) the top digit of a
// (|a - a~| <= 2^(E_a - 8) 256/255, the same for x), every entry obeys
//     |X| <= |sum a~ x~| + 1.005 2^-8 (2^E_a sum |x| + sum |a~| 2^E_x),
// where sum a~ x~ is one slice-pair product (pair (0, 0): 1/21 of the MMAs, 1/6 of the
// operand bytes), sum |x| is taken per psi vector and sum |a~| per operator row.  E_V
// is the ceiling of log2 of the largest such bound over the vector (plus a margin for
// the rounding of the stage-1 result); on random data it exceeds the exact maximum's
// exponent by less than one bit.

// Layout.  A sliced operand ("job") is an array of tiles (vector tile vt, K tile kt),
// each holding the 6 slices of rows_tile vectors x 16 K contiguously (UMMA canonical
// K-major layout without swizzle: 8x8 core matrices of 128 bytes, the two K halves of
// an 8-row group adjacent).  L operands have 128-row tiles (the MMA's M), R operands
// 96-row tiles (its N).  Stage-2 contractions run over (term t, index k) with every
// term's run padded to a multiple of 8 (kcp), so that the stage-1 epilogue writes whole
// 16-byte groups of 8 K.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "plan.h"

namespace dmrg {

constexpr int SPL_S = 6;          // digit slices per operand
constexpr int SPL_PAIRS = 21;     // slice pairs (i, j) with i + j <= 5
constexpr int SPL_TM = 128;       // MMA tile rows (M), L tile height
constexpr int SPL_TN = 96;        // MMA tile columns (N, trimmed to a multiple of 16), R tile height
constexpr int SPL_TK = 16;        // K per tile (one K=16 MMA per slice pair)
constexpr int SPL_LT = SPL_TM * SPL_TK;   // bf16 elements per L slice tile
constexpr int SPL_RT = SPL_TN * SPL_TK;   // bf16 elements per R slice tile
constexpr int SPL_DRAIN_KT = 16;          // K tiles per exact drain (256 K)
constexpr int SPL_ACCS = 5;               // TMEM accumulators (pair levels 0-3 exact, rest)
constexpr int64_t SPL_MAX_K = int64_t(1) << 23;   // longest contraction (s >= 24)
constexpr int SPL_S2_KCHUNK = 512;        // K tiles per stage-2 work item (8192 K)
constexpr int SPL_MAX_DRAINS = 32;        // drains per work item (int64 sums of the epilogue)
constexpr int SPL_KPAD = 8;               // stage-2 runs per term padded to this many K
constexpr int32_t SPL_EXP_NONE = -0x1F1F1F20;     // "no exponent" (an all-zero vector); the
                                                  // sum of two stays far above INT_MIN
constexpr int SPL_ROWS_PER_ITEM = 64;
constexpr int SPL_TILE_K = 256;           // K of one work item of the operator digit pass
constexpr int64_t SPL_MID_CAP = int64_t(64) << 30;   // default intermediate bytes per output chunk

inline int32_t kpad(int32_t k) { return (k + SPL_KPAD - 1) / SPL_KPAD * SPL_KPAD; }

// One split GEMM: D (M x N) = L (M x K) * R (K x N) over kt K tiles.  L and R are
// sliced tile arrays (buffer 0 = operator slices, 1 = per-apply slices).
//   kind 1 (stage 2): F added atomically into the int64 sums at d_off (row stride ldd).
//   kind 0 (stage 1): row r = t*per + i, column n = v*cp + k of the product is entry
//     (vector v*per + i, K = kbase + t*cp + k) of the stage-2 job whose tiles start at
//     d_off (rows_tile dst_rows_tile, dst_kt K tiles, vector exponents at dst_exp); the
//     epilogue writes its 6 digits there relative to that vector's bound E_V (at
//     dst_exp + vector in the apply exponents, raised by the estimate pass).
struct SGemm {
    int64_t l_tiles, r_tiles;   // bf16 element offsets of tile (0, 0)
    int64_t d_off;
    int32_t l_buf, r_buf;
    int32_t M, N, kt;
    int32_t kind;
    int32_t sign;
    int32_t fshift;             // s: F = round(2^s * accumulated slice sums)
    int32_t ldd;
    int32_t per, cp, kbase;
    int32_t dst_rows_tile, dst_kt, dst_exp;
    int32_t er_off, ec_off;     // operator row exponents (op_ex), psi vector exponents (ap_ex)
    int32_t chunk;              // output chunk (host-side: the launch it belongs to)
};

struct SWork { int32_t gemm, mtile, ntile, k0, k1, pad; };

// A contraction run of a sliced operator: nt sub-blocks of kc entries, each padded to
// kcp K.  Vector v of the operand splits into (vg, vr) = (v / vper, v % vper) and
// entry k < kc of sub-block t (K = kbase + t*kcp + k) is at
//     off + t*ts + vg*vgs + vr*vs + k*ks
// in the operator data.
struct SSeg {
    int64_t off, ts, vs, ks, vgs;
    int32_t kc, kcp, nt, vper;
    int32_t kbase, pad;
};

// One sliced operand: vectors [0, npad) (valid below nvalid) along K [0, kt*16) (valid
// below K), rows_tile vectors per tile.  Operator jobs (out_buf 0) have segments and
// are sliced once; top_sums marks a stage-1 operator whose digit pass also sums |d_0|
// per row (for the estimate pass, indexed like the exponents).  Per-apply jobs
// (out_buf 1) are psi jobs (sliced by k_xprep) or stage-2 intermediate jobs (written by
// the stage-1 epilogue).
struct SJob {
    int64_t out_tiles;   // bf16 element offset in the output slice buffer
    int64_t out_exp;     // int32 offset in the output exponent buffer
    int32_t out_buf, rows_tile;
    int32_t nvalid, npad, K, kt;
    int32_t seg0, nseg;
    int32_t top_sums;
    int32_t chunk;       // stage-2 intermediate jobs: their output chunk (host-side)
};

// psi operand of the stage-1 GEMMs of one (psi block, contraction side): vector
// v*cp + k (k < nk valid) holds column k of block q of Davidson vector v (side 0,
// contraction over the block's rows) or row k (side 1, over its columns); entry K of
// the vector is x[v*dim + off + K*ks + k*vs].
struct SXJob {
    int64_t off;
    int32_t job;         // its SJob (tiles and exponents)
    int32_t K, nk, cp, ks, vs;
};

// Rows (term t, vector v) of one segment of one operator job.
struct SSlab { int64_t rows; int32_t job, seg, kbase, pad; };
// A run of up to SPL_ROWS_PER_ITEM rows of one slab, the unit of work of the slicer.
struct SItem { int64_t r0; int32_t slab, nrows; };
// Output tile of the operator digit pass: vectors [8 vg, 8 vg + 8) x K [k0, k0 + SPL_TILE_K)
// of one job; seg is the job's segment that holds K index k0.
struct STile { int32_t job, vg, k0, seg; };

// Output block of the wave function and the stage-2 sums that land on it.  Entry (i, j)
// of Davidson vector v is F[(v*rstack + i)*ld + v*cstack + j] with row exponent
// [er_off + v*rstack + i] and column exponent [ec_off + v*cstack + j] (vectors stack
// along the rows of A-first sums and along the columns of B-first sums).
struct SBlock { int64_t y_off; int32_t rows, cols, p0, np; };
struct SPart {
    int64_t acc_off, er_off, ec_off;
    int32_t er_buf, ec_buf, e_off, ld, rstack, cstack;
};

// Host-side split plan for nv stacked Davidson vectors.
struct SplitHost {
    std::vector<SGemm> gemms;
    std::vector<SSeg> segs;
    std::vector<SJob> jobs;
    std::vector<SXJob> xjobs;
    std::vector<SWork> w1, w2;
    std::vector<std::pair<int32_t, int32_t>> r1, r2;   // per-GEMM ranges of w1 / w2 (per_gemm)
    std::vector<SBlock> blocks;
    std::vector<SPart> parts;
    std::vector<SSlab> slabs;   // operator exponent pass
    std::vector<SItem> items;
    std::vector<STile> tiles;   // operator digit pass
    int64_t op_sl = 0, op_ex = 0;                       // operator buffers (the same in every plan)
    int64_t ap_sl_vs = 0, ap_ex_vs = 0, s2_vs = 0;      // per-apply buffers of this plan
    int64_t ap_ex_mid0 = 0, ap_ex_mid1 = 0;             // exponents of the stage-2 intermediate vectors
    int64_t ap_sl_mid0 = 0;                             // first slice entry of the intermediates
    int nv = 1;   // Davidson vectors stacked in this plan
    // Output chunks: runs of output blocks whose stage-2 intermediate slices share one
    // apply space [ap_sl_mid0, ap_sl_vs); an apply runs estimate, stage 1 and stage 2 of
    // one chunk before the next.  Chunk c owns w1[cw1[c], cw1[c+1]), w2[cw2[c],
    // cw2[c+1]) and (per_gemm) the GEMM ranges r1[cr1[c], cr1[c+1]), r2[cr2[c], cr2[c+1]).
    int n_chunks = 1;
    std::vector<int32_t> cw1, cw2, cr1, cr2;
    std::vector<int32_t> block_chunk;   // output chunk of each wave-function block
};

// A range [lo, hi) of the operator layout staged on the device at once while the
// operators are sliced, and the slicer work (items [item0, item1), tiles [tile0,
// tile1) of the first plan) that reads only inside it.
struct SWindow { int64_t lo, hi, item0, item1, tile0, tile1; };

int64_t cdiv(int64_t a, int64_t b);
// Cuts the operator layout [0, P.ops_len) into windows of at most `target` entries
// (longer where one run of overlapping read ranges is longer), never inside a range
// that one operator job of H or one block's diagonal reads, and orders H.items and
// H.tiles window by window.  Returns the longest window, or DMRG_ERR_BOUNDS (negative)
// with *err.
int64_t build_split_windows(const Plan& P, SplitHost& H, int64_t target, std::vector<SWindow>& W,
                            std::string* err);
constexpr int64_t SPL_STAGE_TARGET = int64_t(1) << 28;   // entries per operator window (2 GB)
// The plans for 1 .. max_nvec stacked vectors (hosts[nv - 1]; their operator slices are
// the same), the operator windows of the first, and the device bytes of the split state
// (the staging buffer of one window as the set-up peak).
int build_split_hosts(const Plan& P, int max_nvec, int64_t mid_cap, std::vector<SplitHost>& hosts,
                      std::vector<SWindow>& W, dmrg_memory* mem, std::string* err);
int32_t fshift_for(int64_t K);
// mid_cap: bytes of stage-2 intermediate slices per output chunk (0: SPL_MID_CAP).
int build_split_plan(const Plan& P, int nv, SplitHost& H, std::string* err, const Schedule& S = Schedule{},
                     int64_t mid_cap = 0);
// (Re)builds the work lists w1, w2 (and their per-GEMM ranges) of H from its GEMMs.
void build_split_work(SplitHost& H, const Schedule& S);
int validate_split_plan(const Plan& P, const SplitHost& H, std::string* err);

}  // namespace dmrg
