// Host-side planner of the two-site H_eff*psi: sector indexing, contraction-order
// choice and the grouped-GEMM work lists that the kernels walk.
//
// Grouping.  All terms with the same shift Delta and parity flag that touch the same
// wave-function block q have identical block shapes (a, b, c, d) and therefore the
// same cheaper contraction order.  Such a group g runs as
//   A-first:  X_g  = s_g [c_t A_t]_t (stacked rows, n_g*a x b) * x_q (b x c)
//             Y_O += sum_t X_{g,t} (a x c) * B_t^T (c x d)      (K = n_g*c)
//   B-first:  Z_g^T = s_g [B_t]_t (stacked rows, n_g*d x c) * x_q^T (c x b)
//             Y_O += sum_t c_t A_t (a x b) * Z_{g,t} (b x d)    (K = n_g*b)
// so stage 1 is one tall GEMM per group and stage 2 one long-K GEMM per output block
// (all groups that land on it), reduced in a fixed order without atomics.
#pragma once
#include <array>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace dmrg {

// Address spaces a descriptor offset refers to.
enum Space : int32_t { SP_OPS = 0, SP_X = 1, SP_SCR = 2, SP_Y = 3, SP_PART = 4 };

// One K-run of a GEMM: nt sub-blocks of kc columns each.  For sub-block t and
// column k (global K index = kbase + t*kc + k):
//   L(i, K) = L[l_off + t*l_ts + i*l_ld + k]
//   R(K, n) = R[r_off + t*r_ts + k*r_ld + n]   (r_trans = 0)
//           = R[r_off + t*r_ts + n*r_ld + k]   (r_trans = 1)
struct Seg {
    int64_t l_off, r_off, l_ts, r_ts;
    int32_t l_space, r_space, l_ld, r_ld;
    int32_t kc, nt, r_trans, pad;
};

// D (M x N, row stride ldd) = alpha * sum over segs [seg0, seg0+nseg) of L*R.
struct Gemm {
    int64_t d_off, K;
    int32_t d_space, ldd, M, N;
    int32_t seg0, nseg;
    double alpha;
};

// One output tile of one GEMM over the K range [k0, k1).  slot < 0: the tile
// stores alpha*acc into D; slot >= 0: it stores acc into partial slot `slot`.
struct Tile {
    int64_t k0, k1;
    int32_t gemm, m0, n0, slot;
};

// D tile = alpha * sum of partial slots [p0, p0+np) in slot order.
struct Reduce {
    int32_t gemm, m0, n0, p0, np, pad;
};

struct PsiBlock { int32_t iL, iR, rows, cols; int64_t off; };

// How the planned GEMMs are cut into work items and launched (what is computed does
// not depend on it).  Stage-2 GEMMs fall into shape classes by contraction length:
// K <= 2048, K <= 16384, longer.
constexpr int N_KCLASS = 3;
inline int kclass(int64_t K) { return K <= 2048 ? 0 : (K <= 16384 ? 1 : 2); }
struct Schedule {
    int32_t fp64_kchunk[N_KCLASS] = {512, 512, 2048};  // K per FP64 stage-2 item (0: whole K)
    int32_t fp64_ctas_per_sm = 0;                      // 0: the occupancy limit
    int32_t split_kchunk[N_KCLASS] = {0, 0, 0};        // K tiles per split stage-2 item (0: adaptive)
    int32_t per_gemm = 0;                              // 1: one launch per grouped GEMM
    int32_t fp64_tile = 0;                             // FP64 output tile shape (FP64_TILE_M/N)
};

struct Group {
    int32_t dn, d2sz, parity;
    int32_t in_block, out_block;
    int32_t order;          // 0 = A-first, 1 = B-first
    int32_t a, b, c, d;
    double sign;            // (-1)^{n_L(in)} for parity groups, else 1
    std::vector<int32_t> terms;
    std::vector<int64_t> a_src, b_src;  // per term: op_data offsets of its A and B blocks
    std::vector<double> a_scale;        // per term: factor of its stacked A copy
    int64_t a_stack = 0, b_stack = 0;   // offsets of the stacked operator copies (device ops)
    int64_t scratch = 0;                // offset of X_g or Z_g^T in the per-vector scratch
};

struct Plan {
    std::vector<int32_t> left, right;   // (n, two_sz, dim) triples
    int32_t nl = 0, nr = 0, tn = 0, t2sz = 0;
    std::vector<PsiBlock> blocks;
    int64_t dim = 0;
    std::vector<int64_t> canon;         // 5 int64 per item, canonical order
    int64_t flops = 0;                  // algorithmic flops per vector
    std::vector<Group> groups;
    std::vector<int32_t> layout;        // groups in operator-layout order (by output block)
    int64_t ops_len = 0;                // doubles in the device operator copy
    int64_t scratch_len = 0;            // doubles of stage-1 intermediates per vector
    // FP64 grouped-GEMM work lists
    std::vector<Seg> segs;
    std::vector<Gemm> gemms;
    std::vector<int32_t> s1gemms, s2gemms;   // GEMM indices of the two stages
    std::vector<Tile> tiles1, tiles2;
    std::vector<Reduce> reduces;
    int64_t n_slots = 0;                // partial slots per vector
    // per-GEMM launch ranges [first, last) into tiles1 / tiles2 (per_gemm schedules)
    std::vector<std::pair<int32_t, int32_t>> ranges1, ranges2;
    int64_t diag_terms = 0;
    bool su2 = false;                   // spin-adapted plan (blocks need not be unique per left sector)
};

// Tile shape of the FP64 kernels (the K extent of stage-2 items is scheduled).
constexpr int FP64_BM = 32, FP64_BN = 32, FP64_BK = 16;   // the default tile (shape 0)
constexpr int FP64_SHAPES = 3;
constexpr int FP64_TILE_M[FP64_SHAPES] = {32, 64, 32}, FP64_TILE_N[FP64_SHAPES] = {32, 32, 64};
inline int fp64_tile_elems(int shape) { return FP64_TILE_M[shape] * FP64_TILE_N[shape]; }   // partial-slot stride

// Validates the inputs and builds the plan; returns 0 or a DMRG_ERR_* code with
// a message in *err.
int build_plan(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
               int32_t tn, int32_t t2sz, const double* coef, const int32_t* delta,
               const int32_t* parity, const int64_t* a_off, const int64_t* b_off,
               int64_t T, int64_t op_len, Plan& P, std::string* err);

// Spin-adapted (SU(2)) plan: sectors are (n, 2S, dim) multiplet tables, terms rank-k
// tensor products coupled to a scalar, blocks rows (term, in, out, offset).  The
// recoupling coefficient of each (term, in block, out block) and the parity sign
// are folded with c_t into the stacked A copies; the work lists are the U(1) ones.
int build_plan_su2(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                   int32_t tn, int32_t t2s, const double* coef, const int32_t* rank2,
                   const int32_t* dn, const int32_t* parity, int64_t T, const int64_t* a_blocks,
                   int64_t n_a, const int64_t* b_blocks, int64_t n_b, int64_t op_len, Plan& P,
                   std::string* err);

// Scalar-coupling recoupling coefficient of the spin-adapted terms (arguments twice
// the spins): <(S_L' S_R') S || sum_mu (-1)^{k-mu} T_mu U_-mu || (S_L S_R) S> for unit
// Clebsch-Gordan-normalised reduced blocks, 0 unless every triangle holds.
double su2_recoupling(int sl_out, int sr_out, int sl_in, int sr_in, int k2, int s2);
constexpr int SU2_MAX_TWO_S = 40;   // spins up to 20 (factorials stay far inside the double range)

// Sorts the items, fills the canonical dump and flop total, lays out the stacked
// operator copies and scratch of P.groups and builds the FP64 work lists.  The stacks
// are laid out output block by output block (groups of one output block in their
// order), so that everything one output block's GEMMs and diagonal read is one
// contiguous range of the layout.
int finish_plan(Plan& P, std::vector<std::array<int64_t, 5>>& items, std::string* err);

// (Re)builds the FP64 tile lists of P for schedule S; returns 0 or DMRG_ERR_INVALID_ARG.
int build_fp64_work(Plan& P, const Schedule& S, std::string* err);
// Checks the ranges of a schedule (not its fit to a plan).
int check_schedule(const Schedule& S, std::string* err);

// Visits the device operator layout in memory order: per group (in P.layout order) its
// stacked scaled A blocks, then its B blocks; sink(src, n, scale) receives n doubles
// to be scaled.
void stream_ops(const Plan& P, const double* op_data,
                const std::function<void(const double*, int64_t, double)>& sink);

}  // namespace dmrg
