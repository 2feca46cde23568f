// Host planner: input validation, sector indexing of the two-site wave function,
// per-(term, block) contraction-order choice by exact integer flop count, grouping
// of terms that share a block, device operator layout and FP64 work lists.
#include "plan.h"

#include <algorithm>
#include <climits>
#include <array>
#include <cstring>
#include <functional>
#include <map>
#include <tuple>

#include "../../include/dmrg_heff.h"

namespace dmrg {
namespace {

struct SectorIndex {
    std::map<std::pair<int32_t, int32_t>, int32_t> idx;
    int find(int32_t n, int32_t s) const {
        auto it = idx.find({n, s});
        return it == idx.end() ? -1 : it->second;
    }
};

int check_table(const int32_t* tab, int32_t n, SectorIndex& si, const char* name, std::string* err) {
    for (int32_t i = 0; i < n; ++i) {
        int32_t q = tab[3 * i], s = tab[3 * i + 1], d = tab[3 * i + 2];
        if (d < 1) {
            *err = std::string(name) + ": sector dimension < 1";
            return DMRG_ERR_INVALID_ARG;
        }
        if (i > 0) {
            int32_t pq = tab[3 * i - 3], ps = tab[3 * i - 2];
            if (!(pq < q || (pq == q && ps < s))) {
                *err = std::string(name) + ": sectors not strictly ascending in (n, two_sz)";
                return DMRG_ERR_INVALID_ARG;
            }
        }
        si.idx[{q, s}] = i;
    }
    return DMRG_OK;
}

}  // namespace

int build_plan(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
               int32_t tn, int32_t t2sz, const double* coef, const int32_t* delta,
               const int32_t* parity, const int64_t* a_off, const int64_t* b_off,
               int64_t T, int64_t op_len, Plan& P, std::string* err) {
    if (nl < 0 || nr < 0 || T < 0 || op_len < 0) {
        *err = "negative size";
        return DMRG_ERR_INVALID_ARG;
    }
    if ((nl > 0 && !left) || (nr > 0 && !right)) {
        *err = "null sector table";
        return DMRG_ERR_INVALID_ARG;
    }
    if (T > 0 && (!coef || !delta || !parity || (nl > 0 && !a_off) || (nr > 0 && !b_off))) {
        *err = "null term array";
        return DMRG_ERR_INVALID_ARG;
    }
    if (T > (int64_t(1) << 30)) {
        *err = "too many terms";
        return DMRG_ERR_INVALID_ARG;
    }
    SectorIndex L, R;
    int rc;
    if ((rc = check_table(left, nl, L, "left", err)) != DMRG_OK) return rc;
    if ((rc = check_table(right, nr, R, "right", err)) != DMRG_OK) return rc;
    P.left.assign(left, left + 3 * nl);
    P.right.assign(right, right + 3 * nr);
    P.nl = nl; P.nr = nr; P.tn = tn; P.t2sz = t2sz;
    auto dl = [&](int i) { return int64_t(left[3 * i + 2]); };
    auto dr = [&](int i) { return int64_t(right[3 * i + 2]); };

    // Operator offsets: each present block must have its output sector and fit.
    for (int64_t t = 0; t < T; ++t) {
        if (parity[t] != 0 && parity[t] != 1) {
            *err = "parity flag must be 0 or 1";
            return DMRG_ERR_INVALID_ARG;
        }
        if (!(coef[t] == coef[t]) || coef[t] - coef[t] != 0.0) {
            *err = "non-finite coefficient";
            return DMRG_ERR_INVALID_ARG;
        }
        const int32_t dn = delta[2 * t], ds = delta[2 * t + 1];
        for (int32_t q = 0; q < nl; ++q) {
            int64_t o = a_off[t * nl + q];
            if (o == -1) continue;
            int p = L.find(left[3 * q] + dn, left[3 * q + 1] + ds);
            if (p < 0) {
                *err = "A block present for a shift whose left output sector is absent";
                return DMRG_ERR_SECTOR_MISMATCH;
            }
            if (o < 0 || o > op_len || dl(p) * dl(q) > op_len - o) {
                *err = "A block offset out of range";
                return DMRG_ERR_INVALID_ARG;
            }
        }
        for (int32_t q = 0; q < nr; ++q) {
            int64_t o = b_off[t * nr + q];
            if (o == -1) continue;
            int p = R.find(right[3 * q] - dn, right[3 * q + 1] - ds);
            if (p < 0) {
                *err = "B block present for a shift whose right output sector is absent";
                return DMRG_ERR_SECTOR_MISMATCH;
            }
            if (o < 0 || o > op_len || dr(p) * dr(q) > op_len - o) {
                *err = "B block offset out of range";
                return DMRG_ERR_INVALID_ARG;
            }
        }
    }

    // Wave-function blocks, ascending in the left sector.
    std::vector<int32_t> block_of_left(nl, -1);
    int64_t off = 0;
    for (int32_t i = 0; i < nl; ++i) {
        int j = R.find(tn - left[3 * i], t2sz - left[3 * i + 1]);
        if (j < 0) continue;
        PsiBlock b{i, j, int32_t(dl(i)), int32_t(dr(j)), off};
        block_of_left[i] = int32_t(P.blocks.size());
        P.blocks.push_back(b);
        off += dl(i) * dr(j);
    }
    P.dim = off;

    // Items and groups.
    std::map<std::tuple<int32_t, int32_t, int32_t, int32_t>, int32_t> gidx;
    std::vector<std::array<int64_t, 5>> items;
    for (int64_t t = 0; t < T; ++t) {
        const int32_t dn = delta[2 * t], ds = delta[2 * t + 1];
        for (int32_t k = 0; k < int32_t(P.blocks.size()); ++k) {
            const PsiBlock& B = P.blocks[k];
            int pL = L.find(left[3 * B.iL] + dn, left[3 * B.iL + 1] + ds);
            int pR = R.find(right[3 * B.iR] - dn, right[3 * B.iR + 1] - ds);
            if (pL < 0 || pR < 0) continue;
            if (a_off[t * nl + B.iL] < 0 || b_off[t * nr + B.iR] < 0) continue;
            const int32_t kout = block_of_left[pL];
            const int64_t a = dl(pL), b = dl(B.iL), c = dr(B.iR), d = dr(pR);
            const int64_t fa = 2 * a * b * c + 2 * a * c * d;
            const int64_t fb = 2 * b * c * d + 2 * a * b * d;
            const int32_t order = fa <= fb ? 0 : 1;
            items.push_back({kout, t, k, order, std::min(fa, fb)});
            auto key = std::make_tuple(dn, ds, parity[t], k);
            auto it = gidx.find(key);
            int32_t g;
            if (it == gidx.end()) {
                g = int32_t(P.groups.size());
                gidx[key] = g;
                Group G;
                G.dn = dn; G.d2sz = ds; G.parity = parity[t];
                G.in_block = k; G.out_block = kout; G.order = order;
                G.a = int32_t(a); G.b = int32_t(b); G.c = int32_t(c); G.d = int32_t(d);
                G.sign = (parity[t] && (left[3 * B.iL] & 1)) ? -1.0 : 1.0;
                P.groups.push_back(G);
            } else {
                g = it->second;
            }
            Group& G = P.groups[g];
            G.terms.push_back(int32_t(t));
            G.a_src.push_back(a_off[t * nl + B.iL]);
            G.b_src.push_back(b_off[t * nr + B.iR]);
            G.a_scale.push_back(coef[t]);
        }
    }
    return finish_plan(P, items, err);
}

int finish_plan(Plan& P, std::vector<std::array<int64_t, 5>>& items, std::string* err) {
    std::sort(items.begin(), items.end());
    P.canon.resize(items.size() * 5);
    P.flops = 0;
    for (size_t i = 0; i < items.size(); ++i) {
        for (int j = 0; j < 5; ++j) P.canon[5 * i + j] = items[i][j];
        P.flops += items[i][4];
    }

    // Device operator layout (output block by output block) and per-vector scratch.
    P.layout.resize(P.groups.size());
    for (size_t g = 0; g < P.groups.size(); ++g) P.layout[g] = int32_t(g);
    std::stable_sort(P.layout.begin(), P.layout.end(),
                     [&](int32_t x, int32_t y) { return P.groups[x].out_block < P.groups[y].out_block; });
    int64_t pos = 0, scr = 0;
    for (int32_t g : P.layout) {
        Group& G = P.groups[g];
        const int64_t n = int64_t(G.terms.size());
        G.a_stack = pos; pos += n * G.a * G.b;
        G.b_stack = pos; pos += n * G.d * G.c;
    }
    for (Group& G : P.groups) {
        const int64_t n = int64_t(G.terms.size());
        G.scratch = scr;
        scr += G.order == 0 ? n * G.a * G.c : n * G.d * G.b;
        if (G.in_block == G.out_block) P.diag_terms += n;
    }
    P.ops_len = pos;
    P.scratch_len = scr;

    // FP64 work lists.  Stage 1: one GEMM per group.
    P.segs.clear(); P.gemms.clear(); P.tiles1.clear(); P.tiles2.clear(); P.reduces.clear();
    std::vector<int32_t> s1gemm;
    for (const Group& G : P.groups) {
        const int32_t n = int32_t(G.terms.size());
        const PsiBlock& B = P.blocks[G.in_block];
        Seg s{};
        Gemm m{};
        if (G.order == 0) {   // X_g = s_g A_stack (n a x b) * x_q (b x c)
            s.l_space = SP_OPS; s.l_off = G.a_stack; s.l_ld = G.b; s.l_ts = 0;
            s.r_space = SP_X; s.r_off = B.off; s.r_ld = G.c; s.r_ts = 0; s.r_trans = 0;
            s.kc = G.b; s.nt = 1;
            m.d_space = SP_SCR; m.d_off = G.scratch; m.ldd = G.c; m.M = n * G.a; m.N = G.c;
            m.K = G.b;
        } else {              // Z_g^T = s_g B_stack (n d x c) * x_q^T (c x b)
            s.l_space = SP_OPS; s.l_off = G.b_stack; s.l_ld = G.c; s.l_ts = 0;
            s.r_space = SP_X; s.r_off = B.off; s.r_ld = G.c; s.r_ts = 0; s.r_trans = 1;
            s.kc = G.c; s.nt = 1;
            m.d_space = SP_SCR; m.d_off = G.scratch; m.ldd = G.b; m.M = n * G.d; m.N = G.b;
            m.K = G.c;
        }
        m.seg0 = int32_t(P.segs.size()); m.nseg = 1; m.alpha = G.sign;
        P.segs.push_back(s);
        s1gemm.push_back(int32_t(P.gemms.size()));
        P.gemms.push_back(m);
    }
    // Stage 2: one GEMM per output block over all its groups.
    std::vector<std::vector<int32_t>> by_out(P.blocks.size());
    for (int32_t g = 0; g < int32_t(P.groups.size()); ++g) by_out[P.groups[g].out_block].push_back(g);
    std::vector<int32_t> s2gemm;
    for (int32_t o = 0; o < int32_t(P.blocks.size()); ++o) {
        if (by_out[o].empty()) continue;
        const PsiBlock& O = P.blocks[o];
        Gemm m{};
        m.d_space = SP_Y; m.d_off = O.off; m.ldd = O.cols; m.M = O.rows; m.N = O.cols;
        m.seg0 = int32_t(P.segs.size()); m.nseg = int32_t(by_out[o].size()); m.alpha = 1.0;
        m.K = 0;
        for (int32_t g : by_out[o]) {
            const Group& G = P.groups[g];
            const int32_t n = int32_t(G.terms.size());
            Seg s{};
            if (G.order == 0) {   // sum_t X_{g,t} (a x c) * B_t^T: R(K,n) = B_t[n][k]
                s.l_space = SP_SCR; s.l_off = G.scratch; s.l_ld = G.c; s.l_ts = int64_t(G.a) * G.c;
                s.r_space = SP_OPS; s.r_off = G.b_stack; s.r_ld = G.c; s.r_ts = int64_t(G.d) * G.c;
                s.r_trans = 1; s.kc = G.c;
            } else {              // sum_t c_t A_t (a x b) * Z_{g,t}: R(K,n) = Z^T[t d + n][k]
                s.l_space = SP_OPS; s.l_off = G.a_stack; s.l_ld = G.b; s.l_ts = int64_t(G.a) * G.b;
                s.r_space = SP_SCR; s.r_off = G.scratch; s.r_ld = G.b; s.r_ts = int64_t(G.d) * G.b;
                s.r_trans = 1; s.kc = G.b;
            }
            s.nt = n;
            m.K += int64_t(s.kc) * n;
            P.segs.push_back(s);
        }
        s2gemm.push_back(int32_t(P.gemms.size()));
        P.gemms.push_back(m);
    }
    P.s1gemms = s1gemm;
    P.s2gemms = s2gemm;
    return build_fp64_work(P, Schedule{}, err);
}

int check_schedule(const Schedule& S, std::string* err) {
    for (int c = 0; c < N_KCLASS; ++c) {
        if (S.fp64_kchunk[c] < 0 || S.fp64_kchunk[c] % FP64_BK || S.fp64_kchunk[c] > (1 << 24)) {
            *err = "schedule: FP64 K chunk must be 0 or a positive multiple of 16";
            return DMRG_ERR_INVALID_ARG;
        }
        if (S.split_kchunk[c] < 0 || S.split_kchunk[c] % 8 || S.split_kchunk[c] > 256) {
            *err = "schedule: split K chunk must be 0 or a multiple of 8 K tiles up to 256";
            return DMRG_ERR_INVALID_ARG;
        }
    }
    if (S.fp64_ctas_per_sm < 0 || S.fp64_ctas_per_sm > 64 || (S.per_gemm != 0 && S.per_gemm != 1) ||
        S.fp64_tile < 0 || S.fp64_tile >= FP64_SHAPES) {
        *err = "schedule: CTAs per SM in [0, 64], per_gemm 0 or 1, fp64_tile 0..2";
        return DMRG_ERR_INVALID_ARG;
    }
    return DMRG_OK;
}

int build_fp64_work(Plan& P, const Schedule& S, std::string* err) {
    int rc = check_schedule(S, err);
    if (rc != DMRG_OK) return rc;
    P.tiles1.clear(); P.tiles2.clear(); P.reduces.clear(); P.ranges1.clear(); P.ranges2.clear();
    const int32_t BM = FP64_TILE_M[S.fp64_tile], BN = FP64_TILE_N[S.fp64_tile];
    for (int32_t gi : P.s1gemms) {
        const Gemm& m = P.gemms[gi];
        for (int32_t m0 = 0; m0 < m.M; m0 += BM)
            for (int32_t n0 = 0; n0 < m.N; n0 += BN) P.tiles1.push_back({0, m.K, gi, m0, n0, -1});
    }
    int64_t slot = 0;
    for (int32_t gi : P.s2gemms) {
        const Gemm& m = P.gemms[gi];
        const int64_t kc = S.fp64_kchunk[kclass(m.K)] > 0 ? S.fp64_kchunk[kclass(m.K)] : m.K;
        const int64_t ns = kc > 0 ? (m.K + kc - 1) / kc : 1;
        for (int32_t m0 = 0; m0 < m.M; m0 += BM)
            for (int32_t n0 = 0; n0 < m.N; n0 += BN) {
                if (ns <= 1) {
                    P.tiles2.push_back({0, m.K, gi, m0, n0, -1});
                    continue;
                }
                P.reduces.push_back({gi, m0, n0, int32_t(slot), int32_t(ns), 0});
                for (int64_t s = 0; s < ns; ++s)
                    P.tiles2.push_back({s * kc, std::min(m.K, (s + 1) * kc), gi, m0, n0, int32_t(slot + s)});
                slot += ns;
                if (slot > INT32_MAX) {   // slot indices are int32 (offsets are formed in int64)
                    *err = "too many partial tiles";
                    return DMRG_ERR_INVALID_ARG;
                }
            }
    }
    P.n_slots = slot;
    // Largest K range first (the kernels take tiles in this order); one launch per GEMM
    // takes each GEMM's tiles as one contiguous range instead.
    auto by_cost = [](const Tile& x, const Tile& y) { return (x.k1 - x.k0) > (y.k1 - y.k0); };
    auto by_gemm = [](const Tile& x, const Tile& y) {
        return x.gemm != y.gemm ? x.gemm < y.gemm : (x.k1 - x.k0) > (y.k1 - y.k0);
    };
    for (int st = 0; st < 2; ++st) {
        std::vector<Tile>& T = st == 0 ? P.tiles1 : P.tiles2;
        if (!S.per_gemm) {
            std::stable_sort(T.begin(), T.end(), by_cost);
            continue;
        }
        std::stable_sort(T.begin(), T.end(), by_gemm);
        auto& R = st == 0 ? P.ranges1 : P.ranges2;
        for (int32_t i = 0; i < int32_t(T.size());) {
            int32_t j = i;
            while (j < int32_t(T.size()) && T[j].gemm == T[i].gemm) ++j;
            R.push_back({i, j});
            i = j;
        }
    }
    return DMRG_OK;
}

void stream_ops(const Plan& P, const double* op_data,
                const std::function<void(const double*, int64_t, double)>& sink) {
    for (int32_t g : P.layout) {
        const Group& G = P.groups[size_t(g)];
        const int64_t na = int64_t(G.a) * G.b, nb = int64_t(G.d) * G.c;
        for (size_t i = 0; i < G.terms.size(); ++i) sink(op_data + G.a_src[i], na, G.a_scale[i]);
        for (size_t i = 0; i < G.terms.size(); ++i) sink(op_data + G.b_src[i], nb, 1.0);
    }
}

}  // namespace dmrg
