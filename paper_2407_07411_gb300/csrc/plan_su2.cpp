// Host planner of the spin-adapted (SU(2)) two-site H_eff*psi.
//
// Sectors are (n, S) multiplets, operators rank-k irreducible tensors given by their
// reduced blocks (Clebsch-Gordan-normalised Wigner-Eckart convention), and term t is
// c_t sum_mu (-1)^{k-mu} T_mu U_-mu times the parity sign.  On the reduced wave function
// of total spin S every (term, A block [q_L' <- q_L], B block [q_R' <- q_R]) whose input
// and output sector pairs couple to S contributes
//     y[q_L', q_R'] += c_t s_t W A x[q_L, q_R] B^T,
//     W = (-1)^{S_L + S_R' + k + S} sqrt((2S_L' + 1)(2S_R' + 1)) {S_L' S_L k; S_R S_R' S},
// the 6j form of the scalar-product recoupling (Edmonds, Angular Momentum in Quantum
// Mechanics, the reduction of a coupled tensor product of rank 0).  Contributions are
// grouped per (input block, output block): every term of a group shares the block
// shapes, and c_t s_t W is folded into its stacked A copy, so the work lists and the
// kernels are those of the U(1) path.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <utility>

#include "../../include/dmrg_heff.h"
#include "plan.h"

namespace dmrg {
namespace {

bool triangle(int a2, int b2, int c2) { return std::abs(a2 - b2) <= c2 && c2 <= a2 + b2 && (a2 + b2 + c2) % 2 == 0; }

long double fact(int n) {
    static const std::array<long double, 171> tab = [] {   // initialised once, thread-safe
        std::array<long double, 171> t{};
        t[0] = 1.0L;
        for (int i = 1; i <= 170; ++i) t[size_t(i)] = t[size_t(i - 1)] * i;
        return t;
    }();
    return tab[size_t(n)];
}

// (a+b-c)! (a-b+c)! (-a+b+c)! / (a+b+c+1)!, twice-spin arguments of a triangle
long double tri(int a, int b, int c) {
    return fact((a + b - c) / 2) * fact((a - b + c) / 2) * fact((-a + b + c) / 2) / fact((a + b + c) / 2 + 1);
}

// Wigner 6j symbol {a b c; d e f} by Racah's single sum (twice-spin arguments).
long double six_j(int a, int b, int c, int d, int e, int f) {
    if (!triangle(a, b, c) || !triangle(a, e, f) || !triangle(d, b, f) || !triangle(d, e, c)) return 0.0L;
    const int al[4] = {(a + b + c) / 2, (a + e + f) / 2, (d + b + f) / 2, (d + e + c) / 2};
    const int be[3] = {(a + b + d + e) / 2, (b + c + e + f) / 2, (c + a + f + d) / 2};
    const int t0 = std::max(std::max(al[0], al[1]), std::max(al[2], al[3]));
    const int t1 = std::min(be[0], std::min(be[1], be[2]));
    long double s = 0.0L;
    for (int t = t0; t <= t1; ++t) {
        long double den = 1.0L;
        for (int i = 0; i < 4; ++i) den *= fact(t - al[i]);
        for (int i = 0; i < 3; ++i) den *= fact(be[i] - t);
        s += ((t & 1) ? -1.0L : 1.0L) * fact(t + 1) / den;
    }
    return std::sqrt(tri(a, b, c) * tri(a, e, f) * tri(d, b, f) * tri(d, e, c)) * s;
}

struct Blk {
    int32_t in, out;
    int64_t off;
};

}  // namespace

double su2_recoupling(int sl_out, int sr_out, int sl_in, int sr_in, int k2, int s2) {
    if (!triangle(sl_in, sr_in, s2) || !triangle(sl_out, sr_out, s2) || !triangle(sl_in, k2, sl_out) ||
        !triangle(sr_in, k2, sr_out))
        return 0.0;
    const int e = (sl_in + sr_out + k2 + s2) / 2;   // an integer once the triangles hold
    const long double w = ((e & 1) ? -1.0L : 1.0L) * std::sqrt((long double)(sl_out + 1) * (sr_out + 1)) *
                          six_j(sl_out, sl_in, k2, sr_in, sr_out, s2);
    return double(w);
}

int build_plan_su2(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr, int32_t tn, int32_t t2s,
                   const double* coef, const int32_t* rank2, const int32_t* dn, const int32_t* parity, int64_t T,
                   const int64_t* a_blocks, int64_t n_a, const int64_t* b_blocks, int64_t n_b, int64_t op_len,
                   Plan& P, std::string* err) {
    auto bad = [&](int code, const char* m) {
        *err = m;
        return code;
    };
    if (nl < 0 || nr < 0 || T < 0 || n_a < 0 || n_b < 0 || op_len < 0) return bad(DMRG_ERR_INVALID_ARG, "negative size");
    if ((nl > 0 && !left) || (nr > 0 && !right)) return bad(DMRG_ERR_INVALID_ARG, "null sector table");
    if (T > 0 && (!coef || !rank2 || !dn || !parity)) return bad(DMRG_ERR_INVALID_ARG, "null term array");
    if ((n_a > 0 && !a_blocks) || (n_b > 0 && !b_blocks)) return bad(DMRG_ERR_INVALID_ARG, "null block list");
    if (T > (int64_t(1) << 30)) return bad(DMRG_ERR_INVALID_ARG, "too many terms");
    if (t2s < 0 || t2s > 2 * SU2_MAX_TWO_S) return bad(DMRG_ERR_INVALID_ARG, "target spin out of range");
    for (int side = 0; side < 2; ++side) {
        const int32_t* tab = side ? right : left;
        const int32_t n = side ? nr : nl;
        for (int32_t i = 0; i < n; ++i) {
            if (tab[3 * i + 2] < 1) return bad(DMRG_ERR_INVALID_ARG, "sector dimension < 1");
            if (tab[3 * i + 1] < 0 || tab[3 * i + 1] > SU2_MAX_TWO_S)
                return bad(DMRG_ERR_INVALID_ARG, "sector spin 2S outside [0, 40]");
            if (i > 0 && !(tab[3 * i - 3] < tab[3 * i] || (tab[3 * i - 3] == tab[3 * i] && tab[3 * i - 2] < tab[3 * i + 1])))
                return bad(DMRG_ERR_INVALID_ARG, "sectors not strictly ascending in (n, two_s)");
        }
    }
    for (int64_t t = 0; t < T; ++t) {
        if (parity[t] != 0 && parity[t] != 1) return bad(DMRG_ERR_INVALID_ARG, "parity flag must be 0 or 1");
        if (!(coef[t] == coef[t]) || coef[t] - coef[t] != 0.0) return bad(DMRG_ERR_INVALID_ARG, "non-finite coefficient");
        if (rank2[t] < 0 || rank2[t] > SU2_MAX_TWO_S) return bad(DMRG_ERR_INVALID_ARG, "tensor rank 2k outside [0, 40]");
    }
    P.left.assign(left, left + 3 * nl);
    P.right.assign(right, right + 3 * nr);
    P.nl = nl; P.nr = nr; P.tn = tn; P.t2sz = t2s;
    P.su2 = true;

    // Block lists per term, validated and sorted by (in, out).
    std::vector<std::vector<Blk>> AB[2] = {std::vector<std::vector<Blk>>(size_t(T)), std::vector<std::vector<Blk>>(size_t(T))};
    for (int side = 0; side < 2; ++side) {
        const int64_t* rows = side ? b_blocks : a_blocks;
        const int64_t nrow = side ? n_b : n_a;
        const int32_t* tab = side ? right : left;
        const int32_t n = side ? nr : nl;
        for (int64_t r = 0; r < nrow; ++r) {
            const int64_t t = rows[4 * r], q = rows[4 * r + 1], p = rows[4 * r + 2], off = rows[4 * r + 3];
            if (t < 0 || t >= T || q < 0 || q >= n || p < 0 || p >= n)
                return bad(DMRG_ERR_INVALID_ARG, "block row: term or sector out of range");
            const int32_t shift = side ? -dn[t] : dn[t];
            if (tab[3 * p] != tab[3 * q] + shift || !triangle(tab[3 * q + 1], rank2[t], tab[3 * p + 1]))
                return bad(DMRG_ERR_SECTOR_MISMATCH, "block row: sectors do not match the term's shift and rank");
            const int64_t sz = int64_t(tab[3 * p + 2]) * tab[3 * q + 2];
            if (off < 0 || off > op_len || sz > op_len - off) return bad(DMRG_ERR_INVALID_ARG, "block offset out of range");
            AB[side][size_t(t)].push_back({int32_t(q), int32_t(p), off});
        }
        for (auto& v : AB[side]) {
            std::sort(v.begin(), v.end(), [](const Blk& x, const Blk& y) { return x.in != y.in ? x.in < y.in : x.out < y.out; });
            for (size_t i = 1; i < v.size(); ++i)
                if (v[i].in == v[i - 1].in && v[i].out == v[i - 1].out)
                    return bad(DMRG_ERR_INVALID_ARG, "block row listed twice");
        }
    }

    // Reduced wave-function blocks, in (left, right) sector order.
    std::vector<int32_t> bidx(size_t(nl) * size_t(nr), -1);
    int64_t off = 0;
    for (int32_t i = 0; i < nl; ++i)
        for (int32_t j = 0; j < nr; ++j) {
            if (left[3 * i] + right[3 * j] != tn || !triangle(left[3 * i + 1], right[3 * j + 1], t2s)) continue;
            bidx[size_t(i) * nr + j] = int32_t(P.blocks.size());
            P.blocks.push_back({i, j, left[3 * i + 2], right[3 * j + 2], off});
            off += int64_t(left[3 * i + 2]) * right[3 * j + 2];
        }
    P.dim = off;

    // Items and groups (one group per (input block, output block)).
    std::map<std::pair<int32_t, int32_t>, int32_t> gidx;
    std::vector<std::array<int64_t, 5>> items;
    for (int64_t t = 0; t < T; ++t) {
        for (const Blk& A : AB[0][size_t(t)])
            for (const Blk& B : AB[1][size_t(t)]) {
                const int32_t kin = bidx[size_t(A.in) * nr + B.in], kout = bidx[size_t(A.out) * nr + B.out];
                if (kin < 0 || kout < 0) continue;
                const int64_t a = left[3 * A.out + 2], b = left[3 * A.in + 2], c = right[3 * B.in + 2],
                              d = right[3 * B.out + 2];
                const int64_t fa = 2 * a * b * c + 2 * a * c * d;
                const int64_t fb = 2 * b * c * d + 2 * a * b * d;
                const int32_t order = fa <= fb ? 0 : 1;
                items.push_back({kout, t, kin, order, std::min(fa, fb)});
                const double w = su2_recoupling(left[3 * A.out + 1], right[3 * B.out + 1], left[3 * A.in + 1],
                                                right[3 * B.in + 1], rank2[t], t2s);
                const double s = (parity[t] && (left[3 * A.in] & 1)) ? -1.0 : 1.0;
                auto key = std::make_pair(kin, kout);
                auto it = gidx.find(key);
                int32_t g;
                if (it == gidx.end()) {
                    g = int32_t(P.groups.size());
                    gidx[key] = g;
                    Group G;
                    G.dn = dn[t]; G.d2sz = 0; G.parity = 0;
                    G.in_block = kin; G.out_block = kout; G.order = order;
                    G.a = int32_t(a); G.b = int32_t(b); G.c = int32_t(c); G.d = int32_t(d);
                    G.sign = 1.0;
                    P.groups.push_back(G);
                } else {
                    g = it->second;
                }
                Group& G = P.groups[size_t(g)];
                G.terms.push_back(int32_t(t));
                G.a_src.push_back(A.off);
                G.b_src.push_back(B.off);
                G.a_scale.push_back(coef[t] * s * w);
            }
    }
    return finish_plan(P, items, err);
}

}  // namespace dmrg
