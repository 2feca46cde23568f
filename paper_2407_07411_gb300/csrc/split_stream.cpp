// Operator windows of the split path: the FP64 operators are never resident on the
// device as a whole.  Set-up streams the operator layout through one device staging
// buffer, a window at a time, and slices each window (and forms its diagonal blocks)
// before the next one is copied.  A window must therefore hold every entry that its
// slicer work reads: the windows are cut only between the ranges that operator jobs
// (and the diagonal blocks) read, which the output-block-ordered layout keeps short.
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "split.h"

namespace dmrg {

namespace {

struct Span { int64_t lo, hi; };

// The layout range [lo, hi) that an operator job reads (empty for a job without rows).
Span job_span(const SplitHost& H, const SJob& J) {
    Span s{INT64_MAX, INT64_MIN};
    if (J.nvalid == 0) return Span{0, 0};
    for (int sg = J.seg0; sg < J.seg0 + J.nseg; ++sg) {
        const SSeg& g = H.segs[size_t(sg)];
        const int ngrp = (J.nvalid - 1) / g.vper, rmax = std::min(J.nvalid, g.vper) - 1;
        const int64_t last = g.off + (g.nt - 1) * g.ts + ngrp * g.vgs + int64_t(rmax) * g.vs + int64_t(g.kc - 1) * g.ks;
        s.lo = std::min(s.lo, g.off);
        s.hi = std::max(s.hi, last + 1);
    }
    return s;
}

}  // namespace

int64_t build_split_windows(const Plan& P, SplitHost& H, int64_t target, std::vector<SWindow>& W,
                            std::string* err) {
    W.clear();
    if (P.ops_len == 0) return 0;
    // every range some slicer job or diagonal block reads
    std::vector<Span> spans(H.jobs.size(), Span{0, 0});
    std::vector<Span> all;
    for (size_t j = 0; j < H.jobs.size(); ++j) {
        if (H.jobs[j].out_buf != 0) continue;
        spans[j] = job_span(H, H.jobs[j]);
        if (spans[j].hi > spans[j].lo) all.push_back(spans[j]);
    }
    std::vector<Span> diag(P.blocks.size(), Span{INT64_MAX, INT64_MIN});
    for (const Group& G : P.groups) {
        if (G.in_block != G.out_block || G.terms.empty()) continue;
        const int64_t n = int64_t(G.terms.size());
        Span& d = diag[size_t(G.in_block)];
        d.lo = std::min({d.lo, G.a_stack, G.b_stack});
        d.hi = std::max({d.hi, G.a_stack + n * G.a * G.a, G.b_stack + n * G.c * G.c});
    }
    for (const Span& d : diag)
        if (d.hi > d.lo) all.push_back(d);
    std::sort(all.begin(), all.end(), [](const Span& x, const Span& y) { return x.lo < y.lo; });
    // components: maximal unions of overlapping ranges; windows: runs of components
    // (and the gaps between them) of at most `target` entries unless one component is
    // longer, covering the layout [0, ops_len) without gaps
    std::vector<int64_t> cuts{0};
    int64_t comp_lo = -1, comp_hi = -1;
    auto close_component = [&]() {
        if (comp_lo < 0) return;
        if (comp_hi - cuts.back() > target && comp_lo > cuts.back()) cuts.push_back(comp_lo);
    };
    for (const Span& s : all) {
        if (s.lo < 0 || s.hi > P.ops_len) {
            *err = "operator window: read range outside the layout";
            return DMRG_ERR_BOUNDS;
        }
        if (comp_lo >= 0 && s.lo < comp_hi) {
            comp_hi = std::max(comp_hi, s.hi);
            continue;
        }
        close_component();
        comp_lo = s.lo;
        comp_hi = s.hi;
    }
    close_component();
    cuts.push_back(P.ops_len);
    int64_t wmax = 0;
    for (size_t w = 0; w + 1 < cuts.size(); ++w) {
        W.push_back(SWindow{cuts[w], cuts[w + 1], 0, 0, 0, 0});
        wmax = std::max(wmax, cuts[w + 1] - cuts[w]);
    }
    auto window_of = [&](const Span& s) -> int64_t {
        const int64_t w = int64_t(std::upper_bound(cuts.begin(), cuts.end(), s.lo) - cuts.begin()) - 1;
        if (w < 0 || w >= int64_t(W.size()) || s.hi > W[size_t(w)].hi) return -1;
        return w;
    };
    for (size_t k = 0; k < diag.size(); ++k)
        if (diag[k].hi > diag[k].lo && window_of(diag[k]) < 0) {
            *err = "operator window: a diagonal block straddles two windows";
            return DMRG_ERR_BOUNDS;
        }
    // slicer work, window by window (each job's work stays in its original order)
    std::vector<int64_t> jw(H.jobs.size(), -1);
    for (size_t j = 0; j < H.jobs.size(); ++j) {
        if (H.jobs[j].out_buf != 0 || spans[j].hi <= spans[j].lo) continue;
        if ((jw[j] = window_of(spans[j])) < 0) {
            *err = "operator window: a job straddles two windows";
            return DMRG_ERR_BOUNDS;
        }
    }
    auto item_w = [&](const SItem& I) { return jw[size_t(H.slabs[size_t(I.slab)].job)]; };
    auto tile_w = [&](const STile& T) { return jw[size_t(T.job)]; };
    for (const SItem& I : H.items)
        if (item_w(I) < 0) {
            *err = "operator window: slicer item without a window";
            return DMRG_ERR_BOUNDS;
        }
    for (const STile& T : H.tiles)
        if (tile_w(T) < 0) {
            *err = "operator window: slicer tile without a window";
            return DMRG_ERR_BOUNDS;
        }
    std::stable_sort(H.items.begin(), H.items.end(),
                     [&](const SItem& x, const SItem& y) { return item_w(x) < item_w(y); });
    std::stable_sort(H.tiles.begin(), H.tiles.end(),
                     [&](const STile& x, const STile& y) { return tile_w(x) < tile_w(y); });
    size_t i = 0, t = 0;
    for (size_t w = 0; w < W.size(); ++w) {
        W[w].item0 = int64_t(i);
        while (i < H.items.size() && item_w(H.items[i]) == int64_t(w)) ++i;
        W[w].item1 = int64_t(i);
        W[w].tile0 = int64_t(t);
        while (t < H.tiles.size() && tile_w(H.tiles[t]) == int64_t(w)) ++t;
        W[w].tile1 = int64_t(t);
    }
    return wmax;
}

int build_split_hosts(const Plan& P, int max_nvec, int64_t mid_cap, std::vector<SplitHost>& hosts,
                      std::vector<SWindow>& W, dmrg_memory* mem, std::string* err) {
    hosts.assign(size_t(max_nvec), SplitHost{});
    int64_t ap_sl = 0, ap_ex = 0, s2 = 0;
    for (int nv = 1; nv <= max_nvec; ++nv) {
        SplitHost& H = hosts[size_t(nv - 1)];
        const int rc = build_split_plan(P, nv, H, err, Schedule{}, mid_cap);
        if (rc != DMRG_OK) return rc;
        if (H.op_sl != hosts[0].op_sl || H.op_ex != hosts[0].op_ex) {
            *err = "operator slice layout differs between plans";
            return DMRG_ERR_BOUNDS;
        }
        ap_sl = std::max(ap_sl, H.ap_sl_vs);
        ap_ex = std::max(ap_ex, H.ap_ex_vs);
        s2 = std::max(s2, H.s2_vs);
    }
    const int64_t wmax = build_split_windows(P, hosts[0], SPL_STAGE_TARGET, W, err);
    if (wmax < 0) return int(wmax);
    *mem = dmrg_memory{};
    mem->operator_slices = 2 * hosts[0].op_sl + 8 * hosts[0].op_ex + 8 * P.dim;
    mem->apply_buffers = 2 * ap_sl + 8 * ap_ex + 8 * s2 + 4;
    mem->setup_peak = 8 * wmax;
    mem->total = mem->operators + mem->operator_slices + mem->apply_buffers;
    return DMRG_OK;
}

}  // namespace dmrg
