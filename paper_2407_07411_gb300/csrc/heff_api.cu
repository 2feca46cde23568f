// C ABI of the library: handle life cycle, device layout of the operators and work
// lists, and the apply entry points.  Every arithmetic step runs in the kernels of
// k_*.cu; this file only validates, allocates, uploads and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "handle.h"
#include "kernels.h"
#include "split.h"

namespace dmrg {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DMRG_ERR_OOM : DMRG_ERR_CUDA;
}

template <class T>
static int upload(const std::vector<T>& v, T** dst, const char* what) {
    *dst = nullptr;
    if (v.empty()) return DMRG_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * v.size());
    if (e != cudaSuccess) return cuda_fail(e, what);
    e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return DMRG_OK;
}

static int dalloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return DMRG_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return DMRG_OK;
}

// Copies the FP64 work lists of the current schedule to the device, growing a buffer
// only when the list outgrew it.
int Handle::upload_fp64_work() {
    auto put = [&](auto& vec, auto** dptr, size_t* cap, const char* what) {
        using T = typename std::remove_reference_t<decltype(vec)>::value_type;
        if (vec.size() > *cap) {
            if (*dptr) cudaFree(*dptr);
            *dptr = nullptr;
            *cap = 0;
            int rc = dalloc(reinterpret_cast<void**>(dptr), sizeof(T) * vec.size(), what);
            if (rc != DMRG_OK) return rc;
            *cap = vec.size();
        }
        if (vec.empty()) return int(DMRG_OK);
        cudaError_t e = cudaMemcpy(*dptr, vec.data(), sizeof(T) * vec.size(), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? int(DMRG_OK) : cuda_fail(e, what);
    };
    int rc;
    if ((rc = put(plan.tiles1, &d_tiles1, &cap_tiles1, "tiles")) != DMRG_OK) return rc;
    if ((rc = put(plan.tiles2, &d_tiles2, &cap_tiles2, "tiles")) != DMRG_OK) return rc;
    if ((rc = put(plan.reduces, &d_red, &cap_red, "reduce jobs")) != DMRG_OK) return rc;
    const size_t part = size_t(plan.n_slots) * fp64_tile_elems(sched.fp64_tile) * size_t(max_nvec);
    if (precision == DMRG_PREC_FP64 && part > cap_part) {
        if (d_part) cudaFree(d_part);
        d_part = nullptr;
        cap_part = 0;
        if ((rc = dalloc(reinterpret_cast<void**>(&d_part), sizeof(double) * part, "partials")) != DMRG_OK) return rc;
        cap_part = part;
    }
    const size_t counters = 2 + plan.ranges1.size() + plan.ranges2.size();
    if (counters > cap_counters) {
        if (d_counters) cudaFree(d_counters);
        d_counters = nullptr;
        cap_counters = 0;
        if ((rc = dalloc(reinterpret_cast<void**>(&d_counters), sizeof(int32_t) * counters, "counters")) != DMRG_OK)
            return rc;
        cap_counters = counters;
    }
    return DMRG_OK;
}

void Handle::drop_graphs() {
    for (GraphEntry& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
}

// Rebuilds the work lists for schedule s (results of every schedule agree: the FP64
// path up to the order of its split-K sums, the split path bit for bit).
int Handle::set_schedule(const Schedule& s) {
    std::string err;
    int rc = check_schedule(s, &err);
    if (rc != DMRG_OK) return fail(rc, err);
    if (!plan_only) {
        cudaError_t e = cudaDeviceSynchronize();   // no apply may still read the old lists
        if (e != cudaSuccess) return cuda_fail(e, "synchronize before rescheduling");
    }
    if ((rc = build_fp64_work(plan, s, &err)) != DMRG_OK) return fail(rc, err);
    sched = s;
    if (precision == DMRG_PREC_SPLIT_BF16 && (rc = split_set_schedule(s)) != DMRG_OK) return rc;
    if (plan_only) return DMRG_OK;
    drop_graphs();
    return upload_fp64_work();
}

Spaces Handle::spaces(const double* x, double* y) const {
    Spaces s;
    s.ops = d_ops; s.x = x; s.scr = d_scr; s.y = y; s.part = d_part;
    s.x_vs = plan.dim; s.y_vs = plan.dim; s.scr_vs = plan.scratch_len;
    s.part_vs = plan.n_slots * fp64_tile_elems(sched.fp64_tile);
    return s;
}

int Handle::apply_fp64(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(y, 0, sizeof(double) * plan.dim * nvec, st);
    if (e != cudaSuccess) return cuda_fail(e, "zero y");
    const size_t n_counters = 2 + plan.ranges1.size() + plan.ranges2.size();
    e = cudaMemsetAsync(d_counters, 0, sizeof(int32_t) * n_counters, st);
    if (e != cudaSuccess) return cuda_fail(e, "zero counters");
    const Spaces sp = spaces(x, y);
    const int shape = sched.fp64_tile, tps = tiles_per_sm[shape];
    const int ctas = sched.fp64_ctas_per_sm > 0 ? std::min(sched.fp64_ctas_per_sm, tps) : tps;
    auto grid_for = [&](size_t n) {
        int64_t items = int64_t(n) * nvec;
        int64_t g = int64_t(n_sm) * ctas;
        return int32_t(items < g ? items : g);
    };
    // one stage: a single persistent launch over its tile list (queue counter 0 for
    // stage 1, 1 for stage 2), or (per_gemm) one launch per GEMM over that GEMM's
    // contiguous tile range (counters 2 .. 2 + #stage-1 GEMMs + #stage-2 GEMMs)
    auto stage = [&](const Tile* d_t, const std::vector<Tile>& tl, const std::vector<std::pair<int32_t, int32_t>>& rg,
                     int32_t* counters) {
        if (!sched.per_gemm)
            return launch_fp64_tiles(d_t, int32_t(tl.size()), d_gemms, d_segs, sp, nvec, counters,
                                     grid_for(tl.size()), st, shape);
        for (size_t r = 0; r < rg.size(); ++r) {
            const int32_t n = rg[r].second - rg[r].first;
            cudaError_t le = launch_fp64_tiles(d_t + rg[r].first, n, d_gemms, d_segs, sp, nvec,
                                               counters + r, grid_for(size_t(n)), st, shape);
            if (le != cudaSuccess) return le;
        }
        return cudaSuccess;
    };
    Profiler::Pending pe;
    if (!plan.tiles1.empty()) {
        prof.begin(kid_s1, st, s1_flops * nvec, s1_bytes * nvec, &pe);
        e = stage(d_tiles1, plan.tiles1, plan.ranges1, sched.per_gemm ? d_counters + 2 : d_counters);
        prof.end(pe, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage-1 tiles");
    }
    if (!plan.tiles2.empty()) {
        prof.begin(kid_s2, st, s2_flops * nvec, s2_bytes * nvec, &pe);
        e = stage(d_tiles2, plan.tiles2, plan.ranges2, sched.per_gemm ? d_counters + 2 + plan.ranges1.size()
                                                                      : d_counters + 1);
        prof.end(pe, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage-2 tiles");
    }
    if (!plan.reduces.empty()) {
        prof.begin(kid_red, st, 0.0, double(plan.reduces.size()) * fp64_tile_elems(shape) * 8.0 * nvec, &pe);
        e = launch_fp64_reduce(d_red, int32_t(plan.reduces.size()), d_gemms, sp, nvec, st, shape);
        prof.end(pe, st);
        if (e != cudaSuccess) return cuda_fail(e, "stage-2 reduce");
    }
    return DMRG_OK;
}

int Handle::apply(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    if (plan_only) return fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    if (nvec < 1 || nvec > max_nvec) return fail(DMRG_ERR_INVALID_ARG, "nvec outside [1, max_nvec]");
    if (plan.dim == 0) return DMRG_OK;
    if (!x || !y) return fail(DMRG_ERR_INVALID_ARG, "null x or y");
    const char* xb = reinterpret_cast<const char*>(x);
    const char* yb = reinterpret_cast<const char*>(y);
    const size_t bytes = sizeof(double) * plan.dim * nvec;
    if (xb < yb + bytes && yb < xb + bytes) return fail(DMRG_ERR_INVALID_ARG, "x and y overlap");
    if (use_graphs && !prof.timing) return apply_graph(x, y, nvec, st);
    return apply_direct(x, y, nvec, st);
}

int Handle::apply_direct(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    if (precision == DMRG_PREC_FP64) return apply_fp64(x, y, nvec, st);
    return apply_split(x, y, nvec, st);
}

// Replays the instantiated graph of this (x, y, nvec), capturing it on the handle's own
// stream first if needed (least recently used graph evicted beyond 64).
int Handle::apply_graph(const double* x, double* y, int32_t nvec, cudaStream_t st) {
    GraphEntry* g = nullptr;
    for (GraphEntry& e : graphs)
        if (e.x == x && e.y == y && e.nvec == nvec) g = &e;
    cudaError_t e;
    if (!g) {
        if (!cap_stream && (e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "capture stream");
        if (graphs.size() >= 64) {
            size_t lru = 0;
            for (size_t i = 1; i < graphs.size(); ++i)
                if (graphs[i].last_use < graphs[lru].last_use) lru = i;
            cudaGraphExecDestroy(graphs[lru].exec);
            graphs.erase(graphs.begin() + lru);
        }
        if ((e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "begin capture");
        prof.counting = false;
        prof.cap_kids.clear(); prof.cap_flops.clear(); prof.cap_bytes.clear();
        const int rc = apply_direct(x, y, nvec, cap_stream);
        prof.counting = true;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap_stream, &graph);
        if (rc != DMRG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        GraphEntry ge{x, y, nvec, nullptr, 0, prof.cap_kids, prof.cap_flops, prof.cap_bytes};
        e = cudaGraphInstantiate(&ge.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
        graphs.push_back(ge);
        g = &graphs.back();
    }
    g->last_use = ++graph_clock;
    if ((e = cudaGraphLaunch(g->exec, st)) != cudaSuccess) return cuda_fail(e, "graph launch");
    for (size_t i = 0; i < g->kids.size(); ++i) {
        prof.launches[g->kids[i]] += 1;
        prof.flops[g->kids[i]] += g->flops[i];
        prof.bytes[g->kids[i]] += g->bytes[i];
    }
    return DMRG_OK;
}

Handle::~Handle() {
    void* ptrs[] = {d_ops, d_scr, d_part, d_tiles1, d_tiles2, d_gemms, d_segs, d_red, d_counters,
                    d_xstage, d_ystage, d_diag_jobs, d_diag};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    release_split();
    release_davidson();
    for (GraphEntry& g : graphs) cudaGraphExecDestroy(g.exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
}

}  // namespace dmrg

using dmrg::Handle;

namespace {

int check_opts(const dmrg_heff_opts* opts, const double* op_data, int64_t op_len, dmrg_heff_opts* o,
               dmrg_heff_t* out) {
    if (!out) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    *o = dmrg_heff_opts{DMRG_PREC_FP64, 0, 1, 0, 0};
    if (opts) *o = *opts;
    if (o->precision != DMRG_PREC_FP64 && o->precision != DMRG_PREC_SPLIT_BF16)
        return dmrg::fail(DMRG_ERR_INVALID_ARG, "unknown precision");
    if (o->max_nvec < 1 || o->max_nvec > 64 || (o->flags & ~(DMRG_FLAG_PLAN_ONLY | DMRG_FLAG_NO_GRAPH)) != 0)
        return dmrg::fail(DMRG_ERR_INVALID_ARG, "max_nvec must be in [1, 64], unknown flags must be 0");
    if (o->n_slices != 0 && o->n_slices != 6)
        return dmrg::fail(DMRG_ERR_UNSUPPORTED, "the split path takes 6 digit slices (n_slices 0 or 6)");
    if (o->split_mid_bytes < 0) return dmrg::fail(DMRG_ERR_INVALID_ARG, "split_mid_bytes must be >= 0");
    if (op_len > 0 && !op_data) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null op_data");
    return DMRG_OK;
}

// Everything after the plan: device operator copy, work lists, precision state, diagonal.
// Takes ownership of h (deleted on failure).
int create_from_plan(Handle* h, const dmrg_heff_opts& o, const double* op_data, dmrg_heff_t* out) {
    int rc = DMRG_OK;
    std::string err;
    h->precision = o.precision;
    h->max_nvec = o.max_nvec;
    h->n_slices = o.n_slices;
    h->split_mid_cap = o.split_mid_bytes;
    h->plan_only = (o.flags & DMRG_FLAG_PLAN_ONLY) != 0;
    h->use_graphs = (o.flags & DMRG_FLAG_NO_GRAPH) == 0;
    if (o.precision == DMRG_PREC_FP64) {
        const dmrg::Plan& P = h->plan;
        dmrg_memory& m = h->mem;
        m.operators = 8 * P.ops_len;
        m.apply_buffers = 8 * int64_t(o.max_nvec) * (P.scratch_len + P.n_slots * dmrg::FP64_BM * dmrg::FP64_BN);
        m.total = m.operators + m.apply_buffers;
    }
    if (h->plan_only) {
        if (o.precision == DMRG_PREC_SPLIT_BF16) {   // host-side split plans, bounds proof, windows
            std::vector<dmrg::SplitHost> hosts;
            std::vector<dmrg::SWindow> win;
            rc = dmrg::build_split_hosts(h->plan, h->max_nvec, h->split_mid_cap, hosts, win, &h->mem, &err);
            if (rc != DMRG_OK) {
                delete h;
                return dmrg::fail(rc, err);
            }
        }
        *out = h;
        return DMRG_OK;
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return dmrg::cuda_fail(e, "cudaGetDevice");
    }
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    for (int sh = 0; sh < dmrg::FP64_SHAPES; ++sh) h->tiles_per_sm[sh] = dmrg::fp64_tiles_per_sm(sh);
    const dmrg::Plan& P = h->plan;
    // Algorithmic work per vector of each stage: flops of the planned order, bytes =
    // operator blocks read once + intermediates written (stage 1) or read (stage 2)
    // + the wave function read (stage 1) or written (stage 2).
    for (const dmrg::Group& G : P.groups) {
        const double n = double(G.terms.size());
        const double a = G.a, b = G.b, c = G.c, d = G.d;
        if (G.order == 0) {
            h->s1_flops += n * 2 * a * b * c; h->s2_flops += n * 2 * a * c * d;
            h->s1_bytes += 8 * n * (a * b + a * c); h->s2_bytes += 8 * n * (a * c + d * c);
        } else {
            h->s1_flops += n * 2 * b * c * d; h->s2_flops += n * 2 * a * b * d;
            h->s1_bytes += 8 * n * (d * c + d * b); h->s2_bytes += 8 * n * (a * b + d * b);
        }
    }
    for (const dmrg::PsiBlock& B : P.blocks) {
        h->s1_bytes += 8.0 * B.rows * B.cols;
        h->s2_bytes += 8.0 * B.rows * B.cols;
    }
    if (o.precision == DMRG_PREC_FP64) {
        h->kid_s1 = h->prof.kernel_id("fp64_tiles/stage1");
        h->kid_s2 = h->prof.kernel_id("fp64_tiles/stage2");
        h->kid_red = h->prof.kernel_id("fp64_reduce");
    }
    auto bail = [&](int code) {
        delete h;
        return code;
    };
    // FP64 handles: the operators in the grouped device layout, streamed through a
    // bounded host buffer (the host never holds a second copy of the operator data).
    // Split handles stream them through the slicer instead and keep only the slices.
    if (P.ops_len > 0 && o.precision == DMRG_PREC_FP64) {
        if ((rc = dmrg::dalloc(reinterpret_cast<void**>(&h->d_ops), sizeof(double) * size_t(P.ops_len),
                               "operators")) != DMRG_OK)
            return bail(rc);
        const size_t cap = size_t(std::min<int64_t>(P.ops_len, int64_t(1) << 25));   // 256 MB
        std::vector<double> stage(cap);
        size_t fill = 0;
        int64_t dst = 0;
        cudaError_t ce = cudaSuccess;
        auto flush = [&]() {
            if (fill > 0 && ce == cudaSuccess)
                ce = cudaMemcpy(h->d_ops + dst, stage.data(), sizeof(double) * fill, cudaMemcpyHostToDevice);
            dst += int64_t(fill);
            fill = 0;
        };
        dmrg::stream_ops(P, op_data, [&](const double* src, int64_t n, double scale) {
            while (n > 0) {
                const int64_t k = std::min<int64_t>(n, int64_t(cap - fill));
                for (int64_t e = 0; e < k; ++e) stage[fill + size_t(e)] = scale * src[e];
                fill += size_t(k);
                src += k;
                n -= k;
                if (fill == cap) flush();
            }
        });
        flush();
        if (ce != cudaSuccess) return bail(dmrg::cuda_fail(ce, "operators"));
        if (dst != P.ops_len) return bail(dmrg::fail(DMRG_ERR_BOUNDS, "operator layout size"));
    }
    const size_t nv = size_t(o.max_nvec);
    if ((rc = dmrg::upload(P.gemms, &h->d_gemms, "gemms")) != DMRG_OK) return bail(rc);
    if ((rc = dmrg::upload(P.segs, &h->d_segs, "segments")) != DMRG_OK) return bail(rc);
    if ((rc = h->upload_fp64_work()) != DMRG_OK) return bail(rc);
    if (o.precision == DMRG_PREC_FP64) {
        if ((rc = dmrg::dalloc(reinterpret_cast<void**>(&h->d_scr), sizeof(double) * P.scratch_len * nv,
                               "stage-1 scratch")) != DMRG_OK)
            return bail(rc);
        if ((rc = h->init_diag()) != DMRG_OK) return bail(rc);
    } else {
        if ((rc = h->init_diag()) != DMRG_OK) return bail(rc);
        if ((rc = h->init_split(op_data)) != DMRG_OK) return bail(rc);
    }
    *out = h;
    return DMRG_OK;
}

}  // namespace

extern "C" {

int dmrg_heff_create(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                     int32_t target_n, int32_t target_2sz, const double* coef, const int32_t* delta,
                     const int32_t* parity, const int64_t* a_off, const int64_t* b_off,
                     int64_t n_terms, const double* op_data, int64_t op_len,
                     const dmrg_heff_opts* opts, dmrg_heff_t* out) {
    dmrg_heff_opts o;
    int rc = check_opts(opts, op_data, op_len, &o, out);
    if (rc != DMRG_OK) return rc;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return dmrg::fail(DMRG_ERR_OOM, "host allocation");
    std::string err;
    rc = dmrg::build_plan(left, nl, right, nr, target_n, target_2sz, coef, delta, parity, a_off, b_off, n_terms,
                          op_len, h->plan, &err);
    if (rc != DMRG_OK) {
        delete h;
        return dmrg::fail(rc, err);
    }
    return create_from_plan(h, o, op_data, out);
}

int dmrg_heff_create_su2(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr, int32_t target_n,
                         int32_t target_2s, const double* coef, const int32_t* rank2, const int32_t* dn,
                         const int32_t* parity, int64_t n_terms, const int64_t* a_blocks, int64_t n_a,
                         const int64_t* b_blocks, int64_t n_b, const double* op_data, int64_t op_len,
                         const dmrg_heff_opts* opts, dmrg_heff_t* out) {
    dmrg_heff_opts o;
    int rc = check_opts(opts, op_data, op_len, &o, out);
    if (rc != DMRG_OK) return rc;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return dmrg::fail(DMRG_ERR_OOM, "host allocation");
    std::string err;
    rc = dmrg::build_plan_su2(left, nl, right, nr, target_n, target_2s, coef, rank2, dn, parity, n_terms, a_blocks,
                              n_a, b_blocks, n_b, op_len, h->plan, &err);
    if (rc != DMRG_OK) {
        delete h;
        return dmrg::fail(rc, err);
    }
    return create_from_plan(h, o, op_data, out);
}

int dmrg_su2_recoupling(int32_t two_sl_out, int32_t two_sr_out, int32_t two_sl_in, int32_t two_sr_in,
                        int32_t two_k, int32_t two_s, double* w) {
    const int32_t a[6] = {two_sl_out, two_sr_out, two_sl_in, two_sr_in, two_k, two_s};
    if (!w) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null output");
    for (int i = 0; i < 6; ++i)
        if (a[i] < 0 || a[i] > (i == 5 ? 2 : 1) * dmrg::SU2_MAX_TWO_S)
            return dmrg::fail(DMRG_ERR_INVALID_ARG, "spin outside [0, 20] (total spin [0, 40])");
    *w = dmrg::su2_recoupling(two_sl_out, two_sr_out, two_sl_in, two_sr_in, two_k, two_s);
    return DMRG_OK;
}

int64_t dmrg_heff_dim(dmrg_heff_t h) { return h ? static_cast<Handle*>(h)->plan.dim : -1; }

int dmrg_heff_flops(dmrg_heff_t h, int64_t* flops) {
    if (!h || !flops) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    *flops = static_cast<Handle*>(h)->plan.flops;
    return DMRG_OK;
}

int dmrg_heff_memory(dmrg_heff_t h, dmrg_memory* m) {
    if (!h || !m) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    *m = static_cast<Handle*>(h)->mem;
    return DMRG_OK;
}

int dmrg_heff_plan_dump(dmrg_heff_t h, int64_t* buf, int64_t* n_rows) {
    if (!h || !n_rows) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null argument");
    const auto& c = static_cast<Handle*>(h)->plan.canon;
    const int64_t rows = int64_t(c.size() / 5);
    if (buf) {
        if (*n_rows < rows) return dmrg::fail(DMRG_ERR_INVALID_ARG, "plan buffer too small");
        std::memcpy(buf, c.data(), sizeof(int64_t) * c.size());
    }
    *n_rows = rows;
    return DMRG_OK;
}

int dmrg_heff_apply(dmrg_heff_t h, const double* x, double* y, int32_t nvec, void* stream) {
    if (!h) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null handle");
    return static_cast<Handle*>(h)->apply(x, y, nvec, static_cast<cudaStream_t>(stream));
}

int dmrg_heff_apply_host(dmrg_heff_t hh, const double* x, double* y, int32_t nvec) {
    if (!hh) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null handle");
    Handle* h = static_cast<Handle*>(hh);
    if (h->plan_only) return dmrg::fail(DMRG_ERR_INVALID_ARG, "plan-only handle");
    if (nvec < 1 || nvec > h->max_nvec) return dmrg::fail(DMRG_ERR_INVALID_ARG, "nvec outside [1, max_nvec]");
    const size_t bytes = sizeof(double) * h->plan.dim * nvec;
    if (bytes == 0) return DMRG_OK;
    if (!x || !y) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null x or y");
    int rc;
    if (!h->d_xstage) {
        const size_t full = sizeof(double) * h->plan.dim * h->max_nvec;
        if ((rc = dmrg::dalloc(reinterpret_cast<void**>(&h->d_xstage), full, "x staging")) != DMRG_OK) return rc;
        if ((rc = dmrg::dalloc(reinterpret_cast<void**>(&h->d_ystage), full, "y staging")) != DMRG_OK) return rc;
    }
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMemcpyAsync(h->d_xstage, x, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "copy x to device");
    if ((rc = h->apply(h->d_xstage, h->d_ystage, nvec, st)) != DMRG_OK) return rc;
    e = cudaMemcpyAsync(y, h->d_ystage, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "copy y to host");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return dmrg::cuda_fail(e, "apply_host synchronize");
    return h->check_status();
}

int dmrg_heff_diagonal(dmrg_heff_t h, double* diag, void* stream) {
    if (!h) return dmrg::fail(DMRG_ERR_INVALID_ARG, "null handle");
    return static_cast<Handle*>(h)->diagonal(diag, static_cast<cudaStream_t>(stream));
}

void dmrg_heff_destroy(dmrg_heff_t h) { delete static_cast<Handle*>(h); }

const char* dmrg_strerror(int code) {
    switch (code) {
        case DMRG_OK: return "ok";
        case DMRG_ERR_INVALID_ARG: return "invalid argument";
        case DMRG_ERR_SECTOR_MISMATCH: return "sector mismatch";
        case DMRG_ERR_OOM: return "out of memory";
        case DMRG_ERR_CUDA: return "CUDA error";
        case DMRG_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case DMRG_ERR_NOT_CONVERGED: return "not converged";
        case DMRG_ERR_BOUNDS: return "out-of-bounds access detected";
        case DMRG_ERR_UNSUPPORTED: return "unsupported option";
        default: return "unknown error code";
    }
}

const char* dmrg_last_error(void) { return dmrg::g_last_error.c_str(); }

}  // extern "C"
