// The opaque handle behind dmrg_heff_t.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/dmrg_heff.h"
#include "kernels.h"
#include "plan.h"

struct dmrg_heff {
    virtual ~dmrg_heff() = default;
};

namespace dmrg {

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// One diagonal contribution list entry: block `blk` of the wave function gets
// sign * sum_t A_stack[t][i][i] * B_stack[t][j][j] over the n terms of a group
// whose output block is its input block (A_stack already carries c_t).
struct DiagJob {
    int64_t a_stack, b_stack, off;
    int32_t n, rows, cols, pad;
    double sign;
};

struct SplitState;
struct DavidsonState;

// One instantiated CUDA graph of an apply for a given (x, y, nvec), and the launch
// accounting it stands for.
struct GraphEntry {
    const double* x;
    double* y;
    int32_t nvec;
    cudaGraphExec_t exec;
    uint64_t last_use;
    std::vector<int> kids;
    std::vector<double> flops, bytes;
};

// Launch accounting of one handle: counts, algorithmic flops/bytes and (when
// timing) CUDA-event pairs recorded on the launching stream.
struct Profiler {
    struct Pending { int id; cudaEvent_t start, stop; };
    struct Rec { int id; cudaEvent_t start, stop; };
    std::vector<std::string> names;
    std::vector<int64_t> launches;
    std::vector<double> flops, bytes, ms;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<Rec> recs;
    bool timing = false;
    bool counting = true;            // false while an apply is being captured
    std::vector<int> cap_kids;       // launches seen during a capture
    std::vector<double> cap_flops, cap_bytes;
    int kernel_id(const char* name);
    cudaEvent_t take_event();
    void begin(int id, cudaStream_t st, double f, double b, Pending* p);
    void end(const Pending& p, cudaStream_t st);
    void reset();
    int collect();
    ~Profiler();
};

struct Handle : dmrg_heff {
    Plan plan;
    int precision = 0, max_nvec = 1, n_slices = 0;
    int device = 0, n_sm = 152;
    int tiles_per_sm[FP64_SHAPES] = {8, 8, 8};   // resident FP64 tile CTAs per SM, per tile shape
    bool plan_only = false;
    dmrg_memory mem{};              // device bytes (plan-only handles: what they would hold)
    int64_t split_mid_cap = 0;      // split path: intermediate bytes per output chunk (0: default)
    double* d_ops = nullptr;
    double* d_scr = nullptr;
    double* d_part = nullptr;
    Tile* d_tiles1 = nullptr;
    Tile* d_tiles2 = nullptr;
    Gemm* d_gemms = nullptr;
    Seg* d_segs = nullptr;
    Reduce* d_red = nullptr;
    int32_t* d_counters = nullptr;
    // current schedule and the capacities of the device work lists it fills
    Schedule sched;
    size_t cap_tiles1 = 0, cap_tiles2 = 0, cap_red = 0, cap_part = 0, cap_counters = 0;
    int upload_fp64_work();
    int set_schedule(const Schedule& s);
    int split_set_schedule(const Schedule& s);   // k_split.cu
    void drop_graphs();
    int autotune(int32_t nvec, int32_t reps, dmrg_tune_report* rep);   // autotune.cu
    const struct SplitHost* split_plan_host(int nv) const;             // k_split.cu
    double* d_xstage = nullptr;
    double* d_ystage = nullptr;
    DiagJob* d_diag_jobs = nullptr;
    int32_t n_diag_jobs = 0;
    double* d_diag = nullptr;       // split handles: the diagonal, formed at set-up
    SplitState* split = nullptr;
    DavidsonState* dav = nullptr;
    Profiler prof;
    // CUDA graphs of the apply (DMRG_FLAG_NO_GRAPH disables them)
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    uint64_t graph_clock = 0;
    int apply_graph(const double* x, double* y, int32_t nvec, cudaStream_t st);
    int apply_direct(const double* x, double* y, int32_t nvec, cudaStream_t st);
    int kid_s1 = -1, kid_s2 = -1, kid_red = -1;
    double s1_flops = 0, s2_flops = 0, s1_bytes = 0, s2_bytes = 0;

    ~Handle() override;
    Spaces spaces(const double* x, double* y) const;
    int apply(const double* x, double* y, int32_t nvec, cudaStream_t st);
    int apply_fp64(const double* x, double* y, int32_t nvec, cudaStream_t st);
    int init_diag();
    int diagonal(double* diag, cudaStream_t st);
    // forms the diagonal blocks whose stacks lie in layout entries [lo, hi) from the
    // layout entries held in ops (entry ops_lo first)
    cudaError_t launch_diag(const double* ops, int64_t ops_lo, int64_t lo, int64_t hi, double* diag,
                            cudaStream_t st);
    // split-precision path (k_split.cu): streams the operators window by window through
    // a device staging buffer into the slicer and the diagonal (no resident FP64 copy)
    int init_split(const double* op_data);
    int apply_split(const double* x, double* y, int32_t nvec, cudaStream_t st);
    void release_split();
    // reads and clears the device status word of the split kernels (synchronises)
    int check_status();
    // Davidson (davidson.cu)
    void release_davidson();
};


}  // namespace dmrg
