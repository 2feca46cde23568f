// Launchers of the library's CUDA kernels (device code in k_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "plan.h"

namespace dmrg {

// Base pointers of the address spaces of plan descriptors, with per-vector strides.
struct Spaces {
    const double* ops;
    const double* x;
    double* scr;
    double* y;
    double* part;
    int64_t x_vs, scr_vs, y_vs, part_vs;
};

// Grouped FP64 tile GEMM over `n_tiles` tiles x `nvec` vectors, tiles taken in
// order from the counter at *counter (zeroed by the caller before the launch).
cudaError_t launch_fp64_tiles(const Tile* tiles, int32_t n_tiles, const Gemm* gemms,
                              const Seg* segs, const Spaces& sp, int32_t nvec, int32_t* counter,
                              int32_t grid, cudaStream_t st, int shape = 0);
// Fixed-order sum of split-K partial tiles into their outputs.
cudaError_t launch_fp64_reduce(const Reduce* red, int32_t n_red, const Gemm* gemms,
                               const Spaces& sp, int32_t nvec, cudaStream_t st, int shape = 0);
// Resident CTAs of the tile kernel per SM (occupancy query).
int fp64_tiles_per_sm(int shape = 0);

}  // namespace dmrg
