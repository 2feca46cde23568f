/*
 * dmrg_profile.h -- measurement entry points of libdmrg_gb300: per-kernel timing of
 * the library's own launches and the FP64 tensor-core peak probe that serves as the
 * roofline denominator of the FP64 path.  The paper has no counterpart; it reports
 * sustained FLOP rates (Performance assessment, Fig. 1) without a kernel breakdown.
 */
#ifndef DMRG_PROFILE_H
#define DMRG_PROFILE_H

#include <stdint.h>

#include "dmrg_heff.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    char    name[48];      /* kernel and launch role, e.g. "fp64_tiles/stage1"          */
    int64_t launches;      /* launches since the last reset                              */
    double  ms_total;      /* summed CUDA-event time of those launches (0 if not timed)  */
    double  flops_total;   /* algorithmic flops of those launches (plan count)           */
    double  bytes_total;   /* algorithmic DRAM bytes of those launches                   */
} dmrg_kernel_stat;

/* enable = 1: record a CUDA event pair around every kernel launch of this handle
 * (on the stream the kernel is launched on) and reset the counters; enable = 0:
 * stop timing (launch counts continue).  Timing adds two event records per launch. */
int dmrg_heff_profile(dmrg_heff_t h, int32_t enable);

/* Per-kernel statistics since the last reset.  stats may be NULL to query *n; else
 * it must hold *n entries.  Waits for the recorded events to complete. */
int dmrg_heff_profile_read(dmrg_heff_t h, dmrg_kernel_stat* stats, int32_t* n);

/* Measures the FP64 tensor-core (DMMA mma.sync m16n8k16) throughput of the current
 * device in TFLOP/s: every SM runs independent MMA chains for ~20 ms. */
int dmrg_probe_fp64_peak(double* tflops);

/* Failure-detection self-test: one GPU thread waits, with the same bounded mbarrier wait
 * the slice-GEMM kernel uses, on a barrier that nothing arrives at, for at most
 * wait_cycles SM clock cycles (1 .. 2^34).  Returns DMRG_ERR_DEVICE_TIMEOUT when the wait
 * ran out and the status word was written, as designed; the CUDA context stays usable.
 * The paper has no counterpart. */
int dmrg_selftest_wait_timeout(int64_t wait_cycles);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_PROFILE_H */
