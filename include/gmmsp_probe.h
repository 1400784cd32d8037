/*
 * gmmsp_probe.h - arithmetic-rate probes of the GPU (no counterpart in the
 * paper: a measurement aid for the roofline of the EM kernels, which are
 * bound by FP32 arithmetic and, in the finalize, by FP64).
 *
 * gmmsp_probe_peaks runs short synthetic kernels on the current CUDA device
 * (each a few milliseconds, bounded loops, no waits) and reports measured
 * rates.  It allocates and frees a small device buffer and synchronises the
 * device.  Returns 0 on success, 2 on a CUDA error (message in err, which may
 * be NULL, up to err_len bytes).
 */
#ifndef GMMSP_PROBE_H
#define GMMSP_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int sm_count;                /* multiprocessors                                  */
    int clock_mhz;               /* maximum SM clock reported by the device          */
    double fp32_fma_tflops;      /* FFMA, all SMs, 2 flops per FMA                   */
    double fp64_fma_tflops;      /* DFMA, all SMs, all lanes active                  */
    double fp64_fma_tflops_lane1;/* DFMA with one active lane per warp (lane-flops)  */
    double mufu_ex2_tops;        /* ex2.approx.f32 results per second, x 1e12        */
    double fp32_fma_latency_clk; /* dependent FFMA chain, SM clocks per FMA          */
    double fp64_fma_latency_clk; /* dependent DFMA chain, SM clocks per DFMA         */
    double fp32x2_fma_tflops;    /* packed fma.rn.f32x2 (two FMAs per instruction),
                                    all SMs, 4 flops per instruction                 */
} gmmsp_peaks;

int gmmsp_probe_peaks(gmmsp_peaks *out, char *err, int err_len);

/*
 * gmmsp_probe_smem_patterns launches one short kernel per shared-memory load
 * pattern of the EM kernels (k_lds_pattern<0..9>: warp-uniform 16-, 8- and
 * 4-byte loads, three-address loads, the posterior-row layouts) and
 * synchronises.  It measures nothing itself: run it under a profiler and read
 * the shared-memory wavefronts per load instruction of each kernel.  Returns 0,
 * or 2 on a CUDA error (message in err).
 */
int gmmsp_probe_smem_patterns(char *err, int err_len);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_PROBE_H */
