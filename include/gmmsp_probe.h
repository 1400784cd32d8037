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
 * gmmsp_probe_fp64_helpers evaluates, for each of the n device doubles x_dev,
 * the FP64 helpers the finalize of the M-step uses instead of FP64 division,
 * square root and logarithm (gmmsp_math.cuh): 1/x and sqrt(x) from an FP32
 * estimate refined by two Newton-Raphson steps, and log2(x) as the exponent
 * plus the FP32 log2 of the mantissa.  Results go to rcp_dev, sqrt_dev
 * (doubles) and log2_dev (floats), n of each, all device memory the caller
 * owns; the kernel is queued on stream (a cudaStream_t) without
 * synchronising.  Inputs must be positive, finite and inside the normal FP32
 * range (the finalize's weights, variances and determinants are).  Returns 0,
 * 1 for NULL pointers or n < 0, 2 on a CUDA launch error (message in err).
 */
int gmmsp_probe_fp64_helpers(const double *x_dev, int n, double *rcp_dev, double *sqrt_dev, float *log2_dev,
                             void *stream, char *err, int err_len);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_PROBE_H */
