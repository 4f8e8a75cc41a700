/*
 * cwo_debug.h -- host-only diagnostic entry points of libcwo_gb300.so.
 *
 * They expose the FP64 host computations the plans are built from, so that tests can check them
 * on a machine without a GPU.  None of them touches a device, except cwo_debug_bounded_wait and
 * cwo_debug_ffma_rate (the last two).  They return CWO_ERR_INVALID_ARG on bad arguments (message
 * in cwo_last_error()).
 */
#ifndef CWO_DEBUG_H
#define CWO_DEBUG_H

#include "cwo.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Axis index -> frequency bin (0 .. p-1) for a padded axis of length p (power of two in
 * [32, 8192]).  Index idx = e*(p/16) + t is register e of thread t in the last forward FFT stage,
 * which holds the output at digit-reversed (DIF) position 16 t + e; along x the same index is
 * the storage column of the 2Nx-wide intermediate.  bins: p ints, caller-owned. */
cwo_status cwo_debug_axis_bins(int p, int* bins);

/* Split order of a zero-padded axis of length p (power of two in [64, 8192]): the p-point DFT of
 * p/2 samples x_n is, exactly, the (p/2)-point DFT of x_n at the even frequencies and that of
 * x_n W_p^n at the odd ones.  Split index i = h (p/2) + idx (h = 0: even, 1: odd; idx a
 * (p/2)-point axis index, see cwo_debug_axis_bins) holds frequency 2 bin(idx) + h.  The column
 * pass at p = 8192 with a cached transfer function stores that table's rows in this order.
 * index: p ints, the p-point axis index of the same frequency; phase_ri: p floats, W_p^n =
 * exp(-2 pi i n / p) for n < p/2 (re, im interleaved) rounded from FP64.  Caller-owned; either
 * may be NULL. */
cwo_status cwo_debug_split_axis(int p, int* index, float* phase_ri);

/* The length-p DFT (forward sign, unscaled) of the Fresnel impulse response sampled on the
 * padded axis, h(d) = exp(i pi (d pitch)^2 / (lambda z)), d = i for i < p/2 else i - p
 * (Eq. fre_conv_prop_d, one separable factor), in natural bin order, FP64.
 * out_ri: 2p doubles (re, im interleaved), caller-owned. */
cwo_status cwo_debug_fresnel_axis(int p, double pitch, double lambda, double z, double* out_ri);

/* Inter-stage twiddle table of an axis of length p: one block per radix-16 stage s but the last,
 * of 8 S_s float4 (S_s = L_s / 16, L_s = p / 16^s), holding the pair
 * (W_{L_s}^{j (2kp+1)}, W_{L_s}^{j (2kp+2)}) at [kp][j], kp = 0..7, j = 0..S_s-1; thread t of the
 * FFT reads j = t mod S_s.  out_ri: 4 floats per float4, sum over the blocks (caller-owned). */
cwo_status cwo_debug_twiddles(int p, float* out_ri);

/* ASM per-axis table {a, W - c0, u_hi, u_lo} of an axis of length p (see cwo_cols.cu) in axis
 * index order.  is_x selects the x-axis variant (frac(z/lambda) and the sign of z folded in).
 * out4: 4p floats. */
cwo_status cwo_debug_asm_axis(int p, double pitch, double lambda, double z, int is_x, float* out4);

/* The ASM transfer function H_A of Eq. ang2 on the padded px x py grid, evaluated on the host
 * by the same per-element code and in the same mode as the column pass of an unshifted ASM plan
 * with these parameters (px, py: padded sizes, powers of two in [32, 8192]).  Layout [iy][ix] in
 * axis index order (frequency of index i: cwo_debug_axis_bins).  *mode_out receives the mode:
 * 0 series tail, 1 closed-form tail, 2 per-element FP64.  out_ri: 2 px py floats,
 * caller-owned host memory. */
cwo_status cwo_debug_asm_h(int px, int py, double dx, double dy, double lambda, double z, int* mode_out,
                           float* out_ri);

/* Host emulation of the shifted angular-spectrum plan of cwo_plan_create_shifted (flags 0) for
 * one [ny][nx] complex64 field: the same shifted, windowed per-axis tables and the three passes
 * (adjoint 0/1).  CWO_ERR_UNSUPPORTED where the plan would evaluate its phase per element in
 * FP64.  in_ri, out_ri: 2 nx ny floats each, caller-owned host memory.  Slow. */
cwo_status cwo_debug_emulate_shifted(int nx, int ny, double dx, double dy, double lambda, double z,
                                     const cwo_shift* shift, int adjoint, const float* in_ri, float* out_ri);

/* Host emulation of the shifted Fresnel plan of cwo_plan_create_shifted_fresnel (flags 0) for one
 * [ny][nx] complex64 field: the same tables and the two separable line passes with the source
 * and destination factors of each axis (adjoint 0/1).  in_ri, out_ri: 2 nx ny floats each,
 * caller-owned host memory.  Slow; meant for small fields. */
cwo_status cwo_debug_emulate_shifted_fresnel(int nx, int ny, double dx0, double dy0, double lambda, double z,
                                             const cwo_shifted_fresnel* params, int adjoint, const float* in_ri,
                                             float* out_ri);

/* Host emulation of the CUDA passes for one [ny][nx] complex64 field (same butterflies, stage
 * positions, tables and transfer-function code, executed serially on the CPU): the three passes
 * of the angular spectrum method, the two separable line passes of the Fresnel form.  type is
 * CWO_ANGULAR or CWO_FRESNEL_CONV; flags 0, CWO_FLAG_LITERAL_SCALE (Fresnel) or CWO_FLAG_CACHE_H
 * (angular spectrum: the column pass of a cached transfer function, which at Py = 2 ny = 8192 is
 * the split form of cwo_debug_split_axis); adjoint 0/1.  in_ri and out_ri: 2 nx ny floats each,
 * caller-owned host memory.  Slow; meant for small fields. */
cwo_status cwo_debug_emulate(int nx, int ny, double dx, double dy, double lambda, double z,
                             int type, unsigned flags, int adjoint, const float* in_ri, float* out_ri);

/* Host emulation of one padded line transform of length p.  inverse = 0: forward transform of
 * p/2 natural-order samples (the upper half is the zero padding) into p values in axis-index
 * order.  inverse = 1: adjoint of p axis-index-order values, returning the first p/2 natural-order
 * outputs (unscaled). */
cwo_status cwo_debug_line_fft(int p, int inverse, const float* in_ri, float* out_ri);

/* Failure path of the bounded mbarrier wait that guards every TMA load (device, current CUDA
 * device, synchronous).  One thread initialises an mbarrier for one arrival; with complete = 0 it
 * never arrives, so the wait can only end by its iteration limit: the kernel must then set the
 * timeout bit (1) in a device status word and return.  With complete = 1 it arrives first and
 * the status word stays 0.  spin_limit: polls before giving up, in [1, 2^20].  *status_out
 * receives the status word.  Returns CWO_ERR_CUDA if the launch or a copy fails. */
cwo_status cwo_debug_bounded_wait(unsigned spin_limit, int complete, int* status_out);

/* FP32 issue-rate calibration (device, asynchronous on cuda_stream): `blocks` CTAs of 256
 * threads, each thread running `iters` (a multiple of 8) steps of 16 independent FP32 fused
 * multiply-adds and writing one float to out_dev[blocks * 256] (device memory of the current
 * device).  The caller times the launch: FP32 instructions = blocks * 256 * iters * 16 (2 flops
 * each).  The paper has no counterpart; it is the measured denominator of the FFT passes'
 * arithmetic roofline. */
cwo_status cwo_debug_ffma_rate(int blocks, int iters, float* out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CWO_DEBUG_H */
