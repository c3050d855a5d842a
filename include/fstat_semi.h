/* Semicoherent stack-slide of coherent 2F over time segments.
 *
 * The paper's Einstein@Home client follows the coherent F-statistic with a
 * semicoherent stage over several data segments (a Hough transform, Section
 * "Einstein@Home"); it prints no algorithm for it.  This is the generic
 * stack-slide form of that stage:
 *
 *   out[sky][m][j] = sum over segments s = 0 .. n_seg-1, in that order, of
 *                    twoF_s[sky][m][i_s(m, j)]                  (FP32 sum)
 *
 * where segment s is a context whose bank is (sky list, f0_s + i df_s for
 * i < n_f_s, spindown list fdot_m) at its reference time t_s, and the
 * semicoherent template (sky, f0 + j df, fdot_m) at t_ref has, at t_s, the
 * frequency f0 + j df + fdot_m (t_s - t_ref).  Its nearest coarse frequency
 * is decided in 32.32 fixed point:
 *
 *   A = ((f0 - f0_s) + fdot_m (t_s - t_ref)) / df_s   (FP64, round to
 *   B = df / df_s                                       nearest, this order)
 *   i_s(m, j) = floor((rint(A 2^32) + j rint(B 2^32) + 2^31) / 2^32)
 *
 * (rint: half to even; integer arithmetic exact).  A lookup with i outside
 * [0, n_f_s) adds nothing and is counted.
 */
#ifndef FSTAT_SEMI_H
#define FSTAT_SEMI_H

#include <stdint.h>

#include "fstat.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FSTAT_SEMI_MAX_SEG 256

/* Sum the segments' 2F along the slid tracks of the semicoherent bank
 * (f0, df, n_f at t_ref; the segments' sky and spindown lists).
 *
 * seg        n_seg contexts (1 .. FSTAT_SEMI_MAX_SEG) on one device, each
 *            after fstat_compute, all with the same sky list and the same
 *            spindown list (compared exactly).  Not modified, except that
 *            seg[0] holds the call's small device scratch.
 * out        DEVICE array of n_sky * n_fdot * n_f floats on that device,
 *            owned by the caller, written in [sky][fdot][f] order.
 * n_outside  host pointer or NULL: the number of (template, segment) lookups
 *            that fell outside a segment's band.  When non-NULL the call
 *            waits for the stream.
 * cuda_stream the stream to run on (NULL: the legacy default stream); the
 *            segments' computes must be ordered before it.
 * Returns FSTAT_OK; FSTAT_EINVAL for null pointers, counts out of range,
 * df / df_s outside [2^-20, 2^20], non-finite grid values, contexts on
 * different devices or with different sky / spindown lists; FSTAT_ESTATE if
 * a segment has not been computed; FSTAT_ECUDA on a CUDA error (the message
 * is in fstat_last_error(seg[0])). */
int fstat_stackslide(fstat_ctx *const *seg, int32_t n_seg, double f0, double df, int32_t n_f, double t_ref,
                     float *out, int64_t *n_outside, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
