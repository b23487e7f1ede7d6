/*
 * opta_debug.h -- verification hooks of libopta.so.
 *
 * Each hook runs one preparation kernel of the library in isolation on
 * caller-owned DEVICE buffers so that tests can compare it with a CPU
 * statement of the same step.  They are not needed to search.  All
 * pointers named *_dev are device pointers; the caller owns every buffer.
 * Images are row-major uint8 with stride == cols.  Each hook synchronises
 * `stream` (a cudaStream_t) and returns an opta_status.
 */
#ifndef OPTA_DEBUG_H
#define OPTA_DEBUG_H

#include "opta.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Local statistics (Algorithm 3's Run-Sum S, Q and Omega) of every m x n
 * window of I: inv_sigma_dev[y*(q-n+1)+x] = 1/Omega (0 for a flat window),
 * Omega = sqrt(Q - S^2/mn), from FP64 integral images. */
opta_status opta_dbg_window_stats(const uint8_t *I_dev, int32_t p, int32_t q,
                                  int32_t m, int32_t n, float *inv_sigma_dev,
                                  void *stream);

/* Spatially varying Gaussian blur (Eq. defblur, Eq. Gauss) rounded to the
 * nearest integer: sigma_map_host is ceil(p/block) x ceil(q/block) floats,
 * each 0 or one of the values allowed by opta_params (radius ceil(3 sigma)
 * <= 9, sigma <= 3).  P_dev receives p x q bytes. */
opta_status opta_dbg_blur(const uint8_t *I_dev, int32_t p, int32_t q,
                          const float *sigma_map_host, int32_t block,
                          uint8_t *P_dev, void *stream);

/* Blur correlation R_oo(x) = rho(P window at x, I window at x)
 * (Algorithm 3); R_dev (nullable if fail_dev is given) receives
 * (p-m+1)(q-n+1) floats.  If fail_dev is
 * not null it receives the lambda test (Eq. misDec) per block of
 * block x block locations by top-left (ceil(p/block) x ceil(q/block)
 * int32, row-major): 1 where a window with a non-flat I block has
 * R_oo < lambda, else 0. */
opta_status opta_dbg_blur_corr(const uint8_t *P_dev, const uint8_t *I_dev,
                               int32_t p, int32_t q, int32_t m, int32_t n,
                               float *R_dev, float lambda, int32_t block,
                               int32_t *fail_dev, void *stream);

/* Pivot auto-correlation (Algorithm 1 with the pivot block read from P):
 * rco_dev[x] = rho(P window at the centre of x's group, I window at x) for
 * odd group side h in {1,3,5,7,9}.  rco_dev may be NULL; n_retained_host
 * (nullable) receives #{x : rho_co(x) < rho_cut} (Algorithm 2's count). */
opta_status opta_dbg_rho_co(const uint8_t *P_dev, const uint8_t *I_dev,
                            int32_t p, int32_t q, int32_t m, int32_t n, int32_t h,
                            float *rco_dev, double rho_cut, int64_t *n_retained_host,
                            void *stream);

/* The prepared state of size (m, n) of a handle: pivot_dev (p x q bytes),
 * rho_co_dev (L floats), sigma_map_host (blocks_y x blocks_x floats).
 * Any pointer may be NULL. */
opta_status optA_debug_maps(opta_handle *h, int32_t m, int32_t n,
                            uint8_t *pivot_dev, float *rho_co_dev,
                            float *sigma_map_host, void *stream);

/* Scan 1 alone (Section 6) for n_t (1..128) templates of one size with the
 * handle's precision: rho_dev receives n_t x G floats (template-major;
 * G = groups of that size, row-major over the group grid) holding rho(t,
 * pivot block at each centre); theta_dev (nullable) n_t x G x 2 floats, the
 * angle interval [lo, hi] certain to contain acos of the exact value. */
opta_status optA_debug_scan1(opta_handle *h, const opta_template *t, int32_t n_t,
                             float *rho_dev, float *theta_dev, void *stream);

/* The survivor evaluation of the search (Eq. rho1 at the locations that
 * fail the elimination test of Eq. SEC) at chosen locations: rho_dev[i] and
 * eps_dev[i] (count floats each, device) receive the FP32 rho of template t
 * at location idx_dev[i] (linear index y * (q - n + 1) + x, device int32,
 * each in 0 .. L - 1) and its error bound (|rho - exact| <= eps), computed
 * by survivor form `form`: 0 one lane per location, 1 one warp per
 * location, -1 the form the search takes for this size.  A template whose
 * values are all integers in 0..255 takes the exact integer form of the
 * numerator, any other the FP32 one.  Nothing is skipped.  Prepares the
 * size if needed; synchronises `stream`.  OPTA_ERR_INVALID_ARG for a bad
 * index range, count < 0 or count > L, or form outside -1..1. */
opta_status opta_dbg_survivors(opta_handle *h, const opta_template *t, const int32_t *idx_dev,
                               int64_t count, int32_t form, float *rho_dev, float *eps_dev,
                               void *stream);

/* The survivor-form threshold of an m x n size on the current device: a
 * template (of bytes on the image itself: u8 = 1; any other: u8 = 0) whose
 * survivor sweep has at least *lane_min entries takes the lane form, else the
 * warp form.  *tuned = 1 when the value was measured by the tuner (the
 * first search of the size on this device), 0 for the default rule. */
opta_status opta_dbg_survivor_lane_min(int32_t m, int32_t n, int32_t u8, int32_t *lane_min,
                                       int32_t *tuned);

/* The kernels' int64 -> float conversion (FP32 pipe, no 64-bit conversion
 * instruction) applied to n device values: out_dev[i] = v_dev[i] rounded to
 * the nearest float (ties to even) for |v| < 2^46, within 1 ulp beyond. */
opta_status opta_dbg_i64_to_f32(const int64_t *v_dev, float *out_dev, int64_t n, void *stream);

/* Failure detection of the tensor-core scan 1 (its mbarrier waits are
 * bounded).  Later scan-1 launches give up any wait for progress after
 * `wait_ns` nanoseconds (0 restores the default of 2 s); with `stall` = 1
 * the thread that issues the MMAs first waits on a barrier that no thread
 * ever arrives at, so every launch runs out of its budget.  A launch that
 * gives up still waits (up to 2 s) for its own copies and MMAs in flight,
 * releases its tensor memory and returns; the search then reports
 * OPTA_ERR_TIMEOUT and the handle stays usable.  Process-wide; for tests. */
void opta_dbg_scan1_wait(uint64_t wait_ns, int32_t stall);

/* Number of kernel launches the library has issued in this process. */
uint64_t opta_dbg_launch_count(void);

/* Enable (1) or disable (0) per-kernel timing: every later launch is
 * bracketed by a CUDA event pair recorded on its stream. */
void opta_dbg_profile_enable(int32_t on);

/* Read and clear the timings recorded so far (waits for their events).
 * Writes up to `capacity` entries: kernel name (NUL-terminated, at most
 * name_stride bytes each, into `names`), total milliseconds and launch
 * count.  Returns the number of distinct kernels recorded. */
int32_t opta_dbg_profile_read(char *names, int32_t name_stride, double *total_ms,
                              int64_t *launches, int32_t capacity);

#ifdef __cplusplus
}
#endif

#endif /* OPTA_DEBUG_H */
