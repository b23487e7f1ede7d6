// Internal declarations shared by the CUDA translation units of libopta.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "opta.h"

namespace opta {

// Unit roundoff of binary32.
constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24

// ---------------------------------------------------------------------------
// Group layout (Section 2, Fig. 1): groups of h x h locations tile the
// location grid from (0, 0); the last group along an axis may be cut short;
// its centre is start + (size - 1) / 2.
// ---------------------------------------------------------------------------
__host__ __device__ inline int group_centre_of(int g, int len, int h) {
    const int start = g * h;
    int size = len - start;
    if (size > h) size = h;
    return start + (size - 1) / 2;
}
__host__ __device__ inline int groups_along(int len, int h) { return (len + h - 1) / h; }

// Sum over the m x n window at (y, x) from an inclusive-prefix integral image
// with row pitch q1 = q + 1 (entry (0, *) and (*, 0) zero).  Integer adds:
// exact, and off the GPU's narrow FP64 pipe.
__device__ inline long long ii_box(const long long *__restrict__ II, int64_t q1, int y, int x,
                                   int m, int n) {
    return II[(int64_t)(y + m) * q1 + x + n] - II[(int64_t)y * q1 + x + n]
         - II[(int64_t)(y + m) * q1 + x] + II[(int64_t)y * q1 + x];
}


// int64 -> FP32 on the FP32 pipe.  The 64-bit integer conversion runs on
// the FP64 pipe, which GB300 has little of; here the value is split into
// two 22-bit chunks and a signed top chunk, each converted exactly by the
// magic-number method (an integer c with |c| < 2^22 added to the bit pattern
// of 1.5 * 2^23 gives the float 1.5 * 2^23 + c; Hacker's Delight, 2nd ed.,
// section 17-2), then summed.  The upper sum is exact for |v| < 2^46 (a
// multiple of 2^22 below 2^46 has at most 24 significant bits), so the
// result is v correctly rounded there; beyond, two roundings (< 1 ulp).
__device__ __forceinline__ float i64_to_f32(long long v) {
    constexpr float kMagic = 12582912.f;                            // 1.5 * 2^23
    const unsigned lo = (unsigned)v & 0x3fffffu;                     // bits 0 .. 21
    const unsigned mid = (unsigned)(v >> 22) & 0x3fffffu;            // bits 22 .. 43
    const int hi = (int)(v >> 44);                                   // bits 44 .. 63 (signed)
    const float flo = __uint_as_float(0x4b400000u + lo) - kMagic;
    const float fmid = __uint_as_float(0x4b400000u + mid) - kMagic;
    const float fhi = __int_as_float(0x4b400000 + hi) - kMagic;
    return fmaf(fhi, 17592186044416.f, fmid * 4194304.f) + flo;     // 2^44, 2^22
}

// a * b - c * d exactly, for 32-bit unsigned a, b and 32-bit signed c, d:
// two widening 32 x 32 -> 64 products (no 64 x 64 multiply)
__device__ __forceinline__ long long mul_sub_wide(unsigned a, unsigned b, int c, int d) {
    return (long long)((unsigned long long)a * b) - (long long)c * (long long)d;
}

// mn * Q - S * S (= mn^2 * variance) of a window of mn 8-bit pixels with sum S
// and square sum Q, as FP32.  Exact in int64 up to 2^23 pixels (the product
// stays below 2^62); larger windows take it from FP64 products.
__device__ inline float win_var(long long mn, long long S, long long Q) {
    if (mn <= (1ll << 23)) return i64_to_f32(mn * Q - S * S);
    return (float)((double)mn * (double)Q - (double)S * (double)S);
}

// Order-preserving map of a float to uint32 (larger float -> larger key).
__device__ inline uint32_t float_key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ inline float key_float(uint32_t k) {
    uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// Safety margins of the elimination test (Section 2, Eq. tranEqq in angle form):
// |rho_co(fp32) - rho_co| <= kEcoBound (exact integer numerator, FP32 finish with
// 1/Omega factors of a few ulp each);
// kAngMargin covers acosf and the subtraction of two angles; kCosMargin cosf.
constexpr float kEcoBound = 2e-6f;
constexpr float kAngMargin = 2e-6f;
constexpr float kCosMargin = 2e-6f;

// Angle interval [lo, hi] that certainly contains acos(rho_true) when
// |rho - rho_true| <= e.
__device__ inline float2 angle_interval(float r, float e) {
    return make_float2(acosf(fminf(1.f, r + e)) - kAngMargin,
                       acosf(fmaxf(-1.f, r - e)) + kAngMargin);
}

// Error bounds of scan 1's rho(t, pivot block): e = A * efac + kScan1EpsB,
// efac = ||P - 128|| / sigma_hat of the centre.  bf16 tensor-core form (the
// exhaustive map's, with 2m rows): the hi/lo bf16 split holds t' to 2^-16
// relative and the TMEM FP32 accumulation adds at most 4u per MMA step
// (m * Kp/16 steps); FP32 CUDA-core forms: k roundings per term.
__host__ __device__ inline float scan1_epsA_mma(int m, int Kp) {
    return ((float)(4 * m * (Kp / 16) + 16) * kU32 + 1.55e-5f) * 1.01f;
}
// Scan 1 on the tensor cores in fp16: the template, scaled by a power of
// two s so that s max|t'| lies in [2^13, 2^14), is split into fp16 hi + lo.
// |v - hi| <= 2^-11 |v| and lo rounds v - hi to 2^-11 of itself or, below
// fp16's normal range, to 2^-25 absolute, so the residual is at most
// 2^-22 |v| + 2^-25 per element; summed against P - 128 and divided by
// s sigma_t Omega_hat (s sigma_t >= s max|t'| >= 2^13) that is at most
// (2^-22 + 2^-38 sqrt(mn)) efac, plus 2^-24 for t' rounded once to FP32.
// The FP32 accumulation in TMEM is bounded as for the bf16 form.
__host__ __device__ inline float scan1_epsA_f16(int m, int n, int Kp) {
    const float mn = (float)m * (float)n;
    return ((float)(4 * m * (Kp / 16) + 16) * kU32 + 2.384185791015625e-7f +
            5.9604644775390625e-8f + 3.637978807091713e-12f * sqrtf(mn)) * 1.01f;
}
__host__ __device__ inline float scan1_epsA_fp32(int k) { return (float)(k + 2) * kU32 * 1.01f; }
constexpr float kScan1EpsB = 8.f * kU32;
// roundings per term of the FP32 scan-1 kernels (centre tiles, one column)
__host__ __device__ inline int centre_rho_kacc(int m, int npad) { return 64 + m * ((npad + 63) / 64) + 1; }
// (the column kernel: a lane's chain over its rows, four columns per step,
// two rows per pass when n / 4 <= 16, then the tail column)
__host__ __device__ inline int centre_column_kacc(int m, int n) {
    const int rpp = n / 4 <= 16 ? 2 : 1, gstep = rpp == 2 ? 16 : 32;
    return ((m + rpp - 1) / rpp) * (4 * ((n / 4 + gstep - 1) / gstep) + 1) + 6;
}

// Angle interval certain to contain acos of a centre's exact rho(t, pivot)
// (the largest bound over the kernels that compute centres of the size).
__device__ inline float2 centre_interval(float rho, float efac, float epsA) {
    return angle_interval(rho, fmaf(epsA, efac, kScan1EpsB));
}

// Per-template device state, one per template in flight.
struct TmplState {
    double mu;          // template mean (FP64)
    double sigma;       // sqrt(sum (t - mu)^2) (FP64)
    float inv_sigma;    // 1 / sigma (0 if flat)
    int flat;           // sigma == 0
    // search pipeline
    unsigned int lo_key;      // float_key of the best certain lower bound on max rho
    int n_surv;               // survivors written
    int n_cand;               // candidates written (the first `topk` are threshold centres)
    int n_topk;               // number of threshold centres
    double thr;               // threshold: max exact rho over the threshold centres
    float thr_lo;             // thr rounded down, minus margin (compare in FP32)
    int best_idx;             // final argmax (linear location index)
    double best_rho;          // final rho (FP64)
    int overflow;             // candidate buffer overflowed (status)
    int n_eval;               // survivors evaluated (not skipped by the running threshold)
    float theta_lim;          // survive iff angular gap <= theta_lim (from thr_lo)
    int n_surv_eff;           // survivors past this index are known to be skippable
    int hat_idx;              // literal mode: maximum on the blurred image (-1 otherwise)
    int n_cand_search;        // literal mode: candidates of the search before the re-match
    int dense;                // 1: every location's rho from the tensor-core map, no gathers
    int n_first;              // survivors the first sweep takes (two-phase sweep)
    int u8;                   // every template value an integer in 0..255 (bytes packed)
    int sum_t;                // sum of the template values (exact when u8)
    int int_op;               // exhaustive map: integer operand t - rint(mu) (see brute_mma.cu)
    float c0;                 // rint(mu) - mu when int_op, else 0
    float tscale;             // scan 1's fp16 planes hold t' * tscale (a power of two putting
    float tscale_inv;         // max |t'| in [2^13, 2^14)); and its inverse
    long long sumsq_t;        // sum of the squared template values (exact when u8)
    int grouped;              // scan 2: survivors kept in the bound pass's order (group order)
};

// Floats of one template's slot in a batch: the centred FP32 template (m rows
// of npad = round_up(n, 8)) and then its values as bytes, four to a 32-bit
// word, in rows of tmpl_row_bytes(n) = round_up(n, 32) bytes with zeros past
// column n (written and meaningful only when TmplState::u8).
__host__ __device__ inline int tmpl_row_bytes(int n) { return (n + 31) & ~31; }
__host__ __device__ inline size_t tmpl_slot_floats(int m, int n) {
    return (size_t)m * ((n + 7) & ~7) + (size_t)m * tmpl_row_bytes(n) / 4;
}

// Survivors are bucketed by their upper bound (bucket 0 = highest) so that
// they are evaluated roughly in decreasing bound order.
constexpr int kUbBuckets = 256;
// Templates of at least kGroupOrderMN pixels whose survivors number at most
// a quarter of the count at which their dense map would take over keep the
// survivors in the order the bound pass found them, in one bucket: the
// members of a group sit next to one another, so the windows of a lane-form
// round overlap and share cache lines (4x fewer L2 sectors at 48 x 48).  With
// so few survivors the running lower bound seldom skips one (the threshold
// centres usually hold the maximum already) and cannot tip the template into
// the dense map, so the bound order buys little; other templates keep it.
constexpr long long kGroupOrderMN = 1024;
// Templates per scan-2 launch (their histograms share one block's shared memory).
constexpr int kScan2MaxT = 16;


// Device pointer and row stride of one template of a batch.
struct TmplIn {
    const float *data;
    int64_t ld;
};

// ---------------------------------------------------------------------------
// Launchers (stream-ordered, return cudaError_t of the launch).
// ---------------------------------------------------------------------------
// Integral images (int64, exact; (p+1) x (q+1), zero first row/col) of A, A*A
// and, if B != null and o2 != null, A*B.
cudaError_t launch_integrals(const uint8_t *A, const uint8_t *B, int p, int q, long long *o0,
                             long long *o1, long long *o2, cudaStream_t s);

// inv_sigma[y*Lx+x] = 1/Omega and efac[y*Lx+x] = ||I-128|| / Omega (0 when flat);
// wsum (nullable) = the window sum S (int32: asked for windows of at most 2^23 pixels).
cudaError_t launch_window_stats(const long long *IIS, const long long *IIQ, int p, int q,
                                int m, int n, float *inv_sigma, float *efac128,
                                cudaStream_t s, int *wsum = nullptr);

// out[i] = i64_to_f32(v[i]) (the conversion the kernels use; tested alone).
cudaError_t launch_i64_to_f32(const long long *v, float *out, int64_t n, cudaStream_t s);
// count += number of zeros of the Ly x Lx map x over the rows EGS samples
// for group side h (kEgsRun; every row when sample == 1); not cleared.
cudaError_t launch_count_zero(const float *x, int Ly, int Lx, int h, int sample,
                              unsigned long long *count, cudaStream_t s);

// Convert a float32 image holding integers in [0,255] into uint8; bad = 1 otherwise.
cudaError_t launch_ingest_f32(const float *src, int64_t ld, int p, int q, uint8_t *dst,
                              int *bad, cudaStream_t s);
cudaError_t launch_ingest_u8(const uint8_t *src, int64_t ld, int p, int q, uint8_t *dst,
                             cudaStream_t s);

// Template statistics: tf (m x npad, FP32, zero padded) and td (m x n, FP64) hold t - mu.
cudaError_t launch_tmpl_prep(const float *t, int64_t ld, int m, int n, int npad,
                             float *tf, double *td, TmplState *st, int topk, cudaStream_t s);
// The same for T templates (tin: T device descriptors), outputs at k * tsz / k * dsz / st + k;
// tsz = tmpl_slot_floats(m, n): each slot also receives the packed bytes.
cudaError_t launch_tmpl_prep_batch(const TmplIn *tin, int T, int m, int n, int npad, float *tf,
                                   size_t tsz, double *td, size_t dsz, TmplState *st, int topk,
                                   cudaStream_t s);

// Exhaustive FP32 map (Eq. rho1 with v = I - 128), plus the certain lower bound key.
cudaError_t launch_zncc_map(const uint8_t *I, int p, int q, const float *tf, int m, int n,
                            int npad, const float *inv_sigma, const float *efac128,
                            TmplState *st, float *map, cudaStream_t s);
// Candidates from a full FP32 map: map + eps >= lower bound.
// Error-bound coefficient of the FP32 CUDA-core map: eps = epsA * efac + 8u.
float zncc_map_epsA(int m, int n);
// Candidates: every location whose map value + eps (epsA * efac + 8u) reaches
// the map's certain lower bound on the maximum.
cudaError_t launch_map_candidates(const float *map, const float *efac128, int64_t L, float epsA,
                                  TmplState *st, int *cand, int cap, cudaStream_t s);

// FP64 recomputation of rho at the candidate locations [0, n_cand) of T
// templates (template k: td + k * dsz, st + k, cand / cand_rho + k * ccap).
// With the batch's template slots (tf + k * tsz, nullable), a template of
// bytes takes exact integer sums and an FP64 finish instead.
cudaError_t launch_refine64(const uint8_t *I, int q, int Lx, const double *td, size_t dsz, int m,
                            int n, int T, TmplState *st, const int *cand, double *cand_rho,
                            int64_t ccap, cudaStream_t s, const float *tf = nullptr, size_t tsz = 0,
                            int npad = 0);
// Final argmax over the candidates and threshold centres (nullable; kTopkMax
// per template) of T templates -> st->best_idx / best_rho.
cudaError_t launch_final_argmax(int T, TmplState *st, const int *cand, const double *cand_rho,
                                int64_t ccap, const int *cand_topk, const double *cand_rho_topk,
                                cudaStream_t s);
// Literal mode: candidates := the (2d+1)^2 neighbourhood of best_idx.
cudaError_t launch_rematch_window(int T, TmplState *st, int Ly, int Lx, int d, int *cand,
                                  int64_t ccap, cudaStream_t s);
// FP64 rho at the threshold centres of T templates (kTopkMax slots each);
// tf / tsz / npad as for launch_refine64.
cudaError_t launch_refine64_topk(const uint8_t *I, int q, int Lx, const double *td, size_t dsz,
                                 int m, int n, int T, TmplState *st, const int *cand_topk,
                                 double *cand_rho_topk, cudaStream_t s, const float *tf = nullptr,
                                 size_t tsz = 0, int npad = 0);

// --- pruned search ---
// rho_tc per group and the angle interval of its true value (tc), for the
// group columns gx >= gx_begin (FP32 CUDA cores).
cudaError_t launch_centre_rho(const uint8_t *P, int p, int q, const float *tf, int m, int n,
                              int npad, int h, int Ly, int Lx, const float *c_inv_sigma,
                              TmplState *st, float *rho_tc, int gx_begin, cudaStream_t s);
// Tensor-core scan 1 for T same-size templates (planes of B), see corr_mma.cu.
// B holds corr_mma_bbytes(m, Kp, N, h) bytes: the template planes ((m + 1)
// rows, row m zero) and the per-launch arrangement of them that follows.
size_t corr_mma_bbytes(int m, int Kp, int N, int h);
cudaError_t launch_corr_mma(const uint8_t *V, int p, int q, void *B, int m, int n, int Kp,
                            int N, int h, int Ly, int Lx, int T, const float *c_inv_sigma,
                            const TmplState *st, float *rho_tc, int64_t gstride, int *err,
                            int *Gx_u_out, cudaStream_t s);
// rho_tc of one group column for a chunk of templates (warp per centre).
cudaError_t launch_centre_column(const uint8_t *P, int q, const float *tf, int m, int n, int npad,
                                 size_t tsz, int h, int Ly, int Lx, int gx, int T,
                                 const float *c_inv_sigma, const TmplState *st, float *rho_tc,
                                 int64_t gstride, cudaStream_t s);
// Angle intervals of scan-1 values (verification output): T x G float2.
cudaError_t launch_centre_intervals(const float *rho_tc, int64_t G, int T, const float *c_efac,
                                    float epsA, float2 *out, cudaStream_t s);
cudaError_t launch_tmpl_split(const float *tf, size_t tsz, int T, int m, int n, int npad, int Kp,
                              int N, const TmplState *st, void *B, cudaStream_t s);
// Threshold centres of T templates: rho_tc of template k at k * gstride;
// tmp_val/tmp_idx: T x 256 x kTopkMax; cand_topk: T x kTopkMax.
cudaError_t launch_topk(const float *rho_tc, int64_t gstride, int Gy, int Gx, int h, int Ly, int Lx,
                        int k, int T, TmplState *st, float *tmp_val, int *tmp_idx, int *cand_topk,
                        cudaStream_t s);
cudaError_t launch_threshold(TmplState *st, const double *cand_rho_topk, int T, cudaStream_t s);
// FP32 rho at the members of the threshold centres' groups (raises lo_key).
cudaError_t launch_group_members(const uint8_t *I, int q, int Ly, int Lx, int h, const int *wsum,
                                 const float *tf, size_t tsz, int m, int n,
                                 int npad, const float *inv_sigma, int T, TmplState *st,
                                 const int *cand_topk, int topk, cudaStream_t s);
// Scan 2 of a batch of T same-size templates: per-template arrays, each at
// its own stride.
struct Scan2Batch {
    int T;
    TmplState *st;                       // T states
    const float *rho_tc;                 // scan-1 rho per centre, template k at k * tc_stride
    int64_t tc_stride;
    const float *c_efac;                 // per centre: ||P - 128|| / sigma_hat
    float epsA;                          // scan-1 error bound factor of the size
    const float *tf;                     // FP32 templates (m x npad), k * tsz
    size_t tsz;
    int *surv;                           // survivor lists (bucket order), k * scap
    float *surv_ub, *surv_rho, *surv_eps;
    int64_t scap;
    int *cand;                           // candidates, k * ccap
    int64_t ccap;
    int *ucnt;                           // unordered survivors found, per template
    int *bucket_cnt, *bucket_cur;        // k * kUbBuckets
    float dense_frac;                    // > 0: a template with more survivors left than
                                         // dense_frac * L after its first sweep takes the
                                         // dense map; < 0: any template with a survivor
                                         // left; 0: none (one sweep)
    int64_t first_budget;                // survivors of the first sweep (dense_frac != 0)
    int64_t L;                           // locations per template
    int phase;                           // sweep: 0 all, 1 the first n_first, 2 the rest
    const uint8_t *Ipad;                 // the search image with rows of qs bytes (16-byte
    int qs;                              // aligned), or null: integer survivors path off
    int lane_min_u8, lane_min_f32;       // a template whose sweep has at least this many
                                         // entries takes the lane form, else the warp form
                                         // (templates of bytes on Ipad / all others)
    unsigned long long *span;            // null, or [earliest block start, latest block end]
    int group_order;                     // 1: the size may keep its survivors in group order
                                         // of the sweep kernels (%globaltimer ns): the tuner
};

// Bound of every location against each template's threshold (group test
// on the group union intervals gco first, members of passing groups only),
// bucket histograms of the survivors, then the survivors in bucket order
// with their upper bound.  ub_map / surv_map (nullable; T == 1 only)
// receive the full maps.
cudaError_t launch_bound_compact(const Scan2Batch &B, const float2 *theta_co, const float2 *gco,
                                 int Ly, int Lx, int h, float *ub_map, uint8_t *surv_map,
                                 cudaStream_t s);
// Per group: the union (lowest lo, highest hi) of its members' angle intervals.
cudaError_t launch_group_co(const float2 *theta_co, int Ly, int Lx, int h, float2 *gco,
                            cudaStream_t s);
// Cut of the skippable buckets, then one bound-ordered sweep over the
// survivors of all T templates (FP32 rho, running lower bound per template).
cudaError_t launch_survivors(const Scan2Batch &B, const uint8_t *I, int pimg, int q, int Lx,
                             const int *wsum, int m, int n, int npad, const float *inv_sigma,
                             cudaStream_t s);
cudaError_t launch_surv_candidates(const Scan2Batch &B, cudaStream_t s);
// rho and its error bound at the B.surv[0..count) locations of B's one
// template (B.T == 1, st prepared) by survivor form `form` (0 one lane per
// survivor, 1 one warp, -1 by B's thresholds), none skipped: into
// B.surv_rho / B.surv_eps.
cudaError_t launch_survivor_eval(const Scan2Batch &B, const uint8_t *I, int pimg, int q, int Lx,
                                 const int *wsum, int m, int n, int npad, const float *inv_sigma,
                                 int count, int form, cudaStream_t s);
// Survivor forms: a template's sweep takes the lane form when it has at least
// lane_min entries, the warp form otherwise.  survivor_lane_min gives the
// thresholds of an m x n size on the current device (byte templates on the
// aligned image: u8 = true), measured by the tuner (tuned = true) or from
// the default rule; set_survivor_lane_min records measured ones.
int survivor_lane_min(int m, int n, bool u8, bool *tuned = nullptr);
void set_survivor_lane_min(int m, int n, bool u8, int lane_min);
constexpr int kLaneNever = 0x7fffffff;

// --- preparation ---
// Blur with per-block sigma-level index (uint8 map; level 0 = copy) and weight table.
cudaError_t launch_blur(const uint8_t *I, int p, int q, const uint8_t *level_map, int block,
                        const float *weights /* [levels][10] */, const int *radius,
                        uint8_t *P, cudaStream_t s);
// Blur correlation R_oo per location straight from P and I (I's windows
// from the window-sum and 1/Omega maps); block fail flags where a non-flat
// window has R < lambda.  R (nullable) receives the map.
cudaError_t launch_blur_corr(const uint8_t *P, const uint8_t *I, const int *wsum,
                             const float *inv_sigma, int p, int q, int m, int n, float lambda,
                             int block, int *fail, float *R, cudaStream_t s);
// Whether the auto-correlation kernel can run group side h for m x n windows
// of a p x q image (its strip of window columns and ring of image rows must
// fit the thread and shared-memory limits).
bool rho_co_supported(int p, int q, int m, int n, int h);
// EGS counts (Algorithm 2's n_r) over a systematic sample of the location
// grid: the group rows g (of side h) with (g / kEgsRun) % sample == 0, in
// runs of kEgsRun group rows; sample = 1 counts every location.
constexpr int kEgsRun = 8;
// Pivot auto-correlation map (rco, nullable) / retained count (count,
// nullable) for odd group side h.  The member windows' statistics come from
// the window-sum and 1/Omega maps of I, the centres' from the pivot itself;
// c_inv_sigma / c_efac (nullable) receive the centres' 1/sigma_hat and
// ||P - 128|| / sigma_hat for scan 1.  With sample > 1 only the count is
// taken, over the sampled group rows (rco, c_inv_sigma and c_efac null).
cudaError_t launch_rho_co(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                          int h, const int *wsum, const float *inv_sigma, float cut, float *rco,
                          unsigned long long *count, float *c_inv_sigma, float *c_efac,
                          cudaStream_t s, int sample = 1);
// Angle intervals of the pivot auto-correlation map (kEcoBound wide).
cudaError_t launch_theta_co(const float *rho_co, int64_t L, float2 *theta_co, cudaStream_t s);

// Device buffers of one exhaustive search (zncc_full and its no-allocation
// variant): integral images ((p+1)(q+1) each), per-location 1/Omega and
// error factor, the rho map and the candidate indices (L each), their FP64
// rho (L), the template as FP32 rows padded to a multiple of 8 columns and
// as FP64 (m n), and its state.  With Ipad (p x round_up(q, 16) bytes), Bt
// (brute_tmpl_bytes) and err (one int) the map is taken on the tensor cores
// for templates brute_mma_supported accepts; otherwise on FP32 CUDA cores.
struct ExhaustiveBufs {
    long long *IIS, *IIQ;
    float *inv, *ef, *map, *tf;
    double *td;
    int *cand;
    double *crho;
    TmplState *st;
    uint8_t *Ipad = nullptr;
    void *Bt = nullptr;
    int *err = nullptr;
    int *wsum = nullptr;   // window sums (the tensor-core map needs them)
};

// The exhaustive map on the tensor cores (brute_mma.cu): templates up to
// 128 x 128; the template tile (bytes) and its error-bound coefficient.
bool brute_mma_supported(int m, int n);
size_t brute_tmpl_bytes(int m, int n);
float brute_mma_epsA(int m, int n);
// Template tiles of T templates (t' at tf + k * tsz, states st + k) into
// B + k * brute_tmpl_bytes; with dense_only, only templates k with st[k].dense.
cudaError_t launch_brute_tmpl(const float *tf, size_t tsz, int T, int m, int n, int npad, void *B,
                              const TmplState *st, int dense_only, cudaStream_t s);
cudaError_t launch_pad_rows(const uint8_t *I, int p, int q, uint8_t *out, int qs, cudaStream_t s);
// rho maps of T templates (tile k at B + k * brute_tmpl_bytes, state st[k],
// map at map + k * map_stride); with dense_only, templates without
// st[k].dense are skipped.  The error factor ||I - 128|| / Omega comes from
// efac, or when efac is null from the window sums wsum and inv_sigma.
cudaError_t launch_brute_mma(const uint8_t *Ipad, int qs, int p, int q, const void *B, int m, int n,
                             const float *inv_sigma, const float *efac, const int *wsum,
                             TmplState *st, float *map, int64_t map_stride, int T, int dense_only,
                             int *err, cudaStream_t s);
// Candidates of the templates of a scan-2 batch that took the dense map
// (held in B.surv_rho + k * B.scap): every location whose rho + eps
// reaches the certain lower bound on the maximum.
cudaError_t launch_dense_candidates(const Scan2Batch &B, const int *wsum, const float *inv_sigma,
                                    int m, int n, cudaStream_t s);
// The exhaustive search of template tdev (m x n, row stride tld, device)
// on the uint8 image I8 (p x q, device): window statistics, rho at every
// location, candidates within the map's error bound of its maximum, their
// FP64 rho and the argmax (lowest row-major index on ties) into *best.
// Synchronises s; returns best->status or OPTA_ERR_CUDA.
opta_status exhaustive_run(const uint8_t *I8, int p, int q, const float *tdev, int64_t tld, int m,
                           int n, const ExhaustiveBufs &b, opta_result *best, cudaStream_t s);

int num_sms();
int topk_blocks(int G, int T);
// Budget of scan 1's waits for progress (0: the default 2 s) and its stall
// switch, for the verification hook opta_dbg_scan1_wait.
void set_scan1_wait(uint64_t wait_ns, int stall);

// Counts every kernel launch of the library and, when per-kernel timing is
// enabled (opta_dbg_profile_enable), brackets it with CUDA events on its stream.
// Raise func's dynamic shared-memory limit on the current device to at
// least `bytes` (the limits already set are kept per kernel and device,
// under a library-wide lock so that host threads may launch concurrently).
cudaError_t ensure_smem(const void *func, size_t bytes);

class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t s);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    void *a_ = nullptr;
};
constexpr int kTopkMax = 16;   // largest supported params.topk

}  // namespace opta
