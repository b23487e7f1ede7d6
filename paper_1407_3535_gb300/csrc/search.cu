// Per-template search kernels: template statistics, the exhaustive FP32 map,
// the pruned path of Sections 2 and 6 (centre rho, threshold, transitive
// bound + compaction, survivors) and the FP64 final argmax.
//
// Error bounds.  Every FP32 correlation produced here carries a certain
// bound eps on |rho_fp32 - rho_exact|: for a dot product accumulated with
// at most k roundings per term (Higham, Accuracy and Stability of
// Numerical Algorithms, Section 3.1) and template values rounded once,
//   |num_fp32 - num| <= (k+2) u ||t'||_2 ||v||_2     (Cauchy-Schwarz),
// so eps = (k+2) u (1.01) ||v||/sigma_v + 8u (the 8u covers the final
// products with 1/sigma).  ||v||/sigma_v ("efac") comes from exact integer
// window sums.  These bounds make the elimination test and the choice of
// FP64 candidates safe.
#include <algorithm>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace opta {

namespace {

__device__ inline float eps_bound(int k, float efac) {
    return (float)(k + 2) * kU32 * 1.01f * efac + 8.f * kU32;
}

__device__ inline double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_max_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of a double (blockDim.x multiple of 32, <= 1024).
__device__ double block_sum_d(double v, double *sh) {
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum_d(r);
        if (lane == 0) sh[0] = r;
    }
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Template statistics (Eq. rho1's mu_t and sigma_t), two FP64 passes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
tmpl_prep_kernel(const float *__restrict__ t, int64_t ld, const TmplIn *__restrict__ tin, int m,
                 int n, int npad, float *tf, size_t tsz, double *td, size_t dsz, TmplState *st,
                 int topk, int pack) {
    __shared__ double sh[32];
    const int mn = m * n;
    // block k prepares template k of the batch
    const int k = blockIdx.x;
    if (tin) { t = tin[k].data; ld = tin[k].ld; }
    tf += k * tsz;
    td += k * dsz;
    st += k;
    double s = 0.0, s2 = 0.0;
    int whole = 1;   // every value an integer in 0..255
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        const float v = t[(int64_t)(i / n) * ld + (i % n)];
        s += (double)v;
        s2 += (double)v * (double)v;   // exact for integers (below 2^53)
        whole &= (v >= 0.f && v <= 255.f && v == rintf(v)) ? 1 : 0;
    }
    whole = __syncthreads_and(whole);
    s = block_sum_d(s, sh);
    s2 = block_sum_d(s2, sh);
    if (pack && whole) {
        // the bytes, four to a word, rows of tmpl_row_bytes(n) bytes
        uint32_t *tb = reinterpret_cast<uint32_t *>(tf + (size_t)m * npad);
        const int wr = tmpl_row_bytes(n) / 4;
        for (int i = threadIdx.x; i < m * wr; i += blockDim.x) {
            const int u = i / wr, v0 = 4 * (i % wr);
            uint32_t w = 0u;
            for (int b = 0; b < 4; ++b)
                if (v0 + b < n) w |= (uint32_t)t[(int64_t)u * ld + v0 + b] << (8 * b);
            tb[i] = w;
        }
    }
    const double mu = s / (double)mn;
    double ss = 0.0;
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        const double d = (double)t[(int64_t)(i / n) * ld + (i % n)] - mu;
        td[i] = d;
        ss += d * d;
    }
    double amax = 0.0;   // max |t'| (for scan 1's fp16 scale)
    for (int i = threadIdx.x; i < m * npad; i += blockDim.x) {
        const int u = i / npad, v = i % npad;
        const float x = v < n ? (float)((double)t[(int64_t)u * ld + v] - mu) : 0.f;
        tf[i] = x;
        amax = fmax(amax, (double)fabsf(x));
    }
    ss = block_sum_d(ss, sh);
    // block maximum of amax (values >= 0: the maximum of the squares' order)
    {
        for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = amax;
        __syncthreads();
        if (threadIdx.x < 32) {
            double r = (int)threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
            if (threadIdx.x == 0) sh[0] = r;
        }
        __syncthreads();
        amax = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sg = sqrt(ss);
        st->mu = mu;
        st->sigma = sg;
        st->inv_sigma = sg > 0.0 ? (float)(1.0 / sg) : 0.f;
        st->flat = sg > 0.0 ? 0 : 1;
        st->lo_key = float_key(-4.f);   // below every correlation
        st->n_surv = 0;
        st->n_cand = 0;
        st->n_topk = topk;
        st->thr = -2.0;
        st->thr_lo = -2.f;
        st->best_idx = -1;
        st->best_rho = 0.0;
        st->overflow = 0;
        st->n_eval = 0;
        st->n_surv_eff = 0x7fffffff;
        st->hat_idx = -1;
        st->n_cand_search = 0;
        st->dense = 0;
        st->n_first = 0;
        st->u8 = pack && whole;
        st->sum_t = whole ? (int)s : 0;   // exact: integers below 2^22
        st->sumsq_t = whole ? (long long)s2 : 0;
        // the exhaustive map's integer operand t - rint(mu) keeps its error
        // bound while sigma_t >= sqrt(mn) / 6 (brute_mma.cu)
        st->int_op = whole && sg >= sqrt((double)mn) / 6.0 ? 1 : 0;
        st->c0 = st->int_op ? (float)(rint(mu) - mu) : 0.f;
        // s = 2^(14 - e) for max|t'| = f 2^e, f in [0.5, 1): s max|t'| in [2^13, 2^14)
        int e = 0;
        if (amax > 0.0) frexp(amax, &e);
        // (k clamped to float's normal range: only templates whose values
        // differ by less than 2^-112 would need more)
        const int k = amax > 0.0 ? max(-126, min(126, 14 - e)) : 0;
        st->tscale = ldexpf(1.f, k);
        st->tscale_inv = ldexpf(1.f, -k);
    }
}

// ---------------------------------------------------------------------------
// Exhaustive FP32 correlation map (brute force, Eq. rho1).
// Tile: 16 output rows x 128 output columns, 256 threads, each thread 8
// consecutive columns.  Template streamed in chunks of MT rows x NT columns.
// ---------------------------------------------------------------------------
constexpr int ZT_Y = 16, ZT_X = 128, ZT_MT = 32, ZT_NT = 128;
constexpr int ZT_W = ZT_X + ZT_NT + 8;           // image tile row length (floats)
constexpr int ZT_ROWS = ZT_Y + ZT_MT - 1;
constexpr size_t ZT_SMEM = (size_t)(ZT_ROWS * ZT_W + ZT_MT * ZT_NT) * sizeof(float);

__device__ inline int zncc_kacc(int m, int npad) {
    return ZT_NT + m * ((npad + ZT_NT - 1) / ZT_NT) + 1;
}

__global__ void __launch_bounds__(256)
zncc_map_kernel(const uint8_t *__restrict__ I, int p, int q, const float *__restrict__ tf,
                int m, int n, int npad, const float *__restrict__ inv_sigma,
                const float *__restrict__ efac, TmplState *st, float *map) {
    extern __shared__ float4 zsm4[];
    float *img = reinterpret_cast<float *>(zsm4);
    float *tm = img + ZT_ROWS * ZT_W;
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int y0 = blockIdx.y * ZT_Y, x0 = blockIdx.x * ZT_X;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    if (st->flat) return;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    for (int u0 = 0; u0 < m; u0 += ZT_MT) {
        const int mt = min(ZT_MT, m - u0);
        for (int v0 = 0; v0 < npad; v0 += ZT_NT) {
            const int nt = min(ZT_NT, npad - v0);
            __syncthreads();
            for (int i = tid; i < ZT_MT * ZT_NT; i += 256) {
                const int u = i / ZT_NT, v = i % ZT_NT;
                tm[i] = (u < mt && v < nt) ? tf[(int64_t)(u0 + u) * npad + v0 + v] : 0.f;
            }
            const int rows = ZT_Y + mt - 1;
            for (int i = tid; i < rows * ZT_W; i += 256) {
                const int r = i / ZT_W, c = i % ZT_W;
                const int gy = y0 + u0 + r, gx = x0 + v0 + c;
                float v = 0.f;
                if (gy < p && gx < q) v = (float)I[(int64_t)gy * q + gx] - 128.f;
                img[i] = v;
            }
            __syncthreads();
            for (int u = 0; u < mt; ++u) {
                const float *row = img + (ty + u) * ZT_W + tx * 8;
                const float *trow = tm + u * ZT_NT;
                float racc[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) racc[k] = 0.f;
                for (int v = 0; v < nt; v += 8) {
                    float w[16], tv[8];
                    const float4 *r4 = reinterpret_cast<const float4 *>(row + v);
                    const float4 *t4 = reinterpret_cast<const float4 *>(trow + v);
                    float4 a = r4[0], b = r4[1], c = r4[2], d = r4[3];
                    float4 e = t4[0], f = t4[1];
                    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
                    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
                    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
                    w[12] = d.x; w[13] = d.y; w[14] = d.z; w[15] = d.w;
                    tv[0] = e.x; tv[1] = e.y; tv[2] = e.z; tv[3] = e.w;
                    tv[4] = f.x; tv[5] = f.y; tv[6] = f.z; tv[7] = f.w;
#pragma unroll
                    for (int j = 0; j < 8; ++j)
#pragma unroll
                        for (int k = 0; k < 8; ++k) racc[k] = fmaf(tv[j], w[k + j], racc[k]);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) acc[k] += racc[k];
            }
        }
    }
    const int y = y0 + ty;
    const int kacc = zncc_kacc(m, npad);
    float lo = -3.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = x0 + tx * 8 + k;
        if (y < Ly && x < Lx) {
            const int64_t i = (int64_t)y * Lx + x;
            const float is = inv_sigma[i];
            const float rho = (acc[k] * st->inv_sigma) * is;
            map[i] = rho;
            const float eps = is > 0.f ? eps_bound(kacc, efac[i]) : 0.f;
            lo = fmaxf(lo, rho - eps);
        }
    }
    lo = warp_max_f(lo);
    if ((tid & 31) == 0 && lo > -2.5f) atomicMax(&st->lo_key, float_key(lo));
}

// Warp-aggregated append of flagged items to list[base...]; returns nothing.
__device__ inline void warp_append(bool flag, int value, int *counter, int *list, int cap,
                                   int *overflow) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (flag) {
        const int pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < cap) list[pos] = value;
        else atomicOr(overflow, 1);
    }
}

__global__ void map_candidates_kernel(const float *__restrict__ map, const float *__restrict__ efac,
                                      int64_t L, float epsA, TmplState *st, int *cand, int cap) {
    if (st->flat) return;
    const float lstar = key_float(st->lo_key);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < L; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool f = false;
        if (i < L) {
            const float ef = efac[i];
            const float eps = ef > 0.f ? fmaf(epsA, ef, 8.f * kU32) : 0.f;
            f = map[i] + eps >= lstar;
        }
        warp_append(f, (int)i, &st->n_cand, cand, cap, &st->overflow);
    }
}

// Eq. rho1 at the window (y, x) for a template of bytes (tb: its rows of
// tmpl_row_bytes(n) / 4 packed words), by the whole block: sum t I, sum I and
// sum I^2 are integers (exact in the block's FP64 sums, all below 2^53), so
// the numerator mn sum tI - sum t sum I and the variances mn sum t^2 -
// (sum t)^2 and mn sum I^2 - (sum I)^2 are exact in int64 and only the FP64
// square root and division round.  Flat window: 0.  Valid in thread 0.
__device__ double block_rho_u8(const uint8_t *__restrict__ I, int q, int y, int x,
                               const uint32_t *__restrict__ tb, int m, int n, const TmplState *st,
                               double *sh) {
    const int wr = tmpl_row_bytes(n) >> 2;
    const int mn = m * n;
    unsigned stb = 0u, sb = 0u, sbb = 0u;   // per thread: below 2^32 for any window of 16 M pixels
    // pixel i = r n + c, stepped by the block size without a division per pixel
    int pr = (int)threadIdx.x / n, pc = (int)threadIdx.x - pr * n;
    const int dr = (int)blockDim.x / n, dc = (int)blockDim.x - dr * n;
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        const unsigned b = I[(int64_t)(y + pr) * q + x + pc];
        const unsigned t = (tb[pr * wr + (pc >> 2)] >> (8 * (pc & 3))) & 255u;
        stb += t * b;
        sb += b;
        sbb += b * b;
        pr += dr;
        pc += dc;
        if (pc >= n) { pc -= n; ++pr; }
    }
    const double Stb = block_sum_d((double)stb, sh);
    const double Sb = block_sum_d((double)sb, sh);
    const double Sbb = block_sum_d((double)sbb, sh);
    double r = 0.0;
    if (threadIdx.x == 0) {
        const long long lmn = mn;
        const long long num = lmn * (long long)Stb - (long long)st->sum_t * (long long)Sb;
        const long long vt = lmn * st->sumsq_t - (long long)st->sum_t * (long long)st->sum_t;
        const long long vb = lmn * (long long)Sbb - (long long)Sb * (long long)Sb;
        r = (vt > 0 && vb > 0) ? (double)num / sqrt((double)vt * (double)vb) : 0.0;
    }
    return r;
}

// ---------------------------------------------------------------------------
// FP64 recomputation of Eq. rho1 at candidate locations (two passes, as the
// definition reads).  One block per candidate.
// Candidates [0, n_cand) of template blockIdx.y of a batch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
refine64_kernel(const uint8_t *__restrict__ I, int q, int Lx, const double *__restrict__ td,
                size_t dsz, int m, int n, TmplState *st, const int *__restrict__ cand,
                double *cand_rho, int64_t ccap, const float *__restrict__ tf, size_t tsz, int npad) {
    __shared__ double sh[32];
    st += blockIdx.y;
    if (st->flat) return;
    td += blockIdx.y * dsz;
    cand += blockIdx.y * ccap;
    cand_rho += blockIdx.y * ccap;
    const int to = (int)min((int64_t)st->n_cand, ccap);
    const int mn = m * n;
    const int r0 = (int)threadIdx.x / n, c0 = (int)threadIdx.x - r0 * n;   // start of this thread
    const int dr = (int)blockDim.x / n, dc = (int)blockDim.x - dr * n;    // its stride in (row, col)
    const uint32_t *tb = tf && st->u8 ? reinterpret_cast<const uint32_t *>(tf + blockIdx.y * tsz + (size_t)m * npad)
                                      : nullptr;
    for (int c = blockIdx.x; c < to; c += gridDim.x) {
        const int idx = cand[c];
        const int y = idx / Lx, x = idx % Lx;
        if (tb) {
            const double r = block_rho_u8(I, q, y, x, tb, m, n, st, sh);
            if (threadIdx.x == 0) cand_rho[c] = r;
            continue;
        }
        const uint8_t *w = I + (int64_t)y * q + x;
        long long si = 0;
        for (int i = threadIdx.x, r = r0, cc = c0; i < mn; i += blockDim.x) {
            si += w[(int64_t)r * q + cc];
            r += dr; cc += dc;
            if (cc >= n) { cc -= n; ++r; }
        }
        const double S = block_sum_d((double)si, sh);
        const double mu = S / (double)mn;
        double num = 0.0, vv = 0.0;
        for (int i = threadIdx.x, r = r0, cc = c0; i < mn; i += blockDim.x) {
            const double d = (double)w[(int64_t)r * q + cc] - mu;
            num += td[i] * d;
            vv += d * d;
            r += dr; cc += dc;
            if (cc >= n) { cc -= n; ++r; }
        }
        num = block_sum_d(num, sh);
        vv = block_sum_d(vv, sh);
        if (threadIdx.x == 0)
            cand_rho[c] = (vv == 0.0 || st->sigma == 0.0) ? 0.0 : num / (sqrt(vv) * st->sigma);
    }
}

// FP64 rho at the threshold centres of a batch: block (j, k) takes centre j
// of template k.
__global__ void __launch_bounds__(256)
refine64_topk_kernel(const uint8_t *__restrict__ I, int q, int Lx, const double *__restrict__ td,
                     size_t dsz, int m, int n, TmplState *st, const int *__restrict__ cand_topk,
                     double *cand_rho_topk, const float *__restrict__ tf, size_t tsz, int npad) {
    __shared__ double sh[32];
    const int j = blockIdx.x, k = blockIdx.y;
    st += k;
    if (st->flat || j >= st->n_topk) return;
    td += k * dsz;
    const int mn = m * n;
    const int idx = cand_topk[k * kTopkMax + j];
    const int y = idx / Lx, x = idx % Lx;
    if (tf && st->u8) {
        const double r = block_rho_u8(I, q, y, x, reinterpret_cast<const uint32_t *>(tf + k * tsz + (size_t)m * npad),
                                      m, n, st, sh);
        if (threadIdx.x == 0) cand_rho_topk[k * kTopkMax + j] = r;
        return;
    }
    long long si = 0;
    for (int i = threadIdx.x; i < mn; i += blockDim.x)
        si += I[(int64_t)(y + i / n) * q + x + (i % n)];
    const double S = block_sum_d((double)si, sh);
    const double mu = S / (double)mn;
    double num = 0.0, vv = 0.0;
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        const double d = (double)I[(int64_t)(y + i / n) * q + x + (i % n)] - mu;
        num += td[i] * d;
        vv += d * d;
    }
    num = block_sum_d(num, sh);
    vv = block_sum_d(vv, sh);
    if (threadIdx.x == 0)
        cand_rho_topk[k * kTopkMax + j] =
            (vv == 0.0 || st->sigma == 0.0) ? 0.0 : num / (sqrt(vv) * st->sigma);
}

// Argmax of (rho64, -index) over the survivor candidates and the threshold
// centres of one template; one block per template of a batch.
__global__ void __launch_bounds__(256)
final_argmax_kernel(TmplState *st, const int *__restrict__ cand,
                    const double *__restrict__ cand_rho, int64_t ccap, const int *__restrict__ ctk,
                    const double *__restrict__ crtk) {
    __shared__ double sv[256];
    __shared__ int si[256];
    st += blockIdx.x;
    cand += blockIdx.x * ccap;
    cand_rho += blockIdx.x * ccap;
    if (ctk) { ctk += blockIdx.x * kTopkMax; crtk += blockIdx.x * kTopkMax; }
    const int nc = (int)min((int64_t)st->n_cand, ccap);
    double bv = -3.0;
    int bi = 0x7fffffff;
    if (!st->flat) {
        for (int c = threadIdx.x; c < nc; c += blockDim.x) {
            const double v = cand_rho[c];
            const int i = cand[c];
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        if (ctk && (int)threadIdx.x < st->n_topk) {
            const double v = crtk[threadIdx.x];
            const int i = ctk[threadIdx.x];
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
    }
    sv[threadIdx.x] = bv; si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double v = sv[threadIdx.x + o];
            const int i = si[threadIdx.x + o];
            if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
                sv[threadIdx.x] = v; si[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (st->flat || si[0] == 0x7fffffff) { st->best_idx = 0; st->best_rho = 0.0; }
        else { st->best_idx = si[0]; st->best_rho = sv[0]; }
    }
}

// Literal mode (Section 4.3): the maximum found on the blurred image becomes
// hat_idx, and the candidates are replaced by its (2d+1) x (2d+1)
// neighbourhood clipped to the location grid, in row-major order (so the
// final argmax's lowest-index tie rule is the row-major one).  One block per
// template of a batch; ccap >= Ly * Lx.
__global__ void __launch_bounds__(256)
rematch_window_kernel(TmplState *st, int Ly, int Lx, int d, int *cand, int64_t ccap) {
    st += blockIdx.x;
    cand += blockIdx.x * ccap;
    if (st->flat) return;
    const int c = st->best_idx;
    const int yc = c / Lx, xc = c - yc * Lx;
    const int y0 = max(0, yc - d), y1 = min(Ly, yc + d + 1);
    const int x0 = max(0, xc - d), x1 = min(Lx, xc + d + 1);
    const int w = x1 - x0, cnt = (y1 - y0) * w;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) cand[i] = (y0 + i / w) * Lx + x0 + i % w;
    __syncthreads();   // every thread has read best_idx before it is replaced
    if (threadIdx.x == 0) {
        st->hat_idx = c;
        st->n_cand_search = st->n_cand;
        st->n_cand = cnt;
    }
}

// ---------------------------------------------------------------------------
// Scan 1 (Section 6): rho(t, pivot block) at every group centre, FP32.
// Tile of 4 x 32 centres, one thread per centre; template in chunks of
// 16 x 64; pivot tile (P - 128) in shared memory.
// ---------------------------------------------------------------------------
constexpr int CT_Y = 4, CT_X = 32, CT_MT = 16, CT_NT = 64;

__global__ void __launch_bounds__(128)
centre_rho_kernel(const uint8_t *__restrict__ P, int p, int q, const float *__restrict__ tf,
                  int m, int n, int npad, int h, int Ly, int Lx,
                  const float *__restrict__ c_inv_sigma, TmplState *st, float *rho_tc,
                  int tile_w, int gx_begin) {
    extern __shared__ float4 csm4[];
    float *tile = reinterpret_cast<float *>(csm4);
    const int tile_rows = (CT_Y - 1) * h + CT_MT;
    float *tm = tile + tile_rows * tile_w;
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int gy0 = blockIdx.y * CT_Y, gx0 = gx_begin + blockIdx.x * CT_X;
    const int ty = threadIdx.x / CT_X, tx = threadIdx.x % CT_X;
    if (st->flat) return;
    const int cy0 = group_centre_of(gy0, Ly, h), cx0 = group_centre_of(gx0, Lx, h);
    const int gy = gy0 + ty, gx = gx0 + tx;
    const bool valid = gy < Gy && gx < Gx;
    const int oy = valid ? group_centre_of(gy, Ly, h) - cy0 : 0;
    const int ox = valid ? group_centre_of(gx, Lx, h) - cx0 : 0;
    float acc = 0.f;
    for (int u0 = 0; u0 < m; u0 += CT_MT) {
        const int mt = min(CT_MT, m - u0);
        for (int v0 = 0; v0 < npad; v0 += CT_NT) {
            const int nt = min(CT_NT, npad - v0);
            __syncthreads();
            for (int i = threadIdx.x; i < CT_MT * CT_NT; i += blockDim.x) {
                const int u = i / CT_NT, v = i % CT_NT;
                tm[i] = (u < mt && v < nt) ? tf[(int64_t)(u0 + u) * npad + v0 + v] : 0.f;
            }
            for (int i = threadIdx.x; i < tile_rows * tile_w; i += blockDim.x) {
                const int r = i / tile_w, c = i % tile_w;
                const int yy = cy0 + u0 + r, xx = cx0 + v0 + c;
                tile[i] = (yy < p && xx < q) ? (float)P[(int64_t)yy * q + xx] - 128.f : 0.f;
            }
            __syncthreads();
            if (valid) {
                for (int u = 0; u < mt; ++u) {
                    const float *row = tile + (oy + u) * tile_w + ox;
                    const float *trow = tm + u * CT_NT;
                    float racc = 0.f;
                    for (int v = 0; v < nt; v += 4) {
                        const float4 tv = *reinterpret_cast<const float4 *>(trow + v);
                        racc = fmaf(tv.x, row[v], racc);
                        racc = fmaf(tv.y, row[v + 1], racc);
                        racc = fmaf(tv.z, row[v + 2], racc);
                        racc = fmaf(tv.w, row[v + 3], racc);
                    }
                    acc += racc;
                }
            }
        }
    }
    if (valid) {
        const int g = gy * Gx + gx;
        const float is = c_inv_sigma[g];
        const float r = (acc * st->inv_sigma) * is;
        rho_tc[g] = r;
    }
}

// rho(t_k, pivot) at the centres of one group column gx (all group rows) for a
// chunk of templates.  Used for the last column when its centre is off the
// uniform grid the tensor-core path covers.  A block takes one template
// (blockIdx.y), holds it in shared memory and walks kColChunk centres, one
// warp per centre at a time, so each template is read from global memory
// once per chunk rather than once per centre.  A template of bytes takes
// Eq. rho1's numerator exactly, m n sum(t P) - sum(t) sum(P), from 4-byte dot
// products (as the survivors do); others take sum(t' (P - 128)) in FP32.
// the largest m n whose sum of byte products fits in u32 (mn 255^2 < 2^32)
constexpr int kU8MaxMN = 32768;
constexpr int kColChunk = 64;
__global__ void __launch_bounds__(256)
centre_column_kernel(const uint8_t *__restrict__ P, int q, const float *__restrict__ tf, int m,
                     int n, int npad, size_t tsz, int h, int Ly, int Lx, int gx, int T,
                     const float *__restrict__ c_inv_sigma,
                     const TmplState *__restrict__ st, float *rho_tc, int64_t gstride) {
    extern __shared__ float4 csm4[];   // the block's template: t' (m x npad) or its bytes (m x wr words)
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int k = blockIdx.y;
    const bool u8 = st[k].u8 != 0 && (long long)m * n <= kU8MaxMN;
    const int wr = tmpl_row_bytes(n) / 4;   // words per packed template row
    {
        const float *src = tf + (size_t)k * tsz + (u8 ? (size_t)m * npad : 0);
        const int n16 = u8 ? m * wr / 4 : m * npad / 4;
        for (int i = threadIdx.x; i < n16; i += blockDim.x)
            csm4[i] = reinterpret_cast<const float4 *>(src)[i];
    }
    __syncthreads();
    const float *tsm = reinterpret_cast<const float *>(csm4);
    const uint32_t *tsw = reinterpret_cast<const uint32_t *>(csm4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cx = group_centre_of(gx, Lx, h);
    const uint8_t *pend = P + (int64_t)(Ly + m - 1) * q;   // end of the p x q pivot
    // four columns per lane and step; half-warps take two rows at once when
    // n / 4 <= 16
    const int n4 = n >> 2;
    const int rpp = n4 <= 16 ? 2 : 1;
    const int lr = rpp == 2 ? lane >> 4 : 0, lg = rpp == 2 ? lane & 15 : lane;
    const int gstep = rpp == 2 ? 16 : 32;
    constexpr float kC = 8388608.f + 128.f;
    const int gy_end = min(Gy, (int)(blockIdx.x + 1) * kColChunk);
    for (int gy = blockIdx.x * kColChunk + warp; gy < gy_end; gy += blockDim.x >> 5) {
        const int cy = group_centre_of(gy, Ly, h);
        const uint8_t *bp = P + (int64_t)cy * q + cx;
        float r = 0.f;
        if (u8) {
            unsigned acc = 0u, sp = 0u;   // sum t P, sum P over the window
            for (int u = lr; u < m; u += rpp) {
                const uint8_t *br = bp + (int64_t)u * q;
                const uint32_t *tr = tsw + u * wr;
                for (int g = lg; g < n4; g += gstep) {
                    // the four pixels from the aligned words around them
                    const uintptr_t ad = reinterpret_cast<uintptr_t>(br + 4 * g);
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(ad & ~(uintptr_t)3);
                    const unsigned sh = 8u * (unsigned)(ad & 3);
                    uint32_t w;
                    if (sh == 0u) {
                        w = wp[0];
                    } else if (reinterpret_cast<const uint8_t *>(wp + 2) <= pend) {
                        w = __funnelshift_r(wp[0], wp[1], sh);
                    } else {
                        const uint8_t *b4 = br + 4 * g;
                        w = (uint32_t)b4[0] | ((uint32_t)b4[1] << 8) | ((uint32_t)b4[2] << 16) |
                            ((uint32_t)b4[3] << 24);
                    }
                    acc = __dp4a(w, tr[g], acc);
                    sp = __dp4a(w, 0x01010101u, sp);
                }
                for (int v = 4 * n4 + lg; v < n; v += gstep) {
                    const unsigned b = br[v];
                    acc += b * ((tr[v >> 2] >> (8 * (v & 3))) & 255u);
                    sp += b;
                }
            }
            acc = __reduce_add_sync(0xffffffffu, acc);
            sp = __reduce_add_sync(0xffffffffu, sp);
            const long long D = mul_sub_wide((unsigned)(m * n), acc, st[k].sum_t, (int)sp);
            r = i64_to_f32(D) / (float)(m * n);
        } else {
            float acc = 0.f;
            for (int u = lr; u < m; u += rpp) {
                const uint8_t *br = bp + (int64_t)u * q;
                const float *tr = tsm + u * npad;
                for (int g = lg; g < n4; g += gstep) {
                    const float4 tv = *reinterpret_cast<const float4 *>(tr + 4 * g);
                    const uint8_t *b4 = br + 4 * g;
                    acc = fmaf(tv.x, __uint_as_float(0x4B000000u | b4[0]) - kC, acc);
                    acc = fmaf(tv.y, __uint_as_float(0x4B000000u | b4[1]) - kC, acc);
                    acc = fmaf(tv.z, __uint_as_float(0x4B000000u | b4[2]) - kC, acc);
                    acc = fmaf(tv.w, __uint_as_float(0x4B000000u | b4[3]) - kC, acc);
                }
                for (int v = 4 * n4 + lg; v < n; v += gstep)
                    acc = fmaf(tr[v], __uint_as_float(0x4B000000u | br[v]) - kC, acc);
            }
            r = warp_sum_f(acc);
        }
        if (lane == 0) {
            const int64_t g = (int64_t)gy * Gx + gx;
            const float is = c_inv_sigma[g];
            rho_tc[k * gstride + g] = (r * st[k].inv_sigma) * is;
        }
    }
}

// ---------------------------------------------------------------------------
// Threshold centres: approximate top-k of rho_tc (any k achieved values give a
// valid threshold; Section 6 uses the single best centre).
// ---------------------------------------------------------------------------
constexpr int TOPK_PER_THREAD = 4;
constexpr int TOPK_MAX = kTopkMax;

__device__ inline void block_topk(float *sv, int *si, int n, int k, float *out_v, int *out_i) {
    // k rounds of block argmax over sv[0..n); chosen entries are set to -inf.
    __shared__ float rv[32];
    __shared__ int rp[32];
    for (int r = 0; r < k; ++r) {
        float bv = -INFINITY; int bp = -1;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            if (sv[j] > bv || (sv[j] == bv && bp >= 0 && si[j] < si[bp])) { bv = sv[j]; bp = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (ov > bv || (ov == bv && op >= 0 && (bp < 0 || si[op] < si[bp]))) { bv = ov; bp = op; }
        }
        if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = bv; rp[threadIdx.x >> 5] = bp; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = -INFINITY; int pp = -1;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
                if (rp[w] >= 0 && (rv[w] > b || (rv[w] == b && (pp < 0 || si[rp[w]] < si[pp])))) { b = rv[w]; pp = rp[w]; }
            out_v[r] = b;
            out_i[r] = pp >= 0 ? si[pp] : -1;
            if (pp >= 0) sv[pp] = -INFINITY;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
topk_stage1_kernel(const float *__restrict__ rho_tc, int G, int64_t gstride, int k, float *tmp_v,
                   int *tmp_i, TmplState *st) {
    __shared__ float sv[256 * TOPK_PER_THREAD];
    __shared__ int si[256 * TOPK_PER_THREAD];
    // blockIdx.y: template of the batch
    st += blockIdx.y;
    rho_tc += blockIdx.y * gstride;
    tmp_v += (size_t)blockIdx.y * 256 * TOPK_MAX;
    tmp_i += (size_t)blockIdx.y * 256 * TOPK_MAX;
    if (st->flat) return;
    float v[TOPK_PER_THREAD];
    int ix[TOPK_PER_THREAD];
#pragma unroll
    for (int j = 0; j < TOPK_PER_THREAD; ++j) { v[j] = -INFINITY; ix[j] = -1; }
    const int chunk = (G + gridDim.x - 1) / gridDim.x;
    const int g0 = blockIdx.x * chunk, g1 = min(G, g0 + chunk);
    // four values in flight per thread, then inserted into its sorted list in
    // index order
    constexpr int kInFlight = 4;
    for (int g = g0 + threadIdx.x; g < g1; g += kInFlight * blockDim.x) {
        float xs[kInFlight];
#pragma unroll
        for (int u = 0; u < kInFlight; ++u) {
            const int gi = g + u * blockDim.x;
            xs[u] = gi < g1 ? rho_tc[gi] : -INFINITY;
        }
#pragma unroll
        for (int u = 0; u < kInFlight; ++u) {
            float x = xs[u];
            int xi = g + u * blockDim.x;
            if (x > v[TOPK_PER_THREAD - 1]) {
#pragma unroll
                for (int j = 0; j < TOPK_PER_THREAD; ++j) {
                    if (x > v[j]) { float tv = v[j]; int ti = ix[j]; v[j] = x; ix[j] = xi; x = tv; xi = ti; }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < TOPK_PER_THREAD; ++j) {
        sv[threadIdx.x * TOPK_PER_THREAD + j] = ix[j] >= 0 ? v[j] : -INFINITY;
        si[threadIdx.x * TOPK_PER_THREAD + j] = ix[j] >= 0 ? ix[j] : 0x7fffffff;
    }
    __syncthreads();
    __shared__ float ov[TOPK_MAX];
    __shared__ int oi[TOPK_MAX];
    block_topk(sv, si, 256 * TOPK_PER_THREAD, k, ov, oi);
    if (threadIdx.x < k) {
        tmp_v[blockIdx.x * TOPK_MAX + threadIdx.x] = ov[threadIdx.x];
        tmp_i[blockIdx.x * TOPK_MAX + threadIdx.x] = oi[threadIdx.x];
    }
}

__global__ void __launch_bounds__(256)
topk_stage2_kernel(const float *__restrict__ tmp_v, const int *__restrict__ tmp_i, int nb, int k,
                   int Gx, int h, int Ly, int Lx, TmplState *st, int *cand) {
    extern __shared__ float t2sm[];
    float *sv = t2sm;
    int *si = reinterpret_cast<int *>(t2sm + nb * k);
    // blockIdx.x: template of the batch; cand: its kTopkMax threshold slots
    st += blockIdx.x;
    tmp_v += (size_t)blockIdx.x * 256 * TOPK_MAX;
    tmp_i += (size_t)blockIdx.x * 256 * TOPK_MAX;
    cand += blockIdx.x * TOPK_MAX;
    if (st->flat) return;
    for (int j = threadIdx.x; j < nb * k; j += blockDim.x) {
        const int b = j / k, r = j % k;
        const int gi = tmp_i[b * TOPK_MAX + r];
        sv[j] = gi >= 0 ? tmp_v[b * TOPK_MAX + r] : -INFINITY;
        si[j] = gi >= 0 ? gi : 0x7fffffff;
    }
    __syncthreads();
    __shared__ float ov[TOPK_MAX];
    __shared__ int oi[TOPK_MAX];
    block_topk(sv, si, nb * k, k, ov, oi);
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (int r = 0; r < k; ++r) {
            const int g = oi[r];
            if (g < 0 || g == 0x7fffffff) continue;
            const int gy = g / Gx, gx = g % Gx;
            const int cy = group_centre_of(gy, Ly, h), cx = group_centre_of(gx, Lx, h);
            cand[cnt++] = cy * Lx + cx;
        }
        st->n_topk = cnt;
    }
}

// thr = max exact rho over the threshold centres; thr_lo = float below thr - 1e-9.
__global__ void threshold_kernel(TmplState *st, const double *__restrict__ cand_rho) {
    st += blockIdx.x;
    cand_rho += blockIdx.x * kTopkMax;
    if (threadIdx.x != 0 || st->flat) return;
    double thr = -2.0;
    for (int c = 0; c < st->n_topk; ++c) thr = fmax(thr, cand_rho[c]);
    st->thr = thr;
    // certain lower bound of the maximum: the exact threshold centres, or any
    // FP32 rho minus its error bound evaluated so far (group members)
    const float lo = fmaxf(__double2float_rd(thr - 1e-9), key_float(st->lo_key));
    st->thr_lo = lo;
    st->lo_key = max(st->lo_key, float_key(lo));
    // cos(gap) + kCosMargin >= thr_lo  <=>  gap <= acos(thr_lo - kCosMargin)
    st->theta_lim = acosf(fminf(1.f, fmaxf(-1.f, lo - kCosMargin))) + kAngMargin;
}

// ---------------------------------------------------------------------------
// Scan 2: interval-safe transitive bound (Eq. tranEqq in angle form) and
// warp-ballot compaction of the locations that fail Eq. SEC.
// ---------------------------------------------------------------------------
// Buckets are uniform in the bound cos(gap): bucket 0 holds the largest bounds.
// Any monotone map is valid; pass 2 recomputes it from the stored gap with the
// same code, so both passes agree.
__device__ inline int gap_bucket(float gap, float lim) {
    if (!(lim > 0.f)) return 0;
    const float x = gap / lim;                 // in [0, 1]
    int b = (int)(x * x * (float)kUbBuckets);  // ~ (1 - cos gap) / (1 - cos lim)
    return b < 0 ? 0 : (b >= kUbBuckets ? kUbBuckets - 1 : b);
}

// Scan 2, group first.  gap = max(0, tc.lo - co.hi, co.lo - tc.hi) is the
// smallest angle between t and a location allowed by the two intervals, so
// rho <= cos(gap); a location survives iff gap <= theta_lim.  Per group the
// union of its members' intervals (gco: lowest lo, highest hi) gives a
// group test that every group holding a survivor passes (FP32 subtraction
// is monotone), so members are read only for the (template, group) pairs
// that pass.  Pass A histograms the survivors by bucket and appends them,
// unordered, with their gap; pass B moves them into bucket order.  Gaps are
// computed with subtractions and maxima only, so every pass that recomputes
// one obtains the same value.
constexpr int SC_PER = 16;
constexpr int kChunkLoc = 256 * SC_PER;
constexpr int kS2MaxT = kScan2MaxT;
constexpr int kPassGroups = 256;   // groups per pass-A tile (one per thread)

__device__ inline float loc_gap(float2 t, float2 c) {
    return fmaxf(0.f, fmaxf(t.x - c.y, c.x - t.y));
}

// Group union intervals of the auto-correlation map (per template size).
__global__ void group_co_kernel(const float2 *__restrict__ theta_co, int Ly, int Lx, int h,
                                float2 *gco) {
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int64_t G = (int64_t)Gy * Gx;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int gy = (int)(g / Gx), gx = (int)(g - (int64_t)gy * Gx);
        const int y0 = gy * h, x0 = gx * h, y1 = min(y0 + h, Ly), x1 = min(x0 + h, Lx);
        float lo = 4.f, hi = -4.f;
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) {
                const float2 c = theta_co[(int64_t)y * Lx + x];
                lo = fminf(lo, c.x);
                hi = fmaxf(hi, c.y);
            }
        gco[g] = make_float2(lo, hi);
    }
}

// Pass A: group tests of a tile of groups against every template of the
// batch, then the members of the passing pairs: bucket histogram and the
// unordered survivor list (index in surv_eps as int, gap in surv_rho) of
// each template.
//
// The group test is taken in cosine space, without an arc cosine per
// (template, group): with l = theta_lim + kAngMargin and the centre's
// interval tv = [acos(min(1, r + e)) - kAngMargin, acos(max(-1, r - e)) +
// kAngMargin],
//   tv.lo - gco.hi <= theta_lim  <=>  gco.hi + l >= pi  or  r + e >= cos(gco.hi + l),
//   gco.lo - tv.hi <= theta_lim  <=>  gco.lo <= l        or  r - e <= cos(gco.lo - l),
// (acos decreasing on [-1, 1]; gco.hi > 0), the cosines from sincos of the
// group's bounds (once per group) and of l (once per template).  A slack of
// kCosSlack covers the rounding of both forms, so every pair that passes
// the angle test passes this one (extra pairs only cost their members'
// exact test).  A passing pair's interval tv is taken once, into shared
// memory, for the gaps of its members.
constexpr float kCosSlack = 8e-6f;
constexpr float kPiF = 3.14159265358979f;

// Templates per queue fill: the passing pairs of kPassTGroup templates (at
// most kPassTGroup x kPassGroups) are queued, their members tested, then the
// next templates'.
constexpr int kPassTGroup = 4;
constexpr int kPassQueue = kPassTGroup * kPassGroups;

__host__ __device__ inline size_t bound_pass_smem(int T) {
    return (size_t)T * kUbBuckets * sizeof(int) + (size_t)kPassQueue * sizeof(float2) +
           (size_t)kPassQueue * sizeof(unsigned short);
}

__global__ void __launch_bounds__(256)
bound_pass_kernel(const Scan2Batch B, const float2 *__restrict__ gco,
                  const float2 *__restrict__ theta_co, int Ly, int Lx, int h) {
    extern __shared__ int bp_sm[];
    __shared__ float lims[kS2MaxT];
    __shared__ float2 lcs[kS2MaxT];        // (cos l, sin l) of l = lim + kAngMargin
    __shared__ int ty0[kPassGroups], tx0[kPassGroups];   // top-left member of the tile's groups
    __shared__ unsigned short memd[81];    // member k of a group: (dy << 8) | dx
    __shared__ int qn;
    const int T = B.T;
    int *hist = bp_sm;                                                            // T x kUbBuckets
    float2 *qtv = reinterpret_cast<float2 *>(bp_sm + T * kUbBuckets);             // interval of entry
    unsigned short *queue = reinterpret_cast<unsigned short *>(qtv + kPassQueue); // (t << 8) | group
    for (int i = threadIdx.x; i < T * kUbBuckets; i += blockDim.x) hist[i] = 0;
    if ((int)threadIdx.x < T) {
        const float lim = B.st[threadIdx.x].flat ? -1.f : B.st[threadIdx.x].theta_lim;
        lims[threadIdx.x] = lim;
        lcs[threadIdx.x] = make_float2(cosf(lim + kAngMargin), sinf(lim + kAngMargin));
    }
    const int hh = h * h;
    for (int k = threadIdx.x; k < hh; k += blockDim.x) memd[k] = (unsigned short)(((k / h) << 8) | (k % h));
    // item / hh for item < 2^24 by one multiply: m = ceil(2^40 / hh) errs by
    // less than item / 2^40 < 2^-16, below the 1 / hh gap to the next integer
    const unsigned long long mhh = ((1ull << 40) + (unsigned long long)hh - 1) / (unsigned long long)hh;
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int64_t G = (int64_t)Gy * Gx;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) qn = 0;
    for (int64_t g0 = (int64_t)blockIdx.x * kPassGroups; g0 < G;
         g0 += (int64_t)gridDim.x * kPassGroups) {
        __syncthreads();
        const int64_t g = g0 + threadIdx.x;
        const float2 gc = g < G ? gco[g] : make_float2(4.f, -4.f);   // empty group: fails
        const float cef = g < G ? B.c_efac[g] : 0.f;
        const float e = fmaf(B.epsA, cef, kScan1EpsB);
        const float shi = sinf(gc.y), chi = cosf(gc.y), slo = sinf(gc.x), clo = cosf(gc.x);
        {
            const int gy = (int)(g / Gx);
            ty0[threadIdx.x] = gy * h;
            tx0[threadIdx.x] = (int)(g - (int64_t)gy * Gx) * h;
        }
        // every template's centre value of this group, loads in flight together
        float rg[kS2MaxT];
#pragma unroll
        for (int t = 0; t < kS2MaxT; ++t) rg[t] = t < T && g < G ? B.rho_tc[t * B.tc_stride + g] : 0.f;
        for (int t0 = 0; t0 < T; t0 += kPassTGroup) {
#pragma unroll
            for (int tt = 0; tt < kPassTGroup; ++tt) {
                const int t = t0 + tt;
                if (t >= T) break;
                const float lim = lims[t];
                bool pass = false;
                if (lim >= 0.f && g < G) {
                    // (constant indices keep rg in registers)
                    static_assert(kS2MaxT == 4 * kPassTGroup, "four template groups");
                    const float r = t0 == 0 ? rg[tt] : t0 == kPassTGroup ? rg[kPassTGroup + tt]
                                  : t0 == 2 * kPassTGroup ? rg[2 * kPassTGroup + tt] : rg[3 * kPassTGroup + tt];
                    const float2 cs = lcs[t];
                    const float l = lim + kAngMargin;
                    const bool c1 = gc.y + l >= kPiF || r + e >= fmaf(chi, cs.x, -shi * cs.y) - kCosSlack;
                    const bool c2 = gc.x <= l || r - e <= fmaf(clo, cs.x, slo * cs.y) + kCosSlack;
                    pass = c1 && c2;
                }
                const unsigned msk = __ballot_sync(0xffffffffu, pass);
                if (msk) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&qn, __popc(msk));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (pass)
                        queue[base + __popc(msk & ((1u << lane) - 1u))] =
                            (unsigned short)((t << 8) | threadIdx.x);
                }
            }
            __syncthreads();
            const int nq = qn;
            // the passing pairs' centre intervals, once each
            for (int k = threadIdx.x; k < nq; k += blockDim.x) {
                const int code = queue[k];
                const int64_t gg = g0 + (code & 255);
                qtv[k] = centre_interval(B.rho_tc[(code >> 8) * B.tc_stride + gg], B.c_efac[gg], B.epsA);
            }
            __syncthreads();
            const int nitem = nq * hh;
            // two items per thread and round: both location reads in flight
            for (int ib = 0; ib < nitem; ib += 2 * blockDim.x) {   // uniform trip count
                int tq[2], liq[2], eqq[2];
                float2 co[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int item = ib + u * blockDim.x + threadIdx.x;
                    tq[u] = 0;
                    liq[u] = -1;   // no location
                    eqq[u] = 0;
                    if (item < nitem) {
                        const int eq = (int)(((unsigned long long)item * mhh) >> 40);
                        const int mem = item - eq * hh;
                        const int code = queue[eq];
                        const int gi = code & 255;
                        const int dd = memd[mem];
                        const int my = ty0[gi] + (dd >> 8), mx = tx0[gi] + (dd & 255);
                        tq[u] = code >> 8;
                        eqq[u] = eq;
                        if (my < Ly && mx < Lx) {
                            liq[u] = my * Lx + mx;
                            co[u] = theta_co[liq[u]];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int t = tq[u];
                    const int li = liq[u];
                    const float gap = li >= 0 ? loc_gap(qtv[eqq[u]], co[u]) : 0.f;
                    const bool f = li >= 0 && gap <= lims[t];
                    if (f) atomicAdd(&hist[t * kUbBuckets + gap_bucket(gap, lims[t])], 1);
                    // append to template t's unordered list, aggregated over
                    // the lanes of the warp that share t
                    const unsigned fm = __ballot_sync(0xffffffffu, f);
                    if (fm) {
                        const unsigned peers = __match_any_sync(0xffffffffu, f ? t : -1);
                        const int leader = __ffs(peers) - 1;
                        int base = 0;
                        if (f && lane == leader) base = atomicAdd(&B.ucnt[t], __popc(peers));
                        base = __shfl_sync(0xffffffffu, base, leader);
                        if (f) {
                            const int64_t pos = base + __popc(peers & ((1u << lane) - 1u));
                            if (pos < B.scap) {
                                reinterpret_cast<int *>(B.surv_eps)[t * B.scap + pos] = li;
                                B.surv_rho[t * B.scap + pos] = gap;
                            } else {
                                atomicOr(&B.st[t].overflow, 1);
                            }
                        }
                    }
                }
            }
            __syncthreads();   // the queue is refilled
            if (threadIdx.x == 0) qn = 0;
            __syncthreads();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < T * kUbBuckets; i += blockDim.x) {
        const int v = hist[i];
        if (v) atomicAdd(&B.bucket_cnt[i], v);
    }
}

// Exclusive scan of the bucket counts into write cursors; total survivors.
// One warp per template: each lane owns kUbBuckets/32 consecutive buckets.
__global__ void bucket_scan_kernel(const Scan2Batch B) {
    TmplState *st = B.st + blockIdx.x;
    if (st->flat) return;
    const int *bucket_cnt = B.bucket_cnt + blockIdx.x * kUbBuckets;
    int *bucket_cur = B.bucket_cur + blockIdx.x * kUbBuckets;
    constexpr int PER = kUbBuckets / 32;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    int loc[PER], sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) { loc[k] = bucket_cnt[lane * PER + k]; sum += loc[k]; }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    // group order for a large template whose survivors are few next to the
    // count at which the dense map would take over (so the bound order's cut
    // has nothing to save): every cursor at the end, one bucket, and the
    // sort keeps each entry's place
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    const bool grouped = B.group_order && B.dense_frac > 0.f &&
                         (double)tot <= 0.25 * (double)B.dense_frac * (double)B.L;
    int acc = incl - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        bucket_cur[lane * PER + k] = grouped ? tot : acc;
        acc += loc[k];
    }
    if (lane == 31) { st->n_surv = incl; st->n_surv_eff = incl; st->grouped = grouped ? 1 : 0; }
}

// Pass B: the unordered survivors of template blockIdx.y into their bucket
// ranges (bucket 0 = largest bound first) with their bound cos(gap) +
// margin; in group order (TmplState::grouped) they keep their places.  Each
// block counts a slice per bucket in shared memory and reserves every
// bucket's part with one global atomic.
__global__ void __launch_bounds__(256)
bound_sort_kernel(const Scan2Batch B) {
    __shared__ int cnt[kUbBuckets];
    __shared__ int basep[kUbBuckets];
    const int t = blockIdx.y;
    TmplState *st = B.st + t;
    if (st->flat) return;
    const int64_t n = min((int64_t)B.ucnt[t], B.scap);
    if ((int64_t)blockIdx.x * kChunkLoc >= n) return;   // uniform
    const float lim = st->theta_lim;
    const int *uidx = reinterpret_cast<const int *>(B.surv_eps) + t * B.scap;
    const float *ugap = B.surv_rho + t * B.scap;
    int *bucket_cur = B.bucket_cur + t * kUbBuckets;
    int *surv = B.surv + t * B.scap;
    float *surv_ub = B.surv_ub + t * B.scap;
    for (int64_t base = (int64_t)blockIdx.x * kChunkLoc; base < n;
         base += (int64_t)gridDim.x * kChunkLoc) {
        if (st->grouped) {
            // in the bound pass's order: a group's members stay next to one
            // another (block-uniform branch)
            for (int64_t e = base + threadIdx.x; e < min(n, base + (int64_t)kChunkLoc); e += blockDim.x) {
                surv[e] = uidx[e];
                surv_ub[e] = cosf(ugap[e]) + kCosMargin;
            }
            continue;
        }
        for (int i = threadIdx.x; i < kUbBuckets; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        float g[SC_PER];
        int ix[SC_PER], bk[SC_PER];
#pragma unroll
        for (int k = 0; k < SC_PER; ++k) {
            const int64_t e = base + k * 256 + threadIdx.x;
            bk[k] = -1;
            if (e < n) {
                g[k] = ugap[e];
                ix[k] = uidx[e];
                bk[k] = gap_bucket(g[k], lim);
                atomicAdd(&cnt[bk[k]], 1);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kUbBuckets; i += blockDim.x) {
            const int c = cnt[i];
            basep[i] = c ? atomicAdd(&bucket_cur[i], c) : 0;
            cnt[i] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SC_PER; ++k) {
            if (bk[k] < 0) continue;
            const int pos = basep[bk[k]] + atomicAdd(&cnt[bk[k]], 1);
            surv[pos] = ix[k];
            surv_ub[pos] = cosf(g[k]) + kCosMargin;
        }
        __syncthreads();
    }
}

// Full bound and survivor maps of one template (verification output).
__global__ void bound_map_kernel(const Scan2Batch B, const float2 *__restrict__ theta_co, int Ly,
                                 int Lx, int h, float *ub_map, uint8_t *surv_map) {
    const TmplState *st = B.st;
    if (st->flat) return;
    const float lim = st->theta_lim;
    const int Gx = groups_along(Lx, h);
    const int64_t L = (int64_t)Ly * Lx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i - (int64_t)y * Lx);
        const int64_t g = (int64_t)(y / h) * Gx + x / h;
        const float gap = loc_gap(centre_interval(B.rho_tc[g], B.c_efac[g], B.epsA), theta_co[i]);
        if (ub_map) ub_map[i] = cosf(gap) + kCosMargin;
        if (surv_map) surv_map[i] = gap <= lim ? 1 : 0;
    }
}

// Angle intervals of the auto-correlation map.
__global__ void theta_co_kernel(const float *__restrict__ rho_co, int64_t L, float2 *theta_co) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x)
        theta_co[i] = angle_interval(rho_co[i], kEcoBound);
}

// ---------------------------------------------------------------------------
// Exact-ish rho (FP32, per-window centring v = I - rint(mu_o)) at the survivors;
// one warp per survivor, template in shared memory when it fits.
// ---------------------------------------------------------------------------
// Per-warp staging of a survivor's window in shared memory: rows are copied
// with 16-byte cp.async (aligned down; zero-filled past the image end) in
// chunks of kStageRows rows, double-buffered, so that each warp keeps many
// loads in flight instead of waiting on one byte load per row.
constexpr int kStageRows = 16;

__device__ inline int stage_width(int n) { return 16 * ((n + 30) / 16); }

__device__ inline void cp_async16(void *dst, const void *src, int bytes) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ inline void stage_rows(const uint8_t *I, const uint8_t *img_end, int q, int y, int x,
                                  int u0, int rows, int n, uint8_t *buf, int WB) {
    const int lane = threadIdx.x & 31;
    const int CW = WB / 16;
    for (int t = lane; t < rows * CW; t += 32) {
        const int r = t / CW, k = t % CW;
        const uint8_t *row = I + (int64_t)(y + u0 + r) * q + x;
        const uint8_t *ga = reinterpret_cast<const uint8_t *>(
            reinterpret_cast<uintptr_t>(row) & ~static_cast<uintptr_t>(15));
        const uint8_t *src = ga + 16 * k;
        const int64_t avail = img_end - src;
        const int bytes = avail >= 16 ? 16 : (avail > 0 ? (int)avail : 0);
        cp_async16(buf + r * WB + 16 * k, bytes > 0 ? src : I, bytes);
    }
    cp_async_commit();
}

// rho at location idx in FP32 with per-window centring v = I - rint(mu_o), by
// the whole warp, and its error bound; results valid in lane 0.  With a
// staging buffer (wbuf: 2 x kStageRows x WB bytes) the window goes through
// shared memory; without, it is read straight from global memory.
// A byte b as the float 2^23 + b (b under the exponent of 2^23): one logic
// operation instead of an integer-to-float conversion.
__device__ __forceinline__ float u8f(uint32_t b) { return __uint_as_float(0x4B000000u | b); }

__device__ inline void warp_rho32(const uint8_t *__restrict__ I, int q, int Lx,
                                  const int *__restrict__ wsum,
                                  const float *__restrict__ tm, int m, int n, int npad,
                                  const float *__restrict__ inv_sigma, float ist, int idx,
                                  uint8_t *wbuf, const uint8_t *img_end, float &rho, float &eps) {
    const int lane = threadIdx.x & 31;
    const long long mn = (long long)m * n;
    const int y = idx / Lx, x = idx % Lx;
    const long long S = wsum[idx];                 // exact window sum (per-size map)
    const float is = inv_sigma[idx];
    // any integer in [0, 255] keeps |v| <= 255; the nearest to the mean keeps it small
    const float a = rintf((float)S / (float)mn);
    const float ca = 8388608.f + a;   // 2^23 + a: u8f(b) - ca = b - a, exactly
    const uint8_t *bp = I + (int64_t)y * q + x;
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    if (wbuf) {
        const int WB = stage_width(n);
        const int nch = (m + kStageRows - 1) / kStageRows;
        stage_rows(I, img_end, q, y, x, 0, min(kStageRows, m), n, wbuf, WB);
        for (int c = 0; c < nch; ++c) {
            const int u0 = c * kStageRows, rows = min(kStageRows, m - u0);
            uint8_t *buf = wbuf + (c & 1) * kStageRows * WB;
            if (c + 1 < nch) {
                stage_rows(I, img_end, q, y, x, u0 + kStageRows, min(kStageRows, m - u0 - kStageRows),
                           n, wbuf + ((c + 1) & 1) * kStageRows * WB, WB);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            // four columns per lane and step (one funnel-shifted word of the
            // staged row, four byte_perm conversions, a 16-byte template
            // read); with n / 4 <= 16 the half-warps take two rows at once
            const int n4 = n >> 2;
            const int rpp = n4 <= 16 ? 2 : 1;               // rows per pass
            const int lr = rpp == 2 ? lane >> 4 : 0;        // this lane's row in the pass
            const int lg = rpp == 2 ? lane & 15 : lane;     // its first column group
            const int gstep = rpp == 2 ? 16 : 32;
            for (int r0 = 0; r0 < rows; r0 += rpp) {
                const int r = r0 + lr;
                float racc = 0.f;
                if (r < rows) {
                    const uint8_t *row = I + (int64_t)(y + u0 + r) * q + x;
                    const int off = (int)(reinterpret_cast<uintptr_t>(row) & 15);
                    const uint8_t *sb = buf + r * WB;
                    const unsigned *sw = reinterpret_cast<const unsigned *>(sb);
                    const float *tr = tm + (u0 + r) * npad;
                    for (int g = lg; g < n4; g += gstep) {
                        const int b0 = off + 4 * g;
                        const unsigned w =
                            __funnelshift_r(sw[b0 >> 2], sw[(b0 >> 2) + 1], 8u * (unsigned)(b0 & 3));
                        const float4 tv = *reinterpret_cast<const float4 *>(tr + 4 * g);
                        racc = fmaf(tv.x, __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7440)) - ca, racc);
                        racc = fmaf(tv.y, __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7441)) - ca, racc);
                        racc = fmaf(tv.z, __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7442)) - ca, racc);
                        racc = fmaf(tv.w, __uint_as_float(__byte_perm(w, 0x4b000000u, 0x7443)) - ca, racc);
                    }
                    for (int v = 4 * n4 + lg; v < n; v += gstep)
                        racc = fmaf(tr[v], u8f(sb[off + v]) - ca, racc);
                }
                if (r0 & 2) acc1 += racc; else acc0 += racc;
            }
            __syncwarp();   // the buffer is refilled two chunks later
        }
    } else {
        int u = 0;
        for (; u + 4 <= m; u += 4) {
            const uint8_t *r0 = bp + (int64_t)u * q;
            const float *t0 = tm + u * npad;
            for (int v = lane; v < n; v += 32) {
                const float i0 = u8f(r0[v]), i1 = u8f(r0[q + v]);
                const float i2 = u8f(r0[2 * (int64_t)q + v]), i3 = u8f(r0[3 * (int64_t)q + v]);
                acc0 = fmaf(t0[v], i0 - ca, acc0);
                acc1 = fmaf(t0[npad + v], i1 - ca, acc1);
                acc2 = fmaf(t0[2 * npad + v], i2 - ca, acc2);
                acc3 = fmaf(t0[3 * npad + v], i3 - ca, acc3);
            }
        }
        for (; u < m; ++u)
            for (int v = lane; v < n; v += 32)
                acc0 = fmaf(tm[u * npad + v], u8f(bp[(int64_t)u * q + v]) - ca, acc0);
    }
    const float acc = warp_sum_f((acc0 + acc2) + (acc1 + acc3));
    rho = 0.f;
    eps = 0.f;
    if (lane == 0) {
        // accumulation depth per lane: per row ceil(n/32) (one column per
        // lane and step) or 4 ceil(n/4 / 16) + 1 (four columns per lane and
        // step, a half-warp per row when n/4 <= 16, then the tail column),
        // then at most m row partial sums into one chain, the chain merges
        // and 5 shuffle levels
        const int kacc = max((n + 31) / 32, 4 * ((n / 4 + 15) / 16) + 1) + m + 8;
        rho = (acc * ist) * is;
        if (is > 0.f) {
            // ||I - a||^2 = Omega^2 + (S - a mn)^2 / mn, so ||I - a|| / Omega =
            // sqrt(1 + dS^2 / mn * (1/Omega)^2) with dS = S - a mn exact
            const long long dS = S - (long long)a * mn;
            const float r2 = (i64_to_f32(dS * dS) / i64_to_f32(mn)) * (is * is);
            eps = eps_bound(kacc, sqrtf(1.f + r2));
        }
    }
}

// Integer form of Eq. rho1's numerator for a template of bytes (TmplState::u8):
//   sum (t - mu_t)(I - mu_I) = (mn * sum t I - sum t * sum I) / mn,
// with sum t I accumulated exactly by 4-byte dot products (dp4a, u8 x u8 into
// u32: at most mn * 255^2 < 2^32 for mn <= kU8MaxMN) and the difference in
// int64.  In the lane form the window's rows come from the aligned copy of
// the image (rows of qs bytes, a multiple of 32) in 32-byte loads: chunk c
// of 32 columns needs the aligned blocks c and c + 1 of the row, from which
// the window's words are selected by the offset o = x mod 32 (word o / 4,
// then a funnel shift by 8 (o mod 4) bits); templates wider than 128 take
// 16-byte loads.  Only the last rounding steps remain: the conversion of
// the integer, the division by mn and the two products with 1/sigma_t and
// 1/Omega (each within a few ulp), so |rho - rho_exact| <= kU8Eps.
constexpr float kU8Eps = 16.f * kU32 * 1.01f;

// warp_rho32 for a template of bytes (TmplState::u8): the staged window's
// words against the packed template words by 4-byte dot products, summed
// exactly in u32 and over the warp; rho from the int64 numerator as in the
// lane form (error <= kU8Eps).  Needs the staging buffer.  Results in lane 0.
__device__ inline void warp_rho_u8(const uint8_t *__restrict__ I, int q, int Lx,
                                   const int *__restrict__ wsum, const uint32_t *__restrict__ tb,
                                   int m, int n, int sum_t, const float *__restrict__ inv_sigma,
                                   float ist, int idx, uint8_t *wbuf, const uint8_t *img_end,
                                   float &rho, float &eps) {
    const int lane = threadIdx.x & 31;
    const int y = idx / Lx, x = idx % Lx;
    const int wr = tmpl_row_bytes(n) / 4;   // words per packed template row
    const int WB = stage_width(n);
    const int nch = (m + kStageRows - 1) / kStageRows;
    const int n4 = n >> 2;
    const int rpp = n4 <= 16 ? 2 : 1;
    const int lr = rpp == 2 ? lane >> 4 : 0;
    const int lg = rpp == 2 ? lane & 15 : lane;
    const int gstep = rpp == 2 ? 16 : 32;
    unsigned acc = 0u;
    stage_rows(I, img_end, q, y, x, 0, min(kStageRows, m), n, wbuf, WB);
    for (int c = 0; c < nch; ++c) {
        const int u0 = c * kStageRows, rows = min(kStageRows, m - u0);
        uint8_t *buf = wbuf + (c & 1) * kStageRows * WB;
        if (c + 1 < nch) {
            stage_rows(I, img_end, q, y, x, u0 + kStageRows, min(kStageRows, m - u0 - kStageRows), n,
                       wbuf + ((c + 1) & 1) * kStageRows * WB, WB);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        for (int r0 = 0; r0 < rows; r0 += rpp) {
            const int r = r0 + lr;
            if (r < rows) {
                const uint8_t *row = I + (int64_t)(y + u0 + r) * q + x;
                const int off = (int)(reinterpret_cast<uintptr_t>(row) & 15);
                const uint8_t *sb = buf + r * WB;
                const unsigned *sw = reinterpret_cast<const unsigned *>(sb);
                const uint32_t *tr = tb + (u0 + r) * wr;
                for (int g = lg; g < n4; g += gstep) {
                    const int b0 = off + 4 * g;
                    const unsigned w =
                        __funnelshift_r(sw[b0 >> 2], sw[(b0 >> 2) + 1], 8u * (unsigned)(b0 & 3));
                    acc = __dp4a(w, tr[g], acc);
                }
                for (int v = 4 * n4 + lg; v < n; v += gstep)
                    acc += (unsigned)sb[off + v] * ((tr[v >> 2] >> (8 * (v & 3))) & 255u);
            }
        }
        __syncwarp();   // the buffer is refilled two chunks later
    }
    acc = __reduce_add_sync(0xffffffffu, acc);
    rho = 0.f;
    eps = 0.f;
    if (lane == 0) {
        const float is = inv_sigma[idx];
        const long long D = mul_sub_wide((unsigned)(m * n), acc, sum_t, wsum[idx]);
        rho = ((i64_to_f32(D) / (float)(m * n)) * ist) * is;
        eps = is > 0.f ? kU8Eps : 0.f;
    }
}

// Copy the template (m x npad floats, npad a multiple of 8) into shared
// memory with 16-byte loads, several in flight per thread.
__device__ inline const float *stage_template(const float *tf, int m, int npad, int in_smem,
                                              float *tsm) {
    if (!in_smem) return tf;
    const float4 *src = reinterpret_cast<const float4 *>(tf);
    float4 *dst = reinterpret_cast<float4 *>(tsm);
    const int n4 = m * npad / 4;
    int i = threadIdx.x;
    for (; i + 3 * (int)blockDim.x < n4; i += 4 * blockDim.x) {
        const float4 a = src[i], b = src[i + blockDim.x], c = src[i + 2 * blockDim.x],
                     d = src[i + 3 * blockDim.x];
        dst[i] = a; dst[i + blockDim.x] = b; dst[i + 2 * blockDim.x] = c; dst[i + 3 * blockDim.x] = d;
    }
    for (; i < n4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    return tsm;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// With B.span: the block's start and end into the sweep's span (every
// thread reaches the end: the sweeps return early only block-uniformly).
__device__ __forceinline__ void span_end(const Scan2Batch &B, unsigned long long t0) {
    if (!B.span) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMin(&B.span[0], t0);
        atomicMax(&B.span[1], gtimer());
    }
}

// Survivors of template blockIdx.y of a batch, in bucket order, skipping
// those whose bound has fallen below the running certain lower bound of the
// maximum.
__device__ __forceinline__ void warp_sweep(const Scan2Batch &B, const uint8_t *__restrict__ I, int q, int Lx,
                                           const int *__restrict__ wsum, int m, int n, int npad,
                                           const float *__restrict__ inv_sigma, int tmpl_in_smem,
                                           int stage, const uint8_t *img_end) {
    extern __shared__ float4 ssm4[];
    TmplState *st = B.st + blockIdx.y;
    if (st->flat) return;
    const float *tf = B.tf + blockIdx.y * B.tsz;
    const int *surv = B.surv + blockIdx.y * B.scap;
    const float *surv_ub = B.surv_ub + blockIdx.y * B.scap;
    float *surv_rho = B.surv_rho + blockIdx.y * B.scap;
    float *surv_eps = B.surv_eps + blockIdx.y * B.scap;
    // blocks whose first entry lies beyond the survivor list have nothing to do
    if (st->dense) return;
    // entries [ns_lo, ns0) of the bound-ordered list in this sweep
    const int ns_all = (int)min((int64_t)min(st->n_surv, st->n_surv_eff), B.scap);
    const int ns_lo = B.phase == 2 ? min(st->n_first, ns_all) : 0;
    const int ns0 = B.phase == 1 ? min(st->n_first, ns_all) : ns_all;
    if (ns_lo + (int)blockIdx.x * (int)(blockDim.x >> 5) >= ns0) return;
    // as many entries as the lane form's threshold: the lane form's template
    if (ns0 - ns_lo >= (st->u8 && B.Ipad != nullptr ? B.lane_min_u8 : B.lane_min_f32)) return;
    // a template of bytes: exact integer sums over the staged window
    const bool u8 = stage && st->u8 && (long long)m * n <= kU8MaxMN;
    const float *tm = nullptr;
    const uint32_t *tb = nullptr;
    if (u8) {
        const uint4 *src = reinterpret_cast<const uint4 *>(tf + (size_t)m * npad);
        tb = reinterpret_cast<const uint32_t *>(src);
        if (tmpl_in_smem) {
            const int n16 = m * (tmpl_row_bytes(n) >> 4);
            for (int i = threadIdx.x; i < n16; i += blockDim.x) reinterpret_cast<uint4 *>(ssm4)[i] = src[i];
            __syncthreads();
            tb = reinterpret_cast<const uint32_t *>(ssm4);
        }
    } else {
        tm = stage_template(tf, m, npad, tmpl_in_smem, reinterpret_cast<float *>(ssm4));
    }
    uint8_t *wbuf = nullptr;
    if (stage) {
        const size_t tb = tmpl_in_smem ? (((size_t)m * npad * sizeof(float) + 15) & ~(size_t)15) : 0;
        wbuf = reinterpret_cast<uint8_t *>(ssm4) + tb +
               (size_t)(threadIdx.x >> 5) * 2 * kStageRows * stage_width(n);
    }
    const int ns = ns0;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const float ist = st->inv_sigma;
    volatile unsigned int *lo_key = &st->lo_key;
    int evaluated = 0;
    // one survivor per warp, interleaved so that all warps advance through
    // the bound-ordered list together; a survivor whose bound has fallen below
    // the running certain lower bound of the maximum is skipped (Eq. SEC with
    // the best rho_tb found so far).  The warp's next 32 entries are read in
    // one round (a lane each), so skipped entries cost no dependent load; the
    // lower bound is read once per round and kept current with the values
    // the warp's own atomic maxima return (a stale bound only skips less).
    float lim = -4.f;
    for (int64_t base = ns_lo + warp; base < ns; base += 32 * (int64_t)nwarps) {
        const int64_t sl = base + (int64_t)lane * nwarps;
        const bool have = sl < ns;
        const float ubl = have ? surv_ub[sl] : -4.f;
        const int idxl = have ? surv[sl] : 0;
        lim = fmaxf(lim, __shfl_sync(0xffffffffu, key_float(*lo_key), 0));
        unsigned pend = __ballot_sync(0xffffffffu, have && ubl >= lim);
        while (pend) {
            const int k = __ffs(pend) - 1;
            pend &= pend - 1;
            const float ub = __shfl_sync(0xffffffffu, ubl, k);
            const int idx = __shfl_sync(0xffffffffu, idxl, k);
            if (ub < lim) continue;
            float rho, eps;
            if (u8)
                warp_rho_u8(I, q, Lx, wsum, tb, m, n, st->sum_t, inv_sigma, ist, idx, wbuf, img_end,
                            rho, eps);
            else
                warp_rho32(I, q, Lx, wsum, tm, m, n, npad, inv_sigma, ist, idx, wbuf, img_end, rho,
                           eps);
            unsigned seen = 0u;
            if (lane == 0) {
                const int64_t s = base + (int64_t)k * nwarps;
                surv_rho[s] = rho;
                surv_eps[s] = eps;
                const unsigned mine = float_key(rho - eps);
                seen = max(atomicMax(&st->lo_key, mine), mine);
                ++evaluated;
            }
            lim = fmaxf(lim, key_float(__shfl_sync(0xffffffffu, seen, 0)));
            __syncwarp();
        }
    }
    if (lane == 0 && evaluated) atomicAdd(&st->n_eval, evaluated);
}

__global__ void __launch_bounds__(256)
survivors_kernel(const Scan2Batch B, const uint8_t *__restrict__ I, int q, int Lx,
                 const int *__restrict__ wsum, int m, int n, int npad,
                 const float *__restrict__ inv_sigma, int tmpl_in_smem, int stage,
                 const uint8_t *img_end) {
    const unsigned long long t0 = B.span ? gtimer() : 0ull;
    warp_sweep(B, I, q, Lx, wsum, m, n, npad, inv_sigma, tmpl_in_smem, stage, img_end);
    span_end(B, t0);
}

// Survivors of small templates (m * n <= kLaneMaxMN): one lane per survivor.
// A warp takes 32 consecutive entries of its interleaved share of the
// bound-ordered list; each lane evaluates its own window from 32-bit words
// (funnel-shifted to the window's alignment), the template comes from
// shared memory by broadcast.  Per-row partial sums keep the accumulation
// depth at n + m + 2, the same error bound as the warp form.
constexpr int kLaneMaxMN = 2304;   // above this the warp form is faster (fewer, longer dot products)

__device__ __forceinline__ unsigned dp4a_chunk(uint4 cur, uint4 nxt, bool k1, bool k2, unsigned sh,
                                               uint4 tv, unsigned acc) {
    const uint32_t w[8] = {cur.x, cur.y, cur.z, cur.w, nxt.x, nxt.y, nxt.z, nxt.w};
    uint32_t a[6], l[5];
#pragma unroll
    for (int j = 0; j < 6; ++j) a[j] = k2 ? w[j + 2] : w[j];
#pragma unroll
    for (int j = 0; j < 5; ++j) l[j] = k1 ? a[j + 1] : a[j];
    acc = __dp4a(__funnelshift_r(l[0], l[1], sh), tv.x, acc);
    acc = __dp4a(__funnelshift_r(l[1], l[2], sh), tv.y, acc);
    acc = __dp4a(__funnelshift_r(l[2], l[3], sh), tv.z, acc);
    acc = __dp4a(__funnelshift_r(l[3], l[4], sh), tv.w, acc);
    return acc;
}

// window_dot_u8 for rows of NC chunks of 32 pixels (n <= 32 NC): 32-byte
// loads (ld.global.nc.v8) of the 32-byte-aligned image copy, whose rows are
// 32-byte aligned, so that a window row costs its 32-byte sectors once each;
// the NC + 1 blocks of R rows are loaded together (R = 4, 2 or 1 as the
// rows widen).  Chunk c needs blocks c and c + 1; its window words are the
// block pair's words o / 4 onward (a three-level selection by the bits of
// o / 4), funnel-shifted by 8 (o mod 4) bits.
__device__ __forceinline__ void ldg_v8(const uint8_t *p, uint32_t (&w)[8]) {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
                   "=r"(w[7])
                 : "l"(p));
}

template <int NC>
__device__ __forceinline__ void load_row32(const uint8_t *__restrict__ rp, int lb, uint32_t (&b)[NC + 1][8]) {
#pragma unroll
    for (int c = 0; c <= NC; ++c) {
        if (c == 0 || 32 * c < lb) {   // a block that holds a byte of the window
            ldg_v8(rp + 32 * c, b[c]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) b[c][k] = 0u;
        }
    }
}

__device__ __forceinline__ unsigned dp4a_chunk32(const uint32_t (&w0)[8], const uint32_t (&w1)[8], bool k1,
                                                 bool k2, bool k4, unsigned sh, uint4 t0, uint4 t1,
                                                 unsigned acc) {
    uint32_t a[12], b[10], l[9];
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        const uint32_t lo = j < 8 ? w0[j] : w1[j - 8];
        const uint32_t hi = j + 4 < 8 ? w0[j + 4] : w1[j - 4];
        a[j] = k4 ? hi : lo;
    }
#pragma unroll
    for (int j = 0; j < 10; ++j) b[j] = k2 ? a[j + 2] : a[j];
#pragma unroll
    for (int j = 0; j < 9; ++j) l[j] = k1 ? b[j + 1] : b[j];
    acc = __dp4a(__funnelshift_r(l[0], l[1], sh), t0.x, acc);
    acc = __dp4a(__funnelshift_r(l[1], l[2], sh), t0.y, acc);
    acc = __dp4a(__funnelshift_r(l[2], l[3], sh), t0.z, acc);
    acc = __dp4a(__funnelshift_r(l[3], l[4], sh), t0.w, acc);
    acc = __dp4a(__funnelshift_r(l[4], l[5], sh), t1.x, acc);
    acc = __dp4a(__funnelshift_r(l[5], l[6], sh), t1.y, acc);
    acc = __dp4a(__funnelshift_r(l[6], l[7], sh), t1.z, acc);
    acc = __dp4a(__funnelshift_r(l[7], l[8], sh), t1.w, acc);
    return acc;
}

template <int NC>
__device__ __forceinline__ unsigned window_dot_u8_rows32(const uint8_t *__restrict__ Ipad, int qs, int y,
                                                         int x, const uint4 *__restrict__ tb, int m,
                                                         int n) {
    constexpr int R = NC <= 1 ? 4 : (NC <= 2 ? 2 : 1);
    const int o = x & 31;
    const unsigned sh = 8u * (unsigned)(o & 3);
    const bool k1 = (o & 4) != 0, k2 = (o & 8) != 0, k4 = (o & 16) != 0;
    const int lb = o + n;
    const uint8_t *rp = Ipad + (int64_t)y * qs + (x - o);
    unsigned acc0 = 0u, acc1 = 0u;
    int u = 0;
#pragma unroll 1
    for (; u + R <= m; u += R, tb += R * 2 * NC, rp += (int64_t)R * qs) {
        uint32_t b[R][NC + 1][8];
#pragma unroll
        for (int r = 0; r < R; ++r) load_row32<NC>(rp + (int64_t)r * qs, lb, b[r]);
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint4 t0 = tb[(r * NC + c) * 2], t1 = tb[(r * NC + c) * 2 + 1];
                if ((r * NC + c) & 1)
                    acc1 = dp4a_chunk32(b[r][c], b[r][c + 1], k1, k2, k4, sh, t0, t1, acc1);
                else
                    acc0 = dp4a_chunk32(b[r][c], b[r][c + 1], k1, k2, k4, sh, t0, t1, acc0);
            }
    }
#pragma unroll 1
    for (; u < m; ++u, tb += 2 * NC, rp += qs) {
        uint32_t b[NC + 1][8];
        load_row32<NC>(rp, lb, b);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (c & 1)
                acc1 = dp4a_chunk32(b[c], b[c + 1], k1, k2, k4, sh, tb[2 * c], tb[2 * c + 1], acc1);
            else
                acc0 = dp4a_chunk32(b[c], b[c + 1], k1, k2, k4, sh, tb[2 * c], tb[2 * c + 1], acc0);
        }
    }
    return acc0 + acc1;
}

// sum over the m x n window at (y, x) of t * I, exactly (tb: the packed
// template rows of tmpl_row_bytes(n) bytes), in 16-byte loads (any n).
__device__ __forceinline__ unsigned window_dot_u8(const uint8_t *__restrict__ Ipad, int qs, int y,
                                                  int x, const uint4 *__restrict__ tb, int m, int n) {
    const int o = x & 15;
    const unsigned sh = 8u * (unsigned)(o & 3);
    const bool k1 = (o & 4) != 0, k2 = (o & 8) != 0;
    const int nch = (n + 15) >> 4;
    const int tstride = tmpl_row_bytes(n) >> 4;   // 16-byte chunks per packed template row
    const int lb = o + n;   // bytes of the aligned row that the window reaches
    const uint4 *rp = reinterpret_cast<const uint4 *>(Ipad + (int64_t)y * qs + (x - o));
    const int qs4 = qs >> 4;
    unsigned acc0 = 0u, acc1 = 0u;
    for (int u = 0; u < m; ++u, rp += qs4, tb += tstride) {
        uint4 cur = __ldg(rp);
        int c = 0;
        for (; c + 2 <= nch; c += 2) {
            const uint4 nx1 = __ldg(rp + c + 1);   // 16 (c + 1) < n <= lb: needed
            const uint4 nx2 = 16 * (c + 2) < lb ? __ldg(rp + c + 2) : make_uint4(0u, 0u, 0u, 0u);
            acc0 = dp4a_chunk(cur, nx1, k1, k2, sh, tb[c], acc0);
            acc1 = dp4a_chunk(nx1, nx2, k1, k2, sh, tb[c + 1], acc1);
            cur = nx2;
        }
        if (c < nch) {
            const uint4 nx1 = 16 * (c + 1) < lb ? __ldg(rp + c + 1) : make_uint4(0u, 0u, 0u, 0u);
            acc0 = dp4a_chunk(cur, nx1, k1, k2, sh, tb[c], acc0);
        }
    }
    return acc0 + acc1;
}

// window_dot_u8 by the 32-byte row form where a row has at most 4 chunks of
// 32 pixels (n <= 128); n is uniform over a block.
__device__ __forceinline__ unsigned window_dot_u8_any(const uint8_t *__restrict__ Ipad, int qs, int y,
                                                      int x, const uint4 *__restrict__ tb, int m,
                                                      int n) {
    switch ((n + 31) >> 5) {
    case 1: return window_dot_u8_rows32<1>(Ipad, qs, y, x, tb, m, n);
    case 2: return window_dot_u8_rows32<2>(Ipad, qs, y, x, tb, m, n);
    case 3: return window_dot_u8_rows32<3>(Ipad, qs, y, x, tb, m, n);
    case 4: return window_dot_u8_rows32<4>(Ipad, qs, y, x, tb, m, n);
    default: return window_dot_u8(Ipad, qs, y, x, tb, m, n);
    }
}

// FP32 form of one lane's window (any template): rows read as 32-bit words
// funnel-shifted to the window's alignment, per-row partial sums.
__device__ __forceinline__ float lane_dot_f32(const uint8_t *__restrict__ I, int q, int y, int x,
                                              const float *__restrict__ tm, int m, int n, int npad,
                                              float ca, uintptr_t iend) {
    float tot = 0.f;
    const uint8_t *wp = I + (int64_t)y * q + x;
    for (int u = 0; u < m; ++u) {
        const uintptr_t ra = reinterpret_cast<uintptr_t>(wp + (int64_t)u * q);
        const uint32_t *wr = reinterpret_cast<const uint32_t *>(ra & ~(uintptr_t)3);
        const unsigned sh = (unsigned)(ra & 3) * 8u;
        const float *tr = tm + u * npad;
        uint32_t w0 = wr[0];
        float racc = 0.f;
        if ((n & 3) == 0 && reinterpret_cast<uintptr_t>(wr + (n >> 2) + 1) <= iend) {
            // whole words of the row inside the image: four template values
            // per 16-byte read (the same for every lane)
            for (int v = 0; v < n; v += 4) {
                const uint32_t w1 = wr[(v >> 2) + 1];
                const uint32_t wv = __funnelshift_r(w0, w1, sh);
                w0 = w1;
                const float4 tv = *reinterpret_cast<const float4 *>(tr + v);
                racc = fmaf(tv.x, __uint_as_float(__byte_perm(wv, 0x4B000000u, 0x7650)) - ca, racc);
                racc = fmaf(tv.y, __uint_as_float(__byte_perm(wv, 0x4B000000u, 0x7651)) - ca, racc);
                racc = fmaf(tv.z, __uint_as_float(__byte_perm(wv, 0x4B000000u, 0x7652)) - ca, racc);
                racc = fmaf(tv.w, __uint_as_float(__byte_perm(wv, 0x4B000000u, 0x7653)) - ca, racc);
            }
        } else {
            for (int v = 0; v < n; v += 4) {
                // the next word, unless it starts past the image
                const uint32_t *nx = wr + (v >> 2) + 1;
                const uint32_t w1 = reinterpret_cast<uintptr_t>(nx) < iend ? *nx : 0u;
                const uint32_t wv = __funnelshift_r(w0, w1, sh);
                w0 = w1;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (v + b < n)
                        racc = fmaf(tr[v + b], __uint_as_float(__byte_perm(wv, 0x4B000000u, 0x7650 + b)) - ca,
                                    racc);
            }
        }
        tot += racc;
    }
    return tot;
}

// Per-warp queue of the entries a lane-form sweep evaluates (shared memory,
// after the template): list position, location and bound of up to
// 31 + 32 kLaneFetch entries, so that every evaluation round has 32 lanes
// busy however many entries the running lower bound skips.  A warp reads
// 32 kLaneFetch entries per round (kLaneFetch coalesced loads in flight per
// lane), which hides the latency of the reads behind one another.
constexpr int kLaneFetch = 4;
constexpr int kLaneQueue = 32 * kLaneFetch + 32;
__host__ __device__ inline size_t lane_tmpl_bytes(int m, int npad) {
    return ((size_t)m * npad * sizeof(float) + 15) & ~(size_t)15;
}

__device__ __forceinline__ void lane_sweep(const Scan2Batch &B, const uint8_t *__restrict__ I, int q, int Lx,
                                           const int *__restrict__ wsum, int m, int n, int npad,
                                           const float *__restrict__ inv_sigma, const uint8_t *img_end) {
    extern __shared__ float4 lsm4[];
    TmplState *st = B.st + blockIdx.y;
    if (st->flat) return;
    const int *surv = B.surv + blockIdx.y * B.scap;
    const float *surv_ub = B.surv_ub + blockIdx.y * B.scap;
    float *surv_rho = B.surv_rho + blockIdx.y * B.scap;
    float *surv_eps = B.surv_eps + blockIdx.y * B.scap;
    if (st->dense) return;
    // entries [ns_lo, ns) of the bound-ordered list in this sweep
    const int ns_all = (int)min((int64_t)min(st->n_surv, st->n_surv_eff), B.scap);
    const int ns_lo = B.phase == 2 ? min(st->n_first, ns_all) : 0;
    const int ns = B.phase == 1 ? min(st->n_first, ns_all) : ns_all;
    // entries per lane and round: kLaneFetch when every warp has that many
    // rounds of 32 or more, else fewer (short lists keep all warps busy)
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int K = max(1, min(kLaneFetch, (ns - ns_lo) / (32 * nwarps)));
    if (ns_lo + (int64_t)blockIdx.x * (blockDim.x >> 5) * 32 * K >= ns) return;   // uniform
    // fewer entries than the lane form's threshold: the warp form's template
    if (ns - ns_lo < (st->u8 && B.Ipad != nullptr ? B.lane_min_u8 : B.lane_min_f32)) return;
    // a template of bytes with the aligned image: exact integer dot products
    const bool u8 = B.Ipad != nullptr && st->u8 && (long long)m * n <= kU8MaxMN;
    const float *tm = nullptr;
    const uint4 *tb = reinterpret_cast<const uint4 *>(lsm4);
    if (u8) {
        const uint4 *src = reinterpret_cast<const uint4 *>(B.tf + blockIdx.y * B.tsz + (size_t)m * npad);
        const int n16 = m * (tmpl_row_bytes(n) >> 4);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) reinterpret_cast<uint4 *>(lsm4)[i] = src[i];
        __syncthreads();
    } else {
        tm = stage_template(B.tf + blockIdx.y * B.tsz, m, npad, 1, reinterpret_cast<float *>(lsm4));
    }
    int *qsl = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(lsm4) + lane_tmpl_bytes(m, npad)) +
               (threadIdx.x >> 5) * (3 * kLaneQueue);
    int *qix = qsl + kLaneQueue;
    float *qub = reinterpret_cast<float *>(qix + kLaneQueue);
    const int sum_t = st->sum_t;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const float ist = st->inv_sigma;
    const long long mn = (long long)m * n;
    const int kacc = n + m + 2;
    volatile unsigned int *lo_key = &st->lo_key;
    const uintptr_t iend = reinterpret_cast<uintptr_t>(img_end);
    float lim = -4.f;
    int evaluated = 0;
    // round r: warp w takes entries ns_lo + 32 K (r nwarps + w) + 32 k + lane
    // (k < K), so all warps advance through the bound order
    // together and the lanes of a warp hold neighbouring entries (of one
    // bucket, mostly from one strip of groups: overlapping windows, shared
    // cache lines); the entries the running lower bound does not skip join
    // the warp's queue, evaluated 32 at a time (the rest once the list is done)
    int qn = 0;
    int64_t base = ns_lo + 32 * K * (int64_t)warp;
    for (;;) {
        const bool more = base < ns;   // warp-uniform
        if (more) {
            lim = fmaxf(lim, __shfl_sync(0xffffffffu, key_float(*lo_key), 0));
            float ub[kLaneFetch];
            int ix[kLaneFetch];
#pragma unroll
            for (int k = 0; k < kLaneFetch; ++k) {
                const int64_t sl = base + 32 * k + lane;
                ub[k] = -4.f;
                ix[k] = 0;
                if (k < K && sl < ns) {
                    ub[k] = surv_ub[sl];
                    ix[k] = surv[sl];
                }
            }
#pragma unroll
            for (int k = 0; k < kLaneFetch; ++k) {
                const bool take = ub[k] >= lim;
                const unsigned mask = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const int pos = qn + __popc(mask & ((1u << lane) - 1u));
                    qsl[pos] = (int)(base + 32 * k + lane);
                    qix[pos] = ix[k];
                    qub[pos] = ub[k];
                }
                qn += __popc(mask);
            }
            base += 32 * K * (int64_t)nwarps;
            __syncwarp();
        }
        // queue entries [qh, qh + cnt), one per lane, while 32 are waiting
        // (all of them once the list is done); after each round one atomic
        // per warp: the largest certain lower bound of the round
        int qh = 0;
        while (qn - qh >= 32 || (!more && qn > qh)) {
            const int cnt = min(qn - qh, 32);
            const bool act = lane < cnt && qub[qh + lane] >= lim;
            float lo = -4.f;
            if (act) {
                const int sl = qsl[qh + lane], idx = qix[qh + lane];
                const int y = idx / Lx, x = idx - y * Lx;
                const int S = wsum[idx];
                const float is = inv_sigma[idx];
                float rho, eps = 0.f;
                if (u8) {
                    const unsigned dot = window_dot_u8_any(B.Ipad, B.qs, y, x, tb, m, n);
                    const long long D = mul_sub_wide((unsigned)mn, dot, sum_t, S);
                    rho = ((i64_to_f32(D) / (float)mn) * ist) * is;
                    if (is > 0.f) eps = kU8Eps;
                } else {
                    const float a = rintf((float)S / (float)mn);
                    // 2^23 + a: byte b - a = float(0x4B0000bb) - ca, exactly
                    const float tot = lane_dot_f32(I, q, y, x, tm, m, n, npad, 8388608.f + a, iend);
                    rho = (tot * ist) * is;
                    if (is > 0.f) {
                        const long long dS = (long long)S - (long long)a * mn;
                        const float r2 = (i64_to_f32(dS * dS) / i64_to_f32(mn)) * (is * is);
                        eps = eps_bound(kacc, sqrtf(1.f + r2));
                    }
                }
                surv_rho[sl] = rho;
                surv_eps[sl] = eps;
                lo = rho - eps;
                ++evaluated;
            }
            const unsigned key = __reduce_max_sync(0xffffffffu, act ? float_key(lo) : 0u);
            unsigned seen = 0u;
            if (lane == 0 && key) seen = max(atomicMax(&st->lo_key, key), key);
            lim = fmaxf(lim, key_float(__shfl_sync(0xffffffffu, seen, 0)));
            qh += cnt;
        }
        if (!more) break;
        // the fewer than 32 entries left to the front of the queue (qh >= 32:
        // no overlap)
        if (qh > 0) {
            const int rem = qn - qh;
            const bool mv = lane < rem;
            int ra = 0, rb = 0;
            float rc = 0.f;
            if (mv) { ra = qsl[qh + lane]; rb = qix[qh + lane]; rc = qub[qh + lane]; }
            __syncwarp();
            if (mv) { qsl[lane] = ra; qix[lane] = rb; qub[lane] = rc; }
            __syncwarp();
            qn = rem;
        }
    }
    evaluated = __reduce_add_sync(0xffffffffu, evaluated);
    if (lane == 0 && evaluated) atomicAdd(&st->n_eval, evaluated);
}

__global__ void __launch_bounds__(256, 2)
survivors_lane_kernel(const Scan2Batch B, const uint8_t *__restrict__ I, int q, int Lx,
                      const int *__restrict__ wsum, int m, int n, int npad,
                      const float *__restrict__ inv_sigma, const uint8_t *img_end) {
    const unsigned long long t0 = B.span ? gtimer() : 0ull;
    lane_sweep(B, I, q, Lx, wsum, m, n, npad, inv_sigma, img_end);
    span_end(B, t0);
}

// After the priority pass: the survivors from the first bucket whose largest
// bound is already below the running lower bound onward can all be skipped.
// bucket_end[b] = end of bucket b in the list; bucket b holds gaps with
// (gap/lim)^2 in [b/NB, (b+1)/NB), i.e. bounds <= cos(lim sqrt(b/NB)) + margin
// (evaluated with a relative slack on the angle and a doubled margin).
__global__ void __launch_bounds__(kUbBuckets)
survivor_cut_kernel(const Scan2Batch B, int phase) {
    __shared__ int first;
    TmplState *st = B.st + blockIdx.x;
    const int *bucket_end = B.bucket_cur + blockIdx.x * kUbBuckets;
    if (st->flat) return;
    if (threadIdx.x == 0) first = kUbBuckets;
    __syncthreads();
    const float lstar = key_float(st->lo_key);
    const float lim = st->theta_lim;
    const int b = threadIdx.x;
    if (b >= 1) {
        const float gmin = lim * sqrtf((float)b / (float)kUbBuckets) * 0.9999f;
        if (cosf(gmin) + 2.f * kCosMargin < lstar) atomicMin(&first, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int eff = first < kUbBuckets ? bucket_end[first - 1] : st->n_surv;
        if (phase <= 1) {
            st->n_surv_eff = eff;
            st->n_first = phase == 1 ? (int)min((int64_t)eff, B.first_budget) : eff;
        } else {
            // after the first sweep (the highest bounds first, so the running
            // lower bound has usually reached the maximum): with many
            // survivors still left, the tensor-core map of every location is
            // cheaper than their gathered evaluation
            const int64_t left = (int64_t)eff - st->n_first;
            if ((B.dense_frac < 0.f && left > 0) ||
                (B.dense_frac > 0.f && (double)left > (double)B.dense_frac * (double)B.L)) {
                st->dense = 1;
                st->n_eval = (int)B.L;
                st->n_surv_eff = st->n_first;
            } else {
                st->n_surv_eff = eff;
            }
        }
    }
}

// Threshold refinement: FP32 rho at every member of the groups of the
// threshold centres (the best match usually lies in the group of one of
// them); raises the certain lower bound of the maximum before scan 2.
__global__ void __launch_bounds__(256)
group_members_kernel(const uint8_t *__restrict__ I, int q, int Ly, int Lx, int h,
                     const int *__restrict__ wsum,
                     const float *__restrict__ tf, size_t tsz, int m, int n, int npad,
                     const float *__restrict__ inv_sigma, TmplState *st,
                     const int *__restrict__ cand, int tmpl_in_smem) {
    extern __shared__ float4 gsm4[];
    // blockIdx.y: template of the batch; blockIdx.x: its threshold centre
    st += blockIdx.y;
    tf += blockIdx.y * tsz;
    cand += blockIdx.y * kTopkMax;
    if (st->flat || (int)blockIdx.x >= st->n_topk) return;
    const float *tm = stage_template(tf, m, npad, tmpl_in_smem, reinterpret_cast<float *>(gsm4));
    const int k = blockIdx.x;
    if (k >= st->n_topk) return;
    const int c = cand[k];
    const int gy = (c / Lx) / h, gx = (c % Lx) / h;
    const int y0 = gy * h, x0 = gx * h;
    const int hy = min(h, Ly - y0), hx = min(h, Lx - x0);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float ist = st->inv_sigma;
    for (int j = warp; j < hy * hx; j += nw) {
        const int idx = (y0 + j / hx) * Lx + x0 + j % hx;
        float rho, eps;
        warp_rho32(I, q, Lx, wsum, tm, m, n, npad, inv_sigma, ist, idx, nullptr, nullptr, rho,
                   eps);
        if ((threadIdx.x & 31) == 0) atomicMax(&st->lo_key, float_key(rho - eps));
    }
}

__global__ void surv_candidates_kernel(const Scan2Batch B) {
    TmplState *st = B.st + blockIdx.y;
    if (st->flat || st->dense) return;
    const int *surv = B.surv + blockIdx.y * B.scap;
    const float *surv_ub = B.surv_ub + blockIdx.y * B.scap;
    const float *surv_rho = B.surv_rho + blockIdx.y * B.scap;
    const float *surv_eps = B.surv_eps + blockIdx.y * B.scap;
    int *cand = B.cand + blockIdx.y * B.ccap;
    const int cap = (int)B.ccap;
    const float lstar = key_float(st->lo_key);
    const int ns = (int)min((int64_t)st->n_surv, B.scap);
    for (int base = blockIdx.x * blockDim.x; base < ns; base += gridDim.x * blockDim.x) {
        const int s = base + threadIdx.x;
        bool f = false;
        // entries whose bound is below the final lower bound were skipped (never
        // written) and cannot be the maximum
        if (s < ns && surv_ub[s] >= lstar) f = surv_rho[s] + surv_eps[s] >= lstar;
        warp_append(f, s < ns ? surv[s] : 0, &st->n_cand, cand, cap, &st->overflow);
    }
}

// Candidates of a template that took the dense map: every location whose
// rho + eps reaches the certain lower bound (eps from the tensor-core map's
// bound, ||I - 128|| / Omega from the window sum and 1/Omega).
__global__ void dense_candidates_kernel(const Scan2Batch B, const int *__restrict__ wsum,
                                        const float *__restrict__ inv_sigma, int mn, float epsA) {
    TmplState *st = B.st + blockIdx.y;
    if (st->flat || !st->dense) return;
    const float *map = B.surv_rho + blockIdx.y * B.scap;
    int *cand = B.cand + blockIdx.y * B.ccap;
    const int cap = (int)B.ccap;
    const float lstar = key_float(st->lo_key);
    const float c128 = 128.f * (float)mn, imn = 1.f / (float)mn;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < B.L; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        bool f = false;
        if (i < B.L) {
            const float is = inv_sigma[i];
            float eps = 0.f;
            if (is > 0.f) {
                const float d = ((float)wsum[i] - c128) * is;
                eps = fmaf(epsA, sqrtf(fmaf(d * d, imn, 1.f)), 8.f * kU32);
            }
            f = map[i] + eps >= lstar;
        }
        warp_append(f, (int)i, &st->n_cand, cand, cap, &st->overflow);
    }
}

}  // namespace

cudaError_t launch_dense_candidates(const Scan2Batch &B, const int *wsum, const float *inv_sigma,
                                    int m, int n, cudaStream_t s) {
    LaunchScope ls("dense_candidates_kernel", s);
    const int bx = std::max(1, num_sms() * 4 / std::min(B.T, 4));
    dense_candidates_kernel<<<dim3(bx, B.T), 256, 0, s>>>(B, wsum, inv_sigma, m * n, brute_mma_epsA(m, n));
    return cudaGetLastError();
}

static int grid_cap(int64_t n, int threads, int per_sm) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_tmpl_prep(const float *t, int64_t ld, int m, int n, int npad, float *tf,
                             double *td, TmplState *st, int topk, cudaStream_t s) {
    LaunchScope ls_tmpl_prep_kernel("tmpl_prep_kernel", s);
    tmpl_prep_kernel<<<1, 1024, 0, s>>>(t, ld, nullptr, m, n, npad, tf, 0, td, 0, st, topk, 0);
    return cudaGetLastError();
}

cudaError_t launch_tmpl_prep_batch(const TmplIn *tin, int T, int m, int n, int npad, float *tf,
                                   size_t tsz, double *td, size_t dsz, TmplState *st, int topk,
                                   cudaStream_t s) {
    LaunchScope ls("tmpl_prep_kernel", s);
    tmpl_prep_kernel<<<T, 1024, 0, s>>>(nullptr, 0, tin, m, n, npad, tf, tsz, td, dsz, st, topk,
                                        tsz >= tmpl_slot_floats(m, n) ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_zncc_map(const uint8_t *I, int p, int q, const float *tf, int m, int n,
                            int npad, const float *inv_sigma, const float *efac128,
                            TmplState *st, float *map, cudaStream_t s) {
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(zncc_map_kernel), ZT_SMEM);
        if (e != cudaSuccess) return e;
    }
    const int Ly = p - m + 1, Lx = q - n + 1;
    dim3 grid((Lx + ZT_X - 1) / ZT_X, (Ly + ZT_Y - 1) / ZT_Y);
    LaunchScope ls_zncc_map_kernel("zncc_map_kernel", s);
    zncc_map_kernel<<<grid, 256, ZT_SMEM, s>>>(I, p, q, tf, m, n, npad, inv_sigma, efac128, st, map);
    return cudaGetLastError();
}

float zncc_map_epsA(int m, int n) {
    const int npad = (n + 7) & ~7;
    const int kacc = ZT_NT + m * ((npad + ZT_NT - 1) / ZT_NT) + 1;
    return (float)(kacc + 2) * kU32 * 1.01f;   // eps_bound's coefficient of efac
}

cudaError_t launch_map_candidates(const float *map, const float *efac128, int64_t L, float epsA,
                                  TmplState *st, int *cand, int cap, cudaStream_t s) {
    LaunchScope ls_map_candidates_kernel("map_candidates_kernel", s);
    map_candidates_kernel<<<grid_cap(L, 256, 8), 256, 0, s>>>(map, efac128, L, epsA, st, cand, cap);
    return cudaGetLastError();
}

cudaError_t launch_refine64(const uint8_t *I, int q, int Lx, const double *td, size_t dsz, int m,
                            int n, int T, TmplState *st, const int *cand, double *cand_rho,
                            int64_t ccap, cudaStream_t s, const float *tf, size_t tsz, int npad) {
    const int bx = std::max(1, num_sms() * 2 / std::min(T, 8));
    LaunchScope ls_refine64_kernel("refine64_kernel", s);
    refine64_kernel<<<dim3(bx, T), 256, 0, s>>>(I, q, Lx, td, dsz, m, n, st, cand, cand_rho, ccap, tf,
                                                tsz, npad);
    return cudaGetLastError();
}

cudaError_t launch_final_argmax(int T, TmplState *st, const int *cand, const double *cand_rho,
                                int64_t ccap, const int *cand_topk, const double *cand_rho_topk,
                                cudaStream_t s) {
    LaunchScope ls_final_argmax_kernel("final_argmax_kernel", s);
    final_argmax_kernel<<<T, 256, 0, s>>>(st, cand, cand_rho, ccap, cand_topk, cand_rho_topk);
    return cudaGetLastError();
}

cudaError_t launch_rematch_window(int T, TmplState *st, int Ly, int Lx, int d, int *cand,
                                  int64_t ccap, cudaStream_t s) {
    if (d < 0 || (int64_t)(2 * d + 1) * (2 * d + 1) > ccap) return cudaErrorInvalidValue;
    LaunchScope ls("rematch_window_kernel", s);
    rematch_window_kernel<<<T, 256, 0, s>>>(st, Ly, Lx, d, cand, ccap);
    return cudaGetLastError();
}

cudaError_t launch_refine64_topk(const uint8_t *I, int q, int Lx, const double *td, size_t dsz,
                                 int m, int n, int T, TmplState *st, const int *cand_topk,
                                 double *cand_rho_topk, cudaStream_t s, const float *tf, size_t tsz,
                                 int npad) {
    LaunchScope ls("refine64_topk_kernel", s);
    refine64_topk_kernel<<<dim3(kTopkMax, T), 256, 0, s>>>(I, q, Lx, td, dsz, m, n, st, cand_topk,
                                                           cand_rho_topk, tf, tsz, npad);
    return cudaGetLastError();
}

cudaError_t launch_centre_rho(const uint8_t *P, int p, int q, const float *tf, int m, int n,
                              int npad, int h, int Ly, int Lx, const float *c_inv_sigma,
                              TmplState *st, float *rho_tc, int gx_begin, cudaStream_t s) {
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int tile_w = ((CT_X - 1) * h + CT_NT + 3) & ~3;
    const int tile_rows = (CT_Y - 1) * h + CT_MT;
    const size_t smem = (size_t)(tile_rows * tile_w + CT_MT * CT_NT) * sizeof(float);
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(centre_rho_kernel), smem);
        if (e != cudaSuccess) return e;
    }
    if (gx_begin >= Gx) return cudaSuccess;
    dim3 grid((Gx - gx_begin + CT_X - 1) / CT_X, (Gy + CT_Y - 1) / CT_Y);
    LaunchScope ls_centre_rho_kernel("centre_rho_kernel", s);
    centre_rho_kernel<<<grid, CT_Y * CT_X, smem, s>>>(P, p, q, tf, m, n, npad, h, Ly, Lx,
                                                     c_inv_sigma, st, rho_tc, tile_w,
                                                     gx_begin);
    return cudaGetLastError();
}

int topk_blocks(int G, int T) {
    // one wave of the GPU over all templates (8 blocks of 256 per SM), each
    // block a slice of at least 2048 centres
    int nb = (num_sms() * 8 + T - 1) / max(T, 1);
    nb = min(nb, (G + 2047) / 2048);
    if (nb > 256) nb = 256;
    if (nb < 1) nb = 1;
    return nb;
}

cudaError_t launch_centre_column(const uint8_t *P, int q, const float *tf, int m, int n, int npad,
                                 size_t tsz, int h, int Ly, int Lx, int gx, int T,
                                 const float *c_inv_sigma, const TmplState *st, float *rho_tc,
                                 int64_t gstride, cudaStream_t s) {
    const int Gy = groups_along(Ly, h);
    if (npad % 4 != 0 || tsz % 4 != 0) return cudaErrorInvalidValue;
    const size_t smem = std::max((size_t)m * npad * sizeof(float), (size_t)m * tmpl_row_bytes(n));
    const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(centre_column_kernel), smem);
    if (e != cudaSuccess) return e;
    LaunchScope ls("centre_column_kernel", s);
    centre_column_kernel<<<dim3((Gy + kColChunk - 1) / kColChunk, T), 256, smem, s>>>(
        P, q, tf, m, n, npad, tsz, h, Ly, Lx, gx, T, c_inv_sigma, st, rho_tc, gstride);
    return cudaGetLastError();
}

cudaError_t launch_topk(const float *rho_tc, int64_t gstride, int Gy, int Gx, int h, int Ly, int Lx,
                        int k, int T, TmplState *st, float *tmp_val, int *tmp_idx, int *cand_topk,
                        cudaStream_t s) {
    const int G = Gy * Gx;
    if (k > TOPK_MAX) k = TOPK_MAX;
    if (k < 1) k = 1;
    const int nb = topk_blocks(G, T);
    {
        LaunchScope ls("topk_stage1_kernel", s);
        topk_stage1_kernel<<<dim3(nb, T), 256, 0, s>>>(rho_tc, G, gstride, k, tmp_val, tmp_idx, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)nb * k * (sizeof(float) + sizeof(int));
    {
        LaunchScope ls("topk_stage2_kernel", s);
        topk_stage2_kernel<<<T, 256, smem, s>>>(tmp_val, tmp_idx, nb, k, Gx, h, Ly, Lx, st, cand_topk);
    }
    return cudaGetLastError();
}

cudaError_t launch_threshold(TmplState *st, const double *cand_rho_topk, int T, cudaStream_t s) {
    LaunchScope ls_threshold_kernel("threshold_kernel", s);
    threshold_kernel<<<T, 32, 0, s>>>(st, cand_rho_topk);
    return cudaGetLastError();
}

cudaError_t launch_bound_compact(const Scan2Batch &B, const float2 *theta_co, const float2 *gco,
                                 int Ly, int Lx, int h, float *ub_map, uint8_t *surv_map,
                                 cudaStream_t s) {
    if (B.T < 1 || B.T > kS2MaxT || ((ub_map || surv_map) && B.T != 1) || h < 1 || h > 9)
        return cudaErrorInvalidValue;
    const int64_t G = (int64_t)groups_along(Ly, h) * groups_along(Lx, h);
    const int64_t tiles = (G + kPassGroups - 1) / kPassGroups;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 8));
    cudaError_t e = cudaMemsetAsync(B.bucket_cnt, 0, (size_t)B.T * kUbBuckets * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.ucnt, 0, (size_t)B.T * sizeof(int), s);
    if (e != cudaSuccess) return e;
    {
        const size_t smem = bound_pass_smem(B.T);
        if ((e = ensure_smem(reinterpret_cast<const void *>(bound_pass_kernel), smem)) != cudaSuccess)
            return e;
        LaunchScope ls("bound_pass_kernel", s);
        bound_pass_kernel<<<grid, 256, smem, s>>>(B, gco, theta_co, Ly, Lx, h);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        LaunchScope ls("bucket_scan_kernel", s);
        bucket_scan_kernel<<<B.T, 32, 0, s>>>(B);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        LaunchScope ls("bound_sort_kernel", s);
        // every template gets the blocks a long list needs; the blocks past a
        // short list's chunks return at once
        bound_sort_kernel<<<dim3(num_sms() * 4, B.T), 256, 0, s>>>(B);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ub_map || surv_map) {
        const int64_t L = (int64_t)Ly * Lx;
        LaunchScope ls("bound_map_kernel", s);
        bound_map_kernel<<<grid_cap(L, 256, 8), 256, 0, s>>>(B, theta_co, Ly, Lx, h, ub_map, surv_map);
        e = cudaGetLastError();
    }
    return e;
}

namespace {
__global__ void centre_intervals_kernel(const float *__restrict__ rho_tc, int64_t G, int T,
                                        const float *__restrict__ c_efac, float epsA, float2 *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)T * G;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = centre_interval(rho_tc[i], c_efac[i % G], epsA);
}
}  // namespace

cudaError_t launch_centre_intervals(const float *rho_tc, int64_t G, int T, const float *c_efac,
                                    float epsA, float2 *out, cudaStream_t s) {
    LaunchScope ls("centre_intervals_kernel", s);
    centre_intervals_kernel<<<grid_cap((int64_t)T * G, 256, 8), 256, 0, s>>>(rho_tc, G, T, c_efac,
                                                                            epsA, out);
    return cudaGetLastError();
}

cudaError_t launch_theta_co(const float *rho_co, int64_t L, float2 *theta_co, cudaStream_t s) {
    LaunchScope ls("theta_co_kernel", s);
    theta_co_kernel<<<grid_cap(L, 256, 16), 256, 0, s>>>(rho_co, L, theta_co);
    return cudaGetLastError();
}

cudaError_t launch_group_co(const float2 *theta_co, int Ly, int Lx, int h, float2 *gco,
                            cudaStream_t s) {
    const int64_t G = (int64_t)groups_along(Ly, h) * groups_along(Lx, h);
    LaunchScope ls("group_co_kernel", s);
    group_co_kernel<<<grid_cap(G, 256, 16), 256, 0, s>>>(theta_co, Ly, Lx, h, gco);
    return cudaGetLastError();
}

static size_t tmpl_smem(int m, int npad, int *in_smem) {
    size_t smem = (size_t)m * npad * sizeof(float);
    *in_smem = smem <= 200 * 1024;
    return *in_smem ? smem : 0;
}

// One sweep (B.phase) over the survivor lists of a batch.
// One sweep: each template of the batch by the lane form
// (survivors_lane_kernel) or the warp form (survivors_kernel), by its entry
// count against B.lane_min_*; a kernel runs only when some template may
// take its form.
static cudaError_t launch_sweep(const Scan2Batch &B, const uint8_t *I, int q, int Lx, const int *wsum,
                                int m, int n, int npad, const float *inv_sigma, int in_smem, int stage,
                                size_t smem, const uint8_t *iend, cudaStream_t s) {
    // one sweep for the whole batch: num_sms * 4 blocks for one template,
    // fewer per template (down to num_sms) when several share the launch
    const int bx = std::max(num_sms(), num_sms() * 4 / std::min(B.T, 4));
    const bool lane = std::min(B.lane_min_u8, B.lane_min_f32) < kLaneNever;
    const bool warp = std::max(B.lane_min_u8, B.lane_min_f32) > 0;
    if (lane) {
        const size_t lsmem = lane_tmpl_bytes(m, npad) + (size_t)8 * 3 * kLaneQueue * sizeof(int);
        {
            const cudaError_t e2 =
                ensure_smem(reinterpret_cast<const void *>(survivors_lane_kernel), lsmem);
            if (e2 != cudaSuccess) return e2;
        }
        LaunchScope ls("survivors_lane_kernel", s);
        survivors_lane_kernel<<<dim3(bx, B.T), 256, lsmem, s>>>(B, I, q, Lx, wsum, m, n, npad,
                                                                inv_sigma, iend);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (warp) {
        LaunchScope ls("survivors_kernel", s);
        survivors_kernel<<<dim3(bx, B.T), 256, smem, s>>>(B, I, q, Lx, wsum, m, n, npad,
                                                          inv_sigma, in_smem, stage, iend);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

// Lane-form thresholds per (device, m, n, bytes): measured by the tuner,
// else the default rule -- FP32 path: the lane form up to kLaneMaxMN
// template pixels at any count, the warp form above; integer path: the lane
// form at any count up to 1024 pixels, above from 8192 entries on.
static std::mutex g_form_mu;
static std::map<std::tuple<int, int, int, int>, int> g_lane_min;

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
    return dev;
}

int survivor_lane_min(int m, int n, bool u8, bool *tuned) {
    const auto key = std::make_tuple(current_device(), m, n, u8 ? 1 : 0);
    {
        std::lock_guard<std::mutex> lk(g_form_mu);
        const auto it = g_lane_min.find(key);
        if (tuned) *tuned = it != g_lane_min.end();
        if (it != g_lane_min.end()) return it->second;
    }
    const int64_t mn = (int64_t)m * n;
    if (!u8) return mn <= kLaneMaxMN ? 0 : kLaneNever;
    return mn <= 1024 ? 0 : 8192;
}

void set_survivor_lane_min(int m, int n, bool u8, int lane_min) {
    const auto key = std::make_tuple(current_device(), m, n, u8 ? 1 : 0);
    std::lock_guard<std::mutex> lk(g_form_mu);
    if (lane_min < 0) g_lane_min.erase(key); else g_lane_min[key] = lane_min;
}

// One template's state for an evaluation of given locations: every entry
// kept (bound above any rho), the whole list in one sweep.
static __global__ void survivor_eval_setup_kernel(TmplState *st, float *surv_ub, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        surv_ub[i] = 2.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->n_surv = count;
        st->n_surv_eff = count;
        st->n_first = 0;
        st->dense = 0;
    }
}

// Shared memory of the warp form (template, then each warp's double-buffered
// staging of kStageRows window rows when the template fits and the rows are
// narrow enough).
static size_t warp_form_smem(int m, int n, int npad, int *in_smem, int *stage) {
    size_t smem = tmpl_smem(m, npad, in_smem);
    smem = (smem + 15) & ~(size_t)15;
    const int WB = 16 * ((n + 30) / 16);
    *stage = *in_smem && n <= 256 ? 1 : 0;
    // (+16: a staged row's last word pair may reach 3 bytes past its row)
    if (*stage) smem += (size_t)8 * 2 * kStageRows * WB + 16;
    return smem;
}

cudaError_t launch_survivors(const Scan2Batch &B, const uint8_t *I, int pimg, int q, int Lx,
                             const int *wsum, int m, int n, int npad, const float *inv_sigma,
                             cudaStream_t s) {
    int in_smem = 0, stage = 0;
    const size_t smem = warp_form_smem(m, n, npad, &in_smem, &stage);
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(survivors_kernel), smem);
        if (e != cudaSuccess) return e;
    }
    const uint8_t *iend = I + (int64_t)q * pimg;
    Scan2Batch Bf = B;
    Bf.lane_min_u8 = survivor_lane_min(m, n, true);
    Bf.lane_min_f32 = survivor_lane_min(m, n, false);
    // buckets whose largest bound is below the certain lower bound already
    // reached (threshold centres and their groups) are cut off, then one sweep
    // -- or, with the dense path on, a first sweep over a bounded head of the
    // list, a second cut that also decides the dense templates, and a second
    // sweep over the rest of the others
    const bool two = B.dense_frac != 0.f;
    cudaError_t e;
    for (int phase = two ? 1 : 0; phase <= (two ? 2 : 0); ++phase) {
        Scan2Batch Bp = Bf;
        Bp.phase = phase;
        {
            LaunchScope ls("survivor_cut_kernel", s);
            survivor_cut_kernel<<<B.T, kUbBuckets, 0, s>>>(Bp, phase);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_sweep(Bp, I, q, Lx, wsum, m, n, npad, inv_sigma, in_smem, stage, smem, iend, s)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t launch_survivor_eval(const Scan2Batch &B, const uint8_t *I, int pimg, int q, int Lx,
                                 const int *wsum, int m, int n, int npad, const float *inv_sigma,
                                 int count, int form, cudaStream_t s) {
    if (B.T != 1 || count < 0 || count > B.scap || form < -1 || form > 1) return cudaErrorInvalidValue;
    if (count == 0) return cudaSuccess;
    int in_smem = 0, stage = 0;
    const size_t smem = warp_form_smem(m, n, npad, &in_smem, &stage);
    cudaError_t e = ensure_smem(reinterpret_cast<const void *>(survivors_kernel), smem);
    if (e != cudaSuccess) return e;
    {
        LaunchScope ls("survivor_eval_setup_kernel", s);
        survivor_eval_setup_kernel<<<grid_cap(count, 256, 4), 256, 0, s>>>(B.st, B.surv_ub, count);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Scan2Batch Bp = B;
    Bp.phase = 0;
    if (form >= 0) Bp.lane_min_u8 = Bp.lane_min_f32 = form == 0 ? 0 : kLaneNever;
    return launch_sweep(Bp, I, q, Lx, wsum, m, n, npad, inv_sigma, in_smem, stage, smem,
                        I + (int64_t)q * pimg, s);
}

cudaError_t launch_surv_candidates(const Scan2Batch &B, cudaStream_t s) {
    LaunchScope ls("surv_candidates_kernel", s);
    const int bx = std::max(1, num_sms() * 4 / std::min(B.T, 4));
    surv_candidates_kernel<<<dim3(bx, B.T), 256, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_group_members(const uint8_t *I, int q, int Ly, int Lx, int h, const int *wsum,
                                 const float *tf, size_t tsz, int m, int n,
                                 int npad, const float *inv_sigma, int T, TmplState *st,
                                 const int *cand_topk, int topk, cudaStream_t s) {
    int in_smem = 0;
    const size_t smem = tmpl_smem(m, npad, &in_smem);
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(group_members_kernel), smem);
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls("group_members_kernel", s);
    group_members_kernel<<<dim3(topk, T), 256, smem, s>>>(I, q, Ly, Lx, h, wsum, tf, tsz, m, n,
                                                          npad, inv_sigma, st, cand_topk, in_smem);
    return cudaGetLastError();
}


}  // namespace opta
