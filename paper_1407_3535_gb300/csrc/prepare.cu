// Preparation kernels (Sections 3-5): spatially varying Gaussian blur
// (Eq. defblur / Eq. Gauss), blur correlation with the lambda test
// (Algorithm 3, Eq. misDec), pivot auto-correlation maps and the EGS
// retained count (Algorithm 1, Algorithm 2 with Eq. co), per-centre pivot
// statistics.
//
// All correlation sums here are exact integer sums (uint8 x uint8 products
// in int32/int64, int64 integral images); only the final quotient is
// rounded, so |rho_co(fp32) - rho_co| <= ~5 u.
#include <algorithm>

#include "common.cuh"

namespace opta {

namespace {

// 4-byte asynchronous global -> shared copies (visible to the issuing thread
// after cp_async_wait_all).
__device__ inline void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int kMaxRadius = 9;

// One CTA per block x block output tile; sigma (level) fixed per tile and
// its radius R a template parameter (taps unrolled).  The tile and its
// R-wide halo (clamped to the image) are staged in shared memory as floats.
// The horizontal pass gives each thread kBlurCB consecutive outputs of one
// row, whose kBlurCB + 2R inputs it reads once into registers (a warp's
// threads take consecutive rows; row strides are odd, so they fall in
// distinct banks); the vertical pass gives each thread kBlurRB consecutive
// rows of one column.  Each output is w0 s0 + sum_j w_j (s_j + s_-j),
// accumulated in that order in FP32, then rounded to the nearest integer.
constexpr int kBlurThreads = 256;
constexpr int kBlurCB = 8;
constexpr int kBlurRB = 16;

__host__ __device__ inline size_t blur_smem_floats(int block, int R) {
    const int ih = block + 2 * R, iw = block + 2 * R;
    return (size_t)ih * (iw | 1) + (size_t)ih * (block | 1) + kBlurCB + 2 * R;
}

template <int R>
__device__ __forceinline__ void blur_tile(const uint8_t *__restrict__ I, int p, int q, int y0,
                                          int x0, int bh, int bw, const float *__restrict__ wg,
                                          uint8_t *P, float *bsm) {
    constexpr int CB = kBlurCB, RB = kBlurRB;
    float w[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) w[k] = wg[k];
    const int iw = bw + 2 * R, ih = bh + 2 * R;
    const int ist = iw | 1, hst = bw | 1;
    float *in = bsm;                 // ih x ist
    float *hb = bsm + ih * ist;      // ih x hst
    {
        // element i = (r, c) of the ih x iw tile, walked in strides of the
        // block (row and column advanced without division); unrolled so
        // that the loads of several elements are in flight together
        const int dr = kBlurThreads / iw, dc = kBlurThreads - dr * iw;
        int r = (int)threadIdx.x / iw, c = (int)threadIdx.x - r * iw;
#pragma unroll 4
        for (int i = threadIdx.x; i < ih * iw; i += kBlurThreads) {
            const int yy = min(max(y0 - R + r, 0), p - 1), xx = min(max(x0 - R + c, 0), q - 1);
            // the byte under the exponent of 2^23 is the float 2^23 + b: minus 2^23, b exactly
            in[r * ist + c] = __uint_as_float(0x4B000000u | I[(int64_t)yy * q + xx]) - 8388608.f;
            r += dr;
            c += dc;
            if (c >= iw) { c -= iw; ++r; }
        }
    }
    __syncthreads();
    const int ng = (bw + CB - 1) / CB;
    for (int item = threadIdx.x; item < ih * ng; item += kBlurThreads) {
        const int g = item / ih, r = item - g * ih;
        const int c0 = g * CB;
        const float *src = in + r * ist + c0;   // reads past the row land in the slack or the
        float sv[CB + 2 * R];                   // next row and only feed outputs past bw
#pragma unroll
        for (int k = 0; k < CB + 2 * R; ++k) sv[k] = src[k];
#pragma unroll
        for (int o = 0; o < CB; ++o) {
            float a = w[0] * sv[o + R];
#pragma unroll
            for (int t = 1; t <= R; ++t) a = fmaf(w[t], sv[o + R + t] + sv[o + R - t], a);
            if (c0 + o < bw) hb[r * hst + c0 + o] = a;
        }
    }
    __syncthreads();
    const int nrg = (bh + RB - 1) / RB;
    for (int item = threadIdx.x; item < bw * nrg; item += kBlurThreads) {
        const int g = item / bw, c = item - g * bw;
        const int r0 = g * RB;
        float sv[RB + 2 * R];
#pragma unroll
        for (int k = 0; k < RB + 2 * R; ++k) sv[k] = r0 + k < ih ? hb[(r0 + k) * hst + c] : 0.f;
#pragma unroll
        for (int o = 0; o < RB; ++o) {
            float a = w[0] * sv[o + R];
#pragma unroll
            for (int t = 1; t <= R; ++t) a = fmaf(w[t], sv[o + R + t] + sv[o + R - t], a);
            if (r0 + o < bh) {
                a = fminf(fmaxf(rintf(a), 0.f), 255.f);
                P[(int64_t)(y0 + r0 + o) * q + x0 + c] = (uint8_t)a;
            }
        }
    }
}

__global__ void __launch_bounds__(kBlurThreads)
blur_kernel(const uint8_t *__restrict__ I, int p, int q, const uint8_t *__restrict__ level_map,
            int block, const float *__restrict__ weights, const int *__restrict__ radius,
            uint8_t *P) {
    extern __shared__ float bsm[];
    const int bq = (q + block - 1) / block;
    const int by = blockIdx.y, bx = blockIdx.x;
    const int y0 = by * block, x0 = bx * block;
    const int lev = level_map[by * bq + bx];
    const int R = lev > 0 ? radius[lev] : 0;
    const int bh = min(block, p - y0), bw = min(block, q - x0);
    const float *w = weights + lev * (kMaxRadius + 1);
    switch (R) {
        case 1: blur_tile<1>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 2: blur_tile<2>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 3: blur_tile<3>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 4: blur_tile<4>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 5: blur_tile<5>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 6: blur_tile<6>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 7: blur_tile<7>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 8: blur_tile<8>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        case 9: blur_tile<9>(I, p, q, y0, x0, bh, bw, w, P, bsm); return;
        default: break;
    }
    // R = 0: the block is copied
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < bh; r += kBlurThreads / 32)
        for (int c = lane; c < bw; c += 32)
            P[(int64_t)(y0 + r) * q + x0 + c] = I[(int64_t)(y0 + r) * q + x0 + c];
}


// ---------------------------------------------------------------------------
// Pivot auto-correlation, Algorithm 1 with running sums.
//
// A CTA owns a strip of GXS groups (horizontally) by a band of GYB groups
// (vertically).  Thread j owns pivot column cx0 + j and keeps, for every
// shift s = (sy, sx) of the group, the column sum
//     colsum_s(r) = sum_{i<m} P(r+i, j) * I(r+i+sy, j+sx)
// which slides down H rows per group row (add the new bottom products,
// subtract the old top ones).  At each centre row the column sums are summed
// over the n pivot columns of each centre, giving the exact cross sum of the
// pivot block and the member block x = c + s.
//
// The slide works on 4-row words: the image rows sit column-major in a
// shared-memory ring (each column's ring slots packed 4 per 32-bit word), the
// pivot rows of one slide batch are packed 4 per word, and one dp4a (four
// uint8 x uint8 products summed into a 32-bit accumulator) takes four rows
// of one shift at once.  A funnel shift realigns the image words to the
// batch's first row and to each sy.
// ---------------------------------------------------------------------------
template <int H>
struct RcoCfg {
    static constexpr int R = (H - 1) / 2;
    static constexpr int NS = H * H;
    // threads per CTA at most (one per pivot column and per image ring
    // column): the H^2 column sums, the next row's slide data held across an
    // emission and the emission's 64-bit finish share 65536 / MAXT registers
    static constexpr int MAXT = H >= 9 ? 448 : (H >= 7 ? 640 : (H >= 5 ? 896 : 1024));
    static constexpr int KW = (H + 3) / 4;           // pivot words per batch
    static constexpr int BATCH = 4 * KW;             // rows per batch (>= H)
    static constexpr int NA = (H + BATCH + 2) / 4;   // aligned image words per column and batch
};

// Ring geometry shared by host and device: RING slots (a multiple of 4, at
// least the m + 2R + 1 rows one slide step needs plus the H rows loaded
// ahead), RW4 words per column, column stride CSW words (odd: conflict-free
// column-parallel reads).
__host__ __device__ inline int rco_ring(int m, int H) { return (m + (H - 1) + 1 + H + 3) & ~3; }
__host__ __device__ inline int rco_csw(int ring) { return (ring >> 2) | 1; }

// Pivot column jc, rows [prow, prow + cnt), packed 4 rows per word (zero
// past cnt, cnt <= BATCH): the loads are issued together.
template <int H>
__device__ __forceinline__ void rco_pcol(unsigned (&pw)[RcoCfg<H>::KW], const uint8_t *__restrict__ P,
                                         int q, int jc, int prow, int cnt) {
    constexpr int KW = RcoCfg<H>::KW;
#pragma unroll
    for (int w = 0; w < KW; ++w) {
        pw[w] = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * w + b;
            if (k < cnt) pw[w] |= (unsigned)P[(int64_t)(prow + k) * q + jc] << (8 * b);
        }
    }
}

// cs[sy][sx] += (or -=) sum_{k<cnt} P(prow+k, jc) * I(prow+k+sy-R, cx0+j+sx-R)
// for the packed pivot words pw of rows [prow, prow + cnt); image row rr
// lives in ring slot (rr + R) % RING.
template <int H, bool SUB>
__device__ __forceinline__ void rco_batch(int (&cs)[H * H], const unsigned (&pw)[RcoCfg<H>::KW],
                                          int prow, const unsigned *ringw, int j, int CSW, int RW4,
                                          int RING) {
    constexpr int KW = RcoCfg<H>::KW, NA = RcoCfg<H>::NA;
    const int slot0 = prow % RING;                  // slot of image row prow - R
    const unsigned sh = (unsigned)(slot0 & 3) * 8u;
    int woff[NA + 1];
    {
        int w = slot0 >> 2;
#pragma unroll
        for (int i = 0; i <= NA; ++i) {
            woff[i] = w;
            w = (w + 1 == RW4) ? 0 : w + 1;
        }
    }
#pragma unroll
    for (int sx = 0; sx < H; ++sx) {
        const unsigned *col = ringw + (j + sx) * CSW;
        unsigned wd[NA + 1];
#pragma unroll
        for (int i = 0; i <= NA; ++i) wd[i] = col[woff[i]];
        unsigned al[NA];                             // byte t = image row prow - R + t
#pragma unroll
        for (int i = 0; i < NA; ++i) al[i] = __funnelshift_r(wd[i], wd[i + 1], sh);
#pragma unroll
        for (int sy = 0; sy < H; ++sy) {
            unsigned acc = 0u;
#pragma unroll
            for (int w = 0; w < KW; ++w) {
                const int t = sy + 4 * w;
                const unsigned x = (t & 3) ? __funnelshift_r(al[t >> 2], al[(t >> 2) + 1], 8 * (t & 3))
                                           : al[t >> 2];
                acc = __dp4a(x, pw[w], acc);
            }
            if (SUB) cs[sy * H + sx] -= (int)acc;
            else cs[sy * H + sx] += (int)acc;
        }
    }
}

// One lane's blocks [k0, k1) of a column-sum row cr (blocks of H columns):
// pr[k] = the sum of blocks k0 .. k - 1, pr[NB + k] = the sum of block k's
// first NBc columns; returns the sum of all the lane's blocks.  NBc is a
// template parameter so that the split of a block costs no selects.
template <int H, int NBc>
__device__ __forceinline__ unsigned rco_blocks(const unsigned *cr, unsigned *pr, int k0, int k1,
                                               int NB) {
    unsigned run = 0u;
    for (int k = k0; k < k1; ++k) {
        const unsigned *cb = cr + k * H;
        unsigned pb = 0u;
#pragma unroll
        for (int c = 0; c < NBc; ++c) pb += cb[c];
        unsigned bs = pb;
#pragma unroll
        for (int c = NBc; c < H; ++c) bs += cb[c];
        pr[k] = run;
        pr[NB + k] = pb;
        run += bs;
    }
    return run;
}

// rco_blocks for the run-time split nb in [0, H) (uniform over the CTA)
template <int H, int NBc = 0>
__device__ __forceinline__ unsigned rco_blocks_nb(int nb, const unsigned *cr, unsigned *pr, int k0,
                                                  int k1, int NB) {
    if constexpr (NBc + 1 < H) {
        if (nb != NBc) return rco_blocks_nb<H, NBc + 1>(nb, cr, pr, k0, k1, NB);
    }
    return rco_blocks<H, NBc>(cr, pr, k0, k1, NB);
}

// Shared-memory words of one CTA (host and device agree on the layout):
// one emission buffer of K * H column-sum rows plus the two rows of the
// pivot statistics, their block prefixes (see block_rows), the per-centre
// statistics, each thread's pivot column sums and the image ring.
struct RcoSmem {
    int hsc, pre, cst, psq, ring, total;
    int nb, bpl, rwc, rwp;   // blocks per row, blocks per lane, words per column row / prefix row
};
template <int H>
__host__ __device__ inline RcoSmem rco_smem(int Wmax, int GXS, int CSW, int K, int n) {
    constexpr int R = RcoCfg<H>::R;
    RcoSmem l;
    l.nb = GXS + n / H + 1;              // blocks of H columns the windows reach
    l.bpl = ((l.nb + 31) / 32) | 1;      // blocks per lane (odd: the lanes' strides miss each other's banks)
    l.rwc = l.nb * H;                    // the columns the blocks read (> Wmax)
    l.rwp = 2 * l.nb + 2;
    const int rows = K * H + 2;
    int o = 0;
    l.hsc = o;  o += rows * l.rwc;
    l.pre = o;  o += rows * l.rwp;
    l.cst = o;  o += 2 * GXS;
    l.psq = o;  o += 2 * RcoCfg<H>::MAXT;
    l.ring = o; o += (Wmax + 2 * R) * CSW;
    l.total = o;
    return l;
}

template <int H>
__global__ void __launch_bounds__(RcoCfg<H>::MAXT, 1)
rho_co_kernel(const uint8_t *__restrict__ P, const uint8_t *__restrict__ I, int p, int q,
              int m, int n, int Ly, int Lx, const int *__restrict__ wsum,
              const float *__restrict__ inv_sigma, int GXS, int GYB, int GYS, int SUB, int K,
              float cut, float *rco, unsigned long long *count, float *c_inv_sigma, float *c_efac) {
    constexpr int R = RcoCfg<H>::R;
    constexpr int NS = RcoCfg<H>::NS;
    constexpr int KW = RcoCfg<H>::KW;
    constexpr int BATCH = RcoCfg<H>::BATCH;
    extern __shared__ unsigned rsm[];
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    // band blockIdx.y: group rows [gy0, gy0 + GYB); runs of SUB bands, runs
    // GYS apart (SUB = 1, GYS = GYB: every group row; GYS > SUB GYB: the
    // sampled runs of a count, each split into SUB bands)
    const int gx0 = blockIdx.x * GXS;
    const int gy0 = (blockIdx.y / SUB) * GYS + (blockIdx.y % SUB) * GYB;
    if (gx0 >= Gx || gy0 >= Gy) return;
    const int gx1 = min(Gx, gx0 + GXS), gy1 = min(Gy, gy0 + GYB);
    const int ngx = gx1 - gx0;
    const int cx0 = group_centre_of(gx0, Lx, H);
    const int W = group_centre_of(gx1 - 1, Lx, H) + n - cx0;   // pivot columns
    const int Wmax = (GXS - 1) * H + n;
    const int RING = rco_ring(m, H), RW4 = RING >> 2, CSW = rco_csw(RING);
    const int nwarps = blockDim.x >> 5;
    const RcoSmem L = rco_smem<H>(Wmax, GXS, CSW, K, n);
    const int NB = L.nb, BPL = L.bpl, RWc = L.rwc, RWp = L.rwp;
    unsigned *hsc = rsm + L.hsc;                                  // (K H + 2) x RWc column sums
    unsigned *pre = rsm + L.pre;                                  // (K H + 2) x RWp block prefixes
    int *cS = reinterpret_cast<int *>(rsm + L.cst);               // per centre: S_hat
    float *cI = reinterpret_cast<float *>(rsm + L.cst + GXS);     // per centre: 1/(mn Omega_hat)
    unsigned *psq = rsm + L.psq;                                  // [2][MAXT] column sums of P, P^2
    unsigned *ringw = rsm + L.ring;                               // (W + 2R) columns x CSW words
    uint8_t *ring8 = reinterpret_cast<uint8_t *>(ringw);
    const int j = threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = j < W;
    const long long mn = (long long)m * n;
    const unsigned mn32 = (unsigned)mn;                           // < 2^17 (see rco_geom)
    const int RW = W + 2 * R;                                     // ring columns used

    // image rows [r0, r0 + cnt) into their ring slots: columns across the
    // threads; a thread's rows are independent loads, issued together
    auto ring_put = [&](int slot, int col, uint8_t v) {
        ring8[(col * CSW + (slot >> 2)) * 4 + (slot & 3)] = v;
    };
    auto img_at = [&](int rr, int col) {
        return I[(int64_t)min(max(rr, 0), p - 1) * q + min(max(cx0 - R + col, 0), q - 1)];
    };
    auto load_rows = [&](int r0, int cnt) {          // any cnt (the initial fill)
        const int slot0 = (r0 + R) % RING;
        for (int col = threadIdx.x; col < RW; col += blockDim.x) {
            int slot = slot0;
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                ring_put(slot, col, img_at(r0 + k, col));
                slot = slot + 1 == RING ? 0 : slot + 1;
            }
        }
    };
    const int jc = cx0 + j;
    // Window sums at the centres.  The strip's centres are H columns apart
    // (centre gxi at column gxi * H), so a row of column sums is cut into
    // blocks of H columns: with n = a H + b, the window of centre gxi is
    // blocks gxi .. gxi + a - 1 plus the first b columns of block gxi + a.
    // One warp per row: each lane sums BPL consecutive blocks, the lane
    // totals are scanned, and the lane writes PrefB[k] (the sum of blocks
    // 0 .. k - 1) and PB[k] (the first b columns of block k).  The image's
    // last group, when shorter than H, has its centre dl columns before its
    // block: its window also takes the last dl columns of the block before
    // and a partial of b2 columns at its end (computed by lane 0).  Columns
    // past the strip hold stale sums; they only reach blocks no window uses.
    const int na = n / H, nb = n - na * H;
    int gxs = -1, dl = 0, a2 = 0, b2 = 0;
    if (gx1 == Gx && ngx >= 2) {
        const int ls = Lx - (Gx - 1) * H;   // size of the image's last group
        if (ls < H) {
            gxs = ngx - 1;
            dl = R - (ls - 1) / 2;
            a2 = (n - dl) / H;
            b2 = n - dl - a2 * H;
        }
    }
    auto block_rows = [&](int nrows) {
        for (int rr = warp; rr < nrows; rr += nwarps) {
            const unsigned *cr = hsc + rr * RWc;
            unsigned *pr = pre + rr * RWp;
            const int k0 = lane * BPL, k1 = min(NB, k0 + BPL);
            // one read of the lane's columns: block partials and prefixes
            // relative to the lane's first block, then the lane offsets
            const unsigned run = rco_blocks_nb<H>(nb, cr, pr, k0, k1, NB);
            unsigned inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            const unsigned off = inc - run;
            for (int k = k0; k < k1; ++k) pr[k] += off;
            if (gxs >= 0 && lane == 0) {
                unsigned s1 = 0u, s2 = 0u;
                for (int c = gxs * H - dl; c < gxs * H; ++c) s1 += cr[c];
                for (int c = (gxs + a2) * H; c < (gxs + a2) * H + b2; ++c) s2 += cr[c];
                pr[2 * NB] = s1;
                pr[2 * NB + 1] = s2;
            }
        }
    };
    // sum of a row over the window of centre gxi (modulo 2^32)
    auto xsum = [&](const unsigned *pr, int gxi) -> unsigned {
        if (gxi == gxs) return pr[2 * NB] + (pr[gxs + a2] - pr[gxs]) + pr[2 * NB + 1];
        return (pr[gxi + na] - pr[gxi]) + pr[NB + gxi + na];
    };

    // constants of this thread's first emission task (centre gxi, shift
    // column sxi): its member column; further tasks (n < H only) take the
    // loop
    const int t0_gxi = (int)threadIdx.x / H, t0_sxi = (int)threadIdx.x - t0_gxi * H;
    int t0_mx;
    bool t0_ok;
    {
        const int gx = gx0 + t0_gxi;
        const int cxg = group_centre_of(gx, Lx, H);
        t0_mx = cxg + t0_sxi - R;
        t0_ok = (int)threadIdx.x < ngx * H && t0_mx >= gx * H && t0_mx < min(gx * H + H, Lx);
    }

    int r = group_centre_of(gy0, Ly, H);
    load_rows(r - R, m + 2 * R + 1);
    int cs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cs[s] = 0;
    // this column's pivot sum and square sum over the window rows, slid with
    // cs and kept in shared memory (read once per group row)
    unsigned *ps_j = psq + j, *pq_j = psq + RcoCfg<H>::MAXT + j;
    __syncthreads();
    if (active) {
        unsigned ps = 0u, pq = 0u;
        for (int b0 = 0; b0 < m; b0 += BATCH) {
            unsigned pw[KW];
            rco_pcol<H>(pw, P, q, jc, r + b0, min(BATCH, m - b0));
            rco_batch<H, false>(cs, pw, r + b0, ringw, j, CSW, RW4, RING);
#pragma unroll
            for (int w = 0; w < KW; ++w) {
                ps = __dp4a(pw[w], 0x01010101u, ps);
                pq = __dp4a(pw[w], pw[w], pq);
            }
        }
        *ps_j = ps;
        *pq_j = pq;
    }
    unsigned local = 0;                      // this thread's locations below the cut
    const int ntask = ngx * H;
    // The next group row's slide data (this column's pivot bytes entering
    // and leaving the window, and the image rows up to r + steps - 1 + m + R
    // for ring column j) is loaded into registers before this row's emission,
    // the image rows stored into the ring after the emission's block pass and
    // the pivot bytes slid after its tasks, so that the loads' latency hides
    // behind the emission and the emission's last barrier also publishes the
    // ring rows (no barrier between one row's tasks and the next row's
    // slide).  The ring slots it overwrites hold rows above r - R that no
    // slide reads again (the emission does not read the ring).
    unsigned pa[KW], pr[KW];
    uint8_t iv[H];
    int steps = 0;                           // rows to the next centre row (<= H)
    auto fetch = [&](int gy) {
        steps = gy < gy1 ? group_centre_of(gy, Ly, H) - r : 0;
        if (steps <= 0) return;
        if (active) {
            rco_pcol<H>(pa, P, q, jc, r + m, steps);
            rco_pcol<H>(pr, P, q, jc, r, steps);
        }
        if (j < RW) {
#pragma unroll
            for (int k = 0; k < H; ++k) iv[k] = k < steps ? img_at(r + m + R + 1 + k, j) : (uint8_t)0;
        }
    };
    for (int gy = gy0; gy < gy1; ++gy) {
        const int cy = group_centre_of(gy, Ly, H);
        if (gy > gy0 && steps > 0) {
            if (active) {
                rco_batch<H, false>(cs, pa, r + m, ringw, j, CSW, RW4, RING);
                rco_batch<H, true>(cs, pr, r, ringw, j, CSW, RW4, RING);
                unsigned dps = 0u, dpq = 0u;
#pragma unroll
                for (int w = 0; w < KW; ++w) {
                    dps += __dp4a(pa[w], 0x01010101u, 0u) - __dp4a(pr[w], 0x01010101u, 0u);
                    dpq += __dp4a(pa[w], pa[w], 0u) - __dp4a(pr[w], pr[w], 0u);
                }
                *ps_j += dps;
                *pq_j += dpq;
            }
            r += steps;
            // (no barrier: the emission reads no ring slot, and its first
            // barrier orders this slide before the next ring stores; the
            // emission's hsc stores do not touch the prefixes that other
            // threads' tasks of the previous row may still read)
        }
        fetch(gy + 1);
        // emission of centre row cy in chunks of K shift rows (sy): the chunk's
        // K H column-sum rows (and, in the first chunk, the column sums of P
        // and P^2 for the pivot statistics) are stored, cut into blocks
        // together and read by the tasks
        const int gys = gy * H, gye = min(gys + H, Ly);
        for (int k0 = 0; k0 < H; k0 += K) {
            const int kn = min(K, H - k0);
            const bool first = k0 == 0;
            const int rb = first ? 2 : 0;              // first shift row of the chunk
            if (!first) __syncthreads();               // the previous chunk's tasks are done
            // this thread's first task's member statistics for the chunk's
            // shift rows, brought into L1 now and read after the scan
#pragma unroll
            for (int syi = 0; syi < H; ++syi) {
                const int my = cy + syi - R;
                if (t0_ok && syi >= k0 && syi < k0 + kn && my >= gys && my < gye) {
                    const int64_t li = (int64_t)my * Lx + t0_mx;
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(wsum + li));
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(inv_sigma + li));
                }
            }
            if (active) {
                if (first) {
                    hsc[j] = *ps_j;
                    hsc[RWc + j] = *pq_j;
                }
#pragma unroll
                for (int syi = 0; syi < H; ++syi) {
                    if (syi < k0 || syi >= k0 + kn) continue;
#pragma unroll
                    for (int sxi = 0; sxi < H; ++sxi)
                        hsc[(rb + (syi - k0) * H + sxi) * RWc + j] = (unsigned)cs[syi * H + sxi];
                }
            }
            __syncthreads();
            block_rows(rb + kn * H);
            __syncthreads();
            if (first) {
                // the next row's image rows into the ring (their loads were
                // issued before this emission)
                if (steps > 0 && j < RW) {
                    int slot = (r + m + 2 * R + 1) % RING;
#pragma unroll
                    for (int k = 0; k < H; ++k) {
                        if (k < steps) ring_put(slot, j, iv[k]);
                        slot = slot + 1 == RING ? 0 : slot + 1;
                    }
                }
                // pivot statistics of this row's centres: window sums of the
                // column sums of P and P^2 (exact, < 2^32)
                if ((int)threadIdx.x < ngx) {
                    const int gx = gx0 + threadIdx.x;
                    const long long Sp = xsum(pre, threadIdx.x), Qp = xsum(pre + RWp, threadIdx.x);
                    const long long var = mn * Qp - Sp * Sp;   // exact
                    cS[threadIdx.x] = (int)Sp;
                    // 1 / (mn Omega_hat) = sqrt(mn / var) / mn
                    const float fmn = i64_to_f32(mn), fv = i64_to_f32(var);
                    cI[threadIdx.x] = var > 0 ? sqrtf(fmn / fv) / fmn : 0.f;
                    if (c_inv_sigma) {
                        // per-centre statistics of scan 1: 1/sigma_hat and ||P - 128|| / sigma_hat
                        const int64_t g = (int64_t)gy * Gx + gx;
                        c_inv_sigma[g] = var > 0 ? sqrtf(fmn / fv) : 0.f;
                        c_efac[g] = var > 0 ? sqrtf(fmn * i64_to_f32(Qp - 256 * Sp + 16384 * mn) / fv) : 0.f;
                    }
                }
                __syncthreads();
            }
            // task = (centre gxi, shift column sxi): X = window sum over pivot
            // columns [c1, c1 + n); rho = (mn X - S_hat S) / (mn Omega_hat
            // Omega): exact integer numerator, FP32 finish (flat windows have
            // 1/Omega = 0 -> 0)
#pragma unroll
            for (int syi = 0; syi < H; ++syi) {
                if (syi < k0 || syi >= k0 + kn) continue;
                const int my = cy + syi - R;
                if (my < gys || my >= gye) continue;   // uniform over the block
                const int row = rb + (syi - k0) * H;
                if (t0_ok) {
                    const int64_t li = (int64_t)my * Lx + t0_mx;
                    const int ws = wsum[li];
                    const float iw = inv_sigma[li];
                    const unsigned X = xsum(pre + (row + t0_sxi) * RWp, t0_gxi);
                    const long long num = mul_sub_wide(mn32, X, cS[t0_gxi], ws);
                    const float rho = (i64_to_f32(num) * iw) * cI[t0_gxi];
                    if (rco) rco[li] = rho;
                    if (rho < cut) ++local;
                }
                for (int task = threadIdx.x + blockDim.x; task < ntask; task += blockDim.x) {
                    const int gxi = task / H, sxi = task - gxi * H;
                    const int gx = gx0 + gxi;
                    const int cxg = group_centre_of(gx, Lx, H);
                    const int mx = cxg + sxi - R;
                    if (mx < gx * H || mx >= min(gx * H + H, Lx)) continue;
                    const int64_t li = (int64_t)my * Lx + mx;
                    const int ws = wsum[li];
                    const float iw = inv_sigma[li];
                    const unsigned X = xsum(pre + (row + sxi) * RWp, gxi);
                    const long long num = mul_sub_wide(mn32, X, cS[gxi], ws);
                    const float rho = (i64_to_f32(num) * iw) * cI[gxi];
                    if (rco) rco[li] = rho;
                    if (rho < cut) ++local;
                }
            }
        }
    }
    if (count) {
        unsigned long long tot = local;
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(count, tot);
    }
}

// R_oo(x) = rho(P window, I window) at every location (Algorithm 3) and the
// lambda test, straight from P and I.  A CTA takes a strip of output columns
// (one thread per input column: the strip's n - 1 extra columns included)
// and a band of output rows.  Each thread slides its column's sums of P, P^2
// and P*I down the window rows, kBcRows output rows per round, into shared
// memory; one warp then turns each such row into running sums along the
// strip (32 consecutive columns per lane, rows padded to 33 words per lane
// so that the lanes' accesses fall in distinct banks), and each window sum
// over n columns is the difference of two running sums (modulo 2^32: the
// window sums themselves fit in 32 bits).  I's window statistics come from
// the window-sum and 1/Omega maps, copied to shared memory (cp.async) for a
// round's rows while its sums slide and are scanned; the slide's image bytes
// of a round are loaded together, four rows per register.
constexpr int kBcRows = 10;                  // output rows per round (3 scanned rows each)
constexpr int kBcThreads = 1024;             // input columns per strip at most
constexpr int kBcLaneW = 33;                 // words per lane in a scanned row
constexpr int kBcRS = 32 * kBcLaneW;         // words per scanned row

__device__ __forceinline__ int bc_addr(int c) { return (c >> 5) * kBcLaneW + (c & 31); }

constexpr size_t kBcSmem = (size_t)3 * kBcRows * kBcRS * sizeof(unsigned) +   // scanned rows
                           (size_t)2 * kBcRows * kBcThreads * sizeof(int);        // member statistics

__global__ void __launch_bounds__(kBcThreads, 1)
blur_corr_kernel(const uint8_t *__restrict__ P, const uint8_t *__restrict__ I, int p, int q,
                 int m, int n, int Ly, int Lx, const int *__restrict__ wsum,
                 const float *__restrict__ inv_sigma, int WO, int BR, float lambda, int block,
                 int *fail, float *R) {
    extern __shared__ unsigned bcs[];        // 3 * kBcRows rows x kBcRS
    int *tws = reinterpret_cast<int *>(bcs + 3 * kBcRows * kBcRS);          // [kBcRows][kBcThreads]
    float *tiw = reinterpret_cast<float *>(tws + kBcRows * kBcThreads);     // [kBcRows][kBcThreads]
    const int x0 = blockIdx.x * WO, y0 = blockIdx.y * BR;
    if (x0 >= Lx || y0 >= Ly) return;
    const int wo = min(WO, Lx - x0), y1 = min(Ly, y0 + BR);
    const int W = wo + n - 1;                // input columns of the strip
    const int j = threadIdx.x, lane = j & 31, warp = j >> 5, nwarps = blockDim.x >> 5;
    const bool active = j < W;
    const int xc = x0 + j;
    const long long mn = (long long)m * n;
    const unsigned mn32 = (unsigned)mn;      // < 2^17 (window sums of products fit 32 bits)
    const float fmn = i64_to_f32(mn);
    const int bq = (q + block - 1) / block;
    const int aj = bc_addr(j);
    const int lane_cnt = W - 32 * lane;      // columns of the strip held by this lane in a scan
    // lambda test: one flag per thread and block row (the thread's x is fixed)
    const int bx = (x0 + j) / block;
    int by = y0 / block, by_end = (by + 1) * block;
    bool failed = false;
    // column sums over the window rows [y, y + m)
    unsigned sp = 0u, sq = 0u, sx = 0u;
    if (active) {
        const uint8_t *pc = P + (int64_t)y0 * q + xc, *ic = I + (int64_t)y0 * q + xc;
#pragma unroll 8
        for (int u = 0; u < m; ++u, pc += q, ic += q) {
            const unsigned pv = *pc, iv = *ic;
            sp += pv;
            sq += pv * pv;
            sx += pv * iv;
        }
    }
    constexpr int kBcW = (kBcRows + 3) / 4;  // packed words per slid image row set
    for (int yr = y0; yr < y1; yr += kBcRows) {
        const int nr = min(kBcRows, y1 - yr);
        // member statistics of the round's locations, copied while the sums slide
        if (j < wo) {
            for (int k = 0; k < nr; ++k) {
                const int64_t li = (int64_t)(yr + k) * Lx + x0 + j;
                cp_async4(tws + k * kBcThreads + j, wsum + li);
                cp_async4(tiw + k * kBcThreads + j, inv_sigma + li);
            }
        }
        cp_async_commit();
        // the column sums of rows yr .. yr + nr - 1, sliding between them
        // (nsl steps: not past the band's last row)
        const int nsl = min(nr, y1 - 1 - yr);
        if (active) {
            const uint8_t *pa = P + (int64_t)(yr + m) * q + xc, *ia = I + (int64_t)(yr + m) * q + xc;
            const uint8_t *po = P + (int64_t)yr * q + xc, *io = I + (int64_t)yr * q + xc;
            unsigned wa[kBcW], wai[kBcW], wo_[kBcW], woi[kBcW];
#pragma unroll
            for (int w = 0; w < kBcW; ++w) wa[w] = wai[w] = wo_[w] = woi[w] = 0u;
#pragma unroll
            for (int k = 0; k < kBcRows; ++k) {
                if (k < nsl) {
                    const int sh = 8 * (k & 3);
                    wa[k >> 2] |= (unsigned)pa[(int64_t)k * q] << sh;
                    wai[k >> 2] |= (unsigned)ia[(int64_t)k * q] << sh;
                    wo_[k >> 2] |= (unsigned)po[(int64_t)k * q] << sh;
                    woi[k >> 2] |= (unsigned)io[(int64_t)k * q] << sh;
                }
            }
#pragma unroll
            for (int k = 0; k < kBcRows; ++k) {
                if (k < nr) {
                    bcs[(3 * k) * kBcRS + aj] = sp;
                    bcs[(3 * k + 1) * kBcRS + aj] = sq;
                    bcs[(3 * k + 2) * kBcRS + aj] = sx;
                    const int sh = 8 * (k & 3);
                    const unsigned a = (wa[k >> 2] >> sh) & 255u, ai = (wai[k >> 2] >> sh) & 255u;
                    const unsigned o = (wo_[k >> 2] >> sh) & 255u, oi = (woi[k >> 2] >> sh) & 255u;
                    sp += a - o;             // zero past the slid rows
                    sq += a * a - o * o;
                    sx += a * ai - o * oi;
                }
            }
        }
        __syncthreads();
        // running sums along each row, one warp per row
        for (int row = warp; row < 3 * nr; row += nwarps) {
            unsigned *lp = bcs + row * kBcRS + lane * kBcLaneW;
            unsigned v[32];
            unsigned tot = 0u;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                v[i] = i < lane_cnt ? lp[i] : 0u;
                tot += v[i];
            }
            unsigned inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            unsigned run = inc - tot;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                run += v[i];
                lp[i] = run;
            }
        }
        cp_async_wait_all();   // this thread's member statistics (read by this thread only)
        __syncthreads();
        if (j < wo) {
            const int x = x0 + j;
            const int a2 = bc_addr(j + n - 1), a1 = j > 0 ? bc_addr(j - 1) : 0;
            const unsigned keep = j > 0 ? 0xffffffffu : 0u;   // running sum before column 0 is 0
            for (int k = 0; k < nr; ++k) {
                const unsigned *r0 = bcs + (3 * k) * kBcRS;
                const unsigned Sp = r0[a2] - (r0[a1] & keep);
                const unsigned Qp = r0[kBcRS + a2] - (r0[kBcRS + a1] & keep);
                const unsigned X = r0[2 * kBcRS + a2] - (r0[2 * kBcRS + a1] & keep);
                const int y = yr + k;
                const int64_t i = (int64_t)y * Lx + x;
                const long long dA = mul_sub_wide(mn32, Qp, (int)Sp, (int)Sp);                  // exact
                const long long num = mul_sub_wide(mn32, X, (int)Sp, tws[k * kBcThreads + j]);   // exact
                const float iw = tiw[k * kBcThreads + j];                    // 0: flat I window
                float r = 0.f;
                if (dA > 0 && iw > 0.f) r = (i64_to_f32(num) * iw) * rsqrtf(i64_to_f32(dA) * fmn);
                if (R) R[i] = r;
                if (y >= by_end) {
                    if (failed && fail) {
                        int *f = fail + by * bq + bx;
                        if (*f == 0) atomicOr(f, 1);
                    }
                    failed = false;
                    by = y / block;
                    by_end = (by + 1) * block;
                }
                failed |= iw > 0.f && r < lambda;
            }
        }
        __syncthreads();   // the next round overwrites the scanned rows
    }
    if (failed && fail && j < wo) {
        int *f = fail + by * bq + bx;
        if (*f == 0) atomicOr(f, 1);
    }
}

struct RcoGeom {
    bool ok;
    int GXS, Wmax, threads, strips, K;
    size_t smem;
};

// Launch geometry: strips of GXS group columns (one thread per pivot column
// of the strip), bands of GYB group rows; shared memory = H slide rows of
// column prefix sums and their warp totals, the per-centre statistics of one
// group row and the packed image ring.
template <int H>
RcoGeom rco_geom(int p, int q, int m, int n) {
    constexpr int MAXT = RcoCfg<H>::MAXT;
    constexpr size_t kSmemMax = 227 * 1024;
    RcoGeom g{};
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    // window sums of uint8 products are kept in 32 bits
    if (n + 2 * H > MAXT || (uint64_t)m * n * 65025u > 0xffffffffull) return g;
    const int csw = rco_csw(rco_ring(m, H));
    auto smem_for = [&](int gxs, int k, int *wmax) {
        *wmax = (gxs - 1) * H + n;
        return (size_t)rco_smem<H>(*wmax, gxs, csw, k, n).total * sizeof(unsigned);
    };
    // the most shift rows per emission (K) that fit beside the image ring
    auto best_k = [&](int gxs, size_t *smem, int *wmax) {
        for (int k = H; k >= 1; --k) {
            *smem = smem_for(gxs, k, wmax);
            if (*smem <= kSmemMax) return k;
        }
        return 0;
    };
    // widest strip within the thread limit, narrowed until the ring and one
    // shift row per emission fit
    g.GXS = std::min((MAXT - n - (H - 1)) / H + 1, Gx);
    g.K = best_k(g.GXS, &g.smem, &g.Wmax);
    while (g.K == 0 && g.GXS > 1) {
        g.GXS = std::max(1, g.GXS - std::max(1, g.GXS / 8));
        g.K = best_k(g.GXS, &g.smem, &g.Wmax);
    }
    g.ok = g.K > 0;
    if (!g.ok) return g;
    // strips of equal width (narrower than the limit: the last strip is not
    // left with a remainder while the others carry the rest), then again the
    // most shift rows per emission at that width
    g.strips = (Gx + g.GXS - 1) / g.GXS;
    g.GXS = (Gx + g.strips - 1) / g.strips;
    g.K = best_k(g.GXS, &g.smem, &g.Wmax);
    // a thread per pivot column and per image ring column (W + 2R of them)
    g.threads = ((g.Wmax + (H - 1) + 31) / 32) * 32;
    (void)Gy;
    return g;
}

template <int H>
cudaError_t launch_rho_co_h(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                            const int *wsum, const float *inv_sigma, float cut, float *rco,
                            unsigned long long *count, float *c_inv_sigma, float *c_efac,
                            int sample, cudaStream_t s) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    const RcoGeom g = rco_geom<H>(p, q, m, n);
    if (!g.ok) return cudaErrorInvalidValue;
    const size_t smem = g.smem;
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(rho_co_kernel<H>), smem);
        if (e != cudaSuccess) return e;
    }
    // one wave: strips x bands CTAs fill the SMs once (each CTA slides its
    // band from one initial build, so fewer, taller bands pay it less often)
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rho_co_kernel<H>, g.threads, smem) !=
            cudaSuccess || bps < 1) {
        cudaGetLastError();
        bps = 1;
    }
    const int Gy = groups_along(Ly, H);
    int GYB, GYS, bands, sub = 1;
    if (sample > 1) {
        // a count over the sampled runs only (kEgsRun group rows, every
        // sample-th run), each run split into sub bands: a band's time is
        // about its rows (its group rows' H rows each, plus the m - 1 rows
        // its windows reach below), so a run is split while the CTAs still
        // fit in fewer waves than the rows saved
        GYS = kEgsRun * sample;
        const int runs = (Gy + GYS - 1) / GYS;
        double best = 0.0;
        for (int d = 1; d <= kEgsRun; d *= 2) {
            const int64_t ctas = (int64_t)g.strips * runs * d;
            const int64_t waves = (ctas + (int64_t)num_sms() * bps - 1) / ((int64_t)num_sms() * bps);
            const double t = (double)waves * (double)((kEgsRun / d) * H + m - 1);
            if (d == 1 || t < best) { best = t; sub = d; }
        }
        GYB = kEgsRun / sub;
        bands = runs * sub;
    } else {
        bands = std::max(1, std::min(Gy, num_sms() * bps / g.strips));
        GYB = (Gy + bands - 1) / bands;
        GYS = GYB;
        bands = (Gy + GYB - 1) / GYB;
    }
    dim3 grid(g.strips, bands);
    // launches are timed under the group side's name, so that the work of
    // each (the H^2 shifts it slides) can be told apart
    static_assert(H >= 1 && H <= 9 && (H & 1), "odd group sides up to 9");
    static const char *const kName[10] = {"", "rho_co_kernel<1>", "", "rho_co_kernel<3>", "",
                                          "rho_co_kernel<5>", "", "rho_co_kernel<7>", "",
                                          "rho_co_kernel<9>"};
    // count-only launches (EGS trials) are timed apart from map emissions
    static const char *const kCountName[10] = {"", "rho_co_count<1>", "", "rho_co_count<3>", "",
                                               "rho_co_count<5>", "", "rho_co_count<7>", "",
                                               "rho_co_count<9>"};
    const bool count_only = !rco && !c_inv_sigma && !c_efac;
    LaunchScope ls_rho_co_kernel(count_only ? kCountName[H] : kName[H], s);
    rho_co_kernel<H><<<grid, g.threads, smem, s>>>(P, I, p, q, m, n, Ly, Lx, wsum, inv_sigma,
                                                   g.GXS, GYB, GYS, sub, g.K, cut, rco, count,
                                                   c_inv_sigma, c_efac);
    return cudaGetLastError();
}

}  // namespace

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_blur(const uint8_t *I, int p, int q, const uint8_t *level_map, int block,
                        const float *weights, const int *radius, uint8_t *P, cudaStream_t s) {
    const int bp = (p + block - 1) / block, bq = (q + block - 1) / block;
    const size_t smem = blur_smem_floats(block, kMaxRadius) * sizeof(float);
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(blur_kernel), smem);
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls_blur_kernel("blur_kernel", s);
    blur_kernel<<<dim3(bq, bp), kBlurThreads, smem, s>>>(I, p, q, level_map, block, weights,
                                                        radius, P);
    return cudaGetLastError();
}

cudaError_t launch_blur_corr(const uint8_t *P, const uint8_t *I, const int *wsum,
                             const float *inv_sigma, int p, int q, int m, int n, float lambda,
                             int block, int *fail, float *R, cudaStream_t s) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    // one thread per strip column; window sums of uint8 products in 32 bits
    if (n > kBcThreads || (uint64_t)m * n * 65025u > 0xffffffffull) return cudaErrorInvalidValue;
    // strips of equal width (one input column per thread), and bands so that
    // all CTAs run in one wave, one per SM
    const int strips = (Lx + (kBcThreads - n + 1) - 1) / (kBcThreads - n + 1);
    const int WO = (Lx + strips - 1) / strips;
    const int threads = ((WO + n - 1) + 31) & ~31;
    int bands = std::max(1, std::min(Ly, num_sms() / strips));
    const int BR = (Ly + bands - 1) / bands;
    bands = (Ly + BR - 1) / BR;
    const size_t smem = kBcSmem;
    {
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(blur_corr_kernel), smem);
        if (e != cudaSuccess) return e;
    }
    LaunchScope ls_blur_corr_kernel("blur_corr_kernel", s);
    blur_corr_kernel<<<dim3(strips, bands), threads, smem, s>>>(P, I, p, q, m, n, Ly, Lx, wsum,
                                                               inv_sigma, WO, BR, lambda, block,
                                                               fail, R);
    return cudaGetLastError();
}

bool rho_co_supported(int p, int q, int m, int n, int h) {
    switch (h) {
        case 1: return rco_geom<1>(p, q, m, n).ok;
        case 3: return rco_geom<3>(p, q, m, n).ok;
        case 5: return rco_geom<5>(p, q, m, n).ok;
        case 7: return rco_geom<7>(p, q, m, n).ok;
        case 9: return rco_geom<9>(p, q, m, n).ok;
        default: return false;
    }
}

cudaError_t launch_rho_co(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                          int h, const int *wsum, const float *inv_sigma, float cut, float *rco,
                          unsigned long long *count, float *c_inv_sigma, float *c_efac,
                          cudaStream_t s, int sample) {
    if (sample > 1 && (rco || c_inv_sigma || c_efac)) return cudaErrorInvalidValue;   // counts only
    switch (h) {
        case 1: return launch_rho_co_h<1>(P, I, p, q, m, n, wsum, inv_sigma, cut, rco, count, c_inv_sigma, c_efac, sample, s);
        case 3: return launch_rho_co_h<3>(P, I, p, q, m, n, wsum, inv_sigma, cut, rco, count, c_inv_sigma, c_efac, sample, s);
        case 5: return launch_rho_co_h<5>(P, I, p, q, m, n, wsum, inv_sigma, cut, rco, count, c_inv_sigma, c_efac, sample, s);
        case 7: return launch_rho_co_h<7>(P, I, p, q, m, n, wsum, inv_sigma, cut, rco, count, c_inv_sigma, c_efac, sample, s);
        case 9: return launch_rho_co_h<9>(P, I, p, q, m, n, wsum, inv_sigma, cut, rco, count, c_inv_sigma, c_efac, sample, s);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace opta
