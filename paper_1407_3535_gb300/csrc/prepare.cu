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

constexpr int kMaxRadius = 9;

// One CTA per block x block output tile; sigma (level) fixed per tile.
__global__ void blur_kernel(const uint8_t *__restrict__ I, int p, int q,
                            const uint8_t *__restrict__ level_map, int block,
                            const float *__restrict__ weights, const int *__restrict__ radius,
                            uint8_t *P) {
    extern __shared__ float bsm[];
    const int bq = (q + block - 1) / block;
    const int by = blockIdx.y, bx = blockIdx.x;
    const int y0 = by * block, x0 = bx * block;
    const int lev = level_map[by * bq + bx];
    const int R = lev > 0 ? radius[lev] : 0;
    const int bh = min(block, p - y0), bw = min(block, q - x0);
    if (R == 0) {
        for (int i = threadIdx.x; i < bh * bw; i += blockDim.x) {
            const int r = i / bw, c = i % bw;
            P[(int64_t)(y0 + r) * q + x0 + c] = I[(int64_t)(y0 + r) * q + x0 + c];
        }
        return;
    }
    const float *w = weights + lev * (kMaxRadius + 1);
    const int iw = bw + 2 * R, ih = bh + 2 * R;
    float *in = bsm;                 // ih x iw
    float *hb = bsm + ih * iw;       // ih x bw
    for (int i = threadIdx.x; i < ih * iw; i += blockDim.x) {
        const int r = i / iw, c = i % iw;
        const int yy = min(max(y0 - R + r, 0), p - 1);
        const int xx = min(max(x0 - R + c, 0), q - 1);
        in[i] = (float)I[(int64_t)yy * q + xx];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ih * bw; i += blockDim.x) {
        const int r = i / bw, c = i % bw;
        const float *src = in + r * iw + c + R;
        float a = w[0] * src[0];
        for (int j = 1; j <= R; ++j) a = fmaf(w[j], src[j] + src[-j], a);
        hb[i] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < bh * bw; i += blockDim.x) {
        const int r = i / bw, c = i % bw;
        const float *src = hb + (r + R) * bw + c;
        float a = w[0] * src[0];
        for (int j = 1; j <= R; ++j) a = fmaf(w[j], src[j * bw] + src[-j * bw], a);
        a = fminf(fmaxf(rintf(a), 0.f), 255.f);
        P[(int64_t)(y0 + r) * q + x0 + c] = (uint8_t)a;
    }
}


// R_oo(x) = rho(P window, I window) (Algorithm 3) and the lambda test.
__global__ void blur_corr_kernel(const int *__restrict__ wsum, const float *__restrict__ inv_sigma,
                                 const long long *__restrict__ PS, const long long *__restrict__ PQ,
                                 const long long *__restrict__ PX, int q, int Ly, int Lx, int m,
                                 int n, float lambda, int block, int *fail, float *R) {
    const int64_t L = (int64_t)Ly * Lx;
    const int64_t q1 = q + 1;
    const long long mn = (long long)m * n;
    const int bq = (q + block - 1) / block;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ii = (int)i;
        const int y = ii / Lx, x = ii - y * Lx;
        const long long Sp = ii_box(PS, q1, y, x, m, n), Qp = ii_box(PQ, q1, y, x, m, n);
        const long long X = ii_box(PX, q1, y, x, m, n);
        const long long dA = mn * Qp - Sp * Sp;                        // exact
        const long long num = mn * X - Sp * (long long)wsum[i];        // exact
        const float iw = inv_sigma[i];                                 // 0: flat I window
        float r = 0.f;
        if (dA > 0 && iw > 0.f)
            r = ((float)num * iw) * (sqrtf((float)mn / (float)dA) / (float)mn);
        if (R) R[i] = r;
        if (fail && iw > 0.f && r < lambda) {
            int *f = fail + (y / block) * bq + (x / block);
            if (*f == 0) atomicOr(f, 1);
        }
    }
}

// Per-centre pivot statistics.
__global__ void centre_stats_kernel(const long long *__restrict__ PS, const long long *__restrict__ PQ,
                                    int q, int m, int n, int h, int Ly, int Lx,
                                    float *c_inv_sigma, float *c_efac) {
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    const int64_t G = (int64_t)Gy * Gx;
    const int64_t q1 = q + 1;
    const double mn = (double)m * n;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int cy = group_centre_of((int)(g / Gx), Ly, h);
        const int cx = group_centre_of((int)(g % Gx), Lx, h);
        const long long S = ii_box(PS, q1, cy, cx, m, n), Q = ii_box(PQ, q1, cy, cx, m, n);
        const long long imn = (long long)m * n;
        const long long var = imn * Q - S * S;   // exact
        float is = 0.f, ef = 0.f;
        if (var > 0) {
            const float fv = (float)var, fmn = (float)mn;
            is = sqrtf(fmn / fv);
            ef = sqrtf(fmn * (float)(Q - 256 * S + 16384 * imn) / fv);
        }
        c_inv_sigma[g] = is;
        c_efac[g] = ef;
    }
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
    static constexpr int MAXT = H >= 9 ? 512 : (H >= 7 ? 640 : 1024);
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

// cs[sy][sx] += (or -=) sum_{k<cnt} P(prow+k, jc) * I(prow+k+sy-R, cx0+j+sx-R)
// for cnt <= BATCH rows; image row rr lives in ring slot (rr + R) % RING.
template <int H, bool SUB>
__device__ __forceinline__ void rco_batch(int (&cs)[H * H], const uint8_t *__restrict__ P, int q,
                                          int jc, int prow, int cnt, const unsigned *ringw, int j,
                                          int CSW, int RW4, int RING) {
    constexpr int KW = RcoCfg<H>::KW, NA = RcoCfg<H>::NA;
    unsigned pw[KW];
#pragma unroll
    for (int w = 0; w < KW; ++w) {
        pw[w] = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * w + b;
            if (k < cnt) pw[w] |= (unsigned)P[(int64_t)(prow + k) * q + jc] << (8 * b);
        }
    }
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

template <int H>
__global__ void __launch_bounds__(RcoCfg<H>::MAXT, 1)
rho_co_kernel(const uint8_t *__restrict__ P, const uint8_t *__restrict__ I, int p, int q,
              int m, int n, int Ly, int Lx, const int *__restrict__ wsum,
              const float *__restrict__ inv_sigma, const long long *__restrict__ PS,
              const long long *__restrict__ PQ, int GXS, int GYB, float cut,
              float *rco, unsigned long long *count) {
    constexpr int R = RcoCfg<H>::R;
    constexpr int NS = RcoCfg<H>::NS;
    constexpr int BATCH = RcoCfg<H>::BATCH;
    extern __shared__ int rsm[];
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    const int gx0 = blockIdx.x * GXS, gy0 = blockIdx.y * GYB;
    if (gx0 >= Gx || gy0 >= Gy) return;
    const int gx1 = min(Gx, gx0 + GXS), gy1 = min(Gy, gy0 + GYB);
    const int cx0 = group_centre_of(gx0, Lx, H);
    const int W = group_centre_of(gx1 - 1, Lx, H) + n - cx0;   // pivot columns
    const int RING = rco_ring(m, H), RW4 = RING >> 2, CSW = rco_csw(RING);
    // per shift column sx: prefix sums of the column sums over the W pivot
    // columns (H x (W+1), unsigned: differences of wrapped prefixes are exact
    // because every window sum is < 2^32), warp totals, per-centre pivot
    // statistics, then the image ring
    unsigned *hs = reinterpret_cast<unsigned *>(rsm);
    unsigned *wtot = hs + H * (W + 1);
    int *cS = reinterpret_cast<int *>(wtot + H * 32);             // per centre: S_hat
    float *cI = reinterpret_cast<float *>(cS + GXS);              // per centre: 1/Omega_hat
    unsigned *ringw = reinterpret_cast<unsigned *>(cI + GXS);     // (W + 2R) columns x CSW words
    uint8_t *ring8 = reinterpret_cast<uint8_t *>(ringw);
    const int j = threadIdx.x;
    const bool active = j < W;
    const int jc = cx0 + j;
    const int64_t q1 = q + 1;
    const long long mn = (long long)m * n;
    const int RW = W + 2 * R;                                     // ring columns used

    // rows [r0, r0 + cnt) into their ring slots, all loads of all rows in flight
    auto load_rows = [&](int r0, int cnt) {
        for (int c = threadIdx.x; c < cnt * RW; c += blockDim.x) {
            const int k = c / RW, col = c - k * RW;
            const int rr = r0 + k;
            const int slot = (rr + R) % RING;
            const int ry = min(max(rr, 0), p - 1);
            const int xx = min(max(cx0 - R + col, 0), q - 1);
            ring8[(col * CSW + (slot >> 2)) * 4 + (slot & 3)] = I[(int64_t)ry * q + xx];
        }
    };

    int r = group_centre_of(gy0, Ly, H);
    load_rows(r - R, m + 2 * R + 1);
    __syncthreads();

    int cs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cs[s] = 0;
    if (active) {
        for (int b0 = 0; b0 < m; b0 += BATCH)
            rco_batch<H, false>(cs, P, q, jc, r + b0, min(BATCH, m - b0), ringw, j, CSW, RW4, RING);
    }
    unsigned long long local = 0;
    for (int gy = gy0; gy < gy1; ++gy) {
        const int cy = group_centre_of(gy, Ly, H);
        const int steps = cy - r;            // 0 for the first row, <= H after
        if (steps > 0) {
            // the batch needs rows up to r + steps - 1 + m + R; load the new ones
            load_rows(r + m + R + 1, steps);
            __syncthreads();
            if (active) {
                rco_batch<H, false>(cs, P, q, jc, r + m, steps, ringw, j, CSW, RW4, RING);
                rco_batch<H, true>(cs, P, q, jc, r, steps, ringw, j, CSW, RW4, RING);
            }
            r += steps;
            __syncthreads();   // nobody reads the dead rows the next batch overwrites
        }
        // pivot statistics of this row's centres (exact sums, FP32 1/Omega_hat)
        for (int i = threadIdx.x; i < gx1 - gx0; i += blockDim.x) {
            const int cx = group_centre_of(gx0 + i, Lx, H);
            const long long Sp = ii_box(PS, q1, cy, cx, m, n), Qp = ii_box(PQ, q1, cy, cx, m, n);
            const long long var = mn * Qp - Sp * Sp;
            cS[i] = (int)Sp;
            cI[i] = var > 0 ? sqrtf((float)mn / (float)var) : 0.f;
        }
        // emit centre row cy, one shift row (sy) at a time: block-wide prefix
        // sums of the column sums turn each n-column window sum into one
        // difference
        const int gys = gy * H, gye = min(gys + H, Ly);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
        for (int syi = 0; syi < H; ++syi) {
            const int my = cy + syi - R;
            if (my < gys || my >= gye) continue;   // uniform over the block
            unsigned v[H];
#pragma unroll
            for (int sxi = 0; sxi < H; ++sxi) v[sxi] = active ? (unsigned)cs[syi * H + sxi] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int sxi = 0; sxi < H; ++sxi) {
                    const unsigned t = __shfl_up_sync(0xffffffffu, v[sxi], o);
                    if (lane >= o) v[sxi] += t;
                }
            }
            __syncthreads();   // previous readers of hs / wtot are done
            if (lane == 31) {
#pragma unroll
                for (int sxi = 0; sxi < H; ++sxi) wtot[sxi * 32 + warp] = v[sxi];
            }
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int sxi = 0; sxi < H; ++sxi) {
                    const unsigned t = lane < nwarps ? wtot[sxi * 32 + lane] : 0u;
                    unsigned inc = t;
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned u2 = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += u2;
                    }
                    wtot[sxi * 32 + lane] = inc - t;
                }
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int sxi = 0; sxi < H; ++sxi)
                    hs[sxi * (W + 1) + j + 1] = v[sxi] + wtot[sxi * 32 + warp];
            }
            if (threadIdx.x < H) hs[threadIdx.x * (W + 1)] = 0u;
            __syncthreads();
            const int ntask = (gx1 - gx0) * H;
            for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
                const int gxi = task / H, sxi = task % H;
                const int gx = gx0 + gxi;
                const int cx = group_centre_of(gx, Lx, H);
                const int mx = cx + sxi - R;
                const int gxs = gx * H, gxe = min(gxs + H, Lx);
                if (mx < gxs || mx >= gxe) continue;
                const unsigned *pre = hs + sxi * (W + 1) + (cx - cx0);
                const long long X = (long long)(unsigned)(pre[n] - pre[0]);
                const int64_t li = (int64_t)my * Lx + mx;
                // rho = (mn X - S_hat S) / (mn Omega_hat Omega): exact integer
                // numerator, FP32 finish (flat windows have 1/Omega = 0 -> 0)
                const long long num = mn * X - (long long)cS[gxi] * (long long)wsum[li];
                const float rho = ((float)num * inv_sigma[li]) * (cI[gxi] / (float)mn);
                if (rco) rco[(int64_t)my * Lx + mx] = rho;
                if (rho < cut) ++local;
            }
        }
    }
    if (count) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
    }
}

struct RcoGeom {
    bool ok;
    int GXS, Wmax, threads, strips, bands, GYB;
    size_t smem;
};

// Launch geometry: strips of GXS group columns (one thread per pivot column
// of the strip), bands of GYB group rows; shared memory = H slide rows of
// column prefix sums and their warp totals, the per-centre statistics of one
// group row and the packed image ring.
template <int H>
RcoGeom rco_geom(int p, int q, int m, int n) {
    constexpr int R = RcoCfg<H>::R;
    constexpr int MAXT = RcoCfg<H>::MAXT;
    constexpr size_t kSmemMax = 227 * 1024;
    RcoGeom g{};
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    // window sums of uint8 products are kept in 32 bits
    if (n + H > MAXT || (uint64_t)m * n * 65025u > 0xffffffffull) return g;
    const int csw = rco_csw(rco_ring(m, H));
    auto smem_for = [&](int gxs, int *wmax) {
        *wmax = (gxs - 1) * H + n;
        return (size_t)H * (*wmax + 1 + 32) * sizeof(unsigned) + 2 * (size_t)gxs * sizeof(float) +
               (size_t)(*wmax + 2 * R) * csw * sizeof(unsigned);
    };
    // widest strip within the thread limit, narrowed until tall windows' ring fits
    g.GXS = std::min((MAXT - n) / H + 1, Gx);
    g.smem = smem_for(g.GXS, &g.Wmax);
    while (g.smem > kSmemMax && g.GXS > 1) {
        g.GXS = std::max(1, g.GXS - std::max(1, g.GXS / 8));
        g.smem = smem_for(g.GXS, &g.Wmax);
    }
    g.ok = g.smem <= kSmemMax;
    g.threads = ((g.Wmax + 31) / 32) * 32;
    g.strips = (Gx + g.GXS - 1) / g.GXS;
    const int target = num_sms() * 2;
    g.bands = (target + g.strips - 1) / g.strips;
    if (g.bands > Gy) g.bands = Gy;
    if (g.bands < 1) g.bands = 1;
    g.GYB = (Gy + g.bands - 1) / g.bands;
    g.bands = (Gy + g.GYB - 1) / g.GYB;
    return g;
}

template <int H>
cudaError_t launch_rho_co_h(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                            const int *wsum, const float *inv_sigma, const long long *PS,
                            const long long *PQ, float cut, float *rco,
                            unsigned long long *count, cudaStream_t s) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    const RcoGeom g = rco_geom<H>(p, q, m, n);
    if (!g.ok) return cudaErrorInvalidValue;
    const size_t smem = g.smem;
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(rho_co_kernel<H>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    dim3 grid(g.strips, g.bands);
    LaunchScope ls_rho_co_kernel("rho_co_kernel", s);
    rho_co_kernel<H><<<grid, g.threads, smem, s>>>(P, I, p, q, m, n, Ly, Lx, wsum, inv_sigma, PS,
                                                   PQ, g.GXS, g.GYB, cut, rco, count);
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
    const int ih = block + 2 * kMaxRadius;
    const size_t smem = (size_t)(ih * ih + ih * block) * sizeof(float);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(blur_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    LaunchScope ls_blur_kernel("blur_kernel", s);
    blur_kernel<<<dim3(bq, bp), 256, smem, s>>>(I, p, q, level_map, block, weights, radius, P);
    return cudaGetLastError();
}

cudaError_t launch_blur_corr(const int *wsum, const float *inv_sigma, const long long *PS,
                             const long long *PQ, const long long *PX, int p, int q, int m, int n,
                             float lambda, int block, int *fail, float *R, cudaStream_t s) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    LaunchScope ls_blur_corr_kernel("blur_corr_kernel", s);
    blur_corr_kernel<<<grid_for((int64_t)Ly * Lx, 256), 256, 0, s>>>(
        wsum, inv_sigma, PS, PQ, PX, q, Ly, Lx, m, n, lambda, block, fail, R);
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
                          int h, const int *wsum, const float *inv_sigma, const long long *PS,
                          const long long *PQ, float cut, float *rco,
                          unsigned long long *count, cudaStream_t s) {
    switch (h) {
        case 1: return launch_rho_co_h<1>(P, I, p, q, m, n, wsum, inv_sigma, PS, PQ, cut, rco, count, s);
        case 3: return launch_rho_co_h<3>(P, I, p, q, m, n, wsum, inv_sigma, PS, PQ, cut, rco, count, s);
        case 5: return launch_rho_co_h<5>(P, I, p, q, m, n, wsum, inv_sigma, PS, PQ, cut, rco, count, s);
        case 7: return launch_rho_co_h<7>(P, I, p, q, m, n, wsum, inv_sigma, PS, PQ, cut, rco, count, s);
        case 9: return launch_rho_co_h<9>(P, I, p, q, m, n, wsum, inv_sigma, PS, PQ, cut, rco, count, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_centre_stats(const long long *PS, const long long *PQ, int p, int q, int m, int n,
                                int h, int Ly, int Lx, float *c_inv_sigma, float *c_efac,
                                cudaStream_t s) {
    const int64_t G = (int64_t)groups_along(Ly, h) * groups_along(Lx, h);
    LaunchScope ls_centre_stats_kernel("centre_stats_kernel", s);
    centre_stats_kernel<<<grid_for(G, 256), 256, 0, s>>>(PS, PQ, q, m, n, h, Ly, Lx,
                                                         c_inv_sigma, c_efac);
    return cudaGetLastError();
}

}  // namespace opta
