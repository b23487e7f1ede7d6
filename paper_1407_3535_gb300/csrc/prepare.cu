// Preparation kernels (Sections 3-5): spatially varying Gaussian blur
// (Eq. defblur / Eq. Gauss), blur correlation with the lambda test
// (Algorithm 3, Eq. misDec), pivot auto-correlation maps and the EGS
// retained count (Algorithm 1, Algorithm 2 with Eq. co), per-centre pivot
// statistics.
//
// All correlation sums here are exact integer sums (uint8 x uint8 products
// in int32/int64; FP64 integral images holding integers); only the final
// quotient is rounded, so |rho_co(fp32) - rho_co| <= ~5 u.
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

__device__ inline double box(const double *II, int64_t q1, int y, int x, int m, int n) {
    return II[(int64_t)(y + m) * q1 + x + n] - II[(int64_t)y * q1 + x + n]
         - II[(int64_t)(y + m) * q1 + x] + II[(int64_t)y * q1 + x];
}

// R_oo(x) = rho(P window, I window) (Algorithm 3) and the lambda test.
__global__ void blur_corr_kernel(const double *__restrict__ IIS, const double *__restrict__ IIQ,
                                 const double *__restrict__ PS, const double *__restrict__ PQ,
                                 const double *__restrict__ PX, int q, int Ly, int Lx, int m,
                                 int n, float lambda, int block, int *fail, float *R) {
    const int64_t L = (int64_t)Ly * Lx;
    const int64_t q1 = q + 1;
    const double mn = (double)m * n;
    const int bq = (q + block - 1) / block;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i % Lx);
        const double S = box(IIS, q1, y, x, m, n), Q = box(IIQ, q1, y, x, m, n);
        const double Sp = box(PS, q1, y, x, m, n), Qp = box(PQ, q1, y, x, m, n);
        const double X = box(PX, q1, y, x, m, n);
        // numerator and variances are exact in FP64 (integers < 2^53); the
        // quotient only drives the lambda decision and is finished in FP32
        const double dB = mn * Q - S * S, dA = mn * Qp - Sp * Sp;
        const double num = mn * X - Sp * S;
        float r = 0.f;
        if (dA > 0.0 && dB > 0.0) r = (float)num / sqrtf((float)dA * (float)dB);
        if (R) R[i] = r;
        if (fail && dB > 0.0 && r < lambda) {
            int *f = fail + (y / block) * bq + (x / block);
            if (*f == 0) atomicOr(f, 1);
        }
    }
}

// Per-centre pivot statistics.
__global__ void centre_stats_kernel(const double *__restrict__ PS, const double *__restrict__ PQ,
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
        const double S = box(PS, q1, cy, cx, m, n), Q = box(PQ, q1, cy, cx, m, n);
        const double var = mn * Q - S * S;   // exact
        float is = 0.f, ef = 0.f;
        if (var > 0.0) {
            const float fv = (float)var, fmn = (float)mn;
            is = sqrtf(fmn / fv);
            ef = sqrtf(fmn * (float)(Q - 256.0 * S + 16384.0 * mn) / fv);
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
// which slides down one row at a time (add the new bottom product, subtract
// the old top one).  At each centre row the column sums are summed over the
// n pivot columns of each centre, giving the exact cross sum of the pivot
// block and the member block x = c + s.  A ring buffer in shared memory holds
// the m + 2R + 1 image rows the slide needs.
// ---------------------------------------------------------------------------
template <int H>
struct RcoCfg {
    static constexpr int R = (H - 1) / 2;
    static constexpr int NS = H * H;
    static constexpr int MAXT = H >= 9 ? 512 : (H >= 7 ? 640 : 1024);
};

template <int H>
__global__ void __launch_bounds__(RcoCfg<H>::MAXT, 1)
rho_co_kernel(const uint8_t *__restrict__ P, const uint8_t *__restrict__ I, int p, int q,
              int m, int n, int Ly, int Lx, const float *__restrict__ wsum,
              const float *__restrict__ inv_sigma, const double *__restrict__ PS,
              const double *__restrict__ PQ, int GXS, int GYB, int ring_w, float cut,
              float *rco, unsigned long long *count) {
    constexpr int R = RcoCfg<H>::R;
    constexpr int NS = RcoCfg<H>::NS;
    extern __shared__ int rsm[];
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    const int gx0 = blockIdx.x * GXS, gy0 = blockIdx.y * GYB;
    if (gx0 >= Gx || gy0 >= Gy) return;
    const int gx1 = min(Gx, gx0 + GXS), gy1 = min(Gy, gy0 + GYB);
    const int cx0 = group_centre_of(gx0, Lx, H);
    const int W = group_centre_of(gx1 - 1, Lx, H) + n - cx0;   // pivot columns
    // ring of image rows: the m + 2R + 1 rows one slide step needs, plus the
    // H rows that the next batch of steps (one group row) loads ahead
    const int RING = m + 2 * R + 1 + H;
    // per shift column sx: prefix sums of the column sums over the W pivot
    // columns (H x (W+1), unsigned: differences of wrapped prefixes are exact
    // because every window sum is < 2^32), warp totals, then the image ring
    unsigned *hs = reinterpret_cast<unsigned *>(rsm);
    unsigned *wtot = hs + H * (W + 1);
    float *cst = reinterpret_cast<float *>(wtot + H * 32);        // per centre: S_hat, 1/Omega_hat
    uint8_t *ring = reinterpret_cast<uint8_t *>(cst + 2 * GXS);   // RING x ring_w bytes
    const int j = threadIdx.x;
    const bool active = j < W;
    const int jc = cx0 + j;
    const int64_t q1 = q + 1;
    const long long mn = (long long)m * n;
    const int RW = W + 2 * R;                                     // ring row width used

    // rows [r0, r0 + cnt) into their ring slots, all loads of all rows in flight
    auto load_rows = [&](int r0, int cnt) {
        for (int c = threadIdx.x; c < cnt * RW; c += blockDim.x) {
            const int k = c / RW, col = c - k * RW;
            const int rr = r0 + k;
            const int slot = (rr + R) % RING;
            const int ry = min(max(rr, 0), p - 1);
            const int xx = min(max(cx0 - R + col, 0), q - 1);
            ring[slot * ring_w + col] = I[(int64_t)ry * q + xx];
        }
    };

    int r = group_centre_of(gy0, Ly, H);
    load_rows(r - R, m + 2 * R + 1);
    __syncthreads();

    int cs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) cs[s] = 0;
    if (active) {
        for (int i = 0; i < m; ++i) {
            const int pv = P[(int64_t)(r + i) * q + jc];
#pragma unroll
            for (int sy = 0; sy < H; ++sy) {
                const uint8_t *row = ring + ((r + i + sy) % RING) * ring_w + j;   // row r+i+sy-R
#pragma unroll
                for (int sx = 0; sx < H; ++sx) cs[sy * H + sx] += pv * (int)row[sx];
            }
        }
    }
    unsigned long long local = 0;
    for (int gy = gy0; gy < gy1; ++gy) {
        const int cy = group_centre_of(gy, Ly, H);
        const int steps = cy - r;            // 0 for the first row, <= H after
        if (steps > 0) {
            // the batch needs rows up to r + steps - 1 + m + R; load the new ones
            load_rows(r + m + R + 1, steps);
            int pold[H], pnew[H];
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const bool ok = active && k < steps;
                pold[k] = ok ? P[(int64_t)(r + k) * q + jc] : 0;
                pnew[k] = ok ? P[(int64_t)(r + k + m) * q + jc] : 0;
            }
            __syncthreads();
            if (active) {
                int so = r % RING, sn = (r + m) % RING;     // slots of rows r - R and r + m - R
#pragma unroll
                for (int k = 0; k < H; ++k) {
                    if (k < steps) {
#pragma unroll
                        for (int sy = 0; sy < H; ++sy) {
                            const int a = so + sy, b = sn + sy;
                            const uint8_t *ro = ring + (a >= RING ? a - RING : a) * ring_w + j;
                            const uint8_t *rn = ring + (b >= RING ? b - RING : b) * ring_w + j;
#pragma unroll
                            for (int sx = 0; sx < H; ++sx)
                                cs[sy * H + sx] += pnew[k] * (int)rn[sx] - pold[k] * (int)ro[sx];
                        }
                        so = (so + 1 == RING) ? 0 : so + 1;
                        sn = (sn + 1 == RING) ? 0 : sn + 1;
                    }
                }
            }
            r += steps;
            __syncthreads();   // nobody reads the dead rows the next batch overwrites
        }
        // pivot statistics of this row's centres (exact sums, FP32 1/Omega_hat)
        for (int i = threadIdx.x; i < gx1 - gx0; i += blockDim.x) {
            const int cx = group_centre_of(gx0 + i, Lx, H);
            const double Sp = box(PS, q1, cy, cx, m, n), Qp = box(PQ, q1, cy, cx, m, n);
            const double var = (double)mn * Qp - Sp * Sp;
            cst[2 * i] = (float)Sp;
            cst[2 * i + 1] = var > 0.0 ? sqrtf((float)mn / (float)var) : 0.f;
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
                const long long num = mn * X - (long long)cst[2 * gxi] * (long long)wsum[li];
                const float rho = ((float)num * inv_sigma[li]) * (cst[2 * gxi + 1] / (float)mn);
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

template <int H>
cudaError_t launch_rho_co_h(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                            const float *wsum, const float *inv_sigma, const double *PS,
                            const double *PQ, float cut, float *rco,
                            unsigned long long *count, cudaStream_t s) {
    constexpr int R = RcoCfg<H>::R;
    constexpr int MAXT = RcoCfg<H>::MAXT;
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int Gy = groups_along(Ly, H), Gx = groups_along(Lx, H);
    if (n + H > MAXT) return cudaErrorInvalidValue;
    int GXS = (MAXT - n) / H + 1;
    if (GXS > Gx) GXS = Gx;
    const int Wmax = (GXS - 1) * H + n;
    const int threads = ((Wmax + 31) / 32) * 32;
    const int strips = (Gx + GXS - 1) / GXS;
    const int target = num_sms() * 2;
    int bands = (target + strips - 1) / strips;
    if (bands > Gy) bands = Gy;
    if (bands < 1) bands = 1;
    int GYB = (Gy + bands - 1) / bands;
    bands = (Gy + GYB - 1) / GYB;
    const int ring_w = ((Wmax + 2 * R) + 15) & ~15;
    const size_t smem = (size_t)H * (Wmax + 1 + 32) * sizeof(unsigned) + 2 * (size_t)GXS * sizeof(float) +
                        (size_t)(m + 2 * R + 1 + H) * ring_w;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(rho_co_kernel<H>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    dim3 grid(strips, bands);
    LaunchScope ls_rho_co_kernel("rho_co_kernel", s);
    rho_co_kernel<H><<<grid, threads, smem, s>>>(P, I, p, q, m, n, Ly, Lx, wsum, inv_sigma, PS, PQ,
                                                 GXS, GYB, ring_w, cut, rco, count);
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

cudaError_t launch_blur_corr(const double *IIS, const double *IIQ, const double *PS,
                             const double *PQ, const double *PX, int p, int q, int m, int n,
                             float lambda, int block, int *fail, float *R, cudaStream_t s) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    LaunchScope ls_blur_corr_kernel("blur_corr_kernel", s);
    blur_corr_kernel<<<grid_for((int64_t)Ly * Lx, 256), 256, 0, s>>>(
        IIS, IIQ, PS, PQ, PX, q, Ly, Lx, m, n, lambda, block, fail, R);
    return cudaGetLastError();
}

cudaError_t launch_rho_co(const uint8_t *P, const uint8_t *I, int p, int q, int m, int n,
                          int h, const float *wsum, const float *inv_sigma, const double *PS,
                          const double *PQ, float cut, float *rco,
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

cudaError_t launch_centre_stats(const double *PS, const double *PQ, int p, int q, int m, int n,
                                int h, int Ly, int Lx, float *c_inv_sigma, float *c_efac,
                                cudaStream_t s) {
    const int64_t G = (int64_t)groups_along(Ly, h) * groups_along(Lx, h);
    LaunchScope ls_centre_stats_kernel("centre_stats_kernel", s);
    centre_stats_kernel<<<grid_for(G, 256), 256, 0, s>>>(PS, PQ, q, m, n, h, Ly, Lx,
                                                         c_inv_sigma, c_efac);
    return cudaGetLastError();
}

}  // namespace opta
