// Local statistics: int64 integral images and per-window sum / sum of squares
// (Algorithm 3's Run-Sum S, Q and Omega = sqrt(Q - S^2/mn); the "four
// operations" per window of Section 3.1).
//
// Pixels are integers in [0,255], so the integral images, the window sums
// taken from them and mn*Q - S^2 (for windows up to 2^23 pixels) are exact
// integers; only the final 1/Omega is rounded (FP32).
#include <atomic>
#include <algorithm>

#include "common.cuh"

namespace opta {

namespace {

constexpr int kRowThreads = 256;

// Row pass: o_k[(y+1)*(q+1) + x+1] = sum_{j<=x} f_k(A[y][j], B[y][j]).
// One block per row; tiles of 4 * 256 pixels: each thread takes 4 consecutive
// pixels, the block scans the thread totals, and consecutive threads write
// consecutive 32-byte runs (coalesced).  Sums are exact in int64.
template <typename T>
__global__ void __launch_bounds__(kRowThreads)
ii_rows_kernel(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B, int p, int q,
               T *o0, T *o1, T *o2) {
    __shared__ long long wsum[3][kRowThreads / 32];
    __shared__ long long carry[3];
    const int y = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint8_t *a = A + (int64_t)y * q;
    const uint8_t *b = B ? B + (int64_t)y * q : nullptr;
    const int64_t q1 = q + 1;
    T *d0 = o0 + (int64_t)(y + 1) * q1;
    T *d1 = o1 + (int64_t)(y + 1) * q1;
    T *d2 = (b && o2) ? o2 + (int64_t)(y + 1) * q1 : nullptr;
    if (tid == 0) {
        d0[0] = 0; d1[0] = 0; if (d2) d2[0] = 0;
        carry[0] = carry[1] = carry[2] = 0;
    }
    __syncthreads();
    for (int x0 = 0; x0 < q; x0 += 4 * kRowThreads) {
        const int xs = x0 + 4 * tid;
        int va[4], vb[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            va[k] = xs + k < q ? a[xs + k] : 0;
            vb[k] = (b && xs + k < q) ? b[xs + k] : 0;
        }
        long long p0[4], p1[4], p2[4];
        long long r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            r0 += va[k]; r1 += va[k] * va[k]; r2 += va[k] * vb[k];
            p0[k] = r0; p1[k] = r1; p2[k] = r2;
        }
        // inclusive warp scan of the thread totals
        long long i0 = r0, i1 = r1, i2 = r2;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t0 = __shfl_up_sync(0xffffffffu, i0, o);
            const long long t1 = __shfl_up_sync(0xffffffffu, i1, o);
            const long long t2 = __shfl_up_sync(0xffffffffu, i2, o);
            if (lane >= o) { i0 += t0; i1 += t1; i2 += t2; }
        }
        if (lane == 31) { wsum[0][warp] = i0; wsum[1][warp] = i1; wsum[2][warp] = i2; }
        __syncthreads();
        long long e0 = carry[0] + i0 - r0, e1 = carry[1] + i1 - r1, e2 = carry[2] + i2 - r2;
        for (int w = 0; w < warp; ++w) { e0 += wsum[0][w]; e1 += wsum[1][w]; e2 += wsum[2][w]; }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (xs + k < q) {
                d0[xs + k + 1] = (T)(e0 + p0[k]);
                d1[xs + k + 1] = (T)(e1 + p1[k]);
                if (d2) d2[xs + k + 1] = (T)(e2 + p2[k]);
            }
        }
        __syncthreads();
        if (tid == kRowThreads - 1) {
            carry[0] = e0 + r0; carry[1] = e1 + r1; carry[2] = e2 + r2;
        }
        __syncthreads();
    }
}

// Column pass over rows 1..p of up to three arrays, 32 columns x 32 row segments.
template <typename T>
__global__ void __launch_bounds__(1024)
ii_cols_kernel(int p, int q, T *o0, T *o1, T *o2) {
    const int64_t q1 = q + 1;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int seg = threadIdx.y;
    const int seglen = (p + 31) / 32;
    const int r0 = 1 + seg * seglen, r1 = min(p + 1, r0 + seglen);
    T a0 = 0, a1 = 0, a2 = 0;
    if (x < q1) {
        for (int r = r0; r < r1; ++r) {
            a0 += o0[r * q1 + x];
            a1 += o1[r * q1 + x];
            if (o2) a2 += o2[r * q1 + x];
        }
    }
    __shared__ T sh[3][32][33];
    sh[0][seg][threadIdx.x] = a0; sh[1][seg][threadIdx.x] = a1; sh[2][seg][threadIdx.x] = a2;
    __syncthreads();
    if (seg == 0) {
        T c0 = 0, c1 = 0, c2 = 0;
        for (int k = 0; k < 32; ++k) {
            const T t0 = sh[0][k][threadIdx.x], t1 = sh[1][k][threadIdx.x], t2 = sh[2][k][threadIdx.x];
            sh[0][k][threadIdx.x] = c0; sh[1][k][threadIdx.x] = c1; sh[2][k][threadIdx.x] = c2;
            c0 += t0; c1 += t1; c2 += t2;
        }
    }
    __syncthreads();
    if (x >= q1) return;
    T c0 = sh[0][seg][threadIdx.x], c1 = sh[1][seg][threadIdx.x], c2 = sh[2][seg][threadIdx.x];
    for (int r = r0; r < r1; ++r) {
        c0 += o0[r * q1 + x]; o0[r * q1 + x] = c0;
        c1 += o1[r * q1 + x]; o1[r * q1 + x] = c1;
        if (o2) { c2 += o2[r * q1 + x]; o2[r * q1 + x] = c2; }
    }
}

// Number of zero entries (flat windows: 1/Omega = 0) of the Ly x Lx map x,
// over the rows EGS samples for group side h (every row when sample == 1):
// rows over blockIdx.y (grid-strided), columns over the x threads.
__global__ void count_zero_kernel(const float *__restrict__ x, int Ly, int Lx, int h, int sample,
                                  unsigned long long *count) {
    unsigned long long c = 0;
    for (int row = blockIdx.y; row < Ly; row += gridDim.y) {
        if (sample > 1 && ((row / h) / kEgsRun) % sample != 0) continue;   // uniform
        const float *xr = x + (int64_t)row * Lx;
        for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < Lx; col += gridDim.x * blockDim.x)
            c += xr[col] == 0.f ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// One thread per location: rows over blockIdx.y (grid-strided), columns over
// blockIdx.x * blockDim.x + threadIdx.x.
__global__ void window_stats_kernel(const long long *__restrict__ IIS,
                                    const long long *__restrict__ IIQ, int q, int Ly, int Lx,
                                    int m, int n, float *inv_sigma, float *efac128, int *wsum) {
    const int64_t q1 = q + 1;
    const long long mn = (long long)m * n;
    const float fmn = i64_to_f32(mn);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= Lx) return;
    for (int y = blockIdx.y; y < Ly; y += gridDim.y) {
        const int64_t i = (int64_t)y * Lx + x;
        const long long S = ii_box(IIS, q1, y, x, m, n);
        const long long Q = ii_box(IIQ, q1, y, x, m, n);
        const float fv = win_var(mn, S, Q);         // mn * Omega^2
        float inv = 0.f, ef = 0.f;
        if (fv > 0.f) {
            // FP32 finish (a few ulp; the error bounds that use 1/Omega allow 8u)
            inv = sqrtf(fmn / fv);
            const long long c2 = Q - 256 * S + 16384 * mn;   // sum (I - 128)^2, exact
            ef = sqrtf(fmn * i64_to_f32(c2) / fv);
        }
        inv_sigma[i] = inv;
        if (efac128) efac128[i] = ef;
        if (wsum) wsum[i] = (int)S;
    }
}

__global__ void i64_to_f32_kernel(const long long *__restrict__ v, float *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = i64_to_f32(v[i]);
}

__global__ void ingest_f32_kernel(const float *__restrict__ src, int64_t ld, int p, int q,
                                  uint8_t *dst, int *bad) {
    const int64_t N = (int64_t)p * q;
    int any = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / q), x = (int)(i % q);
        const float v = src[(int64_t)y * ld + x];
        if (!(v >= 0.f && v <= 255.f && v == rintf(v))) any = 1;
        dst[i] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
    if (any) atomicOr(bad, 1);
}

__global__ void ingest_u8_kernel(const uint8_t *__restrict__ src, int64_t ld, int p, int q,
                                 uint8_t *dst) {
    const int64_t N = (int64_t)p * q;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / q), x = (int)(i % q);
        dst[i] = src[(int64_t)y * ld + x];
    }
}

}  // namespace

int num_sms() {
    // per device: the library may serve several GPUs of one process
    constexpr int kDevs = 64;
    static std::atomic<int> sms[kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
        cudaGetLastError();
        return 132;
    }
    int v = sms[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 132;
    }
    sms[dev].store(v, std::memory_order_relaxed);
    return v;
}

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
static cudaError_t integrals_impl(const uint8_t *A, const uint8_t *B, int p, int q, T *o0, T *o1,
                                  T *o2, cudaStream_t s) {
    const int64_t q1 = q + 1;
    cudaError_t e;
    // first row zero
    if ((e = cudaMemsetAsync(o0, 0, q1 * sizeof(T), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(o1, 0, q1 * sizeof(T), s)) != cudaSuccess) return e;
    if (B && o2 && (e = cudaMemsetAsync(o2, 0, q1 * sizeof(T), s)) != cudaSuccess) return e;
    {
        LaunchScope ls("ii_rows_kernel", s);
        ii_rows_kernel<T><<<p, kRowThreads, 0, s>>>(A, B, p, q, o0, o1, (B ? o2 : nullptr));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        LaunchScope ls("ii_cols_kernel", s);
        ii_cols_kernel<T><<<(int)((q1 + 31) / 32), dim3(32, 32), 0, s>>>(p, q, o0, o1,
                                                                        (B ? o2 : nullptr));
    }
    return cudaGetLastError();
}

cudaError_t launch_integrals(const uint8_t *A, const uint8_t *B, int p, int q, long long *o0,
                             long long *o1, long long *o2, cudaStream_t s) {
    return integrals_impl<long long>(A, B, p, q, o0, o1, o2, s);
}


cudaError_t launch_count_zero(const float *x, int Ly, int Lx, int h, int sample,
                              unsigned long long *count, cudaStream_t s) {
    const int bx = (Lx + 255) / 256;
    const int by = std::max(1, std::min(Ly, (8 * num_sms() + bx - 1) / bx));
    LaunchScope ls("count_zero_kernel", s);
    count_zero_kernel<<<dim3(bx, by), 256, 0, s>>>(x, Ly, Lx, h, sample, count);
    return cudaGetLastError();
}

cudaError_t launch_window_stats(const long long *IIS, const long long *IIQ, int p, int q,
                                int m, int n, float *inv_sigma, float *efac128,
                                cudaStream_t s, int *wsum) {
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int bx = (Lx + 255) / 256;
    const int by = std::max(1, std::min(Ly, (8 * num_sms() + bx - 1) / bx));
    LaunchScope ls_window_stats_kernel("window_stats_kernel", s);
    window_stats_kernel<<<dim3(bx, by), 256, 0, s>>>(IIS, IIQ, q, Ly, Lx, m, n, inv_sigma, efac128,
                                                     wsum);
    return cudaGetLastError();
}

cudaError_t launch_i64_to_f32(const long long *v, float *out, int64_t n, cudaStream_t s) {
    LaunchScope ls("i64_to_f32_kernel", s);
    i64_to_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, out, n);
    return cudaGetLastError();
}

cudaError_t launch_ingest_f32(const float *src, int64_t ld, int p, int q, uint8_t *dst,
                              int *bad, cudaStream_t s) {
    LaunchScope ls_ingest_f32_kernel("ingest_f32_kernel", s);
    ingest_f32_kernel<<<grid_for((int64_t)p * q, 256), 256, 0, s>>>(src, ld, p, q, dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_ingest_u8(const uint8_t *src, int64_t ld, int p, int q, uint8_t *dst,
                             cudaStream_t s) {
    LaunchScope ls_ingest_u8_kernel("ingest_u8_kernel", s);
    ingest_u8_kernel<<<grid_for((int64_t)p * q, 256), 256, 0, s>>>(src, ld, p, q, dst);
    return cudaGetLastError();
}

}  // namespace opta
