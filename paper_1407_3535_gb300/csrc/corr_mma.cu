// Scan 1 (Section 6) on the 5th-generation tensor cores: rho(t, pivot block)
// at every group centre for a batch of same-size templates at once.
//
// For a centre row cy and 128 consecutive centres along x (spacing h):
//
//   D[i][j] = sum_{u<m} sum_{v<Kp} A_u[i][v] * B_u[j][v]
//   A_u[i][v] = P(cy + u, cx0 + h*i + v) - 128            (fp16, exact)
//   B_u[j][v] = template plane j, row u                     (fp16 hi/lo split of s t')
//
// with j = 2t (hi part of template t) and 2t+1 (lo part), so each template's
// numerator is D[i][2t] + D[i][2t+1].  D lives in TMEM; the contraction over
// (u, v) is m * Kp/16 tcgen05.mma instructions of shape 128 x N x 16.
//
// A_u is a Hankel operand: row i is the pivot row shifted by h*i.  It is
// stored once per template row in the K-major "core matrix" layout without
// swizzle: segment w (128 bytes) holds 8 copies b = 0..7 of the 8 pixels
// starting at column cx0 + h*b + 8*w.  Element (i = 8a + b, k = 8c + d) then
// sits at byte (h*a + c)*128 + 16*b + 2*d, i.e. a descriptor with leading
// (K) byte offset 128 and stride (M) byte offset 128*h; core matrices
// overlap, which costs nothing.  B_u arrives by one bulk copy from a buffer
// already laid out as core matrices.
//
// A CTA takes RC centre rows cy_k (k < RC, about h apart) of the same 128
// centres and walks the pivot rows r: the Hankel operand of row r is built
// once and feeds every accumulator k with u_k = r - cy_k in [0, m), against
// template row u_k.  The RC accumulators sit side by side in TMEM (k at
// column k * N), so one MMA of N' = RC * N columns serves all of them: its
// B operand holds, for each 8-wide K block, the tiles of rows u_0 .. u_RC-1
// one after another (a zero tile, row m of the buffer, where u_k is out of
// range).  Two stages (A and B) overlap the build of the next pivot row
// with the MMAs of the current one, and the work is split by warp: lane 0
// of warp 0 issues and commits the MMAs; warps 1-7 build the Hankel
// operand, and warp 1 first queues the B operand of the step; the stages
// change hands through mbarriers (operand and tiles ready, MMAs done), so no
// role waits for another at a CTA barrier.  Where the CTA's centre rows are
// exactly h apart (all but the last, clamped group row), the B operand of
// pivot row r is one contiguous block of a buffer arranged per launch,
// B2[u0 = r - cy_0][c][k] = tile (u0 - k h, c), and arrives by one bulk
// copy: a bulk copy or an MMA costs its issuing thread about a hundred
// cycles, so the step issues one copy and Kp/16 MMAs, not RC * Kp/8 copies
// and RC * Kp/16 MMAs.
//
// The operands are fp16 (kind::f16 with both operands fp16): a pixel
// P - 128 is an integer of at most 8 bits, exact, and converts from a byte by
// one byte permutation and one paired subtraction (tc5::bytes_f16x2); the
// template is scaled by a power of two s (TmplState::tscale, s max|t'| in
// [2^13, 2^14)) and split into fp16 hi + lo, which holds it to about 2^-22;
// the epilogue multiplies by 1/s, exactly.  FP32 accumulation in TMEM is
// bounded by 4u per accumulation step (one step per MMA of a row in range;
// the zero tiles' MMAs add exact zeros) -- scan1_epsA_f16.
// The angle intervals that scan 2 needs are formed there from rho and this
// bound.
#include <cuda_fp16.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "tc5.cuh"

namespace opta {

namespace {

constexpr int kMmaM = 128;
constexpr uint64_t kWaitNs = 2000000000ull;   // every wait gives up after 2 s
// Budget of the waits for progress (operand built, tiles landed, stage
// released) and the stall switch, both set only by the verification hook
// opta_dbg_scan1_wait; the drain at the end (copies and MMAs still in
// flight) always waits up to kWaitNs.
std::atomic<uint64_t> g_wait_ns{kWaitNs};
std::atomic<int> g_stall{0};

__host__ __device__ inline uint32_t round_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

struct CorrMmaArgs {
    const uint8_t *V;          // pivot image, p x q
    int p, q;
    const __half *B;           // [m + 1][Kp/8][N/8][8][8]; row m is zero
    const __half *B2;          // [R2][Kp/8][RC][N/8][8][8]: B2[u0][c][k] = B[u0 - k h][c] (zero outside)
    int R2;                    // rows of B2: m + (RC - 1) h
    int m, n, Kp, N;
    int h, Ly, Lx, Gx, Gx_u;   // Gx_u: leading groups whose centres are uniform (cx0 + h*i)
    int Gy, RC;                // group rows; centre rows per CTA (1, 2 or 4)
    int T;                     // templates (planes 2t, 2t+1)
    const float *c_inv_sigma;  // per group
    const TmplState *st;       // T states
    float *rho_tc;             // [T][gstride]
    int64_t gstride;
    int *err;
    uint64_t wait_ns;          // budget of each wait for progress
    int stall;                 // 1: the issuer first waits on a barrier no thread arrives at
};


constexpr int kMmaThreads = 256;
// The raw words of one operand item (8 pixels from column x of a row):
// three aligned words and the byte shift that aligns them, or, at the right
// edge, the 8 clamped pixels in words 0-1 with no shift.
struct ItemWords {
    uint32_t w0, w1, w2, sh;
};

// the right edge, out of line (the last few items of a row only)
__device__ __noinline__ ItemWords item_words_edge(const uint8_t *row, int x, int q) {
    ItemWords r;
    r.w0 = r.w1 = r.w2 = r.sh = 0u;
    for (int d = 0; d < 4; ++d) r.w0 |= (uint32_t)row[min(x + d, q - 1)] << (8 * d);
    for (int d = 0; d < 4; ++d) r.w1 |= (uint32_t)row[min(x + 4 + d, q - 1)] << (8 * d);
    return r;
}

__device__ __forceinline__ ItemWords item_words(const uint8_t *row, int x, int q) {
    if (x + 12 > q) return item_words_edge(row, x, q);
    // the 12 bytes from the aligned word at or below row + x lie in the row
    ItemWords r;
    const uintptr_t ad = reinterpret_cast<uintptr_t>(row + x);
    const uint32_t *wp = reinterpret_cast<const uint32_t *>(ad & ~(uintptr_t)3);
    r.w0 = wp[0]; r.w1 = wp[1]; r.w2 = wp[2];
    r.sh = (uint32_t)(ad & 3) * 8u;
    return r;
}
// Segments of one copy a builder thread converts per row: WA = 15 h + Kp/8
// <= 151 (h <= 9, Kp <= 128) over 28 runs.
constexpr int kMaxRun = 6;
constexpr int kMaxRC = 4;   // centre rows per CTA (the launcher measures 1 to 4, RC * N <= 256)

__global__ void __launch_bounds__(kMmaThreads, 4) corr_mma_kernel(const CorrMmaArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *a_full = reinterpret_cast<uint64_t *>(smem);   // [2] A written (7 builder warps) and B checked
    uint64_t *b_full = a_full + 2;                           // [2] B tiles landed (transaction bytes)
    uint64_t *mma_done = b_full + 2;                         // [2] MMAs of the stage completed
    uint64_t *stall_bar = mma_done + 2;                      // never completes (verification only)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(stall_bar + 1);
    const int WA = 15 * a.h + a.Kp / 8;
    const uint32_t abytes = (uint32_t)WA * 128u;
    const uint32_t cbytes = (uint32_t)a.RC * a.N * 16u;      // one 8-wide K block of the RC tiles
    const uint32_t bbytes = cbytes * (uint32_t)(a.Kp / 8);
    const uint32_t astride = round_up(abytes, 1024), bstride = round_up(bbytes, 1024);
    uint8_t *Abase = smem + 1024;
    uint8_t *Bbase = Abase + 2 * astride;                    // [2] stages of [Kp/8][RC][N/8] core matrices

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gy0 = blockIdx.y * a.RC;
    const int nrow = min(a.RC, a.Gy - gy0);
    const int gx0 = blockIdx.x * kMmaM;
    const int cx0 = group_centre_of(gx0, a.Lx, a.h);
    int cyk[kMaxRC];
    bool uniform = true;   // centre rows exactly h apart: B2 serves this CTA
#pragma unroll
    for (int k = 0; k < kMaxRC; ++k) {
        cyk[k] = k < nrow ? group_centre_of(gy0 + k, a.Ly, a.h) : 0;
        if (k < nrow && cyk[k] != cyk[0] + k * a.h) uniform = false;
    }

    uint32_t ncols = 32;
    while ((int)ncols < a.RC * a.N) ncols <<= 1;
    if (tid == 0) {
        tc5::mbar_init(&a_full[0], kMmaThreads / 32 - 1);
        tc5::mbar_init(&a_full[1], kMmaThreads / 32 - 1);
        tc5::mbar_init(&b_full[0], 1);
        tc5::mbar_init(&b_full[1], 1);
        tc5::mbar_init(&mma_done[0], 1);
        tc5::mbar_init(&mma_done[1], 1);
        tc5::mbar_init(stall_bar, 1);
        tc5::fence_mbar_init();
    }
    if (warp == 0) {
        tc5::tmem_alloc(tmem_slot, ncols);
        tc5::tmem_relinquish();
    }
    tc5::tc_fence_before();
    __syncthreads();
    tc5::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    const int r_end = group_centre_of(gy0 + nrow - 1, a.Ly, a.h) + a.m;
    // template row u_k of accumulator k at pivot row r (-1: none); every role
    // walks the same rows and counts the same steps
    auto rows_of = [&](int r, int (&uk)[kMaxRC]) {
        int nvalid = 0;
#pragma unroll
        for (int k = 0; k < kMaxRC; ++k) {
            const int u = r - cyk[k];
            uk[k] = (k < nrow && u >= 0 && u < a.m) ? u : -1;
            nvalid += uk[k] >= 0 ? 1 : 0;
        }
        return nvalid;
    };
    if (warp == 0) {
        if (lane == 0) {
            // issuer: step k waits for its stage (operand built, tiles
            // landed), issues Kp/16 MMAs of 128 x RC*N x 16 and commits
            const uint32_t idesc = tc5::idesc_f16_f32(kMmaM, a.RC * a.N);
            const uint64_t ad0 = tc5::smem_desc(tc5::smem_u32(Abase), 128, 128u * a.h);
            const uint64_t ad1 = tc5::smem_desc(tc5::smem_u32(Abase + astride), 128, 128u * a.h);
            const uint64_t bd0 = tc5::smem_desc(tc5::smem_u32(Bbase), cbytes, 128);
            const uint64_t bd1 = tc5::smem_desc(tc5::smem_u32(Bbase + bstride), cbytes, 128);
            // the next 16 K columns: 256 bytes further in A, two K blocks in B
            // (descriptor start addresses count 16-byte units)
            const uint64_t bstep = (uint64_t)((2u * cbytes) >> 4);
            const int nk = a.Kp / 16;
            int step = 0, last = -1;
            // verification of the timeout path: a wait that cannot complete
            if (a.stall && !tc5::mbar_wait(stall_bar, 0u, a.wait_ns)) ok = false;
            for (int r = cyk[0]; ok && r < r_end; ++r) {
                int uk[kMaxRC];
                if (rows_of(r, uk) == 0) continue;
                const int s = step & 1;
                const uint32_t ph = (step >> 1) & 1;
                if (!tc5::mbar_wait(&a_full[s], ph, a.wait_ns)) { ok = false; break; }
                tc5::tc_fence_after();
                const uint64_t ad = s ? ad1 : ad0, bd = s ? bd1 : bd0;
                // the first step initialises every accumulator (tiles of
                // rows out of range are zero)
                for (int kk = 0; kk < nk; ++kk)
                    tc5::mma_bf16(tmem, ad + (uint64_t)(16 * kk), bd + (uint64_t)kk * bstep, idesc,
                                  step > 0 || kk > 0);
                tc5::mma_commit(&mma_done[s]);
                last = step;
                ++step;
            }
            // drain (bounded): the last MMA batch
            if (last >= 0 && !tc5::mbar_wait(&mma_done[last & 1], (last >> 1) & 1, kWaitNs)) ok = false;
        }
    } else {
        // builders (warps 1..7): step k writes A of stage k & 1 once the MMAs
        // of step k - 2 released it (lane 0 waits; the warp follows it);
        // warp 1 first queues the step's B tiles and, before its arrival on
        // a_full, waits until they landed
        const int btid = tid - 32;
        constexpr int kBuilders = kMmaThreads - 32;
        const int ncopy = a.RC * (a.Kp / 8);
        const uint32_t tile_bytes = (uint32_t)a.N * 16u;
        const int runK = (WA + kBuilders / 8 - 1) / (kBuilders / 8);   // segments per thread (<= kMaxRun)
        int step = 0, last_tx = -1;
        for (int r = cyk[0]; r < r_end; ++r) {
            int uk[kMaxRC];
            if (rows_of(r, uk) == 0) continue;
            const int s = step & 1;
            const uint32_t ph = (step >> 1) & 1;
            if (step >= 2) {
                bool w_ok = true;
                if (lane == 0) w_ok = tc5::mbar_wait(&mma_done[s], ph ^ 1u, a.wait_ns);
                w_ok = __shfl_sync(0xffffffffu, w_ok ? 1 : 0, 0) != 0;
                __syncwarp();
                if (!w_ok) { ok = false; break; }
            }
            if (warp == 1) {
                // slot j = c * RC + k <- K block c of template row u_k (row m: zeros)
                if (lane == 0) tc5::mbar_arrive_expect_tx(&b_full[s], bbytes);
                __syncwarp();
                uint8_t *Bs = Bbase + s * bstride;
                const int u0 = r - cyk[0];
                if (uniform && u0 < a.R2) {
                    if (lane == 0) tc5::bulk_g2s(Bs, a.B2 + (size_t)u0 * (bbytes / 2), bbytes, &b_full[s]);
                } else for (int j = lane; j < ncopy; j += 32) {
                    const int k = j % a.RC, c = j / a.RC;
                    int u = -1;
#pragma unroll
                    for (int k2 = 0; k2 < kMaxRC; ++k2)
                        if (k2 == k) u = uk[k2];
                    if (u < 0) u = a.m;
                    tc5::bulk_g2s(Bs + (size_t)j * tile_bytes,
                                  a.B + ((size_t)u * (a.Kp / 8) + c) * (size_t)a.N * 8, tile_bytes,
                                  &b_full[s]);
                }
                last_tx = step;
            }
            // A_r: segment w, copy b = pixels cx0 + h*b + 8w .. +7 of row r
            const uint8_t *row = a.V + (size_t)r * a.q;
            uint8_t *Ab = Abase + s * astride;
            // thread (b, run): copy b of the run of K consecutive segments
            // wb .. wb + K - 1, i.e. the pixels from cx0 + h b + 8 wb on, one
            // contiguous stretch: its words are loaded once, share one byte
            // shift, and item k takes words 2k .. 2k + 2 (a warp stores four
            // segment rows of 128 contiguous bytes)
            {
                const int b = btid & 7, wb = (btid >> 3) * runK;
                const int nk = min(runK, WA - wb);
                const int xr = cx0 + a.h * b + 8 * wb;
                if (nk > 0 && xr + 8 * nk + 4 <= a.q) {
                    const uintptr_t ad = reinterpret_cast<uintptr_t>(row + xr);
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(ad & ~(uintptr_t)3);
                    const uint32_t sh = (uint32_t)(ad & 3) * 8u;
                    uint32_t wv[2 * kMaxRun + 1];
#pragma unroll
                    for (int i = 0; i <= 2 * kMaxRun; ++i) wv[i] = i <= 2 * nk ? wp[i] : 0u;
#pragma unroll
                    for (int k = 0; k < kMaxRun; ++k) {
                        if (k < nk) {
                            const uint32_t lo = __funnelshift_r(wv[2 * k], wv[2 * k + 1], sh);
                            const uint32_t hi = __funnelshift_r(wv[2 * k + 1], wv[2 * k + 2], sh);
                            *reinterpret_cast<uint4 *>(Ab + (wb + k) * 128 + b * 16) =
                                make_uint4(tc5::bytes_f16x2<0>(lo), tc5::bytes_f16x2<2>(lo),
                                           tc5::bytes_f16x2<0>(hi), tc5::bytes_f16x2<2>(hi));
                        }
                    }
                } else {
                    // the right edge of the row: item by item, clamped
                    for (int k = 0; k < nk; ++k) {
                        const ItemWords iw = item_words(row, xr + 8 * k, a.q);
                        const uint32_t lo = __funnelshift_r(iw.w0, iw.w1, iw.sh);
                        const uint32_t hi = __funnelshift_r(iw.w1, iw.w2, iw.sh);
                        *reinterpret_cast<uint4 *>(Ab + (wb + k) * 128 + b * 16) =
                            make_uint4(tc5::bytes_f16x2<0>(lo), tc5::bytes_f16x2<2>(lo),
                                       tc5::bytes_f16x2<0>(hi), tc5::bytes_f16x2<2>(hi));
                    }
                }
            }
            tc5::fence_proxy_async_smem();
            __syncwarp();
            if (warp == 1) {
                bool w_ok = true;
                if (lane == 0) w_ok = tc5::mbar_wait(&b_full[s], ph, a.wait_ns);
                w_ok = __shfl_sync(0xffffffffu, w_ok ? 1 : 0, 0) != 0;
                __syncwarp();
                if (!w_ok) { ok = false; break; }
            }
            if (lane == 0) tc5::mbar_arrive(&a_full[s]);
            ++step;
        }
        // drain (bounded): the tiles of the last step queued
        if (warp == 1 && lane == 0 && last_tx >= 0)
            tc5::mbar_wait(&b_full[last_tx & 1], (last_tx >> 1) & 1, kWaitNs);
    }
    tc5::tc_fence_before();
    ok = __syncthreads_and(ok) != 0;
    tc5::tc_fence_after();

    if (ok) {
        // warp w reads TMEM lanes 32 * (w % 4) .. + 31; warps 0-3 take the
        // even accumulators, warps 4-7 the odd ones
        const int wl = warp & 3;
        const int i = wl * 32 + lane;                   // TMEM lane = accumulator row
        const int gx = gx0 + i;
        const bool valid = gx < a.Gx_u;
        for (int k = warp >> 2; k < nrow; k += 2) {
            const int64_t g = (int64_t)(gy0 + k) * a.Gx + gx;
            const float cis = valid ? a.c_inv_sigma[g] : 0.f;
            for (int c0 = 0; c0 < a.N; c0 += 8) {
                float v[8];
                tc5::tmem_ld8(tmem + ((uint32_t)(wl * 32) << 16) + (uint32_t)(k * a.N + c0), v);
#pragma unroll
                for (int q2 = 0; q2 < 8; q2 += 2) {
                    const int t = (c0 + q2) >> 1;
                    if (valid && t < a.T) {
                        const float num = v[q2] + v[q2 + 1];
                        // num holds t' scaled by the template's power of two
                        a.rho_tc[t * a.gstride + g] = ((num * a.st[t].tscale_inv) * a.st[t].inv_sigma) * cis;
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    tc5::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc5::tmem_dealloc(tmem, ncols);
}

// Template t' (FP32, m x npad) -> hi/lo fp16 planes 2t, 2t+1 of s t' in the B buffer;
// template t = t0 + blockIdx.y, whose t' is at tf + blockIdx.y * tsz.
__global__ void tmpl_split_kernel(const float *__restrict__ tf, size_t tsz, int m, int n, int npad,
                                  int Kp, int N, int t0, const TmplState *__restrict__ st, __half *B) {
    const int t = t0 + blockIdx.y;
    tf += blockIdx.y * tsz;
    const float sc = st[blockIdx.y].tscale;   // a power of two: exact
    const int total = m * Kp;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += gridDim.x * blockDim.x) {
        const int u = idx / Kp, v = idx % Kp;
        const float x = v < n ? tf[u * npad + v] * sc : 0.f;
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        const int64_t base = (((int64_t)u * (Kp / 8) + v / 8) * (N / 8)) * 64 + (v % 8);
        const int j0 = 2 * t, j1 = 2 * t + 1;
        B[base + (int64_t)(j0 / 8) * 64 + (j0 % 8) * 8] = hi;
        B[base + (int64_t)(j1 / 8) * 64 + (j1 % 8) * 8] = lo;
    }
}

// B2[u0][c][k] = B[u0 - k h][c] (a tile of N x 8 fp16, N * 16 bytes), zero
// where u0 - k h is outside [0, m): the B operand of pivot row cy_0 + u0 for
// a CTA whose RC centre rows are h apart, contiguous.
__global__ void b2_arrange_kernel(const uint4 *__restrict__ B, uint4 *__restrict__ B2, int m, int KB,
                                  int N, int RC, int h, int R2) {
    const int64_t total = (int64_t)R2 * KB * RC * N;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx % N);
        int64_t t = idx / N;
        const int k = (int)(t % RC);
        t /= RC;
        const int c = (int)(t % KB);
        const int u0 = (int)(t / KB);
        const int u = u0 - k * h;
        B2[idx] = (u >= 0 && u < m) ? B[((int64_t)u * KB + c) * N + e] : make_uint4(0u, 0u, 0u, 0u);
    }
}

}  // namespace

size_t corr_mma_bbytes(int m, int Kp, int N, int h) {
    size_t b2 = 0;
    for (int rc = 1; rc <= kMaxRC && rc * N <= 256; ++rc)
        b2 = std::max(b2, (size_t)(m + (rc - 1) * h) * rc * Kp * N * 2);
    return round_up((uint32_t)((size_t)(m + 1) * Kp * N * 2), 1024) + b2;
}

size_t corr_mma_smem(int h, int Kp, int N, int RC) {
    const uint32_t WA = 15u * h + Kp / 8;
    return 1024 + 2 * round_up(WA * 128u, 1024) + 2 * (size_t)round_up((uint32_t)RC * N * Kp * 2u, 1024);
}

cudaError_t launch_tmpl_split(const float *tf, size_t tsz, int T, int m, int n, int npad, int Kp,
                              int N, const TmplState *st, void *B, cudaStream_t s) {
    LaunchScope ls("tmpl_split_kernel", s);
    const int total = m * Kp;
    tmpl_split_kernel<<<dim3((total + 255) / 256, T), 256, 0, s>>>(
        tf, tsz, m, n, npad, Kp, N, 0, st, static_cast<__half *>(B));
    return cudaGetLastError();
}

namespace {

// Centre rows per CTA, in the order preferred before measurement: more rows
// amortise each pivot row's operand build over more MMAs, fewer leave TMEM
// room for more resident CTAs.
constexpr int kRcs[] = {2, 1, 3, 4};

struct MmaTuneKey {
    int m, n, N, h, p, q;
    bool operator<(const MmaTuneKey &o) const {
        return std::tie(m, n, N, h, p, q) < std::tie(o.m, o.n, o.N, o.h, o.p, o.q);
    }
};
std::mutex g_tune_mu;
std::map<MmaTuneKey, int> g_tuned;   // chosen centre rows per CTA

}  // namespace

cudaError_t launch_corr_mma(const uint8_t *V, int p, int q, void *B, int m, int n, int Kp,
                            int N, int h, int Ly, int Lx, int T, const float *c_inv_sigma,
                            const TmplState *st, float *rho_tc, int64_t gstride, int *err,
                            int *Gx_u_out, cudaStream_t s) {
    const int Gy = groups_along(Ly, h), Gx = groups_along(Lx, h);
    // centres along x are uniform (g*h + (h-1)/2) except possibly the last group
    int Gx_u = Gx;
    if (group_centre_of(Gx - 1, Lx, h) != (Gx - 1) * h + (h - 1) / 2) Gx_u = Gx - 1;
    *Gx_u_out = Gx_u;
    if (Gx_u <= 0) return cudaSuccess;
    if (N % 16 != 0 || N < 16 || N > 256 || Kp % 16 != 0) return cudaErrorInvalidValue;
    if (15 * h + Kp / 8 > kMaxRun * ((kMmaThreads - 32) / 8)) return cudaErrorInvalidValue;
    // RC accumulators of N columns: one MMA of RC * N <= 256 columns; shared
    // memory within 227 KB
    auto fits = [&](int rc) {
        return rc <= kMaxRC && rc * N <= 256 && rc <= Gy && corr_mma_smem(h, Kp, N, rc) <= 227 * 1024;
    };
    CorrMmaArgs a;
    a.V = V; a.p = p; a.q = q;
    a.B = static_cast<const __half *>(B);
    a.B2 = reinterpret_cast<const __half *>(static_cast<uint8_t *>(B) +
                                            round_up((uint32_t)((size_t)(m + 1) * Kp * N * 2), 1024));
    a.R2 = 0;
    a.m = m; a.n = n; a.Kp = Kp; a.N = N;
    a.h = h; a.Ly = Ly; a.Lx = Lx; a.Gx = Gx; a.Gx_u = Gx_u;
    a.Gy = Gy;
    a.T = T;
    a.c_inv_sigma = c_inv_sigma;
    a.st = st; a.rho_tc = rho_tc; a.gstride = gstride; a.err = err;
    a.wait_ns = g_wait_ns.load();
    a.stall = g_stall.load();
    auto launch = [&](int rc) -> cudaError_t {
        size_t smem = corr_mma_smem(h, Kp, N, rc);
        // never more resident CTAs per SM than TMEM can hold (512 columns):
        // pad the request so that 228 KB / (request + 1 KB) <= 512 / ncols
        int ncols = 32;
        while (ncols < rc * N) ncols <<= 1;
        const int max_ctas = 512 / ncols;
        const size_t floor_req = (size_t)(228 * 1024) / (size_t)(max_ctas + 1) + 1;
        if (smem + 1024 < floor_req) smem = floor_req - 1024 + 16;
        if (smem > 227 * 1024) return cudaErrorInvalidValue;
        const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(corr_mma_kernel), smem);
        if (e != cudaSuccess) return e;
        a.RC = rc;
        a.R2 = m + (rc - 1) * h;
        {
            const int64_t total = (int64_t)a.R2 * (Kp / 8) * rc * N;
            LaunchScope ls2("b2_arrange_kernel", s);
            b2_arrange_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(
                reinterpret_cast<const uint4 *>(a.B), reinterpret_cast<uint4 *>(const_cast<__half *>(a.B2)),
                m, Kp / 8, N, rc, h, a.R2);
            const cudaError_t e2 = cudaGetLastError();
            if (e2 != cudaSuccess) return e2;
        }
        dim3 grid((Gx_u + kMmaM - 1) / kMmaM, (Gy + rc - 1) / rc);
        LaunchScope ls("corr_mma_kernel", s);
        corr_mma_kernel<<<grid, kMmaThreads, smem, s>>>(a);
        return cudaGetLastError();
    };
    // autotuning: the first launch of a shape times every fitting choice of
    // RC on the real operands (all write the same output, after one untimed
    // launch) and keeps the fastest for the launches that follow
    const MmaTuneKey key{m, n, N, h, p, q};
    int chosen = 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) chosen = it->second;
    }
    if (chosen > 0) return launch(chosen);
    std::vector<int> cand;
    for (int rc : kRcs)
        if (fits(rc)) cand.push_back(rc);
    if (cand.empty()) return cudaErrorInvalidValue;
    // a stream being captured into a graph cannot be timed: first choice
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    if (cand.size() == 1 || cap != cudaStreamCaptureStatusNone) return launch(cand[0]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch(cand[0]);
    float best = 1e30f;
    for (int rc : cand) {
        if (e != cudaSuccess) break;
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch(rc);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) { best = ms; chosen = rc; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = chosen;
    return cudaSuccess;   // the measured launches left the output
}

void set_scan1_wait(uint64_t wait_ns, int stall) {
    g_wait_ns.store(wait_ns ? wait_ns : kWaitNs);
    g_stall.store(stall ? 1 : 0);
}

}  // namespace opta
