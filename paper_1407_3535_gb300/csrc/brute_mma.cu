// The exhaustive rho map (Eq. rho1) on the 5th-generation tensor cores: the
// numerator sum_{u<m, v<n} t'(u,v) (I(y+u, x+v) - 128) at every location.
//
// Residue-class form.  For image row r and the 128 columns x0 + i of a tile:
//
//   D_r[i][j] = sum_{v<Kp} A_r[i][v] B[j][v],   A_r[i][v] = I(r, x0+i+v) - 128,
//   B[j][v]   = t'(m-1-j, v)   (template rows as the N columns, reversed),
//
// so D_r[i][j] is template row u = m-1-j's contribution to output row
// y = r - u.  The accumulator of output row y of a band that starts at
// output row y0 is TMEM column y - y0 + m - 1, so image row r = y0 + k adds
// B's column j into column k + j -- the row shift of the correlation becomes
// a column offset of the accumulator, and each image row's Hankel operand is
// built once and meets the whole template in one MMA chain.  An MMA's
// accumulator starts on a 16-column boundary: image row k writes columns
// [c0, c0 + N + 16) with c0 = k - d, d = k mod 16, against the tile shifted
// by d rows (16 zero rows pad the tile on each side; its 8-row core
// matrices are 128 bytes apart, so rows are 16 bytes apart and a shift of d
// rows is a shift of the descriptor's start address).  The hi and lo bf16
// parts of t' are the two halves of K (K = 2 Kp) against the same A.
// Output row y is complete after the MMAs of image row y + m - 1, and no
// MMA after the next 16-column boundary touches its column, so columns are
// read back 16 at a time while later rows' MMAs run.
//
// A persistent CTA per SM walks the work items (template, band of output
// rows, tile of 128 columns); templates a scan-2 launch does not need
// densely are skipped at the top of the loop.  Warp roles (256 threads; a
// band takes all 512 TMEM columns): warp 0 lane 0 loads the template tile
// (one bulk copy, again when the template changes), the image
// rows (2-D tensor-map tiles of 8 rows x BW bytes into a ring) and issues
// the MMAs; warps 1-3 build each image row's Hankel operand from the ring;
// warps 4-7 clear the accumulator columns, then read 8 completed columns at
// a time and write rho = num / (sigma_t sigma_o) with the map's lower bound
// on the maximum.  Every mbarrier wait is bounded (2 s); a CTA that gives up
// waits for its own copies and MMAs in flight, sets *err and returns.
//
// Error bound: as scan 1's (common.cuh, scan1_epsA_mma) with 2 m Kp/16
// accumulation steps per location (hi and lo in the same accumulator).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "tc5.cuh"

namespace opta {

namespace {

constexpr int kBM = 128;                      // locations per tile (TMEM lanes)
constexpr int kBThreads = 256;
constexpr int kNS = 8;                        // operand stages
constexpr int kEB = 16;                       // columns the read-back takes at once
// the operand build runs at most kGate steps ahead of the read-back, so the
// MMAs never complete a batch two batches beyond the one it waits for (its
// two barriers then never run a phase ahead of its waits)
constexpr int kGate = kEB + kNS - 2;
constexpr int kNR = 8;                        // image boxes in the ring
constexpr int kBR = 8;                        // image rows per box
constexpr uint64_t kBWaitNs = 2000000000ull;  // every wait gives up after 2 s
constexpr int kTmemCols = 512;

__host__ __device__ inline uint32_t rup(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

struct BruteGeom {
    int Kp, N, NB, WA, BW;
    uint32_t bbytes, astride, boxbytes;
    size_t off_b, off_a, off_ring, smem;
};

__host__ __device__ inline BruteGeom brute_geom(int m, int n) {
    BruteGeom g;
    g.Kp = (int)rup((uint32_t)n, 16);
    g.N = (int)rup((uint32_t)m, 16);
    g.WA = 15 + g.Kp / 8;                     // 128-byte operand segments per row
    g.BW = (int)rup((uint32_t)(kBM - 1 + g.Kp), 16);   // image bytes per row (pixels x0 .. x0+126+Kp)
    g.NB = g.N + 32;                          // tile rows: 16 zero rows on each side
    g.bbytes = (uint32_t)g.NB * 2u * (uint32_t)g.Kp * 2u;
    g.astride = rup((uint32_t)g.WA * 128u, 1024);
    g.boxbytes = (uint32_t)kBR * (uint32_t)g.BW;
    g.off_b = 1024;
    g.off_a = g.off_b + rup(g.bbytes, 1024);
    g.off_ring = g.off_a + (size_t)kNS * g.astride;
    // a row's last operand words may read up to 16 bytes past the ring
    g.smem = g.off_ring + (size_t)kNR * g.boxbytes + 16;
    return g;
}

struct BruteArgs {
    int p, q, m, n, Ly, Lx, RB;
    int tiles, bands, T;        // work items: T templates x bands x column tiles
    const __nv_bfloat16 *B;     // template k's tile at B + k * (bbytes / 2): [2Kp/8][NB/8][8][8]
    const float *inv_sigma;     // 1/Omega per location (0: flat window)
    const float *efac;          // ||I - 128|| / Omega per location (null: from wsum)
    const int *wsum;            // window sums (the integer operand's mean term; the
                                // error factor when efac is null)
    TmplState *st;              // template k's state at st + k
    float *map;                 // template k's map at map + k * map_stride
    int64_t map_stride;
    int dense_only;             // skip templates without st->dense
    int *err;
    float epsA;
};

__device__ inline bool wait_warp(uint64_t *bar, uint32_t parity, int lane) {
    bool ok = true;
    if (lane == 0) ok = tc5::mbar_wait(bar, parity, kBWaitNs);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    return ok;
}

// AND of `v` over the 128 threads of the read-back warps (named barrier 1).
__device__ inline bool readback_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n"
        " barrier.cta.red.and.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(r)
        : "r"(v ? 1u : 0u)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(kBThreads, 1)
brute_mma_kernel(const __grid_constant__ CUtensorMap tmap, const BruteArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const BruteGeom g = brute_geom(a.m, a.n);
    uint64_t *img_full = reinterpret_cast<uint64_t *>(smem);   // [kNR] image box landed
    uint64_t *a_full = img_full + kNR;                          // [kNS] operand built (3 warps)
    uint64_t *mma_done = a_full + kNS;                          // [kNS] MMAs of the stage completed
    uint64_t *acc_full = mma_done + kNS;                        // [2] a batch of kEB columns done
    uint64_t *b_full = acc_full + 2;                            // template tile landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(b_full + 1);
    volatile int *epi_done = reinterpret_cast<volatile int *>(tmem_slot + 1);   // steps read back
    uint8_t *Bs = smem + g.off_b;
    uint8_t *As = smem + g.off_a;
    uint8_t *ring = smem + g.off_ring;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kNR; ++i) tc5::mbar_init(&img_full[i], 1);
        for (int i = 0; i < kNS; ++i) {
            tc5::mbar_init(&a_full[i], 3);
            tc5::mbar_init(&mma_done[i], 1);
        }
        tc5::mbar_init(&acc_full[0], 1);
        tc5::mbar_init(&acc_full[1], 1);
        tc5::mbar_init(b_full, 1);
        tc5::fence_mbar_init();
    }
    if (warp == 0) {
        tc5::tmem_alloc(tmem_slot, kTmemCols);
        tc5::tmem_relinquish();
    }
    tc5::tc_fence_before();
    __syncthreads();
    tc5::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // Work items (template z, band, column tile), one CTA per SM looping over
    // them.  Every barrier phase follows from running counters over the items
    // this CTA has processed (steps, image boxes, read-back batches, template
    // tiles), which all roles advance alike, so each barrier is waited for
    // phase by phase across items.
    const int per_t = a.tiles * a.bands;
    const int n_items = per_t * a.T;
    int gstep = 0, gbox = 0, gbatch = 0, gtile = 0, curz = -1;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const int z = item / per_t, r = item - z * per_t;
        TmplState *st = a.st + z;
        if (st->flat || (a.dense_only && !st->dense)) continue;   // uniform
        const int by = r / a.tiles, bx = r - by * a.tiles;
        const int x0 = bx * kBM;
        const int y0 = by * a.RB;
        const int yend = min(a.Ly, y0 + a.RB);
        const int nsteps = (yend - y0) + a.m - 1;   // image rows y0 .. yend + m - 2
        const int nbox = (nsteps + kBR - 1) / kBR;
        const int nbatch = (nsteps + kEB - 1) / kEB;
        const bool new_tile = z != curz;
        // the accumulators start at zero: every MMA accumulates
        if (warp >= 4) {
            const uint32_t lanebase = (uint32_t)((warp & 3) * 32) << 16;
            for (int c = 0; c < kTmemCols; c += 8) tc5::tmem_st8_zero(tmem + lanebase + (uint32_t)c);
            tc5::tmem_wait_st();
        }
        if (tid == 0) *epi_done = 0;
        tc5::tc_fence_before();
        __syncthreads();
        tc5::tc_fence_after();

        if (warp == 0) {
            if (lane == 0) {
                const int KS = g.Kp / 16;
                const uint32_t idesc = tc5::idesc_bf16_f32(kBM, g.N + 16);
                const uint32_t blbo = (uint32_t)(g.NB / 8) * 128u;
                if (new_tile) {
                    // (the previous item's MMAs were drained: the tile is free)
                    tc5::mbar_arrive_expect_tx(b_full, g.bbytes);
                    tc5::bulk_g2s(Bs, a.B + (size_t)z * (g.bbytes / 2), g.bbytes, b_full);
                }
                int issued = 0;   // image boxes issued for this item
                for (; issued < min(kNR, nbox); ++issued) {
                    const int gb = gbox + issued;
                    tc5::mbar_arrive_expect_tx(&img_full[gb % kNR], g.boxbytes);
                    tc5::tma_load_2d(ring + (gb % kNR) * g.boxbytes, &tmap, x0, y0 + kBR * issued,
                                     &img_full[gb % kNR]);
                }
                if (new_tile) ok = tc5::mbar_wait(b_full, (uint32_t)(gtile & 1), kBWaitNs);
                const uint32_t bbase = tc5::smem_u32(Bs);
                int last = -1;
                for (int k = 0; ok && k < nsteps; ++k) {
                    const int G = gstep + k, s = G % kNS;
                    if (!tc5::mbar_wait(&a_full[s], (uint32_t)((G / kNS) & 1), kBWaitNs)) {
                        ok = false;
                        break;
                    }
                    // the builders are done with image row k: after a box's last
                    // row its slot takes the box kNR further on
                    if ((k % kBR) == kBR - 1 && issued < nbox) {
                        const int gb = gbox + issued;
                        tc5::mbar_arrive_expect_tx(&img_full[gb % kNR], g.boxbytes);
                        tc5::tma_load_2d(ring + (gb % kNR) * g.boxbytes, &tmap, x0, y0 + kBR * issued,
                                         &img_full[gb % kNR]);
                        ++issued;
                    }
                    tc5::tc_fence_after();
                    const uint32_t abase = tc5::smem_u32(As + s * g.astride);
                    const int dsh = k & 15;
                    const uint32_t d = tmem + (uint32_t)(k - dsh);            // 16-column aligned
                    const uint32_t bsh = bbase + (uint32_t)(16 - dsh) * 16u;   // tile shifted by dsh rows
                    for (int kk = 0; kk < 2 * KS; ++kk) {
                        const int ka = kk < KS ? kk : kk - KS;   // hi and lo halves share A
                        const uint64_t ad = tc5::smem_desc(abase + (uint32_t)ka * 256u, 128, 128);
                        const uint64_t bd = tc5::smem_desc(bsh + (uint32_t)kk * 2u * blbo, blbo, 128);
                        tc5::mma_bf16(d, ad, bd, idesc, true);
                    }
                    tc5::mma_commit(&mma_done[s]);
                    // the read-back's barriers: one phase per batch of kEB steps, so
                    // that each is waited for phase by phase
                    if (k % kEB == kEB - 1 || k == nsteps - 1)
                        tc5::mma_commit(&acc_full[(gbatch + k / kEB) & 1]);
                    last = G;
                }
                // drain (bounded): the item's last MMAs, then every image box in flight
                if (last >= 0 && !tc5::mbar_wait(&mma_done[last % kNS], (uint32_t)((last / kNS) & 1), kBWaitNs))
                    ok = false;
                for (int b = max(0, issued - kNR); b < issued; ++b) {
                    const int gb = gbox + b;
                    if (!tc5::mbar_wait(&img_full[gb % kNR], (uint32_t)((gb / kNR) & 1), kBWaitNs)) ok = false;
                }
            }
        } else if (warp < 4) {
            // operand builders: segment w of stage s holds 8 copies b of the 8
            // pixels from column b + 8w of image row k (a Hankel operand with
            // shift 1: element (i = 8a + b, v = 8c + d) at byte (a + c) * 128 +
            // 16 b + 2 d)
            const int bt = tid - 32;
            for (int k = 0; k < nsteps; ++k) {
                const int G = gstep + k, s = G % kNS;
                if (G >= kNS && !wait_warp(&mma_done[s], (uint32_t)(((G / kNS) & 1) ^ 1), lane)) {
                    ok = false;
                    break;
                }
                if (k > kGate) {
                    bool w_ok = true;
                    if (lane == 0) {
                        const uint64_t t0 = tc5::globaltimer();
                        while (*epi_done < k - kGate) {
                            if (tc5::globaltimer() - t0 > kBWaitNs) { w_ok = false; break; }
                        }
                    }
                    w_ok = __shfl_sync(0xffffffffu, w_ok ? 1 : 0, 0) != 0;
                    __syncwarp();
                    if (!w_ok) { ok = false; break; }
                }
                const int gb = gbox + k / kBR;
                if ((k % kBR) == 0 && !wait_warp(&img_full[gb % kNR], (uint32_t)((gb / kNR) & 1), lane)) {
                    ok = false;
                    break;
                }
                const uint8_t *row = ring + (gb % kNR) * g.boxbytes + (k % kBR) * g.BW;
                uint8_t *Ab = As + s * g.astride;
                for (int j = bt; j < g.WA * 8; j += 96) {
                    const int c = (j & 7) + 8 * (j >> 3);
                    const uint32_t *wp = reinterpret_cast<const uint32_t *>(row + (c & ~3));
                    const uint32_t sh = (uint32_t)(c & 3) * 8u;
                    const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2];
                    const uint32_t lo = __funnelshift_r(w0, w1, sh);
                    const uint32_t hi = __funnelshift_r(w1, w2, sh);
                    *reinterpret_cast<uint4 *>(Ab + (j >> 3) * 128 + (j & 7) * 16) =
                        make_uint4(tc5::bytes_bf16x2<0>(lo), tc5::bytes_bf16x2<2>(lo),
                                   tc5::bytes_bf16x2<0>(hi), tc5::bytes_bf16x2<2>(hi));
                }
                tc5::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc5::mbar_arrive(&a_full[s]);
            }
        } else {
            // read-back: columns [k0, k0 + 16) once the MMAs of step k0 + 15 are
            // done (later MMAs start at column k0 + 16 or beyond)
            const int wl = warp & 3;
            const uint32_t lanebase = (uint32_t)(wl * 32) << 16;
            const int x = x0 + wl * 32 + lane;
            const bool xv = x < a.Lx;
            const float inv_t = st->inv_sigma;
            const float c0 = st->c0;   // integer operand: t' = (t - rint(mu)) + c0
            const float c128 = 128.f * (float)(a.m * a.n), imn = 1.f / (float)(a.m * a.n);
            float *map = a.map + (int64_t)z * a.map_stride;
            float lo = -3.f;
            for (int k0 = 0; k0 < nsteps; k0 += kEB) {
                const int kb = min(k0 + kEB, nsteps) - 1;
                const int batch = gbatch + k0 / kEB;
                // the four warps agree (one barrier per batch) before any leaves;
                // passing it also means all four have seen step kb complete,
                // which is the progress the operand builders wait for
                if (!readback_all(wait_warp(&acc_full[batch & 1], (uint32_t)((batch >> 1) & 1), lane))) {
                    ok = false;
                    break;
                }
                if (tid == 128) *epi_done = kb + 1;
                tc5::tc_fence_after();
                float v[kEB];
                tc5::tmem_ld8(tmem + lanebase + (uint32_t)k0, *reinterpret_cast<float(*)[8]>(&v[0]));
                tc5::tmem_ld8(tmem + lanebase + (uint32_t)k0 + 8u, *reinterpret_cast<float(*)[8]>(&v[8]));
#pragma unroll
                for (int c = 0; c < kEB; ++c) {
                    const int y = y0 + k0 + c - (a.m - 1);
                    if (k0 + c > kb || y < y0 || y >= yend || !xv) continue;
                    const int64_t idx = (int64_t)y * a.Lx + x;
                    const float is = a.inv_sigma[idx];
                    // sum t'(I - 128) = sum (t - rint(mu))(I - 128) + c0 (S - 128 mn),
                    // S - 128 mn exact (integers below 2^24)
                    const float acc = c0 != 0.f ? fmaf(c0, (float)a.wsum[idx] - c128, v[c]) : v[c];
                    const float rho = (acc * inv_t) * is;
                    map[idx] = rho;
                    if (is > 0.f) {
                        float ef;
                        if (a.efac) {
                            ef = a.efac[idx];
                        } else {
                            const float dd = ((float)a.wsum[idx] - c128) * is;
                            ef = sqrtf(fmaf(dd * dd, imn, 1.f));
                        }
                        lo = fmaxf(lo, rho - fmaf(a.epsA, ef, 8.f * kU32));
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) lo = fmaxf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            if (lane == 0 && lo > -2.5f) atomicMax(&st->lo_key, float_key(lo));
        }
        // every role is done with the item (the issuer drained its MMAs and
        // image boxes) before the next one clears the accumulators
        tc5::tc_fence_before();
        ok = __syncthreads_and(ok) != 0;
        tc5::tc_fence_after();
        gstep += nsteps;
        gbox += nbox;
        gbatch += nbatch;
        if (new_tile) ++gtile;
        curz = z;
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    tc5::tc_fence_before();
    __syncthreads();
    tc5::tc_fence_after();
    if (warp == 0) tc5::tmem_dealloc(tmem, kTmemCols);
}

// t' (FP32, m x npad) -> the template tile of NB = N + 32 rows: row 16 + j
// holds template row m-1-j (j < m), every other row is zero; K halves
// hi | lo of the bf16 split, zeros past n columns.
// A template of integers in 0..255 with sigma_t >= sqrt(mn) / 6 (int_op)
// takes instead hi = t - rint(mu) (an integer of at most 8 significant bits:
// exact in bf16) and lo = 0; the epilogue adds c0 (S - 128 mn) with
// c0 = rint(mu) - mu.  Its products are then exact and only the FP32
// accumulation rounds: at most m Kp / 16 steps of u |partial sum|, i.e.
// (m Kp / 16) u (||hi|| / sigma_t) ||I - 128|| / Omega with ||hi|| <=
// sigma_t + sqrt(mn) / 2 <= 4 sigma_t, plus the correction's few roundings
// (each below u ||I - 128|| sqrt(mn) / 2 / (sigma_t Omega) <= 3 u efac):
// within the split's bound brute_mma_epsA, which allows (8 m Kp / 16 + 16) u
// efac besides the split's residual term.
__global__ void brute_tmpl_kernel(const float *__restrict__ tf, size_t tsz, int m, int n, int npad,
                                  int Kp, int NB, const TmplState *st, int dense_only,
                                  __nv_bfloat16 *B) {
    // template blockIdx.y (dense_only: only templates marked dense)
    if (dense_only && !st[blockIdx.y].dense) return;
    const bool int_op = st[blockIdx.y].int_op != 0;
    const float c0 = st[blockIdx.y].c0;
    tf += blockIdx.y * tsz;
    const int total = NB * 2 * Kp;
    B += (size_t)blockIdx.y * total;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int jj = idx / (2 * Kp), kk = idx - jj * 2 * Kp;
        const int v = kk < Kp ? kk : kk - Kp;
        const int u = m - 1 - (jj - 16);
        float x = 0.f;
        if (jj >= 16 && u >= 0 && v < n) x = tf[u * npad + v];
        // t - rint(mu) = t' - c0, recovered exactly by rounding (t' is t - mu
        // within 255 u)
        if (int_op) x = rintf(x - c0);
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 part =
            kk < Kp ? hi : (int_op ? __float2bfloat16_rn(0.f) : __float2bfloat16_rn(x - __bfloat162float(hi)));
        B[((int64_t)(kk / 8) * (NB / 8) + jj / 8) * 64 + (jj % 8) * 8 + kk % 8] = part;
    }
}

__global__ void pad_rows_kernel(const uint8_t *__restrict__ I, int p, int q, uint8_t *out, int qs) {
    const int64_t total = (int64_t)p * qs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / qs), x = (int)(i - (int64_t)y * qs);
        out[i] = x < q ? I[(int64_t)y * q + x] : (uint8_t)0;
    }
}

// The driver's tensor-map encoder, looked up through the runtime (the
// library links no driver symbol, so it loads on machines without one).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool brute_mma_supported(int m, int n) { return m >= 1 && n >= 1 && m <= 128 && n <= 128; }

size_t brute_tmpl_bytes(int m, int n) { return brute_geom(m, n).bbytes; }

float brute_mma_epsA(int m, int n) {
    // 2 m Kp/16 accumulation steps per location: scan 1's bound for 2m rows
    return scan1_epsA_mma(2 * m, (int)rup((uint32_t)n, 16));
}

cudaError_t launch_brute_tmpl(const float *tf, size_t tsz, int T, int m, int n, int npad, void *B,
                              const TmplState *st, int dense_only, cudaStream_t s) {
    if (!st) return cudaErrorInvalidValue;
    const BruteGeom g = brute_geom(m, n);
    const int total = g.NB * 2 * g.Kp;
    LaunchScope ls("brute_tmpl_kernel", s);
    brute_tmpl_kernel<<<dim3((total + 255) / 256, T), 256, 0, s>>>(tf, tsz, m, n, npad, g.Kp, g.NB,
                                                                  st, dense_only,
                                                                  static_cast<__nv_bfloat16 *>(B));
    return cudaGetLastError();
}

cudaError_t launch_pad_rows(const uint8_t *I, int p, int q, uint8_t *out, int qs, cudaStream_t s) {
    const int64_t total = (int64_t)p * qs;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16));
    LaunchScope ls("pad_rows_kernel", s);
    pad_rows_kernel<<<grid, 256, 0, s>>>(I, p, q, out, qs);
    return cudaGetLastError();
}

cudaError_t launch_brute_mma(const uint8_t *Ipad, int qs, int p, int q, const void *B, int m, int n,
                             const float *inv_sigma, const float *efac, const int *wsum,
                             TmplState *st, float *map, int64_t map_stride, int T, int dense_only,
                             int *err, cudaStream_t s) {
    if (!brute_mma_supported(m, n) || qs % 16 != 0 || qs < q || T < 1 || T > 65535 || !wsum)
        return cudaErrorInvalidValue;
    const BruteGeom g = brute_geom(m, n);
    const int Ly = p - m + 1, Lx = q - n + 1;
    // a band's columns: the last MMA writes up to column (nsteps - 1) + N + 16
    // (exclusive) and the last read-back up to nsteps - 1 + 16, both within
    // 512 when nsteps = RB + m - 1 <= 497 - N
    const int rb_max = kTmemCols - 14 - m - g.N;
    if (rb_max < 1) return cudaErrorInvalidValue;
    const int tiles = (Lx + kBM - 1) / kBM;
    // bands: a CTA's time is about its image rows (RB + m - 1 MMA steps) and
    // one CTA runs per SM, so take the band count with the fewest waves x
    // steps (ties: fewer bands)
    const int sms = num_sms();
    const int b_min = (Ly + rb_max - 1) / rb_max;
    int bands = b_min;
    int64_t best = -1;
    for (int b = b_min; b <= std::min(Ly, 8 * b_min + 2 * sms); ++b) {
        const int64_t waves = ((int64_t)tiles * b + sms - 1) / sms;
        const int64_t t = waves * ((Ly + b - 1) / b + m - 1);
        if (best < 0 || t < best) { best = t; bands = b; }
    }
    const int RB = (Ly + bands - 1) / bands;
    bands = (Ly + RB - 1) / RB;

    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[2] = {(cuuint64_t)q, (cuuint64_t)p};
    const cuuint64_t strides[1] = {(cuuint64_t)qs};
    const cuuint32_t box[2] = {(cuuint32_t)g.BW, (cuuint32_t)kBR};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(Ipad), dims,
                               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // one CTA per SM (its band holds all of TMEM): at least half the shared memory
    const size_t smem = std::max<size_t>(g.smem, 116 * 1024);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const cudaError_t e = ensure_smem(reinterpret_cast<const void *>(brute_mma_kernel), smem);
    if (e != cudaSuccess) return e;
    BruteArgs a;
    a.p = p; a.q = q; a.m = m; a.n = n; a.Ly = Ly; a.Lx = Lx; a.RB = RB;
    a.B = static_cast<const __nv_bfloat16 *>(B);
    a.inv_sigma = inv_sigma; a.efac = efac; a.wsum = wsum; a.st = st; a.map = map;
    a.map_stride = map_stride; a.dense_only = dense_only; a.err = err;
    a.epsA = brute_mma_epsA(m, n);
    a.tiles = tiles; a.bands = bands; a.T = T;
    // persistent: one CTA per SM walks the (template, band, tile) items
    const int64_t items = (int64_t)tiles * bands * T;
    if (items > 0x7fffffff) return cudaErrorInvalidValue;
    const int grid = (int)std::min<int64_t>(items, sms);
    LaunchScope ls("brute_mma_kernel", s);
    brute_mma_kernel<<<grid, kBThreads, smem, s>>>(tm, a);
    return cudaGetLastError();
}

}  // namespace opta
