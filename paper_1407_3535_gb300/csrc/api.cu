// C ABI of libopta.so: handle lifecycle, OptA preparation driver
// (Algorithms 2 and 3), per-template search sequencing (Sections 2 and 6)
// and the exhaustive search.  All device work is enqueued on the caller's
// stream; host decisions of the preparation loop read back a few scalars.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>
#include <new>
#include <shared_mutex>
#include <thread>
#include <utility>
#include <vector>

#include "common.cuh"
#include "opta_debug.h"

using namespace opta;

namespace {

opta_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return OPTA_OK;
    cudaGetLastError();   // clear the non-sticky error state
    return e == cudaErrorMemoryAllocation ? OPTA_ERR_OOM : OPTA_ERR_CUDA;
}

#define CK(x)                                                    \
    do {                                                         \
        cudaError_t e__ = (x);                                   \
        if (e__ != cudaSuccess) return map_err(e__);             \
    } while (0)
#define TRY(x)                                                   \
    do {                                                         \
        opta_status s__ = (x);                                   \
        if (s__ != OPTA_OK) return s__;                          \
    } while (0)

constexpr int kMaxRadius = 9;
constexpr int kChunk = 128;   // templates per batch (tensor-core N = 2 * chunk <= 256)
// Device bytes the per-template scan-2 arrays of one batch may take (28 bytes
// per location and template: survivor index, bound, rho, error bound,
// candidate index and its FP64 rho).
constexpr size_t kScan2Budget = (size_t)8 << 30;

// Device allocation that keeps a running byte count (host threads that
// prepare sizes concurrently share it).
struct DevMem {
    std::atomic<size_t> bytes{0};
    template <class T>
    opta_status alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        void *v = nullptr;
        cudaError_t e = cudaMalloc(&v, count * sizeof(T));
        if (e != cudaSuccess) { cudaGetLastError(); return OPTA_ERR_OOM; }
        bytes += count * sizeof(T);
        *p = static_cast<T *>(v);
        return OPTA_OK;
    }
    template <class T>
    void release(T *&p, size_t count) {
        if (p) { cudaFree(p); bytes -= (count ? count : 1) * sizeof(T); p = nullptr; }
    }
};

struct SizeState {
    int m = 0, n = 0, Ly = 0, Lx = 0, Gy = 0, Gx = 0;
    int h = 1, level = 0, n_evals = 0;
    long long cost = 0;
    uint8_t *P = nullptr;          // pivot image (owned unless it aliases the image)
    bool P_owned = false;
    float *inv_sigma = nullptr;    // L
    int *wsum = nullptr;           // L window sums of I
    float *rho_co = nullptr;       // L
    float2 *theta_co = nullptr;    // L angle intervals of rho_co
    float2 *gco = nullptr;         // G union of the members' angle intervals per group
    float *c_inv_sigma = nullptr;  // G
    float *c_efac = nullptr;       // G
    std::vector<float> sigma_map;
    // The image the search runs on (its members) with its window statistics:
    // I with wsum / inv_sigma, or in the literal mode (Section 4.3) the
    // accepted pivot with statistics of its own (owned when M_owned).
    const uint8_t *M = nullptr;
    int *wsumM = nullptr;
    float *invM = nullptr;
    bool M_owned = false;
    int d = 0;                     // literal mode: half-width of the re-match on I
};

}  // namespace

// Search scratch and per-template states of one search context: searches
// of one handle through different contexts may run concurrently (each on
// its own stream); a context runs one search at a time.
struct opta_search_ctx {
    int device = 0;
    DevMem mem;
    std::atomic<bool> busy{false};
    size_t capL = 0, capG = 0, capT = 0, capN = 0;
    size_t capS2 = 0;                         // template slots of the scan-2 arrays (stride capL)
    int *ucnt = nullptr;                      // kScan2MaxT unordered-survivor counters
    float *rho_tc = nullptr;
    int *surv = nullptr;
    float *surv_rho = nullptr, *surv_eps = nullptr, *surv_ub = nullptr;
    int *bucket_cnt = nullptr, *bucket_cur = nullptr;
    int *cand = nullptr;
    double *cand_rho = nullptr;
    float *topk_v = nullptr;                  // chunk x 256 x kTopkMax
    int *topk_i = nullptr;
    int *cand_topk = nullptr;                 // chunk x kTopkMax threshold centres
    double *cand_rho_topk = nullptr;
    TmplIn *tin = nullptr;                    // template descriptors, one slot per template
    float *tf = nullptr, *tstage = nullptr;   // tf: chunk of templates, m x npad each
    double *td = nullptr;                     // chunk of templates, m x n each
    TmplState *states = nullptr;
    // pinned host mirrors, one slot per template (read by copies queued on a
    // stream, so a slot is not rewritten until its search has finished; and
    // copies from pinned memory can be captured in a CUDA graph)
    TmplIn *tin_host = nullptr;
    TmplState *states_host = nullptr;
    int *err_host = nullptr;
    size_t capTS = 0, capB = 0, capRT = 0;    // template-slot, B-buffer, rho_tc capacities
    void *Bmma = nullptr;                     // bf16 hi/lo planes of a chunk (core-matrix layout)
    int *dev_err = nullptr;                   // set by a kernel whose bounded wait gave up
    TmplState *tune_st = nullptr;             // the survivor-form tuner's template state
    unsigned long long *tune_span = nullptr;  // and the span of its timed sweeps
};

struct opta_handle {
    int p = 0, q = 0, device = 0;
    opta_params prm;
    DevMem mem;
    uint8_t *I8 = nullptr;
    uint8_t *Ipad = nullptr;                  // I8 with rows padded to qs bytes (tensor-map copies)
    int qs = 0;
    long long *IIS = nullptr, *IIQ = nullptr;
    std::map<std::pair<int, int>, SizeState *> sizes;
    std::shared_mutex sizes_rw;               // `sizes`: shared while searches use it, exclusive to insert
    cudaMemPool_t pool = nullptr;             // stream-ordered scratch of the preparation
    opta_search_ctx *dctx = nullptr;          // the context of optA_search (created on first use)
    std::mutex prep_mu;                       // one preparation of new sizes at a time
    // blur tables
    float *weights = nullptr;
    int *radius = nullptr;
    std::atomic<bool> busy{false};
};

namespace {

bool valid_params(const opta_params &p) {
    if (!(p.rho_th > -1.0 && p.rho_th < 1.0)) return false;
    if (!(p.rho_max >= -1.0 && p.rho_max <= 1.0)) return false;
    if (!(p.xi >= 0.0)) return false;
    if (p.block < 8 || p.block > 128) return false;
    if (p.n_levels < 0 || p.n_levels > 8) return false;
    for (int i = 0; i < p.n_levels; ++i)
        if (!(p.sigma_levels[i] > 0.f && p.sigma_levels[i] <= 3.0f)) return false;
    if (p.h_max < 1 || p.h_max > 9 || (p.h_max % 2) == 0) return false;
    if (p.fixed_h < 0 || p.fixed_h > 9 || (p.fixed_h > 0 && p.fixed_h % 2 == 0)) return false;
    if (p.topk < 1 || p.topk > kTopkMax) return false;
    if (p.precision != 0 && p.precision != 1) return false;
    if (p.literal != 0 && p.literal != 1) return false;
    if (p.egs_sample < 0 || p.egs_sample > 64) return false;
    if (p.dense < 0 || p.dense > 2) return false;
    if (!(p.dense_cut >= 0.f && p.dense_cut < 1e9f)) return false;
    return true;
}

double lambda_of(double rth, double rmax) {   // Eq. misDec
    const double r = 1.0 + rth * rth * rmax * rmax - (rth * rth + rmax * rmax);
    return rth * rmax + std::sqrt(r > 0.0 ? r : 0.0);
}

// 1-D normalised Gaussian weights for the level table (radius ceil(3 sigma)).
void gauss_table(const opta_params &prm, std::vector<float> &w, std::vector<int> &rad) {
    const int L = prm.n_levels + 1;
    w.assign((size_t)L * (kMaxRadius + 1), 0.f);
    rad.assign(L, 0);
    for (int l = 1; l < L; ++l) {
        const double s = prm.sigma_levels[l - 1];
        const int R = (int)std::ceil(3.0 * s);
        rad[l] = R;
        double tot = 0.0;
        std::vector<double> g(R + 1);
        for (int i = 0; i <= R; ++i) g[i] = std::exp(-(double)(i * i) / (2.0 * s * s));
        for (int i = -R; i <= R; ++i) tot += g[i < 0 ? -i : i];
        for (int i = 0; i <= R; ++i) w[(size_t)l * (kMaxRadius + 1) + i] = (float)(g[i] / tot);
    }
}

opta_status ingest(const opta_image *img, uint8_t *dst, cudaStream_t s) {
    const int p = img->rows, q = img->cols;
    const int64_t ld = img->stride_elems;
    if (img->dtype == OPTA_U8) {
        if (img->on_device) {
            CK(launch_ingest_u8(static_cast<const uint8_t *>(img->data), ld, p, q, dst, s));
        } else {
            CK(cudaMemcpy2DAsync(dst, q, img->data, ld, q, p, cudaMemcpyHostToDevice, s));
        }
        return OPTA_OK;
    }
    // float32: must hold integers in [0, 255]
    const float *src = static_cast<const float *>(img->data);
    float *staging = nullptr;
    int *bad = nullptr;
    CK(cudaMallocAsync(&bad, sizeof(int), s));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    int64_t sld = ld;
    if (!img->on_device) {
        CK(cudaMallocAsync(&staging, (size_t)p * q * sizeof(float), s));
        CK(cudaMemcpy2DAsync(staging, (size_t)q * sizeof(float), src, ld * sizeof(float),
                             (size_t)q * sizeof(float), p, cudaMemcpyHostToDevice, s));
        src = staging;
        sld = q;
    }
    CK(launch_ingest_f32(src, sld, p, q, dst, bad, s));
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (staging) CK(cudaFreeAsync(staging, s));
    CK(cudaFreeAsync(bad, s));
    CK(cudaStreamSynchronize(s));
    return hbad ? OPTA_ERR_UNSUPPORTED : OPTA_OK;
}

bool valid_image(const opta_image *img) {
    return img && img->data && img->rows > 0 && img->cols > 0 &&
           img->stride_elems >= img->cols && (img->dtype == OPTA_U8 || img->dtype == OPTA_F32) &&
           (int64_t)img->rows * img->cols < (int64_t)1 << 31;
}

bool valid_template(const opta_template *t, int p, int q) {
    return t && t->data && t->rows > 0 && t->cols > 0 && t->stride_elems >= t->cols &&
           t->rows <= p && t->cols <= q && t->cols <= 1024;
}

// ---------------------------------------------------------------------------
// Preparation of one template size: Algorithm 3 (OptA) driving Algorithm 2
// (EGS) under the readings documented with the oracle.
// ---------------------------------------------------------------------------
struct PrepScratch {
    uint8_t *Pcur = nullptr, *Pacc = nullptr;
    int *fail = nullptr;
    uint8_t *lvl = nullptr;
    unsigned long long *count = nullptr;
    // literal mode: integral images and window statistics of a candidate pivot
    long long *IIS = nullptr, *IIQ = nullptr;
    int *wsumP = nullptr;
    float *invP = nullptr;
};

// Members of the auto-correlation EGS measures: image M (I, or the candidate
// pivot itself in the literal mode) with its window sums and 1/Omega.
struct Members {
    const uint8_t *M;
    const int *wsum;
    const float *inv;
};

// Location rows EGS counts for group side h: the rows of the group rows g
// with (g / kEgsRun) % sample == 0 (every row when sample == 1).
int64_t egs_rows(int Ly, int h, int sample) {
    if (sample <= 1) return Ly;
    const int Gy = groups_along(Ly, h);
    int64_t rows = 0;
    for (int g0 = 0; g0 < Gy; g0 += kEgsRun * sample) {
        const int g1 = std::min(Gy, g0 + kEgsRun);
        rows += std::min<int64_t>((int64_t)g1 * h, Ly) - (int64_t)g0 * h;
    }
    return rows;
}

// Queue the retained count of group side h (Algorithm 2's n_r) over EGS's
// sample of the location grid into dcount.  Counts only: no map is stored.
opta_status egs_launch(opta_handle *H, SizeState *S, const uint8_t *P, const Members &M, int h,
                       unsigned long long *dcount, cudaStream_t s) {
    const float cut = (float)std::sqrt(1.0 - H->prm.rho_th * H->prm.rho_th);
    const int sample = std::max(1, H->prm.egs_sample);
    CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s));
    if (h == 1 && P == M.M) {
        // pivots equal to the members, one location per group: every member
        // is its own centre, rho_co = 1 except on flat windows (rho_co = 0
        // there), so the retained count is the number of flat windows
        CK(launch_count_zero(M.inv, S->Ly, S->Lx, 1, sample, dcount, s));
    } else {
        CK(launch_rho_co(P, M.M, H->p, H->q, S->m, S->n, h, M.wsum, M.inv, cut, nullptr, dcount,
                         nullptr, nullptr, s, sample));
    }
    S->n_evals++;
    return OPTA_OK;
}

// Wait for k queued counts (group sides hs[]) and turn them into costs
// (groups + retained, Eq. objfunc); a sampled count is scaled to the whole
// grid by Ly / (rows sampled), rounded to the nearest integer.
opta_status egs_read(opta_handle *H, SizeState *S, const int *hs, int k,
                     const unsigned long long *dcount, unsigned long long *host, long long *cost,
                     cudaStream_t s) {
    CK(cudaMemcpyAsync(host, dcount, (size_t)k * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int sample = std::max(1, H->prm.egs_sample);
    for (int i = 0; i < k; ++i) {
        const int64_t rows = egs_rows(S->Ly, hs[i], sample);
        const long long nr = ((long long)host[i] * S->Ly + rows / 2) / rows;
        cost[i] = (long long)groups_along(S->Ly, hs[i]) * groups_along(S->Lx, hs[i]) + nr;
    }
    return OPTA_OK;
}

// Largest odd group side <= hmax the auto-correlation kernel supports for
// m x n windows of a p x q image (0: none).
int h_limit(int p, int q, int m, int n, int hmax) {
    int h = hmax;
    while (h >= 1 && !rho_co_supported(p, q, m, n, h)) h -= 2;
    return h;
}

// Algorithm 2: grow h by 2 while the cost drops by more than xi of the last.
// dcount: two device counters.  The first two sides (h and h + 2, both
// always evaluated when h + 2 is allowed) are queued together and read with
// one wait; each further side takes one more.
opta_status egs(opta_handle *H, SizeState *S, const uint8_t *P, const Members &M, int h_start,
                unsigned long long *dcount, int *h_out, long long *c_out, cudaStream_t s) {
    const int hmax = h_limit(H->p, H->q, S->m, S->n, H->prm.h_max);
    unsigned long long host[2];
    long long cost[2];
    int h = std::min(h_start, hmax);
    const bool pair = h + 2 <= hmax;
    TRY(egs_launch(H, S, P, M, h, dcount, s));
    if (pair) TRY(egs_launch(H, S, P, M, h + 2, dcount + 1, s));
    const int hs[2] = {h, h + 2};
    TRY(egs_read(H, S, hs, pair ? 2 : 1, dcount, host, cost, s));
    long long c = cost[0];
    bool grow = pair;
    long long c2 = cost[1];
    while (grow) {
        if (!((double)(c - c2) > H->prm.xi * (double)c)) break;
        h += 2; c = c2;
        if (h + 2 > hmax) break;
        TRY(egs_launch(H, S, P, M, h + 2, dcount, s));
        const int hn[1] = {h + 2};
        TRY(egs_read(H, S, hn, 1, dcount, host, cost, s));
        c2 = cost[0];
    }
    *h_out = h;
    *c_out = c;
    return OPTA_OK;
}

opta_status blur_to(opta_handle *H, PrepScratch &W, const std::vector<uint8_t> &levels,
                    uint8_t *P, cudaStream_t s) {
    CK(cudaMemcpyAsync(W.lvl, levels.data(), levels.size(), cudaMemcpyHostToDevice, s));
    // (a copy from pageable memory has taken the host data when it returns)
    CK(launch_blur(H->I8, H->p, H->q, W.lvl, H->prm.block, H->weights, H->radius, P, s));
    return OPTA_OK;
}

bool size_ready(opta_handle *H, const std::pair<int, int> &key) {
    std::shared_lock<std::shared_mutex> lk(H->sizes_rw);
    return H->sizes.count(key) != 0;
}

// The prepared state of a size (nullptr if not prepared); the caller holds
// sizes_rw (shared or exclusive) or is the only thread using the handle.
SizeState *size_of(opta_handle *H, const std::pair<int, int> &key) {
    auto it = H->sizes.find(key);
    return it == H->sizes.end() ? nullptr : it->second;
}

// Preparation of one size on stream s.  Scratch comes from the handle's
// stream-ordered pool (allocation and release without a device-wide
// synchronisation), so sizes may be prepared by several host threads at once.
opta_status prepare_size(opta_handle *H, int m, int n, cudaStream_t s) {
    auto key = std::make_pair(m, n);
    if (size_ready(H, key)) return OPTA_OK;
    const int p = H->p, q = H->q;
    if (h_limit(p, q, m, n, 1) < 1) return OPTA_ERR_TOO_LARGE;
    SizeState *S = new (std::nothrow) SizeState();
    if (!S) return OPTA_ERR_OOM;
    S->m = m; S->n = n; S->Ly = p - m + 1; S->Lx = q - n + 1;
    const int64_t L = (int64_t)S->Ly * S->Lx;
    const opta_params &prm = H->prm;
    const int block = prm.block;
    const int bp = (p + block - 1) / block, bq = (q + block - 1) / block;
    S->sigma_map.assign((size_t)bp * bq, 0.f);

    PrepScratch W;
    auto scratch = [&](auto **ptr, size_t bytes) {
        return cudaMallocFromPoolAsync(reinterpret_cast<void **>(ptr), bytes, H->pool, s);
    };
    auto cleanup = [&](opta_status st) {
        void *bufs[] = {W.Pcur, W.Pacc, W.fail, W.lvl, W.count, W.IIS, W.IIQ, W.wsumP, W.invP};
        for (void *b : bufs)
            if (b) cudaFreeAsync(b, s);
        if (st != OPTA_OK) {
            if (S->M_owned) {
                H->mem.release(S->wsumM, L);
                H->mem.release(S->invM, L);
            }
            H->mem.release(S->inv_sigma, L);
            H->mem.release(S->wsum, L);
            H->mem.release(S->rho_co, L);
            H->mem.release(S->theta_co, L);
            H->mem.release(S->gco, (size_t)S->Gy * S->Gx);
            H->mem.release(S->c_inv_sigma, (size_t)S->Gy * S->Gx);
            H->mem.release(S->c_efac, (size_t)S->Gy * S->Gx);
            if (S->P_owned) H->mem.release(S->P, (size_t)p * q);
            delete S;
        }
        return st;
    };
#define PTRY(x) do { opta_status s__ = (x); if (s__ != OPTA_OK) return cleanup(s__); } while (0)
#define PCK(x) do { cudaError_t e__ = (x); if (e__ != cudaSuccess) return cleanup(map_err(e__)); } while (0)

    PTRY(H->mem.alloc(&S->inv_sigma, L));
    PTRY(H->mem.alloc(&S->wsum, L));
    PCK(launch_window_stats(H->IIS, H->IIQ, p, q, m, n, S->inv_sigma, nullptr, s, S->wsum));
    PCK(scratch(&W.count, 2 * sizeof(unsigned long long)));
    const bool literal = prm.literal != 0;
    const Members on_image{H->I8, S->wsum, S->inv_sigma};
    const size_t nII = (size_t)(p + 1) * (q + 1);
    // literal mode: window statistics of pivot P into (wsum, inv) via scratch integrals
    auto pivot_stats = [&](const uint8_t *P, int *wsum, float *inv) -> cudaError_t {
        if (!W.IIS) {
            cudaError_t e = scratch(&W.IIS, nII * sizeof(long long));
            if (e == cudaSuccess) e = scratch(&W.IIQ, nII * sizeof(long long));
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_integrals(P, nullptr, p, q, W.IIS, W.IIQ, nullptr, s);
        if (e == cudaSuccess) e = launch_window_stats(W.IIS, W.IIQ, p, q, m, n, inv, nullptr, s, wsum);
        return e;
    };

    // Level 0: unblurred pivots (P = I).
    int h_best = 1;
    long long c_best = 0;
    bool best_is_image = true;
    if (prm.fixed_h > 0) {
        h_best = std::min(prm.fixed_h, h_limit(p, q, m, n, 9));
    } else {
        PTRY(egs(H, S, H->I8, on_image, 1, W.count, &h_best, &c_best, s));
    }
    int level_best = 0;
    if (prm.blur && prm.n_levels > 0 && prm.fixed_h == 0) {
        PCK(scratch(&W.Pcur, (size_t)p * q));
        PCK(scratch(&W.Pacc, (size_t)p * q));
        PCK(scratch(&W.fail, (size_t)bp * bq * sizeof(int)));
        PCK(scratch(&W.lvl, (size_t)bp * bq));
        const float lam = (float)lambda_of(prm.rho_th, prm.rho_max);
        std::vector<uint8_t> cur_level((size_t)bp * bq, 0);   // accepted level index per block
        std::vector<char> frozen((size_t)bp * bq, 0);
        std::vector<int> fail((size_t)bp * bq);
        for (int k = 1; k <= prm.n_levels; ++k) {
            bool all_frozen = true;
            for (char f : frozen) all_frozen = all_frozen && f;
            if (all_frozen) break;
            std::vector<uint8_t> cand(cur_level);
            for (size_t b = 0; b < cand.size(); ++b) if (!frozen[b]) cand[b] = (uint8_t)k;
            PTRY(blur_to(H, W, cand, W.Pcur, s));
            PCK(cudaMemsetAsync(W.fail, 0, (size_t)bp * bq * sizeof(int), s));
            PCK(launch_blur_corr(W.Pcur, H->I8, S->wsum, S->inv_sigma, p, q, m, n, lam, block,
                                 W.fail, nullptr, s));
            PCK(cudaMemcpyAsync(fail.data(), W.fail, fail.size() * sizeof(int),
                                cudaMemcpyDeviceToHost, s));
            PCK(cudaStreamSynchronize(s));
            bool any = false;
            std::vector<char> new_frozen(frozen);
            for (size_t b = 0; b < cand.size(); ++b) {
                if (!frozen[b] && fail[b]) { cand[b] = cur_level[b]; new_frozen[b] = 1; any = true; }
            }
            if (any) PTRY(blur_to(H, W, cand, W.Pcur, s));
            int hk = 0;
            long long ck = 0;
            if (literal) {
                // Section 4.3: the cost is that of searching the blurred image,
                // so EGS measures its own auto-correlation
                if (!W.wsumP) {
                    PCK(scratch(&W.wsumP, (size_t)L * sizeof(int)));
                    PCK(scratch(&W.invP, (size_t)L * sizeof(float)));
                }
                PCK(pivot_stats(W.Pcur, W.wsumP, W.invP));
                PTRY(egs(H, S, W.Pcur, Members{W.Pcur, W.wsumP, W.invP}, h_best, W.count, &hk, &ck,
                         s));
            } else {
                PTRY(egs(H, S, W.Pcur, on_image, h_best, W.count, &hk, &ck, s));
            }
            if ((double)(c_best - ck) > prm.xi * (double)c_best) {
                cur_level = cand;
                frozen = new_frozen;
                h_best = hk;
                c_best = ck;
                level_best = k;
                std::swap(W.Pcur, W.Pacc);
                best_is_image = false;
            } else {
                break;
            }
        }
        for (size_t b = 0; b < cur_level.size(); ++b)
            S->sigma_map[b] = cur_level[b] ? prm.sigma_levels[cur_level[b] - 1] : 0.f;
    }
    S->h = h_best;
    S->level = level_best;
    S->cost = c_best;
    S->Gy = groups_along(S->Ly, S->h);
    S->Gx = groups_along(S->Lx, S->h);
    const int64_t G = (int64_t)S->Gy * S->Gx;
    if (best_is_image) {
        S->P = H->I8;
        S->P_owned = false;
    } else {
        // the accepted pivot is copied into the size state
        PTRY(H->mem.alloc(&S->P, (size_t)p * q));
        S->P_owned = true;
        PCK(cudaMemcpyAsync(S->P, W.Pacc, (size_t)p * q, cudaMemcpyDeviceToDevice, s));
    }
    S->M = H->I8;
    S->wsumM = S->wsum;
    S->invM = S->inv_sigma;
    if (literal) {
        float smax = 0.f;
        for (float v : S->sigma_map) smax = std::max(smax, v);
        S->d = smax > 0.f ? (int)std::ceil(3.0 * (double)smax) : 0;
        if (!best_is_image) {
            // the search runs on the accepted pivot, with its own statistics
            S->M = S->P;
            S->wsumM = nullptr;
            S->invM = nullptr;
            S->M_owned = true;
            PTRY(H->mem.alloc(&S->wsumM, L));
            PTRY(H->mem.alloc(&S->invM, L));
            PCK(pivot_stats(S->P, S->wsumM, S->invM));
        }
    }
    PTRY(H->mem.alloc(&S->rho_co, L));
    PTRY(H->mem.alloc(&S->theta_co, L));
    PTRY(H->mem.alloc(&S->c_inv_sigma, G));
    PTRY(H->mem.alloc(&S->c_efac, G));
    // the accepted configuration's full map and centre statistics (EGS
    // only counted, over its sample)
    PCK(launch_rho_co(S->P, S->M, p, q, m, n, S->h, S->wsumM, S->invM, 0.f, S->rho_co, nullptr,
                      S->c_inv_sigma, S->c_efac, s));
    PCK(launch_theta_co(S->rho_co, L, S->theta_co, s));
    PTRY(H->mem.alloc(&S->gco, G));
    PCK(launch_group_co(S->theta_co, S->Ly, S->Lx, S->h, S->gco, s));
    PCK(cudaStreamSynchronize(s));
    {
        std::unique_lock<std::shared_mutex> lk(H->sizes_rw);
        H->sizes[key] = S;
    }
    return cleanup(OPTA_OK);
#undef PTRY
#undef PCK
}

// Prepare every size of `todo` not prepared yet.  Several sizes run at once,
// one host thread and stream each (their level loops wait on the host
// between kernels, so one size's waits overlap another's kernels); the work
// queued on `s` before the call is awaited first.
opta_status prepare_sizes(opta_handle *H, const std::vector<std::pair<int, int>> &todo,
                          cudaStream_t s) {
    std::vector<std::pair<int, int>> need;
    for (const auto &k : todo)
        if (!size_ready(H, k) && std::find(need.begin(), need.end(), k) == need.end())
            need.push_back(k);
    if (need.empty()) return OPTA_OK;
    if (need.size() == 1) return prepare_size(H, need[0].first, need[0].second, s);
    cudaEvent_t ready = nullptr;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, s));
    std::vector<opta_status> st(need.size(), OPTA_OK);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        cudaSetDevice(H->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
            cudaGetLastError();
            for (size_t i = next++; i < need.size(); i = next++) st[i] = OPTA_ERR_CUDA;
            if (ws) cudaStreamDestroy(ws);
            return;
        }
        for (size_t i = next++; i < need.size(); i = next++)
            st[i] = prepare_size(H, need[i].first, need[i].second, ws);
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    const size_t nth = std::min<size_t>(need.size(), 8);
    std::vector<std::thread> threads;
    try {
        for (size_t t = 0; t < nth; ++t) threads.emplace_back(worker);
    } catch (...) {
        // no threads to be had: the caller's thread takes the rest
    }
    if (threads.empty()) worker();
    for (auto &t : threads) t.join();
    cudaEventDestroy(ready);
    for (opta_status x : st)
        if (x != OPTA_OK) return x;
    return OPTA_OK;
}

template <class T>
opta_status grow(DevMem &mem, T *&p, size_t old_n, size_t new_n) {
    mem.release(p, old_n);
    return mem.alloc(&p, new_n);
}

// Templates per scan-2 launch for L locations and a chunk of `chunk`.
int scan2_batch(size_t L, int chunk) {
    const size_t per = 28 * std::max<size_t>(L, 1);
    size_t tb = kScan2Budget / per;
    tb = std::min<size_t>(tb, (size_t)std::min(chunk, kScan2MaxT));
    return (int)std::max<size_t>(tb, 1);
}

// Make the search scratch large enough for L locations per template and TB
// scan-2 template slots, G groups (times the templates of one chunk: RT =
// chunk * G), chunk template slots of T = m*npad elements each (TS = chunk *
// T), a B buffer of `Bbytes` and N templates.
opta_status ensure_scratch(opta_search_ctx *X, size_t L, size_t TB, size_t RT, size_t T, size_t TS,
                           size_t Bbytes, size_t N) {
    const size_t G = RT;
    if (L > X->capL || TB > X->capS2) {
        const size_t nL = std::max(L, X->capL), nS = std::max(TB, X->capS2);
        const size_t oldn = X->capL * X->capS2, newn = nL * nS;
        TRY(grow(X->mem, X->surv, oldn, newn));
        TRY(grow(X->mem, X->surv_rho, oldn, newn));
        TRY(grow(X->mem, X->surv_eps, oldn, newn));
        TRY(grow(X->mem, X->surv_ub, oldn, newn));
        TRY(grow(X->mem, X->cand, oldn, newn));
        TRY(grow(X->mem, X->cand_rho, oldn, newn));
        X->capL = nL;
        X->capS2 = nS;
    }
    if (G > X->capG) {
        TRY(grow(X->mem, X->rho_tc, X->capG, G));
        X->capG = G;
    }
    if (!X->topk_v) {
        TRY(X->mem.alloc(&X->topk_v, (size_t)kChunk * 256 * kTopkMax));
        TRY(X->mem.alloc(&X->topk_i, (size_t)kChunk * 256 * kTopkMax));
        TRY(X->mem.alloc(&X->cand_topk, (size_t)kChunk * kTopkMax));
        TRY(X->mem.alloc(&X->cand_rho_topk, (size_t)kChunk * kTopkMax));
        TRY(X->mem.alloc(&X->bucket_cnt, (size_t)kScan2MaxT * kUbBuckets));
        TRY(X->mem.alloc(&X->bucket_cur, (size_t)kScan2MaxT * kUbBuckets));
        TRY(X->mem.alloc(&X->ucnt, (size_t)kScan2MaxT));
    }
    if (T > X->capT) {
        TRY(grow(X->mem, X->tstage, X->capT, T));
        X->capT = T;
    }
    if (TS > X->capTS) {
        TRY(grow(X->mem, X->tf, X->capTS, TS));
        TRY(grow(X->mem, X->td, X->capTS, TS));
        X->capTS = TS;
    }
    if (Bbytes > X->capB) {
        uint8_t *b = static_cast<uint8_t *>(X->Bmma);
        TRY(grow(X->mem, b, X->capB, Bbytes));
        X->Bmma = b;
        X->capB = Bbytes;
    }
    if (!X->dev_err) {
        TRY(X->mem.alloc(&X->dev_err, 1));
        CK(cudaMemset(X->dev_err, 0, sizeof(int)));
    }
    if (N > X->capN) {
        TRY(grow(X->mem, X->states, X->capN, N));
        TRY(grow(X->mem, X->tin, X->capN, N));
        if (X->tin_host) cudaFreeHost(X->tin_host);
        if (X->states_host) cudaFreeHost(X->states_host);
        X->tin_host = nullptr;
        X->states_host = nullptr;
        if (cudaMallocHost(&X->tin_host, N * sizeof(TmplIn)) != cudaSuccess ||
            cudaMallocHost(&X->states_host, N * sizeof(TmplState)) != cudaSuccess) {
            cudaGetLastError();
            return OPTA_ERR_OOM;
        }
        X->capN = N;
    }
    if (!X->err_host) {
        if (cudaMallocHost(&X->err_host, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return OPTA_ERR_OOM;
        }
    }
    return OPTA_OK;
}

bool use_mma(const opta_handle *H) { return H->prm.precision == 1; }

// Whether scan 2 may evaluate an m x n template densely on the tensor cores:
// the exact search of I (not the literal mode's blurred image), sizes the
// tensor-core map supports, and not switched off.
bool dense_usable(const opta_handle *H, int m, int n) {
    return H->prm.dense != 0 && !H->prm.literal && H->Ipad && brute_mma_supported(m, n);
}

// Survivors left after the cut, as a fraction of the locations, above which a
// template takes the dense map.  The tensor-core map costs about the same per
// location at every template size (about 11-19 G locations/s on 4096^2) and a
// gathered survivor about 2 m n flops at 2-3.5 TFLOP/s, which would break
// even near 80 / (m n) of the locations; but the sweep's running lower bound
// skips most survivors of a template with a high maximum (at rho_th = 0.9 on
// the 4096^2 batch it evaluated a fifth of them), so the cut sits higher:
// dense_cut / (m n) (default 100), at most half, counted after a first
// sweep over the head of the bound-ordered list (about a quarter of the dense
// map's cost: 20 L / (m n) survivors), which has usually raised the running
// lower bound to the maximum.  dense = 2: every template with a survivor left.
float dense_frac(const opta_handle *H, int m, int n) {
    if (H->prm.dense == 2) return -1.f;
    const float c = H->prm.dense_cut > 0.f ? H->prm.dense_cut : 100.f;
    return std::min(0.5f, c / ((float)m * (float)n));
}

// Scan-1 error factor A of an m x n size (e = A * ||P - 128|| / sigma_hat +
// kScan1EpsB): the largest over the kernels that compute its centres.
float scan1_eps_factor(const opta_handle *H, int m, int n) {
    const int npad = (n + 7) & ~7, Kp = (n + 15) & ~15;
    if (use_mma(H)) return std::max(scan1_epsA_f16(m, n, Kp), scan1_epsA_fp32(centre_column_kacc(m, n)));
    return scan1_epsA_fp32(centre_rho_kacc(m, npad));
}

// Scratch needed by a batch of templates (sizes already prepared).
// Scratch capacities a batch of templates needs: L locations per template,
// TB scan-2 slots, RT = chunk x G centre values, T / TS template elements of
// a chunk, B bytes of tensor-core operands and N template states.  A size
// not prepared yet is planned at its largest (h = 1: G = L).
struct ScratchPlan {
    size_t L = 0, TB = 1, RT = 0, T = 0, TS = 0, B = 0, N = 0;
};

ScratchPlan plan_scratch(opta_handle *H, const opta_template *t, int n_t) {
    ScratchPlan c;
    std::map<std::pair<int, int>, int> count;
    for (int i = 0; i < n_t; ++i) count[std::make_pair(t[i].rows, t[i].cols)]++;
    for (auto &kv : count) {
        SizeState *S = size_of(H, kv.first);
        const int m = kv.first.first, n = kv.first.second, Kp = (n + 15) & ~15;
        const size_t chunk = (size_t)std::min(kv.second, kChunk);
        const size_t L = (size_t)(H->p - m + 1) * (H->q - n + 1);
        const size_t G = S ? (size_t)S->Gy * S->Gx : L;
        c.L = std::max(c.L, L);
        c.TB = std::max(c.TB, (size_t)scan2_batch(L, (int)chunk));
        c.RT = std::max(c.RT, chunk * G);
        c.T = std::max(c.T, chunk * (size_t)m * n);
        c.TS = std::max(c.TS, chunk * tmpl_slot_floats(m, n));
        const size_t N = ((2 * chunk + 15) / 16) * 16;
        if (use_mma(H)) c.B = std::max(c.B, corr_mma_bbytes(m, Kp, (int)N, S ? S->h : m));
        // the template tiles of a scan-2 launch that may take the dense map
        if (dense_usable(H, m, n))
            c.B = std::max(c.B, (size_t)scan2_batch(L, (int)chunk) * brute_tmpl_bytes(m, n));
    }
    c.N = (size_t)n_t;
    return c;
}

opta_status size_scratch(opta_handle *H, opta_search_ctx *X, const opta_template *t, int n_t) {
    const ScratchPlan c = plan_scratch(H, t, n_t);
    return ensure_scratch(X, c.L, c.TB, c.RT, c.T, c.TS, c.B, c.N);
}

// Template statistics and scan 1 (Section 6: rho(t, pivot) at every centre)
// of templates t[0..n) -- all of one size -- into the chunk slots; states
// st[0..n).  No host synchronisation.
opta_status enqueue_scan1(opta_handle *H, opta_search_ctx *X, const opta_template *const *t, int n, TmplState *st,
                          cudaStream_t s) {
    const int m = t[0]->rows, nn = t[0]->cols, npad = (nn + 7) & ~7, Kp = (nn + 15) & ~15;
    SizeState *S = size_of(H, std::make_pair(m, nn));
    const int64_t G = (int64_t)S->Gy * S->Gx;
    const size_t tsz = tmpl_slot_floats(m, nn), dsz = (size_t)m * nn;
    // template statistics (Eq. rho1's mu_t, sigma_t) of the whole chunk in one launch
    const ptrdiff_t slot0 = st - X->states;
    TmplIn *tin = X->tin_host + slot0;
    for (int k = 0; k < n; ++k) {
        if (t[k]->on_device) {
            tin[k].data = t[k]->data;
            tin[k].ld = t[k]->stride_elems;
        } else {
            float *slot = X->tstage + (size_t)k * m * nn;
            CK(cudaMemcpy2DAsync(slot, (size_t)nn * sizeof(float), t[k]->data,
                                 (size_t)t[k]->stride_elems * sizeof(float),
                                 (size_t)nn * sizeof(float), m, cudaMemcpyHostToDevice, s));
            tin[k].data = slot;
            tin[k].ld = nn;
        }
    }
    CK(cudaMemcpyAsync(X->tin + slot0, tin, n * sizeof(TmplIn), cudaMemcpyHostToDevice, s));
    CK(launch_tmpl_prep_batch(X->tin + slot0, n, m, nn, npad, X->tf, tsz, X->td, dsz, st,
                              H->prm.topk, s));
    // scan 1: rho(t, pivot) at every centre
    if (use_mma(H)) {
        const int N = ((2 * n + 15) / 16) * 16;
        CK(cudaMemsetAsync(X->Bmma, 0, (size_t)(m + 1) * Kp * N * 2, s));   // row m stays zero
        CK(launch_tmpl_split(X->tf, tsz, n, m, nn, npad, Kp, N, st, X->Bmma, s));
        int Gx_u = S->Gx;
        CK(launch_corr_mma(S->P, H->p, H->q, X->Bmma, m, nn, Kp, N, S->h, S->Ly, S->Lx, n,
                           S->c_inv_sigma, st, X->rho_tc, G, X->dev_err, &Gx_u, s));
        for (int gx = Gx_u; gx < S->Gx; ++gx)
            CK(launch_centre_column(S->P, H->q, X->tf, m, nn, npad, tsz, S->h, S->Ly, S->Lx, gx, n,
                                    S->c_inv_sigma, st, X->rho_tc, G, s));
    } else {
        for (int k = 0; k < n; ++k)
            CK(launch_centre_rho(S->P, H->p, H->q, X->tf + k * tsz, m, nn, npad, S->h, S->Ly,
                                 S->Lx, S->c_inv_sigma, st + k, X->rho_tc + k * G, 0, s));
    }
    // threshold (Section 6): top-k centres, their exact rho, the members of
    // their groups -- batched over the chunk
    CK(launch_topk(X->rho_tc, G, S->Gy, S->Gx, S->h, S->Ly, S->Lx, H->prm.topk, n, st, X->topk_v,
                   X->topk_i, X->cand_topk, s));
    CK(launch_refine64_topk(S->M, H->q, S->Lx, X->td, dsz, m, nn, n, st, X->cand_topk,
                            X->cand_rho_topk, s, X->tf, tsz, npad));
    CK(launch_group_members(S->M, H->q, S->Ly, S->Lx, S->h, S->wsumM, X->tf, tsz, m, nn,
                            npad, S->invM, n, st, X->cand_topk, H->prm.topk, s));
    CK(launch_threshold(st, X->cand_rho_topk, n, s));
    return OPTA_OK;
}

// Scan-2 launch descriptor of templates k0 .. k0 + T of a chunk (states st)
// of size S, over the context's scratch; no dense map (dense_frac 0).
Scan2Batch scan2_batch_of(opta_handle *H, opta_search_ctx *X, SizeState *S, TmplState *st, int k0,
                          int T) {
    const int m = S->m, nn = S->n;
    const int64_t L = (int64_t)S->Ly * S->Lx;
    const int64_t G = (int64_t)S->Gy * S->Gx;
    const size_t tsz = tmpl_slot_floats(m, nn);
    Scan2Batch B;
    B.T = T;
    B.st = st + k0;
    B.rho_tc = X->rho_tc + k0 * G;
    B.tc_stride = G;
    B.c_efac = S->c_efac;
    B.epsA = scan1_eps_factor(H, m, nn);
    B.tf = X->tf + k0 * tsz;
    B.tsz = tsz;
    B.surv = X->surv;
    B.surv_ub = X->surv_ub;
    B.surv_rho = X->surv_rho;
    B.surv_eps = X->surv_eps;
    B.scap = (int64_t)X->capL;
    B.cand = X->cand;
    B.ccap = (int64_t)X->capL;
    B.ucnt = X->ucnt;
    B.bucket_cnt = X->bucket_cnt;
    B.bucket_cur = X->bucket_cur;
    B.L = L;
    B.dense_frac = 0.f;
    // the first sweep: about a quarter of the dense map's cost (none when
    // every template with a survivor is to take the dense map)
    B.first_budget = H->prm.dense == 2
                         ? 0
                         : std::max<int64_t>(1024, (int64_t)(20.0 * (double)L / ((double)m * nn)));
    B.phase = 0;
    // survivors of byte templates on the image itself: exact integer sums
    // over the 32-byte-aligned copy
    B.Ipad = S->M == H->I8 ? H->Ipad : nullptr;
    B.qs = H->qs;
    B.lane_min_u8 = survivor_lane_min(m, nn, true);
    B.lane_min_f32 = survivor_lane_min(m, nn, false);
    B.span = nullptr;
    B.group_order = (long long)m * nn >= kGroupOrderMN;
    return B;
}

// Survivor-form tuner.  The lane form (a lane per survivor) has a long
// serial chain per lane and wins once there are enough survivors to fill
// the GPU; the warp form (a warp per survivor) wins on short lists.  The
// first search of a size on a device (outside graph capture) times both on
// synthetic lists of c1 and c2 locations (clusters of 5 x 5, like the
// members of the groups the elimination test keeps) with the batch's first
// template, fits time = a + b count per form and records the count from
// which the lane form is faster, for templates of bytes (when the template
// is one) and for the FP32 path.
opta_status tune_survivor_forms(opta_handle *H, opta_search_ctx *X, SizeState *S, TmplState *st, int k0,
                                cudaStream_t s) {
    const int m = S->m, nn = S->n, npad = (nn + 7) & ~7;
    bool t8 = false, t32 = false;
    survivor_lane_min(m, nn, true, &t8);
    survivor_lane_min(m, nn, false, &t32);
    if (t8 && t32) return OPTA_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) { cudaGetLastError(); return OPTA_OK; }
    if (cap != cudaStreamCaptureStatusNone) return OPTA_OK;
    const int64_t L = (int64_t)S->Ly * S->Lx;
    const int c2 = (int)std::min<int64_t>(L, 32768), c1 = std::min(c2 / 16, 2048);
    if (c1 < 256) return OPTA_OK;   // small maps: the default rule
    if (!X->tune_st) TRY(X->mem.alloc(&X->tune_st, 1));
    if (!X->tune_span) TRY(X->mem.alloc(&X->tune_span, 2));
    // the synthetic list: c2 / 25 cluster centres, seeded
    std::vector<int> idx;
    idx.reserve((size_t)c2);
    uint64_t r = 0x9e3779b97f4a7c15ull;
    auto next = [&r]() { r ^= r << 13; r ^= r >> 7; r ^= r << 17; return r; };
    while ((int)idx.size() < c2) {
        const int cy = 2 + (int)(next() % (uint64_t)std::max(1, S->Ly - 4));
        const int cx = 2 + (int)(next() % (uint64_t)std::max(1, S->Lx - 4));
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                const int y = std::min(std::max(cy + dy, 0), S->Ly - 1);
                const int x = std::min(std::max(cx + dx, 0), S->Lx - 1);
                if ((int)idx.size() < c2) idx.push_back(y * S->Lx + x);
            }
    }
    CK(cudaMemcpyAsync(X->surv, idx.data(), (size_t)c2 * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(X->tune_st, st + k0, sizeof(TmplState), cudaMemcpyDeviceToDevice, s));
    TmplState hs;
    CK(cudaMemcpyAsync(&hs, st + k0, sizeof(TmplState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs.flat) return OPTA_OK;
    Scan2Batch B = scan2_batch_of(H, X, S, st, k0, 1);
    B.st = X->tune_st;
    B.span = X->tune_span;
    // a sweep's time from its own blocks' clocks (first start to last end),
    // free of launch gaps and of any profiler around the launches
    auto timed = [&](int count, int form, float *ms) -> cudaError_t {
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            const unsigned long long init[2] = {~0ull, 0ull};
            unsigned long long span[2] = {0ull, 0ull};
            cudaError_t e = cudaMemcpyAsync(X->tune_span, init, sizeof(init), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = launch_survivor_eval(B, S->M, H->p, H->q, S->Lx, S->wsumM, m, nn, npad, S->invM, count,
                                         form, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(span, X->tune_span, sizeof(span), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            if (span[1] > span[0]) best = std::min(best, (float)((double)(span[1] - span[0]) * 1e-6));
        }
        *ms = best < 1e30f ? best : 0.f;
        return cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    for (int type = 1; type >= 0 && e == cudaSuccess; --type) {
        const bool u8 = type == 1;
        if ((u8 && (t8 || !hs.u8 || !B.Ipad)) || (!u8 && t32)) continue;
        const int flag = u8 ? 1 : 0;   // the FP32 path: the same template as real values
        e = cudaMemcpyAsync(&X->tune_st->u8, &flag, sizeof(int), cudaMemcpyHostToDevice, s);
        float t[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
        for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
            float w = 0.f;
            e = timed(c1, form, &w);   // first launches of the kernels
            if (e == cudaSuccess) e = timed(c1, form, &t[form][0]);
            if (e == cudaSuccess) e = timed(c2, form, &t[form][1]);
        }
        if (e != cudaSuccess) break;
        const double bl = (t[0][1] - t[0][0]) / (double)(c2 - c1), al = t[0][0] - bl * c1;
        const double bw = (t[1][1] - t[1][0]) / (double)(c2 - c1), aw = t[1][0] - bw * c1;
        int lane_min;
        if (bw > bl) {
            const double c = (al - aw) / (bw - bl);
            lane_min = c <= 0.0 ? 0 : (int)std::min<double>(std::ceil(c), (double)kLaneNever - 1);
        } else {
            lane_min = al <= aw ? 0 : kLaneNever;
        }
        set_survivor_lane_min(m, nn, u8, lane_min);
    }
    if (e != cudaSuccess) { cudaGetLastError(); return map_err(e); }
    return OPTA_OK;
}

// Scan 2 (Eq. SEC), survivors and FP64 argmax of the chunk whose scan 1 and
// threshold are done, in batches of scan2_batch() templates per launch.
opta_status enqueue_scan2(opta_handle *H, opta_search_ctx *X, const opta_template *const *t, int n, TmplState *st,
                          float *ub_map, uint8_t *surv_map, cudaStream_t s) {
    const int m = t[0]->rows, nn = t[0]->cols, npad = (nn + 7) & ~7;
    SizeState *S = size_of(H, std::make_pair(m, nn));
    const int64_t L = (int64_t)S->Ly * S->Lx;
    const size_t tsz = tmpl_slot_floats(m, nn), dsz = (size_t)m * nn;
    const int TB = std::min(scan2_batch((size_t)L, n), (int)X->capS2);
    const int64_t scap = (int64_t)X->capL;
    const bool dense = dense_usable(H, m, nn) && S->M == H->I8;
    if (TB < 1 || ((ub_map || surv_map) && n != 1)) return OPTA_ERR_INVALID_ARG;
    for (int k0 = 0; k0 < n; k0 += TB) {
        const int T = std::min(TB, n - k0);
        if (k0 == 0 && !(ub_map || surv_map)) TRY(tune_survivor_forms(H, X, S, st, k0, s));
        Scan2Batch B = scan2_batch_of(H, X, S, st, k0, T);
        B.dense_frac = dense ? dense_frac(H, m, nn) : 0.f;
        CK(launch_bound_compact(B, S->theta_co, S->gco, S->Ly, S->Lx, S->h, ub_map, surv_map, s));
        // the survivor cut marks the templates with many survivors left as
        // dense; the sweep skips them
        CK(launch_survivors(B, S->M, H->p, H->q, S->Lx, S->wsumM, m, nn, npad, S->invM, s));
        if (dense) {
            // their rho at every location on the tensor cores (templates not
            // marked are skipped on the device), into their rho slots
            CK(launch_brute_tmpl(X->tf + k0 * tsz, tsz, T, m, nn, npad, X->Bmma, st + k0, 1, s));
            CK(launch_brute_mma(H->Ipad, H->qs, H->p, H->q, X->Bmma, m, nn, S->invM, nullptr, S->wsumM,
                                st + k0, X->surv_rho, scap, T, 1, X->dev_err, s));
            CK(launch_dense_candidates(B, S->wsumM, S->invM, m, nn, s));
        }
        CK(launch_surv_candidates(B, s));
        CK(launch_refine64(S->M, H->q, S->Lx, X->td + k0 * dsz, dsz, m, nn, T, st + k0, X->cand,
                           X->cand_rho, scap, s, X->tf + k0 * tsz, tsz, npad));
        CK(launch_final_argmax(T, st + k0, X->cand, X->cand_rho, scap, X->cand_topk + k0 * kTopkMax,
                               X->cand_rho_topk + k0 * kTopkMax, s));
        if (H->prm.literal) {
            // Section 4.3: t matched with I in FP64 over the (2d+1)^2
            // neighbourhood of the maximum found on the blurred image
            CK(launch_rematch_window(T, st + k0, S->Ly, S->Lx, S->d, X->cand, scap, s));
            CK(launch_refine64(H->I8, H->q, S->Lx, X->td + k0 * dsz, dsz, m, nn, T, st + k0,
                               X->cand, X->cand_rho, scap, s, X->tf + k0 * tsz, tsz, npad));
            CK(launch_final_argmax(T, st + k0, X->cand, X->cand_rho, scap, nullptr, nullptr, s));
        }
    }
    return OPTA_OK;
}

// Templates grouped by size (stable): order[k] is the input index of the
// template whose state is states[k]; groups holds each size's [begin, end)
// of states.
void group_by_size(const opta_template *t, int n_t, std::vector<int> &order,
                   std::vector<std::pair<int, int>> &groups) {
    order.resize(n_t);
    for (int i = 0; i < n_t; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return std::make_pair(t[a].rows, t[a].cols) < std::make_pair(t[b].rows, t[b].cols);
    });
    groups.clear();
    for (int i = 0; i < n_t;) {
        int j = i;
        while (j < n_t && t[order[j]].rows == t[order[i]].rows && t[order[j]].cols == t[order[i]].cols) ++j;
        groups.emplace_back(i, j);
        i = j;
    }
}

// Scan 1 and scan 2 of the states [b, e) (templates of one size), chunk by chunk.
opta_status enqueue_group(opta_handle *H, opta_search_ctx *X, const opta_template *t,
                          const std::vector<int> &order, int b, int e, cudaStream_t s) {
    std::vector<const opta_template *> chunk;
    for (int i = b; i < e;) {
        const int j = std::min(e, i + kChunk);
        chunk.clear();
        for (int k = i; k < j; ++k) chunk.push_back(&t[order[k]]);
        TRY(enqueue_scan1(H, X, chunk.data(), (int)chunk.size(), X->states + i, s));
        TRY(enqueue_scan2(H, X, chunk.data(), (int)chunk.size(), X->states + i, nullptr, nullptr, s));
        i = j;
    }
    return OPTA_OK;
}

// Group templates by size (stable) and enqueue them chunk by chunk; order[i]
// is the input index of the template whose state is states[i].
opta_status enqueue_all(opta_handle *H, opta_search_ctx *X, const opta_template *t, int n_t, std::vector<int> &order,
                        cudaStream_t s) {
    std::vector<std::pair<int, int>> groups;
    group_by_size(t, n_t, order, groups);
    for (const auto &g : groups) TRY(enqueue_group(H, X, t, order, g.first, g.second, s));
    return OPTA_OK;
}

void fill_result(const TmplState &st, const SizeState *S, int Lx, int64_t L, int h,
                 int64_t n_centres, opta_result *r) {
    std::memset(r, 0, sizeof(*r));
    r->n_locations = L;
    r->group_h = h;
    r->n_centres = n_centres;
    r->n_survivors = st.n_surv;
    r->n_candidates = st.n_cand + st.n_cand_search;
    r->n_evaluated = st.n_eval;
    r->rho_threshold = st.thr;
    if (st.flat) {
        r->y = 0; r->x = 0; r->rho = 0.0;
        r->status = OPTA_ERR_FLAT_TEMPLATE;
        return;
    }
    r->y = st.best_idx / Lx;
    r->x = st.best_idx % Lx;
    r->rho = st.best_rho;
    const int hat = st.hat_idx >= 0 ? st.hat_idx : st.best_idx;
    r->y_hat = hat / Lx;
    r->x_hat = hat % Lx;
    r->rematch_d = st.hat_idx >= 0 ? S->d : 0;
    r->status = st.overflow ? OPTA_ERR_CUDA : OPTA_OK;
}

}  // namespace

namespace opta {

opta_status exhaustive_run(const uint8_t *I8, int p, int q, const float *tdev, int64_t tld, int m,
                           int n, const ExhaustiveBufs &b, opta_result *best, cudaStream_t s) {
    const int npad = (n + 7) & ~7;
    const int Lx = q - n + 1;
    const int64_t L = (int64_t)(p - m + 1) * Lx;
    cudaError_t e;
#define XCK(x) do { if ((e = (x)) != cudaSuccess) return map_err(e); } while (0)
    XCK(launch_integrals(I8, nullptr, p, q, b.IIS, b.IIQ, nullptr, s));
    XCK(launch_window_stats(b.IIS, b.IIQ, p, q, m, n, b.inv, b.ef, s, b.wsum));
    XCK(launch_tmpl_prep(tdev, tld, m, n, npad, b.tf, b.td, b.st, 0, s));
    const bool tc = b.Ipad && b.Bt && b.err && b.wsum && brute_mma_supported(m, n);
    float epsA;
    if (tc) {
        // the map on the tensor cores (bf16 hi/lo split of t', FP32 accumulation)
        const int qs = (q + 15) & ~15;
        XCK(cudaMemsetAsync(b.err, 0, sizeof(int), s));
        XCK(launch_pad_rows(I8, p, q, b.Ipad, qs, s));
        XCK(launch_brute_tmpl(b.tf, 0, 1, m, n, npad, b.Bt, b.st, 0, s));
        XCK(launch_brute_mma(b.Ipad, qs, p, q, b.Bt, m, n, b.inv, b.ef, b.wsum, b.st, b.map, 0, 1, 0,
                             b.err, s));
        epsA = brute_mma_epsA(m, n);
    } else {
        XCK(launch_zncc_map(I8, p, q, b.tf, m, n, npad, b.inv, b.ef, b.st, b.map, s));
        epsA = zncc_map_epsA(m, n);
    }
    XCK(launch_map_candidates(b.map, b.ef, L, epsA, b.st, b.cand, (int)L, s));
    XCK(launch_refine64(I8, q, Lx, b.td, (size_t)m * n, m, n, 1, b.st, b.cand, b.crho, L, s));
    XCK(launch_final_argmax(1, b.st, b.cand, b.crho, L, nullptr, nullptr, s));
    TmplState hs;
    int herr = 0;
    XCK(cudaMemcpyAsync(&hs, b.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (tc) XCK(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    XCK(cudaStreamSynchronize(s));
#undef XCK
    fill_result(hs, nullptr, Lx, L, 1, L, best);
    best->n_survivors = L;
    best->n_evaluated = L;
    if (herr) best->status = OPTA_ERR_TIMEOUT;
    return (opta_status)best->status;
}

}  // namespace opta

namespace {

struct BusyGuard {
    opta_handle *h;
    explicit BusyGuard(opta_handle *hh) : h(hh) { h->busy = true; }
    ~BusyGuard() { h->busy = false; }
};

// Releases a context claimed with compare_exchange on its busy flag.
struct CtxGuard {
    opta_search_ctx *x;
    explicit CtxGuard(opta_search_ctx *xx) : x(xx) {}
    ~CtxGuard() { x->busy.store(false); }
};

void free_ctx(opta_search_ctx *X) {
    void *ptrs[] = {X->rho_tc, X->surv, X->surv_rho, X->surv_eps, X->surv_ub, X->ucnt,
                    X->bucket_cnt, X->bucket_cur, X->Bmma, X->dev_err, X->cand_topk,
                    X->cand_rho_topk, X->tin, X->cand, X->cand_rho, X->topk_v, X->topk_i,
                    X->tf, X->tstage, X->td, X->states, X->tune_st, X->tune_span};
    for (void *p : ptrs) if (p) cudaFree(p);
    if (X->tin_host) cudaFreeHost(X->tin_host);
    if (X->states_host) cudaFreeHost(X->states_host);
    if (X->err_host) cudaFreeHost(X->err_host);
    delete X;
}

}  // namespace

// A captured batched search (optA_graph_*): its own context, the templates'
// device buffers and the instantiated graph.
struct opta_graph {
    opta_handle *h = nullptr;
    opta_search_ctx *X = nullptr;
    int n_t = 0;
    float *tbuf = nullptr;
    std::vector<opta_template> desc;
    std::vector<int> order;
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t nodes = 0;
};

namespace {

void destroy_graph(opta_graph *G) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    if (G->s) cudaStreamDestroy(G->s);
    if (G->tbuf) cudaFree(G->tbuf);
    if (G->X) free_ctx(G->X);
    delete G;
}

opta_status default_ctx(opta_handle *H) {
    if (H->dctx) return OPTA_OK;
    opta_search_ctx *X = new (std::nothrow) opta_search_ctx();
    if (!X) return OPTA_ERR_OOM;
    X->device = H->device;
    H->dctx = X;
    return OPTA_OK;
}

// One search through context X (claimed by the caller): missing sizes are
// prepared first (one preparation at a time per handle), then the prepared
// sizes are read under a shared lock while the search's kernels run on s.
// The search of templates t whose sizes `need` are not prepared yet: the
// scratch is sized first (those sizes at their largest), the missing sizes
// are prepared on worker threads, one stream each, while the search of every
// size already prepared is enqueued on s, and each other size's search is
// enqueued as soon as its preparation has finished -- so the search kernels
// of ready sizes run beside the preparation of the others.  The caller holds
// prep_mu; order receives the state order (see group_by_size).
opta_status search_overlapped(opta_handle *H, opta_search_ctx *X, const opta_template *t, int n_t,
                              const std::vector<std::pair<int, int>> &need, std::vector<int> &order,
                              cudaStream_t s) {
    {
        std::shared_lock<std::shared_mutex> rl(H->sizes_rw);
        TRY(size_scratch(H, X, t, n_t));
    }
    std::vector<std::pair<int, int>> groups;
    group_by_size(t, n_t, order, groups);
    cudaEvent_t ready = nullptr;
    CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CK(cudaEventRecord(ready, s));
    std::mutex mu;
    std::condition_variable cv;
    size_t finished = 0;
    std::vector<opta_status> st(need.size(), OPTA_OK);
    std::atomic<size_t> next{0};
    auto report = [&]() {
        std::lock_guard<std::mutex> lk(mu);
        ++finished;
        cv.notify_one();
    };
    auto worker = [&]() {
        cudaSetDevice(H->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(ws, ready, 0) != cudaSuccess) {
            cudaGetLastError();
            for (size_t i = next++; i < need.size(); i = next++) {
                st[i] = OPTA_ERR_CUDA;
                report();
            }
            if (ws) cudaStreamDestroy(ws);
            return;
        }
        for (size_t i = next++; i < need.size(); i = next++) {
            st[i] = prepare_size(H, need[i].first, need[i].second, ws);
            report();
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    const size_t nth = std::min<size_t>(need.size(), 8);
    std::vector<std::thread> threads;
    try {
        for (size_t k = 0; k < nth; ++k) threads.emplace_back(worker);
    } catch (...) {
        // no threads to be had: the sizes are prepared below, one by one
    }
    std::vector<char> queued(groups.size(), 0);
    opta_status first = OPTA_OK;
    // enqueue the search of every group whose size is prepared (once each)
    auto enqueue_ready = [&]() {
        std::shared_lock<std::shared_mutex> rl(H->sizes_rw);
        for (size_t g = 0; g < groups.size(); ++g) {
            if (queued[g]) continue;
            const opta_template &t0 = t[order[groups[g].first]];
            if (!size_of(H, std::make_pair(t0.rows, t0.cols))) continue;
            queued[g] = 1;
            if (first == OPTA_OK) first = enqueue_group(H, X, t, order, groups[g].first, groups[g].second, s);
        }
    };
    enqueue_ready();
    if (threads.empty()) {
        worker();
        enqueue_ready();
    } else {
        for (size_t seen = 0; seen < need.size();) {
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return finished > seen; });
                seen = finished;
            }
            enqueue_ready();
        }
        for (auto &th : threads) th.join();
    }
    cudaEventDestroy(ready);
    for (opta_status x : st)
        if (x != OPTA_OK) return x;
    return first;
}

opta_status search_in(opta_handle *H, opta_search_ctx *X, const opta_template *t, int32_t n_t,
                      opta_result *out, cudaStream_t s) {
    std::vector<std::pair<int, int>> todo;
    for (int i = 0; i < n_t; ++i) {
        if (!valid_template(&t[i], H->p, H->q)) return OPTA_ERR_INVALID_ARG;
        todo.emplace_back(t[i].rows, t[i].cols);
    }
    std::vector<int> order;
    {
        std::lock_guard<std::mutex> pl(H->prep_mu);
        if (n_t == 0) return prepare_sizes(H, todo, s);
        std::vector<std::pair<int, int>> need;
        for (const auto &k : todo)
            if (!size_ready(H, k) && std::find(need.begin(), need.end(), k) == need.end()) need.push_back(k);
        if (!need.empty()) {
            // sizes prepared here overlap the search of the others
            TRY(search_overlapped(H, X, t, n_t, need, order, s));
        } else {
            std::shared_lock<std::shared_mutex> rl0(H->sizes_rw);
            TRY(size_scratch(H, X, t, n_t));
            TRY(enqueue_all(H, X, t, n_t, order, s));
        }
    }
    std::shared_lock<std::shared_mutex> rl(H->sizes_rw);
    CK(cudaMemcpyAsync(X->states_host, X->states, sizeof(TmplState) * n_t, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(X->err_host, X->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const TmplState *hs = X->states_host;
    const int herr = *X->err_host;
    opta_status first = OPTA_OK;
    for (int k = 0; k < n_t; ++k) {
        const int i = order[k];
        SizeState *S = size_of(H, std::make_pair(t[i].rows, t[i].cols));
        fill_result(hs[k], S, S->Lx, (int64_t)S->Ly * S->Lx, S->h, (int64_t)S->Gy * S->Gx, &out[i]);
        if (herr) out[i].status = OPTA_ERR_TIMEOUT;
    }
    for (int i = 0; i < n_t; ++i)
        if (first == OPTA_OK && out[i].status != OPTA_OK) first = (opta_status)out[i].status;
    if (herr) CK(cudaMemsetAsync(X->dev_err, 0, sizeof(int), s));
    return first;
}

opta_status setup_tables(opta_handle *H) {
    std::vector<float> w;
    std::vector<int> rad;
    gauss_table(H->prm, w, rad);
    TRY(H->mem.alloc(&H->weights, w.size()));
    TRY(H->mem.alloc(&H->radius, rad.size()));
    CK(cudaMemcpy(H->weights, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(H->radius, rad.data(), rad.size() * sizeof(int), cudaMemcpyHostToDevice));
    return OPTA_OK;
}

}  // namespace

// ===========================================================================
// Public ABI
// ===========================================================================
extern "C" {

void opta_params_default(opta_params *prm) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->rho_th = 0.80;
    prm->rho_max = 0.95;
    prm->xi = 0.005;
    prm->block = 64;
    prm->n_levels = 4;
    prm->sigma_levels[0] = 0.5f;
    prm->sigma_levels[1] = 1.0f;
    prm->sigma_levels[2] = 2.0f;
    prm->sigma_levels[3] = 3.0f;
    prm->h_max = 9;
    prm->fixed_h = 0;
    prm->blur = 1;
    prm->topk = 8;
    prm->precision = 1;
    prm->egs_sample = 8;
    prm->dense = 1;
}

const char *opta_status_str(opta_status s) {
    switch (s) {
        case OPTA_OK: return "ok";
        case OPTA_ERR_INVALID_ARG: return "invalid argument";
        case OPTA_ERR_FLAT_TEMPLATE: return "flat template (sigma_t == 0)";
        case OPTA_ERR_OOM: return "out of device memory";
        case OPTA_ERR_CUDA: return "CUDA error";
        case OPTA_ERR_TIMEOUT: return "timeout";
        case OPTA_ERR_BUSY: return "handle busy";
        case OPTA_ERR_UNSUPPORTED: return "unsupported input";
        case OPTA_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the no-alloc entry point";
    }
    return "unknown status";
}

opta_status optA_destroy(opta_handle *h) {
    if (!h) return OPTA_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    for (auto &kv : h->sizes) {
        SizeState *S = kv.second;
        cudaFree(S->inv_sigma); cudaFree(S->wsum); cudaFree(S->rho_co); cudaFree(S->theta_co);
        cudaFree(S->gco);
        cudaFree(S->c_inv_sigma); cudaFree(S->c_efac);
        if (S->P_owned) cudaFree(S->P);
        if (S->M_owned) { cudaFree(S->wsumM); cudaFree(S->invM); }
        delete S;
    }
    void *ptrs[] = {h->I8, h->Ipad, h->IIS, h->IIQ, h->weights, h->radius};
    for (void *p : ptrs) if (p) cudaFree(p);
    if (h->dctx) free_ctx(h->dctx);
    if (h->pool) {
        cudaDeviceSynchronize();   // stream-ordered frees of the preparation have completed
        cudaMemPoolDestroy(h->pool);
    }
    cudaSetDevice(cur);
    delete h;
    return OPTA_OK;
}

opta_status optA_prepare(const opta_image *img, const opta_params *prm, const int32_t *sizes_mn,
                         int32_t n_sizes, void *stream, opta_handle **out) {
    if (!out) return OPTA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_image(img) || n_sizes < 0 || (n_sizes > 0 && !sizes_mn)) return OPTA_ERR_INVALID_ARG;
    opta_params P;
    if (prm) P = *prm; else opta_params_default(&P);
    if (!valid_params(P)) return OPTA_ERR_INVALID_ARG;
    for (int i = 0; i < n_sizes; ++i) {
        const int m = sizes_mn[2 * i], n = sizes_mn[2 * i + 1];
        if (m < 1 || n < 1 || m > img->rows || n > img->cols || n > 1024) return OPTA_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    opta_handle *H = new (std::nothrow) opta_handle();
    if (!H) return OPTA_ERR_OOM;
    cudaGetDevice(&H->device);
    {
        // the preparation's scratch pool keeps its memory between calls
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = H->device;
        if (cudaMemPoolCreate(&H->pool, &props) != cudaSuccess) {
            cudaGetLastError();
            delete H;
            return OPTA_ERR_CUDA;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(H->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    H->prm = P;
    H->p = img->rows;
    H->q = img->cols;
    const int p = H->p, q = H->q;
    auto fail = [&](opta_status st) { optA_destroy(H); return st; };
    opta_status st;
    if ((st = H->mem.alloc(&H->I8, (size_t)p * q)) != OPTA_OK) return fail(st);
    if ((st = ingest(img, H->I8, s)) != OPTA_OK) return fail(st);
    // the image with rows padded to 32 bytes (the tensor-core map's 2-D copies
    // and the survivors' 32-byte loads)
    H->qs = (q + 31) & ~31;
    if ((st = H->mem.alloc(&H->Ipad, (size_t)p * H->qs)) != OPTA_OK) return fail(st);
    {
        const cudaError_t e0 = launch_pad_rows(H->I8, p, q, H->Ipad, H->qs, s);
        if (e0 != cudaSuccess) return fail(map_err(e0));
    }
    const size_t nII = (size_t)(p + 1) * (q + 1);
    if ((st = H->mem.alloc(&H->IIS, nII)) != OPTA_OK) return fail(st);
    if ((st = H->mem.alloc(&H->IIQ, nII)) != OPTA_OK) return fail(st);
    cudaError_t e = launch_integrals(H->I8, nullptr, p, q, H->IIS, H->IIQ, nullptr, s);
    if (e != cudaSuccess) return fail(map_err(e));
    if ((st = setup_tables(H)) != OPTA_OK) return fail(st);
    {
        std::vector<std::pair<int, int>> todo;
        for (int i = 0; i < n_sizes; ++i) todo.emplace_back(sizes_mn[2 * i], sizes_mn[2 * i + 1]);
        if ((st = prepare_sizes(H, todo, s)) != OPTA_OK) return fail(st);
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(map_err(e));
    *out = H;
    return OPTA_OK;
}

opta_status optA_ctx_create(const opta_handle *h, opta_search_ctx **out) {
    if (!h || !out) return OPTA_ERR_INVALID_ARG;
    *out = nullptr;
    opta_search_ctx *X = new (std::nothrow) opta_search_ctx();
    if (!X) return OPTA_ERR_OOM;
    X->device = h->device;
    *out = X;
    return OPTA_OK;
}

opta_status optA_ctx_destroy(opta_search_ctx *X) {
    if (!X) return OPTA_OK;
    if (X->busy.load()) return OPTA_ERR_BUSY;
    free_ctx(X);
    return OPTA_OK;
}

opta_status optA_ctx_memory_bytes(const opta_search_ctx *X, size_t *bytes) {
    if (!X || !bytes) return OPTA_ERR_INVALID_ARG;
    *bytes = X->mem.bytes.load();
    return OPTA_OK;
}

opta_status optA_ctx_bytes_after(opta_handle *h, const opta_search_ctx *X,
                                 const opta_template *t, int32_t n_t, size_t *bytes) {
    if (!h || !X || !bytes || n_t < 0 || (n_t > 0 && !t)) return OPTA_ERR_INVALID_ARG;
    for (int i = 0; i < n_t; ++i)
        if (!valid_template(&t[i], h->p, h->q)) return OPTA_ERR_INVALID_ARG;
    ScratchPlan c;
    {
        std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
        c = plan_scratch(h, t, n_t);
    }
    // the capacities ensure_scratch keeps: the larger of the held and the needed
    const size_t L = std::max(c.L, X->capL), TB = std::max(c.TB, X->capS2);
    const size_t RT = std::max(c.RT, X->capG), T = std::max(c.T, X->capT);
    const size_t TS = std::max(c.TS, X->capTS), B = std::max(c.B, X->capB);
    const size_t N = std::max(c.N, X->capN);
    const size_t fixed = (size_t)kChunk * 256 * kTopkMax * (sizeof(float) + sizeof(int)) +
                         (size_t)kChunk * kTopkMax * (sizeof(int) + sizeof(double)) +
                         (size_t)kScan2MaxT * (2 * kUbBuckets + 1) * sizeof(int) + sizeof(int);
    *bytes = L * TB * (4 * sizeof(float) + sizeof(int) + sizeof(double)) + RT * sizeof(float) +
             T * sizeof(float) + TS * (sizeof(float) + sizeof(double)) + B +
             N * (sizeof(TmplState) + sizeof(TmplIn)) + fixed;
    return OPTA_OK;
}

opta_status optA_search_ctx(opta_handle *h, opta_search_ctx *X, const opta_template *t,
                            int32_t n_t, opta_result *out, void *stream) {
    if (!h || !X || X->device != h->device || n_t < 0 || (n_t > 0 && (!t || !out)))
        return OPTA_ERR_INVALID_ARG;
    bool idle = false;
    if (!X->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard guard(X);
    return search_in(h, X, t, n_t, out, static_cast<cudaStream_t>(stream));
}

opta_status optA_graph_create(opta_handle *h, const opta_template *t, int32_t n_t, void *stream,
                              opta_graph **out) {
    if (!h || !out || n_t < 1 || !t) return OPTA_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n_t; ++i)
        if (!valid_template(&t[i], h->p, h->q)) return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    opta_graph *G = new (std::nothrow) opta_graph();
    if (!G) return OPTA_ERR_OOM;
    G->h = h;
    G->n_t = n_t;
    auto fail = [&](opta_status st) {
        destroy_graph(G);
        return st;
    };
    if (optA_ctx_create(h, &G->X) != OPTA_OK) return fail(OPTA_ERR_OOM);
    // the templates' device buffers (64-byte aligned), filled with the given data
    std::vector<size_t> off(n_t);
    size_t total = 0;
    for (int i = 0; i < n_t; ++i) {
        off[i] = total;
        total += ((size_t)t[i].rows * t[i].cols + 15) & ~(size_t)15;
    }
    if (cudaMalloc(&G->tbuf, total * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(OPTA_ERR_OOM);
    }
    G->desc.resize(n_t);
    for (int i = 0; i < n_t; ++i) {
        opta_template &d = G->desc[i];
        std::memset(&d, 0, sizeof(d));
        d.rows = t[i].rows;
        d.cols = t[i].cols;
        d.stride_elems = t[i].cols;
        d.on_device = 1;
        d.data = G->tbuf + off[i];
        if (cudaMemcpy2DAsync(G->tbuf + off[i], (size_t)d.cols * sizeof(float), t[i].data,
                              (size_t)t[i].stride_elems * sizeof(float), (size_t)d.cols * sizeof(float),
                              d.rows, cudaMemcpyDefault, s) != cudaSuccess) {
            cudaGetLastError();
            return fail(OPTA_ERR_CUDA);
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(map_err(cudaGetLastError()));
    // one search as it runs without the graph: prepares the sizes, grows the
    // scratch to its final size and tunes scan 1's tiles
    {
        std::vector<opta_result> warm(n_t);
        G->X->busy.store(true);
        const opta_status st = search_in(h, G->X, G->desc.data(), n_t, warm.data(), s);
        G->X->busy.store(false);
        if (st != OPTA_OK && st != OPTA_ERR_FLAT_TEMPLATE) return fail(st);
    }
    if (cudaStreamCreateWithFlags(&G->s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(OPTA_ERR_CUDA);
    }
    // capture: the whole batched search, then the copies of its results to
    // the context's pinned mirrors
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    opta_search_ctx *X = G->X;
    if (cudaStreamBeginCapture(G->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return fail(OPTA_ERR_CUDA);
    }
    opta_status st = OPTA_OK;
    if (cudaMemsetAsync(X->dev_err, 0, sizeof(int), G->s) != cudaSuccess) st = OPTA_ERR_CUDA;
    if (st == OPTA_OK) st = enqueue_all(h, X, G->desc.data(), n_t, G->order, G->s);
    if (st == OPTA_OK &&
        (cudaMemcpyAsync(X->states_host, X->states, sizeof(TmplState) * n_t,
                         cudaMemcpyDeviceToHost, G->s) != cudaSuccess ||
         cudaMemcpyAsync(X->err_host, X->dev_err, sizeof(int), cudaMemcpyDeviceToHost, G->s) !=
             cudaSuccess))
        st = OPTA_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(G->s, &graph);
    if (st == OPTA_OK && ec != cudaSuccess) st = map_err(ec);
    if (st != OPTA_OK) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        rl.unlock();
        return fail(st);
    }
    G->graph = graph;
    if (cudaGraphInstantiate(&G->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        rl.unlock();
        return fail(OPTA_ERR_CUDA);
    }
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    G->nodes = nodes;
    *out = G;
    return OPTA_OK;
}

opta_status optA_graph_set_template(opta_graph *G, int32_t i, const opta_template *t, void *stream) {
    if (!G || !t || !t->data || i < 0 || i >= G->n_t) return OPTA_ERR_INVALID_ARG;
    const opta_template &d = G->desc[i];
    if (t->rows != d.rows || t->cols != d.cols || t->stride_elems < t->cols) return OPTA_ERR_INVALID_ARG;
    CK(cudaMemcpy2DAsync(const_cast<float *>(d.data), (size_t)d.cols * sizeof(float), t->data,
                         (size_t)t->stride_elems * sizeof(float), (size_t)d.cols * sizeof(float),
                         d.rows, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)));
    return OPTA_OK;
}

opta_status optA_graph_launch(opta_graph *G, opta_result *out, void *stream) {
    if (!G || !out) return OPTA_ERR_INVALID_ARG;
    opta_search_ctx *X = G->X;
    bool idle = false;
    if (!X->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard cg(X);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaGraphLaunch(G->exec, s));
    CK(cudaStreamSynchronize(s));
    std::shared_lock<std::shared_mutex> rl(G->h->sizes_rw);
    const int herr = *X->err_host;
    opta_status first = OPTA_OK;
    for (int k = 0; k < G->n_t; ++k) {
        const int i = G->order[k];
        const opta_template &d = G->desc[i];
        SizeState *S = size_of(G->h, std::make_pair(d.rows, d.cols));
        fill_result(X->states_host[k], S, S->Lx, (int64_t)S->Ly * S->Lx, S->h,
                    (int64_t)S->Gy * S->Gx, &out[i]);
        if (herr) out[i].status = OPTA_ERR_TIMEOUT;
    }
    for (int i = 0; i < G->n_t; ++i)
        if (first == OPTA_OK && out[i].status != OPTA_OK) first = (opta_status)out[i].status;
    return first;
}

opta_status optA_graph_info(const opta_graph *G, int64_t *nodes) {
    if (!G || !nodes) return OPTA_ERR_INVALID_ARG;
    *nodes = (int64_t)G->nodes;
    return OPTA_OK;
}

opta_status optA_graph_destroy(opta_graph *G) {
    if (!G) return OPTA_OK;
    if (G->X && G->X->busy.load()) return OPTA_ERR_BUSY;
    destroy_graph(G);
    return OPTA_OK;
}

opta_status optA_search(opta_handle *h, const opta_template *t, int32_t n_t, opta_result *out,
                        void *stream) {
    if (!h || n_t < 0 || (n_t > 0 && (!t || !out))) return OPTA_ERR_INVALID_ARG;
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    TRY(default_ctx(h));
    bool idle = false;
    if (!h->dctx->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard cg(h->dctx);
    return search_in(h, h->dctx, t, n_t, out, static_cast<cudaStream_t>(stream));
}

opta_status optA_debug_bounds(opta_handle *h, const opta_template *t, float *ub_map,
                              uint8_t *survived, void *stream) {
    if (!h || !t) return OPTA_ERR_INVALID_ARG;
    if (!valid_template(t, h->p, h->q)) return OPTA_ERR_INVALID_ARG;
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    TRY(default_ctx(h));
    opta_search_ctx *X = h->dctx;
    bool idle = false;
    if (!X->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard cg(X);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> pl(h->prep_mu);
        TRY(prepare_size(h, t->rows, t->cols, s));
    }
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    TRY(size_scratch(h, X, t, 1));
    const opta_template *one = t;
    TRY(enqueue_scan1(h, X, &one, 1, X->states, s));
    TRY(enqueue_scan2(h, X, &one, 1, X->states, ub_map, survived, s));
    TmplState st;
    CK(cudaMemcpyAsync(&st, X->states, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st.flat ? OPTA_ERR_FLAT_TEMPLATE : OPTA_OK;
}

opta_status opta_dbg_survivor_lane_min(int32_t m, int32_t n, int32_t u8, int32_t *lane_min,
                                       int32_t *tuned) {
    if (m < 1 || n < 1 || !lane_min) return OPTA_ERR_INVALID_ARG;
    bool t = false;
    *lane_min = survivor_lane_min(m, n, u8 != 0, &t);
    if (tuned) *tuned = t ? 1 : 0;
    return OPTA_OK;
}

opta_status opta_dbg_survivors(opta_handle *h, const opta_template *t, const int32_t *idx_dev,
                               int64_t count, int32_t form, float *rho_dev, float *eps_dev,
                               void *stream) {
    if (!h || !t || count < 0 || form < -1 || form > 1) return OPTA_ERR_INVALID_ARG;
    if (count > 0 && (!idx_dev || !rho_dev || !eps_dev)) return OPTA_ERR_INVALID_ARG;
    if (!valid_template(t, h->p, h->q)) return OPTA_ERR_INVALID_ARG;
    const int m = t->rows, nn = t->cols, npad = (nn + 7) & ~7;
    const int64_t L = (int64_t)(h->p - m + 1) * (h->q - nn + 1);
    if (count > L || count > INT32_MAX) return OPTA_ERR_INVALID_ARG;
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    TRY(default_ctx(h));
    opta_search_ctx *X = h->dctx;
    bool idle = false;
    if (!X->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard cg(X);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> pl(h->prep_mu);
        TRY(prepare_size(h, m, nn, s));
    }
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    TRY(size_scratch(h, X, t, 1));
    if (count == 0) return OPTA_OK;
    // every index inside the location map before any kernel reads through it
    std::vector<int32_t> hidx((size_t)count);
    CK(cudaMemcpyAsync(hidx.data(), idx_dev, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int32_t v : hidx)
        if (v < 0 || (int64_t)v >= L) return OPTA_ERR_INVALID_ARG;
    SizeState *S = size_of(h, std::make_pair(m, nn));
    const opta_template *one = t;
    TRY(enqueue_scan1(h, X, &one, 1, X->states, s));
    CK(cudaMemcpyAsync(X->surv, idx_dev, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    const Scan2Batch B = scan2_batch_of(h, X, S, X->states, 0, 1);
    CK(launch_survivor_eval(B, S->M, h->p, h->q, S->Lx, S->wsumM, m, nn, npad, S->invM, (int)count, form, s));
    CK(cudaMemcpyAsync(rho_dev, X->surv_rho, (size_t)count * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(eps_dev, X->surv_eps, (size_t)count * sizeof(float), cudaMemcpyDeviceToDevice, s));
    TmplState st;
    CK(cudaMemcpyAsync(&st, X->states, sizeof(st), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st.flat ? OPTA_ERR_FLAT_TEMPLATE : OPTA_OK;
}

opta_status optA_debug_scan1(opta_handle *h, const opta_template *t, int32_t n_t,
                             float *rho_dev, float *theta_dev, void *stream) {
    if (!h || !t || n_t < 1 || n_t > kChunk) return OPTA_ERR_INVALID_ARG;
    for (int i = 0; i < n_t; ++i) {
        if (!valid_template(&t[i], h->p, h->q)) return OPTA_ERR_INVALID_ARG;
        if (t[i].rows != t[0].rows || t[i].cols != t[0].cols) return OPTA_ERR_INVALID_ARG;
    }
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    TRY(default_ctx(h));
    opta_search_ctx *X = h->dctx;
    bool idle = false;
    if (!X->busy.compare_exchange_strong(idle, true)) return OPTA_ERR_BUSY;
    CtxGuard cg(X);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> pl(h->prep_mu);
        TRY(prepare_size(h, t[0].rows, t[0].cols, s));
    }
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    SizeState *S = size_of(h, std::make_pair(t[0].rows, t[0].cols));
    TRY(size_scratch(h, X, t, n_t));
    std::vector<const opta_template *> ptrs(n_t);
    for (int i = 0; i < n_t; ++i) ptrs[i] = &t[i];
    TRY(enqueue_scan1(h, X, ptrs.data(), n_t, X->states, s));
    const size_t G = (size_t)S->Gy * S->Gx;
    if (rho_dev)
        CK(cudaMemcpyAsync(rho_dev, X->rho_tc, n_t * G * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (theta_dev)
        CK(launch_centre_intervals(X->rho_tc, (int64_t)G, n_t, S->c_efac,
                                   scan1_eps_factor(h, t[0].rows, t[0].cols),
                                   reinterpret_cast<float2 *>(theta_dev), s));
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, X->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (herr) {
        CK(cudaMemset(X->dev_err, 0, sizeof(int)));
        return OPTA_ERR_TIMEOUT;
    }
    return OPTA_OK;
}

opta_status optA_size_info(opta_handle *h, int32_t m, int32_t n, opta_size_info *info) {
    if (!h || !info || m < 1 || n < 1 || m > h->p || n > h->q || n > 1024) return OPTA_ERR_INVALID_ARG;
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    {
        std::lock_guard<std::mutex> pl(h->prep_mu);
        TRY(prepare_size(h, m, n, nullptr));
    }
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    SizeState *S = size_of(h, std::make_pair(m, n));
    std::memset(info, 0, sizeof(*info));
    info->m = m; info->n = n;
    info->group_h = S->h;
    info->level = S->level;
    info->cost = S->cost;
    info->n_groups = (int64_t)S->Gy * S->Gx;
    info->blocks_y = (h->p + h->prm.block - 1) / h->prm.block;
    info->blocks_x = (h->q + h->prm.block - 1) / h->prm.block;
    info->n_egs_evals = S->n_evals;
    return OPTA_OK;
}

opta_status optA_debug_maps(opta_handle *h, int32_t m, int32_t n, uint8_t *pivot_dev,
                            float *rho_co_dev, float *sigma_map_host, void *stream) {
    if (!h || m < 1 || n < 1 || m > h->p || n > h->q || n > 1024) return OPTA_ERR_INVALID_ARG;
    if (h->busy) return OPTA_ERR_BUSY;
    BusyGuard guard(h);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> pl(h->prep_mu);
        TRY(prepare_size(h, m, n, s));
    }
    std::shared_lock<std::shared_mutex> rl(h->sizes_rw);
    SizeState *S = size_of(h, std::make_pair(m, n));
    if (pivot_dev)
        CK(cudaMemcpyAsync(pivot_dev, S->P, (size_t)h->p * h->q, cudaMemcpyDeviceToDevice, s));
    if (rho_co_dev)
        CK(cudaMemcpyAsync(rho_co_dev, S->rho_co, (size_t)S->Ly * S->Lx * sizeof(float),
                           cudaMemcpyDeviceToDevice, s));
    if (sigma_map_host)
        std::memcpy(sigma_map_host, S->sigma_map.data(), S->sigma_map.size() * sizeof(float));
    CK(cudaStreamSynchronize(s));
    return OPTA_OK;
}

opta_status optA_memory_bytes(const opta_handle *h, size_t *bytes) {
    if (!h || !bytes) return OPTA_ERR_INVALID_ARG;
    *bytes = h->mem.bytes.load() + (h->dctx ? h->dctx->mem.bytes.load() : 0);
    return OPTA_OK;
}

namespace {
// The exhaustive search's scratch pool of each device: it keeps up to 4 GiB
// between calls (what a repeated search of one image size needs), so calls
// do not map and unmap their scratch every time.
cudaMemPool_t exhaustive_pool() {
    constexpr int kDevs = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kDevs] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
            cudaGetLastError();
            pools[dev] = nullptr;
            return nullptr;
        }
        uint64_t keep = (uint64_t)4 << 30;
        cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return pools[dev];
}
}  // namespace

opta_status zncc_full(const opta_image *img, const opta_template *t, float *rho_map,
                      opta_result *best, void *stream) {
    if (!valid_image(img) || !best) return OPTA_ERR_INVALID_ARG;
    if (!valid_template(t, img->rows, img->cols)) return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int p = img->rows, q = img->cols, m = t->rows, n = t->cols, npad = (n + 7) & ~7;
    const int Ly = p - m + 1, Lx = q - n + 1;
    const int64_t L = (int64_t)Ly * Lx;
    const size_t nII = (size_t)(p + 1) * (q + 1);
    uint8_t *I8 = nullptr;
    long long *IIS = nullptr, *IIQ = nullptr;
    double *td = nullptr;
    float *inv = nullptr, *ef = nullptr, *map = rho_map, *tf = nullptr, *tst = nullptr;
    int *cand = nullptr;
    double *cand_rho = nullptr;
    TmplState *st = nullptr;
    std::vector<void *> owned;
    cudaMemPool_t pool = exhaustive_pool();
    if (!pool) return OPTA_ERR_CUDA;
    auto A = [&](auto **ptr, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMallocFromPoolAsync((void **)ptr, bytes ? bytes : 1, pool, s);
        if (e == cudaSuccess) owned.push_back(*ptr);
        return e;
    };
    auto finish = [&](opta_status stt) {
        for (void *p2 : owned) cudaFreeAsync(p2, s);
        cudaStreamSynchronize(s);
        return stt;
    };
#define ZCK(x) do { cudaError_t e__ = (x); if (e__ != cudaSuccess) return finish(map_err(e__)); } while (0)
    ZCK(A(&I8, (size_t)p * q));
    {
        opta_status stt = ingest(img, I8, s);
        if (stt != OPTA_OK) return finish(stt);
    }
    ZCK(A(&IIS, nII * sizeof(long long)));
    ZCK(A(&IIQ, nII * sizeof(long long)));
    ZCK(A(&inv, L * sizeof(float)));
    ZCK(A(&ef, L * sizeof(float)));
    if (!map) ZCK(A(&map, L * sizeof(float)));
    ZCK(A(&tf, (size_t)m * npad * sizeof(float)));
    ZCK(A(&td, (size_t)m * n * sizeof(double)));
    ZCK(A(&cand, L * sizeof(int)));
    ZCK(A(&cand_rho, L * sizeof(double)));
    ZCK(A(&st, sizeof(TmplState)));
    uint8_t *Ipad = nullptr;
    void *Bt = nullptr;
    int *err = nullptr;
    int *wsum = nullptr;
    if (brute_mma_supported(m, n)) {
        ZCK(A(&Ipad, (size_t)p * ((q + 15) & ~15)));
        ZCK(A(&Bt, brute_tmpl_bytes(m, n)));
        ZCK(A(&err, sizeof(int)));
        ZCK(A(&wsum, L * sizeof(int)));
    }
    const float *tdev = t->data;
    int64_t ld = t->stride_elems;
    if (!t->on_device) {
        ZCK(A(&tst, (size_t)m * n * sizeof(float)));
        ZCK(cudaMemcpy2DAsync(tst, (size_t)n * sizeof(float), t->data,
                              (size_t)t->stride_elems * sizeof(float), (size_t)n * sizeof(float), m,
                              cudaMemcpyHostToDevice, s));
        tdev = tst;
        ld = n;
    }
    const ExhaustiveBufs bufs{IIS, IIQ, inv, ef, map, tf, td, cand, cand_rho, st, Ipad, Bt, err, wsum};
    return finish(exhaustive_run(I8, p, q, tdev, ld, m, n, bufs, best, s));
#undef ZCK
}

// ---------------------------------------------------------------------------
// Verification hooks (opta_debug.h)
// ---------------------------------------------------------------------------
opta_status opta_dbg_window_stats(const uint8_t *I_dev, int32_t p, int32_t q, int32_t m,
                                  int32_t n, float *inv_sigma_dev, void *stream) {
    if (!I_dev || !inv_sigma_dev || p < 1 || q < 1 || m < 1 || n < 1 || m > p || n > q)
        return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nII = (size_t)(p + 1) * (q + 1);
    long long *S = nullptr, *Q = nullptr;
    CK(cudaMallocAsync(&S, nII * sizeof(long long), s));
    CK(cudaMallocAsync(&Q, nII * sizeof(long long), s));
    cudaError_t e = launch_integrals(I_dev, nullptr, p, q, S, Q, nullptr, s);
    if (e == cudaSuccess) e = launch_window_stats(S, Q, p, q, m, n, inv_sigma_dev, nullptr, s);
    cudaFreeAsync(S, s);
    cudaFreeAsync(Q, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    CK(e);
    CK(e2);
    return OPTA_OK;
}

opta_status opta_dbg_blur(const uint8_t *I_dev, int32_t p, int32_t q, const float *sigma_map_host,
                          int32_t block, uint8_t *P_dev, void *stream) {
    if (!I_dev || !P_dev || !sigma_map_host || p < 1 || q < 1 || block < 8 || block > 128)
        return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int bp = (p + block - 1) / block, bq = (q + block - 1) / block;
    // distinct sigma values -> level table
    opta_params prm;
    opta_params_default(&prm);
    prm.n_levels = 0;
    std::vector<uint8_t> lv((size_t)bp * bq, 0);
    for (int b = 0; b < bp * bq; ++b) {
        const float sg = sigma_map_host[b];
        if (!(sg >= 0.f && sg <= 3.0f)) return OPTA_ERR_INVALID_ARG;
        if (sg == 0.f) continue;
        int l = -1;
        for (int k = 0; k < prm.n_levels; ++k) if (prm.sigma_levels[k] == sg) l = k;
        if (l < 0) {
            if (prm.n_levels == 8) return OPTA_ERR_INVALID_ARG;
            prm.sigma_levels[prm.n_levels] = sg;
            l = prm.n_levels++;
        }
        lv[b] = (uint8_t)(l + 1);
    }
    std::vector<float> w;
    std::vector<int> rad;
    gauss_table(prm, w, rad);
    float *dw = nullptr;
    int *dr = nullptr;
    uint8_t *dl = nullptr;
    CK(cudaMallocAsync(&dw, w.size() * sizeof(float), s));
    CK(cudaMallocAsync(&dr, rad.size() * sizeof(int), s));
    CK(cudaMallocAsync(&dl, lv.size(), s));
    CK(cudaMemcpyAsync(dw, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dr, rad.data(), rad.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dl, lv.data(), lv.size(), cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_blur(I_dev, p, q, dl, block, dw, dr, P_dev, s);
    cudaFreeAsync(dw, s);
    cudaFreeAsync(dr, s);
    cudaFreeAsync(dl, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    CK(e);
    CK(e2);
    return OPTA_OK;
}

opta_status opta_dbg_i64_to_f32(const int64_t *v_dev, float *out_dev, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!v_dev || !out_dev))) return OPTA_ERR_INVALID_ARG;
    if (n == 0) return OPTA_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_i64_to_f32(reinterpret_cast<const long long *>(v_dev), out_dev, n, s));
    CK(cudaStreamSynchronize(s));
    return OPTA_OK;
}

opta_status opta_dbg_blur_corr(const uint8_t *P_dev, const uint8_t *I_dev, int32_t p, int32_t q,
                               int32_t m, int32_t n, float *R_dev, float lambda, int32_t block,
                               int32_t *fail_dev, void *stream) {
    if (!P_dev || !I_dev || (!R_dev && !fail_dev) || p < 1 || q < 1 || m < 1 || n < 1 || m > p ||
        n > q)
        return OPTA_ERR_INVALID_ARG;
    if (fail_dev && (block < 1 || block > 4096)) return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nII = (size_t)(p + 1) * (q + 1);
    const size_t L = (size_t)(p - m + 1) * (q - n + 1);
    if (n > 1024) return OPTA_ERR_INVALID_ARG;
    long long *b[2] = {nullptr, nullptr};
    float *inv = nullptr;
    int *ws = nullptr;
    for (auto &x : b) CK(cudaMallocAsync(&x, nII * sizeof(long long), s));
    CK(cudaMallocAsync(&inv, L * sizeof(float), s));
    CK(cudaMallocAsync(&ws, L * sizeof(int), s));
    cudaError_t e = launch_integrals(I_dev, nullptr, p, q, b[0], b[1], nullptr, s);
    if (e == cudaSuccess) e = launch_window_stats(b[0], b[1], p, q, m, n, inv, nullptr, s, ws);
    if (e == cudaSuccess && fail_dev)
        e = cudaMemsetAsync(fail_dev, 0,
                            sizeof(int32_t) * ((p + block - 1) / block) * ((q + block - 1) / block), s);
    if (e == cudaSuccess)
        e = launch_blur_corr(P_dev, I_dev, ws, inv, p, q, m, n, lambda, fail_dev ? block : 64,
                             fail_dev, R_dev, s);
    for (auto &x : b) cudaFreeAsync(x, s);
    cudaFreeAsync(inv, s);
    cudaFreeAsync(ws, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    CK(e);
    CK(e2);
    return OPTA_OK;
}

opta_status opta_dbg_rho_co(const uint8_t *P_dev, const uint8_t *I_dev, int32_t p, int32_t q,
                            int32_t m, int32_t n, int32_t h, float *rco_dev, double rho_cut,
                            int64_t *n_retained_host, void *stream) {
    if (!P_dev || !I_dev || p < 1 || q < 1 || m < 1 || n < 1 || m > p || n > q)
        return OPTA_ERR_INVALID_ARG;
    if (h < 1 || h > 9 || h % 2 == 0 || h_limit(p, q, m, n, h) != h) return OPTA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nII = (size_t)(p + 1) * (q + 1);
    long long *b[2] = {nullptr, nullptr};
    float *inv = nullptr;
    int *ws = nullptr;
    unsigned long long *cnt = nullptr;
    const size_t L = (size_t)(p - m + 1) * (q - n + 1);
    for (auto &x : b) CK(cudaMallocAsync(&x, nII * sizeof(long long), s));
    CK(cudaMallocAsync(&inv, L * sizeof(float), s));
    CK(cudaMallocAsync(&ws, L * sizeof(int), s));
    CK(cudaMallocAsync(&cnt, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    cudaError_t e = launch_integrals(I_dev, nullptr, p, q, b[0], b[1], nullptr, s);
    if (e == cudaSuccess) e = launch_window_stats(b[0], b[1], p, q, m, n, inv, nullptr, s, ws);
    if (e == cudaSuccess)
        e = launch_rho_co(P_dev, I_dev, p, q, m, n, h, ws, inv, (float)rho_cut, rco_dev, cnt,
                          nullptr, nullptr, s);
    unsigned long long hc = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
    for (auto &x : b) cudaFreeAsync(x, s);
    cudaFreeAsync(inv, s);
    cudaFreeAsync(ws, s);
    cudaFreeAsync(cnt, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    CK(e);
    CK(e2);
    if (n_retained_host) *n_retained_host = (int64_t)hc;
    return OPTA_OK;
}

}  // extern "C"
