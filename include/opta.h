/*
 * opta.h -- C ABI of the GB300 OptA template-search library (libopta.so).
 *
 * The problem (Section 1 of Mahmood, Mian & Owens, "Optimizing
 * Auto-correlation for Fast Target Search in Large Search Space"): match a
 * template t (m x n) at every location of a search image I (p x q) and
 * return the location that maximises the correlation coefficient
 *
 *   rho(y,x) = sum_{u,v} (t(u,v)-mu_t)(I(y+u,x+v)-mu_o) / (sigma_t sigma_o)
 *   sigma    = sqrt(sum (.-mu)^2)                             (Eq. rho1)
 *
 * Locations are window top-left corners, y in [0, p-m], x in [0, q-n];
 * images are row-major.  A flat window (sigma_o == 0) has rho := 0.  The
 * result is the maximum of signed rho; ties go to the lowest row-major
 * index.  The returned rho is recomputed in FP64.
 *
 * optA_search skips locations with the transitive bound of Section 2
 * (Eq. tranEqq / Eq. SEC) applied with an explicit floating-point safety
 * margin, so it returns the same location as the exhaustive search
 * (zncc_full) up to exact ties.  optA_prepare does the per-image work of
 * Sections 3-5 (local statistics, spatially varying blur, blur correlation
 * and lambda test, auto-correlation, EGS group size, OptA level loop).
 *
 * Conventions for every entry point:
 *   - Pointers flagged `on_device` are CUDA device pointers on the current
 *     device; others are host pointers.  Inputs are never modified and the
 *     caller keeps ownership of everything it passes.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *     enqueue their GPU work on it; calls that return host results
 *     synchronise that stream before returning.
 *   - No entry point aborts, throws or exits; errors are returned as
 *     opta_status and leave handles valid.
 *   - Not re-entrant per handle: calls on one handle must be serialised.
 */
#ifndef OPTA_H
#define OPTA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum opta_status {
    OPTA_OK = 0,
    OPTA_ERR_INVALID_ARG = 1,   /* null pointer, template larger than image, bad stride/size */
    OPTA_ERR_FLAT_TEMPLATE = 2, /* sigma_t == 0: rho undefined (per-template status) */
    OPTA_ERR_OOM = 3,           /* device allocation failed */
    OPTA_ERR_CUDA = 4,          /* any other CUDA runtime error */
    OPTA_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    OPTA_ERR_BUSY = 6,          /* handle in use */
    OPTA_ERR_UNSUPPORTED = 7,   /* input outside the supported domain (see optA_prepare) */
    OPTA_ERR_TOO_LARGE = 8      /* template size outside optA's limits, or a problem larger
                                   than zncc_full_noalloc's fixed scratch */
} opta_status;

typedef enum opta_dtype {
    OPTA_U8 = 0,   /* uint8 pixels */
    OPTA_F32 = 1   /* float32 pixels */
} opta_dtype;

/* Search image I, p = rows, q = cols, row stride in elements (>= cols). */
typedef struct opta_image {
    int32_t rows;
    int32_t cols;
    int64_t stride_elems;
    int32_t dtype;        /* opta_dtype */
    int32_t on_device;    /* 1: data is a device pointer */
    const void *data;
} opta_image;

/* Template t, m = rows, n = cols, float32, row stride in elements. */
typedef struct opta_template {
    int32_t rows;
    int32_t cols;
    int64_t stride_elems;
    int32_t on_device;
    int32_t reserved;
    const float *data;
} opta_template;

/* Per-template result. */
typedef struct opta_result {
    int32_t y, x;          /* best-match window top-left */
    double rho;            /* rho at (y, x), recomputed in FP64 */
    int64_t n_locations;   /* (p-m+1)(q-n+1) */
    int64_t n_centres;     /* group centres matched (scan 1, Section 6) */
    int64_t n_survivors;   /* locations that failed the elimination test */
    int64_t n_candidates;  /* locations recomputed in FP64 for the final argmax */
    int64_t n_evaluated;   /* survivors whose rho was computed; the others were
                              skipped once the running threshold passed their bound */
    double rho_threshold;  /* scan-1 threshold (max exact rho over the threshold centres) */
    int32_t group_h;       /* group side h (1 for zncc_full) */
    int32_t status;        /* opta_status of this template */
    int32_t y_hat, x_hat;  /* maximum on the image the search ran on: the blurred
                              pivot in the literal mode (Section 4.3), before the
                              local re-match on I; equal to (y, x) otherwise */
    int32_t rematch_d;     /* half-width d of the re-match neighbourhood (literal
                              mode: ceil(3 sigma_max) of the accepted blur map); 0 otherwise */
    int32_t reserved;
} opta_result;

/* Method parameters (Section 7 defaults via opta_params_default). */
typedef struct opta_params {
    double rho_th;          /* 0.80: cost-model threshold of Algorithms 2 and 3 */
    double rho_max;         /* 0.95: rho_max of Eq. misDec */
    double xi;              /* 0.005: relative cost decrement (Section 3.4) */
    int32_t block;          /* 64: side of the blocks that carry one blur sigma */
    int32_t n_levels;       /* number of entries used in sigma_levels (<= 8) */
    float sigma_levels[8];  /* blur levels tried in order: {0.5, 1, 2, 3} */
    int32_t h_max;          /* 9: largest group side tried by EGS (odd) */
    int32_t fixed_h;        /* 0: EGS chooses h; odd h > 0: fixed group side */
    int32_t blur;           /* 1: run the OptA level loop; 0: unblurred pivots */
    int32_t topk;           /* 8: centres re-evaluated on I for the threshold (1..16) */
    int32_t precision;      /* scan 1 (centre rho): 1 = fp16 hi/lo split products on the
                               tensor cores, FP32 accumulation (default); 0 = FP32 CUDA cores */
    int32_t literal;        /* 0 (default): exact search of I with blurred pivots bounding it.
                               1: the procedure of Section 4.3 -- EGS measures the blurred
                               image's own auto-correlation, the pruned search finds the
                               exact maximum on the blurred image Î, and t is then matched
                               with I in FP64 over the (2d+1) x (2d+1) neighbourhood of that
                               location, d = ceil(3 sigma_max) of the accepted blur map.
                               Fast but not exact: the result may miss the maximum on I. */
    int32_t egs_sample;     /* 8: Algorithm 2's retained count n_r is taken over a systematic
                               sample of the location grid -- the group rows g with
                               (g / 8) % egs_sample == 0, in runs of 8 group rows -- and
                               scaled to the grid; 0 or 1 counts every location as
                               Algorithm 2 does.  EGS's trials count only, and the
                               accepted configuration's map is computed once.  Speed
                               only: the search's answer does not depend on it.  <= 64. */
    int32_t dense;          /* 1 (default): a template whose survivors left after a first
                               sweep over the head of scan 2's bound-ordered survivor list
                               (about 20 L/(m n) of them) and a second cut still exceed
                               min(1/2, dense_cut/(m n)) of the locations has
                               rho computed at every location on the tensor cores (the
                               exhaustive map's kernel) instead of survivor by survivor;
                               0: never; 2: every template with a survivor left after the
                               cut, without the first sweep (for tests).
                               Exact search of templates up to 128 x 128 only.  Speed only. */
    float dense_cut;        /* 0 (default) means 100: see `dense` */
    int32_t reserved[3];
} opta_params;

typedef struct opta_handle opta_handle;
typedef struct opta_search_ctx opta_search_ctx;
typedef struct opta_graph opta_graph;

/* Per-template-size preparation summary (see optA_size_info). */
typedef struct opta_size_info {
    int32_t m, n;
    int32_t group_h;        /* chosen group side */
    int32_t level;          /* index of the accepted OptA level (0 = unblurred) */
    int64_t cost;           /* EGS cost of the chosen configuration, in rho evaluations */
    int64_t n_groups;       /* number of groups (centres) */
    int32_t blocks_y, blocks_x;  /* blur-map size */
    int32_t n_egs_evals;    /* auto-correlation maps evaluated by the level loop */
    int32_t reserved;
} opta_size_info;

/* Fill `prm` with the Section 7 defaults: rho_th 0.80, rho_max 0.95,
 * xi 0.005, 64-pixel blur blocks, sigma levels {0.5,1,2,3}, h_max 9, EGS
 * group sizes, blur on, top-8 threshold centres, tensor-core scan 1. */
void opta_params_default(opta_params *prm);

/* Static string for a status code (never NULL). */
const char *opta_status_str(opta_status s);

/*
 * Prepare a device-resident handle for image `img` (Algorithm 3 per
 * template size).  The image is copied; the caller keeps `img->data`.
 * Supported domain: pixel values that are integers in [0, 255] (uint8, or
 * float32 holding such integers); other float images give
 * OPTA_ERR_UNSUPPORTED (use zncc_full for them).  `sizes_mn` lists n_sizes
 * (m, n) pairs to prepare now (may be NULL / 0); other sizes are prepared
 * on first use by optA_search.  Template sizes: n <= 1023 and m * n <=
 * 66051 pixels (e.g. 256 x 256; the group auto-correlation sums are 32-bit),
 * and the rows of one window must fit the kernel's shared-memory ring;
 * larger sizes give OPTA_ERR_TOO_LARGE (zncc_full has no pixel-count limit).
 * The handle owns all device memory it
 * allocates (integral images, blur maps, pivot images, auto-correlation
 * maps, group statistics, search scratch).  `prm` may be NULL (defaults).
 * Synchronises `stream`.
 */
opta_status optA_prepare(const opta_image *img, const opta_params *prm,
                         const int32_t *sizes_mn, int32_t n_sizes,
                         void *stream, opta_handle **out);

/*
 * Best match of each of the n_t templates (Section 2 elimination with the
 * two scans of Section 6).  `t` is a host array of n_t descriptors whose
 * data may be on host or device; sizes may differ.  `out` is a host array
 * of n_t results.  Returns OPTA_OK or the first per-template error; the
 * per-template status is in out[i].status.  Synchronises `stream`.
 */
opta_status optA_search(opta_handle *h, const opta_template *t, int32_t n_t,
                        opta_result *out, void *stream);

/*
 * Search contexts: the scratch memory and per-template state of a search,
 * apart from the prepared images.  A context serves any handle on the
 * device of the handle it was created with.  Searches through different
 * contexts may run at the same time, from different host threads on
 * different streams, on one handle or several, and their kernels overlap on
 * the device; a context runs one search at a time (a second concurrent call
 * returns OPTA_ERR_BUSY).  Sizes not prepared yet are prepared by the first
 * search that needs them, one preparation per handle at a time.
 * optA_search uses a context of its own.  A context grows its scratch on
 * demand and keeps it until it is destroyed (the handles it served may be
 * destroyed first, once no search through it is running on them).
 */
opta_status optA_ctx_create(const opta_handle *h, opta_search_ctx **out);
opta_status optA_ctx_destroy(opta_search_ctx *ctx);
/* Device bytes currently held by the context's scratch. */
opta_status optA_ctx_memory_bytes(const opta_search_ctx *ctx, size_t *bytes);
/* Device bytes `ctx` would hold after searching the n_t templates `t` on
 * handle h: its scratch grows to the larger of what it holds and what the
 * batch needs, and keeps it (sizes not prepared yet are counted at their
 * largest).  For admission control by device memory; no device work. */
opta_status optA_ctx_bytes_after(opta_handle *h, const opta_search_ctx *ctx,
                                 const opta_template *t, int32_t n_t, size_t *bytes);
/* optA_search through context `ctx` (created on h's device). */
opta_status optA_search_ctx(opta_handle *h, opta_search_ctx *ctx, const opta_template *t,
                            int32_t n_t, opta_result *out, void *stream);

/*
 * The batched search as one CUDA graph, for searching the same set of
 * template sizes again and again (new template data each time).
 * optA_graph_create copies the n_t templates (host or device data) into
 * device buffers the graph owns, runs one ordinary search (which prepares
 * the sizes, sizes the scratch and tunes scan 1's tiles), then captures the
 * whole batched search -- every kernel launch and the copy of its results
 * to pinned host memory -- into a graph on a stream of its own.  The graph
 * has its own search context; handle h must outlive it.
 * optA_graph_set_template replaces template i's data (same size; host or
 * device source, queued on `stream`); optA_graph_launch replays the graph
 * on `stream`, waits, and fills out[0..n_t) as optA_search would.
 */
opta_status optA_graph_create(opta_handle *h, const opta_template *t, int32_t n_t, void *stream,
                              opta_graph **out);
opta_status optA_graph_set_template(opta_graph *g, int32_t i, const opta_template *t, void *stream);
opta_status optA_graph_launch(opta_graph *g, opta_result *out, void *stream);
/* Number of nodes (kernel launches, copies, memsets) in the captured graph. */
opta_status optA_graph_info(const opta_graph *g, int64_t *nodes);
opta_status optA_graph_destroy(opta_graph *g);

/*
 * Exhaustive search: rho at all locations and its argmax (Eq. rho1).  Same
 * image domain as optA_prepare (integers in [0, 255]; OPTA_ERR_UNSUPPORTED
 * otherwise).  `rho_map` (nullable) is a DEVICE buffer of
 * (p-m+1)(q-n+1) floats that receives the FP32 rho map; `best` (host)
 * receives the FP64-refined best match.  The map is taken on the tensor
 * cores (bf16 hi/lo split of t - mu_t, FP32 accumulation) for templates up
 * to 128 x 128, on FP32 CUDA cores beyond; either way every candidate
 * within the map's error bound of its maximum is re-evaluated in FP64.
 * Allocates its scratch from a library pool of the current device (stream-
 * ordered; the pool keeps up to 4 GiB between calls) and frees it before
 * returning.  Synchronises.
 */
opta_status zncc_full(const opta_image *img, const opta_template *t,
                      float *rho_map, opta_result *best, void *stream);

/*
 * zncc_full without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they search (a framework allocator owns the device heap, a
 * real-time loop must not call cudaMalloc/cudaFree, which may synchronise
 * the device, or a fixed memory budget).  Same arguments, results and
 * image domain as zncc_full.
 *
 * Scratch: one ~12 MB array in the library's device memory, held by every
 * GPU that loads the library until the process exits.  Limits: p, q <= 4096
 * with p*q <= 262144 pixels, and m * round_up(n, 8) <= 4096 template
 * elements; larger problems return OPTA_ERR_TOO_LARGE before touching the
 * GPU.  The first call on each device looks up the array's device address
 * (on that device, which must be current).  Never call it while `stream`
 * is being captured into a graph: every call reads its result back into
 * host memory and synchronises `stream`.  All calls share the array: calls
 * that overlap on the GPU (e.g. from two streams or threads) race and must
 * be serialised by the caller.  Calls no cudaMalloc/cudaFree.
 */
opta_status zncc_full_noalloc(const opta_image *img, const opta_template *t,
                              float *rho_map, opta_result *best, void *stream);

/*
 * Elimination test of one template over the full location map, for
 * verification: `ub_map` (device, L floats, nullable) receives the
 * margin-widened upper bound of every location, `survived` (device, L
 * bytes, nullable) 1 where the location failed the elimination test.
 * The threshold used is the one optA_search would use.  Synchronises.
 */
opta_status optA_debug_bounds(opta_handle *h, const opta_template *t,
                              float *ub_map, uint8_t *survived, void *stream);

/* Summary of the preparation of size (m, n) (prepared on demand). */
opta_status optA_size_info(opta_handle *h, int32_t m, int32_t n, opta_size_info *info);

/* Device bytes currently owned by the handle (its own search context
 * included, other contexts not). */
opta_status optA_memory_bytes(const opta_handle *h, size_t *bytes);

/* Release the handle and all its device memory (NULL is accepted). */
opta_status optA_destroy(opta_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* OPTA_H */
