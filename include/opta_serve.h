/*
 * opta_serve.h -- serving loop over device-resident prepared images.
 *
 * Not in the paper (which searches one template at a time): a request loop
 * that keeps prepared images resident on one GPU and answers template
 * queries as they arrive.  Requests are searched in batches by a fixed set
 * of workers, each a host thread with its own stream and search context
 * (optA_search_ctx); a worker that finishes a batch takes the next
 * requests waiting for one image, so requests that arrive while other
 * batches are on the GPU join the next free worker (continuous batching)
 * and the batches of different workers overlap on the device.  A batch is
 * admitted only while the workers' search scratch stays within the
 * configured device-memory budget: a batch that would exceed it is cut down,
 * and a single request that cannot fit waits for other workers to release
 * scratch, or fails with OPTA_ERR_OOM when nothing else holds any.
 *
 * Every result equals what optA_search returns for that template alone on
 * the same handle: the search of one template does not depend on the
 * others in its batch (the argmax is exact and its rho comes from the same
 * FP64 evaluation).
 */
#ifndef OPTA_SERVE_H
#define OPTA_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "opta.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opta_server opta_server;

typedef struct opta_server_config {
    int32_t n_workers;       /* concurrent batches (host threads and streams); default 4 */
    int32_t max_batch;       /* requests per batch at most; default 64 */
    int64_t memory_budget;   /* device bytes for the workers' search scratch together;
                                0 = no limit (default) */
    int32_t reserved[8];
} opta_server_config;

/* One finished request.  Times are seconds on the server's steady clock
 * (zero at opta_server_create). */
typedef struct opta_completion {
    uint64_t request_id;
    int32_t image_id;
    int32_t batch_size;      /* requests searched in the same batch (this one included) */
    int32_t worker;
    int32_t status;          /* opta_status of the request (also result.status) */
    double t_submit, t_start, t_done;
    opta_result result;
} opta_completion;

void opta_server_config_default(opta_server_config *cfg);

/* Start the workers on the current device.  `cfg` may be NULL (defaults). */
opta_status opta_server_create(const opta_server_config *cfg, opta_server **out);

/* Prepare `img` as optA_prepare does (same arguments) and keep it resident;
 * *image_id names it in requests.  May be called while requests run. */
opta_status opta_server_add_image(opta_server *srv, const opta_image *img,
                                  const opta_params *prm, const int32_t *sizes_mn,
                                  int32_t n_sizes, int32_t *image_id);

/* Queue one query of image `image_id`.  The template data must be in host
 * memory; it is copied before the call returns.  *request_id (nullable)
 * receives the id its completion carries (ids increase from 1). */
opta_status opta_server_submit(opta_server *srv, int32_t image_id, const opta_template *t,
                               uint64_t *request_id);

/* Move up to `capacity` finished requests into `out` (oldest first),
 * waiting up to timeout_ms milliseconds (< 0: no limit) until at least
 * min_count are available; *n_out receives the number written. */
opta_status opta_server_wait(opta_server *srv, opta_completion *out, int32_t capacity,
                             int32_t min_count, int32_t timeout_ms, int32_t *n_out);

/* Requests submitted and not yet returned by opta_server_wait. */
opta_status opta_server_pending(opta_server *srv, int64_t *n);

/* Device bytes held for resident image `image_id` (its integral images and
 * prepared sizes; *image_bytes, nullable) and by the workers' search scratch
 * together (*scratch_bytes, nullable; what the memory budget limits). */
opta_status opta_server_memory(opta_server *srv, int32_t image_id, int64_t *image_bytes,
                               int64_t *scratch_bytes);

/* Finish the queued requests, stop the workers and release every image
 * and context (NULL is accepted). */
opta_status opta_server_destroy(opta_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* OPTA_SERVE_H */
