/*
 * spect_serve.h -- continuous-batching reconstruction server of libspect.
 *
 * The paper reconstructs one acquisition at a time (Sec. 3, OSEM with the
 * Poisson gradient of Table 1).  This server runs many such reconstructions
 * of different sizes, angle counts and iteration budgets as they arrive:
 * requests wait in a queue and are admitted while fewer than max_slots run
 * and their device footprint fits a fixed HBM budget.  Device state lives in
 * slots, one per acquisition geometry in use, reused by later requests of the
 * same geometry: a plan (tables, attenuation cache, sensitivities), the
 * image, counts and scatter buffers, and a CUDA graph of one OSEM iteration
 * captured when the slot is built and replayed n_iters times per request.
 * Admitting a request uploads its counts and mu and recomputes the slot's
 * attenuation cache and sensitivities; slots run on the server's streams and
 * overlap on the device.  Results are bitwise the
 * same alone or in any mix (no state is shared between requests).
 *
 * Threading: the server owns one scheduler thread; every call below is
 * thread-safe.  Errors: SPECT_* status codes of spect.h.
 */
#ifndef SPECT_SERVE_H
#define SPECT_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "spect.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SPECT_REQ_QUEUED 0
#define SPECT_REQ_RUNNING 1
#define SPECT_REQ_DONE 2
#define SPECT_REQ_FAILED 3
#define SPECT_REQ_CANCELLED 4

typedef struct spect_serve_cfg {
    size_t hbm_budget_bytes; /* device memory the admitted requests may hold together */
    int max_slots;           /* requests on the device at once, 1..256 */
    int n_streams;           /* CUDA streams the requests are spread over, 1..64 */
    int wait_timeout_ms;     /* default bound of spect_serve_wait */
} spect_serve_cfg;

typedef struct spect_request {
    spect_geom geom;         /* size, angles, subsets, PSF and precision flags */
    const float* mu_host;    /* [nx][ny][nz] attenuation map (1/cm); copied at submit */
    const float* y_host;     /* [n_angles][ny][nz] measured counts; copied at submit */
    float s;                 /* constant additive scatter term */
    int n_iters;             /* OSEM iterations (each visits all n_subsets subsets) */
    uint64_t tag;            /* caller's label, not interpreted */
} spect_request;

typedef struct spect_serve_stats {
    uint64_t submitted, admitted, completed, failed, cancelled, rejected;
    uint64_t queued, active, peak_active;
    uint64_t bytes_in_use, peak_bytes;
    uint64_t slots_created;        /* device slots built (one per geometry in use, reused) */
    uint64_t graph_slots;          /* of which replay a captured CUDA graph per iteration */
    double p50_ms, p99_ms, max_ms; /* latency, submit to result on the host */
    double recon_per_s;            /* completed / (last completion - first submit) */
} spect_serve_stats;

typedef struct spect_server spect_server;

/* Start a server (streams and scheduler thread) on the current device. */
int spect_serve_create(const spect_serve_cfg* cfg, spect_server** out);

/* Queue a reconstruction.  The inputs are copied; the caller may free them
 * on return.  SPECT_EBUDGET if the request alone exceeds the budget. */
int spect_serve_submit(spect_server* server, const spect_request* req, uint64_t* id);

/* Current state of a request (SPECT_REQ_*). */
int spect_serve_poll(spect_server* server, uint64_t id, int* state);

/* Wait (at most timeout_ms, or the server's default when <= 0) for a request
 * to end; copy its image [nx][ny][nz] into x_host (if not NULL) and its
 * latency into *latency_ms (if not NULL), then forget the request.  Returns
 * the request's status (SPECT_ECANCELLED for a cancelled one) or
 * SPECT_ETIMEDOUT, in which case the request stays known. */
int spect_serve_wait(spect_server* server, uint64_t id, int timeout_ms, float* x_host, double* latency_ms);

/* Cancel a request that has not been admitted yet (SPECT_ESTATE otherwise). */
int spect_serve_cancel(spect_server* server, uint64_t id);

/* Counters and the latency percentiles of the requests completed so far. */
int spect_serve_stats_get(spect_server* server, spect_serve_stats* out);

/* Let admitted requests finish, cancel queued ones, stop the scheduler and
 * free everything; requests not yet waited for are forgotten. */
int spect_serve_destroy(spect_server* server);

#ifdef __cplusplus
}
#endif

#endif /* SPECT_SERVE_H */
