/*
 * cwo_serve.h -- native serving runtime of libcwo_gb300.so: continuous batching of mixed-size
 * propagation requests on one GPU.
 *
 * The paper's library propagates one field per call (Diffract, Section "CWO class"); a service
 * that receives many independent requests of different sizes, methods and parameters runs many
 * such calls.  This runtime keeps, for every served size, a few slots -- a plan with its tables
 * and scratch resident, a CUDA stream (higher priority for small sizes), an event and
 * input/output buffers -- and one queue per size.  Whenever a slot of a size is free and the
 * device-memory budget admits the batch, up to the slot's capacity of the queued requests of that
 * size are gathered into the slot's input buffer and propagated as one mixed batch
 * (cwo_propagate_items: every item keeps its own type, distance, wavelength and pitch).  Requests
 * that arrive while others run are admitted as soon as a slot and memory free up; batches of
 * different sizes run concurrently on different streams.  Results do not depend on the batch a
 * request travels in (bit for bit).  Completion is observed with cudaEventQuery on the slot's
 * event; no call blocks on the device except cwo_server_create, cwo_server_destroy,
 * cwo_server_warm_up and the serial baseline.
 *
 * Ownership: the caller owns request fields and outputs (device memory of the server's device,
 * [n][n] complex64); a field must stay unchanged, and an output untouched, until its request is
 * done.  The server owns its plans, streams, events and buffers.
 * Errors: every entry point returns a cwo_status (cwo.h); cwo_last_error() describes failures.
 * Thread safety: one server is driven from one thread at a time.
 */
#ifndef CWO_SERVE_H
#define CWO_SERVE_H

#include <stddef.h>

#include "cwo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cwo_server cwo_server;

/* One propagation request. */
typedef struct {
    int n;                  /* field side: one of the server's sizes                               */
    int type;               /* CWO_ANGULAR or CWO_FRESNEL_CONV                                     */
    double z;               /* distance, metres (non-zero for CWO_FRESNEL_CONV), finite            */
    double wavelength;      /* metres, > 0                                                         */
    double pitch;           /* sampling pitch along both axes, metres, > 0                         */
    const void* field;      /* device [n][n] complex64 input                                       */
    void* out;              /* device [n][n] complex64 output, or NULL (result not kept)           */
    double t_arrival;       /* open-loop runs: release time, seconds after the run starts          */
} cwo_request;

typedef struct {
    long long batches;      /* mixed batches launched                                              */
    long long completed;    /* requests completed                                                  */
    size_t mem_in_use;      /* bytes of the batches in flight                                      */
    size_t mem_peak;        /* largest mem_in_use seen                                             */
    size_t mem_budget;      /* the admission budget                                                */
} cwo_server_stats;

/*
 * Create a server on the current device for `nsizes` sizes (powers of two in [16, 4096]) with
 * max_batch[i] requests per batch of sizes[i] and `slots_per_size` slots each (1..8).
 * mem_budget: bytes that batches in flight may hold (plan scratch and tables, gathered inputs and
 * outputs, as cwo_server_batch_bytes counts them); 0 means the sum over all slots at full
 * capacity.  Allocates everything it will use; synchronises the device.
 */
cwo_status cwo_server_create(int nsizes, const int* sizes, const int* max_batch, int slots_per_size,
                             size_t mem_budget, cwo_server** out);

/* Wait for the work in flight and release everything (NULL is accepted). */
cwo_status cwo_server_destroy(cwo_server* srv);

/* Device bytes a batch of b fields of n x n holds while in flight (admission accounting). */
cwo_status cwo_server_batch_bytes(int n, int b, size_t* bytes);

/*
 * Admission rule: how many of `queued` requests one free slot of capacity `capacity` takes now
 * -- up to its capacity, halved until the batch fits the budget next to `in_use` bytes already
 * in flight (0: wait for completions).  bytes(b) = cwo_server_batch_bytes(n, b).  Host only.
 */
cwo_status cwo_server_admit(int queued, int capacity, size_t in_use, size_t budget, int n, int* take);

/*
 * Queue one request; *ticket identifies it.  The request is checked on the host first (size
 * served, type, parameters, one field within the budget, field and out device memory of the
 * server's device holding n*n complex64 values); on failure nothing is queued.  The server keeps
 * a small record (~70 bytes) of every submitted request until it is destroyed, so that
 * cwo_server_done answers for any ticket; an open-loop run keeps none of its own.
 */
cwo_status cwo_server_submit(cwo_server* srv, const cwo_request* req, long long* ticket);

/* Later launches of the server wait for the work enqueued on cuda_stream so far (fields that
 * the caller produced on that stream). */
cwo_status cwo_server_after(cwo_server* srv, void* cuda_stream);

/* Admit what fits and collect what finished; *completed (may be NULL) = requests completed. */
cwo_status cwo_server_step(cwo_server* srv, int* completed);

/* 1 if the request has completed (its output written), 0 if not, -1 for an unknown ticket;
 * *t_done (may be NULL) = observed completion time, seconds after the server was created. */
int cwo_server_done(cwo_server* srv, long long ticket, double* t_done);

/*
 * Open-loop run: request i is released at reqs[i].t_arrival seconds after the call starts
 * (reqs in any order); the call returns when every request has completed.  t_done[i] = observed
 * completion time of request i, seconds after the call started.  Requests are checked as by
 * cwo_server_submit before the run starts.
 */
cwo_status cwo_server_run(cwo_server* srv, const cwo_request* reqs, int nreq, double* t_done);

/*
 * Baseline of the same stream: each request, in arrival order, released at its t_arrival and
 * propagated alone on one stream with the server's first slot of its size, the host waiting for
 * it before the next one.  t_done as in cwo_server_run.
 */
cwo_status cwo_server_run_serial(cwo_server* srv, const cwo_request* reqs, int nreq, double* t_done);

/* Propagate a single and a gathered batch of each type in every slot (zero fields), so that no
 * first-use cost lands in a measured run.  Synchronises the device. */
cwo_status cwo_server_warm_up(cwo_server* srv);

cwo_status cwo_server_get_stats(const cwo_server* srv, cwo_server_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* CWO_SERVE_H */
