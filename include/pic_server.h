/*
 * pic_server.h -- continuous-batching server of independent PIC simulations
 * on one GPU (libpic).
 *
 * A request is a small, independent simulation, for example one member of a
 * parameter scan over the laser-plasma setups of arXiv 2104.11385 Sec. 3.
 * The server keeps every admitted request's state resident in HBM, admits
 * pending requests as slots and memory free up (admission by HBM footprint),
 * and on every tick advances each active request by one PIC step with all their
 * boxes packed into ONE launch of the persistent particle kernel, followed by
 * field and sort kernels batched over the active requests.  Requests join and
 * leave between ticks, so their work overlaps on the device.  The paper's cost
 * measurement runs inside the packed launch (per request, per box).
 *
 * Conventions are those of include/pic_api.h: pic_status return codes, never
 * aborts, messages via pic_server_last_error.  A server handle is not
 * thread-safe.
 */
#ifndef PIC_SERVER_H
#define PIC_SERVER_H
#include "pic_api.h"
#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_server pic_server; /* opaque */

/* Server configuration.
 *   dim, shape_order  shared by every request (one particle-kernel variant).
 *   max_active        at most this many requests on the GPU at once (slots).
 *   hbm_budget_bytes  admission budget: the summed device footprint of the
 *                     requests held (active or finished and not yet released)
 *                     never exceeds it.
 *   stream            cudaStream_t for all device work (NULL: a private one). */
typedef struct {
    int dim, shape_order;
    int max_active;
    int64_t hbm_budget_bytes;
    void* stream;
} pic_server_desc;

/* Initial plasma drawn on the device (a thermal plasma with a density ripple,
 * whose Langmuir oscillation makes every request self-checking):
 *   ppc            macro-electrons per cell (>= 1).
 *   density        n0 of the electrons; a fixed ion background -n0*q cancels
 *                  the mean charge (q = -1, m = 1: omega_pe^2 = n0).
 *   u_th           standard deviation of each momentum component (u = gamma v).
 *   ripple         relative amplitude a of n(x) = n0 (1 + a cos(2 pi x / Lx)),
 *                  carried by the particle weights.
 *   seed           key of the counter-based generator (Philox4x32-10, Salmon
 *                  et al., SC'11): particle i of cell c draws with counter
 *                  (c * ppc + i, 0|1, 0, 0). */
typedef struct {
    int ppc;
    double density, u_th, ripple;
    uint64_t seed;
} pic_plasma_init;

/* Explicit species given as host arrays (copied at submit; same layout as
 * pic_add_species). */
typedef struct {
    double charge, mass;
    int64_t np;
    const double* soa[7];
    const int64_t* ids;
} pic_species_init;

/* One request.
 *   grid       geometry (dim and shape_order must match the server); stream
 *              and absorb_cells are ignored (requests are periodic).
 *   nsteps     PIC steps to run (>= 1).
 *   nspecies   0: the plasma is drawn from `plasma`; 1..4: `species` given. */
typedef struct {
    pic_grid_desc grid;
    int nsteps;
    pic_plasma_init plasma;
    int nspecies;
    pic_species_init species[4];
} pic_request_desc;

enum {
    PIC_REQ_PENDING = 0, /* waiting for a slot and memory   */
    PIC_REQ_ACTIVE = 1,  /* resident, stepping every tick    */
    PIC_REQ_DONE = 2,    /* finished, results resident       */
    PIC_REQ_RELEASED = 3,
    PIC_REQ_CANCELLED = 4, /* withdrawn by pic_server_cancel */
    PIC_REQ_FAILED = 5     /* could not be admitted (see pic_server_tick) */
};

pic_status pic_server_create(const pic_server_desc* desc, pic_server** out);

/* Queues a request.  Its device footprint is computed from the description;
 * a request that could never fit the budget is refused with PIC_ENOMEM.
 * *req_id receives the request id.  Errors: PIC_EINVAL, PIC_ENOMEM. */
pic_status pic_server_submit(pic_server* srv, const pic_request_desc* req, int64_t* req_id);

/* One tick: admits pending requests in submission order while a slot is free
 * and the footprint fits, advances every active request by one step (one
 * packed particle launch), and marks requests that reached their step count
 * DONE.  Synchronises the stream.  *n_active and *n_pending (nullable) receive
 * the counts after the tick.  A request whose admission fails without a
 * device error (its grid or species rejected by pic_init or pic_add_species,
 * or their allocation failing) becomes PIC_REQ_FAILED, with the reason in
 * pic_server_last_error, and the tick goes on with the other requests; a
 * device error poisons the server (PIC_ECUDA, then PIC_ESTATE). */
pic_status pic_server_tick(pic_server* srv, int* n_active, int* n_pending);

/* State and host wall-clock times (seconds, steady clock) of a request:
 * submitted, admitted, finished (negative when not reached); steps done. */
pic_status pic_server_poll(pic_server* srv, int64_t req_id, int* state, double* t_submit,
                           double* t_admit, double* t_done, int* steps_done);

/* Results of a DONE request: one field component (layout of pic_read_fields)
 * or one species' particles (layout of pic_read_particles), host buffers. */
pic_status pic_server_read_fields(pic_server* srv, int64_t req_id, int comp, double* out);
pic_status pic_server_num_particles(pic_server* srv, int64_t req_id, int species, int64_t* np);
pic_status pic_server_read_particles(pic_server* srv, int64_t req_id, int species,
                                     double* const soa_out[7], int64_t* id_out);

/* Frees a DONE request's device state (its footprint leaves the budget). */
pic_status pic_server_release(pic_server* srv, int64_t req_id);

/* Withdraws a request that has not finished, between ticks: a PENDING one
 * leaves the queue without being admitted; an ACTIVE one stops stepping, its
 * device state is freed, and its slot and footprint go back to the server, so
 * the next tick can admit the next pending request into them.  The other
 * requests are unaffected (their state lives in their own slots).  The state
 * becomes PIC_REQ_CANCELLED and the request has no results.  Synchronises the
 * server's stream first.  Errors: PIC_EINVAL (unknown id), PIC_ESTATE (the
 * request is DONE, RELEASED or already CANCELLED: use pic_server_release for a
 * finished one). */
pic_status pic_server_cancel(pic_server* srv, int64_t req_id);

/* Device bytes of a request as admitted (or as estimated while pending). */
pic_status pic_server_footprint(pic_server* srv, int64_t req_id, int64_t* bytes);

/* Totals since creation: ticks, particle updates, packed launches. */
typedef struct {
    int64_t ticks, particle_updates, particle_launches, kernels, admitted, finished;
    int64_t bytes_in_use;
} pic_server_stats;
pic_status pic_server_get_stats(pic_server* srv, pic_server_stats* out);

pic_status pic_server_destroy(pic_server* srv);
const char* pic_server_last_error(const pic_server* srv);

#ifdef __cplusplus
}
#endif
#endif
