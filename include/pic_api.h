/*
 * pic_api.h -- C ABI of libpic: a single-GPU (GB300, sm_103a) particle-in-cell
 * step with in-situ device-side cost measurement per box and the dynamic load
 * balancing that the measurement drives, after
 *   Rowan, Gott, Deslippe, Huebl, Thevenet, Lehe, Vay, "In-Situ Assessment of
 *   Device-Side Compute Work for Dynamic Load Balancing in a GPU-Accelerated
 *   PIC Code", arXiv 2104.11385.
 *
 * Conventions shared by every call:
 *   - Every function returns pic_status; nothing aborts, throws or exits across
 *     the ABI.  On error, pic_last_error(sim) returns a one-line reason.
 *   - After a device-side error (CUDA error, bounded wait that ran out) the
 *     handle is poisoned: every later call on it returns PIC_ESTATE; only
 *     pic_destroy and pic_last_error remain valid.
 *   - Inputs are caller-owned and copied on entry.  Outputs go to caller
 *     buffers of the documented size.  Pointers flagged "on_device" are device
 *     pointers valid on the simulation's device (e.g. from torch); otherwise
 *     they are host pointers.
 *   - Units are normalised: c = eps0 = mu0 = 1.  Positions are physical
 *     coordinates in [0, L) with L = ncell * dx per direction.
 *   - Grid field arrays exchanged through the ABI are dense, periodic,
 *     ncell[0]*ncell[1]*ncell[2] doubles, flat index (k*ny + j)*nx + i (x
 *     fastest), each component at its Yee location: Ex,Jx (i+1/2,j,k),
 *     Ey,Jy (i,j+1/2,k), Ez,Jz (i,j,k+1/2), Bx (i,j+1/2,k+1/2),
 *     By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k).
 *   - 2D3V runs use the (z, x) plane: dim = 2, ncell[1] = 1, box[1] = 1.
 *   - Calls on one handle are not thread-safe; distinct handles are
 *     independent.  Device work is issued on the handle's stream.
 */
#ifndef PIC_API_H
#define PIC_API_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = -1,       /* an argument is out of range or inconsistent       */
    PIC_ENOMEM = -2,       /* device or host allocation failed / does not fit   */
    PIC_ECUDA = -3,        /* a CUDA call failed (handle is then poisoned)      */
    PIC_ETIMEOUT = -4,     /* a bounded device-side wait ran out (poisoned)     */
    PIC_ESTATE = -5,       /* handle poisoned, or call made in the wrong state  */
    PIC_EUNSUPPORTED = -6  /* valid request that libpic does not support       */
} pic_status;

typedef struct pic_sim pic_sim; /* opaque, library-owned */

/* field component ids for pic_read_fields / pic_set_field */
enum {
    PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ,
    PIC_RHO = 9 /* charge density at the nodes (read only): particles + background */
};

/* Grid and decomposition (Sec. 2.1: the domain is cut into boxes, rectilinear
 * regions of cells; a box owns its cells and the particles inside it).
 *   dim          2 (2D3V, (z,x) plane) or 3.
 *   ncell        cells per direction (ncell[1] == 1 when dim == 2).
 *   box          cells per box per direction; must divide ncell.
 *   dx           cell sizes.
 *   dt           time step; <= 0 selects cfl * Courant limit
 *                (dt = cfl / sqrt(sum 1/dx_i^2) over the active directions).
 *   cfl          used only when dt <= 0.
 *   shape_order  1 (linear), 2 (quadratic) or 3 (cubic, the paper's choice in
 *                Sec. 3.1) B-spline particle shape.
 *   absorb_cells 0: periodic in every direction.  > 0: x and y periodic; at
 *                both z ends a damping layer of this many cells scales E and B
 *                each step, and particles entering it are removed.
 *   stream       cudaStream_t on which all device work is issued (NULL: the
 *                legacy default stream).  May be torch's current stream. */
typedef struct {
    int dim;
    int64_t ncell[3];
    int32_t box[3];
    double dx[3];
    double dt;
    double cfl;
    int shape_order;
    int absorb_cells;
    void* stream;
} pic_grid_desc;

/* Creates a simulation with zero fields and no particles on the current CUDA
 * device.  *out receives the handle.  Errors: PIC_EINVAL (bad description),
 * PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_init(const pic_grid_desc* desc, pic_sim** out);

/* Adds a species of macro-particles (Sec. 2.1: weighted markers moved by the
 * Lorentz force).  soa[0..6] = x, y, z, ux, uy, uz, w: np doubles each, where
 * u = gamma*v and w is the number of physical particles per marker.  y is
 * ignored in 2D (may be NULL).  ids: np int64 (NULL: 0..np-1).  All arrays are
 * host pointers (on_device = 0) or device pointers (on_device = 1); they are
 * copied.  Positions must lie in [0, L); with absorb_cells > 0, z must lie
 * outside the damping layers.
 * *species_id_out receives the species index.  Errors: PIC_EINVAL,
 * PIC_ENOMEM, PIC_ECUDA, PIC_ESTATE (after the first pic_step). */
pic_status pic_add_species(pic_sim* sim, double charge, double mass, int64_t np,
                           const double* const soa[7], const int64_t* ids, int on_device,
                           int* species_id_out);

/* Records a uniform neutralising background charge density rho0 (fixed ions).
 * It enters only PIC_RHO reads, never the current. */
pic_status pic_add_background(pic_sim* sim, double rho0);

/* Laser antenna: a soft sheet of Jx in the plane z = k_ant*dz (cell layer
 * k_ant), Jx = (2 a0 / dz) exp(-r^2/w0^2) exp(-((t-t_peak)/tau)^2)
 * sin(omega (t - t_peak)) at the current's time level t = (n+1/2) dt, with
 * r^2 = (x_{i+1/2} - xc)^2 + (y_j - yc)^2 (y term absent in 2D).  A sheet
 * current K radiates |E| = |K|/2 to each side, so the forward wave has
 * amplitude a0 (units m c omega0 / e with omega0 = 1).  The 2D Summit pulse of
 * Sec. 3.1 is the model.  One laser per simulation. */
typedef struct {
    double a0, w0, tau, t_peak, omega, xc, yc;
    int64_t k_ant;
} pic_laser_desc;
pic_status pic_add_laser(pic_sim* sim, const pic_laser_desc* laser);

/* Overwrites one E or B component (comp PIC_EX..PIC_BZ) with a dense array in
 * the layout given at the top of this file (host or device pointer). */
pic_status pic_set_field(pic_sim* sim, int comp, const double* data, int on_device);

/* Field gather kind.  PIC_GATHER_MOMENTUM (default): every component
 * interpolated at its own staggered location with the run's shape order in
 * every direction.  PIC_GATHER_ENERGY: the energy-conserving (Galerkin)
 * gather, one order lower along each direction in which the component sits
 * at half nodes (Ex along x, Bx along y and z, ...; order 0 is the nearest
 * half node), which makes the gather the transpose of the Esirkepov deposit.
 * The paper runs WarpX (Sec. 3), whose Yee-grid runs offer both; it does not
 * say which it used.  May be called at any time; takes effect from the next
 * step.  Synchronises the stream.  Errors: PIC_EINVAL (unknown kind). */
enum { PIC_GATHER_MOMENTUM = 0, PIC_GATHER_ENERGY = 1 };
pic_status pic_set_gather(pic_sim* sim, int kind);

/* Sets the step counter n (time t = n dt, which the laser antenna reads, and
 * the count that load-balancing intervals refer to), for resuming a run from
 * saved state: pic_init + pic_add_species with the saved arrays and ids +
 * pic_set_field for E and B + pic_set_step.  Synchronises.  Errors:
 * PIC_EINVAL (step < 0). */
pic_status pic_set_step(pic_sim* sim, int64_t step);

/* Self-test of the device-side bounded wait (every wait in the kernels is
 * bounded by %globaltimer so that a lost arrival cannot hang the GPU): one CTA
 * waits on an mbarrier that nothing arrives at, gives up after limit_ns
 * (1e3..5e9), records the error and returns.  Expected result: PIC_ETIMEOUT,
 * with the handle poisoned like after any device-side error (later calls
 * return PIC_ESTATE; pic_destroy still works and other handles are
 * unaffected).  Errors: PIC_EINVAL (limit out of range). */
pic_status pic_selftest_bounded_wait(pic_sim* sim, int64_t limit_ns);

/* ---- load balancing (Sec. 2.2) ------------------------------------------- */
enum { PIC_POLICY_KNAPSACK = 0, PIC_POLICY_SFC = 1, PIC_POLICY_BOX_ORDER = 2 };
enum { PIC_COST_HEURISTIC = 0, PIC_COST_DEVICE_CLOCK = 1, PIC_COST_KERNEL_TIME = 2 };
enum { PIC_LB_NONE = 0, PIC_LB_STATIC = 1, PIC_LB_DYNAMIC = 2 };
enum { PIC_SCHED_LISTS = 0, PIC_SCHED_QUEUE = 1 };

/* Parameters of the load-balancing routine (Sec. 2.2; scans in Sec. 3.3).
 *   mode        NONE: work in box order, boxes never split, mapping fixed;
 *               STATIC: balance once, at the first interval, threshold 0;
 *               DYNAMIC: balance every `interval` steps with threshold theta.
 *   interval    steps between load-balancing calls (Sec. 3.3 scans 1..300).
 *   theta       required relative improvement of E to adopt a new mapping
 *               (E_new >= (1 + theta) E_old; Sec. 3.2 uses 0.10).
 *   policy      knapsack or Morton space-filling curve (the paper's two
 *               policies, Sec. 2.2), or BOX_ORDER: a control without cost
 *               input -- the work units (boxes cut by cost as below) in
 *               box-index order, contiguous equal-count pieces per worker,
 *               pulled in that order by the queue schedule; it separates the
 *               gain of cutting heavy boxes from that of cost-driven order.
 *               pic_balance_compute accepts only the paper's two policies.
 *   cost        heuristic (w_p Np + w_c Nc per box), device clock (summed
 *               per-thread clock64 of the particle kernel, per box; the
 *               paper's GPU-clock strategy), or kernel time (summed
 *               %globaltimer span of the box's work units: the in-kernel
 *               analog of the paper's CUPTI kernel duration, without CUPTI).
 *   w_p, w_c    heuristic weights (Sec. 3.3 footnotes: 0.75/0.25 knapsack,
 *               0.02/0.98 SFC).
 *   cap_factor  knapsack cap on units per worker, times the average (1.5).
 *   n_workers   workers the mapping spreads over; 0 = one per persistent CTA.
 *   split       target work units per worker used to cut heavy boxes into
 *               several units (CTAs per box); 0 = library default.
 *   sched       LISTS: each persistent CTA runs its own worker's units;
 *               QUEUE: all CTAs pull units from one list in mapping order. */
typedef struct {
    int mode, interval;
    double theta;
    int policy, cost;
    double w_p, w_c, cap_factor;
    int n_workers, split, sched;
} pic_lb_params;

/* Result of one load-balancing call (the root's view in Sec. 2.2).
 *   e_old, e_new   Eq. 1 efficiencies of the current and proposed mappings
 *                  under the costs just measured.
 *   adopted        1 if the proposed mapping replaced the current one.
 *   n_units        work units in the proposed mapping.
 *   predicted_speedup  Sec. 4 model (1/e_old)^x with x = 0.88 (3D) / 0.91 (2D). */
typedef struct {
    double e_old, e_new;
    int adopted;
    int64_t n_units;
    double predicted_speedup;
    int64_t step; /* steps completed when the call ran */
} pic_lb_result;

/* Stores load-balancing parameters used by pic_step (default: mode NONE). */
pic_status pic_set_lb_params(pic_sim* sim, const pic_lb_params* params);

/* Advances nsteps PIC cycles (Sec. 2.1): field gather, relativistic Boris
 * push, Esirkepov current deposit with in-kernel per-box cost capture, Yee
 * field update, per-box re-sort of particles.  Device work is enqueued on the
 * stream; when the load-balancing interval falls inside the call, the routine
 * of Sec. 2.2 runs at that step (a device->host copy of costs, host mapping,
 * host->device copy of the new work list when adopted).  Errors: PIC_ESTATE,
 * PIC_ECUDA, PIC_ETIMEOUT. */
pic_status pic_step(pic_sim* sim, int nsteps);

/* Waits for the stream and reports any pending device-side error. */
pic_status pic_sync(pic_sim* sim);

/* Per-box cost (Sec. 2.2 strategies).  strategy HEURISTIC: w_p*Np + w_c*Nc
 * with the weights of the last pic_set_lb_params (0.75/0.25 by default);
 * DEVICE_CLOCK: summed thread clock cycles of the particle kernel since the
 * last rebalance (or since the start); KERNEL_TIME: summed nanoseconds
 * (%globaltimer) of the box's work units over the same window.  costs_out: host, nboxes doubles;
 * np_out: host, nboxes int64 particle counts (nullable).  Box index
 * (bz*nby + by)*nbx + bx.  Synchronises the stream. */
pic_status pic_get_box_costs(pic_sim* sim, int strategy, double* costs_out, int64_t* np_out);

/* Runs the load-balancing routine now (Sec. 2.2) with the given parameters
 * (mode NONE is treated as DYNAMIC for an explicit call) and fills *out
 * (nullable).  assign_out: host, nboxes int32 (nullable) receives the worker
 * of each box's first unit under the mapping in force after the call.
 * With cost HEURISTIC the call needs only the particle counts, so it may run
 * before the first step (a balanced start).  Resets the accumulated
 * device-clock costs.  Synchronises the stream. */
pic_status pic_rebalance(pic_sim* sim, const pic_lb_params* params, pic_lb_result* out,
                         int32_t* assign_out);

/* In-kernel cost capture (Sec. 2.2, the device-side measurement this work
 * is about): PIC_CAPTURE_CLOCK accumulates each thread's clock64() deltas
 * over its particle loop into the box's device-clock cost; PIC_CAPTURE_TIME
 * adds each work unit's %globaltimer span to the box's kernel-time cost.
 * Both are on by default.  A strategy whose capture is off reads zero costs
 * (and a load balancer driven by it then sees E = 1 and keeps its mapping);
 * the heuristic strategy needs neither.  Turning capture off measures its
 * overhead (the paper found CUPTI's about 2x).  Takes effect from the next
 * step; synchronises.  Errors: PIC_EINVAL (mask outside 0..3). */
enum { PIC_CAPTURE_CLOCK = 1, PIC_CAPTURE_TIME = 2 };
pic_status pic_set_cost_capture(pic_sim* sim, int mask);

/* E (Eq. 1, c_avg / c_max over workers) of the work-unit mapping in force,
 * with the per-box costs of the current cost window (strategy as in
 * pic_get_box_costs; a box's cost is divided evenly over its work units), as
 * Listing 1 evaluates the current distribution before it proposes a new one.
 * The cost window is the one pic_rebalance reads: it holds everything since
 * the last load-balancing call.  reset_window != 0 starts a new window after
 * the read (the next internal load-balancing call then sees only the steps
 * after it).  Synchronises.  Errors: PIC_EINVAL. */
pic_status pic_get_efficiency(pic_sim* sim, int strategy, int reset_window, double* e_out);

/* Log of the load-balancing calls made so far (by pic_step at its intervals
 * and by pic_rebalance), oldest first: copies min(max, n_total) entries into
 * out (host, nullable when max == 0) and the total count into *n_total. */
pic_status pic_get_lb_log(pic_sim* sim, pic_lb_result* out, int64_t max, int64_t* n_total);

/* Pure host function, the bit-exact test surface of the balancer (Sec. 2.2):
 * maps nboxes boxes with the given costs to n_workers workers.
 *   costs      host, nboxes doubles (>= 0).
 *   box_ijk    host, 3*nboxes int32 box coordinates (bx, by, bz); used by SFC
 *              (Morton key interleaving x, y, z bits from the least
 *              significant end; in 2D, x and z).  May be NULL for knapsack.
 *   policy     PIC_POLICY_KNAPSACK: greedy longest-processing-time-first,
 *              boxes by cost descending (ties: lower index), each to the
 *              least-loaded worker below the cap (ties: lowest id); cap =
 *              max(ceil(nboxes/n), floor(cap_factor*nboxes/n)).
 *              PIC_POLICY_SFC: boxes in Morton order cut into contiguous
 *              pieces; the worker index advances after the box whose running
 *              cost reaches the next multiple of total/n.
 *   assign_out host, nboxes int32.
 *   e_out      host, nullable: Eq. 1 efficiency of the result.
 * Errors: PIC_EINVAL. */
pic_status pic_balance_compute(const double* costs, int64_t nboxes, const int32_t* box_ijk,
                               int dim, int n_workers, int policy, double cap_factor,
                               int32_t* assign_out, double* e_out);

/* Eq. 1 for a given mapping: E = (sum of worker costs / n_workers) / max
 * worker cost, worker cost summed over its boxes in ascending box index; 1 when
 * all workers are idle.  Host pointers. */
pic_status pic_lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes,
                             int n_workers, double* e_out);

/* Copies one field component (PIC_EX..PIC_JZ, PIC_RHO) into out: host or
 * device buffer of ncell[0]*ncell[1]*ncell[2] doubles (layout above).  J is
 * the current of the last step (J^{n+1/2}).  Synchronises the stream. */
pic_status pic_read_fields(pic_sim* sim, int comp, double* out, int on_device);

/* Current number of macro-particles of a species (synchronises). */
pic_status pic_num_particles(pic_sim* sim, int species, int64_t* np_out);

/* Copies a species' particles: soa_out[0..6] = x, y, z, ux, uy, uz, w, each
 * room for pic_num_particles doubles (an entry may be NULL to skip it), and
 * id_out (nullable).  Particles come in the library's internal order (sorted
 * by box); match them by id.  Host or device buffers.  Synchronises. */
pic_status pic_read_particles(pic_sim* sim, int species, double* const soa_out[7],
                              int64_t* id_out, int on_device);

/* Bins caller-owned particles by box (Sec. 2.1: a box owns the particles
 * inside it; Sec. 2.2 moves particles with their box when the mapping
 * changes).  A particle's box is floor(x/dx) wrapped into [0, ncell) divided
 * by the box extent, per direction; box index (bz*nby + by)*nbx + bx.
 *   grid         geometry only: dim, ncell, box, dx; stream (NULL: legacy
 *                default stream).  Other fields are ignored.
 *   x, y, z      device, np doubles each (y unused and may be NULL in 2D).
 *   np           0 <= np < 2^31.
 *   box_off_out  device, nboxes+1 int64: exclusive prefix of the per-box
 *                counts (box b holds perm_out[box_off_out[b] .. box_off_out[b+1])).
 *   perm_out     device, np int64: particle indices grouped by box; the order
 *                inside a box is unspecified.
 * Asynchronous on the stream; per-box cursors are allocated stream-ordered
 * (cudaMallocAsync) and freed before return.  Errors: PIC_EINVAL, PIC_ENOMEM,
 * PIC_ECUDA (message in pic_last_error(NULL)). */
pic_status pic_bin_particles(const pic_grid_desc* grid, const double* x, const double* y,
                             const double* z, int64_t np, int64_t* box_off_out, int64_t* perm_out);

/* Launch configuration of the persistent particle kernel and the work
 * splitting (the autotuner's knobs).  Any field <= 0 keeps its value.
 *   threads       threads per CTA (a multiple of 32, at most 256).
 *   ctas_per_sm   persistent CTAs per SM (1 or 2; 2 selects the kernel
 *                 variant compiled for 128 registers; capped by occupancy).
 *   split         target work units per worker when boxes are cut (the
 *                 number of CTAs that share a heavy box).
 *   tile          cells per tile edge in every active direction: the unit of
 *                 field staging (a guard-extended E/B tile per tile in shared
 *                 memory) and of the particle sort.  Even, dividing every box
 *                 extent, at least 4, and small enough for its staged tile to
 *                 fit in shared memory.  The default is the largest even
 *                 divisor of the box up to 8 (3D) or 16 (2D).  A change
 *                 re-tiles the simulation: tile maps, sort arrays and every
 *                 species' order are rebuilt (synchronises).
 *   ppt           particles per thread per loop iteration (1 or 2): the HBM
 *                 loads of that many particles are issued before the first
 *                 of them is pushed.
 *   precision     arithmetic of the particle push: 1 FP64 (default);
 *                 2 float-float (pairs of FP32 with error-free
 *                 transformations, ~48-bit significand) for gather, Boris and
 *                 deposit weights, with FP64 storage, positions, index math and
 *                 current accumulation -- the mixed-precision variant; 3 FP32
 *                 for gather, Boris and deposit weights with FP64 storage,
 *                 positions and current accumulation (the FP32 variant:
 *                 about 2^-24 per operation, so it meets an FP32-derived
 *                 tolerance, not the FP64 one); 0 keeps the current
 *                 setting.  The autotuner
 *                 never changes it. */
typedef struct {
    int threads, ctas_per_sm, split, precision, tile, ppt;
} pic_launch_cfg;
pic_status pic_set_launch(pic_sim* sim, const pic_launch_cfg* cfg);
pic_status pic_get_launch(const pic_sim* sim, pic_launch_cfg* cfg);

/* Autotuner: times candidate launch configurations on real steps of this
 * simulation (steps_per_candidate steps each, after one warm-up step; the
 * steps advance the simulation) and keeps the fastest.  The search runs by
 * coordinates, each stage keeping the best of the previous ones: tile size
 * (the even divisors of the box from 4 up to 8 in 3D, 32 in 2D, that fit in
 * shared memory) x particles per thread {1, 2}; then threads per CTA
 * {128, 256} x CTAs per SM {1, 2}; then work units per worker {4, 16, 64}
 * (only when load balancing cuts boxes).  The precision is never changed.
 * *best receives the result (nullable).  Synchronises. */
pic_status pic_autotune(pic_sim* sim, int steps_per_candidate, pic_launch_cfg* best);

/* Timing of the last pic_step call, from CUDA events recorded on the
 * simulation's stream around each launch (enabled by pic_set_profiling):
 * milliseconds summed over the call's steps per phase, and launches. */
typedef struct {
    double ms_particle, ms_fields, ms_sort, ms_total;
    int64_t steps, launches, particle_launches;
    int64_t particles_pushed; /* particle updates in those steps */
} pic_stats;
pic_status pic_set_profiling(pic_sim* sim, int on);
pic_status pic_get_stats(pic_sim* sim, pic_stats* out);

/* Measures the FP64 fused multiply-add throughput of the current device, the
 * denominator of the FP64 roofline of the particle kernel (GB300 executes
 * FP64 at a small fraction of its FP32 rate, so the FP64 push is bound by this
 * pipe rather than by HBM).  The paper has no counterpart: it reports no
 * per-kernel rates.  Every SM runs 8 CTAs of 256 threads, each thread 8
 * independent DFMA chains of `iters` iterations (1 <= iters <= 10^7); one
 * warm-up launch, then the best of three launches timed with CUDA events on
 * a private stream.  *tflops_out = 2 x 8 x iters x threads / seconds / 10^12.
 * Allocates and frees a small device buffer.  Errors: PIC_EINVAL, PIC_ECUDA
 * (message in pic_last_error(NULL)). */
pic_status pic_probe_fp64_fma(int64_t iters, double* tflops_out);

/* Releases all resources of the handle (also valid on a poisoned handle). */
pic_status pic_destroy(pic_sim* sim);

/* One-line description of the last error on the handle (never NULL).  With
 * sim == NULL, the last error of a call that had no handle (pic_init, the pure
 * balancer functions). */
const char* pic_last_error(const pic_sim* sim);

#ifdef __cplusplus
}
#endif
#endif
