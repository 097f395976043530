/*
 * pic_shard.h -- box sharding of one simulation across several ranks (GPUs),
 * the setting of arXiv 2104.11385: Sec. 2.1 distributes the boxes of the
 * domain among MPI ranks, each rank owning the fields and the particles of
 * its boxes, with guard cells exchanged between neighbouring boxes; Sec. 2.2
 * (Listing 1) gathers the per-box costs to the root at load-balancing steps,
 * computes the new box-to-rank mapping, and redistributes boxes and
 * particles when it is adopted.
 *
 * Here a rank is one pic_sim handle (normally one per GPU).  Every rank
 * allocates the full-size field arrays (HBM is large enough), but fields are
 * valid only on the boxes it owns plus a ghost layer around them, and it
 * holds only the particles of its own boxes.  The host drives one step as
 *
 *   pic_shard_push              particles of own boxes -> local J (incl. ghosts)
 *   J ghost sum                 each rank adds the J other ranks deposited in its boxes
 *   pic_shard_field_stage 0     B half step on own boxes
 *   B ghost exchange
 *   pic_shard_field_stage 1     E step on own boxes
 *   E ghost exchange
 *   pic_shard_field_stage 2     B half step + damping layers on own boxes
 *   E and B ghost exchange
 *   pic_shard_field_stage 3     periodic guard fill
 *   migration                   pic_shard_take_leaving / pic_shard_read_leaving
 *                               on the sender, pic_shard_add_arriving on the owner
 *   pic_shard_finish            per-tile re-sort, step counter
 *
 * with the exchanges moving packed cell lists (pic_shard_halo_cells,
 * pic_shard_pack, pic_shard_unpack) by any transport (peer copies, NCCL).
 * The physics equals the unsharded step up to the order of floating-point
 * sums.  Conventions of pic_api.h apply (status codes, pic_last_error,
 * poisoned handles).  Cell indices are dense interior indices
 * (k*ny + j)*nx + i.  Particle records exchanged between ranks are in the
 * library's internal units (positions in cells, x/dx) and are only meant to
 * be handed to another rank of the same geometry.
 */
#ifndef PIC_SHARD_H
#define PIC_SHARD_H
#include <stdint.h>

#include "pic_api.h"
#ifdef __cplusplus
extern "C" {
#endif

/* Pure host function (Sec. 2.1 guard cells): the cells of the boxes owned by
 * rank `own` (owner[b] == own) that lie within `halo` cells, periodically, of
 * a box owned by rank `near`; ascending, each once.
 *   grid       geometry only (dim, ncell, box); every active box extent must
 *              be at least `halo`.
 *   owner      host, nboxes int32 ranks (>= 0), box index (bz*nby + by)*nbx + bx.
 *   halo       1..8.
 *   cells_out  host, room for the count (nullable: count only).
 *   n_out      receives the count.
 * J ghost sum: rank `near` sends its J at halo_cells(own = dst, near = src)
 * to rank `own`, which adds it.  E/B ghosts: rank `own` sends its E/B at
 * halo_cells(own = src, near = dst) to rank `near`, which stores it.
 * Errors: PIC_EINVAL. */
pic_status pic_shard_halo_cells(const pic_grid_desc* grid, const int32_t* owner, int own, int near, int halo,
                                int64_t* cells_out, int64_t* n_out);

/* Pure host function (Sec. 2.2 redistribution): the cells of the boxes whose
 * owner changes from rank `src` (old_owner) to rank `dst` (new_owner),
 * ascending.  Arguments as for pic_shard_halo_cells.  Errors: PIC_EINVAL. */
pic_status pic_shard_moved_cells(const pic_grid_desc* grid, const int32_t* old_owner, const int32_t* new_owner,
                                 int src, int dst, int64_t* cells_out, int64_t* n_out);

/* Makes the handle rank `rank` of a sharded run with the given box owners
 * (host, nboxes int32, copied).  From then on the field sub-steps update only
 * the cells of its boxes, and pic_shard_take_leaving sets aside particles
 * whose box another rank owns.  May be called again with a new mapping (a
 * redistribution, Sec. 2.2).  Synchronises.  Errors: PIC_EINVAL, PIC_ENOMEM. */
pic_status pic_shard_set_owner(pic_sim* sim, const int32_t* owner, int rank);

/* Gathers components [first_comp, first_comp + ncomp) (PIC_EX..PIC_JZ) at n
 * cells (device, int64 dense indices) into buf (device, ncomp * n doubles,
 * component-major).  Synchronises.  Errors: PIC_EINVAL, PIC_ECUDA. */
pic_status pic_shard_pack(pic_sim* sim, int first_comp, int ncomp, const int64_t* cells, int64_t n, double* buf);

/* Scatters buf (as produced by pic_shard_pack on another rank) back into the
 * same components at the same cells: stores (add = 0: E/B ghosts, moved
 * boxes) or adds (add = 1: the J ghost sum).  The cells of one call must be
 * distinct.  Synchronises.  Errors: PIC_EINVAL, PIC_ECUDA. */
pic_status pic_shard_unpack(pic_sim* sim, int first_comp, int ncomp, const int64_t* cells, int64_t n,
                            const double* buf, int add);

/* The particle half of a step on this rank's particles: J reset, the
 * persistent gather / Boris / Esirkepov kernel with its in-situ costs, and the
 * fold of guard-cell current into the domain.  Asynchronous on the stream.
 * Errors: PIC_ESTATE (not sharded), PIC_ECUDA. */
pic_status pic_shard_push(pic_sim* sim);

/* One field sub-step on this rank's boxes: 0 B half step, 1 E step with J and
 * the antenna, 2 B half step and damping layers, 3 periodic guard fill (all
 * cells).  Asynchronous.  Errors: PIC_EINVAL, PIC_ESTATE, PIC_ECUDA. */
pic_status pic_shard_field_stage(pic_sim* sim, int stage);

/* Re-derives every particle's tile from its position, as a push does, so that
 * pic_shard_take_leaving can route particles after a change of owners
 * outside a step.  Errors: PIC_ESTATE, PIC_ECUDA. */
pic_status pic_shard_rekey(pic_sim* sim);

/* Sets aside the particles of `species` whose new box belongs to another
 * rank (after pic_shard_push or pic_shard_rekey): they leave the rank's sort
 * and are copied into the handle's outbox, grouped by destination.
 * counts_out: host, nranks int64 (room for every rank in the owner map).
 * Synchronises.  Errors: PIC_EINVAL, PIC_ESTATE, PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_shard_take_leaving(pic_sim* sim, int species, int nranks, int64_t* counts_out);

/* Copies the outbox group of destination `dst` (from the last
 * pic_shard_take_leaving of `species`): soa_out[0..6] device buffers of
 * counts_out[dst] doubles (X, Y, Z in cells, ux, uy, uz, w), ids_out device
 * int64.  Synchronises.  Errors: PIC_EINVAL, PIC_ESTATE, PIC_ECUDA. */
pic_status pic_shard_read_leaving(pic_sim* sim, int species, int dst, double* const soa_out[7], int64_t* ids_out);

/* Appends n particle records (device, as read by pic_shard_read_leaving on
 * another rank) to `species`; they join the next pic_shard_finish sort.
 * Grows the species' buffers when needed.  Synchronises.  Errors:
 * PIC_EINVAL, PIC_ESTATE, PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_shard_add_arriving(pic_sim* sim, int species, int64_t n, const double* const soa[7],
                                  const int64_t* ids);

/* The end of a step: per-tile re-sort of every species (kept and arrived
 * particles) and, with advance = 1, the step counter (advance = 0 after a
 * redistribution outside a step).  Synchronises and reports device errors.
 * Errors: PIC_ESTATE, PIC_ECUDA, PIC_ETIMEOUT. */
pic_status pic_shard_finish(pic_sim* sim, int advance);

#ifdef __cplusplus
}
#endif
#endif
