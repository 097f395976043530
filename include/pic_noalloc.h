/*
 * pic_noalloc.h -- allocation-free entry point of libpic.
 *
 * The paper has no counterpart to this call: it is a service for callers that
 * cannot let a library allocate device memory.  Examples are code that issues
 * work while a CUDA stream capture is open (a cudaMalloc there is illegal in
 * the global capture mode and is not recorded in the graph), frameworks that
 * hand out all device memory from their own pool and forbid foreign
 * allocations, and tight loops that must never reach the allocator.
 */
#ifndef PIC_NOALLOC_H
#define PIC_NOALLOC_H
#include "pic_api.h"
#ifdef __cplusplus
extern "C" {
#endif

/* Largest box count pic_bin_particles_noalloc accepts: its per-box cursors
 * live in a fixed device array of this many int32 (4 MiB), which every GPU
 * that loads libpic holds until the process exits. */
#define PIC_BIN_NOALLOC_MAX_BOXES (1 << 20)

/* Same arguments, outputs and guarantees as pic_bin_particles (include/
 * pic_api.h), but the call allocates nothing: no cudaMalloc, cudaMallocAsync,
 * cudaFree or allocating library routine.  The caller passes the inputs
 * (x, y, z) and the outputs (box_off_out, perm_out); the only scratch, one
 * int32 cursor per box, is a fixed array compiled into the library.
 *   - Boxes beyond PIC_BIN_NOALLOC_MAX_BOXES are rejected with PIC_EINVAL and a
 *     message in pic_last_error(NULL); nothing is launched.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.  The address is kept per device and
 *     CUDA context: after a device reset (cudaDeviceReset) the next call looks
 *     it up again, so that call too belongs outside a capture.  Later calls
 *     issue only a memset and kernel launches on grid->stream and can be
 *     captured into a CUDA graph (global capture mode) and replayed.
 *   - Every call, on every stream, shares the one array, and it keeps the last
 *     call's contents; each call zeroes the part it uses on its stream first.
 *     Calls whose device work overlaps (different streams, or host threads
 *     racing) therefore race on the cursors and give wrong results: order
 *     them on one stream or synchronise between them.
 * Errors: PIC_EINVAL, PIC_ECUDA. */
pic_status pic_bin_particles_noalloc(const pic_grid_desc* grid, const double* x, const double* y,
                                     const double* z, int64_t np, int64_t* box_off_out,
                                     int64_t* perm_out);

#ifdef __cplusplus
}
#endif
#endif
