// pic_internal.h -- device-side data layout of libpic (shared by the .cu files
// of the library only; the CPU oracle never includes it).
//
// HBM layout of one simulation:
//   fields  9 FP64 arrays (Ex Ey Ez Bx By Bz Jx Jy Jz), each padded by guard
//           cells in every active direction (3 per side in x, 4 for cubic
//           shapes; 2 in y and z, 3 for quadratic and cubic): linear shapes
//           give dims (nx+6, ny+4, nz+4), x fastest (ny+4 -> 1 in 2D).  Guards
//           of E and B hold the periodic images after every step, so a tile
//           plus its halo is one rectangular TMA box; J guards collect the
//           current the particle kernel deposits beyond the domain, which the
//           fold kernel adds to the periodic images.  J is one contiguous
//           block of 3 arrays.
//   particles per species, SoA of FP64 X Y Z (global cell units, X = x/dx),
//           ux uy uz (u = gamma v), w, plus int64 id; double-buffered, sorted
//           by tile (tiles numbered box-major, so each box is contiguous).
//   sort    per species: key[cap] (tile of the new position), count and
//           cursor[ntiles+1], off[ntiles+2] (exclusive scan of count).
//   costs   uint64 cost_clock[nboxes] (summed thread clocks), per simulation.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pic_api.h"

#define PIC_G 2        // guard cells per side in y and z of the padded field arrays (+1 for order >= 2)
#define PIC_GX 3       // guard cells per side in x (4 for cubic shapes): a tile's TMA box
                       // starts 1 cell (2 for cubic) below an even tile origin and must
                       // start at an even padded x (x * 8 bytes a multiple of 16)
#define PIC_MAXSP 4    // species per simulation
#define PIC_NCOMP 9

// error codes written by kernels into the device error word
#define PIC_DERR_TMA_TIMEOUT 1
#define PIC_DERR_BOUNDS 2
#define PIC_DERR_SCATTER 4
#define PIC_DERR_WAIT_TIMEOUT 8  // the bounded-wait self-test ran out (as it should)

struct SpeciesDev {
    double q, m;
    double kq;            // q dt / (2 m): half electric kick factor
    double qw_scale;      // q / (dV dt)-style deposit prefactor (per simulation dims)
    double* cur[7];       // X Y Z ux uy uz w  (current, tile-sorted)
    double* alt[7];       // scatter target
    int64_t* id;
    int64_t* id_alt;
    int32_t* key;         // [cap]
    int32_t* count;       // [ntiles+1]
    int32_t* cursor;      // [ntiles+1]
    int64_t* off;         // [ntiles+2]; off[ntiles] = particles kept
    int64_t* np_prev;     // particles in the buffer being scattered
    int64_t cap;
};

struct LaserDev {
    int on;
    int k_ant;
    double a0, w0, tau, t_peak, omega, xc, yc;
};

struct SimDev {
    CUtensorMap tmap[6];  // TMA descriptors of the padded E,B arrays (must stay first)
    int dim, order, nsp, absorb;
    int ec;               // 1: energy-conserving gather (order - 1 along staggered directions)
    int capture;          // in-kernel cost capture: bit 0 clock64 (cost_clock), bit 1 %globaltimer (cost_time)
    int n[3];             // cells per direction
    int pn[3];            // padded extents (n + 2G; 1 for an inactive y)
    int g[3];             // guard width per direction (G or 0)
    int T[3];             // tile extents in cells (T[1] = 1 in 2D)
    int tpb[3];           // tiles per box per direction
    int nb[3];            // boxes per direction
    int bsz[3];           // box extents in cells
    int tiles_per_box, nboxes, ntiles;
    int ebs[3];           // E/B shared tile extents (x padded to even for TMA)
    int jlo;              // a tile's J view starts jlo cells below the tile origin
    double d[3];          // cell sizes
    double nd[3];         // n as doubles (periodic wrap of positions)
    double invd[3];       // 1 / d (0 for the inactive y of 2D runs)
    double dt;
    double dtd[3];        // dt / d
    double jfac[3];       // -1/(dA_perp dt) for the prefix currents (3D); 2D see kernel
    double jyfac2d;       // 1/(dx dz) for the 2D out-of-plane current
    double* F[PIC_NCOMP]; // padded field arrays
    uint64_t* cost_clock; // [nboxes] summed thread clock64 cycles (device-clock cost)
    uint64_t* cost_time;  // [nboxes] summed %globaltimer ns of the box's units (kernel-time cost)
    int64_t* step;        // device step counter
    int32_t* err;         // device error word (shared with the schedule)
    int64_t* scan_part;   // [scan_part_cap] block sums of the multi-block histogram scan
    int64_t scan_part_cap;
    const int32_t* owner; // box sharding: rank owning each box (nullptr: every box is this rank's)
    int rank;             // this simulation's rank when sharded
    LaserDev las;
    SpeciesDev sp[PIC_MAXSP];
};

struct UnitDev {
    int32_t sim, box, chunk, nchunks;
};

struct SchedDev {
    UnitDev* units;       // [cap_units]
    int32_t* list_off;    // [nlists+1] start of each list in units
    int32_t* head;        // [nlists] atomic pull counters
    int32_t* meta;        // [0] = nlists, [1] = steal (0/1)
    int32_t* err;         // device error word
    double* rings;        // [PIC_RING_CTAS_PER_SM x SMs x 8 warps x PIC_RING_DOUBLES] rings of
                          // cell-crossing particles in global memory (FP64, float-float)
};

// global ring scratch: per warp 7 fields x 64 slots of doubles, for up to 4
// persistent CTAs per SM of up to 8 warps
#define PIC_RING_DOUBLES (7 * 64)
#define PIC_RING_CTAS_PER_SM 4
__host__ inline size_t pic_ring_bytes(int nsm) {
    return (size_t)nsm * PIC_RING_CTAS_PER_SM * 8 * PIC_RING_DOUBLES * sizeof(double);
}

// padded linear index of interior cell (i,j,k) of a simulation
__host__ __device__ inline int64_t pidx(const SimDev& s, int i, int j, int k) {
    return ((int64_t)(k + s.g[2]) * s.pn[1] + (j + s.g[1])) * s.pn[0] + (i + s.g[0]);
}

// whether interior cell (i,j,k) lies in a box this simulation owns (always
// when it is not sharded)
__host__ __device__ inline bool cell_owned(const SimDev& s, int i, int j, int k) {
    if (!s.owner) return true;
    const int b = ((k / s.bsz[2]) * s.nb[1] + (j / s.bsz[1])) * s.nb[0] + (i / s.bsz[0]);
    return s.owner[b] == s.rank;
}

// streaming multiprocessors of the current device, queried once per device
// (pic_particles.cu): grid-stride launches cap their grids at a multiple of it
int pic_sm_count();

// ---- kernel launchers (defined in the .cu files) ----
struct LaunchCfg {
    int threads;
    int ctas;
    int minb;     // register budget variant of the particle kernel: 1 or 2 CTAs per SM
    int prec;     // arithmetic of the particle push: 0 FP64, 1 float-float, 2 FP32
    int ppt = 1;  // particles per thread per loop iteration (1 or 2)
};
// dynamic shared memory of the particle kernel; prec 0 FP64, 1 float-float, 2 FP32
size_t pic_particle_smem_bytes(int dim, int order, const int T[3], int threads, int prec);
cudaError_t pic_prepare_particles(int dim, int order, size_t smem);  // outside graph capture
int pic_particle_occupancy(int dim, int order, int minb, int ppt, int threads, size_t smem,
                           int prec);  // resident CTAs per SM
// per-precision, per-dimensionality instantiations (pic_particles_<prec>_<dim>d.cu);
// the dispatchers below (pic_particles.cu) pick one by precision and dim
#define PIC_DECLARE_PARTICLE_TU(SUF)                                                                     \
    cudaError_t pic_launch_particles_##SUF(int order, const LaunchCfg& cfg, size_t smem,                 \
                                           const SchedDev* sched, SimDev* sims, cudaStream_t st);        \
    cudaError_t pic_prepare_particles_##SUF(int order, size_t smem);                                      \
    int pic_particle_occupancy_##SUF(int order, int minb, int ppt, int threads, size_t smem);
PIC_DECLARE_PARTICLE_TU(p0_d3)
PIC_DECLARE_PARTICLE_TU(p0_d2)
PIC_DECLARE_PARTICLE_TU(p1_d3)
PIC_DECLARE_PARTICLE_TU(p1_d2)
PIC_DECLARE_PARTICLE_TU(p2_d3)
PIC_DECLARE_PARTICLE_TU(p2_d2)
// self-test of the device's bounded wait: one CTA waits on an mbarrier that
// nothing arrives at; after limit_ns it sets PIC_DERR_WAIT_TIMEOUT in *err
cudaError_t pic_launch_selftest_wait(int32_t* err, uint64_t limit_ns, cudaStream_t st);
cudaError_t pic_launch_particles(int dim, int order, const LaunchCfg& cfg, size_t smem,
                                 const SchedDev* sched, SimDev* sims, cudaStream_t st);
cudaError_t pic_launch_fields(const SimDev* dsim, const SimDev& hsim, cudaStream_t st);
cudaError_t pic_launch_sort(const SimDev* dsim, const SimDev& hsim, int sp, cudaStream_t st);
cudaError_t pic_launch_initial_keys(const SimDev* dsim, const SimDev& hsim, int sp,
                                    int64_t np, cudaStream_t st);
cudaError_t pic_launch_finish(SimDev* dsim, const SchedDev* sched, cudaStream_t st);
cudaError_t pic_launch_box_counts(const SimDev* dsim, const SimDev& hsim, int64_t* out,
                                  cudaStream_t st);
cudaError_t pic_launch_rho(const SimDev* dsim, const SimDev& hsim, double* rho, double rho0,
                           cudaStream_t st);
cudaError_t pic_launch_unpad(const double* padded, double* dense, const SimDev& hsim,
                             cudaStream_t st);
cudaError_t pic_launch_pad(const double* dense, double* padded, const SimDev& hsim,
                           cudaStream_t st);
cudaError_t pic_launch_guards(const SimDev* dsim, const SimDev& hsim, int first_comp,
                              int ncomp, cudaStream_t st);
// the field update in its sub-steps, for sharded runs that exchange ghost
// cells between them: 0 B half step, 1 E step (with J and the antenna),
// 2 B half step and damping layers, 3 periodic guard fill; and the fold of
// guard-cell current into the domain
cudaError_t pic_launch_field_stage(const SimDev* dsim, const SimDev& hsim, int stage, cudaStream_t st);
cudaError_t pic_launch_fold(const SimDev* dsim, const SimDev& hsim, cudaStream_t st);
// keys and histogram of particles [p0, p1) of species sp from their positions
cudaError_t pic_launch_keys_range(const SimDev* dsim, const SimDev& hsim, int sp, int64_t p0, int64_t p1,
                                  cudaStream_t st);
// multi-simulation launches over a device list of slots (blockIdx.y = slot)
cudaError_t pic_launch_fields_multi(const SimDev* sims, const int* slots, int nslots, int dim,
                                    int64_t max_cells, int64_t max_padded, bool any_absorb,
                                    cudaStream_t st);
cudaError_t pic_launch_zero_j_multi(const SimDev* sims, const int* slots, int nslots,
                                    int64_t max_padded, cudaStream_t st);
cudaError_t pic_launch_sort_multi(SimDev* sims, const int* slots, int nslots, int dim, int64_t max_cap,
                                  cudaStream_t st);
cudaError_t pic_launch_finish_multi(SimDev* sims, const int* slots, int nslots, const SchedDev* sched,
                                    cudaStream_t st);
// dst[j] = src[(j * (2^31 + 11)) mod np] for the 7 SoA arrays (array `skip`
// left alone, -1 for none) and the ids: the one-time input-order scramble
cudaError_t pic_launch_permute(double* const dst[7], const double* const src[7], int64_t* id_dst,
                               const int64_t* id_src, int64_t np, int skip, cudaStream_t st);
cudaError_t pic_launch_to_cells(double* p, int64_t np, double d, int n, cudaStream_t st);
cudaError_t pic_launch_from_cells(const double* src, double* dst, int64_t np, double d,
                                  cudaStream_t st);

// hooks of pic_api.cu used by the request server (not part of the C ABI)
int64_t pic_internal_bytes(const pic_sim* s);
pic_status pic_internal_mirror(pic_sim* s, SimDev* out);
SimDev* pic_internal_device_sim(pic_sim* s);
void pic_internal_mark_external(pic_sim* s);
// records the message returned by pic_last_error(NULL) on this thread
pic_status pic_record_error(pic_status st, const char* msg);
int64_t pic_internal_estimate_bytes(const pic_grid_desc* g, const int64_t* np, int nsp);
const char* pic_internal_error(const pic_sim* s);
