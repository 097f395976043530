/*
 * pic_oracle.h -- plain, slow, FP64 CPU reference ("oracle") for the per-box
 * particle-in-cell step and the load-balancing routine of
 *   Rowan et al., "In-Situ Assessment of Device-Side Compute Work for Dynamic
 *   Load Balancing in a GPU-Accelerated PIC Code" (arXiv 2104.11385).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this code; the tests, the smoke check and the CPU-baseline leg of
 * the benchmark are its only users.  It shares no code with the CUDA path.
 *
 * What it computes (each function cites the passage it follows):
 *   - the explicit PIC cycle of Sec. 2.1 (Maxwell on cells, Lorentz push of
 *     weighted markers, deposited currents), with the schemes the paper leaves
 *     open fixed as: Yee staggering, relativistic Boris push, Esirkepov
 *     charge-conserving deposit, B-spline shapes of order 1, 2 or 3 (the
 *     paper's runs use order 3, Sec. 3.1), gathered with the same order in
 *     every direction or, energy-conserving, one order lower along each
 *     component's staggered directions;
 *   - the load-balance efficiency E = c_avg / c_max (Sec. 2.2, Eq. 1), the
 *     knapsack and Morton space-filling-curve policies (Sec. 2.2), the
 *     improvement threshold (Sec. 2.2, Sec. 3.2) and the performance model
 *     S = (1/E0)^x (Sec. 4, Eq. 2).
 *
 * Units: normalised, c = eps0 = mu0 = 1.  Fields are periodic arrays of
 * n[0]*n[1]*n[2] cells, flat index (k*ny + j)*nx + i, x fastest.  2D3V runs
 * use the (z, x) plane: dim = 2, n[1] = 1, d/dy = 0.
 *
 * Build: gcc -O2 -ffp-contract=off (no FMA contraction, IEEE round-to-nearest).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

/* field component ids: E (0..2), B (3..5), J (6..8) */
enum { ORC_EX = 0, ORC_EY, ORC_EZ, ORC_BX, ORC_BY, ORC_BZ, ORC_JX, ORC_JY, ORC_JZ };

/* dim: 2 or 3; n: cells (nx, ny, nz) with ny == 1 when dim == 2;
 * d: cell sizes; dt: time step; order: shape order 1, 2 or 3;
 * absorb_cells: 0 = fully periodic; > 0 = width (in z cells) of the damping
 * layers at both z ends, where particles are removed.  Returns NULL on bad input.
 * The layers' damping profile, 1 - (p/absorb)^2 / 2 per step at depth p, is a
 * reading of this project (the paper fixes no field boundary): parity
 * unpinned beyond the tests that the layers absorb an outgoing pulse and
 * remove the particles that enter them. */
orc_sim* orc_create(int dim, const int64_t n[3], const double d[3], double dt,
                    int order, int absorb_cells);
void orc_destroy(orc_sim* s);

/* adds a species; the arrays are copied.  y is ignored when dim == 2. */
int orc_add_species(orc_sim* s, double q, double m, int64_t np,
                    const double* x, const double* y, const double* z,
                    const double* ux, const double* uy, const double* uz,
                    const double* w, const int64_t* id);

/* laser antenna (soft current sheet in the plane k = k_ant). */
int orc_set_laser(orc_sim* s, double a0, double w0, double tau, double t_peak,
                  double omega, double xc, double yc, int64_t k_ant);

/* field gather: 0 = the run's order in every direction (default); 1 =
 * energy-conserving: order - 1 along each direction in which the component
 * is staggered (Ex along x, Bx along y and z, ...), order-0 being the box
 * shape on the nearest half node. */
int orc_set_gather(orc_sim* s, int energy_conserving);

int orc_set_field(orc_sim* s, int comp, const double* data);
int orc_get_field(const orc_sim* s, int comp, double* out);
int64_t orc_num_particles(const orc_sim* s, int species);
int orc_get_particles(const orc_sim* s, int species, double* x, double* y, double* z,
                      double* ux, double* uy, double* uz, double* w, int64_t* id);
int64_t orc_step_count(const orc_sim* s);

/* advances nsteps full PIC cycles. */
int orc_step(orc_sim* s, int nsteps);

/* diagnostics: charge density of all species at the nodes, shape S of the
 * run's order (used by the continuity and Gauss checks). */
int orc_deposit_rho(const orc_sim* s, double* rho_out);
/* particle count per box; boxes of bsize cells, box index (bz*nby+by)*nbx+bx. */
int orc_box_counts(const orc_sim* s, const int64_t bsize[3], int64_t* counts_out);

/* box binning of a particle set (Sec. 2.1: a box owns the particles inside
 * it): box of a particle = floor(x/d) wrapped into [0, n), divided by the box
 * extent; box index (bz*nby + by)*nbx + bx.  box_off_out: nboxes+1 exclusive
 * prefix of the per-box counts; perm_out: particle indices in box order, in
 * ascending original index inside a box (stable). */
int orc_bin_particles(int dim, const int64_t n[3], const double d[3], const int64_t bsize[3],
                      const double* x, const double* y, const double* z, int64_t np,
                      int64_t* box_off_out, int64_t* perm_out);

/* ---- pieces exposed for the pin tests ---- */
double orc_shape(int order, double dist);     /* B-spline S(dist), order 0..3 */
/* single-particle gather of all six E/B components at (x,y,z) */
int orc_gather(const orc_sim* s, double x, double y, double z, double eb_out[6]);
/* one Boris push of u given E, B; returns u in place */
void orc_boris(double q, double m, double dt, const double eb[6], double u[3]);

/* ---- load balancing (Sec. 2.2) ---- */
double orc_lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes,
                         int n_workers);
int orc_knapsack(const double* costs, int64_t nboxes, int n_workers,
                 double cap_factor, int32_t* assign_out);
uint64_t orc_morton(int dim, int64_t bx, int64_t by, int64_t bz);
int orc_sfc(const double* costs, const int32_t* box_ijk /* 3 per box */, int64_t nboxes,
            int dim, int n_workers, int32_t* assign_out);
int orc_lb_adopt(double e_old, double e_new, double theta);
double orc_predicted_speedup(double e0, double x);

#ifdef __cplusplus
}
#endif
#endif
