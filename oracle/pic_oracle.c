/*
 * pic_oracle.c -- plain FP64 CPU reference of the per-box PIC step and of the
 * load-balancing routine of arXiv 2104.11385.  TEST INFRASTRUCTURE ONLY: see
 * pic_oracle.h.  Written for a reader checking it against the paper and the
 * published schemes it names; no blocking, fusion or reordering.
 *
 * Scheme readings (the paper names the PIC cycle in Sec. 2.1 and cites
 * Birdsall & Langdon, but fixes no scheme):
 *   - Yee staggering: Ex,Jx at (i+1/2,j,k), Ey,Jy at (i,j+1/2,k),
 *     Ez,Jz at (i,j,k+1/2), Bx at (i,j+1/2,k+1/2), By at (i+1/2,j,k+1/2),
 *     Bz at (i+1/2,j+1/2,k); rho at nodes.
 *   - time levels: x, E, B at n; u at n-1/2; J at n+1/2.
 *   - field update: B half step, E full step with J, B half step.
 *   - relativistic Boris push (Boris 1970).
 *   - Esirkepov charge-conserving deposit (Esirkepov, CPC 135 (2001) 144).
 *   - B-spline shapes of order 1, 2 or 3, every component interpolated at
 *     its own staggered location.  Default ("momentum-conserving" style): the
 *     run's order in every direction.  Energy-conserving variant (the
 *     Galerkin gather of Yee-grid PIC codes): one order lower along each
 *     direction in which the component is staggered, which makes the gather
 *     the transpose of the Esirkepov deposit (checked in the pins).
 * Parity with the CUDA path is checked on these definitions; the physics
 * pins (dispersion, gyration, plasma frequency, continuity, Gauss) are in the
 * tests.  The damping profile of the absorbing z layers (damp_factor) is a
 * reading with no counterpart in the paper (it fixes no field boundary); the
 * tests pin it layer by layer, bit for bit, against hand-computed factors on a
 * uniform field, besides checking that the layers absorb an outgoing pulse.
 */
#include "pic_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAX_SPECIES 8

typedef struct {
    double q, m;
    int64_t np;
    double *x, *y, *z, *ux, *uy, *uz, *w;
    int64_t* id;
} orc_species;

struct orc_sim {
    int dim;
    int64_t n[3];
    double d[3];
    double dt;
    int order;
    int ec;     /* 1: energy-conserving gather (order - 1 along staggered directions) */
    int absorb;
    int64_t step;
    double* f[9]; /* Ex Ey Ez Bx By Bz Jx Jy Jz */
    int nsp;
    orc_species sp[MAX_SPECIES];
    int has_laser;
    double las_a0, las_w0, las_tau, las_tpeak, las_omega, las_xc, las_yc;
    int64_t las_k;
};

/* staggering offsets (in cells) of each component along x, y, z */
static const double STAG[9][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* E */
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}, /* B */
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}, /* J */
};

static int64_t wrap(int64_t i, int64_t n) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t ncells(const orc_sim* s) { return s->n[0] * s->n[1] * s->n[2]; }

static int64_t idx3(const orc_sim* s, int64_t i, int64_t j, int64_t k) {
    return (wrap(k, s->n[2]) * s->n[1] + wrap(j, s->n[1])) * s->n[0] + wrap(i, s->n[0]);
}

/* B-spline shape S(dist): order 0 is the box, 1 on -1/2 <= d < 1/2 (half
 * open, so that exactly one node carries a point); order 1 is the hat 1-|d| on |d|<1; order 2 is
 * 3/4-d^2 on |d|<1/2 and (3/2-|d|)^2/2 on 1/2<=|d|<3/2; order 3 (the paper's
 * choice, Sec. 3.1) is 2/3-d^2+|d|^3/2 on |d|<1 and (2-|d|)^3/6 on 1<=|d|<2. */
double orc_shape(int order, double dist) {
    if (order == 0) return (dist >= -0.5 && dist < 0.5) ? 1.0 : 0.0;
    double a = fabs(dist);
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (order == 2) {
        if (a < 0.5) return 0.75 - a * a;
        if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    }
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

/* first node of the (order+1)-point support of S around the point xi
 * (xi in cell units, measured from the component's own grid origin). */
static int64_t support_start(int order, double xi) {
    if (order == 0) return (int64_t)floor(xi + 0.5);
    if (order == 1) return (int64_t)floor(xi);
    if (order == 2) return (int64_t)floor(xi + 0.5) - 1;
    return (int64_t)floor(xi) - 1;
}

orc_sim* orc_create(int dim, const int64_t n[3], const double d[3], double dt,
                    int order, int absorb_cells) {
    if (dim != 2 && dim != 3) return NULL;
    if (order < 1 || order > 3) return NULL;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return NULL;
    if (dim == 2 && n[1] != 1) return NULL;
    if (absorb_cells < 0 || 2 * (int64_t)absorb_cells >= n[2]) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->dim = dim;
    for (int a = 0; a < 3; a++) { s->n[a] = n[a]; s->d[a] = d[a]; }
    if (dim == 2) s->d[1] = 1.0;
    s->dt = dt;
    s->order = order;
    s->absorb = absorb_cells;
    for (int c = 0; c < 9; c++) s->f[c] = (double*)calloc((size_t)ncells(s), sizeof(double));
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    for (int c = 0; c < 9; c++) free(s->f[c]);
    for (int p = 0; p < s->nsp; p++) {
        orc_species* sp = &s->sp[p];
        free(sp->x); free(sp->y); free(sp->z); free(sp->ux); free(sp->uy); free(sp->uz);
        free(sp->w); free(sp->id);
    }
    free(s);
}

static double* dup(const double* a, int64_t n) {
    double* r = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (a && n > 0) memcpy(r, a, (size_t)n * sizeof(double));
    else memset(r, 0, (size_t)(n > 0 ? n : 1) * sizeof(double));
    return r;
}

int orc_add_species(orc_sim* s, double q, double m, int64_t np,
                    const double* x, const double* y, const double* z,
                    const double* ux, const double* uy, const double* uz,
                    const double* w, const int64_t* id) {
    if (!s || s->nsp >= MAX_SPECIES || np < 0 || m <= 0.0) return -1;
    orc_species* sp = &s->sp[s->nsp];
    sp->q = q; sp->m = m; sp->np = np;
    sp->x = dup(x, np); sp->y = dup(s->dim == 3 ? y : NULL, np); sp->z = dup(z, np);
    sp->ux = dup(ux, np); sp->uy = dup(uy, np); sp->uz = dup(uz, np); sp->w = dup(w, np);
    sp->id = (int64_t*)malloc((size_t)(np > 0 ? np : 1) * sizeof(int64_t));
    for (int64_t p = 0; p < np; p++) sp->id[p] = id ? id[p] : p;
    return s->nsp++;
}

int orc_set_laser(orc_sim* s, double a0, double w0, double tau, double t_peak,
                  double omega, double xc, double yc, int64_t k_ant) {
    if (!s || k_ant < 0 || k_ant >= s->n[2] || w0 <= 0.0 || tau <= 0.0) return -1;
    s->has_laser = 1;
    s->las_a0 = a0; s->las_w0 = w0; s->las_tau = tau; s->las_tpeak = t_peak;
    s->las_omega = omega; s->las_xc = xc; s->las_yc = yc; s->las_k = k_ant;
    return 0;
}

int orc_set_field(orc_sim* s, int comp, const double* data) {
    if (!s || comp < 0 || comp > 8) return -1;
    memcpy(s->f[comp], data, (size_t)ncells(s) * sizeof(double));
    return 0;
}

int orc_get_field(const orc_sim* s, int comp, double* out) {
    if (!s || comp < 0 || comp > 8) return -1;
    memcpy(out, s->f[comp], (size_t)ncells(s) * sizeof(double));
    return 0;
}

int64_t orc_num_particles(const orc_sim* s, int species) {
    if (!s || species < 0 || species >= s->nsp) return -1;
    return s->sp[species].np;
}

int64_t orc_step_count(const orc_sim* s) { return s ? s->step : -1; }

int orc_get_particles(const orc_sim* s, int species, double* x, double* y, double* z,
                      double* ux, double* uy, double* uz, double* w, int64_t* id) {
    if (!s || species < 0 || species >= s->nsp) return -1;
    const orc_species* sp = &s->sp[species];
    size_t nb = (size_t)sp->np * sizeof(double);
    if (x) memcpy(x, sp->x, nb);
    if (y) memcpy(y, sp->y, nb);
    if (z) memcpy(z, sp->z, nb);
    if (ux) memcpy(ux, sp->ux, nb);
    if (uy) memcpy(uy, sp->uy, nb);
    if (uz) memcpy(uz, sp->uz, nb);
    if (w) memcpy(w, sp->w, nb);
    if (id) memcpy(id, sp->id, (size_t)sp->np * sizeof(int64_t));
    return 0;
}

/* ------------------------------------------------------------------ */
/* Field gather: each component interpolated at its own staggered grid  */
/* with S of the run's order in every (active) direction, or, for the   */
/* energy-conserving variant, of order - 1 along the directions in      */
/* which the component sits at half nodes.                              */
/* ------------------------------------------------------------------ */
static double gather_comp(const orc_sim* s, int comp, const double X[3]) {
    int64_t base[3];
    int npts[3];
    double wt[3][4];
    for (int a = 0; a < 3; a++) {
        if (a == 1 && s->dim == 2) { base[a] = 0; npts[a] = 1; wt[a][0] = 1.0; continue; }
        int o = (s->ec && STAG[comp][a] == 0.5) ? s->order - 1 : s->order;
        double xi = X[a] - STAG[comp][a];
        base[a] = support_start(o, xi);
        npts[a] = o + 1;
        for (int l = 0; l < npts[a]; l++) wt[a][l] = orc_shape(o, xi - (double)(base[a] + l));
    }
    double sum = 0.0;
    for (int c = 0; c < npts[2]; c++)
        for (int b = 0; b < npts[1]; b++)
            for (int a = 0; a < npts[0]; a++)
                sum += wt[0][a] * wt[1][b] * wt[2][c] *
                       s->f[comp][idx3(s, base[0] + a, base[1] + b, base[2] + c)];
    return sum;
}

int orc_set_gather(orc_sim* s, int energy_conserving) {
    if (!s || (energy_conserving != 0 && energy_conserving != 1)) return -1;
    s->ec = energy_conserving;
    return 0;
}

int orc_gather(const orc_sim* s, double x, double y, double z, double eb_out[6]) {
    if (!s) return -1;
    double X[3] = {x / s->d[0], s->dim == 3 ? y / s->d[1] : 0.0, z / s->d[2]};
    for (int c = 0; c < 6; c++) eb_out[c] = gather_comp(s, c, X);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Relativistic Boris push (Boris 1970; Birdsall & Langdon Sec. 15-4):  */
/* half electric kick, magnetic rotation, half electric kick.           */
/* ------------------------------------------------------------------ */
void orc_boris(double q, double m, double dt, const double eb[6], double u[3]) {
    double k = q * dt / (2.0 * m);
    double um[3], up[3], ud[3], t[3], sv[3];
    for (int a = 0; a < 3; a++) um[a] = u[a] + k * eb[a];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; a++) t[a] = k * eb[3 + a] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; a++) sv[a] = 2.0 * t[a] / (1.0 + t2);
    /* u' = u- + u- x t */
    ud[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    ud[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    ud[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    /* u+ = u- + u' x s */
    up[0] = um[0] + (ud[1] * sv[2] - ud[2] * sv[1]);
    up[1] = um[1] + (ud[2] * sv[0] - ud[0] * sv[2]);
    up[2] = um[2] + (ud[0] * sv[1] - ud[1] * sv[0]);
    for (int a = 0; a < 3; a++) u[a] = up[a] + k * eb[a];
}

/* ------------------------------------------------------------------ */
/* Esirkepov deposit.  S0, S1: node shape factors at the old and new     */
/* positions on a common window of order+3 nodes whose first node is     */
/* taken from the old position; dS = S1 - S0.  The decomposition weights */
/* W (Esirkepov 2001, Eq. 31 in 3D; the 2D form with the out-of-plane    */
/* current) are prefix-summed along their own direction.                 */
/* ------------------------------------------------------------------ */
#define WMAX 6

static int64_t window_start(int order, double X0) {
    if (order == 1) return (int64_t)floor(X0) - 1;
    if (order == 2) return (int64_t)floor(X0 + 0.5) - 2;
    return (int64_t)floor(X0) - 2;
}

static void node_shapes(int order, double X0, double X1, int64_t base, int L,
                        double S0[WMAX], double DS[WMAX]) {
    for (int l = 0; l < L; l++) {
        double node = (double)(base + l);
        S0[l] = orc_shape(order, X0 - node);
        DS[l] = orc_shape(order, X1 - node) - S0[l];
    }
}

static void deposit3d(orc_sim* s, double qw, const double X0[3], const double X1[3]) {
    int o = s->order, L = o + 3;
    int64_t b[3];
    double S0[3][WMAX], DS[3][WMAX];
    for (int a = 0; a < 3; a++) {
        b[a] = window_start(o, X0[a]);
        node_shapes(o, X0[a], X1[a], b[a], L, S0[a], DS[a]);
    }
    const double dx = s->d[0], dy = s->d[1], dz = s->d[2], dt = s->dt;
    const double cx = -qw / (dy * dz * dt);
    const double cy = -qw / (dx * dz * dt);
    const double cz = -qw / (dx * dy * dt);
    double* Jx = s->f[ORC_JX];
    double* Jy = s->f[ORC_JY];
    double* Jz = s->f[ORC_JZ];
    /* Jx: prefix sum along x of Wx */
    for (int n = 0; n < L; n++)
        for (int m = 0; m < L; m++) {
            double acc = 0.0;
            for (int l = 0; l < L; l++) {
                double W = DS[0][l] * (S0[1][m] * S0[2][n] + 0.5 * DS[1][m] * S0[2][n] +
                                       0.5 * S0[1][m] * DS[2][n] + DS[1][m] * DS[2][n] / 3.0);
                acc += W;
                Jx[idx3(s, b[0] + l, b[1] + m, b[2] + n)] += cx * acc;
            }
        }
    /* Jy: prefix sum along y of Wy */
    for (int n = 0; n < L; n++)
        for (int l = 0; l < L; l++) {
            double acc = 0.0;
            for (int m = 0; m < L; m++) {
                double W = DS[1][m] * (S0[0][l] * S0[2][n] + 0.5 * DS[0][l] * S0[2][n] +
                                       0.5 * S0[0][l] * DS[2][n] + DS[0][l] * DS[2][n] / 3.0);
                acc += W;
                Jy[idx3(s, b[0] + l, b[1] + m, b[2] + n)] += cy * acc;
            }
        }
    /* Jz: prefix sum along z of Wz */
    for (int m = 0; m < L; m++)
        for (int l = 0; l < L; l++) {
            double acc = 0.0;
            for (int n = 0; n < L; n++) {
                double W = DS[2][n] * (S0[0][l] * S0[1][m] + 0.5 * DS[0][l] * S0[1][m] +
                                       0.5 * S0[0][l] * DS[1][m] + DS[0][l] * DS[1][m] / 3.0);
                acc += W;
                Jz[idx3(s, b[0] + l, b[1] + m, b[2] + n)] += cz * acc;
            }
        }
}

/* 2D3V in the (z, x) plane, y invariant: in-plane currents by prefix sums,
 * out-of-plane Jy = q w vy W_y / (dx dz) with the 2D Esirkepov weight. */
static void deposit2d(orc_sim* s, double qw, const double X0[3], const double X1[3], double vy) {
    int o = s->order, L = o + 3;
    int64_t bx = window_start(o, X0[0]), bz = window_start(o, X0[2]);
    double S0x[WMAX], DSx[WMAX], S0z[WMAX], DSz[WMAX];
    node_shapes(o, X0[0], X1[0], bx, L, S0x, DSx);
    node_shapes(o, X0[2], X1[2], bz, L, S0z, DSz);
    const double dx = s->d[0], dz = s->d[2], dt = s->dt;
    const double cx = -qw / (dz * dt);
    const double cz = -qw / (dx * dt);
    const double cyv = qw * vy / (dx * dz);
    double* Jx = s->f[ORC_JX];
    double* Jy = s->f[ORC_JY];
    double* Jz = s->f[ORC_JZ];
    for (int n = 0; n < L; n++) {
        double acc = 0.0;
        for (int l = 0; l < L; l++) {
            acc += DSx[l] * (S0z[n] + 0.5 * DSz[n]);
            Jx[idx3(s, bx + l, 0, bz + n)] += cx * acc;
        }
    }
    for (int l = 0; l < L; l++) {
        double acc = 0.0;
        for (int n = 0; n < L; n++) {
            acc += DSz[n] * (S0x[l] + 0.5 * DSx[l]);
            Jz[idx3(s, bx + l, 0, bz + n)] += cz * acc;
        }
    }
    for (int n = 0; n < L; n++)
        for (int l = 0; l < L; l++) {
            double W = S0x[l] * S0z[n] + 0.5 * DSx[l] * S0z[n] + 0.5 * S0x[l] * DSz[n] +
                       DSx[l] * DSz[n] / 3.0;
            Jy[idx3(s, bx + l, 0, bz + n)] += cyv * W;
        }
}

/* ------------------------------------------------------------------ */
/* Yee FDTD (the field solve named in Sec. 3.3).  Curls with periodic    */
/* index wrap; d/dy terms vanish in 2D.                                  */
/* ------------------------------------------------------------------ */
#define F(c, i, j, k) s->f[c][idx3(s, (i), (j), (k))]

static void push_b_half(orc_sim* s) {
    const double h = 0.5 * s->dt;
    const double ix = 1.0 / s->d[0], iy = (s->dim == 3) ? 1.0 / s->d[1] : 0.0, iz = 1.0 / s->d[2];
    for (int64_t k = 0; k < s->n[2]; k++)
        for (int64_t j = 0; j < s->n[1]; j++)
            for (int64_t i = 0; i < s->n[0]; i++) {
                double cEx = (F(ORC_EZ, i, j + 1, k) - F(ORC_EZ, i, j, k)) * iy -
                             (F(ORC_EY, i, j, k + 1) - F(ORC_EY, i, j, k)) * iz;
                double cEy = (F(ORC_EX, i, j, k + 1) - F(ORC_EX, i, j, k)) * iz -
                             (F(ORC_EZ, i + 1, j, k) - F(ORC_EZ, i, j, k)) * ix;
                double cEz = (F(ORC_EY, i + 1, j, k) - F(ORC_EY, i, j, k)) * ix -
                             (F(ORC_EX, i, j + 1, k) - F(ORC_EX, i, j, k)) * iy;
                F(ORC_BX, i, j, k) -= h * cEx;
                F(ORC_BY, i, j, k) -= h * cEy;
                F(ORC_BZ, i, j, k) -= h * cEz;
            }
}

static void push_e(orc_sim* s) {
    const double dt = s->dt;
    const double ix = 1.0 / s->d[0], iy = (s->dim == 3) ? 1.0 / s->d[1] : 0.0, iz = 1.0 / s->d[2];
    for (int64_t k = 0; k < s->n[2]; k++)
        for (int64_t j = 0; j < s->n[1]; j++)
            for (int64_t i = 0; i < s->n[0]; i++) {
                double cBx = (F(ORC_BZ, i, j, k) - F(ORC_BZ, i, j - 1, k)) * iy -
                             (F(ORC_BY, i, j, k) - F(ORC_BY, i, j, k - 1)) * iz;
                double cBy = (F(ORC_BX, i, j, k) - F(ORC_BX, i, j, k - 1)) * iz -
                             (F(ORC_BZ, i, j, k) - F(ORC_BZ, i - 1, j, k)) * ix;
                double cBz = (F(ORC_BY, i, j, k) - F(ORC_BY, i - 1, j, k)) * ix -
                             (F(ORC_BX, i, j, k) - F(ORC_BX, i, j - 1, k)) * iy;
                F(ORC_EX, i, j, k) += dt * (cBx - F(ORC_JX, i, j, k));
                F(ORC_EY, i, j, k) += dt * (cBy - F(ORC_JY, i, j, k));
                F(ORC_EZ, i, j, k) += dt * (cBz - F(ORC_JZ, i, j, k));
            }
}

/* damping layers at both z ends: E and B in cell layer k scaled by
 * 1 - 0.5 (p/absorb)^2, p = depth of layer k inside the layer (1..absorb). */
static double damp_factor(const orc_sim* s, int64_t k) {
    int64_t A = s->absorb, p = 0;
    if (k < A) p = A - k;
    else if (k > s->n[2] - 1 - A) p = k - (s->n[2] - 1 - A);
    double r = (double)p / (double)A;
    return 1.0 - 0.5 * r * r;
}

static void damp_fields(orc_sim* s) {
    if (s->absorb <= 0) return;
    for (int64_t k = 0; k < s->n[2]; k++) {
        double f = damp_factor(s, k);
        if (f == 1.0) continue;
        for (int c = 0; c < 6; c++)
            for (int64_t j = 0; j < s->n[1]; j++)
                for (int64_t i = 0; i < s->n[0]; i++) F(c, i, j, k) *= f;
    }
}

/* laser antenna: a soft sheet of Jx in the plane k = k_ant at the J time
 * level t = (n + 1/2) dt; a sheet current K = Jx dz radiates |E| = |K|/2 to
 * each side, so Jx = 2 a0 / dz gives the forward wave amplitude a0. */
static void add_antenna(orc_sim* s) {
    if (!s->has_laser) return;
    double t = ((double)s->step + 0.5) * s->dt;
    double tt = (t - s->las_tpeak) / s->las_tau;
    double env = exp(-tt * tt) * sin(s->las_omega * (t - s->las_tpeak));
    double amp = 2.0 * s->las_a0 / s->d[2] * env;
    for (int64_t j = 0; j < s->n[1]; j++)
        for (int64_t i = 0; i < s->n[0]; i++) {
            double x = ((double)i + 0.5) * s->d[0] - s->las_xc;
            double y = (s->dim == 3) ? (double)j * s->d[1] - s->las_yc : 0.0;
            double r2 = x * x + y * y;
            F(ORC_JX, i, j, s->las_k) += amp * exp(-r2 / (s->las_w0 * s->las_w0));
        }
}
#undef F

/* ------------------------------------------------------------------ */
/* One PIC cycle: for every particle gather at x^n, Boris push, deposit  */
/* J^{n+1/2} from x^n to x^{n+1}, boundary; then the field update.       */
/* ------------------------------------------------------------------ */
static void remove_particle(orc_species* sp, int64_t p) {
    int64_t last = sp->np - 1;
    /* keep array order: shift down (slow, obviously order-preserving) */
    for (int64_t r = p; r < last; r++) {
        sp->x[r] = sp->x[r + 1]; sp->y[r] = sp->y[r + 1]; sp->z[r] = sp->z[r + 1];
        sp->ux[r] = sp->ux[r + 1]; sp->uy[r] = sp->uy[r + 1]; sp->uz[r] = sp->uz[r + 1];
        sp->w[r] = sp->w[r + 1]; sp->id[r] = sp->id[r + 1];
    }
    sp->np = last;
}

static double periodic_pos(double x, double L) {
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

static void step_once(orc_sim* s) {
    const int64_t nc = ncells(s);
    for (int c = ORC_JX; c <= ORC_JZ; c++) memset(s->f[c], 0, (size_t)nc * sizeof(double));
    const double L[3] = {s->n[0] * s->d[0], s->n[1] * s->d[1], s->n[2] * s->d[2]};
    const double zlo = (double)s->absorb * s->d[2];
    const double zhi = (double)(s->n[2] - s->absorb) * s->d[2];
    for (int ps = 0; ps < s->nsp; ps++) {
        orc_species* sp = &s->sp[ps];
        int64_t* drop = (int64_t*)malloc((size_t)(sp->np > 0 ? sp->np : 1) * sizeof(int64_t));
        int64_t ndrop = 0;
        for (int64_t p = 0; p < sp->np; p++) {
            double pos[3] = {sp->x[p], s->dim == 3 ? sp->y[p] : 0.0, sp->z[p]};
            double X0[3] = {pos[0] / s->d[0], pos[1] / s->d[1], pos[2] / s->d[2]};
            double eb[6];
            for (int c = 0; c < 6; c++) eb[c] = gather_comp(s, c, X0);
            double u[3] = {sp->ux[p], sp->uy[p], sp->uz[p]};
            orc_boris(sp->q, sp->m, s->dt, eb, u);
            double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double np_[3];
            for (int a = 0; a < 3; a++) np_[a] = pos[a] + s->dt * u[a] / g;
            if (s->dim == 2) np_[1] = 0.0;
            double X1[3] = {np_[0] / s->d[0], np_[1] / s->d[1], np_[2] / s->d[2]};
            double qw = sp->q * sp->w[p];
            if (s->dim == 3) deposit3d(s, qw, X0, X1);
            else deposit2d(s, qw, X0, X1, u[1] / g);
            sp->ux[p] = u[0]; sp->uy[p] = u[1]; sp->uz[p] = u[2];
            sp->x[p] = periodic_pos(np_[0], L[0]);
            if (s->dim == 3) sp->y[p] = periodic_pos(np_[1], L[1]);
            if (s->absorb > 0) {
                sp->z[p] = np_[2];
                if (np_[2] < zlo || np_[2] >= zhi) drop[ndrop++] = p;
            } else {
                sp->z[p] = periodic_pos(np_[2], L[2]);
            }
        }
        for (int64_t r = ndrop - 1; r >= 0; r--) remove_particle(sp, drop[r]);
        free(drop);
    }
    add_antenna(s);
    push_b_half(s);
    push_e(s);
    push_b_half(s);
    damp_fields(s);
    s->step++;
}

int orc_step(orc_sim* s, int nsteps) {
    if (!s || nsteps < 0) return -1;
    for (int t = 0; t < nsteps; t++) step_once(s);
    return 0;
}

int orc_deposit_rho(const orc_sim* s, double* rho) {
    if (!s) return -1;
    const int64_t nc = ncells(s);
    memset(rho, 0, (size_t)nc * sizeof(double));
    const int o = s->order, np1 = o + 1;
    const double vol = s->d[0] * s->d[1] * s->d[2];
    for (int ps = 0; ps < s->nsp; ps++) {
        const orc_species* sp = &s->sp[ps];
        for (int64_t p = 0; p < sp->np; p++) {
            double X[3] = {sp->x[p] / s->d[0], s->dim == 3 ? sp->y[p] / s->d[1] : 0.0,
                           sp->z[p] / s->d[2]};
            int64_t b[3];
            double wt[3][4];
            for (int a = 0; a < 3; a++) {
                if (a == 1 && s->dim == 2) { b[a] = 0; wt[a][0] = 1.0; continue; }
                b[a] = support_start(o, X[a]);
                for (int l = 0; l < np1; l++) wt[a][l] = orc_shape(o, X[a] - (double)(b[a] + l));
            }
            int ny_pts = (s->dim == 2) ? 1 : np1;
            double qw = sp->q * sp->w[p] / vol;
            for (int c = 0; c < np1; c++)
                for (int bb = 0; bb < ny_pts; bb++)
                    for (int a = 0; a < np1; a++)
                        rho[idx3(s, b[0] + a, b[1] + bb, b[2] + c)] +=
                            qw * wt[0][a] * wt[1][bb] * wt[2][c];
        }
    }
    return 0;
}

int orc_box_counts(const orc_sim* s, const int64_t bsize[3], int64_t* counts) {
    if (!s) return -1;
    int64_t nb[3];
    for (int a = 0; a < 3; a++) {
        if (bsize[a] < 1 || s->n[a] % bsize[a] != 0) return -1;
        nb[a] = s->n[a] / bsize[a];
    }
    memset(counts, 0, (size_t)(nb[0] * nb[1] * nb[2]) * sizeof(int64_t));
    for (int ps = 0; ps < s->nsp; ps++) {
        const orc_species* sp = &s->sp[ps];
        for (int64_t p = 0; p < sp->np; p++) {
            double pos[3] = {sp->x[p], s->dim == 3 ? sp->y[p] : 0.0, sp->z[p]};
            int64_t c[3];
            for (int a = 0; a < 3; a++) {
                c[a] = wrap((int64_t)floor(pos[a] / s->d[a]), s->n[a]) / bsize[a];
            }
            counts[(c[2] * nb[1] + c[1]) * nb[0] + c[0]]++;
        }
    }
    return 0;
}

int orc_bin_particles(int dim, const int64_t n[3], const double d[3], const int64_t bsize[3],
                      const double* x, const double* y, const double* z, int64_t np,
                      int64_t* box_off, int64_t* perm) {
    int64_t nb[3];
    for (int a = 0; a < 3; a++) {
        if (bsize[a] < 1 || n[a] % bsize[a] != 0) return -1;
        nb[a] = n[a] / bsize[a];
    }
    if (dim == 2 && n[1] != 1) return -1;
    const int64_t nboxes = nb[0] * nb[1] * nb[2];
    int64_t* box = (int64_t*)malloc((size_t)(np > 0 ? np : 1) * sizeof(int64_t));
    for (int64_t b = 0; b <= nboxes; b++) box_off[b] = 0;
    for (int64_t p = 0; p < np; p++) {
        double pos[3] = {x[p], dim == 3 ? y[p] : 0.0, z[p]};
        int64_t c[3];
        for (int a = 0; a < 3; a++) {
            double dd = (dim == 2 && a == 1) ? 1.0 : d[a];
            c[a] = wrap((int64_t)floor(pos[a] / dd), n[a]) / bsize[a];
        }
        box[p] = (c[2] * nb[1] + c[1]) * nb[0] + c[0];
        box_off[box[p] + 1]++;
    }
    for (int64_t b = 0; b < nboxes; b++) box_off[b + 1] += box_off[b];
    /* stable placement: particles visited in ascending index */
    int64_t* fill = (int64_t*)calloc((size_t)(nboxes > 0 ? nboxes : 1), sizeof(int64_t));
    for (int64_t p = 0; p < np; p++) perm[box_off[box[p]] + fill[box[p]]++] = p;
    free(fill);
    free(box);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Load balancing, Sec. 2.2.                                           */
/* ------------------------------------------------------------------ */

/* Eq. 1: E = c_avg / c_max over workers; a worker's cost is the sum of its
 * boxes' costs (ascending box index); E = 1 when every worker is idle. */
double orc_lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes,
                         int n_workers) {
    if (n_workers < 1) return -1.0;
    double* wc = (double*)calloc((size_t)n_workers, sizeof(double));
    for (int64_t b = 0; b < nboxes; b++) wc[assign[b]] += costs[b];
    double total = 0.0, mx = 0.0;
    for (int w = 0; w < n_workers; w++) {
        total += wc[w];
        if (wc[w] > mx) mx = wc[w];
    }
    free(wc);
    if (mx == 0.0) return 1.0;
    return (total / (double)n_workers) / mx;
}

/* knapsack (Sec. 2.2): spread box costs as evenly as possible over workers,
 * ignoring geometry.  Greedy longest-processing-time-first: boxes by cost
 * descending (ties: lower index first), each to the least-loaded worker
 * (ties: lowest id) among those holding fewer than the box cap, the cap
 * being cap_factor times the average boxes per worker (Sec. 3.3 footnote,
 * 1.5), but at least ceil(nboxes / n_workers). */
int orc_knapsack(const double* costs, int64_t nboxes, int n_workers, double cap_factor,
                 int32_t* assign) {
    if (n_workers < 1 || nboxes < 0) return -1;
    int64_t* order = (int64_t*)malloc((size_t)(nboxes > 0 ? nboxes : 1) * sizeof(int64_t));
    for (int64_t b = 0; b < nboxes; b++) order[b] = b;
    /* insertion sort: plain and stable, fine for the test sizes */
    for (int64_t i = 1; i < nboxes; i++) {
        int64_t v = order[i], j = i - 1;
        while (j >= 0 && costs[order[j]] < costs[v]) { order[j + 1] = order[j]; j--; }
        order[j + 1] = v;
    }
    int64_t cap_ceil = (nboxes + n_workers - 1) / n_workers;
    int64_t cap_f = (int64_t)floor(cap_factor * (double)nboxes / (double)n_workers);
    int64_t cap = cap_f > cap_ceil ? cap_f : cap_ceil;
    double* load = (double*)calloc((size_t)n_workers, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)n_workers, sizeof(int64_t));
    for (int64_t r = 0; r < nboxes; r++) {
        int64_t b = order[r];
        int best = -1;
        for (int w = 0; w < n_workers; w++) {
            if (cnt[w] >= cap) continue;
            if (best < 0 || load[w] < load[best]) best = w;
        }
        assign[b] = best;
        load[best] += costs[b];
        cnt[best]++;
    }
    free(order); free(load); free(cnt);
    return 0;
}

/* Morton Z-order key: bit i of bx goes to bit 3i, of by to 3i+1, of bz to
 * 3i+2; in 2D (z, x plane) bit i of bx goes to 2i and of bz to 2i+1. */
uint64_t orc_morton(int dim, int64_t bx, int64_t by, int64_t bz) {
    uint64_t key = 0;
    if (dim == 3) {
        for (int i = 0; i < 21; i++) {
            key |= (uint64_t)((bx >> i) & 1) << (3 * i);
            key |= (uint64_t)((by >> i) & 1) << (3 * i + 1);
            key |= (uint64_t)((bz >> i) & 1) << (3 * i + 2);
        }
    } else {
        for (int i = 0; i < 32; i++) {
            key |= (uint64_t)((bx >> i) & 1) << (2 * i);
            key |= (uint64_t)((bz >> i) & 1) << (2 * i + 1);
        }
    }
    return key;
}

/* space-filling curve (Sec. 2.2): enumerate boxes along the Morton curve
 * and cut the sequence into contiguous pieces of about equal cost: the
 * worker index advances after the box whose running total reaches the next
 * multiple of total / n_workers. */
int orc_sfc(const double* costs, const int32_t* ijk, int64_t nboxes, int dim, int n_workers,
            int32_t* assign) {
    if (n_workers < 1 || nboxes < 0 || (dim != 2 && dim != 3)) return -1;
    int64_t* order = (int64_t*)malloc((size_t)(nboxes > 0 ? nboxes : 1) * sizeof(int64_t));
    uint64_t* key = (uint64_t*)malloc((size_t)(nboxes > 0 ? nboxes : 1) * sizeof(uint64_t));
    for (int64_t b = 0; b < nboxes; b++) {
        order[b] = b;
        key[b] = orc_morton(dim, ijk[3 * b], ijk[3 * b + 1], ijk[3 * b + 2]);
    }
    for (int64_t i = 1; i < nboxes; i++) {
        int64_t v = order[i], j = i - 1;
        while (j >= 0 && (key[order[j]] > key[v] || (key[order[j]] == key[v] && order[j] > v))) {
            order[j + 1] = order[j];
            j--;
        }
        order[j + 1] = v;
    }
    double total = 0.0;
    for (int64_t r = 0; r < nboxes; r++) total += costs[order[r]];
    double prefix = 0.0;
    int w = 0;
    for (int64_t r = 0; r < nboxes; r++) {
        int64_t b = order[r];
        assign[b] = w;
        prefix += costs[b];
        if (prefix * (double)n_workers >= (double)(w + 1) * total && w < n_workers - 1) w++;
    }
    free(order); free(key);
    return 0;
}

/* the improvement threshold (Sec. 2.2, Sec. 3.2): the proposed mapping is
 * adopted when its efficiency is at least (1 + theta) times the current one. */
int orc_lb_adopt(double e_old, double e_new, double theta) {
    return e_new >= (1.0 + theta) * e_old;
}

/* Sec. 4, Eq. 2: S = (c_max0 / c_avg0)^x = (1 / E0)^x. */
double orc_predicted_speedup(double e0, double x) { return pow(1.0 / e0, x); }
