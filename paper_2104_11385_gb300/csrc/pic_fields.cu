// pic_fields.cu -- the cell side of the PIC cycle: Yee FDTD update (the
// finite-difference time-domain field solve named in arXiv 2104.11385 Sec. 3.3)
// as B half step, E full step with the deposited current (and the laser
// antenna source of Sec. 3.1), B half step; z damping layers; periodic guard
// fill of the padded E/B arrays for the next step's TMA tile loads.
//
// Each cell update reads E,B,J and writes E,B (120 bytes) with 39 FP64
// operations (the time step over the cell size folded into the differences:
// 12 per B half step, 15 for E): on GB300, whose FP64 rate is 1/64 of FP32,
// that is FP64-bound, not HBM-bound.  One warp per x row of cells, lanes
// along x for coalescing; the guard kernels visit only the guard cells.
#include "pic_internal.h"

namespace {

__device__ __forceinline__ int nxt(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int prv(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// multi-simulation launches: blockIdx.y indexes the slot list (nullptr: slot 0)
__device__ __forceinline__ const SimDev& slot_sim(const SimDev* sims, const int* slots) {
    return sims[slots ? slots[blockIdx.y] : 0];
}

// Visits the interior cells this simulation owns, one warp per x row (j, k),
// lanes along x (coalesced): f(i, j, k, o, oi, oj, ok) gets the cell's padded
// index o and those of its periodic neighbours along x, y and z, the next ones
// (FWD) or the previous ones.  Only the row index is divided.
template <int DIM, bool FWD, class F>
__device__ __forceinline__ void for_cells_by_row(const SimDev& S, F&& f) {
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const bool all_owned = S.owner == nullptr;
    const int wpb = blockDim.x >> 5;
    const int64_t rows = (int64_t)ny * nz;
    auto nb = [](int i, int n) { return FWD ? nxt(i, n) : prv(i, n); };
    for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const int k = (int)(r / ny), j = (int)(r - (int64_t)k * ny);
        const int64_t row = pidx(S, 0, j, k);
        const int64_t dj = (DIM == 3) ? pidx(S, 0, nb(j, ny), k) - row : 0;
        const int64_t dk = pidx(S, 0, j, nb(k, nz)) - row;
#pragma unroll 1
        for (int i = threadIdx.x & 31; i < nx; i += 32) {
            if (!all_owned && !cell_owned(S, i, j, k)) continue;
            const int64_t o = row + i;
            f(i, j, k, o, row + nb(i, nx), o + dj, o + dk);
        }
    }
}

template <int DIM>
__global__ void b_half_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots) {
    const SimDev& S = slot_sim(sims, slots);
    // B -= (dt/2) curl E with dt/(2 dx) folded into the differences: two FMAs
    // per component
    const double h = 0.5 * S.dt;
    const double hx = h * S.invd[0], hy = (DIM == 3) ? h * S.invd[1] : 0.0, hz = h * S.invd[2];
    const double* __restrict__ Ex = S.F[0];
    const double* __restrict__ Ey = S.F[1];
    const double* __restrict__ Ez = S.F[2];
    double* __restrict__ Bx = S.F[3];
    double* __restrict__ By = S.F[4];
    double* __restrict__ Bz = S.F[5];
    for_cells_by_row<DIM, true>(S, [&](int, int, int, int64_t o, int64_t oi, int64_t oj, int64_t ok) {
        const double ez = Ez[o], ey = Ey[o], ex = Ex[o];
        Bx[o] = fma(Ey[ok] - ey, hz, fma(-(Ez[oj] - ez), hy, Bx[o]));
        By[o] = fma(Ez[oi] - ez, hx, fma(-(Ex[ok] - ex), hz, By[o]));
        Bz[o] = fma(Ex[oj] - ex, hy, fma(-(Ey[oi] - ey), hx, Bz[o]));
    });
}

// the antenna sheet's current at cell (i, j) of its layer (out of line: the
// exp would otherwise raise the register count of every cell's update)
template <int DIM>
__device__ __noinline__ double antenna_jx(const SimDev& S, double amp, int i, int j) {
    const LaserDev& L = S.las;
    const double x = ((double)i + 0.5) * S.d[0] - L.xc;
    const double y = (DIM == 3) ? (double)j * S.d[1] - L.yc : 0.0;
    return amp * exp(-(x * x + y * y) / (L.w0 * L.w0));
}

template <int DIM>
__global__ void e_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots) {
    const SimDev& S = slot_sim(sims, slots);
    // E += dt (curl B - J) with dt/dx folded into the differences: three FMAs
    // per component
    const double dt = S.dt;
    const double tx = dt * S.invd[0], ty = (DIM == 3) ? dt * S.invd[1] : 0.0, tz = dt * S.invd[2];
    double* __restrict__ Ex = S.F[0];
    double* __restrict__ Ey = S.F[1];
    double* __restrict__ Ez = S.F[2];
    const double* __restrict__ Bx = S.F[3];
    const double* __restrict__ By = S.F[4];
    const double* __restrict__ Bz = S.F[5];
    const double* __restrict__ Jx = S.F[6];
    const double* __restrict__ Jy = S.F[7];
    const double* __restrict__ Jz = S.F[8];
    const LaserDev L = S.las;
    // the antenna's time factor, once per block (FP64 exp and sin are dozens
    // of FP64 instructions, at 1/64 of the FP32 rate)
    __shared__ double s_amp;
    if (threadIdx.x == 0) {
        double a = 0.0;
        if (L.on) {
            double t = ((double)(*S.step) + 0.5) * dt;
            double tt = (t - L.t_peak) / L.tau;
            a = 2.0 * L.a0 / S.d[2] * exp(-tt * tt) * sin(L.omega * (t - L.t_peak));
        }
        s_amp = a;
    }
    __syncthreads();
    const double amp = s_amp;
    for_cells_by_row<DIM, false>(S, [&](int i, int j, int k, int64_t o, int64_t oi, int64_t oj, int64_t ok) {
        const double bx = Bx[o], by = By[o], bz = Bz[o];
        double jx = Jx[o];
        if (L.on && k == L.k_ant) {
            jx += antenna_jx<DIM>(S, amp, i, j);
            const_cast<double*>(Jx)[o] = jx;  // the antenna sheet is part of J^{n+1/2}
        }
        Ex[o] = fma(-dt, jx, fma(bz - Bz[oj], ty, fma(-(by - By[ok]), tz, Ex[o])));
        Ey[o] = fma(-dt, Jy[o], fma(bx - Bx[ok], tz, fma(-(bz - Bz[oi]), tx, Ey[o])));
        Ez[o] = fma(-dt, Jz[o], fma(by - By[oi], tx, fma(-(bx - Bx[oj]), ty, Ez[o])));
    });
}

// E and B of cell layer k scaled by 1 - 0.5 (p/A)^2, p = depth inside the layer
__global__ void damp_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots) {
    const SimDev& S = slot_sim(sims, slots);
    const int A = S.absorb;
    if (A <= 0) return;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const int64_t per_layer = (int64_t)nx * ny;
    const int64_t total = per_layer * 2 * A;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        int layer = (int)(c / per_layer);
        int64_t r = c - (int64_t)layer * per_layer;
        int i = (int)(r % nx), j = (int)(r / nx);
        int k = layer < A ? layer : nz - 2 * A + layer;
        if (!cell_owned(S, i, j, k)) continue;
        int p = k < A ? A - k : k - (nz - 1 - A);
        double q = (double)p / (double)A;
        double f = 1.0 - 0.5 * q * q;
        int64_t o = pidx(S, i, j, k);
#pragma unroll
        for (int comp = 0; comp < 6; ++comp) S.F[comp][o] *= f;
    }
}

// Visits the guard cells of the padded arrays, one warp per padded row (b, e):
// the whole row when it lies in a y or z guard layer, else only the x guards
// at its two ends (at most 8 cells).  f(c, i, j, k) gets the padded index and
// the interior coordinates of the cell (outside [0, n) along some axis).  The
// guards are a few per cent of the padded volume, and no thread divides
// anything but its row index.
template <class F>
__device__ __forceinline__ void for_guard_cells(const SimDev& S, F&& f) {
    const int px = S.pn[0], py = S.pn[1], pz = S.pn[2];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int gl = S.g[0], gx = px - S.n[0];  // left x guards, both x guards
    const int64_t rows = (int64_t)py * pz;
    for (int64_t r = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * wpb) {
        const int e = (int)(r / py), b = (int)(r - (int64_t)e * py);
        const int j = b - S.g[1], k = e - S.g[2];
        const int64_t row0 = r * px;
        if (j < 0 || j >= S.n[1] || k < 0 || k >= S.n[2]) {
            for (int a = lane; a < px; a += 32) f(row0 + a, a - gl, j, k);
        } else if (lane < gx) {
            const int a = lane < gl ? lane : S.n[0] + lane;
            f(row0 + a, a - gl, j, k);
        }
    }
}

__device__ __forceinline__ int wrap_cell(int i, int n) {
    const int r = i % n;
    return r < 0 ? r + n : r;
}

// Current deposited in the guard cells of the padded J arrays (the particle
// kernel's reductions reach up to 2 cells below and 3 above the domain) added
// to its periodic image inside the domain.  Several guard cells share an image
// (edges, corners), hence the reductions; guard cells holding zero are skipped.
__global__ void fold_j_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots) {
    const SimDev& S = slot_sim(sims, slots);
    for_guard_cells(S, [&](int64_t c, int i, int j, int k) {
        const int64_t dst = pidx(S, wrap_cell(i, S.n[0]), wrap_cell(j, S.n[1]), wrap_cell(k, S.n[2]));
#pragma unroll
        for (int comp = 6; comp < 9; ++comp) {
            const double v = S.F[comp][c];
            if (v != 0.0) atomicAdd(S.F[comp] + dst, v);
        }
    });
}

// periodic images into the guard cells of components [c0, c0+nc)
__global__ void guard_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots, int c0,
                             int nc) {
    const SimDev& S = slot_sim(sims, slots);
    for_guard_cells(S, [&](int64_t c, int i, int j, int k) {
        const int64_t src = pidx(S, wrap_cell(i, S.n[0]), wrap_cell(j, S.n[1]), wrap_cell(k, S.n[2]));
        for (int comp = c0; comp < c0 + nc; ++comp) S.F[comp][c] = S.F[comp][src];
    });
}

__global__ void unpad_kernel(const double* __restrict__ src, double* __restrict__ dst, SimDev S) {
    const int64_t ncell = (int64_t)S.n[0] * S.n[1] * S.n[2];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(c % S.n[0]);
        int j = (int)((c / S.n[0]) % S.n[1]);
        int k = (int)(c / ((int64_t)S.n[0] * S.n[1]));
        dst[c] = src[pidx(S, i, j, k)];
    }
}

__global__ void pad_kernel(const double* __restrict__ src, double* __restrict__ dst, SimDev S) {
    const int64_t ncell = (int64_t)S.n[0] * S.n[1] * S.n[2];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(c % S.n[0]);
        int j = (int)((c / S.n[0]) % S.n[1]);
        int k = (int)(c / ((int64_t)S.n[0] * S.n[1]));
        dst[pidx(S, i, j, k)] = src[c];
    }
}

// charge density at the nodes (diagnostic): shape S of the run's order
template <int DIM, int ORDER>
__global__ void rho_kernel(const SimDev* __restrict__ sims, int sp_idx, double* __restrict__ rho) {
    const SimDev& S = sims[0];
    const SpeciesDev& sp = S.sp[sp_idx];
    const int64_t np = sp.off[S.ntiles];
    const double inv_vol = 1.0 / (S.d[0] * S.d[1] * S.d[2]);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        double X[3] = {sp.cur[0][p], DIM == 3 ? sp.cur[1][p] : 0.0, sp.cur[2][p]};
        int s[3];
        double w[3][4];
        for (int a = 0; a < 3; ++a) {
            if (DIM == 2 && a == 1) { s[a] = 0; w[a][0] = 1.0; continue; }
            if (ORDER == 1) {
                s[a] = (int)floor(X[a]);
                double f = X[a] - s[a];
                w[a][0] = 1.0 - f;
                w[a][1] = f;
            } else if (ORDER == 3) {
                const int i = (int)floor(X[a]);
                const double f = X[a] - i, g = 1.0 - f;
                s[a] = i - 1;
                w[a][0] = g * g * g / 6.0;
                w[a][1] = 2.0 / 3.0 - f * f + 0.5 * f * f * f;
                w[a][2] = 2.0 / 3.0 - g * g + 0.5 * g * g * g;
                w[a][3] = f * f * f / 6.0;
            } else {
                int c = (int)floor(X[a] + 0.5);
                double d = X[a] - c;
                s[a] = c - 1;
                w[a][0] = 0.5 * (0.5 - d) * (0.5 - d);
                w[a][1] = 0.75 - d * d;
                w[a][2] = 0.5 * (0.5 + d) * (0.5 + d);
            }
        }
        const double qw = sp.q * sp.cur[6][p] * inv_vol;
        const int ny_pts = (DIM == 3) ? ORDER + 1 : 1;
        for (int c = 0; c <= ORDER; ++c)
            for (int b = 0; b < ny_pts; ++b)
                for (int a = 0; a <= ORDER; ++a) {
                    int i = ((s[0] + a) % S.n[0] + S.n[0]) % S.n[0];
                    int j = (DIM == 3) ? ((s[1] + b) % S.n[1] + S.n[1]) % S.n[1] : 0;
                    int k = ((s[2] + c) % S.n[2] + S.n[2]) % S.n[2];
                    atomicAdd(rho + ((int64_t)k * S.n[1] + j) * S.n[0] + i,
                              qw * w[0][a] * w[1][b] * w[2][c]);
                }
    }
}

// zeroes the J block (three padded arrays) of every listed simulation
__global__ void zero_j_kernel(const SimDev* __restrict__ sims, const int* __restrict__ slots) {
    const SimDev& S = slot_sim(sims, slots);
    const int64_t n = (int64_t)S.pn[0] * S.pn[1] * S.pn[2] * 3;
    double* J = S.F[6];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        J[i] = 0.0;
}

__global__ void fill_kernel(double* p, int64_t n, double v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// padded rows (y, z) of a simulation: one warp each in the guard kernels
int64_t guard_rows(const SimDev& h) { return (int64_t)h.pn[1] * h.pn[2]; }

int blocks_for(int64_t n, int t) {
    int64_t b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > (int64_t)pic_sm_count() * 64) b = (int64_t)pic_sm_count() * 64;
    return (int)b;
}

}  // namespace

cudaError_t pic_launch_fields(const SimDev* dsim, const SimDev& h, cudaStream_t st) {
    const int64_t ncell = (int64_t)h.n[0] * h.n[1] * h.n[2];
    const int nb = blocks_for(ncell, 256);
    fold_j_kernel<<<blocks_for(guard_rows(h) * 32, 256), 256, 0, st>>>(dsim, nullptr);
    if (h.dim == 3) {
        b_half_kernel<3><<<nb, 256, 0, st>>>(dsim, nullptr);
        e_kernel<3><<<nb, 256, 0, st>>>(dsim, nullptr);
        b_half_kernel<3><<<nb, 256, 0, st>>>(dsim, nullptr);
    } else {
        b_half_kernel<2><<<nb, 256, 0, st>>>(dsim, nullptr);
        e_kernel<2><<<nb, 256, 0, st>>>(dsim, nullptr);
        b_half_kernel<2><<<nb, 256, 0, st>>>(dsim, nullptr);
    }
    if (h.absorb > 0) {
        int64_t t = (int64_t)h.n[0] * h.n[1] * 2 * h.absorb;
        damp_kernel<<<blocks_for(t, 256), 256, 0, st>>>(dsim, nullptr);
    }
    return pic_launch_guards(dsim, h, 0, 6, st);
}

cudaError_t pic_launch_fold(const SimDev* dsim, const SimDev& h, cudaStream_t st) {
    fold_j_kernel<<<blocks_for(guard_rows(h) * 32, 256), 256, 0, st>>>(dsim, nullptr);
    return cudaGetLastError();
}

cudaError_t pic_launch_field_stage(const SimDev* dsim, const SimDev& h, int stage, cudaStream_t st) {
    const int64_t ncell = (int64_t)h.n[0] * h.n[1] * h.n[2];
    const int nb = blocks_for(ncell, 256);
    if (stage == 0 || stage == 2) {
        if (h.dim == 3) b_half_kernel<3><<<nb, 256, 0, st>>>(dsim, nullptr);
        else b_half_kernel<2><<<nb, 256, 0, st>>>(dsim, nullptr);
        if (stage == 2 && h.absorb > 0) {
            int64_t t = (int64_t)h.n[0] * h.n[1] * 2 * h.absorb;
            damp_kernel<<<blocks_for(t, 256), 256, 0, st>>>(dsim, nullptr);
        }
    } else if (stage == 1) {
        if (h.dim == 3) e_kernel<3><<<nb, 256, 0, st>>>(dsim, nullptr);
        else e_kernel<2><<<nb, 256, 0, st>>>(dsim, nullptr);
    } else {
        return pic_launch_guards(dsim, h, 0, 6, st);
    }
    return cudaGetLastError();
}

cudaError_t pic_launch_guards(const SimDev* dsim, const SimDev& h, int c0, int nc,
                              cudaStream_t st) {
    guard_kernel<<<blocks_for(guard_rows(h) * 32, 256), 256, 0, st>>>(dsim, nullptr, c0, nc);
    return cudaGetLastError();
}

cudaError_t pic_launch_fields_multi(const SimDev* sims, const int* slots, int nslots, int dim,
                                    int64_t max_cells, int64_t max_padded, bool any_absorb,
                                    cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    const dim3 g(blocks_for(max_cells, 256) / 4 + 1, nslots);
    fold_j_kernel<<<dim3(blocks_for(max_padded, 256) / 4 + 1, nslots), 256, 0, st>>>(sims, slots);
    if (dim == 3) {
        b_half_kernel<3><<<g, 256, 0, st>>>(sims, slots);
        e_kernel<3><<<g, 256, 0, st>>>(sims, slots);
        b_half_kernel<3><<<g, 256, 0, st>>>(sims, slots);
    } else {
        b_half_kernel<2><<<g, 256, 0, st>>>(sims, slots);
        e_kernel<2><<<g, 256, 0, st>>>(sims, slots);
        b_half_kernel<2><<<g, 256, 0, st>>>(sims, slots);
    }
    if (any_absorb) damp_kernel<<<g, 256, 0, st>>>(sims, slots);
    const dim3 gp(blocks_for(max_padded, 256) / 4 + 1, nslots);
    guard_kernel<<<gp, 256, 0, st>>>(sims, slots, 0, 6);
    return cudaGetLastError();
}

cudaError_t pic_launch_zero_j_multi(const SimDev* sims, const int* slots, int nslots,
                                    int64_t max_padded, cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    const dim3 g(blocks_for(3 * max_padded, 256) / 4 + 1, nslots);
    zero_j_kernel<<<g, 256, 0, st>>>(sims, slots);
    return cudaGetLastError();
}

cudaError_t pic_launch_unpad(const double* padded, double* dense, const SimDev& h,
                             cudaStream_t st) {
    const int64_t ncell = (int64_t)h.n[0] * h.n[1] * h.n[2];
    unpad_kernel<<<blocks_for(ncell, 256), 256, 0, st>>>(padded, dense, h);
    return cudaGetLastError();
}

cudaError_t pic_launch_pad(const double* dense, double* padded, const SimDev& h,
                           cudaStream_t st) {
    const int64_t ncell = (int64_t)h.n[0] * h.n[1] * h.n[2];
    pad_kernel<<<blocks_for(ncell, 256), 256, 0, st>>>(dense, padded, h);
    return cudaGetLastError();
}

cudaError_t pic_launch_rho(const SimDev* dsim, const SimDev& h, double* rho, double rho0,
                           cudaStream_t st) {
    const int64_t ncell = (int64_t)h.n[0] * h.n[1] * h.n[2];
    fill_kernel<<<blocks_for(ncell, 256), 256, 0, st>>>(rho, ncell, rho0);
    for (int s = 0; s < h.nsp; ++s) {
        int64_t cap = h.sp[s].cap;
        int nb = blocks_for(cap, 256);
        if (h.dim == 3 && h.order == 1) rho_kernel<3, 1><<<nb, 256, 0, st>>>(dsim, s, rho);
        else if (h.dim == 3 && h.order == 2) rho_kernel<3, 2><<<nb, 256, 0, st>>>(dsim, s, rho);
        else if (h.dim == 3) rho_kernel<3, 3><<<nb, 256, 0, st>>>(dsim, s, rho);
        else if (h.order == 1) rho_kernel<2, 1><<<nb, 256, 0, st>>>(dsim, s, rho);
        else if (h.order == 2) rho_kernel<2, 2><<<nb, 256, 0, st>>>(dsim, s, rho);
        else rho_kernel<2, 3><<<nb, 256, 0, st>>>(dsim, s, rho);
    }
    return cudaGetLastError();
}
