// pic_bin.cu -- binning of caller-owned particles by box (arXiv 2104.11385
// Sec. 2.1: a box owns the particles inside it; Sec. 2.2 moves particles with
// their box when the mapping changes).  A counting sort: per-box histogram
// (warp-aggregated 64-bit atomics), exclusive scan, scatter through per-box
// cursors.  The order of particles inside a box is unspecified.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/pic_api.h"
#include "pic_bin.h"

namespace {

__device__ __forceinline__ int bin_box_of(const BinGeom& g, const double* x, const double* y,
                                          const double* z, int64_t p) {
    const double pos[3] = {x[p], g.dim == 3 ? y[p] : 0.0, z[p]};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (g.dim == 2 && a == 1) {
            c[a] = 0;
            continue;
        }
        long long i = (long long)floor(pos[a] / g.d[a]);
        long long r = i % g.n[a];
        if (r < 0) r += g.n[a];
        c[a] = (int)(r / g.bsz[a]);
    }
    return (c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0];
}

__global__ void bin_count_kernel(BinGeom g, const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ z, int64_t np,
                                 unsigned long long* __restrict__ off) {
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < np; p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= np) break;
        const int b = bin_box_of(g, x, y, z, p);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(off + b + 1, (unsigned long long)__popc(peers));
    }
}

// in-place exclusive scan of off[1..nboxes] (off[0] = 0) by one CTA
__global__ void __launch_bounds__(1024) bin_scan_kernel(int64_t* __restrict__ off, int nboxes) {
    __shared__ int64_t part[1024];
    const int n = nboxes;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = 1 + threadIdx.x * per, i1 = min(n + 1, i0 + per);
    int64_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += off[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int64_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;
    for (int i = i0; i < i1; ++i) {
        run += off[i];
        off[i] = run;
    }
    if (threadIdx.x == 0) off[0] = 0;
}

__global__ void bin_scatter_kernel(BinGeom g, const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ z, int64_t np,
                                   const int64_t* __restrict__ off, int32_t* __restrict__ cursor,
                                   int64_t* __restrict__ perm) {
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < np; p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= np) break;
        const int b = bin_box_of(g, x, y, z, p);
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, b);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(cursor + b, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        perm[off[b] + base + __popc(peers & ((1u << lane) - 1u))] = p;
    }
}

int bin_grid(int64_t np) {
    int64_t b = (np + 255) / 256;
    if (b < 1) b = 1;
    if (b > (int64_t)pic_sm_count() * 16) b = (int64_t)pic_sm_count() * 16;
    return (int)b;
}

}  // namespace

pic_status pic_bin_validate(const pic_grid_desc* grid, const double* x, const double* y,
                            const double* z, int64_t np, const int64_t* box_off_out,
                            const int64_t* perm_out, BinGeom* g, std::string* err) {
    if (!grid || !box_off_out || (np > 0 && (!x || !z || !perm_out || (grid->dim == 3 && !y)))) {
        *err = "null argument";
        return PIC_EINVAL;
    }
    if (grid->dim != 2 && grid->dim != 3) {
        *err = "dim must be 2 or 3";
        return PIC_EINVAL;
    }
    if (np < 0 || np >= ((int64_t)1 << 31)) {
        *err = "np out of range";
        return PIC_EINVAL;
    }
    g->dim = grid->dim;
    int64_t nboxes = 1;
    for (int a = 0; a < 3; ++a) {
        bool act = !(grid->dim == 2 && a == 1);
        if (grid->ncell[a] < 1 || grid->ncell[a] > (1 << 24) || grid->box[a] < 1 ||
            grid->ncell[a] % grid->box[a] != 0 || (!act && grid->ncell[a] != 1) ||
            (act && !(grid->dx[a] > 0.0))) {
            *err = "bad grid or box extents";
            return PIC_EINVAL;
        }
        g->n[a] = (int)grid->ncell[a];
        g->bsz[a] = grid->box[a];
        g->nb[a] = g->n[a] / g->bsz[a];
        g->d[a] = act ? grid->dx[a] : 1.0;
        nboxes *= g->nb[a];
    }
    if (nboxes > (int64_t)1 << 30) {
        *err = "too many boxes";
        return PIC_EINVAL;
    }
    g->nboxes = (int)nboxes;
    return PIC_OK;
}

cudaError_t pic_bin_launch(const BinGeom& g, const double* x, const double* y, const double* z,
                           int64_t np, int64_t* box_off, int64_t* perm, int32_t* cursor,
                           cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(box_off, 0, (size_t)(g.nboxes + 1) * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, (size_t)g.nboxes * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    if (np > 0)
        bin_count_kernel<<<bin_grid(np), 256, 0, st>>>(g, x, y, z, np, (unsigned long long*)box_off);
    bin_scan_kernel<<<1, 1024, 0, st>>>(box_off, g.nboxes);
    if (np > 0) bin_scatter_kernel<<<bin_grid(np), 256, 0, st>>>(g, x, y, z, np, box_off, cursor, perm);
    return cudaGetLastError();
}

namespace {
thread_local std::string g_bin_error;
}

extern "C" pic_status pic_bin_particles(const pic_grid_desc* grid, const double* x, const double* y,
                                        const double* z, int64_t np, int64_t* box_off_out,
                                        int64_t* perm_out) {
    BinGeom g;
    pic_status st = pic_bin_validate(grid, x, y, z, np, box_off_out, perm_out, &g, &g_bin_error);
    if (st != PIC_OK) return pic_record_error(st, g_bin_error.c_str());
    cudaStream_t s = (cudaStream_t)grid->stream;
    int32_t* cursor = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&cursor, (size_t)g.nboxes * sizeof(int32_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pic_record_error(PIC_ENOMEM, "cursor allocation failed");
    }
    e = pic_bin_launch(g, x, y, z, np, box_off_out, perm_out, cursor, s);
    cudaError_t e2 = cudaFreeAsync(cursor, s);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        std::string m = std::string("binning failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
        return pic_record_error(PIC_ECUDA, m.c_str());
    }
    return PIC_OK;
}
