// pic_particles.cu -- re-sort of the particles (scan of the per-tile
// histogram written by the particle kernel, warp-aggregated scatter, buffer
// swap), end-of-step bookkeeping, initial keys, per-box counts, and the
// dispatch of the particle kernel over its two arithmetic variants.
#include <algorithm>
#include <atomic>

#include "pic_internal.h"
#include "pic_sync.cuh"

namespace {

// tile key of a global cell (box-major numbering)
__device__ __forceinline__ int tile_key(const SimDev& S, int ix, int iy, int iz) {
    int bx = ix / S.bsz[0], by = iy / S.bsz[1], bz = iz / S.bsz[2];
    int tx = (ix - bx * S.bsz[0]) / S.T[0];
    int ty = (iy - by * S.bsz[1]) / S.T[1];
    int tz = (iz - bz * S.bsz[2]) / S.T[2];
    int b = (bz * S.nb[1] + by) * S.nb[0] + bx;
    return b * S.tiles_per_box + (tz * S.tpb[1] + ty) * S.tpb[0] + tx;
}

__device__ __forceinline__ void warp_hist_add(int32_t* count, int key) {
    unsigned act = __activemask();
    unsigned peers = __match_any_sync(act, key);
    int lane = threadIdx.x & 31;
    if (lane == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
}

}  // namespace

// ---------------------------------------------------------------------------
// re-sort: scan of the per-tile histogram, scatter, end-of-step bookkeeping
// ---------------------------------------------------------------------------
// multi-simulation launches: blockIdx.y indexes the slot list (nullptr: slot 0);
// sp_idx < 0 takes the species from blockIdx.x (scan, swap) or blockIdx.z (scatter)
__global__ void __launch_bounds__(1024) pic_scan_kernel(SimDev* __restrict__ sims,
                                                        const int* __restrict__ slots, int sp_idx) {
    SimDev& S = sims[slots ? slots[blockIdx.y] : 0];
    if (sp_idx < 0) sp_idx = blockIdx.x;
    if (sp_idx >= S.nsp) return;
    SpeciesDev& sp = S.sp[sp_idx];
    const int N = S.ntiles + 1;  // tiles plus the bucket of removed particles
    __shared__ int64_t s_part[1024];
    __shared__ int64_t s_np_prev;
    if (threadIdx.x == 0) s_np_prev = sp.off[S.ntiles];  // kept count of the buffer just pushed
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per, i1 = min(N, i0 + per);
    int64_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += sp.count[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    // inclusive Hillis-Steele scan of the partial sums
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int64_t v = (threadIdx.x >= (unsigned)o) ? s_part[threadIdx.x - o] : 0;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = s_part[threadIdx.x] - sum;
    for (int i = i0; i < i1; ++i) {
        int c = sp.count[i];
        sp.off[i] = run;
        run += c;
        sp.count[i] = 0;
        sp.cursor[i] = 0;
    }
    if (threadIdx.x == blockDim.x - 1) sp.off[N] = s_part[blockDim.x - 1];
    if (threadIdx.x == 0) *sp.np_prev = s_np_prev;
}

// The same scan for large tile counts, in three launches over blocks of 1024
// entries: block sums; their exclusive scan in one block (which also records
// the kept count of the buffer just pushed and the total); then each block's
// own exclusive scan plus its offset, clearing count and cursor.
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const int64_t before = warp > 0 ? s_warp[warp - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(kScanBlock) pic_scan_part_kernel(SimDev* __restrict__ sims, int sp_idx) {
    SimDev& S = sims[0];
    SpeciesDev& sp = S.sp[sp_idx];
    const int N = S.ntiles + 1;
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    int64_t total;
    block_exclusive_scan(i < N ? (int64_t)sp.count[i] : 0, &total);
    if (threadIdx.x == 0) S.scan_part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) pic_scan_top_kernel(SimDev* __restrict__ sims, int sp_idx, int nparts) {
    SimDev& S = sims[0];
    SpeciesDev& sp = S.sp[sp_idx];
    const int per = (nparts + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per, i1 = min(nparts, i0 + per);
    int64_t sum = 0;
    for (int i = i0; i < i1; ++i) sum += S.scan_part[i];
    int64_t total;
    int64_t run = block_exclusive_scan(sum, &total);
    if (threadIdx.x == 0) *sp.np_prev = sp.off[S.ntiles];  // kept count of the buffer just pushed
    for (int i = i0; i < i1; ++i) {
        const int64_t c = S.scan_part[i];
        S.scan_part[i] = run;
        run += c;
    }
    if (threadIdx.x == 0) sp.off[S.ntiles + 1] = total;
}

__global__ void __launch_bounds__(kScanBlock) pic_scan_final_kernel(SimDev* __restrict__ sims, int sp_idx) {
    SimDev& S = sims[0];
    SpeciesDev& sp = S.sp[sp_idx];
    const int N = S.ntiles + 1;
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int64_t c = i < N ? (int64_t)sp.count[i] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(c, &total);
    if (i < N) {
        sp.off[i] = S.scan_part[blockIdx.x] + ex;
        sp.count[i] = 0;
        sp.cursor[i] = 0;
    }
}

template <int DIM>
__global__ void pic_scatter_kernel(SimDev* __restrict__ sims, const int* __restrict__ slots, int sp_idx) {
    const SimDev& S = sims[slots ? slots[blockIdx.y] : 0];
    if (sp_idx < 0) sp_idx = blockIdx.z;
    if (sp_idx >= S.nsp) return;
    const SpeciesDev& sp = S.sp[sp_idx];
    const int64_t np = *sp.np_prev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < np; p0 += stride) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= np) break;
        const int k = sp.key[p];
        if (k < 0 || k > S.ntiles) {
            atomicOr(S.err, PIC_DERR_SCATTER);
            continue;
        }
        if (k == S.ntiles) continue;  // removed by the absorbing boundary
        unsigned act = __activemask();
        unsigned peers = __match_any_sync(act, k);
        int lane = threadIdx.x & 31;
        int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(sp.cursor + k, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        int rank = __popc(peers & ((1u << lane) - 1u));
        const int64_t dst = sp.off[k] + base + rank;
#pragma unroll
        for (int a = 0; a < 7; ++a) {
            if (DIM == 2 && a == 1) continue;
            sp.alt[a][dst] = sp.cur[a][p];
        }
        sp.id_alt[dst] = sp.id[p];
    }
}

__global__ void pic_swap_kernel(SimDev* __restrict__ sims, const int* __restrict__ slots, int sp_idx) {
    SimDev& S = sims[slots ? slots[blockIdx.y] : 0];
    if (sp_idx < 0) sp_idx = blockIdx.x;
    if (sp_idx >= S.nsp || threadIdx.x != 0) return;
    SpeciesDev& sp = S.sp[sp_idx];
    for (int a = 0; a < 7; ++a) {
        double* t = sp.cur[a];
        sp.cur[a] = sp.alt[a];
        sp.alt[a] = t;
    }
    int64_t* ti = sp.id;
    sp.id = sp.id_alt;
    sp.id_alt = ti;
}

__global__ void pic_finish_kernel(SimDev* __restrict__ sims, const int* __restrict__ slots,
                                  const SchedDev* __restrict__ sd) {
    if (blockIdx.y == 0) {
        const int nlists = sd->meta[0];
        for (int i = threadIdx.x; i < nlists; i += blockDim.x) sd->head[i] = 0;
    }
    if (threadIdx.x == 0) *sims[slots ? slots[blockIdx.y] : 0].step += 1;
}

template <int DIM>
__global__ void pic_initial_keys_kernel(SimDev* __restrict__ sims, int sp_idx, int64_t np) {
    const SimDev& S = sims[0];
    const SpeciesDev& sp = S.sp[sp_idx];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x; p0 < np; p0 += stride) {
        const int64_t p = p0 + threadIdx.x;
        if (p >= np) break;
        int ix = min(max(__double2int_rd(sp.cur[0][p]), 0), S.n[0] - 1);
        int iy = (DIM == 3) ? min(max(__double2int_rd(sp.cur[1][p]), 0), S.n[1] - 1) : 0;
        int iz = min(max(__double2int_rd(sp.cur[2][p]), 0), S.n[2] - 1);
        int key = tile_key(S, ix, iy, iz);
        sp.key[p] = key;
        warp_hist_add(sp.count, key);
    }
}

template <int DIM>
__global__ void pic_keys_range_kernel(SimDev* __restrict__ sims, int sp_idx, int64_t p0, int64_t p1) {
    const SimDev& S = sims[0];
    const SpeciesDev& sp = S.sp[sp_idx];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q0 = p0 + (int64_t)blockIdx.x * blockDim.x; q0 < p1; q0 += stride) {
        const int64_t p = q0 + threadIdx.x;
        if (p >= p1) break;
        int ix = min(max(__double2int_rd(sp.cur[0][p]), 0), S.n[0] - 1);
        int iy = (DIM == 3) ? min(max(__double2int_rd(sp.cur[1][p]), 0), S.n[1] - 1) : 0;
        int iz = min(max(__double2int_rd(sp.cur[2][p]), 0), S.n[2] - 1);
        int key = tile_key(S, ix, iy, iz);
        sp.key[p] = key;
        warp_hist_add(sp.count, key);
    }
}

__global__ void pic_box_counts_kernel(const SimDev* __restrict__ sims, int64_t* out) {
    const SimDev& S = sims[0];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < S.nboxes; b += gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int s = 0; s < S.nsp; ++s)
            c += S.sp[s].off[(b + 1) * S.tiles_per_box] - S.sp[s].off[b * S.tiles_per_box];
        out[b] = c;
    }
}

// physical position -> global cell units X = x / d, wrapped into [0, n)
__global__ void pic_to_cells_kernel(double* p, int64_t np, double d, int n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        double X = p[i] / d;
        if (X < 0.0) X += (double)n;
        if (X >= (double)n) X -= (double)n;
        p[i] = X;
    }
}

__global__ void pic_scale_copy_kernel(const double* __restrict__ s, double* __restrict__ d,
                                      int64_t n, double f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i] * f;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int pic_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// particle kernel: dispatch on the arithmetic of the push and the dimensionality
cudaError_t pic_launch_particles(int dim, int order, const LaunchCfg& cfg, size_t smem,
                                 const SchedDev* sched, SimDev* sims, cudaStream_t st) {
    if (cfg.prec == 2)
        return dim == 3 ? pic_launch_particles_p2_d3(order, cfg, smem, sched, sims, st)
                        : pic_launch_particles_p2_d2(order, cfg, smem, sched, sims, st);
    if (cfg.prec == 1)
        return dim == 3 ? pic_launch_particles_p1_d3(order, cfg, smem, sched, sims, st)
                        : pic_launch_particles_p1_d2(order, cfg, smem, sched, sims, st);
    return dim == 3 ? pic_launch_particles_p0_d3(order, cfg, smem, sched, sims, st)
                    : pic_launch_particles_p0_d2(order, cfg, smem, sched, sims, st);
}

cudaError_t pic_prepare_particles(int dim, int order, size_t smem) {
    cudaError_t e;
    if (dim == 3) {
        e = pic_prepare_particles_p0_d3(order, smem);
        if (e == cudaSuccess) e = pic_prepare_particles_p1_d3(order, smem);
        if (e == cudaSuccess) e = pic_prepare_particles_p2_d3(order, smem);
    } else {
        e = pic_prepare_particles_p0_d2(order, smem);
        if (e == cudaSuccess) e = pic_prepare_particles_p1_d2(order, smem);
        if (e == cudaSuccess) e = pic_prepare_particles_p2_d2(order, smem);
    }
    return e;
}

int pic_particle_occupancy(int dim, int order, int minb, int ppt, int threads, size_t smem, int prec) {
    if (prec == 2)
        return dim == 3 ? pic_particle_occupancy_p2_d3(order, minb, ppt, threads, smem)
                        : pic_particle_occupancy_p2_d2(order, minb, ppt, threads, smem);
    if (prec == 1)
        return dim == 3 ? pic_particle_occupancy_p1_d3(order, minb, ppt, threads, smem)
                        : pic_particle_occupancy_p1_d2(order, minb, ppt, threads, smem);
    return dim == 3 ? pic_particle_occupancy_p0_d3(order, minb, ppt, threads, smem)
                    : pic_particle_occupancy_p0_d2(order, minb, ppt, threads, smem);
}

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (int64_t)pic_sm_count() * 32) b = (int64_t)pic_sm_count() * 32;
    return (int)b;
}

cudaError_t pic_launch_sort(const SimDev* dsim, const SimDev& hsim, int sp, cudaStream_t st) {
    SimDev* d = const_cast<SimDev*>(dsim);
    const int64_t N = (int64_t)hsim.ntiles + 1;
    const int64_t nparts = (N + kScanBlock - 1) / kScanBlock;
    if (N > 8 * kScanBlock && hsim.scan_part && nparts <= hsim.scan_part_cap) {
        pic_scan_part_kernel<<<(int)nparts, kScanBlock, 0, st>>>(d, sp);
        pic_scan_top_kernel<<<1, kScanBlock, 0, st>>>(d, sp, (int)nparts);
        pic_scan_final_kernel<<<(int)nparts, kScanBlock, 0, st>>>(d, sp);
    } else {
        pic_scan_kernel<<<1, 1024, 0, st>>>(d, nullptr, sp);
    }
    int64_t cap = hsim.sp[sp].cap;
    if (hsim.dim == 3) pic_scatter_kernel<3><<<grid_for(cap, 256), 256, 0, st>>>(d, nullptr, sp);
    else pic_scatter_kernel<2><<<grid_for(cap, 256), 256, 0, st>>>(d, nullptr, sp);
    pic_swap_kernel<<<1, 32, 0, st>>>(d, nullptr, sp);
    return cudaGetLastError();
}

cudaError_t pic_launch_sort_multi(SimDev* sims, const int* slots, int nslots, int dim, int64_t max_cap,
                                  cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    pic_scan_kernel<<<dim3(PIC_MAXSP, nslots), 1024, 0, st>>>(sims, slots, -1);
    const dim3 g(grid_for(max_cap, 256) / 4 + 1, nslots, PIC_MAXSP);
    if (dim == 3) pic_scatter_kernel<3><<<g, 256, 0, st>>>(sims, slots, -1);
    else pic_scatter_kernel<2><<<g, 256, 0, st>>>(sims, slots, -1);
    pic_swap_kernel<<<dim3(PIC_MAXSP, nslots), 32, 0, st>>>(sims, slots, -1);
    return cudaGetLastError();
}

cudaError_t pic_launch_finish_multi(SimDev* sims, const int* slots, int nslots, const SchedDev* sched,
                                    cudaStream_t st) {
    if (nslots <= 0) return cudaSuccess;
    pic_finish_kernel<<<dim3(1, nslots), 256, 0, st>>>(sims, slots, sched);
    return cudaGetLastError();
}

cudaError_t pic_launch_initial_keys(const SimDev* dsim, const SimDev& hsim, int sp, int64_t np,
                                    cudaStream_t st) {
    SimDev* d = const_cast<SimDev*>(dsim);
    if (np > 0) {
        if (hsim.dim == 3) pic_initial_keys_kernel<3><<<grid_for(np, 256), 256, 0, st>>>(d, sp, np);
        else pic_initial_keys_kernel<2><<<grid_for(np, 256), 256, 0, st>>>(d, sp, np);
    }
    return cudaGetLastError();
}

cudaError_t pic_launch_keys_range(const SimDev* dsim, const SimDev& hsim, int sp, int64_t p0, int64_t p1,
                                  cudaStream_t st) {
    SimDev* d = const_cast<SimDev*>(dsim);
    if (p1 > p0) {
        if (hsim.dim == 3) pic_keys_range_kernel<3><<<grid_for(p1 - p0, 256), 256, 0, st>>>(d, sp, p0, p1);
        else pic_keys_range_kernel<2><<<grid_for(p1 - p0, 256), 256, 0, st>>>(d, sp, p0, p1);
    }
    return cudaGetLastError();
}

cudaError_t pic_launch_finish(SimDev* dsim, const SchedDev* sched, cudaStream_t st) {
    pic_finish_kernel<<<1, 256, 0, st>>>(dsim, nullptr, sched);
    return cudaGetLastError();
}

cudaError_t pic_launch_box_counts(const SimDev* dsim, const SimDev& hsim, int64_t* out,
                                  cudaStream_t st) {
    pic_box_counts_kernel<<<grid_for(hsim.nboxes, 256), 256, 0, st>>>(dsim, out);
    return cudaGetLastError();
}

// One-time scramble of a species' input order.  Within a tile the re-sort
// keeps the relative order of the particles that stay, so an input generated
// cell by cell would keep a warp's 32 particles in one cell for the whole run,
// all adding to the same J entries, and the shared-memory atomics would
// serialise.  dst[j] = src[(j * P) mod np] with P = 2^31 + 11, a prime above
// any species size (np <= 2^31, so gcd(P, np) = 1), is a bijection that spreads
// consecutive inputs apart; j * P < 2^63 needs no wider product.
struct PermArrays {
    const double* src[7];
    double* dst[7];
    const int64_t* id_src;
    int64_t* id_dst;
};

__global__ void pic_permute_kernel(PermArrays A, int64_t np, int skip) {
    const uint64_t P = 2147483659ull;  // 2^31 + 11, prime
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < np;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)(((uint64_t)j * P) % (uint64_t)np);
#pragma unroll
        for (int a = 0; a < 7; ++a)
            if (a != skip) A.dst[a][j] = A.src[a][i];
        A.id_dst[j] = A.id_src[i];
    }
}

cudaError_t pic_launch_permute(double* const dst[7], const double* const src[7], int64_t* id_dst,
                               const int64_t* id_src, int64_t np, int skip, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    PermArrays A;
    for (int a = 0; a < 7; ++a) {
        A.src[a] = src[a];
        A.dst[a] = dst[a];
    }
    A.id_src = id_src;
    A.id_dst = id_dst;
    const int64_t nb = std::min<int64_t>((np + 255) / 256, (int64_t)pic_sm_count() * 32);
    pic_permute_kernel<<<(int)nb, 256, 0, st>>>(A, np, skip);
    return cudaGetLastError();
}

cudaError_t pic_launch_to_cells(double* p, int64_t np, double d, int n, cudaStream_t st) {
    if (np > 0) pic_to_cells_kernel<<<grid_for(np, 256), 256, 0, st>>>(p, np, d, n);
    return cudaGetLastError();
}

cudaError_t pic_launch_from_cells(const double* src, double* dst, int64_t np, double d,
                                  cudaStream_t st) {
    if (np > 0) pic_scale_copy_kernel<<<grid_for(np, 256), 256, 0, st>>>(src, dst, np, d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bounded-wait self-test: the particle kernel's mbarrier wait on a barrier that
// nothing arrives at.  It must give up after limit_ns, record the error and
// return, leaving the context usable.
// ---------------------------------------------------------------------------
__global__ void pic_selftest_wait_kernel(int32_t* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, limit_ns)) atomicOr(err, PIC_DERR_WAIT_TIMEOUT);
}

cudaError_t pic_launch_selftest_wait(int32_t* err, uint64_t limit_ns, cudaStream_t st) {
    pic_selftest_wait_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}
