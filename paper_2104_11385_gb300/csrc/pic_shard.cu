// pic_shard.cu -- box sharding of one simulation across ranks (include/pic_shard.h):
// the ghost-cell plans of Sec. 2.1 of arXiv 2104.11385 (pure host), packing and
// unpacking of field values at listed cells, the field update restricted to a
// rank's boxes, and the migration of particles whose box another rank owns
// (the redistribution of Sec. 2.2 uses the same path).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/pic_shard.h"
#include "pic_internal.h"
#include "pic_sim.h"

namespace {

struct Geom {
    int dim;
    int64_t n[3];
    int bsz[3], nb[3];
    int64_t nboxes;
};

pic_status geom_from(const pic_grid_desc* g, Geom* o, const char** why) {
    if (!g || (g->dim != 2 && g->dim != 3)) {
        *why = "grid: dim must be 2 or 3";
        return PIC_EINVAL;
    }
    o->dim = g->dim;
    o->nboxes = 1;
    for (int a = 0; a < 3; ++a) {
        const bool act = !(g->dim == 2 && a == 1);
        if (!act && (g->ncell[a] != 1 || g->box[a] != 1)) {
            *why = "grid: 2D runs need ncell[1] == box[1] == 1";
            return PIC_EINVAL;
        }
        if (g->ncell[a] < 1 || g->ncell[a] > (1 << 20) || g->box[a] < 1 || g->ncell[a] % g->box[a] != 0) {
            *why = "grid: box extents must divide ncell";
            return PIC_EINVAL;
        }
        o->n[a] = g->ncell[a];
        o->bsz[a] = g->box[a];
        o->nb[a] = (int)(g->ncell[a] / g->box[a]);
        o->nboxes *= o->nb[a];
    }
    return PIC_OK;
}

// periodic distance (in cells) from coordinate x to the cell interval [c0, c1) of a domain of n cells
int64_t pdist(int64_t x, int64_t c0, int64_t c1, int64_t n) {
    int64_t best = n;
    for (int64_t s = -n; s <= n; s += n) {
        const int64_t lo = c0 + s, hi = c1 + s;
        const int64_t d = x < lo ? lo - x : (x >= hi ? x - hi + 1 : 0);
        best = std::min(best, d);
    }
    return best;
}

pic_status host_fail(pic_status st, const char* msg) { return pic_record_error(st, msg); }

// ---- device side --------------------------------------------------------
__device__ __forceinline__ int64_t dense_to_padded(const SimDev& S, int64_t d) {
    const int i = (int)(d % S.n[0]);
    const int j = (int)((d / S.n[0]) % S.n[1]);
    const int k = (int)(d / ((int64_t)S.n[0] * S.n[1]));
    return pidx(S, i, j, k);
}

__global__ void pack_kernel(const SimDev* __restrict__ sims, int c0, int nc, const int64_t* __restrict__ cells,
                            int64_t n, double* __restrict__ buf) {
    const SimDev& S = sims[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = dense_to_padded(S, cells[q]);
        for (int c = 0; c < nc; ++c) buf[(int64_t)c * n + q] = S.F[c0 + c][o];
    }
}

__global__ void unpack_kernel(const SimDev* __restrict__ sims, int c0, int nc, const int64_t* __restrict__ cells,
                              int64_t n, const double* __restrict__ buf, int add) {
    const SimDev& S = sims[0];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = dense_to_padded(S, cells[q]);
        for (int c = 0; c < nc; ++c) {
            const double v = buf[(int64_t)c * n + q];
            if (add) S.F[c0 + c][o] += v;
            else S.F[c0 + c][o] = v;
        }
    }
}

// destination rank of particle p, or -1 when it stays (or leaves the domain)
__device__ __forceinline__ int leaving_to(const SimDev& S, const SpeciesDev& sp, int64_t p) {
    const int k = sp.key[p];
    if (k < 0 || k >= S.ntiles) return -1;
    const int o = S.owner[k / S.tiles_per_box];
    return o == S.rank ? -1 : o;
}

__global__ void leaving_count_kernel(const SimDev* __restrict__ sims, int spi, int64_t np, int nranks,
                                     int32_t* __restrict__ counts) {
    const SimDev& S = sims[0];
    const SpeciesDev& sp = S.sp[spi];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int d = leaving_to(S, sp, p);
        if (d >= 0 && d < nranks) atomicAdd(counts + d, 1);
        else if (d >= nranks) atomicOr(S.err, PIC_DERR_BOUNDS);
    }
}

struct OutBox {
    double* soa[7];
    int64_t* id;
    const int64_t* off;  // [nranks] start of each destination's group
    int32_t* cursor;     // [nranks]
};

__global__ void leaving_scatter_kernel(SimDev* __restrict__ sims, int spi, int64_t np, int nranks, OutBox ob) {
    SimDev& S = sims[0];
    SpeciesDev& sp = S.sp[spi];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int d = leaving_to(S, sp, p);
        if (d < 0 || d >= nranks) continue;
        const int k = sp.key[p];
        const int64_t slot = ob.off[d] + atomicAdd(ob.cursor + d, 1);
#pragma unroll
        for (int a = 0; a < 7; ++a) ob.soa[a][slot] = sp.cur[a][p];
        ob.id[slot] = sp.id[p];
        // out of this rank's sort: into the bucket of removed particles
        sp.key[p] = S.ntiles;
        atomicSub(sp.count + k, 1);
        atomicAdd(sp.count + S.ntiles, 1);
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    b = std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)pic_sm_count() * 16));
    return (int)b;
}

#define SCU(s, call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            std::string m_ = std::string(#call) + " failed: " + cudaGetErrorString(e_); \
            return pic_sim_fail((s), PIC_ECUDA, m_.c_str());                          \
        }                                                                             \
    } while (0)
#define STRY(x)                         \
    do {                                \
        pic_status st_ = (x);           \
        if (st_ != PIC_OK) return st_;  \
    } while (0)

pic_status sharded(pic_sim* s) {
    STRY(pic_sim_check(s));
    if (s->rank < 0) return pic_sim_fail(s, PIC_ESTATE, "the handle is not sharded (pic_shard_set_owner)");
    return PIC_OK;
}

pic_status read_i64(pic_sim* s, const int64_t* d, int64_t* h) {
    SCU(s, cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream));
    SCU(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

template <class T>
pic_status grow(pic_sim* s, T** p, int64_t n) {
    void* q = nullptr;
    STRY(pic_sim_dalloc(s, &q, (size_t)std::max<int64_t>(n, 1) * sizeof(T)));
    *p = (T*)q;
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_shard_halo_cells(const pic_grid_desc* grid, const int32_t* owner, int own, int near, int halo,
                                int64_t* cells_out, int64_t* n_out) {
    Geom G;
    const char* why = "";
    if (geom_from(grid, &G, &why) != PIC_OK) return host_fail(PIC_EINVAL, why);
    if (!owner || !n_out || halo < 1 || halo > 8 || own < 0 || near < 0 || own == near)
        return host_fail(PIC_EINVAL, "pic_shard_halo_cells: bad arguments");
    for (int a = 0; a < 3; ++a)
        if (!(G.dim == 2 && a == 1) && G.bsz[a] < halo)
            return host_fail(PIC_EINVAL, "pic_shard_halo_cells: a box extent is below the halo");
    for (int64_t b = 0; b < G.nboxes; ++b)
        if (owner[b] < 0) return host_fail(PIC_EINVAL, "pic_shard_halo_cells: negative owner");
    std::vector<int64_t> out;
    std::vector<uint8_t> mask;
    std::vector<uint8_t> nearf[3];
    const int64_t vol = (int64_t)G.bsz[0] * G.bsz[1] * G.bsz[2];
    for (int64_t b = 0; b < G.nboxes; ++b) {
        if (owner[b] != own) continue;
        const int bi[3] = {(int)(b % G.nb[0]), (int)((b / G.nb[0]) % G.nb[1]), (int)(b / ((int64_t)G.nb[0] * G.nb[1]))};
        // neighbour boxes (periodic), each once; a box extent >= halo keeps
        // every cell within halo of this box inside them
        std::vector<int64_t> nbrs;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = (G.dim == 3 ? -1 : 0); dy <= (G.dim == 3 ? 1 : 0); ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int d[3] = {dx, dy, dz};
                    int64_t nb = 0, mul = 1;
                    for (int a = 0; a < 3; ++a) {
                        const int c = ((bi[a] + d[a]) % G.nb[a] + G.nb[a]) % G.nb[a];
                        nb += c * mul;
                        mul *= G.nb[a];
                    }
                    if (owner[nb] == near && std::find(nbrs.begin(), nbrs.end(), nb) == nbrs.end())
                        nbrs.push_back(nb);
                }
        if (nbrs.empty()) continue;
        mask.assign((size_t)vol, 0);
        for (int64_t nb : nbrs) {
            const int ni[3] = {(int)(nb % G.nb[0]), (int)((nb / G.nb[0]) % G.nb[1]),
                               (int)(nb / ((int64_t)G.nb[0] * G.nb[1]))};
            for (int a = 0; a < 3; ++a) {
                nearf[a].assign(G.bsz[a], 0);
                const int64_t c0 = (int64_t)ni[a] * G.bsz[a], c1 = c0 + G.bsz[a];
                for (int x = 0; x < G.bsz[a]; ++x)
                    nearf[a][x] = pdist((int64_t)bi[a] * G.bsz[a] + x, c0, c1, G.n[a]) <= halo ? 1 : 0;
            }
            for (int z = 0; z < G.bsz[2]; ++z)
                for (int y = 0; y < G.bsz[1]; ++y)
                    for (int x = 0; x < G.bsz[0]; ++x)
                        if (nearf[0][x] && nearf[1][y] && nearf[2][z])
                            mask[((int64_t)z * G.bsz[1] + y) * G.bsz[0] + x] = 1;
        }
        for (int z = 0; z < G.bsz[2]; ++z)
            for (int y = 0; y < G.bsz[1]; ++y)
                for (int x = 0; x < G.bsz[0]; ++x)
                    if (mask[((int64_t)z * G.bsz[1] + y) * G.bsz[0] + x]) {
                        const int64_t gi = (int64_t)bi[0] * G.bsz[0] + x, gj = (int64_t)bi[1] * G.bsz[1] + y,
                                      gk = (int64_t)bi[2] * G.bsz[2] + z;
                        out.push_back((gk * G.n[1] + gj) * G.n[0] + gi);
                    }
    }
    std::sort(out.begin(), out.end());
    *n_out = (int64_t)out.size();
    if (cells_out && !out.empty()) std::copy(out.begin(), out.end(), cells_out);
    return PIC_OK;
}

pic_status pic_shard_moved_cells(const pic_grid_desc* grid, const int32_t* old_owner, const int32_t* new_owner,
                                 int src, int dst, int64_t* cells_out, int64_t* n_out) {
    Geom G;
    const char* why = "";
    if (geom_from(grid, &G, &why) != PIC_OK) return host_fail(PIC_EINVAL, why);
    if (!old_owner || !new_owner || !n_out || src < 0 || dst < 0)
        return host_fail(PIC_EINVAL, "pic_shard_moved_cells: bad arguments");
    std::vector<int64_t> out;
    for (int64_t b = 0; b < G.nboxes; ++b) {
        if (old_owner[b] != src || new_owner[b] != dst || src == dst) continue;
        const int bi[3] = {(int)(b % G.nb[0]), (int)((b / G.nb[0]) % G.nb[1]), (int)(b / ((int64_t)G.nb[0] * G.nb[1]))};
        for (int z = 0; z < G.bsz[2]; ++z)
            for (int y = 0; y < G.bsz[1]; ++y)
                for (int x = 0; x < G.bsz[0]; ++x) {
                    const int64_t gi = (int64_t)bi[0] * G.bsz[0] + x, gj = (int64_t)bi[1] * G.bsz[1] + y,
                                  gk = (int64_t)bi[2] * G.bsz[2] + z;
                    out.push_back((gk * G.n[1] + gj) * G.n[0] + gi);
                }
    }
    std::sort(out.begin(), out.end());
    *n_out = (int64_t)out.size();
    if (cells_out && !out.empty()) std::copy(out.begin(), out.end(), cells_out);
    return PIC_OK;
}

pic_status pic_shard_set_owner(pic_sim* s, const int32_t* owner, int rank) {
    STRY(pic_sim_check(s));
    const int64_t nb = s->h.nboxes;
    if (!owner || rank < 0 || rank >= (1 << 20)) return pic_sim_fail(s, PIC_EINVAL, "bad owner map or rank");
    for (int64_t b = 0; b < nb; ++b)
        if (owner[b] < 0 || owner[b] >= (1 << 20)) return pic_sim_fail(s, PIC_EINVAL, "owner out of range");
    if (s->stepped) {
        STRY(pic_sim_sync(s));
        STRY(pic_sim_pull(s));
    }
    if (!s->d_owner) {
        void* p = nullptr;
        STRY(pic_sim_dalloc(s, &p, (size_t)nb * sizeof(int32_t)));
        s->d_owner = (int32_t*)p;
    }
    s->owner.assign(owner, owner + nb);
    s->rank = rank;
    SCU(s, cudaMemcpyAsync(s->d_owner, s->owner.data(), nb * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    s->h.owner = s->d_owner;
    s->h.rank = rank;
    s->graph_dirty = true;
    return pic_sim_upload(s);
}

pic_status pic_shard_pack(pic_sim* s, int c0, int nc, const int64_t* cells, int64_t n, double* buf) {
    STRY(pic_sim_check(s));
    if (c0 < 0 || nc < 1 || c0 + nc > PIC_NCOMP || n < 0 || (n > 0 && (!cells || !buf)))
        return pic_sim_fail(s, PIC_EINVAL, "pic_shard_pack: bad arguments");
    if (!s->stepped) STRY(pic_sim_upload(s));
    if (n > 0) {
        pack_kernel<<<grid_for(n), 256, 0, s->stream>>>(s->d, c0, nc, cells, n, buf);
        SCU(s, cudaGetLastError());
    }
    return pic_sim_sync(s);
}

pic_status pic_shard_unpack(pic_sim* s, int c0, int nc, const int64_t* cells, int64_t n, const double* buf,
                            int add) {
    STRY(pic_sim_check(s));
    if (c0 < 0 || nc < 1 || c0 + nc > PIC_NCOMP || n < 0 || (n > 0 && (!cells || !buf)))
        return pic_sim_fail(s, PIC_EINVAL, "pic_shard_unpack: bad arguments");
    if (!s->stepped) STRY(pic_sim_upload(s));
    if (n > 0) {
        unpack_kernel<<<grid_for(n), 256, 0, s->stream>>>(s->d, c0, nc, cells, n, buf, add ? 1 : 0);
        SCU(s, cudaGetLastError());
    }
    return pic_sim_sync(s);
}

pic_status pic_shard_push(pic_sim* s) {
    STRY(sharded(s));
    STRY(pic_sim_ensure_ready(s));
    STRY(pic_sim_launch_push(s));
    SCU(s, pic_launch_fold(s->d, s->h, s->stream));
    return PIC_OK;
}

pic_status pic_shard_field_stage(pic_sim* s, int stage) {
    STRY(sharded(s));
    if (stage < 0 || stage > 3) return pic_sim_fail(s, PIC_EINVAL, "stage must be 0..3");
    STRY(pic_sim_ensure_ready(s));
    SCU(s, pic_launch_field_stage(s->d, s->h, stage, s->stream));
    return PIC_OK;
}

pic_status pic_shard_rekey(pic_sim* s) {
    STRY(sharded(s));
    STRY(pic_sim_ensure_ready(s));
    STRY(pic_sim_sync(s));
    STRY(pic_sim_pull(s));
    for (int i = 0; i < s->h.nsp; ++i) {
        int64_t np = 0;
        STRY(read_i64(s, s->h.sp[i].off + s->h.ntiles, &np));
        SCU(s, pic_launch_keys_range(s->d, s->h, i, 0, np, s->stream));
    }
    return pic_sim_sync(s);
}

pic_status pic_shard_take_leaving(pic_sim* s, int spi, int nranks, int64_t* counts_out) {
    STRY(sharded(s));
    if (spi < 0 || spi >= s->h.nsp || nranks < 1 || nranks > (1 << 20) || !counts_out)
        return pic_sim_fail(s, PIC_EINVAL, "pic_shard_take_leaving: bad arguments");
    for (int32_t o : s->owner)
        if (o >= nranks) return pic_sim_fail(s, PIC_EINVAL, "an owner is not below nranks");
    STRY(pic_sim_sync(s));
    STRY(pic_sim_pull(s));
    SpeciesDev& sp = s->h.sp[spi];
    int64_t np = 0;
    STRY(read_i64(s, sp.off + s->h.ntiles, &np));
    // per-destination counts, cursors and offsets
    if (!s->d_out_count || (int64_t)s->out_off.size() < nranks + 1) {
        pic_sim_dfree(s, s->d_out_count);
        pic_sim_dfree(s, s->d_out_cursor);
        s->d_out_count = s->d_out_cursor = nullptr;
        // int32 counts | int32 cursors | int64 offsets (at an 8-byte boundary: 2(n+1) int32 before them)
        STRY(grow(s, &s->d_out_count, 4 * (int64_t)(nranks + 1)));
        s->d_out_cursor = s->d_out_count + (nranks + 1);
        s->out_off.assign(nranks + 1, 0);
    }
    const int nr_alloc = (int)s->out_off.size() - 1;
    int64_t* d_off = reinterpret_cast<int64_t*>(s->d_out_count + 2 * (nr_alloc + 1));
    SCU(s, cudaMemsetAsync(s->d_out_count, 0, 2 * (nr_alloc + 1) * sizeof(int32_t), s->stream));
    leaving_count_kernel<<<grid_for(np), 256, 0, s->stream>>>(s->d, spi, np, nranks, s->d_out_count);
    SCU(s, cudaGetLastError());
    std::vector<int32_t> cnt(nranks);
    SCU(s, cudaMemcpyAsync(cnt.data(), s->d_out_count, nranks * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    STRY(pic_sim_sync(s));
    s->out_off.assign(nr_alloc + 1, 0);
    for (int r = 0; r < nranks; ++r) s->out_off[r + 1] = s->out_off[r] + cnt[r];
    for (int r = nranks; r < nr_alloc; ++r) s->out_off[r + 1] = s->out_off[r];
    const int64_t total = s->out_off[nr_alloc];
    if (total > s->out_cap) {
        for (int a = 0; a < 7; ++a) pic_sim_dfree(s, s->out_soa[a]);
        pic_sim_dfree(s, s->out_id);
        const int64_t cap = std::max<int64_t>(total, s->out_cap + s->out_cap / 2);
        for (int a = 0; a < 7; ++a) STRY(grow(s, &s->out_soa[a], cap));
        STRY(grow(s, &s->out_id, cap));
        s->out_cap = cap;
    }
    if (total > 0) {
        SCU(s, cudaMemcpyAsync(d_off, s->out_off.data(), nranks * sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
        OutBox ob;
        for (int a = 0; a < 7; ++a) ob.soa[a] = s->out_soa[a];
        ob.id = s->out_id;
        ob.off = d_off;
        ob.cursor = s->d_out_cursor;
        leaving_scatter_kernel<<<grid_for(np), 256, 0, s->stream>>>(s->d, spi, np, nranks, ob);
        SCU(s, cudaGetLastError());
    }
    STRY(pic_sim_sync(s));
    for (int r = 0; r < nranks; ++r) counts_out[r] = cnt[r];
    s->out_species = spi;
    return PIC_OK;
}

pic_status pic_shard_read_leaving(pic_sim* s, int spi, int dst, double* const soa_out[7], int64_t* ids_out) {
    STRY(sharded(s));
    if (spi != s->out_species || dst < 0 || dst + 1 >= (int)s->out_off.size() || !soa_out)
        return pic_sim_fail(s, PIC_EINVAL, "pic_shard_read_leaving: no such outbox group");
    const int64_t b = s->out_off[dst], n = s->out_off[dst + 1] - b;
    if (n == 0) return PIC_OK;
    for (int a = 0; a < 7; ++a)
        if (soa_out[a])
            SCU(s, cudaMemcpyAsync(soa_out[a], s->out_soa[a] + b, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                   s->stream));
    if (ids_out)
        SCU(s, cudaMemcpyAsync(ids_out, s->out_id + b, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s->stream));
    return pic_sim_sync(s);
}

pic_status pic_shard_add_arriving(pic_sim* s, int spi, int64_t n, const double* const soa[7], const int64_t* ids) {
    STRY(sharded(s));
    if (spi < 0 || spi >= s->h.nsp || n < 0 || (n > 0 && (!soa || !ids)))
        return pic_sim_fail(s, PIC_EINVAL, "pic_shard_add_arriving: bad arguments");
    for (int a = 0; a < 7 && n > 0; ++a)
        if (!soa[a]) return pic_sim_fail(s, PIC_EINVAL, "pic_shard_add_arriving: missing array");
    if (n == 0) return PIC_OK;
    STRY(pic_sim_sync(s));
    STRY(pic_sim_pull(s));
    SpeciesDev& sp = s->h.sp[spi];
    int64_t np = 0;
    STRY(read_i64(s, sp.off + s->h.ntiles, &np));
    const int64_t need = np + n;
    if (need > ((int64_t)1 << 31)) return pic_sim_fail(s, PIC_ENOMEM, "a species would exceed 2^31 particles");
    if (need > sp.cap) {
        // grow: kept particles, their ids and this step's keys move to the new buffers
        const int64_t cap = std::max<int64_t>(need, sp.cap + sp.cap / 2 + 1024);
        double* nc[7];
        double* na[7];
        int64_t *nid = nullptr, *nida = nullptr;
        int32_t* nkey = nullptr;
        for (int a = 0; a < 7; ++a) {
            STRY(grow(s, &nc[a], cap));
            STRY(grow(s, &na[a], cap));
        }
        STRY(grow(s, &nid, cap));
        STRY(grow(s, &nida, cap));
        STRY(grow(s, &nkey, cap));
        for (int a = 0; a < 7; ++a)
            if (np > 0)
                SCU(s, cudaMemcpyAsync(nc[a], sp.cur[a], np * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
        if (np > 0) {
            SCU(s, cudaMemcpyAsync(nid, sp.id, np * sizeof(int64_t), cudaMemcpyDeviceToDevice, s->stream));
            SCU(s, cudaMemcpyAsync(nkey, sp.key, np * sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream));
        }
        SCU(s, cudaStreamSynchronize(s->stream));
        for (int a = 0; a < 7; ++a) {
            pic_sim_dfree(s, sp.cur[a]);
            pic_sim_dfree(s, sp.alt[a]);
            sp.cur[a] = nc[a];
            sp.alt[a] = na[a];
        }
        pic_sim_dfree(s, sp.id);
        pic_sim_dfree(s, sp.id_alt);
        pic_sim_dfree(s, sp.key);
        sp.id = nid;
        sp.id_alt = nida;
        sp.key = nkey;
        sp.cap = cap;
        s->graph_dirty = true;
        STRY(pic_sim_upload(s));
    }
    for (int a = 0; a < 7; ++a)
        SCU(s, cudaMemcpyAsync(sp.cur[a] + np, soa[a], n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    SCU(s, cudaMemcpyAsync(sp.id + np, ids, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s->stream));
    SCU(s, pic_launch_keys_range(s->d, s->h, spi, np, need, s->stream));
    int64_t total = need;
    SCU(s, cudaMemcpyAsync(sp.off + s->h.ntiles, &total, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    return pic_sim_sync(s);
}

pic_status pic_shard_finish(pic_sim* s, int advance) {
    STRY(sharded(s));
    STRY(pic_sim_ensure_ready(s));
    for (int i = 0; i < s->h.nsp; ++i) SCU(s, pic_launch_sort(s->d, s->h, i, s->stream));
    if (advance) {
        SCU(s, pic_launch_finish(s->d, s->ds, s->stream));
        s->step_count++;
    }
    STRY(pic_sim_sync(s));
    return pic_sim_pull(s);
}

}  // extern "C"
