// pic_server.cu -- continuous batching of independent PIC simulations on one
// GPU (include/pic_server.h).
//
// Every admitted request is an ordinary libpic simulation (pic_init +
// pic_add_species) whose SimDev is copied into one slot of a contiguous device
// array.  A tick enqueues, for all active slots at once: the J reset, ONE
// persistent particle-kernel launch whose work units (slot, box, chunk) are the
// boxes of every active request in longest-first order, the Yee update, the
// per-tile re-sort and the step counters -- each a single launch with
// blockIdx.y running over the active slots.  Admission and retirement happen
// between ticks on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/pic_server.h"
#include "pic_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published definition
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// (0, 1) from a 32-bit draw
__device__ __forceinline__ double u01(uint32_t v) { return ((double)v + 0.5) * 2.3283064365386963e-10; }

// thermal electrons with a density ripple: particle i of cell c at a uniform
// point of the cell, momenta N(0, u_th^2) by Box-Muller, weight n0 dV/ppc
// (1 + a cos(2 pi x / Lx))
__global__ void plasma_init_kernel(int dim, int nx, int ny, int nz, double dx, double dy, double dz,
                                   int ppc, double n0, double uth, double ripple, uint2 key,
                                   double* x, double* y, double* z, double* ux, double* uy, double* uz,
                                   double* w, int64_t* id) {
    const int64_t ncell = (int64_t)nx * ny * nz;
    const int64_t np = ncell * ppc;
    const double two_pi = 6.283185307179586;
    const double Lx = nx * dx;
    const double dV = dx * (dim == 3 ? dy : 1.0) * dz;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = p / ppc;
        const int i = (int)(c % nx);
        const int j = (int)((c / nx) % ny);
        const int k = (int)(c / ((int64_t)nx * ny));
        const uint4 a = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), 0u, 0u), key);
        const uint4 b = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), 1u, 0u), key);
        const double px = (i + u01(a.x)) * dx;
        x[p] = px;
        y[p] = dim == 3 ? (j + u01(a.y)) * dy : 0.0;
        z[p] = (k + u01(a.z)) * dz;
        const double r1 = sqrt(-2.0 * log(u01(b.x))), r2 = sqrt(-2.0 * log(u01(b.z)));
        ux[p] = uth * r1 * cos(two_pi * u01(b.y));
        uy[p] = uth * r1 * sin(two_pi * u01(b.y));
        uz[p] = uth * r2 * cos(two_pi * u01(b.w));
        w[p] = n0 * dV / ppc * (1.0 + ripple * cos(two_pi * px / Lx));
        id[p] = p;
    }
}

struct Request {
    int64_t id = 0;
    pic_request_desc desc{};
    std::vector<std::vector<double>> arrays;  // staged explicit species (7 per species)
    std::vector<std::vector<int64_t>> ids;
    int state = PIC_REQ_PENDING;
    pic_sim* sim = nullptr;
    int slot = -1;
    int64_t footprint = 0;
    int64_t nparticles = 0;
    int steps_done = 0;
    double t_submit = -1, t_admit = -1, t_done = -1;
};

}  // namespace

struct pic_server {
    pic_server_desc desc{};
    std::string err = "no error";
    bool poisoned = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 0;
    SimDev* d_sims = nullptr;
    int* d_slots = nullptr;
    SchedDev hs{};
    SchedDev* ds = nullptr;
    int64_t units_cap = 0;
    std::vector<int64_t> slot_owner;  // request id per slot, -1 free
    std::map<int64_t, Request> reqs;
    std::deque<int64_t> pending;
    std::vector<int> active_slots;
    int64_t next_id = 1;
    int64_t bytes_in_use = 0;
    bool dirty = true;
    int64_t max_cells = 0, max_padded = 0, max_cap = 0;
    size_t smem = 0;
    int ctas = 0;
    int threads = 256;
    pic_server_stats stats{};
};

namespace {

pic_status sfail(pic_server* s, pic_status st, const std::string& m) {
    if (s) {
        s->err = m;
        if (st == PIC_ECUDA || st == PIC_ETIMEOUT) s->poisoned = true;
    }
    return st;
}

#define SCU(s, call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sfail((s), PIC_ECUDA, std::string(#call " failed: ") + cudaGetErrorString(e_)); \
    } while (0)

int64_t request_particles(const pic_request_desc& d, int64_t* per_species, int* nsp) {
    if (d.nspecies == 0) {
        const int64_t n = d.grid.ncell[0] * d.grid.ncell[1] * d.grid.ncell[2] * (int64_t)d.plasma.ppc;
        per_species[0] = n;
        *nsp = 1;
        return n;
    }
    int64_t t = 0;
    for (int i = 0; i < d.nspecies; ++i) {
        per_species[i] = d.species[i].np;
        t += d.species[i].np;
    }
    *nsp = d.nspecies;
    return t;
}

pic_status admit(pic_server* s, Request& r, int slot) {
    pic_grid_desc g = r.desc.grid;
    g.stream = s->stream;
    g.absorb_cells = 0;
    g.shape_order = s->desc.shape_order;
    pic_sim* sim = nullptr;
    pic_status st = pic_init(&g, &sim);
    if (st != PIC_OK) return sfail(s, st, std::string("request init: ") + pic_last_error(nullptr));
    r.sim = sim;
    if (r.desc.nspecies == 0) {
        const pic_plasma_init& pl = r.desc.plasma;
        const int64_t np = g.ncell[0] * g.ncell[1] * g.ncell[2] * (int64_t)pl.ppc;
        // the loader's staging buffers are freed (stream-ordered) on every way out
        struct Staging {
            cudaStream_t st;
            double* buf = nullptr;
            int64_t* ids = nullptr;
            ~Staging() {
                if (buf) cudaFreeAsync(buf, st);
                if (ids) cudaFreeAsync(ids, st);
            }
        } stg{s->stream};
        SCU(s, cudaMallocAsync((void**)&stg.buf, (size_t)std::max<int64_t>(np, 1) * 7 * sizeof(double), s->stream));
        SCU(s, cudaMallocAsync((void**)&stg.ids, (size_t)std::max<int64_t>(np, 1) * sizeof(int64_t), s->stream));
        double* buf = stg.buf;
        int64_t* ids = stg.ids;
        if (np > 0) {
            int64_t nb = std::min<int64_t>((np + 255) / 256, (int64_t)s->nsm * 32);
            plasma_init_kernel<<<(int)nb, 256, 0, s->stream>>>(
                g.dim, (int)g.ncell[0], (int)g.ncell[1], (int)g.ncell[2], g.dx[0], g.dx[1], g.dx[2], pl.ppc,
                pl.density, pl.u_th, pl.ripple, make_uint2((uint32_t)pl.seed, (uint32_t)(pl.seed >> 32)),
                buf, buf + np, buf + 2 * np, buf + 3 * np, buf + 4 * np, buf + 5 * np, buf + 6 * np, ids);
            SCU(s, cudaGetLastError());
        }
        SCU(s, cudaStreamSynchronize(s->stream));
        const double* soa[7];
        for (int a = 0; a < 7; ++a) soa[a] = buf + a * np;
        int spid = 0;
        st = pic_add_species(sim, -1.0, 1.0, np, soa, ids, 1, &spid);
        if (st != PIC_OK) return sfail(s, st, std::string("request species: ") + pic_last_error(sim));
        pic_add_background(sim, pl.density);
    } else {
        for (int i = 0; i < r.desc.nspecies; ++i) {
            const pic_species_init& sp = r.desc.species[i];
            const double* soa[7];
            for (int a = 0; a < 7; ++a) soa[a] = r.arrays[7 * i + a].data();
            int spid = 0;
            st = pic_add_species(sim, sp.charge, sp.mass, sp.np, soa, r.ids[i].data(), 0, &spid);
            if (st != PIC_OK) return sfail(s, st, std::string("request species: ") + pic_last_error(sim));
        }
        r.arrays.clear();
        r.ids.clear();
    }
    SimDev mirror;
    st = pic_internal_mirror(sim, &mirror);
    if (st != PIC_OK) return sfail(s, st, std::string("request mirror: ") + pic_internal_error(sim));
    SCU(s, cudaMemcpyAsync(s->d_sims + slot, &mirror, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream));
    SCU(s, cudaStreamSynchronize(s->stream));
    // admission reserved the estimate; the budget holds for the actual bytes
    const int64_t actual = pic_internal_bytes(sim);
    if (s->bytes_in_use + actual > s->desc.hbm_budget_bytes)
        return sfail(s, PIC_ENOMEM, "request footprint " + std::to_string(actual) + " bytes exceeds the HBM budget");
    pic_internal_mark_external(sim);
    r.footprint = actual;
    r.slot = slot;
    r.state = PIC_REQ_ACTIVE;
    r.t_admit = now_s();
    s->slot_owner[slot] = r.id;
    s->bytes_in_use += r.footprint;
    s->stats.admitted++;
    s->dirty = true;
    const int64_t pvol = (int64_t)mirror.pn[0] * mirror.pn[1] * mirror.pn[2];
    s->max_padded = std::max(s->max_padded, pvol);
    s->max_cells = std::max(s->max_cells, (int64_t)mirror.n[0] * mirror.n[1] * mirror.n[2]);
    for (int i = 0; i < mirror.nsp; ++i) s->max_cap = std::max(s->max_cap, mirror.sp[i].cap);
    s->smem = std::max(s->smem, pic_particle_smem_bytes(mirror.dim, mirror.order, mirror.T, s->threads, 0));
    return PIC_OK;
}

// work units of every active request, longest first (ties: lower slot, box)
pic_status rebuild_units(pic_server* s) {
    struct U {
        UnitDev u;
        double cost;
    };
    std::vector<U> all;
    s->active_slots.clear();
    for (int sl = 0; sl < (int)s->slot_owner.size(); ++sl) {
        if (s->slot_owner[sl] < 0) continue;
        const Request& r = s->reqs[s->slot_owner[sl]];
        if (r.state != PIC_REQ_ACTIVE) continue;
        s->active_slots.push_back(sl);
        const pic_grid_desc& g = r.desc.grid;
        int64_t nb = 1;
        for (int a = 0; a < 3; ++a) nb *= g.ncell[a] / g.box[a];
        const double per_box = (double)r.nparticles / (double)nb;
        const int k = (int)std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)std::llround(per_box / 8192.0)));
        for (int64_t b = 0; b < nb; ++b)
            for (int c = 0; c < k; ++c) all.push_back(U{UnitDev{sl, (int32_t)b, c, k}, per_box / k});
    }
    std::stable_sort(all.begin(), all.end(), [](const U& a, const U& b) { return a.cost > b.cost; });
    const int64_t nu = (int64_t)all.size();
    if (nu > s->units_cap) {
        if (s->hs.units) SCU(s, cudaFree(s->hs.units));
        const int64_t cap = std::max<int64_t>(nu, 2 * s->units_cap);
        SCU(s, cudaMalloc(&s->hs.units, (size_t)cap * sizeof(UnitDev)));
        s->units_cap = cap;
        SCU(s, cudaMemcpyAsync(s->ds, &s->hs, sizeof(SchedDev), cudaMemcpyHostToDevice, s->stream));
    }
    std::vector<UnitDev> hu(nu);
    for (int64_t i = 0; i < nu; ++i) hu[i] = all[i].u;
    if (nu > 0)
        SCU(s, cudaMemcpyAsync(s->hs.units, hu.data(), nu * sizeof(UnitDev), cudaMemcpyHostToDevice, s->stream));
    int32_t lo[2] = {0, (int32_t)nu};
    SCU(s, cudaMemcpyAsync(s->hs.list_off, lo, sizeof lo, cudaMemcpyHostToDevice, s->stream));
    int32_t meta[2] = {1, 0};
    SCU(s, cudaMemcpyAsync(s->hs.meta, meta, sizeof meta, cudaMemcpyHostToDevice, s->stream));
    if (!s->active_slots.empty())
        SCU(s, cudaMemcpyAsync(s->d_slots, s->active_slots.data(), s->active_slots.size() * sizeof(int),
                               cudaMemcpyHostToDevice, s->stream));
    SCU(s, cudaStreamSynchronize(s->stream));
    if (!s->active_slots.empty()) {
        SCU(s, pic_prepare_particles(s->desc.dim, s->desc.shape_order, s->smem));
        int per_sm = pic_particle_occupancy(s->desc.dim, s->desc.shape_order, 1, 1, s->threads, s->smem, 0);
        s->ctas = s->nsm * std::max(1, std::min(per_sm, 2));
    }
    s->dirty = false;
    return PIC_OK;
}

Request* find(pic_server* s, int64_t id) {
    auto it = s->reqs.find(id);
    return it == s->reqs.end() ? nullptr : &it->second;
}

}  // namespace

extern "C" {

const char* pic_server_last_error(const pic_server* s) { return s ? s->err.c_str() : "null server"; }

pic_status pic_server_create(const pic_server_desc* d, pic_server** out) {
    if (!d || !out) return pic_record_error(PIC_EINVAL, "null argument");
    *out = nullptr;
    if ((d->dim != 2 && d->dim != 3) || d->shape_order < 1 || d->shape_order > 3 ||
        d->max_active < 1 || d->max_active > 4096 || d->hbm_budget_bytes <= 0)
        return pic_record_error(PIC_EINVAL, "bad server description");
    pic_server* s = new (std::nothrow) pic_server();
    if (!s) return pic_record_error(PIC_ENOMEM, "host allocation failed");
    s->desc = *d;
    cudaDeviceProp prop;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        delete s;
        return pic_record_error(PIC_ECUDA, "no CUDA device");
    }
    s->nsm = prop.multiProcessorCount;
    if (d->stream) {
        s->stream = (cudaStream_t)d->stream;
    } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess) {
        s->own_stream = true;
    } else {
        delete s;
        return pic_record_error(PIC_ECUDA, "stream creation failed");
    }
    bool ok = cudaMalloc(&s->d_sims, sizeof(SimDev) * d->max_active) == cudaSuccess &&
              cudaMalloc(&s->d_slots, sizeof(int) * d->max_active) == cudaSuccess &&
              cudaMalloc(&s->ds, sizeof(SchedDev)) == cudaSuccess &&
              cudaMalloc(&s->hs.list_off, 2 * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&s->hs.head, sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&s->hs.meta, 2 * sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&s->hs.err, sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&s->hs.rings, pic_ring_bytes(s->nsm)) == cudaSuccess;
    if (!ok) {
        pic_server_destroy(s);
        return pic_record_error(PIC_ENOMEM, "server allocation failed");
    }
    cudaMemset(s->hs.head, 0, sizeof(int32_t));
    cudaMemset(s->hs.err, 0, sizeof(int32_t));
    if (cudaMemcpy(s->ds, &s->hs, sizeof(SchedDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        pic_server_destroy(s);
        return pic_record_error(PIC_ECUDA, "server set-up failed");
    }
    s->slot_owner.assign(d->max_active, -1);
    *out = s;
    return PIC_OK;
}

pic_status pic_server_submit(pic_server* s, const pic_request_desc* d, int64_t* req_id) {
    if (!s || !d || !req_id) return sfail(s, PIC_EINVAL, "null argument");
    if (s->poisoned) return PIC_ESTATE;
    const pic_grid_desc& g = d->grid;
    if (g.dim != s->desc.dim || d->nsteps < 1 || d->nspecies < 0 || d->nspecies > 4)
        return sfail(s, PIC_EINVAL, "request dim, nsteps or species count invalid");
    for (int a = 0; a < 3; ++a)
        if (g.ncell[a] < 1 || g.box[a] < 1 || g.ncell[a] % g.box[a] != 0)
            return sfail(s, PIC_EINVAL, "request boxes must divide the grid");
    if (d->nspecies == 0 && (d->plasma.ppc < 1 || !(d->plasma.density >= 0.0) || !(d->plasma.u_th >= 0.0)))
        return sfail(s, PIC_EINVAL, "bad plasma description");
    Request r;
    r.id = s->next_id++;
    r.desc = *d;
    int64_t per[4] = {0, 0, 0, 0};
    int nsp = 0;
    r.nparticles = request_particles(*d, per, &nsp);
    // the grid as admission will create it: the server's shape order (it sets
    // the guard widths), no absorbing layers
    pic_grid_desc ga = g;
    ga.shape_order = s->desc.shape_order;
    ga.absorb_cells = 0;
    r.footprint = pic_internal_estimate_bytes(&ga, per, nsp);
    if (r.footprint > s->desc.hbm_budget_bytes)
        return sfail(s, PIC_ENOMEM, "request footprint " + std::to_string(r.footprint) +
                                        " bytes exceeds the server budget");
    if (d->nspecies > 0) {
        for (int i = 0; i < d->nspecies; ++i) {
            const pic_species_init& sp = d->species[i];
            if (sp.np < 0 || !(sp.mass > 0.0)) return sfail(s, PIC_EINVAL, "bad species");
            for (int a = 0; a < 7; ++a) {
                std::vector<double> v((size_t)sp.np, 0.0);
                if (sp.np > 0 && sp.soa[a]) memcpy(v.data(), sp.soa[a], sp.np * sizeof(double));
                else if (sp.np > 0 && !(a == 1 && g.dim == 2))
                    return sfail(s, PIC_EINVAL, "missing particle array");
                r.arrays.push_back(std::move(v));
            }
            std::vector<int64_t> ids((size_t)sp.np);
            for (int64_t p = 0; p < sp.np; ++p) ids[p] = sp.ids ? sp.ids[p] : p;
            r.ids.push_back(std::move(ids));
        }
        r.desc.nspecies = d->nspecies;
    }
    r.t_submit = now_s();
    *req_id = r.id;
    s->pending.push_back(r.id);
    s->reqs.emplace(r.id, std::move(r));
    return PIC_OK;
}

pic_status pic_server_tick(pic_server* s, int* n_active, int* n_pending) {
    if (!s) return PIC_EINVAL;
    if (s->poisoned) return PIC_ESTATE;
    // admission: submission order, while a slot is free and the footprint fits
    while (!s->pending.empty()) {
        Request& r = s->reqs[s->pending.front()];
        int slot = -1;
        for (int i = 0; i < (int)s->slot_owner.size(); ++i)
            if (s->slot_owner[i] < 0) {
                slot = i;
                break;
            }
        if (slot < 0 || s->bytes_in_use + r.footprint > s->desc.hbm_budget_bytes) break;
        s->pending.pop_front();
        pic_status st = admit(s, r, slot);
        if (st != PIC_OK) {
            // nothing of the request was registered with the server; a device
            // error poisons it, any other failure fails this request alone
            if (r.sim) pic_destroy(r.sim);
            r.sim = nullptr;
            if (s->poisoned) return st;
            r.state = PIC_REQ_FAILED;
            r.t_done = now_s();
            r.arrays.clear();
            r.ids.clear();
        }
    }
    if (s->dirty) {
        pic_status st = rebuild_units(s);
        if (st != PIC_OK) return st;
    }
    const int na = (int)s->active_slots.size();
    if (na > 0) {
        SCU(s, pic_launch_zero_j_multi(s->d_sims, s->d_slots, na, s->max_padded, s->stream));
        LaunchCfg cfg{s->threads, s->ctas, 1, 0};
        SCU(s, pic_launch_particles(s->desc.dim, s->desc.shape_order, cfg, s->smem, s->ds, s->d_sims, s->stream));
        SCU(s, pic_launch_fields_multi(s->d_sims, s->d_slots, na, s->desc.dim, s->max_cells, s->max_padded,
                                       false, s->stream));
        SCU(s, pic_launch_sort_multi(s->d_sims, s->d_slots, na, s->desc.dim, s->max_cap, s->stream));
        SCU(s, pic_launch_finish_multi(s->d_sims, s->d_slots, na, s->ds, s->stream));
        SCU(s, cudaStreamSynchronize(s->stream));
        int32_t e = 0;
        SCU(s, cudaMemcpy(&e, s->hs.err, sizeof e, cudaMemcpyDeviceToHost));
        if (e) return sfail(s, (e & PIC_DERR_TMA_TIMEOUT) ? PIC_ETIMEOUT : PIC_ECUDA,
                            "device-side check failed (error word " + std::to_string(e) + ")");
        s->stats.ticks++;
        s->stats.particle_launches++;
        s->stats.kernels += 1 + 1 + 5 + 3 + 1;
        const double t = now_s();
        for (int sl : s->active_slots) {
            Request& r = s->reqs[s->slot_owner[sl]];
            r.steps_done++;
            s->stats.particle_updates += r.nparticles;
            if (r.steps_done >= r.desc.nsteps) {
                // keep the results: copy the slot's state back to the request's handle
                SCU(s, cudaMemcpy(pic_internal_device_sim(r.sim), s->d_sims + sl, sizeof(SimDev),
                                  cudaMemcpyDeviceToDevice));
                r.state = PIC_REQ_DONE;
                r.t_done = t;
                s->slot_owner[sl] = -1;
                r.slot = -1;
                s->stats.finished++;
                s->dirty = true;
            }
        }
    }
    if (n_active) {
        int c = 0;
        for (int64_t o : s->slot_owner) c += o >= 0;
        *n_active = c;
    }
    if (n_pending) *n_pending = (int)s->pending.size();
    return PIC_OK;
}

pic_status pic_server_poll(pic_server* s, int64_t id, int* state, double* ts, double* ta, double* td,
                           int* steps) {
    if (!s) return PIC_EINVAL;
    Request* r = find(s, id);
    if (!r) return sfail(s, PIC_EINVAL, "unknown request");
    if (state) *state = r->state;
    if (ts) *ts = r->t_submit;
    if (ta) *ta = r->t_admit;
    if (td) *td = r->t_done;
    if (steps) *steps = r->steps_done;
    return PIC_OK;
}

static pic_status done_request(pic_server* s, int64_t id, Request** out) {
    Request* r = find(s, id);
    if (!r) return sfail(s, PIC_EINVAL, "unknown request");
    if (r->state != PIC_REQ_DONE) return sfail(s, PIC_ESTATE, "request is not finished");
    *out = r;
    return PIC_OK;
}

pic_status pic_server_read_fields(pic_server* s, int64_t id, int comp, double* out) {
    if (!s) return PIC_EINVAL;
    Request* r = nullptr;
    pic_status st = done_request(s, id, &r);
    if (st != PIC_OK) return st;
    st = pic_read_fields(r->sim, comp, out, 0);
    return st == PIC_OK ? st : sfail(s, st, pic_internal_error(r->sim));
}

pic_status pic_server_num_particles(pic_server* s, int64_t id, int species, int64_t* np) {
    if (!s) return PIC_EINVAL;
    Request* r = nullptr;
    pic_status st = done_request(s, id, &r);
    if (st != PIC_OK) return st;
    st = pic_num_particles(r->sim, species, np);
    return st == PIC_OK ? st : sfail(s, st, pic_internal_error(r->sim));
}

pic_status pic_server_read_particles(pic_server* s, int64_t id, int species, double* const soa[7],
                                     int64_t* ids) {
    if (!s) return PIC_EINVAL;
    Request* r = nullptr;
    pic_status st = done_request(s, id, &r);
    if (st != PIC_OK) return st;
    st = pic_read_particles(r->sim, species, soa, ids, 0);
    return st == PIC_OK ? st : sfail(s, st, pic_internal_error(r->sim));
}

pic_status pic_server_release(pic_server* s, int64_t id) {
    if (!s) return PIC_EINVAL;
    Request* r = nullptr;
    pic_status st = done_request(s, id, &r);
    if (st != PIC_OK) return st;
    pic_destroy(r->sim);
    r->sim = nullptr;
    s->bytes_in_use -= r->footprint;
    r->state = PIC_REQ_RELEASED;
    return PIC_OK;
}

pic_status pic_server_cancel(pic_server* s, int64_t id) {
    if (!s) return PIC_EINVAL;
    Request* r = find(s, id);
    if (!r) return sfail(s, PIC_EINVAL, "unknown request");
    if (r->state == PIC_REQ_PENDING) {
        s->pending.erase(std::find(s->pending.begin(), s->pending.end(), id));
        r->arrays.clear();
        r->ids.clear();
    } else if (r->state == PIC_REQ_ACTIVE) {
        // no device work of the server is in flight after this: the slot's
        // entry in the packed launch is dropped when the next tick rebuilds
        // its work units (before it launches anything)
        SCU(s, cudaStreamSynchronize(s->stream));
        s->slot_owner[r->slot] = -1;
        r->slot = -1;
        pic_destroy(r->sim);
        r->sim = nullptr;
        s->bytes_in_use -= r->footprint;
        s->dirty = true;
    } else {
        return sfail(s, PIC_ESTATE, "request is finished, released or cancelled");
    }
    r->state = PIC_REQ_CANCELLED;
    return PIC_OK;
}

pic_status pic_server_footprint(pic_server* s, int64_t id, int64_t* bytes) {
    if (!s || !bytes) return PIC_EINVAL;
    Request* r = find(s, id);
    if (!r) return sfail(s, PIC_EINVAL, "unknown request");
    *bytes = r->footprint;
    return PIC_OK;
}

pic_status pic_server_get_stats(pic_server* s, pic_server_stats* out) {
    if (!s || !out) return PIC_EINVAL;
    *out = s->stats;
    out->bytes_in_use = s->bytes_in_use;
    return PIC_OK;
}

pic_status pic_server_destroy(pic_server* s) {
    if (!s) return PIC_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto& kv : s->reqs)
        if (kv.second.sim) pic_destroy(kv.second.sim);
    cudaFree(s->d_sims);
    cudaFree(s->d_slots);
    cudaFree(s->ds);
    cudaFree(s->hs.units);
    cudaFree(s->hs.list_off);
    cudaFree(s->hs.head);
    cudaFree(s->hs.meta);
    cudaFree(s->hs.err);
    cudaFree(s->hs.rings);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return PIC_OK;
}

}  // extern "C"
