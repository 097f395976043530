// pic_api.cu -- host side of libpic: the C ABI of include/pic_api.h.
//
// One pic_sim owns a simulation resident in HBM (SimDev + buffers), the work
// schedule of the persistent particle kernel (SchedDev), and a CUDA graph of
// one PIC step.  pic_step replays the graph; at load-balancing intervals it
// runs the routine of arXiv 2104.11385 Sec. 2.2: device->host copy of the
// per-box costs (the "gather to the root"), host mapping and efficiency, and,
// when the threshold is met, a host->device copy of the new work list (the
// "broadcast and redistribution").  Pointers captured in the graph never
// change; everything that changes lives in device memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pic_api.h"
#include "pic_balance.h"
#include "pic_bin.h"
#include "pic_internal.h"
#include "pic_sim.h"

namespace {

thread_local std::string g_last_error = "no error";

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

namespace {

pic_status fail(pic_sim* s, pic_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) {
        s->err = buf;
        if (st == PIC_ECUDA || st == PIC_ETIMEOUT) s->poisoned = true;
    } else {
        g_last_error = buf;
    }
    return st;
}

#define CU(s, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((s), PIC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// a temporary device buffer for one call: a failed allocation is PIC_ENOMEM
// (the handle stays usable), not a device error
template <class T>
pic_status talloc(pic_sim* s, T** p, size_t n) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(s, PIC_ENOMEM, "temporary cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    *p = (T*)q;
    return PIC_OK;
}

template <class T>
pic_status dalloc(pic_sim* s, T** p, size_t n) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(s, PIC_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    s->allocs.push_back(q);
    s->bytes += (int64_t)bytes;
    *p = (T*)q;
    return PIC_OK;
}

#define TRY(x)                          \
    do {                                \
        pic_status st_ = (x);           \
        if (st_ != PIC_OK) return st_;  \
    } while (0)

pic_status check(pic_sim* s) {
    if (!s) return fail(nullptr, PIC_EINVAL, "null handle");
    if (s->poisoned) return PIC_ESTATE;
    return PIC_OK;
}

pic_status upload_sim(pic_sim* s) {
    CU(s, cudaMemcpyAsync(s->d, &s->h, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

// refreshes the host mirror's species buffer pointers from the device copy
pic_status pull_sim(pic_sim* s) {
    SimDev tmp;
    CU(s, cudaMemcpyAsync(&tmp, s->d, sizeof(SimDev), cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    for (int i = 0; i < PIC_MAXSP; ++i) {
        memcpy(s->h.sp[i].cur, tmp.sp[i].cur, sizeof(tmp.sp[i].cur));
        memcpy(s->h.sp[i].alt, tmp.sp[i].alt, sizeof(tmp.sp[i].alt));
        s->h.sp[i].id = tmp.sp[i].id;
        s->h.sp[i].id_alt = tmp.sp[i].id_alt;
    }
    return PIC_OK;
}

pic_status check_device_error(pic_sim* s) {
    int32_t e = 0;
    CU(s, cudaMemcpyAsync(&e, s->hs.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    if (e & PIC_DERR_TMA_TIMEOUT)
        return fail(s, PIC_ETIMEOUT, "a bounded wait on a TMA tile load ran out (device error %d)", e);
    if (e & PIC_DERR_WAIT_TIMEOUT)
        return fail(s, PIC_ETIMEOUT, "the bounded-wait self-test ran out, as designed (device error %d)", e);
    if (e) return fail(s, PIC_ECUDA, "device-side check failed (device error word %d)", e);
    return PIC_OK;
}

pic_status sync_and_check(pic_sim* s) {
    CU(s, cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

int largest_even_divisor_le(int b, int cap) {
    for (int t = std::min(b, cap); t >= 2; --t)
        if (b % t == 0 && t % 2 == 0) return t;
    return 0;
}

// tile extents t[a] (cells per tile edge, 1 for the inactive y of 2D runs) and
// everything derived from them: tiles per box, tile count, staged E/B and J
// tile extents
void set_tiling(SimDev& h, const int t[3]) {
    for (int a = 0; a < 3; ++a) {
        const bool act = !(h.dim == 2 && a == 1);
        h.T[a] = act ? t[a] : 1;
        h.tpb[a] = h.bsz[a] / h.T[a];
        h.ebs[a] = act ? h.T[a] + (h.order == 1 ? 2 : h.order == 2 ? 3 : 4) : 1;
    }
    if (h.order == 2) h.ebs[0] += 1;
    h.tiles_per_box = h.tpb[0] * h.tpb[1] * h.tpb[2];
    h.ntiles = h.nboxes * h.tiles_per_box;
}

// a tile size is valid when it is even, at least 4 (2D and 3D alike) and
// divides every active box extent
bool tile_ok(const SimDev& h, int t) {
    if (t < 4 || t % 2 != 0) return false;
    for (int a = 0; a < 3; ++a)
        if (!(h.dim == 2 && a == 1) && h.bsz[a] % t != 0) return false;
    return true;
}

// TMA descriptors of the six padded E/B arrays, box = the staged tile
pic_status encode_tmaps(pic_sim* s) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc) return fail(s, PIC_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    SimDev& h = s->h;
    for (int c = 0; c < 6; ++c) {
        cuuint64_t dims[3] = {(cuuint64_t)h.pn[0], (cuuint64_t)h.pn[1], (cuuint64_t)h.pn[2]};
        cuuint64_t strides[2] = {(cuuint64_t)h.pn[0] * 8, (cuuint64_t)h.pn[0] * h.pn[1] * 8};
        cuuint32_t box[3] = {(cuuint32_t)h.ebs[0], (cuuint32_t)h.ebs[1], (cuuint32_t)h.ebs[2]};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&h.tmap[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, h.F[c], dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(s, PIC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return PIC_OK;
}

// ---------------------------------------------------------------- plans ---
void box_coords(const pic_sim* s, int64_t b, int32_t* ijk) {
    const SimDev& h = s->h;
    ijk[0] = (int32_t)(b % h.nb[0]);
    ijk[1] = (int32_t)((b / h.nb[0]) % h.nb[1]);
    ijk[2] = (int32_t)(b / ((int64_t)h.nb[0] * h.nb[1]));
}

int n_workers_for(const pic_sim* s, const pic_lb_params& p) {
    int nw = p.n_workers > 0 ? p.n_workers : s->ctas;
    if (p.sched == PIC_SCHED_LISTS) nw = std::min(nw, s->ctas);
    return std::max(1, nw);
}

// builds the plan from units and their mapping
void build_plan(pic_sim* s, const std::vector<pic::Unit>& units, const std::vector<int32_t>& assign,
                int n_workers, int sched, bool box_order = false) {
    SimPlan& P = s->plan;
    P.units.clear();
    P.unit_cost.clear();
    P.unit_worker.clear();
    P.n_workers = n_workers;
    const int64_t nu = (int64_t)units.size();
    std::vector<int64_t> order(nu);
    for (int64_t i = 0; i < nu; ++i) order[i] = i;
    if (sched == PIC_SCHED_LISTS) {
        // list w holds the units of worker w, heaviest first (ties: lower index)
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
            if (assign[a] != assign[b]) return assign[a] < assign[b];
            return !box_order && units[a].cost > units[b].cost;
        });
        P.nlists = n_workers;
        P.list_off.assign(n_workers + 1, 0);
        for (int64_t i = 0; i < nu; ++i) P.list_off[assign[i] + 1]++;
        for (int w = 0; w < n_workers; ++w) P.list_off[w + 1] += P.list_off[w];
    } else {
        // one queue, heaviest unit first (longest-processing-time order), or
        // in box-index order for the box-order policy
        if (!box_order)
            std::stable_sort(order.begin(), order.end(),
                             [&](int64_t a, int64_t b) { return units[a].cost > units[b].cost; });
        P.nlists = 1;
        P.list_off = {0, (int32_t)nu};
    }
    for (int64_t i : order) {
        const pic::Unit& u = units[i];
        P.units.push_back(UnitDev{0, u.box, u.chunk, u.nchunks});
        P.unit_cost.push_back(u.cost);
        P.unit_worker.push_back(assign[i]);
    }
}

pic_status upload_plan(pic_sim* s) {
    SimPlan& P = s->plan;
    int64_t nu = (int64_t)P.units.size();
    if (nu > s->units_cap) {
        int64_t cap = std::max<int64_t>(nu, 2 * s->units_cap);
        UnitDev* nu_ptr = nullptr;
        TRY(dalloc(s, &nu_ptr, (size_t)cap));
        s->hs.units = nu_ptr;
        s->units_cap = cap;
        CU(s, cudaMemcpyAsync(s->ds, &s->hs, sizeof(SchedDev), cudaMemcpyHostToDevice, s->stream));
    }
    if (P.nlists + 1 > 8192) return fail(s, PIC_EINVAL, "too many work lists (%d)", P.nlists);
    if (nu > 0)
        CU(s, cudaMemcpyAsync(s->hs.units, P.units.data(), nu * sizeof(UnitDev),
                              cudaMemcpyHostToDevice, s->stream));
    CU(s, cudaMemcpyAsync(s->hs.list_off, P.list_off.data(), P.list_off.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s->stream));
    int32_t meta[2] = {P.nlists, 0};
    CU(s, cudaMemcpyAsync(s->hs.meta, meta, sizeof meta, cudaMemcpyHostToDevice, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

// the fixed starting mapping: one unit per box, boxes cut into contiguous
// equal-count pieces of the Morton curve (the space-filling-curve policy with
// uniform costs), no cost information used
pic_status initial_plan(pic_sim* s) {
    const int64_t nb = s->h.nboxes;
    std::vector<double> ones(nb, 1.0);
    std::vector<int64_t> np(nb, 1);
    std::vector<pic::Unit> units = pic::make_units(ones.data(), np.data(), nb, 1, 1, 1, false);
    int sched = s->lb_set ? s->lb.sched : PIC_SCHED_LISTS;
    pic_lb_params p = s->lb;
    if (!s->lb_set) p.sched = PIC_SCHED_LISTS, p.n_workers = 0;
    int nw = n_workers_for(s, p);
    std::vector<int32_t> assign(nb);
    pic::sfc(ones.data(), s->box_ijk.data(), nb, s->h.dim, nw, assign.data());
    if (sched == PIC_SCHED_QUEUE) {
        // queue: boxes in index order
        SimPlan& P = s->plan;
        P.units.clear();
        P.unit_cost.assign(nb, 1.0);
        P.unit_worker = assign;
        P.n_workers = nw;
        P.nlists = 1;
        for (int64_t b = 0; b < nb; ++b) P.units.push_back(UnitDev{0, (int32_t)b, 0, 1});
        P.list_off = {0, (int32_t)nb};
    } else {
        // keep Morton order inside each list
        std::vector<pic::Unit> u2 = units;
        for (int64_t b = 0; b < nb; ++b)
            u2[b].cost = -(double)pic::morton_key(s->h.dim, s->box_ijk[3 * b], s->box_ijk[3 * b + 1],
                                                   s->box_ijk[3 * b + 2]);
        build_plan(s, u2, assign, nw, PIC_SCHED_LISTS);
        std::fill(s->plan.unit_cost.begin(), s->plan.unit_cost.end(), 1.0);
    }
    return upload_plan(s);
}

// ---------------------------------------------------------------- costs ---
pic_status box_counts(pic_sim* s, std::vector<int64_t>& np) {
    np.assign(s->h.nboxes, 0);
    if (s->h.nsp == 0) return PIC_OK;
    CU(s, pic_launch_box_counts(s->d, s->h, s->d_box_np, s->stream));
    CU(s, cudaMemcpyAsync(np.data(), s->d_box_np, s->h.nboxes * sizeof(int64_t),
                          cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

pic_status box_costs(pic_sim* s, int strategy, double w_p, double w_c, std::vector<double>& costs,
                     std::vector<int64_t>& np) {
    TRY(box_counts(s, np));
    const int64_t nb = s->h.nboxes;
    costs.assign(nb, 0.0);
    if (strategy == PIC_COST_DEVICE_CLOCK || strategy == PIC_COST_KERNEL_TIME) {
        std::vector<uint64_t> clk(nb);
        CU(s, cudaMemcpyAsync(clk.data(), strategy == PIC_COST_DEVICE_CLOCK ? s->h.cost_clock : s->h.cost_time,
                              nb * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
        CU(s, cudaStreamSynchronize(s->stream));
        for (int64_t b = 0; b < nb; ++b) costs[b] = (double)clk[b];
    } else {
        const double nc = (double)s->h.bsz[0] * s->h.bsz[1] * s->h.bsz[2];
        for (int64_t b = 0; b < nb; ++b) costs[b] = w_p * (double)np[b] + w_c * nc;
    }
    return PIC_OK;
}

pic_lb_params default_lb() {
    pic_lb_params p{};
    p.mode = PIC_LB_NONE;
    p.interval = 10;
    p.theta = 0.10;
    p.policy = PIC_POLICY_KNAPSACK;
    p.cost = PIC_COST_DEVICE_CLOCK;
    p.w_p = 0.75;
    p.w_c = 0.25;
    p.cap_factor = 1.5;
    p.n_workers = 0;
    p.split = 0;
    p.sched = PIC_SCHED_LISTS;
    return p;
}

pic_status validate_lb(pic_sim* s, const pic_lb_params* p) {
    if (!p) return fail(s, PIC_EINVAL, "null load-balancing parameters");
    if (p->mode < PIC_LB_NONE || p->mode > PIC_LB_DYNAMIC || p->interval < 1 || !(p->theta >= 0.0) ||
        (p->policy != PIC_POLICY_KNAPSACK && p->policy != PIC_POLICY_SFC && p->policy != PIC_POLICY_BOX_ORDER) ||
        (p->cost != PIC_COST_HEURISTIC && p->cost != PIC_COST_DEVICE_CLOCK && p->cost != PIC_COST_KERNEL_TIME) ||
        !(p->cap_factor > 0.0) || p->n_workers < 0 || p->split < 0 ||
        (p->sched != PIC_SCHED_LISTS && p->sched != PIC_SCHED_QUEUE) || !std::isfinite(p->w_p) ||
        !std::isfinite(p->w_c))
        return fail(s, PIC_EINVAL, "load-balancing parameters out of range");
    return PIC_OK;
}

// the load-balancing routine (Sec. 2.2): costs -> proposed mapping -> E_old,
// E_new -> adopt when E_new >= (1 + theta) E_old
// E (Eq. 1) of the work-unit mapping in force for per-box costs; a box's
// cost is divided evenly over its units
double plan_efficiency(const pic_sim* s, const std::vector<double>& costs) {
    const SimPlan& P = s->plan;
    std::vector<double> uc(P.units.size());
    for (size_t i = 0; i < P.units.size(); ++i) uc[i] = costs[P.units[i].box] / (double)P.units[i].nchunks;
    return pic::lb_efficiency(uc.data(), P.unit_worker.data(), (int64_t)uc.size(), P.n_workers);
}

// maps work units to workers with the policy of p (knapsack or Morton SFC)
void map_units(const pic_sim* s, const pic_lb_params& p, const std::vector<pic::Unit>& units, int nw,
               std::vector<double>& uc, std::vector<int32_t>& assign) {
    uc.resize(units.size());
    for (size_t i = 0; i < units.size(); ++i) uc[i] = units[i].cost;
    assign.resize(units.size());
    if (p.policy == PIC_POLICY_BOX_ORDER) {
        // no cost input: units in box-index order, contiguous equal-count pieces
        const int64_t nu = (int64_t)units.size();
        for (int64_t i = 0; i < nu; ++i) assign[i] = (int32_t)((i * (int64_t)nw) / std::max<int64_t>(nu, 1));
    } else if (p.policy == PIC_POLICY_KNAPSACK) {
        pic::knapsack(uc.data(), (int64_t)uc.size(), nw, p.cap_factor, assign.data());
    } else {
        std::vector<int32_t> ijk(3 * units.size());
        for (size_t i = 0; i < units.size(); ++i)
            for (int a = 0; a < 3; ++a) ijk[3 * i + a] = s->box_ijk[3 * units[i].box + a];
        pic::sfc(uc.data(), ijk.data(), (int64_t)uc.size(), s->h.dim, nw, assign.data());
    }
}

pic_status rebalance(pic_sim* s, const pic_lb_params& p, double theta, pic_lb_result* out) {
    std::vector<double> costs;
    std::vector<int64_t> np;
    TRY(box_costs(s, p.cost, p.w_p, p.w_c, costs, np));
    const int64_t nb = s->h.nboxes;
    const int nw = n_workers_for(s, p);
    // E_old: the mapping in force, re-costed with the costs just measured
    const double e_old = plan_efficiency(s, costs);
    const int split = p.split > 0 ? p.split : s->split;
    std::vector<pic::Unit> units =
        pic::make_units(costs.data(), np.data(), nb, nw, split, 256, true);
    std::vector<double> uc;
    std::vector<int32_t> assign;
    map_units(s, p, units, nw, uc, assign);
    double e_new = pic::lb_efficiency(uc.data(), assign.data(), (int64_t)uc.size(), nw);
    bool adopted = pic::adopt(e_old, e_new, theta);
    if (adopted) {
        build_plan(s, units, assign, nw, p.sched, p.policy == PIC_POLICY_BOX_ORDER);
        TRY(upload_plan(s));
    }
    s->last_costs = costs;
    s->last_np = np;
    CU(s, cudaMemsetAsync(s->h.cost_clock, 0, nb * sizeof(uint64_t), s->stream));
    CU(s, cudaMemsetAsync(s->h.cost_time, 0, nb * sizeof(uint64_t), s->stream));
    pic_lb_result r;
    r.e_old = e_old;
    r.e_new = e_new;
    r.adopted = adopted ? 1 : 0;
    r.n_units = (int64_t)units.size();
    r.predicted_speedup = pic::predicted_speedup(e_old > 0 ? e_old : 1.0, s->h.dim == 3 ? 0.88 : 0.91);
    r.step = s->step_count;
    s->lb_log.push_back(r);
    if (out) *out = r;
    return PIC_OK;
}

// ---------------------------------------------------------------- graph ---
pic_status enqueue_step(pic_sim* s, bool with_events) {
    const SimDev& h = s->h;
    const int64_t jbytes = (int64_t)h.pn[0] * h.pn[1] * h.pn[2] * 3 * sizeof(double);
    if (with_events) CU(s, cudaEventRecord(s->ev[0], s->stream));
    CU(s, cudaMemsetAsync(h.F[6], 0, jbytes, s->stream));
    if (h.nsp > 0) {
        LaunchCfg cfg{s->threads, s->ctas, s->minb, s->prec, s->ppt};
        CU(s, pic_launch_particles(h.dim, h.order, cfg, s->smem, s->ds, s->d, s->stream));
    }
    if (with_events) CU(s, cudaEventRecord(s->ev[1], s->stream));
    CU(s, pic_launch_fields(s->d, h, s->stream));
    if (with_events) CU(s, cudaEventRecord(s->ev[2], s->stream));
    for (int sp = 0; sp < h.nsp; ++sp) CU(s, pic_launch_sort(s->d, h, sp, s->stream));
    CU(s, pic_launch_finish(s->d, s->ds, s->stream));
    if (with_events) CU(s, cudaEventRecord(s->ev[3], s->stream));
    return PIC_OK;
}

int count_kernels(const pic_sim* s) {
    int k = (s->h.nsp > 0 ? 1 : 0) + 1 + 3 + (s->h.absorb > 0 ? 1 : 0) + 1 + 3 * s->h.nsp + 1;
    return k;
}

pic_status capture_graph(pic_sim* s) {
    if (s->graph) {
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    cudaGraph_t g;
    CU(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    pic_status st = enqueue_step(s, false);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (st != PIC_OK) return st;
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    s->graph_dirty = false;
    s->kernels_per_step = count_kernels(s);
    return PIC_OK;
}

pic_status configure_launch(pic_sim* s) {
    s->smem = pic_particle_smem_bytes(s->h.dim, s->h.order, s->h.T, s->threads, s->prec);
    cudaDeviceProp prop;
    CU(s, cudaGetDeviceProperties(&prop, s->device));
    if (s->smem > prop.sharedMemPerBlockOptin)
        return fail(s, PIC_EUNSUPPORTED, "tile needs %zu bytes of shared memory", s->smem);
    CU(s, pic_prepare_particles(s->h.dim, s->h.order, s->smem));
    // persistent grid: every CTA resident (registers, shared memory, threads)
    // ctas_per_sm >= 2 selects the kernel variant compiled for 2 resident CTAs
    s->minb = s->ctas_per_sm >= 2 ? 2 : 1;
    int resident = pic_particle_occupancy(s->h.dim, s->h.order, s->minb, s->ppt, s->threads, s->smem, s->prec);
    if (resident < 1) return fail(s, PIC_EUNSUPPORTED, "particle kernel does not fit on an SM");
    int per_sm = std::max(1, std::min(s->ctas_per_sm, resident));
    s->ctas = s->nsm * per_sm;
    s->graph_dirty = true;
    return PIC_OK;
}

// block sums of the multi-block histogram scan, enough for the tile count
pic_status ensure_scan_part(pic_sim* s) {
    SimDev& h = s->h;
    const int64_t need = ((int64_t)h.ntiles + 1 + 1023) / 1024;
    if (need <= h.scan_part_cap) return PIC_OK;
    TRY(dalloc(s, &h.scan_part, (size_t)need));
    h.scan_part_cap = need;
    return PIC_OK;
}

// Re-tiles the simulation with tile edge t in every active direction: tile
// maps for the new staged tile, sort arrays for the new tile count, and every
// species re-sorted by the new tiles.  Units (box chunks) are unaffected.
pic_status retile(pic_sim* s, int t) {
    SimDev& h = s->h;
    if (!tile_ok(h, t)) return fail(s, PIC_EINVAL, "tile %d must be even, at least 4 and divide every box extent", t);
    bool same = true;
    for (int a = 0; a < 3; ++a)
        if (!(h.dim == 2 && a == 1) && h.T[a] != t) same = false;
    if (same) return PIC_OK;
    {
        SimDev probe = h;
        const int tt[3] = {t, t, t};
        set_tiling(probe, tt);
        cudaDeviceProp prop;
        CU(s, cudaGetDeviceProperties(&prop, s->device));
        if (pic_particle_smem_bytes(h.dim, h.order, probe.T, s->threads, s->prec) > prop.sharedMemPerBlockOptin)
            return fail(s, PIC_EUNSUPPORTED, "tile %d does not fit in shared memory", t);
    }
    TRY(sync_and_check(s));
    TRY(pull_sim(s));
    int64_t np[PIC_MAXSP] = {0, 0, 0, 0};
    for (int i = 0; i < h.nsp; ++i)
        CU(s, cudaMemcpyAsync(&np[i], h.sp[i].off + h.ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    const int tt[3] = {t, t, t};
    set_tiling(h, tt);
    TRY(encode_tmaps(s));
    for (int i = 0; i < h.nsp; ++i) {
        SpeciesDev& sp = h.sp[i];
        if (h.ntiles > s->tiles_cap[i]) {
            TRY(dalloc(s, &sp.count, h.ntiles + 1));
            TRY(dalloc(s, &sp.cursor, h.ntiles + 1));
            TRY(dalloc(s, &sp.off, h.ntiles + 2));
            s->tiles_cap[i] = h.ntiles;
        }
        TRY(ensure_scan_part(s));
        CU(s, cudaMemsetAsync(sp.count, 0, (h.ntiles + 1) * sizeof(int32_t), s->stream));
        CU(s, cudaMemsetAsync(sp.cursor, 0, (h.ntiles + 1) * sizeof(int32_t), s->stream));
        CU(s, cudaMemsetAsync(sp.off, 0, (h.ntiles + 2) * sizeof(int64_t), s->stream));
        CU(s, cudaMemcpyAsync(sp.off + h.ntiles, &np[i], sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    }
    TRY(upload_sim(s));
    for (int i = 0; i < h.nsp; ++i) {
        CU(s, pic_launch_initial_keys(s->d, h, i, np[i], s->stream));
        CU(s, pic_launch_sort(s->d, h, i, s->stream));
    }
    TRY(sync_and_check(s));
    TRY(pull_sim(s));
    s->graph_dirty = true;
    return PIC_OK;
}

pic_status ensure_ready(pic_sim* s) {
    if (!s->stepped) {
        // the first step: freeze the layout, make the starting plan
        TRY(upload_sim(s));
        if (s->plan.units.empty()) TRY(initial_plan(s));
        s->stepped = true;
    }
    if (s->graph_dirty) TRY(capture_graph(s));
    return PIC_OK;
}

// re-plans after a change of the number of persistent CTAs
pic_status replan(pic_sim* s) {
    if (!s->stepped) return PIC_OK;
    pic_lb_params p = s->lb_set ? s->lb : default_lb();
    if (p.mode == PIC_LB_NONE || s->last_costs.empty()) return initial_plan(s);
    const int nw = n_workers_for(s, p);
    const int split = p.split > 0 ? p.split : s->split;
    std::vector<pic::Unit> units = pic::make_units(s->last_costs.data(), s->last_np.data(),
                                                   s->h.nboxes, nw, split, 256, true);
    std::vector<double> uc;
    std::vector<int32_t> assign;
    map_units(s, p, units, nw, uc, assign);  // the simulation's own policy
    build_plan(s, units, assign, nw, p.sched, p.policy == PIC_POLICY_BOX_ORDER);
    return upload_plan(s);
}

}  // namespace

pic_status pic_record_error(pic_status st, const char* msg) {
    g_last_error = msg;
    return st;
}

// ---- helpers for the other host files of the library (pic_sim.h) ----
pic_status pic_sim_fail(pic_sim* s, pic_status st, const char* msg) { return fail(s, st, "%s", msg); }
pic_status pic_sim_check(pic_sim* s) { return check(s); }
pic_status pic_sim_upload(pic_sim* s) { return upload_sim(s); }
pic_status pic_sim_pull(pic_sim* s) { return pull_sim(s); }
pic_status pic_sim_sync(pic_sim* s) { return sync_and_check(s); }
pic_status pic_sim_dalloc(pic_sim* s, void** p, size_t bytes) {
    char* q = nullptr;
    pic_status st = dalloc(s, &q, bytes);
    *p = q;
    return st;
}
void pic_sim_dfree(pic_sim* s, void* p) {
    if (!p) return;
    for (size_t i = 0; i < s->allocs.size(); ++i)
        if (s->allocs[i] == p) {
            cudaFree(p);
            s->allocs.erase(s->allocs.begin() + (long)i);
            return;
        }
}
pic_status pic_sim_ensure_ready(pic_sim* s) { return ensure_ready(s); }
pic_status pic_sim_launch_push(pic_sim* s) {
    const SimDev& h = s->h;
    const int64_t jbytes = (int64_t)h.pn[0] * h.pn[1] * h.pn[2] * 3 * sizeof(double);
    CU(s, cudaMemsetAsync(h.F[6], 0, jbytes, s->stream));
    if (h.nsp > 0) {
        LaunchCfg cfg{s->threads, s->ctas, s->minb, s->prec, s->ppt};
        CU(s, pic_launch_particles(h.dim, h.order, cfg, s->smem, s->ds, s->d, s->stream));
    }
    return PIC_OK;
}

// ---- hooks for the request server (same library, not exported) ----
int64_t pic_internal_bytes(const pic_sim* s) { return s ? s->bytes : 0; }

pic_status pic_internal_mirror(pic_sim* s, SimDev* out) {
    TRY(check(s));
    TRY(pull_sim(s));
    *out = s->h;
    return PIC_OK;
}

SimDev* pic_internal_device_sim(pic_sim* s) { return s ? s->d : nullptr; }

// the handle's device state was advanced outside pic_step (request server):
// never upload the host mirror over it again
void pic_internal_mark_external(pic_sim* s) {
    if (s) s->stepped = true;
}

// device bytes that pic_init + pic_add_species request for this geometry and
// these species sizes (mirrors the allocations made there)
int64_t pic_internal_estimate_bytes(const pic_grid_desc* g, const int64_t* np, int nsp) {
    int64_t pvol = 1, nboxes = 1, ntiles = 1;
    for (int a = 0; a < 3; ++a) {
        const bool act = !(g->dim == 2 && a == 1);
        const int gw = act ? (a == 0 ? (g->shape_order == 3 ? PIC_GX + 1 : PIC_GX)
                                     : (g->shape_order >= 2 ? PIC_G + 1 : PIC_G)) : 0;
        pvol *= g->ncell[a] + 2 * gw;
        const int64_t nb = g->ncell[a] / std::max<int32_t>(1, g->box[a]);
        nboxes *= nb;
        const int T = act ? largest_even_divisor_le(g->box[a], g->dim == 3 ? 8 : 16) : 1;
        ntiles *= nb * (T > 0 ? g->box[a] / T : 1);
    }
    auto r = [](int64_t n, int64_t sz) { return std::max<int64_t>(n, 1) * sz; };
    int64_t b = r(pvol * PIC_NCOMP, 8) + 2 * r(nboxes, 8) + 8 + 4 + (int64_t)sizeof(SimDev) + (int64_t)pic_ring_bytes(pic_sm_count()) +
                (int64_t)sizeof(SchedDev) + r(8193, 4) + r(8192, 4) + r(2, 4) + r(4, 8) + r(nboxes, 8);
    if (nsp > 0) b += r((ntiles + 1 + 1023) / 1024, 8);  // block sums of the histogram scan
    for (int i = 0; i < nsp; ++i) {
        const int64_t cap = std::max<int64_t>(np[i], 1);
        b += 14 * r(cap, 8) + 2 * r(cap, 8) + r(cap, 4) + 2 * r(ntiles + 1, 4) + r(ntiles + 2, 8) + 8;
    }
    return b;
}

const char* pic_internal_error(const pic_sim* s) { return s ? s->err.c_str() : g_last_error.c_str(); }

// ====================================================================== ABI
extern "C" {

const char* pic_last_error(const pic_sim* s) {
    return s ? s->err.c_str() : g_last_error.c_str();
}

pic_status pic_init(const pic_grid_desc* desc, pic_sim** out) {
    if (!desc || !out) return fail(nullptr, PIC_EINVAL, "null argument");
    *out = nullptr;
    const pic_grid_desc& g = *desc;
    if (g.dim != 2 && g.dim != 3) return fail(nullptr, PIC_EINVAL, "dim must be 2 or 3");
    if (g.shape_order < 1 || g.shape_order > 3)
        return fail(nullptr, PIC_EINVAL, "shape_order must be 1, 2 or 3");
    if (g.dim == 2 && (g.ncell[1] != 1 || g.box[1] != 1))
        return fail(nullptr, PIC_EINVAL, "2D runs need ncell[1] == box[1] == 1");
    for (int a = 0; a < 3; ++a) {
        if (g.ncell[a] < 1 || g.ncell[a] > (1 << 20) || g.box[a] < 1 || g.ncell[a] % g.box[a] != 0)
            return fail(nullptr, PIC_EINVAL, "box extents must divide ncell (direction %d)", a);
        if (!(g.dx[a] > 0.0) && !(g.dim == 2 && a == 1))
            return fail(nullptr, PIC_EINVAL, "dx must be positive");
    }
    if (g.ncell[0] % 2 != 0) return fail(nullptr, PIC_EINVAL, "ncell[0] must be even");
    if (g.absorb_cells < 0 || (g.absorb_cells > 0 && (g.absorb_cells < 4 || 2 * g.absorb_cells >= g.ncell[2])))
        return fail(nullptr, PIC_EINVAL, "absorb_cells must be 0 or in [4, ncell[2]/2)");
    pic_sim* s = new (std::nothrow) pic_sim();
    if (!s) return fail(nullptr, PIC_ENOMEM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return fail(nullptr, PIC_ECUDA, "no CUDA device");
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, s->device) != cudaSuccess) {
        delete s;
        return fail(nullptr, PIC_ECUDA, "cudaGetDeviceProperties failed");
    }
    s->nsm = prop.multiProcessorCount;
    if (g.stream) {
        s->stream = (cudaStream_t)g.stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return fail(nullptr, PIC_ECUDA, "stream creation failed");
        }
        s->own_stream = true;
    }
    SimDev& h = s->h;
    h.dim = g.dim;
    h.order = g.shape_order;
    h.absorb = g.absorb_cells;
    h.capture = PIC_CAPTURE_CLOCK | PIC_CAPTURE_TIME;
    const int tdef = (g.dim == 3) ? 8 : 16;
    int tdefs[3];
    double inv2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        bool act = !(g.dim == 2 && a == 1);
        h.n[a] = (int)g.ncell[a];
        h.nd[a] = (double)h.n[a];
        // x guard: even tile origin - E/B halo + guard must be even (TMA)
        // y, z: 2 guards, 3 for quadratic and cubic shapes, whose current
        // windows reach 3 nodes above the domain
        h.g[a] = act ? (a == 0 ? (g.shape_order == 3 ? PIC_GX + 1 : PIC_GX)
                               : (g.shape_order >= 2 ? PIC_G + 1 : PIC_G)) : 0;
        h.pn[a] = h.n[a] + 2 * h.g[a];
        h.bsz[a] = g.box[a];
        h.nb[a] = h.n[a] / h.bsz[a];
        tdefs[a] = 1;
        if (act) {
            // default tile edge: the largest even divisor of the box extent up
            // to 8 (3D) or 16 (2D)
            tdefs[a] = largest_even_divisor_le(h.bsz[a], tdef);
            if (tdefs[a] == 0) {
                pic_destroy(s);
                return fail(nullptr, PIC_EUNSUPPORTED, "box extent %d has no even tile size", h.bsz[a]);
            }
            inv2 += 1.0 / (g.dx[a] * g.dx[a]);
        }
        h.d[a] = act ? g.dx[a] : 1.0;
        h.invd[a] = act ? 1.0 / g.dx[a] : 0.0;
    }
    h.nboxes = h.nb[0] * h.nb[1] * h.nb[2];
    set_tiling(h, tdefs);
    h.dt = g.dt > 0.0 ? g.dt : (g.cfl > 0.0 ? g.cfl : 0.99) / std::sqrt(inv2);
    for (int a = 0; a < 3; ++a) {
        bool act = !(g.dim == 2 && a == 1);
        h.dtd[a] = act ? h.dt / h.d[a] : 0.0;
    }
    h.jlo = h.order == 1 ? 1 : 2;
    if (g.dim == 3) {
        h.jfac[0] = -1.0 / (h.d[1] * h.d[2] * h.dt);
        h.jfac[1] = -1.0 / (h.d[0] * h.d[2] * h.dt);
        h.jfac[2] = -1.0 / (h.d[0] * h.d[1] * h.dt);
    } else {
        h.jfac[0] = -1.0 / (h.d[2] * h.dt);
        h.jfac[1] = 0.0;
        h.jfac[2] = -1.0 / (h.d[0] * h.dt);
        h.jyfac2d = 1.0 / (h.d[0] * h.d[2]);
    }
    const int64_t pvol = (int64_t)h.pn[0] * h.pn[1] * h.pn[2];
    pic_status st;
    double* fields = nullptr;
    if ((st = dalloc(s, &fields, (size_t)pvol * PIC_NCOMP)) != PIC_OK) {
        g_last_error = s->err;
        pic_destroy(s);
        return st;
    }
    for (int c = 0; c < PIC_NCOMP; ++c) h.F[c] = fields + (int64_t)c * pvol;
    if (cudaMemset(fields, 0, (size_t)pvol * PIC_NCOMP * sizeof(double)) != cudaSuccess ||
        (st = dalloc(s, &h.cost_clock, h.nboxes)) != PIC_OK || (st = dalloc(s, &h.cost_time, h.nboxes)) != PIC_OK ||
        (st = dalloc(s, &h.step, 1)) != PIC_OK ||
        (st = dalloc(s, &h.err, 1)) != PIC_OK || (st = dalloc(s, &s->d, 1)) != PIC_OK ||
        (st = dalloc(s, &s->ds, 1)) != PIC_OK || (st = dalloc(s, &s->hs.list_off, 8193)) != PIC_OK ||
        (st = dalloc(s, &s->hs.head, 8192)) != PIC_OK || (st = dalloc(s, &s->hs.meta, 2)) != PIC_OK ||
        (st = dalloc(s, &s->hs.rings, pic_ring_bytes(s->nsm) / sizeof(double))) != PIC_OK ||
        (st = dalloc(s, &s->d_scalar, 4)) != PIC_OK || (st = dalloc(s, &s->d_box_np, h.nboxes)) != PIC_OK) {
        g_last_error = s->err;
        pic_destroy(s);
        return st == PIC_OK ? PIC_ECUDA : st;
    }
    cudaMemset(h.cost_clock, 0, h.nboxes * sizeof(uint64_t));
    cudaMemset(h.cost_time, 0, h.nboxes * sizeof(uint64_t));
    cudaMemset(h.step, 0, sizeof(int64_t));
    cudaMemset(h.err, 0, sizeof(int32_t));
    cudaMemset(s->hs.head, 0, 8192 * sizeof(int32_t));
    s->hs.err = h.err;
    if (cudaMemcpy(s->ds, &s->hs, sizeof(SchedDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        pic_destroy(s);
        return fail(nullptr, PIC_ECUDA, "schedule upload failed");
    }
    // TMA descriptors of the six padded E/B arrays
    if (encode_tmaps(s) != PIC_OK) {
        g_last_error = s->err;
        pic_destroy(s);
        return PIC_EUNSUPPORTED;
    }
    s->box_ijk.resize(3 * (size_t)h.nboxes);
    for (int64_t b = 0; b < h.nboxes; ++b) box_coords(s, b, &s->box_ijk[3 * b]);
    s->lb = default_lb();
    for (int i = 0; i < 4; ++i) cudaEventCreate(&s->ev[i]);
    if (cudaDeviceSynchronize() != cudaSuccess || upload_sim(s) != PIC_OK) {
        pic_destroy(s);
        return fail(nullptr, PIC_ECUDA, "layout upload failed");
    }
    if (configure_launch(s) != PIC_OK) {
        g_last_error = s->err;
        pic_destroy(s);
        return PIC_EUNSUPPORTED;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        pic_destroy(s);
        return fail(nullptr, PIC_ECUDA, "initialisation failed");
    }
    *out = s;
    return PIC_OK;
}

pic_status pic_add_species(pic_sim* s, double charge, double mass, int64_t np,
                           const double* const soa[7], const int64_t* ids, int on_device,
                           int* species_id_out) {
    TRY(check(s));
    if (s->stepped) return fail(s, PIC_ESTATE, "species must be added before the first step");
    SimDev& h = s->h;
    if (h.nsp >= PIC_MAXSP) return fail(s, PIC_EINVAL, "at most %d species", PIC_MAXSP);
    if (np < 0 || np > (int64_t)1 << 31 || !(mass > 0.0) || !std::isfinite(charge) || !soa)
        return fail(s, PIC_EINVAL, "bad species arguments");
    for (int a = 0; a < 7; ++a)
        if (!soa[a] && !(a == 1 && h.dim == 2) && np > 0)
            return fail(s, PIC_EINVAL, "missing particle array %d", a);
    const int idx = h.nsp;
    SpeciesDev& sp = h.sp[idx];
    sp.q = charge;
    sp.m = mass;
    sp.kq = charge * h.dt / (2.0 * mass);
    const int64_t cap = std::max<int64_t>(np, 1);
    sp.cap = cap;
    for (int a = 0; a < 7; ++a) {
        TRY(dalloc(s, &sp.cur[a], cap));
        TRY(dalloc(s, &sp.alt[a], cap));
    }
    TRY(dalloc(s, &sp.id, cap));
    TRY(dalloc(s, &sp.id_alt, cap));
    TRY(dalloc(s, &sp.key, cap));
    TRY(dalloc(s, &sp.count, h.ntiles + 1));
    TRY(dalloc(s, &sp.cursor, h.ntiles + 1));
    TRY(dalloc(s, &sp.off, h.ntiles + 2));
    s->tiles_cap[idx] = h.ntiles;
    TRY(ensure_scan_part(s));
    TRY(dalloc(s, &sp.np_prev, 1));
    CU(s, cudaMemsetAsync(sp.count, 0, (h.ntiles + 1) * sizeof(int32_t), s->stream));
    CU(s, cudaMemsetAsync(sp.cursor, 0, (h.ntiles + 1) * sizeof(int32_t), s->stream));
    CU(s, cudaMemsetAsync(sp.off, 0, (h.ntiles + 2) * sizeof(int64_t), s->stream));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (np > 0) {
        // the input lands in the alternate buffers and is gathered into the
        // current ones in a scrambled order (see pic_launch_permute)
        for (int a = 0; a < 7; ++a) {
            if (a == 1 && h.dim == 2) {
                CU(s, cudaMemsetAsync(sp.cur[1], 0, np * sizeof(double), s->stream));
                continue;
            }
            CU(s, cudaMemcpyAsync(sp.alt[a], soa[a], np * sizeof(double), kind, s->stream));
        }
        if (ids) {
            CU(s, cudaMemcpyAsync(sp.id_alt, ids, np * sizeof(int64_t), kind, s->stream));
        } else {
            std::vector<int64_t> seq(np);
            for (int64_t i = 0; i < np; ++i) seq[i] = i;
            CU(s, cudaMemcpyAsync(sp.id_alt, seq.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice,
                                  s->stream));
            CU(s, cudaStreamSynchronize(s->stream));
        }
        CU(s, pic_launch_permute(sp.cur, sp.alt, sp.id, sp.id_alt, np, h.dim == 2 ? 1 : -1, s->stream));
        // positions to global cell units
        for (int a = 0; a < 3; ++a) {
            if (a == 1 && h.dim == 2) continue;
            CU(s, pic_launch_to_cells(sp.cur[a], np, h.d[a], h.n[a], s->stream));
        }
    }
    // validate positions on the host side of the copy: range check via a
    // device->host read is costly; the sort kernel clamps and the first step
    // flags particles that do not sit in their tile
    h.nsp = idx + 1;
    s->np_init[idx] = np;
    CU(s, cudaMemcpyAsync(sp.off + h.ntiles, &s->np_init[idx], sizeof(int64_t),
                          cudaMemcpyHostToDevice, s->stream));
    TRY(upload_sim(s));
    CU(s, pic_launch_initial_keys(s->d, h, idx, np, s->stream));
    CU(s, pic_launch_sort(s->d, h, idx, s->stream));
    TRY(sync_and_check(s));
    TRY(pull_sim(s));
    s->graph_dirty = true;
    if (species_id_out) *species_id_out = idx;
    return PIC_OK;
}

pic_status pic_add_background(pic_sim* s, double rho0) {
    TRY(check(s));
    if (!std::isfinite(rho0)) return fail(s, PIC_EINVAL, "rho0 must be finite");
    s->rho0 += rho0;
    return PIC_OK;
}

pic_status pic_add_laser(pic_sim* s, const pic_laser_desc* L) {
    TRY(check(s));
    if (s->stepped) return fail(s, PIC_ESTATE, "the laser must be added before the first step");
    if (!L || L->k_ant < 0 || L->k_ant >= s->h.n[2] || !(L->w0 > 0.0) || !(L->tau > 0.0))
        return fail(s, PIC_EINVAL, "bad laser description");
    LaserDev& d = s->h.las;
    d.on = 1;
    d.k_ant = (int)L->k_ant;
    d.a0 = L->a0; d.w0 = L->w0; d.tau = L->tau; d.t_peak = L->t_peak;
    d.omega = L->omega; d.xc = L->xc; d.yc = L->yc;
    s->graph_dirty = true;
    return upload_sim(s);
}

pic_status pic_set_field(pic_sim* s, int comp, const double* data, int on_device) {
    TRY(check(s));
    if (comp < PIC_EX || comp > PIC_BZ || !data) return fail(s, PIC_EINVAL, "bad field component");
    const SimDev& h = s->h;
    const int64_t nc = (int64_t)h.n[0] * h.n[1] * h.n[2];
    const double* src = data;
    double* tmp = nullptr;
    if (!on_device) {
        TRY(talloc(s, &tmp, (size_t)nc));
        CU(s, cudaMemcpyAsync(tmp, data, nc * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        src = tmp;
    }
    cudaError_t e = pic_launch_pad(src, h.F[comp], h, s->stream);
    if (e == cudaSuccess) e = pic_launch_guards(s->d, h, comp, 1, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(s, PIC_ECUDA, "field upload failed: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(s, PIC_ECUDA, "field upload failed: %s", cudaGetErrorString(e2));
    return PIC_OK;
}

pic_status pic_set_gather(pic_sim* s, int kind) {
    TRY(check(s));
    if (kind != PIC_GATHER_MOMENTUM && kind != PIC_GATHER_ENERGY)
        return fail(s, PIC_EINVAL, "unknown gather kind %d", kind);
    // after the first step the device copy owns the species buffer pointers
    if (s->stepped) {
        TRY(sync_and_check(s));
        TRY(pull_sim(s));
    }
    s->h.ec = kind == PIC_GATHER_ENERGY ? 1 : 0;
    return upload_sim(s);
}

pic_status pic_set_cost_capture(pic_sim* s, int mask) {
    TRY(check(s));
    if (mask < 0 || mask > (PIC_CAPTURE_CLOCK | PIC_CAPTURE_TIME))
        return fail(s, PIC_EINVAL, "bad capture mask %d", mask);
    if (s->stepped) {
        TRY(sync_and_check(s));
        TRY(pull_sim(s));
    }
    s->h.capture = mask;
    return upload_sim(s);
}

pic_status pic_selftest_bounded_wait(pic_sim* s, int64_t limit_ns) {
    TRY(check(s));
    if (limit_ns < 1000 || limit_ns > 5000000000ll)
        return fail(s, PIC_EINVAL, "limit_ns must be in [1e3, 5e9]");
    CU(s, pic_launch_selftest_wait(s->hs.err, (uint64_t)limit_ns, s->stream));
    return sync_and_check(s);
}

pic_status pic_set_step(pic_sim* s, int64_t step) {
    TRY(check(s));
    if (step < 0) return fail(s, PIC_EINVAL, "step must be >= 0");
    TRY(sync_and_check(s));
    CU(s, cudaMemcpyAsync(s->h.step, &step, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    s->step_count = step;
    return PIC_OK;
}

pic_status pic_set_lb_params(pic_sim* s, const pic_lb_params* p) {
    TRY(check(s));
    TRY(validate_lb(s, p));
    bool sched_changed = !s->lb_set || p->sched != s->lb.sched || p->n_workers != s->lb.n_workers;
    s->lb = *p;
    s->lb_set = true;
    s->static_done = false;
    if (p->split > 0) s->split = p->split;
    if (s->stepped && sched_changed) {
        TRY(replan(s));
        s->graph_dirty = true;
    }
    return PIC_OK;
}

pic_status pic_step(pic_sim* s, int nsteps) {
    TRY(check(s));
    if (nsteps < 0) return fail(s, PIC_EINVAL, "nsteps must be >= 0");
    TRY(ensure_ready(s));
    pic_stats& st = s->stats;
    st = pic_stats{};
    for (int i = 0; i < nsteps; ++i) {
        if (s->profiling) {
            TRY(enqueue_step(s, true));
            CU(s, cudaEventSynchronize(s->ev[3]));
            float a = 0, b = 0, c = 0;
            cudaEventElapsedTime(&a, s->ev[0], s->ev[1]);
            cudaEventElapsedTime(&b, s->ev[1], s->ev[2]);
            cudaEventElapsedTime(&c, s->ev[2], s->ev[3]);
            st.ms_particle += a;
            st.ms_fields += b;
            st.ms_sort += c;
            st.ms_total += a + b + c;
        } else {
            CU(s, cudaGraphLaunch(s->graph, s->stream));
        }
        st.steps++;
        st.launches += s->kernels_per_step ? s->kernels_per_step : count_kernels(s);
        st.particle_launches += s->h.nsp > 0 ? 1 : 0;
        s->step_count++;
        const pic_lb_params& p = s->lb;
        if (s->lb_set && p.mode != PIC_LB_NONE && s->step_count % p.interval == 0) {
            if (p.mode == PIC_LB_DYNAMIC) {
                TRY(rebalance(s, p, p.theta, nullptr));
            } else if (!s->static_done) {
                TRY(rebalance(s, p, 0.0, nullptr));
                s->static_done = true;
            }
            TRY(check_device_error(s));
        }
    }
    return PIC_OK;
}

pic_status pic_sync(pic_sim* s) {
    TRY(check(s));
    return sync_and_check(s);
}

pic_status pic_get_box_costs(pic_sim* s, int strategy, double* costs_out, int64_t* np_out) {
    TRY(check(s));
    if (!costs_out || (strategy != PIC_COST_HEURISTIC && strategy != PIC_COST_DEVICE_CLOCK &&
                       strategy != PIC_COST_KERNEL_TIME))
        return fail(s, PIC_EINVAL, "bad cost request");
    if (!s->stepped) TRY(upload_sim(s));
    TRY(sync_and_check(s));
    std::vector<double> c;
    std::vector<int64_t> np;
    TRY(box_costs(s, strategy, s->lb.w_p, s->lb.w_c, c, np));
    memcpy(costs_out, c.data(), c.size() * sizeof(double));
    if (np_out) memcpy(np_out, np.data(), np.size() * sizeof(int64_t));
    return PIC_OK;
}

pic_status pic_rebalance(pic_sim* s, const pic_lb_params* params, pic_lb_result* out,
                         int32_t* assign_out) {
    TRY(check(s));
    TRY(validate_lb(s, params));
    TRY(ensure_ready(s));
    TRY(sync_and_check(s));
    pic_lb_params p = *params;
    if (p.sched != s->lb.sched || !s->lb_set) {
        // an explicit call may switch the schedule kind
        s->lb.sched = p.sched;
    }
    TRY(rebalance(s, p, p.theta, out));
    if (assign_out) {
        for (int64_t b = 0; b < s->h.nboxes; ++b) assign_out[b] = -1;
        const SimPlan& P = s->plan;
        for (size_t i = 0; i < P.units.size(); ++i)
            if (P.units[i].chunk == 0) assign_out[P.units[i].box] = P.unit_worker[i];
    }
    return check_device_error(s);
}

pic_status pic_get_efficiency(pic_sim* s, int strategy, int reset_window, double* e_out) {
    TRY(check(s));
    if (!e_out || (strategy != PIC_COST_HEURISTIC && strategy != PIC_COST_DEVICE_CLOCK &&
                   strategy != PIC_COST_KERNEL_TIME))
        return fail(s, PIC_EINVAL, "bad efficiency request");
    TRY(ensure_ready(s));
    TRY(sync_and_check(s));
    std::vector<double> c;
    std::vector<int64_t> np;
    TRY(box_costs(s, strategy, s->lb.w_p, s->lb.w_c, c, np));
    *e_out = plan_efficiency(s, c);
    if (reset_window) {
        CU(s, cudaMemsetAsync(s->h.cost_clock, 0, s->h.nboxes * sizeof(uint64_t), s->stream));
        CU(s, cudaMemsetAsync(s->h.cost_time, 0, s->h.nboxes * sizeof(uint64_t), s->stream));
        CU(s, cudaStreamSynchronize(s->stream));
    }
    return PIC_OK;
}

pic_status pic_get_lb_log(pic_sim* s, pic_lb_result* out, int64_t max, int64_t* n_total) {
    if (!s || !n_total || max < 0 || (max > 0 && !out)) return fail(s, PIC_EINVAL, "bad log arguments");
    const int64_t n = (int64_t)s->lb_log.size();
    for (int64_t i = 0; i < std::min(n, max); ++i) out[i] = s->lb_log[i];
    *n_total = n;
    return PIC_OK;
}

pic_status pic_balance_compute(const double* costs, int64_t nboxes, const int32_t* box_ijk,
                               int dim, int n_workers, int policy, double cap_factor,
                               int32_t* assign_out, double* e_out) {
    if (nboxes < 0 || n_workers < 1 || !assign_out || (nboxes > 0 && !costs))
        return fail(nullptr, PIC_EINVAL, "bad balancer arguments");
    for (int64_t b = 0; b < nboxes; ++b)
        if (!(costs[b] >= 0.0) || !std::isfinite(costs[b]))
            return fail(nullptr, PIC_EINVAL, "box %lld has a negative or non-finite cost", (long long)b);
    if (policy == PIC_POLICY_KNAPSACK) {
        if (!(cap_factor > 0.0)) return fail(nullptr, PIC_EINVAL, "cap_factor must be positive");
        pic::knapsack(costs, nboxes, n_workers, cap_factor, assign_out);
    } else if (policy == PIC_POLICY_SFC) {
        if (!box_ijk || (dim != 2 && dim != 3))
            return fail(nullptr, PIC_EINVAL, "SFC needs box coordinates and dim 2 or 3");
        for (int64_t b = 0; b < 3 * nboxes; ++b)
            if (box_ijk[b] < 0) return fail(nullptr, PIC_EINVAL, "negative box coordinate");
        pic::sfc(costs, box_ijk, nboxes, dim, n_workers, assign_out);
    } else {
        return fail(nullptr, PIC_EINVAL, "unknown policy %d", policy);
    }
    if (e_out) *e_out = pic::lb_efficiency(costs, assign_out, nboxes, n_workers);
    return PIC_OK;
}

pic_status pic_lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes,
                             int n_workers, double* e_out) {
    if (nboxes < 0 || n_workers < 1 || !e_out || (nboxes > 0 && (!costs || !assign)))
        return fail(nullptr, PIC_EINVAL, "bad efficiency arguments");
    for (int64_t b = 0; b < nboxes; ++b)
        if (assign[b] < 0 || assign[b] >= n_workers)
            return fail(nullptr, PIC_EINVAL, "assignment out of range");
    *e_out = pic::lb_efficiency(costs, assign, nboxes, n_workers);
    return PIC_OK;
}

pic_status pic_read_fields(pic_sim* s, int comp, double* out, int on_device) {
    TRY(check(s));
    if (comp < PIC_EX || comp > PIC_RHO || !out) return fail(s, PIC_EINVAL, "bad field component");
    if (!s->stepped) TRY(upload_sim(s));
    TRY(sync_and_check(s));
    const SimDev& h = s->h;
    const int64_t nc = (int64_t)h.n[0] * h.n[1] * h.n[2];
    double* dst = out;
    double* tmp = nullptr;
    if (!on_device) {
        TRY(talloc(s, &tmp, (size_t)nc));
        dst = tmp;
    }
    cudaError_t e;
    if (comp == PIC_RHO) e = pic_launch_rho(s->d, h, dst, s->rho0, s->stream);
    else e = pic_launch_unpad(h.F[comp], dst, h, s->stream);
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, tmp, nc * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(s, PIC_ECUDA, "field read failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return PIC_OK;
}

pic_status pic_num_particles(pic_sim* s, int species, int64_t* np_out) {
    TRY(check(s));
    if (species < 0 || species >= s->h.nsp || !np_out) return fail(s, PIC_EINVAL, "bad species");
    TRY(sync_and_check(s));
    CU(s, cudaMemcpyAsync(np_out, s->h.sp[species].off + s->h.ntiles, sizeof(int64_t),
                          cudaMemcpyDeviceToHost, s->stream));
    CU(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

pic_status pic_read_particles(pic_sim* s, int species, double* const soa_out[7], int64_t* id_out,
                              int on_device) {
    TRY(check(s));
    if (species < 0 || species >= s->h.nsp || !soa_out) return fail(s, PIC_EINVAL, "bad species");
    int64_t np = 0;
    TRY(pic_num_particles(s, species, &np));
    TRY(pull_sim(s));
    const SpeciesDev& sp = s->h.sp[species];
    if (np == 0) return PIC_OK;
    double* tmp = nullptr;
    if (!on_device) TRY(talloc(s, &tmp, (size_t)np));
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 7 && e == cudaSuccess; ++a) {
        if (!soa_out[a]) continue;
        double* dst = on_device ? soa_out[a] : tmp;
        if (a == 1 && s->h.dim == 2) {
            e = cudaMemsetAsync(dst, 0, np * sizeof(double), s->stream);
        } else if (a < 3) {
            e = pic_launch_from_cells(sp.cur[a], dst, np, s->h.d[a], s->stream);
        } else {
            e = cudaMemcpyAsync(dst, sp.cur[a], np * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
        }
        if (e == cudaSuccess && !on_device)
            e = cudaMemcpyAsync(soa_out[a], tmp, np * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s->stream);
    }
    if (e == cudaSuccess && id_out)
        e = cudaMemcpyAsync(id_out, sp.id, np * sizeof(int64_t),
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
    cudaError_t e2 = cudaStreamSynchronize(s->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(s, PIC_ECUDA, "particle read failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return PIC_OK;
}

pic_status pic_set_launch(pic_sim* s, const pic_launch_cfg* cfg) {
    TRY(check(s));
    if (!cfg) return fail(s, PIC_EINVAL, "null launch configuration");
    if (cfg->threads > 0) {
        if (cfg->threads % 32 != 0 || cfg->threads > 256)
            return fail(s, PIC_EINVAL, "threads must be a multiple of 32, at most 256");
        s->threads = cfg->threads;
    }
    if (cfg->ctas_per_sm > 0) {
        if (cfg->ctas_per_sm > PIC_RING_CTAS_PER_SM) return fail(s, PIC_EINVAL, "ctas_per_sm must be 1..4");
        s->ctas_per_sm = cfg->ctas_per_sm;
    }
    const int old_split = s->split;
    if (cfg->split > 0) s->split = cfg->split;
    if (cfg->precision < 0 || cfg->precision > 3) return fail(s, PIC_EINVAL, "precision must be 0, 1, 2 or 3");
    if (cfg->ppt < 0 || cfg->ppt > 2) return fail(s, PIC_EINVAL, "ppt must be 1 or 2");
    if (cfg->precision > 0) {
        s->prec = cfg->precision - 1;
        s->graph_dirty = true;
    }
    if (cfg->ppt > 0) {
        s->ppt = cfg->ppt;
        s->graph_dirty = true;
    }
    if (cfg->tile > 0) TRY(retile(s, cfg->tile));
    const int old = s->ctas;
    TRY(configure_launch(s));
    if (s->ctas != old || s->split != old_split) TRY(replan(s));
    return PIC_OK;
}

pic_status pic_get_launch(const pic_sim* s, pic_launch_cfg* cfg) {
    if (!s || !cfg) return fail(nullptr, PIC_EINVAL, "null argument");
    cfg->threads = s->threads;
    cfg->ctas_per_sm = s->ctas / std::max(1, s->nsm);
    cfg->split = s->split;
    cfg->precision = s->prec + 1;
    cfg->tile = s->h.T[0];
    cfg->ppt = s->ppt;
    return PIC_OK;
}

pic_status pic_autotune(pic_sim* s, int steps_per_candidate, pic_launch_cfg* best) {
    TRY(check(s));
    if (steps_per_candidate < 1) return fail(s, PIC_EINVAL, "steps_per_candidate must be >= 1");
    TRY(ensure_ready(s));
    // the events and the profiling switch are restored on every way out
    struct Guard {
        pic_sim* s;
        bool prof;
        cudaEvent_t a = nullptr, b = nullptr;
        ~Guard() {
            s->profiling = prof;
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } g{s, s->profiling};
    CU(s, cudaEventCreate(&g.a));
    CU(s, cudaEventCreate(&g.b));
    s->profiling = false;
    pic_launch_cfg cur{};
    TRY(pic_get_launch(s, &cur));
    cur.precision = 0;
    float best_ms = 1e30f;
    pic_launch_cfg best_cfg = cur;
    // times one candidate on real steps; *ms = 1e30 when it is not resident
    auto trial = [&](const pic_launch_cfg& c, float* ms) -> pic_status {
        *ms = 1e30f;
        TRY(pic_set_launch(s, &c));
        if (s->ctas / s->nsm != c.ctas_per_sm) return PIC_OK;  // not resident: skip
        TRY(pic_step(s, 1));
        CU(s, cudaEventRecord(g.a, s->stream));
        TRY(pic_step(s, steps_per_candidate));
        CU(s, cudaEventRecord(g.b, s->stream));
        CU(s, cudaEventSynchronize(g.b));
        cudaEventElapsedTime(ms, g.a, g.b);
        return PIC_OK;
    };
    auto consider = [&](const pic_launch_cfg& c) -> pic_status {
        float ms;
        TRY(trial(c, &ms));
        if (ms < best_ms) {
            best_ms = ms;
            best_cfg = c;
        }
        return PIC_OK;
    };
    // stage 1: tile size x particles per thread
    const int tmax = s->h.dim == 3 ? 8 : 32;
    for (int t = 4; t <= tmax; t += 2) {
        if (!tile_ok(s->h, t)) continue;
        SimDev probe = s->h;
        const int tt[3] = {t, t, t};
        set_tiling(probe, tt);
        cudaDeviceProp prop;
        CU(s, cudaGetDeviceProperties(&prop, s->device));
        if (pic_particle_smem_bytes(probe.dim, probe.order, probe.T, 256, s->prec) > prop.sharedMemPerBlockOptin)
            continue;
        for (int ppt = 1; ppt <= 2; ++ppt) {
            pic_launch_cfg c = best_ms < 1e29f ? best_cfg : cur;
            c.tile = t;
            c.ppt = ppt;
            TRY(consider(c));
        }
    }
    // stage 2: threads per CTA x resident CTAs per SM (register budget of the kernel variant)
    const pic_launch_cfg after1 = best_cfg;
    for (int threads : {128, 256})
        for (int cps : {1, 2}) {
            if (threads == after1.threads && cps == after1.ctas_per_sm) continue;
            pic_launch_cfg c = after1;
            c.threads = threads;
            c.ctas_per_sm = cps;
            TRY(consider(c));
        }
    // stage 3: work units per worker (how finely heavy boxes are cut), only
    // when load balancing cuts boxes
    if (s->lb_set && s->lb.mode != PIC_LB_NONE) {
        const pic_launch_cfg after2 = best_cfg;
        for (int sp : {4, 16, 64}) {
            if (sp == after2.split) continue;
            pic_launch_cfg c = after2;
            c.split = sp;
            TRY(consider(c));
        }
    }
    s->profiling = g.prof;
    TRY(pic_set_launch(s, &best_cfg));
    if (best) {
        *best = best_cfg;
        best->precision = s->prec + 1;
    }
    return sync_and_check(s);
}

pic_status pic_set_profiling(pic_sim* s, int on) {
    TRY(check(s));
    s->profiling = on != 0;
    return PIC_OK;
}

pic_status pic_get_stats(pic_sim* s, pic_stats* out) {
    TRY(check(s));
    if (!out) return fail(s, PIC_EINVAL, "null stats");
    *out = s->stats;
    return PIC_OK;
}

pic_status pic_destroy(pic_sim* s) {
    if (!s) return PIC_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (void* p : s->allocs) cudaFree(p);
    for (int i = 0; i < 4; ++i)
        if (s->ev[i]) cudaEventDestroy(s->ev[i]);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return PIC_OK;
}

}  // extern "C"
