// pic_sim.h -- the library-side state of one simulation handle and the host
// helpers that pic_api.cu exports to the other host files of the library
// (pic_shard.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/pic_api.h"
#include "pic_internal.h"

// work schedule of the persistent particle kernel
struct SimPlan {
    std::vector<UnitDev> units;      // in list order
    std::vector<int32_t> list_off;   // nlists + 1
    std::vector<double> unit_cost;   // model cost of each unit (list order)
    std::vector<int32_t> unit_worker;
    int nlists = 1;
    int n_workers = 1;
};

struct pic_sim {
    std::string err = "no error";
    bool poisoned = false;
    bool stepped = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    SimDev h{};            // host mirror (species buffer pointers are swapped on the device)
    SimDev* d = nullptr;   // device copy
    SchedDev hs{};
    SchedDev* ds = nullptr;
    int64_t units_cap = 0;
    double rho0 = 0.0;
    std::vector<void*> allocs;
    int64_t bytes = 0;  // device bytes allocated by the handle
    int64_t np_init[PIC_MAXSP] = {0, 0, 0, 0};
    // launch configuration
    int nsm = 0;
    int threads = 256;
    int ctas_per_sm = 1;
    int split = 16;
    int ctas = 0;
    int minb = 1;
    int prec = 0;  // 0 FP64, 1 float-float, 2 FP32 particle push
    int ppt = 1;   // particles per thread per loop iteration
    size_t smem = 0;
    int64_t tiles_cap[PIC_MAXSP] = {0, 0, 0, 0};  // sort arrays allocated for this many tiles
    // load balancing
    pic_lb_params lb{};
    bool lb_set = false;
    bool static_done = false;
    SimPlan plan;
    std::vector<double> last_costs;
    std::vector<int64_t> last_np;
    int64_t step_count = 0;
    std::vector<int32_t> box_ijk;
    // graph
    cudaGraphExec_t graph = nullptr;
    bool graph_dirty = true;
    int kernels_per_step = 0;
    // profiling
    bool profiling = false;
    pic_stats stats{};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // device scratch
    int64_t* d_scalar = nullptr;
    int64_t* d_box_np = nullptr;
    std::vector<pic_lb_result> lb_log;
    // box sharding across ranks (pic_shard.cu): the owner of every box, this
    // handle's rank, the owner map on the device, and the outbox of particles
    // leaving this rank's boxes
    std::vector<int32_t> owner;
    int rank = -1;
    int32_t* d_owner = nullptr;
    double* out_soa[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t* out_id = nullptr;
    int64_t out_cap = 0;
    int32_t* d_out_count = nullptr;  // [nranks + 1] per-destination counts, then cursors
    int32_t* d_out_cursor = nullptr;
    std::vector<int64_t> out_off;     // host: start of each destination's group in the outbox
    int out_species = -1;
};


// helpers defined in pic_api.cu
pic_status pic_sim_fail(pic_sim* s, pic_status st, const char* msg);  // records; ECUDA/ETIMEOUT poison
pic_status pic_sim_check(pic_sim* s);                                 // null or poisoned handle
pic_status pic_sim_upload(pic_sim* s);                                // host mirror -> device copy
pic_status pic_sim_pull(pic_sim* s);                                  // species pointers <- device copy
pic_status pic_sim_sync(pic_sim* s);                                  // stream sync + device error word
pic_status pic_sim_dalloc(pic_sim* s, void** p, size_t bytes);        // tracked device allocation
void pic_sim_dfree(pic_sim* s, void* p);                              // frees a tracked allocation
pic_status pic_sim_ensure_ready(pic_sim* s);                          // first-step set-up, graph
pic_status pic_sim_launch_push(pic_sim* s);                           // J reset + particle kernel
