// pic_bin_noalloc.cu -- pic_bin_particles_noalloc: the box binning of
// pic_bin_particles without any device allocation.
//
// Who needs it: callers that cannot let a library call cudaMalloc -- code that
// enqueues work while a CUDA stream capture is open (an allocation there
// breaks or escapes the capture), frameworks that own every byte of device
// memory through their own pool and forbid foreign allocations, and
// latency-critical loops that must not hit the allocator.  They pass their own
// input and output buffers; the only scratch the binning needs, one cursor per
// box, lives in a fixed file-scope device array instead.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/pic_noalloc.h"
#include "pic_bin.h"

// Per-box cursors of the counting sort.  Every GPU that loads libpic holds
// this array (4 MiB) until the process exits; every call shares it.
static __device__ __align__(256) int32_t g_bin_cursor_scratch[PIC_BIN_NOALLOC_MAX_BOXES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};            // device address of the array, per device
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // id of the context it was looked up in
thread_local std::string g_err;

// Id of the current context (0 when the driver cannot tell): a device reset
// destroys the primary context and the module with the array, so an address
// looked up in an earlier context must not be reused.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrentFn)(CUcontext*);
    typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrentFn)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetIdFn)p;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// The array's name is a host-side stand-in in host code, not a device
// address: look the address up once per device and context, with that device
// current.
pic_status scratch_for_current_device(int32_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        g_err = "no usable current CUDA device";
        return PIC_ECUDA;
    }
    // (before the first runtime call that creates the context the id reads 0;
    // the next call then finds a new id and looks the address up once more)
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] && ctx != g_scratch_ctx[dev]) g_scratch_ptr[dev] = nullptr;
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_cursor_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            g_err = std::string("cudaGetSymbolAddress of the binning scratch failed: ") +
                    cudaGetErrorString(e);
            return PIC_ECUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<int32_t*>(g_scratch_ptr[dev]);
    return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_bin_particles_noalloc(const pic_grid_desc* grid, const double* x,
                                                const double* y, const double* z, int64_t np,
                                                int64_t* box_off_out, int64_t* perm_out) {
    BinGeom g;
    pic_status st = pic_bin_validate(grid, x, y, z, np, box_off_out, perm_out, &g, &g_err);
    if (st != PIC_OK) return pic_record_error(st, g_err.c_str());
    if (g.nboxes > PIC_BIN_NOALLOC_MAX_BOXES) {
        g_err = "pic_bin_particles_noalloc: " + std::to_string(g.nboxes) +
                " boxes exceed the fixed scratch of " + std::to_string(PIC_BIN_NOALLOC_MAX_BOXES) +
                " boxes; use pic_bin_particles";
        return pic_record_error(PIC_EINVAL, g_err.c_str());
    }
    int32_t* cursor = nullptr;
    st = scratch_for_current_device(&cursor);
    if (st != PIC_OK) return pic_record_error(st, g_err.c_str());
    // the cursors keep the previous call's values: pic_bin_launch zeroes the
    // first nboxes of them (and the output offsets) on the stream first
    cudaError_t e = pic_bin_launch(g, x, y, z, np, box_off_out, perm_out, cursor,
                                   (cudaStream_t)grid->stream);
    if (e != cudaSuccess) {
        g_err = std::string("pic_bin_particles_noalloc failed: ") + cudaGetErrorString(e);
        return pic_record_error(PIC_ECUDA, g_err.c_str());
    }
    return PIC_OK;
}
