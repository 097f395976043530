// pic_bin.h -- box binning of caller-owned particles (shared by pic_bin.cu and
// its allocation-free variant).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/pic_api.h"

struct BinGeom {
    int dim;
    int n[3], bsz[3], nb[3];
    double d[3];
    int nboxes;
};

pic_status pic_bin_validate(const pic_grid_desc* grid, const double* x, const double* y,
                            const double* z, int64_t np, const int64_t* box_off_out,
                            const int64_t* perm_out, BinGeom* g, std::string* err);
// box_off: nboxes+1 int64 (output, also the histogram); cursor: nboxes int32 scratch
cudaError_t pic_bin_launch(const BinGeom& g, const double* x, const double* y, const double* z,
                           int64_t np, int64_t* box_off, int64_t* perm, int32_t* cursor,
                           cudaStream_t st);
// streaming multiprocessors of the current device (defined in pic_particles.cu)
int pic_sm_count();
// records the message returned by pic_last_error(NULL) on this thread
pic_status pic_record_error(pic_status st, const char* msg);
