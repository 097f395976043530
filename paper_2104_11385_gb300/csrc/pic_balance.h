// pic_balance.h -- host-side load balancing (arXiv 2104.11385 Sec. 2.2 and Sec. 4).
#pragma once
#include <stdint.h>

#include <vector>

namespace pic {

// Eq. 1: E = c_avg / c_max over workers (1 when every worker is idle)
double lb_efficiency(const double* costs, const int32_t* assign, int64_t nboxes, int n_workers);
// knapsack policy: greedy LPT with a cap of max(ceil(n/w), floor(cap_factor n/w)) boxes per worker
void knapsack(const double* costs, int64_t nboxes, int n_workers, double cap_factor,
              int32_t* assign);
// Morton Z-order key (3D: x,y,z bits interleaved from bit 0; 2D: x,z)
uint64_t morton_key(int dim, int64_t bx, int64_t by, int64_t bz);
// space-filling-curve policy: contiguous cost-balanced pieces of the Morton order
void sfc(const double* costs, const int32_t* ijk, int64_t nboxes, int dim, int n_workers,
         int32_t* assign);
// improvement threshold: adopt when E_new >= (1 + theta) E_old
bool adopt(double e_old, double e_new, double theta);
// Sec. 4, Eq. 2: S = (1/E0)^x
double predicted_speedup(double e0, double x);

struct Unit {
    int32_t box, chunk, nchunks;
    double cost;
};
std::vector<Unit> make_units(const double* costs, const int64_t* np, int64_t nboxes, int n_workers,
                             int split, int64_t min_particles, bool allow_split);

}  // namespace pic
