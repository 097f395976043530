// pic_particles_f32.cu -- FP32 instantiation of the particle kernel (the FP32
// variant: FP64 storage, positions and current sums, FP32 gather, push and
// deposit weights).
#define PIC_PREC 2
#include "pic_particle_kernel.cuh"

cudaError_t pic_launch_particles_p2(int dim, int order, const LaunchCfg& cfg, size_t smem,
                                        const SchedDev* sched, SimDev* sims, cudaStream_t st) {
    PIC_DISPATCH_DO(launch_particles_t, cfg, smem, sched, sims, st);
    return cudaErrorInvalidValue;
}

cudaError_t pic_prepare_particles_p2(int dim, int order, size_t smem) {
    PIC_DISPATCH_DO(prepare_t, smem);
    return cudaErrorInvalidValue;
}

int pic_particle_occupancy_p2(int dim, int order, int minb, int threads, size_t smem) {
    PIC_DISPATCH_DO(occupancy_t, minb, threads, smem);
    return 0;
}
