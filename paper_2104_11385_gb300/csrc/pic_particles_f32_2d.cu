// pic_particles_f32_2d.cu -- FP32 instantiation of the particle kernel (the FP32 variant: FP64 storage and positions, FP32 gather, push and deposit weights, FP64 current sums), 2D shapes of order 1-3.
#define PIC_PREC 2
#define PIC_DIM 2
#include "pic_particle_kernel.cuh"

PIC_DEFINE_PARTICLE_TU(p2_d2)
