// pic_particles_f64_2d.cu -- FP64 instantiation of the particle kernel, 2D shapes of order 1-3.
#define PIC_PREC 0
#define PIC_DIM 2
#include "pic_particle_kernel.cuh"

PIC_DEFINE_PARTICLE_TU(p0_d2)
