// pic_particles_dd_3d.cu -- float-float instantiation of the particle kernel (the mixed-precision variant), 3D shapes of order 1-3.
#define PIC_PREC 1
#define PIC_DIM 3
#include "pic_particle_kernel.cuh"

PIC_DEFINE_PARTICLE_TU(p1_d3)
