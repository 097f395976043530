// pic_particles_f64_3d.cu -- FP64 instantiation of the particle kernel, 3D shapes of order 1-3.
#define PIC_PREC 0
#define PIC_DIM 3
#include "pic_particle_kernel.cuh"

PIC_DEFINE_PARTICLE_TU(p0_d3)

size_t pic_particle_smem_bytes(int dim, int order, const int T[3], int threads, int prec) {
    int ebs[3];
    for (int a = 0; a < 3; ++a) {
        bool act = !(dim == 2 && a == 1);
        ebs[a] = act ? T[a] + (order == 1 ? 2 : order == 2 ? 3 : 4) : 1;
    }
    if (order == 2) ebs[0] += 1;  // even x extent for TMA (16-byte rows)
    // tiles (the x differences for linear FP64; the particle staging buffers
    // for the FP32 variant, prec 2) + alignment slack of the dynamic base; the
    // rings of crossing particles are in global memory
    return smem_plan(ebs, uses_xdiff(prec, order), prec == 2).bytes + 128;
}
