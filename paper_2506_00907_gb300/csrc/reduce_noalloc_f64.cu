// FP64 instantiations of the allocation-free reduction, in a unit of their
// own so that they are built without multiply-add contraction like the
// context's FP64 reduction (every *_f64.cu unit is).
#include "reduce_noalloc.cuh"

namespace lbm {

cudaError_t noalloc_launch_f64(int dim, uint32_t physics, const lbm_case &k, int64_t ps, const void *pops,
                               const uint8_t *flags, double *snap, double *scratch, int nb, cudaStream_t s) {
    if (dim == 2) return launch_noalloc_phys<2, double>(physics, k, ps, pops, flags, snap, scratch, nb, s);
    return launch_noalloc_phys<3, double>(physics, k, ps, pops, flags, snap, scratch, nb, s);
}

}  // namespace lbm
