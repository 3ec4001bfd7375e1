// reduce_noalloc.cu -- an allocation-free variant of the FP64 reduction.
//
// lbm_check() reduces through per-tile partial sums that live in scratch
// memory the context allocated with cudaMalloc when it was created.  Some
// callers cannot allocate device memory: an application that owns every byte
// of the GPU through its own pool or fixed budget, or a monitoring hook that
// must not change the memory footprint of the job it inspects.  For them,
// lbm_reduce_noalloc() computes the same eight numbers for one domain from
// buffers the caller already holds, and keeps its partial sums in a
// file-scope device array instead.  Nothing here calls cudaMalloc, cudaFree
// or an allocating library routine.
#include <cstdio>
#include <cstring>

#include "reduce_noalloc.cuh"

namespace lbm {

// Partial sums of the allocation-free reduction: one record of RED_Q doubles
// per block of 256 nodes, plus one final record.  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[(NOALLOC_MAX_BLOCKS + 1) * RED_Q];

// One block sums nb partial records in a fixed order into out[RED_Q].
__global__ void __launch_bounds__(256) k_reduce_noalloc_final(const double *part, int nb, double *out) {
    __shared__ double sh[256];
    for (int i = 0; i < RED_Q; ++i) {
        double s = 0.0;
        for (int t = threadIdx.x; t < nb; t += blockDim.x) s += part[(int64_t)t * RED_Q + i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] = sh[0];
        __syncthreads();
    }
}

// Device address of g_noalloc_scratch on the current device (in host code
// the symbol itself is only a stand-in).  Looked up on every call: the
// lookup is cheap, and an address kept from an earlier call would be stale
// once the device's primary context has been torn down and recreated.
double *noalloc_scratch(cudaError_t &err) {
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    return err == cudaSuccess ? static_cast<double *>(p) : nullptr;
}

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_reduce_noalloc(int32_t lattice, int32_t prec, uint32_t physics, const lbm_case *cs,
                                         const void *pops, int64_t plane_stride, const uint8_t *flags,
                                         double *snap, double *out, void *stream) {
    if (!cs || !pops || !out || (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) || prec < LBM_FP64 ||
        prec > LBM_BF16S || !(physics & LBM_FLOW))
        return LBM_EINVAL;
    const int dim = lattice == LBM_D2Q9 ? 2 : 3;
    const int64_t N = (int64_t)cs->nx * cs->ny * cs->nz;
    if (cs->nx < 1 || cs->ny < 1 || cs->nz < 1 || (dim == 2 && cs->nz != 1) || plane_stride < N) return LBM_EINVAL;
    if (N > LBM_NOALLOC_MAX_NODES) {
        std::fprintf(stderr, "lbm_reduce_noalloc: %lld nodes exceed the limit of %d nodes\n", (long long)N,
                     LBM_NOALLOC_MAX_NODES);
        return LBM_EINVAL;
    }
    cudaError_t e;
    double *scratch = noalloc_scratch(e);
    if (!scratch) return LBM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((N + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
    switch ((dim == 3 ? 4 : 0) + prec) {
    case 0: e = noalloc_launch_f64(2, physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 1: e = launch_noalloc_phys<2, float>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 2: e = launch_noalloc_phys<2, __half>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 3: e = launch_noalloc_phys<2, __nv_bfloat16>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 4: e = noalloc_launch_f64(3, physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 5: e = launch_noalloc_phys<3, float>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 6: e = launch_noalloc_phys<3, __half>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    default: e = launch_noalloc_phys<3, __nv_bfloat16>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    }
    if (e != cudaSuccess) return LBM_ECUDA;
    // one block sums the partials in a fixed order into the final record
    double *final_rec = scratch + (int64_t)NOALLOC_MAX_BLOCKS * RED_Q;
    k_reduce_noalloc_final<<<1, 256, 0, s>>>(scratch, nb, final_rec);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (cudaMemcpyAsync(out, final_rec, RED_Q * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LBM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ECUDA;
    return out[5] != 0.0 ? LBM_EUNSTABLE : LBM_OK;
}
