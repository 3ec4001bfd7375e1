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
#include <mutex>

#include "reduce.cuh"
#include "lbm.h"

namespace lbm {

// Partial sums of the allocation-free reduction: one record of RED_Q doubles
// per block of 256 nodes, plus one final record.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int NOALLOC_BLOCK = 256;
constexpr int NOALLOC_MAX_BLOCKS = LBM_NOALLOC_MAX_NODES / NOALLOC_BLOCK;
static __device__ __align__(256) double g_noalloc_scratch[(NOALLOC_MAX_BLOCKS + 1) * RED_Q];

// Same per-node work as k_reduce, over a plain node range of one domain whose
// descriptor arrives by value; partials go to scratch[block][RED_Q].
template <int DIM, bool HH, bool HG, class S>
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_reduce_noalloc(const CaseDev<typename Codec<S>::T> c,
                                                                 const void *pops, const uint8_t *flags,
                                                                 double *snap, double *scratch) {
    using PL = Planes<DIM, HH, HG>;
    using T = typename Codec<S>::T;
    __shared__ double sh[RED_Q][32];
    const int n = blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    RecAcc<T> acc;
    acc.zero();
    int nfc = 0;
    if (n < c.N && (!flags || flags[n])) {
        T rho, C, B[3], r2, p2, phi[SNAP_Q], old[SNAP_Q];
        int nf;
        node_phi<PL, S, T>(static_cast<const S *>(pops), c.stride, n, c, rho, C, B, nf, phi);
        // the caller's snapshot: SNAP_Q planes of N doubles
#pragma unroll
        for (int k = 0; k < SNAP_Q; ++k) {
            old[k] = (snap && snap_used<PL>(k)) ? T(snap[(int64_t)k * c.N + n]) : T(0);
            if (snap && snap_used<PL>(k)) snap[(int64_t)k * c.N + n] = (double)phi[k];
        }
        resid_terms<PL, T>(phi, old, r2, p2);
        add_terms<PL, T>(acc, nfc, rho, C, B, nf, r2, p2);
    }
    block_record(acc, nfc, sh, scratch + (int64_t)blockIdx.x * RED_Q);
}

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

template <int DIM, bool HH, bool HG, class S>
cudaError_t launch_noalloc(const lbm_case &k, int64_t plane_stride, const void *pops, const uint8_t *flags,
                           double *snap, double *scratch, int nblocks, cudaStream_t s) {
    using T = typename Codec<S>::T;
    CaseDev<T> c{};
    c.nx = k.nx;
    c.ny = k.ny;
    c.nz = k.nz;
    c.N = k.nx * k.ny * k.nz;
    c.stride = plane_stride;
    c.ax = T(k.accel[0]);
    c.ay = T(k.accel[1]);
    c.az = DIM == 3 ? T(k.accel[2]) : T(0);
    c.ref_rho = T(k.rho0);
    c.ref_C = HH ? T(k.C0) : T(0);
    for (int j = 0; j < 3; ++j) {
        c.ref_B[j] = (HG && j < DIM) ? T(k.B0[j]) : T(0);
        c.B0[j] = j < DIM ? T(k.B0[j]) : T(0);
    }
    k_reduce_noalloc<DIM, HH, HG, S><<<nblocks, NOALLOC_BLOCK, 0, s>>>(c, pops, flags, snap, scratch);
    return cudaGetLastError();
}

template <int DIM, class S>
cudaError_t launch_noalloc_phys(uint32_t physics, const lbm_case &k, int64_t ps, const void *pops,
                                const uint8_t *flags, double *snap, double *scratch, int nb, cudaStream_t s) {
    const bool hh = physics & LBM_CD, hg = physics & LBM_MHD;
    if (hh && hg) return launch_noalloc<DIM, true, true, S>(k, ps, pops, flags, snap, scratch, nb, s);
    if (hh) return launch_noalloc<DIM, true, false, S>(k, ps, pops, flags, snap, scratch, nb, s);
    if (hg) return launch_noalloc<DIM, false, true, S>(k, ps, pops, flags, snap, scratch, nb, s);
    return launch_noalloc<DIM, false, false, S>(k, ps, pops, flags, snap, scratch, nb, s);
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (in host code the symbol itself is only a stand-in).
double *noalloc_scratch(int device, cudaError_t &err) {
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    err = cudaSuccess;
    if (device < 0 || device >= 64) { err = cudaErrorInvalidDevice; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) return nullptr;
        addr[device] = static_cast<double *>(p);
    }
    return addr[device];
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
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return LBM_ECUDA;
    cudaError_t e;
    double *scratch = noalloc_scratch(device, e);
    if (!scratch) return LBM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((N + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
    switch ((dim == 3 ? 4 : 0) + prec) {
    case 0: e = launch_noalloc_phys<2, double>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 1: e = launch_noalloc_phys<2, float>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 2: e = launch_noalloc_phys<2, __half>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 3: e = launch_noalloc_phys<2, __nv_bfloat16>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
    case 4: e = launch_noalloc_phys<3, double>(physics, *cs, plane_stride, pops, flags, snap, scratch, nb, s); break;
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
