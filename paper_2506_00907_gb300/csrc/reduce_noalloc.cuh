// reduce_noalloc.cuh -- kernels of the allocation-free reduction (see
// reduce_noalloc.cu).  Instantiated in reduce_noalloc.cu (FP32 and 16-bit
// storage) and reduce_noalloc_f64.cu (FP64 storage, built like the other FP64
// units without multiply-add contraction, as the context's reduction is).
#pragma once
#include "lbm.h"
#include "reduce.cuh"

namespace lbm {

constexpr int NOALLOC_BLOCK = 256;
constexpr int NOALLOC_MAX_BLOCKS = LBM_NOALLOC_MAX_NODES / NOALLOC_BLOCK;

// Same per-node work as k_reduce, over a plain node range of one domain whose
// descriptor arrives by value; partials go to scratch[block][RED_Q].
template <int DIM, int NC, bool HG, class S>
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_reduce_noalloc(const CaseDev<typename Codec<S>::T> c,
                                                                 const void *pops, const uint8_t *flags,
                                                                 double *snap, double *scratch) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    __shared__ double sh[RED_Q][32];
    const int n = blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    RecAcc<T> acc;
    acc.zero();
    int nfc = 0;
    if (n < c.N && (!flags || flags[n])) {
        T rho, C[MAX_SPECIES], B[3], r2, p2, phi[SNAP_Q], old[SNAP_Q];
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

template <int DIM, int NC, bool HG, class S>
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
    c.ref_C = NC ? T(k.C0) : T(0);
    for (int j = 0; j < 3; ++j) {
        c.ref_B[j] = (HG && j < DIM) ? T(k.B0[j]) : T(0);
        c.B0[j] = j < DIM ? T(k.B0[j]) : T(0);
    }
    k_reduce_noalloc<DIM, NC, HG, S><<<nblocks, NOALLOC_BLOCK, 0, s>>>(c, pops, flags, snap, scratch);
    return cudaGetLastError();
}

template <int DIM, class S>
inline cudaError_t launch_noalloc_phys(uint32_t physics, const lbm_case &k, int64_t ps, const void *pops,
                                const uint8_t *flags, double *snap, double *scratch, int nb, cudaStream_t s) {
    const bool hh = physics & LBM_CD, hg = physics & LBM_MHD;
    if (hh && hg) return launch_noalloc<DIM, true, true, S>(k, ps, pops, flags, snap, scratch, nb, s);
    if (hh) return launch_noalloc<DIM, true, false, S>(k, ps, pops, flags, snap, scratch, nb, s);
    if (hg) return launch_noalloc<DIM, false, true, S>(k, ps, pops, flags, snap, scratch, nb, s);
    return launch_noalloc<DIM, false, false, S>(k, ps, pops, flags, snap, scratch, nb, s);
}

// FP64 storage (reduce_noalloc_f64.cu)
cudaError_t noalloc_launch_f64(int dim, uint32_t physics, const lbm_case &k, int64_t ps, const void *pops,
                               const uint8_t *flags, double *snap, double *scratch, int nb, cudaStream_t s);

}  // namespace lbm
