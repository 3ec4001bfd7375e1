// dispatch.cuh -- type-erased launchers of one (lattice, physics, precision)
// variant of the kernels, so that the C ABI picks a variant at run time.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "kernels_bulk.cuh"
#include "kernels_ring.cuh"
#include "reduce.cuh"

namespace lbm {

// register budgets of k_step (resident 256-thread blocks per SM)
constexpr int kstep_minb(int dim, int i) { return dim == 2 ? 4 + i : 2 + i; }
// nodes per consumer lane of k_step_ring: packed pairs in 2D, one node in 3D
constexpr int kring_npl(int dim) { return dim == 2 ? 2 : 1; }
constexpr int KRING_MINB = 2;

struct KernelSet {
    cudaError_t (*step[3])(const void *params, int npt, int grid, int block, cudaStream_t s);
    cudaError_t (*boundary)(const void *params, int grid, int block, cudaStream_t s);
    cudaError_t (*links)(const void *params, int grid, int block, cudaStream_t s);   // null: links inline
    // unwrapped-pull variants (launch variant 2), budgets kstep_minb(dim, 0..2)
    cudaError_t (*unw[3])(const void *params, int npt, int grid, int block, cudaStream_t s);
    cudaError_t (*init_d)(const void *params, int grid, int block, cudaStream_t s);   // FP64 host-side fields
    cudaError_t (*init_f)(const void *params, int grid, int block, cudaStream_t s);   // FP32 device fields
    cudaError_t (*moments)(const void *params, int grid, int block, cudaStream_t s);
    cudaError_t (*reduce)(const void *params, int grid, int block, cudaStream_t s);
    // bulk-copy variants, one per configuration of BULK_TT / BULK_MB / BULK_NS (null for FP64)
    cudaError_t (*step_bulk[BULK_NCFG])(const void *params, const BulkParams &bp, int grid, size_t smem,
                                        cudaStream_t s);
    const void *step_fn[3];       // kernel symbols (occupancy queries, attributes)
    const void *step_bulk_fn[BULK_NCFG];
    // shared-memory ring variant (null for FP64), ns stages
    cudaError_t (*ring)(const void *params, const BulkParams &bp, int ns, int grid, size_t smem, cudaStream_t s);
    const void *ring_fn;
};

template <int DIM, int NC, bool HG, class S>
struct Launch {
    using T = typename Codec<S>::T;
    template <int MINB>
    static cudaError_t step(const void *p, int npt, int g, int b, cudaStream_t s) {
        k_step<DIM, NC, HG, S, MINB><<<g, b, 0, s>>>(*static_cast<const StepParams<T> *>(p), npt);
        return cudaGetLastError();
    }
    template <int MINB>
    static cudaError_t unw(const void *p, int npt, int g, int b, cudaStream_t s) {
        k_step_unwrapped<DIM, NC, HG, S, MINB><<<g, b, 0, s>>>(*static_cast<const StepParams<T> *>(p), npt);
        return cudaGetLastError();
    }
    static cudaError_t boundary(const void *p, int g, int b, cudaStream_t s) {
        k_boundary<DIM, NC, HG, S><<<g, b, 0, s>>>(*static_cast<const StepParams<T> *>(p));
        return cudaGetLastError();
    }
    static cudaError_t links(const void *p, int g, int b, cudaStream_t s) {
        if constexpr (links_apart<DIM>())
            k_links<DIM, NC, HG, S><<<g, b, 0, s>>>(*static_cast<const StepParams<T> *>(p));
        return cudaGetLastError();
    }
    static cudaError_t init_d(const void *p, int g, int b, cudaStream_t s) {
        k_init<DIM, NC, HG, S, double><<<g, b, 0, s>>>(*static_cast<const InitParams<T, double> *>(p));
        return cudaGetLastError();
    }
    static cudaError_t init_f(const void *p, int g, int b, cudaStream_t s) {
        k_init<DIM, NC, HG, S, float><<<g, b, 0, s>>>(*static_cast<const InitParams<T, float> *>(p));
        return cudaGetLastError();
    }
    static cudaError_t moments(const void *p, int g, int b, cudaStream_t s) {
        k_moments<DIM, NC, HG, S><<<g, b, 0, s>>>(*static_cast<const MomParams<T> *>(p));
        return cudaGetLastError();
    }
    static cudaError_t reduce(const void *p, int g, int b, cudaStream_t s) {
        k_reduce<DIM, NC, HG, S><<<g, b, 0, s>>>(*static_cast<const RedParams<T> *>(p));
        return cudaGetLastError();
    }
    template <int I>
    static cudaError_t step_bulk(const void *p, const BulkParams &bp, int g, size_t smem, cudaStream_t s) {
        k_step_bulk<DIM, NC, HG, S, BULK_MB[I], BULK_TT[I], BULK_NS[I]><<<g, BULK_THREADS, smem, s>>>(
            *static_cast<const StepParams<T> *>(p), bp);
        return cudaGetLastError();
    }
    template <int I>
    static void set_bulk(KernelSet &k) {
        if constexpr (std::is_same<S, double>::value) {
            k.step_bulk[I] = nullptr;
            k.step_bulk_fn[I] = nullptr;
        } else {
            k.step_bulk[I] = &step_bulk<I>;
            k.step_bulk_fn[I] = reinterpret_cast<const void *>(
                &k_step_bulk<DIM, NC, HG, S, BULK_MB[I], BULK_TT[I], BULK_NS[I]>);
        }
    }
    static cudaError_t ring(const void *p, const BulkParams &bp, int ns, int g, size_t smem, cudaStream_t s) {
        if constexpr (std::is_same<S, double>::value) {
            return cudaErrorInvalidValue;
        } else {
            k_step_ring<DIM, NC, HG, S, kring_npl(DIM), KRING_MINB><<<g, RING_THREADS, smem, s>>>(
                *static_cast<const StepParams<T> *>(p), bp, ns);
            return cudaGetLastError();
        }
    }
    static void set_ring(KernelSet &k) {
        if constexpr (std::is_same<S, double>::value) {
            k.ring = nullptr;
            k.ring_fn = nullptr;
        } else {
            k.ring = &ring;
            k.ring_fn = reinterpret_cast<const void *>(&k_step_ring<DIM, NC, HG, S, kring_npl(DIM), KRING_MINB>);
        }
    }
    static KernelSet make() {
        KernelSet k{};
        // the bulk-copy and ring variants serve one concentration species at most,
        // and storage that rounds to nearest (not the stochastic 16-bit rounding)
        if constexpr (NC <= 1 && !Rounding<S>::SR) {
            set_ring(k);
            set_bulk<0>(k);
            set_bulk<1>(k);
            set_bulk<2>(k);
            set_bulk<3>(k);
            set_bulk<4>(k);
            static_assert(BULK_NCFG == 5, "one set_bulk per configuration");
        }
        k.step[0] = &step<kstep_minb(DIM, 0)>;
        k.step[1] = &step<kstep_minb(DIM, 1)>;
        k.step[2] = &step<kstep_minb(DIM, 2)>;
        k.boundary = &boundary;
        k.links = links_apart<DIM>() ? &links : nullptr;
        k.unw[0] = &unw<kstep_minb(DIM, 0)>;
        k.unw[1] = &unw<kstep_minb(DIM, 1)>;
        k.unw[2] = &unw<kstep_minb(DIM, 2)>;
        k.init_d = &init_d;
        k.init_f = &init_f;
        k.moments = &moments;
        k.reduce = &reduce;
        k.step_fn[0] = reinterpret_cast<const void *>(&k_step<DIM, NC, HG, S, kstep_minb(DIM, 0)>);
        k.step_fn[1] = reinterpret_cast<const void *>(&k_step<DIM, NC, HG, S, kstep_minb(DIM, 1)>);
        k.step_fn[2] = reinterpret_cast<const void *>(&k_step<DIM, NC, HG, S, kstep_minb(DIM, 2)>);
        return k;
    }
};

// prec: 0 FP64, 1 FP32, 2 FP16S, 3 BF16S
KernelSet kernels_2d_f64(bool hh, bool hg);
KernelSet kernels_2d_f32(bool hh, bool hg);
KernelSet kernels_2d_f16(bool hh, bool hg);
KernelSet kernels_2d_bf16(bool hh, bool hg);
KernelSet kernels_3d_f64(bool hh, bool hg);
KernelSet kernels_3d_f32(bool hh, bool hg);
KernelSet kernels_3d_f16(bool hh, bool hg);
KernelSet kernels_3d_bf16(bool hh, bool hg);
// several concentration species (nc = 2 or 3; no magnetic field)
constexpr int MAX_COMPILED_SPECIES = 3;
KernelSet species_2d_f64(int nc);
KernelSet species_2d_f32(int nc);
KernelSet species_2d_f16(int nc);
KernelSet species_2d_bf16(int nc);
KernelSet species_3d_f64(int nc);
KernelSet species_3d_f32(int nc);
KernelSet species_3d_f16(int nc);
KernelSet species_3d_bf16(int nc);

}  // namespace lbm

#define LBM_DEFINE_SPECIES_SET(NAME, DIM, S)                              \
    namespace lbm {                                                       \
    KernelSet NAME(int nc) {                                              \
        if (nc == 3) return Launch<DIM, 3, false, S>::make();             \
        return Launch<DIM, 2, false, S>::make();                          \
    }                                                                     \
    }

#define LBM_DEFINE_KERNEL_SET(NAME, DIM, S)                               \
    namespace lbm {                                                       \
    KernelSet NAME(bool hh, bool hg) {                                    \
        if (hh && hg) return Launch<DIM, true, true, S>::make();          \
        if (hh) return Launch<DIM, true, false, S>::make();               \
        if (hg) return Launch<DIM, false, true, S>::make();               \
        return Launch<DIM, false, false, S>::make();                      \
    }                                                                     \
    }
