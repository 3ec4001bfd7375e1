// reduce.cuh -- moments at the current time and the FP64 invariant / residual
// reductions over the stored (shifted, relaxed) populations.
//
// Moments: rho = sum f_rel, u = (sum e f_rel - F/2)/rho (the relaxation adds
// F/2 to the momentum), C = sum h_rel, B = sum g_rel (mass, C and B are
// conserved by the relaxation).
//
// Per node the reduction forms, in the arithmetic precision T of the step,
// rho, C, B, a non-finite count and the residual terms
//   r2 = |phi - phi_prev|^2,  p2 = |phi|^2,  phi = (u, C, B - B0)
// (only the components the lattice and physics can make nonzero; with
// several concentration species, which exclude the magnetic field, phi =
// (u, C_0, C_1, ..)); sums over nodes are FP64.  phi_prev is kept node by node in the snapshot buffer,
// stored in T (FP64 storage: double, otherwise float), and is replaced by phi.
#pragma once
#include "kernels.cuh"

namespace lbm {

// C[k]: species k (k < PL::NCS; the rest 0)
template <class PL, class S, class T>
LBM_DEV void node_moments(const S *src, int64_t stride, int n, const CaseDev<T> &c,
                          T &rho, T (&u)[3], T (&C)[MAX_SPECIES], T (&B)[3], int &nonfinite) {
    using F = typename PL::F;
    T drho = 0;
    T j[3] = {T(0), T(0), T(0)};
    nonfinite = 0;
#pragma unroll
    for (int a = 0; a < PL::QF; ++a) {
        const T v = Codec<S>::ld(src + (int64_t)a * stride + n);
        nonfinite += !isfinite(v);
        drho += v;
        j[0] += T(F::ex(a)) * v;
        j[1] += T(F::ey(a)) * v;
        j[2] += T(F::ez(a)) * v;
    }
    rho = drho + c.ref_rho;
    u[0] = (j[0] - T(0.5) * rho * c.ax) / rho;
    u[1] = (j[1] - T(0.5) * rho * c.ay) / rho;
    u[2] = F::DIM == 3 ? (j[2] - T(0.5) * rho * c.az) / rho : T(0);
    B[0] = B[1] = B[2] = T(0);
#pragma unroll
    for (int k = 0; k < MAX_SPECIES; ++k) {
        C[k] = T(0);
        if (k >= PL::NCS) continue;
        T s = 0;
#pragma unroll
        for (int a = 0; a < PL::QM; ++a) {
            const T v = Codec<S>::ld(src + (int64_t)(PL::H0 + k * PL::QM + a) * stride + n);
            nonfinite += !isfinite(v);
            s += v;
        }
        C[k] = s + species_ref(c, k);
    }
    if constexpr (PL::P > PL::G0) {
#pragma unroll
        for (int k = 0; k < PL::NB; ++k) {
            T s = 0;
#pragma unroll
            for (int a = 0; a < PL::QM; ++a) {
                const int q = PL::G0 + k * PL::QM + a;
                const T v = Codec<S>::ld(src + (int64_t)q * stride + n);
                nonfinite += !isfinite(v);
                s += v;
            }
            B[k] = s + c.ref_B[k];
        }
    }
}

template <class T>
struct MomParams {
    const void *src;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    int32_t case_id;
    double *rho, *u, *C, *B;  // case-relative device outputs (u, B as [N][3])
    int32_t species;          // the species C reports
};

template <int DIM, int NC, bool HG, class S>
__global__ void __launch_bounds__(256) k_moments(const MomParams<typename Codec<S>::T> mp) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    const CaseDev<T> &c = mp.cases[mp.case_id];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= c.N) return;
    if (!(mp.flags[c.node_off + n] & NODE_FLUID)) {
        mp.rho[n] = 0;
        mp.C[n] = 0;
        for (int k = 0; k < 3; ++k) { mp.u[3 * n + k] = 0; mp.B[3 * n + k] = 0; }
        return;
    }
    T rho, u[3], C[MAX_SPECIES], B[3];
    int nf;
    node_moments<PL, S, T>(static_cast<const S *>(mp.src) + c.pop_off, c.stride, n, c, rho, u, C, B, nf);
    mp.rho[n] = (double)rho;
    mp.C[n] = mp.species < NC ? (double)C[mp.species & (MAX_SPECIES - 1)] : 0.0;
    for (int k = 0; k < 3; ++k) { mp.u[3 * n + k] = (double)u[k]; mp.B[3 * n + k] = HG ? (double)B[k] : 0.0; }
}

// ------------------------------------------------------------------ FP64 reductions
// Record per case: (sum rho, sum C, sum Bx, sum By, sum Bz, non-finite count,
// sum |phi - phi_prev|^2, sum |phi|^2).
constexpr int RED_Q = 8;
constexpr int SNAP_Q = 7;

// Snapshot components that can be nonzero: u (DIM components), C_0, then
// B - B0 (DIM) or the further species C_1 .. C_{NC-1}.
template <class PL>
LBM_HD constexpr bool snap_used(int k) {
    constexpr int D = PL::F::DIM;
    constexpr int nc = PL::NCS;
    constexpr bool hg = PL::P > PL::G0;
    return k < 3 ? k < D : (k == 3 ? nc >= 1 : (hg ? k - 4 < D : k - 4 < nc - 1));
}

// The context keeps phi_prev node by node: the used components packed into
// snap_width entries (4 or 8, so that a node's entries are one or two
// 16-byte vectors in FP32).
LBM_HD constexpr int snap_width(int dim, int nc, bool hg) {
    return dim + nc + (hg ? dim : 0) <= 4 ? 4 : 8;
}
template <class PL>
LBM_HD constexpr int snap_slot(int k) {
    int s = 0;
    for (int i = 0; i < k; ++i) s += snap_used<PL>(i) ? 1 : 0;
    return s;
}

// Moments and phi = (u, C, B - B0) of node n.
template <class PL, class S, class T>
LBM_DEV void node_phi(const S *src, int64_t stride, int n, const CaseDev<T> &c, T &rho, T (&C)[MAX_SPECIES],
                      T (&B)[3], int &nf, T (&phi)[SNAP_Q]) {
    T u[3];
    node_moments<PL, S, T>(src, stride, n, c, rho, u, C, B, nf);
    phi[0] = u[0];
    phi[1] = u[1];
    phi[2] = u[2];
    phi[3] = C[0];
    if constexpr (PL::P > PL::G0) {
        phi[4] = B[0] - c.B0[0];
        phi[5] = B[1] - c.B0[1];
        phi[6] = B[2] - c.B0[2];
    } else {
        phi[4] = C[1];
        phi[5] = C[2];
        phi[6] = C[3];
    }
}

// Residual terms r2 = |phi - phi_prev|^2 and p2 = |phi|^2 over the used components.
template <class PL, class T>
LBM_DEV void resid_terms(const T (&phi)[SNAP_Q], const T (&old)[SNAP_Q], T &r2, T &p2) {
    r2 = T(0);
    p2 = T(0);
#pragma unroll
    for (int k = 0; k < SNAP_Q; ++k) {
        if (!snap_used<PL>(k)) continue;
        const T dd = phi[k] - old[k];
        r2 = fmaf_t(dd, dd, r2);
        p2 = fmaf_t(phi[k], phi[k], p2);
    }
}

// Packed snapshot entries of one node: read phi_prev, write phi (vector
// accesses; p is aligned to the node's entries).
template <class PL, class SnapT, class T>
LBM_DEV void snap_exchange(SnapT *p, const T (&phi)[SNAP_Q], T (&old)[SNAP_Q]) {
    constexpr int W = snap_width(PL::F::DIM, PL::NCS, PL::P > PL::G0);
    SnapT v[W];
    if constexpr (sizeof(SnapT) == 4) {
#pragma unroll
        for (int j = 0; j < W / 4; ++j) {
            const float4 x = reinterpret_cast<const float4 *>(p)[j];
            v[4 * j] = x.x; v[4 * j + 1] = x.y; v[4 * j + 2] = x.z; v[4 * j + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < W / 2; ++j) {
            const double2 x = reinterpret_cast<const double2 *>(p)[j];
            v[2 * j] = x.x; v[2 * j + 1] = x.y;
        }
    }
#pragma unroll
    for (int k = 0; k < SNAP_Q; ++k) {
        old[k] = snap_used<PL>(k) ? T(v[snap_slot<PL>(k)]) : T(0);
        if (snap_used<PL>(k)) v[snap_slot<PL>(k)] = SnapT(phi[k]);
    }
    if constexpr (sizeof(SnapT) == 4) {
#pragma unroll
        for (int j = 0; j < W / 4; ++j)
            reinterpret_cast<float4 *>(p)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < W / 2; ++j) reinterpret_cast<double2 *>(p)[j] = make_double2(v[2 * j], v[2 * j + 1]);
    }
}

// Accumulators of the record.  FP64 steps sum in double.  FP32 steps keep
// each running sum as an unevaluated pair hi + lo of floats (Knuth's TwoSum:
// hi + lo equals the exact sum of the added floats up to ~2^-44 relative),
// combine pairs across the warp the same way, and form doubles only for the
// per-block partial records, so that the FP64 units (1/70 of the FP32 rate on
// GB300) see a few operations per block instead of several per node.
template <class T>
struct RecAcc {
    double v[RED_Q];
    LBM_DEV void zero() {
#pragma unroll
        for (int i = 0; i < RED_Q; ++i) v[i] = 0.0;
    }
    LBM_DEV void add(int i, T x) { v[i] += (double)x; }
    LBM_DEV void warp_reduce() {
#pragma unroll
        for (int i = 0; i < RED_Q; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    }
    LBM_DEV double get(int i) const { return v[i]; }
};

LBM_DEV void two_sum(float &hi, float &lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

template <>
struct RecAcc<float> {
    float hi[RED_Q], lo[RED_Q];
    LBM_DEV void zero() {
#pragma unroll
        for (int i = 0; i < RED_Q; ++i) hi[i] = lo[i] = 0.f;
    }
    LBM_DEV void add(int i, float x) { two_sum(hi[i], lo[i], x); }
    LBM_DEV void warp_reduce() {
#pragma unroll
        for (int i = 0; i < RED_Q; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h = __shfl_down_sync(0xffffffffu, hi[i], o);
                const float l = __shfl_down_sync(0xffffffffu, lo[i], o);
                two_sum(hi[i], lo[i], h);
                lo[i] += l;
            }
    }
    LBM_DEV double get(int i) const { return (double)hi[i] + (double)lo[i]; }
};

// Adds the node terms to the record (non-finite count kept as an int).
// Slots 2-4 hold sum B_k, or, with several species (no field), sum C_1..C_3.
template <class PL, class T>
LBM_DEV void add_terms(RecAcc<T> &acc, int &nfc, T rho, const T (&C)[MAX_SPECIES], const T (&B)[3], int nf, T r2,
                       T p2) {
    constexpr int D = PL::F::DIM;
    acc.add(0, rho);
    if constexpr (PL::NCS >= 1) acc.add(1, C[0]);
    if constexpr (PL::P > PL::G0) {
        acc.add(2, B[0]);
        acc.add(3, B[1]);
        if constexpr (D == 3) acc.add(4, B[2]);
    } else {
#pragma unroll
        for (int k = 1; k < PL::NCS; ++k) acc.add(1 + k, C[k]);
    }
    nfc += nf;
    acc.add(6, r2);
    acc.add(7, p2);
}

// Block-wide sum of the record into out[RED_Q] (blockDim.x a multiple of 32,
// at most 1024; sh holds RED_Q x 32 doubles); the warps' records are summed
// in FP64 in a fixed order.
template <class T>
LBM_DEV void block_record(RecAcc<T> &acc, int nfc, double (*sh)[32], double *out) {
    acc.warp_reduce();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nfc += __shfl_down_sync(0xffffffffu, nfc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < RED_Q; ++i) sh[i][warp] = i == 5 ? (double)nfc : acc.get(i);
    }
    __syncthreads();
    if (threadIdx.x < RED_Q) {
        const int nw = (blockDim.x + 31) >> 5;
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
}

template <class T>
struct RedParams {
    const void *src;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    const int2 *tiles;
    int32_t ntiles;
    int32_t tile_nodes;
    void *snap;               // snap_width entries per node, double (FP64 storage) or float
    double *part;             // [ntiles][RED_Q]
};

template <class T>
using SnapOf = typename std::conditional<std::is_same<T, double>::value, double, float>::type;

// One block per tile: partial record of the tile's fluid nodes.
template <int DIM, int NC, bool HG, class S>
__global__ void __launch_bounds__(256) k_reduce(const RedParams<typename Codec<S>::T> rp) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    using SnapT = SnapOf<T>;
    __shared__ double sh[RED_Q][32];
    const int t = blockIdx.x;
    const int2 tile = rp.tiles[t];
    const CaseDev<T> &c = rp.cases[tile.x];
    RecAcc<T> acc;
    acc.zero();
    int nfc = 0;
    for (int i = threadIdx.x; i < rp.tile_nodes; i += blockDim.x) {
        const int n = tile.y + i;
        if (n >= c.N || !(rp.flags[c.node_off + n] & NODE_FLUID)) continue;
        T rho, C[MAX_SPECIES], B[3], r2, p2, phi[SNAP_Q], old[SNAP_Q];
        int nf;
        node_phi<PL, S, T>(static_cast<const S *>(rp.src) + c.pop_off, c.stride, n, c, rho, C, B, nf, phi);
        constexpr int W = snap_width(DIM, NC, HG);
        snap_exchange<PL, SnapT, T>(static_cast<SnapT *>(rp.snap) + (c.node_off + n) * W, phi, old);
        resid_terms<PL, T>(phi, old, r2, p2);
        add_terms<PL, T>(acc, nfc, rho, C, B, nf, r2, p2);
    }
    block_record(acc, nfc, sh, rp.part + (int64_t)t * RED_Q);
}

// One block (256 threads) per case: sums the case's tile partials in a fixed
// order (deterministic for a given tile list).
static __global__ void __launch_bounds__(256) k_reduce_final(const double *part, const int32_t *case_tile_lo,
                                                             double *out) {
    __shared__ double sh[256];
    const int c = blockIdx.x;
    const int lo = case_tile_lo[c], hi = case_tile_lo[c + 1];
    for (int i = 0; i < RED_Q; ++i) {
        double s = 0.0;
        for (int t = lo + (int)threadIdx.x; t < hi; t += blockDim.x) s += part[(int64_t)t * RED_Q + i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c * RED_Q + i] = sh[0];
        __syncthreads();
    }
}

}  // namespace lbm
