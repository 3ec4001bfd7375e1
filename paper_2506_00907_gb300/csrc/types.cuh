// types.cuh -- device-side records shared by the host driver and the kernels.
#pragma once
#include <cstdint>

namespace lbm {

// Division by a run-time constant d (1 <= d, n < 2^31) with a multiply-high
// (Granlund & Montgomery 1994, round-up magic): q = (umulhi(n, m) + n) >> s.
struct FastDiv {
    uint32_t m, s;
};

// Per-case descriptor, one per domain, read warp-uniformly by every tile.
template <class T>
struct CaseDev {
    int32_t nx, ny, nz, N;
    FastDiv div_nx, div_ny;
    int64_t pop_off;      // element offset of the case's first plane in a population buffer
    int64_t stride;       // elements between consecutive planes of the case
    int64_t node_off;     // offset of the case's nodes in the flag / snapshot arrays
    int32_t index;        // the case's position in the case table
    int32_t pad1;
    T om_f, om_h, om_g;   // 1/tau_nu, 1/tau_D, 1/tau_eta
    T omc_f, omc_h, omc_g; // 1 - om (the relaxation p + om (eq - p) = (1 - om) p + om eq)
    T guo;                // 1 - 1/(2 tau_nu): weight of the Guo source
    T ax, ay, az;         // body force per unit mass
    T ref_rho, ref_C;     // storage references: planes hold p - w_a * phi_ref
    T ref_B[3];
    T B0[3];              // B_ext for the residual (phi uses B - B0)
    T sp_om[3], sp_omc[3], sp_ref[3];   // concentration species 1..3: 1/tau_D, 1 - 1/tau_D, C_ref
};

// Relaxation parameters and storage reference of concentration species k
// (species 0 keeps om_h, omc_h, ref_C).
template <class T>
__host__ __device__ __forceinline__ T species_om(const CaseDev<T> &c, int k) { return k == 0 ? c.om_h : c.sp_om[k - 1]; }
template <class T>
__host__ __device__ __forceinline__ T species_omc(const CaseDev<T> &c, int k) { return k == 0 ? c.omc_h : c.sp_omc[k - 1]; }
template <class T>
__host__ __device__ __forceinline__ T species_ref(const CaseDev<T> &c, int k) { return k == 0 ? c.ref_C : c.sp_ref[k - 1]; }

// Surface reaction network of a case (several species, Sec. 4.2.2): reaction
// j runs at rate[j] prod_m C_m^order_jm per unit wall area and time
// (order_jm = byte m of ord[j], 0..2) and produces species i at st[j][i]
// times that rate.
constexpr int MAX_SPECIES = 4;
constexpr int MAX_REACT = 4;
template <class T>
struct ReactDev {
    int32_t n;
    uint32_t ord[MAX_REACT];
    T rate[MAX_REACT];
    T st[MAX_REACT][MAX_SPECIES];
};

// Per-link record with the wall formula of the link folded into coefficients
// (the host derives them from the link kind, d and the wall data), acting on
// the stored (shifted) populations s = p - w phi_ref:
//   s_a(A, t+1) = c0 + ca s_a(A) + cap s_a'(A) + cape s_a'(E)
//               + cphi phi_X + sum_j cB[j] B_X,j
// with the relaxed populations at t, phi_X = -d phi(E) + (1 + d) phi(A)
// (Eq. 13) of the link's own field (rho for f, C for h, B_k for g_k), and
// B_X the extrapolated magnetic field vector (moving flux walls of g, Eq. 24).
// Given-pressure links (open boundaries, Eq. 42/44) add cphi * (4.5 (e.u_X)^2 -
// 1.5 |u_X|^2) with u_X = -d u(E) + (1 + d) u(A) (Eq. 13) and e = cB (LINK_NEED_U).
// Velocity links of an oscillating wall (LINK_WALL_T) keep their steady cphi in
// cB[0]; a clock kernel writes cphi = cB[0] cos(omega t + phase) before each step.
// Reaction links of species i (LINK_NEED_REACT, kernels with several species
// only) add cB[0] R_i(C_X) with R_i the case's network rate at every species'
// C_X = (1 + d) C(A) - d C(E) (Eq. 13).
enum : uint8_t { LINK_NEED_PHI = 1, LINK_NEED_B = 2, LINK_NEED_U = 4, LINK_WALL_T = 8, LINK_NEED_REACT = 16 };

template <class T>
struct alignas(16) LinkDev {
    int32_t nodeA;        // case-relative node indices
    int32_t nodeE;        // = nodeA when E is solid (then d = 1/2)
    uint8_t plane_a;      // plane of the unknown direction a
    uint8_t plane_ap;     // plane of the opposite direction a'
    uint8_t phi_plane0;   // first plane of the link's field
    uint8_t flags;        // LINK_NEED_PHI | LINK_NEED_B | LINK_NEED_U | LINK_WALL_T
    int32_t cs;           // case index
    T d, c0, ca, cap, cape, cphi;
    T cB[3];
    T ref_phi;            // storage reference of the link's field (phi = sum of stored + ref_phi)
};

// The value a link gives its unknown population in the coming step, and the
// plane it replaces (written by the link kernel, read by the boundary kernel).
template <class T>
struct LinkOut {
    T v;
    int32_t plane;
};

// Boundary record of a fluid node that owns links.
// One boundary node (a fluid node with at least one wall link): the boundary
// kernel takes one record per thread.
struct BRec {
    int32_t node;         // case-relative node index
    int32_t lo, hi;       // link range [lo, hi) in the global link array
    int32_t cs;           // case index
};

enum : uint8_t { NODE_FLUID = 1, NODE_BOUNDARY = 2 };

}  // namespace lbm
