// kernels.cuh -- the fused coupled lattice-Boltzmann step and its helpers.
//
// Storage: one structure-of-arrays plane per population, x fastest.  The two
// buffers hold the RELAXED populations, shifted by their rest value:
// s_a(x, t) = p_rel,a(x, t) - w_a phi_ref (phi_ref = rho0, C0 or B0_k of the
// case).  The shift keeps the stored numbers small so that FP32 and 16-bit
// storage resolve the deviations that carry the flow, and the arithmetic below
// works on the shifted values directly (sum_a w_a = 1, sum_a w_a e_a = 0).
// One thread per node:
//   1. pull s(x, t+1) = s_rel(x - e_a, t) for every plane (Eq. 1, 3, 5);
//   2. boundary nodes replace the populations that come from solid nodes by
//      their wall-link formulas (Sec. 3-4), evaluated from the relaxed
//      populations at A and E and the moments at t recovered from them (mass,
//      C and B are conserved by the relaxation);
//   3. moments, equilibria (Eq. 2, 4, 6 with the magnetic stress), BGK
//      relaxation with the Guo source, store s_rel(x, t+1) to the other buffer.
// Every step is one launch over a flat list of node tiles of all cases.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "lattice.cuh"
#include "types.cuh"

#define LBM_DEV __device__ __forceinline__

namespace lbm {

// ------------------------------------------------------------------ storage
template <class S> struct Codec;
template <> struct Codec<double> {
    using T = double;
    LBM_DEV static double ld(const double *p) { return __ldg(p); }
    LBM_DEV static double ld_shared(const double *p) { return *p; }
    LBM_DEV static void st(double *p, double v) { *p = v; }
};
template <> struct Codec<float> {
    using T = float;
    LBM_DEV static float ld(const float *p) { return __ldg(p); }
    LBM_DEV static float ld_shared(const float *p) { return *p; }
    LBM_DEV static void st(float *p, float v) { *p = v; }
};
template <> struct Codec<__half> {
    using T = float;
    LBM_DEV static float ld(const __half *p) { return __half2float(__ldg(p)); }
    LBM_DEV static float ld_shared(const __half *p) { return __half2float(*p); }
    LBM_DEV static void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Codec<__nv_bfloat16> {
    using T = float;
    LBM_DEV static float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    LBM_DEV static float ld_shared(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    LBM_DEV static void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

LBM_DEV uint32_t fast_div(uint32_t n, FastDiv d) { return (__umulhi(n, d.m) + n) >> d.s; }

LBM_DEV float fmaf_t(float a, float b, float c) { return fmaf(a, b, c); }
LBM_DEV double fmaf_t(double a, double b, double c) { return a * b + c; }   // FP64 serves parity: no fused rounding

template <class T>
struct StepParams {
    const void *src;
    void *dst;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    const int2 *tiles;        // (case, first node) per tile of blockDim.x nodes
    int32_t ntiles;
    const BRec *brec;
    const int32_t *brow;
    const LinkDev<T> *links;
};

// ------------------------------------------------------------------ equilibria
// Shifted equilibria e_a - w_a phi_ref, written with the deviations
// drho = rho - rho_ref, dC = C - C_ref, dB = B - B_ref so that nothing large
// cancels.
// Eq. 2 plus the magnetic stress w/(2 cs^4) [1/2|B|^2 (|e|^2 - D cs^2) - ((e.B)^2 - cs^2 |B|^2)].
// mag[k] = 4.5 (1/2 |B|^2 (k - D/3) + |B|^2/3) is the isotropic part for |e|^2 = k.
template <class F, bool HG, class T>
LBM_DEV T feq_dir(int a, T drho, T rho, const T (&u)[3], T usq15, const T (&B)[3], const T (&mag)[3]) {
    const T ex = T(F::ex(a)), ey = T(F::ey(a)), ez = T(F::ez(a));
    const T w = T(F::w(a));
    const T eu = ex * u[0] + ey * u[1] + ez * u[2];
    T feq = drho + rho * (eu * (T(3) + T(4.5) * eu) - usq15);
    if constexpr (HG) {
        const T eB = ex * B[0] + ey * B[1] + ez * B[2];
        const int ee = F::ex(a) * F::ex(a) + F::ey(a) * F::ey(a) + F::ez(a) * F::ez(a);
        feq += (ee == 0 ? mag[0] : (ee == 1 ? mag[1] : mag[2])) - T(4.5) * eB * eB;
    }
    return w * feq;
}

template <class F, class T>
LBM_DEV void mag_classes(T Bsq, T (&mag)[3]) {
    constexpr T third = T(1) / T(3);
#pragma unroll
    for (int k = 0; k < 3; ++k) mag[k] = T(4.5) * (T(0.5) * Bsq * (T(k) - T(F::DIM) * third) + Bsq * third);
}
// Eq. 4 with c_h^2 = 1/4
template <class M, class T>
LBM_DEV T heq_dir(int a, T dC, T C, const T (&u)[3]) {
    const T eu = T(M::ex(a)) * u[0] + T(M::ey(a)) * u[1] + T(M::ez(a)) * u[2];
    return T(M::w(a)) * (dC + T(4) * C * eu);
}
// Eq. 6, component k, with c_g^2 = 1/4
template <class M, class T>
LBM_DEV T geq_dir(int a, int k, T dBk, const T (&B)[3], const T (&u)[3]) {
    const T ex = T(M::ex(a)), ey = T(M::ey(a)), ez = T(M::ez(a));
    const T eu = ex * u[0] + ey * u[1] + ez * u[2];
    const T eB = ex * B[0] + ey * B[1] + ez * B[2];
    return T(M::w(a)) * (dBk + T(4) * (eu * B[k] - eB * u[k]));
}

// ------------------------------------------------------------------ collision
// In place: s (shifted populations at x, t) -> s_rel (Eq. 1, 3, 5).
template <class PL, bool HH, bool HG, class T>
LBM_DEV void collide(T (&p)[PL::P], const CaseDev<T> &c) {
    using F = typename PL::F;
    using M = typename PL::M;
    constexpr int QF = PL::QF, QM = PL::QM, NB = PL::NB, DIM = F::DIM;
    T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int a = 0; a < QF; ++a) {
        drho += p[a];
        if (F::ex(a)) jx += T(F::ex(a)) * p[a];
        if (F::ey(a)) jy += T(F::ey(a)) * p[a];
        if (F::ez(a)) jz += T(F::ez(a)) * p[a];
    }
    const T rho = drho + c.ref_rho;
    // Guo forcing: u = (sum e f + F/2) / rho with F = rho * accel
    const T Fx = rho * c.ax, Fy = rho * c.ay, Fz = DIM == 3 ? rho * c.az : T(0);
    const T inv = T(1) / rho;
    const T ux = (jx + T(0.5) * Fx) * inv;
    const T uy = (jy + T(0.5) * Fy) * inv;
    const T uz = DIM == 3 ? (jz + T(0.5) * Fz) * inv : T(0);
    const T usq15 = T(1.5) * (ux * ux + uy * uy + uz * uz);
    T B[3] = {T(0), T(0), T(0)}, dB[3] = {T(0), T(0), T(0)};
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            T s = 0;
#pragma unroll
            for (int a = 0; a < QM; ++a) s += p[PL::G0 + k * QM + a];
            dB[k] = s;
            B[k] = s + c.ref_B[k];
        }
    }
    T mag[3] = {T(0), T(0), T(0)};
    if constexpr (HG) mag_classes<F, T>(B[0] * B[0] + B[1] * B[1] + B[2] * B[2], mag);
    const T u[3] = {ux, uy, uz};
    const T uF = ux * Fx + uy * Fy + uz * Fz;
#pragma unroll
    for (int a = 0; a < QF; ++a) {
        const T ex = T(F::ex(a)), ey = T(F::ey(a)), ez = T(F::ez(a));
        const T w = T(F::w(a));
        const T feq = feq_dir<F, HG, T>(a, drho, rho, u, usq15, B, mag);
        const T eu = ex * ux + ey * uy + ez * uz;
        const T eF = ex * Fx + ey * Fy + ez * Fz;
        // Guo source (1 - 1/(2 tau)) w [3 (e - u).F + 9 (e.u)(e.F)]
        const T S = c.guo * w * (T(3) * (eF - uF) + T(9) * eu * eF);
        p[a] = fmaf_t(c.om_f, feq, fmaf_t(c.omc_f, p[a], S));
    }
    if constexpr (HH) {
        T dC = 0;
#pragma unroll
        for (int a = 0; a < QM; ++a) dC += p[PL::H0 + a];
        const T C = dC + c.ref_C;
#pragma unroll
        for (int a = 0; a < QM; ++a)
            p[PL::H0 + a] = fmaf_t(c.om_h, heq_dir<M, T>(a, dC, C, u), c.omc_h * p[PL::H0 + a]);
    }
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
#pragma unroll
            for (int a = 0; a < QM; ++a) {
                const int q = PL::G0 + k * QM + a;
                p[q] = fmaf_t(c.om_g, geq_dir<M, T>(a, k, dB[k], B, u), c.omc_g * p[q]);
            }
        }
    }
}

// ------------------------------------------------------------------ wall links
template <class S, class T>
LBM_DEV T field_sum(const S *src, int stride, int q0, int nq, int node) {
    T s = 0;
    for (int j = 0; j < nq; ++j) s += Codec<S>::ld(src + ((q0 + j) * stride + node));
    return s;
}

template <class PL, class S, class T>
LBM_DEV T eval_link(const LinkDev<T> &L, const S *src, const CaseDev<T> &c) {
    const int st = (int)c.stride;
    const T paA = Codec<S>::ld(src + ((int)L.plane_a * st + L.nodeA));
    const T papA = Codec<S>::ld(src + ((int)L.plane_ap * st + L.nodeA));
    const T papE = Codec<S>::ld(src + ((int)L.plane_ap * st + L.nodeE));
    T v = L.c0 + L.ca * paA + L.cap * papA + L.cape * papE;
    if (L.flags & LINK_NEED_PHI) {
        const int nq = L.phi_plane0 < PL::QF ? PL::QF : PL::QM;
        const T phA = field_sum<S, T>(src, st, L.phi_plane0, nq, L.nodeA) + L.ref_phi;
        const T phE = field_sum<S, T>(src, st, L.phi_plane0, nq, L.nodeE) + L.ref_phi;
        v += L.cphi * ((T(1) + L.d) * phA - L.d * phE);
    }
    if constexpr (PL::G0 < PL::P) {
        if (L.flags & LINK_NEED_B) {
#pragma unroll
            for (int k = 0; k < PL::NB; ++k) {
                const int q0 = PL::G0 + k * PL::QM;
                const T bA = field_sum<S, T>(src, st, q0, PL::QM, L.nodeA) + c.ref_B[k];
                const T bE = field_sum<S, T>(src, st, q0, PL::QM, L.nodeE) + c.ref_B[k];
                v += L.cB[k] * ((T(1) + L.d) * bA - L.d * bE);
            }
        }
    }
    return v;
}

// Applies every link of boundary node n (row r of the case) to p.
template <class PL, class S, class T>
LBM_DEV void apply_links(T (&p)[PL::P], const StepParams<T> &prm, const CaseDev<T> &c, const S *src, int n, int r) {
    int lo = prm.brow[c.brow_off + r];
    const int hi0 = prm.brow[c.brow_off + r + 1];
    int hi = hi0;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (prm.brec[mid].node < n) lo = mid + 1; else hi = mid;
    }
    if (lo < hi0 && prm.brec[lo].node == n) {
        const BRec br = prm.brec[lo];
        for (int li = br.lo; li < br.hi; ++li) {
            const LinkDev<T> L = prm.links[li];
            const T v = eval_link<PL, S, T>(L, src, c);
            // select per plane (an indexed store would move p to local memory)
            const int pa = L.plane_a;
#pragma unroll
            for (int q = 0; q < PL::P; ++q) p[q] = (q == pa) ? v : p[q];
        }
    }
}

// node coordinates of case-relative index n; r = y + ny*z is the row
template <int DIM, class T>
LBM_DEV void coords(const CaseDev<T> &c, int n, int &x, int &y, int &z, int &r) {
    r = (int)fast_div((uint32_t)n, c.div_nx);
    x = n - r * c.nx;
    if constexpr (DIM == 3) {
        z = (int)fast_div((uint32_t)r, c.div_ny);
        y = r - z * c.ny;
    } else {
        z = 0;
        y = r;
    }
}

// ------------------------------------------------------------------ fused step
template <int DIM, bool HH, bool HG, class S>
LBM_DEV void step_node(const StepParams<typename Codec<S>::T> &prm, const CaseDev<typename Codec<S>::T> &c, int n,
                       uint8_t fl) {
    using PL = Planes<DIM, HH, HG>;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    const S *src = static_cast<const S *>(prm.src) + c.pop_off;
    S *dst = static_cast<S *>(prm.dst) + c.pop_off;
    const int nx = c.nx, ny = c.ny;
    int x, y, z, r;
    coords<DIM, T>(c, n, x, y, z, r);
    // source node x - e_a with periodic wrap: index of x-1 is xi[0] (e_x = +1)
    const int xi[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
    const int yi[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
    int zi[3] = {0, 0, 0};
    if constexpr (DIM == 3) {
        const int nz = c.nz, nxy = nx * ny;
        zi[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
        zi[1] = z * nxy;
        zi[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
    }
    // in-case indices are 32-bit (the host keeps P * stride below 2^31)
    const int st32 = (int)c.stride;
    T p[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int src_node = xi[1 - PL::ex(q)] + yi[1 - PL::ey(q)] + zi[1 - PL::ez(q)];
        p[q] = Codec<S>::ld(src + (q * st32 + src_node));
    }
    if (fl & NODE_BOUNDARY) apply_links<PL, S, T>(p, prm, c, src, n, r);
    collide<PL, HH, HG, T>(p, c);
#pragma unroll
    for (int q = 0; q < P; ++q) Codec<S>::st(dst + (q * st32 + n), p[q]);
}

// Tiles of blockDim.x * npt nodes; each thread takes nodes tid, tid + blockDim.x, ...
// The next tile's record and the thread's first flag are fetched one tile ahead.
template <int DIM, bool HH, bool HG, class S>
__global__ void __launch_bounds__(256, DIM == 2 ? 4 : 2) k_step(const StepParams<typename Codec<S>::T> prm, const int npt) {
    using T = typename Codec<S>::T;
    int t = blockIdx.x;
    if (t >= prm.ntiles) return;
    int2 tile = prm.tiles[t];
    for (; t < prm.ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        const int2 next = tn < prm.ntiles ? prm.tiles[tn] : tile;
        const CaseDev<T> &c = prm.cases[tile.x];
        for (int k = 0; k < npt; ++k) {
            const int n = tile.y + (int)threadIdx.x + k * (int)blockDim.x;
            if (n >= c.N) break;
            const uint8_t fl = prm.flags[c.node_off + n];
            if (fl & NODE_FLUID) step_node<DIM, HH, HG, S>(prm, c, n, fl);
        }
        tile = next;
    }
}

// ------------------------------------------------------------------ initial state
// Equilibrium (Eq. 2, 4, 6) of the given fields, relaxed once, stored shifted
// as s_rel(x, 0).  Fields are case-relative arrays (u, B as [N][3]); null means
// the case defaults.  Solid nodes store zero.
template <class T, class FT>
struct InitParams {
    void *dst;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    int32_t case_id;
    const FT *rho, *u, *C, *B;
    T rho0, C0, B0[3];
};

template <int DIM, bool HH, bool HG, class S, class FT>
__global__ void __launch_bounds__(256) k_init(const InitParams<typename Codec<S>::T, FT> ip) {
    using PL = Planes<DIM, HH, HG>;
    using F = typename PL::F;
    using M = typename PL::M;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    const CaseDev<T> &c = ip.cases[ip.case_id];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= c.N) return;
    S *dst = static_cast<S *>(ip.dst) + c.pop_off;
    const int st32 = (int)c.stride;
    if (!(ip.flags[c.node_off + n] & NODE_FLUID)) {
#pragma unroll
        for (int q = 0; q < P; ++q) Codec<S>::st(dst + (q * st32 + n), T(0));
        return;
    }
    const T rho = ip.rho ? T(ip.rho[n]) : ip.rho0;
    T u[3] = {T(0), T(0), T(0)}, B[3] = {ip.B0[0], ip.B0[1], ip.B0[2]};
    if (ip.u) for (int k = 0; k < 3; ++k) u[k] = T(ip.u[3 * n + k]);
    if (ip.B) for (int k = 0; k < 3; ++k) B[k] = T(ip.B[3 * n + k]);
    if (DIM == 2) { u[2] = T(0); B[2] = T(0); }
    const T C = ip.C ? T(ip.C[n]) : ip.C0;
    T p[P];
    const T usq15 = T(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    T mag[3] = {T(0), T(0), T(0)};
    if constexpr (HG) mag_classes<F, T>(B[0] * B[0] + B[1] * B[1] + B[2] * B[2], mag);
    const T drho = rho - c.ref_rho;
#pragma unroll
    for (int a = 0; a < PL::QF; ++a) p[a] = feq_dir<F, HG, T>(a, drho, rho, u, usq15, B, mag);
    if constexpr (HH) {
#pragma unroll
        for (int a = 0; a < PL::QM; ++a) p[PL::H0 + a] = heq_dir<M, T>(a, C - c.ref_C, C, u);
    }
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < PL::NB; ++k)
#pragma unroll
            for (int a = 0; a < PL::QM; ++a) p[PL::G0 + k * PL::QM + a] = geq_dir<M, T>(a, k, B[k] - c.ref_B[k], B, u);
    }
    collide<PL, HH, HG, T>(p, c);
#pragma unroll
    for (int q = 0; q < P; ++q) Codec<S>::st(dst + (q * st32 + n), p[q]);
}

// ------------------------------------------------------------------ moments
// Moments at the current time from the stored relaxed populations:
// rho = sum f_rel, u = (sum e f_rel - F/2)/rho (the relaxation adds F/2 to the
// momentum), C = sum h_rel, B = sum g_rel.
template <class PL, class S, class T>
LBM_DEV void node_moments(const S *src, int64_t stride, int n, const CaseDev<T> &c,
                          T &rho, T (&u)[3], T &C, T (&B)[3], int &nonfinite) {
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
    C = 0;
    B[0] = B[1] = B[2] = T(0);
    if constexpr (PL::G0 > PL::H0) {
        T s = 0;
#pragma unroll
        for (int a = 0; a < PL::QM; ++a) {
            const T v = Codec<S>::ld(src + (int64_t)(PL::H0 + a) * stride + n);
            nonfinite += !isfinite(v);
            s += v;
        }
        C = s + c.ref_C;
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
};

template <int DIM, bool HH, bool HG, class S>
__global__ void __launch_bounds__(256) k_moments(const MomParams<typename Codec<S>::T> mp) {
    using PL = Planes<DIM, HH, HG>;
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
    T rho, u[3], C, B[3];
    int nf;
    node_moments<PL, S, T>(static_cast<const S *>(mp.src) + c.pop_off, c.stride, n, c, rho, u, C, B, nf);
    mp.rho[n] = (double)rho;
    mp.C[n] = HH ? (double)C : 0.0;
    for (int k = 0; k < 3; ++k) { mp.u[3 * n + k] = (double)u[k]; mp.B[3 * n + k] = HG ? (double)B[k] : 0.0; }
}

// ------------------------------------------------------------------ FP64 reductions
// One block per tile: partial sums (rho, C, Bx, By, Bz, non-finite count,
// |phi - phi_prev|^2, |phi|^2) in FP64, written to part[tile][8]; the previous
// phi = (u, C, B - B0) lives in snap[7][total nodes] (FP64) and is replaced.
constexpr int RED_Q = 8;
constexpr int SNAP_Q = 7;

template <class T>
struct RedParams {
    const void *src;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    const int2 *tiles;
    int32_t ntiles;
    int32_t tile_nodes;
    double *snap;
    int64_t snap_stride;
    double *part;             // [ntiles][RED_Q]
};

LBM_DEV double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int DIM, bool HH, bool HG, class S>
__global__ void __launch_bounds__(256) k_reduce(const RedParams<typename Codec<S>::T> rp) {
    using PL = Planes<DIM, HH, HG>;
    using T = typename Codec<S>::T;
    __shared__ double sh[RED_Q][32];
    const int t = blockIdx.x;
    const int2 tile = rp.tiles[t];
    const CaseDev<T> &c = rp.cases[tile.x];
    double acc[RED_Q];
#pragma unroll
    for (int i = 0; i < RED_Q; ++i) acc[i] = 0.0;
    for (int i = threadIdx.x; i < rp.tile_nodes; i += blockDim.x) {
        const int n = tile.y + i;
        if (n >= c.N || !(rp.flags[c.node_off + n] & NODE_FLUID)) continue;
        T rho, u[3], C, B[3];
        int nf;
        node_moments<PL, S, T>(static_cast<const S *>(rp.src) + c.pop_off, c.stride, n, c, rho, u, C, B, nf);
        acc[0] = rho;
        acc[1] = HH ? (double)C : 0.0;
        acc[2] = HG ? (double)B[0] : 0.0;
        acc[3] = HG ? (double)B[1] : 0.0;
        acc[4] = HG ? (double)B[2] : 0.0;
        acc[5] = nf;
        const double phi[SNAP_Q] = {(double)u[0], (double)u[1], (double)u[2],
                                    HH ? (double)C : 0.0,
                                    HG ? (double)B[0] - (double)c.B0[0] : 0.0,
                                    HG ? (double)B[1] - (double)c.B0[1] : 0.0,
                                    HG ? (double)B[2] - (double)c.B0[2] : 0.0};
        double *sp = rp.snap + c.node_off + n;
#pragma unroll
        for (int k = 0; k < SNAP_Q; ++k) {
            const double old = sp[k * rp.snap_stride];
            const double dd = phi[k] - old;
            acc[6] += dd * dd;
            acc[7] += phi[k] * phi[k];
            sp[k * rp.snap_stride] = phi[k];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < RED_Q; ++i) {
        const double v = warp_sum(acc[i]);
        if (lane == 0) sh[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < RED_Q) {
        const int nw = (blockDim.x + 31) >> 5;
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
        rp.part[(int64_t)t * RED_Q + threadIdx.x] = s;
    }
}

// One block (256 threads) per case: sums the case's tile partials in a fixed
// order (deterministic for a given tile list).
inline __global__ void __launch_bounds__(256) k_reduce_final(const double *part, const int32_t *case_tile_lo,
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
