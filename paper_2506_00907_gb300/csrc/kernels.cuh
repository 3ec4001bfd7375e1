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
    LBM_DEV static double ld_raw(const double *p) { return __ldg(p); }
    LBM_DEV static double ld_shared(const double *p) { return *p; }
    LBM_DEV static void st(double *p, double v) { *p = v; }
};
template <> struct Codec<float> {
    using T = float;
    LBM_DEV static float ld(const float *p) { return __ldg(p); }
    LBM_DEV static float ld_raw(const float *p) { return __ldg(p); }
    LBM_DEV static float ld_shared(const float *p) { return *p; }
    LBM_DEV static void st(float *p, float v) { *p = v; }
};
// FP16 storage holds the offsets times 2^12 (exact: a power of two), so that
// offsets down to 1.5e-8 keep FP16's full 11-bit significand instead of
// falling into its subnormal range below 6.1e-5 (the induced magnetic field
// and the second-order parts of f^eq are that small); |offset| < 16 fits.
constexpr float H_SCALE = 4096.0f;
constexpr float H_UNSCALE = 1.0f / 4096.0f;
// log2 of the factor between stored and true offsets.  The bulk-node paths
// relax the stored values as they are, with the factor folded into the
// collision's constants (a power of two: the results are exactly those of
// the unscaled arithmetic, scaled).
template <class S> struct StoreScale { static constexpr int L2 = 0; };
template <> struct StoreScale<__half> { static constexpr int L2 = 12; };
template <> struct Codec<__half> {
    using T = float;
    LBM_DEV static float ld(const __half *p) { return __half2float(__ldg(p)) * H_UNSCALE; }
    LBM_DEV static float ld_raw(const __half *p) { return __half2float(__ldg(p)); }       // as stored
    LBM_DEV static float ld_shared(const __half *p) { return __half2float(*p) * H_UNSCALE; }
    LBM_DEV static void st(__half *p, float v) { *p = __float2half_rn(v * H_SCALE); }
};
template <> struct Codec<__nv_bfloat16> {
    using T = float;
    LBM_DEV static float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    LBM_DEV static float ld_raw(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    LBM_DEV static float ld_shared(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    LBM_DEV static void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

LBM_DEV uint32_t fast_div(uint32_t n, FastDiv d) { return (__umulhi(n, d.m) + n) >> d.s; }

// ------------------------------------------------------------------ stochastic rounding (16-bit storage)
// 16-bit storage rounds stochastically: a value is rounded up in magnitude
// with the probability of its distance to the lower neighbour (in units of
// their spacing), so that the rounding error has zero mean.  Round to nearest,
// at a steady state, makes the same error every step, which the flow
// integrates over its diffusion time; and a change smaller than half a
// spacing per step is lost every step, so slow transients stall.  The
// conversion instruction that takes random bits (cvt.rs, sm_100a and later)
// rounds two FP32 values to an FP16 or BF16 pair, each lane from its own half
// of a 32-bit random word.  Planes are rounded in pairs: a direction and its
// opposite (the member whose leading component is +1 in the low lane), rest
// planes alone in the low lane.  The random word of (step, node, pair) comes
// from a multiply-xorshift integer hash of the step and the node (constants
// of Wellons' "lowbias32"), then one multiplication by a constant of the
// pair's low plane, so every launch variant draws the same bits for the same
// population in the same lane.
template <class S> struct Rounding { static constexpr bool SR = false; };
template <> struct Rounding<__nv_bfloat16> { static constexpr bool SR = true; };
template <> struct Rounding<__half> { static constexpr bool SR = true; };

LBM_DEV uint32_t sr_node_hash(uint32_t step, uint32_t node) {
    uint32_t x = node * 0x9E3779B1u ^ step * 0x85EBCA77u;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// the random word of the pair whose low plane is q, at the node whose hash is h
LBM_DEV uint32_t sr_word(uint32_t h, int q) { return h * (0x2545F491u + 0x9E3779B9u * (uint32_t)q); }

// (lo, hi) rounded stochastically to one 32-bit word of two 16-bit values
// (values as stored: FP16 ones already scaled)
template <class S> LBM_DEV uint32_t sr_pack(float lo, float hi, uint32_t r);
template <> LBM_DEV uint32_t sr_pack<__half>(float lo, float hi, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
template <> LBM_DEV uint32_t sr_pack<__nv_bfloat16>(float lo, float hi, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
template <class S> LBM_DEV void store_bits(S *p, uint32_t w) { *reinterpret_cast<unsigned short *>(p) = (unsigned short)w; }

// the value as stored (SCALED: it already is)
template <class S, bool SCALED>
LBM_DEV float to_stored(float v) {
    if constexpr (StoreScale<S>::L2 != 0 && !SCALED) return v * float(1 << StoreScale<S>::L2);
    else return v;
}
// stores rest plane q of a node whose hash is h (SCALED: v is a stored value)
template <class S, bool SCALED = false>
LBM_DEV void store_pop(S *p, float v, uint32_t h, int q) {
    if constexpr (Rounding<S>::SR)
        store_bits(p, sr_pack<S>(to_stored<S, SCALED>(v), 0.0f, sr_word(h, q)));
    else
        Codec<S>::st(p, v);
}
// stores the pair of planes qp (low lane) and its opposite (high lane)
template <class S, bool SCALED = false, class V>
LBM_DEV void store_pop_pair(S *pp, S *pm, V vp, V vm, uint32_t h, int qp) {
    if constexpr (Rounding<S>::SR) {
        const uint32_t d = sr_pack<S>(to_stored<S, SCALED>(vp), to_stored<S, SCALED>(vm), sr_word(h, qp));
        store_bits(pp, d);
        store_bits(pm, d >> 16);
    } else {
        Codec<S>::st(pp, vp);
        Codec<S>::st(pm, vm);
    }
}
template <class S, bool SCALED = false>
LBM_DEV void store_pop(S *p, double v, uint32_t, int) { Codec<S>::st(p, v); }

LBM_DEV float fmaf_t(float a, float b, float c) { return fmaf(a, b, c); }
LBM_DEV double fmaf_t(double a, double b, double c) { return a * b + c; }   // FP64 serves parity: no fused rounding

template <class T>
struct StepParams {
    const void *src;
    void *dst;
    const uint8_t *flags;
    const CaseDev<T> *cases;
    const int2 *tiles;        // (case, first node) per tile of every node (bulk-copy and ring variants)
    int32_t ntiles;
    const int4 *spans;        // (case, lo, hi, 0): nodes [lo, hi) are bulk fluid (k_step, k_step_unwrapped)
    int32_t nspans;
    const BRec *brec;         // boundary nodes of all cases
    int32_t nbrec;
    const LinkDev<T> *links;
    LinkOut<T> *linkout;      // per link: its value for the coming step (k_links writes, k_boundary reads)
    int32_t nlinks;
    const int32_t *tile_brec; // boundary records of tile t: [tile_brec[t], tile_brec[t + 1])
    const ReactDev<T> *react; // surface reaction network per case (kernels with several species)
    const uint32_t *ctr_rd;   // the step count (stochastic rounding); the step's main kernel writes
    uint32_t *ctr_wr;         // count + 1 into the other slot (slots swap every step, as src and dst)
};

// block 0 of a step's main kernel advances the device step count
template <class T>
LBM_DEV void advance_step_count(const StepParams<T> &prm) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *prm.ctr_wr = *prm.ctr_rd + 1u;
}

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
//
// The relaxed flow populations are a quadratic polynomial in e_a.  With
// m = rho u = j + F/2 (Guo), om = 1/tau, g = 1 - 1/(2 tau), the BGK update
// of Eq. 1 with the equilibrium of Eq. 2 plus the magnetic stress and the
// Guo source w_a g [3 (e_a - u).F + 9 (e_a.u)(e_a.F)] collects into
//   s_rel,a = (1 - om) s_a + w_a (A + V.e_a + e_a.Tm.e_a)
//   A  = om (drho - 1.5 m.u + 0.75 (2 - D) |B|^2) - 3 g u.F
//   V  = 3 (om m + g F)
//   Tm = 4.5 [om (m u^T - B B^T) + g (u F^T + F u^T)] + 2.25 om |B|^2 I
// (the isotropic magnetic part 4.5 (|B|^2/2 (|e|^2 - D/3) + |B|^2/3) is
// 2.25 |B|^2 |e|^2 + 0.75 (2 - D) |B|^2).  Opposite directions share the even
// part A + e.Tm.e and differ in the sign of V.e.  Eq. 4 and 6 are linear in
// e_a: h_rel = (1 - om_h) h + om_h w (dC + 4 C e.u) and, per component k,
// g_rel = (1 - om_g) g + om_g w (dB_k + 4 e.(u B_k - B u_k)).
// The collision is written once over an arithmetic type V:
//   double  FP64 storage: plain operators (the FP64 translation units are
//           compiled without multiply-add contraction, so every product rounds)
//   F1      one node in FP32: every operation is an explicit round-to-nearest
//           intrinsic, so a product is fused into a sum only where fma_v says so
//   F2      two nodes in FP32 with the packed f32x2 instructions of sm_100 and
//           later; each lane rounds exactly as F1 does, so the result of a node
//           does not depend on which of the two forms computed it.
// Constants of the case are scalars T; products of scalars are formed in T
// before they meet a V.
struct F1 {
    float v;
    F1() = default;
    LBM_DEV F1(float x) : v(x) {}
};
LBM_DEV F1 operator+(F1 a, F1 b) { return F1(__fadd_rn(a.v, b.v)); }
LBM_DEV F1 operator-(F1 a, F1 b) { return F1(__fsub_rn(a.v, b.v)); }
LBM_DEV F1 operator*(F1 a, F1 b) { return F1(__fmul_rn(a.v, b.v)); }
LBM_DEV F1 fma_v(F1 a, F1 b, F1 c) { return F1(__fmaf_rn(a.v, b.v, c.v)); }
LBM_DEV F1 neg_v(F1 a) { return F1(-a.v); }
LBM_DEV F1 recip_v(F1 a) { return F1(__frcp_rn(a.v)); }

struct F2 {
    float2 v;
    F2() = default;
    LBM_DEV F2(float x) : v(make_float2(x, x)) {}
    LBM_DEV F2(float x, float y) : v(make_float2(x, y)) {}
};
LBM_DEV F2 operator+(F2 a, F2 b) { F2 r; r.v = __fadd2_rn(a.v, b.v); return r; }
// a - b = fma(b, -1, a): one rounding of the exact difference, as in the scalar subtraction
LBM_DEV F2 operator-(F2 a, F2 b) { F2 r; r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v); return r; }
LBM_DEV F2 operator*(F2 a, F2 b) { F2 r; r.v = __fmul2_rn(a.v, b.v); return r; }
LBM_DEV F2 fma_v(F2 a, F2 b, F2 c) { F2 r; r.v = __ffma2_rn(a.v, b.v, c.v); return r; }
LBM_DEV F2 neg_v(F2 a) { return F2(-a.v.x, -a.v.y); }
LBM_DEV F2 recip_v(F2 a) { return F2(__frcp_rn(a.v.x), __frcp_rn(a.v.y)); }

LBM_DEV double fma_v(double a, double b, double c) { return a * b + c; }
LBM_DEV double neg_v(double a) { return -a; }
LBM_DEV double recip_v(double a) { return 1.0 / a; }

// sum_a e_ai s_a over a lattice with e_ai in {-1, 0, 1}: (sum over +1) - (sum over -1);
// get(q) returns plane q
template <class L, int Q, class V, class Get>
LBM_DEV V axis_sum(Get &&get, int q0, int i) {
    V pos, neg;
    bool hp = false, hn = false;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int e = i == 0 ? L::ex(a) : (i == 1 ? L::ey(a) : L::ez(a));
        if (e > 0) {
            pos = hp ? pos + get(q0 + a) : get(q0 + a);
            hp = true;
        } else if (e < 0) {
            neg = hn ? neg + get(q0 + a) : get(q0 + a);
            hn = true;
        }
    }
    return pos - neg;
}

template <class V, class Get>
LBM_DEV V plane_sum(Get &&get, int q0, int n) {
    V s = get(q0);
#pragma unroll
    for (int a = 1; a < n; ++a) s = s + get(q0 + a);
    return s;
}

// first nonzero component of e_a
template <class L>
LBM_HD constexpr int lead_sign(int a) { return L::ex(a) ? L::ex(a) : (L::ey(a) ? L::ey(a) : L::ez(a)); }

// The collision over accessors: getm(q) reads plane q for the moments,
// getr(q) reads it again for its relaxation, put(q, v) takes the relaxed
// value of a rest plane and put2(qp, qm, vp, vm) those of a direction qp
// (leading component +1) and its opposite qm.  Every plane is read by getr
// once, before it is written.
// With SL2 > 0 the planes hold the offsets times 2^SL2: the moments are
// scaled back once, and the relaxed values come out scaled through the
// weights (exact: powers of two).
template <class PL, int NC, bool HG, class V, class T, int SL2 = 0, class GetM, class GetR, class Put, class Put2>
LBM_DEV void collide_g(GetM &&getm, GetR &&getr, Put &&put, Put2 &&put2, const CaseDev<T> &c) {
    using F = typename PL::F;
    using M = typename PL::M;
    constexpr int QF = PL::QF, QM = PL::QM, NB = PL::NB, DIM = F::DIM;
    constexpr double SC = double(1 << SL2);
    auto unscale = [](V v) -> V {
        if constexpr (SL2 != 0) return v * V(T(1.0 / SC));
        else return v;
    };
    const V drho = unscale(plane_sum<V>(getm, 0, QF));
    V j[3];
#pragma unroll
    for (int i = 0; i < DIM; ++i) j[i] = unscale(axis_sum<F, QF, V>(getm, 0, i));
    const V rho = drho + V(c.ref_rho);
    const V inv = recip_v(rho);
    const T acc[3] = {c.ax, c.ay, c.az};
    V Fo[3], m[3], u[3];
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        Fo[i] = rho * V(acc[i]);
        m[i] = fma_v(Fo[i], V(T(0.5)), j[i]);
        u[i] = m[i] * inv;
    }
    V B[3], nB[3], dB[3];
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            dB[k] = unscale(plane_sum<V>(getm, PL::G0 + k * QM, QM));
            B[k] = dB[k] + V(c.ref_B[k]);
            nB[k] = neg_v(B[k]);
        }
    }
    const T om = c.om_f, g = c.guo;
    V mu = m[0] * u[0], uF = u[0] * Fo[0], Bsq;
    if constexpr (HG) Bsq = B[0] * B[0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) {
        mu = fma_v(m[i], u[i], mu);
        uF = fma_v(u[i], Fo[i], uF);
        if constexpr (HG) Bsq = fma_v(B[i], B[i], Bsq);
    }
    V A = fma_v(mu, V(T(-1.5)), drho);
    if constexpr (HG && DIM == 3) A = fma_v(Bsq, V(T(-0.75)), A);   // 0.75 (2 - D) |B|^2 vanishes in 2D
    A = fma_v(A, V(om), V(T(-3) * g) * uF);
    // Td: Tm_ii (with the field) or Tm_ii / 4.5 (without: the even parts then
    // accumulate 4.5 Td with one fused operation per term)
    V Vv[3], Td[3], Tc[3];                                           // Tc: 2 Tm_xy, 2 Tm_xz, 2 Tm_yz
    V mag;
    if constexpr (HG) mag = V(T(2.25) * om) * Bsq;
    const T g2 = T(2) * g;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        Vv[i] = fma_v(m[i], V(om), V(g) * Fo[i]) * V(T(3));
        V t = m[i] * u[i];
        if constexpr (HG) t = fma_v(B[i], nB[i], t);
        const V s = fma_v(t, V(om), (V(g2) * u[i]) * Fo[i]);
        if constexpr (HG) Td[i] = fma_v(s, V(T(4.5)), mag);
        else Td[i] = s;
    }
#pragma unroll
    for (int pr = 0; pr < (DIM == 3 ? 3 : 1); ++pr) {
        const int i = pr == 2 ? 1 : 0, k = pr == 0 ? 1 : 2;
        V t = m[i] * u[k];
        if constexpr (HG) t = fma_v(nB[i], B[k], t);
        Tc[pr] = fma_v(t, V(om), V(g) * fma_v(u[i], Fo[k], Fo[i] * u[k])) * V(T(9));
    }
    const V omc = V(c.omc_f);
    put(0, fma_v(getr(0), omc, A * V(T(F::w(0) * SC))));                 // rest: even part A only
#pragma unroll
    for (int a = 1; a < QF; ++a) {
        const int b = F::opp(a);
        if (b < a) continue;                                         // done with its pair
        // the member of the pair whose leading component is +1 gets even + odd
        const int ap = lead_sign<F>(a) > 0 ? a : b, am = lead_sign<F>(a) > 0 ? b : a;
        const int e[3] = {F::ex(ap), F::ey(ap), F::ez(ap)};
        V even = A, odd;
        bool first = true;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            if (e[i]) {
                if constexpr (HG) even = even + Td[i];
                else even = fma_v(Td[i], V(T(4.5)), even);
                odd = first ? Vv[i] : (e[i] > 0 ? odd + Vv[i] : odd - Vv[i]);
                first = false;
            }
        }
#pragma unroll
        for (int pr = 0; pr < (DIM == 3 ? 3 : 1); ++pr) {
            const int i = pr == 2 ? 1 : 0, k = pr == 0 ? 1 : 2;
            const int s2 = e[i] * e[k];
            if (s2) even = s2 > 0 ? even + Tc[pr] : even - Tc[pr];
        }
        const V w = V(T(F::w(ap) * SC));
        const V we = even * w, wo = odd * w;
        const V vp = fma_v(getr(ap), omc, we + wo);
        put2(ap, am, vp, fma_v(getr(am), omc, we - wo));
    }
    const T w0 = T(M::w(0) * SC), w1 = T(M::w(1) * SC);
#pragma unroll
    for (int sp = 0; sp < NC; ++sp) {              // every concentration species, its own tau_D and C_ref
        const int h0 = PL::H0 + sp * QM;
        const V dC = unscale(plane_sum<V>(getm, h0, QM));
        const V C = dC + V(species_ref(c, sp));
        const T oh = species_om(c, sp);
        const V ohc = V(species_omc(c, sp));
        const V ev = V(oh * w1) * dC, f4 = V(T(4) * oh * w1) * C;
        put(h0, fma_v(getr(h0), ohc, V(oh * w0) * dC));
#pragma unroll
        for (int a = 1; a < QM; ++a) {
            const int b = M::opp(a);
            if (b < a) continue;
            const int ap = lead_sign<M>(a) > 0 ? a : b, am = lead_sign<M>(a) > 0 ? b : a;
            const int i = M::ex(a) ? 0 : (M::ey(a) ? 1 : 2);
            const V od = f4 * u[i];
            const V vp = fma_v(getr(h0 + ap), ohc, ev + od);
            put2(h0 + ap, h0 + am, vp, fma_v(getr(h0 + am), ohc, ev - od));
        }
    }
    if constexpr (HG) {
        const T og = c.om_g;
        const V ogc = V(c.omc_g);
        const V og1 = V(og * w1), og4 = V(T(4) * og * w1), og0 = V(og * w0);
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int q0 = PL::G0 + k * QM;
            const V ev = og1 * dB[k];
            put(q0, fma_v(getr(q0), ogc, og0 * dB[k]));
#pragma unroll
            for (int a = 1; a < QM; ++a) {
                const int b = M::opp(a);
                if (b < a) continue;
                const int ap = lead_sign<M>(a) > 0 ? a : b, am = lead_sign<M>(a) > 0 ? b : a;
                const int i = M::ex(a) ? 0 : (M::ey(a) ? 1 : 2);
                if (i == k) {                                        // u_k B_k - B_k u_k = 0
                    const V vp = fma_v(getr(q0 + ap), ogc, ev);
                    put2(q0 + ap, q0 + am, vp, fma_v(getr(q0 + am), ogc, ev));
                } else {
                    const V od = og4 * fma_v(u[i], B[k], nB[i] * u[k]);
                    const V vp = fma_v(getr(q0 + ap), ogc, ev + od);
                    put2(q0 + ap, q0 + am, vp, fma_v(getr(q0 + am), ogc, ev - od));
                }
            }
        }
    }
}

// in place on a register array
template <class PL, int NC, bool HG, class V, class T, int SL2 = 0>
LBM_DEV void collide_v(V (&p)[PL::P], const CaseDev<T> &c) {
    auto get = [&](int q) -> V { return p[q]; };
    auto put = [&](int q, V v) { p[q] = v; };
    auto put2 = [&](int qp, int qm, V vp, V vm) {
        p[qp] = vp;
        p[qm] = vm;
    };
    collide_g<PL, NC, HG, V, T, SL2>(get, get, put, put2, c);
}

// one node: FP64 as is, FP32 through F1 (SL2: values scaled by 2^SL2)
template <class PL, int NC, bool HG, class T, int SL2 = 0>
LBM_DEV void collide(T (&p)[PL::P], const CaseDev<T> &c) {
    if constexpr (sizeof(T) == 8) {
        collide_v<PL, NC, HG, T, T, SL2>(p, c);
    } else {
        F1 v[PL::P];
#pragma unroll
        for (int q = 0; q < PL::P; ++q) v[q] = F1(p[q]);
        collide_v<PL, NC, HG, F1, float, SL2>(v, c);
#pragma unroll
        for (int q = 0; q < PL::P; ++q) p[q] = v[q].v;
    }
}

// ------------------------------------------------------------------ wall links
template <int NQ, class S, class T>
LBM_DEV T field_sum(const S *src, int stride, int q0, int node) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) s += Codec<S>::ld(src + ((q0 + j) * stride + node));
    return s;
}

// The reaction increment of a link of species i (Sec. 4.2.2, text after
// Eq. 23): every species' C_m(X) by Eq. 13 from its own C at A and E, the
// network's production rate R_i at them, times the link's weight (cB[0],
// folded with the M scheme's 1/(d + 1/2) on the host).
template <class PL, class S, class T>
LBM_DEV T reaction_term(const LinkDev<T> &L, const S *src, int st, const CaseDev<T> &c, const ReactDev<T> &R) {
    constexpr int NC = PL::NCS;
    T CX[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const T CA = field_sum<PL::QM, S, T>(src, st, PL::H0 + m * PL::QM, L.nodeA) + species_ref(c, m);
        const T CE = field_sum<PL::QM, S, T>(src, st, PL::H0 + m * PL::QM, L.nodeE) + species_ref(c, m);
        CX[m] = (T(1) + L.d) * CA - L.d * CE;
    }
    const int i = ((int)L.phi_plane0 - PL::H0) / PL::QM;
    T Ri = T(0);
#pragma unroll
    for (int j = 0; j < MAX_REACT; ++j) {
        if (j >= R.n) break;
        T r = R.rate[j];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const uint32_t o = (R.ord[j] >> (8 * m)) & 0xffu;
            if (o >= 1) r = r * CX[m];
            if (o >= 2) r = r * CX[m];
        }
        Ri = Ri + R.st[j][i] * r;
    }
    return L.cB[0] * Ri;
}

template <class PL, class S, class T>
LBM_DEV T eval_link(const LinkDev<T> &L, const S *src, const CaseDev<T> &c, const ReactDev<T> *react) {
    const int st = (int)c.stride;
    const T paA = Codec<S>::ld(src + ((int)L.plane_a * st + L.nodeA));
    const T papA = Codec<S>::ld(src + ((int)L.plane_ap * st + L.nodeA));
    const T papE = Codec<S>::ld(src + ((int)L.plane_ap * st + L.nodeE));
    T v = L.c0 + L.ca * paA + L.cap * papA + L.cape * papE;
    if (L.flags & LINK_NEED_PHI) {
        T phA, phE;
        if (L.phi_plane0 < PL::QF) {
            phA = field_sum<PL::QF, S, T>(src, st, L.phi_plane0, L.nodeA);
            phE = field_sum<PL::QF, S, T>(src, st, L.phi_plane0, L.nodeE);
        } else {
            phA = field_sum<PL::QM, S, T>(src, st, L.phi_plane0, L.nodeA);
            phE = field_sum<PL::QM, S, T>(src, st, L.phi_plane0, L.nodeE);
        }
        phA += L.ref_phi;
        phE += L.ref_phi;
        v += L.cphi * ((T(1) + L.d) * phA - L.d * phE);
    }
    // given-pressure links exist only in flow-only cases
    if constexpr (PL::P == PL::QF) if (L.flags & LINK_NEED_U) {
        // fluid velocity at A and E from the relaxed populations:
        // u = (sum e s_rel - F/2) / rho, with F = rho * accel
        T rA = 0, rE = 0, jA[3] = {0, 0, 0}, jE[3] = {0, 0, 0};
#pragma unroll
        for (int q = 0; q < PL::QF; ++q) {
            const T vA = Codec<S>::ld(src + (q * st + L.nodeA));
            const T vE = Codec<S>::ld(src + (q * st + L.nodeE));
            rA += vA;
            rE += vE;
            if (PL::ex(q)) { jA[0] += T(PL::ex(q)) * vA; jE[0] += T(PL::ex(q)) * vE; }
            if (PL::ey(q)) { jA[1] += T(PL::ey(q)) * vA; jE[1] += T(PL::ey(q)) * vE; }
            if (PL::ez(q)) { jA[2] += T(PL::ez(q)) * vA; jE[2] += T(PL::ez(q)) * vE; }
        }
        rA += L.ref_phi;
        rE += L.ref_phi;
        const T acc[3] = {c.ax, c.ay, c.az};
        T eu = 0, uu = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T uX = (T(1) + L.d) * (jA[k] / rA - T(0.5) * acc[k]) - L.d * (jE[k] / rE - T(0.5) * acc[k]);
            eu += L.cB[k] * uX;
            uu += uX * uX;
        }
        v += L.cphi * (T(4.5) * eu * eu - T(1.5) * uu);
    }
    if constexpr (PL::NCS >= 2) {
        if (L.flags & LINK_NEED_REACT) v += reaction_term<PL, S, T>(L, src, st, c, *react);
    }
    if constexpr (PL::G0 < PL::P) {
        if (L.flags & LINK_NEED_B) {
#pragma unroll
            for (int k = 0; k < PL::NB; ++k) {
                const int q0 = PL::G0 + k * PL::QM;
                const T bA = field_sum<PL::QM, S, T>(src, st, q0, L.nodeA) + c.ref_B[k];
                const T bE = field_sum<PL::QM, S, T>(src, st, q0, L.nodeE) + c.ref_B[k];
                v += L.cB[k] * ((T(1) + L.d) * bA - L.d * bE);
            }
        }
    }
    return v;
}

// Replaces the populations of boundary node A that come from solid nodes by
// the wall formulas of its links [lo, hi).
// Links are taken LCH at a time so that their records and the populations
// they read are all in flight together.
template <class PL, class S, class T, int LCH>
LBM_DEV void apply_links(T (&p)[PL::P], const StepParams<T> &prm, const CaseDev<T> &c, const S *src, int lo, int hi) {
    for (int base = lo; base < hi; base += LCH) {
        LinkDev<T> L[LCH];
        T v[LCH];
#pragma unroll
        for (int j = 0; j < LCH; ++j)
            if (base + j < hi) L[j] = prm.links[base + j];
#pragma unroll
        for (int j = 0; j < LCH; ++j)
            v[j] = base + j < hi ? eval_link<PL, S, T>(L[j], src, c, PL::NCS >= 2 ? prm.react + c.index : nullptr) : T(0);
#pragma unroll
        for (int j = 0; j < LCH; ++j) {
            if (base + j >= hi) break;
            // select per plane (an indexed store would move p to local memory)
            const int pa = L[j].plane_a;
#pragma unroll
            for (int q = 0; q < PL::P; ++q) p[q] = (q == pa) ? v[j] : p[q];
        }
    }
}

// The same with the values already computed by k_links.
template <class PL, class T>
LBM_DEV void apply_links_pre(T (&p)[PL::P], const StepParams<T> &prm, int lo, int hi) {
    for (int j = lo; j < hi; ++j) {
        const LinkOut<T> o = prm.linkout[j];
#pragma unroll
        for (int q = 0; q < PL::P; ++q) p[q] = (q == o.plane) ? o.v : p[q];
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

// 16-bit populations two to a 32-bit register: plane q in half (q & 1) of word q >> 1
// (values as stored)
template <class S> struct Pack16;
template <> struct Pack16<__half> {
    LBM_DEV static uint32_t raw(const __half *p) { return __ldg(reinterpret_cast<const unsigned short *>(p)); }
    LBM_DEV static float get(uint32_t w, int hi) {
        const __half2 h = *reinterpret_cast<const __half2 *>(&w);
        return hi ? __high2float(h) : __low2float(h);
    }
};
template <> struct Pack16<__nv_bfloat16> {
    LBM_DEV static uint32_t raw(const __nv_bfloat16 *p) {
        return __ldg(reinterpret_cast<const unsigned short *>(p));
    }
    LBM_DEV static float get(uint32_t w, int hi) { return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16)); }
};

// Stores every plane of a node in the pairs of collide_g: rest planes alone,
// a direction with its opposite (the same lanes and random words as the
// collision's own put and put2).
template <class PL, int NC, bool HG, class S, bool SCALED, class V>
LBM_DEV void store_node(S *dp, int os, const V (&p)[PL::P], uint32_t h) {
    using F = typename PL::F;
    using M = typename PL::M;
    auto pairs = [&](auto L, int q0, int nq) {
        using LL = decltype(L);
#pragma unroll
        for (int a = 1; a < nq; ++a) {
            const int b = LL::opp(a);
            if (b < a) continue;
            const int ap = lead_sign<LL>(a) > 0 ? a : b, am = lead_sign<LL>(a) > 0 ? b : a;
            store_pop_pair<S, SCALED>(dp + (q0 + ap) * os, dp + (q0 + am) * os, p[q0 + ap], p[q0 + am], h, q0 + ap);
        }
    };
    store_pop<S, SCALED>(dp, p[0], h, 0);
    pairs(F{}, 0, PL::QF);
#pragma unroll
    for (int sp = 0; sp < NC; ++sp) {
        const int h0 = PL::H0 + sp * PL::QM;
        store_pop<S, SCALED>(dp + h0 * os, p[h0], h, h0);
        pairs(M{}, h0, PL::QM);
    }
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < PL::NB; ++k) {
            const int q0 = PL::G0 + k * PL::QM;
            store_pop<S, SCALED>(dp + q0 * os, p[q0], h, q0);
            pairs(M{}, q0, PL::QM);
        }
    }
}

// ------------------------------------------------------------------ fused step
// One node: pull, (boundary nodes: wall links [lo, hi)), collide, store
// plane q to out[q * ostride] (out = 0: the node's entries of the target buffer).
// LINKS: 0 a bulk node; 1 a wall-link node whose links are evaluated here
// (LCH at a time); 2 a wall-link node whose link values k_links computed.
template <int DIM, int NC, bool HG, class S, int LINKS, int LCH = 4>
LBM_DEV void step_node(const StepParams<typename Codec<S>::T> &prm, const CaseDev<typename Codec<S>::T> &c, int n,
                       int lo, int hi, S *out = nullptr, int ostride = 0) {
    using PL = Planes<DIM, NC, HG>;
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
    // in-case offsets are 32-bit (the host keeps P * stride below 2^31) and
    // taken from one 64-bit pointer per node: the source of plane q is
    // sp[q * stride + (wrapped neighbour offset of e_q)]
    const int st32 = (int)c.stride;
    const S *__restrict__ sp = src + n;
    S *__restrict__ dp = out ? out : dst + n;
    const int os = out ? ostride : st32;
    const int ox[3] = {xi[0] - x, 0, xi[2] - x};
    const int oy[3] = {yi[0] - yi[1], 0, yi[2] - yi[1]};
    const int oz[3] = {zi[0] - zi[1], 0, zi[2] - zi[1]};
    if constexpr (!LINKS && sizeof(S) == 2 && P > 24) {
        // many 16-bit planes (3D with fields): the pulled values stay packed two
        // to a register; the moments and then the relaxation each convert them
        // (the empty asm keeps the second conversion from reusing the first),
        // and every relaxed value is stored as soon as it is formed.  Same
        // arithmetic as the array path below.
        uint32_t pk[(P + 1) / 2];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const uint32_t w = Pack16<S>::raw(sp + (q * st32 + ox[1 - PL::ex(q)] + oy[1 - PL::ey(q)] + oz[1 - PL::ez(q)]));
            pk[q >> 1] = (q & 1) ? (pk[q >> 1] | (w << 16)) : w;
        }
        auto getm = [&](int q) -> F1 { return F1(Pack16<S>::get(pk[q >> 1], q & 1)); };
        auto getr = [&](int q) -> F1 {
            uint32_t w = pk[q >> 1];
            asm("" : "+r"(w));
            return F1(Pack16<S>::get(w, q & 1));
        };
        const uint32_t h = Rounding<S>::SR ? sr_node_hash(*prm.ctr_rd, (uint32_t)(c.node_off + n)) : 0u;
        auto put = [&](int q, F1 v) { store_pop<S, true>(dp + q * os, v.v, h, q); };
        auto put2 = [&](int qp, int qm, F1 vp, F1 vm) {
            store_pop_pair<S, true>(dp + qp * os, dp + qm * os, vp.v, vm.v, h, qp);
        };
        collide_g<PL, NC, HG, F1, float, StoreScale<S>::L2>(getm, getr, put, put2, c);
        return;
    }
    // bulk nodes relax the values as stored; wall-link nodes the true offsets
    // (the link formulas take them)
    constexpr int SL2 = LINKS ? 0 : StoreScale<S>::L2;
    T p[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const S *a = sp + (q * st32 + ox[1 - PL::ex(q)] + oy[1 - PL::ey(q)] + oz[1 - PL::ez(q)]);
        p[q] = SL2 ? Codec<S>::ld_raw(a) : Codec<S>::ld(a);
    }
    if constexpr (LINKS == 1) apply_links<PL, S, T, LCH>(p, prm, c, src, lo, hi);
    if constexpr (LINKS == 2) apply_links_pre<PL, T>(p, prm, lo, hi);
    collide<PL, NC, HG, T, SL2>(p, c);
    const uint32_t h = Rounding<S>::SR ? sr_node_hash(*prm.ctr_rd, (uint32_t)(c.node_off + n)) : 0u;
    store_node<PL, NC, HG, S, SL2 != 0>(dp, os, p, h);
}

// Bulk nodes (fluid, no wall link) over the span list: span t holds nodes
// [lo, hi) of one case, all bulk fluid, at most blockDim.x * npt of them; each
// thread takes nodes lo + tid, lo + tid + blockDim.x, ...  No node flag is
// read: solid and wall-link nodes are in no span (k_boundary relaxes the
// latter).
// MINB: resident 256-thread blocks per SM the kernel is compiled for (its
// register budget, 65536 / (256 MINB) registers per thread).
template <int DIM, int NC, bool HG, class S, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step(const StepParams<typename Codec<S>::T> prm, const int npt) {
    using T = typename Codec<S>::T;
    advance_step_count(prm);
    for (int t = blockIdx.x; t < prm.nspans; t += gridDim.x) {
        const int4 sp = prm.spans[t];
        // the descriptor by value: the stores below cannot alias it, so it stays in registers
        const CaseDev<T> c = prm.cases[sp.x];
        for (int k = 0; k < npt; ++k) {
            const int n = sp.y + (int)threadIdx.x + k * (int)blockDim.x;
            if (n >= sp.z) break;
            step_node<DIM, NC, HG, S, 0>(prm, c, n, 0, 0);
        }
    }
}

// ------------------------------------------------------------------ unwrapped pulls (launch variant 2)
// One bulk node n: every plane's pull is read unwrapped, at n - s_q with s_q
// the flat offset of e_q, so that a plane's address is the node's own plus a
// per-case constant (q * stride - s_q); the pool's guard bands keep these
// reads inside the allocation.  A node on a periodic edge of its case then
// reloads the planes whose source wraps (a short branch taken by those lanes
// only).  16-bit populations stay packed two to a register until the
// collision reads them (once for the moments, once for the relaxation).  Same
// arithmetic as step_node: the bits are those of k_step.
template <class S> struct Raw16 {
    LBM_DEV static uint32_t ld(const S *p) { return __ldg(reinterpret_cast<const unsigned short *>(p)); }
    LBM_DEV static float get(uint32_t w, int hi);
};
template <> LBM_DEV float Raw16<__half>::get(uint32_t w, int hi) {
    __half2 h;
    memcpy(&h, &w, 4);
    return hi ? __high2float(h) : __low2float(h);
}
template <> LBM_DEV float Raw16<__nv_bfloat16>::get(uint32_t w, int hi) {
    return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
}

template <int DIM, int NC, bool HG, class S>
LBM_DEV void step_node_unwrapped(const StepParams<typename Codec<S>::T> &prm, const CaseDev<typename Codec<S>::T> &c,
                                 const int n) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    constexpr bool PACK = sizeof(S) == 2;
    const S *__restrict__ src = static_cast<const S *>(prm.src) + c.pop_off;
    S *__restrict__ dp = static_cast<S *>(prm.dst) + c.pop_off + n;
    const int nx = c.nx, ny = c.ny, nxy = nx * ny;
    const int st = (int)c.stride;
    const S *__restrict__ sp = src + n;
    // raw pulls: 16-bit values two to a 32-bit word (plane q in half q & 1 of
    // word q >> 1), wider types as they are
    uint32_t pk[PACK ? (P + 1) / 2 : 1];
    T p[PACK ? 1 : P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int o = q * st - (PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy);
        if constexpr (PACK) {
            const uint32_t w = Raw16<S>::ld(sp + o);
            pk[q >> 1] = (q & 1) ? (pk[q >> 1] | (w << 16)) : w;
        } else {
            p[q] = Codec<S>::ld(sp + o);
        }
    }
    int x, y, z, r;
    coords<DIM, T>(c, n, x, y, z, r);
    const int nz = c.nz;
    if (x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || (DIM == 3 && (z == 0 || z == nz - 1))) {
        const int N = c.N;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            int corr = 0;
            if (PL::ex(q) > 0 && x == 0) corr += nx;
            if (PL::ex(q) < 0 && x == nx - 1) corr -= nx;
            if (PL::ey(q) > 0 && y == 0) corr += nxy;
            if (PL::ey(q) < 0 && y == ny - 1) corr -= nxy;
            if (DIM == 3 && PL::ez(q) > 0 && z == 0) corr += N;
            if (DIM == 3 && PL::ez(q) < 0 && z == nz - 1) corr -= N;
            if (corr != 0) {
                const int o = q * st - (PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy) + corr;
                if constexpr (PACK) {
                    const uint32_t w = Raw16<S>::ld(sp + o);
                    pk[q >> 1] = (q & 1) ? ((pk[q >> 1] & 0x0000ffffu) | (w << 16)) : ((pk[q >> 1] & 0xffff0000u) | w);
                } else {
                    p[q] = Codec<S>::ld(sp + o);
                }
            }
        }
    }
    if constexpr (PACK) {
        auto getm = [&](int q) -> F1 { return F1(Raw16<S>::get(pk[q >> 1], q & 1)); };
        auto getr = [&](int q) -> F1 {
            uint32_t w = pk[q >> 1];
            asm("" : "+r"(w));                 // convert again rather than keep the moments' copy alive
            return F1(Raw16<S>::get(w, q & 1));
        };
        const uint32_t h = Rounding<S>::SR ? sr_node_hash(*prm.ctr_rd, (uint32_t)(c.node_off + n)) : 0u;
        auto put = [&](int q, F1 v) { store_pop<S, true>(dp + q * st, v.v, h, q); };
        auto put2 = [&](int qp, int qm, F1 vp, F1 vm) {
            store_pop_pair<S, true>(dp + qp * st, dp + qm * st, vp.v, vm.v, h, qp);
        };
        collide_g<PL, NC, HG, F1, float, StoreScale<S>::L2>(getm, getr, put, put2, c);
    } else {
        collide<PL, NC, HG, T>(p, c);
#pragma unroll
        for (int q = 0; q < P; ++q) Codec<S>::st(dp + q * st, p[q]);
    }
}

// Bulk nodes over the span list with unwrapped pulls (launch variant 2):
// the same node order and tiling as k_step.
template <int DIM, int NC, bool HG, class S, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_unwrapped(const StepParams<typename Codec<S>::T> prm, const int npt) {
    using T = typename Codec<S>::T;
    advance_step_count(prm);
    for (int t = blockIdx.x; t < prm.nspans; t += gridDim.x) {
        const int4 spn = prm.spans[t];
        const CaseDev<T> c = prm.cases[spn.x];
        for (int k = 0; k < npt; ++k) {
            const int n = spn.y + (int)threadIdx.x + k * (int)blockDim.x;
            if (n >= spn.z) break;
            step_node_unwrapped<DIM, NC, HG, S>(prm, c, n);
        }
    }
}

// 3D walls (curved walls give a node many links) evaluate their links in a
// kernel of their own ahead of k_boundary, so that the links of a node run in
// parallel instead of one after another; 2D walls (a few links per node, the
// wall-link kernel far off the critical path) evaluate them inside
// k_boundary and save the launch.  (Measured on GB300: MHD pipe FP16 and FP32
// against the Hartmann batch.)
template <int DIM>
LBM_HD constexpr bool links_apart() { return DIM == 3; }
// In 2D and for 16-bit 3D storage the inline link evaluation is built lean
// (links one at a time, a small register budget), so that its blocks take few
// of the registers the bulk step's blocks would use; FP64 needs the full budget.
template <class S, int DIM>
LBM_HD constexpr bool boundary_lean() { return sizeof(S) == 2 || (DIM == 2 && sizeof(S) == 4); }
template <class S, int DIM>
LBM_HD constexpr int boundary_minb() {
    return links_apart<DIM>() ? (sizeof(S) == 8 ? 2 : 6) : (boundary_lean<S, DIM>() ? 8 : 1);
}

// Wall links, one thread per link: the value each link gives its unknown
// population in the coming step (from the relaxed populations at t, which the
// step only reads), with the plane it replaces.  It runs on the side stream
// ahead of k_boundary.  Links of frozen cases are evaluated too (their values
// are not used).
template <int DIM, int NC, bool HG, class S>
__global__ void __launch_bounds__(256) k_links(const StepParams<typename Codec<S>::T> prm) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= prm.nlinks) return;
    const LinkDev<T> L = prm.links[i];
    const CaseDev<T> &c = prm.cases[L.cs];
    const S *src = static_cast<const S *>(prm.src) + c.pop_off;
    LinkOut<T> o;
    o.v = eval_link<PL, S, T>(L, src, c, PL::NCS >= 2 ? prm.react + c.index : nullptr);
    o.plane = L.plane_a;
    prm.linkout[i] = o;
}

// Boundary nodes: one thread per record of the compact boundary list (the
// nodes of a wall row are consecutive records, so a warp works along a wall).
// It runs beside the bulk step on a side stream.
template <int DIM, int NC, bool HG, class S>
__global__ void __launch_bounds__(128, boundary_minb<S, DIM>()) k_boundary(const StepParams<typename Codec<S>::T> prm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= prm.nbrec) return;
    const BRec b = prm.brec[i];
    const CaseDev<typename Codec<S>::T> c = prm.cases[b.cs];
    if constexpr (links_apart<DIM>())
        step_node<DIM, NC, HG, S, 2>(prm, c, b.node, b.lo, b.hi);
    else
        step_node<DIM, NC, HG, S, 1, boundary_lean<S, DIM>() ? 1 : 4>(prm, c, b.node, b.lo, b.hi);
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
    T C0s[MAX_SPECIES];       // initial C of every species (species 0: C0 unless the field C is given)
};

template <int DIM, int NC, bool HG, class S, class FT>
__global__ void __launch_bounds__(256) k_init(const InitParams<typename Codec<S>::T, FT> ip) {
    using PL = Planes<DIM, NC, HG>;
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
#pragma unroll
    for (int sp = 0; sp < NC; ++sp) {
        const T Cs = sp == 0 ? C : ip.C0s[sp];
#pragma unroll
        for (int a = 0; a < PL::QM; ++a) p[PL::H0 + sp * PL::QM + a] = heq_dir<M, T>(a, Cs - species_ref(c, sp), Cs, u);
    }
    if constexpr (HG) {
#pragma unroll
        for (int k = 0; k < PL::NB; ++k)
#pragma unroll
            for (int a = 0; a < PL::QM; ++a) p[PL::G0 + k * PL::QM + a] = geq_dir<M, T>(a, k, B[k] - c.ref_B[k], B, u);
    }
    collide<PL, NC, HG, T>(p, c);
#pragma unroll
    for (int q = 0; q < P; ++q) Codec<S>::st(dst + (q * st32 + n), p[q]);
}

}  // namespace lbm
