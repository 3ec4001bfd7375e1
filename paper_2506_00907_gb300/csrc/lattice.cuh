// lattice.cuh -- compile-time lattice descriptions for the fused step.
//
// Flow: D2Q9 / D3Q19 (Sec. 2.1, c_s^2 = 1/3).  Concentration and the vector
// magnetic field: D2Q5 / D3Q7 (Sec. 2.2-2.3) with c^2 = 1/4, i.e. rest weight
// 1/2 (2D) or 1/4 (3D) and 1/8 for every moving direction; the paper does not
// print these weights, its parameter sets (Sec. 5.3, 5.4, 6) all imply
// c_h^2 = c_g^2 = c^2/4.
// Direction numbering is part of the C ABI (include/lbm.h).
#pragma once

#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int DIM = 2;
    // 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y)
    LBM_HD static constexpr int ex(int a) {
        return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0;
    }
    LBM_HD static constexpr int ey(int a) {
        return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0;
    }
    LBM_HD static constexpr int ez(int) { return 0; }
    LBM_HD static constexpr double w(int a) { return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
    LBM_HD static constexpr int opp(int a) { return a == 0 ? 0 : (a < 5 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5); }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int DIM = 3;
    // 0 rest; axis pairs 1/2 (x), 3/4 (y), 5/6 (z); edge pairs
    // 7 (+x+y) 8 (-x-y) 9 (+x-y) 10 (-x+y) 11 (+x+z) 12 (-x-z) 13 (+x-z) 14 (-x+z)
    // 15 (+y+z) 16 (-y-z) 17 (+y-z) 18 (-y+z)
    LBM_HD static constexpr int ex(int a) {
        return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
             : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
    }
    LBM_HD static constexpr int ey(int a) {
        return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
             : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
    }
    LBM_HD static constexpr int ez(int a) {
        return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
             : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
    }
    LBM_HD static constexpr double w(int a) { return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
    LBM_HD static constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
};

struct D2Q5 {
    static constexpr int Q = 5;
    static constexpr int DIM = 2;
    LBM_HD static constexpr int ex(int a) { return a == 1 ? 1 : (a == 3 ? -1 : 0); }
    LBM_HD static constexpr int ey(int a) { return a == 2 ? 1 : (a == 4 ? -1 : 0); }
    LBM_HD static constexpr int ez(int) { return 0; }
    LBM_HD static constexpr double w(int a) { return a == 0 ? 0.5 : 0.125; }
    LBM_HD static constexpr int opp(int a) { return a == 0 ? 0 : ((a + 1) % 4) + 1; }
};

struct D3Q7 {
    static constexpr int Q = 7;
    static constexpr int DIM = 3;
    LBM_HD static constexpr int ex(int a) { return a == 1 ? 1 : (a == 2 ? -1 : 0); }
    LBM_HD static constexpr int ey(int a) { return a == 3 ? 1 : (a == 4 ? -1 : 0); }
    LBM_HD static constexpr int ez(int a) { return a == 5 ? 1 : (a == 6 ? -1 : 0); }
    LBM_HD static constexpr double w(int a) { return a == 0 ? 0.25 : 0.125; }
    LBM_HD static constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
};

// The concatenated population planes of one node: f (QF planes), then the
// NC concentration species h_0 .. h_{NC-1} (QM each), then g_0 .. g_{DIM-1}
// (QM each, if MHD).
template <int DIM, int NC, bool HG>
struct Planes {
    using F = typename std::conditional<DIM == 2, D2Q9, D3Q19>::type;
    using M = typename std::conditional<DIM == 2, D2Q5, D3Q7>::type;
    static constexpr int QF = F::Q;
    static constexpr int QM = M::Q;
    static constexpr int NB = DIM;
    static constexpr int NCS = NC;       // concentration species
    static constexpr int H0 = QF;
    static constexpr int G0 = QF + NC * QM;
    static constexpr int P = G0 + (HG ? NB * QM : 0);
    LBM_HD static constexpr int dir(int q) { return q < QF ? q : (q < G0 ? (q - H0) % QM : (q - G0) % QM); }
    LBM_HD static constexpr int ex(int q) { return q < QF ? F::ex(q) : M::ex(dir(q)); }
    LBM_HD static constexpr int ey(int q) { return q < QF ? F::ey(q) : M::ey(dir(q)); }
    LBM_HD static constexpr int ez(int q) { return q < QF ? F::ez(q) : M::ez(dir(q)); }
    LBM_HD static constexpr double w(int q) { return q < QF ? F::w(q) : M::w(dir(q)); }
};

}  // namespace lbm
