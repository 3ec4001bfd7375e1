// links.cu -- host-side wall-link builders of the C ABI (no GPU needed):
// flat channel walls (Sec. 4-5) and the curved pipe wall with surface
// segmentation and conservative flux splitting (Sec. 6, Eq. 48).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lattice.cuh"
#include "lbm.h"

namespace {

struct Dirs {
    int q;
    int e[19][3];
};

template <class L>
Dirs dirs() {
    Dirs d{};
    d.q = L::Q;
    for (int a = 0; a < L::Q; ++a) {
        d.e[a][0] = L::ex(a);
        d.e[a][1] = L::ey(a);
        d.e[a][2] = L::ez(a);
    }
    return d;
}

Dirs field_dirs(int dim, int field) {
    if (field == 0) return dim == 2 ? dirs<lbm::D2Q9>() : dirs<lbm::D3Q19>();
    return dim == 2 ? dirs<lbm::D2Q5>() : dirs<lbm::D3Q7>();
}

std::vector<int> enabled_fields(int dim, uint32_t physics) {
    std::vector<int> f{0};
    if (physics & LBM_CD) f.push_back(1);
    if (physics & LBM_MHD)
        for (int k = 0; k < dim; ++k) f.push_back(2 + k);
    return f;
}

struct Grid {
    int nx, ny, nz;
    int64_t idx(int x, int y, int z) const {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
        return x + (int64_t)nx * (y + (int64_t)ny * z);
    }
};

lbm_link make_link(int64_t node, int field, int dir, const lbm_wall_bc &bc, double d, double k0, double k1) {
    lbm_link l;
    std::memset(&l, 0, sizeof l);
    l.node = (uint32_t)node;
    l.field = (uint8_t)field;
    l.dir = (uint8_t)dir;
    l.kind = (uint8_t)bc.kind;
    l.d = d;
    for (int k = 0; k < 3; ++k) l.u_wall[k] = bc.u_wall[k];
    l.phi_wall = bc.phi_wall;
    l.k0 = k0;
    l.k1 = k1;
    return l;
}

lbm_status emit(const std::vector<lbm_link> &v, lbm_link *links, size_t cap, size_t *nlinks) {
    if (nlinks) *nlinks = v.size();
    if (!links) return LBM_OK;
    if (cap < v.size()) return LBM_EINVAL;
    std::copy(v.begin(), v.end(), links);
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_build_channel(int32_t dim, int32_t nx, int32_t ny, int32_t nz, int32_t axis, double d_lo,
                             double d_hi, uint32_t physics, const lbm_wall_bc *bc, uint8_t *solid,
                             lbm_link *links, size_t cap, size_t *nlinks) {
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1)) return LBM_EINVAL;
    if (axis < 0 || axis >= dim || !bc || !solid) return LBM_EINVAL;
    if (!(d_lo > 0 && d_lo <= 1) || !(d_hi > 0 && d_hi <= 1)) return LBM_EINVAL;
    const Grid g{nx, ny, nz};
    const int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
    if (n_axis < 3) return LBM_EINVAL;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t n = 0; n < N; ++n) {
        const int c[3] = {(int)(n % nx), (int)((n / nx) % ny), (int)(n / ((int64_t)nx * ny))};
        solid[n] = (c[axis] == 0 || c[axis] == n_axis - 1) ? 1 : 0;
    }
    std::vector<lbm_link> out;
    for (int field : enabled_fields(dim, physics)) {
        const Dirs D = field_dirs(dim, field);
        for (int64_t n = 0; n < N; ++n) {
            if (solid[n]) continue;
            const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            for (int a = 1; a < D.q; ++a) {
                const int64_t b = g.idx(x - D.e[a][0], y - D.e[a][1], z - D.e[a][2]);
                if (!solid[b]) continue;
                // the upstream solid layer is the low wall when e_a points up the axis
                const int side = D.e[a][axis] > 0 ? 0 : 1;
                const lbm_wall_bc &w = bc[side * 5 + field];
                const double d = side == 0 ? d_lo : d_hi;
                // flat wall: one D2Q5/D3Q7 link per interface element of area dx^2 (Eq. 23)
                out.push_back(make_link(n, field, a, w, d, w.kappa0, w.kappa1));
            }
        }
    }
    return emit(out, links, cap, nlinks);
}

lbm_status lbm_build_pipe(int32_t nx, int32_t ny, int32_t nz, double R, uint32_t physics, const lbm_wall_bc *bc,
                          uint8_t *solid, lbm_link *links, size_t cap, size_t *nlinks) {
    if (nx < 1 || ny < 3 || nz < 3 || !(R > 0) || !bc || !solid) return LBM_EINVAL;
    const Grid g{nx, ny, nz};
    const double cy = 0.5 * (ny - 1), cz = 0.5 * (nz - 1);
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t n = 0; n < N; ++n) {
        const int y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        const double ry = y - cy, rz = z - cz;
        solid[n] = (ry * ry + rz * rz < R * R) ? 0 : 1;
    }
    // surface segments of the outer-layer solid points, per axial slice
    const Dirs D7 = dirs<lbm::D3Q7>();
    std::vector<double> S(N, 0.0), nrm_y(N, 0.0), nrm_z(N, 0.0);
    for (int x = 0; x < nx; ++x) {
        struct P { double th; int64_t n; };
        std::vector<P> pts;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y) {
                const int64_t n = g.idx(x, y, z);
                if (!solid[n]) continue;
                bool outer = false;
                for (int a = 1; a < 7; ++a)
                    if (!solid[g.idx(x + D7.e[a][0], y + D7.e[a][1], z + D7.e[a][2])]) outer = true;
                if (outer) pts.push_back(P{std::atan2(z - cz, y - cy), n});
            }
        std::sort(pts.begin(), pts.end(), [](const P &a, const P &b) { return a.th < b.th || (a.th == b.th && a.n < b.n); });
        const size_t m = pts.size();
        const double two_pi = 2.0 * M_PI;
        for (size_t i = 0; i < m; ++i) {
            const double th_next = pts[(i + 1) % m].th + (i + 1 == m ? two_pi : 0.0);
            const double th_prev = pts[(i + m - 1) % m].th - (i == 0 ? two_pi : 0.0);
            const int64_t n = pts[i].n;
            S[n] = 0.5 * (th_next - th_prev) * R;
            const int y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            const double ry = y - cy, rz = z - cz, r = std::sqrt(ry * ry + rz * rz);
            nrm_y[n] = -ry / r;   // inward normal (into the fluid)
            nrm_z[n] = -rz / r;
        }
    }
    std::vector<lbm_link> out;
    for (int field : enabled_fields(3, physics)) {
        const Dirs D = field_dirs(3, field);
        const lbm_wall_bc &w = bc[field];
        for (int64_t n = 0; n < N; ++n) {
            if (solid[n]) continue;
            const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
            const double ay = y - cy, az = z - cz;
            for (int a = 1; a < D.q; ++a) {
                const int ex = D.e[a][0], ey = D.e[a][1], ez = D.e[a][2];
                const int64_t b = g.idx(x - ex, y - ey, z - ez);
                if (!solid[b]) continue;
                // wall point X = A - d e_a on the circle, d in (0, 1]
                const double ee = (double)(ey * ey + ez * ez);
                const double ae = ay * ey + az * ez;
                double d = (ae + std::sqrt(ae * ae + ee * (R * R - (ay * ay + az * az)))) / ee;
                d = std::min(1.0, std::max(d, 1e-12));
                double k0 = 0.0, k1 = 0.0;
                if ((w.kind == LBM_W_FLUX || w.kind == LBM_W_FLUX_SIMPLIFIED) && field != 0) {
                    const double proj = ey * nrm_y[b] + ez * nrm_z[b];
                    double tot = 0.0;
                    const int bx = (int)(b % nx), by = (int)((b / nx) % ny), bz = (int)(b / ((int64_t)nx * ny));
                    for (int c = 1; c < 7; ++c) {
                        const double pc = D7.e[c][1] * nrm_y[b] + D7.e[c][2] * nrm_z[b];
                        if (pc > 0 && !solid[g.idx(bx + D7.e[c][0], by + D7.e[c][1], bz + D7.e[c][2])]) tot += pc;
                    }
                    const double share = (proj > 0 && tot > 0) ? proj / tot : 0.0;
                    k0 = w.kappa0 * S[b] * share;
                    k1 = w.kappa1 * S[b] * share;
                }
                out.push_back(make_link(n, field, a, w, d, k0, k1));
            }
        }
    }
    return emit(out, links, cap, nlinks);
}

}  // extern "C"
