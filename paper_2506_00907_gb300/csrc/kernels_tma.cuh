// kernels_tma.cuh -- the fused step with a bulk-copy (TMA) prefetch pipeline.
//
// Same arithmetic as k_step (kernels.cuh); only the way the pulled populations
// reach the registers differs.  A persistent block walks the tile list; for
// the NEXT tile one elected thread issues, per population plane q, one
// cp.async.bulk of the contiguous source window [start - s_q, start + len - s_q)
// (s_q = flat index offset of e_q) into shared memory, completing on an
// mbarrier with an expected byte count, while the whole block computes the
// current tile from the other shared-memory stage.  The bytes in flight per
// SM are then set by the stage size, not by registers and occupancy.
//
// Interior nodes read their source at smem[i + base_q]; nodes on the edge of
// the periodic box (whose source wraps) look their source up in the window
// and fall back to a direct load when it is outside.  Windows are aligned to
// 16 bytes as cp.async.bulk requires and clamped to the plane.
//
// Every mbarrier wait is bounded: on timeout the block records an error code
// in err[0], waits (bounded) for its own copies and returns.
#pragma once
#include "kernels.cuh"

namespace lbm {

struct TmaParams {
    int32_t tile_nodes;       // nodes per tile (a multiple of blockDim.x)
    int32_t cap;              // elements per plane per stage (multiple of 16 bytes)
    int32_t stages;           // ring depth, 2..TMA_MAX_STAGES
    int32_t *err;             // error word (0 = ok)
};

constexpr uint32_t TMA_SPIN_LIMIT = 1u << 24;
constexpr int TMA_MAX_STAGES = 4;

// shared memory before the stage buffers: mbarriers + the window table [stage][2P]
__host__ __device__ constexpr int tma_header_bytes(int P) {
    return ((8 * TMA_MAX_STAGES + TMA_MAX_STAGES * 2 * P * 4 + 127) / 128) * 128;
}

LBM_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

LBM_DEV void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
LBM_DEV void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
LBM_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
LBM_DEV void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// window of plane q for a tile: element range [lo, hi) of the plane, aligned
// to 16 bytes and clamped to the plane's padded extent
template <class PL, class S>
LBM_DEV void plane_window(int q, int start, int len, int nx, int nxy, int N, int &lo, int &hi) {
    constexpr int A = 16 / (int)sizeof(S);
    const int s = PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy;
    const int a = start - s, b = start + len - s;
    lo = a < 0 ? 0 : (a / A) * A;
    const int top = ((N + A - 1) / A) * A;
    const int h = ((b + A - 1) / A) * A;
    hi = h > top ? top : h;
    if (hi < lo) hi = lo;
}

// Issued by one thread: the windows of tile t into stage st.
template <class PL, class S, class T>
LBM_DEV void tma_issue(const StepParams<T> &prm, const TmaParams &tp, int t, int st, uint64_t *bar, int *win,
                       S *stage_buf) {
    constexpr int P = PL::P;
    const int2 tile = prm.tiles[t];
    const CaseDev<T> &c = prm.cases[tile.x];
    const int len = min(tp.tile_nodes, c.N - tile.y);
    const S *src = static_cast<const S *>(prm.src) + c.pop_off;
    int *w = win + st * 2 * P;
    uint32_t total = 0;
    for (int q = 0; q < P; ++q) {
        int lo, hi;
        plane_window<PL, S>(q, tile.y, len, c.nx, c.nx * c.ny, c.N, lo, hi);
        w[q] = lo;
        w[P + q] = hi;
        total += (uint32_t)(hi - lo) * (uint32_t)sizeof(S);
    }
    mbar_arrive_expect_tx(&bar[st], total);
    S *dstb = stage_buf + (size_t)st * P * tp.cap;
    for (int q = 0; q < P; ++q) {
        const int lo = w[q], hi = w[P + q];
        if (hi > lo)
            bulk_g2s(dstb + (size_t)q * tp.cap, src + (int64_t)q * c.stride + lo, (uint32_t)(hi - lo) * (uint32_t)sizeof(S),
                     &bar[st]);
    }
}

template <int DIM, bool HH, bool HG, class S, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_tma(const StepParams<typename Codec<S>::T> prm, const TmaParams tp) {
    using PL = Planes<DIM, HH, HG>;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);                            // [stages]
    int *win = reinterpret_cast<int *>(smem + 8 * TMA_MAX_STAGES);                  // [stages][2P]
    S *stage_buf = reinterpret_cast<S *>(smem + tma_header_bytes(P));
    const int tid = threadIdx.x;
    const int NS = tp.stages;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // prologue: the first NS - 1 tiles of this block
    if (tid == 0)
        for (int k = 0; k < NS - 1; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < prm.ntiles) tma_issue<PL, S, T>(prm, tp, t, k, bar, win, stage_buf);
        }
    uint32_t phases = 0u;     // bit k = parity to wait for on stage k
    int st = 0, k_iter = 0;
    for (int t = blockIdx.x; t < prm.ntiles; t += gridDim.x, ++k_iter) {
        // keep NS - 1 tiles in flight: tile k_iter + NS - 1 goes to the stage freed last iteration
        const int ahead = t + (NS - 1) * gridDim.x;
        if (tid == 0 && ahead < prm.ntiles) tma_issue<PL, S, T>(prm, tp, ahead, (k_iter + NS - 1) % NS, bar, win, stage_buf);
        uint32_t spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&bar[st], (phases >> st) & 1u)) {
            if (++spins > TMA_SPIN_LIMIT) { ok = false; break; }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(tp.err, 1);
                // let this block's copies land before the block exits (bounded)
                for (int s2 = 0; s2 < NS; ++s2)
                    for (uint32_t k = 0; k < TMA_SPIN_LIMIT && !mbar_try_wait(&bar[s2], (phases >> s2) & 1u); ++k) {
                    }
            }
            return;
        }
        phases ^= 1u << st;

        const int2 tile = prm.tiles[t];
        const CaseDev<T> &c = prm.cases[tile.x];
        const S *src = static_cast<const S *>(prm.src) + c.pop_off;
        S *dst = static_cast<S *>(prm.dst) + c.pop_off;
        const S *sb = stage_buf + (size_t)st * P * tp.cap;
        const int *wlo = win + st * 2 * P;
        const int *whi = wlo + P;
        const int nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
        const int len = min(tp.tile_nodes, c.N - tile.y);
        const int st32 = (int)c.stride;
        for (int i = tid; i < len; i += blockDim.x) {
            const int n = tile.y + i;
            const uint8_t fl = prm.flags[c.node_off + n];
            if (fl != NODE_FLUID) continue;         // solid, or a boundary node (k_boundary)
            int x, y, z, r;
            coords<DIM, T>(c, n, x, y, z, r);
            const bool edge = x == 0 || x == nx - 1 || y == 0 || y == ny - 1 ||
                              (DIM == 3 && (z == 0 || z == nz - 1));
            T p[P];
            if (!edge) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int s = PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy;
                    p[q] = (T)Codec<S>::ld_shared(sb + (size_t)q * tp.cap + (n - s - wlo[q]));
                }
            } else {
                const int xi[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
                const int yi[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
                int zi[3] = {0, 0, 0};
                if constexpr (DIM == 3) {
                    zi[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
                    zi[1] = z * nxy;
                    zi[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
                }
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int sn = xi[1 - PL::ex(q)] + yi[1 - PL::ey(q)] + zi[1 - PL::ez(q)];
                    p[q] = (sn >= wlo[q] && sn < whi[q])
                               ? (T)Codec<S>::ld_shared(sb + (size_t)q * tp.cap + (sn - wlo[q]))
                               : Codec<S>::ld(src + (q * st32 + sn));
                }
            }
            collide<PL, HH, HG, T>(p, c);
#pragma unroll
            for (int q = 0; q < P; ++q) Codec<S>::st(dst + (q * st32 + n), p[q]);
        }
        __syncthreads();   // every thread is done with stage st before it is refilled
        st = st + 1 == NS ? 0 : st + 1;
    }
}

}  // namespace lbm
