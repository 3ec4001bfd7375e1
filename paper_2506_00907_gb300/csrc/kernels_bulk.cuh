// kernels_bulk.cuh -- the fused bulk step with bulk-copy (TMA) loads and stores.
//
// Same arithmetic as k_step (kernels.cuh); only the way populations move
// between HBM and the registers differs.  A persistent block walks the tile
// list.  For the NEXT tile one elected thread issues, per population plane q,
// one cp.async.bulk of the contiguous source window [start - s_q, start + len
// - s_q) (s_q = flat index offset of e_q; aligned outward to 16 bytes and
// clamped to the plane) into one of two shared-memory stages, completing on an
// mbarrier with an expected byte count, while the block computes the current
// tile from the other stage.  Results go to a shared-memory output tile that
// the elected thread writes back with one cp.async.bulk store per plane.  HBM
// then sees a few kilobytes of contiguous traffic per plane and tile instead
// of 2- or 4-byte accesses per thread.
//
// Every node looks its source up in the window and falls back to a direct
// load when the periodic wrap puts the source outside it.  Solid and
// boundary nodes get zeros in the output tile; k_boundary, launched after
// this kernel on the same stream, writes the boundary nodes.
//
// Every mbarrier wait is bounded: on timeout the block records an error code
// in err[0], waits (bounded) for its own copies and returns.
#pragma once
#include "kernels.cuh"

namespace lbm {

struct BulkParams {
    int32_t tile_nodes;       // nodes per tile (a multiple of 16 bytes of elements)
    int32_t cap;              // window elements per plane and stage (tile_nodes + 16 bytes of elements)
    int32_t *err;             // error word (0 = ok)
};

constexpr uint32_t BULK_SPIN_LIMIT = 1u << 24;
constexpr int BULK_STAGES = 2;

// shared memory before the stage buffers: mbarriers + window table [stage][2P]
__host__ __device__ constexpr int bulk_header_bytes(int P) {
    return ((16 * BULK_STAGES + BULK_STAGES * 2 * P * 4 + 127) / 128) * 128;
}
// total dynamic shared memory of one block
__host__ __device__ constexpr size_t bulk_smem_bytes(int P, int tile, int cap, int elem) {
    return (size_t)bulk_header_bytes(P) + (size_t)BULK_STAGES * P * cap * elem + (size_t)P * tile * elem;
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
LBM_DEV void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
LBM_DEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
LBM_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
LBM_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
LBM_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// window of plane q for a tile: element range [lo, hi) of the plane, aligned
// to 16 bytes and clamped to the plane's extent rounded up to 16 bytes
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
LBM_DEV void bulk_issue(const StepParams<T> &prm, const BulkParams &bp, int t, int st, uint64_t *bar, int *win,
                        S *stage_buf) {
    constexpr int P = PL::P;
    const int2 tile = prm.tiles[t];
    const CaseDev<T> &c = prm.cases[tile.x];
    const int len = min(bp.tile_nodes, c.N - tile.y);
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
    S *dstb = stage_buf + (size_t)st * P * bp.cap;
    for (int q = 0; q < P; ++q) {
        const int lo = w[q], hi = w[P + q];
        if (hi > lo)
            bulk_g2s(dstb + (size_t)q * bp.cap, src + (int64_t)q * c.stride + lo,
                     (uint32_t)(hi - lo) * (uint32_t)sizeof(S), &bar[st]);
    }
}

template <int DIM, bool HH, bool HG, class S, int MINB>
__global__ void __launch_bounds__(256, MINB) k_step_bulk(const StepParams<typename Codec<S>::T> prm,
                                                         const BulkParams bp) {
    using PL = Planes<DIM, HH, HG>;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    constexpr int A = 16 / (int)sizeof(S);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);                            // [BULK_STAGES]
    int *win = reinterpret_cast<int *>(smem + 16 * BULK_STAGES);                    // [BULK_STAGES][2P]
    S *stage_buf = reinterpret_cast<S *>(smem + bulk_header_bytes(P));
    S *out = stage_buf + (size_t)BULK_STAGES * P * bp.cap;                         // [P][tile_nodes]
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < BULK_STAGES; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0 && (int)blockIdx.x < prm.ntiles) bulk_issue<PL, S, T>(prm, bp, blockIdx.x, 0, bar, win, stage_buf);
    int k_iter = 0;
    for (int t = blockIdx.x; t < prm.ntiles; t += gridDim.x, ++k_iter) {
        const int st = k_iter & 1;
        // the other stage was consumed in the previous iteration (everyone passed its barriers)
        const int tn = t + gridDim.x;
        if (tid == 0 && tn < prm.ntiles) bulk_issue<PL, S, T>(prm, bp, tn, st ^ 1, bar, win, stage_buf);
        uint32_t spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&bar[st], (k_iter >> 1) & 1)) {
            if (++spins > BULK_SPIN_LIMIT) { ok = false; break; }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(bp.err, 1);
                // let this block's copies land before the block exits (bounded)
                for (uint32_t k = 0; k < BULK_SPIN_LIMIT && !mbar_try_wait(&bar[st ^ 1], ((k_iter + 1) >> 1) & 1); ++k) {
                }
                bulk_wait_all();
            }
            return;
        }
        if (tid == 0) bulk_wait_read();       // the previous tile's stores are done reading `out`
        __syncthreads();
        const int2 tile = prm.tiles[t];
        const CaseDev<T> c = prm.cases[tile.x];
        const S *src = static_cast<const S *>(prm.src) + c.pop_off;
        const S *sb = stage_buf + (size_t)st * P * bp.cap;
        const int *wlo = win + st * 2 * P;
        const int *whi = wlo + P;
        const int nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
        const int len = min(bp.tile_nodes, c.N - tile.y);
        const int st32 = (int)c.stride;
        for (int i = tid; i < len; i += blockDim.x) {
            const int n = tile.y + i;
            const uint8_t fl = prm.flags[c.node_off + n];
            if (fl != NODE_FLUID) {                 // solid, or a boundary node (k_boundary writes it)
#pragma unroll
                for (int q = 0; q < P; ++q) Codec<S>::st(out + q * bp.tile_nodes + i, T(0));
                continue;
            }
            int x, y, z, r;
            coords<DIM, T>(c, n, x, y, z, r);
            const int xi[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
            const int yi[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
            int zi[3] = {0, 0, 0};
            if constexpr (DIM == 3) {
                zi[0] = (z == 0 ? nz - 1 : z - 1) * nxy;
                zi[1] = z * nxy;
                zi[2] = (z == nz - 1 ? 0 : z + 1) * nxy;
            }
            T p[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                const int sn = xi[1 - PL::ex(q)] + yi[1 - PL::ey(q)] + zi[1 - PL::ez(q)];
                const int lo = wlo[q];
                p[q] = (unsigned)(sn - lo) < (unsigned)(whi[q] - lo)
                           ? (T)Codec<S>::ld_shared(sb + (size_t)q * bp.cap + (sn - lo))
                           : Codec<S>::ld(src + (q * st32 + sn));
            }
            collide<PL, HH, HG, T>(p, c);
#pragma unroll
            for (int q = 0; q < P; ++q) Codec<S>::st(out + q * bp.tile_nodes + i, p[q]);
        }
        // a ragged last tile stores up to the next 16 bytes: zeros there, inside the plane's padding
        const int lenA = ((len + A - 1) / A) * A;
        for (int i = len + tid; i < lenA; i += blockDim.x)
#pragma unroll
            for (int q = 0; q < P; ++q) Codec<S>::st(out + q * bp.tile_nodes + i, T(0));
        fence_async_smem();                       // generic-proxy writes of `out` before the async-proxy stores
        __syncthreads();
        if (tid == 0) {
            S *dst = static_cast<S *>(prm.dst) + c.pop_off;
            for (int q = 0; q < P; ++q)
                bulk_s2g(dst + (int64_t)q * c.stride + tile.y, out + q * bp.tile_nodes,
                         (uint32_t)lenA * (uint32_t)sizeof(S));
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
}

}  // namespace lbm
