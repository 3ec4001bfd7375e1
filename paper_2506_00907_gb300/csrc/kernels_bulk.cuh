// kernels_bulk.cuh -- the fused step with bulk-copy (TMA) loads and stores.
//
// Same arithmetic as k_step (kernels.cuh); only the way populations move
// between HBM and the registers differs.  Persistent blocks of 256 threads
// walk the tile list (tiles of TT nodes).  While a block computes tile k, the
// lanes of warp 0 keep one cp.async.bulk per population plane in flight for
// each of the next NS - 1 tiles, copying the plane's source window
// ([start - s_q, start + len - s_q), s_q the flat index offset of e_q,
// aligned outward to 16 bytes and clamped to the plane) into a ring of NS
// shared-memory stages, each completing on its own mbarrier.  Results go to
// one of two output tiles in shared memory, which the same lanes write back
// with one cp.async.bulk store per plane.  HBM then sees kilobytes of contiguous traffic per plane
// and tile instead of 2- or 4-byte accesses per thread.
//
// Interior nodes read their source at a fixed offset in the window; nodes on
// the periodic edges look their wrapped source up in the window and load it
// directly when it lies outside.  Wall-link (boundary) nodes of the tile are
// computed after the bulk nodes by the whole block, from global memory, into
// the output tile; solid nodes and the ragged end of the last tile get zeros.
//
// Every mbarrier wait is bounded: on timeout the block records an error code
// in err[0], waits (bounded) for its own copies and returns.
#pragma once
#include "kernels.cuh"

namespace lbm {

struct BulkParams {
    int32_t *err;             // error word (0 = ok)
};

constexpr uint32_t BULK_SPIN_LIMIT = 1u << 24;
constexpr int BULK_THREADS = 256;

// compiled (tile nodes, resident 256-thread blocks per SM of the register
// budget, input stages = tiles in flight + 1)
constexpr int BULK_NCFG = 5;
constexpr int BULK_TT[BULK_NCFG] = {128, 256, 256, 512, 512};
constexpr int BULK_MB[BULK_NCFG] = {2, 2, 4, 1, 2};
constexpr int BULK_NS[BULK_NCFG] = {3, 3, 3, 2, 2};
constexpr int BULK_MAX_NS = 4;

template <int P, int TT, int ELEM, int NS>
struct BulkLayout {
    static constexpr int A = 16 / ELEM;             // elements per 16 bytes
    static constexpr int CAP = TT + A;              // window elements per plane and stage
    static constexpr int BAR = 0;                   // NS mbarriers
    static constexpr int WLO = 8 * BULK_MAX_NS;     // [NS][P] window starts
    static constexpr int WHI = WLO + NS * P * 4;    // [NS][P] window ends
    static constexpr int HDR = ((WHI + NS * P * 4 + 127) / 128) * 128;
    static constexpr int IN = HDR;                  // [NS][P][CAP] windows
    static constexpr int OUT = IN + NS * P * CAP * ELEM;  // [2][P][TT] output tiles
    static constexpr int BYTES = OUT + 2 * P * TT * ELEM;
};

// the same total for run-time arguments (host side)
__host__ __device__ constexpr int bulk_layout_bytes(int P, int TT, int ELEM, int NS) {
    return ((8 * BULK_MAX_NS + 2 * NS * P * 4 + 127) / 128) * 128 + NS * P * (TT + 16 / ELEM) * ELEM +
           2 * P * TT * ELEM;
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
LBM_DEV void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
LBM_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
LBM_DEV void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp 0: the windows of tile t into stage st (lane q handles planes q, q + 32).
template <class PL, class S, class T, int TT, int NS>
LBM_DEV void bulk_issue(const StepParams<T> &prm, int t, int st, unsigned char *smem) {
    constexpr int P = PL::P;
    constexpr int NJ = (P + 31) / 32;
    using L = BulkLayout<P, TT, (int)sizeof(S), NS>;
    constexpr int A = L::A;
    const int lane = threadIdx.x & 31;
    const int2 tile = prm.tiles[t];
    const CaseDev<T> &c = prm.cases[tile.x];
    const int len = min(TT, c.N - tile.y);
    const int nx = c.nx, nxy = c.nx * c.ny;
    const int top = ((c.N + A - 1) / A) * A;
    int *wlo = reinterpret_cast<int *>(smem + L::WLO) + st * P;
    int *whi = reinterpret_cast<int *>(smem + L::WHI) + st * P;
    int lo[NJ], hi[NJ];
    uint32_t bytes = 0;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int q = lane + 32 * j;
        lo[j] = hi[j] = 0;
        if (q < P) {
            const int s = PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy;
            const int a = tile.y - s, b = tile.y + len - s;
            lo[j] = a < 0 ? 0 : (a / A) * A;
            const int h = ((b + A - 1) / A) * A;
            hi[j] = h > top ? top : h;
            if (hi[j] < lo[j]) hi[j] = lo[j];
            wlo[q] = lo[j];
            whi[q] = hi[j];
            bytes += (uint32_t)(hi[j] - lo[j]) * (uint32_t)sizeof(S);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::BAR) + st;
    if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
    __syncwarp();
    const S *src = static_cast<const S *>(prm.src) + c.pop_off;
    S *in = reinterpret_cast<S *>(smem + L::IN) + (size_t)st * P * L::CAP;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int q = lane + 32 * j;
        if (q < P && hi[j] > lo[j])
            bulk_g2s(in + (size_t)q * L::CAP, src + (int64_t)q * c.stride + lo[j],
                     (uint32_t)(hi[j] - lo[j]) * (uint32_t)sizeof(S), bar);
    }
}

template <int DIM, int NC, bool HG, class S, int MINB, int TT, int NS>
__global__ void __launch_bounds__(BULK_THREADS, MINB) k_step_bulk(const StepParams<typename Codec<S>::T> prm,
                                                                  const BulkParams bp) {
    using PL = Planes<DIM, NC, HG>;
    using T = typename Codec<S>::T;
    constexpr int P = PL::P;
    using L = BulkLayout<P, TT, (int)sizeof(S), NS>;
    static_assert(L::BYTES == bulk_layout_bytes(P, TT, (int)sizeof(S), NS), "layout");
    static_assert(NS >= 2 && NS <= BULK_MAX_NS, "stages");
    constexpr int A = L::A;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::BAR);
    const int tid = threadIdx.x;
    advance_step_count(prm);
    const bool w0 = tid < 32;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the first NS - 1 tiles of this block go into stages 0 .. NS - 2
    if (w0)
        for (int k = 0; k < NS - 1; ++k) {
            const int t0 = blockIdx.x + k * gridDim.x;
            if (t0 < prm.ntiles) bulk_issue<PL, S, T, TT, NS>(prm, t0, k, smem);
        }
    int k_iter = 0;
    for (int t = blockIdx.x; t < prm.ntiles; t += gridDim.x, ++k_iter) {
        const int st = k_iter % NS;
        const int ob = k_iter & 1;
        // NS - 1 tiles ahead: tile k_iter + NS - 1 goes to the stage consumed in the previous iteration;
        // output tile ob was last used two iterations ago
        const int ta = t + (NS - 1) * gridDim.x;
        if (w0) {
            if (ta < prm.ntiles) bulk_issue<PL, S, T, TT, NS>(prm, ta, (k_iter + NS - 1) % NS, smem);
            bulk_wait_read_1();            // the stores of two tiles ago are done reading output tile ob
        }
        uint32_t spins = 0;
        bool ok = true;
        while (!mbar_try_wait(&bar[st], (k_iter / NS) & 1)) {
            if (++spins > BULK_SPIN_LIMIT) { ok = false; break; }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(bp.err, 1);
            if (w0) {
                // let this block's copies in flight land before the block exits (bounded waits)
                for (int d = 1; d < NS; ++d) {
                    const int kk = k_iter + d;
                    for (uint32_t k = 0; k < BULK_SPIN_LIMIT && !mbar_try_wait(&bar[kk % NS], (kk / NS) & 1); ++k) {
                    }
                }
                bulk_wait_all();
            }
            return;
        }
        const int2 tile = prm.tiles[t];
        const CaseDev<T> c = prm.cases[tile.x];
        const S *src = static_cast<const S *>(prm.src) + c.pop_off;
        const S *in = reinterpret_cast<const S *>(smem + L::IN) + (size_t)st * P * L::CAP;
        S *out = reinterpret_cast<S *>(smem + L::OUT) + (size_t)ob * P * TT;
        const int *wlo = reinterpret_cast<const int *>(smem + L::WLO) + st * P;
        const int *whi = reinterpret_cast<const int *>(smem + L::WHI) + st * P;
        const int nx = c.nx, ny = c.ny, nz = c.nz, nxy = nx * ny;
        const int len = min(TT, c.N - tile.y);
        const int st32 = (int)c.stride;
        for (int i = tid; i < len; i += BULK_THREADS) {
            const int n = tile.y + i;
            const uint8_t fl = prm.flags[c.node_off + n];
            if (fl != NODE_FLUID) {
                if (!(fl & NODE_BOUNDARY))       // solid: zeros (boundary nodes are written below)
#pragma unroll
                    for (int q = 0; q < P; ++q) Codec<S>::st(out + q * TT + i, T(0));
                continue;
            }
            int x, y, z, r;
            coords<DIM, T>(c, n, x, y, z, r);
            const bool edge = x == 0 || x == nx - 1 || y == 0 || y == ny - 1 ||
                              (DIM == 3 && (z == 0 || z == nz - 1));
            T p[P];
            if (!edge) {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const int s = PL::ex(q) + PL::ey(q) * nx + PL::ez(q) * nxy;
                    p[q] = (T)Codec<S>::ld_shared(in + q * L::CAP + (n - s - wlo[q]));
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
                    const int lo = wlo[q];
                    p[q] = (unsigned)(sn - lo) < (unsigned)(whi[q] - lo)
                               ? (T)Codec<S>::ld_shared(in + q * L::CAP + (sn - lo))
                               : Codec<S>::ld(src + (q * st32 + sn));
                }
            }
            collide<PL, NC, HG, T>(p, c);
#pragma unroll
            for (int q = 0; q < P; ++q) Codec<S>::st(out + q * TT + i, p[q]);
        }
        // boundary nodes of the tile, from global memory, into the output tile
        // (one link at a time: these nodes are few, registers matter more here)
        const int b_lo = prm.tile_brec[t], b_hi = prm.tile_brec[t + 1];
        for (int b = b_lo + tid; b < b_hi; b += BULK_THREADS) {
            const BRec rec = prm.brec[b];
            step_node<DIM, NC, HG, S, 1, 1>(prm, c, rec.node, rec.lo, rec.hi, out + (rec.node - tile.y), TT);
        }
        // a ragged last tile stores up to the next 16 bytes: zeros there, inside the plane's padding
        const int lenA = ((len + A - 1) / A) * A;
        for (int i = len + tid; i < lenA; i += BULK_THREADS)
#pragma unroll
            for (int q = 0; q < P; ++q) Codec<S>::st(out + q * TT + i, T(0));
        fence_async_smem();                       // generic-proxy writes of `out` before the async-proxy stores
        __syncthreads();
        if (w0) {
            S *dst = static_cast<S *>(prm.dst) + c.pop_off;
#pragma unroll
            for (int j = 0; j < (P + 31) / 32; ++j) {
                const int q = tid + 32 * j;
                if (q < P)
                    bulk_s2g(dst + (int64_t)q * c.stride + tile.y, out + q * TT, (uint32_t)lenA * (uint32_t)sizeof(S));
            }
            bulk_commit();
        }
    }
    if (w0) bulk_wait_all();
}

}  // namespace lbm
