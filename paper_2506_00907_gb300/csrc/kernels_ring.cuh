// kernels_ring.cuh -- the fused step fed through a ring of shared-memory stages.
//
// Same arithmetic as k_step (kernels.cuh); the populations reach the
// registers differently.  A block is one producer warp and RING_CW consumer
// warps.  The producer walks the block's tiles (t = blockIdx.x, + gridDim.x,
// ...) and, for each, fills a free stage: every population plane's source
// window ([start - s_q, start + len - s_q), s_q the flat index offset of e_q,
// widened to 16 bytes) and the tile's node flags with one cp.async.bulk each,
// completing on the stage's `full` mbarrier, and the tile record and its case
// descriptor (fetched one tile ahead) written by its lanes.  Consumers wait on
// `full`, read everything they need from the stage into registers, arrive on
// the stage's `empty` mbarrier (which frees it for the producer), then relax
// their nodes and store the results straight to global memory.  There is no
// block-wide barrier in the loop: the producer runs up to NS tiles ahead.
//
// NPL = 2: each consumer lane takes two x-adjacent nodes and relaxes them
// together with packed f32x2 arithmetic (collide_v<F2>); planes whose window
// shift is even are read as one 32- or 64-bit word.  NPL = 1: one node per
// lane (F1).  Both give the bits of the one-node kernel.
//
// Nodes on a periodic edge, and nodes whose partner in the pair is not bulk
// fluid, take the one-node path from global memory (step_node).  Wall-link
// nodes are left to k_boundary, as for k_step.
//
// Every mbarrier wait is bounded: on timeout the warp records an error code
// in err[0] and raises the block's abort word; the producer then stops
// issuing, waits (bounded) for its copies in flight and returns.
#pragma once
#include <cstddef>

#include "kernels_bulk.cuh"

namespace lbm {

constexpr int RING_CW = 8;                         // consumer warps per block
constexpr int RING_THREADS = (RING_CW + 1) * 32;   // + the producer warp
constexpr int RING_MAX_NS = 8;                     // stages
constexpr int RING_MAX_QF = 20;                    // window shifts per stage (>= 19 lattice vectors)

// shared memory: full[NS], empty[NS] mbarriers and the abort word, then per
// stage a metadata block (the tile record, a copy of its case descriptor, the
// window shifts and the node flags of the tile), then the windows [NS][P][CAP]
__host__ __device__ constexpr int ring_tile(int npl) { return RING_CW * 32 * npl; }
__host__ __device__ constexpr int ring_cap(int npl, int elem) { return ring_tile(npl) + 16 / elem; }
constexpr int RING_FULL = 0;
constexpr int RING_EMPTY = 8 * RING_MAX_NS;
constexpr int RING_ABORT = 16 * RING_MAX_NS;
constexpr int RING_META = 256;
constexpr int RM_TILE = 0;                         // int2
constexpr int RM_CASE = 16;                        // CaseDev<float>
constexpr int RM_SHIFT = 208;                      // int[RING_MAX_QF]: window index of the tile's first pull source
constexpr int RM_FLAGS = 288;                      // uint8_t[tile nodes, rounded up to 16]
__host__ __device__ constexpr int ring_meta_bytes(int npl) { return ((RM_FLAGS + ring_tile(npl) + 127) / 128) * 128; }
__host__ __device__ constexpr int ring_win_off(int npl, int ns) { return RING_META + ns * ring_meta_bytes(npl); }
__host__ __device__ constexpr int ring_smem_bytes(int P, int npl, int elem, int ns) {
    return ring_win_off(npl, ns) + ns * P * ring_cap(npl, elem) * elem;
}
static_assert(sizeof(CaseDev<float>) <= RM_SHIFT - RM_CASE, "case descriptor slot");
static_assert(RM_SHIFT + 4 * RING_MAX_QF <= RM_FLAGS, "shift slot");

LBM_DEV void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait for the completion of phase `parity`; false on timeout or when
// the block's abort word is raised
LBM_DEV bool ring_wait(uint64_t *bar, uint32_t parity, volatile int *abort_word) {
    for (uint32_t k = 0; k < BULK_SPIN_LIMIT; ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 255) == 255 && *abort_word) return false;
    }
    return false;
}

// the flow plane with the lattice vector of plane q (every vector of the
// D2Q5/D3Q7 lattices is one of D2Q9/D3Q19)
template <class PL>
LBM_HD constexpr int flow_dir(int q) {
    for (int a = 0; a < PL::QF; ++a)
        if (PL::F::ex(a) == PL::ex(q) && PL::F::ey(a) == PL::ey(q) && PL::F::ez(a) == PL::ez(q)) return a;
    return 0;
}

// two consecutive values from shared memory (aligned to their pair size) and
// the packed store of two results
template <class S> struct PairMem;
template <> struct PairMem<float> {
    LBM_DEV static float2 lds(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    LBM_DEV static void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <> struct PairMem<__half> {
    LBM_DEV static float2 lds(const __half *p) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        return make_float2(v.x * H_UNSCALE, v.y * H_UNSCALE);
    }
    LBM_DEV static void st(__half *p, float2 v) {
        *reinterpret_cast<__half2 *>(p) = __float22half2_rn(make_float2(v.x * H_SCALE, v.y * H_SCALE));
    }
};
template <> struct PairMem<__nv_bfloat16> {
    LBM_DEV static float2 lds(const __nv_bfloat16 *p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    LBM_DEV static void st(__nv_bfloat16 *p, float2 v) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
    }
};

// Producer: one tile into stage st.  `tile` is its record and the lanes hold
// its case descriptor as 32-bit words (lane w: words w and w + 32), fetched
// one tile ahead.  The lanes copy both into the stage's metadata and compute
// the plane windows; lane q copies planes q, q + 32 and the last lane the
// tile's node flags, all completing on the stage's `full` mbarrier.
constexpr int RING_CW_WORDS = (int)(sizeof(CaseDev<float>) / 4);
static_assert(RING_CW_WORDS <= 64, "case words per lane");
template <int OFF>
LBM_DEV int case_word(int wa, int wb) {
    return __shfl_sync(0xffffffffu, OFF / 4 < 32 ? wa : wb, (OFF / 4) & 31);
}
template <int OFF>
LBM_DEV int64_t case_word64(int wa, int wb) {
    const uint32_t lo = (uint32_t)case_word<OFF>(wa, wb), hi = (uint32_t)case_word<OFF + 4>(wa, wb);
    return (int64_t)(((uint64_t)hi << 32) | lo);
}

template <class PL, class S, int NPL>
LBM_DEV void ring_issue(const StepParams<float> &prm, int2 tile, int wa, int wb, int st, unsigned char *smem,
                        int ns) {
    constexpr int P = PL::P;
    constexpr int NJ = (P + 31) / 32;
    constexpr int TT = ring_tile(NPL);
    constexpr int A = 16 / (int)sizeof(S);
    constexpr int CAP = ring_cap(NPL, (int)sizeof(S));
    using CD = CaseDev<float>;
    const int lane = threadIdx.x & 31;
    unsigned char *meta = smem + RING_META + st * ring_meta_bytes(NPL);
    if (lane == 0) *reinterpret_cast<int2 *>(meta + RM_TILE) = tile;
    int *mcase = reinterpret_cast<int *>(meta + RM_CASE);
    if (lane < RING_CW_WORDS) mcase[lane] = wa;
    if (lane + 32 < RING_CW_WORDS) mcase[lane + 32] = wb;
    const int nx = case_word<offsetof(CD, nx)>(wa, wb), ny = case_word<offsetof(CD, ny)>(wa, wb);
    const int N = case_word<offsetof(CD, N)>(wa, wb);
    const int64_t pop_off = case_word64<offsetof(CD, pop_off)>(wa, wb);
    const int64_t stride = case_word64<offsetof(CD, stride)>(wa, wb);
    const int64_t node_off = case_word64<offsetof(CD, node_off)>(wa, wb);
    const int len = min(TT, N - tile.y);
    const int nxy = nx * ny;
    const int top = ((N + A - 1) / A) * A;
    int *shift = reinterpret_cast<int *>(meta + RM_SHIFT);
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
            if (q < PL::QF) shift[q] = a - lo[j];          // window index of the pull source of the tile's first node
            bytes += (uint32_t)(hi[j] - lo[j]) * (uint32_t)sizeof(S);
        }
    }
    // flags of the tile: node_off and tile.y are multiples of 64, the flag array is padded to 64 per case
    const uint32_t fbytes = (uint32_t)((len + 15) / 16) * 16u;
    if (lane == 31) bytes += fbytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    __syncwarp();                                            // metadata before the arrival that publishes it
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + RING_FULL) + st;
    if (lane == 0) mbar_arrive_expect_tx(full, bytes);
    __syncwarp();
    const S *src = static_cast<const S *>(prm.src) + pop_off;
    S *win = reinterpret_cast<S *>(smem + ring_win_off(NPL, ns)) + (size_t)st * P * CAP;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int q = lane + 32 * j;
        if (q < P && hi[j] > lo[j])
            bulk_g2s(win + (size_t)q * CAP, src + (int64_t)q * stride + lo[j],
                     (uint32_t)(hi[j] - lo[j]) * (uint32_t)sizeof(S), full);
    }
    if (lane == 31) bulk_g2s(meta + RM_FLAGS, prm.flags + node_off + tile.y, fbytes, full);
}

// Consumer loads.  Two nodes (local, local + 1 of the tile; both bulk fluid,
// off the periodic edges): plane q's window shift has the parity of s_q
// (window starts are even), so planes of even shift are read as one word.
template <class PL, class S, int PX, int PXY>
LBM_DEV void ring_load_pair(F2 (&v)[PL::P], const S *win, const int *shift, int local) {
    constexpr int CAP = ring_cap(2, (int)sizeof(S));
    int sh[PL::QF];
#pragma unroll
    for (int d = 0; d < PL::QF; ++d) sh[d] = shift[d] + local;
#pragma unroll
    for (int q = 0; q < PL::P; ++q) {
        const int par = (PL::ex(q) + PL::ey(q) * PX + PL::ez(q) * PXY) & 1;
        const S *e = win + q * CAP + sh[flow_dir<PL>(q)];
        if (par == 0) {
            const float2 w = PairMem<S>::lds(e);
            v[q] = F2(w.x, w.y);
        } else {
            v[q] = F2(Codec<S>::ld_shared(e), Codec<S>::ld_shared(e + 1));
        }
    }
}

// one node
template <class PL, class S>
LBM_DEV void ring_load_one(float (&p)[PL::P], const S *win, const int *shift, int local) {
    constexpr int CAP = ring_cap(1, (int)sizeof(S));
#pragma unroll
    for (int q = 0; q < PL::P; ++q) p[q] = Codec<S>::ld_shared(win + q * CAP + shift[flow_dir<PL>(q)] + local);
}

template <int DIM, int NC, bool HG, class S, int NPL, int MINB>
__global__ void __launch_bounds__(RING_THREADS, MINB) k_step_ring(const StepParams<float> prm, const BulkParams bp,
                                                                  const int ns) {
    using PL = Planes<DIM, NC, HG>;
    constexpr int P = PL::P;
    constexpr int CAP = ring_cap(NPL, (int)sizeof(S));
    static_assert(PL::QF <= RING_MAX_QF, "window shifts");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + RING_FULL);
    uint64_t *empty = reinterpret_cast<uint64_t *>(smem + RING_EMPTY);
    volatile int *abort_word = reinterpret_cast<volatile int *>(smem + RING_ABORT);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    advance_step_count(prm);
    if (threadIdx.x == 0) {
        for (int k = 0; k < ns; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], RING_CW);
        }
        *abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == RING_CW) {
        // ---------------------------------------------------------- producer
        // the block's tiles are k = 0, 1, ...: t = blockIdx.x + k gridDim.x.
        // Lane i holds the record of tile k = 32 b + i of the current batch b;
        // the case words of tile k + 1 are fetched while tile k is issued.
        const int ntile_blk = prm.ntiles > (int)blockIdx.x ? (prm.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
        auto batch = [&](int b) {
            const int kk = 32 * b + lane;
            return kk < ntile_blk ? prm.tiles[blockIdx.x + kk * gridDim.x] : make_int2(0, 0);
        };
        auto words = [&](int2 tl, int &wa, int &wb) {
            const int *cw = reinterpret_cast<const int *>(prm.cases + tl.x);
            wa = lane < RING_CW_WORDS ? cw[lane] : 0;
            wb = lane + 32 < RING_CW_WORDS ? cw[lane + 32] : 0;
        };
        int2 rec = batch(0);
        int2 tile = make_int2(__shfl_sync(0xffffffffu, rec.x, 0), __shfl_sync(0xffffffffu, rec.y, 0));
        int wa = 0, wb = 0;
        if (ntile_blk > 0) words(tile, wa, wb);
        int k = 0;
        bool ok = true;
        for (; k < ntile_blk; ++k) {
            // next tile's record and case words (their loads overlap the wait below)
            const int kn = k + 1;
            if ((kn & 31) == 0 && kn < ntile_blk) rec = batch(kn >> 5);
            const int2 tn = make_int2(__shfl_sync(0xffffffffu, rec.x, kn & 31), __shfl_sync(0xffffffffu, rec.y, kn & 31));
            int wan = 0, wbn = 0;
            if (kn < ntile_blk) words(tn, wan, wbn);
            const int st = k % ns;
            if (k >= ns && !ring_wait(&empty[st], (uint32_t)((k / ns) - 1) & 1u, abort_word)) {
                ok = false;
                break;
            }
            ring_issue<PL, S, NPL>(prm, tile, wa, wb, st, smem, ns);
            tile = tn;
            wa = wan;
            wb = wbn;
        }
        if (!ok && lane == 0) {
            if (!*abort_word) atomicExch(bp.err, 1);
            *abort_word = 1;
        }
        // the block stays resident until every copy it issued has landed
        if (lane == 0)
            for (int kk = k - 1; kk >= 0 && kk >= k - ns; --kk)
                for (uint32_t s = 0; s < BULK_SPIN_LIMIT && !mbar_try_wait(&full[kk % ns], (uint32_t)(kk / ns) & 1u);
                     ++s) {
                }
        return;
    }
    // -------------------------------------------------------------- consumers
    for (int k = 0;; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t >= prm.ntiles) break;
        const int st = k % ns;
        if (!ring_wait(&full[st], (uint32_t)(k / ns) & 1u, abort_word)) {
            if (lane == 0) {
                atomicExch(bp.err, 1);
                *abort_word = 1;
            }
            return;
        }
        // everything this warp needs from the stage goes to registers first;
        // the stage is released before the relaxation and the stores
        const unsigned char *meta = smem + RING_META + st * ring_meta_bytes(NPL);
        const int2 tile = *reinterpret_cast<const int2 *>(meta + RM_TILE);
        const CaseDev<float> c = *reinterpret_cast<const CaseDev<float> *>(meta + RM_CASE);
        const S *win = reinterpret_cast<const S *>(smem + ring_win_off(NPL, ns)) + (size_t)st * P * CAP;
        const int *shift = reinterpret_cast<const int *>(meta + RM_SHIFT);
        const uint8_t *flags = meta + RM_FLAGS;
        const int local = (warp * 32 + lane) * NPL;
        const int n0 = tile.y + local;
        uint8_t f0 = 0, f1 = 0;
        bool fast = false;
        if (n0 < c.N) {
            int x, y, z, r;
            coords<DIM, float>(c, n0, x, y, z, r);
            const bool yz_in = y >= 1 && y + 1 <= c.ny - 1 && (DIM == 2 || (z >= 1 && z + 1 <= c.nz - 1));
            f0 = flags[local];
            if constexpr (NPL == 2) {
                f1 = n0 + 1 < c.N ? flags[local + 1] : uint8_t(0);
                fast = f0 == NODE_FLUID && f1 == NODE_FLUID && yz_in && x >= 1 && x + 2 <= c.nx - 1;
            } else {
                fast = f0 == NODE_FLUID && yz_in && x >= 1 && x + 1 <= c.nx - 1;
            }
        }
        S *dst = static_cast<S *>(prm.dst) + c.pop_off;
        const int st32 = (int)c.stride;
        if constexpr (NPL == 2) {
            F2 v[P];
            if (fast) {
                const int px = c.nx & 1, pxy = (c.nx * c.ny) & 1;
                if (!px)
                    ring_load_pair<PL, S, 0, 0>(v, win, shift, local);
                else if (DIM == 2 || !pxy)
                    ring_load_pair<PL, S, 1, 0>(v, win, shift, local);
                else
                    ring_load_pair<PL, S, 1, 1>(v, win, shift, local);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            if (fast) {
                collide_v<PL, NC, HG, F2, float>(v, c);
                S *__restrict__ dp = dst + n0;
#pragma unroll
                for (int q = 0; q < P; ++q) PairMem<S>::st(dp + q * st32, v[q].v);
            } else {
                if (f0 == NODE_FLUID) step_node<DIM, NC, HG, S, 0>(prm, c, n0, 0, 0);
                if (f1 == NODE_FLUID) step_node<DIM, NC, HG, S, 0>(prm, c, n0 + 1, 0, 0);
            }
        } else {
            float p[P];
            if (fast) ring_load_one<PL, S>(p, win, shift, local);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
            if (fast) {
                collide<PL, NC, HG, float>(p, c);
                S *__restrict__ dp = dst + n0;
#pragma unroll
                for (int q = 0; q < P; ++q) Codec<S>::st(dp + q * st32, p[q]);
            } else if (f0 == NODE_FLUID) {
                step_node<DIM, NC, HG, S, 0>(prm, c, n0, 0, 0);
            }
        }
    }
}

}  // namespace lbm
