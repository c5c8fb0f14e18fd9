// Fused 2D red-black sweep fed by the tensor memory accelerator (TMA):
// tensor-map tile loads (cp.async.bulk.tensor) completing on an mbarrier,
// persistent blocks, two stages.
//
// Same tile algorithm and per-cell arithmetic as rbgs_fused2d_block (a whole
// sweep per launch: red cells of the tile and a one-cell ring from the staged
// x, then the tile's black cells, x -> xout).  Every operand the tile reads
// -- x with a 2-cell halo, the faces of both axes, bt and W -- arrives as one
// TMA box per array, requested by one thread; elements beyond the grid are
// filled with zeros by the TMA unit and never read.  Each block walks tiles
// with a grid stride and requests tile k+2 while it computes tile k.
//
// Boxes start two cells left of the tile (so the innermost coordinate, in
// scalars, is a multiple of 16 bytes) and are laid out densely in shared
// memory: element (i, j) of an array sits at row j - row0, column i - (i0 - 2).
// Row strides must be multiples of 16 bytes: always true in FP64; in FP32 the
// level needs an even n0, and the axis-0 faces (n0 + 1 per row) come from a
// copy with an even row pitch kept for this purpose.
//
// Waits on an mbarrier are bounded: after kAsyncSpinLimit polls the kernel
// sets bit 8 of *err, waits (bounded again) for its own loads still in flight,
// and returns; the host reports MG_ERR_TIMEOUT.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "mg_kernels.cuh"

namespace cmg {

constexpr int kAsyncStages = 2;
constexpr long long kAsyncSpinLimit = 1LL << 26;
constexpr int kErrAsyncTimeout = 8;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Tile loads of a 2D / 3D box at the given coordinates into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy ones (a stage is re-filled after it was read).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// The maps of one level and precision: x and xalt (a sweep reads one of them),
// axis-0 faces, axis-1 faces, bt, W.
struct TmaLevel {
    CUtensorMap x[2], g0, g1, bt, w;
};

// Staged boxes of one tile: 0 x, 1 axis-0 faces, 2 axis-1 faces, 3 bt, 4 W.
template <typename R, int TX, int TY>
struct TmaTile {
    using V2 = typename Vec<R>::v2;
    using Q4 = typename Vec<R>::q4;
    static constexpr int W2 = TX + 4;    // box width, cells (from i0 - 2)
    __host__ __device__ static constexpr int rows(int a) { return a == 0 ? TY + 4 : (a == 2 ? TY + 3 : TY + 2); }
    __host__ __device__ static constexpr int row0(int a) { return a == 0 ? -2 : -1; }
    __host__ __device__ static constexpr int esz(int a) { return a == 4 ? (int)sizeof(Q4) : (int)sizeof(V2); }
    __host__ __device__ static constexpr int bytes(int a) { return rows(a) * W2 * esz(a); }
    __host__ __device__ static constexpr int slot(int a) { return (bytes(a) + 127) / 128 * 128; }
    __host__ __device__ static constexpr int off(int a) { return a == 0 ? 0 : off(a - 1) + slot(a - 1); }
    static constexpr int stage_bytes = off(4) + slot(4);
    static constexpr int tx_bytes = bytes(0) + bytes(1) + bytes(2) + bytes(3) + bytes(4);
};

template <typename R, int TX, int TY>
constexpr int tma_smem_bytes() {
    return kAsyncStages * TmaTile<R, TX, TY>::stage_bytes + 128;   // + the barriers
}

// Requests tile (bx, by) into a stage (one thread).
template <typename R, int TX, int TY>
__device__ __forceinline__ void tma_issue(const CUtensorMap *mx, const CUtensorMap *mg0, const CUtensorMap *mg1,
                                          const CUtensorMap *mbt, const CUtensorMap *mw, int bx, int by,
                                          unsigned char *stage, uint64_t *bar) {
    using T = TmaTile<R, TX, TY>;
    const int i0 = bx * TX, j0 = by * TY;
    const int cx = 2 * (i0 - 2);                 // scalars: two per cell
    mbar_arrive_expect_tx(bar, (uint32_t)T::tx_bytes);
    tma_load_2d(stage + T::off(0), mx, cx, j0 - 2, bar);
    tma_load_2d(stage + T::off(1), mg0, cx, j0 - 1, bar);
    tma_load_2d(stage + T::off(2), mg1, cx, j0 - 1, bar);
    tma_load_2d(stage + T::off(3), mbt, cx, j0 - 1, bar);
    tma_load_3d(stage + T::off(4), mw, 0, i0 - 2, j0 - 1, bar);
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(256, 1)
    k_rbgs_fused2d_tma(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mg0,
                       const __grid_constant__ CUtensorMap mg1, const __grid_constant__ CUtensorMap mbt,
                       const __grid_constant__ CUtensorMap mw, const __grid_constant__ Level<R> L,
                       typename Vec<R>::v2 *__restrict__ xout, int *__restrict__ err) {
    pdl_entry();
    using T = TmaTile<R, TX, TY>;
    using V2 = typename Vec<R>::v2;
    using Q4 = typename Vec<R>::q4;
    constexpr int W2 = T::W2;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(tma_smem + kAsyncStages * T::stage_bytes);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int n0 = L.n0, n1 = L.n1;
    const int gx = (n0 + TX - 1) / TX, gy = (n1 + TY - 1) / TY;
    const int tiles = gx * gy;
    if (tid == 0) {
        for (int s = 0; s < kAsyncStages; s++) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
        for (int s = 0; s < kAsyncStages; s++) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < tiles) tma_issue<R, TX, TY>(&mx, &mg0, &mg1, &mbt, &mw, t % gx, t / gx, tma_smem + s * T::stage_bytes,
                                                &bars[s]);
        }
    }
    __syncthreads();
    bool failed = false;
    int k = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, k++) {
        const int s = k % kAsyncStages;
        const uint32_t parity = (uint32_t)((k / kAsyncStages) & 1);
        long long spins = 0;
        while (!mbar_try_wait(&bars[s], parity)) {
            if (++spins > kAsyncSpinLimit) { failed = true; break; }
        }
        if (__syncthreads_or(failed)) { failed = true; break; }
        unsigned char *stage = tma_smem + s * T::stage_bytes;
        V2 *xs = reinterpret_cast<V2 *>(stage + T::off(0));          // rows j0-2 .., in place for the red phase
        const V2 *g0 = reinterpret_cast<const V2 *>(stage + T::off(1));   // rows j0-1 ..
        const V2 *g1 = reinterpret_cast<const V2 *>(stage + T::off(2));   // face rows j0-1 ..
        const V2 *bts = reinterpret_cast<const V2 *>(stage + T::off(3));  // rows j0-1 ..
        const Q4 *ws = reinterpret_cast<const Q4 *>(stage + T::off(4));   // rows j0-1 ..
        const int bx = t % gx, by = t / gx;
        const int i0 = bx * TX, j0 = by * TY;
        // neighbour sums as offdiag_tile2d; (lx, ly) = (gi - i0 + 2, gj - j0 + 2)
        auto offd = [&](int gi, int gj, int lx, int ly, R &sT, R &sp) {
            sT = R(0);
            sp = R(0);
            const int rf = ly - 1;                                   // rows from j0 - 1
            if (gi > 0)      { V2 g = g0[rf * W2 + lx];     V2 u = xs[ly * W2 + lx - 1];   sT += g.x * u.x; sp += g.y * u.y; }
            if (gi < n0 - 1) { V2 g = g0[rf * W2 + lx + 1]; V2 u = xs[ly * W2 + lx + 1];   sT += g.x * u.x; sp += g.y * u.y; }
            if (gj > 0)      { V2 g = g1[rf * W2 + lx];     V2 u = xs[(ly - 1) * W2 + lx]; sT += g.x * u.x; sp += g.y * u.y; }
            if (gj < n1 - 1) { V2 g = g1[(rf + 1) * W2 + lx]; V2 u = xs[(ly + 1) * W2 + lx]; sT += g.x * u.x; sp += g.y * u.y; }
        };
        auto update = [&](int lx, int ly, R sT, R sp) -> V2 {
            const V2 bt = bts[(ly - 1) * W2 + lx];
            const Q4 W = ws[(ly - 1) * W2 + lx];
            return mk2<R>(bt.x - W.a * sT - W.b * sp, bt.y - W.c * sT - W.d * sp);
        };
        // red cells ((i + j) even) of the tile and its one-cell ring
        constexpr int kRedPerRow = (TX + 2) / 2;
        for (int q = tid; q < (TY + 2) * kRedPerRow; q += 256) {
            const int ry = q / kRedPerRow, rx = q - ry * kRedPerRow;
            const int gj = j0 - 1 + ry;
            const int gi = i0 - 1 + 2 * rx + ((i0 - 1 + gj) & 1);
            if (gi < 0 || gi >= n0 || gj < 0 || gj >= n1) continue;
            const int lx = gi - i0 + 2, ly = gj - j0 + 2;
            R sT, sp;
            offd(gi, gj, lx, ly, sT, sp);
            xs[ly * W2 + lx] = update(lx, ly, sT, sp);
        }
        __syncthreads();
        // black cells of the tile, one per thread (no warp mixes colours), in place
        constexpr int kBlackPerRow = TX / 2;
        for (int q = tid; q < TY * kBlackPerRow; q += 256) {
            const int ty = q / kBlackPerRow, rx = q - ty * kBlackPerRow;
            const int gj = j0 + ty;
            const int gi = i0 + 2 * rx + ((i0 + gj + 1) & 1);
            if (gi >= n0 || gj >= n1) continue;
            const int lx = gi - i0 + 2, ly = ty + 2;
            R sT, sp;
            offd(gi, gj, lx, ly, sT, sp);
            xs[ly * W2 + lx] = update(lx, ly, sT, sp);
        }
        __syncthreads();
        // the tile, both colours, coalesced
        for (int q = tid; q < TY * TX; q += 256) {
            const int ty = q / TX, tx = q - ty * TX;
            const int gi = i0 + tx, gj = j0 + ty;
            if (gi < n0 && gj < n1) xout[(long long)gj * n0 + gi] = xs[(ty + 2) * W2 + tx + 2];
        }
        __syncthreads();                      // every thread is done with stage s
        const int tn = t + kAsyncStages * gridDim.x;
        if (tid == 0 && tn < tiles) {
            fence_proxy_async_smem();
            tma_issue<R, TX, TY>(&mx, &mg0, &mg1, &mbt, &mw, tn % gx, tn / gx, stage, &bars[s]);
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(err, kErrAsyncTimeout);
        // wait, bounded, for this block's loads still in flight before leaving
        for (int s = 0; s < kAsyncStages; s++) {
            const int kk = k + s;
            long long spins = 0;
            while (!mbar_try_wait(&bars[kk % kAsyncStages], (uint32_t)((kk / kAsyncStages) & 1)) &&
                   ++spins < kAsyncSpinLimit) {
            }
        }
    }
}

}  // namespace cmg
