// CUDA kernels of the coupled p-T multigrid: set-up, smoothing, residual,
// restriction, prolongation, coarsest solve, norms.  Templated on the real
// type R (double: FP64 path and the FP64 side of mixed precision; float: the
// inner cycles of mixed precision) and on the dimension.
//
// The system each level holds is described in mg_types.cuh.
#pragma once
#include <cooperative_groups.h>

#include "mg_types.cuh"

namespace cmg {

constexpr int kBX = 32;   // block shape of the 2D/3D cell kernels
constexpr int kBY = 8;
constexpr int kReduceThreads = 256;

template <typename R> __device__ __forceinline__ typename Vec<R>::v2 mk2(R a, R b);
template <> __device__ __forceinline__ double2 mk2<double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 mk2<float>(float a, float b) { return make_float2(a, b); }

template <typename V> __device__ __forceinline__ V ldg2(const V *p) { return __ldg(p); }
// Loads of data that a kernel may itself have written in an earlier stage (the
// cluster tail): NC = false reads through L2 (coherent), NC = true through the
// read-only path.
template <bool NC, typename V> __device__ __forceinline__ V ldv(const V *p) { return NC ? __ldg(p) : __ldcg(p); }

__device__ __forceinline__ void block_coords(int local, int gx, int gy, int &bx, int &by, int &bz) {
    bx = local % gx;
    by = (local / gx) % gy;
    bz = local / (gx * gy);
}

// Tiles of a (gx, gy, gz) geometry.  P false: the launch grid is that
// geometry, a block per tile (no index arithmetic before the loads).  P true,
// a persistent launch: the grid is one wave (SMs x resident blocks per SM, at
// most the number of tiles) and each block walks the tiles with a grid
// stride, so no partial last wave leaves SMs idle.
#define CMG_TILES(P, gx, gy, gz, body)                                                     \
    do {                                                                                 \
        if (!(P)) {                                                                      \
            const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;                 \
            body;                                                                        \
        } else {                                                                         \
            const int tiles_ = (gx) * (gy) * (gz);                                       \
            for (int v_ = blockIdx.x; v_ < tiles_; v_ += gridDim.x) {                    \
                int bx, by, bz;                                                          \
                block_coords(v_, (gx), (gy), bx, by, bz);                                \
                body;                                                                    \
            }                                                                            \
        }                                                                                \
    } while (0)
__device__ __forceinline__ dq ldgq(const dq *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 u = __ldg(q), v = __ldg(q + 1);
    return dq{u.x, u.y, v.x, v.y};
}
__device__ __forceinline__ fq ldgq(const fq *p) {
    float4 u = __ldg(reinterpret_cast<const float4 *>(p));
    return fq{u.x, u.y, u.z, u.w};
}

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  A kernel
// of a cycle launched with the programmatic-serialisation attribute is set up
// while the kernel before it in the stream drains: its blocks are scheduled
// as that kernel's last blocks exit, and pdl_entry() (griddepcontrol.wait)
// returns once that kernel has completed and its writes are visible.  Every
// such kernel calls it before it reads or writes anything.  Launched without
// the attribute it returns at once.  No kernel triggers its dependents early
// (griddepcontrol.launch_dependents): blocks of the next grid scheduled while
// this one still runs land on the SMs that free first, and small FP64 grids
// packed onto a few SMs' FP64 pipes made the FP64 step 4% slower.
__device__ __forceinline__ void pdl_entry() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }


// Off-diagonal part of the two rows: sT = sum over interior faces of G^T_f T_nb,
// sp = sum of G^p_f p_nb + l4 * sT (the p-row's T-Laplacian term, Eq. 28).
// Neighbours beyond the grid contribute nothing (homogeneous boundary values;
// inhomogeneous Dirichlet data are folded into the right-hand side).
template <typename R, int DIM, bool WITH_L4 = true, bool NC = true>
__device__ __forceinline__ void offdiag(const Level<R> &L, const typename Vec<R>::v2 *__restrict__ x,
                                        int i, int j, int k, long long c, R &sT, R &sp) {
    using V2 = typename Vec<R>::v2;
    const int n0 = L.n0, n1 = L.n1;
    sT = R(0);
    sp = R(0);
    const long long f0 = (long long)i + (long long)(n0 + 1) * ((long long)j + (long long)n1 * k);
    if (i > 0)      { V2 g = ldg2(L.G0 + f0);     V2 u = ldv<NC>(x + c - 1);  sT += g.x * u.x; sp += g.y * u.y; }
    if (i < n0 - 1) { V2 g = ldg2(L.G0 + f0 + 1); V2 u = ldv<NC>(x + c + 1);  sT += g.x * u.x; sp += g.y * u.y; }
    const long long f1 = (long long)i + (long long)n0 * ((long long)j + (long long)(n1 + 1) * k);
    if (j > 0)      { V2 g = ldg2(L.G1 + f1);      V2 u = ldv<NC>(x + c - n0); sT += g.x * u.x; sp += g.y * u.y; }
    if (j < n1 - 1) { V2 g = ldg2(L.G1 + f1 + n0); V2 u = ldv<NC>(x + c + n0); sT += g.x * u.x; sp += g.y * u.y; }
    if (DIM == 3) {
        const long long pl = (long long)n0 * n1;
        if (k > 0)        { V2 g = ldg2(L.G2 + c);      V2 u = ldv<NC>(x + c - pl); sT += g.x * u.x; sp += g.y * u.y; }
        if (k < L.n2 - 1) { V2 g = ldg2(L.G2 + c + pl); V2 u = ldv<NC>(x + c + pl); sT += g.x * u.x; sp += g.y * u.y; }
    }
    if (WITH_L4) sp += __ldg(L.l4 + c) * sT;
}

// Gauss-Seidel update of one cell from its plain neighbour sums.  In the FP32
// cycles a cell next to a large coefficient jump (its FP32 W marked with a NaN
// first entry at set-up) applies its 2x2 block in FP64 instead: the FP64 W
// and Dinv b of the same level, the neighbour sums promoted.
template <typename R>
__device__ __noinline__ typename Vec<R>::v2 gs_update_fp64(const Level<R> &L, long long c, R sT, R sp) {
    const dq W = ldgq(L.W64 + c);
    const double2 bt = __ldcg(L.bt64 + c);
    const double t = (double)sT, p = (double)sp;
    return mk2<R>((R)(bt.x - W.a * t - W.b * p), (R)(bt.y - W.c * t - W.d * p));
}

template <typename R, bool NC = true>
__device__ __forceinline__ typename Vec<R>::v2 gs_update(const Level<R> &L, long long c, R sT, R sp) {
    const auto bt = ldv<NC>(L.bt + c);
    const auto W = ldgq(L.W + c);
    if (sizeof(R) == 4 && W.a != W.a) return gs_update_fp64<R>(L, c, sT, sp);
    return mk2<R>(bt.x - W.a * sT - W.b * sp, bt.y - W.c * sT - W.d * sp);
}

// ---------------------------------------------------------------------------
// Smoothing: one colour of a red-black block Gauss-Seidel sweep.  Each thread
// owns one cell of the colour (red: i+j+k even) and solves its two rows for
// (T_i, p_i):  x_i = Dinv_i (b_i - offdiag_i) = bt_i - W_i (sT, sp).
// Neighbours are of the other colour and are not written by this launch.
// ---------------------------------------------------------------------------
// The work of thread block (bx, by, bz) of the launch geometry
// (ceil(ceil(n0/2)/32), ceil(n1/8), n2); shared with the batched kernels.
template <typename R, int DIM, bool NC = true>
__device__ __forceinline__ void rbgs_colour_block(const Level<R> &L, int colour, int bx, int by, int bz) {
    using V2 = typename Vec<R>::v2;
    const int j = by * kBY + threadIdx.y;
    const int k = DIM == 3 ? bz : 0;
    if (j >= L.n1) return;
    const int par = (j + k + colour) & 1;
    const int i = 2 * (bx * kBX + (int)threadIdx.x) + par;
    if (i >= L.n0) return;
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    R sT, sp;
    offdiag<R, DIM, false, NC>(L, L.x, i, j, k, c, sT, sp);
    L.x[c] = gs_update<R, NC>(L, c, sT, sp);
}

// Two rows per thread (rows j and j + 8 of a 32 x 16 block of colour cells):
// both updates are formed before either is stored, so their loads overlap,
// and half as many blocks make a launch (a grid whose block count would leave
// a partial last wave can then fit one wave).  Same per-cell arithmetic.
template <typename R, int DIM>
__global__ void __launch_bounds__(kBX * kBY, 7) k_rbgs_colour2(Level<R> L, int colour) {
    pdl_entry();
    using V2 = typename Vec<R>::v2;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    V2 out[2];
    long long cid[2];
    bool ok[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int j = (int)blockIdx.y * 2 * kBY + r * kBY + (int)threadIdx.y;
        const int par = (j + k + colour) & 1;
        const int i = 2 * ((int)blockIdx.x * kBX + (int)threadIdx.x) + par;
        ok[r] = j < L.n1 && i < L.n0;
        cid[r] = cell_id(i, j, k, L.n0, L.n1);
        if (ok[r]) {
            R sT, sp;
            offdiag<R, DIM, false>(L, L.x, i, j, k, cid[r], sT, sp);
            out[r] = gs_update<R>(L, cid[r], sT, sp);
        }
    }
#pragma unroll
    for (int r = 0; r < 2; r++)
        if (ok[r]) L.x[cid[r]] = out[r];
}

template <typename R, int DIM, bool P>
__global__ void __launch_bounds__(kBX * kBY, 8) k_rbgs_colour(Level<R> L, int colour) {
    pdl_entry();
    CMG_TILES(P, ((L.n0 + 1) / 2 + kBX - 1) / kBX, (L.n1 + kBY - 1) / kBY, DIM == 3 ? L.n2 : 1,
              (rbgs_colour_block<R, DIM>(L, colour, bx, by, bz)));
}


// ---------------------------------------------------------------------------
// The stop test of a solve run as one graph (mg_solve_async): the V-cycles
// repeat inside a WHILE graph node whose condition this one-thread kernel
// sets.  init: the initial norms n0 (norms[0..1]), no cycle yet; otherwise a
// cycle has run and norms holds its norms.  The rule is mg_solve's: stop when
// both fields fell by rtol (rtol <= 0: never), or at the start when both
// initial norms are zero; the loop ends at max_it cycles whatever the norms
// (so a non-finite norm still ends it).
// ---------------------------------------------------------------------------
struct AsyncStat {
    double n0[2], nk[2];
    int it;        // cycles (outer steps) run
    int ok;        // the stop test was met
};

__device__ __forceinline__ bool async_converged(const double n0[2], const double nk[2], double rtol) {
    if (!(rtol > 0.0)) return false;
    for (int f = 0; f < 2; f++) {
        const double q = n0[f] > 0.0 ? nk[f] / n0[f] : 0.0;
        if (!(q <= rtol)) return false;
    }
    return true;
}

__global__ void k_async_stop(const double *__restrict__ norms, AsyncStat *__restrict__ st, int max_it, double rtol,
                             cudaGraphConditionalHandle cond, int init) {
    pdl_entry();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool ok;
    if (init) {
        st->n0[0] = st->nk[0] = norms[0];
        st->n0[1] = st->nk[1] = norms[1];
        st->it = 0;
        ok = async_converged(st->n0, st->nk, rtol) || (st->n0[0] == 0.0 && st->n0[1] == 0.0);
    } else {
        st->it += 1;
        st->nk[0] = norms[0];
        st->nk[1] = norms[1];
        ok = async_converged(st->n0, st->nk, rtol);
    }
    st->ok = ok ? 1 : 0;
    cudaGraphSetConditional(cond, (!ok && st->it < max_it) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Weighted block Jacobi (the other smoother): every cell solves its two rows
// against the previous iterate xin, z_i = bt_i - W_i (sT, sp) with sT, sp the
// neighbour sums of xin, and moves a fraction omega of the way:
// xout_i = xin_i + omega (z_i - xin_i).  xin and xout are distinct buffers.
// ---------------------------------------------------------------------------
template <typename R, int DIM>
__device__ __forceinline__ void wjac_block(const Level<R> &L, const typename Vec<R>::v2 *__restrict__ xin,
                                           typename Vec<R>::v2 *__restrict__ xout, R omega, int bx, int by, int bz) {
    const int i = bx * kBX + (int)threadIdx.x;
    const int j = by * kBY + (int)threadIdx.y;
    const int k = DIM == 3 ? bz : 0;
    if (i >= L.n0 || j >= L.n1) return;
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    R sT, sp;
    offdiag<R, DIM, false>(L, xin, i, j, k, c, sT, sp);
    const auto z = gs_update<R>(L, c, sT, sp);
    const auto xo = ldg2(xin + c);
    xout[c] = mk2<R>(xo.x + omega * (z.x - xo.x), xo.y + omega * (z.y - xo.y));
}

template <typename R, int DIM, bool P>
__global__ void __launch_bounds__(kBX * kBY, 8) k_wjac(Level<R> L, const typename Vec<R>::v2 *__restrict__ xin,
                                                      typename Vec<R>::v2 *__restrict__ xout, R omega) {
    pdl_entry();
    CMG_TILES(P, (L.n0 + kBX - 1) / kBX, (L.n1 + kBY - 1) / kBY, DIM == 3 ? L.n2 : 1,
              (wjac_block<R, DIM>(L, xin, xout, omega, bx, by, bz)));
}

// ---------------------------------------------------------------------------
// Fused 2D sweep: one launch does a whole red-black sweep (red, then black)
// from xin to xout.  A CTA owns a TX x TY tile.  It stages xin with a
// halo of 2 in shared memory, updates the red cells of the tile and of a
// one-cell ring around it (the ring's red values are what the tile's black
// cells see; neighbouring CTAs compute the same values), then the tile's
// black cells, and writes the tile.  Reading xin and writing xout (distinct
// buffers) keeps CTAs from seeing each other's updates.  Same arithmetic as
// two k_rbgs_colour launches.
// ---------------------------------------------------------------------------
constexpr int kFTX = 64, kFTY = 16;   // tile of the batched kernels and the default

// Tile shapes a handle can select per level (index = mg_tuning tile value).
constexpr int kTileShapes = 3;
constexpr int kTileX[kTileShapes] = {64, 32, 32};
constexpr int kTileY[kTileShapes] = {16, 16, 8};

template <typename R, int TX>
__device__ __forceinline__ void offdiag_tile2d(const Level<R> &L, const typename Vec<R>::v2 (*xs)[TX + 4], int lx,
                                               int ly, int i, int j, long long c, R &sT, R &sp) {
    using V2 = typename Vec<R>::v2;
    const int n0 = L.n0, n1 = L.n1;
    sT = R(0);
    sp = R(0);
    const long long f0 = (long long)i + (long long)(n0 + 1) * j;
    if (i > 0)      { V2 g = ldg2(L.G0 + f0);     V2 u = xs[ly][lx - 1]; sT += g.x * u.x; sp += g.y * u.y; }
    if (i < n0 - 1) { V2 g = ldg2(L.G0 + f0 + 1); V2 u = xs[ly][lx + 1]; sT += g.x * u.x; sp += g.y * u.y; }
    const long long f1 = (long long)i + (long long)n0 * j;
    if (j > 0)      { V2 g = ldg2(L.G1 + f1);      V2 u = xs[ly - 1][lx]; sT += g.x * u.x; sp += g.y * u.y; }
    if (j < n1 - 1) { V2 g = ldg2(L.G1 + f1 + n0); V2 u = xs[ly + 1][lx]; sT += g.x * u.x; sp += g.y * u.y; }
}

// Tile (bx, by) of the launch geometry (ceil(n0/TX), ceil(n1/TY)); shared with
// the batched kernels (which call it repeatedly: it starts with a barrier so
// the previous tile's readers are done with the shared stage).
template <typename R, int TX = kFTX, int TY = kFTY>
__device__ __forceinline__ void rbgs_fused2d_block(const Level<R> &L, const typename Vec<R>::v2 *__restrict__ xin,
                                                   typename Vec<R>::v2 *__restrict__ xout, int bx, int by) {
    using V2 = typename Vec<R>::v2;
    __shared__ V2 xs[TY + 4][TX + 4];
    const int n0 = L.n0, n1 = L.n1;
    const int i0 = bx * TX, j0 = by * TY;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    __syncthreads();
    // stage xin, halo 2 (cells beyond the grid are never read)
    for (int q = tid; q < (TY + 4) * (TX + 4); q += 256) {
        const int ly = q / (TX + 4), lx = q - ly * (TX + 4);
        const int gi = i0 + lx - 2, gj = j0 + ly - 2;
        if (gi >= 0 && gi < n0 && gj >= 0 && gj < n1) xs[ly][lx] = ldg2(xin + (long long)gj * n0 + gi);
    }
    __syncthreads();
    // red cells ((i + j) even) of the tile and its one-cell ring
    constexpr int kRedPerRow = (TX + 2) / 2;
    for (int q = tid; q < (TY + 2) * kRedPerRow; q += 256) {
        const int ry = q / kRedPerRow, rx = q - ry * kRedPerRow;
        const int gj = j0 - 1 + ry;
        const int gi = i0 - 1 + 2 * rx + ((i0 - 1 + gj) & 1);
        if (gi < 0 || gi >= n0 || gj < 0 || gj >= n1) continue;
        const int lx = gi - i0 + 2, ly = gj - j0 + 2;
        const long long c = (long long)gj * n0 + gi;
        R sT, sp;
        offdiag_tile2d<R, TX>(L, xs, lx, ly, gi, gj, c, sT, sp);
        xs[ly][lx] = gs_update<R>(L, c, sT, sp);
    }
    __syncthreads();
    // black cells of the tile, one per thread (a warp never mixes colours, so
    // no FP64 issue slot goes to a predicated-off lane); in place in xs, where
    // black cells read only red values
    constexpr int kBlackPerRow = TX / 2;
    for (int q = tid; q < TY * kBlackPerRow; q += 256) {
        const int ty = q / kBlackPerRow, rx = q - ty * kBlackPerRow;
        const int gj = j0 + ty;
        const int gi = i0 + 2 * rx + ((i0 + gj + 1) & 1);
        if (gi >= n0 || gj >= n1) continue;
        const int lx = gi - i0 + 2, ly = ty + 2;
        const long long c = (long long)gj * n0 + gi;
        R sT, sp;
        offdiag_tile2d<R, TX>(L, xs, lx, ly, gi, gj, c, sT, sp);
        xs[ly][lx] = gs_update<R>(L, c, sT, sp);
    }
    __syncthreads();
    // the tile, both colours, coalesced
    for (int q = tid; q < TY * TX; q += 256) {
        const int ty = q / TX, tx = q - ty * TX;
        const int gi = i0 + tx, gj = j0 + ty;
        if (gi < n0 && gj < n1) xout[(long long)gj * n0 + gi] = xs[ty + 2][tx + 2];
    }
}

// FP32: 8 resident blocks per SM (at most 32 registers): the sweep is bound by
// memory latency, so occupancy is what feeds it.  FP64: 4.
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 8 : 4)
    k_rbgs_fused2d(Level<R> L, const typename Vec<R>::v2 *__restrict__ xin, typename Vec<R>::v2 *__restrict__ xout) {
    pdl_entry();
    rbgs_fused2d_block<R, TX, TY>(L, xin, xout, blockIdx.x, blockIdx.y);
}

// Two red-black sweeps on one tile (temporal blocking): x staged with a halo
// of 4, then the red cells of the tile and a 3-cell ring, the black cells of
// a 2-cell ring, the red cells of a 1-cell ring, the black cells of the tile.
// Each phase reads only values the phase before it left in its ring (or the
// staged x), so every cell of the tile ends as after two full sweeps, with
// the same update in the same order: the result is the other kernels' bit
// for bit.  Faces, W and bt of the ring are read once from DRAM and the
// second time from L1; xin -> xout.
template <typename R, int TX, int TY>
__device__ __forceinline__ void rbgs_fused2d_x2_block(const Level<R> &L, const typename Vec<R>::v2 *__restrict__ xin,
                                                      typename Vec<R>::v2 *__restrict__ xout, int bx, int by) {
    using V2 = typename Vec<R>::v2;
    constexpr int H = 4, SX = TX + 2 * H, SY = TY + 2 * H;
    __shared__ V2 xs[SY][SX];
    const int n0 = L.n0, n1 = L.n1;
    const int i0 = bx * TX, j0 = by * TY;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    for (int q = tid; q < SY * SX; q += 256) {
        const int ly = q / SX, lx = q - ly * SX;
        const int gi = i0 + lx - H, gj = j0 + ly - H;
        if (gi >= 0 && gi < n0 && gj >= 0 && gj < n1) xs[ly][lx] = ldg2(xin + (long long)gj * n0 + gi);
    }
    __syncthreads();
    // phase p = 0..3: colour (p even: red), ring width 3 - p
#pragma unroll 1
    for (int p = 0; p < 4; p++) {
        const int ring = 3 - p, par = p & 1;            // par 0: red ((i + j) even), 1: black
        const int w = TX + 2 * ring, hgt = TY + 2 * ring;
        const int per_row = w / 2;                      // TX even: each row holds w / 2 cells of a colour
        for (int q = tid; q < hgt * per_row; q += 256) {
            const int ry = q / per_row, rx = q - ry * per_row;
            const int gj = j0 - ring + ry;
            const int gi = i0 - ring + 2 * rx + ((i0 - ring + gj + par) & 1);
            if (gi < 0 || gi >= n0 || gj < 0 || gj >= n1) continue;
            const int lx = gi - i0 + H, ly = gj - j0 + H;
            const long long c = (long long)gj * n0 + gi;
            R sT, sp;
            offdiag_tile2d<R, SX - 4>(L, xs, lx, ly, gi, gj, c, sT, sp);
            xs[ly][lx] = gs_update<R>(L, c, sT, sp);
        }
        __syncthreads();
    }
    for (int q = tid; q < TY * TX; q += 256) {
        const int ty = q / TX, tx = q - ty * TX;
        const int gi = i0 + tx, gj = j0 + ty;
        if (gi < n0 && gj < n1) xout[(long long)gj * n0 + gi] = xs[ty + H][tx + H];
    }
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 4)
    k_rbgs_fused2d_x2(Level<R> L, const typename Vec<R>::v2 *__restrict__ xin, typename Vec<R>::v2 *__restrict__ xout) {
    pdl_entry();
    rbgs_fused2d_x2_block<R, TX, TY>(L, xin, xout, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Residual of the children, restricted: coarse b = mean of the 2^DIM
// children's residuals (plain mean in the row-scaled form = volume-weighted
// mean of the physical residuals).  Also zeroes the coarse initial guess.
//
// RED: the fine level has just ended a red-black sweep, whose second colour
// (black, i+j+k odd) solved its 2x2 blocks against the final red values, so
// the black residuals vanish (in exact arithmetic; computed, they are
// rounding noise of b - A x) and only the red children (even child index
// popcount) are evaluated.
// ---------------------------------------------------------------------------
template <typename R, int DIM, bool NC = true, bool RED = false>
__device__ __forceinline__ void residual_restrict_block(const Level<R> &F, const Level<R> &C, int bx, int by, int bz) {
    using V2 = typename Vec<R>::v2;
    const int I = bx * kBX + threadIdx.x;
    const int J = by * kBY + threadIdx.y;
    const int K = DIM == 3 ? bz : 0;
    if (I >= C.n0 || J >= C.n1) return;
    R aT = R(0), ap = R(0);
#pragma unroll
    for (int q = 0; q < (1 << DIM); q++) {
        if (RED && (__popc(q) & 1)) continue;
        const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = DIM == 3 ? 2 * K + (q >> 2) : 0;
        const long long c = cell_id(i, j, k, F.n0, F.n1);
        R sT, sp;
        offdiag<R, DIM, true, NC>(F, F.x, i, j, k, c, sT, sp);
        const V2 bb = ldv<NC>(F.b + c), xx = ldv<NC>(F.x + c);
        const auto Dd = ldgq(F.D + c);
        const R rT = ((bb.x - sT) - Dd.a * xx.x) - Dd.b * xx.y;   // two FMAs per row
        const R rp = ((bb.y - sp) - Dd.c * xx.x) - Dd.d * xx.y;
        // the sums start from child 0 (always evaluated): no FP64 addition to 0
        aT = q == 0 ? rT : aT + rT;
        ap = q == 0 ? rp : ap + rp;
    }
    const R w = R(1) / R(1 << DIM);
    const long long cc = cell_id(I, J, K, C.n0, C.n1);
    const R bT = aT * w, bp = ap * w;
    C.b[cc] = mk2<R>(bT, bp);
    const auto Di = ldgq(C.Dinv + cc);
    C.bt[cc] = mk2<R>(Di.a * bT + Di.b * bp, Di.c * bT + Di.d * bp);
    C.x[cc] = mk2<R>(R(0), R(0));
}

template <typename R, int DIM, bool RED, bool P>
__global__ void __launch_bounds__(kBX * kBY) k_residual_restrict(Level<R> F, Level<R> C) {
    pdl_entry();
    CMG_TILES(P, (C.n0 + kBX - 1) / kBX, (C.n1 + kBY - 1) / kBY, DIM == 3 ? C.n2 : 1,
              (residual_restrict_block<R, DIM, true, RED>(F, C, bx, by, bz)));
}

// ---------------------------------------------------------------------------
// Prolongation and correction: fine x += cell-centred bi/tri-linear
// interpolation of the coarse correction (weight 3/4 towards the parent and
// 1/4 towards the next coarse cell per axis).  Beyond the grid the ghost
// reflects the parent: same value at walls and the axis, opposite sign at
// Dirichlet faces (the correction vanishes there).
// ---------------------------------------------------------------------------
template <typename R, int DIM, bool NC = true>
__device__ __forceinline__ void prolong_add_block(const Level<R> &C, const Level<R> &F, const BcFlags &bc, int bx,
                                                  int by, int bz) {
    using V2 = typename Vec<R>::v2;
    const int i = bx * kBX + threadIdx.x;
    const int j = by * kBY + threadIdx.y;
    const int k = DIM == 3 ? bz : 0;
    if (i >= F.n0 || j >= F.n1) return;
    const int P[3] = {i >> 1, j >> 1, k >> 1};
    const int s[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
    const int nC[3] = {C.n0, C.n1, C.n2};
    // neighbour index per axis; `neg` marks a ghost beyond a Dirichlet face
    int Qn[3];
    bool neg[3];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int t = P[a] + s[a];
        if (t < 0)           { Qn[a] = P[a]; neg[a] = bc.dir[a][0] != 0; }
        else if (t >= nC[a]) { Qn[a] = P[a]; neg[a] = bc.dir[a][1] != 0; }
        else                 { Qn[a] = t;    neg[a] = false; }
    }
    // per-axis weights 3/4 (parent) and 1/4 (neighbour); products are exact
    // constants, signs are applied by selection, not arithmetic
    R aT = R(0), ap = R(0);
#pragma unroll
    for (int q = 0; q < (1 << DIM); q++) {
        int Q[3] = {P[0], P[1], DIM == 3 ? P[2] : 0};
        bool flip = false;
        int nq = 0;
#pragma unroll
        for (int a = 0; a < DIM; a++)
            if ((q >> a) & 1) { Q[a] = Qn[a]; flip ^= neg[a]; nq++; }
        const R w = DIM == 2 ? (nq == 0 ? R(9.0 / 16) : nq == 1 ? R(3.0 / 16) : R(1.0 / 16))
                             : (nq == 0 ? R(27.0 / 64) : nq == 1 ? R(9.0 / 64) : nq == 2 ? R(3.0 / 64) : R(1.0 / 64));
        const V2 e = ldv<NC>(C.x + cell_id(Q[0], Q[1], Q[2], C.n0, C.n1));
        const R ws = flip ? -w : w;   // the ghost's sign goes on the constant weight: no FP64 negations
        aT += ws * e.x;
        ap += ws * e.y;
    }
    const long long c = cell_id(i, j, k, F.n0, F.n1);
    V2 xv = NC ? F.x[c] : __ldcg(F.x + c);
    xv.x += aT;
    xv.y += ap;
    F.x[c] = xv;
}

template <typename R, int DIM, bool P>
__global__ void __launch_bounds__(kBX * kBY) k_prolong_add(Level<R> C, Level<R> F, BcFlags bc) {
    pdl_entry();
    CMG_TILES(P, (F.n0 + kBX - 1) / kBX, (F.n1 + kBY - 1) / kBY, DIM == 3 ? F.n2 : 1,
              (prolong_add_block<R, DIM>(C, F, bc, bx, by, bz)));
}

// ---------------------------------------------------------------------------
// Coarsest level: x = Minv b with the dense inverse of the level's matrix
// (unknown order: (T, p) per cell).  One warp per row, fixed summation order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_coarse_matvec(const R *__restrict__ Minv, const R *__restrict__ b, R *__restrict__ x, int n) {
    pdl_entry();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const R *row = Minv + (long long)warp * n;
    R acc = R(0);
    for (int c = lane; c < n; c += 32) acc += row[c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) x[warp] = acc;
}

// ---------------------------------------------------------------------------
// Norms.  Per cell z = Dinv (b - offdiag(x)) - x = Dinv r: the block-Jacobi
// scaled residual, invariant under the row scaling.  Each block writes its
// partial sums of z_T^2 and z_p^2; k_reduce_norms sums them in a fixed order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_sum2(double &a, double &b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    __shared__ double sa[32], sb[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, w = tid >> 5;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = (nthr + 31) >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Last-block completion: after a block stored its partial, the block that
// draws the final ticket sums all partials in index order (deterministic),
// writes sqrt of the two sums to out and re-arms the ticket counter.
__device__ __forceinline__ void finish_norms(double2 *partial, int nblocks, unsigned int *ticket, double *out) {
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthr = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)nblocks - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int q = tid; q < nblocks; q += nthr) {
        const double2 v = __ldcg(partial + q);
        a += v.x;
        b += v.y;
    }
    block_sum2(a, b);
    if (tid == 0) {
        out[0] = sqrt(a);
        out[1] = sqrt(b);
        *ticket = 0u;
    }
}

// Norm and FP64-residual tiles cover 64 x 32 cells (x, y) of one z-plane,
// eight per thread (four rows unrolled, for loads in flight).  The solo
// kernels run one persistent wave: each thread
// accumulates the squares of all its tiles' cells with FMAs and the block
// reduces once, so the FP64 reduction tree (shuffles, then one warp) is spread
// over many cells; on a part with few FP64 units per SM it would otherwise
// cost as much as the cells themselves.  (The batched kernels reduce per tile.)
constexpr int kNormCols = 64;
constexpr int kNormRows = 4;   // rows per thread: the tile spans kBY * kNormRows rows
__host__ __device__ __forceinline__ int norm_gx(int n0) { return (n0 + kNormCols - 1) / kNormCols; }
__host__ __device__ __forceinline__ int norm_gy(int n1) { return (n1 + kBY * kNormRows - 1) / (kBY * kNormRows); }

template <int DIM>
__device__ __forceinline__ void norm_cell(const Level<double> &L, int i, int j, int k, double &zT2, double &zp2) {
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    double sT, sp;
    offdiag<double, DIM, false>(L, L.x, i, j, k, c, sT, sp);
    const double2 xx = ldg2(L.x + c);
    const double2 u = gs_update<double>(L, c, sT, sp);   // = Dinv (b - offdiag)
    const double zT = u.x - xx.x;
    const double zp = u.y - xx.y;
    zT2 = fma(zT, zT, zT2);
    zp2 = fma(zp, zp, zp2);
}

// Sums of (Dinv r)_T^2 and (Dinv r)_p^2 over tile (bx, by, bz) of the norm
// grid (ceil(n0/64), ceil(n1/32), n2), added to zT2, zp2 (norm_block: reduced
// over the block, valid in thread 0).
//
// RED: x has just come out of a red-black sweep, so the block residual of
// the black cells is exactly zero (z = gs_update - x recomputes the very
// update that produced x, bit for bit) and each thread visits the one red
// cell of its column pair per row.
template <int DIM, bool RED = false>
__device__ __forceinline__ void norm_tile(const Level<double> &L, int bx, int by, int bz, double &zT2, double &zp2) {
    const int k = DIM == 3 ? bz : 0;
#pragma unroll
    for (int r = 0; r < kNormRows; r++) {
        const int j = (by * kNormRows + r) * kBY + threadIdx.y;
        if (j >= L.n1) continue;
        if (RED) {
            const int i = bx * kNormCols + 2 * threadIdx.x + ((j + k) & 1);
            if (i < L.n0) norm_cell<DIM>(L, i, j, k, zT2, zp2);
        } else {
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int i = bx * kNormCols + e * kBX + threadIdx.x;
                if (i < L.n0) norm_cell<DIM>(L, i, j, k, zT2, zp2);
            }
        }
    }
}

template <int DIM, bool RED = false>
__device__ __forceinline__ double2 norm_block(const Level<double> &L, int bx, int by, int bz) {
    double zT2 = 0.0, zp2 = 0.0;
    norm_tile<DIM, RED>(L, bx, by, bz, zT2, zp2);
    block_sum2(zT2, zp2);
    return make_double2(zT2, zp2);
}

template <int DIM, bool RED, bool P>
__global__ void __launch_bounds__(kBX * kBY) k_norm_partials(Level<double> L, double2 *__restrict__ partial,
                                                           unsigned int *__restrict__ ticket, double *__restrict__ out) {
    pdl_entry();
    double zT2 = 0.0, zp2 = 0.0;     // a block's tiles accumulate, then one reduction
    CMG_TILES(P, norm_gx(L.n0), norm_gy(L.n1), DIM == 3 ? L.n2 : 1, (norm_tile<DIM, RED>(L, bx, by, bz, zT2, zp2)));
    block_sum2(zT2, zp2);
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blk] = make_double2(zT2, zp2);
    finish_norms(partial, gridDim.x * gridDim.y * gridDim.z, ticket, out);
}

// FP64 residual of the finest level for mixed precision: r = b - A x is
// written (rounded) as the FP32 right-hand side of the correction problem,
// the FP32 correction is zeroed, and the norm partials of Dinv r are formed.
template <int DIM>
__device__ __forceinline__ void residual64_to32_cell(const Level<double> &L, float2 *__restrict__ b32,
                                                     float2 *__restrict__ bt32, float2 *__restrict__ e32,
                                                     double2 *__restrict__ r_out, double2 *__restrict__ r_out2, int i,
                                                     int j, int k, double &zT2, double &zp2) {
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    double sT, sp;
    offdiag<double, DIM>(L, L.x, i, j, k, c, sT, sp);
    const double2 bb = ldg2(L.b + c), xx = ldg2(L.x + c);
    const dq Dd = ldgq(L.D + c);
    const dq Di = ldgq(L.Dinv + c);
    const double rT = ((bb.x - sT) - Dd.a * xx.x) - Dd.b * xx.y;   // two FMAs per row
    const double rp = ((bb.y - sp) - Dd.c * xx.x) - Dd.d * xx.y;
    const double zT = Di.a * rT + Di.b * rp;
    const double zp = Di.c * rT + Di.d * rp;
    zT2 = fma(zT, zT, zT2);
    zp2 = fma(zp, zp, zp2);
    b32[c] = make_float2((float)rT, (float)rp);
    bt32[c] = make_float2((float)zT, (float)zp);     // Dinv r for the FP32 sweeps
    if (L.jflag && L.jflag[c]) L.bt[c] = make_double2(zT, zp);   // and in FP64 where they apply the block in FP64
    e32[c] = make_float2(0.f, 0.f);
    if (r_out) {                                     // the initial residual of the defect correction:
        r_out[c] = make_double2(rT, rp);             // r0 over b (only this thread reads b[c], before this store),
        r_out2[c] = make_double2(0.0, 0.0);          // and the correction starts at zero
    }
}

// Block (bx, by, bz) of the norm grid.
template <int DIM>
__device__ __forceinline__ void residual64_to32_tile(const Level<double> &L, float2 *__restrict__ b32,
                                                     float2 *__restrict__ bt32, float2 *__restrict__ e32,
                                                     double2 *__restrict__ r_out, double2 *__restrict__ r_out2, int bx,
                                                     int by, int bz, double &zT2, double &zp2) {
    const int k = DIM == 3 ? bz : 0;
#pragma unroll
    for (int r = 0; r < kNormRows; r++) {
        const int j = (by * kNormRows + r) * kBY + threadIdx.y;
        if (j >= L.n1) continue;
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int i = bx * kNormCols + e * kBX + threadIdx.x;
            if (i < L.n0) residual64_to32_cell<DIM>(L, b32, bt32, e32, r_out, r_out2, i, j, k, zT2, zp2);
        }
    }
}

template <int DIM>
__device__ __forceinline__ double2 residual64_to32_block(const Level<double> &L, float2 *__restrict__ b32,
                                                         float2 *__restrict__ bt32, float2 *__restrict__ e32,
                                                         double2 *__restrict__ r_out, double2 *__restrict__ r_out2, int bx,
                                                         int by, int bz) {
    double zT2 = 0.0, zp2 = 0.0;
    residual64_to32_tile<DIM>(L, b32, bt32, e32, r_out, r_out2, bx, by, bz, zT2, zp2);
    block_sum2(zT2, zp2);
    return make_double2(zT2, zp2);
}

template <int DIM, bool P>
__global__ void __launch_bounds__(kBX * kBY) k_residual64_to32(Level<double> L, float2 *__restrict__ b32,
                                                             float2 *__restrict__ bt32, float2 *__restrict__ e32,
                                                             double2 *__restrict__ r_out,
                                                             double2 *__restrict__ r_out2,
                                                             double2 *__restrict__ partial,
                                                             unsigned int *__restrict__ ticket,
                                                             double *__restrict__ out) {
    pdl_entry();
    double zT2 = 0.0, zp2 = 0.0;
    CMG_TILES(P, norm_gx(L.n0), norm_gy(L.n1), DIM == 3 ? L.n2 : 1,
              (residual64_to32_tile<DIM>(L, b32, bt32, e32, r_out, r_out2, bx, by, bz, zT2, zp2)));
    block_sum2(zT2, zp2);
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x == 0 && threadIdx.y == 0) partial[blk] = make_double2(zT2, zp2);
    finish_norms(partial, gridDim.x * gridDim.y * gridDim.z, ticket, out);
}

// x += delta: the solution from the initial guess and the accumulated correction
__global__ void k_add_pairs(double2 *__restrict__ x, const double2 *__restrict__ delta, long long N) {
    pdl_entry();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double2 a = x[c], d = delta[c];
        x[c] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// x64 += e32 (the refinement update; mixed solves pass the correction delta as x64)
__global__ void k_add_correction(double2 *__restrict__ x, const float2 *__restrict__ e, long long N) {
    pdl_entry();
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float2 d = e[c];
        double2 v = x[c];
        v.x += (double)d.x;
        v.y += (double)d.y;
        x[c] = v;
    }
}

// Sums the partials in a fixed order; out[0..1] = sqrt of the sums.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_norms(const double2 *__restrict__ partial, int n,
                                                                 double *__restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        a += partial[q].x;
        b += partial[q].y;
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        out[0] = sqrt(a);
        out[1] = sqrt(b);
    }
}

// ---------------------------------------------------------------------------
// Finest-level right-hand side: b0 = s_i (lambda_T, lambda_p) minus the
// Dirichlet boundary data of the rows.
// ---------------------------------------------------------------------------
struct BcVals {
    int dir[3][2];
    double T[3][2], p[3][2];
};

// Dirichlet data of a boundary cell's rows: G^T g_T and G^p g_p + l4 G^T g_T.
// Called for cells on the grid's boundary only, as a real call: its
// conditional FP64 products would otherwise be issued (predicated off) for
// every interior cell too, and FP64 issue slots are this part's scarce unit.
template <int DIM>
__device__ __noinline__ double2 boundary_rows(const Level<double> &L, const BcVals &bv, int i, int j, int k) {
    const int n0 = L.n0, n1 = L.n1;
    double gT = 0.0, gp = 0.0;
    const long long f0 = (long long)i + (long long)(n0 + 1) * ((long long)j + (long long)n1 * k);
    if (i == 0 && bv.dir[0][0])      { double2 g = L.G0[f0];     gT += g.x * bv.T[0][0]; gp += g.y * bv.p[0][0]; }
    if (i == n0 - 1 && bv.dir[0][1]) { double2 g = L.G0[f0 + 1]; gT += g.x * bv.T[0][1]; gp += g.y * bv.p[0][1]; }
    const long long f1 = (long long)i + (long long)n0 * ((long long)j + (long long)(n1 + 1) * k);
    if (j == 0 && bv.dir[1][0])      { double2 g = L.G1[f1];      gT += g.x * bv.T[1][0]; gp += g.y * bv.p[1][0]; }
    if (j == n1 - 1 && bv.dir[1][1]) { double2 g = L.G1[f1 + n0]; gT += g.x * bv.T[1][1]; gp += g.y * bv.p[1][1]; }
    if (DIM == 3) {
        const long long c = cell_id(i, j, k, n0, n1), pl = (long long)n0 * n1;
        if (k == 0 && bv.dir[2][0])        { double2 g = L.G2[c];      gT += g.x * bv.T[2][0]; gp += g.y * bv.p[2][0]; }
        if (k == L.n2 - 1 && bv.dir[2][1]) { double2 g = L.G2[c + pl]; gT += g.x * bv.T[2][1]; gp += g.y * bv.p[2][1]; }
    }
    gp += L.l4[cell_id(i, j, k, n0, n1)] * gT;
    return make_double2(gT, gp);
}

template <int DIM>
__device__ __forceinline__ bool on_boundary(const Level<double> &L, int i, int j, int k) {
    return i == 0 || i == L.n0 - 1 || j == 0 || j == L.n1 - 1 || (DIM == 3 && (k == 0 || k == L.n2 - 1));
}

// Block (bx, by, bz) of the cell grid; xin (may be NULL) is also copied into L.x.
// AXI: the rows carry the factor s_i = r_i (else 1, with no arithmetic).
template <int DIM, bool AXI>
__device__ __forceinline__ void prep_rhs_cells(const Level<double> &L, const double2 *__restrict__ rhs,
                                               const double2 *__restrict__ xin, const BcVals &bv, double r0,
                                               double h, int bx, int by, int bz) {
    const int i = bx * kBX + threadIdx.x;
    const int j = by * kBY + threadIdx.y;
    const int k = DIM == 3 ? bz : 0;
    if (i >= L.n0 || j >= L.n1) return;
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    const double2 q = rhs[c];
    double bT = q.x, bp = q.y;
    if (AXI) {
        const double s = r0 + (i + 0.5) * h;
        bT = s * q.x;
        bp = s * q.y;
    }
    if (on_boundary<DIM>(L, i, j, k)) {
        const double2 g = boundary_rows<DIM>(L, bv, i, j, k);
        bT -= g.x;
        bp -= g.y;
    }
    L.b[c] = make_double2(bT, bp);
    const dq Di = ldgq(L.Dinv + c);
    L.bt[c] = make_double2(Di.a * bT + Di.b * bp, Di.c * bT + Di.d * bp);
    if (xin) L.x[c] = xin[c];
}

template <int DIM>
__device__ __forceinline__ void prep_rhs_block(const Level<double> &L, const double2 *__restrict__ rhs,
                                               const double2 *__restrict__ xin, const BcVals &bv, int axisym,
                                               double r0, double h, int bx, int by, int bz) {
    if (axisym) prep_rhs_cells<DIM, true>(L, rhs, xin, bv, r0, h, bx, by, bz);
    else prep_rhs_cells<DIM, false>(L, rhs, xin, bv, r0, h, bx, by, bz);
}

template <int DIM>
__global__ void __launch_bounds__(kBX * kBY) k_prep_rhs(const __grid_constant__ Level<double> L,
                                                      const double2 *__restrict__ rhs, const __grid_constant__ BcVals bv,
                                                      int axisym, double r0, double h) {
    pdl_entry();
    CMG_TILES(false, (L.n0 + kBX - 1) / kBX, (L.n1 + kBY - 1) / kBY, DIM == 3 ? L.n2 : 1,
              (prep_rhs_block<DIM>(L, rhs, nullptr, bv, axisym, r0, h, bx, by, bz)));
}

// y = L(x) (Eqs. 27-28): offdiag + boundary data + D x is s_i times the rows.
template <int DIM>
__global__ void __launch_bounds__(kBX * kBY) k_apply_paper(const __grid_constant__ Level<double> L,
                                                         const __grid_constant__ BcVals bv, int axisym, double r0,
                                                         double h, double2 *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= L.n0 || j >= L.n1) return;
    const long long c = cell_id(i, j, k, L.n0, L.n1);
    double sT, sp, gT = 0.0, gp = 0.0;
    offdiag<double, DIM>(L, L.x, i, j, k, c, sT, sp);
    if (on_boundary<DIM>(L, i, j, k)) {
        const double2 g = boundary_rows<DIM>(L, bv, i, j, k);
        gT = g.x;
        gp = g.y;
    }
    const double2 xx = L.x[c];
    const dq Dd = L.D[c];
    const double s = axisym ? r0 + (i + 0.5) * h : 1.0;
    y[c] = make_double2((sT + gT + Dd.a * xx.x + Dd.b * xx.y) / s, (sp + gp + Dd.c * xx.x + Dd.d * xx.y) / s);
}

// ---------------------------------------------------------------------------
// Set-up kernels (FP64).  One launch per level: the finest level from the
// caller's arrays, every coarser level from the level below.  Each cell
// computes all 2*DIM of its face coefficients (a face shared by two cells is
// computed identically by both) and stores the faces it owns: its low faces,
// and its high faces on the high boundary.  It then forms its 2x2 block D and
// the inverse.  The scaled local terms S = s [[l1, l2], [0, l3]] are kept per
// level for the next coarsening.
// ---------------------------------------------------------------------------
struct SetupOut {                 // one level's outputs
    double2 *G[3];
    dq *S, *D, *Dinv, *W;
    double *l4;
    float2 *G32[3];               // FP32 copies (mixed precision), or NULL
    fq *D32, *Dinv32, *W32;
    float *l432;
    float2 *G0p;                  // 2D mixed: FP32 axis-0 faces again, row pitch p0 (even), or NULL
    int p0, n0;
    // finest level of mixed precision with jump marking on: per-cell mark,
    // count of marked cells, and the face-coefficient ratio that marks a cell
    unsigned char *jflag;
    int *jcount;
    double jratio;
};

struct SetupGeom {
    int n[3];
    int axisym;
    double r0, h;                 // this level's spacing
    double ih2;                   // 1 / h^2 (finest level)
    double fac[3][2];             // boundary factor per axis / side: 2 Dirichlet, 0 wall/axis
};

// Finite test on the bit pattern (integer pipe, not the scarce FP64 pipe).
__device__ __forceinline__ bool finite_bits(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

template <int DIM>
__device__ __forceinline__ void finish_cell(const SetupOut &o, long long c, const long long fid[3][2], int own[3][2],
                                            const double2 g[3][2], dq S, double l4, int *err) {
    double sT = g[0][0].x, sp = g[0][0].y;   // face sums (the faces are finite and >= 0)
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            if (a | sd) {
                sT += g[a][sd].x;
                sp += g[a][sd].y;
            }
            if (own[a][sd]) {
                o.G[a][fid[a][sd]] = g[a][sd];
                if (o.G32[a]) o.G32[a][fid[a][sd]] = make_float2((float)g[a][sd].x, (float)g[a][sd].y);
                if (a == 0 && o.G0p) {
                    const long long f = fid[0][sd], row = f / (o.n0 + 1);
                    o.G0p[f - row * (o.n0 + 1) + row * o.p0] = make_float2((float)g[0][sd].x, (float)g[0][sd].y);
                }
            }
        }
    o.S[c] = S;
    o.l4[c] = l4;
    dq D{S.a - sT, S.b, S.c - l4 * sT, S.d - sp};
    const double det = D.a * D.d - D.b * D.c;
    if ((__double_as_longlong(det) & 0x7fffffffffffffffLL) == 0 || !finite_bits(det)) atomicOr(err, 2);
    const double id = 1.0 / det;
    const dq Di{D.d * id, -D.b * id, -D.c * id, D.a * id};
    const dq Wc{Di.a + Di.b * l4, Di.b, Di.c + Di.d * l4, Di.d};
    o.D[c] = D;
    o.Dinv[c] = Di;
    o.W[c] = Wc;
    if (o.D32) {
        o.D32[c] = fq{(float)D.a, (float)D.b, (float)D.c, (float)D.d};
        o.Dinv32[c] = fq{(float)Di.a, (float)Di.b, (float)Di.c, (float)Di.d};
        o.W32[c] = fq{(float)Wc.a, (float)Wc.b, (float)Wc.c, (float)Wc.d};
        o.l432[c] = (float)l4;
    }
}

__device__ __forceinline__ void face_ids(const int n[3], int i, int j, int k, long long fid[3][2]) {
    const long long f0 = (long long)i + (long long)(n[0] + 1) * ((long long)j + (long long)n[1] * k);
    const long long f1 = (long long)i + (long long)n[0] * ((long long)j + (long long)(n[1] + 1) * k);
    const long long f2 = (long long)i + (long long)n[0] * ((long long)j + (long long)n[1] * k);
    fid[0][0] = f0; fid[0][1] = f0 + 1;
    fid[1][0] = f1; fid[1][1] = f1 + n[0];
    fid[2][0] = f2; fid[2][1] = f2 + (long long)n[0] * n[1];
}

// The caller's coefficient arrays of one problem.
struct SetupIn {
    const double *lam;            // [N][4]
    const double *fa[3], *fk[3];  // 1/rho and k on the faces of each axis
};

// Finest level from lambda [N][4] and the per-axis arrays of 1/rho and k:
// block (bx, by, bz) of the cell grid (ceil(n0/32), ceil(n1/8), n2).
// AXI: faces carry r_f and the rows s_i = r_i; boundary faces (rare, a
// separate branch) carry the boundary factor.
template <int DIM, bool AXI>
__device__ __forceinline__ void setup_fine_cells(const SetupGeom &gm, const SetupIn &in, const SetupOut &o, int *err,
                                                 int bx, int by, int bz) {
    const int i = bx * kBX + threadIdx.x;
    const int j = by * kBY + threadIdx.y;
    const int k = DIM == 3 ? bz : 0;
    if (i >= gm.n[0] || j >= gm.n[1]) return;
    const double *lam = in.lam;
    const long long c = cell_id(i, j, k, gm.n[0], gm.n[1]);
    const double l1 = lam[4 * c], l2 = lam[4 * c + 1], l3 = lam[4 * c + 2], l4 = lam[4 * c + 3];
    bool bad = !finite_bits(l1) || !finite_bits(l2) || !finite_bits(l3) || !finite_bits(l4);
    const double s = AXI ? gm.r0 + (i + 0.5) * gm.h : 1.0;
    const double ih2 = gm.ih2;
    const double *const *fa = in.fa, *const *fk = in.fk;
    const int pos[3] = {i, j, k};
    long long fid[3][2];
    face_ids(gm.n, i, j, k, fid);
    int own[3][2];
    double2 g[3][2];
    double kf[3][2], af[3][2], wf[3][2];
    bool edge = false;
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            const int fpos = pos[a] + sd;
            // w = rho_f / h^2 (times r_f or r_i on axisymmetric grids)
            double w = ih2;
            if (AXI) w *= (a == 0 ? gm.r0 + (i + sd) * gm.h : s);
            const double al = fa[a][fid[a][sd]], kk = fk[a][fid[a][sd]];
            bad = bad || !finite_bits(al) || !finite_bits(kk);
            kf[a][sd] = kk;
            af[a][sd] = al;
            wf[a][sd] = w;
            g[a][sd] = make_double2(kk * w, al * w);
            own[a][sd] = sd == 0 || fpos == gm.n[a];
            edge = edge || fpos == 0 || fpos == gm.n[a];
        }
    if (edge) {
        // boundary faces: w times the factor (2 Dirichlet, 0 wall / axis)
#pragma unroll
        for (int a = 0; a < DIM; a++)
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int fpos = pos[a] + sd;
                if (fpos == 0 || fpos == gm.n[a]) {
                    const double w = wf[a][sd] * (fpos == 0 ? gm.fac[a][0] : gm.fac[a][1]);
                    g[a][sd] = make_double2(kf[a][sd] * w, af[a][sd] * w);
                }
            }
    }
    if (bad) atomicOr(err, 1);
    const dq S = AXI ? dq{s * l1, s * l2, 0.0, s * l3} : dq{l1, l2, 0.0, l3};
    finish_cell<DIM>(o, c, fid, own, g, S, l4, err);
    if (o.jflag) {
        // a coefficient jump at this cell: its interior faces' k or 1/rho
        // differ by more than the ratio; its 2x2 block is then applied in FP64
        // by the FP32 cycles (marked by a NaN first entry of its FP32 W)
        double kmin = 0.0, kmax = 0.0, amin = 0.0, amax = 0.0;
        bool any = false;
#pragma unroll
        for (int a = 0; a < DIM; a++)
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int fpos = pos[a] + sd;
                if (fpos == 0 || fpos == gm.n[a]) continue;
                const double kk = kf[a][sd], al = af[a][sd];
                kmin = any ? fmin(kmin, kk) : kk;
                kmax = any ? fmax(kmax, kk) : kk;
                amin = any ? fmin(amin, al) : al;
                amax = any ? fmax(amax, al) : al;
                any = true;
            }
        const bool jump = any && (kmax > o.jratio * kmin || amax > o.jratio * amin);
        o.jflag[c] = jump ? 1 : 0;
        if (jump) {
            reinterpret_cast<float *>(o.W32 + c)[0] = __int_as_float(0x7fc00000);
            atomicAdd(o.jcount, 1);
        }
    }
}

template <int DIM>
__device__ __forceinline__ void setup_fine_block(const SetupGeom &gm, const SetupIn &in, const SetupOut &o, int *err,
                                                 int bx, int by, int bz) {
    if (gm.axisym) setup_fine_cells<DIM, true>(gm, in, o, err, bx, by, bz);
    else setup_fine_cells<DIM, false>(gm, in, o, err, bx, by, bz);
}

template <int DIM>
__global__ void __launch_bounds__(kBX * kBY) k_setup_fine(SetupGeom gm, SetupIn in, SetupOut o, int *__restrict__ err) {
    pdl_entry();
    CMG_TILES(false, (gm.n[0] + kBX - 1) / kBX, (gm.n[1] + kBY - 1) / kBY, DIM == 3 ? gm.n[2] : 1,
              (setup_fine_block<DIM>(gm, in, o, err, bx, by, bz)));
}

// Coarse level from the level below: S = mean of the children's S, l4 the
// volume-weighted mean of theirs, each face the sum of its 2^(DIM-1) fine
// faces / 2^(DIM+1) (area-weighted mean coefficient re-discretised at 2h).
// The level below, as the coarsening reads it.
struct SetupFine {
    int n0, n1;
    const dq *S;
    const double *l4;
    const double2 *G[3];
    double h;
};

template <int DIM, bool AXI>
__device__ __forceinline__ void setup_coarse_cells(const SetupGeom &cg, const SetupFine &F, const SetupOut &o,
                                                   int *err, int bx, int by, int bz) {
    const int I = bx * kBX + threadIdx.x;
    const int J = by * kBY + threadIdx.y;
    const int K = DIM == 3 ? bz : 0;
    if (I >= cg.n[0] || J >= cg.n[1]) return;
    const int fn0 = F.n0, fn1 = F.n1;
    const dq *Sf = F.S;
    const double *l4f = F.l4;
    const double hf = F.h;
    const long long cc = cell_id(I, J, K, cg.n[0], cg.n[1]);
    // S = s [[l1, l2], [0, l3]] on every level: its lower-left entry is zero
    // by construction and is neither summed nor scaled
    double a0 = 0, a1 = 0, a3 = 0, v4 = 0, vs = 0;
#pragma unroll
    for (int q = 0; q < (1 << DIM); q++) {
        const int i = 2 * I + (q & 1);
        const long long f = cell_id(i, 2 * J + ((q >> 1) & 1), DIM == 3 ? 2 * K + (q >> 2) : 0, fn0, fn1);
        const dq sf = Sf[f];
        // sums start from the first child: an addition to 0.0 would still take an FP64 issue slot
        if (q == 0) { a0 = sf.a; a1 = sf.b; a3 = sf.d; }
        else { a0 += sf.a; a1 += sf.b; a3 += sf.d; }
        if (AXI) {
            const double sc = cg.r0 + (i + 0.5) * hf;
            if (q == 0) { v4 = sc * l4f[f]; vs = sc; }
            else { v4 += sc * l4f[f]; vs += sc; }
        } else {
            v4 = q == 0 ? l4f[f] : v4 + l4f[f];
        }
    }
    const double wb = 1.0 / (1 << DIM);
    const dq S{a0 * wb, a1 * wb, 0.0, a3 * wb};
    const double l4 = AXI ? v4 / vs : v4 * wb;   // volume-weighted mean (a power-of-two mean is exact as a product)
    const int P[3] = {I, J, K};
    const int fm[3][2] = {{fn0 + 1, fn1}, {fn0, fn1 + 1}, {fn0, fn1}};   // fine face array dims (x, y) per axis
    const double2 *const *Gf = F.G;
    long long fid[3][2];
    face_ids(cg.n, I, J, K, fid);
    int own[3][2];
    double2 g[3][2];
    const double wf = 1.0 / (1 << (DIM + 1));
#pragma unroll
    for (int a = 0; a < DIM; a++)
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            double sT = 0.0, sp = 0.0;
#pragma unroll
            for (int q = 0; q < (1 << (DIM - 1)); q++) {
                int off[3] = {0, 0, 0}, bit = 0;
#pragma unroll
                for (int b = 0; b < DIM; b++) {
                    if (b == a) continue;
                    off[b] = (q >> bit) & 1;
                    bit++;
                }
                int fpos[3];
#pragma unroll
                for (int b = 0; b < 3; b++) fpos[b] = (b == a) ? 2 * (P[b] + sd) : 2 * P[b] + off[b];
                if (DIM == 2) fpos[2] = 0;
                const double2 v = Gf[a][(long long)fpos[0] + (long long)fm[a][0] * ((long long)fpos[1] +
                                                                                  (long long)fm[a][1] * fpos[2])];
                if (q == 0) { sT = v.x; sp = v.y; }
                else { sT += v.x; sp += v.y; }
            }
            g[a][sd] = make_double2(sT * wf, sp * wf);
            own[a][sd] = sd == 0 || P[a] + sd == cg.n[a];
        }
    finish_cell<DIM>(o, cc, fid, own, g, S, l4, err);
}

template <int DIM>
__device__ __forceinline__ void setup_coarse_block(const SetupGeom &cg, const SetupFine &F, const SetupOut &o,
                                                   int *err, int bx, int by, int bz) {
    if (cg.axisym) setup_coarse_cells<DIM, true>(cg, F, o, err, bx, by, bz);
    else setup_coarse_cells<DIM, false>(cg, F, o, err, bx, by, bz);
}

template <int DIM>
__global__ void __launch_bounds__(kBX * kBY) k_setup_coarse(SetupGeom cg, SetupFine F, SetupOut o,
                                                          int *__restrict__ err) {
    pdl_entry();
    CMG_TILES(false, (cg.n[0] + kBX - 1) / kBX, (cg.n[1] + kBY - 1) / kBY, DIM == 3 ? cg.n[2] : 1,
              (setup_coarse_block<DIM>(cg, F, o, err, bx, by, bz)));
}

// FP32 copy of an FP64 array (the coarsest inverse of mixed precision).
__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

// Dense matrix of the coarsest level (M zeroed beforehand): rows 2c, 2c+1
// hold D_c on the diagonal block; on a neighbour, G^T in the T-row, G^p and
// l4 G^T in the p-row.
template <int DIM>
__global__ void k_coarse_assemble(int n0, int n1, int n2, const double2 *__restrict__ G0,
                                  const double2 *__restrict__ G1, const double2 *__restrict__ G2,
                                  const dq *__restrict__ D, const double *__restrict__ l4, double *__restrict__ M) {
    pdl_entry();
    const long long N = (long long)n0 * n1 * n2;
    const long long n = 2 * N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % n0), j = (int)((c / n0) % n1), k = (int)(c / ((long long)n0 * n1));
        const dq d = D[c];
        M[(2 * c) * n + 2 * c] = d.a;
        M[(2 * c) * n + 2 * c + 1] = d.b;
        M[(2 * c + 1) * n + 2 * c] = d.c;
        M[(2 * c + 1) * n + 2 * c + 1] = d.d;
        const long long f0 = (long long)i + (long long)(n0 + 1) * ((long long)j + (long long)n1 * k);
        const long long f1 = (long long)i + (long long)n0 * ((long long)j + (long long)(n1 + 1) * k);
        const double w4 = l4[c];
        auto put = [&](long long nb, double2 g) {
            M[(2 * c) * n + 2 * nb] = g.x;
            M[(2 * c + 1) * n + 2 * nb] = w4 * g.x;
            M[(2 * c + 1) * n + 2 * nb + 1] = g.y;
        };
        if (i > 0) put(c - 1, G0[f0]);
        if (i < n0 - 1) put(c + 1, G0[f0 + 1]);
        if (j > 0) put(c - n0, G1[f1]);
        if (j < n1 - 1) put(c + n0, G1[f1 + n0]);
        if (DIM == 3) {
            const long long pl = (long long)n0 * n1;
            if (k > 0) put(c - pl, G2[c]);
            if (k < n2 - 1) put(c + pl, G2[c + pl]);
        }
    }
}

// Coarsest inverse for n <= kBandSmemMax in two kernels.  GB300's FP64 pipe
// issues one warp instruction per 16 clocks per SM and single chains of FP64
// work are latency-bound, so both kernels spread each step over a block:
//
// k_band_lu_warp: one block, the matrix in shared memory.  The banded LU with
//   partial pivoting of k_band_lu below (the pivot chosen by comparing |a| as
//   integers: the bit patterns of non-negative doubles order like the values,
//   lowest row on ties), factors written back to M, piv[k], dinv[k] = 1/u_kk.
// k_band_inv_cols_warp: one block per 32 columns, one column j of the inverse
//   per lane and row groups on threadIdx.y: L U x = P e_j with the vectors in
//   shared memory (column-interleaved) and the factors read as broadcasts;
//   writes Minv (and Minv32).
constexpr int kBandSmemMax = 128;

__device__ __forceinline__ long long abs_bits(double v) {
    return __double_as_longlong(v) & 0x7fffffffffffffffLL;
}

// One block of kLUThreads threads, the matrix in shared memory.
constexpr int kLUThreads = 256;

__device__ __forceinline__ void band_lu_warp_block(double *__restrict__ M, int n, int kl, int ku,
                                                   int *__restrict__ piv, double *__restrict__ dinv,
                                                   int *__restrict__ err) {
    extern __shared__ double a[];
    __shared__ int prow, bad;
    __shared__ double pinv;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5;
    for (int q = tid; q < n * n; q += nthr) a[q] = M[q];
    if (tid == 0) bad = 0;
    __syncthreads();
    const int ur = kl + ku;
    const long long kInfBits = 0x7ff0000000000000LL;
    int k = 0;
    for (; k < n; k++) {
        const int rlast = min(n - 1, k + kl), clast = min(n - 1, k + ur);
        if (warp == 0) {
            long long best = -1;
            int br = k;
            for (int r = k + lane; r <= rlast; r += 32) {
                const long long v = abs_bits(a[r * n + k]);
                if (v > best) { best = v; br = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
                const int orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ov > best || (ov == best && orr < br)) { best = ov; br = orr; }
            }
            if (lane == 0) {
                if (best <= 0 || best >= kInfBits) bad = 1;   // zero, infinite or NaN pivot
                else {
                    prow = br;
                    piv[k] = br;
                    pinv = 1.0 / a[br * n + k];
                    dinv[k] = pinv;
                }
            }
        }
        __syncthreads();
        if (bad) break;
        const int p = prow;
        if (p != k)
            for (int c = k + tid; c <= clast; c += nthr) {
                const double t = a[k * n + c];
                a[k * n + c] = a[p * n + c];
                a[p * n + c] = t;
            }
        __syncthreads();
        const double ip = pinv;
        for (int r = k + 1 + tid; r <= rlast; r += nthr) a[r * n + k] *= ip;
        __syncthreads();
        const int w = clast - k, rows = rlast - k;
        for (int q = tid; q < rows * w; q += nthr) {
            const int r = k + 1 + q / w, c = k + 1 + q % w;
            const double l = a[r * n + k];
            if (abs_bits(l) != 0) a[r * n + c] -= l * a[k * n + c];
        }
        __syncthreads();
    }
    if (bad) {
        // leave an identity permutation behind so that no later reader
        // indexes out of range, then report
        for (int q = k + tid; q < n; q += nthr) {
            piv[q] = q;
            dinv[q] = 0.0;
        }
        if (tid == 0) atomicOr(err, 4);
        return;
    }
    for (int q = tid; q < n * n; q += nthr) M[q] = a[q];
}

__global__ void __launch_bounds__(kLUThreads) k_band_lu_warp(double *__restrict__ M, int n, int kl, int ku,
                                                             int *__restrict__ piv, double *__restrict__ dinv,
                                                             int *__restrict__ err) {
    band_lu_warp_block(M, n, kl, ku, piv, dinv, err);
}

// Columns 32 * col_block + lane of the inverse from the factors of
// k_band_lu_warp, one column per lane and kInvRows row groups (threadIdx.y)
// per column; does nothing when the factorisation reported a zero pivot.
// The factors' band is staged in shared memory first: the substitutions are
// 2n dependent steps, and a global load in each (a column of M, one sector
// per row) would put an L2 round trip on every step.
constexpr int kInvRows = 8;

// Shared-memory layout of the staged factors: a band of width kl + ku + kl + 1
// (row r holds columns r - kl .. r + kl + ku, U's reach after pivoting), or the
// dense matrix where the band would be at least as wide.
__host__ __device__ __forceinline__ int inv_band_width(int n, int kl, int ku) {
    const int bw = kl + (kl + ku) + 1;
    return bw >= n ? n : bw;
}

// Dynamic shared memory of band_inv_cols_warp_block, in doubles.
__host__ __device__ __forceinline__ long long inv_smem_doubles(int n, int kl, int ku) {
    return 32LL * n + 32LL * kInvRows + (long long)n * inv_band_width(n, kl, ku);
}

__device__ __forceinline__ void band_inv_cols_warp_block(const double *__restrict__ M, const int *__restrict__ piv,
                                                         const double *__restrict__ dinv, int n, int kl, int ku,
                                                         double *__restrict__ Minv, float *__restrict__ Minv32,
                                                         int col_block, const int *__restrict__ err) {
    extern __shared__ double ysm[];   // y[i][lane], n x 32; partial sums kInvRows x 32; the staged factors
    if (*(volatile const int *)err & 4) return;
    double *part = ysm + n * 32;
    double *fac = part + kInvRows * 32;
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = lane + 32 * ty;
    const int j = col_block * 32 + lane;
    const int bw = inv_band_width(n, kl, ku);
    const bool dense = bw == n;
    // factor entry (r, c), c within r - kl .. r + kl + ku
    auto F = [&](int r, int c) -> double { return dense ? fac[r * n + c] : fac[r * bw + (c - r + kl)]; };
    for (int q = tid; q < n * bw; q += 32 * kInvRows) {
        const int r = q / bw, o = q - r * bw;
        const int c = dense ? o : r - kl + o;
        fac[q] = (c >= 0 && c < n) ? __ldg(M + (long long)r * n + c) : 0.0;
    }
    for (int i = ty; i < n; i += kInvRows) ysm[i * 32 + lane] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < n; k++) {                      // P and L, in the factorisation's order
        const int p = min(max(__ldg(piv + k), k), n - 1);
        if (p != k && ty == 0) {
            const double t = ysm[k * 32 + lane];
            ysm[k * 32 + lane] = ysm[p * 32 + lane];
            ysm[p * 32 + lane] = t;
        }
        __syncthreads();
        const double yk = ysm[k * 32 + lane];
        const int rlast = min(n - 1, k + kl);
        for (int r = k + 1 + ty; r <= rlast; r += kInvRows) {
            const double l = F(r, k);
            if (abs_bits(l) != 0) ysm[r * 32 + lane] -= l * yk;
        }
        __syncthreads();
    }
    const int ur = kl + ku;
    for (int i = n - 1; i >= 0; i--) {                 // U
        const int clast = min(n - 1, i + ur);
        double s = 0.0;
        for (int c = i + 1 + ty; c <= clast; c += kInvRows) {
            const double u = F(i, c);
            if (abs_bits(u) != 0) s += u * ysm[c * 32 + lane];
        }
        part[ty * 32 + lane] = s;
        __syncthreads();
        if (ty == 0) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < kInvRows; q++) t += part[q * 32 + lane];
            ysm[i * 32 + lane] = (ysm[i * 32 + lane] - t) * __ldg(dinv + i);
        }
        __syncthreads();
    }
    if (j < n)
        for (int i = ty; i < n; i += kInvRows) {
            const double v = ysm[i * 32 + lane];
            Minv[(long long)i * n + j] = v;
            if (Minv32) Minv32[(long long)i * n + j] = (float)v;
        }
}

__global__ void __launch_bounds__(32 * kInvRows) k_band_inv_cols_warp(const double *__restrict__ M,
                                                                      const int *__restrict__ piv,
                                                                      const double *__restrict__ dinv, int n, int kl,
                                                                      int ku, double *__restrict__ Minv,
                                                                      float *__restrict__ Minv32,
                                                                      const int *__restrict__ err) {
    band_inv_cols_warp_block(M, piv, dinv, n, kl, ku, Minv, Minv32, blockIdx.x, err);
}

// Coarsest inverse for kBandSmemMax < n <= 1024 in three kernels that exploit
// the band of the coarsest matrix (cells in lexicographic order, two unknowns
// each: entries lie within kl = 2 * (largest neighbour cell offset) + 1 of the
// diagonal).
//
// 1. k_band_lu: LU with partial pivoting restricted to the band, one block:
//    per column k the pivot is the largest |a_rk| for k <= r <= k + kl, rows
//    k and pivot are swapped over the columns the band can reach (k .. k + kl
//    + ku, U's band after pivoting), multipliers l_rk = a_rk / a_kk are stored
//    below the diagonal and the window rows k+1..k+kl, columns k+1..k+kl+ku
//    is updated.  piv[k] = pivot row; dinv[k] = 1 / u_kk.  err |= 4 on a zero
//    pivot.
// 2. k_band_inv_cols: thread j solves L U x = P e_j (row swaps and the unit
//    lower factor forward, U backward) into W[j][*].
// 3. k_transpose: Minv[i][j] = W[j][i].
// One 32 x 32 block factors one matrix (shared with the batched kernel).
__device__ __forceinline__ void band_lu_block(double *__restrict__ M, int n, int kl, int ku, int *__restrict__ piv,
                                              double *__restrict__ dinv, int *__restrict__ err) {
    __shared__ int prow;
    __shared__ double pinv;
    __shared__ int bad;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + 32 * ty;
    const int ur = kl + ku;                      // reach of U after pivoting
    if (tid == 0) bad = 0;
    __syncthreads();
    int k = 0;
    for (; k < n; k++) {
        const int rlast = min(n - 1, k + kl), clast = min(n - 1, k + ur);
        if (ty == 0) {
            double best = -1.0;
            int br = k;
            for (int r = k + tx; r <= rlast; r += 32) {
                const double v = fabs(M[(long long)r * n + k]);
                if (v > best) { best = v; br = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, best, o);
                const int orr = __shfl_down_sync(0xffffffffu, br, o);
                if (ov > best || (ov == best && orr < br)) { best = ov; br = orr; }
            }
            if (tx == 0) {
                prow = br;
                piv[k] = br;
                if (!(best > 0.0)) bad = 1;
                else {
                    pinv = 1.0 / M[(long long)br * n + k];
                    dinv[k] = pinv;
                }
            }
        }
        __syncthreads();
        if (bad) break;
        const int p = prow;
        if (p != k)
            for (int c = k + tid; c <= clast; c += 1024) {
                const double t = M[(long long)k * n + c];
                M[(long long)k * n + c] = M[(long long)p * n + c];
                M[(long long)p * n + c] = t;
            }
        __syncthreads();
        const double ip = pinv;
        for (int r = k + 1 + tid; r <= rlast; r += 1024) M[(long long)r * n + k] *= ip;
        __syncthreads();
        for (int r = k + 1 + ty; r <= rlast; r += 32) {
            const double l = M[(long long)r * n + k];
            if (l != 0.0)
                for (int c = k + 1 + tx; c <= clast; c += 32) M[(long long)r * n + c] -= l * M[(long long)k * n + c];
        }
        __syncthreads();
    }
    if (bad) {
        // identity permutation from the failing column on, then report
        for (int q = k + tid; q < n; q += 1024) {
            piv[q] = q;
            dinv[q] = 0.0;
        }
        if (tid == 0) atomicOr(err, 4);
    }
}

__global__ void __launch_bounds__(1024) k_band_lu(double *__restrict__ M, int n, int kl, int ku,
                                                  int *__restrict__ piv, double *__restrict__ dinv,
                                                  int *__restrict__ err) {
    band_lu_block(M, n, kl, ku, piv, dinv, err);
}

// Column j of the inverse into W[j][*] (one thread).
__device__ __forceinline__ void band_inv_col(const double *__restrict__ M, const int *__restrict__ piv,
                                             const double *__restrict__ dinv, int n, int kl, int ku,
                                             double *__restrict__ W, const int *__restrict__ err, int j) {
    if (j >= n || (*(volatile const int *)err & 4)) return;
    double *y = W + (long long)j * n;
    for (int i = 0; i < n; i++) y[i] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++) {              // P and L, in the order the factorisation applied them
        const int p = min(max(piv[k], k), n - 1);
        if (p != k) {
            const double t = y[k];
            y[k] = y[p];
            y[p] = t;
        }
        const double yk = y[k];
        if (yk != 0.0) {
            const int rlast = min(n - 1, k + kl);
            for (int r = k + 1; r <= rlast; r++) y[r] -= M[(long long)r * n + k] * yk;
        }
    }
    const int ur = kl + ku;
    for (int i = n - 1; i >= 0; i--) {         // U
        double s = y[i];
        const int clast = min(n - 1, i + ur);
        for (int c = i + 1; c <= clast; c++) s -= M[(long long)i * n + c] * y[c];
        y[i] = s * dinv[i];
    }
}

__global__ void k_band_inv_cols(const double *__restrict__ M, const int *__restrict__ piv,
                                const double *__restrict__ dinv, int n, int kl, int ku, double *__restrict__ W,
                                const int *__restrict__ err) {
    band_inv_col(M, piv, dinv, n, kl, ku, W, err, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_transpose(const double *__restrict__ W, double *__restrict__ Minv, int n) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)n * n;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / n), j = (int)(q - (long long)i * n);
        Minv[q] = W[(long long)j * n + i];
    }
}

// ---------------------------------------------------------------------------
// Coarsest inverse for kBandSmemMax < n (the coarsest grids of sizes with an
// odd factor of 9 or more, up to 31 x 31 cells) in two kernels, both exact in
// FP64 with the same banded partial pivoting as k_band_lu:
//
// 1. k_band_lu_window: one block.  Only the active window of the band, rows
//    k..k+kl and columns k..k+kl+ku, is live at step k; it sits in shared
//    memory, circular in both directions, and the row that enters after the
//    step is loaded from global memory while the step computes.  The factors
//    leave in compact band layouts: Lb[k][q] = l_{k+1+q,k} (q < kl) and
//    Uc[c][o] = u_{c-o,c} (1 <= o <= kl+ku, column c of U), with piv[k] and
//    dinv[k] = 1 / u_kk.
// 2. k_band_inv_block: each warp of a block computes one column j of the
//    inverse, y = U^-1 L^-1 P e_j (the row swaps and multipliers in the order
//    the factorisation applied them, then U from the last row up), with y in
//    shared memory; the block's warps walk the same steps together, so each
//    chunk of kInvChunk rows of Lb / Uc is staged in shared memory once for
//    all of them.  The columns are written back as row segments of Minv (and
//    of the FP32 copy).
// ---------------------------------------------------------------------------
constexpr int kWinThreads = 1024;
constexpr int kLuAhead = 8;           // steps by which the windowed LU loads the rows entering it ahead
constexpr int kInvChunk = 32;
constexpr long long kWinSmemMax = 200 * 1024;

// Shared memory of k_band_lu_window for bandwidths kl, ku (bytes).
inline long long band_window_smem(int kl, int ku) {
    const long long R = kl + 1, C = kl + ku + 1;
    return 8LL * (R * C + C + R);
}

// Shared memory of k_band_inv_block with `warps` warps per block (bytes).
inline long long band_inv_block_smem(int n, int kl, int ku, int warps) {
    const long long C = kl + ku + 1;
    return 8LL * ((long long)warps * n + (long long)kInvChunk * (kl + C + 1)) + 4LL * kInvChunk;
}

// Slot arithmetic without divisions: a window row or column index moves by
// at most one period, so one conditional subtraction wraps it.
__device__ __forceinline__ int wrap(int v, int m) { return v >= m ? v - m : v; }

// One pivot step of the windowed LU (see band_lu_window_block).  `pre` holds
// column k + 1 + tid of the row that enters the window after this step, and
// receives the one that enters kLuAhead steps later.  Returns false on a zero
// pivot.
__device__ __forceinline__ bool band_lu_window_step(const double *__restrict__ M, int n, int kl, int R, int C, int ur,
                                                    int k, int ks, int kc, double *W, double *urow, double *lmul,
                                                    int *__restrict__ piv, double *__restrict__ dinv,
                                                    double *__restrict__ Lb, double *__restrict__ Uc, double &pre,
                                                    int &s_piv, int &s_bad, double &s_pinv) {
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5, nty = blockDim.x >> 5;
    const int rlast = min(n - 1, k + kl), clast = min(n - 1, k + ur);
    if (tid < 32) {
        // pivot: largest |a_rk|, the first such row on ties.  |a| is compared
        // as its bit pattern with the sign cleared (monotone for non-negative
        // doubles), on the integer pipe instead of GB300's scarce FP64 one.
        long long best = -1;
        int br = k;
        for (int r = k + tid, rs = wrap(ks + tid, R); r <= rlast; r += 32, rs = wrap(rs + 32 - (32 / R) * R, R)) {
            const long long v = __double_as_longlong(W[rs * C + kc]) & 0x7fffffffffffffffLL;
            if (v > best) { best = v; br = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_down_sync(0xffffffffu, best, o);
            const int orr = __shfl_down_sync(0xffffffffu, br, o);
            if (ov > best || (ov == best && orr < br)) { best = ov; br = orr; }
        }
        if (tid == 0) {
            s_piv = br;
            piv[k] = br;
            if (best <= 0) s_bad = 1;               // an exactly zero column below the diagonal
        }
    }
    __syncthreads();
    if (s_bad) return false;
    const int p = s_piv;
    if (tid <= clast - k) {                        // swap rows k and p; keep row k of U
        const int cs = wrap(kc + tid, C);
        const double a = W[ks * C + cs];
        double b = a;
        if (p != k) {
            const int ps = wrap(ks + (p - k), R) * C + cs;
            b = W[ps];
            W[ps] = a;
            W[ks * C + cs] = b;
        }
        urow[tid] = b;
        // one reciprocal per step: GB300's FP64 pipe issues ~2 operations per clock per SM,
        // and a division in every thread of the block would cost more than the step's update
        if (tid == 0) s_pinv = 1.0 / b;
    }
    __syncthreads();
    const double pinv = s_pinv;
    if (tid >= 1 && tid <= clast - k) Uc[(long long)(k + tid) * C + tid] = urow[tid];
    if (tid == 0) dinv[k] = pinv;
    if (tid < rlast - k) {                         // multipliers of rows k+1..rlast; column k leaves the window
        const int rs = wrap(ks + 1 + tid, R) * C + kc;
        const double l = W[rs] * pinv;
        lmul[tid] = l;
        Lb[(long long)k * kl + tid] = l;
        W[rs] = 0.0;
    }
    __syncthreads();
    const int nr = rlast - k, ncl = clast - k;
    for (int i = ty; i < nr; i += nty) {           // rows k+1..rlast by warp, columns k+1..clast by lane
        const double l = lmul[i];
        double *row = W + wrap(ks + 1 + i, R) * C;
        for (int jj = tx; jj < ncl; jj += 32) row[wrap(kc + 1 + jj, C)] -= l * urow[1 + jj];
    }
    if (tid < C) W[ks * C + wrap(kc + 1 + tid, C)] = pre;   // row k + R enters the retired slot (zeros beyond n)
    {
        const int r = k + R + kLuAhead, c = k + kLuAhead + 1 + tid;
        pre = (tid < C && r < n && c < n) ? M[(long long)r * n + c] : 0.0;
    }
    __syncthreads();
    return true;
}

__device__ __forceinline__ void band_lu_window_block(const double *__restrict__ M, int n, int kl, int ku,
                                                     int *__restrict__ piv, double *__restrict__ dinv,
                                                     double *__restrict__ Lb, double *__restrict__ Uc,
                                                     int *__restrict__ err) {
    extern __shared__ double wsm[];
    __shared__ int s_piv, s_bad;
    __shared__ double s_pinv;
    const int R = kl + 1, ur = kl + ku, C = ur + 1;
    double *W = wsm;                  // R x C window: entry (r, c) at (r mod R) * C + (c mod C)
    double *urow = W + R * C;         // row k of U after the swap (columns k..k+ur)
    double *lmul = urow + C;          // multipliers of rows k+1..k+kl
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int q = tid; q < R * C; q += nthr) {
        const int r = q / C, c = q - r * C;
        W[q] = (r < n && c < n) ? M[(long long)r * n + c] : 0.0;
    }
    if (tid == 0) s_bad = 0;
    // the rows entering the window, kLuAhead steps ahead: pre[a] serves the
    // steps k = a (mod kLuAhead); the step loop is unrolled by kLuAhead so
    // every slot is a register that its load has kLuAhead steps to fill
    double pre[kLuAhead];
#pragma unroll
    for (int a = 0; a < kLuAhead; a++) {
        const int r = R + a, c = a + 1 + tid;
        pre[a] = (tid < C && r < n && c < n) ? M[(long long)r * n + c] : 0.0;
    }
    __syncthreads();
    int k = 0, ks = 0, kc = 0;        // k mod R, k mod C
    bool ok = true;
    for (; k < n && ok;) {
#pragma unroll
        for (int a = 0; a < kLuAhead; a++) {
            if (k < n && ok) {
                ok = band_lu_window_step(M, n, kl, R, C, ur, k, ks, kc, W, urow, lmul, piv, dinv, Lb, Uc, pre[a],
                                         s_piv, s_bad, s_pinv);
                if (ok) {
                    k++;
                    ks = wrap(ks + 1, R);
                    kc = wrap(kc + 1, C);
                }
            }
        }
    }
    if (!ok) {
        for (int q = k + tid; q < n; q += nthr) {
            piv[q] = q;
            dinv[q] = 0.0;
        }
        if (tid == 0) atomicOr(err, 4);
    }
}

__global__ void __launch_bounds__(kWinThreads) k_band_lu_window(const double *__restrict__ M, int n, int kl, int ku,
                                                                int *__restrict__ piv, double *__restrict__ dinv,
                                                                double *__restrict__ Lb, double *__restrict__ Uc,
                                                                int *__restrict__ err) {
    band_lu_window_block(M, n, kl, ku, piv, dinv, Lb, Uc, err);
}

// ---------------------------------------------------------------------------
// The windowed LU blocked over a thread-block cluster (k_band_lu_blocked).
// The single-block kernel runs every step's rank-1 update of the whole window
// on one SM, whose FP64 pipe bounds it.  Here the columns are grouped in
// panels of kLuNb; panel b belongs to CTA b mod kLuClusterCtas, which keeps
// each of its columns j as the vector of rows j - (kl + ku) .. j + kl (every
// row a step can reach it in).  For panel b the owner runs the panel's steps
// on the panel's own columns only (pivot, swap, multipliers, row of U,
// update), then publishes the pivots and multipliers; after one cluster
// barrier every CTA applies those steps, in order, to each of its columns
// after the panel that they reach (swap, row of U, update), one warp per
// column.  Every entry receives the same multiply-adds in the same order as
// in the unblocked factorisation, so the factors are the single-block
// kernel's bit for bit.  A panel becomes resident kLuNb + kl + ku columns
// before its first step, in a slot freed long before.  A zero pivot stops
// every CTA after the same barrier; a last barrier keeps each CTA's shared
// memory alive until no other CTA reads it.
// ---------------------------------------------------------------------------
constexpr int kLuClusterCtas = 8;
constexpr int kLuNb = 16;
constexpr int kLuBlockedThreads = 512;

struct LuBlockedShape {
    int ur, C, Lc, NP, S, npan, bsz;
};

__host__ __device__ inline LuBlockedShape lu_blocked_shape(int n, int kl, int ku) {
    LuBlockedShape g;
    g.ur = kl + ku;
    g.C = g.ur + 1;
    g.Lc = g.ur + kl + 1;                                   // rows j - ur .. j + kl of column j
    g.NP = (kLuNb + g.ur + kLuNb - 1) / kLuNb;              // panels a panel's steps reach
    g.S = (g.NP + kLuClusterCtas - 1) / kLuClusterCtas + 1; // resident panels per CTA
    g.npan = (n + kLuNb - 1) / kLuNb;
    g.bsz = kLuNb * kl + kLuNb + 1;                         // multipliers, pivots, stop flag
    return g;
}

// Shared memory of k_band_lu_blocked (bytes), at least 116 KB: more than half
// of an SM's, so that no two CTAs of a cluster share an SM's FP64 pipe.
inline long long band_blocked_smem(int n, int kl, int ku) {
    const LuBlockedShape g = lu_blocked_shape(n, kl, ku);
    const long long need = 8LL * ((long long)g.S * kLuNb * g.Lc + 3LL * g.bsz + kLuNb);
    return need > 116LL * 1024 ? need : 116LL * 1024;
}

__device__ __forceinline__ void band_lu_blocked_block(const double *__restrict__ M, int n, int kl, int ku,
                                                      int *__restrict__ piv, double *__restrict__ dinv,
                                                      double *__restrict__ Lb, double *__restrict__ Uc,
                                                      int *__restrict__ err, double *sm) {
    namespace cg = cooperative_groups;
    constexpr int P = kLuClusterCtas, NB = kLuNb;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ long long s_best;
    __shared__ int s_p;
    __shared__ double s_pinv;
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const LuBlockedShape g = lu_blocked_shape(n, kl, ku);
    const int ur = g.ur, C = g.C, Lc = g.Lc;
    double *store = sm;                                     // S x NB x Lc
    double *bc = store + (long long)g.S * NB * Lc;          // 2 x bsz: this CTA's broadcasts
    double *loc = bc + 2 * g.bsz;                           // bsz: the panel owner's, copied
    double *urow = loc + g.bsz;                             // NB: row p of U in the panel's columns
    // column j of a panel this CTA owns
    auto colp = [&](int j) {
        const int b = j / NB;
        return store + ((long long)((b / P) % g.S) * NB + (j - b * NB)) * Lc;
    };
    auto load_panel = [&](int b) {
        if (b >= g.npan || b % P != rank) return;
        double *base = colp(b * NB);
        for (int q = tid; q < NB * Lc; q += nt) {
            const int c = q / Lc, idx = q - c * Lc, j = b * NB + c, r = j - ur + idx;
            base[q] = (j < n && r >= 0 && r < n) ? M[(long long)r * n + j] : 0.0;
        }
    };
    for (int b = 0; b < g.NP && b < g.npan; b++) load_panel(b);
    __syncthreads();
    int kfail = n;
    for (int b = 0; b < g.npan; b++) {
        const int o = b % P, k0 = b * NB, k1 = min(n, k0 + NB);
        double *bs = bc + (b & 1) * g.bsz;
        if (rank == o) {                                    // the same branch in every thread of this CTA
            if (tid == 0) bs[NB * kl + NB] = -1.0;
            for (int p = k0; p < k1; p++) {
                double *cp = colp(p);
                const int rl = min(n - 1, p + kl), nr = rl - p;
                if (tid < 32) {                             // pivot: largest |a|, first row on ties
                    long long best = -1;
                    int br = p;
                    for (int r = p + tid; r <= rl; r += 32) {
                        const long long v = __double_as_longlong(cp[r - p + ur]) & 0x7fffffffffffffffLL;
                        if (v > best) { best = v; br = r; }
                    }
                    for (int off = 16; off > 0; off >>= 1) {
                        const long long ov = __shfl_down_sync(0xffffffffu, best, off);
                        const int orr = __shfl_down_sync(0xffffffffu, br, off);
                        if (ov > best || (ov == best && orr < br)) { best = ov; br = orr; }
                    }
                    if (tid == 0) {
                        s_best = best;
                        s_p = br;
                    }
                }
                __syncthreads();
                if (s_best <= 0) {                          // a zero column: stop here, every CTA at this panel
                    if (tid == 0) bs[NB * kl + NB] = (double)p;
                    __syncthreads();
                    break;
                }
                const int pp = s_p;
                if (tid < k1 - p) {                         // swap rows p and pp in the panel's columns p..k1-1
                    const int j = p + tid;
                    double *cj = colp(j);
                    const int ia = p - j + ur, ib = pp - j + ur;
                    const double a = cj[ia];
                    cj[ia] = cj[ib];
                    cj[ib] = a;
                }
                __syncthreads();
                if (tid == 0) {
                    s_pinv = 1.0 / cp[ur];
                    piv[p] = pp;
                    dinv[p] = s_pinv;
                    bs[NB * kl + (p - k0)] = (double)pp;
                }
                __syncthreads();
                const double pinv = s_pinv;
                for (int q = tid; q < nr; q += nt) {
                    const double l = cp[ur + 1 + q] * pinv;
                    bs[(p - k0) * kl + q] = l;
                    Lb[(long long)p * kl + q] = l;
                }
                if (tid < k1 - p - 1) {                     // row p of U in the panel's columns p+1..k1-1
                    const int j = p + 1 + tid;
                    const double u = colp(j)[p - j + ur];
                    urow[tid] = u;
                    Uc[(long long)j * C + (j - p)] = u;
                }
                __syncthreads();
                for (int c = warp; c < k1 - p - 1; c += nw) {   // the panel's columns by warp, rows by lane
                    const int j = p + 1 + c;
                    double *cj = colp(j);
                    const double u = urow[c];
                    for (int q = lane; q < nr; q += 32) cj[p + 1 + q - j + ur] -= bs[(p - k0) * kl + q] * u;
                }
                __syncthreads();
            }
        }
        cl.sync();                                          // panel b's broadcast is visible cluster-wide
        const double *ob = cl.map_shared_rank(bs, o);
        for (int q = tid; q < g.bsz; q += nt) loc[q] = ob[q];
        __syncthreads();
        const int stop = (int)loc[NB * kl + NB];            // read by every thread of every CTA
        const int kend = stop >= 0 ? stop : k1;             // the panel's steps that ran
        // this CTA's columns k1 .. min(n - 1, kend - 1 + ur), a warp each: panel b's steps, in order
        const int hi = min(n - 1, kend - 1 + ur);
        if (stop < 0 && k1 <= hi) {
            const int pb = k1 / NB;                         // first panel after b
            const int b1 = pb + ((rank - pb) % P + P) % P;  // this CTA's first panel >= pb
            for (int c = warp; c < g.S * NB; c += nw) {
                const int j = (b1 + (c / NB) * P) * NB + (c % NB);
                if (j > hi) continue;
                double *cj = colp(j);
                for (int p = max(k0, j - ur); p < kend; p++) {
                    const int pp = (int)loc[NB * kl + (p - k0)];
                    const int ia = p - j + ur, ib = pp - j + ur;
                    if (lane == 0 && pp != p) {
                        const double a = cj[ia];
                        cj[ia] = cj[ib];
                        cj[ib] = a;
                    }
                    __syncwarp();
                    const double u = cj[ia];
                    if (lane == 0) Uc[(long long)j * C + (j - p)] = u;
                    const int nr = min(n - 1, p + kl) - p;
                    for (int q = lane; q < nr; q += 32) cj[p + 1 + q - j + ur] -= loc[(p - k0) * kl + q] * u;
                    __syncwarp();
                }
            }
        }
        if (stop >= 0) {
            kfail = stop;
            break;
        }
        __syncthreads();
        load_panel(b + g.NP);
        __syncthreads();
    }
    if (kfail < n && rank == 0) {
        for (int q = kfail + tid; q < n; q += nt) {
            piv[q] = q;
            dinv[q] = 0.0;
        }
        if (tid == 0) atomicOr(err, 4);
    }
    cl.sync();                                              // no CTA leaves while another may still read it
}

__global__ void __launch_bounds__(kLuBlockedThreads) k_band_lu_blocked(const double *__restrict__ M, int n, int kl,
                                                                       int ku, int *__restrict__ piv,
                                                                       double *__restrict__ dinv,
                                                                       double *__restrict__ Lb,
                                                                       double *__restrict__ Uc,
                                                                       int *__restrict__ err) {
    extern __shared__ double lbsm[];
    band_lu_blocked_block(M, n, kl, ku, piv, dinv, Lb, Uc, err, lbsm);
}

// Columns j0 .. j0 + warps - 1 of the inverse (block of warps x 32 threads).
__device__ __forceinline__ void band_inv_block(const double *__restrict__ Lb, const double *__restrict__ Uc,
                                               const int *__restrict__ piv, const double *__restrict__ dinv, int n,
                                               int kl, int ku, double *__restrict__ Minv, float *__restrict__ Minv32,
                                               const int *__restrict__ err, int j0) {
    if (*(volatile const int *)err & 4) return;
    extern __shared__ double ism[];
    const int C = kl + ku + 1, ur = kl + ku;
    const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x, nthr = blockDim.x;
    double *y = ism + (long long)w * n;                      // this warp's column
    double *Lc = ism + (long long)warps * n;                 // kInvChunk rows of Lb
    double *Ucc = Lc + kInvChunk * kl;                       // kInvChunk rows of Uc
    double *dc = Ucc + kInvChunk * C;                        // kInvChunk of dinv
    int *pc = reinterpret_cast<int *>(dc + kInvChunk);       // kInvChunk of piv
    const int j = j0 + w;
    const bool live = j < n;
    for (int i = lane; i < n; i += 32) y[i] = (live && i == j) ? 1.0 : 0.0;
    // forward: P and L; columns j < n start at max(0, j - kl): earlier steps only swap and scale zeros
    const int kstart = max(0, j0 - kl);
    for (int kb = kstart; kb < n; kb += kInvChunk) {
        const int cnt = min(kInvChunk, n - kb);
        __syncthreads();
        for (int q = tid; q < cnt * kl; q += nthr) Lc[q] = Lb[(long long)kb * kl + q];
        for (int q = tid; q < cnt; q += nthr) pc[q] = piv[kb + q];
        __syncthreads();
        for (int t = 0; t < cnt; t++) {
            const int k = kb + t;
            const int p = pc[t];
            if (p != k && lane == 0) {
                const double a = y[k];
                y[k] = y[p];
                y[p] = a;
            }
            __syncwarp();
            const double yk = y[k];
            const int m = min(kl, n - 1 - k);
            for (int q = lane; q < m; q += 32) y[k + 1 + q] -= Lc[t * kl + q] * yk;
            __syncwarp();
        }
    }
    // backward: U, from the last row up, column-wise: y_i = y_i / u_ii, then
    // y_{i-o} -= u_{i-o,i} y_i
    for (int ib = n - 1; ib >= 0; ib -= kInvChunk) {
        const int cnt = min(kInvChunk, ib + 1);
        __syncthreads();
        for (int q = tid; q < cnt * C; q += nthr) Ucc[q] = Uc[(long long)(ib - cnt + 1) * C + q];
        for (int q = tid; q < cnt; q += nthr) dc[q] = dinv[ib - cnt + 1 + q];
        __syncthreads();
        for (int t = cnt - 1; t >= 0; t--) {
            const int i = ib - cnt + 1 + t;
            const double yi = y[i] * dc[t];
            __syncwarp();
            if (lane == 0) y[i] = yi;
            const int m = min(ur, i);
            for (int o = 1 + lane; o <= m; o += 32) y[i - o] -= Ucc[t * C + o] * yi;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int q = tid; q < n * warps; q += nthr) {            // row segments Minv[i][j0 .. j0 + warps)
        const int i = q / warps, ww = q - i * warps;
        if (j0 + ww < n) {
            const double v = ism[(long long)ww * n + i];
            Minv[(long long)i * n + j0 + ww] = v;
            if (Minv32) Minv32[(long long)i * n + j0 + ww] = (float)v;
        }
    }
}

__global__ void __launch_bounds__(256) k_band_inv_block(const double *__restrict__ Lb, const double *__restrict__ Uc,
                                                        const int *__restrict__ piv, const double *__restrict__ dinv,
                                                        int n, int kl, int ku, double *__restrict__ Minv,
                                                        float *__restrict__ Minv32, const int *__restrict__ err) {
    band_inv_block(Lb, Uc, piv, dinv, n, kl, ku, Minv, Minv32, err, blockIdx.x * (blockDim.x >> 5));
}

// ---------------------------------------------------------------------------
// The coarsest solve from the factors (mg_options.coarse_solve AUTO on the
// windowed path): x = U^-1 L^-1 P b with the factors k_band_lu_window leaves
// (Lb, piv; Uc with each column scaled by its reciprocal pivot, see
// k_scale_uc), one block of kLuSolveThreads per system, in FP64 whatever R
// is.  The steps are those of one column of k_band_inv_block with b in place
// of e_j: the row swaps and multipliers in the order the factorisation
// applied them, then U from the last row up.  A step's multiply-adds are
// spread over the block's four warps, one per SM sub-partition: GB300's FP64
// pipe issues a warp's FMA over many cycles, so one warp would take four
// times as long per step.  One barrier per step, two for a forward step that
// swaps rows: every thread reads the pivot row's value itself (and, for a
// swap, y_k, before thread 0 overwrites it); the thread that updates the
// pivot row starts from the value swapped out of row k.  In the backward
// step the scaled column puts no division on the chain (x = dinv y at the
// end, all threads).  y sits in
// shared memory; the rows of Lb (and piv) or Uc the next kLuSolveRows steps
// use are staged by asynchronous 8-byte copies one chunk ahead,
// double-buffered.  With the coarsest matrix singular (err & 4, reported by
// the solve) x is set to 0.
// ---------------------------------------------------------------------------
constexpr int kLuSolveRows = 16;
constexpr int kLuSolveThreads = 128;

// Shared memory of k_coarse_lu (bytes): y, then two chunks each of Lb rows,
// Uc rows and piv.
inline long long coarse_lu_smem(int n, int kl, int ku) {
    const long long C = kl + ku + 1;
    return 8LL * (n + 2LL * kLuSolveRows * (kl + C)) + 4LL * 2 * kLuSolveRows;
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Uc[i][o] *= dinv[i] (1 <= o <= kl + ku): column i of U over its pivot, so
// that the backward step updates with y_i itself (one system, grid-stride).
__device__ __forceinline__ void scale_uc(double *__restrict__ Uc, const double *__restrict__ dinv, int n, int kl,
                                         int ku, const int *__restrict__ err, long long start, long long stride) {
    if (*(volatile const int *)err & 4) return;
    const int ur = kl + ku, C = ur + 1;
    for (long long q = start; q < (long long)n * ur; q += stride) {
        const int i = (int)(q / ur), o = 1 + (int)(q - (long long)i * ur);
        Uc[(long long)i * C + o] *= dinv[i];
    }
}

__global__ void k_scale_uc(double *__restrict__ Uc, const double *__restrict__ dinv, int n, int kl, int ku,
                           const int *__restrict__ err) {
    scale_uc(Uc, dinv, n, kl, ku, err, blockIdx.x * (long long)blockDim.x + threadIdx.x,
             (long long)gridDim.x * blockDim.x);
}

template <typename R>
__device__ void coarse_lu_solve_block(const double *__restrict__ Lb, const double *__restrict__ Uc,
                                      const int *__restrict__ piv, const double *__restrict__ dinv, int n, int kl,
                                      int ku, const R *__restrict__ b, R *__restrict__ x,
                                      const int *__restrict__ err, double *sm) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (*(volatile const int *)err & 4) {
        for (int i = tid; i < n; i += nt) x[i] = R(0);
        return;
    }
    const int C = kl + ku + 1, ur = kl + ku;
    double *y = sm;
    double *Lbuf = y + n;                                      // 2 x kLuSolveRows x kl
    double *Ubuf = Lbuf + 2 * kLuSolveRows * kl;                // 2 x kLuSolveRows x C
    int *pbuf = reinterpret_cast<int *>(Ubuf + 2 * kLuSolveRows * C);   // 2 x kLuSolveRows
    const int nch = (n + kLuSolveRows - 1) / kLuSolveRows;
    for (int i = tid; i < n; i += nt) y[i] = (double)b[i];
    // forward: rows k0 .. k0 + cnt - 1 of Lb and piv per chunk
    auto stage_l = [&](int k0, int buf) {
        const int cnt = min(kLuSolveRows, n - k0);
        const double *src = Lb + (long long)k0 * kl;
        double *dst = Lbuf + buf * kLuSolveRows * kl;
        for (int q = tid; q < cnt * kl; q += nt) cp_async8(dst + q, src + q);
        for (int q = tid; q < cnt; q += nt) cp_async4(pbuf + buf * kLuSolveRows + q, piv + k0 + q);
        cp_async_commit();
    };
    stage_l(0, 0);
    for (int c = 0; c < nch; c++) {
        const int k0 = c * kLuSolveRows, cnt = min(kLuSolveRows, n - k0), buf = c & 1;
        __syncthreads();                        // chunk c - 1, in the other buffer, is done with
        if (c + 1 < nch) {
            stage_l(k0 + kLuSolveRows, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const double *Lc = Lbuf + buf * kLuSolveRows * kl;
        const int *pc = pbuf + buf * kLuSolveRows;
        for (int t = 0; t < cnt; t++) {
            const int k = k0 + t, p = pc[t];
            const double yk = y[p];                // y_k after the swap (p == k: no swap)
            double a = 0.0;
            if (p != k) {                          // the same branch in every thread
                a = y[k];
                __syncthreads();                   // both read everywhere before either changes
                if (tid == 0) y[k] = yk;
            }
            const int m = min(kl, n - 1 - k);
            for (int q = tid; q < m; q += nt) {
                const int r = k + 1 + q;
                const double v = r == p ? a : y[r];
                y[r] = v - Lc[t * kl + q] * yk;
            }
            __syncthreads();
        }
    }
    // backward: rows hi - cnt + 1 .. hi of the scaled Uc per chunk, from the last row up
    auto stage_u = [&](int hi, int buf) {
        const int cnt = min(kLuSolveRows, hi + 1), lo = hi - cnt + 1;
        const double *src = Uc + (long long)lo * C;
        double *dst = Ubuf + buf * kLuSolveRows * C;
        for (int q = tid; q < cnt * C; q += nt) cp_async8(dst + q, src + q);
        cp_async_commit();
    };
    stage_u(n - 1, 0);
    for (int c = 0; c < nch; c++) {
        const int hi = n - 1 - c * kLuSolveRows, cnt = min(kLuSolveRows, hi + 1), lo = hi - cnt + 1, buf = c & 1;
        __syncthreads();
        if (c + 1 < nch) {
            stage_u(hi - kLuSolveRows, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const double *Ucc = Ubuf + buf * kLuSolveRows * C;
        for (int t = cnt - 1; t >= 0; t--) {
            const int i = lo + t;
            const double yi = y[i];
            const int m = min(ur, i);
            for (int o = 1 + tid; o <= m; o += nt) y[i - o] -= Ucc[t * C + o] * yi;
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) x[i] = (R)(y[i] * dinv[i]);
}

template <typename R>
__global__ void __launch_bounds__(kLuSolveThreads) k_coarse_lu(const double *__restrict__ Lb,
                                                               const double *__restrict__ Uc,
                                                               const int *__restrict__ piv,
                                                               const double *__restrict__ dinv, int n, int kl, int ku,
                                                               const R *__restrict__ b, R *__restrict__ x,
                                                               const int *__restrict__ err) {
    pdl_entry();
    extern __shared__ double lusm[];
    coarse_lu_solve_block<R>(Lb, Uc, piv, dinv, n, kl, ku, b, x, err, lusm);
}

}  // namespace cmg
