// The bottom of a V-cycle in one launch on a thread-block cluster.
//
// Every level from a first "tail" level (at most kTailMaxCells cells) down to
// the coarsest runs as stages of one kernel: pre-smoothing colours,
// restriction, the coarsest solve, prolongation, post-smoothing colours, with
// a hardware cluster barrier (release / acquire) between stages.  Launched
// separately, each of these small stages costs a kernel launch for very
// little work.
//
// State lives in shared memory.  Each level's cells are cut into slabs (rows
// in 2D, z-planes in 3D); CTA r of the cluster owns slabs [r*chunk,
// (r+1)*chunk) and keeps their x, b and bt (= Dinv b) in its own shared
// memory.  A stage updates only the cells its CTA owns; neighbour values in
// other CTAs' slabs are read through distributed shared memory.  For the
// smallest levels a single CTA can own everything (no cluster; block barriers,
// which cost far less than cluster barriers, between stages).  Coefficients
// (faces, D, Dinv, W, l4, the coarsest inverse) are read-only here and come
// from global memory through the read-only cache.  On entry the first tail
// level's b and bt are read from global memory (where the restriction from
// the level above left them) and x starts at zero; on exit its x goes back to
// global memory for the prolongation to the level above.
//
// Each stage repeats the separate kernels' per-cell arithmetic operation for
// operation (same operands, same order, same fused multiply-adds), so a solve
// with the tail equals one without it bit for bit.
#pragma once
#include <cooperative_groups.h>

#include "mg_kernels.cuh"

namespace cmg {

constexpr int kTailCells = 4096;       // default: first level below the finest with at most this many cells
constexpr int kTailMaxLevels = 12;
constexpr int kTailCtas = 8;           // CTAs of the cluster (portable cluster size)
constexpr int kTailMaxCells = 16384;   // largest first tail level a tuning may choose
constexpr int kTailThreads = kBX * kBY;

template <typename R>
struct TailLevel {
    Level<R> g;          // the level in global memory (coefficients; x, b, bt of the first tail level)
    int S;               // slabs: n1 (2D) or n2 (3D)
    int chunk;           // slabs per CTA
    int slab;            // cells per slab: n0 (2D) or n0 * n1 (3D)
    int off;             // this level's offset in each CTA's shared memory, in pairs: x, then b, then bt
    int cap;             // chunk * slab: pairs per array
};

template <typename R>
struct TailArgs {
    TailLevel<R> L[kTailMaxLevels];   // first tail level .. coarsest
    int nlev;
    BcFlags bc;
    const R *Minv;
    int nc;
    int nu1, nu2;
};

// Shared-memory pairs one CTA needs for levels L[0..nlev).
template <typename R>
inline int tail_layout(TailArgs<R> &A, int dim, int ctas) {
    int off = 0;
    for (int l = 0; l < A.nlev; l++) {
        TailLevel<R> &T = A.L[l];
        T.S = dim == 3 ? T.g.n2 : T.g.n1;
        T.slab = dim == 3 ? T.g.n0 * T.g.n1 : T.g.n0;
        T.chunk = (T.S + ctas - 1) / ctas;
        T.cap = T.chunk * T.slab;
        T.off = off;
        off += 3 * T.cap;
    }
    return off;
}

template <typename R>
struct TailCta {
    using V2 = typename Vec<R>::v2;
    V2 *sm;              // this CTA's shared memory
    int rank;
};

// Address (generic, possibly in another CTA's shared memory) of array a
// (0 x, 1 b, 2 bt) of cell (i, j, k) of tail level T.  A single-CTA tail
// (CL false) owns every slab.
template <typename R, int DIM, bool CL>
__device__ __forceinline__ typename Vec<R>::v2 *tail_at(const TailCta<R> &C, const TailLevel<R> &T, int a, int i,
                                                        int j, int k) {
    namespace cg = cooperative_groups;
    const int s = DIM == 3 ? k : j;
    const int w = DIM == 3 ? i + T.g.n0 * j : i;
    if (!CL) return C.sm + T.off + a * T.cap + s * T.slab + w;
    const int owner = s / T.chunk;
    typename Vec<R>::v2 *p = C.sm + T.off + a * T.cap + (s - owner * T.chunk) * T.slab + w;
    if (owner == C.rank) return p;
    return cg::this_cluster().map_shared_rank(p, owner);
}

// Barrier between stages: the cluster's (release / acquire), or the block's.
template <bool CL>
__device__ __forceinline__ void tail_sync() {
    if (CL) cooperative_groups::this_cluster().sync();
    else __syncthreads();
}

// offdiag() on tail storage: the same faces, neighbours and order.
template <typename R, int DIM, bool CL, bool WITH_L4>
__device__ __forceinline__ void tail_offdiag(const TailCta<R> &C, const TailLevel<R> &T, int i, int j, int k,
                                             long long c, R &sT, R &sp) {
    using V2 = typename Vec<R>::v2;
    const Level<R> &L = T.g;
    const int n0 = L.n0, n1 = L.n1;
    sT = R(0);
    sp = R(0);
    const long long f0 = (long long)i + (long long)(n0 + 1) * ((long long)j + (long long)n1 * k);
    if (i > 0)      { V2 g = ldg2(L.G0 + f0);     V2 u = *tail_at<R, DIM, CL>(C, T, 0, i - 1, j, k); sT += g.x * u.x; sp += g.y * u.y; }
    if (i < n0 - 1) { V2 g = ldg2(L.G0 + f0 + 1); V2 u = *tail_at<R, DIM, CL>(C, T, 0, i + 1, j, k); sT += g.x * u.x; sp += g.y * u.y; }
    const long long f1 = (long long)i + (long long)n0 * ((long long)j + (long long)(n1 + 1) * k);
    if (j > 0)      { V2 g = ldg2(L.G1 + f1);      V2 u = *tail_at<R, DIM, CL>(C, T, 0, i, j - 1, k); sT += g.x * u.x; sp += g.y * u.y; }
    if (j < n1 - 1) { V2 g = ldg2(L.G1 + f1 + n0); V2 u = *tail_at<R, DIM, CL>(C, T, 0, i, j + 1, k); sT += g.x * u.x; sp += g.y * u.y; }
    if (DIM == 3) {
        const long long pl = (long long)n0 * n1;
        if (k > 0)        { V2 g = ldg2(L.G2 + c);      V2 u = *tail_at<R, DIM, CL>(C, T, 0, i, j, k - 1); sT += g.x * u.x; sp += g.y * u.y; }
        if (k < L.n2 - 1) { V2 g = ldg2(L.G2 + c + pl); V2 u = *tail_at<R, DIM, CL>(C, T, 0, i, j, k + 1); sT += g.x * u.x; sp += g.y * u.y; }
    }
    if (WITH_L4) sp += __ldg(L.l4 + c) * sT;
}

// Slabs [s0, s1) of level T that this CTA owns.
template <typename R>
__device__ __forceinline__ void tail_owned(const TailCta<R> &C, const TailLevel<R> &T, int &s0, int &s1) {
    s0 = C.rank * T.chunk;
    s1 = min(T.S, s0 + T.chunk);
}

// One colour of a red-black sweep over the owned cells (rbgs_colour_block's update).
template <typename R, int DIM, bool CL>
__device__ __forceinline__ void tail_colour(const TailCta<R> &C, const TailLevel<R> &T, int colour) {
    const Level<R> &L = T.g;
    int s0, s1;
    tail_owned(C, T, s0, s1);
    const int half = (L.n0 + 1) / 2;
    const int rows = DIM == 3 ? L.n1 : 1;                 // rows of a slab
    const int per = rows * half;
    for (int q = threadIdx.x + kBX * threadIdx.y; q < (s1 - s0) * per; q += kTailThreads) {
        const int sl = q / per, rem = q - sl * per;
        const int r = rem / half, m = rem - r * half;
        const int j = DIM == 3 ? r : s0 + sl;
        const int k = DIM == 3 ? s0 + sl : 0;
        const int i = 2 * m + ((j + k + colour) & 1);
        if (i >= L.n0) continue;
        const long long c = cell_id(i, j, k, L.n0, L.n1);
        R sT, sp;
        tail_offdiag<R, DIM, CL, false>(C, T, i, j, k, c, sT, sp);
        typename Vec<R>::v2 *xp = tail_at<R, DIM, CL>(C, T, 0, i, j, k);
        const auto bt = *tail_at<R, DIM, CL>(C, T, 2, i, j, k);
        const auto W = ldgq(L.W + c);
        *xp = mk2<R>(bt.x - W.a * sT - W.b * sp, bt.y - W.c * sT - W.d * sp);
    }
}

// Restriction of the residual from F to its coarse level Cl over the coarse
// cells this CTA owns (residual_restrict_block's arithmetic).
template <typename R, int DIM, bool CL, bool RED>
__device__ __forceinline__ void tail_restrict(const TailCta<R> &C, const TailLevel<R> &F, const TailLevel<R> &Cl) {
    using V2 = typename Vec<R>::v2;
    const Level<R> &FL = F.g, &CG = Cl.g;
    int s0, s1;
    tail_owned(C, Cl, s0, s1);
    for (int q = threadIdx.x + kBX * threadIdx.y; q < (s1 - s0) * Cl.slab; q += kTailThreads) {
        const int sl = q / Cl.slab, w = q - sl * Cl.slab;
        const int I = w % CG.n0;
        const int J = DIM == 3 ? w / CG.n0 : s0 + sl;
        const int K = DIM == 3 ? s0 + sl : 0;
        R aT = R(0), ap = R(0);
#pragma unroll
        for (int qq = 0; qq < (1 << DIM); qq++) {
            if (RED && (__popc(qq) & 1)) continue;
            const int i = 2 * I + (qq & 1), j = 2 * J + ((qq >> 1) & 1), k = DIM == 3 ? 2 * K + (qq >> 2) : 0;
            const long long c = cell_id(i, j, k, FL.n0, FL.n1);
            R sT, sp;
            tail_offdiag<R, DIM, CL, true>(C, F, i, j, k, c, sT, sp);
            const V2 bb = *tail_at<R, DIM, CL>(C, F, 1, i, j, k), xx = *tail_at<R, DIM, CL>(C, F, 0, i, j, k);
            const auto Dd = ldgq(FL.D + c);
            const R rT = ((bb.x - sT) - Dd.a * xx.x) - Dd.b * xx.y;   // two FMAs per row
            const R rp = ((bb.y - sp) - Dd.c * xx.x) - Dd.d * xx.y;
            // the sums start from child 0 (always evaluated): no FP64 addition to 0
            aT = qq == 0 ? rT : aT + rT;
            ap = qq == 0 ? rp : ap + rp;
        }
        const R wgt = R(1) / R(1 << DIM);
        const long long cc = cell_id(I, J, K, CG.n0, CG.n1);
        const R bT = aT * wgt, bp = ap * wgt;
        *tail_at<R, DIM, CL>(C, Cl, 1, I, J, K) = mk2<R>(bT, bp);
        const auto Di = ldgq(CG.Dinv + cc);
        *tail_at<R, DIM, CL>(C, Cl, 2, I, J, K) = mk2<R>(Di.a * bT + Di.b * bp, Di.c * bT + Di.d * bp);
        *tail_at<R, DIM, CL>(C, Cl, 0, I, J, K) = mk2<R>(R(0), R(0));
    }
}

// Prolongation of Cl's x into F's owned cells (prolong_add_block's arithmetic).
template <typename R, int DIM, bool CL>
__device__ __forceinline__ void tail_prolong(const TailCta<R> &C, const TailLevel<R> &Cl, const TailLevel<R> &F,
                                             const BcFlags &bc) {
    using V2 = typename Vec<R>::v2;
    const Level<R> &FL = F.g, &CG = Cl.g;
    int s0, s1;
    tail_owned(C, F, s0, s1);
    for (int q = threadIdx.x + kBX * threadIdx.y; q < (s1 - s0) * F.slab; q += kTailThreads) {
        const int sl = q / F.slab, w = q - sl * F.slab;
        const int i = w % FL.n0;
        const int j = DIM == 3 ? w / FL.n0 : s0 + sl;
        const int k = DIM == 3 ? s0 + sl : 0;
        const int P[3] = {i >> 1, j >> 1, k >> 1};
        const int s[3] = {(i & 1) ? 1 : -1, (j & 1) ? 1 : -1, (k & 1) ? 1 : -1};
        const int nC[3] = {CG.n0, CG.n1, CG.n2};
        int Qn[3];
        bool neg[3];
#pragma unroll
        for (int a = 0; a < DIM; a++) {
            const int t = P[a] + s[a];
            if (t < 0)           { Qn[a] = P[a]; neg[a] = bc.dir[a][0] != 0; }
            else if (t >= nC[a]) { Qn[a] = P[a]; neg[a] = bc.dir[a][1] != 0; }
            else                 { Qn[a] = t;    neg[a] = false; }
        }
        R aT = R(0), ap = R(0);
#pragma unroll
        for (int qq = 0; qq < (1 << DIM); qq++) {
            int Q[3] = {P[0], P[1], DIM == 3 ? P[2] : 0};
            bool flip = false;
            int nq = 0;
#pragma unroll
            for (int a = 0; a < DIM; a++)
                if ((qq >> a) & 1) { Q[a] = Qn[a]; flip ^= neg[a]; nq++; }
            const R wq = DIM == 2 ? (nq == 0 ? R(9.0 / 16) : nq == 1 ? R(3.0 / 16) : R(1.0 / 16))
                                  : (nq == 0 ? R(27.0 / 64) : nq == 1 ? R(9.0 / 64) : nq == 2 ? R(3.0 / 64) : R(1.0 / 64));
            const V2 e = *tail_at<R, DIM, CL>(C, Cl, 0, Q[0], Q[1], Q[2]);
            const R ws = flip ? -wq : wq;
            aT += ws * e.x;
            ap += ws * e.y;
        }
        V2 *xp = tail_at<R, DIM, CL>(C, F, 0, i, j, k);
        V2 xv = *xp;
        xv.x += aT;
        xv.y += ap;
        *xp = xv;
    }
}

// CL: launched as a cluster of CTAs (distributed shared memory); else one CTA.
template <typename R, int DIM, bool CL>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(const __grid_constant__ TailArgs<R> A) {
    pdl_entry();
    namespace cg = cooperative_groups;
    using V2 = typename Vec<R>::v2;
    extern __shared__ __align__(16) unsigned char tail_smem[];
    TailCta<R> C{reinterpret_cast<V2 *>(tail_smem), CL ? (int)cg::this_cluster().block_rank() : 0};
    const int tid = threadIdx.x + kBX * threadIdx.y;
    {   // entry: the first tail level's b and bt from global memory, x = 0
        const TailLevel<R> &T = A.L[0];
        int s0, s1;
        tail_owned(C, T, s0, s1);
        const long long g0 = (long long)s0 * T.slab;
        for (int q = tid; q < (s1 - s0) * T.slab; q += kTailThreads) {
            C.sm[T.off + q] = mk2<R>(R(0), R(0));
            C.sm[T.off + T.cap + q] = __ldcg(T.g.b + g0 + q);
            C.sm[T.off + 2 * T.cap + q] = __ldcg(T.g.bt + g0 + q);
        }
    }
    tail_sync<CL>();                    // every CTA resident and loaded before any remote read
    for (int l = 0; l + 1 < A.nlev; l++) {
        for (int q = 0; q < A.nu1; q++)
            for (int colour = 0; colour < 2; colour++) {
                tail_colour<R, DIM, CL>(C, A.L[l], colour);
                tail_sync<CL>();
            }
        if (A.nu1 > 0) tail_restrict<R, DIM, CL, true>(C, A.L[l], A.L[l + 1]);
        else tail_restrict<R, DIM, CL, false>(C, A.L[l], A.L[l + 1]);
        tail_sync<CL>();
    }
    {   // coarsest: x = Minv b for the unknowns of the owned cells, one warp per row
        const TailLevel<R> &T = A.L[A.nlev - 1];
        int s0, s1;
        tail_owned(C, T, s0, s1);
        const int lane = threadIdx.x, warp = threadIdx.y;
        const int r0 = 2 * s0 * T.slab, r1 = 2 * s1 * T.slab;
        for (int row = r0 + warp; row < r1; row += kBY) {
            R acc = R(0);
            for (int c = lane; c < A.nc; c += 32) {
                const int cell = c >> 1;
                const int n0 = T.g.n0, n1 = T.g.n1;
                const int i = cell % n0, j = (cell / n0) % n1, k = cell / (n0 * n1);
                const V2 bv = *tail_at<R, DIM, CL>(C, T, 1, i, j, k);
                acc += __ldg(A.Minv + (long long)row * A.nc + c) * ((c & 1) ? bv.y : bv.x);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const int cell = row >> 1;
                const int n0 = T.g.n0, n1 = T.g.n1;
                const int i = cell % n0, j = (cell / n0) % n1, k = cell / (n0 * n1);
                R *xp = reinterpret_cast<R *>(tail_at<R, DIM, CL>(C, T, 0, i, j, k));
                xp[row & 1] = acc;
            }
        }
        tail_sync<CL>();
    }
    for (int l = A.nlev - 2; l >= 0; l--) {
        tail_prolong<R, DIM, CL>(C, A.L[l + 1], A.L[l], A.bc);
        tail_sync<CL>();
        for (int q = 0; q < A.nu2; q++)
            for (int colour = 0; colour < 2; colour++) {
                tail_colour<R, DIM, CL>(C, A.L[l], colour);
                tail_sync<CL>();
            }
    }
    {   // exit: the first tail level's x to global memory
        const TailLevel<R> &T = A.L[0];
        int s0, s1;
        tail_owned(C, T, s0, s1);
        const long long g0 = (long long)s0 * T.slab;
        for (int q = tid; q < (s1 - s0) * T.slab; q += kTailThreads) T.g.x[g0 + q] = C.sm[T.off + q];
    }
    tail_sync<CL>();                    // no CTA leaves while another may still read its shared memory
}

}  // namespace cmg
