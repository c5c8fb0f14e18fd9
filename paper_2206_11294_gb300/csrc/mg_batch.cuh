// Batched solve of many independent problems of uneven sizes (C ABI:
// mg_batch_create / mg_batch_solve / mg_batch_destroy).
//
// The problems are existing handles (each with its own hierarchy and
// coefficients).  Their V-cycles are aligned at the finest level: stage d of
// the down phase smooths and restricts depth d of every problem deeper than
// d + 1 levels, one coarse stage solves every problem's coarsest level, and
// the up phase mirrors the down phase.  Each stage is ONE persistent kernel
// over a table of virtual blocks (level, block) spanning all problems; the
// whole cycle, with the per-problem stopping test, is captured once as a CUDA
// graph and replayed until every problem has stopped.  Convergence is decided
// on the device per problem with the same rule as mg_solve, and a stopped
// problem's blocks do nothing, so each problem runs exactly the cycles it
// would run alone, through the same per-block device functions.
//
// Included by mg_capi.cu (it needs the handle's layout).

namespace {

struct BLevel {                 // one (problem, level), device side
    Level<double> d;
    Level<float> f;
    double2 *xalt;
    float2 *xalt32;
    double2 *delta;             // finest level, mixed precision: the correction from the initial guess
                                // (the handle's staging area); x keeps the initial guess
    BcFlags bc;
    int problem;
};

struct BProb {                  // one problem, device side
    double2 *partial;
    unsigned int *ticket;
    const double *Minv;
    const float *Minv32;
    const double *Lb, *Uc;      // the coarsest level's factors, when its solve uses them (k_coarse_lu)
    const int *piv;
    const double *dinv;
    const int *err;
    int kl;
    int nc;
    int coarse;                 // index of its coarsest level in the BLevel table
    int npartial;
    float2 *x32_0;              // finest-level FP32 correction (mixed)
};

struct BSetupLevel {            // one (problem, level) of the batched set-up
    SetupGeom gm;
    SetupOut out;
    SetupFine fine;             // the level below (coarse levels only)
    int problem;
    int *err;                   // the problem's set-up error flags
};

struct BIo {                    // one problem's solve inputs, device side
    const double2 *rhs;
    const double2 *xin;         // initial guess (device), or NULL when already in place
    double2 *xout;              // result destination (device), or NULL
    BcVals bv;
    int axisym;
    double r0, h;
};

struct BState {                 // per-problem solve state, device side
    double n0[2];
    double nk[2];
    int cycles;
    int active;
};

constexpr int kBatchThreads = 256;
constexpr int kBatchBlocksPerSM = 8;    // default persistent blocks per SM

template <typename R> __device__ __forceinline__ const Level<R> &pick(const BLevel &L);
template <> __device__ __forceinline__ const Level<double> &pick<double>(const BLevel &L) { return L.d; }
template <> __device__ __forceinline__ const Level<float> &pick<float>(const BLevel &L) { return L.f; }
template <typename R> __device__ __forceinline__ typename Vec<R>::v2 *pick_alt(const BLevel &L);
template <> __device__ __forceinline__ double2 *pick_alt<double>(const BLevel &L) { return L.xalt; }
template <> __device__ __forceinline__ float2 *pick_alt<float>(const BLevel &L) { return L.xalt32; }

template <typename R, int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_rbgs_colour(const BLevel *__restrict__ lv,
                                                                const BState *__restrict__ st,
                                                                const int2 *__restrict__ tab, int n, int colour) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> L = pick<R>(B);
        const int gx = ((L.n0 + 1) / 2 + kBX - 1) / kBX, gy = (L.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        rbgs_colour_block<R, DIM>(L, colour, bx, by, bz);
    }
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(kBatchThreads, sizeof(R) == 4 ? 8 : 4)
    kb_rbgs_fused2d(const BLevel *__restrict__ lv, const BState *__restrict__ st, const int2 *__restrict__ tab, int n,
                    int to_alt) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> L = pick<R>(B);
        typename Vec<R>::v2 *xa = pick_alt<R>(B);
        const int gx = (L.n0 + TX - 1) / TX;
        const int bx = e.y % gx, by = e.y / gx;
        if (to_alt) rbgs_fused2d_block<R, TX, TY>(L, L.x, xa, bx, by);
        else rbgs_fused2d_block<R, TX, TY>(L, xa, L.x, bx, by);
    }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_restrict(const BLevel *__restrict__ lv,
                                                             const BState *__restrict__ st,
                                                             const int2 *__restrict__ tab, int n, int red) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> F = pick<R>(B);
        const Level<R> Cc = pick<R>(lv[e.x + 1]);
        const int gx = (Cc.n0 + kBX - 1) / kBX, gy = (Cc.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        if (red) residual_restrict_block<R, DIM, true, true>(F, Cc, bx, by, bz);
        else residual_restrict_block<R, DIM, true, false>(F, Cc, bx, by, bz);
    }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_prolong(const BLevel *__restrict__ lv,
                                                            const BState *__restrict__ st,
                                                            const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> F = pick<R>(B);
        const Level<R> Cc = pick<R>(lv[e.x + 1]);
        const BcFlags bc = B.bc;
        const int gx = (F.n0 + kBX - 1) / kBX, gy = (F.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        prolong_add_block<R, DIM>(Cc, F, bc, bx, by, bz);
    }
}

// Coarsest solves of all problems: one warp per row of x = Minv b.
template <typename R>
__global__ void __launch_bounds__(kBatchThreads) kb_coarse(const BLevel *__restrict__ lv,
                                                           const BProb *__restrict__ pr,
                                                           const BState *__restrict__ st,
                                                           const int2 *__restrict__ tab, int n) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        if (!st[e.x].active) continue;
        const BProb &P = pr[e.x];
        const int row = e.y * (kBatchThreads / 32) + warp;
        if (row >= P.nc) continue;
        const Level<R> C = pick<R>(lv[P.coarse]);
        const R *Mi = (const R *)(sizeof(R) == 8 ? (const void *)P.Minv : (const void *)P.Minv32);
        const R *b = reinterpret_cast<const R *>(C.b);
        R acc = R(0);
        for (int c = lane; c < P.nc; c += 32) acc += Mi[(long long)row * P.nc + c] * b[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) reinterpret_cast<R *>(C.x)[row] = acc;
    }
}

// Coarsest solves of the problems that keep the factors (ids): one block each.
template <typename R>
__global__ void __launch_bounds__(kLuSolveThreads) kb_coarse_lu(const BLevel *__restrict__ lv,
                                                                const BProb *__restrict__ pr,
                                                                const BState *__restrict__ st,
                                                                const int *__restrict__ ids) {
    extern __shared__ double blusm[];
    const int p = ids[blockIdx.x];
    if (!st[p].active) return;
    const BProb &P = pr[p];
    const Level<R> C = pick<R>(lv[P.coarse]);
    coarse_lu_solve_block<R>(P.Lb, P.Uc, P.piv, P.dinv, P.nc, P.kl, P.kl, reinterpret_cast<const R *>(C.b),
                             reinterpret_cast<R *>(C.x), P.err, blusm);
}


template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_setup_fine(const BSetupLevel *__restrict__ sl,
                                                               const SetupIn *__restrict__ in,
                                                               const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BSetupLevel &L = sl[e.x];
        const int gx = (L.gm.n[0] + kBX - 1) / kBX, gy = (L.gm.n[1] + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        setup_fine_block<DIM>(L.gm, in[L.problem], L.out, L.err, bx, by, bz);
    }
}

template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_setup_coarse(const BSetupLevel *__restrict__ sl,
                                                                 const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BSetupLevel &L = sl[e.x];
        const int gx = (L.gm.n[0] + kBX - 1) / kBX, gy = (L.gm.n[1] + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        setup_coarse_block<DIM>(L.gm, L.fine, L.out, L.err, bx, by, bz);
    }
}

// Dense coarsest matrices of all problems (zeroed first by kb_zero_coarse).
struct BCoarse {
    int n[3];
    const double2 *G0, *G1, *G2;
    const dq *D;
    const double *l4;
    double *M;
    double *Minv;
    float *Minv32;
    int *piv;
    double *dinv;
    double *Mwork;                // banded path: columns of the inverse before the transpose
    int nc, kl;
    int *err;
};

// Banded path of the coarsest inverses (kBandSmemMax < nc), all problems in
// three launches: one 32 x 32 block per problem factors; a 2D grid solves
// the columns (x: column blocks, y: problem); a 2D grid transposes (and
// rounds the FP32 copy for mixed precision).
__global__ void __launch_bounds__(1024) kb_band_lu_big(const BCoarse *__restrict__ co, const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.x]];
    band_lu_block(C.M, C.nc, C.kl, C.kl, C.piv, C.dinv, C.err);
}

__global__ void __launch_bounds__(128) kb_band_inv_cols_big(const BCoarse *__restrict__ co,
                                                            const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.y]];
    band_inv_col(C.M, C.piv, C.dinv, C.nc, C.kl, C.kl, C.Mwork, C.err, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void kb_transpose_big(const BCoarse *__restrict__ co, const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.y]];
    const int n = C.nc;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (long long)n * n;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / n), j = (int)(q - (long long)i * n);
        const double v = C.Mwork[(long long)j * n + i];
        C.Minv[q] = v;
        if (C.Minv32) C.Minv32[q] = (float)v;
    }
}

__global__ void __launch_bounds__(kBatchThreads) kb_zero_coarse(const BCoarse *__restrict__ co, int count) {
    for (int p = blockIdx.y; p < count; p += gridDim.y) {
        const long long m = (long long)co[p].nc * co[p].nc;
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x)
            co[p].M[q] = 0.0;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_coarse_assemble(const BCoarse *__restrict__ co, int count) {
    for (int p = blockIdx.y; p < count; p += gridDim.y) {
        const BCoarse &C = co[p];
        const long long N = (long long)C.n[0] * C.n[1] * C.n[2];
        const long long n = 2 * N;
        for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
            const int i = (int)(c % C.n[0]), j = (int)((c / C.n[0]) % C.n[1]), k = (int)(c / ((long long)C.n[0] * C.n[1]));
            const dq d = C.D[c];
            double *M = C.M;
            M[(2 * c) * n + 2 * c] = d.a;
            M[(2 * c) * n + 2 * c + 1] = d.b;
            M[(2 * c + 1) * n + 2 * c] = d.c;
            M[(2 * c + 1) * n + 2 * c + 1] = d.d;
            const long long f0 = (long long)i + (long long)(C.n[0] + 1) * ((long long)j + (long long)C.n[1] * k);
            const long long f1 = (long long)i + (long long)C.n[0] * ((long long)j + (long long)(C.n[1] + 1) * k);
            const double w4 = C.l4[c];
            auto put = [&](long long nb, double2 g) {
                M[(2 * c) * n + 2 * nb] = g.x;
                M[(2 * c + 1) * n + 2 * nb] = w4 * g.x;
                M[(2 * c + 1) * n + 2 * nb + 1] = g.y;
            };
            if (i > 0) put(c - 1, C.G0[f0]);
            if (i < C.n[0] - 1) put(c + 1, C.G0[f0 + 1]);
            if (j > 0) put(c - C.n[0], C.G1[f1]);
            if (j < C.n[1] - 1) put(c + C.n[0], C.G1[f1 + C.n[0]]);
            if (DIM == 3) {
                const long long pl = (long long)C.n[0] * C.n[1];
                if (k > 0) put(c - pl, C.G2[c]);
                if (k < C.n[2] - 1) put(c + pl, C.G2[c + pl]);
            }
        }
    }
}

// Windowed path of the coarsest inverses (window_path): one block per problem
// factors (the factors in the problem's work array: Lb, then Uc); a 2D grid
// of warp groups (x: column groups, y: problem) computes the inverse.
__global__ void __launch_bounds__(kWinThreads) kb_band_lu_window(const BCoarse *__restrict__ co,
                                                                  const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.x]];
    band_lu_window_block(C.M, C.nc, C.kl, C.kl, C.piv, C.dinv, C.Mwork, C.Mwork + (long long)C.nc * C.kl, C.err);
}

// Columns of U over their pivots (scale_uc), for the problems that keep the factors: a 2D grid (x: chunks of a
// problem's entries, y: problem).
__global__ void __launch_bounds__(256) kb_scale_uc(const BCoarse *__restrict__ co, const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.y]];
    scale_uc(C.Mwork + (long long)C.nc * C.kl, C.dinv, C.nc, C.kl, C.kl, C.err,
             blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// The blocked LU on one cluster per problem (band_lu_blocked_block): cluster c factors problem ids[c].
__global__ void __launch_bounds__(kLuBlockedThreads) kb_band_lu_blocked(const BCoarse *__restrict__ co,
                                                                        const int *__restrict__ ids) {
    extern __shared__ double bbsm[];
    const BCoarse &C = co[ids[blockIdx.x / kLuClusterCtas]];
    band_lu_blocked_block(C.M, C.nc, C.kl, C.kl, C.piv, C.dinv, C.Mwork, C.Mwork + (long long)C.nc * C.kl, C.err,
                          bbsm);
}

__global__ void __launch_bounds__(256) kb_band_inv_block(const BCoarse *__restrict__ co, const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.y]];
    const int j0 = blockIdx.x * (blockDim.x >> 5);
    if (j0 >= C.nc) return;
    band_inv_block(C.Mwork, C.Mwork + (long long)C.nc * C.kl, C.piv, C.dinv, C.nc, C.kl, C.kl, C.Minv, C.Minv32,
                   C.err, j0);
}

// Coarsest inverses of the problems listed in ids (nc <= kBandSmemMax): the
// single-warp LU, one block per problem; then the columns, one warp per 32.
__global__ void __launch_bounds__(kLUThreads) kb_band_lu_warp(const BCoarse *__restrict__ co,
                                                               const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.x]];
    band_lu_warp_block(C.M, C.nc, C.kl, C.kl, C.piv, C.dinv, C.err);
}

__global__ void __launch_bounds__(32 * kInvRows) kb_band_inv_cols_warp(const BCoarse *__restrict__ co,
                                                                      const int *__restrict__ ids) {
    const BCoarse &C = co[ids[blockIdx.y]];
    if ((int)blockIdx.x * 32 >= C.nc) return;
    band_inv_cols_warp_block(C.M, C.piv, C.dinv, C.nc, C.kl, C.kl, C.Minv, C.Minv32, blockIdx.x, C.err);
}

// Finest-level right-hand sides (and initial guesses) of all problems.
template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_prep(const BLevel *__restrict__ lv, const BIo *__restrict__ io,
                                                         const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        const BIo &P = io[B.problem];
        const Level<double> &L = B.d;    // in global memory: the boundary call takes its address
        const int gx = (L.n0 + kBX - 1) / kBX, gy = (L.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        prep_rhs_block<DIM>(L, P.rhs, P.xin, P.bv, P.axisym, P.r0, P.h, bx, by, bz);
    }
}

// A problem's flags: err[0] set-up errors, err[2] its finest-level cells marked
// for FP64 block updates (mixed precision).
__global__ void kb_zero_err(const BCoarse *__restrict__ co, int count) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < count; p += gridDim.x * blockDim.x) {
        co[p].err[0] = 0;
        co[p].err[2] = 0;
    }
}

__global__ void kb_gather_err(const BCoarse *__restrict__ co, int count, int *__restrict__ out) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < count; p += gridDim.x * blockDim.x) {
        out[p] = co[p].err[0];
        out[count + p] = co[p].err[2];
    }
}

// Results of all problems to the callers' device arrays.
__global__ void __launch_bounds__(kBatchThreads) kb_copy_out(const BLevel *__restrict__ lv, const BIo *__restrict__ io,
                                                             const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        double2 *dst = io[B.problem].xout;
        const long long c = (long long)e.y * kBatchThreads + threadIdx.x;
        if (dst && c < B.d.N) dst[c] = B.d.x[c];
    }
}

__device__ __forceinline__ bool batch_converged(const double n0[2], const double nk[2], double rtol) {
    if (!(rtol > 0.0)) return false;
    for (int f = 0; f < 2; f++) {
        const double q = n0[f] > 0.0 ? nk[f] / n0[f] : 0.0;
        if (!(q <= rtol)) return false;
    }
    return true;
}

// After a block stored its partial: the problem's last block sums them (in
// order), updates that problem's state with mg_solve's stopping rule and
// counts it in active_count if it continues.
__device__ __forceinline__ void batch_finish(const BProb &P, BState &S, int local, double2 s, int initial,
                                             double rtol, int max_cycles, int *active_count) {
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    if (tid == 0) {
        P.partial[local] = s;
        __threadfence();
        last = atomicAdd(P.ticket, 1u) == (unsigned)P.npartial - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int q = tid; q < P.npartial; q += nthr) {
        const double2 v = __ldcg(P.partial + q);
        a += v.x;
        b += v.y;
    }
    block_sum2(a, b);
    if (tid == 0) {
        const double nk[2] = {sqrt(a), sqrt(b)};
        *P.ticket = 0u;
        if (initial) {
            S.n0[0] = nk[0];
            S.n0[1] = nk[1];
            S.nk[0] = nk[0];
            S.nk[1] = nk[1];
            S.cycles = 0;
            const bool ok = batch_converged(S.n0, nk, rtol) || (nk[0] == 0.0 && nk[1] == 0.0);
            S.active = (!ok && max_cycles > 0) ? 1 : 0;
        } else {
            S.nk[0] = nk[0];
            S.nk[1] = nk[1];
            S.cycles += 1;
            const bool ok = batch_converged(S.n0, nk, rtol);
            S.active = (!ok && S.cycles < max_cycles) ? 1 : 0;
        }
        atomicAdd(active_count, S.active);
    }
}

// Stopping norm of every (active) problem's finest level (FP64 path).
template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_norm(const BLevel *__restrict__ lv, const BProb *__restrict__ pr,
                                                         BState *__restrict__ st, const int2 *__restrict__ tab, int n,
                                                         int initial, int red, double rtol, int max_cycles,
                                                         int *__restrict__ active_count) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        __syncthreads();
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        const int p = B.problem;
        if (!initial && !st[p].active) continue;
        const Level<double> L = B.d;
        int bx, by, bz;
        block_coords(e.y, norm_gx(L.n0), norm_gy(L.n1), bx, by, bz);
        const double2 s = (red && !initial) ? norm_block<DIM, true>(L, bx, by, bz) : norm_block<DIM, false>(L, bx, by, bz);
        batch_finish(pr[p], st[p], e.y, s, initial, rtol, max_cycles, active_count);
    }
}

// Mixed precision: FP64 residual into the FP32 correction problem, with the norm.
template <int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_residual64(const BLevel *__restrict__ lv,
                                                               const BProb *__restrict__ pr, BState *__restrict__ st,
                                                               const int2 *__restrict__ tab, int n, int initial,
                                                               double rtol, int max_cycles,
                                                               int *__restrict__ active_count) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        __syncthreads();
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        const int p = B.problem;
        if (!initial && !st[p].active) continue;
        Level<double> L = B.d;
        int bx, by, bz;
        block_coords(e.y, norm_gx(L.n0), norm_gy(L.n1), bx, by, bz);
        // defect correction: the initial call stores r0 = b - A x0 over b and sets delta = 0; later calls
        // form r0 - A delta
        if (!initial) L.x = B.delta;
        const double2 s = residual64_to32_block<DIM>(L, B.f.b, B.f.bt, B.f.x, initial ? L.b : nullptr,
                                                     initial ? B.delta : nullptr, bx, by, bz);
        batch_finish(pr[p], st[p], e.y, s, initial, rtol, max_cycles, active_count);
    }
}

// Mixed precision, at the end: x = x0 + delta.
__global__ void __launch_bounds__(kBatchThreads) kb_finish_correction(const BLevel *__restrict__ lv,
                                                                      const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        const long long c = (long long)e.y * kBatchThreads + threadIdx.x;
        if (c >= B.d.N) continue;
        const double2 a = B.d.x[c], d = B.delta[c];
        B.d.x[c] = make_double2(a.x + d.x, a.y + d.y);
    }
}

// Mixed precision: delta += e32 on the finest level of active problems.
__global__ void __launch_bounds__(kBatchThreads) kb_add_correction(const BLevel *__restrict__ lv,
                                                                   const BState *__restrict__ st,
                                                                   const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const long long c = (long long)e.y * kBatchThreads + threadIdx.x;
        if (c >= B.d.N) continue;
        const float2 d = B.f.x[c];
        double2 xv = B.delta[c];
        xv.x += (double)d.x;
        xv.y += (double)d.y;
        B.delta[c] = xv;
    }
}

}  // namespace

struct mg_batch {
    int count;
    int dim;
    mg_options opt;
    cudaStream_t stream;
    int device;
    std::vector<mg_handle *> h;
    int dmax;
    // device tables
    char *mem;
    BLevel *lv;
    BProb *pr;
    BState *st;
    int *active_count;
    int *active_h;                    // pinned
    int2 *tabs;
    // table slices: {offset, count}
    std::vector<std::pair<long long, int>> colour, restr, prolong;
    std::vector<std::pair<long long, int>> fusedt[kTileShapes];   // per tile shape, per depth
    // kernel choices (mg_batch_set_tuning): per depth, and the persistent grid
    int bsweep[kMaxLevels], btile[kMaxLevels];
    int blocks_per_sm, sms;
    std::pair<long long, int> norm, coarse, cells0, cells0g;   // cells0g: level-0 cell grids
    cudaGraphExec_t graph;
    long long graph_kernels;
    long long launches;
    // batched set-up and I/O
    BSetupLevel *sl;
    SetupIn *sin;
    BCoarse *co;
    BIo *io;
    int *inv_ids;
    int *big_ids;                     // problems on the banded path (device)
    int *win_ids;                     // problems on the windowed banded path (device)
    std::vector<int> win_coarse;      // their indices
    bool win_factors = false;         // the windowed-path problems solve from their factors (no inverse)
    size_t lu_smem = 0;               // shared memory of kb_coarse_lu
    int max_nc_win = 0;
    size_t win_smem = 0, win_inv_smem = 0;
    int win_warps = 8;
    int max_nc_big;
    int n_inv_smem;
    size_t inv_smem_bytes;
    size_t inv_cols_smem_bytes;       // the inverse-columns kernel (staged factors)
    int max_nc_small;
    std::vector<int> big_coarse;      // problems whose coarsest inverse takes the banded three-kernel path
    std::pair<long long, int> setup_fine_tab;
    std::vector<std::pair<long long, int>> setup_tab;   // depth 1.. (all levels at that depth)
    char *host_io;                    // pinned staging for the per-call pointer tables
    int *err_d, *err_h;               // per-problem set-up error flags (device, pinned host)
};

namespace {

// Persistent grid: at most blocks_per_sm blocks per SM, each looping over the table.
unsigned batch_grid(const mg_batch *b, int n) {
    const int cap = b->sms * b->blocks_per_sm;
    return (unsigned)std::max(1, std::min(n, cap));
}

template <typename R, int TX, int TY>
void b_fused_pair(mg_batch *b, cudaStream_t s, int d, int t) {
    const int2 *ft = b->tabs + b->fusedt[t][d].first;
    const int nf = b->fusedt[t][d].second;
    kb_rbgs_fused2d<R, TX, TY><<<batch_grid(b, nf), kBlock, 0, s>>>(b->lv, b->st, ft, nf, 1);
    kb_rbgs_fused2d<R, TX, TY><<<batch_grid(b, nf), kBlock, 0, s>>>(b->lv, b->st, ft, nf, 0);
}

template <typename R, int DIM>
void b_smooth(mg_batch *b, cudaStream_t s, int d, int sweeps) {
    const int2 *ct = b->tabs + b->colour[d].first;
    const int nc = b->colour[d].second;
    int q = 0;
    if (DIM == 2 && b->bsweep[d] == MG_SWEEP_FUSED) {
        const int t = b->btile[d];
        for (; q + 1 < sweeps; q += 2) {
            if (t == 1) b_fused_pair<R, kTileX[1], kTileY[1]>(b, s, d, 1);
            else if (t == 2) b_fused_pair<R, kTileX[2], kTileY[2]>(b, s, d, 2);
            else b_fused_pair<R, kTileX[0], kTileY[0]>(b, s, d, 0);
            b->launches += 2;
        }
    }
    for (; q < sweeps; q++) {
        kb_rbgs_colour<R, DIM><<<batch_grid(b, nc), kBlock, 0, s>>>(b->lv, b->st, ct, nc, 0);
        kb_rbgs_colour<R, DIM><<<batch_grid(b, nc), kBlock, 0, s>>>(b->lv, b->st, ct, nc, 1);
        b->launches += 2;
    }
}

template <typename R, int DIM>
void b_vcycle(mg_batch *b, cudaStream_t s) {
    for (int d = 0; d + 1 < b->dmax; d++) {
        if (b->colour[d].second == 0) continue;
        b_smooth<R, DIM>(b, s, d, b->opt.nu1);
        const int nr = b->restr[d].second;
        kb_restrict<R, DIM><<<batch_grid(b, nr), kBlock, 0, s>>>(b->lv, b->st, b->tabs + b->restr[d].first, nr,
                                                              b->opt.nu1 > 0);
        b->launches++;
    }
    const int ncs = b->coarse.second;
    if (ncs > 0) {
        kb_coarse<R><<<batch_grid(b, ncs), kBatchThreads, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->coarse.first, ncs);
        b->launches++;
    }
    if (b->win_factors) {
        raise_smem_limit((const void *)kb_coarse_lu<R>, (int)b->lu_smem);
        kb_coarse_lu<R><<<(unsigned)b->win_coarse.size(), kLuSolveThreads, b->lu_smem, s>>>(b->lv, b->pr, b->st,
                                                                                            b->win_ids);
        b->launches++;
    }
    for (int d = b->dmax - 2; d >= 0; d--) {
        if (b->colour[d].second == 0) continue;
        const int np = b->prolong[d].second;
        kb_prolong<R, DIM><<<batch_grid(b, np), kBlock, 0, s>>>(b->lv, b->st, b->tabs + b->prolong[d].first, np);
        b->launches++;
        b_smooth<R, DIM>(b, s, d, b->opt.nu2);
    }
}

template <int DIM>
void b_norm(mg_batch *b, cudaStream_t s, int initial) {
    cudaMemsetAsync(b->active_count, 0, sizeof(int), s);
    const int n = b->norm.second;
    if (b->opt.precision == MG_FP64)
        kb_norm<DIM><<<batch_grid(b, n), kBlock, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->norm.first, n, initial,
                                                      b->opt.nu2 > 0, b->opt.rtol, b->opt.max_cycles,
                                                      b->active_count);
    else
        kb_residual64<DIM><<<batch_grid(b, n), kBlock, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->norm.first, n, initial,
                                                            b->opt.rtol, b->opt.max_cycles, b->active_count);
    b->launches++;
    cudaMemcpyAsync(b->active_h, b->active_count, sizeof(int), cudaMemcpyDeviceToHost, s);
}

// Captures body on the first handle's private stream and times the graph on
// the batch's stream: one warm-up replay, then the best of three.
template <typename F>
mg_status b_time_graph(mg_batch *b, double *ms, F &&body) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaStream_t cs = b->h[0]->cap;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const long long before = b->launches;
    body(cs);
    b->launches = before;
    const cudaError_t le = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("batch autotune capture: ") + cudaGetErrorString(e));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, b->stream);
    for (int t = 0; t < 3 && e == cudaSuccess; t++) {
        e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        if (e == cudaSuccess && f < best) best = f;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(ex);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("batch autotune timing: ") + cudaGetErrorString(e));
    *ms = best;
    return MG_OK;
}

template <typename R, int DIM>
mg_status b_autotune_impl(mg_batch *b, int reps, double *cycle_ms) {
    mg_status st;
    for (int d = 0; d + 1 < b->dmax; d++) {
        if (b->colour[d].second == 0) continue;
        const int ncand = DIM == 2 ? 1 + kTileShapes : 1;
        double best = 1e30;
        int kind = MG_SWEEP_COLOUR, tile = 0;
        for (int c = 0; c < ncand; c++) {
            b->bsweep[d] = c == 0 ? MG_SWEEP_COLOUR : MG_SWEEP_FUSED;
            b->btile[d] = c == 0 ? 0 : c - 1;
            double ms = 0.0;
            st = b_time_graph(b, &ms, [&](cudaStream_t s) {
                for (int r = 0; r < reps; r++) b_smooth<R, DIM>(b, s, d, 2);
            });
            if (st) return st;
            if (ms < best) { best = ms; kind = b->bsweep[d]; tile = b->btile[d]; }
        }
        b->bsweep[d] = kind;
        b->btile[d] = tile;
    }
    const int cand[] = {1, 2, 4, 8, 16, 32};
    double best = 1e30;
    int pick = kBatchBlocksPerSM;
    for (int c : cand) {
        b->blocks_per_sm = c;
        double ms = 0.0;
        st = b_time_graph(b, &ms, [&](cudaStream_t s) {
            for (int r = 0; r < reps; r++) b_vcycle<R, DIM>(b, s);
        });
        if (st) return st;
        if (ms < best) { best = ms; pick = c; }
    }
    b->blocks_per_sm = pick;
    if (cycle_ms) *cycle_ms = best / reps;
    return MG_OK;
}

void b_get_tuning(const mg_batch *b, mg_batch_tuning *t) {
    std::memset(t, 0, sizeof(*t));
    t->depths = b->dmax;
    for (int d = 0; d < MG_MAX_LEVELS; d++) {
        t->sweep[d] = d < b->dmax ? b->bsweep[d] : MG_SWEEP_COLOUR;
        t->tile[d] = d < b->dmax ? b->btile[d] : 0;
    }
    t->blocks_per_sm = b->blocks_per_sm;
}

void b_drop_graph(mg_batch *b) {
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
}

template <int DIM>
void b_step(mg_batch *b, cudaStream_t s) {
    if (b->opt.precision == MG_FP64) {
        b_vcycle<double, DIM>(b, s);
    } else {
        for (int q = 0; q < b->opt.inner_cycles; q++) b_vcycle<float, DIM>(b, s);
        const int n = b->cells0.second;
        kb_add_correction<<<batch_grid(b, n), kBatchThreads, 0, s>>>(b->lv, b->st, b->tabs + b->cells0.first, n);
        b->launches++;
    }
    b_norm<DIM>(b, s, 0);
}

bool same_options(const mg_options &a, const mg_options &c) {
    return a.nu1 == c.nu1 && a.nu2 == c.nu2 && a.precision == c.precision && a.rtol == c.rtol &&
           a.max_cycles == c.max_cycles && a.inner_cycles == c.inner_cycles && a.cycle == c.cycle &&
           a.smoother == c.smoother && a.fp64_jump_ratio == c.fp64_jump_ratio && a.coarse_solve == c.coarse_solve;
}

void add_blocks(std::vector<int2> &t, int level_index, long long blocks) {
    for (long long q = 0; q < blocks; q++) t.push_back(make_int2(level_index, (int)q));
}

}  // namespace

extern "C" {

mg_status mg_batch_create(int count, mg_handle *const *handles, mg_batch **out) {
    if (!out || !handles || count < 1) return fail(MG_ERR_INVALID_ARG, "mg_batch_create: bad arguments");
    *out = nullptr;
    for (int q = 0; q < count; q++) {
        if (!handles[q]) return fail(MG_ERR_INVALID_ARG, "mg_batch_create: NULL handle");
        const mg_handle *h0 = handles[0], *h = handles[q];
        if (h->grid.dim != h0->grid.dim || !same_options(h->opt, h0->opt) || h->stream != h0->stream ||
            h->device != h0->device)
            return fail(MG_ERR_INVALID_ARG,
                        "mg_batch_create: handles must share dim, options (nu1, nu2, precision, rtol, "
                        "max_cycles, inner_cycles), stream and device");
    }
    if (handles[0]->opt.cycle != MG_CYCLE_V) return fail(MG_ERR_INVALID_ARG, "mg_batch_create: batches run V-cycles");
    if (handles[0]->opt.smoother != MG_SMOOTH_RBGS)
        return fail(MG_ERR_INVALID_ARG, "mg_batch_create: batches smooth by red-black block Gauss-Seidel");
    mg_batch *b = new (std::nothrow) mg_batch();
    if (!b) return fail(MG_ERR_OOM, "host allocation failed");
    b->count = count;
    b->dim = handles[0]->grid.dim;
    b->opt = handles[0]->opt;
    b->stream = handles[0]->stream;
    b->device = handles[0]->device;
    b->h.assign(handles, handles + count);
    DeviceGuard dg(b->device);
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || b->sms < 1) {
        cudaGetLastError();
        b->sms = 152;
    }
    b->blocks_per_sm = kBatchBlocksPerSM;
    for (int d = 0; d < kMaxLevels; d++) {
        b->bsweep[d] = (b->dim == 2 && b->opt.precision == MG_MIXED) ? MG_SWEEP_FUSED : MG_SWEEP_COLOUR;
        b->btile[d] = 0;
    }
    // host-side tables
    std::vector<BLevel> lv;
    std::vector<BProb> pr(count);
    std::vector<int> base(count);
    b->dmax = 0;
    for (int p = 0; p < count; p++) {
        const mg_handle *h = handles[p];
        base[p] = (int)lv.size();
        b->dmax = std::max(b->dmax, h->nlev);
        for (int l = 0; l < h->nlev; l++) {
            const LevelBuf &L = h->L[l];
            BLevel d;
            std::memset(&d, 0, sizeof(d));
            d.d = view<double>(L);
            if (h->opt.precision == MG_MIXED) d.f = view<float>(L);
            d.xalt = L.xalt;
            d.xalt32 = L.xalt32;
            d.delta = l == 0 ? reinterpret_cast<double2 *>(h->stage) : nullptr;
            d.bc = bc_flags(h->grid);
            d.problem = p;
            lv.push_back(d);
        }
        pr[p].partial = h->partial;
        pr[p].ticket = h->ticket;
        pr[p].Minv = h->Minv;
        pr[p].Minv32 = h->Minv32;
        pr[p].Lb = h->coarse_factors ? h->Mwork : nullptr;
        pr[p].Uc = h->coarse_factors ? h->Mwork + (long long)h->nc * h->coarse_kl : nullptr;
        pr[p].piv = h->piv;
        pr[p].dinv = h->dinv;
        pr[p].err = h->err_d;
        pr[p].kl = h->coarse_kl;
        pr[p].nc = h->nc;
        pr[p].coarse = base[p] + h->nlev - 1;
        pr[p].npartial = h->npartial;
        pr[p].x32_0 = h->L[0].x32;
    }
    std::vector<int2> tabs;
    auto slice = [&](std::vector<int2> &t) {
        std::pair<long long, int> s{(long long)tabs.size(), (int)t.size()};
        tabs.insert(tabs.end(), t.begin(), t.end());
        return s;
    };
    const int dim = b->dim;
    for (int d = 0; d + 1 < b->dmax; d++) {
        std::vector<int2> tc, tf[kTileShapes], tr, tp;
        for (int p = 0; p < count; p++) {
            const mg_handle *h = handles[p];
            if (h->nlev - 1 <= d) continue;
            const LevelBuf &F = h->L[d], &Cl = h->L[d + 1];
            const int li = base[p] + d;
            add_blocks(tc, li, (long long)cell_grid(F, dim, (F.n[0] + 1) / 2).x * cell_grid(F, dim, 1).y *
                                   cell_grid(F, dim, 1).z);
            if (dim == 2)
                for (int t = 0; t < kTileShapes; t++)
                    add_blocks(tf[t], li, (long long)((F.n[0] + kTileX[t] - 1) / kTileX[t]) *
                                              ((F.n[1] + kTileY[t] - 1) / kTileY[t]));
            const dim3 gc = cell_grid(Cl, dim, Cl.n[0]);
            add_blocks(tr, li, (long long)gc.x * gc.y * gc.z);
            const dim3 gf = cell_grid(F, dim, F.n[0]);
            add_blocks(tp, li, (long long)gf.x * gf.y * gf.z);
        }
        b->colour.push_back(slice(tc));
        for (int t = 0; t < kTileShapes; t++) b->fusedt[t].push_back(slice(tf[t]));
        b->restr.push_back(slice(tr));
        b->prolong.push_back(slice(tp));
    }
    std::vector<int2> tn, tnorm, tco, tcell;
    for (int p = 0; p < count; p++) {
        const mg_handle *h = handles[p];
        const dim3 g0 = cell_grid(h->L[0], dim, h->L[0].n[0]);
        add_blocks(tn, base[p], (long long)g0.x * g0.y * g0.z);
        const dim3 gn = norm_grid(h->L[0], dim);
        add_blocks(tnorm, base[p], (long long)gn.x * gn.y * gn.z);
        if (!h->coarse_factors)
            for (int r = 0; r < (h->nc + 7) / 8; r++) tco.push_back(make_int2(p, r));
        add_blocks(tcell, base[p], (h->L[0].N + kBatchThreads - 1) / kBatchThreads);
    }
    b->cells0g = slice(tn);
    b->norm = slice(tnorm);
    b->coarse = slice(tco);
    b->cells0 = slice(tcell);
    b->setup_fine_tab = b->cells0g;
    for (int d = 1; d < b->dmax; d++) {
        std::vector<int2> ts;
        for (int p = 0; p < count; p++) {
            const mg_handle *h = handles[p];
            if (h->nlev <= d) continue;
            const dim3 gl = cell_grid(h->L[d], dim, h->L[d].n[0]);
            add_blocks(ts, base[p] + d, (long long)gl.x * gl.y * gl.z);
        }
        b->setup_tab.push_back(slice(ts));
    }
    // set-up descriptors, one per (problem, level), same indexing as lv
    std::vector<BSetupLevel> sl(lv.size());
    std::vector<BCoarse> co(count);
    std::vector<int> inv_ids;
    for (int p = 0; p < count; p++) {
        const mg_handle *h = handles[p];
        const bool mixed = h->opt.precision == MG_MIXED;
        double hl = h->grid.h;
        for (int l = 0; l < h->nlev; l++) {
            BSetupLevel &S = sl[base[p] + l];
            std::memset(&S, 0, sizeof(S));
            for (int a = 0; a < 3; a++) {
                S.gm.n[a] = h->L[l].n[a];
                for (int sd = 0; sd < 2; sd++)
                    S.gm.fac[a][sd] = (a < dim && h->grid.bc[a][sd] == MG_BC_DIRICHLET) ? 2.0 : 0.0;
            }
            S.gm.axisym = h->grid.axisym;
            S.gm.r0 = h->grid.r0;
            S.gm.h = hl;
            S.gm.ih2 = 1.0 / (hl * hl);
            S.out = setup_out(h->L[l], mixed);
            if (l > 0) S.fine = setup_fine_of(h->L[l - 1], hl / 2.0);
            S.problem = p;
            S.err = h->err_d;
            hl *= 2.0;
        }
        const LevelBuf &c = h->L[h->nlev - 1];
        BCoarse &C = co[p];
        for (int a = 0; a < 3; a++) C.n[a] = c.n[a];
        C.G0 = c.G[0];
        C.G1 = c.G[1];
        C.G2 = dim == 3 ? c.G[2] : c.G[0];
        C.D = c.D;
        C.l4 = c.l4;
        C.M = h->Mtmp;
        C.Minv = h->Minv;
        C.Minv32 = mixed ? h->Minv32 : nullptr;
        C.piv = h->piv;
        C.dinv = h->dinv;
        C.Mwork = h->Mwork;
        C.nc = h->nc;
        const int off = dim == 3 ? c.n[0] * c.n[1] : c.n[0];
        C.kl = std::min(h->nc - 1, 2 * off + 1);
        C.err = h->err_d;
        if (h->nc <= kBandSmemMax) {
            inv_ids.push_back(p);
            b->inv_smem_bytes = std::max(b->inv_smem_bytes, sizeof(double) * (size_t)h->nc * h->nc);
            b->inv_cols_smem_bytes = std::max(b->inv_cols_smem_bytes,
                                              sizeof(double) * (size_t)inv_smem_doubles(h->nc, C.kl, C.kl));
            b->max_nc_small = std::max(b->max_nc_small, h->nc);
        } else if (window_path(h->nc, C.kl)) {
            b->win_coarse.push_back(p);
            b->win_factors = h->coarse_factors;      // one coarse_solve option for the whole batch
            b->lu_smem = std::max(b->lu_smem, (size_t)coarse_lu_smem(h->nc, C.kl, C.kl));
            b->max_nc_win = std::max(b->max_nc_win, h->nc);
            b->win_smem = std::max(b->win_smem, (size_t)band_window_smem(C.kl, C.kl));
            b->win_warps = std::min(b->win_warps, inv_block_warps(h->nc, C.kl));
        } else {
            b->big_coarse.push_back(p);
            b->max_nc_big = std::max(b->max_nc_big, h->nc);
        }
    }
    for (int p : b->win_coarse)          // the staging of the common warp count
        b->win_inv_smem = std::max(b->win_inv_smem, (size_t)band_inv_block_smem(co[p].nc, co[p].kl, co[p].kl,
                                                                                 b->win_warps));
    b->n_inv_smem = (int)inv_ids.size();
    // one device allocation for the tables
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) / 256 * 256;
        const size_t o = off;
        off += bytes;
        return o;
    };
    const size_t o_lv = take(sizeof(BLevel) * lv.size()), o_pr = take(sizeof(BProb) * count),
                 o_st = take(sizeof(BState) * count), o_ac = take(sizeof(int)),
                 o_tab = take(sizeof(int2) * std::max<size_t>(1, tabs.size())),
                 o_sl = take(sizeof(BSetupLevel) * sl.size()), o_sin = take(sizeof(SetupIn) * count),
                 o_co = take(sizeof(BCoarse) * count), o_io = take(sizeof(BIo) * count),
                 o_ids = take(sizeof(int) * std::max<size_t>(1, inv_ids.size())), o_err = take(sizeof(int) * 2 * count),
                 o_big = take(sizeof(int) * std::max<size_t>(1, b->big_coarse.size())),
                 o_win = take(sizeof(int) * std::max<size_t>(1, b->win_coarse.size()));
    cudaError_t e = cudaMalloc(&b->mem, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(MG_ERR_OOM, "batch table allocation failed");
    }
    b->lv = reinterpret_cast<BLevel *>(b->mem + o_lv);
    b->pr = reinterpret_cast<BProb *>(b->mem + o_pr);
    b->st = reinterpret_cast<BState *>(b->mem + o_st);
    b->active_count = reinterpret_cast<int *>(b->mem + o_ac);
    b->tabs = reinterpret_cast<int2 *>(b->mem + o_tab);
    b->sl = reinterpret_cast<BSetupLevel *>(b->mem + o_sl);
    b->sin = reinterpret_cast<SetupIn *>(b->mem + o_sin);
    b->co = reinterpret_cast<BCoarse *>(b->mem + o_co);
    b->io = reinterpret_cast<BIo *>(b->mem + o_io);
    b->inv_ids = reinterpret_cast<int *>(b->mem + o_ids);
    b->big_ids = reinterpret_cast<int *>(b->mem + o_big);
    b->win_ids = reinterpret_cast<int *>(b->mem + o_win);
    b->err_d = reinterpret_cast<int *>(b->mem + o_err);
    if (cudaMemcpy(b->lv, lv.data(), sizeof(BLevel) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->pr, pr.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        (tabs.size() && cudaMemcpy(b->tabs, tabs.data(), sizeof(int2) * tabs.size(), cudaMemcpyHostToDevice) !=
                            cudaSuccess) ||
        cudaMemcpy(b->sl, sl.data(), sizeof(BSetupLevel) * sl.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->co, co.data(), sizeof(BCoarse) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        (inv_ids.size() && cudaMemcpy(b->inv_ids, inv_ids.data(), sizeof(int) * inv_ids.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
        (b->win_coarse.size() && cudaMemcpy(b->win_ids, b->win_coarse.data(), sizeof(int) * b->win_coarse.size(),
                                            cudaMemcpyHostToDevice) != cudaSuccess) ||
        (b->big_coarse.size() && cudaMemcpy(b->big_ids, b->big_coarse.data(), sizeof(int) * b->big_coarse.size(),
                                            cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(b->st, 0, sizeof(BState) * count) != cudaSuccess ||
        cudaMallocHost(&b->host_io, std::max(sizeof(SetupIn), sizeof(BIo)) * count) != cudaSuccess ||
        cudaMallocHost(&b->err_h, sizeof(int) * 2 * count) != cudaSuccess ||
        cudaMallocHost(&b->active_h, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        mg_batch_destroy(b);
        return fail(MG_ERR_CUDA, "batch table upload failed");
    }
    *out = b;
    return MG_OK;
}

mg_status mg_batch_solve(mg_batch *b, const double *const *rhs, double *const *x, int on_device, mg_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!b || !rhs || !x) return fail(MG_ERR_INVALID_ARG, "mg_batch_solve: bad arguments");
    for (int p = 0; p < b->count; p++) {
        mg_status st = check_handle(b->h[p], true);
        if (st) return st;
        if (!rhs[p] || !x[p]) return fail(MG_ERR_INVALID_ARG, "mg_batch_solve: NULL rhs or x");
    }
    DeviceGuard dg(b->device);
    cudaStream_t s = b->stream;
    for (int p = 0; p < b->count; p++) CK(cudaStreamWaitEvent(s, b->h[p]->ev_inv, 0));   // per-handle set-ups
    {
        BIo *io = reinterpret_cast<BIo *>(b->host_io);
        for (int p = 0; p < b->count; p++) {
            mg_handle *h = b->h[p];
            BIo &o = io[p];
            std::memset(&o, 0, sizeof(o));
            o.bv = bc_vals(h->grid);
            o.axisym = h->grid.axisym;
            o.r0 = h->grid.r0;
            o.h = h->grid.h;
            if (on_device) {
                if (!aligned16(rhs[p]) || !aligned16(x[p]))
                    return fail(MG_ERR_INVALID_ARG, "device pair arrays must be 16-byte aligned");
                o.rhs = reinterpret_cast<const double2 *>(rhs[p]);
                o.xin = reinterpret_cast<const double2 *>(x[p]);
                o.xout = reinterpret_cast<double2 *>(x[p]);
            } else {
                CK(cudaMemcpyAsync(h->stage, rhs[p], sizeof(double2) * h->L[0].N, cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(h->L[0].x, x[p], sizeof(double2) * h->L[0].N, cudaMemcpyHostToDevice, s));
                o.rhs = reinterpret_cast<const double2 *>(h->stage);
            }
        }
        CK(cudaMemcpyAsync(b->io, io, sizeof(BIo) * b->count, cudaMemcpyHostToDevice, s));
        const int n = b->cells0g.second;
        if (b->dim == 2) kb_prep<2><<<batch_grid(b, n), kBlock, 0, s>>>(b->lv, b->io, b->tabs + b->cells0g.first, n);
        else kb_prep<3><<<batch_grid(b, n), kBlock, 0, s>>>(b->lv, b->io, b->tabs + b->cells0g.first, n);
        b->launches++;
        CK(cudaGetLastError());
    }
    if (b->dim == 2) b_norm<2>(b, s, 1);
    else b_norm<3>(b, s, 1);
    const bool mixed = b->opt.precision == MG_MIXED;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    int active = *b->active_h;
    if (active > 0 && !b->graph) {
        cudaGraph_t graph = nullptr;
        // capture on the first handle's private stream
        cudaStream_t cs = b->h[0]->cap;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        const long long before = b->launches;
        if (b->dim == 2) b_step<2>(b, cs);
        else b_step<3>(b, cs);
        b->graph_kernels = b->launches - before;
        b->launches = before;
        const cudaError_t le = cudaGetLastError();    // a launch refused while capturing
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(MG_ERR_CUDA, std::string("batch graph capture: a launch failed: ") + cudaGetErrorString(le));
        }
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    int steps = 0;
    while (active > 0 && steps <= b->opt.max_cycles) {
        CK(cudaGraphLaunch(b->graph, s));
        b->launches += b->graph_kernels;
        CK(cudaStreamSynchronize(s));
        active = *b->active_h;
        steps++;
    }
    if (mixed) {
        const int n = b->cells0.second;
        kb_finish_correction<<<batch_grid(b, n), kBatchThreads, 0, s>>>(b->lv, b->tabs + b->cells0.first, n);
        b->launches++;
    }
    std::vector<BState> host(b->count);
    CK(cudaMemcpyAsync(host.data(), b->st, sizeof(BState) * b->count, cudaMemcpyDeviceToHost, s));
    if (on_device) {
        const int n = b->cells0.second;
        kb_copy_out<<<batch_grid(b, n), kBatchThreads, 0, s>>>(b->lv, b->io, b->tabs + b->cells0.first, n);
        b->launches++;
        CK(cudaGetLastError());
    } else {
        for (int p = 0; p < b->count; p++) {
            mg_status st = x_out(b->h[p], x[p], 0);
            if (st) return st;
        }
    }
    CK(cudaStreamSynchronize(s));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    bool all_ok = true;
    for (int p = 0; p < b->count; p++) {
        const BState &S = host[p];
        const mg_handle *h = b->h[p];
        const bool zero = S.n0[0] == 0.0 && S.n0[1] == 0.0;
        bool ok = zero || !(h->opt.rtol > 0.0) || converged(S.n0, S.nk, h->opt.rtol);
        if (S.cycles == 0 && converged(S.n0, S.n0, h->opt.rtol)) ok = true;
        all_ok = all_ok && ok;
        if (stats) {
            mg_stats &o = stats[p];
            std::memset(&o, 0, sizeof(o));
            o.cycles = h->opt.precision == MG_FP64 ? S.cycles : S.cycles * h->opt.inner_cycles;
            o.outer = S.cycles;
            o.r0[0] = S.n0[0];
            o.r0[1] = S.n0[1];
            o.rfinal[0] = S.nk[0];
            o.rfinal[1] = S.nk[1];
            o.seconds = secs;
            o.status = ok ? MG_OK : MG_ERR_NOT_CONVERGED;
            o.levels = h->nlev;
            o.fp64_cells = h->jcells;
        }
    }
    if (!all_ok) return fail(MG_ERR_NOT_CONVERGED, "at least one problem did not converge in max_cycles");
    return MG_OK;
}

mg_status mg_batch_set_coeffs(mg_batch *b, const double *const *lambda, const double *const *face_alpha,
                              const double *const *face_k, int on_device) {
    if (!b || !lambda || !face_alpha || !face_k) return fail(MG_ERR_INVALID_ARG, "mg_batch_set_coeffs: bad arguments");
    const int dim = b->dim;
    for (int p = 0; p < b->count; p++) {
        if (!lambda[p]) return fail(MG_ERR_INVALID_ARG, "NULL lambda");
        for (int a = 0; a < dim; a++)
            if (!face_alpha[3 * p + a] || !face_k[3 * p + a]) return fail(MG_ERR_INVALID_ARG, "NULL face array");
    }
    DeviceGuard dg(b->device);
    cudaStream_t s = b->stream;
    for (int p = 0; p < b->count; p++) CK(cudaStreamWaitEvent(s, b->h[p]->ev_inv, 0));   // in-flight inverses
    SetupIn *in = reinterpret_cast<SetupIn *>(b->host_io);
    for (int p = 0; p < b->count; p++) {
        mg_handle *h = b->h[p];
        h->coeffs_set = false;
        const LevelBuf &f = h->L[0];
        SetupIn &q = in[p];
        std::memset(&q, 0, sizeof(q));
        if (on_device) {
            q.lam = lambda[p];
            for (int a = 0; a < dim; a++) {
                q.fa[a] = face_alpha[3 * p + a];
                q.fk[a] = face_k[3 * p + a];
            }
        } else {
            double *st = reinterpret_cast<double *>(h->stage);
            CK(cudaMemcpyAsync(st, lambda[p], sizeof(double) * 4 * f.N, cudaMemcpyHostToDevice, s));
            q.lam = st;
            double *ptr = st + 4 * f.N;
            for (int a = 0; a < dim; a++) {
                CK(cudaMemcpyAsync(ptr, face_alpha[3 * p + a], sizeof(double) * f.nf[a], cudaMemcpyHostToDevice, s));
                q.fa[a] = ptr;
                ptr += f.nf[a];
                CK(cudaMemcpyAsync(ptr, face_k[3 * p + a], sizeof(double) * f.nf[a], cudaMemcpyHostToDevice, s));
                q.fk[a] = ptr;
                ptr += f.nf[a];
            }
        }
    }
    CK(cudaMemcpyAsync(b->sin, in, sizeof(SetupIn) * b->count, cudaMemcpyHostToDevice, s));
    kb_zero_err<<<(b->count + 255) / 256, 256, 0, s>>>(b->co, b->count);
    const int nf = b->setup_fine_tab.second;
    if (dim == 2) kb_setup_fine<2><<<batch_grid(b, nf), kBlock, 0, s>>>(b->sl, b->sin, b->tabs + b->setup_fine_tab.first, nf);
    else kb_setup_fine<3><<<batch_grid(b, nf), kBlock, 0, s>>>(b->sl, b->sin, b->tabs + b->setup_fine_tab.first, nf);
    b->launches += 2;
    for (size_t d = 0; d < b->setup_tab.size(); d++) {
        const int n = b->setup_tab[d].second;
        if (n == 0) continue;
        if (dim == 2) kb_setup_coarse<2><<<batch_grid(b, n), kBlock, 0, s>>>(b->sl, b->tabs + b->setup_tab[d].first, n);
        else kb_setup_coarse<3><<<batch_grid(b, n), kBlock, 0, s>>>(b->sl, b->tabs + b->setup_tab[d].first, n);
        b->launches++;
    }
    const unsigned gy = (unsigned)std::min(b->count, 65535);
    kb_zero_coarse<<<dim3(16, gy), kBatchThreads, 0, s>>>(b->co, b->count);
    if (dim == 2) kb_coarse_assemble<2><<<dim3(4, gy), kBatchThreads, 0, s>>>(b->co, b->count);
    else kb_coarse_assemble<3><<<dim3(4, gy), kBatchThreads, 0, s>>>(b->co, b->count);
    b->launches += 2;
    if (b->n_inv_smem > 0) {
        CK(raise_smem_limit((const void *)kb_band_lu_warp, (int)(sizeof(double) * kBandSmemMax * kBandSmemMax)));
        kb_band_lu_warp<<<b->n_inv_smem, kLUThreads, b->inv_smem_bytes, s>>>(b->co, b->inv_ids);
        CK(raise_smem_limit((const void *)kb_band_inv_cols_warp, (int)b->inv_cols_smem_bytes));
        kb_band_inv_cols_warp<<<dim3((b->max_nc_small + 31) / 32, b->n_inv_smem), dim3(32, kInvRows),
                                b->inv_cols_smem_bytes, s>>>(b->co, b->inv_ids);
        b->launches += 2;
    }
    if (!b->win_coarse.empty()) {           // the windowed LU, a block per problem, then the inverse's columns
        const unsigned nw = (unsigned)b->win_coarse.size();
        CK(raise_smem_limit((const void *)kb_band_lu_window, (int)b->win_smem));
        CK(raise_smem_limit((const void *)kb_band_inv_block, (int)b->win_inv_smem));
        {   // blocked over one cluster per problem where every problem's shared memory fits and all the clusters
            // run at once (one SM per CTA), else one block each: a second wave of clusters would cost more than
            // the blocked LU saves over all problems factoring side by side
            size_t bsm = 0;
            bool blocked = (long long)nw * kLuClusterCtas <= (long long)b->sms;
            for (int p : b->win_coarse) {
                const mg_handle *hp = b->h[p];
                blocked = blocked && lu_blocked_ok(hp->nc, hp->coarse_kl);
                bsm = std::max(bsm, (size_t)band_blocked_smem(hp->nc, hp->coarse_kl, hp->coarse_kl));
            }
            if (blocked)
                CK(launch_cluster(kb_band_lu_blocked, s, (int)nw, kLuBlockedThreads, bsm, (const BCoarse *)b->co,
                                  (const int *)b->win_ids));
            else
                kb_band_lu_window<<<nw, kWinThreads, b->win_smem, s>>>(b->co, b->win_ids);
        }
        b->launches++;
        if (b->win_factors)                 // the cycles solve from Lb and the scaled Uc (kb_coarse_lu)
            kb_scale_uc<<<dim3(64, nw), 256, 0, s>>>(b->co, b->win_ids);
        else
            kb_band_inv_block<<<dim3((unsigned)((b->max_nc_win + b->win_warps - 1) / b->win_warps), nw),
                                32 * b->win_warps, b->win_inv_smem, s>>>(b->co, b->win_ids);
        b->launches++;
    }
    if (!b->big_coarse.empty()) {           // medium coarsest levels: the banded path, all at once
        const unsigned nb = (unsigned)b->big_coarse.size();
        kb_band_lu_big<<<nb, dim3(32, 32, 1), 0, s>>>(b->co, b->big_ids);
        kb_band_inv_cols_big<<<dim3((unsigned)((b->max_nc_big + 127) / 128), nb), 128, 0, s>>>(b->co, b->big_ids);
        kb_transpose_big<<<dim3(64, nb), 256, 0, s>>>(b->co, b->big_ids);
        b->launches += 3;
    }
    kb_gather_err<<<(b->count + 255) / 256, 256, 0, s>>>(b->co, b->count, b->err_d);
    b->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b->err_h, b->err_d, sizeof(int) * 2 * b->count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int p = 0; p < b->count; p++) b->h[p]->jcells = b->h[p]->L[0].jflag ? b->err_h[b->count + p] : 0;
    for (int p = 0; p < b->count; p++) {
        const int e = b->err_h[p];
        if (e & 1) return fail(MG_ERR_INVALID_COEFF, "problem " + std::to_string(p) + ": non-finite coefficient");
        if (e & 2) return fail(MG_ERR_INVALID_COEFF, "problem " + std::to_string(p) + ": singular local block");
        if (e & 4) return fail(MG_ERR_INVALID_COEFF, "problem " + std::to_string(p) + ": singular coarsest matrix");
    }
    for (int p = 0; p < b->count; p++) b->h[p]->coeffs_set = true;
    return MG_OK;
}

mg_status mg_batch_get_tuning(const mg_batch *b, mg_batch_tuning *out) {
    if (!b || !out) return fail(MG_ERR_INVALID_ARG, "mg_batch_get_tuning: NULL argument");
    b_get_tuning(b, out);
    return MG_OK;
}

mg_status mg_batch_set_tuning(mg_batch *b, const mg_batch_tuning *t) {
    if (!b || !t) return fail(MG_ERR_INVALID_ARG, "mg_batch_set_tuning: NULL argument");
    for (int d = 0; d < b->dmax; d++) {
        if (t->sweep[d] != MG_SWEEP_COLOUR && t->sweep[d] != MG_SWEEP_FUSED)
            return fail(MG_ERR_INVALID_ARG, "sweep kind must be MG_SWEEP_COLOUR or MG_SWEEP_FUSED");
        if (t->sweep[d] == MG_SWEEP_FUSED && b->dim != 2)
            return fail(MG_ERR_INVALID_ARG, "fused sweeps are for 2D grids");
        if (t->tile[d] < 0 || t->tile[d] >= kTileShapes) return fail(MG_ERR_INVALID_ARG, "tile shape out of range");
    }
    if (t->blocks_per_sm < 1 || t->blocks_per_sm > 32)
        return fail(MG_ERR_INVALID_ARG, "blocks_per_sm must be in [1, 32]");
    DeviceGuard dg(b->device);
    CK(cudaStreamSynchronize(b->stream));
    for (int d = 0; d < b->dmax; d++) {
        b->bsweep[d] = t->sweep[d];
        b->btile[d] = t->tile[d];
    }
    b->blocks_per_sm = t->blocks_per_sm;
    b_drop_graph(b);
    return MG_OK;
}

mg_status mg_batch_autotune(mg_batch *b, int reps, mg_batch_tuning *out, double *cycle_ms) {
    if (!b) return fail(MG_ERR_INVALID_ARG, "batch is NULL");
    if (reps < 1 || reps > 1000) return fail(MG_ERR_INVALID_ARG, "reps must be in [1, 1000]");
    for (int p = 0; p < b->count; p++)
        if (!b->h[p]->coeffs_set) return fail(MG_ERR_STATE, "mg_batch_autotune: a problem has no coefficients");
    DeviceGuard dg(b->device);
    cudaStream_t s = b->stream;
    CK(cudaStreamSynchronize(s));
    for (int p = 0; p < b->count; p++) CK(cudaStreamWaitEvent(s, b->h[p]->ev_inv, 0));
    // scratch state to zeros and every problem active: all candidates run on
    // the same finite data over the whole batch
    for (int p = 0; p < b->count; p++)
        for (int l = 0; l < b->h[p]->nlev; l++) {
            const LevelBuf &L = b->h[p]->L[l];
            void *ptrs[8] = {L.x, L.b, L.bt, L.xalt, L.x32, L.b32, L.bt32, L.xalt32};
            const size_t sz[8] = {16, 16, 16, 16, 8, 8, 8, 8};
            for (int q = 0; q < 8; q++)
                if (ptrs[q]) CK(cudaMemsetAsync(ptrs[q], 0, sz[q] * (size_t)L.N, s));
        }
    std::vector<BState> act(b->count);
    std::memset(act.data(), 0, sizeof(BState) * b->count);
    for (auto &a : act) a.active = 1;
    CK(cudaMemcpyAsync(b->st, act.data(), sizeof(BState) * b->count, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    const bool mixed = b->opt.precision == MG_MIXED;
    mg_status st;
    if (b->dim == 2) st = mixed ? b_autotune_impl<float, 2>(b, reps, cycle_ms) : b_autotune_impl<double, 2>(b, reps, cycle_ms);
    else st = mixed ? b_autotune_impl<float, 3>(b, reps, cycle_ms) : b_autotune_impl<double, 3>(b, reps, cycle_ms);
    b_drop_graph(b);
    CK(cudaStreamSynchronize(s));
    if (st) return st;
    if (out) b_get_tuning(b, out);
    return MG_OK;
}

mg_status mg_batch_counters(const mg_batch *b, long long *launches) {
    if (!b) return fail(MG_ERR_INVALID_ARG, "batch is NULL");
    if (launches) *launches = b->launches;
    return MG_OK;
}

mg_status mg_batch_destroy(mg_batch *b) {
    if (!b) return MG_OK;
    DeviceGuard dg(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->active_h) cudaFreeHost(b->active_h);
    if (b->host_io) cudaFreeHost(b->host_io);
    if (b->err_h) cudaFreeHost(b->err_h);
    if (b->mem) cudaFree(b->mem);
    delete b;
    return MG_OK;
}

}  // extern "C"
