// Host side of the C ABI declared in include/coupledmg.h: argument checks,
// the device hierarchy (one arena), coefficient set-up, the V-cycle launch
// sequence (captured once per handle as a CUDA graph and replayed), the FP64
// defect-correction loop and the mixed-precision refinement loop.
//
// The outer loop is the paper's (Sec. 3, after Eq. 34): residual, stop test,
// correction solve by one multigrid V-cycle, update.  The FP64 path runs the
// V-cycle in place on x, which equals "correction from zero, then add" for a
// linear cycle.  The mixed path solves the correction in FP32 from zero and
// adds it in FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "coupledmg.h"
#include "mg_host.h"
#include "mg_kernels.cuh"
#include "mg_tail.cuh"
#include "mg_async.cuh"
#include "mg_assemble.cuh"
#include "mg_momentum.cuh"

using namespace cmg;

namespace {

constexpr int kMaxLevels = 32;
constexpr int kMaxCoarseUnknowns = 2048;
constexpr int kSetupGraphs = 4;
constexpr size_t kAlign = 256;
constexpr size_t kTailSmemMax = 200 * 1024;   // shared memory a tail CTA may use

thread_local std::string g_err;

mg_status fail(mg_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(MG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

struct LevelBuf {
    int n[3];
    long long N;
    long long nf[3];
    double2 *x, *b;
    double2 *xalt;          // ping-pong partner of x for fused sweeps (2D) and Jacobi sweeps
    double2 *G[3];
    dq *S;                  // scaled local terms s [[l1, l2], [0, l3]] (set-up)
    dq *D, *Dinv, *W;
    double *l4;
    double2 *bt;            // Dinv b
    float2 *x32, *b32, *bt32;
    float2 *xalt32;
    float2 *G32[3];
    float2 *G32p0;          // FP32 axis-0 faces with an even row pitch p0 (2D mixed: tensor-map loads)
    int p0;
    fq *D32, *Dinv32, *W32;
    float *l4_32;
    unsigned char *jflag;   // finest level, mixed: cells whose 2x2 block the FP32 cycles apply in FP64
    int *jcount;            // their count (device)
    double jratio;          // the face-coefficient ratio that marks them
};

}  // namespace

mg_status cmg::set_error(mg_status s, const char *msg) {
    g_err = msg ? msg : "";
    return s;
}

// The grid alone: dimensions, spacing, boundary kinds and values.
mg_status cmg::check_grid_geom(const mg_grid *g) {
    if (!g) return fail(MG_ERR_INVALID_ARG, "grid must not be NULL");
    if (g->dim != 2 && g->dim != 3) return fail(MG_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (g->axisym && g->dim != 2) return fail(MG_ERR_INVALID_ARG, "axisymmetric grids are 2D (r, z)");
    for (int a = 0; a < 3; a++) {
        if (g->n[a] < 1) return fail(MG_ERR_INVALID_ARG, "every n[a] must be >= 1");
        if (a >= g->dim && g->n[a] != 1) return fail(MG_ERR_INVALID_ARG, "n[2] must be 1 for a 2D grid");
    }
    if (g->n[0] > (1 << 28) || g->n[1] > 8 * 65535 || g->n[2] > 65535)
        return fail(MG_ERR_INVALID_ARG, "grid too large for the launch geometry (n1 <= 524280, n2 <= 65535)");
    if (!(g->h > 0.0) || !std::isfinite(g->h)) return fail(MG_ERR_INVALID_ARG, "h must be positive and finite");
    if (g->axisym && (!(g->r0 >= 0.0) || !std::isfinite(g->r0)))
        return fail(MG_ERR_INVALID_ARG, "r0 must be >= 0 and finite");
    for (int a = 0; a < g->dim; a++)
        for (int s = 0; s < 2; s++) {
            const int k = g->bc[a][s];
            if (k != MG_BC_WALL && k != MG_BC_DIRICHLET && k != MG_BC_AXIS)
                return fail(MG_ERR_INVALID_ARG, "unknown boundary kind");
            if (k == MG_BC_AXIS && !(g->axisym && a == 0 && s == 0 && g->r0 == 0.0))
                return fail(MG_ERR_INVALID_ARG, "MG_BC_AXIS only on the low-r side of an axisymmetric grid with r0 = 0");
            if (k == MG_BC_DIRICHLET && (!std::isfinite(g->bc_T[a][s]) || !std::isfinite(g->bc_p[a][s])))
                return fail(MG_ERR_INVALID_ARG, "Dirichlet values must be finite");
        }
    if (g->axisym && g->r0 == 0.0 && g->bc[0][0] == MG_BC_DIRICHLET)
        return fail(MG_ERR_INVALID_ARG, "the symmetry axis (r0 = 0) cannot carry a Dirichlet condition");
    return MG_OK;
}

struct mg_handle {
    mg_grid grid;
    mg_options opt;
    int device;
    cudaStream_t stream;   // caller's stream: all work runs here
    cudaStream_t cap;      // private stream used only to capture graphs
    cudaStream_t aux;      // private stream: the coarsest inverse, overlapping the solve's start
    cudaEvent_t ev_asm;    // coarsest matrix assembled (main stream)
    cudaEvent_t ev_inv;    // coarsest inverse ready (aux stream); cycle graphs wait on it
    cudaEvent_t ev_last;   // end of the last call that returned with work pending on the stream
    int *errh;             // pinned host copy of err_d
    long long jcells;      // finest-level cells whose 2x2 block the FP32 cycles apply in FP64 (last set-up)
    int nlev;
    LevelBuf L[kMaxLevels];
    char *arena;
    size_t arena_bytes;
    bool owns_arena;
    char *stage;
    size_t stage_bytes;
    int nc;                // unknowns of the coarsest level
    int tail_lev;          // first level of the cluster tail (nlev: no tail)
    int tail_ctas;         // CTAs of the tail's cluster (8, or 16 where allowed)
    int sweep[kMaxLevels]; // per level: MG_SWEEP_COLOUR or MG_SWEEP_FUSED
    int tile[kMaxLevels];  // per level: fused tile shape (index into kTileX / kTileY)
    int persistent;        // colour sweeps, restriction, prolongation: one persistent wave (1) or a block per tile (0)
    int overlap;           // cycle and set-up kernels as programmatic dependent launches (1) or in plain order (0)
    TmaLevel *tmaps;       // tensor maps per (level, precision, tile), built on first use (host memory)
    unsigned char *tmap_ok;
    double *Minv, *Mtmp;   // coarse inverse (NULL when the cycles solve from the factors); assembled matrix
    bool coarse_factors;   // the cycles solve the coarsest level from its LU factors (k_coarse_lu)
    int coarse_kl;         // the coarsest matrix's lower (= upper) bandwidth
    double *Mwork;         // coarse inverse: columns before the transpose (banded path); the window path's factors
    int *piv;              // coarse inverse: pivot rows (banded path)
    double *dinv;          // coarse inverse: reciprocal pivots (banded path)
    float *Minv32;
    double2 *partial;
    int npartial;
    double *norms_d;       // device: [2] latest norms
    unsigned int *ticket;  // device: last-block counter of the norm kernels (re-armed by them)
    int *err_d;
    double *norms_h;       // pinned host: [0..1] latest norms, [2..3] initial norms of a solve
    bool x_stale;          // the handle's x ran an iteration the stop test did not allow: not copied back
    bool coeffs_set;
    cudaGraphExec_t g64, g32;   // FP64 cycle+norm; mixed inner cycles+update+residual
    cudaGraphExec_t gcorr;      // fixed FP64 cycles without norms (correction solves of the momentum predictor)
    cudaGraphExec_t gasync;     // a whole solve with the stop test on the device (mg_solve_async)
    long long async_kernels_pre;   // its kernels outside the loop, and per loop iteration
    long long async_kernels_body;
    cudaStream_t cap2;          // private stream: captures the loop body of gasync
    AsyncStat *astat_d;         // device: the async solve's norms and cycle count
    AsyncStat *astat_h;         // pinned host copy, written at the end of the async solve
    cudaEvent_t ev_a0, ev_a1;   // bracket the last async solve (device time)
    bool async_pending;         // an async solve was enqueued and its statistics not yet read
    bool cond_body;             // capturing a conditional body: no event nodes
    long long graph_kernels_corr;
    struct SetupGraph {         // set-up of the levels for the input pointers in key
        cudaGraphExec_t exec;
        const void *key[7];
        long long kernels;
    } gsetup[kSetupGraphs];     // a few input sets (e.g. double-buffered inputs), replaced round-robin
    int gsetup_next;
    // instrumentation
    long long enq;              // kernels launched since the last reset (graph nodes per replay)
    long long graph_kernels64, graph_kernels32;
    int timing;
    cudaEvent_t ev[2];          // start / end of the timed finest-level smoothing pass
    double smooth_ms;
    long long smooth_launches;
    long long smooth_sweeps;
};

namespace {

// ---------------------------------------------------------------- validation
bool can_coarsen(const int n[3], int dim, int coarse_min) {
    for (int a = 0; a < dim; a++)
        if (n[a] % 2 != 0 || n[a] / 2 < coarse_min) return false;
    return true;
}

mg_status check_grid(const mg_grid *g, const mg_options *o) {
    if (!g || !o) return fail(MG_ERR_INVALID_ARG, "grid and options must not be NULL");
    const mg_status st = check_grid_geom(g);
    if (st) return st;
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 > 16 || o->nu2 > 16 || o->nu1 + o->nu2 == 0)
        return fail(MG_ERR_INVALID_ARG, "nu1, nu2 must be in 0..16 and not both zero");
    if (o->precision != MG_FP64 && o->precision != MG_MIXED) return fail(MG_ERR_INVALID_ARG, "unknown precision");
    if (o->max_cycles < 0 || o->coarse_min < 1 || o->inner_cycles < 1 || o->inner_cycles > 64)
        return fail(MG_ERR_INVALID_ARG, "max_cycles >= 0, coarse_min >= 1, inner_cycles in 1..64");
    if (!std::isfinite(o->rtol)) return fail(MG_ERR_INVALID_ARG, "rtol must be finite");
    if (o->cycle != MG_CYCLE_V && o->cycle != MG_CYCLE_W && o->cycle != MG_CYCLE_F)
        return fail(MG_ERR_INVALID_ARG, "cycle must be MG_CYCLE_V, MG_CYCLE_W or MG_CYCLE_F");
    if (o->smoother != MG_SMOOTH_RBGS && o->smoother != MG_SMOOTH_WJAC)
        return fail(MG_ERR_INVALID_ARG, "smoother must be MG_SMOOTH_RBGS or MG_SMOOTH_WJAC");
    if (o->smoother == MG_SMOOTH_WJAC && !(o->omega > 0.0 && o->omega <= 1.0))
        return fail(MG_ERR_INVALID_ARG, "omega must be in (0, 1] for weighted block Jacobi");
    if (!(o->fp64_jump_ratio == 0.0 || (o->fp64_jump_ratio >= 1.0 && std::isfinite(o->fp64_jump_ratio))))
        return fail(MG_ERR_INVALID_ARG, "fp64_jump_ratio must be 0 (off) or a finite ratio >= 1");
    if (o->coarse_solve != MG_COARSE_AUTO && o->coarse_solve != MG_COARSE_INVERSE)
        return fail(MG_ERR_INVALID_ARG, "coarse_solve must be MG_COARSE_AUTO or MG_COARSE_INVERSE");
    int n[3] = {g->n[0], g->n[1], g->n[2]}, lev = 1;
    while (can_coarsen(n, g->dim, o->coarse_min) && lev < kMaxLevels) {
        for (int a = 0; a < g->dim; a++) n[a] /= 2;
        lev++;
    }
    const long long nc = 2LL * n[0] * n[1] * n[2];
    if (nc > kMaxCoarseUnknowns)
        return fail(MG_ERR_INVALID_ARG, "coarsest level has " + std::to_string(nc) + " unknowns (limit " +
                                             std::to_string(kMaxCoarseUnknowns) +
                                             "): choose sizes with more factors of two");
    return MG_OK;
}

// ---------------------------------------------------------------- arena plan
struct Planner {
    char *base;       // NULL while sizing
    size_t off = 0;
    template <typename T> T *take(long long count) {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (size_t)count;
        return p;
    }
};

dim3 cell_grid(const LevelBuf &l, int dim, int xthreads) {
    return dim3((unsigned)((xthreads + kBX - 1) / kBX), (unsigned)((l.n[1] + kBY - 1) / kBY),
                (unsigned)(dim == 3 ? l.n[2] : 1));
}

// Blocks of the norm / FP64-residual kernels (64 x 32 cells each).
dim3 norm_grid(const LevelBuf &l, int dim) {
    return dim3((unsigned)norm_gx(l.n[0]), (unsigned)norm_gy(l.n[1]), (unsigned)(dim == 3 ? l.n[2] : 1));
}

bool window_path(int n, int kl);

// Lays out every buffer; with base == NULL only computes the size.
void plan(mg_handle *h, char *base, size_t *bytes) {
    Planner P{base};
    const mg_grid &g = h->grid;
    const bool mixed = h->opt.precision == MG_MIXED;
    int n[3] = {g.n[0], g.n[1], g.n[2]};
    h->nlev = 0;
    for (;;) {
        LevelBuf &l = h->L[h->nlev];
        std::memset(&l, 0, sizeof(l));
        for (int a = 0; a < 3; a++) l.n[a] = n[a];
        l.N = (long long)n[0] * n[1] * n[2];
        for (int a = 0; a < 3; a++) {
            l.nf[a] = 1;
            for (int b = 0; b < 3; b++) l.nf[a] *= (b == a) ? n[b] + 1 : n[b];
        }
        l.x = P.take<double2>(l.N);
        l.b = P.take<double2>(l.N);
        const bool pingpong = g.dim == 2 || h->opt.smoother == MG_SMOOTH_WJAC;
        if (pingpong) l.xalt = P.take<double2>(l.N);
        for (int a = 0; a < g.dim; a++) l.G[a] = P.take<double2>(l.nf[a]);
        l.S = P.take<dq>(l.N);
        l.D = P.take<dq>(l.N);
        l.Dinv = P.take<dq>(l.N);
        l.W = P.take<dq>(l.N);
        l.l4 = P.take<double>(l.N);
        l.bt = P.take<double2>(l.N);
        if (mixed) {
            l.x32 = P.take<float2>(l.N);
            l.b32 = P.take<float2>(l.N);
            if (pingpong) l.xalt32 = P.take<float2>(l.N);
            for (int a = 0; a < g.dim; a++) l.G32[a] = P.take<float2>(l.nf[a]);
            if (g.dim == 2) {
                l.p0 = (n[0] + 2) & ~1;
                l.G32p0 = P.take<float2>((long long)l.p0 * n[1]);
            }
            l.D32 = P.take<fq>(l.N);
            l.Dinv32 = P.take<fq>(l.N);
            l.W32 = P.take<fq>(l.N);
            l.l4_32 = P.take<float>(l.N);
            l.bt32 = P.take<float2>(l.N);
            if (h->nlev == 0 && h->opt.fp64_jump_ratio > 0.0) {
                l.jflag = P.take<unsigned char>(l.N);
                l.jratio = h->opt.fp64_jump_ratio;
            }
        }
        h->nlev++;
        if (!can_coarsen(n, g.dim, h->opt.coarse_min) || h->nlev == kMaxLevels) break;
        for (int a = 0; a < g.dim; a++) n[a] /= 2;
    }
    const LevelBuf &f = h->L[0];
    const LevelBuf &c = h->L[h->nlev - 1];
    h->nc = (int)(2 * c.N);
    // band of the coarsest matrix: the farthest neighbour cell is n0 (2D) or
    // n0*n1 (3D) cells away, two unknowns per cell
    h->coarse_kl = std::min(h->nc - 1, 2 * (g.dim == 3 ? c.n[0] * c.n[1] : c.n[0]) + 1);
    h->coarse_factors = h->opt.coarse_solve == MG_COARSE_AUTO && window_path(h->nc, h->coarse_kl);
    // The cluster tail takes the levels below the finest whose cells fit
    // kTailCells, when there are at least two of them (and the coarsest
    // level has an inverse: the tail multiplies by it).
    h->tail_lev = h->nlev;
    for (int l = 1; l < h->nlev && h->opt.smoother == MG_SMOOTH_RBGS; l++)
        if (h->L[l].N <= kTailCells) { h->tail_lev = l; break; }
    if (h->nlev - h->tail_lev < 2 || h->nlev - h->tail_lev > kTailMaxLevels || h->coarse_factors)
        h->tail_lev = h->nlev;
    h->tail_ctas = kTailCtas;
    h->persistent = 0;
    h->overlap = 1;
    // Default kernel choices until mg_autotune / mg_set_tuning: FP32 cycles
    // (mixed precision) sweep fused in 2D; FP64 sweeps are bound by GB300's
    // FP64 pipe, where the fused kernel's recomputed ring costs more than the
    // DRAM traffic it saves, so they run as colour launches.
    for (int l = 0; l < kMaxLevels; l++) {
        h->sweep[l] = (g.dim == 2 && mixed) ? MG_SWEEP_FUSED : MG_SWEEP_COLOUR;
        h->tile[l] = 0;
    }
    long long sumnf = 0;
    for (int a = 0; a < g.dim; a++) sumnf += f.nf[a];
    // lambda, then 1/rho and k of every axis (host-side coefficient intake)
    h->stage_bytes = (size_t)(32 * f.N + 16 * sumnf);
    h->stage = P.take<char>((long long)h->stage_bytes);
    h->Minv = h->coarse_factors ? nullptr : P.take<double>((long long)h->nc * h->nc);
    h->Mtmp = P.take<double>((long long)h->nc * h->nc);
    const bool big = h->nc > kBandSmemMax;
    h->Mwork = big ? P.take<double>((long long)h->nc * h->nc) : nullptr;
    h->piv = P.take<int>(h->nc);
    h->dinv = P.take<double>(h->nc);
    h->Minv32 = mixed && !h->coarse_factors ? P.take<float>((long long)h->nc * h->nc) : nullptr;
    const dim3 gg = norm_grid(f, g.dim);
    h->npartial = (int)(gg.x * gg.y * gg.z);
    h->partial = P.take<double2>(h->npartial);
    h->norms_d = P.take<double>(8);
    h->ticket = P.take<unsigned int>(1);
    h->err_d = P.take<int>(4);            // [0] set-up flags, [1] bounded waits that gave up (per solve), [2] jump cells
    if (h->L[0].jflag) h->L[0].jcount = h->err_d + 2;
    h->astat_d = P.take<AsyncStat>(1);
    *bytes = P.off + kAlign;
}

template <typename R> Level<R> view(const LevelBuf &l);
template <> Level<double> view<double>(const LevelBuf &l) {
    return Level<double>{l.n[0], l.n[1], l.n[2], l.N, l.x, l.b, l.G[0], l.G[1], l.G[2], l.D, l.Dinv, l.l4, l.W, l.bt,
                         l.W, l.bt, l.jflag};
}
template <> Level<float> view<float>(const LevelBuf &l) {
    return Level<float>{l.n[0], l.n[1], l.n[2], l.N, l.x32, l.b32, l.G32[0], l.G32[1], l.G32[2], l.D32, l.Dinv32,
                        l.l4_32, l.W32, l.bt32, l.W, l.bt, nullptr};
}

BcFlags bc_flags(const mg_grid &g) {
    BcFlags f;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) f.dir[a][s] = (a < g.dim && g.bc[a][s] == MG_BC_DIRICHLET) ? 1 : 0;
    return f;
}

BcVals bc_vals(const mg_grid &g) {
    BcVals v;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) {
            v.dir[a][s] = (a < g.dim && g.bc[a][s] == MG_BC_DIRICHLET) ? 1 : 0;
            v.T[a][s] = g.bc_T[a][s];
            v.p[a][s] = g.bc_p[a][s];
        }
    return v;
}

dim3 kBlock(kBX, kBY, 1);

// One persistent wave for a grid-stride kernel over `tiles` tiles: SMs x the
// kernel's resident blocks per SM (from the occupancy calculator, cached per
// kernel and device), at most the number of tiles.
unsigned wave(const void *kernel, long long tiles, int dyn_smem = 0) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;   // (kernel, device) -> SMs x blocks per SM
    int dev = 0;
    cudaGetDevice(&dev);
    int slots = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find({kernel, dev});
        if (it != cache.end()) slots = it->second;
    }
    if (slots == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBX * kBY, dyn_smem) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
            per = 4;
        }
        slots = std::max(1, sms * std::max(1, per));
        std::lock_guard<std::mutex> g(mu);
        cache[{kernel, dev}] = slots;
    }
    return (unsigned)std::max(1LL, std::min(tiles, (long long)slots));
}

long long tiles_of(const dim3 &g) { return (long long)g.x * g.y * g.z; }



// Raises a kernel's dynamic shared-memory limit to at least `bytes`, never
// lowers it.  The limit is a process-wide attribute of the function: setting
// it per launch would race with other threads launching the same kernel with
// more shared memory (their launch fails), so it only grows, under a lock.
cudaError_t raise_smem_limit(const void *fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    int &cur = limit[{fn, dev}];
    if (bytes <= cur) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

unsigned lin_blocks(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// ---------------------------------------------------------------- V-cycle
inline void counted(const mg_handle *h, long long n = 1) { const_cast<mg_handle *>(h)->enq += n; }

// Launches one kernel of a cycle or a set-up in stream s.  With the handle's
// overlap on, as a programmatic dependent of the kernel before it (each of
// these kernels starts with pdl_entry): it is set up while that kernel
// drains.  `cluster` > 0: thread-block clusters of that size.
template <typename... KArgs, typename... Args>
void launch_k(const mg_handle *h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
              int cluster, Args &&...args) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na = 0;
    if (cluster > 0) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = (unsigned)cluster;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        na++;
    }
    if (h->overlap) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        na++;
    }
    cfg.attrs = attr;
    cfg.numAttrs = (unsigned)na;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename R> typename Vec<R>::v2 *xalt_of(const LevelBuf &l);
template <> double2 *xalt_of<double>(const LevelBuf &l) { return l.xalt; }
template <> float2 *xalt_of<float>(const LevelBuf &l) { return l.xalt32; }

template <typename R, int TX, int TY>
void launch_fused(const mg_handle *h, const LevelBuf &lb, const Level<R> &v, cudaStream_t s) {
    const dim3 gf((unsigned)((lb.n[0] + TX - 1) / TX), (unsigned)((lb.n[1] + TY - 1) / TY), 1);
    typename Vec<R>::v2 *xa = xalt_of<R>(lb);
    launch_k(h, k_rbgs_fused2d<R, TX, TY>, gf, kBlock, 0, s, 0, v, v.x, xa);
    launch_k(h, k_rbgs_fused2d<R, TX, TY>, gf, kBlock, 0, s, 0, v, xa, v.x);
}

// Two sweeps in one launch (k_rbgs_fused2d_x2): src -> dst.
template <typename R, int TX, int TY>
void launch_fused_x2(const mg_handle *h, const LevelBuf &lb, const Level<R> &v, const typename Vec<R>::v2 *src,
                     typename Vec<R>::v2 *dst, cudaStream_t s) {
    const dim3 gf((unsigned)((lb.n[0] + TX - 1) / TX), (unsigned)((lb.n[1] + TY - 1) / TY), 1);
    launch_k(h, k_rbgs_fused2d_x2<R, TX, TY>, gf, kBlock, 0, s, 0, v, src, dst);
}

// ---------------------------------------------------------------- TMA sweeps
// Shared memory of the TMA fused sweep with tile `tile`.
template <typename R>
int async_smem(int tile) {
    switch (tile) {
        case 1: return tma_smem_bytes<R, kTileX[1], kTileY[1]>();
        case 2: return tma_smem_bytes<R, kTileX[2], kTileY[2]>();
        default: return tma_smem_bytes<R, kTileX[0], kTileY[0]>();
    }
}
constexpr int kSmemOptInMax = 227 * 1024;

// Whether level l can run the TMA sweep with this tile in precision R.
template <typename R>
bool async_ok(const mg_handle *h, int l, int tile) {
    if (h->grid.dim != 2 || async_smem<R>(tile) > kSmemOptInMax) return false;
    if (sizeof(R) == 4 && ((h->L[l].n[0] & 1) || !h->L[l].G32p0)) return false;   // FP32 rows: 8 n0 bytes
    if (sizeof(R) == 4 && h->L[l].jflag) return false;   // its staged W has no FP64 branch for marked cells
    return true;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static EncodeTiled fn = []() -> EncodeTiled {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

// A 2D map over rows of `width` scalars (row pitch `pitch` scalars), box bx x by.
bool map2d(CUtensorMap *m, bool f32, void *base, long long width, long long pitch, long long rows, int bx, int by) {
    const EncodeTiled enc = encode_tiled();
    if (!enc) return false;
    const long long es = f32 ? 4 : 8;
    const cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(pitch * es)};
    const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The 2x2 blocks W as a 3D map (4 scalars, n0 cells, n1 rows), box 4 x bx x by.
bool map3d_w(CUtensorMap *m, bool f32, void *base, long long n0, long long n1, int bx, int by) {
    const EncodeTiled enc = encode_tiled();
    if (!enc) return false;
    const long long es = f32 ? 4 : 8;
    const cuuint64_t dims[3] = {4, (cuuint64_t)n0, (cuuint64_t)n1};
    const cuuint64_t strides[2] = {(cuuint64_t)(4 * es), (cuuint64_t)(4 * es * n0)};
    const cuuint32_t box[3] = {4, (cuuint32_t)bx, (cuuint32_t)by};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of level l for the TMA sweep with tile (TX, TY), built once per handle.
template <typename R, int TX, int TY>
const TmaLevel *tma_maps(const mg_handle *hc, int l, int tile) {
    mg_handle *h = const_cast<mg_handle *>(hc);
    const int prec = sizeof(R) == 4 ? 1 : 0;
    const int idx = (l * 2 + prec) * kTileShapes + tile;
    if (!h->tmaps) {
        h->tmaps = new (std::nothrow) TmaLevel[kMaxLevels * 2 * kTileShapes];
        h->tmap_ok = new (std::nothrow) unsigned char[kMaxLevels * 2 * kTileShapes]();
        if (!h->tmaps || !h->tmap_ok) return nullptr;
    }
    if (h->tmap_ok[idx]) return &h->tmaps[idx];
    const LevelBuf &b = h->L[l];
    const long long n0 = b.n[0], n1 = b.n[1];
    const bool f32 = prec == 1;
    TmaLevel &m = h->tmaps[idx];
    void *x = f32 ? (void *)b.x32 : (void *)b.x, *xa = f32 ? (void *)b.xalt32 : (void *)b.xalt;
    void *g0 = f32 ? (void *)b.G32p0 : (void *)b.G[0];
    const long long p0 = f32 ? b.p0 : n0 + 1;
    void *g1 = f32 ? (void *)b.G32[1] : (void *)b.G[1];
    void *bt = f32 ? (void *)b.bt32 : (void *)b.bt;
    void *w = f32 ? (void *)b.W32 : (void *)b.W;
    const int W2 = 2 * (TX + 4);
    const bool ok = map2d(&m.x[0], f32, x, 2 * n0, 2 * n0, n1, W2, TY + 4) &&
                    map2d(&m.x[1], f32, xa, 2 * n0, 2 * n0, n1, W2, TY + 4) &&
                    map2d(&m.g0, f32, g0, 2 * (n0 + 1), 2 * p0, n1, W2, TY + 2) &&
                    map2d(&m.g1, f32, g1, 2 * n0, 2 * n0, n1 + 1, W2, TY + 3) &&
                    map2d(&m.bt, f32, bt, 2 * n0, 2 * n0, n1, W2, TY + 2) &&
                    map3d_w(&m.w, f32, w, n0, n1, TX + 4, TY + 2);
    if (!ok) return nullptr;
    h->tmap_ok[idx] = 1;
    return &m;
}

template <typename R, int TX, int TY>
void launch_fused_tma(const mg_handle *h, int l, int tile, const Level<R> &v, cudaStream_t s) {
    const TmaLevel *m = tma_maps<R, TX, TY>(h, l, tile);
    if (!m) return;                           // refused by mg_set_tuning before it can get here
    const LevelBuf &lb = h->L[l];
    const int smem = tma_smem_bytes<R, TX, TY>();
    const void *fn = (const void *)k_rbgs_fused2d_tma<R, TX, TY>;
    raise_smem_limit(fn, smem);
    const long long tiles = (long long)((lb.n[0] + TX - 1) / TX) * ((lb.n[1] + TY - 1) / TY);
    const unsigned grid = wave(fn, tiles, smem);
    typename Vec<R>::v2 *xa = xalt_of<R>(lb);
    launch_k(h, k_rbgs_fused2d_tma<R, TX, TY>, grid, kBlock, smem, s, 0, m->x[0], m->g0, m->g1, m->bt, m->w, v, xa, h->err_d + 1);
    launch_k(h, k_rbgs_fused2d_tma<R, TX, TY>, grid, kBlock, smem, s, 0, m->x[1], m->g0, m->g1, m->bt, m->w, v, v.x, h->err_d + 1);
}

// `sweeps` red-black sweeps on level l with the given kernel choice.  Fused
// (2D only): pairs of sweeps run as fused launches x -> xalt -> x.  Fused
// pairs (MG_SWEEP_FUSED2, 2D only): each pair of sweeps is one launch from
// the buffer that holds the level's values to the other one.  A leftover odd
// sweep (and every non-fused sweep) runs as two colour launches in place.
// alt: the values start in xalt (only after fused pairs).  Returns whether
// they end in xalt.  The values are the same, bit for bit, for every choice.
template <typename R, int DIM>
bool enqueue_sweeps(const mg_handle *h, cudaStream_t s, int l, int sweeps, int kind, int tile, bool alt = false) {
    using V2 = typename Vec<R>::v2;
    const LevelBuf &lb = h->L[l];
    Level<R> v = view<R>(lb);
    V2 *const xm = v.x, *const xa = xalt_of<R>(lb);
    if (alt) v.x = xa;
    int q = 0;
    if (DIM == 2 && kind == MG_SWEEP_FUSED2) {
        for (; q + 1 < sweeps; q += 2) {
            V2 *dst = v.x == xm ? xa : xm;
            if (tile == 1) launch_fused_x2<R, kTileX[1], kTileY[1]>(h, lb, v, v.x, dst, s);
            else if (tile == 2) launch_fused_x2<R, kTileX[2], kTileY[2]>(h, lb, v, v.x, dst, s);
            else launch_fused_x2<R, kTileX[0], kTileY[0]>(h, lb, v, v.x, dst, s);
            v.x = dst;
            counted(h);
        }
    }
    if (DIM == 2 && kind == MG_SWEEP_FUSED) {
        for (; q + 1 < sweeps; q += 2) {
            if (tile == 1) launch_fused<R, kTileX[1], kTileY[1]>(h, lb, v, s);
            else if (tile == 2) launch_fused<R, kTileX[2], kTileY[2]>(h, lb, v, s);
            else launch_fused<R, kTileX[0], kTileY[0]>(h, lb, v, s);
            counted(h, 2);
        }
    }
    if (DIM == 2 && kind == MG_SWEEP_ASYNC) {
        for (; q + 1 < sweeps; q += 2) {
            if (tile == 1) launch_fused_tma<R, kTileX[1], kTileY[1]>(h, l, 1, v, s);
            else if (tile == 2) launch_fused_tma<R, kTileX[2], kTileY[2]>(h, l, 2, v, s);
            else launch_fused_tma<R, kTileX[0], kTileY[0]>(h, l, 0, v, s);
            counted(h, 2);
        }
    }
    const dim3 gr = cell_grid(lb, DIM, (lb.n[0] + 1) / 2);
    if (kind == MG_SWEEP_COLOUR2) {
        const dim3 g2(gr.x, (unsigned)((lb.n[1] + 2 * kBY - 1) / (2 * kBY)), gr.z);
        for (; q < sweeps; q++) {
            launch_k(h, k_rbgs_colour2<R, DIM>, g2, kBlock, 0, s, 0, v, 0);
            launch_k(h, k_rbgs_colour2<R, DIM>, g2, kBlock, 0, s, 0, v, 1);
            counted(h, 2);
        }
    }
    for (; q < sweeps; q++) {
        if (h->persistent) {
            const unsigned gw = wave((const void *)k_rbgs_colour<R, DIM, true>, tiles_of(gr));
            launch_k(h, k_rbgs_colour<R, DIM, true>, gw, kBlock, 0, s, 0, v, 0);
            launch_k(h, k_rbgs_colour<R, DIM, true>, gw, kBlock, 0, s, 0, v, 1);
        } else {
            launch_k(h, k_rbgs_colour<R, DIM, false>, gr, kBlock, 0, s, 0, v, 0);
            launch_k(h, k_rbgs_colour<R, DIM, false>, gr, kBlock, 0, s, 0, v, 1);
        }
        counted(h, 2);
    }
    return v.x != xm;
}

// `sweeps` weighted block Jacobi sweeps on level l, alternating x -> xalt ->
// x; after an odd number the result is copied back into x.
template <typename R, int DIM>
void enqueue_wjac(const mg_handle *h, cudaStream_t s, int l, int sweeps) {
    using V2 = typename Vec<R>::v2;
    const LevelBuf &lb = h->L[l];
    Level<R> v = view<R>(lb);
    V2 *a = v.x, *b = xalt_of<R>(lb);
    const R omega = (R)h->opt.omega;
    const dim3 gr = cell_grid(lb, DIM, lb.n[0]);
    for (int q = 0; q < sweeps; q++) {
        if (h->persistent)
            launch_k(h, k_wjac<R, DIM, true>, wave((const void *)k_wjac<R, DIM, true>, tiles_of(gr)), kBlock, 0, s, 0, v, a, b, omega);
        else
            launch_k(h, k_wjac<R, DIM, false>, gr, kBlock, 0, s, 0, v, a, b, omega);
        counted(h);
        std::swap(a, b);
    }
    if (a != v.x) cudaMemcpyAsync(v.x, a, sizeof(V2) * lb.N, cudaMemcpyDeviceToDevice, s);
}

// Returns whether the level's values end in xalt (fused pairs only; alt:
// they start there).
template <typename R, int DIM>
bool enqueue_smooth(const mg_handle *h, cudaStream_t s, int l, int sweeps, bool alt = false) {
    if (h->opt.smoother == MG_SMOOTH_WJAC) {
        enqueue_wjac<R, DIM>(h, s, l, sweeps);
        return false;
    }
    return enqueue_sweeps<R, DIM>(h, s, l, sweeps, h->sweep[l], h->tile[l], alt);
}

// Fused pairs leave a level's values in xalt after an odd number of pairs;
// a V-cycle needs them back in x at its end: nu1 / 2 + nu2 / 2 even.
bool fused2_ok(const mg_options &o, int dim) {
    return dim == 2 && o.smoother == MG_SMOOTH_RBGS && (o.nu1 / 2 + o.nu2 / 2) % 2 == 0;
}

// Red-black Gauss-Seidel leaves the residual of the colour swept last at zero,
// so the restriction after pre-smoothing evaluates the red children only and
// the norm after post-smoothing the red cells only; Jacobi leaves no such zeros.
bool red_only_after_sweeps(const mg_handle *h) { return h->opt.smoother == MG_SMOOTH_RBGS; }

// The tail kernel runs red-black V-cycles.
bool tail_runs(const mg_handle *h) { return h->opt.cycle == MG_CYCLE_V && h->opt.smoother == MG_SMOOTH_RBGS; }

// Kernel launches and sweeps of one call of enqueue_smooth.
void smooth_launches(int kind, bool dim2, int sweeps, long long *launches, long long *sweeps_out) {
    const bool fused = dim2 && (kind == MG_SWEEP_FUSED || kind == MG_SWEEP_ASYNC || kind == MG_SWEEP_FUSED2);
    const int fused_pairs = fused ? sweeps / 2 : 0;
    *launches = (kind == MG_SWEEP_FUSED2 ? 1LL : 2LL) * fused_pairs + 2LL * (sweeps - 2 * fused_pairs);
    *sweeps_out = sweeps;
}

template <typename R> const R *coarse_inverse(const mg_handle *h);
template <> const double *coarse_inverse<double>(const mg_handle *h) { return h->Minv; }
template <> const float *coarse_inverse<float>(const mg_handle *h) { return h->Minv32; }

// Levels tail_lev .. coarsest as one launch of k_vcycle_tail on one cluster.
template <typename R>
TailArgs<R> tail_args(const mg_handle *h, int first, int ctas, size_t *smem) {
    TailArgs<R> A;
    std::memset(&A, 0, sizeof(A));
    A.nlev = h->nlev - first;
    for (int q = 0; q < A.nlev; q++) A.L[q].g = view<R>(h->L[first + q]);
    const int pairs = tail_layout(A, h->grid.dim, ctas);
    *smem = (size_t)pairs * sizeof(typename Vec<R>::v2);
    A.bc = bc_flags(h->grid);
    A.Minv = coarse_inverse<R>(h);
    A.nc = h->nc;
    A.nu1 = h->opt.nu1;
    A.nu2 = h->opt.nu2;
    return A;
}

template <typename R, int DIM>
void enqueue_tail(const mg_handle *h, cudaStream_t s) {
    size_t smem = 0;
    TailArgs<R> A = tail_args<R>(h, h->tail_lev, h->tail_ctas, &smem);
    if (h->tail_ctas == 1) {                  // one CTA, no cluster
        raise_smem_limit((const void *)k_vcycle_tail<R, DIM, false>, (int)kTailSmemMax);
        launch_k(h, k_vcycle_tail<R, DIM, false>, 1, kBlock, smem, s, 0, A);
        return;
    }
    raise_smem_limit((const void *)k_vcycle_tail<R, DIM, true>, (int)kTailSmemMax);
    launch_k(h, k_vcycle_tail<R, DIM, true>, dim3((unsigned)h->tail_ctas, 1, 1), kBlock, smem, s, h->tail_ctas, A);
}

template <typename R, int DIM>
void enqueue_vcycle(const mg_handle *h, cudaStream_t s, int l, int type);

template <typename R, int DIM>
// One cycle from level l: V, or (type) W / F, whose coarse-grid correction
// visits level l + 1 twice (W then W, F then V), the second visit continuing
// from the first one's coarse solution, except at the exactly solved coarsest
// level.  The tail kernel runs V-cycles only, so W and F cycles never use it.
void enqueue_vcycle(const mg_handle *h, cudaStream_t s, int l, int type) {
    const LevelBuf &lb = h->L[l];
    if (l == h->tail_lev && tail_runs(h)) {
        // the coarsest inverse is computed on the aux stream after each set-up
        // (a conditional body may hold no event node: the async solve waits first)
        if (!h->cond_body) cudaStreamWaitEvent(s, h->ev_inv, cudaEventWaitExternal);
        enqueue_tail<R, DIM>(h, s);
        counted(h);
        return;
    }
    if (l == h->nlev - 1) {
        const Level<R> v = view<R>(lb);
        // the coarsest inverse (or factors) is computed on the aux stream after each set-up
        if (!h->cond_body) cudaStreamWaitEvent(s, h->ev_inv, cudaEventWaitExternal);
        if (h->coarse_factors) {
            const long long sm = coarse_lu_smem(h->nc, h->coarse_kl, h->coarse_kl);
            raise_smem_limit((const void *)k_coarse_lu<R>, (int)sm);
            launch_k(h, k_coarse_lu<R>, 1, kLuSolveThreads, (size_t)sm, s, 0, h->Mwork, h->Mwork + (long long)h->nc * h->coarse_kl, h->piv,
                                                     h->dinv, h->nc, h->coarse_kl, h->coarse_kl,
                                                     reinterpret_cast<const R *>(v.b), reinterpret_cast<R *>(v.x),
                                                     h->err_d);
            counted(h);
            return;
        }
        const int threads = 256;
        const unsigned blocks = (unsigned)((h->nc * 32LL + threads - 1) / threads);
        launch_k(h, k_coarse_matvec<R>, blocks, threads, 0, s, 0, coarse_inverse<R>(h), reinterpret_cast<const R *>(v.b),
                                                      reinterpret_cast<R *>(v.x), h->nc);
        counted(h);
        return;
    }
    const LevelBuf &cb = h->L[l + 1];
    // timing brackets one smoothing pass of the finest level per cycle: the
    // pre-smoothing, or the post-smoothing when there is none (two event nodes
    // per cycle, not four: each costs the step a little)
    const bool tm_pre = h->timing && !h->cond_body && l == 0 && h->opt.nu1 > 0;
    const bool tm_post = h->timing && !h->cond_body && l == 0 && h->opt.nu1 == 0;
    if (tm_pre) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
    const bool alt = enqueue_smooth<R, DIM>(h, s, l, h->opt.nu1);
    if (tm_pre) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
    // the level's values, where the smoothing left them
    Level<R> vl = view<R>(lb);
    if (alt) vl.x = xalt_of<R>(lb);
    const dim3 rg = cell_grid(cb, DIM, cb.n[0]);
    if (h->opt.nu1 > 0 && red_only_after_sweeps(h)) {
        if (h->persistent)
            launch_k(h, k_residual_restrict<R, DIM, true, true>, wave((const void *)k_residual_restrict<R, DIM, true, true>, tiles_of(rg)), kBlock, 0, s, 0, vl,
                                                                                                          view<R>(cb));
        else
            launch_k(h, k_residual_restrict<R, DIM, true, false>, rg, kBlock, 0, s, 0, vl, view<R>(cb));
    } else {
        if (h->persistent)
            launch_k(h, k_residual_restrict<R, DIM, false, true>, wave((const void *)k_residual_restrict<R, DIM, false, true>, tiles_of(rg)), kBlock, 0, s, 0, 
                    vl, view<R>(cb));
        else
            launch_k(h, k_residual_restrict<R, DIM, false, false>, rg, kBlock, 0, s, 0, vl, view<R>(cb));
    }
    counted(h);
    enqueue_vcycle<R, DIM>(h, s, l + 1, type);
    if (type != MG_CYCLE_V && l + 1 < h->nlev - 1)
        enqueue_vcycle<R, DIM>(h, s, l + 1, type == MG_CYCLE_W ? MG_CYCLE_W : MG_CYCLE_V);
    const dim3 pg = cell_grid(lb, DIM, lb.n[0]);
    if (h->persistent)
        launch_k(h, k_prolong_add<R, DIM, true>, wave((const void *)k_prolong_add<R, DIM, true>, tiles_of(pg)), kBlock, 0, s, 0, 
            view<R>(cb), vl, bc_flags(h->grid));
    else
        launch_k(h, k_prolong_add<R, DIM, false>, pg, kBlock, 0, s, 0, view<R>(cb), vl, bc_flags(h->grid));
    counted(h);
    if (tm_post) cudaEventRecordWithFlags(h->ev[0], s, cudaEventRecordExternal);
    const bool alt_end = enqueue_smooth<R, DIM>(h, s, l, h->opt.nu2, alt);
    if (tm_post) cudaEventRecordWithFlags(h->ev[1], s, cudaEventRecordExternal);
    // (fused pairs are allowed only where the pairs of a cycle are even in number)
    if (alt_end)
        cudaMemcpyAsync(view<R>(lb).x, xalt_of<R>(lb), sizeof(typename Vec<R>::v2) * lb.N, cudaMemcpyDeviceToDevice,
                        s);
}

// after_sweep: x has just come out of a red-black sweep (red cells only).
template <int DIM>
void enqueue_norm(const mg_handle *h, cudaStream_t s, bool after_sweep) {
    const LevelBuf &f = h->L[0];
    const dim3 ng = norm_grid(f, DIM);
    if (after_sweep) {
        if (h->persistent)
            launch_k(h, k_norm_partials<DIM, true, true>, wave((const void *)k_norm_partials<DIM, true, true>, tiles_of(ng)), kBlock, 0, s, 0, view<double>(f), h->partial, h->ticket, h->norms_d);
        else
            launch_k(h, k_norm_partials<DIM, true, false>, ng, kBlock, 0, s, 0, view<double>(f), h->partial, h->ticket, h->norms_d);
    } else {
        if (h->persistent)
            launch_k(h, k_norm_partials<DIM, false, true>, wave((const void *)k_norm_partials<DIM, false, true>, tiles_of(ng)), kBlock, 0, s, 0, view<double>(f), h->partial, h->ticket, h->norms_d);
        else
            launch_k(h, k_norm_partials<DIM, false, false>, ng, kBlock, 0, s, 0, view<double>(f), h->partial, h->ticket, h->norms_d);
    }
    counted(h);
}

// Mixed precision solves for the correction delta from the initial guess x0
// (the paper's defect correction, the steps after Eq. 34): x keeps x0, delta
// lives in the staging area (at least 32 bytes per cell, free once prep has
// run).
double2 *mixed_delta(const mg_handle *h) { return reinterpret_cast<double2 *>(h->stage); }

// FP64 residual of the finest level, as the FP32 right-hand side, with its
// norms.  initial: r0 = b - A x0, written over b, and delta set to zero;
// otherwise r = r0 - A delta.  Forming b - A x every step instead subtracts
// terms of the size of b (lambda_T ~ 1e16 at these units) and leaves a
// rounding floor that a good initial guess puts near the tolerance.
template <int DIM>
void enqueue_residual_to32(const mg_handle *h, cudaStream_t s, bool initial = false) {
    const LevelBuf &f = h->L[0];
    const dim3 ng = norm_grid(f, DIM);
    Level<double> v = view<double>(f);
    double2 *delta = mixed_delta(h);
    if (!initial) v.x = delta;
    double2 *r_out = initial ? f.b : nullptr;
    double2 *r_out2 = initial ? delta : nullptr;
    if (h->persistent)
        launch_k(h, k_residual64_to32<DIM, true>, wave((const void *)k_residual64_to32<DIM, true>, tiles_of(ng)), kBlock, 0, s, 0, 
            v, f.b32, f.bt32, f.x32, r_out, r_out2, h->partial, h->ticket, h->norms_d);
    else
        launch_k(h, k_residual64_to32<DIM, false>, ng, kBlock, 0, s, 0, v, f.b32, f.bt32, f.x32, r_out, r_out2, h->partial,
                                                             h->ticket, h->norms_d);
    counted(h);
}

// Fills wave()'s cache for this handle's kernels outside any stream capture.
template <typename R, int DIM>
void warm_waves_r() {
    wave((const void *)k_rbgs_colour<R, DIM, true>, 1);
    wave((const void *)k_residual_restrict<R, DIM, true, true>, 1);
    wave((const void *)k_residual_restrict<R, DIM, false, true>, 1);
    wave((const void *)k_prolong_add<R, DIM, true>, 1);
}

template <int DIM>
void warm_waves() {
    warm_waves_r<double, DIM>();
    warm_waves_r<float, DIM>();
    wave((const void *)k_norm_partials<DIM, true, true>, 1);
    wave((const void *)k_norm_partials<DIM, false, true>, 1);
    wave((const void *)k_residual64_to32<DIM, true>, 1);
}

// FP64: one V-cycle, then the stopping norm, copied to pinned host memory.
template <int DIM>
void enqueue_cycle64(const mg_handle *h, cudaStream_t s) {
    enqueue_vcycle<double, DIM>(h, s, 0, h->opt.cycle);
    enqueue_norm<DIM>(h, s, h->opt.nu2 > 0 && red_only_after_sweeps(h));
    cudaMemcpyAsync(h->norms_h, h->norms_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

// Mixed: FP32 V-cycles on the correction, FP64 update, FP64 residual + norm.
template <int DIM>
void enqueue_step32(const mg_handle *h, cudaStream_t s) {
    for (int q = 0; q < h->opt.inner_cycles; q++) enqueue_vcycle<float, DIM>(h, s, 0, h->opt.cycle);
    const LevelBuf &f = h->L[0];
    launch_k(h, k_add_correction, lin_blocks(f.N), 256, 0, s, 0, mixed_delta(h), f.x32, f.N);
    counted(h);
    enqueue_residual_to32<DIM>(h, s);
    cudaMemcpyAsync(h->norms_h, h->norms_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
}

template <typename F>
mg_status capture(mg_handle *h, cudaGraphExec_t *out, long long *kernels, F &&body) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    const long long before = h->enq;
    body(h->cap);
    *kernels = h->enq - before;
    h->enq = before;
    const cudaError_t le = cudaGetLastError();        // a launch refused while capturing
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(MG_ERR_CUDA, std::string("graph capture: a launch failed: ") + cudaGetErrorString(le));
    }
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return MG_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Brings a [N][2] pair array to the device: the caller's pointer itself when
// on_device, else a copy in the staging area.
mg_status pair_in(mg_handle *h, const double *src, int on_device, const double2 **dev) {
    const long long N = h->L[0].N;
    if (on_device) {
        if (!aligned16(src)) return fail(MG_ERR_INVALID_ARG, "device pair arrays must be 16-byte aligned");
        *dev = reinterpret_cast<const double2 *>(src);
        return MG_OK;
    }
    CK(cudaMemcpyAsync(h->stage, src, sizeof(double2) * N, cudaMemcpyHostToDevice, h->stream));
    *dev = reinterpret_cast<const double2 *>(h->stage);
    return MG_OK;
}

mg_status x_in(mg_handle *h, const double *x, int on_device) {
    const long long N = h->L[0].N;
    if (on_device && !aligned16(x)) return fail(MG_ERR_INVALID_ARG, "device pair arrays must be 16-byte aligned");
    CK(cudaMemcpyAsync(h->L[0].x, x, sizeof(double2) * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
    return MG_OK;
}

mg_status x_out(mg_handle *h, double *x, int on_device) {
    const long long N = h->L[0].N;
    CK(cudaMemcpyAsync(x, h->L[0].x, sizeof(double2) * N, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    return MG_OK;
}

template <int DIM>
void enqueue_prep(mg_handle *h, const double2 *rhs, cudaStream_t s) {
    const LevelBuf &f = h->L[0];
    launch_k(h, k_prep_rhs<DIM>, cell_grid(f, DIM, f.n[0]), kBlock, 0, s, 0, view<double>(f), rhs, bc_vals(h->grid),
                                                                          h->grid.axisym, h->grid.r0, h->grid.h);
    counted(h);
}

mg_status prep(mg_handle *h, const double *rhs, const double *x, int on_device) {
    const double2 *r = nullptr;
    mg_status st = pair_in(h, rhs, on_device, &r);
    if (st) return st;
    if ((st = x_in(h, x, on_device))) return st;
    if (h->grid.dim == 2) enqueue_prep<2>(h, r, h->stream);
    else enqueue_prep<3>(h, r, h->stream);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status sync_norms(mg_handle *h, double out[2]) {
    CK(cudaStreamSynchronize(h->stream));
    out[0] = h->norms_h[0];
    out[1] = h->norms_h[1];
    return MG_OK;
}

// After a synchronised cycle: add the finest-level smoothing time it recorded.
mg_status accumulate_timing(mg_handle *h) {
    if (!h->timing || h->L[0].N == 0 || h->nlev < 2) return MG_OK;
    float a = 0.f;
    CK(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    h->smooth_ms += (double)a;
    long long l1, s1;
    const int sw = h->opt.nu1 > 0 ? h->opt.nu1 : h->opt.nu2;
    if (h->opt.smoother == MG_SMOOTH_WJAC) {
        l1 = sw;                 // one Jacobi kernel per sweep
        s1 = sw;
    } else {
        smooth_launches(h->sweep[0], h->grid.dim == 2, sw, &l1, &s1);
    }
    h->smooth_launches += l1;
    h->smooth_sweeps += s1;
    return MG_OK;
}

bool converged(const double n0[2], const double nk[2], double rtol) {
    if (!(rtol > 0.0)) return false;
    for (int f = 0; f < 2; f++) {
        const double q = n0[f] > 0.0 ? nk[f] / n0[f] : 0.0;
        if (!(q <= rtol)) return false;
    }
    return true;
}

// The coarsest inverse above kBandSmemMax unknowns takes the windowed LU and
// the block-column inverse when the band's window and the inverse's staging
// fit a block's shared memory and the factors fit the n x n work array;
// otherwise the three global-memory kernels.
int inv_block_warps(int n, int kl) {
    for (int w = 8; w > 1; w /= 2)
        if (band_inv_block_smem(n, kl, kl, w) <= kWinSmemMax) return w;
    return 1;
}

bool window_path(int n, int kl) {
    return n > kBandSmemMax && band_window_smem(kl, kl) <= kWinSmemMax &&
           band_inv_block_smem(n, kl, kl, inv_block_warps(n, kl)) <= kWinSmemMax &&
           (long long)n * (kl + 2LL * kl + 1) <= (long long)n * n;
}

// The windowed path's LU blocked over one cluster per coarsest matrix
// (k_band_lu_blocked; the same factors as k_band_lu_window) where its shared
// memory fits.
bool lu_blocked_ok(int n, int kl) { return band_blocked_smem(n, kl, kl) <= kWinSmemMax; }

// Launches kern on `clusters` clusters of kLuClusterCtas CTAs of `threads` threads.
template <typename... Args>
cudaError_t launch_cluster(void (*kern)(Args...), cudaStream_t s, int clusters, int threads, size_t smem,
                           Args... args) {
    cudaError_t e = raise_smem_limit((const void *)kern, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(kLuClusterCtas * clusters), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kLuClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_lu_blocked(cudaStream_t s, const double *M, int n, int kl, int *piv, double *dinv, double *Lb,
                              double *Uc, int *err) {
    return launch_cluster(k_band_lu_blocked, s, 1, kLuBlockedThreads, (size_t)band_blocked_smem(n, kl, kl), M, n, kl,
                          kl, piv, dinv, Lb, Uc, err);
}

// ---------------------------------------------------------------- set-up
SetupOut setup_out(const LevelBuf &l, bool mixed) {
    SetupOut o;
    std::memset(&o, 0, sizeof(o));
    for (int a = 0; a < 3; a++) {
        o.G[a] = l.G[a];
        o.G32[a] = mixed ? l.G32[a] : nullptr;
    }
    o.S = l.S;
    o.D = l.D;
    o.Dinv = l.Dinv;
    o.W = l.W;
    o.l4 = l.l4;
    if (mixed) {
        o.D32 = l.D32;
        o.Dinv32 = l.Dinv32;
        o.W32 = l.W32;
        o.l432 = l.l4_32;
        o.G0p = l.G32p0;
        o.p0 = l.p0;
        o.n0 = l.n[0];
        o.jflag = l.jflag;
        o.jcount = l.jcount;
        o.jratio = l.jratio;
    }
    return o;
}

SetupFine setup_fine_of(const LevelBuf &F, double h) {
    SetupFine s;
    s.n0 = F.n[0];
    s.n1 = F.n[1];
    s.S = F.S;
    s.l4 = F.l4;
    for (int a = 0; a < 3; a++) s.G[a] = F.G[a] ? F.G[a] : F.G[0];
    s.h = h;
    return s;
}

// The set-up of every level on stream s: flag reset, the finest level from
// the inputs, each coarser level from the one below, and the coarsest matrix.
template <int DIM>
void enqueue_setup_levels(mg_handle *h, cudaStream_t s, const SetupGeom &gm, const SetupIn &in) {
    const bool mixed = h->opt.precision == MG_MIXED;
    const LevelBuf &f = h->L[0];
    cudaMemsetAsync(h->err_d, 0, sizeof(int), s);
    if (f.jflag) cudaMemsetAsync(h->err_d + 2, 0, sizeof(int), s);
    launch_k(h, k_setup_fine<DIM>, cell_grid(f, DIM, f.n[0]), kBlock, 0, s, 0, gm, in, setup_out(f, mixed), h->err_d);
    counted(h);
    double hl = h->grid.h;
    for (int l = 1; l < h->nlev; l++) {
        const LevelBuf &F = h->L[l - 1];
        const LevelBuf &C = h->L[l];
        SetupGeom cg = gm;
        for (int a = 0; a < 3; a++) cg.n[a] = C.n[a];
        cg.h = 2.0 * hl;
        launch_k(h, k_setup_coarse<DIM>, cell_grid(C, DIM, C.n[0]), kBlock, 0, s, 0, cg, setup_fine_of(F, hl),
                 setup_out(C, mixed), h->err_d);
        counted(h);
        hl *= 2.0;
    }
    const LevelBuf &c = h->L[h->nlev - 1];
    cudaMemsetAsync(h->Mtmp, 0, sizeof(double) * h->nc * h->nc, s);
    launch_k(h, k_coarse_assemble<DIM>, lin_blocks(c.N), 256, 0, s, 0, c.n[0], c.n[1], c.n[2], c.G[0], c.G[1],
             DIM == 3 ? c.G[2] : nullptr, c.D, c.l4, h->Mtmp);
    counted(h);
}

template <int DIM>
mg_status setup_hierarchy(mg_handle *h, const double *lam, const double *const fa[3], const double *const fk[3],
                          int on_device) {
    const mg_grid &g = h->grid;
    cudaStream_t s = h->stream;
    const bool mixed = h->opt.precision == MG_MIXED;
    LevelBuf &f = h->L[0];
    // the previous set-up's coarsest inverse must be done before anything is overwritten
    CK(cudaStreamWaitEvent(s, h->ev_inv, 0));
    const double *lam_d = lam;
    const double *fad[3] = {nullptr, nullptr, nullptr}, *fkd[3] = {nullptr, nullptr, nullptr};
    if (!on_device) {
        double *st = reinterpret_cast<double *>(h->stage);
        CK(cudaMemcpyAsync(st, lam, sizeof(double) * 4 * f.N, cudaMemcpyHostToDevice, s));
        lam_d = st;
        double *p = st + 4 * f.N;
        for (int a = 0; a < DIM; a++) {
            CK(cudaMemcpyAsync(p, fa[a], sizeof(double) * f.nf[a], cudaMemcpyHostToDevice, s));
            fad[a] = p;
            p += f.nf[a];
            CK(cudaMemcpyAsync(p, fk[a], sizeof(double) * f.nf[a], cudaMemcpyHostToDevice, s));
            fkd[a] = p;
            p += f.nf[a];
        }
    } else {
        for (int a = 0; a < DIM; a++) {
            fad[a] = fa[a];
            fkd[a] = fk[a];
        }
    }
    SetupGeom gm;
    std::memset(&gm, 0, sizeof(gm));
    for (int a = 0; a < 3; a++) {
        gm.n[a] = f.n[a];
        for (int sd = 0; sd < 2; sd++)
            gm.fac[a][sd] = (a < DIM && g.bc[a][sd] == MG_BC_DIRICHLET) ? 2.0 : 0.0;
    }
    gm.axisym = g.axisym;
    gm.r0 = g.r0;
    gm.h = g.h;
    gm.ih2 = 1.0 / (g.h * g.h);
    SetupIn in;
    in.lam = lam_d;
    for (int a = 0; a < 3; a++) {
        in.fa[a] = a < DIM ? fad[a] : nullptr;
        in.fk[a] = a < DIM ? fkd[a] : nullptr;
    }
    // The level work is one CUDA graph per handle, captured again only when
    // the input pointers change: launched one kernel at a time from the host,
    // the small coarse levels would leave the device waiting on launches.
    // The coarsest matrix is assembled (and its inverse started below) before
    // the host waits for the flags of the level kernels, so the device runs
    // the whole set-up without a gap.  With invalid coefficients the inverse
    // works on non-finite values (bounded loops, no fault) and the call fails;
    // the next set-up waits for it before overwriting anything.
    const void *key[7] = {lam_d, in.fa[0], in.fa[1], in.fa[2], in.fk[0], in.fk[1], in.fk[2]};
    mg_handle::SetupGraph *sg = nullptr;
    for (auto &cand : h->gsetup)
        if (cand.exec && std::memcmp(key, cand.key, sizeof(key)) == 0) sg = &cand;
    if (!sg) {
        sg = &h->gsetup[h->gsetup_next];
        h->gsetup_next = (h->gsetup_next + 1) % kSetupGraphs;
        if (sg->exec) {
            cudaGraphExecDestroy(sg->exec);
            sg->exec = nullptr;
        }
        const mg_status e =
            capture(h, &sg->exec, &sg->kernels, [&](cudaStream_t cs) { enqueue_setup_levels<DIM>(h, cs, gm, in); });
        if (e) return e;
        std::memcpy(sg->key, key, sizeof(key));
    }
    CK(cudaGraphLaunch(sg->exec, s));
    h->enq += sg->kernels;
    const LevelBuf &c = h->L[h->nlev - 1];
    // The coarsest inverse runs on the aux stream, overlapping the caller's
    // next work and the start of the next solve (whose cycles wait for it
    // before their coarsest solve).  A singular coarsest matrix is reported by
    // mg_solve.
    CK(cudaEventRecord(h->ev_asm, s));
    CK(cudaStreamWaitEvent(h->aux, h->ev_asm, 0));
    cudaStream_t a = h->aux;
    // band of the coarsest matrix: the farthest neighbour cell is n0 (2D)
    // or n0*n1 (3D) cells away, two unknowns per cell
    const int off = DIM == 3 ? c.n[0] * c.n[1] : c.n[0];
    const int kl = std::min(h->nc - 1, 2 * off + 1);
    if (h->nc <= kBandSmemMax) {
        const size_t smem_lu = sizeof(double) * (size_t)h->nc * h->nc;
        CK(raise_smem_limit((const void *)k_band_lu_warp, (int)(sizeof(double) * kBandSmemMax * kBandSmemMax)));
        k_band_lu_warp<<<1, kLUThreads, smem_lu, a>>>(h->Mtmp, h->nc, kl, kl, h->piv, h->dinv, h->err_d);
        const int smem_inv = (int)(sizeof(double) * inv_smem_doubles(h->nc, kl, kl));
        CK(raise_smem_limit((const void *)k_band_inv_cols_warp,
                            (int)(sizeof(double) * inv_smem_doubles(kBandSmemMax, kBandSmemMax - 1, kBandSmemMax - 1))));
        k_band_inv_cols_warp<<<(h->nc + 31) / 32, dim3(32, kInvRows), smem_inv,
                               a>>>(h->Mtmp, h->piv, h->dinv, h->nc, kl, kl, h->Minv, mixed ? h->Minv32 : nullptr,
                                    h->err_d);
    } else if (window_path(h->nc, kl)) {
        // the band's active window in shared memory, then the columns of the inverse, a warp each
        const long long wsm = band_window_smem(kl, kl);
        const int warps = inv_block_warps(h->nc, kl);
        const long long ism = band_inv_block_smem(h->nc, kl, kl, warps);
        CK(raise_smem_limit((const void *)k_band_lu_window, (int)wsm));
        CK(raise_smem_limit((const void *)k_band_inv_block, (int)ism));
        double *Lb = h->Mwork, *Uc = h->Mwork + (long long)h->nc * kl;
        if (lu_blocked_ok(h->nc, kl))
            CK(launch_lu_blocked(a, h->Mtmp, h->nc, kl, h->piv, h->dinv, Lb, Uc, h->err_d));
        else
            k_band_lu_window<<<1, kWinThreads, (size_t)wsm, a>>>(h->Mtmp, h->nc, kl, kl, h->piv, h->dinv, Lb, Uc,
                                                                 h->err_d);
        if (h->coarse_factors)           // the cycles solve from Lb and the scaled Uc (k_coarse_lu)
            k_scale_uc<<<lin_blocks((long long)h->nc * 2 * kl), 256, 0, a>>>(Uc, h->dinv, h->nc, kl, kl, h->err_d);
        else
            k_band_inv_block<<<(h->nc + warps - 1) / warps, 32 * warps, (size_t)ism, a>>>(
                Lb, Uc, h->piv, h->dinv, h->nc, kl, kl, h->Minv, mixed ? h->Minv32 : nullptr, h->err_d);
    } else {
        k_band_lu<<<1, dim3(32, 32, 1), 0, a>>>(h->Mtmp, h->nc, kl, kl, h->piv, h->dinv, h->err_d);
        k_band_inv_cols<<<(h->nc + 127) / 128, 128, 0, a>>>(h->Mtmp, h->piv, h->dinv, h->nc, kl, kl, h->Mwork,
                                                            h->err_d);
        k_transpose<<<lin_blocks((long long)h->nc * h->nc), 256, 0, a>>>(h->Mwork, h->Minv, h->nc);
        if (mixed)
            k_to_f32<<<lin_blocks((long long)h->nc * h->nc), 256, 0, a>>>(h->Minv, h->Minv32,
                                                                         (long long)h->nc * h->nc);
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(h->ev_inv, a));
    counted(h, h->nc <= kBandSmemMax || window_path(h->nc, kl) ? 2 : 4);
    // flags 1 and 2 come from the level kernels, which precede this copy on
    // the stream (the inverse on the private stream keeps running)
    CK(cudaMemcpyAsync(h->errh, h->err_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (f.jflag) CK(cudaMemcpyAsync(h->errh + 2, h->err_d + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->jcells = f.jflag ? h->errh[2] : 0;
    const int err = *h->errh;
    if (err & 1) return fail(MG_ERR_INVALID_COEFF, "non-finite coefficient in lambda or the face arrays");
    if (err & 2) return fail(MG_ERR_INVALID_COEFF, "a local 2x2 block is singular or not finite");
    return MG_OK;
}

// ---------------------------------------------------------------- solves
// The stop-test loop of both precisions.  `initial` enqueues the initial
// norms (into norms_d); g is the graph of one iteration, which copies its
// norms to norms_h[0..1]; an iteration is `per_iter` V-cycles.  The first
// iteration is launched before the initial norms are read, so one host wait
// serves both: it only changes the handle's own x, which mg_solve does not
// copy back (x_stale) when the initial state already meets the stop test.
template <typename FInit>
mg_status run_loop(mg_handle *h, mg_stats *st, cudaGraphExec_t g, long long kernels, int per_iter, FInit &&initial) {
    double n0[2], nk[2];
    initial(h->stream);
    CK(cudaMemcpyAsync(h->norms_h + 2, h->norms_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    const bool ahead = h->opt.max_cycles >= 1 && h->opt.rtol < 1.0;
    if (ahead) {
        CK(cudaGraphLaunch(g, h->stream));
        h->enq += kernels;
    }
    CK(cudaStreamSynchronize(h->stream));
    n0[0] = nk[0] = h->norms_h[2];
    n0[1] = nk[1] = h->norms_h[3];
    int it = 0;
    bool ok = converged(n0, nk, h->opt.rtol) || (n0[0] == 0.0 && n0[1] == 0.0);
    if (ahead) {
        if (ok) {
            h->x_stale = true;
        } else {
            nk[0] = h->norms_h[0];
            nk[1] = h->norms_h[1];
            mg_status e = accumulate_timing(h);
            if (e) return e;
            it = 1;
            ok = converged(n0, nk, h->opt.rtol);
        }
    }
    while (!ok && it < h->opt.max_cycles) {
        CK(cudaGraphLaunch(g, h->stream));
        h->enq += kernels;
        mg_status e = sync_norms(h, nk);
        if (!e) e = accumulate_timing(h);
        if (e) return e;
        it++;
        ok = converged(n0, nk, h->opt.rtol);
    }
    st->cycles = it * per_iter;
    st->outer = it;
    st->r0[0] = n0[0];
    st->r0[1] = n0[1];
    st->rfinal[0] = nk[0];
    st->rfinal[1] = nk[1];
    st->status = (ok || !(h->opt.rtol > 0.0)) ? MG_OK : MG_ERR_NOT_CONVERGED;
    return MG_OK;
}

template <int DIM>
mg_status solve64(mg_handle *h, mg_stats *st) {
    if (!h->g64) {
        const mg_status e = capture(h, &h->g64, &h->graph_kernels64, [&](cudaStream_t s) { enqueue_cycle64<DIM>(h, s); });
        if (e) return e;
    }
    return run_loop(h, st, h->g64, h->graph_kernels64, 1,
                    [&](cudaStream_t s) { enqueue_norm<DIM>(h, s, false); });
}

template <int DIM>
mg_status solve_mixed(mg_handle *h, mg_stats *st) {
    if (!h->g32) {
        const mg_status e = capture(h, &h->g32, &h->graph_kernels32, [&](cudaStream_t s) { enqueue_step32<DIM>(h, s); });
        if (e) return e;
    }
    // r0 = b - A x0 once, delta from A delta = r0 by FP32 cycles with the
    // FP64 residual r0 - A delta after each outer step, then x = x0 + delta
    const LevelBuf &f = h->L[0];
    const mg_status e = run_loop(h, st, h->g32, h->graph_kernels32, h->opt.inner_cycles,
                                 [&](cudaStream_t s) { enqueue_residual_to32<DIM>(h, s, true); });
    if (e) return e;
    if (!h->x_stale) {
        launch_k(h, k_add_pairs, lin_blocks(f.N), 256, 0, h->stream, 0, f.x, mixed_delta(h), f.N);
        counted(h);
        CK(cudaGetLastError());
    }
    return MG_OK;
}

// opt.max_cycles FP64 cycles from x = 0 with no stopping norms and no host wait: a fixed linear map of rhs, the
// correction solve of the momentum predictor's outer loop.  The result stays in L[0].x.
template <int DIM>
mg_status correction_cycles(mg_handle *h, const double2 *rhs) {
    if (!h->gcorr) {
        const mg_status e = capture(h, &h->gcorr, &h->graph_kernels_corr, [&](cudaStream_t s) {
            for (int q = 0; q < h->opt.max_cycles; q++) enqueue_vcycle<double, DIM>(h, s, 0, h->opt.cycle);
        });
        if (e) return e;
    }
    const LevelBuf &f = h->L[0];
    CK(cudaMemsetAsync(f.x, 0, sizeof(double2) * f.N, h->stream));
    enqueue_prep<DIM>(h, rhs, h->stream);
    CK(cudaGetLastError());
    CK(cudaGraphLaunch(h->gcorr, h->stream));
    h->enq += h->graph_kernels_corr;
    return MG_OK;
}

// The same correction enqueued on stream s without a graph of its own (for
// a caller that captures it into its graph): x = 0, the prepared right-hand
// side rhs, max_cycles cycles without norms.  A mixed-precision handle runs
// them in FP32 (right-hand side rounded from the FP64 one, as for an outer
// step of its solves) and leaves the correction, widened, in the FP64 x.
template <int DIM>
mg_status enqueue_correction(mg_handle *h, cudaStream_t s, const double2 *rhs) {
    const LevelBuf &f = h->L[0];
    CK(cudaMemsetAsync(f.x, 0, sizeof(double2) * f.N, s));
    enqueue_prep<DIM>(h, rhs, s);
    if (h->opt.precision == MG_MIXED) {
        enqueue_residual_to32<DIM>(h, s, true);        // x = 0: b32 = b, bt32 = Dinv b, e32 = 0
        for (int q = 0; q < h->opt.max_cycles; q++) enqueue_vcycle<float, DIM>(h, s, 0, h->opt.cycle);
        launch_k(h, k_add_correction, lin_blocks(f.N), 256, 0, s, 0, f.x, f.x32, f.N);
        counted(h);
    } else {
        for (int q = 0; q < h->opt.max_cycles; q++) enqueue_vcycle<double, DIM>(h, s, 0, h->opt.cycle);
    }
    CK(cudaGetLastError());
    return MG_OK;
}

// A whole solve as one graph, for mg_solve_async: the initial norms and a
// first stop test, then a WHILE node whose body is one iteration of the
// solve (FP64: a cycle and its norms; mixed: the FP32 cycles, the update and
// the FP64 residual with its norms) ending in the stop test, then (mixed) x =
// x0 + delta and the copy of the statistics to pinned host memory.  The same
// kernels in the same order as mg_solve, so the result is the same bit for
// bit.  The body holds no event node (graph rules): the caller's stream waits
// for the coarsest inverse before launching the graph.
template <int DIM>
mg_status capture_async(mg_handle *h) {
    const bool mixed = h->opt.precision == MG_MIXED;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    const long long before = h->enq;
    cudaError_t e = cudaSuccess;
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNode_t node = nullptr;
    cudaGraph_t body = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaStreamCaptureStatus cs;
    if (mixed) enqueue_residual_to32<DIM>(h, h->cap, true);
    else enqueue_norm<DIM>(h, h->cap, false);
    long long pre = h->enq - before;
    e = cudaStreamGetCaptureInfo(h->cap, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
    // the condition starts at 0 on every launch (the loop runs only if the
    // first stop test below asks for it); the body's stop test ends the loop
    // after max_cycles iterations at the latest
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        launch_k(h, k_async_stop, 1, 32, 0, h->cap, 0, h->norms_d, h->astat_d, h->opt.max_cycles, h->opt.rtol, cond, 1);
        pre++;
        e = cudaStreamGetCaptureInfo(h->cap, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
    }
    if (e == cudaSuccess) {
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // the rest zero-initialised
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &np);
        if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(h->cap, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    long long per = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(h->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const long long b0 = h->enq;
        h->cond_body = true;
        if (mixed) {
            for (int q = 0; q < h->opt.inner_cycles; q++) enqueue_vcycle<float, DIM>(h, h->cap2, 0, h->opt.cycle);
            const LevelBuf &f = h->L[0];
            launch_k(h, k_add_correction, lin_blocks(f.N), 256, 0, h->cap2, 0, mixed_delta(h), f.x32, f.N);
            counted(h);
            enqueue_residual_to32<DIM>(h, h->cap2);
        } else {
            enqueue_vcycle<double, DIM>(h, h->cap2, 0, h->opt.cycle);
            enqueue_norm<DIM>(h, h->cap2, h->opt.nu2 > 0 && red_only_after_sweeps(h));
        }
        launch_k(h, k_async_stop, 1, 32, 0, h->cap2, 0, h->norms_d, h->astat_d, h->opt.max_cycles, h->opt.rtol, cond, 0);
        counted(h);
        h->cond_body = false;
        per = h->enq - b0;
        const cudaError_t le = cudaGetLastError();
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(h->cap2, &out);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    long long post = 0;
    if (e == cudaSuccess) {
        if (mixed) {
            const LevelBuf &f = h->L[0];
            launch_k(h, k_add_pairs, lin_blocks(f.N), 256, 0, h->cap, 0, f.x, mixed_delta(h), f.N);
            post++;
        }
        e = cudaMemcpyAsync(h->astat_h, h->astat_d, sizeof(AsyncStat), cudaMemcpyDeviceToHost, h->cap);
    }
    h->enq = before;
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ee = cudaStreamEndCapture(h->cap, &graph);
    if (e == cudaSuccess) e = le != cudaSuccess ? le : ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gasync, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->gasync = nullptr;
        h->cond_body = false;
        return fail(MG_ERR_CUDA, std::string("async solve graph: ") + cudaGetErrorString(e));
    }
    h->async_kernels_pre = pre + post;
    h->async_kernels_body = per;
    return MG_OK;
}

// The device error flags a solve reports (singular coarsest matrix, a bounded wait that gave up); one host wait.
mg_status handle_errors(mg_handle *h) {
    CK(cudaStreamWaitEvent(h->stream, h->ev_inv, 0));
    CK(cudaMemcpyAsync(h->errh, h->err_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->errh[0] & 4) return fail(MG_ERR_INVALID_COEFF, "the coarsest-level matrix is singular");
    if (h->errh[1] & kErrAsyncTimeout) return fail(MG_ERR_TIMEOUT, "an asynchronous copy did not complete in time");
    return MG_OK;
}

mg_status check_handle(const mg_handle *h, bool need_coeffs) {
    if (!h) return fail(MG_ERR_INVALID_ARG, "handle is NULL");
    if (need_coeffs && !h->coeffs_set) return fail(MG_ERR_STATE, "mg_set_coeffs has not succeeded on this handle");
    return MG_OK;
}

// ---------------------------------------------------------------- tuning
bool tail_level_ok(const mg_handle *h, int l, int ctas = kTailCtas) {
    if (h->coarse_factors) return false;     // the tail multiplies by the coarsest inverse
    if (!(l >= 1 && h->nlev - l >= 2 && h->nlev - l <= kTailMaxLevels && h->L[l].N <= kTailMaxCells)) return false;
    size_t smem = 0;
    if (h->opt.precision == MG_MIXED) tail_args<float>(h, l, ctas, &smem);
    else tail_args<double>(h, l, ctas, &smem);
    return smem <= kTailSmemMax;
}

// 8 CTAs is a portable cluster size; 16 needs the kernel's opt-in and a
// device that can place such a cluster.
template <typename R, int DIM>
bool tail_ctas_allowed(int ctas) {
    if (ctas == 1 || ctas == kTailCtas) return true;
    if (ctas != 16) return false;
    if (cudaFuncSetAttribute(k_vcycle_tail<R, DIM, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = kBlock;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 16;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_tail<R, DIM, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

bool tail_ctas_ok(const mg_handle *h, int ctas) {
    const bool mixed = h->opt.precision == MG_MIXED;
    if (h->grid.dim == 2) return mixed ? tail_ctas_allowed<float, 2>(ctas) : tail_ctas_allowed<double, 2>(ctas);
    return mixed ? tail_ctas_allowed<float, 3>(ctas) : tail_ctas_allowed<double, 3>(ctas);
}

void drop_graphs(mg_handle *h) {
    if (h->g64) { cudaGraphExecDestroy(h->g64); h->g64 = nullptr; }
    if (h->gasync) { cudaGraphExecDestroy(h->gasync); h->gasync = nullptr; }
    if (h->gcorr) { cudaGraphExecDestroy(h->gcorr); h->gcorr = nullptr; }
    if (h->g32) { cudaGraphExecDestroy(h->g32); h->g32 = nullptr; }
}

// Captures body as a graph and times it with CUDA events on the handle's
// stream: one warm-up replay, then `launches` replays, each bracketed by
// events and waited for (the solve's own pattern: one graph launch per cycle,
// then a host synchronisation, so each time includes the launch overhead).
// Returns the median.
template <typename F>
mg_status time_graph(mg_handle *h, int launches, double *ms, F &&body) {
    cudaGraphExec_t ex = nullptr;
    long long kernels = 0;
    mg_status st = capture(h, &ex, &kernels, body);
    if (st) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> t;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    for (int q = 0; q < launches && e == cudaSuccess; q++) {
        e = cudaEventRecord(e0, h->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        if (e == cudaSuccess) t.push_back(f);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(ex);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("autotune timing: ") + cudaGetErrorString(e));
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return MG_OK;
}

template <typename R, int DIM>
mg_status autotune_impl(mg_handle *h, int reps, double *vcycle_ms) {
    mg_status st;
    // sweeps, level by level (the coarsest level is solved, not smoothed);
    // the Jacobi smoother has a single kernel
    for (int l = 0; l + 1 < h->nlev && h->opt.smoother == MG_SMOOTH_RBGS; l++) {
        // candidates: colour, colour with two rows per thread, then (2D) fused, TMA-fed fused and fused pairs
        // per tile
        const int ncand = DIM == 2 ? 2 + 3 * kTileShapes : 2;
        double best = 1e30;
        int kind = MG_SWEEP_COLOUR, tile = 0;
        for (int c = 0; c < ncand; c++) {
            const int ck = c == 0   ? MG_SWEEP_COLOUR
                           : c == 1 ? MG_SWEEP_COLOUR2
                           : c < 2 + kTileShapes ? MG_SWEEP_FUSED
                           : c < 2 + 2 * kTileShapes ? MG_SWEEP_ASYNC : MG_SWEEP_FUSED2;
            const int ct = c < 2 ? 0 : (c - 2) % kTileShapes;
            if (ck == MG_SWEEP_ASYNC && !async_ok<R>(h, l, ct)) continue;
            if (ck == MG_SWEEP_FUSED2 && !fused2_ok(h->opt, DIM)) continue;
            double ms = 0.0;
            st = time_graph(h, 5, &ms, [&](cudaStream_t s) {
                for (int r = 0; r < reps; r++) enqueue_sweeps<R, DIM>(h, s, l, 2, ck, ct);
            });
            if (st) return st;
            if (ms < best) { best = ms; kind = ck; tile = ct; }
        }
        h->sweep[l] = kind;
        h->tile[l] = tile;
    }
    // the cluster tail: none, or each allowed first level and cluster size
    std::vector<std::pair<int, int>> cand{{h->nlev, kTailCtas}};
    const bool wide = tail_ctas_allowed<R, DIM>(16);
    for (int l = 1; l < h->nlev && tail_runs(h); l++) {     // the tail runs red-black V-cycles only
        if (tail_level_ok(h, l, 1)) cand.push_back({l, 1});
        if (tail_level_ok(h, l, kTailCtas)) cand.push_back({l, kTailCtas});
        if (wide && tail_level_ok(h, l, 16)) cand.push_back({l, 16});
    }
    double best = 1e30;
    std::pair<int, int> pick = cand[0];
    int pick_p = 0;
    for (int persist = 0; persist < 2; persist++)
        for (const auto &c : cand) {
            h->tail_lev = c.first;
            h->tail_ctas = c.second;
            h->persistent = persist;
            double ms = 0.0;
            st = time_graph(h, 4 * reps + 1, &ms,
                            [&](cudaStream_t s) { enqueue_vcycle<R, DIM>(h, s, 0, h->opt.cycle); });
            if (st) return st;
            if (ms < best) { best = ms; pick = c; pick_p = persist; }
        }
    h->tail_lev = pick.first;
    h->tail_ctas = pick.second;
    h->persistent = pick_p;
    // dependent launches on or off for the chosen kernels: plain stream order
    // only where it is faster by more than the timing's noise (1%)
    double ms_on = 0.0, ms_off = 0.0;
    const int overlap = h->overlap;
    for (int ov = 1; ov >= 0; ov--) {
        h->overlap = ov;
        st = time_graph(h, 4 * reps + 1, ov ? &ms_on : &ms_off,
                        [&](cudaStream_t s) { enqueue_vcycle<R, DIM>(h, s, 0, h->opt.cycle); });
        if (st) {
            h->overlap = overlap;
            return st;
        }
    }
    h->overlap = ms_off < 0.99 * ms_on ? 0 : 1;
    if (vcycle_ms) *vcycle_ms = h->overlap ? ms_on : ms_off;
    return MG_OK;
}

void get_tuning(const mg_handle *h, mg_tuning *t) {
    std::memset(t, 0, sizeof(*t));
    t->levels = h->nlev;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        t->sweep[l] = l < h->nlev ? h->sweep[l] : MG_SWEEP_COLOUR;
        t->tile[l] = l < h->nlev ? h->tile[l] : 0;
    }
    t->tail_level = h->tail_lev;
    t->tail_ctas = h->tail_ctas;
    t->persistent = h->persistent;
    t->overlap = h->overlap;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

mg_status mg_default_options(mg_options *o) {
    if (!o) return fail(MG_ERR_INVALID_ARG, "options is NULL");
    o->nu1 = 2;
    o->nu2 = 2;
    o->precision = MG_FP64;
    o->rtol = 1e-10;
    o->max_cycles = 50;
    o->coarse_min = 4;
    o->inner_cycles = 1;
    o->cycle = MG_CYCLE_V;
    o->smoother = MG_SMOOTH_RBGS;
    o->omega = 0.8;
    o->fp64_jump_ratio = 2.0;
    o->coarse_solve = MG_COARSE_AUTO;
    return MG_OK;
}

mg_status mg_workspace_size(const mg_grid *grid, const mg_options *opt, size_t *bytes) {
    mg_status st = check_grid(grid, opt);
    if (st) return st;
    if (!bytes) return fail(MG_ERR_INVALID_ARG, "bytes is NULL");
    mg_handle tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    tmp.grid = *grid;
    tmp.opt = *opt;
    plan(&tmp, nullptr, bytes);
    return MG_OK;
}

mg_status mg_create(const mg_grid *grid, const mg_options *opt, void *workspace, size_t workspace_bytes, void *stream,
                    mg_handle **out) {
    mg_status st = check_grid(grid, opt);
    if (st) return st;
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mg_handle *h = new (std::nothrow) mg_handle;
    if (!h) return fail(MG_ERR_OOM, "host allocation failed");
    std::memset(h, 0, sizeof(*h));
    h->grid = *grid;
    h->opt = *opt;
    h->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&h->device);
    size_t need = 0;
    plan(h, nullptr, &need);
    char *base = nullptr;
    if (workspace) {
        if (workspace_bytes < need) {
            delete h;
            return fail(MG_ERR_BUDGET, "workspace of " + std::to_string(workspace_bytes) + " bytes, need " +
                                           std::to_string(need));
        }
        base = static_cast<char *>(workspace);
    } else {
        cudaError_t e = cudaMalloc(&base, need);
        if (e != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return fail(MG_ERR_OOM, std::string("cudaMalloc of the hierarchy failed: ") + cudaGetErrorString(e));
        }
        h->owns_arena = true;
    }
    char *aligned = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(base) + kAlign - 1) / kAlign * kAlign);
    h->arena = base;
    h->arena_bytes = need;
    size_t dummy;
    plan(h, aligned, &dummy);
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&h->ev_a0) != cudaSuccess || cudaEventCreate(&h->ev_a1) != cudaSuccess ||
        cudaMallocHost(&h->astat_h, sizeof(AsyncStat)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_asm, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_inv, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_last, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&h->errh, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&h->norms_h, 8 * sizeof(double)) != cudaSuccess ||
        cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(h);
        return fail(MG_ERR_CUDA, "stream or pinned buffer creation failed");
    }
    if (h->grid.dim == 2) warm_waves<2>();
    else warm_waves<3>();
    cudaGetLastError();
    *out = h;
    return MG_OK;
}

mg_status mg_set_coeffs(mg_handle *h, const double *lambda, const double *const face_alpha[3],
                        const double *const face_k[3], int on_device) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (!lambda || !face_alpha || !face_k) return fail(MG_ERR_INVALID_ARG, "NULL coefficient pointer");
    for (int a = 0; a < h->grid.dim; a++)
        if (!face_alpha[a] || !face_k[a]) return fail(MG_ERR_INVALID_ARG, "NULL face array");
    if (on_device) {
        if ((reinterpret_cast<uintptr_t>(lambda) & 7u) != 0) return fail(MG_ERR_INVALID_ARG, "lambda misaligned");
        for (int a = 0; a < h->grid.dim; a++)
            if ((reinterpret_cast<uintptr_t>(face_alpha[a]) & 7u) || (reinterpret_cast<uintptr_t>(face_k[a]) & 7u))
                return fail(MG_ERR_INVALID_ARG, "face array misaligned");
    }
    DeviceGuard dg(h->device);
    h->coeffs_set = false;
    st = h->grid.dim == 2 ? setup_hierarchy<2>(h, lambda, face_alpha, face_k, on_device)
                          : setup_hierarchy<3>(h, lambda, face_alpha, face_k, on_device);
    // the set-up is still running: mg_set_stream orders the next stream after it
    const cudaError_t e = cudaEventRecord(h->ev_last, h->stream);
    if (st == MG_OK && e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("set-up: ") + cudaGetErrorString(e));
    if (st == MG_OK) h->coeffs_set = true;
    return st;
}

mg_status mg_solve(mg_handle *h, const double *rhs, double *x, int on_device, mg_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (!rhs || !x) return fail(MG_ERR_INVALID_ARG, "rhs and x must not be NULL");
    DeviceGuard dg(h->device);
    CK(cudaMemsetAsync(h->err_d + 1, 0, sizeof(int), h->stream));
    h->x_stale = false;
    if ((st = prep(h, rhs, x, on_device))) return st;
    mg_stats s;
    std::memset(&s, 0, sizeof(s));
    s.levels = h->nlev;
    s.fp64_cells = h->jcells;
    const int dim = h->grid.dim;
    if (h->opt.precision == MG_FP64) st = dim == 2 ? solve64<2>(h, &s) : solve64<3>(h, &s);
    else st = dim == 2 ? solve_mixed<2>(h, &s) : solve_mixed<3>(h, &s);
    if (st) return st;
    if (!h->x_stale && (st = x_out(h, x, on_device))) return st;
    CK(cudaStreamWaitEvent(h->stream, h->ev_inv, 0));
    CK(cudaMemcpyAsync(h->errh, h->err_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->errh[0] & 4) return fail(MG_ERR_INVALID_COEFF, "the coarsest-level matrix is singular");
    if (h->errh[1] & kErrAsyncTimeout) return fail(MG_ERR_TIMEOUT, "an asynchronous copy did not complete in time");
    s.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = s;
    if (s.status != MG_OK) {
        g_err = "not converged after " + std::to_string(h->opt.max_cycles) + " cycles";
        return (mg_status)s.status;
    }
    return MG_OK;
}

mg_status mg_solve_async(mg_handle *h, const double *rhs, double *x, void *event) {
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (!rhs || !x) return fail(MG_ERR_INVALID_ARG, "rhs and x must not be NULL");
    if (!aligned16(rhs) || !aligned16(x)) return fail(MG_ERR_INVALID_ARG, "device pair arrays must be 16-byte aligned");
    DeviceGuard dg(h->device);
    if (!h->gasync) {
        st = h->grid.dim == 2 ? capture_async<2>(h) : capture_async<3>(h);
        if (st) return st;
    }
    CK(cudaMemsetAsync(h->err_d + 1, 0, sizeof(int), h->stream));
    h->x_stale = false;
    if ((st = prep(h, rhs, x, 1))) return st;
    CK(cudaStreamWaitEvent(h->stream, h->ev_inv, 0));
    CK(cudaEventRecord(h->ev_a0, h->stream));
    CK(cudaGraphLaunch(h->gasync, h->stream));
    if ((st = x_out(h, x, 1))) return st;
    CK(cudaMemcpyAsync(h->errh, h->err_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaEventRecord(h->ev_a1, h->stream));
    if (event) CK(cudaEventRecord(reinterpret_cast<cudaEvent_t>(event), h->stream));
    CK(cudaEventRecord(h->ev_last, h->stream));
    h->async_pending = true;
    return MG_OK;
}

mg_status mg_solve_async_stats(mg_handle *h, mg_stats *stats) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (!h->async_pending) return fail(MG_ERR_STATE, "no mg_solve_async to report on");
    DeviceGuard dg(h->device);
    CK(cudaEventSynchronize(h->ev_a1));
    h->async_pending = false;
    const AsyncStat a = *h->astat_h;
    h->enq += h->async_kernels_pre + (long long)a.it * h->async_kernels_body + 1;   // + the right-hand side's prep
    mg_stats s;
    std::memset(&s, 0, sizeof(s));
    s.levels = h->nlev;
    s.fp64_cells = h->jcells;
    const int per = h->opt.precision == MG_MIXED ? h->opt.inner_cycles : 1;
    s.cycles = a.it * per;
    s.outer = a.it;
    for (int f = 0; f < 2; f++) {
        s.r0[f] = a.n0[f];
        s.rfinal[f] = a.nk[f];
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_a0, h->ev_a1));
    s.seconds = ms * 1e-3;
    s.status = (a.ok || !(h->opt.rtol > 0.0)) ? MG_OK : MG_ERR_NOT_CONVERGED;
    if (h->errh[0] & 4) return fail(MG_ERR_INVALID_COEFF, "the coarsest-level matrix is singular");
    if (h->errh[1] & kErrAsyncTimeout) return fail(MG_ERR_TIMEOUT, "an asynchronous copy did not complete in time");
    if (stats) *stats = s;
    if (s.status != MG_OK) {
        g_err = "not converged after " + std::to_string(h->opt.max_cycles) + " cycles";
        return (mg_status)s.status;
    }
    return MG_OK;
}

mg_status mg_apply(mg_handle *h, const double *x, double *y, int on_device) {
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (!x || !y) return fail(MG_ERR_INVALID_ARG, "x and y must not be NULL");
    if (on_device && !aligned16(y)) return fail(MG_ERR_INVALID_ARG, "device pair arrays must be 16-byte aligned");
    DeviceGuard dg(h->device);
    if ((st = x_in(h, x, on_device))) return st;
    const LevelBuf &f = h->L[0];
    double2 *yd = on_device ? reinterpret_cast<double2 *>(y) : reinterpret_cast<double2 *>(h->stage);
    if (h->grid.dim == 2)
        k_apply_paper<2><<<cell_grid(f, 2, f.n[0]), kBlock, 0, h->stream>>>(view<double>(f), bc_vals(h->grid),
                                                                            h->grid.axisym, h->grid.r0, h->grid.h, yd);
    else
        k_apply_paper<3><<<cell_grid(f, 3, f.n[0]), kBlock, 0, h->stream>>>(view<double>(f), bc_vals(h->grid),
                                                                            h->grid.axisym, h->grid.r0, h->grid.h, yd);
    counted(h);
    CK(cudaGetLastError());
    if (!on_device) CK(cudaMemcpyAsync(y, yd, sizeof(double2) * f.N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

mg_status mg_smooth(mg_handle *h, const double *rhs, double *x, int sweeps, int on_device) {
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (!rhs || !x || sweeps < 0) return fail(MG_ERR_INVALID_ARG, "bad arguments to mg_smooth");
    DeviceGuard dg(h->device);
    if ((st = prep(h, rhs, x, on_device))) return st;
    const bool alt = h->grid.dim == 2 ? enqueue_smooth<double, 2>(h, h->stream, 0, sweeps)
                                      : enqueue_smooth<double, 3>(h, h->stream, 0, sweeps);
    if (alt)          // an odd number of fused pairs: the values are in xalt
        CK(cudaMemcpyAsync(h->L[0].x, h->L[0].xalt, sizeof(double2) * h->L[0].N, cudaMemcpyDeviceToDevice,
                           h->stream));
    CK(cudaGetLastError());
    if ((st = x_out(h, x, on_device))) return st;
    CK(cudaStreamSynchronize(h->stream));
    return MG_OK;
}

// ---------------------------------------------------------------- assembly and update
namespace {
bool device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

mg_status check_phase(const mg_phase &P) {
    const double v[8] = {P.Gamma, P.Pi, P.b, P.q, P.cp, P.cv, P.k, P.mu};
    for (double x : v)
        if (!std::isfinite(x)) return fail(MG_ERR_INVALID_ARG, "phase parameters must be finite");
    if (!(P.Gamma > 1.0)) return fail(MG_ERR_INVALID_ARG, "phase Gamma must be > 1");
    if (!(P.cv > 0.0) || !(P.cp > P.cv)) return fail(MG_ERR_INVALID_ARG, "phase heat capacities need cp > cv > 0");
    if (P.b < 0.0 || P.k < 0.0 || P.mu < 0.0) return fail(MG_ERR_INVALID_ARG, "phase b, k and mu must be >= 0");
    return MG_OK;
}

PhaseK phase_k(const mg_phase &P) {
    PhaseK K;
    K.Gamma = P.Gamma;
    K.Pi = P.Pi;
    K.b = P.b;
    K.q = P.q;
    K.cp = P.cp;
    K.k = P.k;
    K.shift = P.Gamma * P.Pi / (P.Gamma - 1.0);
    K.inv_g1 = 1.0 / (P.Gamma - 1.0);
    K.cpcv = P.cp - P.cv;
    K.g1cv = (P.Gamma - 1.0) * P.cv;
    K.gam_over_G = (P.cp / P.cv) / P.Gamma;
    K.inv_cp = 1.0 / P.cp;
    return K;
}
}  // namespace

mg_status mg_assemble_async(const mg_grid *grid, const mg_phase phases[2], double dt, int flags,
                            const mg_state *s, const mg_assembly *out, void *stream) {
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (!phases || !s || !out) return fail(MG_ERR_INVALID_ARG, "phases, state and out must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite");
    if (flags & ~(MG_ASSEMBLE_LAMBDA4_PRINTED | MG_ASSEMBLE_HARMONIC_K))
        return fail(MG_ERR_INVALID_ARG, "unknown assembly flags");
    for (int q = 0; q < 2; q++)
        if ((st = check_phase(phases[q]))) return st;
    const int dim = grid->dim;
    bool ok = device_ptr(s->C) && device_ptr(s->m1) && device_ptr(s->m2) && device_ptr(s->E) &&
              device_ptr(out->lambda) && device_ptr(out->rhs) && (!out->x0 || device_ptr(out->x0));
    for (int a = 0; a < dim; a++)
        ok = ok && device_ptr(s->mom[a]) && device_ptr(s->uf[a]) && device_ptr(out->face_alpha[a]) &&
             device_ptr(out->face_k[a]);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "every array must be a device pointer of the current device");
    if (!aligned16(out->lambda) || !aligned16(out->rhs) || (out->x0 && !aligned16(out->x0)))
        return fail(MG_ERR_INVALID_ARG, "lambda, rhs and x0 must be 16-byte aligned");
    AssembleArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < 3; a++) A.n[a] = grid->n[a];
    A.axisym = grid->axisym;
    A.r0 = grid->r0;
    A.h = grid->h;
    A.inv_h = 1.0 / grid->h;
    A.inv_dt = 1.0 / dt;
    A.inv_dt2 = 1.0 / (dt * dt);
    A.l4_scale = (flags & MG_ASSEMBLE_LAMBDA4_PRINTED) ? 1.0 : 1.0 / dt;
    A.harmonic_k = (flags & MG_ASSEMBLE_HARMONIC_K) ? 1 : 0;
    A.ph[0] = phase_k(phases[0]);
    A.ph[1] = phase_k(phases[1]);
    A.C = s->C;
    A.m1 = s->m1;
    A.m2 = s->m2;
    A.E = s->E;
    for (int a = 0; a < dim; a++) {
        A.mom[a] = s->mom[a];
        A.uf[a] = s->uf[a];
        A.fa[a] = out->face_alpha[a];
        A.fk[a] = out->face_k[a];
    }
    A.lam = reinterpret_cast<double2 *>(out->lambda);
    A.rhs = reinterpret_cast<double2 *>(out->rhs);
    A.x0 = reinterpret_cast<double2 *>(out->x0);
    const dim3 gr((unsigned)((grid->n[0] + kBX - 1) / kBX), (unsigned)((grid->n[1] + kBY - 1) / kBY),
                  (unsigned)(dim == 3 ? grid->n[2] : 1));
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dim == 3) k_assemble<3, false><<<gr, kBlock, 0, cs>>>(A);
    else if (grid->axisym) k_assemble<2, true><<<gr, kBlock, 0, cs>>>(A);
    else k_assemble<2, false><<<gr, kBlock, 0, cs>>>(A);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_correct_async(const mg_grid *grid, double dt, double sigma, const double *x, const double *C,
                           const double *kappa, const double *const face_alpha[3], const double *const uf_star[3],
                           double *const uf_out[3], double *p1, double *p2, void *stream) {
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (!face_alpha || !uf_star || !uf_out) return fail(MG_ERR_INVALID_ARG, "face array lists must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(sigma))
        return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite, sigma finite");
    const int dim = grid->dim;
    bool ok = device_ptr(x) && device_ptr(C) && device_ptr(kappa) && device_ptr(p1) && device_ptr(p2);
    for (int a = 0; a < dim; a++)
        ok = ok && device_ptr(face_alpha[a]) && device_ptr(uf_star[a]) && device_ptr(uf_out[a]);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "every array must be a device pointer of the current device");
    if (!aligned16(x)) return fail(MG_ERR_INVALID_ARG, "x must be 16-byte aligned");
    CorrectArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < 3; a++) {
        A.n[a] = grid->n[a];
        for (int sd = 0; sd < 2; sd++) {
            A.dir[a][sd] = a < dim && grid->bc[a][sd] == MG_BC_DIRICHLET;
            A.gp[a][sd] = a < dim ? grid->bc_p[a][sd] : 0.0;
        }
    }
    A.dt = dt;
    A.inv_h = 1.0 / grid->h;
    A.two_inv_h = 2.0 / grid->h;
    A.sigma = sigma;
    A.x = reinterpret_cast<const double2 *>(x);
    A.C = C;
    A.kappa = kappa;
    for (int a = 0; a < dim; a++) {
        A.fa[a] = face_alpha[a];
        A.uf[a] = uf_star[a];
        A.uo[a] = uf_out[a];
    }
    A.p1 = p1;
    A.p2 = p2;
    const dim3 gr((unsigned)((grid->n[0] + kBX - 1) / kBX), (unsigned)((grid->n[1] + kBY - 1) / kBY),
                  (unsigned)(dim == 3 ? grid->n[2] : 1));
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dim == 3) k_correct<3><<<gr, kBlock, 0, cs>>>(A);
    else k_correct<2><<<gr, kBlock, 0, cs>>>(A);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_energy_async(const mg_grid *grid, const mg_phase phases[2], double dt, const double *x, const double *C,
                          const double *p1, const double *p2, const double *const uf[3], const double *E1,
                          const double *E2, double *E1_out, double *E2_out, void *stream) {
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (!phases || !uf) return fail(MG_ERR_INVALID_ARG, "phases and uf must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite");
    for (int q = 0; q < 2; q++)
        if ((st = check_phase(phases[q]))) return st;
    const int dim = grid->dim;
    bool ok = device_ptr(x) && device_ptr(C) && device_ptr(p1) && device_ptr(p2) && device_ptr(E1) &&
              device_ptr(E2) && device_ptr(E1_out) && device_ptr(E2_out);
    for (int a = 0; a < dim; a++) ok = ok && device_ptr(uf[a]);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "every array must be a device pointer of the current device");
    if (!aligned16(x)) return fail(MG_ERR_INVALID_ARG, "x must be 16-byte aligned");
    bool alias = E1_out == E2_out || E1_out == E2 || E2_out == E1;
    for (const double *o : {(const double *)E1_out, (const double *)E2_out}) {
        alias = alias || o == x || o == C || o == p1 || o == p2;
        for (int a = 0; a < dim; a++) alias = alias || o == uf[a];
    }
    if (alias) return fail(MG_ERR_INVALID_ARG, "E1_out and E2_out may alias only their own phase's input");
    EnergyArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < 3; a++) {
        A.n[a] = grid->n[a];
        for (int sd = 0; sd < 2; sd++) {
            A.dir[a][sd] = a < dim && grid->bc[a][sd] == MG_BC_DIRICHLET;
            A.gT[a][sd] = a < dim ? grid->bc_T[a][sd] : 0.0;
            A.gp[a][sd] = a < dim ? grid->bc_p[a][sd] : 0.0;
        }
    }
    A.r0 = grid->r0;
    A.h = grid->h;
    A.inv_h = 1.0 / grid->h;
    A.half_inv_h = 0.5 / grid->h;
    A.two_inv_h = 2.0 / grid->h;
    A.dt = dt;
    for (int q = 0; q < 2; q++) {
        A.k[q] = phases[q].k;
        A.mu[q] = phases[q].mu;
    }
    A.x = reinterpret_cast<const double2 *>(x);
    A.C = C;
    A.p1 = p1;
    A.p2 = p2;
    for (int a = 0; a < dim; a++) A.uf[a] = uf[a];
    A.E1 = E1;
    A.E2 = E2;
    A.E1o = E1_out;
    A.E2o = E2_out;
    const dim3 gr((unsigned)((grid->n[0] + kBX - 1) / kBX), (unsigned)((grid->n[1] + kBY - 1) / kBY),
                  (unsigned)(dim == 3 ? grid->n[2] : 1));
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dim == 3) k_energy<3, false, kBX, kBY><<<gr, kBlock, 0, cs>>>(A);
    else if (grid->axisym) k_energy<2, true, kBX, kBY><<<gr, kBlock, 0, cs>>>(A);
    else k_energy<2, false, kBX, kBY><<<gr, kBlock, 0, cs>>>(A);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_residual_norms(mg_handle *h, const double *rhs, const double *x, int on_device, double out[2]) {
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (!rhs || !x || !out) return fail(MG_ERR_INVALID_ARG, "bad arguments to mg_residual_norms");
    DeviceGuard dg(h->device);
    if ((st = prep(h, rhs, x, on_device))) return st;
    if (h->grid.dim == 2) enqueue_norm<2>(h, h->stream, false);
    else enqueue_norm<3>(h, h->stream, false);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->norms_h, h->norms_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync_norms(h, out);
}

mg_status mg_get_tuning(const mg_handle *h, mg_tuning *out) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    get_tuning(h, out);
    return MG_OK;
}

mg_status mg_set_tuning(mg_handle *h, const mg_tuning *t) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (!t) return fail(MG_ERR_INVALID_ARG, "tuning is NULL");
    for (int l = 0; l < h->nlev; l++) {
        if (t->sweep[l] != MG_SWEEP_COLOUR && t->sweep[l] != MG_SWEEP_FUSED && t->sweep[l] != MG_SWEEP_ASYNC &&
            t->sweep[l] != MG_SWEEP_COLOUR2 && t->sweep[l] != MG_SWEEP_FUSED2)
            return fail(MG_ERR_INVALID_ARG, "sweep kind must be MG_SWEEP_COLOUR, MG_SWEEP_COLOUR2, MG_SWEEP_FUSED, "
                                            "MG_SWEEP_ASYNC or MG_SWEEP_FUSED2");
        if ((t->sweep[l] == MG_SWEEP_FUSED || t->sweep[l] == MG_SWEEP_ASYNC || t->sweep[l] == MG_SWEEP_FUSED2) &&
            h->grid.dim != 2)
            return fail(MG_ERR_INVALID_ARG, "fused sweeps are for 2D grids");
        if (t->sweep[l] == MG_SWEEP_FUSED2 && l + 1 < h->nlev && !fused2_ok(h->opt, h->grid.dim))
            return fail(MG_ERR_INVALID_ARG, "fused sweep pairs need red-black smoothing with nu1 / 2 + nu2 / 2 even");
        if (t->tile[l] < 0 || t->tile[l] >= kTileShapes) return fail(MG_ERR_INVALID_ARG, "tile shape out of range");
        if (t->sweep[l] == MG_SWEEP_ASYNC && l + 1 < h->nlev &&
            !(h->opt.precision == MG_MIXED ? async_ok<float>(h, l, t->tile[l]) : async_ok<double>(h, l, t->tile[l])))
            return fail(MG_ERR_INVALID_ARG, "async sweep does not fit this level (shared memory per block, or an "
                                            "odd FP32 row length)");
    }
    const bool no_tail = t->tail_level >= h->nlev;
    if (!no_tail && (t->tail_ctas != 1 && t->tail_ctas != kTailCtas && t->tail_ctas != 16))
        return fail(MG_ERR_INVALID_ARG, "tail cluster size must be 1, 8, or 16 where the device allows it");
    if (!no_tail && !tail_level_ok(h, t->tail_level, t->tail_ctas))
        return fail(MG_ERR_INVALID_ARG, "tail level must be >= 1, leave 2 to 12 levels, have <= 16384 cells "
                                        "and fit the tail's shared memory");
    DeviceGuard dg(h->device);
    if (!no_tail && !tail_ctas_ok(h, t->tail_ctas))
        return fail(MG_ERR_INVALID_ARG, "tail cluster size must be 1, 8, or 16 where the device allows it");
    if (t->persistent != 0 && t->persistent != 1) return fail(MG_ERR_INVALID_ARG, "persistent must be 0 or 1");
    if (t->overlap != 0 && t->overlap != 1) return fail(MG_ERR_INVALID_ARG, "overlap must be 0 or 1");
    CK(cudaStreamSynchronize(h->stream));
    for (int l = 0; l < h->nlev; l++) {
        h->sweep[l] = t->sweep[l];
        h->tile[l] = t->tile[l];
    }
    h->tail_lev = no_tail ? h->nlev : t->tail_level;
    h->tail_ctas = no_tail ? kTailCtas : t->tail_ctas;
    h->persistent = t->persistent;
    h->overlap = t->overlap;
    drop_graphs(h);
    return MG_OK;
}

mg_status mg_autotune(mg_handle *h, int reps, mg_tuning *out, double *vcycle_ms) {
    mg_status st = check_handle(h, true);
    if (st) return st;
    if (reps < 1 || reps > 1000) return fail(MG_ERR_INVALID_ARG, "reps must be in [1, 1000]");
    DeviceGuard dg(h->device);
    CK(cudaStreamSynchronize(h->stream));
    // scratch state to zeros: every candidate then runs on the same finite data
    for (int l = 0; l < h->nlev; l++) {
        const LevelBuf &b = h->L[l];
        void *ptrs[8] = {b.x, b.b, b.bt, b.xalt, b.x32, b.b32, b.bt32, b.xalt32};
        const size_t sz[8] = {16, 16, 16, 16, 8, 8, 8, 8};
        for (int q = 0; q < 8; q++)
            if (ptrs[q]) CK(cudaMemsetAsync(ptrs[q], 0, sz[q] * (size_t)b.N, h->stream));
    }
    const int timing = h->timing;
    h->timing = 0;
    const bool mixed = h->opt.precision == MG_MIXED;
    if (h->grid.dim == 2) st = mixed ? autotune_impl<float, 2>(h, reps, vcycle_ms) : autotune_impl<double, 2>(h, reps, vcycle_ms);
    else st = mixed ? autotune_impl<float, 3>(h, reps, vcycle_ms) : autotune_impl<double, 3>(h, reps, vcycle_ms);
    h->timing = timing;
    drop_graphs(h);
    CK(cudaStreamSynchronize(h->stream));
    if (st) return st;
    if (out) get_tuning(h, out);
    return MG_OK;
}

mg_status mg_set_timing(mg_handle *h, int enable) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    DeviceGuard dg(h->device);
    CK(cudaStreamSynchronize(h->stream));
    if (enable && !h->ev[0])
        for (int q = 0; q < 2; q++) CK(cudaEventCreate(&h->ev[q]));
    // re-capture the cycle graphs with (or without) the event nodes when that changes
    if ((enable ? 1 : 0) != h->timing) drop_graphs(h);
    h->timing = enable ? 1 : 0;
    h->enq = 0;
    h->smooth_ms = 0.0;
    h->smooth_launches = 0;
    h->smooth_sweeps = 0;
    return MG_OK;
}

mg_status mg_counters(const mg_handle *h, long long *launches, double *smooth_ms, long long *smooth_launches,
                      long long *smooth_sweeps, long long *smooth_cells) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (launches) *launches = h->enq;
    if (smooth_ms) *smooth_ms = h->smooth_ms;
    if (smooth_launches) *smooth_launches = h->smooth_launches;
    if (smooth_sweeps) *smooth_sweeps = h->smooth_sweeps;
    if (smooth_cells) *smooth_cells = h->L[0].N;
    return MG_OK;
}

mg_status mg_set_stream(mg_handle *h, void *stream) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    DeviceGuard dg(h->device);
    // Only mg_set_coeffs and mg_solve_async return with the handle's work
    // still running; the new stream waits (on the device) for the end of the
    // last of them.  The old stream's later work, another handle's, is not
    // waited for, and the host does not block.
    const cudaStream_t next = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaStreamWaitEvent(next, h->ev_last, 0));
    h->stream = next;
    return MG_OK;
}

mg_status mg_set_device(int device) {
    CK(cudaSetDevice(device));
    return MG_OK;
}

mg_status mg_levels(const mg_handle *h, int *levels, int *n_out) {
    mg_status st = check_handle(h, false);
    if (st) return st;
    if (levels) *levels = h->nlev;
    if (n_out)
        for (int l = 0; l < h->nlev; l++)
            for (int a = 0; a < 3; a++) n_out[3 * l + a] = h->L[l].n[a];
    return MG_OK;
}

mg_status mg_destroy(mg_handle *h) {
    if (!h) return MG_OK;
    DeviceGuard dg(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->g64) cudaGraphExecDestroy(h->g64);
    if (h->gasync) cudaGraphExecDestroy(h->gasync);
    if (h->gcorr) cudaGraphExecDestroy(h->gcorr);
    for (auto &sg : h->gsetup)
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (h->g32) cudaGraphExecDestroy(h->g32);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->cap2) cudaStreamDestroy(h->cap2);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_a0) cudaEventDestroy(h->ev_a0);
    if (h->ev_a1) cudaEventDestroy(h->ev_a1);
    if (h->astat_h) cudaFreeHost(h->astat_h);
    if (h->ev_asm) cudaEventDestroy(h->ev_asm);
    if (h->ev_inv) cudaEventDestroy(h->ev_inv);
    if (h->ev_last) cudaEventDestroy(h->ev_last);
    if (h->errh) cudaFreeHost(h->errh);
    for (int q = 0; q < 2; q++)
        if (h->ev[q]) cudaEventDestroy(h->ev[q]);
    if (h->norms_h) cudaFreeHost(h->norms_h);
    if (h->owns_arena && h->arena) cudaFree(h->arena);
    delete[] h->tmaps;
    delete[] h->tmap_ok;
    delete h;
    return MG_OK;
}

#include "mg_momentum_api.cuh"
#include "mg_composite_api.cuh"

const char *mg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

#include "mg_batch.cuh"
