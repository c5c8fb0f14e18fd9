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
    BcFlags bc;
    int problem;
};

struct BProb {                  // one problem, device side
    double2 *partial;
    unsigned int *ticket;
    const double *Minv;
    const float *Minv32;
    int nc;
    int coarse;                 // index of its coarsest level in the BLevel table
    int npartial;
    float2 *x32_0;              // finest-level FP32 correction (mixed)
};

struct BState {                 // per-problem solve state, device side
    double n0[2];
    double nk[2];
    int cycles;
    int active;
};

constexpr int kBatchThreads = 256;
constexpr int kBatchBlocksPerSM = 8;
constexpr int kSMs = 152;

template <typename R> __device__ __forceinline__ const Level<R> &pick(const BLevel &L);
template <> __device__ __forceinline__ const Level<double> &pick<double>(const BLevel &L) { return L.d; }
template <> __device__ __forceinline__ const Level<float> &pick<float>(const BLevel &L) { return L.f; }
template <typename R> __device__ __forceinline__ typename Vec<R>::v2 *pick_alt(const BLevel &L);
template <> __device__ __forceinline__ double2 *pick_alt<double>(const BLevel &L) { return L.xalt; }
template <> __device__ __forceinline__ float2 *pick_alt<float>(const BLevel &L) { return L.xalt32; }

__device__ __forceinline__ void block_coords(int local, int gx, int gy, int &bx, int &by, int &bz) {
    bx = local % gx;
    by = (local / gx) % gy;
    bz = local / (gx * gy);
}

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

template <typename R>
__global__ void __launch_bounds__(kBatchThreads) kb_rbgs_fused2d(const BLevel *__restrict__ lv,
                                                                 const BState *__restrict__ st,
                                                                 const int2 *__restrict__ tab, int n, int to_alt) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> L = pick<R>(B);
        typename Vec<R>::v2 *xa = pick_alt<R>(B);
        const int gx = (L.n0 + kFTX - 1) / kFTX;
        const int bx = e.y % gx, by = e.y / gx;
        if (to_alt) rbgs_fused2d_block<R>(L, L.x, xa, bx, by);
        else rbgs_fused2d_block<R>(L, xa, L.x, bx, by);
    }
}

template <typename R, int DIM>
__global__ void __launch_bounds__(kBatchThreads) kb_restrict(const BLevel *__restrict__ lv,
                                                             const BState *__restrict__ st,
                                                             const int2 *__restrict__ tab, int n) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        if (!st[B.problem].active) continue;
        const Level<R> F = pick<R>(B);
        const Level<R> Cc = pick<R>(lv[e.x + 1]);
        const int gx = (Cc.n0 + kBX - 1) / kBX, gy = (Cc.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        residual_restrict_block<R, DIM>(F, Cc, bx, by, bz);
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
                                                         int initial, double rtol, int max_cycles,
                                                         int *__restrict__ active_count) {
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        __syncthreads();
        const int2 e = tab[v];
        const BLevel &B = lv[e.x];
        const int p = B.problem;
        if (!initial && !st[p].active) continue;
        const Level<double> L = B.d;
        const int gx = (L.n0 + kBX - 1) / kBX, gy = (L.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        const double2 s = norm_block<DIM>(L, bx, by, bz);
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
        const Level<double> L = B.d;
        const int gx = (L.n0 + kBX - 1) / kBX, gy = (L.n1 + kBY - 1) / kBY;
        int bx, by, bz;
        block_coords(e.y, gx, gy, bx, by, bz);
        const double2 s = residual64_to32_block<DIM>(L, B.f.b, B.f.x, bx, by, bz);
        batch_finish(pr[p], st[p], e.y, s, initial, rtol, max_cycles, active_count);
    }
}

// Mixed precision: x64 += e32 on the finest level of active problems.
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
        double2 xv = B.d.x[c];
        xv.x += (double)d.x;
        xv.y += (double)d.y;
        B.d.x[c] = xv;
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
    std::vector<std::pair<long long, int>> colour, fused, restr, prolong;
    std::pair<long long, int> norm, coarse, cells0;
    cudaGraphExec_t graph;
    long long graph_kernels;
    long long launches;
};

namespace {

unsigned batch_grid(int n) {
    const int cap = kSMs * kBatchBlocksPerSM;
    return (unsigned)std::max(1, std::min(n, cap));
}

template <typename R, int DIM>
void b_smooth(mg_batch *b, cudaStream_t s, int d, int sweeps) {
    const int2 *ct = b->tabs + b->colour[d].first;
    const int nc = b->colour[d].second;
    int q = 0;
    if (fused_sweeps<R, DIM>()) {
        const int2 *ft = b->tabs + b->fused[d].first;
        const int nf = b->fused[d].second;
        for (; q + 1 < sweeps; q += 2) {
            kb_rbgs_fused2d<R><<<batch_grid(nf), kBlock, 0, s>>>(b->lv, b->st, ft, nf, 1);
            kb_rbgs_fused2d<R><<<batch_grid(nf), kBlock, 0, s>>>(b->lv, b->st, ft, nf, 0);
            b->launches += 2;
        }
    }
    for (; q < sweeps; q++) {
        kb_rbgs_colour<R, DIM><<<batch_grid(nc), kBlock, 0, s>>>(b->lv, b->st, ct, nc, 0);
        kb_rbgs_colour<R, DIM><<<batch_grid(nc), kBlock, 0, s>>>(b->lv, b->st, ct, nc, 1);
        b->launches += 2;
    }
}

template <typename R, int DIM>
void b_vcycle(mg_batch *b, cudaStream_t s) {
    for (int d = 0; d + 1 < b->dmax; d++) {
        if (b->colour[d].second == 0) continue;
        b_smooth<R, DIM>(b, s, d, b->opt.nu1);
        const int nr = b->restr[d].second;
        kb_restrict<R, DIM><<<batch_grid(nr), kBlock, 0, s>>>(b->lv, b->st, b->tabs + b->restr[d].first, nr);
        b->launches++;
    }
    const int ncs = b->coarse.second;
    kb_coarse<R><<<batch_grid(ncs), kBatchThreads, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->coarse.first, ncs);
    b->launches++;
    for (int d = b->dmax - 2; d >= 0; d--) {
        if (b->colour[d].second == 0) continue;
        const int np = b->prolong[d].second;
        kb_prolong<R, DIM><<<batch_grid(np), kBlock, 0, s>>>(b->lv, b->st, b->tabs + b->prolong[d].first, np);
        b->launches++;
        b_smooth<R, DIM>(b, s, d, b->opt.nu2);
    }
}

template <int DIM>
void b_norm(mg_batch *b, cudaStream_t s, int initial) {
    cudaMemsetAsync(b->active_count, 0, sizeof(int), s);
    const int n = b->norm.second;
    if (b->opt.precision == MG_FP64)
        kb_norm<DIM><<<batch_grid(n), kBlock, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->norm.first, n, initial,
                                                      b->opt.rtol, b->opt.max_cycles, b->active_count);
    else
        kb_residual64<DIM><<<batch_grid(n), kBlock, 0, s>>>(b->lv, b->pr, b->st, b->tabs + b->norm.first, n, initial,
                                                            b->opt.rtol, b->opt.max_cycles, b->active_count);
    b->launches++;
    cudaMemcpyAsync(b->active_h, b->active_count, sizeof(int), cudaMemcpyDeviceToHost, s);
}

template <int DIM>
void b_step(mg_batch *b, cudaStream_t s) {
    if (b->opt.precision == MG_FP64) {
        b_vcycle<double, DIM>(b, s);
    } else {
        for (int q = 0; q < b->opt.inner_cycles; q++) b_vcycle<float, DIM>(b, s);
        const int n = b->cells0.second;
        kb_add_correction<<<batch_grid(n), kBatchThreads, 0, s>>>(b->lv, b->st, b->tabs + b->cells0.first, n);
        b->launches++;
    }
    b_norm<DIM>(b, s, 0);
}

bool same_options(const mg_options &a, const mg_options &c) {
    return a.nu1 == c.nu1 && a.nu2 == c.nu2 && a.precision == c.precision && a.rtol == c.rtol &&
           a.max_cycles == c.max_cycles && a.inner_cycles == c.inner_cycles;
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
    mg_batch *b = new (std::nothrow) mg_batch();
    if (!b) return fail(MG_ERR_OOM, "host allocation failed");
    b->count = count;
    b->dim = handles[0]->grid.dim;
    b->opt = handles[0]->opt;
    b->stream = handles[0]->stream;
    b->device = handles[0]->device;
    b->h.assign(handles, handles + count);
    DeviceGuard dg(b->device);
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
            d.bc = bc_flags(h->grid);
            d.problem = p;
            lv.push_back(d);
        }
        pr[p].partial = h->partial;
        pr[p].ticket = h->ticket;
        pr[p].Minv = h->Minv;
        pr[p].Minv32 = h->Minv32;
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
        std::vector<int2> tc, tf, tr, tp;
        for (int p = 0; p < count; p++) {
            const mg_handle *h = handles[p];
            if (h->nlev - 1 <= d) continue;
            const LevelBuf &F = h->L[d], &Cl = h->L[d + 1];
            const int li = base[p] + d;
            add_blocks(tc, li, (long long)cell_grid(F, dim, (F.n[0] + 1) / 2).x * cell_grid(F, dim, 1).y *
                                   cell_grid(F, dim, 1).z);
            if (dim == 2)
                add_blocks(tf, li, (long long)((F.n[0] + kFTX - 1) / kFTX) * ((F.n[1] + kFTY - 1) / kFTY));
            const dim3 gc = cell_grid(Cl, dim, Cl.n[0]);
            add_blocks(tr, li, (long long)gc.x * gc.y * gc.z);
            const dim3 gf = cell_grid(F, dim, F.n[0]);
            add_blocks(tp, li, (long long)gf.x * gf.y * gf.z);
        }
        b->colour.push_back(slice(tc));
        b->fused.push_back(slice(tf));
        b->restr.push_back(slice(tr));
        b->prolong.push_back(slice(tp));
    }
    std::vector<int2> tn, tco, tcell;
    for (int p = 0; p < count; p++) {
        const mg_handle *h = handles[p];
        const dim3 g0 = cell_grid(h->L[0], dim, h->L[0].n[0]);
        add_blocks(tn, base[p], (long long)g0.x * g0.y * g0.z);
        for (int r = 0; r < (h->nc + 7) / 8; r++) tco.push_back(make_int2(p, r));
        add_blocks(tcell, base[p], (h->L[0].N + kBatchThreads - 1) / kBatchThreads);
    }
    b->norm = slice(tn);
    b->coarse = slice(tco);
    b->cells0 = slice(tcell);
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
                 o_tab = take(sizeof(int2) * std::max<size_t>(1, tabs.size()));
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
    if (cudaMemcpy(b->lv, lv.data(), sizeof(BLevel) * lv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->pr, pr.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        (tabs.size() && cudaMemcpy(b->tabs, tabs.data(), sizeof(int2) * tabs.size(), cudaMemcpyHostToDevice) !=
                            cudaSuccess) ||
        cudaMemset(b->st, 0, sizeof(BState) * count) != cudaSuccess ||
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
    for (int p = 0; p < b->count; p++) {
        mg_status st = prep(b->h[p], rhs[p], x[p], on_device);
        if (st) return st;
    }
    cudaStream_t s = b->stream;
    if (b->dim == 2) b_norm<2>(b, s, 1);
    else b_norm<3>(b, s, 1);
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
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
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
    std::vector<BState> host(b->count);
    CK(cudaMemcpyAsync(host.data(), b->st, sizeof(BState) * b->count, cudaMemcpyDeviceToHost, s));
    for (int p = 0; p < b->count; p++) {
        mg_status st = x_out(b->h[p], x[p], on_device);
        if (st) return st;
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
        }
    }
    if (!all_ok) return fail(MG_ERR_NOT_CONVERGED, "at least one problem did not converge in max_cycles");
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
    if (b->mem) cudaFree(b->mem);
    delete b;
    return MG_OK;
}

}  // extern "C"
