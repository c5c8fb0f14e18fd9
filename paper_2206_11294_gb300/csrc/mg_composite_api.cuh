// C ABI of the refined-patch (adaptive) grid solve: mg_composite_*.
// Included by mg_capi.cu (it drives a base-grid handle's V-cycle).
#include "mg_composite.cuh"

struct mg_composite {
    mg_grid base;
    int box[2][2];
    mg_options opt;
    int device;
    cudaStream_t stream;
    CfGeom g, g0;              // with the grid's Dirichlet values, and with zeros (correction problems)
    mg_handle *hb;             // the base grid's hierarchy: the FAC cycle's base correction
    long long Nb, Nf, nfb[2], nff[2];
    char *arena;
    // the caller's coefficients, copied (physical, unscaled)
    double *lamb, *fab[2], *fkb[2], *lamf, *faf[2], *fkf[2];
    // the base hierarchy's coefficients (covered cells from the patch)
    double *clam, *cfa[2], *cfk[2];
    double2 *rb, *rf, *sb, *sf, *df, *zb, *xb, *xf, *bb, *bf;
    double *partial, *norms_d, *norms_h;
    unsigned int *ticket;
    int nblk;
    bool coeffs_set;
    cudaGraphExec_t gcyc;      // one FAC cycle and the new residuals (captured at the first solve)
};

namespace {

CfCoef cf_coef(const mg_composite *m) {
    CfCoef k;
    k.lamb = m->lamb;
    k.lamf = m->lamf;
    for (int a = 0; a < 2; a++) {
        k.fab[a] = m->fab[a];
        k.fkb[a] = m->fkb[a];
        k.faf[a] = m->faf[a];
        k.fkf[a] = m->fkf[a];
    }
    return k;
}

dim3 cf_grid2(int nx, int ny) { return dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + 7) / 8), 1); }

// (T, p) norms of the current residuals rb, rf into norms_h (after the stream is synchronised)
void cf_enqueue_norms(mg_composite *m) {
    k_cf_norms<<<m->nblk, 256, 0, m->stream>>>(m->g, m->rb, m->rf, m->Nb, m->Nf, m->partial, m->ticket, m->norms_d);
    cudaMemcpyAsync(m->norms_h, m->norms_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
}

// The composite residuals r = b - L(x) of the current x.
void cf_enqueue_residual(mg_composite *m, cudaStream_t s) {
    const CfCoef k = cf_coef(m);
    k_cf_rows_base<<<cf_grid2(m->g.n0, m->g.n1), dim3(32, 8), 0, s>>>(m->g, k, m->xb, m->xf, m->bb, m->rb);
    k_cf_rows_fine<<<cf_grid2(m->g.m0, m->g.m1), dim3(32, 8), 0, s>>>(m->g, k, m->xb, m->xf, m->bf, m->rf);
}

void cf_enqueue_sweeps(mg_composite *m, cudaStream_t s, const double2 *rhs, int sweeps) {
    const CfCoef k = cf_coef(m);
    const dim3 gr = cf_grid2((m->g.m0 + 1) / 2, m->g.m1);
    for (int q = 0; q < sweeps; q++)
        for (int colour = 0; colour < 2; colour++)
            k_cf_rbgs_fine<<<gr, dim3(32, 8), 0, s>>>(m->g0, k, m->zb, rhs, m->df, colour);
}

// One FAC cycle on the residuals rb, rf, x += the correction, and the
// residuals of the new x.
mg_status cf_enqueue_fac_cycle(mg_composite *m, cudaStream_t s) {
    const CfCoef k = cf_coef(m);
    CK(cudaMemsetAsync(m->df, 0, sizeof(double2) * m->Nf, s));
    cf_enqueue_sweeps(m, s, m->rf, m->opt.nu1);
    // the patch residual of the correction (zero base values), then the base right-hand side
    k_cf_rows_fine<<<cf_grid2(m->g.m0, m->g.m1), dim3(32, 8), 0, s>>>(m->g0, k, m->zb, m->df, m->rf, m->sf);
    k_cf_base_rhs<<<cf_grid2(m->g.n0, m->g.n1), dim3(32, 8), 0, s>>>(m->g0, k, m->rb, m->df, m->sf, m->sb);
    // one V-cycle of the base hierarchy from zero; the result is in its finest level's x
    mg_status st = enqueue_correction<2>(m->hb, s, m->sb);
    if (st) return st;
    const double2 *db = m->hb->L[0].x;
    k_cf_prolong_ghost<<<cf_grid2(m->g.m0, m->g.m1), dim3(32, 8), 0, s>>>(m->g0, k, db, m->rf, m->df, m->sf);
    cf_enqueue_sweeps(m, s, m->sf, m->opt.nu2);
    const dim3 ug = cf_grid2(std::max(m->g.n0, m->g.m0), std::max(m->g.n1, m->g.m1));
    k_cf_update<<<ug, dim3(32, 8), 0, s>>>(m->g, m->xb, m->xf, db, m->df);
    cf_enqueue_residual(m, s);
    CK(cudaGetLastError());
    return MG_OK;
}

// The FAC cycle as one graph, captured on the base handle's private capture
// stream (the caller's stream may be the legacy default stream, which cannot
// be captured).  Every pointer it uses is fixed for the handle's life.
mg_status cf_capture(mg_composite *m) {
    cudaStream_t cs = m->hb->cap;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const mg_status st = cf_enqueue_fac_cycle(m, cs);
    const cudaError_t le = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (st || le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        if (st) return st;
        return fail(MG_ERR_CUDA, std::string("FAC cycle capture: ") + cudaGetErrorString(le ? le : e));
    }
    e = cudaGraphInstantiate(&m->gcyc, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        m->gcyc = nullptr;
        return fail(MG_ERR_CUDA, std::string("FAC cycle graph instantiate: ") + cudaGetErrorString(e));
    }
    return MG_OK;
}

mg_status cf_check_pair(const double *p) {
    if (!p) return fail(MG_ERR_INVALID_ARG, "NULL array");
    if (!aligned16(p)) return fail(MG_ERR_INVALID_ARG, "pair arrays must be 16-byte aligned");
    return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_composite_create(const mg_grid *grid, const int box[2][2], const mg_options *opt, void *stream,
                              mg_composite **out) {
    if (!out || !box) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (grid->dim != 2 || grid->axisym) return fail(MG_ERR_INVALID_ARG, "refined-patch grids are 2D Cartesian");
    for (int a = 0; a < 2; a++) {
        if (!(0 <= box[a][0] && box[a][0] < box[a][1] && box[a][1] <= grid->n[a]))
            return fail(MG_ERR_INVALID_ARG, "the box must be a non-empty range of base cells on each axis");
        for (int sd = 0; sd < 2; sd++)
            if (grid->bc[a][sd] == MG_BC_AXIS) return fail(MG_ERR_INVALID_ARG, "no symmetry axis on a Cartesian grid");
    }
    mg_options o;
    if (opt) o = *opt;
    else mg_default_options(&o);
    if (o.precision != MG_FP64 && o.precision != MG_MIXED)
        return fail(MG_ERR_INVALID_ARG, "precision must be MG_FP64 or MG_MIXED");
    if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 16 || o.nu2 > 16 || o.nu1 + o.nu2 == 0)
        return fail(MG_ERR_INVALID_ARG, "nu1, nu2 must be in 0..16 and not both zero");
    mg_composite *m = new (std::nothrow) mg_composite();
    if (!m) return fail(MG_ERR_OOM, "host allocation failed");
    m->base = *grid;
    std::memcpy(m->box, box, sizeof(m->box));
    m->opt = o;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&m->device);
    CfGeom &g = m->g;
    std::memset(&g, 0, sizeof(g));
    g.n0 = grid->n[0];
    g.n1 = grid->n[1];
    for (int a = 0; a < 2; a++) {
        g.b0[a] = box[a][0];
        g.b1[a] = box[a][1];
        for (int sd = 0; sd < 2; sd++) {
            g.dir[a][sd] = grid->bc[a][sd] == MG_BC_DIRICHLET;
            g.gT[a][sd] = g.dir[a][sd] ? grid->bc_T[a][sd] : 0.0;
            g.gp[a][sd] = g.dir[a][sd] ? grid->bc_p[a][sd] : 0.0;
        }
        g.iface[a][0] = box[a][0] > 0;
        g.iface[a][1] = box[a][1] < grid->n[a];
    }
    g.m0 = 2 * (box[0][1] - box[0][0]);
    g.m1 = 2 * (box[1][1] - box[1][0]);
    g.H = grid->h;
    g.h = 0.5 * grid->h;
    g.rh2 = 1.0 / (g.h * g.h);
    g.rif = 1.0 / (1.5 * g.h * g.h);
    g.rdf = 1.0 / (0.5 * g.h * g.h);
    g.rH2 = 1.0 / (g.H * g.H);
    g.rdb = 1.0 / (0.5 * g.H * g.H);
    g.rbif = 1.0 / (1.5 * g.H * g.H);
    m->g0 = g;
    std::memset(m->g0.gT, 0, sizeof(m->g0.gT));
    std::memset(m->g0.gp, 0, sizeof(m->g0.gp));
    // the base hierarchy: the same grid with zero Dirichlet values (its cycles solve for corrections)
    mg_grid bg = *grid;
    std::memset(bg.bc_T, 0, sizeof(bg.bc_T));
    std::memset(bg.bc_p, 0, sizeof(bg.bc_p));
    mg_options bo = o;
    bo.rtol = 0.0;
    bo.max_cycles = 1;
    bo.cycle = MG_CYCLE_V;
    bo.smoother = MG_SMOOTH_RBGS;
    st = mg_create(&bg, &bo, nullptr, 0, stream, &m->hb);
    if (st) {
        delete m;
        return st;
    }
    m->Nb = (long long)g.n0 * g.n1;
    m->Nf = (long long)g.m0 * g.m1;
    m->nfb[0] = (long long)(g.n0 + 1) * g.n1;
    m->nfb[1] = (long long)g.n0 * (g.n1 + 1);
    m->nff[0] = (long long)(g.m0 + 1) * g.m1;
    m->nff[1] = (long long)g.m0 * (g.m1 + 1);
    m->nblk = 152 * 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) / 256 * 256;
        const size_t o2 = off;
        off += bytes;
        return o2;
    };
    const size_t o_lamb = take(32 * m->Nb), o_lamf = take(32 * m->Nf), o_clam = take(32 * m->Nb);
    size_t o_fb[2][3], o_ff[2][2];
    for (int a = 0; a < 2; a++) {
        for (int q = 0; q < 3; q++) o_fb[a][q] = take(8 * m->nfb[a]);    // fa, fk, and the hierarchy's fa / fk pair
        for (int q = 0; q < 2; q++) o_ff[a][q] = take(8 * m->nff[a]);
    }
    const size_t o_cfk[2] = {take(8 * m->nfb[0]), take(8 * m->nfb[1])};
    const size_t o_pairs_b = take(16 * m->Nb * 5), o_pairs_f = take(16 * m->Nf * 5);
    const size_t o_part = take(8 * 4 * (size_t)m->nblk), o_norm = take(8 * 4), o_tick = take(4);
    if (cudaMalloc(&m->arena, off + 256) != cudaSuccess) {
        cudaGetLastError();
        mg_destroy(m->hb);
        delete m;
        return fail(MG_ERR_OOM, "refined-patch arrays: device allocation failed");
    }
    char *A = m->arena;
    m->lamb = reinterpret_cast<double *>(A + o_lamb);
    m->lamf = reinterpret_cast<double *>(A + o_lamf);
    m->clam = reinterpret_cast<double *>(A + o_clam);
    for (int a = 0; a < 2; a++) {
        m->fab[a] = reinterpret_cast<double *>(A + o_fb[a][0]);
        m->fkb[a] = reinterpret_cast<double *>(A + o_fb[a][1]);
        m->cfa[a] = reinterpret_cast<double *>(A + o_fb[a][2]);
        m->cfk[a] = reinterpret_cast<double *>(A + o_cfk[a]);
        m->faf[a] = reinterpret_cast<double *>(A + o_ff[a][0]);
        m->fkf[a] = reinterpret_cast<double *>(A + o_ff[a][1]);
    }
    double2 *pb = reinterpret_cast<double2 *>(A + o_pairs_b), *pf = reinterpret_cast<double2 *>(A + o_pairs_f);
    m->rb = pb;
    m->sb = pb + m->Nb;
    m->zb = pb + 2 * m->Nb;
    m->xb = pb + 3 * m->Nb;
    m->bb = pb + 4 * m->Nb;
    m->rf = pf;
    m->sf = pf + m->Nf;
    m->df = pf + 2 * m->Nf;
    m->xf = pf + 3 * m->Nf;
    m->bf = pf + 4 * m->Nf;
    m->partial = reinterpret_cast<double *>(A + o_part);
    m->norms_d = reinterpret_cast<double *>(A + o_norm);
    m->ticket = reinterpret_cast<unsigned int *>(A + o_tick);
    if (cudaMallocHost(&m->norms_h, 4 * sizeof(double)) != cudaSuccess ||
        cudaMemsetAsync(m->zb, 0, sizeof(double2) * m->Nb, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->ticket, 0, sizeof(unsigned int), m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        mg_composite_destroy(m);
        return fail(MG_ERR_CUDA, "refined-patch set-up failed");
    }
    *out = m;
    return MG_OK;
}

mg_status mg_composite_set_coeffs(mg_composite *m, const double *lam_b, const double *const fa_b[3],
                                  const double *const fk_b[3], const double *lam_f, const double *const fa_f[3],
                                  const double *const fk_f[3]) {
    if (!m || !lam_b || !fa_b || !fk_b || !lam_f || !fa_f || !fk_f) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    for (int a = 0; a < 2; a++)
        if (!fa_b[a] || !fk_b[a] || !fa_f[a] || !fk_f[a]) return fail(MG_ERR_INVALID_ARG, "NULL face array");
    DeviceGuard dg(m->device);
    cudaStream_t s = m->stream;
    CK(cudaMemcpyAsync(m->lamb, lam_b, 32 * m->Nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->lamf, lam_f, 32 * m->Nf, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->clam, lam_b, 32 * m->Nb, cudaMemcpyDeviceToDevice, s));
    for (int a = 0; a < 2; a++) {
        CK(cudaMemcpyAsync(m->fab[a], fa_b[a], 8 * m->nfb[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(m->fkb[a], fk_b[a], 8 * m->nfb[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(m->cfa[a], fa_b[a], 8 * m->nfb[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(m->cfk[a], fk_b[a], 8 * m->nfb[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(m->faf[a], fa_f[a], 8 * m->nff[a], cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(m->fkf[a], fk_f[a], 8 * m->nff[a], cudaMemcpyDeviceToDevice, s));
    }
    const int bx = m->g.b1[0] - m->g.b0[0], by = m->g.b1[1] - m->g.b0[1];
    k_cf_cover<<<cf_grid2(bx, by), dim3(32, 8), 0, s>>>(m->g, cf_coef(m), m->clam, m->cfa[0], m->cfa[1], m->cfk[0],
                                                        m->cfk[1]);
    CK(cudaGetLastError());
    const double *pa[3] = {m->cfa[0], m->cfa[1], nullptr}, *pk[3] = {m->cfk[0], m->cfk[1], nullptr};
    mg_status st = mg_set_coeffs(m->hb, m->clam, pa, pk, 1);
    if (st) return st;
    m->coeffs_set = true;
    return MG_OK;
}

mg_status mg_composite_apply(mg_composite *m, const double *xb, const double *xf, double *yb, double *yf) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "NULL handle");
    if (!m->coeffs_set) return fail(MG_ERR_STATE, "mg_composite_set_coeffs has not succeeded");
    mg_status st;
    if ((st = cf_check_pair(xb)) || (st = cf_check_pair(xf)) || (st = cf_check_pair(yb)) || (st = cf_check_pair(yf)))
        return st;
    DeviceGuard dg(m->device);
    const CfCoef k = cf_coef(m);
    const double2 *xb2 = reinterpret_cast<const double2 *>(xb), *xf2 = reinterpret_cast<const double2 *>(xf);
    k_cf_rows_base<<<cf_grid2(m->g.n0, m->g.n1), dim3(32, 8), 0, m->stream>>>(m->g, k, xb2, xf2, nullptr,
                                                                             reinterpret_cast<double2 *>(yb));
    k_cf_rows_fine<<<cf_grid2(m->g.m0, m->g.m1), dim3(32, 8), 0, m->stream>>>(m->g, k, xb2, xf2, nullptr,
                                                                             reinterpret_cast<double2 *>(yf));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(m->stream));
    return MG_OK;
}

mg_status mg_composite_solve(mg_composite *m, const double *bb, const double *bf, double *xb, double *xf,
                             int cycles, double *norms) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "NULL handle");
    if (!m->coeffs_set) return fail(MG_ERR_STATE, "mg_composite_set_coeffs has not succeeded");
    if (cycles < 0 || cycles > 10000) return fail(MG_ERR_INVALID_ARG, "cycles must be in 0..10000");
    mg_status st;
    if ((st = cf_check_pair(bb)) || (st = cf_check_pair(bf)) || (st = cf_check_pair(xb)) || (st = cf_check_pair(xf)))
        return st;
    DeviceGuard dg(m->device);
    cudaStream_t s = m->stream;
    CK(cudaMemcpyAsync(m->bb, bb, 16 * m->Nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->bf, bf, 16 * m->Nf, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->xb, xb, 16 * m->Nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(m->xf, xf, 16 * m->Nf, cudaMemcpyDeviceToDevice, s));
    if (cycles > 0 && !m->gcyc && (st = cf_capture(m))) return st;
    cf_enqueue_residual(m, s);
    for (int k = 0;; k++) {
        if (norms) {
            cf_enqueue_norms(m);
            CK(cudaStreamSynchronize(s));
            for (int q = 0; q < 4; q++) norms[4 * k + q] = m->norms_h[q];
        }
        if (k == cycles) break;
        CK(cudaGraphLaunch(m->gcyc, s));
    }
    const int bx = m->g.b1[0] - m->g.b0[0], by = m->g.b1[1] - m->g.b0[1];
    k_cf_covered_mean<<<cf_grid2(bx, by), dim3(32, 8), 0, s>>>(m->g, m->xb, m->xf);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(xb, m->xb, 16 * m->Nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(xf, m->xf, 16 * m->Nf, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamWaitEvent(s, m->hb->ev_inv, 0));
    CK(cudaMemcpyAsync(m->hb->errh, m->hb->err_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (m->hb->errh[0] & 4) return fail(MG_ERR_INVALID_COEFF, "the base grid's coarsest-level matrix is singular");
    return MG_OK;
}

mg_status mg_composite_autotune(mg_composite *m, int reps, double *vcycle_ms) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "NULL handle");
    if (!m->coeffs_set) return fail(MG_ERR_STATE, "mg_composite_set_coeffs has not succeeded");
    DeviceGuard dg(m->device);
    const mg_status st = mg_autotune(m->hb, reps, nullptr, vcycle_ms);
    // the FAC cycle graph holds the base hierarchy's former kernel choices
    if (m->gcyc) {
        cudaGraphExecDestroy(m->gcyc);
        m->gcyc = nullptr;
    }
    return st;
}

mg_status mg_composite_destroy(mg_composite *m) {
    if (!m) return MG_OK;
    DeviceGuard dg(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->gcyc) cudaGraphExecDestroy(m->gcyc);
    if (m->hb) mg_destroy(m->hb);
    if (m->arena) cudaFree(m->arena);
    if (m->norms_h) cudaFreeHost(m->norms_h);
    delete m;
    return MG_OK;
}

}  // extern "C"
