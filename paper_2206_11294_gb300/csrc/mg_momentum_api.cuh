// C ABI of the implicit momentum predictor (mg_momentum_*) and of the steps either side of it
// (mg_momentum_rhs_async, mg_provisional_async).  Included by mg_capi.cu inside its extern "C" block, after the
// handle, the correction cycles (correction_cycles, handle_errors) and the argument helpers it uses.
#pragma once

struct mg_momentum {
    mg_grid grid;
    int flags, device;
    cudaStream_t stream;
    mg_handle *hA, *hB;                // correction hierarchies: (u_0, u_1) and, in 3D, (u_2, unused)
    long long N, nblocks;
    double dt;
    bool have_coeffs;
    char *arena;
    double *rho_dt, *wgt, *mu;         // rho / dt, dt / rho and mu per cell (owned copies)
    double *r0[3], *delta[3];          // initial residual and accumulated correction, per component
    double *inv_diag[3];               // 1 / diagonal of the component-diagonal operator, per component
    double nu;                         // Jacobi bound of the last set-up: max over rows of 2 off / diag
    bool jacobi;                       // corrections by point-Jacobi (no hierarchy set up)
    double *V, *Z;                     // Krylov basis (kKryM + 1 vectors of dim N) and one work vector
    double *kpart, *kdot_d, *kdot_h;   // dot partials, dots (device), dots (pinned host)
    double2 *lamA, *lamB, *rA, *rB;
    double *fA[2][3], *fB[3], *fzero[3];
    double *partial, *norm_d, *norm_h;
};

namespace {
mg_grid momentum_inner_grid(const mg_grid &g) {
    mg_grid gin = g;
    for (int a = 0; a < 3; a++)
        for (int sd = 0; sd < 2; sd++) {
            const int bc = g.bc[a][sd];
            gin.bc[a][sd] = a >= g.dim ? bc : bc == MG_BC_WALL ? MG_BC_DIRICHLET : bc == MG_BC_AXIS ? MG_BC_AXIS
                                                                                                 : MG_BC_WALL;
            gin.bc_T[a][sd] = gin.bc_p[a][sd] = 0.0;
        }
    return gin;
}

dim3 cell_grid(const mg_grid &g) {
    return dim3((unsigned)((g.n[0] + kBX - 1) / kBX), (unsigned)((g.n[1] + kBY - 1) / kBY),
                (unsigned)(g.dim == 3 ? g.n[2] : 1));
}

MomArgs momentum_args(const mg_momentum *m) {
    MomArgs A;
    std::memset(&A, 0, sizeof(A));
    const mg_grid &g = m->grid;
    for (int a = 0; a < 3; a++) {
        A.n[a] = g.n[a];
        for (int sd = 0; sd < 2; sd++) A.wall[a][sd] = a < g.dim && g.bc[a][sd] == MG_BC_WALL;
    }
    A.no_slip = (m->flags & MG_MOMENTUM_NO_SLIP) ? 1 : 0;
    A.r0 = g.r0;
    A.h = g.h;
    A.inv_h = 1.0 / g.h;
    A.half_inv_h = 0.5 / g.h;
    A.two_inv_h = 2.0 / g.h;
    A.inv_dt = 1.0 / m->dt;
    A.dt = m->dt;
    A.rho_dt = m->rho_dt;
    A.wgt = m->wgt;
    A.mu = m->mu;
    return A;
}

mg_status launch_momentum(const mg_momentum *m, const MomArgs &A, bool apply) {
    const dim3 gr = cell_grid(m->grid);
    cudaStream_t s = m->stream;
    if (apply) {
        if (m->grid.dim == 3) k_mom_residual<3, false, true, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
        else if (m->grid.axisym) k_mom_residual<2, true, true, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
        else k_mom_residual<2, false, true, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
    } else {
        if (m->grid.dim == 3) k_mom_residual<3, false, false, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
        else if (m->grid.axisym) k_mom_residual<2, true, false, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
        else k_mom_residual<2, false, false, kBX, kBY><<<gr, kBlock, 0, s>>>(A);
    }
    CK(cudaGetLastError());
    return MG_OK;
}

// r = R - A(u) into the correction right-hand sides (and into r_out, if given); returns ||dt r / rho||_2 (one
// host wait).
mg_status momentum_residual(mg_momentum *m, const double *const R[3], const double *const u[3], double *const r_out[3],
                            double *norm) {
    MomArgs A = momentum_args(m);
    for (int a = 0; a < m->grid.dim; a++) {
        A.u[a] = u[a];
        A.R[a] = R[a];
        A.r_out[a] = r_out ? r_out[a] : nullptr;
    }
    A.rA = m->rA;
    A.rB = m->rB;
    A.partial = m->partial;
    mg_status st = launch_momentum(m, A, false);
    if (st) return st;
    k_mom_norm<<<1, 1024, 0, m->stream>>>(m->partial, m->nblocks, m->norm_d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(m->norm_h, m->norm_d, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    *norm = std::sqrt(m->norm_h[0]);
    return MG_OK;
}

// ---- restarted GMRES on A delta = r0, right-preconditioned by the correction solve
// nd weighted dots <V_d, w> (d < nd, V_d at V + d * stride) read back to out; one host wait.
mg_status kry_dots(mg_momentum *m, const double *V, int nd, const double *w, double *out) {
    const long long N = m->N, stride = (long long)m->grid.dim * N;
    k_kry_dots<<<kKryBlocks, 256, 0, m->stream>>>(N, m->grid.dim, m->wgt, V, stride, nd, w, m->kpart);
    k_kry_reduce<<<1, 32 * nd, 0, m->stream>>>(m->kpart, kKryBlocks, nd, m->kdot_d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(m->kdot_h, m->kdot_d, nd * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    for (int d = 0; d < nd; d++) out[d] = m->kdot_h[d];
    return MG_OK;
}

int lin_grid(long long M) { return (int)std::min<long long>((M + 255) / 256, 152LL * 16); }

// z = M^-1 v (the fixed multigrid correction, a linear map), or z += M^-1 v with add.
mg_status kry_precond(mg_momentum *m, const double *v, double *const z[3], bool add) {
    const long long N = m->N;
    const int dim = m->grid.dim;
    mg_status st;
    if (dim == 3) {
        k_kry_pack<3><<<lin_grid(N), 256, 0, m->stream>>>(N, v, m->rA, m->rB);
        CK(cudaGetLastError());
        if ((st = correction_cycles<3>(m->hA, m->rA)) || (st = correction_cycles<3>(m->hB, m->rB))) return st;
        if (add) k_kry_unpack<3, true><<<lin_grid(N), 256, 0, m->stream>>>(N, m->hA->L[0].x, m->hB->L[0].x, z[0], z[1], z[2]);
        else k_kry_unpack<3, false><<<lin_grid(N), 256, 0, m->stream>>>(N, m->hA->L[0].x, m->hB->L[0].x, z[0], z[1], z[2]);
    } else {
        k_kry_pack<2><<<lin_grid(N), 256, 0, m->stream>>>(N, v, m->rA, nullptr);
        CK(cudaGetLastError());
        if ((st = correction_cycles<2>(m->hA, m->rA))) return st;
        if (add) k_kry_unpack<2, true><<<lin_grid(N), 256, 0, m->stream>>>(N, m->hA->L[0].x, nullptr, z[0], z[1], nullptr);
        else k_kry_unpack<2, false><<<lin_grid(N), 256, 0, m->stream>>>(N, m->hA->L[0].x, nullptr, z[0], z[1], nullptr);
    }
    CK(cudaGetLastError());
    return MG_OK;
}

// GMRES(kKryM) from delta (in m->delta) on A delta = r0 (in m->r0); r: the norm of r0 - A delta on entry and exit.
mg_status momentum_gmres(mg_momentum *m, double target, int max_iters, int *iters, int *precs, double *r) {
    const int dim = m->grid.dim;
    const long long N = m->N, M = (long long)dim * N;
    const double *r0c[3] = {m->r0[0], m->r0[1], m->r0[2]};
    const double *dc[3] = {m->delta[0], m->delta[1], m->delta[2]};
    auto vec = [&](int d) { return m->V + d * M; };
    auto comps = [&](double *v, double *out[3]) {
        for (int q = 0; q < 3; q++) out[q] = q < dim ? v + q * N : nullptr;
    };
    mg_status st;
    for (;;) {
        double *v0[3];
        comps(vec(0), v0);
        if ((st = momentum_residual(m, r0c, dc, v0, r))) return st;
        if (!std::isfinite(*r)) return fail(MG_ERR_INVALID_COEFF, "non-finite momentum residual");
        if (*r <= target || *iters >= max_iters) return MG_OK;
        KryCoef none;
        std::memset(&none, 0, sizeof(none));
        k_kry_orth<<<lin_grid(M), 256, 0, m->stream>>>(M, nullptr, 0, 0, none, 1.0 / *r, vec(0));
        CK(cudaGetLastError());
        double H[kKryM + 1][kKryM], g[kKryM + 1], cs[kKryM], sn[kKryM];
        std::memset(H, 0, sizeof(H));
        std::memset(g, 0, sizeof(g));
        g[0] = *r;
        int kk = 0;
        for (int j = 0; j < kKryM; j++) {
            double *z[3], *w[3];
            comps(m->Z, z);
            comps(vec(j + 1), w);
            if ((st = kry_precond(m, vec(j), z, false))) return st;
            *precs += 1;
            MomArgs A = momentum_args(m);
            for (int q = 0; q < dim; q++) {
                A.u[q] = z[q];
                A.y[q] = w[q];
            }
            if ((st = launch_momentum(m, A, true))) return st;
            KryCoef h, h2;
            std::memset(&h, 0, sizeof(h));
            std::memset(&h2, 0, sizeof(h2));
            if ((st = kry_dots(m, m->V, j + 1, vec(j + 1), h.c))) return st;
            k_kry_orth<<<lin_grid(M), 256, 0, m->stream>>>(M, m->V, M, j + 1, h, 1.0, vec(j + 1));
            CK(cudaGetLastError());
            if ((st = kry_dots(m, m->V, j + 1, vec(j + 1), h2.c))) return st;      // second pass (CGS2)
            k_kry_orth<<<lin_grid(M), 256, 0, m->stream>>>(M, m->V, M, j + 1, h2, 1.0, vec(j + 1));
            CK(cudaGetLastError());
            double nn;
            if ((st = kry_dots(m, vec(j + 1), 1, vec(j + 1), &nn))) return st;
            const double hn = std::sqrt(std::max(nn, 0.0));
            for (int i = 0; i <= j; i++) H[i][j] = h.c[i] + h2.c[i];
            H[j + 1][j] = hn;
            for (int i = 0; i < j; i++) {                     // earlier rotations
                const double a = H[i][j], b = H[i + 1][j];
                H[i][j] = cs[i] * a + sn[i] * b;
                H[i + 1][j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[j][j], b = H[j + 1][j], den = std::hypot(a, b);
            cs[j] = den > 0.0 ? a / den : 1.0;
            sn[j] = den > 0.0 ? b / den : 0.0;
            H[j][j] = den;
            H[j + 1][j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            kk = j + 1;
            *iters += 1;
            if (hn > 0.0) {
                k_kry_orth<<<lin_grid(M), 256, 0, m->stream>>>(M, nullptr, 0, 0, none, 1.0 / hn, vec(j + 1));
                CK(cudaGetLastError());
            }
            if (std::fabs(g[j + 1]) <= target || *iters >= max_iters || !(hn > 0.0)) break;
        }
        KryCoef y;
        std::memset(&y, 0, sizeof(y));
        for (int i = kk - 1; i >= 0; i--) {                   // H y = g, upper triangular
            double s = g[i];
            for (int l = i + 1; l < kk; l++) s -= H[i][l] * y.c[l];
            y.c[i] = H[i][i] != 0.0 ? s / H[i][i] : 0.0;
        }
        k_kry_combine<<<lin_grid(M), 256, 0, m->stream>>>(M, m->V, M, kk, y, m->Z);
        CK(cudaGetLastError());
        double *d[3] = {m->delta[0], m->delta[1], m->delta[2]};
        if ((st = kry_precond(m, m->Z, d, true))) return st;    // delta += M^-1 (V y)
        *precs += 1;
    }
}

bool momentum_ptrs(const mg_momentum *m, const double *const v[3]) {
    if (!v) return false;
    for (int a = 0; a < m->grid.dim; a++)
        if (!device_ptr(v[a])) return false;
    return true;
}
}  // namespace

mg_status mg_momentum_destroy(mg_momentum *m) {
    if (!m) return MG_OK;
    DeviceGuard dg(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    mg_destroy(m->hA);
    mg_destroy(m->hB);
    if (m->arena) cudaFree(m->arena);
    if (m->norm_h) cudaFreeHost(m->norm_h);
    if (m->kdot_h) cudaFreeHost(m->kdot_h);
    delete m;
    return MG_OK;
}

mg_status mg_momentum_create(const mg_grid *grid, int flags, const mg_options *inner, void *stream,
                             mg_momentum **out) {
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (flags & ~(MG_MOMENTUM_NO_SLIP | MG_MOMENTUM_MULTIGRID | MG_MOMENTUM_KRYLOV))
        return fail(MG_ERR_INVALID_ARG, "unknown momentum flags");
    mg_options opt;
    if (inner) {
        opt = *inner;
    } else {
        mg_default_options(&opt);
        opt.max_cycles = 1;
    }
    if (opt.max_cycles < 1) return fail(MG_ERR_INVALID_ARG, "inner max_cycles must be >= 1");
    if (opt.precision != MG_FP64) return fail(MG_ERR_INVALID_ARG, "the correction solves run in FP64 (MG_FP64)");
    opt.rtol = 0.0;
    const mg_grid gin = momentum_inner_grid(*grid);
    mg_momentum *m = new (std::nothrow) mg_momentum;
    if (!m) return fail(MG_ERR_OOM, "host allocation failed");
    std::memset(m, 0, sizeof(*m));
    m->grid = *grid;
    m->flags = flags;
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&m->device);
    const int dim = grid->dim;
    if ((st = mg_create(&gin, &opt, nullptr, 0, stream, &m->hA)) ||
        (dim == 3 && (st = mg_create(&gin, &opt, nullptr, 0, stream, &m->hB)))) {
        const std::string msg = g_err;
        mg_momentum_destroy(m);
        return fail(st, msg);
    }
    m->N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    const dim3 gr = cell_grid(*grid);
    m->nblocks = (long long)gr.x * gr.y * gr.z;
    long long nf[3] = {0, 0, 0};
    for (int a = 0; a < dim; a++)
        nf[a] = (long long)(grid->n[0] + (a == 0)) * (grid->n[1] + (a == 1)) * (grid->n[2] + (a == 2));
    // one arena: offsets rounded to 256 bytes
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t N = (size_t)m->N;
    const size_t o_rho = take(N * 8), o_wgt = take(N * 8), o_mu = take(N * 8), o_lamA = take(N * 32),
                 o_rA = take(N * 16);
    size_t o_r0[3] = {}, o_d[3] = {}, o_id[3] = {};
    for (int a = 0; a < dim; a++) {
        o_r0[a] = take(N * 8);
        o_d[a] = take(N * 8);
        o_id[a] = take(N * 8);
    }
    const size_t o_lamB = dim == 3 ? take(N * 32) : 0, o_rB = dim == 3 ? take(N * 16) : 0;
    size_t o_f[4][3] = {};
    for (int q = 0; q < (dim == 3 ? 4 : 2); q++)
        for (int a = 0; a < dim; a++) o_f[q][a] = take((size_t)nf[a] * 8);
    const size_t o_part = take((size_t)m->nblocks * 8), o_norm = take(8);
    const bool kry = (flags & MG_MOMENTUM_KRYLOV) != 0;
    const size_t o_V = kry ? take((size_t)(kKryM + 1) * dim * N * 8) : 0, o_Z = kry ? take((size_t)dim * N * 8) : 0,
                 o_kp = kry ? take((size_t)(kKryM + 1) * kKryBlocks * 8) : 0, o_kd = kry ? take((kKryM + 1) * 8) : 0;
    DeviceGuard dg(m->device);
    if (cudaMalloc(&m->arena, off) != cudaSuccess || cudaMallocHost(&m->norm_h, sizeof(double)) != cudaSuccess ||
        (kry && cudaMallocHost(&m->kdot_h, (kKryM + 1) * sizeof(double)) != cudaSuccess)) {
        cudaGetLastError();
        mg_momentum_destroy(m);
        return fail(MG_ERR_OOM, "device allocation failed");
    }
    auto at = [&](size_t o) { return m->arena + o; };
    m->rho_dt = reinterpret_cast<double *>(at(o_rho));
    m->wgt = reinterpret_cast<double *>(at(o_wgt));
    m->mu = reinterpret_cast<double *>(at(o_mu));
    m->lamA = reinterpret_cast<double2 *>(at(o_lamA));
    m->rA = reinterpret_cast<double2 *>(at(o_rA));
    for (int a = 0; a < dim; a++) {
        m->r0[a] = reinterpret_cast<double *>(at(o_r0[a]));
        m->delta[a] = reinterpret_cast<double *>(at(o_d[a]));
        m->inv_diag[a] = reinterpret_cast<double *>(at(o_id[a]));
    }
    if (dim == 3) {
        m->lamB = reinterpret_cast<double2 *>(at(o_lamB));
        m->rB = reinterpret_cast<double2 *>(at(o_rB));
    }
    for (int a = 0; a < dim; a++) {
        m->fA[0][a] = reinterpret_cast<double *>(at(o_f[0][a]));
        m->fA[1][a] = reinterpret_cast<double *>(at(o_f[1][a]));
        if (dim == 3) {
            m->fB[a] = reinterpret_cast<double *>(at(o_f[2][a]));
            m->fzero[a] = reinterpret_cast<double *>(at(o_f[3][a]));
            CK(cudaMemsetAsync(m->fzero[a], 0, (size_t)nf[a] * 8, m->stream));
        }
    }
    m->partial = reinterpret_cast<double *>(at(o_part));
    m->norm_d = reinterpret_cast<double *>(at(o_norm));
    if (kry) {
        m->V = reinterpret_cast<double *>(at(o_V));
        m->Z = reinterpret_cast<double *>(at(o_Z));
        m->kpart = reinterpret_cast<double *>(at(o_kp));
        m->kdot_d = reinterpret_cast<double *>(at(o_kd));
    }
    CK(cudaStreamSynchronize(m->stream));
    *out = m;
    return MG_OK;
}

mg_status mg_momentum_set_coeffs(mg_momentum *m, double dt, const double *rho, const double *mu) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "momentum handle is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite");
    DeviceGuard dg(m->device);
    if (!device_ptr(rho) || !device_ptr(mu))
        return fail(MG_ERR_INVALID_ARG, "rho and mu must be device pointers of the handle's device");
    m->have_coeffs = false;
    const mg_grid &g = m->grid;
    const int dim = g.dim;
    MomCoeffArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < 3; a++) {
        A.n[a] = g.n[a];
        for (int sd = 0; sd < 2; sd++) A.wall[a][sd] = a < dim && g.bc[a][sd] == MG_BC_WALL;
    }
    A.no_slip = (m->flags & MG_MOMENTUM_NO_SLIP) ? 1 : 0;
    A.r0 = g.r0;
    A.h = g.h;
    A.dt = dt;
    A.inv_dt = 1.0 / dt;
    A.inv_h2 = 1.0 / (g.h * g.h);
    A.rho = rho;
    A.mu = mu;
    A.partial = m->partial;        // one Jacobi bound per block
    for (int a = 0; a < dim; a++) A.inv_diag[a] = m->inv_diag[a];
    A.rho_dt = m->rho_dt;
    A.wgt = m->wgt;
    A.mu_o = m->mu;
    A.lamA = m->lamA;
    A.lamB = m->lamB;
    for (int a = 0; a < dim; a++) {
        A.fA[0][a] = m->fA[0][a];
        A.fA[1][a] = m->fA[1][a];
        A.fB[a] = m->fB[a];
    }
    const dim3 gr = cell_grid(g);
    if (dim == 3) k_mom_diag<3, false><<<gr, kBlock, 0, m->stream>>>(A);
    else if (g.axisym) k_mom_diag<2, true><<<gr, kBlock, 0, m->stream>>>(A);
    else k_mom_diag<2, false><<<gr, kBlock, 0, m->stream>>>(A);
    CK(cudaGetLastError());
    k_mom_max<<<1, 1024, 0, m->stream>>>(m->partial, m->nblocks, m->norm_d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(m->norm_h, m->norm_d, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    const double nu = m->norm_h[0];
    if (!std::isfinite(nu)) return fail(MG_ERR_INVALID_COEFF, "non-finite momentum coefficients");
    m->nu = nu;
    // Point-Jacobi corrections contract the residual by at least nu per step; below kJacobiNu they beat a V-cycle
    // and need no hierarchy.
    constexpr double kJacobiNu = 0.01;
    m->jacobi = !(m->flags & MG_MOMENTUM_MULTIGRID) && nu <= kJacobiNu;
    if (!m->jacobi) {
        if (dim == 3) k_mom_hier<3, false><<<gr, kBlock, 0, m->stream>>>(A);
        else if (g.axisym) k_mom_hier<2, true><<<gr, kBlock, 0, m->stream>>>(A);
        else k_mom_hier<2, false><<<gr, kBlock, 0, m->stream>>>(A);
        CK(cudaGetLastError());
        const double *faA[3] = {m->fA[1][0], m->fA[1][1], m->fA[1][2]};
        const double *fkA[3] = {m->fA[0][0], m->fA[0][1], m->fA[0][2]};
        mg_status st = mg_set_coeffs(m->hA, reinterpret_cast<const double *>(m->lamA), faA, fkA, 1);
        if (st) return st;
        if (dim == 3) {
            const double *faB[3] = {m->fzero[0], m->fzero[1], m->fzero[2]};
            const double *fkB[3] = {m->fB[0], m->fB[1], m->fB[2]};
            if ((st = mg_set_coeffs(m->hB, reinterpret_cast<const double *>(m->lamB), faB, fkB, 1))) return st;
        }
    }
    m->dt = dt;
    m->have_coeffs = true;
    return MG_OK;
}

mg_status mg_momentum_apply(mg_momentum *m, const double *const u[3], double *const y[3]) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "momentum handle is NULL");
    if (!m->have_coeffs) return fail(MG_ERR_STATE, "mg_momentum_set_coeffs has not succeeded on this handle");
    DeviceGuard dg(m->device);
    if (!momentum_ptrs(m, u) || !momentum_ptrs(m, y))
        return fail(MG_ERR_INVALID_ARG, "u and y must be device pointers of the handle's device");
    for (int a = 0; a < m->grid.dim; a++)
        for (int b = 0; b < m->grid.dim; b++)
            if (y[a] == u[b]) return fail(MG_ERR_INVALID_ARG, "y must not alias u");
    MomArgs A = momentum_args(m);
    for (int a = 0; a < m->grid.dim; a++) {
        A.u[a] = u[a];
        A.y[a] = y[a];
    }
    mg_status st = launch_momentum(m, A, true);
    if (st) return st;
    CK(cudaStreamSynchronize(m->stream));
    return MG_OK;
}

mg_status mg_momentum_solve(mg_momentum *m, const double *const R[3], double *const u[3], double rtol, int max_iters,
                            mg_momentum_stats *stats) {
    if (!m) return fail(MG_ERR_INVALID_ARG, "momentum handle is NULL");
    if (!m->have_coeffs) return fail(MG_ERR_STATE, "mg_momentum_set_coeffs has not succeeded on this handle");
    if (!std::isfinite(rtol) || max_iters < 0) return fail(MG_ERR_INVALID_ARG, "rtol must be finite, max_iters >= 0");
    DeviceGuard dg(m->device);
    if (!momentum_ptrs(m, R) || !momentum_ptrs(m, u))
        return fail(MG_ERR_INVALID_ARG, "R and u must be device pointers of the handle's device");
    const int dim = m->grid.dim;
    for (int a = 0; a < dim; a++)
        for (int b = 0; b < dim; b++)
            if (R[a] == u[b]) return fail(MG_ERR_INVALID_ARG, "R must not alias u");
    const auto t0 = std::chrono::steady_clock::now();
    // Correction form: r0 = R - A(u0) once, then r = r0 - A(delta) and u = u0 + delta at the end.  Forming
    // R - A(u) at every step would stall at the rounding of R (rho u / dt), far above the residual when dt is
    // small and u0 is close to the solution.
    const double *uc[3] = {u[0], dim > 1 ? u[1] : nullptr, dim > 2 ? u[2] : nullptr};
    const double *r0c[3] = {m->r0[0], m->r0[1], m->r0[2]};
    const double *dc[3] = {m->delta[0], m->delta[1], m->delta[2]};
    double r0 = 0.0, r = 0.0;
    CK(cudaMemsetAsync(m->hA->err_d + 1, 0, sizeof(int), m->stream));
    if (dim == 3) CK(cudaMemsetAsync(m->hB->err_d + 1, 0, sizeof(int), m->stream));
    mg_status st = momentum_residual(m, R, uc, m->r0, &r0);
    if (st) return st;
    for (int a = 0; a < dim; a++) CK(cudaMemsetAsync(m->delta[a], 0, (size_t)m->N * 8, m->stream));
    if (!std::isfinite(r0)) return fail(MG_ERR_INVALID_COEFF, "non-finite momentum residual");
    r = r0;
    int it = 0, cycles = 0;
    mg_status result = MG_OK;
    if (m->V && !m->jacobi && !(r == 0.0 || (rtol > 0.0 && r <= rtol * r0))) {
        int precs = 0;
        const double target = rtol > 0.0 ? rtol * r0 : 0.0;
        if ((st = momentum_gmres(m, target, max_iters, &it, &precs, &r))) return st;
        cycles = precs * m->hA->opt.max_cycles * (dim == 3 ? 2 : 1);
        if (!(r == 0.0 || (rtol > 0.0 && r <= rtol * r0))) result = rtol > 0.0 ? MG_ERR_NOT_CONVERGED : MG_OK;
    }
    for (; !m->V || m->jacobi;) {
        if (r == 0.0 || (rtol > 0.0 && r <= rtol * r0)) break;
        if (it >= max_iters) {
            result = rtol > 0.0 ? MG_ERR_NOT_CONVERGED : MG_OK;
            break;
        }
        const int blocks = (int)std::min<long long>((m->N + 255) / 256, 152LL * 16);
        double *const *d = m->delta;
        double *const *id = m->inv_diag;
        if (m->jacobi) {
            if (dim == 3)
                k_mom_jacobi<3><<<blocks, 256, 0, m->stream>>>(m->N, m->rA, m->rB, id[0], id[1], id[2], d[0], d[1],
                                                               d[2]);
            else
                k_mom_jacobi<2><<<blocks, 256, 0, m->stream>>>(m->N, m->rA, nullptr, id[0], id[1], nullptr, d[0],
                                                               d[1], nullptr);
        } else {
            if (dim == 3) {
                if ((st = correction_cycles<3>(m->hA, m->rA)) || (st = correction_cycles<3>(m->hB, m->rB))) return st;
                cycles += 2 * m->hA->opt.max_cycles;
            } else {
                if ((st = correction_cycles<2>(m->hA, m->rA))) return st;
                cycles += m->hA->opt.max_cycles;
            }
            const double2 *xa = m->hA->L[0].x, *xb = dim == 3 ? m->hB->L[0].x : nullptr;
            if (dim == 3) k_mom_update<3><<<blocks, 256, 0, m->stream>>>(m->N, xa, xb, d[0], d[1], d[2]);
            else k_mom_update<2><<<blocks, 256, 0, m->stream>>>(m->N, xa, xb, d[0], d[1], nullptr);
        }
        CK(cudaGetLastError());
        if ((st = momentum_residual(m, r0c, dc, nullptr, &r))) return st;
        it++;
        if (!std::isfinite(r)) return fail(MG_ERR_INVALID_COEFF, "non-finite momentum residual");
    }
    if (it > 0) {
        const int blocks = (int)std::min<long long>((m->N + 255) / 256, 152LL * 16);
        double *const *d = m->delta;
        if (dim == 3) k_mom_add<3><<<blocks, 256, 0, m->stream>>>(m->N, d[0], d[1], d[2], u[0], u[1], u[2]);
        else k_mom_add<2><<<blocks, 256, 0, m->stream>>>(m->N, d[0], d[1], nullptr, u[0], u[1], nullptr);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(m->stream));
        if (!m->jacobi && ((st = handle_errors(m->hA)) || (dim == 3 && (st = handle_errors(m->hB))))) return st;
    }
    if (stats) {
        stats->iterations = it;
        stats->cycles = cycles;
        stats->r0 = r0;
        stats->rfinal = r;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->status = result;
        stats->jacobi = m->jacobi ? 1 : 0;
        stats->nu = m->nu;
    }
    if (result) return fail(result, "momentum solve did not reach rtol in max_iters steps");
    return MG_OK;
}

namespace {
MomSideArgs side_args(const mg_grid *grid, double dt) {
    MomSideArgs A;
    std::memset(&A, 0, sizeof(A));
    for (int a = 0; a < 3; a++) {
        A.n[a] = grid->n[a];
        for (int sd = 0; sd < 2; sd++) {
            A.dir[a][sd] = a < grid->dim && grid->bc[a][sd] == MG_BC_DIRICHLET;
            A.gp[a][sd] = a < grid->dim ? grid->bc_p[a][sd] : 0.0;
        }
    }
    A.inv_h = 1.0 / grid->h;
    A.two_inv_h = 2.0 / grid->h;
    A.half_inv_h = 0.5 / grid->h;
    A.dt = dt;
    A.inv_dt = 1.0 / dt;
    return A;
}
}  // namespace

mg_status mg_momentum_rhs_async(const mg_grid *grid, double dt, double sigma, const double *const mom[3],
                                const double *p, const double *kappa, const double *C, double *const R[3],
                                void *stream) {
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (!mom || !R) return fail(MG_ERR_INVALID_ARG, "mom and R must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(sigma))
        return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite, sigma finite");
    const int dim = grid->dim;
    bool ok = device_ptr(p) && device_ptr(kappa) && device_ptr(C);
    for (int a = 0; a < dim; a++) ok = ok && device_ptr(mom[a]) && device_ptr(R[a]);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "every array must be a device pointer of the current device");
    for (int a = 0; a < dim; a++)
        if (R[a] == p || R[a] == C || R[a] == kappa) return fail(MG_ERR_INVALID_ARG, "R must not alias p, C or kappa");
    MomSideArgs A = side_args(grid, dt);
    A.sigma = sigma;
    A.p = p;
    A.C = C;
    A.kappa = kappa;
    for (int a = 0; a < dim; a++) {
        A.mom[a] = mom[a];
        A.R[a] = R[a];
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dim == 3) k_mom_rhs<3><<<cell_grid(*grid), kBlock, 0, cs>>>(A);
    else k_mom_rhs<2><<<cell_grid(*grid), kBlock, 0, cs>>>(A);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status mg_provisional_async(const mg_grid *grid, double dt, const double *rho, const double *p,
                               const double *const u_pred[3], double *const uf_out[3], void *stream) {
    mg_status st = check_grid_geom(grid);
    if (st) return st;
    if (!u_pred || !uf_out) return fail(MG_ERR_INVALID_ARG, "u_pred and uf_out must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(MG_ERR_INVALID_ARG, "dt must be positive and finite");
    const int dim = grid->dim;
    bool ok = device_ptr(rho) && device_ptr(p);
    for (int a = 0; a < dim; a++) ok = ok && device_ptr(u_pred[a]) && device_ptr(uf_out[a]);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "every array must be a device pointer of the current device");
    for (int a = 0; a < dim; a++) {
        if (uf_out[a] == rho || uf_out[a] == p) return fail(MG_ERR_INVALID_ARG, "uf_out must not alias an input");
        for (int b = 0; b < dim; b++)
            if (uf_out[a] == u_pred[b]) return fail(MG_ERR_INVALID_ARG, "uf_out must not alias an input");
    }
    MomSideArgs A = side_args(grid, dt);
    A.p = p;
    A.rho = rho;
    for (int a = 0; a < dim; a++) {
        A.u[a] = u_pred[a];
        A.uf[a] = uf_out[a];
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (dim == 3) k_provisional<3><<<cell_grid(*grid), kBlock, 0, cs>>>(A);
    else k_provisional<2><<<cell_grid(*grid), kBlock, 0, cs>>>(A);
    CK(cudaGetLastError());
    return MG_OK;
}

