/*
 * Plain FP64 CPU oracle for the coupled pressure-temperature solve on an
 * adaptive (refined-patch) grid: the paper's production grids are coarsened
 * away from the bubble (Sec. 5.2, the rigid-wall collapse runs), i.e. finer
 * cells near the interface and coarser ones elsewhere.
 *
 * TEST INFRASTRUCTURE ONLY, like coupled_oracle.c (whose functions it reuses
 * by including that file): nothing in the product path links, loads or calls
 * it.  Build: gcc -O2 -ffp-contract=off, one thread.
 *
 * The composite grid (2D Cartesian)
 * ---------------------------------
 * A uniform base grid of spacing H covers the domain.  One box of base cells,
 * [box[0][0], box[0][1]) x [box[1][0], box[1][1]), is refined 2:1 into a patch
 * of fine cells of spacing h = H / 2.  The unknowns are the fine cells and the
 * base cells outside the box ("valid" cells); base cells under the box are
 * covered.
 *
 * The operator is Eqs. 27-28 on every valid cell, with the finite-volume
 * divergence of each cell built from its faces:
 *   - between two fine or two valid base cells: the uniform-grid flux;
 *   - on the domain boundary: wall (no flux) or Dirichlet (value h/2 away);
 *   - at the coarse-fine interface (a patch side inside the domain), seen from
 *     a fine cell: the flux towards the adjacent base cell C is
 *       c_f (u~ - u_f) / (1.5 h),
 *     u~ = u_C + s (u_{C+t} - u_{C-t}) / 8: the coarse field at the fine cell's
 *     tangential position (a quarter of C's width above or below its centre,
 *     s = +1 / -1), taken from C's tangential neighbours (outside the domain:
 *     the wall or Dirichlet ghost of the base grid).  1.5 h is the distance
 *     from the fine centre to the coarse centre, so the flux is the two-point
 *     difference between those values, exact for fields linear in both
 *     directions;
 *   - at the interface seen from the base cell C: the sum of the fluxes of the
 *     fine faces that make up C's face (each counted once, with opposite
 *     sign), so the composite operator is conservative: the fluxes through
 *     the interface cancel in any sum of cell integrals.
 *
 * Solver: the paper's defect-correction loop with a fast adaptive composite
 * (FAC) cycle as the correction solve: red-black block Gauss-Seidel sweeps on
 * the patch (interface ghosts from the base correction, zero before it), the
 * patch residual restricted onto the covered base cells and the valid base
 * cells' residual corrected for the patch's interface fluxes, one V-cycle of
 * the uniform base-grid multigrid (base coefficients outside the patch, the
 * patch's coarsened under it), the base correction prolonged onto the patch
 * (cell-centred bilinear), and post sweeps on the patch.
 *
 * Parity unpinned: none (tests/test_oracle_composite.py pins every function).
 */
#include "coupled_oracle.c"

typedef struct {
    orc_grid base;    /* dim 2, axisym 0 */
    int box[2][2];    /* per axis: first and one-past-last refined base cell */
} orc_cgrid;

/* The patch as a uniform grid of spacing h: the domain's boundary conditions
 * on the sides where the box reaches the domain boundary; the interface sides
 * are marked in iface[axis][side]. */
static orc_grid patch_grid(const orc_cgrid *cg, int iface[2][2])
{
    orc_grid f = cg->base;
    f.h = 0.5 * cg->base.h;
    for (int a = 0; a < 2; a++) {
        f.n[a] = 2 * (cg->box[a][1] - cg->box[a][0]);
        iface[a][0] = cg->box[a][0] > 0;
        iface[a][1] = cg->box[a][1] < cg->base.n[a];
        for (int s = 0; s < 2; s++)
            if (iface[a][s]) { f.bc[a][s] = BC_WALL; f.bcT[a][s] = 0.0; f.bcp[a][s] = 0.0; }
    }
    f.n[2] = 1;
    return f;
}

static int covered(const orc_cgrid *cg, int I, int J)
{
    return I >= cg->box[0][0] && I < cg->box[0][1] && J >= cg->box[1][0] && J < cg->box[1][1];
}

/* Value of field `fld` (0 = T, 1 = p) of base cell (I, J), or across the
 * domain boundary its ghost: mirror at a wall, 2 g - u at a Dirichlet side
 * (g = 0 when homogeneous).  (I, J) may be one cell outside along either axis
 * or both (a corner: the rule of each side in turn, x first). */
static double base_value(const orc_grid *g, const double *xb, int I, int J, int fld, int homogeneous)
{
    int c[3] = {I, J, 0}, out[2] = {-1, -1};
    if (I < 0) { c[0] = 0; out[0] = 0; }
    if (I >= g->n[0]) { c[0] = g->n[0] - 1; out[0] = 1; }
    if (J < 0) { c[1] = 0; out[1] = 0; }
    if (J >= g->n[1]) { c[1] = g->n[1] - 1; out[1] = 1; }
    double u = xb[2 * cell_id(g, c) + fld];
    for (int ax = 0; ax < 2; ax++) {
        int side = out[ax];
        if (side < 0 || g->bc[ax][side] != BC_DIRICHLET) continue;
        double gv = homogeneous ? 0.0 : (fld == 0 ? g->bcT[ax][side] : g->bcp[ax][side]);
        u = 2.0 * gv - u;
    }
    return u;
}

/* u~ of the fine cell (fi, fj) of the patch across its interface side (a, s):
 * the coarse field at the fine cell's tangential position. */
static double ghost_value(const orc_cgrid *cg, const double *xb, int a, int s, int fi, int fj, int fld,
                          int homogeneous)
{
    const orc_grid *g = &cg->base;
    int t = 1 - a;
    int f[2] = {fi, fj};
    int C[2];
    C[a] = s == 0 ? cg->box[a][0] - 1 : cg->box[a][1];
    C[t] = cg->box[t][0] + f[t] / 2;
    double sgn = (f[t] & 1) ? 1.0 : -1.0;
    int Cp[2] = {C[0], C[1]}, Cm[2] = {C[0], C[1]};
    Cp[t] += 1;
    Cm[t] -= 1;
    double uc = base_value(g, xb, C[0], C[1], fld, homogeneous);
    double up = base_value(g, xb, Cp[0], Cp[1], fld, homogeneous);
    double um = base_value(g, xb, Cm[0], Cm[1], fld, homogeneous);
    return uc + sgn * (up - um) / 8.0;
}

/* div(c grad u) of fine cell (fi, fj) in the composite operator.  xf: patch
 * unknowns (stride 2, field fld), xb: base unknowns. */
static double fine_div(const orc_cgrid *cg, const orc_grid *fg, int iface[2][2], double *const coef[3],
                       const double *xf, const double *xb, int fi, int fj, int fld, int homogeneous)
{
    int c[3] = {fi, fj, 0};
    long i = cell_id(fg, c);
    double h = fg->h, sum = 0.0;
    double u = xf[2 * i + fld];
    for (int a = 0; a < 2; a++)
        for (int s = 0; s < 2; s++) {
            int f[3] = {fi, fj, 0};
            f[a] += s;
            int nb[3] = {fi, fj, 0};
            nb[a] += s ? 1 : -1;
            double cf = coef[a][face_id(fg, a, f)];
            if (nb[a] >= 0 && nb[a] < fg->n[a]) {
                sum += cf * (xf[2 * cell_id(fg, nb) + fld] - u) / (h * h);
            } else if (iface[a][s]) {
                double gu = ghost_value(cg, xb, a, s, fi, fj, fld, homogeneous);
                sum += cf * (gu - u) / (1.5 * h * h);
            } else if (fg->bc[a][s] == BC_DIRICHLET) {
                double gv = homogeneous ? 0.0 : (fld == 0 ? fg->bcT[a][s] : fg->bcp[a][s]);
                sum += cf * (gv - u) / (0.5 * h * h);
            }
        }
    return sum;
}

/* div(c grad u) of valid base cell (I, J): uniform-grid fluxes, except the
 * faces it shares with the patch, whose flux is the sum of the fine faces'. */
static double base_div(const orc_cgrid *cg, const orc_grid *fg, int iface[2][2], double *const bcoef[3],
                       double *const fcoef[3], const double *xf, const double *xb, int I, int J, int fld,
                       int homogeneous)
{
    const orc_grid *g = &cg->base;
    int c[3] = {I, J, 0};
    double H = g->h, sum = 0.0;
    double u = xb[2 * cell_id(g, c) + fld];
    for (int a = 0; a < 2; a++)
        for (int s = 0; s < 2; s++) {
            int f[3] = {I, J, 0};
            f[a] += s;
            int nb[3] = {I, J, 0};
            nb[a] += s ? 1 : -1;
            if (nb[a] >= 0 && nb[a] < g->n[a] && covered(cg, nb[0], nb[1])) {
                /* interface: the two fine faces of this face, fluxes from the fine side */
                int t = 1 - a;
                int side = s ? 0 : 1;               /* the patch side this face belongs to */
                int fi_n = side == 0 ? 0 : fg->n[a] - 1;   /* the fine cells along it */
                for (int q = 0; q < 2; q++) {
                    int ff[2];
                    ff[a] = fi_n;
                    ff[t] = 2 * (c[t] - cg->box[t][0]) + q;
                    int fc[3] = {ff[0], ff[1], 0};
                    int fface[3] = {ff[0], ff[1], 0};
                    fface[a] += side;               /* the fine cell's face on the interface */
                    double cf = fcoef[a][face_id(fg, a, fface)];
                    double uf = xf[2 * cell_id(fg, fc) + fld];
                    double gu = ghost_value(cg, xb, a, side, ff[0], ff[1], fld, homogeneous);
                    /* flux into the fine cell is h cf (gu - uf) / (1.5 h); into C the opposite,
                       over C's volume H^2 */
                    sum += (0.5 * H) * cf * (uf - gu) / (1.5 * 0.5 * H) / (H * H);
                }
                (void)iface;
            } else if (nb[a] >= 0 && nb[a] < g->n[a]) {
                double cf = bcoef[a][face_id(g, a, f)];
                sum += cf * (xb[2 * cell_id(g, nb) + fld] - u) / (H * H);
            } else if (g->bc[a][s] == BC_DIRICHLET) {
                double cf = bcoef[a][face_id(g, a, f)];
                double gv = homogeneous ? 0.0 : (fld == 0 ? g->bcT[a][s] : g->bcp[a][s]);
                sum += cf * (gv - u) / (0.5 * H * H);
            }
        }
    return sum;
}

/* y = L(x) of Eqs. 27-28 on the composite grid.  Base arrays have the base
 * grid's cells (covered cells: y = 0, x ignored); patch arrays the patch's.
 * homogeneous != 0: zero Dirichlet values. */
void orc_cf_apply(const orc_cgrid *cg, const double *lamb, double *const fab[3], double *const fkb[3],
                  const double *lamf, double *const faf[3], double *const fkf[3], const double *xb,
                  const double *xf, double *yb, double *yf, int homogeneous)
{
    int iface[2][2];
    orc_grid fg = patch_grid(cg, iface);
    const orc_grid *g = &cg->base;
    for (long i = 0; i < ncells(g); i++) {
        int c[3];
        cell_of(g, i, c);
        if (covered(cg, c[0], c[1])) { yb[2 * i] = yb[2 * i + 1] = 0.0; continue; }
        double lapT = base_div(cg, &fg, iface, fkb, fkf, xf, xb, c[0], c[1], 0, homogeneous);
        double lapp = base_div(cg, &fg, iface, fab, faf, xf, xb, c[0], c[1], 1, homogeneous);
        const double *l = lamb + 4 * i;
        yb[2 * i] = lapT + l[0] * xb[2 * i] + l[1] * xb[2 * i + 1];
        yb[2 * i + 1] = lapp + l[2] * xb[2 * i + 1] + l[3] * lapT;
    }
    for (long i = 0; i < ncells(&fg); i++) {
        int c[3];
        cell_of(&fg, i, c);
        double lapT = fine_div(cg, &fg, iface, fkf, xf, xb, c[0], c[1], 0, homogeneous);
        double lapp = fine_div(cg, &fg, iface, faf, xf, xb, c[0], c[1], 1, homogeneous);
        const double *l = lamf + 4 * i;
        yf[2 * i] = lapT + l[0] * xf[2 * i] + l[1] * xf[2 * i + 1];
        yf[2 * i + 1] = lapp + l[2] * xf[2 * i + 1] + l[3] * lapT;
    }
}

/* The patch as a multigrid level for its sweeps: the interface sides become
 * Dirichlet sides with zero value whose face coefficients are a third of the
 * fine ones, so that their flux c (0 - u) / (0.5 h) / 3 is the interface flux
 * c (u~ - u) / (1.5 h) with u~ = 0; a nonzero u~ enters the right-hand side. */
static int patch_level(const orc_cgrid *cg, const double *lamf, double *const faf[3], double *const fkf[3],
                       level *P, int iface[2][2])
{
    orc_grid fg = patch_grid(cg, iface);
    for (int a = 0; a < 2; a++)
        for (int s = 0; s < 2; s++)
            if (iface[a][s]) fg.bc[a][s] = BC_DIRICHLET;
    memset(fg.bcT, 0, sizeof(fg.bcT));
    memset(fg.bcp, 0, sizeof(fg.bcp));
    if (alloc_level(P, &fg)) return -2;
    memcpy(P->lam, lamf, sizeof(double) * 4 * P->N);
    for (int a = 0; a < 2; a++) {
        long m = nfaces(&fg, a);
        memcpy(P->fa[a], faf[a], sizeof(double) * m);
        memcpy(P->fk[a], fkf[a], sizeof(double) * m);
        int dims[3] = {fg.n[0], fg.n[1], 1};
        dims[a] += 1;
        for (long id = 0; id < m; id++) {
            int pos = a == 0 ? (int)(id % dims[0]) : (int)((id / dims[0]) % dims[1]);
            if ((pos == 0 && iface[a][0]) || (pos == fg.n[a] && iface[a][1])) {
                P->fa[a][id] /= 3.0;
                P->fk[a][id] /= 3.0;
            }
        }
    }
    return 0;
}

/* The interface part of the patch rows for base values xb: what the ghosts
 * u~ add to each fine cell's T-row and p-row (the p-row's l4 div(k grad T)
 * included). */
static void patch_ghost_terms(const orc_cgrid *cg, const level *P, int iface[2][2], double *const fkf[3],
                              double *const faf[3], const double *xb, double *out)
{
    const orc_grid *fg = &P->g;
    double h = fg->h;
    for (long i = 0; i < P->N; i++) {
        int c[3];
        cell_of(fg, i, c);
        double gT = 0.0, gp = 0.0;
        for (int a = 0; a < 2; a++)
            for (int s = 0; s < 2; s++) {
                if (!iface[a][s]) continue;
                if ((s == 0 && c[a] != 0) || (s == 1 && c[a] != fg->n[a] - 1)) continue;
                int f[3] = {c[0], c[1], 0};
                f[a] += s;
                long fid = face_id(fg, a, f);
                gT += fkf[a][fid] * ghost_value(cg, xb, a, s, c[0], c[1], 0, 1) / (1.5 * h * h);
                gp += faf[a][fid] * ghost_value(cg, xb, a, s, c[0], c[1], 1, 1) / (1.5 * h * h);
            }
        out[2 * i] = gT;
        out[2 * i + 1] = gp + P->lam[4 * i + 3] * gT;
    }
}

/* The valid base cells' rows' dependence on the patch values xf through the
 * interface fluxes, with zero base values (the reflux of a patch correction). */
static void base_reflux_terms(const orc_cgrid *cg, const orc_grid *fg, int iface[2][2], const double *lamb,
                              double *const fkf[3], double *const faf[3], const double *xf, double *out,
                              double *zero_b)
{
    const orc_grid *g = &cg->base;
    for (long i = 0; i < ncells(g); i++) {
        int c[3];
        cell_of(g, i, c);
        out[2 * i] = out[2 * i + 1] = 0.0;
        if (covered(cg, c[0], c[1])) continue;
        /* base_div with zero base values and the base faces' own terms removed:
           only the interface faces carry patch values */
        double tT = 0.0, tp = 0.0;
        double H = g->h;
        for (int a = 0; a < 2; a++)
            for (int s = 0; s < 2; s++) {
                int nb[3] = {c[0], c[1], 0};
                nb[a] += s ? 1 : -1;
                if (!(nb[a] >= 0 && nb[a] < g->n[a] && covered(cg, nb[0], nb[1]))) continue;
                int t = 1 - a, side = s ? 0 : 1;
                int fi_n = side == 0 ? 0 : fg->n[a] - 1;
                for (int q = 0; q < 2; q++) {
                    int ff[2];
                    ff[a] = fi_n;
                    ff[t] = 2 * (c[t] - cg->box[t][0]) + q;
                    int fc[3] = {ff[0], ff[1], 0};
                    int fface[3] = {ff[0], ff[1], 0};
                    fface[a] += side;
                    long fid = face_id(fg, a, fface);
                    long fci = cell_id(fg, fc);
                    tT += (0.5 * H) * fkf[a][fid] * xf[2 * fci] / (1.5 * 0.5 * H) / (H * H);
                    tp += (0.5 * H) * faf[a][fid] * xf[2 * fci + 1] / (1.5 * 0.5 * H) / (H * H);
                }
            }
        out[2 * i] = tT;
        out[2 * i + 1] = tp + lamb[4 * i + 3] * tT;
    }
    (void)iface;
    (void)zero_b;
}

/* Fine correction += bilinear prolongation of the base correction eb onto
 * the patch (the fine cells' positions inside the whole domain; base cells
 * outside the domain by their homogeneous ghosts). */
static void prolong_to_patch(const orc_cgrid *cg, const level *P, const double *eb, double *xf)
{
    const orc_grid *g = &cg->base;
    for (long i = 0; i < P->N; i++) {
        int c[3];
        cell_of(&P->g, i, c);
        int gi = 2 * cg->box[0][0] + c[0], gj = 2 * cg->box[1][0] + c[1];   /* in a full fine grid */
        int Pc[2] = {gi / 2, gj / 2};
        int sg[2] = {(gi & 1) ? 1 : -1, (gj & 1) ? 1 : -1};
        for (int fld = 0; fld < 2; fld++) {
            double add = 0.0;
            for (int q = 0; q < 4; q++) {
                double w = 1.0;
                int Q[2] = {Pc[0], Pc[1]};
                for (int a = 0; a < 2; a++) {
                    if ((q >> a) & 1) { w *= 0.25; Q[a] += sg[a]; }
                    else w *= 0.75;
                }
                add += w * base_value(g, eb, Q[0], Q[1], fld, 1);
            }
            xf[2 * i + fld] += add;
        }
    }
}

/* The base grid's coefficients under the patch, for the base correction:
 * covered cells take the mean of their four children's l1..l4 and every base
 * face of a covered cell the mean of its two fine faces (the coarsening of
 * the hierarchy), so the base correction sees the patch's own coefficients. */
static void cover_with_patch(const orc_cgrid *cg, const orc_grid *pg, const double *lamf, double *const faf[3],
                             double *const fkf[3], level *B)
{
    const orc_grid *g = &cg->base;
    for (long I = 0; I < ncells(g); I++) {
        int c[3];
        cell_of(g, I, c);
        if (!covered(cg, c[0], c[1])) continue;
        for (int t = 0; t < 4; t++) {
            double acc = 0.0;
            for (int q = 0; q < 4; q++) {
                int fc[3] = {2 * (c[0] - cg->box[0][0]) + (q & 1), 2 * (c[1] - cg->box[1][0]) + (q >> 1), 0};
                acc += lamf[4 * cell_id(pg, fc) + t];
            }
            B->lam[4 * I + t] = acc / 4.0;
        }
        for (int a = 0; a < 2; a++)
            for (int s = 0; s < 2; s++) {
                int F[3] = {c[0], c[1], 0};
                F[a] += s;
                double sa = 0.0, sk = 0.0;
                for (int q = 0; q < 2; q++) {
                    int f[3] = {2 * (F[0] - cg->box[0][0]), 2 * (F[1] - cg->box[1][0]), 0};
                    f[1 - a] += q;
                    long fid = face_id(pg, a, f);
                    sa += faf[a][fid];
                    sk += fkf[a][fid];
                }
                B->fa[a][face_id(g, a, F)] = sa / 2.0;
                B->fk[a][face_id(g, a, F)] = sk / 2.0;
            }
    }
}

/*
 * Solve L(x) = b on the composite grid by the defect-correction loop with
 * one FAC cycle per step (see the header), `cycles` steps.  Base arrays
 * cover the base grid (covered cells: on return the volume-weighted mean of
 * their fine children); patch arrays the patch.  hist (nullable, 4 *
 * (cycles + 1)): per step the L2 norms of the T and p residuals over the
 * valid base cells, then over the patch.  Returns 0 or a negative code.
 */
int orc_cf_fac_solve(const orc_cgrid *cg, const double *lamb, double *const fab[3], double *const fkb[3],
                     const double *lamf, double *const faf[3], double *const fkf[3], const double *bb,
                     const double *bf, double *xb, double *xf, int nu1, int nu2, int coarse_min, int cycles,
                     double *hist)
{
    int iface[2][2];
    level P;
    if (patch_level(cg, lamf, faf, fkf, &P, iface)) return -2;
    orc_grid fgi = patch_grid(cg, iface);
    const orc_grid *g = &cg->base;
    long Nb = ncells(g), Nf = P.N;
    int nlev = orc_num_levels(g, coarse_min);
    level *Ls = calloc(nlev, sizeof(level));
    double *rb = malloc(sizeof(double) * 2 * Nb), *rf = malloc(sizeof(double) * 2 * Nf);
    double *tb = malloc(sizeof(double) * 2 * Nb), *tf = malloc(sizeof(double) * 2 * Nf);
    int rc = 0;
    if (!Ls || !rb || !rf || !tb || !tf) { rc = -2; goto done; }
    if (alloc_level(&Ls[0], g)) { rc = -2; goto done; }
    memset(Ls[0].g.bcT, 0, sizeof(Ls[0].g.bcT));
    memset(Ls[0].g.bcp, 0, sizeof(Ls[0].g.bcp));
    fill_level0(&Ls[0], lamb, fab, fkb);
    cover_with_patch(cg, &P.g, lamf, faf, fkf, &Ls[0]);
    for (int l = 1; l < nlev; l++)
        if (coarsen(&Ls[l - 1], &Ls[l])) { rc = -2; goto done; }
    smoother sm = {0, 0.0};
    for (int k = 0;; k++) {
        /* step 1: the composite residual */
        orc_cf_apply(cg, lamb, fab, fkb, lamf, faf, fkf, xb, xf, rb, rf, 0);
        double n4[4] = {0, 0, 0, 0};
        for (long i = 0; i < Nb; i++) {
            int c[3];
            cell_of(g, i, c);
            if (covered(cg, c[0], c[1])) { rb[2 * i] = rb[2 * i + 1] = 0.0; continue; }
            rb[2 * i] = bb[2 * i] - rb[2 * i];
            rb[2 * i + 1] = bb[2 * i + 1] - rb[2 * i + 1];
            n4[0] += rb[2 * i] * rb[2 * i];
            n4[1] += rb[2 * i + 1] * rb[2 * i + 1];
        }
        for (long i = 0; i < Nf; i++) {
            rf[2 * i] = bf[2 * i] - rf[2 * i];
            rf[2 * i + 1] = bf[2 * i + 1] - rf[2 * i + 1];
            n4[2] += rf[2 * i] * rf[2 * i];
            n4[3] += rf[2 * i + 1] * rf[2 * i + 1];
        }
        if (hist) for (int q = 0; q < 4; q++) hist[4 * k + q] = sqrt(n4[q]);
        if (k == cycles) break;
        /* step 3: the correction by one FAC cycle from zero */
        memcpy(P.rhs, rf, sizeof(double) * 2 * Nf);
        memset(P.u, 0, sizeof(double) * 2 * Nf);
        for (int s = 0; s < nu1; s++) smooth(&P, &sm, NULL, NULL);
        level_residual(&P);                                   /* P.r: the patch residual */
        base_reflux_terms(cg, &fgi, iface, lamb, fkf, faf, P.u, tb, NULL);
        for (long I = 0; I < Nb; I++) {
            int c[3];
            cell_of(g, I, c);
            if (!covered(cg, c[0], c[1])) {
                Ls[0].rhs[2 * I] = rb[2 * I] - tb[2 * I];
                Ls[0].rhs[2 * I + 1] = rb[2 * I + 1] - tb[2 * I + 1];
            } else {                                          /* mean of the four children */
                double s0 = 0.0, s1 = 0.0;
                for (int q = 0; q < 4; q++) {
                    int fc[3] = {2 * (c[0] - cg->box[0][0]) + (q & 1), 2 * (c[1] - cg->box[1][0]) + (q >> 1), 0};
                    long f = cell_id(&P.g, fc);
                    s0 += P.r[2 * f];
                    s1 += P.r[2 * f + 1];
                }
                Ls[0].rhs[2 * I] = s0 / 4.0;
                Ls[0].rhs[2 * I + 1] = s1 / 4.0;
            }
        }
        memset(Ls[0].u, 0, sizeof(double) * 2 * Nb);
        rc = mgcycle(Ls, 0, nlev, nu1, nu2, 0, &sm);
        if (rc) goto done;
        prolong_to_patch(cg, &P, Ls[0].u, P.u);
        patch_ghost_terms(cg, &P, iface, fkf, faf, Ls[0].u, tf);
        for (long i = 0; i < 2 * Nf; i++) P.rhs[i] = rf[i] - tf[i];
        for (int s = 0; s < nu2; s++) smooth(&P, &sm, NULL, NULL);
        /* step 4: update the valid cells */
        for (long I = 0; I < Nb; I++) {
            int c[3];
            cell_of(g, I, c);
            if (covered(cg, c[0], c[1])) continue;
            xb[2 * I] += Ls[0].u[2 * I];
            xb[2 * I + 1] += Ls[0].u[2 * I + 1];
        }
        for (long i = 0; i < 2 * Nf; i++) xf[i] += P.u[i];
    }
    /* covered base cells: the mean of their children */
    for (long I = 0; I < Nb; I++) {
        int c[3];
        cell_of(g, I, c);
        if (!covered(cg, c[0], c[1])) continue;
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < 4; q++) {
            int fc[3] = {2 * (c[0] - cg->box[0][0]) + (q & 1), 2 * (c[1] - cg->box[1][0]) + (q >> 1), 0};
            long f = cell_id(&P.g, fc);
            s0 += xf[2 * f];
            s1 += xf[2 * f + 1];
        }
        xb[2 * I] = s0 / 4.0;
        xb[2 * I + 1] = s1 / 4.0;
    }
done:
    if (Ls) for (int l = 0; l < nlev; l++) free_level(&Ls[l]);
    free(Ls);
    free_level(&P);
    free(rb); free(rf); free(tb); free(tf);
    return rc;
}

/* Exact solution of the composite system by Gaussian elimination on the
 * unknowns of the valid base cells and the patch (small grids only).  Covered
 * base cells of xb receive the mean of their children. */
int orc_cf_dense_solve(const orc_cgrid *cg, const double *lamb, double *const fab[3], double *const fkb[3],
                       const double *lamf, double *const faf[3], double *const fkf[3], const double *bb,
                       const double *bf, double *xb, double *xf)
{
    int iface[2][2];
    orc_grid fg = patch_grid(cg, iface);
    const orc_grid *g = &cg->base;
    long Nb = ncells(g), Nf = ncells(&fg);
    long *map = malloc(sizeof(long) * Nb);
    long nv = 0;
    for (long I = 0; I < Nb; I++) {
        int c[3];
        cell_of(g, I, c);
        map[I] = covered(cg, c[0], c[1]) ? -1 : nv++;
    }
    long n = 2 * (nv + Nf);
    double *M = malloc(sizeof(double) * n * n), *z = malloc(sizeof(double) * n);
    double *eb = calloc(2 * Nb, sizeof(double)), *ef = calloc(2 * Nf, sizeof(double));
    double *yb = malloc(sizeof(double) * 2 * Nb), *yf = malloc(sizeof(double) * 2 * Nf);
    int rc = 0;
    if (!map || !M || !z || !eb || !ef || !yb || !yf) { rc = -2; goto done; }
    for (long j = 0; j < n; j++) {
        long u = j / 2;
        int fld = (int)(j % 2);
        double *slot;
        if (u < nv) {
            long I = 0;
            for (; I < Nb; I++) if (map[I] == u) break;
            slot = eb + 2 * I + fld;
        } else {
            slot = ef + 2 * (u - nv) + fld;
        }
        *slot = 1.0;
        orc_cf_apply(cg, lamb, fab, fkb, lamf, faf, fkf, eb, ef, yb, yf, 1);
        *slot = 0.0;
        for (long I = 0; I < Nb; I++)
            if (map[I] >= 0) {
                M[(2 * map[I]) * n + j] = yb[2 * I];
                M[(2 * map[I] + 1) * n + j] = yb[2 * I + 1];
            }
        for (long i = 0; i < Nf; i++) {
            M[(2 * (nv + i)) * n + j] = yf[2 * i];
            M[(2 * (nv + i) + 1) * n + j] = yf[2 * i + 1];
        }
    }
    orc_cf_apply(cg, lamb, fab, fkb, lamf, faf, fkf, eb, ef, yb, yf, 0);     /* the affine part */
    for (long I = 0; I < Nb; I++)
        if (map[I] >= 0) {
            z[2 * map[I]] = bb[2 * I] - yb[2 * I];
            z[2 * map[I] + 1] = bb[2 * I + 1] - yb[2 * I + 1];
        }
    for (long i = 0; i < Nf; i++) {
        z[2 * (nv + i)] = bf[2 * i] - yf[2 * i];
        z[2 * (nv + i) + 1] = bf[2 * i + 1] - yf[2 * i + 1];
    }
    rc = gauss_solve(n, M, z);
    if (rc) goto done;
    for (long I = 0; I < Nb; I++)
        if (map[I] >= 0) { xb[2 * I] = z[2 * map[I]]; xb[2 * I + 1] = z[2 * map[I] + 1]; }
    for (long i = 0; i < Nf; i++) { xf[2 * i] = z[2 * (nv + i)]; xf[2 * i + 1] = z[2 * (nv + i) + 1]; }
    for (long I = 0; I < Nb; I++) {
        int c[3];
        cell_of(g, I, c);
        if (map[I] >= 0) continue;
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < 4; q++) {
            int fc[3] = {2 * (c[0] - cg->box[0][0]) + (q & 1), 2 * (c[1] - cg->box[1][0]) + (q >> 1), 0};
            long f = cell_id(&fg, fc);
            s0 += xf[2 * f];
            s1 += xf[2 * f + 1];
        }
        xb[2 * I] = s0 / 4.0;
        xb[2 * I + 1] = s1 / 4.0;
    }
done:
    free(map); free(M); free(z); free(eb); free(ef); free(yb); free(yf);
    return rc;
}
