/*
 * Plain FP64 CPU oracle for the coupled pressure-temperature Poisson-Helmholtz
 * solve (Saade, Lohse & Fuster, "A multigrid solver for the coupled
 * pressure-temperature equations in an all-Mach solver with VoF", Sec. 3,
 * Eqs. 27-34 and the defect-correction loop that follows them).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the package smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or constant with the CUDA
 * library: it is written directly from the paper's equations, slowly and
 * plainly, in the physical (un-scaled) finite-volume form.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no FMA
 * contraction, single thread), so every operation rounds as written.  That is
 * the build every comparison uses.  A second build adds -fopenmp only to time
 * the oracle on all host cores: the pragmas below split the loops over the
 * cells of one level (of one colour in a red-black sweep, whose cells do not
 * read each other), so each cell's arithmetic is unchanged; only the order in
 * which the stopping norm's squares are summed differs.
 *
 * What is computed
 * ----------------
 * Unknown per cell: a = (T, p), in the paper's order (Sec. 3, the operator
 * form L(a) = b following Eq. 34).  Per-cell inputs lambda1..lambda4 (Eqs.
 * 29-32), right-hand side (lambda_T, lambda_p) (Eqs. 33-34), face coefficients
 * 1/rho and k on every face (Eqs. 27-28).
 *
 *   T-row (Eq. 27):  div(k grad T) + l1 T + l2 p                 = lambda_T
 *   p-row (Eq. 28):  div((1/rho) grad p) + l3 p + l4 div(k grad T) = lambda_p
 *
 * Cell-centred finite volumes on a uniform grid of spacing h:
 *   div(c grad u)_i = (1/V_i) sum_faces A_f c_f (u_nb - u_i) / d_f
 * with d_f = h between two cells, d_f = h/2 to a Dirichlet boundary value,
 * and no flux through a wall (Neumann) or through the symmetry axis.
 * Cartesian: V = h^dim, A = h^(dim-1).  Axisymmetric (axis 0 = r, axis 1 = z):
 * V_i = r_i h^2, A_f = r_f h on r-faces and r_i h on z-faces (the common
 * factor 2*pi cancels).
 *
 * Parity unpinned: none.  Every function below is pinned by the CPU tests
 * (closed-form grid modes, dense solves, an independently assembled sparse
 * operator, second-order convergence, symmetry, the zero-coupling limit).
 *
 * The multigrid (the paper names the solver type but not its parts) is this
 * library's reading, written out plainly:
 *   - the system is solved in its printed form (Eqs. 27-28), the p-row
 *     keeping its l4 div(k grad T) term;
 *   - V(nu1, nu2) cycle, red-black block Gauss-Seidel (red = even i+j+k,
 *     red first), each cell's two equations solved exactly for (T_i, p_i);
 *     or, as the other smoother, weighted block Jacobi: every cell's two
 *     equations solved against the previous iterate's neighbours, the cell
 *     then moving a fraction omega of the way to that solution;
 *   - restriction: volume-weighted mean of the 2^dim children;
 *   - prolongation: cell-centred bi/tri-linear (weights 3/4 and 1/4 per axis),
 *     reflecting ghosts (same value at walls and the axis, opposite sign at
 *     Dirichlet faces);
 *   - coarse operator: Eqs. 27-28 re-discretised at 2h with area-weighted
 *     mean face coefficients and volume-weighted mean l1..l4; coarsen while
 *     every dimension is even and halves to at least coarse_min;
 *   - coarsest level solved exactly by Gaussian elimination;
 *   - outer loop = the paper's defect correction: res = b - L(a); stop when
 *     small; else solve L(da) ~= res by one V-cycle from da = 0; a += da.
 *   - stopping norm, per field: || D^{-1} r ||_2 over cells, where r is the
 *     residual and D the 2x2 block of each cell's own unknowns in its two
 *     equations; stop when both fields' norms fell by rtol relative to the
 *     initial ones.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the loops below run on: 1 in the comparison build. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

enum { BC_WALL = 0, BC_DIRICHLET = 1, BC_AXIS = 2 };

typedef struct {
    int dim;          /* 2 or 3 */
    int axisym;       /* 1: dim == 2, axis 0 is r, axis 1 is z */
    int n[3];         /* cells per axis; n[2] = 1 when dim == 2 */
    double h;         /* uniform spacing */
    double r0;        /* axisymmetric: radius of the low-r boundary (0 = axis) */
    int bc[3][2];     /* per axis, low / high side: BC_WALL, BC_DIRICHLET, BC_AXIS */
    double bcT[3][2]; /* Dirichlet values of T */
    double bcp[3][2]; /* Dirichlet values of p */
} orc_grid;

/* One multigrid level, physical form. */
typedef struct {
    orc_grid g;
    long N;
    double *lam;      /* N x 4: l1..l4 of Eqs. 29-32 (coarse levels: volume-weighted means) */
    double *fa[3];    /* 1/rho on faces, per axis */
    double *fk[3];    /* k on faces, per axis */
    double *rhs;      /* N x 2 */
    double *u;        /* N x 2 */
    double *r;        /* N x 2 */
} level;

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

static long cell_id(const orc_grid *g, const int c[3])
{
    return c[0] + (long)g->n[0] * (c[1] + (long)g->n[1] * c[2]);
}

static long nfaces(const orc_grid *g, int a)
{
    long m = 1;
    for (int b = 0; b < 3; b++) m *= (b == a) ? g->n[b] + 1 : g->n[b];
    return m;
}

/* Face at position f (f[a] in 0..n[a]) of the faces normal to axis a. */
static long face_id(const orc_grid *g, int a, const int f[3])
{
    int m[3] = {g->n[0], g->n[1], g->n[2]};
    m[a] += 1;
    return f[0] + (long)m[0] * (f[1] + (long)m[1] * f[2]);
}

static long ncells(const orc_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static void cell_of(const orc_grid *g, long id, int c[3])
{
    c[0] = (int)(id % g->n[0]);
    c[1] = (int)((id / g->n[0]) % g->n[1]);
    c[2] = (int)(id / ((long)g->n[0] * g->n[1]));
}

static double r_cell(const orc_grid *g, int i) { return g->r0 + (i + 0.5) * g->h; }
static double r_face(const orc_grid *g, int i) { return g->r0 + i * g->h; }

static double volume(const orc_grid *g, const int c[3])
{
    if (g->axisym) return r_cell(g, c[0]) * g->h * g->h;
    return g->dim == 2 ? g->h * g->h : g->h * g->h * g->h;
}

/* Area of the face normal to axis a at face position f, belonging to cell c. */
static double area(const orc_grid *g, int a, const int f[3], const int c[3])
{
    if (g->axisym) return (a == 0 ? r_face(g, f[0]) : r_cell(g, c[0])) * g->h;
    return g->dim == 2 ? g->h : g->h * g->h;
}

/* ------------------------------------------------------------------ */
/* div(c grad u) at one cell, Eqs. 27-28                               */
/* ------------------------------------------------------------------ */

/* u is strided (stride 2, field offset already applied); bcv: Dirichlet
 * values per axis/side, or NULL for homogeneous boundary values. */
static double div_flux(const orc_grid *g, double *const coef[3], const double *u,
                       double bcv[3][2], const int c[3])
{
    long i = cell_id(g, c);
    double sum = 0.0;
    for (int a = 0; a < g->dim; a++) {
        for (int side = 0; side < 2; side++) {
            int f[3] = {c[0], c[1], c[2]};
            f[a] += side;                       /* low face c[a], high face c[a]+1 */
            int nb[3] = {c[0], c[1], c[2]};
            nb[a] += side ? 1 : -1;
            double A = area(g, a, f, c);
            double cf = coef[a][face_id(g, a, f)];
            if (nb[a] >= 0 && nb[a] < g->n[a]) {
                sum += A * cf * (u[2 * cell_id(g, nb)] - u[2 * i]) / g->h;
            } else if (g->bc[a][side] == BC_DIRICHLET) {
                double gv = bcv ? bcv[a][side] : 0.0;
                sum += A * cf * (gv - u[2 * i]) / (0.5 * g->h);
            }                                   /* wall or axis: no flux */
        }
    }
    return sum / volume(g, c);
}

/* sigma_i: minus the coefficient of u_i in div(c grad u)_i. */
static double div_flux_diag(const orc_grid *g, double *const coef[3], const int c[3])
{
    double sum = 0.0;
    for (int a = 0; a < g->dim; a++) {
        for (int side = 0; side < 2; side++) {
            int f[3] = {c[0], c[1], c[2]};
            f[a] += side;
            int nbi = c[a] + (side ? 1 : -1);
            double A = area(g, a, f, c);
            double cf = coef[a][face_id(g, a, f)];
            if (nbi >= 0 && nbi < g->n[a]) sum += A * cf / g->h;
            else if (g->bc[a][side] == BC_DIRICHLET) sum += A * cf / (0.5 * g->h);
        }
    }
    return sum / volume(g, c);
}

/* ------------------------------------------------------------------ */
/* The paper's operator L(a), Eqs. 27-28                               */
/* ------------------------------------------------------------------ */

/* y = L(x).  homogeneous != 0 uses zero Dirichlet values (the linear part);
 * otherwise the grid's Dirichlet values enter (the affine operator). */
void orc_apply_paper(const orc_grid *g, const double *lam, double *const fa[3],
                     double *const fk[3], const double *x, double *y, int homogeneous)
{
    long N = ncells(g);
    double (*vT)[2] = homogeneous ? NULL : (double (*)[2])g->bcT;
    double (*vp)[2] = homogeneous ? NULL : (double (*)[2])g->bcp;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        int c[3];
        cell_of(g, i, c);
        double lapT = div_flux(g, fk, x + 0, vT, c);
        double lapp = div_flux(g, fa, x + 1, vp, c);
        const double *l = lam + 4 * i;
        double T = x[2 * i], p = x[2 * i + 1];
        y[2 * i]     = lapT + l[0] * T + l[1] * p;              /* Eq. 27 */
        y[2 * i + 1] = lapp + l[2] * p + l[3] * lapT;           /* Eq. 28 */
    }
}

/* ------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting                    */
/* ------------------------------------------------------------------ */

/* Solves M z = rhs in place (M is n x n row-major, destroyed; rhs -> z).
 * Returns 0, or -1 if a pivot is exactly zero. */
static int gauss_solve(long n, double *M, double *rhs)
{
    for (long k = 0; k < n; k++) {
        long piv = k;
        double best = fabs(M[k * n + k]);
        for (long r = k + 1; r < n; r++)
            if (fabs(M[r * n + k]) > best) { best = fabs(M[r * n + k]); piv = r; }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (long cc = 0; cc < n; cc++) {
                double t = M[k * n + cc]; M[k * n + cc] = M[piv * n + cc]; M[piv * n + cc] = t;
            }
            double t = rhs[k]; rhs[k] = rhs[piv]; rhs[piv] = t;
        }
        for (long r = k + 1; r < n; r++) {
            double m = M[r * n + k] / M[k * n + k];
            if (m == 0.0) continue;
            for (long cc = k; cc < n; cc++) M[r * n + cc] -= m * M[k * n + cc];
            rhs[r] -= m * rhs[k];
        }
    }
    for (long k = n - 1; k >= 0; k--) {
        double s = rhs[k];
        for (long cc = k + 1; cc < n; cc++) s -= M[k * n + cc] * rhs[cc];
        rhs[k] = s / M[k * n + k];
    }
    return 0;
}

/* Exact solution of L(x) = b (Eqs. 27-28, with the grid's Dirichlet values)
 * by assembling the 2N x 2N matrix column by column and eliminating.
 * Only for small grids.  Returns 0, -1 (singular) or -2 (allocation). */
int orc_dense_solve(const orc_grid *g, const double *lam, double *const fa[3],
                    double *const fk[3], const double *b, double *x)
{
    long N = ncells(g), n = 2 * N;
    double *M = malloc(sizeof(double) * n * n);
    double *e = calloc(n, sizeof(double));
    double *col = malloc(sizeof(double) * n);
    double *z = malloc(sizeof(double) * n);
    if (!M || !e || !col || !z) { free(M); free(e); free(col); free(z); return -2; }
    for (long j = 0; j < n; j++) {
        e[j] = 1.0;
        orc_apply_paper(g, lam, fa, fk, e, col, 1);
        for (long r = 0; r < n; r++) M[r * n + j] = col[r];
        e[j] = 0.0;
    }
    /* affine part: L(0) carries the Dirichlet values */
    orc_apply_paper(g, lam, fa, fk, e, col, 0);
    for (long r = 0; r < n; r++) z[r] = b[r] - col[r];
    int rc = gauss_solve(n, M, z);
    if (rc == 0) memcpy(x, z, sizeof(double) * n);
    free(M); free(e); free(col); free(z);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Eqs. 27-28 on one level                                              */
/* ------------------------------------------------------------------ */

/* The two rows of Eqs. 27-28 at cell c of a level:
 *   T-row: div(k grad T) + l1 T + l2 p
 *   p-row: div((1/rho) grad p) + l3 p + l4 div(k grad T)              */
static void paper_row(const level *L, const double *u, double *const bcT2, double *const bcp2,
                      const int c[3], double out[2])
{
    long i = cell_id(&L->g, c);
    const double *l = L->lam + 4 * i;
    double lapT = div_flux(&L->g, L->fk, u + 0, (double (*)[2])bcT2, c);
    double lapp = div_flux(&L->g, L->fa, u + 1, (double (*)[2])bcp2, c);
    out[0] = lapT + l[0] * u[2 * i] + l[1] * u[2 * i + 1];
    out[1] = lapp + l[2] * u[2 * i + 1] + l[3] * lapT;
}

/* Coefficients of (T_i, p_i) in cell i's two rows:
 *   [[l1 - sigma_k, l2], [-l4 sigma_k, l3 - sigma_a]]                  */
static void diag_block(const level *L, const int c[3], double D[4])
{
    long i = cell_id(&L->g, c);
    const double *l = L->lam + 4 * i;
    double sk = div_flux_diag(&L->g, L->fk, c);
    double sa = div_flux_diag(&L->g, L->fa, c);
    D[0] = l[0] - sk;
    D[1] = l[1];
    D[2] = -l[3] * sk;
    D[3] = l[2] - sa;
}

static void solve2(const double D[4], const double s[2], double z[2])
{
    double det = D[0] * D[3] - D[1] * D[2];
    z[0] = (D[3] * s[0] - D[1] * s[1]) / det;
    z[1] = (D[0] * s[1] - D[2] * s[0]) / det;
}

/* r = rhs - L(u) on a level (homogeneous boundary values). */
static void level_residual(level *L)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L->N; i++) {
        int c[3];
        cell_of(&L->g, i, c);
        double e[2];
        paper_row(L, L->u, NULL, NULL, c, e);
        L->r[2 * i] = L->rhs[2 * i] - e[0];
        L->r[2 * i + 1] = L->rhs[2 * i + 1] - e[1];
    }
}

/* One red-black block Gauss-Seidel sweep: for every cell of one colour,
 * solve that cell's two equations for (T_i, p_i) holding all other
 * unknowns fixed; red cells (even i+j+k) first, then black. */
static void rbgs_sweep(level *L, double *const bcT2, double *const bcp2)
{
    for (int colour = 0; colour < 2; colour++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < L->N; i++) {
            int c[3];
            cell_of(&L->g, i, c);
            if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
            double e[2], D[4], s[2], z[2];
            paper_row(L, L->u, bcT2, bcp2, c, e);
            diag_block(L, c, D);
            /* rhs minus the off-diagonal part of the rows: rhs - (L(u) - D u_i) */
            s[0] = L->rhs[2 * i] - (e[0] - (D[0] * L->u[2 * i] + D[1] * L->u[2 * i + 1]));
            s[1] = L->rhs[2 * i + 1] - (e[1] - (D[2] * L->u[2 * i] + D[3] * L->u[2 * i + 1]));
            solve2(D, s, z);
            L->u[2 * i] = z[0];
            L->u[2 * i + 1] = z[1];
        }
    }
}

/* One weighted block Jacobi sweep: every cell's two equations are solved
 * for (T_i, p_i) with all other unknowns held at the previous iterate (the
 * same z_i as a Gauss-Seidel update, but from old neighbours only), and the
 * cell moves a fraction omega of the way: u_i <- u_i + omega (z_i - u_i). */
static int wjac_sweep(level *L, double *const bcT2, double *const bcp2, double omega)
{
    double *z = malloc(sizeof(double) * 2 * L->N);
    if (!z) return -2;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L->N; i++) {
        int c[3];
        cell_of(&L->g, i, c);
        double e[2], D[4], s[2];
        paper_row(L, L->u, bcT2, bcp2, c, e);
        diag_block(L, c, D);
        s[0] = L->rhs[2 * i] - (e[0] - (D[0] * L->u[2 * i] + D[1] * L->u[2 * i + 1]));
        s[1] = L->rhs[2 * i + 1] - (e[1] - (D[2] * L->u[2 * i] + D[3] * L->u[2 * i + 1]));
        solve2(D, s, z + 2 * i);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < 2 * L->N; i++) L->u[i] = L->u[i] + omega * (z[i] - L->u[i]);
    free(z);
    return 0;
}

/* The smoother of a cycle: kind 0 = red-black block Gauss-Seidel, 1 =
 * weighted block Jacobi with weight omega. */
typedef struct {
    int kind;
    double omega;
} smoother;

static int smooth(level *L, const smoother *sm, double *const bcT2, double *const bcp2)
{
    if (sm->kind == 1) return wjac_sweep(L, bcT2, bcp2, sm->omega);
    rbgs_sweep(L, bcT2, bcp2);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Hierarchy                                                           */
/* ------------------------------------------------------------------ */

static int alloc_level(level *L, const orc_grid *g)
{
    memset(L, 0, sizeof(*L));
    L->g = *g;
    L->N = ncells(g);
    L->lam = calloc(4 * L->N, sizeof(double));
    L->rhs = calloc(2 * L->N, sizeof(double));
    L->u = calloc(2 * L->N, sizeof(double));
    L->r = calloc(2 * L->N, sizeof(double));
    int ok = L->lam && L->rhs && L->u && L->r;
    for (int a = 0; a < 3; a++) {
        long m = a < g->dim ? nfaces(g, a) : 1;
        L->fa[a] = calloc(m, sizeof(double));
        L->fk[a] = calloc(m, sizeof(double));
        ok = ok && L->fa[a] && L->fk[a];
    }
    return ok ? 0 : -2;
}

static void free_level(level *L)
{
    free(L->lam); free(L->rhs); free(L->u); free(L->r);
    for (int a = 0; a < 3; a++) { free(L->fa[a]); free(L->fk[a]); }
}

static int can_coarsen(const orc_grid *g, int coarse_min)
{
    for (int a = 0; a < g->dim; a++)
        if (g->n[a] % 2 != 0 || g->n[a] / 2 < coarse_min) return 0;
    return 1;
}

/* Coarse level at spacing 2h: area-weighted mean face coefficients and
 * volume-weighted mean l1..l4 of the children. */
static int coarsen(const level *F, level *C)
{
    orc_grid g = F->g;
    for (int a = 0; a < g.dim; a++) g.n[a] /= 2;
    g.h = 2.0 * F->g.h;
    memset(g.bcT, 0, sizeof(g.bcT));
    memset(g.bcp, 0, sizeof(g.bcp));
    if (alloc_level(C, &g)) return -2;

    int nchild = 1 << g.dim;
#pragma omp parallel for schedule(static)
    for (long I = 0; I < C->N; I++) {
        int cc[3];
        cell_of(&C->g, I, cc);
        double vsum = 0.0, acc[4] = {0, 0, 0, 0};
        for (int q = 0; q < nchild; q++) {
            int fc[3] = {2 * cc[0] + (q & 1), 2 * cc[1] + ((q >> 1) & 1),
                         g.dim == 3 ? 2 * cc[2] + ((q >> 2) & 1) : 0};
            double V = volume(&F->g, fc);
            const double *l = F->lam + 4 * cell_id(&F->g, fc);
            for (int t = 0; t < 4; t++) acc[t] += V * l[t];
            vsum += V;
        }
        for (int t = 0; t < 4; t++) C->lam[4 * I + t] = acc[t] / vsum;
    }

    for (int a = 0; a < g.dim; a++) {
        long m = nfaces(&C->g, a);
        int dims[3] = {C->g.n[0], C->g.n[1], C->g.n[2]};
        dims[a] += 1;
#pragma omp parallel for schedule(static)
        for (long id = 0; id < m; id++) {
            int Fp[3] = {(int)(id % dims[0]), (int)((id / dims[0]) % dims[1]),
                         (int)(id / ((long)dims[0] * dims[1]))};
            double asum = 0.0, sa = 0.0, sk = 0.0, pa = 0.0, pk = 0.0;
            int nsub = 1 << (g.dim - 1);
            for (int q = 0; q < nsub; q++) {
                int f[3], cfine[3], bit = 0;
                for (int b = 0; b < 3; b++) {
                    if (b == a) { f[b] = 2 * Fp[b]; continue; }
                    if (b >= g.dim) { f[b] = 0; continue; }
                    f[b] = 2 * Fp[b] + ((q >> bit) & 1);
                    bit++;
                }
                /* the fine cell owning this face on its low side (for the
                 * radius of an axisymmetric z-face) */
                for (int b = 0; b < 3; b++) cfine[b] = f[b];
                if (cfine[a] >= F->g.n[a]) cfine[a] = F->g.n[a] - 1;
                double A = area(&F->g, a, f, cfine);
                long fid = face_id(&F->g, a, f);
                asum += A;
                sa += A * F->fa[a][fid];
                sk += A * F->fk[a][fid];
                pa += F->fa[a][fid] / nsub;
                pk += F->fk[a][fid] / nsub;
            }
            /* a face of zero area (the symmetry axis) carries no flux; its
             * coefficient is the plain mean so that it stays finite */
            C->fa[a][id] = asum > 0.0 ? sa / asum : pa;
            C->fk[a][id] = asum > 0.0 ? sk / asum : pk;
        }
    }
    return 0;
}

/* coarse rhs = volume-weighted mean of the children's residuals */
static void restrict_residual(const level *F, level *C)
{
    int nchild = 1 << C->g.dim;
#pragma omp parallel for schedule(static)
    for (long I = 0; I < C->N; I++) {
        int cc[3];
        cell_of(&C->g, I, cc);
        double vsum = 0.0, s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < nchild; q++) {
            int fc[3] = {2 * cc[0] + (q & 1), 2 * cc[1] + ((q >> 1) & 1),
                         C->g.dim == 3 ? 2 * cc[2] + ((q >> 2) & 1) : 0};
            double V = volume(&F->g, fc);
            long f = cell_id(&F->g, fc);
            s0 += V * F->r[2 * f];
            s1 += V * F->r[2 * f + 1];
            vsum += V;
        }
        C->rhs[2 * I] = s0 / vsum;
        C->rhs[2 * I + 1] = s1 / vsum;
        C->u[2 * I] = 0.0;
        C->u[2 * I + 1] = 0.0;
    }
}

/* fine u += bi/tri-linear interpolation of the coarse correction */
static void prolong_add(const level *C, level *F)
{
    int dim = F->g.dim;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < F->N; i++) {
        int c[3];
        cell_of(&F->g, i, c);
        int P[3] = {c[0] / 2, c[1] / 2, dim == 3 ? c[2] / 2 : 0};
        int s[3] = {(c[0] & 1) ? 1 : -1, (c[1] & 1) ? 1 : -1, (c[2] & 1) ? 1 : -1};
        double add0 = 0.0, add1 = 0.0;
        for (int q = 0; q < (1 << dim); q++) {
            double w = 1.0, sign = 1.0;
            int Q[3] = {P[0], P[1], P[2]};
            for (int a = 0; a < dim; a++) {
                if ((q >> a) & 1) {
                    w *= 0.25;
                    int t = P[a] + s[a];
                    if (t < 0 || t >= C->g.n[a]) {
                        int side = t < 0 ? 0 : 1;
                        if (C->g.bc[a][side] == BC_DIRICHLET) sign = -sign;
                    } else {
                        Q[a] = t;
                    }
                } else {
                    w *= 0.75;
                }
            }
            long qi = cell_id(&C->g, Q);
            add0 += w * sign * C->u[2 * qi];
            add1 += w * sign * C->u[2 * qi + 1];
        }
        F->u[2 * i] += add0;
        F->u[2 * i + 1] += add1;
    }
}

/* Exact solve of the coarsest level's Eqs. 27-28 (homogeneous). */
static int coarse_solve(level *L)
{
    long n = 2 * L->N;
    double *M = malloc(sizeof(double) * n * n);
    double *z = malloc(sizeof(double) * n);
    double *saveu = L->u;
    double *e = calloc(n, sizeof(double));
    if (!M || !z || !e) { free(M); free(z); free(e); return -2; }
    L->u = e;
    for (long j = 0; j < n; j++) {
        e[j] = 1.0;
        for (long i = 0; i < L->N; i++) {
            int c[3];
            double out[2];
            cell_of(&L->g, i, c);
            paper_row(L, e, NULL, NULL, c, out);
            M[(2 * i) * n + j] = out[0];
            M[(2 * i + 1) * n + j] = out[1];
        }
        e[j] = 0.0;
    }
    L->u = saveu;
    memcpy(z, L->rhs, sizeof(double) * n);
    int rc = gauss_solve(n, M, z);
    if (rc == 0) memcpy(L->u, z, sizeof(double) * n);
    free(M); free(z); free(e);
    return rc;
}

/* One multigrid cycle from level l: pre-smoothing, restriction of the
 * residual, the coarse-grid correction, prolongation, post-smoothing.
 * type 0 (V): one coarse cycle; 1 (W): two W-cycles on the coarser level;
 * 2 (F): an F-cycle then a V-cycle on the coarser level.  The second coarse
 * cycle continues from the first one's coarse solution with the same
 * restricted right-hand side; at the coarsest level the exact solve is done
 * once (a second exact solve would give the same values). */
static int mgcycle(level *Ls, int l, int nlev, int nu1, int nu2, int type, const smoother *sm)
{
    level *L = &Ls[l];
    int rc;
    if (l == nlev - 1) return coarse_solve(L);
    for (int s = 0; s < nu1; s++)
        if ((rc = smooth(L, sm, NULL, NULL))) return rc;
    level_residual(L);
    restrict_residual(L, &Ls[l + 1]);
    rc = mgcycle(Ls, l + 1, nlev, nu1, nu2, type, sm);
    if (rc) return rc;
    if (type != 0 && l + 1 < nlev - 1) {
        rc = mgcycle(Ls, l + 1, nlev, nu1, nu2, type == 1 ? 1 : 0, sm);
        if (rc) return rc;
    }
    prolong_add(&Ls[l + 1], L);
    for (int s = 0; s < nu2; s++)
        if ((rc = smooth(L, sm, NULL, NULL))) return rc;
    return 0;
}

/* Fill level 0 from the paper's inputs. */
static void fill_level0(level *L, const double *lam, double *const fa[3], double *const fk[3])
{
    memcpy(L->lam, lam, sizeof(double) * 4 * L->N);
    for (int a = 0; a < L->g.dim; a++) {
        long m = nfaces(&L->g, a);
        memcpy(L->fa[a], fa[a], sizeof(double) * m);
        memcpy(L->fk[a], fk[a], sizeof(double) * m);
    }
}

/* Per-field || D^{-1} res ||_2 with D the cell's 2x2 diagonal block. */
static void scaled_norms(const level *L0, const double *res, double out[2])
{
    double s0 = 0.0, s1 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s0, s1)
    for (long i = 0; i < L0->N; i++) {
        int c[3];
        cell_of(&L0->g, i, c);
        double D[4], z[2];
        diag_block(L0, c, D);
        solve2(D, res + 2 * i, z);
        s0 += z[0] * z[0];
        s1 += z[1] * z[1];
    }
    out[0] = sqrt(s0);
    out[1] = sqrt(s1);
}

/* Number of levels the hierarchy of this grid has. */
int orc_num_levels(const orc_grid *g, int coarse_min)
{
    orc_grid t = *g;
    int n = 1;
    while (can_coarsen(&t, coarse_min)) {
        for (int a = 0; a < t.dim; a++) t.n[a] /= 2;
        n++;
    }
    return n;
}

/*
 * Solve L(x) = b (Eqs. 27-34) by the defect-correction loop with one
 * V(nu1, nu2) cycle (or W, F: cycle_type 1, 2) as the correction solve,
 * smoothed by red-black block Gauss-Seidel (smoother_kind 0) or weighted
 * block Jacobi with weight omega (smoother_kind 1).
 *   x       in: initial guess a~; out: result
 *   rtol    stop when both per-field norms fell by rtol (rtol <= 0: run
 *           exactly max_cycles cycles)
 *   hist    optional, 2 * (max_cycles + 1) doubles: per-field norms before
 *           each cycle and after the last
 * Returns the number of cycles run (>= 0) or a negative error code.
 */
int orc_mg_solve(const orc_grid *g, const double *lam, double *const fa[3], double *const fk[3],
                 const double *b, double *x, int nu1, int nu2, int coarse_min, int max_cycles,
                 double rtol, double *hist, int cycle_type, int smoother_kind, double omega)
{
    smoother sm = {smoother_kind, omega};
    int nlev = orc_num_levels(g, coarse_min);
    level *Ls = calloc(nlev, sizeof(level));
    double *res = NULL;
    int rc = 0, cycles = 0;
    if (!Ls) return -2;
    if (alloc_level(&Ls[0], g)) { rc = -2; goto done; }
    /* level 0 of the correction problem has homogeneous boundary values */
    memset(Ls[0].g.bcT, 0, sizeof(Ls[0].g.bcT));
    memset(Ls[0].g.bcp, 0, sizeof(Ls[0].g.bcp));
    fill_level0(&Ls[0], lam, fa, fk);
    for (int l = 1; l < nlev; l++)
        if (coarsen(&Ls[l - 1], &Ls[l])) { rc = -2; goto done; }

    long N = Ls[0].N;
    res = malloc(sizeof(double) * 2 * N);
    if (!res) { rc = -2; goto done; }

    double n0[2] = {0, 0};
    for (int k = 0;; k++) {
        /* step 1: res = b - L(x) */
        orc_apply_paper(g, lam, fa, fk, x, res, 0);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < 2 * N; i++) res[i] = b[i] - res[i];
        double nk[2];
        scaled_norms(&Ls[0], res, nk);
        if (hist) { hist[2 * k] = nk[0]; hist[2 * k + 1] = nk[1]; }
        if (k == 0) { n0[0] = nk[0]; n0[1] = nk[1]; }
        /* step 2: stop when small enough */
        if (k == max_cycles) break;
        if (rtol > 0.0) {
            double q0 = n0[0] > 0.0 ? nk[0] / n0[0] : 0.0;
            double q1 = n0[1] > 0.0 ? nk[1] / n0[1] : 0.0;
            if (q0 <= rtol && q1 <= rtol) break;
        }
        /* step 3: L(da) ~= res by one V-cycle from da = 0 */
        memcpy(Ls[0].rhs, res, sizeof(double) * 2 * N);
        memset(Ls[0].u, 0, sizeof(double) * 2 * N);
        rc = mgcycle(Ls, 0, nlev, nu1, nu2, cycle_type, &sm);
        if (rc) goto done;
        /* step 4: a += da */
#pragma omp parallel for schedule(static)
        for (long i = 0; i < 2 * N; i++) x[i] += Ls[0].u[i];
        cycles = k + 1;
    }
    rc = cycles;
done:
    if (Ls) for (int l = 0; l < nlev; l++) free_level(&Ls[l]);
    free(Ls);
    free(res);
    return rc;
}

/* In-place red-black block Gauss-Seidel sweeps on level 0 with the grid's
 * Dirichlet values (used to check single sweeps). */
int orc_rbgs_sweeps(const orc_grid *g, const double *lam, double *const fa[3],
                    double *const fk[3], const double *b, double *x, int sweeps)
{
    level L;
    if (alloc_level(&L, g)) { free_level(&L); return -2; }
    fill_level0(&L, lam, fa, fk);
    memcpy(L.rhs, b, sizeof(double) * 2 * L.N);
    memcpy(L.u, x, sizeof(double) * 2 * L.N);
    for (int s = 0; s < sweeps; s++) rbgs_sweep(&L, &L.g.bcT[0][0], &L.g.bcp[0][0]);
    memcpy(x, L.u, sizeof(double) * 2 * L.N);
    free_level(&L);
    return 0;
}

/* Weighted block Jacobi sweeps on level 0 with the grid's Dirichlet values. */
int orc_wjac_sweeps(const orc_grid *g, const double *lam, double *const fa[3],
                    double *const fk[3], const double *b, double *x, int sweeps, double omega)
{
    level L;
    int rc = 0;
    if (alloc_level(&L, g)) { free_level(&L); return -2; }
    fill_level0(&L, lam, fa, fk);
    memcpy(L.rhs, b, sizeof(double) * 2 * L.N);
    memcpy(L.u, x, sizeof(double) * 2 * L.N);
    for (int s = 0; s < sweeps && rc == 0; s++) rc = wjac_sweep(&L, &L.g.bcT[0][0], &L.g.bcp[0][0], omega);
    memcpy(x, L.u, sizeof(double) * 2 * L.N);
    free_level(&L);
    return rc;
}

/* Per-field || D^{-1} res ||_2 of the current x (the stopping norm). */
int orc_residual_norms(const orc_grid *g, const double *lam, double *const fa[3],
                       double *const fk[3], const double *b, const double *x, double out[2])
{
    level L;
    long N = ncells(g);
    double *res = malloc(sizeof(double) * 2 * N);
    if (!res || alloc_level(&L, g)) { free(res); return -2; }
    fill_level0(&L, lam, fa, fk);
    orc_apply_paper(g, lam, fa, fk, x, res, 0);
    for (long i = 0; i < 2 * N; i++) res[i] = b[i] - res[i];
    scaled_norms(&L, res, out);
    free(res);
    free_level(&L);
    return 0;
}

/* Coarse-level data of the hierarchy, for comparing set-up steps:
 * writes level l's l1..l4 (N_l x 4) and face coefficients. */
int orc_level_coeffs(const orc_grid *g, const double *lam, double *const fa[3],
                     double *const fk[3], int coarse_min, int l, double *B_out,
                     double *const fa_out[3], double *const fk_out[3])
{
    int nlev = orc_num_levels(g, coarse_min);
    if (l < 0 || l >= nlev) return -1;
    level *Ls = calloc(l + 1, sizeof(level));
    int rc = 0;
    if (!Ls) return -2;
    if (alloc_level(&Ls[0], g)) { rc = -2; goto done; }
    fill_level0(&Ls[0], lam, fa, fk);
    for (int q = 1; q <= l; q++)
        if (coarsen(&Ls[q - 1], &Ls[q])) { rc = -2; goto done; }
    memcpy(B_out, Ls[l].lam, sizeof(double) * 4 * Ls[l].N);
    for (int a = 0; a < g->dim; a++) {
        long m = nfaces(&Ls[l].g, a);
        memcpy(fa_out[a], Ls[l].fa[a], sizeof(double) * m);
        memcpy(fk_out[a], Ls[l].fk[a], sizeof(double) * m);
    }
done:
    for (int q = 0; q <= l; q++) free_level(&Ls[q]);
    free(Ls);
    return rc;
}

/* y at selected cells only: out[2*q..] = L(x) of Eqs. 27-28 at cell ids[q]
 * (with the grid's Dirichlet values).  For checking residuals of large
 * solutions at sampled cells. */
void orc_apply_rows(const orc_grid *g, const double *lam, double *const fa[3], double *const fk[3],
                    const double *x, const long *ids, long nids, double *out)
{
    double (*vT)[2] = (double (*)[2])g->bcT;
    double (*vp)[2] = (double (*)[2])g->bcp;
    for (long q = 0; q < nids; q++) {
        long i = ids[q];
        int c[3];
        cell_of(g, i, c);
        double lapT = div_flux(g, fk, x + 0, vT, c);
        double lapp = div_flux(g, fa, x + 1, vp, c);
        const double *l = lam + 4 * i;
        double T = x[2 * i], p = x[2 * i + 1];
        out[2 * q]     = lapT + l[0] * T + l[1] * p;            /* Eq. 27 */
        out[2 * q + 1] = lapp + l[2] * p + l[3] * lapT;         /* Eq. 28 */
    }
}

/* ------------------------------------------------------------------ */
/* The grid transfers alone (pinned separately by the CPU tests)       */
/* ------------------------------------------------------------------ */

/* The grid of the next coarser level: every n_a halved, spacing 2h, the
 * same boundary kinds and r0, homogeneous boundary values. */
static orc_grid coarse_grid_of(const orc_grid *g)
{
    orc_grid c = *g;
    for (int a = 0; a < c.dim; a++) c.n[a] /= 2;
    c.h = 2.0 * g->h;
    memset(c.bcT, 0, sizeof(c.bcT));
    memset(c.bcp, 0, sizeof(c.bcp));
    return c;
}

/* Restriction of a fine residual r (N x 2 on grid g, every n_a even) to the
 * coarse right-hand side bc (N/2^dim x 2), as a V-cycle forms it. */
int orc_restrict(const orc_grid *g, const double *r, double *bc)
{
    level F, C;
    orc_grid cg = coarse_grid_of(g);
    int rc = alloc_level(&F, g) || alloc_level(&C, &cg) ? -2 : 0;
    if (rc == 0) {
        memcpy(F.r, r, sizeof(double) * 2 * F.N);
        restrict_residual(&F, &C);
        memcpy(bc, C.rhs, sizeof(double) * 2 * C.N);
    }
    free_level(&F);
    free_level(&C);
    return rc;
}

/* Prolongation of a coarse correction uc (on the coarse grid of g) added to
 * the fine unknowns uf (N x 2 on grid g), as a V-cycle applies it. */
int orc_prolong_add(const orc_grid *g, const double *uc, double *uf)
{
    level F, C;
    orc_grid cg = coarse_grid_of(g);
    int rc = alloc_level(&F, g) || alloc_level(&C, &cg) ? -2 : 0;
    if (rc == 0) {
        memcpy(C.u, uc, sizeof(double) * 2 * C.N);
        memcpy(F.u, uf, sizeof(double) * 2 * F.N);
        prolong_add(&C, &F);
        memcpy(uf, F.u, sizeof(double) * 2 * F.N);
    }
    free_level(&F);
    free_level(&C);
    return rc;
}
