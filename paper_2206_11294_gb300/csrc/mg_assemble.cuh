// The steps on either side of the solve, per cell on the device (FP64).
//
// Before it (k_assemble): from the advected state of a time step (Eq. Yadv:
// volume fraction C, partial densities m_i = C_i rho_i, averaged total energy,
// averaged momentum, face velocities u*) the pressure p^(adv) by the mixture's
// NASG equation of state (Eq. 20), the temperature T^(adv) (Eq. 23), the
// thermal dilation (Eq. 10) and sound speed (Eq. 11) of each phase, the
// coefficients lambda_1..lambda_4, lambda_T, lambda_p (Eqs. 29-34) and the face
// coefficients 1/rho and k that mg_set_coeffs and mg_solve take.
//
// After it (k_correct): the face velocity u^{n+1} = u* - dt (1/rho)_f grad p
// (Eq. unp1) with the solve operator's face gradients, and the phase pressures
// p_1 = p + (1 - C) sigma kappa, p_2 = p - C sigma kappa (Eqs. 37-38).
//
// Overlines are volume-fraction averages of the phase expressions, written in
// the partial densities: C_i (1 - rho_i b_i) = C_i - m_i b_i, C_i rho_i q_i =
// m_i q_i, C_i / rho_i = C_i^2 / m_i, so pure cells need no special case; a
// phase with C_i = 0 contributes nothing.
#pragma once
#include "mg_types.cuh"

namespace cmg {

// Per-phase constants, derived on the host from the NASG parameters.
struct PhaseK {
    double Gamma, Pi, b, q, cp, k;
    double shift;          // Gamma Pi / (Gamma - 1)
    double inv_g1;         // 1 / (Gamma - 1)
    double cpcv;           // c_p - c_v
    double g1cv;           // (Gamma - 1) c_v          (Eq. 10)
    double gam_over_G;     // gamma / Gamma, gamma = c_p / c_v
    double inv_cp;         // 1 / c_p
};

struct AssembleArgs {
    int n[3];
    int axisym;
    double r0, h, inv_h;
    double inv_dt, inv_dt2, l4_scale;   // l4_scale: 1/dt (restored lambda_4) or 1 (as printed)
    int harmonic_k;                     // face k: 2 k_L k_R / (k_L + k_R) of the cells' mixture k, else C_f-weighted
    PhaseK ph[2];
    const double *C, *m1, *m2, *E;
    const double *mom[3];
    const double *uf[3];
    double2 *lam;          // [N][2 pairs]: (l1, l2), (l3, l4)
    double2 *rhs;          // [N]: (lambda_T, lambda_p)
    double2 *x0;           // [N]: (T, p) or NULL
    double *fa[3], *fk[3];
};

__device__ __forceinline__ long long face_index(const int n[3], int a, int i, int j, int k) {
    const long long n0 = n[0] + (a == 0), n1 = n[1] + (a == 1);
    return (long long)i + n0 * ((long long)j + n1 * k);
}

// One phase's share of the lambda averages at (T, p): beta C_i, the bracket of
// Eq. 8 times C_i, and beta / (rho c_p) times C_i.
__device__ __forceinline__ void phase_terms(const PhaseK &P, double Ci, double mi, double T, double p, double &beta_c,
                                            double &bracket_c, double &bover_c) {
    const double beta = P.g1cv / (P.g1cv * T + P.b * (p + P.Pi));       // Eq. 10
    if (!(Ci > 0.0)) {
        beta_c = bracket_c = bover_c = 0.0;
        return;
    }
    // C_i gamma / (rho_i c_i^2) with c_i^2 of Eq. 11: gamma (C_i - m_i b_i) / (Gamma (p + Pi))
    const double comp = P.gam_over_G * (Ci - mi * P.b) / (p + P.Pi);
    const double c_over_rho = Ci * Ci / mi;                              // C_i / rho_i
    const double bcp = beta * c_over_rho * P.inv_cp;                     // C_i beta / (rho_i c_p)
    beta_c = Ci * beta;
    bracket_c = comp - beta * T * bcp;
    bover_c = bcp;
}

template <int DIM, bool AXI>
__global__ void __launch_bounds__(256) k_assemble(const __grid_constant__ AssembleArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const int n0 = A.n[0], n1 = A.n[1];
    const long long c = (long long)i + (long long)n0 * ((long long)j + (long long)n1 * k);
    const double C = A.C[c], m1 = A.m1[c], m2 = A.m2[c], E = A.E[c];
    const double C2 = 1.0 - C;
    const double rho = m1 + m2;
    double mm = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const double u = A.mom[a][c];
        mm = a == 0 ? u * u : mm + u * u;
    }
    const double kinetic = 0.5 * mm / rho;
    const PhaseK &P1 = A.ph[0], &P2 = A.ph[1];
    const double free1 = C - m1 * P1.b, free2 = C2 - m2 * P2.b;
    // Eq. 20
    const double shift = (P1.shift * free1 + m1 * P1.q) + (P2.shift * free2 + m2 * P2.q);
    const double denom = free1 * P1.inv_g1 + free2 * P2.inv_g1;
    const double p = (E - kinetic - shift) / denom;
    // Eq. 23
    const double T = ((free1 * p + P1.Pi * free1) + (free2 * p + P2.Pi * free2)) / (m1 * P1.cpcv + m2 * P2.cpcv);
    double b1, k1, o1, b2, k2, o2;
    phase_terms(P1, C, m1, T, p, b1, k1, o1);
    phase_terms(P2, C2, m2, T, p, b2, k2, o2);
    const double rho_cp = m1 * P1.cp + m2 * P2.cp;
    // div u* (axisymmetric r-faces weighted by r_f / r_i)
    double div = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int pos[3] = {i, j, k};
        const long long flo = face_index(A.n, a, i, j, k);
        const long long fhi = face_index(A.n, a, pos[0] + (a == 0), pos[1] + (a == 1), pos[2] + (a == 2));
        const double ulo = A.uf[a][flo], uhi = A.uf[a][fhi];
        double t;
        if (AXI && a == 0) {
            const double ri = A.r0 + (i + 0.5) * A.h;
            t = ((ri + 0.5 * A.h) * uhi - (ri - 0.5 * A.h) * ulo) / (ri * A.h);
        } else {
            t = (uhi - ulo) * A.inv_h;
        }
        div = a == 0 ? t : div + t;
    }
    const double l1 = -rho_cp * A.inv_dt;                 // Eq. 29
    const double l2 = (b1 + b2) * T * A.inv_dt;           // Eq. 30
    const double l3 = -(k1 + k2) * A.inv_dt2;             // Eq. 31
    const double l4 = (o1 + o2) * A.l4_scale;             // Eq. 32
    A.lam[2 * c] = make_double2(l1, l2);
    A.lam[2 * c + 1] = make_double2(l3, l4);
    A.rhs[c] = make_double2(l1 * T + l2 * p, l3 * p + div * A.inv_dt);   // Eqs. 33-34
    if (A.x0) A.x0[c] = make_double2(T, p);
    // faces owned by this cell: the low face of each axis, and the high face on the high boundary
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int pos[3] = {i, j, k};
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            const int fpos = pos[a] + sd;
            if (sd == 1 && fpos != A.n[a]) continue;
            const bool edge = fpos == 0 || fpos == A.n[a];
            const long long cn = edge ? c : c - (a == 0 ? 1LL : a == 1 ? (long long)n0 : (long long)n0 * n1);
            const double Cn = edge ? C : A.C[cn];
            const double rf = edge ? rho : 0.5 * (rho + (A.m1[cn] + A.m2[cn]));
            double kf;
            if (A.harmonic_k) {                     // uniform over the launch
                const double kc = C * P1.k + C2 * P2.k, kn = Cn * P1.k + (1.0 - Cn) * P2.k;
                kf = edge ? kc : 2.0 * kn * kc / (kn + kc);      // series conduction through the two half cells
            } else {
                const double Cf = edge ? C : 0.5 * (C + Cn);
                kf = Cf * P1.k + (1.0 - Cf) * P2.k;
            }
            const long long f = face_index(A.n, a, pos[0] + (a == 0 ? sd : 0), pos[1] + (a == 1 ? sd : 0),
                                           pos[2] + (a == 2 ? sd : 0));
            A.fa[a][f] = 1.0 / rf;
            A.fk[a][f] = kf;
        }
    }
}

struct CorrectArgs {
    int n[3];
    int dir[3][2];           // Dirichlet faces
    double gp[3][2];         // their pressure values
    double dt, inv_h, two_inv_h, sigma;
    const double2 *x;        // [N] (T, p)
    const double *C, *kappa;
    const double *fa[3], *uf[3];
    double *uo[3];
    double *p1, *p2;
};

template <int DIM>
__global__ void __launch_bounds__(256) k_correct(const __grid_constant__ CorrectArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const int n0 = A.n[0], n1 = A.n[1];
    const long long c = (long long)i + (long long)n0 * ((long long)j + (long long)n1 * k);
    const double p = A.x[c].y;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int pos[3] = {i, j, k};
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            const int fpos = pos[a] + sd;
            if (sd == 1 && fpos != A.n[a]) continue;
            double g;
            if (fpos == 0) {
                g = A.dir[a][0] ? (p - A.gp[a][0]) * A.two_inv_h : 0.0;     // towards the low boundary value
            } else if (fpos == A.n[a]) {
                g = A.dir[a][1] ? (A.gp[a][1] - p) * A.two_inv_h : 0.0;
            } else {
                const long long cn = c - (a == 0 ? 1LL : a == 1 ? (long long)n0 : (long long)n0 * n1);
                g = (p - A.x[cn].y) * A.inv_h;
            }
            const long long f = face_index(A.n, a, pos[0] + (a == 0 ? sd : 0), pos[1] + (a == 1 ? sd : 0),
                                           pos[2] + (a == 2 ? sd : 0));
            A.uo[a][f] = A.uf[a][f] - A.dt * A.fa[a][f] * g;
        }
    }
    const double sk = A.sigma * A.kappa[c];
    const double Cc = A.C[c];
    A.p1[c] = p + (1.0 - Cc) * sk;
    A.p2[c] = p - Cc * sk;
}

// ---------------------------------------------------------------- Eq. 39
// Phase total energies at the end of the step: (C_i rho_i e_T,i)^{n+1} =
// (C_i rho_i e_T,i)^(adv) + dt C_i div F_i, with the face flux of axis a
//   F_i = -p_i,f u_f + mu_i (S . u)_{a,f} + k_i (dT/dx_a)_f,   S = grad u + grad u^T.
// Cell velocities are the means of their two face velocities; on a face the
// normal velocity is the face's own, the tangential ones and p_i the means of
// the two cells, the normal derivatives the difference across the face and the
// tangential derivatives the mean of the two cells' (central, one-sided in the
// first and last cell).  Walls and the axis carry no flux; a Dirichlet face
// carries -g_p u_f + k_i 2 (g_T - T)/h towards the boundary value.
//
// A block computes every face flux of its tile into shared memory through one
// code path (faces on the tile's edge are computed by both blocks that share
// them, by the same instructions on the same inputs, so both get the same
// bits), then each cell takes the divergence.  The update is conservative:
// summed over the cells with their volumes, (E_i^{n+1} - E_i) / (dt C_i)
// telescopes to the fluxes through the boundary faces.
struct EnergyArgs {
    int n[3];
    int dir[3][2];                 // Dirichlet faces
    double gT[3][2], gp[3][2];     // their values
    double r0, h, inv_h, half_inv_h, two_inv_h, dt;
    double k[2], mu[2];
    const double2 *x;              // [N] (T, p)
    const double *C, *p1, *p2;
    const double *uf[3];
    const double *E1, *E2;
    double *E1o, *E2o;
};

// Cell velocities of a block's tile and a one-cell halo (planes k-1..k+1 in 3D), staged in shared memory: the
// mean of each cell's two faces of each axis.  Every cell an interior face flux of the tile reads - its two cells
// and their neighbours for the tangential derivatives - lies in this region; staged cells outside the grid hold 0
// and are never read (derivatives are clamped to the grid).
template <int DIM, int TX, int TY>
struct EnergyTile {
    static constexpr int SX = TX + 2, SY = TY + 2, SZ = DIM == 3 ? 3 : 1, NS = SX * SY * SZ;
    int i0, j0, k0;
    const double *U;                 // [DIM][NS]
    __device__ __forceinline__ double u(int q, int i, int j, int k) const {
        return U[q * NS + (i - i0 + 1) + SX * ((j - j0 + 1) + SY * (DIM == 3 ? k - k0 + 1 : 0))];
    }
};

// d u_a / d x_b at a cell from the staged velocities: central inside, one-sided in the first and last cell.
template <int DIM, int TX, int TY>
__device__ __forceinline__ double cell_du(const EnergyArgs &A, const EnergyTile<DIM, TX, TY> &S, int a, int b,
                                          const int pos[3]) {
    const int nb = A.n[b];
    if (nb < 2) return 0.0;
    int up[3] = {pos[0], pos[1], pos[2]}, dn[3] = {pos[0], pos[1], pos[2]};
    up[b] = pos[b] + 1 < nb ? pos[b] + 1 : pos[b];
    dn[b] = pos[b] > 0 ? pos[b] - 1 : pos[b];
    const double d = S.u(a, up[0], up[1], up[2]) - S.u(a, dn[0], dn[1], dn[2]);
    return d * (up[b] - dn[b] == 2 ? A.half_inv_h : A.inv_h);
}

// (F_1, F_2) on the face of axis a at face position f (f[a] in 0..n[a]).
template <int DIM, int TX, int TY>
__device__ __forceinline__ double2 energy_face_flux(const EnergyArgs &A, const EnergyTile<DIM, TX, TY> &S, int a,
                                                    const int f[3]) {
    const int fa = f[a];
    const double u_f = A.uf[a][face_index(A.n, a, f[0], f[1], f[2])];
    if (fa == 0 || fa == A.n[a]) {
        const int side = fa == 0 ? 0 : 1;
        if (!A.dir[a][side]) return make_double2(0.0, 0.0);
        int c[3] = {f[0], f[1], f[2]};
        if (side) c[a] = fa - 1;
        const double Tb = A.x[(long long)c[0] + (long long)A.n[0] * ((long long)c[1] + (long long)A.n[1] * c[2])].x;
        const double dT = (side == 0 ? Tb - A.gT[a][0] : A.gT[a][1] - Tb) * A.two_inv_h;
        const double pw = -A.gp[a][side] * u_f;
        return make_double2(pw + A.k[0] * dT, pw + A.k[1] * dT);
    }
    int L[3] = {f[0], f[1], f[2]};
    L[a] = fa - 1;
    const int *R = f;
    const long long cl = (long long)L[0] + (long long)A.n[0] * ((long long)L[1] + (long long)A.n[1] * L[2]);
    const long long cr = (long long)R[0] + (long long)A.n[0] * ((long long)R[1] + (long long)A.n[1] * R[2]);
    const double dTdn = (A.x[cr].x - A.x[cl].x) * A.inv_h;
    double visc = 0.0;
#pragma unroll
    for (int b = 0; b < DIM; b++) {
        const double ubL = S.u(b, L[0], L[1], L[2]), ubR = S.u(b, R[0], R[1], R[2]);
        double s, ub;
        if (b == a) {
            s = 2.0 * (ubR - ubL) * A.inv_h;
            ub = u_f;
        } else {
            s = 0.5 * (cell_du<DIM, TX, TY>(A, S, a, b, L) + cell_du<DIM, TX, TY>(A, S, a, b, R)) + (ubR - ubL) * A.inv_h;
            ub = 0.5 * (ubL + ubR);
        }
        visc = b == 0 ? s * ub : visc + s * ub;
    }
    const double pf1 = 0.5 * (A.p1[cl] + A.p1[cr]), pf2 = 0.5 * (A.p2[cl] + A.p2[cr]);
    return make_double2(-pf1 * u_f + A.mu[0] * visc + A.k[0] * dTdn, -pf2 * u_f + A.mu[1] * visc + A.k[1] * dTdn);
}

template <int DIM, bool AXI, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_energy(const __grid_constant__ EnergyArgs A) {
    constexpr int NX = (TX + 1) * TY, NY = TX * (TY + 1), NZ = DIM == 3 ? 2 * TX * TY : 0;
    using Tile = EnergyTile<DIM, TX, TY>;
    __shared__ double2 F[NX + NY + NZ];
    __shared__ double U[DIM * Tile::NS];
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k = DIM == 3 ? (int)blockIdx.z : 0;
    const int tid = threadIdx.x + TX * threadIdx.y;
    for (int t = tid; t < DIM * Tile::NS; t += TX * TY) {
        const int q = t / Tile::NS, v = t - q * Tile::NS;
        const int si = v % Tile::SX, sj = (v / Tile::SX) % Tile::SY, sk = v / (Tile::SX * Tile::SY);
        const int ci = i0 - 1 + si, cj = j0 - 1 + sj, ck = DIM == 3 ? k - 1 + sk : 0;
        double val = 0.0;
        if (ci >= 0 && ci < A.n[0] && cj >= 0 && cj < A.n[1] && ck >= 0 && ck < A.n[2]) {
            const long long f = face_index(A.n, q, ci, cj, ck);
            const long long st = q == 0 ? 1LL : q == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1];
            val = 0.5 * (A.uf[q][f] + A.uf[q][f + st]);
        }
        U[t] = val;
    }
    __syncthreads();
    const Tile S{i0, j0, k, U};
    for (int t = tid; t < NX + NY + NZ; t += TX * TY) {
        int a, f[3];
        if (t < NX) {
            a = 0;
            f[0] = i0 + t % (TX + 1);
            f[1] = j0 + t / (TX + 1);
            f[2] = k;
        } else if (t < NX + NY) {
            const int u = t - NX;
            a = 1;
            f[0] = i0 + u % TX;
            f[1] = j0 + u / TX;
            f[2] = k;
        } else {
            const int u = t - NX - NY;
            a = 2;
            f[0] = i0 + u % TX;
            f[1] = j0 + (u / TX) % TY;
            f[2] = k + u / (TX * TY);
        }
        bool in = true;
#pragma unroll
        for (int b = 0; b < 3; b++) in = in && f[b] < A.n[b] + (b == a);
        F[t] = in ? energy_face_flux<DIM, TX, TY>(A, S, a, f) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int li = threadIdx.x, lj = threadIdx.y, i = i0 + li, j = j0 + lj;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const long long c = (long long)i + (long long)A.n[0] * ((long long)j + (long long)A.n[1] * k);
    double2 lo[3], hi[3];
    lo[0] = F[lj * (TX + 1) + li];
    hi[0] = F[lj * (TX + 1) + li + 1];
    lo[1] = F[NX + lj * TX + li];
    hi[1] = F[NX + (lj + 1) * TX + li];
    if (DIM == 3) {
        lo[2] = F[NX + NY + lj * TX + li];
        hi[2] = F[NX + NY + TX * TY + lj * TX + li];
    }
    double d1 = 0.0, d2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        double t1, t2;
        if (AXI && a == 0) {
            const double ri = A.r0 + (i + 0.5) * A.h;
            const double wl = ri - 0.5 * A.h, wh = ri + 0.5 * A.h, s = 1.0 / (ri * A.h);
            t1 = (wh * hi[0].x - wl * lo[0].x) * s;
            t2 = (wh * hi[0].y - wl * lo[0].y) * s;
        } else {
            t1 = (hi[a].x - lo[a].x) * A.inv_h;
            t2 = (hi[a].y - lo[a].y) * A.inv_h;
        }
        d1 = a == 0 ? t1 : d1 + t1;
        d2 = a == 0 ? t2 : d2 + t2;
    }
    const double Cc = A.C[c];
    A.E1o[c] = A.E1[c] + A.dt * Cc * d1;
    A.E2o[c] = A.E2[c] + A.dt * (1.0 - Cc) * d2;
}

}  // namespace cmg
