// Device-side types of the coupled p-T multigrid (sm_103a).
//
// Every level stores Eqs. 27-28 with each cell's two rows multiplied by
// s_i = V_i / h^dim (1 on Cartesian grids, r_i on axisymmetric ones):
//
//   T-row:  sum_f G^T_f (T_nb - T_i) + s l1 T_i + s l2 p_i              = s lambda_T
//   p-row:  sum_f G^p_f (p_nb - p_i) + s l3 p_i + l4 sum_f G^T_f (T_nb - T_i) = s lambda_p
//
// The scaling makes every face coefficient G_f = c_f * rho_f / h^2 the same
// for both cells of the face (rho_f = r_f on r-faces, r_i on z-faces, 1 on
// Cartesian grids), so restriction becomes a plain average of children and
// face coefficients coarsen by a plain sum.  Boundary faces carry G = 0
// (wall, axis) or twice the interior value (Dirichlet: the boundary value
// sits h/2 away); their Dirichlet data move to the right-hand side once.
//
// Per level and cell:
//   x, b      pair (T, p)                      R2  (double2 / float2)
//   D         the 2x2 block of (T_i, p_i) in the cell's two rows:
//             [[s l1 - sum G^T, s l2], [-l4 sum G^T, s l3 - sum G^p]]
//   Dinv      its inverse                      R4  (row-major 2x2)
//   l4        the p-row's weight of the T-Laplacian (Eq. 32)
//   W         Dinv [[1, 0], [l4, 1]]: a cell's update from its neighbour sums
//   bt        Dinv b, formed once per right-hand side
// so that a Gauss-Seidel update is  x_i = bt_i - W_i (sT, sp)  with sT, sp the
// plain neighbour sums of the T- and p-Laplacians.
// Per face, one array per axis:
//   G         (G^T, G^p) = (k, 1/rho) times rho_f / h^2 times the boundary factor
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cmg {

struct __align__(32) dq { double a, b, c, d; };   // 2x2 block, row-major
struct __align__(16) fq { float a, b, c, d; };

template <typename R> struct Vec;
template <> struct Vec<double> { using v2 = double2; using q4 = dq; };
template <> struct Vec<float>  { using v2 = float2;  using q4 = fq; };

template <typename R>
struct Level {
    int n0, n1, n2;                 // cells per axis (n2 = 1 in 2D)
    long long N;                    // cells
    typename Vec<R>::v2 *x;         // unknowns (T, p)
    typename Vec<R>::v2 *b;         // right-hand side of this level
    const typename Vec<R>::v2 *G0, *G1, *G2;   // face coefficients, axes 0..2
    const typename Vec<R>::q4 *D, *Dinv;
    const R *l4;
    const typename Vec<R>::q4 *W;   // Dinv [[1, 0], [l4, 1]]
    typename Vec<R>::v2 *bt;        // Dinv b
    // FP32 levels of mixed precision: the same level's FP64 W and Dinv b.  A
    // cell whose FP32 W has a NaN first entry (set at set-up for cells at a
    // large coefficient jump) is updated with these, in FP64.
    const dq *W64;
    double2 *bt64;
    // Finest level of mixed precision: 1 for those cells (the FP64 residual
    // then stores their Dinv r in FP64); NULL elsewhere.
    const unsigned char *jflag;
};

// Dirichlet flags per axis and side (prolongation ghost signs).
struct BcFlags {
    int dir[3][2];
};

__host__ __device__ inline long long cell_id(int i, int j, int k, int n0, int n1) {
    return (long long)i + (long long)n0 * ((long long)j + (long long)n1 * k);
}

}  // namespace cmg
