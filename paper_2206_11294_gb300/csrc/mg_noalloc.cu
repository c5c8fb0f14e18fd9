// mg_residual_norms_noalloc: the per-field stopping norms ||D^-1 r||_2 of a
// state x, computed straight from the caller's coefficient arrays without any
// device allocation.
//
// Who needs it: callers whose device memory is owned entirely by another
// allocator (a framework's caching allocator, a fixed arena sized up front) or
// whose time-stepping loop must not call cudaMalloc/cudaFree, which can
// synchronise the whole device.  Such callers cannot create an mg_handle (its
// hierarchy is device memory) just to monitor a residual.
//
// Scratch: the per-block partial sums live in the file-scope array below
// (1 MiB on each device, held until the process exits; with lazy module
// loading the array and the kernels are loaded on the first call on that
// device).  Host code must not pass the array's name to a kernel (in host
// code it is only a stand-in symbol); its device address is looked up with
// cudaGetSymbolAddress by the first call made while that device is current.
#include <mutex>
#include <string>

#include "coupledmg.h"
#include "mg_host.h"
#include "mg_types.cuh"

namespace cmg {
namespace {

constexpr int kNA_BX = 32, kNA_BY = 8;      // cells per block: 32 x 8 (x 1 in z)
constexpr int kNoAllocMaxBlocks = 65536;   // at most 16,777,216 cells
constexpr int kMaxDevices = 64;

// Block-wide sums of two values in a fixed order (result in thread 0).
__device__ __forceinline__ void na_block_sum2(double &a, double &b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    __shared__ double sa[32], sb[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, w = tid >> 5;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = (nthr + 31) >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Sums the n partials in a fixed order; out[0..1] = square roots.
__global__ void __launch_bounds__(256) k_na_reduce(const double2 *__restrict__ partial, int n,
                                                   double *__restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        a += partial[q].x;
        b += partial[q].y;
    }
    na_block_sum2(a, b);
    if (threadIdx.x == 0) {
        out[0] = sqrt(a);
        out[1] = sqrt(b);
    }
}

static __device__ __align__(256) double2 g_norm_scratch[kNoAllocMaxBlocks];

std::mutex g_addr_mutex;
double2 *g_addr[kMaxDevices] = {};

struct RawGeom {
    int n[3];
    int axisym;
    double r0, h;
    int dir[3][2];          // Dirichlet sides
    double gT[3][2], gp[3][2];
};

// rho_f of a face normal to axis a of cell column i: r_f on r-faces, r_i on
// z-faces (axisymmetric); 1 on Cartesian grids.  G_f = c_f rho_f / h^2.
__device__ __forceinline__ double face_rho(const RawGeom &g, int a, int i, int fi) {
    if (!g.axisym) return 1.0;
    return a == 0 ? g.r0 + fi * g.h : g.r0 + (i + 0.5) * g.h;
}

// Variant of k_norm_partials that reads the caller's raw inputs (lambda,
// 1/rho and k on faces, rhs, x) and builds each cell's rows of Eqs. 27-28 on
// the fly; partial sums go to the static scratch array.
template <int DIM>
__global__ void __launch_bounds__(kNA_BX * kNA_BY) k_norm_partials_raw(RawGeom g, const double *__restrict__ lam,
                                                               const double *__restrict__ fa0,
                                                               const double *__restrict__ fa1,
                                                               const double *__restrict__ fa2,
                                                               const double *__restrict__ fk0,
                                                               const double *__restrict__ fk1,
                                                               const double *__restrict__ fk2,
                                                               const double2 *__restrict__ rhs,
                                                               const double2 *__restrict__ x,
                                                               double2 *__restrict__ partial) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    double zT2 = 0.0, zp2 = 0.0;
    if (i < g.n[0] && j < g.n[1]) {
        const int n0 = g.n[0], n1 = g.n[1];
        const long long c = cell_id(i, j, k, n0, n1);
        const double2 xc = x[c];
        const double ih2 = 1.0 / (g.h * g.h);
        double lapT = 0.0, lapp = 0.0, sigT = 0.0, sigp = 0.0;
        const int pos[3] = {i, j, k};
        const double *fa[3] = {fa0, fa1, fa2};
        const double *fk[3] = {fk0, fk1, fk2};
#pragma unroll
        for (int a = 0; a < DIM; a++) {
            int m[3] = {n0, n1, g.n[2]};
            m[a] += 1;
#pragma unroll
            for (int side = 0; side < 2; side++) {
                int f[3] = {i, j, k};
                f[a] += side;
                const long long fid = (long long)f[0] + (long long)m[0] * ((long long)f[1] + (long long)m[1] * f[2]);
                const int nbpos = pos[a] + (side ? 1 : -1);
                const double w = face_rho(g, a, i, f[0]) * ih2;
                if (nbpos >= 0 && nbpos < g.n[a]) {
                    int nb[3] = {i, j, k};
                    nb[a] = nbpos;
                    const double2 u = x[cell_id(nb[0], nb[1], nb[2], n0, n1)];
                    const double GT = fk[a][fid] * w, Gp = fa[a][fid] * w;
                    lapT += GT * (u.x - xc.x);
                    lapp += Gp * (u.y - xc.y);
                    sigT += GT;
                    sigp += Gp;
                } else if (g.dir[a][side]) {
                    const double GT = 2.0 * fk[a][fid] * w, Gp = 2.0 * fa[a][fid] * w;
                    lapT += GT * (g.gT[a][side] - xc.x);
                    lapp += Gp * (g.gp[a][side] - xc.y);
                    sigT += GT;
                    sigp += Gp;
                }
            }
        }
        const double s = g.axisym ? g.r0 + (i + 0.5) * g.h : 1.0;
        const double l1 = lam[4 * c], l2 = lam[4 * c + 1], l3 = lam[4 * c + 2], l4 = lam[4 * c + 3];
        const double2 bb = rhs[c];
        // residual of the s-scaled rows (Eqs. 27-28)
        const double rT = s * bb.x - (lapT + s * (l1 * xc.x + l2 * xc.y));
        const double rp = s * bb.y - (lapp + s * l3 * xc.y + l4 * lapT);
        // the cell's 2x2 block and D^-1 r
        const double Da = s * l1 - sigT, Db = s * l2, Dc = -l4 * sigT, Dd = s * l3 - sigp;
        const double det = Da * Dd - Db * Dc;
        const double zT = (Dd * rT - Db * rp) / det;
        const double zp = (Da * rp - Dc * rT) / det;
        zT2 = zT * zT;
        zp2 = zp * zp;
    }
    na_block_sum2(zT2, zp2);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = make_double2(zT2, zp2);
}

mg_status scratch_address(double2 **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(MG_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess || !p)
            return set_error(MG_ERR_CUDA, (std::string("cudaGetSymbolAddress of the norm scratch failed: ") +
                                           cudaGetErrorString(e)).c_str());
        g_addr[dev] = static_cast<double2 *>(p);
    }
    *out = g_addr[dev];
    return MG_OK;
}

bool misaligned(const void *p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

}  // namespace
}  // namespace cmg

using namespace cmg;

extern "C" mg_status mg_residual_norms_noalloc(const mg_grid *grid, const double *lambda,
                                               const double *const face_alpha[3], const double *const face_k[3],
                                               const double *rhs, const double *x, double *out, void *stream) {
    if (!grid || !lambda || !face_alpha || !face_k || !rhs || !x || !out)
        return set_error(MG_ERR_INVALID_ARG, "NULL argument");
    // the grid rules of mg_create: dimensions, spacing, boundary kinds and values
    const mg_status gst = check_grid_geom(grid);
    if (gst) return gst;
    const int dim = grid->dim;
    for (int a = 0; a < dim; a++)
        if (!face_alpha[a] || !face_k[a]) return set_error(MG_ERR_INVALID_ARG, "NULL face array");
    if (misaligned(rhs, 16) || misaligned(x, 16) || misaligned(lambda, 8) || misaligned(out, 8))
        return set_error(MG_ERR_INVALID_ARG, "device arrays misaligned (pairs need 16 bytes)");
    const dim3 block(kNA_BX, kNA_BY, 1);
    const dim3 gridd((grid->n[0] + kNA_BX - 1) / kNA_BX, (grid->n[1] + kNA_BY - 1) / kNA_BY,
                     dim == 3 ? grid->n[2] : 1);
    const long long nblocks = (long long)gridd.x * gridd.y * gridd.z;
    if (grid->n[1] > 8 * 65535 || grid->n[2] > 65535 || nblocks > kNoAllocMaxBlocks)
        return set_error(MG_ERR_INVALID_ARG,
                         ("grid needs " + std::to_string(nblocks) + " blocks of 32x8 cells; the allocation-free "
                          "norm holds partial sums for at most " + std::to_string(kNoAllocMaxBlocks) +
                          " (16,777,216 cells as 256^3 or 4096^2)").c_str());
    RawGeom g;
    for (int a = 0; a < 3; a++) g.n[a] = grid->n[a];
    g.axisym = grid->axisym;
    g.r0 = grid->r0;
    g.h = grid->h;
    for (int a = 0; a < 3; a++)
        for (int s = 0; s < 2; s++) {
            g.dir[a][s] = (a < dim && grid->bc[a][s] == MG_BC_DIRICHLET) ? 1 : 0;
            g.gT[a][s] = grid->bc_T[a][s];
            g.gp[a][s] = grid->bc_p[a][s];
        }
    double2 *scratch = nullptr;
    mg_status st = scratch_address(&scratch);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double *f2a = dim == 3 ? face_alpha[2] : face_alpha[0];
    const double *f2k = dim == 3 ? face_k[2] : face_k[0];
    if (dim == 2)
        k_norm_partials_raw<2><<<gridd, block, 0, s>>>(g, lambda, face_alpha[0], face_alpha[1], f2a, face_k[0],
                                                       face_k[1], f2k, reinterpret_cast<const double2 *>(rhs),
                                                       reinterpret_cast<const double2 *>(x), scratch);
    else
        k_norm_partials_raw<3><<<gridd, block, 0, s>>>(g, lambda, face_alpha[0], face_alpha[1], f2a, face_k[0],
                                                       face_k[1], f2k, reinterpret_cast<const double2 *>(rhs),
                                                       reinterpret_cast<const double2 *>(x), scratch);
    k_na_reduce<<<1, 256, 0, s>>>(scratch, (int)nblocks, out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(MG_ERR_CUDA, cudaGetErrorString(e));
    return MG_OK;
}
