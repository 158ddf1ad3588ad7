// The Galerkin projection applied as G* = D (D^H D)^-1 D^H, row by row.
//
// For each tensor row i the compatible projection of Sec. 2.2 (Eqs.
// eql_discrete2, linequil2ast) is (G X)_ij = D_j sum_l conj(D_l) X_il /
// sum_m |D_m|^2, with D the rotated-scheme derivative of App. A (Eq. kas).
// That derivative is, by construction, a finite difference: up to 1/(4h),
//   (D_j f)(n)   = sum_{a in {0,1}^3} s_j(a) f(n + a),
//   (D_j^T g)(n) = sum_{a in {0,1}^3} s_j(a) g(n - a),   s_j(a) = +1 if a_j = 1 else -1,
// so the projection is a divergence stencil (9 fields -> 3), a scalar Laplace
// solve in Fourier space (3 fields instead of 9: OP_LAPINV, which also
// carries the two 1/(4h) factors), and a gradient stencil (3 -> 9), plus the
// zero mode of the mixed control (the stress-controlled components of the
// mean are kept).  Identical to the Fourier-space projection up to round-off.
#include "common.cuh"
#include "rve_internal.h"

namespace {

// 32-bit voxel indexing (grids up to 512^3 = 2^27 voxels)
struct Grid3 {
  int n0, n1, n2;
  unsigned nvox;
};

__device__ __forceinline__ void coords(const Grid3& g, unsigned v, int& x, int& y, int& z) {
  const unsigned plane = (unsigned)g.n0 * (unsigned)g.n1;
  z = (int)(v / plane);
  const unsigned r = v - (unsigned)z * plane;
  y = (int)(r / (unsigned)g.n0);
  x = (int)(r - (unsigned)y * (unsigned)g.n0);
}

// voxel indices of the 8 corners n + sgn * a, a in {0,1}^3 (corner index a0 + 2 a1 + 4 a2)
__device__ __forceinline__ void corners(const Grid3& g, int x, int y, int z, int sgn, unsigned* m) {
  int xs = x + sgn, ys = y + sgn, zs = z + sgn;
  xs = xs < 0 ? xs + g.n0 : (xs >= g.n0 ? xs - g.n0 : xs);
  ys = ys < 0 ? ys + g.n1 : (ys >= g.n1 ? ys - g.n1 : ys);
  zs = zs < 0 ? zs + g.n2 : (zs >= g.n2 ? zs - g.n2 : zs);
  const unsigned r00 = (unsigned)g.n0 * ((unsigned)y + (unsigned)g.n1 * (unsigned)z);
  const unsigned r10 = (unsigned)g.n0 * ((unsigned)ys + (unsigned)g.n1 * (unsigned)z);
  const unsigned r01 = (unsigned)g.n0 * ((unsigned)y + (unsigned)g.n1 * (unsigned)zs);
  const unsigned r11 = (unsigned)g.n0 * ((unsigned)ys + (unsigned)g.n1 * (unsigned)zs);
  m[0] = r00 + x; m[1] = r00 + xs; m[2] = r10 + x; m[3] = r10 + xs;
  m[4] = r01 + x; m[5] = r01 + xs; m[6] = r11 + x; m[7] = r11 + xs;
}

// (D_0 f, D_1 f, D_2 f) from the 8 corner values, without the 1/(4h) factor
__device__ __forceinline__ void corner_diffs(const double* c, double* d) {
  const double p00 = c[0] + c[4], p10 = c[1] + c[5], p01 = c[2] + c[6], p11 = c[3] + c[7];  // pairs along z
  d[0] = (p10 + p11) - (p00 + p01);
  d[1] = (p01 + p11) - (p00 + p10);
  d[2] = ((c[4] - c[0]) + (c[5] - c[1])) + ((c[6] - c[2]) + (c[7] - c[3]));
}

// d_i = sum_l D_l^T X_il (unscaled); partial sums of the 9 input fields for their means
__global__ void __launch_bounds__(RVE_RED_THREADS) k_div(Grid3 g, const double* __restrict__ X, double* __restrict__ d,
                                                         double* __restrict__ ds, double* __restrict__ partial,
                                                         unsigned int* __restrict__ ticket, int check_done) {
  __shared__ double sh[32];
  if (check_done && ds[DS_DONE] != 0.0) return;
  double mean[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) mean[c] = 0.0;
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nvox; v += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(g, v, x, y, z);
    unsigned m[8];
    corners(g, x, y, z, -1, m);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double* f = X + (size_t)(3 * i + l) * g.nvox;
        double c[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) c[a] = __ldg(f + m[a]);
        mean[3 * i + l] += c[0];
        // D_l^T at n: corners n - a weighted +1 where a_l = 1, -1 where a_l = 0
        double dd[3];
        corner_diffs(c, dd);
        acc += dd[l];
      }
      d[(size_t)i * g.nvox + v] = acc;
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const double s = blk_sum(mean[c], sh);
    if (threadIdx.x == 0) partial[(size_t)c * gridDim.x + blockIdx.x] = s;
  }
  double tot[9];
  if (last_block_sums(partial, 9, ticket, sh, tot) && threadIdx.x == 0) {
    for (int c = 0; c < 9; ++c) ds[DS_XMEAN + c] = tot[c] / (double)g.nvox;
  }
}

struct ZeroMode {
  double add[9];      // keep_ij * (-shift_ij); the kept mean itself is read from ds
  int keep[9];
};

// Y_ij = D_j u_i (unscaled) + keep_ij (mean_ij - shift_ij); partial of sum Y^2 -> ds[DS_NORM]
__global__ void __launch_bounds__(RVE_RED_THREADS) k_grad(Grid3 g, const double* __restrict__ u, double* __restrict__ Y,
                                                          ZeroMode zm, double* __restrict__ ds,
                                                          double* __restrict__ partial, unsigned int* __restrict__ ticket) {
  __shared__ double sh[32];
  double off[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) off[c] = zm.keep[c] ? ds[DS_XMEAN + c] + zm.add[c] : 0.0;
  double acc = 0.0;
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nvox; v += gridDim.x * blockDim.x) {
    int x, y, z;
    coords(g, v, x, y, z);
    unsigned m[8];
    corners(g, x, y, z, +1, m);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* f = u + (size_t)i * g.nvox;
      double c[8], d[3];
#pragma unroll
      for (int a = 0; a < 8; ++a) c[a] = __ldg(f + m[a]);
      corner_diffs(c, d);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double yv = d[j] + off[3 * i + j];
        Y[(size_t)(3 * i + j) * g.nvox + v] = yv;
        acc = fma(yv, yv, acc);
      }
    }
  }
  const double s = blk_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  double tot;
  if (last_block_sums(partial, 1, ticket, sh, &tot) && threadIdx.x == 0) ds[DS_NORM] = tot;
}

// CG step fused with the gradient: q_ij = D_j u_i + keep_ij mean(t_ij);
// x += alpha p; r -= alpha q; rr' = r . r; beta = rr'/rr; iteration count; done test.
__global__ void __launch_bounds__(RVE_RED_THREADS) k_grad_cg(Grid3 g, const double* __restrict__ u, ZeroMode zm,
                                                             double* __restrict__ x, double* __restrict__ r,
                                                             const double* __restrict__ p, double* __restrict__ ds,
                                                             double* __restrict__ partial,
                                                             unsigned int* __restrict__ ticket) {
  __shared__ double sh[32];
  if (ds[DS_DONE] != 0.0) return;
  const double alpha = ds[DS_ALPHA];
  double off[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) off[c] = zm.keep[c] ? ds[DS_XMEAN + c] : 0.0;
  double acc = 0.0;
  for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < g.nvox; v += gridDim.x * blockDim.x) {
    int xx, yy, zz;
    coords(g, v, xx, yy, zz);
    unsigned m[8];
    corners(g, xx, yy, zz, +1, m);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double* f = u + (size_t)i * g.nvox;
      double c[8], d[3];
#pragma unroll
      for (int a = 0; a < 8; ++a) c[a] = __ldg(f + m[a]);
      corner_diffs(c, d);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const size_t e = (size_t)(3 * i + j) * g.nvox + v;
        const double q = d[j] + off[3 * i + j];
        x[e] = fma(alpha, p[e], x[e]);
        const double rv = fma(-alpha, q, r[e]);
        r[e] = rv;
        acc = fma(rv, rv, acc);
      }
    }
  }
  const double s = blk_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  double tot;
  if (last_block_sums(partial, 1, ticket, sh, &tot) && threadIdx.x == 0) {
    ds[DS_BETA] = tot / ds[DS_RR];
    ds[DS_RR] = tot;
    ds[DS_ITERS] += 1.0;
    if (!(tot > ds[DS_STOP])) ds[DS_DONE] = 1.0;
  }
}

Grid3 grid_of(const rve_s* h) {
  Grid3 g;
  g.n0 = h->n0; g.n1 = h->n1; g.n2 = h->n2;
  g.nvox = (unsigned)h->nvox;
  return g;
}

ZeroMode zero_mode(const uint8_t* mask, const double* shift) {
  ZeroMode z;
  for (int c = 0; c < 9; ++c) {
    z.keep[c] = mask[c] ? 0 : 1;
    z.add[c] = (z.keep[c] && shift) ? -shift[c] : 0.0;
  }
  return z;
}

}  // namespace

cudaError_t launch_div(const rve_s* h, const double* X, double* d, int check_done, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    k_div<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(grid_of(h), X, d, h->dscal, h->partial,
                                                     (unsigned int*)(h->dcount + 4), check_done);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad(const rve_s* h, const double* u, double* Y, const uint8_t* mask, const double* shift,
                        cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    k_grad<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(grid_of(h), u, Y, zero_mode(mask, shift), h->dscal,
                                                      h->partial, (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_cg(const rve_s* h, const double* u, const uint8_t* mask, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    k_grad_cg<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(grid_of(h), u, zero_mode(mask, nullptr), h->x, h->r, h->p,
                                                         h->dscal, h->partial, (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}
