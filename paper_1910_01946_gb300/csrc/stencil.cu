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

// Tiled stencils.  A tile is tx x ty voxels of one z plane (128 threads,
// tx a power of two dividing n0, ty = 128 / tx).  Each thread loads the two
// planes the stencil needs at its position (and the halo threads at the
// one-voxel halo), stores the z-pair sum (or difference) of every field in
// shared memory, and the x/y corner sums then share those partial sums
// between neighbouring voxels: 3 additions per field and voxel instead of 7.
// Blocks loop over tiles, so the grid (and the reduction partials) stay bounded.
constexpr int NT = 128;
constexpr int SMAX = 196;       // max (ty + 1)(tx + 1) over tx in {2, 4, ..., 32}
constexpr int MAX_BLOCKS = 4096;
// k_div reduces the field means per thread at the end: its grid is capped
// (rve_s::div_blocks, four blocks per SM unless the autotuner picks another)
// so that each thread first accumulates several tiles and the reduction is
// amortised

struct Tiling {
  int tx, ty, bx, by, ntiles, nblocks;
};

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// d_i = sum_l D_l^T X_il (unscaled); partial sums of the 9 input fields for
// their means.  V is the field type (double, or float for the mixed-precision
// conjugate gradients); block and grid sums are accumulated in double.
template <typename V>
__global__ void __launch_bounds__(NT) k_div(Grid3 g, Tiling T, const V* __restrict__ X,
                                           V* __restrict__ d, double* __restrict__ ds,
                                           double* __restrict__ partial, unsigned int* __restrict__ ticket,
                                           int check_done, unsigned mean_mask) {
  __shared__ V S[9][SMAX];
  __shared__ double sh[320];
  if (check_done && ds[DS_DONE] != 0.0) return;
  const int W = T.tx + 1;     // row pitch of the staged tile (with its halo)
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int lt = tx + T.tx * ty;
  const int H = T.tx + 1 + T.ty;   // halo: row y0 - 1 (x0 - 1 .. x0 + tx - 1), column x0 - 1
  const unsigned plane = (unsigned)g.n0 * g.n1;
  V mean[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) mean[f] = (V)0;
  for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x) {
    const int bxi = t % T.bx, byi = (t / T.bx) % T.by, z = t / (T.bx * T.by);
    const int x0 = bxi * T.tx, y0 = byi * T.ty;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = y < g.n1;
    const int ym = inside ? y : 0;
    const int zp = wrapi(z - 1, g.n2);
    const unsigned rz = (unsigned)z * plane, rzp = (unsigned)zp * plane;
    const unsigned own = (unsigned)ym * g.n0 + x;
#pragma unroll
    for (int f = 0; f < 9; ++f) {
      const V* F = X + (size_t)f * g.nvox;
      const bool diff = (f % 3) == 2;      // the z-derivative field of each row
      const V a = __ldg(F + rz + own), bm = __ldg(F + rzp + own);
      S[f][(ty + 1) * W + tx + 1] = diff ? bm - a : a + bm;
      if (inside && ((mean_mask >> f) & 1u)) mean[f] += a;
    }
    // the halo is spread over the first H linear threads (whole warps), not
    // given to one lane of every warp: a divergent FP64 instruction costs the
    // pipe as much as a full one
    for (int hh = lt; hh < H; hh += NT) {
      int sidx, gx, gy;
      if (hh <= T.tx) {
        sidx = hh;
        gx = wrapi(x0 - 1 + hh, g.n0);
        gy = wrapi(y0 - 1, g.n1);
      } else {
        const int j = hh - T.tx - 1;
        sidx = (j + 1) * W;
        gx = wrapi(x0 - 1, g.n0);
        gy = (y0 + j < g.n1) ? y0 + j : 0;   // rows past n1 are never a neighbour here
      }
      const unsigned o = (unsigned)gy * g.n0 + gx;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        const V* F = X + (size_t)f * g.nvox;
        const V a = __ldg(F + rz + o), bm = __ldg(F + rzp + o);
        S[f][sidx] = (f % 3) == 2 ? bm - a : a + bm;
      }
    }
    __syncthreads();
    if (inside) {
      const int c11 = (ty + 1) * W + tx + 1;                          // this voxel
      const int c10 = c11 - 1, c01 = c11 - W, c00 = c11 - W - 1;      // x-1, y-1, both
      const unsigned v = rz + (unsigned)y * g.n0 + x;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V* A = S[3 * i];
        const V* B = S[3 * i + 1];
        const V* Cz = S[3 * i + 2];
        const V d0 = (A[c10] + A[c00]) - (A[c11] + A[c01]);
        const V d1 = (B[c01] + B[c00]) - (B[c11] + B[c10]);
        const V d2 = (Cz[c11] + Cz[c10]) + (Cz[c01] + Cz[c00]);
        d[(size_t)i * g.nvox + v] = d0 + d1 + d2;
      }
    }
    __syncthreads();
  }
  double bs[9];
  blk_sums9<V>(mean, mean_mask, sh, bs);       // unselected means: zero partials
  if (tx == 0 && ty == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) partial[(size_t)c * gridDim.x + blockIdx.x] = bs[c];
  }
  double tot[9];
  if (last_block_sums(partial, 9, ticket, sh, tot, mean_mask) && tx == 0 && ty == 0) {
    for (int c = 0; c < 9; ++c) ds[DS_XMEAN + c] = tot[c] / (double)g.nvox;
  }
}

struct ZeroMode {
  double add[9];      // keep_ij * (-shift_ij); the kept mean itself is read from ds
  int keep[9];
};

// Forward gradient of the three potentials, D_j u_i (unscaled), plus the zero
// mode.  CG = false: Y = q, partial of sum Y^2 -> ds[DS_NORM].  CG = true:
// x += alpha p, r -= alpha q, rr' = r . r, beta, iteration count, done test.
template <bool CG, typename V>
__global__ void __launch_bounds__(NT) k_grad_t(Grid3 g, Tiling T, const V* __restrict__ u, ZeroMode zm,
                                              double* __restrict__ Y, V* __restrict__ x,
                                              V* __restrict__ r, const V* __restrict__ p,
                                              double* __restrict__ ds, double* __restrict__ partial,
                                              unsigned int* __restrict__ ticket) {
  __shared__ V SP[3][SMAX], SM[3][SMAX];
  __shared__ double sh[320];
  if (CG && ds[DS_DONE] != 0.0) return;
  const V alpha = CG ? (V)ds[DS_ALPHA] : (V)0;
  V off[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) off[c] = zm.keep[c] ? (V)(ds[DS_XMEAN + c] + zm.add[c]) : (V)0;
  const int W = T.tx + 1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int lt = tx + T.tx * ty;
  const int H = T.tx + 1 + T.ty;
  const unsigned plane = (unsigned)g.n0 * g.n1;
  V acc = (V)0;
  for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x) {
    const int bxi = t % T.bx, byi = (t / T.bx) % T.by, z = t / (T.bx * T.by);
    const int x0 = bxi * T.tx, y0 = byi * T.ty;
    const int xi = x0 + tx, yi = y0 + ty;
    const bool inside = yi < g.n1;
    // high halo: row y0 + ty and column x0 + tx.  When n1 cuts the tile, the
    // +1 neighbour of the last inside row is the first outside thread row,
    // whose threads load row wrap(n1) = 0 (ym), so the halo row is not used.
    const int xh = wrapi(x0 + T.tx, g.n0), yh = (y0 + T.ty) % g.n1, ym = inside ? yi : 0;
    const int zn = wrapi(z + 1, g.n2);
    const unsigned rz = (unsigned)z * plane, rzn = (unsigned)zn * plane;
    const unsigned own = (unsigned)ym * g.n0 + xi;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const V* F = u + (size_t)i * g.nvox;
      const V a = __ldg(F + rz + own), c = __ldg(F + rzn + own);
      SP[i][ty * W + tx] = a + c;
      SM[i][ty * W + tx] = c - a;
    }
    // high halo (row y0 + ty: x0 .. x0 + tx, the last one the corner; column
    // x0 + tx), spread over the first H linear threads
    for (int hh = lt; hh < H; hh += NT) {
      int sidx, gx, gy;
      if (hh <= T.tx) {
        sidx = T.ty * W + hh;
        gx = hh < T.tx ? x0 + hh : xh;
        gy = yh;
      } else {
        const int j = hh - T.tx - 1;
        sidx = j * W + T.tx;
        gx = xh;
        gy = (y0 + j < g.n1) ? y0 + j : 0;   // row n1 wraps to row 0
      }
      const unsigned o = (unsigned)gy * g.n0 + gx;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V* F = u + (size_t)i * g.nvox;
        const V a = __ldg(F + rz + o), c = __ldg(F + rzn + o);
        SP[i][sidx] = a + c;
        SM[i][sidx] = c - a;
      }
    }
    __syncthreads();
    if (inside) {
      const unsigned v = rz + (unsigned)yi * g.n0 + xi;
      const int c00 = ty * W + tx, c10 = c00 + 1, c01 = c00 + W, c11 = c00 + W + 1;   // +x, +y, both
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const V* Pp = SP[i];
        const V* Mm = SM[i];
        const V q0 = (Pp[c10] + Pp[c11]) - (Pp[c00] + Pp[c01]);
        const V q1 = (Pp[c01] + Pp[c11]) - (Pp[c00] + Pp[c10]);
        const V q2 = (Mm[c00] + Mm[c10]) + (Mm[c01] + Mm[c11]);
        const V qv[3] = {q0 + off[3 * i], q1 + off[3 * i + 1], q2 + off[3 * i + 2]};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const size_t e = (size_t)(3 * i + j) * g.nvox + v;
          if (CG) {
            x[e] = fma(alpha, p[e], x[e]);
            const V rv = fma(-alpha, qv[j], r[e]);
            r[e] = rv;
            acc = fma(rv, rv, acc);
          } else {
            Y[e] = (double)qv[j];
            acc = fma(qv[j], qv[j], acc);
          }
        }
      }
    }
    __syncthreads();
  }
  const double s = blk_sum_v<V>(acc, sh);
  if (tx == 0 && ty == 0) partial[blockIdx.x] = s;
  double tot;
  if (last_block_sums(partial, 1, ticket, sh, &tot) && tx == 0 && ty == 0) {
    if (CG) {
      ds[DS_BETA] = tot / ds[DS_RR];
      ds[DS_RR] = tot;
      ds[DS_ITERS] += 1.0;
      if (!(tot > ds[DS_STOP])) ds[DS_DONE] = 1.0;
    } else {
      ds[DS_NORM] = tot;
    }
  }
}

Tiling tiling_of(const rve_s* h) {
  Tiling T;
  int tx = 1;
  while (tx * 2 <= 32 && h->n0 % (tx * 2) == 0) tx *= 2;
  T.tx = tx;
  T.ty = NT / tx;
  T.bx = h->n0 / tx;
  T.by = (h->n1 + T.ty - 1) / T.ty;
  T.ntiles = T.bx * T.by * h->n2;
  T.nblocks = T.ntiles < MAX_BLOCKS ? T.ntiles : MAX_BLOCKS;
  return T;
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

int stencil_tiles(const rve_s* h) { return tiling_of(h).ntiles; }

cudaError_t launch_div(const rve_s* h, const double* X, double* d, int check_done, unsigned mean_mask,
                       cudaStream_t s) {
  Tiling T = tiling_of(h);
  if ((T.tx + 1) * (T.ty + 1) > SMAX) return cudaErrorInvalidValue;   // n0 odd: not a valid grid
  if (T.nblocks > h->div_blocks) T.nblocks = h->div_blocks;
  {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    k_div<double><<<T.nblocks, dim3(T.tx, T.ty), 0, s>>>(grid_of(h), T, X, d, h->dscal, h->partial,
                                                         (unsigned int*)(h->dcount + 4), check_done, mean_mask);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad(const rve_s* h, const double* u, double* Y, const uint8_t* mask, const double* shift,
                        cudaStream_t s) {
  const Tiling T = tiling_of(h);
  if ((T.tx + 1) * (T.ty + 1) > SMAX) return cudaErrorInvalidValue;   // n0 odd: not a valid grid
  {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    k_grad_t<false, double><<<T.nblocks, dim3(T.tx, T.ty), 0, s>>>(grid_of(h), T, u, zero_mode(mask, shift), Y,
                                                                   nullptr, nullptr, nullptr, h->dscal, h->partial,
                                                                   (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_cg(const rve_s* h, const double* u, const uint8_t* mask, cudaStream_t s) {
  const Tiling T = tiling_of(h);
  if ((T.tx + 1) * (T.ty + 1) > SMAX) return cudaErrorInvalidValue;   // n0 odd: not a valid grid
  {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    k_grad_t<true, double><<<T.nblocks, dim3(T.tx, T.ty), 0, s>>>(grid_of(h), T, u, zero_mode(mask, nullptr),
                                                                  nullptr, h->x, h->r, h->p, h->dscal, h->partial,
                                                                  (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_div32(const rve_s* h, const float* X, float* d, unsigned mean_mask, cudaStream_t s) {
  // the same capped grid as in FP64: one tile per block (2048 blocks at 64^3)
  // measured slower (41.5 against 34.6 us) than a few tiles per block
  Tiling T = tiling_of(h);
  if ((T.tx + 1) * (T.ty + 1) > SMAX) return cudaErrorInvalidValue;   // n0 odd: not a valid grid
  if (T.nblocks > h->div_blocks) T.nblocks = h->div_blocks;
  {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    k_div<float><<<T.nblocks, dim3(T.tx, T.ty), 0, s>>>(grid_of(h), T, X, d, h->dscal, h->partial,
                                                        (unsigned int*)(h->dcount + 4), 1, mean_mask);
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_cg32(const rve_s* h, const float* u, const uint8_t* mask, cudaStream_t s) {
  const Tiling T = tiling_of(h);
  if ((T.tx + 1) * (T.ty + 1) > SMAX) return cudaErrorInvalidValue;   // n0 odd: not a valid grid
  {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    k_grad_t<true, float><<<T.nblocks, dim3(T.tx, T.ty), 0, s>>>(grid_of(h), T, u, zero_mode(mask, nullptr), nullptr,
                                                                 h->x32, h->r32, h->p32, h->dscal, h->partial,
                                                                 (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}
