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

template <typename V> struct V2T;
template <> struct V2T<double> { typedef double2 t; };
template <> struct V2T<float> { typedef float2 t; };

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

// ---------------------------------------------------------------- row-strip stencils
// For n0 = 32 NPL (NPL = 1..4) the stencils run one warp per run of
// consecutive rows (x lines), walked as strips within z planes, a whole x
// line per warp with
// NPL adjacent points per lane (x = NPL lane + k), loaded as vectors.  The
// stencil is applied separably, so every partial sum is formed once and
// shared: z pairs (or differences), then y pairs of those, then the x step.
// Within a lane the x -/+ 1 neighbour is the lane's own next point; across
// lanes one value per field row comes by a warp shuffle (the line is
// periodic and complete in the warp: no halo, no block barrier).  Each row
// keeps the previous row's z pairs in registers and issues the next row's
// loads before its own arithmetic.  Per voxel this is 30 FP64 additions for
// the divergence (against 42 in the tiled form, which recomputes the shared
// pairs) and 24 for the gradient (against 33).
constexpr int RW = 4;            // warps per block

template <typename V, int NPL>
__device__ __forceinline__ void load_row(const V* __restrict__ src, V (&v)[NPL]) {
  if constexpr (NPL == 2 || NPL == 4) {
    typedef typename V2T<V>::t V2;
#pragma unroll
    for (int k = 0; k < NPL; k += 2) {
      const V2 w = __ldg(reinterpret_cast<const V2*>(src) + k / 2);
      v[k] = w.x;
      v[k + 1] = w.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NPL; ++k) v[k] = __ldg(src + k);
  }
}

// The rows (x lines) of the grid, n1 n2 of them in (z, y) order, split into
// one contiguous run per warp of the grid, the runs differing in length by
// at most one row: every SM gets the same work whatever the grid's shape.  A
// run is walked as strips, each the part of the run inside one z plane; a
// strip starts with a priming row (the partial sums of its row before or
// after).  next() sets the next strip (z, ya .. yb - 1) and is false once
// the run is done.
struct RowRange {
  unsigned r, e, n1;
  int z, ya, yb;
  __device__ bool next() {
    if (r >= e) return false;
    z = (int)(r / n1);
    ya = (int)(r - (unsigned)z * n1);
    const unsigned left = e - r, room = n1 - (unsigned)ya;
    yb = ya + (int)(left < room ? left : room);
    r += (unsigned)(yb - ya);
    return true;
  }
};

__device__ __forceinline__ RowRange row_range(const Grid3& g, int warps_per_block) {
  const unsigned long long rows = (unsigned long long)g.n1 * g.n2;
  const unsigned long long nw = (unsigned long long)gridDim.x * warps_per_block;
  const unsigned long long w = (unsigned long long)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  RowRange rr;
  rr.r = (unsigned)(rows * w / nw);
  rr.e = (unsigned)(rows * (w + 1) / nw);
  rr.n1 = (unsigned)g.n1;
  rr.z = rr.ya = rr.yb = 0;
  return rr;
}

// Divergence d_i = sum_l D_l^T X_il (unscaled), as k_div.  Per voxel and row
// i of X (fields A = X_i0, B = X_i1, C = X_i2): z pairs A = X(z) + X(z-1),
// B likewise, C = X(z-1) - X(z); then with YS_A = A(y) + A(y-1),
// YD_B = B(y-1) - B(y), YS_C = C(y) + C(y-1) and Q = YD_B + YS_C,
//   d_i(x) = (Q - YS_A)(x) + (Q + YS_A)(x - 1).
template <typename V, int NPL>
__global__ void __launch_bounds__(32 * RW) k_div_rows(Grid3 g, const V* __restrict__ X,
                                                     V* __restrict__ d, double* __restrict__ ds,
                                                     double* __restrict__ partial, unsigned int* __restrict__ ticket,
                                                     int check_done, unsigned mean_mask) {
  __shared__ double sh[320];
  if (check_done && ds[DS_DONE] != 0.0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int left = (lane + 31) & 31;
  // the next row's loads are issued ahead of this row's arithmetic where the
  // registers allow it (up to three points per lane)
  constexpr bool PF = NPL <= 3;
  V mean[9];
#pragma unroll
  for (int f = 0; f < 9; ++f) mean[f] = (V)0;
  RowRange rr = row_range(g, RW);
  while (rr.next()) {                                   // warp-uniform: one strip of one plane
    const int z = rr.z, ya = rr.ya, yb = rr.yb;
    const unsigned plane = (unsigned)g.n0 * g.n1;
    const unsigned rz = (unsigned)z * plane, rzp = (unsigned)wrapi(z - 1, g.n2) * plane;
    V a[9][NPL], b[9][NPL];                             // loads of one row: plane z, plane z - 1
    auto load = [&](int y) {
      const unsigned row = (unsigned)y * g.n0 + NPL * lane;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        load_row<V, NPL>(X + (size_t)f * g.nvox + rz + row, a[f]);
        load_row<V, NPL>(X + (size_t)f * g.nvox + rzp + row, b[f]);
      }
    };
    V zp[9][NPL];                                       // z pairs of the previous row
    load(wrapi(ya - 1, g.n1));
#pragma unroll
    for (int f = 0; f < 9; ++f)
#pragma unroll
      for (int k = 0; k < NPL; ++k) zp[f][k] = (f % 3 == 2) ? b[f][k] - a[f][k] : a[f][k] + b[f][k];
    if (PF) load(ya);
    for (int y = ya; y < yb; ++y) {
      if (!PF) load(y);
      V zc[9][NPL];
#pragma unroll
      for (int f = 0; f < 9; ++f)
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
          zc[f][k] = (f % 3 == 2) ? b[f][k] - a[f][k] : a[f][k] + b[f][k];
          if ((mean_mask >> f) & 1u) mean[f] += a[f][k];
        }
      if (PF && y + 1 < yb) load(y + 1);                // in flight during this row's arithmetic
      const unsigned row = rz + (unsigned)y * g.n0 + NPL * lane;
      if constexpr (sizeof(V) == 8) {
        // FP64: the x step of the three y sums in one pair (e1, e2), one
        // value per row from the left lane
        V e1[3][NPL], e2[3][NPL], e2l[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < NPL; ++k) {
            const V ysa = zc[3 * i][k] + zp[3 * i][k];
            const V ydb = zp[3 * i + 1][k] - zc[3 * i + 1][k];
            const V ysc = zc[3 * i + 2][k] + zp[3 * i + 2][k];
            const V q = ydb + ysc;
            e1[i][k] = q - ysa;
            e2[i][k] = q + ysa;
          }
        // the left neighbour's last point, for the three rows at once
#pragma unroll
        for (int i = 0; i < 3; ++i) e2l[i] = __shfl_sync(0xffffffffu, e2[i][NPL - 1], left);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < NPL; ++k)
            d[(size_t)i * g.nvox + row + k] = e1[i][k] + (k == 0 ? e2l[i] : e2[i][k - 1]);
      } else {
        // FP32 (the mixed-precision CG): each directional term is formed as a
        // difference of its own y sums before the terms are added, so the
        // small y differences are never rounded at the scale of the large z
        // pairs (the grouping of the tiled kernel); three values per row
        // cross lanes
        V ysa[3][NPL], ydb[3][NPL], ysc[3][NPL], l[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < NPL; ++k) {
            ysa[i][k] = zc[3 * i][k] + zp[3 * i][k];
            ydb[i][k] = zp[3 * i + 1][k] - zc[3 * i + 1][k];
            ysc[i][k] = zc[3 * i + 2][k] + zp[3 * i + 2][k];
          }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          l[i][0] = __shfl_sync(0xffffffffu, ysa[i][NPL - 1], left);
          l[i][1] = __shfl_sync(0xffffffffu, ydb[i][NPL - 1], left);
          l[i][2] = __shfl_sync(0xffffffffu, ysc[i][NPL - 1], left);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < NPL; ++k) {
            const V am = k == 0 ? l[i][0] : ysa[i][k > 0 ? k - 1 : 0];
            const V bm = k == 0 ? l[i][1] : ydb[i][k > 0 ? k - 1 : 0];
            const V cm = k == 0 ? l[i][2] : ysc[i][k > 0 ? k - 1 : 0];
            const V d0 = am - ysa[i][k];
            const V d1 = ydb[i][k] + bm;
            const V d2 = ysc[i][k] + cm;
            d[(size_t)i * g.nvox + row + k] = d0 + d1 + d2;
          }
      }
#pragma unroll
      for (int f = 0; f < 9; ++f)
#pragma unroll
        for (int k = 0; k < NPL; ++k) zp[f][k] = zc[f][k];
    }
  }
  // means: one transposed warp reduction of the (up to nine) selected fields,
  // the block's warps combined in shared memory, then the grid's last block
  V m16[16];
#pragma unroll
  for (int f = 0; f < 16; ++f) m16[f] = f < 9 ? mean[f] : (V)0;
  const V w = warp_sums16<V>(m16);
  const int slot = slot16_of_lane(lane);
  if ((lane & 1) == 0 && slot < 9) sh[warp * 16 + slot] = (double)w;
  __syncthreads();
  if (threadIdx.x < 9) {
    double t = 0.0;
    for (int q = 0; q < RW; ++q) t += sh[q * 16 + threadIdx.x];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = ((mean_mask >> threadIdx.x) & 1u) ? t : 0.0;
  }
  double tot[9];
  if (last_block_sums(partial, 9, ticket, sh, tot, mean_mask) && threadIdx.x == 0) {
    for (int c = 0; c < 9; ++c) ds[DS_XMEAN + c] = tot[c] / (double)g.nvox;
  }
}

// Gradient of the three potentials q_ij = D_j u_i (unscaled) plus the zero
// mode, as k_grad_t.  Per potential: z pair SP = u(z) + u(z+1) and
// difference SM = u(z+1) - u(z); YS = SP(y) + SP(y+1), YD = SP(y+1) - SP(y),
// YM = SM(y) + SM(y+1); q_i0 = YS(x+1) - YS(x), q_i1 = YD(x) + YD(x+1),
// q_i2 = YM(x) + YM(x+1).  CG as in k_grad_t.
template <bool CG, typename V, int NPL>
__global__ void __launch_bounds__(32 * RW, NPL <= 2 ? 4 : 1) k_grad_rows(Grid3 g, const V* __restrict__ u,
                                                      ZeroMode zm, double* __restrict__ Y, V* __restrict__ x,
                                                      V* __restrict__ r, const V* __restrict__ p,
                                                      double* __restrict__ ds, double* __restrict__ partial,
                                                      unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  if (CG && ds[DS_DONE] != 0.0) return;
  const V alpha = CG ? (V)ds[DS_ALPHA] : (V)0;
  V off[9];
#pragma unroll
  for (int c = 0; c < 9; ++c)          // (in the CG update the zero mode carries no shift)
    off[c] = zm.keep[c] ? (CG ? (V)ds[DS_XMEAN + c] : (V)(ds[DS_XMEAN + c] + zm.add[c])) : (V)0;
  const int lane = threadIdx.x & 31;
  const int right = (lane + 1) & 31;
  V acc = (V)0;
  RowRange rr = row_range(g, RW);
  while (rr.next()) {                                   // warp-uniform: one strip of one plane
    const int z = rr.z, ya = rr.ya, yb = rr.yb;
    const unsigned plane = (unsigned)g.n0 * g.n1;
    const unsigned rz = (unsigned)z * plane, rzn = (unsigned)wrapi(z + 1, g.n2) * plane;
    V a[3][NPL], c[3][NPL];                             // loads of one row: plane z, plane z + 1
    auto load = [&](int y) {
      const unsigned row = (unsigned)y * g.n0 + NPL * lane;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        load_row<V, NPL>(u + (size_t)i * g.nvox + rz + row, a[i]);
        load_row<V, NPL>(u + (size_t)i * g.nvox + rzn + row, c[i]);
      }
    };
    V sp[3][NPL], sm[3][NPL];                           // z pair and difference of the current row
    load(ya);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < NPL; ++k) { sp[i][k] = a[i][k] + c[i][k]; sm[i][k] = c[i][k] - a[i][k]; }
    load(ya + 1 < g.n1 ? ya + 1 : 0);
    for (int y = ya; y < yb; ++y) {
      V spn[3][NPL], smn[3][NPL];                       // row y + 1
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < NPL; ++k) { spn[i][k] = a[i][k] + c[i][k]; smn[i][k] = c[i][k] - a[i][k]; }
      if (y + 1 < yb) load(y + 2 < g.n1 ? y + 2 : 0);
      const unsigned row = rz + (unsigned)y * g.n0 + NPL * lane;
      V ys[3][NPL], yd[3][NPL], ym[3][NPL], rs[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
          ys[i][k] = sp[i][k] + spn[i][k];
          yd[i][k] = spn[i][k] - sp[i][k];
          ym[i][k] = sm[i][k] + smn[i][k];
        }
      // the right neighbour's first point of the three sums, nine at once
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rs[i][0] = __shfl_sync(0xffffffffu, ys[i][0], right);
        rs[i][1] = __shfl_sync(0xffffffffu, yd[i][0], right);
        rs[i][2] = __shfl_sync(0xffffffffu, ym[i][0], right);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        V qv[3][NPL];
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
          const V ysr = k + 1 < NPL ? ys[i][k + 1 < NPL ? k + 1 : 0] : rs[i][0];
          const V ydr = k + 1 < NPL ? yd[i][k + 1 < NPL ? k + 1 : 0] : rs[i][1];
          const V ymr = k + 1 < NPL ? ym[i][k + 1 < NPL ? k + 1 : 0] : rs[i][2];
          qv[0][k] = ysr - ys[i][k];
          qv[1][k] = yd[i][k] + ydr;
          qv[2][k] = ym[i][k] + ymr;
#pragma unroll
          for (int j = 0; j < 3; ++j)
            if (zm.keep[3 * i + j]) qv[j][k] += off[3 * i + j];
        }
        if (CG) {
          // the row's p, x and r of this tensor row are loaded together, so
          // that their latencies overlap
          V pv[3][NPL], xv[3][NPL], rv[3][NPL];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const size_t e = (size_t)(3 * i + j) * g.nvox + row;
            load_row<V, NPL>(p + e, pv[j]);
            load_row<V, NPL>(x + e, xv[j]);
            load_row<V, NPL>(r + e, rv[j]);
          }
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
              const size_t e = (size_t)(3 * i + j) * g.nvox + row + k;
              x[e] = fma(alpha, pv[j][k], xv[j][k]);
              const V rn = fma(-alpha, qv[j][k], rv[j][k]);
              r[e] = rn;
              acc = fma(rn, rn, acc);
            }
        } else {
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
              Y[(size_t)(3 * i + j) * g.nvox + row + k] = (double)qv[j][k];
              acc = fma(qv[j][k], qv[j][k], acc);
            }
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < NPL; ++k) { sp[i][k] = spn[i][k]; sm[i][k] = smn[i][k]; }
    }
  }
  const double s = blk_sum_v<V>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  double tot;
  if (last_block_sums(partial, 1, ticket, sh, &tot) && threadIdx.x == 0) {
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

struct RowShape {
  int npl, nblocks;
};

// One wave of resident blocks: blocks_per_sm on every SM, at most `cap`
// (the divergence passes h->div_blocks, which the autotuner varies), and no
// more warps than rows.  The rows are split evenly over the warps (RowRange).
RowShape row_shape_for(const rve_s* h, int blocks_per_sm, int cap) {
  RowShape r{0, 0};
  if (h->n0 % 32 != 0 || h->n0 > 128) return r;
  r.npl = h->n0 / 32;
  const long rows = (long)h->n1 * h->n2;
  long nb = (long)h->num_sms * (blocks_per_sm > 0 ? blocks_per_sm : 1);
  if (cap > 0 && cap < nb) nb = cap;
  if (nb > rows / RW) nb = rows / RW;
  if (nb > 4096) nb = 4096;
  r.nblocks = (int)(nb > 0 ? nb : 1);
  return r;
}

template <typename K>
int resident_blocks(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 32 * RW, 0) != cudaSuccess) n = 1;
  return n;
}

template <typename V, int NPL>
cudaError_t div_rows_n(const rve_s* h, const V* X, V* d, int check_done, unsigned mean_mask, cudaStream_t s,
                       const Grid3& g) {
  static const int bps = resident_blocks(k_div_rows<V, NPL>);
  const RowShape rs = row_shape_for(h, bps, h->div_blocks);
  k_div_rows<V, NPL><<<rs.nblocks, 32 * RW, 0, s>>>(g, X, d, h->dscal, h->partial, (unsigned int*)(h->dcount + 4),
                                                    check_done, mean_mask);
  return cudaGetLastError();
}

template <typename V>
cudaError_t div_rows(const rve_s* h, int npl, const V* X, V* d, int check_done, unsigned mean_mask, cudaStream_t s,
                     const Grid3& g) {
  switch (npl) {
    case 1: return div_rows_n<V, 1>(h, X, d, check_done, mean_mask, s, g);
    case 2: return div_rows_n<V, 2>(h, X, d, check_done, mean_mask, s, g);
    case 3: return div_rows_n<V, 3>(h, X, d, check_done, mean_mask, s, g);
    default: return div_rows_n<V, 4>(h, X, d, check_done, mean_mask, s, g);
  }
}

template <bool CG, typename V, int NPL>
cudaError_t grad_rows_n(const rve_s* h, const V* u, const ZeroMode& zm, double* Y, V* x, V* r, const V* p,
                        cudaStream_t s, const Grid3& g) {
  static const int bps = resident_blocks(k_grad_rows<CG, V, NPL>);
  const RowShape rs = row_shape_for(h, bps, 0);
  k_grad_rows<CG, V, NPL><<<rs.nblocks, 32 * RW, 0, s>>>(g, u, zm, Y, x, r, p, h->dscal, h->partial,
                                                         (unsigned int*)(h->dcount + 4));
  return cudaGetLastError();
}

template <bool CG, typename V>
cudaError_t grad_rows(const rve_s* h, int npl, const V* u, const ZeroMode& zm, double* Y, V* x, V* r, const V* p,
                      cudaStream_t s, const Grid3& g) {
  switch (npl) {
    case 1: return grad_rows_n<CG, V, 1>(h, u, zm, Y, x, r, p, s, g);
    case 2: return grad_rows_n<CG, V, 2>(h, u, zm, Y, x, r, p, s, g);
    case 3: return grad_rows_n<CG, V, 3>(h, u, zm, Y, x, r, p, s, g);
    default: return grad_rows_n<CG, V, 4>(h, u, zm, Y, x, r, p, s, g);
  }
}

// points per lane of the row-strip stencils for this grid (0: tiled stencils).
// The FP64 divergence takes them up to n0 = 128; the gradient with its fused
// vector update up to n0 = 64 (beyond that its register demand leaves too
// few warps to cover the update's loads, measured 1.8x slower at 128^3).  The
// FP32 stencils of the mixed-precision CG take them up to n0 = 64: on the
// hardest sweep RVE (96^3, 183 grains, plastic onset) the FP32 CG stalls on
// the non-symmetric tangent and the Newton path is chaotic in the rounding
// order of the projection; it is known to converge with the tiled order there.
int row_npl(const rve_s* h, bool gradient = false, bool fp32 = false) {
  const int lim = (gradient || fp32) ? 64 : 128;
  if (!h->row_stencils || h->n0 % 32 != 0 || h->n0 > lim) return 0;
  return h->n0 / 32;
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
  if (const int npl = row_npl(h)) {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    return div_rows<double>(h, npl, X, d, check_done, mean_mask, s, grid_of(h));
  }
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
  if (const int npl = row_npl(h, true)) {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    return grad_rows<false, double>(h, npl, u, zero_mode(mask, shift), Y, nullptr, nullptr, nullptr, s, grid_of(h));
  }
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
  if (const int npl = row_npl(h, true)) {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    return grad_rows<true, double>(h, npl, u, zero_mode(mask, nullptr), nullptr, h->x, h->r, h->p, s, grid_of(h));
  }
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
  if (const int npl = row_npl(h, false, true)) {
    ProfScope ps_(h, RVE_K_STENCIL, s);
    return div_rows<float>(h, npl, X, d, 1, mean_mask, s, grid_of(h));
  }
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
  if (const int npl = row_npl(h, true, true)) {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    return grad_rows<true, float>(h, npl, u, zero_mode(mask, nullptr), nullptr, h->x32, h->r32, h->p32, s, grid_of(h));
  }
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
