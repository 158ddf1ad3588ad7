// Device helpers shared by the kernels of the GB300 path: complex arithmetic,
// the FCC slip-system table in the crystal frame and small 3x3 algebra.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RVE_HD __host__ __device__ __forceinline__

struct cplx { double x, y; };
RVE_HD cplx cmk(double a, double b) { cplx c; c.x = a; c.y = b; return c; }
RVE_HD cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
RVE_HD cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
RVE_HD cplx cmul(cplx a, cplx b) { return cmk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)); }
RVE_HD cplx cconj(cplx a) { return cmk(a.x, -a.y); }
RVE_HD cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
// multiply by (sign * i): sign = -1 forward, +1 inverse
RVE_HD cplx cmul_i(cplx a, int sign) { return sign > 0 ? cmk(-a.y, a.x) : cmk(a.y, -a.x); }

// FCC {111}<110> slip systems, crystal frame, unnormalised integer vectors.
// Plane normals m' in {(111), (-111), (1-11), (11-1)} (|m'| = sqrt 3), three
// <110> directions s' (|s'| = sqrt 2) per plane; the unit Schmid tensor is
// s (x) m = s' m'^T / sqrt 6.  The order is the one the whole library (and its
// field outputs) uses for slip-system indices 0..11.
// As compile-time functions: the loops over systems are unrolled everywhere,
// so every coefficient built from these is a constant there.
__host__ __device__ constexpr int fcc_s(int a, int i) {
  constexpr signed char t[12][3] = {
      {0, 1, -1}, {-1, 0, 1}, {1, -1, 0},
      {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
      {0, 1, 1}, {1, 0, -1}, {1, 1, 0},
      {0, 1, 1}, {1, 0, 1}, {1, -1, 0}};
  return t[a][i];
}
__host__ __device__ constexpr int fcc_m(int a, int i) {
  constexpr signed char t[12][3] = {
      {1, 1, 1}, {1, 1, 1}, {1, 1, 1},
      {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
      {1, -1, 1}, {1, -1, 1}, {1, -1, 1},
      {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
  return t[a][i];
}

// acc + c x for a small integer coefficient c that is a compile-time
// constant (a product of slip-table entries): c = 0 adds nothing and c = +-1
// is an addition or a subtraction, so no FP64 instruction is spent on the
// table's zeros and ones.  (The compiler may not drop a product with 0.0 on
// its own: for an infinite or NaN x it is not zero.)  `first` marks an empty
// accumulator, whose first term is taken exactly.
__device__ __forceinline__ double cacc(double acc, bool& first, int c, double x) {
  if (c == 0) return acc;
  double r;
  if (first) r = c == 1 ? x : (c == -1 ? -x : (double)c * x);
  else r = c == 1 ? acc + x : (c == -1 ? acc - x : fma((double)c, x, acc));
  first = false;
  return r;
}

// M += g s^a (x) m^a / sqrt 6 (the unit Schmid tensor of system a)
__device__ __forceinline__ void add_schmid(double* M, int a, double g) {
  const double gs = g * 0.40824829046386301637;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      bool f = false;
      M[3 * i + j] = cacc(M[3 * i + j], f, fcc_s(a, i) * fcc_m(a, j), gs);
    }
}

// Voigt order of a symmetric tensor: 11, 22, 33, 23, 13, 12
#define V_I(a) ((a) < 3 ? (a) : ((a) == 3 ? 1 : 0))
#define V_J(a) ((a) < 3 ? (a) : ((a) == 5 ? 1 : 2))

RVE_HD void mat3_mul(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = fma(A[3 * i], B[j], fma(A[3 * i + 1], B[3 + j], A[3 * i + 2] * B[6 + j]));
}
// C = A^T B
RVE_HD void mat3_tmul(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = fma(A[i], B[j], fma(A[3 + i], B[3 + j], A[6 + i] * B[6 + j]));
}
// C = A B^T
RVE_HD void mat3_mult(const double* A, const double* B, double* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = fma(A[3 * i], B[3 * j], fma(A[3 * i + 1], B[3 * j + 1], A[3 * i + 2] * B[3 * j + 2]));
}
RVE_HD double mat3_inv(const double* A, double* B) {
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  double id = 1.0 / det;
  B[0] = c00 * id;
  B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  B[3] = c01 * id;
  B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  B[6] = c02 * id;
  B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return det;
}

// ---- deterministic reductions shared by the reducing kernels ----
// linear thread index and block size (1-D or 2-D blocks)
__device__ __forceinline__ int lin_tid() { return threadIdx.x + blockDim.x * threadIdx.y; }
__device__ __forceinline__ int lin_nthreads() { return blockDim.x * blockDim.y; }

// block-wide sum, result in linear thread 0 (all threads must call it; the
// block size is a multiple of 32)
__device__ __forceinline__ double blk_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int t = lin_tid();
  const int lane = t & 31, wid = t >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (t == 0) {
    const int nw = (lin_nthreads() + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sh[w];
  }
  __syncthreads();
  return s;
}

// Block-wide sum of a value of the field type V: the warp stage adds in V
// (FP32 shuffles for the mixed-precision loop, where FP64 additions would
// cost the narrow FP64 pipe), the warps' sums are added in double.  For
// V = double it is blk_sum.
template <typename V>
__device__ __forceinline__ double blk_sum_v(V v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int t = lin_tid();
  const int lane = t & 31, wid = t >> 5;
  if (lane == 0) sh[wid] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (t == 0) {
    const int nw = (lin_nthreads() + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sh[w];
  }
  __syncthreads();
  return s;
}

// Block-wide sums of up to nine values at once (bit c of `which` selects
// value c): the shuffle trees of all values are interleaved and one pair of
// barriers serves them all.  Each value is summed in the same order as
// blk_sum_v (the same bits).  Results in out[] of linear thread 0 (0 for
// unselected values).  sh: at least 10 * 32 doubles.
template <typename V>
__device__ __forceinline__ void blk_sums9(V* v, unsigned which, double* sh, double* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if ((which >> c) & 1u) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  const int t = lin_tid();
  const int lane = t & 31, wid = t >> 5;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if ((which >> c) & 1u) sh[32 * c + wid] = (double)v[c];
  }
  __syncthreads();
  if (t < 9 && ((which >> t) & 1u)) {
    const int nw = (lin_nthreads() + 31) >> 5;
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[32 * t + w];
    sh[288 + t] = s;
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int c = 0; c < 9; ++c) out[c] = ((which >> c) & 1u) ? sh[288 + c] : 0.0;
  }
  __syncthreads();
}

// Sums over a warp of 16 values per lane by transposed halving: at the level
// of shuffle distance o (16, 8, 4, 2) every lane keeps half of its values and
// adds the partner's copy of that half, so the four levels cost 8 + 4 + 2 + 1
// additions, and one more level (distance 1) completes the sums: 16 FP64
// additions per warp instead of 16 x 5 for separate shuffle trees (every
// FP64 instruction counts on this GPU's narrow FP64 pipe).  On return lane
// L holds the warp total of value slot16_of_lane(L) (each slot in two lanes).
__device__ __forceinline__ int slot16_of_lane(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
template <typename V>
__device__ __forceinline__ V warp_sums16(V* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const int o = 2 * h;               // shuffle distance 16, 8, 4, 2
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const V send = hi ? v[k] : v[k + h];
      const V keep = hi ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// After every block has written partial[c * gridDim.x + blockIdx.x] for
// c < nval (nval <= 9): the block that takes the last ticket sums each value
// whose bit is set in `which` over the blocks in block order (deterministic)
// into out[c] (thread 0; 0 for the others) and returns true; every other block
// returns false.  The partials of all values are loaded together and summed
// by one fused block reduction, so the tail costs one round trip to L2 rather
// than one per value.  sh: at least 10 * 32 doubles.
__device__ __forceinline__ bool last_block_sums(const double* partial, int nval, unsigned int* ticket, double* sh,
                                                double* out, unsigned which = 0x1FFu) {
  __shared__ bool last;
  const int t = lin_tid();
  __threadfence();
  __syncthreads();
  if (t == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return false;
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  // four partials per value in flight at a time (the loads of one group are
  // issued before its additions, which keep the order of i: the sums are
  // those of the plain loop, bit for bit)
  const int n = (int)gridDim.x, nt = lin_nthreads();
  int i = t;
  for (; i + 3 * nt < n; i += 4 * nt) {
    double v[4][9];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 9; ++c)
        v[q][c] = (c < nval && ((which >> c) & 1u)) ? __ldcg(partial + (size_t)c * n + i + q * nt) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (c < nval && ((which >> c) & 1u)) acc[c] += v[q][c];
  }
  for (; i < n; i += nt) {
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if (c < nval && ((which >> c) & 1u)) acc[c] += __ldcg(partial + (size_t)c * n + i);
  }
  double res[9];
  blk_sums9<double>(acc, which & ((1u << nval) - 1u), sh, res);
  if (t == 0) {
    for (int c = 0; c < nval; ++c) out[c] = res[c];
    *ticket = 0u;
  }
  return true;
}
