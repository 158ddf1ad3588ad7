// Vector kernels of the Newton / conjugate-gradient solve (Sec. 2.2,
// Eq. linequil2ast), the increment predictor, the commit of the internal
// variables (Kocks-Mecking SSD update, Eq. kocks, integrated implicitly over
// the increment) and the volume averages.  All reductions are deterministic:
// a fixed grid writes one partial per block, a single block sums the
// partials in a fixed order and derives the CG scalars on the device.
#include <algorithm>

#include "common.cuh"
#include "rve_internal.h"

namespace {

// k_macro and k_mean9 reduce 27 and 9 values per thread at the end (five
// shuffle additions each, FP64): one block per SM amortises that over many voxels
constexpr int MACRO_BLOCKS = 152;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sh[w];
  }
  __syncthreads();
  return s;
}

// Last-block finalisation: every block has written its partial; the block
// that takes the last ticket sums the partials in block order (deterministic)
// and returns the total in thread 0 (other threads and blocks get NaN).
__device__ __forceinline__ double last_block_sum(const double* partial, unsigned int* ticket, double* sh) {
  __shared__ bool last;
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return NAN;
  double acc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(partial + i);
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) *ticket = 0u;
  return s;
}

// p = r (first) or r + beta p; t = K : p; pKp = p . t; alpha = rr / pKp.
// Returns at once when the CG loop has converged (done != 0).
__global__ void __launch_bounds__(RVE_RED_THREADS, 3) k_tangent_apply(size_t nvox, const double* __restrict__ K,
                                                                      const double* __restrict__ r, double* __restrict__ p,
                                                                      double* __restrict__ t, double* __restrict__ ds,
                                                                      double* __restrict__ partial,
                                                                      unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  if (ds[DS_DONE] != 0.0) return;
  // the first iteration of a solve (the counter is reset by the CG init and
  // bumped by each completed iteration): every launch of the loop has the
  // same arguments, so chunks of iterations can be replayed as a CUDA graph
  const bool first = ds[DS_ITERS] == 0.0;
  const double beta = first ? 0.0 : ds[DS_BETA];
  double acc = 0.0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
    double pv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double rv = r[k * nvox + v];
      pv[k] = first ? rv : fma(beta, p[k * nvox + v], rv);
      p[k * nvox + v] = pv[k];
    }
    // three rows of K (27 streamed loads in flight) per stage
#pragma unroll
    for (int ib = 0; ib < 3; ++ib) {
      double kk[27];
#pragma unroll
      for (int e = 0; e < 27; ++e) kk[e] = __ldcs(K + (size_t)(27 * ib + e) * nvox + v);
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < 9; ++j) s = fma(kk[9 * ii + j], pv[j], s);
        t[(3 * ib + ii) * nvox + v] = s;
        acc = fma(pv[3 * ib + ii], s, acc);
      }
    }
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_PKP] = tot;
    ds[DS_ALPHA] = ds[DS_RR] / tot;
  }
}

// x += alpha p; r -= alpha q; rr' = r . r; beta = rr' / rr; one more
// iteration counted; done once rr' <= stop.
__global__ void __launch_bounds__(RVE_RED_THREADS) k_cg_update(size_t n, double* __restrict__ x, double* __restrict__ r,
                                                               const double* __restrict__ p, const double* __restrict__ q,
                                                               double* __restrict__ ds, double* __restrict__ partial,
                                                               unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  if (ds[DS_DONE] != 0.0) return;
  const double alpha = ds[DS_ALPHA];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    x[e] = fma(alpha, p[e], x[e]);
    const double rv = fma(-alpha, q[e], r[e]);
    r[e] = rv;
    acc = fma(rv, rv, acc);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_BETA] = tot / ds[DS_RR];
    ds[DS_RR] = tot;
    ds[DS_ITERS] += 1.0;
    if (!(tot > ds[DS_STOP])) ds[DS_DONE] = 1.0;   // also stops on NaN
  }
}

// Mixed precision: the same CG step with FP32 tangent and vectors (warp sums
// in FP32, block and grid sums in FP64).  p = r (first) or r + beta p; t = K : p; alpha = rr / p.t
__global__ void __launch_bounds__(RVE_RED_THREADS, 2) k_tangent_apply32(size_t nvox, const float* __restrict__ K,
                                                                     const float* __restrict__ r, float* __restrict__ p,
                                                                     float* __restrict__ t, double* __restrict__ ds,
                                                                     double* __restrict__ partial,
                                                                     unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  if (ds[DS_DONE] != 0.0) return;
  const bool first = ds[DS_ITERS] == 0.0;
  const float beta = first ? 0.0f : (float)ds[DS_BETA];
  float acc = 0.0f;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
    // all 81 tangent loads are issued before any arithmetic: in FP32 the
    // kernel is bound by HBM, and one round trip per voxel instead of one per
    // row keeps enough bytes in flight
    float kk[81], pv[9];
#pragma unroll
    for (int e = 0; e < 81; ++e) kk[e] = __ldcs(K + (size_t)e * nvox + v);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float rv = r[k * nvox + v];
      pv[k] = first ? rv : fmaf(beta, p[k * nvox + v], rv);
      p[k * nvox + v] = pv[k];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float sacc = 0.0f;
#pragma unroll
      for (int j = 0; j < 9; ++j) sacc = fmaf(kk[9 * i + j], pv[j], sacc);
      t[i * nvox + v] = sacc;
      acc = fmaf(pv[i], sacc, acc);
    }
  }
  const double s = blk_sum_v<float>(acc, sh);   // warp stage in FP32
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_PKP] = tot;
    ds[DS_ALPHA] = ds[DS_RR] / tot;
  }
}

// ---- TMA-staged FP32 tangent apply ----
// The FP32 CG step is bound by HBM: 324 of its 396 bytes per voxel are the
// tangent.  A persistent block per SM streams 256-voxel tiles of the 81
// tangent rows and of r and p (99 rows) into shared memory with bulk
// asynchronous copies (one 1 KB copy per row, completion counted on an
// mbarrier), double-buffered, so the copy engine keeps the bytes in flight
// instead of per-thread loads.
constexpr int TA_TV = 256;                       // voxels per tile = threads per block
constexpr int TA_ROWS = 81 + 9 + 9;              // K, r, p
constexpr int TA_STAGE = TA_ROWS * TA_TV;        // floats per stage
constexpr unsigned TA_STAGE_BYTES = TA_STAGE * sizeof(float);
constexpr size_t TA_SMEM = 2 * (size_t)TA_STAGE_BYTES + 64;
constexpr unsigned WAIT_LIMIT = RVE_WAIT_POLLS_DEFAULT;   // bounded mbarrier polls, then an error flag

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
               ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// the same with an L2 evict-first policy: the tangent is read once per
// iteration and should not push the CG vectors the next kernels read out of L2
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("{\n .reg .b64 pol;\n createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n"
               " cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], pol;\n}"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// wait for the phase of the given parity; false after `limit` polls (0: gives
// up without polling)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = WAIT_LIMIT) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// issue the 99 row copies of tile `tile` into a stage buffer (threads 0..98)
__device__ __forceinline__ void ta_issue(const float* __restrict__ K, const float* __restrict__ r,
                                         const float* __restrict__ p, size_t nvox, long tile, float* buf,
                                         uint64_t* bar) {
  const size_t v0 = (size_t)tile * TA_TV;
  const size_t nv = (nvox - v0) < (size_t)TA_TV ? nvox - v0 : (size_t)TA_TV;
  const unsigned bytes = (unsigned)(nv * sizeof(float));   // nvox is a multiple of 4: a 16-byte multiple
  if (threadIdx.x == 0) mbar_expect_tx(bar, TA_ROWS * bytes);
  const int e = threadIdx.x;
  if (e < TA_ROWS) {
    if (e < 81)
      bulk_g2s_stream(buf + e * TA_TV, K + (size_t)e * nvox + v0, bytes, bar);
    else
      bulk_g2s(buf + e * TA_TV, (e < 90 ? r + (size_t)(e - 81) * nvox : p + (size_t)(e - 90) * nvox) + v0, bytes, bar);
  }
}

__global__ void __launch_bounds__(TA_TV, 1) k_tangent_apply32_tma(size_t nvox, const float* __restrict__ K,
                                                                 const float* __restrict__ r, float* __restrict__ p,
                                                                 float* __restrict__ t, double* __restrict__ ds,
                                                                 double* __restrict__ partial,
                                                                 unsigned int* __restrict__ ticket,
                                                                 unsigned tile_wait_polls) {
  extern __shared__ __align__(128) unsigned char ta_smem[];
  float* stage[2] = {reinterpret_cast<float*>(ta_smem), reinterpret_cast<float*>(ta_smem) + TA_STAGE};
  uint64_t* bar = reinterpret_cast<uint64_t*>(ta_smem + 2 * (size_t)TA_STAGE_BYTES);
  __shared__ double sh[320];
  if (ds[DS_DONE] != 0.0) return;
  const bool first = ds[DS_ITERS] == 0.0;
  const float beta = first ? 0.0f : (float)ds[DS_BETA];
  const long ntiles = (long)((nvox + TA_TV - 1) / TA_TV);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  long tile = blockIdx.x;
  // pending[b]: stage b has copies in flight that no wait has seen land
  bool pending[2] = {tile < ntiles, tile + gridDim.x < ntiles};
  if (pending[0]) ta_issue(K, r, p, nvox, tile, stage[0], &bar[0]);
  if (pending[1]) ta_issue(K, r, p, nvox, tile + gridDim.x, stage[1], &bar[1]);
  float acc = 0.0f;
  bool ok = true;
  unsigned phase[2] = {0u, 0u};
  for (int k = 0; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    // the decision to go on is the whole block's: a barrier inside the loop
    // follows.  The per-tile wait gives up after tile_wait_polls polls.
    if (!__syncthreads_and(mbar_wait(&bar[b], phase[b], tile_wait_polls) ? 1 : 0)) { ok = false; break; }
    pending[b] = false;
    phase[b] ^= 1u;
    const size_t v = (size_t)tile * TA_TV + threadIdx.x;
    if (v < nvox) {
      const float* Ks = stage[b];
      float pv[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const float rv = Ks[(81 + c) * TA_TV + threadIdx.x];
        pv[c] = first ? rv : fmaf(beta, Ks[(90 + c) * TA_TV + threadIdx.x], rv);
        p[c * nvox + v] = pv[c];
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        float sacc = 0.0f;
#pragma unroll
        for (int j = 0; j < 9; ++j) sacc = fmaf(Ks[(9 * i + j) * TA_TV + threadIdx.x], pv[j], sacc);
        t[i * nvox + v] = sacc;
        acc = fmaf(pv[i], sacc, acc);
      }
    }
    __syncthreads();                              // every thread is done with this stage
    const long next = tile + 2 * (long)gridDim.x;
    if (next < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      ta_issue(K, r, p, nvox, next, stage[b], &bar[b]);
      pending[b] = true;
    }
  }
  if (!ok) {
    // a wait gave up: flag it, and before the block exits give every stage
    // that still has copies in flight the full bounded wait, so that no copy
    // lands in shared memory after the block has left
    if (threadIdx.x == 0) ds[DS_ERR] = 1.0;
    if (pending[0]) mbar_wait(&bar[0], phase[0]);
    if (pending[1]) mbar_wait(&bar[1], phase[1]);
  }
  const double s = blk_sum_v<float>(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_PKP] = tot;
    ds[DS_ALPHA] = ds[DS_RR] / tot;
  }
}

// x32 = 0; r32 = -R (rounded); rr; stop = eta^2 rr; iteration count 0
__global__ void __launch_bounds__(RVE_RED_THREADS) k_cg_init32(size_t n, float* __restrict__ x, float* __restrict__ r,
                                                               const double* __restrict__ R, double* __restrict__ ds,
                                                               double eta, double* __restrict__ partial,
                                                               unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    x[e] = 0.0f;
    const float rv = (float)(-R[e]);
    r[e] = rv;
    acc += (double)rv * (double)rv;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_RR] = tot;
    ds[DS_STOP] = eta * eta * tot;
    ds[DS_ITERS] = 0.0;
    ds[DS_DONE] = (tot > 0.0) ? 0.0 : 1.0;
  }
}

__global__ void k_widen(size_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    b[e] = (double)a[e];
}

// x = 0; r = -R; rr = r . r; stop = eta^2 rr; iteration count 0
__global__ void __launch_bounds__(RVE_RED_THREADS) k_cg_init(size_t n, double* __restrict__ x, double* __restrict__ r,
                                                             const double* __restrict__ R, double* __restrict__ ds,
                                                             double eta, double* __restrict__ partial,
                                                             unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    x[e] = 0.0;
    const double rv = -R[e];
    r[e] = rv;
    acc = fma(rv, rv, acc);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
  const double tot = last_block_sum(partial, ticket, sh);
  if (threadIdx.x == 0 && !isnan(tot)) {
    ds[DS_RR] = tot;
    ds[DS_STOP] = eta * eta * tot;
    ds[DS_ITERS] = 0.0;
    ds[DS_DONE] = (tot > 0.0) ? 0.0 : 1.0;
  }
}

__global__ void __launch_bounds__(RVE_RED_THREADS) k_norm2(size_t n, const double* __restrict__ a, double* __restrict__ partial) {
  __shared__ double sh[320];
  double acc = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    acc = fma(a[e], a[e], acc);
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ partial, int nparts, int nval,
                                                       int mode, double* __restrict__ ds) {
  __shared__ double sh[320];
  for (int c = 0; c < nval; ++c) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[(size_t)c * nparts + i];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) {
      if (mode == RED_PKP_ALPHA) {
        ds[DS_PKP] = s;
        ds[DS_ALPHA] = ds[DS_RR] / s;
      } else if (mode == RED_RR_BETA) {
        ds[DS_BETA] = s / ds[DS_RR];
        ds[DS_RR] = s;
      } else if (mode == RED_RR_INIT) {
        ds[DS_RR] = s;
      } else if (mode == RED_NORM) {
        ds[DS_NORM] = s;
      } else {  // RED_MACRO: 27 averages -> mean P, mean sigma, mean F
        ds[DS_MEANP + c] = s;
      }
    }
  }
}

__global__ void k_axpy(size_t n, double* __restrict__ y, const double* __restrict__ x, double a) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

struct Nine { double v[9]; };

__global__ void k_predictor(size_t nvox, double* F, const double* Fc,
                            const double* __restrict__ dFl, Nine shift, double ratio, int extrapolate) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double f = Fc[k * nvox + v] + shift.v[k];
      if (extrapolate) f = fma(ratio, dFl[k * nvox + v], f);
      F[k * nvox + v] = f;
    }
  }
}

// Commit: Fp <- R (I + sum dgam s (x) m) R^T Fp; rho_SSD by implicit Kocks-Mecking;
// S_c <- S; dF_last <- F - F_c; F_c <- F.
__global__ void __launch_bounds__(128) k_commit(size_t nvox, const int32_t* __restrict__ grain,
                                                const double* __restrict__ grainR, const double* __restrict__ dgam,
                                                const double* __restrict__ S, const double* __restrict__ ell,
                                                const double* __restrict__ F, double* __restrict__ Fc,
                                                double* __restrict__ dFl, double* __restrict__ Fp,
                                                double* __restrict__ Sc, double* __restrict__ rho,
                                                const double* __restrict__ P, double* __restrict__ Pc, double b, double yc) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  double R[9], M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  const int g = grain[v];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __ldg(grainR + 9 * g + k);
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const double d = dgam[a * nvox + v];
    add_schmid(M, a, d);
    const double ad = fabs(d);
    const double r0 = rho[a * nvox + v];
    rho[a * nvox + v] = (r0 + ad / (b * ell[a * nvox + v])) / (1.0 + 2.0 * yc * ad / b);
  }
  double T[9], Ms[9], Fpo[9], Fpn[9];
  mat3_mult(M, R, T);
  mat3_mul(R, T, Ms);      // R M R^T
#pragma unroll
  for (int k = 0; k < 9; ++k) Fpo[k] = Fp[k * nvox + v];
  mat3_mul(Ms, Fpo, Fpn);
#pragma unroll
  for (int k = 0; k < 9; ++k) Fp[k * nvox + v] = Fpn[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) Sc[k * nvox + v] = S[k * nvox + v];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double f = F[k * nvox + v];
    dFl[k * nvox + v] = f - Fc[k * nvox + v];
    Fc[k * nvox + v] = f;
    Pc[k * nvox + v] = P[k * nvox + v];
  }
}

__device__ __forceinline__ void cauchy(const double* P, const double* F, double* sig) {
  double T[9];
  mat3_mult(P, F, T);      // P F^T
  const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                   F[2] * (F[3] * F[7] - F[4] * F[6]);
#pragma unroll
  for (int k = 0; k < 9; ++k) sig[k] = T[k] / J;
}

// partial sums of P, sigma, F (27 values) over the committed state
__global__ void __launch_bounds__(RVE_RED_THREADS) k_macro(size_t nvox, const double* __restrict__ P,
                                                           const double* __restrict__ F, double* __restrict__ partial) {
  __shared__ double sh[320];
  double acc[27];
#pragma unroll
  for (int c = 0; c < 27; ++c) acc[c] = 0.0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
    double Pv[9], Fv[9], sg[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { Pv[k] = P[k * nvox + v]; Fv[k] = F[k * nvox + v]; }
    cauchy(Pv, Fv, sg);
#pragma unroll
    for (int k = 0; k < 9; ++k) { acc[k] += Pv[k]; acc[9 + k] += sg[k]; acc[18 + k] += Fv[k]; }
  }
  for (int g = 0; g < 3; ++g) {
    double bs[9];
    blk_sums9<double>(acc + 9 * g, 0x1FFu, sh, bs);
    if (threadIdx.x == 0)
      for (int c = 0; c < 9; ++c) partial[(size_t)(9 * g + c) * gridDim.x + blockIdx.x] = bs[c];
  }
}

// derived output fields: 0 = Cauchy stress (9), 1 = von Mises (1), 2 = S in the sample frame (6)
__global__ void k_output(size_t nvox, int which, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
                         const double* __restrict__ P, const double* __restrict__ F, const double* __restrict__ Sc,
                         double* __restrict__ out) {
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  if (which == 2) {
    double R[9], Sf[9], T[9], Ss[9];
    const int g = grain[v];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = __ldg(grainR + 9 * g + k);
    double s6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) s6[k] = Sc[k * nvox + v];
    Sf[0] = s6[0]; Sf[4] = s6[1]; Sf[8] = s6[2];
    Sf[5] = Sf[7] = s6[3]; Sf[2] = Sf[6] = s6[4]; Sf[1] = Sf[3] = s6[5];
    mat3_mult(Sf, R, T);
    mat3_mul(R, T, Ss);    // R S R^T
    const int vi[6] = {0, 4, 8, 5, 2, 1};
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k * nvox + v] = Ss[vi[k]];
    return;
  }
  double Pv[9], Fv[9], sg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) { Pv[k] = P[k * nvox + v]; Fv[k] = F[k * nvox + v]; }
  cauchy(Pv, Fv, sg);
  if (which == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) out[k * nvox + v] = sg[k];
  } else {
    const double m = (sg[0] + sg[4] + sg[8]) / 3.0;
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double d = 0.5 * (sg[3 * i + j] + sg[3 * j + i]) - (i == j ? m : 0.0);
        s2 += d * d;
      }
    out[v] = sqrt(1.5 * s2);
  }
}

unsigned grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_tangent_apply(const rve_s* h, cudaStream_t s) {
  // one wave of resident blocks (three per SM): each thread covers more
  // voxels, so the block reduction of p . t is spread over more of them, and
  // no partial last wave trails
  const int blocks = std::min(RVE_RED_BLOCKS, 3 * h->num_sms);
  {
    ProfScope ps_(h, RVE_K_TANGENT_APPLY, s);
    k_tangent_apply<<<blocks, RVE_RED_THREADS, 0, s>>>(h->nvox, h->K[h->cur], h->r, h->p, h->t, h->dscal,
                                                       h->partial, (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_update(const rve_s* h, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_CG_UPDATE, s);
    k_cg_update<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, h->x, h->r, h->p, h->q, h->dscal, h->partial,
                                                           (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const rve_s* h, double eta, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_cg_init<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, h->x, h->r, h->R, h->dscal, eta, h->partial,
                                                         (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_norm2(const rve_s* h, const double* a, int ncomp, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_REDUCE, s);
    k_norm2<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>((size_t)ncomp * h->nvox, a, h->partial);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_final(h, RED_NORM, s);
}

cudaError_t launch_reduce_final(const rve_s* h, int mode, cudaStream_t s) {
  const int nval = mode == RED_MACRO ? 27 : 1;
  const int nparts = mode == RED_MACRO ? MACRO_BLOCKS : RVE_RED_BLOCKS;
  {
    ProfScope ps_(h, RVE_K_REDUCE, s);
    k_reduce_final<<<1, 1024, 0, s>>>(h->partial, nparts, nval, mode, h->dscal);
  }
  return cudaGetLastError();
}

cudaError_t launch_axpy_F(const rve_s* h, double lambda, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_axpy<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, h->F, h->x, lambda);
  }
  return cudaGetLastError();
}

cudaError_t launch_predictor(const rve_s* h, const double* dFb, const double* dFb_prev, double ratio,
                             int extrapolate, cudaStream_t s) {
  Nine sh;
  for (int k = 0; k < 9; ++k) sh.v[k] = dFb[k] - (extrapolate ? ratio * dFb_prev[k] : 0.0);
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_predictor<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, h->F, h->F_c, h->dF_last, sh, ratio, extrapolate);
  }
  return cudaGetLastError();
}

cudaError_t launch_shift_F(const rve_s* h, const double* shift, cudaStream_t s) {
  Nine sh;
  for (int k = 0; k < 9; ++k) sh.v[k] = shift[k];
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_predictor<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, h->F, h->F, h->dF_last, sh, 0.0, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_commit(const rve_s* h, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_commit<<<grid_for(h->nvox, 128), 128, 0, s>>>(h->nvox, h->grain, h->grainR, h->dgam[h->cur], h->S[h->cur],
                                                  h->ell, h->F, h->F_c, h->dF_last, h->Fp, h->S_c, h->rho_ssd,
                                                  h->P[h->cur], h->P_c, h->mat.b, h->mat.yc);
  }
  return cudaGetLastError();
}

cudaError_t launch_macro(const rve_s* h, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_REDUCE, s);
    k_macro<<<MACRO_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, h->P_c, h->F_c, h->partial);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_final(h, RED_MACRO, s);
}

cudaError_t launch_output_field(const rve_s* h, int which, const double* P, const double* S, double* dst,
                               cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_output<<<grid_for(h->nvox, 128), 128, 0, s>>>(h->nvox, which, h->grain, h->grainR, P, h->F_c, S, dst);
  }
  return cudaGetLastError();
}

cudaError_t vec_init() {
  return cudaFuncSetAttribute(k_tangent_apply32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TA_SMEM);
}

cudaError_t launch_tangent_apply32(const rve_s* h, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_TANGENT_APPLY, s);
    if (h->tma_apply)   // persistent: one block per SM
      k_tangent_apply32_tma<<<h->num_sms, TA_TV, TA_SMEM, s>>>(h->nvox, reinterpret_cast<const float*>(h->K[h->cur]),
                                                               h->r32, h->p32, h->t32, h->dscal, h->partial,
                                                               (unsigned int*)(h->dcount + 4), h->wait_polls);
    else
      k_tangent_apply32<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, reinterpret_cast<const float*>(h->K[h->cur]),
                                                                   h->r32, h->p32, h->t32, h->dscal, h->partial,
                                                                   (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_cg_init32(const rve_s* h, double eta, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_cg_init32<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, h->x32, h->r32, h->R, h->dscal, eta,
                                                           h->partial, (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_widen_x(const rve_s* h, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_widen<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, h->x32, h->x);
  }
  return cudaGetLastError();
}

cudaError_t launch_widen(const rve_s* h, const float* a, double* b, size_t n, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_widen<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(n, a, b);
  }
  return cudaGetLastError();
}

// ---- BiCGStab support (FP64): w = K : v; fused dot products; linear combinations
namespace {

template <typename KT>
__global__ void __launch_bounds__(RVE_RED_THREADS, 2) k_kmul(size_t nvox, const KT* __restrict__ K,
                                                             const double* __restrict__ in, double* __restrict__ out) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
    double pv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) pv[k] = in[k * nvox + v];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < 9; ++j) s = fma((double)__ldcs(K + (size_t)(9 * i + j) * nvox + v), pv[j], s);
      out[i * nvox + v] = s;
    }
  }
}

// up to three dot products a_k . b_k at once -> ds[slot + k]
__global__ void __launch_bounds__(RVE_RED_THREADS) k_dots(size_t n, int np, const double* __restrict__ a0,
                                                          const double* __restrict__ b0, const double* __restrict__ a1,
                                                          const double* __restrict__ b1, const double* __restrict__ a2,
                                                          const double* __restrict__ b2, double* __restrict__ ds,
                                                          int slot, double* __restrict__ partial,
                                                          unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    acc[0] = fma(a0[e], b0[e], acc[0]);
    if (np > 1) acc[1] = fma(a1[e], b1[e], acc[1]);
    if (np > 2) acc[2] = fma(a2[e], b2[e], acc[2]);
  }
  for (int c = 0; c < np; ++c) {
    const double s = blk_sum(acc[c], sh);
    if (threadIdx.x == 0) partial[(size_t)c * gridDim.x + blockIdx.x] = s;
  }
  double tot[3];
  if (last_block_sums(partial, np, ticket, sh, tot) && threadIdx.x == 0)
    for (int c = 0; c < np; ++c) ds[slot + c] = tot[c];
}

// out = c0 a0 + c1 a1 + c2 a2 (a1, a2 nullable; out may alias an input)
__global__ void k_lincomb(size_t n, double* out, double c0, const double* a0, double c1, const double* a1,
                          double c2, const double* a2) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    double v = c0 * a0[e];
    if (a1) v = fma(c1, a1[e], v);
    if (a2) v = fma(c2, a2[e], v);
    out[e] = v;
  }
}

// Means of the nine components of a field -> ds[slot + c] (last-block sum).
__global__ void __launch_bounds__(RVE_RED_THREADS) k_mean9(size_t nvox, const double* __restrict__ x,
                                                          double* __restrict__ ds, int slot,
                                                          double* __restrict__ partial,
                                                          unsigned int* __restrict__ ticket) {
  __shared__ double sh[320];
  double acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = 0.0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] += x[c * nvox + v];
  }
  double bs[9];
  blk_sums9<double>(acc, 0x1FFu, sh, bs);
  if (threadIdx.x == 0)
    for (int c = 0; c < 9; ++c) partial[(size_t)c * gridDim.x + blockIdx.x] = bs[c];
  double tot[9];
  if (last_block_sums(partial, 9, ticket, sh, tot) && threadIdx.x == 0)
    for (int c = 0; c < 9; ++c) ds[slot + c] = tot[c] / (double)nvox;
}

// x_c -= mean(x_c) on the components whose bit is set
__global__ void k_sub_means(size_t nvox, double* __restrict__ x, const double* __restrict__ ds, int slot,
                            unsigned bits) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c)
      if ((bits >> c) & 1u) x[c * nvox + v] -= ds[slot + c];
  }
}

}  // namespace

cudaError_t launch_zero_means(const rve_s* h, double* x, unsigned bits, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_REDUCE, s);
    k_mean9<<<MACRO_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, x, h->dscal, DS_XMEAN, h->partial,
                                                       (unsigned int*)(h->dcount + 4));
  }
  if (cudaError_t e = cudaGetLastError()) return e;
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_sub_means<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, x, h->dscal, DS_XMEAN, bits);
  }
  return cudaGetLastError();
}

cudaError_t launch_kmul(const rve_s* h, const double* in, double* out, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_TANGENT_APPLY, s);
    if (h->opt.precision == 1)   // the tangent is stored as float in mixed precision
      k_kmul<float><<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, reinterpret_cast<const float*>(h->K[h->cur]),
                                                               in, out);
    else
      k_kmul<double><<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(h->nvox, h->K[h->cur], in, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_dots(const rve_s* h, int np, const double* a0, const double* b0, const double* a1,
                        const double* b1, const double* a2, const double* b2, int slot, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_REDUCE, s);
    k_dots<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, np, a0, b0, a1, b1, a2, b2, h->dscal, slot,
                                                      h->partial, (unsigned int*)(h->dcount + 4));
  }
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const rve_s* h, double* out, double c0, const double* a0, double c1, const double* a1,
                           double c2, const double* a2, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_OTHER, s);
    k_lincomb<<<RVE_RED_BLOCKS, RVE_RED_THREADS, 0, s>>>(9 * h->nvox, out, c0, a0, c1, a1, c2, a2);
  }
  return cudaGetLastError();
}
