// Hand-written batched 3-D real FFT of tensor-component fields (FP64, and
// FP32 for the mixed-precision conjugate gradients), with the frequency-space operators of the method fused between the
// forward and inverse transforms along z:
//   - the Galerkin projection with mixed control (Sec. 2.2, Eqs. weakarbi,
//     eql_discrete2) built from the rotated-scheme frequencies (App. A, Eq. kas);
//   - the Nye tensor G_ij = -eps_jkl d_k Fp_il (App. B, Eq. nyeindexfourier)
//     with the same rotated-scheme derivative.
//
// Layout.  Real fields: [c][z][y][x] (x fastest).  Half spectrum:
// [c][z][y][kx], kx = 0..n0/2.  Passes (each a kernel, each transform staged
// in shared memory and done by a mixed-radix 8/4/2/3 Stockham autosort):
//   X  (R2C): two real rows y, y+1 packed as one complex row, one length-n0
//             FFT, then the two half spectra are separated;
//   Y  (C2C): tiles of consecutive kx columns, length-n1 FFTs;
//   Z  (C2C + operator + C2C): the three fields of one tensor row i for a tile
//             of (kx, ky) pencils (both operators act row by row), forward
//             z FFT, operator, inverse z FFT;
//   Y^-1, X^-1 (C2R).  The 1/nvox scaling is folded into the operator.
#include "common.cuh"
#include "rve_internal.h"

namespace {

// complex value and storage pair type of a real type R (double or float)
template <typename R> struct CX { R x, y; };
template <typename R> struct V2T;
template <> struct V2T<double> { typedef double2 t; };
template <> struct V2T<float> { typedef float2 t; };
template <typename R> using V2 = typename V2T<R>::t;

template <typename R> __device__ __forceinline__ CX<R> mk(R a, R b) { CX<R> c; c.x = a; c.y = b; return c; }
template <typename R> __device__ __forceinline__ CX<R> add(CX<R> a, CX<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ CX<R> sub(CX<R> a, CX<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ CX<R> scl(CX<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
template <typename R> __device__ __forceinline__ V2<R> st2(R a, R b) { V2<R> v; v.x = a; v.y = b; return v; }

struct PlanDev {
  int n, npass;
  int radix[RVE_MAX_RADIX_PASSES];
};

PlanDev to_dev(const FFTPlan& p) {
  PlanDev d;
  d.n = p.n;
  d.npass = p.npass;
  for (int i = 0; i < RVE_MAX_RADIX_PASSES; ++i) d.radix[i] = p.radix[i];
  return d;
}

// a * w or a * conj(w) (w from the forward table) with the sign fixed at
// compile time, so the negation folds into the FMA operands; float
// transforms read the float table
template <int SIGN, typename R>
__device__ __forceinline__ CX<R> twiddle(CX<R> a, const V2<R>* tw, int idx) {
  const V2<R> w = __ldg(tw + idx);
  if (SIGN < 0) return mk<R>(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
  return mk<R>(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}

template <int SIGN, typename R>
__device__ __forceinline__ CX<R> mul_i(CX<R> a) { return SIGN > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x); }

// One Stockham pass of radix R over `howmany` contiguous transforms of length
// N from src to dst (both shared memory).
template <int SIGN, typename RT>
__device__ void stockham_pass(const CX<RT>* __restrict__ src, CX<RT>* __restrict__ dst, int N, int howmany,
                              int R, int Ns, const V2<RT>* tw) {
  typedef CX<RT> cplx;
  const int nb = N / R;
  const int total = nb * howmany;
  const int twstep = N / (Ns * R);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int tr = b / nb;
    const int j = b - tr * nb;
    const int k = j % Ns;
    const cplx* X = src + tr * N;
    cplx* Y = dst + tr * N;
    const int d = (j / Ns) * Ns * R + k;
    if (R == 8) {
      // radix 8 as a radix-2 step (a_m +/- a_{m+4}), the factors W8^m on the
      // differences, then two radix-4 DFTs (even and odd outputs)
      cplx a[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) a[m] = X[j + m * nb];
      if (k) {
#pragma unroll
        for (int m = 1; m < 8; ++m) a[m] = twiddle<SIGN, RT>(a[m], tw, m * k * twstep);
      }
      const RT r2 = (RT)0.70710678118654752440;    // 1/sqrt(2)
      cplx b[4], c[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) { b[m] = add(a[m], a[m + 4]); c[m] = sub(a[m], a[m + 4]); }
      // c1 *= W8^(sign), c2 *= -/+ i, c3 *= W8^(3 sign)
      {
        const cplx c1 = c[1], c3 = c[3];
        if (SIGN < 0) {
          c[1] = mk<RT>(r2 * (c1.x + c1.y), r2 * (c1.y - c1.x));
          c[3] = mk<RT>(r2 * (c3.y - c3.x), -r2 * (c3.x + c3.y));
        } else {
          c[1] = mk<RT>(r2 * (c1.x - c1.y), r2 * (c1.x + c1.y));
          c[3] = mk<RT>(-r2 * (c3.x + c3.y), r2 * (c3.x - c3.y));
        }
        c[2] = mul_i<SIGN, RT>(c[2]);
      }
      const cplx t0 = add(b[0], b[2]), t1 = sub(b[0], b[2]), t2 = add(b[1], b[3]), t3 = mul_i<SIGN, RT>(sub(b[1], b[3]));
      const cplx u0 = add(c[0], c[2]), u1 = sub(c[0], c[2]), u2 = add(c[1], c[3]), u3 = mul_i<SIGN, RT>(sub(c[1], c[3]));
      Y[d] = add(t0, t2);
      Y[d + 4 * Ns] = sub(t0, t2);
      Y[d + 2 * Ns] = add(t1, t3);
      Y[d + 6 * Ns] = sub(t1, t3);
      Y[d + Ns] = add(u0, u2);
      Y[d + 5 * Ns] = sub(u0, u2);
      Y[d + 3 * Ns] = add(u1, u3);
      Y[d + 7 * Ns] = sub(u1, u3);
    } else if (R == 4) {
      cplx a0 = X[j], a1 = X[j + nb], a2 = X[j + 2 * nb], a3 = X[j + 3 * nb];
      if (k) {
        a1 = twiddle<SIGN, RT>(a1, tw, k * twstep);
        a2 = twiddle<SIGN, RT>(a2, tw, 2 * k * twstep);
        a3 = twiddle<SIGN, RT>(a3, tw, 3 * k * twstep);
      }
      cplx t0 = add(a0, a2), t1 = sub(a0, a2), t2 = add(a1, a3), t3 = mul_i<SIGN, RT>(sub(a1, a3));
      Y[d] = add(t0, t2);
      Y[d + Ns] = add(t1, t3);
      Y[d + 2 * Ns] = sub(t0, t2);
      Y[d + 3 * Ns] = sub(t1, t3);
    } else if (R == 2) {
      cplx a0 = X[j], a1 = X[j + nb];
      if (k) a1 = twiddle<SIGN, RT>(a1, tw, k * twstep);
      Y[d] = add(a0, a1);
      Y[d + Ns] = sub(a0, a1);
    } else {  // R == 3
      cplx a0 = X[j], a1 = X[j + nb], a2 = X[j + 2 * nb];
      if (k) {
        a1 = twiddle<SIGN, RT>(a1, tw, k * twstep);
        a2 = twiddle<SIGN, RT>(a2, tw, 2 * k * twstep);
      }
      const RT s3 = (RT)0.86602540378443864676;  // sqrt(3)/2
      cplx t = add(a1, a2);
      cplx u = scl(mul_i<SIGN, RT>(sub(a1, a2)), s3);
      cplx m = mk<RT>(fma((RT)-0.5, t.x, a0.x), fma((RT)-0.5, t.y, a0.y));
      Y[d] = add(a0, t);
      Y[d + Ns] = add(m, u);
      Y[d + 2 * Ns] = sub(m, u);
    }
  }
}

// Full transform of `howmany` contiguous length-N sequences; the caller has
// synchronised after filling `a`.  Returns the buffer that holds the result.
template <int SIGN, typename RT>
__device__ CX<RT>* block_fft(CX<RT>* a, CX<RT>* b, const PlanDev& pl, int howmany, const V2<RT>* tw) {
  int Ns = 1;
  for (int p = 0; p < pl.npass; ++p) {
    const int R = pl.radix[p];
    stockham_pass<SIGN, RT>(a, b, pl.n, howmany, R, Ns, tw);
    __syncthreads();
    CX<RT>* t = a; a = b; b = t;
    Ns *= R;
  }
  return a;
}

// ---------------------------------------------------------------- pass X (R2C)
// in: real fields (type R); spec: half spectrum (pairs of R)
template <typename R>
__global__ void __launch_bounds__(256) k_fft_x_r2c(const R* __restrict__ in, V2<R>* __restrict__ spec,
                                                   int n0, int n1, int n2, int nkx, int rpb, PlanDev pl,
                                                   const V2<R>* __restrict__ tw, const double* __restrict__ done) {
  typedef CX<R> cplx;
  if (done && *done != 0.0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx* a = reinterpret_cast<cplx*>(smraw);
  cplx* b = a + rpb * n0;
  const int f = blockIdx.z, z = blockIdx.y, j0 = blockIdx.x * rpb;
  const size_t nvox = (size_t)n0 * n1 * n2;
  const R* src = in + f * nvox + (size_t)z * n1 * n0;
  for (int e = threadIdx.x; e < rpb * n0; e += blockDim.x) {
    const int jj = e / n0, x = e - jj * n0;
    const int y0 = 2 * (j0 + jj);
    a[e] = mk<R>(src[(size_t)y0 * n0 + x], src[(size_t)(y0 + 1) * n0 + x]);
  }
  __syncthreads();
  cplx* res = block_fft<-1, R>(a, b, pl, rpb, tw);
  V2<R>* dst = spec + ((size_t)f * n2 + z) * n1 * nkx;
  // the two half spectra are Z(k) +/- conj(Z(n0 - k)) without the factor 1/2
  // of the split: every operator applied between the z passes carries it in
  // its 1/nvox (SPEC_SCALE), exactly, as a power of two
  for (int e = threadIdx.x; e < rpb * nkx; e += blockDim.x) {
    const int jj = e / nkx, k = e - jj * nkx;
    const cplx zk = res[jj * n0 + k];
    const cplx zc = res[jj * n0 + (k == 0 ? 0 : n0 - k)];
    const cplx zm = mk<R>(zc.x, -zc.y);
    const cplx s = add(zk, zm), d = sub(zk, zm);
    const int y0 = 2 * (j0 + jj);
    dst[(size_t)y0 * nkx + k] = st2<R>(s.x, s.y);
    dst[(size_t)(y0 + 1) * nkx + k] = st2<R>(d.y, -d.x);
  }
}

// ---------------------------------------------------------------- pass X^-1 (C2R)
template <typename R>
__global__ void __launch_bounds__(256) k_fft_x_c2r(const V2<R>* __restrict__ spec, R* __restrict__ out,
                                                   int n0, int n1, int n2, int nkx, int rpb, PlanDev pl,
                                                   const V2<R>* __restrict__ tw, const double* __restrict__ done) {
  typedef CX<R> cplx;
  if (done && *done != 0.0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx* a = reinterpret_cast<cplx*>(smraw);
  cplx* b = a + rpb * n0;
  const int f = blockIdx.z, z = blockIdx.y, j0 = blockIdx.x * rpb;
  const size_t nvox = (size_t)n0 * n1 * n2;
  const V2<R>* src = spec + ((size_t)f * n2 + z) * n1 * nkx;
  for (int e = threadIdx.x; e < rpb * n0; e += blockDim.x) {
    const int jj = e / n0, k = e - jj * n0;
    const int y0 = 2 * (j0 + jj);
    cplx A, B;
    if (k < nkx) {
      V2<R> u = src[(size_t)y0 * nkx + k], v = src[(size_t)(y0 + 1) * nkx + k];
      A = mk<R>(u.x, u.y); B = mk<R>(v.x, v.y);
    } else {
      V2<R> u = src[(size_t)y0 * nkx + (n0 - k)], v = src[(size_t)(y0 + 1) * nkx + (n0 - k)];
      A = mk<R>(u.x, -u.y); B = mk<R>(v.x, -v.y);
    }
    a[e] = mk<R>(A.x - B.y, A.y + B.x);  // A + i B
  }
  __syncthreads();
  cplx* res = block_fft<+1, R>(a, b, pl, rpb, tw);
  R* dst = out + f * nvox + (size_t)z * n1 * n0;
  for (int e = threadIdx.x; e < rpb * n0; e += blockDim.x) {
    const int jj = e / n0, x = e - jj * n0;
    const int y0 = 2 * (j0 + jj);
    dst[(size_t)y0 * n0 + x] = res[e].x;
    dst[(size_t)(y0 + 1) * n0 + x] = res[e].y;
  }
}

// ---------------------------------------------------------------- pass Y (C2C)
template <int SIGN, typename R>
__global__ void __launch_bounds__(256) k_fft_y(V2<R>* __restrict__ spec, int n1, int n2, int nkx, int tx,
                                               PlanDev pl, const V2<R>* __restrict__ tw,
                                               const double* __restrict__ done) {
  typedef CX<R> cplx;
  if (done && *done != 0.0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx* a = reinterpret_cast<cplx*>(smraw);
  cplx* b = a + tx * n1;
  const int f = blockIdx.z, z = blockIdx.y, kx0 = blockIdx.x * tx;
  V2<R>* base = spec + ((size_t)f * n2 + z) * n1 * nkx;
  for (int e = threadIdx.x; e < tx * n1; e += blockDim.x) {
    const int y = e / tx, t = e - y * tx;
    const int kx = kx0 + t;
    V2<R> v = kx < nkx ? base[(size_t)y * nkx + kx] : st2<R>((R)0, (R)0);
    a[t * n1 + y] = mk<R>(v.x, v.y);
  }
  __syncthreads();
  cplx* res = block_fft<SIGN, R>(a, b, pl, tx, tw);
  for (int e = threadIdx.x; e < tx * n1; e += blockDim.x) {
    const int y = e / tx, t = e - y * tx;
    const int kx = kx0 + t;
    if (kx < nkx) {
      cplx v = res[t * n1 + y];
      base[(size_t)y * nkx + kx] = st2<R>(v.x, v.y);
    }
  }
}

struct OpTables {
  const double* lapw;   // OP_LAPINV weight per spectrum point, SPEC_SCALE included (FP64 path)
  const double* s20; const double* s21; const double* s22;
  const double* c20; const double* c21; const double* c22;
  const double* tan0; const double* tan1; const double* tan2;
  const int8_t* nyq0; const int8_t* nyq1; const int8_t* nyq2;
  const double2* ph0; const double2* ph1; const double2* ph2;
  const double* xi0; const double* xi1; const double* xi2;
};

// The forward transform leaves the spectrum at 1 / SPEC_SCALE = 2 times its
// value (see the X pass); the operators scale by SPEC_SCALE / nvox.
constexpr double SPEC_SCALE = 0.5;

// Inverse-Laplacian weight of OP_LAPINV at one frequency, with SPEC_SCALE:
// SPEC_SCALE / (64 nvox sum_m s2_m prod_{j!=m} c2_j), 0 where it vanishes
__device__ __forceinline__ double lapinv_weight(const OpTables& T, double inv_nvox, int kx, int ky, int kz) {
  const double sx = T.s20[kx], sy = T.s21[ky], sz = T.s22[kz];
  const double cx = T.c20[kx], cy = T.c21[ky], cz = T.c22[kz];
  const double lap = fma(sx, cy * cz, fma(cx, sy * cz, cx * cy * sz));
  return lap > 0.0 ? (SPEC_SCALE * inv_nvox) / (64.0 * lap) : 0.0;
}

// Operator at one frequency on the three fields of a tensor row (in double).
__device__ __forceinline__ void apply_op(const OpTables& T, const SpecParams& sp, int i, int kx, int ky, int kz,
                                         size_t kidx, cplx& X0, cplx& X1, cplx& X2) {
  cplx Y0, Y1, Y2;
  const double sc = SPEC_SCALE * sp.inv_nvox;
  if (sp.op == OP_LAPINV) {
    const double w = T.lapw ? __ldg(T.lapw + kidx) : lapinv_weight(T, sp.inv_nvox, kx, ky, kz);
    Y0 = cscale(X0, w); Y1 = cscale(X1, w); Y2 = cscale(X2, w);
  } else if (sp.op == OP_PROJECT) {
    if (kx == 0 && ky == 0 && kz == 0) {
      if (sp.mean_out) {
        sp.mean_out[3 * i + 0] = X0.x * sc;
        sp.mean_out[3 * i + 1] = X1.x * sc;
        sp.mean_out[3 * i + 2] = X2.x * sc;
      }
      const double nv = 1.0 / sp.inv_nvox;
      Y0 = sp.keep[3 * i + 0] ? cmk((SPEC_SCALE * X0.x - nv * sp.shift[3 * i + 0]) * sp.inv_nvox, X0.y * sc) : cmk(0.0, 0.0);
      Y1 = sp.keep[3 * i + 1] ? cmk((SPEC_SCALE * X1.x - nv * sp.shift[3 * i + 1]) * sp.inv_nvox, X1.y * sc) : cmk(0.0, 0.0);
      Y2 = sp.keep[3 * i + 2] ? cmk((SPEC_SCALE * X2.x - nv * sp.shift[3 * i + 2]) * sp.inv_nvox, X2.y * sc) : cmk(0.0, 0.0);
    } else {
      const int q0 = T.nyq0[kx], q1 = T.nyq1[ky], q2 = T.nyq2[kz];
      double u0, u1, u2;
      if (q0 + q1 + q2 >= 2) {
        u0 = u1 = u2 = 0.0;
      } else if (q0 + q1 + q2 == 1) {
        u0 = q0; u1 = q1; u2 = q2;
      } else {
        const double t0 = T.tan0[kx], t1 = T.tan1[ky], t2 = T.tan2[kz];
        const double inv = rsqrt(fma(t0, t0, fma(t1, t1, t2 * t2)));
        u0 = t0 * inv; u1 = t1 * inv; u2 = t2 * inv;
      }
      // (G X)_ij = u_j sum_l X_il u_l  (scaled by SPEC_SCALE / nvox)
      cplx s = cmk(fma(X0.x, u0, fma(X1.x, u1, X2.x * u2)), fma(X0.y, u0, fma(X1.y, u1, X2.y * u2)));
      s = cscale(s, sc);
      Y0 = cscale(s, u0); Y1 = cscale(s, u1); Y2 = cscale(s, u2);
    }
  } else if (sp.op == OP_CURL_STD) {
    // the standard spectral derivative i xi_k / h (no rotated stencil)
    const double scd = 4.0 * sp.inv4h * sc;
    const cplx D0 = cmk(0.0, T.xi0[kx] * scd), D1 = cmk(0.0, T.xi1[ky] * scd), D2 = cmk(0.0, T.xi2[kz] * scd);
    Y0 = csub(cmul(D2, X1), cmul(D1, X2));
    Y1 = csub(cmul(D0, X2), cmul(D2, X0));
    Y2 = csub(cmul(D1, X0), cmul(D0, X1));
  } else {  // OP_CURL: G_ij = -eps_jkl D_k Fp_il
    const double2 e0 = T.ph0[kx], e1 = T.ph1[ky], e2 = T.ph2[kz];
    const cplx p0 = cmk(1.0 + e0.x, e0.y), p1 = cmk(1.0 + e1.x, e1.y), p2 = cmk(1.0 + e2.x, e2.y);
    const cplx m0 = cmk(e0.x - 1.0, e0.y), m1 = cmk(e1.x - 1.0, e1.y), m2 = cmk(e2.x - 1.0, e2.y);
    const double scd = sp.inv4h * sc;
    const cplx D0 = cscale(cmul(m0, cmul(p1, p2)), scd);
    const cplx D1 = cscale(cmul(p0, cmul(m1, p2)), scd);
    const cplx D2 = cscale(cmul(p0, cmul(p1, m2)), scd);
    Y0 = csub(cmul(D2, X1), cmul(D1, X2));
    Y1 = csub(cmul(D0, X2), cmul(D2, X0));
    Y2 = csub(cmul(D1, X0), cmul(D0, X1));
  }
  X0 = Y0; X1 = Y1; X2 = Y2;
}

// inverse-Laplacian weight in float for the float path (SPEC_SCALE included
// through the caller's scale)
__device__ __forceinline__ float lapinv_weight_f(const OpTables& T, float scale, int kx, int ky, int kz) {
  const float sx = (float)T.s20[kx], sy = (float)T.s21[ky], sz = (float)T.s22[kz];
  const float cx = (float)T.c20[kx], cy = (float)T.c21[ky], cz = (float)T.c22[kz];
  const float lap = fmaf(sx, cy * cz, fmaf(cx, sy * cz, cx * cy * sz));
  return lap > 0.0f ? scale / (64.0f * lap) : 0.0f;
}

// the OP_LAPINV weight of every spectrum point (layout of one field's half
// spectrum, [kz][ky][kx]), built once per handle
__global__ void k_lapinv_table(double* __restrict__ w, OpTables T, int nkx, int n1, int n2, double inv_nvox) {
  const size_t n = (size_t)nkx * n1 * n2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(e % nkx), ky = (int)((e / nkx) % n1), kz = (int)(e / ((size_t)nkx * n1));
    w[e] = lapinv_weight(T, inv_nvox, kx, ky, kz);
  }
}

// ---------------------------------------------------------------- pass Z + operator
template <typename R>
__global__ void __launch_bounds__(256) k_fft_z_op(V2<R>* __restrict__ spec, int n1, int n2, int nkx, int tx,
                                                  PlanDev pl, const V2<R>* __restrict__ tw, OpTables T,
                                                  SpecParams sp, const double* __restrict__ done) {
  typedef CX<R> cx;
  if (done && *done != 0.0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int cnt = 3 * tx * n2;
  cx* a = reinterpret_cast<cx*>(smraw);
  cx* b = a + cnt;
  const int i = blockIdx.z, ky = blockIdx.y, kx0 = blockIdx.x * tx;
  const size_t zstride = (size_t)n1 * nkx;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int c = e / (tx * n2);
    const int rem = e - c * tx * n2;
    const int z = rem / tx, t = rem - z * tx;
    const int kx = kx0 + t;
    const size_t f = 3 * i + c;
    V2<R> v = kx < nkx ? spec[(f * n2 + z) * zstride + (size_t)ky * nkx + kx] : st2<R>((R)0, (R)0);
    a[(c * tx + t) * n2 + z] = mk<R>(v.x, v.y);
  }
  __syncthreads();
  cx* res = block_fft<-1, R>(a, b, pl, 3 * tx, tw);
  cx* oth = (res == a) ? b : a;
  const float inv_nvox_f = (float)(SPEC_SCALE * sp.inv_nvox);
  for (int e = threadIdx.x; e < tx * n2; e += blockDim.x) {
    const int t = e / n2, z = e - t * n2;
    const int kx = kx0 + t;
    cx Y0 = res[(0 * tx + t) * n2 + z], Y1 = res[(1 * tx + t) * n2 + z], Y2 = res[(2 * tx + t) * n2 + z];
    if (kx >= nkx) {
      Y0 = Y1 = Y2 = mk<R>((R)0, (R)0);
    } else if (sizeof(R) == 4) {
      // float path: the inverse Laplacian is the only operator it carries
      const R w = (R)lapinv_weight_f(T, inv_nvox_f, kx, ky, z);
      Y0 = scl(Y0, w); Y1 = scl(Y1, w); Y2 = scl(Y2, w);
    } else {
      cplx X0 = cmk((double)Y0.x, (double)Y0.y), X1 = cmk((double)Y1.x, (double)Y1.y),
           X2 = cmk((double)Y2.x, (double)Y2.y);
      apply_op(T, sp, i, kx, ky, z, ((size_t)z * gridDim.y + ky) * nkx + kx, X0, X1, X2);
      Y0 = mk<R>((R)X0.x, (R)X0.y); Y1 = mk<R>((R)X1.x, (R)X1.y); Y2 = mk<R>((R)X2.x, (R)X2.y);
    }
    oth[(0 * tx + t) * n2 + z] = Y0;
    oth[(1 * tx + t) * n2 + z] = Y1;
    oth[(2 * tx + t) * n2 + z] = Y2;
  }
  __syncthreads();
  cx* res2 = block_fft<+1, R>(oth, res, pl, 3 * tx, tw);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int c = e / (tx * n2);
    const int rem = e - c * tx * n2;
    const int z = rem / tx, t = rem - z * tx;
    const int kx = kx0 + t;
    if (kx < nkx) {
      const size_t f = 3 * i + c;
      cx v = res2[(c * tx + t) * n2 + z];
      spec[(f * n2 + z) * zstride + (size_t)ky * nkx + kx] = st2<R>(v.x, v.y);
    }
  }
}

// Tile sizes: as large as shared memory allows (up to 1024 complex per
// transform batch, 512 in the z pass that holds three fields), shrunk while
// the grid would fill less than four blocks per SM, down to 256 elements.

int rows_per_block(int n0, int n1, int n2, int nf, int fill) {
  int r = 1024 / n0;
  if (r < 1) r = 1;
  if (r > n1 / 2) r = n1 / 2;
  while (r > 1 && (n1 / 2) % r) --r;
  while (r > 1 && (long)(n1 / 2 / r) * n2 * nf < fill && r * n0 > 256) {
    int q = r / 2;
    while (q > 1 && (n1 / 2) % q) --q;
    r = q;
  }
  return r;
}
int tile_y(int n1, int n2, int nkx, int nf, int fill) {
  int t = 1024 / n1;
  if (t > 16) t = 16;
  if (t < 1) t = 1;
  while (t > 1 && (long)((nkx + t - 1) / t) * n2 * nf < fill && t * n1 > 256) t /= 2;
  return t;
}
int tile_z(int n1, int n2, int nkx, int nf, int fill) {
  int t = 512 / n2;
  if (t > 16) t = 16;
  if (t < 1) t = 1;
  while (t > 1 && (long)((nkx + t - 1) / t) * n1 * (nf / 3) < fill && 3 * t * n2 > 256) t /= 2;
  return t;
}
// threads for a block holding `elems` complex values: one per `per` values
// (the x and y passes: one butterfly of the plan's largest radix, its first
// pass, per thread; the z pass, whose tiles are narrow and few per SM, keeps
// one thread per four values for the warps that hide its latency)
int threads_for(int elems, int per) {
  int t = (elems / per + 31) / 32 * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}
int first_radix(const FFTPlan& pl) { return pl.npass > 0 ? pl.radix[0] : 4; }

OpTables op_tables(const rve_s* h) {
  OpTables T;
  T.lapw = h->lapw;
  T.tan0 = h->ax[0].tanh_; T.tan1 = h->ax[1].tanh_; T.tan2 = h->ax[2].tanh_;
  T.nyq0 = h->ax[0].nyq; T.nyq1 = h->ax[1].nyq; T.nyq2 = h->ax[2].nyq;
  T.ph0 = h->ax[0].ph; T.ph1 = h->ax[1].ph; T.ph2 = h->ax[2].ph;
  T.xi0 = h->ax[0].xi; T.xi1 = h->ax[1].xi; T.xi2 = h->ax[2].xi;
  T.s20 = h->ax[0].s2; T.s21 = h->ax[1].s2; T.s22 = h->ax[2].s2;
  T.c20 = h->ax[0].c2; T.c21 = h->ax[1].c2; T.c22 = h->ax[2].c2;
  return T;
}

template <typename R> const V2<R>* twt(const rve_s* h, int a);
template <> const double2* twt<double>(const rve_s* h, int a) { return h->ax[a].tw; }
template <> const float2* twt<float>(const rve_s* h, int a) { return h->ax[a].tw32; }
template <typename R> V2<R>* spect(const rve_s* h);
template <> double2* spect<double>(const rve_s* h) { return h->spec; }
template <> float2* spect<float>(const rve_s* h) { return h->spec32; }

template <typename R>
cudaError_t fwd(const rve_s* h, const R* in, cudaStream_t s, const double* done, int nf) {
  const int rpb = rows_per_block(h->n0, h->n1, h->n2, nf, h->fft_fill);
  dim3 gx(h->n1 / 2 / rpb, h->n2, nf);
  size_t shx = 2 * (size_t)rpb * h->n0 * sizeof(CX<R>);
  {
    ProfScope ps_(h, h->fft_cat >= 0 ? h->fft_cat : RVE_K_FFT_X_R2C, s);
    k_fft_x_r2c<R><<<gx, threads_for(rpb * h->n0, first_radix(h->plan[0])), shx, s>>>(in, spect<R>(h), h->n0, h->n1, h->n2, h->nkx, rpb,
                                                             to_dev(h->plan[0]), twt<R>(h, 0), done);
  }
  const int ty = tile_y(h->n1, h->n2, h->nkx, nf, h->fft_fill_y);
  dim3 gy((h->nkx + ty - 1) / ty, h->n2, nf);
  size_t shy = 2 * (size_t)ty * h->n1 * sizeof(CX<R>);
  {
    ProfScope ps_(h, h->fft_cat >= 0 ? h->fft_cat : RVE_K_FFT_Y, s);
    k_fft_y<-1, R><<<gy, threads_for(ty * h->n1, first_radix(h->plan[1])), shy, s>>>(spect<R>(h), h->n1, h->n2, h->nkx, ty,
                                                            to_dev(h->plan[1]), twt<R>(h, 1), done);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t zop(const rve_s* h, const SpecParams& sp, cudaStream_t s, const double* done, int nf) {
  const int tz = tile_z(h->n1, h->n2, h->nkx, nf, h->fft_fill_z);
  dim3 g((h->nkx + tz - 1) / tz, h->n1, nf / 3);
  size_t sh = 2 * 3 * (size_t)tz * h->n2 * sizeof(CX<R>);
  const int zthreads = threads_for(3 * tz * h->n2, 4);
  {
    ProfScope ps_(h, h->fft_cat >= 0 ? h->fft_cat : RVE_K_FFT_Z_OP, s);
    k_fft_z_op<R><<<g, zthreads, sh, s>>>(spect<R>(h), h->n1, h->n2, h->nkx, tz, to_dev(h->plan[2]), twt<R>(h, 2),
                                          op_tables(h), sp, done);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t inv(const rve_s* h, R* out, cudaStream_t s, const double* done, int nf) {
  const int ty = tile_y(h->n1, h->n2, h->nkx, nf, h->fft_fill_y);
  dim3 gy((h->nkx + ty - 1) / ty, h->n2, nf);
  size_t shy = 2 * (size_t)ty * h->n1 * sizeof(CX<R>);
  {
    ProfScope ps_(h, h->fft_cat >= 0 ? h->fft_cat : RVE_K_FFT_Y_INV, s);
    k_fft_y<+1, R><<<gy, threads_for(ty * h->n1, first_radix(h->plan[1])), shy, s>>>(spect<R>(h), h->n1, h->n2, h->nkx, ty,
                                                            to_dev(h->plan[1]), twt<R>(h, 1), done);
  }
  const int rpb = rows_per_block(h->n0, h->n1, h->n2, nf, h->fft_fill);
  dim3 gx(h->n1 / 2 / rpb, h->n2, nf);
  size_t shx = 2 * (size_t)rpb * h->n0 * sizeof(CX<R>);
  {
    ProfScope ps_(h, h->fft_cat >= 0 ? h->fft_cat : RVE_K_FFT_X_C2R, s);
    k_fft_x_c2r<R><<<gx, threads_for(rpb * h->n0, first_radix(h->plan[0])), shx, s>>>(spect<R>(h), out, h->n0, h->n1, h->n2, h->nkx, rpb,
                                                             to_dev(h->plan[0]), twt<R>(h, 0), done);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lapinv_table(const rve_s* h, cudaStream_t s) {
  if (!h->lapw) return cudaSuccess;
  k_lapinv_table<<<RVE_RED_BLOCKS, 256, 0, s>>>(h->lapw, op_tables(h), h->nkx, h->n1, h->n2, 1.0 / (double)h->nvox);
  return cudaGetLastError();
}

void make_plan(int n, FFTPlan* p, int max_radix) {
  p->n = n;
  p->npass = 0;
  int m = n;
  while (max_radix >= 8 && m % 8 == 0) { p->radix[p->npass++] = 8; m /= 8; }
  while (m % 4 == 0) { p->radix[p->npass++] = 4; m /= 4; }
  if (m % 2 == 0) { p->radix[p->npass++] = 2; m /= 2; }
  while (m % 3 == 0) { p->radix[p->npass++] = 3; m /= 3; }
  if (m != 1) p->npass = -1;  // unsupported length
}

cudaError_t launch_fft_forward(const rve_s* h, const double* in, cudaStream_t s, const double* done, int nf) {
  return fwd<double>(h, in, s, done, nf);
}
cudaError_t launch_fft_op(const rve_s* h, const SpecParams& sp, cudaStream_t s, const double* done, int nf) {
  return zop<double>(h, sp, s, done, nf);
}
cudaError_t launch_fft_inverse(const rve_s* h, double* out, cudaStream_t s, const double* done, int nf) {
  return inv<double>(h, out, s, done, nf);
}
cudaError_t launch_fft_forward32(const rve_s* h, const float* in, cudaStream_t s, const double* done) {
  return fwd<float>(h, in, s, done, 3);
}
cudaError_t launch_fft_lapinv32(const rve_s* h, const SpecParams& sp, cudaStream_t s, const double* done) {
  return zop<float>(h, sp, s, done, 3);
}
cudaError_t launch_fft_inverse32(const rve_s* h, float* out, cudaStream_t s, const double* done) {
  return inv<float>(h, out, s, done, 3);
}
