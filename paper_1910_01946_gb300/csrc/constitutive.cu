// Per-voxel kernels of the strain-gradient crystal-plasticity model (FP64,
// one voxel per thread, structure-of-arrays fields):
//
//   k_hardening    GND densities from the Nye tensor by the minimum-norm
//                  inverse of G = A rho (Eqs. defA2, mingnd), the Taylor
//                  critical resolved shear stress (Eq. Taylor_hard, with the
//                  lattice friction tau0 and Taylor coefficient alpha) and the
//                  mean free path (Eq. meanfree), frozen for the increment.
//   k_constitutive the implicit update of Sec. 2.1 (Eqs. 1-5, power law,
//                  Eq. Piola) by Newton on the second Piola-Kirchhoff stress S,
//                  and the consistent tangent dP/dF (Eq. linequil2ast).
//
// Everything inside a voxel is done in its grain's crystal frame, where the
// stiffness is cubic (three constants) and the Schmid tensors s (x) m are
// compile-time constants with entries 0, +-1/sqrt6: with X~ = R^T X R for
// every second-order tensor (R: crystal -> sample), the update is covariant,
// so F is rotated in and P, dP/dF are rotated out.
//
// Time integration (the paper gives none): backward Euler,
//   Fp = (I + sum_a dgam^a s^a (x) m^a) Fp_prev,
//   dgam^a = dt gdot0 |tau^a / tauc^a|^n sgn tau^a,  tau^a = S : s^a (x) m^a,
// residual r(S) = S - C : (Fe^T Fe - I)/2, Fe = F Fp^-1, solved from a warm
// start with the exact Jacobian and step halving (a step is taken only if it
// lowers max|r| and keeps every |dgam| <= dgam_max).
#include <algorithm>

#include "common.cuh"
#include "rve_internal.h"

namespace {

constexpr double INV_SQRT6 = 0.40824829046386301637;

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  while (n) {
    if (n & 1) r *= x;
    x *= x;
    n >>= 1;
  }
  return r;
}

// |x|^n and |x|^(n-1) of the flow rule: the exponent n = 20 of the materials
// here (rate sensitivity m = 1/n = 0.05) in five and six multiplications,
// the same products in the same order as ipow's (bit-identical)
__device__ __forceinline__ double pow_n(const Consts& c, double x) {
  if (c.n_int == 20) {
    const double x2 = x * x, x4 = x2 * x2, x8 = x4 * x4, x16 = x8 * x8;
    return x4 * x16;
  }
  return c.n_int ? ipow(x, c.n_int) : pow(x, c.n);
}
__device__ __forceinline__ double pow_n1(const Consts& c, double x) {
  if (c.n_int == 20) {
    const double x2 = x * x, x3 = x * x2, x4 = x2 * x2, x8 = x4 * x4, x16 = x8 * x8;
    return x3 * x16;
  }
  return c.n_int ? ipow(x, c.n_int - 1) : pow(x, c.n - 1.0);
}

// Coefficients of tau^a = S : s^a (x) m^a (times sqrt 6) on the Voigt
// components (11, 22, 33, 23, 13, 12) of a symmetric S
__host__ __device__ constexpr int tau_coef(int a, int k) {
  return k < 3 ? fcc_s(a, k) * fcc_m(a, k)
               : (k == 3 ? fcc_s(a, 1) * fcc_m(a, 2) + fcc_s(a, 2) * fcc_m(a, 1)
                         : (k == 4 ? fcc_s(a, 0) * fcc_m(a, 2) + fcc_s(a, 2) * fcc_m(a, 0)
                                   : fcc_s(a, 0) * fcc_m(a, 1) + fcc_s(a, 1) * fcc_m(a, 0)));
}

// tau^a = S : s^a (x) m^a for symmetric S in Voigt order (11,22,33,23,13,12)
__device__ __forceinline__ double resolved(const double* S, int a) {
  bool first = true;
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) t = cacc(t, first, tau_coef(a, k), S[k]);
  return t * INV_SQRT6;
}

// cubic stiffness applied to a symmetric strain given by its tensor components
// (E11, E22, E33, E23, E13, E12) -> stress in Voigt order
__device__ __forceinline__ void cubic(const Consts& c, const double* E, double* S) {
  S[0] = fma(c.C11, E[0], c.C12 * (E[1] + E[2]));
  S[1] = fma(c.C11, E[1], c.C12 * (E[0] + E[2]));
  S[2] = fma(c.C11, E[2], c.C12 * (E[0] + E[1]));
  S[3] = 2.0 * c.C44 * E[3];
  S[4] = 2.0 * c.C44 * E[4];
  S[5] = 2.0 * c.C44 * E[5];
}

__device__ __forceinline__ void sym_full(const double* v, double* X) {
  X[0] = v[0]; X[4] = v[1]; X[8] = v[2];
  X[5] = X[7] = v[3];
  X[2] = X[6] = v[4];
  X[1] = X[3] = v[5];
}

struct Eval {
  double tau[12], dg[12];
  double Minv[9];
  double Ce[6];   // symmetric, Voigt order
  double r[6];
  double rn;      // max |r|, +inf when rejected
};

// Evaluate the residual at S; A = FeTr^T FeTr (full 3x3, symmetric); tinv =
// 1 / tauc (divisions cost several FP64 instructions each: every kernel forms
// the twelve reciprocals once per voxel and multiplies).
__device__ void evaluate(const Consts& c, const double* S, const double* A, const double* tinv, double dt, Eval& e) {
  double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const double t = resolved(S, a);
    const double x = t * tinv[a];
    const double ax = fabs(x);
    const double xn = pow_n(c, ax);
    double g = dt * c.gdot0 * xn;
    bad |= !(g <= c.dgam_max);
    g = copysign(g, x);
    e.tau[a] = t;
    e.dg[a] = g;
  }
  if (bad) {
    e.rn = INFINITY;
    return;
  }
#pragma unroll
  for (int a = 0; a < 12; ++a) add_schmid(M, a, e.dg[a]);
  mat3_inv(M, e.Minv);
  double B[9], Ce[9];
  mat3_mul(A, e.Minv, B);
  mat3_tmul(e.Minv, B, Ce);
  e.Ce[0] = Ce[0]; e.Ce[1] = Ce[4]; e.Ce[2] = Ce[8];
  e.Ce[3] = 0.5 * (Ce[5] + Ce[7]); e.Ce[4] = 0.5 * (Ce[2] + Ce[6]); e.Ce[5] = 0.5 * (Ce[1] + Ce[3]);
  double E[6] = {0.5 * (e.Ce[0] - 1.0), 0.5 * (e.Ce[1] - 1.0), 0.5 * (e.Ce[2] - 1.0),
                 0.5 * e.Ce[3], 0.5 * e.Ce[4], 0.5 * e.Ce[5]};
  double Sn[6];
  cubic(c, E, Sn);
  double rn = 0.0;
  bool fin = true;     // fmax drops a NaN operand: test every component
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    e.r[k] = S[k] - Sn[k];
    rn = fmax(rn, fabs(e.r[k]));
    fin = fin && isfinite(e.r[k]);
  }
  e.rn = (fin && isfinite(rn)) ? rn : INFINITY;
}

// J = I - sum_a c^a (x) w^a with c^a = -dgp^a C : sym(Ce S0^a Minv) and w^a =
// d tau^a / dS.  C is linear, so the sum is accumulated before it:
// J = I - C : N, N = sum_a T^a (x) w^a, T^a = -dgp^a sym(Ce S0^a Minv), and
// the cubic stiffness is applied to the six columns of N once instead of to
// each system's T^a.
__device__ void jacobian(const Consts& c, const Eval& e, const double* tinv, double dt, double* J, double* dgp) {
  double N[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) N[i] = 0.0;
  double Cf[9];
  sym_full(e.Ce, Cf);
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const double x = fabs(e.tau[a] * tinv[a]);
    const double xn1 = pow_n1(c, x);
    const double gp = dt * c.gdot0 * c.n * xn1 * tinv[a];
    dgp[a] = gp;
    // u = Ce s', w = Minv^T m'  (times 1/sqrt6 folded in below)
    double u[3], w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      bool fu = true, fw = true;
      u[i] = w[i] = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        u[i] = cacc(u[i], fu, fcc_s(a, k), Cf[3 * i + k]);
        w[i] = cacc(w[i], fw, fcc_m(a, k), e.Minv[3 * k + i]);
      }
    }
    const double f = -gp * INV_SQRT6;
    const double T[6] = {f * u[0] * w[0], f * u[1] * w[1], f * u[2] * w[2], 0.5 * f * (u[1] * w[2] + u[2] * w[1]),
                         0.5 * f * (u[0] * w[2] + u[2] * w[0]), 0.5 * f * (u[0] * w[1] + u[1] * w[0])};
    // N += T (x) d tau^a / dS, skipping the zero coefficients
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (tau_coef(a, j) != 0) N[6 * i + j] = fma(T[i], (double)tau_coef(a, j) * INV_SQRT6, N[6 * i + j]);
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    double col[6], cc[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) col[i] = N[6 * i + j];
    cubic(c, col, cc);
#pragma unroll
    for (int i = 0; i < 6; ++i) J[6 * i + j] = (i == j) ? 1.0 - cc[i] : -cc[i];
  }
}

// LU with partial pivoting of a 6x6 matrix in place (the diagonal holds the
// reciprocal pivots); piv[k] = row swapped into k
__device__ void lu6(double* J, int* piv) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    int p = k;
    double best = fabs(J[6 * k + k]);
#pragma unroll
    for (int i = k + 1; i < 6; ++i) {
      const double v = fabs(J[6 * i + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    // the swap of rows k and p as selects over the candidate rows: every index
    // is a compile-time constant, so J stays in registers (a runtime row
    // index would place the whole matrix in local memory)
#pragma unroll
    for (int i = k + 1; i < 6; ++i) {
      const bool sw = p == i;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const double a = J[6 * k + j], b = J[6 * i + j];
        J[6 * k + j] = sw ? b : a;
        J[6 * i + j] = sw ? a : b;
      }
    }
    const double inv = 1.0 / J[6 * k + k];
    J[6 * k + k] = inv;                 // the solves multiply by the reciprocal pivot
#pragma unroll
    for (int i = k + 1; i < 6; ++i) {
      const double l = J[6 * i + k] * inv;
      J[6 * i + k] = l;
#pragma unroll
      for (int j = k + 1; j < 6; ++j) J[6 * i + j] = fma(-l, J[6 * k + j], J[6 * i + j]);
    }
  }
}

__device__ void lu6_solve(const double* LU, const int* piv, double* b) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int p = piv[k];
#pragma unroll
    for (int i = k + 1; i < 6; ++i) {      // swap b[k], b[p] by selects (registers only)
      const bool sw = p == i;
      const double x = b[k], y = b[i];
      b[k] = sw ? y : x;
      b[i] = sw ? x : y;
    }
  }
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) b[i] = fma(-LU[6 * i + j], b[j], b[i]);
#pragma unroll
  for (int i = 5; i >= 0; --i) {
#pragma unroll
    for (int j = i + 1; j < 6; ++j) b[i] = fma(-LU[6 * i + j], b[j], b[i]);
    b[i] *= LU[6 * i + i];
  }
}

__global__ void __launch_bounds__(128) k_hardening(
    size_t nvox, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
    const double* __restrict__ qhat, const double* __restrict__ Apinv, const int32_t* __restrict__ screw_of,
    const double* __restrict__ nye, const double* __restrict__ rho_ssd, const double* __restrict__ Fp,
    double* __restrict__ rho18, double* __restrict__ rho_gnd, double* __restrict__ tauc, double* __restrict__ ell,
    double* __restrict__ Fp0inv, Consts c) {
  __shared__ double sq[144], sA[162];
  __shared__ int sscrew[12];
  for (int i = threadIdx.x; i < 144; i += blockDim.x) sq[i] = qhat[i];
  for (int i = threadIdx.x; i < 162; i += blockDim.x) sA[i] = Apinv[i];
  if (threadIdx.x < 12) sscrew[threadIdx.x] = screw_of[threadIdx.x];
  __syncthreads();
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  double R[9], G[9], T[9], Gt[9];
  const int g = grain[v];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __ldg(grainR + 9 * g + k);
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = nye[k * nvox + v];
  mat3_mul(G, R, T);
  mat3_tmul(R, T, Gt);       // R^T G R
  double r18[18];
#pragma unroll
  for (int a = 0; a < 18; ++a) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) s = fma(sA[9 * a + k], Gt[k], s);
    r18[a] = s;
    rho18[a * nvox + v] = s;
  }
  double rho[12], sum = 0.0;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const double gd = c.gnd_enabled ? fabs(r18[a]) + 0.5 * fabs(r18[12 + sscrew[a]]) : 0.0;
    rho_gnd[a * nvox + v] = gd;
    rho[a] = rho_ssd[a * nvox + v] + gd;
    sum += rho[a];
  }
  const double amb = c.alpha * c.mu * c.b;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 12; ++b) s = fma(sq[12 * a + b], rho[b], s);
    tauc[a * nvox + v] = fma(amb, sqrt(s), c.tau0);
    ell[a * nvox + v] = c.K / sqrt(sum - rho[a]);
  }
  double Fpv[9], Fi[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Fpv[k] = Fp[k * nvox + v];
  mat3_inv(Fpv, Fi);
  mat3_mul(Fi, R, T);
  mat3_tmul(R, T, Gt);       // R^T Fp^-1 R
#pragma unroll
  for (int k = 0; k < 9; ++k) Fp0inv[k * nvox + v] = Gt[k];
}

// State of one voxel at the start of an evaluation: rotation, F~ = R^T F R
// (F with the line-search step applied), the crystal-frame Fp_prev^-1, the
// trial elastic right Cauchy-Green tensor A = (F~ Fp_prev^-1)^T (F~ Fp_prev^-1)
// and the frozen critical resolved shear stresses.
struct VoxelIn {
  double R[9], Ft[9], Fpi0[9], A[9], tinv[12];   // tinv = 1 / tauc
};

__device__ __forceinline__ void load_voxel(size_t nvox, size_t v, const int32_t* __restrict__ grain,
                                           const double* __restrict__ grainR, const double* __restrict__ Fin,
                                           const double* __restrict__ xdir, double lambda,
                                           const double* __restrict__ Fp0inv, const double* __restrict__ tauc_g,
                                           VoxelIn& in) {
  double Fs[9], T[9], FeTr[9];
  const int g = grain[v];
#pragma unroll
  for (int k = 0; k < 9; ++k) in.R[k] = __ldg(grainR + 9 * g + k);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double f = Fin[k * nvox + v];
    if (lambda != 0.0) f = fma(lambda, xdir[k * nvox + v], f);
    Fs[k] = f;
    in.Fpi0[k] = Fp0inv[k * nvox + v];
  }
  mat3_mul(Fs, in.R, T);
  mat3_tmul(in.R, T, in.Ft);              // F~ = R^T F R
  mat3_mul(in.Ft, in.Fpi0, FeTr);
  mat3_tmul(FeTr, FeTr, in.A);
#pragma unroll
  for (int a = 0; a < 12; ++a) in.tinv[a] = 1.0 / tauc_g[a * nvox + v];
}

// P = Fe S Fp^-T = F~ (Fp^-1 S Fp^-T) in the crystal frame, rotated to the
// sample frame, with Fp^-1 = Fp_prev^-1 M^-1 (Eq. Piola)
__device__ __forceinline__ void piola(const VoxelIn& in, const double* S, const double* Minv, double* P) {
  double Fpinv[9], Sf[9], W[9], Q[9], Pt[9], U[9];
  mat3_mul(in.Fpi0, Minv, Fpinv);
  sym_full(S, Sf);
  mat3_mult(Sf, Fpinv, W);
  mat3_mul(Fpinv, W, Q);
  mat3_mul(in.Ft, Q, Pt);
  mat3_mult(Pt, in.R, U);
  mat3_mul(in.R, U, P);
}

// Local Newton on S at one voxel (data-dependent iteration counts): writes S,
// dgam and P; returns the Newton iterations, residual evaluations and whether
// it failed.
__device__ __forceinline__ void local_voxel(size_t nvox, size_t v, const int32_t* __restrict__ grain,
                                            const double* __restrict__ grainR, const double* __restrict__ Fin,
                                            const double* __restrict__ xdir, double lambda,
                                            const double* __restrict__ Fp0inv, const double* __restrict__ tauc_g,
                                            const double* __restrict__ Swarm, double* __restrict__ Sout,
                                            double* __restrict__ dgout, double* __restrict__ Pout, double dt,
                                            const Consts& c, int& iters, int& evals, int& failed) {
  VoxelIn in;
  load_voxel(nvox, v, grain, grainR, Fin, xdir, lambda, Fp0inv, tauc_g, in);
  const double* A = in.A;
  const double* tinv = in.tinv;      // 1 / tauc
  double S[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) S[k] = Swarm[k * nvox + v];

  Eval e;
  evaluate(c, S, A, tinv, dt, e);
  ++evals;
  if (!(e.rn < INFINITY)) {             // warm start rejected: restart from the elastic-free state
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k] = 0.0;
    evaluate(c, S, A, tinv, dt, e);
    ++evals;
  }
  double J[36], dgp[12];
  int piv[6];
  bool conv = e.rn <= c.local_tol_abs;
  while (!conv && iters < c.max_local) {
    jacobian(c, e, tinv, dt, J, dgp);
    lu6(J, piv);
    double d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = -e.r[k];
    lu6_solve(J, piv, d);
    double lam = 1.0;
    bool acc = false;
    for (int hv = 0; hv <= c.max_halvings; ++hv) {
      double St[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) St[k] = fma(lam, d[k], S[k]);
      Eval et;
      evaluate(c, St, A, tinv, dt, et);
      ++evals;
      if (et.rn < e.rn) {
#pragma unroll
        for (int k = 0; k < 6; ++k) S[k] = St[k];
        e = et;
        acc = true;
        break;
      }
      lam *= 0.5;
    }
    ++iters;
    if (!acc) {                          // no decrease: round-off floor or failure
      conv = e.rn <= c.floor_abs;
      break;
    }
    conv = e.rn <= c.local_tol_abs;
  }
  failed = conv ? 0 : 1;
#pragma unroll
  for (int k = 0; k < 6; ++k) Sout[k * nvox + v] = S[k];
#pragma unroll
  for (int a = 0; a < 12; ++a) dgout[a * nvox + v] = e.dg[a];
  double P[9];
  piola(in, S, e.Minv, P);
#pragma unroll
  for (int k = 0; k < 9; ++k) Pout[k * nvox + v] = P[k];
}

// Local update over all voxels.  The number of local Newton iterations
// differs from voxel to voxel (grains near their yield point need several),
// so the kernel is persistent and balanced dynamically: each warp takes the
// next chunk of 32 voxels from a device counter (counters[6], zeroed before
// the launch) until none is left, and an SM whose voxels converge quickly
// takes more chunks.  Each voxel's arithmetic is the same as with a fixed
// assignment.
__global__ void __launch_bounds__(128) k_local(
    size_t nvox, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
    const double* __restrict__ Fin, const double* __restrict__ xdir, double lambda,
    const double* __restrict__ Fp0inv, const double* __restrict__ tauc_g, const double* __restrict__ Swarm,
    double* __restrict__ Sout, double* __restrict__ dgout, double* __restrict__ Pout,
    int32_t* __restrict__ counters, double dt, Consts c) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long nchunks = (long)((nvox + 31) / 32);
  int mx = 0, nf = 0;
  unsigned si = 0, se = 0;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(&counters[6], 1);
    chunk = __shfl_sync(full, chunk, 0);
    if (chunk >= nchunks) break;
    const size_t v = (size_t)chunk * 32 + lane;
    int iters = 0, failed = 0, evals = 0;
    if (v < nvox)
      local_voxel(nvox, v, grain, grainR, Fin, xdir, lambda, Fp0inv, tauc_g, Swarm, Sout, dgout, Pout, dt, c,
                  iters, evals, failed);
    mx = max(mx, iters);
    nf += failed;
    si += (unsigned)iters;
    se += (unsigned)evals;
  }
  // counters: warp-aggregated
  mx = __reduce_max_sync(full, mx);
  nf = __reduce_add_sync(full, nf);
  si = __reduce_add_sync(full, si);
  se = __reduce_add_sync(full, se);
  if (lane == 0) {
    if (mx) atomicMax(&counters[0], mx);
    if (nf) atomicAdd(&counters[1], nf);
    // 64-bit totals of local Newton iterations and residual evaluations (work accounting)
    unsigned long long* tot = reinterpret_cast<unsigned long long*>(counters + 8);
    atomicAdd(&tot[0], (unsigned long long)si);
    atomicAdd(&tot[1], (unsigned long long)se);
  }
}

// The consistent tangent at the converged S: the same work for every voxel
// (no data-dependent iterations), so whole warps stay converged.
//
// For a direction dF~ = a b^T of the crystal-frame deformation gradient,
// dE = sym(u w^T) with u = Fe^T a, w = Fp^-T b, and
//   dP~ = F~ dQ + a (Q b)^T,  dQ = Fp^-1 dS Fp^-T - (dFpi W + (dFpi W)^T),
// where dS = J^-1 C : dE, dM = sum_a dgp^a tau^a(dS) s^a (x) m^a,
// dFpi = Fp^-1 dM M^-1, W = S Fp^-T and Q = Fp^-1 S Fp^-T.  Everything but
// a (Q b)^T is linear in the six components of dE, so F~ dQ is formed once
// for each unit dE (the columns of H, 9 x 6, in shared memory) and each of
// the nine directions costs H dE plus the rank-one term and the rotation:
// six solves through the chain instead of nine.
constexpr int TAN_THREADS = 64;

__global__ void __launch_bounds__(TAN_THREADS) k_tangent(
    size_t nvox, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
    const double* __restrict__ Fin, const double* __restrict__ xdir, double lambda,
    const double* __restrict__ Fp0inv, const double* __restrict__ tauc_g, const double* __restrict__ Sin,
    double* __restrict__ Kout, double dt, Consts c, int k32) {
  __shared__ double Hs[54 * TAN_THREADS];     // H[9 m + ij] of this thread at Hs[(9 m + ij) T + tid]
  double* H = Hs + threadIdx.x;
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nvox) {
    VoxelIn in;
    load_voxel(nvox, v, grain, grainR, Fin, xdir, lambda, Fp0inv, tauc_g, in);
    const double* R = in.R;
    const double* Ft = in.Ft;
    const double* Fpi0 = in.Fpi0;
    const double* tinv = in.tinv;      // 1 / tauc
    double S[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k] = Sin[k * nvox + v];
    Eval e;
    evaluate(c, S, in.A, tinv, dt, e);
    double J[36], dgp[12];
    int piv[6];
    jacobian(c, e, tinv, dt, J, dgp);
    lu6(J, piv);
    double Fpinv[9], Fe[9], Sf[9], W[9], Q[9];
    mat3_mul(Fpi0, e.Minv, Fpinv);
    mat3_mul(Ft, Fpinv, Fe);
    sym_full(S, Sf);
    mat3_mult(Sf, Fpinv, W);             // W = S Fpinv^T
    mat3_mul(Fpinv, W, Q);               // Q = Fpinv S Fpinv^T
    // H: F~ dQ for the six unit strain increments (tensor components
    // E11, E22, E33, E23, E13, E12, as `cubic` takes them)
#pragma unroll 1
    for (int m = 0; m < 6; ++m) {
      double dE[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) dE[k] = k == m ? 1.0 : 0.0;
      double dS[6];
      cubic(c, dE, dS);
      lu6_solve(J, piv, dS);
      double dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int a = 0; a < 12; ++a) add_schmid(dM, a, dgp[a] * resolved(dS, a));
      double t1[9], dFpi[9], dQ[9], dSf[9], t2[9], dPt[9];
      mat3_mul(dM, e.Minv, t1);
      mat3_mul(Fpinv, t1, dFpi);        // (negated below)
      mat3_mul(dFpi, W, t1);            // dFpinv W with dFpinv = -dFpi
      sym_full(dS, dSf);
      mat3_mult(dSf, Fpinv, t2);
      mat3_mul(Fpinv, t2, dQ);          // Fpinv dS Fpinv^T
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dQ[3 * i + j] -= t1[3 * i + j] + t1[3 * j + i];
      mat3_mul(Ft, dQ, dPt);
#pragma unroll
      for (int ij = 0; ij < 9; ++ij) H[(9 * m + ij) * TAN_THREADS] = dPt[ij];
    }
#pragma unroll 1
    for (int kl = 0; kl < 9; ++kl) {
      const int kk = kl / 3, ll = kl % 3;
      double a3[3], b3[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) { a3[p] = R[3 * kk + p]; b3[p] = R[3 * ll + p]; }
      // dF~ = a b^T; dE = sym(Fe^T a (Fpinv^T b)^T)
      double u[3], w[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        u[i] = Fe[i] * a3[0] + Fe[3 + i] * a3[1] + Fe[6 + i] * a3[2];
        w[i] = Fpinv[i] * b3[0] + Fpinv[3 + i] * b3[1] + Fpinv[6 + i] * b3[2];
      }
      const double dE[6] = {u[0] * w[0], u[1] * w[1], u[2] * w[2], 0.5 * (u[1] * w[2] + u[2] * w[1]),
                            0.5 * (u[0] * w[2] + u[2] * w[0]), 0.5 * (u[0] * w[1] + u[1] * w[0])};
      double qb[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) qb[j] = Q[3 * j] * b3[0] + Q[3 * j + 1] * b3[1] + Q[3 * j + 2] * b3[2];
      double dPt[9];
#pragma unroll
      for (int ij = 0; ij < 9; ++ij) {
        double t = a3[ij / 3] * qb[ij % 3];
#pragma unroll
        for (int m = 0; m < 6; ++m) t = fma(H[(9 * m + ij) * TAN_THREADS], dE[m], t);
        dPt[ij] = t;
      }
      double U[9], dP[9];
      mat3_mult(dPt, R, U);
      mat3_mul(R, U, dP);
#pragma unroll
      for (int ij = 0; ij < 9; ++ij) {
        if (k32)   // mixed precision: the tangent only drives the FP32 conjugate gradients
          reinterpret_cast<float*>(Kout)[(size_t)(9 * ij + kl) * nvox + v] = (float)dP[ij];
        else
          Kout[(size_t)(9 * ij + kl) * nvox + v] = dP[ij];
      }
    }
  }
}


// ---- forward-mode sensitivities with respect to theta = (tau0, K, alpha, b) ----
// One parameter per launch: dth = the unit direction of that parameter.

__device__ __forceinline__ double sgn(double x) { return (double)((x > 0.0) - (x < 0.0)); }

// X~ = R^T X R
__device__ __forceinline__ void to_crystal(const double* R, const double* X, double* Xt) {
  double T[9];
  mat3_mul(X, R, T);
  mat3_tmul(R, T, Xt);
}
// X = R X~ R^T
__device__ __forceinline__ void to_sample(const double* R, const double* Xt, double* X) {
  double T[9];
  mat3_mult(Xt, R, T);
  mat3_mul(R, T, X);
}

// d tauc and d l from the Nye tensor of dFp_{k-1} (sample frame), d rho_SSD,k-1
// and dth, at the start-of-increment state (rho18 of the increment, rho_SSD,k-1):
//   d rho18 = A^+ dG~ - rho18 db / b  (A is proportional to b),
//   d rho_GND^a = sgn(rho18_e^a) d rho18_e^a + 1/2 sgn(rho18_s) d rho18_s,
//   d tauc^a = dtau0 + mu (dalpha b X^a + alpha db X^a + alpha b dX^a),
//   X^a = sqrt(sum_b q^ab rho^b),  d l^a = dK / Y^a - K dY^a / Y^a^2,
//   Y^a = sqrt(sum_{b != a} rho^b).
__global__ void __launch_bounds__(128) k_hard_jvp(
    size_t nvox, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
    const double* __restrict__ qhat, const double* __restrict__ Apinv, const int32_t* __restrict__ screw_of,
    const double* __restrict__ dnye, const double* __restrict__ rho18, const double* __restrict__ rho_ssd,
    const double* __restrict__ drho, double* __restrict__ dtauc, double* __restrict__ dell, Consts c, Theta dth) {
  __shared__ double sq[144], sA[162];
  __shared__ int sscrew[12];
  for (int i = threadIdx.x; i < 144; i += blockDim.x) sq[i] = qhat[i];
  for (int i = threadIdx.x; i < 162; i += blockDim.x) sA[i] = Apinv[i];
  if (threadIdx.x < 12) sscrew[threadIdx.x] = screw_of[threadIdx.x];
  __syncthreads();
  const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvox) return;
  double R[9], G[9], Gt[9];
  const int g = grain[v];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = __ldg(grainR + 9 * g + k);
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = dnye[k * nvox + v];
  to_crystal(R, G, Gt);
  double r18[18], d18[18];
#pragma unroll
  for (int a = 0; a < 18; ++a) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) s = fma(sA[9 * a + k], Gt[k], s);
    r18[a] = rho18[a * nvox + v];
    d18[a] = s - r18[a] * (dth.db / c.b);
  }
  double rho[12], dr[12], sum = 0.0, dsum = 0.0;
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    const int sa = 12 + sscrew[a];
    double gd = 0.0, dgd = 0.0;
    if (c.gnd_enabled) {
      gd = fabs(r18[a]) + 0.5 * fabs(r18[sa]);
      dgd = sgn(r18[a]) * d18[a] + 0.5 * sgn(r18[sa]) * d18[sa];
    }
    rho[a] = rho_ssd[a * nvox + v] + gd;
    dr[a] = drho[a * nvox + v] + dgd;
    sum += rho[a];
    dsum += dr[a];
  }
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    double s = 0.0, ds = 0.0;
#pragma unroll
    for (int b = 0; b < 12; ++b) {
      s = fma(sq[12 * a + b], rho[b], s);
      ds = fma(sq[12 * a + b], dr[b], ds);
    }
    const double X = sqrt(s), dX = ds / (2.0 * X);
    dtauc[a * nvox + v] = dth.dtau0 + c.mu * (dth.dalpha * c.b * X + c.alpha * dth.db * X + c.alpha * c.b * dX);
    const double Y = sqrt(sum - rho[a]), dY = (dsum - dr[a]) / (2.0 * Y);
    dell[a * nvox + v] = dth.dK / Y - c.K * dY / (Y * Y);
  }
}

// Directional derivative of the converged local update along (dF, dFp_{k-1},
// dtauc), in the crystal frame (see the tangent kernel for the notation):
//   J dS = C : sym(Fe^T dFe) with dFe = dF~ Fp^-1 + F~ dFp0inv M^-1
//          + F~ Fp0^-1 dMinv|_tauc (the change of Fe at fixed S),
//   d dgam^a = dgam'(tau^a) (S0^a : dS) - n dgam^a dtauc^a / tauc^a,
//   dFp^-1 = dFp0inv M^-1 - Fp^-1 dM M^-1,
//   dP = dF Q + F dQ, Q = Fp^-1 S Fp^-T,  dFp = dM Fp0 + M dFp0.
// mode 0 (dF = 0): writes dP.  mode 1: writes dFp_k and d rho_SSD,k (the
// implicit Kocks-Mecking commit differentiated) and reduces the mean of dP
// into mean_out[9].
__global__ void __launch_bounds__(128) k_local_jvp(
    size_t nvox, const int32_t* __restrict__ grain, const double* __restrict__ grainR,
    const double* __restrict__ Fin, const double* __restrict__ Fp0inv, const double* __restrict__ tauc_g,
    const double* __restrict__ Sin, const double* __restrict__ dFin, const double* __restrict__ dFp0_g,
    const double* __restrict__ dtauc_g, const double* __restrict__ ell_g, const double* __restrict__ dell_g,
    const double* __restrict__ rho_g, const double* __restrict__ drho_g, double* __restrict__ dP_out,
    double* __restrict__ dFp_out, double* __restrict__ drho_out, double* __restrict__ partial,
    unsigned int* __restrict__ ticket, double* __restrict__ mean_out, double dt, Consts c, Theta dth, int mode) {
  __shared__ double sh[320];
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (size_t)gridDim.x * blockDim.x) {
    VoxelIn in;
    load_voxel(nvox, v, grain, grainR, Fin, nullptr, 0.0, Fp0inv, tauc_g, in);
    const double* R = in.R;
    double S[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) S[k] = Sin[k * nvox + v];
    Eval e;
    evaluate(c, S, in.A, in.tinv, dt, e);
    double J[36], dgp[12];
    int piv[6];
    jacobian(c, e, in.tinv, dt, J, dgp);
    lu6(J, piv);
    double X[9], dFt[9], dFp0t[9], dtc[12];
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = mode ? dFin[k * nvox + v] : 0.0;
    to_crystal(R, X, dFt);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = dFp0_g[k * nvox + v];
    to_crystal(R, X, dFp0t);
#pragma unroll
    for (int a = 0; a < 12; ++a) dtc[a] = dtauc_g[a * nvox + v];
    double Fpinv[9], Fe[9], FeTr[9], T1[9], T2[9], dFpi0[9], dFe[9];
    mat3_mul(in.Fpi0, e.Minv, Fpinv);
    mat3_mul(in.Ft, Fpinv, Fe);
    mat3_mul(in.Ft, in.Fpi0, FeTr);
    mat3_mul(in.Fpi0, dFp0t, T1);
    mat3_mul(T1, in.Fpi0, dFpi0);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFpi0[k] = -dFpi0[k];
    // the change of M^-1 through tauc at fixed S
    double ddg[12], dM[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      ddg[a] = -c.n * e.dg[a] * in.tinv[a] * dtc[a];
      add_schmid(dM, a, ddg[a]);
    }
    double dMinv[9];
    mat3_mul(e.Minv, dM, T1);
    mat3_mul(T1, e.Minv, dMinv);                 // negated below
    mat3_mul(dFt, Fpinv, dFe);
    mat3_mul(in.Ft, dFpi0, T1);
    mat3_mul(T1, e.Minv, T2);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFe[k] += T2[k];
    mat3_mul(FeTr, dMinv, T2);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFe[k] -= T2[k];
    mat3_tmul(Fe, dFe, T1);                      // Fe^T dFe
    double dE[6] = {T1[0], T1[4], T1[8], 0.5 * (T1[5] + T1[7]), 0.5 * (T1[2] + T1[6]), 0.5 * (T1[1] + T1[3])};
    double dS[6];
    cubic(c, dE, dS);
    lu6_solve(J, piv, dS);
#pragma unroll
    for (int a = 0; a < 9; ++a) dM[a] = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      ddg[a] = fma(dgp[a], resolved(dS, a), ddg[a]);
      add_schmid(dM, a, ddg[a]);
    }
    // dFp^-1 = dFp0inv M^-1 - Fp^-1 dM M^-1
    double dFpinv[9];
    mat3_mul(dFpi0, e.Minv, dFpinv);
    mat3_mul(Fpinv, dM, T1);
    mat3_mul(T1, e.Minv, T2);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFpinv[k] -= T2[k];
    double Sf[9], dSf[9], W[9], Q[9], dQ[9];
    sym_full(S, Sf);
    sym_full(dS, dSf);
    mat3_mult(Sf, Fpinv, W);                     // S Fp^-T
    mat3_mul(Fpinv, W, Q);
    // dQ = dFpinv S Fp^-T + Fp^-1 dS Fp^-T + (dFpinv S Fp^-T)^T
    double A3[9];
    mat3_mul(dFpinv, W, A3);
    mat3_mult(dSf, Fpinv, T1);
    mat3_mul(Fpinv, T1, T2);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dQ[3 * i + j] = A3[3 * i + j] + A3[3 * j + i] + T2[3 * i + j];
    double dPt[9];
    mat3_mul(dFt, Q, dPt);
    mat3_mul(in.Ft, dQ, T1);
#pragma unroll
    for (int k = 0; k < 9; ++k) dPt[k] += T1[k];
    double dP[9];
    to_sample(R, dPt, dP);
    if (mode == 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) dP_out[k * nvox + v] = dP[k];
      continue;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] += dP[k];
    // dFp = dM Fp0 + M dFp0 (crystal frame), M = I + sum dgam S0
    double Fp0[9], Mm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, dFpt[9];
    mat3_inv(in.Fpi0, Fp0);
#pragma unroll
    for (int a = 0; a < 12; ++a) add_schmid(Mm, a, e.dg[a]);
    mat3_mul(dM, Fp0, dFpt);
    mat3_mul(Mm, dFp0t, T1);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFpt[k] += T1[k];
    to_sample(R, dFpt, X);
#pragma unroll
    for (int k = 0; k < 9; ++k) dFp_out[k * nvox + v] = X[k];
    // rho_k = (rho + a / (b l)) / D, D = 1 + 2 yc a / b, a = |dgam|
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const double ag = fabs(e.dg[a]), da = sgn(e.dg[a]) * ddg[a];
      const double l = ell_g[a * nvox + v], dl = dell_g[a * nvox + v];
      const double bl = c.b * l;
      const double D = 1.0 + 2.0 * c.yc * ag / c.b;
      const double dD = 2.0 * c.yc * (da / c.b - ag * dth.db / (c.b * c.b));
      const double rk = (rho_g[a * nvox + v] + ag / bl) / D;
      const double dnum = drho_g[a * nvox + v] + da / bl - ag * (dth.db * l + c.b * dl) / (bl * bl);
      drho_out[a * nvox + v] = (dnum - rk * dD) / D;
    }
  }
  if (mode == 0) return;
  double bs[9];
  blk_sums9<double>(acc, 0x1FFu, sh, bs);
  if (threadIdx.x == 0)
    for (int k = 0; k < 9; ++k) partial[(size_t)k * gridDim.x + blockIdx.x] = bs[k];
  double tot[9];
  if (last_block_sums(partial, 9, ticket, sh, tot) && threadIdx.x == 0)
    for (int k = 0; k < 9; ++k) mean_out[k] = tot[k] / (double)nvox;
}

}  // namespace

cudaError_t launch_hardening(const rve_s* h, cudaStream_t s) {
  const unsigned blocks = (unsigned)((h->nvox + 127) / 128);
  {
    ProfScope ps_(h, RVE_K_HARDENING, s);
    k_hardening<<<blocks, 128, 0, s>>>(h->nvox, h->grain, h->grainR, h->qhat, h->Apinv, h->screw_of, h->nye,
                                     h->rho_ssd, h->Fp, h->rho18, h->rho_gnd, h->tauc, h->ell, h->Fp0inv, h->cst);
  }
  return cudaGetLastError();
}

cudaError_t launch_local(const rve_s* h, double dt, double lambda, int out_buf, int warm_buf, cudaStream_t s) {
  // persistent: as many blocks as are resident at once (no more than the chunks need)
  static const int per_sm = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_local, 128, 0) != cudaSuccess || n < 1) n = 1;
    return n;
  }();
  const long need = (long)((h->nvox + 127) / 128);
  const unsigned blocks = (unsigned)std::min<long>(need, (long)per_sm * h->num_sms);
  const double* warm = warm_buf < 0 ? h->S_c : h->S[warm_buf];
  if (cudaError_t e = cudaMemsetAsync(h->dcount + 6, 0, sizeof(int32_t), s)) return e;
  {
    ProfScope ps_(h, RVE_K_CONSTITUTIVE, s);
    k_local<<<blocks, 128, 0, s>>>(h->nvox, h->grain, h->grainR, h->F, h->x, lambda, h->Fp0inv, h->tauc, warm,
                                   h->S[out_buf], h->dgam[out_buf], h->P[out_buf], h->dcount, dt, h->cst);
  }
  return cudaGetLastError();
}

cudaError_t launch_tangent(const rve_s* h, double dt, double lambda, int buf, cudaStream_t s) {
  const unsigned blocks = (unsigned)((h->nvox + TAN_THREADS - 1) / TAN_THREADS);
  {
    ProfScope ps_(h, RVE_K_TANGENT_BUILD, s);
    k_tangent<<<blocks, TAN_THREADS, 0, s>>>(h->nvox, h->grain, h->grainR, h->F, h->x, lambda, h->Fp0inv,
                                             h->tauc, h->S[buf], h->K[buf], dt, h->cst, h->opt.precision == 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_constitutive(const rve_s* h, double dt, double lambda, int out_buf, int warm_buf,
                                cudaStream_t s) {
  if (cudaError_t e = launch_local(h, dt, lambda, out_buf, warm_buf, s)) return e;
  return launch_tangent(h, dt, lambda, out_buf, s);
}

constexpr int JVP_BLOCKS = 4 * 152;

cudaError_t launch_hard_jvp(const rve_s* h, const double* dnye, const double* drho, double* dtauc, double* dell,
                            Theta dth, cudaStream_t s) {
  const unsigned blocks = (unsigned)((h->nvox + 127) / 128);
  {
    ProfScope ps_(h, RVE_K_HARDENING, s);
    k_hard_jvp<<<blocks, 128, 0, s>>>(h->nvox, h->grain, h->grainR, h->qhat, h->Apinv, h->screw_of, dnye, h->rho18,
                                      h->rho_ssd, drho, dtauc, dell, h->cst, dth);
  }
  return cudaGetLastError();
}

cudaError_t launch_local_jvp(const rve_s* h, double dt, int mode, const double* dF, const double* dFp0,
                             const double* dtauc, const double* dell, const double* drho, double* dP,
                             double* dFp_out, double* drho_out, double* mean_out, Theta dth, cudaStream_t s) {
  {
    ProfScope ps_(h, RVE_K_CONSTITUTIVE, s);
    k_local_jvp<<<JVP_BLOCKS, 128, 0, s>>>(h->nvox, h->grain, h->grainR, h->F, h->Fp0inv, h->tauc, h->S[h->cur], dF,
                                           dFp0, dtauc, h->ell, dell, h->rho_ssd, drho, dP, dFp_out, drho_out,
                                           h->partial, (unsigned int*)(h->dcount + 4), mean_out, dt, h->cst, dth,
                                           mode);
  }
  return cudaGetLastError();
}
