// Internal declarations of the GB300 path: the handle, the per-handle device
// tables and the launch wrappers of every kernel (defined in fft.cu,
// constitutive.cu and vec.cu; orchestrated by rve_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/rve.h"

#define RVE_MAX_RADIX_PASSES 12
#define RVE_RED_BLOCKS 1216      // 152 SMs x 8: grid of the reducing kernels
#define RVE_RED_THREADS 256
#define RVE_WAIT_POLLS_DEFAULT (1u << 22)   // bounded mbarrier polls of the staged FP32 tangent apply

struct FFTPlan {
  int n;                                  // transform length
  int npass;                              // number of radix passes
  int radix[RVE_MAX_RADIX_PASSES];
};

// Operator applied in frequency space between the forward and inverse z passes.
//   OP_PROJECT: 9 fields, (G X)_ij = n_j sum_l X_il n_l with the zero-mode mixed control
//   OP_CURL:    9 fields, G_ij = -eps_jkl D_k X_il
//   OP_LAPINV:  3 fields, each multiplied by 1 / (64 nvox sum_m s2_m prod_{j!=m} c2_j),
//               the inverse of D^H D for the unscaled rotated-scheme stencils (0 where it vanishes)
//   OP_CURL_STD: 9 fields, G_ij = -eps_jkl D_k X_il with the standard (continuous)
//               spectral derivative D_k = i xi_k / h (Nyquist: 0), for comparison
enum SpecOp { OP_PROJECT = 0, OP_CURL = 1, OP_LAPINV = 2, OP_CURL_STD = 3 };

struct SpecParams {
  int op;
  int keep[9];          // zero mode: 1 = keep (stress-controlled) component
  double shift[9];      // zero mode: subtract nvox * shift[c] (the prescribed Pbar)
  double inv_nvox;
  double inv4h;         // 1 / (4 h) for the curl
  double* mean_out;     // nullable: receives X^(0) / nvox (9 doubles) before the shift
};

// Device tables per axis (in the workspace).
struct AxisTables {
  const double2* tw;    // e^{-2 pi i t / n}, t = 0..n-1
  const double* tanh_;  // tan(pi k' / n) for the frequency index k (signed k'), Nyquist: 0
  const int8_t* nyq;    // 1 at the Nyquist index of an even n
  const double2* ph;    // e^{i xi_k}, exactly -1 at Nyquist
  const double* s2;     // sin^2(xi_k / 2)
  const double* c2;     // cos^2(xi_k / 2)
  const float2* tw32;   // the twiddles rounded to float (mixed precision)
  const double* xi;     // xi_k = 2 pi k' / n (signed k'), 0 at Nyquist: the standard frequency
};

// Unit direction in the material parameters (tau0, K, alpha, b) of one
// sensitivity
struct Theta {
  double dtau0, dK, dalpha, db;
};

struct Consts {        // material constants read by the hardening and constitutive kernels
  double C11, C12, C44, mu, b, tau0, alpha, gdot0, n, K, yc;
  int n_int;            // n if it is a positive integer <= 64, else 0 (use pow)
  int gnd_enabled;
  double local_tol_abs, floor_abs, dgam_max;
  int max_local, max_halvings;
};

// Launch accounting: every kernel launch goes through prof_begin/prof_end.
struct Prof {
  bool on = false;
  int64_t launches[RVE_K_COUNT] = {0};
  double ms[RVE_K_COUNT] = {0};
  struct Pending { int cat; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  // A stream capture in progress records into `cap`: launch counts per
  // category, and (when timing) event pairs taken from its spare events and
  // recorded as external event nodes of the graph.  The graph owns them.
  struct Capture {
    int64_t launches[RVE_K_COUNT] = {0};
    std::vector<Pending> events;
    std::vector<cudaEvent_t> spare;
  };
  Capture* cap = nullptr;
  std::vector<Pending> borrowed;   // graph-owned pairs replayed since the last resolve
  cudaEvent_t take();
  void begin(int cat, cudaStream_t s, cudaEvent_t* a);
  void end(int cat, cudaStream_t s, cudaEvent_t a);
  void resolve();      // after a host synchronisation
  void reset();
  void destroy();
};

// One captured chunk of CG iterations (see cg_chunk in rve_api.cu).
struct CgGraph {
  cudaGraphExec_t exec = nullptr;
  int cur = -1;            // tangent buffer the chunk reads
  unsigned key = 0;        // strain mask bits
  bool timed = false;      // captured with profiling events
  Prof::Capture rec;
};
constexpr int RVE_CG_GRAPHS = 4;

struct rve_s {
  int n0, n1, n2, nkx;
  size_t nvox, nspec;   // nspec = nkx * n1 * n2
  int ngrains;
  rve_material mat;
  rve_options opt;
  double mu, h;
  Consts cst;
  cudaStream_t stream;
  int device;           // CUDA device current at rve_create
  FFTPlan plan[3];
  AxisTables ax[3];

  // device state (all carved from the caller's workspace)
  int32_t* grain;       // nvox
  double* grainR;       // 9 * ngrains (crystal -> sample)
  double* qhat;         // 144 interaction matrix (row-major alpha, beta)
  double* Apinv;        // 162: A^+ (18 x 9, crystal frame, divided by b)
  int32_t* screw_of;    // 12
  double *F_c, *Fp, *S_c, *rho_ssd, *dF_last, *P_c;  // committed
  double *nye, *rho18, *rho_gnd, *tauc, *ell, *Fp0inv;  // per increment
  double* F;            // Newton iterate
  double *P[2], *K[2], *S[2], *dgam[2];             // evaluation double buffer
  int cur;
  bool K_stale = false;   // the converged evaluation's tangent is not built yet (built on request)
  CgGraph graphs[RVE_CG_GRAPHS];
  int graph_next = 0;
  int num_sms = 152;        // of the handle's device
  // launch shapes (rve_options.autotune times candidates at create):
  int div_blocks = 4 * 152; // grid cap of the divergence stencil
  int fft_fill = 4 * 152;   // block count the FFT tile rules aim for: x passes
  int fft_fill_y = 8 * 152; // y passes
  int fft_fill_z = 4 * 152; // z pass
  bool autotuned = false;
  bool tma_apply = false;   // FP32 tangent apply staged by bulk copies (rve_options.tma)
  int fft_cat = -1;         // >= 0: the FFT passes are counted in this category (the Nye curl)
  bool row_stencils = true; // row-strip stencils where the grid suits them (n0 = 32, 64, 96, 128)
  unsigned wait_polls = RVE_WAIT_POLLS_DEFAULT;   // its per-tile wait limit (rve_set_wait_limit)
  // forward-mode sensitivities (rve_sensitivity_enable): state tangents
  // dFp (9) and d rho_SSD (12) per parameter, double-buffered so that a
  // failed increment leaves them untouched; scratch fields; d<P>/d theta of
  // the last increment
  bool sens_on = false;
  int sens_cur = 0;
  double sens_tol = 0.0;
  double *sd_Fp[2][RVE_NTHETA], *sd_rho[2][RVE_NTHETA];
  double *s_dnye, *s_dtauc, *s_dell, *s_dP, *s_mean;
  double sens_dP[RVE_NTHETA * 9];
  int sens_valid = 0;
  double *R, *x, *r, *p, *t, *q;
  double *bv, *bs;      // BiCGStab vectors v and s
  double2* spec;        // 9 * nspec
  double* lapw;         // nspec: inverse-Laplacian weight of the projection's Laplace solve
  // mixed precision (precision == 1): FP32 conjugate-gradient state
  float2* spec32;       // 3 * nspec
  float *x32, *r32, *p32, *t32, *du32;   // 9, 9, 9, 9, 6 components
  double* partial;      // 4 * RVE_RED_BLOCKS
  double* dscal;        // device scalars (see DS_*)
  int32_t* dcount;      // device counters: [0] local max iters, [1] local failures, [4] last-block ticket,
                        // [6] next voxel chunk of the local update, [8..11] 64-bit work totals
  double* hscal;        // pinned host mirror of dscal
  int32_t* hcount;      // pinned host mirror of dcount

  // host-side history
  double Pmacro[9], Smacro[9];
  double dFbar_prev[9];
  double dt_prev;
  int increment;
  std::string err;
  mutable Prof prof;
};

// bracket one kernel launch of category `cat` on stream `s`
struct ProfScope {
  Prof& p; int cat; cudaStream_t s; cudaEvent_t a = nullptr;
  ProfScope(const rve_s* h, int c, cudaStream_t st) : p(h->prof), cat(c), s(st) { p.begin(cat, s, &a); }
  ~ProfScope() { p.end(cat, s, a); }
};

// device scalar slots
enum { DS_RR = 0, DS_PKP = 1, DS_ALPHA = 2, DS_BETA = 3, DS_NORM = 4, DS_STOP = 5, DS_DONE = 6, DS_ITERS = 7,
       DS_MEANP = 8,
       DS_MEANSIG = 17, DS_MEANF = 26, DS_DOT = 35,
       DS_ERR = 40,      // nonzero: a kernel gave up a bounded wait (sticky)
       DS_XMEAN = 48 };

// ---- fft.cu ----
// `done` (nullable, device): when *done != 0 every block returns at once (the
// conjugate-gradient loop has converged on the device)
// nf: number of fields transformed (9, or 3 for OP_LAPINV)
cudaError_t launch_fft_forward(const rve_s* h, const double* in, cudaStream_t s, const double* done = nullptr,
                               int nf = 9);
cudaError_t launch_fft_op(const rve_s* h, const SpecParams& sp, cudaStream_t s, const double* done = nullptr,
                          int nf = 9);
cudaError_t launch_fft_inverse(const rve_s* h, double* out, cudaStream_t s, const double* done = nullptr,
                               int nf = 9);
// radix passes 8 (up to max_radix), 4, 2, 3.  The x and y passes take radix 8
// (two shared-memory round trips for 64 points instead of three); the z pass,
// whose narrow tiles leave few threads per block, is faster with radix 4
void make_plan(int n, FFTPlan* p, int max_radix = 8);
// fills h->lapw (once, at create)
cudaError_t launch_lapinv_table(const rve_s* h, cudaStream_t s);
cudaError_t launch_fft_forward32(const rve_s* h, const float* in, cudaStream_t s, const double* done);
cudaError_t launch_fft_lapinv32(const rve_s* h, const SpecParams& sp, cudaStream_t s, const double* done);
cudaError_t launch_fft_inverse32(const rve_s* h, float* out, cudaStream_t s, const double* done);

// ---- stencil.cu: G* = D (D^H D)^-1 D^H with real-space rotated-scheme stencils ----
// number of tiles the stencils cover (their grids loop over them)
int stencil_tiles(const rve_s* h);
// mean_mask: bit c set = the mean of field c is reduced into ds[DS_XMEAN + c]
// (others read 0)
cudaError_t launch_div(const rve_s* h, const double* X, double* d, int check_done, unsigned mean_mask,
                       cudaStream_t s);
cudaError_t launch_grad(const rve_s* h, const double* u, double* Y, const uint8_t* mask, const double* shift,
                        cudaStream_t s);
cudaError_t launch_grad_cg(const rve_s* h, const double* u, const uint8_t* mask, cudaStream_t s);
cudaError_t launch_div32(const rve_s* h, const float* X, float* d, unsigned mean_mask, cudaStream_t s);
cudaError_t launch_grad_cg32(const rve_s* h, const float* u, const uint8_t* mask, cudaStream_t s);

// ---- constitutive.cu ----
cudaError_t launch_hardening(const rve_s* h, cudaStream_t s);
// local update (S, dgam, P) at F + lambda x into buffer out_buf, warm-started
// from S[warm_buf] (or the committed S when warm_buf < 0)
cudaError_t launch_local(const rve_s* h, double dt, double lambda, int out_buf, int warm_buf, cudaStream_t s);
// consistent tangent K[buf] at F + lambda x and the converged S[buf]
cudaError_t launch_tangent(const rve_s* h, double dt, double lambda, int buf, cudaStream_t s);
// sensitivities (one parameter direction per launch): d tauc, d l from the
// Nye tensor of dFp_{k-1} and d rho_SSD,k-1; the directional derivative of
// the converged local update (mode 0: dP at dF = 0; mode 1: dFp_k,
// d rho_SSD,k and the mean of dP into mean_out[9])
cudaError_t launch_hard_jvp(const rve_s* h, const double* dnye, const double* drho, double* dtauc, double* dell,
                            Theta dth, cudaStream_t s);
cudaError_t launch_local_jvp(const rve_s* h, double dt, int mode, const double* dF, const double* dFp0,
                             const double* dtauc, const double* dell, const double* drho, double* dP,
                             double* dFp_out, double* drho_out, double* mean_out, Theta dth, cudaStream_t s);
// both
cudaError_t launch_constitutive(const rve_s* h, double dt, double lambda, int out_buf, int warm_buf,
                                cudaStream_t s);

// ---- vec.cu ----
cudaError_t launch_tangent_apply(const rve_s* h, cudaStream_t s);
cudaError_t launch_cg_update(const rve_s* h, cudaStream_t s);
cudaError_t launch_norm2(const rve_s* h, const double* a, int ncomp, cudaStream_t s);
cudaError_t launch_reduce_final(const rve_s* h, int mode, cudaStream_t s);
cudaError_t launch_cg_init(const rve_s* h, double eta, cudaStream_t s);
cudaError_t launch_tangent_apply32(const rve_s* h, cudaStream_t s);
// one-time kernel attributes (shared-memory sizes); before any launch or capture
cudaError_t vec_init();
cudaError_t launch_cg_init32(const rve_s* h, double eta, cudaStream_t s);
cudaError_t launch_widen_x(const rve_s* h, cudaStream_t s);
cudaError_t launch_widen(const rve_s* h, const float* a, double* b, size_t n, cudaStream_t s);
// x_c -= mean(x_c) for the components whose bit is set (uses DS_XMEAN)
cudaError_t launch_zero_means(const rve_s* h, double* x, unsigned bits, cudaStream_t s);
cudaError_t launch_kmul(const rve_s* h, const double* in, double* out, cudaStream_t s);
cudaError_t launch_dots(const rve_s* h, int np, const double* a0, const double* b0, const double* a1,
                        const double* b1, const double* a2, const double* b2, int slot, cudaStream_t s);
cudaError_t launch_lincomb(const rve_s* h, double* out, double c0, const double* a0, double c1, const double* a1,
                           double c2, const double* a2, cudaStream_t s);
cudaError_t launch_axpy_F(const rve_s* h, double lambda, cudaStream_t s);
cudaError_t launch_predictor(const rve_s* h, const double* dFb, const double* dFb_prev, double ratio,
                             int extrapolate, cudaStream_t s);
// F += shift on every voxel (components as given)
cudaError_t launch_shift_F(const rve_s* h, const double* shift, cudaStream_t s);
cudaError_t launch_commit(const rve_s* h, cudaStream_t s);
cudaError_t launch_macro(const rve_s* h, cudaStream_t s);
cudaError_t launch_output_field(const rve_s* h, int which, const double* P, const double* S, double* dst,
                               cudaStream_t s);

enum { RED_PKP_ALPHA = 0, RED_RR_BETA = 1, RED_NORM = 2, RED_RR_INIT = 3, RED_MACRO = 4 };
