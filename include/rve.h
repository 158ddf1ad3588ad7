/*
 * rve.h - C ABI of the GB300 FFT-Galerkin strain-gradient crystal-plasticity
 * increment (Haouala, Lucarini, LLorca, Segurado, arXiv:1910.01946).
 *
 * One handle holds one voxelised FCC polycrystal (a representative volume
 * element, RVE) and advances it one strain increment per rve_step:
 *   - Nye tensor G = -curl Fp by the rotated-scheme spectral derivative
 *     (App. A Eq. kas, App. B Eq. nyeindexfourier);
 *   - GND densities by the minimum-norm inverse of Eq. defA2 (Eq. mingnd);
 *   - Taylor hardening (Eq. Taylor_hard) and mean free path (Eq. meanfree);
 *   - per-voxel implicit crystal-plasticity update and consistent tangent
 *     (Sec. 2.1, Eqs. 1-5, power law, Eq. Piola);
 *   - Newton-Raphson with conjugate gradients on the Galerkin equilibrium
 *     G*(K : dF) = -G*(P - Pbar) under mixed macroscopic control
 *     (Sec. 2.2, Eqs. weakarbi, eql_discrete2, linequil2ast);
 *   - commit of Fp, S and the SSD densities (Kocks-Mecking, Eq. kocks).
 *
 * Conventions for every entry point below:
 *   - voxel index v = x + n0*(y + n1*z) (x fastest); voxels are cubes of
 *     edge h = L/n0 (rve_options.L);
 *   - 3x3 tensors are row-major, component index 3*i + j;
 *   - fields are structure-of-arrays: component c of voxel v at [c*nvox + v];
 *   - units: MPa for moduli and stresses, metres for lengths, m^-2 for
 *     dislocation densities, seconds for time;
 *   - all device memory is the caller's: rve_create carves its state out of
 *     one caller-owned device workspace of rve_workspace_bytes() bytes, which
 *     must outlive the handle; the library itself calls no cudaMalloc for
 *     field storage (it allocates only a small pinned host scalar block);
 *   - every call is issued on the CUDA stream given at rve_create and
 *     returns an rve_status; no exception or abort crosses the ABI.  On a
 *     non-OK status rve_last_error() gives a message.  A device error
 *     (RVE_ECUDA) leaves the handle unusable; every other status leaves the
 *     last committed increment in place and the handle usable.
 */
#ifndef RVE_H
#define RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RVE_OK = 0,
  RVE_EINVAL = 1,         /* bad argument: sizes, pointers, out-of-range values */
  RVE_ENOMEM = 2,         /* workspace too small */
  RVE_ECUDA = 3,          /* a CUDA call failed */
  RVE_ENOCONV_LOCAL = 4,  /* a voxel's implicit update did not converge */
  RVE_ENOCONV_CG = 5,     /* conjugate gradients hit max_cg */
  RVE_ENOCONV_NEWTON = 6, /* Newton-Raphson hit max_newton or could not decrease the residual */
  RVE_ENAN = 7,           /* a non-finite residual (a non-finite value in the state, e.g. set through
                             rve_set_fields); reported before RVE_ENOCONV_LOCAL */
  RVE_ETIMEOUT = 8        /* a bounded wait inside a kernel gave up (see rve_set_wait_limit); the
                             kernel drained its own copies first, nothing was committed and the
                             handle stays usable */
} rve_status;

typedef struct rve_s rve_t;

/* Material (Sec. 2.1, Tables 1-2).  Critical resolved shear stress
 *   tauc^a = tau0 + alpha mu b sqrt(sum_b q^ab (rho_SSD^b + rho_GND^b)),
 * the paper's Eq. Taylor_hard being tau0 = 0, alpha = 1, unnormalised q. */
typedef struct {
  double C11, C12, C44;  /* cubic elastic constants [MPa] */
  double b;              /* Burgers vector length [m] */
  double mu;             /* shear modulus in the Taylor law [MPa]; <= 0: 3 C44 (C11-C12)/(4 C44 + C11 - C12) */
  double tau0;           /* lattice friction [MPa] */
  double alpha;          /* Taylor coefficient [-] */
  double q[6];           /* interaction coefficients: self, coplanar, collinear, Hirth, glissile, Lomer (Table 1) */
  int32_t q_normalise;   /* nonzero: divide q by its self coefficient */
  double gdot0;          /* reference slip rate [1/s] */
  double n;              /* power-law exponent (Table 1 rate sensitivity m = 0.05 -> n = 1/m = 20) */
  double K;              /* similitude coefficient in the mean free path (Eq. meanfree) [-] */
  double yc;             /* annihilation distance (Eq. kocks) [m] */
  double rho0_total;     /* initial SSD density summed over the 12 systems [m^-2] */
  int32_t gnd_enabled;   /* 0: GND densities switched off ("infinite grain size", Sec. 3) */
} rve_material;

typedef struct {
  double L;              /* RVE edge along x [m]; voxel edge h = L / n0 */
  double newton_tol;     /* stop when rms(G*(P - Pbar)) <= newton_tol * max(|<P>|, 1e-4 mu) */
  double cg_tol;         /* CG relative residual */
  double local_tol;      /* local update: max |r| <= local_tol * mu */
  int32_t max_newton, max_cg, max_local, max_halvings;
  int32_t extrapolate;   /* nonzero: predict the increment from the previous one */
  int32_t precision;     /* 0: FP64 throughout.  1: mixed -- the conjugate gradients (tangent storage,
                            stencils, FFT, vectors) in FP32; the local update, tangent computation,
                            equilibrium residual and Newton update in FP64, so the converged
                            increment is the FP64 one (outer Newton refinement) */
  int32_t cg_adaptive;   /* nonzero: CG relative tolerance max(cg_tol, min(1e-2, current relative
                            residual)) (inexact Newton; the converged increment is the same) */
  int32_t krylov;        /* linear solver of the Newton step: 0 conjugate gradients (the paper's
                            solver), and when no step along the CG direction (converged or cut
                            off at max_cg) lowers the residual, the same Newton iteration solved
                            again with BiCGStab (the consistent tangent is not symmetric);
                            1 BiCGStab only; 2 conjugate gradients only */
  int32_t graphs;        /* nonzero: chunks of 8 CG iterations are captured once into a CUDA graph
                            and replayed with one launch (needs a stream other than the legacy
                            default stream; ignored there).  Results are bit-identical. */
  int32_t tma;           /* nonzero: the FP32 tangent apply streams the tangent through shared
                            memory with bulk asynchronous copies (precision 1 only) */
  int32_t autotune;      /* nonzero: rve_create times candidate launch shapes on the handle's own
                            buffers and keeps the fastest (grid of the divergence stencil, FFT
                            tile sizes, staged or plain FP32 tangent apply; see rve_get_tuning).
                            The choice follows measured times, so two tuned handles may differ in
                            reduction order: equal results to round-off, not bit for bit. */
  int32_t stencils;      /* divergence and gradient stencils of the projection: 0 row strips (one
                            warp per x line, separable, no halo) where n0 is 32, 64, 96 or 128, else
                            tiles; 1 tiles always.  Equal results to round-off. */
  int32_t continuation;  /* 0..6: when Newton-Raphson fails on an increment (RVE_ENOCONV_NEWTON,
                            _CG or _LOCAL), solve the same increment again from its start with the
                            macroscopic load in 2^k equal stages, k = 1 .. continuation, each stage
                            starting from the previous one's solution.  The hardening stays frozen
                            over the increment and the last stage solves its own equations: the
                            converged increment is the same, only the path to it differs.  With
                            continuation > 0 the direct solve is given max(8, max_newton / 4)
                            iterations, each stage max_newton. */
} rve_options;

#define RVE_MAX_NEWTON_LOG 64
typedef struct {
  int32_t converged;
  int32_t newton_iters;
  int32_t cg_iters_total;
  int32_t local_max_iters;
  int32_t local_failures;
  int32_t halvings;
  int32_t bicgstab_solves;                      /* Newton steps solved by BiCGStab */
  int32_t load_stages;                          /* 1, or the stages of the load continuation that solved it */
  int64_t local_iters_total;                    /* local Newton iterations summed over voxels and evaluations */
  int64_t local_evals_total;                    /* local residual evaluations, likewise */
  double residual;                              /* final relative residual */
  double seconds;                               /* host wall time of the call */
  int32_t cg_iters[RVE_MAX_NEWTON_LOG];         /* per Newton iteration */
  double residuals[RVE_MAX_NEWTON_LOG + 1];     /* relative residual per Newton iteration */
} rve_step_info;

/* Field selectors for rve_get_fields / rve_set_fields (double unless noted).
 * Committed state (the end of the last converged increment):
 *   F, P, FP, SIGMA (Cauchy P F^T / det F): 9 components; S: 6 (Voigt 11, 22,
 *   33, 23, 13, 12; second Piola-Kirchhoff stress in the intermediate
 *   configuration, sample axes); RHO_SSD: 12 (slip systems); VM: 1 (von Mises
 *   stress of the Cauchy stress); GRAIN: 1 (int32).
 * Hardening of the last increment (computed from Fp at its start, or by
 * rve_eval_hardening from the committed Fp):
 *   NYE: 9; RHO_GND18: 18 (12 edge segments in slip-system order, then 6
 *   screw segments along [0 1 -1], [1 0 -1], [1 -1 0], [0 1 1], [1 0 1],
 *   [1 1 0]); RHO_GND, TAUC: 12.
 * Last local evaluation (the converged one after rve_step, or the one made by
 * rve_eval_constitutive):
 *   P_EVAL: 9; S_EVAL: 6; DGAM: 12 (slip increments); TANGENT: 81
 *   (K_ijkl = dP_ij / dF_kl at component 27*i + 9*j + 3*k + l).  rve_step does
 *   not build the tangent of the converged evaluation (no solve needs it); the
 *   first TANGENT request, or rve_eval_hardening, builds it from that state. */
enum {
  RVE_FIELD_F = 0, RVE_FIELD_P = 1, RVE_FIELD_FP = 2, RVE_FIELD_S = 3,
  RVE_FIELD_SIGMA = 4, RVE_FIELD_RHO_SSD = 5, RVE_FIELD_RHO_GND = 6,
  RVE_FIELD_RHO_GND18 = 7, RVE_FIELD_NYE = 8, RVE_FIELD_VM = 9,
  RVE_FIELD_TAUC = 10, RVE_FIELD_DGAM = 11, RVE_FIELD_TANGENT = 12,
  RVE_FIELD_GRAIN = 13, RVE_FIELD_P_EVAL = 14, RVE_FIELD_S_EVAL = 15
};

/* Bytes of device workspace needed for an n0 x n1 x n2 grid of n_grains
 * grains at the given precision (rve_options.precision).  n0 and n1 must be
 * even, every size a product of 2s and 3s with 2 <= n0, n1 <= 512 and
 * 1 <= n2 <= 512.  Returns 0 for unsupported sizes, grain counts or precision. */
size_t rve_workspace_bytes(int n0, int n1, int n2, int n_grains, int precision);

/* Create a handle.
 *   grain_id: host, n0*n1*n2 int32 in [0, n_grains), voxel order as above;
 *   quat: host, 4*n_grains doubles (w, x, y, z), rotation crystal -> sample
 *         (normalised here);
 *   mat, opt: host structs, copied;
 *   d_workspace: device pointer, 256-byte aligned, ws_bytes >= rve_workspace_bytes();
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Initial state: F = Fp = I, S = 0, rho_SSD = rho0_total / 12 on every system.
 * Errors: RVE_EINVAL (sizes, ids, pointers, options), RVE_ENOMEM (workspace),
 * RVE_ECUDA. */
rve_status rve_create(const int32_t* grain_id, int n0, int n1, int n2,
                      const double* quat, int n_grains,
                      const rve_material* mat, const rve_options* opt,
                      void* d_workspace, size_t ws_bytes, void* cuda_stream,
                      rve_t** out);

/* One strain increment of length dt (Sec. 2.2).  dFbar: host, 9 increments
 * of the macroscopic deformation gradient, used where strain_mask[c] != 0
 * (strain-controlled); Pbar: host, 9 prescribed macroscopic first
 * Piola-Kirchhoff stresses, used where strain_mask[c] == 0.  info: host,
 * may be NULL.  On any status but RVE_OK the state is the last committed
 * increment (the call is atomic). */
rve_status rve_step(rve_t* rve, const double dFbar[9], const uint8_t strain_mask[9],
                    const double Pbar[9], double dt, rve_step_info* info);

/* Batched increments (the grain-size study of Sec. 3-4 runs many RVEs of
 * different sizes): n independent handles (different sizes, grain counts,
 * materials) each advance one increment, concurrently.  One host thread per
 * handle drives that handle's own stream, so the kernels of different RVEs
 * overlap on the GPU (the batched grain-size sweep).  dFbar, strain_mask and
 * Pbar hold 9 values per handle, dt one; info and status (nullable) receive
 * one entry per handle.  Each handle behaves exactly as under rve_step
 * (atomic on failure).  Handles must be distinct; for overlap they must use
 * different streams.  Returns RVE_OK if every step succeeded, else the status
 * of the first handle (in index order) that failed. */
rve_status rve_step_batch(rve_t* const* rves, int n, const double* dFbar, const uint8_t* strain_mask,
                          const double* Pbar, const double* dt, rve_step_info* info, rve_status* status);

/* Volume averages of the first Piola-Kirchhoff stress and of the Cauchy
 * stress P F^T / det F over the committed state; host outputs. */
rve_status rve_get_macro_stress(rve_t* rve, double P[9], double sigma[9]);

/* Copy one field (see the selectors) to dst (host or device memory per
 * dst_is_device); bytes >= ncomp * nvox * element size, else RVE_EINVAL. */
rve_status rve_get_fields(rve_t* rve, uint32_t which, void* dst, size_t bytes, int dst_is_device);

/* Overwrite one committed state field (F, FP or RHO_SSD) from src (host or
 * device per src_is_device, bytes == ncomp * nvox * 8).  Used to set up a
 * test state; other selectors give RVE_EINVAL. */
rve_status rve_set_fields(rve_t* rve, uint32_t which, const void* src, size_t bytes, int src_is_device);

/* Kernel-level entry points on the committed state (used for per-step parity
 * checks):
 *   rve_eval_hardening: Nye tensor, GND densities and tauc from the committed
 *     Fp and SSD densities (fields NYE, RHO_GND18, RHO_GND, TAUC);
 *   rve_eval_constitutive: rve_eval_hardening, then the local update and
 *     tangent at the committed F over an increment dt from the committed Fp
 *     (warm start: the committed S); fields P_EVAL, S_EVAL, DGAM, TANGENT.
 *     local_max_iters / local_failures (host, nullable) receive the largest
 *     local iteration count and the number of voxels that did not converge;
 *   rve_project: Y = G*(X) for device fields X, Y (9 * nvox doubles each,
 *     may alias) under the given strain mask (zero mode: components with
 *     strain_mask[c] == 0 kept, the others zeroed). */
rve_status rve_eval_hardening(rve_t* rve);
/* Nye tensor of the committed Fp alone (field NYE), G_ij = -eps_jkl d_k Fp_il,
 * with the derivative of scheme 0: the rotated-scheme discrete derivative the
 * method uses (App. A Eq. kas, App. B Eq. nyeindexfourier), or 1: the
 * standard spectral derivative i xi_k / h (the continuous frequencies App. A
 * contrasts it with; 0 at the Nyquist frequency), which rings (Gibbs
 * oscillations) where Fp jumps across a grain boundary (App. B).  The
 * hardening fields are left as they were.  Errors: RVE_EINVAL for another
 * scheme. */
rve_status rve_eval_nye(rve_t* rve, int scheme);
rve_status rve_eval_constitutive(rve_t* rve, double dt, int32_t* local_max_iters, int32_t* local_failures);
rve_status rve_project(rve_t* rve, const uint8_t strain_mask[9], const double* d_X, double* d_Y);

/* Checkpoint: host buffer of rve_checkpoint_bytes() bytes holding F, Fp, S,
 * rho_SSD, the previous increment and the macro history; rve_restore checks
 * sizes and a magic/version word (RVE_EINVAL on mismatch). */
size_t rve_checkpoint_bytes(const rve_t* rve);
rve_status rve_checkpoint(rve_t* rve, void* host_buf, size_t bytes);
rve_status rve_restore(rve_t* rve, const void* host_buf, size_t bytes);

/* Kernel accounting (no counterpart in the paper: instrumentation for the
 * measurements).  Every kernel launch is counted per category (always on).
 * With rve_profile(rve, 1) each launch is also bracketed by CUDA events on
 * the handle's stream and its device time accumulated per category (the
 * events are resolved at the library's own host synchronisation points);
 * rve_profile(rve, 0) stops timing.  Both calls reset the counters.
 * rve_kernel_stats copies RVE_K_COUNT launch counts and milliseconds (host
 * arrays, either may be NULL). */
enum {
  RVE_K_FFT_X_R2C = 0, RVE_K_FFT_Y = 1, RVE_K_FFT_Z_OP = 2, RVE_K_FFT_X_C2R = 3,
  RVE_K_CONSTITUTIVE = 4, RVE_K_HARDENING = 5, RVE_K_TANGENT_APPLY = 6, RVE_K_CG_UPDATE = 7,
  RVE_K_REDUCE = 8, RVE_K_OTHER = 9, RVE_K_STENCIL = 10, RVE_K_TANGENT_BUILD = 11,
  RVE_K_FFT_CURL = 12,   /* all five passes of the nine-field Nye-curl FFT (the other FFT
                            categories count the three-field transforms of the projection) */
  RVE_K_FFT_Y_INV = 13,  /* the inverse y pass (RVE_K_FFT_Y counts the forward one) */
  RVE_K_COUNT = 14
};
rve_status rve_profile(rve_t* rve, int enable);
/* The launch shapes in use (no counterpart in the paper): out[0] grid cap of
 * the divergence stencil (blocks),
 * out[1] block count the FFT tile rules aim for in the x passes, out[2] 1 if
 * the FP32 tangent apply is staged by bulk copies, out[3] 1 if the autotuner
 * chose them, out[4] and out[5] the FFT block counts aimed for in the y
 * passes and the z pass (host array of 6). */
rve_status rve_get_tuning(rve_t* rve, int32_t out[6]);
rve_status rve_kernel_stats(rve_t* rve, int64_t* launches, double* ms);

/* Device time of the hand-written FFT alone (no counterpart in the paper:
 * instrumentation for the comparison with a vendor FFT): nf real fields of
 * the handle's grid (nf = 3: the projection's transforms, with its
 * inverse-Laplacian weight fused between the z passes; nf = 9: the nine-field
 * transforms with the Galerkin projection fused) forward and back, `reps`
 * times on the handle's stream and buffers, timed with CUDA events.  fp32 = 1
 * times the FP32 transforms of the mixed-precision conjugate gradients (nf =
 * 3, precision 1 handles only).  ms (host): average time of one forward +
 * inverse pair.  Overwrites the handle's scratch (not its committed state).
 * Errors: RVE_EINVAL for other nf / fp32 combinations. */
rve_status rve_time_fft(rve_t* rve, int nf, int fp32, int reps, double* ms);

/* Poll limit of the per-tile wait in the staged FP32 tangent apply
 * (rve_options.tma, precision 1; no counterpart in the paper: a bounded wait
 * of the GPU design).  Each block of that kernel waits on an mbarrier for its
 * bulk copies; after `polls` unsuccessful polls (default 4194304; 0 gives up
 * at the first wait without polling) the block raises a device flag, waits at
 * the default limit for every copy it still has in flight, and leaves.  The
 * host finds the flag after the CG chunk and rve_step returns RVE_ETIMEOUT
 * with the last committed increment intact; the handle stays usable.  A
 * small limit makes that recovery path run on purpose (tests).  Drops the
 * captured CG graphs, which carry the limit as a kernel argument. */
rve_status rve_set_wait_limit(rve_t* rve, uint32_t polls);

/* Allocation-free Galerkin projection (no counterpart in the paper; an
 * addition for callers that cannot allocate device memory).
 *
 * Y = G*(X) for device fields X and Y (9 * n0*n1*n2 doubles each, layout as
 * above, may alias) on an n0 x n1 x n2 grid of edge L along x, under
 * strain_mask (host, 9 bytes): the same linear map as rve_project, computed in
 * the nine-field Fourier form (rve_project uses the stencil-factored form), so
 * the two agree to round-off.  It needs no handle and no workspace: the FFT
 * spectrum and frequency tables live in one static device array of
 * RVE_NOALLOC_SPEC_BYTES plus about 64 KiB, which every GPU that loads the
 * library holds until the process exits.  Meant for code that must not call
 * cudaMalloc: for example a plug-in running under a host application whose
 * memory manager has already reserved the device memory, or a time-critical
 * loop that cannot afford cudaMalloc/cudaFree's implicit device-wide
 * synchronisation.  This entry point calls no cudaMalloc, cudaFree or other
 * allocating routine, and copies nothing from the host.
 *
 * Work is queued on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without waiting: synchronise the stream before
 * reading Y.  The first call on a device looks up the device address of the
 * static array (cudaGetSymbolAddress, once per device, with that device
 * current) and, like every call whose grid differs from the previous call's on
 * that device, launches one small kernel that writes the frequency tables into
 * the array; make that first call before any stream capture.  All calls share
 * the one array, which keeps the last call's contents: calls that overlap on
 * the GPU (different streams, or different host threads) race on it.  The
 * cached address and tables do not survive cudaDeviceReset: do not call this
 * entry point after resetting the device in the same process.
 *
 * Errors: RVE_EINVAL for bad pointers, L <= 0 or unsupported sizes (as in
 * rve_workspace_bytes); RVE_ENOMEM when 9 * (n0/2 + 1) * n1 * n2 * 16 bytes of
 * spectrum exceed RVE_NOALLOC_SPEC_BYTES (64^3 fits; 96^3 does not);
 * RVE_ECUDA when a CUDA call fails. */
#define RVE_NOALLOC_SPEC_BYTES ((size_t)32 * 1024 * 1024)
rve_status rve_project_noalloc(int n0, int n1, int n2, double L, const uint8_t strain_mask[9],
                               const double* d_X, double* d_Y, void* cuda_stream);

/* Sensitivities of the macroscopic stress with respect to the material
 * parameters theta = (tau0 [MPa], K [-], alpha [-], b [m]) (differentiation of
 * the incremental solve; the paper fits such parameters to Hall-Petch data in
 * Sec. 4).  Forward mode through the same discrete equations rve_step solves:
 * the hardening (Eqs. Taylor_hard, meanfree, with the GND densities of
 * Eqs. defA2 / mingnd scaling as 1/b), the implicit local update, the
 * equilibrium G*(K : dF) = -G*(dP|_dF=0) with the converged increment's
 * consistent tangent (Eq. linequil2ast; one linear solve per parameter and
 * increment, CG with a BiCGStab retry in FP64, BiCGStab in mixed precision),
 * and the implicit Kocks-Mecking commit (Eq. kocks).  The state tangents
 * dFp and d rho_SSD carry the load history.
 *
 * rve_sensitivity_bytes: device bytes the tangents and scratch need.
 * rve_sensitivity_enable: d_workspace is caller-owned device memory (256-byte
 *   aligned, >= rve_sensitivity_bytes, outliving the handle); the tangents
 *   start at zero, i.e. the current state is taken as independent of theta
 *   (exact from the initial state).  tol: relative tolerance of the linear
 *   solves, used as given by both the CG and the BiCGStab solve (<= 0: the
 *   larger of rve_options.cg_tol and 1e-9, BiCGStab at no less than 1e-12).
 *   From then on every rve_step also updates the sensitivities before it
 *   commits; a solve that reaches max_cg in both solvers fails the step
 *   (RVE_ENOCONV_CG, rve_step_info.converged 0) with nothing committed.
 *   rve_restore zeroes the tangents.
 * rve_get_stress_sensitivity: dP[9 * j + 3 * i + k] = d<P_ik> / d theta_j of
 *   the last converged increment (host array of 36); RVE_EINVAL when there is
 *   none. */
#define RVE_NTHETA 4
size_t rve_sensitivity_bytes(const rve_t* rve);
rve_status rve_sensitivity_enable(rve_t* rve, void* d_workspace, size_t bytes, double tol);
rve_status rve_get_stress_sensitivity(rve_t* rve, double dP[RVE_NTHETA * 9]);

const char* rve_last_error(const rve_t* rve);
void rve_destroy(rve_t* rve);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
