// C ABI and host orchestration of one strain increment (Sec. 2.2 of the
// paper): Nye tensor and hardening, predictor, Newton-Raphson with conjugate
// gradients on G*(K : dF) = -G*(P - Pbar) (Eq. linequil2ast), backtracking
// on the residual norm, commit.  Every kernel runs on the caller's stream;
// the host reads back only a few scalars per iteration.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "rve_internal.h"

namespace {

const uint32_t CKPT_MAGIC = 0x43455652u;  // "RVEC"
const uint32_t CKPT_VERSION = 1;

#define RVE_CUDA(h, call)                                                          \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return RVE_ECUDA;                                                            \
    }                                                                              \
  } while (0)

#define RVE_TRY(call)                   \
  do {                                  \
    rve_status s_ = (call);             \
    if (s_ != RVE_OK) return s_;        \
  } while (0)

rve_status fail(rve_s* h, rve_status s, const char* msg);

bool good_len(int n, int lo) {
  if (n < lo || n > 512) return false;
  FFTPlan p;
  make_plan(n, &p);
  return p.npass >= 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout: carve() walks the same sequence for sizing and for
// assigning pointers.
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    size_t o = off;
    off = align256(off + count * sizeof(T));
    return base ? reinterpret_cast<T*>(base + o) : nullptr;
  }
};

void carve(rve_s* h, Carver& c) {
  const size_t nv = h->nvox;
  h->grain = c.take<int32_t>(nv);
  h->grainR = c.take<double>(9 * (size_t)h->ngrains);
  h->qhat = c.take<double>(144);
  h->Apinv = c.take<double>(162);
  h->screw_of = c.take<int32_t>(12);
  const int ns[3] = {h->n0, h->n1, h->n2};
  for (int a = 0; a < 3; ++a) {
    h->ax[a].tw = c.take<double2>(ns[a]);
    h->ax[a].tanh_ = c.take<double>(ns[a]);
    h->ax[a].nyq = c.take<int8_t>(ns[a]);
    h->ax[a].ph = c.take<double2>(ns[a]);
    h->ax[a].s2 = c.take<double>(ns[a]);
    h->ax[a].c2 = c.take<double>(ns[a]);
    h->ax[a].xi = c.take<double>(ns[a]);
  }
  h->F_c = c.take<double>(9 * nv);
  h->Fp = c.take<double>(9 * nv);
  h->S_c = c.take<double>(6 * nv);
  h->rho_ssd = c.take<double>(12 * nv);
  h->dF_last = c.take<double>(9 * nv);
  h->P_c = c.take<double>(9 * nv);
  h->nye = c.take<double>(9 * nv);
  h->rho18 = c.take<double>(18 * nv);
  h->rho_gnd = c.take<double>(12 * nv);
  h->tauc = c.take<double>(12 * nv);
  h->ell = c.take<double>(12 * nv);
  h->Fp0inv = c.take<double>(9 * nv);
  h->F = c.take<double>(9 * nv);
  for (int b = 0; b < 2; ++b) {
    h->P[b] = c.take<double>(9 * nv);
    h->K[b] = c.take<double>(81 * nv);
    h->S[b] = c.take<double>(6 * nv);
    h->dgam[b] = c.take<double>(12 * nv);
  }
  h->R = c.take<double>(9 * nv);
  h->x = c.take<double>(9 * nv);
  h->r = c.take<double>(9 * nv);
  h->p = c.take<double>(9 * nv);
  h->t = c.take<double>(9 * nv);
  h->q = c.take<double>(9 * nv);
  h->bv = c.take<double>(9 * nv);
  h->bs = c.take<double>(9 * nv);
  h->spec = c.take<double2>(9 * h->nspec);
  h->lapw = c.take<double>(h->nspec);
  if (h->opt.precision == 1) {
    for (int a = 0; a < 3; ++a) h->ax[a].tw32 = c.take<float2>(ns[a]);
    h->spec32 = c.take<float2>(3 * h->nspec);
    h->x32 = c.take<float>(9 * nv);
    h->r32 = c.take<float>(9 * nv);
    h->p32 = c.take<float>(9 * nv);
    h->t32 = c.take<float>(9 * nv);
    h->du32 = c.take<float>(6 * nv);
  } else {
    for (int a = 0; a < 3; ++a) h->ax[a].tw32 = nullptr;
    h->spec32 = nullptr;
    h->x32 = h->r32 = h->p32 = h->t32 = h->du32 = nullptr;
  }
  h->partial = c.take<double>(9 * 4096 + 27 * (size_t)RVE_RED_BLOCKS);
  h->dscal = c.take<double>(64);
  h->dcount = c.take<int32_t>(16);
}

// ---- host tables (crystallography written from the geometry of FCC slip) ----
const int SL_S[12][3] = {{0, 1, -1}, {-1, 0, 1}, {1, -1, 0}, {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
                         {0, 1, 1}, {1, 0, -1}, {1, 1, 0}, {0, 1, 1}, {1, 0, 1}, {1, -1, 0}};
const int SL_M[12][3] = {{1, 1, 1}, {1, 1, 1}, {1, 1, 1}, {-1, 1, 1}, {-1, 1, 1}, {-1, 1, 1},
                         {1, -1, 1}, {1, -1, 1}, {1, -1, 1}, {1, 1, -1}, {1, 1, -1}, {1, 1, -1}};
const int SCREW[6][3] = {{0, 1, -1}, {1, 0, -1}, {1, -1, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

int idot(const int* a, const int* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// interaction class of systems (a, b): 0 self, 1 coplanar, 2 collinear,
// 3 Hirth, 4 glissile junction, 5 Lomer-Cottrell lock
int interaction_class(int a, int b) {
  if (a == b) return 0;
  const int* sa = SL_S[a]; const int* sb = SL_S[b];
  const int* ma = SL_M[a]; const int* mb = SL_M[b];
  const int mm = idot(ma, mb);
  if (mm == 3 || mm == -3) return 1;              // same plane (|m| = sqrt 3)
  const int ss = idot(sa, sb);                     // |s|^2 = 2
  if (ss == 2 || ss == -2) return 2;               // same Burgers direction
  if (ss == 0) return 3;                           // perpendicular Burgers vectors
  int j[3];
  const int sg = ss > 0 ? 1 : -1;                  // junction b = b_a - sign(b_a.b_b) b_b
  for (int k = 0; k < 3; ++k) j[k] = sa[k] - sg * sb[k];
  return (idot(j, ma) == 0 || idot(j, mb) == 0) ? 4 : 5;
}

// Gauss-Jordan inverse with partial pivoting (n x n, row-major); false if singular
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    for (int j = 0; j < n; ++j) { std::swap(A[k * n + j], A[p * n + j]); std::swap(I[k * n + j], I[p * n + j]); }
    const double d = 1.0 / A[k * n + k];
    for (int j = 0; j < n; ++j) { A[k * n + j] *= d; I[k * n + j] *= d; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A[i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) { A[i * n + j] -= f * A[k * n + j]; I[i * n + j] -= f * I[k * n + j]; }
    }
  }
  A = I;
  return true;
}

void build_tables(const rve_material& m, std::vector<double>& q, std::vector<double>& Ap, std::vector<int32_t>& screw) {
  q.assign(144, 0.0);
  const double norm = m.q_normalise ? m.q[0] : 1.0;
  for (int a = 0; a < 12; ++a)
    for (int b = 0; b < 12; ++b) q[12 * a + b] = m.q[interaction_class(a, b)] / norm;
  // A (9 x 18), crystal frame, unit b and t: columns = vec(b (x) t)
  double A[9][18];
  for (int a = 0; a < 18; ++a) {
    double bv[3], tv[3];
    if (a < 12) {
      const double is2 = 1.0 / std::sqrt(2.0), is3 = 1.0 / std::sqrt(3.0);
      double s[3], mm[3];
      for (int k = 0; k < 3; ++k) { s[k] = SL_S[a][k] * is2; mm[k] = SL_M[a][k] * is3; }
      for (int k = 0; k < 3; ++k) bv[k] = s[k];
      tv[0] = mm[1] * s[2] - mm[2] * s[1];   // t = m x s
      tv[1] = mm[2] * s[0] - mm[0] * s[2];
      tv[2] = mm[0] * s[1] - mm[1] * s[0];
    } else {
      const double is2 = 1.0 / std::sqrt(2.0);
      for (int k = 0; k < 3; ++k) bv[k] = tv[k] = SCREW[a - 12][k] * is2;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[3 * i + j][a] = bv[i] * tv[j];
  }
  std::vector<double> AAt(81, 0.0);
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      double s = 0.0;
      for (int a = 0; a < 18; ++a) s += A[i][a] * A[j][a];
      AAt[9 * i + j] = s;
    }
  invert(AAt, 9);
  Ap.assign(162, 0.0);   // A^T (A A^T)^-1 / b
  for (int a = 0; a < 18; ++a)
    for (int j = 0; j < 9; ++j) {
      double s = 0.0;
      for (int i = 0; i < 9; ++i) s += A[i][a] * AAt[9 * i + j];
      Ap[9 * a + j] = s / m.b;
    }
  screw.assign(12, 0);
  for (int a = 0; a < 12; ++a)
    for (int d = 0; d < 6; ++d) {
      const int v = idot(SL_S[a], SCREW[d]);
      if (v == 2 || v == -2) screw[a] = d;
    }
}

void quat_to_R(const double* qin, double* R) {
  double w = qin[0], x = qin[1], y = qin[2], z = qin[3];
  const double n = std::sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

rve_status read_scalars(rve_s* h) {
  RVE_CUDA(h, cudaMemcpyAsync(h->hscal, h->dscal, 64 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  RVE_CUDA(h, cudaMemcpyAsync(h->hcount, h->dcount, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->prof.on) h->prof.resolve();
  return RVE_OK;
}


SpecParams project_params(const rve_s* h, const uint8_t* mask, const double* shift, double* mean_out) {
  SpecParams sp;
  sp.op = OP_PROJECT;
  for (int c = 0; c < 9; ++c) {
    sp.keep[c] = mask[c] ? 0 : 1;
    sp.shift[c] = shift ? shift[c] : 0.0;
  }
  sp.inv_nvox = 1.0 / (double)h->nvox;
  sp.inv4h = 0.25 / h->h;
  sp.mean_out = mean_out;
  return sp;
}

rve_status run_project(rve_s* h, const double* in, double* out, const SpecParams& sp) {
  RVE_CUDA(h, launch_fft_forward(h, in, h->stream));
  RVE_CUDA(h, launch_fft_op(h, sp, h->stream));
  RVE_CUDA(h, launch_fft_inverse(h, out, h->stream));
  return RVE_OK;
}

// Y = G*(X) (minus the prescribed mean `shift` on the kept components) as
// divergence stencil, scalar Laplace solve by FFT, gradient stencil; leaves
// mean(X) in DS_XMEAN and sum Y^2 in DS_NORM.  Scratch: the first six
// components of q (divergence, then the Laplace solution).
// bits of the stress-controlled components: the zero mode keeps their means
unsigned kept_means(const uint8_t* mask) {
  unsigned m = 0;
  for (int c = 0; c < 9; ++c)
    if (!mask[c]) m |= 1u << c;
  return m;
}

// all_means: reduce the means of all nine fields (the residual's scale is the
// norm of the mean stress); otherwise only the kept ones
rve_status run_project_stencil(rve_s* h, const double* X, double* Y, const uint8_t* mask, const double* shift,
                               bool all_means = false) {
  double* d = h->q;
  double* u = h->q + 3 * h->nvox;
  SpecParams sp = project_params(h, mask, nullptr, nullptr);
  sp.op = OP_LAPINV;
  RVE_CUDA(h, launch_div(h, X, d, 0, all_means ? 0x1FFu : kept_means(mask), h->stream));
  RVE_CUDA(h, launch_fft_forward(h, d, h->stream, nullptr, 3));
  RVE_CUDA(h, launch_fft_op(h, sp, h->stream, nullptr, 3));
  RVE_CUDA(h, launch_fft_inverse(h, u, h->stream, nullptr, 3));
  RVE_CUDA(h, launch_grad(h, u, Y, mask, shift, h->stream));
  return RVE_OK;
}

// the nine-field curl transforms, counted in their own profiling category
rve_status run_curl(rve_s* h, const double* in, double* out) {
  SpecParams sp = project_params(h, (const uint8_t*)"\0\0\0\0\0\0\0\0\0", nullptr, nullptr);
  sp.op = OP_CURL;
  h->fft_cat = RVE_K_FFT_CURL;
  const rve_status st = run_project(h, in, out, sp);
  h->fft_cat = -1;
  return st;
}

rve_status run_hardening(rve_s* h) {
  RVE_TRY(run_curl(h, h->Fp, h->nye));
  RVE_CUDA(h, launch_hardening(h, h->stream));
  return RVE_OK;
}

// evaluate the local update at F + lambda x into buffer `out` and the
// residual R = G*(P - Pbar); returns rms(R) and the mean of P
rve_status eval_residual(rve_s* h, double dt, double lambda, int out, int warm, const uint8_t* mask,
                         const double* Pbar_m, double* rabs, double* scale, int* lmax, int* lfail) {
  RVE_CUDA(h, cudaMemsetAsync(h->dcount, 0, 2 * sizeof(int32_t), h->stream));
  RVE_CUDA(h, launch_local(h, dt, lambda, out, warm, h->stream));
  RVE_TRY(run_project_stencil(h, h->P[out], h->R, mask, Pbar_m, true));
  RVE_TRY(read_scalars(h));
  *rabs = std::sqrt(h->hscal[DS_NORM] / (double)h->nvox);
  double pn = 0.0;
  for (int c = 0; c < 9; ++c) pn += h->hscal[DS_XMEAN + c] * h->hscal[DS_XMEAN + c];
  *scale = std::fmax(std::sqrt(pn), 1e-4 * h->mu);
  *lmax = h->hcount[0];
  *lfail = h->hcount[1];
  return RVE_OK;
}

// CG on G*(K : x) = -R from x = 0 to relative residual eta.  Iterations are
// queued in chunks; the device stops the loop itself (every CG kernel returns
// at once after convergence), the host looks at the flag once per chunk.
const int CG_CHUNK = 8;

void release_graph(CgGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  for (auto& p : g.rec.events) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto e : g.rec.spare) cudaEventDestroy(e);
  g.rec = Prof::Capture();
  g.cur = -1;
}

// Issue one full chunk of CG iterations.  With rve_options.graphs (and a
// stream other than the legacy default stream, which cannot be captured) the
// chunk is captured once per (tangent buffer, strain mask, profiling) into a
// CUDA graph and replayed with a single launch: every launch of the chunk has
// the same arguments and all iteration state lives on the device.  Up to
// RVE_CG_GRAPHS captured chunks are kept per handle.
template <class Issue>
rve_status cg_chunk(rve_s* h, const uint8_t* mask, Issue issue) {
  if (!h->opt.graphs || h->stream == nullptr) return issue();
  const unsigned key = kept_means(mask);
  CgGraph* g = nullptr;
  for (auto& c : h->graphs)
    if (c.exec && c.cur == h->cur && c.key == key && c.timed == h->prof.on) g = &c;
  if (!g) {
    g = &h->graphs[h->graph_next];
    h->graph_next = (h->graph_next + 1) % RVE_CG_GRAPHS;
    release_graph(*g);
    if (h->prof.on) {
      // two events per launch: created before the capture starts
      for (int k = 0; k < 2 * 16 * CG_CHUNK; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) break;
        g->rec.spare.push_back(e);
      }
    }
    RVE_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->prof.cap = &g->rec;
    const rve_status st = issue();
    h->prof.cap = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
    if (st != RVE_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      release_graph(*g);
      if (st != RVE_OK) return st;
      RVE_CUDA(h, ec);
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g->exec = nullptr;
      release_graph(*g);
      RVE_CUDA(h, ei);
    }
    g->cur = h->cur;
    g->key = key;
    g->timed = h->prof.on;
  }
  RVE_CUDA(h, cudaGraphLaunch(g->exec, h->stream));
  for (int c = 0; c < RVE_K_COUNT; ++c) h->prof.launches[c] += g->rec.launches[c];
  if (g->timed) h->prof.borrowed.insert(h->prof.borrowed.end(), g->rec.events.begin(), g->rec.events.end());
  return RVE_OK;
}

rve_status cg_solve(rve_s* h, const uint8_t* mask, double eta, int* iters, bool* ok) {
  RVE_CUDA(h, launch_cg_init(h, eta, h->stream));
  SpecParams sp = project_params(h, mask, nullptr, nullptr);
  sp.op = OP_LAPINV;
  const double* done = h->dscal + DS_DONE;
  double* d = h->q;
  double* u = h->q + 3 * h->nvox;
  int issued = 0;
  *ok = false;
  while (issued < h->opt.max_cg) {
    const int chunk = std::min(CG_CHUNK, h->opt.max_cg - issued);
    auto issue = [&]() -> rve_status {
      for (int i = 0; i < chunk; ++i) {
        // t = K : p, then q = G*(t) as div -> Laplace solve -> grad fused with the update
        RVE_CUDA(h, launch_tangent_apply(h, h->stream));
        RVE_CUDA(h, launch_div(h, h->t, d, 1, kept_means(mask), h->stream));
        RVE_CUDA(h, launch_fft_forward(h, d, h->stream, done, 3));
        RVE_CUDA(h, launch_fft_op(h, sp, h->stream, done, 3));
        RVE_CUDA(h, launch_fft_inverse(h, u, h->stream, done, 3));
        RVE_CUDA(h, launch_grad_cg(h, u, mask, h->stream));
      }
      return RVE_OK;
    };
    RVE_TRY(chunk == CG_CHUNK ? cg_chunk(h, mask, issue) : issue());
    issued += chunk;
    RVE_TRY(read_scalars(h));
    if (h->hscal[DS_DONE] != 0.0) break;
  }
  *iters = (int)h->hscal[DS_ITERS];
  *ok = h->hscal[DS_DONE] != 0.0 && std::isfinite(h->hscal[DS_RR]);
  return RVE_OK;
}

// Mixed precision: the same CG in FP32 (tangent, vectors, stencils, FFT);
// the solution is widened to FP64 for the Newton update.  The FP32 loop
// cannot go below a relative residual of about 1e-6, so eta >= 1e-5.
rve_status cg_solve32(rve_s* h, const uint8_t* mask, double eta, int* iters, bool* ok) {
  eta = std::fmax(eta, 1e-5);
  RVE_CUDA(h, launch_cg_init32(h, eta, h->stream));
  SpecParams sp = project_params(h, mask, nullptr, nullptr);
  sp.op = OP_LAPINV;
  const double* done = h->dscal + DS_DONE;
  float* d = h->du32;
  float* u = h->du32 + 3 * h->nvox;
  int issued = 0;
  *ok = false;
  while (issued < h->opt.max_cg) {
    const int chunk = std::min(CG_CHUNK, h->opt.max_cg - issued);
    auto issue = [&]() -> rve_status {
      for (int i = 0; i < chunk; ++i) {
        RVE_CUDA(h, launch_tangent_apply32(h, h->stream));
        RVE_CUDA(h, launch_div32(h, h->t32, d, kept_means(mask), h->stream));
        RVE_CUDA(h, launch_fft_forward32(h, d, h->stream, done));
        RVE_CUDA(h, launch_fft_lapinv32(h, sp, h->stream, done));
        RVE_CUDA(h, launch_fft_inverse32(h, u, h->stream, done));
        RVE_CUDA(h, launch_grad_cg32(h, u, mask, h->stream));
      }
      return RVE_OK;
    };
    RVE_TRY(chunk == CG_CHUNK ? cg_chunk(h, mask, issue) : issue());
    issued += chunk;
    RVE_TRY(read_scalars(h));
    if (h->hscal[DS_ERR] != 0.0) {
      // every block drained its copies before it left; the context is intact
      RVE_CUDA(h, cudaMemsetAsync(h->dscal + DS_ERR, 0, sizeof(double), h->stream));
      return fail(h, RVE_ETIMEOUT, "a bounded wait for a staged copy gave up");
    }
    if (h->hscal[DS_DONE] != 0.0) break;
  }
  RVE_CUDA(h, launch_widen_x(h, h->stream));
  *iters = (int)h->hscal[DS_ITERS];
  *ok = h->hscal[DS_DONE] != 0.0 && std::isfinite(h->hscal[DS_RR]);
  // FP32 rounding leaves a small incompatible part in the iterate, which the
  // projected residual cannot see; one FP64 projection puts the correction
  // back in the range of G* (compatible fluctuation plus the stress-controlled
  // mean), so F stays compatible to FP64 round-off
  RVE_TRY(run_project_stencil(h, h->x, h->x, mask, nullptr));
  return RVE_OK;
}

// BiCGStab (van der Vorst) on G*(K : x) = -R from x = 0, in FP64 (the
// tangent is read as stored).  The consistent tangent is not symmetric; when
// conjugate gradients stall on it (plastic onset in large RVEs) this is the
// fallback.  r^ = r0 = -R.  Two operator applications and three host reads
// of fused dot products per iteration.
rve_status bicgstab_solve(rve_s* h, const uint8_t* mask, double eta, int* iters, bool* ok) {
  cudaStream_t st = h->stream;
  double* x = h->x; double* r = h->r; double* p = h->p; double* v = h->bv; double* sv = h->bs;
  double* t = h->t;
  const double* R = h->R;        // r^ = -R
  auto dots = [&](int np, const double* a0, const double* b0, const double* a1, const double* b1,
                  const double* a2, const double* b2, double* out) -> rve_status {
    RVE_CUDA(h, launch_dots(h, np, a0, b0, a1, b1, a2, b2, DS_DOT, st));
    RVE_TRY(read_scalars(h));
    for (int k = 0; k < np; ++k) out[k] = h->hscal[DS_DOT + k];
    return RVE_OK;
  };
  auto apply = [&](const double* in, double* out) -> rve_status {   // out = G*(K : in)
    RVE_CUDA(h, launch_kmul(h, in, t, st));
    RVE_TRY(run_project_stencil(h, t, out, mask, nullptr));
    return RVE_OK;
  };
  RVE_CUDA(h, launch_lincomb(h, x, 0.0, R, 0.0, nullptr, 0.0, nullptr, st));
  RVE_CUDA(h, launch_lincomb(h, r, -1.0, R, 0.0, nullptr, 0.0, nullptr, st));
  RVE_CUDA(h, launch_lincomb(h, p, 0.0, R, 0.0, nullptr, 0.0, nullptr, st));
  RVE_CUDA(h, launch_lincomb(h, v, 0.0, R, 0.0, nullptr, 0.0, nullptr, st));
  double d[3];
  RVE_TRY(dots(1, r, r, nullptr, nullptr, nullptr, nullptr, d));
  const double stop = eta * eta * d[0];
  double rho = 1.0, alpha = 1.0, omega = 1.0, rho_new = d[0];   // r^ . r0 = r0 . r0
  *ok = !(d[0] > 0.0);
  int k = 0;
  for (; k < h->opt.max_cg && !*ok; ++k) {
    if (rho_new == 0.0 || !std::isfinite(rho_new)) break;
    const double beta = (rho_new / rho) * (alpha / omega);
    RVE_CUDA(h, launch_lincomb(h, p, 1.0, r, beta, p, -beta * omega, v, st));     // p = r + beta (p - omega v)
    RVE_TRY(apply(p, v));
    RVE_TRY(dots(1, R, v, nullptr, nullptr, nullptr, nullptr, d));
    const double rv = -d[0];
    if (rv == 0.0 || !std::isfinite(rv)) break;
    alpha = rho_new / rv;
    RVE_CUDA(h, launch_lincomb(h, sv, 1.0, r, -alpha, v, 0.0, nullptr, st));      // s = r - alpha v
    RVE_TRY(apply(sv, t));                                                        // t = A s (in place)
    RVE_TRY(dots(3, t, sv, t, t, sv, sv, d));
    if (!(d[2] > stop)) {                                                         // s small enough
      RVE_CUDA(h, launch_lincomb(h, x, 1.0, x, alpha, p, 0.0, nullptr, st));
      *ok = true;
      ++k;
      break;
    }
    if (!(d[1] > 0.0)) break;
    omega = d[0] / d[1];
    RVE_CUDA(h, launch_lincomb(h, x, 1.0, x, alpha, p, omega, sv, st));           // x += alpha p + omega s
    RVE_CUDA(h, launch_lincomb(h, r, 1.0, sv, -omega, t, 0.0, nullptr, st));      // r = s - omega t
    RVE_TRY(dots(2, R, r, r, r, nullptr, nullptr, d));
    rho = rho_new;
    rho_new = -d[0];
    if (!(d[1] > stop)) { *ok = true; ++k; break; }
    if (omega == 0.0) break;
  }
  *iters = k;
  return RVE_OK;
}

// Forward-mode sensitivities of the converged increment (before its commit):
// for each parameter direction, the Nye tensor of dFp_{k-1} (9-field Fourier
// curl), d tauc and d l, the local update's derivative at dF = 0, the
// equilibrium solve G*(K : dF) = -G*(dP|_dF=0) with the converged tangent, and
// the local derivative along dF, which also gives dFp_k, d rho_SSD,k and
// d<P>.  The new state tangents go to the other buffer (swapped at commit).
rve_status sens_update(rve_s* h, const uint8_t* mask, double dt) {
  const int cur = h->cur, sc = h->sens_cur, sn = 1 - h->sens_cur;
  RVE_CUDA(h, launch_tangent(h, dt, 0.0, cur, h->stream));
  // the sensitivities need a few more digits than their uses (gradients
  // checked to 1e-5 against differences): 1e-9 by default
  const double eta = h->sens_tol > 0 ? h->sens_tol : std::fmax(h->opt.cg_tol, 1e-9);
  for (int j = 0; j < RVE_NTHETA; ++j) {
    Theta th{j == 0 ? 1.0 : 0.0, j == 1 ? 1.0 : 0.0, j == 2 ? 1.0 : 0.0, j == 3 ? 1.0 : 0.0};
    RVE_TRY(run_curl(h, h->sd_Fp[sc][j], h->s_dnye));
    RVE_CUDA(h, launch_hard_jvp(h, h->s_dnye, h->sd_rho[sc][j], h->s_dtauc, h->s_dell, th, h->stream));
    RVE_CUDA(h, launch_local_jvp(h, dt, 0, nullptr, h->sd_Fp[sc][j], h->s_dtauc, h->s_dell, h->sd_rho[sc][j],
                                 h->s_dP, nullptr, nullptr, nullptr, th, h->stream));
    RVE_TRY(run_project_stencil(h, h->s_dP, h->R, mask, nullptr));
    int it = 0;
    bool ok = false;
    if (h->opt.precision == 0 && h->opt.krylov != 1) RVE_TRY(cg_solve(h, mask, eta, &it, &ok));
    // an explicit tolerance is honoured as given; the default one is kept
    // above what FP64 BiCGStab can reach
    if (!ok) RVE_TRY(bicgstab_solve(h, mask, h->sens_tol > 0 ? eta : std::fmax(eta, 1e-12), &it, &ok));
    if (!ok) return fail(h, RVE_ENOCONV_CG, "the sensitivity solve did not converge");
    RVE_CUDA(h, launch_zero_means(h, h->x, 0x1FFu & ~kept_means(mask), h->stream));
    RVE_CUDA(h, launch_local_jvp(h, dt, 1, h->x, h->sd_Fp[sc][j], h->s_dtauc, h->s_dell, h->sd_rho[sc][j],
                                 nullptr, h->sd_Fp[sn][j], h->sd_rho[sn][j], h->s_mean + 9 * j, th, h->stream));
  }
  RVE_CUDA(h, cudaMemcpyAsync(h->sens_dP, h->s_mean, sizeof(h->sens_dP), cudaMemcpyDeviceToHost, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  for (double v : h->sens_dP)
    if (!std::isfinite(v)) return fail(h, RVE_ENAN, "non-finite stress sensitivity");
  return RVE_OK;
}

// Launch-shape autotuner (rve_options.autotune): at create, on the handle's
// own buffers, time each candidate of three choices on its stream and keep
// the fastest -- the grid cap of the divergence stencil, the block count the
// FFT tile rules aim for, and (mixed precision) the staged or the plain
// tangent apply.  Device scalars are reset afterwards; the handle's state is
// as after an untuned create.
rve_status autotune(rve_s* h) {
  cudaStream_t st = h->stream;
  cudaEvent_t e0, e1;
  RVE_CUDA(h, cudaEventCreate(&e0));
  RVE_CUDA(h, cudaEventCreate(&e1));
  const bool f32 = h->opt.precision == 1;
  const uint8_t mask[9] = {1, 0, 0, 1, 0, 0, 1, 1, 0};
  if (f32) {
    RVE_CUDA(h, cudaMemsetAsync(h->t32, 0, 9 * h->nvox * sizeof(float), st));
    RVE_CUDA(h, cudaMemsetAsync(h->r32, 0, 9 * h->nvox * sizeof(float), st));
  }
  auto timed = [&](auto&& launch, float* ms) -> rve_status {
    for (int w = 0; w < 2; ++w) RVE_CUDA(h, launch());
    RVE_CUDA(h, cudaEventRecord(e0, st));
    for (int k = 0; k < 5; ++k) RVE_CUDA(h, launch());
    RVE_CUDA(h, cudaEventRecord(e1, st));
    RVE_CUDA(h, cudaEventSynchronize(e1));
    RVE_CUDA(h, cudaEventElapsedTime(ms, e0, e1));
    return RVE_OK;
  };
  const int sms = h->num_sms;
  // divergence grid cap
  {
    // multiples of the SM count, and grids that split the tiles evenly
    const int nt = stencil_tiles(h);
    const int cand[9] = {2 * sms, 3 * sms, 4 * sms, 6 * sms, 8 * sms, nt / 8, nt / 4, nt / 2, nt};
    float best = 1e30f;
    int pick = h->div_blocks;
    for (int c : cand) {
      if (c < 1 || c > 4096) continue;
      h->div_blocks = c;
      float ms = 0.f;
      RVE_TRY(timed([&]() {
        return f32 ? launch_div32(h, h->t32, h->du32, kept_means(mask), st)
                   : launch_div(h, h->F, h->q, 0, kept_means(mask), st);
      }, &ms));
      if (ms < best) { best = ms; pick = c; }
    }
    h->div_blocks = pick;
  }
  // FFT tile fill targets of the x, y and z passes, one at a time with the
  // others held (forward, Laplace solve, inverse of three fields)
  for (int* target : {&h->fft_fill, &h->fft_fill_y, &h->fft_fill_z}) {
    SpecParams sp = project_params(h, mask, nullptr, nullptr);
    sp.op = OP_LAPINV;
    const int cand[4] = {2 * sms, 4 * sms, 8 * sms, 16 * sms};
    float best = 1e30f;
    int pick = *target;
    for (int c : cand) {
      *target = c;
      float ms = 0.f;
      RVE_TRY(timed([&]() -> cudaError_t {
        if (f32) {
          if (cudaError_t e = launch_fft_forward32(h, h->du32, st, nullptr)) return e;
          if (cudaError_t e = launch_fft_lapinv32(h, sp, st, nullptr)) return e;
          return launch_fft_inverse32(h, h->du32 + 3 * h->nvox, st, nullptr);
        }
        if (cudaError_t e = launch_fft_forward(h, h->q, st, nullptr, 3)) return e;
        if (cudaError_t e = launch_fft_op(h, sp, st, nullptr, 3)) return e;
        return launch_fft_inverse(h, h->q + 3 * h->nvox, st, nullptr, 3);
      }, &ms));
      if (ms < best) { best = ms; pick = c; }
    }
    *target = pick;
  }
  // staged or plain FP32 tangent apply (the tangent buffer's contents do not matter)
  if (f32 && h->tma_apply) {
    float ms[2] = {0.f, 0.f};
    for (int v = 0; v < 2; ++v) {
      h->tma_apply = v == 1;
      RVE_TRY(timed([&]() { return launch_tangent_apply32(h, st); }, &ms[v]));
    }
    h->tma_apply = ms[1] <= ms[0];
  }
  RVE_CUDA(h, cudaMemsetAsync(h->dscal, 0, 64 * sizeof(double), st));
  RVE_CUDA(h, cudaMemsetAsync(h->dcount, 0, 16 * sizeof(int32_t), st));
  RVE_CUDA(h, cudaStreamSynchronize(st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->prof.reset();
  h->autotuned = true;
  return RVE_OK;
}

// The tangent of the evaluation that ended the last increment, built on
// request (rve_step skips it): same F, S, frozen hardening and step.
rve_status build_stale_tangent(rve_s* h) {
  if (!h->K_stale) return RVE_OK;
  RVE_CUDA(h, launch_tangent(h, h->dt_prev, 0.0, h->cur, h->stream));
  h->K_stale = false;
  return RVE_OK;
}

rve_status fail(rve_s* h, rve_status s, const char* msg) {
  h->err = msg;
  return s;
}

int ncomp_of(uint32_t which) {
  switch (which) {
    case RVE_FIELD_F: case RVE_FIELD_P: case RVE_FIELD_FP: case RVE_FIELD_SIGMA: case RVE_FIELD_NYE:
    case RVE_FIELD_P_EVAL: return 9;
    case RVE_FIELD_S: case RVE_FIELD_S_EVAL: return 6;
    case RVE_FIELD_RHO_SSD: case RVE_FIELD_RHO_GND: case RVE_FIELD_TAUC: case RVE_FIELD_DGAM: return 12;
    case RVE_FIELD_RHO_GND18: return 18;
    case RVE_FIELD_VM: case RVE_FIELD_GRAIN: return 1;
    case RVE_FIELD_TANGENT: return 81;
    default: return 0;
  }
}

}  // namespace

cudaEvent_t Prof::take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::begin(int cat, cudaStream_t s, cudaEvent_t* a) {
  if (cap) {
    ++cap->launches[cat];
    if (!on || cap->spare.size() < 2) return;
    *a = cap->spare.back();
    cap->spare.pop_back();
    cudaEventRecordWithFlags(*a, s, cudaEventRecordExternal);
    return;
  }
  ++launches[cat];
  if (!on) return;
  *a = take();
  if (*a) cudaEventRecord(*a, s);
}

void Prof::end(int cat, cudaStream_t s, cudaEvent_t a) {
  if (!on || !a) return;
  if (cap) {
    cudaEvent_t b = cap->spare.back();
    cap->spare.pop_back();
    cudaEventRecordWithFlags(b, s, cudaEventRecordExternal);
    cap->events.push_back({cat, a, b});
    return;
  }
  cudaEvent_t b = take();
  if (!b) { pool.push_back(a); return; }
  cudaEventRecord(b, s);
  pending.push_back({cat, a, b});
}

void Prof::resolve() {
  for (auto& p : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.cat] += t;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  for (auto& p : borrowed) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.cat] += t;
  }
  borrowed.clear();
}

void Prof::reset() {
  resolve();
  for (int k = 0; k < RVE_K_COUNT; ++k) { launches[k] = 0; ms[k] = 0.0; }
}

void Prof::destroy() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

extern "C" {

size_t rve_workspace_bytes(int n0, int n1, int n2, int n_grains, int precision) {
  if ((precision != 0 && precision != 1) || n_grains < 1) return 0;
  if (!good_len(n0, 2) || !good_len(n1, 2) || !good_len(n2, 1) || (n0 & 1) || (n1 & 1)) return 0;
  rve_s h;
  h.n0 = n0; h.n1 = n1; h.n2 = n2; h.nkx = n0 / 2 + 1;
  h.nvox = (size_t)n0 * n1 * n2;
  h.nspec = (size_t)h.nkx * n1 * n2;
  h.ngrains = n_grains;
  h.opt.precision = precision;
  Carver c{nullptr};
  carve(&h, c);
  return c.off;
}

rve_status rve_create(const int32_t* grain_id, int n0, int n1, int n2, const double* quat, int n_grains,
                      const rve_material* mat, const rve_options* opt, void* d_workspace, size_t ws_bytes,
                      void* cuda_stream, rve_t** out) {
  if (!out) return RVE_EINVAL;
  *out = nullptr;
  if (!grain_id || !quat || !mat || !opt || !d_workspace) return RVE_EINVAL;
  const size_t need = rve_workspace_bytes(n0, n1, n2, n_grains, opt->precision);
  if (need == 0) return RVE_EINVAL;
  if (ws_bytes < need) return RVE_ENOMEM;
  if (reinterpret_cast<uintptr_t>(d_workspace) & 255) return RVE_EINVAL;
  if (!(mat->C11 > 0 && mat->C44 > 0 && mat->C11 > mat->C12 && mat->b > 0 && mat->gdot0 > 0 && mat->n >= 1 &&
        mat->K > 0 && mat->yc >= 0 && mat->rho0_total > 0 && mat->tau0 >= 0 && mat->alpha >= 0 &&
        mat->q[0] > 0 && opt->L > 0 && opt->newton_tol > 0 && opt->cg_tol > 0 && opt->local_tol > 0 &&
        opt->max_newton > 0 && opt->max_cg > 0 && opt->max_local > 0 && opt->max_halvings >= 0 &&
        opt->krylov >= 0 && opt->krylov <= 2 && (opt->stencils == 0 || opt->stencils == 1) &&
        opt->continuation >= 0 && opt->continuation <= 6))
    return RVE_EINVAL;
  const size_t nvox = (size_t)n0 * n1 * n2;
  for (size_t v = 0; v < nvox; ++v)
    if (grain_id[v] < 0 || grain_id[v] >= n_grains) return RVE_EINVAL;
  for (int g = 0; g < n_grains; ++g) {
    const double* qq = quat + 4 * g;
    const double nn = qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3];
    if (!(nn > 0) || !std::isfinite(nn)) return RVE_EINVAL;
  }

  rve_s* h = new (std::nothrow) rve_s();
  if (!h) return RVE_ENOMEM;
  h->n0 = n0; h->n1 = n1; h->n2 = n2; h->nkx = n0 / 2 + 1;
  h->nvox = nvox;
  h->nspec = (size_t)h->nkx * n1 * n2;
  h->ngrains = n_grains;
  h->mat = *mat;
  h->opt = *opt;
  h->stream = (cudaStream_t)cuda_stream;
  h->device = 0;
  cudaGetDevice(&h->device);
  if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || h->num_sms < 1)
    h->num_sms = 152;
  h->div_blocks = 4 * h->num_sms;
  h->fft_fill = 8 * h->num_sms;     // x passes: radix-8 rows leave 8 threads per row, so more, smaller tiles
  h->fft_fill_y = 8 * h->num_sms;   // the y passes run faster with smaller tiles (measured at 64^3)
  h->fft_fill_z = 4 * h->num_sms;
  h->tma_apply = opt->tma != 0 && opt->precision == 1 && vec_init() == cudaSuccess;
  h->row_stencils = opt->stencils == 0;
  h->h = opt->L / n0;
  h->mu = mat->mu > 0 ? mat->mu : 3.0 * mat->C44 * (mat->C11 - mat->C12) / (4.0 * mat->C44 + mat->C11 - mat->C12);
  h->cur = 0;
  h->increment = 0;
  h->dt_prev = 1.0;
  for (int c = 0; c < 9; ++c) { h->dFbar_prev[c] = 0.0; h->Pmacro[c] = 0.0; h->Smacro[c] = 0.0; }
  make_plan(n0, &h->plan[0]);
  make_plan(n1, &h->plan[1]);
  make_plan(n2, &h->plan[2], 4);
  Consts& c = h->cst;
  c.C11 = mat->C11; c.C12 = mat->C12; c.C44 = mat->C44; c.mu = h->mu; c.b = mat->b;
  c.tau0 = mat->tau0; c.alpha = mat->alpha; c.gdot0 = mat->gdot0; c.n = mat->n; c.K = mat->K; c.yc = mat->yc;
  c.n_int = (mat->n == std::floor(mat->n) && mat->n >= 1 && mat->n <= 64) ? (int)mat->n : 0;
  c.gnd_enabled = mat->gnd_enabled ? 1 : 0;
  c.local_tol_abs = opt->local_tol * h->mu;
  c.floor_abs = 10.0 * c.local_tol_abs;
  c.dgam_max = 0.1;
  c.max_local = opt->max_local;
  c.max_halvings = 40;

  Carver cv{static_cast<char*>(d_workspace)};
  carve(h, cv);
  if (cudaMallocHost((void**)&h->hscal, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&h->hcount, 16 * sizeof(int32_t)) != cudaSuccess) {
    delete h;
    return RVE_ECUDA;
  }
  auto bad = [&](cudaError_t e) {
    if (e == cudaSuccess) return false;
    h->err = cudaGetErrorString(e);
    return true;
  };
  // tables
  std::vector<double> R(9 * (size_t)n_grains), q, Ap;
  std::vector<int32_t> screw;
  for (int g = 0; g < n_grains; ++g) quat_to_R(quat + 4 * g, &R[9 * g]);
  build_tables(*mat, q, Ap, screw);
  const int ns[3] = {n0, n1, n2};
  std::vector<double2> tw[3], ph[3];
  std::vector<double> tn[3], s2[3], c2[3], xi[3];
  std::vector<int8_t> nq[3];
  const double PI = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) {
    const int n = ns[a];
    tw[a].resize(n); ph[a].resize(n); tn[a].resize(n); nq[a].resize(n); s2[a].resize(n); c2[a].resize(n);
    xi[a].resize(n);
    for (int t = 0; t < n; ++t) {
      const double ang = 2.0 * PI * (double)t / n;
      tw[a][t] = make_double2(std::cos(ang), -std::sin(ang));
      const bool nyq = (2 * t == n);
      const int ks = (2 * t <= n) ? t : t - n;
      nq[a][t] = nyq ? 1 : 0;
      tn[a][t] = nyq ? 0.0 : std::tan(PI * (double)ks / n);
      ph[a][t] = nyq ? make_double2(-1.0, 0.0) : make_double2(std::cos(ang), std::sin(ang));
      const double sh = std::sin(PI * (double)t / n), chf = std::cos(PI * (double)t / n);
      s2[a][t] = nyq ? 1.0 : (t == 0 ? 0.0 : sh * sh);     // sin^2(xi/2), xi = 2 pi t / n
      c2[a][t] = nyq ? 0.0 : (t == 0 ? 1.0 : chf * chf);   // cos^2(xi/2)
      xi[a][t] = nyq ? 0.0 : 2.0 * PI * (double)ks / n;     // standard frequency
    }
    // exact values at the quarter points
    for (int t = 0; t < n; ++t) {
      if (4 * t == n) { tw[a][t] = make_double2(0.0, -1.0); ph[a][t] = make_double2(0.0, 1.0); }
      if (4 * t == 3 * n) { tw[a][t] = make_double2(0.0, 1.0); ph[a][t] = make_double2(0.0, -1.0); }
      if (2 * t == n) tw[a][t] = make_double2(-1.0, 0.0);
    }
    tw[a][0] = make_double2(1.0, 0.0);
    ph[a][0] = make_double2(1.0, 0.0);
  }
  cudaStream_t s = h->stream;
  bool fail_ = bad(cudaMemcpyAsync(h->grain, grain_id, nvox * sizeof(int32_t), cudaMemcpyHostToDevice, s)) ||
               bad(cudaMemcpyAsync(h->grainR, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, s)) ||
               bad(cudaMemcpyAsync(h->qhat, q.data(), 144 * sizeof(double), cudaMemcpyHostToDevice, s)) ||
               bad(cudaMemcpyAsync(h->Apinv, Ap.data(), 162 * sizeof(double), cudaMemcpyHostToDevice, s)) ||
               bad(cudaMemcpyAsync(h->screw_of, screw.data(), 12 * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  for (int a = 0; a < 3 && !fail_; ++a) {
    fail_ = bad(cudaMemcpyAsync((void*)h->ax[a].tw, tw[a].data(), ns[a] * sizeof(double2), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].tanh_, tn[a].data(), ns[a] * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].nyq, nq[a].data(), ns[a] * sizeof(int8_t), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].ph, ph[a].data(), ns[a] * sizeof(double2), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].s2, s2[a].data(), ns[a] * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].c2, c2[a].data(), ns[a] * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync((void*)h->ax[a].xi, xi[a].data(), ns[a] * sizeof(double), cudaMemcpyHostToDevice, s));
    if (!fail_ && h->opt.precision == 1) {
      std::vector<float2> t32(ns[a]);
      for (int t = 0; t < ns[a]; ++t) t32[t] = make_float2((float)tw[a][t].x, (float)tw[a][t].y);
      fail_ = bad(cudaMemcpyAsync((void*)h->ax[a].tw32, t32.data(), ns[a] * sizeof(float2), cudaMemcpyHostToDevice, s)) ||
              bad(cudaStreamSynchronize(s));
    }
  }
  // initial state: F = Fp = I, S = 0, rho_SSD = rho0 / 12, dF_last = 0
  if (!fail_) {
    std::vector<double> ident(9 * nvox, 0.0), rho(12 * nvox, mat->rho0_total / 12.0);
    for (int k = 0; k < 9; k += 4)
      for (size_t v = 0; v < nvox; ++v) ident[k * nvox + v] = 1.0;
    fail_ = bad(cudaMemcpyAsync(h->F_c, ident.data(), 9 * nvox * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync(h->Fp, ident.data(), 9 * nvox * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync(h->F, ident.data(), 9 * nvox * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemcpyAsync(h->rho_ssd, rho.data(), 12 * nvox * sizeof(double), cudaMemcpyHostToDevice, s)) ||
            bad(cudaMemsetAsync(h->S_c, 0, 6 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->S[0], 0, 6 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->S[1], 0, 6 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->P_c, 0, 9 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->P[0], 0, 9 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->dF_last, 0, 9 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->nye, 0, 9 * nvox * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->dscal, 0, 64 * sizeof(double), s)) ||
            bad(cudaMemsetAsync(h->dcount, 0, 16 * sizeof(int32_t), s)) ||
            bad(launch_lapinv_table(h, s)) ||
            bad(cudaStreamSynchronize(s));
  }
  if (!fail_ && opt->autotune) fail_ = autotune(h) != RVE_OK;
  if (fail_) {
    cudaFreeHost(h->hscal);
    cudaFreeHost(h->hcount);
    delete h;
    return RVE_ECUDA;
  }
  *out = h;
  return RVE_OK;
}

// Newton-Raphson on the equilibrium G*(P(F) - Pbar) = 0 of one increment
// (Sec. 2.2, Eq. linequil2ast) from the iterate in h->F, with the hardening
// of the increment frozen.  The first local evaluation is warm-started from
// S[warm] (the committed S when warm < 0).  On RVE_OK h->cur holds the
// converged evaluation.  Iteration counts accumulate into loc.
static rve_status newton_solve(rve_s* h, double dt, const uint8_t* mask, const double* Pb, int warm,
                               rve_step_info& loc, int max_iters) {
  int cur = warm < 0 ? 0 : 1 - warm;
  double rabs, scale;
  int lmax, lfail;
  h->cur = cur;
  rve_status st = eval_residual(h, dt, 0.0, cur, warm, mask, Pb, &rabs, &scale, &lmax, &lfail);
  if (st != RVE_OK) return st;
  loc.local_max_iters = std::max(loc.local_max_iters, lmax);
  loc.local_failures = lfail;
  double res = rabs / scale;
  if (loc.newton_iters <= RVE_MAX_NEWTON_LOG) loc.residuals[loc.newton_iters] = res;
  int it = 0;
  for (;;) {
    loc.residual = res;
    // a non-finite value anywhere in the state or the load path poisons the
    // residual; it is reported as such even though the local update at the
    // voxels concerned also fails
    if (!std::isfinite(res)) return (fail(h, RVE_ENAN, "non-finite residual"));
    if (lfail) return (fail(h, RVE_ENOCONV_LOCAL, "local update did not converge"));
    if (res <= h->opt.newton_tol) break;
    if (it >= max_iters) return fail(h, RVE_ENOCONV_NEWTON, "Newton-Raphson reached its iteration limit");
    // the tangent is built only at iterates that get a Krylov solve: not at
    // rejected line-search trials, not at the iterate that ends the increment
    if (cudaError_t e = launch_tangent(h, dt, 0.0, cur, h->stream)) {
      h->err = cudaGetErrorString(e);
      return RVE_ECUDA;
    }
    int ncg = 0;
    bool cgok = false;
    // inexact Newton: with cg_adaptive the linear solve only needs to be as
    // accurate as the current residual (forcing term min(1e-2, res)); the
    // converged increment does not depend on it
    const double eta = h->opt.cg_adaptive ? std::fmax(h->opt.cg_tol, std::fmin(1e-2, res)) : h->opt.cg_tol;
    double lam = 1.0, rt = 0.0, sct = 0.0;
    int lm = 0, lf = 0;
    bool acc = false;
    // krylov 0: conjugate gradients (the paper's solver); when no step along
    // the CG direction lowers the residual, the iteration is solved again with
    // BiCGStab.  A CG solve cut off at max_cg still gives its direction a line
    // search first: the truncated iterate is a damped step (CG iterates grow in
    // norm from zero), which on an ill-conditioned tangent often does better
    // than a fully solved BiCGStab step.  1: BiCGStab only; 2: CG only.
    const int attempts = h->opt.krylov == 0 ? 2 : 1;
    for (int att = 0; att < attempts && !acc; ++att) {
      const bool use_bicg = h->opt.krylov == 1 || att == 1;
      if (use_bicg) {
        // trials of the rejected CG line search overwrote R: rebuild it from
        // the current iterate's stress (its tangent K[cur] is untouched)
        if (att == 1) RVE_TRY(run_project_stencil(h, h->P[cur], h->R, mask, Pb));
        st = bicgstab_solve(h, mask, h->opt.precision == 1 ? std::fmax(eta, 1e-10) : eta, &ncg, &cgok);
        ++loc.bicgstab_solves;
      } else {
        st = h->opt.precision == 1 ? cg_solve32(h, mask, eta, &ncg, &cgok) : cg_solve(h, mask, eta, &ncg, &cgok);
      }
      if (st != RVE_OK) return st;
      // dF has zero strain-controlled means by construction (every Krylov vector
      // is a projection); remove what round-off left there, which a long or
      // stalled solve with a large dF would otherwise carry into <F>
      RVE_CUDA(h, launch_zero_means(h, h->x, 0x1FFu & ~kept_means(mask), h->stream));
      if (loc.newton_iters < RVE_MAX_NEWTON_LOG) loc.cg_iters[loc.newton_iters] += ncg;
      loc.cg_iters_total += ncg;
      // backtracking on phi(lam) = rms(R(F + lam dF))^2 with sufficient decrease;
      // after a rejected trial the next lam minimises the quadratic through
      // phi(0), the Newton slope -2 phi(0) and phi(lam), kept in [0.1, 0.5] lam.
      // A trial at which some voxel's local update fails (the step asks for
      // slips above the local cap) is halved on a budget of its own: the
      // current iterate itself has a converged local state, so a small enough
      // step always passes.
      lam = 1.0;
      const double f0 = rabs * rabs;
      int shrink = 0, local_cuts = 0;
      while (shrink <= h->opt.max_halvings && local_cuts <= 40) {
        st = eval_residual(h, dt, lam, 1 - cur, cur, mask, Pb, &rt, &sct, &lm, &lf);
        if (st != RVE_OK) return st;
        if (lf == 0 && rt < rabs * (1.0 - 1e-4 * lam)) { acc = true; break; }
        double next = 0.5 * lam;
        if (lf == 0 && std::isfinite(rt)) {
          const double c = (rt * rt - f0 * (1.0 - 2.0 * lam)) / (lam * lam);
          if (c > 0.0) next = std::fmin(std::fmax(f0 / c, 0.1 * lam), 0.5 * lam);
          ++shrink;
        } else {
          ++local_cuts;
        }
        lam = next;
        ++loc.halvings;
      }
    }
    if (!acc) {
      if (lf) return (fail(h, RVE_ENOCONV_LOCAL, "local update did not converge in the line search"));
      if (!cgok) return (fail(h, RVE_ENOCONV_CG, "the Krylov solve did not converge"));
      return (fail(h, RVE_ENOCONV_NEWTON, "no step along the Newton direction lowers the residual"));
    }
    if (cudaError_t e = launch_axpy_F(h, lam, h->stream)) {
      h->err = cudaGetErrorString(e);
      return RVE_ECUDA;
    }
    cur = 1 - cur;
    h->cur = cur;
    rabs = rt;
    res = rt / sct;
    loc.local_max_iters = lm > loc.local_max_iters ? lm : loc.local_max_iters;
    ++loc.newton_iters;
    ++it;
    if (loc.newton_iters <= RVE_MAX_NEWTON_LOG) loc.residuals[loc.newton_iters] = res;
  }
  return RVE_OK;
}

// statuses after which the increment is tried again with the load in stages
static bool retryable(rve_status st) {
  return st == RVE_ENOCONV_NEWTON || st == RVE_ENOCONV_CG || st == RVE_ENOCONV_LOCAL;
}

rve_status rve_step(rve_t* h, const double dFbar[9], const uint8_t strain_mask[9], const double Pbar[9], double dt,
                    rve_step_info* info) {
  if (!h || !dFbar || !strain_mask || !Pbar || !(dt > 0) || !std::isfinite(dt)) return RVE_EINVAL;
  for (int c = 0; c < 9; ++c)
    if (!std::isfinite(dFbar[c]) || !std::isfinite(Pbar[c])) return fail(h, RVE_EINVAL, "non-finite load");
  const auto t0 = std::chrono::steady_clock::now();
  rve_step_info loc;
  std::memset(&loc, 0, sizeof(loc));
  uint8_t mask[9];
  double dFb[9], Pb[9];
  for (int c = 0; c < 9; ++c) {
    mask[c] = strain_mask[c] ? 1 : 0;
    dFb[c] = mask[c] ? dFbar[c] : 0.0;
    Pb[c] = mask[c] ? 0.0 : Pbar[c];
  }
  auto finish = [&](rve_status st) {
    const unsigned long long* tot = reinterpret_cast<const unsigned long long*>(h->hcount + 8);
    loc.local_iters_total = (int64_t)tot[0];
    loc.local_evals_total = (int64_t)tot[1];
    loc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = loc;
    return st;
  };
  RVE_CUDA(h, cudaMemsetAsync(h->dcount + 8, 0, 4 * sizeof(int32_t), h->stream));
  RVE_CUDA(h, cudaMemsetAsync(h->dscal + DS_ERR, 0, sizeof(double), h->stream));
  h->K_stale = false;
  rve_status st = run_hardening(h);
  if (st != RVE_OK) return finish(st);
  const int extrap = (h->opt.extrapolate && h->increment > 0) ? 1 : 0;
  const double ratio = dt / h->dt_prev;
  if (cudaError_t e = launch_predictor(h, dFb, h->dFbar_prev, ratio, extrap, h->stream)) {
    h->err = cudaGetErrorString(e);
    return finish(RVE_ECUDA);
  }
  // with continuation available, the direct solve gets a quarter of max_newton
  // (at least 8): an increment that needs more goes to the staged load at once
  const int direct_max = h->opt.continuation > 0 ? std::max(8, h->opt.max_newton / 4) : h->opt.max_newton;
  st = newton_solve(h, dt, mask, Pb, -1, loc, std::min(direct_max, h->opt.max_newton));
  loc.load_stages = 1;
  // Load continuation: when Newton fails on the increment (typically at the
  // plastic onset of a large, strongly non-linear RVE), the same increment is
  // solved again from its start with the macroscopic load applied in 2^k equal
  // stages (k = 1 .. continuation), each stage's solution the starting point
  // of the next.  The hardening stays frozen and the last stage solves the
  // increment's own equations, so the converged increment is the same; only
  // the path to it changes.
  for (int lev = 1; retryable(st) && lev <= h->opt.continuation; ++lev) {
    const int nst = 1 << lev;
    loc.load_stages = nst;
    st = RVE_OK;
    for (int k = 1; k <= nst && st == RVE_OK; ++k) {
      const double th = (double)k / nst;
      double dFs[9], Ps[9];
      for (int c = 0; c < 9; ++c) { dFs[c] = dFb[c] / nst; Ps[c] = th * Pb[c]; }
      cudaError_t e;
      if (k == 1) {
        double dF1[9];
        for (int c = 0; c < 9; ++c) dF1[c] = th * dFb[c];
        e = launch_predictor(h, dF1, h->dFbar_prev, th * ratio, extrap, h->stream);
      } else {
        e = launch_shift_F(h, dFs, h->stream);
      }
      if (e != cudaSuccess) {
        h->err = cudaGetErrorString(e);
        return finish(RVE_ECUDA);
      }
      st = newton_solve(h, dt, mask, Ps, k == 1 ? -1 : h->cur, loc, h->opt.max_newton);
    }
  }
  if (st != RVE_OK) return finish(st);
  if (h->sens_on) {
    h->sens_valid = 0;
    st = sens_update(h, mask, dt);
    if (st != RVE_OK) return finish(st);      // nothing committed
  }
  loc.converged = 1;
  if (cudaError_t e = launch_commit(h, h->stream)) {
    h->err = cudaGetErrorString(e);
    return finish(RVE_ECUDA);
  }
  if (cudaError_t e = launch_macro(h, h->stream)) {
    h->err = cudaGetErrorString(e);
    return finish(RVE_ECUDA);
  }
  st = read_scalars(h);
  if (st != RVE_OK) return finish(st);
  for (int c = 0; c < 9; ++c) {
    h->Pmacro[c] = h->hscal[DS_MEANP + c] / (double)h->nvox;
    h->Smacro[c] = h->hscal[DS_MEANSIG + c] / (double)h->nvox;
    h->dFbar_prev[c] = dFb[c];
  }
  h->dt_prev = dt;
  ++h->increment;
  h->K_stale = !h->sens_on;                   // sens_update built the converged tangent
  if (h->sens_on) {
    h->sens_cur = 1 - h->sens_cur;
    h->sens_valid = 1;
  }
  return finish(RVE_OK);
}

rve_status rve_step_batch(rve_t* const* hs, int n, const double* dFbar, const uint8_t* strain_mask,
                          const double* Pbar, const double* dt, rve_step_info* info, rve_status* status) {
  if (!hs || n <= 0 || !dFbar || !strain_mask || !Pbar || !dt) return RVE_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return RVE_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return RVE_EINVAL;
  }
  std::vector<rve_status> st(n, RVE_OK);
  auto run = [&](int i) {
    cudaSetDevice(hs[i]->device);
    st[i] = rve_step(hs[i], dFbar + 9 * i, strain_mask + 9 * i, Pbar + 9 * i, dt[i], info ? info + i : nullptr);
  };
  std::vector<std::thread> threads;
  int started = 0;
  try {
    threads.reserve(n);
    for (; started < n; ++started) threads.emplace_back(run, started);
  } catch (...) {
    // no more threads: the remaining handles run on this thread
  }
  for (int i = started; i < n; ++i) run(i);
  for (auto& t : threads) t.join();
  rve_status first = RVE_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = st[i];
    if (first == RVE_OK && st[i] != RVE_OK) first = st[i];
  }
  return first;
}

rve_status rve_get_macro_stress(rve_t* h, double P[9], double sigma[9]) {
  if (!h || !P || !sigma) return RVE_EINVAL;
  for (int c = 0; c < 9; ++c) { P[c] = h->Pmacro[c]; sigma[c] = h->Smacro[c]; }
  return RVE_OK;
}

rve_status rve_get_fields(rve_t* h, uint32_t which, void* dst, size_t bytes, int dst_is_device) {
  if (!h || !dst) return RVE_EINVAL;
  const int nc = ncomp_of(which);
  if (nc == 0) return fail(h, RVE_EINVAL, "unknown field selector");
  const size_t esz = which == RVE_FIELD_GRAIN ? sizeof(int32_t) : sizeof(double);
  const size_t need = (size_t)nc * h->nvox * esz;
  if (bytes < need) return fail(h, RVE_EINVAL, "destination too small");
  const void* src = nullptr;
  switch (which) {
    case RVE_FIELD_F: src = h->F_c; break;
    case RVE_FIELD_P: src = h->P_c; break;
    case RVE_FIELD_FP: src = h->Fp; break;
    case RVE_FIELD_RHO_SSD: src = h->rho_ssd; break;
    case RVE_FIELD_RHO_GND: src = h->rho_gnd; break;
    case RVE_FIELD_RHO_GND18: src = h->rho18; break;
    case RVE_FIELD_NYE: src = h->nye; break;
    case RVE_FIELD_TAUC: src = h->tauc; break;
    case RVE_FIELD_DGAM: src = h->dgam[h->cur]; break;
    case RVE_FIELD_TANGENT:
      RVE_TRY(build_stale_tangent(h));
      if (h->opt.precision == 1) {   // stored as float: widen into the other evaluation buffer
        double* tmp = h->K[1 - h->cur];
        RVE_CUDA(h, launch_widen(h, reinterpret_cast<const float*>(h->K[h->cur]), tmp, 81 * h->nvox, h->stream));
        src = tmp;
      } else {
        src = h->K[h->cur];
      }
      break;
    case RVE_FIELD_GRAIN: src = h->grain; break;
    case RVE_FIELD_P_EVAL: src = h->P[h->cur]; break;
    case RVE_FIELD_SIGMA:
      RVE_CUDA(h, launch_output_field(h, 0, h->P_c, h->S_c, h->q, h->stream));
      src = h->q; break;
    case RVE_FIELD_VM:
      RVE_CUDA(h, launch_output_field(h, 1, h->P_c, h->S_c, h->q, h->stream));
      src = h->q; break;
    case RVE_FIELD_S:
      RVE_CUDA(h, launch_output_field(h, 2, h->P_c, h->S_c, h->q, h->stream));
      src = h->q; break;
    case RVE_FIELD_S_EVAL:
      RVE_CUDA(h, launch_output_field(h, 2, h->P_c, h->S[h->cur], h->q, h->stream));
      src = h->q; break;
  }
  RVE_CUDA(h, cudaMemcpyAsync(dst, src, need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

rve_status rve_set_fields(rve_t* h, uint32_t which, const void* src, size_t bytes, int src_is_device) {
  if (!h || !src) return RVE_EINVAL;
  double* dst = nullptr;
  int nc = 0;
  switch (which) {
    case RVE_FIELD_F: dst = h->F_c; nc = 9; break;
    case RVE_FIELD_FP: dst = h->Fp; nc = 9; break;
    case RVE_FIELD_RHO_SSD: dst = h->rho_ssd; nc = 12; break;
    default: return fail(h, RVE_EINVAL, "field cannot be set");
  }
  if (bytes != (size_t)nc * h->nvox * sizeof(double)) return fail(h, RVE_EINVAL, "wrong byte count");
  RVE_CUDA(h, cudaMemcpyAsync(dst, src, bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

rve_status rve_eval_hardening(rve_t* h) {
  if (!h) return RVE_EINVAL;
  RVE_TRY(build_stale_tangent(h));   // before the frozen hardening state changes
  RVE_TRY(run_hardening(h));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

rve_status rve_eval_nye(rve_t* h, int scheme) {
  if (!h || (scheme != 0 && scheme != 1)) return RVE_EINVAL;
  if (scheme == 0) {
    RVE_TRY(run_curl(h, h->Fp, h->nye));
  } else {
    SpecParams sp = project_params(h, (const uint8_t*)"\0\0\0\0\0\0\0\0\0", nullptr, nullptr);
    sp.op = OP_CURL_STD;
    h->fft_cat = RVE_K_FFT_CURL;
    const rve_status st = run_project(h, h->Fp, h->nye, sp);
    h->fft_cat = -1;
    RVE_TRY(st);
  }
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

rve_status rve_eval_constitutive(rve_t* h, double dt, int32_t* local_max_iters, int32_t* local_failures) {
  if (!h || !(dt > 0)) return RVE_EINVAL;
  RVE_TRY(run_hardening(h));
  RVE_CUDA(h, cudaMemcpyAsync(h->F, h->F_c, 9 * h->nvox * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  RVE_CUDA(h, cudaMemsetAsync(h->dcount, 0, 2 * sizeof(int32_t), h->stream));
  RVE_CUDA(h, launch_constitutive(h, dt, 0.0, h->cur, -1, h->stream));
  h->K_stale = false;
  RVE_TRY(read_scalars(h));
  if (local_max_iters) *local_max_iters = h->hcount[0];
  if (local_failures) *local_failures = h->hcount[1];
  return RVE_OK;
}

rve_status rve_project(rve_t* h, const uint8_t strain_mask[9], const double* d_X, double* d_Y) {
  if (!h || !strain_mask || !d_X || !d_Y) return RVE_EINVAL;
  uint8_t mask[9];
  for (int c = 0; c < 9; ++c) mask[c] = strain_mask[c] ? 1 : 0;
  RVE_TRY(run_project_stencil(h, d_X, d_Y, mask, nullptr));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

struct CkptHeader {
  uint32_t magic, version;
  int32_t n0, n1, n2, ngrains, increment, cur;
  double dt_prev;
  double dFbar_prev[9], Pmacro[9], Smacro[9];
};

size_t rve_checkpoint_bytes(const rve_t* h) {
  if (!h) return 0;
  return sizeof(CkptHeader) + (size_t)(9 + 9 + 6 + 12 + 9 + 9) * h->nvox * sizeof(double);
}

rve_status rve_checkpoint(rve_t* h, void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < rve_checkpoint_bytes(h)) return RVE_EINVAL;
  CkptHeader hd;
  hd.magic = CKPT_MAGIC; hd.version = CKPT_VERSION;
  hd.n0 = h->n0; hd.n1 = h->n1; hd.n2 = h->n2; hd.ngrains = h->ngrains;
  hd.increment = h->increment; hd.cur = 0; hd.dt_prev = h->dt_prev;
  for (int c = 0; c < 9; ++c) { hd.dFbar_prev[c] = h->dFbar_prev[c]; hd.Pmacro[c] = h->Pmacro[c]; hd.Smacro[c] = h->Smacro[c]; }
  char* p = static_cast<char*>(host_buf);
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const double* bufs[6] = {h->F_c, h->Fp, h->S_c, h->rho_ssd, h->dF_last, h->P_c};
  const int nc[6] = {9, 9, 6, 12, 9, 9};
  for (int b = 0; b < 6; ++b) {
    const size_t n = (size_t)nc[b] * h->nvox * sizeof(double);
    RVE_CUDA(h, cudaMemcpyAsync(p, bufs[b], n, cudaMemcpyDeviceToHost, h->stream));
    p += n;
  }
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  return RVE_OK;
}

rve_status rve_restore(rve_t* h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < rve_checkpoint_bytes(h)) return RVE_EINVAL;
  CkptHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (hd.magic != CKPT_MAGIC || hd.version != CKPT_VERSION || hd.n0 != h->n0 || hd.n1 != h->n1 || hd.n2 != h->n2 ||
      hd.ngrains != h->ngrains || !(hd.dt_prev > 0) || hd.increment < 0)
    return fail(h, RVE_EINVAL, "checkpoint does not match this handle");
  const char* p = static_cast<const char*>(host_buf) + sizeof(hd);
  double* bufs[6] = {h->F_c, h->Fp, h->S_c, h->rho_ssd, h->dF_last, h->P_c};
  const int nc[6] = {9, 9, 6, 12, 9, 9};
  for (int b = 0; b < 6; ++b) {
    const size_t n = (size_t)nc[b] * h->nvox * sizeof(double);
    RVE_CUDA(h, cudaMemcpyAsync(bufs[b], p, n, cudaMemcpyHostToDevice, h->stream));
    p += n;
  }
  RVE_CUDA(h, cudaMemcpyAsync(h->S[0], h->S_c, 6 * h->nvox * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  RVE_CUDA(h, cudaMemcpyAsync(h->P[0], h->P_c, 9 * h->nvox * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->cur = 0;
  h->K_stale = false;
  if (h->sens_on) {                           // the restored state is taken as parameter-independent
    for (int j = 0; j < RVE_NTHETA; ++j) {
      RVE_CUDA(h, cudaMemsetAsync(h->sd_Fp[h->sens_cur][j], 0, 9 * h->nvox * sizeof(double), h->stream));
      RVE_CUDA(h, cudaMemsetAsync(h->sd_rho[h->sens_cur][j], 0, 12 * h->nvox * sizeof(double), h->stream));
    }
    RVE_CUDA(h, cudaStreamSynchronize(h->stream));
    h->sens_valid = 0;
  }
  h->increment = hd.increment;
  h->dt_prev = hd.dt_prev;
  for (int c = 0; c < 9; ++c) { h->dFbar_prev[c] = hd.dFbar_prev[c]; h->Pmacro[c] = hd.Pmacro[c]; h->Smacro[c] = hd.Smacro[c]; }
  return RVE_OK;
}

size_t rve_sensitivity_bytes(const rve_t* h) {
  if (!h) return 0;
  return (2 * RVE_NTHETA * (9 + 12) + 9 + 12 + 12 + 9) * align256(h->nvox * sizeof(double)) + 256 +
         align256(RVE_NTHETA * 9 * sizeof(double));
}

rve_status rve_sensitivity_enable(rve_t* h, void* d_workspace, size_t bytes, double tol) {
  if (!h || !d_workspace || bytes < rve_sensitivity_bytes(h) || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
    return RVE_EINVAL;
  Carver c{static_cast<char*>(d_workspace)};
  const size_t nv = h->nvox;
  for (int b = 0; b < 2; ++b)
    for (int j = 0; j < RVE_NTHETA; ++j) {
      h->sd_Fp[b][j] = c.take<double>(9 * nv);
      h->sd_rho[b][j] = c.take<double>(12 * nv);
    }
  h->s_dnye = c.take<double>(9 * nv);
  h->s_dtauc = c.take<double>(12 * nv);
  h->s_dell = c.take<double>(12 * nv);
  h->s_dP = c.take<double>(9 * nv);
  h->s_mean = c.take<double>(RVE_NTHETA * 9);
  if (c.off > bytes) return fail(h, RVE_EINVAL, "sensitivity workspace too small");
  RVE_CUDA(h, cudaMemsetAsync(d_workspace, 0, c.off, h->stream));
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->sens_on = true;
  h->sens_cur = 0;
  h->sens_tol = tol;
  h->sens_valid = 0;
  return RVE_OK;
}

rve_status rve_get_stress_sensitivity(rve_t* h, double dP[RVE_NTHETA * 9]) {
  if (!h || !dP) return RVE_EINVAL;
  if (!h->sens_on || !h->sens_valid) return fail(h, RVE_EINVAL, "no sensitivity of a converged increment");
  for (int k = 0; k < RVE_NTHETA * 9; ++k) dP[k] = h->sens_dP[k];
  return RVE_OK;
}

rve_status rve_time_fft(rve_t* h, int nf, int fp32, int reps, double* ms) {
  if (!h || !ms || reps < 1 || !(nf == 3 || nf == 9) || (fp32 && (nf != 3 || h->opt.precision != 1)))
    return RVE_EINVAL;
  const uint8_t mask[9] = {1, 0, 0, 1, 0, 0, 1, 1, 0};
  SpecParams sp = project_params(h, mask, nullptr, nullptr);
  sp.op = nf == 3 ? OP_LAPINV : OP_PROJECT;
  cudaStream_t s = h->stream;
  auto pair = [&]() -> cudaError_t {
    cudaError_t e;
    if (fp32) {
      if ((e = launch_fft_forward32(h, h->t32, s, nullptr)) != cudaSuccess) return e;
      if ((e = launch_fft_lapinv32(h, sp, s, nullptr)) != cudaSuccess) return e;
      return launch_fft_inverse32(h, h->x32, s, nullptr);
    }
    if ((e = launch_fft_forward(h, h->R, s, nullptr, nf)) != cudaSuccess) return e;
    if ((e = launch_fft_op(h, sp, s, nullptr, nf)) != cudaSuccess) return e;
    return launch_fft_inverse(h, h->t, s, nullptr, nf);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RVE_CUDA(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fail(h, RVE_ECUDA, "cudaEventCreate"); }
  cudaError_t err = pair();                       // warm-up
  if (err == cudaSuccess) err = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) err = pair();
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RVE_CUDA(h, err);
  *ms = (double)t / reps;
  return RVE_OK;
}

rve_status rve_set_wait_limit(rve_t* h, uint32_t polls) {
  if (!h) return RVE_EINVAL;
  h->wait_polls = polls;
  // captured CG chunks carry the old limit as a kernel argument
  for (auto& g : h->graphs) release_graph(g);
  return RVE_OK;
}

rve_status rve_get_tuning(rve_t* h, int32_t out[6]) {
  if (!h || !out) return RVE_EINVAL;
  out[0] = h->div_blocks;
  out[1] = h->fft_fill;
  out[4] = h->fft_fill_y;
  out[5] = h->fft_fill_z;
  out[2] = h->tma_apply ? 1 : 0;
  out[3] = h->autotuned ? 1 : 0;
  return RVE_OK;
}

rve_status rve_profile(rve_t* h, int enable) {
  if (!h) return RVE_EINVAL;
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->prof.reset();
  h->prof.on = enable != 0;
  return RVE_OK;
}

rve_status rve_kernel_stats(rve_t* h, int64_t* launches, double* ms) {
  if (!h) return RVE_EINVAL;
  RVE_CUDA(h, cudaStreamSynchronize(h->stream));
  h->prof.resolve();
  for (int k = 0; k < RVE_K_COUNT; ++k) {
    if (launches) launches[k] = h->prof.launches[k];
    if (ms) ms[k] = h->prof.ms[k];
  }
  return RVE_OK;
}

const char* rve_last_error(const rve_t* h) { return h ? h->err.c_str() : "null handle"; }

void rve_destroy(rve_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs) release_graph(g);
  h->prof.destroy();
  cudaFreeHost(h->hscal);
  cudaFreeHost(h->hcount);
  delete h;
}

}  // extern "C"
