// Galerkin projection Y = G*(X) for callers that cannot allocate device
// memory.  The spectrum scratch and the per-axis frequency tables live in one
// file-scope static device array instead of a caller-provided workspace; the
// FFT and projection kernels are the same ones the handle-based path runs.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "rve_internal.h"

namespace {

constexpr size_t SPEC_MAX_BYTES = RVE_NOALLOC_SPEC_BYTES;
constexpr int AXIS_MAX = 512;
constexpr size_t AXIS_BYTES = AXIS_MAX * (sizeof(double2) + sizeof(double) + sizeof(int8_t) + sizeof(double2));
constexpr size_t TABLE_BYTES = 3 * ((AXIS_BYTES + 255) & ~(size_t)255);

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPEC_MAX_BYTES + TABLE_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the static scratch for the current device.  Looked up
// once per device (with that device current): in host code the symbol's name
// is only a host-side stand-in, not a device address.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool supported(int n, int lo) {
  if (n < lo || n > AXIS_MAX) return false;
  FFTPlan p;
  make_plan(n, &p);
  return p.npass >= 0;
}

}  // namespace

extern "C" rve_status rve_project_noalloc(int n0, int n1, int n2, double L, const uint8_t strain_mask[9],
                                          const double* d_X, double* d_Y, void* cuda_stream) {
  if (!strain_mask || !d_X || !d_Y || !(L > 0)) return RVE_EINVAL;
  if (!supported(n0, 2) || !supported(n1, 2) || !supported(n2, 1) || (n0 & 1) || (n1 & 1)) return RVE_EINVAL;
  rve_s h;
  h.n0 = n0; h.n1 = n1; h.n2 = n2; h.nkx = n0 / 2 + 1;
  h.nvox = (size_t)n0 * n1 * n2;
  h.nspec = (size_t)h.nkx * n1 * n2;
  if (9 * h.nspec * sizeof(double2) > SPEC_MAX_BYTES) return RVE_ENOMEM;
  h.h = L / n0;
  h.stream = (cudaStream_t)cuda_stream;
  make_plan(n0, &h.plan[0]);
  make_plan(n1, &h.plan[1]);
  make_plan(n2, &h.plan[2]);

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return RVE_ECUDA;
  char* tab = static_cast<char*>(base) + SPEC_MAX_BYTES;
  h.spec = reinterpret_cast<double2*>(base);

  // frequency tables of the three axes, built on the host into fixed arrays
  const int ns[3] = {n0, n1, n2};
  const double PI = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) {
    const int n = ns[a];
    double2 tw[AXIS_MAX], ph[AXIS_MAX];
    double tn[AXIS_MAX];
    int8_t nq[AXIS_MAX];
    for (int t = 0; t < n; ++t) {
      const double ang = 2.0 * PI * (double)t / n;
      const bool nyq = (2 * t == n);
      const int ks = (2 * t <= n) ? t : t - n;
      tw[t] = make_double2(std::cos(ang), -std::sin(ang));
      nq[t] = nyq ? 1 : 0;
      tn[t] = nyq ? 0.0 : std::tan(PI * (double)ks / n);
      ph[t] = nyq ? make_double2(-1.0, 0.0) : make_double2(std::cos(ang), std::sin(ang));
      if (4 * t == n) { tw[t] = make_double2(0.0, -1.0); ph[t] = make_double2(0.0, 1.0); }
      if (4 * t == 3 * n) { tw[t] = make_double2(0.0, 1.0); ph[t] = make_double2(0.0, -1.0); }
      if (nyq) tw[t] = make_double2(-1.0, 0.0);
    }
    tw[0] = make_double2(1.0, 0.0);
    ph[0] = make_double2(1.0, 0.0);
    char* ax = tab + a * ((AXIS_BYTES + 255) & ~(size_t)255);
    double2* dtw = reinterpret_cast<double2*>(ax);
    double2* dph = dtw + AXIS_MAX;
    double* dtn = reinterpret_cast<double*>(dph + AXIS_MAX);
    int8_t* dnq = reinterpret_cast<int8_t*>(dtn + AXIS_MAX);
    // pageable sources: each copy is staged before the call returns
    if (cudaMemcpyAsync(dtw, tw, n * sizeof(double2), cudaMemcpyHostToDevice, h.stream) != cudaSuccess ||
        cudaMemcpyAsync(dph, ph, n * sizeof(double2), cudaMemcpyHostToDevice, h.stream) != cudaSuccess ||
        cudaMemcpyAsync(dtn, tn, n * sizeof(double), cudaMemcpyHostToDevice, h.stream) != cudaSuccess ||
        cudaMemcpyAsync(dnq, nq, n * sizeof(int8_t), cudaMemcpyHostToDevice, h.stream) != cudaSuccess)
      return RVE_ECUDA;
    h.ax[a].tw = dtw;
    h.ax[a].ph = dph;
    h.ax[a].tanh_ = dtn;
    h.ax[a].nyq = dnq;
  }

  SpecParams sp;
  sp.op = OP_PROJECT;
  for (int c = 0; c < 9; ++c) {
    sp.keep[c] = strain_mask[c] ? 0 : 1;
    sp.shift[c] = 0.0;
  }
  sp.inv_nvox = 1.0 / (double)h.nvox;
  sp.inv4h = 0.25 / h.h;
  sp.mean_out = nullptr;
  if (launch_fft_forward(&h, d_X, h.stream) != cudaSuccess) return RVE_ECUDA;
  if (launch_fft_op(&h, sp, h.stream) != cudaSuccess) return RVE_ECUDA;
  if (launch_fft_inverse(&h, d_Y, h.stream) != cudaSuccess) return RVE_ECUDA;
  return RVE_OK;
}
