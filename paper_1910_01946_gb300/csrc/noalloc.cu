// Galerkin projection Y = G*(X) for callers that cannot allocate device
// memory.  The spectrum scratch and the per-axis frequency tables live in one
// file-scope static device array instead of a caller-provided workspace.  It
// computes the same linear map as the handle path's rve_project, but in the
// nine-field Fourier form (forward FFT of all nine fields, the projection at
// every frequency, inverse FFT) rather than the stencil-factored form; the
// two agree to round-off.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "rve_internal.h"

namespace {

constexpr size_t SPEC_MAX_BYTES = RVE_NOALLOC_SPEC_BYTES;
constexpr int AXIS_MAX = 512;
constexpr size_t AXIS_BYTES = AXIS_MAX * (sizeof(double2) + sizeof(double2) + sizeof(double) + sizeof(int8_t));
constexpr size_t AXIS_PITCH = (AXIS_BYTES + 255) & ~(size_t)255;
constexpr size_t TABLE_BYTES = 3 * AXIS_PITCH;

// Held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SPEC_MAX_BYTES + TABLE_BYTES];

// Per device: the scratch's device address (looked up once, with that device
// current: in host code the symbol's name is only a host-side stand-in, not a
// device address) and the grid whose frequency tables the scratch holds.
constexpr int MAX_DEVICES = 64;
struct DeviceSlot {
  void* addr = nullptr;
  int n[3] = {0, 0, 0};
};
std::mutex g_mutex;
DeviceSlot g_slot[MAX_DEVICES];

// Frequency tables of one axis of length n in the layout the FFT kernels read
// (twiddles e^{-2 pi i t / n}; phases e^{i xi_t}, exactly -1 at Nyquist;
// tan(pi k / n) for the signed index k, 0 at Nyquist; Nyquist flags), built
// on the device, so no call copies anything from the host.  sincospi gives
// the quarter-turn values exactly.
__global__ void k_axis_tables(unsigned char* tab, int n0, int n1, int n2) {
  const int a = blockIdx.y;
  const int n = a == 0 ? n0 : (a == 1 ? n1 : n2);
  unsigned char* ax = tab + a * AXIS_PITCH;
  double2* tw = reinterpret_cast<double2*>(ax);
  double2* ph = tw + AXIS_MAX;
  double* tn = reinterpret_cast<double*>(ph + AXIS_MAX);
  int8_t* nq = reinterpret_cast<int8_t*>(tn + AXIS_MAX);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const bool nyq = 2 * t == n;
    const int ks = (2 * t <= n) ? t : t - n;
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    tw[t] = nyq ? make_double2(-1.0, 0.0) : make_double2(c, -s);
    ph[t] = nyq ? make_double2(-1.0, 0.0) : make_double2(c, s);
    double sh, ch;
    sincospi((double)ks / (double)n, &sh, &ch);
    tn[t] = nyq ? 0.0 : sh / ch;
    nq[t] = nyq ? 1 : 0;
  }
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
  if (!strain_mask || !d_X || !d_Y || !(L > 0) || !std::isfinite(L)) return RVE_EINVAL;
  if (!supported(n0, 2) || !supported(n1, 2) || !supported(n2, 1) || (n0 & 1) || (n1 & 1)) return RVE_EINVAL;
  rve_s h{};     // every table pointer the FFT kernels do not use stays null
  h.n0 = n0; h.n1 = n1; h.n2 = n2; h.nkx = n0 / 2 + 1;
  h.nvox = (size_t)n0 * n1 * n2;
  h.nspec = (size_t)h.nkx * n1 * n2;
  if (9 * h.nspec * sizeof(double2) > SPEC_MAX_BYTES) return RVE_ENOMEM;
  h.h = L / n0;
  h.stream = (cudaStream_t)cuda_stream;
  make_plan(n0, &h.plan[0]);
  make_plan(n1, &h.plan[1]);
  make_plan(n2, &h.plan[2], 4);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ECUDA;
  if (dev < 0 || dev >= MAX_DEVICES) return RVE_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSlot& sl = g_slot[dev];
    if (!sl.addr) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RVE_ECUDA;
      sl.addr = p;
    }
    base = static_cast<unsigned char*>(sl.addr);
    if (sl.n[0] != n0 || sl.n[1] != n1 || sl.n[2] != n2) {
      k_axis_tables<<<dim3(2, 3), 256, 0, h.stream>>>(base + SPEC_MAX_BYTES, n0, n1, n2);
      if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
      sl.n[0] = n0; sl.n[1] = n1; sl.n[2] = n2;
    }
  }
  h.spec = reinterpret_cast<double2*>(base);
  for (int a = 0; a < 3; ++a) {
    unsigned char* ax = base + SPEC_MAX_BYTES + a * AXIS_PITCH;
    const double2* tw = reinterpret_cast<const double2*>(ax);
    h.ax[a].tw = tw;
    h.ax[a].ph = tw + AXIS_MAX;
    h.ax[a].tanh_ = reinterpret_cast<const double*>(tw + 2 * AXIS_MAX);
    h.ax[a].nyq = reinterpret_cast<const int8_t*>(h.ax[a].tanh_ + AXIS_MAX);
  }

  SpecParams sp{};
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
