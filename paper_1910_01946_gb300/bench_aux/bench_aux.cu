// Measurement helpers for bench.py, built into their own library
// (libbench_aux.so), never into librve.so:
//   - aux_fp64_peak: the FP64 FMA rate of the device, timed live (chains of
//     independent DFMA per thread, CUDA events), the denominator of the FP64
//     roofline fractions;
//   - aux_cufft_time: cuFFT's batched 3-D real transforms (D2Z + Z2D, or
//     R2C + C2R in FP32) on the same grid and field count as the library's
//     hand-written FFT, for the timed comparison.  cuFFT is a comparison
//     here, not part of the product path.
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_dfma_loop(int iters, double b, double c, double* out) {
  double a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  if (s == 1234.5678) out[0] = s;      // never true for the arguments used; keeps the chains live
}

}  // namespace

extern "C" {

// FP64 FMA throughput of the current device: `blocks_per_sm` x SMs blocks
// of 256 threads, each thread `iters` x 8 independent DFMA (2 flops each).
// Returns 0 on success; gflops and ms are the best of `reps` timed launches.
int aux_fp64_peak(int blocks_per_sm, int iters, int reps, double* gflops, double* ms) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = blocks_per_sm * sms;
  k_dfma_loop<<<blocks, 256>>>(iters / 4 + 1, 0.999999, 1e-7, out);    // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    k_dfma_loop<<<blocks, 256>>>(iters, 0.999999, 1e-7, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return 2;
  const double flops = 2.0 * CHAINS * (double)iters * blocks * 256.0;
  *ms = best;
  *gflops = flops / (best * 1e-3) / 1e9;
  return 0;
}

// cuFFT batched 3-D real transforms of nf fields on an n0 x n1 x n2 grid (x
// fastest, the library's layout): forward (D2Z / R2C) then inverse (Z2D /
// C2R), out of place, on buffers allocated here.  ms: average device time
// of one forward + inverse pair over `reps` pairs (CUDA events, after a
// warm-up pair).  Returns 0 on success.
int aux_cufft_time(int n0, int n1, int n2, int nf, int fp32, int reps, double* ms) {
  const size_t nvox = (size_t)n0 * n1 * n2;
  const size_t nspec = (size_t)(n0 / 2 + 1) * n1 * n2;
  const size_t rbytes = nf * nvox * (fp32 ? sizeof(float) : sizeof(double));
  const size_t cbytes = nf * nspec * (fp32 ? sizeof(cufftComplex) : sizeof(cufftDoubleComplex));
  void *rbuf = nullptr, *cbuf = nullptr;
  if (cudaMalloc(&rbuf, rbytes) != cudaSuccess) return 1;
  if (cudaMalloc(&cbuf, cbytes) != cudaSuccess) { cudaFree(rbuf); return 1; }
  cudaMemset(rbuf, 0, rbytes);
  int n[3] = {n2, n1, n0};                     // slowest first
  int inembed[3] = {n2, n1, n0};
  int onembed[3] = {n2, n1, n0 / 2 + 1};
  cufftHandle fwd = 0, inv = 0;
  int rc = 0;
  if (cufftPlanMany(&fwd, 3, n, inembed, 1, (int)nvox, onembed, 1, (int)nspec, fp32 ? CUFFT_R2C : CUFFT_D2Z, nf) !=
          CUFFT_SUCCESS ||
      cufftPlanMany(&inv, 3, n, onembed, 1, (int)nspec, inembed, 1, (int)nvox, fp32 ? CUFFT_C2R : CUFFT_Z2D, nf) !=
          CUFFT_SUCCESS)
    rc = 3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto pair = [&]() -> bool {
    if (fp32)
      return cufftExecR2C(fwd, (cufftReal*)rbuf, (cufftComplex*)cbuf) == CUFFT_SUCCESS &&
             cufftExecC2R(inv, (cufftComplex*)cbuf, (cufftReal*)rbuf) == CUFFT_SUCCESS;
    return cufftExecD2Z(fwd, (cufftDoubleReal*)rbuf, (cufftDoubleComplex*)cbuf) == CUFFT_SUCCESS &&
           cufftExecZ2D(inv, (cufftDoubleComplex*)cbuf, (cufftDoubleReal*)rbuf) == CUFFT_SUCCESS;
  };
  if (rc == 0 && !pair()) rc = 4;
  if (rc == 0) {
    cudaDeviceSynchronize();
    cudaEventRecord(e0);
    for (int r = 0; r < reps && rc == 0; ++r)
      if (!pair()) rc = 4;
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / reps;
  }
  if (cudaGetLastError() != cudaSuccess && rc == 0) rc = 2;
  if (fwd) cufftDestroy(fwd);
  if (inv) cufftDestroy(inv);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(rbuf);
  cudaFree(cbuf);
  return rc;
}

}  // extern "C"
