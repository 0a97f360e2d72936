// Checks rcp_halley (paper_1705_05783_gb300/csrc/rcp64.h) against IEEE 1/d on
// 2^22 values d = m 2^e, m uniform in [1, 2), e uniform in [-300, 300], both
// signs; prints the largest error in ulps, the largest relative error and the
// share of results equal to 1/d.  Run by tests/test_gpu_rcp64.py.
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>

#include "rcp64.h"

__global__ void k_check(int n, unsigned long long seed, long long* ulps, double* rel) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long s = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  s ^= s >> 33; s *= 0xff51afd7ed558ccdull; s ^= s >> 33; s *= 0xc4ceb9fe1a85ec53ull; s ^= s >> 33;
  const double m = 1.0 + (double)(s >> 12) * (1.0 / 4503599627370496.0);
  const int ex = (int)((s >> 3) % 601) - 300;
  const double d = (s & 1) ? -ldexp(m, ex) : ldexp(m, ex);
  const double ref = 1.0 / d, x = cams::rcp_halley(d);
  const long long a = __double_as_longlong(x), b = __double_as_longlong(ref);
  ulps[i] = a > b ? a - b : b - a;
  rel[i] = fabs(x - ref) / fabs(ref);
}

int main() {
  const int n = 1 << 22;
  long long* du; double* dr;
  if (cudaMalloc(&du, sizeof(long long) * n) != cudaSuccess) return 2;
  if (cudaMalloc(&dr, sizeof(double) * n) != cudaSuccess) return 2;
  k_check<<<n / 256, 256>>>(n, 20170516ull, du, dr);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  long long* hu = new long long[n];
  double* hr = new double[n];
  cudaMemcpy(hu, du, sizeof(long long) * n, cudaMemcpyDeviceToHost);
  cudaMemcpy(hr, dr, sizeof(double) * n, cudaMemcpyDeviceToHost);
  long long mu = 0, same = 0;
  double mr = 0.0;
  for (int i = 0; i < n; ++i) {
    if (hu[i] > mu) mu = hu[i];
    if (hr[i] > mr) mr = hr[i];
    same += hu[i] == 0;
  }
  printf("max_ulp %lld max_rel %.6e equal %.6f\n", mu, mr, (double)same / n);
  return 0;
}
