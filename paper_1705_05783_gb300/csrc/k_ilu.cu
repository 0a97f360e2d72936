// ILU(0) second-stage smoother (Sec. 3, Table 1 step 6) for the 7-point
// matrix in natural order.  For this stencil ILU(0) only changes the
// diagonal: d_i = a_ii - sum_{j in {i-1, i-nx, i-nx*ny}} a_ij a_ji / d_j, and
// M = (D + L_A) D^{-1} (D + U_A) with L_A, U_A the strict triangles of A.
//
// Level-scheduled version: the cells of hyperplane x+y+z = L depend only on
// hyperplane L-1 (forward) or L+1 (backward), so each hyperplane is one
// launch of one thread per (y, z) pair.
#include "cams_internal.h"

namespace cams {

namespace {

__global__ void k_ilu_factor_level(Geo g, int L, const double* __restrict__ Ad,
                                   const double* __restrict__ Ax, const double* __restrict__ Ay,
                                   const double* __restrict__ Az, double* dinv, int* status) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)g.ny * g.nz) return;
  const int y = (int)(t % g.ny), z = (int)(t / g.ny);
  const int x = L - y - z;
  if (x < 0 || x >= g.nx) return;
  const long long i = x + g.sy * y + g.sz * z;
  double d = Ad[i];
  if (x > 0) d -= Ax[i] * Ax[i] * dinv[i - 1];
  if (y > 0) d -= Ay[i] * Ay[i] * dinv[i - g.sy];
  if (z > 0) d -= Az[i] * Az[i] * dinv[i - g.sz];
  if (!(d != 0.0) || !isfinite(d)) {
    atomicOr(status, kStatSingular);
    d = 1.0;
  }
  dinv[i] = 1.0 / d;
}

// w_i = d_i^{-1} (r_i - sum_{lower} a_ij w_j), r = f - A p computed in place.
__global__ void k_ilu_fwd_level(Geo g, int L, const double* __restrict__ Ad,
                                const double* __restrict__ Ax, const double* __restrict__ Ay,
                                const double* __restrict__ Az, const double* __restrict__ f,
                                const double* __restrict__ p, const double* __restrict__ dinv,
                                double* w) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)g.ny * g.nz) return;
  const int y = (int)(t % g.ny), z = (int)(t / g.ny);
  const int x = L - y - z;
  if (x < 0 || x >= g.nx) return;
  const long long i = x + g.sy * y + g.sz * z;
  double r = f[i] - Ad[i] * p[i];
  double s = 0.0;
  if (x > 0) { r -= Ax[i] * p[i - 1]; s += Ax[i] * w[i - 1]; }
  if (x < g.nx - 1) r -= Ax[i + 1] * p[i + 1];
  if (y > 0) { r -= Ay[i] * p[i - g.sy]; s += Ay[i] * w[i - g.sy]; }
  if (y < g.ny - 1) r -= Ay[i + g.sy] * p[i + g.sy];
  if (z > 0) { r -= Az[i] * p[i - g.sz]; s += Az[i] * w[i - g.sz]; }
  if (z < g.nz - 1) r -= Az[i + g.sz] * p[i + g.sz];
  w[i] = (r - s) * dinv[i];
}

// x_i = w_i - d_i^{-1} sum_{upper} a_ij x_j (in place in w), p_i += x_i.
__global__ void k_ilu_bwd_level(Geo g, int L, const double* __restrict__ Ax,
                                const double* __restrict__ Ay, const double* __restrict__ Az,
                                const double* __restrict__ dinv, double* w, double* p) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)g.ny * g.nz) return;
  const int y = (int)(t % g.ny), z = (int)(t / g.ny);
  const int x = L - y - z;
  if (x < 0 || x >= g.nx) return;
  const long long i = x + g.sy * y + g.sz * z;
  double s = 0.0;
  if (x < g.nx - 1) s += Ax[i + 1] * w[i + 1];
  if (y < g.ny - 1) s += Ay[i + g.sy] * w[i + g.sy];
  if (z < g.nz - 1) s += Az[i + g.sz] * w[i + g.sz];
  const double xi = w[i] - dinv[i] * s;
  w[i] = xi;
  p[i] += xi;
}

}  // namespace

cudaError_t launch_ilu_factor(const Geo& g, Buffers& b, cudaStream_t s) {
  const long long nt = (long long)g.ny * g.nz;
  const int blocks = (int)((nt + 255) / 256);
  const int levels = g.nx + g.ny + g.nz - 2;
  for (int L = 0; L < levels; ++L)
    k_ilu_factor_level<<<blocks, 256, 0, s>>>(g, L, b.Ad, b.Ax, b.Ay, b.Az, b.dinv, b.status);
  return cudaGetLastError();
}

cudaError_t launch_ilu_smooth(const Geo& g, Buffers& b, cudaStream_t s) {
  const long long nt = (long long)g.ny * g.nz;
  const int blocks = (int)((nt + 255) / 256);
  const int levels = g.nx + g.ny + g.nz - 2;
  for (int L = 0; L < levels; ++L)
    k_ilu_fwd_level<<<blocks, 256, 0, s>>>(g, L, b.Ad, b.Ax, b.Ay, b.Az, b.f, b.p, b.dinv, b.w);
  for (int L = levels - 1; L >= 0; --L)
    k_ilu_bwd_level<<<blocks, 256, 0, s>>>(g, L, b.Ax, b.Ay, b.Az, b.dinv, b.w, b.p);
  return cudaGetLastError();
}

}  // namespace cams
