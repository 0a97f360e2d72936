// Fine-grid streaming kernels: static transmissibilities (a1), density and
// linear-system population (a2, Eqs. 3-6 and Eq. 19), the basis operators of
// Eqs. 8-11, residual SpMV with a fused 2-norm, and deterministic reductions.
//
// All kernels are one thread per cell over the x-fastest layout, so every
// array access of a warp is a coalesced 256-byte run; the six neighbour
// reads of the 7-point stencil hit L1/L2 (each value is read by up to seven
// cells).  FP64 throughout.
#include "cams_internal.h"

namespace cams {

namespace {

__device__ __forceinline__ void cell_xyz(const Geo& g, long long i, int& x, int& y, int& z) {
  xyz_of(g, i, x, y, z);
}

// Block-wide sum; every thread passes its value, thread 0 gets the total.
// Fixed shape, fixed order: bit-reproducible for a fixed launch.
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

__global__ void k_transmissibility(Geo g, double mu, const double* __restrict__ kx,
                                   const double* __restrict__ ky, const double* __restrict__ kz,
                                   int dirichlet, double* Tx, double* Ty, double* Tz, double* Tbw,
                                   double* Tbe) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  cell_xyz(g, i, x, y, z);
  const double ax = g.dy * g.dz, ay = g.dx * g.dz, az = g.dx * g.dy;
  const double lx = kx[i] / mu, ly = ky[i] / mu, lz = kz[i] / mu;
  // TPFA: T = A / (h/(2 lambda_a) + h/(2 lambda_b)) on internal faces
  Tx[i] = x > 0 ? ax / (g.dx / (2.0 * (kx[i - 1] / mu)) + g.dx / (2.0 * lx)) : 0.0;
  Ty[i] = y > 0 ? ay / (g.dy / (2.0 * (ky[i - g.sy] / mu)) + g.dy / (2.0 * ly)) : 0.0;
  Tz[i] = z > 0 ? az / (g.dz / (2.0 * (kz[i - g.sz] / mu)) + g.dz / (2.0 * lz)) : 0.0;
  if (dirichlet) {
    const long long f = y + (long long)g.ny * z;
    if (x == 0) Tbw[f] = ax / (g.dx / (2.0 * lx));
    if (x == g.nx - 1) Tbe[f] = ax / (g.dx / (2.0 * lx));
  }
}

__global__ void k_density(long long N, FluidK fl, const double* __restrict__ p, double* rho) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < N) rho[i] = rho_of(fl, p[i]);
}

// Table 1 step 1: A = C + A~, f, eps (Eq. 19) and per-block sums of eps^2.
// fixm (null when no cell is fixed) marks the prescribed-pressure cells of
// Test Case 2 (Sec. 4.2.2), which are eliminated symmetrically: a face with a
// fixed end stores no coupling, a free cell moves w p_j of a fixed
// neighbour j to its right-hand side (p_j holds the prescribed value), and a
// fixed row reads p_i = p_i with a unit diagonal and eps_i = 0.
//
// full (Reading R22): the full-Jacobian step adds what Eq. 3 leaves out of
// the derivative of the equation over rho, rows times V rho: per face (i, j),
// h = T (p_i - p_j) / 2 gives h rho'_i on the diagonal and h rho'_j at (i, j);
// the diagonal also takes - Phi_i rho'_i / rho_i (Phi_i the mass flux
// leaving i).  A p^{nu+1} = f keeps meaning A dp = -F, so f takes X p^nu over
// the free columns.  A is then not symmetric: Ax.. hold the row's lower
// couplings a_{i,i-e}, Axu.. the transposed ones a_{i-e,i}, both at cell i.
__global__ void k_assemble(Geo g, FluidK fl, double dt, int dirichlet, double pw, double pe,
                           double rhow, double rhoe, const double* __restrict__ p,
                           const double* __restrict__ rho, const double* __restrict__ rhon,
                           const double* __restrict__ Tx, const double* __restrict__ Ty,
                           const double* __restrict__ Tz, const double* __restrict__ Tbw,
                           const double* __restrict__ Tbe, const double* __restrict__ src,
                           const unsigned char* __restrict__ fixm, double* Ad, double* Ax,
                           double* Ay, double* Az, double* Cacc, double* f, double* eps,
                           double* red, int full, double* Axu, double* Ayu, double* Azu) {
  double e2 = 0.0;
  const double inv_dt = 1.0 / dt, inv_V = 1.0 / g.V;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, i, x, y, z);
    const double pi = p[i], ri = rho[i];
    const bool fi = fixm && fixm[i];
    double flux = 0.0, dsum = 0.0, rhsb = 0.0;
    // Reading R4: face density = arithmetic mean of the two cell densities
#define CAMS_FACE(cond, T, j, lowslot)                              \
    if (cond) {                                                     \
      const double w = (T) * (0.5 * (ri + rho[j]));                 \
      dsum += w;                                                    \
      flux += w * (pi - p[j]);                                      \
      if (fixm && (fi || fixm[j])) {                                \
        if (!fi) rhsb += w * p[j];                                  \
      } else {                                                      \
        lowslot;                                                    \
      }                                                             \
    }
    double ax = 0.0, ay = 0.0, az = 0.0;
    CAMS_FACE(x > 0, Tx[i], i - 1, ax = -w)
    CAMS_FACE(x < g.nx - 1, Tx[i + 1], i + 1, (void)0)
    CAMS_FACE(y > 0, Ty[i], i - g.sy, ay = -w)
    CAMS_FACE(y < g.ny - 1, Ty[i + g.sy], i + g.sy, (void)0)
    CAMS_FACE(z > 0, Tz[i], i - g.sz, az = -w)
    CAMS_FACE(z < g.nz - 1, Tz[i + g.sz], i + g.sz, (void)0)
#undef CAMS_FACE
    if (dirichlet) {
      const long long fi2 = y + (long long)g.ny * z;
      if (x == 0) {
        const double wb = Tbw[fi2] * rhow;
        dsum += wb; flux += wb * (pi - pw); rhsb += wb * pw;
      }
      if (x == g.nx - 1) {
        const double wb = Tbe[fi2] * rhoe;
        dsum += wb; flux += wb * (pi - pe); rhsb += wb * pe;
      }
    }
    const double rn = rhon[i];
    // d rho / dp: c rho for the exponential law (rho_i already holds
    // rho0 exp(c p_i)), rho0 eta for the linear one
    const double drho = fl.law == 0 ? fl.c * ri : fl.rho0 * fl.c;
    // FP64 divisions are long dependent sequences on this GPU: one per cell
    const double rinv = 1.0 / ri;
    const double phidt = fl.phi * inv_dt;
    // Eq. 4 with d phi/dp = 0, then the row scaling V rho (Reading R7)
    const double cc = phidt * rn * drho * rinv * rinv;
    const double C = g.V * ri * cc;
    const double q = src ? src[i] * inv_V : 0.0;
    const double b = -phidt + phidt * rn * rinv + q;   // Eq. 5
    double xdiag = 0.0, xp = 0.0;
    if (full) {
      double axu = 0.0, ayu = 0.0, azu = 0.0;
#define CAMS_JFACE(cond, T, j, lowslot)                                        \
      if (cond) {                                                              \
        const double h = 0.5 * (T) * (pi - p[j]);                              \
        xdiag += h * drho;                                                     \
        if (!(fixm && (fi || fixm[j]))) {                                      \
          const double drj = fl.law == 0 ? fl.c * rho[j] : fl.rho0 * fl.c;     \
          xp += h * drj * p[j];                                                \
          lowslot;                                                             \
        }                                                                      \
      }
      // a lower face also gives the transposed entry a_{j,i} = -w - h rho'_i
      CAMS_JFACE(x > 0, Tx[i], i - 1,
                 (ax += h * drj, axu = -(Tx[i] * (0.5 * (ri + rho[i - 1]))) - h * drho))
      CAMS_JFACE(x < g.nx - 1, Tx[i + 1], i + 1, (void)0)
      CAMS_JFACE(y > 0, Ty[i], i - g.sy,
                 (ay += h * drj, ayu = -(Ty[i] * (0.5 * (ri + rho[i - g.sy]))) - h * drho))
      CAMS_JFACE(y < g.ny - 1, Ty[i + g.sy], i + g.sy, (void)0)
      CAMS_JFACE(z > 0, Tz[i], i - g.sz,
                 (az += h * drj, azu = -(Tz[i] * (0.5 * (ri + rho[i - g.sz]))) - h * drho))
      CAMS_JFACE(z < g.nz - 1, Tz[i + g.sz], i + g.sz, (void)0)
#undef CAMS_JFACE
      xdiag -= flux * drho * rinv;
      Axu[i] = axu; Ayu[i] = ayu; Azu[i] = azu;
    }
    Ax[i] = ax; Ay[i] = ay; Az[i] = az;
    Cacc[i] = C;
    double e = 0.0;
    if (fi) {
      Ad[i] = 1.0;
      f[i] = pi;
    } else {
      double fv = g.V * ri * b + rhsb + C * pi;
      if (full) {
        Ad[i] = C + dsum + xdiag;
        fv += xdiag * pi + xp;
      } else {
        Ad[i] = C + dsum;
      }
      f[i] = fv;
      e = q - phidt + phidt * rn * rinv - flux * inv_V * rinv;  // Eq. 19
    }
    eps[i] = e;
    e2 += e * e;
  }
  const double s = block_sum(e2);
  if (threadIdx.x == 0) red[blockIdx.x] = s;
}

// Prescribed cells in list order (a repeated cell keeps its last value):
// mark the cell and put its value into the iterate.
__global__ void k_fix_cells(int n, const int* __restrict__ cell, const double* __restrict__ val,
                            unsigned char* fixm, double* p, long long N) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int k = 0; k < n; ++k) {
    const int c = cell[k];
    if (c >= 0 && c < N) {
      fixm[c] = 1;
      p[c] = val[k];
    }
  }
}

__global__ void k_add_sources(int n, const int* __restrict__ cell, const double* __restrict__ rate,
                              double* src, long long N) {
  // single thread: repeated cells add up in list order (deterministic)
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int k = 0; k < n; ++k) {
    const int c = cell[k];
    if (c >= 0 && c < N) src[c] += rate[k];
  }
}

__global__ void k_sumsq_partial(const double* __restrict__ x, long long N, double* red) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  s = block_sum(s);
  if (threadIdx.x == 0) red[blockIdx.x] = s;
}

__global__ void k_finish_sum(const double* __restrict__ red, int n, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += red[i];
  s = block_sum(s);
  if (threadIdx.x == 0) out[0] = s;
}

// r = f - A p and per-block sums of r^2 (kNS: Axu.. hold the couplings to
// the upper neighbours; otherwise A is symmetric and Ax.. serve both).  Warps take whole
// x-rows (lanes along x, coalesced), so the cell coordinates cost one
// division per row.  r32 (null unless wanted): r rounded to FP32 once, for
// the mixed preconditioner's restriction and smoothing steps, which would
// otherwise each round it again (an FP64-unit conversion per cell).
template <bool kNS>
__global__ void k_residual(Geo g, const double* __restrict__ Ad, const double* __restrict__ Ax,
                           const double* __restrict__ Ay, const double* __restrict__ Az,
                           const double* __restrict__ Axu, const double* __restrict__ Ayu,
                           const double* __restrict__ Azu, const double* __restrict__ f,
                           const double* __restrict__ p, double* r, float* r32, double* red) {
  double s2 = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const unsigned rows = (unsigned)g.ny * (unsigned)g.nz;
  for (unsigned row = blockIdx.x * nw + warp; row < rows; row += gridDim.x * nw) {
    const int y = (int)(row % (unsigned)g.ny), z = (int)(row / (unsigned)g.ny);
    const long long base = g.sy * y + g.sz * z;
    for (int x = lane; x < g.nx; x += 32) {
      const long long i = base + x;
      double a = f[i] - Ad[i] * p[i];
      if (x > 0) a -= Ax[i] * p[i - 1];
      if (x < g.nx - 1) a -= (kNS ? Axu : Ax)[i + 1] * p[i + 1];
      if (y > 0) a -= Ay[i] * p[i - g.sy];
      if (y < g.ny - 1) a -= (kNS ? Ayu : Ay)[i + g.sy] * p[i + g.sy];
      if (z > 0) a -= Az[i] * p[i - g.sz];
      if (z < g.nz - 1) a -= (kNS ? Azu : Az)[i + g.sz] * p[i + g.sz];
      if (r) r[i] = a;
      if (r32) r32[i] = (float)a;
      s2 += a * a;
    }
  }
  s2 = block_sum(s2);
  if (threadIdx.x == 0) red[blockIdx.x] = s2;
}

// Basis operators A_b (Eqs. 8-11, Reading R10: internal faces only).
// Prescribed cells (fixm, null when none) are eliminated as in A: no
// coupling across a face with a fixed end, the free row keeps the face on
// its diagonal, a fixed row is a unit row.
__global__ void k_basis_operator(Geo g, FluidK fl, int kind, double dt,
                                 const double* __restrict__ Tx, const double* __restrict__ Ty,
                                 const double* __restrict__ Tz, const double* __restrict__ rho,
                                 const double* __restrict__ Cacc, const double* __restrict__ pn,
                                 const unsigned char* __restrict__ fixm, double* Abd, double* Abx,
                                 double* Aby, double* Abz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  cell_xyz(g, i, x, y, z);
  const bool fi = fixm && fixm[i];
  if (fi) {
    Abd[i] = 1.0; Abx[i] = 0.0; Aby[i] = 0.0; Abz[i] = 0.0;
    return;
  }
  // (B1), (B2): rho_f-weighted faces, the couplings of A; (B3), (B4): T
  const double ri = kind <= 2 ? rho[i] : 0.0;
  double bx = 0.0, by = 0.0, bz = 0.0, d = 0.0;
#define CAMS_BFACE(cond, T, j, lowslot)                                 \
  if (cond) {                                                           \
    const double w = kind <= 2 ? (T) * (0.5 * (ri + rho[j])) : (T);     \
    d += w;                                                             \
    if (!(fixm && fixm[j])) { lowslot; }                                \
  }
  CAMS_BFACE(x > 0, Tx[i], i - 1, bx = -w)
  CAMS_BFACE(x < g.nx - 1, Tx[i + 1], i + 1, (void)0)
  CAMS_BFACE(y > 0, Ty[i], i - g.sy, by = -w)
  CAMS_BFACE(y < g.ny - 1, Ty[i + g.sy], i + g.sy, (void)0)
  CAMS_BFACE(z > 0, Tz[i], i - g.sz, bz = -w)
  CAMS_BFACE(z < g.nz - 1, Tz[i + g.sz], i + g.sz, (void)0)
#undef CAMS_BFACE
  if (kind == 1) d += Cacc[i];
  if (kind == 3) {
    const double pp = pn[i];
    const double r = rho_of(fl, pp);
    const double dr = fl.law == 0 ? fl.c * fl.rho0 * exp(fl.c * pp) : fl.rho0 * fl.c;
    d += g.V * (fl.phi * r * dr / (dt * r * r));   // V c^n, Eq. 4 at p = p^n
  }
  Abd[i] = d; Abx[i] = bx; Aby[i] = by; Abz[i] = bz;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_transmissibility(const Geo& g, double mu, const double* kx, const double* ky,
                                    const double* kz, int dirichlet, Buffers& b, cudaStream_t s) {
  k_transmissibility<<<blocks_for(g.N, 256), 256, 0, s>>>(g, mu, kx, ky, kz, dirichlet, b.Tx,
                                                          b.Ty, b.Tz, b.Tbw, b.Tbe); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_density(const Geo& g, const FluidK& fl, const double* p, double* rho,
                           cudaStream_t s) {
  k_density<<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, fl, p, rho); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const Geo& g, const FluidK& fl, double dt, int dirichlet, double pw,
                            double pe, const unsigned char* fixm, bool full, Buffers& b,
                            cudaStream_t s) {
  FluidK f2 = fl;
  const double rhow = fl.law == 0 ? fl.rho0 * std::exp(fl.c * pw) : fl.rho0 * (1.0 + fl.c * pw);
  const double rhoe = fl.law == 0 ? fl.rho0 * std::exp(fl.c * pe) : fl.rho0 * (1.0 + fl.c * pe);
  k_assemble<<<kRedBlocks, kRedThreads, 0, s>>>(g, f2, dt, dirichlet, pw, pe, rhow, rhoe, b.p,
                                                b.rho, b.rhon, b.Tx, b.Ty, b.Tz, b.Tbw, b.Tbe,
                                                b.src, fixm, b.Ad, b.Ax, b.Ay, b.Az, b.Cacc, b.f,
                                                b.eps, b.red, full ? 1 : 0, b.Axu, b.Ayu,
                                                b.Azu); count_launches(1);
  k_finish_sum<<<1, 1024, 0, s>>>(b.red, kRedBlocks, b.scal); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_add_sources(int n, const int* cell, const double* rate, double* src,
                               long long N, cudaStream_t s) {
  k_add_sources<<<1, 32, 0, s>>>(n, cell, rate, src, N); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fix_cells(int n, const int* cell, const double* val, unsigned char* fixm,
                             double* p, long long N, cudaStream_t s) {
  k_fix_cells<<<1, 32, 0, s>>>(n, cell, val, fixm, p, N); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* x, long long N, double* red, double* out, cudaStream_t s) {
  k_sumsq_partial<<<kRedBlocks, kRedThreads, 0, s>>>(x, N, red); count_launches(1);
  k_finish_sum<<<1, 1024, 0, s>>>(red, kRedBlocks, out); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Geo& g, const Buffers& b, const double* p, double* r,
                            double* red, double* out, cudaStream_t s) {
  // the FP32 copy goes with the handle's own residual vector (mixed precision)
  float* r32 = (r && r == b.r) ? b.f32.r : nullptr;
  if (b.Axu != b.Ax)
    k_residual<true><<<kRedBlocks, kRedThreads, 0, s>>>(g, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu,
                                                        b.Azu, b.f, p, r, r32, red);
  else
    k_residual<false><<<kRedBlocks, kRedThreads, 0, s>>>(g, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu,
                                                         b.Azu, b.f, p, r, r32, red);
  count_launches(1);
  k_finish_sum<<<1, 1024, 0, s>>>(red, kRedBlocks, out); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_basis_operator(const Geo& g, const FluidK& fl, int kind, double dt,
                                  const unsigned char* fixm, Buffers& b, cudaStream_t s) {
  k_basis_operator<<<blocks_for(g.N, 256), 256, 0, s>>>(g, fl, kind, dt, b.Tx, b.Ty, b.Tz, b.rho,
                                                        b.Cacc, b.pn, fixm, b.Abd, b.Abx, b.Aby,
                                                        b.Abz); count_launches(1);
  return cudaGetLastError();
}

}  // namespace cams
