// ILU(0) second-stage smoother (Sec. 3, Table 1 step 6) for the 7-point
// matrix in natural order.  For this stencil ILU(0) only changes the
// diagonal: d_i = a_ii - sum_{j in {i-1, i-nx, i-nx*ny}} a_ij a_ji / d_j, and
// M = (D + L_A) D^{-1} (D + U_A) with L_A, U_A the strict triangles of A.
// One smoothing step p <- p + M^{-1}(f - A p) is
//   rd = D^{-1} (f - A p)                         (parallel)
//   w_i = rd_i - sum_{j<i} (a_ij / d_i) w_j       (forward wavefront)
//   z_i = w_i  - sum_{j>i} (a_ij / d_i) z_j       (backward wavefront)
//   p += z
// with the couplings pre-scaled by the row pivot once per factorisation, so
// every cell of a sweep is a chain of at most three FMAs.
//
// Two schedules of the same arithmetic (bitwise identical results):
//  * level-scheduled: one launch per hyperplane x+y+z = L (reference);
//  * pipelined: one persistent launch per sweep.  A thread owns an x-row
//    (y, z); a CTA owns a TY x TZ block of rows and steps through x in
//    lockstep, row (ty, tz) lagging one cell per row hop (ty + tz), so the
//    values it needs from rows y-1 and z-1 were produced one step earlier
//    and are exchanged in shared memory.  Row blocks that border other CTAs
//    read those CTAs' boundary rows from global memory (L2, bypassing L1)
//    after an acquire-poll of the producer's progress counter, which the
//    producer publishes with release semantics every kBatch steps; every
//    row loads the operands of its next kBatch cells with independent loads
//    at the start of a batch, and a row that borders another tile fetches
//    kBatch boundary values per poll.  Tiles
//    are claimed through an atomic ticket in anti-diagonal order, so a CTA
//    only ever waits on tiles already claimed by running CTAs: no
//    co-residency assumption, no deadlock.  Every wait has an iteration
//    limit; on expiry the kernel sets an abort flag and the status word and
//    all CTAs leave.
#include <cuda/atomic>

#include "cams_internal.h"

namespace cams {

namespace {

constexpr int kBatch = 8;                    // steps per batch of cross-tile loads / publications
constexpr long long kSpinLimit = 1LL << 22;  // polls before a wait gives up (~ seconds)

// ----------------------------------------------------------- factor ---

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

// Row-pivot-scaled couplings: L_d[i] = a_{i,i-e_d} / d_i, U_d[i] = a_{i,i+e_d} / d_i.
__global__ void k_ilu_scale(Geo g, const double* __restrict__ Ax, const double* __restrict__ Ay,
                            const double* __restrict__ Az, const double* __restrict__ dinv,
                            double* Lx, double* Ly, double* Lz, double* Ux, double* Uy, double* Uz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const int x = (int)(i % g.nx);
  const int y = (int)((i / g.nx) % g.ny);
  const int z = (int)(i / g.sz);
  const double di = dinv[i];
  Lx[i] = Ax[i] * di;
  Ly[i] = Ay[i] * di;
  Lz[i] = Az[i] * di;
  Ux[i] = x < g.nx - 1 ? Ax[i + 1] * di : 0.0;
  Uy[i] = y < g.ny - 1 ? Ay[i + g.sy] * di : 0.0;
  Uz[i] = z < g.nz - 1 ? Az[i + g.sz] * di : 0.0;
}

// rd = D^{-1} (f - A p)
__global__ void k_resid_scaled(Geo g, const double* __restrict__ Ad, const double* __restrict__ Ax,
                               const double* __restrict__ Ay, const double* __restrict__ Az,
                               const double* __restrict__ f, const double* __restrict__ p,
                               const double* __restrict__ dinv, double* rd) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const int x = (int)(i % g.nx);
  const int y = (int)((i / g.nx) % g.ny);
  const int z = (int)(i / g.sz);
  double a = f[i] - Ad[i] * p[i];
  if (x > 0) a -= Ax[i] * p[i - 1];
  if (x < g.nx - 1) a -= Ax[i + 1] * p[i + 1];
  if (y > 0) a -= Ay[i] * p[i - g.sy];
  if (y < g.ny - 1) a -= Ay[i + g.sy] * p[i + g.sy];
  if (z > 0) a -= Az[i] * p[i - g.sz];
  if (z < g.nz - 1) a -= Az[i + g.sz] * p[i + g.sz];
  rd[i] = a * dinv[i];
}

// ------------------------------------------------- per-cell operators ---
// Each sweep is "value_i = op(i, values of the three upstream neighbours)".
// load() fetches the operands of one cell (issued a batch ahead, so the
// loads overlap); apply() combines them with the upstream values.

struct FwdSolve {   // w_i = rd_i - Lz w_{z-1} - Ly w_{y-1} - Lx w_{x-1}
  const double *rd, *Lx, *Ly, *Lz;
  double* w;
  struct In { double rd, lx, ly, lz; };
  __device__ __forceinline__ In load(long long i) const {
    return In{__ldg(rd + i), __ldg(Lx + i), __ldg(Ly + i), __ldg(Lz + i)};
  }
  __device__ __forceinline__ double apply(const In& a, long long i, bool hx, double vx, bool hy,
                                          double vy, bool hz, double vz) const {
    double v = a.rd;
    if (hz) v = fma(-a.lz, vz, v);
    if (hy) v = fma(-a.ly, vy, v);
    if (hx) v = fma(-a.lx, vx, v);
    w[i] = v;
    return v;
  }
};

struct BwdSolve {   // z_i = w_i - Uz z_{z+1} - Uy z_{y+1} - Ux z_{x+1};  p_i += z_i
  const double *Ux, *Uy, *Uz;
  double *w, *p;
  struct In { double w, ux, uy, uz, p; };
  __device__ __forceinline__ In load(long long i) const {
    return In{w[i], __ldg(Ux + i), __ldg(Uy + i), __ldg(Uz + i), p[i]};
  }
  __device__ __forceinline__ double apply(const In& a, long long i, bool hx, double vx, bool hy,
                                          double vy, bool hz, double vz) const {
    double v = a.w;
    if (hz) v = fma(-a.uz, vz, v);
    if (hy) v = fma(-a.uy, vy, v);
    if (hx) v = fma(-a.ux, vx, v);
    w[i] = v;
    p[i] = a.p + v;
    return v;
  }
};

struct Factor {     // d_i = a_ii - a_{i,x-1}^2 / d_{x-1} - a_{i,y-1}^2 / d_{y-1} - a_{i,z-1}^2 / d_{z-1}
  const double *Ad, *Ax, *Ay, *Az;
  double* dinv;
  int* status;
  struct In { double d, ax, ay, az; };
  __device__ __forceinline__ In load(long long i) const {
    return In{__ldg(Ad + i), __ldg(Ax + i), __ldg(Ay + i), __ldg(Az + i)};
  }
  __device__ __forceinline__ double apply(const In& a, long long i, bool hx, double vx, bool hy,
                                          double vy, bool hz, double vz) const {
    double d = a.d;
    if (hx) d -= a.ax * a.ax * vx;
    if (hy) d -= a.ay * a.ay * vy;
    if (hz) d -= a.az * a.az * vz;
    if (!(d != 0.0) || !isfinite(d)) {
      atomicOr(status, kStatSingular);
      d = 1.0;
    }
    const double v = 1.0 / d;
    dinv[i] = v;
    return v;
  }
};

// ---------------------------------------------------- level schedule ---

template <class Op, bool kBackward>
__global__ void k_sweep_level(Geo g, int L, Op op, const double* vals) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)g.ny * g.nz) return;
  const int y = (int)(t % g.ny), z = (int)(t / g.ny);
  const int xf = L - y - z;                 // position along the sweep
  if (xf < 0 || xf >= g.nx) return;
  // the backward sweep visits hyperplane L of the mirrored grid
  const int x = kBackward ? g.nx - 1 - xf : xf;
  const int yy = kBackward ? g.ny - 1 - y : y;
  const int zz = kBackward ? g.nz - 1 - z : z;
  const long long i = x + g.sy * yy + g.sz * zz;
  const typename Op::In in = op.load(i);
  if (!kBackward) {
    const bool hx = x > 0, hy = yy > 0, hz = zz > 0;
    op.apply(in, i, hx, hx ? vals[i - 1] : 0.0, hy, hy ? vals[i - g.sy] : 0.0, hz,
             hz ? vals[i - g.sz] : 0.0);
  } else {
    const bool hx = x < g.nx - 1, hy = yy < g.ny - 1, hz = zz < g.nz - 1;
    op.apply(in, i, hx, hx ? vals[i + 1] : 0.0, hy, hy ? vals[i + g.sy] : 0.0, hz,
             hz ? vals[i + g.sz] : 0.0);
  }
}

// ------------------------------------------------ pipelined schedule ---

__device__ __forceinline__ void tile_of_ticket(int t, int nty, int ntz, int& Y, int& Z) {
  // anti-diagonals d = Y + Z in increasing order, Y ascending within one
  for (int d = 0;; ++d) {
    const int ylo = d - (ntz - 1) > 0 ? d - (ntz - 1) : 0;
    const int yhi = d < nty - 1 ? d : nty - 1;
    const int cnt = yhi - ylo + 1;
    if (t < cnt) {
      Y = ylo + t;
      Z = d - Y;
      return;
    }
    t -= cnt;
  }
}

// Wait until *ctr >= need (acquire).  Returns false on abort or timeout.
__device__ __forceinline__ bool wait_at_least(int* ctr, int need, int* abort_flag, int* status) {
  cuda::atomic_ref<int, cuda::thread_scope_device> a(*ctr);
  cuda::atomic_ref<int, cuda::thread_scope_device> ab(*abort_flag);
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (a.load(cuda::memory_order_acquire) >= need) return true;
    if (ab.load(cuda::memory_order_relaxed)) return false;
    __nanosleep(64);
  }
  atomicOr(status, kStatTimeout);
  ab.store(1, cuda::memory_order_relaxed);
  return false;
}

// ctrl: [0] ticket, [1] abort flag, [2 + tile] progress (steps completed).
// The backward sweep runs the same schedule on the mirrored grid
// (x -> nx-1-x, y -> ny-1-y, z -> nz-1-z).  Steps are grouped in batches of
// kBatch.  At the start of a batch every row loads the operands of its
// kBatch cells of that batch (independent loads: one memory round trip per
// batch), and a row that borders an upstream tile waits once for the
// producer to be a whole batch ahead and then fetches that batch's boundary
// values with independent L2 loads; producers publish at the end of each
// batch.
template <int TY, int TZ, class Op, bool kBackward>
__global__ void __launch_bounds__(TY* TZ, 1) k_sweep_pipe(Geo g, Op op, const double* vals, int* ctrl,
                                                          int* status) {
  __shared__ double buf[2][TZ][TY];
  __shared__ double yin[TZ][kBatch];   // boundary values from the tile below in y (ty == 0 rows)
  __shared__ double zin[TY][kBatch];   // boundary values from the tile below in z (tz == 0 rows)
  __shared__ int s_tile;
  const int ty = threadIdx.x % TY, tz = threadIdx.x / TY;
  const int nty = (g.ny + TY - 1) / TY, ntz = (g.nz + TZ - 1) / TZ;
  const int ntiles = nty * ntz;
  const int nsteps = g.nx + TY + TZ - 2;
  int* progress = ctrl + 2;
  for (;;) {
    __syncthreads();                           // s_tile of the previous tile is consumed
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctrl[0], 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) return;
    int Y, Z;                                  // tile in mirrored coordinates
    tile_of_ticket(t, nty, ntz, Y, Z);
    const int ym = Y * TY + ty, zm = Z * TZ + tz;   // my row, mirrored coordinates
    const bool valid = ym < g.ny && zm < g.nz;
    const int y = kBackward ? g.ny - 1 - ym : ym;
    const int z = kBackward ? g.nz - 1 - zm : zm;
    const long long row = (long long)y * g.sy + (long long)z * g.sz;
    const long long sy = kBackward ? -g.sy : g.sy, sz = kBackward ? -g.sz : g.sz;
    const bool hy = ym > 0, hz = zm > 0;       // upstream neighbours exist
    const bool ext_y = valid && ty == 0 && hy; // my y-neighbour lives in another tile
    const bool ext_z = valid && tz == 0 && hz;
    int* dep_y = ext_y ? &progress[(Y - 1) + nty * Z] : nullptr;
    int* dep_z = ext_z ? &progress[Y + nty * (Z - 1)] : nullptr;
    const bool boundary = (ty == TY - 1) || (tz == TZ - 1);
    double vprev = 0.0;
    bool fail = false;
    for (int s0 = 0; s0 < nsteps; s0 += kBatch) {
      // operands of my cells in this batch
      typename Op::In in[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int k = s0 + u - ty - tz;
        if (valid && k >= 0 && k < g.nx) in[u] = op.load(row + (kBackward ? g.nx - 1 - k : k));
      }
      // boundary values from upstream tiles
      const int last = min(s0 + kBatch - 1, nsteps - 1);
      if (ext_y && !fail) {
        if (!wait_at_least(dep_y, min(last + TY, nsteps), ctrl + 1, status)) fail = true;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int k = s0 + u - ty - tz;
          double v = 0.0;
          if (!fail && k >= 0 && k < g.nx) v = __ldcg(vals + (row + (kBackward ? g.nx - 1 - k : k) - sy));
          yin[tz][u] = v;
        }
      }
      if (ext_z && !fail) {
        if (!wait_at_least(dep_z, min(last + TZ, nsteps), ctrl + 1, status)) fail = true;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int k = s0 + u - ty - tz;
          double v = 0.0;
          if (!fail && k >= 0 && k < g.nx) v = __ldcg(vals + (row + (kBackward ? g.nx - 1 - k : k) - sz));
          zin[ty][u] = v;
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int s = s0 + u;
        if (s >= nsteps) break;                // uniform over the CTA
        const int k = s - ty - tz;             // cell of my row at this step
        double v = 0.0;
        if (valid && k >= 0 && k < g.nx && !fail) {
          const int x = kBackward ? g.nx - 1 - k : k;
          double vy = 0.0, vz = 0.0;
          if (hy) vy = (ty > 0) ? buf[(s - 1) & 1][tz][ty - 1] : yin[tz][u];
          if (hz) vz = (tz > 0) ? buf[(s - 1) & 1][tz - 1][ty] : zin[ty][u];
          v = op.apply(in[u], row + x, k > 0, vprev, hy, vy, hz, vz);
          vprev = v;
        }
        buf[s & 1][tz][ty] = v;
        const bool publish = (u == kBatch - 1) || (s + 1 == nsteps);
        if (publish && boundary) __threadfence();
        if (__syncthreads_or(fail)) {
          if (threadIdx.x == 0) {
            cuda::atomic_ref<int, cuda::thread_scope_device> ab(ctrl[1]);
            ab.store(1, cuda::memory_order_relaxed);
          }
          return;
        }
        if (publish && threadIdx.x == 0) {
          cuda::atomic_ref<int, cuda::thread_scope_device> pr(progress[Y + nty * Z]);
          pr.store(s + 1, cuda::memory_order_release);
        }
      }
    }
  }
}

// Self-test of the bounded wait: waits on a counter that nothing sets.
__global__ void k_wait_selftest(int* ctrl, int* status) {
  if (threadIdx.x == 0) wait_at_least(&ctrl[2], 1, &ctrl[1], status);
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

constexpr int kTY = 8, kTZ = 8;

}  // namespace

int ilu_ctrl_ints(const Geo& g) {
  return 2 + ((g.ny + kTY - 1) / kTY) * ((g.nz + kTZ - 1) / kTZ);
}

cudaError_t launch_ilu_factor(const Geo& g, Buffers& b, bool pipelined, int grid, cudaStream_t s) {
  const int levels = g.nx + g.ny + g.nz - 2;
  int n = 1;
  if (!pipelined) {
    const int blocks = blocks_for((long long)g.ny * g.nz, 256);
    for (int L = 0; L < levels; ++L)
      k_ilu_factor_level<<<blocks, 256, 0, s>>>(g, L, b.Ad, b.Ax, b.Ay, b.Az, b.dinv, b.status);
    n += levels;
  } else {
    cudaError_t e = cudaMemsetAsync(b.ctrl, 0, sizeof(int) * (size_t)ilu_ctrl_ints(g), s);
    if (e != cudaSuccess) return e;
    Factor fa{b.Ad, b.Ax, b.Ay, b.Az, b.dinv, b.status};
    k_sweep_pipe<kTY, kTZ, Factor, false><<<grid, kTY * kTZ, 0, s>>>(g, fa, b.dinv, b.ctrl, b.status);
    n += 1;
  }
  k_ilu_scale<<<blocks_for(g.N, 256), 256, 0, s>>>(g, b.Ax, b.Ay, b.Az, b.dinv, b.Lx, b.Ly, b.Lz,
                                                   b.Ux, b.Uy, b.Uz);
  count_launches(n);
  return cudaGetLastError();
}

cudaError_t launch_ilu_resid(const Geo& g, Buffers& b, cudaStream_t s) {
  k_resid_scaled<<<blocks_for(g.N, 256), 256, 0, s>>>(g, b.Ad, b.Ax, b.Ay, b.Az, b.f, b.p, b.dinv,
                                                      b.r);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ilu_sweep(const Geo& g, Buffers& b, bool backward, bool pipelined, int grid,
                             cudaStream_t s) {
  FwdSolve fw{b.r, b.Lx, b.Ly, b.Lz, b.w};
  BwdSolve bw{b.Ux, b.Uy, b.Uz, b.w, b.p};
  if (!pipelined) {
    const int blocks = blocks_for((long long)g.ny * g.nz, 256);
    const int levels = g.nx + g.ny + g.nz - 2;
    for (int L = 0; L < levels; ++L) {
      if (!backward) k_sweep_level<FwdSolve, false><<<blocks, 256, 0, s>>>(g, L, fw, b.w);
      else k_sweep_level<BwdSolve, true><<<blocks, 256, 0, s>>>(g, L, bw, b.w);
    }
    count_launches(levels);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(b.ctrl, 0, sizeof(int) * (size_t)ilu_ctrl_ints(g), s);
  if (e != cudaSuccess) return e;
  if (!backward) k_sweep_pipe<kTY, kTZ, FwdSolve, false><<<grid, kTY * kTZ, 0, s>>>(g, fw, b.w, b.ctrl, b.status);
  else k_sweep_pipe<kTY, kTZ, BwdSolve, true><<<grid, kTY * kTZ, 0, s>>>(g, bw, b.w, b.ctrl, b.status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(const Geo& g, Buffers& b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.ctrl, 0, sizeof(int) * (size_t)ilu_ctrl_ints(g), s);
  if (e != cudaSuccess) return e;
  k_wait_selftest<<<1, 32, 0, s>>>(b.ctrl, b.status);
  count_launches(1);
  return cudaGetLastError();
}

int ilu_pipe_grid(const Geo& g, int num_sms) {
  const int ntiles = ((g.ny + kTY - 1) / kTY) * ((g.nz + kTZ - 1) / kTZ);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_pipe<kTY, kTZ, FwdSolve, false>,
                                                kTY * kTZ, 0);
  const int cap = num_sms * (per_sm > 0 ? per_sm : 1);
  return ntiles < cap ? ntiles : cap;
}

}  // namespace cams
