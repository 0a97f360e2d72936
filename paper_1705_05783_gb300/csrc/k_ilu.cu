// ILU(0) second-stage smoother (Sec. 3, Table 1 step 6) for the 7-point
// matrix in natural order.  For this stencil ILU(0) only changes the
// diagonal: d_i = a_ii - sum_{j in {i-1, i-nx, i-nx*ny}} a_ij a_ji / d_j, and
// M = (D + L_A) D^{-1} (D + U_A) with L_A, U_A the strict triangles of A.
// One smoothing step x <- x + M^{-1}(b - A x) is
//   rd = D^{-1} (b - A x)                         (parallel)
//   w_i = rd_i - sum_{j<i} (a_ij / d_i) w_j       (forward wavefront)
//   z_i = w_i  - sum_{j>i} (a_ij / d_i) z_j       (backward wavefront)
//   x += z
// with the couplings pre-scaled by the row pivot once per factorisation, so
// every cell of a sweep is a chain of at most three FMAs.  For a
// nonsymmetric A (the full-Jacobian step) the pivot recurrence takes the
// products a_{i,j} a_{j,i}, formed once per factorisation.  In FP64 (b, x) =
// (f, p).  In the mixed-precision preconditioner the smoother runs in FP32
// on the correction equation A delta = r, (b, x) = (r, delta), with an FP32
// copy of A; r is the FP64 residual and p += delta is taken in FP64.
//
// Layout.  The sweep vectors (rd, the scaled couplings, w, z) are stored
// "skewed tile-major": the (y, z) cross-section is cut into tiles of
// kIluTY x kIluTZ = 32 x-rows, one warp each, and cell (x, y, z) of tile T,
// row (ty, tz) sits at record T * ns + x + ty + tz, slot ty + kIluTY * tz
// (ns >= nx + kIluTY + kIluTZ - 2 records per tile, 32 values per record,
// plus kPad spare records at both ends).  A tile advances one "step" s at a
// time and row (ty, tz) works on x = s - ty - tz, so the 32 cells of one
// step are one contiguous record.  Slots that hold no cell (the pipeline's
// fill and drain, rows beyond the grid) are zero in rd and in the
// couplings, so every step runs the same branch-free arithmetic; the values
// computed there are never read by a cell.  Pivots (dinv) stay in natural
// order.
//
// Two schedules of the same arithmetic (bitwise identical results):
//  * level-scheduled: one launch per hyperplane x+y+z = L (reference);
//  * pipelined: one persistent launch per sweep.  Each warp takes a whole
//    tile and steps through it; the values a row needs from rows y-1 and
//    z-1 of its own tile were produced by the neighbouring lanes one step
//    earlier and arrive by warp shuffle.  Operands are staged into a
//    shared-memory ring kG - 1 groups ahead by bulk copies (the TMA
//    engine; one per operand and group of kU records).  Values from
//    another tile are read from the sweep's output vector itself, which is
//    pre-filled with a signalling-NaN sentinel that no arithmetic produces:
//    a value is ready once it differs from the sentinel, so no flags or
//    fences are needed (values are written and read with single-copy atomic
//    relaxed accesses at device scope); they are fetched one group ahead and
//    re-polled only when still unset.  Tiles are claimed through an atomic
//    ticket in anti-diagonal order, so a warp only ever waits on tiles
//    already claimed by running warps: no co-residency assumption, no
//    deadlock.  Every wait has an iteration limit; on expiry the kernel sets
//    an abort flag and the status word and all warps leave.  One CTA of
//    four warps per SM keeps one sweeping warp per FP64 pipe.
//  The backward sweep runs the same schedule on the mirrored grid; with the
//  tiling fixed by the forward direction, its steps read the same records in
//  reverse order.  x += z follows as a separate coalesced pass (k_apply_z).
#include "cams_internal.h"
#include "tc_ptx.h"

namespace cams {

namespace {

constexpr int kTY = kIluTY, kTZ = kIluTZ, kR = kIluR;
static_assert(kR == 32, "a tile is one warp");
constexpr int kWarps = 4;                    // tiles in flight per CTA (one per FP64 pipe)
constexpr int kU = 4;                        // steps per group (straight-line code)
constexpr int kG = 3;                        // operand ring slots (groups staged kG - 1 ahead)
constexpr int kPad = 3 * kU;                 // spare records at both ends of a vector
constexpr bool kBulkStage = false;           // skewed operands staged by bulk copies
constexpr int kL2Ahead = 0;                  // groups of skewed operands prefetched into L2 ahead
constexpr bool kFetchFirst = true;           // cross-tile loads issued before the group's staging
constexpr long long kSpinLimit = 1LL << 22;  // polls before a wait gives up (~ a second)
constexpr int kFastPolls = 64;               // in-loop polls before a wait starts to sleep

// Bit pattern of a value and the "not computed yet" sentinel: a signalling
// NaN.  IEEE arithmetic never produces a signalling NaN, so no computed
// value carries this pattern.
template <class T>
struct Word;
template <>
struct Word<double> {
  using U = unsigned long long;
  static constexpr U kNotReady = 0x7FF4DEADBEEF0001ull;
  static __device__ __forceinline__ double value(U u) { return __longlong_as_double((long long)u); }
};
template <>
struct Word<float> {
  using U = unsigned;
  static constexpr U kNotReady = 0x7FA5A5A1u;
  static __device__ __forceinline__ float value(U u) { return __uint_as_float(u); }
};

template <class T>
__device__ __forceinline__ T not_ready() {
  return Word<T>::value(Word<T>::kNotReady);
}

struct Skew {
  int nty, ntz, ns;   // tiles in y and z, records per tile (a multiple of kU)
};

inline Skew make_skew(const Geo& g) {
  const int ns = g.nx + kTY + kTZ - 2;
  return Skew{(g.ny + kTY - 1) / kTY, (g.nz + kTZ - 1) / kTZ, (ns + kU - 1) / kU * kU};
}

__device__ __forceinline__ long long skew_index(const Skew& k, int x, int y, int z) {
  const int Y = y / kTY, ty = y - Y * kTY, Z = z / kTZ, tz = z - Z * kTZ;
  return ((long long)(Y + k.nty * Z) * k.ns + x + ty + tz + kPad) * kR + ty + kTY * tz;
}

// ---- relaxed device-scope accesses, copies (8- or 4-byte values) ----
__device__ __forceinline__ unsigned long long ld_relaxed(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const float* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// ld_relaxed when `pred` holds, else 0 (a predicated load: no branch).
__device__ __forceinline__ unsigned long long ld_relaxed_if(bool pred, const double* p) {
  unsigned long long v = 0ull;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.relaxed.gpu.global.b64 %0, [%1];\n\t}"
      : "+l"(v)
      : "l"(p), "r"((unsigned)pred));
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_if(bool pred, const float* p) {
  unsigned v = 0u;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q ld.relaxed.gpu.global.b32 %0, [%1];\n\t}"
      : "+r"(v)
      : "l"(p), "r"((unsigned)pred));
  return v;
}

__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void publish(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}
__device__ __forceinline__ void publish(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

__device__ __forceinline__ void cp_async(double* smem_dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(float* smem_dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------ parallel parts ---

// Row-pivot-scaled couplings, stored skewed:
// L_d = a_{i,i-e_d} / d_i, U_d = a_{i,i+e_d} / d_i.
template <class T>
__global__ void k_ilu_scale(Geo g, Skew sk, const T* __restrict__ Ax, const T* __restrict__ Ay,
                            const T* __restrict__ Az, const T* __restrict__ Axu,
                            const T* __restrict__ Ayu, const T* __restrict__ Azu,
                            const T* __restrict__ dinv, T* Lx, T* Ly, T* Lz, T* Ux, T* Uy,
                            T* Uz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  xyz_of(g, i, x, y, z);
  const long long j = skew_index(sk, x, y, z);
  const T di = dinv[i];
  Lx[j] = Ax[i] * di;
  Ly[j] = Ay[i] * di;
  Lz[j] = Az[i] * di;
  Ux[j] = x < g.nx - 1 ? Axu[i + 1] * di : T(0);
  Uy[j] = y < g.ny - 1 ? Ayu[i + g.sy] * di : T(0);
  Uz[j] = z < g.nz - 1 ? Azu[i + g.sz] * di : T(0);
}

// The two conversions between the natural layout and the skewed sweep
// layout run as tile transposes: one CTA per (tile, kXC positions along x).
// Rows are read or written in the natural layout by warps along x
// (coalesced); records are written or read in the skewed layout by warps
// whose lanes are the tile's 32 rows (one 128- or 256-byte record each);
// shared memory holds the kR x kXC block in between.
constexpr int kXC = 64;
static_assert(kR % 8 == 0 && kXC % 32 == 0, "the transposes take 8 warps of 32 lanes");

// rd = D^{-1} (b - A x), stored skewed; b is read in its own precision and
// rounded to T.  kNS: Axu.. hold the couplings to the upper neighbours (A
// not symmetric); otherwise Ax.. serve both.
template <class B, class T, bool kNS>
__global__ void __launch_bounds__(256) k_resid_scaled(Geo g, Skew sk, const T* __restrict__ Ad,
                                                      const T* __restrict__ Ax,
                                                      const T* __restrict__ Ay,
                                                      const T* __restrict__ Az,
                                                      const T* __restrict__ Axu,
                                                      const T* __restrict__ Ayu,
                                                      const T* __restrict__ Azu,
                                                      const B* __restrict__ bv,
                                                      const T* __restrict__ xv,
                                                      const T* __restrict__ dinv, T* rd) {
  __shared__ T blk[kR][kXC + 1];
  const int tile = blockIdx.x, x0 = blockIdx.y * kXC;
  const int Y = tile % sk.nty, Z = tile / sk.nty;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // (both loops unrolled, with predicates instead of early exits, so that a
  // thread's loads of all its cells are in flight together; 256 threads)
#pragma unroll
  for (int rr = 0; rr < kR / 8; ++rr) {
    const int r = warp + rr * 8;
    const int y = Y * kTY + r % kTY, z = Z * kTZ + r / kTY;
#pragma unroll
    for (int hh = 0; hh < kXC / 32; ++hh) {
      const int h = lane + 32 * hh;
      const int x = x0 + h;
      if (y < g.ny && z < g.nz && x < g.nx) {
        const long long i = x + g.sy * y + g.sz * z;
        T a = T(bv[i]) - Ad[i] * xv[i];
        if (x > 0) a -= Ax[i] * xv[i - 1];
        if (x < g.nx - 1) a -= (kNS ? Axu : Ax)[i + 1] * xv[i + 1];
        if (y > 0) a -= Ay[i] * xv[i - g.sy];
        if (y < g.ny - 1) a -= (kNS ? Ayu : Ay)[i + g.sy] * xv[i + g.sy];
        if (z > 0) a -= Az[i] * xv[i - g.sz];
        if (z < g.nz - 1) a -= (kNS ? Azu : Az)[i + g.sz] * xv[i + g.sz];
        blk[r][h] = a * dinv[i];
      }
    }
  }
  __syncthreads();
  // record q holds row (ty, tz) = (lane % kTY, lane / kTY) at x = q - ty - tz
  const int ty = lane % kTY, tz = lane / kTY;
  const bool row_ok = Y * kTY + ty < g.ny && Z * kTZ + tz < g.nz;
  for (int q = x0 + warp; q < x0 + kXC + kTY + kTZ - 2; q += nwarp) {
    const int x = q - ty - tz;
    if (row_ok && x >= x0 && x < x0 + kXC && x < g.nx)
      rd[((long long)tile * sk.ns + q + kPad) * kR + lane] = blk[lane][x - x0];
  }
}

// x += z (the correction of one smoothing step), z stored skewed.
template <class T>
__global__ void __launch_bounds__(256) k_apply_z(Geo g, Skew sk, const T* __restrict__ zs, T* xv) {
  __shared__ T blk[kR][kXC + 1];
  const int tile = blockIdx.x, x0 = blockIdx.y * kXC;
  const int Y = tile % sk.nty, Z = tile / sk.nty;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int ty = lane % kTY, tz = lane / kTY;
  const bool row_ok = Y * kTY + ty < g.ny && Z * kTZ + tz < g.nz;
  for (int q = x0 + warp; q < x0 + kXC + kTY + kTZ - 2; q += nwarp) {
    const int x = q - ty - tz;
    if (row_ok && x >= x0 && x < x0 + kXC && x < g.nx)
      blk[lane][x - x0] = zs[((long long)tile * sk.ns + q + kPad) * kR + lane];
  }
  __syncthreads();
  // all of a thread's x values are loaded before any is written back (the
  // stores through xv would otherwise order every later load after them);
  // 256 threads
  T xo[kR / 8][kXC / 32];
#pragma unroll
  for (int rr = 0; rr < kR / 8; ++rr) {
    const int r = warp + rr * 8;
    const int y = Y * kTY + r % kTY, z = Z * kTZ + r / kTY;
#pragma unroll
    for (int hh = 0; hh < kXC / 32; ++hh) {
      const int x = x0 + lane + 32 * hh;
      xo[rr][hh] = (y < g.ny && z < g.nz && x < g.nx) ? xv[x + g.sy * y + g.sz * z] : T(0);
    }
  }
#pragma unroll
  for (int rr = 0; rr < kR / 8; ++rr) {
    const int r = warp + rr * 8;
    const int y = Y * kTY + r % kTY, z = Z * kTZ + r / kTY;
#pragma unroll
    for (int hh = 0; hh < kXC / 32; ++hh) {
      const int h = lane + 32 * hh, x = x0 + h;
      if (y < g.ny && z < g.nz && x < g.nx) xv[x + g.sy * y + g.sz * z] = xo[rr][hh] + blk[r][h];
    }
  }
}

inline dim3 transpose_grid(const Geo& g, const Skew& sk) {
  return dim3(sk.nty * sk.ntz, (g.nx + kXC - 1) / kXC);
}

template <class T>
__global__ void k_fill_not_ready(long long n, T* a, T* b) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  a[i] = not_ready<T>();
  if (b) b[i] = not_ready<T>();
}

// FP32 copy of the 7-point matrix (mixed precision)
__global__ void k_matrix_to_single(long long n, const double* __restrict__ Ad,
                                   const double* __restrict__ Ax, const double* __restrict__ Ay,
                                   const double* __restrict__ Az, float* sd, float* sx, float* sy,
                                   float* sz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  sd[i] = (float)Ad[i];
  sx[i] = (float)Ax[i];
  sy[i] = (float)Ay[i];
  sz[i] = (float)Az[i];
}

// FP32 copies of three arrays (the transposed couplings of a nonsymmetric A)
__global__ void k_three_to_single(long long n, const double* __restrict__ a,
                                  const double* __restrict__ b, const double* __restrict__ c,
                                  float* sa, float* sb, float* sc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  sa[i] = (float)a[i];
  sb[i] = (float)b[i];
  sc[i] = (float)c[i];
}

// Q_d[i] = a_{i,i-e_d} a_{i-e_d,i}: the pivot recurrence's products
template <class T>
__global__ void k_pivot_products(long long n, const T* __restrict__ Ax, const T* __restrict__ Ay,
                                 const T* __restrict__ Az, const T* __restrict__ Axu,
                                 const T* __restrict__ Ayu, const T* __restrict__ Azu, T* Qx,
                                 T* Qy, T* Qz) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Qx[i] = Ax[i] * Axu[i];
  Qy[i] = Ay[i] * Ayu[i];
  Qz[i] = Az[i] * Azu[i];
}

// p += delta (mixed precision: the FP32 correction enters the FP64 iterate)
__global__ void k_add_correction(long long n, const float* __restrict__ d, double* p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  p[i] += (double)d[i];
}

// ------------------------------------------------- per-cell operators ---
// Each sweep is "value = op(cell, operands, values of the three upstream
// neighbours)", with 0 standing for a neighbour outside the grid (its
// coupling is 0 as well).  src(a, i, j) is the address of operand a of the
// cell with natural index i and skewed index j; apply() combines the
// operands with the upstream values and publishes the result.  `cell` is
// false on the pipeline's fill/drain slots and on rows beyond the grid:
// there the result is discarded and nothing outside the slot is written.
//
// The two solves also keep the sentinels of the pipelined schedule: the
// forward sweep marks z "not computed" as it passes (the backward sweep that
// follows publishes into z), and the backward sweep does the same for w once
// it has consumed it (the next forward sweep publishes into w).
template <class T>
struct FwdSolve {   // w = rd - Lx w_{x-1} - Ly w_{y-1} - Lz w_{z-1}
  using Scalar = T;
  static constexpr int kN = 4;
  static constexpr bool kSkewIn = true, kSkewOut = true;
  const T *rd, *Lx, *Ly, *Lz;
  T *w, *z;
  __device__ __forceinline__ const T* src(int a, long long, long long j) const {
    return (a == 0 ? rd : a == 1 ? Lx : a == 2 ? Ly : Lz) + j;
  }
  __device__ __forceinline__ T apply(const T* in, long long, long long j, bool, T vx, T vy,
                                     T vz) const {
    const T v = fma(-in[1], vx, fma(-in[2], vy, fma(-in[3], vz, in[0])));
    publish(w + j, v);
    z[j] = not_ready<T>();
    return v;
  }
};

template <class T>
struct BwdSolve {   // z = w - Ux z_{x+1} - Uy z_{y+1} - Uz z_{z+1}  (x += z follows)
  using Scalar = T;
  static constexpr int kN = 4;
  static constexpr bool kSkewIn = true, kSkewOut = true;
  const T *Ux, *Uy, *Uz;
  T *w, *z;
  __device__ __forceinline__ const T* src(int a, long long, long long j) const {
    return (a == 0 ? w : a == 1 ? Ux : a == 2 ? Uy : Uz) + j;
  }
  __device__ __forceinline__ T apply(const T* in, long long, long long j, bool, T vx, T vy,
                                     T vz) const {
    const T v = fma(-in[1], vx, fma(-in[2], vy, fma(-in[3], vz, in[0])));
    publish(z + j, v);
    w[j] = not_ready<T>();
    return v;
  }
};

// d = a_ii - a_{i,x-1}^2 / d_{x-1} - a_{i,y-1}^2 / d_{y-1} - a_{i,z-1}^2 / d_{z-1};
// kProd: the operands are the products a_{i,i-e} a_{i-e,i} (nonsymmetric A)
template <class T, bool kProd = false>
struct Factor {
  using Scalar = T;
  static constexpr int kN = 4;
  static constexpr bool kSkewIn = false, kSkewOut = false;
  const T *Ad, *Ax, *Ay, *Az;
  T* dinv;
  int* status;
  __device__ __forceinline__ const T* src(int a, long long i, long long) const {
    return (a == 0 ? Ad : a == 1 ? Ax : a == 2 ? Ay : Az) + i;
  }
  __device__ __forceinline__ T apply(const T* in, long long i, long long, bool cell, T vx, T vy,
                                     T vz) const {
    T d = in[0];
    if constexpr (kProd) {
      d -= in[1] * vx;
      d -= in[2] * vy;
      d -= in[3] * vz;
    } else {
      d -= in[1] * in[1] * vx;
      d -= in[2] * in[2] * vy;
      d -= in[3] * in[3] * vz;
    }
    if (cell && (!(d != T(0)) || !isfinite(d))) {
      atomicOr(status, kStatSingular);
      d = T(1);
    }
    const T v = T(1) / d;
    if (cell) publish(dinv + i, v);
    return v;
  }
};

// ---------------------------------------------------- level schedule ---

template <class Op, bool kBackward>
__global__ void k_sweep_level(Geo g, Skew sk, int L, Op op, const typename Op::Scalar* vals) {
  using T = typename Op::Scalar;
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
  const long long j = skew_index(sk, x, yy, zz);
  T in[Op::kN];
#pragma unroll
  for (int a = 0; a < Op::kN; ++a) in[a] = *op.src(a, i, j);
  const int e = kBackward ? 1 : -1;
  const bool hx = kBackward ? x < g.nx - 1 : x > 0;
  const bool hy = kBackward ? yy < g.ny - 1 : yy > 0;
  const bool hz = kBackward ? zz < g.nz - 1 : zz > 0;
  auto at = [&](int dx, int dy, int dz) {
    return Op::kSkewOut ? vals[skew_index(sk, x + dx, yy + dy, zz + dz)]
                        : vals[i + dx + g.sy * dy + g.sz * dz];
  };
  op.apply(in, i, j, true, hx ? at(e, 0, 0) : T(0), hy ? at(0, e, 0) : T(0),
           hz ? at(0, 0, e) : T(0));
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

// Polls *p until it holds a published value; returns its bits, or the
// sentinel after an abort or a timeout (the status word and the abort flag
// are then set).  A light loop (one address, a short sleep between polls)
// for the long wait before a tile's first step: heavy polling there slows
// the tile's first steps and every tile downstream of it.
template <class T>
__device__ __forceinline__ typename Word<T>::U wait_bits(const T* p, int* abort_flag, int* status) {
  unsigned nap = 32;
  for (long long it = 0; it < kSpinLimit; ++it) {
    const typename Word<T>::U b = ld_relaxed(p);
    if (b != Word<T>::kNotReady) return b;
    if ((it & 63) == 63 && ld_relaxed_int(abort_flag)) return Word<T>::kNotReady;
    __nanosleep(nap);
    nap = nap < 256 ? 2 * nap : 256;      // back off while the upstream tile is far away
  }
  atomicOr(status, kStatTimeout);
  atomicExch(abort_flag, 1);
  return Word<T>::kNotReady;
}

// Shared-memory edge values between the warps of one CTA (volatile: every
// access is performed; aligned 4- and 8-byte accesses are single-copy atomic).
template <class T>
__device__ __forceinline__ typename Word<T>::U ld_shared_bits(const T* p) {
  return *reinterpret_cast<const volatile typename Word<T>::U*>(p);
}
template <class T>
__device__ __forceinline__ void st_shared(T* p, T v) {
  *reinterpret_cast<volatile T*>(p) = v;
}

// wait_bits for a value another warp of this CTA writes into shared memory
template <class T>
__device__ __forceinline__ typename Word<T>::U wait_shared(const T* p, int* abort_flag,
                                                          int* status) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    const typename Word<T>::U b = ld_shared_bits(p);
    if (b != Word<T>::kNotReady) return b;
    if ((it & 63) == 63) {
      if (ld_relaxed_int(abort_flag)) return Word<T>::kNotReady;
      __nanosleep(20);
    }
  }
  atomicOr(status, kStatTimeout);
  atomicExch(abort_flag, 1);
  return Word<T>::kNotReady;
}

// One tile of a sweep, run by one warp: the tile at (Ym, Zm) in the sweep
// frame (mirrored for the backward sweep).  ringw, bars, phase: this warp's
// operand ring, its slot barriers and their phase bits (kept across tiles).
// Values from other tiles are read from `out`.  Before its first step the
// tile waits (lightly) for the upstream values of its first group; steps
// then run in groups of kU: a group's prologue stages the operands of the
// group kG - 1 ahead and prefetches the next group's cross-tile
// values; values still unset are re-polled together; the kU steps
// themselves are straight-line code.  Returns false after an abort or a
// timeout (the warp's copies drained).
//
// With kCta, the upstream tile in y (z) may be run by another warp of the
// same CTA: then ey (ez) is this lane's shared-memory edge buffer, indexed
// by x in the sweep frame, which that warp fills; py / pz are the edge
// buffers this lane fills for the downstream warps of the CTA (null: none).
template <class Op, bool kBackward, bool kCta = false>
__device__ __forceinline__ bool sweep_tile(const Geo& g, const Skew& sk, const Op& op,
                                           const typename Op::Scalar* out, int* abort_flag,
                                           int* status, typename Op::Scalar* ringw,
                                           uint64_t* bars, uint32_t& phase, int lane, int Ym,
                                           int Zm, const typename Op::Scalar* ey = nullptr,
                                           const typename Op::Scalar* ez = nullptr,
                                           typename Op::Scalar* py = nullptr,
                                           typename Op::Scalar* pz = nullptr) {
  using T = typename Op::Scalar;
  using U = typename Word<T>::U;
  constexpr U kNR = Word<T>::kNotReady;
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int kN = Op::kN;
  const int tym = lane % kTY, tzm = lane / kTY;   // row within the tile, sweep frame
  const int ty = kBackward ? kTY - 1 - tym : tym, tz = kBackward ? kTZ - 1 - tzm : tzm;
  const int slot = ty + kTY * tz;                 // my slot of a record
  const long long rec = (long long)sk.ns * kR;    // one tile's records
  const long long dj = kBackward ? -kR : kR;      // skewed index change per step
  const long long di = kBackward ? -1 : 1;        // natural index change per step
  // cross-tile neighbour of an edge row, relative to my own index
  const long long offy_s = (kBackward ? 1 : -1) * (rec - (long long)(kTY - 1) * (kR + 1));
  const long long offz_s =
      (kBackward ? 1 : -1) * ((long long)sk.nty * rec - (long long)(kTZ - 1) * (kR + kTY));
  const long long offy_n = kBackward ? g.sy : -g.sy, offz_n = kBackward ? g.sz : -g.sz;
  const int Y = kBackward ? sk.nty - 1 - Ym : Ym, Z = kBackward ? sk.ntz - 1 - Zm : Zm;
  const int y = Y * kTY + ty, z = Z * kTZ + tz;
  const bool valid = y < g.ny && z < g.nz;
  const bool hy = valid && (kBackward ? y < g.ny - 1 : y > 0);   // upstream rows exist
  const bool hz = valid && (kBackward ? z < g.nz - 1 : z > 0);
  const bool ext_y = hy && tym == 0;                              // ... in another tile
  const bool ext_z = hz && tzm == 0;
  const bool sy = kCta && ext_y && ey != nullptr;                 // ... another warp of my CTA
  const bool sz = kCta && ext_z && ez != nullptr;
  const bool gy = ext_y && !sy, gz = ext_z && !sz;                // ... another CTA (via L2)
  // indices at sweep step 0.  x in the sweep frame is step - xoff; the
  // backward sweep walks the tile's records from the last one down, and its
  // first ns - (nx + kTY + kTZ - 2) steps are padding.
  const int xoff = tym + tzm + (kBackward ? sk.ns - (g.nx + kTY + kTZ - 2) : 0);
  const long long j0 =
      ((long long)(Y + sk.nty * Z) * sk.ns + (kBackward ? sk.ns - 1 : 0) + kPad) * kR + slot;
  const int yc = valid ? y : 0, zc = valid ? z : 0;               // rows beyond the grid read row 0
  const long long row = (long long)yc * g.sy + (long long)zc * g.sz;
  const long long i0 = row + (kBackward ? g.nx - 1 + xoff : -xoff);
  const long long o0 = Op::kSkewOut ? j0 : i0;
  const long long od = Op::kSkewOut ? dj : di;
  const long long oy0 = o0 + (Op::kSkewOut ? offy_s : offy_n);
  const long long oz0 = o0 + (Op::kSkewOut ? offz_s : offz_n);
  // Operands of steps gs .. gs+kU-1 into ring slot q, laid out
  // [slot][operand][step][lane].  Skewed operands (the solves'): the group's
  // kU records of one operand are contiguous, so one lane issues a bulk copy
  // per operand (the TMA engine, completing on the slot's mbarrier; the
  // backward sweep's records arrive in reverse step order).  Bulk copies do
  // not queue in front of the cross-tile loads of the critical path the way
  // per-lane copies do.  Groups past the tile are not staged (nor waited
  // for).  Natural operands (the factorisation's): per-lane cp.async,
  // clamped to my row (read, then discarded).
  constexpr bool kBulk = Op::kSkewIn && kBulkStage;
  T* const ring = ringw + lane;                    // where my cp.async copies land
  const T* const ring_rd = ringw + (kBulk ? slot : lane);   // a bulk copy keeps record order
  const long long jr0 = j0 - slot;                 // record of step 0
  int issued = -1;                                 // last group staged (bulk)
  auto stage = [&](int gs, int q) {
    if constexpr (kBulk) {
      if (gs >= sk.ns) return;
      __syncwarp();                                // the slot's previous reads are done
      if (lane == 0) {
        tc::mbar_arrive_expect_tx(bars + q, (uint32_t)(kN * kU * kR * sizeof(T)));
        const long long rs = kBackward ? jr0 - (long long)(gs + kU - 1) * kR : jr0 + (long long)gs * kR;
#pragma unroll
        for (int a = 0; a < kN; ++a)
          tc::bulk_g2s(ringw + (q * kN + a) * kU * kR, op.src(a, 0, rs),
                       (uint32_t)(kU * kR * sizeof(T)), bars + q);
      }
      issued = gs / kU;
    } else {
      if (gs >= sk.ns) {                           // past the tile: an empty group
        cp_async_commit();
        return;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        long long i = i0 + (gs + u) * di;
        i = i < row ? row : i;
        i = i > row + g.nx - 1 ? row + g.nx - 1 : i;
        const long long j = j0 + (gs + u) * dj;
#pragma unroll
        for (int a = 0; a < kN; ++a) cp_async(ring + ((q * kN + a) * kU + u) * kR, op.src(a, i, j));
      }
      cp_async_commit();
    }
  };
  // the operands of group gq (slot gq % kG) have landed; false after a timeout
  auto landed = [&](int gq) -> bool {
    if constexpr (kBulk) {
      const int q = gq % kG;
      if (!tc::mbar_wait(bars + q, (phase >> q) & 1u, kSpinLimit)) {
        if (lane == 0) {
          atomicOr(status, kStatTimeout);
          atomicExch(abort_flag, 1);
        }
        return false;
      }
      phase ^= 1u << q;
    } else {
      cp_async_wait<kG - 1>();
    }
    return true;
  };
  // before leaving early: wait (bounded) for the copies still in flight
  auto drain = [&](int next) {
    if constexpr (kBulk) {
      for (int gq = next; gq <= issued; ++gq)
        if (!landed(gq)) break;
    } else {
      cp_async_wait<0>();
    }
  };
  // values of steps gs .. gs+kU-1 read from `out` (0 where none is needed)
  auto fetch = [&](int gs, U* cy, U* cz) {
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int xq = gs + u - xoff;
      const bool in_row = xq >= 0 && xq < g.nx;
      cy[u] = ld_relaxed_if(gy && in_row, out + oy0 + (gs + u) * od);
      cz[u] = ld_relaxed_if(gz && in_row, out + oz0 + (gs + u) * od);
    }
  };
  // skewed operands of the group at step gs into L2 (the TMA engine; no
  // completion to wait for)
  auto l2_prefetch = [&](int gs) {
    if (gs >= sk.ns || lane != 0) return;
    const long long rs = kBackward ? jr0 - (long long)(gs + kU - 1) * kR : jr0 + (long long)gs * kR;
#pragma unroll
    for (int a = 0; a < kN; ++a)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(op.src(a, 0, rs)),
                   "r"((uint32_t)(kU * kR * sizeof(T)))
                   : "memory");
  };
  if constexpr (kL2Ahead > 0 && Op::kSkewIn) {
#pragma unroll 1
    for (int gq = kG - 1; gq < kL2Ahead; ++gq) l2_prefetch(gq * kU);
  }
  // the operands of the first kG - 1 groups do not depend on other tiles:
  // their copies overlap the first wait
#pragma unroll 1
  for (int gq = 0; gq < kG - 1; ++gq) stage(gq * kU, gq);
  {
    // The first group's upstream values (the first wait is the long one).
    // A tile publishes in step order, and among my edge lanes the one with
    // the largest skew needs the latest value, so that lane alone polls for
    // each direction (tz = 3 in y, ty = 7 in z): few pollers keep L2 quiet
    // for the tiles that are running.
    // (Every lane takes part in both shuffles.)
    const int xq = kU - 1 - xoff;
    bool ok = true;
    const bool in_row = xq >= 0 && xq < g.nx;
    const bool need_y = ext_y && in_row, need_z = ext_z && in_row;
    const bool des_y = __shfl_sync(kAll, need_y, tym + (kTZ - 1) * kTY);   // tz = 3 of my column
    const bool des_z = __shfl_sync(kAll, need_z, (kTY - 1) + tzm * kTY);   // ty = 7 of my row
    const bool last_y = tzm == kTZ - 1 || !des_y;
    const bool last_z = tym == kTY - 1 || !des_z;
    if (gy && in_row && last_y) ok &= wait_bits(out + oy0 + (kU - 1) * od, abort_flag, status) != kNR;
    if (gz && in_row && last_z) ok &= wait_bits(out + oz0 + (kU - 1) * od, abort_flag, status) != kNR;
    if (kCta && sy && in_row && last_y) ok &= wait_shared(ey + xq, abort_flag, status) != kNR;
    if (kCta && sz && in_row && last_z) ok &= wait_shared(ez + xq, abort_flag, status) != kNR;
    if (__any_sync(kAll, !ok)) {
      drain(0);
      return false;
    }
  }
  U cy[kU], cz[kU];
  fetch(0, cy, cz);
  T vprev = T(0), from_y = T(0), from_z = T(0);
  int q = 0;
  for (int s0 = 0; s0 < sk.ns; s0 += kU) {
    U ny_[kU], nz_[kU];
    if constexpr (kFetchFirst) fetch(s0 + kU, ny_, nz_);
    if constexpr (kL2Ahead > 0 && Op::kSkewIn) l2_prefetch(s0 + kL2Ahead * kU);
    stage(s0 + (kG - 1) * kU, q == 0 ? kG - 1 : q - 1);
    if constexpr (!kFetchFirst) fetch(s0 + kU, ny_, nz_);
    if (kCta && (sy || sz)) {   // edge values of this group from my CTA's shared memory
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int xq = s0 + u - xoff;
        const bool in_row = xq >= 0 && xq < g.nx;
        if (sy) cy[u] = in_row ? ld_shared_bits(ey + xq) : U(0);
        if (sz) cz[u] = in_row ? ld_shared_bits(ez + xq) : U(0);
      }
    }
    // values still unset: re-poll them together (one round trip per poll)
    bool pending = false;
#pragma unroll
    for (int u = 0; u < kU; ++u) pending |= (cy[u] == kNR) | (cz[u] == kNR);
    if (__any_sync(kAll, pending)) {
      bool fail = false;
      for (long long it = 0; pending && !fail; ++it) {
        pending = false;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          if (cy[u] == kNR) {
            cy[u] = sy ? ld_shared_bits(ey + (s0 + u - xoff)) : ld_relaxed(out + oy0 + (s0 + u) * od);
            pending |= cy[u] == kNR;
          }
          if (cz[u] == kNR) {
            cz[u] = sz ? ld_shared_bits(ez + (s0 + u - xoff)) : ld_relaxed(out + oz0 + (s0 + u) * od);
            pending |= cz[u] == kNR;
          }
        }
        if (pending && it >= kFastPolls) {
          if (it >= kSpinLimit) {
            atomicOr(status, kStatTimeout);
            atomicExch(abort_flag, 1);
            fail = true;
          } else if ((it & 15) == 0 && ld_relaxed_int(abort_flag)) {
            fail = true;
          } else {
            __nanosleep(100);
          }
        }
      }
      if (__any_sync(kAll, fail)) {
        drain(s0 / kU);
        return false;
      }
    }
    if constexpr (kBulk) {
      if (!__all_sync(kAll, landed(s0 / kU))) {
        drain(s0 / kU + 1);
        return false;
      }
    } else {
      cp_async_wait<kG - 1>();
    }
    T in[kU][kN];
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int a = 0; a < kN; ++a)
        in[u][a] = ring_rd[((q * kN + a) * kU + (kBulk && kBackward ? kU - 1 - u : u)) * kR];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int s = s0 + u;
      const int xs = s - xoff;
      const bool cell = valid && xs >= 0 && xs < g.nx;
      const T vy = hy ? (tym > 0 ? from_y : Word<T>::value(cy[u])) : T(0);
      const T vz = hz ? (tzm > 0 ? from_z : Word<T>::value(cz[u])) : T(0);
      const T vx = xs > 0 ? vprev : T(0);
      const T v = op.apply(in[u], i0 + s * di, j0 + s * dj, cell, vx, vy, vz);
      if (kCta) {   // feed the downstream warps of my CTA
        if (py != nullptr && cell) st_shared(py + xs, v);
        if (pz != nullptr && cell) st_shared(pz + xs, v);
      }
      // rows y-1 / z-1 of my tile computed my next neighbours just now
      from_y = __shfl_up_sync(kAll, v, 1);
      from_z = __shfl_up_sync(kAll, v, kTY);
      vprev = v;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      cy[u] = ny_[u];
      cz[u] = nz_[u];
    }
    q = q == kG - 1 ? 0 : q + 1;
  }
  if constexpr (!kBulk) cp_async_wait<0>();   // (every bulk group staged was waited for)
  return true;
}

// Shared memory of the sweep kernels: the warps' operand rings
// [kWarps][kG][Op::kN][kU][32], then one mbarrier per ring slot
// [kWarps][kG] (then, in k_sweep_cta, the edge buffers).
template <class Op>
constexpr int ring_bytes() {
  return (int)sizeof(typename Op::Scalar) * kWarps * kG * Op::kN * kU * kR;
}
constexpr int bar_bytes() { return (int)sizeof(uint64_t) * kWarps * kG; }

// This warp's ring and slot barriers (initialised: one arrival each).
template <class Op>
__device__ __forceinline__ void warp_ring(unsigned char* smem_raw, int warp, int lane,
                                          typename Op::Scalar*& ringw, uint64_t*& bars) {
  ringw = reinterpret_cast<typename Op::Scalar*>(smem_raw) + warp * (kG * Op::kN * kU * kR);
  bars = reinterpret_cast<uint64_t*>(smem_raw + ring_bytes<Op>()) + warp * kG;
  if (lane == 0) {
    for (int q = 0; q < kG; ++q) tc::mbar_init(bars + q, 1);
    tc::fence_proxy_async();
  }
  __syncwarp();
}

// ctrl: [0] ticket, [1] abort flag.  `out` is the vector the operator
// publishes into (pre-filled with the sentinel on every cell).  Each warp
// claims tiles on its own.
template <class Op, bool kBackward>
__global__ void __launch_bounds__(32 * kWarps, 1) k_sweep_warp(Geo g, Skew sk, Op op,
                                                                const typename Op::Scalar* out,
                                                                int* ctrl, int* status) {
  using T = typename Op::Scalar;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* ringw;
  uint64_t* bars;
  warp_ring<Op>(smem_raw, warp, lane, ringw, bars);
  uint32_t phase = 0;
  const int ntiles = sk.nty * sk.ntz;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&ctrl[0], 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) return;
    int Ym, Zm;
    tile_of_ticket(t, sk.nty, sk.ntz, Ym, Zm);
    if (!sweep_tile<Op, kBackward>(g, sk, op, out, ctrl + 1, status, ringw, bars, phase, lane, Ym,
                                   Zm))
      return;
  }
}

// The 4 warps of a CTA take a 2 x 2 block of tiles (16 x 8 x-rows) together:
// warp w runs tile (2 CY + (w & 1), 2 CZ + (w >> 1)) of CTA block (CY, CZ)
// in the sweep frame.  Edges between the block's tiles pass through shared
// memory (12 buffers of nx values per warp pair, kNotReady until written);
// edges between blocks pass through L2 as in k_sweep_warp.  Blocks are
// claimed by ticket in anti-diagonal order; a CTA resets its edge buffers
// between blocks.  Shared memory: the operand rings, then the edges:
// [2 (block column wz)][4 (tz)][nx] in y, then [2 (wy)][8 (ty)][nx] in z.
template <class Op, bool kBackward>
__global__ void __launch_bounds__(32 * kWarps, 1) k_sweep_cta(Geo g, Skew sk, Op op,
                                                               const typename Op::Scalar* out,
                                                               int* ctrl, int* status) {
  static_assert(kWarps == 4, "a CTA block is 2 x 2 tiles");
  using T = typename Op::Scalar;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_ticket;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tym = lane % kTY, tzm = lane / kTY;
  const int wy = warp & 1, wz = warp >> 1;
  T* ringw;
  uint64_t* bars;
  warp_ring<Op>(smem_raw, warp, lane, ringw, bars);
  uint32_t phase = 0;
  T* edges = reinterpret_cast<T*>(smem_raw + ring_bytes<Op>() + bar_bytes());
  const long long nx = g.nx;
  T* ey_row = edges + (wz * kTZ + tzm) * nx;                  // y-edge of block column wz, row tz
  T* ez_row = edges + 2 * kTZ * nx + (wy * kTY + tym) * nx;    // z-edge of block row wy, row ty
  const T* ey = wy == 1 ? ey_row : nullptr;                     // I read what warp (0, wz) writes
  const T* ez = wz == 1 ? ez_row : nullptr;                     // ... what warp (wy, 0) writes
  T* py = (wy == 0 && tym == kTY - 1) ? ey_row : nullptr;
  T* pz = (wz == 0 && tzm == kTZ - 1) ? ez_row : nullptr;
  const int ncy = (sk.nty + 1) / 2, ncz = (sk.ntz + 1) / 2, nblocks = ncy * ncz;
  const int nedge = 2 * (kTZ + kTY) * g.nx;
  for (;;) {
    if (threadIdx.x == 0) {
      int t = atomicAdd(&ctrl[0], 1);
      if (ld_relaxed_int(ctrl + 1)) t = nblocks;   // after an abort: stop
      s_ticket = t;
    }
    __syncthreads();
    const int t = s_ticket;
    if (t >= nblocks) return;
    for (int e = threadIdx.x; e < nedge; e += blockDim.x) edges[e] = not_ready<T>();
    __syncthreads();
    int CY, CZ;
    tile_of_ticket(t, ncy, ncz, CY, CZ);
    const int Ym = 2 * CY + wy, Zm = 2 * CZ + wz;
    if (Ym < sk.nty && Zm < sk.ntz)
      sweep_tile<Op, kBackward, true>(g, sk, op, out, ctrl + 1, status, ringw, bars, phase, lane,
                                      Ym, Zm, ey, ez, py, pz);
    // a warp that failed falls through: the others see the abort flag in
    // their waits, and the next claim ends the CTA
    __syncthreads();
  }
}

// Bounded wait used by the self-test: polls a counter that nothing sets.
__device__ __forceinline__ bool wait_at_least(int* ctr, int need, int* abort_flag, int* status) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    if (ld_relaxed_int(ctr) >= need) return true;
    if (ld_relaxed_int(abort_flag)) return false;
    __nanosleep(64);
  }
  atomicOr(status, kStatTimeout);
  atomicExch(abort_flag, 1);
  return false;
}

__global__ void k_wait_selftest(int* ctrl, int* status) {
  if (threadIdx.x == 0) wait_at_least(&ctrl[2], 1, &ctrl[1], status);
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

template <class Op>
constexpr int warp_smem() {
  return ring_bytes<Op>() + bar_bytes();
}

template <class Op>
int cta_smem(const Geo& g) {
  return warp_smem<Op>() + (int)sizeof(typename Op::Scalar) * 2 * (kTZ + kTY) * g.nx;
}

// sms: the device's SM count; cta: run k_sweep_cta (else k_sweep_warp).
// One CTA per SM: more sweeping warps per SM would share the FP64 pipes.
template <class Op, bool kBackward>
cudaError_t launch_sweep(const Geo& g, const Skew& sk, int sms, bool cta, const Op& op,
                         const typename Op::Scalar* out, Buffers& b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.ctrl, 0, sizeof(int) * (size_t)ilu_ctrl_ints(g), s);
  if (e != cudaSuccess) return e;
  if (cta) {
    const int blocks = ((sk.nty + 1) / 2) * ((sk.ntz + 1) / 2);
    k_sweep_cta<Op, kBackward><<<blocks < sms ? blocks : sms, 32 * kWarps, cta_smem<Op>(g), s>>>(
        g, sk, op, out, b.ctrl, b.status);
  } else {
    const int ctas = (sk.nty * sk.ntz + kWarps - 1) / kWarps;
    k_sweep_warp<Op, kBackward><<<ctas < sms ? ctas : sms, 32 * kWarps, warp_smem<Op>(), s>>>(
        g, sk, op, out, b.ctrl, b.status);
  }
  return cudaGetLastError();
}

template <class Op, bool kBackward>
void set_sweep_smem() {
  raise_smem_limit(k_sweep_warp<Op, kBackward>, warp_smem<Op>());
}

template <class Op, bool kBackward>
bool set_cta_smem(const Geo& g) {
  return raise_smem_limit(k_sweep_cta<Op, kBackward>, cta_smem<Op>(g)) == cudaSuccess;
}

// The vectors of one precision's smoother.
template <class T>
struct IluSet {
  const T *Ad, *Ax, *Ay, *Az;
  const T *Axu, *Ayu, *Azu;
  T *Qx, *Qy, *Qz;
  T* dinv;
  T *Lx, *Ly, *Lz, *Ux, *Uy, *Uz;
  T *rds, *w, *z;
};

IluSet<double> set_of(Buffers& b, double*) {
  return IluSet<double>{b.Ad,   b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, b.Qx, b.Qy, b.Qz,
                        b.dinv, b.Lx, b.Ly, b.Lz, b.Ux,  b.Uy,  b.Uz,  b.rds, b.w, b.z};
}
IluSet<float> set_of(Buffers& b, float*) {
  const SingleBuffers& f = b.f32;
  return IluSet<float>{f.Ad,   f.Ax, f.Ay, f.Az, f.Axu, f.Ayu, f.Azu, f.Qx, f.Qy, f.Qz,
                       f.dinv, f.Lx, f.Ly, f.Lz, f.Ux,  f.Uy,  f.Uz,  f.rds, f.w, f.z};
}

// The pivot sweep (level-scheduled or pipelined); returns the launch count.
template <class Op>
int factor_sweep(const Geo& g, const Skew& sk, Buffers& b, bool pipelined, int sms, bool cta,
                 const Op& fa, typename Op::Scalar* dinv, cudaStream_t s, cudaError_t& e) {
  using T = typename Op::Scalar;
  e = cudaSuccess;
  if (!pipelined) {
    const int blocks = blocks_for((long long)g.ny * g.nz, 256);
    const int levels = g.nx + g.ny + g.nz - 2;
    for (int L = 0; L < levels; ++L)
      k_sweep_level<Op, false><<<blocks, 256, 0, s>>>(g, sk, L, fa, dinv);
    return levels;
  }
  k_fill_not_ready<T><<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, dinv, nullptr);
  e = launch_sweep<Op, false>(g, sk, sms, cta, fa, dinv, b, s);
  return 2;
}

template <class T>
cudaError_t factor_impl(const Geo& g, Buffers& b, bool pipelined, int sms, bool cta, bool nonsym,
                        cudaStream_t s) {
  const Skew sk = make_skew(g);
  const IluSet<T> v = set_of(b, (T*)nullptr);
  int n = 1;
  cudaError_t e;
  if (nonsym) {
    k_pivot_products<T><<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, v.Ax, v.Ay, v.Az, v.Axu, v.Ayu,
                                                             v.Azu, v.Qx, v.Qy, v.Qz);
    ++n;
    Factor<T, true> fa{v.Ad, v.Qx, v.Qy, v.Qz, v.dinv, b.status};
    n += factor_sweep(g, sk, b, pipelined, sms, cta, fa, v.dinv, s, e);
  } else {
    Factor<T> fa{v.Ad, v.Ax, v.Ay, v.Az, v.dinv, b.status};
    n += factor_sweep(g, sk, b, pipelined, sms, cta, fa, v.dinv, s, e);
  }
  if (e != cudaSuccess) return e;
  if (pipelined) {
    // sweep outputs start "not computed"; the sweeps keep it so from here on
    const long long S = ilu_skew_len(g);
    k_fill_not_ready<T><<<blocks_for(S, 256), 256, 0, s>>>(S, v.w, v.z);
    ++n;
  }
  k_ilu_scale<T><<<blocks_for(g.N, 256), 256, 0, s>>>(g, sk, v.Ax, v.Ay, v.Az, v.Axu, v.Ayu,
                                                      v.Azu, v.dinv, v.Lx, v.Ly, v.Lz, v.Ux,
                                                      v.Uy, v.Uz);
  count_launches(n);
  return cudaGetLastError();
}

template <class T>
cudaError_t sweep_impl(const Geo& g, Buffers& b, bool backward, bool pipelined, int sms, bool cta,
                       T* xv, cudaStream_t s) {
  const Skew sk = make_skew(g);
  const IluSet<T> v = set_of(b, (T*)nullptr);
  FwdSolve<T> fw{v.rds, v.Lx, v.Ly, v.Lz, v.w, v.z};
  BwdSolve<T> bw{v.Ux, v.Uy, v.Uz, v.w, v.z};
  if (!pipelined) {
    const int blocks = blocks_for((long long)g.ny * g.nz, 256);
    const int levels = g.nx + g.ny + g.nz - 2;
    for (int L = 0; L < levels; ++L) {
      if (!backward) k_sweep_level<FwdSolve<T>, false><<<blocks, 256, 0, s>>>(g, sk, L, fw, v.w);
      else k_sweep_level<BwdSolve<T>, true><<<blocks, 256, 0, s>>>(g, sk, L, bw, v.z);
    }
    count_launches(levels);
  } else {
    cudaError_t e = !backward ? launch_sweep<FwdSolve<T>, false>(g, sk, sms, cta, fw, v.w, b, s)
                              : launch_sweep<BwdSolve<T>, true>(g, sk, sms, cta, bw, v.z, b, s);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  (void)xv;
  return cudaGetLastError();
}

template <class T>
cudaError_t apply_impl(const Geo& g, Buffers& b, T* xv, cudaStream_t s) {
  const Skew sk = make_skew(g);
  const IluSet<T> v = set_of(b, (T*)nullptr);
  k_apply_z<T><<<transpose_grid(g, sk), 256, 0, s>>>(g, sk, v.z, xv);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

long long ilu_skew_len(const Geo& g) {
  const Skew k = make_skew(g);
  return ((long long)k.nty * k.ntz * k.ns + 2 * kPad) * kR;
}

int ilu_ctrl_ints(const Geo& g) {
  (void)g;
  return 4;                                    // ticket, abort flag, self-test counter
}

int ilu_pipe_grid(const Geo& g, int num_sms) {
  (void)g;
  set_sweep_smem<FwdSolve<double>, false>();
  set_sweep_smem<BwdSolve<double>, true>();
  set_sweep_smem<Factor<double>, false>();
  set_sweep_smem<FwdSolve<float>, false>();
  set_sweep_smem<BwdSolve<float>, true>();
  set_sweep_smem<Factor<float>, false>();
  set_sweep_smem<Factor<double, true>, false>();
  set_sweep_smem<Factor<float, true>, false>();
  return num_sms;
}

bool ilu_cta_ok(const Geo& g, int max_smem) {
  if (cta_smem<FwdSolve<double>>(g) > max_smem) return false;   // FP64 needs the most
  bool ok = set_cta_smem<FwdSolve<double>, false>(g) && set_cta_smem<BwdSolve<double>, true>(g) &&
            set_cta_smem<Factor<double>, false>(g) && set_cta_smem<FwdSolve<float>, false>(g) &&
            set_cta_smem<BwdSolve<float>, true>(g) && set_cta_smem<Factor<float>, false>(g) &&
            set_cta_smem<Factor<double, true>, false>(g) &&
            set_cta_smem<Factor<float, true>, false>(g);
  cudaGetLastError();
  return ok;
}

cudaError_t launch_ilu_factor(const Geo& g, Buffers& b, bool pipelined, int sms, bool cta,
                              bool single, bool nonsym, cudaStream_t s) {
  if (single) {
    k_matrix_to_single<<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, b.Ad, b.Ax, b.Ay, b.Az, b.f32.Ad,
                                                            b.f32.Ax, b.f32.Ay, b.f32.Az);
    count_launches(1);
    if (nonsym) {
      k_three_to_single<<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, b.Axu, b.Ayu, b.Azu, b.f32.Axu,
                                                             b.f32.Ayu, b.f32.Azu);
      count_launches(1);
    }
    return factor_impl<float>(g, b, pipelined, sms, cta, nonsym, s);
  }
  return factor_impl<double>(g, b, pipelined, sms, cta, nonsym, s);
}

cudaError_t launch_ilu_resid(const Geo& g, Buffers& b, bool single, cudaStream_t s) {
  const Skew sk = make_skew(g);
  if (single) {
    const SingleBuffers& f = b.f32;
    // b = the outer residual's FP32 copy (written with it by launch_residual)
    if (f.Axu != f.Ax)
      k_resid_scaled<float, float, true><<<transpose_grid(g, sk), 256, 0, s>>>(
          g, sk, f.Ad, f.Ax, f.Ay, f.Az, f.Axu, f.Ayu, f.Azu, f.r, f.d, f.dinv, f.rds);
    else
      k_resid_scaled<float, float, false><<<transpose_grid(g, sk), 256, 0, s>>>(
          g, sk, f.Ad, f.Ax, f.Ay, f.Az, f.Axu, f.Ayu, f.Azu, f.r, f.d, f.dinv, f.rds);
  } else {
    if (b.Axu != b.Ax)
      k_resid_scaled<double, double, true><<<transpose_grid(g, sk), 256, 0, s>>>(
          g, sk, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, b.f, b.p, b.dinv, b.rds);
    else
      k_resid_scaled<double, double, false><<<transpose_grid(g, sk), 256, 0, s>>>(
          g, sk, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, b.f, b.p, b.dinv, b.rds);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ilu_sweep(const Geo& g, Buffers& b, bool backward, bool pipelined, int sms,
                             bool cta, bool single, cudaStream_t s) {
  return single ? sweep_impl<float>(g, b, backward, pipelined, sms, cta, b.f32.d, s)
                : sweep_impl<double>(g, b, backward, pipelined, sms, cta, b.p, s);
}

cudaError_t launch_ilu_apply(const Geo& g, Buffers& b, bool single, cudaStream_t s) {
  return single ? apply_impl<float>(g, b, b.f32.d, s) : apply_impl<double>(g, b, b.p, s);
}

cudaError_t launch_add_correction(const Geo& g, Buffers& b, cudaStream_t s) {
  k_add_correction<<<blocks_for(g.N, 256), 256, 0, s>>>(g.N, b.f32.d, b.p);
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

}  // namespace cams
