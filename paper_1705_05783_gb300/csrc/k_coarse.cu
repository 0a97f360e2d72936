// Coarse-scale kernels of Sec. 3: Galerkin operator R A P (Eq. 13) for MSFE
// (R = P^T) and MSFV (Eq. 7), restriction R r, coarse direct solve and
// prolongation P p_c (Eqs. 12, 15).
//
// P is stored per fine cell as 8 slots (slot-major arrays); slot bit d says
// whether the coarse node is the lower (0) or upper (1) one along d among the
// nodes spanning the cell's dual block (a cell on a vertex plane of d uses
// bit 0 for that plane's node and never bit 1).
//
// P is FP64, or FP32 in the mixed-precision preconditioner; products with P
// are formed and summed in FP64 either way.
//
// Deterministic reductions only: every sum over fine cells is a fixed-shape
// block tree, and every sum over blocks runs in a fixed block order, so the
// MSFE matrix is bitwise symmetric.
#include "cams_internal.h"
#include "rcp64.h"

namespace cams {

namespace {

__device__ __forceinline__ int nd_of(const Geo& g, int d) { return d == 0 ? g.nx : (d == 1 ? g.ny : g.nz); }
__device__ __forceinline__ long long sd_of(const Geo& g, int d) { return d == 0 ? 1 : (d == 1 ? g.sy : g.sz); }

// Coarse node index along d of the cell coordinate x for slot bit `bit`
// (-1 when that node does not exist).
__device__ __forceinline__ int corner_d(const CGeo& c, int d, int x, int bit) {
  const int b = c.b[d], o = c.o[d], s = x - o;
  int J;
  if (s >= 0 && s % b == 0) J = bit ? -1 : s / b;          // on a vertex plane
  else {
    const int j = s >= 0 ? s / b + 1 : 0;                   // interval index
    J = bit ? j : j - 1;
  }
  return (J >= 0 && J < c.nc[d]) ? J : -1;
}

// Cell range [lo, hi] along d of dual block index j (0..nc): the cells from
// the lower vertex plane (inclusive) to the upper one (exclusive).
__device__ __forceinline__ void dual_range(const CGeo& c, const Geo& g, int d, int j, int& lo, int& hi) {
  const int n = nd_of(g, d);
  lo = j == 0 ? 0 : (j - 1) * c.b[d] + c.o[d];
  hi = j == c.nc[d] ? n - 1 : j * c.b[d] + c.o[d] - 1;
}

// Warp sums in the accumulation type TA, the sum over warps in FP64.
template <int K, class TA>
__device__ void block_sum_k(TA (&v)[K], double* sh /* K*32 */, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (sizeof(TA) == 4) {
    // FP32 sums: lane k % 32 collects sum k, so that each warp converts its
    // sums to FP64 in ceil(K / 32) instructions instead of K (a conversion is
    // an FP64-unit instruction, as slow with one active lane as with 32)
    constexpr int kW = (K + 31) / 32;
    TA mine[kW];
#pragma unroll
    for (int w = 0; w < kW; ++w) mine[w] = TA(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      TA t = v[k];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (lane == k % 32) mine[k / 32] = t;
    }
#pragma unroll
    for (int w = 0; w < kW; ++w)
      if (32 * w + lane < K) sh[(32 * w + lane) * 32 + wid] = (double)mine[w];
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      TA t = v[k];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) sh[k * 32 + wid] = (double)t;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[k * 32 + w];
    out[k] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ int sym_idx(int s, int t) {   // upper triangle of 8x8, s <= t
  return s * 8 - (s * (s - 1)) / 2 + (t - s);
}

// A = sum over the coupled faces of w_f (e_i - e_j)(e_i - e_j)^T + diag(D):
// D_i is the row sum of A (the accumulation term, the Dirichlet faces and,
// for a free cell, the faces to prescribed cells; 1 on a prescribed row).
// Axu.. hold the couplings to the upper neighbours (the same arrays as
// Ax.. for a symmetric A).
__device__ __forceinline__ double row_sum(const Geo& g, const double* __restrict__ Ad,
                                          const double* __restrict__ Ax,
                                          const double* __restrict__ Ay,
                                          const double* __restrict__ Az,
                                          const double* __restrict__ Axu,
                                          const double* __restrict__ Ayu,
                                          const double* __restrict__ Azu, long long i, int x, int y,
                                          int z) {
  double s = Ad[i] + Ax[i] + Ay[i] + Az[i];
  if (x < g.nx - 1) s += Axu[i + 1];
  if (y < g.ny - 1) s += Ayu[i + g.sy];
  if (z < g.nz - 1) s += Azu[i + g.sz];
  return s;
}

// MSFE: per dual block, the 8x8 block sum over its cells and its low-side
// faces of  D_i P_i P_i^T + w_f (P_i - P_j)(P_i - P_j)^T.  The products and
// each thread's and warp's sums are in P's precision (FP32 for the mixed
// preconditioner, whose FP64 instruction count would otherwise bind the
// kernel), the sum over the block's warps in FP64.
template <class TP>
__global__ void __launch_bounds__(256) k_galerkin_fe_local(
    Geo g, CGeo c, const TP* __restrict__ P, const double* __restrict__ Ad,
    const double* __restrict__ Ax, const double* __restrict__ Ay, const double* __restrict__ Az,
    double* loc) {
  __shared__ double sh[36 * 32];
  const int ndx = c.nc[0] + 1, ndy = c.nc[1] + 1;
  const int D = blockIdx.x;
  const int j[3] = {D % ndx, (D / ndx) % ndy, D / (ndx * ndy)};
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) dual_range(c, g, d, j[d], lo[d], hi[d]);
  const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
  const int ncell = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
  using TA = TP;
  TA acc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) acc[k] = TA(0);
  for (int l = threadIdx.x; l < ncell; l += blockDim.x) {
    const int x = lo[0] + l % ex, y = lo[1] + (l / ex) % ey, z = lo[2] + l / (ex * ey);
    const long long i = x + g.sy * y + g.sz * z;
    TA pi[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) pi[s] = P[(long long)s * g.N + i];
    const TA Dd = (TA)row_sum(g, Ad, Ax, Ay, Az, Ax, Ay, Az, i, x, y, z);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const TA a = Dd * pi[s];
#pragma unroll
      for (int t = s; t < 8; ++t) acc[sym_idx(s, t)] += a * pi[t];
    }
    const int xc[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (xc[d] >= nd_of(g, d) - 1) continue;
      const long long jn = i + sd_of(g, d);
      const TA w = (TA)(-(d == 0 ? Ax[jn] : (d == 1 ? Ay[jn] : Az[jn])));
      const bool inside = xc[d] + 1 <= hi[d];
      TA dv[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        TA pj;
        if (inside) pj = P[(long long)s * g.N + jn];
        else pj = (s & (1 << d)) ? P[(long long)(s & ~(1 << d)) * g.N + jn] : TA(0);
        dv[s] = pi[s] - pj;
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const TA a = w * dv[s];
#pragma unroll
        for (int t = s; t < 8; ++t) acc[sym_idx(s, t)] += a * dv[t];
      }
    }
  }
  block_sum_k<36>(acc, sh, loc + (long long)D * 36);
}

// Gather the dual-block blocks into the 27-point coarse stencil, in a fixed
// block order (so entry (I,J) and (J,I) add identical terms in one order).
__global__ void k_galerkin_fe_gather(CGeo c, const double* __restrict__ loc, double* Acs) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= 27LL * c.Nc) return;
  const int I = (int)(q / 27), t = (int)(q % 27);
  const int off[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
  const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
  int Jc[3];
  for (int d = 0; d < 3; ++d) {
    Jc[d] = Ic[d] + off[d];
    if (Jc[d] < 0 || Jc[d] >= c.nc[d]) { Acs[q] = 0.0; return; }
  }
  const int ndx = c.nc[0] + 1, ndy = c.nc[1] + 1;
  double sum = 0.0;
  // dual blocks having I and J as corners: along d, j in {I, I+1} and {J, J+1}
  for (int jz = Ic[2]; jz <= Ic[2] + 1; ++jz)
    for (int jy = Ic[1]; jy <= Ic[1] + 1; ++jy)
      for (int jx = Ic[0]; jx <= Ic[0] + 1; ++jx) {
        const int jj[3] = {jx, jy, jz};
        int sI = 0, sJ = 0;
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          // corner bit of node K along d in dual block j: upper if j == K, lower if j == K + 1
          if (jj[d] == Ic[d]) sI |= 1 << d;
          else if (jj[d] != Ic[d] + 1) ok = false;
          if (jj[d] == Jc[d]) sJ |= 1 << d;
          else if (jj[d] != Jc[d] + 1) ok = false;
        }
        if (!ok) continue;
        const int D = jx + ndx * (jy + ndy * jz);
        const int a = sI < sJ ? sI : sJ, b = sI < sJ ? sJ : sI;
        sum += loc[(long long)D * 36 + sym_idx(a, b)];
      }
  Acs[q] = sum;
}

// MSFV: row I of R A P = sum over the cells of primal block I of (A P)_i,
// i.e. D_i P_i plus the fluxes w (P_i - P_j) through the block's faces.
// For a symmetric A the faces inside the block cancel and are skipped; with
// nonsym every face of every cell is taken, w = -a_{i,j} of the row.
template <class TP>
__global__ void __launch_bounds__(256) k_galerkin_fv(
    Geo g, CGeo c, const TP* __restrict__ P, const double* __restrict__ Ad,
    const double* __restrict__ Ax, const double* __restrict__ Ay, const double* __restrict__ Az,
    const double* __restrict__ Axu, const double* __restrict__ Ayu,
    const double* __restrict__ Azu, int nonsym, double* Acs) {
  extern __shared__ double acc[];   // 27 * blockDim
  const int I = blockIdx.x;
  const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
  const int bx = c.b[0], by = c.b[1], bz = c.b[2];
  const int nb = bx * by * bz;
  const int T = blockDim.x, tid = threadIdx.x;
  for (int k = 0; k < 27; ++k) acc[k * T + tid] = 0.0;
  auto add_cell = [&](long long cell, const int* xc, double scale) {
    for (int s = 0; s < 8; ++s) {
      const double v = (double)P[(long long)s * g.N + cell];
      if (v == 0.0) continue;
      int t = 0, mul = 1;
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        const int J = corner_d(c, d, xc[d], (s >> d) & 1);
        if (J < 0) { ok = false; break; }
        t += (J - Ic[d] + 1) * mul;
        mul *= 3;
      }
      if (ok) acc[t * T + tid] += scale * v;
    }
  };
  for (int l = tid; l < nb; l += T) {
    const int x = Ic[0] * bx + l % bx, y = Ic[1] * by + (l / bx) % by, z = Ic[2] * bz + l / (bx * by);
    const long long i = x + g.sy * y + g.sz * z;
    const int xc[3] = {x, y, z};
    add_cell(i, xc, row_sum(g, Ad, Ax, Ay, Az, Axu, Ayu, Azu, i, x, y, z));
    for (int d = 0; d < 3; ++d) {
      const int bd = c.b[d];
      for (int side = 0; side < 2; ++side) {
        const bool onface = side == 0 ? (xc[d] == Ic[d] * bd) : (xc[d] == Ic[d] * bd + bd - 1);
        if (!onface && !nonsym) continue;
        const int xn = xc[d] + (side == 0 ? -1 : 1);
        if (xn < 0 || xn >= nd_of(g, d)) continue;
        const long long jn = side == 0 ? i - sd_of(g, d) : i + sd_of(g, d);
        // row i's coupling to jn, stored at the upper cell of the face
        const double w = side == 0 ? -(d == 0 ? Ax[i] : (d == 1 ? Ay[i] : Az[i]))
                                   : -(d == 0 ? Axu[jn] : (d == 1 ? Ayu[jn] : Azu[jn]));
        add_cell(i, xc, w);
        int xcn[3] = {xc[0], xc[1], xc[2]};
        xcn[d] = xn;
        add_cell(jn, xcn, -w);
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < 27; k += T) {
    double s = 0.0;
    for (int q = 0; q < T; ++q) s += acc[k * T + q];
    Acs[(long long)I * 27 + k] = s;
  }
}

// MSFE for a nonsymmetric A (the full-Jacobian step): row I of P^T A P =
// sum over the cells i of basis function I's support of P_iI (A P)_i, with
// (A P)_i = D_i P_i + sum over the six faces of w (P_i - P_j), w = -a_{i,j}.
// One CTA per coarse node; sums in FP64.
template <class TP>
__global__ void __launch_bounds__(128) k_galerkin_fe_ns(
    Geo g, CGeo c, const TP* __restrict__ P, const double* __restrict__ Ad,
    const double* __restrict__ Ax, const double* __restrict__ Ay, const double* __restrict__ Az,
    const double* __restrict__ Axu, const double* __restrict__ Ayu,
    const double* __restrict__ Azu, double* Acs) {
  extern __shared__ double acc[];   // 27 * blockDim
  const int I = blockIdx.x;
  const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
  const int T = blockDim.x, tid = threadIdx.x;
  for (int k = 0; k < 27; ++k) acc[k * T + tid] = 0.0;
  // support of basis function I along d: strictly between the neighbouring vertex planes
  int lo[3], ext[3];
  for (int d = 0; d < 3; ++d) {
    const int X = Ic[d] * c.b[d] + c.o[d];
    lo[d] = max(0, X - c.b[d] + 1);
    ext[d] = min(nd_of(g, d) - 1, X + c.b[d] - 1) - lo[d] + 1;
  }
  // the slot of coarse node I in a cell's P row, -1 if none
  auto slot_of_I = [&](const int* xc) {
    int sl = 0;
    for (int d = 0; d < 3; ++d) {
      if (corner_d(c, d, xc[d], 0) == Ic[d]) continue;
      if (corner_d(c, d, xc[d], 1) == Ic[d]) { sl |= 1 << d; continue; }
      return -1;
    }
    return sl;
  };
  auto add_cell = [&](long long cell, const int* xc, double scale) {
    for (int s = 0; s < 8; ++s) {
      const double v = (double)P[(long long)s * g.N + cell];
      if (v == 0.0) continue;
      int t = 0, mul = 1;
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        const int J = corner_d(c, d, xc[d], (s >> d) & 1);
        const int o = J - Ic[d] + 1;
        if (J < 0 || o < 0 || o > 2) { ok = false; break; }
        t += o * mul;
        mul *= 3;
      }
      if (ok) acc[t * T + tid] += scale * v;
    }
  };
  const int ncell = ext[0] * ext[1] * ext[2];
  for (int l = tid; l < ncell; l += T) {
    const int xc[3] = {lo[0] + l % ext[0], lo[1] + (l / ext[0]) % ext[1],
                       lo[2] + l / (ext[0] * ext[1])};
    const long long i = xc[0] + g.sy * xc[1] + g.sz * xc[2];
    const int sI = slot_of_I(xc);
    if (sI < 0) continue;
    const double wI = (double)P[(long long)sI * g.N + i];
    if (wI == 0.0) continue;
    add_cell(i, xc, wI * row_sum(g, Ad, Ax, Ay, Az, Axu, Ayu, Azu, i, xc[0], xc[1], xc[2]));
    for (int d = 0; d < 3; ++d) {
      for (int side = 0; side < 2; ++side) {
        const int xn = xc[d] + (side == 0 ? -1 : 1);
        if (xn < 0 || xn >= nd_of(g, d)) continue;
        const long long jn = side == 0 ? i - sd_of(g, d) : i + sd_of(g, d);
        const double w = side == 0 ? -(d == 0 ? Ax[i] : (d == 1 ? Ay[i] : Az[i]))
                                   : -(d == 0 ? Axu[jn] : (d == 1 ? Ayu[jn] : Azu[jn]));
        if (w == 0.0) continue;
        add_cell(i, xc, wI * w);
        int xcn[3] = {xc[0], xc[1], xc[2]};
        xcn[d] = xn;
        add_cell(jn, xcn, -wI * w);
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < 27; k += T) {
    double s = 0.0;
    for (int q = 0; q < T; ++q) s += acc[k * T + q];
    Acs[(long long)I * 27 + k] = s;
  }
}

// Natural-order 27-point stencil -> column-major band in the reordered
// index.  General (MSFV): Bc[col*(2m+1) + (row - col + m)].  Symmetric
// (MSFE): lower triangle only, W[col*(m+1) + (row - col)].
template <class TB>
__global__ void k_band_fill(CGeo c, int m, int sym, const double* __restrict__ Acs,
                            const int* __restrict__ perm, TB* band) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= 27LL * c.Nc) return;
  const int I = (int)(q / 27), t = (int)(q % 27);
  const int off[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
  const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
  int J = 0, mul = 1;
  for (int d = 0; d < 3; ++d) {
    const int v = Ic[d] + off[d];
    if (v < 0 || v >= c.nc[d]) return;
    J += v * mul;
    mul *= c.nc[d];
  }
  const int row = perm[I], col = perm[J];
  if (sym) {
    if (row >= col) band[(long long)col * (m + 1) + (row - col)] = (TB)Acs[q];
  } else {
    band[(long long)col * (2 * m + 1) + (row - col + m)] = (TB)Acs[q];
  }
}

// ---- symmetric (MSFE) coarse matrix: blocked right-looking band LDL^T ----
// One launch per block of kTB columns [c0, c1].  Each CTA factors the
// kTB x kTB diagonal block in shared memory (redundantly: cheaper than a
// separate launch), forms the panel rows l_rq (q in the block) of the
// kTB-row tiles it owns, and subtracts  sum_q l_rq d_q l_cq  from its tile of
// the trailing band.  Diagonal-tile CTAs write their panel rows to the
// factor Lc (column-major: Lc[q*(m+1) + (r-q)], Lc[q*(m+1)] = d_q).  The
// working band W is only read in the block columns and only written right of
// them, so CTAs of one launch never race.
//
// On this GPU an FP64 warp instruction holds its sub-partition's FP64 unit
// for about 64 cycles whatever the number of active lanes, and a dependent
// FP64 instruction waits as long, so the factorisation's time is the number
// of FP64 warp instructions on its pivot chain.  The kernel keeps that
// number small: one thread per element of the diagonal block's lower
// triangle, the elements right of column 0 in warps 0-3 (at most one warp
// per sub-partition issues at each pivot: one product and one FMA), the
// reciprocal of the next pivot formed by its owner as soon as that pivot is
// final, from the hardware estimate and one Halley step instead of a
// division, the pivot tests on the bit pattern instead of FP64 compares, the
// panel rows solved by four threads per row (one warp per sub-partition),
// and the products d_q l_cq kept from the elimination instead of recomputed.
constexpr int kTB = 16;
constexpr int kTri = kTB * (kTB + 1) / 2;   // lower-triangle elements of a diagonal block

// 1/d of a pivot (rcp64.h), and whether d is positive and finite, tested on
// its bit pattern instead of by FP64 compares; a non-positive or non-finite
// pivot is replaced by 1 and reported.
__device__ __forceinline__ double pivot_rcp(double d, bool& bad) {
  const long long b = __double_as_longlong(d);
  bad = !(b > 0 && b < 0x7FF0000000000000LL);
  return rcp_halley(bad ? 1.0 : d);
}
// the same for a pivot of either sign (band LU): nonzero and finite
__device__ __forceinline__ double pivot_rcp_signed(double d, bool& bad) {
  const long long a = __double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFLL;
  bad = !(a > 0 && a < 0x7FF0000000000000LL);
  return rcp_halley(bad ? 1.0 : d);
}

template <class T>
__device__ __forceinline__ T band_at(const T* W, int m, int r, int c) {
  // lower band, column-major; 0 outside the band
  return (r - c <= m && r >= c) ? W[(long long)c * (m + 1) + (r - c)] : T(0);
}

// T: the precision of the factorisation (FP64, or FP32 for the mixed
// preconditioner's coarse solve)
template <class T>
__global__ void __launch_bounds__(256) k_ldlt_block(int N, int m, int c0, const T* __restrict__ Wr,
                                                    T* W, T* Lc, int* status) {
  __shared__ T A[kTB][kTB + 1];        // diagonal block; column q keeps d_q l_rq
  __shared__ T L[kTB][kTB + 1];        // l_rq below the diagonal
  __shared__ T rinv[kTB];              // 1 / d_q
  __shared__ T V[2 * kTB][kTB + 1];    // panel rows: a_rq in, l_rq out
  __shared__ T VD[2 * kTB][kTB + 1];   // d_q l_rq of the panel rows
  const int c1 = min(c0 + kTB, N) - 1;
  const int tb = c1 - c0 + 1;
  const int tid = threadIdx.x;
  // my tile of the trailing triangle, enumerated row by row (bj <= bi)
  const int rlo = c1 + 1;
  const int rhi = min(c1 + m, N - 1);
  const int nb = rhi >= rlo ? (rhi - rlo + kTB) / kTB : 0;
  int bi = 0, bj = 0;
  {
    int t = blockIdx.x;
    while (t > bi) { t -= bi + 1; ++bi; }
    bj = t;
  }
  const bool have_tile = nb > 0 && bi < nb;
  const int r0 = rlo + bi * kTB, cc0 = rlo + bj * kTB;
  // Programmatic dependent launch: the next block's launch may begin now;
  // its CTAs wait below until this grid has completed and its writes are
  // visible (a no-op when launched without the attribute).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // --- stage the diagonal block and the 2 kTB panel rows ---
  // (consecutive threads take consecutive rows of one band column: the
  // column is contiguous in the band)
  {
    const int r = tid % kTB, q = tid / kTB;
    A[r][q] = (r < tb && q <= r) ? band_at(Wr, m, c0 + r, c0 + q) : T(0);
  }
  for (int e = tid; e < 2 * kTB * kTB; e += blockDim.x) {
    const int k = e % (2 * kTB), q = e / (2 * kTB);
    const int r = (k < kTB ? r0 + k : cc0 + k - kTB);
    V[k][q] = (have_tile && r <= rhi && q < tb) ? band_at(Wr, m, r, c0 + q) : T(0);
  }
  // element of the diagonal block's lower triangle owned by this thread:
  // those right of column 0, row by row in threads 0..119 (warps 0-3).
  // Column 0 is scaled at the first pivot by the threads of column 1, which
  // form the same products.
  int er = 0, ec = -1;
  if (tid < kTri - kTB) {
    int t = tid, r = 1;
    while (t >= r) { t -= r; ++r; }
    er = r;
    ec = t + 1;
  }
  __syncthreads();
  if (tid == 0) {
    bool bad;
    rinv[0] = pivot_rcp(A[0][0], bad);
    if (bad && blockIdx.x == 0) atomicOr(status, kStatSingular);
  }
  // panel rows, four threads a row in warps 4-7
  const int pk = (tid - 128) >> 2, pt = tid & 3;
  const int src0 = (threadIdx.x & 31) & ~3;
  T v[kTB / 4];
  if (tid >= 128) {
#pragma unroll
    for (int j = 0; j < kTB / 4; ++j) v[j] = V[pk][4 * j + pt];
  }
  __syncthreads();
  // --- factor the diagonal block (warps 0-3): at pivot q, column q is
  // scaled and the trailing triangle updated, a_rc -= (a_rq / d_q) a_cq.
  // Beside it (warps 4-7), step q of the panel rows: l_rq = (a_rq -
  // sum_{k<q} l_rk d_k l_qk) / d_q, which needs only column q and 1/d_q,
  // final once pivot q-1 is done, so the panel runs one pivot behind the
  // factorisation under the same barriers instead of after it ---
#pragma unroll
  for (int q = 0; q < kTB; ++q) {
    if (q < tb) {                                // uniform across the CTA
      if (tid < 128) {
        if (ec >= q && er > q && er < tb) {
          const T t = A[er][q] * rinv[q];
          if (ec == q) {
            L[er][q] = t;
          } else {
            if (q == 0 && ec == 1) L[er][0] = t;
            const T vv = fma(-t, A[ec][q], A[er][ec]);
            A[er][ec] = vv;
            if (er == q + 1 && ec == q + 1) {   // the next pivot is final
              bool bad;
              rinv[q + 1] = pivot_rcp(vv, bad);
              if (bad && blockIdx.x == 0) atomicOr(status, kStatSingular);
            }
          }
        }
      } else {
        T l = T(0);
        if (pt == (q & 3)) {
          VD[pk][q] = v[q >> 2];
          l = v[q >> 2] * rinv[q];
          v[q >> 2] = l;
        }
        l = __shfl_sync(0xffffffffu, l, src0 | (q & 3));
#pragma unroll
        for (int j = 0; j < kTB / 4; ++j)
          if (4 * j + 3 > q && 4 * j + pt > q) v[j] = fma(-l, A[4 * j + pt][q], v[j]);
      }
      __syncthreads();
    }
  }
  if (tid >= 128) {
#pragma unroll
    for (int j = 0; j < kTB / 4; ++j) V[pk][4 * j + pt] = v[j];
  }
  __syncthreads();
  if (have_tile) {
    // W[r][c] -= sum_q l_rq d_q l_cq, one element a thread
    const int a = tid / kTB, b = tid % kTB;
    const int r = r0 + a, cc = cc0 + b;
    if (r <= rhi && cc <= rhi && cc <= r && r - cc <= m) {
      T s = T(0);
      for (int q = 0; q < tb; ++q) s = fma(V[a][q], VD[kTB + b][q], s);
      W[(long long)cc * (m + 1) + (r - cc)] -= s;
    }
    // diagonal tiles publish their panel rows
    if (bi == bj) {
      const int a2 = tid / kTB, q = tid % kTB;
      const int r2 = r0 + a2, col = c0 + q;
      if (r2 <= rhi && q < tb && r2 - col <= m) Lc[(long long)col * (m + 1) + (r2 - col)] = V[a2][q];
    }
  }
  // the first CTA publishes the diagonal block: l below, d_q on the diagonal
  if (blockIdx.x == 0 && ec >= 0 && er < tb && er - ec <= m)
    Lc[(long long)(c0 + ec) * (m + 1) + (er - ec)] = er == ec ? A[er][er] : L[er][ec];
  if (blockIdx.x == 0 && tid < tb && tid <= m)   // column 0
    Lc[(long long)c0 * (m + 1) + tid] = tid == 0 ? A[0][0] : L[tid][0];
}

// Row-major copy of L for the backward substitution: Lr[k*(m+1) + a] = l_{k,k-a}.
__global__ void k_ldlt_rows(int N, int m, const double* __restrict__ Lc, double* Lr) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)N * (m + 1)) return;
  const int k = (int)(e / (m + 1)), a = (int)(e % (m + 1));
  Lr[e] = (a == 0) ? Lc[(long long)k * (m + 1)] : (k - a >= 0 ? Lc[(long long)(k - a) * (m + 1) + a] : 0.0);
}

// ---- the mixed preconditioner's coarse solve by the inverse factor ----
// With the FP32 factor L D L^T of the coarse matrix, Z = L^{-1} (unit lower
// triangular, dense below the diagonal) is formed once per factorisation,
// and every solve is x = Z^T (D^{-1} (Z b)): two matrix-vector products over
// the lower triangle of Z, which stream Z from memory, in place of a
// substitution whose N forward and N backward steps depend on one another.
// In exact arithmetic the result is the substitution's.
//
// Column j of Z solves L z = e_j: z_i = 0 (i < j), z_j = 1, and
// z_i = -sum_{k=max(j,i-m)}^{i-1} l_ik z_k.  A CTA takes 16 consecutive
// columns and walks their rows in blocks of 32, one row a lane; its 32 warps
// are 4 column groups (kZC columns each, one 16-byte ring entry) x 8.  The
// band entries l_ik of a block's 32 rows (columns k from max(first column,
// r0 - m) to r0 + 31) are staged in shared memory two blocks ahead
// (cp.async with zero fill; three tile buffers).  Each column group keeps
// its values of the last m + 32 rows in a ring in shared memory, written
// twice so that any window of them is contiguous.  The sum over the rows
// before a block is split into a far part (rows of the blocks before the
// previous one) and a near part (the previous block's rows): while the
// first warp of each group finishes block b's rows one after the other
// (each broadcast by shuffle to the rows below it), the other seven already
// sum the far part of block b + 1; the near part is then shared by all
// eight.  (16 columns a CTA measured 0.69 ms a 4000-node formation against
// 0.84 with 32 and 1.14 with 8.)  Z is column-major with leading dimension
// ldz (a multiple of 128); rows i >= j of column j are written, the others
// are never read.
constexpr int kZC = 4;    // columns of Z per column group (one 16-byte ring entry)
constexpr int kZG = 4;    // column groups per CTA: 16 columns
constexpr int kZQ = 8;    // warps per column group
constexpr int kZT = 32 * kZG * kZQ;   // threads per CTA
constexpr int kZCols = kZG * kZC;     // columns per CTA

__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void add4(float4& a, const float4& b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

// acc += sum over rows k in [k0, k1) of l_ik y_k (lane = row i - r0), with
// Lt the tile whose first column is kb and R the column group's ring
__device__ __forceinline__ void zband(float4& acc, const float* Lt, int kb, const float4* R,
                                      int mask, int k0, int k1, int lane) {
  const float* lp = Lt + (k0 - kb) * 32 + lane;
  const float4* yp = R + (k0 & mask);              // contiguous: the ring is written twice
#pragma unroll 8
  for (int t = 0; t < k1 - k0; ++t) {
    const float l = lp[t * 32];
    const float4 y = yp[t];
    acc.x = fmaf(l, y.x, acc.x);
    acc.y = fmaf(l, y.y, acc.y);
    acc.z = fmaf(l, y.z, acc.z);
    acc.w = fmaf(l, y.w, acc.w);
  }
}

__global__ void __launch_bounds__(kZT, 1) k_coarse_zinv(int N, int m, int ring,
                                                      const float* __restrict__ Lc, float* Z,
                                                      long long ldz) {
  // [3][m + 32][32] band tiles, [2][kZQ - 1][kZG][32] float4 far sums,
  // [kZQ - 1][kZG][32] float4 near sums, [kZG][2 ring] float4 rings
  extern __shared__ __align__(16) float zsm[];
  const int tw = m + 32;                           // tile columns
  float* tiles = zsm;
  float4* farp = reinterpret_cast<float4*>(zsm + 3 * tw * 32);
  float4* nearp = farp + 2 * (kZQ - 1) * kZG * 32;
  float4* rings = nearp + (kZQ - 1) * kZG * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cg = warp % kZG, kq = warp / kZG;
  const int J0 = blockIdx.x * kZCols;              // the CTA's first column
  const int j0 = J0 + cg * kZC;                    // the column group's first column
  const bool active = j0 < N;
  float4* R = rings + (size_t)cg * 2 * ring;
  const int mask = ring - 1, mp = m + 1;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = tid; t < kZG * 2 * ring; t += kZT) rings[t] = zero4;
  for (int t = tid; t < 3 * (kZQ - 1) * kZG * 32; t += kZT) farp[t] = zero4;   // far and near sums
  // tile of block r0: Lt[(k - kb) * 32 + (i - r0)] = l_ik inside the band, else 0
  auto load_tile = [&](int r0, float* Lt) {
    const int kb = max(J0, r0 - m);
    const int n = (r0 + 32 - kb) * 32;
    for (int e = tid; e < n; e += kZT) {
      const int k = kb + (e >> 5), i = r0 + (e & 31), d = i - k;
      const bool v = i < N && d >= 1 && d <= m;
      cp_async4_zfill(Lt + e, v ? Lc + (long long)k * mp + d : Lc, v);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int nblk = (N - J0 + 31) / 32;
  load_tile(J0, tiles);
  if (nblk > 1) load_tile(J0 + 32, tiles + tw * 32);
  for (int b = 0; b < nblk; ++b) {
    const int r0 = J0 + 32 * b;
    const float* Lt = tiles + (b % 3) * tw * 32;
    const float* Ln = tiles + ((b + 1) % 3) * tw * 32;
    if (b + 2 < nblk) {
      load_tile(r0 + 64, tiles + ((b + 2) % 3) * tw * 32);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();                               // tiles b, b+1 in; rows < r0 in the rings
    const int kb = max(J0, r0 - m);
    // near part of block b: the previous block's rows, an eighth per warp
    float4 acc = zero4;
    if (active) {
      const int nlo = max(max(j0, r0 - m), r0 - 32), n = r0 - nlo;
      if (n > 0) zband(acc, Lt, kb, R, mask, nlo + (n * kq) / kZQ, nlo + (n * (kq + 1)) / kZQ, lane);
      if (kq > 0) nearp[((kq - 1) * kZG + cg) * 32 + lane] = acc;
    }
    __syncthreads();
    if (active && kq == 0) {
#pragma unroll
      for (int q = 0; q < kZQ - 1; ++q) {
        add4(acc, nearp[(q * kZG + cg) * 32 + lane]);
        add4(acc, farp[(((b & 1) * (kZQ - 1) + q) * kZG + cg) * 32 + lane]);
      }
      float a4[kZC] = {acc.x, acc.y, acc.z, acc.w};
      // the block's rows, in order
      float y[kZC];
#pragma unroll
      for (int c = 0; c < kZC; ++c) y[c] = 0.f;
      for (int kk = 0; kk < 32 && r0 + kk < N; ++kk) {
        const int k = r0 + kk;
        if (lane == kk) {
#pragma unroll
          for (int c = 0; c < kZC; ++c) {
            const int j = j0 + c;
            y[c] = k == j ? 1.f : (k > j ? -a4[c] : 0.f);
          }
        }
        const float l = Lt[(k - kb) * 32 + lane];   // 0 for rows at or above k
#pragma unroll
        for (int c = 0; c < kZC; ++c) a4[c] = fmaf(l, __shfl_sync(0xffffffffu, y[c], kk), a4[c]);
      }
      const int i = r0 + lane;
      if (i < N) {
        const float4 yv = make_float4(y[0], y[1], y[2], y[3]);
        R[i & mask] = yv;
        R[(i & mask) + ring] = yv;
#pragma unroll
        for (int c = 0; c < kZC; ++c) {
          const int j = j0 + c;
          if (j < N && i >= j) Z[(long long)j * ldz + i] = y[c];
        }
      }
    } else if (active && b + 1 < nblk) {
      // far part of block b + 1 (rows of the blocks before b), a seventh per warp
      const int r1 = r0 + 32, kb1 = max(J0, r1 - m);
      const int flo = max(j0, r1 - m), n = r0 - flo;
      float4 f = zero4;
      if (n > 0) {
        const int w = kq - 1;
        zband(f, Ln, kb1, R, mask, flo + (n * w) / (kZQ - 1), flo + (n * (w + 1)) / (kZQ - 1), lane);
      }
      farp[((((b + 1) & 1) * (kZQ - 1) + (kq - 1)) * kZG + cg) * 32 + lane] = f;
    }
    __syncthreads();                               // ring written; tile b is refilled next
  }
}

// Partial sums of Z b: CTA (strip s, chunk c) adds, for the 128 rows
// i0 = 128 s .. i0 + 127, the columns j of chunk c (256 columns) with
// j <= i; each lane takes four consecutive rows (one 16-byte load per
// column), each warp 32 columns, and the warps' sums meet in shared memory.
// part[c * ldz + i].  b is the FP64 restricted residual, rounded to FP32.
constexpr int kZS = 128;   // rows per strip
constexpr int kZK = 256;   // columns per chunk
__global__ void __launch_bounds__(256) k_coarse_zlower(int N, const float* __restrict__ Z,
                                                       long long ldz, const double* __restrict__ rhs,
                                                       float* part) {
  __shared__ float4 red[8][32];
  __shared__ float bs[kZK];                        // the chunk's b, rounded to FP32 once
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kZS, c = blockIdx.y, jc = c * kZK;
  if (jc > i0 + kZS - 1 || jc >= N) return;        // the whole chunk lies above the strip
  // (an FP64 -> FP32 conversion is an FP64-unit instruction: one per
  // element here, not one per element and warp in the loop below)
  for (int e = threadIdx.x; e < kZK; e += blockDim.x) bs[e] = jc + e < N ? (float)rhs[jc + e] : 0.f;
  __syncthreads();
  const int ib = i0 + 4 * lane;                    // my rows ib .. ib + 3
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int jlo = jc + warp * 32, jhi = min(min(jlo + 32, N), i0 + kZS);
#pragma unroll 8
  for (int j = jlo; j < jhi; ++j) {
    const float4 z = *reinterpret_cast<const float4*>(Z + (long long)j * ldz + ib);
    const float bj = bs[j - jc];
    // rows above the diagonal or past N hold no value of Z
    acc.x += (ib + 0 >= j && ib + 0 < N) ? z.x * bj : 0.f;
    acc.y += (ib + 1 >= j && ib + 1 < N) ? z.y * bj : 0.f;
    acc.z += (ib + 2 >= j && ib + 2 < N) ? z.z * bj : 0.f;
    acc.w += (ib + 3 >= j && ib + 3 < N) ? z.w * bj : 0.f;
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    float4 s = red[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) {
      s.x += red[w][lane].x;
      s.y += red[w][lane].y;
      s.z += red[w][lane].z;
      s.w += red[w][lane].w;
    }
    *reinterpret_cast<float4*>(part + (long long)c * ldz + ib) = s;
  }
}

// t_i = (Z b)_i / d_i: the chunks' partial sums in chunk order.
__global__ void k_coarse_tsum(int N, int m, const float* __restrict__ Lc,
                              const float* __restrict__ part, long long ldz, float* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float s = 0.f;
  for (int c = 0; c * kZK <= i; ++c) s += part[(long long)c * ldz + i];
  t[i] = s / Lc[(long long)i * (m + 1)];
}

// x = Z^T t: one warp per column j (its rows i >= j are contiguous), 16-byte
// loads from the aligned row j & ~3 on.
__global__ void __launch_bounds__(256) k_coarse_zupper(int N, const float* __restrict__ Z,
                                                       long long ldz, const float* __restrict__ t,
                                                       float* x) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= N) return;
  const float* col = Z + (long long)j * ldz;
  float acc = 0.f;
#pragma unroll 4
  for (int i = (j & ~3) + 4 * lane; i < N; i += 128) {
    const float4 z = *reinterpret_cast<const float4*>(col + i);
    const float4 v = *reinterpret_cast<const float4*>(t + i);
    acc += (i + 0 >= j) ? z.x * v.x : 0.f;
    acc += (i + 1 >= j && i + 1 < N) ? z.y * v.y : 0.f;
    acc += (i + 2 >= j && i + 2 < N) ? z.z * v.z : 0.f;
    acc += (i + 3 >= j && i + 3 < N) ? z.w * v.w : 0.f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[j] = acc;
}

// L D L^T x = b, one CTA.  y lives in shared memory; the factor is streamed
// through shared memory in chunks of kSC consecutive columns (forward, from
// the column-major Lc) or rows (backward, from the row-major Lr), each chunk
// a contiguous run copied with cp.async while the previous one is applied.
constexpr int kSC = 16;

__device__ __forceinline__ void cp_async16(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// copy `n` doubles (n even, both addresses 16-byte aligned) into shared memory
__device__ __forceinline__ void stage(double* dst, const double* src, int n) {
  for (int e = 2 * threadIdx.x; e < n; e += 2 * blockDim.x) cp_async16(dst + e, src + e);
  cp_async_commit();
}

__global__ void __launch_bounds__(256) k_ldlt_solve(int N, int m, const double* __restrict__ Lc,
                                                    const double* __restrict__ Lr, const double* __restrict__ rc,
                                                    double* pc) {
  extern __shared__ __align__(16) double sm[];
  const int mp = m + 1;
  const int chunk = kSC * mp;                  // even: mp is even by construction
  double* buf0 = sm;
  double* buf1 = sm + chunk;
  double* y = sm + 2 * chunk;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N; i += nt) y[i] = rc[i];
  const int nchunks = (N + kSC - 1) / kSC;
  // forward with the unit lower factor, column by column
  stage(buf0, Lc, min(kSC, N) * mp);
  for (int ck = 0; ck < nchunks; ++ck) {
    double* cur = (ck & 1) ? buf1 : buf0;
    double* nxt = (ck & 1) ? buf0 : buf1;
    cp_async_wait_all();
    __syncthreads();
    if (ck + 1 < nchunks) {
      const int k1 = (ck + 1) * kSC;
      stage(nxt, Lc + (long long)k1 * mp, min(kSC, N - k1) * mp);
    }
    const int k0 = ck * kSC;
    for (int c = 0; c < kSC && k0 + c < N; ++c) {
      const int k = k0 + c;
      const double yk = y[k];
      const int amax = min(m, N - 1 - k);
      for (int a = 1 + tid; a <= amax; a += nt) y[k + a] -= cur[c * mp + a] * yk;
      __syncthreads();
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < N; i += nt) y[i] /= Lc[(long long)i * mp];
  // backward with L^T: rows of L from the last chunk down
  const int last0 = (nchunks - 1) * kSC;
  stage(buf0, Lr + (long long)last0 * mp, (N - last0) * mp);
  for (int ck = nchunks - 1, it = 0; ck >= 0; --ck, ++it) {
    double* cur = (it & 1) ? buf1 : buf0;
    double* nxt = (it & 1) ? buf0 : buf1;
    cp_async_wait_all();
    __syncthreads();
    if (ck > 0) stage(nxt, Lr + (long long)(ck - 1) * kSC * mp, kSC * mp);
    const int k0 = ck * kSC;
    for (int c = min(kSC, N - k0) - 1; c >= 0; --c) {
      const int k = k0 + c;
      const double xk = y[k];
      const int amax = min(m, k);
      for (int a = 1 + tid; a <= amax; a += nt) y[k - a] -= cur[c * mp + a] * xk;
      __syncthreads();
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < N; i += nt) pc[i] = y[i];
}

// ---- L D L^T x = b across a thread-block cluster ----
// The rows are cut into blocks of kCB.  With L_IJ the blocks of the unit
// lower factor, the forward solve L y = b is, block by block,
//   y_J = s_J - M_J y_{J-1},  s_J = L_JJ^{-1} (b_J - sum_{I <= J-2} L_JI y_I),
//   M_J = L_JJ^{-1} L_{J,J-1},
// so once y_{J-1} is known only one kCB x kCB product remains; s_J needs
// y_{J-2} and is formed one block earlier.  The backward solve
// L^T x = D^{-1} y is the same with the transposed blocks:
//   x_I = s'_I - M'_I x_{I+1},  M'_I = L_II^{-T} L_{I+1,I}^T.
// k_coarse_prep computes L_JJ^{-1}, M_J, M'_J and 1/d after each
// factorisation.  k_coarse_solve_cluster deals the blocks round-robin to the
// kCC CTAs of one cluster; each CTA keeps a copy of y and x in shared memory
// (kNotReady until written) and the owner of a block stores its values into
// every CTA's copy through distributed shared memory.
constexpr int kCB = 32;                      // rows per block
constexpr int kCBlocks = 3;                  // per block: L_JJ^{-1}, M_J, M'_J
constexpr int kCC = 8;                       // CTAs per cluster
constexpr unsigned long long kCNotReady = 0x7FF4DEADBEEF0002ull;   // signalling NaN
constexpr unsigned kCNotReady32 = 0x7FA5A5A2u;                      // signalling NaN (FP32)
constexpr long long kCSpinLimit = 1LL << 22;

__device__ __forceinline__ double lower_at(const double* Lc, int N, int m, int r, int c) {
  // strictly lower entry of the unit factor (column-major band), 0 elsewhere
  return (r < N && c >= 0 && r > c && r - c <= m) ? Lc[(long long)c * (m + 1) + (r - c)] : 0.0;
}

// One CTA per block J: blk[J] = { L_JJ^{-1}, M_J, M'_J } (kCB x kCB each,
// row-major), dinv[i] = 1 / d_i.  Rows past N act as identity rows.
__global__ void __launch_bounds__(256) k_coarse_prep(int N, int m, const double* __restrict__ Lc,
                                                     double* blk, double* dinv) {
  __shared__ double Lj[kCB][kCB + 1];
  __shared__ double Li[kCB][kCB + 1];
  __shared__ double Lo[kCB][kCB + 1];
  const int J = blockIdx.x, NB = gridDim.x, base = J * kCB, tid = threadIdx.x;
  double* out = blk + (long long)J * kCBlocks * kCB * kCB;
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int r = e / kCB, q = e % kCB;
    Lj[r][q] = q == r ? 1.0 : lower_at(Lc, N, m, base + r, base + q);
  }
  if (tid < kCB && base + tid < N) dinv[base + tid] = 1.0 / Lc[(long long)(base + tid) * (m + 1)];
  __syncthreads();
  // inverse of the unit lower block, one column per thread (forward substitution)
  if (tid < kCB) {
    const int c = tid;
    for (int r = 0; r < kCB; ++r) {
      double s = r == c ? 1.0 : 0.0;
      if (r > c) {
        for (int q = c; q < r; ++q) s -= Lj[r][q] * Li[q][c];
      }
      Li[r][c] = s;
    }
  }
  __syncthreads();
  for (int e = tid; e < kCB * kCB; e += blockDim.x) out[e] = Li[e / kCB][e % kCB];
  // M_J = L_JJ^{-1} L_{J,J-1}
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int r = e / kCB, q = e % kCB;
    Lo[r][q] = J > 0 ? lower_at(Lc, N, m, base + r, base - kCB + q) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int r = e / kCB, q = e % kCB;
    double s = 0.0;
    for (int k = 0; k < kCB; ++k) s += Li[r][k] * Lo[k][q];
    out[kCB * kCB + e] = s;
  }
  __syncthreads();
  // M'_J = L_JJ^{-T} L_{J+1,J}^T :  M'[c][q] = sum_k Li[k][c] L[(J+1)B + q][JB + k]
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int q = e / kCB, kk = e % kCB;
    Lo[q][kk] = J + 1 < NB ? lower_at(Lc, N, m, base + kCB + q, base + kk) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int c = e / kCB, q = e % kCB;
    double s = 0.0;
    for (int kk = 0; kk < kCB; ++kk) s += Li[kk][c] * Lo[q][kk];
    out[2 * kCB * kCB + e] = s;
  }
}

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v into the same shared-memory location of every CTA of the cluster
__device__ __forceinline__ void cl_broadcast(const double* local, double v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
#pragma unroll
  for (int rk = 0; rk < kCC; ++rk) {
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rk));
    asm volatile("st.relaxed.cluster.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
  }
}
__device__ __forceinline__ void cl_broadcast(const float* local, float v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(local);
#pragma unroll
  for (int rk = 0; rk < kCC; ++rk) {
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rk));
    asm volatile("st.relaxed.cluster.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
  }
}
__device__ __forceinline__ unsigned long long ld_cl(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.cluster.shared::cta.b64 %0, [%1];"
               : "=l"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_cl(const float* p) {
  unsigned v;
  asm volatile("ld.relaxed.cluster.shared::cta.b32 %0, [%1];"
               : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}
// the "not yet written" pattern of each precision, and its value
template <class T> struct CWord;
template <> struct CWord<double> {
  static constexpr unsigned long long kNR = kCNotReady;
  static __device__ __forceinline__ double value(unsigned long long b) { return __longlong_as_double((long long)b); }
};
template <> struct CWord<float> {
  static constexpr unsigned kNR = kCNotReady32;
  static __device__ __forceinline__ float value(unsigned b) { return __uint_as_float(b); }
};
__device__ __forceinline__ int ld_abort(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Waits until the 4 values at p are written; false after an abort or a timeout.
template <class T>
__device__ __forceinline__ bool wait4(const T* p, T* v, int* abort_flag, int* status) {
  for (long long it = 0; it < kCSpinLimit; ++it) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const auto b = ld_cl(p + k);
      v[k] = CWord<T>::value(b);
      ok &= b != CWord<T>::kNR;
    }
    if (ok) return true;
    if ((it & 63) == 63) {
      if (ld_abort(abort_flag)) return false;
      __nanosleep(32);
    }
  }
  atomicOr(status, kStatTimeout);
  atomicExch(abort_flag, 1);
  return false;
}

// sum over the 8 lanes of an aligned lane group (every lane gets the sum)
template <class T>
__device__ __forceinline__ T sum8(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// 256 threads: thread (r = tid / 8, h = tid % 8) owns row r of a block and
// the 4 columns 4h .. 4h+3 of every kCB x kCB product.  T: the precision of
// the substitution (the factor's blocks come in that precision; the
// right-hand side is FP64, rounded to T).
template <class T>
__global__ void __launch_bounds__(256, 1) k_coarse_solve_cluster(
    int N, int m, const T* __restrict__ Lc, const T* __restrict__ Lr,
    const T* __restrict__ blk, const T* __restrict__ dinv,
    const double* __restrict__ rc, T* pc, int* abort_flag, int* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  __shared__ T uv[kCB];
  const int NB = (N + kCB - 1) / kCB, Np = NB * kCB;
  T* y = sm;
  T* x = sm + Np;
  const int rank = (int)cl_rank();
  const int tid = threadIdx.x, r = tid >> 3, h = tid & 7;
  const int W = (m + kCB - 1) / kCB;           // blocks of the band left of a diagonal block
  for (int i = tid; i < 2 * Np; i += blockDim.x) sm[i] = CWord<T>::value(CWord<T>::kNR);
  cl_sync();
  bool ok = true;
  // ---- forward: L y = b ----
  for (int J = rank; J < NB; J += kCC) {
    const int base = J * kCB, row = base + r;
    T acc = (h == 0 && row < N) ? T(rc[row]) : T(0);
    for (int I = J - W > 0 ? J - W : 0; I <= J - 2; ++I) {
      T yv[4] = {0.0, 0.0, 0.0, 0.0};
      ok = ok && wait4(y + I * kCB + 4 * h, yv, abort_flag, status);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = I * kCB + 4 * h + k;
        const T l = (row < N && row - c <= m) ? Lr[(long long)row * (m + 1) + (row - c)] : 0.0;
        acc -= l * yv[k];
      }
    }
    acc = sum8(acc);
    if (h == 0) uv[r] = acc;
    __syncthreads();
    const T* Li = blk + (long long)J * kCBlocks * kCB * kCB;
    T s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += Li[r * kCB + 4 * h + k] * uv[4 * h + k];
    s = sum8(s);
    if (J > 0) {
      const T* M = Li + kCB * kCB;
      T yv[4] = {0.0, 0.0, 0.0, 0.0};
      ok = ok && wait4(y + (J - 1) * kCB + 4 * h, yv, abort_flag, status);
      T t = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) t += M[r * kCB + 4 * h + k] * yv[k];
      s -= sum8(t);
    }
    __syncthreads();
    if (h == 0) cl_broadcast(y + row, ok ? s : 0.0);
  }
  // ---- backward: L^T x = D^{-1} y ----
  const int lastJ = NB - 1 - ((NB - 1 - rank) % kCC + kCC) % kCC;
  for (int I = lastJ; I >= 0; I -= kCC) {
    const int base = I * kCB, col = base + r;
    T acc = 0.0;
    if (h == 0) {
      T yv[4] = {0.0, 0.0, 0.0, 0.0};
      ok = ok && wait4(y + base + (r & ~3), yv, abort_flag, status);
      acc = col < N ? yv[r & 3] * dinv[col] : 0.0;
    }
    for (int J = I + W < NB - 1 ? I + W : NB - 1; J >= I + 2; --J) {
      T xv[4] = {0.0, 0.0, 0.0, 0.0};
      ok = ok && wait4(x + J * kCB + 4 * h, xv, abort_flag, status);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int rw = J * kCB + 4 * h + k;
        const T l = (rw < N && col < N && rw - col <= m) ? Lc[(long long)col * (m + 1) + (rw - col)] : 0.0;
        acc -= l * xv[k];
      }
    }
    acc = sum8(acc);
    if (h == 0) uv[r] = acc;
    __syncthreads();
    const T* Li = blk + (long long)I * kCBlocks * kCB * kCB;
    T s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += Li[(4 * h + k) * kCB + r] * uv[4 * h + k];
    s = sum8(s);
    if (I + 1 < NB) {
      const T* Mt = Li + 2 * kCB * kCB;
      T xv[4] = {0.0, 0.0, 0.0, 0.0};
      ok = ok && wait4(x + (I + 1) * kCB + 4 * h, xv, abort_flag, status);
      T t = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) t += Mt[r * kCB + 4 * h + k] * xv[k];
      s -= sum8(t);
    }
    __syncthreads();
    if (h == 0) {
      cl_broadcast(x + col, ok ? s : 0.0);
      if (col < N) pc[col] = s;
    }
  }
  cl_sync();   // no CTA leaves while others may still store into its shared memory
}

// Symmetric band solve for coarse grids whose vectors do not fit shared
// memory (N_c of tens of thousands): the block recurrences of
// k_coarse_solve_cluster, run by one CTA block after block, with y and x in
// global memory (they stay in L2).  Per block of kCB rows: the band's part
// from the solved blocks (four independent partial sums per thread, so the
// FP64 additions overlap), then the kCB x kCB inverse of the diagonal block.
__global__ void __launch_bounds__(256, 1) k_coarse_solve_global(
    int N, int m, const double* __restrict__ Lc, const double* __restrict__ Lr,
    const double* __restrict__ blk, const double* __restrict__ dinv,
    const double* __restrict__ rc, double* y, double* pc) {
  __shared__ double uv[kCB];
  const int NB = (N + kCB - 1) / kCB;
  const int tid = threadIdx.x, r = tid >> 3, h = tid & 7;
  // ---- forward: L y = b ----
  for (int J = 0; J < NB; ++J) {
    const int base = J * kCB, row = base + r;
    const int lo = row - m > 0 ? row - m : 0;
    double a4[4] = {0.0, 0.0, 0.0, 0.0};
    if (row < N)
      for (int c = lo + h; c < base; c += 8)
        a4[(c >> 3) & 3] -= Lr[(long long)row * (m + 1) + (row - c)] * y[c];
    double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    acc = sum8(acc);
    if (h == 0) uv[r] = (row < N ? rc[row] : 0.0) + acc;
    __syncthreads();
    const double* Li = blk + (long long)J * kCBlocks * kCB * kCB;
    double sy = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) sy += Li[r * kCB + 4 * h + k] * uv[4 * h + k];
    sy = sum8(sy);
    if (h == 0 && row < N) y[row] = sy;
    __syncthreads();                           // y of this block is visible to the CTA
  }
  // ---- backward: L^T x = D^{-1} y ----
  for (int I = NB - 1; I >= 0; --I) {
    const int base = I * kCB, col = base + r;
    const int hi = col + m < N - 1 ? col + m : N - 1;
    double a4[4] = {0.0, 0.0, 0.0, 0.0};
    if (col < N)
      for (int rw = base + kCB + h; rw <= hi; rw += 8)
        a4[(rw >> 3) & 3] -= Lc[(long long)col * (m + 1) + (rw - col)] * pc[rw];
    double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    acc = sum8(acc);
    if (h == 0) uv[r] = (col < N ? y[col] * dinv[col] : 0.0) + acc;
    __syncthreads();
    const double* Li = blk + (long long)I * kCBlocks * kCB * kCB;
    double sx = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) sx += Li[(4 * h + k) * kCB + r] * uv[4 * h + k];
    sx = sum8(sx);
    if (h == 0 && col < N) pc[col] = sx;
    __syncthreads();
  }
}

// ---- general coarse matrix (MSFV, or MSFE of a nonsymmetric A): band LU ----
// without pivoting, in column blocks of kTB like k_ldlt_block.  Column-major
// band B[col*(2m+1) + (row-col+m)].  One launch per column block c0..c1:
// every CTA factors the diagonal block D = L_D U_D, forms its kTB rows of
// the L panel (A U_D^{-1}, rows c1+1..c1+m) and its kTB columns of the U
// panel (L_D^{-1} A, columns c1+1..c1+m), and updates its tile of the
// trailing window (rows and columns c1+1..c1+m, all inside the band).  The
// factor goes to F (same layout: U on and above the diagonal, the
// multipliers of L below), so no CTA reads a value another one rewrites.
__device__ __forceinline__ double gband_at(const double* B, int m, int r, int c) {
  return (r - c <= m && c - r <= m) ? B[(long long)c * (2 * m + 1) + (r - c + m)] : 0.0;
}

__global__ void __launch_bounds__(256) k_lu_block(int N, int m, int c0, const double* __restrict__ Br,
                                                  double* B, double* F, int* status) {
  __shared__ double D[kTB][kTB + 1];        // diagonal block: U on and above, work below
  __shared__ double L[kTB][kTB + 1];        // its multipliers l_rq (r > q)
  __shared__ double dinv[kTB];              // 1 / u_qq
  __shared__ double V[kTB][kTB + 1];        // my L-panel rows: a_rq in, l_rq out
  __shared__ double H[kTB][kTB + 1];        // my U-panel columns: H[q][k] = a_{q, cc0+k} in, u out
  const int w = 2 * m + 1;
  const int c1 = min(c0 + kTB, N) - 1;
  const int tb = c1 - c0 + 1;
  const int tid = threadIdx.x;
  const int rlo = c1 + 1;
  const int rhi = min(c1 + m, N - 1);
  const int nb = rhi >= rlo ? (rhi - rlo + kTB) / kTB : 0;
  const int bi = nb > 0 ? (int)blockIdx.x / nb : 0, bj = nb > 0 ? (int)blockIdx.x % nb : 0;
  const bool have_tile = nb > 0 && bi < nb;
  const int r0 = rlo + bi * kTB, cc0 = rlo + bj * kTB;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  {
    const int r = tid / kTB, q = tid % kTB;
    D[r][q] = (r < tb && q < tb) ? gband_at(Br, m, c0 + r, c0 + q) : 0.0;
    V[r][q] = (have_tile && r0 + r <= rhi && q < tb) ? gband_at(Br, m, r0 + r, c0 + q) : 0.0;
    H[q][r] = (have_tile && cc0 + r <= rhi && q < tb) ? gband_at(Br, m, c0 + q, cc0 + r) : 0.0;
    L[r][q] = 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    bool bad;
    dinv[0] = pivot_rcp_signed(D[0][0], bad);
    if (bad && blockIdx.x == 0) atomicOr(status, kStatSingular);
  }
  __syncthreads();
  // --- D = L_D U_D, one element a thread ---
  const int er = tid / kTB, ec = tid % kTB;
  for (int q = 0; q < tb; ++q) {
    if (er > q && er < tb) {
      const double t = D[er][q] * dinv[q];
      if (ec == q) {
        L[er][q] = t;
      } else if (ec > q && ec < tb) {
        const double v = fma(-t, D[q][ec], D[er][ec]);
        D[er][ec] = v;
        if (er == q + 1 && ec == q + 1) {     // the next pivot is final
          bool bad;
          dinv[q + 1] = pivot_rcp_signed(v, bad);
          if (bad && blockIdx.x == 0) atomicOr(status, kStatSingular);
        }
      }
    }
    __syncthreads();
  }
  // --- panels: row k of V by thread k of warp 0, column k of H by thread k
  // of warp 1 (two sub-partitions: their FP64 chains run side by side) ---
  if (tid < kTB) {
    const int k = tid;
    for (int q = 0; q < tb; ++q) {
      double s = V[k][q];
      for (int j = 0; j < q; ++j) s = fma(-V[k][j], D[j][q], s);
      V[k][q] = s * dinv[q];
    }
  } else if (tid >= 32 && tid < 32 + kTB) {
    const int k = tid - 32;
    for (int q = 0; q < tb; ++q) {
      double s = H[q][k];
      for (int j = 0; j < q; ++j) s = fma(-L[q][j], H[j][k], s);
      H[q][k] = s;
    }
  }
  __syncthreads();
  if (have_tile) {
    // trailing tile: B[r][c] -= sum_q l_rq u_qc (|r - c| < m inside the window)
    const int a = tid / kTB, bc = tid % kTB;
    const int r = r0 + a, c = cc0 + bc;
    if (r <= rhi && c <= rhi) {
      double s = 0.0;
      for (int q = 0; q < tb; ++q) s = fma(V[a][q], H[q][bc], s);
      B[(long long)c * w + (r - c + m)] -= s;
    }
    // the first tile column publishes the L rows, the first tile row the U columns
    const int k = tid / kTB, q = tid % kTB;
    if (bj == 0 && q < tb) {
      const int rr = r0 + k, col = c0 + q;
      if (rr <= rhi && rr - col <= m) F[(long long)col * w + (rr - col + m)] = V[k][q];
    }
    if (bi == 0 && q < tb) {
      const int row = c0 + q, col = cc0 + k;
      if (col <= rhi && col - row <= m) F[(long long)col * w + (row - col + m)] = H[q][k];
    }
  }
  // the first CTA publishes the diagonal block
  if (blockIdx.x == 0 && er < tb && ec < tb && er - ec <= m && ec - er <= m)
    F[(long long)(c0 + ec) * w + (er - ec + m)] = er > ec ? L[er][ec] : D[er][ec];
}

// L U x = b, one CTA, with the band LU's columns streamed through shared
// memory in chunks of kSC (as in k_ldlt_solve; 8-byte copies, since a band
// column of 2m+1 doubles starts on an 8-byte boundary only): forward with the
// multipliers l_{k+a,k} of column k, backward with u_{k-a,k} and the pivot.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src));
}

__global__ void __launch_bounds__(256) k_band_lu_solve(int N, int m, const double* __restrict__ Bc,
                                                       const double* __restrict__ rc, double* pc) {
  extern __shared__ __align__(16) double sm[];
  const int w = 2 * m + 1, mp = m + 1;
  const int chunk = kSC * mp;
  double* buf0 = sm;
  double* buf1 = sm + chunk;
  double* y = sm + 2 * chunk;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N; i += nt) y[i] = rc[i];
  const int nchunks = (N + kSC - 1) / kSC;
  // dst[c*mp + a] = l_{k0+c+a, k0+c}, a = 1..m
  auto stage_l = [&](double* dst, int k0) {
    const int nc = min(kSC, N - k0);
    for (int e = tid; e < nc * m; e += nt) {
      const int c = e / m, a = e - c * m + 1;
      cp_async8(dst + c * mp + a, Bc + (long long)(k0 + c) * w + m + a);
    }
    cp_async_commit();
  };
  // dst[c*mp + a] = u_{k0+c-a, k0+c}, a = 0..m (a = 0: the pivot)
  auto stage_u = [&](double* dst, int k0) {
    const int nc = min(kSC, N - k0);
    for (int e = tid; e < nc * mp; e += nt) {
      const int c = e / mp, a = e - c * mp;
      cp_async8(dst + c * mp + a, Bc + (long long)(k0 + c) * w + m - a);
    }
    cp_async_commit();
  };
  stage_l(buf0, 0);
  for (int ck = 0; ck < nchunks; ++ck) {
    double* cur = (ck & 1) ? buf1 : buf0;
    double* nxt = (ck & 1) ? buf0 : buf1;
    cp_async_wait_all();
    __syncthreads();
    if (ck + 1 < nchunks) stage_l(nxt, (ck + 1) * kSC);
    const int k0 = ck * kSC;
    for (int c = 0; c < kSC && k0 + c < N; ++c) {
      const int k = k0 + c;
      const double yk = y[k];
      const int amax = min(m, N - 1 - k);
      for (int a = 1 + tid; a <= amax; a += nt) y[k + a] -= cur[c * mp + a] * yk;
      __syncthreads();
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int last0 = (nchunks - 1) * kSC;
  stage_u(buf0, last0);
  for (int ck = nchunks - 1, it = 0; ck >= 0; --ck, ++it) {
    double* cur = (it & 1) ? buf1 : buf0;
    double* nxt = (it & 1) ? buf0 : buf1;
    cp_async_wait_all();
    __syncthreads();
    if (ck > 0) stage_u(nxt, (ck - 1) * kSC);
    const int k0 = ck * kSC;
    for (int c = min(kSC, N - k0) - 1; c >= 0; --c) {
      const int k = k0 + c;
      const double xk = y[k] / cur[c * mp];
      __syncthreads();                         // every thread has read y[k]
      if (tid == 0) y[k] = xk;
      const int amax = min(m, k);
      for (int a = 1 + tid; a <= amax; a += nt) y[k - a] -= cur[c * mp + a] * xk;
      __syncthreads();
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < N; i += nt) pc[i] = y[i];
}

// MSFE restriction, part 1: per dual block the 8 sums  sum_i P_i[s] r_i.
template <class TP, class TR>
__global__ void __launch_bounds__(256) k_restrict_fe_local(Geo g, CGeo c, const TP* __restrict__ P,
                                                           const TR* __restrict__ r, double* part) {
  __shared__ double sh[8 * 32];
  const int ndx = c.nc[0] + 1, ndy = c.nc[1] + 1;
  const int D = blockIdx.x;
  const int j[3] = {D % ndx, (D / ndx) % ndy, D / (ndx * ndy)};
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) dual_range(c, g, d, j[d], lo[d], hi[d]);
  const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
  const int ncell = (ex > 0 && ey > 0 && ez > 0) ? ex * ey * ez : 0;
  // products, each thread's and each warp's sums in P's precision, the sum
  // over the block's warps in FP64
  TP tacc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (threadIdx.x < ncell) {
    // thread t takes cells t, t + blockDim.x, ... of the block in x-fastest
    // order; the cell's coordinates advance by a fixed mixed-radix step
    // instead of being divided out of l
    const int st = blockDim.x;
    const int sx = st % ex, sy = (st / ex) % ey, sz = st / (ex * ey);
    int x = threadIdx.x % ex, y = (threadIdx.x / ex) % ey, z = threadIdx.x / (ex * ey);
    for (int l = threadIdx.x; l < ncell; l += st) {
      const long long i = (lo[0] + x) + g.sy * (lo[1] + y) + g.sz * (lo[2] + z);
      const TP ri = (TP)r[i];
#pragma unroll
      for (int s = 0; s < 8; ++s) tacc[s] += P[(long long)s * g.N + i] * ri;
      x += sx;
      y += sy;
      z += sz;
      if (x >= ex) { x -= ex; ++y; }
      if (y >= ey) { y -= ey; ++z; }
    }
  }
  block_sum_k<8>(tacc, sh, part + (long long)D * 8);
}

// MSFE restriction, part 2: coarse node J sums its (up to 8) dual blocks.
__global__ void k_restrict_fe_gather(CGeo c, const double* __restrict__ part, const int* __restrict__ perm,
                                     double* rc) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= c.Nc) return;
  const int Jc[3] = {J % c.nc[0], (J / c.nc[0]) % c.nc[1], J / (c.nc[0] * c.nc[1])};
  const int ndx = c.nc[0] + 1, ndy = c.nc[1] + 1;
  double s = 0.0;
  for (int bz = 0; bz < 2; ++bz)
    for (int by = 0; by < 2; ++by)
      for (int bx = 0; bx < 2; ++bx) {
        // dual block j = J + bit: J is its lower corner (slot bit 0) when bit = 1
        const int jx = Jc[0] + bx, jy = Jc[1] + by, jz = Jc[2] + bz;
        const int slot = (bx ? 0 : 1) | (by ? 0 : 2) | (bz ? 0 : 4);
        const int D = jx + ndx * (jy + ndy * jz);
        s += part[(long long)D * 8 + slot];
      }
  rc[perm[J]] = s;
}

// MSFV restriction: block sums of r.
__global__ void __launch_bounds__(256) k_restrict_fv(Geo g, CGeo c, const double* __restrict__ r,
                                                     const int* __restrict__ perm, double* rc) {
  __shared__ double sh[32];
  const int I = blockIdx.x;
  const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
  const int bx = c.b[0], by = c.b[1], bz = c.b[2];
  double acc[1] = {0.0};
  if ((int)threadIdx.x < bx * by * bz) {
    // cells t, t + blockDim.x, ... in x-fastest order, coordinates advanced
    // by a fixed mixed-radix step (as in k_restrict_fe_local)
    const int st = blockDim.x;
    const int sx = st % bx, sy = (st / bx) % by, sz = st / (bx * by);
    int x = threadIdx.x % bx, y = (threadIdx.x / bx) % by, z = threadIdx.x / (bx * by);
    for (int l = threadIdx.x; l < bx * by * bz; l += st) {
      acc[0] += r[(Ic[0] * bx + x) + g.sy * (Ic[1] * by + y) + g.sz * (Ic[2] * bz + z)];
      x += sx;
      y += sy;
      z += sz;
      if (x >= bx) { x -= bx; ++y; }
      if (y >= by) { y -= by; ++z; }
    }
  }
  double out;
  block_sum_k<1>(acc, sh, &out);
  // block_sum_k writes through thread 0 only when K == 1
  if (threadIdx.x == 0) rc[perm[I]] = out;
}

// p += P p_c (FP64), or delta = P p_c (the mixed-precision preconditioner:
// P, p_c and delta in FP32); the sum is formed in p_c's precision.  Warps
// take whole x-rows.  A row's y and z corners are fixed, so its coarse
// values (4 corner pairs x the coarse x-nodes) are staged in the warp's
// shared memory once per row, and each cell's two x-corners come from the
// per-x table jxt: a cell costs its 8 P loads and 8 shared reads, with no
// index division and no gather through the permutation.
template <class TP, class TC, class TO, bool kSet>
__global__ void k_prolong(Geo g, CGeo c, const TP* __restrict__ P, const TC* __restrict__ pc,
                          const int* __restrict__ perm, const int* __restrict__ jxt, TO* p) {
  extern __shared__ __align__(16) unsigned char prolong_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int ncx = c.nc[0];
  TC* cv = reinterpret_cast<TC*>(prolong_smem) + (size_t)warp * 4 * ncx;
  const unsigned rows = (unsigned)g.ny * (unsigned)g.nz;
  for (unsigned row = blockIdx.x * nw + warp; row < rows; row += gridDim.x * nw) {
    const int y = (int)(row % (unsigned)g.ny), z = (int)(row / (unsigned)g.ny);
    const int Jy[2] = {corner_d(c, 1, y, 0), corner_d(c, 1, y, 1)};
    const int Jz[2] = {corner_d(c, 2, z, 0), corner_d(c, 2, z, 1)};
    // corner pair k = (y bit, z bit) = (k & 1, k >> 1), the slot's bits 1 and 2
    unsigned ok = 0;
    __syncwarp();                                // the previous row's reads are done
    for (int k = 0; k < 4; ++k) {
      const int jy = Jy[k & 1], jz = Jz[k >> 1];
      if (jy < 0 || jz < 0) continue;            // uniform across the warp
      ok |= 1u << k;
      for (int jx = lane; jx < ncx; jx += 32) cv[k * ncx + jx] = pc[perm[jx + ncx * (jy + c.nc[1] * jz)]];
    }
    __syncwarp();
    const long long base = g.sy * y + g.sz * z;
    for (int x = lane; x < g.nx; x += 32) {
      const long long i = base + x;
      const int Jx[2] = {jxt[2 * x], jxt[2 * x + 1]};
      TC s = TC(0);
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) {
        const int jx = Jx[sl & 1], k = (sl >> 1) & 3;
        if (jx < 0 || !((ok >> k) & 1u)) continue;
        s += (TC)P[(long long)sl * g.N + i] * cv[k * ncx + jx];
      }
      if (kSet) p[i] = (TO)s;
      else p[i] += (TO)s;
    }
  }
}

__global__ void k_to_single(int n, const double* __restrict__ a, float* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

}  // namespace

cudaError_t launch_galerkin_fe(const Geo& g, const CGeo& c, bool single, bool nonsym, Buffers& b,
                               cudaStream_t s) {
  if (nonsym) {
    const int T = 128;
    if (single)
      k_galerkin_fe_ns<float><<<c.Nc, T, 27 * T * sizeof(double), s>>>(
          g, c, b.f32.P, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, b.Acs);
    else
      k_galerkin_fe_ns<double><<<c.Nc, T, 27 * T * sizeof(double), s>>>(
          g, c, b.P, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, b.Acs);
    count_launches(1);
    return cudaGetLastError();
  }
  const int nd = (c.nc[0] + 1) * (c.nc[1] + 1) * (c.nc[2] + 1);
  if (single)
    k_galerkin_fe_local<float><<<nd, 256, 0, s>>>(g, c, b.f32.P, b.Ad, b.Ax, b.Ay, b.Az, b.loc);
  else
    k_galerkin_fe_local<double><<<nd, 256, 0, s>>>(g, c, b.P, b.Ad, b.Ax, b.Ay, b.Az, b.loc);
  count_launches(1);
  k_galerkin_fe_gather<<<(27 * c.Nc + 255) / 256, 256, 0, s>>>(c, b.loc, b.Acs); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_galerkin_fv(const Geo& g, const CGeo& c, bool single, bool nonsym, Buffers& b,
                               cudaStream_t s) {
  const int T = 128;
  if (single)
    k_galerkin_fv<float><<<c.Nc, T, 27 * T * sizeof(double), s>>>(
        g, c, b.f32.P, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, nonsym ? 1 : 0, b.Acs);
  else
    k_galerkin_fv<double><<<c.Nc, T, 27 * T * sizeof(double), s>>>(
        g, c, b.P, b.Ad, b.Ax, b.Ay, b.Az, b.Axu, b.Ayu, b.Azu, nonsym ? 1 : 0, b.Acs);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_band_fill(const CGeo& c, int m, int sym, Buffers& b, cudaStream_t s) {
  const size_t len = sym ? (size_t)c.Nc * (m + 1) : (size_t)c.Nc * (2 * m + 1);
  cudaError_t e = cudaMemsetAsync(b.band, 0, sizeof(double) * len, s);
  if (e != cudaSuccess) return e;
  k_band_fill<double><<<(27 * c.Nc + 255) / 256, 256, 0, s>>>(c, m, sym, b.Acs, b.perm, b.band);
  count_launches(1);
  return cudaGetLastError();
}

// The symmetric band factorisation: one launch per block of kTB columns,
// each allowed to start while the previous one drains (programmatic
// dependent launch; the kernel waits for its predecessor).
template <class T>
static cudaError_t ldlt_launches(int Nc, int m, T* band, T* Lc, int* status, cudaStream_t s,
                                 int& launches) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  for (int c0 = 0; c0 < Nc; c0 += kTB) {
    const int c1 = (c0 + kTB < Nc ? c0 + kTB : Nc) - 1;
    const int rhi = (c1 + m < Nc - 1) ? c1 + m : Nc - 1;
    const int nb = rhi > c1 ? (rhi - c1 - 1 + kTB) / kTB : 0;
    const int grid = nb > 0 ? nb * (nb + 1) / 2 : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = c0 == 0 ? 0 : 1;      // the first block follows the band fill normally
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_ldlt_block<T>, Nc, m, c0, (const T*)band, band, Lc,
                                       status);
    if (e != cudaSuccess) return e;
    ++launches;
  }
  return cudaSuccess;
}

long long coarse_ldz(int Nc) { return ((long long)Nc + kZS - 1) / kZS * kZS; }

static int coarse_ring(int m) {
  int r = 32;
  while (r < m + 32) r *= 2;
  return r;
}

static int zinv_smem(int m) {
  return (int)sizeof(float) * 3 * (m + 32) * 32 +
         (int)sizeof(float4) * (3 * (kZQ - 1) * kZG * 32 + kZG * 2 * coarse_ring(m));
}

long long coarse_part_len(int Nc) { return ((long long)Nc + kZK - 1) / kZK * coarse_ldz(Nc); }

bool coarse_inverse_ok(int Nc, int m) {
  // forming Z costs about Nc^2 m / 2 FP32 FMAs and holds Nc x ldz floats
  const double work = (double)Nc * (double)Nc * (double)m;
  const double bytes = 4.0 * (double)Nc * (double)coarse_ldz(Nc);
  return Nc > 0 && work <= 2e10 && bytes <= 1073741824.0 && zinv_smem(m) <= 200 * 1024;
}

cudaError_t launch_coarse_factor_inv(const CGeo& c, int m, Buffers& b, cudaStream_t s) {
  // the FP64 band L D L^T (the coarse-system factorisation stays FP64), then
  // its FP32 copy, from which k_coarse_zinv forms Z
  const int Nc = c.Nc;
  cudaError_t e = launch_band_fill(c, m, 1, b, s);
  if (e != cudaSuccess) return e;
  int launches = 0;
  e = ldlt_launches<double>(Nc, m, b.band, b.Lc, b.status, s, launches);
  if (e != cudaSuccess) return e;
  const long long n = (long long)Nc * (m + 1);
  k_to_single<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, b.Lc, b.f32.Lc);
  count_launches(launches + 1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_zinv(int Nc, int m, Buffers& b, cudaStream_t s) {
  const int smem = zinv_smem(m);
  cudaError_t e = raise_smem_limit(k_coarse_zinv, smem);
  if (e != cudaSuccess) return e;
  k_coarse_zinv<<<(Nc + kZCols - 1) / kZCols, kZT, smem, s>>>(Nc, m, coarse_ring(m), b.f32.Lc, b.f32.Z,
                                                  coarse_ldz(Nc));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_f32(int Nc, int m, Buffers& b, cudaStream_t s) {
  SingleBuffers& f = b.f32;
  const long long ldz = coarse_ldz(Nc);
  const dim3 grid((unsigned)((Nc + kZS - 1) / kZS), (unsigned)((Nc + kZK - 1) / kZK));
  k_coarse_zlower<<<grid, 256, 0, s>>>(Nc, f.Z, ldz, b.rc, f.zpart);
  k_coarse_tsum<<<(Nc + 255) / 256, 256, 0, s>>>(Nc, m, f.Lc, f.zpart, ldz, f.tc);
  k_coarse_zupper<<<(Nc + 7) / 8, 256, 0, s>>>(Nc, f.Z, ldz, f.tc, f.pc);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_band_factor(int Nc, int m, int sym, Buffers& b, cudaStream_t s) {
  // one launch per column block, each allowed to start while the previous
  // one drains (programmatic dependent launch; the kernel waits for it)
  int launches = 0;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  if (!sym) {
    for (int c0 = 0; c0 < Nc; c0 += kTB) {
      const int c1 = (c0 + kTB < Nc ? c0 + kTB : Nc) - 1;
      const int rhi = (c1 + m < Nc - 1) ? c1 + m : Nc - 1;
      const int nb = rhi > c1 ? (rhi - c1 - 1 + kTB) / kTB : 0;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nb > 0 ? nb * nb : 1);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = c0 == 0 ? 0 : 1;    // the first block follows the band fill normally
      cudaError_t e = cudaLaunchKernelEx(&cfg, k_lu_block, Nc, m, c0, (const double*)b.band,
                                         b.band, b.Fc, b.status);
      if (e != cudaSuccess) return e;
      ++launches;
    }
    count_launches(launches);
    return cudaGetLastError();
  }
  cudaError_t e = ldlt_launches<double>(Nc, m, b.band, b.Lc, b.status, s, launches);
  if (e != cudaSuccess) return e;
  const long long n = (long long)Nc * (m + 1);
  k_ldlt_rows<<<(int)((n + 255) / 256), 256, 0, s>>>(Nc, m, b.Lc, b.Lr);
  k_coarse_prep<<<(Nc + kCB - 1) / kCB, 256, 0, s>>>(Nc, m, b.Lc, b.cblk, b.cdinv);
  count_launches(launches + 2);
  if (b.f32.Lc) {
    // FP32 copy of the factor for the mixed-precision substitution
    const long long nb = coarse_blocks_len(Nc);
    k_to_single<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, b.Lc, b.f32.Lc);
    k_to_single<<<(int)((n + 255) / 256), 256, 0, s>>>((int)n, b.Lr, b.f32.Lr);
    k_to_single<<<(int)((nb + 255) / 256), 256, 0, s>>>((int)nb, b.cblk, b.f32.cblk);
    k_to_single<<<(Nc + 255) / 256, 256, 0, s>>>(Nc, b.cdinv, b.f32.cdinv);
    count_launches(4);
  }
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Geo& g, const CGeo& c, int kind, const double* r, bool single,
                            Buffers& b, cudaStream_t s) {
  if (kind == 0) {
    const int nd = (c.nc[0] + 1) * (c.nc[1] + 1) * (c.nc[2] + 1);
    // mixed precision: the FP32 copy of the handle's residual (written with it)
    if (single && r == b.r) k_restrict_fe_local<float, float><<<nd, 256, 0, s>>>(g, c, b.f32.P, b.f32.r, b.loc);
    else if (single) k_restrict_fe_local<float, double><<<nd, 256, 0, s>>>(g, c, b.f32.P, r, b.loc);
    else k_restrict_fe_local<double, double><<<nd, 256, 0, s>>>(g, c, b.P, r, b.loc);
    count_launches(1);
    k_restrict_fe_gather<<<(c.Nc + 127) / 128, 128, 0, s>>>(c, b.loc, b.perm, b.rc); count_launches(1);
  } else {
    k_restrict_fv<<<c.Nc, 256, 0, s>>>(g, c, r, b.perm, b.rc); count_launches(1);
  }
  return cudaGetLastError();
}

long long coarse_blocks_len(int Nc) {
  return (long long)((Nc + kCB - 1) / kCB) * kCBlocks * kCB * kCB;
}

// the device's opt-in shared memory per CTA
static int coarse_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 48 * 1024;
  return v;
}

static int coarse_cluster_smem(int Nc, int bytes = 8) {
  return bytes * 2 * ((Nc + kCB - 1) / kCB) * kCB;
}

bool coarse_cluster_ok(int Nc, int max_smem) {
  const int smem = coarse_cluster_smem(Nc);
  if (smem > max_smem) return false;
  if (raise_smem_limit(k_coarse_solve_cluster<double>, smem) != cudaSuccess ||
      raise_smem_limit(k_coarse_solve_cluster<float>, coarse_cluster_smem(Nc, 4)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCC);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kCC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_coarse_solve_cluster<double>, &cfg) != cudaSuccess) n = 0;
  cudaGetLastError();
  return n > 0;
}

cudaError_t launch_band_solve(int Nc, int m, int sym, bool cluster, bool single, Buffers& b,
                              cudaStream_t s) {
  if (sym && cluster) {
    cudaError_t e = cudaMemsetAsync(b.cabort, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCC);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = (size_t)coarse_cluster_smem(Nc, single ? 4 : 8);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (single) {
      // FP32 substitution with the FP64 factor's FP32 copy; the result goes
      // straight to the FP32 prolongation
      const SingleBuffers& f = b.f32;
      e = cudaLaunchKernelEx(&cfg, k_coarse_solve_cluster<float>, Nc, m, (const float*)f.Lc,
                             (const float*)f.Lr, (const float*)f.cblk, (const float*)f.cdinv,
                             (const double*)b.rc, b.f32.pc, b.cabort, b.status);
    } else {
      e = cudaLaunchKernelEx(&cfg, k_coarse_solve_cluster<double>, Nc, m, (const double*)b.Lc,
                             (const double*)b.Lr, (const double*)b.cblk, (const double*)b.cdinv,
                             (const double*)b.rc, b.pc, b.cabort, b.status);
    }
    count_launches(1);
    return e;
  }
  if (sym) {
    const int smem = (int)sizeof(double) * (2 * kSC * (m + 1) + Nc);
    if (smem <= coarse_smem_optin()) {
      cudaError_t e = raise_smem_limit(k_ldlt_solve, smem);
      if (e != cudaSuccess) return e;
      k_ldlt_solve<<<1, 256, smem, s>>>(Nc, m, b.Lc, b.Lr, b.rc, b.pc);
    } else {
      // vectors in global memory (b.ywork holds y)
      k_coarse_solve_global<<<1, 256, 0, s>>>(Nc, m, b.Lc, b.Lr, b.cblk, b.cdinv, b.rc, b.ywork,
                                             b.pc);
    }
  } else {
    const int smem = (int)sizeof(double) * (2 * kSC * (m + 1) + Nc);
    cudaError_t e = raise_smem_limit(k_band_lu_solve, smem);
    if (e != cudaSuccess) return e;
    k_band_lu_solve<<<1, 256, smem, s>>>(Nc, m, b.Fc, b.rc, b.pc);
  }
  count_launches(1);
  if (single) {
    k_to_single<<<(Nc + 255) / 256, 256, 0, s>>>(Nc, b.pc, b.f32.pc);
    count_launches(1);
  }
  return cudaGetLastError();
}

// warps a CTA for k_prolong: 8, fewer when the staged coarse values of 8
// warps would not fit in 48 KB of shared memory
static int prolong_warps(const CGeo& c, int elem) {
  const int per = 4 * c.nc[0] * elem;
  int w = 8;
  while (w > 1 && w * per > 48 * 1024) --w;
  return w;
}

template <class TP, class TC, class TO, bool kSet>
static cudaError_t prolong(const Geo& g, const CGeo& c, const TP* P, const TC* pc, Buffers& b, TO* p,
                           cudaStream_t s) {
  const int w = prolong_warps(c, (int)sizeof(TC));
  const int smem = w * 4 * c.nc[0] * (int)sizeof(TC);
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit(k_prolong<TP, TC, TO, kSet>, smem);
    if (e != cudaSuccess) return e;
  }
  const int blocks = (int)(((long long)g.ny * g.nz + w - 1) / w);   // one warp per x-row
  k_prolong<TP, TC, TO, kSet><<<blocks, 32 * w, smem, s>>>(g, c, P, pc, b.perm, b.jxt, p);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(const Geo& g, const CGeo& c, bool single, Buffers& b,
                               cudaStream_t s) {
  // the coarse solution of the mixed preconditioner is already in b.f32.pc
  if (single) return prolong<float, float, float, true>(g, c, b.f32.P, b.f32.pc, b, b.f32.d, s);
  return prolong<double, double, double, false>(g, c, b.P, b.pc, b, b.p, s);
}

cudaError_t launch_prolong_to_p(const Geo& g, const CGeo& c, bool single, Buffers& b,
                                cudaStream_t s) {
  if (single) return prolong<float, double, double, false>(g, c, b.f32.P, b.pc, b, b.p, s);
  return prolong<double, double, double, false>(g, c, b.P, b.pc, b, b.p, s);
}

}  // namespace cams
