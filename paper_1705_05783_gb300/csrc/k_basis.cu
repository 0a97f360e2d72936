// Multiscale basis construction (Sec. 3, Eqs. 8-12) with the wirebasket
// reduced-problem conditions, and the adaptive-update flags of Sec. 4.1.2.
//
// Every edge segment, face patch and dual-block interior is one local SPD
// problem  M_e P_e = -A_b[e, lower] P[lower]  (level-(k+1) neighbours lumped
// onto the diagonal).  One CTA solves one entity: it orders the entity's
// cells with the shortest direction fastest, which makes M_e banded with
// half-width m = product of the two shortest extents, and runs a
// right-looking banded LDL^T whose active (m+1)x(m+1) window lives in shared
// memory as a ring of rows.  All right-hand sides (one per corner vertex,
// 2^free) are carried through the forward elimination in shared memory; the
// finished rows of L stream to a per-CTA scratch slice (L2-resident) for the
// backward substitution.  No atomics, so the result is deterministic.  The
// local solve and P are FP64, or FP32 for the mixed-precision preconditioner
// (the basis operator is read in FP64 and rounded).
//
// The same kernels in their kCF form apply the correction functions of
// Table 1 step 4 (Sec. 3): the same local systems with one right-hand side,
// the fine residual r minus the couplings to the correction values Psi
// already found on the lower levels (zero on the vertices), launched level
// by level like the basis stages.
#include "cams_internal.h"

namespace cams {

namespace {

__device__ __forceinline__ double coupling(const Geo& g, const double* Abx, const double* Aby,
                                           const double* Abz, int d, long long i) {
  // A_b entry between i and i - e_d (stored at the upper cell)
  return d == 0 ? Abx[i] : (d == 1 ? Aby[i] : Abz[i]);
}

__device__ __forceinline__ long long gstride(const Geo& g, int d) {
  return d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
}

__device__ __forceinline__ int gextent(const Geo& g, int d) {
  return d == 0 ? g.nx : (d == 1 ? g.ny : g.nz);
}

// global slot (bits over x,y,z) of the entity's r-th right-hand side
__device__ __forceinline__ int slot_of(int r, int free_mask) {
  int s = 0, k = 0;
  for (int d = 0; d < 3; ++d)
    if (free_mask & (1 << d)) {
      if (r & (1 << k)) s |= 1 << d;
      ++k;
    }
  return s;
}

struct Local {
  int c[3];        // coordinates
  long long i;     // global cell
};

__device__ __forceinline__ Local local_cell(const Entity& E, int l) {
  Local L;
  const int L0 = E.L[E.ord[0]], L1 = E.L[E.ord[1]];
  int t[3];
  t[0] = l % L0;
  t[1] = (l / L0) % L1;
  t[2] = l / (L0 * L1);
  for (int k = 0; k < 3; ++k) L.c[E.ord[k]] = E.org[E.ord[k]] + t[k];
  return L;
}

__device__ __forceinline__ int local_stride(const Entity& E, int d) {
  const int L0 = E.L[E.ord[0]], L1 = E.L[E.ord[1]];
  return d == E.ord[0] ? 1 : (d == E.ord[1] ? L0 : L0 * L1);
}

// Build row l of M (lower band, ring slot) and the right-hand sides of row l:
// one per corner vertex for the basis functions, or (kCF) the single
// correction-function right-hand side r_i - sum over lower neighbours j of
// a_ij Psi_j.
template <class T, bool kCF>
__device__ void build_row(const Geo& g, const Entity& E, int l, T* Wrow, T* Yrow,
                          const double* Abd, const double* Abx, const double* Aby,
                          const double* Abz, const T* P, const double* rin, const T* psi) {
  Local c = local_cell(E, l);
  const long long i = c.c[0] + g.sy * c.c[1] + g.sz * c.c[2];
  for (int dd = 0; dd <= E.m; ++dd) Wrow[dd] = T(0);
  if constexpr (kCF) {
    Yrow[0] = T(rin[i]);
  } else {
    for (int r = 0; r < E.nrhs; ++r) Yrow[r] = T(0);
  }
  double diag = Abd[i];
  for (int d = 0; d < 3; ++d) {
    const int n_d = gextent(g, d);
    if (n_d == 1) continue;
    const long long sd = gstride(g, d);
    const double lo = c.c[d] > 0 ? coupling(g, Abx, Aby, Abz, d, i) : 0.0;          // to i - e_d
    const double up = c.c[d] < n_d - 1 ? coupling(g, Abx, Aby, Abz, d, i + sd) : 0.0; // to i + e_d
    if (!(E.free_mask & (1 << d))) {
      // lattice direction: neighbours are one level higher -> lumped
      diag += lo;
      diag += up;
      continue;
    }
    // free direction: inside the box -> band entry; outside -> known data
    if (c.c[d] > E.org[d]) {
      Wrow[local_stride(E, d)] = T(lo);
    } else if (c.c[d] > 0) {
      const long long j = i - sd;
      if constexpr (kCF) {
        Yrow[0] -= T(lo) * psi[j];
      } else {
        for (int r = 0; r < E.nrhs; ++r) {
          const int s = slot_of(r, E.free_mask);
          if (!(s & (1 << d))) Yrow[r] -= T(lo) * P[(long long)s * g.N + j];
        }
      }
    }
    if (c.c[d] < E.org[d] + E.L[d] - 1) {
      // upper in-box neighbour: its entry is stored in the neighbour's row
    } else if (c.c[d] < n_d - 1) {
      const long long j = i + sd;
      if constexpr (kCF) {
        Yrow[0] -= T(up) * psi[j];
      } else {
        for (int r = 0; r < E.nrhs; ++r) {
          const int s = slot_of(r, E.free_mask);
          if (s & (1 << d)) Yrow[r] -= T(up) * P[(long long)(s & ~(1 << d)) * g.N + j];
        }
      }
    }
  }
  Wrow[0] = T(diag);
}

template <class T>
__global__ void k_vertices(Geo g, CGeo c, T* P) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= c.Nc) return;
  const int Jx = J % c.nc[0], Jy = (J / c.nc[0]) % c.nc[1], Jz = J / (c.nc[0] * c.nc[1]);
  const long long v = (Jx * c.b[0] + c.o[0]) + g.sy * (Jy * c.b[1] + c.o[1]) +
                      g.sz * (Jz * c.b[2] + c.o[2]);
  for (int s = 0; s < 8; ++s) P[(long long)s * g.N + v] = (s == 0) ? T(1) : T(0);
}

template <class T, bool kCF>
__global__ void __launch_bounds__(256) k_entity_solve(
    Geo g, const Entity* __restrict__ ents, int count, const unsigned char* __restrict__ flag,
    int adaptive, const double* __restrict__ Abd, const double* __restrict__ Abx,
    const double* __restrict__ Aby, const double* __restrict__ Abz, T* P, double* snap,
    T* lscratch, long long lstride, int* status, const double* __restrict__ rin, T* psi,
    double* padd) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* Lg = lscratch + (long long)blockIdx.x * lstride;
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    if (flag && !flag[e]) continue;
    const Entity E = ents[e];
    const int n = E.n, m = E.m, nr = kCF ? 1 : E.nrhs, mp = m + 1;
    T* W = sm;                      // mp * mp ring
    T* Y = W + mp * mp;             // n * nr
    T* lcol = Y + n * nr;           // mp
    T* ucol = lcol + mp;            // mp
    // rows 0..m go to the ring; rows beyond the first window are staged in
    // the scratch slice (row l at l*mp) until they enter the ring
    for (int l = tid; l < n; l += nt) {
      T* row = (l <= m) ? W + l * mp : Lg + (long long)l * mp;
      build_row<T, kCF>(g, E, l, row, Y + l * nr, Abd, Abx, Aby, Abz, P, rin, psi);
    }
    __syncthreads();
    // banded LDL^T with forward elimination of the right-hand sides.  The
    // reciprocal pivot 1/d_k is formed once, by the thread that completes
    // d_k, and kept in the factor (slot 0 of row k) for the D^{-1} step.
    __shared__ T s_inv;
    const int lnr = __ffs(nr) - 1;                 // nr is a power of two
    if (tid == 0) {
      T d0 = W[0];
      if (!(d0 > T(0)) || !isfinite(d0)) {
        atomicOr(status, kStatSingular);
        d0 = T(1);
      }
      s_inv = T(1) / d0;
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      const int amax = min(m, n - 1 - k);
      const int ks = k % mp;                       // ring slot of row k
      const T inv = s_inv;
      for (int a = 1 + tid; a <= amax; a += nt) {
        int sl = ks + a;
        if (sl >= mp) sl -= mp;
        T* w = W + sl * mp + a;
        const T u = *w;
        ucol[a] = u;
        lcol[a] = u * inv;
        *w = u * inv;
      }
      // row k is final: store (1/d_k, l_{k,k-1}, ..., l_{k,k-m})
      for (int dd = tid; dd <= m; dd += nt) Lg[(long long)k * mp + dd] = (dd == 0) ? inv : W[ks * mp + dd];
      __syncthreads();
      // rank-1 update of the trailing window (lower triangle only): warp w
      // takes rows a = 1 + w, 1 + w + nw, ..., its lanes the columns b <= a
      for (int a = 1 + (tid >> 5); a <= amax; a += nt >> 5) {
        int sl = ks + a;
        if (sl >= mp) sl -= mp;
        T* wr = W + sl * mp + a;                   // wr[-b] = W(k+a, k+b)
        const T la = lcol[a];
        for (int bb = 1 + (tid & 31); bb <= a; bb += 32) wr[-bb] -= la * ucol[bb];
        if (a == 1 && (tid & 31) == 0) {           // d_{k+1} is final: its reciprocal
          T d1 = wr[-1];
          if (!(d1 > T(0)) || !isfinite(d1)) {
            atomicOr(status, kStatSingular);
            d1 = T(1);
          }
          s_inv = T(1) / d1;
        }
      }
      for (int t = tid; t < (amax << lnr); t += nt) {
        const int a = (t >> lnr) + 1, r = t & (nr - 1);
        Y[(k + a) * nr + r] -= lcol[a] * Y[k * nr + r];
      }
      // the slot of row k receives row k + m + 1
      const int nxt = k + m + 1;
      if (nxt < n) {
        T* dst = W + ks * mp;
        // copy the band part that was prepared in the scratch row
        for (int dd = tid; dd <= m; dd += nt) dst[dd] = Lg[(long long)nxt * mp + dd];
      }
      __syncthreads();
    }
    // D^{-1}
    for (int t = tid; t < n * nr; t += nt) Y[t] *= Lg[(long long)(t >> lnr) * mp];
    __syncthreads();
    // backward substitution with L^T
    for (int k = n - 1; k > 0; --k) {
      const int amax = min(m, k);
      for (int t = tid; t < (amax << lnr); t += nt) {
        const int dd = (t >> lnr) + 1, r = t & (nr - 1);
        Y[(k - dd) * nr + r] -= Lg[(long long)k * mp + dd] * Y[k * nr + r];
      }
      __syncthreads();
    }
    // write the basis values (slots on lattice bits stay zero), or the
    // correction values (and p += Psi when padd is given)
    for (int l = tid; l < n; l += nt) {
      Local c = local_cell(E, l);
      const long long i = c.c[0] + g.sy * c.c[1] + g.sz * c.c[2];
      if constexpr (kCF) {
        psi[i] = Y[l];
        if (padd) padd[i] += (double)Y[l];
        continue;
      }
      for (int s = 0; s < 8; ++s) P[(long long)s * g.N + i] = T(0);
      for (int r = 0; r < nr; ++r) P[(long long)slot_of(r, E.free_mask) * g.N + i] = Y[l * nr + r];
      if (adaptive) {
        snap[0 * g.N + i] = Abd[i];
        snap[1 * g.N + i] = c.c[0] > 0 ? Abx[i] : 0.0;
        snap[2 * g.N + i] = c.c[0] < g.nx - 1 ? Abx[i + 1] : 0.0;
        snap[3 * g.N + i] = c.c[1] > 0 ? Aby[i] : 0.0;
        snap[4 * g.N + i] = c.c[1] < g.ny - 1 ? Aby[i + g.sy] : 0.0;
        snap[5 * g.N + i] = c.c[2] > 0 ? Abz[i] : 0.0;
        snap[6 * g.N + i] = c.c[2] < g.nz - 1 ? Abz[i + g.sz] : 0.0;
      }
    }
    __syncthreads();
  }
}

// ---- blocked variant for the large local problems (dual-block interiors) ----
// The per-pivot rank-1 update above issues several instructions per FMA
// (ring addressing, partial warps), which bounds it.  Here pivots go in
// panels of kKB: the panel's columns are eliminated pivot by pivot (only
// within the panel), then the trailing window takes one rank-kKB update in
// 4x4 register tiles, and the right-hand sides one kKB-term update.  The
// ring holds m + kKB rows; the backward substitution also goes kKB rows at a
// time, with those rows of L staged in shared memory.  Same arithmetic as the
// per-pivot kernel up to the order of the additions.
constexpr int kKB = 8;
constexpr int kLPS = kKB + 1;   // panel row stride (odd: no shared-memory bank conflicts)

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

template <class T, bool kCF>
__global__ void __launch_bounds__(256) k_entity_solve_blk(
    Geo g, const Entity* __restrict__ ents, int count, const unsigned char* __restrict__ flag,
    int adaptive, const double* __restrict__ Abd, const double* __restrict__ Abx,
    const double* __restrict__ Aby, const double* __restrict__ Abz, T* P, double* snap,
    T* lscratch, long long lstride, int* status, const double* __restrict__ rin, T* psi,
    double* padd, unsigned char* gwork, long long gbytes) {
  // the working window, right-hand sides and panel: dynamic shared memory,
  // or this CTA's slice of gwork when an entity's window is too large for it
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = gwork ? reinterpret_cast<T*>(gwork + (long long)blockIdx.x * gbytes)
                : reinterpret_cast<T*>(sm_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* Lg = lscratch + (long long)blockIdx.x * lstride;
  __shared__ T s_d[kKB], s_dinv[kKB];
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    if (flag && !flag[e]) continue;
    const Entity E = ents[e];
    const int n = E.n, m = E.m, nr = kCF ? 1 : E.nrhs, mp = m + 1, R = m + kKB;
    const int lnr = __ffs(nr) - 1;                 // nr is a power of two
    T* W = sm;                                     // ring: row i in slot i % R, entry (i, i-dd) at dd
    T* Y = W + round4(R * mp);                     // n x nr right-hand sides
    T* Lp = Y + round4(n * nr);                    // panel: Lp[(i-k)*kLPS + q] = l_{i,k+q}
    T* Ls = W;                                     // backward sweep: kKB staged rows of L
    for (int l = tid; l < n; l += nt) {
      T* row = (l < R) ? W + l * mp : Lg + (long long)l * mp;
      build_row<T, kCF>(g, E, l, row, Y + l * nr, Abd, Abx, Aby, Abz, P, rin, psi);
    }
    __syncthreads();
    for (int k = 0; k < n; k += kKB) {
      const int kb = min(kKB, n - k);
      const int k_slot = k % R;                    // ring slot of row k
      const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
      for (int t = tid; t < (m + kKB) * kLPS; t += nt) Lp[t] = T(0);
      if constexpr (sizeof(T) == 4) {
        // FP32: the panel's diagonal block by one warp, then its rows below
        // by one thread a row (three barriers a panel)
        __syncthreads();
        // --- the panel's kb x kb diagonal block, by warp 0: lane r holds row
        // k+r (x[c] = a_{k+r,k+c}, c <= r); after pivot c, lanes r > c hold
        // l_{k+r,k+c} and have updated their later entries.  Then the
        // right-hand sides of the panel's rows, lane r' < nr one column. ---
        if (warp == 0) {
          T x[kKB];
          int rs = k_slot + lane;                    // slot of row k+lane
          if (rs >= R) rs -= R;
  #pragma unroll
          for (int c = 0; c < kKB; ++c)
            x[c] = (lane < kb && c <= lane && lane - c <= m) ? W[rs * mp + (lane - c)] : T(0);
  #pragma unroll
          for (int c = 0; c < kKB; ++c) {
            if (c < kb) {                            // uniform
              T d = __shfl_sync(0xffffffffu, x[c], c);
              if (!(d > T(0)) || !isfinite(d)) {
                if (lane == 0) atomicOr(status, kStatSingular);
                d = T(1);
              }
              const T dinv = T(1) / d;
              if (lane == c) { s_d[c] = d; s_dinv[c] = dinv; }
              if (lane > c && lane < kb) x[c] *= dinv;
              // x[c'] -= l_{r,c} d_c l_{c',c} for c < c' <= r (the diagonal too)
  #pragma unroll
              for (int cp = c + 1; cp < kKB; ++cp) {
                const T lcp = __shfl_sync(0xffffffffu, x[c], cp);
                if (cp <= lane && lane < kb) x[cp] -= x[c] * d * lcp;
              }
            }
          }
          if (lane < kb) {
  #pragma unroll
            for (int c = 0; c < kKB; ++c) {
              if (c < lane) {
                if (lane - c <= m) W[rs * mp + (lane - c)] = x[c];
                Lp[lane * kLPS + c] = x[c];
              }
            }
          }
          if (lane == 0)
            for (int q = kb; q < kKB; ++q) { s_d[q] = T(0); s_dinv[q] = T(0); }
          // forward substitution of the panel's rows in the right-hand sides
  #pragma unroll
          for (int r = 1; r < kKB; ++r) {
  #pragma unroll
            for (int c = 0; c < kKB; ++c) {
              if (c < r) {
                const T l = __shfl_sync(0xffffffffu, x[c], r);
                if (r < kb && lane < nr) Y[(k + r) * nr + lane] -= l * Y[(k + c) * nr + lane];
              }
            }
          }
        }
        __syncthreads();
        // --- the panel's rows below the block, one thread a row:
        // l_{i,k+c} = (a_{i,k+c} - sum_{c'<c} t_{c'} l_{k+c,k+c'}) / d_c, with
        // t_{c'} = l_{i,k+c'} d_{c'} (the entries outside the band are zero) ---
        {
          const int amax = min(kb + m - 1, n - 1 - k);   // rows k+kb .. k+amax
          for (int a = kb + tid; a <= amax; a += nt) {
            int sl = k_slot + a;
            if (sl >= R) sl -= R;
            T* wrow = W + sl * mp;
            T t[kKB];
  #pragma unroll
            for (int c = 0; c < kKB; ++c) {
              T v = (c < kb && a - c <= m) ? wrow[a - c] : T(0);
  #pragma unroll
              for (int cp = 0; cp < c; ++cp) v -= t[cp] * Lp[c * kLPS + cp];
              t[c] = v;
              const T l = v * s_dinv[c];
              if (c < kb && a - c <= m) {
                wrow[a - c] = l;
                Lp[a * kLPS + c] = l;
              }
            }
          }
        }
        __syncthreads();
      } else {
        // FP64: pivot by pivot across the CTA (one barrier a pivot), the
        // order of operations the FP64 parity bar was established with
        if (tid == 0) {
          T d = W[k_slot * mp];
          if (!(d > T(0)) || !isfinite(d)) { atomicOr(status, kStatSingular); d = T(1); }
          s_d[0] = d;
          s_dinv[0] = T(1) / d;
          for (int q = kb; q < kKB; ++q) { s_d[q] = T(0); s_dinv[q] = T(0); }
        }
        __syncthreads();
        {  // scale column k: l_{i,k} = a_{i,k} / d_k
          const int rmax = min(m, n - 1 - k);
          const T dinv = s_dinv[0];
          for (int a = 1 + tid; a <= rmax; a += nt) {
            int sl = k_slot + a;
            if (sl >= R) sl -= R;
            T* w = W + sl * mp + a;
            const T l = *w * dinv;
            *w = l;
            Lp[a * kLPS] = l;
          }
        }
        __syncthreads();
        // --- the panel's pivots, eliminating within the panel only.  Warp c
        // updates column k+q+1+c; warp 0 then also forms pivot q+1 and scales
        // its column, so one barrier per pivot suffices. ---
        for (int q = 0; q < kb; ++q) {
          const int kq = k + q;
          const int rmax = min(m, n - 1 - kq);       // rows kq+1 .. kq+rmax hold column kq
          const T dq = s_d[q];
          const int ncol = kb - 1 - q;
          for (int c = warp; c < ncol; c += nwarp) {
            //   a_{i,k+q'} -= l_{i,kq} d_q l_{k+q',kq},  rows k+q' .. kq+rmax
            const int qp = q + 1 + c;
            const T u = Lp[qp * kLPS + q] * dq;
            int base = k_slot + qp;                  // slot of row k+q'
            if (base >= R) base -= R;
            for (int a = lane; a < rmax - c; a += 32) {
              int sl = base + a;
              if (sl >= R) sl -= R;
              T* w = W + sl * mp + a;
              *w -= Lp[(qp + a) * kLPS + q] * u;
            }
            if (c == 0) {
              // column k+q+1 is final: its pivot, then l_{i,k+q+1} for rows
              // k+q+2 .. k+q+1+rmax1
              __syncwarp();
              T d = W[base * mp];
              if (!(d > T(0)) || !isfinite(d)) {
                if (lane == 0) atomicOr(status, kStatSingular);
                d = T(1);
              }
              const T dinv = T(1) / d;
              if (lane == 0) { s_d[q + 1] = d; s_dinv[q + 1] = dinv; }
              const int rmax1 = min(m, n - 1 - (kq + 1));
              for (int a = 1 + lane; a <= rmax1; a += 32) {
                int sl = base + a;
                if (sl >= R) sl -= R;
                T* w = W + sl * mp + a;
                const T l = *w * dinv;
                *w = l;
                Lp[(qp + a) * kLPS + qp] = l;
              }
            }
          }
          // right-hand sides of the panel's later rows
          for (int t = tid; t < (ncol << lnr); t += nt) {
            const int i = kq + 1 + (t >> lnr), r = t & (nr - 1);
            Y[i * nr + r] -= Lp[(i - k) * kLPS + q] * Y[kq * nr + r];
          }
          __syncthreads();
        }
      }
      // --- rank-kb update of the trailing window and of the right-hand sides ---
      const int me = min(m, n - (k + kb));        // trailing rows k+kb .. k+kb+me-1
      if (me > 0) {
        const int nT = (me + 3) >> 2;
        const int ntile = nT * (nT + 1) / 2;
        for (int t = tid; t < ntile; t += nt) {
          int tu = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
          while (tu * (tu + 1) / 2 > t) --tu;
          while ((tu + 1) * (tu + 2) / 2 <= t) ++tu;
          const int tv = t - tu * (tu + 1) / 2;
          T acc[4][4];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
          const int u0 = 4 * tu, v0 = 4 * tv;
#pragma unroll
          for (int q = 0; q < kKB; ++q) {
            const T dq = s_d[q];
            T av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              av[r] = (u0 + r < me) ? Lp[(kb + u0 + r) * kLPS + q] : T(0);
              bv[r] = (v0 + r < me) ? Lp[(kb + v0 + r) * kLPS + q] * dq : T(0);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[r][c] += av[r] * bv[c];
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int u = u0 + r;
            if (u >= me) continue;
            int sl = k_slot + kb + u;              // row k+kb+u, < 2R
            if (sl >= R) sl -= R;
            T* wrow = W + sl * mp;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const int v = v0 + c;
              if (v < me && v <= u) wrow[u - v] -= acc[r][c];
            }
          }
        }
        for (int t = tid; t < (me << lnr); t += nt) {
          const int u = t >> lnr, r = t & (nr - 1);
          const int i = k + kb + u;
          T s = T(0);
#pragma unroll
          for (int q = 0; q < kKB; ++q)
            if (q < kb) s += Lp[(kb + u) * kLPS + q] * Y[(k + q) * nr + r];
          Y[i * nr + r] -= s;
        }
      }
      __syncthreads();
      // --- rows k .. k+kb-1 are final: to the scratch (1/d_i, l_{i,i-1..i-m});
      //     their slots take rows k+R .. k+R+kb-1 ---
      for (int qq = 0; qq < kb; ++qq) {
        const int i = k + qq;
        int sl = k_slot + qq;
        if (sl >= R) sl -= R;
        for (int dd = tid; dd < mp; dd += nt) {
          T* w = W + sl * mp + dd;
          Lg[(long long)i * mp + dd] = (dd == 0) ? s_dinv[qq] : *w;
          const int inew = i + R;
          if (inew < n) *w = Lg[(long long)inew * mp + dd];
        }
      }
      __syncthreads();
    }
    // D^{-1}
    for (int t = tid; t < (n << lnr); t += nt) Y[t] *= Lg[(long long)(t >> lnr) * mp];
    __syncthreads();
    // backward substitution with L^T, kKB rows at a time from the end
    for (int b1 = n - 1; b1 > 0; b1 -= kKB) {
      const int b0 = max(0, b1 - kKB + 1);
      const int nb = b1 - b0 + 1;
      for (int t = tid; t < nb * mp; t += nt) Ls[t] = Lg[(long long)b0 * mp + t];
      __syncthreads();
      if (tid < 32) {                              // inside the block, row by row
        for (int kk = b1; kk > b0; --kk) {
          for (int t = tid; t < ((kk - b0) << lnr); t += 32) {
            const int j = b0 + (t >> lnr), r = t & (nr - 1);
            if (kk - j <= m) Y[j * nr + r] -= Ls[(kk - b0) * mp + (kk - j)] * Y[kk * nr + r];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      const int jlo = max(0, b0 - m);
      for (int t = tid; t < ((b0 - jlo) << lnr); t += nt) {
        const int j = jlo + (t >> lnr), r = t & (nr - 1);
        T s = T(0);
        for (int kk = b0; kk <= b1; ++kk)
          if (kk - j <= m) s += Ls[(kk - b0) * mp + (kk - j)] * Y[kk * nr + r];
        Y[j * nr + r] -= s;
      }
      __syncthreads();
    }
    // write the basis values (slots on lattice bits stay zero), or the
    // correction values (and p += Psi when padd is given)
    for (int l = tid; l < n; l += nt) {
      Local c = local_cell(E, l);
      const long long i = c.c[0] + g.sy * c.c[1] + g.sz * c.c[2];
      if constexpr (kCF) {
        psi[i] = Y[l];
        if (padd) padd[i] += (double)Y[l];
        continue;
      }
      for (int s = 0; s < 8; ++s) P[(long long)s * g.N + i] = T(0);
      for (int r = 0; r < nr; ++r) P[(long long)slot_of(r, E.free_mask) * g.N + i] = Y[l * nr + r];
      if (adaptive) {
        snap[0 * g.N + i] = Abd[i];
        snap[1 * g.N + i] = c.c[0] > 0 ? Abx[i] : 0.0;
        snap[2 * g.N + i] = c.c[0] < g.nx - 1 ? Abx[i + 1] : 0.0;
        snap[3 * g.N + i] = c.c[1] > 0 ? Aby[i] : 0.0;
        snap[4 * g.N + i] = c.c[1] < g.ny - 1 ? Aby[i + g.sy] : 0.0;
        snap[5 * g.N + i] = c.c[2] > 0 ? Abz[i] : 0.0;
        snap[6 * g.N + i] = c.c[2] < g.nz - 1 ? Abz[i + g.sz] : 0.0;
      }
    }
    __syncthreads();
  }
}

__device__ double block_max(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  return v;
}

__device__ __forceinline__ double rel_change(double a, double s) {
  if (s != 0.0) return fabs(a - s) / fabs(s);
  return a != 0.0 ? INFINITY : 0.0;
}

// Sec. 4.1.2 (Reading R15): largest relative change of the A_b rows of the
// entity's cells since its last build.
__global__ void k_adapt_flags(Geo g, const Entity* __restrict__ ents, int count, double theta,
                              const double* __restrict__ Abd, const double* __restrict__ Abx,
                              const double* __restrict__ Aby, const double* __restrict__ Abz,
                              const double* __restrict__ snap, unsigned char* flag) {
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const Entity E = ents[e];
    double mx = 0.0;
    for (int l = threadIdx.x; l < E.n; l += blockDim.x) {
      Local c = local_cell(E, l);
      const long long i = c.c[0] + g.sy * c.c[1] + g.sz * c.c[2];
      const double a[7] = {Abd[i],
                           c.c[0] > 0 ? Abx[i] : 0.0, c.c[0] < g.nx - 1 ? Abx[i + 1] : 0.0,
                           c.c[1] > 0 ? Aby[i] : 0.0, c.c[1] < g.ny - 1 ? Aby[i + g.sy] : 0.0,
                           c.c[2] > 0 ? Abz[i] : 0.0, c.c[2] < g.nz - 1 ? Abz[i + g.sz] : 0.0};
      for (int q = 0; q < 7; ++q) mx = fmax(mx, rel_change(a[q], snap[q * g.N + i]));
    }
    mx = block_max(mx);
    if (threadIdx.x == 0) flag[e] = (mx > theta) ? 1 : 0;
  }
}

// An entity is also rebuilt when a lower-level entity it touches was.
__global__ void k_adapt_propagate(Geo g, const Entity* __restrict__ ents, int first, int count,
                                  const int* __restrict__ ent_of_cell, unsigned char* flag) {
  for (int e = blockIdx.x; e < count; e += gridDim.x) {
    const Entity E = ents[first + e];
    int hit = 0;
    for (int l = threadIdx.x; l < E.n; l += blockDim.x) {
      Local c = local_cell(E, l);
      const long long i = c.c[0] + g.sy * c.c[1] + g.sz * c.c[2];
      for (int d = 0; d < 3; ++d) {
        if (!(E.free_mask & (1 << d))) continue;
        const long long sd = gstride(g, d);
        if (c.c[d] == E.org[d] && c.c[d] > 0) {
          const int o = ent_of_cell[i - sd];
          if (o >= 0 && flag[o]) hit = 1;
        }
        if (c.c[d] == E.org[d] + E.L[d] - 1 && c.c[d] < gextent(g, d) - 1) {
          const int o = ent_of_cell[i + sd];
          if (o >= 0 && flag[o]) hit = 1;
        }
      }
    }
    hit = __syncthreads_or(hit);
    if (threadIdx.x == 0 && hit) flag[first + e] = 1;
  }
}

__global__ void k_count_flags(int count, const unsigned char* __restrict__ flag, double* out) {
  __shared__ int sh[32];
  int c = 0;
  for (int e = threadIdx.x; e < count; e += blockDim.x) c += flag[e];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    out[0] = (double)t;
  }
}

}  // namespace

cudaError_t launch_vertices(const Geo& g, const CGeo& c, Buffers& b, bool single, cudaStream_t s) {
  if (single) k_vertices<float><<<(c.Nc + 127) / 128, 128, 0, s>>>(g, c, b.f32.P);
  else k_vertices<double><<<(c.Nc + 127) / 128, 128, 0, s>>>(g, c, b.P);
  count_launches(1);
  return cudaGetLastError();
}

// Shared memory of one entity's local solve (bytes).
int entity_smem_bytes(const Entity& E, bool single, bool blocked) {
  const int mp = E.m + 1;
  const int elems = blocked ? round4((E.m + kKB) * mp) + round4(E.n * E.nrhs) + (E.m + kKB) * kLPS
                            : mp * mp + E.n * E.nrhs + 2 * mp;
  return elems * (int)(single ? sizeof(float) : sizeof(double));
}

// A window in global memory belongs to the blocked solver only, and each
// CTA's slice must keep every element aligned (the slices are 256 bytes apart).
static bool window_ok(bool blocked, long long gbytes, const Buffers& b) {
  return gbytes == 0 || (blocked && gbytes % 256 == 0 && b.lwork != nullptr);
}

cudaError_t launch_entity_solve(const Geo& g, const Entity* ents, const unsigned char* flag,
                                int count, int smem, int grid, long long lstride, int adaptive,
                                bool single, bool blocked, long long gbytes, Buffers& b,
                                cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!window_ok(blocked, gbytes, b)) return cudaErrorInvalidValue;
  if (grid > count) grid = count;
  if (single) {
    float* ls = reinterpret_cast<float*>(b.lscratch);
    if (blocked)
      k_entity_solve_blk<float, false><<<grid, 256, gbytes ? 0 : smem, s>>>(
          g, ents, count, flag, adaptive, b.Abd, b.Abx, b.Aby, b.Abz, b.f32.P, b.snap, ls, lstride,
          b.status, nullptr, nullptr, nullptr, gbytes ? b.lwork : nullptr, gbytes);
    else
      k_entity_solve<float, false><<<grid, 256, smem, s>>>(
          g, ents, count, flag, adaptive, b.Abd, b.Abx, b.Aby, b.Abz, b.f32.P, b.snap, ls, lstride,
          b.status, nullptr, nullptr, nullptr);
  } else {
    if (blocked)
      k_entity_solve_blk<double, false><<<grid, 256, gbytes ? 0 : smem, s>>>(
          g, ents, count, flag, adaptive, b.Abd, b.Abx, b.Aby, b.Abz, b.P, b.snap, b.lscratch,
          lstride, b.status, nullptr, nullptr, nullptr, gbytes ? b.lwork : nullptr, gbytes);
    else
      k_entity_solve<double, false><<<grid, 256, smem, s>>>(
          g, ents, count, flag, adaptive, b.Abd, b.Abx, b.Aby, b.Abz, b.P, b.snap, b.lscratch,
          lstride, b.status, nullptr, nullptr, nullptr);
  }
  count_launches(1);
  return cudaGetLastError();
}

// Correction functions of one level's entities from the residual b.r: in
// FP64 into b.cf with p += Psi; in mixed precision into the FP32 correction
// b.f32.d (which the caller zeroed: its vertex values are Psi's).
cudaError_t launch_entity_cf(const Geo& g, const Entity* ents, int count, int smem, int grid,
                             long long lstride, bool single, bool blocked, long long gbytes,
                             Buffers& b, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!window_ok(blocked, gbytes, b)) return cudaErrorInvalidValue;
  if (grid > count) grid = count;
  if (single) {
    float* ls = reinterpret_cast<float*>(b.lscratch);
    if (blocked)
      k_entity_solve_blk<float, true><<<grid, 256, gbytes ? 0 : smem, s>>>(
          g, ents, count, nullptr, 0, b.Abd, b.Abx, b.Aby, b.Abz, b.f32.P, nullptr, ls, lstride,
          b.status, b.r, b.f32.d, nullptr, gbytes ? b.lwork : nullptr, gbytes);
    else
      k_entity_solve<float, true><<<grid, 256, smem, s>>>(
          g, ents, count, nullptr, 0, b.Abd, b.Abx, b.Aby, b.Abz, b.f32.P, nullptr, ls, lstride,
          b.status, b.r, b.f32.d, nullptr);
  } else {
    if (blocked)
      k_entity_solve_blk<double, true><<<grid, 256, gbytes ? 0 : smem, s>>>(
          g, ents, count, nullptr, 0, b.Abd, b.Abx, b.Aby, b.Abz, b.P, nullptr, b.lscratch,
          lstride, b.status, b.r, b.cf, b.p, gbytes ? b.lwork : nullptr, gbytes);
    else
      k_entity_solve<double, true><<<grid, 256, smem, s>>>(
          g, ents, count, nullptr, 0, b.Abd, b.Abx, b.Aby, b.Abz, b.P, nullptr, b.lscratch,
          lstride, b.status, b.r, b.cf, b.p);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t set_entity_smem(int smem) {
  cudaError_t e = raise_smem_limit(k_entity_solve<double, false>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve<float, false>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve_blk<double, false>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve_blk<float, false>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve<double, true>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve<float, true>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve_blk<double, true>, smem);
  if (e == cudaSuccess) e = raise_smem_limit(k_entity_solve_blk<float, true>, smem);
  return e;
}

cudaError_t launch_adapt_flags(const Geo& g, const Entity* ents, int count, double theta,
                               Buffers& b, unsigned char* flag, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_adapt_flags<<<count < 4096 ? count : 4096, 256, 0, s>>>(g, ents, count, theta, b.Abd, b.Abx,
                                                           b.Aby, b.Abz, b.snap, flag); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adapt_propagate(const Geo& g, int first, int count, Buffers& b,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_adapt_propagate<<<count < 4096 ? count : 4096, 256, 0, s>>>(g, b.ents, first, count,
                                                               b.ent_of_cell, b.flag); count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(int count, const unsigned char* flag, double* out, cudaStream_t s) {
  k_count_flags<<<1, 1024, 0, s>>>(count, flag, out); count_launches(1);
  return cudaGetLastError();
}

}  // namespace cams
