// Kernels of the learned basis surrogate: a small 3D convolutional network
// trained and evaluated on the GPU by these kernels alone.
//
// Layout: activations [B][C][S][S][S] (x fastest), FP32; weights
// [co][ci][27] with tap t = (dx+1) + 3 (dy+1) + 9 (dz+1) for the offsets
// d in {-1, 0, 1}^3; biases [co].  Every convolution is a 3x3x3
// cross-correlation with zero padding, output size = input size:
//   y[b][co][v] = bias[co] + sum_ci sum_t w[co][ci][t] x[b][ci][v + d(t)].
// Reductions run in a fixed order (no atomics), so results are
// bit-reproducible for a given launch.
#include "cams_internal.h"

namespace cams {

namespace {

constexpr int kCoB = 8;        // output (or input) channels per thread
constexpr int kNetThreads = 256;

__device__ __forceinline__ void tap_offset(int t, int& dx, int& dy, int& dz) {
  dx = t % 3 - 1;
  dy = (t / 3) % 3 - 1;
  dz = t / 9 - 1;
}

// y = conv(x) + bias, optionally ReLU.  Each thread takes kVox voxels
// (kNetThreads apart) and kCoB output channels, so a weight read from shared
// memory feeds kVox FMAs and an input read kCoB.
// grid (ceil(S^3/(256 kVox)), ceil(co/8), B).
constexpr int kVox = 1;   // measured: 4 voxels a thread ran slower (fewer, fuller blocks)

__global__ void __launch_bounds__(kNetThreads) k_conv_fwd(int S, int ci, int co,
                                                          const float* __restrict__ x,
                                                          const float* __restrict__ w,
                                                          const float* __restrict__ bias,
                                                          int relu, float* __restrict__ y) {
  extern __shared__ float ws[];                 // [kCoB][ci][27]
  const int S3 = S * S * S;
  const int co0 = blockIdx.y * kCoB, b = blockIdx.z;
  const int nco = min(kCoB, co - co0);
  for (int e = threadIdx.x; e < kCoB * ci * 27; e += blockDim.x) {
    const int c = e / (ci * 27);
    ws[e] = c < nco ? w[(long long)(co0 + c) * ci * 27 + (e - c * ci * 27)] : 0.0f;
  }
  __syncthreads();
  int vv[kVox], vx[kVox], vy[kVox], vz[kVox];
#pragma unroll
  for (int k = 0; k < kVox; ++k) {
    vv[k] = blockIdx.x * (kNetThreads * kVox) + k * kNetThreads + threadIdx.x;
    const int v = min(vv[k], S3 - 1);
    vx[k] = v % S; vy[k] = (v / S) % S; vz[k] = v / (S * S);
  }
  if (vv[0] >= S3) return;
  float acc[kVox][kCoB];
#pragma unroll
  for (int k = 0; k < kVox; ++k)
#pragma unroll
    for (int c = 0; c < kCoB; ++c) acc[k][c] = c < nco ? bias[co0 + c] : 0.0f;
  const float* xb = x + (long long)b * ci * S3;
  for (int i = 0; i < ci; ++i) {
    const float* xc = xb + (long long)i * S3;
    for (int t = 0; t < 27; ++t) {
      int dx, dy, dz;
      tap_offset(t, dx, dy, dz);
      float xv[kVox];
#pragma unroll
      for (int k = 0; k < kVox; ++k) {
        const int ux = vx[k] + dx, uy = vy[k] + dy, uz = vz[k] + dz;
        xv[k] = (ux < 0 || ux >= S || uy < 0 || uy >= S || uz < 0 || uz >= S) ? 0.0f
                                                                               : xc[ux + S * (uy + S * uz)];
      }
#pragma unroll
      for (int c = 0; c < kCoB; ++c) {
        const float wv = ws[(c * ci + i) * 27 + t];
#pragma unroll
        for (int k = 0; k < kVox; ++k) acc[k][c] += wv * xv[k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kVox; ++k) {
    if (vv[k] >= S3) continue;
    float* yb = y + ((long long)b * co + co0) * S3 + vv[k];
#pragma unroll
    for (int c = 0; c < kCoB; ++c)
      if (c < nco) yb[(long long)c * S3] = relu ? fmaxf(acc[k][c], 0.0f) : acc[k][c];
  }
}

// gx[b][i][v] = sum_co sum_t w[co][i][t] gy[b][co][v - d(t)], times the ReLU
// mask (xact > 0) of the layer input when xact is given.
// grid (ceil(S^3/256), ceil(ci/8), B).
__global__ void __launch_bounds__(kNetThreads) k_conv_bwd_data(int S, int ci, int co,
                                                               const float* __restrict__ gy,
                                                               const float* __restrict__ w,
                                                               const float* __restrict__ xact,
                                                               float* __restrict__ gx) {
  extern __shared__ float ws[];                 // [kCoB][co][27]: w[c][i0 + k][t] at (k*co + c)*27 + t
  const int S3 = S * S * S;
  const int ci0 = blockIdx.y * kCoB, b = blockIdx.z;
  const int nci = min(kCoB, ci - ci0);
  for (int e = threadIdx.x; e < kCoB * co * 27; e += blockDim.x) {
    const int k = e / (co * 27), rem = e - k * co * 27, c = rem / 27, t = rem - c * 27;
    ws[e] = k < nci ? w[((long long)c * ci + ci0 + k) * 27 + t] : 0.0f;
  }
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= S3) return;
  const int vx = v % S, vy = (v / S) % S, vz = v / (S * S);
  float acc[kCoB];
#pragma unroll
  for (int k = 0; k < kCoB; ++k) acc[k] = 0.0f;
  const float* gb = gy + (long long)b * co * S3;
  for (int c = 0; c < co; ++c) {
    const float* gc = gb + (long long)c * S3;
    for (int t = 0; t < 27; ++t) {
      int dx, dy, dz;
      tap_offset(t, dx, dy, dz);
      const int ux = vx - dx, uy = vy - dy, uz = vz - dz;
      if (ux < 0 || ux >= S || uy < 0 || uy >= S || uz < 0 || uz >= S) continue;
      const float g = gc[ux + S * (uy + S * uz)];
#pragma unroll
      for (int k = 0; k < kCoB; ++k) acc[k] += ws[(k * co + c) * 27 + t] * g;
    }
  }
  const long long o = ((long long)b * ci + ci0) * S3 + v;
#pragma unroll
  for (int k = 0; k < kCoB; ++k) {
    if (k >= nci) continue;
    float val = acc[k];
    if (xact && !(xact[o + (long long)k * S3] > 0.0f)) val = 0.0f;
    gx[o + (long long)k * S3] = val;
  }
}

// gw[o][i][t] = sum_b sum_v gy[b][o][v] x[b][i][v + d(t)]; gbias[o] = sum gy[b][o][v].
// One CTA per (o, i): grid (ci, co).
__global__ void __launch_bounds__(kNetThreads) k_conv_bwd_w(int B, int S, int ci, int co,
                                                            const float* __restrict__ x,
                                                            const float* __restrict__ gy,
                                                            float* __restrict__ gw,
                                                            float* __restrict__ gbias) {
  __shared__ float red[28][kNetThreads / 32];
  const int i = blockIdx.x, o = blockIdx.y;
  const int S3 = S * S * S;
  float acc[28];
#pragma unroll
  for (int t = 0; t < 28; ++t) acc[t] = 0.0f;
  for (int b = 0; b < B; ++b) {
    const float* xc = x + ((long long)b * ci + i) * S3;
    const float* gc = gy + ((long long)b * co + o) * S3;
    for (int v = threadIdx.x; v < S3; v += blockDim.x) {
      const float g = gc[v];
      if (g == 0.0f) continue;
      const int vx = v % S, vy = (v / S) % S, vz = v / (S * S);
      acc[27] += g;
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
        const int ux = vx + dx, uy = vy + dy, uz = vz + dz;
        if (ux < 0 || ux >= S || uy < 0 || uy >= S || uz < 0 || uz >= S) continue;
        acc[t] += g * xc[ux + S * (uy + S * uz)];
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 28; ++t) {
    float s = acc[t];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) red[t][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < 28) {
    float s = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
    if (threadIdx.x < 27) gw[((long long)o * ci + i) * 27 + threadIdx.x] = s;
    else if (i == 0) gbias[o] = s;
  }
}

// Masked mean-squared error: loss = sum_mask (p - t)^2 / count,
// grad = 2 (p - t) mask / count.  Per-block partial sums, then one block.
__global__ void k_mse_partial(long long n, const float* __restrict__ p, const float* __restrict__ t,
                              const float* __restrict__ mask, float inv_count, float* grad,
                              double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float mk = mask[e];
    const float d = (p[e] - t[e]) * mk;
    grad[e] = 2.0f * d * inv_count;
    s += (double)d * (double)d;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tsum += red[k];
    part[blockIdx.x] = tsum;
  }
}

__global__ void k_mse_final(int nb, const double* __restrict__ part, double inv_count, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < nb; ++k) s += part[k];
  out[0] = s * inv_count;
}

// Energy norm of the interior error (the norm the coarse space pays in):
// e = mask (p - t), relative face couplings w = exp(x[b][d][u]) for the face
// between u and its lower neighbour along d (x: the network input, whose
// channels 0-2 are the log couplings), E = sum_faces w (e_u - e_v)^2 / count,
// grad = mask dE/dp.  One thread per (patch, channel, cell), grid-stride.
__device__ __forceinline__ float e_at(const float* p, const float* t, const float* mk, long long o) {
  return (p[o] - t[o]) * mk[o];
}

__global__ void k_energy_partial(int B, int S, int C, int cx, const float* __restrict__ p,
                                 const float* __restrict__ t, const float* __restrict__ mk,
                                 const float* __restrict__ x, float inv_count, float* grad,
                                 double* part) {
  __shared__ double red[32];
  const int S3 = S * S * S;
  const long long n = (long long)B * C * S3;
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(e % S3);
    const long long bc = e / S3;
    const int b = (int)(bc / C);
    const int l[3] = {v % S, (v / S) % S, v / (S * S)};
    const int st[3] = {1, S, S * S};
    const float ev = e_at(p, t, mk, e);
    float gsum = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float* xd = x + ((long long)b * cx + d) * S3;
      if (l[d] > 0) {                          // face to the lower neighbour
        const float w = expf(xd[v]);
        const float diff = ev - e_at(p, t, mk, e - st[d]);
        acc += (double)(w * diff * diff);
        gsum += w * diff;
      }
      if (l[d] < S - 1) {                      // face to the upper neighbour
        const float w = expf(xd[v + st[d]]);
        gsum += w * (ev - e_at(p, t, mk, e + st[d]));
      }
    }
    grad[e] = 2.0f * gsum * mk[e] * inv_count;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tsum += red[k];
    part[blockIdx.x] = tsum;
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void k_adam(long long n, float* p, const float* __restrict__ g, float* m, float* v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float ge = g[e];
  const float me = b1 * m[e] + (1.0f - b1) * ge;
  const float ve = b2 * v[e] + (1.0f - b2) * ge * ge;
  m[e] = me;
  v[e] = ve;
  p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
}

constexpr int kMseBlocks = 512;

}  // namespace

cudaError_t launch_conv_fwd(int B, int S, int ci, int co, const float* x, const float* w,
                            const float* bias, int relu, float* y, cudaStream_t s) {
  const int S3 = S * S * S;
  const int smem = kCoB * ci * 27 * (int)sizeof(float);
  cudaError_t e = raise_smem_limit(k_conv_fwd, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((S3 + kNetThreads * kVox - 1) / (kNetThreads * kVox), (co + kCoB - 1) / kCoB, B);
  k_conv_fwd<<<grid, kNetThreads, smem, s>>>(S, ci, co, x, w, bias, relu, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_conv_bwd(int B, int S, int ci, int co, const float* x, const float* w,
                            const float* gy, const float* xact, float* gx, float* gw,
                            float* gbias, cudaStream_t s) {
  const int S3 = S * S * S;
  if (gx) {
    const int smem = kCoB * co * 27 * (int)sizeof(float);
    cudaError_t e = raise_smem_limit(k_conv_bwd_data, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((S3 + kNetThreads - 1) / kNetThreads, (ci + kCoB - 1) / kCoB, B);
    k_conv_bwd_data<<<grid, kNetThreads, smem, s>>>(S, ci, co, gy, w, xact, gx);
    count_launches(1);
  }
  k_conv_bwd_w<<<dim3(ci, co), kNetThreads, 0, s>>>(B, S, ci, co, x, gy, gw, gbias);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mse(long long n, const float* p, const float* t, const float* mask,
                       double count, float* grad, double* part, double* loss, cudaStream_t s) {
  k_mse_partial<<<kMseBlocks, 256, 0, s>>>(n, p, t, mask, (float)(1.0 / count), grad, part);
  k_mse_final<<<1, 32, 0, s>>>(kMseBlocks, part, 1.0 / count, loss);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_energy(int B, int S, int C, int cx, const float* p, const float* t,
                          const float* mask, const float* x, double count, float* grad, double* part,
                          double* loss, cudaStream_t s) {
  k_energy_partial<<<kMseBlocks, 256, 0, s>>>(B, S, C, cx, p, t, mask, x, (float)(1.0 / count), grad,
                                              part);
  k_mse_final<<<1, 32, 0, s>>>(kMseBlocks, part, 1.0 / count, loss);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(int)((n + 255) / 256), 256, 0, s>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  count_launches(1);
  return cudaGetLastError();
}

int mse_partial_blocks() { return kMseBlocks; }

// ---------------------------------------------------------------------
// The surrogate's patches.  A full interior dual block is the box of
// (b+1)^3 cells from one vertex plane to the next in every direction
// (S = b+1); its 8 basis functions are those of its corner nodes, corner
// bits (cx, cy, cz).  At local coordinate l (0..b) along d the value of the
// function with corner bit c_d sits in the cell's P slot with bit d = c_d
// between the planes; on the plane l = 0 only c_d = 0 has support (slot bit
// 0), on l = b only c_d = 1 (slot bit 0).  The baseline is the multilinear
// interpolant of the corner values, the exact discrete basis function of a
// homogeneous medium; the network predicts the deviation from it.
namespace {

template <class TP>
__device__ __forceinline__ float patch_value(const Geo& g, const TP* P, long long i, const int* l, int b,
                                             int corner) {
  int slot = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int cd = (corner >> d) & 1;
    if (l[d] == 0) { if (cd) return 0.0f; }
    else if (l[d] == b) { if (!cd) return 0.0f; }
    else if (cd) slot |= 1 << d;
  }
  return (float)P[(long long)slot * g.N + i];
}

__device__ __forceinline__ float baseline(const int* l, int b, int corner) {
  float v = 1.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float t = (float)l[d] / (float)b;
    v *= ((corner >> d) & 1) ? t : 1.0f - t;
  }
  return v;
}

// One CTA per patch: x [12][S^3] (log couplings minus their patch mean, the
// relative accumulation term, the boundary deviations of the 8 functions),
// optionally target/mask [8][S^3] (deviation everywhere, mask 1 inside).
template <class TP>
__global__ void __launch_bounds__(256) k_patch_inputs(Geo g, int b, const int* __restrict__ org,
                                                      const TP* __restrict__ P,
                                                      const double* __restrict__ Abd,
                                                      const double* __restrict__ Abx,
                                                      const double* __restrict__ Aby,
                                                      const double* __restrict__ Abz, float* x,
                                                      float* target, float* mask) {
  __shared__ float red[32];
  __shared__ float s_mean;
  const int S = b + 1, S3 = S * S * S;
  const int pidx = blockIdx.x;
  const int ox = org[3 * pidx], oy = org[3 * pidx + 1], oz = org[3 * pidx + 2];
  float* xp = x + (long long)pidx * kNetIn * S3;
  // mean of the log couplings over the patch
  float s = 0.0f;
  for (int v = threadIdx.x; v < S3; v += blockDim.x) {
    const int l[3] = {v % S, (v / S) % S, v / (S * S)};
    const long long i = (ox + l[0]) + g.sy * (oy + l[1]) + g.sz * (oz + l[2]);
    s += logf(fmaxf((float)-Abx[i], 1e-30f)) + logf(fmaxf((float)-Aby[i], 1e-30f)) +
         logf(fmaxf((float)-Abz[i], 1e-30f));
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    s_mean = t / (3.0f * (float)S3);
  }
  __syncthreads();
  const float mean = s_mean;
  for (int v = threadIdx.x; v < S3; v += blockDim.x) {
    const int l[3] = {v % S, (v / S) % S, v / (S * S)};
    const long long i = (ox + l[0]) + g.sy * (oy + l[1]) + g.sz * (oz + l[2]);
    const float wx = (float)-Abx[i], wy = (float)-Aby[i], wz = (float)-Abz[i];
    xp[0 * S3 + v] = logf(fmaxf(wx, 1e-30f)) - mean;
    xp[1 * S3 + v] = logf(fmaxf(wy, 1e-30f)) - mean;
    xp[2 * S3 + v] = logf(fmaxf(wz, 1e-30f)) - mean;
    const double wsum = -(Abx[i] + Aby[i] + Abz[i] + Abx[i + 1] + Aby[i + g.sy] + Abz[i + g.sz]);
    xp[3 * S3 + v] = wsum > 0.0 ? (float)((Abd[i] - wsum) / wsum) : 0.0f;
    const bool inside = l[0] > 0 && l[0] < b && l[1] > 0 && l[1] < b && l[2] > 0 && l[2] < b;
    for (int c = 0; c < 8; ++c) {
      const float dev = patch_value(g, P, i, l, b, c) - baseline(l, b, c);
      xp[(4 + c) * S3 + v] = inside ? 0.0f : dev;
      if (target) {
        target[((long long)pidx * 8 + c) * S3 + v] = dev;
        mask[((long long)pidx * 8 + c) * S3 + v] = inside ? 1.0f : 0.0f;
      }
    }
  }
}

// P at the patches' interior cells = baseline + the network's deviation.
template <class TP>
__global__ void __launch_bounds__(256) k_patch_apply(Geo g, int b, const int* __restrict__ org,
                                                     const float* __restrict__ y, TP* P) {
  const int S = b + 1, S3 = S * S * S;
  const int pidx = blockIdx.x;
  const int ox = org[3 * pidx], oy = org[3 * pidx + 1], oz = org[3 * pidx + 2];
  for (int v = threadIdx.x; v < S3; v += blockDim.x) {
    const int l[3] = {v % S, (v / S) % S, v / (S * S)};
    if (!(l[0] > 0 && l[0] < b && l[1] > 0 && l[1] < b && l[2] > 0 && l[2] < b)) continue;
    const long long i = (ox + l[0]) + g.sy * (oy + l[1]) + g.sz * (oz + l[2]);
    for (int c = 0; c < 8; ++c)
      P[(long long)c * g.N + i] = (TP)(baseline(l, b, c) + y[((long long)pidx * 8 + c) * S3 + v]);
  }
}

// Residual gate: for each function, ||D^{-1} A_b P|| over the interior
// cells against ||D^{-1} (the part of A_b P from the boundary values)||,
// D = diag(A_b) (the Jacobi scaling keeps high-permeability cells from
// dominating both norms); the patch's flag (1 = solve exactly) is set when
// the largest ratio over its 8 functions exceeds tol.
template <class TP>
__global__ void __launch_bounds__(256) k_patch_gate(Geo g, int b, const int* __restrict__ org,
                                                    const int* __restrict__ ent, const TP* __restrict__ P,
                                                    const double* __restrict__ Abd,
                                                    const double* __restrict__ Abx,
                                                    const double* __restrict__ Aby,
                                                    const double* __restrict__ Abz, double tol,
                                                    unsigned char* flag, float* ratio_out) {
  __shared__ float red[2][8][8];
  const int S = b + 1, S3 = S * S * S;
  const int pidx = blockIdx.x;
  const int ox = org[3 * pidx], oy = org[3 * pidx + 1], oz = org[3 * pidx + 2];
  float rr[8], bb[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) { rr[c] = 0.0f; bb[c] = 0.0f; }
  for (int v = threadIdx.x; v < S3; v += blockDim.x) {
    const int l[3] = {v % S, (v / S) % S, v / (S * S)};
    if (!(l[0] > 0 && l[0] < b && l[1] > 0 && l[1] < b && l[2] > 0 && l[2] < b)) continue;
    const long long i = (ox + l[0]) + g.sy * (oy + l[1]) + g.sz * (oz + l[2]);
    const double cpl[6] = {Abx[i], Abx[i + 1], Aby[i], Aby[i + g.sy], Abz[i], Abz[i + g.sz]};
    const long long nbi[6] = {i - 1, i + 1, i - g.sy, i + g.sy, i - g.sz, i + g.sz};
    const double dinv = 1.0 / Abd[i];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      double r = Abd[i] * (double)patch_value(g, P, i, l, b, c), f = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        int ln[3] = {l[0], l[1], l[2]};
        ln[k >> 1] += (k & 1) ? 1 : -1;
        const double t = cpl[k] * (double)patch_value(g, P, nbi[k], ln, b, c);
        r += t;
        const bool nb_inside = ln[0] > 0 && ln[0] < b && ln[1] > 0 && ln[1] < b && ln[2] > 0 && ln[2] < b;
        if (!nb_inside) f += t;
      }
      r *= dinv;
      f *= dinv;
      rr[c] += (float)(r * r);
      bb[c] += (float)(f * f);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float a = rr[c], q = bb[c];
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      q += __shfl_down_sync(0xffffffffu, q, off);
    }
    if (lane == 0) { red[0][c][wid] = a; red[1][c][wid] = q; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float worst = 0.0f;
    for (int c = 0; c < 8; ++c) {
      float a = 0.0f, q = 0.0f;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += red[0][c][k]; q += red[1][c][k]; }
      const float ratio = q > 0.0f ? sqrtf(a / q) : (a > 0.0f ? INFINITY : 0.0f);
      worst = fmaxf(worst, ratio);
    }
    if (ratio_out) ratio_out[pidx] = worst;
    flag[ent[pidx]] = (worst > (float)tol || !isfinite(worst)) ? 1 : 0;
  }
}

}  // namespace

cudaError_t launch_patch_inputs(const Geo& g, int b, int n, const int* org, bool single,
                                const Buffers& bf, float* x, float* target, float* mask,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (single)
    k_patch_inputs<float><<<n, 256, 0, s>>>(g, b, org, bf.f32.P, bf.Abd, bf.Abx, bf.Aby, bf.Abz, x,
                                            target, mask);
  else
    k_patch_inputs<double><<<n, 256, 0, s>>>(g, b, org, bf.P, bf.Abd, bf.Abx, bf.Aby, bf.Abz, x,
                                             target, mask);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_patch_apply(const Geo& g, int b, int n, const int* org, const float* y,
                               bool single, Buffers& bf, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (single) k_patch_apply<float><<<n, 256, 0, s>>>(g, b, org, y, bf.f32.P);
  else k_patch_apply<double><<<n, 256, 0, s>>>(g, b, org, y, bf.P);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_patch_gate(const Geo& g, int b, int n, const int* org, const int* ent,
                              double tol, bool single, Buffers& bf, unsigned char* flag,
                              float* ratio, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (single)
    k_patch_gate<float><<<n, 256, 0, s>>>(g, b, org, ent, bf.f32.P, bf.Abd, bf.Abx, bf.Aby, bf.Abz,
                                          tol, flag, ratio);
  else
    k_patch_gate<double><<<n, 256, 0, s>>>(g, b, org, ent, bf.P, bf.Abd, bf.Abx, bf.Aby, bf.Abz, tol,
                                           flag, ratio);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cams
