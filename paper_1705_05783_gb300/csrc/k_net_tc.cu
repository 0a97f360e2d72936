// The learned surrogate's 3x3x3 convolutions on the tensor cores: tcgen05
// MMAs with BF16 operands and FP32 accumulation in tensor memory.
//
// Implicit GEMM over a zero-padded patch.  A patch of S^3 voxels with C
// channels is stored "chunked and padded": the (S+2)^3 grid with a zero
// border, voxels in flat order r = px + S'(py + S' pz) (S' = S + 2), channels
// in chunks of 8 (16 bytes): element (r, c) at ((c / 8) * RP + r) * 8 + c % 8,
// RP rows per chunk plane (the padded grid plus spare zero rows).  For an
// output row r the 27 input rows of its stencil are r + off(t),
// off = dx + S' dy + S'^2 dz, so the A operand of one tap for 128 consecutive
// output rows is 128 consecutive input rows: a shared-memory descriptor
// starting off(t) rows further, no im2col copy.  Rows of one 8-channel chunk
// are 16 bytes apart, so any run of 8 rows is one 128-byte core matrix of the
// no-swizzle K-major layout (SBO = 128 bytes between row groups, LBO = RP x 16
// bytes between the two chunks of a K = 16 step).  The weights of a tap, N x
// C in the same layout, are the B operand; D = A B^T (128 x N, FP32) sits in
// 128 lanes x N columns of tensor memory.
//
// Output rows are computed in tiles of 128 from the first interior voxel
// (r = h, h = S'^2 + S' + 1) to the last; border rows inside those tiles
// are written as zeros, so a layer's output is the next layer's zero-padded
// input.  One CTA of 128 threads (one per tensor-memory lane) runs one patch
// at a time: the patch's input and all weights in shared memory, one thread
// issues the 27 x C/16 MMAs of a tile and commits them to an mbarrier, and
// the four warps read the accumulator back (bias, ReLU, BF16 or FP32 out).
#include <cuda_bf16.h>

#include "cams_internal.h"
#include "tc_ptx.h"

namespace cams {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTile = 128;
constexpr long long kTcWait = 1LL << 24;   // polls of the MMA barrier before giving up

struct TcGeom {
  int S, Sp, h, nt, RP;
};

inline TcGeom tc_geom(int S) {
  TcGeom G;
  G.S = S;
  G.Sp = S + 2;
  G.h = G.Sp * G.Sp + G.Sp + 1;
  const int span = G.Sp * G.Sp * G.Sp - 2 * G.h;
  G.nt = (span + kTile - 1) / kTile;
  G.RP = (2 * G.h + G.nt * kTile + 7) / 8 * 8;
  return G;
}

__device__ __forceinline__ bool interior(const TcGeom& G, int r, int& vox) {
  const int n3 = G.Sp * G.Sp * G.Sp;
  if (r >= n3) return false;
  const int px = r % G.Sp, py = (r / G.Sp) % G.Sp, pz = r / (G.Sp * G.Sp);
  if (px < 1 || px > G.S || py < 1 || py > G.S || pz < 1 || pz > G.S) return false;
  vox = (px - 1) + G.S * ((py - 1) + G.S * (pz - 1));
  return true;
}

// FP32 activations [B][C][S^3] -> BF16 chunked-padded [B][KC][RP][8] (KC
// chunks of 8 channels, channels >= C zero).  Only rows of the output-tile
// range are written; the rest stay zero from the buffer's initialisation.
__global__ void k_tc_pack(int B, TcGeom G, int C, int KC, const float* __restrict__ x,
                          __nv_bfloat16* __restrict__ out) {
  const long long rows = (long long)G.nt * kTile;
  const long long n = (long long)B * KC * rows;
  const int S3 = G.S * G.S * G.S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = G.h + (int)(e % rows);
    const long long bk = e / rows;
    const int kc = (int)(bk % KC);
    const long long b = bk / KC;
    int vox;
    const bool in = interior(G, r, vox);
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = kc * 8 + k;
      v[k] = __float2bfloat16_rn(in && c < C ? x[(b * C + c) * S3 + vox] : 0.0f);
    }
    *reinterpret_cast<uint4*>(out + ((b * KC + kc) * G.RP + r) * 8) = *reinterpret_cast<uint4*>(v);
  }
}

// One layer: y = conv(x; w) + bias (ReLU when relu).  x: BF16 chunked-padded
// with KCin chunks (KCin even).  w: FP32 [co][ci][27] (ci <= 8 KCin real
// input channels), bias [co].  N: the MMA's N (co rounded up to 16).
// kOutBf16: y is BF16 chunked-padded with co / 8 chunks (the next layer's
// input); else y is FP32 [B][co][S^3].
template <int N, bool kOutBf16>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(int B, TcGeom G, int KCin, int ci,
                                                             int co, const __nv_bfloat16* __restrict__ x,
                                                             const float* __restrict__ w,
                                                             const float* __restrict__ bias, int relu,
                                                             void* __restrict__ yv,
                                                             int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // [input: KCin x RP x 16 B][weights: 27 x KCin x N x 16 B][mbarrier][tmem slot]
  unsigned char* xs = smem;
  const int xbytes = KCin * G.RP * 16;
  unsigned char* ws = smem + xbytes;
  const int wbytes = 27 * KCin * N * 16;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + xbytes + wbytes);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + xbytes + wbytes + 16);
  const int t = threadIdx.x, warp = t >> 5;
  const int S3 = G.S * G.S * G.S;
  // weights into the B layout: tap t, chunk kc, row n at ((t KCin + kc) N + n) 16 B
  for (int e = t; e < 27 * KCin * N * 8; e += kTcThreads) {
    const int k = e % 8, n = (e / 8) % N, kc = (e / (8 * N)) % KCin, tap = e / (8 * N * KCin);
    const int c = kc * 8 + k;
    const float v = (n < co && c < ci) ? w[((long long)n * ci + c) * 27 + tap] : 0.0f;
    reinterpret_cast<__nv_bfloat16*>(ws)[e] = __float2bfloat16_rn(v);
  }
  if (t == 0) tc::mbar_init(bar, 1);
  if (warp == 0) tc::tmem_alloc(slot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTile, N);
  const uint32_t xs_a = tc::smem_u32(xs), ws_a = tc::smem_u32(ws);
  uint32_t phase = 0;
  bool ok = true;
  for (int b = blockIdx.x; b < B && ok; b += gridDim.x) {
    // the patch's input rows into shared memory (16-byte copies)
    const uint4* src = reinterpret_cast<const uint4*>(x + (long long)b * KCin * G.RP * 8);
    uint4* dst = reinterpret_cast<uint4*>(xs);
    for (int e = t; e < KCin * G.RP; e += kTcThreads) dst[e] = src[e];
    tc::fence_proxy_async();
    __syncthreads();
    for (int m = 0; m < G.nt; ++m) {
      const int row0 = G.h + m * kTile;
      if (t == 0) {
        tc::fence_after_sync();
        bool acc = false;
        for (int tap = 0; tap < 27; ++tap) {
          const int off = (tap % 3 - 1) + G.Sp * ((tap / 3) % 3 - 1) + G.Sp * G.Sp * (tap / 9 - 1);
          for (int ks = 0; ks < KCin / 2; ++ks) {
            const uint64_t a = tc::smem_desc(xs_a + ((2 * ks) * G.RP + row0 + off) * 16,
                                             G.RP * 16, 128);
            const uint64_t bd = tc::smem_desc(ws_a + ((tap * KCin + 2 * ks) * N) * 16, N * 16, 128);
            tc::mma_bf16(tmem, a, bd, kIdesc, acc);
            acc = true;
          }
        }
        tc::mma_commit(bar);
      }
      if (!tc::mbar_wait(bar, phase, kTcWait)) {
        atomicOr(status, kStatTimeout);
        ok = false;
        tc::mbar_wait(bar, phase, kTcWait);   // one more bounded wait before TMEM is freed
      }
      phase ^= 1u;
      tc::fence_after_sync();
      // epilogue: thread t holds output row row0 + t (tensor-memory lane t)
      const int r = row0 + t;
      int vox = 0;
      const bool in = interior(G, r, vox);
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int n0 = 0; n0 < N; n0 += 16) {
        float v[16];
        tc::tmem_ld16(tl + n0, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int n = n0 + k;
          float y = n < co ? v[k] + bias[n] : 0.0f;
          if (relu) y = fmaxf(y, 0.0f);
          v[k] = in ? y : 0.0f;
        }
        if constexpr (kOutBf16) {
          __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(yv);
          const int KCo = (co + 7) / 8;
#pragma unroll
          for (int h8 = 0; h8 < 2; ++h8) {
            const int kc = n0 / 8 + h8;
            if (kc >= KCo) continue;
            __align__(16) __nv_bfloat16 o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = __float2bfloat16_rn(v[h8 * 8 + k]);
            *reinterpret_cast<uint4*>(y + (((long long)b * KCo + kc) * G.RP + r) * 8) =
                *reinterpret_cast<uint4*>(o);
          }
        } else {
          float* y = reinterpret_cast<float*>(yv);
          if (in)
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (n0 + k < co) y[((long long)b * co + n0 + k) * S3 + vox] = v[k];
        }
      }
      tc::fence_before_sync();
      __syncthreads();   // the accumulator is read out before the next tile's MMAs
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

int tc_smem_bytes(const TcGeom& G, int KCin, int N) { return KCin * G.RP * 16 + 27 * KCin * N * 16 + 64; }

template <int N, bool kOutBf16>
cudaError_t launch_conv_tc_n(int B, const TcGeom& G, int KCin, int ci, int co,
                             const __nv_bfloat16* x, const float* w, const float* bias, int relu,
                             void* y, int* status, int sms, cudaStream_t s) {
  const int smem = tc_smem_bytes(G, KCin, N);
  cudaError_t e = raise_smem_limit(k_conv_tc<N, kOutBf16>, smem);
  if (e != cudaSuccess) return e;
  const int grid = B < sms ? B : sms;
  k_conv_tc<N, kOutBf16><<<grid, kTcThreads, smem, s>>>(B, G, KCin, ci, co, x, w, bias, relu, y,
                                                        status);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

long long net_tc_act_elems(int B, int S, int C) {
  const TcGeom G = tc_geom(S);
  const int KC = (C + 15) / 16 * 2;
  return (long long)B * KC * G.RP * 8;
}

bool net_tc_fits(int S, int max_smem) {
  const TcGeom G = tc_geom(S);
  return tc_smem_bytes(G, 4, 32) <= max_smem;
}

cudaError_t launch_tc_pack(int B, int S, int C, const float* x, void* out, cudaStream_t s) {
  const TcGeom G = tc_geom(S);
  const int KC = (C + 15) / 16 * 2;
  const long long n = (long long)B * KC * G.nt * kTile;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_tc_pack<<<blocks, 256, 0, s>>>(B, G, C, KC, x, static_cast<__nv_bfloat16*>(out));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_conv_tc(int B, int S, int ci, int co, const void* xv, const float* w,
                           const float* bias, int relu, bool out_bf16, void* y, int* status,
                           int sms, cudaStream_t s) {
  const TcGeom G = tc_geom(S);
  const __nv_bfloat16* x = static_cast<const __nv_bfloat16*>(xv);
  const int KCin = (ci + 15) / 16 * 2;
  if (co <= 16) {
    return out_bf16 ? launch_conv_tc_n<16, true>(B, G, KCin, ci, co, x, w, bias, relu, y, status, sms, s)
                    : launch_conv_tc_n<16, false>(B, G, KCin, ci, co, x, w, bias, relu, y, status, sms, s);
  }
  if (co <= 32) {
    return out_bf16 ? launch_conv_tc_n<32, true>(B, G, KCin, ci, co, x, w, bias, relu, y, status, sms, s)
                    : launch_conv_tc_n<32, false>(B, G, KCin, ci, co, x, w, bias, relu, y, status, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace cams
