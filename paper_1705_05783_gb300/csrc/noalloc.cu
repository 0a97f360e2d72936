// Residual and 2-norm of a 7-point system with no device allocation.
//
// Some callers cannot call cudaMalloc: frameworks that hand all device memory
// to their own pool or arena (a cudaMalloc behind the pool's back can fail or
// fragment it), and time-critical loops that must not pay the device-wide
// synchronisation that cudaMalloc/cudaFree imply.  This entry point serves
// them: the caller passes the system and the output buffers, and the
// reduction's scratch (one partial sum per block of cells plus the total)
// lives in a file-scope static device array instead of a handle allocation.
//
// The array exists once per device that loads the library and stays there
// until the process exits.  In host code its name is only a host-side stand-in,
// so its device address is looked up with cudaGetSymbolAddress, with the
// device current: on the first call on a device, and again whenever the
// device's current context differs from the one the address was taken in (the
// module is loaded anew after cudaDeviceReset, and the array may move).
// Every call shares the array: calls that overlap on the GPU (different
// streams, or several host threads) race on it and must be serialised by the
// caller.  Each call overwrites every slot it reads, so nothing left by an
// earlier call leaks into a result.
#include <cmath>
#include <mutex>
#include <string>

#include "cams_internal.h"

namespace {

constexpr int kCellsPerBlock = 8192;    // cells summed by one CTA
constexpr int kMaxBlocks = 32768;       // partial sums the scratch holds (256 KiB)
constexpr long long kMaxCells = (long long)kCellsPerBlock * kMaxBlocks;   // 268,435,456
constexpr int kMaxDevices = 64;

// cuCtxGetCurrent of the driver API, reached through the runtime (no link
// against libcuda); its CUcontext is held as an opaque pointer.
using CtxGetCurrentFn = int (*)(void**);

// partial sums [0, kMaxBlocks) and the total at [kMaxBlocks]
static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks + 1];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};      // context the address was taken in
CtxGetCurrentFn g_ctx_get = nullptr;
bool g_ctx_get_tried = false;

// The calling thread's current context, or null when it cannot be told.
void* current_context() {
  if (!g_ctx_get_tried) {
    g_ctx_get_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
    else
      cudaGetLastError();
  }
  void* ctx = nullptr;
  if (!g_ctx_get || g_ctx_get(&ctx) != 0) return nullptr;
  return ctx;
}

__device__ double block_sum_na(double v) {
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

// Block b owns cells [b*kCellsPerBlock, (b+1)*kCellsPerBlock); same per-cell
// arithmetic as the engine's residual kernel.
__global__ void k_residual_noalloc(cams::Geo g, const double* __restrict__ Ad,
                                   const double* __restrict__ Ax, const double* __restrict__ Ay,
                                   const double* __restrict__ Az, const double* __restrict__ f,
                                   const double* __restrict__ p, double* r, double* scratch) {
  const long long lo = (long long)blockIdx.x * kCellsPerBlock;
  const long long hi = lo + kCellsPerBlock < g.N ? lo + kCellsPerBlock : g.N;
  double s2 = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
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
    if (r) r[i] = a;
    s2 += a * a;
  }
  s2 = block_sum_na(s2);
  if (threadIdx.x == 0) scratch[blockIdx.x] = s2;
}

// total of the partial sums, in block order (deterministic)
__global__ void k_finish_noalloc(int nblocks, double* scratch) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += scratch[b];
  s = block_sum_na(s);
  if (threadIdx.x == 0) scratch[kMaxBlocks] = s;
}

int fail_na(int code, const std::string& msg) {
  cams::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int cams_residual_norm_noalloc(int nx, int ny, int nz, const double* diag,
                                          const double* ax, const double* ay, const double* az,
                                          const double* f, const double* p, double* r,
                                          double* norm_out, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1) return fail_na(CAMS_EINVAL, "grid sizes must be >= 1");
  const long long N = (long long)nx * ny * nz;
  if (N > kMaxCells)
    return fail_na(CAMS_EINVAL, "cams_residual_norm_noalloc: the grid has " + std::to_string(N) +
                                    " cells; at most " + std::to_string(kMaxCells) +
                                    " are supported (the static scratch holds " +
                                    std::to_string(kMaxBlocks) + " partial sums of " +
                                    std::to_string(kCellsPerBlock) + " cells)");
  if (!diag || !ax || !ay || !az || !f || !p) return fail_na(CAMS_EINVAL, "null input pointer");
  if (!r && !norm_out) return fail_na(CAMS_EINVAL, "no output requested");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(CAMS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(CAMS_EINVAL, "device ordinal out of range");
  double* scratch = nullptr;
  {
    // set-up, once per device and context, with that device current
    std::lock_guard<std::mutex> lock(g_mutex);
    void* ctx = current_context();
    if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&scratch), g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail_na(CAMS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = scratch;
      g_scratch_ctx[dev] = current_context();   // the lookup made the primary context current
    }
    scratch = g_scratch_addr[dev];
  }
  cams::Geo g{};
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.N = N;
  g.sy = nx; g.sz = (long long)nx * ny;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblocks = (int)((N + kCellsPerBlock - 1) / kCellsPerBlock);
  k_residual_noalloc<<<nblocks, 256, 0, s>>>(g, diag, ax, ay, az, f, p, r, scratch);
  k_finish_noalloc<<<1, 1024, 0, s>>>(nblocks, scratch);
  cams::count_launches(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_na(CAMS_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (norm_out) {
    double s2 = 0.0;
    e = cudaMemcpyAsync(&s2, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_na(CAMS_ECUDA, std::string("read-back: ") + cudaGetErrorString(e));
    *norm_out = std::sqrt(s2);
  } else {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_na(CAMS_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
  }
  return CAMS_OK;
}
