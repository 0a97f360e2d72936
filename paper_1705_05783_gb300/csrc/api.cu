// C-ABI and host-side control of the C-AMS engine: setup (static
// transmissibilities and wirebasket tables), linear-system population, the
// adaptive operator update, the C-AMS iteration of Table 1 and the Newton
// loop of Sec. 4.1.1.  Every numerical step is a kernel of this library; the
// host only sequences launches and reads back one scalar per stopping test.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cams_internal.h"

using namespace cams;

struct cams_handle {
  int dev = 0;
  cudaStream_t stream = nullptr;
  cams_grid grid{};
  cams_fluid fluid{};
  cams_options opt{};
  Geo g{};
  CGeo c{};
  FluidK fl{};
  Buffers b{};
  // wirebasket
  std::vector<Entity> ents;
  int lev_first[4] = {0, 0, 0, 0}, lev_count[4] = {0, 0, 0, 0}, lev_smem[4] = {0, 0, 0, 0};
  int lev_grid[4] = {0, 0, 0, 0};
  bool lev_blocked[4] = {false, false, false, false};
  long long lev_lstride[4] = {0, 0, 0, 0};
  long long lev_gbytes[4] = {0, 0, 0, 0};   // > 0: the level's windows in b.lwork, bytes per CTA
  long long lwork_len = 0;
  long long lscratch_len = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int d_active = 0;
  int n_dual = 0;
  // coarse band
  int mc = 0;
  std::vector<int> perm;        // band position of each natural coarse index
  bool coarse_ldlt = false;     // b.Lc holds the L D L^T of the current R A P
  // state
  bool built = false;
  bool assembled = false;
  bool have_src = false;
  bool have_fix = false;        // prescribed cells in the current boundary conditions
  int fix_cap = 0;              // capacity of b.fixc / b.fixv
  double dt = 0.0;
  int dirichlet = 0;
  double pw = 0.0, pe = 0.0, rhow = 1.0, rhoe = 1.0;
  int last_rebuilt = 0;
  long long launch_base = 0;
  bool single = false;          // mixed precision: FP32 preconditioner (b.f32)
  bool ilu_pipelined = true;    // false: level-scheduled sweeps (CAMS_ILU_LEVEL=1)
  bool ilu_cta = false;         // 2 x 2 tile blocks per CTA, else one tile per warp
  bool coarse_cluster = false;  // MSFE coarse solve across a cluster (CAMS_COARSE_CLUSTER=0: one CTA)
  bool coarse_inv = false;      // mixed MSFE: FP32 factor and inverse factor (CAMS_COARSE_INV=0: off)
  int ilu_grid = 1;
  // learned surrogate of the interior basis stage (cams_set_surrogate)
  double surr_tol = 0.0;           // > 0: enabled
  int surr_b = 0, surr_n = 0, surr_chunk = 0, surr_accepted = 0;
  float* net = nullptr;            // device parameters (kNetParams)
  int* surr_org = nullptr;         // device: lower corner of each full interior's patch
  int* surr_ent = nullptr;         // device: its entity index
  float *surr_x = nullptr, *surr_h1 = nullptr, *surr_h2 = nullptr, *surr_y = nullptr;
  void *surr_ta = nullptr, *surr_tb = nullptr;   // BF16 activations of the tensor-core path
  bool surr_tc = false;                           // the network runs on the tensor cores
  int sms = 0;                                    // SM count of the handle's device
  float* surr_ratio = nullptr;     // device: gate ratio of each full interior (last build)
  // the C-AMS iteration as a CUDA graph (captured once, replayed per iteration)
  bool graphs = true;               // CAMS_GRAPHS=0 launches every kernel directly
  cudaGraphExec_t step_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t aux_stream = nullptr;   // the ILU(0) factorisation beside the coarse one
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  long long step_launches = 0;
  // the whole inner loop of a linearisation as one graph: a conditional WHILE
  // node around one iteration, the residual norm and the stopping test
  bool loop_graph = true;           // CAMS_LOOP_GRAPH=0 keeps the host-driven loop
  cudaGraphExec_t loop_exec = nullptr;
  long long loop_body_launches = 0;
  // per-kernel-class profiling (cams_profile)
  bool prof = false;
  struct Pending { int cls; cudaEvent_t a, b; long long k0, k1; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_acc[3 * CAMS_PROF_CLASSES] = {};
  std::string err;
};

namespace {

std::string g_setup_error = "no error";

int fail(cams_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_setup_error = msg;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(h, CAMS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
int dalloc(cams_handle* h, T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(h, CAMS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return CAMS_OK;
}

cudaMemcpyKind kind_in(const cams_handle* h) {
  return h->opt.memspace == CAMS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}
cudaMemcpyKind kind_out(const cams_handle* h) {
  return h->opt.memspace == CAMS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

double rho_host(const FluidK& f, double p) {
  return f.law == 0 ? f.rho0 * std::exp(f.c * p) : f.rho0 * (1.0 + f.c * p);
}

void prof_flush(cams_handle* h);

// device status word -> status code (and reset)
int check_status(cams_handle* h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->b.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->prof) prof_flush(h);
  if (st) CK(cudaMemsetAsync(h->b.status, 0, sizeof(int), h->stream));
  if (st & kStatTimeout) return fail(h, CAMS_ETIMEOUT, "a device-side wait exceeded its limit");
  if (st & kStatSingular) return fail(h, CAMS_ESINGULAR, "zero or non-finite pivot in a local or coarse factorisation");
  if (st & kStatNan) return fail(h, CAMS_ENAN, "non-finite value");
  return CAMS_OK;
}

int read_scalar(cams_handle* h, double* out) {
  CK(cudaMemcpyAsync(out, h->b.scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->prof) prof_flush(h);
  return CAMS_OK;
}

// ------------------------------------------------------------- profiling --

namespace lc {
std::atomic<long long> total{0};
thread_local long long mine = 0;     // launches issued by this thread
}

cudaEvent_t pool_get(cams_handle* h) {
  if (h->pool.empty()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = h->pool.back();
  h->pool.pop_back();
  return e;
}

// Accumulate the timed launches whose events have completed (call after a
// stream synchronisation) and recycle their events.
void prof_flush(cams_handle* h) {
  for (auto& q : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      h->prof_acc[3 * q.cls + 0] += 1.0;
      h->prof_acc[3 * q.cls + 1] += ms;
      h->prof_acc[3 * q.cls + 2] += (double)(q.k1 - q.k0);
    }
    h->pool.push_back(q.a);
    h->pool.push_back(q.b);
  }
  h->pending.clear();
}

struct ProfScope {
  cams_handle* h;
  int cls;
  cudaEvent_t a = nullptr;
  long long k0 = 0;
  ProfScope(cams_handle* hh, int c) : h(hh), cls(c) {
    if (!h->prof) return;
    a = pool_get(h);
    k0 = cams::launches_total();
    if (a) cudaEventRecord(a, h->stream);
  }
  ~ProfScope() {
    if (!h->prof || !a) return;
    cudaEvent_t b = pool_get(h);
    if (!b) { h->pool.push_back(a); return; }
    cudaEventRecord(b, h->stream);
    h->pending.push_back({cls, a, b, k0, cams::launches_total()});
    if (h->pending.size() > 4096) {   // bound the number of live events
      cudaEventSynchronize(b);
      prof_flush(h);
    }
  }
};

// One kernel class: events bracket the launcher when profiling is on.
#define LAUNCH(cls, call)          \
  do {                             \
    ProfScope ps_(h, cls);         \
    CK(call);                      \
  } while (0)

// ---------------------------------------------------------------- tables --

void build_entities(cams_handle* h, std::vector<int>& ent_of_cell) {
  const Geo& g = h->g;
  const CGeo& c = h->c;
  const int n[3] = {g.nx, g.ny, g.nz};
  bool active[3];
  h->d_active = 0;
  for (int d = 0; d < 3; ++d) {
    active[d] = n[d] > 1;
    h->d_active += active[d];
  }
  // per direction: list of (org, L, is_free)
  struct Choice { int org, L, free_; };
  std::vector<Choice> ch[3];
  for (int d = 0; d < 3; ++d) {
    if (!active[d]) { ch[d].push_back({0, 1, 0}); continue; }
    for (int I = 0; I < c.nc[d]; ++I) ch[d].push_back({I * c.b[d] + c.o[d], 1, 0});
    for (int j = 0; j <= c.nc[d]; ++j) {
      const int lo = j == 0 ? 0 : (j - 1) * c.b[d] + c.o[d] + 1;
      const int hi = j == c.nc[d] ? n[d] - 1 : j * c.b[d] + c.o[d] - 1;
      if (lo <= hi) ch[d].push_back({lo, hi - lo + 1, 1});
    }
  }
  h->ents.clear();
  for (int lev = 1; lev <= 3; ++lev) {
    h->lev_first[lev] = (int)h->ents.size();
    for (const Choice& cz : ch[2])
      for (const Choice& cy : ch[1])
        for (const Choice& cx : ch[0]) {
          if (cx.free_ + cy.free_ + cz.free_ != lev) continue;
          Entity E{};
          E.org[0] = cx.org; E.org[1] = cy.org; E.org[2] = cz.org;
          E.L[0] = cx.L; E.L[1] = cy.L; E.L[2] = cz.L;
          E.level = lev;
          E.free_mask = cx.free_ | (cy.free_ << 1) | (cz.free_ << 2);
          int ord[3] = {0, 1, 2};
          std::stable_sort(ord, ord + 3, [&](int a, int b2) { return E.L[a] < E.L[b2]; });
          for (int k = 0; k < 3; ++k) E.ord[k] = ord[k];
          E.n = E.L[0] * E.L[1] * E.L[2];
          const int st[3] = {1, E.L[ord[0]], E.L[ord[0]] * E.L[ord[1]]};
          E.m = 0;
          for (int k = 0; k < 3; ++k)
            if (E.L[ord[k]] > 1) E.m = std::max(E.m, st[k]);
          E.nrhs = 1 << (cx.free_ + cy.free_ + cz.free_);
          const int id = (int)h->ents.size();
          for (int z = 0; z < E.L[2]; ++z)
            for (int y = 0; y < E.L[1]; ++y)
              for (int x = 0; x < E.L[0]; ++x)
                ent_of_cell[(E.org[0] + x) + g.sy * (E.org[1] + y) + g.sz * (E.org[2] + z)] = id;
          h->ents.push_back(E);
        }
    h->lev_count[lev] = (int)h->ents.size() - h->lev_first[lev];
  }
}

int alloc_all(cams_handle* h) {
  const long long N = h->g.N;
  Buffers& b = h->b;
  int rc;
#define AL(ptr, n) if ((rc = dalloc(h, &(ptr), (size_t)(n))) != CAMS_OK) return rc
  AL(b.Tx, N); AL(b.Ty, N); AL(b.Tz, N);
  AL(b.Tbw, (long long)h->g.ny * h->g.nz); AL(b.Tbe, (long long)h->g.ny * h->g.nz);
  AL(b.p, N); AL(b.pn, N); AL(b.rho, N); AL(b.rhon, N);
  AL(b.Ad, N); AL(b.Ax, N); AL(b.Ay, N); AL(b.Az, N); AL(b.Cacc, N);
  if (h->opt.jacobian) {
    // A is not symmetric: its transposed couplings and the pivot products
    AL(b.Axu, N); AL(b.Ayu, N); AL(b.Azu, N);
    if (!h->single) { AL(b.Qx, N); AL(b.Qy, N); AL(b.Qz, N); }
  } else {
    b.Axu = b.Ax; b.Ayu = b.Ay; b.Azu = b.Az;
  }
  AL(b.f, N); AL(b.eps, N);
  AL(b.Abd, N); AL(b.Abx, N); AL(b.Aby, N); AL(b.Abz, N);
  if (h->opt.basis != 4) AL(b.snap, 7 * N);
  if (!h->single) AL(b.P, 8 * N);
  if (h->single) {
    SingleBuffers& f = b.f32;
    const long long S = ilu_skew_len(h->g);
    AL(f.Ad, N); AL(f.Ax, N); AL(f.Ay, N); AL(f.Az, N); AL(f.dinv, N); AL(f.d, N); AL(f.r, N);
    if (h->opt.jacobian) {
      AL(f.Axu, N); AL(f.Ayu, N); AL(f.Azu, N); AL(f.Qx, N); AL(f.Qy, N); AL(f.Qz, N);
    } else {
      f.Axu = f.Ax; f.Ayu = f.Ay; f.Azu = f.Az;
    }
    AL(f.P, 8 * N); AL(f.pc, h->c.Nc);
    AL(f.Lc, (size_t)h->c.Nc * (h->mc + 1)); AL(f.Lr, (size_t)h->c.Nc * (h->mc + 1));
    AL(f.cblk, coarse_blocks_len(h->c.Nc)); AL(f.cdinv, h->c.Nc);
    if (h->coarse_inv) {
      AL(f.Z, (size_t)h->c.Nc * (size_t)coarse_ldz(h->c.Nc));
      AL(f.tc, coarse_ldz(h->c.Nc));
      AL(f.zpart, coarse_part_len(h->c.Nc));
    }
    AL(f.Lx, S); AL(f.Ly, S); AL(f.Lz, S); AL(f.Ux, S); AL(f.Uy, S); AL(f.Uz, S);
    AL(f.rds, S); AL(f.w, S); AL(f.z, S);
    // slots that hold no cell must read as zero (the sweeps run branch-free over them)
    for (float* v : {f.Lx, f.Ly, f.Lz, f.Ux, f.Uy, f.Uz, f.rds, f.w, f.z})
      if (cudaMemset(v, 0, sizeof(float) * (size_t)S) != cudaSuccess)
        return fail(h, CAMS_ECUDA, "cudaMemset failed");
  }
  AL(b.ent_of_cell, N);
  AL(b.ents, h->ents.size());
  AL(b.flag, h->ents.size());
  AL(b.lscratch, (size_t)h->lscratch_len);
  if (h->lwork_len > 0) AL(b.lwork, (size_t)h->lwork_len);
  AL(b.loc, (size_t)h->n_dual * 36);
  AL(b.Acs, 27LL * h->c.Nc);
  AL(b.band, (size_t)h->c.Nc * (2 * h->mc + 1));
  AL(b.Fc, (size_t)h->c.Nc * (2 * h->mc + 1));
  AL(b.Lc, (size_t)h->c.Nc * (h->mc + 1)); AL(b.Lr, (size_t)h->c.Nc * (h->mc + 1));
  AL(b.cblk, coarse_blocks_len(h->c.Nc)); AL(b.cdinv, h->c.Nc); AL(b.cabort, 1);
  AL(b.perm, h->c.Nc);
  AL(b.jxt, 2LL * h->g.nx);
  AL(b.rc, h->c.Nc); AL(b.pc, h->c.Nc); AL(b.ywork, h->c.Nc);
  AL(b.dinv, N);
  {
    const long long S = ilu_skew_len(h->g);   // >= N
    AL(b.Lx, S); AL(b.Ly, S); AL(b.Lz, S); AL(b.Ux, S); AL(b.Uy, S); AL(b.Uz, S);
    AL(b.rds, S); AL(b.w, S); AL(b.z, S);
    // slots that hold no cell must read as zero (the sweeps run branch-free over them)
    for (double* v : {b.Lx, b.Ly, b.Lz, b.Ux, b.Uy, b.Uz, b.rds, b.w, b.z})
      if (cudaMemset(v, 0, sizeof(double) * (size_t)S) != cudaSuccess)
        return fail(h, CAMS_ECUDA, "cudaMemset failed");
  }
  AL(b.ctrl, ilu_ctrl_ints(h->g));
  AL(b.r, N);
  if (h->opt.cf && !h->single) {
    AL(b.cf, N);
    // vertex cells are in no entity: their correction value stays zero
    if (cudaMemset(b.cf, 0, sizeof(double) * (size_t)N) != cudaSuccess)
      return fail(h, CAMS_ECUDA, "cudaMemset failed");
  }
  AL(b.red, kRedBlocks);
  AL(b.scal, 8);
  AL(b.status, 1);
#undef AL
  return CAMS_OK;
}

void free_all(cams_handle* h) {
  Buffers& b = h->b;
  void* ptrs[] = {b.Tx, b.Ty, b.Tz, b.Tbw, b.Tbe, b.p, b.pn, b.rho, b.rhon, b.Ad, b.Ax, b.Ay,
                  b.Az, b.Cacc, b.f, b.eps, b.src, b.Abd, b.Abx, b.Aby, b.Abz, b.snap, b.P,
                  b.ent_of_cell, b.ents, b.flag, b.lscratch, b.loc, b.Acs, b.band, b.perm, b.jxt, b.rc,
                  b.pc, b.dinv, b.r, b.rds, b.w, b.z, b.red, b.scal, b.status, b.Lx, b.Ly, b.Lz,
                  b.Ux, b.Uy, b.Uz, b.ctrl, b.Lc, b.Lr, b.cblk, b.cdinv, b.cabort, b.fixm,
                  b.fixc, b.fixv, b.cf, b.Qx, b.Qy, b.Qz, b.Fc, b.ywork, b.lwork,
                  // the transposed couplings are separate arrays only for a nonsymmetric A
                  b.Axu != b.Ax ? b.Axu : nullptr, b.Ayu != b.Ay ? b.Ayu : nullptr,
                  b.Azu != b.Az ? b.Azu : nullptr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  const SingleBuffers& f = b.f32;
  void* fptrs[] = {f.Ad, f.Ax, f.Ay, f.Az, f.dinv, f.Lx, f.Ly, f.Lz, f.Ux, f.Uy, f.Uz,
                   f.rds, f.w, f.z, f.d, f.r, f.P, f.pc, f.Qx, f.Qy, f.Qz, f.Lc, f.Lr, f.cblk, f.cdinv,
                   f.Z, f.tc, f.zpart, f.Axu != f.Ax ? f.Axu : nullptr, f.Ayu != f.Ay ? f.Ayu : nullptr,
                   f.Azu != f.Az ? f.Azu : nullptr};
  for (void* p : fptrs)
    if (p) cudaFree(p);
  h->b = Buffers{};
}

int validate(const cams_grid* gr, const cams_fluid* fl, const cams_options* o) {
  if (!gr || !fl || !o) return fail(nullptr, CAMS_EINVAL, "null argument");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 1) return fail(nullptr, CAMS_EINVAL, "grid sizes must be >= 1");
  if (!(gr->dx > 0 && gr->dy > 0 && gr->dz > 0)) return fail(nullptr, CAMS_EINVAL, "cell sizes must be > 0");
  if (!(fl->phi > 0 && fl->mu > 0 && fl->rho0 > 0)) return fail(nullptr, CAMS_EINVAL, "phi, mu, rho0 must be > 0");
  if (fl->law != CAMS_RHO_EXP && fl->law != CAMS_RHO_LINEAR) return fail(nullptr, CAMS_EINVAL, "unknown density law");
  const int n[3] = {gr->nx, gr->ny, gr->nz};
  for (int d = 0; d < 3; ++d) {
    const int b = o->coarse[d];
    if (n[d] == 1) {
      if (b != 1) return fail(nullptr, CAMS_EINVAL, "an inactive direction needs coarse size 1");
    } else if (b < 2 || n[d] % b != 0) {
      return fail(nullptr, CAMS_EINVAL, "coarse size must be >= 2 and divide the grid size");
    }
  }
  if (o->basis < 1 || o->basis > 4) return fail(nullptr, CAMS_EINVAL, "basis must be 1..4");
  if (o->restriction < 0 || o->restriction > 2) return fail(nullptr, CAMS_EINVAL, "restriction must be 0, 1 or 2");
  if (o->n_pre < 0 || o->n_post < 0) return fail(nullptr, CAMS_EINVAL, "smoothing counts must be >= 0");
  if (o->max_newton < 1 || o->max_newton > kMaxNewton) return fail(nullptr, CAMS_EINVAL, "max_newton must be 1..64");
  if (o->max_cams < 1) return fail(nullptr, CAMS_EINVAL, "max_cams must be >= 1");
  if (o->memspace != CAMS_HOST && o->memspace != CAMS_DEVICE) return fail(nullptr, CAMS_EINVAL, "bad memspace");
  if (o->precision != CAMS_PREC_FP64 && o->precision != CAMS_PREC_MIXED)
    return fail(nullptr, CAMS_EINVAL, "precision must be CAMS_PREC_FP64 or CAMS_PREC_MIXED");
  if (o->cf != 0 && o->cf != 1) return fail(nullptr, CAMS_EINVAL, "cf must be 0 or 1");
  if (o->jacobian != 0 && o->jacobian != 1) return fail(nullptr, CAMS_EINVAL, "jacobian must be 0 or 1");
  if ((long long)gr->nx * gr->ny * gr->nz > (1LL << 31) - 1) return fail(nullptr, CAMS_EINVAL, "grid too large");
  return CAMS_OK;
}

// ------------------------------------------------------------ surrogate --

void free_surrogate(cams_handle* h) {
  void* ptrs[] = {h->net, h->surr_org, h->surr_ent, h->surr_x, h->surr_h1, h->surr_h2, h->surr_y,
                  h->surr_ta, h->surr_tb,
                  h->surr_ratio};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  h->net = nullptr; h->surr_org = h->surr_ent = nullptr;
  h->surr_x = h->surr_h1 = h->surr_h2 = h->surr_y = h->surr_ratio = nullptr;
  h->surr_ta = h->surr_tb = nullptr;
  h->surr_tc = false;
  h->surr_tol = 0.0; h->surr_n = 0; h->surr_chunk = 0;
}

// The full dual-block interiors ((b-1)^3 cells) with their patch corners.
int surrogate_tables(cams_handle* h) {
  const int b = h->c.b[0];
  std::vector<int> org, ent;
  for (int e = h->lev_first[3]; e < h->lev_first[3] + h->lev_count[3]; ++e) {
    const Entity& E = h->ents[e];
    if (E.L[0] != b - 1 || E.L[1] != b - 1 || E.L[2] != b - 1) continue;
    for (int d = 0; d < 3; ++d) org.push_back(E.org[d] - 1);
    ent.push_back(e);
  }
  h->surr_b = b;
  h->surr_n = (int)ent.size();
  if (h->surr_n == 0) return CAMS_OK;
  int rc = dalloc(h, &h->surr_org, org.size());
  if (!rc) rc = dalloc(h, &h->surr_ent, ent.size());
  if (rc) return rc;
  CK(cudaMemcpy(h->surr_org, org.data(), sizeof(int) * org.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->surr_ent, ent.data(), sizeof(int) * ent.size(), cudaMemcpyHostToDevice));
  return CAMS_OK;
}

// y = network(x) for n patches (x: n x kNetIn x S^3, y: n x kNetOut x S^3).
cudaError_t net_forward(cams_handle* h, int n, const float* x, float* y) {
  const int S = h->surr_b + 1;
  const float* p = h->net;
  const float *w1 = p, *b1 = w1 + kNetHid * kNetIn * 27;
  const float *w2 = b1 + kNetHid, *b2 = w2 + kNetHid * kNetHid * 27;
  const float *w3 = b2 + kNetHid, *b3 = w3 + kNetHid * kNetHid * 27;
  const float *w4 = b3 + kNetHid, *b4 = w4 + kNetOut * kNetHid * 27;
  if (h->surr_tc) {
    // tensor cores: BF16 activations, FP32 accumulation; the last layer writes FP32
    cudaError_t e = launch_tc_pack(n, S, kNetIn, x, h->surr_ta, h->stream);
    if (e == cudaSuccess) e = launch_conv_tc(n, S, kNetIn, kNetHid, h->surr_ta, w1, b1, 1, true, h->surr_tb, h->b.status, h->sms, h->stream);
    if (e == cudaSuccess) e = launch_conv_tc(n, S, kNetHid, kNetHid, h->surr_tb, w2, b2, 1, true, h->surr_ta, h->b.status, h->sms, h->stream);
    if (e == cudaSuccess) e = launch_conv_tc(n, S, kNetHid, kNetHid, h->surr_ta, w3, b3, 1, true, h->surr_tb, h->b.status, h->sms, h->stream);
    if (e == cudaSuccess) e = launch_conv_tc(n, S, kNetHid, kNetOut, h->surr_tb, w4, b4, 0, false, y, h->b.status, h->sms, h->stream);
    return e;
  }
  cudaError_t e = launch_conv_fwd(n, S, kNetIn, kNetHid, x, w1, b1, 1, h->surr_h1, h->stream);
  if (e == cudaSuccess) e = launch_conv_fwd(n, S, kNetHid, kNetHid, h->surr_h1, w2, b2, 1, h->surr_h2, h->stream);
  if (e == cudaSuccess) e = launch_conv_fwd(n, S, kNetHid, kNetHid, h->surr_h2, w3, b3, 1, h->surr_h1, h->stream);
  if (e == cudaSuccess) e = launch_conv_fwd(n, S, kNetHid, kNetOut, h->surr_h1, w4, b4, 0, y, h->stream);
  return e;
}

// Interior stage by the surrogate: predict every full interior, keep the
// predictions that pass the residual gate (flag 0), leave flag 1 for the
// exact solve.  Called with every level-3 flag set to 1.
int surrogate_interiors(cams_handle* h) {
  Buffers& b = h->b;
  const int S = h->surr_b + 1;
  for (int p0 = 0; p0 < h->surr_n; p0 += h->surr_chunk) {
    const int n = std::min(h->surr_chunk, h->surr_n - p0);
    CK(launch_patch_inputs(h->g, h->surr_b, n, h->surr_org + 3 * p0, h->single, b, h->surr_x,
                           nullptr, nullptr, h->stream));
    CK(net_forward(h, n, h->surr_x, h->surr_y));
    CK(launch_patch_apply(h->g, h->surr_b, n, h->surr_org + 3 * p0, h->surr_y, h->single, b,
                          h->stream));
  }
  (void)S;
  CK(launch_patch_gate(h->g, h->surr_b, h->surr_n, h->surr_org, h->surr_ent, h->surr_tol,
                       h->single, b, b.flag, h->surr_ratio, h->stream));
  CK(launch_count_flags(h->lev_count[3], b.flag + h->lev_first[3], b.scal, h->stream));
  double cnt = 0.0;
  int rc = read_scalar(h, &cnt);
  if (rc) return rc;
  h->surr_accepted = h->lev_count[3] - (int)cnt;
  return CAMS_OK;
}

// ----------------------------------------------------------- operations --

// True when fine cell i is a coarse node (a vertex of the wirebasket).
bool is_coarse_node(const cams_handle* h, long long i) {
  const int n[3] = {h->g.nx, h->g.ny, h->g.nz};
  const int xc[3] = {(int)(i % n[0]), (int)((i / n[0]) % n[1]), (int)(i / ((long long)n[0] * n[1]))};
  for (int d = 0; d < 3; ++d) {
    const int sft = xc[d] - h->c.o[d];
    if (sft < 0 || sft % h->c.b[d] != 0) return false;
  }
  return true;
}

// Prescribed cell-centre pressures: validated on the host, copied into the
// handle's list, then marked in b.fixm and written into the iterate b.p
// (which must already hold this call's pressure).
int set_fixed(cams_handle* h, const cams_bc* bc) {
  const int n = bc ? bc->n_fix : 0;
  if (n < 0) return fail(h, CAMS_EINVAL, "n_fix < 0");
  h->have_fix = false;
  if (n == 0) return CAMS_OK;
  if (!bc->fix_cell || !bc->fix_value) return fail(h, CAMS_EINVAL, "null fixed-cell arrays");
  std::vector<int> cells(n);
  CK(cudaMemcpyAsync(cells.data(), bc->fix_cell, sizeof(int) * n,
                     h->opt.memspace == CAMS_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < n; ++k) {
    if (cells[k] < 0 || cells[k] >= h->g.N) return fail(h, CAMS_EINVAL, "fixed cell out of range");
    if (is_coarse_node(h, cells[k])) return fail(h, CAMS_EINVAL, "a fixed cell is a coarse node");
  }
  Buffers& b = h->b;
  if (!b.fixm) {
    int rc = dalloc(h, &b.fixm, (size_t)h->g.N);
    if (rc) return rc;
  }
  if (n > h->fix_cap) {
    if (b.fixc) cudaFree(b.fixc);
    if (b.fixv) cudaFree(b.fixv);
    b.fixc = nullptr;
    b.fixv = nullptr;
    h->fix_cap = 0;
    int rc = dalloc(h, &b.fixc, n);
    if (rc) return rc;
    rc = dalloc(h, &b.fixv, n);
    if (rc) return rc;
    h->fix_cap = n;
  }
  CK(cudaMemcpyAsync(b.fixc, cells.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(b.fixv, bc->fix_value, sizeof(double) * n, kind_in(h), h->stream));
  CK(cudaMemsetAsync(b.fixm, 0, (size_t)h->g.N, h->stream));
  CK(launch_fix_cells(n, b.fixc, b.fixv, b.fixm, b.p, h->g.N, h->stream));
  // the host copy of the cell list must outlive the copy above
  CK(cudaStreamSynchronize(h->stream));
  h->have_fix = true;
  return CAMS_OK;
}

int set_sources(cams_handle* h, const cams_bc* bc) {
  int rcf = set_fixed(h, bc);
  if (rcf) return rcf;
  h->dirichlet = bc ? bc->dirichlet : 0;
  h->pw = bc ? bc->p_west : 0.0;
  h->pe = bc ? bc->p_east : 0.0;
  h->rhow = rho_host(h->fl, h->pw);
  h->rhoe = rho_host(h->fl, h->pe);
  const int n = bc ? bc->n_src : 0;
  if (n < 0) return fail(h, CAMS_EINVAL, "n_src < 0");
  if (n == 0) { h->have_src = false; return CAMS_OK; }
  if (!bc->src_cell || !bc->src_rate) return fail(h, CAMS_EINVAL, "null source arrays");
  if (!h->b.src) {
    int rc = dalloc(h, &h->b.src, (size_t)h->g.N);
    if (rc) return rc;
  }
  CK(cudaMemsetAsync(h->b.src, 0, sizeof(double) * h->g.N, h->stream));
  int* dcell = nullptr;
  double* drate = nullptr;
  if (h->opt.memspace == CAMS_HOST) {
    for (int k = 0; k < n; ++k)
      if (bc->src_cell[k] < 0 || bc->src_cell[k] >= h->g.N) return fail(h, CAMS_EINVAL, "source cell out of range");
    int rc = dalloc(h, &dcell, n);
    if (rc) return rc;
    rc = dalloc(h, &drate, n);
    if (rc) { cudaFree(dcell); return rc; }
    cudaMemcpyAsync(dcell, bc->src_cell, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(drate, bc->src_rate, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
  }
  cudaError_t e = launch_add_sources(n, dcell ? dcell : bc->src_cell, drate ? drate : bc->src_rate,
                                     h->b.src, h->g.N, h->stream);
  if (dcell) {
    cudaStreamSynchronize(h->stream);
    cudaFree(dcell);
    cudaFree(drate);
  }
  CK(e);
  h->have_src = true;
  return CAMS_OK;
}

int assemble(cams_handle* h, double* eps_norm) {
  Buffers& b = h->b;
  double* src_saved = b.src;
  if (!h->have_src) b.src = nullptr;
  {
    ProfScope ps_(h, CAMS_PROF_ASSEMBLE);
    cudaError_t e = launch_density(h->g, h->fl, b.p, b.rho, h->stream);
    if (e == cudaSuccess) e = launch_assemble(h->g, h->fl, h->dt, h->dirichlet, h->pw, h->pe,
                                                   h->have_fix ? b.fixm : nullptr,
                                                   h->opt.jacobian != 0, b, h->stream);
    b.src = src_saved;
    CK(e);
  }
  double s2;
  int rc = read_scalar(h, &s2);
  if (rc) return rc;
  if (!std::isfinite(s2)) return fail(h, CAMS_ENAN, "non-finite nonlinear error norm");
  if (eps_norm) *eps_norm = std::sqrt(s2);
  h->assembled = true;
  return CAMS_OK;
}

int update_operators(cams_handle* h, int force, int* n_rebuilt) {
  if (!h->assembled) return fail(h, CAMS_EINVAL, "cams_assemble must come first");
  Buffers& b = h->b;
  const cams_options& o = h->opt;
  const int ne = (int)h->ents.size();
  const bool nonsym = o.jacobian != 0;
  // The ILU(0) factorisation needs only A: it runs on a second stream while
  // the basis, R A P and the coarse factorisation (latency-bound chains that
  // leave most SMs idle) run on the handle's stream, and the handle's stream
  // waits for it at the end.  With per-class profiling on, everything stays
  // on one stream so that each class is timed alone.
  const bool overlap = !h->prof;
  if (overlap) {
    if (!h->aux_stream) {
      CK(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(h->ev_fork, h->stream));
    CK(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
    CK(launch_ilu_factor(h->g, b, h->ilu_pipelined, h->ilu_grid, h->ilu_cta, h->single, nonsym,
                         h->aux_stream));
    CK(cudaEventRecord(h->ev_join, h->aux_stream));
  }
  LAUNCH(CAMS_PROF_BASIS_OP, launch_basis_operator(h->g, h->fl, o.basis, h->dt,
                                                     h->have_fix ? b.fixm : nullptr, b, h->stream));
  const bool adaptive = o.basis != 4;
  int rebuilt = 0;
  if (!h->built || force || o.adapt_theta < 0) {
    CK(cudaMemsetAsync(b.flag, 1, ne, h->stream));
    rebuilt = ne;
  } else if (o.basis == 4) {
    // (B4) depends on the transmissibilities only: its operator cannot
    // change, so the relative-change test of Sec. 4.1.2 flags nothing.
    rebuilt = 0;
  } else {
    {
      ProfScope ps_(h, CAMS_PROF_ADAPT);
      CK(launch_adapt_flags(h->g, b.ents, ne, o.adapt_theta, b, b.flag, h->stream));
      for (int lev = 2; lev <= 3; ++lev)
        CK(launch_adapt_propagate(h->g, h->lev_first[lev], h->lev_count[lev], b, h->stream));
      CK(launch_count_flags(ne, b.flag, b.scal, h->stream));
    }
    double cnt;
    int rc = read_scalar(h, &cnt);
    if (rc) return rc;
    rebuilt = (int)cnt;
  }
  if (rebuilt > 0) {
    ProfScope ps_(h, CAMS_PROF_BASIS);
    if (!h->built) CK(launch_vertices(h->g, h->c, b, h->single, h->stream));
    h->surr_accepted = 0;
    for (int lev = 1; lev <= 3; ++lev) {
      const int f = h->lev_first[lev];
      if (lev == 3 && h->surr_tol > 0.0 && h->surr_n > 0 && rebuilt == ne) {
        const int rc = surrogate_interiors(h);
        if (rc) return rc;
      }
      CK(launch_entity_solve(h->g, b.ents + f, b.flag + f, h->lev_count[lev], h->lev_smem[lev],
                             h->lev_grid[lev], h->lev_lstride[lev], adaptive ? 1 : 0, h->single,
                             h->lev_blocked[lev], h->lev_gbytes[lev], b, h->stream));
    }
  }
  h->built = true;
  h->last_rebuilt = rebuilt;
  if (n_rebuilt) *n_rebuilt = rebuilt;
  // Galerkin coarse operator and its factorisation
  // restriction 2 iterates with MSFE (its MSFV correction closes the step)
  if (o.restriction != 1)
    LAUNCH(CAMS_PROF_GALERKIN, launch_galerkin_fe(h->g, h->c, h->single, nonsym, b, h->stream));
  else
    LAUNCH(CAMS_PROF_GALERKIN, launch_galerkin_fv(h->g, h->c, h->single, nonsym, b, h->stream));
  {
    ProfScope ps_(h, CAMS_PROF_COARSE_FACTOR);
    // MSFE with a symmetric A: R A P = P^T A P is symmetric (LDL^T), else band LU
    const int sym = o.restriction != 1 && !nonsym;
    h->coarse_ldlt = sym != 0;
    if (h->coarse_inv) {
      CK(launch_coarse_factor_inv(h->c, h->mc, b, h->stream));
    } else {
      CK(launch_band_fill(h->c, h->mc, sym, b, h->stream));
      CK(launch_band_factor(h->c.Nc, h->mc, sym, b, h->stream));
    }
  }
  if (h->coarse_inv) LAUNCH(CAMS_PROF_COARSE_INV, launch_coarse_zinv(h->c.Nc, h->mc, b, h->stream));
  if (overlap)
    CK(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  else
    LAUNCH(CAMS_PROF_ILU_FACTOR, launch_ilu_factor(h->g, b, h->ilu_pipelined, h->ilu_grid,
                                                    h->ilu_cta, h->single, nonsym, h->stream));
  return check_status(h);
}

int residual_norm(cams_handle* h, double* out) {
  LAUNCH(CAMS_PROF_RESIDUAL, launch_residual(h->g, h->b, h->b.p, h->b.r, h->b.red, h->b.scal, h->stream));
  double s2;
  int rc = read_scalar(h, &s2);
  if (rc) return rc;
  if (!std::isfinite(s2)) return fail(h, CAMS_ENAN, "non-finite residual norm");
  *out = std::sqrt(s2);
  return CAMS_OK;
}

// One ILU(0) smoothing step: p <- p + M^{-1}(f - A p) in FP64, or in mixed
// precision delta <- delta + M^{-1}(r - A delta) in FP32 (r the FP64
// residual of the current p).
int ilu_smooth(cams_handle* h) {
  const bool s = h->single;
  LAUNCH(CAMS_PROF_ILU_RESID, launch_ilu_resid(h->g, h->b, s, h->stream));
  LAUNCH(CAMS_PROF_ILU_FWD, launch_ilu_sweep(h->g, h->b, false, h->ilu_pipelined, h->ilu_grid, h->ilu_cta, s, h->stream));
  LAUNCH(CAMS_PROF_ILU_BWD, launch_ilu_sweep(h->g, h->b, true, h->ilu_pipelined, h->ilu_grid, h->ilu_cta, s, h->stream));
  LAUNCH(CAMS_PROF_ILU_APPLY, launch_ilu_apply(h->g, h->b, s, h->stream));
  return CAMS_OK;
}

// One C-AMS iteration (Table 1 steps 4-7 with ILU(0) smoothing).  On entry
// b.r holds f - A p for the current p (residual_norm computed it).
//
// Mixed precision runs the same iteration on the correction: delta =
// P (R A P)^{-1} R r, then n_post smoothing steps on A delta = r, then
// p += delta; f - A(p + delta) = r - A delta, so this is the FP64
// iteration with the preconditioner rounded to FP32.  Pre-smoothing steps
// are applied the same way and added to p before the coarse correction.
// With options.cf the pre-smoothing stage starts with the correction
// functions of r (Table 1 step 4): p += Psi, level by level.
int cams_step_direct(cams_handle* h) {
  Buffers& b = h->b;
  const bool s = h->single;
  if (h->opt.n_pre > 0 || h->opt.cf) {
    if (s) CK(cudaMemsetAsync(b.f32.d, 0, sizeof(float) * h->g.N, h->stream));
    if (h->opt.cf) {
      ProfScope ps_(h, CAMS_PROF_BASIS);         // the same local solves as the basis stages
      for (int lev = 1; lev <= 3; ++lev) {
        const int f = h->lev_first[lev];
        CK(launch_entity_cf(h->g, b.ents + f, h->lev_count[lev], h->lev_smem[lev],
                            h->lev_grid[lev], h->lev_lstride[lev], s, h->lev_blocked[lev],
                            h->lev_gbytes[lev], b,
                            h->stream));
      }
    }
    for (int k = 0; k < h->opt.n_pre; ++k) {
      int rc = ilu_smooth(h);
      if (rc) return rc;
    }
    if (s) LAUNCH(CAMS_PROF_UPDATE, launch_add_correction(h->g, b, h->stream));
    LAUNCH(CAMS_PROF_RESIDUAL, launch_residual(h->g, b, b.p, b.r, b.red, b.scal, h->stream));
  }
  const int fv = h->opt.restriction == 1;
  LAUNCH(CAMS_PROF_RESTRICT, launch_restrict(h->g, h->c, fv, b.r, s, b, h->stream));
  if (h->coarse_inv)
    LAUNCH(CAMS_PROF_COARSE_SOLVE, launch_coarse_solve_f32(h->c.Nc, h->mc, b, h->stream));
  else
    LAUNCH(CAMS_PROF_COARSE_SOLVE, launch_band_solve(h->c.Nc, h->mc, !fv && !h->opt.jacobian,
                                                     h->coarse_cluster, s, b, h->stream));
  LAUNCH(CAMS_PROF_PROLONG, launch_prolong_add(h->g, h->c, s, b, h->stream));
  for (int k = 0; k < h->opt.n_post; ++k) {
    int rc = ilu_smooth(h);
    if (rc) return rc;
  }
  if (s) LAUNCH(CAMS_PROF_UPDATE, launch_add_correction(h->g, b, h->stream));
  return CAMS_OK;
}

// Capture one iteration's launches (no host reads happen inside it) on a
// private stream into a graph.  Every pointer and size it uses is fixed for
// the handle's lifetime, so the graph is captured once and replayed on the
// handle's current stream.
int capture_step(cams_handle* h) {
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaStream_t own = h->stream;
  cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(h, CAMS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  h->stream = h->cap_stream;
  const long long l0 = lc::mine;
  const int rc = cams_step_direct(h);
  const long long l1 = lc::mine;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &graph);
  h->stream = own;
  lc::total -= l1 - l0;                        // captured, not launched
  lc::mine -= l1 - l0;
  if (rc || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : fail(h, CAMS_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&h->step_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->step_exec = nullptr;
    cudaGetLastError();
    return fail(h, CAMS_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
  }
  h->step_launches = l1 - l0;
  return CAMS_OK;
}

// Device side of the inner loop's stopping test (Sec. 4.1.1): scal[0] holds
// ||f - A p||^2 of the current iterate (the residual kernel's sum),
// scal[1] the same at the start of the linearisation, scal[2] the
// iterations run.  The test is the host loop's, in the same FP64 operations:
// continue while ||r|| >= lin_rtol ||r^0|| (and finite) and fewer than
// max_cams iterations have run.
__global__ void k_loop_begin(double* scal) {
  scal[1] = scal[0];
  scal[2] = 0.0;
}
__global__ void k_loop_ctrl(cudaGraphConditionalHandle cond, double* scal, int max_cams,
                            double lin_rtol) {
  const double its = scal[2] + 1.0;
  scal[2] = its;
  const double rn = sqrt(scal[0]), r0 = sqrt(scal[1]);
  const bool more = its < (double)max_cams && isfinite(rn) && !(rn < lin_rtol * r0);
  cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// Capture the inner loop: a graph holding one conditional WHILE node whose
// body is one C-AMS iteration, the residual norm and k_loop_ctrl (which
// sets the node's condition).  Like the single-iteration graph it is
// captured once (every pointer and size is fixed for the handle's life).
int capture_loop(cams_handle* h) {
  if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  // (the parameter union has no default constructor: zeroed raw storage)
  alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)] = {};
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(h, CAMS_ECUDA, std::string("loop graph: ") + cudaGetErrorString(e));
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t own = h->stream;
  e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return fail(h, CAMS_ECUDA, std::string("loop graph capture: ") + cudaGetErrorString(e));
  }
  h->stream = h->cap_stream;
  const long long l0 = lc::mine;
  int rc = cams_step_direct(h);
  if (!rc) {
    cudaError_t e2 = launch_residual(h->g, h->b, h->b.p, h->b.r, h->b.red, h->b.scal, h->stream);
    if (e2 == cudaSuccess) {
      k_loop_ctrl<<<1, 1, 0, h->stream>>>(cond, h->b.scal, h->opt.max_cams, h->opt.lin_rtol);
      count_launches(1);
      e2 = cudaGetLastError();
    }
    if (e2 != cudaSuccess) rc = fail(h, CAMS_ECUDA, std::string("loop graph body: ") + cudaGetErrorString(e2));
  }
  const long long l1 = lc::mine;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(h->cap_stream, &captured);
  h->stream = own;
  lc::total -= l1 - l0;                        // captured, not launched
  lc::mine -= l1 - l0;
  if (rc || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc ? rc : fail(h, CAMS_ECUDA, std::string("loop graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&h->loop_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->loop_exec = nullptr;
    cudaGetLastError();
    return fail(h, CAMS_ECUDA, std::string("loop graph instantiation: ") + cudaGetErrorString(e));
  }
  h->loop_body_launches = l1 - l0;
  return CAMS_OK;
}

// The inner loop of one linearisation on the device: from the residual of
// the current iterate (residual_norm just computed it), C-AMS iterations
// until ||r|| < lin_rtol ||r^0|| or max_cams.  *its and *rn receive the
// count and the final ||r||.  Returns CAMS_EINVAL (nothing launched) when
// the loop graph is unavailable, so the caller keeps its host loop.
int inner_loop_graph(cams_handle* h, int* its, double* rn) {
  if (h->prof || !h->graphs || !h->loop_graph) return CAMS_EINVAL;
  if (!h->loop_exec) {
    const int rc = capture_loop(h);
    if (rc) {
      h->loop_graph = false;                   // keep the host loop for this handle
      return CAMS_EINVAL;
    }
  }
  k_loop_begin<<<1, 1, 0, h->stream>>>(h->b.scal);
  count_launches(1);
  CK(cudaGetLastError());
  CK(cudaGraphLaunch(h->loop_exec, h->stream));
  double sc[3];
  CK(cudaMemcpyAsync(sc, h->b.scal, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *its = (int)sc[2];
  count_launches((long long)*its * h->loop_body_launches);
  if (!std::isfinite(sc[0])) return fail(h, CAMS_ENAN, "non-finite residual norm");
  *rn = std::sqrt(sc[0]);
  return CAMS_OK;
}

// One C-AMS iteration: the captured graph, or direct launches while
// per-kernel-class profiling is on (its events bracket every class).
int cams_step(cams_handle* h) {
  if (h->prof || !h->graphs) return cams_step_direct(h);
  if (!h->step_exec) {
    const int rc = capture_step(h);
    if (rc) {
      h->graphs = false;                       // keep the direct launches for this handle
      return cams_step_direct(h);
    }
  }
  CK(cudaGraphLaunch(h->step_exec, h->stream));
  count_launches(h->step_launches);
  return CAMS_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// Workspace of the tensor-core network entry points: a status word, then
// two BF16 activation buffers of 32 channels.
long long tc_work_bytes(int B, int S) {
  if (B < 1 || S < 1) return -1;
  return 256 + 2 * ((2 * net_tc_act_elems(B, S, kNetHid) + 255) / 256 * 256);
}

// Shared driver of the two tensor-core entry points: zero the workspace,
// run `body` on its two activation buffers, wait and read the status word.
template <class F>
int run_tc(int B, int S, void* work, long long work_bytes, cudaStream_t s, F body) {
  const long long need = tc_work_bytes(B, S);
  if (!work || work_bytes < need)
    return fail(nullptr, CAMS_EINVAL, "tensor-core workspace missing or smaller than "
                                      "cams_net_tc_work_bytes(B, S)");
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return fail(nullptr, CAMS_ECUDA, "no CUDA device available");
  if (!net_tc_fits(S, (int)prop.sharedMemPerBlockOptin))
    return fail(nullptr, CAMS_EINVAL, "the patch does not fit the tensor-core kernel's shared memory");
  char* base = static_cast<char*>(work);
  int* status = reinterpret_cast<int*>(base);
  const long long half = (need - 256) / 2;
  void* ta = base + 256;
  void* tb = base + 256 + half;
  cudaError_t e = cudaMemsetAsync(work, 0, (size_t)need, s);
  if (e == cudaSuccess) e = body(ta, tb, status, prop.multiProcessorCount);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  if (st & kStatTimeout) return fail(nullptr, CAMS_ETIMEOUT, "a tensor-core barrier wait exceeded its limit");
  return CAMS_OK;
}

}  // namespace

namespace cams {
void set_global_error(const std::string& msg) { g_setup_error = msg; }
void count_launches(long long n) {
  lc::total += n;
  lc::mine += n;
}

cudaError_t raise_smem_limit(const void* func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
long long launches_total() { return lc::total.load(); }
}  // namespace cams

// =================================================================== ABI ==

extern "C" {

int cams_setup(const cams_grid* grid, const cams_fluid* fluid, const cams_options* opt,
               const double* kx, const double* ky, const double* kz, cams_handle** out) {
  if (!out) return fail(nullptr, CAMS_EINVAL, "out is null");
  *out = nullptr;
  int rc = validate(grid, fluid, opt);
  if (rc) return rc;
  if (!kx) return fail(nullptr, CAMS_EINVAL, "kx is null");
  if (!ky) ky = kx;
  if (!kz) kz = kx;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(nullptr, CAMS_ECUDA, "no CUDA device available");
  cams_handle* h = new (std::nothrow) cams_handle();
  if (!h) return fail(nullptr, CAMS_ENOMEM, "host allocation failed");
  h->grid = *grid;
  h->fluid = *fluid;
  h->opt = *opt;
  h->single = opt->precision == CAMS_PREC_MIXED;
  cudaGetDevice(&h->dev);
  Geo& g = h->g;
  g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
  g.N = (long long)g.nx * g.ny * g.nz;
  g.sy = g.nx; g.sz = (long long)g.nx * g.ny;
  g.dx = grid->dx; g.dy = grid->dy; g.dz = grid->dz;
  g.V = grid->dx * grid->dy * grid->dz;
  h->fl = FluidK{fluid->law, fluid->c_or_eta, fluid->rho0, fluid->mu, fluid->phi};
  CGeo& c = h->c;
  const int n[3] = {g.nx, g.ny, g.nz};
  c.Nc = 1;
  for (int d = 0; d < 3; ++d) {
    c.b[d] = opt->coarse[d];
    c.o[d] = opt->coarse[d] / 2;
    c.nc[d] = n[d] / opt->coarse[d];
    c.Nc *= c.nc[d];
  }
  h->n_dual = (c.nc[0] + 1) * (c.nc[1] + 1) * (c.nc[2] + 1);
  // wirebasket entity tables
  std::vector<int> eoc((size_t)g.N, -1);
  build_entities(h, eoc);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->dev) != cudaSuccess) {
    delete h;
    return fail(nullptr, CAMS_ECUDA, "cudaGetDeviceProperties failed");
  }
  int smem_max = 0;
  for (int lev = 1; lev <= 3; ++lev) {
    int sm = 0, mmax = 0;
    long long ls = 0;
    for (int e = h->lev_first[lev]; e < h->lev_first[lev] + h->lev_count[lev]; ++e)
      mmax = std::max(mmax, h->ents[e].m);
    // wide bands (the 3D dual-block interiors) take the blocked local solver
    h->lev_blocked[lev] = mmax >= 16;
    for (int e = h->lev_first[lev]; e < h->lev_first[lev] + h->lev_count[lev]; ++e) {
      const Entity& E = h->ents[e];
      sm = std::max(sm, entity_smem_bytes(E, h->single, h->lev_blocked[lev]));
      ls = std::max(ls, (long long)E.n * (E.m + 1));
    }
    h->lev_smem[lev] = sm;
    h->lev_lstride[lev] = ls;
    if (h->lev_blocked[lev] && sm > (int)prop.sharedMemPerBlockOptin) {
      // the blocked solver's window in global memory (the 15^3 interiors of
      // 16^3 blocks): per CTA the same bytes, 256-byte aligned
      h->lev_gbytes[lev] = ((long long)sm + 255) / 256 * 256;
      continue;
    }
    smem_max = std::max(smem_max, sm);
  }
  if (smem_max > (int)prop.sharedMemPerBlockOptin) {
    delete h;
    return fail(nullptr, CAMS_EINVAL, "dual-coarse blocks too large for the shared-memory local solver");
  }
  if (set_entity_smem(std::max(smem_max, 1)) != cudaSuccess) {
    delete h;
    return fail(nullptr, CAMS_ECUDA, "cudaFuncSetAttribute failed");
  }
  for (int lev = 1; lev <= 3; ++lev) {
    const int per_sm = h->lev_gbytes[lev] ? 2 :
        std::max(1, (int)(prop.sharedMemPerMultiprocessor / std::max(h->lev_smem[lev] + 1024, 1)));
    h->lev_grid[lev] = std::min(h->lev_count[lev], prop.multiProcessorCount * std::min(per_sm, 8));
    h->lscratch_len = std::max(h->lscratch_len, (long long)h->lev_grid[lev] * h->lev_lstride[lev]);
    h->lwork_len = std::max(h->lwork_len, (long long)h->lev_grid[lev] * h->lev_gbytes[lev]);
  }
  // coarse ordering: fastest = fewest coarse cells
  int ordc[3] = {0, 1, 2};
  std::stable_sort(ordc, ordc + 3, [&](int a, int b2) { return c.nc[a] < c.nc[b2]; });
  const int na = c.nc[ordc[0]], nb = c.nc[ordc[1]], ncc = c.nc[ordc[2]];
  h->mc = (na > 1 ? 1 : 0) + (nb > 1 ? na : 0) + (ncc > 1 ? na * nb : 0);
  // an odd half-width makes m + 1 even, so every band column starts on a
  // 16-byte boundary (the substitution streams columns with 16-byte copies);
  // the extra diagonal is structurally zero
  if (h->mc % 2 == 0) h->mc += 1;
  std::vector<int> perm(c.Nc);
  for (int I = 0; I < c.Nc; ++I) {
    const int Ic[3] = {I % c.nc[0], (I / c.nc[0]) % c.nc[1], I / (c.nc[0] * c.nc[1])};
    perm[I] = Ic[ordc[0]] + na * (Ic[ordc[1]] + nb * Ic[ordc[2]]);
  }
  {
    // the mixed preconditioner's symmetric (MSFE) coarse solve by the FP32
    // inverse factor, where its work and memory stay small
    const char* ci = std::getenv("CAMS_COARSE_INV");
    h->coarse_inv = h->single && opt->restriction != 1 && !opt->jacobian &&
                    !(ci && ci[0] == '0') && coarse_inverse_ok(c.Nc, h->mc);
  }
  rc = alloc_all(h);
  if (rc) {
    const std::string msg = h->err;
    free_all(h);
    delete h;
    return fail(nullptr, rc, msg);
  }
  for (auto& x : h->ev) cudaEventCreate(&x);
  h->launch_base = launches_total();
  {
    const char* gr = std::getenv("CAMS_GRAPHS");
    h->graphs = !(gr && gr[0] == '0');
    const char* lg = std::getenv("CAMS_LOOP_GRAPH");
    h->loop_graph = !(lg && lg[0] == '0');
    const char* lv = std::getenv("CAMS_ILU_LEVEL");
    h->ilu_pipelined = !(lv && lv[0] == '1');
    h->ilu_grid = ilu_pipe_grid(h->g, prop.multiProcessorCount);
    // One tile per warp for both precisions (with the cross-tile loads
    // issued ahead of the operand copies it measured faster than 2 x 2 tile
    // blocks per CTA: 143 against 161 us a 4M-cell FP32 sweep).
    // CAMS_ILU_CTA=1 forces the tile blocks.
    const char* ct = std::getenv("CAMS_ILU_CTA");
    const bool want = ct && ct[0] == '1';
    h->ilu_cta = want && ilu_cta_ok(h->g, (int)prop.sharedMemPerBlockOptin);
    const char* cc = std::getenv("CAMS_COARSE_CLUSTER");
    h->coarse_cluster = !(cc && cc[0] == '0') &&
                        coarse_cluster_ok(h->c.Nc, (int)prop.sharedMemPerBlockOptin);
  }
  // copy tables and compute transmissibilities
  cudaStream_t s = h->stream;
  cudaMemcpyAsync(h->b.ents, h->ents.data(), sizeof(Entity) * h->ents.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->b.ent_of_cell, eoc.data(), sizeof(int) * g.N, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->b.perm, perm.data(), sizeof(int) * c.Nc, cudaMemcpyHostToDevice, s);
  {
    // the two coarse x-corners of every x (the prolongation's per-x table):
    // on a vertex plane the lower one only, else the nodes either side
    std::vector<int> jxt(2 * (size_t)g.nx);
    for (int x = 0; x < g.nx; ++x)
      for (int bit = 0; bit < 2; ++bit) {
        const int sft = x - c.o[0];
        int J;
        if (sft >= 0 && sft % c.b[0] == 0) J = bit ? -1 : sft / c.b[0];
        else {
          const int j = sft >= 0 ? sft / c.b[0] + 1 : 0;
          J = bit ? j : j - 1;
        }
        jxt[2 * x + bit] = (J >= 0 && J < c.nc[0]) ? J : -1;
      }
    cudaMemcpyAsync(h->b.jxt, jxt.data(), sizeof(int) * jxt.size(), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  h->perm = perm;
  cudaMemsetAsync(h->b.status, 0, sizeof(int), s);
  cudaMemsetAsync(h->b.Tbw, 0, sizeof(double) * g.ny * g.nz, s);
  cudaMemsetAsync(h->b.Tbe, 0, sizeof(double) * g.ny * g.nz, s);
  const double* k3[3] = {kx, ky, kz};
  double* dk[3] = {nullptr, nullptr, nullptr};
  if (opt->memspace == CAMS_HOST) {
    for (int d = 0; d < 3; ++d)
      for (long long i = 0; i < g.N; ++i)
        if (!(k3[d][i] > 0.0) || !std::isfinite(k3[d][i])) {
          free_all(h);
          delete h;
          return fail(nullptr, CAMS_EINVAL, "permeability must be positive and finite");
        }
    // stage through the work vectors r, f, eps (overwritten by the next assembly)
    double* stage[3] = {h->b.r, h->b.f, h->b.eps};
    for (int d = 0; d < 3; ++d) {
      cudaMemcpyAsync(stage[d], k3[d], sizeof(double) * g.N, cudaMemcpyHostToDevice, s);
      dk[d] = stage[d];
    }
  } else {
    for (int d = 0; d < 3; ++d) dk[d] = const_cast<double*>(k3[d]);
  }
  cudaError_t e = launch_transmissibility(g, fluid->mu, dk[0], dk[1], dk[2], 1, h->b, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    std::string msg = std::string("setup: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return fail(nullptr, CAMS_ECUDA, msg);
  }
  *out = h;
  return CAMS_OK;
}

int cams_set_permeability(cams_handle* h, const double* kx, const double* ky, const double* kz) {
  if (!h) return CAMS_EINVAL;
  if (!kx) return fail(h, CAMS_EINVAL, "kx is null");
  if (!ky) ky = kx;
  if (!kz) kz = kx;
  const Geo& g = h->g;
  const double* k3[3] = {kx, ky, kz};
  double* dk[3];
  if (h->opt.memspace == CAMS_HOST) {
    for (int d = 0; d < 3; ++d)
      for (long long i = 0; i < g.N; ++i)
        if (!(k3[d][i] > 0.0) || !std::isfinite(k3[d][i]))
          return fail(h, CAMS_EINVAL, "permeability must be positive and finite");
    double* stage[3] = {h->b.r, h->b.f, h->b.eps};
    for (int d = 0; d < 3; ++d) {
      CK(cudaMemcpyAsync(stage[d], k3[d], sizeof(double) * g.N, cudaMemcpyHostToDevice, h->stream));
      dk[d] = stage[d];
    }
  } else {
    for (int d = 0; d < 3; ++d) dk[d] = const_cast<double*>(k3[d]);
  }
  CK(launch_transmissibility(g, h->fluid.mu, dk[0], dk[1], dk[2], 1, h->b, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->built = false;
  h->assembled = false;
  return CAMS_OK;
}

int cams_selftest_wait(cams_handle* h) {
  if (!h) return CAMS_EINVAL;
  CK(launch_wait_selftest(h->g, h->b, h->stream));
  return check_status(h);
}

int cams_profile(cams_handle* h, int enable) {
  if (!h) return CAMS_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  prof_flush(h);
  h->prof = enable != 0;
  if (h->prof)
    for (double& v : h->prof_acc) v = 0.0;
  return CAMS_OK;
}

int cams_set_stream(cams_handle* h, void* stream) {
  if (!h) return CAMS_EINVAL;
  h->stream = static_cast<cudaStream_t>(stream);
  return CAMS_OK;
}

int cams_set_schedule(cams_handle* h, int ilu_cta, int coarse_cluster) {
  if (!h) return CAMS_EINVAL;
  if (ilu_cta < -1 || ilu_cta > 1 || coarse_cluster < -1 || coarse_cluster > 1)
    return fail(h, CAMS_EINVAL, "schedule values must be -1, 0 or 1");
  if (ilu_cta >= 0 && !h->ilu_pipelined)
    return fail(h, CAMS_EINVAL, "the level-scheduled sweeps have no tile schedule");
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, h->dev));
  if (ilu_cta == 1 && !h->ilu_cta && !ilu_cta_ok(h->g, (int)prop.sharedMemPerBlockOptin))
    return fail(h, CAMS_EINVAL, "2x2 tile blocks do not fit this grid's shared memory");
  if (coarse_cluster == 1 && !h->coarse_cluster &&
      !coarse_cluster_ok(h->c.Nc, (int)prop.sharedMemPerBlockOptin))
    return fail(h, CAMS_EINVAL, "the cluster coarse solve is not available for this coarse grid");
  CK(cudaStreamSynchronize(h->stream));
  if (ilu_cta >= 0) h->ilu_cta = ilu_cta == 1;
  if (coarse_cluster >= 0) h->coarse_cluster = coarse_cluster == 1;
  if (h->step_exec) {                          // it holds the previous schedule's kernels
    CK(cudaGraphExecDestroy(h->step_exec));
    h->step_exec = nullptr;
  }
  if (h->loop_exec) {
    CK(cudaGraphExecDestroy(h->loop_exec));
    h->loop_exec = nullptr;
  }
  return CAMS_OK;
}

int cams_get_schedule(cams_handle* h, int* ilu_cta, int* coarse_cluster) {
  if (!h) return CAMS_EINVAL;
  if (ilu_cta) *ilu_cta = h->ilu_cta ? 1 : 0;
  if (coarse_cluster) *coarse_cluster = h->coarse_cluster ? 1 : 0;
  return CAMS_OK;
}

int cams_assemble(cams_handle* h, const double* p_nu, const double* p_n, double dt,
                  const cams_bc* bc, double* eps_norm_out) {
  if (!h) return CAMS_EINVAL;
  if (!p_nu || !p_n) return fail(h, CAMS_EINVAL, "null pressure");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, CAMS_EINVAL, "dt must be > 0");
  h->dt = dt;
  CK(cudaMemcpyAsync(h->b.p, p_nu, sizeof(double) * h->g.N, kind_in(h), h->stream));
  CK(cudaMemcpyAsync(h->b.pn, p_n, sizeof(double) * h->g.N, kind_in(h), h->stream));
  int rc = set_sources(h, bc);
  if (rc) return rc;
  CK(launch_density(h->g, h->fl, h->b.pn, h->b.rhon, h->stream));
  double en = 0.0;
  rc = assemble(h, &en);
  if (rc) return rc;
  if (eps_norm_out) *eps_norm_out = en;
  return CAMS_OK;
}

int cams_update_basis(cams_handle* h, int force, int* n_rebuilt_out) {
  if (!h) return CAMS_EINVAL;
  return update_operators(h, force, n_rebuilt_out);
}

// Restriction 2 (Sec. 4.3): after the step's Newton loop has converged with
// MSFE, one MSFV coarse correction of the last linearisation (A, f at the
// converged p) with the current basis: p += P (R_FV A P)^{-1} R_FV (f - A p).
// The restricted residual then vanishes on every primal block.  FP64 in
// either precision (the mixed preconditioner's FP32 P is read and widened).
int closing_msfv(cams_handle* h) {
  Buffers& b = h->b;
  LAUNCH(CAMS_PROF_GALERKIN, launch_galerkin_fv(h->g, h->c, h->single, h->opt.jacobian != 0, b,
                                                h->stream));
  {
    ProfScope ps_(h, CAMS_PROF_COARSE_FACTOR);
    CK(launch_band_fill(h->c, h->mc, 0, b, h->stream));
    CK(launch_band_factor(h->c.Nc, h->mc, 0, b, h->stream));
  }
  LAUNCH(CAMS_PROF_RESIDUAL, launch_residual(h->g, b, b.p, b.r, b.red, b.scal, h->stream));
  LAUNCH(CAMS_PROF_RESTRICT, launch_restrict(h->g, h->c, 1, b.r, h->single, b, h->stream));
  LAUNCH(CAMS_PROF_COARSE_SOLVE, launch_band_solve(h->c.Nc, h->mc, 0, false, false, b, h->stream));
  LAUNCH(CAMS_PROF_PROLONG, launch_prolong_to_p(h->g, h->c, h->single, b, h->stream));
  return check_status(h);
}

int cams_iterate(cams_handle* h, int n, double* res_norms) {
  if (!h) return CAMS_EINVAL;
  if (!h->built) return fail(h, CAMS_EINVAL, "cams_update_basis must come first");
  double rn;
  int rc = residual_norm(h, &rn);
  if (rc) return rc;
  if (res_norms) res_norms[0] = rn;
  for (int k = 0; k < n; ++k) {
    rc = cams_step(h);
    if (rc) return rc;
    rc = residual_norm(h, &rn);
    if (rc) return rc;
    if (res_norms) res_norms[k + 1] = rn;
  }
  return check_status(h);
}

int cams_solve(cams_handle* h, const double* p_n, double dt, const cams_bc* bc, double* p_inout,
               cams_stats* stats) {
  if (!h) return CAMS_EINVAL;
  if (!p_n || !p_inout) return fail(h, CAMS_EINVAL, "null pressure");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(h, CAMS_EINVAL, "dt must be > 0");
  cams_stats st;
  std::memset(&st, 0, sizeof(st));
  cudaEvent_t* ev = h->ev;
  float t_asm = 0, t_pre = 0, t_it = 0;
  cudaEventRecord(ev[0], h->stream);
  h->dt = dt;
  CK(cudaMemcpyAsync(h->b.pn, p_n, sizeof(double) * h->g.N, kind_in(h), h->stream));
  CK(cudaMemcpyAsync(h->b.p, p_inout, sizeof(double) * h->g.N, kind_in(h), h->stream));
  int rc = set_sources(h, bc);
  if (rc) return rc;
  CK(launch_density(h->g, h->fl, h->b.pn, h->b.rhon, h->stream));
  const cams_options& o = h->opt;
  double e0 = 0.0;
  int result = CAMS_ENOCONV;
  for (int nu = 0; nu <= o.max_newton; ++nu) {
    cudaEventRecord(ev[1], h->stream);
    double en;
    rc = assemble(h, &en);
    if (rc) return rc;
    cudaEventRecord(ev[2], h->stream);
    cudaEventSynchronize(ev[2]);
    t_asm += elapsed(ev[1], ev[2]);
    if (nu == 0) e0 = en;
    if (nu < 65) st.eps_hist[nu] = en;
    const double ref = o.tol_abs ? 1.0 : e0;
    if (en == 0.0 || en < o.nl_tol * ref) {
      st.converged = 1;
      result = CAMS_OK;
      break;
    }
    if (nu == o.max_newton) break;
    int nb = 0;
    cudaEventRecord(ev[1], h->stream);
    rc = update_operators(h, 0, &nb);
    if (rc) return rc;
    cudaEventRecord(ev[2], h->stream);
    cudaEventSynchronize(ev[2]);
    t_pre += elapsed(ev[1], ev[2]);
    st.basis_rebuilt += nb;
    double r0, rn = 0.0;
    rc = residual_norm(h, &r0);
    if (rc) return rc;
    int its = 0;
    rc = inner_loop_graph(h, &its, &rn);
    if (rc == CAMS_EINVAL) {                   // host-driven loop (profiling on, or no loop graph)
      rc = CAMS_OK;
      while (its < o.max_cams) {
        rc = cams_step(h);
        if (rc) return rc;
        ++its;
        rc = residual_norm(h, &rn);
        if (rc) return rc;
        if (rn < o.lin_rtol * r0) break;
      }
    }
    if (rc) return rc;
    cudaEventRecord(ev[3], h->stream);
    cudaEventSynchronize(ev[3]);
    t_it += elapsed(ev[2], ev[3]);
    st.res_final = rn;
    st.cams_its += its;
    if (st.newton_its < 64) st.cams_per_newton[st.newton_its] = its;
    st.newton_its += 1;
  }
  if (result == CAMS_OK && o.restriction == 2 && st.newton_its > 0) {
    rc = closing_msfv(h);
    if (rc) return rc;
  }
  rc = check_status(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(p_inout, h->b.p, sizeof(double) * h->g.N, kind_out(h), h->stream));
  cudaEventRecord(ev[3], h->stream);
  CK(cudaStreamSynchronize(h->stream));
  st.t_assemble = t_asm;
  st.t_precond = t_pre;
  st.t_iterate = t_it;
  st.t_total = elapsed(ev[0], ev[3]);
  if (stats) *stats = st;
  if (result == CAMS_ENOCONV) fail(h, CAMS_ENOCONV, "max_newton reached without convergence");
  return result;
}

int cams_ensemble_solve(int n, cams_handle* const* h, const double* const* p_n, const double* dt,
                        const cams_bc* const* bc, double* const* p_inout, cams_stats* stats,
                        int* status, int n_workers) {
  if (n < 0) return fail(nullptr, CAMS_EINVAL, "n < 0");
  if (n == 0) return CAMS_OK;
  if (!h || !p_n || !dt || !bc || !p_inout || !status)
    return fail(nullptr, CAMS_EINVAL, "null ensemble array");
  {
    std::vector<cams_handle*> v(h, h + n);
    for (cams_handle* x : v)
      if (!x) return fail(nullptr, CAMS_EINVAL, "null handle in the ensemble");
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end())
      return fail(nullptr, CAMS_EINVAL, "a handle appears twice in the ensemble");
  }
  int nw = n_workers > 0 ? n_workers : (int)std::thread::hardware_concurrency();
  nw = std::max(1, std::min(nw, n));
  for (int k = 0; k < n; ++k) status[k] = CAMS_OK;
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaStream_t s = nullptr;
    int sdev = -1;
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      cams_handle* hk = h[k];
      if (cudaSetDevice(hk->dev) != cudaSuccess || cudaStreamSynchronize(hk->stream) != cudaSuccess) {
        status[k] = fail(hk, CAMS_ECUDA, "cannot reach the handle's device or stream");
        continue;
      }
      if (sdev != hk->dev) {
        if (s) cudaStreamDestroy(s);
        s = nullptr;
        sdev = -1;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
          s = nullptr;
          status[k] = fail(hk, CAMS_ECUDA, "cudaStreamCreate failed");
          continue;
        }
        sdev = hk->dev;
      }
      cudaStream_t own = hk->stream;
      hk->stream = s;
      status[k] = cams_solve(hk, p_n[k], dt[k], bc[k], p_inout[k], stats ? &stats[k] : nullptr);
      hk->stream = own;
    }
    if (s) {
      cudaSetDevice(sdev);
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nw; ++w) {
    try {
      pool.emplace_back(worker);
    } catch (...) {
      break;   // fewer workers: the remaining ones take the members
    }
  }
  worker();
  for (std::thread& t : pool) t.join();
  for (int k = 0; k < n; ++k)
    if (status[k] != CAMS_OK) return status[k];
  return CAMS_OK;
}

int cams_set_surrogate(cams_handle* h, const float* params, double gate_tol) {
  if (!h) return CAMS_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  free_surrogate(h);
  if (!(gate_tol > 0.0)) return CAMS_OK;
  if (!params) return fail(h, CAMS_EINVAL, "null surrogate parameters");
  const CGeo& c = h->c;
  if (h->g.nx < 2 || h->g.ny < 2 || h->g.nz < 2 || c.b[0] != c.b[1] || c.b[0] != c.b[2] || c.b[0] < 3)
    return fail(h, CAMS_EINVAL, "the surrogate needs a 3D grid with cubic coarse blocks (b >= 3)");
  int rc = surrogate_tables(h);
  if (rc) { free_surrogate(h); return rc; }
  const long long S3 = (long long)(h->surr_b + 1) * (h->surr_b + 1) * (h->surr_b + 1);
  h->surr_chunk = std::max(1, std::min(h->surr_n, 1024));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, h->dev));
  h->sms = prop.multiProcessorCount;
  // the tensor-core network when a patch and the weights fit shared memory
  const char* tcv = std::getenv("CAMS_NET_TC");
  h->surr_tc = !(tcv && tcv[0] == '0') &&
               net_tc_fits(h->surr_b + 1, (int)prop.sharedMemPerBlockOptin);
  rc = dalloc(h, &h->net, (size_t)kNetParams);
  if (!rc) rc = dalloc(h, &h->surr_x, (size_t)(h->surr_chunk * kNetIn * S3));
  if (h->surr_tc) {
    const size_t n = (size_t)net_tc_act_elems(h->surr_chunk, h->surr_b + 1, kNetHid);
    unsigned short *ta = nullptr, *tb = nullptr;     // BF16 storage
    if (!rc) rc = dalloc(h, &ta, n);
    if (!rc) rc = dalloc(h, &tb, n);
    h->surr_ta = ta;
    h->surr_tb = tb;
    // rows outside the output-tile range are never written: they hold the zero border
    if (!rc && (cudaMemset(ta, 0, 2 * n) != cudaSuccess || cudaMemset(tb, 0, 2 * n) != cudaSuccess))
      rc = fail(h, CAMS_ECUDA, "cudaMemset failed");
  } else {
    if (!rc) rc = dalloc(h, &h->surr_h1, (size_t)(h->surr_chunk * kNetHid * S3));
    if (!rc) rc = dalloc(h, &h->surr_h2, (size_t)(h->surr_chunk * kNetHid * S3));
  }
  if (!rc) rc = dalloc(h, &h->surr_y, (size_t)(h->surr_chunk * kNetOut * S3));
  if (!rc) rc = dalloc(h, &h->surr_ratio, (size_t)h->surr_n);
  if (rc) { free_surrogate(h); return rc; }
  CK(cudaMemcpy(h->net, params, sizeof(float) * kNetParams, cudaMemcpyHostToDevice));
  h->surr_tol = gate_tol;
  return CAMS_OK;
}

int cams_surrogate_data(cams_handle* h, int max_patches, float* x, float* target, float* mask,
                        int* n_out) {
  if (!h || !n_out) return CAMS_EINVAL;
  if (!h->built) return fail(h, CAMS_EINVAL, "cams_update_basis must come first");
  if (h->surr_n == 0 && !h->surr_org) {
    const CGeo& c = h->c;
    if (h->g.nx < 2 || h->g.ny < 2 || h->g.nz < 2 || c.b[0] != c.b[1] || c.b[0] != c.b[2] || c.b[0] < 3)
      return fail(h, CAMS_EINVAL, "the surrogate needs a 3D grid with cubic coarse blocks (b >= 3)");
    int rc = surrogate_tables(h);
    if (rc) return rc;
  }
  if (max_patches <= 0) {           // how many there are
    *n_out = h->surr_n;
    return CAMS_OK;
  }
  const int n = std::min(max_patches, h->surr_n);
  *n_out = n;
  if (n == 0) return CAMS_OK;
  if (!x || !target || !mask) return fail(h, CAMS_EINVAL, "null patch arrays");
  CK(launch_patch_inputs(h->g, h->surr_b, n, h->surr_org, h->single, h->b, x, target, mask,
                         h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAMS_OK;
}

int cams_net_conv_forward(int B, int S, int ci, int co, const float* x, const float* w,
                          const float* bias, int relu, float* y, void* stream) {
  if (B < 0 || S < 1 || ci < 1 || co < 1 || !x || !w || !bias || !y)
    return fail(nullptr, CAMS_EINVAL, "bad convolution arguments");
  if (B == 0) return CAMS_OK;
  cudaError_t e = launch_conv_fwd(B, S, ci, co, x, w, bias, relu, y, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  return CAMS_OK;
}

int cams_net_conv_backward(int B, int S, int ci, int co, const float* x, const float* w,
                           const float* gy, const float* xact, float* gx, float* gw,
                           float* gbias, void* stream) {
  if (B < 1 || S < 1 || ci < 1 || co < 1 || !x || !w || !gy || !gw || !gbias)
    return fail(nullptr, CAMS_EINVAL, "bad convolution arguments");
  cudaError_t e = launch_conv_bwd(B, S, ci, co, x, w, gy, xact, gx, gw, gbias,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  return CAMS_OK;
}

long long cams_net_tc_work_bytes(int B, int S) { return tc_work_bytes(B, S); }

int cams_net_conv_forward_tc(int B, int S, int ci, int co, const float* x, const float* w,
                             const float* bias, int relu, float* y, void* work,
                             long long work_bytes, void* stream) {
  if (B < 0 || S < 1 || ci < 1 || ci > kNetHid || co < 1 || co > kNetHid || !x || !w || !bias || !y)
    return fail(nullptr, CAMS_EINVAL, "bad convolution arguments");
  if (B == 0) return CAMS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return run_tc(B, S, work, work_bytes, s, [&](void* ta, void*, int* status, int sms) {
    cudaError_t e = launch_tc_pack(B, S, ci, x, ta, s);
    if (e == cudaSuccess) e = launch_conv_tc(B, S, ci, co, ta, w, bias, relu, false, y, status, sms, s);
    return e;
  });
}

int cams_net_forward_tc(int B, int S, const float* x, const float* params, float* y, void* work,
                        long long work_bytes, void* stream) {
  if (B < 0 || S < 1 || !x || !params || !y) return fail(nullptr, CAMS_EINVAL, "bad network arguments");
  if (B == 0) return CAMS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float *w1 = params, *b1 = w1 + kNetHid * kNetIn * 27;
  const float *w2 = b1 + kNetHid, *b2 = w2 + kNetHid * kNetHid * 27;
  const float *w3 = b2 + kNetHid, *b3 = w3 + kNetHid * kNetHid * 27;
  const float *w4 = b3 + kNetHid, *b4 = w4 + kNetOut * kNetHid * 27;
  return run_tc(B, S, work, work_bytes, s, [&](void* ta, void* tb, int* status, int sms) {
    cudaError_t e = launch_tc_pack(B, S, kNetIn, x, ta, s);
    if (e == cudaSuccess) e = launch_conv_tc(B, S, kNetIn, kNetHid, ta, w1, b1, 1, true, tb, status, sms, s);
    if (e == cudaSuccess) e = launch_conv_tc(B, S, kNetHid, kNetHid, tb, w2, b2, 1, true, ta, status, sms, s);
    if (e == cudaSuccess) e = launch_conv_tc(B, S, kNetHid, kNetHid, ta, w3, b3, 1, true, tb, status, sms, s);
    if (e == cudaSuccess) e = launch_conv_tc(B, S, kNetHid, kNetOut, tb, w4, b4, 0, false, y, status, sms, s);
    return e;
  });
}

int cams_net_mse(long long n, const float* pred, const float* target, const float* mask,
                 double count, float* grad, double* loss, double* scratch, void* stream) {
  if (n < 1 || !(count > 0.0) || !pred || !target || !mask || !grad || !loss || !scratch)
    return fail(nullptr, CAMS_EINVAL, "bad loss arguments");
  cudaError_t e = launch_mse(n, pred, target, mask, count, grad, scratch, loss,
                             static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  return CAMS_OK;
}

int cams_net_energy(int B, int S, int C, int cx, const float* pred, const float* target,
                    const float* mask, const float* x, double count, float* grad, double* loss,
                    double* scratch, void* stream) {
  if (B < 1 || S < 2 || C < 1 || cx < 3 || !(count > 0.0) || !pred || !target || !mask || !x ||
      !grad || !loss || !scratch)
    return fail(nullptr, CAMS_EINVAL, "bad energy-loss arguments");
  cudaError_t e = launch_energy(B, S, C, cx, pred, target, mask, x, count, grad, scratch, loss,
                                static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  return CAMS_OK;
}

int cams_net_adam(long long n, float* p, const float* g, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int step, void* stream) {
  if (n < 1 || step < 1 || !p || !g || !m || !v) return fail(nullptr, CAMS_EINVAL, "bad Adam arguments");
  cudaError_t e = launch_adam(n, p, g, m, v, lr, beta1, beta2, eps, step,
                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, CAMS_ECUDA, cudaGetErrorString(e));
  return CAMS_OK;
}

int cams_get(cams_handle* h, int what, double* dst) {
  if (!h || !dst) return CAMS_EINVAL;
  const long long N = h->g.N;
  Buffers& b = h->b;
  const cudaMemcpyKind k = kind_out(h);
  cudaStream_t s = h->stream;
  switch (what) {
    case CAMS_Q_TRANS:
      CK(cudaMemcpyAsync(dst, b.Tx, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + N, b.Ty, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + 2 * N, b.Tz, sizeof(double) * N, k, s));
      break;
    case CAMS_Q_MATRIX:
      CK(cudaMemcpyAsync(dst, b.Ad, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + N, b.Ax, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + 2 * N, b.Ay, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + 3 * N, b.Az, sizeof(double) * N, k, s));
      break;
    case CAMS_Q_MATRIX_UPPER:
      CK(cudaMemcpyAsync(dst, b.Axu, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + N, b.Ayu, sizeof(double) * N, k, s));
      CK(cudaMemcpyAsync(dst + 2 * N, b.Azu, sizeof(double) * N, k, s));
      break;
    case CAMS_Q_RHS: CK(cudaMemcpyAsync(dst, b.f, sizeof(double) * N, k, s)); break;
    case CAMS_Q_EPS: CK(cudaMemcpyAsync(dst, b.eps, sizeof(double) * N, k, s)); break;
    case CAMS_Q_PRESSURE: CK(cudaMemcpyAsync(dst, b.p, sizeof(double) * N, k, s)); break;
    case CAMS_Q_PROLONG: {
      if (!h->single) {
        CK(cudaMemcpyAsync(dst, b.P, sizeof(double) * 8 * N, k, s));
        break;
      }
      std::vector<float> tf(8 * N);
      std::vector<double> td(8 * N);
      CK(cudaMemcpyAsync(tf.data(), b.f32.P, sizeof(float) * 8 * N, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (long long i = 0; i < 8 * N; ++i) td[i] = tf[i];
      CK(cudaMemcpyAsync(dst, td.data(), sizeof(double) * 8 * N,
                         h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      CK(cudaStreamSynchronize(s));
      break;
    }
    case CAMS_Q_COARSE: CK(cudaMemcpyAsync(dst, b.Acs, sizeof(double) * 27 * h->c.Nc, k, s)); break;
    case CAMS_Q_COARSE_FACTOR:
      if (!h->coarse_ldlt) return fail(h, CAMS_EINVAL, "the coarse matrix was not factored by L D L^T");
      CK(cudaMemcpyAsync(dst, b.Lc, sizeof(double) * h->c.Nc * (h->mc + 1), k, s));
      break;
    case CAMS_Q_ILU_DIAG: {
      // d_i = 1 / dinv_i, formed in the residual work vector
      std::vector<double> tmp(N);
      if (h->single) {
        std::vector<float> tf(N);
        CK(cudaMemcpyAsync(tf.data(), b.f32.dinv, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (long long i = 0; i < N; ++i) tmp[i] = 1.0 / (double)tf[i];
      } else {
        CK(cudaMemcpyAsync(tmp.data(), b.dinv, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (long long i = 0; i < N; ++i) tmp[i] = 1.0 / tmp[i];
      }
      CK(cudaMemcpyAsync(dst, tmp.data(), sizeof(double) * N,
                         h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      break;
    }
    case CAMS_Q_PROFILE: {
      CK(cudaStreamSynchronize(s));
      prof_flush(h);
      CK(cudaMemcpyAsync(dst, h->prof_acc, sizeof(h->prof_acc),
                         h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      break;
    }
    case CAMS_Q_LAUNCHES: {
      const double v = (double)(launches_total() - h->launch_base);
      CK(cudaMemcpyAsync(dst, &v, sizeof(double),
                         h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      CK(cudaStreamSynchronize(s));
      break;
    }
    case CAMS_Q_SURR_RATIO: {
      if (!h->surr_ratio) return fail(h, CAMS_EINVAL, "no surrogate on this handle");
      std::vector<float> tf(h->surr_n);
      std::vector<double> td(h->surr_n);
      CK(cudaMemcpyAsync(tf.data(), h->surr_ratio, sizeof(float) * h->surr_n, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int k = 0; k < h->surr_n; ++k) td[k] = tf[k];
      CK(cudaMemcpyAsync(dst, td.data(), sizeof(double) * h->surr_n,
                         h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s));
      break;
    }
    case CAMS_Q_RESIDUAL: {
      CK(launch_residual(h->g, b, b.p, b.r, b.red, b.scal, s));
      CK(cudaMemcpyAsync(dst, b.r, sizeof(double) * N, k, s));
      break;
    }
    default: return fail(h, CAMS_EINVAL, "unknown quantity");
  }
  CK(cudaStreamSynchronize(s));
  return CAMS_OK;
}

int cams_get_int(cams_handle* h, int what, int* dst) {
  if (!h || !dst) return CAMS_EINVAL;
  const long long N = h->g.N;
  if (what == CAMS_Q_SIZES) {
    dst[0] = (int)N; dst[1] = h->c.Nc; dst[2] = h->c.nc[0]; dst[3] = h->c.nc[1]; dst[4] = h->c.nc[2];
    dst[5] = (int)h->ents.size(); dst[6] = h->last_rebuilt; dst[7] = h->surr_accepted;
    return CAMS_OK;
  }
  if (what == CAMS_Q_COARSE_ORDER) {
    std::vector<int> v(h->c.Nc + 1);
    v[0] = h->mc;
    std::copy(h->perm.begin(), h->perm.end(), v.begin() + 1);
    CK(cudaMemcpyAsync(dst, v.data(), sizeof(int) * v.size(),
                       h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CAMS_OK;
  }
  if (what != CAMS_Q_PROLONG_J) return fail(h, CAMS_EINVAL, "unknown integer quantity");
  // coarse column of every slot, from the geometry (host computation)
  std::vector<int> J((size_t)8 * N);
  const CGeo& c = h->c;
  const int n[3] = {h->g.nx, h->g.ny, h->g.nz};
  for (long long i = 0; i < N; ++i) {
    const int xc[3] = {(int)(i % n[0]), (int)((i / n[0]) % n[1]), (int)(i / ((long long)n[0] * n[1]))};
    int cj[3][2];
    for (int d = 0; d < 3; ++d)
      for (int bit = 0; bit < 2; ++bit) {
        const int sft = xc[d] - c.o[d];
        int v;
        if (sft >= 0 && sft % c.b[d] == 0) v = bit ? -1 : sft / c.b[d];
        else {
          const int j = sft >= 0 ? sft / c.b[d] + 1 : 0;
          v = bit ? j : j - 1;
        }
        cj[d][bit] = (v >= 0 && v < c.nc[d]) ? v : -1;
      }
    for (int s = 0; s < 8; ++s) {
      const int a = cj[0][s & 1], b2 = cj[1][(s >> 1) & 1], z = cj[2][(s >> 2) & 1];
      J[(size_t)s * N + i] = (a < 0 || b2 < 0 || z < 0) ? -1 : a + c.nc[0] * (b2 + c.nc[1] * z);
    }
  }
  CK(cudaMemcpyAsync(dst, J.data(), sizeof(int) * 8 * N,
                     h->opt.memspace == CAMS_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CAMS_OK;
}

const char* cams_last_error(cams_handle* h) {
  return h ? h->err.c_str() : g_setup_error.c_str();
}

void cams_destroy(cams_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->aux_stream) cudaStreamSynchronize(h->aux_stream);
  free_surrogate(h);
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  if (h->loop_exec) cudaGraphExecDestroy(h->loop_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (auto& x : h->ev)
    if (x) cudaEventDestroy(x);
  prof_flush(h);
  for (auto& x : h->pool) cudaEventDestroy(x);
  free_all(h);
  delete h;
}

}  // extern "C"
