// Internal declarations of the C-AMS engine: handle layout, entity tables
// and the launchers of every kernel.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cams.h"

namespace cams {

constexpr int kMaxNewton = 64;

// Grid geometry as seen by the kernels.
struct Geo {
  int nx, ny, nz;
  long long N;
  long long sy, sz;    // strides of y and z (nx, nx*ny)
  double dx, dy, dz, V;
};

#ifdef __CUDACC__
// (x, y, z) of cell i.  Grids are below 2^31 cells (checked at setup), so
// 32-bit division will do (64-bit division is a long instruction sequence).
__device__ __forceinline__ void xyz_of(const Geo& g, long long i, int& x, int& y, int& z) {
  const unsigned u = (unsigned)i, nx = (unsigned)g.nx, ny = (unsigned)g.ny;
  const unsigned t = u / nx;
  x = (int)(u - t * nx);
  const unsigned s = t / ny;
  y = (int)(t - s * ny);
  z = (int)s;
}
#endif

// Coarse-grid geometry: primal block size b, coarse-node offset o = b/2,
// number of coarse cells nc per direction (inactive directions: b = 1,
// o = 0, nc = 1).
struct CGeo {
  int b[3], o[3], nc[3];
  int Nc;
};

// One local entity of the wirebasket: an edge segment (level 1), face patch
// (level 2) or dual-block interior (level 3).  It is the box of cells
// [org, org + L) where every lattice (non-free) direction has L = 1.
// The local solve orders the cells with dimension ord[0] fastest and ord[2]
// slowest (ascending extent) so that the band half-width m is minimal.
struct Entity {
  int org[3];
  int L[3];
  int level;
  int free_mask;    // bit d set when direction d is free
  int ord[3];
  int n;            // cells
  int m;            // band half-width of the local matrix
  int nrhs;         // 2^(number of free directions)
};

// Fluid parameters passed by value to kernels.
struct FluidK {
  int law;
  double c, rho0, mu, phi;
};

__host__ __device__ inline double rho_of(const FluidK& f, double p) {
#ifdef __CUDA_ARCH__
  return f.law == 0 ? f.rho0 * exp(f.c * p) : f.rho0 * (1.0 + f.c * p);
#else
  return 0.0;
#endif
}

// FP32 copies used by the mixed-precision preconditioner (allocated only
// when cams_options.precision is CAMS_PREC_MIXED).
struct SingleBuffers {
  float *Ad = nullptr, *Ax = nullptr, *Ay = nullptr, *Az = nullptr;   // A in FP32
  float *Axu = nullptr, *Ayu = nullptr, *Azu = nullptr;   // transposed couplings (alias Ax.. if symmetric)
  float *Qx = nullptr, *Qy = nullptr, *Qz = nullptr;      // ILU(0) pivot products (nonsymmetric A)
  float* dinv = nullptr;                                  // 1 / ILU(0) pivots
  float *Lx = nullptr, *Ly = nullptr, *Lz = nullptr;      // scaled couplings, skewed
  float *Ux = nullptr, *Uy = nullptr, *Uz = nullptr;
  float *rds = nullptr, *w = nullptr, *z = nullptr;       // smoother vectors, skewed
  float* d = nullptr;                                     // the correction delta (N)
  float* r = nullptr;                                     // the outer residual rounded to FP32 (N)
  float* P = nullptr;                                     // 8N, slot-major
  float* pc = nullptr;                                    // coarse solution (band order)
  // FP32 copy of the symmetric coarse factor (the substitution's operands)
  float *Lc = nullptr, *Lr = nullptr, *cblk = nullptr, *cdinv = nullptr;
  // the inverse-factor coarse solve: Z = L^{-1} of the FP32 copy Lc of the
  // FP64 factor (Nc x coarse_ldz(Nc), column-major), the partial sums of
  // Z b and t = D^{-1} Z b
  float *Z = nullptr, *tc = nullptr, *zpart = nullptr;
};

// Device buffers, one allocation each, owned by the handle.
struct Buffers {
  double *Tx = nullptr, *Ty = nullptr, *Tz = nullptr;     // transmissibilities (lower faces)
  double *Tbw = nullptr, *Tbe = nullptr;                  // Dirichlet faces (ny*nz)
  double *p = nullptr, *pn = nullptr;                     // iterate, previous time level
  double *rho = nullptr, *rhon = nullptr;
  double *Ad = nullptr, *Ax = nullptr, *Ay = nullptr, *Az = nullptr;  // A = C + A~
  // a_{i-e_d, i} stored at the upper cell i (Ax.. hold a_{i, i-e_d}); the same
  // arrays as Ax, Ay, Az while A is symmetric (the lagged Newton step)
  double *Axu = nullptr, *Ayu = nullptr, *Azu = nullptr;
  double *Qx = nullptr, *Qy = nullptr, *Qz = nullptr;     // a_{i,i-e_d} a_{i-e_d,i} (nonsymmetric A)
  double *Cacc = nullptr;                                 // V rho c (diagonal of C)
  double *f = nullptr, *eps = nullptr;
  double *src = nullptr;                                  // dense Q_i (N) or null
  unsigned char* fixm = nullptr;                          // prescribed-cell mask (N) or null
  int* fixc = nullptr;                                    // prescribed cells (list)
  double* fixv = nullptr;                                 // their pressures
  double *Abd = nullptr, *Abx = nullptr, *Aby = nullptr, *Abz = nullptr;  // basis operator
  double *snap = nullptr;                                 // 7N snapshot (adaptive)
  double *P = nullptr;                                    // 8N, slot-major
  int* ent_of_cell = nullptr;                             // N, -1 on vertices
  Entity* ents = nullptr;                                 // all entities, level-sorted
  unsigned char* flag = nullptr;                          // per entity
  double* lscratch = nullptr;                             // local L factors, per resident CTA
  unsigned char* lwork = nullptr;                         // local solver windows too large for shared memory
  double* loc = nullptr;                                  // FE local 8x8 blocks per dual block (64 each)
  double* Acs = nullptr;                                  // 27*Nc coarse stencil
  double* band = nullptr;                                 // coarse band (column-major)
  double* Fc = nullptr;                                   // its LU factor (general band layout)
  double *Lc = nullptr, *Lr = nullptr;                    // LDL^T factor, column/row-major
  double *cblk = nullptr, *cdinv = nullptr;               // block inverses / products, 1/d
  int* cabort = nullptr;                                  // abort flag of the cluster solve
  int* perm = nullptr;                                    // coarse natural -> band order
  int* jxt = nullptr;                                     // per x: the two coarse x-corners (-1: none)
  double *rc = nullptr, *pc = nullptr;                    // coarse vectors (band order)
  double* ywork = nullptr;                                // forward-solve vector of the global band solve
  double* dinv = nullptr;                                 // 1 / ILU(0) pivots
  // ILU(0) sweep vectors, skewed tile-major (ilu_skew_len elements each)
  double *Lx = nullptr, *Ly = nullptr, *Lz = nullptr;     // a_{i,i-e_d} / d_i
  double *Ux = nullptr, *Uy = nullptr, *Uz = nullptr;     // a_{i,i+e_d} / d_i
  double *rds = nullptr, *w = nullptr, *z = nullptr;      // D^{-1} r, forward / backward sweeps
  int* ctrl = nullptr;                                    // wavefront tickets, abort flag
  double* r = nullptr;                                    // residual (natural order)
  double* cf = nullptr;                                   // correction function Psi (N; FP64 with options.cf)
  double* red = nullptr;                                  // reduction partials
  double* scal = nullptr;                                 // reduced scalars (device)
  int* status = nullptr;                                  // device status word
  SingleBuffers f32;                                      // mixed precision only
};

// Bits of the device status word (set by kernels, read by the host).
enum : int { kStatSingular = 1, kStatNan = 2, kStatTimeout = 4, kStatBounds = 8 };

// Message returned by cams_last_error(NULL).
void set_global_error(const std::string& msg);

// Raise (never lower) a kernel's dynamic shared-memory limit on the current
// device to at least `bytes`.  Handles of different sizes share the kernels,
// so the limit is the largest any of them asked for; thread-safe.
cudaError_t raise_smem_limit(const void* func, int bytes);
template <class F>
cudaError_t raise_smem_limit(F* func, int bytes) {
  return raise_smem_limit(reinterpret_cast<const void*>(func), bytes);
}

// Kernels launched by this library in this process (read per handle as a
// difference around its calls).
void count_launches(long long n);
long long launches_total();

// Reductions use a fixed grid so results are bit-reproducible.
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

// ---- launchers (each returns the launch error) ----
cudaError_t launch_transmissibility(const Geo& g, double mu, const double* kx, const double* ky,
                                    const double* kz, int dirichlet, Buffers& b, cudaStream_t s);
cudaError_t launch_density(const Geo& g, const FluidK& fl, const double* p, double* rho,
                           cudaStream_t s);
// fixm: prescribed-cell mask (N bytes) or null; full: the full-Jacobian
// step (writes the transposed couplings b.Axu.., distinct arrays then)
cudaError_t launch_assemble(const Geo& g, const FluidK& fl, double dt, int dirichlet, double pw,
                            double pe, const unsigned char* fixm, bool full, Buffers& b,
                            cudaStream_t s);
cudaError_t launch_add_sources(int n, const int* cell, const double* rate, double* src,
                               long long N, cudaStream_t s);
cudaError_t launch_fix_cells(int n, const int* cell, const double* val, unsigned char* fixm,
                             double* p, long long N, cudaStream_t s);
cudaError_t launch_sumsq(const double* x, long long N, double* red, double* out, cudaStream_t s);
cudaError_t launch_residual(const Geo& g, const Buffers& b, const double* p, double* r,
                            double* red, double* out, cudaStream_t s);
cudaError_t launch_basis_operator(const Geo& g, const FluidK& fl, int kind, double dt,
                                  const unsigned char* fixm, Buffers& b, cudaStream_t s);
cudaError_t launch_adapt_flags(const Geo& g, const Entity* ents, int count, double theta,
                               Buffers& b, unsigned char* flag, cudaStream_t s);
cudaError_t launch_adapt_propagate(const Geo& g, int first, int count, Buffers& b,
                                   cudaStream_t s);
cudaError_t launch_count_flags(int count, const unsigned char* flag, double* out, cudaStream_t s);
// single: P and the local solves in FP32 (mixed precision), else FP64.
cudaError_t launch_vertices(const Geo& g, const CGeo& c, Buffers& b, bool single, cudaStream_t s);
// blocked: panels of pivots with a register-tiled trailing update (large
// local problems); otherwise one pivot at a time.
// gbytes > 0: the blocked solver's window lives in b.lwork, gbytes per CTA
// (entities whose window exceeds shared memory), else in shared memory
cudaError_t launch_entity_solve(const Geo& g, const Entity* ents, const unsigned char* flag,
                                int count, int smem, int grid, long long lstride, int adaptive,
                                bool single, bool blocked, long long gbytes, Buffers& b,
                                cudaStream_t s);
int entity_smem_bytes(const Entity& E, bool single, bool blocked);
cudaError_t launch_entity_cf(const Geo& g, const Entity* ents, int count, int smem, int grid,
                             long long lstride, bool single, bool blocked, long long gbytes,
                             Buffers& b, cudaStream_t s);
cudaError_t set_entity_smem(int smem);
// nonsym: A is not symmetric (the full-Jacobian step)
cudaError_t launch_galerkin_fe(const Geo& g, const CGeo& c, bool single, bool nonsym, Buffers& b,
                               cudaStream_t s);
cudaError_t launch_galerkin_fv(const Geo& g, const CGeo& c, bool single, bool nonsym, Buffers& b,
                               cudaStream_t s);
cudaError_t launch_band_fill(const CGeo& c, int m, int sym, Buffers& b, cudaStream_t s);
cudaError_t launch_band_factor(int Nc, int m, int sym, Buffers& b, cudaStream_t s);
// The mixed preconditioner's symmetric coarse solve by the explicit inverse
// factor: the FP64 band LDL^T of the Galerkin matrix, its FP32 copy and
// Z = L^{-1} of that copy, then per solve f32.pc = Z^T D^{-1} Z rc.
// coarse_inverse_ok bounds its work and memory.
bool coarse_inverse_ok(int Nc, int m);
long long coarse_ldz(int Nc);        // leading dimension of Z (and length of t)
long long coarse_part_len(int Nc);   // partial sums of Z b
cudaError_t launch_coarse_factor_inv(const CGeo& c, int m, Buffers& b, cudaStream_t s);
cudaError_t launch_coarse_zinv(int Nc, int m, Buffers& b, cudaStream_t s);
cudaError_t launch_coarse_solve_f32(int Nc, int m, Buffers& b, cudaStream_t s);
cudaError_t launch_restrict(const Geo& g, const CGeo& c, int kind, const double* r, bool single,
                            Buffers& b, cudaStream_t s);
// the coarse solution into b.pc; with single into b.f32.pc for the FP32
// prolongation (the symmetric cluster solve then substitutes in FP32 with
// the FP32 copy of the factor)
cudaError_t launch_band_solve(int Nc, int m, int sym, bool cluster, bool single, Buffers& b,
                              cudaStream_t s);
long long coarse_blocks_len(int Nc);
bool coarse_cluster_ok(int Nc, int max_smem);
// FP64: p += P p_c; single: delta = P p_c (FP32 P and delta)
cudaError_t launch_prolong_add(const Geo& g, const CGeo& c, bool single, Buffers& b,
                               cudaStream_t s);
// p += P p_c in FP64 whatever the precision of P
cudaError_t launch_prolong_to_p(const Geo& g, const CGeo& c, bool single, Buffers& b,
                                cudaStream_t s);
// single: the FP32 smoother of the mixed-precision preconditioner (on
// A delta = r, vectors in b.f32); otherwise the FP64 smoother on A p = f.
// sms: the SM count (from ilu_pipe_grid); cta: tiles in 2 x 2 blocks per CTA
// with shared-memory edges (ilu_cta_ok), else one tile per warp.
// nonsym: pivots from the products a_{i,i-e} a_{i-e,i} (b.Qx.., formed here)
cudaError_t launch_ilu_factor(const Geo& g, Buffers& b, bool pipelined, int sms, bool cta,
                              bool single, bool nonsym, cudaStream_t s);
cudaError_t launch_ilu_resid(const Geo& g, Buffers& b, bool single, cudaStream_t s);
cudaError_t launch_ilu_sweep(const Geo& g, Buffers& b, bool backward, bool pipelined, int sms,
                             bool cta, bool single, cudaStream_t s);
// x += z after the backward sweep (single: delta in FP32, else p)
cudaError_t launch_ilu_apply(const Geo& g, Buffers& b, bool single, cudaStream_t s);
bool ilu_cta_ok(const Geo& g, int max_smem);
cudaError_t launch_add_correction(const Geo& g, Buffers& b, cudaStream_t s);   // p += delta
int ilu_ctrl_ints(const Geo& g);
// Rows per wavefront tile (y, z) and the length of a skewed sweep vector.
constexpr int kIluTY = 8, kIluTZ = 4, kIluR = kIluTY * kIluTZ;   // one warp per tile
long long ilu_skew_len(const Geo& g);
int ilu_pipe_grid(const Geo& g, int num_sms);
cudaError_t launch_wait_selftest(const Geo& g, Buffers& b, cudaStream_t s);

// ---- learned basis surrogate (k_net.cu) ----
constexpr int kNetIn = 12, kNetHid = 32, kNetOut = 8;
constexpr long long kNetParams = (long long)kNetHid * kNetIn * 27 + kNetHid +
                                 2 * ((long long)kNetHid * kNetHid * 27 + kNetHid) +
                                 (long long)kNetOut * kNetHid * 27 + kNetOut;
cudaError_t launch_conv_fwd(int B, int S, int ci, int co, const float* x, const float* w,
                            const float* bias, int relu, float* y, cudaStream_t s);
cudaError_t launch_conv_bwd(int B, int S, int ci, int co, const float* x, const float* w,
                            const float* gy, const float* xact, float* gx, float* gw,
                            float* gbias, cudaStream_t s);
cudaError_t launch_mse(long long n, const float* p, const float* t, const float* mask,
                       double count, float* grad, double* part, double* loss, cudaStream_t s);
cudaError_t launch_adam(long long n, float* p, const float* g, float* m, float* v, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s);
cudaError_t launch_energy(int B, int S, int C, int cx, const float* p, const float* t,
                          const float* mask, const float* x, double count, float* grad, double* part,
                          double* loss, cudaStream_t s);
int mse_partial_blocks();
// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) path of the
// network (k_net_tc.cu).  Activations between layers are BF16 "chunked and
// padded" (a zero border around the patch, channels in chunks of 8); a
// buffer of net_tc_act_elems(B, S, C) BF16 values must start zeroed (only
// rows inside the output-tile range are ever written).
long long net_tc_act_elems(int B, int S, int C);
bool net_tc_fits(int S, int max_smem);
// FP32 [B][C][S^3] -> BF16 chunked-padded
cudaError_t launch_tc_pack(int B, int S, int C, const float* x, void* out, cudaStream_t s);
// one layer from a BF16 chunked-padded input: BF16 chunked-padded output
// (out_bf16, the next layer's input) or FP32 [B][co][S^3]; status gets
// kStatTimeout if an MMA barrier wait gives up
cudaError_t launch_conv_tc(int B, int S, int ci, int co, const void* x, const float* w,
                           const float* bias, int relu, bool out_bf16, void* y, int* status,
                           int sms, cudaStream_t s);
// patches of the full interior dual blocks: org = lower corner (x, y, z) per patch
cudaError_t launch_patch_inputs(const Geo& g, int b, int n, const int* org, bool single,
                                const Buffers& bf, float* x, float* target, float* mask,
                                cudaStream_t s);
cudaError_t launch_patch_apply(const Geo& g, int b, int n, const int* org, const float* y,
                               bool single, Buffers& bf, cudaStream_t s);
cudaError_t launch_patch_gate(const Geo& g, int b, int n, const int* org, const int* ent,
                              double tol, bool single, Buffers& bf, unsigned char* flag,
                              float* ratio, cudaStream_t s);

}  // namespace cams
