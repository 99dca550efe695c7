// Internal declarations shared by the libtsu translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsu.h"

namespace tsu {

constexpr int kMaxSing = 32;

struct DepthParams {
  double background, eps, c1, c2;
  int32_t mollifier, nsing;
  tsu_sing sing[kMaxSing];
};

// Geometry and coefficients every stencil launch needs.
struct StencilGeom {
  int32_t nx, ny;
  int64_t ld;
  double cx, cy;  // tau^2/dx^2, tau^2/dy^2
  double tau;
  double dxdy;
};

// Workspace of the steppers: a ticket counter and a device status word in the first 256 bytes,
// then per-CTA FP64 energy partials.
// The same workspace also holds, after the partials, the receiver table of the warp-blocked pass:
// tile t's entries are rec_ent[rec_off[t] .. rec_off[t + 1]) (int4: row, col, receiver, 0), for
// at most rec_tiles_cap tiles and rec_ent_cap receivers.
struct EnergyWs {
  unsigned int* counter;
  int* status;
  double* partials;
  int64_t capacity;  // number of partial slots
  int* rec_off;
  int4* rec_ent;
  int64_t rec_tiles_cap;
  int32_t rec_ent_cap;
  void* flow;              // the persistent warp-blocked pass's counters and energy partials, or nullptr
  int64_t flow_tiles_cap;  // tiles it holds room for
};

// The persistent warp-blocked pass (k_leapfrog_wtb_flow): energy partials of kFlowSlots passes
// in flight at once, for grids of at most kFlowMaxTiles tiles.  Its region of the workspace: a
// 128-byte header (task counter, per-slot tile counts and last reduced pass), a done counter per
// tile, then [kFlowSlots][4][tiles rounded up to 4] doubles.
constexpr int kFlowSlots = 8;
constexpr int64_t kFlowMaxTiles = 32768;
inline size_t flow_bytes(int64_t tiles) {
  const size_t t4 = (size_t)(tiles + 3) / 4 * 4;
  return 128 + (t4 * sizeof(int) + 15) / 16 * 16 + (size_t)kFlowSlots * 4 * t4 * sizeof(double);
}

// receivers the warp-blocked pass records itself (longer lists go one step per pass)
constexpr int32_t kWtbMaxReceivers = 2048;

// Rows per CTA of the one-step passes when the caller does not choose: 32, halved (down to 4)
// until the grid has at least 4 CTAs per SM (152 SMs), so that small grids still fill the GPU.
inline int auto_rows(int64_t ld, int64_t ny, int64_t cols_per_cta) {
  const int64_t cx = (ld + cols_per_cta - 1) / cols_per_cta;
  int rows = 32;
  while (rows > 4 && cx * ((ny - 2 + rows - 1) / rows) < 4 * 152) rows /= 2;
  return rows;
}

size_t energy_ws_bytes(int64_t ny, int64_t ld);

// Argument checks shared by the entry points (tsu_api.cu, tsu_noalloc.cu).  Each returns TSU_OK,
// or a status code after writing a message into err[0 .. n).
int check_grid(const tsu_grid* g, char* err, size_t n);
int check_dtype(int dtype, char* err, size_t n);
int check_field(const void* p, const char* name, char* err, size_t n);
// tau finite and positive, the medium's extrema consistent (positive depth, or a face family that
// is identically zero) and tau inside the leapfrog bound
int check_medium(const tsu_grid* g, double tau, const tsu_medium* m, char* err, size_t n);
int check_state(const tsu_state* st, bool need_roles, char* err, size_t n);
EnergyWs energy_ws_carve(void* ws, size_t bytes, int64_t ny, int64_t ld);

// Host-side mollifier normalisers, computed once by double-exponential quadrature.
double friedrichs_c1();
double friedrichs_c2();

cudaError_t launch_make_depth(const tsu_grid& g, const DepthParams& p, int dtype, void* hx, void* hy,
                              double* ext_dev, cudaStream_t s);

// Deterministic reductions (k_reduce.cu): kReduceBlocks per-block FP64 partials, then one block.
constexpr int kReduceBlocks = 152 * 4;
cudaError_t launch_sum_partials(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t s);
// out[0] = sum (a - b)^2, out[1] = sum b^2 over nodes i < nx; partials: 2 kReduceBlocks doubles
cudaError_t launch_diff_norms(const tsu_grid& g, int dtype, const void* a, const void* b, double* partials,
                              double* out, cudaStream_t s);
// d h_eps / d eps at the faces (k_depth.cu), and its contraction with face gradients
cudaError_t launch_depth_deps(const tsu_grid& g, const DepthParams& p, int dtype, void* dhx, void* dhy,
                              cudaStream_t s);
cudaError_t launch_eps_gradient(const tsu_grid& g, const DepthParams& p, const double* gx, const double* gy,
                                double* partials, double* out, cudaStream_t s);

// Optional per-step side outputs of a stencil pass.
struct PassOut {
  double* energy;           // one double, or nullptr
  EnergyWs ews;
  int32_t nrec;
  const int64_t* rec_idx;
  void* trace;              // nrec elements, or nullptr
  void* ckpt_a;             // checkpoint slot field 0 (u^{n-1} or u^n), or nullptr
  void* ckpt_b;             // checkpoint slot field 1
};

cudaError_t launch_init(const StencilGeom& g, int dtype, int form, const void* hx, const void* hy,
                        const void* u0, const void* u1, tsu_state* st, cudaStream_t s);

// CTAs of one launch of the one-step pass (launch_step) for this grid, element type and rows per
// CTA (rows <= 0: the automatic choice): one energy partial sum each.
int64_t one_step_ctas(int64_t ld, int64_t ny, int dtype, int rows);

// One leapfrog pass (standard or increment form) over the interior; store=false computes only
// the side outputs (energy of the current pair, traces).
cudaError_t launch_step(const StencilGeom& g, int dtype, int form, const void* hx, const void* hy,
                        const void* u_prev, const void* u_cur, void* v, void* u_next, const PassOut& o,
                        bool store, int rows, cudaStream_t s);

// Temporally blocked FP32 pass (k_step_tb.cu): k in {4, 8} steps per launch.
bool tb_supported_depth(int k);
int64_t tb_energy_slots(int64_t ny, int64_t ld, int k, int rows);
cudaError_t launch_step_tb(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                           const void* p, void* out_a, void* out_b, double* energy, const EnergyWs& ews, int* status,
                           int rows, int debug_flags, cudaStream_t s);

// Warp-blocked FP32 pass (k_step_wtb.cu): k in {2, 4} steps per launch, no CTA barriers.
bool wtb_supported_depth(int k);
int64_t wtb_tiles(int64_t ny, int64_t ld, int rows);
int wtb_auto_rows(int64_t ny, int64_t ld, int k);
int64_t wtb_energy_slots(int64_t ny, int64_t ld, int k, int rows);
// traces (optional): traces[t * nrec + r] = u^{n+t}[rec_idx[r]] for t = 0 .. k-1
cudaError_t launch_step_wtb(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                            const void* p, void* out_a, void* out_b, double* energy, const EnergyWs& ews, int rows,
                            cudaStream_t s, int32_t nrec = 0, const int64_t* rec_idx = nullptr,
                            void* traces = nullptr);
int wtb_seg_rows(int64_t ny, int64_t ld);
// the receiver table of the warp-blocked pass for this grid and rows per chunk (one CTA, into the
// workspace): every interior receiver under the tile whose output region holds it
cudaError_t launch_wtb_rec_table(const StencilGeom& g, int rows, const int64_t* rec_idx, int32_t nrec,
                                 const EnergyWs& ews, cudaStream_t s);
// traces of receivers on the boundary or outside the grid (0) for nsteps steps: the warp-blocked
// pass records interior receivers only
cudaError_t launch_wtb_trace_edges(const StencilGeom& g, const int64_t* rec_idx, int32_t nrec, void* traces,
                                   int64_t nsteps, cudaStream_t s);
// segment variant: u^{n+t} into seg + (t - 1) seg_stride for t = 1 .. k (elements), v^{n+k} into
// v_out (increment form; unused in the standard form)
// rows per tile of the persistent pass (k_leapfrog_wtb_flow) on this device
int wtb_flow_rows(int64_t ny, int64_t ld);
// whether the automatic kernel choice takes the persistent pass for this grid
bool wtb_flow_preferred(int64_t ny, int64_t ld);
// All nsteps / 4 passes of the warp-blocked pass (increment form, K = 4) in one persistent
// launch: pass p reads (u, v)[p & 1] and writes (u, v)[(p + 1) & 1]; energy (K doubles per pass)
// or nullptr; debug bit 1: the failure-detection test hook (tsu_step_opts.reserved).  *ran =
// false and nothing enqueued when the device, the workspace or the grid do not allow it.
cudaError_t launch_step_wtb_flow(const StencilGeom& g, const void* hx, const void* hy, void* const u[2], void* const v[2],
                                 double* energy, const EnergyWs& ews, int rows, int64_t npass, int debug, cudaStream_t s,
                                 bool* ran);
cudaError_t launch_step_wtb_seg(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                                const void* p, void* seg, int64_t seg_stride, void* v_out, int rows, cudaStream_t s);
// batched warp-blocked pass: descriptors of wtb_args_bytes() each, int4 tiles (problem, strip, chunk);
// wtb_strips(ld) strips per row of tiles
int64_t wtb_strips(int64_t ld);
size_t wtb_args_bytes();
void wtb_fill_args(void* dst, const StencilGeom& g, const void* hx, const void* hy, const void* u, const void* p,
                   void* out_a, void* out_b, int rows);
cudaError_t launch_step_wtb_batched(int form, int k, const void* probs_dev, size_t stride, const void* tiles_dev,
                                    int64_t ntiles, cudaStream_t s);

// Batched family (k_step_tb.cu): per-problem descriptors (tb_args_bytes() each, filled on the
// host by tb_fill_args) and an int4 tile table (problem, strip, chunk, 0).
size_t tb_args_bytes();
int tb_strip_width(int k);
void tb_fill_args(void* dst, const StencilGeom& g, const void* hx, const void* hy, const void* u, const void* p,
                  void* out_a, void* out_b, int* status, int rows);
cudaError_t launch_step_tb_batched(int form, int k, const void* probs_dev, const void* tiles_dev, int64_t ntiles,
                                   cudaStream_t s);

// Adjoint (k_adjoint.cu).
// Receivers bucketed by the adjoint-pass CTA owning their node (off[ncta+1], ord[nrec]) and the
// values g[r] injected into lam^n by that CTA after its stores; off == nullptr: no injection.
struct RecBuckets {
  const int* off;
  const int* ord;
  const int64_t* idx;
  const void* g;
};
void adjoint_pass_shape(const StencilGeom& g, int dtype, int64_t* gridx, int64_t* gridy, int* rows,
                        int64_t* cols_per_cta);
cudaError_t launch_rec_bucket(const StencilGeom& g, int dtype, const int64_t* idx, int32_t nrec, int* off, int* ord,
                              int* cta_of, cudaStream_t s);
// One reverse step (mode kAdjStep / kAdjStepInc) or the start (kAdjStart / kAdjStartInc).  The
// increment modes read mu = lam^{n+1} - lam^{n+2} from lam_pp and write mu^n into mu_out (which may
// be lam_pp); see k_adjoint.cu.
enum { kAdjStep = 0, kAdjStart = 1, kAdjStepInc = 2, kAdjStartInc = 3 };
cudaError_t launch_adjoint_pass(const StencilGeom& g, int dtype, int mode, const void* hx, const void* hy,
                                const void* lam, const void* lam_pp, void* lam_out, void* mu_out, const void* u,
                                void* gx, void* gy, void* g_u1, const RecBuckets& rb, cudaStream_t s);
cudaError_t launch_inject(const StencilGeom& g, int dtype, void* lam, const void* gvals, const int64_t* idx,
                          int32_t nrec, cudaStream_t s);
// K = 2 or 4 adjoint steps per pass, FP32, increment form (k_adjoint_wtb.cu): from lam^{n+1},
// mu^{n+1} = lam^{n+1} - lam^{n+2} and u[f] = u^{n-f} (f < K), the steps n .. n-K+1; stores
// lam^{n-K+1} into out_lam and mu^{n-K+1} into out_mu and adds the K steps' face gradients into
// gx, gy.  Receivers through a per-tile table (off[ntiles+1], int4 (row, col, receiver, 0)
// entries, <= 4 per receiver) built by launch_rec_tiles for the same K and rows; gv[f] = g^{n-f}
// at the receivers.
int adjoint_wtb_rows(int k, int64_t ny, int64_t ld);
int64_t adjoint_wtb_tiles(int64_t ny, int64_t ld, int rows);
cudaError_t launch_rec_tiles(const StencilGeom& g, int k, const int64_t* idx, int32_t nrec, int rows, int* off,
                             int4* ent, cudaStream_t s);
cudaError_t launch_adjoint_wtb(const StencilGeom& g, int k, int rows, const void* hx, const void* hy,
                               const void* lam1, const void* mu1, const void* const* u, void* out_lam, void* out_mu,
                               void* gx, void* gy, const int* rec_off, const int4* rec, const void* const* gv,
                               cudaStream_t s);
cudaError_t launch_flush(const StencilGeom& g, void* g32x, void* g32y, double* gx, double* gy, cudaStream_t s);

// Implicit comparator (k_implicit.cu): the factorized scheme (I - s B_x)(I - s B_y) w = B u.
// Transposed fields have nx rows of ldT = roundup(ny, 32) elements.  Factor layout (elements):
// mx [ny][ld], myT [nx][ldT], kyT [nx][ldT]; workspace: zT [nx][ldT] then one scratch field of
// max(ny ld, nx ldT) elements.
struct ImplicitGeom {
  int32_t nx, ny;
  int64_t ld, ldT;
  double cx, cy, tau, sigma;
};
int64_t implicit_ldT(int32_t ny);
size_t implicit_factor_elems(const tsu_grid& g);
// workspace bytes: a 256-byte header (status word at byte 4), [nx][ldT] + max(ny ld, nx ldT) elements
size_t implicit_ws_bytes(const tsu_grid& g, size_t elem);
cudaError_t launch_implicit_factor(const ImplicitGeom& g, int dtype, const void* hx, const void* hy, void* fac,
                                   cudaStream_t s);
// start = true: u^0 = u0 on interior nodes (0 elsewhere; u0 may be u), v = tau u1 + w^0 / 2,
// u = u^0 + v; else nsteps steps (v += w^n, u += v) in place
cudaError_t launch_implicit(const ImplicitGeom& g, int dtype, const void* hx, const void* hy, const void* fac,
                            const void* u0, void* u, void* v, const void* u1, int64_t nsteps, bool start, void* ws,
                            cudaStream_t s);

}  // namespace tsu
