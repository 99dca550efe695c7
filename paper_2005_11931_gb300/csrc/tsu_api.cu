// C ABI of libtsu: argument validation, error reporting and launch sequencing.  All compute is
// in the kernels of k_*.cu; this file only checks arguments and enqueues work on the caller's
// stream.  See include/tsu.h for the contract of every entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <vector>

#include "tsu_internal.h"

namespace {
thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(TSU_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// the shared checks (tsu::check_*) with this file's thread-local message buffer
int check_grid(const tsu_grid* g) { return tsu::check_grid(g, g_err, sizeof g_err); }
int check_dtype(int dtype) { return tsu::check_dtype(dtype, g_err, sizeof g_err); }
int check_field(const void* p, const char* name) { return tsu::check_field(p, name, g_err, sizeof g_err); }
int check_cfl(const tsu_grid* g, double tau, const tsu_medium* m) {
  return tsu::check_medium(g, tau, m, g_err, sizeof g_err);
}
int check_state(const tsu_state* st, bool need_roles) { return tsu::check_state(st, need_roles, g_err, sizeof g_err); }

// first buffer index that is neither cur nor aux
int scratch_index(const tsu_state* st, int skip) {
  for (int b = 0; b < st->nbuf; ++b)
    if (b != st->cur && b != st->aux && b != skip) return b;
  return -1;
}

tsu::StencilGeom geom(const tsu_grid* g, double tau) {
  tsu::StencilGeom s;
  s.nx = g->nx;
  s.ny = g->ny;
  s.ld = g->ld;
  s.cx = tau * tau / (g->dx * g->dx);
  s.cy = tau * tau / (g->dy * g->dy);
  s.tau = tau;
  s.dxdy = g->dx * g->dy;
  return s;
}

size_t elem_size(int dtype) { return dtype == TSU_F32 ? 4 : 8; }

#define TRY(x)                    \
  do {                            \
    int _rc = (x);                \
    if (_rc != TSU_OK) return _rc; \
  } while (0)
}  // namespace

namespace tsu {

namespace {
int errf(char* err, size_t n, int code, const char* fmt, ...) {
  if (err && n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, n, fmt, ap);
    va_end(ap);
  }
  return code;
}
}  // namespace

int check_grid(const tsu_grid* g, char* err, size_t n) {
  if (!g) return errf(err, n, TSU_EINVAL, "grid is NULL");
  if (g->nx < 3 || g->ny < 3) return errf(err, n, TSU_EINVAL, "grid needs nx, ny >= 3 (got %d x %d)", g->nx, g->ny);
  if (g->ld < g->nx || (g->ld % 4) != 0)
    return errf(err, n, TSU_EINVAL, "ld must be >= nx and a multiple of 4 (ld=%lld nx=%d)", (long long)g->ld, g->nx);
  if (!(g->dx > 0.0) || !(g->dy > 0.0) || !isfinite(g->dx) || !isfinite(g->dy))
    return errf(err, n, TSU_EINVAL, "dx, dy must be positive and finite");
  if ((int64_t)g->ny * g->ld >= ((int64_t)1 << 40)) return errf(err, n, TSU_EINVAL, "grid too large");
  return TSU_OK;
}

int check_dtype(int dtype, char* err, size_t n) {
  if (dtype != TSU_F32 && dtype != TSU_F64) return errf(err, n, TSU_EINVAL, "dtype must be TSU_F32 or TSU_F64");
  return TSU_OK;
}

int check_field(const void* p, const char* name, char* err, size_t n) {
  if (!p) return errf(err, n, TSU_EINVAL, "%s is NULL", name);
  if (((uintptr_t)p & 15u) != 0) return errf(err, n, TSU_EINVAL, "%s is not 16-byte aligned", name);
  return TSU_OK;
}

// One face family's extrema: a positive depth (0 < min <= max, Sec. 2: 0 < c0 <= h_j), or a
// family that is identically zero (min = max = 0: the equation decouples into 1D problems along
// the other direction, the paper's 1D setting).
static int check_family(double mn, double mx, const char* name, char* err, size_t n) {
  if (!(mx >= 0.0) || !isfinite(mx) || !isfinite(mn))
    return errf(err, n, TSU_EINVAL, "medium: %s extrema must be finite with max >= 0", name);
  if (mx == 0.0 && mn == 0.0) return TSU_OK;
  if (!(mn > 0.0) || mn > mx)
    return errf(err, n, TSU_ENONPOS, "medium: %s face depth minimum %.6g is not in (0, max = %.6g]", name, mn, mx);
  return TSU_OK;
}

// both families (and not both identically zero)
static int check_positive(const tsu_medium* m, char* err, size_t n) {
  int rc = check_family(m->hx_min, m->hx_max, "hx", err, n);
  if (rc != TSU_OK) return rc;
  rc = check_family(m->hy_min, m->hy_max, "hy", err, n);
  if (rc != TSU_OK) return rc;
  if (m->hx_max == 0.0 && m->hy_max == 0.0) return errf(err, n, TSU_ENONPOS, "medium: every face depth is 0");
  return TSU_OK;
}

int check_medium(const tsu_grid* g, double tau, const tsu_medium* m, char* err, size_t n) {
  if (!m) return errf(err, n, TSU_EINVAL, "medium is NULL");
  if (!(tau > 0.0) || !isfinite(tau)) return errf(err, n, TSU_EINVAL, "tau must be positive and finite");
  const int rc = check_positive(m, err, n);
  if (rc != TSU_OK) return rc;
  const double q = tau * tau * (m->hx_max / (g->dx * g->dx) + m->hy_max / (g->dy * g->dy));
  if (!(q <= 1.0))
    return errf(err, n, TSU_ECFL, "tau^2 (hx_max/dx^2 + hy_max/dy^2) = %.6g > 1: leapfrog unstable", q);
  return TSU_OK;
}

int check_state(const tsu_state* st, bool need_roles, char* err, size_t n) {
  if (!st) return errf(err, n, TSU_EINVAL, "state is NULL");
  if (st->form != TSU_FORM_STANDARD && st->form != TSU_FORM_INCREMENT) return errf(err, n, TSU_EINVAL, "bad form");
  const int need = st->form == TSU_FORM_STANDARD ? 2 : 3;
  if (st->nbuf < need || st->nbuf > 4)
    return errf(err, n, TSU_EINVAL, "state needs %d..4 buffers for this form (nbuf = %d)", need, st->nbuf);
  for (int b = 0; b < st->nbuf; ++b) {
    if (!st->buf[b] || ((uintptr_t)st->buf[b] & 15u))
      return errf(err, n, TSU_EINVAL, "state buf[%d] NULL or misaligned", b);
  }
  if (need_roles) {
    if (st->cur < 0 || st->cur >= st->nbuf || st->aux < 0 || st->aux >= st->nbuf || st->cur == st->aux)
      return errf(err, n, TSU_EINVAL, "state cur/aux invalid (%d, %d)", st->cur, st->aux);
  }
  return TSU_OK;
}

}  // namespace tsu

extern "C" {

int tsu_version(void) { return 100; }

const char* tsu_last_error(void) { return g_err; }

double tsu_tau_for(const tsu_grid* g, double hx_max, double hy_max, double cfl) {
  if (!g || !(g->dx > 0) || !(g->dy > 0) || !(cfl > 0) || cfl > 1 || !(hx_max >= 0) || !(hy_max >= 0)) return 0.0;
  const double s = hx_max / (g->dx * g->dx) + hy_max / (g->dy * g->dy);
  if (!(s > 0)) return 0.0;
  return cfl / sqrt(s);
}

double tsu_tau_courant(const tsu_grid* g, const tsu_medium* m, double courant) {
  if (!g || !m || !(g->dx > 0) || !(g->dy > 0) || !(courant > 0) || !isfinite(courant)) return 0.0;
  const double hmax = m->hx_max > m->hy_max ? m->hx_max : m->hy_max;
  if (!(hmax > 0) || !isfinite(hmax)) return 0.0;
  return courant * (g->dx < g->dy ? g->dx : g->dy) / sqrt(hmax);
}

// validated depth descriptor -> device parameters
static int depth_params(const tsu_depth* d, tsu::DepthParams* p_out) {
  if (!d) return fail(TSU_EINVAL, "depth is NULL");
  if (!(d->eps > 0.0) || !isfinite(d->eps)) return fail(TSU_EINVAL, "eps must be positive");
  if (d->nsing < 0 || d->nsing > tsu::kMaxSing) return fail(TSU_EINVAL, "nsing must be in [0, %d]", tsu::kMaxSing);
  if (d->nsing > 0 && !d->sing) return fail(TSU_EINVAL, "sing is NULL");
  if (d->mollifier != TSU_GAUSS && d->mollifier != TSU_FRIEDRICHS) return fail(TSU_EINVAL, "bad mollifier");
  tsu::DepthParams p;
  memset(&p, 0, sizeof p);
  p.background = d->background;
  p.eps = d->eps;
  p.mollifier = d->mollifier;
  p.nsing = d->nsing;
  p.c1 = tsu::friedrichs_c1();
  p.c2 = tsu::friedrichs_c2();
  for (int k = 0; k < d->nsing; ++k) {
    const tsu_sing& s = d->sing[k];
    if (s.kind < TSU_LINE_X || s.kind > TSU_STEP_Y) return fail(TSU_EINVAL, "sing[%d]: bad kind %d", k, s.kind);
    if (s.power < 1 || s.power > 8) return fail(TSU_EINVAL, "sing[%d]: power must be in [1, 8]", k);
    p.sing[k] = s;
  }
  *p_out = p;
  return TSU_OK;
}

int tsu_make_depth(const tsu_grid* g, const tsu_depth* d, int dtype, void* hx, void* hy, double* ext_dev,
                   double* ext_host, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_field(hx, "hx"));
  TRY(check_field(hy, "hy"));
  if (!ext_dev || ((uintptr_t)ext_dev & 7u)) return fail(TSU_EINVAL, "ext_dev must be a device double[4]");
  tsu::DepthParams p;
  TRY(depth_params(d, &p));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = tsu::launch_make_depth(*g, p, dtype, hx, hy, ext_dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_make_depth launch");
  if (ext_host) {
    e = cudaMemcpyAsync(ext_host, ext_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_make_depth extrema");
    if (!(ext_host[0] > 0.0) || !(ext_host[2] > 0.0))
      return fail(TSU_ENONPOS, "face depth minimum <= 0 (min hx = %.6g, min hy = %.6g)", ext_host[0], ext_host[2]);
  }
  return TSU_OK;
}

int tsu_depth_eps_derivative(const tsu_grid* g, const tsu_depth* d, int dtype, void* dhx, void* dhy, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_field(dhx, "dhx"));
  TRY(check_field(dhy, "dhy"));
  tsu::DepthParams p;
  TRY(depth_params(d, &p));
  cudaError_t e = tsu::launch_depth_deps(*g, p, dtype, dhx, dhy, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_depth_eps_derivative launch");
  return TSU_OK;
}

size_t tsu_reduce_workspace(void) { return 256 + 2 * (size_t)tsu::kReduceBlocks * sizeof(double); }

static int check_reduce(double* out_dev, void* ws, size_t ws_bytes) {
  if (!out_dev || ((uintptr_t)out_dev & 7u)) return fail(TSU_EINVAL, "out_dev must be a device double array");
  if (!ws || ws_bytes < tsu_reduce_workspace())
    return fail(TSU_ENOMEM, "reduction workspace %zu B < %zu B", ws_bytes, tsu_reduce_workspace());
  if ((uintptr_t)ws & 15u) return fail(TSU_EINVAL, "workspace must be 16-byte aligned");
  return TSU_OK;
}

int tsu_depth_eps_gradient(const tsu_grid* g, const tsu_depth* d, const double* g_hx, const double* g_hy,
                           double* out_dev, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_field(g_hx, "g_hx"));
  TRY(check_field(g_hy, "g_hy"));
  TRY(check_reduce(out_dev, ws, ws_bytes));
  tsu::DepthParams p;
  TRY(depth_params(d, &p));
  cudaError_t e = tsu::launch_eps_gradient(*g, p, g_hx, g_hy, (double*)((char*)ws + 256), out_dev,
                                           (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_depth_eps_gradient launch");
  return TSU_OK;
}

int tsu_diff_norms(const tsu_grid* g, int dtype, const void* a, const void* b, double* out_dev, void* ws,
                   size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_field(a, "a"));
  TRY(check_field(b, "b"));
  TRY(check_reduce(out_dev, ws, ws_bytes));
  cudaError_t e = tsu::launch_diff_norms(*g, dtype, a, b, (double*)((char*)ws + 256), out_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_diff_norms launch");
  return TSU_OK;
}

int tsu_init(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, const void* u0, const void* u1,
             tsu_state* st, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_cfl(g, tau, m));
  TRY(check_field(m->hx, "hx"));
  TRY(check_field(m->hy, "hy"));
  TRY(check_field(u0, "u0"));
  if (u1) TRY(check_field(u1, "u1"));
  TRY(check_state(st, false));
  cudaError_t e = tsu::launch_init(geom(g, tau), dtype, st->form, m->hx, m->hy, u0, u1, st, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_init launch");
  st->cur = st->form == TSU_FORM_STANDARD ? 1 : 0;
  st->aux = st->form == TSU_FORM_STANDARD ? 0 : 1;
  st->step = 1;
  return TSU_OK;
}

int tsu_step_workspace(const tsu_grid* g, int dtype, size_t* bytes) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  if (!bytes) return fail(TSU_EINVAL, "bytes is NULL");
  *bytes = tsu::energy_ws_bytes(g->ny, g->ld);
  return TSU_OK;
}


int tsu_step_n(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, tsu_state* st, int64_t nsteps,
               const tsu_step_opts* opts, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_cfl(g, tau, m));
  TRY(check_field(m->hx, "hx"));
  TRY(check_field(m->hy, "hy"));
  TRY(check_state(st, true));
  if (nsteps < 0) return fail(TSU_EINVAL, "nsteps must be >= 0");
  tsu_step_opts o;
  memset(&o, 0, sizeof o);
  if (opts) o = *opts;
  if (o.nrec < 0) return fail(TSU_EINVAL, "nrec must be >= 0");
  if (o.traces && (o.nrec == 0 || !o.rec_idx)) return fail(TSU_EINVAL, "traces need nrec > 0 and rec_idx");
  if (o.ckpt && (o.ckpt_every < 1 || o.ckpt_slots < 1 || !aligned16(o.ckpt)))
    return fail(TSU_EINVAL, "checkpoints need ckpt_every >= 1, ckpt_slots >= 1 and an aligned store");
  if (o.kernel < 0 || o.kernel > 4) return fail(TSU_EINVAL, "kernel must be 0..4");
  if (o.rows < 0) return fail(TSU_EINVAL, "rows must be >= 0");
  if (o.tdepth != 0 && o.kernel == 3 && !tsu::tb_supported_depth(o.tdepth))
    return fail(TSU_EINVAL, "kernel 3: tdepth must be 0, 4 or 8");
  if (o.tdepth != 0 && o.kernel == 2 && !tsu::wtb_supported_depth(o.tdepth))
    return fail(TSU_EINVAL, "kernel 2: tdepth must be 0, 2 or 4");
  const bool have_ws = ws && ws_bytes >= tsu::energy_ws_bytes(g->ny, g->ld);
  tsu::EnergyWs ews{};
  if (o.energy && !ws) return fail(TSU_ENOMEM, "energy needs a workspace (tsu_step_workspace)");
  if (ws && !have_ws)
    return fail(TSU_ENOMEM, "workspace %zu B < %zu B", ws_bytes, tsu::energy_ws_bytes(g->ny, g->ld));
  if (have_ws) {
    ews = tsu::energy_ws_carve(ws, ws_bytes, g->ny, g->ld);
    cudaError_t e = cudaMemsetAsync(ews.counter, 0, sizeof(unsigned int), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n workspace reset");
  }
  // kernel choice: the temporally blocked passes need FP32 fields, four state buffers and a
  // workspace (status word).  The warp-blocked pass records receivers itself and takes
  // checkpoints between its launches, so checkpoint steps must fall on launch boundaries
  // (ckpt_every a multiple of its depth, the call starting on a checkpoint's residue); the
  // CTA-blocked pass takes neither.
  const int wdepth = o.tdepth ? o.tdepth : 4;
  const bool blocked_base = dtype == TSU_F32 && st->nbuf == 4 && have_ws;
  const bool ckpt_aligned = !o.ckpt || (o.ckpt_every % wdepth == 0 && ((st->step - 1) % wdepth + wdepth) % wdepth == 0);
  // receivers: every warp of the blocked pass scans the whole list once per launch, so long lists
  // go one step per pass (whose first CTA gathers them)
  const bool wtb_possible = blocked_base && ckpt_aligned && (!o.traces || o.nrec <= tsu::kWtbMaxReceivers);
  const bool tb_possible = blocked_base && !o.traces && !o.ckpt;
  if (o.kernel == 2 && !wtb_possible)
    return fail(TSU_EINVAL, "kernel 2 needs FP32, nbuf = 4, a workspace and checkpoints on its launch boundaries");
  const bool flow_possible = blocked_base && st->form == TSU_FORM_INCREMENT && !o.traces && !o.ckpt &&
                             (o.tdepth == 0 || o.tdepth == 4);
  if (o.kernel == 4 && !flow_possible)
    return fail(TSU_EINVAL, "kernel 4 needs FP32 in the increment form, nbuf = 4, a workspace, depth 4 and no "
                            "traces or checkpoints");
  if (o.kernel == 3 && !tb_possible)
    return fail(TSU_EINVAL, "kernel 3 needs FP32, nbuf = 4, a workspace and no traces/checkpoints");
  // kernel 2: warp-blocked pass, tdepth steps per launch (default 4); also the automatic choice
  // (kernel 0) whenever it is possible: it beat one step per pass at every size measured (1024^2
  // to 16384^2).  All passes give the same bits, so the choice never changes a result.
  int wrows = o.rows ? (o.rows < 16 ? 16 : o.rows) : tsu::wtb_auto_rows(g->ny, g->ld, wdepth);
  const bool use_wtb = wtb_possible && nsteps >= wdepth && tsu::wtb_supported_depth(wdepth) &&
                       (o.kernel == 2 || o.kernel == 0 || o.kernel == 4);
  // kernel 3: CTA-blocked pass, on request only
  const int tdepth = o.tdepth ? o.tdepth : 8;
  int tb_rows = o.rows ? o.rows : 128;
  if (tb_rows < 16) tb_rows = 16;
  const bool use_tb = !use_wtb && tb_possible && nsteps >= tdepth && o.kernel == 3;
  const tsu::StencilGeom sg = geom(g, tau);
  const size_t field_bytes = (size_t)g->ny * g->ld * elem_size(dtype);
  cudaStream_t s = (cudaStream_t)stream;
  int64_t k = 0;
  if (use_wtb && o.traces) {
    cudaError_t e = tsu::launch_wtb_rec_table(sg, wrows, o.rec_idx, o.nrec, ews, s);
    if (e == cudaSuccess) e = tsu::launch_wtb_trace_edges(sg, o.rec_idx, o.nrec, o.traces, nsteps / wdepth * wdepth, s);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n receiver table");
  }
  if (use_wtb && flow_possible && (o.kernel == 4 || (o.kernel == 0 && tsu::wtb_flow_preferred(g->ny, g->ld)))) {
    // kernel 4, and the automatic choice for grids of 2K to 12K per side: every pass of the call
    // in one persistent launch (the same states; 2048^2 611 against 481 GLUPS, 4096^2 988 against
    // 826, 8192^2 1030-1052 against 963)
    const int64_t npass = nsteps / wdepth;
    const int f1 = scratch_index(st, -1), f2 = scratch_index(st, f1);
    void* const uu[2] = {st->buf[st->cur], st->buf[f1]};
    void* const vv[2] = {st->buf[st->aux], st->buf[f2]};
    const int frows = o.rows ? wrows : tsu::wtb_flow_rows(g->ny, g->ld);
    bool ran = false;
    cudaError_t e =
        tsu::launch_step_wtb_flow(sg, m->hx, m->hy, uu, vv, o.energy, ews, frows, npass, o.reserved, s, &ran);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n persistent warp-blocked launch");
    if (ran) {
      k = npass * wdepth;
      if (npass & 1) {
        st->cur = f1;
        st->aux = f2;
      }
      st->step += k;
    }
  }
  if (use_wtb) {
    for (; k + wdepth <= nsteps; k += wdepth) {
      const int64_t n = st->step;  // state holds u^n: checkpoint (u^{n-1}, u^n) or (u^n, v^n)
      if (o.ckpt && ((n - 1) % o.ckpt_every) == 0 && (n - 1) / o.ckpt_every < o.ckpt_slots) {
        char* slot = (char*)o.ckpt + (size_t)((n - 1) / o.ckpt_every) * 2 * field_bytes;
        const void* a0 = st->form == TSU_FORM_STANDARD ? st->buf[st->aux] : st->buf[st->cur];
        const void* a1 = st->form == TSU_FORM_STANDARD ? st->buf[st->cur] : st->buf[st->aux];
        cudaError_t e = cudaMemcpyAsync(slot, a0, field_bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(slot + field_bytes, a1, field_bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n checkpoint");
      }
      const int f1 = scratch_index(st, -1), f2 = scratch_index(st, f1);
      void* tr = o.traces ? (char*)o.traces + (size_t)k * o.nrec * elem_size(dtype) : nullptr;
      cudaError_t e = tsu::launch_step_wtb(sg, st->form, wdepth, m->hx, m->hy, st->buf[st->cur], st->buf[st->aux],
                                           st->buf[f1], st->buf[f2], o.energy ? o.energy + k : nullptr, ews, wrows, s,
                                           o.nrec, o.rec_idx, tr);
      if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n warp-blocked launch");
      st->cur = f1;
      st->aux = f2;
      st->step += wdepth;
    }
  }
  if (use_tb) {
    for (; k + tdepth <= nsteps; k += tdepth) {
      const int f1 = scratch_index(st, -1), f2 = scratch_index(st, f1);
      cudaError_t e = tsu::launch_step_tb(sg, st->form, tdepth, m->hx, m->hy, st->buf[st->cur], st->buf[st->aux],
                                          st->buf[f1], st->buf[f2], o.energy ? o.energy + k : nullptr, ews,
                                          ews.status, tb_rows, o.reserved, s);
      if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n temporally blocked launch");
      st->cur = f1;
      st->aux = f2;
      st->step += tdepth;
    }
  }
  for (; k < nsteps; ++k) {
    tsu::PassOut po{};
    po.energy = o.energy ? o.energy + k : nullptr;
    po.ews = ews;
    po.nrec = o.nrec;
    po.rec_idx = o.rec_idx;
    po.trace = o.traces ? (char*)o.traces + (size_t)k * o.nrec * elem_size(dtype) : nullptr;
    const int64_t n = st->step;  // state holds u^n
    if (o.ckpt && ((n - 1) % o.ckpt_every) == 0 && (n - 1) / o.ckpt_every < o.ckpt_slots) {
      char* slot = (char*)o.ckpt + (size_t)((n - 1) / o.ckpt_every) * 2 * field_bytes;
      po.ckpt_a = slot;
      po.ckpt_b = slot + field_bytes;
    }
    cudaError_t e;
    if (st->form == TSU_FORM_STANDARD) {
      e = tsu::launch_step(sg, dtype, st->form, m->hx, m->hy, st->buf[st->aux], st->buf[st->cur], nullptr,
                           st->buf[st->aux], po, true, (use_tb || use_wtb) ? 0 : o.rows, s);
    } else {
      const int f = scratch_index(st, -1);
      e = tsu::launch_step(sg, dtype, st->form, m->hx, m->hy, nullptr, st->buf[st->cur], st->buf[st->aux],
                           st->buf[f], po, true, (use_tb || use_wtb) ? 0 : o.rows, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n launch");
    if (st->form == TSU_FORM_STANDARD) {
      const int t = st->cur;
      st->cur = st->aux;
      st->aux = t;
    } else {
      st->cur = scratch_index(st, -1);
    }
    st->step += 1;
  }
  return TSU_OK;
}

// ---------------------------------------------------------------------------------------------
// Adjoint: workspace = 4 multiplier fields + 2 segment buffers of (E+1) recomputed states, the
// restore field (u^{m-1} or v^m) and a second v [+ 2 FP32 gradient accumulators for FP32 fields]
// + receiver tables
// ---------------------------------------------------------------------------------------------
static int64_t adjoint_ctas(const tsu_grid* g, int dtype) {
  int64_t gx, gy, cpc;
  int rows;
  tsu::adjoint_pass_shape(geom(g, 1.0), dtype, &gx, &gy, &rows, &cpc);
  return gx * gy;
}

// steps per pass of the FP32 segment recompute (warp-blocked, intermediate states stored)
constexpr int kRecomputeDepth = 4;
// steps per pass of the FP32 reverse sweep (2 or 4); leftover steps of a segment run one per pass
constexpr int kAdjointDepth = 4;

// fields of dtype before the FP32 accumulators: 4 multiplier fields, then two segment buffers of
// E + 3
static int64_t adjoint_fields(int form, int64_t every) {
  (void)form;
  return 4 + 2 * (every + 3);
}

// receiver tables: the one-step pass's (per CTA) and the K-step pass's (per tile, <= 4 per receiver)
static size_t adjoint_bucket_bytes(const tsu_grid* g, int dtype, int32_t nrec) {
  const size_t nr = nrec > 0 ? (size_t)nrec : 0;
  const size_t one = ((size_t)(adjoint_ctas(g, dtype) + 1) + 2 * nr) * sizeof(int);
  const int rowsk = tsu::adjoint_wtb_rows(kAdjointDepth, g->ny, g->ld);
  const size_t blk = ((size_t)tsu::adjoint_wtb_tiles(g->ny, g->ld, rowsk) + 1) * sizeof(int) + 16 + 4 * nr * 16;
  return (one + 15) / 16 * 16 + blk;
}

static size_t adjoint_ws_bytes(const tsu_grid* g, int dtype, int form, int64_t every, int32_t nrec) {
  const size_t fb = (size_t)g->ny * g->ld * elem_size(dtype);
  size_t b = (size_t)adjoint_fields(form, every) * fb;
  if (dtype == TSU_F32) b += 2 * (size_t)g->ny * g->ld * sizeof(float);
  const size_t buckets = adjoint_bucket_bytes(g, dtype, nrec);
  return b + (buckets + 255) / 256 * 256 + 256;
}

int tsu_adjoint_workspace(const tsu_grid* g, int dtype, int form, int64_t nsteps, int64_t ckpt_every, int32_t nrec,
                          size_t* bytes) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  if (!bytes) return fail(TSU_EINVAL, "bytes is NULL");
  if (form != TSU_FORM_STANDARD && form != TSU_FORM_INCREMENT) return fail(TSU_EINVAL, "bad form");
  if (nsteps < 1 || ckpt_every < 1 || nrec < 0) return fail(TSU_EINVAL, "nsteps, ckpt_every >= 1 and nrec >= 0");
  *bytes = adjoint_ws_bytes(g, dtype, form, ckpt_every, nrec);
  return TSU_OK;
}

}  // extern "C"

// One auxiliary (non-blocking) stream per device and host thread with its events, created on
// first use, for overlapping the adjoint's segment recompute with its reverse sweep.  Per thread,
// so that adjoints enqueued from several host threads never share the events that order them.
// The thread owns them: they are destroyed when the thread exits (work still in flight on the
// stream completes first; CUDA releases a busy stream once it is idle).
namespace {
std::atomic<int> g_aux_live{0};

struct AuxStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t start = nullptr, computed[2] = {nullptr, nullptr}, swept[2] = {nullptr, nullptr};
  AuxStream() = default;
  AuxStream(const AuxStream&) = delete;
  AuxStream& operator=(const AuxStream&) = delete;
  ~AuxStream() {  // also releases a partial creation; errors at process teardown are ignored
    int prev = -1;
    const bool switch_dev = cudaGetDevice(&prev) == cudaSuccess && dev >= 0 && prev != dev;
    if (switch_dev) cudaSetDevice(dev);
    cudaEvent_t* evs[5] = {&start, &computed[0], &computed[1], &swept[0], &swept[1]};
    for (cudaEvent_t* e : evs)
      if (*e) cudaEventDestroy(*e);
    if (s) {
      cudaStreamDestroy(s);
      g_aux_live.fetch_sub(1);
    }
    if (switch_dev) cudaSetDevice(prev);
  }
};

struct AuxSet {
  std::unique_ptr<AuxStream> dev[64];
};
thread_local AuxSet g_aux;

AuxStream* aux_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!g_aux.dev[dev]) {
    std::unique_ptr<AuxStream> a(new AuxStream());
    a->dev = dev;
    bool ok = cudaStreamCreateWithFlags(&a->s, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) g_aux_live.fetch_add(1);
    else a->s = nullptr;
    ok = ok && cudaEventCreateWithFlags(&a->start, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b) {
      ok = cudaEventCreateWithFlags(&a->computed[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&a->swept[b], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) return nullptr;  // the destructor releases what was created
    g_aux.dev[dev] = std::move(a);
  }
  return g_aux.dev[dev].get();
}
}  // namespace

extern "C" {

int tsu_aux_streams(void) { return g_aux_live.load(); }

int64_t tsu_ckpt_slots(int64_t nsteps, int64_t ckpt_every) {
  if (nsteps < 2 || ckpt_every < 1) return 0;
  return (nsteps - 2) / ckpt_every + 1;
}

int tsu_adjoint(const tsu_grid* g, int dtype, int form, double tau, const tsu_medium* m, int64_t nsteps,
                int64_t ckpt_every, const void* ckpt, const void* u0, int32_t nrec, const int64_t* rec_idx,
                const void* dtraces, double* g_hx, double* g_hy, void* g_u0, void* g_u1, void* ws, size_t ws_bytes,
                void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_cfl(g, tau, m));
  TRY(check_field(m->hx, "hx"));
  TRY(check_field(m->hy, "hy"));
  TRY(check_field(u0, "u0"));
  TRY(check_field(g_hx, "g_hx"));
  TRY(check_field(g_hy, "g_hy"));
  TRY(check_field(g_u0, "g_u0"));
  TRY(check_field(g_u1, "g_u1"));
  if (form != TSU_FORM_STANDARD && form != TSU_FORM_INCREMENT) return fail(TSU_EINVAL, "bad form");
  if (nsteps < 1 || ckpt_every < 1) return fail(TSU_EINVAL, "nsteps and ckpt_every must be >= 1");
  int64_t C = tsu_ckpt_slots(nsteps, ckpt_every);
  if (C > 0) TRY(check_field(ckpt, "ckpt"));
  if (nrec < 0 || (nrec > 0 && (!rec_idx || !dtraces))) return fail(TSU_EINVAL, "receivers need rec_idx and dtraces");
  const size_t need = adjoint_ws_bytes(g, dtype, form, ckpt_every, nrec);
  if (!ws || ws_bytes < need) return fail(TSU_ENOMEM, "adjoint workspace %zu B < %zu B", ws_bytes, need);
  TRY(check_field(ws, "workspace"));
  cudaStream_t s = (cudaStream_t)stream;
  const tsu::StencilGeom sg = geom(g, tau);
  const size_t es = elem_size(dtype);
  const size_t fb = (size_t)g->ny * g->ld * es;
  char* w = (char*)ws;
  // four multiplier fields.  FP64 (standard form): lam4[i1] = lam^{n+1}, lam4[i2] = lam^{n+2}.
  // FP32 (increment form): lam4[i1] = lam^{n+1}, lam4[i2] = mu^{n+1} = lam^{n+1} - lam^{n+2}.  The
  // other two receive the outputs of a K-step pass (which may not overwrite inputs that
  // neighbouring tiles' halos still read).
  char* lam4[4] = {w, w + fb, w + 2 * fb, w + 3 * fb};
  int i1 = 0, i2 = 1;
  const bool inc = dtype == TSU_F32;
  // two segment buffers, each seg[k] = u^{m_c + k} (k = 0..E) followed by the restore field
  // (u^{m_c - 1} or v) and a second v field (the blocked recompute writes v to the other one);
  // the recompute of one segment overlaps the reverse sweep of the other
  char* segbuf[2] = {w + 4 * fb, w + 4 * fb + (size_t)(ckpt_every + 3) * fb};
  char* g32 = w + (size_t)adjoint_fields(form, ckpt_every) * fb;  // FP32 accumulators [2][ny][ld]
  const size_t f32b = (size_t)g->ny * g->ld * sizeof(float);
  void* accx = dtype == TSU_F32 ? (void*)g32 : (void*)g_hx;
  void* accy = dtype == TSU_F32 ? (void*)(g32 + f32b) : (void*)g_hy;
  char* bk = (dtype == TSU_F32 ? g32 + 2 * f32b : g32);  // receiver buckets (ints)
  int* b_off = (int*)bk;
  int* b_ord = b_off + (adjoint_ctas(g, dtype) + 1);
  int* b_cta = b_ord + (nrec > 0 ? nrec : 0);
  // K-step pass (FP32): tile table of receivers
  const bool blocked = dtype == TSU_F32;
  const int rowsk = tsu::adjoint_wtb_rows(kAdjointDepth, g->ny, g->ld);
  char* bk2 = bk + ((((size_t)(adjoint_ctas(g, dtype) + 1) + 2 * (size_t)(nrec > 0 ? nrec : 0)) * sizeof(int) + 15) /
                    16 * 16);
  int* t_off = (int*)bk2;
  int4* t_ent = (int4*)(bk2 + (((size_t)tsu::adjoint_wtb_tiles(g->ny, g->ld, rowsk) + 1) * sizeof(int) + 15) / 16 * 16);
  auto segp = [&](int b, int64_t k) { return (void*)(segbuf[b] + (size_t)k * fb); };
  const int recompute_rows = tsu::wtb_seg_rows(g->ny, g->ld);
  auto extra = [&](int b, int q = 0) { return (void*)(segbuf[b] + (size_t)(ckpt_every + 1 + q) * fb); };
  AuxStream* aux = aux_stream();
  if (!aux) return fail(TSU_ECUDA, "tsu_adjoint: could not create the recompute stream");
  cudaError_t e = cudaMemsetAsync(ws, 0, need - 256, s);
  if (e == cudaSuccess && nrec > 0) e = tsu::launch_rec_bucket(sg, dtype, rec_idx, nrec, b_off, b_ord, b_cta, s);
  if (e == cudaSuccess && nrec > 0 && blocked)
    e = tsu::launch_rec_tiles(sg, kAdjointDepth, rec_idx, nrec, rowsk, t_off, t_ent, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g_hx, 0, (size_t)g->ny * g->ld * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g_hy, 0, (size_t)g->ny * g->ld * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint reset");
  auto free_pair = [&](int* oa, int* ob) {
    *oa = *ob = -1;
    for (int k = 0; k < 4; ++k)
      if (k != i1 && k != i2) (*oa < 0 ? *oa : *ob) = k;
  };
  // one step back.  FP64: lam^n written over lam^{n+2}.  FP32: mu^n in place, lam^n into a free field.
  auto step_back = [&](int64_t n, const void* un) -> cudaError_t {
    tsu::RecBuckets rb{};
    if (nrec > 0) rb = {b_off, b_ord, rec_idx, (const char*)dtraces + (size_t)(n - 1) * nrec * es};
    if (inc) {
      int oa, ob;
      free_pair(&oa, &ob);
      cudaError_t r = tsu::launch_adjoint_pass(sg, dtype, tsu::kAdjStepInc, m->hx, m->hy, lam4[i1], lam4[i2],
                                               lam4[oa], lam4[i2], un, accx, accy, nullptr, rb, s);
      i1 = oa;  // lam^n; mu^n stays in lam4[i2]
      return r;
    }
    cudaError_t r = tsu::launch_adjoint_pass(sg, dtype, tsu::kAdjStep, m->hx, m->hy, lam4[i1], lam4[i2], lam4[i2],
                                             nullptr, un, accx, accy, nullptr, rb, s);
    const int t = i1;  // now lam4[i1] = lam^n, lam4[i2] = lam^{n+1}
    i1 = i2;
    i2 = t;
    return r;
  };
  // kAdjointDepth steps back (n .. n-K+1) in one pass (FP32), u[f] = u^{n-f}: lam^{n-K+1} and
  // mu^{n-K+1} into the two free multiplier fields
  auto steps_back = [&](int64_t n, const void* const* u) -> cudaError_t {
    int oa, ob;
    free_pair(&oa, &ob);
    const void* gv[kAdjointDepth];
    for (int f = 0; f < kAdjointDepth; ++f)
      gv[f] = nrec > 0 ? (const char*)dtraces + (size_t)(n - 1 - f) * nrec * es : nullptr;
    cudaError_t r = tsu::launch_adjoint_wtb(sg, kAdjointDepth, rowsk, m->hx, m->hy, lam4[i1], lam4[i2], u, lam4[oa],
                                            lam4[ob], accx, accy, nrec > 0 ? t_off : nullptr, t_ent,
                                            nrec > 0 ? gv : nullptr, s);
    i1 = oa;  // lam^{n-K+1}
    i2 = ob;  // mu^{n-K+1}
    return r;
  };
  if (C == 0) {  // nsteps == 1: lam^1 = g^1 (the gradient term of n = 1 vanishes with lam^2 = 0)
    e = step_back(1, (void*)lam4[3]);  // a zero field no pass writes here: u is not used with lam^2 = 0
    if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint pass");
  }
  // the recompute stream starts after the resets above
  e = cudaEventRecord(aux->start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(aux->s, aux->start, 0);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint stream setup");
  for (int64_t c = C - 1, idx = 0; c >= 0; --c, ++idx) {
    const int b = (int)(idx & 1);
    const int64_t mc = 1 + c * ckpt_every;
    const int64_t mend = (mc + ckpt_every < nsteps) ? mc + ckpt_every : nsteps;
    // recompute stream: wait until the sweep that last read buffer b is done, restore the
    // checkpointed state, recompute u^{mc+1}..u^{mend} into seg[b][1..]
    if (idx >= 2) e = cudaStreamWaitEvent(aux->s, aux->swept[b], 0);
    const char* slot = (const char*)ckpt + (size_t)c * 2 * fb;
    if (e == cudaSuccess) {
      if (form == TSU_FORM_STANDARD) {
        e = cudaMemcpyAsync(extra(b), slot, fb, cudaMemcpyDeviceToDevice, aux->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(segp(b, 0), slot + fb, fb, cudaMemcpyDeviceToDevice, aux->s);
      } else {
        e = cudaMemcpyAsync(segp(b, 0), slot, fb, cudaMemcpyDeviceToDevice, aux->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(extra(b), slot + fb, fb, cudaMemcpyDeviceToDevice, aux->s);
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint restore");
    tsu::PassOut none{};
    int64_t k = 0;
    int vq = 0;  // increment form: v^{m_c + k} in extra(b, vq)
    if (dtype == TSU_F32) {  // kRecomputeDepth steps per pass, every intermediate state stored
      for (; k + kRecomputeDepth <= mend - mc; k += kRecomputeDepth) {
        const void* p = form == TSU_FORM_STANDARD ? (k == 0 ? extra(b) : segp(b, k - 1)) : extra(b, vq);
        e = tsu::launch_step_wtb_seg(sg, form, kRecomputeDepth, m->hx, m->hy, segp(b, k), p, segp(b, k + 1),
                                     (int64_t)(fb / es), form == TSU_FORM_STANDARD ? nullptr : extra(b, vq ^ 1),
                                     recompute_rows, aux->s);
        if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint recompute");
        vq ^= 1;
      }
    }
    for (; k < mend - mc; ++k) {
      if (form == TSU_FORM_STANDARD)
        e = tsu::launch_step(sg, dtype, form, m->hx, m->hy, k == 0 ? extra(b) : segp(b, k - 1), segp(b, k), nullptr,
                             segp(b, k + 1), none, true, 0, aux->s);
      else
        e = tsu::launch_step(sg, dtype, form, m->hx, m->hy, nullptr, segp(b, k), extra(b, vq), segp(b, k + 1), none,
                             true, 0, aux->s);
      if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint recompute");
    }
    e = cudaEventRecord(aux->computed[b], aux->s);
    // caller's stream: the reverse sweep over this segment once its states are there
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, aux->computed[b], 0);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint stream order");
    const int64_t nlo = (c == 0) ? 1 : mc + 1;
    for (int64_t n = mend; n >= nlo;) {
      if (blocked && n - (kAdjointDepth - 1) >= nlo) {
        const void* u[kAdjointDepth];
        for (int f = 0; f < kAdjointDepth; ++f) u[f] = segp(b, n - f - mc);
        e = steps_back(n, u);
        n -= kAdjointDepth;
      } else {
        e = step_back(n, segp(b, n - mc));
        n -= 1;
      }
      if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint pass");
    }
    if (dtype == TSU_F32) {
      e = tsu::launch_flush(sg, accx, accy, g_hx, g_hy, s);
      if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint flush");
    }
    e = cudaEventRecord(aux->swept[b], s);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint stream order");
  }
  // the start: dJ/du0 = (I + B/2) lam^1 - lam^2 (= mu^1 + B lam^1 / 2), dJ/du1 = tau lam^1, face
  // terms with u^0 and weight 1/2
  e = tsu::launch_adjoint_pass(sg, dtype, inc ? tsu::kAdjStartInc : tsu::kAdjStart, m->hx, m->hy, lam4[i1], lam4[i2],
                               g_u0, nullptr, u0, accx, accy, g_u1, tsu::RecBuckets{}, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g_u0, 0, (size_t)g->ld * es, s);  // boundary rows of the outputs
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)g_u0 + (size_t)(g->ny - 1) * g->ld * es, 0, (size_t)g->ld * es, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g_u1, 0, (size_t)g->ld * es, s);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)g_u1 + (size_t)(g->ny - 1) * g->ld * es, 0, (size_t)g->ld * es, s);
  if (e == cudaSuccess && dtype == TSU_F32) e = tsu::launch_flush(sg, accx, accy, g_hx, g_hy, s);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_adjoint start");
  return TSU_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched family
// ---------------------------------------------------------------------------------------------
// kernel 2 (warp-blocked, default, tdepth 2 or 4, default 4) or 3 (CTA-blocked, tdepth 4 or 8,
// default 8); descriptor size and strip width follow the kernel
static int batch_kernel(const tsu_batch_opts* opts) { return (opts && opts->kernel) ? opts->kernel : 2; }

// rows per chunk of problem i under these options (rows: the call's uniform choice)
static int batch_rows_of(const tsu_batch_opts* opts, int i, int rows) {
  return (opts && opts->rows_per_problem && opts->rows_per_problem[i] > 0) ? opts->rows_per_problem[i] : rows;
}

static int batch_layout(int32_t nprob, const tsu_problem* probs, const tsu_batch_opts* opts, int* k_out,
                        int* rows_out, int64_t* ntiles_out, size_t* bytes_out) {
  if (nprob < 1 || !probs) return fail(TSU_EINVAL, "need at least one problem");
  const int kern = batch_kernel(opts);
  if (kern != 2 && kern != 3) return fail(TSU_EINVAL, "batch kernel must be 2 or 3");
  const int k = (opts && opts->tdepth) ? opts->tdepth : (kern == 2 ? 4 : 8);
  if (kern == 3 && !tsu::tb_supported_depth(k)) return fail(TSU_EINVAL, "kernel 3: tdepth must be 4 or 8");
  if (kern == 2 && !tsu::wtb_supported_depth(k)) return fail(TSU_EINVAL, "kernel 2: tdepth must be 2 or 4");
  if (opts && (opts->order < 0 || opts->order > 2)) return fail(TSU_EINVAL, "order must be 0, 1 or 2");
  for (int i = 0; i < nprob; ++i) TRY(check_grid(&probs[i].grid));
  auto strips = [&](int64_t ld) {
    return kern == 2 ? tsu::wtb_strips(ld) : (ld + tsu::tb_strip_width(k) - 1) / tsu::tb_strip_width(k);
  };
  auto tiles_at = [&](int r) {
    int64_t t = 0;
    for (int i = 0; i < nprob; ++i) {
      const int ri = batch_rows_of(opts, i, r);
      t += strips(probs[i].grid.ld) * ((probs[i].grid.ny - 2 + ri - 1) / ri);
    }
    return t;
  };
  // rows per chunk: 80 (64-problem family of 512^2..2048^2, FP32 GLUPS of the flux-form pass at
  // 56/64/80/128 rows: 927/932/934/889), fewer (down to 16) while the family's tiles would not
  // fill one wave of the GPU (small problems)
  int rows = (opts && opts->rows) ? opts->rows : 80;
  if (!(opts && opts->rows) && kern == 2)
    while (rows > 16 && tiles_at(rows) < (int64_t)152 * 3 * 4) rows = rows > 32 ? rows / 2 : 16;
  for (int i = 0; i < nprob; ++i)
    if (batch_rows_of(opts, i, rows) < 16) return fail(TSU_EINVAL, "problem %d: rows must be >= 16", i);
  const size_t ab = kern == 2 ? tsu::wtb_args_bytes() : tsu::tb_args_bytes();
  const int64_t ntiles = tiles_at(rows);
  *k_out = k;
  *rows_out = rows;
  *ntiles_out = ntiles;
  *bytes_out = 256 + 3 * (size_t)nprob * ab + (size_t)ntiles * 16;
  return TSU_OK;
}

int tsu_batch_workspace(int32_t nprob, const tsu_problem* probs, const tsu_batch_opts* opts, size_t* bytes) {
  g_err[0] = 0;
  if (!bytes) return fail(TSU_EINVAL, "bytes is NULL");
  int k, rows;
  int64_t nt;
  return batch_layout(nprob, probs, opts, &k, &rows, &nt, bytes);
}

int tsu_batch_run(int32_t nprob, const tsu_problem* probs, const tsu_batch_opts* opts, void* ws, size_t ws_bytes,
                  void* stream) {
  g_err[0] = 0;
  int k, rows;
  int64_t ntiles;
  size_t need;
  TRY(batch_layout(nprob, probs, opts, &k, &rows, &ntiles, &need));
  if (!ws || ws_bytes < need) return fail(TSU_ENOMEM, "batch workspace %zu B < %zu B", ws_bytes, need);
  TRY(check_field(ws, "workspace"));
  const int form = probs[0].state ? probs[0].state->form : -1;
  for (int i = 0; i < nprob; ++i) {
    const tsu_problem& p = probs[i];
    TRY(check_cfl(&p.grid, p.tau, &p.medium));
    TRY(check_field(p.medium.hx, "hx"));
    TRY(check_field(p.medium.hy, "hy"));
    TRY(check_state(p.state, true));
    if (p.state->form != form) return fail(TSU_EINVAL, "problem %d: all problems need the same form", i);
    if (p.state->nbuf != 4) return fail(TSU_EINVAL, "problem %d: nbuf must be 4", i);
    if (p.nsteps < 0) return fail(TSU_EINVAL, "problem %d: nsteps < 0", i);
  }
  const int kern = batch_kernel(opts);
  const size_t ab = kern == 2 ? tsu::wtb_args_bytes() : tsu::tb_args_bytes();
  // problems in decreasing order of blocked rounds: round r launches a prefix of the tile table,
  // the tiles of the problems that still have a round to go.  Problems with equal round counts
  // form a group whose tiles are packed in the order the options ask for.
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return probs[a].nsteps / k > probs[b].nsteps / k; });
  const int pack = opts ? opts->order : 0;
  std::vector<int32_t> tiles;  // int4 per tile
  std::vector<int64_t> prefix(nprob);  // tiles up to the end of the group of order[i]
  tiles.reserve((size_t)ntiles * 4);
  auto put = [&](int i, int c, int st) {
    tiles.push_back(i);
    tiles.push_back(st);
    tiles.push_back(c);
    tiles.push_back(0);
  };
  auto strips_of = [&](int i) {
    const int64_t ld = probs[i].grid.ld;
    return (int)(kern == 2 ? tsu::wtb_strips(ld) : (ld + tsu::tb_strip_width(k) - 1) / tsu::tb_strip_width(k));
  };
  auto chunks_of = [&](int i) {
    const int ri = batch_rows_of(opts, i, rows);
    return (int)((probs[i].grid.ny - 2 + ri - 1) / ri);
  };
  for (int g0 = 0; g0 < nprob;) {
    int g1 = g0;
    while (g1 < nprob && probs[order[g1]].nsteps / k == probs[order[g0]].nsteps / k) ++g1;
    if (pack == 2) {  // chunk c of every problem of the group, then c + 1 ...
      int cmax = 0;
      for (int oi = g0; oi < g1; ++oi) cmax = std::max(cmax, chunks_of(order[oi]));
      for (int c = 0; c < cmax; ++c)
        for (int oi = g0; oi < g1; ++oi)
          if (c < chunks_of(order[oi]))
            for (int st = 0; st < strips_of(order[oi]); ++st) put(order[oi], c, st);
    } else {
      for (int pass = 0; pass < (pack == 1 ? 2 : 1); ++pass)
        for (int oi = g0; oi < g1; ++oi) {
          const int i = order[oi], nc = chunks_of(i), ri = batch_rows_of(opts, i, rows);
          const bool ragged = (probs[i].grid.ny - 2) % ri != 0;
          for (int c = 0; c < nc; ++c) {
            // order 1: full chunks in the first pass, a ragged last chunk in the second
            if (pack == 1 && (pass == 1) != (ragged && c == nc - 1)) continue;
            for (int st = 0; st < strips_of(i); ++st) put(i, c, st);
          }
        }
    }
    for (int oi = g0; oi < g1; ++oi) prefix[oi] = (int64_t)tiles.size() / 4;
    g0 = g1;
  }
  if ((int64_t)tiles.size() / 4 != ntiles) return fail(TSU_EINVAL, "tile table size mismatch");
  // descriptor sets: launch 0, then the two role assignments that alternate from launch 1 on
  std::vector<unsigned char> host(3 * (size_t)nprob * ab, 0);
  std::vector<tsu_state> sim(nprob);
  char* base = (char*)ws;
  int* status = (int*)(base + 4);
  for (int i = 0; i < nprob; ++i) sim[i] = *probs[i].state;
  for (int set = 0; set < 3; ++set) {
    for (int i = 0; i < nprob; ++i) {
      tsu_state& st = sim[i];
      const int f1 = scratch_index(&st, -1), f2 = scratch_index(&st, f1);
      void* dst = &host[((size_t)set * nprob + i) * ab];
      const int ri = batch_rows_of(opts, i, rows);
      if (kern == 2)
        tsu::wtb_fill_args(dst, geom(&probs[i].grid, probs[i].tau), probs[i].medium.hx, probs[i].medium.hy,
                           st.buf[st.cur], st.buf[st.aux], st.buf[f1], st.buf[f2], ri);
      else
        tsu::tb_fill_args(dst, geom(&probs[i].grid, probs[i].tau), probs[i].medium.hx, probs[i].medium.hy,
                          st.buf[st.cur], st.buf[st.aux], st.buf[f1], st.buf[f2], status, ri);
      st.cur = f1;
      st.aux = f2;
    }
  }
  for (int i = 0; i < nprob; ++i) {  // the inputs of launch 3 must be those of launch 1
    tsu_state t = *probs[i].state;
    int cur1 = -1, aux1 = -1;
    for (int q = 1; q <= 3; ++q) {
      const int f1 = scratch_index(&t, -1), f2 = scratch_index(&t, f1);
      t.cur = f1;
      t.aux = f2;
      if (q == 1) {
        cur1 = t.cur;
        aux1 = t.aux;
      }
    }
    if (t.cur != cur1 || t.aux != aux1) return fail(TSU_EINVAL, "problem %d: unexpected buffer roles", i);
  }
  cudaStream_t s = (cudaStream_t)stream;
  char* desc = base + 256;
  char* tdev = desc + 3 * (size_t)nprob * ab;
  cudaError_t e = cudaMemcpyAsync(desc, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tdev, tiles.data(), tiles.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffers go out of scope
  if (e != cudaSuccess) return cuda_fail(e, "tsu_batch_run upload");
  // every launch of the run: the blocked rounds, then the leftover single steps per problem
  auto enqueue = [&]() -> int {
    const int64_t rounds_max = probs[order[0]].nsteps / k;
    for (int64_t r = 0; r < rounds_max; ++r) {
      // tiles of the problems that still have a full round
      int64_t nt = 0;
      for (int oi = 0; oi < nprob; ++oi)
        if (probs[order[oi]].nsteps / k > r) nt = prefix[oi];
      const int set = r == 0 ? 0 : ((r & 1) ? 1 : 2);
      cudaError_t le = kern == 2
                           ? tsu::launch_step_wtb_batched(form, k, desc + (size_t)set * nprob * ab, ab, tdev, nt, s)
                           : tsu::launch_step_tb_batched(form, k, desc + (size_t)set * nprob * ab, tdev, nt, s);
      if (le != cudaSuccess) return cuda_fail(le, "tsu_batch_run launch");
    }
    for (int i = 0; i < nprob; ++i) {
      tsu_state* st = probs[i].state;
      const int64_t rounds = probs[i].nsteps / k;
      for (int64_t r = 0; r < rounds; ++r) {
        const int f1 = scratch_index(st, -1), f2 = scratch_index(st, f1);
        st->cur = f1;
        st->aux = f2;
      }
      st->step += rounds * k;
      const int64_t left = probs[i].nsteps - rounds * k;
      if (left > 0) {
        tsu_step_opts o;
        memset(&o, 0, sizeof o);
        o.kernel = 1;
        const int rc = tsu_step_n(&probs[i].grid, TSU_F32, probs[i].tau, &probs[i].medium, st, left, &o, nullptr, 0,
                                  stream);
        if (rc != TSU_OK) return rc;
      }
    }
    return TSU_OK;
  };
  if (!(opts && opts->graph)) return enqueue();
  // the same launches captured into one CUDA graph and launched once (the executable graph is
  // released right away; CUDA frees it when the launch completes)
  if (!s) return fail(TSU_EINVAL, "graph launch needs a non-default stream");
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_batch_run capture");
  const int rc = enqueue();
  cudaGraph_t gr = nullptr;
  e = cudaStreamEndCapture(s, &gr);
  if (rc != TSU_OK) {
    if (gr) cudaGraphDestroy(gr);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "tsu_batch_run capture");
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_batch_run graph instantiate");
  e = cudaGraphLaunch(ge, s);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_batch_run graph launch");
  return TSU_OK;
}

int tsu_sync_status(void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!ws || ws_bytes < 256) return fail(TSU_EINVAL, "workspace missing");
  int h = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, (char*)ws + 4, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)ws + 4, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_sync_status");
  if (h != TSU_OK) return fail(h, "device reported status %d (a bounded wait expired)", h);
  return TSU_OK;
}

int tsu_observe(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, const tsu_state* st,
                double* energy_dev, int32_t nrec, const int64_t* rec_idx, void* trace, void* ws, size_t ws_bytes,
                void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_cfl(g, tau, m));
  TRY(check_field(m->hx, "hx"));
  TRY(check_field(m->hy, "hy"));
  TRY(check_state(st, true));
  if (trace && (nrec <= 0 || !rec_idx)) return fail(TSU_EINVAL, "trace needs nrec > 0 and rec_idx");
  tsu::PassOut po{};
  if (energy_dev) {
    if (!ws || ws_bytes < tsu::energy_ws_bytes(g->ny, g->ld))
      return fail(TSU_ENOMEM, "energy needs a workspace of %zu B", tsu::energy_ws_bytes(g->ny, g->ld));
    po.ews = tsu::energy_ws_carve(ws, ws_bytes, g->ny, g->ld);
    po.energy = energy_dev;
    cudaError_t e = cudaMemsetAsync(po.ews.counter, 0, sizeof(unsigned int), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_observe workspace reset");
  }
  po.nrec = nrec;
  po.rec_idx = rec_idx;
  po.trace = trace;
  if (!energy_dev && !trace) return TSU_OK;
  cudaError_t e = st->form == TSU_FORM_STANDARD
                      ? tsu::launch_step(geom(g, tau), dtype, st->form, m->hx, m->hy, st->buf[st->aux],
                                         st->buf[st->cur], nullptr, nullptr, po, false, 0, (cudaStream_t)stream)
                      : tsu::launch_step(geom(g, tau), dtype, st->form, m->hx, m->hy, nullptr, st->buf[st->cur],
                                         st->buf[st->aux], nullptr, po, false, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_observe launch");
  return TSU_OK;
}

// ---- implicit comparator (Sec. 3.3) -------------------------------------------------------------

static tsu::ImplicitGeom implicit_geom(const tsu_grid* g, double tau, double sigma) {
  tsu::ImplicitGeom ig;
  ig.nx = g->nx;
  ig.ny = g->ny;
  ig.ld = g->ld;
  ig.ldT = tsu::implicit_ldT(g->ny);
  ig.cx = tau * tau / (g->dx * g->dx);
  ig.cy = tau * tau / (g->dy * g->dy);
  ig.tau = tau;
  ig.sigma = sigma;
  return ig;
}

// sigma >= 1/4: stable for every tau; below, the explicit bound scaled by (1 - 4 sigma)
static int check_implicit(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m) {
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  if (!m) return fail(TSU_EINVAL, "medium is NULL");
  TRY(check_field(m->hx, "hx"));
  TRY(check_field(m->hy, "hy"));
  if (!(tau > 0.0) || !isfinite(tau)) return fail(TSU_EINVAL, "tau must be positive and finite");
  if (!(sigma >= 0.0) || !isfinite(sigma)) return fail(TSU_EINVAL, "sigma must be >= 0 and finite");
  TRY(tsu::check_positive(m, g_err, sizeof g_err));
  if (sigma < 0.25) {
    const double q = tau * tau * (m->hx_max / (g->dx * g->dx) + m->hy_max / (g->dy * g->dy));
    if (q * (1.0 - 4.0 * sigma) > 1.0)
      return fail(TSU_ECFL, "sigma = %.6g < 1/4 and tau^2 (hx_max/dx^2 + hy_max/dy^2) (1 - 4 sigma) = %.6g > 1",
                  sigma, q * (1.0 - 4.0 * sigma));
  }
  return TSU_OK;
}

static int check_implicit_state(const tsu_state* st, bool need_roles) {
  if (!st) return fail(TSU_EINVAL, "state is NULL");
  if (st->form != TSU_FORM_INCREMENT) return fail(TSU_EINVAL, "the implicit scheme runs in the increment form");
  if (st->nbuf < 2 || st->nbuf > 4) return fail(TSU_EINVAL, "state needs 2..4 buffers (nbuf = %d)", st->nbuf);
  for (int b = 0; b < st->nbuf; ++b)
    if (!st->buf[b] || !aligned16(st->buf[b])) return fail(TSU_EINVAL, "state buf[%d] NULL or misaligned", b);
  if (need_roles && (st->cur < 0 || st->cur >= st->nbuf || st->aux < 0 || st->aux >= st->nbuf || st->cur == st->aux))
    return fail(TSU_EINVAL, "state cur/aux invalid (%d, %d)", st->cur, st->aux);
  return TSU_OK;
}

int tsu_implicit_sizes(const tsu_grid* g, int dtype, size_t* factor_bytes, size_t* ws_bytes) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  if (!factor_bytes || !ws_bytes) return fail(TSU_EINVAL, "output pointer is NULL");
  *factor_bytes = tsu::implicit_factor_elems(*g) * elem_size(dtype);
  *ws_bytes = tsu::implicit_ws_bytes(*g, elem_size(dtype));
  return TSU_OK;
}

int tsu_implicit_factor(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m, void* factor,
                        size_t factor_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_implicit(g, dtype, tau, sigma, m));
  TRY(check_field(factor, "factor"));
  const size_t need = tsu::implicit_factor_elems(*g) * elem_size(dtype);
  if (factor_bytes < need) return fail(TSU_ENOMEM, "factor needs %zu B (got %zu)", need, factor_bytes);
  cudaError_t e = tsu::launch_implicit_factor(implicit_geom(g, tau, sigma), dtype, m->hx, m->hy, factor,
                                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_implicit_factor launch");
  return TSU_OK;
}

int tsu_implicit_init(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m, const void* factor,
                      const void* u0, const void* u1, tsu_state* st, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_implicit(g, dtype, tau, sigma, m));
  TRY(check_field(factor, "factor"));
  TRY(check_field(u0, "u0"));
  if (u1) TRY(check_field(u1, "u1"));
  TRY(check_implicit_state(st, false));
  TRY(check_field(ws, "workspace"));
  const size_t need = tsu::implicit_ws_bytes(*g, elem_size(dtype));
  if (ws_bytes < need) return fail(TSU_ENOMEM, "workspace needs %zu B (got %zu)", need, ws_bytes);
  const tsu::ImplicitGeom ig = implicit_geom(g, tau, sigma);
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e =
      tsu::launch_implicit(ig, dtype, m->hx, m->hy, factor, u0, st->buf[0], st->buf[1], u1, 1, true, ws, s);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_implicit_init launch");
  st->cur = 0;
  st->aux = 1;
  st->step = 1;
  return TSU_OK;
}

int tsu_implicit_step_n(const tsu_grid* g, int dtype, double tau, double sigma, const tsu_medium* m,
                        const void* factor, tsu_state* st, int64_t nsteps, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  TRY(check_implicit(g, dtype, tau, sigma, m));
  TRY(check_field(factor, "factor"));
  TRY(check_implicit_state(st, true));
  if (nsteps < 0) return fail(TSU_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return TSU_OK;
  TRY(check_field(ws, "workspace"));
  const size_t need = tsu::implicit_ws_bytes(*g, elem_size(dtype));
  if (ws_bytes < need) return fail(TSU_ENOMEM, "workspace needs %zu B (got %zu)", need, ws_bytes);
  cudaError_t e = tsu::launch_implicit(implicit_geom(g, tau, sigma), dtype, m->hx, m->hy, factor, nullptr,
                                       st->buf[st->cur], st->buf[st->aux], nullptr, nsteps, false, ws,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tsu_implicit_step_n launch");
  st->step += nsteps;
  return TSU_OK;
}

}  // extern "C"
