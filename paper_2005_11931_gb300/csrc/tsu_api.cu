// C ABI of libtsu: argument validation, error reporting and launch sequencing.  All compute is
// in the kernels of k_*.cu; this file only checks arguments and enqueues work on the caller's
// stream.  See include/tsu.h for the contract of every entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

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

int check_grid(const tsu_grid* g) {
  if (!g) return fail(TSU_EINVAL, "grid is NULL");
  if (g->nx < 3 || g->ny < 3) return fail(TSU_EINVAL, "grid needs nx, ny >= 3 (got %d x %d)", g->nx, g->ny);
  if (g->ld < g->nx || (g->ld % 4) != 0)
    return fail(TSU_EINVAL, "ld must be >= nx and a multiple of 4 (ld=%lld nx=%d)", (long long)g->ld, g->nx);
  if (!(g->dx > 0.0) || !(g->dy > 0.0)) return fail(TSU_EINVAL, "dx, dy must be positive");
  if ((int64_t)g->ny * g->ld >= ((int64_t)1 << 40)) return fail(TSU_EINVAL, "grid too large");
  return TSU_OK;
}

int check_dtype(int dtype) {
  if (dtype != TSU_F32 && dtype != TSU_F64) return fail(TSU_EINVAL, "dtype must be TSU_F32 or TSU_F64");
  return TSU_OK;
}

int check_field(const void* p, const char* name) {
  if (!p) return fail(TSU_EINVAL, "%s is NULL", name);
  if (!aligned16(p)) return fail(TSU_EINVAL, "%s is not 16-byte aligned", name);
  return TSU_OK;
}

int check_cfl(const tsu_grid* g, double tau, const tsu_medium* m) {
  if (!m) return fail(TSU_EINVAL, "medium is NULL");
  if (!(tau > 0.0) || !isfinite(tau)) return fail(TSU_EINVAL, "tau must be positive and finite");
  if (!(m->hx_max >= 0.0) || !(m->hy_max >= 0.0)) return fail(TSU_EINVAL, "medium maxima must be >= 0");
  const double q = tau * tau * (m->hx_max / (g->dx * g->dx) + m->hy_max / (g->dy * g->dy));
  if (q > 1.0)
    return fail(TSU_ECFL, "tau^2 (hx_max/dx^2 + hy_max/dy^2) = %.6g > 1: leapfrog unstable", q);
  return TSU_OK;
}

int check_state(const tsu_state* st, bool need_roles) {
  if (!st) return fail(TSU_EINVAL, "state is NULL");
  if (st->form != TSU_FORM_STANDARD && st->form != TSU_FORM_INCREMENT) return fail(TSU_EINVAL, "bad form");
  const int need = st->form == TSU_FORM_STANDARD ? 2 : 3;
  if (st->nbuf < need || st->nbuf > 4)
    return fail(TSU_EINVAL, "state needs %d..4 buffers for this form (nbuf = %d)", need, st->nbuf);
  for (int b = 0; b < st->nbuf; ++b) {
    if (!st->buf[b] || ((uintptr_t)st->buf[b] & 15u)) return fail(TSU_EINVAL, "state buf[%d] NULL or misaligned", b);
  }
  if (need_roles) {
    if (st->cur < 0 || st->cur >= st->nbuf || st->aux < 0 || st->aux >= st->nbuf || st->cur == st->aux)
      return fail(TSU_EINVAL, "state cur/aux invalid (%d, %d)", st->cur, st->aux);
  }
  return TSU_OK;
}

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

extern "C" {

int tsu_version(void) { return 100; }

const char* tsu_last_error(void) { return g_err; }

double tsu_tau_for(const tsu_grid* g, double hx_max, double hy_max, double cfl) {
  if (!g || !(g->dx > 0) || !(g->dy > 0) || !(cfl > 0) || cfl > 1 || !(hx_max >= 0) || !(hy_max >= 0)) return 0.0;
  const double s = hx_max / (g->dx * g->dx) + hy_max / (g->dy * g->dy);
  if (!(s > 0)) return 0.0;
  return cfl / sqrt(s);
}

int tsu_make_depth(const tsu_grid* g, const tsu_depth* d, int dtype, void* hx, void* hy, double* ext_dev,
                   double* ext_host, void* stream) {
  g_err[0] = 0;
  TRY(check_grid(g));
  TRY(check_dtype(dtype));
  TRY(check_field(hx, "hx"));
  TRY(check_field(hy, "hy"));
  if (!ext_dev || ((uintptr_t)ext_dev & 7u)) return fail(TSU_EINVAL, "ext_dev must be a device double[4]");
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
  if (o.kernel < 0 || o.kernel > 3) return fail(TSU_EINVAL, "kernel must be 0..3");
  if (o.rows < 0) return fail(TSU_EINVAL, "rows must be >= 0");
  tsu::EnergyWs ews{};
  if (o.energy) {
    if (!ws) return fail(TSU_ENOMEM, "energy needs a workspace (tsu_step_workspace)");
    if (ws_bytes < tsu::energy_ws_bytes(g->ny, g->ld))
      return fail(TSU_ENOMEM, "workspace %zu B < %zu B", ws_bytes, tsu::energy_ws_bytes(g->ny, g->ld));
    ews = tsu::energy_ws_carve(ws, ws_bytes, g->ny, g->ld);
    cudaError_t e = cudaMemsetAsync(ews.counter, 0, sizeof(unsigned int), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tsu_step_n workspace reset");
  }
  const tsu::StencilGeom sg = geom(g, tau);
  const size_t field_bytes = (size_t)g->ny * g->ld * elem_size(dtype);
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t k = 0; k < nsteps; ++k) {
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
                           st->buf[st->aux], po, true, o.rows, s);
    } else {
      const int f = scratch_index(st, -1);
      e = tsu::launch_step(sg, dtype, st->form, m->hx, m->hy, nullptr, st->buf[st->cur], st->buf[st->aux],
                           st->buf[f], po, true, o.rows, s);
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

}  // extern "C"
