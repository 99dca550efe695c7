// tsu_step_n_noalloc: leapfrog steps with the per-step energy, for callers that must not allocate
// device memory.
//
// tsu_step_n takes its energy-reduction scratch (a ticket counter and one FP64 partial sum per
// CTA) from a workspace the caller allocates.  Some callers cannot do that: code that runs while
// another component owns the device allocator (a host application that hands this library only
// its input and output buffers), real-time loops where an allocation could stall, and plugins
// whose host forbids allocation from inside their callbacks.  This entry point takes the scratch
// from a fixed array in the library's own device memory instead, so the caller passes only the
// state, the medium and the energy output.
//
// The array below lives for as long as the library is loaded, on every GPU that uses it.  Its
// device address is looked up once per device (cudaGetSymbolAddress, with that device current)
// by the first call made on the device.  That first call should therefore happen before any
// stream capture begins.  Every call on a device shares the one array and leaves its last
// contents behind; each call zeroes the counter it needs before its first launch.  Calls whose
// work overlaps on the GPU (different streams, no ordering between them) race on the array and
// give wrong energies: order such calls on one stream or with events.
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "tsu_internal.h"

namespace {

// At most this many CTAs of the one-step pass (one FP64 partial each): with 128 threads x one
// 16-byte vector per thread and 32 rows per CTA this covers every grid with
// ceil(ld / 512) * ceil((ny - 2) / 32) <= 65536 in FP32 (e.g. 16384^2) and half of that in FP64.
constexpr int64_t kNoallocPartials = 65536;
constexpr size_t kNoallocBytes = 256 + (size_t)kNoallocPartials * sizeof(double);  // 512 KiB + 256 B
constexpr int kNoallocRows = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

thread_local char g_noalloc_err[256] = "";

int na_fail(int code, const char* msg) {
  snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
  return code;
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

bool al16(const void* p) { return p && (((uintptr_t)p) & 15u) == 0; }

}  // namespace

extern "C" {

// Message of the last failure of tsu_step_n_noalloc on the calling thread.
const char* tsu_noalloc_last_error(void) { return g_noalloc_err; }

int tsu_step_n_noalloc(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, tsu_state* st,
                       int64_t nsteps, double* energy, void* stream) {
  g_noalloc_err[0] = 0;
  if (!g || !m || !st) return na_fail(TSU_EINVAL, "grid, medium or state is NULL");
  if (g->nx < 3 || g->ny < 3 || g->ld < g->nx || (g->ld % 4) != 0 || !(g->dx > 0) || !(g->dy > 0))
    return na_fail(TSU_EINVAL, "bad grid (nx, ny >= 3, ld >= nx, ld % 4 == 0, dx, dy > 0)");
  if (dtype != TSU_F32 && dtype != TSU_F64) return na_fail(TSU_EINVAL, "dtype must be TSU_F32 or TSU_F64");
  if (nsteps < 0) return na_fail(TSU_EINVAL, "nsteps must be >= 0");
  if (!(tau > 0.0) || !(m->hx_max >= 0.0) || !(m->hy_max >= 0.0))
    return na_fail(TSU_EINVAL, "tau must be positive and the medium maxima >= 0");
  if (tau * tau * (m->hx_max / (g->dx * g->dx) + m->hy_max / (g->dy * g->dy)) > 1.0)
    return na_fail(TSU_ECFL, "tau^2 (hx_max/dx^2 + hy_max/dy^2) > 1: leapfrog unstable");
  if (!al16(m->hx) || !al16(m->hy)) return na_fail(TSU_EINVAL, "hx, hy NULL or not 16-byte aligned");
  const int need = st->form == TSU_FORM_STANDARD ? 2 : (st->form == TSU_FORM_INCREMENT ? 3 : 99);
  if (st->nbuf < need || st->nbuf > 4) return na_fail(TSU_EINVAL, "bad form or too few state buffers");
  for (int b = 0; b < st->nbuf; ++b)
    if (!al16(st->buf[b])) return na_fail(TSU_EINVAL, "state buffer NULL or not 16-byte aligned");
  if (st->cur < 0 || st->cur >= st->nbuf || st->aux < 0 || st->aux >= st->nbuf || st->cur == st->aux)
    return na_fail(TSU_EINVAL, "state cur/aux invalid");
  // one partial per CTA of the one-step pass; refuse grids the fixed array cannot hold
  const int64_t cols = (int64_t)128 * (dtype == TSU_F32 ? 4 : 2);
  const int64_t ctas = ((g->ld + cols - 1) / cols) * ((g->ny - 2 + kNoallocRows - 1) / kNoallocRows);
  if (energy && ctas > kNoallocPartials)
    return na_fail(TSU_ENOMEM, "grid too large for the fixed scratch of tsu_step_n_noalloc "
                               "(more than 65536 energy partial sums); use tsu_step_n with a workspace");
  if (nsteps == 0) return TSU_OK;
  cudaStream_t s = (cudaStream_t)stream;
  tsu::EnergyWs ews{};
  if (energy) {
    void* base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return na_fail(TSU_ECUDA, cudaGetErrorString(e));
    ews.counter = (unsigned int*)base;
    ews.status = (int*)((char*)base + 4);
    ews.partials = (double*)((char*)base + 256);
    ews.capacity = kNoallocPartials;
    e = cudaMemsetAsync(base, 0, 256, s);  // the ticket counter must start at zero
    if (e != cudaSuccess) return na_fail(TSU_ECUDA, cudaGetErrorString(e));
  }
  tsu::StencilGeom sg;
  sg.nx = g->nx;
  sg.ny = g->ny;
  sg.ld = g->ld;
  sg.cx = tau * tau / (g->dx * g->dx);
  sg.cy = tau * tau / (g->dy * g->dy);
  sg.tau = tau;
  sg.dxdy = g->dx * g->dy;
  for (int64_t k = 0; k < nsteps; ++k) {
    tsu::PassOut po{};
    po.energy = energy ? energy + k : nullptr;
    po.ews = ews;
    cudaError_t e;
    if (st->form == TSU_FORM_STANDARD) {
      e = tsu::launch_step(sg, dtype, st->form, m->hx, m->hy, st->buf[st->aux], st->buf[st->cur], nullptr,
                           st->buf[st->aux], po, true, kNoallocRows, s);
    } else {
      int f = -1;
      for (int b = 0; b < st->nbuf && f < 0; ++b)
        if (b != st->cur && b != st->aux) f = b;
      e = tsu::launch_step(sg, dtype, st->form, m->hx, m->hy, nullptr, st->buf[st->cur], st->buf[st->aux],
                           st->buf[f], po, true, kNoallocRows, s);
      if (e == cudaSuccess) st->cur = f;
    }
    if (e != cudaSuccess) return na_fail(TSU_ECUDA, cudaGetErrorString(e));
    if (st->form == TSU_FORM_STANDARD) {
      const int t = st->cur;
      st->cur = st->aux;
      st->aux = t;
    }
    st->step += 1;
  }
  return TSU_OK;
}

}  // extern "C"
