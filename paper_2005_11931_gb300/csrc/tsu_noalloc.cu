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

}  // namespace

extern "C" {

// Message of the last failure of tsu_step_n_noalloc on the calling thread.
const char* tsu_noalloc_last_error(void) { return g_noalloc_err; }

int tsu_step_n_noalloc(const tsu_grid* g, int dtype, double tau, const tsu_medium* m, tsu_state* st,
                       int64_t nsteps, double* energy, void* stream) {
  g_noalloc_err[0] = 0;
  char* err = g_noalloc_err;
  const size_t n = sizeof g_noalloc_err;
  // the same checks as tsu_step_n, in the same order, so that both refuse the same inputs
  int rc = tsu::check_grid(g, err, n);
  if (rc == TSU_OK) rc = tsu::check_dtype(dtype, err, n);
  if (rc == TSU_OK) rc = tsu::check_medium(g, tau, m, err, n);
  if (rc == TSU_OK) rc = tsu::check_field(m->hx, "hx", err, n);
  if (rc == TSU_OK) rc = tsu::check_field(m->hy, "hy", err, n);
  if (rc == TSU_OK) rc = tsu::check_state(st, true, err, n);
  if (rc != TSU_OK) return rc;
  if (nsteps < 0) return na_fail(TSU_EINVAL, "nsteps must be >= 0");
  if (energy && (((uintptr_t)energy) & 7u)) return na_fail(TSU_EINVAL, "energy must be a device double array");
  // one partial per CTA of the one-step pass; refuse grids the fixed array cannot hold
  if (energy && tsu::one_step_ctas(g->ld, g->ny, dtype, kNoallocRows) > kNoallocPartials)
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
