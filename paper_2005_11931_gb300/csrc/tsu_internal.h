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

// Workspace for the energy reduction: a ticket counter then per-CTA FP64 partials.
struct EnergyWs {
  unsigned int* counter;
  double* partials;
  int64_t capacity;  // number of partial slots
};

size_t energy_ws_bytes(int64_t ny, int64_t ld);
EnergyWs energy_ws_carve(void* ws, size_t bytes, int64_t ny, int64_t ld);

// Host-side mollifier normalisers, computed once by double-exponential quadrature.
double friedrichs_c1();
double friedrichs_c2();

cudaError_t launch_make_depth(const tsu_grid& g, const DepthParams& p, int dtype, void* hx, void* hy,
                              double* ext_dev, cudaStream_t s);

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

// One leapfrog pass (standard or increment form) over the interior; store=false computes only
// the side outputs (energy of the current pair, traces).
cudaError_t launch_step(const StencilGeom& g, int dtype, int form, const void* hx, const void* hy,
                        const void* u_prev, const void* u_cur, void* v, void* u_next, const PassOut& o,
                        bool store, int rows, cudaStream_t s);

}  // namespace tsu
