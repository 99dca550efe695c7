// Leapfrog stepping of the regularised 2D tsunami equation (arXiv:2005.11931, Sec. 2 eq. (2.1),
// Sec. 3.3 box and grid), register-streaming kernel:
//
//   u^{n+1} = 2u^n - u^{n-1} + B u^n,   B u = cx fx(u) + cy fy(u)
//   fx(u)_ij = hx_ij (u_i+1 - u_i) - hx_i-1,j (u_i - u_i-1),  fy likewise in j.
//
// Each thread owns V consecutive columns (one 16-byte vector) and marches down a block of rows
// keeping u^n of rows j-1, j, j+1 and hy of row j-1 in registers, so every field element comes
// from HBM once per step (20 B per lattice update in FP32).  x-neighbours come from the adjacent
// lanes by warp shuffles; the two lanes at a warp edge read the one neighbour column directly.
// The same pass optionally yields the discrete energy of the pair it reads (the leapfrog analogue
// of (CL-01), Theorem 2.1), receiver samples and a checkpoint copy.
//
// FP64 fields are evaluated with explicitly rounded operations in the order of the definition
// (no fused multiply-add), FP32 fields with fused multiply-adds.
#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

// Energy accumulator of one thread: compensated in the field type, FP64 across threads.
template <typename T>
struct EAcc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Deterministic CTA reduction of one double, then a last-CTA-done reduction of all partials
// in CTA order into *out (scaled).
__device__ void energy_reduce(double v, const EnergyWs& ews, double* out, double scale, int64_t cta,
                              int64_t ncta) {
  __shared__ double red[32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q];
    ews.partials[cta] = s;
    __threadfence();
    unsigned int t = atomicAdd(ews.counter, 1u);
    last = (t == (unsigned int)(ncta - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < ncta; q += blockDim.x) s += __ldcg(&ews.partials[q]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += red[q];
    *out = t * scale;
    *ews.counter = 0u;
  }
}

// ---- the pass ---------------------------------------------------------------------------------
// FORM 0: standard (p = u^{n-1}, out = u^{n+1} written over p's buffer when u_next == u_prev)
// FORM 1: increment (p = v^n updated in place, out = u^{n+1} into u_next)
template <typename T, int FORM, bool STORE, bool ENERGY>
__global__ void __launch_bounds__(128) k_leapfrog(const int32_t nx, const int32_t ny, const int64_t ld,
                                                  const typename ArithOf<T>::type ar,
                                                  const T* __restrict__ hx, const T* __restrict__ hy,
                                                  const T* __restrict__ u, const T* p_in, T* p_out,
                                                  T* u_next, const int rows, PassOut o, double escale) {
  constexpr int V = Vec<T>::V;
  const int lane = threadIdx.x & 31;
  int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
  const bool active = i0 < ld;
  if (!active) i0 = 0;  // keep the lane for shuffles; it reads a valid vector and stores nothing
  const int j0 = 1 + blockIdx.y * rows;
  const int j1 = min(j0 + rows, ny - 1);

  // receivers: u^n at the receiver nodes, by the first CTA (u is read-only in this pass)
  if (o.trace && blockIdx.x == 0 && blockIdx.y == 0) {
    const int64_t total = (int64_t)ny * ld;
    for (int r = threadIdx.x; r < o.nrec; r += blockDim.x) {
      const int64_t q = o.rec_idx[r];
      ((T*)o.trace)[r] = (q >= 0 && q < total) ? u[q] : T(0);  // out-of-range receivers read 0
    }
  }

  EAcc<T> acc;
  if (j0 < j1) {
    Pack<T> um = ld_vec(u + (int64_t)(j0 - 1) * ld + i0);
    Pack<T> uc = ld_vec(u + (int64_t)j0 * ld + i0);
    Pack<T> hym = ld_vec(hy + (int64_t)(j0 - 1) * ld + i0);
    for (int j = j0; j < j1; ++j) {
      const int64_t row = (int64_t)j * ld + i0;
      const Pack<T> un = ld_vec(u + row + ld);
      const Pack<T> pv = ld_vec_cg(p_in + row);
      const Pack<T> hxv = ld_vec(hx + row);
      const Pack<T> hyv = ld_vec(hy + row);
      // neighbour columns across lanes
      T ul = __shfl_up_sync(0xffffffffu, uc.a[V - 1], 1);
      T hl = __shfl_up_sync(0xffffffffu, hxv.a[V - 1], 1);
      T ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
      if (lane == 0) {
        ul = (i0 > 0) ? u[row - 1] : T(0);
        hl = (i0 > 0) ? hx[row - 1] : T(0);
      }
      if (lane == 31) ur = (i0 + V < ld) ? u[row + V] : T(0);
      Pack<T> out, pout;
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t i = i0 + e;
        const T xl = (e == 0) ? ul : uc.a[e - 1];
        const T xr = (e == V - 1) ? ur : uc.a[e + 1];
        const T hxl = (e == 0) ? hl : hxv.a[e - 1];
        const T b = ar.b(hxv.a[e], hxl, hyv.a[e], hym.a[e], uc.a[e], xl, xr, un.a[e], um.a[e]);
        const bool interior = (i >= 1) && (i <= nx - 2);
        T unew, up;
        if constexpr (FORM == 0) {
          up = pv.a[e];
          unew = ar.lf(uc.a[e], up, b);
        } else {
          up = uc.a[e] - pv.a[e];
          const T vnew = ar.add(pv.a[e], b);
          unew = ar.add(uc.a[e], vnew);
          pout.a[e] = interior ? vnew : T(0);
        }
        out.a[e] = interior ? unew : T(0);
        if constexpr (ENERGY) {
          if (interior) {
            const T d = uc.a[e] - up;
            acc.add(d * d - b * up);
          }
        }
      }
      if (o.ckpt_a && active) {  // checkpoint copy of the state read by this pass
        st_vec((T*)o.ckpt_a + row, FORM == 0 ? pv : uc);
        st_vec((T*)o.ckpt_b + row, FORM == 0 ? uc : pv);
      }
      if constexpr (STORE) {
        if (active) {
          st_vec(u_next + row, out);
          if constexpr (FORM == 1) st_vec(p_out + row, pout);
        }
      }
      um = uc;
      uc = un;
      hym = hyv;
    }
  }
  if (o.ckpt_a && active) {  // boundary rows of the checkpoint slot are zero
    Pack<T> z;
#pragma unroll
    for (int e = 0; e < V; ++e) z.a[e] = T(0);
    if (j0 == 1) {
      st_vec((T*)o.ckpt_a + i0, z);
      st_vec((T*)o.ckpt_b + i0, z);
    }
    if (j1 == ny - 1) {
      st_vec((T*)o.ckpt_a + (int64_t)(ny - 1) * ld + i0, z);
      st_vec((T*)o.ckpt_b + (int64_t)(ny - 1) * ld + i0, z);
    }
  }
  if constexpr (ENERGY) {
    energy_reduce(active ? acc.value() : 0.0, o.ews, o.energy, escale,
                  (int64_t)blockIdx.y * gridDim.x + blockIdx.x, (int64_t)gridDim.x * gridDim.y);
  }
}

// Taylor start: u^0 (boundary zeroed) and u^1 = (u^0 + tau u1) + B u^0 / 2; for the increment
// form also v^1 = tau u1 + B u^0 / 2.
template <typename T>
__device__ __forceinline__ T u0_at(const T* u0, int32_t nx, int32_t ny, int64_t ld, int64_t i, int64_t j) {
  return (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) ? u0[j * ld + i] : T(0);
}

template <typename T>
__global__ void k_init(const int32_t nx, const int32_t ny, const int64_t ld, const typename ArithOf<T>::type ar,
                       const T tau, const T* __restrict__ hx, const T* __restrict__ hy, const T* __restrict__ u0,
                       const T* __restrict__ u1, T* __restrict__ o_u0, T* __restrict__ o_u1, T* __restrict__ o_v) {
  const int64_t total = (int64_t)ny * ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / ld, i = k - j * ld;
    const bool interior = (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2);
    T a = u0_at(u0, nx, ny, ld, i, j), cur = T(0), v = T(0);
    if (interior) {
      const T b = ar.b(hx[k], hx[k - 1], hy[k], hy[k - ld], a, u0_at(u0, nx, ny, ld, i - 1, j),
                       u0_at(u0, nx, ny, ld, i + 1, j), u0_at(u0, nx, ny, ld, i, j + 1),
                       u0_at(u0, nx, ny, ld, i, j - 1));
      const T w = u1 ? u1[k] : T(0);
      if constexpr (sizeof(T) == 8) {
        cur = __dadd_rn(__dadd_rn(a, __dmul_rn(tau, w)), __dmul_rn(0.5, b));
        v = __dadd_rn(__dmul_rn(tau, w), __dmul_rn(0.5, b));
      } else {
        cur = (a + tau * w) + 0.5f * b;
        v = tau * w + 0.5f * b;
      }
    }
    if (o_u0) o_u0[k] = a;
    o_u1[k] = cur;
    if (o_v) o_v[k] = v;
  }
}

template <typename T>
typename ArithOf<T>::type make_arith(const StencilGeom& g) {
  typename ArithOf<T>::type a;
  a.cx = (T)g.cx;
  a.cy = (T)g.cy;
  return a;
}

constexpr int kStepThreads = 128;

// launch geometry of the pass: CTAs of 128 threads x one vector each across, rows per CTA down
template <typename T>
dim3 step_grid(int64_t ld, int64_t ny, int& rows) {
  const int64_t cols_per_cta = (int64_t)kStepThreads * Vec<T>::V;
  if (rows <= 0) rows = auto_rows(ld, ny, cols_per_cta);
  return dim3((unsigned)((ld + cols_per_cta - 1) / cols_per_cta), (unsigned)((ny - 2 + rows - 1) / rows));
}

template <typename T, int FORM>
cudaError_t step_t(const StencilGeom& g, const void* hx, const void* hy, const void* u_prev, const void* u_cur,
                   void* v, void* u_next, const PassOut& o, bool store, int rows, cudaStream_t s) {
  const int threads = kStepThreads;
  const dim3 grid = step_grid<T>(g.ld, g.ny, rows);
  const auto ar = make_arith<T>(g);
  const T* p_in = (const T*)(FORM == 0 ? u_prev : v);
  T* p_out = (T*)v;
  T* out = (T*)u_next;
  // E = dxdy / (2 tau^2) * sum_nodes [(u^n - u^{n-1})^2 - (B u^n) u^{n-1}]
  const double scale = g.dxdy / (2.0 * g.tau * g.tau);
  if (o.energy) {
    if ((int64_t)grid.x * grid.y > o.ews.capacity) return cudaErrorInvalidValue;
    if (store)
      k_leapfrog<T, FORM, true, true><<<grid, threads, 0, s>>>(g.nx, g.ny, g.ld, ar, (const T*)hx, (const T*)hy,
                                                               (const T*)u_cur, p_in, p_out, out, rows, o, scale);
    else
      k_leapfrog<T, FORM, false, true><<<grid, threads, 0, s>>>(g.nx, g.ny, g.ld, ar, (const T*)hx, (const T*)hy,
                                                                (const T*)u_cur, p_in, p_out, out, rows, o, scale);
  } else {
    if (store)
      k_leapfrog<T, FORM, true, false><<<grid, threads, 0, s>>>(g.nx, g.ny, g.ld, ar, (const T*)hx, (const T*)hy,
                                                                (const T*)u_cur, p_in, p_out, out, rows, o, scale);
    else
      k_leapfrog<T, FORM, false, false><<<grid, threads, 0, s>>>(g.nx, g.ny, g.ld, ar, (const T*)hx,
                                                                 (const T*)hy, (const T*)u_cur, p_in, p_out, out,
                                                                 rows, o, scale);
  }
  return cudaGetLastError();
}

}  // namespace

int64_t one_step_ctas(int64_t ld, int64_t ny, int dtype, int rows) {
  const dim3 grid = dtype == TSU_F32 ? step_grid<float>(ld, ny, rows) : step_grid<double>(ld, ny, rows);
  return (int64_t)grid.x * grid.y;
}

cudaError_t launch_step(const StencilGeom& g, int dtype, int form, const void* hx, const void* hy,
                        const void* u_prev, const void* u_cur, void* v, void* u_next, const PassOut& o, bool store,
                        int rows, cudaStream_t s) {
  if (dtype == TSU_F32)
    return form == TSU_FORM_STANDARD ? step_t<float, 0>(g, hx, hy, u_prev, u_cur, v, u_next, o, store, rows, s)
                                     : step_t<float, 1>(g, hx, hy, u_prev, u_cur, v, u_next, o, store, rows, s);
  return form == TSU_FORM_STANDARD ? step_t<double, 0>(g, hx, hy, u_prev, u_cur, v, u_next, o, store, rows, s)
                                   : step_t<double, 1>(g, hx, hy, u_prev, u_cur, v, u_next, o, store, rows, s);
}

cudaError_t launch_init(const StencilGeom& g, int dtype, int form, const void* hx, const void* hy, const void* u0,
                        const void* u1, tsu_state* st, cudaStream_t s) {
  const int64_t total = (int64_t)g.ny * g.ld;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  // standard: buf[0] = u^0, buf[1] = u^1; increment: buf[0] = u^1, buf[1] = v^1; the rest zeroed
  void* o_u0 = form == TSU_FORM_STANDARD ? st->buf[0] : nullptr;
  void* o_u1 = form == TSU_FORM_STANDARD ? st->buf[1] : st->buf[0];
  void* o_v = form == TSU_FORM_STANDARD ? nullptr : st->buf[1];
  const size_t esz = dtype == TSU_F32 ? 4 : 8;
  for (int b = 2; b < st->nbuf; ++b) {
    cudaError_t e = cudaMemsetAsync(st->buf[b], 0, (size_t)total * esz, s);
    if (e != cudaSuccess) return e;
  }
  if (dtype == TSU_F32)
    k_init<float><<<(unsigned)blocks, 256, 0, s>>>(g.nx, g.ny, g.ld, make_arith<float>(g), (float)g.tau,
                                                    (const float*)hx, (const float*)hy, (const float*)u0,
                                                    (const float*)u1, (float*)o_u0, (float*)o_u1, (float*)o_v);
  else
    k_init<double><<<(unsigned)blocks, 256, 0, s>>>(g.nx, g.ny, g.ld, make_arith<double>(g), g.tau,
                                                     (const double*)hx, (const double*)hy, (const double*)u0,
                                                     (const double*)u1, (double*)o_u0, (double*)o_u1, (double*)o_v);
  return cudaGetLastError();
}

// one partial per CTA of the register-streaming pass (at most ceil(ld/128) column groups x
// (ny - 2) row blocks), or per CTA and level of the temporally blocked pass (at least 16 rows per
// chunk, depth <= 8)
static int64_t energy_slots(int64_t ny, int64_t ld) {
  const int64_t plain = ((ld + 127) / 128) * (ny > 2 ? ny - 2 : 1);
  const int64_t tb = tb_energy_slots(ny, ld, 8, 16);
  return plain > tb ? plain : tb;
}

// the warp-blocked pass's receiver table: tiles + 1 offsets (at least 16 rows per chunk) and
// kWtbMaxReceivers entries
static int64_t rec_table_tiles(int64_t ny, int64_t ld) { return wtb_tiles(ny, ld, 16); }
static size_t rec_off_bytes(int64_t ny, int64_t ld) { return ((size_t)rec_table_tiles(ny, ld) + 1) * sizeof(int); }

static size_t align16(size_t n) { return (n + 15) / 16 * 16; }

static int64_t flow_tiles(int64_t ny, int64_t ld) {
  const int64_t t = rec_table_tiles(ny, ld);
  return t < kFlowMaxTiles ? t : kFlowMaxTiles;
}

size_t energy_ws_bytes(int64_t ny, int64_t ld) {
  return 256 + align16((size_t)energy_slots(ny, ld) * sizeof(double)) +
         align16(rec_off_bytes(ny, ld)) + (size_t)kWtbMaxReceivers * sizeof(int4) + flow_bytes(flow_tiles(ny, ld));
}

EnergyWs energy_ws_carve(void* ws, size_t bytes, int64_t ny, int64_t ld) {
  EnergyWs e{};
  e.counter = (unsigned int*)ws;
  e.status = (int*)((char*)ws + 4);
  e.partials = (double*)((char*)ws + 256);
  e.capacity = energy_slots(ny, ld);
  char* t = (char*)ws + 256 + align16((size_t)e.capacity * sizeof(double));
  const size_t off = align16(rec_off_bytes(ny, ld));
  if (bytes >= energy_ws_bytes(ny, ld)) {
    e.rec_off = (int*)t;
    e.rec_ent = (int4*)(t + off);
    e.rec_tiles_cap = rec_table_tiles(ny, ld);
    e.rec_ent_cap = kWtbMaxReceivers;
    e.flow = t + off + (size_t)kWtbMaxReceivers * sizeof(int4);
    e.flow_tiles_cap = flow_tiles(ny, ld);
  }
  return e;
}

}  // namespace tsu
