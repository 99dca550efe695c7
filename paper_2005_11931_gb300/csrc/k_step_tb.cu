// Temporally blocked leapfrog pass: K steps of
//   u^{n+1} = 2u^n - u^{n-1} + B u^n       (standard form)   or
//   v^{n+1} = v^n + B u^n, u^{n+1} = u^n + v^{n+1}   (increment form)
// per read of the fields from HBM (arXiv:2005.11931, Sec. 2 eq. (2.1) on the Sec. 3.3 box; the
// scheme and operator are those of k_step.cu).
//
// A CTA owns a strip of W = 256 - 2K output columns and a chunk of output rows.  It streams the
// input rows of the extended strip (W + 2K columns: the dependency cone of K steps) down the chunk:
// one elected thread issues 1D bulk-async copies (cp.async.bulk + mbarrier transaction counts)
// of u^n, u^{n-1} (or v^n), hx and hy into a ring of shared-memory stages, P rows ahead.  Each
// thread owns one column; for every time level t = 0..K it keeps the last three rows it computed
// in registers, so the y-neighbours never leave the thread.  x-neighbours of level t-1 come from a
// per-level shared row written one input row earlier; the rows are double buffered by row parity,
// so one CTA barrier per input row orders all K levels.  Level t lags the input by t rows; level K
// (and K-1 in the standard form) are written to the two scratch buffers of the state.
//
// HBM traffic per K steps: 16 B read + 8 B written per node (x (W+2K)/W for the halo columns,
// x (L+2K)/L for the halo rows of an L-row chunk), i.e. ~3 B per lattice update at K = 8.
//
// Every mbarrier wait is bounded; on expiry the CTA records TSU_ETIMEOUT in the status word,
// drains its own copies (bounded) and returns.
#include <string.h>

#include "async_copy.cuh"
#include "stencil_common.cuh"
#include "tsu_internal.h"

namespace tsu {
namespace {
using namespace dev;

constexpr int kTbThreads = 256;  // columns of the extended strip, one per thread
constexpr int kTbPrefetch = 3;   // rows in flight ahead of the row being consumed

template <int K>
struct TbShape {
  static constexpr int WE = kTbThreads;      // extended strip width
  static constexpr int W = WE - 2 * K;       // output columns per strip
  static constexpr int S = K + 2 + kTbPrefetch;  // ring stages
};

// Shared memory layout (floats): ring[S][4][WE], lrow[K-1][2][WE], zero[WE]; then mbarriers.
template <int K>
constexpr size_t tb_smem_bytes() {
  return sizeof(float) * ((size_t)TbShape<K>::S * 4 * kTbThreads + (size_t)(K - 1) * 2 * kTbThreads + kTbThreads) +
         sizeof(uint64_t) * TbShape<K>::S + 64;
}

// 16-byte aligned so that an array of descriptors has the same stride on the host (which packs
// them) and on the device (which indexes them).
struct alignas(16) TbArgs {
  int32_t nx, ny;
  int64_t ld;
  float cx, cy;
  const float* hx;
  const float* hy;
  const float* u;   // u^n
  const float* p;   // u^{n-1} (standard) or v^n (increment)
  float* out_a;     // u^{n+K}
  float* out_b;     // u^{n+K-1} (standard) or v^{n+K} (increment)
  int rows;         // output rows per chunk
  double* energy;   // K doubles or nullptr
  EnergyWs ews;
  double escale;
  int* status;
  uint64_t wait_limit_ns;  // bound of every mbarrier wait
  int skip_row;            // test hook: a row whose copy is never issued (-1: none)
};

template <int K>
__device__ void tb_energy_reduce(float (&es)[K], float (&ec)[K], const TbArgs& a, int64_t cta, int64_t ncta) {
  __shared__ double red[K][kTbThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    double v = (double)es[t] - (double)ec[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[t][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int q = 0; q < kTbThreads / 32; ++q) s += red[threadIdx.x][q];
    a.ews.partials[(int64_t)threadIdx.x * ncta + cta] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int tk = atomicAdd(a.ews.counter, 1u);
    last = (tk == (unsigned int)(ncta - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA sums the partials of level t in warp t, all levels at once (fixed order)
  static_assert(K <= kTbThreads / 32, "one warp per level");
  if (w < K) {
    double s = 0.0;
    for (int64_t q = lane; q < ncta; q += 32) s += __ldcg(&a.ews.partials[(int64_t)w * ncta + q]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) a.energy[w] = s * a.escale;
  }
  if (threadIdx.x == 0) *a.ews.counter = 0u;
}

template <int K, int FORM, bool ENERGY>
__device__ __forceinline__ void tb_body(const TbArgs& a, const int strip, const int chunk, const int64_t cta,
                                        const int64_t ncta) {
  using Sh = TbShape<K>;
  constexpr int WE = Sh::WE, W = Sh::W, S = Sh::S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);             // [S][4][WE]
  float* lrow = ring + (size_t)S * 4 * WE;                      // [K-1][2][WE]
  float* zrow = lrow + (size_t)(K - 1) * 2 * WE;                // [WE]
  uint64_t* bars = reinterpret_cast<uint64_t*>(zrow + WE);      // [S]
  __shared__ int fills[S];                                      // fills issued per stage (thread 0)

  const int tid = threadIdx.x;
  const int64_t x0 = (int64_t)strip * W;                        // first output column
  const int64_t xs = x0 - K;                                    // first column of the extended strip
  const int64_t c = xs + tid;                                   // this thread's column
  const int y0 = 1 + chunk * a.rows;
  const int y1 = min(y0 + a.rows, a.ny - 1);
  const int r_first = y0 - K;                                   // first input row streamed
  const int r_last = y1 + K - 1;                                // last input row streamed
  const int nit = r_last - r_first + 1;
  const int lo_row = max(r_first, 0), hi_row = min(r_last, a.ny - 1);  // rows actually loaded
  // copy window of every row: columns [cg0, cg1) of the array land at smem offset (cg0 - xs)
  const int64_t cg0 = xs < 0 ? 0 : xs;
  const int64_t cg1 = (xs + WE) < a.ld ? (xs + WE) : a.ld;
  const uint32_t seg_bytes = cg1 > cg0 ? (uint32_t)((cg1 - cg0) * sizeof(float)) : 0u;
  const int soff = (int)(cg0 - xs);

  // zero every staging buffer once (edge strips keep zeros outside the copied window)
  for (int k = tid; k < S * 4 * WE + (K - 1) * 2 * WE + WE; k += kTbThreads) ring[k] = 0.0f;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&bars[s], 1);
      fills[s] = 0;
    }
    fence_barrier_init();
  }
  fence_proxy_async();
  __syncthreads();

  // Only rows in [lo_row, hi_row] are loaded; row r uses stage (r - lo_row) % S and is that
  // stage's fill number (r - lo_row) / S, whose completion has mbarrier phase parity fill & 1.
  auto issue = [&](int r) {  // thread 0 only
    if (r < lo_row || r > hi_row || seg_bytes == 0 || r == a.skip_row) return;
    const int st = (r - lo_row) % S;
    fills[st] += 1;
    float* dst = ring + (size_t)st * 4 * WE + soff;
    const int64_t go = (int64_t)r * a.ld + cg0;
    mbar_expect_tx(&bars[st], 4 * seg_bytes);
    bulk_g2s(dst + 0 * WE, a.u + go, seg_bytes, &bars[st]);
    bulk_g2s(dst + 1 * WE, a.p + go, seg_bytes, &bars[st]);
    bulk_g2s(dst + 2 * WE, a.hx + go, seg_bytes, &bars[st]);
    bulk_g2s(dst + 3 * WE, a.hy + go, seg_bytes, &bars[st]);
  };
  auto stage = [&](int r) -> const float* {  // 4 x WE floats of row r (zeros outside the loaded rows)
    if (r < lo_row || r > hi_row || seg_bytes == 0) return nullptr;
    return ring + (size_t)((r - lo_row) % S) * 4 * WE;
  };

  if (tid == 0)
    for (int r = r_first; r <= r_first + kTbPrefetch; ++r) issue(r);

  // register windows: w[t][0] = latest row of level t, [1] the one before, [2] the one before that
  float w[K + 1][3];
  float vw[K][2];  // increment form: v of levels 0..K-1, latest two rows
#pragma unroll
  for (int t = 0; t <= K; ++t) w[t][0] = w[t][1] = w[t][2] = 0.0f;
#pragma unroll
  for (int t = 0; t < K; ++t) vw[t][0] = vw[t][1] = 0.0f;
  float es[K], ec[K];
#pragma unroll
  for (int t = 0; t < K; ++t) es[t] = ec[t] = 0.0f;

  const bool col_interior = (c >= 1) && (c <= a.nx - 2);
  const bool col_out = (tid >= K) && (tid < K + W) && (c < a.ld);
  const int tl = tid > 0 ? tid - 1 : 0, tr = tid < WE - 1 ? tid + 1 : WE - 1;
  bool timed_out = false;

  for (int it = 0; it < nit; ++it) {
    const int r_in = r_first + it;
    if (r_in >= lo_row && r_in <= hi_row && seg_bytes) {
      const uint32_t parity = (uint32_t)(((r_in - lo_row) / S) & 1);
      if (!mbar_wait_bounded(&bars[(r_in - lo_row) % S], parity, a.wait_limit_ns)) timed_out = true;
    }
    const float* s0 = stage(r_in);
    // ---- level 0: input row r_in
#pragma unroll
    for (int t = 0; t <= K; ++t) {
      w[t][2] = w[t][1];
      w[t][1] = w[t][0];
    }
    w[0][0] = s0 ? s0[tid] : 0.0f;
    if constexpr (FORM == 1) {
      vw[0][1] = vw[0][0];
      vw[0][0] = s0 ? s0[WE + tid] : 0.0f;
    }
    // ---- levels 1..K
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int rt = r_in - t;
      const float* st = stage(rt);
      const float* sd = stage(rt - 1);
      float ul, ur, up_or_v;
      if (t == 1) {
        ul = st ? st[tl] : 0.0f;
        ur = st ? st[tr] : 0.0f;
        up_or_v = st ? st[WE + tid] : 0.0f;  // u^{n-1} or v^n at row rt
      } else {
        const float* lr = lrow + ((size_t)(t - 2) * 2 + ((it - 1) & 1)) * WE;
        ul = lr[tl];
        ur = lr[tr];
        if constexpr (FORM == 0)
          up_or_v = w[t - 2][2];
        else
          up_or_v = vw[t - 1][1];
      }
      const float hxr = st ? st[2 * WE + tid] : 0.0f;
      const float hxl = st ? st[2 * WE + tl] : 0.0f;
      const float hyu = st ? st[3 * WE + tid] : 0.0f;
      const float hyd = sd ? sd[3 * WE + tid] : 0.0f;
      const float uc = w[t - 1][1], uu = w[t - 1][0], ud = w[t - 1][2];
      const dev::ArithF32 ar{a.cx, a.cy};
      const float b = ar.b(hxr, hxl, hyu, hyd, uc, ul, ur, uu, ud);
      const bool node = col_interior && rt >= 1 && rt <= a.ny - 2;
      float unew, vnew = 0.0f, upv;
      if constexpr (FORM == 0) {
        upv = up_or_v;
        unew = ar.lf(uc, upv, b);
      } else {
        upv = uc - up_or_v;
        vnew = ar.add(up_or_v, b);
        unew = ar.add(uc, vnew);
      }
      unew = node ? unew : 0.0f;
      vnew = node ? vnew : 0.0f;
      w[t][0] = unew;
      if constexpr (FORM == 1) {
        if (t < K) {
          vw[t][1] = vw[t][0];
          vw[t][0] = vnew;
        }
      }
      if (t < K) lrow[((size_t)(t - 1) * 2 + (it & 1)) * WE + tid] = unew;
      if constexpr (ENERGY) {
        if (node && col_out && rt >= y0 && rt < y1) {
          const float d = uc - upv;
          const float y = (d * d - b * upv) - ec[t - 1];
          const float s = es[t - 1] + y;
          ec[t - 1] = (s - es[t - 1]) - y;
          es[t - 1] = s;
        }
      }
      if (t == K && col_out && rt >= y0 && rt < y1) {
        a.out_a[(int64_t)rt * a.ld + c] = unew;
        if constexpr (FORM == 1) a.out_b[(int64_t)rt * a.ld + c] = vnew;
      }
      if constexpr (FORM == 0) {
        if (t == K - 1 && col_out && rt >= y0 && rt < y1) a.out_b[(int64_t)rt * a.ld + c] = unew;
      }
    }
    // one barrier per input row; any expired wait makes the whole CTA stop
    if (__syncthreads_or(timed_out)) {
      timed_out = true;
      break;
    }
    if (tid == 0) issue(r_in + kTbPrefetch + 1);
  }

  if (timed_out) {
    if (tid == 0) {
      atomicExch(a.status, (int)TSU_ETIMEOUT);
      // drain: wait (bounded) for the last fill issued into every stage, so that no copy lands
      // in shared memory after the CTA has exited
      for (int s = 0; s < S; ++s) {
        if (fills[s] == 0) continue;
        const uint32_t par = (uint32_t)((fills[s] - 1) & 1);
        mbar_wait_bounded(&bars[s], par, a.wait_limit_ns);
      }
    }
    __syncthreads();
    return;
  }
  if constexpr (ENERGY) tb_energy_reduce<K>(es, ec, a, cta, ncta);
}

template <int K, int FORM, bool ENERGY>
__global__ void __launch_bounds__(kTbThreads, 2) k_leapfrog_tb(const TbArgs a) {
  tb_body<K, FORM, ENERGY>(a, blockIdx.x, blockIdx.y, (int64_t)blockIdx.y * gridDim.x + blockIdx.x,
                           (int64_t)gridDim.x * gridDim.y);
}

// Batched family: CTA b works on tile tiles[b] = (problem, strip, chunk) of problem descriptor
// probs[problem]; one launch advances every problem of the family by K steps.
template <int K, int FORM>
__global__ void __launch_bounds__(kTbThreads, 2) k_leapfrog_tb_batched(const TbArgs* __restrict__ probs,
                                                                       const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const TbArgs a = probs[t.x];
  tb_body<K, FORM, false>(a, t.y, t.z, 0, 1);
}

template <int K, int FORM>
cudaError_t tb_launch(const TbArgs& a, cudaStream_t s) {
  constexpr size_t smem = tb_smem_bytes<K>();
  dim3 grid((unsigned)((a.ld + TbShape<K>::W - 1) / TbShape<K>::W), (unsigned)((a.ny - 2 + a.rows - 1) / a.rows));
  if (a.energy) {
    if ((int64_t)grid.x * grid.y * K > a.ews.capacity) return cudaErrorInvalidValue;
    auto kern = k_leapfrog_tb<K, FORM, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTbThreads, smem, s>>>(a);
  } else {
    auto kern = k_leapfrog_tb<K, FORM, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTbThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <int K, int FORM>
cudaError_t tb_launch_batched(const TbArgs* probs, const int4* tiles, int64_t ntiles, cudaStream_t s) {
  constexpr size_t smem = tb_smem_bytes<K>();
  auto kern = k_leapfrog_tb_batched<K, FORM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)ntiles, kTbThreads, smem, s>>>(probs, tiles);
  return cudaGetLastError();
}

}  // namespace

bool tb_supported_depth(int k) { return k == 4 || k == 8; }

size_t tb_args_bytes() {
  static_assert(sizeof(TbArgs) % 16 == 0, "descriptor stride must be a multiple of 16 bytes");
  return sizeof(TbArgs);
}

int tb_strip_width(int k) { return kTbThreads - 2 * k; }

void tb_fill_args(void* dst, const StencilGeom& g, const void* hx, const void* hy, const void* u, const void* p,
                  void* out_a, void* out_b, int* status, int rows) {
  TbArgs a{};
  a.nx = g.nx;
  a.ny = g.ny;
  a.ld = g.ld;
  a.cx = (float)g.cx;
  a.cy = (float)g.cy;
  a.hx = (const float*)hx;
  a.hy = (const float*)hy;
  a.u = (const float*)u;
  a.p = (const float*)p;
  a.out_a = (float*)out_a;
  a.out_b = (float*)out_b;
  a.rows = rows;
  a.energy = nullptr;
  a.escale = 0.0;
  a.status = status;
  a.wait_limit_ns = 2000000000ull;
  a.skip_row = -1;
  memcpy(dst, &a, sizeof a);
}

cudaError_t launch_step_tb_batched(int form, int k, const void* probs_dev, const void* tiles_dev, int64_t ntiles,
                                   cudaStream_t s) {
  const TbArgs* p = (const TbArgs*)probs_dev;
  const int4* t = (const int4*)tiles_dev;
  if (k == 4) return form == TSU_FORM_STANDARD ? tb_launch_batched<4, 0>(p, t, ntiles, s)
                                               : tb_launch_batched<4, 1>(p, t, ntiles, s);
  if (k == 8) return form == TSU_FORM_STANDARD ? tb_launch_batched<8, 0>(p, t, ntiles, s)
                                               : tb_launch_batched<8, 1>(p, t, ntiles, s);
  return cudaErrorInvalidValue;
}

int64_t tb_energy_slots(int64_t ny, int64_t ld, int k, int rows) {
  const int W = kTbThreads - 2 * k;
  return ((ld + W - 1) / W) * ((ny - 2 + rows - 1) / rows) * k;
}

cudaError_t launch_step_tb(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                           const void* p, void* out_a, void* out_b, double* energy, const EnergyWs& ews, int* status,
                           int rows, int debug_flags, cudaStream_t s) {
  TbArgs a;
  // test hook (debug_flags & 1): never issue the copy of the chunk's second loaded row, so that
  // the consumers' bounded wait expires; the wait limit is then 20 ms instead of 2 s
  a.skip_row = (debug_flags & 1) ? 2 : -1;
  a.wait_limit_ns = (debug_flags & 1) ? 20000000ull : 2000000000ull;
  a.nx = g.nx;
  a.ny = g.ny;
  a.ld = g.ld;
  a.cx = (float)g.cx;
  a.cy = (float)g.cy;
  a.hx = (const float*)hx;
  a.hy = (const float*)hy;
  a.u = (const float*)u;
  a.p = (const float*)p;
  a.out_a = (float*)out_a;
  a.out_b = (float*)out_b;
  a.rows = rows;
  a.energy = energy;
  a.ews = ews;
  a.escale = g.dxdy / (2.0 * g.tau * g.tau);
  a.status = status;
  if (k == 4) return form == TSU_FORM_STANDARD ? tb_launch<4, 0>(a, s) : tb_launch<4, 1>(a, s);
  if (k == 8) return form == TSU_FORM_STANDARD ? tb_launch<8, 0>(a, s) : tb_launch<8, 1>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace tsu
