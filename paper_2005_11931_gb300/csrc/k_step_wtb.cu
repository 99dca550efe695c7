// Warp-blocked leapfrog pass: K = 2 or 4 steps of the scheme of k_step.cu per read of the fields
// from HBM (arXiv:2005.11931, Sec. 2 eq. (2.1) on the Sec. 3.3 box), without any CTA barrier.
//
// Every warp works alone on a tile: a strip of 128 columns (one float4 per lane) of which the
// middle 120 are output (a 4-column halo on each side covers the K-step dependency cone), and a
// chunk of L output rows it streams down.  Strip s reads columns 120 s - x .. 120 s - x + 127 and
// outputs the middle 120, with x = 8 or 4 per launch.  At x = 8 its reads start on a 32-byte
// sector (rows of a multiple of 8 floats): a row of a field touches 16 sectors, the one at each
// side shared with the neighbouring strip, and its writes start 16 bytes into one.  At x = 4 the
// writes are sector-aligned and a read touches 17 sectors, two of them half used.  Measured on
// GB300 (FP32 GLUPS, x = 8 against x = 4): the persistent pass 1049 against 969 at 8192^2 (DRAM
// reads per pass 1.199 against 1.251 GB), 988 against 919-932 at 4096^2; the batched family 974
// against 929; the receiver-recording pass (2048^2 adjoint workload) 33.9 against 35.1 ms.  The
// launch-per-pass pass without receivers, its tiles running in lockstep, moves the same DRAM
// bytes either way, but at x = 8 it makes 47 % more L2 read-sector requests and runs slower:
// 850 against 963 at 8192^2, 766 against 824 at 4096^2, 989 against 1076 at 16384^2; it keeps
// x = 4.  Each thread stages its own float4 of every input row
// (u^n, u^{n-1} or v^n, hx, hy) through a private ring in shared memory with 16-byte cp.async
// copies, P rows ahead, and reads back only what it copied itself (cp.async.wait_group), so no
// thread waits for another.  Time level t lags the input by t rows; for each level the thread
// keeps its four columns of the latest rows in registers, with the y face fluxes below the current
// row, and evaluates every face flux once: the x flux left of its first column comes from the
// lane on the left, the right neighbour of its last column from the lane on the right (shuffles).
// Level K is written with level K-1 (standard form) or v (increment form) of the same row.
//
// HBM traffic per K steps: 16 B read + 8 B written per node, x 128/120 for the halo columns and
// x (L + 2K)/L for the halo rows: 6.4 B per lattice update at K = 4.
//
// The segment variant (k_leapfrog_wtb_seg) also writes every intermediate level u^{n+1} ..
// u^{n+K-1}: the states the reverse sweep of the adjoint reads, recomputed from a checkpoint at
// 4 + (16 + 4)/K B per node and step instead of 24 B for one step per pass.
#include <string.h>

#include <atomic>

#include <type_traits>

#include "async_copy.cuh"
#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

constexpr int kWtbWarps = 4;       // warps (independent tiles) per CTA
constexpr int kWtbOut = 120;       // output columns per strip
constexpr int kWtbXAligned = 8;    // strip offset x with sector-aligned reads
constexpr int kWtbXLockstep = 4;   // strip offset x with sector-aligned writes
// strips over the columns 0 .. ld - 1 (strip s outputs 120 s + 4 - x .. 120 s + 123 - x), and the
// strip whose output columns hold column i
__host__ __device__ __forceinline__ int64_t wtb_nstrips(int64_t ld, int x) {
  return (ld + x - 4 + kWtbOut - 1) / kWtbOut;
}
__host__ __device__ __forceinline__ int64_t wtb_strip_of(int64_t i, int x) { return (i + x - 4) / kWtbOut; }
constexpr int kWtbPre = 2;         // rows in flight ahead of the one being consumed
// Tiles are sized for one wave of three CTAs per SM (the kernels are bounded to 128 registers so
// that four fit: 8192^2 801 against 792 GLUPS unbounded at 130 registers, 16384^2 952 against
// 922; sizing the tiles for four CTAs instead lost 4-8 % on 2048^2 and 4096^2).
constexpr int kWtbCtasPerSm = 3;

template <int K>
struct WtbShape {
  // rings of power-of-two length (slot = row index & (S - 1))
  static constexpr int SA = 4;                // (u, p) rows: in flight (2) + current + previous
  static constexpr int SB = 8;                // (hx, hy) rows: the levels' rows (K), the input row, in flight (2)
  static_assert(kWtbPre + 2 <= SA && K + 1 + kWtbPre <= SB, "ring too short");
  // bytes per thread
  static constexpr int bytes = (SA * 2 + SB * 2) * 16;
};

// 16-byte aligned: arrays of descriptors have the same stride on the host and the device.
struct alignas(16) WtbArgs {
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
  int xoff;         // strip s reads the columns 120 s - xoff .. 120 s - xoff + 127 (4 or 8)
  int64_t nstrips, ntiles;
  double* energy;   // K doubles or nullptr
  EnergyWs ews;
  double escale;
  float* seg;       // segment variant: u^{n+t} at seg + (t - 1) seg_stride, t = 1 .. K - 1
  int64_t seg_stride;
  float* traces;           // traces[t * nrec + r] = u^{n+t} at receiver r, t = 0 .. K - 1
  int32_t nrec;
  const int* rec_off;      // receiver table: tile t's entries rec_ent[rec_off[t] .. rec_off[t + 1])
  const int4* rec_ent;     // (row, col, receiver, 0)
};



template <int K>
__device__ void wtb_energy(float (&es)[K], float (&ec)[K], const WtbArgs& a) {
  __shared__ double red[K][kWtbWarps];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < K; ++t) {
    double v = (double)es[t] - (double)ec[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[t][w] = v;
  }
  __syncthreads();
  const int64_t ncta = gridDim.x;
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int q = 0; q < kWtbWarps; ++q) s += red[threadIdx.x][q];
    a.ews.partials[(int64_t)threadIdx.x * ncta + blockIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int tk = atomicAdd(a.ews.counter, 1u);
    last = (tk == (unsigned int)(ncta - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA sums the partials of level t in warp t, all levels at once (a fixed order: lane
  // l takes the CTAs l, l + 32, ..., then a shuffle tree), so the pass ends one L2 round trip
  // after its last tile rather than K
  static_assert(K <= kWtbWarps, "one warp per level");
  if (w < K) {
    double s = 0.0;
    for (int64_t q = lane; q < ncta; q += 32) s += __ldcg(&a.ews.partials[(int64_t)w * ncta + q]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) a.energy[w] = s * a.escale;
  }
  if (threadIdx.x == 0) *a.ews.counter = 0u;
}

// One tile's K steps: input state (in_u, in_p), output state (o_a, o_b).  FLOW: the tile's
// per-level energy sums go to fpart[t * fstride + tile_id] (warp-reduced as wtb_energy does)
// instead of into the CTA's partial.
template <int K, int FORM, bool ENERGY, bool ALL, bool REC = false, bool UNROLL2 = false, bool FLOW = false>
__device__ __forceinline__ void wtb_body(const WtbArgs& a, const bool tile_ok, const int64_t strip,
                                         const int64_t chunk, const int64_t tile_id, const float* in_u,
                                         const float* in_p, float* o_a, float* o_b, double* fpart = nullptr,
                                         const int64_t fstride = 0) {
  using Sh = WtbShape<K>;
  extern __shared__ __align__(16) unsigned char wtb_smem[];
  const int lane = threadIdx.x & 31;
  // this thread's private ring: A[SA][2] float4 (u, p), B[SB][2] float4 (hx, hy)
  float* ringA = reinterpret_cast<float*>(wtb_smem) + (size_t)threadIdx.x * 4;
  const int stride = kWtbWarps * 32 * 4;  // floats between consecutive float4 slots of one thread
  auto slotA = [&](unsigned s, int f) { return ringA + (size_t)(s * 2 + f) * stride; };
  auto slotB = [&](unsigned s, int f) { return ringA + (size_t)(Sh::SA * 2 + s * 2 + f) * stride; };

  // first column read (lane 0, halo); the persistent pass always takes the aligned layout
  const int64_t xs = strip * kWtbOut - (FLOW ? kWtbXAligned : a.xoff);
  const int64_t c0 = xs + 4 * lane;  // first of this lane's four columns
  const int y0 = 1 + (int)chunk * a.rows;
  const int y1 = tile_ok ? min(y0 + a.rows, a.ny - 1) : y0;
  const int r_first = y0 - K, nit = tile_ok ? (y1 - y0) + 2 * K : 0;
  const bool col_in = c0 >= 0 && c0 < a.ld;  // the whole float4 lies in the row (ld % 4 == 0)
  const bool col_out = lane >= 1 && lane <= 30 && col_in;
  bool node_col[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) node_col[e] = (c0 + e >= 1) && (c0 + e <= a.nx - 2);

  // ALL (the segment recompute, whose fields exceed the L2 on the grids it runs on): the first 2K
  // input rows of a tile are the last rows the tile above reads, at its end; they are copied with
  // a priority to stay in the L2 until then
  [[maybe_unused]] const uint64_t keep = ALL ? l2_evict_last() : 0ull;
  auto issue = [&](int r) {  // copies of input row r into the rings (zeros outside the grid)
    const bool ok = col_in && r >= 0 && r < a.ny;
    const int64_t go = ok ? (int64_t)r * a.ld + c0 : 0;
    const unsigned sa = (unsigned)(r - r_first) & (Sh::SA - 1), sb = (unsigned)(r - r_first) & (Sh::SB - 1);
    if (ALL && r - r_first < 2 * K) {
      cp16_hint(slotA(sa, 0), in_u + go, ok, keep);
      cp16_hint(slotA(sa, 1), in_p + go, ok, keep);
      cp16_hint(slotB(sb, 0), a.hx + go, ok, keep);
      cp16_hint(slotB(sb, 1), a.hy + go, ok, keep);
    } else {
      cp16(slotA(sa, 0), in_u + go, ok);
      cp16(slotA(sa, 1), in_p + go, ok);
      cp16(slotB(sb, 0), a.hx + go, ok);
      cp16(slotB(sb, 1), a.hy + go, ok);
    }
  };
  auto ringB = [&](int r, int f) -> P4 {  // hx (f = 0) or hy (f = 1) of row r, zeros outside
    if (r < r_first) return kZeroP4;
    return lds_p4(slotB((unsigned)(r - r_first) & (Sh::SB - 1), f));
  };

  // registers: w[t][0..2] = level t at its latest three rows, v[t][0..1] likewise (increment form)
  P4 w[K + 1][3];
  P4 vv[K][2];
  P4 gb[K];  // gb[t - 1]: level t's y flux at the faces below its current row
#pragma unroll
  for (int t = 0; t <= K; ++t)
#pragma unroll
    for (int q = 0; q < 3; ++q) w[t][q] = kZeroP4;
#pragma unroll
  for (int t = 0; t < K; ++t) vv[t][0] = vv[t][1] = gb[t] = kZeroP4;
  const f2x cx2 = pk(a.cx, a.cx), cy2 = pk(a.cy, a.cy), ncx2 = pk(-a.cx, -a.cx), ncy2 = pk(-a.cy, -a.cy);
  // receivers whose node this tile owns (output columns and rows), from the call's receiver
  // table (k_wtb_rec_table): one per lane; more than 32 in one tile are read back from the
  // table at every record.  Receivers on the boundary or outside the grid belong to no tile:
  // k_trace_edges records them once per call.
  int rec_row = -1, rec_col = 0, rec_r = 0, rec_count = 0, rec_lo = 0;
  if constexpr (REC) {
    if (tile_ok) {
      rec_lo = a.rec_off[tile_id];
      rec_count = a.rec_off[tile_id + 1] - rec_lo;
      if (lane < rec_count) {
        const int4 e = a.rec_ent[rec_lo + lane];
        rec_row = e.x;
        rec_col = e.y;
        rec_r = e.z;
      }
    }
  }
  // rows the tile's receivers lie on, from rec_rmin to rec_rmax: other rows skip the ballot
  int rec_rmin = 0, rec_rmax = -1;
  if constexpr (REC) {
    if (rec_count > 32) {
      rec_rmin = y0;
      rec_rmax = y1 - 1;
    } else if (rec_count > 0) {
      rec_rmin = __reduce_min_sync(0xffffffffu, lane < rec_count ? rec_row : 0x7fffffff);
      rec_rmax = __reduce_max_sync(0xffffffffu, lane < rec_count ? rec_row : -1);
    }
  }
  // trace of level t (u^{n+t}) at row r: the owning lane stores its element
  auto record = [&](int t, int r, const P4& v) {
    if constexpr (REC) {
      if (r < rec_rmin || r > rec_rmax) return;
      const float2 v01 = upk(v.p[0]), v23 = upk(v.p[1]);
      auto put = [&](int col, int rr) {
        const int64_t e = col - c0;
        if (e >= 0 && e < 4)  // selects, not an indexed register array
          a.traces[(int64_t)t * a.nrec + rr] = e == 0 ? v01.x : e == 1 ? v01.y : e == 2 ? v23.x : v23.y;
      };
      if (rec_count <= 32) {
        unsigned m = __ballot_sync(0xffffffffu, rec_row == r);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          put(__shfl_sync(0xffffffffu, rec_col, src), __shfl_sync(0xffffffffu, rec_r, src));
        }
      } else {
        for (int q = rec_lo; q < rec_lo + rec_count; ++q) {
          const int4 e = a.rec_ent[q];
          if (e.x == r) put(e.y, e.z);
        }
      }
    }
  };
  float es[K], ec[K];  // compensated per-level energy sums of this thread
#pragma unroll
  for (int t = 0; t < K; ++t) es[t] = ec[t] = 0.f;

  for (int q = 0; q < kWtbPre; ++q) {
    if (q < nit) issue(r_first + q);
    cp_commit();
  }
  // Iterations whose levels all lie on interior output rows of a strip without boundary columns
  // take the fast path: no masking, no range checks (the edge path handles the rest).
  const bool interior_strip = (xs >= 1) && (xs + 127 <= (int64_t)a.nx - 2);
  // RECNOW: the iteration's rows (r_in - K .. r_in) reach the tile's receiver rows; iterations
  // that do not run a copy of the row code without any receiver test
  // MODE 0: every level's row is an output row of an interior strip; 1 (RMASK, the segment pass
  // only): rows of an interior strip inside the grid, some of them outside the tile's output
  // rows (the tile's first 2K and last K - 1 iterations), whose results are only kept from
  // stores and the energy; 2 (EDGE): everything else, masked node by node.  In the other passes
  // a third copy of the row code (twice over with two rows per loop trip) cost more than it
  // saved: the persistent pass ran 449 against 611 GLUPS at 2048^2, 890 against 988 at 4096^2;
  // the segment pass gains (the 2048^2 adjoint 68.6 against 70.4 ms).
  auto iterate = [&](auto mode_tag, auto rec_tag, const int it) {
    constexpr bool EDGE = decltype(mode_tag)::value == 2;
    constexpr bool RMASK = decltype(mode_tag)::value == 1;
    constexpr bool RECNOW = REC && decltype(rec_tag)::value;
    const int r_in = r_first + it;
    const unsigned sa = (unsigned)it & (Sh::SA - 1);
    // ---- level 0: the input row
#pragma unroll
    for (int t = 0; t <= K; ++t) {
      w[t][2] = w[t][1];
      w[t][1] = w[t][0];
    }
    w[0][0] = lds_p4(slotA(sa, 0));
    if constexpr (RECNOW) {
      if (r_in >= y0 && r_in < y1) record(0, r_in, w[0][0]);
    }
    if constexpr (FORM == 1) {
      vv[0][1] = vv[0][0];
      vv[0][0] = lds_p4(slotA(sa, 1));
    }
    // ---- levels 1..K
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int rt = r_in - t;
      const unsigned sb = (unsigned)(it - t) & (Sh::SB - 1);  // ring slot of row rt (rows >= r_first)
      const P4 hxv = EDGE ? ringB(rt, 0) : lds_p4(slotB(sb, 0));
      const P4 hyv = EDGE ? ringB(rt, 1) : lds_p4(slotB(sb, 1));  // the faces above row rt
      const P4 uc = w[t - 1][1], uu = w[t - 1][0];
      P4 pc;  // u^{n-1} (standard) or v at row rt of the level below
      if (t == 1) {
        if constexpr (FORM == 1)
          pc = vv[0][1];
        else
          pc = (!EDGE || it >= 1) ? lds_p4(slotA((unsigned)(it - 1) & (Sh::SA - 1), 1)) : kZeroP4;
      } else {
        if constexpr (FORM == 0)
          pc = w[t - 2][2];
        else
          pc = vv[t - 1][1];
      }
      const float2 c01 = upk(uc.p[0]), c23 = upk(uc.p[1]);
      const float ur = __shfl_down_sync(0xffffffffu, c01.x, 1);
      // x fluxes at the faces right of the four columns, F = hx (u_right - u), and the one left
      // of column 0 from the lane on the left (its fourth flux)
      const f2x fr01 = mul2(hxv.p[0], pk(__fsub_rn(c01.y, c01.x), __fsub_rn(c23.x, c01.y)));
      const f2x fr23 = mul2(hxv.p[1], pk(__fsub_rn(c23.y, c23.x), __fsub_rn(ur, c23.y)));
      const float2 F01 = upk(fr01), F23 = upk(fr23);
      const float fl = __shfl_up_sync(0xffffffffu, F23.y, 1);
      const bool row_in = !EDGE || (rt >= 1 && rt <= a.ny - 2);
      const bool row_out = !(EDGE || RMASK) || (rt >= y0 && rt < y1);
      P4 bv, un, fx, gy;
      fx.p[0] = pk(__fsub_rn(F01.x, fl), __fsub_rn(F01.y, F01.x));
      fx.p[1] = pk(__fsub_rn(F23.x, F01.y), __fsub_rn(F23.y, F23.x));
      [[maybe_unused]] P4 vn = kZeroP4;
      // increment form: -B u from the negated coefficients (negation is exact, so v - (-B u)
      // rounds as v + B u), which the energy term below uses without another negation
      const f2x ccx = FORM == 1 ? ncx2 : cx2, ccy = FORM == 1 ? ncy2 : cy2;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // y flux at the faces above row rt; the one below is this level's flux of the row before
        gy.p[q] = mul2(hyv.p[q], sub2(uu.p[q], uc.p[q]));
        bv.p[q] = fma2(ccx, fx.p[q], mul2(ccy, sub2(gy.p[q], gb[t - 1].p[q])));
      }
      gb[t - 1] = gy;
      [[maybe_unused]] float erow = 0.f;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // energy term of the pair (u^{n-1}, u^n) at this node: (u^n - u^{n-1})^2 - (B u^n) u^{n-1}
        float2 ef = make_float2(0.f, 0.f);
        if constexpr (FORM == 0) {
          const f2x up = pc.p[q];
          un.p[q] = add2(sub2(add2(uc.p[q], uc.p[q]), up), bv.p[q]);  // (2 u - u_prev) + B u, 2 u exact
          if constexpr (ENERGY) {
            const f2x d = sub2(uc.p[q], up);
            ef = upk(sub2(mul2(d, d), mul2(bv.p[q], up)));
          }
        } else {
          vn.p[q] = sub2(pc.p[q], bv.p[q]);  // v^{n+1} = v^n + B u^n (bv holds -B u^n)
          un.p[q] = add2(uc.p[q], vn.p[q]);
          // (u^n - u^{n-1})^2 - (B u^n) u^{n-1} with u^n - u^{n-1} = v^n and u^{n-1} = u^n - v^n:
          // v^n (v^n + B u^n) - (B u^n) u^n = v^n v^{n+1} + (-B u^n) u^n
          if constexpr (ENERGY) ef = upk(fma2(bv.p[q], uc.p[q], mul2(pc.p[q], vn.p[q])));
        }
        if constexpr (EDGE) {
          const bool n0 = row_in && node_col[2 * q], n1 = row_in && node_col[2 * q + 1];
          const float2 uq = upk(un.p[q]);
          un.p[q] = pk(n0 ? uq.x : 0.f, n1 ? uq.y : 0.f);
          if constexpr (FORM == 1) {
            const float2 vq = upk(vn.p[q]);
            vn.p[q] = pk(n0 ? vq.x : 0.f, n1 ? vq.y : 0.f);
          }
          if constexpr (ENERGY) {
            const bool o = row_out && col_out;
            erow += (n0 && o ? ef.x : 0.f) + (n1 && o ? ef.y : 0.f);
          }
        } else if constexpr (ENERGY) {
          // lanes that are not output are masked once at the end
          if constexpr (RMASK)
            erow += row_out ? ef.x + ef.y : 0.f;
          else
            erow += ef.x + ef.y;
        }
      }
      if constexpr (ENERGY) {
        const float y = erow - ec[t - 1];
        const float sum = es[t - 1] + y;
        ec[t - 1] = (sum - es[t - 1]) - y;
        es[t - 1] = sum;
      }
      w[t][0] = un;
      if constexpr (RECNOW) {
        if (t < K && row_out) record(t, rt, un);
      }
      if constexpr (ALL) {
        if (t < K && row_out && col_out) stg_p4(a.seg + (int64_t)(t - 1) * a.seg_stride + (int64_t)rt * a.ld + c0, un);
      }
      if constexpr (FORM == 1) {
        if (t < K) {
          vv[t][1] = vv[t][0];
          vv[t][0] = vn;
        }
      }
      if (t == K && row_out && col_out) {
        const int64_t o = (int64_t)rt * a.ld + c0;
        stg_p4(o_a + o, un);
        if constexpr (FORM == 1)
          stg_p4(o_b + o, vn);
        else if constexpr (!ALL)
          stg_p4(o_b + o, w[K - 1][1]);  // level K-1 at the same row (the segment has it already)
      }
    }
  };
  auto row = [&](const int it) {
    const int r_in = r_first + it;
    if (it + kWtbPre < nit) issue(r_in + kWtbPre);
    cp_commit();
    cp_wait<kWtbPre>();  // this thread's copies of row r_in have landed
    // rows r_in - K .. r_in - 1 of the levels: all output rows, or all inside the grid.  Levels
    // whose rows lie above the tile's first input row (the first K iterations) read ring slots of
    // the tile before; those rows are outside the dependency cone of the output rows and feed
    // nothing that is kept.
    const bool edge = !(interior_strip && r_in - K >= y0 && r_in - 1 < y1);
    using M0 = std::integral_constant<int, 0>;
    using M1 = std::integral_constant<int, 1>;
    using M2 = std::integral_constant<int, 2>;
    if (REC && r_in >= rec_rmin && r_in - K <= rec_rmax) {
      if (edge)
        iterate(M2(), std::integral_constant<bool, true>(), it);
      else
        iterate(M0(), std::integral_constant<bool, true>(), it);
    } else {
      if constexpr (ALL && !REC) {
        if (edge && interior_strip && r_in - K >= 1 && r_in - 1 <= a.ny - 2) {
          iterate(M1(), std::integral_constant<bool, false>(), it);
          return;
        }
      }
      if (edge)
        iterate(M2(), std::integral_constant<bool, false>(), it);
      else
        iterate(M0(), std::integral_constant<bool, false>(), it);
    }
  };
  int it = 0;
  if constexpr (UNROLL2) {
    // Two rows per trip: the window shifts of one row become register renames in the other.
    // The empty asm statements keep the compiler from interleaving the two rows (which raises
    // the register count past the bound and spills): 8192^2 912 against 896 GLUPS, 4096^2 742
    // against 709, 16384^2 1030 against 1037.
#pragma unroll 1
    for (; it + 1 < nit; it += 2) {
      row(it);
      asm volatile("" ::: "memory");
      row(it + 1);
      asm volatile("" ::: "memory");
    }
    if (it < nit) row(it);
  } else {
    for (; it < nit; ++it) row(it);
  }
  if constexpr (ENERGY) {
    if (!col_out) {  // fast-path sums of halo lanes and lanes beyond the row
#pragma unroll
      for (int t = 0; t < K; ++t) es[t] = ec[t] = 0.f;
    }
  }
  cp_wait<0>();
  if constexpr (ENERGY) {
    if constexpr (FLOW) {
#pragma unroll
      for (int t = 0; t < K; ++t) {
        double v = (double)es[t] - (double)ec[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) fpart[(int64_t)t * fstride + tile_id] = v;
      }
    } else {
      wtb_energy<K>(es, ec, a);
    }
  }
}

// Strip and chunk of a single-problem tile.  The tiles of the two outer strips (masked on every
// row, the slowest) come first, so that a launch does not end on them (8192^2 979 against 938
// GLUPS, 4096^2 831 against 771); the other strips follow chunk by chunk.  32-bit arithmetic:
// the launchers refuse 2^31 tiles or more.
__device__ __forceinline__ void wtb_tile_coords(const int64_t tile, const WtbArgs& a, uint32_t& strip,
                                                uint32_t& chunk) {
  const uint32_t t = (uint32_t)tile, ns = (uint32_t)a.nstrips, nchunks = (uint32_t)a.ntiles / ns;
  if (ns < 3) {
    strip = t % ns;
    chunk = t / ns;
  } else if (t < 2 * nchunks) {
    strip = (t & 1) ? ns - 1 : 0;
    chunk = t >> 1;
  } else {
    const uint32_t r = t - 2 * nchunks, inner = ns - 2;
    chunk = r / inner;
    strip = 1 + (r - chunk * inner);
  }
}

template <int K, int FORM, bool ENERGY, bool REC>
__global__ void __launch_bounds__(kWtbWarps * 32, 4) k_leapfrog_wtb(const WtbArgs a) {
  const int64_t tile = (int64_t)blockIdx.x * kWtbWarps + (threadIdx.x >> 5);
  const bool ok = tile < a.ntiles;
  uint32_t strip = 0, chunk = 0;
  if (ok) wtb_tile_coords(tile, a, strip, chunk);
  wtb_body<K, FORM, ENERGY, false, REC, !REC>(a, ok, strip, chunk, tile, a.u, a.p, a.out_a, a.out_b);
}

template <int K, int FORM>
__global__ void __launch_bounds__(kWtbWarps * 32, 4) k_leapfrog_wtb_seg(const WtbArgs a) {
  const int64_t tile = (int64_t)blockIdx.x * kWtbWarps + (threadIdx.x >> 5);
  const bool ok = tile < a.ntiles;
  uint32_t strip = 0, chunk = 0;
  if (ok) wtb_tile_coords(tile, a, strip, chunk);
  wtb_body<K, FORM, false, true, false, true>(a, ok, strip, chunk, 0, a.u, a.p, a.out_a, a.out_b);
}

// Batched family: warp w of CTA b works on tile tiles[4 b + w] = (problem, strip, chunk) of
// descriptor probs[problem]; one launch advances every problem by K steps.
template <int K, int FORM>
__global__ void __launch_bounds__(kWtbWarps * 32, 4) k_leapfrog_wtb_batched(const WtbArgs* __restrict__ probs,
                                                                        const int4* __restrict__ tiles,
                                                                        const int64_t ntiles) {
  const int64_t tile = (int64_t)blockIdx.x * kWtbWarps + (threadIdx.x >> 5);
  const bool ok = tile < ntiles;
  const int4 t = ok ? tiles[tile] : make_int4(0, 0, 0, 0);
  const WtbArgs a = probs[t.x];
  wtb_body<K, FORM, false, false>(a, ok, t.y, t.z, 0, a.u, a.p, a.out_a, a.out_b);
}

// The tile index wtb_tile_coords maps to (strip, chunk).
__device__ __forceinline__ int64_t wtb_tile_index(const int64_t strip, const int64_t chunk, const int64_t ns,
                                                  const int64_t nchunks) {
  if (ns < 3) return chunk * ns + strip;
  if (strip == 0) return 2 * chunk;
  if (strip == ns - 1) return 2 * chunk + 1;
  return 2 * nchunks + chunk * (ns - 2) + (strip - 1);
}

// The receiver table of one call (one CTA): every interior receiver under the tile whose output
// region (strip s: columns 120 s .. 120 s + 119; chunk c: rows 1 + c rows ..) holds its node.
// Counts per tile, an inclusive scan (off[t] = the end of tile t), then each entry placed by an
// atomic decrement (off[t] ends at the start of tile t; off[ntiles] = the total).  The order of a
// tile's entries is not fixed, and nothing depends on it: each receiver has its own trace slot.
__global__ void __launch_bounds__(1024) k_wtb_rec_table(const int32_t nx, const int32_t ny, const int64_t ld,
                                                        const int rows, const int64_t nstrips, const int64_t ntiles,
                                                        const int64_t* rec_idx, const int32_t nrec, int* off,
                                                        int4* ent) {
  __shared__ int wsum[32];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t nchunks = ntiles / nstrips;
  auto tile_of = [&](const int r, int& j, int& i) -> int64_t {
    const int64_t v = rec_idx[r];
    if (v < 0 || v >= (int64_t)ny * ld) return -1;
    const int64_t jj = v / ld, ii = v - jj * ld;
    if (jj < 1 || jj > ny - 2 || ii < 1 || ii > nx - 2) return -1;
    j = (int)jj;
    i = (int)ii;
    return wtb_tile_index(wtb_strip_of(ii, kWtbXAligned), (jj - 1) / rows, nstrips, nchunks);
  };
  for (int64_t t = threadIdx.x; t <= ntiles; t += blockDim.x) off[t] = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
    int j, i;
    const int64_t t = tile_of(r, j, i);
    if (t >= 0) atomicAdd(&off[t], 1);
  }
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    int v = t < ntiles ? off[t] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += n;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      int x = lane < nw ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += n;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    const int incl = v + (w > 0 ? wsum[w - 1] : 0) + carry;
    if (t < ntiles) off[t] = incl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[ntiles] = carry;
  __syncthreads();
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
    int j = 0, i = 0;
    const int64_t t = tile_of(r, j, i);
    if (t >= 0) ent[atomicSub(&off[t], 1) - 1] = make_int4(j, i, r, 0);
  }
}

// traces[k nrec + r] = 0 for k < nsteps at every receiver r whose node is on the boundary or
// outside the grid (Dirichlet: u = 0 there); the warp-blocked pass records only interior nodes.
__global__ void k_trace_edges(const int32_t nx, const int32_t ny, const int64_t ld, const int64_t* rec_idx,
                              const int32_t nrec, float* traces, const int64_t nsteps) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
    const int64_t v = rec_idx[r];
    bool interior = false;
    if (v >= 0 && v < (int64_t)ny * ld) {
      const int64_t j = v / ld, i = v - j * ld;
      interior = j >= 1 && j <= ny - 2 && i >= 1 && i <= nx - 2;
    }
    if (!interior)
      for (int64_t k = 0; k < nsteps; ++k) traces[k * nrec + r] = 0.f;
  }
}

// ---- all K-step passes of a call in one persistent launch --------------------------------------
// Each warp takes tasks (pass, tile) in increasing order from a counter, and starts one once the
// 3 x 3 tiles around it have finished the pass before.  Those tiles are the ones whose outputs
// it reads as its halo, and the ones that read the buffer it is about to overwrite.  So a tile's
// next pass begins while far-away tiles still finish the current one, instead of every SM
// waiting for the slowest tile at the end of each launch.  Passes alternate between two
// (u, v) pairs.  Every wait is bounded (TSU_ETIMEOUT in the status word).  A task waits only for
// tasks handed out before it, which running warps hold, so every wait ends.  A
// tile's energy sums go to a slot of kFlowSlots per-pass partials.  The task that finishes a
// pass last sums them in the order wtb_energy uses, so the energies, like the states, equal those
// of the launch-per-pass path bit for bit.
struct WtbFlow {
  float* u[2];  // pass p reads (u, v)[p & 1] and writes (u, v)[(p + 1) & 1]
  float* v[2];
  double* energy;  // K doubles per pass, or nullptr
  unsigned int* next;
  int* count;    // [kFlowSlots] tiles that finished the pass held by the slot
  int* reduced;  // [kFlowSlots] the last pass whose partials the slot gave up
  int* done;     // [ntiles] passes finished
  double* part;  // [kFlowSlots][K][nt4]
  int* status;
  int64_t npass, nt4;
  uint64_t limit_ns;
  int hold;  // test hook of the failure detection: 1 = tile 0 never reports a pass done
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// bounded wait for *p >= target
__device__ bool wait_ge(const int* p, const int target, const uint64_t limit_ns) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = global_ns();
  for (long long it = 0; it < kSpinCap; ++it) {
    __nanosleep(100);
    if (ld_acquire(p) >= target) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

template <bool ENERGY>
__global__ void __launch_bounds__(kWtbWarps * 32, 4) k_leapfrog_wtb_flow(const WtbArgs a, const WtbFlow f) {
  constexpr int K = 4;
  const int lane = threadIdx.x & 31;
  // 32-bit task numbers (the launcher keeps npass * ntiles below 2^31); what the body does not
  // need is recomputed from the task number after it
  for (;;) {
    unsigned int task = 0;
    if (lane == 0) task = atomicAdd(f.next, 1u);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= (unsigned int)f.npass * (unsigned int)a.ntiles) break;
    const unsigned int nt = (unsigned int)a.ntiles;
    const unsigned int pass = task / nt, tile = task - pass * nt;
    uint32_t strip = 0, chunk = 0;
    wtb_tile_coords(tile, a, strip, chunk);
    const unsigned int slot = pass % kFlowSlots;
    bool ok = true;
    if (lane < 9 && pass > 0) {
      const int ns = (int)a.nstrips, nch = (int)(nt / (unsigned int)ns);
      const int sx = (int)strip + lane % 3 - 1, cy = (int)chunk + lane / 3 - 1;
      if (sx >= 0 && sx < ns && cy >= 0 && cy < nch)
        ok = wait_ge(f.done + wtb_tile_index(sx, cy, ns, nch), (int)pass, f.limit_ns);
    }
    if (ENERGY && lane == 9 && pass >= kFlowSlots)
      ok = wait_ge(f.reduced + slot, (int)(pass - kFlowSlots), f.limit_ns);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicExch(f.status, (int)TSU_ETIMEOUT);
      break;
    }
    {
      const int q = (int)(pass & 1);
      wtb_body<K, 1, ENERGY, false, false, true, true>(a, true, strip, chunk, tile, f.u[q], f.v[q], f.u[q ^ 1],
                                                       f.v[q ^ 1], f.part + (int64_t)slot * K * f.nt4, f.nt4);
    }
    __syncwarp();
    if (lane == 0 && !(f.hold && tile == 0)) {
      __threadfence();
      st_release(f.done + tile, (int)(pass + 1));
    }
    if constexpr (ENERGY) {
      int last = 0;
      if (lane == 0) last = atomicAdd(f.count + slot, 1) == (int)(nt - 1) ? 1 : 0;
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence();
        // CTA c of the launch-per-pass path held tiles 4c .. 4c + 3: its partial, then the sum
        // over CTAs lane by lane and a shuffle tree, as wtb_energy
        const int64_t ncta = f.nt4 / kWtbWarps;
        for (int t = 0; t < K; ++t) {
          const double* pt = f.part + ((int64_t)slot * K + t) * f.nt4;
          double sum = 0.0;
          for (int64_t c = lane; c < ncta; c += 32) {
            double cs = 0.0;
            for (int w = 0; w < kWtbWarps; ++w) cs += __ldcg(pt + c * kWtbWarps + w);
            sum += cs;
          }
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
          if (lane == 0) f.energy[(int64_t)pass * K + t] = sum * a.escale;
        }
        if (lane == 0) {
          f.count[slot] = 0;
          __threadfence();
          st_release(f.reduced + slot, (int)pass);
        }
      }
    }
  }
}

// counters and partials of the persistent pass (one launch before it)
__global__ void k_wtb_flow_init(const WtbFlow f, const int64_t ntiles) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, n = (int64_t)gridDim.x * blockDim.x;
  if (i == 0) *f.next = 0u;
  if (i < kFlowSlots) {
    f.count[i] = 0;
    f.reduced[i] = -1;
  }
  for (int64_t k = i; k < ntiles; k += n) f.done[k] = 0;
  for (int64_t k = i; k < (int64_t)kFlowSlots * 4 * f.nt4; k += n) f.part[k] = 0.0;
}

template <int K, int FORM, bool ENERGY, bool REC>
cudaError_t wtb_launch_kernel(const WtbArgs& a, unsigned grid, size_t smem, cudaStream_t s) {
  auto kern = k_leapfrog_wtb<K, FORM, ENERGY, REC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kWtbWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int K, int FORM>
cudaError_t wtb_launch(const WtbArgs& a, cudaStream_t s) {
  if (a.ntiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // wtb_tile_coords is 32-bit
  const size_t smem = (size_t)WtbShape<K>::bytes * kWtbWarps * 32;
  const unsigned grid = (unsigned)((a.ntiles + kWtbWarps - 1) / kWtbWarps);
  const bool rec = a.traces && a.nrec > 0;
  if (a.energy) {
    if ((int64_t)grid * K > a.ews.capacity) return cudaErrorInvalidValue;
    return rec ? wtb_launch_kernel<K, FORM, true, true>(a, grid, smem, s)
               : wtb_launch_kernel<K, FORM, true, false>(a, grid, smem, s);
  }
  return rec ? wtb_launch_kernel<K, FORM, false, true>(a, grid, smem, s)
             : wtb_launch_kernel<K, FORM, false, false>(a, grid, smem, s);
}

template <int K, int FORM>
cudaError_t wtb_launch_seg(const WtbArgs& a, cudaStream_t s) {
  if (a.ntiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // wtb_tile_coords is 32-bit
  const size_t smem = (size_t)WtbShape<K>::bytes * kWtbWarps * 32;
  auto kern = k_leapfrog_wtb_seg<K, FORM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((a.ntiles + kWtbWarps - 1) / kWtbWarps), kWtbWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int K, int FORM>
cudaError_t wtb_launch_batched(const WtbArgs* probs, const int4* tiles, int64_t ntiles, cudaStream_t s) {
  const size_t smem = (size_t)WtbShape<K>::bytes * kWtbWarps * 32;
  auto kern = k_leapfrog_wtb_batched<K, FORM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((ntiles + kWtbWarps - 1) / kWtbWarps), kWtbWarps * 32, smem, s>>>(probs, tiles, ntiles);
  return cudaGetLastError();
}

}  // namespace

bool wtb_supported_depth(int k) { return k == 2 || k == 4; }

int64_t wtb_strips(int64_t ld) { return wtb_nstrips(ld, kWtbXAligned); }

cudaError_t launch_wtb_rec_table(const StencilGeom& g, int rows, const int64_t* rec_idx, int32_t nrec,
                                 const EnergyWs& ews, cudaStream_t s) {
  const int64_t nstrips = wtb_nstrips(g.ld, kWtbXAligned);  // the layout of the receiver-recording pass
  const int64_t ntiles = nstrips * ((g.ny - 2 + rows - 1) / rows);
  if (!ews.rec_off || ntiles > ews.rec_tiles_cap || nrec > ews.rec_ent_cap || ntiles >= ((int64_t)1 << 31))
    return cudaErrorInvalidValue;
  k_wtb_rec_table<<<1, 1024, 0, s>>>(g.nx, g.ny, g.ld, rows, nstrips, ntiles, rec_idx, nrec, ews.rec_off,
                                     ews.rec_ent);
  return cudaGetLastError();
}

cudaError_t launch_wtb_trace_edges(const StencilGeom& g, const int64_t* rec_idx, int32_t nrec, void* traces,
                                   int64_t nsteps, cudaStream_t s) {
  if (nrec <= 0 || nsteps <= 0) return cudaSuccess;
  k_trace_edges<<<(unsigned)((nrec + 127) / 128), 128, 0, s>>>(g.nx, g.ny, g.ld, rec_idx, nrec, (float*)traces,
                                                               nsteps);
  return cudaGetLastError();
}

size_t wtb_args_bytes() {
  static_assert(sizeof(WtbArgs) % 16 == 0, "descriptor stride must be a multiple of 16 bytes");
  return sizeof(WtbArgs);
}

void wtb_fill_args(void* dst, const StencilGeom& g, const void* hx, const void* hy, const void* u, const void* p,
                   void* out_a, void* out_b, int rows) {
  WtbArgs a{};
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
  a.xoff = kWtbXAligned;
  a.nstrips = wtb_nstrips(g.ld, a.xoff);
  a.ntiles = a.nstrips * ((g.ny - 2 + rows - 1) / rows);
  a.energy = nullptr;
  memcpy(dst, &a, sizeof a);
}

cudaError_t launch_step_wtb_batched(int form, int k, const void* probs_dev, size_t stride, const void* tiles_dev,
                                    int64_t ntiles, cudaStream_t s) {
  if (stride != sizeof(WtbArgs)) return cudaErrorInvalidValue;
  const WtbArgs* p = (const WtbArgs*)probs_dev;
  const int4* t = (const int4*)tiles_dev;
  if (k == 2) return form == TSU_FORM_STANDARD ? wtb_launch_batched<2, 0>(p, t, ntiles, s)
                                               : wtb_launch_batched<2, 1>(p, t, ntiles, s);
  if (k == 4) return form == TSU_FORM_STANDARD ? wtb_launch_batched<4, 0>(p, t, ntiles, s)
                                               : wtb_launch_batched<4, 1>(p, t, ntiles, s);
  return cudaErrorInvalidValue;
}

int64_t wtb_tiles(int64_t ny, int64_t ld, int rows) {
  return wtb_nstrips(ld, kWtbXAligned) * ((ny - 2 + rows - 1) / rows);  // the larger count of the two layouts
}

// Rows per chunk.  When one wave of 152 SMs x 3 CTAs x 4 warps holds every tile at no more than
// 160 rows each, the fewest rows (>= 16) that do so.  Larger grids take several waves; the chunk
// count is then the largest that keeps the tiles within m whole waves of 4 CTAs per SM (the
// register bound lets four reside), for the smallest m whose chunks have at most 160 rows, so
// that the last wave is full.
int wtb_seg_rows(int64_t ny, int64_t ld) {
  const int64_t strips = wtb_nstrips(ld, kWtbXAligned);
  const int64_t inner = ny - 2;
  const int64_t one_wave = (int64_t)152 * kWtbCtasPerSm * kWtbWarps / strips;
  if (one_wave >= 1) {
    const int64_t rows = (inner + one_wave - 1) / one_wave;
    if (rows <= 160) return (int)(rows < 16 ? 16 : rows);
  }
  const int64_t wave4 = (int64_t)152 * 4 * kWtbWarps;
  for (int64_t m = 1;; ++m) {
    const int64_t chunks = m * wave4 / strips;
    if (chunks < 1) continue;
    const int64_t rows = (inner + chunks - 1) / chunks;
    if (rows <= 160) return (int)(rows < 16 ? 16 : rows);
  }
}

// Measured FP32 GLUPS of this pass (increment form, energy every step, K = 4):
//   8192^2 (69 strips): 894 at 117 rows (the rule's: 4830 tiles, 2 full waves of 4 CTAs per SM),
//   883 at 96, 869 at 140, 866 at 240 (one wave), 858 at 160 (1.48 waves), 850 at 128;
//   16384^2: 1012-1023 at every row count from 96 to 240;  4096^2: 709 at 79 (the rule's, one
//   wave of 3 CTAs per SM), 615 at 96, 502 at 160;  2048^2: 407 at 21 (the rule's).  One step per
//   pass for comparison (scalar version): 247 at 4096^2, 256 at 2048^2, 102 at 1024^2.
int wtb_auto_rows(int64_t ny, int64_t ld, int k) {
  (void)k;
  return wtb_seg_rows(ny, ld);
}

int64_t wtb_energy_slots(int64_t ny, int64_t ld, int k, int rows) {
  return ((wtb_tiles(ny, ld, rows) + kWtbWarps - 1) / kWtbWarps) * k;
}

cudaError_t launch_step_wtb(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                            const void* p, void* out_a, void* out_b, double* energy, const EnergyWs& ews, int rows,
                            cudaStream_t s, int32_t nrec, const int64_t* rec_idx, void* traces) {
  WtbArgs a{};
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
  // strips cover columns [0, ld); receivers: the layout the receiver table is built for
  a.xoff = (traces && nrec > 0) ? kWtbXAligned : kWtbXLockstep;
  a.nstrips = wtb_nstrips(g.ld, a.xoff);
  a.ntiles = a.nstrips * ((g.ny - 2 + rows - 1) / rows);
  a.energy = energy;
  a.ews = ews;
  a.escale = g.dxdy / (2.0 * g.tau * g.tau);
  a.seg = nullptr;
  a.seg_stride = 0;
  a.nrec = traces ? nrec : 0;
  a.traces = (float*)traces;
  a.rec_off = ews.rec_off;
  a.rec_ent = ews.rec_ent;
  if (a.nrec > 0 && !a.rec_off) return cudaErrorInvalidValue;
  if (k == 2) return form == TSU_FORM_STANDARD ? wtb_launch<2, 0>(a, s) : wtb_launch<2, 1>(a, s);
  if (k == 4) return form == TSU_FORM_STANDARD ? wtb_launch<4, 0>(a, s) : wtb_launch<4, 1>(a, s);
  return cudaErrorInvalidValue;
}

namespace {
using FlowKernel = void (*)(const WtbArgs, const WtbFlow);
// resident CTAs of the persistent passes on this device (0: not available), once per device
std::atomic<int> g_flow_ctas[64];
int flow_resident_ctas() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  int v = g_flow_ctas[dev].load();
  if (v != 0) return v > 0 ? v : 0;
  int nsm = 0, per_sm = 0;
  const size_t smem = (size_t)WtbShape<4>::bytes * kWtbWarps * 32;
  bool ok = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  const FlowKernel kerns[2] = {k_leapfrog_wtb_flow<false>, k_leapfrog_wtb_flow<true>};
  for (int e = 0; ok && e < 2; ++e) {
    int q = 0;
    ok = cudaFuncSetAttribute(kerns[e], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, kerns[e], kWtbWarps * 32, smem) == cudaSuccess && q >= 1;
    per_sm = e ? (q < per_sm ? q : per_sm) : q;
  }
  (void)cudaGetLastError();  // a refused query leaves no error behind
  v = ok ? per_sm * nsm : -1;
  g_flow_ctas[dev].store(v);
  return v > 0 ? v : 0;
}

// The persistent launch: one CTA per resident slot (more would only wait), its counters reset
// first.  A plain launch suffices: warps take tasks in order, so every task a warp waits for is
// held by a warp already running, resident or not.
cudaError_t flow_launch(const WtbArgs& a, WtbFlow& f, void* region, int64_t npass, FlowKernel kern, cudaStream_t s,
                        bool* ran) {
  const int ctas = flow_resident_ctas();
  if (ctas <= 0 || npass <= 0 || npass * a.ntiles >= ((int64_t)1 << 31)) return cudaSuccess;
  const size_t smem = (size_t)WtbShape<4>::bytes * kWtbWarps * 32;
  int64_t grid = ctas;
  const int64_t need = (npass * a.ntiles + kWtbWarps - 1) / kWtbWarps;
  if (grid > need) grid = need;
  char* base = (char*)region;
  f.nt4 = (a.ntiles + 3) / 4 * 4;
  f.next = (unsigned int*)base;
  f.count = (int*)(base + 8);
  f.reduced = (int*)(base + 8 + 4 * kFlowSlots);
  f.done = (int*)(base + 128);
  f.part = (double*)(base + 128 + ((size_t)f.nt4 * sizeof(int) + 15) / 16 * 16);
  f.npass = npass;
  f.limit_ns = f.hold ? 20000000ull : 2000000000ull;
  k_wtb_flow_init<<<64, 256, 0, s>>>(f, a.ntiles);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kWtbWarps * 32, smem, s>>>(a, f);
  e = cudaGetLastError();
  if (e == cudaSuccess) *ran = true;
  return e;
}
}  // namespace

// Rows per tile of the persistent pass: tiles about 1.2 x the resident warps, so that every warp
// has a tile of each pass and finishing tiles are followed at once by the next pass's (2048^2:
// 610 GLUPS at 16 rows, 544 at 24, 495 at 32; 4096^2: 940 at 48 rows, 889 at 32, 857 at 64),
// at least 16 rows and no more than the launch-per-pass rule gives, nor 96 (with sector-aligned
// reads, 8192^2: 1040 at 96 rows, 1044 at 80, 1030 at the launch-per-pass rule's 117, 1004 at
// 140; 12288^2: 1042 at 96, 1002 at the rule's).
int wtb_flow_rows(int64_t ny, int64_t ld) {
  const int ctas = flow_resident_ctas();
  const int r0 = wtb_seg_rows(ny, ld) < 96 ? wtb_seg_rows(ny, ld) : 96;
  if (ctas <= 0) return r0;
  const int64_t strips = wtb_nstrips(ld, kWtbXAligned);
  const int64_t warps = (int64_t)ctas * kWtbWarps;
  int64_t rows = ((ny - 2) * strips * 5 + warps * 6 - 1) / (warps * 6);
  if (rows > r0) rows = r0;
  return (int)(rows < 16 ? 16 : rows);
}

// Whether the automatic choice takes the persistent pass: when its tiles number between half and
// 6 times the resident warps.  Measured, FP32 GLUPS with the energy, launch per pass against
// persistent, with the persistent pass's rows rule and sector-aligned reads: 6144^2 914 / 1037,
// 8192^2 963 / 1030-1052, 12288^2 1013 / 1042 (13184 tiles of 96 rows, 5.4 times the warps),
// 16384^2 997 / 996 (23427 tiles); earlier, with unaligned reads, 1024^2 201 / 196, 2048^2 484 /
// 591, 3072^2 697 / 821, 4096^2 820 / 921.
bool wtb_flow_preferred(int64_t ny, int64_t ld) {
  const int ctas = flow_resident_ctas();
  if (ctas <= 0) return false;
  const int64_t warps = (int64_t)ctas * kWtbWarps;
  const int64_t tiles = wtb_tiles(ny, ld, wtb_flow_rows(ny, ld));
  return tiles * 2 >= warps && tiles <= warps * 6;
}

cudaError_t launch_step_wtb_flow(const StencilGeom& g, const void* hx, const void* hy, void* const u[2], void* const v[2],
                                 double* energy, const EnergyWs& ews, int rows, int64_t npass, int debug, cudaStream_t s,
                                 bool* ran) {
  *ran = false;
  WtbArgs a{};
  wtb_fill_args(&a, g, hx, hy, u[0], v[0], u[1], v[1], rows);
  a.ews = ews;
  a.escale = g.dxdy / (2.0 * g.tau * g.tau);
  if (!ews.flow || !ews.status || a.ntiles > ews.flow_tiles_cap) return cudaSuccess;
  WtbFlow f{};
  for (int q = 0; q < 2; ++q) {
    f.u[q] = (float*)u[q];
    f.v[q] = (float*)v[q];
  }
  f.energy = energy;
  f.status = ews.status;
  f.hold = (debug & 2) ? 1 : 0;
  return flow_launch(a, f, ews.flow, npass,
                     energy ? k_leapfrog_wtb_flow<true> : k_leapfrog_wtb_flow<false>, s, ran);
}

cudaError_t launch_step_wtb_seg(const StencilGeom& g, int form, int k, const void* hx, const void* hy, const void* u,
                                const void* p, void* seg, int64_t seg_stride, void* v_out, int rows, cudaStream_t s) {
  WtbArgs a{};
  wtb_fill_args(&a, g, hx, hy, u, p, (float*)seg + (int64_t)(k - 1) * seg_stride, v_out, rows);
  a.seg = (float*)seg;
  a.seg_stride = seg_stride;
  if (k == 2) return form == TSU_FORM_STANDARD ? wtb_launch_seg<2, 0>(a, s) : wtb_launch_seg<2, 1>(a, s);
  if (k == 4) return form == TSU_FORM_STANDARD ? wtb_launch_seg<4, 0>(a, s) : wtb_launch_seg<4, 1>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace tsu
