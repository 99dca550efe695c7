// K adjoint steps per pass, K = 2 or 4 (the paper has no adjoint; this is the exact reverse of
// the scheme of k_step.cu, arXiv:2005.11931 Sec. 2 eq. (2.1) on the Sec. 3.3 box), warp-blocked
// like k_step_wtb.cu, in the increment form of the recursion (mu^n = lam^n - lam^{n+1}, see
// k_adjoint.cu).  Level k = 1..K computes step m = n - k + 1 from level k - 1:
//   mu^m  = mu^{m+1} + B lam^{m+1} + g^m,   lam^m = lam^{m+1} + mu^m
//   dJ/dhx_ij  += -cx (lam^{m+1}_{i+1} - lam^{m+1}_i)(u^m_{i+1} - u^m_i)   (hy likewise)
// (level 0 = (lam^{n+1}, mu^{n+1}) is the input).  Every warp owns a tile: 128
// columns (one float4 per lane; the middle 120 are output, a 4-column halo covers the K-step
// cone; strip s reads the columns 120 s - 8 .. 120 s + 119, so each row read starts on a 32-byte
// sector) by a chunk of rows it streams down; level k lags the input row by k rows.  Each thread
// copies its own float4 of every input row through a private cp.async ring: lam^{n+1},
// mu^{n+1}, hx and hy at the input row (the faces one row behind), u^{n-f} f rows behind, where
// level f + 1 needs it; so nothing in the row loop waits on memory.  The ring keeps the previous
// row of every field, so the levels read u, the input multipliers and the faces of the two
// newest rows from it; only older rows live in registers (168 per thread: 3 CTAs per SM).  The
// face gradients of a row are summed over the K steps in registers (carried from level to
// level) and added to the FP32 accumulators once per pass, by a vector reduction in the L2.
// Only the last level is stored (lam and mu: the next pass's input).  Receiver values are added to mu (and so to lam) in registers, in
// every tile whose extended region holds the receiver (halo copies included): the lanes hold the
// tile's entries and a ballot per row and level finds the ones on it.  Arithmetic runs on paired
// FP32 instructions; B lam is evaluated in flux form (each face flux rounded once, shared by the
// two nodes beside it), the one-step adjoint pass in fused multiply-add form: the two round
// differently, within the FP32 adjoint's tolerance.
#include <string.h>

#include "async_copy.cuh"
#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

constexpr int kAwWarps = 4;
constexpr int kAwOut = 120;
// strips over the columns 0 .. ld - 1: strip s outputs 120 s - 4 .. 120 s + 115
__host__ __device__ __forceinline__ int64_t aw_nstrips(int64_t ld) { return (ld + 4 + kAwOut - 1) / kAwOut; }
constexpr int kAwPre = 2;
constexpr int kAwRing = 4;  // slots per field: the previous row, the current one, 2 in flight
// resident CTAs per SM: the launch bound the kernel is compiled for (K = 2 at <= 168 registers per
// thread, K = 4 at <= 168 as well; checked against -Xptxas -v), and what the rows rule sizes for
template <int K>
constexpr int aw_ctas_per_sm() { return 3; }
// ring fields: lam^{n+1}, mu^{n+1}, hx, hy, u^n .. u^{n-K+1}
template <int K>
constexpr int aw_fields() { return K + 4; }

// acc[0..3] += v (one rounding each, as acc + v): the FP32 gradient accumulators of a row are
// added to in the L2, without a read back into the SM.  Every node gets exactly one such add per
// pass (only the tile that owns a row adds to it), so the sums do not depend on timing.
__device__ __forceinline__ void red_add4(float* acc, const P4& v) {
  const float2 a = upk(v.p[0]), b = upk(v.p[1]);
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(acc), "f"(a.x), "f"(a.y), "f"(b.x),
               "f"(b.y)
               : "memory");
}

template <int K>
struct AwArgs {
  int32_t nx, ny;
  int64_t ld;
  float cx, cy;
  const float* hx;
  const float* hy;
  const float* lam1;   // lam^{n+1}
  const float* mu1;    // mu^{n+1} = lam^{n+1} - lam^{n+2}
  const float* u[K];   // u^n, u^{n-1}, ..., u^{n-K+1}
  float* out_a;        // lam^{n-K+1} (level K)
  float* out_b;        // mu^{n-K+1}
  float* gx;           // FP32 face-gradient accumulators
  float* gy;
  int rows;
  int64_t nstrips, ntiles;
  const int* rec_off;  // per tile [ntiles + 1], or nullptr
  const int4* rec;     // (row, col, receiver, 0)
  const float* g[K];   // g^n, g^{n-1}, ... at the receivers
};

template <int K>
__global__ void __launch_bounds__(kAwWarps * 32, aw_ctas_per_sm<K>()) k_adjoint_wtb(const AwArgs<K> a) {
  constexpr int NF = aw_fields<K>();
  constexpr int F_L1 = 0, F_MU = 1, F_HX = 2, F_HY = 3, F_U = 4;
  static_assert(K >= 2, "levels 1 and 2 read hx, hy from the ring, the others from registers");
  extern __shared__ __align__(16) unsigned char aw_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kAwWarps + warp;
  const bool tile_ok = tile < a.ntiles;
  const int64_t strip = tile_ok ? tile % a.nstrips : 0, chunk = tile_ok ? tile / a.nstrips : 0;
  const int64_t xs = strip * kAwOut - 8;  // first column read (lane 0, halo)
  const int64_t c0 = xs + 4 * lane;
  const int y0 = 1 + (int)chunk * a.rows;
  const int y1 = tile_ok ? min(y0 + a.rows, a.ny - 1) : y0;
  const int r_first = y0 - K, nit = tile_ok ? (y1 - y0) + 2 * K : 0;
  const bool col_in = c0 >= 0 && c0 < a.ld;
  const bool col_out = lane >= 1 && lane <= 30 && col_in;
  bool node_col[4], face_x[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    node_col[e] = (c0 + e >= 1) && (c0 + e <= a.nx - 2);
    face_x[e] = (c0 + e <= a.nx - 2);  // x-face (i, i+1) exists
  }
  // per-thread ring: [kAwRing][NF] float4; slot q & 3 holds what iteration q consumes, and the
  // previous slot stays valid through an iteration (the copies issued at iteration q fill slot
  // q + 2)
  float* ring = reinterpret_cast<float*>(aw_smem) + (size_t)threadIdx.x * 4;
  const int stride = kAwWarps * 32 * 4;
  auto slot = [&](unsigned s, int f) { return ring + (size_t)((s & (kAwRing - 1)) * NF + f) * stride; };
  // The first 2K input rows of a tile are the last rows the tile above reads, at its end: they
  // are copied with a priority to stay in the L2 until then.
  const uint64_t keep = l2_evict_last();
  auto issue = [&](int q) {  // the copies consumed at iteration q (input row r_first + q)
    const int r = r_first + q;
    auto copy = [&](int f, const float* src, int row) {
      const bool ok = col_in && row >= 0 && row < a.ny;
      const float* g = src + (ok ? (int64_t)row * a.ld + c0 : 0);
      if (q < 2 * K)
        cp16_hint(slot((unsigned)q, f), g, ok, keep);
      else
        cp16(slot((unsigned)q, f), g, ok);
    };
    copy(F_L1, a.lam1, r);
    copy(F_MU, a.mu1, r);
    copy(F_HX, a.hx, r - 1);
    copy(F_HY, a.hy, r - 1);
#pragma unroll
    for (int f = 0; f < K; ++f) copy(F_U + f, a.u[f], r - f);
  };
  // per-thread column constants (the columns of a thread never change): node and face masks
  // folded into the coefficients of the gradient terms
  f2x node2[2], gcx2[2], gcy2[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = 2 * q;
    node2[q] = pk(node_col[e] ? 1.f : 0.f, node_col[e + 1] ? 1.f : 0.f);
    gcx2[q] = pk(face_x[e] ? -a.cx : 0.f, face_x[e + 1] ? -a.cx : 0.f);
    gcy2[q] = pk(node_col[e] ? -a.cy : 0.f, node_col[e + 1] ? -a.cy : 0.f);
  }
  const f2x cx2 = pk(a.cx, a.cx), cy2 = pk(a.cy, a.cy);
  // register windows, index 0 = newest row.  Level 0 (lam^{n+1}, mu^{n+1}), u and the faces of
  // the two newest rows are read from the ring; what older rows the levels need is kept here.
  P4 W[K][2];       // lam of level k = 1..K-1 at rows r - k, r - k - 1
  P4 GP[K];         // GP[k - 1]: level k's y flux of lam at the faces below its current row
  P4 MW[K][2];      // mu of level k = 1..K-1 at rows r - k, r - k - 1
  P4 HXO[K], HYO[K];  // hx, hy at rows r - 3 .. r - K (index k - 1 for level k >= 3)
  P4 cx_[K], cy_[K];  // gradient sums of levels 1..j at the row level j + 1 reaches next
  P4 g0 = kZeroP4;    // y-face (0, 1) terms of the levels that have passed row 1
#pragma unroll
  for (int k = 0; k < K; ++k) {
    W[k][0] = W[k][1] = GP[k] = kZeroP4;
    MW[k][0] = MW[k][1] = kZeroP4;
    HXO[k] = HYO[k] = kZeroP4;
    cx_[k] = cy_[k] = kZeroP4;
  }

  const int q_lo = (tile_ok && a.rec_off) ? a.rec_off[tile] : 0, q_hi = (tile_ok && a.rec_off) ? a.rec_off[tile + 1] : 0;
  // the tile's first 32 receiver entries, one per lane (row -1: none), with their K values
  int pr_row = -1, pr_col = 0;
  float pr_g[K];
#pragma unroll
  for (int k = 0; k < K; ++k) pr_g[k] = 0.f;
  if (q_lo + lane < q_hi) {
    const int4 rq = a.rec[q_lo + lane];
    pr_row = rq.x;
    pr_col = rq.y;
#pragma unroll
    for (int k = 0; k < K; ++k) pr_g[k] = a.g[k][rq.z];
  }
  // add g^{n-k} (k = kg) at the entries on row p to the lane's four multipliers (warp-uniform
  // loop bounds; kg is a constant once the level loop is unrolled)
  auto inject = [&](int p, P4& l, const int kg) {
    for (int qb = q_lo; qb < q_hi; qb += 32) {
      int row = pr_row, col = pr_col;
      float val = pr_g[kg];
      if (qb != q_lo) {  // more than 32 entries: the rest from memory
        row = -1;
        if (qb + lane < q_hi) {
          const int4 rq = a.rec[qb + lane];
          row = rq.x;
          col = rq.y;
          val = a.g[kg][rq.z];
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, row == p);
      while (m) {
        const int src_lane = __ffs(m) - 1;
        m &= m - 1;
        const int c = __shfl_sync(0xffffffffu, col, src_lane);
        const float v = __shfl_sync(0xffffffffu, val, src_lane);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (c == c0 + e) {
            float2 x = upk(l.p[e >> 1]);
            if (e & 1)
              x.y += v;
            else
              x.x += v;
            l.p[e >> 1] = pk(x.x, x.y);
          }
        }
      }
    }
  };
  // One reverse step at a row: b = B lam and mu_out = mu + b on interior nodes (0 elsewhere), and
  // the face-gradient terms -cx (lam_{i+1} - lam_i)(u_{i+1} - u_i), -cy (lam_{j+1} - lam_j)
  // (u_{j+1} - u_j) of that step with the state u (rows: uc, uu = uc + 1 for lam; us, usu for u).
  // B lam in flux form, as the forward passes evaluate B u: each face's flux h (lam_right -
  // lam_left) once, the x flux left of the lane's first column from the lane on the left, the y
  // flux below the row carried in gp from the level's previous row; the lam differences are the
  // gradient terms' too.
  auto level = [&](const P4& uc, const P4& uu, const P4& hx, const P4& hyu, P4& gp, const P4& mu, const P4& us,
                   const P4& usu, const bool row_in, P4& mout, P4& gx, P4& gy) {
    const float2 c01 = upk(uc.p[0]), c23 = upk(uc.p[1]);
    const float2 s01 = upk(us.p[0]), s23 = upk(us.p[1]);
    const float ur = __shfl_down_sync(0xffffffffu, c01.x, 1);
    const float sr = __shfl_down_sync(0xffffffffu, s01.x, 1);
    // lam and u differences at the x faces right of the four columns
    const f2x dl[2] = {pk(__fsub_rn(c01.y, c01.x), __fsub_rn(c23.x, c01.y)),
                       pk(__fsub_rn(c23.y, c23.x), __fsub_rn(ur, c23.y))};
    const f2x du[2] = {pk(__fsub_rn(s01.y, s01.x), __fsub_rn(s23.x, s01.y)),
                       pk(__fsub_rn(s23.y, s23.x), __fsub_rn(sr, s23.y))};
    const f2x F01 = mul2(hx.p[0], dl[0]), F23 = mul2(hx.p[1], dl[1]);
    const float2 f01 = upk(F01), f23 = upk(F23);
    const float fl = __shfl_up_sync(0xffffffffu, f23.y, 1);
    const f2x fx[2] = {pk(__fsub_rn(f01.x, fl), __fsub_rn(f01.y, f01.x)),
                       pk(__fsub_rn(f23.x, f01.y), __fsub_rn(f23.y, f23.x))};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const f2x dy = sub2(uu.p[q], uc.p[q]);
      const f2x g = mul2(hyu.p[q], dy);
      const f2x b = fma2(cx2, fx[q], mul2(cy2, sub2(g, gp.p[q])));
      gp.p[q] = g;
      mout.p[q] = row_in ? mul2(add2(mu.p[q], b), node2[q]) : 0ull;
      gx.p[q] = mul2(gcx2[q], mul2(dl[q], du[q]));
      gy.p[q] = mul2(gcy2[q], mul2(dy, sub2(usu.p[q], us.p[q])));
    }
  };

  // One iteration: input row r_in = r_first + it; level k = 1..nl computes row r_in - k.  Level k
  // first matters at iteration 2k - 1 (its earlier rows lie above the cone of the tile's output
  // rows; the iteration before its first needed row yields the y flux below that row), so the
  // first 2K - 1 iterations run levels k <= (it + 1) / 2 only.
  auto iterate = [&](const int it, const int nl) {
    const int r_in = r_first + it;
    // hx, hy of row r - 3 leave the ring at this iteration's copies: keep them (and shift the
    // older rows) first
#pragma unroll
    for (int k = K - 1; k >= 3; --k) {
      HXO[k] = HXO[k - 1];
      HYO[k] = HYO[k - 1];
    }
    HXO[2] = lds_p4(slot((unsigned)(it - 2), F_HX));
    HYO[2] = lds_p4(slot((unsigned)(it - 2), F_HY));
    if (it + kAwPre < nit) issue(it + kAwPre);
    cp_commit();
    cp_wait<kAwPre>();
    const unsigned s = (unsigned)it, sp = (unsigned)(it - 1);
    P4 pend_x = kZeroP4, pend_y = kZeroP4;
#pragma unroll
    for (int k = 1; k <= K; ++k) {
      if (k > nl) continue;  // a constant once the loops are unrolled
      const int pk_row = r_in - k;
      // level k - 1 at rows r - k (centre) and r - k + 1; level 0 from the ring
      const P4 lc = k == 1 ? lds_p4(slot(sp, F_L1)) : W[k - 1][1];
      const P4 lu = k == 1 ? lds_p4(slot(s, F_L1)) : W[k - 1][0];
      const P4 mc = k == 1 ? lds_p4(slot(sp, F_MU)) : MW[k - 1][1];
      // u^{n-k+1} at rows r - k and r - k + 1 (copied at the previous and this iteration)
      const P4 us = lds_p4(slot(sp, F_U + k - 1)), usu = lds_p4(slot(s, F_U + k - 1));
      // hx, hy of row r - k: in the ring for k = 1, 2 (copied at iterations it, it - 1)
      const P4 hxk = k <= 2 ? lds_p4(slot((unsigned)(it - k + 1), F_HX)) : HXO[k - 1];
      const P4 hyk = k <= 2 ? lds_p4(slot((unsigned)(it - k + 1), F_HY)) : HYO[k - 1];
      P4 mk, gxk, gyk;
      level(lc, lu, hxk, hyk, GP[k - 1], mc, us, usu, pk_row >= 1 && pk_row <= a.ny - 2, mk, gxk, gyk);
      if (pk_row == 1) {  // y-face (0, 1): lam and u vanish on row 0, the term is -cy lam_1 u_1
#pragma unroll
        for (int q = 0; q < 2; ++q) g0.p[q] = add2(g0.p[q], mul2(gcy2[q], mul2(lc.p[q], us.p[q])));
      }
      inject(pk_row, mk, k - 1);  // g^m into mu^m (receivers are interior nodes)
      P4 lk;  // lam^m = lam^{m+1} + mu^m (0 wherever mu^m and lam^{m+1} are)
#pragma unroll
      for (int q = 0; q < 2; ++q) lk.p[q] = add2(lc.p[q], mk.p[q]);
      const bool store_row = col_out && pk_row >= y0 && pk_row < y1;
      if (k < K) {
        W[k][1] = W[k][0];
        W[k][0] = lk;
        MW[k][1] = MW[k][0];
        MW[k][0] = mk;
      }
      // gradient sums: level k adds to the sum of levels 1..k-1 at this row (carried from the
      // previous iteration); the new sum is kept until level k + 1 has read the old one
      P4 sx, sy;
      if (k == 1) {
        sx = gxk;
        sy = gyk;
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          sx.p[q] = add2(cx_[k - 1].p[q], gxk.p[q]);
          sy.p[q] = add2(cy_[k - 1].p[q], gyk.p[q]);
        }
        cx_[k - 1] = pend_x;
        cy_[k - 1] = pend_y;
      }
      if (k < K) {
        pend_x = sx;
        pend_y = sy;
      } else if (store_row) {
        const int64_t o = (int64_t)pk_row * a.ld + c0;
        stg_p4(a.out_a + o, lk);
        stg_p4(a.out_b + o, mk);
        red_add4(a.gx + o, sx);
        red_add4(a.gy + o, sy);
        if (pk_row == 1) red_add4(a.gy + c0, g0);  // y-face (0, 1) of all K steps
      }
    }
  };

  for (int q = 0; q < kAwPre; ++q) {
    if (q < nit) issue(q);
    cp_commit();
  }
  int it = 0;
  if (nit > 0) {  // every tile has nit >= 2K + 1 iterations
#pragma unroll
    for (int f = 0; f < 2 * K - 1; ++f) iterate(f, (f + 1) / 2);
    it = 2 * K - 1;
  }
#pragma unroll 1
  for (; it < nit; ++it) iterate(it, K);
  cp_wait<0>();
}

// Receivers of the K-step pass: for every tile whose extended region (columns 120 s - 8 ..
// 120 s + 119, rows y0 - (K - 1) .. y1 + (K - 2), where the levels before the last need the
// values) holds a receiver's interior node, one entry (row, col, r, 0), tiles in order,
// receivers in order within a tile (at most 4 per receiver).  One thread; nrec is small.
__global__ void k_rec_tiles(const int32_t nx, const int32_t ny, const int64_t ld, const int64_t* idx,
                            const int32_t nrec, const int rows, const int above, const int below,
                            const int64_t nstrips, const int64_t ntiles, int* off, int4* ent) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t nchunks = ntiles / nstrips;
  for (int64_t t = 0; t <= ntiles; ++t) off[t] = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int r = 0; r < nrec; ++r) {
      const int64_t q = idx[r];
      if (q < 0 || q >= (int64_t)ny * ld) continue;
      const int64_t j = q / ld, i = q - j * ld;
      if (!(i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2)) continue;
      const int64_t s_lo = (i + 8) / kAwOut - 1, c_lo = (j - 1) / rows - 1;
      for (int64_t sc = s_lo; sc <= s_lo + 2; ++sc) {
        if (sc < 0 || sc >= nstrips || i < sc * kAwOut - 8 || i >= sc * kAwOut + 120) continue;
        for (int64_t ch = c_lo; ch <= c_lo + 2; ++ch) {
          if (ch < 0 || ch >= nchunks) continue;
          const int64_t y0 = 1 + ch * rows, y1 = (y0 + rows < ny - 1) ? y0 + rows : ny - 1;
          if (j < y0 - above || j > y1 + below) continue;
          const int64_t t = ch * nstrips + sc;
          if (pass == 0)
            off[t + 1] += 1;
          else
            ent[off[t]++] = make_int4((int)j, (int)i, r, 0);
        }
      }
    }
    if (pass == 0) {
      for (int64_t t = 0; t < ntiles; ++t) off[t + 1] += off[t];
    } else {
      for (int64_t t = ntiles; t >= 1; --t) off[t] = off[t - 1];
      off[0] = 0;
    }
  }
}

template <int K>
cudaError_t aw_launch(const StencilGeom& g, int rows, const void* hx, const void* hy, const void* lam1,
                      const void* mu1, const void* const* u, void* out_a, void* out_b, void* gx, void* gy,
                      const int* rec_off, const int4* rec, const void* const* gv, cudaStream_t s);

}  // namespace

// Rows per chunk: the fewest that still fit all tiles into one wave (152 SMs x the resident CTAs
// of 4 warps), between 16 (halo rows cost (rows + 2K) / rows) and 64.  Tiles of a second, partly
// filled wave would leave most SMs idle while it runs.
int adjoint_wtb_rows(int k, int64_t ny, int64_t ld) {
  const int64_t strips = aw_nstrips(ld);
  const int64_t wave_tiles = (int64_t)152 * (k == 2 ? aw_ctas_per_sm<2>() : aw_ctas_per_sm<4>()) * kAwWarps;
  const int64_t chunks = wave_tiles / strips;
  if (chunks < 1) return 64;
  const int64_t rows = (ny - 2 + chunks - 1) / chunks;
  return (int)(rows < 16 ? 16 : rows > 64 ? 64 : rows);
}

int64_t adjoint_wtb_tiles(int64_t ny, int64_t ld, int rows) {
  return aw_nstrips(ld) * ((ny - 2 + rows - 1) / rows);
}

cudaError_t launch_rec_tiles(const StencilGeom& g, int k, const int64_t* idx, int32_t nrec, int rows, int* off,
                             int4* ent, cudaStream_t s) {
  const int64_t nstrips = aw_nstrips(g.ld);
  k_rec_tiles<<<1, 32, 0, s>>>(g.nx, g.ny, g.ld, idx, nrec, rows, k - 1, k - 2, nstrips,
                               adjoint_wtb_tiles(g.ny, g.ld, rows), off, ent);
  return cudaGetLastError();
}

namespace {
template <int K>
cudaError_t aw_launch(const StencilGeom& g, int rows, const void* hx, const void* hy, const void* lam1,
                      const void* mu1, const void* const* u, void* out_a, void* out_b, void* gx, void* gy,
                      const int* rec_off, const int4* rec, const void* const* gv, cudaStream_t s) {
  AwArgs<K> a;
  a.nx = g.nx;
  a.ny = g.ny;
  a.ld = g.ld;
  a.cx = (float)g.cx;
  a.cy = (float)g.cy;
  a.hx = (const float*)hx;
  a.hy = (const float*)hy;
  a.lam1 = (const float*)lam1;
  a.mu1 = (const float*)mu1;
  for (int f = 0; f < K; ++f) {
    a.u[f] = (const float*)u[f];
    a.g[f] = gv ? (const float*)gv[f] : nullptr;
  }
  a.out_a = (float*)out_a;
  a.out_b = (float*)out_b;
  a.gx = (float*)gx;
  a.gy = (float*)gy;
  a.rows = rows;
  a.nstrips = aw_nstrips(g.ld);
  a.ntiles = adjoint_wtb_tiles(g.ny, g.ld, rows);
  a.rec_off = rec_off;
  a.rec = rec;
  const size_t smem = (size_t)kAwRing * aw_fields<K>() * 16 * kAwWarps * 32;
  cudaError_t e = cudaFuncSetAttribute(k_adjoint_wtb<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_adjoint_wtb<K><<<(unsigned)((a.ntiles + kAwWarps - 1) / kAwWarps), kAwWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_adjoint_wtb(const StencilGeom& g, int k, int rows, const void* hx, const void* hy,
                               const void* lam1, const void* mu1, const void* const* u, void* out_lam, void* out_mu,
                               void* gx, void* gy, const int* rec_off, const int4* rec, const void* const* gv,
                               cudaStream_t s) {
  if (k == 2) return aw_launch<2>(g, rows, hx, hy, lam1, mu1, u, out_lam, out_mu, gx, gy, rec_off, rec, gv, s);
  if (k == 4) return aw_launch<4>(g, rows, hx, hy, lam1, mu1, u, out_lam, out_mu, gx, gy, rec_off, rec, gv, s);
  return cudaErrorInvalidValue;
}

}  // namespace tsu
