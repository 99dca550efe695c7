// Two adjoint steps per pass (the paper has no adjoint; this is the exact reverse of the scheme of
// k_step.cu, arXiv:2005.11931 Sec. 2 eq. (2.1) on the Sec. 3.3 box), warp-blocked like
// k_step_wtb.cu:
//   lam^n     = g^n     + 2 lam^{n+1} - lam^{n+2} + B lam^{n+1}
//   lam^{n-1} = g^{n-1} + 2 lam^n     - lam^{n+1} + B lam^n
//   dJ/dhx_ij += -cx [ (lam^{n+1}_{i+1}-lam^{n+1}_i)(u^n_{i+1}-u^n_i)
//                    + (lam^n_{i+1}  -lam^n_i  )(u^{n-1}_{i+1}-u^{n-1}_i) ]   (dJ/dhy likewise)
// Every warp owns a tile: 128 columns (one float4 per lane; the middle 120 are output, a
// 4-column halo covers the two-step cone) by a chunk of rows it streams down.  Each thread copies
// its own float4 of the six input rows (lam^{n+1}, lam^{n+2}, u^n, u^{n-1}, hx, hy) through a
// private cp.async ring; level 1 (lam^n) lags the input by one row, level 2 (lam^{n-1}) by two.
// The face gradients of both steps are added in registers, so the FP32 accumulators are read and
// written once per two steps; their rows travel through the same ring, two rows behind the
// inputs, so no load waits inside the row loop.  Receiver values g^n, g^{n-1} are added to the
// multipliers in registers, in every tile whose extended region holds the receiver (halo copies
// included): the lanes hold the tile's entries and a ballot per row finds the ones on it.
#include <string.h>

#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

constexpr int kAwWarps = 4;
constexpr int kAwOut = 120;
constexpr int kAwPre = 2;
constexpr int kAwRing = 4;  // slots per field: in flight (2) + current, power of two
constexpr int kAwFields = 8;  // lam^{n+1}, lam^{n+2}, u^n, u^{n-1}, hx, hy, then gx, gy two rows behind

__device__ __forceinline__ void cp16(void* smem, const void* gmem, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct AwArgs {
  int32_t nx, ny;
  int64_t ld;
  float cx, cy;
  const float* hx;
  const float* hy;
  const float* lam1;  // lam^{n+1}
  const float* lam2;  // lam^{n+2}
  const float* un;    // u^n
  const float* um;    // u^{n-1}
  float* out1;        // lam^n
  float* out2;        // lam^{n-1}
  float* gx;          // FP32 face-gradient accumulators
  float* gy;
  int rows;
  int64_t nstrips, ntiles;
  const int* rec_off;  // per tile [ntiles + 1], or nullptr
  const int4* rec;     // (row, col, receiver, 0)
  const float* g1;     // g^n at the receivers
  const float* g2;     // g^{n-1}
};

__global__ void __launch_bounds__(kAwWarps * 32) k_adjoint_wtb2(const AwArgs a) {
  extern __shared__ __align__(16) unsigned char aw_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile = (int64_t)blockIdx.x * kAwWarps + warp;
  const bool tile_ok = tile < a.ntiles;
  const int64_t strip = tile_ok ? tile % a.nstrips : 0, chunk = tile_ok ? tile / a.nstrips : 0;
  const int64_t xs = strip * kAwOut - 4;
  const int64_t c0 = xs + 4 * lane;
  const int y0 = 1 + (int)chunk * a.rows;
  const int y1 = tile_ok ? min(y0 + a.rows, a.ny - 1) : y0;
  const int r_first = y0 - 2, nit = tile_ok ? (y1 - y0) + 4 : 0;
  const bool col_in = c0 >= 0 && c0 < a.ld;
  const bool col_out = lane >= 1 && lane <= 30 && col_in;
  bool node_col[4], face_x[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    node_col[e] = (c0 + e >= 1) && (c0 + e <= a.nx - 2);
    face_x[e] = (c0 + e <= a.nx - 2);  // x-face (i, i+1) exists
  }
  // per-thread ring: [kAwRing][kAwFields] float4
  float* ring = reinterpret_cast<float*>(aw_smem) + (size_t)threadIdx.x * 4;
  const int stride = kAwWarps * 32 * 4;
  auto slot = [&](unsigned s, int f) { return ring + (size_t)(s * kAwFields + f) * stride; };
  const float* src[6] = {a.lam1, a.lam2, a.un, a.um, a.hx, a.hy};
  auto issue = [&](int r) {
    const bool ok = col_in && r >= 0 && r < a.ny;
    const int64_t go = ok ? (int64_t)r * a.ld + c0 : 0;
    const unsigned s = (unsigned)(r - r_first) & (kAwRing - 1);
#pragma unroll
    for (int f = 0; f < 6; ++f) cp16(slot(s, f), src[f] + go, ok);
    // accumulators of row r - 2, the row level 2 finishes when row r is consumed; only rows this
    // tile owns are read (no other tile writes them, and this tile writes each once)
    const bool acc = col_out && r - 2 >= y0 && r - 2 < y1;
    const int64_t ga = acc ? (int64_t)(r - 2) * a.ld + c0 : 0;
    cp16(slot(s, 6), a.gx + ga, acc);
    cp16(slot(s, 7), a.gy + ga, acc);
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
  // windows (index 0 = newest row)
  P4 w0[3] = {kZeroP4, kZeroP4, kZeroP4};  // lam^{n+1} rows r, r-1, r-2
  P4 w1[3] = {kZeroP4, kZeroP4, kZeroP4};  // lam^n rows r-1, r-2, r-3
  P4 L2[2] = {kZeroP4, kZeroP4};           // lam^{n+2} rows r, r-1
  P4 U[2] = {kZeroP4, kZeroP4};            // u^n rows r, r-1
  P4 M[3] = {kZeroP4, kZeroP4, kZeroP4};   // u^{n-1} rows r, r-1, r-2
  P4 HX[3] = {kZeroP4, kZeroP4, kZeroP4};  // hx rows r, r-1, r-2
  P4 HY[4] = {kZeroP4, kZeroP4, kZeroP4, kZeroP4};  // hy rows r .. r-3
  P4 gpx = kZeroP4, gpy = kZeroP4;  // face gradients of step n at the previous level-1 row
  P4 g0ya = kZeroP4;                // y-face (0, 1) of step n, carried to the level-2 row 1
  const int q_lo = (tile_ok && a.rec_off) ? a.rec_off[tile] : 0, q_hi = (tile_ok && a.rec_off) ? a.rec_off[tile + 1] : 0;
  // the tile's first 32 receiver entries, one per lane (row -1: none)
  int pr_row = -1, pr_col = 0;
  float pr_g1 = 0.f, pr_g2 = 0.f;
  if (q_lo + lane < q_hi) {
    const int4 rq = a.rec[q_lo + lane];
    pr_row = rq.x;
    pr_col = rq.y;
    pr_g1 = a.g1[rq.z];
    pr_g2 = a.g2[rq.z];
  }
  // add g at the entries on row p to the lane's four multipliers (warp-uniform loop bounds)
  auto inject = [&](int p, P4& l, bool second) {
    for (int qb = q_lo; qb < q_hi; qb += 32) {
      int row = pr_row, col = pr_col;
      float val = second ? pr_g2 : pr_g1;
      if (qb != q_lo) {  // more than 32 entries: the rest from memory
        row = -1;
        if (qb + lane < q_hi) {
          const int4 rq = a.rec[qb + lane];
          row = rq.x;
          col = rq.y;
          val = second ? a.g2[rq.z] : a.g1[rq.z];
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
  // One reverse step at a row: lam_out = (2 lam - lam_pp) + B lam on interior nodes (0 elsewhere),
  // and the face-gradient terms -cx (lam_{i+1} - lam_i)(u_{i+1} - u_i), -cy (lam_{j+1} - lam_j)
  // (u_{j+1} - u_j) of that step with the state u (rows: uc, uu = uc + 1 for lam; us, usu for u).
  auto level = [&](const P4& uc, const P4& uu, const P4& ud, const P4& hx, const P4& hyu, const P4& hyd,
                   const P4& lpp, const P4& us, const P4& usu, const bool row_in, P4& lout, P4& gx, P4& gy) {
    const float2 c01 = upk(uc.p[0]), c23 = upk(uc.p[1]);
    const float2 h01 = upk(hx.p[0]), h23 = upk(hx.p[1]);
    const float2 s01 = upk(us.p[0]), s23 = upk(us.p[1]);
    const float ul = __shfl_up_sync(0xffffffffu, c23.y, 1);
    const float ur = __shfl_down_sync(0xffffffffu, c01.x, 1);
    const float hl = __shfl_up_sync(0xffffffffu, h23.y, 1);
    const float sr = __shfl_down_sync(0xffffffffu, s01.x, 1);
    const f2x mid = pk(c01.y, c23.x), right1 = pk(c23.y, ur);
    const f2x lpair[2] = {pk(ul, c01.x), mid}, rpair[2] = {mid, right1};
    const f2x hlpair[2] = {pk(hl, h01.x), pk(h01.y, h23.x)};
    const f2x srpair[2] = {pk(s01.y, s23.x), pk(s23.y, sr)};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const f2x b = stencil2(hlpair[q], hx.p[q], hyd.p[q], hyu.p[q], uc.p[q], lpair[q], rpair[q], uu.p[q], ud.p[q],
                             cx2, cy2);
      const f2x v = add2(sub2(add2(uc.p[q], uc.p[q]), lpp.p[q]), b);  // (2 lam - lam_pp) + B lam
      lout.p[q] = row_in ? mul2(v, node2[q]) : 0ull;
      gx.p[q] = mul2(gcx2[q], mul2(sub2(rpair[q], uc.p[q]), sub2(srpair[q], us.p[q])));
      gy.p[q] = mul2(gcy2[q], mul2(sub2(uu.p[q], uc.p[q]), sub2(usu.p[q], us.p[q])));
    }
  };

  for (int q = 0; q < kAwPre; ++q) {
    if (q < nit) issue(r_first + q);
    cp_commit();
  }
  for (int it = 0; it < nit; ++it) {
    const int r_in = r_first + it;
    if (it + kAwPre < nit) issue(r_in + kAwPre);
    cp_commit();
    cp_wait<kAwPre>();
    const unsigned s = (unsigned)it & (kAwRing - 1);
    // shift histories and take the new row
    w0[2] = w0[1]; w0[1] = w0[0]; w0[0] = lds_p4(slot(s, 0));
    L2[1] = L2[0]; L2[0] = lds_p4(slot(s, 1));
    U[1] = U[0]; U[0] = lds_p4(slot(s, 2));
    M[2] = M[1]; M[1] = M[0]; M[0] = lds_p4(slot(s, 3));
    HX[2] = HX[1]; HX[1] = HX[0]; HX[0] = lds_p4(slot(s, 4));
    HY[3] = HY[2]; HY[2] = HY[1]; HY[1] = HY[0]; HY[0] = lds_p4(slot(s, 5));

    // ---- level 1: lam^n at row p1 = r_in - 1, and the face gradients of step n there
    const int p1 = r_in - 1;
    P4 l1, g1x, g1y;
    level(w0[1], w0[0], w0[2], HX[1], HY[1], HY[2], L2[1], U[1], U[0], p1 >= 1 && p1 <= a.ny - 2, l1, g1x, g1y);
    if (p1 == 1) {  // y-face (0, 1): lam and u vanish on row 0, the term is -cy lam_1 u_1
#pragma unroll
      for (int q = 0; q < 2; ++q) g0ya.p[q] = mul2(gcy2[q], mul2(w0[1].p[q], U[1].p[q]));
    }
    inject(p1, l1, false);  // receivers on this row (extended region)
    w1[2] = w1[1]; w1[1] = w1[0]; w1[0] = l1;
    if (col_out && p1 >= y0 && p1 < y1) stg_p4(a.out1 + (int64_t)p1 * a.ld + c0, l1);

    // ---- level 2: lam^{n-1} at row p2 = r_in - 2, and the face gradients of step n-1 there
    const int p2 = r_in - 2;
    P4 l2, g2x, g2y;
    level(w1[1], w1[0], w1[2], HX[2], HY[2], HY[3], w0[2], M[2], M[1], p2 >= 1 && p2 <= a.ny - 2, l2, g2x, g2y);
    inject(p2, l2, true);
    if (col_out && p2 >= y0 && p2 < y1) {
      const int64_t o = (int64_t)p2 * a.ld + c0;
      stg_p4(a.out2 + o, l2);
      // both steps' face gradients of row p2: step n was computed one iteration ago
      P4 ax = lds_p4(slot(s, 6)), ay = lds_p4(slot(s, 7));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        ax.p[q] = add2(ax.p[q], add2(gpx.p[q], g2x.p[q]));
        ay.p[q] = add2(ay.p[q], add2(gpy.p[q], g2y.p[q]));
      }
      stg_p4(a.gx + o, ax);
      stg_p4(a.gy + o, ay);
      if (p2 == 1) {  // y-face (0, 1) of both steps
        const ulonglong2 r0 = __ldcg(reinterpret_cast<const ulonglong2*>(a.gy + c0));  // once per tile column
        P4 a0{{r0.x, r0.y}};
#pragma unroll
        for (int q = 0; q < 2; ++q)
          a0.p[q] = add2(a0.p[q], add2(g0ya.p[q], mul2(gcy2[q], mul2(w1[1].p[q], M[2].p[q]))));
        stg_p4(a.gy + c0, a0);
      }
    }
    gpx = g1x;
    gpy = g1y;
  }
  cp_wait<0>();
}

// Receivers of the two-step pass: for every tile whose extended region (columns 120 s - 4 ..
// 120 s + 123, rows y0 - 1 .. y1) holds a receiver's interior node, one entry (row, col, r, 0),
// tiles in order, receivers in order within a tile.  One thread; nrec is small.
__global__ void k_rec_tiles(const int32_t nx, const int32_t ny, const int64_t ld, const int64_t* idx,
                            const int32_t nrec, const int rows, const int64_t nstrips, const int64_t ntiles, int* off,
                            int4* ent) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t nchunks = ntiles / nstrips;
  for (int64_t t = 0; t <= ntiles; ++t) off[t] = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int r = 0; r < nrec; ++r) {
      const int64_t q = idx[r];
      if (q < 0 || q >= (int64_t)ny * ld) continue;
      const int64_t j = q / ld, i = q - j * ld;
      if (!(i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2)) continue;
      const int64_t s_lo = (i + 4) / kAwOut - 1, c_lo = (j - 1) / rows - 1;
      for (int64_t sc = s_lo; sc <= s_lo + 2; ++sc) {
        if (sc < 0 || sc >= nstrips || i < sc * kAwOut - 4 || i >= sc * kAwOut + 124) continue;
        for (int64_t ch = c_lo; ch <= c_lo + 2; ++ch) {
          if (ch < 0 || ch >= nchunks) continue;
          const int64_t y0 = 1 + ch * rows, y1 = (y0 + rows < ny - 1) ? y0 + rows : ny - 1;
          if (j < y0 - 1 || j > y1) continue;
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

}  // namespace

// Rows per chunk: the fewest that still fit all tiles into one wave (152 SMs x 3 resident CTAs of
// 4 warps at 148 registers), between 16 (halo rows cost (rows + 4) / rows) and 64.  Tiles of a
// second, partly filled wave would leave most SMs idle while it runs.
int adjoint_wtb2_rows(int64_t ny, int64_t ld) {
  const int64_t strips = (ld + kAwOut - 1) / kAwOut;
  const int64_t wave_tiles = 152 * 3 * kAwWarps;
  const int64_t chunks = wave_tiles / strips;
  if (chunks < 1) return 64;
  const int64_t rows = (ny - 2 + chunks - 1) / chunks;
  return (int)(rows < 16 ? 16 : rows > 64 ? 64 : rows);
}

int64_t adjoint_wtb2_tiles(int64_t ny, int64_t ld, int rows) {
  return ((ld + kAwOut - 1) / kAwOut) * ((ny - 2 + rows - 1) / rows);
}

cudaError_t launch_rec_tiles(const StencilGeom& g, const int64_t* idx, int32_t nrec, int rows, int* off, int4* ent,
                             cudaStream_t s) {
  const int64_t nstrips = (g.ld + kAwOut - 1) / kAwOut;
  k_rec_tiles<<<1, 32, 0, s>>>(g.nx, g.ny, g.ld, idx, nrec, rows, nstrips, adjoint_wtb2_tiles(g.ny, g.ld, rows), off,
                               ent);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_wtb2(const StencilGeom& g, int rows, const void* hx, const void* hy, const void* lam1,
                                const void* lam2, const void* un, const void* um, void* out1, void* out2, void* gx,
                                void* gy, const int* rec_off, const int4* rec, const void* g1, const void* g2,
                                cudaStream_t s) {
  AwArgs a;
  a.nx = g.nx;
  a.ny = g.ny;
  a.ld = g.ld;
  a.cx = (float)g.cx;
  a.cy = (float)g.cy;
  a.hx = (const float*)hx;
  a.hy = (const float*)hy;
  a.lam1 = (const float*)lam1;
  a.lam2 = (const float*)lam2;
  a.un = (const float*)un;
  a.um = (const float*)um;
  a.out1 = (float*)out1;
  a.out2 = (float*)out2;
  a.gx = (float*)gx;
  a.gy = (float*)gy;
  a.rows = rows;
  a.nstrips = (g.ld + kAwOut - 1) / kAwOut;
  a.ntiles = adjoint_wtb2_tiles(g.ny, g.ld, rows);
  a.rec_off = rec_off;
  a.rec = rec;
  a.g1 = (const float*)g1;
  a.g2 = (const float*)g2;
  const size_t smem = (size_t)kAwRing * kAwFields * 16 * kAwWarps * 32;
  cudaError_t e = cudaFuncSetAttribute(k_adjoint_wtb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_adjoint_wtb2<<<(unsigned)((a.ntiles + kAwWarps - 1) / kAwWarps), kAwWarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace tsu
