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

struct F4 {
  float a[4];
};
__device__ __forceinline__ F4 lds4(const float* s) {
  const float4 v = *reinterpret_cast<const float4*>(s);
  return F4{{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ void stg4(float* g, const F4& v) {
  *reinterpret_cast<float4*>(g) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
}
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
  const F4 Z{{0.f, 0.f, 0.f, 0.f}};
  const ArithF32 ar{a.cx, a.cy};
  // windows (index 0 = newest row)
  F4 w0[3] = {Z, Z, Z};      // lam^{n+1} rows r, r-1, r-2
  F4 w1[3] = {Z, Z, Z};      // lam^n rows r-1, r-2, r-3
  F4 L2[2] = {Z, Z};         // lam^{n+2} rows r, r-1
  F4 U[2] = {Z, Z};          // u^n rows r, r-1
  F4 M[3] = {Z, Z, Z};       // u^{n-1} rows r, r-1, r-2
  F4 HX[3] = {Z, Z, Z};      // hx rows r, r-1, r-2
  F4 HY[4] = {Z, Z, Z, Z};   // hy rows r .. r-3
  float gpx[4] = {0.f, 0.f, 0.f, 0.f}, gpy[4] = {0.f, 0.f, 0.f, 0.f};  // step n at the previous level-1 row
  float g0ya[4] = {0.f, 0.f, 0.f, 0.f};  // y-face (0, 1) of step n, carried to the level-2 row 1
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
  auto inject = [&](int p, F4& l, bool second) {
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
        for (int e = 0; e < 4; ++e)
          if (c == c0 + e) l.a[e] += v;
      }
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
    w0[2] = w0[1]; w0[1] = w0[0]; w0[0] = lds4(slot(s, 0));
    L2[1] = L2[0]; L2[0] = lds4(slot(s, 1));
    U[1] = U[0]; U[0] = lds4(slot(s, 2));
    M[2] = M[1]; M[1] = M[0]; M[0] = lds4(slot(s, 3));
    HX[2] = HX[1]; HX[1] = HX[0]; HX[0] = lds4(slot(s, 4));
    HY[3] = HY[2]; HY[2] = HY[1]; HY[1] = HY[0]; HY[0] = lds4(slot(s, 5));

    // ---- level 1: lam^n at row p1 = r_in - 1, and the face gradients of step n there
    const int p1 = r_in - 1;
    F4 l1;
    float g1x[4], g1y[4];
    {
      const F4 uc = w0[1], uu = w0[0], ud = w0[2];
      const float ul = __shfl_up_sync(0xffffffffu, uc.a[3], 1);
      const float ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
      const float hl = __shfl_up_sync(0xffffffffu, HX[1].a[3], 1);
      const float unr = __shfl_down_sync(0xffffffffu, U[1].a[0], 1);
      const bool row_in = p1 >= 1 && p1 <= a.ny - 2;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float xl = (e == 0) ? ul : uc.a[e - 1];
        const float xr = (e == 3) ? ur : uc.a[e + 1];
        const float hxl = (e == 0) ? hl : HX[1].a[e - 1];
        const float b = ar.b(HX[1].a[e], hxl, HY[1].a[e], HY[2].a[e], uc.a[e], xl, xr, uu.a[e], ud.a[e]);
        const float v = ar.lf(uc.a[e], L2[1].a[e], b);
        l1.a[e] = (row_in && node_col[e]) ? v : 0.f;
        const float uxr = (e == 3) ? unr : U[1].a[e + 1];
        g1x[e] = face_x[e] ? -a.cx * ((xr - uc.a[e]) * (uxr - U[1].a[e])) : 0.f;
        g1y[e] = node_col[e] ? -a.cy * ((uu.a[e] - uc.a[e]) * (U[0].a[e] - U[1].a[e])) : 0.f;
        if (p1 == 1) g0ya[e] = node_col[e] ? -a.cy * (uc.a[e] * U[1].a[e]) : 0.f;  // face (0, 1)
      }
    }
    inject(p1, l1, false);  // receivers on this row (extended region)
    w1[2] = w1[1]; w1[1] = w1[0]; w1[0] = l1;
    if (col_out && p1 >= y0 && p1 < y1) stg4(a.out1 + (int64_t)p1 * a.ld + c0, l1);

    // ---- level 2: lam^{n-1} at row p2 = r_in - 2, and the face gradients of step n-1 there
    const int p2 = r_in - 2;
    {
      const F4 uc = w1[1], uu = w1[0], ud = w1[2];
      const float ul = __shfl_up_sync(0xffffffffu, uc.a[3], 1);
      const float ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
      const float hl = __shfl_up_sync(0xffffffffu, HX[2].a[3], 1);
      const float umr = __shfl_down_sync(0xffffffffu, M[2].a[0], 1);
      const bool row_in = p2 >= 1 && p2 <= a.ny - 2;
      F4 l2;
      float g2x[4], g2y[4], g0b[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float xl = (e == 0) ? ul : uc.a[e - 1];
        const float xr = (e == 3) ? ur : uc.a[e + 1];
        const float hxl = (e == 0) ? hl : HX[2].a[e - 1];
        const float b = ar.b(HX[2].a[e], hxl, HY[2].a[e], HY[3].a[e], uc.a[e], xl, xr, uu.a[e], ud.a[e]);
        const float v = ar.lf(uc.a[e], w0[2].a[e], b);
        l2.a[e] = (row_in && node_col[e]) ? v : 0.f;
        const float uxr = (e == 3) ? umr : M[2].a[e + 1];
        g2x[e] = face_x[e] ? -a.cx * ((xr - uc.a[e]) * (uxr - M[2].a[e])) : 0.f;
        g2y[e] = node_col[e] ? -a.cy * ((uu.a[e] - uc.a[e]) * (M[1].a[e] - M[2].a[e])) : 0.f;
        g0b[e] = node_col[e] ? -a.cy * (uc.a[e] * M[2].a[e]) : 0.f;
      }
      inject(p2, l2, true);
      if (col_out && p2 >= y0 && p2 < y1) {
        const int64_t o = (int64_t)p2 * a.ld + c0;
        stg4(a.out2 + o, l2);
        // both steps' face gradients of row p2: step n was computed one iteration ago
        F4 ax = lds4(slot(s, 6)), ay = lds4(slot(s, 7));
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ax.a[e] += gpx[e] + g2x[e];
          ay.a[e] += gpy[e] + g2y[e];
        }
        stg4(a.gx + o, ax);
        stg4(a.gy + o, ay);
        if (p2 == 1) {  // y-face (0, 1): lam and u vanish on row 0
          const float4 r0 = __ldcg(reinterpret_cast<const float4*>(a.gy + c0));  // once per tile column
          F4 a0{{r0.x, r0.y, r0.z, r0.w}};
#pragma unroll
          for (int e = 0; e < 4; ++e) a0.a[e] += g0ya[e] + g0b[e];
          stg4(a.gy + c0, a0);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      gpx[e] = g1x[e];
      gpy[e] = g1y[e];
    }
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
