// Implicit comparator (arXiv:2005.11931 Sec. 3.3: the 2D problem solved by an implicit scheme
// whose systems are tridiagonal along grid lines).  The scheme is read as the factorized scheme
// with weight s:
//   (I - s B_x)(I - s B_y) w^n = B u^n,   v^{n+1} = v^n + w^n,   u^{n+1} = u^n + v^{n+1},
// started by w^0 from B u^0 and v^1 = tau u1 + w^0 / 2, u^1 = u^0 + v^1.  B_x u = cx fx(u) and
// B_y u = cy fy(u) are the two halves of the explicit operator (flux form).
//
// Each factor is one tridiagonal system per grid line.  Their LU factors do not change in time,
// so the pivots are computed once (k_imp_factor_x / _y: m = 1 / pivot).  A step is then two
// passes, one per direction, each a forward and a backward substitution over every line:
//   forward   d_k = alpha_k d_{k-1} + beta_k,   alpha_k = s c h_{k-1/2} m_k, beta_k = m_k r_k
//   backward  z_k = gamma_k z_{k+1} + d_k,      gamma_k = s c h_{k+1/2} m_k
// Both are first-order linear recurrences, i.e. compositions of affine maps.  One warp owns a
// line and walks it in segments of 128 nodes (4 consecutive nodes per lane, one 16-byte load
// per field and lane): each lane composes its four maps, a 5-step warp scan (Kogge-Stone, by
// shuffles) composes the lanes' maps, and the value carried in from the previous segment turns
// them into the 128 results.  So every line is solved by 32 threads with coalesced loads instead
// of one thread, and the cyclic reduction of the paper's GPU code is not needed.
//
// The x pass (k_imp_x) reads rows of the row-major fields and computes r = B u^n on the way; the
// y pass (k_imp_y) needs columns, so the x pass writes its result z transposed (zT[i][j]) through
// a shared-memory tile of R rows x 128 columns, and the y pass reads rows of zT, then writes w
// back to row-major order through the same kind of tile, fused with the update of v and u.
// Forward results wait for the backward substitution in a global scratch line (mostly L2).
#include <cooperative_groups.h>
#include <string.h>

#include <atomic>

#include "async_copy.cuh"
#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

constexpr int kImpSeg = 128;  // nodes per warp segment
// the workspace starts with a header whose int at byte 4 is the status word (as for tsu_step_n)
constexpr size_t kImpWsHeader = 256;

template <typename T>
struct V4 {
  T a[4];
};
__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return V4<float>{{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 v0 = *reinterpret_cast<const double2*>(p);
  const double2 v1 = *reinterpret_cast<const double2*>(p + 2);
  return V4<double>{{v0.x, v0.y, v1.x, v1.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  *reinterpret_cast<double2*>(p) = make_double2(v.a[0], v.a[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v.a[2], v.a[3]);
}
template <typename T>
__device__ __forceinline__ V4<T> zero4() {
  return V4<T>{{T(0), T(0), T(0), T(0)}};
}

// explicitly rounded arithmetic (no contraction left to the compiler)
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// An affine map x -> A x + B, composed over a segment by a warp scan.  `up`: maps of lower lanes
// come first (forward substitution); otherwise higher lanes come first (backward).
template <typename T, bool UP>
__device__ __forceinline__ void warp_scan(T& A, T& B, const int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T A2 = UP ? __shfl_up_sync(0xffffffffu, A, off) : __shfl_down_sync(0xffffffffu, A, off);
    const T B2 = UP ? __shfl_up_sync(0xffffffffu, B, off) : __shfl_down_sync(0xffffffffu, B, off);
    if (UP ? lane >= off : lane + off < 32) {
      B = fma_(A, B2, B);
      A = mul_(A, A2);
    }
  }
}

// Solve x_e = c_e x_{prev} + d_e over the 4 nodes of each lane and the 32 lanes of a segment
// (node order e = 0..3, lane 0..31 when UP, the reverse otherwise), starting from `carry` (the
// value before the segment); returns the 4 results and updates carry to the segment's last.
template <typename T, bool UP>
__device__ __forceinline__ V4<T> segment_solve(const V4<T>& c, const V4<T>& d, T& carry, const int lane) {
  T A = T(1), B = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = UP ? q : 3 - q;
    B = fma_(c.a[e], B, d.a[e]);
    A = mul_(c.a[e], A);
  }
  warp_scan<T, UP>(A, B, lane);
  // the value entering this lane: the scanned map of the neighbour before it applied to carry
  const T A1 = UP ? __shfl_up_sync(0xffffffffu, A, 1) : __shfl_down_sync(0xffffffffu, A, 1);
  const T B1 = UP ? __shfl_up_sync(0xffffffffu, B, 1) : __shfl_down_sync(0xffffffffu, B, 1);
  const bool first = UP ? lane == 0 : lane == 31;
  T x = first ? carry : fma_(A1, carry, B1);
  V4<T> out;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = UP ? q : 3 - q;
    x = fma_(c.a[e], x, d.a[e]);
    out.a[e] = x;
  }
  carry = __shfl_sync(0xffffffffu, x, UP ? 31 : 0);
  return out;
}

// segment_solve over the NS segments of a whole line (segment 0 first when UP, NS - 1 first
// otherwise), starting from 0.  The segments' warp scans do not depend on one another, so they
// run interleaved; only the carries pass from segment to segment.  Every result rounds exactly as
// in NS calls of segment_solve.
template <typename T, bool UP, int NS>
__device__ __forceinline__ void line_solve(const V4<T> (&c)[NS], const V4<T> (&d)[NS], V4<T> (&out)[NS],
                                           const int lane) {
  T A[NS], B[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A[s] = T(1);
    B[s] = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = UP ? q : 3 - q;
      B[s] = fma_(c[s].a[e], B[s], d[s].a[e]);
      A[s] = mul_(c[s].a[e], A[s]);
    }
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const T A2 = UP ? __shfl_up_sync(0xffffffffu, A[s], off) : __shfl_down_sync(0xffffffffu, A[s], off);
      const T B2 = UP ? __shfl_up_sync(0xffffffffu, B[s], off) : __shfl_down_sync(0xffffffffu, B[s], off);
      if (UP ? lane >= off : lane + off < 32) {
        B[s] = fma_(A[s], B2, B[s]);
        A[s] = mul_(A[s], A2);
      }
    }
  }
  T A1[NS], B1[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    A1[s] = UP ? __shfl_up_sync(0xffffffffu, A[s], 1) : __shfl_down_sync(0xffffffffu, A[s], 1);
    B1[s] = UP ? __shfl_up_sync(0xffffffffu, B[s], 1) : __shfl_down_sync(0xffffffffu, B[s], 1);
  }
  const bool first = UP ? lane == 0 : lane == 31;
  T carry = T(0);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int s = UP ? k : NS - 1 - k;
    T x = first ? carry : fma_(A1[s], carry, B1[s]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = UP ? q : 3 - q;
      x = fma_(c[s].a[e], x, d[s].a[e]);
      out[s].a[e] = x;
    }
    if (k + 1 < NS) carry = __shfl_sync(0xffffffffu, x, UP ? 31 : 0);
  }
}

// The coefficients of one segment's recurrences, shared by every kernel that solves the lines
// (so that all of them round alike).  x pass, forward: r = B u in flux form over the lane's four
// nodes (rows uc, uu = row + 1, ud = row - 1; faces hxv, hyu above and hyd below; pivots m), with
// the neighbours across the lane's edges (ul, hl: node and face before it; ur: node after it);
// alpha_k = s cx h_{k-1/2} m_k, beta_k = m_k r_k, both 0 off the unknowns (m = 0 there).
template <typename T>
__device__ __forceinline__ void imp_x_coeffs(const T cx, const T cy, const T sx, const V4<T>& uc, const V4<T>& uu,
                                             const V4<T>& ud, const V4<T>& hxv, const V4<T>& hyu, const V4<T>& hyd,
                                             const V4<T>& m, const T ul, const T hl, const T ur, V4<T>& alpha,
                                             V4<T>& beta) {
  T fl = mul_(hl, sub_(uc.a[0], ul));  // x flux left of the lane's first node
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const T right = e < 3 ? uc.a[e + 1] : ur;
    const T fr = mul_(hxv.a[e], sub_(right, uc.a[e]));
    const T fx = sub_(fr, fl);
    const T fy = sub_(mul_(hyu.a[e], sub_(uu.a[e], uc.a[e])), mul_(hyd.a[e], sub_(uc.a[e], ud.a[e])));
    const T r = fma_(cx, fx, mul_(cy, fy));
    const T hprev = e == 0 ? hl : hxv.a[e - 1];
    const bool unk = m.a[e] != T(0);
    alpha.a[e] = unk ? mul_(mul_(sx, hprev), m.a[e]) : T(0);
    beta.a[e] = unk ? mul_(m.a[e], r) : T(0);
    fl = fr;
  }
}
// x pass, backward: gamma_k = s cx h_{k+1/2} m_k
template <typename T>
__device__ __forceinline__ V4<T> imp_x_gamma(const T sx, const V4<T>& m, const V4<T>& hxv) {
  V4<T> gamma;
#pragma unroll
  for (int e = 0; e < 4; ++e) gamma.a[e] = m.a[e] != T(0) ? mul_(mul_(sx, hxv.a[e]), m.a[e]) : T(0);
  return gamma;
}
// y pass, forward: z = the x pass's result along the column, k = s cy hy (kl: the face before the
// lane's first node)
template <typename T>
__device__ __forceinline__ void imp_y_coeffs(const V4<T>& z, const V4<T>& m, const V4<T>& k, const T kl,
                                             V4<T>& alpha, V4<T>& beta) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const T kprev = e == 0 ? kl : k.a[e - 1];
    const bool unk = m.a[e] != T(0);
    alpha.a[e] = unk ? mul_(kprev, m.a[e]) : T(0);
    beta.a[e] = unk ? mul_(m.a[e], z.a[e]) : T(0);
  }
}
// y pass, backward
template <typename T>
__device__ __forceinline__ V4<T> imp_y_gamma(const V4<T>& m, const V4<T>& k) {
  V4<T> gamma;
#pragma unroll
  for (int e = 0; e < 4; ++e) gamma.a[e] = m.a[e] != T(0) ? mul_(k.a[e], m.a[e]) : T(0);
  return gamma;
}

template <typename T>
struct ImpArgs {
  int32_t nx, ny;
  int64_t ld, ldT;
  T cx, cy, sx;      // tau^2/dx^2, tau^2/dy^2, s cx
  T tau;
  const T* hx;
  const T* hy;
  const T* mx;       // [ny][ld]  1 / pivot of the x systems (0 off the unknowns)
  const T* myT;      // [nx][ldT] 1 / pivot of the y systems
  const T* kyT;      // [nx][ldT] s cy hy (face j+1/2 of column i)
  const T* u;        // u^n (read by the x pass)
  T* zT;             // [nx][ldT] (I - s B_x)^{-1} B u^n, transposed
  T* scratch;        // forward results, one line per warp
  T* v;              // updated in place by the y pass
  T* uo;             // updated in place by the y pass
  const T* u1;       // start only: initial velocity or nullptr
  int* status;       // status word of the workspace (TSU_ETIMEOUT when a bounded wait ran out)
  int start;
};

// x pass: one warp per row j; R rows per CTA.  NS > 0: lines of at most NS segments (small
// grids) keep each segment's forward results, pivots and faces in registers (the loops unrolled,
// so the next segment's loads are issued ahead of this one's scan) and the backward substitution
// reads nothing back from memory; NS = 0: any length, forward results through the scratch line.
template <typename T, int R, int NS>
__global__ void __launch_bounds__(R * 32) k_imp_x(const ImpArgs<T> a) {
  __shared__ T tile[R][kImpSeg + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j0 = blockIdx.x * R, j = j0 + w;
  const bool row_in = j >= 1 && j <= a.ny - 2;  // rows with unknowns
  const int nseg = (a.nx - 1 + kImpSeg - 1) / kImpSeg;
  const int64_t base = (int64_t)j * a.ld;
  T* line = a.scratch + (row_in ? base : 0);
  // forward: r = B u, then d_k = alpha_k d_{k-1} + beta_k
  T carry = T(0), cu = T(0), ch = T(0);  // d, u and hx at the node before the segment
  auto forward = [&](const int s, V4<T>& d, V4<T>& m, V4<T>& hxv) {
    const int64_t c0 = (int64_t)s * kImpSeg + 4 * lane;
    const bool in = row_in && c0 < a.ld;
    V4<T> uc = zero4<T>(), uu = zero4<T>(), ud = zero4<T>(), hyu = zero4<T>(), hyd = zero4<T>();
    m = zero4<T>();
    hxv = zero4<T>();
    T ur_own = T(0);
    if (in) {
      uc = ld4(a.u + base + c0);
      uu = ld4(a.u + base + a.ld + c0);
      ud = ld4(a.u + base - a.ld + c0);
      hxv = ld4(a.hx + base + c0);
      hyu = ld4(a.hy + base + c0);
      hyd = ld4(a.hy + base - a.ld + c0);
      m = ld4(a.mx + base + c0);
      if (lane == 31 && c0 + 4 < a.ld) ur_own = a.u[base + c0 + 4];
    }
    T ul = __shfl_up_sync(0xffffffffu, uc.a[3], 1), hl = __shfl_up_sync(0xffffffffu, hxv.a[3], 1);
    T ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
    if (lane == 0) {
      ul = cu;
      hl = ch;
    }
    if (lane == 31) ur = ur_own;
    V4<T> alpha, beta;
    imp_x_coeffs(a.cx, a.cy, a.sx, uc, uu, ud, hxv, hyu, hyd, m, ul, hl, ur, alpha, beta);
    d = segment_solve<T, true>(alpha, beta, carry, lane);
    cu = __shfl_sync(0xffffffffu, uc.a[3], 31);
    ch = __shfl_sync(0xffffffffu, hxv.a[3], 31);
  };
  // backward: z_k = gamma_k z_{k+1} + d_k, written transposed through the tile
  auto backward = [&](const int s, const V4<T>& d, const V4<T>& m, const V4<T>& hxv) {
    const V4<T> z = segment_solve<T, false>(imp_x_gamma(a.sx, m, hxv), d, carry, lane);
#pragma unroll
    for (int e = 0; e < 4; ++e) tile[w][4 * lane + e] = z.a[e];
    __syncthreads();
    // column c of the segment, rows j0 .. j0 + R - 1: R consecutive elements of zT
    for (int q = threadIdx.x; q < kImpSeg * R; q += R * 32) {
      const int cc = q / R, rr = q - cc * R;
      const int64_t c = (int64_t)s * kImpSeg + cc;
      if (c < a.nx) a.zT[c * a.ldT + j0 + rr] = tile[rr][cc];
    }
    __syncthreads();
  };
  if constexpr (NS > 0) {
    V4<T> dk[NS], mk[NS], hk[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s < nseg) forward(s, dk[s], mk[s], hk[s]);
    carry = T(0);
#pragma unroll
    for (int s = NS - 1; s >= 0; --s)
      if (s < nseg) backward(s, dk[s], mk[s], hk[s]);
  } else {
    for (int s = 0; s < nseg; ++s) {
      V4<T> d, m, hxv;
      forward(s, d, m, hxv);
      const int64_t c0 = (int64_t)s * kImpSeg + 4 * lane;
      if (row_in && c0 < a.ld) st4(line + c0, d);
    }
    carry = T(0);
    for (int s = nseg - 1; s >= 0; --s) {
      const int64_t c0 = (int64_t)s * kImpSeg + 4 * lane;
      V4<T> d = zero4<T>(), m = zero4<T>(), hxv = zero4<T>();
      if (row_in && c0 < a.ld) {
        d = ld4(line + c0);
        m = ld4(a.mx + base + c0);
        hxv = ld4(a.hx + base + c0);
      }
      backward(s, d, m, hxv);
    }
  }
}

// y pass: one warp per column i (a row of zT); R columns per CTA; w written back row-major and
// folded into v and u.  Each segment's fields are loaded one segment ahead, and the v and u each
// thread updates after a segment's scan are read before the scan (4096^2 FP32: 136 against 239
// us per pass).  The x pass does not load ahead: at 72 registers instead of 48 it ran slower.
// NS > 0: columns of at most NS segments keep the forward results and coefficients in registers,
// as in the x pass.
template <typename T, int R, int NS>
__global__ void __launch_bounds__(R * 32) k_imp_y(const ImpArgs<T> a) {
  constexpr int kPer = kImpSeg * R / (R * 32);  // tile entries each thread writes back: 4
  __shared__ T tile[R][kImpSeg + 1];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * R, i = i0 + wp;
  const bool col_in = i >= 1 && i <= a.nx - 2;
  const int nseg = (a.ny - 1 + kImpSeg - 1) / kImpSeg;
  const int64_t base = (int64_t)i * a.ldT;
  T* line = a.scratch + (col_in ? base : 0);
  auto load3 = [&](int s, const T* first, V4<T>& x, V4<T>& m, V4<T>& k) {
    x = m = k = zero4<T>();
    const int64_t c0 = (int64_t)s * kImpSeg + 4 * lane;
    if (s >= 0 && s < nseg && col_in && c0 < a.ldT) {
      x = ld4(first + c0);
      m = ld4(a.myT + base + c0);
      k = ld4(a.kyT + base + c0);
    }
  };
  T carry = T(0), ck = T(0);  // d and s cy hy at the node before the segment
  auto forward = [&](const V4<T>& z, const V4<T>& m, const V4<T>& k) {
    T kl = __shfl_up_sync(0xffffffffu, k.a[3], 1);
    if (lane == 0) kl = ck;
    V4<T> alpha, beta;
    imp_y_coeffs(z, m, k, kl, alpha, beta);
    const V4<T> d = segment_solve<T, true>(alpha, beta, carry, lane);
    ck = __shfl_sync(0xffffffffu, k.a[3], 31);
    return d;
  };
  auto backward = [&](const int s, const V4<T>& d, const V4<T>& m, const V4<T>& k) {
    // the nodes this thread updates after the scan (row jj, column ii of the tile), read now
    T vq[kPer], uq[kPer], u1q[kPer];
    int64_t oq[kPer];
#pragma unroll
    for (int p = 0; p < kPer; ++p) {
      const int q = threadIdx.x + p * R * 32;
      const int cc = q / R, rr = q - cc * R;
      const int jj = s * kImpSeg + cc, ii = i0 + rr;
      const bool node = jj >= 1 && jj <= a.ny - 2 && ii >= 1 && ii <= a.nx - 2;
      oq[p] = node ? (int64_t)jj * a.ld + ii : -1;
      vq[p] = uq[p] = u1q[p] = T(0);
      if (node) {
        uq[p] = a.uo[oq[p]];
        if (a.start)
          u1q[p] = a.u1 ? a.u1[oq[p]] : T(0);
        else
          vq[p] = a.v[oq[p]];
      }
    }
    const V4<T> wv = segment_solve<T, false>(imp_y_gamma(m, k), d, carry, lane);
#pragma unroll
    for (int e = 0; e < 4; ++e) tile[wp][4 * lane + e] = wv.a[e];
    __syncthreads();
    // row j of the segment, columns i0 .. i0 + R - 1: v += w (or the start), u += v
#pragma unroll
    for (int p = 0; p < kPer; ++p) {
      if (oq[p] < 0) continue;
      const int q = threadIdx.x + p * R * 32;
      const int cc = q / R, rr = q - cc * R;
      const T wt = tile[rr][cc];
      const T vn = a.start ? fma_(a.tau, u1q[p], mul_(T(0.5), wt)) : vq[p] + wt;
      a.v[oq[p]] = vn;
      a.uo[oq[p]] = uq[p] + vn;
    }
    __syncthreads();
  };
  if constexpr (NS > 0) {
    V4<T> dk[NS], mk[NS], kk[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s < nseg) {
        V4<T> z;
        load3(s, a.zT + base, z, mk[s], kk[s]);
        dk[s] = forward(z, mk[s], kk[s]);
      }
    carry = T(0);
#pragma unroll
    for (int s = NS - 1; s >= 0; --s)
      if (s < nseg) backward(s, dk[s], mk[s], kk[s]);
  } else {
    V4<T> z, m, k;
    load3(0, a.zT + base, z, m, k);
    for (int s = 0; s < nseg; ++s) {
      V4<T> nz, nm, nk;
      load3(s + 1, a.zT + base, nz, nm, nk);
      const int64_t c0 = (int64_t)s * kImpSeg + 4 * lane;
      const V4<T> d = forward(z, m, k);
      if (col_in && c0 < a.ldT) st4(line + c0, d);
      z = nz;
      m = nm;
      k = nk;
    }
    carry = T(0);
    V4<T> d;
    load3(nseg - 1, line, d, m, k);
    for (int s = nseg - 1; s >= 0; --s) {
      V4<T> nd, nm, nk;
      load3(s - 1, line, nd, nm, nk);
      backward(s, d, m, k);
      d = nd;
      m = nm;
      k = nk;
    }
  }
}

// ---- every step of a small grid in one cluster (FP32, at most 256 x 256 nodes) -------------------
// The fields of such a grid fit in the shared memory of one cluster of NC = 8 CTAs (lines of at
// most 129 nodes, one segment) or NC = 16 (at most 256 nodes, two segments).  CTA c owns rows
// 16 c .. 16 c + 15 (their u and v in shared memory; faces and x pivots in the registers of the
// warps solving them) and columns 16 c .. 16 c + 15 (y pivots and coefficients in registers, the
// x pass's result along them in shared memory), read from memory once.  It also keeps copies of
// the two rows next to its edge rows (u in shared memory, v in registers), updated as their
// owners update them.  One step: the update v += w, u += v of the own and the copied rows from
// the previous step's w; the x pass (warp w solves row 16 c + w and stores each result into the
// CTA owning its column); the y pass (warp w solves column 16 c + w and stores each w into the
// CTA owning its row and, for edge rows, into the neighbour holding the copy).
//
// Every hand-over is an asynchronous store into the receiver's shared memory that completes its
// bytes on one of the receiver's two barriers (zb and wb received), so there is no cluster-wide
// barrier and no fence in the loop: a CTA waits only for the bytes it needs, and knows how many
// from the shape (every CTA's rows and columns lie in the solved segments; a line of NS segments
// is solved whole, the nodes beyond the grid are zeros and add exact zeros).  The bytes of the
// next step cannot arrive early: a CTA stores into zb of step n + 1 only after its own wb of
// step n, which needs every CTA's y pass of step n, i.e. every zb of step n read.
//
// The arithmetic is that of k_imp_x / k_imp_y (imp_x_coeffs ... segment_solve), so the states equal
// those of the two-kernel steps bit for bit; the launches, not memory, had bounded those on small
// grids (Table 1 run at 256^2: 3.3 us per pass).
constexpr int kCluLines = 16, kCluLen = 256;
// The x pass's results for the CTA's 16 columns, zb[j][.] (every row j of the grid), and the y
// pass's results for its 16 rows, wb[i][.] (every column i): a lane hands over the four values of
// its four consecutive nodes, which fall in one owner's 16 lines, as one 16-byte store.  The
// four 16-byte chunks of a line are swizzled by bits 3-4 of the other index (clu_pos), so that
// a warp reading one line's values across 32 lanes (4 rows apart) meets at most 4-way bank
// conflicts (rows 20 floats apart).
constexpr int kCluGroup = 20;
struct CluSmem {
  float u[kCluLines][kCluLen];
  float zb[kCluLen][kCluGroup], wb[kCluLen][kCluGroup];
  // the rows next to the edge rows (h = 0: row 16 c - 1, h = 1: row 16 c + 16); the w of each
  // comes in the 16-byte chunk of four rows that holds it (as its last row for h = 0, its first
  // for h = 1)
  float uh[2][kCluLen], wbh[2][kCluLen][4];
  uint64_t full[2];  // zb, wb (with wbh) of the current step received
};
constexpr uint64_t kCluWaitNs = 2000000000ull;  // bound of every wait (a step takes microseconds)

// offset of line q (0..15 within the owner) in entry n of zb / wb
__device__ __forceinline__ int clu_pos(const int n, const int q) {
  return ((((q >> 2) ^ (n >> 3)) & 3) << 2) | (q & 3);
}

template <int NC>
__global__ void __launch_bounds__(kCluLines * 32, 1) k_imp_cluster(const ImpArgs<float> a, const int64_t nsteps) {
  constexpr int NS = NC / 8;  // segments of kImpSeg nodes per line
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char clu_raw[];
  CluSmem& sm = *reinterpret_cast<CluSmem*>(clu_raw);
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int j0 = rank * kCluLines, i0 = rank * kCluLines;
  const int nth = blockDim.x;
  if (threadIdx.x == 0) {
    mbar_init(&sm.full[0], 1);
    mbar_init(&sm.full[1], 1);
    fence_barrier_init();
  }
  // the CTA's part of the grid, zeros beyond the grid; a start call (a.start) reads u^0 = u0 on
  // the interior nodes and 0 on the boundary, with v^0 = 0
  const bool first = a.start != 0;
  auto u_at = [&](const int jj, const int c) -> float {
    const bool take = jj >= 0 && jj < a.ny && c < a.ld &&
                      (!first || (jj >= 1 && jj <= a.ny - 2 && c >= 1 && c <= a.nx - 2));
    return take ? a.u[(int64_t)jj * a.ld + c] : 0.f;
  };
  {  // the loads first, then the stores: one round trip to memory
    float uv[kCluLen / 32];
#pragma unroll
    for (int k = 0; k < kCluLen / 32; ++k) {
      const int q = threadIdx.x + k * kCluLines * 32;
      uv[k] = u_at(j0 + q / kCluLen, q % kCluLen);
    }
#pragma unroll
    for (int k = 0; k < kCluLen / 32; ++k) {
      const int q = threadIdx.x + k * kCluLines * 32;
      sm.u[q / kCluLen][q % kCluLen] = uv[k];
    }
  }
  for (int q = threadIdx.x; q < kCluLen * kCluGroup; q += nth) {
    (&sm.zb[0][0])[q] = 0.f;
    (&sm.wb[0][0])[q] = 0.f;
  }
  for (int q = threadIdx.x; q < 2 * kCluLen; q += nth) {
    const int h = q / kCluLen, c = q - h * kCluLen;
    const int j = h == 0 ? j0 - 1 : j0 + kCluLines;
    sm.uh[h][c] = u_at(j, c);
    sm.wbh[h][c][0] = sm.wbh[h][c][1] = sm.wbh[h][c][2] = sm.wbh[h][c][3] = 0.f;
  }
  // bytes received per step: the x pass of each of the NC * 16 rows hands over 16 columns (64 B),
  // the y pass of each column 16 rows (64 B) and, per copied row, the 16-byte chunk holding its w
  const uint32_t zbytes = NC * kCluLines * 64;
  const uint32_t wbytes = NC * kCluLines * 64 + ((rank > 0 ? 1 : 0) + (rank + 1 < NC ? 1 : 0)) * NC * kCluLines * 16;
  const int j = j0 + wp, i = i0 + wp;
  const bool row_in = j >= 1 && j <= a.ny - 2, col_in = i >= 1 && i <= a.nx - 2;
  // What does not change from step to step stays in registers: the lane's faces and pivots of
  // row j (x pass; hxl: the face before the lane's first node) and of column i (y pass; kyl
  // likewise), zeros off the solved lines and beyond the grid.
  V4<float> hxk[NS], hyu[NS], hyd[NS], mxk[NS], myk[NS], kyk[NS];
  float hxl[NS], kyl[NS];
  {
    float ch = 0.f, ck = 0.f;
#pragma unroll
    for (int sg = 0; sg < NS; ++sg) {
      const int c0 = sg * kImpSeg + 4 * lane;
      hxk[sg] = hyu[sg] = hyd[sg] = mxk[sg] = myk[sg] = kyk[sg] = zero4<float>();
      if (row_in && c0 < a.ld) {
        const int64_t o = (int64_t)j * a.ld + c0;
        hxk[sg] = ld4(a.hx + o);
        hyu[sg] = ld4(a.hy + o);
        hyd[sg] = ld4(a.hy + o - a.ld);
        mxk[sg] = ld4(a.mx + o);
      }
      if (col_in && c0 < a.ldT) {
        const int64_t t = (int64_t)i * a.ldT + c0;
        myk[sg] = ld4(a.myT + t);
        kyk[sg] = ld4(a.kyT + t);
      }
      hxl[sg] = __shfl_up_sync(0xffffffffu, hxk[sg].a[3], 1);
      kyl[sg] = __shfl_up_sync(0xffffffffu, kyk[sg].a[3], 1);
      if (lane == 0) {
        hxl[sg] = ch;
        kyl[sg] = ck;
      }
      ch = __shfl_sync(0xffffffffu, hxk[sg].a[3], 31);
      ck = __shfl_sync(0xffffffffu, kyk[sg].a[3], 31);
    }
  }
  // v += w, u += v on the interior nodes of the own rows and of the two copied rows (the previous
  // step's y pass left w in wb and wbh).  Thread t takes rows 4 g .. 4 g + 3 of column c (g, c
  // from t and t + 512), whose v it holds in registers: their four w are one 16-byte chunk of wb,
  // read whole (8 lanes a wavefront), and lanes along c read u without bank conflicts; then column
  // ch of copied row h (from t), whose v it holds too.
  const int hh = threadIdx.x / kCluLen, ch = threadIdx.x - hh * kCluLen;
  const int jh = hh == 0 ? j0 - 1 : j0 + kCluLines;
  V4<float> vk[2];
  float vhk = (!first && jh >= 0 && jh < a.ny && ch < a.ld) ? a.v[(int64_t)jh * a.ld + ch] : 0.f;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int q = threadIdx.x + k * kCluLines * 32;
    const int g = q / kCluLen, c = q - g * kCluLen;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j0 + 4 * g + e;
      vk[k].a[e] = (!first && jj < a.ny && c < a.ld) ? a.v[(int64_t)jj * a.ld + c] : 0.f;
    }
  }
  cl.sync();  // every CTA's barriers initialised and buffers filled before the first store
  // START: the start rule v = tau u1 + w / 2 instead of v += w (own rows only: a start call is
  // one step, the copied rows are not read again)
  auto update = [&](const bool START) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int q = threadIdx.x + k * kCluLines * 32;
      const int g = q / kCluLen, c = q - g * kCluLen;
      if (c < 1 || c > a.nx - 2) continue;
      const V4<float> w = ld4(&sm.wb[c][clu_pos(c, 4 * g)]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 4 * g + e, jj = j0 + r;
        if (jj >= 1 && jj <= a.ny - 2) {
          if (START) {
            const float u1 = a.u1 ? a.u1[(int64_t)jj * a.ld + c] : 0.f;
            vk[k].a[e] = fma_(a.tau, u1, mul_(0.5f, w.a[e]));
          } else {
            vk[k].a[e] = vk[k].a[e] + w.a[e];
          }
          sm.u[r][c] = sm.u[r][c] + vk[k].a[e];
        }
      }
    }
    if (jh >= 1 && jh <= a.ny - 2 && ch >= 1 && ch <= a.nx - 2) {
      vhk = vhk + sm.wbh[hh][ch][hh == 0 ? 3 : 0];
      sm.uh[hh][ch] = sm.uh[hh][ch] + vhk;
    }
  };
  bool dead = false;  // a wait ran out: stop and report TSU_ETIMEOUT
  for (int64_t n = 0; n < nsteps; ++n) {
    if (n > 0) {
      if (!dead) dead = !mbar_wait_bounded<true>(&sm.full[1], (uint32_t)((n - 1) & 1), kCluWaitNs);
      if (!dead) update(false);
    }
    if (threadIdx.x == 0 && !dead) {  // this step's phase of both barriers
      mbar_expect_tx(&sm.full[0], zbytes);
      mbar_expect_tx(&sm.full[1], wbytes);
    }
    if (__syncthreads_or(dead)) break;
    // ---- x pass: row j
    {
      const float* ur_row = wp + 1 < kCluLines ? sm.u[wp + 1] : sm.uh[1];  // row j + 1
      const float* ud_row = wp > 0 ? sm.u[wp - 1] : sm.uh[0];             // row j - 1
      float cu = 0.f;
      V4<float> alpha[NS], beta[NS];
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) {
        const int c0 = sg * kImpSeg + 4 * lane;
        const bool in = row_in && c0 < a.ld;
        V4<float> uc = zero4<float>(), uu = zero4<float>(), ud = zero4<float>();
        float ur_own = 0.f;
        if (in) {
          uc = ld4(&sm.u[wp][c0]);
          uu = ld4(ur_row + c0);
          ud = ld4(ud_row + c0);
          if (lane == 31 && c0 + 4 < a.ld) ur_own = sm.u[wp][c0 + 4];
        }
        float ul = __shfl_up_sync(0xffffffffu, uc.a[3], 1);
        float ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
        if (lane == 0) ul = cu;
        if (lane == 31) ur = ur_own;
        imp_x_coeffs(a.cx, a.cy, a.sx, uc, uu, ud, hxk[sg], hyu[sg], hyd[sg], mxk[sg], ul, hxl[sg], ur, alpha[sg],
                     beta[sg]);
        cu = __shfl_sync(0xffffffffu, uc.a[3], 31);
      }
      V4<float> dk[NS], gamma[NS], zk[NS];
      line_solve<float, true, NS>(alpha, beta, dk, lane);
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) gamma[sg] = imp_x_gamma(a.sx, mxk[sg], hxk[sg]);
      line_solve<float, false, NS>(gamma, dk, zk, lane);
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) {
        const V4<float>& z = zk[sg];
        // columns c0 .. c0 + 3 (0 beyond the grid) into their owner's zb row j
        const int c0 = sg * kImpSeg + 4 * lane, o = c0 / kCluLines;
        st_async(cluster_addr(&sm.zb[j][clu_pos(j, c0 % kCluLines)], o), z.a[0], z.a[1], z.a[2], z.a[3],
                 cluster_addr(&sm.full[0], o));
      }
    }
    if (!dead) dead = !mbar_wait_bounded<true>(&sm.full[0], (uint32_t)(n & 1), kCluWaitNs);
    dead = __any_sync(0xffffffffu, dead);
    // ---- y pass: column i
    if (!dead) {
      V4<float> alpha[NS], beta[NS];
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) {
        const int c0 = sg * kImpSeg + 4 * lane;
        V4<float> z = zero4<float>();
        if (col_in && c0 < a.ldT) {
#pragma unroll
          for (int e = 0; e < 4; ++e) z.a[e] = sm.zb[c0 + e][clu_pos(c0 + e, wp)];
        }
        imp_y_coeffs(z, myk[sg], kyk[sg], kyl[sg], alpha[sg], beta[sg]);
      }
      V4<float> dk[NS], gamma[NS], wk[NS];
      line_solve<float, true, NS>(alpha, beta, dk, lane);
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) gamma[sg] = imp_y_gamma(myk[sg], kyk[sg]);
      line_solve<float, false, NS>(gamma, dk, wk, lane);
#pragma unroll
      for (int sg = 0; sg < NS; ++sg) {
        const V4<float>& wv = wk[sg];
        // rows c0 .. c0 + 3 into their owner's wb entry i; the owner's first row is the copied
        // row below of CTA o - 1, its last row the copied row above of CTA o + 1
        const int c0 = sg * kImpSeg + 4 * lane;
        const int o = c0 / kCluLines, q = c0 % kCluLines;
        st_async(cluster_addr(&sm.wb[i][clu_pos(i, q)], o), wv.a[0], wv.a[1], wv.a[2], wv.a[3],
                 cluster_addr(&sm.full[1], o));
        const int oh = q == 0 ? o - 1 : q == kCluLines - 4 ? o + 1 : -1;
        if (oh >= 0 && oh < NC)
          st_async(cluster_addr(&sm.wbh[q == 0 ? 1 : 0][i][0], oh), wv.a[0], wv.a[1], wv.a[2], wv.a[3],
                   cluster_addr(&sm.full[1], oh));
      }
    }
  }
  dead = __syncthreads_or(dead);
  if (!dead && nsteps > 0) {
    dead = !mbar_wait_bounded<true>(&sm.full[1], (uint32_t)((nsteps - 1) & 1), kCluWaitNs);
    if (!dead) update(first);
  }
  if (__syncthreads_or(dead) && threadIdx.x == 0) atomicExch(a.status, (int)TSU_ETIMEOUT);
  for (int q = threadIdx.x; q < kCluLines * kCluLen; q += nth) {
    const int r = q / kCluLen, c = q - r * kCluLen;
    const int jj = j0 + r;
    if (jj < a.ny && c < a.ld) a.uo[(int64_t)jj * a.ld + c] = sm.u[r][c];
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int q = threadIdx.x + k * kCluLines * 32;
    const int g = q / kCluLen, c = q - g * kCluLen;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = j0 + 4 * g + e;
      if (jj < a.ny && c < a.ld) a.v[(int64_t)jj * a.ld + c] = vk[k].a[e];
    }
  }
  cl.sync();  // no CTA leaves while another may still store into its shared memory
}

// Pivots of the x systems, one thread per row (once per medium and tau): for the unknowns
// i = 1..nx-2 of row j, a_i = -s cx hx_{i-1}, b_i = 1 + s cx (hx_{i-1} + hx_i), c_i = -s cx hx_i,
// p_i = b_i - a_i c_{i-1} / p_{i-1}; stores 1 / p_i (FP64 arithmetic).
template <typename T>
__global__ void k_imp_factor_x(int32_t nx, int32_t ny, int64_t ld, double sx, const T* hx, T* mx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 1 || j > ny - 2) return;
  const int64_t base = (int64_t)j * ld;
  double cprev = 0.0;  // c_{i-1} / p_{i-1}
  for (int i = 1; i <= nx - 2; ++i) {
    const double hl = (double)hx[base + i - 1], hr = (double)hx[base + i];
    const double p = (1.0 + sx * (hl + hr)) - (-(sx * hl)) * cprev;
    mx[base + i] = (T)(1.0 / p);
    cprev = -(sx * hr) / p;
  }
}

// Pivots of the y systems, one thread per column, stored transposed, with s cy hy transposed.
template <typename T>
__global__ void k_imp_factor_y(int32_t nx, int32_t ny, int64_t ld, int64_t ldT, double sy, const T* hy, T* myT,
                               T* kyT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  const int64_t base = (int64_t)i * ldT;
  for (int j = 0; j + 1 < ny; ++j) kyT[base + j] = (T)(sy * (double)hy[(int64_t)j * ld + i]);
  if (i < 1 || i > nx - 2) return;
  double cprev = 0.0;
  for (int j = 1; j <= ny - 2; ++j) {
    const double hd = (double)hy[(int64_t)(j - 1) * ld + i], hu = (double)hy[(int64_t)j * ld + i];
    const double p = (1.0 + sy * (hd + hu)) - (-(sy * hd)) * cprev;
    myT[base + j] = (T)(1.0 / p);
    cprev = -(sy * hu) / p;
  }
}

template <typename T>
__global__ void k_imp_prepare(int32_t nx, int32_t ny, int64_t ld, const T* u0, T* u, T* v) {
  const int64_t total = (int64_t)ny * ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / ld, i = k - j * ld;
    const bool interior = i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2;
    u[k] = interior ? u0[k] : T(0);
    v[k] = T(0);
  }
}

template <typename T, int R, int NS>
cudaError_t launch_pair(const ImpArgs<T>& a, cudaStream_t s) {
  k_imp_x<T, R, NS><<<(unsigned)((a.ny + R - 1) / R), R * 32, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_imp_y<T, R, NS><<<(unsigned)((a.nx + R - 1) / R), R * 32, 0, s>>>(a);
  return cudaGetLastError();
}

// Multi-step calls on a stream that can be captured run as one CUDA graph of all their launches
// (two per step): on small grids the launches, not the passes, took the time (Table 1 run at 256^2,
// FP32: 1.27 ms for 100 steps launched one by one, 0.66 ms as a graph).  The executable graph is
// kept per host thread with the exact arguments it was captured with and launched again when a
// call repeats them (the same problem stepped again); any other call captures a new one.
constexpr int64_t kImpGraphMinSteps = 4;

struct ImpGraphCache {
  unsigned char key[256];
  size_t key_len = 0;
  cudaGraphExec_t exec = nullptr;
  ImpGraphCache() = default;
  ImpGraphCache(const ImpGraphCache&) = delete;
  ImpGraphCache& operator=(const ImpGraphCache&) = delete;
  ~ImpGraphCache() {
    if (exec) cudaGraphExecDestroy(exec);  // errors at process teardown are ignored
  }
};
thread_local ImpGraphCache g_imp_graph;

bool imp_capturable(cudaStream_t s) {
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return false;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusNone;
}

// segments per line of the longer direction: up to 2 or 4 keep the lines in registers (256^2,
// 512^2 and smaller), beyond that the generic passes
template <typename T, int R>
cudaError_t imp_steps(const ImpArgs<T>& a, int64_t nsteps, cudaStream_t s) {
  const int nseg = (int)(((a.nx > a.ny ? a.nx : a.ny) - 1 + kImpSeg - 1) / kImpSeg);
  for (int64_t n = 0; n < nsteps; ++n) {
    cudaError_t e;
    if constexpr (R == 8)
      e = nseg <= 2 ? launch_pair<T, R, 2>(a, s) : nseg <= 4 ? launch_pair<T, R, 4>(a, s) : launch_pair<T, R, 0>(a, s);
    else
      e = launch_pair<T, R, 0>(a, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T, int R>
cudaError_t imp_steps_graph(const ImpArgs<T>& a, int64_t nsteps, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  struct Key {
    ImpArgs<T> a;
    int64_t nsteps;
    cudaStream_t s;
    int dev, r;
  } k;
  static_assert(sizeof(Key) <= sizeof(g_imp_graph.key), "graph key too large");
  memset(&k, 0, sizeof k);
  k.a = a;
  k.nsteps = nsteps;
  k.s = s;
  k.dev = dev;
  k.r = R;
  ImpGraphCache& c = g_imp_graph;
  if (!(c.exec && c.key_len == sizeof k && memcmp(c.key, &k, sizeof k) == 0)) {
    if (c.exec) cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
    c.key_len = 0;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = imp_steps<T, R>(a, nsteps, s);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(s, &gr);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return le != cudaSuccess ? le : e;
    }
    e = cudaGraphInstantiate(&c.exec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      c.exec = nullptr;
      return e;
    }
    memcpy(c.key, &k, sizeof k);
    c.key_len = sizeof k;
  }
  return cudaGraphLaunch(c.exec, s);
}

// Whether this device can place one cluster of k_imp_cluster<NC> (queried once per device and NC:
// cluster size 16 is non-portable): 0 not asked yet, 1 yes, 2 no.
std::atomic<int> g_clu_ok[2][64];

// 0: the grid does not fit one cluster; else the cluster size
int imp_cluster_ctas(const ImpArgs<float>& a) {
  if (a.ld > kCluLen || a.ldT > kCluLen) return 0;
  if (a.nx <= 8 * kCluLines + 1 && a.ny <= 8 * kCluLines + 1) return 8;  // node 128 is a boundary node
  if (a.nx <= 16 * kCluLines && a.ny <= 16 * kCluLines) return 16;
  return 0;
}

// Every step of the call in one cluster launch; *ran = false (and nothing launched) when the
// device cannot place the cluster.
template <int NC>
cudaError_t imp_cluster_launch(const ImpArgs<float>& a, int64_t nsteps, cudaStream_t s, bool* ran) {
  *ran = false;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC);
  cfg.blockDim = dim3(kCluLines * 32);
  cfg.dynamicSmemBytes = sizeof(CluSmem);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  std::atomic<int>& flag = g_clu_ok[NC == 16 ? 1 : 0][dev];
  int ok = flag.load();
  if (ok == 0) {
    ok = 2;
    if ((NC <= 8 ||
         cudaFuncSetAttribute(k_imp_cluster<NC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) &&
        cudaFuncSetAttribute(k_imp_cluster<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CluSmem)) ==
            cudaSuccess) {
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, k_imp_cluster<NC>, &cfg) == cudaSuccess && clusters >= 1) ok = 1;
    }
    (void)cudaGetLastError();  // a refused query leaves no error behind
    flag.store(ok);
  }
  if (ok != 1) return cudaSuccess;
  e = cudaLaunchKernelEx(&cfg, k_imp_cluster<NC>, a, nsteps);
  if (e == cudaSuccess) *ran = true;
  return e;
}

// start: u0 (may be u) and u1 -> the state after the start step; otherwise nsteps steps of (u, v)
template <typename T>
cudaError_t imp_run(const ImplicitGeom& g, const void* hx, const void* hy, const void* fac, const void* u0, void* u,
                    void* v, const void* u1, int64_t nsteps, bool start, void* ws, cudaStream_t s) {
  ImpArgs<T> a;
  memset(&a, 0, sizeof a);  // the graph cache compares the bytes
  a.nx = g.nx;
  a.ny = g.ny;
  a.ld = g.ld;
  a.ldT = g.ldT;
  a.cx = (T)g.cx;
  a.cy = (T)g.cy;
  a.sx = (T)(g.sigma * g.cx);
  a.tau = (T)g.tau;
  a.hx = (const T*)hx;
  a.hy = (const T*)hy;
  a.mx = (const T*)fac;
  a.myT = a.mx + (int64_t)g.ny * g.ld;
  a.kyT = a.myT + (int64_t)g.nx * g.ldT;
  a.u = (const T*)u;
  a.status = (int*)((char*)ws + 4);
  a.zT = (T*)((char*)ws + kImpWsHeader);
  a.scratch = a.zT + (int64_t)g.nx * g.ldT;
  a.v = (T*)v;
  a.uo = (T*)u;
  a.u1 = (const T*)u1;
  // 8 lines per CTA (a 32-byte run per transposed column); 16 (64-byte runs) for FP32 grids of
  // 2048^2 and up (Table 1 runs, FP32: 4096^2 23.2 against 27.2 ms, 2048^2 7.3 against 7.4 ms;
  // FP64, bound by the FP64 pipe, gains nothing and lost at 1024^2)
  const bool wide = sizeof(T) == 4 && g.nx >= 2048 && g.ny >= 2048;
  a.start = start ? 1 : 0;
  const int64_t n = start ? 1 : nsteps;
  if constexpr (sizeof(T) == 4) {  // small FP32 grids: every step in one cluster
    const int nc = imp_cluster_ctas(a);
    if (nc > 0 && n >= 1) {
      ImpArgs<T> c = a;
      if (start) c.u = (const T*)u0;  // the cluster reads u0 itself: no prepare pass
      bool ran = false;
      const cudaError_t e =
          nc == 8 ? imp_cluster_launch<8>(c, n, s, &ran) : imp_cluster_launch<16>(c, n, s, &ran);
      if (e != cudaSuccess || ran) return e;
    }
  }
  if (start) {  // u <- u0 on interior nodes, v <- 0, then the start step
    k_imp_prepare<T><<<152 * 8, 256, 0, s>>>(g.nx, g.ny, g.ld, (const T*)u0, (T*)u, (T*)v);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!start && n >= kImpGraphMinSteps && imp_capturable(s))
    return wide ? imp_steps_graph<T, 16>(a, n, s) : imp_steps_graph<T, 8>(a, n, s);
  return wide ? imp_steps<T, 16>(a, n, s) : imp_steps<T, 8>(a, n, s);
}

}  // namespace

int64_t implicit_ldT(int32_t ny) { return ((int64_t)ny + 31) / 32 * 32; }

size_t implicit_factor_elems(const tsu_grid& g) {
  return (size_t)g.ny * g.ld + 2 * (size_t)g.nx * implicit_ldT(g.ny);
}

size_t implicit_ws_bytes(const tsu_grid& g, size_t elem) {
  const size_t t = (size_t)g.nx * implicit_ldT(g.ny), r = (size_t)g.ny * g.ld;
  return kImpWsHeader + (t + (t > r ? t : r)) * elem;
}

cudaError_t launch_implicit_factor(const ImplicitGeom& g, int dtype, const void* hx, const void* hy, void* fac,
                                   cudaStream_t s) {
  const size_t es = dtype == TSU_F32 ? 4 : 8;
  tsu_grid tg{g.nx, g.ny, g.ld, 0.0, 0.0};
  cudaError_t e = cudaMemsetAsync(fac, 0, implicit_factor_elems(tg) * es, s);
  if (e != cudaSuccess) return e;
  const double sx = g.sigma * g.cx, sy = g.sigma * g.cy;
  const unsigned bx = (unsigned)((g.ny + 127) / 128), by = (unsigned)((g.nx + 127) / 128);
  if (dtype == TSU_F32) {
    float* mx = (float*)fac;
    float* myT = mx + (int64_t)g.ny * g.ld;
    float* kyT = myT + (int64_t)g.nx * g.ldT;
    k_imp_factor_x<float><<<bx, 128, 0, s>>>(g.nx, g.ny, g.ld, sx, (const float*)hx, mx);
    k_imp_factor_y<float><<<by, 128, 0, s>>>(g.nx, g.ny, g.ld, g.ldT, sy, (const float*)hy, myT, kyT);
  } else {
    double* mx = (double*)fac;
    double* myT = mx + (int64_t)g.ny * g.ld;
    double* kyT = myT + (int64_t)g.nx * g.ldT;
    k_imp_factor_x<double><<<bx, 128, 0, s>>>(g.nx, g.ny, g.ld, sx, (const double*)hx, mx);
    k_imp_factor_y<double><<<by, 128, 0, s>>>(g.nx, g.ny, g.ld, g.ldT, sy, (const double*)hy, myT, kyT);
  }
  return cudaGetLastError();
}

cudaError_t launch_implicit(const ImplicitGeom& g, int dtype, const void* hx, const void* hy, const void* fac,
                            const void* u0, void* u, void* v, const void* u1, int64_t nsteps, bool start, void* ws,
                            cudaStream_t s) {
  return dtype == TSU_F32 ? imp_run<float>(g, hx, hy, fac, u0, u, v, u1, nsteps, start, ws, s)
                          : imp_run<double>(g, hx, hy, fac, u0, u, v, u1, nsteps, start, ws, s);
}

}  // namespace tsu
