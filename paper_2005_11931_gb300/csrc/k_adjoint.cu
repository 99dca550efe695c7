// Discrete adjoint of the leapfrog scheme (the paper has no adjoint; this is the exact reverse of
// the scheme of k_step.cu, whose PDE is arXiv:2005.11931 Sec. 2 eq. (2.1) on the Sec. 3.3 box).
//
// For a receiver functional J(traces), g^n = S^T dJ/dtrace^n, the multipliers obey
//   lam^n = g^n + (2I + B) lam^{n+1} - lam^{n+2},  n = S..1,   lam^{S+1} = lam^{S+2} = 0,
//   dJ/du0 = (I + B/2) lam^1 - lam^2,  dJ/du1 = tau lam^1,
//   dJ/dhx_ij += -cx (lam^{n+1}_{i+1,j} - lam^{n+1}_ij)(u^n_{i+1,j} - u^n_ij)   (n = 1..S-1, and
//                with -cx/2, lam^1 and u^0 for the start), dJ/dhy likewise in j.
// k_adjoint_pass computes lam^n from lam^{n+1} (5-point) and lam^{n+2} (centre), written over
// lam^{n+2}, with the same register-streaming layout as the forward pass, and accumulates both
// face gradients from lam^{n+1} and the recomputed forward state u^n.  FP32 runs the recursion in
// increment form, mu^n = lam^n - lam^{n+1}:
//   mu^n = mu^{n+1} + B lam^{n+1} + g^n,  lam^n = lam^{n+1} + mu^n,  dJ/du0 = mu^1 + B lam^1 / 2,
// algebraically the same recursion; it keeps the multipliers accurate over thousands of steps in
// FP32 for the reason the forward's increment form does (the change per step is far below one ulp
// of lam).  In FP32 the face gradients are summed in FP32 over one checkpoint segment and flushed
// into FP64 per segment.
#include "stencil_common.cuh"

namespace tsu {
namespace {
using namespace dev;

template <typename T>
struct AccOf;
template <>
struct AccOf<float> { using type = float; };
template <>
struct AccOf<double> { using type = double; };

// MODE 0 (kAdjStep):     lam_out = (2 lam_c - lam_pp) + B lam_c          (the recursion)
// MODE 1 (kAdjStart):    lam_out = (lam_c - lam_pp) + B lam_c / 2 = dJ/du0; g_u1 = tau lam_c
// MODE 2 (kAdjStepInc):  lam_pp holds mu^{n+1}: mu_out = mu^{n+1} + B lam_c (may be lam_pp itself:
//                        every node reads only its own mu), lam_out = lam_c + mu_out
// MODE 3 (kAdjStartInc): lam_pp holds mu^1: lam_out = mu^1 + B lam_c / 2 = dJ/du0; g_u1 = tau lam_c
template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_adjoint_pass(const int32_t nx, const int32_t ny, const int64_t ld,
                                                      const typename AdjArithOf<T>::type ar, const T gwx, const T gwy,
                                                      const T tau, const T* __restrict__ hx, const T* __restrict__ hy,
                                                      const T* __restrict__ lam, const T* lam_pp, T* lam_out, T* mu_out,
                                                      const T* __restrict__ u, typename AccOf<T>::type* gx,
                                                      typename AccOf<T>::type* gy, T* g_u1, const int rows,
                                                      const RecBuckets rb) {
  using A = typename AccOf<T>::type;
  constexpr int V = Vec<T>::V;
  const int lane = threadIdx.x & 31;
  int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
  const bool active = i0 < ld;
  if (!active) i0 = 0;
  const int j0 = 1 + blockIdx.y * rows;
  const int j1 = min(j0 + rows, ny - 1);
  if (j0 >= j1) return;  // uniform per CTA

  // u^n with its boundary nodes read as zero (the start pass reads the caller's u0)
  auto umask = [&](Pack<T> v, int j) {
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int64_t i = i0 + e;
      if (!(i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2)) v.a[e] = T(0);
    }
    return v;
  };
  auto u_at = [&](int64_t i, int j) -> T {
    return (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) ? u[(int64_t)j * ld + i] : T(0);
  };

  Pack<T> lm = ld_vec(lam + (int64_t)(j0 - 1) * ld + i0);
  Pack<T> lc = ld_vec(lam + (int64_t)j0 * ld + i0);
  Pack<T> hym = ld_vec(hy + (int64_t)(j0 - 1) * ld + i0);
  Pack<T> uc = umask(ld_vec(u + (int64_t)j0 * ld + i0), j0);
  for (int j = j0; j < j1; ++j) {
    const int64_t row = (int64_t)j * ld + i0;
    const Pack<T> ln = ld_vec(lam + row + ld);
    const Pack<T> lp = ld_vec_l2(lam_pp + row);
    const Pack<T> hxv = ld_vec(hx + row);
    const Pack<T> hyv = ld_vec(hy + row);
    const Pack<T> un = umask(ld_vec(u + row + ld), j + 1);
    T ll = __shfl_up_sync(0xffffffffu, lc.a[V - 1], 1);
    T hl = __shfl_up_sync(0xffffffffu, hxv.a[V - 1], 1);
    T lr = __shfl_down_sync(0xffffffffu, lc.a[0], 1);
    T ur = __shfl_down_sync(0xffffffffu, uc.a[0], 1);
    if (lane == 0) {
      ll = (i0 > 0) ? lam[row - 1] : T(0);
      hl = (i0 > 0) ? hx[row - 1] : T(0);
    }
    if (lane == 31) {
      lr = (i0 + V < ld) ? lam[row + V] : T(0);
      ur = u_at(i0 + V, j);
    }
    Pack<T> out, gu1, mo;
    A gxv[V], gyv[V], gy0[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int64_t i = i0 + e;
      const T xl = (e == 0) ? ll : lc.a[e - 1];
      const T xr = (e == V - 1) ? lr : lc.a[e + 1];
      const T hxl = (e == 0) ? hl : hxv.a[e - 1];
      const T b = ar.b(hxv.a[e], hxl, hyv.a[e], hym.a[e], lc.a[e], xl, xr, ln.a[e], lm.a[e]);
      const bool interior = (i >= 1) && (i <= nx - 2);
      T val;
      if constexpr (MODE == 0) {
        val = ar.lf(lc.a[e], lp.a[e], b);
      } else if constexpr (MODE == 2) {
        const T mu = ar.add(lp.a[e], b);
        mo.a[e] = interior ? mu : T(0);
        val = ar.add(lc.a[e], mu);
      } else {
        const T d = (MODE == 1) ? lc.a[e] - lp.a[e] : lp.a[e];  // lam^1 - lam^2 = mu^1
        if constexpr (sizeof(T) == 8)
          val = __dadd_rn(MODE == 1 ? __dsub_rn(lc.a[e], lp.a[e]) : lp.a[e], __dmul_rn(0.5, b));
        else
          val = d + 0.5f * b;
        gu1.a[e] = interior ? tau * lc.a[e] : T(0);
      }
      out.a[e] = interior ? val : T(0);
      // face gradients: x-face (i, i+1) on this row, y-face (j, j+1) on this column
      const T uxr = (e == V - 1) ? ur : uc.a[e + 1];
      const T dlx = xr - lc.a[e], dux = uxr - uc.a[e];
      const T dly = ln.a[e] - lc.a[e], duy = un.a[e] - uc.a[e];
      gxv[e] = (i <= nx - 2) ? (A)(gwx * (dlx * dux)) : A(0);
      gyv[e] = interior ? (A)(gwy * (dly * duy)) : A(0);
      gy0[e] = interior ? (A)(gwy * (lc.a[e] * uc.a[e])) : A(0);  // y-face (0, 1), used on row 1
    }
    if (active) {
      st_vec(lam_out + row, out);
      if constexpr (MODE == 2) st_vec(mu_out + row, mo);
      if constexpr (MODE == 1 || MODE == 3) st_vec(g_u1 + row, gu1);
      // the accumulators have the field's vector width (float4 / double2): 16-byte read-modify-write
      Pack<A> ax = ld_vec_l2(gx + row), ay = ld_vec_l2(gy + row);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        ax.a[e] += gxv[e];
        ay.a[e] += gyv[e];
      }
      st_vec(gx + row, ax);
      st_vec(gy + row, ay);
      if (j == 1) {
        Pack<A> a0 = ld_vec_l2(gy + i0);
#pragma unroll
        for (int e = 0; e < V; ++e) a0.a[e] += gy0[e];
        st_vec(gy + i0, a0);
      }
    }
    lm = lc;
    lc = ln;
    hym = hyv;
    uc = un;
  }
  // receiver injection lam^n += g^n (and mu^n += g^n in increment form) at this CTA's receivers,
  // in receiver order, after the CTA's own stores (visible to the CTA after the barrier)
  if (rb.off) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      for (int q = rb.off[cta]; q < rb.off[cta + 1]; ++q) {
        const int r = rb.ord[q];
        const T gv = ((const T*)rb.g)[r];
        lam_out[rb.idx[r]] += gv;
        if constexpr (MODE == 2) mu_out[rb.idx[r]] += gv;
      }
    }
  }
}

// Receivers grouped by the CTA of the adjoint pass that owns their node (interior nodes only),
// in receiver order: off[ncta + 1], ord[nrec].  One thread; nrec and ncta are small.
__global__ void k_rec_bucket(const int32_t nx, const int32_t ny, const int64_t ld, const int64_t* idx,
                             const int32_t nrec, const int64_t cols_per_cta, const int rows, const int64_t gridx,
                             const int64_t ncta, int* off, int* ord, int* cta_of) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int64_t c = 0; c <= ncta; ++c) off[c] = 0;
  for (int r = 0; r < nrec; ++r) {
    const int64_t q = idx[r];
    int c = -1;
    if (q >= 0 && q < (int64_t)ny * ld) {
      const int64_t j = q / ld, i = q - j * ld;
      if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) c = (int)(((j - 1) / rows) * gridx + i / cols_per_cta);
    }
    cta_of[r] = c;
    if (c >= 0) off[c + 1] += 1;
  }
  for (int64_t c = 0; c < ncta; ++c) off[c + 1] += off[c];
  // stable fill with off[c] as the cursor of bucket c, then shift the cursors back to the starts
  for (int r = 0; r < nrec; ++r)
    if (cta_of[r] >= 0) ord[off[cta_of[r]]++] = r;
  for (int64_t c = ncta; c >= 1; --c) off[c] = off[c - 1];
  off[0] = 0;
}

// lam[rec_idx[r]] += g[r] for interior receiver nodes (boundary receivers record a constant 0)
template <typename T>
__global__ void k_inject(const int32_t nx, const int32_t ny, const int64_t ld, T* lam, const T* g, const int64_t* idx,
                         const int32_t nrec) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrec) return;
  const int64_t q = idx[r];
  if (q < 0 || q >= (int64_t)ny * ld) return;
  const int64_t j = q / ld, i = q - j * ld;
  if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) atomicAdd(&lam[q], g[r]);
}

__global__ void k_flush(const int64_t total, float* g32x, float* g32y, double* gx, double* gy) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    gx[k] += (double)g32x[k];
    gy[k] += (double)g32y[k];
    g32x[k] = 0.0f;
    g32y[k] = 0.0f;
  }
}

template <typename T>
typename AdjArithOf<T>::type arith(const StencilGeom& g) {
  typename AdjArithOf<T>::type a;
  a.cx = (T)g.cx;
  a.cy = (T)g.cy;
  return a;
}

}  // namespace

void adjoint_pass_shape(const StencilGeom& g, int dtype, int64_t* gridx, int64_t* gridy, int* rows,
                        int64_t* cols_per_cta) {
  const int64_t cpc = (int64_t)128 * (dtype == TSU_F32 ? 4 : 2);
  const int r = auto_rows(g.ld, g.ny, cpc);
  *cols_per_cta = cpc;
  *rows = r;
  *gridx = (g.ld + cpc - 1) / cpc;
  *gridy = (g.ny - 2 + r - 1) / r;
}

namespace {
template <typename T, int MODE>
void pass_mode(dim3 grid, const StencilGeom& g, T gwx, T gwy, const void* hx, const void* hy, const void* lam,
               const void* lam_pp, void* lam_out, void* mu_out, const void* u, void* gx, void* gy, void* g_u1,
               int rows, const RecBuckets& rb, cudaStream_t s) {
  using A = typename AccOf<T>::type;
  k_adjoint_pass<T, MODE><<<grid, 128, 0, s>>>(g.nx, g.ny, g.ld, arith<T>(g), gwx, gwy, (T)g.tau, (const T*)hx,
                                               (const T*)hy, (const T*)lam, (const T*)lam_pp, (T*)lam_out,
                                               (T*)mu_out, (const T*)u, (A*)gx, (A*)gy, (T*)g_u1, rows, rb);
}

template <typename T>
cudaError_t pass_t(const StencilGeom& g, int mode, const void* hx, const void* hy, const void* lam,
                   const void* lam_pp, void* lam_out, void* mu_out, const void* u, void* gx, void* gy, void* g_u1,
                   const RecBuckets& rb, cudaStream_t s) {
  int64_t gx_, gy_, cpc;
  int rows;
  adjoint_pass_shape(g, sizeof(T) == 4 ? TSU_F32 : TSU_F64, &gx_, &gy_, &rows, &cpc);
  dim3 grid((unsigned)gx_, (unsigned)gy_);
  const bool start = mode == kAdjStart || mode == kAdjStartInc;
  const T w = start ? T(0.5) : T(1);
  const T gwx = -(T)g.cx * w, gwy = -(T)g.cy * w;
  switch (mode) {
    case kAdjStep:
      pass_mode<T, 0>(grid, g, gwx, gwy, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rows, rb, s);
      break;
    case kAdjStart:
      pass_mode<T, 1>(grid, g, gwx, gwy, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rows, rb, s);
      break;
    case kAdjStepInc:
      pass_mode<T, 2>(grid, g, gwx, gwy, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rows, rb, s);
      break;
    case kAdjStartInc:
      pass_mode<T, 3>(grid, g, gwx, gwy, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rows, rb, s);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_rec_bucket(const StencilGeom& g, int dtype, const int64_t* idx, int32_t nrec, int* off, int* ord,
                              int* cta_of, cudaStream_t s) {
  int64_t gx_, gy_, cpc;
  int rows;
  adjoint_pass_shape(g, dtype, &gx_, &gy_, &rows, &cpc);
  k_rec_bucket<<<1, 32, 0, s>>>(g.nx, g.ny, g.ld, idx, nrec, cpc, rows, gx_, gx_ * gy_, off, ord, cta_of);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_pass(const StencilGeom& g, int dtype, int mode, const void* hx, const void* hy,
                                const void* lam, const void* lam_pp, void* lam_out, void* mu_out, const void* u,
                                void* gx, void* gy, void* g_u1, const RecBuckets& rb, cudaStream_t s) {
  return dtype == TSU_F32 ? pass_t<float>(g, mode, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rb, s)
                          : pass_t<double>(g, mode, hx, hy, lam, lam_pp, lam_out, mu_out, u, gx, gy, g_u1, rb, s);
}

cudaError_t launch_inject(const StencilGeom& g, int dtype, void* lam, const void* gvals, const int64_t* idx,
                          int32_t nrec, cudaStream_t s) {
  if (nrec <= 0) return cudaSuccess;
  const int threads = 128;
  const unsigned blocks = (unsigned)((nrec + threads - 1) / threads);
  if (dtype == TSU_F32)
    k_inject<float><<<blocks, threads, 0, s>>>(g.nx, g.ny, g.ld, (float*)lam, (const float*)gvals, idx, nrec);
  else
    k_inject<double><<<blocks, threads, 0, s>>>(g.nx, g.ny, g.ld, (double*)lam, (const double*)gvals, idx, nrec);
  return cudaGetLastError();
}

cudaError_t launch_flush(const StencilGeom& g, void* g32x, void* g32y, double* gx, double* gy, cudaStream_t s) {
  const int64_t total = (int64_t)g.ny * g.ld;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_flush<<<(unsigned)blocks, 256, 0, s>>>(total, (float*)g32x, (float*)g32y, gx, gy);
  return cudaGetLastError();
}

}  // namespace tsu
