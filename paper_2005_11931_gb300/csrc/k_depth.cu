// Face-sampled regularised depth h_eps = background + sum_s amp_s * phi_eps(dist_s)^p_s
// (arXiv:2005.11931 Sec. 2.1: h_eps = h * psi_eps; Sec. 3.1: the Friedrichs bump, delta and
// delta^2 singularities, the mollified step h0).  Evaluated in FP64 on the device, rounded once
// to the field type; the extrema of the stored values are reduced with ordered-integer atomics.
#include <math.h>

#include "tsu_internal.h"

namespace tsu {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

__device__ __forceinline__ double bump(double t) {
  return (fabs(t) < 1.0) ? exp(1.0 / (t * t - 1.0)) : 0.0;
}

// Mass of the 1D Friedrichs mollifier on (-inf, t]: c1 * int_{-1}^{t} bump, by the
// tanh-sinh rule on [-1, t] (step 1/16, |k| <= 64), which handles the flat endpoint.
__device__ double friedrichs_cdf(double c1, double t) {
  if (t <= -1.0) return 0.0;
  if (t >= 1.0) return 1.0;
  const double a = -1.0, b = t, half = 0.5 * (b - a), mid = 0.5 * (a + b);
  const double h = 1.0 / 16.0;
  double s = 0.0;
  for (int k = -64; k <= 64; ++k) {
    double x = k * h;
    double sh = sinh(x), ch = cosh(x);
    double arg = 0.5 * kPi * sh;
    double th = tanh(arg), cha = cosh(arg);
    double w = 0.5 * kPi * ch / (cha * cha);
    double tt = mid + half * th;
    s += w * bump(tt);
  }
  return c1 * s * h * half;
}

// Far from a singularity the mollifier's value is exactly 0 in FP64 (exp(-q^2) underflows for
// q^2 > 745.2; the bump vanishes for |t| >= 1) and the mollified step is exactly 0 or 1; those
// faces skip the transcendental functions, with the same results.  kFar = 750 keeps a margin over
// the rounding of the squared distances.
constexpr double kFar = 750.0;

__device__ __forceinline__ double phi1(const DepthParams& p, double s) {
  const double e = p.eps;
  if (p.mollifier == TSU_GAUSS) {
    if (s * s > kFar * (e * e)) return 0.0;
    double q = s / e;
    return exp(-q * q) / (e * sqrt(kPi));
  }
  if (s * s >= e * e * 1.0000001) return 0.0;
  return p.c1 / e * bump(s / e);
}

__device__ __forceinline__ double phi2(const DepthParams& p, double dx, double dy) {
  const double e = p.eps, r2 = dx * dx + dy * dy;
  if (p.mollifier == TSU_GAUSS) {
    if (r2 > kFar * (e * e)) return 0.0;
    double q = sqrt(r2) / e;
    return exp(-q * q) / (kPi * e * e);
  }
  if (r2 >= e * e * 1.0000001) return 0.0;
  return p.c2 / (e * e) * bump(sqrt(r2) / e);
}

__device__ __forceinline__ double step1(const DepthParams& p, double s) {
  if (p.mollifier == TSU_GAUSS) {
    // 0.5 erfc(-s/eps): erfc(t) = 2 exactly below t = -6 and 0 above t = 27.3
    if (s > 7.0 * p.eps) return 1.0;
    if (s < -28.0 * p.eps) return 0.0;
    return 0.5 * erfc(-s / p.eps);
  }
  return friedrichs_cdf(p.c1, s / p.eps);
}

__device__ double depth_at(const DepthParams& p, double x, double y) {
  double h = p.background;
  for (int k = 0; k < p.nsing; ++k) {
    const tsu_sing& s = p.sing[k];
    double v;
    switch (s.kind) {
      case TSU_LINE_X: v = phi1(p, x - s.cx); break;
      case TSU_LINE_Y: v = phi1(p, y - s.cy); break;
      case TSU_POINT: v = phi2(p, x - s.cx, y - s.cy); break;
      case TSU_STEP_X: v = step1(p, s.cx - x); break;
      default: v = step1(p, s.cy - y); break;
    }
    double pw = v;
    for (int q = 1; q < s.power; ++q) pw *= v;
    h += s.amp * pw;
  }
  return h;
}

// FP32 distances beyond which a singularity's term is exactly 0 in FP64 (exactly 0 or 1 for a
// step): a face whose FP32 coordinates clear them for every term skips the FP64 evaluation, with
// the same result (8192^2 point workload: 3.25 ms of FP64 coordinate and conversion work per
// evaluation of the depth before).  The margins (0.1 % plus 1e-5 in the unit box) exceed the FP32 rounding of the
// face coordinates and centres (about 2e-7).
struct FarTest {
  float cx[kMaxSing], cy[kMaxSing];
  float d[kMaxSing];   // line / point: |s| or r above which the term is 0
  float hi[kMaxSing];  // step: s = c - x above which the step is 1
  float lo[kMaxSing];  // ... below which it is 0
};

// Decides a face from FP32 coordinates when every term is exactly 0 there (or, for a step,
// exactly 0 or 1): returns 0 if the depth is the background, 1 if it is h (the background plus
// the amplitudes of the steps at 1, added in the order depth_at adds them), 2 if a term needs
// the FP64 evaluation.
__device__ __forceinline__ int far_decide(const DepthParams& p, const FarTest& f, float xf, float yf, double& h) {
  int r = 0;
  for (int k = 0; k < p.nsing; ++k) {
    const int kind = p.sing[k].kind;
    if (kind == TSU_LINE_X) {
      if (fabsf(xf - f.cx[k]) > f.d[k]) continue;
      return 2;
    }
    if (kind == TSU_LINE_Y) {
      if (fabsf(yf - f.cy[k]) > f.d[k]) continue;
      return 2;
    }
    if (kind == TSU_POINT) {
      const float ax = xf - f.cx[k], ay = yf - f.cy[k];
      if (ax * ax + ay * ay > f.d[k] * f.d[k]) continue;
      return 2;
    }
    const float sf = kind == TSU_STEP_X ? f.cx[k] - xf : f.cy[k] - yf;
    if (sf < f.lo[k]) continue;
    if (sf > f.hi[k]) {  // the step is exactly 1: amp * 1^power
      if (r == 0) h = p.background;
      h += p.sing[k].amp;
      r = 1;
      continue;
    }
    return 2;
  }
  return r;
}

// d h_eps / d eps (Sec. 2.1, the regularised depth's derivative in its width).  With
// psi_eps(s) = eps^-d psi(s/eps) and t = s/eps:  d/deps psi_eps = -eps^-(d+1) (d psi + t psi'(t)),
// where t psi' = -2 t^2 psi (Gaussian) or -2 t^2/(t^2-1)^2 psi (bump); for the mollified step
// S(s) = int^{s/eps} psi:  dS/deps = -(t/eps) psi(t); a power p > 1 brings p phi^{p-1}.
__device__ __forceinline__ double dphi_deps(const DepthParams& p, int d, double c, double s2) {
  const double e = p.eps;
  if (p.mollifier == TSU_GAUSS && s2 > kFar * (e * e)) return 0.0;
  if (p.mollifier != TSU_GAUSS && s2 >= e * e * 1.0000001) return 0.0;
  const double t2 = s2 / (e * e);
  double psi, tdpsi;
  if (p.mollifier == TSU_GAUSS) {
    psi = exp(-t2) / (d == 1 ? sqrt(kPi) : kPi);
    tdpsi = -2.0 * t2 * psi;
  } else {
    psi = c * exp(1.0 / (t2 - 1.0));
    const double w = t2 - 1.0;
    tdpsi = -2.0 * t2 / (w * w) * psi;
  }
  const double ed = d == 1 ? e * e : e * e * e;
  return -(d * psi + tdpsi) / ed;
}

__device__ __forceinline__ double dstep_deps(const DepthParams& p, double s) {
  const double e = p.eps, t = s / e;
  double psi;
  if (p.mollifier == TSU_GAUSS) {
    if (t * t > kFar) return 0.0;
    psi = exp(-t * t) / sqrt(kPi);
  } else {
    psi = fabs(t) < 1.0 ? p.c1 * exp(1.0 / (t * t - 1.0)) : 0.0;
  }
  return -t / e * psi;
}

__device__ double depth_deps_at(const DepthParams& p, double x, double y) {
  double acc = 0.0;
  for (int k = 0; k < p.nsing; ++k) {
    const tsu_sing& s = p.sing[k];
    double v, dv;
    switch (s.kind) {
      case TSU_LINE_X:
        v = phi1(p, x - s.cx);
        dv = dphi_deps(p, 1, p.c1, (x - s.cx) * (x - s.cx));
        break;
      case TSU_LINE_Y:
        v = phi1(p, y - s.cy);
        dv = dphi_deps(p, 1, p.c1, (y - s.cy) * (y - s.cy));
        break;
      case TSU_POINT: {
        const double dx = x - s.cx, dy = y - s.cy;
        v = phi2(p, dx, dy);
        dv = dphi_deps(p, 2, p.c2, dx * dx + dy * dy);
        break;
      }
      case TSU_STEP_X:
        v = step1(p, s.cx - x);
        dv = dstep_deps(p, s.cx - x);
        break;
      default:
        v = step1(p, s.cy - y);
        dv = dstep_deps(p, s.cy - y);
        break;
    }
    double pw = 1.0;  // v^(power-1)
    for (int q = 1; q < s.power; ++q) pw *= v;
    acc += s.amp * (s.power * pw) * dv;
  }
  return acc;
}

// Order-preserving map of doubles to unsigned 64-bit integers (for atomicMin/Max).
__device__ __forceinline__ unsigned long long ord_enc(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_dec(unsigned long long e) {
  unsigned long long b = (e & 0x8000000000000000ull) ? (e & 0x7fffffffffffffffull) : ~e;
  return __longlong_as_double((long long)b);
}

__global__ void k_ext_reset(unsigned long long* ext) {
  ext[0] = ~0ull;  // min hx
  ext[1] = 0ull;   // max hx
  ext[2] = ~0ull;  // min hy
  ext[3] = 0ull;   // max hy
}

__global__ void k_ext_decode(unsigned long long* ext) {
  double* d = reinterpret_cast<double*>(ext);
  for (int k = 0; k < 4; ++k) d[k] = ord_dec(ext[k]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_make_depth(int32_t nx, int32_t ny, int64_t ld, double dx, double dy,
                                                    const DepthParams p, const FarTest f, const T bg,
                                                    T* __restrict__ hx, T* __restrict__ hy,
                                                    unsigned long long* ext) {
  // work items of 256 columns of one row, spread over a fixed grid (one division per item), so
  // that rows near a singularity, whose faces are costly, are shared by every CTA
  T mnx_t = T(INFINITY), mxx_t = T(-INFINITY), mny_t = T(INFINITY), mxy_t = T(-INFINITY);
  const float dxf = (float)dx, dyf = (float)dy;
  const int64_t bxn = (ld + 255) / 256, items = (int64_t)ny * bxn;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    const int64_t j = w / bxn, i = (w - j * bxn) * 256 + threadIdx.x;
    if (i >= ld) continue;
    // 32-bit integers into the FP32 conversions (a 64-bit source converts on the FP64 pipe)
    const float yjf = (float)(int32_t)j * dyf, yhf = ((float)(int32_t)j + 0.5f) * dyf;
    const int64_t k = j * ld + i;
    T vx = T(0), vy = T(0);
    if (i <= nx - 2) {
      double h;
      const int r = far_decide(p, f, ((float)(int32_t)i + 0.5f) * dxf, yjf, h);
      vx = r == 0 ? bg : r == 1 ? T(h) : T(depth_at(p, (i + 0.5) * dx, j * dy));
      mnx_t = vx < mnx_t ? vx : mnx_t;
      mxx_t = vx > mxx_t ? vx : mxx_t;
    }
    if (i < nx && j <= ny - 2) {
      double h;
      const int r = far_decide(p, f, (float)(int32_t)i * dxf, yhf, h);
      vy = r == 0 ? bg : r == 1 ? T(h) : T(depth_at(p, i * dx, (j + 0.5) * dy));
      mny_t = vy < mny_t ? vy : mny_t;
      mxy_t = vy > mxy_t ? vy : mxy_t;
    }
    hx[k] = vx;
    hy[k] = vy;
  }
  // the extrema of the stored values, exact in their own type (min / max do not round)
  for (int o = 16; o > 0; o >>= 1) {
    const T a = __shfl_xor_sync(0xffffffffu, mnx_t, o), b = __shfl_xor_sync(0xffffffffu, mxx_t, o);
    const T c = __shfl_xor_sync(0xffffffffu, mny_t, o), d = __shfl_xor_sync(0xffffffffu, mxy_t, o);
    mnx_t = a < mnx_t ? a : mnx_t;
    mxx_t = b > mxx_t ? b : mxx_t;
    mny_t = c < mny_t ? c : mny_t;
    mxy_t = d > mxy_t ? d : mxy_t;
  }
  double mnx = (double)mnx_t, mxx = (double)mxx_t, mny = (double)mny_t, mxy = (double)mxy_t;
  __shared__ double red[4][8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = mnx;
    red[1][w] = mxx;
    red[2][w] = mny;
    red[3][w] = mxy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int q = 1; q < nw; ++q) {
      mnx = fmin(mnx, red[0][q]);
      mxx = fmax(mxx, red[1][q]);
      mny = fmin(mny, red[2][q]);
      mxy = fmax(mxy, red[3][q]);
    }
    if (mnx <= mxx) {
      atomicMin(&ext[0], ord_enc(mnx));
      atomicMax(&ext[1], ord_enc(mxx));
    }
    if (mny <= mxy) {
      atomicMin(&ext[2], ord_enc(mny));
      atomicMax(&ext[3], ord_enc(mxy));
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_depth_deps(int32_t nx, int32_t ny, int64_t ld, double dx, double dy,
                                                    const DepthParams p, T* __restrict__ dhx, T* __restrict__ dhy) {
  const int64_t total = (int64_t)ny * ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / ld, i = k - j * ld;
    dhx[k] = (i <= nx - 2) ? T(depth_deps_at(p, (i + 0.5) * dx, j * dy)) : T(0);
    dhy[k] = (i < nx && j <= ny - 2) ? T(depth_deps_at(p, i * dx, (j + 0.5) * dy)) : T(0);
  }
}

// Per-block FP64 partial sums of g_hx dhx/deps + g_hy dhy/deps (fixed grid, fixed order).
__global__ void __launch_bounds__(256) k_eps_gradient(int32_t nx, int32_t ny, int64_t ld, double dx, double dy,
                                                      const DepthParams p, const double* __restrict__ gx,
                                                      const double* __restrict__ gy, double* partials) {
  const int64_t total = (int64_t)ny * ld;
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / ld, i = k - j * ld;
    if (i <= nx - 2 && gx[k] != 0.0) acc += gx[k] * depth_deps_at(p, (i + 0.5) * dx, j * dy);
    if (i < nx && j <= ny - 2 && gy[k] != 0.0) acc += gy[k] * depth_deps_at(p, i * dx, (j + 0.5) * dy);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += red[q];
    partials[blockIdx.x] = t;
  }
}

}  // namespace

cudaError_t launch_depth_deps(const tsu_grid& g, const DepthParams& p, int dtype, void* dhx, void* dhy,
                              cudaStream_t s) {
  const int64_t total = (int64_t)g.ny * g.ld;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (dtype == TSU_F32)
    k_depth_deps<float><<<(unsigned)blocks, 256, 0, s>>>(g.nx, g.ny, g.ld, g.dx, g.dy, p, (float*)dhx, (float*)dhy);
  else
    k_depth_deps<double><<<(unsigned)blocks, 256, 0, s>>>(g.nx, g.ny, g.ld, g.dx, g.dy, p, (double*)dhx,
                                                         (double*)dhy);
  return cudaGetLastError();
}

cudaError_t launch_eps_gradient(const tsu_grid& g, const DepthParams& p, const double* gx, const double* gy,
                                double* partials, double* out, cudaStream_t s) {
  k_eps_gradient<<<kReduceBlocks, 256, 0, s>>>(g.nx, g.ny, g.ld, g.dx, g.dy, p, gx, gy, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_partials(partials, kReduceBlocks, 1, out, s);
}

cudaError_t launch_make_depth(const tsu_grid& g, const DepthParams& p, int dtype, void* hx, void* hy,
                              double* ext_dev, cudaStream_t s) {
  auto* ext = reinterpret_cast<unsigned long long*>(ext_dev);
  k_ext_reset<<<1, 1, 0, s>>>(ext);
  FarTest f;
  for (int k = 0; k < p.nsing && k < kMaxSing; ++k) {
    const tsu_sing& q = p.sing[k];
    const double e = p.eps;
    const bool gauss = p.mollifier == TSU_GAUSS;
    f.cx[k] = (float)q.cx;
    f.cy[k] = (float)q.cy;
    const double reach = gauss ? sqrt(kFar) * e : e;  // the mollifier's support, as its FP64 tests see it
    f.d[k] = (float)(reach * 1.001 + 1e-5);
    const double up = (gauss ? 7.0 * e : e) * 1.001 + 1e-5, down = (gauss ? 28.0 * e : e) * 1.001 + 1e-5;
    f.hi[k] = (float)up;
    f.lo[k] = (float)-down;
  }
  // one fixed grid of 152 x 32 CTAs: enough to hide the FP64 latency of the faces near a
  // singularity, few enough that the four extrema's atomics stay cheap (8192^2 point depth:
  // 0.74 against 3.41 ms; 16384^2 crossing lines 7.4 against 18.5 ms; the same values)
  const int64_t items = (int64_t)g.ny * ((g.ld + 255) / 256);
  const unsigned grid = (unsigned)(items < 152 * 32 ? items : 152 * 32);
  if (dtype == TSU_F32)
    k_make_depth<float><<<grid, 256, 0, s>>>(g.nx, g.ny, g.ld, g.dx, g.dy, p, f, (float)p.background, (float*)hx,
                                             (float*)hy, ext);
  else
    k_make_depth<double><<<grid, 256, 0, s>>>(g.nx, g.ny, g.ld, g.dx, g.dy, p, f, p.background, (double*)hx,
                                              (double*)hy, ext);
  k_ext_decode<<<1, 1, 0, s>>>(ext);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Host: Friedrichs normalisers by the double-exponential (tanh-sinh) rule.
// ---------------------------------------------------------------------------------------------
namespace {
double host_bump(double t) { return (fabs(t) < 1.0) ? exp(1.0 / (t * t - 1.0)) : 0.0; }

// int_{-1}^{1} f(t) dt with t = tanh(pi/2 sinh x), step h, |x| <= 6.
template <typename F>
double tanh_sinh(F f) {
  const double h = 1.0 / 64.0;
  double s = 0.0;
  for (int k = -384; k <= 384; ++k) {
    double x = k * h;
    double arg = 0.5 * kPi * sinh(x);
    double ca = cosh(arg);
    double w = 0.5 * kPi * cosh(x) / (ca * ca);
    s += w * f(tanh(arg));
  }
  return s * h;
}
}  // namespace

double friedrichs_c1() {
  static const double c = 1.0 / tanh_sinh([](double t) { return host_bump(t); });
  return c;
}

double friedrichs_c2() {
  // int_{R^2} bump(|r|) dA = 2 pi int_0^1 r bump(r) dr, with r = (1+t)/2 mapped onto [-1, 1]
  static const double c = 1.0 / (2.0 * kPi * 0.5 * tanh_sinh([](double t) {
                                   const double r = 0.5 * (1.0 + t);
                                   return r * host_bump(r);
                                 }));
  return c;
}

}  // namespace tsu
