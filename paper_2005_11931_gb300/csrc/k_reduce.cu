// Deterministic FP64 reductions over a field: fixed grid, per-block partial sums, then one block
// that adds them in a fixed order.  Used to compare two fields (the eps-family studies of
// arXiv:2005.11931 Sec. 3.2 measure how far apart the regularised solutions are) and by the
// eps-gradient of the depth.
#include "tsu_internal.h"

namespace tsu {
namespace {

// out[c] = sum over partials[c][0 .. nblocks-1], c < ncomp, in index order (one block).
__global__ void __launch_bounds__(256) k_sum_partials(const double* partials, int nblocks, int ncomp, double* out) {
  __shared__ double red[256];
  for (int c = 0; c < ncomp; ++c) {
    double t = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) t += partials[(int64_t)c * nblocks + q];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
    __syncthreads();
  }
}

// partials[0][b] = sum (a - b)^2, partials[1][b] = sum b^2 over the nodes i < nx this block visits.
template <typename T>
__global__ void __launch_bounds__(256) k_diff_norms(int32_t nx, int32_t ny, int64_t ld, const T* __restrict__ a,
                                                    const T* __restrict__ b, double* partials) {
  const int64_t total = (int64_t)ny * ld;
  double sd = 0.0, sb = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / ld, i = k - j * ld;
    if (i < nx) {
      const double x = (double)a[k], y = (double)b[k], d = x - y;
      sd += d * d;
      sb += y * y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  __shared__ double red[2][8];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sd;
    red[1][threadIdx.x >> 5] = sb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < 8; ++q) {
      t0 += red[0][q];
      t1 += red[1][q];
    }
    partials[blockIdx.x] = t0;
    partials[gridDim.x + blockIdx.x] = t1;
  }
}

}  // namespace

cudaError_t launch_sum_partials(const double* partials, int nblocks, int ncomp, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(partials, nblocks, ncomp, out);
  return cudaGetLastError();
}

cudaError_t launch_diff_norms(const tsu_grid& g, int dtype, const void* a, const void* b, double* partials,
                              double* out, cudaStream_t s) {
  if (dtype == TSU_F32)
    k_diff_norms<float><<<kReduceBlocks, 256, 0, s>>>(g.nx, g.ny, g.ld, (const float*)a, (const float*)b, partials);
  else
    k_diff_norms<double><<<kReduceBlocks, 256, 0, s>>>(g.nx, g.ny, g.ld, (const double*)a, (const double*)b,
                                                       partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_partials(partials, kReduceBlocks, 2, out, s);
}

}  // namespace tsu
