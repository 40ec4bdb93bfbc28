// Kernels of the batch of independent fits: per-instance residual statistics.
#include "mfa_internal.cuh"

namespace mfa {

// One CTA per instance: sum of squares and max |E| of E = Q - D over the
// instance's values (FP64, fixed order within the CTA).  out[2i] = sum E^2,
// out[2i+1] = max |E|.
template <typename TQ>
__global__ void __launch_bounds__(256) k_batch_residual(const double* __restrict__ D, const TQ* __restrict__ Q,
                                                        const long long* __restrict__ off,
                                                        const long long* __restrict__ len, double* __restrict__ out) {
  const int i = blockIdx.x;
  const long long o = off[i], n = len[i];
  double s2 = 0.0, emax = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    const double e = (double)Q[o + k] - D[o + k];
    s2 = fma(e, e, s2);
    emax = fmax(emax, fabs(e));
  }
  for (int sft = 16; sft > 0; sft >>= 1) {
    s2 += __shfl_down_sync(0xffffffffu, s2, sft);
    emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, sft));
  }
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = s2;
    red[1][w] = emax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[0][k];
      b = fmax(b, red[1][k]);
    }
    out[2 * i] = a;
    out[2 * i + 1] = b;
  }
}

template <typename TQ>
void launch_batch_residual(const double* D, const TQ* Q, const long long* off, const long long* len, int count,
                           double* out, cudaStream_t st) {
  if (count > 0) k_batch_residual<TQ><<<count, 256, 0, st>>>(D, Q, off, len, out);
}

template void launch_batch_residual<float>(const double*, const float*, const long long*, const long long*, int,
                                           double*, cudaStream_t);
template void launch_batch_residual<double>(const double*, const double*, const long long*, const long long*, int,
                                            double*, cudaStream_t);

}  // namespace mfa
