// Masks for removed DOFs (fully fictitious cells dropped, Sec. 4.3.2): the
// removed DOFs keep their slots in the level vectors and blocks; these
// kernels keep the assembled blocks factorisable and the vectors zero there.
#include <cuda_runtime.h>

#include "fcm_internal.h"

namespace fcm {
namespace {

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

// Removed DOFs in assembled blocks (fully fictitious cells dropped): a DOF
// whose row is empty has a zero diagonal.  Phase 0 flags those rows and puts
// a unit diagonal there (the block stays factorisable); phase 1 zeroes the
// flagged rows and columns of the inverse.
__global__ void mask_empty_rows_kernel(long long count, int n, int phase, double* mats,
                                       unsigned char* flags) {
  const long long tot = phase == 0 ? count * n : count * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    if (phase == 0) {
      const long long b = e / n;
      const int i = (int)(e - b * n);
      double* d = mats + (size_t)b * n * n + (size_t)i * n + i;
      const bool empty = *d == 0.0;
      flags[e] = empty ? 1 : 0;
      if (empty) *d = 1.0;
    } else {
      const long long b = e / ((long long)n * n);
      const int rc = (int)(e - b * n * n);
      const int r = rc / n, c = rc - r * n;
      if (flags[b * n + r] || flags[b * n + c]) mats[e] = 0.0;
    }
  }
}

// v[i] = 0 where the scalar DOF i % M is not kept.
template <typename T>
__global__ void mask_vec_kernel(long long N, long long M, const unsigned char* __restrict__ keep,
                                T* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    if (!keep[i % M]) v[i] = (T)0;
}

void launch_mask_empty_rows(long long count, int n, int phase, double* mats,
                            unsigned char* flags, cudaStream_t s) {
  if (count == 0) return;
  const long long tot = phase == 0 ? count * n : count * n * n;
  mask_empty_rows_kernel<<<grid_for(tot), 256, 0, s>>>(count, n, phase, mats, flags);
}

template <typename T>
void launch_mask_vec(long long N, long long M, const unsigned char* keep, T* v, cudaStream_t s) {
  mask_vec_kernel<T><<<grid_for(N), 256, 0, s>>>(N, M, keep, v);
}
template void launch_mask_vec<double>(long long, long long, const unsigned char*, double*,
                                      cudaStream_t);
template void launch_mask_vec<float>(long long, long long, const unsigned char*, float*,
                                     cudaStream_t);

}  // namespace fcm
