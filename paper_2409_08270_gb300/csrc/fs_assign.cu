// Closed-form optimal assignment (Sec. 3.2 "Regularized ILP for Noise
// Reduction", Sec. 3.3 Eq. 7, Supp. Sec. 6 Listing 1).
//
// Per Gaussian i with row A[i, :] and S = sum_e A[i, e] (taken once), for each
// label e: others = S - A_e; both are L1-normalised by
// n = max(|others| + |A_e|, 1e-12); the Gaussian belongs to e iff
// A_e/n > others/n + gamma (a tie is not a membership).  One thread per
// Gaussian; the decision is made in the table's precision.
#include <math.h>

#include "fs_internal.h"

namespace fs {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) assign_kernel(const T* __restrict__ table, int64_t n, int E,
                                                     T gamma, uint64_t* __restrict__ bits,
                                                     int32_t* __restrict__ label,
                                                     float* __restrict__ margin) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T* row = table + i * E;
  T S = 0;
  for (int e = 0; e < E; ++e) S += row[e];
  uint64_t b = 0;
  int members = 0, lab = -1;
  float mmin = INFINITY;
  const T one = 1;
  for (int e = 0; e < E; ++e) {
    const T a = row[e];
    const T others = S - a;
    T nrm = fabs(others) + fabs(a);
    if (nrm < T(1e-12)) nrm = T(1e-12);
    if (a / nrm > others / nrm + gamma) {
      if (e < 64) b |= (1ull << e);
      ++members;
      lab = e;
    }
    if (S > 0) {
      const T mg = fabs((one - gamma) * a - (one + gamma) * others) / S;
      mmin = fminf(mmin, static_cast<float>(mg));
    }
  }
  if (bits) bits[i] = b;
  if (label) label[i] = members == 1 ? lab : -1;
  if (margin) margin[i] = mmin;
}

}  // namespace

cudaError_t launch_assign(const void* table, int table_dtype, int64_t n, int E, float gamma,
                          uint64_t* member_bits, int32_t* label, float* margin,
                          cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((n + threads - 1) / threads);
  if (table_dtype == 0)
    assign_kernel<float><<<blocks, threads, 0, stream>>>(static_cast<const float*>(table), n, E,
                                                         gamma, member_bits, label, margin);
  else
    assign_kernel<double><<<blocks, threads, 0, stream>>>(static_cast<const double*>(table), n, E,
                                                          static_cast<double>(gamma), member_bits,
                                                          label, margin);
  return cudaGetLastError();
}

}  // namespace fs
