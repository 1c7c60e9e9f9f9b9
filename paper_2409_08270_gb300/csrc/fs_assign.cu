// Closed-form optimal assignment (Sec. 3.2 "Regularized ILP for Noise
// Reduction", Sec. 3.3 Eq. 7, Supp. Sec. 6 Listing 1).
//
// Per Gaussian i with row A[i, :] and S = sum_e A[i, e] (taken once), for each
// label e: others = S - A_e; both are L1-normalised by
// n = max(|others| + |A_e|, 1e-12); the Gaussian belongs to e iff
// A_e/n > others/n + gamma (a tie is not a membership), evaluated as
// A_e - others > gamma n.  One thread per Gaussian; the decision is made in
// the table's precision.
#include <math.h>

#include "fs_internal.h"

namespace fs {

namespace {

struct Decision {
  uint64_t bits;
  int32_t label;
  float margin;
};

// The comparison a/n > others/n + gamma is taken as a - others > gamma n
// (n > 0: the same decision, without a division per label: FP64 divisions
// are costly on this part), and the margins share one reciprocal of S.
template <typename T>
__device__ __forceinline__ Decision decide(const T* row, int E, T gamma) {
  T S = 0;
  for (int e = 0; e < E; ++e) S += row[e];
  uint64_t b = 0;
  int members = 0, lab = -1;
  float mmin = INFINITY;
  const T one = 1;
  const T inv_s = S > 0 ? one / S : T(0);
  for (int e = 0; e < E; ++e) {
    const T a = row[e];
    const T others = S - a;
    T nrm = fabs(others) + fabs(a);
    if (nrm < T(1e-12)) nrm = T(1e-12);
    if (a - others > gamma * nrm) {
      if (e < 64) b |= (1ull << e);
      ++members;
      lab = e;
    }
    if (S > 0) {
      const T mg = fabs((one - gamma) * a - (one + gamma) * others) * inv_s;
      mmin = fminf(mmin, static_cast<float>(mg));
    }
  }
  return {b, members == 1 ? lab : -1, mmin};
}

template <typename T>
__global__ void __launch_bounds__(256) assign_kernel(const T* __restrict__ table, int64_t n, int E,
                                                     T gamma, uint64_t* __restrict__ bits,
                                                     int32_t* __restrict__ label,
                                                     float* __restrict__ margin) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Decision d = decide<T>(table + i * E, E, gamma);
  if (bits) bits[i] = d.bits;
  if (label) label[i] = d.label;
  if (margin) margin[i] = d.margin;
}

// The same with the block's rows staged through shared memory: rows of E
// values at a stride of E are read by consecutive threads at consecutive
// addresses (the direct form above reads one row per thread, E * 8 bytes
// apart).  128 rows per block.
constexpr int kAssignRows = 128;
template <typename T>
__global__ void __launch_bounds__(kAssignRows) assign_staged_kernel(
    const T* __restrict__ table, int64_t n, int E, T gamma, uint64_t* __restrict__ bits,
    int32_t* __restrict__ label, float* __restrict__ margin) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rows = reinterpret_cast<T*>(smem_raw);
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kAssignRows;
  const int n_rows = static_cast<int>(min(static_cast<int64_t>(kAssignRows), n - i0));
  const int count = n_rows * E;
  const T* src = table + i0 * E;
  for (int k = threadIdx.x; k < count; k += kAssignRows) rows[k] = src[k];
  __syncthreads();
  if (static_cast<int>(threadIdx.x) >= n_rows) return;
  const int64_t i = i0 + threadIdx.x;
  const Decision d = decide<T>(rows + threadIdx.x * E, E, gamma);
  if (bits) bits[i] = d.bits;
  if (label) label[i] = d.label;
  if (margin) margin[i] = d.margin;
}

__global__ void __launch_bounds__(256) round_table_kernel(int64_t count,
                                                          const double* __restrict__ src,
                                                          float* __restrict__ dst) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = static_cast<float>(src[i]);
}

// Rows re-evaluated in FP64: row j of R belongs to Gaussian F[j].  The row
// replaces the table's (rounded to its type) and the decision is taken again
// in FP64.
template <typename TableT>
__global__ void __launch_bounds__(256) assign_rows_kernel(
    const double* __restrict__ R, const uint32_t* __restrict__ F, int64_t n_rows, int E,
    double gamma, TableT* __restrict__ table, uint64_t* __restrict__ bits,
    int32_t* __restrict__ label, float* __restrict__ margin) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n_rows) return;
  const double* row = R + j * E;
  const int64_t i = F[j];
  for (int e = 0; e < E; ++e) table[i * E + e] = static_cast<TableT>(row[e]);
  const Decision d = decide<double>(row, E, gamma);
  if (bits) bits[i] = d.bits;
  if (label) label[i] = d.label;
  if (margin) margin[i] = d.margin;
}

// flag[i] = 1 iff Gaussian i belongs to none of the objects in `remove`
__global__ void __launch_bounds__(256) keep_flag_kernel(int64_t n,
                                                        const uint64_t* __restrict__ bits,
                                                        uint64_t remove,
                                                        uint32_t* __restrict__ flag) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (bits[i] & remove) ? 0u : 1u;
}

__global__ void __launch_bounds__(256) keep_scatter_kernel(int64_t n,
                                                           const uint32_t* __restrict__ flag,
                                                           const uint32_t* __restrict__ offs,
                                                           int32_t* __restrict__ keep) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) keep[offs[i]] = static_cast<int32_t>(i);
}

}  // namespace

cudaError_t launch_keep_flags(int64_t n, const uint64_t* member_bits, uint64_t remove,
                              uint32_t* flag, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  keep_flag_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(n, member_bits,
                                                                              remove, flag);
  return cudaGetLastError();
}

cudaError_t launch_keep_scatter(int64_t n, const uint32_t* flag, const uint32_t* offs,
                                int32_t* keep, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  keep_scatter_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(n, flag, offs,
                                                                                 keep);
  return cudaGetLastError();
}

cudaError_t launch_assign(const void* table, int table_dtype, int64_t n, int E, float gamma,
                          uint64_t* member_bits, int32_t* label, float* margin,
                          cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const size_t elem = table_dtype == 0 ? 4 : 8;
  const size_t smem = static_cast<size_t>(kAssignRows) * E * elem;
  if (E > 4 && smem <= 48 * 1024) {
    const unsigned blocks = static_cast<unsigned>((n + kAssignRows - 1) / kAssignRows);
    if (table_dtype == 0)
      assign_staged_kernel<float><<<blocks, kAssignRows, smem, stream>>>(
          static_cast<const float*>(table), n, E, gamma, member_bits, label, margin);
    else
      assign_staged_kernel<double><<<blocks, kAssignRows, smem, stream>>>(
          static_cast<const double*>(table), n, E, static_cast<double>(gamma), member_bits,
          label, margin);
    return cudaGetLastError();
  }
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

cudaError_t launch_round_table(int64_t count, const double* src, float* dst,
                               cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  const int threads = 256;
  round_table_kernel<<<static_cast<unsigned>((count + threads - 1) / threads), threads, 0,
                       stream>>>(count, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_assign_rows(const double* R, const uint32_t* F, int64_t n_rows, int E,
                               float gamma, void* table, int table_dtype, uint64_t* member_bits,
                               int32_t* label, float* margin, cudaStream_t stream) {
  if (n_rows == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = static_cast<unsigned>((n_rows + threads - 1) / threads);
  if (table_dtype == 0)
    assign_rows_kernel<float><<<blocks, threads, 0, stream>>>(
        R, F, n_rows, E, static_cast<double>(gamma), static_cast<float*>(table), member_bits,
        label, margin);
  else
    assign_rows_kernel<double><<<blocks, threads, 0, stream>>>(
        R, F, n_rows, E, static_cast<double>(gamma), static_cast<double*>(table), member_bits,
        label, margin);
  return cudaGetLastError();
}

}  // namespace fs
