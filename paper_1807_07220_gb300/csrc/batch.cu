// Staging kernels of batched solves: copies between caller buffers and the
// contexts' buffers through device pointer tables (one launch instead of one
// copy call per array), the shared tolerance, and the per-context results.
#include "common.cuh"

namespace tg {
namespace {

// table layout: 5 entries per context (f, bflux, ux, uy, p); entries [t0, t1)
// of every context are copied; a NULL source writes zeros when zero_if_null
__global__ void k_copy_table(const double* const* __restrict__ src, double* const* __restrict__ dst,
                             const long long* __restrict__ cnt, int t0, int t1, int zero_if_null) {
  pdl_entry();
  const int per = t1 - t0;
  const int j = blockIdx.y / per, t = t0 + blockIdx.y % per;
  const int e = 5 * j + t;
  const double* a = src[e];
  double* b = dst[e];
  const long long m = cnt[e];
  if (!b) return;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
       k += (long long)gridDim.x * blockDim.x) {
    if (a) b[k] = a[k];
    else if (zero_if_null) b[k] = 0.0;
  }
}

__global__ void k_fill_scalars(const double* __restrict__ v, double* const* __restrict__ dst, int m) {
  pdl_entry();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) dst[j][0] = v[0];
}

__global__ void k_gather_states(PcgState* const* __restrict__ st, int* __restrict__ out, int m) {
  pdl_entry();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) {
    out[2 * j] = st[j]->iter;
    out[2 * j + 1] = st[j]->status;
  }
}

}  // namespace

void launch_copy_table(const double* const* src, double* const* dst, const long long* cnt, int m, int t0, int t1,
                       int zero_if_null, cudaStream_t s) {
  TG_COUNT(1);
  dim3 grid(64, m * (t1 - t0));
  launch(k_copy_table, dim3(grid), dim3(256), 0, s, src, dst, cnt, t0, t1, zero_if_null);
}
void launch_fill_scalars(const double* v, double* const* dst, int m, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_fill_scalars, dim3((m + 127) / 128), dim3(128), 0, s, v, dst, m);
}
void launch_gather_states(PcgState* const* st, int* out, int m, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_gather_states, dim3((m + 127) / 128), dim3(128), 0, s, st, out, m);
}

}  // namespace tg
