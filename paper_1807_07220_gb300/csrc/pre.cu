// Section 3 preprocessing (a discrete flux vbar with B_h vbar = F_h built from
// a coarse RT0 solve and per-block zero-flux Neumann solves), the residual of
// the reduced system in stream-function form, the final velocity update and
// the pressure recovery.  Face arrays ux, uy hold physical normal velocities
// including the prescribed boundary values.
#include "common.cuh"

namespace tg {
namespace {

constexpr int kThreads = 256;

inline int grid_for(long long m) {
  long long g = (m + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

// In-place inclusive prefix sum of v[0..m) by one CTA (each thread scans a
// contiguous chunk, then the chunk totals are scanned by warp 0).
__device__ void block_inclusive_scan(double* v, int m) {
  __shared__ double tot[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int chunk = (m + T - 1) / T, lo = min(m, t * chunk), hi = min(m, lo + chunk);
  double run = 0.0;
  for (int k = lo; k < hi; ++k) {
    run += v[k];
    v[k] = run;
  }
  // exclusive scan of the chunk totals: shuffle scan inside each warp, then
  // the warp totals by warp 0
  __shared__ double wtot[32];
  const int lane = t & 31, w = t >> 5;
  double x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  if (w == 0) {
    double v = (lane < (T >> 5)) ? wtot[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wtot[lane] = v - ((lane < (T >> 5)) ? wtot[lane] : 0.0);   // exclusive warp offsets
  }
  __syncthreads();
  tot[t] = wtot[w] + x - run;   // exclusive offset of thread t
  __syncthreads();
  const double off = tot[t];
  for (int k = lo; k < hi; ++k) v[k] += off;
  __syncthreads();
}

__device__ double block_reduce_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// boundary lift: outward normal velocity bflux -> face values; interior 0
__global__ void k_lift(const double* __restrict__ bflux, double* __restrict__ ux,
                       double* __restrict__ uy, int n) {
  pdl_entry();
  const long long m = (long long)(n + 1) * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    {  // x-face (i, j), index j*(n+1)+i
      const int i = (int)(t % (n + 1)), j = (int)(t / (n + 1));
      double v = 0.0;
      if (bflux) {
        if (i == 0) v = -bflux[j];
        else if (i == n) v = bflux[n + j];
      }
      ux[t] = v;
    }
    {  // y-face (i, j), index j*n+i
      const int i = (int)(t % n), j = (int)(t / n);
      double v = 0.0;
      if (bflux) {
        if (j == 0) v = -bflux[2 * n + i];
        else if (j == n) v = bflux[3 * n + i];
      }
      uy[t] = v;
    }
  }
}

__device__ __forceinline__ double cell_outflow(const double* ux, const double* uy, int n, int i, int j,
                                               double h) {
  return h * (ux[(long long)j * (n + 1) + i + 1] - ux[(long long)j * (n + 1) + i] +
              uy[(long long)(j + 1) * n + i] - uy[(long long)j * n + i]);
}

// per block: FH = sum_c (h^2 f_c - outflow_c), absF = sum_c (|h^2 f_c| + |outflow_c| terms)
__global__ void k_block_sources(const double* __restrict__ f, const double* __restrict__ ux,
                                const double* __restrict__ uy, double* __restrict__ FH,
                                double* __restrict__ absF, int n, int b) {
  pdl_entry();
  __shared__ double sa[32], sb[32];
  const int nc = n / b, blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const double h = 1.0 / n;
  double a = 0.0, s = 0.0;
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
    const int i = I * b + t % b, j = J * b + t / b;
    const double F = h * h * f[(long long)j * n + i];
    a += F - cell_outflow(ux, uy, n, i, j, h);
    s += fabs(F) + h * (fabs(ux[(long long)j * (n + 1) + i + 1]) + fabs(ux[(long long)j * (n + 1) + i]) +
                        fabs(uy[(long long)(j + 1) * n + i]) + fabs(uy[(long long)j * n + i]));
  }
  a = warp_sum(a);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += sa[w];
      tb += sb[w];
    }
    FH[blk] = ta;
    absF[blk] = tb;
  }
}

// Particular coarse RT0 coefficients with B_H g = F_H: all vertical transport
// in the first block column (cumulative row totals), then horizontal transport
// along each block row (cumulative remaining sources).  gx[(J)*(nc+1) + I] is
// the normal value on the vertical coarse edge x = I H of block row J, gy[J*nc+I]
// on the horizontal edge y = J H of block column I (boundary edges zero).
__global__ void k_rt_particular(const double* __restrict__ FH, const double* __restrict__ absF,
                                double* __restrict__ gx, double* __restrict__ gy, int nc, double H,
                                int nblocks, PcgState* st) {
  pdl_entry();
  extern __shared__ double sm[];
  double* rowt = sm;            // nc row totals -> flux above each block row (column 0)
  double* fh = sm + nc;         // block sources staged in shared memory
  double a = 0.0, ab = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    const double v = FH[k];
    fh[k] = v;
    a += v;
    ab += absF[k];
  }
  const double tot = block_reduce_sum(a), abt = block_reduce_sum(ab);
  if (threadIdx.x == 0 && fabs(tot) > 1e-12 * fmax(abt, 1e-300)) {
    st->status |= kStIncompatible;
    st->done = 1;
  }
  for (int k = threadIdx.x; k < (nc + 1) * nc; k += blockDim.x) {
    gx[k] = 0.0;
    gy[k] = 0.0;
  }
  for (int J = threadIdx.x; J < nc; J += blockDim.x) {
    double row = 0.0;
    for (int I = 0; I < nc; ++I) row += fh[J * nc + I];
    rowt[J] = row;
  }
  __syncthreads();
  block_inclusive_scan(rowt, nc);   // rowt[J] = flux through the edge above row J (column 0)
  for (int J = threadIdx.x; J < nc; J += blockDim.x) {
    const double below = (J > 0) ? rowt[J - 1] : 0.0;
    const double above = (J + 1 < nc) ? rowt[J] : 0.0;
    if (J + 1 < nc) gy[(J + 1) * nc + 0] = above / H;
    double run = 0.0;
    for (int I = 0; I + 1 < nc; ++I) {
      double s = fh[J * nc + I];
      if (I == 0) s -= (above - below);
      run += s;
      gx[J * (nc + 1) + I + 1] = run / H;
    }
  }
}

// u += interpolation of the coarse RT0 field g onto the interior fine faces
__global__ void k_add_rt_field(const double* __restrict__ gx, const double* __restrict__ gy,
                               double* __restrict__ ux, double* __restrict__ uy, int n, int b) {
  pdl_entry();
  const int nc = n / b;
  const long long m = (long long)(n + 1) * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    {
      const int i = (int)(t % (n + 1)), j = (int)(t / (n + 1));
      if (i > 0 && i < n) {
        const int I0 = i / b, J = j / b;
        const double w = (double)(i - I0 * b) / b;
        const double a0 = gx[J * (nc + 1) + I0];
        const double a1 = (I0 + 1 <= nc) ? gx[J * (nc + 1) + I0 + 1] : 0.0;
        ux[t] += (1.0 - w) * a0 + (w > 0.0 ? w * a1 : 0.0);
      }
    }
    {
      const int i = (int)(t % n), j = (int)(t / n);
      if (j > 0 && j < n) {
        const int J0 = j / b, I = i / b;
        const double w = (double)(j - J0 * b) / b;
        const double a0 = gy[J0 * nc + I];
        const double a1 = (J0 + 1 <= nc) ? gy[(J0 + 1) * nc + I] : 0.0;
        uy[t] += (1.0 - w) * a0 + (w > 0.0 ? w * a1 : 0.0);
      }
    }
  }
}

// (A u)_f / h on x-face (i, j) and y-face (i, j) (exact RT0 mass, cell kinv)
__device__ __forceinline__ double Au_x(const double* ux, const double* kinv, int n, int i, int j) {
  const double kL = (i > 0) ? kinv[(long long)j * n + i - 1] : 0.0;
  const double kR = (i < n) ? kinv[(long long)j * n + i] : 0.0;
  const double* u = ux + (long long)j * (n + 1) + i;
  double v = (kL + kR) * (1.0 / 3.0) * u[0];
  if (i > 0) v += kL * (1.0 / 6.0) * u[-1];
  if (i < n) v += kR * (1.0 / 6.0) * u[1];
  return v * (1.0 / n);  // h^2 / h
}
__device__ __forceinline__ double Au_y(const double* uy, const double* kinv, int n, int i, int j) {
  const double kB = (j > 0) ? kinv[(long long)(j - 1) * n + i] : 0.0;
  const double kT = (j < n) ? kinv[(long long)j * n + i] : 0.0;
  const double* u = uy + (long long)j * n + i;
  double v = (kB + kT) * (1.0 / 3.0) * u[0];
  if (j > 0) v += kB * (1.0 / 6.0) * u[-n];
  if (j < n) v += kT * (1.0 / 6.0) * u[n];
  return v * (1.0 / n);
}

// rho = C^T (-A u) at the interior nodes (the residual of the reduced system)
__global__ void k_face_residual(const double* __restrict__ ux, const double* __restrict__ uy,
                                const double* __restrict__ kinv, double* __restrict__ rho, int n) {
  pdl_entry();
  // Au_x / Au_y already carry the 1/h of C^T: rho = sum of (-A u)/h over the four faces
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    double v = 0.0;
    if (i > 0 && j > 0) {
      v = -Au_x(ux, kinv, n, i, j - 1) + Au_x(ux, kinv, n, i, j) + Au_y(uy, kinv, n, i - 1, j) -
          Au_y(uy, kinv, n, i, j);
    }
    rho[t] = v;
  }
}

// u += C psi on the interior faces
__global__ void k_add_curl(const double* __restrict__ psi, double* __restrict__ ux,
                           double* __restrict__ uy, int n) {
  pdl_entry();
  const long long m = (long long)(n + 1) * n;
  const double inv_h = (double)n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    {
      const int i = (int)(t % (n + 1)), j = (int)(t / (n + 1));
      if (i > 0 && i < n) {
        const double top = (j + 1 < n) ? psi[(long long)(j + 1) * n + i] : 0.0;
        ux[t] += (top - psi[(long long)j * n + i]) * inv_h;
      }
    }
    {
      const int i = (int)(t % n), j = (int)(t / n);
      if (j > 0 && j < n) {
        const double right = (i + 1 < n) ? psi[(long long)j * n + i + 1] : 0.0;
        uy[t] -= (right - psi[(long long)j * n + i]) * inv_h;
      }
    }
  }
}

// Particular zero-flux field on each block carrying the block's remaining
// divergence s_c = h^2 f_c - outflow_c (zero mean per block after the coarse
// RT0 step): vertical transport in the block's first column, then horizontal
// transport along each row.
__global__ void k_block_particular(const double* __restrict__ f, double* __restrict__ ux,
                                   double* __restrict__ uy, int n, int b) {
  pdl_entry();
  __shared__ double s[kMaxB * kMaxB];
  __shared__ double up[kMaxB + 1];
  const int nc = n / b, blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const double h = 1.0 / n;
  for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
    const int i = I * b + t % b, j = J * b + t / b;
    s[t] = h * h * f[(long long)j * n + i] - cell_outflow(ux, uy, n, i, j, h);
  }
  __syncthreads();
  if (threadIdx.x < b) {
    double row = 0.0;
    for (int a = 0; a < b; ++a) row += s[threadIdx.x * b + a];
    up[threadIdx.x + 1] = row;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    up[0] = 0.0;
    for (int c = 1; c <= b; ++c) up[c] += up[c - 1];
    up[b] = 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < b) {
    // vertical flux through y-face (I b, J b + c), c >= 1, column 0 of the block
    // flux / h = flux * n (products, not FP64 divisions, in the loop)
    if (c >= 1) uy[(long long)(J * b + c) * n + I * b] += up[c] * (double)n;
    double run = 0.0;
    for (int a = 0; a + 1 < b; ++a) {
      double v = s[c * b + a];
      if (a == 0) v -= (up[c + 1] - up[c]);
      run += v;
      ux[(long long)(J * b + c) * (n + 1) + I * b + a + 1] += run * (double)n;
    }
  }
}

// pressure: integrate A u = B^T p along each row (x-faces), then fit one
// offset per row to the y-face equations in least squares, zero mean.
// Warm start: stream function of the x-face part of w = u0 - vbar, one CTA
// per node column i: psi(i, 0) = 0, psi(i, j+1) = psi(i, j) + h w_x(i, j)
// (exact when w is divergence free with zero boundary flux, the form of every
// PCG iterate); column 0 is boundary.  col: n doubles of scratch per column.
__global__ void k_psi_from_faces(const double* __restrict__ ux0, const double* __restrict__ vx,
                                 double* __restrict__ colbuf, double* __restrict__ psi, int n) {
  pdl_entry();
  const int i = blockIdx.x;
  const double h = 1.0 / n;
  double* col = colbuf + (long long)i * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const long long f = (long long)j * (n + 1) + i;
    col[j] = (i == 0) ? 0.0 : h * (ux0[f] - vx[f]);
  }
  __syncthreads();
  block_inclusive_scan(col, n);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    psi[(long long)j * n + i] = (i == 0 || j == 0) ? 0.0 : col[j - 1];
}

__global__ void k_pressure_rows(const double* __restrict__ ux, const double* __restrict__ kinv,
                                double* __restrict__ rowp, int n) {
  pdl_entry();
  const int j = blockIdx.x;
  double* row = rowp + (long long)j * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = (i == 0) ? 0.0 : -Au_x(ux, kinv, n, i, j);
  __syncthreads();
  block_inclusive_scan(row, n);
}

__global__ void k_pressure_steps(const double* __restrict__ uy, const double* __restrict__ kinv,
                                 const double* __restrict__ rowp, double* __restrict__ step,
                                 double* __restrict__ rowsum, int n) {
  pdl_entry();
  __shared__ double sh[32];
  const int j = blockIdx.x;  // row j -> j+1 (j < n-1); row sums for all rows
  double a = 0.0, rs = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    rs += rowp[(long long)j * n + i];
    if (j + 1 < n)
      a += rowp[(long long)j * n + i] - rowp[(long long)(j + 1) * n + i] - Au_y(uy, kinv, n, i, j + 1);
  }
  a = warp_sum(a);
  rs = warp_sum(rs);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    step[j] = (j + 1 < n) ? t / n : 0.0;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = rs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    rowsum[j] = t;
  }
}

// step[j] (row j -> j+1) becomes the offset c_j = sum_{k<j} step[k] of row j;
// step[n] receives the mean of the pressure.
__global__ void k_pressure_offsets(double* __restrict__ step, const double* __restrict__ rowsum,
                                   int n) {
  pdl_entry();
  extern __shared__ double c[];
  for (int j = threadIdx.x; j < n; j += blockDim.x) c[j] = (j == 0) ? 0.0 : step[j - 1];
  __syncthreads();
  block_inclusive_scan(c, n);
  double part = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    step[j] = c[j];
    part += rowsum[j] + (double)n * c[j];
  }
  const double tot = block_reduce_sum(part);
  if (threadIdx.x == 0) step[n] = tot / ((double)n * n);
}

__global__ void k_pressure_final(const double* __restrict__ rowp, const double* __restrict__ off,
                                 double* __restrict__ p, int n) {
  pdl_entry();
  const long long nn = (long long)n * n;
  const double mean = off[n];
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x)
    p[t] = rowp[t] + off[t / n] - mean;
}

// max_c |outflow_c - h^2 f_c| and max_c |h^2 f_c| per CTA
__global__ void k_div_error(const double* __restrict__ ux, const double* __restrict__ uy,
                            const double* __restrict__ f, double* __restrict__ part, int n) {
  pdl_entry();
  __shared__ double sa[32], sb[32];
  const long long nn = (long long)n * n;
  const double h = 1.0 / n;
  double a = 0.0, m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    const double F = h * h * f[t];
    a = fmax(a, fabs(cell_outflow(ux, uy, n, i, j, h) - F));
    m = fmax(m, fabs(F));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = fmax(a, sa[w]);
      m = fmax(m, sb[w]);
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = m;
  }
}

__global__ void k_div_error_final(const double* __restrict__ part, int g, double* __restrict__ out) {
  pdl_entry();
  double a = 0.0, m = 0.0;
  for (int k = threadIdx.x; k < g; k += 32) {
    a = fmax(a, part[2 * k]);
    m = fmax(m, part[2 * k + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  if (threadIdx.x == 0) out[0] = (m > 0.0) ? a / m : a;
}

}  // namespace

void launch_lift(const double* bflux, double* ux, double* uy, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_lift, dim3(grid_for((long long)(n + 1) * n)), dim3(kThreads), 0, s, bflux, ux, uy, n);
}
void launch_block_sources(const double* f, const double* ux, const double* uy, double* FH, double* absF,
                          int n, int b, cudaStream_t s) {
  const int nc = n / b;
  TG_COUNT(1);
  launch(k_block_sources, dim3(nc * nc), dim3(kThreads), 0, s, f, ux, uy, FH, absF, n, b);
}
// The RT0 particular flux runs in one CTA with (nc + nblocks) FP64 values in
// dynamic shared memory; grids whose values exceed the default 48 KB get the
// larger carve-out here, before any capture (0 when they exceed the device).
int configure_rt_particular(int nc, int nblocks) {
  const size_t shm = sizeof(double) * (size_t)(nc + nblocks);
  if (shm <= 48 * 1024) return 0;
  int dev = 0, maxopt = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      shm > (size_t)maxopt)
    return -1;
  return cudaFuncSetAttribute(k_rt_particular, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) == cudaSuccess
             ? 0
             : -1;
}
void launch_rt_particular(const double* FH, const double* absF, double* gx, double* gy, int nc, double H,
                          int nblocks, PcgState* st, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_rt_particular, dim3(1), dim3(256), sizeof(double) * (size_t)(nc + nblocks), s, FH, absF, gx, gy, nc, H, nblocks, st);
}
void launch_add_rt_field(const double* gx, const double* gy, double* ux, double* uy, int n, int b,
                         cudaStream_t s) {
  TG_COUNT(1);
  launch(k_add_rt_field, dim3(grid_for((long long)(n + 1) * n)), dim3(kThreads), 0, s, gx, gy, ux, uy, n, b);
}
void launch_face_residual(const double* ux, const double* uy, const double* kinv, double* rho, int n,
                          cudaStream_t s) {
  TG_COUNT(1);
  launch(k_face_residual, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, ux, uy, kinv, rho, n);
}
void launch_add_curl(const double* psi, double* ux, double* uy, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_add_curl, dim3(grid_for((long long)(n + 1) * n)), dim3(kThreads), 0, s, psi, ux, uy, n);
}
void launch_block_particular(const double* f, double* ux, double* uy, int n, int b, cudaStream_t s) {
  const int nc = n / b;
  TG_COUNT(1);
  launch(k_block_particular, dim3(nc * nc), dim3(32), 0, s, f, ux, uy, n, b);
}
void launch_psi_from_faces(const double* ux0, const double* vx, double* colbuf, double* psi, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_psi_from_faces, dim3(n), dim3(256), 0, s, ux0, vx, colbuf, psi, n);
}

void launch_pressure(const double* ux, const double* uy, const double* kinv, double* p, double* work,
                     int n, cudaStream_t s) {
  double* rowp = work;
  double* step = work + (long long)n * n;
  double* rowsum = step + n + 1;
  TG_COUNT(1);
  launch(k_pressure_rows, dim3(n), dim3(256), 0, s, ux, kinv, rowp, n);
  TG_COUNT(1);
  launch(k_pressure_steps, dim3(n), dim3(128), 0, s, uy, kinv, rowp, step, rowsum, n);
  TG_COUNT(1);
  launch(k_pressure_offsets, dim3(1), dim3(256), sizeof(double) * (size_t)n, s, step, rowsum, n);
  TG_COUNT(1);
  launch(k_pressure_final, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, rowp, step, p, n);
}
void launch_div_error(const double* ux, const double* uy, const double* f, double* part, double* out,
                      int n, cudaStream_t s) {
  const int g = grid_for((long long)n * n) > kRedGrid ? kRedGrid : grid_for((long long)n * n);
  TG_COUNT(1);
  launch(k_div_error, dim3(g), dim3(kThreads), 0, s, ux, uy, f, part, n);
  TG_COUNT(1);
  launch(k_div_error_final, dim3(1), dim3(32), 0, s, part, g, out);
}

}  // namespace tg
