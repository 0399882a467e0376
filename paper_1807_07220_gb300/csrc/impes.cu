// Two-phase flow by IMPES (Section 6.2): the total mobility that turns the
// saturation into the pressure equation's permeability (eqs. mobility,
// pressure equ), and the explicit upstream-weighted saturation update of eq.
// DisSatEq_Implicit with a CFL time step.
//
// Relative permeabilities k_rw = s^2, k_ro = (1 - s)^2; porosity 1; cell
// volume h^2.  Sources f > 0 inject water, f < 0 produce at the cell's
// fractional flow; a boundary face with inward flux injects water, one with
// outward flux carries its cell's fractional flow.
#include <algorithm>
#include <mutex>

#include "../../include/tgms.h"
#include "common.cuh"

namespace tg {
namespace {

constexpr int kTrThreads = 256;
constexpr int kTrMaxGrid = 4096;

// partial maxima of the CFL reduction, the reduction's arrival counter and
// the time step, shared by every call on a device (calls must not overlap)
__device__ double g_tr_part[kTrMaxGrid];
__device__ unsigned int g_tr_count;
__device__ double g_tr_dt;

__device__ __forceinline__ double frac_flow(double s, double mw, double mo) {
  const double w = s * s / mw;
  return w / (w + (1.0 - s) * (1.0 - s) / mo);
}

__global__ void k_total_mobility(const double* __restrict__ kappa, const double* __restrict__ s, long long nn,
                                 double mw, double mo, double* __restrict__ out) {
  pdl_entry();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = s[t];
    out[t] = kappa[t] * (v * v / mw + (1.0 - v) * (1.0 - v) / mo);
  }
}

// largest total outflow of a cell (outgoing face fluxes u h plus the sink
// h^2 max(-f, 0)); the last CTA forms dt = cfl h^2 / (F_max sigma), or takes
// dt_fixed when it is positive
__global__ void k_transport_outflow(const double* __restrict__ ux, const double* __restrict__ uy,
                                    const double* __restrict__ f, int n, double cfl, double sigma,
                                    double dt_fixed) {
  pdl_entry();
  __shared__ double sh[kTrThreads / 32];
  __shared__ bool last;
  const double h = 1.0 / n;
  const long long nn = (long long)n * n;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    const double ul = ux[(long long)j * (n + 1) + i], ur = ux[(long long)j * (n + 1) + i + 1];
    const double ub = uy[(long long)j * n + i], ut = uy[(long long)(j + 1) * n + i];
    const double out = (((fmax(ur, 0.0) + fmax(-ul, 0.0)) + fmax(ut, 0.0)) + fmax(-ub, 0.0)) * h +
                       h * h * fmax(-f[t], 0.0);
    m = fmax(m, out);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, sh[w]);
    g_tr_part[blockIdx.x] = b;
    __threadfence();
    last = (atomicAdd(&g_tr_count, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last CTA reduces the partial maxima with all its threads
  __threadfence();
  double fmx = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) fmx = fmax(fmx, __ldcg(g_tr_part + k));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fmx = fmax(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = fmx;
  __syncthreads();
  if (threadIdx.x != 0) return;
  fmx = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fmx = fmax(fmx, sh[w]);
  g_tr_count = 0;
  g_tr_dt = (dt_fixed > 0.0) ? dt_fixed : ((fmx > 0.0) ? cfl * h * h / (fmx * sigma) : 0.0);
}

// s_out = s + dt / h^2 (q+ - sum of upstream-weighted water fluxes out + f_w(s) q-).
// One CTA per kTx x kTy tile of cells: f_w of the tile and its one-cell halo
// is formed once in shared memory (one division per cell instead of five).
constexpr int kTx = 32, kTy = 8;
__global__ void __launch_bounds__(kTx * kTy) k_transport(const double* __restrict__ s, const double* __restrict__ ux,
                                                        const double* __restrict__ uy, const double* __restrict__ f,
                                                        int n, double mw, double mo, double* __restrict__ s_out) {
  pdl_entry();
  __shared__ double fw[kTy + 2][kTx + 2];
  const double h = 1.0 / n, dt = g_tr_dt;
  const int i0 = blockIdx.x * kTx, j0 = blockIdx.y * kTy;
  for (int t = threadIdx.x; t < (kTx + 2) * (kTy + 2); t += blockDim.x) {
    const int a = t % (kTx + 2), c = t / (kTx + 2);
    const int i = i0 + a - 1, j = j0 + c - 1;
    fw[c][a] = (i >= 0 && i < n && j >= 0 && j < n) ? frac_flow(s[(long long)j * n + i], mw, mo) : 0.0;
  }
  __syncthreads();
  const int a = threadIdx.x % kTx, c = threadIdx.x / kTx;
  const int i = i0 + a, j = j0 + c;
  if (i >= n || j >= n) return;
  const long long t = (long long)j * n + i;
  const double fc = fw[c + 1][a + 1];
  const double ul = ux[(long long)j * (n + 1) + i], ur = ux[(long long)j * (n + 1) + i + 1];
  const double ub = uy[(long long)j * n + i], ut = uy[(long long)(j + 1) * n + i];
  double upl, upr, upb, upt;   // fraction carried by each face: the cell the flow leaves; water from outside
  if (i == 0) upl = (ul > 0.0) ? 1.0 : fc;
  else upl = (ul >= 0.0) ? fw[c + 1][a] : fc;
  if (i == n - 1) upr = (ur >= 0.0) ? fc : 1.0;
  else upr = (ur >= 0.0) ? fc : fw[c + 1][a + 2];
  if (j == 0) upb = (ub > 0.0) ? 1.0 : fc;
  else upb = (ub >= 0.0) ? fw[c][a + 1] : fc;
  if (j == n - 1) upt = (ut >= 0.0) ? fc : 1.0;
  else upt = (ut >= 0.0) ? fc : fw[c + 2][a + 1];
  const double net = (ur * h * upr - ul * h * upl) + (ut * h * upt - ub * h * upb);
  const double qp = h * h * fmax(f[t], 0.0), qm = h * h * fmin(f[t], 0.0);
  s_out[t] = s[t] + dt / (h * h) * ((qp - net) + fc * qm);
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return TG_OK;
  return (e == cudaErrorMemoryAllocation) ? TG_ERR_OOM : TG_ERR_CUDA;
}

int grid_for_cells(long long nn) {
  long long g = (nn + kTrThreads - 1) / kTrThreads;
  return (int)std::max<long long>(1, std::min<long long>(g, kTrMaxGrid));
}

// sigma = largest df_w/ds = 2 s (1 - s) / (mu_w mu_o lambda^2) over 20001
// equally spaced saturations of [0, 1]
double max_slope(double mw, double mo) {
  const int samples = 20001;
  double best = 0.0;
  for (int k = 0; k < samples; ++k) {
    const double s = k / (samples - 1.0);
    const double lam = s * s / mw + (1.0 - s) * (1.0 - s) / mo;
    best = std::max(best, 2.0 * s * (1.0 - s) / (mw * mo * lam * lam));
  }
  return best;
}

}  // namespace
}  // namespace tg

using namespace tg;

extern "C" {

int tg_total_mobility(const double* kappa, const double* s, int n, double mu_w, double mu_o, double* kappa_out,
                      void* stream) {
  if (!kappa || !s || !kappa_out || n < 1 || !(mu_w > 0) || !(mu_o > 0)) return TG_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nn = (long long)n * n;
  launch(k_total_mobility, dim3(grid_for_cells(nn)), dim3(kTrThreads), 0, st, kappa, s, nn, mu_w, mu_o, kappa_out);
  int rc = cuda_rc(cudaStreamSynchronize(st));
  return rc ? rc : cuda_rc(cudaGetLastError());
}

int tg_transport_step(const double* s, const double* ux, const double* uy, const double* f, int n, double cfl,
                      double dt_fixed, double mu_w, double mu_o, double* s_out, double* dt, void* stream) {
  if (!s || !ux || !uy || !f || !s_out || n < 1 || !(mu_w > 0) || !(mu_o > 0) || (dt_fixed <= 0 && !(cfl > 0)))
    return TG_ERR_INVALID_ARG;
  if (s == s_out) return TG_ERR_INVALID_ARG;   // neighbours are read while cells are written
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nn = (long long)n * n;
  static std::mutex mu;
  static double sigma_cache[2] = {-1.0, -1.0}, sigma_val = 0.0;
  double sigma;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (sigma_cache[0] != mu_w || sigma_cache[1] != mu_o) {
      sigma_val = max_slope(mu_w, mu_o);
      sigma_cache[0] = mu_w;
      sigma_cache[1] = mu_o;
    }
    sigma = sigma_val;
  }
  const int grid = grid_for_cells(nn);
  launch(k_transport_outflow, dim3(grid), dim3(kTrThreads), 0, st, ux, uy, f, n, cfl, sigma, dt_fixed);
  launch(k_transport, dim3((n + kTx - 1) / kTx, (n + kTy - 1) / kTy), dim3(kTx * kTy), 0, st, s, ux, uy, f, n, mu_w,
         mu_o, s_out);
  TG_COUNT(2);
  int rc = TG_OK;
  if (dt) rc = cuda_rc(cudaMemcpyFromSymbolAsync(dt, g_tr_dt, sizeof(double), 0, cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
  return rc ? rc : cuda_rc(cudaGetLastError());
}

}  // extern "C"
