// Nested-dissection solve of the SPD coarse system (Section 5: the coarse
// problem, like every subdomain problem, is solved by a direct method).
//
// One level of dissection by coarse block rows.  A coarse unknown couples to
// another only through a coarse block that both basis functions cover, so the
// unknowns of one row of coarse nodes (the nodal functions of the row and the
// zero-flux functions of its horizontal coarse faces) separate the unknowns
// below the row from those above it.  S - 1 such rows split the rest into S
// strips of block rows whose interiors are mutually uncoupled.  The factor
// keeps, per strip t, the inverse of the interior block A_t and
// X_t = A_t^{-1} A_{t,S}; and the inverse of the separator Schur complement
// Sigma = A_SS - sum_t A_{S,t} X_t.  All FP64.  A solve reads
// sum_t (n_t^2 + 2 n_t m_t) + NS^2 matrix entries (n_t interior and m_t
// adjacent separator unknowns of strip t, NS separator unknowns in all)
// instead of the D^2 of the dense inverse, in four launches.
#include <algorithm>
#include <vector>

#include "../../include/tgms.h"
#include "common.cuh"

namespace tg {
namespace {

constexpr int kThreads = 256;

// out[i * ldo + j] = K[rows[i] * D + cols[j]]
__global__ void k_nd_gather(const double* __restrict__ K, long long D, const int* __restrict__ rows, int nr,
                            const int* __restrict__ cols, int ncol, double* __restrict__ out, long long ldo) {
  const long long m = (long long)nr * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / ncol), j = (int)(t % ncol);
    out[i * ldo + j] = K[(long long)rows[i] * D + cols[j]];
  }
}

// out (nc x nr, ld ldo) = in (nr x nc, ld ldi)^T
__global__ void k_nd_transpose(const double* __restrict__ in, int nr, int ncol, long long ldi,
                               double* __restrict__ out, long long ldo) {
  const long long m = (long long)nr * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % nr), j = (int)(t / nr);
    out[j * ldo + i] = in[i * ldi + j];
  }
}

// c[i] = sum of the slot partials of the unknown at position i
__global__ void k_nd_rhs(const double* __restrict__ part, const int* __restrict__ gatherp, double* __restrict__ c,
                         int D, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gatherp[4 * i + k];
      if (g >= 0) v += part[g];
    }
    c[i] = v;
  }
}

// One warp's dot product of a matrix row (read once, through the
// non-coherent path) with x, kDot = 8 loads of each in flight per lane
// before any is used, so a row of n entries costs n / 256 memory round trips
// (the ragged GEMVs: 46.4 -> 42.3 and 25.0 -> 19.3 us per launch at 1024^2
// with 8 x 8 blocks; the separator GEMV, whose x is staged in shared memory,
// measured slower with it and keeps four accumulators).
constexpr int kDot = 8;
__device__ __forceinline__ double row_dot(const double* __restrict__ mr, const double* __restrict__ xr, int len,
                                          int lane) {
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int base = 0; base < len; base += 32 * kDot) {
    double m[kDot], x[kDot];
#pragma unroll
    for (int u = 0; u < kDot; ++u) {
      const int j = base + lane + 32 * u;
      m[u] = j < len ? __ldg(mr + j) : 0.0;
      x[u] = j < len ? xr[j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kDot; ++u) a[u & 3] = fma(m[u], x[u], a[u & 3]);
  }
  return warp_sum((a[0] + a[1]) + (a[2] + a[3]));
}

// Ragged batch of dense GEMVs, one warp per row.  kBack = false:
// out[row.out] = acc (w and the X_t^T c_t contributions); kBack = true:
// d[perm[row.out]] = w[row.out] - acc (the interior unknowns).
template <bool kBack>
__global__ void __launch_bounds__(kThreads) k_nd_gemv(const double* __restrict__ M, const NdRow* __restrict__ rows,
                                                      int nrows, const double* __restrict__ x,
                                                      const double* __restrict__ w, double* __restrict__ out,
                                                      const int* __restrict__ perm, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + warp; r < nrows; r += gridDim.x * nw) {
    const NdRow row = rows[r];
    const double acc = row_dot(M + row.m, x + row.x0, row.len, lane);
    if (lane == 0) {
      if constexpr (kBack) out[perm[row.out]] = w[row.out] - acc;
      else out[row.out] = acc;
    }
  }
}

// Separator solve: every CTA stages g = c_S - (contributions of the strips
// below and above each separator) in shared memory, then y_S = Sigma^{-1} g
// one warp per row; y_S goes to ysep (for the interiors) and to d.
__global__ void __launch_bounds__(kThreads) k_nd_sep(const double* __restrict__ Y, int NS, int DI,
                                                     const double* __restrict__ c, const double* __restrict__ wh,
                                                     double* __restrict__ ysep, double* __restrict__ d,
                                                     const int* __restrict__ perm, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  extern __shared__ double g[];
  for (int i = threadIdx.x; i < NS; i += blockDim.x) g[i] = c[DI + i] - wh[DI + i] - wh[DI + NS + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < NS; row += gridDim.x * nw) {
    const double* yr = Y + (long long)row * NS;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = lane;
    for (; j + 96 < NS; j += 128) {
      a0 += __ldg(yr + j) * g[j];
      a1 += __ldg(yr + j + 32) * g[j + 32];
      a2 += __ldg(yr + j + 64) * g[j + 64];
      a3 += __ldg(yr + j + 96) * g[j + 96];
    }
    for (; j < NS; j += 32) a0 += __ldg(yr + j) * g[j];
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) {
      ysep[row] = acc;
      d[perm[DI + row]] = acc;
    }
  }
}

int grid_cap(long long cnt, int per, int cap) {
  long long g = (cnt + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

int ck(cudaError_t e) {
  if (e == cudaSuccess) return TG_OK;
  return e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA;
}

// Strip boundaries r_0 = 0 < r_1 < ... < r_S = nc (block rows), evenly split.
std::vector<int> strip_rows(int S, int nc) {
  std::vector<int> r(S + 1);
  for (int t = 0; t <= S; ++t) r[t] = (int)((long long)t * nc / S);
  return r;
}

}  // namespace

int sm_count();

void nd_free(NdFactor& f) {
  cudaFree(f.perm);
  cudaFree(f.gatherp);
  cudaFree(f.M);
  cudaFree(f.rows_a);
  cudaFree(f.rows_b);
  f = NdFactor{};
}

int nd_build(const double* K, int D, const std::vector<int>& key, int nc, const int* gather, NdFactor& f,
             int* status, cudaStream_t s) {
  if (nc < 4 || D <= 0 || (int)key.size() != D) {
    nd_free(f);
    return TG_ERR_UNSUPPORTED;
  }
  const int nkeys = 2 * nc;
  std::vector<std::vector<int>> byk(nkeys);
  for (int u = 0; u < D; ++u) {
    if (key[u] < 1 || key[u] >= nkeys) {
      nd_free(f);
      return TG_ERR_UNSUPPORTED;
    }
    byk[key[u]].push_back(u);
  }
  // number of strips: the fewest matrix entries read per solve, every strip
  // at least two block rows, the separators within the staged limit
  int S = 0;
  double best = 0.0;
  for (int cand = 2; cand <= nc / 2; ++cand) {
    const std::vector<int> r = strip_rows(cand, nc);
    std::vector<double> nt(cand, 0.0), ns(cand - 1, 0.0);
    double NS = 0.0;
    for (int t = 0; t < cand; ++t)
      for (int k = 2 * r[t] + 1; k < 2 * r[t + 1]; ++k) nt[t] += (double)byk[k].size();
    for (int q = 0; q + 1 < cand; ++q) NS += (ns[q] = (double)byk[2 * r[q + 1]].size());
    if (NS > kNdSepMax) continue;
    double entries = NS * NS;
    for (int t = 0; t < cand; ++t) {
      const double m = (t >= 1 ? ns[t - 1] : 0.0) + (t + 1 < cand ? ns[t] : 0.0);
      entries += nt[t] * nt[t] + 2.0 * nt[t] * m;
    }
    if (S == 0 || entries < best) {
      S = cand;
      best = entries;
    }
  }
  if (S == 0) {
    nd_free(f);
    return TG_ERR_UNSUPPORTED;
  }
  const std::vector<int> r = strip_rows(S, nc);

  // order: interiors strip by strip, then the separators
  std::vector<int> perm;
  perm.reserve(D);
  std::vector<int> o(S + 1, 0), sepoff(S, 0);
  for (int t = 0; t < S; ++t) {
    o[t] = (int)perm.size();
    for (int k = 2 * r[t] + 1; k < 2 * r[t + 1]; ++k) perm.insert(perm.end(), byk[k].begin(), byk[k].end());
  }
  const int DI = (int)perm.size();
  o[S] = DI;
  for (int q = 0; q + 1 < S; ++q) {
    sepoff[q] = (int)perm.size() - DI;
    const std::vector<int>& v = byk[2 * r[q + 1]];
    perm.insert(perm.end(), v.begin(), v.end());
  }
  const int NS = (int)perm.size() - DI;
  sepoff[S - 1] = NS;
  if ((int)perm.size() != D) {   // a key outside every strip and separator
    nd_free(f);
    return TG_ERR_UNSUPPORTED;
  }

  // matrix layout and row tables
  std::vector<long long> offa(S), offe(S);
  std::vector<int> nt(S), st0(S), mt(S);
  long long total = 0;
  for (int t = 0; t < S; ++t) {
    nt[t] = o[t + 1] - o[t];
    st0[t] = sepoff[std::max(t - 1, 0)];
    mt[t] = sepoff[std::min(t + 1, S - 1)] - st0[t];
    offa[t] = total;
    total += (long long)(nt[t] + mt[t]) * nt[t];
  }
  for (int t = 0; t < S; ++t) {
    offe[t] = total;
    total += (long long)nt[t] * mt[t];
  }
  const long long y_off = total;
  total += (long long)NS * NS;
  std::vector<NdRow> ra, rb;
  ra.reserve((size_t)DI + 2 * NS);
  rb.reserve(DI);
  for (int t = 0; t < S; ++t) {
    for (int i = 0; i < nt[t]; ++i) ra.push_back(NdRow{offa[t] + (long long)i * nt[t], o[t], nt[t], o[t] + i});
    for (int j = 0; j < mt[t]; ++j) {
      const int p = st0[t] + j;
      const int slot = (t >= 1 && p < sepoff[t]) ? 1 : 0;   // 1: the strip lies above separator t - 1
      ra.push_back(NdRow{offa[t] + (long long)(nt[t] + j) * nt[t], o[t], nt[t], DI + slot * NS + p});
    }
    for (int i = 0; i < nt[t]; ++i) rb.push_back(NdRow{offe[t] + (long long)i * mt[t], st0[t], mt[t], o[t] + i});
  }
  // slot ids in position order
  std::vector<int> g4((size_t)4 * D), gp((size_t)4 * D);
  int rc = ck(cudaMemcpy(g4.data(), gather, sizeof(int) * g4.size(), cudaMemcpyDeviceToHost));
  if (rc) return rc;
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < 4; ++k) gp[4 * (size_t)i + k] = g4[4 * (size_t)perm[i] + k];

  // the buffers of a factor of the same structure are kept (graphs hold their addresses)
  const bool reuse = f.M && f.D == D && f.DI == DI && f.NS == NS && f.strips == S && f.total == total &&
                     f.nrows_a == (int)ra.size() && f.nrows_b == (int)rb.size();
  if (!reuse) {
    nd_free(f);
    rc = ck(cudaMalloc(&f.perm, sizeof(int) * D));
    if (!rc) rc = ck(cudaMalloc(&f.gatherp, sizeof(int) * 4 * (size_t)D));
    if (!rc) rc = ck(cudaMalloc(&f.M, sizeof(double) * (size_t)total));
    if (!rc) rc = ck(cudaMalloc(&f.rows_a, sizeof(NdRow) * std::max<size_t>(1, ra.size())));
    if (!rc) rc = ck(cudaMalloc(&f.rows_b, sizeof(NdRow) * std::max<size_t>(1, rb.size())));
  }
  // Per-strip work (the interior block, its inverse, X_t and X_t^T) runs on
  // up to kNdStreams streams; strips of fewer than 3 kGjBlock unknowns are
  // inverted by one CTA (k_gj_small) rather than one launch per pivot.  The
  // Schur updates of Sigma follow in two colours (even strips, then odd:
  // strips of one colour touch disjoint separator blocks), then Sigma^{-1}.
  constexpr int kNdStreams = 8;
  const int nss = std::min(S, kNdStreams);
  std::vector<cudaStream_t> ss(nss, nullptr);
  std::vector<cudaEvent_t> ev(nss + 1, nullptr);
  std::vector<double*> G(nss, nullptr);
  double *T = nullptr, *GS = nullptr;
  int* bad = nullptr;
  size_t max_n2 = 1, sum_t = 1;
  for (int t = 0; t < S; ++t) {
    max_n2 = std::max(max_n2, (size_t)nt[t] * nt[t]);
    sum_t += (size_t)nt[t] * mt[t];
  }
  std::vector<long long> toff(S + 1, 0);   // per strip A_{t,S} (kept for the Schur updates)
  for (int t = 0; t < S; ++t) toff[t + 1] = toff[t] + (long long)nt[t] * mt[t];
  for (int k = 0; k < nss && !rc; ++k) {
    rc = ck(cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking));
    if (!rc) rc = ck(cudaMalloc(&G[k], sizeof(double) * max_n2));
  }
  for (int k = 0; k <= nss && !rc; ++k) rc = ck(cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming));
  if (!rc) rc = ck(cudaMalloc(&T, sizeof(double) * sum_t));
  if (!rc) rc = ck(cudaMalloc(&GS, sizeof(double) * std::max<size_t>(1, (size_t)NS * NS)));
  if (!rc) rc = ck(cudaMalloc(&bad, sizeof(int)));
  if (!rc) rc = ck(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (!rc) rc = ck(cudaMemcpyAsync(f.perm, perm.data(), sizeof(int) * D, cudaMemcpyHostToDevice, s));
  if (!rc) rc = ck(cudaMemcpyAsync(f.gatherp, gp.data(), sizeof(int) * gp.size(), cudaMemcpyHostToDevice, s));
  if (!rc && !ra.empty())
    rc = ck(cudaMemcpyAsync(f.rows_a, ra.data(), sizeof(NdRow) * ra.size(), cudaMemcpyHostToDevice, s));
  if (!rc && !rb.empty())
    rc = ck(cudaMemcpyAsync(f.rows_b, rb.data(), sizeof(NdRow) * rb.size(), cudaMemcpyHostToDevice, s));
  // the streams start after what s has enqueued, and s continues after all of them
  auto fork = [&]() {
    cudaEventRecord(ev[nss], s);
    for (int k = 0; k < nss; ++k) cudaStreamWaitEvent(ss[k], ev[nss], 0);
  };
  auto join = [&]() {
    for (int k = 0; k < nss; ++k) {
      cudaEventRecord(ev[k], ss[k]);
      cudaStreamWaitEvent(s, ev[k], 0);
    }
  };
  if (!rc) {
    const int* ps = f.perm + DI;
    double* Y = f.M + y_off;
    // Sigma starts as A_SS
    k_nd_gather<<<grid_cap((long long)NS * NS, 256, 4096), 256, 0, s>>>(K, D, ps, NS, ps, NS, Y, NS);
    fork();
    for (int t = 0; t < S; ++t) {
      const int n = nt[t], m = mt[t];
      if (n == 0) continue;
      cudaStream_t st = ss[t % nss];
      const int* pt = f.perm + o[t];
      double* Ai = f.M + offa[t];
      double* X = f.M + offe[t];
      double* Tt = T + toff[t];
      k_nd_gather<<<grid_cap((long long)n * n, 256, 4096), 256, 0, st>>>(K, D, pt, n, pt, n, Ai, n);
      if (n < 3 * kGjBlock) launch_gj_small(Ai, n, bad, st);                           // A_t^{-1}
      else launch_gauss_jordan(Ai, G[t % nss], n, status, st);
      if (m == 0) continue;
      k_nd_gather<<<grid_cap((long long)n * m, 256, 4096), 256, 0, st>>>(K, D, pt, n, ps + st0[t], m, Tt, m);
      launch_dgemm(n, m, n, 1.0, Ai, n, 1, Tt, m, 1, 0.0, X, m, st);                   // X_t = A_t^{-1} A_{t,S}
      k_nd_transpose<<<grid_cap((long long)n * m, 256, 4096), 256, 0, st>>>(X, n, m, m, Ai + (long long)n * n, n);
    }
    join();
    for (int colour = 0; colour < 2; ++colour) {   // Sigma -= A_{S,t} X_t
      fork();
      for (int t = colour, q = 0; t < S; t += 2, ++q) {
        const int n = nt[t], m = mt[t];
        if (n == 0 || m == 0) continue;
        launch_dgemm(m, m, n, -1.0, T + toff[t], 1, m, f.M + offe[t], m, 1, 1.0,
                     Y + (long long)st0[t] * NS + st0[t], NS, ss[q % nss]);
      }
      join();
    }
    launch_gauss_jordan(Y, GS, NS, status, s);                                         // Sigma^{-1}
    rc = ck(cudaStreamSynchronize(s));
  }
  int h_bad = 0;
  if (!rc) rc = ck(cudaMemcpy(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (!rc && h_bad) rc = TG_ERR_BREAKDOWN;   // a strip block with a non-positive pivot: not SPD
  for (int k = 0; k < nss; ++k) {
    if (ss[k]) cudaStreamDestroy(ss[k]);
    cudaFree(G[k]);
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  cudaFree(T);
  cudaFree(GS);
  cudaFree(bad);
  if (!rc) rc = ck(cudaGetLastError());
  if (!rc && NS * sizeof(double) > 48 * 1024)
    rc = ck(cudaFuncSetAttribute(k_nd_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(NS * sizeof(double))));
  if (rc) {
    if (!reuse) nd_free(f);   // kept buffers stay allocated: a captured solve must not read freed memory
    return rc;
  }
  f.D = D;
  f.DI = DI;
  f.NS = NS;
  f.strips = S;
  f.nrows_a = (int)ra.size();
  f.nrows_b = (int)rb.size();
  f.y_off = y_off;
  f.total = total;
  f.bytes = 8.0 * (double)total;   // every stored entry is read once per solve
  return TG_OK;
}

void launch_nd_solve(const NdFactor& f, const double* part, double* d, const PcgState* st, cudaStream_t s) {
  const int D = f.D;
  double* c = d + D;
  double* wh = d + 2 * (size_t)D;
  double* ysep = d + 4 * (size_t)D;
  const int cap = 8 * sm_count();
  TG_COUNT(4);
  launch(k_nd_rhs, dim3(grid_cap(D, kThreads, cap)), dim3(kThreads), 0, s, part, (const int*)f.gatherp, c, D, st);
  launch(k_nd_gemv<false>, dim3(grid_cap(f.nrows_a, kThreads / 32, cap)), dim3(kThreads), 0, s, (const double*)f.M,
         (const NdRow*)f.rows_a, f.nrows_a, (const double*)c, (const double*)nullptr, wh, (const int*)nullptr, st);
  launch(k_nd_sep, dim3(grid_cap(f.NS, kThreads / 32, 2 * sm_count())), dim3(kThreads), sizeof(double) * (size_t)f.NS,
         s, (const double*)(f.M + f.y_off), f.NS, f.DI, (const double*)c, (const double*)wh, ysep, d,
         (const int*)f.perm, st);
  launch(k_nd_gemv<true>, dim3(grid_cap(f.nrows_b, kThreads / 32, cap)), dim3(kThreads), 0, s, (const double*)f.M,
         (const NdRow*)f.rows_b, f.nrows_b, (const double*)ysep, (const double*)wh, d, (const int*)f.perm, st);
}

}  // namespace tg
