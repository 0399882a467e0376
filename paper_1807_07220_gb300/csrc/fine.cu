// Kernels of one PCG iteration on the reduced (divergence-free) problem in
// stream-function form: fine operator, vector updates with on-device
// scalars, patch smoother (eq. smooth), coarse restriction / solve /
// prolongation (eq. coarsepre).
//
// Scalar reductions use the "last CTA" pattern: every CTA writes its partial
// sum, fences, and bumps an arrival counter; the CTA that arrives last sums
// the partials in a fixed order and updates PcgState.  Consumers read the
// scalars in the next kernel, so no CTA ever reads a value written in its own
// launch.  Every kernel of the loop returns at once when PcgState::done is set.
#include <cstdlib>
#include <type_traits>

#include "common.cuh"

namespace tg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// Writes this CTA's partial and returns true in every thread of the CTA that
// arrived last (whose threads may then read all partials of the launch).
__device__ __forceinline__ bool arrive_last(double partial, double* part, unsigned int* counter) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = partial;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ bool arrive_last_linear(double partial, double* part, unsigned int* counter,
                                                   unsigned int bid, unsigned int nblk) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[bid] = partial;
    __threadfence();
    const unsigned int t = atomicAdd(counter, 1u);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Exact float -> double from the IEEE 754 fields (sign kept, exponent
// rebiased from 127 to 1023, the 23 fraction bits moved to the top of the 52)
// on the integer pipe: the FP64 pipe, the bound of the kernels that widen a
// preconditioned vector, stays free.  Zeros, subnormals, infinities and NaNs
// take the conversion instruction.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}
__device__ __forceinline__ double widen(double d) { return d; }

// Sums K arrays of m partials (array k at part + k m) in the CTA that
// arrived last, with all of its threads: thread t adds entries t, t + T, ...
// of every array (the loads of one pass issued before its adds), then one
// block-wide tree.  The order is fixed by m and the block size, so the sums
// are reproducible.  Every thread of the CTA must call it; out is valid in
// thread 0.
template <int K>
__device__ __forceinline__ void block_sum_partials(const double* part, int m, double (&out)[K]) {
  __shared__ double shp[K][32];
  double s[K];
#pragma unroll
  for (int k = 0; k < K; ++k) s[k] = 0.0;
  int t = threadIdx.x;
  for (; t + 3 * (int)blockDim.x < m; t += 4 * blockDim.x) {
    double v[K][4];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int u = 0; u < 4; ++u) v[k][u] = __ldcg(part + (long long)k * m + t + u * blockDim.x);
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] += (v[k][0] + v[k][1]) + (v[k][2] + v[k][3]);
  }
  for (; t < m; t += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) s[k] += __ldcg(part + (long long)k * m + t);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s[k] = warp_sum(s[k]);
    if (l == 0) shp[k][w] = s[k];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = warp_sum(l < nw ? shp[k][l] : 0.0);
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_apply_operator(const double* __restrict__ psi,
                                                             const double* __restrict__ kinv,
                                                             double* __restrict__ out, int n) {
  pdl_entry();
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    out[t] = (i == 0 || j == 0) ? 0.0 : stencil_apply<double, double, double>(psi, kinv, n, i, j);
  }
}

__global__ void __launch_bounds__(kThreads) k_apply_operator_f32(const double* __restrict__ psi,
                                                                 const float* __restrict__ kinv,
                                                                 double* __restrict__ out, int n) {
  pdl_entry();
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    out[t] = (i == 0 || j == 0) ? 0.0 : (double)stencil_apply<double, float, float>(psi, kinv, n, i, j);
  }
}

// out = r - K z  (inner residual of the two-grid cycle, precision TC)
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_residual(const double* __restrict__ r,
                                                       const TC* __restrict__ z,
                                                       const TC* __restrict__ kinv,
                                                       TC* __restrict__ out, int n,
                                                       const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    TC v = (TC)0;
    if (i != 0 && j != 0) v = (TC)r[t] - stencil_apply<TC, TC, TC>(z, kinv, n, i, j);
    out[t] = v;
  }
}

// q = K p_new with p_new = z_prev + beta p_old formed on the fly in a shared
// (32+2) x (8R+2) halo tile (each p_new value computed once), p_new and q
// written, z_next zeroed for the coming smoother accumulation, and
// alpha = rz / (p_new, q) by the last CTA.  Each thread takes R nodes of a
// column (rows ty, ty + 8, ...): on GB300 the kernel is bound by the FP64
// pipe, and R > 1 spreads the CTA's FP64 sum and the halo over more nodes.
constexpr int kTx = 32, kTy = 8;
template <typename TC, int R>
__global__ void __launch_bounds__(kThreads) k_pcg_apply_p(const TC* __restrict__ zprev,
                                                          const double* __restrict__ pold,
                                                          double* __restrict__ pnew, double* __restrict__ q,
                                                          TC* __restrict__ znext,
                                                          const double* __restrict__ kcoef, double* part,
                                                          PcgState* st, int n) {
  pdl_entry();
  // the stop flag is tested once the halo tile is loaded, so its load is not
  // a round trip of its own (the vectors stay valid after convergence, and
  // nothing global is written before the test)
  const int done = st->done;
  constexpr int kRows = kTy * R;
  __shared__ double P[kRows + 2][kTx + 2];
  __shared__ double sh[32];
  const double beta = st->beta;
  const int i0 = blockIdx.x * kTx, j0 = blockIdx.y * kRows;
  for (int t = threadIdx.x; t < (kTx + 2) * (kRows + 2); t += blockDim.x) {
    const int a = t % (kTx + 2), c = t / (kTx + 2);
    const int i = i0 - 1 + a, j = j0 - 1 + c;
    double v = 0.0;
    if (i >= 1 && j >= 1 && i < n && j < n) {
      const long long id = (long long)j * n + i;
      v = widen(zprev[id]) + beta * pold[id];
    }
    P[c][a] = v;
  }
  __syncthreads();
  if (done) return;
  const int tx = threadIdx.x % kTx, ty0 = threadIdx.x / kTx;
  const int i = i0 + tx;
  const long long nn = (long long)n * n;
  // K p with the node coefficients (c0, cE, cN, cNE, cNW); the west, south,
  // south-west and south-east couplings are the neighbours' east, north,
  // north-east and north-west ones (K is symmetric)
  const double* c0 = kcoef;
  const double* cE = kcoef + nn;
  const double* cN = kcoef + 2 * nn;
  const double* cNE = kcoef + 3 * nn;
  const double* cNW = kcoef + 4 * nn;
  double acc = 0.0;
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int ty = ty0 + kTy * u, j = j0 + ty;
    if (i < n && j < n) {
      const long long id = (long long)j * n + i;
      const double p0 = P[ty + 1][tx + 1];
      double qv = 0.0;
      if (i >= 1 && j >= 1) {
        qv = c0[id] * p0;
        qv = fma(cE[id], P[ty + 1][tx + 2], qv);
        qv = fma(cN[id], P[ty + 2][tx + 1], qv);
        qv = fma(cNE[id], P[ty + 2][tx + 2], qv);
        qv = fma(cNW[id], P[ty + 2][tx], qv);
        qv = fma(cE[id - 1], P[ty + 1][tx], qv);
        qv = fma(cN[id - n], P[ty][tx + 1], qv);
        qv = fma(cNE[id - n - 1], P[ty][tx], qv);
        qv = fma(cNW[id - n + 1], P[ty][tx + 2], qv);
      }
      pnew[id] = p0;
      q[id] = qv;
      znext[id] = (TC)0;
      acc = fma(p0, qv, acc);
    }
  }
  acc = block_sum(acc, sh);
  const unsigned int bid = blockIdx.y * gridDim.x + blockIdx.x, nblk = gridDim.x * gridDim.y;
  if (arrive_last_linear(acc, part, &st->counter[0], bid, nblk)) {
    double sum[1];
    block_sum_partials<1>(part, nblk, sum);
    const double pq = sum[0];
    if (threadIdx.x == 0) {
      st->counter[0] = 0;
      st->pq = pq;
      const double alpha = st->rz / pq;
      if (!(pq > 0.0) || !isfinite(alpha)) {
        st->status |= kStBreakdown;
        st->done = 1;
        st->alpha = 0.0;
      } else {
        st->alpha = alpha;
        if (st->iter < kMaxHist) st->alphas[st->iter] = alpha;
      }
    }
  }
}

// (r, r), (r, z) and (z, q) of the iteration's new residual r and
// preconditioned residual z: the last CTA counts the iteration and tests
// convergence on (r, r) (the stopping rule), then forms beta
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_pcg_dots(const double* __restrict__ r,
                                                       const TC* __restrict__ z,
                                                       const double* __restrict__ q,
                                                       double* part, PcgState* st, int n) {
  pdl_entry();
  const int done = st->done;   // tested after the loads (see k_pcg_apply_p)
  const long long nn = (long long)n * n;
  double a = 0.0, b = 0.0, c = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // four grid strides per pass, all loads issued before the sums (same
  // order of the sums as one stride at a time)
  for (; t + 3 * stride < nn; t += 4 * stride) {
    double zv[4], rv[4], qv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zv[u] = widen(z[t + u * stride]);
      rv[u] = r[t + u * stride];
      qv[u] = q[t + u * stride];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a += rv[u] * zv[u];
      b += zv[u] * qv[u];
      c += rv[u] * rv[u];
    }
  }
  for (; t < nn; t += stride) {
    const double zv = widen(z[t]), rv = r[t];
    a += rv * zv;
    b += zv * q[t];
    c += rv * rv;
  }
  if (done) return;
  // the three CTA sums in one pass (one barrier instead of three block sums)
  {
    __shared__ double sh3[3][32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) {
      sh3[0][w] = a;
      sh3[1][w] = b;
      sh3[2][w] = c;
    }
    __syncthreads();
    if (w == 0) {
      a = warp_sum(l < nw ? sh3[0][l] : 0.0);
      b = warp_sum(l < nw ? sh3[1][l] : 0.0);
      c = warp_sum(l < nw ? sh3[2][l] : 0.0);
    }
  }
  // three partial arrays: part[0..grid), part[grid..2 grid), part[2 grid..3 grid)
  if (threadIdx.x == 0) {
    part[gridDim.x + blockIdx.x] = b;
    part[2 * gridDim.x + blockIdx.x] = c;
  }
  if (arrive_last(a, part, &st->counter[2])) {
    double sum[3];
    block_sum_partials<3>(part, gridDim.x, sum);
    const double rz = sum[0], zq = sum[1], rr = sum[2];
    if (threadIdx.x == 0) {
      st->counter[2] = 0;
      st->rr = rr;
      st->iter += 1;
      if (rr <= st->rtol2 * st->rr0) {
        st->done = 1;
        return;
      } else if (!isfinite(rr)) {
        st->status |= kStBreakdown;
        st->done = 1;
        return;
      } else if (st->iter >= st->maxit) {
        st->status |= kStMaxIter;
        st->done = 1;
        return;
      }
      const double beta = st->flexible ? (-st->alpha * zq / st->rz) : (rz / st->rz);
      if (!(rz > 0.0) || !isfinite(beta)) {
        st->status |= kStBreakdown;
        st->done = 1;
      }
      st->zq = zq;
      st->beta = beta;
      if (st->iter - 1 < kMaxHist) st->betas[st->iter - 1] = beta;
      st->rz_prev = st->rz;
      st->rz = rz;
    }
  }
}

// scalar state at the start of a solve (rtol read from device memory so that
// an instantiated graph serves every tolerance)
__global__ void k_pcg_reset(PcgState* st, const double* __restrict__ rtol, int maxit, int flexible) {
  pdl_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->rz = st->rz_prev = st->rr0 = st->rr = 0.0;
  st->alpha = st->beta = st->pq = st->zq = 0.0;
  st->rtol2 = rtol[0] * rtol[0];
  st->iter = 0;
  st->maxit = maxit;
  st->done = 0;
  st->status = 0;
  st->flexible = flexible;
  for (int k = 0; k < 4; ++k) st->counter[k] = 0u;
}

// loop condition of the graph's while node: continue while not done
__global__ void k_set_condition(cudaGraphConditionalHandle cond, const PcgState* st) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// x = 0, rr0 = (r, r)
__global__ void __launch_bounds__(kThreads) k_pcg_init(double* __restrict__ x,
                                                       const double* __restrict__ r, double* part,
                                                       PcgState* st, int n) {
  pdl_entry();
  __shared__ double sh[32];
  const long long nn = (long long)n * n;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    x[t] = 0.0;
    acc += r[t] * r[t];
  }
  acc = block_sum(acc, sh);
  if (arrive_last(acc, part, &st->counter[3])) {
    double sum[1];
    block_sum_partials<1>(part, gridDim.x, sum);
    const double rr = sum[0];
    if (threadIdx.x == 0) {
      st->counter[3] = 0;
      st->rr0 = rr;
      st->rr = rr;
      st->iter = 0;
      if (rr == 0.0) st->done = 1;
      if (!isfinite(rr)) {
        st->status |= kStBreakdown;
        st->done = 1;
      }
    }
  }
}

// warm start: r = rho - K x (FP64), rr = (r, r); the stopping reference is the
// zero-guess residual, rr0 = (rho, rho), so a good guess needs fewer iterations
// for the same target
__global__ void __launch_bounds__(kThreads) k_pcg_init_warm(const double* __restrict__ x,
                                                            const double* __restrict__ rho,
                                                            const double* __restrict__ kinv,
                                                            double* __restrict__ r, double* part,
                                                            PcgState* st, int n) {
  pdl_entry();
  __shared__ double sh[32];
  const long long nn = (long long)n * n;
  double a = 0.0, b = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    double v = 0.0;
    if (i != 0 && j != 0) v = rho[t] - stencil_apply<double, double, double>(x, kinv, n, i, j);
    r[t] = v;
    a += v * v;
    b += rho[t] * rho[t];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = b;
  if (arrive_last(a, part, &st->counter[3])) {
    double sum[2];
    block_sum_partials<2>(part, gridDim.x, sum);
    const double rr = sum[0], rr0 = sum[1];
    if (threadIdx.x == 0) {
      st->counter[3] = 0;
      st->rr0 = rr0;
      st->rr = rr;
      st->iter = 0;
      if (rr0 == 0.0 || rr <= st->rtol2 * rr0) st->done = 1;
      if (!isfinite(rr) || !isfinite(rr0)) {
        st->status |= kStBreakdown;
        st->done = 1;
      }
    }
  }
}

// p = z, rz = (r, z)
template <typename TC>
__global__ void __launch_bounds__(kThreads) k_pcg_init_rz(const double* __restrict__ r,
                                                          const TC* __restrict__ z,
                                                          double* __restrict__ p, double* part,
                                                          PcgState* st, int n) {
  pdl_entry();
  if (st->done) return;
  __shared__ double sh[32];
  const long long nn = (long long)n * n;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const double zv = widen(z[t]);
    p[t] = zv;
    acc += r[t] * zv;
  }
  acc = block_sum(acc, sh);
  if (arrive_last(acc, part, &st->counter[3])) {
    double sum[1];
    block_sum_partials<1>(part, gridDim.x, sum);
    const double rz = sum[0];
    if (threadIdx.x == 0) {
      st->counter[3] = 0;
      st->rz = rz;
      st->rz_prev = rz;
      st->beta = 0.0;
      if (!(rz > 0.0) || !isfinite(rz)) {
        st->status |= kStBreakdown;
        st->done = 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Smoother: one CTA per oversampled patch.  Gather the residual on the
// patch's interior nodes, multiply by the stored inverse of the local
// operator (row per warp, vectorised loads), scatter eta * result with
// atomics (patches overlap).
template <typename TS> struct Vec;
template <> struct Vec<double> { static constexpr int W = 2; };
template <> struct Vec<float> { static constexpr int W = 4; };
template <> struct Vec<__nv_bfloat16> { static constexpr int W = 8; };

// raw vector chunk of W storage elements (16 bytes) and its dot product
template <typename TS> struct Chunk;
template <> struct Chunk<double> { using T = double2; };
template <> struct Chunk<float> { using T = float4; };
template <> struct Chunk<__nv_bfloat16> { using T = uint4; };
template <typename TS>
__device__ __forceinline__ typename Chunk<TS>::T load_chunk(const TS* m) {
  return __ldg(reinterpret_cast<const typename Chunk<TS>::T*>(m));
}
template <typename TC>
__device__ __forceinline__ TC dot_raw(const double2& v, const TC* x) {
  return (TC)(v.x * (double)x[0] + v.y * (double)x[1]);
}
template <typename TC>
__device__ __forceinline__ TC dot_raw(const float4& v, const TC* x) {
  return (TC)(v.x * x[0] + v.y * x[1] + v.z * x[2] + v.w * x[3]);
}
template <typename TC>
__device__ __forceinline__ TC dot_raw(const uint4& v, const TC* x) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
  TC acc = (TC)0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    acc += f.x * x[2 * k] + f.y * x[2 * k + 1];
  }
  return acc;
}
template <typename TC>
__device__ __forceinline__ TC dot_chunk_smem(const double* m, const TC* x) {
  return dot_raw<TC>(*reinterpret_cast<const double2*>(m), x);
}
template <typename TC>
__device__ __forceinline__ TC dot_chunk_smem(const float* m, const TC* x) {
  return dot_raw<TC>(*reinterpret_cast<const float4*>(m), x);
}
template <typename TC>
__device__ __forceinline__ TC dot_chunk_smem(const __nv_bfloat16* m, const TC* x) {
  return dot_raw<TC>(*reinterpret_cast<const uint4*>(m), x);
}
template <typename TS> struct RowsPerPass { static constexpr int R = 4; };
template <> struct RowsPerPass<double> { static constexpr int R = 2; };

// Register-staged smoother tiles: kCB bytes per lane load (8 or 16) and kR
// rows reduced together per pass.  A 368-entry bfloat16 row is 46 16-byte
// chunks (two passes of 32 lanes, 72% of the slots used) or 92 8-byte chunks
// (three passes, 96%); the autotuner picks per handle.
template <typename TS, int kCB> struct LdChunk;
template <> struct LdChunk<double, 16> { using T = double2; };
template <> struct LdChunk<float, 16> { using T = float4; };
template <> struct LdChunk<float, 8> { using T = float2; };
template <> struct LdChunk<__nv_bfloat16, 16> { using T = uint4; };
template <> struct LdChunk<__nv_bfloat16, 8> { using T = uint2; };
template <> struct LdChunk<__half, 16> { using T = uint4; };
template <> struct LdChunk<__half, 8> { using T = uint2; };
template <typename TS, int kCB>
__device__ __forceinline__ typename LdChunk<TS, kCB>::T load_tile(const TS* m) {
  return __ldg(reinterpret_cast<const typename LdChunk<TS, kCB>::T*>(m));
}
template <typename TC>
__device__ __forceinline__ TC dot_raw(const float2& v, const TC* x) {
  return (TC)(v.x * x[0] + v.y * x[1]);
}
template <typename TC>
__device__ __forceinline__ TC dot_raw(const uint2& v, const TC* x) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
  TC acc = (TC)0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    acc += f.x * x[2 * k] + f.y * x[2 * k + 1];
  }
  return acc;
}
// FP16 chunks (8 or 4 halves), products in FP32
template <typename TC, typename V>
__device__ __forceinline__ TC dot_half(const V& v, const TC* x) {
  constexpr int P = (int)(sizeof(V) / sizeof(__half2));
  const __half2* h = reinterpret_cast<const __half2*>(&v);
  TC acc = (TC)0;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const float2 f = __half22float2(h[k]);
    acc += f.x * x[2 * k] + f.y * x[2 * k + 1];
  }
  return acc;
}
template <typename TS, typename TC, typename V>
__device__ __forceinline__ TC dot_tile(const V& v, const TC* x) {
  if constexpr (std::is_same<TS, __half>::value) return dot_half<TC>(v, x);
  else return dot_raw<TC>(v, x);
}

template <typename TC>
__device__ __forceinline__ TC dot_chunk(const double* m, const TC* x) {
  const double2 v = *reinterpret_cast<const double2*>(m);
  return (TC)(v.x * (double)x[0] + v.y * (double)x[1]);
}
template <typename TC>
__device__ __forceinline__ TC dot_chunk(const float* m, const TC* x) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(m));
  return (TC)(v.x * x[0] + v.y * x[1] + v.z * x[2] + v.w * x[3]);
}
template <typename TC>
__device__ __forceinline__ TC dot_chunk(const __nv_bfloat16* m, const TC* x) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(m));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
  TC acc = (TC)0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(h[k]);
    acc += f.x * x[2 * k] + f.y * x[2 * k + 1];
  }
  return acc;
}

constexpr int kPatchLd = ((kMaxPatchNodes + 7) / 8) * 8;
constexpr int kRowsPerWarp = kRowsPerGroup;

// The rows of all patch inverses are cut into groups of kRowsPerWarp rows;
// gofs[p] is the first group of patch p.  The grid is one wave of CTAs and
// CTA k owns the contiguous group range [k G/grid, (k+1) G/grid): for each
// patch it touches it gathers the patch residual into shared memory, then its
// warps stream their groups (vector loads, the rows of a group in flight
// together) and scatter eta * (M x) with atomics (patches overlap).
// With kFused the sweep also performs the PCG update: the residual it
// smooths is r_new = r_old - alpha q, formed at gather time; the CTA that owns
// the first row group of patch p writes r_new and x += alpha p on the nodes of
// block p (blocks partition the nodes, and r_old is never written here).
// (r_new, r_new) and the stopping test are left to k_pcg_dots, which reads
// r_new anyway.
struct FuseArgs {
  const double* r_old;
  double* r_new;
  const double* q;
  double* x;
  const double* p;
  double* part;
  PcgState* st;
  int nc, b;
  void* zclear;         // mode 1: z buffer zeroed on the owned nodes (or NULL)
  const void* zin;      // mode 2: z before the sweep (TC), read for the residual
  const void* kin;      // mode 2: inverse permeabilities (TC)
};

// the chains of a lock-step group (k_smoother_multi): per chain the vector
// gathered (mode 2: r; mode 1 reads fa.r_old), the output z, the PCG state
// and the fused-update arguments; slots k .. kGroup-1 are absent
template <typename TC>
struct ChainSet {
  const double* r[kGroup];
  TC* zacc[kGroup];
  const PcgState* st[kGroup];
  FuseArgs fa[kGroup];
  int k;
};

// q / nx for a patch node q < kPatchLd and a patch side nx <= kMaxPatchSide:
// q * ceil(2^16 / nx) / 2^16 exceeds q / nx by less than kPatchLd / 2^16 < 1 / nx,
// so the shift gives the exact quotient with two integer operations
__device__ __forceinline__ int patch_row(int q, int mul16) { return (q * mul16) >> 16; }
__device__ __forceinline__ int patch_mul16(int nx) { return (65536 + nx - 1) / nx; }
static_assert(kMaxPatchSide * kPatchLd < 65536 && kPatchLd * 65536LL < (1LL << 31),
              "the multiply-shift quotient stays exact and q * mul16 fits an int");

// The residual of patch p gathered into xs[0 .. fill) (zero past nloc), with
// the fused work of kFused (see k_smoother): mode 1 forms r - alpha q and,
// where this CTA owns block p, writes r and x += alpha p there and clears
// the other z buffer; mode 2 forms r - K z_in and the owner seeds the output
// with z_in.
// the residual at patch node q (zero past nloc), as the sweep of kFused forms it
template <typename TC, typename TR, int kFused>
__device__ __forceinline__ TC smoother_value(const PatchGeo& g, int q, const TR* __restrict__ r, int n,
                                             const FuseArgs& fa, double alpha, int mul16) {
  TC v = (TC)0;
  if (q < g.nloc) {
    const int c = patch_row(q, mul16), a = q - c * g.nx;
    const long long id = (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a);
    if constexpr (kFused == 1) v = (TC)(fa.r_old[id] - alpha * fa.q[id]);
    else if constexpr (kFused == 2)
      v = (TC)r[id] - stencil_apply<TC, TC, TC>((const TC*)fa.zin, (const TC*)fa.kin, n, g.x0 + 1 + a,
                                                g.y0 + 1 + c);
    else v = (TC)r[id];
  }
  return v;
}
template <typename TC, int kFused>
__device__ __forceinline__ void smoother_owner(int p, bool owner, TC* __restrict__ zacc, int n, const FuseArgs& fa,
                                               double alpha);
template <typename TC, typename TR, int kFused>
__device__ __forceinline__ void smoother_gather(const PatchGeo& g, int p, bool owner, const TR* __restrict__ r,
                                                TC* __restrict__ zacc, int n, const FuseArgs& fa, double alpha,
                                                TC* xs, int fill) {
  const int mul16 = patch_mul16(g.nx);
  for (int q = threadIdx.x; q < fill; q += blockDim.x)
    xs[q] = smoother_value<TC, TR, kFused>(g, q, r, n, fa, alpha, mul16);
  smoother_owner<TC, kFused>(p, owner, zacc, n, fa, alpha);
}
template <typename TC, int kFused>
__device__ __forceinline__ void smoother_owner(int p, bool owner, TC* __restrict__ zacc, int n, const FuseArgs& fa,
                                               double alpha) {
  if (kFused == 1 && owner) {   // this CTA owns block p
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      const double rv = fa.r_old[id] - alpha * fa.q[id];
      fa.r_new[id] = rv;
      fa.x[id] += alpha * fa.p[id];
      if (fa.zclear) ((TC*)fa.zclear)[id] = (TC)0;
    }
  }
  if (kFused == 2 && owner) {   // the owner seeds the output with z_in
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      atomicAdd(zacc + id, ((const TC*)fa.zin)[id]);
    }
  }
}

// kFused: 0 plain sweep z += eta S r; 1 first sweep of an iteration (r - alpha q
// formed at gather time, r and x updated by the block owners); 2 last sweep
// with the residual formed at gather time,
// r_in = r - K z_in, into a z buffer that the owners seed with z_in.
template <typename TC, typename TS, typename TR, int kFused, int kCB, int kR, bool kPipe>
__global__ void __launch_bounds__(kThreads) k_smoother(const PatchGeo* __restrict__ geo,
                                                       const int* __restrict__ gofs, int npatch,
                                                       const TS* __restrict__ pinv,
                                                       const TR* __restrict__ r,
                                                       TC* __restrict__ zacc, TC eta, int n,
                                                       const PcgState* st, FuseArgs fa,
                                                       const float* __restrict__ rscale) {
  pdl_entry();
  const int done = st ? st->done : 0;   // tested after the first loads (see k_pcg_apply_p)
  __shared__ __align__(16) TC xs[kPatchLd];
  __shared__ double shr[32];
  const double alpha = (kFused == 1) ? fa.st->alpha : 0.0;
  const int G = gofs[npatch];
  const long long per = ((long long)G + gridDim.x - 1) / gridDim.x;
  const int g0 = (int)min((long long)G, blockIdx.x * per), g1 = (int)min((long long)G, g0 + per);
  // last patch with gofs[p] <= g0: gofs is strictly increasing (every patch
  // has at least one row group), so exactly one thread finds p with
  // gofs[p] <= g0 < gofs[p+1] in one round of loads (none when g0 = G: the
  // CTA is empty and p = npatch - 1 as a bisection would give)
  __shared__ int sp;
  if (threadIdx.x == 0) sp = npatch - 1;
  __syncthreads();
  for (int t = threadIdx.x; t < npatch; t += blockDim.x)
    if (gofs[t] <= g0 && gofs[t + 1] > g0) sp = t;
  __syncthreads();
  if (done) return;
  int p = sp;
  constexpr int W = kCB / (int)sizeof(TS);
  constexpr int kIter = (kPatchLd + 32 * W - 1) / (32 * W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (; g0 < g1 && p < npatch && gofs[p] < g1; ++p) {
    const PatchGeo g = geo[p];
    __syncthreads();
    smoother_gather<TC, TR, kFused>(g, p, gofs[p] >= g0, r, zacc, n, fa, alpha, xs, g.ld);
    __syncthreads();
    const int ga = max(g0, gofs[p]) - gofs[p], gb = min(g1, gofs[p + 1]) - gofs[p];
    const TS* M = pinv + g.off;
    constexpr int R = kR;
    constexpr int P = kRowsPerWarp / R;   // passes per row group
    using V = typename LdChunk<TS, kCB>::T;
    // every load of R rows first (predicated, zero-filled) ...
    auto load_rows = [&](V (&buf)[R][kIter], int row0) {
#pragma unroll
      for (int it = 0; it < kIter; ++it) {
        const int col = (it * 32 + lane) * W;
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (col < g.ld && row0 + k < g.nloc) buf[k][it] = load_tile<TS, kCB>(M + (long long)(row0 + k) * g.ld + col);
          else buf[k][it] = V{};
        }
      }
    };
    // ... then the arithmetic, the warp reductions and the scatter
    auto reduce_rows = [&](const V (&buf)[R][kIter], int row0) {
      TC acc[R];
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] = (TC)0;
#pragma unroll
      for (int it = 0; it < kIter; ++it) {
        const int col = (it * 32 + lane) * W;
        if (col < g.ld) {
#pragma unroll
          for (int k = 0; k < R; ++k) acc[k] += dot_tile<TS, TC>(buf[k][it], xs + col);
        }
      }
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] = warp_sum(acc[k]);
      if (lane < R && row0 + lane < g.nloc) {
        TC v = acc[0];
#pragma unroll
        for (int k = 1; k < R; ++k)
          if (lane == k) v = acc[k];
        const int q = row0 + lane, a = q % g.nx, c = q / g.nx;
        if constexpr (std::is_same<TS, __half>::value) v *= (TC)rscale[(long long)gofs[p] * kRowsPerWarp + q];
        atomicAdd(zacc + (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a), eta * v);
      }
    };
    if constexpr (!kPipe) {
      for (int grp = ga + warp; grp < gb; grp += nw) {
#pragma unroll
        for (int pass = 0; pass < P; ++pass) {
          const int row0 = grp * kRowsPerWarp + pass * R;
          V buf[R][kIter];
          load_rows(buf, row0);
          reduce_rows(buf, row0);
        }
      }
    } else {
      // software pipeline: the rows of pass t+1 are in flight while pass t is reduced
      const int ngrp = (gb > ga + warp) ? (gb - ga - warp + nw - 1) / nw : 0;
      const int nseq = ngrp * P;
      auto row_at = [&](int t) { return (ga + warp + (t / P) * nw) * kRowsPerWarp + (t % P) * R; };
      V bA[R][kIter], bB[R][kIter];
      if (nseq > 0) load_rows(bA, row_at(0));
      for (int t = 0; t < nseq; t += 2) {
        if (t + 1 < nseq) load_rows(bB, row_at(t + 1));
        reduce_rows(bA, row_at(t));
        if (t + 1 < nseq) {
          if (t + 2 < nseq) load_rows(bA, row_at(t + 2));
          reduce_rows(bB, row_at(t + 1));
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core variant (tile shape kShapeTensor, BF16 / FP16 storage).  The
// CUDA-core sweep spends two instructions per stored 2-byte entry (unpack,
// FMA) plus a warp reduction per row, and at grids whose inverses stay in L2
// that instruction stream, not the bytes, bounds it.  Here a warp takes
// 16-row tiles of a patch inverse: per 16 x 16 tile one 16-byte load per lane
// (the tiles are stored in A-fragment order) and one mma.m16n8k16 against
// B = [x_hi x_mid x_lo 0 ...], the residual split into three 2-byte parts
// (x = x_hi + x_mid + x_lo to 2^-24 relative), FP32 accumulation.  The row
// result is the sum of the first three accumulator columns.  FP16 storage
// scales the residual by a per-patch power of two (its largest magnitude in
// [2^14, 2^15)) before the split and undoes it with the row scale.  Gather
// and fused modes are those of k_smoother, with 16-row tiles (tofs) in place
// of 4-row groups.  When the wave holds at least one CTA per patch, each
// patch's tiles are cut evenly among k = grid / npatch CTAs (one gather per
// CTA, no search); otherwise CTAs take equal contiguous tile ranges, as
// k_smoother takes row groups.
static_assert((kMaxPatchNodes + kTile - 1) / kTile * kTile <= kPatchLd, "the tile rows must fit the shared residual");
constexpr int kTileBatch = 8;   // tiles of a row in flight per lane

template <typename TS> struct MmaTile;
template <> struct MmaTile<__nv_bfloat16> {
  static __device__ __forceinline__ unsigned short to16(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
  static __device__ __forceinline__ float from16(unsigned short v) {
    return __bfloat162float(__ushort_as_bfloat16(v));
  }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint4& a, const uint2& b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  }
};
template <> struct MmaTile<__half> {
  static __device__ __forceinline__ unsigned short to16(float x) { return __half_as_ushort(__float2half_rn(x)); }
  static __device__ __forceinline__ float from16(unsigned short v) { return __half2float(__ushort_as_half(v)); }
  static __device__ __forceinline__ void mma(float (&d)[4], const uint4& a, const uint2& b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
  }
};
// part k (0, 1, 2) of x: each part is the 2-byte rounding of what the
// previous parts leave (each difference is exact in FP32)
template <typename TS>
__device__ __forceinline__ unsigned part16(float x, int k) {
  unsigned short v = MmaTile<TS>::to16(x);
  for (int t = 0; t < k; ++t) {
    x -= MmaTile<TS>::from16(v);
    v = MmaTile<TS>::to16(x);
  }
  return v;
}

template <typename TC, typename TS, typename TR, int kFused>
__global__ void __launch_bounds__(kThreads, 4) k_smoother_mma(const PatchGeo* __restrict__ geo,
                                                           const int* __restrict__ tofs,
                                                           const int* __restrict__ gofs, int npatch,
                                                           const TS* __restrict__ tiles,
                                                           const TR* __restrict__ r,
                                                           TC* __restrict__ zacc, TC eta, int n,
                                                           const PcgState* st, FuseArgs fa,
                                                           const float* __restrict__ rscale) {
  pdl_entry();
  const int done = st ? st->done : 0;   // tested after the first loads (see k_pcg_apply_p)
  constexpr bool kHalf = std::is_same<TS, __half>::value;
  __shared__ __align__(16) TC xs[kPatchLd];
  __shared__ __align__(16) uint2 xb[(kPatchLd / kTile) * 12];
  const double alpha = (kFused == 1) ? fa.st->alpha : 0.0;
  int t0, t1;
  __shared__ int sp;
  if (gridDim.x >= (unsigned)npatch && gridDim.x % npatch == 0) {
    const int k = gridDim.x / npatch, pp = blockIdx.x / k, piece = blockIdx.x % k;
    const int base = tofs[pp], nt = tofs[pp + 1] - base;
    t0 = base + piece * nt / k;
    t1 = base + (piece + 1) * nt / k;
    if (threadIdx.x == 0) sp = pp;
    __syncthreads();
  } else {
    const int RT = tofs[npatch];
    const long long per = ((long long)RT + gridDim.x - 1) / gridDim.x;
    t0 = (int)min((long long)RT, blockIdx.x * per);
    t1 = (int)min((long long)RT, t0 + per);
    // the patch holding tile t0 (tofs strictly increasing; see k_smoother)
    if (threadIdx.x == 0) sp = npatch - 1;
    __syncthreads();
    for (int t = threadIdx.x; t < npatch; t += blockDim.x)
      if (tofs[t] <= t0 && tofs[t + 1] > t0) sp = t;
    __syncthreads();
  }
  if (done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int p = sp; t0 < t1 && p < npatch && tofs[p] < t1; ++p) {
    const PatchGeo g = geo[p];
    const int T = tiles_per_side(g.nloc);
    __syncthreads();
    float sx = 1.0f, unscale = 1.0f;
    if constexpr (!kHalf) {
      // BF16 needs no scale: each thread gathers a pair of adjacent nodes and
      // writes its three parts straight into the B fragments (lane 4 k + c of
      // k-tile j holds columns 16 j + 2 c + {0, 1} in its first word, + 8 in
      // its second)
      const int mul16 = patch_mul16(g.nx);
      for (int t = threadIdx.x; t < T * (kTile / 2); t += blockDim.x) {
        const int q0 = 2 * t, j = q0 / kTile, w = q0 % kTile, c = (w & 7) >> 1, half = w >> 3;
        const float v0 = (float)smoother_value<TC, TR, kFused>(g, q0, r, n, fa, alpha, mul16);
        const float v1 = (float)smoother_value<TC, TR, kFused>(g, q0 + 1, r, n, fa, alpha, mul16);
#pragma unroll
        for (int k = 0; k < 3; ++k)
          reinterpret_cast<unsigned*>(&xb[j * 12 + 4 * k + c])[half] = part16<TS>(v0, k) | (part16<TS>(v1, k) << 16);
      }
      smoother_owner<TC, kFused>(p, tofs[p] >= t0, zacc, n, fa, alpha);
    } else {
      smoother_gather<TC, TR, kFused>(g, p, tofs[p] >= t0, r, zacc, n, fa, alpha, xs, T * kTile);
      __syncthreads();
      // every warp forms the patch's residual scale
      float m = 0.0f;
      for (int q = lane; q < g.nloc; q += 32) m = fmaxf(m, fabsf((float)xs[q]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (m > 0.0f) {
        int e = 0;
        frexpf(m, &e);
        sx = ldexpf(1.0f, 15 - e);
        unscale = ldexpf(1.0f, e - 15);
      }
      // B fragments: lane l < 12 of k-tile j holds part l / 4 of x at columns
      // 16 j + 2 (l % 4) + {0, 1} and the same + 8; lanes 12..31 hold zeros
      for (int e = threadIdx.x; e < T * 12; e += blockDim.x) {
        const int j = e / 12, l = e % 12, k = l >> 2, c0 = kTile * j + 2 * (l & 3);
        auto pk = [&](int q) { return part16<TS>((float)xs[q] * sx, k); };
        xb[e] = make_uint2(pk(c0) | (pk(c0 + 1) << 16), pk(c0 + 8) | (pk(c0 + 9) << 16));
      }
    }
    __syncthreads();
    const int ta = max(t0, tofs[p]) - tofs[p], tb = min(t1, tofs[p + 1]) - tofs[p];
    const uint4* A = reinterpret_cast<const uint4*>(tiles + g.toff) + lane;
    for (int i = ta + warp; i < tb; i += nw) {
      // two accumulators (even and odd k-tiles), so consecutive mma do not wait on each other
      float d[4] = {0.0f, 0.0f, 0.0f, 0.0f}, d2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const uint4* Ai = A + (long long)i * T * 32;
      for (int j0 = 0; j0 < T; j0 += kTileBatch) {
        uint4 a[kTileBatch];
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) a[u] = (j0 + u < T) ? __ldg(Ai + (j0 + u) * 32) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < kTileBatch; ++u) {
          if (j0 + u < T) {   // uniform over the warp
            const uint2 bv = (lane < 12) ? xb[(j0 + u) * 12 + lane] : make_uint2(0u, 0u);
            if (u & 1) MmaTile<TS>::mma(d2, a[u], bv);
            else MmaTile<TS>::mma(d, a[u], bv);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) d[k] += d2[k];
      // lane 4 g holds columns 0 and 1 (hi, mid) of rows g and g + 8, lane 4 g + 1 column 2 (lo)
      const float lo0 = __shfl_down_sync(0xffffffffu, d[0], 1), lo1 = __shfl_down_sync(0xffffffffu, d[2], 1);
      if ((lane & 3) == 0) {
        const float y[2] = {d[0] + d[1] + lo0, d[2] + d[3] + lo1};
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int q = kTile * i + (lane >> 2) + 8 * hh;
          if (q < g.nloc) {
            TC v = (TC)y[hh];
            if constexpr (kHalf) v *= (TC)(rscale[(long long)gofs[p] * kRowsPerWarp + q] * unscale);
            const int c2 = patch_row(q, patch_mul16(g.nx)), a2 = q - c2 * g.nx;
            atomicAdd(zacc + (long long)(g.y0 + 1 + c2) * n + (g.x0 + 1 + a2), eta * v);
          }
        }
      }
    }
  }
}

// Lock-step tensor-core sweep (k_smoother_multi on the tile layout): up to
// kGroup chains share every A-fragment load; chains 0 and 1 are the columns
// 0-2 and 3-5 of one B operand, chains 2 and 3 of a second, so a tile costs
// one load per lane and one or two mma.  Each chain keeps its own gather,
// fused updates and (FP16) residual scale, and its row sums follow the
// single-chain order ((hi + mid) + lo).
template <typename TC, typename TS, int kFused>
__global__ void __launch_bounds__(kThreads, 4) k_smoother_mma_multi(const PatchGeo* __restrict__ geo,
                                                                    const int* __restrict__ tofs,
                                                                    const int* __restrict__ gofs, int npatch,
                                                                    const TS* __restrict__ tiles, TC eta, int n,
                                                                    ChainSet<TC> cs,
                                                                    const float* __restrict__ rscale) {
  pdl_entry();
  constexpr bool kHalf = std::is_same<TS, __half>::value;
  constexpr int kPairs = kGroup / 2;
  __shared__ __align__(16) TC xs[kGroup][kPatchLd];
  __shared__ __align__(16) uint2 xb[kPairs][(kPatchLd / kTile) * 24];
  bool act[kGroup];
  int any = 0;
#pragma unroll
  for (int c = 0; c < kGroup; ++c) {
    act[c] = (c < cs.k) && !cs.st[c]->done;
    any |= act[c];
  }
  if (!any) return;
  const bool pair_act[kPairs] = {act[0] || act[1], act[2] || act[3]};
  double alpha[kGroup];
#pragma unroll
  for (int c = 0; c < kGroup; ++c) alpha[c] = (kFused == 1 && act[c]) ? cs.fa[c].st->alpha : 0.0;
  int t0, t1;
  __shared__ int sp;
  if (gridDim.x >= (unsigned)npatch && gridDim.x % npatch == 0) {
    const int k = gridDim.x / npatch, pp = blockIdx.x / k, piece = blockIdx.x % k;
    const int base = tofs[pp], nt = tofs[pp + 1] - base;
    t0 = base + piece * nt / k;
    t1 = base + (piece + 1) * nt / k;
    if (threadIdx.x == 0) sp = pp;
    __syncthreads();
  } else {
    const int RT = tofs[npatch];
    const long long per = ((long long)RT + gridDim.x - 1) / gridDim.x;
    t0 = (int)min((long long)RT, blockIdx.x * per);
    t1 = (int)min((long long)RT, t0 + per);
    if (threadIdx.x == 0) sp = npatch - 1;
    __syncthreads();
    for (int t = threadIdx.x; t < npatch; t += blockDim.x)
      if (tofs[t] <= t0 && tofs[t + 1] > t0) sp = t;
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int p = sp; t0 < t1 && p < npatch && tofs[p] < t1; ++p) {
    const PatchGeo g = geo[p];
    const int T = tiles_per_side(g.nloc);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kGroup; ++c)
      if (act[c])
        smoother_gather<TC, double, kFused>(g, p, tofs[p] >= t0, cs.r[c], cs.zacc[c], n, cs.fa[c], alpha[c], xs[c],
                                            T * kTile);
    __syncthreads();
    float sx[kGroup], unscale[kGroup];
#pragma unroll
    for (int c = 0; c < kGroup; ++c) {
      sx[c] = 1.0f;
      unscale[c] = 1.0f;
      if constexpr (kHalf) {
        if (act[c]) {
          float m = 0.0f;
          for (int q = lane; q < g.nloc; q += 32) m = fmaxf(m, fabsf((float)xs[c][q]));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (m > 0.0f) {
            int e = 0;
            frexpf(m, &e);
            sx[c] = ldexpf(1.0f, 15 - e);
            unscale[c] = ldexpf(1.0f, e - 15);
          }
        }
      }
    }
    // B fragments: lane l < 24 of k-tile j of pair P holds part (l / 4) % 3 of
    // chain 2 P + l / 12 at columns 16 j + 2 (l % 4) + {0, 1} and + 8
    for (int e = threadIdx.x; e < kPairs * T * 24; e += blockDim.x) {
      const int P = e / (T * 24), r2 = e % (T * 24), j = r2 / 24, l = r2 % 24;
      const int c = 2 * P + l / 12, k = (l >> 2) % 3, c0 = kTile * j + 2 * (l & 3);
      uint2 w = make_uint2(0u, 0u);
      if (act[c]) {
        auto pk = [&](int q) { return part16<TS>((float)xs[c][q] * sx[c], k); };
        w = make_uint2(pk(c0) | (pk(c0 + 1) << 16), pk(c0 + 8) | (pk(c0 + 9) << 16));
      }
      xb[P][j * 24 + l] = w;
    }
    __syncthreads();
    const int ta = max(t0, tofs[p]) - tofs[p], tb = min(t1, tofs[p + 1]) - tofs[p];
    const uint4* A = reinterpret_cast<const uint4*>(tiles + g.toff) + lane;
    for (int i = ta + warp; i < tb; i += nw) {
      float d[kPairs][4] = {}, d2[kPairs][4] = {};
      const uint4* Ai = A + (long long)i * T * 32;
      for (int j0 = 0; j0 < T; j0 += 6) {
        uint4 a[6];
#pragma unroll
        for (int u = 0; u < 6; ++u) a[u] = (j0 + u < T) ? __ldg(Ai + (j0 + u) * 32) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          if (j0 + u < T) {   // uniform over the warp
#pragma unroll
            for (int P = 0; P < kPairs; ++P) {
              if (!pair_act[P]) continue;
              const uint2 bv = (lane < 24) ? xb[P][(j0 + u) * 24 + lane] : make_uint2(0u, 0u);
              if (u & 1) MmaTile<TS>::mma(d2[P], a[u], bv);
              else MmaTile<TS>::mma(d[P], a[u], bv);
            }
          }
        }
      }
#pragma unroll
      for (int P = 0; P < kPairs; ++P) {
        if (!pair_act[P]) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) d[P][k] += d2[P][k];
        // chain 2P: columns 0, 1 on lane 4g, column 2 on lane 4g + 1; chain
        // 2P + 1: column 3 on lane 4g + 1, columns 4, 5 on lane 4g + 2
        float y[2][2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const float c0v = d[P][2 * hh], c1v = d[P][2 * hh + 1];
          const float n0 = __shfl_down_sync(0xffffffffu, c0v, 1), n1 = __shfl_down_sync(0xffffffffu, c1v, 1);
          const float m0 = __shfl_down_sync(0xffffffffu, c0v, 2), m1 = __shfl_down_sync(0xffffffffu, c1v, 2);
          y[0][hh] = (c0v + c1v) + n0;
          y[1][hh] = (n1 + m0) + m1;
        }
        if ((lane & 3) == 0) {
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int c = 2 * P + cc;
            if (!act[c]) continue;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int q = kTile * i + (lane >> 2) + 8 * hh;
              if (q < g.nloc) {
                TC v = (TC)y[cc][hh];
                if constexpr (kHalf) v *= (TC)(rscale[(long long)gofs[p] * kRowsPerWarp + q] * unscale[c]);
                const int c2 = patch_row(q, patch_mul16(g.nx)), a2 = q - c2 * g.nx;
                atomicAdd(cs.zacc[c] + (long long)(g.y0 + 1 + c2) * n + (g.x0 + 1 + a2), eta * v);
              }
            }
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Band variant (tile shape kShapeBand): each local problem is solved from its
// band Cholesky factor by the two triangular solves, as the paper's direct
// subdomain solvers do, instead of a product with the stored dense inverse.
// One warp per patch: the residual is gathered into shared memory, then both
// sweeps are right-looking: lane 0 forms the row's value from its pending
// sum, broadcasts it, and lane d adds its band entry's term to the pending
// sum of row j + d (forward) or j - d (backward), held in its registers.
// Lane d loads entry d of four rows at once (the layouts interleave rows in
// groups of four) and keeps 16 rows in flight (8 for FP64, whose wider
// registers would otherwise cost the single wave of patches).  The entries do
// not depend on the sweep, so the chain from row to row is a subtraction, a
// product and two shuffles.  The factor is read once per sweep: n_loc (w + 1)
// values against n_loc^2 for the dense inverse.
constexpr int kBandWarps = 4;   // patches per CTA
template <typename TC>
constexpr int kBandGroupsOf = sizeof(TC) == 8 ? kBandPF / 8 : kBandPF / 4;   // row groups in flight per lane
// the sweeps round n_loc up to a multiple of kBandPF: the rows they touch
// must stay inside the shared residual
static_assert(kPatchLd % kBandPF == 0, "row rounding must stay inside the shared residual");
template <typename TC>
struct BandQuad {
  TC v[4];
};
__device__ __forceinline__ BandQuad<float> band_quad(const float* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ BandQuad<double> band_quad(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}
// lanes past the stored band load nothing and hold zeros
template <typename TC>
__device__ __forceinline__ void band_quad_if(bool ln, const TC* p, BandQuad<TC>& q) {
  if (ln) {
    q = band_quad(p);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) q.v[k] = (TC)0;
  }
}
// four consecutive right-hand sides / solution values of the shared patch
// vector (16-byte aligned quads): one shared-memory access per four rows
// instead of one per row
__device__ __forceinline__ void xs_ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void xs_ld4(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void xs_st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void xs_st4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
template <typename TC, typename TR, int kFused>
__global__ void __launch_bounds__(32 * kBandWarps) k_smoother_band(const PatchGeo* __restrict__ geo, int npatch,
                                                                   const TC* __restrict__ band, int ldb,
                                                                   long long pstride, const TR* __restrict__ r,
                                                                   TC* __restrict__ zacc, TC eta, int n,
                                                                   const PcgState* st, FuseArgs fa) {
  pdl_entry();
  if (st && st->done) return;
  __shared__ __align__(16) TC xs_all[kBandWarps][kPatchLd];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kBandWarps + warp;
  if (p >= npatch) return;   // warp-uniform; no block-wide barrier below
  TC* xs = xs_all[warp];
  const PatchGeo g = geo[p];
  const int nloc = g.nloc, w = g.nx + 1;
  const TC* Lc = band + (long long)p * pstride;
  const double alpha = (kFused == 1) ? fa.st->alpha : 0.0;
  for (int q = lane; q < nloc; q += 32) {
    const int a = q % g.nx, c = q / g.nx;
    const long long id = (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a);
    TC v;
    if constexpr (kFused == 1) v = (TC)(fa.r_old[id] - alpha * fa.q[id]);
    else if constexpr (kFused == 2)
      v = (TC)r[id] - stencil_apply<TC, TC, TC>((const TC*)fa.zin, (const TC*)fa.kin, n, g.x0 + 1 + a, g.y0 + 1 + c);
    else v = (TC)r[id];
    xs[q] = v;
  }
  if (kFused == 1) {   // block p's owner work
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = lane; t < b * b; t += 32) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      fa.r_new[id] = fa.r_old[id] - alpha * fa.q[id];
      fa.x[id] += alpha * fa.p[id];
      if (fa.zclear) ((TC*)fa.zclear)[id] = (TC)0;
    }
  }
  if (kFused == 2) {   // the owner seeds the output with z_in
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = lane; t < b * b; t += 32) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      atomicAdd(zacc + id, ((const TC*)fa.zin)[id]);
    }
  }
  // rows past the matrix up to a multiple of kBandPF: zero right-hand side,
  // zero band entries (padding), so they add nothing
  const int nrow = ((nloc + kBandPF - 1) / kBandPF) * kBandPF;
  for (int q = nloc + lane; q < nrow; q += 32) xs[q] = (TC)0;
  __syncwarp();
  // pending sums live in registers: after row j, lane d holds the pending sum
  // of row j + 1 + d (forward) or j - 1 - d (backward); a shuffle down by one
  // lane moves them along as the sweep advances.  Lane d reads entry (j, d) of
  // the column layout (L_{j+d, j}) in the forward sweep and of the row layout
  // (L_{j, j-d}) in the backward one, four rows per load; the padded layouts
  // make every read in range and zero outside the band.
  const bool ln = (lane < ldb);   // lanes past the stored band read nothing
  const long long gs = 4LL * ldb; // one group of four rows
  constexpr int kG = kBandGroupsOf<TC>, kRows = 4 * kG;   // nrow is a multiple of kRows
  static_assert(kBandPF % kRows == 0, "rows per pass must divide the row rounding");
  {
    // group holding rows 0..3, lane's entries
    const TC* G0 = Lc + (long long)(kBandPad / 4) * gs + (ln ? 4 * lane : 0);
    BandQuad<TC> pf[kG];
#pragma unroll
    for (int i = 0; i < kG; ++i) band_quad_if(ln, G0 + i * gs, pf[i]);
    TC acc = (TC)0;
    for (int j0 = 0; j0 < nrow; j0 += kRows) {
      const TC* gp = G0 + (long long)(j0 / 4 + kG) * gs;
#pragma unroll
      for (int i = 0; i < kG; ++i) {
        const BandQuad<TC> cur = pf[i];
        band_quad_if(ln, gp + i * gs, pf[i]);
        TC xv[4], yv[4];
        xs_ld4(xs + j0 + 4 * i, xv);              // rows j0 + 4 i .. + 3
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const TC cj = cur.v[k];
          TC y = (xv[k] - acc) * cj;             // meaningful in lane 0
          y = __shfl_sync(0xffffffffu, y, 0);
          yv[k] = y;
          if (lane != 0) acc = fma(cj, y, acc);
          acc = __shfl_down_sync(0xffffffffu, acc, 1);
        }
        if (lane == 0) xs_st4(xs + j0 + 4 * i, yv);
      }
    }
  }
  __syncwarp();
  {
    // row layout, group holding rows nrow - 4 .. nrow - 1 (row j at v[j % 4])
    const TC* H0 = Lc + pstride / 2 + (long long)((kBandPad + nrow) / 4 - 1) * gs + (ln ? 4 * lane : 0);
    BandQuad<TC> pf[kG];
#pragma unroll
    for (int i = 0; i < kG; ++i) band_quad_if(ln, H0 - i * gs, pf[i]);
    TC acc = (TC)0;
    for (int j0 = nrow - 1; j0 >= 0; j0 -= kRows) {
      const TC* gp = H0 - (long long)((nrow - 1 - j0) / 4 + kG) * gs;
#pragma unroll
      for (int i = 0; i < kG; ++i) {
        const BandQuad<TC> cur = pf[i];
        band_quad_if(ln, gp - i * gs, pf[i]);
        TC xv[4], yv[4];
        xs_ld4(xs + j0 - 4 * i - 3, xv);          // rows j0 - 4 i - 3 .. j0 - 4 i
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const TC cj = cur.v[3 - k];
          TC x = (xv[3 - k] - acc) * cj;         // meaningful in lane 0
          x = __shfl_sync(0xffffffffu, x, 0);
          yv[3 - k] = x;
          if (lane != 0) acc = fma(cj, x, acc);
          acc = __shfl_down_sync(0xffffffffu, acc, 1);
        }
        if (lane == 0) xs_st4(xs + j0 - 4 * i - 3, yv);
      }
    }
  }
  __syncwarp();
  for (int q = lane; q < nloc; q += 32) {
    const int a = q % g.nx, c = q / g.nx;
    atomicAdd(zacc + (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a), eta * xs[q]);
  }
}

// FP32 band sweeps with a deeper read-ahead (the handles with FP32 factors).
// The sweep's per-row dependency chain (a broadcast and a shift by
// shuffles, a subtraction, a product, an FMA) takes far less than an HBM
// round trip per 16 rows, so the register read-ahead of k_smoother_band
// leaves the warp waiting on loads.  Here each lane copies its own 16-byte
// entry quads (entry d of four rows, the grouped layout) with cp.async into
// a per-warp shared-memory ring of kBandRing row groups, kBandRing - 1
// groups (44 rows) ahead of the row being solved; a lane reads only what it
// copied, so no cross-lane synchronisation is needed, and copies are issued
// only for stored row groups.  Same arithmetic and order as k_smoother_band.
constexpr int kBandRing = 12;
__device__ __forceinline__ void band_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void band_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void band_cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename TR, int kFused>
__global__ void __launch_bounds__(32 * kBandWarps) k_smoother_band_ring(const PatchGeo* __restrict__ geo, int npatch,
                                                                        const float* __restrict__ band, int ldb,
                                                                        long long pstride,
                                                                        const TR* __restrict__ r,
                                                                        float* __restrict__ zacc, float eta, int n,
                                                                        const PcgState* st, FuseArgs fa) {
  pdl_entry();
  if (st && st->done) return;
  __shared__ __align__(16) float xs_all[kBandWarps][kPatchLd];
  __shared__ __align__(16) float4 ring_all[kBandWarps][kBandRing][kBandLd];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kBandWarps + warp;
  if (p >= npatch) return;   // warp-uniform; no block-wide barrier below
  float* xs = xs_all[warp];
  float4(*ring)[kBandLd] = ring_all[warp];
  const PatchGeo g = geo[p];
  const int nloc = g.nloc;
  const float* Lc = band + (long long)p * pstride;
  const bool ln = (lane < ldb);   // lanes past the stored band copy and read nothing (ldb <= kBandLd)
  const long long gs = 4LL * ldb; // one group of four rows
  const int nrow = ((nloc + kBandPF - 1) / kBandPF) * kBandPF;
  const int ngrp = nrow / 4;
  // the first groups of the forward sweep are in flight during the gather
  const float* G0 = Lc + (long long)(kBandPad / 4) * gs + (ln ? 4 * lane : 0);
#pragma unroll
  for (int i = 0; i < kBandRing - 1; ++i) {
    if (ln && i < ngrp) band_cp_async16(&ring[i][lane], G0 + i * gs);
    band_cp_commit();
  }
  const double alpha = (kFused == 1) ? fa.st->alpha : 0.0;
  for (int q = lane; q < nloc; q += 32) {
    const int a = q % g.nx, c = q / g.nx;
    const long long id = (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a);
    float v;
    if constexpr (kFused == 1) v = (float)(fa.r_old[id] - alpha * fa.q[id]);
    else if constexpr (kFused == 2)
      v = (float)r[id] - stencil_apply<float, float, float>((const float*)fa.zin, (const float*)fa.kin, n,
                                                           g.x0 + 1 + a, g.y0 + 1 + c);
    else v = (float)r[id];
    xs[q] = v;
  }
  if (kFused == 1) {   // block p's owner work
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = lane; t < b * b; t += 32) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      fa.r_new[id] = fa.r_old[id] - alpha * fa.q[id];
      fa.x[id] += alpha * fa.p[id];
      if (fa.zclear) ((float*)fa.zclear)[id] = 0.0f;
    }
  }
  if (kFused == 2) {   // the owner seeds the output with z_in
    const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
    for (int t = lane; t < b * b; t += 32) {
      const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
      atomicAdd(zacc + id, ((const float*)fa.zin)[id]);
    }
  }
  for (int q = nloc + lane; q < nrow; q += 32) xs[q] = 0.0f;
  __syncwarp();
  // forward sweep, column layout: group k of rows 4k .. 4k + 3 in slot k % kBandRing
  {
    float acc = 0.0f;
    for (int k = 0; k < ngrp; ++k) {
      // group k + kBandRing - 1 into the slot read in the previous step
      if (ln && k + kBandRing - 1 < ngrp)
        band_cp_async16(&ring[(k + kBandRing - 1) % kBandRing][lane], G0 + (long long)(k + kBandRing - 1) * gs);
      band_cp_commit();
      band_cp_wait<kBandRing - 1>();   // group k has landed
      const float4 cur = ln ? ring[k % kBandRing][lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float cv[4] = {cur.x, cur.y, cur.z, cur.w};
      float xv[4], yv[4];
      xs_ld4(xs + 4 * k, xv);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float cj = cv[t];
        float y = (xv[t] - acc) * cj;             // meaningful in lane 0
        y = __shfl_sync(0xffffffffu, y, 0);
        yv[t] = y;
        if (lane != 0) acc = fmaf(cj, y, acc);
        acc = __shfl_down_sync(0xffffffffu, acc, 1);
      }
      if (lane == 0) xs_st4(xs + 4 * k, yv);
    }
  }
  band_cp_wait<0>();
  __syncwarp();
  // backward sweep, row layout: group holding rows nrow - 4 - 4k .. nrow - 1 - 4k
  {
    const float* H0 = Lc + pstride / 2 + (long long)((kBandPad + nrow) / 4 - 1) * gs + (ln ? 4 * lane : 0);
#pragma unroll
    for (int i = 0; i < kBandRing - 1; ++i) {
      if (ln && i < ngrp) band_cp_async16(&ring[i][lane], H0 - i * gs);
      band_cp_commit();
    }
    float acc = 0.0f;
    for (int k = 0; k < ngrp; ++k) {
      if (ln && k + kBandRing - 1 < ngrp)
        band_cp_async16(&ring[(k + kBandRing - 1) % kBandRing][lane], H0 - (long long)(k + kBandRing - 1) * gs);
      band_cp_commit();
      band_cp_wait<kBandRing - 1>();
      const float4 cur = ln ? ring[k % kBandRing][lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float cv[4] = {cur.x, cur.y, cur.z, cur.w};
      float xv[4], yv[4];
      xs_ld4(xs + nrow - 4 - 4 * k, xv);            // rows nrow - 4 - 4 k .. nrow - 1 - 4 k
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float cj = cv[3 - t];
        float x = (xv[3 - t] - acc) * cj;         // meaningful in lane 0
        x = __shfl_sync(0xffffffffu, x, 0);
        yv[3 - t] = x;
        if (lane != 0) acc = fmaf(cj, x, acc);
        acc = __shfl_down_sync(0xffffffffu, acc, 1);
      }
      if (lane == 0) xs_st4(xs + nrow - 4 - 4 * k, yv);
    }
  }
  band_cp_wait<0>();
  __syncwarp();
  for (int q = lane; q < nloc; q += 32) {
    const int a = q % g.nx, c = q / g.nx;
    atomicAdd(zacc + (long long)(g.y0 + 1 + c) * n + (g.x0 + 1 + a), eta * xs[q]);
  }
}

// ---------------------------------------------------------------------------
// Lock-step variant for several right-hand sides of one instance: one read of
// every patch inverse serves up to kGroup PCG chains that run the same
// five-kernel iteration (each chain its own vectors, scalars and state).
// Each chain's rows are reduced exactly as k_smoother reduces them (same
// lanes, same order), so a chain's results do not depend on its group.
// Chains whose PCG has finished (or that are absent, slot >= k) are skipped.
template <typename TC, typename TS, int kFused, int kCB, int kR>
__global__ void __launch_bounds__(kThreads) k_smoother_multi(const PatchGeo* __restrict__ geo,
                                                             const int* __restrict__ gofs, int npatch,
                                                             const TS* __restrict__ pinv, TC eta, int n,
                                                             ChainSet<TC> cs, const float* __restrict__ rscale) {
  pdl_entry();
  __shared__ __align__(16) TC xs[kGroup][kPatchLd];
  __shared__ double shr[32];
  bool act[kGroup];
  int any = 0;
#pragma unroll
  for (int c = 0; c < kGroup; ++c) {
    act[c] = (c < cs.k) && !cs.st[c]->done;
    any |= act[c];
  }
  if (!any) return;
  double alpha[kGroup];
#pragma unroll
  for (int c = 0; c < kGroup; ++c) alpha[c] = (kFused == 1 && act[c]) ? cs.fa[c].st->alpha : 0.0;
  const int G = gofs[npatch];
  const long long per = ((long long)G + gridDim.x - 1) / gridDim.x;
  const int g0 = (int)min((long long)G, blockIdx.x * per), g1 = (int)min((long long)G, g0 + per);
  __shared__ int sp;
  if (threadIdx.x == 0) sp = npatch - 1;
  __syncthreads();
  for (int t = threadIdx.x; t < npatch; t += blockDim.x)
    if (gofs[t] <= g0 && gofs[t + 1] > g0) sp = t;
  __syncthreads();
  int p = sp;
  constexpr int W = kCB / (int)sizeof(TS);
  constexpr int kIter = (kPatchLd + 32 * W - 1) / (32 * W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (; g0 < g1 && p < npatch && gofs[p] < g1; ++p) {
    const PatchGeo g = geo[p];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kGroup; ++c) {
      if (!act[c]) continue;
      const FuseArgs& fa = cs.fa[c];
      for (int q = threadIdx.x; q < g.ld; q += blockDim.x) {
        TC v = (TC)0;
        if (q < g.nloc) {
          const int a = q % g.nx, cc = q / g.nx;
          const long long id = (long long)(g.y0 + 1 + cc) * n + (g.x0 + 1 + a);
          if constexpr (kFused == 1) v = (TC)(fa.r_old[id] - alpha[c] * fa.q[id]);
          else if constexpr (kFused == 2)
            v = (TC)cs.r[c][id] - stencil_apply<TC, TC, TC>((const TC*)fa.zin, (const TC*)fa.kin, n, g.x0 + 1 + a,
                                                            g.y0 + 1 + cc);
          else v = (TC)cs.r[c][id];
        }
        xs[c][q] = v;
      }
      if (kFused == 1 && gofs[p] >= g0) {   // this CTA owns block p
        const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
          const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
          const double rv = fa.r_old[id] - alpha[c] * fa.q[id];
          fa.r_new[id] = rv;
          fa.x[id] += alpha[c] * fa.p[id];
          if (fa.zclear) ((TC*)fa.zclear)[id] = (TC)0;
        }
      }
      if (kFused == 2 && gofs[p] >= g0) {   // the owner seeds the output with z_in
        const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
          const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
          atomicAdd(cs.zacc[c] + id, ((const TC*)fa.zin)[id]);
        }
      }
    }
    __syncthreads();
    const int ga = max(g0, gofs[p]) - gofs[p], gb = min(g1, gofs[p + 1]) - gofs[p];
    const TS* M = pinv + g.off;
    constexpr int R = kR;
    constexpr int P = kRowsPerWarp / R;
    using V = typename LdChunk<TS, kCB>::T;
    for (int grp = ga + warp; grp < gb; grp += nw) {
#pragma unroll
      for (int pass = 0; pass < P; ++pass) {
        const int row0 = grp * kRowsPerWarp + pass * R;
        V buf[R][kIter];
#pragma unroll
        for (int it = 0; it < kIter; ++it) {
          const int col = (it * 32 + lane) * W;
#pragma unroll
          for (int k = 0; k < R; ++k) {
            if (col < g.ld && row0 + k < g.nloc) buf[k][it] = load_tile<TS, kCB>(M + (long long)(row0 + k) * g.ld + col);
            else buf[k][it] = V{};
          }
        }
#pragma unroll
        for (int c = 0; c < kGroup; ++c) {
          if (!act[c]) continue;
          TC acc[R];
#pragma unroll
          for (int k = 0; k < R; ++k) acc[k] = (TC)0;
#pragma unroll
          for (int it = 0; it < kIter; ++it) {
            const int col = (it * 32 + lane) * W;
            if (col < g.ld) {
#pragma unroll
              for (int k = 0; k < R; ++k) acc[k] += dot_tile<TS, TC>(buf[k][it], &xs[c][col]);
            }
          }
#pragma unroll
          for (int k = 0; k < R; ++k) acc[k] = warp_sum(acc[k]);
          if (lane < R && row0 + lane < g.nloc) {
            TC v = acc[0];
#pragma unroll
            for (int k = 1; k < R; ++k)
              if (lane == k) v = acc[k];
            const int q = row0 + lane, a = q % g.nx, cc = q / g.nx;
            if constexpr (std::is_same<TS, __half>::value) v *= (TC)rscale[(long long)gofs[p] * kRowsPerWarp + q];
            atomicAdd(cs.zacc[c] + (long long)(g.y0 + 1 + cc) * n + (g.x0 + 1 + a), eta * v);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TMA variant of the smoother: the CTA's rows are streamed into a ring of
// shared-memory stages by 1-D bulk copies (cp.async.bulk, completion counted
// on one mbarrier per stage); a stage holds up to 8 consecutive rows of one
// patch (contiguous in memory) and each warp reduces one row of it.  Every
// wait on an mbarrier is bounded; on expiry the kernel raises kStTimeout,
// drains its own copies (bounded again) and returns.
__device__ int g_timeout_flag;   // raised by any expired bounded wait (read and cleared by the host)
constexpr int kStageRows = 8;
constexpr long long kWaitLimit = 1LL << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Failure-detection probe: one warp waits, bounded by 2^limit_log2 polls, on
// an mbarrier that it completes first (complete != 0) or that nothing ever
// completes; an expired wait raises g_timeout_flag exactly as the smoother's
// waits do.
__global__ void k_wait_probe(int complete, long long limit) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = smem_addr(&bar);
  if (threadIdx.x == 0) mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  if (threadIdx.x == 0 && complete)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
  __syncwarp();
  bool ok = false;
  for (long long i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(b, 0);
  if (!ok && threadIdx.x == 0) atomicOr(&g_timeout_flag, 1);
}

__device__ __forceinline__ void bulk_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <typename TS> struct Stages { static constexpr int N = 4; };
template <> struct Stages<double> { static constexpr int N = 3; };
template <> struct Stages<__nv_bfloat16> { static constexpr int N = 6; };

// stage k of the CTA's row list: patch, first row, row count
struct StageDesc {
  int patch, row0, rows;
};
__device__ __forceinline__ StageDesc stage_of(int k, int p0, int npatch, int g0, int g1,
                                              const int* __restrict__ gofs, const PatchGeo* __restrict__ geo) {
  for (int p = p0; p < npatch && gofs[p] < g1; ++p) {
    const int ra = kRowsPerGroup * (max(g0, gofs[p]) - gofs[p]);
    const int rb = min(geo[p].nloc, kRowsPerGroup * (min(g1, gofs[p + 1]) - gofs[p]));
    const int ns = (rb - ra + kStageRows - 1) / kStageRows;
    if (k < ns) return StageDesc{p, ra + k * kStageRows, min(kStageRows, rb - ra - k * kStageRows)};
    k -= ns;
  }
  return StageDesc{-1, 0, 0};
}

template <typename TC, typename TS, typename TR, bool kFused>
__global__ void __launch_bounds__(kThreads) k_smoother_tma(const PatchGeo* __restrict__ geo,
                                                           const int* __restrict__ gofs, int npatch,
                                                           const TS* __restrict__ pinv,
                                                           const TR* __restrict__ r,
                                                           TC* __restrict__ zacc, TC eta, int n,
                                                           PcgState* st, FuseArgs fa) {
  pdl_entry();
  if (st && st->done) return;
  constexpr int NS = Stages<TS>::N;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(16) TC xs[kPatchLd];
  __shared__ __align__(8) unsigned long long bars[NS];
  __shared__ double shr[32];
  __shared__ int s_nst, s_p0;
  TS* buf = reinterpret_cast<TS*>(dsm);
  const int stage_elems = kStageRows * kPatchLd;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double alpha = (kFused == 1) ? fa.st->alpha : 0.0;
  const int G = gofs[npatch];
  const long long per = ((long long)G + gridDim.x - 1) / gridDim.x;
  const int g0 = (int)min((long long)G, blockIdx.x * per), g1 = (int)min((long long)G, g0 + per);
  if (tid == 0) {
    int p = 0, hi = npatch - 1;  // last patch with gofs[p] <= g0
    while (p < hi) {
      const int mid = (p + hi + 1) >> 1;
      if (gofs[mid] <= g0) p = mid;
      else hi = mid - 1;
    }
    int cnt = 0;
    for (int q = p; g0 < g1 && q < npatch && gofs[q] < g1; ++q) {
      const int ra = kRowsPerGroup * (max(g0, gofs[q]) - gofs[q]);
      const int rb = min(geo[q].nloc, kRowsPerGroup * (min(g1, gofs[q + 1]) - gofs[q]));
      cnt += (rb - ra + kStageRows - 1) / kStageRows;
    }
    s_nst = cnt;
    s_p0 = p;
    for (int b = 0; b < NS; ++b) mbar_init(smem_addr(&bars[b]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nst = s_nst, p0 = s_p0;
  auto issue = [&](int k) {
    const StageDesc d = stage_of(k, p0, npatch, g0, g1, gofs, geo);
    const PatchGeo g = geo[d.patch];
    const unsigned bytes = (unsigned)(d.rows * g.ld * (int)sizeof(TS));
    const unsigned bar = smem_addr(&bars[k % NS]);
    mbar_expect_tx(bar, bytes);
    bulk_copy(smem_addr(buf + (size_t)(k % NS) * stage_elems), pinv + g.off + (long long)d.row0 * g.ld, bytes, bar);
  };
  if (tid == 0)
    for (int k = 0; k < NS && k < nst; ++k) issue(k);
  int cur = -1;
  PatchGeo g{};
  bool ok = true;
  int k = 0;
  for (; k < nst; ++k) {
    const StageDesc d = stage_of(k, p0, npatch, g0, g1, gofs, geo);
    if (d.patch != cur) {
      __syncthreads();
      cur = d.patch;
      g = geo[cur];
      for (int q = tid; q < g.ld; q += blockDim.x) {
        TC v = (TC)0;
        if (q < g.nloc) {
          const long long id = (long long)(g.y0 + 1 + q / g.nx) * n + (g.x0 + 1 + q % g.nx);
          if (kFused) v = (TC)(fa.r_old[id] - alpha * fa.q[id]);
          else v = (TC)r[id];
        }
        xs[q] = v;
      }
      __syncthreads();
    }
    // every thread observes the stage's completion; the CTA leaves together if
    // any thread's bounded wait expired
    const int mine = mbar_wait(smem_addr(&bars[k % NS]), (unsigned)((k / NS) & 1)) ? 1 : 0;
    if (!__syncthreads_and(mine)) {
      ok = false;
      break;
    }
    if (warp < d.rows) {
      const TS* row = buf + (size_t)(k % NS) * stage_elems + (size_t)warp * g.ld;
      constexpr int W = Vec<TS>::W;
      TC acc = (TC)0;
      for (int col = lane * W; col < g.ld; col += 32 * W) acc += dot_chunk_smem<TC>(row + col, xs + col);
      acc = warp_sum(acc);
      if (lane == 0) {
        const int q = d.row0 + warp;
        atomicAdd(zacc + (long long)(g.y0 + 1 + q / g.nx) * n + (g.x0 + 1 + q % g.nx), eta * acc);
      }
    }
    __syncthreads();   // stage buffer free again
    if (tid == 0 && k + NS < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(k + NS);
    }
  }
  if (!ok) {
    // raise the status, then drain this CTA's own copies (bounded) before leaving
    if (tid == 0) {
      atomicOr(&g_timeout_flag, 1);
      if (st) {
        atomicOr(&st->status, kStTimeout);
        st->done = 1;
      }
      for (int j = k; j < nst && j < k + NS; ++j) mbar_wait(smem_addr(&bars[j % NS]), (unsigned)((j / NS) & 1));
    }
    return;
  }
  if (kFused) {
    // block owners: r_new = r_old - alpha q and x += alpha p on their block's nodes
    for (int p = p0; g0 < g1 && p < npatch && gofs[p] < g1; ++p) {
      if (gofs[p] < g0) continue;
      const int I = p % fa.nc, J = p / fa.nc, b = fa.b;
      for (int t = tid; t < b * b; t += blockDim.x) {
        const long long id = (long long)(J * b + t / b) * n + I * b + t % b;
        const double rv = fa.r_old[id] - alpha * fa.q[id];
        fa.r_new[id] = rv;
        fa.x[id] += alpha * fa.p[id];
        if (fa.zclear) ((TC*)fa.zclear)[id] = (TC)0;
      }
    }
  }
}

// Inner residual r - K z on each block's owned nodes fused with the coarse
// restriction (partial inner products with the block's basis tiles).
template <typename TC, typename TS>
__global__ void __launch_bounds__(kThreads) k_resid_restrict(const int* __restrict__ slot_ptr,
                                                             const TS* __restrict__ owned,
                                                             const double* __restrict__ r,
                                                             const TC* __restrict__ z,
                                                             const TC* __restrict__ kinv,
                                                             double* __restrict__ part, int nc, int b,
                                                             int n, const PcgState* st) {
  pdl_entry();
  const int done = st ? st->done : 0;   // tested after the loads (see k_pcg_apply_p)
  __shared__ TC vals[kMaxB * kMaxB];
  const int blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const int bb = b * b, t = threadIdx.x;
  if (t < bb) {
    const int i = I * b + t % b, j = J * b + t / b;
    vals[t] = (i != 0 && j != 0) ? (TC)r[(long long)j * n + i] - stencil_apply<TC, TC, TC>(z, kinv, n, i, j)
                                 : (TC)0;
  }
  __syncthreads();
  if (done) return;
  // one warp per slot: no barrier per slot
  const int s0 = slot_ptr[blk], s1 = slot_ptr[blk + 1];
  const int warp = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
  for (int s = s0 + warp; s < s1; s += nw) {
    TC acc = (TC)0;
    for (int e = lane; e < bb; e += 32) acc += vals[e] * (TC)to_f(owned[(long long)s * bb + e]);
    acc = warp_sum(acc);
    if (lane == 0) part[s] = (double)acc;
  }
}

// ---------------------------------------------------------------------------
// Coarse restriction: per block, the partial inner products of the residual
// with each basis function restricted to the block's owned nodes.
template <typename TC, typename TS>
__global__ void __launch_bounds__(kThreads) k_restrict(const int* __restrict__ slot_ptr,
                                                       const TS* __restrict__ owned,
                                                       const TC* __restrict__ v,
                                                       double* __restrict__ part, int nc, int b,
                                                       int n, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  __shared__ TC vals[kMaxB * kMaxB];
  const int blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const int bb = b * b, t = threadIdx.x;
  if (t < bb) vals[t] = v[(long long)(J * b + t / b) * n + I * b + t % b];
  __syncthreads();
  // one warp per slot: no barrier per slot
  const int s0 = slot_ptr[blk], s1 = slot_ptr[blk + 1];
  const int warp = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
  for (int s = s0 + warp; s < s1; s += nw) {
    TC acc = (TC)0;
    for (int e = lane; e < bb; e += 32) acc += vals[e] * (TC)to_f(owned[(long long)s * bb + e]);
    acc = warp_sum(acc);
    if (lane == 0) part[s] = (double)acc;
  }
}

// Coarse solve d = K_H^{-1} c, c[u] = sum of the partials of u's slots.
__global__ void __launch_bounds__(kThreads) k_coarse_solve(const double* __restrict__ part,
                                                           const int* __restrict__ gather,
                                                           const double* __restrict__ Kinv,
                                                           double* __restrict__ d, int D,
                                                           const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  extern __shared__ double cvec[];
  for (int u = threadIdx.x; u < D; u += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gather[4 * u + k];
      if (g >= 0) s += part[g];
    }
    cvec[u] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < D; row += gridDim.x * nw) {
    const double* kr = Kinv + (long long)row * D;
    double acc = 0.0;
    for (int col = lane; col < D; col += 32) acc += kr[col] * cvec[col];
    acc = warp_sum(acc);
    if (lane == 0) d[row] = acc;
  }
}

// Large coarse systems: the right-hand side c[u] = sum of u's slot partials is
// formed once (k_coarse_rhs), then every CTA copies it into shared memory and
// streams its rows of K_H^{-1} with four independent accumulators per lane.
__global__ void k_coarse_rhs(const double* __restrict__ part, const int* __restrict__ gather,
                             double* __restrict__ c, int D, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < D; u += gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gather[4 * u + k];
      if (g >= 0) v += part[g];
    }
    c[u] = v;
  }
}

// Double-float GEMV (mixed-precision handles): d = Kinv c with Kinv and c
// as FP32 pairs (hi + lo), each product formed exactly by TwoProduct (the FMA
// residual of hi * hi) plus the two cross terms, and accumulated by
// compensated summation (Knuth's TwoSum), per lane and in the warp
// reduction; about 48 significant bits, on the FP32 pipe.  The FP64 GEMV
// reads the same 8 bytes per entry but is bound by this part's FP64 rate.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_fma(float& h, float& l, float2 k, float2 c) {
  const float p = k.x * c.x;
  float pe = fmaf(k.x, c.x, -p);   // the exact rounding error of k.x * c.x
  pe = fmaf(k.x, c.y, fmaf(k.y, c.x, pe));
  float sum, err;
  two_sum(h, p, sum, err);
  h = sum;
  l += err + pe;
}
__global__ void k_coarse_rhs_df(const double* __restrict__ part, const int* __restrict__ gather,
                                float2* __restrict__ c, int D, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < D; u += gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gather[4 * u + k];
      if (g >= 0) v += part[g];
    }
    const float hi = (float)v;
    c[u] = make_float2(hi, (float)(v - (double)hi));
  }
}
// kStage: the right-hand side staged in shared memory (D * 8 bytes, up to
// kCoarseStageMax); above that it is read from global memory (L1/L2)
constexpr int kCoarseStageMax = 24 * 1024;
template <bool kStage>
__global__ void __launch_bounds__(kThreads) k_coarse_gemv_df(const float2* __restrict__ c,
                                                             const float2* __restrict__ Kdf,
                                                             double* __restrict__ d, int D, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  extern __shared__ float2 cdf_sh[];
  const float2* cdf = c;
  if constexpr (kStage) {
    for (int u = threadIdx.x; u < D; u += blockDim.x) cdf_sh[u] = c[u];
    __syncthreads();
    cdf = cdf_sh;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < D; row += gridDim.x * nw) {
    const float2* kr = Kdf + (long long)row * D;
    // sixteen loads in flight per lane, four independent accumulator pairs
    float hh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ll[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int col = lane;
    for (; col + 480 < D; col += 512) {
      float2 kk[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) kk[u] = __ldg(kr + col + 32 * u);
#pragma unroll
      for (int u = 0; u < 16; ++u) df_fma(hh[u & 3], ll[u & 3], kk[u], cdf[col + 32 * u]);
    }
    for (; col < D; col += 32) df_fma(hh[0], ll[0], __ldg(kr + col), cdf[col]);
    float h, l, e, h2, e2;
    two_sum(hh[0], hh[1], h, e);
    two_sum(hh[2], hh[3], h2, e2);
    l = (ll[0] + ll[1]) + (ll[2] + ll[3]) + e + e2;
    two_sum(h, h2, h, e);
    l += e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
      two_sum(h, oh, h, e);
      l += ol + e;
    }
    if (lane == 0) d[row] = (double)h + (double)l;
  }
}
__global__ void k_split_df(const double* __restrict__ a, float2* __restrict__ b, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const double x = a[i];
    const float hi = (float)x;
    b[i] = make_float2(hi, (float)(x - (double)hi));
  }
}
template <bool kStage>
__global__ void __launch_bounds__(kThreads) k_coarse_gemv(const double* __restrict__ c,
                                                          const double* __restrict__ Kinv,
                                                          double* __restrict__ d, int D, const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  extern __shared__ double cvec_sh[];
  const double* cvec = c;
  if constexpr (kStage) {
    for (int u = threadIdx.x; u < D; u += blockDim.x) cvec_sh[u] = c[u];
    __syncthreads();
    cvec = cvec_sh;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < D; row += gridDim.x * nw) {
    const double* kr = Kinv + (long long)row * D;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int col = lane;
    for (; col + 96 < D; col += 128) {
      a0 += __ldg(kr + col) * cvec[col];
      a1 += __ldg(kr + col + 32) * cvec[col + 32];
      a2 += __ldg(kr + col + 64) * cvec[col + 64];
      a3 += __ldg(kr + col + 96) * cvec[col + 96];
    }
    for (; col < D; col += 32) a0 += __ldg(kr + col) * cvec[col];
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) d[row] = acc;
  }
}

// Coarse prolongation: v += sum_s d[coef(s)] * tile_s on each block's owned nodes.
template <typename TC, typename TS>
__global__ void __launch_bounds__(kThreads) k_prolong(const int* __restrict__ slot_ptr,
                                                      const Slot* __restrict__ slots,
                                                      const TS* __restrict__ owned,
                                                      const double* __restrict__ d,
                                                      TC* __restrict__ v, int nc, int b, int n,
                                                      const PcgState* st) {
  pdl_entry();
  if (st && st->done) return;
  const int blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const int bb = b * b, t = threadIdx.x;
  if (t >= bb) return;
  TC acc = (TC)0;
  const int s0 = slot_ptr[blk], s1 = slot_ptr[blk + 1];
  for (int s = s0; s < s1; ++s) acc += (TC)d[slots[s].coef] * (TC)to_f(owned[(long long)s * bb + t]);
  v[(long long)(J * b + t / b) * n + I * b + t % b] += acc;
}

// Small coarse systems (D <= kCoarseSplit, at most kFuseSlots slots per block):
// the coarse solve and the prolongation in one kernel.  Each CTA (one block)
// forms the whole right-hand side c, computes d_u = (K_H^{-1} c)_u only for
// the unknowns of its own slots (warp per row, the lane order of
// k_coarse_solve, so d is bit-identical), then adds sum_s d * tile_s on its
// owned nodes exactly as k_prolong does.
constexpr int kFuseSlots = 64;
template <typename TC, typename TS>
__global__ void __launch_bounds__(kThreads) k_coarse_prolong(const double* __restrict__ part,
                                                             const int* __restrict__ gather,
                                                             const double* __restrict__ Kinv, int D,
                                                             const int* __restrict__ slot_ptr,
                                                             const Slot* __restrict__ slots,
                                                             const TS* __restrict__ owned, TC* __restrict__ v,
                                                             int nc, int b, int n, const PcgState* st) {
  pdl_entry();
  const int done = st ? st->done : 0;   // tested after the loads (see k_pcg_apply_p)
  __shared__ double cvec[kCoarseSplit];
  __shared__ double dloc[kFuseSlots];
  for (int u = threadIdx.x; u < D; u += blockDim.x) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int g = gather[4 * u + k];
      if (g >= 0) sum += part[g];
    }
    cvec[u] = sum;
  }
  __syncthreads();
  if (done) return;
  const int blk = blockIdx.x, I = blk % nc, J = blk / nc;
  const int s0 = slot_ptr[blk], m = slot_ptr[blk + 1] - s0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < m; j += nw) {
    const double* kr = Kinv + (long long)slots[s0 + j].coef * D;
    double acc = 0.0;
    for (int col = lane; col < D; col += 32) acc += kr[col] * cvec[col];
    acc = warp_sum(acc);
    if (lane == 0) dloc[j] = acc;
  }
  __syncthreads();
  const int bb = b * b, t = threadIdx.x;
  if (t >= bb) return;
  TC acc = (TC)0;
  for (int j = 0; j < m; ++j) acc += (TC)dloc[j] * (TC)to_f(owned[(long long)(s0 + j) * bb + t]);
  v[(long long)(J * b + t / b) * n + I * b + t % b] += acc;
}

// node coefficients of K (FP64): c0, cE, cN, cNE, cNW, cells outside the domain as 0
__global__ void k_stencil_coefs(const double* __restrict__ kinv, double* __restrict__ kcoef, int n) {
  pdl_entry();
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    auto cell = [&](int ci, int cj) { return (ci >= 0 && cj >= 0 && ci < n && cj < n) ? kinv[(long long)cj * n + ci] : 0.0; };
    const double k00 = cell(i - 1, j - 1), k10 = cell(i, j - 1), k01 = cell(i - 1, j), k11 = cell(i, j);
    kcoef[t] = (2.0 / 3.0) * (k00 + k10 + k01 + k11);
    kcoef[nn + t] = -(1.0 / 6.0) * (k10 + k11);
    kcoef[2 * nn + t] = -(1.0 / 6.0) * (k01 + k11);
    kcoef[3 * nn + t] = -(1.0 / 3.0) * k11;
    kcoef[4 * nn + t] = -(1.0 / 3.0) * k01;
  }
}

template <typename TA, typename TB>
__global__ void k_convert(const TA* __restrict__ a, TB* __restrict__ b, long long m) {
  pdl_entry();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x)
    b[t] = (TB)a[t];
}

inline int grid_for(long long m) {
  long long g = (m + kThreads - 1) / kThreads;
  if (g > kRedGrid) g = kRedGrid;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// ---- launchers ---------------------------------------------------------------
void launch_apply_operator(const double* psi, const double* kinv, double* out, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_apply_operator, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, psi, kinv, out, n);
}
void launch_apply_operator_f32(const double* psi, const float* kinv, double* out, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_apply_operator_f32, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, psi, kinv, out, n);
}

template <typename TC>
void launch_residual(const double* r, const TC* z, const TC* kinv, TC* out, int n, const PcgState* st,
                     cudaStream_t s) {
  TG_COUNT(1);
  launch(k_residual<TC>, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, r, z, kinv, out, n, st);
}
template void launch_residual<double>(const double*, const double*, const double*, double*, int,
                                      const PcgState*, cudaStream_t);
template void launch_residual<float>(const double*, const float*, const float*, float*, int,
                                     const PcgState*, cudaStream_t);

int sm_count();
template <typename TC>
void launch_pcg_dots(const double* r, const TC* z, const double* q, double* part, PcgState* st, int n,
                     cudaStream_t s) {
  TG_COUNT(1);
  // FP64-pipe bound at large n: two CTAs per SM, so fewer per-CTA FP64 tree
  // sums; at small n at least four elements per thread (one pass of loads),
  // so fewer CTAs arrive at the reduction
  const long long nn = (long long)n * n;
  const long long g4 = std::max<long long>(1, (nn + 4LL * kThreads - 1) / (4LL * kThreads));
  launch(k_pcg_dots<TC>, dim3((unsigned)std::min<long long>(g4, 2LL * sm_count())), dim3(kThreads), 0, s, r, z, q,
         part, st, n);
}
void launch_pcg_init(double* x, const double* r, double* part, PcgState* st, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_pcg_init, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, x, r, part, st, n);
}
template <typename TC>
void launch_pcg_init_rz(const double* r, const TC* z, double* p, double* part, PcgState* st, int n,
                        cudaStream_t s) {
  TG_COUNT(1);
  launch(k_pcg_init_rz<TC>, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, r, z, p, part, st, n);
}
#define TG_INST_TC(TC)                                                                              \
  template void launch_pcg_dots<TC>(const double*, const TC*, const double*, double*, PcgState*,   \
                                    int, cudaStream_t);                                             \
  template void launch_pcg_init_rz<TC>(const double*, const TC*, double*, double*, PcgState*, int, \
                                       cudaStream_t);
TG_INST_TC(double)
TG_INST_TC(float)

int sm_count() {
  static int cnt = 0;
  if (!cnt) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev);
    if (cnt <= 0) cnt = 1;
  }
  return cnt;
}

// resident CTAs per SM of a smoother instantiation (queried once, at setup)
template <typename TC, typename TS, typename TR, int kFused, int kCB, int kR, bool kPipe>
int smoother_per_sm() {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smoother<TC, TS, TR, kFused, kCB, kR, kPipe>, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  return per_sm;
}

// one wave of CTAs, but at least 8 row groups per CTA (every warp busy)
inline int wave_grid(int per_sm, int ngroups) {
  int grid = per_sm * sm_count();
  const int min_groups_per_cta = 8;
  if (grid * min_groups_per_cta > ngroups) grid = (ngroups + min_groups_per_cta - 1) / min_groups_per_cta;
  return grid < 1 ? 1 : grid;
}

// TMA smoother: dynamic shared memory of the stage ring, resident CTAs per SM
template <typename TS>
size_t tma_smem() { return (size_t)Stages<TS>::N * kStageRows * kPatchLd * sizeof(TS); }

template <typename TC, typename TS, typename TR, bool kFused>
int tma_per_sm() {
  static int per_sm = 0;
  if (!per_sm) {
    const size_t shm = tma_smem<TS>();
    cudaFuncSetAttribute(k_smoother_tma<TC, TS, TR, kFused>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smoother_tma<TC, TS, TR, kFused>, kThreads, shm);
    if (per_sm <= 0) per_sm = 1;
  }
  return per_sm;
}

// Smoother tile shapes: 0 = 16-byte loads, default rows per pass (4; 2 for
// FP64); 1 = 16-byte loads, 2 rows; 2 = 8-byte loads, 4 rows; 3 = 8-byte
// loads, 2 rows; 4 = TMA bulk copies into a shared-memory ring; 5 and 6 =
// shapes 3 and 1 software-pipelined (the next pass's rows in flight while the
// current pass is reduced).  FP64 storage has shapes 0 and 4 only (others map
// to 0).
template <typename TC, typename TS, typename TR, int kFused, int kCB, int kR, bool kPipe = false>
void smoother_go(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv, const TR* r,
                 TC* zacc, double eta, int n, const PcgState* st, const FuseArgs& fa, const float* rscale,
                 cudaStream_t s) {
  const int grid = wave_grid(smoother_per_sm<TC, TS, TR, kFused, kCB, kR, kPipe>(), ngroups);
  launch(k_smoother<TC, TS, TR, kFused, kCB, kR, kPipe>, dim3(grid), dim3(kThreads), 0, s, geo, gofs, npatch, pinv, r, zacc, (TC)eta, n, st, fa, rscale);
}

template <typename TC, typename TS, typename TR, int kFused>
int smoother_mma_per_sm() {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smoother_mma<TC, TS, TR, kFused>, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  return per_sm;
}

// tensor-core sweep: one wave of CTAs, at least one 16-row tile per warp
template <typename TC, typename TS, typename TR, int kFused>
void smoother_mma_go(const PatchGeo* geo, const int* gofs, int npatch, const TR* r, TC* zacc, double eta, int n,
                     const PcgState* st, const FuseArgs& fa, const float* rscale, const BandRef& band,
                     cudaStream_t s) {
  int grid = smoother_mma_per_sm<TC, TS, TR, kFused>() * sm_count();
  const int min_tiles_per_cta = kThreads / 32;
  if (grid * min_tiles_per_cta > band.ntiles) grid = (band.ntiles + min_tiles_per_cta - 1) / min_tiles_per_cta;
  if (grid >= npatch) grid = grid / npatch * npatch;
  if (grid < 1) grid = 1;
  launch(k_smoother_mma<TC, TS, TR, kFused>, dim3(grid), dim3(kThreads), 0, s, geo, band.tofs, gofs, npatch,
         (const TS*)band.tp, r, zacc, (TC)eta, n, st, fa, rscale);
}

template <typename TC, typename TS, typename TR, int kFused>
void smoother_shape(int shape, const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                    const TR* r, TC* zacc, double eta, int n, const PcgState* st, const FuseArgs& fa,
                    const float* rscale, cudaStream_t s, BandRef band = {}) {
  TG_COUNT(1);
  if (is_band_shape(shape) && band.p) {
    if constexpr (std::is_same<TC, float>::value) {
      if (shape == kShapeBand) {
        launch(k_smoother_band<TC, TR, kFused>, dim3((npatch + kBandWarps - 1) / kBandWarps),
               dim3(32 * kBandWarps), 0, s, geo, npatch, (const TC*)band.p, band.ldb, band.stride, r, zacc, (TC)eta,
               n, st, fa);
        return;
      }
      launch(k_smoother_band_ring<TR, kFused>, dim3((npatch + kBandWarps - 1) / kBandWarps), dim3(32 * kBandWarps),
             0, s, geo, npatch, (const float*)band.p, band.ldb, band.stride, r, zacc, (float)eta, n, st, fa);
    } else {
      launch(k_smoother_band<TC, TR, kFused>, dim3((npatch + kBandWarps - 1) / kBandWarps), dim3(32 * kBandWarps), 0,
             s, geo, npatch, (const TC*)band.p, band.ldb, band.stride, r, zacc, (TC)eta, n, st, fa);
    }
    return;
  }
  if (is_band_shape(shape)) shape = 0;
  if (shape == kShapeTensor) {
    if constexpr (sizeof(TS) == 2) {
      if (band.tp) {
        smoother_mma_go<TC, TS, TR, kFused>(geo, gofs, npatch, r, zacc, eta, n, st, fa, rscale, band, s);
        return;
      }
    }
    shape = 0;
  }
  constexpr bool kHalf = std::is_same<TS, __half>::value;
  // the TMA ring has no row scaling and no residual-fused mode
  if ((kHalf || kFused == 2) && shape == 4) shape = 0;
  if (shape == 4) {
    if constexpr (!kHalf && kFused != 2) {
      int grid = tma_per_sm<TC, TS, TR, kFused == 1>() * sm_count();
      if (grid * 2 > ngroups) grid = (ngroups + 1) / 2;
      launch(k_smoother_tma<TC, TS, TR, kFused == 1>, dim3(grid < 1 ? 1 : grid), dim3(kThreads), tma_smem<TS>(), s,
             geo, gofs, npatch, pinv, r, zacc, (TC)eta, n, const_cast<PcgState*>(st), fa);
    }
    return;
  }
  if constexpr (std::is_same<TS, double>::value) {
    smoother_go<TC, TS, TR, kFused, 16, 2>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s);
  } else {
    switch (shape) {
      case 1: smoother_go<TC, TS, TR, kFused, 16, 2>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
      case 2: smoother_go<TC, TS, TR, kFused, 8, 4>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
      case 3: smoother_go<TC, TS, TR, kFused, 8, 2>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
      case 5: smoother_go<TC, TS, TR, kFused, 8, 2, true>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
      case 6: smoother_go<TC, TS, TR, kFused, 16, 2, true>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
      default: smoother_go<TC, TS, TR, kFused, 16, 4>(geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, fa, rscale, s); break;
    }
  }
}

// occupancy queries of every shape of one instantiation (outside any capture)
template <typename TC, typename TS, typename TR, int kFused>
void smoother_prepare() {
  if constexpr (!std::is_same<TS, __half>::value && kFused != 2) tma_per_sm<TC, TS, TR, kFused == 1>();
  if constexpr (std::is_same<TS, double>::value) {
    smoother_per_sm<TC, TS, TR, kFused, 16, 2, false>();
  } else {
    smoother_per_sm<TC, TS, TR, kFused, 16, 4, false>();
    smoother_per_sm<TC, TS, TR, kFused, 16, 2, false>();
    smoother_per_sm<TC, TS, TR, kFused, 8, 4, false>();
    smoother_per_sm<TC, TS, TR, kFused, 8, 2, false>();
    smoother_per_sm<TC, TS, TR, kFused, 8, 2, true>();
    smoother_per_sm<TC, TS, TR, kFused, 16, 2, true>();
  }
  if constexpr (sizeof(TS) == 2) smoother_mma_per_sm<TC, TS, TR, kFused>();
}

template <typename TC, typename TS, typename TR>
void launch_smoother(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv, const TR* r,
                     TC* zacc, double eta, int n, const PcgState* st, cudaStream_t s, int shape,
                     const float* rscale, BandRef band) {
  smoother_shape<TC, TS, TR, false>(shape, geo, gofs, npatch, ngroups, pinv, r, zacc, eta, n, st, FuseArgs{},
                                    rscale, s, band);
}

template <typename TC, typename TS>
void launch_smoother_update(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                            const double* r_old, double* r_new, const double* q, double* x, const double* p,
                            TC* zacc, double eta, int n, int nc, int b, double* part, PcgState* st,
                            cudaStream_t s, int shape, const float* rscale, TC* zclear, BandRef band) {
  FuseArgs fa{r_old, r_new, q, x, p, part, st, nc, b, zclear, nullptr, nullptr};
  smoother_shape<TC, TS, double, 1>(shape, geo, gofs, npatch, ngroups, pinv, r_old, zacc, eta, n, st, fa,
                                    rscale, s, band);
}

template <typename TC, typename TS>
void launch_smoother_resid(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                           const double* r, const TC* zin, const TC* kin, TC* zout, double eta, int n, int nc, int b,
                           const PcgState* st, cudaStream_t s, int shape, const float* rscale, BandRef band) {
  FuseArgs fa{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nc, b, nullptr, zin, kin};
  smoother_shape<TC, TS, double, 2>(shape, geo, gofs, npatch, ngroups, pinv, r, zout, eta, n, st, fa, rscale, s,
                                    band);
}
template <typename TC, typename TS, int kFused, int kCB, int kR>
int smoother_multi_per_sm() {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smoother_multi<TC, TS, kFused, kCB, kR>, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  return per_sm;
}

template <typename TC, typename TS, int kFused, int kCB, int kR>
void smoother_multi_go(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv, double eta,
                       int n, const ChainSet<TC>& cs, const float* rscale, cudaStream_t s) {
  const int grid = wave_grid(smoother_multi_per_sm<TC, TS, kFused, kCB, kR>(), ngroups);
  launch(k_smoother_multi<TC, TS, kFused, kCB, kR>, dim3(grid), dim3(kThreads), 0, s, geo, gofs, npatch, pinv,
         (TC)eta, n, cs, rscale);
}

// tile shapes of the lock-step sweep: the non-pipelined register shapes
// (TMA and pipelined shapes map to 0, 3 and 1 as in the single-chain sweep's
// families; FP64 storage uses 16-byte loads, 2 rows)
template <typename TC, typename TS, int kFused>
void smoother_multi_shape(int shape, const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                          double eta, int n, const ChainSet<TC>& cs, const float* rscale, cudaStream_t s) {
  TG_COUNT(1);
  if constexpr (std::is_same<TS, double>::value) {
    smoother_multi_go<TC, TS, kFused, 16, 2>(geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s);
  } else {
    switch (shape) {
      case 1: case 6: smoother_multi_go<TC, TS, kFused, 16, 2>(geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s); break;
      case 2: smoother_multi_go<TC, TS, kFused, 8, 4>(geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s); break;
      case 3: case 5: smoother_multi_go<TC, TS, kFused, 8, 2>(geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s); break;
      default: smoother_multi_go<TC, TS, kFused, 16, 4>(geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s); break;
    }
  }
}

template <typename TC, typename TS, int kFused>
void smoother_mma_multi_go(const PatchGeo* geo, const int* gofs, int npatch, double eta, int n,
                           const ChainSet<TC>& cs, const float* rscale, const BandRef& t, cudaStream_t s) {
  static int per_sm = 0;
  if (!per_sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smoother_mma_multi<TC, TS, kFused>, kThreads, 0);
    if (per_sm <= 0) per_sm = 1;
  }
  int grid = per_sm * sm_count();
  const int min_tiles_per_cta = kThreads / 32;
  if (grid * min_tiles_per_cta > t.ntiles) grid = (t.ntiles + min_tiles_per_cta - 1) / min_tiles_per_cta;
  if (grid >= npatch) grid = grid / npatch * npatch;
  if (grid < 1) grid = 1;
  TG_COUNT(1);
  launch(k_smoother_mma_multi<TC, TS, kFused>, dim3(grid), dim3(kThreads), 0, s, geo, t.tofs, gofs, npatch,
         (const TS*)t.tp, (TC)eta, n, cs, rscale);
}

template <typename TC, typename TS>
void launch_smoother_multi(int mode, const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                           const ChainPtrs* chains, int k, double eta, int n, int nc, int b, cudaStream_t s, int shape,
                           const float* rscale, const BandRef* tiles) {
  ChainSet<TC> cs{};
  cs.k = k;
  for (int c = 0; c < kGroup; ++c) {
    const ChainPtrs& q = chains[c < k ? c : 0];   // absent slots repeat chain 0's pointers (never used)
    cs.r[c] = q.r;
    cs.zacc[c] = (TC*)q.zacc;
    cs.st[c] = q.st;
    cs.fa[c] = FuseArgs{q.r_old, q.r_new, q.q, q.x, q.p, q.part, q.st, nc, b, q.zclear, q.zin, q.kin};
  }
  if constexpr (sizeof(TS) == 2) {
    if (shape == kShapeTensor && tiles && tiles->tp) {   // the tensor-core tiles, one A load for every chain
      if (mode == 1) smoother_mma_multi_go<TC, TS, 1>(geo, gofs, npatch, eta, n, cs, rscale, *tiles, s);
      else smoother_mma_multi_go<TC, TS, 2>(geo, gofs, npatch, eta, n, cs, rscale, *tiles, s);
      return;
    }
  }
  if (mode == 1)
    smoother_multi_shape<TC, TS, 1>(shape, geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s);
  else
    smoother_multi_shape<TC, TS, 2>(shape, geo, gofs, npatch, ngroups, pinv, eta, n, cs, rscale, s);
}
template void launch_smoother_multi<double, double>(int, const PatchGeo*, const int*, int, int, const double*,
                                                    const ChainPtrs*, int, double, int, int, int, cudaStream_t, int,
                                                    const float*, const BandRef*);
template void launch_smoother_multi<float, float>(int, const PatchGeo*, const int*, int, int, const float*,
                                                  const ChainPtrs*, int, double, int, int, int, cudaStream_t, int,
                                                  const float*, const BandRef*);
template void launch_smoother_multi<float, __nv_bfloat16>(int, const PatchGeo*, const int*, int, int,
                                                          const __nv_bfloat16*, const ChainPtrs*, int, double, int,
                                                          int, int, cudaStream_t, int, const float*, const BandRef*);
template void launch_smoother_multi<float, __half>(int, const PatchGeo*, const int*, int, int, const __half*,
                                                   const ChainPtrs*, int, double, int, int, int, cudaStream_t, int,
                                                   const float*, const BandRef*);

// set the graph's loop condition: continue while any chain of a group runs
__global__ void k_set_condition_any(cudaGraphConditionalHandle cond, StateSet ss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned go = 0u;
    for (int c = 0; c < ss.k; ++c) go |= ss.st[c]->done ? 0u : 1u;
    cudaGraphSetConditional(cond, go);
  }
}
void launch_set_condition_any(cudaGraphConditionalHandle cond, const PcgState* const* st, int k, cudaStream_t s) {
  StateSet ss{};
  ss.k = k;
  for (int c = 0; c < k && c < kGroup; ++c) ss.st[c] = st[c];
  TG_COUNT(1);
  launch(k_set_condition_any, dim3(1), dim3(32), 0, s, cond, ss);
}

template void launch_smoother_resid<double, double>(const PatchGeo*, const int*, int, int, const double*,
                                                    const double*, const double*, const double*, double*, double,
                                                    int, int, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother_resid<float, float>(const PatchGeo*, const int*, int, int, const float*, const double*,
                                                  const float*, const float*, float*, double, int, int, int,
                                                  const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother_resid<float, __nv_bfloat16>(const PatchGeo*, const int*, int, int,
                                                          const __nv_bfloat16*, const double*, const float*,
                                                          const float*, float*, double, int, int, int,
                                                          const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother_resid<float, __half>(const PatchGeo*, const int*, int, int, const __half*,
                                                   const double*, const float*, const float*, float*, double, int,
                                                   int, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother_update<double, double>(const PatchGeo*, const int*, int, int, const double*,
                                                     const double*, double*, const double*, double*,
                                                     const double*, double*, double, int, int, int, double*,
                                                     PcgState*, cudaStream_t, int, const float*, double*, BandRef);
template void launch_smoother_update<float, float>(const PatchGeo*, const int*, int, int, const float*,
                                                   const double*, double*, const double*, double*,
                                                   const double*, float*, double, int, int, int, double*,
                                                   PcgState*, cudaStream_t, int, const float*, float*, BandRef);
template void launch_smoother_update<float, __nv_bfloat16>(const PatchGeo*, const int*, int, int,
                                                           const __nv_bfloat16*, const double*, double*,
                                                           const double*, double*, const double*, float*, double,
                                                           int, int, int, double*, PcgState*, cudaStream_t, int,
                                                           const float*, float*, BandRef);
template void launch_smoother_update<float, __half>(const PatchGeo*, const int*, int, int, const __half*,
                                                    const double*, double*, const double*, double*, const double*,
                                                    float*, double, int, int, int, double*, PcgState*, cudaStream_t,
                                                    int, const float*, float*, BandRef);

template <typename TC>
void launch_pcg_apply_p(const TC* zprev, const double* pold, double* pnew, double* q, TC* znext,
                        const double* kcoef, double* part, PcgState* st, int n, cudaStream_t s) {
  TG_COUNT(1);
  // rows per thread: the most that still leaves at least two CTAs per SM
  const int gx = (n + kTx - 1) / kTx;
  auto ctas = [&](int r) { return (long long)gx * ((n + kTy * r - 1) / (kTy * r)); };
  const int sms = sm_count();
  if (ctas(4) >= 2LL * sms) {
    launch(k_pcg_apply_p<TC, 4>, dim3(gx, (n + 4 * kTy - 1) / (4 * kTy)), dim3(kThreads), 0, s, zprev, pold, pnew, q,
           znext, kcoef, part, st, n);
  } else if (ctas(2) >= 2LL * sms) {
    launch(k_pcg_apply_p<TC, 2>, dim3(gx, (n + 2 * kTy - 1) / (2 * kTy)), dim3(kThreads), 0, s, zprev, pold, pnew, q,
           znext, kcoef, part, st, n);
  } else {
    launch(k_pcg_apply_p<TC, 1>, dim3(gx, (n + kTy - 1) / kTy), dim3(kThreads), 0, s, zprev, pold, pnew, q, znext,
           kcoef, part, st, n);
  }
}
template void launch_pcg_apply_p<double>(const double*, const double*, double*, double*, double*, const double*,
                                         double*, PcgState*, int, cudaStream_t);
template void launch_pcg_apply_p<float>(const float*, const double*, double*, double*, float*, const double*,
                                        double*, PcgState*, int, cudaStream_t);

template void launch_smoother<double, double, double>(const PatchGeo*, const int*, int, int, const double*, const double*, double*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, float, double>(const PatchGeo*, const int*, int, int, const float*, const double*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, float, float>(const PatchGeo*, const int*, int, int, const float*, const float*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, __nv_bfloat16, double>(const PatchGeo*, const int*, int, int, const __nv_bfloat16*, const double*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, __nv_bfloat16, float>(const PatchGeo*, const int*, int, int, const __nv_bfloat16*, const float*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, __half, double>(const PatchGeo*, const int*, int, int, const __half*, const double*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);
template void launch_smoother<float, __half, float>(const PatchGeo*, const int*, int, int, const __half*, const float*, float*,
                                      double, int, const PcgState*, cudaStream_t, int, const float*, BandRef);

template <typename TC, typename TS>
void launch_resid_restrict(const CoarseSpace& cs, double* part, int nblocks, int nc, int b, int n, const double* r,
                           const TC* z, const TC* kinv, const PcgState* st, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_resid_restrict<TC, TS>, dim3(nblocks), dim3(kThreads), 0, s, cs.slot_ptr, (const TS*)cs.owned, r, z, kinv, part, nc, b, n, st);
}
template void launch_resid_restrict<double, double>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                                    const double*, const double*, const PcgState*, cudaStream_t);
template void launch_resid_restrict<float, float>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                                  const float*, const float*, const PcgState*, cudaStream_t);
template void launch_resid_restrict<float, __nv_bfloat16>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                                          const float*, const float*, const PcgState*, cudaStream_t);

template <typename TC, typename TS>
void launch_restrict(const CoarseSpace& cs, double* part, int nblocks, int nc, int b, int n, const TC* v,
                     const PcgState* st, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_restrict<TC, TS>, dim3(nblocks), dim3(kThreads), 0, s, cs.slot_ptr, (const TS*)cs.owned, v, part, nc, b, n, st);
}
int sm_count();
template <typename TC, typename TS, typename TR, int kFused> void smoother_prepare();
void launch_wait_probe(int complete, int limit_log2, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(complete, 1LL << limit_log2);
}

int read_and_clear_timeout() {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_timeout_flag, sizeof(int));
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_timeout_flag, &zero, sizeof(int));
  }
  return v;
}

void configure_kernels(int max_coarse_dim) {
  sm_count();
  smoother_prepare<double, double, double, false>();
  smoother_prepare<float, float, double, false>();
  smoother_prepare<float, float, float, false>();
  smoother_prepare<float, __nv_bfloat16, double, false>();
  smoother_prepare<float, __nv_bfloat16, float, false>();
  smoother_prepare<double, double, double, true>();
  smoother_prepare<float, float, double, true>();
  smoother_prepare<float, __nv_bfloat16, double, true>();
  smoother_prepare<float, __half, double, false>();
  smoother_prepare<float, __half, float, false>();
  smoother_prepare<float, __half, double, true>();
  smoother_prepare<double, double, double, 2>();
  smoother_prepare<float, float, double, 2>();
  smoother_prepare<float, __nv_bfloat16, double, 2>();
  smoother_prepare<float, __half, double, 2>();
  const size_t shm = sizeof(double) * (size_t)(max_coarse_dim > 0 ? max_coarse_dim : 1);
  if (shm > 48 * 1024) {
    const int stage = (int)std::min(shm, sizeof(double) * (size_t)kCoarseStageMax);
    cudaFuncSetAttribute(k_coarse_gemv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage);
    cudaFuncSetAttribute(k_coarse_gemv_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage);   // float2: 8 B
  }
}
void launch_pcg_init_warm(const double* x, const double* rho, const double* kinv, double* r, double* part,
                          PcgState* st, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_pcg_init_warm, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, x, rho, kinv, r, part, st, n);
}
void launch_pcg_reset(PcgState* st, const double* rtol, int maxit, int flexible, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_pcg_reset, dim3(1), dim3(32), 0, s, st, rtol, maxit, flexible);
}
void launch_set_condition(cudaGraphConditionalHandle cond, const PcgState* st, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_set_condition, dim3(1), dim3(32), 0, s, cond, st);
}
void launch_coarse_solve(const CoarseSpace& cs, const double* part, double* coefs, const PcgState* st,
                         cudaStream_t s) {
  if (cs.solver == 2) {   // nested-dissection factor (coarse_nd.cu)
    launch_nd_solve(cs.nd, part, coefs, st, s);
    return;
  }
  const size_t shm = sizeof(double) * (size_t)cs.D;
  if (cs.D > kCoarseSplit) {
    double* rhs = coefs + cs.D;
    TG_COUNT(2);
    int grid = (cs.D + 7) / 8;
    if (grid > 2 * sm_count()) grid = 2 * sm_count();
    const bool stage = cs.D <= kCoarseStageMax;
    if (cs.Kdf) {   // double-float copy (mixed precision): rhs as FP32 pairs in the same space
      float2* rdf = reinterpret_cast<float2*>(rhs);
      grid = std::min((cs.D + 7) / 8, 4 * sm_count());
      launch(k_coarse_rhs_df, dim3((cs.D + kThreads - 1) / kThreads), dim3(kThreads), 0, s, part, cs.gather, rdf,
             cs.D, st);
      if (stage)
        launch(k_coarse_gemv_df<true>, dim3(grid), dim3(kThreads), sizeof(float2) * (size_t)cs.D, s,
               (const float2*)rdf, (const float2*)cs.Kdf, coefs, cs.D, st);
      else
        launch(k_coarse_gemv_df<false>, dim3(grid), dim3(kThreads), 0, s, (const float2*)rdf, (const float2*)cs.Kdf,
               coefs, cs.D, st);
      return;
    }
    launch(k_coarse_rhs, dim3((cs.D + kThreads - 1) / kThreads), dim3(kThreads), 0, s, part, cs.gather, rhs, cs.D, st);
    if (stage) launch(k_coarse_gemv<true>, dim3(grid), dim3(kThreads), shm, s, rhs, cs.Kinv, coefs, cs.D, st);
    else launch(k_coarse_gemv<false>, dim3(grid), dim3(kThreads), 0, s, rhs, cs.Kinv, coefs, cs.D, st);
    return;
  }
  int grid = (cs.D + 7) / 8;
  if (grid > 2 * 152) grid = 2 * 152;
  if (grid < 1) grid = 1;
  TG_COUNT(1);
  launch(k_coarse_solve, dim3(grid), dim3(kThreads), shm, s, part, cs.gather, cs.Kinv, coefs, cs.D, st);
}
template <typename TC, typename TS>
void launch_prolong(const CoarseSpace& cs, const double* coefs, int nblocks, int nc, int b, int n, TC* v,
                    const PcgState* st, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_prolong<TC, TS>, dim3(nblocks), dim3(kThreads), 0, s, cs.slot_ptr, cs.slots, (const TS*)cs.owned, coefs, v, nc, b, n, st);
}
template <typename TC, typename TS>
void launch_coarse_correct(const CoarseSpace& cs, const double* part, double* coefs, int nblocks, int nc, int b, int n,
                           TC* v, const PcgState* st, cudaStream_t s) {
  if (cs.solver == 1 && cs.D <= kCoarseSplit && cs.max_slots_per_block <= kFuseSlots && b * b <= kThreads) {
    TG_COUNT(1);
    launch(k_coarse_prolong<TC, TS>, dim3(nblocks), dim3(kThreads), 0, s, part, cs.gather, cs.Kinv, cs.D, cs.slot_ptr,
           cs.slots, (const TS*)cs.owned, v, nc, b, n, st);
    return;
  }
  launch_coarse_solve(cs, part, coefs, st, s);
  launch_prolong<TC, TS>(cs, coefs, nblocks, nc, b, n, v, st, s);
}
template void launch_coarse_correct<double, double>(const CoarseSpace&, const double*, double*, int, int, int, int,
                                                    double*, const PcgState*, cudaStream_t);
template void launch_coarse_correct<float, float>(const CoarseSpace&, const double*, double*, int, int, int, int,
                                                  float*, const PcgState*, cudaStream_t);
template void launch_coarse_correct<float, __nv_bfloat16>(const CoarseSpace&, const double*, double*, int, int, int,
                                                          int, float*, const PcgState*, cudaStream_t);
template void launch_restrict<double, double>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                              const PcgState*, cudaStream_t);
template void launch_restrict<float, float>(const CoarseSpace&, double*, int, int, int, int, const float*,
                                            const PcgState*, cudaStream_t);
template void launch_restrict<float, __nv_bfloat16>(const CoarseSpace&, double*, int, int, int, int, const float*,
                                                    const PcgState*, cudaStream_t);
template void launch_restrict<double, float>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                             const PcgState*, cudaStream_t);
template void launch_restrict<double, __nv_bfloat16>(const CoarseSpace&, double*, int, int, int, int, const double*,
                                                     const PcgState*, cudaStream_t);
template void launch_prolong<double, double>(const CoarseSpace&, const double*, int, int, int, int, double*,
                                             const PcgState*, cudaStream_t);
template void launch_prolong<float, float>(const CoarseSpace&, const double*, int, int, int, int, float*,
                                           const PcgState*, cudaStream_t);
template void launch_prolong<float, __nv_bfloat16>(const CoarseSpace&, const double*, int, int, int, int, float*,
                                                   const PcgState*, cudaStream_t);

void launch_split_df(const double* a, float2* b, long long m, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_split_df, dim3(grid_for(m)), dim3(kThreads), 0, s, a, b, m);
}

void launch_stencil_coefs(const double* kinv, double* kcoef, int n, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_stencil_coefs, dim3(grid_for((long long)n * n)), dim3(kThreads), 0, s, kinv, kcoef, n);
}

template <typename TA, typename TB>
void launch_convert(const TA* a, TB* b, long long m, cudaStream_t s) {
  TG_COUNT(1);
  launch(k_convert<TA, TB>, dim3(grid_for(m)), dim3(kThreads), 0, s, a, b, m);
}
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, long long, cudaStream_t);

}  // namespace tg
