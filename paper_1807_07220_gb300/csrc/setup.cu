// Setup kernels (Step 2 of Section 5): local operators and their factors,
// snapshot spaces (eq. snapshot_eqn), local spectral problems (eqs.
// spectral_1, spectral_eqn), coarse basis tiles and the FP64 coarse matrix.
//
// Local operators are principal submatrices of K = C^T A_h C on the interior
// nodes of a cell rectangle (a block K_i or an oversampled block K_i^+): the
// zero-flux local saddle problems of the paper restricted to their
// divergence-free subspace.  Rectangles are given as int4 {x0, y0, nx, ny}:
// cell origin and interior node counts; local node (a, c) is global node
// (x0+1+a, y0+1+c), index c*nx + a, and the natural ordering gives band width
// w = nx + 1.  Band storage: row j holds L_{j, j-d} at j*(wmax+1) + d.
#include <algorithm>

#include "common.cuh"

namespace tg {
namespace {

__device__ __forceinline__ double kat(const double* kinv, int n, int i, int j) {
  return kinv[(long long)j * n + i];
}

__global__ void k_kinv(const double* __restrict__ kappa, double* __restrict__ kinv,
                       float* __restrict__ kinv32, int* status, int n) {
  const long long nn = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const double k = kappa[t];
    double v = 1.0;
    if (!(k > 0.0) || !isfinite(k)) atomicOr(status, kStBadKappa);
    else v = 1.0 / k;
    kinv[t] = v;
    kinv32[t] = (float)v;
  }
}

// lower band rows of the local operator of each rectangle
// slot (optional): band slot of matrix m (default m), so a compacted list of
// rectangles can update a band array indexed by the full matrix numbering
__global__ void k_assemble_band(const double* __restrict__ kinv, const int4* __restrict__ rects,
                                const int* __restrict__ slot, double* __restrict__ band, int wmax, int nmax, int n) {
  const int4 r = rects[blockIdx.x];
  const int nx = r.z, nloc = r.z * r.w, ldb = wmax + 1;
  double* B = band + (long long)(slot ? slot[blockIdx.x] : blockIdx.x) * nmax * ldb;
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
    const int a = q % nx, c = q / nx;
    const int i = r.x + 1 + a, j = r.y + 1 + c;
    const double k00 = kat(kinv, n, i - 1, j - 1), k10 = kat(kinv, n, i, j - 1);
    const double k01 = kat(kinv, n, i - 1, j), k11 = kat(kinv, n, i, j);
    double* row = B + (long long)q * ldb;
    for (int d = 0; d <= wmax; ++d) row[d] = 0.0;
    row[0] = (2.0 / 3.0) * (k00 + k10 + k01 + k11);
    if (a >= 1) row[1] = -(1.0 / 6.0) * (k00 + k01);                 // west
    if (c >= 1) {
      row[nx] = -(1.0 / 6.0) * (k00 + k10);                          // south
      if (a >= 1) row[nx + 1] = -(1.0 / 3.0) * k00;                  // south-west
      if (a + 1 < nx) row[nx - 1] = -(1.0 / 3.0) * k10;              // south-east
    }
  }
}

// right-looking band Cholesky, one CTA per matrix, band in shared memory.
// Column j: r = 1/sqrt(K_jj) comes from shared memory; every thread takes,
// for its pair (d1, d2), 1 <= d2 <= d1 <= w (one pair per thread,
// w (w + 1) / 2 <= blockDim), the scaled entries l1 = K_{j+d1, j} r,
// l2 = K_{j+d2, j} r; after a barrier it subtracts l1 l2 from K_{j+d1, j+d2}
// and the (d1, d1) thread stores l1.  The (1, 1) thread makes the last update
// of the next pivot, so it forms the next r at once (one reciprocal square
// root per column, not one per thread: FP64 is scarce on this GPU).  Two
// barriers per column.
__global__ void k_band_cholesky(double* __restrict__ band, const int4* __restrict__ rects,
                                const int* __restrict__ slot, int wmax, int nmax, int* status) {
  extern __shared__ double L[];
  const int4 r = rects[blockIdx.x];
  const int nx = r.z, nloc = r.z * r.w, w = nx + 1, ldb = wmax + 1;
  double* B = band + (long long)(slot ? slot[blockIdx.x] : blockIdx.x) * nmax * ldb;
  for (int t = threadIdx.x; t < nloc * ldb; t += blockDim.x) L[t] = B[t];
  // this thread's pair: t = d1 (d1 - 1) / 2 + (d2 - 1)
  const int t = threadIdx.x;
  int d1 = 1;
  while (d1 * (d1 + 1) / 2 <= t) ++d1;
  const int d2 = t - d1 * (d1 - 1) / 2 + 1;
  const bool has_pair = (d1 <= w);
  __shared__ double rsh;   // 1/sqrt of the current pivot
  __syncthreads();
  auto pivot_rsqrt = [&](int j) {
    double piv = L[(long long)j * ldb];
    if (!(piv > 0.0) || !isfinite(piv)) {
      atomicOr(status, kStNotSpd);
      piv = 1.0;
      L[(long long)j * ldb] = 1.0;
    }
    rsh = rsqrt(piv);
  };
  if (threadIdx.x == 0 && nloc > 0) pivot_rsqrt(0);
  __syncthreads();
  for (int j = 0; j < nloc; ++j) {
    const double rj = rsh;
    const bool act = has_pair && (j + d1 < nloc);
    double l1 = 0.0, l2 = 0.0;
    if (act) {
      l1 = L[(long long)(j + d1) * ldb + d1] * rj;
      l2 = L[(long long)(j + d2) * ldb + d2] * rj;
    }
    __syncthreads();
    if (act) {
      L[(long long)(j + d1) * ldb + (d1 - d2)] -= l1 * l2;
      if (d1 == d2) L[(long long)(j + d1) * ldb + d1] = l1;
    }
    if (threadIdx.x == 0) {
      L[(long long)j * ldb] *= rj;                // sqrt(K_jj) = K_jj / sqrt(K_jj)
      if (j + 1 < nloc) pivot_rsqrt(j + 1);       // pair (1, 1) just updated K_{j+1, j+1}
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nloc * ldb; q += blockDim.x) B[q] = L[q];
}

// Entries of the dense inverse from the band factor: thread t solves
// L L^T x = e_t for column t, and only rows j >= t are formed (the inverse is
// symmetric: entry (r, c) is read from scratch at row max(r, c), column
// min(r, c)).  CTA (m, y) takes columns c0 .. c0 + blockDim - 1 of matrix m,
// c0 = y blockDim (further chunks strided by gridDim.y blockDim), so that a
// few matrices still spread over many SMs.  Both triangular solves are
// right-looking: once a value is known its band column is added at once to
// the pending sums of the next w rows, which a private ring per thread in
// shared memory holds (ring[k * blockDim + thread]).  The chain of dependent
// FP64 operations from one row to the next is then a subtraction and a
// product (FP64 latency bounds this kernel when it runs on few matrices);
// the w updates per row are independent.  Every thread sweeps the rows in
// the same order, so band entries read from shared memory are broadcasts.
// scratch (row-major, rows j, columns t) holds nloc x nloc per matrix.
__global__ void k_band_inverse(const double* __restrict__ band, const int4* __restrict__ rects,
                               const int* __restrict__ slot, int first, int wmax, int nmax,
                               double* __restrict__ scratch) {
  extern __shared__ double sh[];
  const int m = first + blockIdx.x;
  const int4 r = rects[m];
  const int nx = r.z, nloc = r.z * r.w, w = nx + 1, ldb = wmax + 1, rl = wmax + 1;
  double* L = sh;
  double* rd = sh + (long long)nmax * ldb;
  double* ring = rd + nmax;
  const double* B = band + (long long)(slot ? slot[m] : m) * nmax * ldb;
  for (int t = threadIdx.x; t < nloc * ldb; t += blockDim.x) L[t] = B[t];
  __syncthreads();
  for (int t = threadIdx.x; t < nloc; t += blockDim.x) rd[t] = 1.0 / L[(long long)t * ldb];
  __syncthreads();
  double* X = scratch + (long long)blockIdx.x * nmax * nmax;
  double* my = ring + threadIdx.x;   // my[k * blockDim]: pending sum of the row in ring slot k
  const int T = blockDim.x;
  for (int c0 = blockIdx.y * T; c0 < nloc; c0 += gridDim.y * T) {
    const int t = c0 + threadIdx.x;
    const bool col = (t < nloc);
    for (int q = 0; q < rl; ++q) my[q * T] = 0.0;
    // forward, L y = e_t: y_j = (delta_jt - sum_{i<j} L_ji y_i) / L_jj (y_j = 0 for j < t)
    int pos = 0;   // ring slot of row j
    for (int j = c0; j < nloc; ++j) {
      const double y = (col && j >= t) ? (((j == t) ? 1.0 : 0.0) - my[pos * T]) * rd[j] : 0.0;
      my[pos * T] = 0.0;
      if (col && j >= t) X[(long long)j * nloc + t] = y;
      // L_{j+d, j} = L[(j + d) ldb + d]: add y_j's terms to the next rows
      const int dmax = min(w, nloc - 1 - j);
      const double* Lc = L + (long long)(j + 1) * ldb + 1;
      int q = pos;
      for (int d = 1; d <= dmax; ++d) {
        q = (q + 1 == rl) ? 0 : q + 1;
        my[q * T] = fma(Lc[(d - 1) * (ldb + 1)], y, my[q * T]);
      }
      pos = (pos + 1 == rl) ? 0 : pos + 1;
    }
    // backward, L^T x = y for rows j >= t: x_j = (y_j - sum_{i>j} L_ij x_i) / L_jj
    for (int q = 0; q < rl; ++q) my[q * T] = 0.0;
    pos = 0;       // ring slot of row j, counted from the last row
    for (int j = nloc - 1; j >= c0; --j) {
      const bool act = col && j >= t;
      double x = 0.0;
      if (act) {
        x = (X[(long long)j * nloc + t] - my[pos * T]) * rd[j];
        X[(long long)j * nloc + t] = x;
      }
      my[pos * T] = 0.0;
      // L_{j, j-d} = L[j ldb + d]: add x_j's terms to the rows above
      const int dmax = min(w, j);
      const double* Lr = L + (long long)j * ldb;
      int q = pos;
      for (int d = 1; d <= dmax; ++d) {
        q = (q + 1 == rl) ? 0 : q + 1;
        my[q * T] = fma(Lr[d], x, my[q * T]);
      }
      pos = (pos + 1 == rl) ? 0 : pos + 1;
    }
  }
}

// The same inverse for few matrices, with G lanes per column: the pending
// sums of a column's rows are split among its G lanes by row (row r belongs to
// lane r mod G), so each lane makes about w / G of the w updates per row, and
// the lane owning row j forms y_j (x_j in the backward sweep) and passes it to
// the others by a shuffle.  This cuts the FP64 instructions a warp issues per
// row about G-fold (FP64 issue bounds the first columns' long sweeps when one
// matrix is refactored alone).  CTA (m, y) takes blockDim / G columns; ring of
// pending sums per column in shared memory, slot of row r = r mod (wmax + 1).
template <int G>
__global__ void k_band_inverse_grp(const double* __restrict__ band, const int4* __restrict__ rects,
                                   const int* __restrict__ slot, int first, int wmax, int nmax,
                                   double* __restrict__ scratch) {
  extern __shared__ double sh[];
  const int m = first + blockIdx.x;
  const int4 r = rects[m];
  const int nx = r.z, nloc = r.z * r.w, w = nx + 1, ldb = wmax + 1, rl = wmax + 1;
  const int C = blockDim.x / G;   // columns per CTA
  double* L = sh;
  double* rd = sh + (long long)nmax * ldb;
  double* ring = rd + nmax;   // ring[col * rl + slot]
  const double* B = band + (long long)(slot ? slot[m] : m) * nmax * ldb;
  for (int t = threadIdx.x; t < nloc * ldb; t += blockDim.x) L[t] = B[t];
  __syncthreads();
  for (int t = threadIdx.x; t < nloc; t += blockDim.x) rd[t] = 1.0 / L[(long long)t * ldb];
  __syncthreads();
  double* X = scratch + (long long)blockIdx.x * nmax * nmax;
  const int cl = threadIdx.x / G, sub = threadIdx.x % G;
  const int lane = threadIdx.x & 31, base = lane - sub;   // first lane of this column's group
  double* my = ring + (long long)cl * rl;
  for (int c0 = blockIdx.y * C; c0 < nloc; c0 += gridDim.y * C) {
    const int t = c0 + cl;
    const bool col = (t < nloc);
    for (int q = sub; q < rl; q += G) my[q] = 0.0;
    __syncwarp();
    // forward, L y = e_t, rows j >= t (y_j = 0 above)
    for (int j = c0; j < nloc; ++j) {
      const int o = j % G;
      double y = 0.0;
      if (sub == o && col && j >= t) {
        const int q = j % rl;
        y = (((j == t) ? 1.0 : 0.0) - my[q]) * rd[j];
        my[q] = 0.0;
        X[(long long)j * nloc + t] = y;
      }
      y = __shfl_sync(0xffffffffu, y, base + o);
      if (col && j >= t) {
        const int dmax = min(w, nloc - 1 - j);
        // rows j + d owned by this lane: (j + d) % G == sub
        for (int d = (sub - j % G + G) % G; d <= dmax; d += G) {
          if (d == 0) continue;
          const int rr = j + d;
          my[rr % rl] = fma(L[(long long)rr * ldb + d], y, my[rr % rl]);
        }
      }
      __syncwarp();
    }
    for (int q = sub; q < rl; q += G) my[q] = 0.0;
    __syncwarp();
    // backward, L^T x = y for rows j >= t
    for (int j = nloc - 1; j >= c0; --j) {
      const int o = j % G;
      double x = 0.0;
      if (sub == o && col && j >= t) {
        const int q = j % rl;
        x = (X[(long long)j * nloc + t] - my[q]) * rd[j];
        my[q] = 0.0;
        X[(long long)j * nloc + t] = x;
      }
      x = __shfl_sync(0xffffffffu, x, base + o);
      if (col && j >= t) {
        const int dmax = min(w, j);
        // rows j - d owned by this lane: (j - d) % G == sub
        for (int d = (j % G - sub + G) % G; d <= dmax; d += G) {
          if (d == 0) continue;
          const int rr = j - d;
          my[rr % rl] = fma(L[(long long)j * ldb + d], x, my[rr % rl]);
        }
      }
      __syncwarp();
    }
  }
}

template <typename TS>
__global__ void k_store_inverse(const double* __restrict__ scratch, const PatchGeo* __restrict__ geo,
                                int first, int nmax, TS* __restrict__ pinv) {
  const PatchGeo g = geo[first + blockIdx.x];
  const double* X = scratch + (long long)blockIdx.x * nmax * nmax;
  TS* M = pinv + g.off;
  const long long tot = (long long)g.nloc * g.ld;
  for (long long t = threadIdx.x + (long long)blockIdx.y * blockDim.x; t < tot;
       t += (long long)blockDim.x * gridDim.y) {
    const int row = (int)(t / g.ld), col = (int)(t % g.ld);
    // lower triangle formed (rows >= columns): symmetric read
    const double v = (col < g.nloc) ? X[(long long)max(row, col) * g.nloc + min(row, col)] : 0.0;
    M[t] = from_d<TS>(v);
  }
}

// FP16 storage of the inverses: row q of patch p is multiplied by 2^(15 - e),
// e the binary exponent of its largest magnitude (frexp: max = m 2^e,
// m in [1/2, 1)), so the row maximum lands in [2^14, 2^15) below the FP16
// limit and the smallest entries keep most of their precision; the power-of-
// two factor is exact and rscale holds its inverse.  One warp per row.
__global__ void k_store_inverse_f16(const double* __restrict__ scratch, const PatchGeo* __restrict__ geo,
                                    const int* __restrict__ pidx, const int* __restrict__ gofs, int first, int nmax,
                                    __half* __restrict__ pinv, float* __restrict__ rscale) {
  const int c = first + blockIdx.x;
  const PatchGeo g = geo[c];
  const int p = pidx ? pidx[c] : c;   // patch number (geo may be a compacted list)
  const double* X = scratch + (long long)blockIdx.x * nmax * nmax;
  __half* M = pinv + g.off;
  const int lane = threadIdx.x & 31, nw = (blockDim.x >> 5) * gridDim.y;
  const int warp = (threadIdx.x >> 5) + blockIdx.y * (blockDim.x >> 5);
  // lower triangle formed (rows >= columns): entry (row, col) read symmetrically
  auto at = [&](int row, int col) { return X[(long long)max(row, col) * g.nloc + min(row, col)]; };
  for (int row = warp; row < g.nloc; row += nw) {
    double mx = 0.0;
    for (int col = lane; col < g.nloc; col += 32) mx = fmax(mx, fabs(at(row, col)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    const double sc = ldexp(1.0, 15 - e);
    for (int col = lane; col < g.ld; col += 32)
      M[(long long)row * g.ld + col] = __double2half(col < g.nloc ? at(row, col) * sc : 0.0);
    if (lane == 0) rscale[(long long)gofs[p] * kRowsPerGroup + row] = (float)ldexp(1.0, e - 15);
  }
}

// Patch inverses in the tensor-core tile layout (see kShapeTensor): entry e
// of lane l of tile (i, j) is M(16 i + l / 4 + 8 ((e >> 1) & 1),
// 16 j + 2 (l % 4) + (e & 1) + 8 (e >> 2)), the A-fragment order of
// mma.m16n8k16, zero outside the matrix.  FP16 rows are divided by their
// rscale (a power of two, so the stored value equals the row layout's).
template <typename TS>
__global__ void k_store_inverse_tiles(const double* __restrict__ scratch, const PatchGeo* __restrict__ geo,
                                      const int* __restrict__ gofs, const int* __restrict__ pidx, int first, int nmax,
                                      TS* __restrict__ tiles, const float* __restrict__ rscale) {
  const int c = first + blockIdx.x;
  const PatchGeo g = geo[c];
  const int p = pidx ? pidx[c] : c;
  const double* X = scratch + (long long)blockIdx.x * nmax * nmax;
  TS* out = tiles + g.toff;
  const int T = tiles_per_side(g.nloc);
  const long long tot = (long long)T * T * kTile * kTile;
  for (long long t = threadIdx.x + (long long)blockIdx.y * blockDim.x; t < tot;
       t += (long long)blockDim.x * gridDim.y) {
    const int tile = (int)(t >> 8), w = (int)(t & 255);
    const int lane = w >> 3, e = w & 7;
    const int i = tile / T, j = tile % T;
    const int row = kTile * i + (lane >> 2) + 8 * ((e >> 1) & 1);
    const int col = kTile * j + 2 * (lane & 3) + (e & 1) + 8 * (e >> 2);
    double v = 0.0;
    if (row < g.nloc && col < g.nloc) {
      v = X[(long long)max(row, col) * g.nloc + min(row, col)];   // lower triangle formed: symmetric read
      if (rscale) v /= (double)rscale[(long long)gofs[p] * kRowsPerGroup + row];
    }
    out[t] = from_d<TS>(v);
  }
}

// band factor of compact patch c (band rows L[j][d] = L_{j, j-d}) in the
// smoother's two padded band layouts at out + ids[c] * stride: column layout
// (entry (j, d >= 1) = L_{j+d, j}) then row layout (entry (j, d >= 1) =
// L_{j, j-d}); entry (j, 0) = 1 / L_jj in both, zero outside the matrix;
// rows in groups of four, interleaved by entry (the order the sweeps load)
template <typename TB>
__global__ void k_store_band(const double* __restrict__ band, const int4* __restrict__ rects,
                             const int* __restrict__ ids, int wmax, int nmax, long long stride, TB* __restrict__ out) {
  const int c = blockIdx.x;
  const int4 r = rects[c];
  const int nloc = r.z * r.w, ldb = wmax + 1;
  const double* B = band + (long long)c * nmax * ldb;
  TB* O = out + (long long)(ids ? ids[c] : c) * stride;
  const long long tot = stride / 2;   // one layout: band_rows(nmax) rows in groups of four, ldb wide
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int e = (int)(t % (4 * ldb));
    const int j = (int)(t / (4 * ldb)) * 4 + (e & 3) - kBandPad, d = e >> 2;
    double vc = 0.0, vr = 0.0;
    if (j >= 0 && j < nloc && d < ldb) {
      if (d == 0) {
        vc = vr = 1.0 / B[(long long)j * ldb];
      } else {
        if (j + d < nloc) vc = B[(long long)(j + d) * ldb + d];   // L_{j+d, j}
        if (j - d >= 0) vr = B[(long long)j * ldb + d];           // L_{j, j-d}
      }
    }
    O[t] = (TB)vc;
    O[tot + t] = (TB)vr;
  }
}

// flag[m] = 1 if any cell of rectangle m (cells x0 <= i <= x0 + nx,
// y0 <= j <= y0 + ny) gets a new inverse permeability: 1/kappa computed as
// k_kinv does, compared bit for bit with the stored value
__global__ void k_rect_changed(const double* __restrict__ kappa, const double* __restrict__ kinv_old,
                               const int4* __restrict__ rects, int n, unsigned char* __restrict__ flag) {
  const int4 r = rects[blockIdx.x];
  const int cw = r.z + 1, ch = r.w + 1;
  int ch_any = 0;
  for (int t = threadIdx.x; t < cw * ch; t += blockDim.x) {
    const long long c = (long long)(r.y + t / cw) * n + r.x + t % cw;
    const double k = kappa[c];
    const double v = (k > 0.0 && isfinite(k)) ? 1.0 / k : 1.0;
    if (v != kinv_old[c]) ch_any = 1;
  }
  ch_any = __syncthreads_or(ch_any);
  if (threadIdx.x == 0) flag[blockIdx.x] = (unsigned char)ch_any;
}

// ---------------------------------------------------------------------------
// Snapshot spaces.  For block K = (I, J) and an interior side s (0 L, 1 R,
// 2 B, 3 T) the snapshot space of Section 4.1 restricted to K is spanned by
//   fn 0:    the unit-flux function RT_s + C psi (coarse RT0 half-function of
//            side s plus the energy-minimising divergence-free correction,
//            psi = 0 on dK) -- the MsFEM function of eq. msfem on K;
//   fn k>=1: C psi with psi = 1 at the k-th interior node of side s, zero on
//            the rest of dK, discrete-harmonic (K psi = 0) inside K.
// (Any delta_l snapshot is (1/b) fn0 plus a combination of the fn k >= 1;
// the span is the same.)  Outputs the closed-block psi of every function and
// the Gram matrix int_K kappa^{-1} u_a . u_b.

// normal value of RT_s at fine x-face column i' (local 0..b) / y-face row
__device__ __forceinline__ double rt_value(int side, int t, int b) {
  const double x = (double)t / b;
  return (side == 0 || side == 2) ? 1.0 - x : x;
}

__device__ __forceinline__ void side_node(int side, int k, int b, int& a, int& c) {
  if (side == 0) { a = 0; c = k; }
  else if (side == 1) { a = b; c = k; }
  else if (side == 2) { a = k; c = 0; }
  else { a = k; c = b; }
}

__device__ __forceinline__ bool side_interior(int side, int I, int J, int nc) {
  return (side == 0) ? I >= 1 : (side == 1) ? I + 1 < nc : (side == 2) ? J >= 1 : J + 1 < nc;
}

__device__ __forceinline__ void warp_band_solve_s(const double* L, int ldb, int nloc, int w, double* x) {
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < nloc; ++j) {
    double yj = 0.0;
    if (lane == 0) {
      yj = x[j] / L[j * ldb];
      x[j] = yj;
    }
    yj = __shfl_sync(0xffffffffu, yj, 0);
    __syncwarp();
    for (int d = 1 + lane; d <= w; d += 32)
      if (j + d < nloc) x[j + d] -= L[(j + d) * ldb + d] * yj;
    __syncwarp();
  }
  for (int j = nloc - 1; j >= 0; --j) {
    double xj = 0.0;
    if (lane == 0) {
      xj = x[j] / L[j * ldb];
      x[j] = xj;
    }
    xj = __shfl_sync(0xffffffffu, xj, 0);
    __syncwarp();
    for (int d = 1 + lane; d <= w; d += 32)
      if (j - d >= 0) x[j - d] -= L[j * ldb + d] * xj;
    __syncwarp();
  }
}

// position k (1..b-1) of closed-block node (a, c) among the interior nodes of
// side s, or 0 if the node is not one of them
__device__ __forceinline__ int side_position(int side, int a, int c, int b) {
  if (side == 0) return (a == 0 && c >= 1 && c <= b - 1) ? c : 0;
  if (side == 1) return (a == b && c >= 1 && c <= b - 1) ? c : 0;
  if (side == 2) return (c == 0 && a >= 1 && a <= b - 1) ? a : 0;
  return (c == b && a >= 1 && a <= b - 1) ? a : 0;
}

__device__ __forceinline__ int face_of_side(int side, int I, int J, int nc) {
  const int nV = nc * (nc - 1);
  if (side == 0) return J * (nc - 1) + (I - 1);
  if (side == 1) return J * (nc - 1) + I;
  if (side == 2) return nV + (J - 1) * nc + I;
  return nV + J * nc + I;
}

// Function fn of a side is sum_j coef_j f_j over the snapshot functions above
// (coef = e_fn when the coefficient array is NULL): boundary data
// psi = coef_j on the j-th interior node of the side, forcing coef_0 times the
// RT_s forcing, interior solved with the block's band factor.
// Dynamic shared memory: L[(b-1)^2 (b+1)] | psi[nfn (b+1)^2] | kloc[b^2] |
// coefficient rows [nfn b] | solve lines [warps (b-1)^2]
constexpr int kGramChunk = 8;   // cells per pass of the snapshot Gram
__global__ void k_snapshots(const double* __restrict__ kinv, const double* __restrict__ blk_band,
                            const double* __restrict__ coef, int nfn, const unsigned char* __restrict__ mask,
                            double* __restrict__ psiS, double* __restrict__ gram, int n, int b) {
  extern __shared__ double sm[];
  const int nc = n / b;
  const int blk = blockIdx.x >> 2, side = blockIdx.x & 3;
  const int I = blk % nc, J = blk / nc;
  if (!side_interior(side, I, J, nc)) return;
  if (mask && !mask[blockIdx.x]) return;
  const int nx = b - 1, nloc = nx * nx, ldb = b + 1, w = b;  // block band width w = nx + 1
  const int nb1 = b + 1, ncl = nb1 * nb1;
  double* L = sm;
  double* psi = L + nloc * ldb;
  double* kl = psi + nfn * ncl;
  double* cf = kl + b * b;
  const double h = 1.0 / n;
  const double* Bg = blk_band + (long long)blk * nloc * ldb;
  for (int t = threadIdx.x; t < nloc * ldb; t += blockDim.x) L[t] = Bg[t];
  for (int t = threadIdx.x; t < b * b; t += blockDim.x)
    kl[t] = kinv[(long long)(J * b + t / b) * n + I * b + t % b];
  const double* crow = coef ? coef + (long long)face_of_side(side, I, J, nc) * nfn * b : nullptr;
  for (int t = threadIdx.x; t < nfn * b; t += blockDim.x)
    cf[t] = crow ? crow[t] : ((t / b == t % b) ? 1.0 : 0.0);
  __syncthreads();
  // closed psi: boundary data, interior = right-hand side
  for (int t = threadIdx.x; t < nfn * ncl; t += blockDim.x) {
    const int fn = t / ncl, node = t % ncl, a = node % nb1, c = node / nb1;
    const int pos = side_position(side, a, c, b);
    psi[t] = pos ? cf[fn * b + pos] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nfn * ncl; t += blockDim.x) {
    const int fn = t / ncl, node = t % ncl, a = node % nb1, c = node / nb1;
    if (!(a >= 1 && a <= b - 1 && c >= 1 && c <= b - 1)) continue;
    const double k00 = kl[(c - 1) * b + a - 1], k10 = kl[(c - 1) * b + a];
    const double k01 = kl[c * b + a - 1], k11 = kl[c * b + a];
    double rhs = 0.0;
    const double c0 = cf[fn * b];
    if (c0 != 0.0) {
      // -C^T A RT_s at node (a, c); A RT_s / h on a face = h * (...) with RT values
      if (side <= 1) {
        // x-faces (a, c-1) [node on top] and (a, c) [node at bottom]; cells row c-1 / c
        auto ax = [&](double kL, double kR) {
          return h * ((kL + kR) / 3.0 * rt_value(side, a, b) +
                      (kL * rt_value(side, a - 1, b) + kR * rt_value(side, a + 1, b)) / 6.0);
        };
        rhs = -c0 * (ax(k00, k10) - ax(k01, k11));
      } else {
        auto ay = [&](double kB, double kT) {
          return h * ((kB + kT) / 3.0 * rt_value(side, c, b) +
                      (kB * rt_value(side, c - 1, b) + kT * rt_value(side, c + 1, b)) / 6.0);
        };
        // y-faces (a-1, c) [node on the right] and (a, c) [node on the left]
        rhs = -c0 * (-ay(k00, k01) + ay(k10, k11));
      }
    }
    // boundary data: interior entries of P are being overwritten with
    // right-hand sides by other threads, and the data field is zero there
    const double* P = psi + fn * ncl;
    auto at = [&](int da, int dc) {
      const int aa = a + da, cc = c + dc;
      const bool in = (aa >= 1 && aa <= b - 1 && cc >= 1 && cc <= b - 1);
      return in ? 0.0 : P[cc * nb1 + aa];
    };
    double kp = (2.0 / 3.0) * (k00 + k10 + k01 + k11) * at(0, 0);
    kp -= (1.0 / 6.0) * ((k00 + k10) * at(0, -1) + (k01 + k11) * at(0, 1) + (k00 + k01) * at(-1, 0) +
                         (k10 + k11) * at(1, 0));
    kp -= (1.0 / 3.0) * (k00 * at(-1, -1) + k10 * at(1, -1) + k01 * at(-1, 1) + k11 * at(1, 1));
    psi[t] = rhs - kp;  // interior slot used as right-hand side
  }
  __syncthreads();
  // solve: warp per function, in a compact interior vector stored in the
  // function's own interior slots (copied to a temporary line first)
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* tmp = cf + nfn * b;  // nw * nloc scratch
    double* x = tmp + warp * nloc;
    for (int fn = warp; fn < nfn; fn += nw) {
      double* P = psi + fn * ncl;
      for (int q = lane; q < nloc; q += 32) x[q] = P[(1 + q / nx) * nb1 + 1 + q % nx];
      __syncwarp();
      warp_band_solve_s(L, ldb, nloc, w, x);
      for (int q = lane; q < nloc; q += 32) P[(1 + q / nx) * nb1 + 1 + q % nx] = x[q];
      __syncwarp();
    }
  }
  __syncthreads();
  double* outp = psiS + ((long long)blk * 4 + side) * b * ncl;
  for (int t = threadIdx.x; t < nfn * ncl; t += blockDim.x) outp[t] = psi[t];
  // Gram: G[fa][fb] = sum over the block's cells of u_a^T (kappa^{-1} M) u_b,
  // with u_f the cell's four face values (h times the normal velocity of
  // coef_{f,0} RT_s + C psi_f on the left, right, bottom and top faces) and
  // M the RT0 mass pattern (1/3 on a face, 1/6 between opposite faces).  The
  // cells go in chunks of kGramChunk: the chunk's u and kappa^{-1} M u of every
  // function are formed once in shared memory, then one thread per pair
  // (fa <= fb) adds their inner products.
  double* Ug = cf + nfn * b + (blockDim.x >> 5) * nloc;   // [nfn][kGramChunk][4]
  double* Wg = Ug + nfn * kGramChunk * 4;                  // [nfn][kGramChunk][4]
  double* G = gram + ((long long)blk * 4 + side) * b * b;
  const int npair = nfn * (nfn + 1) / 2;
  int fa = -1, fb = -1;
  if ((int)threadIdx.x < npair) {
    int rem = threadIdx.x;
    fa = 0;
    while (rem >= nfn - fa) { rem -= nfn - fa; ++fa; }
    fb = fa + rem;
  }
  double e = 0.0;
  for (int c0 = 0; c0 < b * b; c0 += kGramChunk) {
    for (int t = threadIdx.x; t < nfn * kGramChunk; t += blockDim.x) {
      const int fn = t / kGramChunk, cell = c0 + t % kGramChunk;
      double u[4] = {0.0, 0.0, 0.0, 0.0}, k = 0.0;
      if (cell < b * b) {
        const int a = cell % b, c = cell / b;
        const int n00 = c * nb1 + a, n10 = n00 + 1, n01 = n00 + nb1, n11 = n01 + 1;
        const double* P = psi + fn * ncl;
        const double cfn = cf[fn * b];
        u[0] = P[n01] - P[n00];
        u[1] = P[n11] - P[n10];
        u[2] = -(P[n10] - P[n00]);
        u[3] = -(P[n11] - P[n01]);
        if (side <= 1) {
          u[0] += cfn * h * rt_value(side, a, b);
          u[1] += cfn * h * rt_value(side, a + 1, b);
        } else {
          u[2] += cfn * h * rt_value(side, c, b);
          u[3] += cfn * h * rt_value(side, c + 1, b);
        }
        k = kl[cell];
      }
      double* Uc = Ug + (long long)t * 4;
      double* Wc = Wg + (long long)t * 4;
      Uc[0] = u[0]; Uc[1] = u[1]; Uc[2] = u[2]; Uc[3] = u[3];
      Wc[0] = k * (u[0] / 3.0 + u[1] / 6.0);
      Wc[1] = k * (u[0] / 6.0 + u[1] / 3.0);
      Wc[2] = k * (u[2] / 3.0 + u[3] / 6.0);
      Wc[3] = k * (u[2] / 6.0 + u[3] / 3.0);
    }
    __syncthreads();
    if (fa >= 0) {
      const double* Ua = Ug + fa * kGramChunk * 4;
      const double* Wb = Wg + fb * kGramChunk * 4;
#pragma unroll 4
      for (int i = 0; i < kGramChunk * 4; ++i) e = fma(Ua[i], Wb[i], e);
    }
    __syncthreads();
  }
  if (fa >= 0) {
    G[fa * b + fb] = e;
    G[fb * b + fa] = e;
  }
}

// ---------------------------------------------------------------------------
// Per coarse face: local spectral problem a c = lambda s c (eq. spectral_1)
// in the basis {m, d_1..d_{b-1}} of the snapshot space (m: unit-flux MsFEM
// function on omega_i, d_k: harmonic extensions of psi = e_k on E_i).
//   s = H^{-1} (Gram_{K1} + Gram_{K2} + div term), div term 2 on (m, m);
//   a = N diag(kappa_e^{-1}) N^T with N the normal values on the fine faces
//       of E_i (fine-face trace product, kappa_e^{-1} the mean of the two
//       adjacent cells).
// Solved as L_a^{-1} s L_a^{-T} y = mu y (a = L_a L_a^T, mu = 1/lambda) by
// Jacobi rotations (jacobi_warp on the face's warp; jacobi_serial for the
// small Ritz problems), so the selected (small lambda = large mu) pairs carry
// full relative accuracy.  Then the selected span is split into one function with
// unit m-coefficient (unit flux through E_i, min-norm combination) and
// nsel-1 zero-flux functions (a Householder complement of the m-coefficients).
constexpr int kJ = kMaxB;

__device__ void jacobi_serial(double (*A)[kJ], double (*V)[kJ], int m) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  double scale = 0.0;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) scale += A[i][j] * A[i][j];
  scale = sqrt(scale);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        if (i != j) off += A[i][j] * A[i][j];
    if (sqrt(off) <= 1e-15 * scale) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p][q];
        if (apq == 0.0) continue;
        const double diff = A[q][q] - A[p][p];
        double t;
        if (fabs(diff) > 1e150 * fabs(apq)) {
          t = apq / diff;
        } else {
          const double tau = diff / (2.0 * apq);
          t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
        }
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        A[p][q] = A[q][p] = 0.0;
        for (int k = 0; k < m; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// The same Jacobi iteration on one warp (all 32 lanes call it): the m
// indices, padded to an even count m2, meet in m2 - 1 rounds of m2 / 2
// disjoint pairs per sweep (round-robin ordering).  Each round, one lane per
// pair forms its rotation from the current A (the formula of jacobi_serial);
// the rotations, which commute, are then applied to the columns of A, to its
// rows and to the columns of V with the work spread over the warp.  Same
// stopping test.
__device__ void jacobi_warp(double (*A)[kJ], double (*V)[kJ], int m, int lane) {
  __shared__ double rc[kJ / 2], rs[kJ / 2];
  __shared__ int rp[kJ / 2], rq[kJ / 2], rot[kJ / 2];
  for (int t = lane; t < m * m; t += 32) V[t / m][t % m] = (t / m == t % m) ? 1.0 : 0.0;
  const int m2 = m + (m & 1), np = m2 / 2;
  double loc = 0.0;
  for (int t = lane; t < m * m; t += 32) loc += A[t / m][t % m] * A[t / m][t % m];
  const double scale = sqrt(warp_sum(loc));
  __syncwarp();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int t = lane; t < m * m; t += 32)
      if (t / m != t % m) off += A[t / m][t % m] * A[t / m][t % m];
    off = warp_sum(off);   // the same value in every lane
    if (sqrt(off) <= 1e-15 * scale) break;
    for (int r = 0; r < m2 - 1; ++r) {
      if (lane < np) {
        int p = lane == 0 ? r : (r + lane) % (m2 - 1);
        int q = lane == 0 ? m2 - 1 : (r - lane + (m2 - 1)) % (m2 - 1);
        if (p > q) { const int x = p; p = q; q = x; }
        double c = 1.0, sn = 0.0;
        int did = 0;
        if (q < m && A[p][q] != 0.0) {   // the padding index rotates nothing
          const double apq = A[p][q], diff = A[q][q] - A[p][p];
          double t;
          if (fabs(diff) > 1e150 * fabs(apq)) {
            t = apq / diff;
          } else {
            const double tau = diff / (2.0 * apq);
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
          }
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
          did = 1;
        }
        rp[lane] = p; rq[lane] = q; rc[lane] = c; rs[lane] = sn; rot[lane] = did;
      }
      __syncwarp();
      for (int t = lane; t < m * np; t += 32) {   // columns of A: (row i, pair k)
        const int i = t / np, k = t % np;
        if (!rot[k]) continue;
        const int p = rp[k], q = rq[k];
        const double c = rc[k], sn = rs[k], aip = A[i][p], aiq = A[i][q];
        A[i][p] = c * aip - sn * aiq;
        A[i][q] = sn * aip + c * aiq;
      }
      __syncwarp();
      for (int t = lane; t < m * np; t += 32) {   // rows of A and columns of V: (index j, pair k)
        const int j = t / np, k = t % np;
        if (!rot[k]) continue;
        const int p = rp[k], q = rq[k];
        const double c = rc[k], sn = rs[k];
        const double apj = A[p][j], aqj = A[q][j];
        A[p][j] = c * apj - sn * aqj;
        A[q][j] = sn * apj + c * aqj;
        const double vjp = V[j][p], vjq = V[j][q];
        V[j][p] = c * vjp - sn * vjq;
        V[j][q] = sn * vjp + c * vjq;
      }
      __syncwarp();
      if (lane < np && rot[lane]) A[rp[lane]][rq[lane]] = A[rq[lane]][rp[lane]] = 0.0;
      __syncwarp();
    }
  }
}

__device__ bool cholesky_serial(double (*A)[kJ], int m) {  // lower factor in place
  for (int j = 0; j < m; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = A[i][j];
      for (int k = 0; k < j; ++k) v -= A[i][k] * A[j][k];
      A[i][j] = v / d;
    }
    for (int k = j + 1; k < m; ++k) A[j][k] = 0.0;
  }
  return true;
}

__device__ __forceinline__ void face_geometry(int f, int nc, int& kind, int& I, int& J) {
  const int nV = nc * (nc - 1);
  if (f < nV) { kind = 0; I = f % (nc - 1) + 1; J = f / (nc - 1); }
  else { kind = 1; I = (f - nV) % nc; J = (f - nV) / nc + 1; }
}

// mean inverse permeability of the two cells at fine face l of coarse face (kind, I, J)
__device__ __forceinline__ double face_kinv(const double* kinv, int n, int b, int kind, int I, int J, int l) {
  double kl, kr;
  if (kind == 0) { kl = kinv[(long long)(J * b + l) * n + I * b - 1]; kr = kinv[(long long)(J * b + l) * n + I * b]; }
  else { kl = kinv[(long long)(J * b - 1) * n + I * b + l]; kr = kinv[(long long)(J * b) * n + I * b + l]; }
  return 0.5 * (kl + kr);
}

// normal values on fine faces l of E_i of {m, d_1..d_{b-1}}: Nl[0] = 1;
// d_k = +-1/h on faces k-1 (node k above / right) and k
__device__ __forceinline__ void normal_values(int kind, int l, int b, double h, double* Nl) {
  for (int k = 0; k < b; ++k) Nl[k] = 0.0;
  Nl[0] = 1.0;
  const double sg = (kind == 0) ? 1.0 : -1.0;
  if (l + 1 <= b - 1) Nl[l + 1] = sg / h;   // face l has node l+1 as its upper/right end
  if (l >= 1) Nl[l] = -sg / h;              // and node l as its lower/left end
}

__global__ void k_face_spectral(SpectralArgs A) {
  // one warp per face: lane 0 assembles the problem and selects the
  // functions, the warp runs the Jacobi iteration
  const int lane = threadIdx.x;
  __shared__ double S[kJ][kJ], Aa[kJ][kJ], V[kJ][kJ], C[kJ][kJ];
  __shared__ double mu[kJ], lamv[kJ], wv[kJ];
  __shared__ int ord[kJ];
  __shared__ int go;
  const int n = A.n, b = A.b, nc = n / b;
  const int f = blockIdx.x;
  if (A.fmask && !A.fmask[f]) return;
  int kind, I, J;
  face_geometry(f, nc, kind, I, J);
  int blk1, side1, blk2, side2;
  if (kind == 0) { blk1 = J * nc + I - 1; side1 = 1; blk2 = J * nc + I; side2 = 0; }
  else { blk1 = (J - 1) * nc + I; side1 = 3; blk2 = J * nc + I; side2 = 2; }
  const double h = 1.0 / n, H = b * h;
  const bool learned = (A.prof != nullptr);
  const int m_fn = learned ? A.jpred[f] : b;    // functions of the face
  if (lane == 0) {
    go = 0;
    if (A.jeff) A.jeff[f] = m_fn;
    for (int k = 0; k < b; ++k) A.lam[(long long)f * b + k] = INFINITY;
    if (learned && m_fn < 1) {                     // nothing predicted: exact problem
      A.fallback[f] = 1;
    } else {
      // flux weights: coefficient of m in each function
      for (int i = 0; i < m_fn; ++i) wv[i] = learned ? A.ccoef[((long long)f * A.kmax + i) * b] : (i == 0 ? 1.0 : 0.0);
      const double* G1 = A.gram + ((long long)blk1 * 4 + side1) * b * b;
      const double* G2 = A.gram + ((long long)blk2 * 4 + side2) * b * b;
      // s = H^{-1} (Gram_{K1} + Gram_{K2} + div term), div term 2 w_i w_j
      for (int i = 0; i < m_fn; ++i)
        for (int j = 0; j < m_fn; ++j) S[i][j] = (G1[i * b + j] + G2[i * b + j] + 2.0 * wv[i] * wv[j]) / H;
      // a = N diag(kappa_e^{-1}) N^T, N the normal values of the functions on E_i
      for (int i = 0; i < m_fn; ++i)
        for (int j = 0; j < m_fn; ++j) Aa[i][j] = 0.0;
      for (int l = 0; l < b; ++l) {
        const double ke = face_kinv(A.kinv, n, b, kind, I, J, l);
        double Nl[kJ];
        if (learned) {
          for (int i = 0; i < m_fn; ++i) Nl[i] = A.prof[((long long)f * A.kmax + i) * b + l];
        } else {
          normal_values(kind, l, b, h, Nl);
        }
        for (int i = 0; i < m_fn; ++i)
          for (int j = 0; j < m_fn; ++j) Aa[i][j] += ke * Nl[i] * Nl[j];
      }
      if (!cholesky_serial(Aa, m_fn)) {
        atomicOr(A.status, kStNotSpd);
      } else {
        // S <- L^{-1} S L^{-T}
        for (int col = 0; col < m_fn; ++col)
          for (int i = 0; i < m_fn; ++i) {
            double v = S[i][col];
            for (int k = 0; k < i; ++k) v -= Aa[i][k] * S[k][col];
            S[i][col] = v / Aa[i][i];
          }
        for (int row = 0; row < m_fn; ++row)
          for (int i = 0; i < m_fn; ++i) {
            double v = S[row][i];
            for (int k = 0; k < i; ++k) v -= Aa[i][k] * S[row][k];
            S[row][i] = v / Aa[i][i];
          }
        for (int i = 0; i < m_fn; ++i)
          for (int j = 0; j < i; ++j) {
            const double v = 0.5 * (S[i][j] + S[j][i]);
            S[i][j] = S[j][i] = v;
          }
        go = 1;
      }   // Cholesky of a
    }   // functions to solve for
  }   // lane 0
  __syncwarp();
  if (!go) return;
  jacobi_warp(S, V, m_fn, lane);
  __syncwarp();
  if (lane != 0) return;
  for (int k = 0; k < m_fn; ++k) { mu[k] = S[k][k]; ord[k] = k; }
  // descending mu = ascending lambda (stable insertion sort)
  for (int i = 1; i < m_fn; ++i) {
    const int o = ord[i];
    int j = i - 1;
    while (j >= 0 && mu[ord[j]] < mu[o]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = o;
  }
  for (int k = 0; k < m_fn; ++k) {
    lamv[k] = 1.0 / mu[ord[k]];
    A.lam[(long long)f * b + k] = lamv[k];
  }
  int m = 0;
  while (m < m_fn && lamv[m] < A.eig_tol) ++m;
  if (m < 1) m = 1;
  if (A.max_basis > 0 && m > A.max_basis) m = A.max_basis;
  if (A.mode != 0) m = 1;
  if (learned) {
    const int fb = (lamv[0] >= A.eig_tol) ? 1 : 0;
    A.fallback[f] = fb;
    if (fb) return;
  }
  if (!learned) A.nsel[f] = m;
  // coefficient vectors c_k = L^{-T} y_k / sqrt(mu_k) (s-orthonormal); the
  // labels need the klab lowest modes, selected or not
  const int mc = A.labels ? max(m, min(A.klab, m_fn)) : m;
  for (int k = 0; k < mc; ++k) {
    const int o = ord[k];
    for (int i = m_fn - 1; i >= 0; --i) {
      double v = V[i][o];
      for (int r = i + 1; r < m_fn; ++r) v -= Aa[r][i] * C[r][k];
      C[i][k] = v / Aa[i][i];
    }
    const double sc = 1.0 / sqrt(mu[o]);
    for (int i = 0; i < m_fn; ++i) C[i][k] *= sc;
  }
  if (A.labels) {
    // whitened profiles y_k = a^{1/2} N^T c_k of the min(klab, b) lowest modes,
    // orthonormalised by modified Gram-Schmidt (twice), zero-padded
    const int ml = min(A.klab, m_fn);
    float* out = A.labels + (long long)f * A.klab * b;
    double P[kJ][kJ];
    for (int k = 0; k < ml; ++k)
      for (int l = 0; l < b; ++l) {
        double Nl[kJ];
        normal_values(kind, l, b, h, Nl);
        double g = 0.0;
        for (int i = 0; i < m_fn; ++i) g += Nl[i] * C[i][k];
        P[k][l] = sqrt(face_kinv(A.kinv, n, b, kind, I, J, l)) * g;   // whitened y = a^{1/2} g
      }
    for (int k = 0; k < ml; ++k) {
      for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q < k; ++q) {
          double d = 0.0;
          for (int l = 0; l < b; ++l) d += P[q][l] * P[k][l];
          for (int l = 0; l < b; ++l) P[k][l] -= d * P[q][l];
        }
      double nr = 0.0;
      for (int l = 0; l < b; ++l) nr += P[k][l] * P[k][l];
      nr = sqrt(nr);
      for (int l = 0; l < b; ++l) P[k][l] = (nr > 0.0) ? P[k][l] / nr : 0.0;
    }
    for (int k = 0; k < A.klab; ++k)
      for (int l = 0; l < b; ++l) out[k * b + l] = (k < ml) ? (float)P[k][l] : 0.0f;
  }
  double* fc = A.fcoef + (long long)f * b;
  double* zc = A.zcoef + (long long)f * (b - 1) * b;
  if (A.mode != 0) {  // MsFEM / RT0: the unit-flux MsFEM function alone
    for (int i = 0; i < b; ++i) fc[i] = (i == 0) ? 1.0 : 0.0;
    return;
  }
  // net flux of each selected function: t_k = sum_i w_i C[i][k]
  double t[kJ];
  double tn = 0.0, cmax = 0.0;
  for (int k = 0; k < m; ++k) {
    double v = 0.0;
    for (int i = 0; i < m_fn; ++i) v += wv[i] * C[i][k];
    t[k] = v;
    tn += v * v;
  }
  for (int k = 0; k < m; ++k)
    for (int i = 0; i < m_fn; ++i) cmax = fmax(cmax, fabs(C[i][k]));
  if (learned && !(sqrt(tn) > 1e-6 * cmax)) {
    // the kept predicted functions carry no net flux through E_i: exact problem
    A.fallback[f] = 1;
    return;
  }
  if (!(sqrt(tn) > 1e-12 * cmax)) {
    atomicOr(A.status, kStDegenerate);
    for (int i = 0; i < b; ++i) fc[i] = (!learned && i == 0) ? 1.0 : 0.0;
    return;
  }
  if (learned) A.nsel[f] = m;
  // unit-flux function: the min-norm combination with sum_k t_k a_k = 1
  for (int i = 0; i < b; ++i) {
    double v = 0.0;
    if (i < m_fn)
      for (int k = 0; k < m; ++k) v += C[i][k] * t[k] / tn;
    fc[i] = v;
  }
  if (!learned) fc[0] = 1.0;
  if (m > 1) {
    // Householder H = I - 2 v v^T / v^T v with v = t + sign(t0) |t| e0 maps t to -sign |t| e0;
    // columns 1..m-1 of H span t^perp: the zero-flux functions
    double v[kJ];
    for (int k = 0; k < m; ++k) v[k] = t[k];
    const double tnorm = sqrt(tn);
    v[0] += (v[0] >= 0.0 ? tnorm : -tnorm);
    double vv = 0.0;
    for (int k = 0; k < m; ++k) vv += v[k] * v[k];
    for (int q = 1; q < m; ++q) {
      for (int i = 0; i < b; ++i) {
        double acc = 0.0;
        if (i < m_fn)
          for (int k = 0; k < m; ++k) {
            const double Hkq = ((k == q) ? 1.0 : 0.0) - 2.0 * v[k] * v[q] / vv;
            acc += C[i][k] * Hkq;
          }
        zc[(long long)(q - 1) * b + i] = (!learned && i == 0) ? 0.0 : acc;
      }
    }
  }
}

// Predicted whitened profiles of a face (network output, k x b, y_l =
// a_l^{1/2} g_l) -> an orthonormal basis of the directions of their span with
// G^T G eigenvalue > thr, converted to flux profiles g = a^{-1/2} y, and each
// direction's coefficients over {m, d_1..d_{b-1}}: c_0 = the mean normal
// value, d_j = sg h sum_{l<j} (g_l - c_0) (inverse of the normal-value map).
__global__ void k_pred_basis(const float* __restrict__ y, const double* __restrict__ kinv, int k, int n, int b,
                             double thr, double* __restrict__ prof, double* __restrict__ ccoef,
                             int* __restrict__ jpred, int nfaces) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfaces) return;
  const int nc = n / b;
  int kind, I, J;
  face_geometry(f, nc, kind, I, J);
  const double h = 1.0 / n, sg = (kind == 0) ? 1.0 : -1.0;
  constexpr int kK = 8;
  double Gm[kJ][kJ], Vm[kJ][kJ];
  const float* Y = y + (long long)f * k * b;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double v = 0.0;
      for (int l = 0; l < b; ++l) v += (double)Y[i * b + l] * (double)Y[j * b + l];
      Gm[i][j] = v;
    }
  jacobi_serial(Gm, Vm, k);
  int order[kK];
  int r = 0;
  for (int i = 0; i < k; ++i)
    if (Gm[i][i] > thr) order[r++] = i;
  // largest eigenvalue first
  for (int i = 1; i < r; ++i) {
    const int o = order[i];
    int j = i - 1;
    while (j >= 0 && Gm[order[j]][order[j]] < Gm[o][o]) { order[j + 1] = order[j]; --j; }
    order[j + 1] = o;
  }
  jpred[f] = r;
  for (int q = 0; q < k; ++q) {
    double* P = prof + ((long long)f * k + q) * b;
    double* Cc = ccoef + ((long long)f * k + q) * b;
    if (q >= r) {
      for (int l = 0; l < b; ++l) { P[l] = 0.0; Cc[l] = 0.0; }
      continue;
    }
    const int o = order[q];
    const double sc = 1.0 / sqrt(Gm[o][o]);
    double mean = 0.0;
    for (int l = 0; l < b; ++l) {
      double g = 0.0;
      for (int i = 0; i < k; ++i) g += (double)Y[i * b + l] * Vm[i][o];
      P[l] = g * sc / sqrt(face_kinv(kinv, n, b, kind, I, J, l));
      mean += P[l];
    }
    mean /= b;
    Cc[0] = mean;
    double run = 0.0;
    for (int j = 1; j < b; ++j) {
      run += P[j - 1] - mean;
      Cc[j] = sg * h * run;
    }
  }
}

// ---------------------------------------------------------------------------
// Basis tiles.  For a slot of block K = (I, J):
//   theta_m (corner m): Hat_m + sum over the two sides E of K at m of
//       c_{E,m} (psi_m(E) + sum_j fcoef_E[j] psi_dj(E)),  c = +-1/H the
//       coarse curl of the nodal delta at m;
//   z_{E,k}: sum_j zcoef_E[k-1][j] psi_dj(E).
// rt_only: theta_m = Hat_m (coarse RT0 space).
// A face's functions are the first jeff[face] functions of its sides (b
// snapshot functions, or the predicted ones of the learned space); fcoef and
// zcoef are combinations of them.
template <typename TS>
__global__ void k_build_tiles(const Slot* __restrict__ slots, const double* __restrict__ psiS,
                              const double* __restrict__ fcoef, const double* __restrict__ zcoef,
                              const int* __restrict__ jeff, double* __restrict__ closed, TS* __restrict__ owned,
                              int rt_only, int n, int b) {
  const int nc = n / b, nb1 = b + 1, ncl = nb1 * nb1;
  const Slot sl = slots[blockIdx.x];
  const int I = sl.block % nc, J = sl.block / nc;
  const double H = (double)b / n;
  for (int t = threadIdx.x; t < ncl; t += blockDim.x) {
    const int a = t % nb1, c = t / nb1;
    const double x = (double)a / b, y = (double)c / b;
    double v = 0.0;
    if (sl.kind == 0) {
      int sA, sB;
      double cA, cB;
      switch (sl.which) {
        case 0: v = (1 - x) * (1 - y); sA = 0; cA = -1.0; sB = 2; cB = +1.0; break;   // BL
        case 1: v = x * (1 - y);       sA = 1; cA = -1.0; sB = 2; cB = -1.0; break;   // BR
        case 2: v = (1 - x) * y;       sA = 0; cA = +1.0; sB = 3; cB = +1.0; break;   // TL
        default: v = x * y;            sA = 1; cA = +1.0; sB = 3; cB = -1.0; break;   // TR
      }
      if (!rt_only) {
        const int sides[2] = {sA, sB};
        const double cs[2] = {cA / H, cB / H};
        for (int e = 0; e < 2; ++e) {
          const int face = face_of_side(sides[e], I, J, nc);
          const double* P = psiS + ((long long)sl.block * 4 + sides[e]) * b * ncl;
          const double* fc = fcoef + (long long)face * b;
          const int nf = jeff ? jeff[face] : b;
          double xi = 0.0;
          for (int jj = 0; jj < nf; ++jj) xi += fc[jj] * P[(long long)jj * ncl + t];
          v += cs[e] * xi;
        }
      }
    } else {
      const double* P = psiS + ((long long)sl.block * 4 + sl.which) * b * ncl;
      const double* zc = zcoef + ((long long)sl.face * (b - 1) + (sl.k - 1)) * b;
      const int nf = jeff ? jeff[sl.face] : b;
      for (int jj = 0; jj < nf; ++jj) v += zc[jj] * P[(long long)jj * ncl + t];
    }
    // the Galerkin matrix is assembled from the rounded values, so that the
    // coarse step is the exact K-orthogonal projection onto the span that the
    // restriction and prolongation actually use
    const TS vr = from_d<TS>(v);
    closed[(long long)blockIdx.x * ncl + t] = (double)to_f(vr);
    if (a < b && c < b) owned[(long long)blockIdx.x * b * b + c * b + a] = vr;
  }
}

// Energies a(phi_sa, phi_sb) restricted to block blk for every pair of the
// block's slots (closed (b+1)^2 node tiles, stream-function form: per cell
// the four face fluxes of each function, weighted by kinv, with the exact
// RT0 cell mass: same-face products / 3 + opposite-face products / 6).
// One warp per pair, lanes over the cells (fixed shuffle order: the result
// is the same on every call); pairs spread over gridDim.y CTAs per block;
// blocks with bmask[blk] == 0 are skipped.
__global__ void __launch_bounds__(256) k_pair_energy(const int* __restrict__ slot_ptr, const double* __restrict__ closed,
                              const double* __restrict__ kinv, const long long* __restrict__ pair_ptr,
                              const unsigned char* __restrict__ bmask, double* __restrict__ pairE, int n, int b) {
  const int nc = n / b, blk = blockIdx.x, I = blk % nc, J = blk / nc;
  if (bmask && !bmask[blk]) return;
  const int s0 = slot_ptr[blk], m = slot_ptr[blk + 1] - s0;
  const int nb1 = b + 1, ncl = nb1 * nb1;
  double* E = pairE + pair_ptr[blk];
  const int npair = m * (m + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = blockIdx.y * nw + warp; t < npair; t += gridDim.y * nw) {
    int sa = 0, rem = t;
    while (rem >= m - sa) { rem -= m - sa; ++sa; }
    const int sb = sa + rem;
    const double* Pa = closed + (long long)(s0 + sa) * ncl;
    const double* Pb = closed + (long long)(s0 + sb) * ncl;
    double e = 0.0;
    for (int cell = lane; cell < b * b; cell += 32) {
      const int a = cell % b, c = cell / b;
      const int n00 = c * nb1 + a, n10 = n00 + 1, n01 = n00 + nb1, n11 = n01 + 1;
      const double aL = Pa[n01] - Pa[n00], aR = Pa[n11] - Pa[n10];
      const double aB = Pa[n00] - Pa[n10], aT = Pa[n01] - Pa[n11];
      const double bL = Pb[n01] - Pb[n00], bR = Pb[n11] - Pb[n10];
      const double bB = Pb[n00] - Pb[n10], bT = Pb[n01] - Pb[n11];
      const double k = kinv[(long long)(J * b + c) * n + I * b + a];
      // (same-face products) / 3 + (opposite-face products) / 6, times 6
      e += k * (2.0 * (aL * bL + aR * bR + aB * bB + aT * bT) + (aL * bR + aR * bL + aB * bT + aT * bB));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) {
      e /= 6.0;
      E[sa * m + sb] = e;
      E[sb * m + sa] = e;
    }
  }
}

// K[u][*] += pair energies of u's slots (one thread per row: deterministic);
// blocks with bmask[blk] == 0 contribute nothing
__global__ void k_assemble_coarse(const int* __restrict__ slot_ptr, const Slot* __restrict__ slots,
                                  const int* __restrict__ gather, const long long* __restrict__ pair_ptr,
                                  const double* __restrict__ pairE, const unsigned char* __restrict__ bmask,
                                  double* __restrict__ K, int D) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= D) return;
  double* row = K + (long long)u * D;
  for (int g = 0; g < 4; ++g) {
    const int s = gather[4 * u + g];
    if (s < 0) continue;
    const int blk = slots[s].block, s0 = slot_ptr[blk], m = slot_ptr[blk + 1] - s0;
    if (bmask && !bmask[blk]) continue;
    const double* E = pairE + pair_ptr[blk] + (long long)(s - s0) * m;
    for (int t = 0; t < m; ++t) row[slots[s0 + t].coef] += E[t];
  }
}

// one Gauss-Jordan elimination step on an SPD matrix: B = GJ_k(A)
__global__ void k_gj_step(const double* __restrict__ A, double* __restrict__ B, int D, int k,
                          int* status) {
  const long long m = (long long)D * D;
  __shared__ double ipk;   // the pivot's reciprocal, once per CTA
  if (threadIdx.x == 0) {
    const double p = A[(long long)k * D + k];
    if (!(p > 0.0) && blockIdx.x == 0) atomicOr(status, kStNotSpd);
    ipk = 1.0 / p;
  }
  __syncthreads();
  const double ip = ipk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / D), j = (int)(t % D);
    double v;
    if (i == k && j == k) v = ip;
    else if (i == k) v = A[t] * ip;
    else if (j == k) v = -A[t] * ip;
    else v = A[t] - A[(long long)i * D + k] * A[(long long)k * D + j] * ip;
    B[t] = v;
  }
}

// ---- low-rank update of a Galerkin inverse ---------------------------------
// The Galerkin matrix is linear in 1/kappa, so a change delta of 1/kappa
// changes it by Delta = Galerkin(delta), nonzero only in the rows and columns
// S of basis functions whose support meets a changed cell.  With B the old
// inverse, X = B[:, S], P = B[S, S]^{-1} (the Schur complement of the old
// matrix on S) and P + Delta[S, S] the new one, the new inverse is
// B + X M X^T, M = -P (P + Delta[S, S])^{-1} Delta[S, S] (symmetric).

// delta = 1/kappa_new - kinv_old, 1/kappa_new computed as k_kinv computes it
__global__ void k_kinv_delta(const double* __restrict__ kappa, const double* __restrict__ kinv_old,
                             double* __restrict__ delta, long long nn) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nn;
       t += (long long)gridDim.x * blockDim.x) {
    const double k = kappa[t];
    const double v = (k > 0.0 && isfinite(k)) ? 1.0 / k : 1.0;
    delta[t] = v - kinv_old[t];
  }
}

// flag[i] = 1 if row i of the D x D matrix K has a nonzero (one warp per row)
__global__ void k_row_nonzero(const double* __restrict__ K, int D, unsigned char* __restrict__ flag) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= D) return;
  const double* r = K + (long long)warp * D;
  int nz = 0;
  for (int j = lane; j < D; j += 32) nz |= (r[j] != 0.0);
  nz = __any_sync(0xffffffffu, nz);
  if (lane == 0) flag[warp] = (unsigned char)nz;
}

// out[i * s + a] = K[row(i) * D + S[a]], row(i) = i (rows_all) or S[i]
__global__ void k_gather_cols(const double* __restrict__ K, int D, const int* __restrict__ S, int s, int rows,
                              int rows_all, double* __restrict__ out) {
  const long long tot = (long long)rows * s;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / s), a = (int)(t % s);
    const int r = rows_all ? i : S[i];
    out[t] = K[(long long)r * D + S[a]];
  }
}

// in-place Gauss-Jordan inverse of an SPD s x s matrix by one CTA (the pivot
// row and column are staged in shared memory before each elimination step)
__global__ void k_gj_small(double* __restrict__ A, int s, int* __restrict__ bad) {
  extern __shared__ double st[];   // 2 s
  __shared__ double ipk;
  double* rows = st;
  double* colk = st + s;
  const int tot = s * s;
  for (int k = 0; k < s; ++k) {
    if (threadIdx.x == 0) {   // the reciprocal once per step
      double p = A[(long long)k * s + k];
      if (!(p > 0.0) || !isfinite(p)) {
        *bad = 1;
        p = 1.0;
      }
      ipk = 1.0 / p;
    }
    __syncthreads();
    const double ip = ipk;
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
      rows[j] = A[(long long)k * s + j] * ip;
      colk[j] = A[(long long)j * s + k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = t / s, j = t % s;
      double v;
      if (i == k && j == k) v = ip;
      else if (i == k) v = rows[j];
      else if (j == k) v = -colk[i] * ip;
      else v = fma(-colk[i], rows[j], A[t]);
      A[t] = v;
    }
    __syncthreads();
  }
}

// C = alpha op(A) op(B) + beta C, FP64, C m x n row-major with leading
// dimension ldc; op(A)(i, k) = A[i * ars + k * acs], op(B)(k, j) = B[k * brs + j * bcs].
// 64 x 64 tiles of C per CTA, 16-deep slices of k staged in shared memory,
// each of the 256 threads accumulating a 4 x 4 sub-tile
__global__ void __launch_bounds__(256) k_dgemm(int m, int n, int kdim, double alpha, const double* __restrict__ A,
                                               long long ars, long long acs, const double* __restrict__ B,
                                               long long brs, long long bcs, double beta, double* __restrict__ C,
                                               long long ldc) {
  __shared__ double sa[16][64 + 1];
  __shared__ double sb[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < kdim; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      const int r = t / 16, kk = t % 16;       // A tile element (row r, depth kk)
      const int gi = i0 + r, gk = k0 + kk;
      sa[kk][r] = (gi < m && gk < kdim) ? A[gi * ars + gk * acs] : 0.0;
      const int c = t % 64, kb = t / 64;       // B tile element (depth kb, column c)
      const int gj = j0 + c, gkb = k0 + kb;
      sb[kb][c] = (gj < n && gkb < kdim) ? B[gkb * brs + gj * bcs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = sa[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sb[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * c;
      if (gi < m && gj < n) {
        double* cp = C + gi * ldc + gj;
        *cp = alpha * acc[r][c] + (beta != 0.0 ? beta * *cp : 0.0);
      }
    }
}

// in-place Gauss-Jordan inverse of the kb x kb SPD diagonal block at A
// (leading dimension lda) by one CTA; a non-positive pivot raises status
// (the pivot's reciprocal is formed once per step and the pivot row scaled
// by it, so each entry costs one FMA: FP64 throughput bounds this kernel)
__global__ void k_gj_block(double* __restrict__ A, long long lda, int kb, int* status) {
  __shared__ double rows[kGjBlock], colk[kGjBlock], ipk;
  const int tot = kb * kb;
  for (int k = 0; k < kb; ++k) {
    if (threadIdx.x == 0) {
      double p = A[(long long)k * lda + k];
      if (!(p > 0.0) || !isfinite(p)) {
        atomicOr(status, kStNotSpd);
        p = 1.0;
      }
      ipk = 1.0 / p;
    }
    __syncthreads();
    const double ip = ipk;
    for (int j = threadIdx.x; j < kb; j += blockDim.x) {
      rows[j] = A[(long long)k * lda + j] * ip;   // pivot row / p
      colk[j] = A[(long long)j * lda + k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = t / kb, j = t % kb;
      double* a = A + (long long)i * lda + j;
      if (i == k && j == k) *a = ip;
      else if (i == k) *a = rows[j];
      else if (j == k) *a = -colk[i] * ip;
      else *a = fma(-colk[i], rows[j], *a);
    }
    __syncthreads();
  }
}

// dst (rows x cols, leading dimension ldd) = src (leading dimension lds)
__global__ void k_copy2d(double* __restrict__ dst, long long ldd, const double* __restrict__ src, long long lds,
                         int rows, int cols) {
  const long long tot = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / cols), j = (int)(t % cols);
    dst[(long long)i * ldd + j] = src[(long long)i * lds + j];
  }
}

// B (D x D) += T X^T for a small rank m (T, X: D x m row-major), one thread
// per entry: the rank-|S| correction of a coarse inverse when |S| is small
__global__ void k_rank_update(double* __restrict__ B, int D, const double* __restrict__ T,
                              const double* __restrict__ X, int m) {
  const long long tot = (long long)D * D;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / D), j = (int)(t % D);
    double acc = B[t];
    for (int a = 0; a < m; ++a) acc = fma(T[(long long)i * m + a], X[(long long)j * m + a], acc);
    B[t] = acc;
  }
}

// A (s x s) = (A + A^T) / 2, one thread per pair i < j
__global__ void k_symmetrize(double* __restrict__ A, int s) {
  const long long tot = (long long)s * s;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / s), j = (int)(t % s);
    if (i < j) {
      const double v = 0.5 * (A[t] + A[(long long)j * s + i]);
      A[t] = v;
      A[(long long)j * s + i] = v;
    }
  }
}

// y += x elementwise
__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, long long cnt) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt;
       t += (long long)gridDim.x * blockDim.x)
    y[t] += x[t];
}

}  // namespace

// ---- launchers ---------------------------------------------------------------
void launch_kinv(const double* kappa, double* kinv, float* kinv32, int* status, int n, cudaStream_t s) {
  long long nn = (long long)n * n;
  int g = (int)((nn + 255) / 256);
  if (g > 4096) g = 4096;
  k_kinv<<<g, 256, 0, s>>>(kappa, kinv, kinv32, status, n);
}
void launch_assemble_band(const double* kinv, const int4* rects, double* band, int nmat, int wmax, int nmax,
                          int n, cudaStream_t s, const int* slot) {
  if (nmat == 0) return;
  k_assemble_band<<<nmat, 128, 0, s>>>(kinv, rects, slot, band, wmax, nmax, n);
}
void launch_band_cholesky(double* band, const int4* rects, int nmat, int wmax, int nmax, int* status,
                          cudaStream_t s, const int* slot) {
  if (nmat == 0) return;
  const size_t shm = sizeof(double) * (size_t)nmax * (wmax + 1);
  // one thread per pair (d1, d2) of the band: w (w + 1) / 2 <= blockDim
  const int threads = std::max(32, ((wmax * (wmax + 1) / 2 + 31) / 32) * 32);
  cudaFuncSetAttribute(k_band_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  k_band_cholesky<<<nmat, threads, shm, s>>>(band, rects, slot, wmax, nmax, status);
}
static int sm_count_setup() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return sms;
}

// CTAs per matrix so that `count` matrices fill about two waves of the SMs
// (at most one per 32 columns or rows of a matrix of side nmax)
static int split_for(int count, int nmax, int granule) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  const int want = (2 * sms + count - 1) / count;
  return std::max(1, std::min(want, (nmax + granule - 1) / granule));
}

void launch_band_inverse(const double* band, const int4* rects, int first, int count, int wmax, int nmax,
                         double* scratch, cudaStream_t s, const int* slot) {
  if (count == 0) return;
  if (count * ((nmax + 31) / 32) < sm_count_setup()) {
    // few matrices: a warp per column, 4 columns per CTA (measured against
    // 8 and 16 lanes per column: one-cell update 1.50 against 1.72 and 1.61 ms)
    constexpr int G = 32, kThr = 128;
    const int C = kThr / G, split = (nmax + C - 1) / C;
    const size_t shm = sizeof(double) * ((size_t)nmax * (wmax + 1) + nmax + (size_t)C * (wmax + 1));
    cudaFuncSetAttribute(k_band_inverse_grp<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_band_inverse_grp<G><<<dim3(count, split), kThr, shm, s>>>(band, rects, slot, first, wmax, nmax, scratch);
    return;
  }
  // one thread per column, the columns of a matrix split over `split` CTAs,
  // as far as the ring fits beside the band
  const int split = split_for(count, nmax, 32);
  const size_t band_b = sizeof(double) * ((size_t)nmax * (wmax + 1) + nmax);
  int threads = std::min(1024, (((nmax + split - 1) / split + 31) / 32) * 32);
  while (threads > 32 && band_b + sizeof(double) * (size_t)threads * (wmax + 1) > (size_t)kMaxDynSmem) threads -= 32;
  const size_t shm = band_b + sizeof(double) * (size_t)threads * (wmax + 1);
  cudaFuncSetAttribute(k_band_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  k_band_inverse<<<dim3(count, split), threads, shm, s>>>(band, rects, slot, first, wmax, nmax, scratch);
}
template <typename TB>
void launch_store_band(const double* band, const int4* rects, const int* ids, int count, int wmax, int nmax,
                       long long stride, TB* out, cudaStream_t s) {
  if (count == 0) return;
  k_store_band<TB><<<count, 256, 0, s>>>(band, rects, ids, wmax, nmax, stride, out);
}
template void launch_store_band<double>(const double*, const int4*, const int*, int, int, int, long long, double*,
                                        cudaStream_t);
template void launch_store_band<float>(const double*, const int4*, const int*, int, int, int, long long, float*,
                                       cudaStream_t);
void launch_rect_changed(const double* kappa, const double* kinv_old, const int4* rects, int nrect, int n,
                         unsigned char* flag, cudaStream_t s) {
  if (nrect == 0) return;
  k_rect_changed<<<nrect, 256, 0, s>>>(kappa, kinv_old, rects, n, flag);
}
template <typename TS>
void launch_store_inverse(const double* scratch, const PatchGeo* geo, int first, int count, int nmax,
                          TS* pinv, cudaStream_t s) {
  if (count == 0) return;
  k_store_inverse<TS><<<dim3(count, split_for(count, nmax, 8)), 256, 0, s>>>(scratch, geo, first, nmax, pinv);
}
template void launch_store_inverse<double>(const double*, const PatchGeo*, int, int, int, double*,
                                           cudaStream_t);
template void launch_store_inverse<float>(const double*, const PatchGeo*, int, int, int, float*,
                                          cudaStream_t);
template void launch_store_inverse<__nv_bfloat16>(const double*, const PatchGeo*, int, int, int,
                                                  __nv_bfloat16*, cudaStream_t);

void launch_store_inverse_f16(const double* scratch, const PatchGeo* geo, const int* gofs, int first, int count,
                              int nmax, __half* pinv, float* rscale, cudaStream_t s, const int* pidx) {
  if (count == 0) return;
  k_store_inverse_f16<<<dim3(count, split_for(count, nmax, 8)), 256, 0, s>>>(scratch, geo, pidx, gofs, first, nmax,
                                                                             pinv, rscale);
}
template <typename TS>
void launch_store_inverse_tiles(const double* scratch, const PatchGeo* geo, const int* gofs, const int* pidx,
                                int first, int count, int nmax, TS* tiles, const float* rscale, cudaStream_t s) {
  if (count == 0) return;
  k_store_inverse_tiles<TS><<<dim3(count, split_for(count, nmax, 8)), 256, 0, s>>>(scratch, geo, gofs, pidx, first,
                                                                                   nmax, tiles, rscale);
}
template void launch_store_inverse_tiles<__nv_bfloat16>(const double*, const PatchGeo*, const int*, const int*, int,
                                                        int, int, __nv_bfloat16*, const float*, cudaStream_t);
template void launch_store_inverse_tiles<__half>(const double*, const PatchGeo*, const int*, const int*, int, int,
                                                 int, __half*, const float*, cudaStream_t);
void launch_snapshots(const double* kinv, const double* blk_band, const double* coef, int nfn,
                      const unsigned char* mask, double* psiS, double* gram, int n, int b, cudaStream_t s) {
  const int nc = n / b, nloc = (b - 1) * (b - 1), threads = 256;
  if (!coef) nfn = b;
  const size_t shm = sizeof(double) * ((size_t)nloc * (b + 1) + (size_t)nfn * (b + 1) * (b + 1) +
                                       (size_t)b * b + (size_t)nfn * b + (size_t)(threads / 32) * nloc +
                                       2 * (size_t)nfn * kGramChunk * 4);
  cudaFuncSetAttribute(k_snapshots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  k_snapshots<<<nc * nc * 4, threads, shm, s>>>(kinv, blk_band, coef, nfn, mask, psiS, gram, n, b);
}
void launch_face_spectral(const SpectralArgs& a, int nfaces, cudaStream_t s) {
  if (nfaces == 0) return;
  k_face_spectral<<<nfaces, 32, 0, s>>>(a);
}
void launch_pred_basis(const float* y, const double* kinv, int k, int n, int b, double thr, double* prof,
                       double* ccoef, int* jpred, int nfaces, cudaStream_t s) {
  if (nfaces == 0) return;
  k_pred_basis<<<(nfaces + 63) / 64, 64, 0, s>>>(y, kinv, k, n, b, thr, prof, ccoef, jpred, nfaces);
}
template <typename TS>
void launch_build_tiles(const CoarseSpace& cs, const double* psiS, const double* fcoef, const double* zcoef,
                        const int* jeff, int rt_only, int n, int b, cudaStream_t s) {
  if (cs.nslots == 0) return;
  k_build_tiles<TS><<<cs.nslots, 128, 0, s>>>(cs.slots, psiS, fcoef, zcoef, jeff, cs.closed, (TS*)cs.owned,
                                               rt_only, n, b);
}
template void launch_build_tiles<double>(const CoarseSpace&, const double*, const double*, const double*,
                                         const int*, int, int, int, cudaStream_t);
template void launch_build_tiles<float>(const CoarseSpace&, const double*, const double*, const double*,
                                        const int*, int, int, int, cudaStream_t);
template void launch_build_tiles<__nv_bfloat16>(const CoarseSpace&, const double*, const double*,
                                                const double*, const int*, int, int, int, cudaStream_t);

void launch_galerkin(const CoarseSpace& cs, const double* kinv, int nblocks, int n, int b, double* pairE,
                     const long long* pair_ptr, double* K, cudaStream_t s, const unsigned char* bmask) {
  if (cs.D == 0) return;
  // one warp per pair of slots: enough CTAs per block for its pairs
  const int mx = std::max(1, cs.max_slots_per_block), pairs = mx * (mx + 1) / 2;
  const int ysplit = std::max(1, std::min(64, (pairs + 7) / 8));
  k_pair_energy<<<dim3(nblocks, ysplit), 256, 0, s>>>(cs.slot_ptr, cs.closed, kinv, pair_ptr, bmask, pairE, n, b);
  cudaMemsetAsync(K, 0, sizeof(double) * (size_t)cs.D * cs.D, s);
  k_assemble_coarse<<<(cs.D + 127) / 128, 128, 0, s>>>(cs.slot_ptr, cs.slots, cs.gather, pair_ptr, pairE, bmask,
                                                        K, cs.D);
}
static int grid_of(long long cnt, int threads, int cap) {
  long long g = (cnt + threads - 1) / threads;
  return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

void launch_kinv_delta(const double* kappa, const double* kinv_old, double* delta, int n, cudaStream_t s) {
  const long long nn = (long long)n * n;
  k_kinv_delta<<<grid_of(nn, 256, 4096), 256, 0, s>>>(kappa, kinv_old, delta, nn);
}
void launch_row_nonzero(const double* K, int D, unsigned char* flag, cudaStream_t s) {
  if (D == 0) return;
  k_row_nonzero<<<(int)(((long long)D * 32 + 255) / 256), 256, 0, s>>>(K, D, flag);
}
void launch_gather_cols(const double* K, int D, const int* S, int s_cnt, int rows, bool rows_all, double* out,
                        cudaStream_t s) {
  if (rows == 0 || s_cnt == 0) return;
  k_gather_cols<<<grid_of((long long)rows * s_cnt, 256, 4096), 256, 0, s>>>(K, D, S, s_cnt, rows,
                                                                           rows_all ? 1 : 0, out);
}
void launch_gj_small(double* A, int s_cnt, int* bad, cudaStream_t s) {
  if (s_cnt == 0) return;
  k_gj_small<<<1, 1024, sizeof(double) * 2 * (size_t)s_cnt, s>>>(A, s_cnt, bad);
}
void launch_dgemm(int m, int n, int k, double alpha, const double* A, long long ars, long long acs,
                  const double* B, long long brs, long long bcs, double beta, double* C, long long ldc,
                  cudaStream_t s) {
  if (m == 0 || n == 0) return;
  k_dgemm<<<dim3((n + 63) / 64, (m + 63) / 64), 256, 0, s>>>(m, n, k, alpha, A, ars, acs, B, brs, bcs, beta, C, ldc);
}
void launch_rank_update(double* B, int D, const double* T, const double* X, int m, cudaStream_t s) {
  if (D == 0 || m == 0) return;
  k_rank_update<<<grid_of((long long)D * D, 256, 4096), 256, 0, s>>>(B, D, T, X, m);
}
void launch_symmetrize(double* A, int s_cnt, cudaStream_t s) {
  if (s_cnt == 0) return;
  k_symmetrize<<<grid_of((long long)s_cnt * s_cnt, 256, 1024), 256, 0, s>>>(A, s_cnt);
}
void launch_add(double* y, const double* x, long long cnt, cudaStream_t s) {
  if (cnt == 0) return;
  k_add<<<grid_of(cnt, 256, 4096), 256, 0, s>>>(y, x, cnt);
}
// Inverse of an SPD D x D matrix in place.  Small matrices: D pivot steps of
// k_gj_step (ping-pong with B).  Larger ones: Gauss-Jordan by blocks of kb =
// kGjBlock pivots, so that the bulk of the work is one rank-kb update of the
// whole matrix per block (a GEMM) instead of D passes over it.  With P the
// inverse of the pivot block, C = A[:, blk] and R = P A[blk, :] (taken before
// the update):  A -= C R;  A[:, blk] = -C P;  A[blk, :] = R;  A[blk, blk] = P,
// which is the scalar step of k_gj_step applied to kb pivots at once.  B holds
// P, C and R (kb (kb + 2 D) doubles <= D^2).
void launch_gauss_jordan(double* A, double* B, int D, int* status, cudaStream_t s) {
  const long long m = (long long)D * D;
  if (D < 3 * kGjBlock) {
    int g = (int)((m + 255) / 256);
    if (g > 2048) g = 2048;
    for (int k = 0; k < D; ++k) {
      if (k % 2 == 0) k_gj_step<<<g, 256, 0, s>>>(A, B, D, k, status);
      else k_gj_step<<<g, 256, 0, s>>>(B, A, D, k, status);
    }
    if (D % 2 == 1) cudaMemcpyAsync(A, B, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s);
    return;
  }
  double* P = B;
  double* C = B + (long long)kGjBlock * kGjBlock;
  double* R = C + (long long)D * kGjBlock;
  for (int k0 = 0; k0 < D; k0 += kGjBlock) {
    const int kb = std::min(kGjBlock, D - k0);
    double* Akk = A + (long long)k0 * D + k0;
    k_gj_block<<<1, 1024, 0, s>>>(Akk, D, kb, status);                                   // P in place
    k_copy2d<<<grid_of((long long)kb * kb, 256, 64), 256, 0, s>>>(P, kb, Akk, D, kb, kb);
    k_copy2d<<<grid_of((long long)D * kb, 256, 2048), 256, 0, s>>>(C, kb, A + k0, D, D, kb);   // C = A[:, blk]
    launch_dgemm(kb, D, kb, 1.0, P, kb, 1, A + (long long)k0 * D, D, 1, 0.0, R, D, s);    // R = P A[blk, :]
    launch_dgemm(D, D, kb, -1.0, C, kb, 1, R, D, 1, 1.0, A, D, s);                       // A -= C R
    launch_dgemm(D, kb, kb, -1.0, C, kb, 1, P, kb, 1, 0.0, A + k0, D, s);                // A[:, blk] = -C P
    k_copy2d<<<grid_of((long long)kb * D, 256, 2048), 256, 0, s>>>(A + (long long)k0 * D, D, R, D, kb, D);
    k_copy2d<<<grid_of((long long)kb * kb, 256, 64), 256, 0, s>>>(Akk, D, P, kb, kb, kb);
  }
}

}  // namespace tg
