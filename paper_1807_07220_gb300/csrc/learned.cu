// Learned coarse basis: the network's face inputs, a three-layer perceptron
// evaluated and trained with bfloat16 tensor-core GEMMs (mma.sync m16n8k16,
// FP32 accumulation), its subspace loss and Adam, and the training-data entry
// point (labels from the exact spectral problems of Section 4.2).
//
// Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3.  Master parameters are
// FP32 (one vector: W1 | b1 | W2 | b2 | W3 | b3, weights row-major out x in);
// the GEMMs read bfloat16 copies of the weights and bfloat16 activations.
// Rounding points (the oracle's emulation rounds at the same places): the
// weight copies, the two hidden activations, dL/dy and the two hidden
// gradients are bfloat16; y, the weight gradients and the bias gradients
// are FP32.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/tgms.h"
#include "common.cuh"

struct tg_mlp {
  int b = 0, k = 0, hidden = 0, din = 0, dout = 0;
  long long np = 0;
  long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* wb = nullptr;    // bfloat16 copy of p
  int t = 0;                      // Adam steps taken
  cudaStream_t stream = nullptr;
  // activations and gradients for up to cap samples
  int cap = 0;
  __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *dy = nullptr, *dh1 = nullptr, *dh2 = nullptr;
  float* y = nullptr;
  double* lacc = nullptr;         // loss accumulator
};

namespace tg {
namespace {

constexpr int kMaxBatch = 4096;

// ---------------------------------------------------------------------------
// Face inputs: log10(kappa)/3 on omega_i plus a one-cell halo (clamped at the
// domain boundary), rows along the coarse edge E_i, columns across it (K^1
// first); a horizontal edge is transposed onto the vertical layout.
__global__ void k_face_inputs(const double* __restrict__ kappa, int n, int b, __nv_bfloat16* __restrict__ x) {
  const int nc = n / b, nV = nc * (nc - 1);
  const int f = blockIdx.x;
  int kind, I, J;
  if (f < nV) { kind = 0; I = f % (nc - 1) + 1; J = f / (nc - 1); }
  else { kind = 1; I = (f - nV) % nc; J = (f - nV) / nc + 1; }
  const int R = b + 2, C = 2 * b + 2;
  const int along0 = (kind == 0 ? J * b : I * b) - 1;
  const int across0 = (kind == 0 ? (I - 1) * b : (J - 1) * b) - 1;
  for (int t = threadIdx.x; t < R * C; t += blockDim.x) {
    const int r = t / C, c = t % C;
    const int al = min(max(along0 + r, 0), n - 1), ac = min(max(across0 + c, 0), n - 1);
    const double kv = (kind == 0) ? kappa[(long long)al * n + ac] : kappa[(long long)ac * n + al];
    x[(long long)f * R * C + t] = __float2bfloat16_rn((float)(log10(kv) / 3.0));
  }
}

// ---------------------------------------------------------------------------
// C (M x N) = A (M x K) B (K x N) on bfloat16 tensor cores, FP32 accumulation.
// A(m, k) = A[row(m) * sam + k * sak], B(k, n) = B[krow(k) * sbk + n * sbn]
// (row / krow: optional gathers); out(m, n) at m * som + n.
enum : int { kEpiF32 = 0, kEpiReluBf16 = 1, kEpiMaskBf16 = 2 };

struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  long long sam, sak;
  const int* arow;
  const __nv_bfloat16* B;
  long long sbk, sbn;
  const int* brow;
  const float* bias;           // [N] or NULL
  int epi;
  float* outf;                 // kEpiF32
  __nv_bfloat16* outh;         // kEpiReluBf16 / kEpiMaskBf16
  long long som;
  const __nv_bfloat16* mask;   // kEpiMaskBf16: out *= (mask(m, n) > 0), same layout as out
};

constexpr int kBM = 64, kBN = 64, kBK = 32, kLds = kBK + 8;

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 64 x 64 tile per CTA, four warps of 32 x 32, K in steps of 32 staged in
// shared memory (A row-major, B column-major: k contiguous for both).
__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[kBM][kLds];
  __shared__ __align__(16) __nv_bfloat16 Bs[kBN][kLds];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  for (int k0 = 0; k0 < g.K; k0 += kBK) {
#pragma unroll 4
    for (int i = 0; i < (kBM * kBK) / 128; ++i) {
      const int e = tid + i * 128;
      int r, kk;
      if (g.sak == 1) { r = e / kBK; kk = e % kBK; }
      else { r = e % kBM; kk = e / kBM; }
      const int gm = m0 + r, gk = k0 + kk;
      __nv_bfloat16 v = zero;
      if (gm < g.M && gk < g.K) {
        const long long row = g.arow ? (long long)g.arow[gm] : (long long)gm;
        v = g.A[row * g.sam + (long long)gk * g.sak];
      }
      As[r][kk] = v;
    }
#pragma unroll 4
    for (int i = 0; i < (kBN * kBK) / 128; ++i) {
      const int e = tid + i * 128;
      int nn, kk;
      if (g.sbk == 1) { nn = e / kBK; kk = e % kBK; }
      else { nn = e % kBN; kk = e / kBN; }
      const int gn = n0 + nn, gk = k0 + kk;
      __nv_bfloat16 v = zero;
      if (gn < g.N && gk < g.K) {
        const long long krow = g.brow ? (long long)g.brow[gk] : (long long)gk;
        v = g.B[krow * g.sbk + (long long)gn * g.sbn];
      }
      Bs[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kBK; ks += 16) {
      const int kq = ks + (lane & 3) * 2;
      uint32_t a[2][4], bq[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = wm * 32 + mt * 16 + (lane >> 2);
        a[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r0][kq]);
        a[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kq]);
        a[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r0][kq + 8]);
        a[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kq + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn * 32 + nt * 8 + (lane >> 2);
        bq[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kq]);
        bq[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kq + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], bq[nt]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + wm * 32 + mt * 16 + (lane >> 2) + (q >> 1) * 8;
        const int c = n0 + wn * 32 + nt * 8 + (lane & 3) * 2 + (q & 1);
        if (r >= g.M || c >= g.N) continue;
        float v = acc[mt][nt][q];
        if (g.bias) v += g.bias[c];
        const long long o = (long long)r * g.som + c;
        if (g.epi == kEpiF32) {
          g.outf[o] = v;
        } else if (g.epi == kEpiReluBf16) {
          g.outh[o] = __float2bfloat16_rn(fmaxf(v, 0.0f));
        } else {
          g.outh[o] = __float2bfloat16_rn(__bfloat162float(g.mask[o]) > 0.0f ? v : 0.0f);
        }
      }
}

// Subspace loss, one warp per sample: E = G G^T - Q Q^T (b x b, G the b x k
// predicted profiles, Q the label); loss += ||E||_F^2 / batch;
// dL/dy = (4 / batch) E G, rounded to bfloat16.
__global__ void k_subspace_loss(const float* __restrict__ Y, const float* __restrict__ Q,
                                const int* __restrict__ rows, int batch, int b, int k, double* __restrict__ loss,
                                __nv_bfloat16* __restrict__ dY) {
  extern __shared__ float smf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int s = blockIdx.x * nw + warp;
  const int bk = b * k;
  float* G = smf + warp * (2 * bk + b * b);
  float* Qs = G + bk;
  float* E = Qs + bk;
  float part = 0.0f;
  if (s < batch) {
    const long long qrow = rows ? (long long)rows[s] : (long long)s;
    for (int t = lane; t < bk; t += 32) {
      G[t] = Y[(long long)s * bk + t];
      Qs[t] = Q[qrow * bk + t];
    }
    __syncwarp();
    for (int t = lane; t < b * b; t += 32) {
      const int l = t / b, mm = t % b;
      float e = 0.0f;
      for (int j = 0; j < k; ++j) e += G[j * b + l] * G[j * b + mm] - Qs[j * b + l] * Qs[j * b + mm];
      E[t] = e;
      part += e * e;
    }
    __syncwarp();
    const float sc = 4.0f / (float)batch;
    for (int t = lane; t < bk; t += 32) {
      const int j = t / b, l = t % b;
      float d = 0.0f;
      for (int mm = 0; mm < b; ++mm) d += E[l * b + mm] * G[j * b + mm];
      dY[(long long)s * bk + t] = __float2bfloat16_rn(sc * d);
    }
  }
  part = warp_sum(part);
  if (lane == 0 && s < batch) atomicAdd(loss, (double)part / (double)batch);
}

// column sums of a bfloat16 matrix (bias gradients)
__global__ void k_colsum(const __nv_bfloat16* __restrict__ D, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float acc = 0.0f;
  for (int r = 0; r < rows; ++r) acc += __bfloat162float(D[(long long)r * cols + c]);
  out[c] = acc;
}

// Adam (Kingma & Ba 2015): c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, long long np, float lr, float c1,
                       float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    p[i] = pi;
    wb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb, long long np) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(p[i]);
}

// flags any index outside [0, limit)
__global__ void k_check_rows(const int* __restrict__ rows, long long count, int limit, int* __restrict__ bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = rows[i];
    if (r < 0 || r >= limit) atomicOr(bad, 1);
  }
}

__global__ void k_loss_out(double* __restrict__ acc, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (out) *out = (float)*acc;
    *acc = 0.0;
  }
}

void gemm(const GemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return;
  dim3 grid((a.N + kBN - 1) / kBN, (a.M + kBM - 1) / kBM);
  k_gemm_bf16<<<grid, 128, 0, s>>>(a);
  TG_COUNT(1);
}

GemmArgs gemm_args(int M, int N, int K) {
  GemmArgs a{};
  a.M = M; a.N = N; a.K = K;
  return a;
}

// forward pass over `batch` rows of x (gathered through rows when not NULL)
void forward_rows(const tg_mlp* net, int batch, const __nv_bfloat16* x, const int* rows, float* y,
                  __nv_bfloat16* h1, __nv_bfloat16* h2, cudaStream_t s) {
  GemmArgs a = gemm_args(batch, net->hidden, net->din);
  a.A = x; a.sam = net->din; a.sak = 1; a.arow = rows;
  a.B = net->wb + net->oW1; a.sbk = 1; a.sbn = net->din;
  a.bias = net->p + net->ob1; a.epi = kEpiReluBf16; a.outh = h1; a.som = net->hidden;
  gemm(a, s);
  a = gemm_args(batch, net->hidden, net->hidden);
  a.A = h1; a.sam = net->hidden; a.sak = 1;
  a.B = net->wb + net->oW2; a.sbk = 1; a.sbn = net->hidden;
  a.bias = net->p + net->ob2; a.epi = kEpiReluBf16; a.outh = h2; a.som = net->hidden;
  gemm(a, s);
  a = gemm_args(batch, net->dout, net->hidden);
  a.A = h2; a.sam = net->hidden; a.sak = 1;
  a.B = net->wb + net->oW3; a.sbk = 1; a.sbn = net->hidden;
  a.bias = net->p + net->ob3; a.epi = kEpiF32; a.outf = y; a.som = net->dout;
  gemm(a, s);
}

// loss and gradient (into net->g) of `batch` rows; loss added to net->lacc
void loss_backward(tg_mlp* net, int batch, const __nv_bfloat16* x, const float* q, const int* rows,
                   cudaStream_t s) {
  const int hid = net->hidden, din = net->din, dout = net->dout;
  forward_rows(net, batch, x, rows, net->y, net->h1, net->h2, s);
  {
    const int warps = 4;
    const size_t shm = sizeof(float) * warps * (2 * net->b * net->k + net->b * net->b);
    k_subspace_loss<<<(batch + warps - 1) / warps, 32 * warps, shm, s>>>(net->y, q, rows, batch, net->b, net->k,
                                                                          net->lacc, net->dy);
    TG_COUNT(1);
  }
  GemmArgs a = gemm_args(dout, hid, batch);           // dW3 = dY^T H2
  a.A = net->dy; a.sam = 1; a.sak = dout;
  a.B = net->h2; a.sbk = hid; a.sbn = 1;
  a.epi = kEpiF32; a.outf = net->g + net->oW3; a.som = hid;
  gemm(a, s);
  k_colsum<<<(dout + 127) / 128, 128, 0, s>>>(net->dy, batch, dout, net->g + net->ob3);
  a = gemm_args(batch, hid, dout);                    // dH2 = (dY W3) * [H2 > 0]
  a.A = net->dy; a.sam = dout; a.sak = 1;
  a.B = net->wb + net->oW3; a.sbk = hid; a.sbn = 1;
  a.epi = kEpiMaskBf16; a.outh = net->dh2; a.som = hid; a.mask = net->h2;
  gemm(a, s);
  a = gemm_args(hid, hid, batch);                     // dW2 = dH2^T H1
  a.A = net->dh2; a.sam = 1; a.sak = hid;
  a.B = net->h1; a.sbk = hid; a.sbn = 1;
  a.epi = kEpiF32; a.outf = net->g + net->oW2; a.som = hid;
  gemm(a, s);
  k_colsum<<<(hid + 127) / 128, 128, 0, s>>>(net->dh2, batch, hid, net->g + net->ob2);
  a = gemm_args(batch, hid, hid);                     // dH1 = (dH2 W2) * [H1 > 0]
  a.A = net->dh2; a.sam = hid; a.sak = 1;
  a.B = net->wb + net->oW2; a.sbk = hid; a.sbn = 1;
  a.epi = kEpiMaskBf16; a.outh = net->dh1; a.som = hid; a.mask = net->h1;
  gemm(a, s);
  a = gemm_args(hid, din, batch);                     // dW1 = dH1^T X
  a.A = net->dh1; a.sam = 1; a.sak = hid;
  a.B = x; a.sbk = din; a.sbn = 1; a.brow = rows;
  a.epi = kEpiF32; a.outf = net->g + net->oW1; a.som = din;
  gemm(a, s);
  k_colsum<<<(hid + 127) / 128, 128, 0, s>>>(net->dh1, batch, hid, net->g + net->ob1);
  TG_COUNT(3);
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return TG_OK;
  return (e == cudaErrorMemoryAllocation) ? TG_ERR_OOM : TG_ERR_CUDA;
}

int ensure_capacity(tg_mlp* net, int batch) {
  if (batch <= net->cap) return TG_OK;
  cudaFree(net->h1); cudaFree(net->h2); cudaFree(net->dy); cudaFree(net->dh1); cudaFree(net->dh2);
  cudaFree(net->y);
  net->h1 = net->h2 = net->dy = net->dh1 = net->dh2 = nullptr;
  net->y = nullptr;
  net->cap = 0;
  const size_t hb = sizeof(__nv_bfloat16) * (size_t)batch * net->hidden;
  const size_t ob = (size_t)batch * net->dout;
  int rc = TG_OK;
  if ((rc = cuda_rc(cudaMalloc(&net->h1, hb))) || (rc = cuda_rc(cudaMalloc(&net->h2, hb))) ||
      (rc = cuda_rc(cudaMalloc(&net->dh1, hb))) || (rc = cuda_rc(cudaMalloc(&net->dh2, hb))) ||
      (rc = cuda_rc(cudaMalloc(&net->dy, sizeof(__nv_bfloat16) * ob))) ||
      (rc = cuda_rc(cudaMalloc(&net->y, sizeof(float) * ob))))
    return rc;
  net->cap = batch;
  return TG_OK;
}

}  // namespace

void launch_face_inputs(const double* kappa, int n, int b, __nv_bfloat16* x, cudaStream_t s) {
  const int nc = n / b, nfaces = 2 * nc * (nc - 1);
  if (nfaces == 0) return;
  k_face_inputs<<<nfaces, 128, 0, s>>>(kappa, n, b, x);
  TG_COUNT(1);
}

void mlp_dims(const tg_mlp* net, int* b, int* k, int* hidden, int* din, int* dout) {
  *b = net->b; *k = net->k; *hidden = net->hidden; *din = net->din; *dout = net->dout;
}

void mlp_forward(const tg_mlp* net, int batch, const __nv_bfloat16* x, float* y, __nv_bfloat16* h1,
                 __nv_bfloat16* h2, cudaStream_t s) {
  forward_rows(net, batch, x, nullptr, y, h1, h2, s);
}

}  // namespace tg

using namespace tg;

extern "C" {

int tg_mlp_shape(int b, int k, int hidden, int* din, int* dout, long long* nparam) {
  if (b < 2 || b > kMaxB || k < 1 || k > 8 || hidden < 1 || hidden > 4096) return TG_ERR_INVALID_ARG;
  const int di = (b + 2) * (2 * b + 2), dd = k * b;
  if (din) *din = di;
  if (dout) *dout = dd;
  if (nparam) *nparam = (long long)hidden * di + hidden + (long long)hidden * hidden + hidden +
                        (long long)dd * hidden + dd;
  return TG_OK;
}

void tg_mlp_destroy(tg_mlp* net) {
  if (!net) return;
  cudaFree(net->p); cudaFree(net->g); cudaFree(net->m); cudaFree(net->v); cudaFree(net->wb);
  cudaFree(net->h1); cudaFree(net->h2); cudaFree(net->dy); cudaFree(net->dh1); cudaFree(net->dh2);
  cudaFree(net->y); cudaFree(net->lacc);
  delete net;
}

int tg_mlp_create(int b, int k, int hidden, const float* params, void* stream, tg_mlp** out) {
  if (!out || !params) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  int din = 0, dout = 0;
  long long np = 0;
  int rc = tg_mlp_shape(b, k, hidden, &din, &dout, &np);
  if (rc) return rc;
  tg_mlp* net = new tg_mlp();
  net->b = b; net->k = k; net->hidden = hidden; net->din = din; net->dout = dout; net->np = np;
  net->oW1 = 0;
  net->ob1 = net->oW1 + (long long)hidden * din;
  net->oW2 = net->ob1 + hidden;
  net->ob2 = net->oW2 + (long long)hidden * hidden;
  net->oW3 = net->ob2 + hidden;
  net->ob3 = net->oW3 + (long long)dout * hidden;
  net->stream = static_cast<cudaStream_t>(stream);
  cudaStream_t s = net->stream;
  if ((rc = cuda_rc(cudaMalloc(&net->p, sizeof(float) * np))) ||
      (rc = cuda_rc(cudaMalloc(&net->g, sizeof(float) * np))) ||
      (rc = cuda_rc(cudaMalloc(&net->m, sizeof(float) * np))) ||
      (rc = cuda_rc(cudaMalloc(&net->v, sizeof(float) * np))) ||
      (rc = cuda_rc(cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * np))) ||
      (rc = cuda_rc(cudaMalloc(&net->lacc, sizeof(double))))) {
    tg_mlp_destroy(net);
    return rc;
  }
  cudaMemcpyAsync(net->p, params, sizeof(float) * np, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(net->m, 0, sizeof(float) * np, s);
  cudaMemsetAsync(net->v, 0, sizeof(float) * np, s);
  cudaMemsetAsync(net->g, 0, sizeof(float) * np, s);
  cudaMemsetAsync(net->lacc, 0, sizeof(double), s);
  k_to_bf16<<<(int)std::min<long long>((np + 255) / 256, 4096), 256, 0, s>>>(net->p, net->wb, np);
  rc = cuda_rc(cudaStreamSynchronize(s));
  if (rc == TG_OK) rc = cuda_rc(cudaGetLastError());
  if (rc) {
    tg_mlp_destroy(net);
    return rc;
  }
  *out = net;
  return TG_OK;
}

int tg_mlp_params(const tg_mlp* net, float* params) {
  if (!net || !params) return TG_ERR_INVALID_ARG;
  int rc = cuda_rc(cudaMemcpyAsync(params, net->p, sizeof(float) * net->np, cudaMemcpyDeviceToDevice, net->stream));
  if (rc) return rc;
  return cuda_rc(cudaStreamSynchronize(net->stream));
}

int tg_mlp_forward(tg_mlp* net, int batch, const uint16_t* x, float* y) {
  if (!net || !x || !y || batch < 0) return TG_ERR_INVALID_ARG;
  cudaStream_t s = net->stream;
  const __nv_bfloat16* xb = reinterpret_cast<const __nv_bfloat16*>(x);
  for (int r0 = 0; r0 < batch; r0 += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, batch - r0);
    int rc = ensure_capacity(net, cnt);
    if (rc) return rc;
    forward_rows(net, cnt, xb + (long long)r0 * net->din, nullptr, y + (long long)r0 * net->dout, net->h1, net->h2,
                 s);
  }
  int rc = cuda_rc(cudaStreamSynchronize(s));
  return rc ? rc : cuda_rc(cudaGetLastError());
}

int tg_mlp_loss_grad(tg_mlp* net, int batch, const uint16_t* x, const float* q, double* loss, float* grad) {
  if (!net || !x || !q || batch < 1 || batch > kMaxBatch) return TG_ERR_INVALID_ARG;
  int rc = ensure_capacity(net, batch);
  if (rc) return rc;
  cudaStream_t s = net->stream;
  cudaMemsetAsync(net->lacc, 0, sizeof(double), s);
  loss_backward(net, batch, reinterpret_cast<const __nv_bfloat16*>(x), q, nullptr, s);
  double h_loss = 0.0;
  if ((rc = cuda_rc(cudaMemcpyAsync(&h_loss, net->lacc, sizeof(double), cudaMemcpyDeviceToHost, s)))) return rc;
  if (grad && (rc = cuda_rc(cudaMemcpyAsync(grad, net->g, sizeof(float) * net->np, cudaMemcpyDeviceToDevice, s))))
    return rc;
  if ((rc = cuda_rc(cudaStreamSynchronize(s)))) return rc;
  if ((rc = cuda_rc(cudaGetLastError()))) return rc;
  if (loss) *loss = h_loss;
  return TG_OK;
}

int tg_mlp_train(tg_mlp* net, int nsamples, const uint16_t* x, const float* q, const int* order, int nsteps,
                 int batch, float lr, float* loss_hist) {
  if (!net || !x || !q || !order || nsamples < 1 || nsteps < 0 || batch < 1 || batch > kMaxBatch || !(lr > 0))
    return TG_ERR_INVALID_ARG;
  int rc = ensure_capacity(net, batch);
  if (rc) return rc;
  cudaStream_t s = net->stream;
  const __nv_bfloat16* xb = reinterpret_cast<const __nv_bfloat16*>(x);
  {
    // every index must address a row of x and q before any kernel gathers through it
    int* bad = nullptr;
    int hbad = 0;
    if ((rc = cuda_rc(cudaMalloc(&bad, sizeof(int))))) return rc;
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    const long long cnt = (long long)nsteps * batch;
    if (cnt > 0)
      k_check_rows<<<(int)std::min<long long>((cnt + 255) / 256, 1024), 256, 0, s>>>(order, cnt, nsamples, bad);
    rc = cuda_rc(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s));
    cudaFree(bad);
    if (rc) return rc;
    if (hbad) return TG_ERR_INVALID_ARG;
  }
  cudaMemsetAsync(net->lacc, 0, sizeof(double), s);
  const int agrid = (int)std::min<long long>((net->np + 255) / 256, 2048);
  for (int st = 0; st < nsteps; ++st) {
    loss_backward(net, batch, xb, q, order + (long long)st * batch, s);
    net->t += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, net->t)), c2 = 1.0 / (1.0 - std::pow(0.999, net->t));
    k_adam<<<agrid, 256, 0, s>>>(net->p, net->g, net->m, net->v, net->wb, net->np, lr, (float)c1, (float)c2);
    k_loss_out<<<1, 32, 0, s>>>(net->lacc, loss_hist ? loss_hist + st : nullptr);
    TG_COUNT(2);
  }
  rc = cuda_rc(cudaStreamSynchronize(s));
  return rc ? rc : cuda_rc(cudaGetLastError());
}

}  // extern "C"
