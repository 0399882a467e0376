// Learned coarse basis: the network's face inputs, a three-layer perceptron
// evaluated and trained with bfloat16 tensor-core GEMMs (tcgen05.mma with TMA
// operand loads and TMEM accumulators, gemm_tc.cu; FP32 accumulation), its
// subspace loss and Adam, and the training-data entry point (labels from the
// exact spectral problems of Section 4.2).
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
  // K-major, 16-byte-strided GEMM operands (gathered, transposed or padded)
  __nv_bfloat16 *pa = nullptr, *pb = nullptr;
  long long pack_cap = 0;         // entries of pa and of pb
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

inline int pad8(int x) { return (x + 7) / 8 * 8; }

// entries each pack buffer needs for batches of up to `rows` samples
long long pack_need(const tg_mlp* net, int rows) {
  const long long M = std::max({rows, net->hidden, net->din, net->dout});
  const long long K = std::max({pad8(net->din), pad8(rows), pad8(net->hidden), pad8(net->dout)});
  return M * K;
}

int ensure_pack(tg_mlp* net, int rows) {
  const long long need = pack_need(net, rows);
  if (need <= net->pack_cap) return TG_OK;
  cudaFree(net->pa);
  cudaFree(net->pb);
  net->pa = net->pb = nullptr;
  net->pack_cap = 0;
  if (cudaMalloc(&net->pa, sizeof(__nv_bfloat16) * need) != cudaSuccess ||
      cudaMalloc(&net->pb, sizeof(__nv_bfloat16) * need) != cudaSuccess)
    return TG_ERR_OOM;
  net->pack_cap = need;
  return TG_OK;
}

// a row-major (rows x K, stride ld) operand as the GEMM takes it: in place when
// its base and stride meet the TMA rules, else copied (padded) into buf
TcOperand operand(const __nv_bfloat16* p, int rows, int K, int ld, __nv_bfloat16* buf, cudaStream_t s) {
  if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0 && ld % 8 == 0) return TcOperand{p, rows, K, ld};
  pack_kmajor(p, ld, 1, nullptr, nullptr, rows, K, pad8(K), buf, s);
  return TcOperand{buf, rows, K, pad8(K)};
}
// the transpose of a row-major (K x rows, stride ld) matrix, with its rows
// optionally gathered through kmap, as a K-major (rows x K) operand in buf
TcOperand transposed(const __nv_bfloat16* p, int rows, int K, int ld, const int* kmap, __nv_bfloat16* buf,
                     cudaStream_t s) {
  pack_kmajor(p, 1, ld, nullptr, kmap, rows, K, pad8(K), buf, s);
  return TcOperand{buf, rows, K, pad8(K)};
}

// forward pass over `batch` rows of x (gathered through rows when not NULL)
int forward_rows(tg_mlp* net, int batch, const __nv_bfloat16* x, const int* rows, float* y, __nv_bfloat16* h1,
                 __nv_bfloat16* h2, cudaStream_t s) {
  const int hid = net->hidden, din = net->din, dout = net->dout;
  const __nv_bfloat16 *W1 = net->wb + net->oW1, *W2 = net->wb + net->oW2, *W3 = net->wb + net->oW3;
  // H1 = relu(X W1^T + b1)
  pack_kmajor(x, din, 1, rows, nullptr, batch, din, pad8(din), net->pa, s);
  int rc = gemm_tc(TcOperand{net->pa, batch, din, pad8(din)}, operand(W1, hid, din, din, net->pb, s), batch, hid,
                   din, net->p + net->ob1, kEpiReluBf16, nullptr, h1, hid, nullptr, s);
  // H2 = relu(H1 W2^T + b2)
  if (!rc)
    rc = gemm_tc(operand(h1, batch, hid, hid, net->pa, s), operand(W2, hid, hid, hid, net->pb, s), batch, hid, hid,
                 net->p + net->ob2, kEpiReluBf16, nullptr, h2, hid, nullptr, s);
  // Y = H2 W3^T + b3
  if (!rc)
    rc = gemm_tc(operand(h2, batch, hid, hid, net->pa, s), operand(W3, dout, hid, hid, net->pb, s), batch, dout,
                 hid, net->p + net->ob3, kEpiF32, y, nullptr, dout, nullptr, s);
  return rc;
}

// loss and gradient (into net->g) of `batch` rows; loss added to net->lacc
int loss_backward(tg_mlp* net, int batch, const __nv_bfloat16* x, const float* q, const int* rows, cudaStream_t s) {
  const int hid = net->hidden, din = net->din, dout = net->dout;
  const __nv_bfloat16 *W2 = net->wb + net->oW2, *W3 = net->wb + net->oW3;
  int rc = forward_rows(net, batch, x, rows, net->y, net->h1, net->h2, s);
  if (rc) return rc;
  {
    const int warps = 4;
    const size_t shm = sizeof(float) * warps * (2 * net->b * net->k + net->b * net->b);
    k_subspace_loss<<<(batch + warps - 1) / warps, 32 * warps, shm, s>>>(net->y, q, rows, batch, net->b, net->k,
                                                                          net->lacc, net->dy);
    TG_COUNT(1);
  }
  // dW3 = dY^T H2 (contraction over the batch)
  rc = gemm_tc(transposed(net->dy, dout, batch, dout, nullptr, net->pa, s),
               transposed(net->h2, hid, batch, hid, nullptr, net->pb, s), dout, hid, batch, nullptr, kEpiF32,
               net->g + net->oW3, nullptr, hid, nullptr, s);
  k_colsum<<<(dout + 127) / 128, 128, 0, s>>>(net->dy, batch, dout, net->g + net->ob3);
  // dH2 = (dY W3) * [H2 > 0]
  if (!rc)
    rc = gemm_tc(operand(net->dy, batch, dout, dout, net->pa, s), transposed(W3, hid, dout, hid, nullptr, net->pb, s),
                 batch, hid, dout, nullptr, kEpiMaskBf16, nullptr, net->dh2, hid, net->h2, s);
  // dW2 = dH2^T H1
  if (!rc)
    rc = gemm_tc(transposed(net->dh2, hid, batch, hid, nullptr, net->pa, s),
                 transposed(net->h1, hid, batch, hid, nullptr, net->pb, s), hid, hid, batch, nullptr, kEpiF32,
                 net->g + net->oW2, nullptr, hid, nullptr, s);
  k_colsum<<<(hid + 127) / 128, 128, 0, s>>>(net->dh2, batch, hid, net->g + net->ob2);
  // dH1 = (dH2 W2) * [H1 > 0]
  if (!rc)
    rc = gemm_tc(operand(net->dh2, batch, hid, hid, net->pa, s), transposed(W2, hid, hid, hid, nullptr, net->pb, s),
                 batch, hid, hid, nullptr, kEpiMaskBf16, nullptr, net->dh1, hid, net->h1, s);
  // dW1 = dH1^T X (the batch's rows of x)
  if (!rc)
    rc = gemm_tc(transposed(net->dh1, hid, batch, hid, nullptr, net->pa, s),
                 transposed(x, din, batch, din, rows, net->pb, s), hid, din, batch, nullptr, kEpiF32,
                 net->g + net->oW1, nullptr, din, nullptr, s);
  k_colsum<<<(hid + 127) / 128, 128, 0, s>>>(net->dh1, batch, hid, net->g + net->ob1);
  TG_COUNT(3);
  return rc;
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

int mlp_forward(const tg_mlp* cnet, int batch, const __nv_bfloat16* x, float* y, __nv_bfloat16* h1,
                __nv_bfloat16* h2, cudaStream_t s) {
  tg_mlp* net = const_cast<tg_mlp*>(cnet);   // the parameters stay; only the pack scratch may grow
  int rc = ensure_pack(net, std::min(batch, kMaxBatch));
  for (int r0 = 0; r0 < batch && !rc; r0 += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, batch - r0);
    rc = forward_rows(net, cnt, x + (long long)r0 * net->din, nullptr, y + (long long)r0 * net->dout,
                      h1 + (long long)r0 * net->hidden, h2 + (long long)r0 * net->hidden, s);
  }
  return rc;
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
  cudaFree(net->y); cudaFree(net->lacc); cudaFree(net->pa); cudaFree(net->pb);
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
    if (!rc) rc = ensure_pack(net, cnt);
    if (!rc)
      rc = forward_rows(net, cnt, xb + (long long)r0 * net->din, nullptr, y + (long long)r0 * net->dout, net->h1,
                        net->h2, s);
    if (rc) return rc;
  }
  int rc = cuda_rc(cudaStreamSynchronize(s));
  if (!rc) rc = cuda_rc(cudaGetLastError());
  if (!rc && read_and_clear_gemm_timeout()) rc = TG_ERR_DEVICE_TIMEOUT;
  return rc;
}

int tg_mlp_loss_grad(tg_mlp* net, int batch, const uint16_t* x, const float* q, double* loss, float* grad) {
  if (!net || !x || !q || batch < 1 || batch > kMaxBatch) return TG_ERR_INVALID_ARG;
  int rc = ensure_capacity(net, batch);
  if (!rc) rc = ensure_pack(net, batch);
  if (rc) return rc;
  cudaStream_t s = net->stream;
  cudaMemsetAsync(net->lacc, 0, sizeof(double), s);
  if ((rc = loss_backward(net, batch, reinterpret_cast<const __nv_bfloat16*>(x), q, nullptr, s))) return rc;
  double h_loss = 0.0;
  if ((rc = cuda_rc(cudaMemcpyAsync(&h_loss, net->lacc, sizeof(double), cudaMemcpyDeviceToHost, s)))) return rc;
  if (grad && (rc = cuda_rc(cudaMemcpyAsync(grad, net->g, sizeof(float) * net->np, cudaMemcpyDeviceToDevice, s))))
    return rc;
  if ((rc = cuda_rc(cudaStreamSynchronize(s)))) return rc;
  if ((rc = cuda_rc(cudaGetLastError()))) return rc;
  if (read_and_clear_gemm_timeout()) return TG_ERR_DEVICE_TIMEOUT;
  if (loss) *loss = h_loss;
  return TG_OK;
}

int tg_mlp_train(tg_mlp* net, int nsamples, const uint16_t* x, const float* q, const int* order, int nsteps,
                 int batch, float lr, float* loss_hist) {
  if (!net || !x || !q || !order || nsamples < 1 || nsteps < 0 || batch < 1 || batch > kMaxBatch || !(lr > 0))
    return TG_ERR_INVALID_ARG;
  int rc = ensure_capacity(net, batch);
  if (!rc) rc = ensure_pack(net, batch);
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
    if ((rc = loss_backward(net, batch, xb, q, order + (long long)st * batch, s))) return rc;
    net->t += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, net->t)), c2 = 1.0 / (1.0 - std::pow(0.999, net->t));
    k_adam<<<agrid, 256, 0, s>>>(net->p, net->g, net->m, net->v, net->wb, net->np, lr, (float)c1, (float)c2);
    k_loss_out<<<1, 32, 0, s>>>(net->lacc, loss_hist ? loss_hist + st : nullptr);
    TG_COUNT(2);
  }
  rc = cuda_rc(cudaStreamSynchronize(s));
  if (!rc) rc = cuda_rc(cudaGetLastError());
  if (!rc && read_and_clear_gemm_timeout()) rc = TG_ERR_DEVICE_TIMEOUT;
  return rc;
}

}  // extern "C"
