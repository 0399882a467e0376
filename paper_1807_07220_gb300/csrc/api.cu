// C ABI of libtgms (declared in include/tgms.h): handle management, host-side
// index tables of the coarse space, and the orchestration of the setup
// (Step 2 of Section 5) and solve (Steps 1, 3, 4) kernels.
//
// A handle holds everything that depends on kappa only (setup) plus one
// solve context; a context holds the vectors, the PCG scalars and the coarse
// scratch of one right-hand side.  A solve is one CUDA graph: for each
// context a chain  prefix (preprocessing, PCG start) -> while node (two PCG
// iterations per pass) -> epilogue.  A batch puts the chains of many contexts
// (several handles, several right-hand sides each) into one graph, where they
// run concurrently.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/tgms.h"
#include "common.cuh"

using namespace tg;

namespace tg {
unsigned long long g_kernel_launches = 0;
bool g_pdl = false;
}

namespace {
struct Ctx;
}

struct tg_handle {
  int n = 0, b = 0, nc = 0, ov = 0, nblocks = 0, npatch = 0, nfaces = 0;
  double h = 0, H = 0, eig_tol = 0;
  tg_options opt{};
  cudaStream_t stream = nullptr;
  // permeability
  double* kinv = nullptr;
  float* kinv32 = nullptr;
  double* kcoef = nullptr;  // 5 n^2 node coefficients of the FP64 outer operator
  int* d_status = nullptr;
  // smoother
  PatchGeo* d_pgeo = nullptr;
  int* d_gofs = nullptr;    // first row group of each patch (+ total)
  int ngroups = 0;
  void* pinv = nullptr;
  void* pband = nullptr;    // band factors of the patches in the arithmetic type (tile shape kShapeBand)
  bool dense = true;        // the dense patch inverses (and tiles) are formed (dense_inverses_needed)
  void* ptiles = nullptr;   // 2-byte storage: the inverses in the tensor-core tile layout (kShapeTensor)
  int* d_tofs = nullptr;    // first 16-row tile of each patch (+ total)
  BandRef band;
  float* rscale = nullptr;  // FP16 storage: inverse row scales
  // block factors (snapshots) and dense block inverses (preprocessing)
  double* blk_band = nullptr;
  PatchGeo* d_bgeo = nullptr;
  int* d_bgofs = nullptr;
  int bgroups = 0;
  double* binv = nullptr;
  float* binv32 = nullptr;  // mixed precision: FP32 block inverses
  // spectral data
  double* lam = nullptr;
  std::vector<int> nsel;
  std::vector<double> lam_h;
  int velocity_basis = 0;
  int snapshot_solves = 0;   // local block solves of the coarse-space setup
  int fallback_faces = 0;    // learned space: faces that took the exact problem
  int refactored_patches = 0, refactored_blocks = 0;   // factored by the last setup or update
  int update_rank[2] = {-1, -1};   // last update: rows of the low-rank Galerkin-inverse update (cs, rt); -1 full
  bool regraph = false;      // a coarse space changed solver: the solve context (and its graph) is re-created
  int shape = 0;             // smoother tile shape (autotuned or from the options)
  float shape_us[kSmootherShapes] = {};   // autotuner: time per smoother launch of each shape (0: not tried)
  // coarse spaces: preconditioner and coarse RT0 (preprocessing)
  CoarseSpace cs, rt;
  int* h_flag = nullptr;    // pinned
  Ctx* ctx = nullptr;       // default solve context (tg_solve and the operator hooks)
  // grow-only device scratch of the setup steps, kept between permeability
  // updates (an update then allocates nothing); released after a setup
  void* scr[16] = {};
  size_t scr_cap[16] = {};
};

namespace {

// per right-hand-side solve state
struct Ctx {
  tg_handle* h = nullptr;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *rho = nullptr, *phi = nullptr;
  double *p2 = nullptr, *r2 = nullptr;   // ping-pong partners of p and r
  void *zacc = nullptr, *zacc2 = nullptr, *rin = nullptr;
  double *ux = nullptr, *uy = nullptr, *fd = nullptr, *bd = nullptr, *pd = nullptr, *pw = nullptr;
  double *part = nullptr, *gx = nullptr, *gy = nullptr, *FH = nullptr, *absF = nullptr, *diverr = nullptr;
  double *cs_part = nullptr, *cs_coefs = nullptr, *rt_part = nullptr, *rt_coefs = nullptr;
  PcgState* st = nullptr;
  double* d_rtol = nullptr;
  void* slab = nullptr;       // the device memory of every vector above (one allocation)
  double* h_rtol = nullptr;   // pinned
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // one-chain graphs of tg_solve (zero initial guess) and tg_solve_warm
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr, exec_warm = nullptr;
  unsigned long long k_prefix = 0, k_prefix_warm = 0, k_body = 0, k_epi = 0;
  bool warm = false;            // enqueue the warm-start prefix
  double* ux0 = nullptr;        // warm start: staged x-face velocities of the guess
  // profiling: events around smoother launches (profile == 1)
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0;
  std::vector<cudaEvent_t> prof_op_ev;   // and around the operator launches
  int prof_op_used = 0;
};

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return TG_OK;
  return (e == cudaErrorMemoryAllocation) ? TG_ERR_OOM : TG_ERR_CUDA;
}

#define TG_CK(call)                        \
  do {                                     \
    const int _rc = cuda_err((call));      \
    if (_rc != TG_OK) return _rc;          \
  } while (0)

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cuda_err(cudaMalloc((void**)p, sizeof(T) * count));
}

// scratch slots of the setup steps; a function uses only its own slots and
// those of no caller that is live across the call
enum Scr {
  kScrDelta,   // update: change of 1/kappa (n^2)
  kScrRect,    // rectangles of a compact list
  kScrFlag,    // per-rectangle or per-row flags
  kScrGeo,     // layouts of a compact list
  kScrIds,     // indices of a compact list
  kScrBand,    // band factors of patches
  kScrInv,     // dense local inverses of a batch
  kScrDense,   // D x D Galerkin matrix or its change
  kScrPPtr,    // pair-energy offsets per block
  kScrPairE,   // pair energies
  kScrX,       // low-rank update: B[:, S]
  kScrT,       // X M
  kScrSmall,   // four |S| x |S| matrices
  kScrBad,     // pivot flag
  kScrBlkMask, // update: blocks with a changed cell
  kScrCount
};

template <typename T>
int scratch(tg_handle* h, Scr slot, size_t count, T** out) {
  const size_t bytes = sizeof(T) * std::max<size_t>(1, count);
  if (h->scr_cap[slot] < bytes) {
    cudaFree(h->scr[slot]);
    h->scr[slot] = nullptr;
    h->scr_cap[slot] = 0;
    if (cudaMalloc(&h->scr[slot], bytes) != cudaSuccess) {
      cudaGetLastError();
      *out = nullptr;
      return TG_ERR_OOM;
    }
    h->scr_cap[slot] = bytes;
  }
  *out = static_cast<T*>(h->scr[slot]);
  return TG_OK;
}

void scratch_release(tg_handle* h) {
  for (int k = 0; k < kScrCount; ++k) {
    cudaFree(h->scr[k]);
    h->scr[k] = nullptr;
    h->scr_cap[k] = 0;
  }
}

void free_space(CoarseSpace& c) {
  cudaFree(c.slot_ptr);
  cudaFree(c.slots);
  cudaFree(c.gather);
  cudaFree(c.closed);
  cudaFree(c.owned);
  cudaFree(c.Kinv);
  cudaFree(c.Kdf);
  nd_free(c.nd);
  c = CoarseSpace{};
}

// bytes per stored patch-inverse entry and per coarse-tile entry
size_t ts_size(int precision) {
  return precision == TG_PREC_F64 ? 8 : precision == TG_PREC_F32 ? 4 : 2;
}
size_t tile_size(int precision) {
  return precision == TG_PREC_F64 ? 8 : 4;
}

int status_to_err(int st) {
  if (st & kStTimeout) return TG_ERR_DEVICE_TIMEOUT;
  if (st & kStBadKappa) return TG_ERR_INVALID_ARG;
  if (st & kStIncompatible) return TG_ERR_INCOMPATIBLE_SOURCE;
  if (st & kStNotSpd) return TG_ERR_BREAKDOWN;
  if (st & kStDegenerate) return TG_ERR_DEGENERATE_BASIS;
  if (st & kStBreakdown) return TG_ERR_BREAKDOWN;
  if (st & kStMaxIter) return TG_ERR_MAXITER;
  return TG_OK;
}

int read_status(tg_handle* h, int* out) {
  TG_CK(cudaMemcpyAsync(h->h_flag, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  TG_CK(cudaStreamSynchronize(h->stream));
  *out = *h->h_flag;
  return TG_OK;
}

// Host-side index tables of a coarse space in per-block slot form.
//   theta unknowns: interior coarse nodes (mI, mJ), 1 <= mI, mJ <= nc-1,
//     index (mJ-1)(nc-1) + (mI-1);
//   z unknowns: nsel[f]-1 per coarse face f, after all theta unknowns.
int build_space(tg_handle* h, CoarseSpace& c, const std::vector<int>& nsel, bool rt_only) {
  const int nc = h->nc, b = h->b;
  const int nV = nc * (nc - 1), nfaces = 2 * nc * (nc - 1);
  const int ntheta = (nc - 1) * (nc - 1);
  std::vector<int> zbase(nfaces + 1, ntheta);
  for (int f = 0; f < nfaces; ++f) zbase[f + 1] = zbase[f] + (rt_only ? 0 : std::max(0, nsel[f] - 1));
  c.D = zbase[nfaces];
  std::vector<Slot> slots;
  std::vector<int> ptr(h->nblocks + 1, 0);
  auto face_of_side = [&](int side, int I, int J) {
    if (side == 0) return J * (nc - 1) + (I - 1);
    if (side == 1) return J * (nc - 1) + I;
    if (side == 2) return nV + (J - 1) * nc + I;
    return nV + J * nc + I;
  };
  for (int blk = 0; blk < h->nblocks; ++blk) {
    const int I = blk % nc, J = blk / nc;
    ptr[blk] = (int)slots.size();
    const int cI[4] = {I, I + 1, I, I + 1}, cJ[4] = {J, J, J + 1, J + 1};
    for (int k = 0; k < 4; ++k)
      if (cI[k] >= 1 && cI[k] <= nc - 1 && cJ[k] >= 1 && cJ[k] <= nc - 1)
        slots.push_back(Slot{blk, 0, k, 0, -1, (cJ[k] - 1) * (nc - 1) + (cI[k] - 1)});
    if (!rt_only) {
      const bool inner[4] = {I >= 1, I + 1 < nc, J >= 1, J + 1 < nc};
      for (int s = 0; s < 4; ++s) {
        if (!inner[s]) continue;
        const int f = face_of_side(s, I, J);
        for (int k = 1; k < nsel[f]; ++k) slots.push_back(Slot{blk, 1, s, k, f, zbase[f] + k - 1});
      }
    }
  }
  ptr[h->nblocks] = (int)slots.size();
  c.nslots = (int)slots.size();
  // coarse row keys (nested-dissection ordering of the coarse system)
  c.key.assign(c.D, 0);
  for (int u = 0; u < ntheta; ++u) c.key[u] = 2 * (u / (nc - 1) + 1);
  for (int f = 0; f < nfaces; ++f)
    for (int u = zbase[f]; u < zbase[f + 1]; ++u) c.key[u] = f < nV ? 2 * (f / (nc - 1)) + 1 : 2 * ((f - nV) / nc + 1);
  std::vector<int> gather((size_t)std::max(c.D, 1) * 4, -1);
  for (int s = 0; s < c.nslots; ++s) {
    int* g = &gather[(size_t)slots[s].coef * 4];
    int k = 0;
    while (k < 4 && g[k] >= 0) ++k;
    if (k == 4) return TG_ERR_UNSUPPORTED;
    g[k] = s;
  }
  c.max_slots_per_block = 0;
  for (int blk = 0; blk < h->nblocks; ++blk)
    c.max_slots_per_block = std::max(c.max_slots_per_block, ptr[blk + 1] - ptr[blk]);
  const size_t ts = tile_size(h->opt.precision);
  if (dalloc(&c.slot_ptr, ptr.size()) || dalloc(&c.slots, slots.size()) || dalloc(&c.gather, gather.size()) ||
      dalloc(&c.closed, (size_t)c.nslots * (b + 1) * (b + 1)) || dalloc(&c.Kinv, (size_t)c.D * c.D))
    return TG_ERR_OOM;
  const size_t tsz = rt_only ? 8 : ts;  // the RT0 space of the preprocessing is FP64
  TG_CK(cudaMalloc(&c.owned, std::max<size_t>(1, (size_t)c.nslots * b * b * tsz)));
  TG_CK(cudaMemcpyAsync(c.slot_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, h->stream));
  if (!slots.empty())
    TG_CK(cudaMemcpyAsync(c.slots, slots.data(), sizeof(Slot) * slots.size(), cudaMemcpyHostToDevice,
                          h->stream));
  TG_CK(cudaMemcpyAsync(c.gather, gather.data(), sizeof(int) * gather.size(), cudaMemcpyHostToDevice,
                        h->stream));
  TG_CK(cudaStreamSynchronize(h->stream));  // host vectors go out of scope
  return TG_OK;
}

// tiles, Galerkin matrix and its inverse
int galerkin_inverse(tg_handle* h, CoarseSpace& c);

int finish_space(tg_handle* h, CoarseSpace& c, const double* psiS, const double* fcoef, const double* zcoef,
                 const int* jeff, bool rt_only) {
  const int b = h->b, n = h->n;
  if (c.nslots > 0) {
    if (rt_only || h->opt.precision == TG_PREC_F64)
      launch_build_tiles<double>(c, psiS, fcoef, zcoef, jeff, rt_only ? 1 : 0, n, b, h->stream);
    else
      launch_build_tiles<float>(c, psiS, fcoef, zcoef, jeff, 0, n, b, h->stream);
  }
  return galerkin_inverse(h, c);
}

// Galerkin matrix R_H K R_H^T of a coarse space from its FP64 closed tiles,
// with the cell weights kinv (1/kappa, or a change of it: the matrix is
// linear in them), into K (D x D, device)
int assemble_galerkin(tg_handle* h, const CoarseSpace& c, const double* kinv, double* K,
                      const unsigned char* bmask = nullptr) {
  const int b = h->b, n = h->n;
  std::vector<int> ptr(h->nblocks + 1);
  TG_CK(cudaMemcpy(ptr.data(), c.slot_ptr, sizeof(int) * ptr.size(), cudaMemcpyDeviceToHost));
  std::vector<long long> pptr(h->nblocks + 1, 0);
  for (int k = 0; k < h->nblocks; ++k) {
    const long long m = ptr[k + 1] - ptr[k];
    pptr[k + 1] = pptr[k] + m * m;
  }
  long long* d_pptr = nullptr;
  double* pairE = nullptr;
  int rc = (scratch(h, kScrPPtr, pptr.size(), &d_pptr) || scratch(h, kScrPairE, (size_t)pptr.back(), &pairE))
               ? TG_ERR_OOM : TG_OK;
  if (!rc)
    rc = cuda_err(cudaMemcpyAsync(d_pptr, pptr.data(), sizeof(long long) * pptr.size(), cudaMemcpyHostToDevice,
                                  h->stream));
  if (!rc) {
    launch_galerkin(c, kinv, h->nblocks, n, b, pairE, d_pptr, K, h->stream, bmask);
    rc = cuda_err(cudaStreamSynchronize(h->stream));
  }
  return rc ? rc : cuda_err(cudaGetLastError());
}

// The double-float copy of the preconditioner's coarse inverse, formed again
// after every change of Kinv (mixed-precision handles whose coarse solve is a
// separate GEMV, D > kCoarseSplit; FP64 handles and the preprocessing's RT0
// space keep the FP64 GEMV)
int refresh_coarse_df(tg_handle* h, CoarseSpace& c) {
  if (&c != &h->cs || h->opt.precision == TG_PREC_F64 || c.D <= kCoarseSplit || c.solver == 2) return TG_OK;
  if (!c.Kdf && dalloc(&c.Kdf, (size_t)c.D * c.D)) return TG_ERR_OOM;
  launch_split_df(c.Kinv, c.Kdf, (long long)c.D * c.D, h->stream);
  return cuda_err(cudaStreamSynchronize(h->stream));
}

// Which solver a coarse space of this handle takes (1 dense inverse, 2 nested
// dissection; the latter needs at least 4 coarse blocks per side)
int coarse_solver_for(const tg_handle* h, const CoarseSpace& c) {
  if (h->nc < 4) return 1;
  if (h->opt.coarse_solver == TG_COARSE_SOLVER_ND) return 2;
  if (h->opt.coarse_solver == TG_COARSE_SOLVER_AUTO && c.D > kNdAutoMin && !c.updated_dense) return 2;
  return 1;
}

// Galerkin matrix of a coarse space with the handle's current kappa, and its
// inverse (dense Gauss-Jordan) or nested-dissection factor
int galerkin_inverse(tg_handle* h, CoarseSpace& c) {
  if (c.D == 0) return cuda_err(cudaGetLastError());
  c.low_rank_updates = 0;
  if (coarse_solver_for(h, c) == 2) {
    int rc = assemble_galerkin(h, c, h->kinv, c.Kinv);   // Kinv holds the matrix itself
    if (!rc) rc = nd_build(c.Kinv, c.D, c.key, h->nc, c.gather, c.nd, h->d_status, h->stream);
    if (rc == TG_OK) {
      c.solver = 2;
      cudaFree(c.Kdf);
      c.Kdf = nullptr;
      return cuda_err(cudaGetLastError());
    }
    if (rc != TG_ERR_UNSUPPORTED) return rc;
  }
  c.solver = 1;
  nd_free(c.nd);
  double* tmp = nullptr;
  if (scratch(h, kScrDense, (size_t)c.D * c.D, &tmp)) return TG_ERR_OOM;
  int rc = assemble_galerkin(h, c, h->kinv, c.Kinv);
  if (!rc) {
    launch_gauss_jordan(c.Kinv, tmp, c.D, h->d_status, h->stream);
    rc = cuda_err(cudaStreamSynchronize(h->stream));
  }
  if (rc == TG_OK) rc = refresh_coarse_df(h, c);
  if (rc == TG_OK) rc = cuda_err(cudaGetLastError());
  return rc;
}

// The Galerkin inverse after 1/kappa changed by delta (device, n x n; zero on
// unchanged cells), with the handle's kinv already the new one.  The change
// of the Galerkin matrix, Galerkin(delta), is nonzero only in the rows and
// columns S of basis functions that meet a changed cell; with B the current
// inverse, X = B[:, S] and P = B[S, S]^{-1} the new inverse is
//   B + X M X^T,  M = -P (P + Delta_SS)^{-1} Delta_SS
// (the Sherman-Morrison-Woodbury identity written with SPD inverses only:
// P and P + Delta_SS are the Schur complements on S of the old and new
// matrices).  O(D^2 |S|) instead of O(D^3).  Falls back to the full inverse
// when |S| is large, after kMaxLowRankUpdates updates in a row (rounding of
// the updates accumulates) or when a small inverse meets a non-positive pivot.
// bmask (device, optional): the blocks that hold a changed cell.
int galerkin_update(tg_handle* h, CoarseSpace& c, const double* delta, const unsigned char* bmask, int* rank) {
  constexpr int kMaxLowRankUpdates = 64;
  *rank = -1;
  if (c.D == 0) return cuda_err(cudaGetLastError());
  // a nested-dissection factor is formed again in full; under
  // TG_COARSE_SOLVER_AUTO the space turns to the dense inverse instead, so
  // that the next changes are low-rank updates
  if (c.solver == 2 && h->opt.coarse_solver == TG_COARSE_SOLVER_AUTO) {
    c.updated_dense = true;
    h->regraph = true;
  }
  if (c.solver == 2 || c.low_rank_updates >= kMaxLowRankUpdates) return galerkin_inverse(h, c);
  cudaStream_t s = h->stream;
  const int D = c.D;
  double* dK = nullptr;
  unsigned char* d_flag = nullptr;
  if (scratch(h, kScrDense, (size_t)D * D, &dK) || scratch(h, kScrFlag, (size_t)D, &d_flag)) return TG_ERR_OOM;
  int rc = assemble_galerkin(h, c, delta, dK, bmask);
  std::vector<unsigned char> flag(D);
  if (!rc) {
    launch_row_nonzero(dK, D, d_flag, s);
    rc = cuda_err(cudaMemcpyAsync(flag.data(), d_flag, D, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  }
  std::vector<int> S;
  for (int i = 0; i < D && !rc; ++i)
    if (flag[i]) S.push_back(i);
  const int m = (int)S.size();
  if (rc || m == 0 || m > kGjSmallMax || 4 * m > D) {
    if (rc) return rc;
    if (m == 0) *rank = 0;
    return m == 0 ? TG_OK : galerkin_inverse(h, c);
  }
  int* d_S = nullptr;
  int* d_bad = nullptr;
  double *X = nullptr, *P = nullptr, *Q = nullptr, *dS = nullptr, *W = nullptr, *T = nullptr;
  double* small = nullptr;
  const size_t mm2 = (size_t)m * m;
  rc = (scratch(h, kScrIds, (size_t)m, &d_S) || scratch(h, kScrBad, 1, &d_bad) || scratch(h, kScrX, (size_t)D * m, &X) ||
        scratch(h, kScrSmall, 4 * mm2, &small) || scratch(h, kScrT, (size_t)D * m, &T))
           ? TG_ERR_OOM : TG_OK;
  if (!rc) {
    P = small;
    Q = small + mm2;
    dS = small + 2 * mm2;
    W = small + 3 * mm2;
  }
  int bad = 0;
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_S, S.data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  if (!rc) {
    const long long mm = (long long)m * m;
    launch_gather_cols(c.Kinv, D, d_S, m, D, true, X, s);      // X = B[:, S]
    launch_gather_cols(c.Kinv, D, d_S, m, m, false, P, s);     // B_SS
    launch_gather_cols(dK, D, d_S, m, m, false, dS, s);        // Delta_SS
    launch_gj_small(P, m, d_bad, s);                           // P = B_SS^{-1}
    cudaMemcpyAsync(Q, P, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s);
    launch_add(Q, dS, mm, s);
    launch_gj_small(Q, m, d_bad, s);                           // Q = (P + Delta_SS)^{-1}
    launch_dgemm(m, m, m, 1.0, Q, m, 1, dS, m, 1, 0.0, W, m, s);     // W = Q Delta_SS
    launch_dgemm(m, m, m, -1.0, P, m, 1, W, m, 1, 0.0, Q, m, s);     // M = -P W (into Q)
    launch_symmetrize(Q, m, s);
    launch_dgemm(D, m, m, 1.0, X, m, 1, Q, m, 1, 0.0, T, m, s);      // T = X M
    rc = cuda_err(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
    if (!rc && !bad) {
      if (m <= 8) launch_rank_update(c.Kinv, D, T, X, m, s);             // B += T X^T
      else launch_dgemm(D, D, m, 1.0, T, m, 1, X, 1, m, 1.0, c.Kinv, D, s);
      rc = cuda_err(cudaStreamSynchronize(s));
    }
  }
  if (rc) return rc;
  if (bad) return galerkin_inverse(h, c);
  ++c.low_rank_updates;
  *rank = m;
  rc = refresh_coarse_df(h, c);
  return rc ? rc : cuda_err(cudaGetLastError());
}

// extreme eigenvalues of the Lanczos tridiagonal by Sturm bisection (report only)
double lanczos_cond(const PcgState& st) {
  const int m = std::min(st.iter, kMaxHist);
  if (m <= 0) return 1.0;
  std::vector<double> d(m), e(m > 1 ? m - 1 : 1, 0.0);
  for (int j = 0; j < m; ++j) d[j] = 1.0 / st.alphas[j] + (j > 0 ? st.betas[j - 1] / st.alphas[j - 1] : 0.0);
  for (int j = 0; j + 1 < m; ++j) e[j] = std::sqrt(std::max(0.0, st.betas[j])) / st.alphas[j];
  double lo = 1e300, hi = -1e300;
  for (int j = 0; j < m; ++j) {
    const double rad = (j > 0 ? std::fabs(e[j - 1]) : 0.0) + (j + 1 < m ? std::fabs(e[j]) : 0.0);
    lo = std::min(lo, d[j] - rad);
    hi = std::max(hi, d[j] + rad);
  }
  auto count_below = [&](double x) {  // eigenvalues < x
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int j = 1; j < m; ++j) {
      if (q == 0.0) q = 1e-300;
      q = d[j] - x - e[j - 1] * e[j - 1] / q;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  auto kth = [&](int k) {  // k-th smallest (0-based)
    double a = lo, c = hi;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a + c);
      if (count_below(mid) > k) c = mid;
      else a = mid;
    }
    return 0.5 * (a + c);
  };
  const double lmin = kth(0), lmax = kth(m - 1);
  return (lmin > 0) ? lmax / lmin : INFINITY;
}

int validate_grid(const tg_grid* g) {
  if (!g) return TG_ERR_INVALID_ARG;
  if (g->nx != g->ny || g->bx != g->by) return TG_ERR_UNSUPPORTED;
  if (g->nx < 2 || g->bx < 2 || g->nx % g->bx != 0) return TG_ERR_INVALID_ARG;
  if (g->nx / g->bx < 2) return TG_ERR_INVALID_ARG;   // one coarse block: no coarse faces, empty coarse space
  if (g->bx > kMaxB) return TG_ERR_UNSUPPORTED;
  if (g->overlap < 1) return TG_ERR_INVALID_ARG;   // singular preconditioner (no patch covers the coarse lines)
  if (g->overlap > kMaxOverlap) return TG_ERR_UNSUPPORTED;
  if ((long long)g->nx * g->nx > (1LL << 30)) return TG_ERR_UNSUPPORTED;
  return TG_OK;
}


// ---- solve contexts ---------------------------------------------------------
void ctx_free(Ctx* c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->exec_warm) cudaGraphExecDestroy(c->exec_warm);
  if (c->cap) cudaStreamDestroy(c->cap);
  cudaFree(c->ux0);
  cudaFree(c->slab);
  if (c->h_rtol) cudaFreeHost(c->h_rtol);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->prof_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->prof_op_ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

int ctx_alloc(tg_handle* h, Ctx** out) {
  *out = nullptr;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return TG_ERR_OOM;
  c->h = h;
  const int n = h->n, nc = h->nc;
  const long long nn = (long long)n * n, nf = (long long)(n + 1) * n;
  const size_t tc = (h->opt.precision == TG_PREC_F64) ? 8 : 4;
  // partials: reductions over up to max(kRedGrid, stencil tiles) CTAs, and the
  // last smoothing sweep's two dot products over its one-wave grid
  const long long npart = 4 * std::max<long long>(2048, (long long)((n + 31) / 32) * ((n + 7) / 8));
  // Every device vector of the context is carved from one allocation (a
  // batch creates nrhs + 1 contexts per instance: one cudaMalloc each instead
  // of 29).  Each vector starts on a 256-byte boundary and is followed by a
  // gap of at least 512 bytes.
  struct Part {
    void** ptr;
    size_t bytes;
  };
  const size_t d8 = sizeof(double);
  auto cnt = [](long long v) { return (size_t)std::max<long long>(v, 1); };   // empty vectors get one element
  const Part parts[] = {
      {(void**)&c->x, d8 * cnt(nn)},          {(void**)&c->r, d8 * cnt(nn)},
      {(void**)&c->p, d8 * cnt(nn)},          {(void**)&c->q, d8 * cnt(nn)},
      {(void**)&c->rho, d8 * cnt(nn)},        {(void**)&c->phi, d8 * cnt(nn)},
      {(void**)&c->p2, d8 * cnt(nn)},         {(void**)&c->r2, d8 * cnt(nn)},
      {(void**)&c->ux, d8 * cnt(nf)},         {(void**)&c->uy, d8 * cnt(nf)},
      {(void**)&c->fd, d8 * cnt(nn)},         {(void**)&c->bd, d8 * cnt(4LL * n)},
      {(void**)&c->pd, d8 * cnt(nn)},         {(void**)&c->pw, d8 * cnt(nn + 2LL * n + 2)},
      {(void**)&c->part, d8 * cnt(npart)},    {(void**)&c->gx, d8 * cnt((nc + 1LL) * nc)},
      {(void**)&c->gy, d8 * cnt((nc + 1LL) * nc)}, {(void**)&c->FH, d8 * cnt(h->nblocks)},
      {(void**)&c->absF, d8 * cnt(h->nblocks)}, {(void**)&c->diverr, d8 * 2},
      {(void**)&c->cs_part, d8 * cnt(h->cs.nslots)}, {(void**)&c->cs_coefs, d8 * cnt(5LL * h->cs.D)},
      {(void**)&c->rt_part, d8 * cnt(h->rt.nslots)}, {(void**)&c->rt_coefs, d8 * cnt(5LL * h->rt.D)},
      {(void**)&c->st, sizeof(PcgState)},     {(void**)&c->d_rtol, d8},
      {(void**)&c->zacc, tc * cnt(nn)},       {(void**)&c->zacc2, tc * cnt(nn)},
      {(void**)&c->rin, tc * cnt(nn)},
  };
  constexpr size_t kAlign = 256, kGap = 512;
  size_t off[sizeof(parts) / sizeof(parts[0])], total = 0;
  for (size_t k = 0; k < sizeof(parts) / sizeof(parts[0]); ++k) {
    total = (total + kAlign - 1) / kAlign * kAlign;
    off[k] = total;
    total += parts[k].bytes + kGap;
  }
  int rc = cuda_err(cudaMalloc(&c->slab, total));
  for (size_t k = 0; !rc && k < sizeof(parts) / sizeof(parts[0]); ++k) *parts[k].ptr = (char*)c->slab + off[k];
  if (!rc) rc = cuda_err(cudaMallocHost(&c->h_rtol, sizeof(double)));
  for (auto& e : c->ev)
    if (!rc) rc = cuda_err(cudaEventCreate(&e));
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  if (!rc && h->opt.profile) {
    c->prof_ev.resize(2048);
    for (auto& e : c->prof_ev)
      if (!rc) rc = cuda_err(cudaEventCreate(&e));
    c->prof_op_ev.resize(1024);
    for (auto& e : c->prof_op_ev)
      if (!rc) rc = cuda_err(cudaEventCreate(&e));
  }
  if (!rc) rc = cuda_err(cudaMemsetAsync(c->st, 0, sizeof(PcgState), h->stream));
  if (rc) {
    ctx_free(c);
    return rc;
  }
  *out = c;
  return TG_OK;
}

// ---- the two-grid preconditioner (Section 5), zacc must be zero on entry ----
void prof_mark(Ctx* c, cudaStream_t s) {
  if (c->h->opt.profile && c->prof_used < (int)c->prof_ev.size()) cudaEventRecord(c->prof_ev[c->prof_used++], s);
}
void prof_op_mark(Ctx* c, cudaStream_t s) {
  if (c->h->opt.profile && c->prof_op_used < (int)c->prof_op_ev.size())
    cudaEventRecord(c->prof_op_ev[c->prof_op_used++], s);
}

template <typename TC, typename TS>
void precondition(Ctx* c, const double* r, TC* zacc, const PcgState* st, cudaStream_t s) {
  tg_handle* h = c->h;
  const int n = h->n;
  const TC* kin = std::is_same<TC, double>::value ? (const TC*)h->kinv : (const TC*)h->kinv32;
  TC* rin = (TC*)c->rin;
  const TS* pinv = (const TS*)h->pinv;
  const double eta = h->opt.eta;
  if (h->opt.cycle == TG_CYCLE_ADDITIVE) {
    // z = S r + P r: both parts from r
    prof_mark(c, s);
    launch_smoother<TC, TS, double>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, r, zacc, eta, n, st, s,
                                    h->shape, h->rscale, h->band);
    prof_mark(c, s);
    if (h->cs.D > 0) {
      launch_restrict<double, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r, st, s);
      launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, zacc, st, s);
    }
    return;
  }
  for (int k = 0; k < h->opt.m1; ++k) {
    if (k == 0) {
      prof_mark(c, s);
      launch_smoother<TC, TS, double>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, r, zacc, eta, n, st, s,
                                      h->shape, h->rscale, h->band);
      prof_mark(c, s);
    } else {
      launch_residual<TC>(r, zacc, kin, rin, n, st, s);
      prof_mark(c, s);
      launch_smoother<TC, TS, TC>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, rin, zacc, eta, n, st, s, h->shape,
                                  h->rscale, h->band);
      prof_mark(c, s);
    }
  }
  if (h->cs.D > 0) {
    launch_resid_restrict<TC, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r, zacc, kin, st, s);
    launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, zacc, st, s);
  }
  for (int k = 0; k < h->opt.m2; ++k) {
    launch_residual<TC>(r, zacc, kin, rin, n, st, s);
    prof_mark(c, s);
    launch_smoother<TC, TS, TC>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, rin, zacc, eta, n, st, s, h->shape,
                                h->rscale, h->band);
    prof_mark(c, s);
  }
}

// Section 3: vbar into (ux, uy), and rho = C^T(-A vbar) (the PCG right-hand side)
void enqueue_preprocess(Ctx* c, const double* f, const double* bflux, double* ux, double* uy, cudaStream_t s) {
  tg_handle* h = c->h;
  const int n = h->n, b = h->b;
  const long long nn = (long long)n * n;
  launch_lift(bflux, ux, uy, n, s);
  launch_block_sources(f, ux, uy, c->FH, c->absF, n, b, s);
  launch_rt_particular(c->FH, c->absF, c->gx, c->gy, h->nc, h->H, h->nblocks, c->st, s);
  launch_add_rt_field(c->gx, c->gy, ux, uy, n, b, s);
  if (h->rt.D > 0) {
    launch_face_residual(ux, uy, h->kinv, c->rho, n, s);
    launch_restrict<double, double>(h->rt, c->rt_part, h->nblocks, h->nc, b, n, c->rho, nullptr, s);
    cudaMemsetAsync(c->phi, 0, sizeof(double) * nn, s);
    launch_coarse_correct<double, double>(h->rt, c->rt_part, c->rt_coefs, h->nblocks, h->nc, b, n, c->phi, nullptr, s);
    launch_add_curl(c->phi, ux, uy, n, s);
  }
  launch_block_particular(f, ux, uy, n, b, s);
  launch_face_residual(ux, uy, h->kinv, c->rho, n, s);
  // phi = K_K^{-1} rho on every block's interior nodes: the smoother's GEMV
  // with the dense block inverses (blocks do not overlap, eta = 1).  phi is a
  // stream function, so its precision cannot change the divergence of vbar;
  // it only moves the PCG starting point, and mixed-precision handles use
  // FP32 inverses and FP32 accumulation (in the free inner-residual buffer).
  if (h->binv) {
    cudaMemsetAsync(c->phi, 0, sizeof(double) * nn, s);
    launch_smoother<double, double, double>(h->d_bgeo, h->d_bgofs, h->nblocks, h->bgroups, h->binv, c->rho, c->phi,
                                            1.0, n, nullptr, s);
  } else {
    float* phi32 = (float*)c->rin;
    cudaMemsetAsync(phi32, 0, sizeof(float) * nn, s);
    launch_smoother<float, float, double>(h->d_bgeo, h->d_bgofs, h->nblocks, h->bgroups, h->binv32, c->rho, phi32,
                                          1.0, n, nullptr, s);
    launch_convert<float, double>(phi32, c->phi, nn, s);
  }
  launch_add_curl(c->phi, ux, uy, n, s);
  launch_face_residual(ux, uy, h->kinv, c->rho, n, s);
}

// reset + preprocessing + PCG start (r = rho, x = 0, z = M r, p = z)
template <typename TC, typename TS>
void enqueue_prefix(Ctx* c, cudaStream_t s) {
  tg_handle* h = c->h;
  const int n = h->n;
  const long long nn = (long long)n * n;
  launch_pcg_reset(c->st, c->d_rtol, std::min(h->opt.max_iter, kMaxHist), h->opt.flexible, s);
  enqueue_preprocess(c, c->fd, c->bd, c->ux, c->uy, s);
  if (c->warm) {
    // x0 = stream function of the guess minus vbar; r = rho - K x0
    launch_psi_from_faces(c->ux0, c->ux, c->pw, c->x, n, s);
    launch_pcg_init_warm(c->x, c->rho, h->kinv, c->r, c->part, c->st, n, s);
  } else {
    cudaMemcpyAsync(c->r, c->rho, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
    launch_pcg_init(c->x, c->r, c->part, c->st, n, s);
  }
  cudaMemsetAsync(c->zacc, 0, sizeof(TC) * nn, s);
  precondition<TC, TS>(c, c->r, (TC*)c->zacc, c->st, s);
  launch_pcg_init_rz<TC>(c->r, (const TC*)c->zacc, c->p, c->part, c->st, n, s);
}

// one PCG iteration (every kernel returns at once when st->done is set).
// parity 0 reads (p, r, zacc) and writes (p2, r2, zacc2); parity 1 the reverse.
//   q = K p_new, p_new = z_prev + beta p_old                (operator kernel)
//   r_new = r_old - alpha q, x += alpha p_new, z = S r_new  (first smoothing)
//   z += P (r_new - K z)                                    (coarse correction)
//   z += S (r_new - K z)                                    (post-smoothing)
//   beta from (r_new, z) and (z, q)
template <typename TC, typename TS>
void enqueue_iteration(Ctx* c, int parity, cudaStream_t s) {
  tg_handle* h = c->h;
  const int n = h->n;
  double* p_old = parity ? c->p2 : c->p;
  double* p_new = parity ? c->p : c->p2;
  double* r_old = parity ? c->r2 : c->r;
  double* r_new = parity ? c->r : c->r2;
  const TC* kin = std::is_same<TC, double>::value ? (const TC*)h->kinv : (const TC*)h->kinv32;
  TC* rin = (TC*)c->rin;
  const TS* pinv = (const TS*)h->pinv;
  const double eta = h->opt.eta;
  PcgState* st = c->st;
  // the five-kernel form gathers r - K z per patch node inside the last
  // sweep; the band sweep (one warp per patch) gathers better from a
  // separately formed residual, so band handles take the general form
  if (h->opt.m1 == 1 && h->opt.m2 == 1 && h->opt.cycle == TG_CYCLE_TWO_GRID && !is_band_shape(h->shape)) {
    // The cycle of Section 6 (m1 = m2 = 1) in five kernels.  z ends every
    // iteration in zacc (A); zacc2 (B) holds the intermediate z.  The first
    // sweep accumulates into B and clears A (dead once p is formed), the
    // coarse step adds into B, and the last sweep forms r - K z_B at gather
    // time and accumulates z_B + S(r - K z_B) into A.
    TC* zA = (TC*)c->zacc;
    TC* zB = (TC*)c->zacc2;
    prof_op_mark(c, s);
    launch_pcg_apply_p<TC>(zA, p_old, p_new, c->q, zB, h->kcoef, c->part, st, n, s);
    prof_op_mark(c, s);
    prof_mark(c, s);
    launch_smoother_update<TC, TS>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, r_old, r_new, c->q, c->x,
                                   p_new, zB, eta, n, h->nc, h->b, c->part, st, s, h->shape, h->rscale, zA, h->band);
    prof_mark(c, s);
    if (h->cs.D > 0) {
      launch_resid_restrict<TC, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r_new, zB, kin, st, s);
      launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, zB, st, s);
    }
    prof_mark(c, s);
    launch_smoother_resid<TC, TS>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, r_new, zB, kin, zA, eta, n,
                                  h->nc, h->b, st, s, h->shape, h->rscale, h->band);
    prof_mark(c, s);
    launch_pcg_dots<TC>(r_new, zA, c->q, c->part, st, n, s);
    return;
  }
  TC* z_prev = (TC*)(parity ? c->zacc2 : c->zacc);
  TC* z_cur = (TC*)(parity ? c->zacc : c->zacc2);
  prof_op_mark(c, s);
  launch_pcg_apply_p<TC>(z_prev, p_old, p_new, c->q, z_cur, h->kcoef, c->part, st, n, s);
  prof_op_mark(c, s);
  prof_mark(c, s);
  launch_smoother_update<TC, TS>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, r_old, r_new, c->q, c->x,
                                 p_new, z_cur, eta, n, h->nc, h->b, c->part, st, s, h->shape, h->rscale, nullptr,
                                 h->band);
  prof_mark(c, s);
  if (h->opt.cycle == TG_CYCLE_ADDITIVE) {
    // z = S r + P r: the coarse part restricts r itself
    if (h->cs.D > 0) {
      launch_restrict<double, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r_new, st, s);
      launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, z_cur, st, s);
    }
    launch_pcg_dots<TC>(r_new, z_cur, c->q, c->part, st, n, s);
    return;
  }
  for (int k = 1; k < h->opt.m1; ++k) {
    launch_residual<TC>(r_new, z_cur, kin, rin, n, st, s);
    prof_mark(c, s);
    launch_smoother<TC, TS, TC>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, rin, z_cur, eta, n, st, s, h->shape,
                                h->rscale, h->band);
    prof_mark(c, s);
  }
  if (h->cs.D > 0) {
    launch_resid_restrict<TC, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r_new, z_cur, kin, st, s);
    launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, z_cur, st, s);
  }
  for (int k = 0; k < h->opt.m2; ++k) {
    launch_residual<TC>(r_new, z_cur, kin, rin, n, st, s);
    prof_mark(c, s);
    launch_smoother<TC, TS, TC>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, rin, z_cur, eta, n, st, s, h->shape,
                                h->rscale, h->band);
    prof_mark(c, s);
  }
  launch_pcg_dots<TC>(r_new, z_cur, c->q, c->part, st, n, s);
}

// Step 4: v = vbar + C x, pressure, conservation check
void enqueue_epilogue(Ctx* c, cudaStream_t s) {
  tg_handle* h = c->h;
  launch_add_curl(c->x, c->ux, c->uy, h->n, s);
  launch_pressure(c->ux, c->uy, h->kinv, c->pd, c->pw, h->n, s);
  launch_div_error(c->ux, c->uy, c->fd, c->part, c->diverr, h->n, s);
}

// Appends the chain  prefix -> while(two iterations) -> epilogue  of one
// context to `graph` (roots: no dependencies), captured on stream cs.
template <typename TC, typename TS>
int add_chain_t(Ctx* c, cudaGraph_t graph, cudaStream_t cs) {
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaStreamCaptureStatus cst;
  unsigned long long k0 = g_kernel_launches;
  TG_CK(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enqueue_prefix<TC, TS>(c, cs);
  TG_CK(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  cudaGraph_t g2 = nullptr;
  TG_CK(cudaStreamEndCapture(cs, &g2));
  (c->warm ? c->k_prefix_warm : c->k_prefix) = g_kernel_launches - k0;
  cudaGraphConditionalHandle cond;
  TG_CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  TG_CK(cudaGraphAddNode(&wnode, graph, tail.data(), nullptr, tail.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  k0 = g_kernel_launches;
  TG_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enqueue_iteration<TC, TS>(c, 0, cs);
  enqueue_iteration<TC, TS>(c, 1, cs);
  launch_set_condition(cond, c->st, cs);
  TG_CK(cudaStreamEndCapture(cs, &body));
  c->k_body = g_kernel_launches - k0;
  k0 = g_kernel_launches;
  TG_CK(cudaStreamBeginCaptureToGraph(cs, graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  enqueue_epilogue(c, cs);
  TG_CK(cudaStreamEndCapture(cs, &g2));
  c->k_epi = g_kernel_launches - k0;
  return TG_OK;
}

// one PCG iteration of a lock-step group: the per-chain kernels of the
// five-kernel iteration in sequence, with both smoothing sweeps shared by the
// k chains (one read of the patch inverses for all of them).  Forking the
// per-chain kernels (or the prefixes and epilogues) into parallel branches of
// the graph measured slower: 364 against 281 ms per step on the 64 x 4 batch.
template <typename TC, typename TS>
void enqueue_group_iteration(Ctx* const* cs, int k, int parity, cudaStream_t s) {
  tg_handle* h = cs[0]->h;
  if (is_band_shape(h->shape)) {   // no lock-step band sweep: each chain's own iteration
    for (int i = 0; i < k; ++i) enqueue_iteration<TC, TS>(cs[i], parity, s);
    return;
  }
  const int n = h->n;
  const TC* kin = std::is_same<TC, double>::value ? (const TC*)h->kinv : (const TC*)h->kinv32;
  const TS* pinv = (const TS*)h->pinv;
  ChainPtrs m1[kGroup] = {}, m2[kGroup] = {};
  for (int i = 0; i < k; ++i) {
    Ctx* c = cs[i];
    double* p_old = parity ? c->p2 : c->p;
    double* p_new = parity ? c->p : c->p2;
    double* r_old = parity ? c->r2 : c->r;
    double* r_new = parity ? c->r : c->r2;
    TC* zA = (TC*)c->zacc;
    TC* zB = (TC*)c->zacc2;
    launch_pcg_apply_p<TC>(zA, p_old, p_new, c->q, zB, h->kcoef, c->part, c->st, n, s);
    m1[i] = ChainPtrs{r_old, r_new, c->q, c->x, p_new, c->part, c->st, zA, nullptr, nullptr, r_old, zB};
    m2[i] = ChainPtrs{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, c->st, nullptr, zB, kin, r_new, zA};
  }
  launch_smoother_multi<TC, TS>(1, h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, m1, k, h->opt.eta, n, h->nc,
                                h->b, s, h->shape, h->rscale, &h->band);
  if (h->cs.D > 0) {
    for (int i = 0; i < k; ++i) {
      Ctx* c = cs[i];
      const double* r_new = parity ? c->r : c->r2;
      TC* zB = (TC*)c->zacc2;
      launch_resid_restrict<TC, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, r_new, zB, kin, c->st, s);
      launch_coarse_correct<TC, tile_t<TS>>(h->cs, c->cs_part, c->cs_coefs, h->nblocks, h->nc, h->b, n, zB, c->st, s);
    }
  }
  launch_smoother_multi<TC, TS>(2, h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, pinv, m2, k, h->opt.eta, n, h->nc,
                                h->b, s, h->shape, h->rscale, &h->band);
  for (int i = 0; i < k; ++i) {
    Ctx* c = cs[i];
    const double* r_new = parity ? c->r : c->r2;
    launch_pcg_dots<TC>(r_new, (const TC*)c->zacc, c->q, c->part, c->st, n, s);
  }
}

// Appends one lock-step group of k (<= kGroup) contexts of the same handle:
// their prefixes, one while node whose body runs two group iterations and
// loops while any chain runs, then their epilogues.
template <typename TC, typename TS>
int add_group_t(Ctx* const* cs, int k, cudaGraph_t graph, cudaStream_t cap) {
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaStreamCaptureStatus cst;
  TG_CK(cudaStreamBeginCaptureToGraph(cap, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) enqueue_prefix<TC, TS>(cs[i], cap);
  TG_CK(cudaStreamGetCaptureInfo(cap, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  cudaGraph_t g2 = nullptr;
  TG_CK(cudaStreamEndCapture(cap, &g2));
  cudaGraphConditionalHandle cond;
  TG_CK(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  TG_CK(cudaGraphAddNode(&wnode, graph, tail.data(), nullptr, tail.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const PcgState* states[kGroup] = {};
  for (int i = 0; i < k; ++i) states[i] = cs[i]->st;
  TG_CK(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  enqueue_group_iteration<TC, TS>(cs, k, 0, cap);
  enqueue_group_iteration<TC, TS>(cs, k, 1, cap);
  launch_set_condition_any(cond, states, k, cap);
  TG_CK(cudaStreamEndCapture(cap, &body));
  TG_CK(cudaStreamBeginCaptureToGraph(cap, graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) enqueue_epilogue(cs[i], cap);
  TG_CK(cudaStreamEndCapture(cap, &g2));
  return TG_OK;
}

int add_group(Ctx* const* cs, int k, cudaGraph_t graph, cudaStream_t cap) {
  switch (cs[0]->h->opt.precision) {
    case TG_PREC_F64: return add_group_t<double, double>(cs, k, graph, cap);
    case TG_PREC_F32: return add_group_t<float, float>(cs, k, graph, cap);
    case TG_PREC_F16: return add_group_t<float, __half>(cs, k, graph, cap);
    default: return add_group_t<float, __nv_bfloat16>(cs, k, graph, cap);
  }
}

int add_chain(Ctx* c, cudaGraph_t graph, cudaStream_t cs) {
  switch (c->h->opt.precision) {
    case TG_PREC_F64: return add_chain_t<double, double>(c, graph, cs);
    case TG_PREC_F32: return add_chain_t<float, float>(c, graph, cs);
    case TG_PREC_F16: return add_chain_t<float, __half>(c, graph, cs);
    default: return add_chain_t<float, __nv_bfloat16>(c, graph, cs);
  }
}

// host-driven loop (profile mode): same kernels, events around the smoother
template <typename TC, typename TS>
int run_loop_t(Ctx* c, unsigned long long* launches) {
  tg_handle* h = c->h;
  cudaStream_t s = h->stream;
  const unsigned long long k0 = g_kernel_launches;
  enqueue_prefix<TC, TS>(c, s);
  cudaEventRecord(c->ev[1], s);
  const int maxit = std::min(h->opt.max_iter, kMaxHist);
  for (int it = 0; it < maxit; ++it) {
    enqueue_iteration<TC, TS>(c, it & 1, s);
    if ((it + 1) % 2 == 0 || it + 1 == maxit) {
      TG_CK(cudaMemcpyAsync(h->h_flag, &c->st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      TG_CK(cudaStreamSynchronize(s));
      if (*h->h_flag) break;
    }
  }
  cudaEventRecord(c->ev[2], s);
  enqueue_epilogue(c, s);
  *launches = g_kernel_launches - k0;
  return cuda_err(cudaGetLastError());
}

int run_loop(Ctx* c, unsigned long long* launches) {
  switch (c->h->opt.precision) {
    case TG_PREC_F64: return run_loop_t<double, double>(c, launches);
    case TG_PREC_F32: return run_loop_t<float, float>(c, launches);
    case TG_PREC_F16: return run_loop_t<float, __half>(c, launches);
    default: return run_loop_t<float, __nv_bfloat16>(c, launches);
  }
}

// kappa and the quantities derived from it cell by cell
int setup_kappa(tg_handle* h, const double* kd, bool update = false) {
  const long long nn = (long long)h->n * h->n;
  cudaStream_t s = h->stream;
  if (!update) {
    TG_CK(cudaMallocHost(&h->h_flag, sizeof(int)));
    TG_CK(cudaMalloc(&h->d_status, sizeof(int)));
    if (dalloc(&h->kinv, nn) || dalloc(&h->kinv32, nn) || dalloc(&h->kcoef, 5 * nn)) return TG_ERR_OOM;
  }
  TG_CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), s));
  launch_kinv(kd, h->kinv, h->kinv32, h->d_status, h->n, s);
  launch_stencil_coefs(h->kinv, h->kcoef, h->n, s);
  int st = 0;
  int rc = read_status(h, &st);
  if (rc) return rc;
  return st ? status_to_err(st) : TG_OK;
}

// rectangles and smoother layout of the oversampled patches K_i^+
struct PatchLayout {
  std::vector<int4> rect;
  std::vector<PatchGeo> geo;
  long long off = 0;   // total stored elements
  long long toff = 0;  // total elements of the tile layout
  std::vector<int> tofs;   // first 16-row tile of each patch (+ total)
  int wmax = 0, nmax = 0;
};

PatchLayout patch_layout(const tg_handle* h) {
  const int n = h->n, b = h->b, nc = h->nc;
  PatchLayout L;
  L.rect.resize(h->npatch);
  L.geo.resize(h->npatch);
  for (int J = 0; J < nc; ++J)
    for (int I = 0; I < nc; ++I) {
      const int k = J * nc + I;
      const int x0 = std::max(0, I * b - h->ov), x1 = std::min(n, (I + 1) * b + h->ov);
      const int y0 = std::max(0, J * b - h->ov), y1 = std::min(n, (J + 1) * b + h->ov);
      PatchGeo g{};
      g.x0 = x0; g.y0 = y0; g.nx = x1 - x0 - 1; g.ny = y1 - y0 - 1;
      g.nloc = g.nx * g.ny;
      g.ld = ((g.nloc + 7) / 8) * 8;
      g.off = L.off;
      L.off += (long long)g.nloc * g.ld;
      const int T = tiles_per_side(g.nloc);
      g.toff = L.toff;
      L.toff += (long long)T * T * kTile * kTile;
      L.geo[k] = g;
      L.rect[k] = make_int4(x0, y0, g.nx, g.ny);
      L.wmax = std::max(L.wmax, g.nx + 1);
      L.nmax = std::max(L.nmax, g.nloc);
    }
  L.tofs.assign(h->npatch + 1, 0);
  for (int k = 0; k < h->npatch; ++k) L.tofs[k + 1] = L.tofs[k] + tiles_per_side(L.geo[k].nloc);
  return L;
}

std::vector<int4> block_rects(const tg_handle* h) {
  std::vector<int4> r(h->nblocks);
  for (int J = 0; J < h->nc; ++J)
    for (int I = 0; I < h->nc; ++I) r[J * h->nc + I] = make_int4(I * h->b, J * h->b, h->b - 1, h->b - 1);
  return r;
}

// changed[m] = 1 where a cell of rect[m] gets a new 1/kappa from kappa (device);
// run before kinv is overwritten
int changed_rects(tg_handle* h, const double* kappa, const std::vector<int4>& rect,
                  std::vector<unsigned char>& changed) {
  cudaStream_t s = h->stream;
  changed.assign(rect.size(), 1);
  if (rect.empty()) return TG_OK;
  int4* d_rect = nullptr;
  unsigned char* d_flag = nullptr;
  int rc = (scratch(h, kScrRect, rect.size(), &d_rect) || scratch(h, kScrFlag, rect.size(), &d_flag)) ? TG_ERR_OOM
                                                                                                      : TG_OK;
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_rect, rect.data(), sizeof(int4) * rect.size(), cudaMemcpyHostToDevice, s));
  if (!rc) {
    launch_rect_changed(kappa, h->kinv, d_rect, (int)rect.size(), h->n, d_flag, s);
    rc = cuda_err(cudaMemcpyAsync(changed.data(), d_flag, rect.size(), cudaMemcpyDeviceToHost, s));
  }
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  return rc;
}

// indices m with sel[m] set (sel NULL: all of 0..count-1)
std::vector<int> selected(int count, const std::vector<unsigned char>* sel) {
  std::vector<int> ids;
  ids.reserve(count);
  for (int m = 0; m < count; ++m)
    if (!sel || (*sel)[m]) ids.push_back(m);
  return ids;
}

// Whether the dense patch inverses (and their tensor-core tiles) are formed:
// FP64 handles and handles given a dense tile shape always; handles whose
// shape the autotuner picks only while the inverses, counted at two bytes an
// entry, stay within 1.5 times the L2.  Above that the band form was the
// faster one at every size measured (the autotuner's warm per-launch times,
// FP16: 448^2 / b = 16, 208 MB, 39.4 against 41.1 us; 512^2 / 16, 272 MB,
// 39.4 against 51.7; 768^2 / 8, 285 MB, 57.8 against 87.8; 1024^2 / 16, 1.1
// GB, 80 against 186), while at 384^2 / 16 (153 MB) the dense tensor-core
// form still won (28.8 against 37.4 us).  The inverses cost most of the
// patch setup and of the handle's memory.
bool dense_inverses_needed(const tg_handle* h, long long entries) {
  if (h->opt.precision == TG_PREC_F64) return true;
  if (h->opt.smoother_shape >= 0) return !is_band_shape(h->opt.smoother_shape);
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
      l2 <= 0) {
    cudaGetLastError();
    return true;
  }
  return 2.0 * (double)entries <= 1.5 * (double)l2;
}

// oversampled patches K_i^+: local operators, band Cholesky, dense inverses.
// update: the storage exists and only the patches in `changed` (NULL: all)
// are factored again
int setup_patches(tg_handle* h, bool update = false, const std::vector<unsigned char>* changed = nullptr) {
  const int n = h->n;
  cudaStream_t s = h->stream;
  const PatchLayout L = patch_layout(h);
  const int wmax = L.wmax, nmax = L.nmax;
  std::vector<int> gofs(h->npatch + 1, 0);
  for (int k = 0; k < h->npatch; ++k) gofs[k + 1] = gofs[k] + (L.geo[k].nloc + kRowsPerGroup - 1) / kRowsPerGroup;
  h->ngroups = gofs[h->npatch];
  if (!update) {
    if (dalloc(&h->d_gofs, gofs.size()) || dalloc(&h->d_pgeo, L.geo.size())) return TG_ERR_OOM;
    TG_CK(cudaMemcpyAsync(h->d_gofs, gofs.data(), sizeof(int) * gofs.size(), cudaMemcpyHostToDevice, s));
    TG_CK(cudaMemcpyAsync(h->d_pgeo, L.geo.data(), sizeof(PatchGeo) * L.geo.size(), cudaMemcpyHostToDevice, s));
    h->dense = dense_inverses_needed(h, L.off);
    if (h->dense) {
      TG_CK(cudaMalloc(&h->pinv, std::max<size_t>(1, (size_t)L.off * ts_size(h->opt.precision))));
      if (h->opt.precision == TG_PREC_F16 && dalloc(&h->rscale, (size_t)h->ngroups * kRowsPerGroup))
        return TG_ERR_OOM;
    }
    // band factors for the band smoother: FP64 handles in FP64, the others in FP32
    h->band.ldb = wmax + 1;   // stored row width: the widest band plus the reciprocal diagonal
    if (h->band.ldb > kBandLd) return TG_ERR_UNSUPPORTED;
    h->band.stride = 2LL * band_rows(nmax) * h->band.ldb;   // column and row layouts
    const size_t esz = (h->opt.precision == TG_PREC_F64) ? sizeof(double) : sizeof(float);
    TG_CK(cudaMalloc(&h->pband, std::max<size_t>(1, (size_t)h->npatch * h->band.stride * esz)));
    h->band.p = h->pband;
    // 2-byte storage: the same inverses in the tensor-core tile layout
    if (h->dense && (h->opt.precision == TG_PREC_BF16 || h->opt.precision == TG_PREC_F16)) {
      TG_CK(cudaMalloc(&h->ptiles, std::max<size_t>(1, (size_t)L.toff * 2)));
      if (dalloc(&h->d_tofs, L.tofs.size())) return TG_ERR_OOM;
      TG_CK(cudaMemcpyAsync(h->d_tofs, L.tofs.data(), sizeof(int) * L.tofs.size(), cudaMemcpyHostToDevice, s));
      h->band.tp = h->ptiles;
      h->band.tofs = h->d_tofs;
      h->band.ntiles = L.tofs.back();
    }
  }
  // the patches to factor, as a compact list: rectangles, layouts, numbers
  const std::vector<int> ids = selected(h->npatch, update ? changed : nullptr);
  const int cnt = (int)ids.size();
  h->refactored_patches = cnt;
  if (cnt == 0) return TG_OK;
  std::vector<int4> crect(cnt);
  std::vector<PatchGeo> cgeo(cnt);
  for (int c = 0; c < cnt; ++c) {
    crect[c] = L.rect[ids[c]];
    cgeo[c] = L.geo[ids[c]];
  }
  int4* d_rect = nullptr;
  PatchGeo* d_geo = nullptr;
  int* d_ids = nullptr;
  double *band = nullptr, *inv = nullptr;
  const int batch = std::max(1, std::min(cnt, (int)((256LL << 20) / (8LL * nmax * nmax))));
  int rc = (scratch(h, kScrRect, cnt, &d_rect) || scratch(h, kScrGeo, cnt, &d_geo) ||
            scratch(h, kScrIds, cnt, &d_ids) || scratch(h, kScrBand, (size_t)cnt * nmax * (wmax + 1), &band) ||
            (h->dense && scratch(h, kScrInv, (size_t)batch * nmax * nmax, &inv)))
               ? TG_ERR_OOM : TG_OK;
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_rect, crect.data(), sizeof(int4) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_geo, cgeo.data(), sizeof(PatchGeo) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) {
    launch_assemble_band(h->kinv, d_rect, band, cnt, wmax, nmax, n, s);
    launch_band_cholesky(band, d_rect, cnt, wmax, nmax, h->d_status, s);
    if (h->opt.precision == TG_PREC_F64)
      launch_store_band<double>(band, d_rect, d_ids, cnt, wmax, nmax, h->band.stride, (double*)h->pband, s);
    else
      launch_store_band<float>(band, d_rect, d_ids, cnt, wmax, nmax, h->band.stride, (float*)h->pband, s);
    for (int first = 0; h->dense && first < cnt; first += batch) {
      const int m = std::min(batch, cnt - first);
      launch_band_inverse(band, d_rect, first, m, wmax, nmax, inv, s);
      if (h->opt.precision == TG_PREC_F64)
        launch_store_inverse<double>(inv, d_geo, first, m, nmax, (double*)h->pinv, s);
      else if (h->opt.precision == TG_PREC_F32)
        launch_store_inverse<float>(inv, d_geo, first, m, nmax, (float*)h->pinv, s);
      else if (h->opt.precision == TG_PREC_F16) {
        launch_store_inverse_f16(inv, d_geo, h->d_gofs, first, m, nmax, (__half*)h->pinv, h->rscale, s, d_ids);
        launch_store_inverse_tiles<__half>(inv, d_geo, h->d_gofs, d_ids, first, m, nmax, (__half*)h->ptiles,
                                           h->rscale, s);
      } else {
        launch_store_inverse<__nv_bfloat16>(inv, d_geo, first, m, nmax, (__nv_bfloat16*)h->pinv, s);
        launch_store_inverse_tiles<__nv_bfloat16>(inv, d_geo, h->d_gofs, d_ids, first, m, nmax,
                                                  (__nv_bfloat16*)h->ptiles, nullptr, s);
      }
    }
    rc = cuda_err(cudaStreamSynchronize(s));
  }
  if (rc) return rc;
  return cuda_err(cudaGetLastError());
}

// coarse blocks: band Cholesky factors of the local operators (snapshots) and,
// with inverses, their dense inverses (preprocessing).  update: the storage
// exists and only the blocks in `changed` (NULL: all) are factored again
int setup_blocks(tg_handle* h, bool inverses, bool update = false,
                 const std::vector<unsigned char>* changed = nullptr) {
  const int b = h->b, n = h->n;
  cudaStream_t s = h->stream;
  const std::vector<int4> brect = block_rects(h);
  const int bw = b, bn = (b - 1) * (b - 1);
  std::vector<PatchGeo> bgeo(h->nblocks);
  std::vector<int> bgofs(h->nblocks + 1, 0);
  long long boff = 0;
  for (int k = 0; k < h->nblocks; ++k) {
    PatchGeo g{};
    g.x0 = brect[k].x; g.y0 = brect[k].y; g.nx = g.ny = b - 1;
    g.nloc = bn;
    g.ld = ((bn + 7) / 8) * 8;
    g.off = boff;
    boff += (long long)g.nloc * g.ld;
    bgeo[k] = g;
    bgofs[k + 1] = bgofs[k] + (bn + kRowsPerGroup - 1) / kRowsPerGroup;
  }
  const bool f64 = (h->opt.precision == TG_PREC_F64);
  if (!update) {
    if (dalloc(&h->blk_band, (size_t)h->nblocks * std::max(bn, 1) * (bw + 1))) return TG_ERR_OOM;
    if (inverses) {
      h->bgroups = bgofs[h->nblocks];
      if (dalloc(&h->d_bgeo, bgeo.size()) || dalloc(&h->d_bgofs, bgofs.size()) ||
          (f64 ? dalloc(&h->binv, (size_t)boff) : dalloc(&h->binv32, (size_t)boff)))
        return TG_ERR_OOM;
      TG_CK(cudaMemcpyAsync(h->d_bgeo, bgeo.data(), sizeof(PatchGeo) * bgeo.size(), cudaMemcpyHostToDevice, s));
      TG_CK(cudaMemcpyAsync(h->d_bgofs, bgofs.data(), sizeof(int) * bgofs.size(), cudaMemcpyHostToDevice, s));
    }
  }
  // the blocks to factor, as a compact list; their bands stay in the full
  // numbering (the snapshot solves read them), so the kernels get the slots
  const std::vector<int> ids = selected(h->nblocks, update ? changed : nullptr);
  const int cnt = (int)ids.size();
  h->refactored_blocks = cnt;
  if (cnt == 0 || bn == 0) return cuda_err(cudaStreamSynchronize(s));
  std::vector<int4> crect(cnt);
  std::vector<PatchGeo> cgeo(cnt);
  for (int c = 0; c < cnt; ++c) {
    crect[c] = brect[ids[c]];
    cgeo[c] = bgeo[ids[c]];
  }
  int4* d_rect = nullptr;
  PatchGeo* d_geo = nullptr;
  int* d_ids = nullptr;
  double* bscratch = nullptr;
  const int bbatch = std::max(1, std::min(cnt, (int)((256LL << 20) / (8LL * bn * bn))));
  int rc = (scratch(h, kScrRect, cnt, &d_rect) || scratch(h, kScrGeo, cnt, &d_geo) || scratch(h, kScrIds, cnt, &d_ids) ||
            (inverses && scratch(h, kScrInv, (size_t)bbatch * bn * bn, &bscratch)))
               ? TG_ERR_OOM : TG_OK;
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_rect, crect.data(), sizeof(int4) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_geo, cgeo.data(), sizeof(PatchGeo) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
  if (!rc) {
    launch_assemble_band(h->kinv, d_rect, h->blk_band, cnt, bw, bn, n, s, d_ids);
    launch_band_cholesky(h->blk_band, d_rect, cnt, bw, bn, h->d_status, s, d_ids);
    if (inverses) {
      // dense inverses of the block operators, smoother layout
      for (int first = 0; first < cnt; first += bbatch) {
        const int m = std::min(bbatch, cnt - first);
        launch_band_inverse(h->blk_band, d_rect, first, m, bw, bn, bscratch, s, d_ids);
        if (f64) launch_store_inverse<double>(bscratch, d_geo, first, m, bn, h->binv, s);
        else launch_store_inverse<float>(bscratch, d_geo, first, m, bn, h->binv32, s);
      }
    }
    rc = cuda_err(cudaStreamSynchronize(s));
  }
  return rc;
}

// buffers of the per-face spectral problems (Section 4)
struct SpectralBufs {
  double *psiS = nullptr, *gram = nullptr, *fcoef = nullptr, *zcoef = nullptr;
  int *d_nsel = nullptr, *d_jeff = nullptr;
};

void free_spectral(SpectralBufs& sb) {
  cudaFree(sb.psiS);
  cudaFree(sb.gram);
  cudaFree(sb.fcoef);
  cudaFree(sb.zcoef);
  cudaFree(sb.d_nsel);
  cudaFree(sb.d_jeff);
  sb = SpectralBufs{};
}

int alloc_spectral(tg_handle* h, SpectralBufs& sb) {
  const int b = h->b, F = h->nfaces;
  if (!h->lam && dalloc(&h->lam, (size_t)F * b)) return TG_ERR_OOM;
  if (dalloc(&sb.psiS, (size_t)h->nblocks * 4 * b * (b + 1) * (b + 1)) ||
      dalloc(&sb.gram, (size_t)h->nblocks * 4 * b * b) || dalloc(&sb.d_nsel, F) || dalloc(&sb.d_jeff, F) ||
      dalloc(&sb.fcoef, (size_t)F * b) || dalloc(&sb.zcoef, (size_t)F * (b - 1) * b))
    return TG_ERR_OOM;
  TG_CK(cudaMemsetAsync(sb.zcoef, 0, sizeof(double) * (size_t)F * (b - 1) * b, h->stream));
  TG_CK(cudaMemsetAsync(sb.fcoef, 0, sizeof(double) * (size_t)F * b, h->stream));
  return TG_OK;
}

SpectralArgs spectral_args(tg_handle* h, SpectralBufs& sb) {
  SpectralArgs A;
  A.kinv = h->kinv;
  A.gram = sb.gram;
  A.eig_tol = h->eig_tol;
  A.max_basis = h->opt.max_basis;
  A.mode = (h->opt.coarse_space == TG_COARSE_MSFEM) ? 1 : 0;
  A.n = h->n;
  A.b = h->b;
  A.lam = h->lam;
  A.nsel = sb.d_nsel;
  A.fcoef = sb.fcoef;
  A.zcoef = sb.zcoef;
  A.status = h->d_status;
  A.jeff = sb.d_jeff;
  return A;
}

// exact snapshot spaces and spectral problems (all faces, or the masked ones)
void spectral_exact(tg_handle* h, SpectralBufs& sb, const unsigned char* smask, const unsigned char* fmask,
                    float* labels, int klab) {
  launch_snapshots(h->kinv, h->blk_band, nullptr, h->b, smask, sb.psiS, sb.gram, h->n, h->b, h->stream);
  SpectralArgs A = spectral_args(h, sb);
  A.fmask = fmask;
  A.labels = labels;
  A.klab = klab;
  launch_face_spectral(A, h->nfaces, h->stream);
}

// learned space: predicted profiles -> Rayleigh-Ritz on their span; faces whose
// smallest Ritz value is >= eig_tol take the exact problem
int spectral_learned(tg_handle* h, const double* kd, SpectralBufs& sb) {
  const int F = h->nfaces, b = h->b, n = h->n;
  cudaStream_t s = h->stream;
  int k = h->opt.learned_k;
  const float* Y = h->opt.face_profiles;
  float* ybuf = nullptr;
  __nv_bfloat16 *x = nullptr, *h1 = nullptr, *h2 = nullptr;
  double *prof = nullptr, *ccoef = nullptr;
  int *jpred = nullptr, *fb = nullptr;
  unsigned char *fmask = nullptr, *smask = nullptr;
  int rc = TG_OK;
  if (!Y) {
    int nb = 0, hid = 0, din = 0, dout = 0;
    mlp_dims(h->opt.net, &nb, &k, &hid, &din, &dout);
    if (nb != b) return TG_ERR_INVALID_ARG;
    if (dalloc(&x, (size_t)F * din) || dalloc(&h1, (size_t)F * hid) || dalloc(&h2, (size_t)F * hid) ||
        dalloc(&ybuf, (size_t)F * dout))
      rc = TG_ERR_OOM;
    if (!rc) {
      launch_face_inputs(kd, n, b, x, s);
      rc = mlp_forward(h->opt.net, F, x, ybuf, h1, h2, s);
      Y = ybuf;
    }
  }
  if (!rc && (dalloc(&prof, (size_t)F * k * b) || dalloc(&ccoef, (size_t)F * k * b) || dalloc(&jpred, F) ||
              dalloc(&fb, F) || dalloc(&fmask, F) || dalloc(&smask, (size_t)h->nblocks * 4)))
    rc = TG_ERR_OOM;
  std::vector<int> hfb(F, 0);
  if (!rc) {
    cudaMemsetAsync(fb, 0, sizeof(int) * F, s);
    launch_pred_basis(Y, h->kinv, k, n, b, 0.25, prof, ccoef, jpred, F, s);
    launch_snapshots(h->kinv, h->blk_band, ccoef, k, nullptr, sb.psiS, sb.gram, n, b, s);
    SpectralArgs A = spectral_args(h, sb);
    A.prof = prof;
    A.ccoef = ccoef;
    A.jpred = jpred;
    A.kmax = k;
    A.fallback = fb;
    launch_face_spectral(A, F, s);
    rc = cuda_err(cudaMemcpyAsync(hfb.data(), fb, sizeof(int) * F, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
    if (!rc && read_and_clear_gemm_timeout()) rc = TG_ERR_DEVICE_TIMEOUT;   // the network's GEMMs
  }
  int nfb = 0;
  for (int v : hfb) nfb += v;
  h->fallback_faces = nfb;
  h->snapshot_solves = 2 * F * k + 2 * nfb * b;
  if (!rc && nfb > 0) {
    const int nc = h->nc, nV = nc * (nc - 1);
    std::vector<unsigned char> hf(F, 0), hs((size_t)h->nblocks * 4, 0);
    for (int f = 0; f < F; ++f) {
      if (!hfb[f]) continue;
      hf[f] = 1;
      if (f < nV) {
        const int I = f % (nc - 1) + 1, J = f / (nc - 1);
        hs[(size_t)(J * nc + I - 1) * 4 + 1] = 1;
        hs[(size_t)(J * nc + I) * 4 + 0] = 1;
      } else {
        const int I = (f - nV) % nc, J = (f - nV) / nc + 1;
        hs[(size_t)((J - 1) * nc + I) * 4 + 3] = 1;
        hs[(size_t)(J * nc + I) * 4 + 2] = 1;
      }
    }
    rc = cuda_err(cudaMemcpyAsync(fmask, hf.data(), F, cudaMemcpyHostToDevice, s));
    if (!rc) rc = cuda_err(cudaMemcpyAsync(smask, hs.data(), hs.size(), cudaMemcpyHostToDevice, s));
    if (!rc) {
      spectral_exact(h, sb, smask, fmask, nullptr, 0);
      rc = cuda_err(cudaStreamSynchronize(s));
    }
  }
  cudaFree(ybuf); cudaFree(x); cudaFree(h1); cudaFree(h2);
  cudaFree(prof); cudaFree(ccoef); cudaFree(jpred); cudaFree(fb); cudaFree(fmask); cudaFree(smask);
  if (rc) return rc;
  return cuda_err(cudaGetLastError());
}

int read_spectral(tg_handle* h, SpectralBufs& sb) {
  cudaStream_t s = h->stream;
  TG_CK(cudaMemcpyAsync(h->nsel.data(), sb.d_nsel, sizeof(int) * h->nfaces, cudaMemcpyDeviceToHost, s));
  h->lam_h.resize((size_t)h->nfaces * h->b);
  TG_CK(cudaMemcpyAsync(h->lam_h.data(), h->lam, sizeof(double) * h->lam_h.size(), cudaMemcpyDeviceToHost, s));
  int st = 0;
  int rc = read_status(h, &st);
  if (rc) return rc;
  if (st) return status_to_err(st);
  h->velocity_basis = 0;
  for (int v : h->nsel) h->velocity_basis += v;
  return TG_OK;
}

// preconditioner coarse space from the spectral data (or RT0)
int setup_coarse(tg_handle* h, SpectralBufs& sb) {
  const bool rt_mode = (h->opt.coarse_space == TG_COARSE_RT0);
  int rc = build_space(h, h->cs, h->nsel, rt_mode);
  if (!rc) rc = finish_space(h, h->cs, sb.psiS, sb.fcoef, sb.zcoef, sb.d_jeff, rt_mode);
  return rc;
}

// Smoother autotuner: times every tile shape on this handle's own patch
// inverses (one warm-up and five timed launches each, CUDA events on the
// handle's stream, scratch vectors of its own) and keeps the fastest.  When
// that is a band form, the two band forms are compared again from an
// evicted L2, as they run in a solve.
constexpr size_t kAutotuneFlushBytes = 256ull << 20;   // twice the 129 MB L2
template <typename TC, typename TS>
int autotune_smoother_t(tg_handle* h) {
  const long long nn = (long long)h->n * h->n;
  cudaStream_t s = h->stream;
  TC *rin = nullptr, *z = nullptr;
  if (dalloc(&rin, nn) || dalloc(&z, nn)) {
    cudaFree(rin);
    return TG_ERR_OOM;
  }
  // L2 eviction buffer for the band candidates (absent without band factors)
  float band_cold[2] = {0.0f, 0.0f};   // shapes kShapeBand, kShapeBandRing, from an evicted L2
  unsigned char* flush = nullptr;
  if (h->band.p && cudaMalloc(&flush, kAutotuneFlushBytes) != cudaSuccess) {
    cudaGetLastError();   // no eviction buffer: the band candidates are timed warm
    flush = nullptr;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_err(cudaEventCreate(&e0));
  if (!rc) rc = cuda_err(cudaEventCreate(&e1));
  if (!rc) rc = cuda_err(cudaMemsetAsync(rin, 0, sizeof(TC) * nn, s));
  if (!rc) rc = cuda_err(cudaMemsetAsync(z, 0, sizeof(TC) * nn, s));
  const bool f64 = std::is_same<TS, double>::value, f16 = std::is_same<TS, __half>::value;
  const bool bf16 = std::is_same<TS, __nv_bfloat16>::value;
  const int cand_bf16[] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9}, cand_f32[] = {0, 1, 2, 3, 4, 5, 6, 7, 9},
            cand_f64[] = {0, 4, 7}, cand_f16[] = {0, 1, 2, 3, 5, 6, 7, 8, 9};
  // FP16: no TMA ring; the tensor-core tiles exist for 2-byte storage only;
  // FP64 factors have one band form
  const int cand_band[] = {7, 9};   // handles without dense inverses (dense_inverses_needed)
  const int* cand = !h->dense ? cand_band : f64 ? cand_f64 : f16 ? cand_f16 : bf16 ? cand_bf16 : cand_f32;
  const int ncand = !h->dense ? 2 : f64 ? 3 : f16 ? 9 : bf16 ? 10 : 9;
  float best = 1e30f;
  int best_shape = 0;
  for (int i = 0; i < ncand && !rc; ++i) {
    const int shape = cand[i];
    auto go = [&]() {
      // the band form runs from a separately formed residual: time that launch with it
      if (is_band_shape(shape))
        launch_residual<TC>(h->kinv, z, (const TC*)(std::is_same<TC, double>::value ? (const void*)h->kinv
                                                                                     : (const void*)h->kinv32),
                            rin, h->n, nullptr, s);
      launch_smoother<TC, TS, TC>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, (const TS*)h->pinv, rin, z,
                                  h->opt.eta, h->n, nullptr, s, shape, h->rscale, h->band);
    };
    go();
    float ms = 0.0f;
    cudaEventRecord(e0, s);
    for (int k = 0; k < 5; ++k) go();
    cudaEventRecord(e1, s);
    rc = cuda_err(cudaEventSynchronize(e1));
    if (!rc) rc = cuda_err(cudaGetLastError());
    if (!rc) cudaEventElapsedTime(&ms, e0, e1);
    h->shape_us[shape] = ms * 1000.0f / 5.0f;
    if (is_band_shape(shape) && flush && !rc) {
      // the two band forms differ only in how far they read ahead, which
      // matters where the factors stream from HBM, as they do in a solve (the
      // iteration's other kernels pass through L2 between two sweeps): they
      // are also timed each from an evicted L2
      float cold = 0.0f;
      for (int k = 0; k < 5 && !rc; ++k) {
        cudaMemsetAsync(flush, 0, kAutotuneFlushBytes, s);
        cudaEventRecord(e0, s);
        go();
        cudaEventRecord(e1, s);
        rc = cuda_err(cudaEventSynchronize(e1));
        float one = 0.0f;
        if (!rc) cudaEventElapsedTime(&one, e0, e1);
        cold += one;
      }
      if (!rc) rc = cuda_err(cudaGetLastError());
      band_cold[shape == kShapeBand ? 0 : 1] = cold * 1000.0f / 5.0f;
    }
    if (!rc && h->shape_us[shape] < best) {
      best = h->shape_us[shape];
      best_shape = shape;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(rin);
  cudaFree(z);
  cudaFree(flush);
  // dense against band on the warm times; between the two band forms, the
  // one faster from an evicted L2
  if (!rc && is_band_shape(best_shape) && band_cold[0] > 0.0f && band_cold[1] > 0.0f)
    best_shape = band_cold[1] < band_cold[0] ? kShapeBandRing : kShapeBand;
  if (!rc) h->shape = best_shape;
  return rc;
}

int choose_smoother_shape(tg_handle* h) {
  if (h->opt.smoother_shape >= 0) {
    h->shape = h->opt.smoother_shape;
    if (h->opt.precision == TG_PREC_F16 && h->shape == 4) h->shape = 0;   // no TMA ring for FP16
    if (h->shape == kShapeTensor && !h->ptiles) h->shape = 0;            // tiles exist for 2-byte storage only
    if (h->shape == kShapeBandRing && h->opt.precision == TG_PREC_F64) h->shape = kShapeBand;   // FP64 factors
    return TG_OK;
  }
  if (h->opt.precision == TG_PREC_F64) return autotune_smoother_t<double, double>(h);
  if (h->opt.precision == TG_PREC_F32) return autotune_smoother_t<float, float>(h);
  if (h->opt.precision == TG_PREC_F16) return autotune_smoother_t<float, __half>(h);
  return autotune_smoother_t<float, __nv_bfloat16>(h);
}

int setup_impl(tg_handle* h, const double* kappa) {
  const long long nn = (long long)h->n * h->n;
  cudaStream_t s = h->stream;
  const double* kd = kappa;
  double* kcopy = nullptr;
  struct Guard {
    double*& p;
    ~Guard() { cudaFree(p); }
  } guard{kcopy};
  if (h->opt.pointer_mode == TG_PTR_HOST) {
    if (dalloc(&kcopy, nn)) return TG_ERR_OOM;
    TG_CK(cudaMemcpyAsync(kcopy, kappa, sizeof(double) * nn, cudaMemcpyHostToDevice, s));
    kd = kcopy;
  }
  int rc = setup_kappa(h, kd);
  if (!rc) rc = setup_patches(h);
  if (!rc) rc = setup_blocks(h, true);
  if (rc) return rc;

  // ---- snapshot spaces and local spectral problems (Section 4) ----
  h->nsel.assign(h->nfaces, 1);
  SpectralBufs sb{};
  if (h->nfaces > 0 && h->opt.coarse_space != TG_COARSE_RT0) {
    rc = alloc_spectral(h, sb);
    if (!rc) {
      if (h->opt.coarse_space == TG_COARSE_LEARNED) {
        rc = spectral_learned(h, kd, sb);
      } else {
        spectral_exact(h, sb, nullptr, nullptr, nullptr, 0);
        h->snapshot_solves = 2 * h->nfaces * h->b;
      }
    }
    if (!rc) rc = read_spectral(h, sb);
  } else {
    h->velocity_basis = h->nfaces;
  }
  // ---- coarse spaces: preconditioner (GMsFEM / MsFEM / RT0 / learned) and RT0 ----
  if (!rc) rc = setup_coarse(h, sb);
  free_spectral(sb);
  if (rc) return rc;
  std::vector<int> ones(h->nfaces, 1);
  if ((rc = build_space(h, h->rt, ones, true))) return rc;
  if ((rc = finish_space(h, h->rt, nullptr, nullptr, nullptr, nullptr, true))) return rc;
  int st = 0;
  if ((rc = read_status(h, &st))) return rc;
  if (st) return status_to_err(st);

  configure_kernels(std::max(h->cs.D, h->rt.D));
  if (configure_rt_particular(h->nc, h->nblocks)) return TG_ERR_UNSUPPORTED;   // coarse grid beyond one CTA's memory
  if ((rc = choose_smoother_shape(h))) return rc;
  if ((rc = ctx_alloc(h, &h->ctx))) return rc;
  TG_CK(cudaStreamSynchronize(s));
  return cuda_err(cudaGetLastError());
}

// New permeability for an existing handle (time-dependent runs, Section 6.2):
// everything that depends on kappa is recomputed into the handle's existing
// buffers (so instantiated solve graphs stay valid), and the preconditioner's
// coarse space is either kept (coarse == 0: the basis of the first setup,
// with its Galerkin matrix recomputed for the new kappa, as the paper keeps
// the initial multiscale space) or rebuilt by the handle's method (coarse ==
// 1: exact spectral, MsFEM or learned; the solve context is re-created).
int update_kappa_impl(tg_handle* h, const double* kappa, int coarse) {
  const long long nn = (long long)h->n * h->n;
  cudaStream_t s = h->stream;
  const double* kd = kappa;
  double* kcopy = nullptr;
  struct Guard {
    double*& p;
    ~Guard() { cudaFree(p); }
  } guard{kcopy};
  if (h->opt.pointer_mode == TG_PTR_HOST) {
    if (dalloc(&kcopy, nn)) return TG_ERR_OOM;
    TG_CK(cudaMemcpyAsync(kcopy, kappa, sizeof(double) * nn, cudaMemcpyHostToDevice, s));
    kd = kcopy;
  }
  // only patches and blocks with a cell whose 1/kappa changed get new
  // factors: their operators depend on kappa through 1/kappa alone, so the
  // others are bitwise what a fresh setup computes (in two-phase flow most of
  // the domain away from the front keeps its saturation and mobility)
  std::vector<unsigned char> pchg, bchg;
  double* delta = nullptr;   // change of 1/kappa, for the low-rank updates of the coarse inverses
  if (scratch(h, kScrDelta, nn, &delta)) return TG_ERR_OOM;
  launch_kinv_delta(kd, h->kinv, delta, h->n, s);
  int rc = changed_rects(h, kd, patch_layout(h).rect, pchg);
  if (!rc) rc = changed_rects(h, kd, block_rects(h), bchg);
  unsigned char* d_bmask = nullptr;
  if (!rc) rc = scratch(h, kScrBlkMask, bchg.size(), &d_bmask);
  if (!rc) rc = cuda_err(cudaMemcpyAsync(d_bmask, bchg.data(), bchg.size(), cudaMemcpyHostToDevice, s));
  if (!rc) rc = setup_kappa(h, kd, true);
  if (!rc) rc = setup_patches(h, true, &pchg);
  if (!rc) rc = setup_blocks(h, true, true, &bchg);
  if (rc) return rc;
  h->update_rank[0] = h->update_rank[1] = -1;
  const bool rebuild = (coarse == 1 && h->opt.coarse_space != TG_COARSE_RT0 && h->nfaces > 0);
  if (coarse == 2) {
    rc = galerkin_inverse(h, h->cs);
  } else if (!rebuild) {
    rc = galerkin_update(h, h->cs, delta, d_bmask, &h->update_rank[0]);
  } else {
    SpectralBufs sb{};
    rc = alloc_spectral(h, sb);
    if (!rc) {
      if (h->opt.coarse_space == TG_COARSE_LEARNED) {
        rc = spectral_learned(h, kd, sb);
      } else {
        spectral_exact(h, sb, nullptr, nullptr, nullptr, 0);
        h->snapshot_solves = 2 * h->nfaces * h->b;
        h->fallback_faces = 0;
      }
    }
    if (!rc) rc = read_spectral(h, sb);
    if (!rc) {
      free_space(h->cs);
      rc = setup_coarse(h, sb);
    }
    free_spectral(sb);
    if (rc) return rc;
    ctx_free(h->ctx);
    h->ctx = nullptr;
    configure_kernels(std::max(h->cs.D, h->rt.D));
    rc = ctx_alloc(h, &h->ctx);
  }
  if (!rc) rc = (coarse == 2) ? galerkin_inverse(h, h->rt) : galerkin_update(h, h->rt, delta, d_bmask, &h->update_rank[1]);
  if (!rc && h->regraph) {   // the solve graph captured the other coarse solver
    h->regraph = false;
    ctx_free(h->ctx);
    h->ctx = nullptr;
    rc = ctx_alloc(h, &h->ctx);
  }
  if (rc) return rc;
  int st = 0;
  if ((rc = read_status(h, &st))) return rc;
  if (st) return status_to_err(st);
  TG_CK(cudaStreamSynchronize(s));
  return cuda_err(cudaGetLastError());
}

// replaces a learned coarse space by the exact one of Section 4.2 and
// re-creates the default solve context
int rebuild_exact(tg_handle* h) {
  SpectralBufs sb{};
  const int saved = h->opt.coarse_space;
  h->opt.coarse_space = TG_COARSE_GMSFEM;
  int rc = alloc_spectral(h, sb);
  if (!rc) {
    spectral_exact(h, sb, nullptr, nullptr, nullptr, 0);
    rc = read_spectral(h, sb);
  }
  if (!rc) {
    free_space(h->cs);
    rc = setup_coarse(h, sb);
  }
  free_spectral(sb);
  h->opt.coarse_space = saved;
  if (rc) return rc;
  h->snapshot_solves += 2 * h->nfaces * h->b;
  h->fallback_faces = h->nfaces;
  ctx_free(h->ctx);
  h->ctx = nullptr;
  configure_kernels(std::max(h->cs.D, h->rt.D));
  if ((rc = ctx_alloc(h, &h->ctx))) return rc;
  TG_CK(cudaStreamSynchronize(h->stream));
  return cuda_err(cudaGetLastError());
}

template <typename TC, typename TS>
int hook_precond(tg_handle* h, const double* rho, double* z, int which) {
  Ctx* c = h->ctx;
  const int n = h->n;
  const long long nn = (long long)n * n;
  TC* zacc = (TC*)c->zacc;
  TG_CK(cudaMemsetAsync(zacc, 0, sizeof(TC) * nn, h->stream));
  if (which == 0) {
    launch_smoother<TC, TS, double>(h->d_pgeo, h->d_gofs, h->npatch, h->ngroups, (const TS*)h->pinv, rho, zacc,
                                    h->opt.eta, n, nullptr, h->stream, h->shape, h->rscale, h->band);
  } else if (which == 1) {
    if (h->cs.D > 0) {
      TC* rin = (TC*)c->rin;
      if (std::is_same<TC, double>::value)
        TG_CK(cudaMemcpyAsync(rin, rho, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
      else
        launch_convert<double, float>(rho, (float*)rin, nn, h->stream);
      launch_restrict<TC, tile_t<TS>>(h->cs, c->cs_part, h->nblocks, h->nc, h->b, n, rin, nullptr, h->stream);
      launch_coarse_solve(h->cs, c->cs_part, c->cs_coefs, nullptr, h->stream);
      launch_prolong<TC, tile_t<TS>>(h->cs, c->cs_coefs, h->nblocks, h->nc, h->b, n, zacc, nullptr, h->stream);
    }
  } else {
    precondition<TC, TS>(c, rho, zacc, nullptr, h->stream);
  }
  if (std::is_same<TC, double>::value)
    TG_CK(cudaMemcpyAsync(z, zacc, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
  else
    launch_convert<float, double>((const float*)zacc, z, nn, h->stream);
  TG_CK(cudaStreamSynchronize(h->stream));
  TG_CK(cudaGetLastError());
  return read_and_clear_timeout() ? TG_ERR_DEVICE_TIMEOUT : TG_OK;
}

int hook_dispatch(tg_handle* h, const double* rho, double* z, int which) {
  g_pdl = (h->opt.launch_overlap != 0);
  if (!h || !rho || !z) return TG_ERR_INVALID_ARG;
  switch (h->opt.precision) {
    case TG_PREC_F64: return hook_precond<double, double>(h, rho, z, which);
    case TG_PREC_F32: return hook_precond<float, float>(h, rho, z, which);
    case TG_PREC_F16: return hook_precond<float, __half>(h, rho, z, which);
    default: return hook_precond<float, __nv_bfloat16>(h, rho, z, which);
  }
}

// ---- batches ------------------------------------------------------------------
}  // namespace

struct tg_batch {
  std::vector<tg_handle*> handles;   // owned
  std::vector<Ctx*> ctx;             // ninst * nrhs, instance-major (owned)
  int nrhs = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  // device tables: per context the staging buffers and sizes
  double** d_src = nullptr;    // 5 m caller pointers: f, bflux, ux, uy, p
  double** d_buf = nullptr;    // 5 m context buffers: fd, bd, ux, uy, pd
  long long* d_cnt = nullptr;  // 5 m element counts
  double** h_src = nullptr;    // pinned staging of the caller pointers
  double* d_rtol = nullptr;    // shared tolerance; each context's d_rtol is set from it
  double** d_ctx_rtol = nullptr;
  PcgState** d_ctx_state = nullptr;  // PCG state per context
  int* d_out = nullptr;         // 2 m: iter, status
  int* h_out = nullptr;         // pinned
  double* h_rtol = nullptr;     // pinned
};

namespace {

void batch_free(tg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (Ctx* c : b->ctx) ctx_free(c);
  for (tg_handle* h : b->handles) tg_destroy(h);
  void* ptrs[] = {b->d_src, b->d_buf, b->d_cnt, b->d_rtol, b->d_ctx_rtol, b->d_ctx_state, b->d_out};
  for (void* p : ptrs) cudaFree(p);
  if (b->h_src) cudaFreeHost(b->h_src);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->h_rtol) cudaFreeHost(b->h_rtol);
  delete b;
}

}  // namespace

// ============================================================================
extern "C" {

int tg_default_options(tg_options* opt) {
  if (!opt) return TG_ERR_INVALID_ARG;
  opt->eta = 0.2;
  opt->m1 = 1;
  opt->m2 = 1;
  opt->precision = TG_PREC_F64;
  opt->flexible = 0;
  opt->max_iter = 1000;
  opt->pointer_mode = TG_PTR_DEVICE;
  opt->coarse_space = TG_COARSE_GMSFEM;
  opt->max_basis = 0;
  opt->profile = 0;
  opt->net = nullptr;
  opt->face_profiles = nullptr;
  opt->learned_k = 4;
  opt->learned_max_iter = 0;
  opt->smoother_shape = -1;
  opt->launch_overlap = 0;
  opt->cycle = TG_CYCLE_TWO_GRID;
  opt->batch_lockstep = 1;
  opt->batch_nets = nullptr;
  opt->batch_nnets = 0;
  opt->coarse_solver = TG_COARSE_SOLVER_AUTO;
  return TG_OK;
}

int tg_probe_bounded_wait(int complete, int limit_log2, void* stream) {
  if (limit_log2 < 0 || limit_log2 > 22) return TG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  read_and_clear_timeout();   // start from a clear flag
  launch_wait_probe(complete, limit_log2, s);
  int rc = cuda_err(cudaStreamSynchronize(s));
  if (!rc) rc = cuda_err(cudaGetLastError());
  if (rc) return rc;
  return read_and_clear_timeout() ? TG_ERR_DEVICE_TIMEOUT : TG_OK;
}

const char* tg_strerror(int code) {
  switch (code) {
    case TG_OK: return "success";
    case TG_ERR_INVALID_ARG: return "invalid argument (sizes, block size, kappa <= 0 or not finite, NULL)";
    case TG_ERR_INCOMPATIBLE_SOURCE: return "incompatible source: sum of F differs from the net boundary outflow";
    case TG_ERR_BREAKDOWN: return "breakdown: a matrix that must be positive definite is not (PCG or a factor)";
    case TG_ERR_MAXITER: return "PCG did not converge within max_iter";
    case TG_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait expired";
    case TG_ERR_CUDA: return "CUDA runtime error";
    case TG_ERR_OOM: return "device memory allocation failed";
    case TG_ERR_UNSUPPORTED: return "configuration not supported by this build";
    case TG_ERR_DEGENERATE_BASIS: return "a coarse face has no selected function with net flux";
    default: return "unknown error code";
  }
}

int tg_setup(const double* kappa, const tg_grid* grid, double eig_tol, const tg_options* opt, void* stream,
             tg_handle** out) {
  if (!out) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!kappa || !opt) return TG_ERR_INVALID_ARG;
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (!(opt->eta > 0) || opt->m1 < 0 || opt->m2 < 0 || opt->m1 + opt->m2 < 1 || opt->max_iter < 1 ||
      opt->precision < 0 || opt->precision > 3 || opt->coarse_space < 0 || opt->coarse_space > 3 ||
      !(eig_tol > 0) || (opt->pointer_mode != TG_PTR_HOST && opt->pointer_mode != TG_PTR_DEVICE))
    return TG_ERR_INVALID_ARG;
  if (opt->cycle != TG_CYCLE_TWO_GRID && opt->cycle != TG_CYCLE_ADDITIVE) return TG_ERR_INVALID_ARG;
  if (opt->coarse_solver < TG_COARSE_SOLVER_AUTO || opt->coarse_solver > TG_COARSE_SOLVER_ND)
    return TG_ERR_INVALID_ARG;
  if (opt->cycle == TG_CYCLE_TWO_GRID && opt->m1 < 1) return TG_ERR_UNSUPPORTED;
  if (opt->smoother_shape < -1 || opt->smoother_shape >= kSmootherShapes) return TG_ERR_INVALID_ARG;
  if (opt->coarse_space == TG_COARSE_LEARNED) {
    if (!opt->face_profiles && !opt->net) return TG_ERR_INVALID_ARG;
    if (opt->face_profiles && (opt->learned_k < 1 || opt->learned_k > 8)) return TG_ERR_INVALID_ARG;
    if (opt->learned_max_iter < 0) return TG_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TG_ERR_CUDA;
  tg_handle* h = new (std::nothrow) tg_handle();
  if (!h) return TG_ERR_OOM;
  h->n = grid->nx;
  h->b = grid->bx;
  h->nc = h->n / h->b;
  h->ov = grid->overlap;
  h->nblocks = h->nc * h->nc;
  h->npatch = h->nblocks;
  h->nfaces = 2 * h->nc * (h->nc - 1);
  h->h = 1.0 / h->n;
  h->H = (double)h->b / h->n;
  h->eig_tol = eig_tol;
  h->opt = *opt;
  h->stream = (cudaStream_t)stream;
  rc = setup_impl(h, kappa);
  if (rc) {
    tg_destroy(h);
    return rc;
  }
  cudaStreamSynchronize(h->stream);
  scratch_release(h);
  *out = h;
  return TG_OK;
}

}  // extern "C"

namespace {

int solve_impl(tg_handle* h, const double* f, const double* bflux, double rtol, const double* ux0, double* ux,
               double* uy, double* p, int* iters, tg_report* rep) {
  g_pdl = (h->opt.launch_overlap != 0);
  Ctx* c = h->ctx;
  const int n = h->n;
  const long long nn = (long long)n * n, nf = (long long)(n + 1) * n;
  cudaStream_t s = h->stream;
  const cudaMemcpyKind in = (h->opt.pointer_mode == TG_PTR_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind out = (h->opt.pointer_mode == TG_PTR_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  // stage inputs into context buffers (the instantiated graph only references those)
  TG_CK(cudaMemcpyAsync(c->fd, f, sizeof(double) * nn, in, s));
  if (bflux) TG_CK(cudaMemcpyAsync(c->bd, bflux, sizeof(double) * 4 * n, in, s));
  else TG_CK(cudaMemsetAsync(c->bd, 0, sizeof(double) * 4 * n, s));
  c->warm = (ux0 != nullptr);
  if (c->warm) {
    if (!c->ux0 && dalloc(&c->ux0, (size_t)nf)) return TG_ERR_OOM;
    TG_CK(cudaMemcpyAsync(c->ux0, ux0, sizeof(double) * nf, in, s));
  }
  *c->h_rtol = rtol;
  TG_CK(cudaMemcpyAsync(c->d_rtol, c->h_rtol, sizeof(double), cudaMemcpyHostToDevice, s));
  unsigned long long launches = 0;
  int rc = TG_OK;
  cudaEventRecord(c->ev[0], s);
  if (h->opt.profile) {
    c->prof_used = 0;
    c->prof_op_used = 0;
    rc = run_loop(c, &launches);
  } else {
    cudaGraphExec_t& ex = c->warm ? c->exec_warm : c->exec;
    if (!ex) {
      cudaGraph_t g = nullptr;
      TG_CK(cudaGraphCreate(&g, 0));
      rc = add_chain(c, g, c->cap);
      if (!rc) rc = cuda_err(cudaGraphInstantiate(&ex, g, 0));
      cudaGraphDestroy(g);
      if (rc) return rc;
    }
    TG_CK(cudaGraphLaunch(ex, s));
  }
  cudaEventRecord(c->ev[3], s);
  if (rc) return rc;
  TG_CK(cudaMemcpyAsync(ux, c->ux, sizeof(double) * nf, out, s));
  TG_CK(cudaMemcpyAsync(uy, c->uy, sizeof(double) * nf, out, s));
  TG_CK(cudaMemcpyAsync(p, c->pd, sizeof(double) * nn, out, s));
  PcgState* full = new (std::nothrow) PcgState();
  if (!full) return TG_ERR_OOM;
  double diverr = 0.0;
  rc = cuda_err(cudaMemcpyAsync(full, c->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_err(cudaMemcpyAsync(&diverr, c->diverr, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!rc) rc = cuda_err(cudaStreamSynchronize(s));
  if (!rc) rc = cuda_err(cudaGetLastError());
  if (rc) {
    delete full;
    return rc;
  }
  if (!h->opt.profile) {
    // the while node ran the two-iteration body once per pair of iterations
    const unsigned long long passes = (unsigned long long)std::max((full->iter + 1) / 2, 1);
    launches = (c->warm ? c->k_prefix_warm : c->k_prefix) + passes * c->k_body + c->k_epi;
  }
  if (iters) *iters = full->iter;
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->iters = full->iter;
    rep->rel_residual = (full->rr0 > 0) ? std::sqrt(full->rr / full->rr0) : 0.0;
    rep->converged = (full->rr <= full->rtol2 * full->rr0) ? 1 : 0;
    rep->cond_estimate = lanczos_cond(*full);
    rep->velocity_basis = h->velocity_basis;
    rep->coarse_dim = h->velocity_basis + h->nc * h->nc + 1;
    rep->coarse_unknowns = h->cs.D;
    rep->max_div_error = diverr;
    rep->kernel_launches = (int)launches;
    rep->graph = h->opt.profile ? 0 : 1;
    rep->snapshot_solves = h->snapshot_solves;
    rep->fallback_faces = h->fallback_faces;
    rep->smoother_shape = h->shape;
    for (int k = 0; k < kSmootherShapes; ++k) rep->shape_us[k] = h->shape_us[k];
    rep->refactored_patches = h->refactored_patches;
    rep->refactored_blocks = h->refactored_blocks;
    rep->update_rank[0] = h->update_rank[0];
    rep->update_rank[1] = h->update_rank[1];
    rep->coarse_solver = h->cs.solver == 2 ? TG_COARSE_SOLVER_ND : TG_COARSE_SOLVER_DENSE;
    rep->coarse_solve_mb = (h->cs.solver == 2 ? h->cs.nd.bytes : 8.0 * (double)h->cs.D * h->cs.D) * 1e-6;
    float ms = 0;
    if (h->opt.profile) {
      cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
      rep->preprocess_ms = ms;
      cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]);
      rep->pcg_ms = ms;
      cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
      rep->epilogue_ms = ms;
      double sm = 0.0;
      for (int k = 0; k + 1 < c->prof_used; k += 2) {
        cudaEventElapsedTime(&ms, c->prof_ev[k], c->prof_ev[k + 1]);
        sm += ms;
      }
      rep->smoother_ms = sm;
      rep->smoother_launches = c->prof_used / 2;
      double om = 0.0;
      for (int k = 0; k + 1 < c->prof_op_used; k += 2) {
        cudaEventElapsedTime(&ms, c->prof_op_ev[k], c->prof_op_ev[k + 1]);
        om += ms;
      }
      rep->operator_ms = om;
      rep->operator_launches = c->prof_op_used / 2;
    } else {
      cudaEventElapsedTime(&ms, c->ev[0], c->ev[3]);
      rep->pcg_ms = ms;  // whole graph
    }
  }
  int status = full->status;
  delete full;
  if (read_and_clear_timeout()) status |= kStTimeout;
  return status_to_err(status);
}

int solve_entry(tg_handle* h, const double* f, const double* bflux, double rtol, const double* ux0, double* ux,
                double* uy, double* p, int* iters, tg_report* rep) {
  if (!h || !f || !ux || !uy || !p || !(rtol > 0) || !(rtol < 1)) return TG_ERR_INVALID_ARG;
  int it = 0;
  int rc = solve_impl(h, f, bflux, rtol, ux0, ux, uy, p, &it, rep);
  int refit = 0;
  if ((rc == TG_OK || rc == TG_ERR_MAXITER) && h->opt.coarse_space == TG_COARSE_LEARNED &&
      h->opt.learned_max_iter > 0 && it > h->opt.learned_max_iter && h->fallback_faces < h->nfaces) {
    // the learned space needed too many iterations: exact space, solve again
    int rb = rebuild_exact(h);
    if (rb) return rb;
    rc = solve_impl(h, f, bflux, rtol, ux0, ux, uy, p, &it, rep);
    refit = 1;
  }
  if (iters) *iters = it;
  if (rep) rep->learned_fallback = refit;
  return rc;
}

}  // namespace

extern "C" {

int tg_solve(tg_handle* h, const double* f, const double* bflux, double rtol, double* ux, double* uy, double* p,
             int* iters, tg_report* rep) {
  return solve_entry(h, f, bflux, rtol, nullptr, ux, uy, p, iters, rep);
}

int tg_solve_warm(tg_handle* h, const double* f, const double* bflux, double rtol, const double* ux0,
                  const double* uy0, double* ux, double* uy, double* p, int* iters, tg_report* rep) {
  (void)uy0;   // the x-face velocities determine the guess's stream function
  if (!ux0) return TG_ERR_INVALID_ARG;
  return solve_entry(h, f, bflux, rtol, ux0, ux, uy, p, iters, rep);
}

int tg_update_kappa(tg_handle* h, const double* kappa, int coarse) {
  if (!h || !kappa || coarse < 0 || coarse > 2) return TG_ERR_INVALID_ARG;
  return update_kappa_impl(h, kappa, coarse);
}

void tg_destroy(tg_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  ctx_free(h->ctx);
  void* ptrs[] = {h->kinv, h->kinv32, h->d_status, h->d_pgeo, h->d_gofs, h->pinv, h->pband, h->ptiles, h->d_tofs,
                  h->rscale, h->blk_band, h->lam, h->d_bgeo, h->d_bgofs, h->binv, h->binv32, h->kcoef};
  for (void* ptr : ptrs) cudaFree(ptr);
  free_space(h->cs);
  free_space(h->rt);
  scratch_release(h);
  if (h->h_flag) cudaFreeHost(h->h_flag);
  delete h;
}

int tg_apply_operator(tg_handle* h, const double* psi, double* out, int precision) {
  if (!h || !psi || !out || precision < 0 || precision > 1) return TG_ERR_INVALID_ARG;
  if (precision == 0) launch_apply_operator(psi, h->kinv, out, h->n, h->stream);
  else launch_apply_operator_f32(psi, h->kinv32, out, h->n, h->stream);
  TG_CK(cudaStreamSynchronize(h->stream));
  return cuda_err(cudaGetLastError());
}

int tg_apply_smoother(tg_handle* h, const double* rho, double* z) { return hook_dispatch(h, rho, z, 0); }
int tg_apply_coarse(tg_handle* h, const double* rho, double* z) { return hook_dispatch(h, rho, z, 1); }
int tg_apply_preconditioner(tg_handle* h, const double* rho, double* z) { return hook_dispatch(h, rho, z, 2); }

int tg_coarse_info(tg_handle* h, int* nfaces, int* velocity_basis, int* nsel, double* lambda) {
  if (!h) return TG_ERR_INVALID_ARG;
  if (nfaces) *nfaces = h->nfaces;
  if (velocity_basis) *velocity_basis = h->velocity_basis;
  if (nsel) std::memcpy(nsel, h->nsel.data(), sizeof(int) * h->nsel.size());
  if (lambda && !h->lam_h.empty()) std::memcpy(lambda, h->lam_h.data(), sizeof(double) * h->lam_h.size());
  return TG_OK;
}

int tg_preprocess(tg_handle* h, const double* f, const double* bflux, double* ux, double* uy) {
  if (!h || !f || !ux || !uy) return TG_ERR_INVALID_ARG;
  g_pdl = (h->opt.launch_overlap != 0);
  Ctx* c = h->ctx;
  const int n = h->n;
  const long long nn = (long long)n * n, nf = (long long)(n + 1) * n;
  cudaStream_t s = h->stream;
  TG_CK(cudaMemcpyAsync(c->fd, f, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (bflux) TG_CK(cudaMemcpyAsync(c->bd, bflux, sizeof(double) * 4 * n, cudaMemcpyDeviceToDevice, s));
  else TG_CK(cudaMemsetAsync(c->bd, 0, sizeof(double) * 4 * n, s));
  *c->h_rtol = 0.5;
  TG_CK(cudaMemcpyAsync(c->d_rtol, c->h_rtol, sizeof(double), cudaMemcpyHostToDevice, s));
  launch_pcg_reset(c->st, c->d_rtol, 1, 0, s);
  enqueue_preprocess(c, c->fd, c->bd, c->ux, c->uy, s);
  TG_CK(cudaMemcpyAsync(ux, c->ux, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
  TG_CK(cudaMemcpyAsync(uy, c->uy, sizeof(double) * nf, cudaMemcpyDeviceToDevice, s));
  PcgState head{};
  TG_CK(cudaMemcpyAsync(&head, c->st, offsetof(PcgState, alphas), cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  TG_CK(cudaGetLastError());
  if (head.status & kStIncompatible) return TG_ERR_INCOMPATIBLE_SOURCE;
  return TG_OK;
}

int tg_setup_batch(int ninst, const double* const* kappa, const tg_grid* grids, double eig_tol,
                   const tg_options* opt, int nrhs, void* stream, tg_batch** out) {
  if (!out) return TG_ERR_INVALID_ARG;
  *out = nullptr;
  if (ninst < 1 || nrhs < 1 || !kappa || !grids || !opt || opt->pointer_mode != TG_PTR_DEVICE || opt->profile)
    return TG_ERR_INVALID_ARG;
  tg_batch* B = new (std::nothrow) tg_batch();
  if (!B) return TG_ERR_OOM;
  B->nrhs = nrhs;
  B->stream = (cudaStream_t)stream;
  int rc = TG_OK;
  // Instances of one grid size, block size and oversampling have the same
  // patches, hence the same smoother launches: the tile shape the autotuner
  // picks for the first of them is given to the others, which skip the
  // autotuner (and, when it is a band shape, the dense patch inverses).
  struct Tuned {
    int nx, bx, overlap, shape;
  };
  std::vector<Tuned> tuned;
  for (int i = 0; i < ninst && !rc; ++i) {
    tg_handle* h = nullptr;
    tg_options oi = *opt;
    if (opt->smoother_shape < 0)
      for (const Tuned& t : tuned)
        if (t.nx == grids[i].nx && t.bx == grids[i].bx && t.overlap == grids[i].overlap) oi.smoother_shape = t.shape;
    if (opt->coarse_space == TG_COARSE_LEARNED && opt->batch_nets) {
      // the network trained for this instance's block size
      oi.net = nullptr;
      for (int k = 0; k < opt->batch_nnets && !oi.net; ++k) {
        if (!opt->batch_nets[k]) continue;
        int nb = 0, nk = 0, hid = 0, din = 0, dout = 0;
        mlp_dims(opt->batch_nets[k], &nb, &nk, &hid, &din, &dout);
        if (nb == grids[i].bx) oi.net = opt->batch_nets[k];
      }
      if (!oi.net) {
        rc = TG_ERR_INVALID_ARG;
        break;
      }
    }
    rc = tg_setup(kappa[i], &grids[i], eig_tol, &oi, stream, &h);
    if (!rc) {
      B->handles.push_back(h);
      if (oi.smoother_shape < 0) tuned.push_back(Tuned{grids[i].nx, grids[i].bx, grids[i].overlap, h->shape});
    }
  }
  // contexts: the handle's own context serves its first right-hand side
  for (int i = 0; i < ninst && !rc; ++i) {
    for (int k = 0; k < nrhs && !rc; ++k) {
      Ctx* c = nullptr;
      if (k == 0) {
        c = B->handles[i]->ctx;
        B->handles[i]->ctx = nullptr;   // now owned by the batch
        rc = ctx_alloc(B->handles[i], &B->handles[i]->ctx);
      } else {
        rc = ctx_alloc(B->handles[i], &c);
      }
      if (!rc) B->ctx.push_back(c);
    }
  }
  const int m = ninst * nrhs;
  if (!rc && (dalloc(&B->d_src, 5 * m) || dalloc(&B->d_buf, 5 * m) || dalloc(&B->d_cnt, 5 * m) ||
              dalloc(&B->d_rtol, 1) || dalloc(&B->d_ctx_rtol, m) || dalloc(&B->d_ctx_state, m) ||
              dalloc(&B->d_out, 2 * m)))
    rc = TG_ERR_OOM;
  if (!rc) rc = cuda_err(cudaMallocHost(&B->h_src, sizeof(double*) * 5 * m));
  if (!rc) rc = cuda_err(cudaMallocHost(&B->h_out, sizeof(int) * 2 * m));
  if (!rc) rc = cuda_err(cudaMallocHost(&B->h_rtol, sizeof(double)));
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  if (!rc) {
    std::vector<double*> buf(5 * m), rt(m);
    std::vector<long long> cnt(5 * m);
    std::vector<PcgState*> stp(m);
    for (int j = 0; j < m; ++j) {
      Ctx* c = B->ctx[j];
      const long long n = c->h->n, nn = n * n, nf = (n + 1) * n;
      double* bufs[5] = {c->fd, c->bd, c->ux, c->uy, c->pd};
      const long long cn[5] = {nn, 4 * n, nf, nf, nn};
      for (int t = 0; t < 5; ++t) {
        buf[5 * j + t] = bufs[t];
        cnt[5 * j + t] = cn[t];
      }
      rt[j] = c->d_rtol;
      stp[j] = c->st;
    }
    rc = cuda_err(cudaMemcpy(B->d_buf, buf.data(), sizeof(double*) * buf.size(), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_err(cudaMemcpy(B->d_cnt, cnt.data(), sizeof(long long) * cnt.size(), cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_err(cudaMemcpy(B->d_ctx_rtol, rt.data(), sizeof(double*) * m, cudaMemcpyHostToDevice));
    if (!rc) rc = cuda_err(cudaMemcpy(B->d_ctx_state, stp.data(), sizeof(PcgState*) * m, cudaMemcpyHostToDevice));
  }
  if (!rc) {
    // one graph: the chains of all contexts, independent of each other
    cudaGraph_t g = nullptr;
    rc = cuda_err(cudaGraphCreate(&g, 0));
    g_pdl = (opt->launch_overlap != 0);
    // the right-hand sides of an instance advance in lock step (groups of up
    // to kGroup sharing the smoother sweeps) when the cycle is the five-kernel
    // one; otherwise every context is an independent chain
    const bool lockstep = opt->batch_lockstep && nrhs > 1 && opt->m1 == 1 && opt->m2 == 1 &&
                          opt->cycle == TG_CYCLE_TWO_GRID;
    for (int i = 0; i < ninst && !rc; ++i) {
      // a band smoother has no lock-step sweep: its right-hand sides run as
      // independent branches (in a group they would follow one another)
      const bool ls = lockstep && !is_band_shape(B->handles[i]->shape);
      for (int k0 = 0; k0 < nrhs && !rc; k0 += ls ? kGroup : 1) {
        const int k = ls ? std::min(kGroup, nrhs - k0) : 1;
        Ctx* const* cs = &B->ctx[(size_t)i * nrhs + k0];
        rc = (k > 1) ? add_group(cs, k, g, B->cap) : add_chain(cs[0], g, B->cap);
      }
    }
    if (!rc) rc = cuda_err(cudaGraphInstantiate(&B->exec, g, 0));
    if (g) cudaGraphDestroy(g);
  }
  if (rc) {
    batch_free(B);
    return rc;
  }
  *out = B;
  return TG_OK;
}

int tg_solve_batch(tg_batch* B, const double* const* f, const double* const* bflux, double rtol,
                   double* const* ux, double* const* uy, double* const* p, int* iters, int* status) {
  if (!B || !f || !ux || !uy || !p || !(rtol > 0) || !(rtol < 1)) return TG_ERR_INVALID_ARG;
  const int m = (int)B->ctx.size();
  cudaStream_t s = B->stream;
  for (int j = 0; j < m; ++j) {
    if (!f[j] || !ux[j] || !uy[j] || !p[j]) return TG_ERR_INVALID_ARG;
    B->h_src[5 * j + 0] = const_cast<double*>(f[j]);
    B->h_src[5 * j + 1] = bflux ? const_cast<double*>(bflux[j]) : nullptr;
    B->h_src[5 * j + 2] = ux[j];
    B->h_src[5 * j + 3] = uy[j];
    B->h_src[5 * j + 4] = p[j];
  }
  *B->h_rtol = rtol;
  TG_CK(cudaMemcpyAsync(B->d_src, B->h_src, sizeof(double*) * 5 * m, cudaMemcpyHostToDevice, s));
  TG_CK(cudaMemcpyAsync(B->d_rtol, B->h_rtol, sizeof(double), cudaMemcpyHostToDevice, s));
  // inputs: caller -> context buffers (f, bflux or zeros), tolerances
  launch_copy_table((const double* const*)B->d_src, B->d_buf, B->d_cnt, m, 0, 2, 1, s);
  launch_fill_scalars(B->d_rtol, B->d_ctx_rtol, m, s);
  TG_CK(cudaGraphLaunch(B->exec, s));
  // outputs: context buffers -> caller (ux, uy, p), then iterations and status
  launch_copy_table((const double* const*)B->d_buf, (double* const*)B->d_src, B->d_cnt, m, 2, 5, 0, s);
  launch_gather_states(B->d_ctx_state, B->d_out, m, s);
  TG_CK(cudaMemcpyAsync(B->h_out, B->d_out, sizeof(int) * 2 * m, cudaMemcpyDeviceToHost, s));
  TG_CK(cudaStreamSynchronize(s));
  TG_CK(cudaGetLastError());
  int worst = TG_OK;
  for (int j = 0; j < m; ++j) {
    if (iters) iters[j] = B->h_out[2 * j];
    if (status) status[j] = status_to_err(B->h_out[2 * j + 1]);
    const int e = status_to_err(B->h_out[2 * j + 1]);
    if (e != TG_OK && (worst == TG_OK || e > worst)) worst = e;   // MAXITER (-4) before harder errors
  }
  if (read_and_clear_timeout()) worst = TG_ERR_DEVICE_TIMEOUT;
  return worst;
}

void tg_destroy_batch(tg_batch* B) { batch_free(B); }

int tg_batch_size(tg_batch* B, int* ninst, int* nrhs) {
  if (!B) return TG_ERR_INVALID_ARG;
  if (ninst) *ninst = (int)B->handles.size();
  if (nrhs) *nrhs = B->nrhs;
  return TG_OK;
}

int tg_face_data(const double* kappa, const tg_grid* grid, double eig_tol, int k, void* stream, uint16_t* x,
                 float* q, int* nsel, double* lambda) {
  if (!kappa || !x || !q || k < 1 || k > 8 || !(eig_tol > 0)) return TG_ERR_INVALID_ARG;
  int rc = validate_grid(grid);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TG_ERR_CUDA;
  tg_handle* h = new (std::nothrow) tg_handle();
  if (!h) return TG_ERR_OOM;
  h->n = grid->nx;
  h->b = grid->bx;
  h->nc = h->n / h->b;
  h->ov = grid->overlap;
  h->nblocks = h->nc * h->nc;
  h->npatch = h->nblocks;
  h->nfaces = 2 * h->nc * (h->nc - 1);
  h->h = 1.0 / h->n;
  h->H = (double)h->b / h->n;
  h->eig_tol = eig_tol;
  tg_default_options(&h->opt);
  h->stream = (cudaStream_t)stream;
  SpectralBufs sb{};
  rc = setup_kappa(h, kappa);
  if (!rc) rc = setup_blocks(h, false);
  if (!rc && h->nfaces > 0) {
    h->nsel.assign(h->nfaces, 1);
    rc = alloc_spectral(h, sb);
    if (!rc) {
      spectral_exact(h, sb, nullptr, nullptr, q, k);
      launch_face_inputs(kappa, h->n, h->b, reinterpret_cast<__nv_bfloat16*>(x), h->stream);
      rc = read_spectral(h, sb);
    }
    if (!rc && nsel) rc = cuda_err(cudaMemcpyAsync(nsel, sb.d_nsel, sizeof(int) * h->nfaces, cudaMemcpyDeviceToDevice, h->stream));
    if (!rc && lambda)
      rc = cuda_err(cudaMemcpyAsync(lambda, h->lam, sizeof(double) * h->nfaces * h->b, cudaMemcpyDeviceToDevice, h->stream));
    if (!rc) rc = cuda_err(cudaStreamSynchronize(h->stream));
  }
  free_spectral(sb);
  tg_destroy(h);
  return rc;
}

}  // extern "C"
