// Internal declarations shared by the libtgms translation units.
//
// Device data layout (n x n fine cells, h = 1/n, blocks of b x b cells,
// nc = n/b blocks per side):
//   node vectors ("psi vectors"): n*n, node (i, j) at j*n + i; nodes with
//     i == 0 or j == 0 are boundary nodes and are kept at zero; nodes with
//     i == n or j == n are implicit zeros;
//   cell arrays: n*n, cell (i, j) at j*n + i;
//   face arrays: ux (n+1)*n at j*(n+1)+i, uy n*(n+1) at j*n+i;
//   block (I, J) owns the nodes [I b, (I+1) b) x [J b, (J+1) b); its closed
//     node set [I b, (I+1) b] x [J b, (J+1) b] is stored locally as
//     (a, c) -> c*(b+1) + a; its interior nodes a, c in [1, b-1] as
//     (c-1)*(b-1) + (a-1);
//   patch (= oversampled block K_i^+) interior nodes: x0 < i < x1,
//     y0 < j < y1 for the clipped cell rectangle [x0, x1) x [y0, y1),
//     local index (j-y0-1)*nx + (i-x0-1).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>
#include <vector>

struct tg_mlp;   // network of the learned coarse basis (learned.cu)

namespace tg {

constexpr int kMaxB = 16;                 // largest supported block size b
constexpr int kMaxOverlap = 2;
constexpr int kMaxPatchSide = kMaxB + 2 * kMaxOverlap - 1;   // interior nodes per side
constexpr int kMaxDynSmem = 227 * 1024;   // dynamic shared memory per CTA (opt-in limit)
constexpr int kMaxPatchNodes = kMaxPatchSide * kMaxPatchSide;
constexpr int kMaxHist = 4096;            // PCG coefficient history
constexpr int kRedGrid = 512;             // CTAs of grid-stride reduction kernels

// status bits raised by device code
enum : int {
  kStOk = 0,
  kStBadKappa = 1,
  kStNotSpd = 2,
  kStBreakdown = 4,
  kStIncompatible = 8,
  kStDegenerate = 16,
  kStMaxIter = 32,
  kStTimeout = 64,      // a bounded device-side wait expired
};

struct PatchGeo {
  int x0, y0;      // lower-left cell of the clipped patch rectangle
  int nx, ny;      // interior nodes per side
  int nloc;        // nx * ny
  int ld;          // row stride of the stored inverse (multiple of 8)
  long long off;   // element offset of the stored inverse
  long long toff;  // element offset of the inverse in the tensor-core tile layout (2-byte storage)
};

// Scalars of the PCG iteration, updated only by the last CTA of a
// reduction kernel (so no CTA reads a value written in its own kernel).
struct PcgState {
  double rz;        // (r, z) of the current iterate
  double rz_prev;   // (r, z) of the previous iterate (flexible beta)
  double rr0;       // ||r_0||^2
  double rr;        // ||r||^2
  double rtol2;     // rtol^2
  double alpha, beta, pq, zq;
  int iter;         // completed iterations
  int maxit;
  int done;         // 1: stop (converged, breakdown or max_iter)
  int status;       // kSt* bits
  int flexible;
  unsigned int counter[4];   // arrival counters of last-CTA reductions
  double alphas[kMaxHist];
  double betas[kMaxHist];
};

// One coarse-space slot: a basis function restricted to one block.
struct Slot {
  int block;
  int kind;        // 0: nodal function theta_m (corner), 1: zero-flux function z_{E,k}
  int which;       // corner (0 BL, 1 BR, 2 TL, 3 TR) or side (0 L, 1 R, 2 B, 3 T)
  int k;           // zero-flux index (1..nsel-1)
  int face;        // coarse face of the side (kind 1) or -1
  int coef;        // coarse unknown
};

// One row of a ragged batch of dense GEMVs: out = sum_j M[m + j] * x[x0 + j], j < len.
struct NdRow {
  long long m;
  int x0, len, out;
};

// Nested-dissection factor of an SPD coarse system (coarse_nd.cu), one level:
// the coarse unknowns are split by coarse block rows into S strips whose
// interiors do not couple to each other, and S - 1 separators (the unknowns
// of one row of coarse nodes: the nodal functions of that row and the
// zero-flux functions of its horizontal coarse faces).  With the unknowns
// ordered interiors first (strip by strip), separators last, A_t the
// interior blocks, X_t = A_t^{-1} A_{t,S} and Sigma = A_SS - sum_t A_{S,t} X_t
// the separator Schur complement, the solve of K y = c is
//   w_t = A_t^{-1} c_t,  g = c_S - sum_t X_t^T c_t,  y_S = Sigma^{-1} g,
//   y_t = w_t - X_t y_S,
// each a batch of dense FP64 GEMVs with blocks stored as explicit inverses.
struct NdFactor {
  int D = 0, DI = 0, NS = 0;   // unknowns, interior unknowns, separator unknowns
  int strips = 0;
  int* perm = nullptr;         // D: unknown at each position of the interiors-then-separators order (device)
  int* gatherp = nullptr;      // 4 D: slot ids of the unknown at each position (device)
  double* M = nullptr;         // per strip [A_t^{-1}; X_t^T] (rows of width n_t), then the X_t, then Sigma^{-1}
  NdRow* rows_a = nullptr;     // rows of the [A_t^{-1}; X_t^T] blocks (device)
  NdRow* rows_b = nullptr;     // rows of the X_t blocks (device)
  int nrows_a = 0, nrows_b = 0;
  long long y_off = 0;         // element offset of Sigma^{-1} in M
  long long total = 0;         // entries of M
  double bytes = 0;            // matrix bytes read by one solve
};

// Coarse space in per-block slot form.
struct CoarseSpace {
  int D = 0;                 // coarse unknowns
  int nslots = 0;
  int* slot_ptr = nullptr;   // nblocks+1, CSR over blocks (device)
  Slot* slots = nullptr;     // device
  int* gather = nullptr;     // D*4 global slot ids (-1 = none) (device)
  double* closed = nullptr;  // nslots*(b+1)^2 FP64 tiles (device)
  void* owned = nullptr;     // nslots*b*b tiles: FP64 (FP64 handles), else FP32 (device)
  double* Kinv = nullptr;    // D*D inverse of the Galerkin matrix (device)
  // mixed-precision handles with D > kCoarseSplit: Kinv as double-float
  // pairs (hi, lo: FP32, hi + lo = Kinv to ~2^-48), applied on the FP32 pipe
  float2* Kdf = nullptr;
  int low_rank_updates = 0;  // low-rank updates of Kinv since it was last inverted in full
  int max_slots_per_block = 0;
  // coarse row key of every unknown (host): 2 j for the nodal functions of
  // coarse node row j and the zero-flux functions of the horizontal faces at
  // y = j H (support in block rows j - 1 and j), 2 J + 1 for the zero-flux
  // functions of the vertical faces in block row J (support in row J only)
  std::vector<int> key;
  // solver of the coarse system: 1 = dense inverse Kinv, 2 = nested
  // dissection (nd; Kinv then holds the Galerkin matrix itself)
  int solver = 1;
  NdFactor nd;
  // TG_COARSE_SOLVER_AUTO: set at the first low-rank update request (a
  // change of kappa with the basis kept); the space keeps the dense inverse
  // from then on, whose low-rank updates cost far less than new factors
  bool updated_dense = false;
};

// Nested-dissection coarse solver (coarse_nd.cu)
constexpr int kNdSepMax = 16384;   // separator unknowns staged in shared memory by the separator GEMV
constexpr int kNdAutoMin = 768;    // TG_COARSE_SOLVER_AUTO takes nested dissection above this many unknowns
// Factor of the SPD matrix K (D x D, device, row-major) with row keys `key`
// and nc coarse blocks per side; gather (device, 4 D) gives the slots of each
// unknown.  Returns TG_ERR_UNSUPPORTED when fewer than 2 strips of at least 2
// block rows exist; sets kStNotSpd in *status on a non-positive pivot.  A
// factor of the same structure (same keys and slots, e.g. after a change of
// kappa with the coarse basis kept) is formed again in the buffers it already
// has, so CUDA graphs that captured its solve stay valid.
int nd_build(const double* K, int D, const std::vector<int>& key, int nc, const int* gather, NdFactor& f,
             int* status, cudaStream_t s);
void nd_free(NdFactor& f);
// d = K^{-1} c, c[u] = sum of the partials of u's slots; work: 4 D doubles
// after d (device).  Four launches.
void launch_nd_solve(const NdFactor& f, const double* part, double* d, const PcgState* st, cudaStream_t s);

constexpr int kCoarseSplit = 1024;   // coarse systems larger than this form their right-hand side once
// Kinv (m entries) into double-float pairs: hi = fl32(x), lo = fl32(x - hi)
void launch_split_df(const double* a, float2* b, long long m, cudaStream_t s);
// shared memory of the RT0 particular-flux kernel for nc x nc blocks; -1 if the device cannot hold it
int configure_rt_particular(int nc, int nblocks);

// ---- small device helpers --------------------------------------------------
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double to_f(double x) { return x; }

template <typename T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn((float)x);
}
template <> __device__ __forceinline__ __half from_d<__half>(double x) { return __double2half(x); }

// Coarse basis tiles are stored in the preconditioner precision, except with
// 2-byte patch inverses (BF16, FP16), whose tiles stay FP32: they are a small
// fraction of the bytes, and BF16 tiles (8 significant bits) cost PCG
// iterations at large grids.
template <typename TS> struct TileOf { using T = TS; };
template <> struct TileOf<__half> { using T = float; };
template <> struct TileOf<__nv_bfloat16> { using T = float; };
template <typename TS> using tile_t = typename TileOf<TS>::T;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 9-point stencil of K = C^T A_h C at interior node (i, j) (1 <= i, j < n),
// written with the inverse permeabilities of the four cells around the node:
// k00 = (i-1, j-1), k10 = (i, j-1), k01 = (i-1, j), k11 = (i, j).
template <typename TV, typename TK, typename TA>
__device__ __forceinline__ TA stencil_apply(const TV* __restrict__ psi, const TK* __restrict__ kinv,
                                            int n, int i, int j) {
  const long long c = (long long)j * n + i;
  const bool e = (i + 1 < n), N = (j + 1 < n);
  const TA p0 = (TA)psi[c];
  const TA pw = (TA)psi[c - 1];
  const TA ps = (TA)psi[c - n];
  const TA psw = (TA)psi[c - n - 1];
  const TA pe = e ? (TA)psi[c + 1] : (TA)0;
  const TA pse = e ? (TA)psi[c - n + 1] : (TA)0;
  const TA pn = N ? (TA)psi[c + n] : (TA)0;
  const TA pnw = N ? (TA)psi[c + n - 1] : (TA)0;
  const TA pne = (e && N) ? (TA)psi[c + n + 1] : (TA)0;
  const TA k11 = (TA)kinv[c], k01 = (TA)kinv[c - 1];
  const TA k10 = (TA)kinv[c - n], k00 = (TA)kinv[c - n - 1];
  const TA third = (TA)(1.0 / 3.0), sixth = (TA)(1.0 / 6.0);
  TA out = (TA)(2.0 / 3.0) * (k00 + k10 + k01 + k11) * p0;
  out -= sixth * ((k00 + k10) * ps + (k01 + k11) * pn + (k00 + k01) * pw + (k10 + k11) * pe);
  out -= third * (k00 * psw + k10 * pse + k01 * pnw + k11 * pne);
  return out;
}

// Programmatic dependent launch.  Every solve-path kernel starts here: it
// waits until the grid it depends on has completed and its writes are visible
// (a no-op when the launch carried no programmatic dependency), then lets the
// next grid in the stream begin launching.  The next grid can only launch
// once every CTA of this one has executed the trigger, so its waiting CTAs
// never hold resources that this grid still needs.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Sum of a partial array by one warp in a fixed order (deterministic).
__device__ __forceinline__ double warp_sum_array(const double* a, int m) {
  double s = 0.0;
  for (int k = threadIdx.x & 31; k < m; k += 32) s += a[k];
  return warp_sum(s);
}

}  // namespace tg

// ---- launchers (host functions, implemented in the kernel files) ----------
namespace tg {

// number of kernels enqueued by the launchers below (host counter)
extern unsigned long long g_kernel_launches;
#define TG_COUNT(k) (::tg::g_kernel_launches += (unsigned long long)(k))

// Solve-path kernels are launched with the programmatic-stream-serialization
// attribute when g_pdl is set (tg_options.launch_overlap, read at enqueue /
// capture time), so a kernel's launch overlaps the tail of its predecessor.
// Off by default: measured slower on GB300 for this kernel chain.
extern bool g_pdl;
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t shm, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = shm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = g_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

void configure_kernels(int max_coarse_dim);
// batched solves (batch.cu)
void launch_copy_table(const double* const* src, double* const* dst, const long long* cnt, int m, int t0, int t1,
                       int zero_if_null, cudaStream_t s);
void launch_fill_scalars(const double* v, double* const* dst, int m, cudaStream_t s);
void launch_gather_states(PcgState* const* st, int* out, int m, cudaStream_t s);
int read_and_clear_timeout();   // 1 if a bounded device wait expired since the last call
// Lock-step groups of right-hand sides (batched solves): up to kGroup PCG
// chains of one instance share each read of the patch inverses.  Per chain:
// mode 1 (first sweep) reads r_old, q, x, p, part, st, zclear and writes into
// zacc; mode 2 (last sweep) reads r, zin, kin, st and writes into zacc.
constexpr int kGroup = 4;
struct ChainPtrs {
  const double* r_old;
  double* r_new;
  const double* q;
  double* x;
  const double* p;
  double* part;
  PcgState* st;
  void* zclear;
  const void* zin;
  const void* kin;
  const double* r;
  void* zacc;
};
struct StateSet {
  const PcgState* st[kGroup];
  int k;
};
struct BandRef;
// tiles (optional): the tensor-core tile layout of the same inverses, used
// when shape is kShapeTensor (2-byte storage)
template <typename TC, typename TS>
void launch_smoother_multi(int mode, const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                           const ChainPtrs* chains, int k, double eta, int n, int nc, int b, cudaStream_t s, int shape,
                           const float* rscale, const BandRef* tiles = nullptr);
// graph loop condition: 1 while any of the k chains is not done
void launch_set_condition_any(cudaGraphConditionalHandle cond, const PcgState* const* st, int k, cudaStream_t s);

// one warp waits (at most 2^limit_log2 polls) on an mbarrier it completes
// first (complete != 0) or that nothing completes (the wait expires)
void launch_wait_probe(int complete, int limit_log2, cudaStream_t s);
void launch_pcg_reset(PcgState* st, const double* rtol, int maxit, int flexible, cudaStream_t s);
// warm start: r = rho - K x, rr = |r|^2, rr0 = |rho|^2 (stopping reference)
void launch_pcg_init_warm(const double* x, const double* rho, const double* kinv, double* r, double* part,
                          PcgState* st, int n, cudaStream_t s);
// warm start: x = stream function of the x-face part of ux0 - vx (colbuf: n*n scratch)
void launch_psi_from_faces(const double* ux0, const double* vx, double* colbuf, double* psi, int n, cudaStream_t s);
void launch_set_condition(cudaGraphConditionalHandle cond, const PcgState* st, cudaStream_t s);

// fine operator / vectors (fine.cu)
void launch_apply_operator(const double* psi, const double* kinv, double* out, int n, cudaStream_t s);
void launch_apply_operator_f32(const double* psi, const float* kinv, double* out, int n, cudaStream_t s);

template <typename TC>
void launch_residual(const double* r, const TC* z, const TC* kinv, TC* out, int n, const PcgState* st,
                     cudaStream_t s);

template <typename TC>
void launch_pcg_dots(const double* r, const TC* z, const double* q, double* part, PcgState* st,
                     int n, cudaStream_t s);
void launch_pcg_init(double* x, const double* r, double* part, PcgState* st, int n, cudaStream_t s);
template <typename TC>
void launch_pcg_init_rz(const double* r, const TC* z, double* p, double* part, PcgState* st, int n,
                        cudaStream_t s);

// Smoother tile shapes (chosen per handle by the autotuner): 0 = 16-byte
// loads, 4 rows per pass (2 for FP64); 1 = 16-byte loads, 2 rows; 2 = 8-byte
// loads, 4 rows; 3 = 8-byte loads, 2 rows; 4 = TMA bulk copies into a
// shared-memory ring; 5 = shape 3 and 6 = shape 1, software-pipelined (the
// next pass's rows in flight while the current one is reduced).  FP64 storage
// uses shape 0 for 1..3, 5, 6; FP16 storage uses shape 0 for 4.
constexpr int kSmootherShapes = 10;
constexpr int kShapeBand = 7;   // smoother from the patches' band Cholesky factors (two triangular solves)
// The band form with FP32 factors read ahead through a shared-memory ring
// (cp.async, 44 rows ahead instead of 16 in registers); FP64 factors run
// shape 7.  The autotuner keeps whichever band form is faster per handle.
constexpr int kShapeBandRing = 9;
__host__ __device__ inline bool is_band_shape(int shape) { return shape == kShapeBand || shape == kShapeBandRing; }
// The patch inverses applied on the tensor cores (2-byte storage; FP32 and
// FP64 storage use shape 0): 16 x 16 tiles stored in the A-fragment order
// of mma.m16n8k16, the residual split into three 2-byte parts as the
// columns of B.  Tile layout of patch p at toff (elements): T = ceil(nloc /
// 16) tiles per side, tile (i, j) (rows 16 i.., columns 16 j..) at
// toff + (i T + j) 256, lane l's eight entries at + 8 l: entries e = 0..7 are
// (row 16 i + l / 4 + 8 ((e >> 1) & 1), column 16 j + 2 (l % 4) + (e & 1) +
// 8 (e >> 2)), zero outside the matrix; FP16 rows carry the row scaling of
// the row layout.
constexpr int kShapeTensor = 8;
constexpr int kTile = 16;
__host__ __device__ inline int tiles_per_side(int nloc) { return (nloc + kTile - 1) / kTile; }
// band factors of the oversampled patches in the arithmetic type, two
// layouts per patch (patch p at p * stride, the second at + stride / 2):
// column layout, entry (j, d) = L_{j+d, j} (the column below the diagonal;
// read by the forward sweep), and row layout, entry (j, d) = L_{j, j-d} (the
// row left of the diagonal; read by the backward sweep); d = 0 holds 1 / L_jj
// in both.  Rows are stored in groups of four, interleaved by entry: with
// R = j + kBandPad, entry (j, d) sits at (R / 4) * 4 ldb + 4 d + R % 4, so
// lane d of a warp loads entries (j..j+3, d) of a group as one 16-byte vector
// (two for FP64) and a group is one contiguous, 16-byte aligned block.
// band_rows(nmax) rows, -kBandPad .. roundup(nmax, kBandPF) + kBandPad - 1,
// are stored, zero outside the matrix and the band, so the sweeps read them
// without bounds checks.
// ldb (BandRef): entries per stored row, the handle's widest band plus the
// reciprocal diagonal (21 at b = 16, 13 at b = 8); kBandLd bounds it
constexpr int kBandLd = 24;    // the band is at most kMaxPatchSide + 1 = 20 wide
constexpr int kBandPF = 16;    // row rounding of the sweeps, and at most the rows they keep in flight per lane
constexpr int kBandPad = 16;   // rows of zeros before and after: the read-ahead runs past the last row
static_assert(kBandPad >= kBandPF && kBandPad % 4 == 0 && kBandPF % 4 == 0,
              "read-ahead must stay inside the padding, in whole row groups");
inline long long band_rows(int nmax) {
  return (long long)(nmax + kBandPF - 1) / kBandPF * kBandPF + 2 * kBandPad;
}
// the patch factors in the layouts other than the dense rows: band factors
// (shape kShapeBand) and tensor-core tiles (shape kShapeTensor; tofs[p] the
// first 16-row tile of patch p in the global tile order, tofs[npatch] their
// total, as gofs is for 4-row groups)
struct BandRef {
  const void* p = nullptr;
  int ldb = 0;
  long long stride = 0;
  const void* tp = nullptr;
  const int* tofs = nullptr;
  int ntiles = 0;
};
// rscale: FP16 storage only, one power-of-two factor per stored row (index
// gofs[p] * kRowsPerGroup + row) that undoes the row's scaling.
template <typename TC, typename TS, typename TR>
void launch_smoother(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv, const TR* r,
                     TC* zacc, double eta, int n, const PcgState* st, cudaStream_t s, int shape = 0,
                     const float* rscale = nullptr, BandRef band = {});
template <typename TC, typename TS>
void launch_smoother_update(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                            const double* r_old, double* r_new, const double* q, double* x, const double* p,
                            TC* zacc, double eta, int n, int nc, int b, double* part, PcgState* st,
                            cudaStream_t s, int shape = 0, const float* rscale = nullptr, TC* zclear = nullptr,
                            BandRef band = {});
// last smoothing sweep with the residual formed at gather time:
// zout (zeroed beforehand) = zin + eta sum_i E_i M_i E_i^T (r - K zin)
template <typename TC, typename TS>
void launch_smoother_resid(const PatchGeo* geo, const int* gofs, int npatch, int ngroups, const TS* pinv,
                           const double* r, const TC* zin, const TC* kin, TC* zout, double eta, int n, int nc, int b,
                           const PcgState* st, cudaStream_t s, int shape, const float* rscale, BandRef band = {});
template <typename TC>
void launch_pcg_apply_p(const TC* zprev, const double* pold, double* pnew, double* q, TC* znext,
                        const double* kcoef, double* part, PcgState* st, int n, cudaStream_t s);
void launch_stencil_coefs(const double* kinv, double* kcoef, int n, cudaStream_t s);
template <typename TC, typename TS>
void launch_resid_restrict(const CoarseSpace& cs, double* part, int nblocks, int nc, int b, int n, const double* r,
                           const TC* z, const TC* kinv, const PcgState* st, cudaStream_t s);
constexpr int kRowsPerGroup = 4;   // rows of a patch inverse streamed together by one warp

// per-solve scratch of the coarse step: part (one entry per slot), coefs (D)
template <typename TC, typename TS>
void launch_restrict(const CoarseSpace& cs, double* part, int nblocks, int nc, int b, int n, const TC* v,
                     const PcgState* st, cudaStream_t s);
// v += Psi K_H^{-1} c (c formed from the slot partials): one fused kernel for
// small coarse systems, else the coarse solve then the prolongation
template <typename TC, typename TS>
void launch_coarse_correct(const CoarseSpace& cs, const double* part, double* coefs, int nblocks, int nc, int b, int n,
                           TC* v, const PcgState* st, cudaStream_t s);
// coefs: 2 D doubles; d = coefs[0, D), the second half is right-hand-side scratch
void launch_coarse_solve(const CoarseSpace& cs, const double* part, double* coefs, const PcgState* st,
                         cudaStream_t s);
template <typename TC, typename TS>
void launch_prolong(const CoarseSpace& cs, const double* coefs, int nblocks, int nc, int b, int n, TC* v,
                    const PcgState* st, cudaStream_t s);

template <typename TA, typename TB>
void launch_convert(const TA* a, TB* b, long long m, cudaStream_t s);

// preprocessing and epilogue (pre.cu)
void launch_lift(const double* bflux, double* ux, double* uy, int n, cudaStream_t s);
void launch_block_sources(const double* f, const double* ux, const double* uy, double* FH,
                          double* absF, int n, int b, cudaStream_t s);
void launch_rt_particular(const double* FH, const double* absF, double* gx, double* gy, int nc,
                          double H, int nblocks, PcgState* st, cudaStream_t s);
void launch_add_rt_field(const double* gx, const double* gy, double* ux, double* uy, int n, int b,
                         cudaStream_t s);
void launch_face_residual(const double* ux, const double* uy, const double* kinv, double* rho,
                          int n, cudaStream_t s);
void launch_add_curl(const double* psi, double* ux, double* uy, int n, cudaStream_t s);
void launch_block_particular(const double* f, double* ux, double* uy, int n, int b, cudaStream_t s);
void launch_pressure(const double* ux, const double* uy, const double* kinv, double* p,
                     double* work, int n, cudaStream_t s);
void launch_div_error(const double* ux, const double* uy, const double* f, double* part,
                      double* out, int n, cudaStream_t s);

// setup (setup.cu)
void launch_kinv(const double* kappa, double* kinv, float* kinv32, int* status, int n,
                 cudaStream_t s);
// slot (optional, NULL = identity): the band of rectangle m is band slot
// slot[m], so a compacted list of rectangles updates bands kept in the full
// numbering
void launch_assemble_band(const double* kinv, const int4* rects, double* band, int nmat, int wmax,
                          int nmax, int n, cudaStream_t s, const int* slot = nullptr);
void launch_band_cholesky(double* band, const int4* rects, int nmat, int wmax, int nmax,
                          int* status, cudaStream_t s, const int* slot = nullptr);
void launch_band_inverse(const double* band, const int4* rects, int first, int count, int wmax,
                         int nmax, double* scratch, cudaStream_t s, const int* slot = nullptr);
// band factors (Cholesky bands of compact patches c, rows L[j][d] =
// L_{j,j-d}) into the smoother's band layout (BandRef) of patches ids[c]
template <typename TB>
void launch_store_band(const double* band, const int4* rects, const int* ids, int count, int wmax, int nmax,
                       long long stride, TB* out, cudaStream_t s);
// flag[m] = 1 where some cell of rectangle m gets a new 1/kappa (bitwise
// comparison against kinv_old, computed as launch_kinv computes it)
void launch_rect_changed(const double* kappa, const double* kinv_old, const int4* rects, int nrect, int n,
                         unsigned char* flag, cudaStream_t s);
template <typename TS>
void launch_store_inverse(const double* scratch, const PatchGeo* geo, int first, int count,
                          int nmax, TS* pinv, cudaStream_t s);
// FP16 storage: each row scaled by a power of two that puts its largest
// magnitude in [2^14, 2^15); rscale receives the inverse factor.  pidx
// (optional): patch numbers of a compacted geo list
void launch_store_inverse_f16(const double* scratch, const PatchGeo* geo, const int* gofs, int first, int count,
                              int nmax, __half* pinv, float* rscale, cudaStream_t s, const int* pidx = nullptr);
// The same inverses in the tensor-core tile layout (kShapeTensor; TS 2-byte).
// FP16: each row scaled as the row layout scales it (rscale, written by
// launch_store_inverse_f16 before, indexed through gofs and pidx).
template <typename TS>
void launch_store_inverse_tiles(const double* scratch, const PatchGeo* geo, const int* gofs, const int* pidx,
                                int first, int count, int nmax, TS* tiles, const float* rscale, cudaStream_t s);
// Snapshot functions of every (block, side): nfn functions per side whose
// coefficient vectors over {m, d_1..d_{b-1}} are coef[face][fn][0..b-1]
// (coef NULL: the unit vectors, nfn = b).  Sides with mask[blk*4+side] == 0
// are skipped (mask NULL: all).  psiS keeps b functions per side, gram b x b.
void launch_snapshots(const double* kinv, const double* blk_band, const double* coef, int nfn,
                      const unsigned char* mask, double* psiS, double* gram, int n, int b, cudaStream_t s);

// Arguments of the per-face spectral problems.
struct SpectralArgs {
  const double* kinv = nullptr;
  const double* gram = nullptr;
  double eig_tol = 0;
  int max_basis = 0;
  int mode = 0;                 // 0 spectral selection, 1 the unit-flux MsFEM function alone
  int n = 0, b = 0;
  double* lam = nullptr;        // [F][b] eigen- or Ritz values ascending (INFINITY padded)
  int* nsel = nullptr;          // [F]
  double* fcoef = nullptr;      // [F][b] unit-flux combination of the face's functions
  double* zcoef = nullptr;      // [F][b-1][b] zero-flux combinations
  int* status = nullptr;
  // learned mode (prof != NULL): the face's functions are jpred[f] predicted
  // ones with orthonormal flux profiles prof[f][i][.] and coefficients
  // ccoef[f][i][.] over {m, d_j}; Ritz pairs on their span
  const double* prof = nullptr;
  const double* ccoef = nullptr;
  const int* jpred = nullptr;
  int kmax = 0;
  int* fallback = nullptr;      // [F] out: 1 when the smallest Ritz value is >= eig_tol
  const unsigned char* fmask = nullptr;   // [F] faces to process (NULL: all)
  int* jeff = nullptr;          // [F] out: functions behind fcoef / zcoef
  float* labels = nullptr;      // [F][klab][b] out (exact mode): orthonormal profiles of the klab lowest modes
  int klab = 0;
};
void launch_face_spectral(const SpectralArgs& a, int nfaces, cudaStream_t s);
// predicted whitened profiles (network output y, faces x k x b FP32) ->
// flux profiles of an orthonormal basis of their span, their coefficients
// over {m, d_j}, and the count kept per face
void launch_pred_basis(const float* y, const double* kinv, int k, int n, int b, double thr, double* prof,
                       double* ccoef, int* jpred, int nfaces, cudaStream_t s);
template <typename TS>
void launch_build_tiles(const CoarseSpace& cs, const double* psiS, const double* fcoef,
                        const double* zcoef, const int* jeff, int rt_only, int n, int b, cudaStream_t s);
// bmask (optional): only blocks with bmask[blk] != 0 contribute (the weights
// kinv are zero on the cells of the others)
void launch_galerkin(const CoarseSpace& cs, const double* kinv, int nblocks, int n, int b,
                     double* pairE, const long long* pair_ptr, double* K, cudaStream_t s,
                     const unsigned char* bmask = nullptr);
void launch_gauss_jordan(double* A, double* B, int D, int* status, cudaStream_t s);
// low-rank update of a Galerkin inverse after a change of 1/kappa on few cells
// (setup.cu): delta = 1/kappa - kinv_old; row flags of nonzero rows; gathers
// out[i][a] = K[row(i)][S[a]] (row(i) = i if rows_all, else S[i]); in-place
// SPD inverse of a small matrix (s <= kGjSmallMax) by one CTA, *bad set on a
// non-positive pivot; FP64 GEMM C = alpha op(A) op(B) + beta C with element
// strides (op(A)(i,k) = A[i*ars + k*acs]); (A + A^T)/2; y += x
constexpr int kGjSmallMax = 1024;
constexpr int kGjBlock = 64;       // pivots per block of the blocked Gauss-Jordan inverse
void launch_kinv_delta(const double* kappa, const double* kinv_old, double* delta, int n, cudaStream_t s);
void launch_row_nonzero(const double* K, int D, unsigned char* flag, cudaStream_t s);
void launch_gather_cols(const double* K, int D, const int* S, int s_cnt, int rows, bool rows_all, double* out,
                        cudaStream_t s);
void launch_gj_small(double* A, int s_cnt, int* bad, cudaStream_t s);
void launch_dgemm(int m, int n, int k, double alpha, const double* A, long long ars, long long acs,
                  const double* B, long long brs, long long bcs, double beta, double* C, long long ldc,
                  cudaStream_t s);
void launch_symmetrize(double* A, int s_cnt, cudaStream_t s);
// B (D x D) += T X^T, T and X D x m row-major (small m: one thread per entry)
void launch_rank_update(double* B, int D, const double* T, const double* X, int m, cudaStream_t s);
void launch_add(double* y, const double* x, long long cnt, cudaStream_t s);  // result in A

// learned coarse basis (learned.cu)
void launch_face_inputs(const double* kappa, int n, int b, __nv_bfloat16* x, cudaStream_t s);
// network dimensions; y (batch x dout) = net(x) with caller scratch h1, h2 (batch x hidden)
void mlp_dims(const tg_mlp* net, int* b, int* k, int* hidden, int* din, int* dout);

// Tensor-core GEMM of the network (gemm_tc.cu): C (M x N) = A (M x K) B (N x K)^T,
// bfloat16 operands K-major (rows x K, row stride ld entries, ld a multiple of
// 8 and the base 16-byte aligned), FP32 accumulation, fused epilogue.
enum : int { kEpiF32 = 0, kEpiReluBf16 = 1, kEpiMaskBf16 = 2 };
struct TcOperand {
  const __nv_bfloat16* p;
  int rows, K, ld;
};
int gemm_tc(const TcOperand& a, const TcOperand& b, int M, int N, int K, const float* bias, int epi, float* outf,
            __nv_bfloat16* outh, long long som, const __nv_bfloat16* mask, cudaStream_t s);
// dst[r * ld + k] = src[(rmap ? rmap[r] : r) * s_row + (kmap ? kmap[k] : k) * s_k], zero for K <= k < ld
void pack_kmajor(const __nv_bfloat16* src, long long s_row, long long s_k, const int* rmap, const int* kmap, int R,
                 int K, int ld, __nv_bfloat16* dst, cudaStream_t s);
int read_and_clear_gemm_timeout();   // 1 if a bounded wait of the GEMM expired since the last call
int mlp_forward(const tg_mlp* net, int batch, const __nv_bfloat16* x, float* y, __nv_bfloat16* h1,
                 __nv_bfloat16* h2, cudaStream_t s);

}  // namespace tg
