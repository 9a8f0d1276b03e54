// Internal declarations shared by the libpairgal translation units.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/pairgal.h"

#define PG_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) return e__;                     \
  } while (0)

namespace pg {

template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Kernel launches issued by this library from the calling host thread (all
// plans); a launcher calls launched() right after each <<<...>>> instead of
// cudaGetLastError() (whose error state is per thread too).
std::atomic<long long>& launch_counter();
inline cudaError_t launched() {
  launch_counter().fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- scan (pg_scan.cu) -----------------------------------------------------
// Exclusive scan of `nseg` independent segments of `len` elements each:
// out[s*len + i] = sum_{j<i} in[s*len + j]; seg_total[s] = the segment sum.
// `tmp` must hold scan_tmp_elems(len, nseg) int64 values.
size_t scan_tmp_elems(int64_t len, int nseg);
cudaError_t scan_u8_i32(const uint8_t* in, int32_t* out, int64_t len, int nseg,
                        int64_t* seg_total, int64_t* tmp, cudaStream_t s);
cudaError_t scan_i32_i32(const int32_t* in, int32_t* out, int64_t len, int nseg,
                         int64_t* seg_total, int64_t* tmp, cudaStream_t s);

// ---- positions and pairs (pg_pairs.cu, compiled without FMA contraction) ----
cudaError_t launch_transform(int64_t n, double L, double rsd, const double* in_aos,
                             const float* vel, double* out_aos, double* x, double* y,
                             double* z, cudaStream_t s);
cudaError_t launch_widen_f32(int64_t n, const float* in, double* out, cudaStream_t s);
cudaError_t launch_check_finite(int64_t n, const double* aos, int32_t* flag, cudaStream_t s);
cudaError_t launch_wsum(int64_t n, const float* w, double* partial, double* out2,
                        cudaStream_t s);

struct PairGeom {
  double L, halfL;
  int nc;                 // cells per side (1, or >= 3)
  double cell_scale;      // nc / L
  int n_s, n_mu;
  double e2[65];          // squared s edges (grid: squared d_perp edges)
  int grid;               // 1: (d_perp, d_par) grid, pe = |d_par| edges
  double pe[65];
};

struct CellList {
  int32_t* cell_id;      // [n]
  int32_t* count;        // [ncell + 1]
  int32_t* start;        // [ncell + 1]
  int32_t* cursor;       // [ncell]
  int32_t* perm;         // [n] sorted slot -> input index
  double* xs; double* ys; double* zs;   // [n] sorted positions
  float* ws;             // [n] sorted weights (or unused)
  int64_t* tmp;          // scan temp
  int64_t* tot;          // [1]
};

cudaError_t launch_cells(const PairGeom& g, int64_t n, const double* x, const double* y,
                         const double* z, const float* w, CellList& cl, cudaStream_t s);

struct PairOut {
  unsigned long long* dd;    // [P] counts
  unsigned long long* ddq;   // [P] Q32.32 weight sums
  unsigned long long* cursor;// [1] fill cursor of the unsorted list
  int64_t capacity;
  int32_t* bin; int32_t* i; int32_t* j;
  double* mx; double* my; double* mz; double* wp;   // unsorted list
};
cudaError_t launch_pairs(const PairGeom& g, int64_t n, const CellList& cl, bool use_w,
                         bool fill, PairOut& po, cudaStream_t s);
// Groups the unsorted pair list by bin: slot = offset[bin] + atomic cursor.
cudaError_t launch_pair_scatter(int64_t np, const PairOut& po, unsigned long long* bin_cursor,
                                int32_t* sbin, int32_t* si, int32_t* sj, double* smid_aos,
                                double* sx, double* sy, double* sz, double* sw,
                                cudaStream_t s);

// ---- mass assignment (pg_mesh.cu, compiled without FMA contraction) --------
struct DepGeom {
  int N;
  double dx;              // L / N
  int assign;             // 0 NGP, 1 CIC, 2 TSC
};

// Nodes and weights of one axis of a point's assignment footprint (Sec. 3.5),
// u = x / dx; returns the node count (1 NGP, 2 CIC, 3 TSC). NGP: node
// floor(u + 1/2). CIC: floor(u) and the next node, weights 1 - f and f.
// TSC: the nearest node c = floor(u + 1/2) and its neighbours, weights
// (1/2)(1/2 - d)^2, 3/4 - d^2, (1/2)(1/2 + d)^2, d = u - c. Every operation
// rounds once (no contraction), so the weights are bit-reproducible.
__device__ __forceinline__ int axis_nodes(const DepGeom& g, double u, int* idx, double* wt) {
  const int N = g.N;
  if (g.assign == 0) {
    int i = (int)floor(__dadd_rn(u, 0.5)) % N;
    if (i < 0) i += N;
    idx[0] = i;
    wt[0] = 1.0;
    return 1;
  }
  if (g.assign == 1) {
    const double i0 = floor(u);
    const double fr = __dsub_rn(u, i0);
    int i = (int)i0 % N;
    if (i < 0) i += N;
    idx[0] = i;
    idx[1] = (i + 1 == N) ? 0 : i + 1;
    wt[0] = __dsub_rn(1.0, fr);
    wt[1] = fr;
    return 2;
  }
  const double c = floor(__dadd_rn(u, 0.5));
  const double d = __dsub_rn(u, c);
  int i = (int)c % N;
  if (i < 0) i += N;
  idx[0] = (i == 0) ? N - 1 : i - 1;
  idx[1] = i;
  idx[2] = (i + 1 == N) ? 0 : i + 1;
  const double t0 = __dsub_rn(0.5, d), t2 = __dadd_rn(0.5, d);
  wt[0] = __dmul_rn(0.5, __dmul_rn(t0, t0));
  wt[1] = __dsub_rn(0.75, __dmul_rn(d, d));
  wt[2] = __dmul_rn(0.5, __dmul_rn(t2, t2));
  return 3;
}
// Points: SoA x,y,z (FP64, in [0,L)), weight FP64 or null; pbin: per point
// bin index relative to the batch (null = all in bin 0).
cudaError_t launch_mark_lines(const DepGeom& g, int64_t n, const double* x, const double* y,
                              const double* z, const int32_t* pbin, int bin0,
                              uint8_t* flags, cudaStream_t s);
cudaError_t launch_line_compact(int N, int nb, const uint8_t* flags, const int32_t* idx,
                                const int64_t* line_base, int32_t* line_y, int32_t* line_bin,
                                int32_t* line_z,
                                cudaStream_t s);
cudaError_t launch_line_bases(int nb, const int64_t* seg_total, int64_t* line_base,
                              int64_t* n_lines_total, cudaStream_t s);
cudaError_t launch_deposit_lines(const DepGeom& g, int64_t n, const double* x, const double* y,
                                 const double* z, const double* w, const int32_t* pbin,
                                 int bin0, const int32_t* idx, const int64_t* line_base,
                                 unsigned long long* lines_q, unsigned long long* qsum,
                                 cudaStream_t s);
cudaError_t launch_deposit_dense(const DepGeom& g, int64_t n, const double* aos,
                                 const double* w, unsigned long long* mesh, cudaStream_t s);
cudaError_t launch_check_bins(int64_t n, const int32_t* bin, int nb, int32_t* bad, cudaStream_t s);
cudaError_t launch_lines_scatter(int N, int64_t n_lines, const unsigned long long* lines_q,
                                const int32_t* line_y, const int32_t* line_z,
                                const int32_t* line_bin, unsigned long long* mesh,
                                cudaStream_t s);
cudaError_t launch_field_scale(int nb, const unsigned long long* qsum, int N, double* scale,
                               cudaStream_t s);

// ---- FFT passes (pg_fft_f32.cu / pg_fft_f64.cu) -----------------------------
// Layout of a half-spectrum array, offsets in complex elements: element
// (z, y, kx) at z*zs + yoff(y) + xoff(kx), with
//   yoff(y)  = (y >> ks)*hs + (y & (2^ks - 1))*ys   (y in blocks of 2^ks rows)
//   xoff(kx) = (kx >> txs)*ts + (kx & (2^txs - 1))  (kx in tiles of 2^txs)
// The defaults ts = 1, txs = 0 keep kx contiguous. The plan's own spectra are
// [y / 8][z][kx / TX][y % 8][kx % TX] with TX = 64 bytes of complex values
// (8 in FP32, 4 in FP64), the width of every column tile: a y-pass item (one
// z plane, one kx tile, all ky) writes whole 512-byte blocks, and a z-pass
// item (one ky, one kx tile, all z) reads one 64-byte row of each block, a
// z stride of 8 P apart, as in the untiled [y / 8][z][y % 8][kx]. The stage
// entry points keep [z][y][kx] (ks large: one block; kx contiguous).
struct Lay {
  int64_t zs, ys, hs;
  int ks;
  int64_t ts = 1;
  int txs = 0;
};
__host__ __device__ __forceinline__ int64_t yoff(const Lay& L, int y) {
  return (int64_t)(y >> L.ks) * L.hs + (int64_t)(y & ((1 << L.ks) - 1)) * L.ys;
}
__host__ __device__ __forceinline__ int64_t xoff(const Lay& L, int kx) {
  return (int64_t)(kx >> L.txs) * L.ts + (kx & ((1 << L.txs) - 1));
}
inline Lay lay_zy(int N, int P) { return {(int64_t)N * P, (int64_t)P, 0, 30}; }
constexpr int kYBlockShift = 3;   // 8 ky rows per block
// kx tile shift of the plan layout: 64-byte tiles
template <typename R> constexpr int tile_shift() { return sizeof(R) == 4 ? 3 : 2; }
template <typename R>
inline Lay lay_plan(int N, int P) {
  constexpr int txs = tile_shift<R>();
  const int K = 1 << kYBlockShift, TX = 1 << txs;
  return {(int64_t)K * P, (int64_t)TX, (int64_t)N * K * P, kYBlockShift, (int64_t)K * TX, txs};
}

// Spectra are complex R pairs; P = row pitch in complex elements (>= N/2+1).
template <typename R>
struct FftPasses {
  using C = typename CT<R>::C;
  static int cols();   // B: kx columns per CTA in the y/z passes
  // X pass, R2C of compact int64 Q32.32 lines: f = q * scale[line_bin].
  static cudaError_t x_r2c_lines(int N, const int64_t* q, const int32_t* line_bin,
                                 const double* scale, int64_t n_lines, C* spec, int P,
                                 const C* tw, cudaStream_t s);
  // X pass, R2C of a dense real mesh [N][N][N].
  static cudaError_t x_r2c_dense(int N, const R* f, C* spec, int P, const C* tw,
                                 cudaStream_t s);
  // Y pass forward over the compact lines of nb meshes (idx == null: dense lines
  // l = z*N + y of one mesh). S[b] = [z][ky][P].
  static cudaError_t y_fwd(int N, int nb, const C* spec, int P, const int32_t* idx,
                           const int64_t* seg_total, const int64_t* line_base,
                           const int32_t* line_y, C* S, int64_t S_stride, Lay L, const C* tw,
                           cudaStream_t s);
  // Z pass forward in place: S[z][ky][kx] -> F[kz][ky][kx].
  // Dense column passes in place (persistent and TMA fed where the pitch
  // allows a tensor map; err receives a device wait timeout)
  static cudaError_t z_fwd(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s);
  // Z pass fused: for each of nb meshes, forward z, times conj(Fg) / N^3
  // (gg: P = |Fg|^2 / N^3 from Fg itself), k = 0 set to zero, inverse z, and
  // only the |z| <= w rows written: Wz[b] = [2w+1][ky][P]. Persistent and
  // TMA fed; S must be [nb][N][N][P] contiguous (S_stride = N*N*P) and P*sizeof(C)
  // a multiple of 16. A bounded wait that gives up sets *err (device) nonzero.
  static cudaError_t z_corr(int N, int nb, const C* S, const C* Fg, bool gg, int w, C* Wz,
                            int64_t Wz_stride, int P, Lay L, const C* tw, int* err, cudaStream_t s);
  // Inverse y on the window rows: Wz[b][zw][ky] -> Wy[b][zw][yw], |y| <= w.
  static cudaError_t y_inv_win(int N, int nb, const C* Wz, int64_t Wz_stride, int w, C* Wy,
                               int64_t Wy_stride, int P, const C* tw, int* err, cudaStream_t s);
  // Inverse x (C2R) on the window lines, x offsets |x| <= w, times `scale`:
  // Cwin[b] = [zw][yw][xw] real, (2w+1)^3 per mesh.
  static cudaError_t x_c2r_win(int N, int nb, const C* Wy, int64_t Wy_stride, int w,
                               R* Cwin, int64_t Cwin_stride, int P, double scale,
                               const C* tw, cudaStream_t s);
  // Dense inverse passes for the stage entry point: full y, full x.
  static cudaError_t z_inv_full(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s);
  static cudaError_t y_inv_full(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s);
  static cudaError_t x_c2r_full(int N, const C* S, int P, R* out, const C* tw,
                                cudaStream_t s);
  static cudaError_t set_smem_limits();
  // Adjoint passes. x R2C of n_lines real lines (line l at f + l*N).
  static cudaError_t x_r2c_real(int N, const R* f, int64_t n_lines, C* spec, int P, const C* tw,
                                cudaStream_t s);
  // Batched adjoint passes over nb pair meshes; window spectra are compact,
  // Xw[b] = [W][N][P] over the window z planes (window rank zr), W = 2w+1.
  // True when the fused passes fit this N and w (shared memory, TMA box).
  static bool adj_fits(int N, int w);
  // Y pass of the window lines (spec line (b*W + zr)*W + ry) into Xw.
  static cudaError_t y_fwd_win(int N, int nb, const C* spec, int P, int w, C* Xw,
                               int64_t Xw_stride, Lay XL, const C* tw, int* err, cudaStream_t s);
  // Both sides of the adjoint z pass: A[kz][ky][kx] += sum_b F_b conj(X_b)
  // (F_b the z transform of S[b], [nb][N][N][P] contiguous; X_b that of
  // Xw[b] zero-padded), and Y_b = inverse z of X_b Fg (k = 0 zeroed) written
  // over S[b].
  static cudaError_t zadj(int N, int nb, C* S, int64_t S_stride, Lay L, const C* Xw,
                          int64_t Xw_stride, Lay XL, const C* Fg, C* A, int w, int P, const C* tw,
                          int* err, cudaStream_t s);
  // A = 2 Re(X) F_g over the half spectrum (layout L), X the z transform of
  // the compact window spectra of mesh 0 of Xw (layout XL, zero outside the
  // W window planes), taken from the W rows alone. Needs err (a bounded TMA
  // wait that runs out sets it to PG_ERR_TIMEOUT's device code).
  static cudaError_t zwin_acc(int N, const C* Xw, int64_t Xw_stride, Lay XL, Lay L, int P, int w,
                              const C* Fg, C* A, const C* tw, int* err, cudaStream_t s);
  // Inverse y of Y[b] at the compact lines of the batch (numbering of the
  // forward deposit: idx, seg_total, line_base, line_y) into hspec[line][P].
  static cudaError_t y_inv_lines(int N, int nb, const C* Y, int64_t Y_stride, Lay L, int P,
                                 const int32_t* idx, const int64_t* seg_total,
                                 const int64_t* line_base, const int32_t* line_y, C* hspec,
                                 const C* tw, int* err, cudaStream_t s);
  // out[l][x] = scale * C2R of row (line_z[l], line_y[l]) of S; line_y ==
  // null: of the compact line S + l*P.
  static cudaError_t x_c2r_lines(int N, const C* S, int P, Lay L, int64_t n_lines, const int32_t* line_y,
                                 const int32_t* line_z, R* out, double scale, const C* tw,
                                 cudaStream_t s);
};

// ---- smooth-W estimator (pg_smooth.cu) ----------------------------------------
// Parameters of the Gauss-sigmoid W of eq. weighting (Mpc/h, h/Mpc).
struct SmoothW {
  double sigma, r_s, s0, r_cut;
};
// Inputs and outputs of the final ratios (all device pointers).
struct SmoothArgs {
  int P, n_mu;
  const double* vbin;              // [P] pair-bin volumes
  double L;
  const unsigned long long* ddq;   // [P] Q32.32 weighted pair counts
  const double* wsum;              // [2] sum w, sum w^2
  const double* pairs;             // [P][2] sum w g, sum w over the bin's pairs
  const double* gal;               // [2] the same over the galaxies
  const double* wc;                // [2] sum W C^2, sum W C over the mesh offsets
  double *xi_ss, *num, *b_pg, *q_eff, *den, *xi_dw;
};
// W on every mesh offset (minimum image), real [z][y][x], line of sight z.
template <typename R>
cudaError_t launch_w_mesh(int N, double dx, const SmoothW& p, R* out, cudaStream_t s);
// out[kz][ky][kx] (pitch P) = scale * A * B (mode 0) or scale * |B|^2 (mode
// 1), k = 0 zeroed; A, B in layout L.
template <typename R>
cudaError_t launch_spec_mul(int N, int P, Lay L, const typename CT<R>::C* A, const typename CT<R>::C* B,
                            int mode, double scale, typename CT<R>::C* out, cudaStream_t s);
// g[k] = dense real field G [z][y][x] at the points, assignment weights.
template <typename R>
cudaError_t launch_interp(const DepGeom& geo, int64_t n, const double* x, const double* y, const double* z,
                          const R* G, double* g, cudaStream_t s);
// Per-segment sums of w g and w (w null: 1), one CTA per segment.
cudaError_t launch_seg_sums(int nseg, const int64_t* off, const double* g, const double* w, double* sums,
                            cudaStream_t s);
// out[0] = sum W C^2, out[1] = sum W C over the mesh offsets; part holds
// 2 * wc_partials(N) doubles (one partial per block of the reduction).
int wc_partials(int N);
template <typename R>
cudaError_t launch_wc_sums(int N, double dx, const SmoothW& p, const R* Cm, double* part, double* out,
                           cudaStream_t s);
cudaError_t launch_smooth_final(const SmoothArgs& a, cudaStream_t s);

// ---- adjoint of the smooth-W estimator (pg_smooth_adj.cu) ------------------------
struct SmoothAdjArgs {
  int P;
  const double* vbin;              // [P] pair-bin volumes
  double L;
  const unsigned long long* ddq;   // [P] Q32.32 weighted pair counts
  const double* wsum;              // [2] sum w, sum w^2
  const double* out;               // forward outputs: xi_ss[P], num[P], b_pg[P], q_eff[P], den, xi_dw
  const double* g;                 // upstream gradients in the same layout (zeros where absent)
  double* sa;                      // out: num bar [P], xi bar [P], RR [P], den bar, xi_w bar, npairs bar
};
cudaError_t launch_sadj_ratios(const SmoothAdjArgs& a, cudaStream_t s);
cudaError_t launch_sadj_pairs(int64_t np, int P, const int32_t* pbin, const double* pw, const double* gp,
                              const int32_t* pi, const int32_t* pj, const double* wgal, const double* psums,
                              const double* out, const double* sa, double* gpbar, double* wbar, cudaStream_t s);
cudaError_t launch_sadj_gbar(int64_t n, int P, const double* sa, const double* gal, const double* wgal,
                             double* gjbar, cudaStream_t s);
template <typename R>
cudaError_t launch_scatter(const DepGeom& geo, int64_t n, const double* x, const double* y, const double* z,
                           const double* v, R* mesh, cudaStream_t s);
template <typename R>
cudaError_t launch_cbar(int N, double dx, const SmoothW& p, const double* wc, const double* sa, int P, R* Cm,
                        cudaStream_t s);
template <typename R>
cudaError_t launch_spec_combine(int N, int P, Lay L, const typename CT<R>::C* Wk, const typename CT<R>::C* A,
                                const typename CT<R>::C* B, const typename CT<R>::C* Fg, double cs, double scale,
                                typename CT<R>::C* out, cudaStream_t s);
cudaError_t launch_sadj_gal(int64_t n, int P, const double* fj, const double* Tsum, const unsigned long long* qsum,
                            double n3, const double* gj, const double* gal, const double* sa, const double* wgal,
                            double* wbar, cudaStream_t s);

// ---- binning and ratios (pg_bin.cu) -----------------------------------------
// Cells per chunk of the binning pass: each list is cut into chunks of at
// most this many cells, summed by one CTA each.
constexpr int kBinChunk = 4096;
inline int bin_chunks(const std::vector<int64_t>& list_off) {
  int64_t n = 0;
  for (size_t l = 0; l + 1 < list_off.size(); ++l) n += (list_off[l + 1] - list_off[l] + kBinChunk - 1) / kBinChunk;
  return (int)n;
}
// Sums C and C^2 over every list of nb window meshes into out [nb][n_lists][2]
// (FP64): per-chunk partial sums into part [nb][n_chunks][2], then each list's
// partials in chunk order, so the result does not depend on scheduling.
template <typename R>
cudaError_t launch_bin_sums(int nb, int n_lists, const R* Cwin, int64_t Cwin_stride,
                            const int32_t* cells, const int64_t* list_off, int n_chunks, double* part,
                            double* out, cudaStream_t s);

// Volume of every pair bin p = k * n_mu + m (the RR normalisation of
// eq. 2PCF_d_collapsed): a (s, mu) bin is 1/n_mu of the spherical shell
// (4 pi / 3)(s_hi^3 - s_lo^3); a (d_perp, d_par) grid cell is the annulus
// pi (p_hi^2 - p_lo^2) times 2 (l_hi - l_lo), both signs of d_par. In grid
// mode wcoef[p] = 2 (l_hi - l_lo), the weight of xi(p) in w(d_perp) (the
// integral over d_par of eq. 2PCF_los_integrated_explicit).
inline void pair_bin_volumes(int grid, int n_s, const double* s_edges, int n_mu, const double* par_edges,
                             std::vector<double>& vbin, std::vector<double>& wcoef) {
  vbin.assign((size_t)n_s * n_mu, 0.0);
  wcoef.assign(grid ? (size_t)n_s * n_mu : 0, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n_s; ++k)
    for (int m = 0; m < n_mu; ++m) {
      const double lo = s_edges[k], hi = s_edges[k + 1];
      if (grid) {
        const double dl = par_edges[m + 1] - par_edges[m];
        vbin[(size_t)k * n_mu + m] = pi * (hi * hi - lo * lo) * (2.0 * dl);
        wcoef[(size_t)k * n_mu + m] = 2.0 * dl;
      } else {
        vbin[(size_t)k * n_mu + m] = (4.0 * pi / 3.0) * (hi * hi * hi - lo * lo * lo) / (double)n_mu;
      }
    }
}

struct RatioArgs {
  int P, Q;                       // pair bins, (r, mu_r) bins
  int n_s, n_mu;
  const double* vbin;             // device [P] pair-bin volumes
  const double* wcoef;            // device [P] weight of xi(p) in w_perp[p / n_mu] (grid), or null
  double L;
  const unsigned long long* dd;   // [P]
  const unsigned long long* ddq;  // [P]
  const double* wsum;             // [2] sum w, sum w^2
  const double* sum_pg;           // [P][Q+1][2]
  const unsigned char* pg_valid;  // [P] 1 if the bin's mesh was correlated
  const double* sum_gg;           // [Q+1][2]
  int gg_valid;
  const int64_t* list_off;        // [Q+2]
  // outputs (device)
  double *dd_w, *xi_ss, *xi_pg, *xi_gg, *b_pg, *q_eff, *q_eff_sq, *xi_dw, *b_pg_agg,
      *q_eff_agg, *xi_dw_agg, *o_sum_pg, *o_sum_pg_agg, *o_sum_gg, *o_sum2_gg, *o_sum_gg_agg, *w_perp;
  int64_t *o_dd, *n_cells, *n_cells_agg;
};
cudaError_t launch_ratios(const RatioArgs& a, cudaStream_t s);

// ---- adjoint (pg_adjoint.cu) ----------------------------------------------------
struct OutSet {   // device arrays with the pg_result layout (any may be null)
  const double *xi_pg, *xi_gg, *b_pg, *q_eff, *q_eff_sq, *xi_dw, *b_pg_agg, *q_eff_agg,
      *xi_dw_agg, *xi_ss, *dd_w, *w_perp;
};
struct AdjRatioArgs {
  int P, Q, n_mu;
  const double* vbin;              // [P] pair-bin volumes
  const double* wcoef;             // [P] weight of xi(p) in w_perp[p / n_mu], or null
  double L;
  const unsigned long long* ddq;
  const double* wsum;
  const double* sum_pg;            // [P][Q+1][2]
  const unsigned char* pg_valid;
  const double* sum_gg;            // [Q+1][2]
  int gg_valid;
  const int64_t* list_off;
  OutSet o;                        // forward outputs (for gating non-finite ones)
  OutSet g;                        // upstream gradients
  double* tmp;                     // [P][Q+1][3] scratch
  double *Sbar, *Gbar, *G2bar, *DDbar, *wsbar;   // [P][Q+1], [Q+1], [Q+1], [P], [2]
};
cudaError_t launch_adjoint_ratios(const AdjRatioArgs& a, cudaStream_t s);
template <typename R>
cudaError_t launch_window_field(int N, int w, const int32_t* cell_bin, const uint8_t* cell_agg, int Q,
                                const double* sbar, const double* gbar, const double* g2bar,
                                const R* cgg, R* lines, cudaStream_t s);
template <typename R>
cudaError_t launch_gather(const DepGeom& geo, int64_t n, const double* x, const double* y,
                          const double* z, const double* wt, const int32_t* idx, const R* lines,
                          double* g, double* partial, double* T, cudaStream_t s);
cudaError_t launch_pair_chain(int64_t np, const double* g, const double* T,
                              const unsigned long long* qsum, double n3, const double* ddbar,
                              const int32_t* pi, const int32_t* pj, const double* wgal,
                              double* wbar, cudaStream_t s);
cudaError_t launch_hod_weights(int64_t n, const double* mass, const int32_t* kind, const float* kh,
                               const double theta[5], float* w, double* dw, double* d2w,
                               cudaStream_t s);

// ---- HOD-parameter derivatives of the pair-count statistics (pg_hod.cu) ----
// Per value: [0] the value, [1..5] d/dtheta_j, [6..20] d2/dtheta_j dtheta_k
// for j <= k in row order (00 01 02 03 04 11 12 13 14 22 23 24 33 34 44).
constexpr int kHodVals = 21;
constexpr int kHodNormBlocks = 256;
// sum w and sum w^2 with their derivatives: partial [kHodNormBlocks][2 * 21]
// then out[2 * 21] (first sum w, then sum w^2), fixed-order sums
cudaError_t launch_hod_norm(int64_t n, const float* w, const double* dw, const double* d2w,
                            double* partial, double* out, cudaStream_t s);
// DD_b = sum over the pairs of bin b of w_i w_j with its derivatives:
// out[P][21]. The bins' pair ranges are cut into chunks of at most
// kHodChunk pairs; chunks = [starts (n_chunks) | ends (n_chunks) | first
// chunk of each bin (P + 1)]; partial [n_chunks][21] scratch. Each bin's
// chunks are added in order (deterministic).
constexpr int64_t kHodChunk = 4096;
cudaError_t launch_hod_pair_sums(int P, int64_t n_chunks, const int64_t* chunks, const int32_t* pi,
                                 const int32_t* pj, const float* w, const double* dw,
                                 const double* d2w, double* partial, double* out, cudaStream_t s);
// xi_b = DD_b / (R vbin_b / L^3) - 1, R = ((sum w)^2 - sum w^2)/2, with its
// derivatives (quotient rule): xi[P][21]; with wcoef (the grid), also
// w(d_perp)_k = sum_m wcoef[k n_mu + m] xi[k n_mu + m]: wp[n_s][21]
cudaError_t launch_hod_xi(int n_s, int n_mu, const double* dd, const double* norm,
                          const double* vbin, const double* wcoef, double inv_L3, double* xi,
                          double* wp, cudaStream_t s);
cudaError_t launch_hod_chain(int64_t n, const double* wbar, const double* dw, double* partial,
                             double* out5, cudaStream_t s);
cudaError_t launch_gal_final(int64_t n, const double* g, const double* T,
                             const unsigned long long* qsum, double n3, const double* wsbar,
                             const double* wgal, double* wbar, cudaStream_t s);

}  // namespace pg
