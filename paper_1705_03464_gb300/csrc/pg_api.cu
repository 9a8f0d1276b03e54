// C ABI of libpairgal: plans, workspace and the forward pipeline.
//
// pg_forward runs the path of Sec. 2.1-2.2 and 3.2-3.6 on one device stream:
//   positions (eq. RSD) -> cell list -> (s, mu) pairs and DD -> galaxy mesh ->
//   galaxy spectrum -> galaxy auto-correlation window -> for each batch of
//   pair bins: midpoint meshes -> spectra -> cross-spectrum with the galaxy
//   spectrum and inverse (z, then y, then x on the |r| <= r_max window) ->
//   (r, mu_r) sums -> ratios.
// Host code only sizes buffers, builds plan geometry (twiddle table, cell
// lists of the window) and launches kernels; every step of the path runs on
// the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <memory>
#include <new>
#include <vector>

#include "pg_internal.cuh"
#include "pg_tma.cuh"

using namespace pg;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  size_t* acct = nullptr;   // if set, growth is booked here instead of the caller's counter
  cudaError_t ensure(size_t want, size_t* total) {
    if (acct) total = acct;
    if (want <= bytes) return cudaSuccess;
    if (p) { cudaFree(p); *total -= bytes; p = nullptr; bytes = 0; }
    if (want == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) { p = nullptr; return e; }
    bytes = want;
    *total += want;
    return cudaSuccess;
  }
  void release(size_t* total) {
    if (acct) total = acct;
    if (p) { cudaFree(p); *total -= bytes; }
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

pg_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PG_OK;
  if (e == cudaErrorMemoryAllocation) return PG_ERR_OOM;
  return PG_ERR_CUDA;
}

#define PG_TRY(expr)                            \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) {                    \
      (void)cudaGetLastError();                 \
      return from_cuda(e_);                     \
    }                                           \
  } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

// Mesh-sized scratch of the forward and backward passes: line buffers,
// spectra, windows, adjoint spectra. Plans of one mesh size and precision on
// one device may share it (pg_plan_create_shared); every call uses it as
// scratch only, so plans that share it must not run concurrently.
struct Workspace {
  int device = 0, N = 0, precision = 0;
  size_t total = 0;
  int64_t cap_lines = -1;
  // count of writes to S (pair spectra, or S used as scratch): a forward
  // records it after its last batch, and the backward of that forward reuses
  // the batch's spectra only if nothing has written S since
  uint64_t s_seq = 0;
  // the same for F_g and the galaxy correlation window cggw (written together
  // by a galaxy pass), which the backward of the last forward reuses
  uint64_t fg_seq = 0;
  DevBuf flags, lidx, seg_total, line_base, n_lines, stmp, line_y, line_bin, line_z, lines_q, qsum,
      scale, spec, S, Fg, Wz, Wy, Cwin, tmpfft, As, Xw, wlines, cggw;
  DevBuf* all_bufs[23] = {&flags, &lidx, &seg_total, &line_base, &n_lines, &stmp, &line_y, &line_bin,
                          &line_z, &lines_q, &qsum, &scale, &spec, &S, &Fg, &Wz, &Wy, &Cwin,
                          &tmpfft, &As, &Xw, &wlines, &cggw};
  Workspace() {
    for (DevBuf* b : all_bufs) b->acct = &total;
  }
  ~Workspace() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    cudaDeviceSynchronize();
    for (DevBuf* b : all_bufs) b->release(&total);
    cudaSetDevice(cur);
  }
};

struct pg_plan {
  explicit pg_plan(std::shared_ptr<Workspace> w)
      : wsp(std::move(w)), flags(wsp->flags), lidx(wsp->lidx), seg_total(wsp->seg_total),
        line_base(wsp->line_base), n_lines(wsp->n_lines), stmp(wsp->stmp), line_y(wsp->line_y),
        line_bin(wsp->line_bin), lines_q(wsp->lines_q), qsum(wsp->qsum), scale(wsp->scale),
        spec(wsp->spec), S(wsp->S), Fg(wsp->Fg), Wz(wsp->Wz), Wy(wsp->Wy), Cwin(wsp->Cwin),
        tmpfft(wsp->tmpfft), line_z(wsp->line_z), wlines(wsp->wlines), As(wsp->As),
        Xw(wsp->Xw), cggw(wsp->cggw), cap_lines(wsp->cap_lines) {}
  std::shared_ptr<Workspace> wsp;
  pg_params prm;
  std::vector<double> s_edges, r_edges, par_edges;
  int device = 0;
  int N = 0, M1 = 0, P = 0;       // mesh, half-spectrum length, row pitch
  int w = 0, W = 0;               // window half size, side
  int nPB = 0, nQ = 0, nL = 0;    // pair bins, (r, mu_r) bins, lists (nQ + 1)
  int nbmax = 1;                  // pair meshes per batch
  double dx = 0.0;
  PairGeom geom;
  size_t total = 0;
  int64_t n_cells_listed = 0;
  int n_bin_chunks = 0;           // chunks of the binning pass over all lists
  std::vector<int64_t> h_list_off;

  // plan geometry
  DevBuf tw, cells, list_off, s_edges_d, vbin_d, wcoef_d;
  // catalogue
  DevBuf in_pos, in_vel, in_w, x, y, z, gw, flag, wpart, wsum;
  DevBuf cell_id, ccount, cstart, ccursor, perm, xs, ys, zs, ws, ctmp, ctot;
  // pairs
  DevBuf dd, ddq, pcursor, ubin, ui, uj, umx, umy, umz, uwp;
  DevBuf pbin, px, py, pz, pw, bcursor;
  // meshes (the workspace's)
  DevBuf &flags, &lidx, &seg_total, &line_base, &n_lines, &stmp, &line_y, &line_bin, &lines_q,
      &qsum, &scale;
  DevBuf &spec, &S, &Fg, &Wz, &Wy, &Cwin, &tmpfft;
  DevBuf sums_pg, sums_gg, pg_valid, bin_part;
  // adjoint: line z, window lines, spectrum A, compact window spectra,
  // galaxy-window correlation, pair galaxy indices, window cell bins,
  // scalar adjoints, upstream gradients, gathers
  DevBuf &line_z, &wlines, &As, &Xw, &cggw;
  DevBuf psi, psj, cell_bin, cell_agg;
  DevBuf adjb, gout, gp, gj, part;
  // HOD-parameter derivatives of the pair counts: bin offsets, sums, partials, outputs
  DevBuf hd;
  // smooth-W estimator: W's spectrum (cached for wk_key), a spectrum of
  // scratch, bin offsets, sums, partial sums and outputs
  DevBuf Wk, Gs, sm_off, sm_sums, sm_part, sm_out;
  SmoothW wk_key{};
  bool wk_valid = false;
  // the last successful pg_forward_smooth call, which pg_backward_smooth
  // differentiates (its G at the points, sums and outputs stay in the plan);
  // adjoint scratch: upstream gradients, scalar adjoints, point adjoints,
  // two dense meshes and two spectra
  bool smooth_ok = false;
  SmoothW smooth_w{};
  int64_t smooth_np = 0;
  DevBuf sa_g, sa_v, sa_gp, sa_gj, sa_fj, sa_mesh, sa_spec;
  // state of the last successful forward call, which pg_backward differentiates
  bool fwd_ok = false, last_has_w = false;
  int64_t last_n = 0;
  std::vector<unsigned long long> last_hdd;
  // the last forward's final pair batch [reuse_b0, reuse_b1), whose spectra
  // stay in S while the workspace's write count equals reuse_seq
  uint64_t reuse_seq = 0;
  int reuse_b0 = -1, reuse_b1 = -1;
  // the workspace's galaxy-pass count after the last forward's galaxy pass
  uint64_t fg_seq_fwd = ~0ull;
  // outputs
  DevBuf out;
  int64_t cap_gal = -1, cap_pairs = -1;
  int64_t& cap_lines;

  // measurement: event pairs around each launch site of a profiled call
  bool prof_on = false;
  std::vector<cudaEvent_t> events;
  struct Rec { int fam; int ev0, ev1; long long launches; };
  std::vector<Rec> recs;
  int next_event = 0;
  double fam_bytes[PG_N_FAMILIES] = {};
  pg_kernel_stat stats[PG_N_FAMILIES] = {};
  int64_t last_launches = 0;
};

std::atomic<long long>& pg::launch_counter() {
  // per host thread: a call counts the launches it issued, also while other
  // threads drive other plans (the multi-stream batch driver)
  static thread_local std::atomic<long long> c{0};
  return c;
}

namespace {

size_t csize(const pg_plan* p) { return p->prm.precision ? sizeof(double2) : sizeof(float2); }
size_t rsize(const pg_plan* p) { return p->prm.precision ? sizeof(double) : sizeof(float); }

const char* kFamNames[PG_N_FAMILIES] = {"positions", "cells", "pairs", "deposit", "fft_x_r2c",
                                        "fft_y_fwd", "fft_z_fwd", "fft_z_corr", "fft_y_inv",
                                        "fft_x_c2r", "bin", "ratios", "adj_ratios",
                                        "adj_window", "adj_z", "adj_y_inv",
                                        "adj_x_c2r", "adj_gather", "adj_galaxy", "smooth"};

// Times the launches issued inside its scope (one kernel family) with a pair
// of CUDA events on the call's stream, and books the family's algorithmic
// bytes. Costs nothing when profiling is off.
struct ProfScope {
  pg_plan* p;
  int fam;
  cudaStream_t s;
  int ev0 = -1;
  long long l0 = 0;
  ProfScope(pg_plan* p_, int fam_, cudaStream_t s_, double bytes) : p(p_), fam(fam_), s(s_) {
    p->fam_bytes[fam] += bytes;
    l0 = launch_counter().load();
    if (!p->prof_on) return;
    ev0 = take();
    if (ev0 >= 0) cudaEventRecord(p->events[ev0], s);
  }
  int take() {
    if (p->next_event >= (int)p->events.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      p->events.push_back(e);
    }
    return p->next_event++;
  }
  ~ProfScope() {
    long long l1 = launch_counter().load();
    if (!p->prof_on || ev0 < 0) {
      p->stats[fam].launches += l1 - l0;
      return;
    }
    int ev1 = take();
    if (ev1 < 0) return;
    cudaEventRecord(p->events[ev1], s);
    p->recs.push_back({fam, ev0, ev1, l1 - l0});
  }
};

void prof_begin(pg_plan* p) {
  p->recs.clear();
  p->next_event = 0;
  for (int f = 0; f < PG_N_FAMILIES; ++f) {
    p->fam_bytes[f] = 0.0;
    memset(&p->stats[f], 0, sizeof(pg_kernel_stat));
    strncpy(p->stats[f].name, kFamNames[f], sizeof(p->stats[f].name) - 1);
  }
}

// After the call's final synchronisation.
void prof_end(pg_plan* p) {
  for (const auto& r : p->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->events[r.ev0], p->events[r.ev1]) == cudaSuccess)
      p->stats[r.fam].ms += ms;
    p->stats[r.fam].launches += r.launches;
  }
  for (int f = 0; f < PG_N_FAMILIES; ++f) p->stats[f].bytes = p->fam_bytes[f];
}

cudaError_t ensure_gal(pg_plan* p, int64_t n) {
  if (n <= p->cap_gal) return cudaSuccess;
  int64_t c = std::max<int64_t>(n, 1);
  size_t* t = &p->total;
  PG_CUDA_TRY(p->x.ensure(8 * c, t));
  PG_CUDA_TRY(p->y.ensure(8 * c, t));
  PG_CUDA_TRY(p->z.ensure(8 * c, t));
  PG_CUDA_TRY(p->gw.ensure(8 * c, t));
  PG_CUDA_TRY(p->cell_id.ensure(4 * c, t));
  PG_CUDA_TRY(p->perm.ensure(4 * c, t));
  PG_CUDA_TRY(p->xs.ensure(8 * c, t));
  PG_CUDA_TRY(p->ys.ensure(8 * c, t));
  PG_CUDA_TRY(p->zs.ensure(8 * c, t));
  PG_CUDA_TRY(p->ws.ensure(4 * c, t));
  p->cap_gal = c;
  return cudaSuccess;
}

cudaError_t ensure_pairs(pg_plan* p, int64_t np) {
  if (np <= p->cap_pairs) return cudaSuccess;
  int64_t c = std::max<int64_t>(np + np / 8, 1024);
  size_t* t = &p->total;
  PG_CUDA_TRY(p->ubin.ensure(4 * c, t));
  PG_CUDA_TRY(p->ui.ensure(4 * c, t));
  PG_CUDA_TRY(p->uj.ensure(4 * c, t));
  PG_CUDA_TRY(p->umx.ensure(8 * c, t));
  PG_CUDA_TRY(p->umy.ensure(8 * c, t));
  PG_CUDA_TRY(p->umz.ensure(8 * c, t));
  PG_CUDA_TRY(p->uwp.ensure(8 * c, t));
  PG_CUDA_TRY(p->pbin.ensure(4 * c, t));
  PG_CUDA_TRY(p->px.ensure(8 * c, t));
  PG_CUDA_TRY(p->py.ensure(8 * c, t));
  PG_CUDA_TRY(p->pz.ensure(8 * c, t));
  PG_CUDA_TRY(p->pw.ensure(8 * c, t));
  PG_CUDA_TRY(p->psi.ensure(4 * c, t));
  PG_CUDA_TRY(p->psj.ensure(4 * c, t));
  p->cap_pairs = c;
  return cudaSuccess;
}

cudaError_t ensure_lines(pg_plan* p, int64_t nl) {
  if (nl <= p->cap_lines) return cudaSuccess;
  int64_t c = std::max<int64_t>(nl, 64);
  size_t* t = &p->total;
  PG_CUDA_TRY(p->line_y.ensure(4 * c, t));
  PG_CUDA_TRY(p->line_bin.ensure(4 * c, t));
  PG_CUDA_TRY(p->line_z.ensure(4 * c, t));
  PG_CUDA_TRY(p->lines_q.ensure(8 * (size_t)c * p->N, t));
  PG_CUDA_TRY(p->spec.ensure(csize(p) * (size_t)c * p->P, t));
  p->cap_lines = c;
  return cudaSuccess;
}

// Shared scratch at the sizes this plan needs. Called by the entry points,
// on the calling thread, never at plan creation: growing a buffer frees the
// old one, which another plan's calls may still be using.
cudaError_t ensure_shared(pg_plan* p) {
  size_t* t = &p->total;
  const int64_t NN = (int64_t)p->N * p->N;
  const int nb = p->nbmax;
  PG_CUDA_TRY(p->flags.ensure((size_t)nb * NN, t));
  PG_CUDA_TRY(p->lidx.ensure(4 * (size_t)nb * NN, t));
  PG_CUDA_TRY(p->seg_total.ensure(8 * nb, t));
  PG_CUDA_TRY(p->line_base.ensure(8 * nb, t));
  PG_CUDA_TRY(p->n_lines.ensure(8, t));
  PG_CUDA_TRY(p->stmp.ensure(8 * scan_tmp_elems(NN, nb), t));
  PG_CUDA_TRY(p->qsum.ensure(8 * nb, t));
  PG_CUDA_TRY(p->scale.ensure(8 * nb, t));
  const size_t plane = csize(p) * (size_t)NN * p->P;
  const void* s_before = p->S.p;
  PG_CUDA_TRY(p->S.ensure(plane * nb, t));
  if (p->S.p != s_before) ++p->wsp->s_seq;   // contents gone
  const void* fg_before = p->Fg.p;
  const void* cg_before = p->cggw.p;
  PG_CUDA_TRY(p->Fg.ensure(plane, t));
  PG_CUDA_TRY(p->cggw.ensure(rsize(p) * (size_t)p->W * p->W * p->W, t));
  if (p->Fg.p != fg_before || p->cggw.p != cg_before) ++p->wsp->fg_seq;   // contents gone
  PG_CUDA_TRY(p->Wz.ensure(csize(p) * (size_t)p->W * p->N * p->P * nb, t));
  PG_CUDA_TRY(p->Wy.ensure(csize(p) * (size_t)p->W * p->W * p->P * nb, t));
  PG_CUDA_TRY(p->Cwin.ensure(rsize(p) * (size_t)p->W * p->W * p->W * nb, t));
  return cudaSuccess;
}

// Buffers whose size depends only on the plan.
cudaError_t ensure_fixed(pg_plan* p) {
  size_t* t = &p->total;
  const int64_t NN = (int64_t)p->N * p->N;
  const int64_t ncell = (int64_t)p->geom.nc * p->geom.nc * p->geom.nc;
  const int nb = p->nbmax;
  PG_CUDA_TRY(p->flag.ensure(64, t));
  PG_CUDA_TRY(p->wpart.ensure(sizeof(double) * 2 * 256, t));
  PG_CUDA_TRY(p->wsum.ensure(sizeof(double) * 2, t));
  PG_CUDA_TRY(p->ccount.ensure(4 * (ncell + 1), t));
  PG_CUDA_TRY(p->cstart.ensure(4 * (ncell + 1), t));
  PG_CUDA_TRY(p->ccursor.ensure(4 * (ncell + 1), t));
  PG_CUDA_TRY(p->ctmp.ensure(8 * scan_tmp_elems(ncell + 1, 1), t));
  PG_CUDA_TRY(p->ctot.ensure(8, t));
  PG_CUDA_TRY(p->dd.ensure(8 * p->nPB, t));
  PG_CUDA_TRY(p->ddq.ensure(8 * p->nPB, t));
  PG_CUDA_TRY(p->pcursor.ensure(8, t));
  PG_CUDA_TRY(p->bcursor.ensure(8 * p->nPB, t));
  PG_CUDA_TRY(p->sums_pg.ensure(sizeof(double) * 2 * (size_t)p->nPB * p->nL, t));
  PG_CUDA_TRY(p->sums_gg.ensure(sizeof(double) * 2 * (size_t)p->nL, t));
  PG_CUDA_TRY(p->pg_valid.ensure(p->nPB, t));
  PG_CUDA_TRY(p->bin_part.ensure(sizeof(double) * 2 * (size_t)std::max(p->n_bin_chunks, 1) * p->nbmax, t));
  // outputs: doubles [P*Q]*5 + [P]*6 + [Q]*4 + 4, int64 [P] + [Q] + 1
  const size_t nd = (size_t)p->nPB * p->nQ * 5 + (size_t)p->nPB * 6 + (size_t)p->nQ * 4 + 8;
  const size_t ni = (size_t)p->nPB + p->nQ + 2;
  PG_CUDA_TRY(p->out.ensure(sizeof(double) * nd + sizeof(int64_t) * ni, t));
  return cudaSuccess;
}

// Geometry of the (r, mu_r) bins over the offset window [-w, w]^3, with the
// same FP64 comparisons as the binning definition: R2 = a^2+b^2+c^2,
// r^2 = R2 dx^2 against squared edges, mu_r = |c|/sqrt(R2), bin =
// min(n_mur - 1, floor(n_mur mu_r)). List Q holds the aggregate support.
void build_cell_lists(const pg_plan* p, std::vector<int32_t>& cells, std::vector<int64_t>& off) {
  const int w = p->w, W = p->W, nQ = p->nQ, nmur = p->prm.n_mur;
  const double dx2 = p->dx * p->dx;
  std::vector<double> e2(p->r_edges.size());
  for (size_t i = 0; i < e2.size(); ++i) e2[i] = p->r_edges[i] * p->r_edges[i];
  const double cut2 = p->prm.r_perp_cut * p->prm.r_perp_cut;
  std::vector<std::vector<int32_t>> lists(nQ + 1);
  for (int c = -w; c <= w; ++c)
    for (int b = -w; b <= w; ++b)
      for (int a = -w; a <= w; ++a) {
        const int64_t R2 = (int64_t)a * a + (int64_t)b * b + (int64_t)c * c;
        const double r2 = (double)R2 * dx2;
        if (r2 < e2[0] || !(r2 < e2[p->nQ / nmur])) continue;
        int k = 0;
        while (k + 1 < (int)e2.size() - 1 && !(r2 < e2[k + 1])) ++k;
        const double mu = R2 > 0 ? (double)std::abs(c) / sqrt((double)R2) : 0.0;
        int m = (int)floor((double)nmur * mu);
        if (m > nmur - 1) m = nmur - 1;
        const int32_t cell = ((c + w) * W + (b + w)) * W + (a + w);
        lists[k * nmur + m].push_back(cell);
        if (cut2 <= 0.0 || (double)((int64_t)a * a + (int64_t)b * b) * dx2 >= cut2) lists[nQ].push_back(cell);
      }
  off.assign(nQ + 2, 0);
  for (int q = 0; q <= nQ; ++q) off[q + 1] = off[q] + (int64_t)lists[q].size();
  cells.clear();
  cells.reserve(off[nQ + 1]);
  for (int q = 0; q <= nQ; ++q) cells.insert(cells.end(), lists[q].begin(), lists[q].end());
}

template <typename R>
cudaError_t build_twiddles(pg_plan* p) {
  using C = typename CT<R>::C;
  const int N = p->N;
  std::vector<C> h(N);
  for (int j = 0; j < N; ++j) {
    const double a = 2.0 * M_PI * (double)j / (double)N;
    h[j].x = (R)cos(a);
    h[j].y = (R)(-sin(a));
  }
  // exact values at the quarter points
  h[0].x = 1; h[0].y = 0;
  if (N % 4 == 0) {
    h[N / 4].x = 0; h[N / 4].y = -1;
    h[N / 2].x = -1; h[N / 2].y = 0;
    h[3 * N / 4].x = 0; h[3 * N / 4].y = 1;
  }
  PG_CUDA_TRY(p->tw.ensure(sizeof(C) * N, &p->total));
  return cudaMemcpy(p->tw.p, h.data(), sizeof(C) * N, cudaMemcpyHostToDevice);
}

// Deposits one set of points (bins [bin0, bin0 + nb) of a bin-sorted list, or
// one galaxy set when pbin == null) into compact lines and returns the line
// count; leaves per-mesh scale = N^3 / Q in p->scale.
cudaError_t deposit_batch(pg_plan* p, int64_t n, const double* x, const double* y,
                          const double* z, const double* w, const int32_t* pbin, int bin0,
                          int nb, int64_t* n_lines_out, cudaStream_t s) {
  const int64_t NN = (int64_t)p->N * p->N;
  DepGeom g{p->N, p->dx, p->prm.assign};
  int64_t nl = 0;
  {
    // flags + scan + numbering: NN bytes written and read, NN int32 written
    ProfScope ps(p, PG_FAM_DEPOSIT, s, (double)nb * NN * 6 + 32.0 * n);
    PG_CUDA_TRY(cudaMemsetAsync(p->flags.p, 0, (size_t)nb * NN, s));
    PG_CUDA_TRY(launch_mark_lines(g, n, x, y, z, pbin, bin0, p->flags.as<uint8_t>(), s));
    PG_CUDA_TRY(scan_u8_i32(p->flags.as<uint8_t>(), p->lidx.as<int32_t>(), NN, nb,
                            p->seg_total.as<int64_t>(), p->stmp.as<int64_t>(), s));
    PG_CUDA_TRY(launch_line_bases(nb, p->seg_total.as<int64_t>(), p->line_base.as<int64_t>(),
                                  p->n_lines.as<int64_t>(), s));
  }
  PG_CUDA_TRY(cudaMemcpyAsync(&nl, p->n_lines.p, 8, cudaMemcpyDeviceToHost, s));
  PG_CUDA_TRY(cudaStreamSynchronize(s));
  PG_CUDA_TRY(ensure_lines(p, nl));
  {
    ProfScope ps(p, PG_FAM_DEPOSIT, s, (double)nl * p->N * 8 + 40.0 * n * (p->prm.assign == 2 ? 27 : p->prm.assign ? 8 : 1));
    PG_CUDA_TRY(launch_line_compact(p->N, nb, p->flags.as<uint8_t>(), p->lidx.as<int32_t>(),
                                    p->line_base.as<int64_t>(), p->line_y.as<int32_t>(),
                                    p->line_bin.as<int32_t>(), p->line_z.as<int32_t>(), s));
    PG_CUDA_TRY(cudaMemsetAsync(p->lines_q.p, 0, (size_t)nl * p->N * 8, s));
    PG_CUDA_TRY(cudaMemsetAsync(p->qsum.p, 0, 8 * (size_t)nb, s));
    PG_CUDA_TRY(launch_deposit_lines(g, n, x, y, z, w, pbin, bin0, p->lidx.as<int32_t>(),
                                     p->line_base.as<int64_t>(),
                                     p->lines_q.as<unsigned long long>(),
                                     p->qsum.as<unsigned long long>(), s));
    PG_CUDA_TRY(launch_field_scale(nb, p->qsum.as<unsigned long long>(), p->N, p->scale.as<double>(), s));
  }
  *n_lines_out = nl;
  return cudaSuccess;
}

// Spectrum of deposited lines: x pass then y pass into S (nb meshes).
template <typename R>
cudaError_t lines_to_S(pg_plan* p, int nb, int64_t nl, typename CT<R>::C* S, int64_t S_stride,
                       cudaStream_t s) {
  using C = typename CT<R>::C;
  if (S == p->S.as<C>()) ++p->wsp->s_seq;
  const C* tw = p->tw.as<C>();
  const double cs = (double)sizeof(C), M1 = p->M1, N = p->N;
  {
    ProfScope ps(p, PG_FAM_FFT_X_R2C, s, (double)nl * (N * 8.0 + M1 * cs));
    PG_CUDA_TRY(FftPasses<R>::x_r2c_lines(p->N, p->lines_q.as<int64_t>(), p->line_bin.as<int32_t>(),
                                          p->scale.as<double>(), nl, p->spec.as<C>(), p->P, tw, s));
  }
  ProfScope ps(p, PG_FAM_FFT_Y_FWD, s, (double)nl * M1 * cs + (double)nb * N * N * M1 * cs);
  return FftPasses<R>::y_fwd(p->N, nb, p->spec.as<C>(), p->P, p->lidx.as<int32_t>(),
                             p->seg_total.as<int64_t>(), p->line_base.as<int64_t>(),
                             p->line_y.as<int32_t>(), S, S_stride, lay_plan<R>(p->N, p->P), tw, s);
}

// Correlation window of nb meshes against Fg (or Fg with itself) and its bin
// sums into `sums` ([nb][nL][2]).
template <typename R>
cudaError_t correlate_window(pg_plan* p, int nb, bool gg, double* sums, cudaStream_t s) {
  using C = typename CT<R>::C;
  const C* tw = p->tw.as<C>();
  const int64_t S_stride = (int64_t)p->N * p->N * p->P;
  const int64_t Wz_stride = (int64_t)p->W * p->N * p->P;
  const int64_t Wy_stride = (int64_t)p->W * p->W * p->P;
  const int64_t Cw_stride = (int64_t)p->W * p->W * p->W;
  const double inv_n3 = 1.0 / ((double)p->N * p->N * p->N);
  const double cs = (double)sizeof(C), M1 = p->M1, N = p->N, W = p->W;
  {
    // reads each mesh's spectrum once and F_g once (later meshes of the batch
    // find F_g in L2); writes the z window of each mesh
    ProfScope ps(p, PG_FAM_FFT_Z_CORR, s,
                 (gg ? 0.0 : nb * N * N * M1 * cs) + N * N * M1 * cs + nb * W * N * M1 * cs);
    PG_CUDA_TRY(FftPasses<R>::z_corr(p->N, nb, p->S.as<C>(), p->Fg.as<C>(), gg, p->w,
                                     p->Wz.as<C>(), Wz_stride, p->P, lay_plan<R>(p->N, p->P), tw,
                                     p->flag.as<int32_t>() + 1, s));
  }
  {
    ProfScope ps(p, PG_FAM_FFT_Y_INV, s, nb * (W * N * M1 * cs + W * W * M1 * cs));
    PG_CUDA_TRY(FftPasses<R>::y_inv_win(p->N, nb, p->Wz.as<C>(), Wz_stride, p->w, p->Wy.as<C>(),
                                        Wy_stride, p->P, tw, p->flag.as<int32_t>() + 1, s));
  }
  {
    ProfScope ps(p, PG_FAM_FFT_X_C2R, s, nb * (W * W * M1 * cs + W * W * W * (double)sizeof(R)));
    PG_CUDA_TRY(FftPasses<R>::x_c2r_win(p->N, nb, p->Wy.as<C>(), Wy_stride, p->w, p->Cwin.as<R>(),
                                        Cw_stride, p->P, inv_n3, tw, s));
  }
  ProfScope ps(p, PG_FAM_BIN, s, nb * (double)p->n_cells_listed * (4.0 + (double)sizeof(R)));
  return launch_bin_sums<R>(nb, p->nL, p->Cwin.as<R>(), Cw_stride, p->cells.as<int32_t>(),
                            p->list_off.as<int64_t>(), p->n_bin_chunks, p->bin_part.as<double>(), sums, s);
}

// Galaxy spectrum into Fg from points (SoA), then the galaxy window sums.
template <typename R>
cudaError_t galaxy_pass(pg_plan* p, int64_t n, const double* x, const double* y, const double* z,
                        const double* w, bool do_gg, cudaStream_t s) {
  using C = typename CT<R>::C;
  int64_t nl = 0;
  ++p->wsp->fg_seq;
  PG_CUDA_TRY(deposit_batch(p, n, x, y, z, w, nullptr, 0, 1, &nl, s));
  PG_CUDA_TRY(lines_to_S<R>(p, 1, nl, p->Fg.as<C>(), 0, s));
  {
    ProfScope ps(p, PG_FAM_FFT_Z_FWD, s, 2.0 * p->N * p->N * p->M1 * (double)sizeof(C));
    PG_CUDA_TRY(FftPasses<R>::z_fwd(p->N, p->Fg.as<C>(), p->P, lay_plan<R>(p->N, p->P), p->tw.as<C>(),
                                    p->flag.as<int32_t>() + 1, s));
  }
  if (do_gg) PG_CUDA_TRY(correlate_window<R>(p, 1, true, p->sums_gg.as<double>(), s));
  return cudaSuccess;
}

struct OutPtrs {
  double *dd_w, *xi_ss, *xi_pg, *xi_gg, *b_pg, *q_eff, *q_eff_sq, *xi_dw, *b_pg_agg, *q_eff_agg,
      *xi_dw_agg, *sum_pg, *sum_pg_agg, *sum_gg, *sum2_gg, *sum_gg_agg, *w_perp;
  int64_t *dd, *n_cells, *n_cells_agg;
};

// Output arrays carved out of one device block (the forward outputs in
// p->out; the same layout holds the upstream gradients of pg_backward).
OutPtrs out_layout_of(pg_plan* p, double* base) {
  const size_t PQ = (size_t)p->nPB * p->nQ, P = p->nPB, Q = p->nQ;
  double* d = base;
  OutPtrs o;
  o.xi_pg = d; d += PQ;
  o.b_pg = d; d += PQ;
  o.q_eff = d; d += PQ;
  o.q_eff_sq = d; d += PQ;
  o.sum_pg = d; d += PQ;
  o.dd_w = d; d += P;
  o.xi_ss = d; d += P;
  o.b_pg_agg = d; d += P;
  o.q_eff_agg = d; d += P;
  o.sum_pg_agg = d; d += P;
  o.w_perp = d; d += P;   // n_s <= P used
  o.xi_gg = d; d += Q;
  o.xi_dw = d; d += Q;
  o.sum_gg = d; d += Q;
  o.sum2_gg = d; d += Q;
  o.xi_dw_agg = d; d += 1;
  o.sum_gg_agg = d; d += 2;
  d += 5;
  int64_t* i = reinterpret_cast<int64_t*>(d);
  o.dd = i; i += P;
  o.n_cells = i; i += Q;
  o.n_cells_agg = i;
  return o;
}

OutPtrs out_layout(pg_plan* p) { return out_layout_of(p, p->out.as<double>()); }

cudaError_t copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
}

// a1-a3 on device positions; leaves the bin-sorted pair list in p->p*, counts
// in p->dd / p->ddq and the host copy of the counts in hdd.
cudaError_t positions_and_pairs(pg_plan* p, int64_t n, const double* d_pos, const float* d_vel,
                                const float* d_w, std::vector<unsigned long long>& hdd,
                                int64_t* np_out, int* nonfinite, cudaStream_t s) {
  PG_CUDA_TRY(ensure_gal(p, n));
  {
    ProfScope ps(p, PG_FAM_POSITIONS, s, 24.0 * n * 2 + (d_vel ? 12.0 * n : 0.0) + (d_w ? 4.0 * n : 0.0));
    PG_CUDA_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));   // [0] non-finite input, [1] device timeout
    PG_CUDA_TRY(launch_check_finite(n, d_pos, p->flag.as<int32_t>(), s));
    PG_CUDA_TRY(launch_transform(n, p->prm.box_L, p->prm.rsd_factor, d_pos, d_vel, nullptr,
                                 p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), s));
    PG_CUDA_TRY(launch_wsum(n, d_w, p->wpart.as<double>(), p->wsum.as<double>(), s));
  }
  CellList cl{p->cell_id.as<int32_t>(), p->ccount.as<int32_t>(), p->cstart.as<int32_t>(),
              p->ccursor.as<int32_t>(), p->perm.as<int32_t>(), p->xs.as<double>(),
              p->ys.as<double>(), p->zs.as<double>(), p->ws.as<float>(), p->ctmp.as<int64_t>(),
              p->ctot.as<int64_t>()};
  {
    ProfScope ps(p, PG_FAM_CELLS, s, 24.0 * n * 2 + 16.0 * n);
    PG_CUDA_TRY(launch_cells(p->geom, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(),
                             d_w, cl, s));
  }
  PG_CUDA_TRY(cudaMemsetAsync(p->dd.p, 0, 8 * p->nPB, s));
  PG_CUDA_TRY(cudaMemsetAsync(p->ddq.p, 0, 8 * p->nPB, s));
  PairOut po{};
  po.dd = p->dd.as<unsigned long long>();
  po.ddq = p->ddq.as<unsigned long long>();
  {
    ProfScope ps(p, PG_FAM_PAIRS, s, 28.0 * n);
    PG_CUDA_TRY(launch_pairs(p->geom, n, cl, d_w != nullptr, false, po, s));
  }
  hdd.assign(p->nPB, 0ull);
  int32_t hflag = 0;
  PG_CUDA_TRY(cudaMemcpyAsync(hdd.data(), p->dd.p, 8 * p->nPB, cudaMemcpyDeviceToHost, s));
  PG_CUDA_TRY(cudaMemcpyAsync(&hflag, p->flag.p, 4, cudaMemcpyDeviceToHost, s));
  PG_CUDA_TRY(cudaStreamSynchronize(s));
  *nonfinite = hflag;
  int64_t np = 0;
  for (auto v : hdd) np += (int64_t)v;
  *np_out = np;
  PG_CUDA_TRY(ensure_pairs(p, np));
  PG_CUDA_TRY(cudaMemsetAsync(p->pcursor.p, 0, 8, s));
  po.cursor = p->pcursor.as<unsigned long long>();
  po.capacity = p->cap_pairs;
  po.bin = p->ubin.as<int32_t>(); po.i = p->ui.as<int32_t>(); po.j = p->uj.as<int32_t>();
  po.mx = p->umx.as<double>(); po.my = p->umy.as<double>(); po.mz = p->umz.as<double>();
  po.wp = p->uwp.as<double>();
  ProfScope ps(p, PG_FAM_PAIRS, s, 28.0 * n + 2.0 * 44.0 * np);
  PG_CUDA_TRY(launch_pairs(p->geom, n, cl, d_w != nullptr, true, po, s));
  std::vector<unsigned long long> off(p->nPB, 0ull);
  for (int b = 1; b < p->nPB; ++b) off[b] = off[b - 1] + hdd[b - 1];
  PG_CUDA_TRY(cudaMemcpyAsync(p->bcursor.p, off.data(), 8 * p->nPB, cudaMemcpyHostToDevice, s));
  PG_CUDA_TRY(launch_pair_scatter(np, po, p->bcursor.as<unsigned long long>(), p->pbin.as<int32_t>(),
                                  p->psi.as<int32_t>(), p->psj.as<int32_t>(), nullptr,
                                  p->px.as<double>(), p->py.as<double>(),
                                  p->pz.as<double>(), p->pw.as<double>(), s));
  // the scatter reads the host offsets before this function's vector dies
  return cudaStreamSynchronize(s);
}

// Pair-bin batches of at most nbmax contiguous bins for the forward and the
// backward: formed from the last nonempty bin down, so that only the first
// batch can be short (the backward reuses the last, full one), with empty
// bins trimmed off the ends of each batch. Increasing bin order.
std::vector<std::pair<int, int>> bin_batches(const std::vector<unsigned long long>& hdd, int nbmax) {
  std::vector<std::pair<int, int>> out;
  int b1 = (int)hdd.size();
  for (;;) {
    while (b1 > 0 && hdd[b1 - 1] == 0) --b1;
    if (b1 <= 0) break;
    int b0 = std::max(0, b1 - nbmax);
    while (b0 < b1 && hdd[b0] == 0) ++b0;
    out.push_back({b0, b1});
    b1 = b0;
  }
  std::reverse(out.begin(), out.end());
  return out;
}

template <typename R>
pg_status forward_impl(pg_plan* p, int64_t n, const double* d_pos, const float* d_vel,
                       const float* d_w, pg_result* out, cudaStream_t s) {
  std::vector<unsigned long long> hdd;
  int64_t np = 0;
  int nonfinite = 0;
  p->fwd_ok = false;
  p->smooth_ok = false;
  prof_begin(p);
  const long long launches0 = launch_counter().load();
  PG_TRY(positions_and_pairs(p, n, d_pos, d_vel, d_w, hdd, &np, &nonfinite, s));
  if (nonfinite) return PG_ERR_INVALID_ARG;
  // galaxy weights widened to FP64 for the deposit
  const double* gw = nullptr;
  if (d_w) {
    PG_TRY(launch_widen_f32(n, d_w, p->gw.as<double>(), s));
    gw = p->gw.as<double>();
  }
  const bool have_gal = n > 0;
  p->fg_seq_fwd = ~0ull;
  if (have_gal) {
    PG_TRY((galaxy_pass<R>(p, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gw, true, s)));
    // the galaxy window kept for the backward (Cwin is overwritten by the pair batches)
    PG_TRY(cudaMemcpyAsync(p->cggw.p, p->Cwin.p, rsize(p) * (size_t)p->W * p->W * p->W,
                           cudaMemcpyDeviceToDevice, s));
    p->fg_seq_fwd = p->wsp->fg_seq;
  }
  std::vector<unsigned char> valid(p->nPB, 0);
  for (int b = 0; b < p->nPB; ++b) valid[b] = (have_gal && hdd[b] > 0) ? 1 : 0;
  PG_TRY(cudaMemcpyAsync(p->pg_valid.p, valid.data(), p->nPB, cudaMemcpyHostToDevice, s));
  // pair bins in batches of contiguous bin ranges
  std::vector<int64_t> off(p->nPB + 1, 0);
  for (int b = 0; b < p->nPB; ++b) off[b + 1] = off[b] + (int64_t)hdd[b];
  using C = typename CT<R>::C;
  const int64_t S_stride = (int64_t)p->N * p->N * p->P;
  p->reuse_b0 = p->reuse_b1 = -1;
  const auto batches = have_gal ? bin_batches(hdd, p->nbmax) : std::vector<std::pair<int, int>>{};
  for (const auto& bb : batches) {
    const int b0 = bb.first, b1 = bb.second;
    const int nb = b1 - b0;
    const int64_t pn = off[b1] - off[b0];
    int64_t nl = 0;
    PG_TRY(deposit_batch(p, pn, p->px.as<double>() + off[b0], p->py.as<double>() + off[b0],
                         p->pz.as<double>() + off[b0], p->pw.as<double>() + off[b0],
                         p->pbin.as<int32_t>() + off[b0], b0, nb, &nl, s));
    PG_TRY(lines_to_S<R>(p, nb, nl, p->S.as<C>(), S_stride, s));
    PG_TRY(correlate_window<R>(p, nb, false, p->sums_pg.as<double>() + (size_t)b0 * p->nL * 2, s));
    p->reuse_seq = p->wsp->s_seq;   // the correlation only reads S
    p->reuse_b0 = b0;
    p->reuse_b1 = b1;
  }
  // ratios
  OutPtrs o = out_layout(p);
  RatioArgs ra{};
  ra.P = p->nPB; ra.Q = p->nQ; ra.n_s = p->prm.n_s; ra.n_mu = p->prm.n_mu;
  ra.vbin = p->vbin_d.as<double>();
  ra.wcoef = p->prm.pair_grid ? p->wcoef_d.as<double>() : nullptr;
  ra.w_perp = o.w_perp;
  ra.L = p->prm.box_L;
  ra.dd = p->dd.as<unsigned long long>();
  ra.ddq = p->ddq.as<unsigned long long>();
  ra.wsum = p->wsum.as<double>();
  ra.sum_pg = p->sums_pg.as<double>();
  ra.pg_valid = p->pg_valid.as<unsigned char>();
  ra.sum_gg = p->sums_gg.as<double>();
  ra.gg_valid = have_gal ? 1 : 0;
  ra.list_off = p->list_off.as<int64_t>();
  ra.dd_w = o.dd_w; ra.xi_ss = o.xi_ss; ra.xi_pg = o.xi_pg; ra.xi_gg = o.xi_gg; ra.b_pg = o.b_pg;
  ra.q_eff = o.q_eff; ra.q_eff_sq = o.q_eff_sq; ra.xi_dw = o.xi_dw; ra.b_pg_agg = o.b_pg_agg;
  ra.q_eff_agg = o.q_eff_agg; ra.xi_dw_agg = o.xi_dw_agg; ra.o_sum_pg = o.sum_pg;
  ra.o_sum_pg_agg = o.sum_pg_agg; ra.o_sum_gg = o.sum_gg; ra.o_sum2_gg = o.sum2_gg;
  ra.o_sum_gg_agg = o.sum_gg_agg; ra.o_dd = o.dd; ra.n_cells = o.n_cells;
  ra.n_cells_agg = o.n_cells_agg;
  {
    ProfScope ps(p, PG_FAM_RATIOS, s, 0.0);
    PG_TRY(launch_ratios(ra, s));
  }
  if (out) {
    const size_t PQ = sizeof(double) * p->nPB * p->nQ, Pd = sizeof(double) * p->nPB,
                 Qd = sizeof(double) * p->nQ;
    PG_TRY(copy_out(out->dd, o.dd, 8 * p->nPB, s));
    PG_TRY(copy_out(out->dd_w, o.dd_w, Pd, s));
    PG_TRY(copy_out(out->xi_ss, o.xi_ss, Pd, s));
    PG_TRY(copy_out(out->xi_pg, o.xi_pg, PQ, s));
    PG_TRY(copy_out(out->xi_gg, o.xi_gg, Qd, s));
    PG_TRY(copy_out(out->b_pg, o.b_pg, PQ, s));
    PG_TRY(copy_out(out->q_eff, o.q_eff, PQ, s));
    PG_TRY(copy_out(out->q_eff_sq, o.q_eff_sq, PQ, s));
    PG_TRY(copy_out(out->xi_dw, o.xi_dw, Qd, s));
    PG_TRY(copy_out(out->b_pg_agg, o.b_pg_agg, Pd, s));
    PG_TRY(copy_out(out->q_eff_agg, o.q_eff_agg, Pd, s));
    PG_TRY(copy_out(out->xi_dw_agg, o.xi_dw_agg, 8, s));
    PG_TRY(copy_out(out->n_cells, o.n_cells, 8 * p->nQ, s));
    PG_TRY(copy_out(out->n_cells_agg, o.n_cells_agg, 8, s));
    PG_TRY(copy_out(out->sum_pg, o.sum_pg, PQ, s));
    PG_TRY(copy_out(out->sum_pg_agg, o.sum_pg_agg, Pd, s));
    PG_TRY(copy_out(out->sum_gg, o.sum_gg, Qd, s));
    PG_TRY(copy_out(out->sum2_gg, o.sum2_gg, Qd, s));
    PG_TRY(copy_out(out->sum_gg_agg, o.sum_gg_agg, 16, s));
    PG_TRY(copy_out(out->w_perp, o.w_perp, sizeof(double) * p->prm.n_s, s));
  }
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  p->last_launches = launch_counter().load() - launches0;
  if (herr) return PG_ERR_TIMEOUT;
  p->fwd_ok = true;
  p->last_n = n;
  p->last_has_w = d_w != nullptr;
  p->last_hdd = hdd;
  if (p->prof_on) prof_end(p);
  else
    for (int f = 0; f < PG_N_FAMILIES; ++f) p->stats[f].bytes = p->fam_bytes[f];
  return PG_OK;
}

}  // namespace

namespace {

// Plan-time geometry of the adjoint: for every window cell its (r, mu_r) bin
// (-1 if none) and aggregate flag.
cudaError_t build_window_geometry(pg_plan* p, const std::vector<int32_t>& cells) {
  const int W = p->W;
  const int64_t W3 = (int64_t)W * W * W;
  std::vector<int32_t> cb(W3, -1);
  std::vector<uint8_t> ca(W3, 0);
  for (int q = 0; q <= p->nQ; ++q)
    for (int64_t i = p->h_list_off[q]; i < p->h_list_off[q + 1]; ++i) {
      if (q < p->nQ) cb[cells[i]] = q;
      else ca[cells[i]] = 1;
    }
  size_t* t = &p->total;
  PG_CUDA_TRY(p->cell_bin.ensure(4 * W3, t));
  PG_CUDA_TRY(p->cell_agg.ensure(W3, t));
  PG_CUDA_TRY(cudaMemcpy(p->cell_bin.p, cb.data(), 4 * W3, cudaMemcpyHostToDevice));
  return cudaMemcpy(p->cell_agg.p, ca.data(), W3, cudaMemcpyHostToDevice);
}

// The galaxy auto-correlation term of the adjoint, A = 2 Re(X) F_g, X the
// spectrum of the gg window adjoint field (gbar, g2bar and the galaxy
// correlation window): its W^2 window lines through the x pass, the window
// y pass into the compact window spectra (mesh slot 0), and the pruned z
// transform fused with the product with F_g.
template <typename R>
cudaError_t galaxy_window_term(pg_plan* p, const double* gbar, const double* g2bar, int64_t Xw_stride,
                               Lay XL, cudaStream_t s) {
  using C = typename CT<R>::C;
  const C* tw = p->tw.as<C>();
  int* err = p->flag.as<int32_t>() + 1;
  const int64_t nl = (int64_t)p->W * p->W;
  PG_CUDA_TRY(launch_window_field<R>(p->N, p->w, p->cell_bin.as<int32_t>(), p->cell_agg.as<uint8_t>(),
                                     p->nQ, nullptr, gbar, g2bar, p->cggw.as<R>(), p->wlines.as<R>(), s));
  PG_CUDA_TRY(FftPasses<R>::x_r2c_real(p->N, p->wlines.as<R>(), nl, p->spec.as<C>(), p->P, tw, s));
  PG_CUDA_TRY(FftPasses<R>::y_fwd_win(p->N, 1, p->spec.as<C>(), p->P, p->w, p->Xw.as<C>(), Xw_stride, XL,
                                      tw, err, s));
  return FftPasses<R>::zwin_acc(p->N, p->Xw.as<C>(), Xw_stride, XL, lay_plan<R>(p->N, p->P), p->P, p->w,
                                p->Fg.as<C>(), p->As.as<C>(), tw, err, s);
}

// Reverse sweep of the last forward call (see pg_backward in pairgal.h).
template <typename R>
cudaError_t backward_impl(pg_plan* p, const pg_result* gin, double* wbar, cudaStream_t s) {
  using C = typename CT<R>::C;
  const C* tw = p->tw.as<C>();
  const int N = p->N, P = p->nPB, Lq = p->nL;
  const int64_t n = p->last_n;
  const int64_t NN = (int64_t)N * N;
  const int64_t spec_elems = NN * p->P;
  const int64_t W3 = (int64_t)p->W * p->W * p->W;
  const double n3 = (double)N * N * N;
  const double scale6 = 1.0 / (n3 * n3);
  const DepGeom geo{N, p->dx, p->prm.assign};
  size_t* t = &p->total;
  // buffers of the reverse sweep
  int64_t np_max = 0;
  for (auto v : p->last_hdd) np_max = std::max<int64_t>(np_max, (int64_t)v);
  const int W = p->W, nbmax = p->nbmax;
  const int64_t W2 = (int64_t)W * W;
  const int64_t Xw_stride = (int64_t)W * N * p->P;
  const Lay L = lay_plan<R>(N, p->P);
  // compact window spectra [ky / 8][zr][kx / TX][ky % 8][kx % TX] per mesh
  constexpr int txs = tile_shift<R>();
  const Lay XL{(int64_t)8 * p->P, (int64_t)1 << txs, (int64_t)W * 8 * p->P, kYBlockShift,
               (int64_t)8 << txs, txs};
  PG_CUDA_TRY(ensure_lines(p, nbmax * W2));
  PG_CUDA_TRY(p->As.ensure(sizeof(C) * spec_elems, t));
  PG_CUDA_TRY(p->Xw.ensure(sizeof(C) * Xw_stride * nbmax, t));
  PG_CUDA_TRY(p->cggw.ensure(sizeof(R) * W3, t));
  PG_CUDA_TRY(p->wlines.ensure(sizeof(R) * W2 * N * nbmax, t));
  const size_t nadj = (size_t)P * Lq * 4 + 2 * Lq + P + 4;
  PG_CUDA_TRY(p->adjb.ensure(sizeof(double) * nadj, t));
  PG_CUDA_TRY(p->gp.ensure(sizeof(double) * std::max<int64_t>(np_max, 1), t));
  PG_CUDA_TRY(p->gj.ensure(sizeof(double) * std::max<int64_t>(n, 1), t));
  PG_CUDA_TRY(p->part.ensure(sizeof(double) * (cdiv(std::max<int64_t>(std::max(n, np_max), 1), 256) + 4), t));
  double* Sbar = p->adjb.as<double>();
  double* tmp = Sbar + (size_t)P * Lq;
  double* Gbar = tmp + (size_t)P * Lq * 3;
  double* G2bar = Gbar + Lq;
  double* DDbar = G2bar + Lq;
  double* wsbar = DDbar + P;
  double* Tdev = wsbar + 2;
  // upstream gradients to the device, in the forward output layout
  PG_CUDA_TRY(p->gout.ensure(p->out.bytes, t));
  OutPtrs go = out_layout_of(p, p->gout.as<double>());
  OutPtrs fo = out_layout(p);
  const size_t PQ = sizeof(double) * P * p->nQ, Pd = sizeof(double) * P, Qd = sizeof(double) * p->nQ;
  OutSet g{}, o{};
  auto up = [&](const double* h, double* d, size_t bytes, const double*& slot) -> cudaError_t {
    if (!h) { slot = nullptr; return cudaSuccess; }
    slot = d;
    return cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s);
  };
  if (gin) {
    PG_CUDA_TRY(up(gin->xi_pg, go.xi_pg, PQ, g.xi_pg));
    PG_CUDA_TRY(up(gin->xi_gg, go.xi_gg, Qd, g.xi_gg));
    PG_CUDA_TRY(up(gin->b_pg, go.b_pg, PQ, g.b_pg));
    PG_CUDA_TRY(up(gin->q_eff, go.q_eff, PQ, g.q_eff));
    PG_CUDA_TRY(up(gin->q_eff_sq, go.q_eff_sq, PQ, g.q_eff_sq));
    PG_CUDA_TRY(up(gin->xi_dw, go.xi_dw, Qd, g.xi_dw));
    PG_CUDA_TRY(up(gin->b_pg_agg, go.b_pg_agg, Pd, g.b_pg_agg));
    PG_CUDA_TRY(up(gin->q_eff_agg, go.q_eff_agg, Pd, g.q_eff_agg));
    PG_CUDA_TRY(up(gin->xi_dw_agg, go.xi_dw_agg, 8, g.xi_dw_agg));
    PG_CUDA_TRY(up(gin->xi_ss, go.xi_ss, Pd, g.xi_ss));
    PG_CUDA_TRY(up(gin->dd_w, go.dd_w, Pd, g.dd_w));
    if (p->prm.pair_grid) PG_CUDA_TRY(up(gin->w_perp, go.w_perp, sizeof(double) * p->prm.n_s, g.w_perp));
  }
  o = OutSet{fo.xi_pg, fo.xi_gg, fo.b_pg, fo.q_eff, fo.q_eff_sq, fo.xi_dw, fo.b_pg_agg, fo.q_eff_agg,
             fo.xi_dw_agg, fo.xi_ss, fo.dd_w, fo.w_perp};
  AdjRatioArgs ra{};
  ra.P = P; ra.Q = p->nQ; ra.n_mu = p->prm.n_mu;
  ra.vbin = p->vbin_d.as<double>();
  ra.wcoef = p->prm.pair_grid ? p->wcoef_d.as<double>() : nullptr;
  ra.L = p->prm.box_L;
  ra.ddq = p->ddq.as<unsigned long long>();
  ra.wsum = p->wsum.as<double>();
  ra.sum_pg = p->sums_pg.as<double>();
  ra.pg_valid = p->pg_valid.as<unsigned char>();
  ra.sum_gg = p->sums_gg.as<double>();
  ra.gg_valid = n > 0 ? 1 : 0;
  ra.list_off = p->list_off.as<int64_t>();
  ra.o = o;
  ra.g = g;
  ra.tmp = tmp;
  ra.Sbar = Sbar; ra.Gbar = Gbar; ra.G2bar = G2bar; ra.DDbar = DDbar; ra.wsbar = wsbar;
  {
    ProfScope ps(p, PG_FAM_ADJ_RATIOS, s, 0.0);
    PG_CUDA_TRY(launch_adjoint_ratios(ra, s));
  }
  PG_CUDA_TRY(cudaMemsetAsync(wbar, 0, sizeof(double) * std::max<int64_t>(n, 1), s));
  if (n == 0) return cudaSuccess;
  const double* gw = p->last_has_w ? p->gw.as<double>() : nullptr;
  // galaxy spectrum and galaxy correlation window: the forward's, unless a
  // galaxy pass (of any plan sharing the workspace) has run since
  if (p->fg_seq_fwd != p->wsp->fg_seq) {
    PG_CUDA_TRY((galaxy_pass<R>(p, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gw, true, s)));
    PG_CUDA_TRY(cudaMemcpyAsync(p->cggw.p, p->Cwin.p, sizeof(R) * W3, cudaMemcpyDeviceToDevice, s));
    p->fg_seq_fwd = p->wsp->fg_seq;
  }
  const double cs = (double)sizeof(C), rs = (double)sizeof(R), M1 = p->M1, Nd = N;
  {
    // A = 2 Re(F[Cbar_gg]) F_g: F_g read, A written once
    ProfScope ps(p, PG_FAM_ADJ_GALAXY, s, 2.0 * NN * M1 * cs);
    PG_CUDA_TRY(galaxy_window_term<R>(p, Gbar, G2bar, Xw_stride, XL, s));
  }
  // the pair meshes in the forward's batches: S_b recomputed, the compact
  // window spectra X_b, A += F_b conj(X_b), Y_b = z-inverse of X_b F_g over
  // S's memory, its y inverse at the lines of the batch, their x C2R, and the
  // gather at the pairs
  const int64_t S_stride = NN * p->P;
  int* err = p->flag.as<int32_t>() + 1;
  R* hl = reinterpret_cast<R*>(p->lines_q.p);   // the deposit's lines are consumed by the x pass
  std::vector<int64_t> off(P + 1, 0), hbase(nbmax, 0);
  for (int b = 0; b < P; ++b) off[b + 1] = off[b] + (int64_t)p->last_hdd[b];
  // the forward's batches, last first (the adjoint z pass takes the meshes
  // of a batch last first too, so A accumulates in descending bin order for
  // any batching); the first of them is the forward's final batch, whose
  // spectra are still in S unless something has written S since
  const auto batches = bin_batches(p->last_hdd, nbmax);
  for (auto it = batches.rbegin(); it != batches.rend(); ++it) {
    const int b0 = it->first, b1 = it->second;
    const int nb = b1 - b0;
    const bool reuse = it == batches.rbegin() && b0 == p->reuse_b0 && b1 == p->reuse_b1 &&
                       p->reuse_seq == p->wsp->s_seq;
    int64_t nl = 0;
    PG_CUDA_TRY(deposit_batch(p, off[b1] - off[b0], p->px.as<double>() + off[b0],
                              p->py.as<double>() + off[b0], p->pz.as<double>() + off[b0],
                              p->pw.as<double>() + off[b0], p->pbin.as<int32_t>() + off[b0], b0, nb,
                              &nl, s));
    PG_CUDA_TRY(cudaMemcpyAsync(hbase.data(), p->line_base.p, sizeof(int64_t) * nb,
                                cudaMemcpyDeviceToHost, s));
    if (!reuse) PG_CUDA_TRY(lines_to_S<R>(p, nb, nl, p->S.as<C>(), S_stride, s));
    const double dnb = nb, Wd = W, spec1 = NN * M1 * cs, win1 = Wd * Nd * M1 * cs;
    {
      ProfScope ps(p, PG_FAM_ADJ_WINDOW, s,
                   dnb * (2.0 * W2 * Nd * rs + 2.0 * W2 * M1 * cs + win1));
      for (int j = 0; j < nb; ++j)
        PG_CUDA_TRY(launch_window_field<R>(N, p->w, p->cell_bin.as<int32_t>(), p->cell_agg.as<uint8_t>(),
                                           p->nQ, Sbar + (size_t)(b0 + j) * Lq, nullptr, nullptr,
                                           p->cggw.as<R>(), p->wlines.as<R>() + j * W2 * N, s));
      PG_CUDA_TRY(FftPasses<R>::x_r2c_real(N, p->wlines.as<R>(), nb * W2, p->spec.as<C>(), p->P, tw, s));
      PG_CUDA_TRY(FftPasses<R>::y_fwd_win(N, nb, p->spec.as<C>(), p->P, p->w, p->Xw.as<C>(), Xw_stride,
                                          XL, tw, err, s));
    }
    {
      // S and the compact window spectra of every mesh in, Y_b out; A read
      // and written once (F_g from L2, counted once)
      ProfScope ps(p, PG_FAM_ADJ_Z, s, dnb * (2.0 * spec1 + win1) + 3.0 * spec1);
      PG_CUDA_TRY(FftPasses<R>::zadj(N, nb, p->S.as<C>(), S_stride, L, p->Xw.as<C>(), Xw_stride, XL,
                                     p->Fg.as<C>(), p->As.as<C>(), p->w, p->P, tw, err, s));
      ++p->wsp->s_seq;   // Y_b written over S
    }
    {
      // Y_b in (planes that hold lines; counted whole), the lines out
      ProfScope ps(p, PG_FAM_ADJ_Y_INV, s, dnb * spec1 + (double)nl * M1 * cs);
      PG_CUDA_TRY(FftPasses<R>::y_inv_lines(N, nb, p->S.as<C>(), S_stride, L, p->P, p->lidx.as<int32_t>(),
                                            p->seg_total.as<int64_t>(), p->line_base.as<int64_t>(),
                                            p->line_y.as<int32_t>(), p->spec.as<C>(), tw, err, s));
    }
    {
      ProfScope ps(p, PG_FAM_ADJ_X_C2R, s, (double)nl * (M1 * cs + Nd * rs));
      PG_CUDA_TRY(FftPasses<R>::x_c2r_lines(N, p->spec.as<C>(), p->P, L, nl, nullptr, nullptr, hl, scale6,
                                            tw, s));
    }
    PG_CUDA_TRY(cudaStreamSynchronize(s));   // hbase
    ProfScope ps(p, PG_FAM_ADJ_GATHER, s, 96.0 * (double)(off[b1] - off[b0]));
    for (int j = 0; j < nb; ++j) {
      const int b = b0 + j;
      const int64_t npb = (int64_t)p->last_hdd[b], o0 = off[b];
      if (npb == 0) continue;
      PG_CUDA_TRY(launch_gather<R>(geo, npb, p->px.as<double>() + o0, p->py.as<double>() + o0,
                                   p->pz.as<double>() + o0, p->pw.as<double>() + o0,
                                   p->lidx.as<int32_t>() + (size_t)j * NN, hl + hbase[j] * N,
                                   p->gp.as<double>(), p->part.as<double>(), Tdev, s));
      PG_CUDA_TRY(launch_pair_chain(npb, p->gp.as<double>(), Tdev, p->qsum.as<unsigned long long>() + j,
                                    n3, DDbar + b, p->psi.as<int32_t>() + o0, p->psj.as<int32_t>() + o0,
                                    gw, wbar, s));
    }
  }
  // galaxy side: f_g adjoint = N^-6 IDFT[A] at the galaxy lines
  ProfScope ps(p, PG_FAM_ADJ_GALAXY, s, 4.0 * NN * M1 * cs + 96.0 * (double)n);
  PG_CUDA_TRY(FftPasses<R>::z_inv_full(N, p->As.as<C>(), p->P, L, tw, p->flag.as<int32_t>() + 1, s));
  PG_CUDA_TRY(FftPasses<R>::y_inv_full(N, p->As.as<C>(), p->P, L, tw, p->flag.as<int32_t>() + 1, s));
  int64_t nlg = 0;
  PG_CUDA_TRY(deposit_batch(p, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gw, nullptr,
                            0, 1, &nlg, s));
  hl = reinterpret_cast<R*>(p->lines_q.p);   // ensure_lines may have moved it
  PG_CUDA_TRY(FftPasses<R>::x_c2r_lines(N, p->As.as<C>(), p->P, L, nlg, p->line_y.as<int32_t>(),
                                        p->line_z.as<int32_t>(), hl, scale6, tw, s));
  PG_CUDA_TRY(launch_gather<R>(geo, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gw,
                               p->lidx.as<int32_t>(), hl, p->gj.as<double>(), p->part.as<double>(),
                               Tdev, s));
  return launch_gal_final(n, p->gj.as<double>(), Tdev, p->qsum.as<unsigned long long>(), n3, wsbar,
                          gw, wbar, s);
}

// The smooth-W estimator (Sec. 2.1 eq. bpg_final with eq. weighting): one
// convolution G = W * delta_g on the mesh, G at every pair midpoint and
// galaxy, weighted means per pair bin and over the galaxies, xi(d_w) from
// the measured C_gg (eq. xi_dw), and the ratios (eq. Qeff_notsq).
template <typename R>
pg_status smooth_impl(pg_plan* p, const SmoothW& wp, int64_t n, const double* d_pos, const float* d_vel,
                      const float* d_w, pg_smooth_result* out, cudaStream_t s) {
  using C = typename CT<R>::C;
  std::vector<unsigned long long> hdd;
  int64_t np = 0;
  int nonfinite = 0;
  p->fwd_ok = false;
  p->smooth_ok = false;
  prof_begin(p);
  const long long launches0 = launch_counter().load();
  PG_TRY(positions_and_pairs(p, n, d_pos, d_vel, d_w, hdd, &np, &nonfinite, s));
  if (nonfinite) return PG_ERR_INVALID_ARG;
  const int N = p->N, P = p->nPB;
  const int64_t NN = (int64_t)N * N;
  size_t* t = &p->total;
  const double cs = (double)sizeof(C), rs = (double)sizeof(R), spec = (double)NN * p->M1 * cs,
               real_b = (double)NN * N * rs;
  PG_TRY(p->Gs.ensure(sizeof(C) * NN * p->P, t));
  PG_TRY(p->Wk.ensure(sizeof(C) * NN * p->P, t));
  PG_TRY(p->sm_off.ensure(sizeof(int64_t) * (P + 3), t));
  PG_TRY(p->sm_sums.ensure(sizeof(double) * (2 * P + 4), t));
  PG_TRY(p->sm_part.ensure(sizeof(double) * 2 * wc_partials(N), t));
  PG_TRY(p->sm_out.ensure(sizeof(double) * (4 * P + 2), t));
  PG_TRY(p->gp.ensure(sizeof(double) * std::max<int64_t>(np, 1), t));
  PG_TRY(p->gj.ensure(sizeof(double) * std::max<int64_t>(n, 1), t));
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (int b = 0; b < P; ++b) out->dd[b] = (int64_t)hdd[b];
  if (n == 0) {
    for (int b = 0; b < P; ++b) out->xi_ss[b] = out->num[b] = out->b_pg[b] = out->q_eff[b] = nan;
    out->den[0] = out->xi_dw[0] = nan;
    p->last_launches = launch_counter().load() - launches0;
    if (p->prof_on) prof_end(p);
    return PG_OK;
  }
  const double* gw = nullptr;
  if (d_w) {
    PG_TRY(launch_widen_f32(n, d_w, p->gw.as<double>(), s));
    gw = p->gw.as<double>();
  }
  const Lay L = lay_plan<R>(N, p->P), Z = lay_zy(N, p->P);
  const C* tw = p->tw.as<C>();
  R* real = reinterpret_cast<R*>(p->S.p);   // shared scratch: at least one spectrum, so N^3 reals
  ++p->wsp->s_seq;
  C* Gs = p->Gs.as<C>();
  C* Wk = p->Wk.as<C>();
  PG_TRY((galaxy_pass<R>(p, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gw, false, s)));
  {
    ProfScope ps(p, PG_FAM_SMOOTH, s, 9.0 * spec + 2.0 * real_b);
    if (!p->wk_valid || memcmp(&p->wk_key, &wp, sizeof(SmoothW)) != 0) {
      // W's spectrum: W on the mesh offsets, then the dense R2C passes
      PG_TRY(launch_w_mesh<R>(N, p->dx, wp, real, s));
      PG_TRY(FftPasses<R>::x_r2c_dense(N, real, Gs, p->P, tw, s));
      PG_TRY(FftPasses<R>::y_fwd(N, 1, Gs, p->P, nullptr, nullptr, nullptr, nullptr, Wk, 0, L, tw, s));
      PG_TRY(FftPasses<R>::z_fwd(N, Wk, p->P, L, tw, p->flag.as<int32_t>() + 1, s));
      p->wk_key = wp;
      p->wk_valid = true;
    }
    // G = W * delta_g = N^-3 IDFT[W~ F_g] (k = 0 zeroed), dense [z][y][x]
    PG_TRY(launch_spec_mul<R>(N, p->P, L, Wk, p->Fg.as<C>(), 0, 1.0 / ((double)NN * N), Gs, s));
    PG_TRY(FftPasses<R>::z_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<R>::y_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<R>::x_c2r_full(N, Gs, p->P, real, tw, s));
    // G at the galaxies and at the pair midpoints (grouped by bin)
    const DepGeom geo{N, p->dx, p->prm.assign};
    PG_TRY(launch_interp<R>(geo, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), real,
                            p->gj.as<double>(), s));
    PG_TRY(launch_interp<R>(geo, np, p->px.as<double>(), p->py.as<double>(), p->pz.as<double>(), real,
                            p->gp.as<double>(), s));
    std::vector<int64_t> off(P + 3, 0);
    for (int b = 0; b < P; ++b) off[b + 1] = off[b] + (int64_t)hdd[b];
    off[P + 1] = 0;
    off[P + 2] = n;
    int64_t* doff = p->sm_off.as<int64_t>();
    PG_TRY(cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (P + 3), cudaMemcpyHostToDevice, s));
    double* sums = p->sm_sums.as<double>();
    PG_TRY(launch_seg_sums(P, doff, p->gp.as<double>(), p->pw.as<double>(), sums, s));
    PG_TRY(launch_seg_sums(1, doff + P + 1, p->gj.as<double>(), gw, sums + 2 * P, s));
    // C_gg = N^-6 IDFT[|F_g|^2] (k = 0 zeroed), then sum W C^2 and sum W C
    PG_TRY(launch_spec_mul<R>(N, p->P, L, nullptr, p->Fg.as<C>(), 1, 1.0 / ((double)NN * NN * NN), Gs, s));
    PG_TRY(FftPasses<R>::z_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<R>::y_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<R>::x_c2r_full(N, Gs, p->P, real, tw, s));
    PG_TRY(launch_wc_sums<R>(N, p->dx, wp, real, p->sm_part.as<double>(), sums + 2 * P + 2, s));
    double* o = p->sm_out.as<double>();
    SmoothArgs a{};
    a.P = P;
    a.n_mu = p->prm.n_mu;
    a.vbin = p->vbin_d.as<double>();
    a.L = p->prm.box_L;
    a.ddq = p->ddq.as<unsigned long long>();
    a.wsum = p->wsum.as<double>();
    a.pairs = sums;
    a.gal = sums + 2 * P;
    a.wc = sums + 2 * P + 2;
    a.xi_ss = o;
    a.num = o + P;
    a.b_pg = o + 2 * P;
    a.q_eff = o + 3 * P;
    a.den = o + 4 * P;
    a.xi_dw = o + 4 * P + 1;
    PG_TRY(launch_smooth_final(a, s));
  }
  std::vector<double> h(4 * P + 2);
  PG_TRY(cudaMemcpyAsync(h.data(), p->sm_out.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  if (herr) return PG_ERR_TIMEOUT;
  for (int b = 0; b < P; ++b) {
    out->xi_ss[b] = h[b];
    out->num[b] = h[P + b];
    out->b_pg[b] = h[2 * P + b];
    out->q_eff[b] = h[3 * P + b];
  }
  out->den[0] = h[4 * P];
  out->xi_dw[0] = h[4 * P + 1];
  p->smooth_ok = true;
  p->smooth_w = wp;
  p->smooth_np = np;
  p->last_n = n;
  p->last_has_w = d_w != nullptr;
  p->last_launches = launch_counter().load() - launches0;
  if (p->prof_on) prof_end(p);
  else
    for (int f = 0; f < PG_N_FAMILIES; ++f) p->stats[f].bytes = p->fam_bytes[f];
  return PG_OK;
}

// Reverse sweep of the last pg_forward_smooth call (see pg_backward_smooth in
// pairgal.h): ratio adjoints -> pair terms, their weight chain and the
// adjoint weights of G at the points -> their deposit -> in k space the
// W convolution of that mesh plus the xi_w term 2/N^3 Cbar * delta -> fbar ->
// the rho / Q chain at the galaxies.
template <typename R>
cudaError_t smooth_backward_impl(pg_plan* p, const pg_smooth_result* gin, double* wbar, cudaStream_t s) {
  using C = typename CT<R>::C;
  const C* tw = p->tw.as<C>();
  const int N = p->N, P = p->nPB;
  const int64_t n = p->last_n, np = p->smooth_np;
  const int64_t NN = (int64_t)N * N, N3 = NN * N, spec = NN * p->P;
  const double n3 = (double)N3;
  size_t* t = &p->total;
  PG_CUDA_TRY(p->sa_g.ensure(sizeof(double) * (4 * P + 2), t));
  PG_CUDA_TRY(p->sa_v.ensure(sizeof(double) * (3 * P + 5), t));
  PG_CUDA_TRY(p->sa_gp.ensure(sizeof(double) * std::max<int64_t>(np, 1), t));
  PG_CUDA_TRY(p->sa_gj.ensure(sizeof(double) * std::max<int64_t>(n, 1), t));
  PG_CUDA_TRY(p->sa_fj.ensure(sizeof(double) * std::max<int64_t>(n, 1), t));
  PG_CUDA_TRY(p->sa_mesh.ensure(sizeof(R) * 2 * N3, t));
  PG_CUDA_TRY(p->sa_spec.ensure(sizeof(C) * 2 * spec, t));
  // upstream gradients in the forward output layout, zeros where absent
  std::vector<double> hg(4 * P + 2, 0.0);
  auto put = [&](const double* src, int off, int cnt) {
    if (src)
      for (int i = 0; i < cnt; ++i) hg[off + i] = src[i];
  };
  if (gin) {
    put(gin->xi_ss, 0, P);
    put(gin->num, P, P);
    put(gin->b_pg, 2 * P, P);
    put(gin->q_eff, 3 * P, P);
    put(gin->den, 4 * P, 1);
    put(gin->xi_dw, 4 * P + 1, 1);
  }
  PG_CUDA_TRY(cudaMemcpyAsync(p->sa_g.p, hg.data(), sizeof(double) * hg.size(), cudaMemcpyHostToDevice, s));
  const double* wgal = p->last_has_w ? p->gw.as<double>() : nullptr;
  const double cs = (double)sizeof(C), rs = (double)sizeof(R);
  ProfScope ps(p, PG_FAM_SMOOTH, s, 14.0 * spec * cs + 8.0 * N3 * rs);
  // the galaxy spectrum and its Q again: the workspace's F_g and mesh totals
  // may have served another plan since the forward
  PG_CUDA_TRY((galaxy_pass<R>(p, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), wgal, false, s)));
  double* sa = p->sa_v.as<double>();
  const double* sums = p->sm_sums.as<double>();   // pairs [P][2], galaxies [2], sum W C^2, sum W C
  SmoothAdjArgs a{};
  a.P = P;
  a.vbin = p->vbin_d.as<double>();
  a.L = p->prm.box_L;
  a.ddq = p->ddq.as<unsigned long long>();
  a.wsum = p->wsum.as<double>();
  a.out = p->sm_out.as<double>();
  a.g = p->sa_g.as<double>();
  a.sa = sa;
  PG_CUDA_TRY(launch_sadj_ratios(a, s));
  PG_CUDA_TRY(cudaMemsetAsync(wbar, 0, sizeof(double) * std::max<int64_t>(n, 1), s));
  PG_CUDA_TRY(launch_sadj_pairs(np, P, p->pbin.as<int32_t>(), p->pw.as<double>(), p->gp.as<double>(),
                                p->psi.as<int32_t>(), p->psj.as<int32_t>(), wgal, sums, p->sm_out.as<double>(), sa,
                                p->sa_gp.as<double>(), wbar, s));
  PG_CUDA_TRY(launch_sadj_gbar(n, P, sa, sums + 2 * P, wgal, p->sa_gj.as<double>(), s));
  // the adjoint weights of G deposited on the mesh (transpose of the interpolation)
  R* gbar = p->sa_mesh.as<R>();
  R* cbar = gbar + N3;
  PG_CUDA_TRY(cudaMemsetAsync(gbar, 0, sizeof(R) * N3, s));
  const DepGeom geo{N, p->dx, p->prm.assign};
  PG_CUDA_TRY(launch_scatter<R>(geo, np, p->px.as<double>(), p->py.as<double>(), p->pz.as<double>(),
                                p->sa_gp.as<double>(), gbar, s));
  PG_CUDA_TRY(launch_scatter<R>(geo, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(),
                                p->sa_gj.as<double>(), gbar, s));
  // C = N^-6 IDFT[|F_g|^2] (k = 0 zeroed) again, then Cbar over it
  const Lay L = lay_plan<R>(N, p->P), Z = lay_zy(N, p->P);
  C* Gs = p->Gs.as<C>();
  PG_CUDA_TRY(launch_spec_mul<R>(N, p->P, L, nullptr, p->Fg.as<C>(), 1, 1.0 / (n3 * n3), Gs, s));
  PG_CUDA_TRY(FftPasses<R>::z_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
  PG_CUDA_TRY(FftPasses<R>::y_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
  PG_CUDA_TRY(FftPasses<R>::x_c2r_full(N, Gs, p->P, cbar, tw, s));
  PG_CUDA_TRY(launch_cbar<R>(N, p->dx, p->smooth_w, sums + 2 * P + 2, sa, P, cbar, s));
  // spectra of Gbar and Cbar in the plan layout
  C* A = p->sa_spec.as<C>();
  C* B = A + spec;
  const R* meshes[2] = {gbar, cbar};
  C* specs[2] = {A, B};
  for (int k = 0; k < 2; ++k) {
    PG_CUDA_TRY(FftPasses<R>::x_r2c_dense(N, meshes[k], Gs, p->P, tw, s));
    PG_CUDA_TRY(FftPasses<R>::y_fwd(N, 1, Gs, p->P, nullptr, nullptr, nullptr, nullptr, specs[k], 0, L, tw, s));
    PG_CUDA_TRY(FftPasses<R>::z_fwd(N, specs[k], p->P, L, tw, p->flag.as<int32_t>() + 1, s));
  }
  // fbar = N^-3 IDFT[W~ F[Gbar] + (2 / N^3) F[Cbar] F_g], k = 0 zeroed, into the first mesh
  PG_CUDA_TRY(launch_spec_combine<R>(N, p->P, L, p->Wk.as<C>(), A, B, p->Fg.as<C>(), 2.0 / n3, 1.0 / n3, Gs, s));
  PG_CUDA_TRY(FftPasses<R>::z_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
  PG_CUDA_TRY(FftPasses<R>::y_inv_full(N, Gs, p->P, Z, tw, p->flag.as<int32_t>() + 1, s));
  PG_CUDA_TRY(FftPasses<R>::x_c2r_full(N, Gs, p->P, gbar, tw, s));
  // fbar at the galaxies, T = sum_j w_j fbar(x_j) (sm_off + P + 1 holds {0, n}), the rho / Q chain
  PG_CUDA_TRY(launch_interp<R>(geo, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), gbar,
                               p->sa_fj.as<double>(), s));
  PG_CUDA_TRY(launch_seg_sums(1, p->sm_off.as<int64_t>() + P + 1, p->sa_fj.as<double>(), wgal, sa + 3 * P + 3, s));
  PG_CUDA_TRY(launch_sadj_gal(n, P, p->sa_fj.as<double>(), sa + 3 * P + 3, p->qsum.as<unsigned long long>(), n3,
                              p->gj.as<double>(), sums + 2 * P, sa, wgal, wbar, s));
  return cudaStreamSynchronize(s);   // hg
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char* pg_status_string(pg_status s) {
  switch (s) {
    case PG_OK: return "ok";
    case PG_ERR_INVALID_ARG: return "invalid argument";
    case PG_ERR_UNSUPPORTED: return "unsupported configuration";
    case PG_ERR_OOM: return "device out of memory";
    case PG_ERR_CUDA: return "CUDA error";
    case PG_ERR_TIMEOUT: return "device wait timed out";
    case PG_ERR_UNIMPLEMENTED: return "not implemented";
    case PG_ERR_CAPACITY: return "output buffer too small";
  }
  return "unknown status";
}

}  // extern "C"

namespace {
pg_status plan_create(const pg_params* prm, const pg_plan* share, pg_plan** out) {
  if (!prm || !out) return PG_ERR_INVALID_ARG;
  *out = nullptr;
  const pg_params& q = *prm;
  if (!(q.box_L > 0.0) || !isfinite(q.box_L)) return PG_ERR_INVALID_ARG;
  if (q.n_s < 1 || q.n_s > 64 || q.n_mu < 1 || q.n_mu > 64 || q.n_r < 1 || q.n_r > 64 ||
      q.n_mur < 1 || q.n_mur > 64 || !q.s_edges || !q.r_edges)
    return PG_ERR_INVALID_ARG;
  if (q.assign < 0 || q.assign > 2) return PG_ERR_INVALID_ARG;
  if (q.precision != 0 && q.precision != 1) return PG_ERR_INVALID_ARG;
  if (!is_pow2(q.mesh_n) || q.mesh_n < 32 || q.mesh_n > 1024) return PG_ERR_UNSUPPORTED;
  for (int i = 0; i < q.n_s; ++i)
    if (!(q.s_edges[i] < q.s_edges[i + 1]) || !(q.s_edges[0] >= 0.0)) return PG_ERR_INVALID_ARG;
  for (int i = 0; i < q.n_r; ++i)
    if (!(q.r_edges[i] < q.r_edges[i + 1]) || !(q.r_edges[0] >= 0.0)) return PG_ERR_INVALID_ARG;
  if (!(q.s_edges[q.n_s] < 0.5 * q.box_L) || !(q.r_edges[q.n_r] < 0.5 * q.box_L))
    return PG_ERR_INVALID_ARG;
  if (q.pair_grid != 0 && q.pair_grid != 1) return PG_ERR_INVALID_ARG;
  if (q.pair_grid) {
    if (!q.par_edges || !(q.par_edges[0] >= 0.0)) return PG_ERR_INVALID_ARG;
    for (int i = 0; i < q.n_mu; ++i)
      if (!(q.par_edges[i] < q.par_edges[i + 1])) return PG_ERR_INVALID_ARG;
    const double pm = q.s_edges[q.n_s], lm = q.par_edges[q.n_mu];
    if (!(sqrt(pm * pm + lm * lm) < 0.5 * q.box_L)) return PG_ERR_INVALID_ARG;
  }
  if (!isfinite(q.rsd_factor) || !(q.r_perp_cut >= 0.0)) return PG_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  std::shared_ptr<Workspace> ws;
  if (share) {
    ws = share->wsp;
    if (ws->device != dev || ws->N != q.mesh_n || ws->precision != q.precision) return PG_ERR_INVALID_ARG;
  } else {
    ws = std::shared_ptr<Workspace>(new (std::nothrow) Workspace());
    if (!ws) return PG_ERR_OOM;
    ws->device = dev;
    ws->N = q.mesh_n;
    ws->precision = q.precision;
  }
  pg_plan* p = new (std::nothrow) pg_plan(ws);
  if (!p) return PG_ERR_OOM;
  p->prm = q;
  p->s_edges.assign(q.s_edges, q.s_edges + q.n_s + 1);
  p->r_edges.assign(q.r_edges, q.r_edges + q.n_r + 1);
  p->prm.s_edges = p->s_edges.data();
  p->prm.r_edges = p->r_edges.data();
  if (q.pair_grid) p->par_edges.assign(q.par_edges, q.par_edges + q.n_mu + 1);
  p->prm.par_edges = q.pair_grid ? p->par_edges.data() : nullptr;
  cudaGetDevice(&p->device);
  p->N = q.mesh_n;
  p->M1 = p->N / 2 + 1;
  // row pitch: a multiple of 64 bytes, so that every 64-byte tile row a TMA
  // box reads is one aligned DRAM access
  {
    const int per64 = q.precision ? 4 : 8;   // complex elements per 64 bytes
    p->P = (p->M1 + per64 - 1) / per64 * per64;
  }
  p->dx = q.box_L / (double)q.mesh_n;
  const double r_max = q.r_edges[q.n_r];
  p->w = (int)ceil(r_max / p->dx);
  p->W = 2 * p->w + 1;
  if (p->W > p->N || p->w >= p->N / 2) { delete p; return PG_ERR_INVALID_ARG; }
  p->nPB = q.n_s * q.n_mu;
  p->nQ = q.n_r * q.n_mur;
  p->nL = p->nQ + 1;
  const double plane = (double)(q.precision ? 16 : 8) * p->N * p->N * p->P;
  int nb = q.bins_per_batch;
  if (nb <= 0) nb = (int)std::max(1.0, std::min(16.0, 72e9 / plane));
  if (q.precision == 1 && q.bins_per_batch <= 0) nb = 1;
  p->nbmax = std::min(nb, std::min(p->nPB, 64));
  // cell list for pairs: cells of side >= s_max (slightly larger, for rounding)
  PairGeom& g = p->geom;
  memset(&g, 0, sizeof(g));
  g.L = q.box_L;
  g.halfL = 0.5 * q.box_L;
  // largest pair separation: s_max, or on the grid the corner of the
  // (d_perp, d_par) cylinder
  const double smax = q.pair_grid ? sqrt(q.s_edges[q.n_s] * q.s_edges[q.n_s] + q.par_edges[q.n_mu] * q.par_edges[q.n_mu])
                                  : q.s_edges[q.n_s];
  // clamped in FP64 before the conversion: a tiny s_max gives a ratio far
  // above INT_MAX
  const double ncr = floor(q.box_L / (smax * (1.0 + 1e-9)));
  int nc = ncr > 256.0 ? 256 : (int)ncr;
  if (nc < 3) nc = 1;
  g.nc = nc;
  g.cell_scale = (double)nc / q.box_L;
  g.n_s = q.n_s;
  g.n_mu = q.n_mu;
  for (int i = 0; i <= q.n_s; ++i) g.e2[i] = q.s_edges[i] * q.s_edges[i];
  g.grid = q.pair_grid;
  if (q.pair_grid)
    for (int i = 0; i <= q.n_mu; ++i) g.pe[i] = q.par_edges[i];
  cudaError_t e = q.precision ? build_twiddles<double>(p) : build_twiddles<float>(p);
  std::vector<int32_t> cells;
  build_cell_lists(p, cells, p->h_list_off);
  p->n_cells_listed = (int64_t)cells.size();
  p->n_bin_chunks = bin_chunks(p->h_list_off);
  if (e == cudaSuccess) e = build_window_geometry(p, cells);
  if (e == cudaSuccess) e = p->cells.ensure(4 * std::max<size_t>(cells.size(), 1), &p->total);
  if (e == cudaSuccess && !cells.empty())
    e = cudaMemcpy(p->cells.p, cells.data(), 4 * cells.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = p->list_off.ensure(8 * p->h_list_off.size(), &p->total);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->list_off.p, p->h_list_off.data(), 8 * p->h_list_off.size(), cudaMemcpyHostToDevice);
  {
    std::vector<double> vb, wc;
    pair_bin_volumes(q.pair_grid, q.n_s, q.s_edges, q.n_mu, q.par_edges, vb, wc);
    if (e == cudaSuccess) e = p->vbin_d.ensure(8 * vb.size(), &p->total);
    if (e == cudaSuccess) e = cudaMemcpy(p->vbin_d.p, vb.data(), 8 * vb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && q.pair_grid) e = p->wcoef_d.ensure(8 * wc.size(), &p->total);
    if (e == cudaSuccess && q.pair_grid)
      e = cudaMemcpy(p->wcoef_d.p, wc.data(), 8 * wc.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = p->s_edges_d.ensure(8 * p->s_edges.size(), &p->total);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->s_edges_d.p, p->s_edges.data(), 8 * p->s_edges.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ensure_fixed(p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    pg_plan_destroy(p);
    return from_cuda(e);
  }
  *out = p;
  return PG_OK;
}
}  // namespace

extern "C" {

pg_status pg_plan_create(const pg_params* prm, pg_plan** out) { return plan_create(prm, nullptr, out); }

pg_status pg_plan_create_shared(const pg_params* prm, const pg_plan* share_with, pg_plan** out) {
  if (!share_with) return PG_ERR_INVALID_ARG;
  return plan_create(prm, share_with, out);
}

void pg_plan_destroy(pg_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  DevBuf* all[] = {&p->tw, &p->cells, &p->list_off, &p->s_edges_d, &p->vbin_d, &p->wcoef_d, &p->in_pos, &p->in_vel, &p->in_w,
                   &p->x, &p->y, &p->z, &p->gw, &p->flag, &p->wpart, &p->wsum, &p->cell_id, &p->ccount,
                   &p->cstart, &p->ccursor, &p->perm, &p->xs, &p->ys, &p->zs, &p->ws, &p->ctmp,
                   &p->ctot, &p->dd, &p->ddq, &p->pcursor, &p->ubin, &p->ui, &p->uj, &p->umx,
                   &p->umy, &p->umz, &p->uwp, &p->pbin, &p->px, &p->py, &p->pz, &p->pw,
                   &p->bcursor, &p->sums_pg, &p->sums_gg, &p->pg_valid, &p->bin_part, &p->out, &p->psi,
                   &p->psj, &p->cell_bin, &p->cell_agg, &p->adjb, &p->gout, &p->gp, &p->gj, &p->part, &p->Wk, &p->Gs,
                   &p->sm_off, &p->sm_sums, &p->sm_part, &p->sm_out, &p->sa_g, &p->sa_v, &p->sa_gp,
                   &p->sa_gj, &p->sa_fj, &p->sa_mesh, &p->sa_spec, &p->hd};
  for (DevBuf* b : all) b->release(&p->total);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  cudaSetDevice(cur);
  delete p;
}

pg_status pg_plan_reserve(pg_plan* p, int64_t n_gal_max, int64_t n_pairs_max) {
  if (!p || n_gal_max < 0 || n_pairs_max < 0) return PG_ERR_INVALID_ARG;
  PG_TRY(ensure_shared(p));
  PG_TRY(ensure_gal(p, n_gal_max));
  PG_TRY(ensure_pairs(p, n_pairs_max));
  const int64_t NN = (int64_t)p->N * p->N;
  const int64_t per = p->prm.assign == 2 ? 9 : p->prm.assign ? 4 : 1;
  PG_TRY(ensure_lines(p, std::min<int64_t>(NN * p->nbmax, std::max(per * n_gal_max, per * n_pairs_max))));
  return PG_OK;
}

size_t pg_workspace_bytes(const pg_plan* p) { return p ? p->total + p->wsp->total : 0; }

pg_status pg_backward_smooth(pg_plan* p, const pg_smooth_result* grad_out, double* d_grad_w, void* stream) {
  if (!p || !d_grad_w) return PG_ERR_INVALID_ARG;
  if (!p->smooth_ok) return PG_ERR_INVALID_ARG;
  if (p->N > 1024) return PG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(ensure_shared(p));
  prof_begin(p);
  const long long launches0 = launch_counter().load();
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  cudaError_t e = p->prm.precision ? smooth_backward_impl<double>(p, grad_out, d_grad_w, s)
                                   : smooth_backward_impl<float>(p, grad_out, d_grad_w, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return from_cuda(e);
  }
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  p->last_launches = launch_counter().load() - launches0;
  if (herr) return PG_ERR_TIMEOUT;
  if (p->prof_on) prof_end(p);
  return PG_OK;
}

pg_status pg_backward(pg_plan* p, const pg_result* grad_out, double* d_grad_w, void* stream) {
  if (!p || !d_grad_w) return PG_ERR_INVALID_ARG;
  if (!p->fwd_ok) return PG_ERR_INVALID_ARG;
  p->smooth_ok = false;   // the backward reuses the plan's point buffers
  const bool fits = p->prm.precision ? FftPasses<double>::adj_fits(p->N, p->w)
                                     : FftPasses<float>::adj_fits(p->N, p->w);
  if (!fits) return PG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(ensure_shared(p));
  prof_begin(p);
  const long long launches0 = launch_counter().load();
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  cudaError_t e = p->prm.precision ? backward_impl<double>(p, grad_out, d_grad_w, s)
                                   : backward_impl<float>(p, grad_out, d_grad_w, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return from_cuda(e);
  }
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  p->last_launches = launch_counter().load() - launches0;
  if (p->prof_on) prof_end(p);
  else
    for (int f = 0; f < PG_N_FAMILIES; ++f) p->stats[f].bytes = p->fam_bytes[f];
  return herr ? PG_ERR_TIMEOUT : PG_OK;
}

pg_status pg_hod_weights(int64_t n, const double* d_mass, const int32_t* d_kind, const float* d_kh,
                         const double* h_theta, float* d_w, double* d_dw_dtheta, void* stream) {
  if (n < 0 || !h_theta || (n > 0 && (!d_mass || !d_kind || !d_kh || !d_w))) return PG_ERR_INVALID_ARG;
  if (!(h_theta[2] > 0.0)) return PG_ERR_INVALID_ARG;
  PG_TRY(launch_hod_weights(n, d_mass, d_kind, d_kh, h_theta, d_w, d_dw_dtheta, nullptr,
                            static_cast<cudaStream_t>(stream)));
  return PG_OK;
}

pg_status pg_hod_weights2(int64_t n, const double* d_mass, const int32_t* d_kind, const float* d_kh,
                          const double* h_theta, float* d_w, double* d_dw_dtheta,
                          double* d_d2w_dtheta2, void* stream) {
  if (n < 0 || !h_theta || (n > 0 && (!d_mass || !d_kind || !d_kh || !d_w || !d_dw_dtheta || !d_d2w_dtheta2)))
    return PG_ERR_INVALID_ARG;
  if (!(h_theta[2] > 0.0)) return PG_ERR_INVALID_ARG;
  PG_TRY(launch_hod_weights(n, d_mass, d_kind, d_kh, h_theta, d_w, d_dw_dtheta, d_d2w_dtheta2,
                            static_cast<cudaStream_t>(stream)));
  return PG_OK;
}

pg_status pg_hod_pair_derivs(pg_plan* p, int64_t n, const double* d_pos, const float* d_vel,
                             const float* d_w, const double* d_dw_dtheta, const double* d_d2w_dtheta2,
                             double* h_xi, double* h_w_perp, void* stream) {
  if (!p || n < 0 || !h_xi || (n > 0 && (!d_pos || !d_w || !d_dw_dtheta || !d_d2w_dtheta2)))
    return PG_ERR_INVALID_ARG;
  if (p->prm.rsd_factor != 0.0 && n > 0 && !d_vel) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->fwd_ok = false;   // the pair buffers are reused
  p->smooth_ok = false;
  prof_begin(p);
  const long long launches0 = launch_counter().load();
  std::vector<unsigned long long> hdd;
  int64_t np = 0;
  int nonfinite = 0;
  PG_TRY(positions_and_pairs(p, n, d_pos, d_vel, d_w, hdd, &np, &nonfinite, s));
  if (nonfinite) return PG_ERR_INVALID_ARG;
  const int P = p->nPB, n_s = p->prm.n_s;
  // each bin's pair range [off_b, off_b + hdd_b) cut into chunks of kHodChunk
  std::vector<int64_t> cstart, cend, cfirst(P + 1, 0);
  {
    int64_t o = 0;
    for (int b = 0; b < P; ++b) {
      cfirst[b] = (int64_t)cstart.size();
      for (int64_t q = o; q < o + (int64_t)hdd[b]; q += kHodChunk) {
        cstart.push_back(q);
        cend.push_back(std::min<int64_t>(q + kHodChunk, o + (int64_t)hdd[b]));
      }
      o += (int64_t)hdd[b];
    }
    cfirst[P] = (int64_t)cstart.size();
  }
  const int64_t nch = (int64_t)cstart.size();
  std::vector<int64_t> chunks;
  chunks.reserve(2 * nch + P + 1);
  chunks.insert(chunks.end(), cstart.begin(), cstart.end());
  chunks.insert(chunks.end(), cend.begin(), cend.end());
  chunks.insert(chunks.end(), cfirst.begin(), cfirst.end());
  // chunk table, pair sums [P][21], chunk partials [nch][21], weight sums
  // [2][21] and their partials, xi [P][21], w_perp [n_s][21]
  const size_t n_ch = chunks.size(), n_dd = (size_t)P * kHodVals, n_pp = (size_t)std::max<int64_t>(nch, 1) * kHodVals,
               n_norm = 2 * kHodVals, n_part = (size_t)kHodNormBlocks * 2 * kHodVals,
               n_xi = (size_t)P * kHodVals, n_wp = (size_t)n_s * kHodVals;
  PG_TRY(p->hd.ensure(8 * (n_ch + n_dd + n_pp + n_norm + n_part + n_xi + n_wp), &p->total));
  int64_t* d_ch = p->hd.as<int64_t>();
  double* d_dd = p->hd.as<double>() + n_ch;
  double* d_pp = d_dd + n_dd;
  double* d_norm = d_pp + n_pp;
  double* d_part = d_norm + n_norm;
  double* d_xi = d_part + n_part;
  double* d_wp = d_xi + n_xi;
  PG_TRY(cudaMemcpyAsync(d_ch, chunks.data(), 8 * n_ch, cudaMemcpyHostToDevice, s));
  {
    ProfScope ps(p, PG_FAM_PAIRS, s, (8.0 + 4.0 * 2 + 2.0 * (4.0 + 40.0 + 120.0)) * (double)np +
                                         (4.0 + 40.0 + 120.0) * (double)n);
    PG_TRY(launch_hod_norm(n, d_w, d_dw_dtheta, d_d2w_dtheta2, d_part, d_norm, s));
    PG_TRY(launch_hod_pair_sums(P, nch, d_ch, p->psi.as<int32_t>(), p->psj.as<int32_t>(), d_w, d_dw_dtheta,
                                d_d2w_dtheta2, d_pp, d_dd, s));
    const double L = p->prm.box_L;
    PG_TRY(launch_hod_xi(n_s, p->prm.n_mu, d_dd, d_norm, p->vbin_d.as<double>(),
                         p->prm.pair_grid ? p->wcoef_d.as<double>() : nullptr, 1.0 / (L * L * L), d_xi,
                         d_wp, s));
  }
  PG_TRY(cudaMemcpyAsync(h_xi, d_xi, 8 * n_xi, cudaMemcpyDeviceToHost, s));
  if (h_w_perp) {
    if (p->prm.pair_grid) {
      PG_TRY(cudaMemcpyAsync(h_w_perp, d_wp, 8 * n_wp, cudaMemcpyDeviceToHost, s));
    } else {
      for (size_t i = 0; i < n_wp; ++i) h_w_perp[i] = std::numeric_limits<double>::quiet_NaN();
    }
  }
  PG_TRY(cudaStreamSynchronize(s));
  p->last_launches = launch_counter().load() - launches0;
  if (p->prof_on) prof_end(p);
  return PG_OK;
}

pg_status pg_hod_chain(pg_plan* p, int64_t n, const double* d_wbar, const double* d_dw_dtheta,
                       double* h_grad_theta, void* stream) {
  if (!p || n < 0 || !h_grad_theta || (n > 0 && (!d_wbar || !d_dw_dtheta))) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(p->part.ensure(sizeof(double) * (5 * (cdiv(std::max<int64_t>(n, 1), 256) + 2)), &p->total));
  double* part = p->part.as<double>();
  const int64_t nblk = std::max<int64_t>(1, cdiv(n, 256));
  PG_TRY(launch_hod_chain(n, d_wbar, d_dw_dtheta, part, part + 5 * nblk, s));
  PG_TRY(cudaMemcpyAsync(h_grad_theta, part + 5 * nblk, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  return PG_OK;
}

pg_status pg_selftest_wait(pg_plan* p, double limit_ms, void* stream) {
  if (!p || !(limit_ms > 0.0) || limit_ms > 5000.0) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  PG_TRY(pg::launch_wait_selftest((uint64_t)(limit_ms * 1e6), p->flag.as<int32_t>() + 1, s));
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  return herr ? PG_ERR_TIMEOUT : PG_OK;
}

pg_status pg_plan_set_profiling(pg_plan* p, int32_t enable) {
  if (!p) return PG_ERR_INVALID_ARG;
  p->prof_on = enable != 0;
  return PG_OK;
}

pg_status pg_plan_last_stats(const pg_plan* p, pg_kernel_stat* out, int64_t* total_launches) {
  if (!p) return PG_ERR_INVALID_ARG;
  if (out) memcpy(out, p->stats, sizeof(p->stats));
  if (total_launches) *total_launches = p->last_launches;
  return PG_OK;
}

pg_status pg_forward(pg_plan* p, int64_t n, const double* d_pos, const float* d_vel,
                     const float* d_w, pg_result* out, void* stream) {
  if (!p || n < 0 || (n > 0 && !d_pos)) return PG_ERR_INVALID_ARG;
  if (p->prm.rsd_factor != 0.0 && n > 0 && !d_vel) return PG_ERR_INVALID_ARG;
  if (n > INT32_MAX / 2) return PG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(ensure_shared(p));
  return p->prm.precision ? forward_impl<double>(p, n, d_pos, d_vel, d_w, out, s)
                          : forward_impl<float>(p, n, d_pos, d_vel, d_w, out, s);
}

pg_status pg_forward_smooth(pg_plan* p, const pg_smooth_params* w, int64_t n, const double* d_pos,
                            const float* d_vel, const float* d_w, pg_smooth_result* out, void* stream) {
  if (!p || !w || !out || n < 0 || (n > 0 && !d_pos)) return PG_ERR_INVALID_ARG;
  if (!out->dd || !out->xi_ss || !out->num || !out->b_pg || !out->q_eff || !out->den || !out->xi_dw)
    return PG_ERR_INVALID_ARG;
  if (!(w->sigma > 0.0) || !isfinite(w->sigma) || !isfinite(w->r_s) || !isfinite(w->s0) ||
      !(w->r_cut >= 0.0) || !isfinite(w->r_cut))
    return PG_ERR_INVALID_ARG;
  if (p->prm.rsd_factor != 0.0 && n > 0 && !d_vel) return PG_ERR_INVALID_ARG;
  if (n > INT32_MAX / 2) return PG_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(ensure_shared(p));
  const SmoothW wp{w->sigma, w->r_s, w->s0, w->r_cut};
  return p->prm.precision ? smooth_impl<double>(p, wp, n, d_pos, d_vel, d_w, out, s)
                          : smooth_impl<float>(p, wp, n, d_pos, d_vel, d_w, out, s);
}

pg_status pg_forward_host(pg_plan* p, int64_t n, const double* h_pos, const float* h_vel,
                          const float* h_w, pg_result* out, void* stream) {
  if (!p || n < 0 || (n > 0 && !h_pos)) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t c = (size_t)std::max<int64_t>(n, 1);
  PG_TRY(p->in_pos.ensure(24 * c, &p->total));
  if (n > 0) PG_TRY(cudaMemcpyAsync(p->in_pos.p, h_pos, 24 * (size_t)n, cudaMemcpyHostToDevice, s));
  const float* dv = nullptr;
  const float* dw = nullptr;
  if (h_vel) {
    PG_TRY(p->in_vel.ensure(12 * c, &p->total));
    if (n > 0) PG_TRY(cudaMemcpyAsync(p->in_vel.p, h_vel, 12 * (size_t)n, cudaMemcpyHostToDevice, s));
    dv = p->in_vel.as<float>();
  }
  if (h_w) {
    PG_TRY(p->in_w.ensure(4 * c, &p->total));
    if (n > 0) PG_TRY(cudaMemcpyAsync(p->in_w.p, h_w, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    dw = p->in_w.as<float>();
  }
  return pg_forward(p, n, p->in_pos.as<double>(), dv, dw, out, stream);
}

pg_status pg_transform_positions(int64_t n, double L, double rsd, const double* d_in,
                                 const float* d_vel, double* d_out, void* stream) {
  if (n < 0 || !(L > 0.0) || (n > 0 && (!d_in || !d_out))) return PG_ERR_INVALID_ARG;
  if (rsd != 0.0 && n > 0 && !d_vel) return PG_ERR_INVALID_ARG;
  PG_TRY(launch_transform(n, L, rsd, d_in, d_vel, d_out, nullptr, nullptr, nullptr,
                          static_cast<cudaStream_t>(stream)));
  return PG_OK;
}

pg_status pg_find_pairs(pg_plan* p, int64_t n, const double* d_pos, const float* d_w,
                        int64_t* d_dd, int64_t* d_ddq, int64_t capacity, int32_t* d_bin,
                        int32_t* d_i, int32_t* d_j, double* d_mid, double* d_wp,
                        int64_t* h_n_pairs, void* stream) {
  if (!p || n < 0 || (n > 0 && !d_pos) || capacity < 0) return PG_ERR_INVALID_ARG;
  if (capacity > 0 && (!d_bin || !d_i || !d_j || !d_mid || !d_wp)) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(ensure_gal(p, n));
  p->fwd_ok = false;   // the plan's pair and position buffers are reused
  p->smooth_ok = false;
  // positions are taken as given (already wrapped); split them to SoA
  PG_TRY(launch_transform(n, p->prm.box_L, 0.0, d_pos, nullptr, nullptr, p->x.as<double>(),
                          p->y.as<double>(), p->z.as<double>(), s));
  CellList cl{p->cell_id.as<int32_t>(), p->ccount.as<int32_t>(), p->cstart.as<int32_t>(),
              p->ccursor.as<int32_t>(), p->perm.as<int32_t>(), p->xs.as<double>(),
              p->ys.as<double>(), p->zs.as<double>(), p->ws.as<float>(), p->ctmp.as<int64_t>(),
              p->ctot.as<int64_t>()};
  PG_TRY(launch_cells(p->geom, n, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), d_w, cl, s));
  PG_TRY(cudaMemsetAsync(p->dd.p, 0, 8 * p->nPB, s));
  PG_TRY(cudaMemsetAsync(p->ddq.p, 0, 8 * p->nPB, s));
  PairOut po{};
  po.dd = p->dd.as<unsigned long long>();
  po.ddq = p->ddq.as<unsigned long long>();
  PG_TRY(launch_pairs(p->geom, n, cl, d_w != nullptr, false, po, s));
  std::vector<unsigned long long> hdd(p->nPB);
  PG_TRY(cudaMemcpyAsync(hdd.data(), p->dd.p, 8 * p->nPB, cudaMemcpyDeviceToHost, s));
  if (d_dd) PG_TRY(cudaMemcpyAsync(d_dd, p->dd.p, 8 * p->nPB, cudaMemcpyDeviceToDevice, s));
  if (d_ddq) PG_TRY(cudaMemcpyAsync(d_ddq, p->ddq.p, 8 * p->nPB, cudaMemcpyDeviceToDevice, s));
  PG_TRY(cudaStreamSynchronize(s));
  int64_t np = 0;
  for (auto v : hdd) np += (int64_t)v;
  if (h_n_pairs) *h_n_pairs = np;
  if (capacity == 0) return PG_OK;
  if (np > capacity) return PG_ERR_CAPACITY;
  PG_TRY(ensure_pairs(p, np));
  PG_TRY(cudaMemsetAsync(p->pcursor.p, 0, 8, s));
  po.cursor = p->pcursor.as<unsigned long long>();
  po.capacity = p->cap_pairs;
  po.bin = p->ubin.as<int32_t>(); po.i = p->ui.as<int32_t>(); po.j = p->uj.as<int32_t>();
  po.mx = p->umx.as<double>(); po.my = p->umy.as<double>(); po.mz = p->umz.as<double>();
  po.wp = p->uwp.as<double>();
  PG_TRY(launch_pairs(p->geom, n, cl, d_w != nullptr, true, po, s));
  std::vector<unsigned long long> off(p->nPB, 0ull);
  for (int b = 1; b < p->nPB; ++b) off[b] = off[b - 1] + hdd[b - 1];
  PG_TRY(cudaMemcpyAsync(p->bcursor.p, off.data(), 8 * p->nPB, cudaMemcpyHostToDevice, s));
  PG_TRY(launch_pair_scatter(np, po, p->bcursor.as<unsigned long long>(), d_bin, d_i, d_j, d_mid,
                             nullptr, nullptr, nullptr, d_wp, s));
  PG_TRY(cudaStreamSynchronize(s));
  return PG_OK;
}

pg_status pg_deposit_dense(int64_t n, const double* d_pts, const double* d_w, double L,
                           int32_t N, int32_t assign, int64_t* d_mesh, void* stream) {
  if (n < 0 || !(L > 0.0) || N < 1 || N > 4096 || assign < 0 || assign > 2 || !d_mesh ||
      (n > 0 && !d_pts))
    return PG_ERR_INVALID_ARG;
  DepGeom g{N, L / (double)N, assign};
  PG_TRY(launch_deposit_dense(g, n, d_pts, d_w, reinterpret_cast<unsigned long long*>(d_mesh),
                              static_cast<cudaStream_t>(stream)));
  return PG_OK;
}

pg_status pg_deposit_lines(pg_plan* p, int64_t n, const double* d_pts, const double* d_w,
                           const int32_t* d_bin, int32_t nb, int64_t* d_mesh, int64_t* h_qsum,
                           int64_t* h_n_lines, void* stream) {
  if (!p || n < 0 || (n > 0 && !d_pts) || !d_mesh || nb < 1 || nb > p->nbmax || (!d_bin && nb != 1))
    return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = p->N;
  PG_TRY(ensure_shared(p));
  PG_TRY(ensure_gal(p, std::max<int64_t>(n, 1)));
  p->fwd_ok = false;   // the plan's line buffers are reused
  p->smooth_ok = false;
  if (d_bin) {   // mesh indices outside [0, nb) would write outside the line flags
    int32_t bad = 0;
    PG_TRY(cudaMemsetAsync(p->flag.p, 0, 4, s));
    PG_TRY(launch_check_bins(n, d_bin, nb, p->flag.as<int32_t>(), s));
    PG_TRY(cudaMemcpyAsync(&bad, p->flag.p, 4, cudaMemcpyDeviceToHost, s));
    PG_TRY(cudaStreamSynchronize(s));
    if (bad) return PG_ERR_INVALID_ARG;
  }
  PG_TRY(cudaMemsetAsync(d_mesh, 0, 8 * (size_t)nb * N * N * N, s));
  PG_TRY(launch_transform(n, p->prm.box_L, 0.0, d_pts, nullptr, nullptr, p->xs.as<double>(),
                          p->ys.as<double>(), p->zs.as<double>(), s));
  int64_t nl = 0;
  PG_TRY(deposit_batch(p, n, p->xs.as<double>(), p->ys.as<double>(), p->zs.as<double>(), d_w,
                       d_bin, 0, nb, &nl, s));
  PG_TRY(launch_lines_scatter(p->N, nl, p->lines_q.as<unsigned long long>(), p->line_y.as<int32_t>(),
                              p->line_z.as<int32_t>(), p->line_bin.as<int32_t>(),
                              reinterpret_cast<unsigned long long*>(d_mesh), s));
  if (h_qsum) PG_TRY(cudaMemcpyAsync(h_qsum, p->qsum.p, 8 * (size_t)nb, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  if (h_n_lines) *h_n_lines = nl;
  return PG_OK;
}

// After a stage entry point's passes: synchronises and reports a device
// wait that gave up (the column passes' bounded TMA waits).
pg_status stage_status(pg_plan* p, cudaStream_t s) {
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  return herr ? PG_ERR_TIMEOUT : PG_OK;
}

pg_status pg_fft_r2c_3d(pg_plan* p, const void* d_in, void* d_out, void* stream) {
  if (!p || !d_in || !d_out) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  const int N = p->N, P = N / 2 + 1;
  if (p->prm.precision) {
    using C = double2;
    PG_TRY(FftPasses<double>::x_r2c_dense(N, (const double*)d_in, (C*)d_out, P, p->tw.as<C>(), s));
    PG_TRY(FftPasses<double>::y_fwd(N, 1, (C*)d_out, P, nullptr, nullptr, nullptr, nullptr, (C*)d_out, 0,
                                    lay_zy(N, P), p->tw.as<C>(), s));
    PG_TRY(FftPasses<double>::z_fwd(N, (C*)d_out, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
  } else {
    using C = float2;
    PG_TRY(FftPasses<float>::x_r2c_dense(N, (const float*)d_in, (C*)d_out, P, p->tw.as<C>(), s));
    PG_TRY(FftPasses<float>::y_fwd(N, 1, (C*)d_out, P, nullptr, nullptr, nullptr, nullptr, (C*)d_out, 0,
                                   lay_zy(N, P), p->tw.as<C>(), s));
    PG_TRY(FftPasses<float>::z_fwd(N, (C*)d_out, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
  }
  return stage_status(p, s);
}

pg_status pg_fft_c2r_3d(pg_plan* p, const void* d_in, void* d_out, void* stream) {
  if (!p || !d_in || !d_out) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  const int N = p->N, P = N / 2 + 1;
  const size_t bytes = csize(p) * (size_t)N * N * P;
  PG_TRY(p->tmpfft.ensure(bytes, &p->total));
  PG_TRY(cudaMemcpyAsync(p->tmpfft.p, d_in, bytes, cudaMemcpyDeviceToDevice, s));
  if (p->prm.precision) {
    using C = double2;
    C* t = p->tmpfft.as<C>();
    PG_TRY(FftPasses<double>::z_inv_full(N, t, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<double>::y_inv_full(N, t, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<double>::x_c2r_full(N, t, P, (double*)d_out, p->tw.as<C>(), s));
  } else {
    using C = float2;
    C* t = p->tmpfft.as<C>();
    PG_TRY(FftPasses<float>::z_inv_full(N, t, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<float>::y_inv_full(N, t, P, lay_zy(N, P), p->tw.as<C>(), p->flag.as<int32_t>() + 1, s));
    PG_TRY(FftPasses<float>::x_c2r_full(N, t, P, (float*)d_out, p->tw.as<C>(), s));
  }
  return stage_status(p, s);
}

pg_status pg_correlate_points(pg_plan* p, int64_t n_a, const double* d_a, const double* d_wa,
                              int64_t n_b, const double* d_b, const double* d_wb, double* h_sum,
                              double* h_sum2, double* h_agg, int64_t* h_ncells, void* stream) {
  if (!p || n_a <= 0 || n_b <= 0 || !d_a || !d_b) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nmax = std::max(n_a, n_b);
  PG_TRY(ensure_shared(p));
  PG_TRY(cudaMemsetAsync(p->flag.p, 0, 8, s));
  PG_TRY(ensure_gal(p, nmax));
  p->fwd_ok = false;   // the plan's spectra and sums are reused
  p->smooth_ok = false;
  // set b -> Fg; set a -> one "pair" mesh in S[0]
  PG_TRY(launch_transform(n_b, p->prm.box_L, 0.0, d_b, nullptr, nullptr, p->x.as<double>(),
                          p->y.as<double>(), p->z.as<double>(), s));
  pg_status st = PG_OK;
  auto run = [&](auto tag) -> cudaError_t {
    using R = decltype(tag);
    using C = typename CT<R>::C;
    PG_CUDA_TRY((galaxy_pass<R>(p, n_b, p->x.as<double>(), p->y.as<double>(), p->z.as<double>(), d_wb, false, s)));
    PG_CUDA_TRY(launch_transform(n_a, p->prm.box_L, 0.0, d_a, nullptr, nullptr, p->xs.as<double>(),
                                 p->ys.as<double>(), p->zs.as<double>(), s));
    int64_t nl = 0;
    PG_CUDA_TRY(deposit_batch(p, n_a, p->xs.as<double>(), p->ys.as<double>(), p->zs.as<double>(),
                              d_wa, nullptr, 0, 1, &nl, s));
    PG_CUDA_TRY(lines_to_S<R>(p, 1, nl, p->S.as<C>(), 0, s));
    return correlate_window<R>(p, 1, false, p->sums_pg.as<double>(), s);
  };
  cudaError_t e = p->prm.precision ? run(double{}) : run(float{});
  if (e != cudaSuccess) { (void)cudaGetLastError(); return from_cuda(e); }
  std::vector<double> sums(2 * p->nL);
  int32_t herr = 0;
  PG_TRY(cudaMemcpyAsync(sums.data(), p->sums_pg.p, 16 * p->nL, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaMemcpyAsync(&herr, p->flag.as<int32_t>() + 1, 4, cudaMemcpyDeviceToHost, s));
  PG_TRY(cudaStreamSynchronize(s));
  if (herr) return PG_ERR_TIMEOUT;
  for (int q = 0; q < p->nQ; ++q) {
    if (h_sum) h_sum[q] = sums[2 * q];
    if (h_sum2) h_sum2[q] = sums[2 * q + 1];
    if (h_ncells) h_ncells[q] = p->h_list_off[q + 1] - p->h_list_off[q];
  }
  if (h_agg) { h_agg[0] = sums[2 * p->nQ]; h_agg[1] = sums[2 * p->nQ + 1]; }
  return st;
}

}  // extern "C"
