// Many-mock drivers and batch-size autotuner (host code over the public C
// ABI). pg_run_batch: a batch of mocks of uneven size (box, mesh, catalogue)
// runs its forward calls in order on one stream; a host thread builds the
// plans of the mocks ahead (cell lists, window geometry, twiddles) while the
// current mock runs on the GPU, and plans of one mesh size and precision
// share their mesh scratch, so the device holds one scratch per distinct mesh
// size. pg_run_batch_streams: several runner threads, each with its own
// stream, plans and scratch, claim mocks from one work queue, so that one
// mock's host-side phases (plan building, the pair-count and line-count
// readbacks that size its launches) overlap another mock's GPU work.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pairgal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

bool same_problem(const pg_params& a, const pg_params& b) {
  if (a.box_L != b.box_L || a.mesh_n != b.mesh_n || a.assign != b.assign || a.n_s != b.n_s ||
      a.n_mu != b.n_mu || a.n_r != b.n_r || a.n_mur != b.n_mur || a.rsd_factor != b.rsd_factor ||
      a.r_perp_cut != b.r_perp_cut || a.precision != b.precision || a.bins_per_batch != b.bins_per_batch)
    return false;
  for (int i = 0; i <= a.n_s; ++i)
    if (a.s_edges[i] != b.s_edges[i]) return false;
  for (int i = 0; i <= a.n_r; ++i)
    if (a.r_edges[i] != b.r_edges[i]) return false;
  if (a.pair_grid != b.pair_grid) return false;
  if (a.pair_grid)
    for (int i = 0; i <= a.n_mu; ++i)
      if (a.par_edges[i] != b.par_edges[i]) return false;
  return true;
}

// p-quantile (0..1) of v by the nearest-rank rule.
double quantile(std::vector<double> v, double p) {
  if (v.empty()) return NAN;
  std::sort(v.begin(), v.end());
  size_t k = (size_t)ceil(p * (double)v.size());
  k = std::min(std::max<size_t>(k, 1), v.size());
  return v[k - 1];
}

}  // namespace

extern "C" {

pg_status pg_run_batch(const pg_mock* mocks, int32_t n_mocks, double* latency_ms, pg_batch_stats* stats,
                       void* stream) {
  if (n_mocks < 0 || (n_mocks > 0 && !mocks)) return PG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n_mocks; ++i)
    if (!mocks[i].out || mocks[i].n_gal < 0 || (mocks[i].n_gal > 0 && !mocks[i].h_pos))
      return PG_ERR_INVALID_ARG;
  const Clock::time_point t_batch = Clock::now();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PG_ERR_CUDA;
  constexpr int kAhead = 2;   // plans built ahead of the mock that runs

  // plan of mock i: plans[slot[i]]; slot -1 until the builder has it
  std::vector<pg_plan*> plans;
  std::vector<int> slot(n_mocks, -1);
  std::vector<pg_status> build_status(n_mocks, PG_OK);
  std::mutex mu;
  std::condition_variable cv;
  int32_t built = 0, running = 0;
  bool stop = false;
  int32_t n_workspaces = 0;

  std::thread builder([&] {
    cudaSetDevice(dev);
    // first plan of each (mesh_n, precision): the others share its scratch
    std::vector<std::pair<std::pair<int32_t, int32_t>, const pg_plan*>> donors;
    for (int32_t i = 0; i < n_mocks; ++i) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || i <= running + kAhead; });
        if (stop) return;
      }
      const pg_params& q = mocks[i].params;
      int found = -1;
      for (int32_t j = 0; j < i && found < 0; ++j)
        if (slot[j] >= 0 && same_problem(mocks[j].params, q)) found = slot[j];
      pg_status st = PG_OK;
      if (found < 0) {
        const pg_plan* donor = nullptr;
        for (const auto& d : donors)
          if (d.first.first == q.mesh_n && d.first.second == q.precision) donor = d.second;
        pg_plan* p = nullptr;
        st = donor ? pg_plan_create_shared(&q, donor, &p) : pg_plan_create(&q, &p);
        if (st == PG_OK) {
          if (!donor) donors.push_back({{q.mesh_n, q.precision}, p});
          std::lock_guard<std::mutex> lk(mu);
          plans.push_back(p);
          found = (int)plans.size() - 1;
          if (!donor) ++n_workspaces;
        }
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        build_status[i] = st;
        slot[i] = found;
        built = i + 1;
      }
      cv.notify_all();
    }
  });

  pg_status first_err = PG_OK;
  std::vector<double> lat;
  int64_t launches = 0;
  for (int32_t i = 0; i < n_mocks; ++i) {
    const Clock::time_point t0 = Clock::now();
    pg_plan* p = nullptr;
    pg_status st;
    {
      std::unique_lock<std::mutex> lk(mu);
      running = i;
      cv.notify_all();
      cv.wait(lk, [&] { return built > i; });
      st = build_status[i];
      if (st == PG_OK) p = plans[slot[i]];
    }
    if (st == PG_OK) {
      const pg_mock& m = mocks[i];
      st = pg_forward_host(p, m.n_gal, m.h_pos, m.h_vel, m.h_w, m.out, stream);
      int64_t nl = 0;
      if (st == PG_OK && pg_plan_last_stats(p, nullptr, &nl) == PG_OK) launches += nl;
    }
    const double ms = ms_since(t0);
    if (latency_ms) latency_ms[i] = st == PG_OK ? ms : NAN;
    if (st == PG_OK) lat.push_back(ms);
    if (st != PG_OK && first_err == PG_OK) first_err = st;
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
    running = n_mocks;
  }
  cv.notify_all();
  builder.join();
  const double wall = ms_since(t_batch);
  const int32_t n_plans = (int32_t)plans.size();
  for (pg_plan* p : plans) pg_plan_destroy(p);
  if (stats) {
    stats->wall_ms = wall;
    stats->mocks_per_s = wall > 0 ? 1e3 * (double)lat.size() / wall : 0.0;
    stats->p50_ms = quantile(lat, 0.50);
    stats->p99_ms = quantile(lat, 0.99);
    stats->n_plans = n_plans;
    stats->n_workspaces = n_workspaces;
    stats->gpu_launches = launches;
  }
  return first_err;
}

pg_status pg_run_batch_streams(const pg_mock* mocks, int32_t n_mocks, int32_t n_streams, double* latency_ms,
                               pg_batch_stats* stats, void* stream) {
  if (n_streams == 1) return pg_run_batch(mocks, n_mocks, latency_ms, stats, stream);
  if (n_mocks < 0 || (n_mocks > 0 && !mocks) || n_streams < 1 || n_streams > 8) return PG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n_mocks; ++i)
    if (!mocks[i].out || mocks[i].n_gal < 0 || (mocks[i].n_gal > 0 && !mocks[i].h_pos))
      return PG_ERR_INVALID_ARG;
  const Clock::time_point t_batch = Clock::now();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PG_ERR_CUDA;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  // the runners start after the caller's queued work and the caller's stream
  // waits for the runners at the end
  cudaEvent_t start_ev = nullptr;
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess) return PG_ERR_CUDA;
  if (cudaEventRecord(start_ev, caller) != cudaSuccess) {
    cudaEventDestroy(start_ev);
    return PG_ERR_CUDA;
  }
  std::mutex mu;
  int32_t next = 0;   // the work queue: the next mock to claim
  std::vector<pg_status> status(n_mocks, PG_OK);
  std::vector<double> lat_all(n_mocks, NAN);
  std::vector<int64_t> launches(n_streams, 0);
  std::vector<int32_t> n_plans(n_streams, 0), n_ws(n_streams, 0);
  std::vector<cudaStream_t> streams(n_streams, nullptr);
  std::vector<cudaEvent_t> done(n_streams, nullptr);
  pg_status setup = PG_OK;
  for (int k = 0; k < n_streams && setup == PG_OK; ++k) {
    if (cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(streams[k], start_ev, 0) != cudaSuccess)
      setup = PG_ERR_CUDA;
  }
  auto runner = [&](int k) {
    cudaSetDevice(dev);
    // this runner's plans (one per distinct problem) and scratch (one per
    // mesh size and precision): plans are not shared between runners
    std::vector<std::pair<const pg_params*, pg_plan*>> plans;
    std::vector<std::pair<std::pair<int32_t, int32_t>, const pg_plan*>> donors;
    for (;;) {
      int32_t i;
      {
        std::lock_guard<std::mutex> lk(mu);
        i = next++;
      }
      if (i >= n_mocks) break;
      const Clock::time_point t0 = Clock::now();
      const pg_params& q = mocks[i].params;
      pg_plan* p = nullptr;
      for (const auto& e : plans)
        if (same_problem(*e.first, q)) p = e.second;
      pg_status st = PG_OK;
      if (!p) {
        const pg_plan* donor = nullptr;
        for (const auto& d : donors)
          if (d.first.first == q.mesh_n && d.first.second == q.precision) donor = d.second;
        st = donor ? pg_plan_create_shared(&q, donor, &p) : pg_plan_create(&q, &p);
        if (st == PG_OK) {
          plans.push_back({&q, p});
          if (!donor) {
            donors.push_back({{q.mesh_n, q.precision}, p});
            ++n_ws[k];
          }
        }
      }
      if (st == PG_OK) {
        const pg_mock& m = mocks[i];
        st = pg_forward_host(p, m.n_gal, m.h_pos, m.h_vel, m.h_w, m.out, streams[k]);
        int64_t nl = 0;
        if (st == PG_OK && pg_plan_last_stats(p, nullptr, &nl) == PG_OK) launches[k] += nl;
      }
      status[i] = st;
      if (st == PG_OK) lat_all[i] = ms_since(t0);
    }
    cudaEventRecord(done[k], streams[k]);
    n_plans[k] = (int32_t)plans.size();
    for (auto it = plans.rbegin(); it != plans.rend(); ++it) pg_plan_destroy(it->second);
  };
  if (setup == PG_OK) {
    std::vector<std::thread> threads;
    for (int k = 0; k < n_streams; ++k) threads.emplace_back(runner, k);
    for (auto& t : threads) t.join();
    for (int k = 0; k < n_streams; ++k) cudaStreamWaitEvent(caller, done[k], 0);
  }
  for (int k = 0; k < n_streams; ++k) {
    if (done[k]) cudaEventDestroy(done[k]);
    if (streams[k]) cudaStreamDestroy(streams[k]);
  }
  cudaEventDestroy(start_ev);
  if (setup != PG_OK) return setup;
  pg_status first_err = PG_OK;
  std::vector<double> lat;
  for (int32_t i = 0; i < n_mocks; ++i) {
    if (latency_ms) latency_ms[i] = lat_all[i];
    if (status[i] == PG_OK) lat.push_back(lat_all[i]);
    else if (first_err == PG_OK) first_err = status[i];
  }
  const double wall = ms_since(t_batch);
  if (stats) {
    stats->wall_ms = wall;
    stats->mocks_per_s = wall > 0 ? 1e3 * (double)lat.size() / wall : 0.0;
    stats->p50_ms = quantile(lat, 0.50);
    stats->p99_ms = quantile(lat, 0.99);
    stats->n_plans = 0;
    stats->n_workspaces = 0;
    stats->gpu_launches = 0;
    for (int k = 0; k < n_streams; ++k) {
      stats->n_plans += n_plans[k];
      stats->n_workspaces += n_ws[k];
      stats->gpu_launches += launches[k];
    }
  }
  return first_err;
}

pg_status pg_autotune(const pg_params* params, int64_t n_gal, const double* h_pos, const float* h_vel,
                      const float* h_w, const int32_t* candidates, int32_t n_cand, int32_t* best,
                      double* ms_out, void* stream) {
  if (!params || !candidates || n_cand <= 0 || !best || n_gal < 0 || (n_gal > 0 && !h_pos))
    return PG_ERR_INVALID_ARG;
  for (int32_t k = 0; k < n_cand; ++k)
    if (candidates[k] <= 0) return PG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PG_ERR_CUDA;
  }
  // outputs of the trial runs go to scratch host arrays
  const size_t PQ = (size_t)params->n_s * params->n_mu * params->n_r * params->n_mur;
  const size_t Pn = (size_t)params->n_s * params->n_mu, Qn = (size_t)params->n_r * params->n_mur;
  std::vector<double> d5(PQ * 5 + Pn * 8 + Qn * 4 + 4);
  std::vector<int64_t> i3(Pn + Qn + 2);
  pg_result r;
  memset(&r, 0, sizeof(r));
  double* dp = d5.data();
  r.xi_pg = dp; dp += PQ;
  r.b_pg = dp; dp += PQ;
  r.q_eff = dp; dp += PQ;
  r.q_eff_sq = dp; dp += PQ;
  r.dd_w = dp; dp += Pn;
  r.xi_ss = dp; dp += Pn;
  r.b_pg_agg = dp; dp += Pn;
  r.q_eff_agg = dp; dp += Pn;
  r.sum_pg_agg = dp; dp += Pn;
  r.xi_gg = dp; dp += Qn;
  r.xi_dw = dp; dp += Qn;
  r.sum_gg = dp; dp += Qn;
  r.sum2_gg = dp; dp += Qn;
  r.sum_pg = dp; dp += PQ;
  r.xi_dw_agg = dp++;
  r.sum_gg_agg = dp;
  dp += 2;
  r.dd = i3.data();
  r.n_cells = i3.data() + Pn;
  r.n_cells_agg = i3.data() + Pn + Qn;
  pg_status st = PG_OK;
  pg_plan* first = nullptr;
  std::vector<pg_plan*> made;
  double best_ms = INFINITY;
  for (int32_t k = 0; k < n_cand && st == PG_OK; ++k) {
    pg_params q = *params;
    q.bins_per_batch = candidates[k];
    pg_plan* p = nullptr;
    st = first ? pg_plan_create_shared(&q, first, &p) : pg_plan_create(&q, &p);
    if (st != PG_OK) break;
    made.push_back(p);
    if (!first) first = p;
    st = pg_forward_host(p, n_gal, h_pos, h_vel, h_w, &r, stream);   // warm-up
    if (st != PG_OK) break;
    cudaEventRecord(e0, s);
    st = pg_forward_host(p, n_gal, h_pos, h_vel, h_w, &r, stream);
    cudaEventRecord(e1, s);
    if (st != PG_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[k] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      *best = candidates[k];
    }
  }
  for (auto it = made.rbegin(); it != made.rend(); ++it) pg_plan_destroy(*it);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // extern "C"
