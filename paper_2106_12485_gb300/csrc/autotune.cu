// autotune.cu -- host autotuner of the particle kernel's settings.
//
// The tile is the unit of work of the push (one CTA per tile) and of the
// particle sort, so its size trades shared-memory staging and guard-cell
// overhead (small tiles) against CTA count and load balance (large tiles,
// few particles).  The resident CTAs per SM set how many tiles are in
// flight on an SM (the paper's regions per core, Sec. 4.3).  The cell-order
// re-sort interval trades the cost of rewriting the store against the
// faster particle kernel on a store whose neighbouring slots hold
// neighbouring cells.  zpic_autotune times the tile-size candidates;
// zpic_autotune_all times them, then the CTA counts at the best tile, then
// the re-sort intervals at the best of both.  Both run on a copy reduced to
// at most 1024 x 1024 cells (same cell size, time step, species, densities
// and momenta; profiles, window and laser placed at the same distance from
// the right edge), keep the fastest per configuration class, and
// zpic_create uses the choice for settings a configuration leaves at 0.
// zpic_batch_autotune tunes the same three settings for a whole batch, by
// timing the batch itself with each candidate applied to every member: one
// batched launch per stage runs one tile size (the 16 x 16 one compiled
// for it), and the per-class choices, made for a simulation that has the
// GPU to itself, favour small tiles that fill the GPU with one small grid
// (measured on the 256-simulation sweep: per-class tiles, 223 of them
// 8 x 8, made its particle kernel 1.7 times slower than 16 x 16 for all).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/zpic.h"

namespace zp {
int set_last_error(int code, const char *msg);
}

namespace {

// Side of the reduced copy: large enough that every candidate gives many
// waves of CTAs (at 256 x 256 the GPU is under-filled by 16 x 16 tiles and
// smaller tiles win for that reason alone; measured on the 2048^2 plasma:
// 16 x 16 is fastest at full size, 12 x 12 on a 256^2 copy).
constexpr int kMaxSide = 1024;

std::mutex g_mu;
std::map<std::string, std::pair<int, int>> g_tuned;
std::map<std::string, zpic_tuning> g_tuned_all;
std::map<std::string, zpic_tuning> g_tuned_batch;

// The class of a configuration: what decides the best tile size is the
// precision, the particles per cell of each species (the work per tile),
// the boundary and window, the current filter and the reduced grid shape.
std::string class_key(const zpic_config &c) {
  std::string k = "p" + std::to_string(c.precision) + " n" +
                  std::to_string(std::min(c.nx, kMaxSide)) + "x" +
                  std::to_string(std::min(c.ny, kMaxSide)) + " b" +
                  std::to_string(c.bc_x) + " w" +
                  std::to_string(c.moving_window) + " f" +
                  std::to_string(c.flags & ZPIC_FILTER_J);
  for (int s = 0; s < c.n_species; ++s)
    k += " s" + std::to_string(c.species[s].ppc_x * c.species[s].ppc_y) + ":" +
         std::to_string(c.species[s].profile);
  return k;
}

zpic_config reduced(const zpic_config &c) {
  zpic_config r = c;
  const double dx = c.box_x / c.nx, dy = c.box_y / c.ny;
  r.nx = std::min(c.nx, kMaxSide);
  r.ny = std::min(c.ny, kMaxSide);
  r.box_x = r.nx * dx;
  r.box_y = r.ny * dy;
  const double fx = r.box_x / c.box_x;
  for (int s = 0; s < c.n_species; ++s) {
    zpic_species &p = r.species[s];
    if (p.profile == ZPIC_PROFILE_SLAB) {
      p.x0 = c.species[s].x0 * fx;
      p.x1 = c.species[s].x1 * fx;
    } else if (p.profile == ZPIC_PROFILE_RAMP) {
      p.x0 = r.box_x - (c.box_x - c.species[s].x0);  // same gap to the edge
    }
  }
  if (c.laser.enabled) {
    r.laser.x0 = r.box_x - (c.box_x - c.laser.x0);
    r.laser.y_center = c.laser.y_center * r.box_y / c.box_y;
  }
  r.energy_every = 0;
  r.flags &= ~ZPIC_TRACK_IDS;
  return r;
}

// Host wall time of `steps` steps after `warm` warm-up steps (ms per
// step), or a negative value if the candidate cannot run (e.g. too large
// for shared memory).
double time_candidate(const zpic_config &r, int steps, int warm = 3) {
  zpic_sim *h = nullptr;
  if (zpic_create(&r, &h) != ZPIC_OK) return -1.0;
  double ms = -1.0;
  if (zpic_step(h, warm) == ZPIC_OK && zpic_sync(h) == ZPIC_OK) {
    const auto t0 = std::chrono::steady_clock::now();
    if (zpic_step(h, steps) == ZPIC_OK && zpic_sync(h) == ZPIC_OK) {
      const auto t1 = std::chrono::steady_clock::now();
      ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / steps;
    }
  }
  zpic_destroy(h);
  return ms;
}

// A batch's key: its members' classes in order.
std::string batch_key(const zpic_config *cfgs, int n) {
  std::string k = "batch " + std::to_string(n);
  for (int i = 0; i < n; ++i) k += " | " + class_key(cfgs[i]);
  return k;
}

// Host wall time per step of the whole batch with `steps` timed steps
// after `warm`, or a negative value if it cannot run.
double time_batch(const std::vector<zpic_config> &cfgs, int steps,
                  int warm = 3) {
  zpic_batch *b = nullptr;
  if (zpic_batch_create(cfgs.data(), (int)cfgs.size(), &b) != ZPIC_OK)
    return -1.0;
  double ms = -1.0;
  if (zpic_batch_step(b, warm) == ZPIC_OK && zpic_batch_sync(b) == ZPIC_OK) {
    const auto t0 = std::chrono::steady_clock::now();
    if (zpic_batch_step(b, steps) == ZPIC_OK && zpic_batch_sync(b) == ZPIC_OK) {
      const auto t1 = std::chrono::steady_clock::now();
      ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / steps;
    }
  }
  zpic_batch_destroy(b);
  return ms;
}

const int kCand[][2] = {{16, 16}, {8, 8}, {12, 12}, {24, 24}, {32, 32},
                        {32, 16}, {16, 32}};
constexpr int kNCand = sizeof(kCand) / sizeof(kCand[0]);

const int kCtaCand[] = {1, 2, 3};
const int kSortCand[] = {-1, 10, 20, 40};
constexpr int kSortWarm = 40, kSortSteps = 80;

}  // namespace

namespace zp {
// The settings zpic_batch_autotune chose for this batch, if it has run.
bool tuned_batch(const zpic_config *cfgs, int n, zpic_tuning *t) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_tuned_batch.find(batch_key(cfgs, n));
  if (it == g_tuned_batch.end()) return false;
  *t = it->second;
  return true;
}

// The settings zpic_autotune_all chose for c's class, if it has run.
bool tuned_setting(const zpic_config &c, zpic_tuning *t) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_tuned_all.find(class_key(c));
  if (it == g_tuned_all.end()) return false;
  *t = it->second;
  return true;
}

// The tuned tile size of c's class, if zpic_autotune has run for it.
bool tuned_tile(const zpic_config &c, int *tx, int *ty) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_tuned.find(class_key(c));
  if (it == g_tuned.end()) return false;
  *tx = it->second.first;
  *ty = it->second.second;
  return true;
}
}  // namespace zp

extern "C" {

int zpic_autotune(const zpic_config *cfg, int steps, int *best_tile_x,
                  int *best_tile_y, double *ms_per_step, int cap,
                  int *n_candidates) {
  if (!cfg || !best_tile_x || !best_tile_y)
    return zp::set_last_error(ZPIC_EINVAL, "NULL argument");
  if (steps < 1 || steps > 10000)
    return zp::set_last_error(ZPIC_EINVAL, "steps out of range");
  if (n_candidates) *n_candidates = kNCand;
  const std::string key = class_key(*cfg);
  if (!ms_per_step) {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      *best_tile_x = it->second.first;
      *best_tile_y = it->second.second;
      return ZPIC_OK;
    }
  }
  double best = -1.0;
  int bx = 16, by = 16;
  int status = ZPIC_OK;
  for (int k = 0; k < kNCand; ++k) {
    zpic_config r = reduced(*cfg);
    r.tile_x = kCand[k][0];
    r.tile_y = kCand[k][1];
    const double ms = time_candidate(r, steps);
    if (ms_per_step && k < cap) ms_per_step[k] = ms;
    if (ms > 0 && (best < 0 || ms < best)) {
      best = ms;
      bx = kCand[k][0];
      by = kCand[k][1];
    }
  }
  if (best < 0)
    return zp::set_last_error(ZPIC_ECUDA, "no tile size candidate could run");
  {
    std::lock_guard<std::mutex> g(g_mu);
    g_tuned[key] = {bx, by};
  }
  *best_tile_x = bx;
  *best_tile_y = by;
  return status;
}

int zpic_autotune_all(const zpic_config *cfg, int steps, zpic_tuning *best,
                      double *ms_per_candidate, int cap, int *n_candidates) {
  if (!cfg || !best) return zp::set_last_error(ZPIC_EINVAL, "NULL argument");
  if (steps < 1 || steps > 10000)
    return zp::set_last_error(ZPIC_EINVAL, "steps out of range");
  const int n_cta = cfg->precision == ZPIC_FP64 ? 2 : 3;
  const int n_sort = (int)(sizeof(kSortCand) / sizeof(kSortCand[0]));
  const int total = kNCand + n_cta + n_sort;
  if (n_candidates) *n_candidates = total;
  int k_out = 0;
  auto record = [&](double ms) {
    if (ms_per_candidate && k_out < cap) ms_per_candidate[k_out] = ms;
    ++k_out;
  };
  zpic_config base = reduced(*cfg);
  base.sort_every = -1;
  base.push_ctas_per_sm = 0;
  // tile size
  double bt = -1.0;
  int bx = 16, by = 16;
  for (int k = 0; k < kNCand; ++k) {
    zpic_config r = base;
    r.tile_x = kCand[k][0];
    r.tile_y = kCand[k][1];
    const double ms = time_candidate(r, steps);
    record(ms);
    if (ms > 0 && (bt < 0 || ms < bt)) {
      bt = ms;
      bx = kCand[k][0];
      by = kCand[k][1];
    }
  }
  if (bt < 0)
    return zp::set_last_error(ZPIC_ECUDA, "no tile size candidate could run");
  base.tile_x = bx;
  base.tile_y = by;
  // resident CTAs per SM
  double bc = -1.0;
  int ctas = 0;
  for (int k = 0; k < n_cta; ++k) {
    zpic_config r = base;
    r.push_ctas_per_sm = kCtaCand[k];
    const double ms = time_candidate(r, steps);
    record(ms);
    if (ms > 0 && (bc < 0 || ms < bc)) {
      bc = ms;
      ctas = kCtaCand[k];
    }
  }
  base.push_ctas_per_sm = ctas;
  // re-sort interval, over a window long enough for the order to decay
  double bs = -1.0;
  int sort = -1;
  for (int k = 0; k < n_sort; ++k) {
    zpic_config r = base;
    r.sort_every = kSortCand[k];
    const double ms = time_candidate(r, kSortSteps, kSortWarm);
    record(ms);
    if (ms > 0 && (bs < 0 || ms < bs)) {
      bs = ms;
      sort = kSortCand[k];
    }
  }
  zpic_tuning t{};
  t.tile_x = bx;
  t.tile_y = by;
  t.push_ctas_per_sm = ctas;
  t.sort_every = sort;
  t.ms_per_step = bs;
  {
    const std::string key = class_key(*cfg);
    std::lock_guard<std::mutex> g(g_mu);
    g_tuned[key] = {bx, by};
    g_tuned_all[key] = t;
  }
  *best = t;
  return ZPIC_OK;
}

int zpic_batch_autotune(const zpic_config *cfgs, int n, int steps,
                        zpic_tuning *best, double *ms_per_candidate, int cap,
                        int *n_candidates) {
  if (!cfgs || !best) return zp::set_last_error(ZPIC_EINVAL, "NULL argument");
  if (n < 2) return zp::set_last_error(ZPIC_EINVAL, "a batch has 2 or more simulations");
  if (steps < 1 || steps > 10000)
    return zp::set_last_error(ZPIC_EINVAL, "steps out of range");
  const int n_cta = cfgs[0].precision == ZPIC_FP64 ? 2 : 3;
  const int n_sort = (int)(sizeof(kSortCand) / sizeof(kSortCand[0]));
  if (n_candidates) *n_candidates = kNCand + n_cta + n_sort;
  int k_out = 0;
  auto record = [&](double ms) {
    if (ms_per_candidate && k_out < cap) ms_per_candidate[k_out] = ms;
    ++k_out;
  };
  // every member gets the candidate; energy records are not needed
  std::vector<zpic_config> v(cfgs, cfgs + n);
  for (auto &c : v) {
    c.energy_every = 0;
    c.flags &= ~ZPIC_TRACK_IDS;
    c.sort_every = -1;
    c.push_ctas_per_sm = 0;
  }
  double bt = -1.0;
  int bx = 16, by = 16;
  for (int k = 0; k < kNCand; ++k) {
    for (auto &c : v) {
      c.tile_x = kCand[k][0];
      c.tile_y = kCand[k][1];
    }
    const double ms = time_batch(v, steps);
    record(ms);
    if (ms > 0 && (bt < 0 || ms < bt)) {
      bt = ms;
      bx = kCand[k][0];
      by = kCand[k][1];
    }
  }
  if (bt < 0)
    return zp::set_last_error(ZPIC_ECUDA, "no tile size candidate could run");
  for (auto &c : v) {
    c.tile_x = bx;
    c.tile_y = by;
  }
  double bc = -1.0;
  int ctas = 0;
  for (int k = 0; k < n_cta; ++k) {
    for (auto &c : v) c.push_ctas_per_sm = kCtaCand[k];
    const double ms = time_batch(v, steps);
    record(ms);
    if (ms > 0 && (bc < 0 || ms < bc)) {
      bc = ms;
      ctas = kCtaCand[k];
    }
  }
  for (auto &c : v) c.push_ctas_per_sm = ctas;
  double bs = -1.0;
  int sort = -1;
  for (int k = 0; k < n_sort; ++k) {
    for (auto &c : v) c.sort_every = kSortCand[k];
    const double ms = time_batch(v, kSortSteps, kSortWarm);
    record(ms);
    if (ms > 0 && (bs < 0 || ms < bs)) {
      bs = ms;
      sort = kSortCand[k];
    }
  }
  zpic_tuning t{};
  t.tile_x = bx;
  t.tile_y = by;
  t.push_ctas_per_sm = ctas;
  t.sort_every = sort;
  t.ms_per_step = bs;
  {
    std::lock_guard<std::mutex> g(g_mu);
    g_tuned_batch[batch_key(cfgs, n)] = t;
  }
  *best = t;
  return ZPIC_OK;
}

int zpic_autotune_candidates(int *tile_xy, int cap) {
  if (!tile_xy && cap > 0) return zp::set_last_error(ZPIC_EINVAL, "NULL buffer");
  for (int k = 0; k < kNCand && k < cap; ++k) {
    tile_xy[2 * k] = kCand[k][0];
    tile_xy[2 * k + 1] = kCand[k][1];
  }
  return kNCand;
}

}  // extern "C"
