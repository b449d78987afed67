// zpic_api.cu -- host implementation of the C ABI declared in include/zpic.h.
//
// A zpic_batch owns everything: per-simulation device buffers (fields, tile
// stores, outboxes, diagnostics), the descriptor table read by the kernels,
// the (sim, tile) work lists, the status word, the overflow buffer and one
// CUDA graph of a whole step (push+deposit -> Yee -> migrate -> end-of-step).
// A zpic_sim is a view of one simulation of a batch; zpic_create makes a
// batch of one and returns its only view.
//
// Steps run asynchronously.  Kernels hold back every step after one that
// raised an error; zpic_sync reads the status word, and when particles were
// parked in the overflow buffer it re-sorts the affected stores with more
// capacity and re-issues the steps that were held back.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/zpic.h"
#include "zpic_dev.cuh"
#include "zpic_kernels.h"

using namespace zp;

// ---------------------------------------------------------------------------
// errors, allocator
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}
namespace zp {
// error reporting for the ABI entry points defined in other files
int set_last_error(int code, const char *msg) { return fail(code, msg); }
bool tuned_tile(const zpic_config &c, int *tx, int *ty);  // autotune.cu
bool tuned_setting(const zpic_config &c, zpic_tuning *t);  // autotune.cu
bool tuned_batch(const zpic_config *cfgs, int n, zpic_tuning *t);  // autotune.cu
}  // namespace zp

static int cuda_fail(cudaError_t e, const char *what) {
  return fail(ZPIC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define ZP_CU(x)                                        \
  do {                                                  \
    cudaError_t e_ = (x);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);    \
  } while (0)
#define ZP_TRY(x)                \
  do {                           \
    int r_ = (x);                \
    if (r_ != ZPIC_OK) return r_; \
  } while (0)

// Host-side fault injection for tests (environment variable ZPIC_FAULT, read
// at every check): "alloc" makes every device allocation fail, "launch"
// makes every kernel or graph launch report a failure without launching
// anything, "timeout" makes zpic_sync report a bounded device wait that gave
// up.  Nothing reaches the GPU, so the injected failures cannot fault it.
static bool fault(const char *kind) {
  const char *v = std::getenv("ZPIC_FAULT");
  return v && std::strcmp(v, kind) == 0;
}

// NVTX range over an ABI call (header-only NVTX3: free unless a profiler
// such as Nsight Systems is attached)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static zpic_alloc_fn g_alloc = nullptr;
static zpic_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

namespace {

struct DevMem {
  void *p = nullptr;
  size_t bytes = 0;
};

// Waits for a stream when it goes out of scope: a call that queued copies
// to or from the caller's host memory on a side stream returns only when
// they are done, on its error paths too.
struct StreamDrain {
  cudaStream_t s;
  ~StreamDrain() {
    if (s) cudaStreamSynchronize(s);
  }
};

class Allocator {
 public:
  explicit Allocator(cudaStream_t s)
      : stream_(s), alloc_(g_alloc), free_(g_free), ctx_(g_alloc_ctx) {}
  void *get(size_t bytes, size_t *total) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (alloc_) {
      p = alloc_(bytes, stream_, ctx_);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) *total += bytes;
    return p;
  }
  void put(void *p, size_t bytes, size_t *total) {
    if (!p) return;
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (free_)
      free_(p, bytes, stream_, ctx_);
    else
      cudaFree(p);
    *total -= bytes;
  }
  cudaStream_t stream_;

 private:
  zpic_alloc_fn alloc_;
  zpic_free_fn free_;
  void *ctx_;
};

int validate(const zpic_config *c) {
  if (!c) return fail(ZPIC_EINVAL, "config is NULL");
  if (c->nx < 4 || c->ny < 4) return fail(ZPIC_EINVAL, "nx, ny must be >= 4");
  if ((long long)c->nx * c->ny > (1ll << 30))
    return fail(ZPIC_EINVAL, "grid too large");
  if (!(c->box_x > 0) || !(c->box_y > 0) || !(c->dt > 0))
    return fail(ZPIC_EINVAL, "box and dt must be positive");
  if (c->precision != ZPIC_FP32 && c->precision != ZPIC_FP64)
    return fail(ZPIC_EINVAL, "precision must be ZPIC_FP32 or ZPIC_FP64");
  if (c->bc_x != ZPIC_BC_PERIODIC && c->bc_x != ZPIC_BC_OPEN)
    return fail(ZPIC_EINVAL, "bc_x must be periodic or open");
  if (c->moving_window && c->bc_x != ZPIC_BC_OPEN)
    return fail(ZPIC_EINVAL, "moving window needs bc_x = ZPIC_BC_OPEN");
  if (c->n_species < 0 || c->n_species > ZPIC_MAX_SPECIES)
    return fail(ZPIC_EINVAL, "n_species out of range");
  if (c->energy_every < 0) return fail(ZPIC_EINVAL, "energy_every < 0");
  if (c->tile_x < 0 || c->tile_y < 0 || c->tile_x == 1 || c->tile_y == 1 ||
      c->tile_x > 32 || c->tile_y > 32)
    return fail(ZPIC_EINVAL, "tile sizes must be 0 or in [2, 32]");
  if (c->capacity_slack < 0 || c->capacity_slack > 16)
    return fail(ZPIC_EINVAL, "capacity_slack out of range");
  if (c->flags & ~(ZPIC_TRACK_IDS | ZPIC_FILTER_J | ZPIC_DETERMINISTIC))
    return fail(ZPIC_EINVAL, "unknown flags");
  if (c->sort_every < -1)
    return fail(ZPIC_EINVAL, "sort_every must be -1, 0 or positive");
  if (c->push_ctas_per_sm < 0 || c->push_ctas_per_sm > 8)
    return fail(ZPIC_EINVAL, "push_ctas_per_sm must be in [0, 8]");
  const double dx = c->box_x / c->nx, dy = c->box_y / c->ny;
  const double cfl = 1.0 / std::sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy));
  if (!(c->dt < cfl)) return fail(ZPIC_ECFL, "dt violates the Courant limit");
  for (int s = 0; s < c->n_species; ++s) {
    const zpic_species &p = c->species[s];
    if (!(p.q_over_m != 0) || !std::isfinite(p.q_over_m))
      return fail(ZPIC_EINVAL, "species q_over_m must be nonzero");
    if (p.ppc_x < 1 || p.ppc_y < 1 || p.ppc_x * p.ppc_y > 4096)
      return fail(ZPIC_EINVAL, "species ppc out of range");
    if (p.profile < ZPIC_PROFILE_NONE || p.profile > ZPIC_PROFILE_RAMP)
      return fail(ZPIC_EINVAL, "unknown density profile");
    if (p.profile != ZPIC_PROFILE_NONE && !(p.n0 > 0))
      return fail(ZPIC_EINVAL, "density n0 must be positive");
    if (p.profile == ZPIC_PROFILE_RAMP && !(p.x1 >= 0))
      return fail(ZPIC_EINVAL, "ramp length must be >= 0");
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(p.u_th[a]) || !std::isfinite(p.u_fl[a]) ||
          p.u_th[a] < 0)
        return fail(ZPIC_EINVAL, "bad thermal or drift momentum");
  }
  if (c->laser.enabled) {
    const zpic_laser &l = c->laser;
    if (!(l.w0 > 0) || !(l.fwhm > 0) || !(l.omega0 > 0))
      return fail(ZPIC_EINVAL, "laser w0, fwhm, omega0 must be positive");
  }
  return ZPIC_OK;
}

// Columns [lo, hi) with a nonzero initial density.
void profile_columns(const zpic_species &p, int nx, double dx, int *lo,
                     int *hi) {
  *lo = 0;
  *hi = 0;
  if (p.profile == ZPIC_PROFILE_NONE) return;
  if (p.profile == ZPIC_PROFILE_UNIFORM) {
    *hi = nx;
    return;
  }
  int a = nx, b = 0;
  for (int i = 0; i < nx; ++i) {
    const double xc = (i + 0.5) * dx;
    bool on;
    if (p.profile == ZPIC_PROFILE_SLAB)
      on = xc >= p.x0 && xc < p.x1;
    else  // ramp: positive density beyond x0
      on = xc > p.x0;
    if (on) {
      a = std::min(a, i);
      b = std::max(b, i + 1);
    }
  }
  if (b > a) {
    *lo = a;
    *hi = b;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// batch implementation
// ---------------------------------------------------------------------------

struct BatchBase {
  virtual ~BatchBase() {}
  virtual int init(const zpic_config *cfgs, int n) = 0;
  virtual int step(int n) = 0;
  virtual int sync() = 0;
  virtual int set_stream(void *s) = 0;
  virtual int get_fields(int sim, int which, void *dst, size_t cap,
                         int want_f64) = 0;
  virtual int set_fields_f64(int sim, int which, const double *src,
                             size_t n) = 0;
  virtual int num_particles(int sim, int sp, int64_t *n) = 0;
  virtual int get_particles(int sim, int sp, int t0, int t1,
                            const zpic_particles *dst, size_t *nw) = 0;
  virtual int set_particles(int sim, int sp, const zpic_particles *src) = 0;
  virtual int energy(int sim, zpic_energy_rec *dst, size_t cap,
                     size_t *nw) = 0;
  virtual int info(int sim, zpic_info *out) = 0;
  virtual int field_energy(int sim, double *wE, double *wB) = 0;
  virtual int tile_counts(int sim, int sp, int32_t *dst, size_t cap) = 0;
  virtual int get_state(int sim, zpic_state *out) = 0;
  virtual int set_state(int sim, const zpic_state *in) = 0;
  virtual int phasespace(int sim, int sp, int qx, int qy, const double *range,
                         int nbx, int nby, double *dst, size_t cap) = 0;
  virtual int profile_enable(int en) = 0;
  virtual int profile_read(char *names, size_t name_len, double *ms,
                           int32_t *launches, int cap, int *n, int reset) = 0;
  int n_sims = 0;
};

struct zpic_batch {
  std::unique_ptr<BatchBase> impl;
  std::vector<zpic_sim *> views;
};
struct zpic_sim {
  zpic_batch *b;
  int index;
  bool owns;
};

namespace {

template <typename R>
struct SpeciesHost {
  zpic_species cfg{};
  bool has_w = false, has_id = false;
  double q0 = 0.0;       // charge of a weight-1 particle
  double w_max = 0.0;    // largest weight given through set_particles
  long long total_cap = 0;
  DevMem store[2];                              // two copies of the store
  DevMem off, cap, cnt, ob_cnt, arr;            // per tile
  DevMem ob_ix, ob_iy, ob_id, ob_x, ob_y, ob_ux, ob_uy, ob_uz, ob_w;
  int ob_cap = 0;
  std::vector<int> h_cnt;                       // last counts read
  std::vector<int> h_cap;                       // current tile capacities
};

template <typename R>
struct SimHost {
  zpic_config cfg{};
  int nx, ny, ld, tx, ty, ntx, nty, ntiles, ybx, yby;
  int sort_every = -1;     // re-sort interval (-1: never)
  int ctas = 0;            // resident push CTAs per SM (0: all that fit)
  double dx, dy, dt;
  DevMem fields;           // 18 planes of ny * ld
  DevMem part_kin, part_fld, epart, hist, small, energy_rows;
  int hist_cap = 0;
  std::vector<SpeciesHost<R>> sp;
  SimDev<R> dev{};         // host copy of the descriptor
};

template <typename R>
struct Timer {
  std::string name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double ms = 0;
  int launches = 0;
};

template <typename R>
class Batch : public BatchBase {
 public:
  ~Batch() override { release(); }

  int init(const zpic_config *cfgs, int n) override {
    n_sims = n;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
      cudaGetLastError();
      return fail(ZPIC_ECUDA, "no CUDA device");
    }
    ZP_CU(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking));
    stream_ = own_stream_;
    ZP_CU(cudaStreamCreateWithFlags(&cpy_, cudaStreamNonBlocking));
    ZP_CU(cudaEventCreateWithFlags(&ev_pos_, cudaEventDisableTiming));
    ZP_CU(cudaEventCreateWithFlags(&ev_mom_, cudaEventDisableTiming));
    alloc_.reset(new Allocator(stream_));
    sims_.resize(n);
    for (int i = 0; i < n; ++i) ZP_TRY(init_sim(i, cfgs[i]));
    // status and overflow buffer
    st_mem_.p = alloc_->get(sizeof(BatchStatus), &bytes_);
    if (!st_mem_.p) return fail(ZPIC_ENOMEM, "status");
    st_mem_.bytes = sizeof(BatchStatus);
    ZP_TRY(reset_status());
    long long total = 0;
    for (auto &s : sims_)
      for (auto &p : s.sp) total += p.total_cap;
    ovf_cap_ = (int)std::min<long long>(1 << 26, std::max<long long>(1 << 14, total / 64));
    ZP_TRY(alloc_overflow());
    ZP_CU(cudaMallocHost(&h_st_, sizeof(BatchStatus)));
    ZP_TRY(upload_descriptors());
    ZP_TRY(build_items());
    // initial loads and laser fields
    for (int i = 0; i < n; ++i) ZP_TRY(initial_state(i));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  // ---- stepping ------------------------------------------------------------

  int step(int n) override {
    if (n < 0) return fail(ZPIC_EINVAL, "negative step count");
    if (sticky_) return sticky_;
    ZP_TRY(enqueue(n));
    target_ += n;
    return ZPIC_OK;
  }

  int sync() override {
    if (sticky_) return sticky_;
    // re-sort and re-issue as long as every round advances the step count
    int stalled = 0, last_step = -1;
    for (;;) {
      ZP_CU(cudaStreamSynchronize(stream_));
      if (fault("timeout")) {
        sticky_ = fail(ZPIC_ETIMEOUT, "injected: a bounded device wait gave up");
        return sticky_;
      }
      ZP_TRY(read_status());
      const BatchStatus &st = *h_st_;
      if (st.step == last_step) {
        if (++stalled > 3) break;
      } else {
        stalled = 0;
      }
      last_step = st.step;
      if (st.error & ERR_LOST) {
        sticky_ = fail(ZPIC_EOVERFLOW, "particle storage exhausted");
        return sticky_;
      }
      if (st.error & ERR_TIMEOUT) {
        sticky_ = fail(ZPIC_ETIMEOUT, "a bounded wait for a particle copy gave up");
        return sticky_;
      }
      if (st.error & ERR_STORE) {
        sticky_ = fail(ZPIC_ECUDA, "particle store corrupted (particle outside its tile)");
        return sticky_;
      }
      if (st.error & ERR_NAN) {
        sticky_ = fail(ZPIC_ENAN, "non-finite energy");
        return sticky_;
      }
      if (st.error & ERR_OVERFLOW) {
        ZP_TRY(resort_all());
        const long long left = target_ - st.step;
        if (left > 0) ZP_TRY(enqueue((int)left));
        continue;
      }
      return ZPIC_OK;
    }
    sticky_ = fail(ZPIC_EOVERFLOW, "repeated tile overflow");
    return sticky_;
  }

  int set_stream(void *s) override {
    ZP_CU(cudaStreamSynchronize(stream_));
    stream_ = s ? (cudaStream_t)s : own_stream_;
    alloc_->stream_ = stream_;
    invalidate_graph();
    return ZPIC_OK;
  }

  // ---- fields ---------------------------------------------------------------

  int get_fields(int si, int which, void *dst, size_t cap,
                 int want_f64) override {
    if (!dst || which < 0 || which > 8) return fail(ZPIC_EINVAL, "bad field");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    const size_t n = (size_t)S.nx * S.ny;
    if (cap < n) return fail(ZPIC_ECAP, "field buffer too small");
    const int step = h_st_->step;
    const R *src;
    if (which < 6)
      src = which < 3 ? S.dev.E[step & 1][which] : S.dev.B[step & 1][which - 3];
    else if (S.dev.Jf[0])
      src = S.dev.Jf[which - 6];  // the filtered current
    else if (sizeof(R) == 4)
      return get_current_fixed(S, S.dev.Jq[(step + 1) & 1][which - 6],
                               S.dev.jscale[which - 6], dst, want_f64);
    else if (S.dev.jfixed)
      return get_current_fixed64(S, S.dev.J[(step + 1) & 1][which - 6],
                                 S.dev.jscale_d[which - 6], dst, want_f64);
    else
      src = S.dev.J[(step + 1) & 1][which - 6];  // last step's current
    const bool same = want_f64 == (sizeof(R) == 8);
    if (same) {
      ZP_CU(cudaMemcpy2DAsync(dst, S.nx * sizeof(R), src, S.ld * sizeof(R),
                              S.nx * sizeof(R), S.ny, cudaMemcpyDeviceToHost,
                              stream_));
      ZP_CU(cudaStreamSynchronize(stream_));
      return ZPIC_OK;
    }
    std::vector<R> tmp(n);
    ZP_CU(cudaMemcpy2DAsync(tmp.data(), S.nx * sizeof(R), src, S.ld * sizeof(R),
                            S.nx * sizeof(R), S.ny, cudaMemcpyDeviceToHost,
                            stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    if (want_f64) {
      double *d = (double *)dst;
      for (size_t k = 0; k < n; ++k) d[k] = (double)tmp[k];
    } else {
      float *d = (float *)dst;
      for (size_t k = 0; k < n; ++k) d[k] = (float)tmp[k];
    }
    return ZPIC_OK;
  }

  // FP32 current: int64 fixed-point sums, scaled as the kernels do
  // (fixed_to_float, times the float scale)
  int get_current_fixed(SimHost<R> &S, const long long *src, float scale,
                        void *dst, int want_f64) {
    const size_t n = (size_t)S.nx * S.ny;
    std::vector<long long> q(n);
    ZP_CU(cudaMemcpy2DAsync(q.data(), S.nx * sizeof(long long), src,
                            S.ld * sizeof(long long), S.nx * sizeof(long long),
                            S.ny, cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    for (size_t k = 0; k < n; ++k) {
      const float v = fixed_to_float(q[k]) * scale;
      if (want_f64)
        ((double *)dst)[k] = v;
      else
        ((float *)dst)[k] = v;
    }
    return ZPIC_OK;
  }

  // FP64 with ZPIC_DETERMINISTIC: int64 fixed-point sums in the J words,
  // scaled as the kernels do ((double) value * scale)
  int get_current_fixed64(SimHost<R> &S, const R *src, double scale,
                          void *dst, int want_f64) {
    const size_t n = (size_t)S.nx * S.ny;
    std::vector<long long> q(n);
    ZP_CU(cudaMemcpy2DAsync(q.data(), S.nx * sizeof(long long), src,
                            S.ld * sizeof(long long), S.nx * sizeof(long long),
                            S.ny, cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    for (size_t k = 0; k < n; ++k) {
      const double v = (double)q[k] * scale;
      if (want_f64)
        ((double *)dst)[k] = v;
      else
        ((float *)dst)[k] = (float)v;
    }
    return ZPIC_OK;
  }

  int set_fields_f64(int si, int which, const double *src,
                     size_t n) override {
    if (!src || which < 0 || which > 5) return fail(ZPIC_EINVAL, "bad field");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (n != (size_t)S.nx * S.ny) return fail(ZPIC_EINVAL, "size != nx*ny");
    std::vector<R> tmp(n);
    for (size_t k = 0; k < n; ++k) tmp[k] = (R)src[k];
    const int step = h_st_->step;
    R *d = which < 3 ? S.dev.E[step & 1][which] : S.dev.B[step & 1][which - 3];
    ZP_CU(cudaMemcpy2DAsync(d, S.ld * sizeof(R), tmp.data(), S.nx * sizeof(R),
                            S.nx * sizeof(R), S.ny, cudaMemcpyHostToDevice,
                            stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  // ---- particles ------------------------------------------------------------

  int num_particles(int si, int s, int64_t *n) override {
    if (!n) return fail(ZPIC_EINVAL, "NULL count");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (s < 0 || s >= (int)S.sp.size()) return fail(ZPIC_EINVAL, "species");
    ZP_TRY(read_counts(si, s));
    long long t = 0;
    for (int c : S.sp[s].h_cnt) t += c;
    *n = t;
    return ZPIC_OK;
  }

  int get_particles(int si, int s, int t0, int t1, const zpic_particles *d,
                    size_t *nw) override {
    if (!d || !d->ix || !d->iy || !d->x || !d->y || !d->ux || !d->uy || !d->uz)
      return fail(ZPIC_EINVAL, "NULL particle array");
    if (d->precision != ZPIC_FP32 && d->precision != ZPIC_FP64)
      return fail(ZPIC_EINVAL, "bad precision");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (s < 0 || s >= (int)S.sp.size()) return fail(ZPIC_EINVAL, "species");
    if (t1 < 0) t1 = S.ntiles;
    if (t0 < 0 || t0 > t1 || t1 > S.ntiles)
      return fail(ZPIC_EINVAL, "tile range");
    ZP_TRY(read_counts(si, s));
    int pc = 0;
    ZP_TRY(particle_copy(si, &pc));
    SpeciesHost<R> &P = S.sp[s];
    std::vector<long long> off(std::max(1, t1 - t0));
    long long n = 0;
    for (int t = t0; t < t1; ++t) {
      off[t - t0] = n;
      n += P.h_cnt[t];
    }
    if (nw) *nw = (size_t)n;
    if ((size_t)n > d->cap) return fail(ZPIC_ECAP, "particle buffer too small");
    ZP_TRY(ensure_staging(n + 1));
    ZP_CU(cudaMemcpyAsync(stg_off_.p, off.data(), sizeof(long long) * off.size(),
                          cudaMemcpyHostToDevice, stream_));
    const bool same = (d->precision == ZPIC_FP64) == (sizeof(R) == 8);
    if (same) {
      // compaction in kChunks tile ranges on the library stream; each
      // range's copies to the host run on the transfer stream while the
      // next range is compacted
      StreamDrain drain{cpy_};
      constexpr int kChunks = 4;
      const int nt = t1 - t0;
      void *dsts[9] = {d->ix, d->iy, d->id, d->x, d->y, d->ux, d->uy, d->uz,
                       d->w};
      const void *srcs[9] = {stg_.ix, stg_.iy, stg_.id, stg_.x, stg_.y,
                             stg_.ux, stg_.uy, stg_.uz, stg_.w};
      const size_t esz[9] = {4, 4, 4, sizeof(R), sizeof(R), sizeof(R),
                             sizeof(R), sizeof(R), sizeof(R)};
      for (int c = 0; c < kChunks; ++c) {
        const int a = t0 + (int)((long long)nt * c / kChunks);
        const int b = t0 + (int)((long long)nt * (c + 1) / kChunks);
        if (a == b) continue;
        ZP_CU(launch_compact<R>(S.dev.sp[s], pc, S.tx, S.ty,
                                S.ntx, a, b - a,
                                (const long long *)stg_off_.p + (a - t0),
                                stg_, stream_));
        const long long p0 = off[a - t0], p1 = b < t1 ? off[b - t0] : n;
        if (p1 == p0) continue;
        ZP_CU(cudaEventRecord(ev_pos_, stream_));
        ZP_CU(cudaStreamWaitEvent(cpy_, ev_pos_, 0));
        for (int k = 0; k < 9; ++k) {
          if (!dsts[k]) continue;
          ZP_CU(cudaMemcpyAsync((char *)dsts[k] + esz[k] * p0,
                                (const char *)srcs[k] + esz[k] * p0,
                                esz[k] * (p1 - p0), cudaMemcpyDeviceToHost,
                                cpy_));
        }
      }
      ZP_CU(cudaStreamSynchronize(cpy_));
      ZP_CU(cudaStreamSynchronize(stream_));
      return ZPIC_OK;
    }
    ZP_CU(launch_compact<R>(S.dev.sp[s], pc, S.tx, S.ty, S.ntx,
                            t0, t1 - t0, (const long long *)stg_off_.p, stg_,
                            stream_));
    ZP_CU(cudaMemcpyAsync(d->ix, stg_.ix, 4 * n, cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaMemcpyAsync(d->iy, stg_.iy, 4 * n, cudaMemcpyDeviceToHost, stream_));
    if (d->id)
      ZP_CU(cudaMemcpyAsync(d->id, stg_.id, 4 * n, cudaMemcpyDeviceToHost, stream_));
    R *srcs[6] = {stg_.x, stg_.y, stg_.ux, stg_.uy, stg_.uz, stg_.w};
    void *dsts[6] = {d->x, d->y, d->ux, d->uy, d->uz, d->w};
    std::vector<R> tmp;
    for (int a = 0; a < 6; ++a) {
      if (!dsts[a]) continue;
      if (same) {
        ZP_CU(cudaMemcpyAsync(dsts[a], srcs[a], sizeof(R) * n,
                              cudaMemcpyDeviceToHost, stream_));
      } else {
        tmp.resize(n);
        ZP_CU(cudaMemcpyAsync(tmp.data(), srcs[a], sizeof(R) * n,
                              cudaMemcpyDeviceToHost, stream_));
        ZP_CU(cudaStreamSynchronize(stream_));
        if (d->precision == ZPIC_FP64)
          for (long long k = 0; k < n; ++k) ((double *)dsts[a])[k] = tmp[k];
        else
          for (long long k = 0; k < n; ++k) ((float *)dsts[a])[k] = (float)tmp[k];
      }
    }
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  int set_particles(int si, int s, const zpic_particles *src) override {
    if (!src || (src->n > 0 && (!src->ix || !src->iy || !src->x || !src->y ||
                                !src->ux || !src->uy || !src->uz)))
      return fail(ZPIC_EINVAL, "NULL particle array");
    if (src->precision != ZPIC_FP32 && src->precision != ZPIC_FP64)
      return fail(ZPIC_EINVAL, "bad precision");
    if (src->n > (size_t)INT_MAX) return fail(ZPIC_EINVAL, "too many particles");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (s < 0 || s >= (int)S.sp.size()) return fail(ZPIC_EINVAL, "species");
    const long long n = (long long)src->n;
    ZP_TRY(ensure_staging(n + 1));
    const bool same = (src->precision == ZPIC_FP64) == (sizeof(R) == 8);
    StreamDrain drain{cpy_};
    ZP_CU(cudaMemcpyAsync(stg_.ix, src->ix, 4 * n, cudaMemcpyHostToDevice, stream_));
    ZP_CU(cudaMemcpyAsync(stg_.iy, src->iy, 4 * n, cudaMemcpyHostToDevice, stream_));
    const void *srcs[6] = {src->x, src->y, src->ux, src->uy, src->uz, src->w};
    R *dsts[6] = {stg_.x, stg_.y, stg_.ux, stg_.uy, stg_.uz, stg_.w};
    cudaEvent_t moments_done = nullptr;
    if (same) {
      // cells and positions first, on the library stream: the tile count
      // (which reads only those) runs while momenta, weights and ids are
      // still arriving over the transfer stream
      for (int a = 0; a < 2; ++a)
        ZP_CU(cudaMemcpyAsync(dsts[a], srcs[a], sizeof(R) * n,
                              cudaMemcpyHostToDevice, stream_));
      ZP_CU(cudaEventRecord(ev_pos_, stream_));
      ZP_CU(cudaStreamWaitEvent(cpy_, ev_pos_, 0));
      for (int a = 2; a < 6; ++a)
        if (srcs[a])
          ZP_CU(cudaMemcpyAsync(dsts[a], srcs[a], sizeof(R) * n,
                                cudaMemcpyHostToDevice, cpy_));
      if (src->id)
        ZP_CU(cudaMemcpyAsync(stg_.id, src->id, 4 * n, cudaMemcpyHostToDevice, cpy_));
      ZP_CU(cudaEventRecord(ev_mom_, cpy_));
      moments_done = ev_mom_;
    } else if (src->id) {
      ZP_CU(cudaMemcpyAsync(stg_.id, src->id, 4 * n, cudaMemcpyHostToDevice, stream_));
    }
    std::vector<R> tmp;
    for (int a = 0; a < 6 && !same; ++a) {
      // other precision: converted on the host, one plane at a time
      if (!srcs[a]) continue;
      tmp.resize(n);
      if (src->precision == ZPIC_FP64)
        for (long long k = 0; k < n; ++k) tmp[k] = (R)((const double *)srcs[a])[k];
      else
        for (long long k = 0; k < n; ++k) tmp[k] = (R)((const float *)srcs[a])[k];
      ZP_CU(cudaMemcpyAsync(dsts[a], tmp.data(), sizeof(R) * n,
                            cudaMemcpyHostToDevice, stream_));
      ZP_CU(cudaStreamSynchronize(stream_));
    }
    if (src->w) {
      S.sp[s].has_w = true;
      double wm = 0.0;
      for (long long k = 0; k < n; ++k) {
        const double v = src->precision == ZPIC_FP64
                             ? ((const double *)src->w)[k]
                             : (double)((const float *)src->w)[k];
        if (!std::isfinite(v) || v < 0)
          return fail(ZPIC_EINVAL, "weights must be finite and >= 0");
        wm = std::max(wm, v);
      }
      S.sp[s].w_max = std::max(S.sp[s].w_max, wm);
      set_deposit_units(S);
    }
    ZP_TRY(rebuild_species(si, s, n, src->w != nullptr, src->id != nullptr,
                           true, moments_done));
    return ZPIC_OK;
  }

  // ---- diagnostics ---------------------------------------------------------

  int energy(int si, zpic_energy_rec *dst, size_t cap, size_t *nw) override {
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    int n = 0;
    if (S.cfg.energy_every > 0)
      ZP_CU(cudaMemcpy(&n, S.dev.hist_n, sizeof(int), cudaMemcpyDeviceToHost));
    if (nw) *nw = (size_t)n;
    if (n == 0 || (!dst && cap == 0)) return ZPIC_OK;  // size query
    if (!dst) return fail(ZPIC_EINVAL, "NULL energy buffer");
    if (cap < (size_t)n) return fail(ZPIC_ECAP, "energy buffer too small");
    ZP_CU(cudaMemcpy(dst, S.dev.hist, sizeof(zpic_energy_rec) * n,
                     cudaMemcpyDeviceToHost));
    return ZPIC_OK;
  }

  int field_energy(int si, double *wE, double *wB) override {
    if (!wE || !wB) return fail(ZPIC_EINVAL, "NULL output");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    const int cur = h_st_->step & 1;
    FieldPtrs<R> f;
    for (int c = 0; c < 3; ++c) {
      f.e[c] = S.dev.E[cur][c];
      f.b[c] = S.dev.B[cur][c];
    }
    double *scratch = (double *)S.energy_rows.p;
    ZP_CU(launch_field_energy<R>(f, S.nx, S.ny, S.ld, S.dx, S.dy, scratch,
                                 stream_));
    double out[2];
    ZP_CU(cudaMemcpyAsync(out, scratch + 2 * (size_t)S.ny, sizeof(out),
                          cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    *wE = out[0];
    *wB = out[1];
    return ZPIC_OK;
  }

  int info(int si, zpic_info *o) override {
    if (!o) return fail(ZPIC_EINVAL, "NULL info");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    std::memset(o, 0, sizeof(*o));
    o->nx = S.nx;
    o->ny = S.ny;
    o->ld = S.ld;
    o->dx = S.dx;
    o->dy = S.dy;
    o->dt = S.dt;
    o->tile_x = S.tx;
    o->tile_y = S.ty;
    o->ntiles_x = S.ntx;
    o->ntiles_y = S.nty;
    o->precision = sizeof(R) == 8 ? ZPIC_FP64 : ZPIC_FP32;
    o->step = h_st_->step;
    int nsh = 0;
    ZP_CU(cudaMemcpy(&nsh, S.dev.n_shift, sizeof(int), cudaMemcpyDeviceToHost));
    o->n_shift = nsh;
    o->n_species = (int)S.sp.size();
    for (int s = 0; s < (int)S.sp.size(); ++s) {
      ZP_TRY(read_counts(si, s));
      long long t = 0;
      for (int c : S.sp[s].h_cnt) t += c;
      o->n_particles[s] = t;
      o->capacity[s] = S.sp[s].total_cap;
    }
    o->resorts = resorts_;
    o->device_bytes = bytes_;
    o->sort_every = S.sort_every;
    o->push_ctas_per_sm = resolved_ctas();
    ZP_CU(cudaMemcpy(&o->sorts, S.dev.sorts, sizeof(int),
                     cudaMemcpyDeviceToHost));
    ZP_CU(cudaMemcpy(o->push_variants, S.dev.variants,
                     sizeof(int) * kMaxSpecies, cudaMemcpyDeviceToHost));
    return ZPIC_OK;
  }

  // ---- checkpoint / restart --------------------------------------------------

  int get_state(int si, zpic_state *o) override {
    if (!o) return fail(ZPIC_EINVAL, "NULL state");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    int small[2 + kMaxSpecies];
    ZP_CU(cudaMemcpy(small + 1, S.dev.n_shift, sizeof(int) * (1 + kMaxSpecies),
                     cudaMemcpyDeviceToHost));
    std::memset(o, 0, sizeof(*o));
    o->step = h_st_->step;
    o->n_shift = small[1];
    for (int s = 0; s < kMaxSpecies; ++s) o->removed[s] = small[2 + s];
    return ZPIC_OK;
  }

  int set_state(int si, const zpic_state *in) override {
    if (!in) return fail(ZPIC_EINVAL, "NULL state");
    if (n_sims != 1)
      return fail(ZPIC_EINVAL, "set_state on a batch of several simulations");
    if (in->step < 0 || in->step > INT_MAX / 2 || in->n_shift < 0)
      return fail(ZPIC_EINVAL, "step or n_shift out of range");
    for (int s = 0; s < kMaxSpecies; ++s)
      if (in->removed[s] < 0 || in->removed[s] > INT_MAX)
        return fail(ZPIC_EINVAL, "removed count out of range");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    const int old_step = h_st_->step, new_step = (int)in->step;
    if ((old_step ^ new_step) & 1) {
      // the current copies are those of the step parity: swap the roles of
      // the two field copies and of the two particle stores (J of the
      // current copy stays zero, as a step expects)
      for (int c = 0; c < 3; ++c) {
        std::swap(S.dev.E[0][c], S.dev.E[1][c]);
        std::swap(S.dev.B[0][c], S.dev.B[1][c]);
        std::swap(S.dev.J[0][c], S.dev.J[1][c]);
        std::swap(S.dev.Jq[0][c], S.dev.Jq[1][c]);
      }
      for (int s = 0; s < (int)S.sp.size(); ++s) {
        std::swap(S.dev.sp[s].buf[0], S.dev.sp[s].buf[1]);
        std::swap(S.sp[s].store[0], S.sp[s].store[1]);
      }
    }
    int small[2 + kMaxSpecies] = {0};
    small[1] = in->n_shift;
    for (int s = 0; s < kMaxSpecies; ++s) small[2 + s] = (int)in->removed[s];
    ZP_CU(cudaMemcpyAsync(S.dev.hist_n, small, sizeof(int) * (2 + kMaxSpecies),
                          cudaMemcpyHostToDevice, stream_));
    S.dev.hist_skip = S.cfg.energy_every > 0 ? new_step / S.cfg.energy_every : 0;
    h_st_->step = new_step;
    target_ = new_step;
    ZP_TRY(reset_status());
    ZP_TRY(upload_descriptors());
    return ZPIC_OK;
  }

  // ---- phase-space report ---------------------------------------------------

  int phasespace(int si, int s, int qx, int qy, const double *range, int nbx,
                 int nby, double *dst, size_t cap) override {
    if (!range || !dst) return fail(ZPIC_EINVAL, "NULL range or buffer");
    if (qx < ZPIC_PS_X || qx > ZPIC_PS_UZ || qy < ZPIC_PS_X || qy > ZPIC_PS_UZ)
      return fail(ZPIC_EINVAL, "bad phase-space quantity");
    if (nbx < 1 || nby < 1 || nbx > 4096 || nby > 4096)
      return fail(ZPIC_EINVAL, "bin counts must be in [1, 4096]");
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(range[k])) return fail(ZPIC_EINVAL, "range not finite");
    if (!(range[1] > range[0]) || !(range[3] > range[2]))
      return fail(ZPIC_EINVAL, "empty range");
    if (cap < (size_t)nbx * nby) return fail(ZPIC_ECAP, "histogram buffer too small");
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (s < 0 || s >= (int)S.sp.size()) return fail(ZPIC_EINVAL, "species");
    const size_t bytes = sizeof(double) * (size_t)nbx * nby;
    DevMem h;
    if (!dalloc(h, bytes)) return fail(ZPIC_ENOMEM, "histogram");
    PhaseSpaceSpec ps;
    ps.qx = qx;
    ps.qy = qy;
    ps.nbx = nbx;
    ps.nby = nby;
    ps.lo[0] = range[0];
    ps.lo[1] = range[2];
    ps.scale[0] = (double)nbx / (range[1] - range[0]);
    ps.scale[1] = (double)nby / (range[3] - range[2]);
    ps.q0 = std::fabs(S.sp[s].q0);
    int pc = 0;
    if (particle_copy(si, &pc) != ZPIC_OK) {
      dfree(h);
      return ZPIC_ECUDA;
    }
    cudaError_t e = cudaMemsetAsync(h.p, 0, bytes, stream_);
    if (e == cudaSuccess)
      e = launch_phasespace<R>(S.dev.sp[s], pc, S.tx, S.ty, S.ntx,
                               S.ntiles, ps, (double *)h.p, stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, h.p, bytes, cudaMemcpyDeviceToHost, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    dfree(h);
    if (e != cudaSuccess) return cuda_fail(e, "phase space");
    return ZPIC_OK;
  }

  int tile_counts(int si, int s, int32_t *dst, size_t cap) override {
    ZP_TRY(sync());
    SimHost<R> &S = sims_[si];
    if (!dst || s < 0 || s >= (int)S.sp.size())
      return fail(ZPIC_EINVAL, "bad argument");
    if (cap < (size_t)S.ntiles) return fail(ZPIC_ECAP, "buffer too small");
    ZP_TRY(read_counts(si, s));
    std::memcpy(dst, S.sp[s].h_cnt.data(), sizeof(int) * S.ntiles);
    return ZPIC_OK;
  }

  // ---- kernel timing --------------------------------------------------------

  int profile_enable(int en) override {
    profiling_ = en != 0;
    return ZPIC_OK;
  }

  int profile_read(char *names, size_t name_len, double *ms, int32_t *launches,
                   int cap, int *n, int reset) override {
    ZP_CU(cudaStreamSynchronize(stream_));
    int k = 0;
    for (auto &t : timers_) {
      for (auto &e : t.ev) {
        float v = 0;
        ZP_CU(cudaEventElapsedTime(&v, e.first, e.second));
        t.ms += v;
        t.launches += 1;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
      t.ev.clear();
      if (k < cap) {
        if (names && name_len > 0) {
          std::strncpy(names + (size_t)k * name_len, t.name.c_str(), name_len - 1);
          names[(size_t)k * name_len + name_len - 1] = 0;
        }
        if (ms) ms[k] = t.ms;
        if (launches) launches[k] = t.launches;
      }
      ++k;
      if (reset) {
        t.ms = 0;
        t.launches = 0;
      }
    }
    if (n) *n = k;
    return ZPIC_OK;
  }

 private:
  // ---- setup ---------------------------------------------------------------

  void *dalloc(DevMem &m, size_t bytes) {
    if (fault("alloc")) {
      m.p = nullptr;
      m.bytes = 0;
      return nullptr;
    }
    m.p = alloc_->get(bytes, &bytes_);
    m.bytes = m.p ? bytes : 0;
    return m.p;
  }
  void dfree(DevMem &m) {
    if (m.p) alloc_->put(m.p, m.bytes, &bytes_);
    m.p = nullptr;
    m.bytes = 0;
  }

  int init_sim(int i, const zpic_config &c) {
    SimHost<R> &S = sims_[i];
    S.cfg = c;
    S.nx = c.nx;
    S.ny = c.ny;
    S.ld = (c.nx + 31) & ~31;
    S.dx = c.box_x / c.nx;
    S.dy = c.box_y / c.ny;
    S.dt = c.dt;
    int tx = c.tile_x, ty = c.tile_y;
    if (tx == 0 && ty == 0 && !tuned_tile(c, &tx, &ty)) tx = ty = 16;
    S.tx = std::min(tx ? tx : 16, c.nx);
    S.ty = std::min(ty ? ty : 16, c.ny);
    if (push_smem_bytes<R>(S.tx, S.ty, true) > 226 * 1024)
      return fail(ZPIC_EINVAL, "tile too large for shared memory");
    S.ntx = (S.nx + S.tx - 1) / S.tx;
    S.nty = (S.ny + S.ty - 1) / S.ty;
    S.ntiles = S.ntx * S.nty;
    S.ybx = (S.nx + kYeeX - 1) / kYeeX;
    S.yby = (S.ny + yee_rows<R>() - 1) / yee_rows<R>();
    const size_t plane = (size_t)S.ny * S.ld;
    const bool filter = (c.flags & ZPIC_FILTER_J) != 0;
    // E, B: 12 planes of R; J: 6 planes of 8-byte values; Jf: 3 planes of R
    const size_t eb_bytes = 12 * plane * sizeof(R);
    const size_t j_bytes = 6 * plane * 8;
    if (!dalloc(S.fields, eb_bytes + j_bytes + (filter ? 3 * plane * sizeof(R) : 0)))
      return fail(ZPIC_ENOMEM, "fields");
    ZP_CU(cudaMemsetAsync(S.fields.p, 0, S.fields.bytes, stream_));
    R *f = (R *)S.fields.p;
    SimDev<R> &D = S.dev;
    D.nx = S.nx;
    D.ny = S.ny;
    D.ld = S.ld;
    D.tx = S.tx;
    D.ty = S.ty;
    D.ntx = S.ntx;
    D.nty = S.nty;
    D.ybx = S.ybx;
    D.yby = S.yby;
    D.open_x = c.bc_x == ZPIC_BC_OPEN;
    D.jfixed = sizeof(R) == 8 && (c.flags & ZPIC_DETERMINISTIC) ? 1 : 0;
    D.moving_window = c.moving_window ? 1 : 0;
    D.energy_every = c.energy_every;
    D.nsp = c.n_species;
    D.dx = (R)S.dx;
    D.dy = (R)S.dy;
    D.dt = (R)S.dt;
    D.dt_dx = (R)(S.dt / S.dx);
    D.dt_dy = (R)(S.dt / S.dy);
    D.dx_d = S.dx;
    D.dy_d = S.dy;
    D.dt_d = S.dt;
    char *jb = (char *)S.fields.p + eb_bytes;
    for (int a = 0; a < 2; ++a)
      for (int c3 = 0; c3 < 3; ++c3) {
        D.E[a][c3] = f + (size_t)(a * 6 + c3) * plane;
        D.B[a][c3] = f + (size_t)(a * 6 + 3 + c3) * plane;
        char *j = jb + (size_t)(a * 3 + c3) * plane * 8;
        D.Jq[a][c3] = sizeof(R) == 4 ? (long long *)j : nullptr;
        D.J[a][c3] = sizeof(R) == 8 ? (R *)j : nullptr;
      }
    R *jf = (R *)(jb + j_bytes);
    for (int c3 = 0; c3 < 3; ++c3)
      D.Jf[c3] = filter ? jf + (size_t)c3 * plane : nullptr;
    if (!dalloc(S.part_kin, sizeof(double) * S.ntiles * kMaxSpecies) ||
        !dalloc(S.part_fld, sizeof(double) * 2 * S.ybx * S.yby) ||
        !dalloc(S.epart, sizeof(double) * 2 * kEndSlicesMax * kEndQ))
      return fail(ZPIC_ENOMEM, "partials");
    ZP_CU(cudaMemsetAsync(S.part_kin.p, 0, S.part_kin.bytes, stream_));
    ZP_CU(cudaMemsetAsync(S.part_fld.p, 0, S.part_fld.bytes, stream_));
    D.part_kin = (double *)S.part_kin.p;
    D.part_fld = (double *)S.part_fld.p;
    ZP_CU(cudaMemsetAsync(S.epart.p, 0, S.epart.bytes, stream_));
    D.epart = (double *)S.epart.p;
    D.end_g = end_slices(S.ntiles, c.n_species, S.ybx * S.yby);
    S.hist_cap = c.energy_every > 0 ? 4096 : 1;
    if (!dalloc(S.hist, sizeof(zpic_energy_rec) * S.hist_cap))
      return fail(ZPIC_ENOMEM, "history");
    ZP_CU(cudaMemsetAsync(S.hist.p, 0, S.hist.bytes, stream_));
    D.hist = (zpic_energy_rec *)S.hist.p;
    D.hist_cap = S.hist_cap;
    D.hist_skip = 0;
    if (!dalloc(S.energy_rows, sizeof(double) * (2 * (size_t)S.ny + 2)))
      return fail(ZPIC_ENOMEM, "energy scratch");
    if (!dalloc(S.small, sizeof(int) * (5 + 3 * kMaxSpecies)))
      return fail(ZPIC_ENOMEM, "counters");
    ZP_CU(cudaMemsetAsync(S.small.p, 0, S.small.bytes, stream_));
    D.hist_n = (int *)S.small.p;
    D.n_shift = (int *)S.small.p + 1;
    D.removed = (int *)S.small.p + 2;
    D.ob_need = (int *)S.small.p + 2 + kMaxSpecies;
    D.eticket = (int *)S.small.p + 2 + 2 * kMaxSpecies;
    D.variants = (int *)S.small.p + 3 + 2 * kMaxSpecies;
    D.pswap = (int *)S.small.p + 3 + 3 * kMaxSpecies;
    D.sorts = (int *)S.small.p + 4 + 3 * kMaxSpecies;
    // cell-order re-sort interval and resident push CTAs: the configured
    // values, else those the autotuner chose for the class, else never / all
    // that fit
    {
      zpic_tuning t{};
      const bool tuned = tuned_setting(c, &t);
      S.sort_every = c.sort_every > 0 ? c.sort_every
                     : (c.sort_every == 0 && tuned ? t.sort_every : -1);
      S.ctas = c.push_ctas_per_sm > 0 ? c.push_ctas_per_sm
               : (tuned ? t.push_ctas_per_sm : 0);
      D.sort_every = S.sort_every > 0 ? S.sort_every : 0;
    }

    // species: initial per-tile counts from the profile, then capacities
    S.sp.resize(c.n_species);
    const double slack = c.capacity_slack > 0 ? c.capacity_slack : 0.25;
    for (int s = 0; s < c.n_species; ++s) {
      SpeciesHost<R> &P = S.sp[s];
      P.cfg = c.species[s];
      P.has_id = (c.flags & ZPIC_TRACK_IDS) != 0;
      // per-particle weights only where the density is not 1 everywhere
      P.has_w = P.cfg.profile == ZPIC_PROFILE_RAMP ||
                (P.cfg.profile != ZPIC_PROFILE_NONE && P.cfg.n0 != 1.0);
      const int ppc = P.cfg.ppc_x * P.cfg.ppc_y;
      int lo, hi;
      profile_columns(P.cfg, S.nx, S.dx, &lo, &hi);
      std::vector<int> cnt(S.ntiles, 0);
      for (int t = 0; t < S.ntiles; ++t) {
        const int x0 = (t % S.ntx) * S.tx, y0 = (t / S.ntx) * S.ty;
        const int tw = std::min(S.tx, S.nx - x0), th = std::min(S.ty, S.ny - y0);
        const int ca = std::max(x0, lo), cb = std::min(x0 + tw, hi);
        cnt[t] = cb > ca ? (cb - ca) * th * ppc : 0;
      }
      const double nominal = (double)ppc * S.tx * S.ty;
      P.ob_cap = ((std::max(64, (int)std::ceil(nominal * (c.moving_window ? 0.25 : 0.125))) + 31) / 32) * 32;
      if ((long long)P.ob_cap * S.ntiles >= INT_MAX)
        return fail(ZPIC_EINVAL, "outbox index range exceeded (grid x ppc too large)");
      ZP_TRY(alloc_store(i, s, cnt, slack, nominal,
                         full_tile_cap(nominal, slack, window_plasma(S, P))));
      // the initial load writes cnt particles per tile directly
      ZP_CU(cudaMemcpyAsync(P.cnt.p, cnt.data(), sizeof(int) * S.ntiles,
                            cudaMemcpyHostToDevice, stream_));
      P.h_cnt = cnt;
      SpeciesDev<R> &Q = D.sp[s];
      const double qm = P.cfg.q_over_m;
      const double q0 = (qm > 0 ? 1.0 : -1.0) / ppc;
      Q.qm = (R)qm;
      Q.hq = (R)(0.5 * qm * S.dt);
      Q.q0 = (R)q0;
      P.q0 = q0;
      Q.qx = (R)(q0 * S.dx / S.dt);
      Q.qy = (R)(q0 * S.dy / S.dt);
      Q.kin_scale = q0 / qm * S.dx * S.dy;
      Q.ob_cap = P.ob_cap;
      if (c.moving_window && P.cfg.profile != ZPIC_PROFILE_NONE) {
        Q.inj_ppc_x = P.cfg.ppc_x;
        Q.inj_ppc_y = P.cfg.ppc_y;
        // window plasma: uniform -> step at 0; ramp -> given ramp
        Q.ramp_x0 = P.cfg.profile == ZPIC_PROFILE_RAMP ? P.cfg.x0 : -1e300;
        Q.ramp_len = P.cfg.profile == ZPIC_PROFILE_RAMP ? P.cfg.x1 : 0.0;
        Q.n0 = P.cfg.n0;
        Q.id_base = (long long)S.nx * S.ny * ppc;
      }
    }
    set_deposit_units(S);
    return ZPIC_OK;
  }

  // Deposit factors and the scale of the FP32 fixed-point current tiles:
  // one unit Uq = max over species of |q0| x (largest weight), so a single
  // segment adds at most one unit to any current value.
  void set_deposit_units(SimHost<R> &S) {
    double uq = 0.0;
    for (auto &P : S.sp) {
      double wmax = std::max(1.0, P.w_max);
      if (P.cfg.profile != ZPIC_PROFILE_NONE) wmax = std::max(wmax, P.cfg.n0);
      uq = std::max(uq, std::fabs(P.q0) * wmax);
    }
    if (!(uq > 0)) uq = 1.0;
    const double cx = S.dx / S.dt, cy = S.dy / S.dt;
    const bool fp32 = sizeof(R) == 4;
    // FP64 fixed point: contributions in units of 2^-47 Uq
    const double u47 = std::ldexp(1.0, 47);
    for (int s = 0; s < (int)S.sp.size(); ++s) {
      SpeciesDev<R> &Q = S.dev.sp[s];
      const double q0 = S.sp[s].q0;
      if (fp32) {
        Q.dq[0] = Q.dq[1] = Q.dq[2] = (R)(q0 / uq * 65536.0);
      } else if (S.dev.jfixed) {
        Q.dq[0] = Q.dq[1] = Q.dq[2] = (R)(q0 / uq * u47);
      } else {
        Q.dq[0] = (R)(q0 * cx);
        Q.dq[1] = (R)(q0 * cy);
        Q.dq[2] = (R)q0;
      }
    }
    const double u30 = std::ldexp(1.0, -30);
    S.dev.jscale[0] = fp32 ? (float)(uq * cx * u30) : 1.0f;
    S.dev.jscale[1] = fp32 ? (float)(uq * cy * u30) : 1.0f;
    S.dev.jscale[2] = fp32 ? (float)(uq * u30) : 1.0f;
    const double i47 = std::ldexp(1.0, -47);
    S.dev.jscale_d[0] = uq * cx * i47;
    S.dev.jscale_d[1] = uq * cy * i47;
    S.dev.jscale_d[2] = uq * i47;
  }

  // Allocates the tile store of species s for per-tile counts cnt.
  // Room every tile of a species gets: its full density plus the slack; a
  // plasma that flows through a moving window is compressed as it passes
  // the laser (wake, channel walls), so its tiles get room for twice their
  // full density.
  static int full_tile_cap(double nominal, double slack, bool window_plasma) {
    const double f = window_plasma ? std::max(1.0 + slack, 2.0) : 1.0 + slack;
    return std::max(64, (int)std::ceil(nominal * f));
  }
  static bool window_plasma(const SimHost<R> &S, const SpeciesHost<R> &P) {
    return S.cfg.moving_window && P.cfg.profile != ZPIC_PROFILE_NONE;
  }

  // Capacity of tile t: room for its count plus the slack, and at least
  // min_cap, the species' full density of a tile plus the slack.  An empty
  // tile can thus fill at the species' density (a cloud front moving in, a
  // window injecting plasma) without a re-sort; only compression beyond
  // that density overflows.
  int alloc_store(int si, int s, const std::vector<int> &cnt, double slack,
                  double nominal, int min_cap) {
    SimHost<R> &S = sims_[si];
    SpeciesHost<R> &P = S.sp[s];
    std::vector<int> off(S.ntiles), cap(S.ntiles);
    // plasma flowing through a moving window meets the same wake in every
    // tile it reaches: once a tile has been compressed beyond the room every
    // tile gets, every tile gets room for that tile's count plus the slack,
    // so the wake does not overflow each new tile it reaches in turn (a
    // re-sort per few tens of steps on the 4096 x 512 LWFA while its window
    // fills; room as if the whole window held the densest tile's plasma)
    if (window_plasma(S, P)) {
      int mx = 0;
      for (int t = 0; t < S.ntiles; ++t) mx = std::max(mx, cnt[t]);
      if (mx > min_cap)
        min_cap = (int)std::min<double>(INT_MAX / 2, std::ceil(mx * (1.0 + slack)));
    }
    // densest tile within two tiles of each tile (a compressed structure
    // moving through the tiles reaches its neighbours next)
    std::vector<int> near(S.ntiles, 0);
    for (int t = 0; t < S.ntiles; ++t) {
      const int tx = t % S.ntx, ty = t / S.ntx;
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          const int x = tx + dx, y = (ty + dy + S.nty) % S.nty;
          if (x < 0 || x >= S.ntx) continue;
          near[t] = std::max(near[t], cnt[y * S.ntx + x]);
        }
    }
    long long tot = 0;
    for (int t = 0; t < S.ntiles; ++t) {
      long long c = std::max<long long>((long long)std::ceil(cnt[t] * (1.0 + slack)),
                                        (long long)cnt[t] + 64);
      c = std::max<long long>(c, min_cap);
      // a tile keeps the capacity it had (density structures such as a
      // laser wake stay in the same tiles and come back after a dip), and a
      // tile that outgrew its capacity at least doubles it, so a tile that
      // keeps filling needs few re-sorts
      if (!P.h_cap.empty()) {
        c = std::max<long long>(c, P.h_cap[t]);
        if (cnt[t] > P.h_cap[t]) c = std::max<long long>(c, 2LL * P.h_cap[t]);
      }
      // a tile near one compressed beyond the species' full density plus
      // the slack may be compressed next (a wake, a filament, a channel wall
      // moving through the tiles): room for twice that density before it
      // overflows.  Thermal scatter of a uniform plasma around its density
      // stays below the threshold, so its capacities stay put and repeated
      // uploads and re-sorts reuse the store's memory.
      if (near[t] > nominal * (1.0 + slack))
        c = std::max<long long>(c, 2LL * near[t]);
      c = (c + 31) / 32 * 32;
      if (tot + c > INT_MAX) return fail(ZPIC_ENOMEM, "species store exceeds 2^31");
      off[t] = (int)tot;
      cap[t] = (int)c;
      tot += c;
    }
    P.total_cap = tot;
    const size_t cb = ((size_t)2 * tot + 255) & ~size_t(255);
    const size_t ib = ((size_t)4 * tot + 255) & ~size_t(255);
    const size_t rb = (sizeof(R) * (size_t)tot + 255) & ~size_t(255);
    const size_t block = cb + (P.has_id ? ib : 0) + rb * (5 + (P.has_w ? 1 : 0));
    // each copy is one block of planes; a block that is large enough (and
    // not more than twice too large) is kept, so a re-sort or an upload of
    // the same size allocates nothing (the data it held is no longer needed:
    // callers have moved the particles to the staging area).  A new block
    // gets 1/8 headroom: tile capacities never shrink, so they creep up with
    // the scatter of the counts between uploads, and that growth should not
    // cost a free and an allocation of gigabytes each time.
    const size_t block_new = (block + block / 8 + 255) & ~size_t(255);
    for (int b = 0; b < 2; ++b) {
      if (P.store[b].p && P.store[b].bytes >= block && P.store[b].bytes <= 2 * block)
        continue;
      dfree(P.store[b]);
      if (!dalloc(P.store[b], block_new) && !dalloc(P.store[b], block))
        return fail(ZPIC_ENOMEM, "particle store");
    }
    if (!P.off.p) {
      if (!dalloc(P.off, 4 * S.ntiles) || !dalloc(P.cap, 4 * S.ntiles) ||
          !dalloc(P.cnt, 4 * S.ntiles) || !dalloc(P.ob_cnt, 4 * S.ntiles) ||
          !dalloc(P.arr, 4 * S.ntiles))
        return fail(ZPIC_ENOMEM, "tile tables");
      ZP_CU(cudaMemsetAsync(P.ob_cnt.p, 0, 4 * S.ntiles, stream_));
      ZP_CU(cudaMemsetAsync(P.arr.p, 0, 4 * S.ntiles, stream_));
    }
    if (!P.ob_ix.p) {  // outbox planes (again after the outbox grew)
      const size_t nob = (size_t)P.ob_cap * S.ntiles;
      if (!dalloc(P.ob_ix, 4 * nob) || !dalloc(P.ob_iy, 4 * nob) ||
          !dalloc(P.ob_x, sizeof(R) * nob) || !dalloc(P.ob_y, sizeof(R) * nob) ||
          !dalloc(P.ob_ux, sizeof(R) * nob) || !dalloc(P.ob_uy, sizeof(R) * nob) ||
          !dalloc(P.ob_uz, sizeof(R) * nob))
        return fail(ZPIC_ENOMEM, "outbox");
    }
    if (P.has_w && !P.ob_w.p &&
        !dalloc(P.ob_w, sizeof(R) * (size_t)P.ob_cap * S.ntiles))
      return fail(ZPIC_ENOMEM, "outbox w");
    if (P.has_id && !P.ob_id.p &&
        !dalloc(P.ob_id, 4 * (size_t)P.ob_cap * S.ntiles))
      return fail(ZPIC_ENOMEM, "outbox id");
    ZP_CU(cudaMemcpyAsync(P.off.p, off.data(), 4 * S.ntiles,
                          cudaMemcpyHostToDevice, stream_));
    ZP_CU(cudaMemcpyAsync(P.cap.p, cap.data(), 4 * S.ntiles,
                          cudaMemcpyHostToDevice, stream_));
    P.h_cap = cap;
    ZP_CU(cudaStreamSynchronize(stream_));  // host vectors go out of scope
    SpeciesDev<R> &Q = S.dev.sp[s];
    for (int b = 0; b < 2; ++b) {
      char *c = (char *)P.store[b].p;
      Planes<R> &L = Q.buf[b];
      L.cell = (uint16_t *)c;
      c += cb;
      L.id = nullptr;
      if (P.has_id) {
        L.id = (int *)c;
        c += ib;
      }
      R **reals[5] = {&L.x, &L.y, &L.ux, &L.uy, &L.uz};
      for (int a = 0; a < 5; ++a) {
        *reals[a] = (R *)c;
        c += rb;
      }
      L.w = P.has_w ? (R *)c : nullptr;
    }
    Q.off = (int *)P.off.p;
    Q.cap = (int *)P.cap.p;
    Q.cnt = (int *)P.cnt.p;
    Q.ob_cnt = (int *)P.ob_cnt.p;
    Q.arr = (int *)P.arr.p;
    Q.ob_ix = (int *)P.ob_ix.p;
    Q.ob_iy = (int *)P.ob_iy.p;
    Q.ob_id = (int *)P.ob_id.p;
    Q.ob_x = (R *)P.ob_x.p;
    Q.ob_y = (R *)P.ob_y.p;
    Q.ob_ux = (R *)P.ob_ux.p;
    Q.ob_uy = (R *)P.ob_uy.p;
    Q.ob_uz = (R *)P.ob_uz.p;
    Q.ob_w = (R *)P.ob_w.p;
    return ZPIC_OK;
  }

  int alloc_overflow() {
    const size_t n = (size_t)ovf_cap_;
    DevMem *ints[5] = {&ov_sim_, &ov_sp_, &ov_ix_, &ov_iy_, &ov_id_};
    DevMem *reals[6] = {&ov_x_, &ov_y_, &ov_ux_, &ov_uy_, &ov_uz_, &ov_w_};
    for (DevMem *m : ints)
      if (!dalloc(*m, 4 * n)) return fail(ZPIC_ENOMEM, "overflow buffer");
    for (DevMem *m : reals)
      if (!dalloc(*m, sizeof(R) * n)) return fail(ZPIC_ENOMEM, "overflow buffer");
    ovf_.cap = ovf_cap_;
    ovf_.sim = (int *)ov_sim_.p;
    ovf_.species = (int *)ov_sp_.p;
    ovf_.ix = (int *)ov_ix_.p;
    ovf_.iy = (int *)ov_iy_.p;
    ovf_.id = (int *)ov_id_.p;
    ovf_.x = (R *)ov_x_.p;
    ovf_.y = (R *)ov_y_.p;
    ovf_.ux = (R *)ov_ux_.p;
    ovf_.uy = (R *)ov_uy_.p;
    ovf_.uz = (R *)ov_uz_.p;
    ovf_.w = (R *)ov_w_.p;
    return ZPIC_OK;
  }

  int reset_status() {
    BatchStatus b{};
    b.err_step = INT_MAX;
    if (h_st_) b.step = h_st_->step;
    ZP_CU(cudaMemcpyAsync(st_mem_.p, &b, sizeof(b), cudaMemcpyHostToDevice,
                          stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    if (h_st_) *h_st_ = b;
    return ZPIC_OK;
  }

  int read_status() {
    ZP_CU(cudaMemcpyAsync(h_st_, st_mem_.p, sizeof(BatchStatus),
                          cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  int upload_descriptors() {
    // the single-simulation push kernel takes the descriptor by value, so a
    // captured graph holds a copy: capture again after any change (and only
    // then: an upload or re-sort that leaves every descriptor as it was
    // keeps the graph)
    ZP_CU(cudaStreamSynchronize(stream_));
    std::vector<SimDev<R>> h(n_sims);
    for (int i = 0; i < n_sims; ++i) h[i] = sims_[i].dev;
    if (sims_dev_.p && uploaded_.size() == h.size() &&
        std::memcmp(uploaded_.data(), h.data(), sizeof(SimDev<R>) * n_sims) == 0)
      return ZPIC_OK;
    invalidate_graph();
    uploaded_ = h;
    if (!sims_dev_.p && !dalloc(sims_dev_, sizeof(SimDev<R>) * n_sims))
      return fail(ZPIC_ENOMEM, "descriptors");
    ZP_CU(cudaMemcpyAsync(sims_dev_.p, h.data(), sizeof(SimDev<R>) * n_sims,
                          cudaMemcpyHostToDevice, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  // Work lists: particle tiles sorted by decreasing load (longest first),
  // Yee blocks in grid order.
  int build_items() {
    std::vector<std::pair<long long, int2>> load;
    int yee_n = 0;
    max_tx_ = max_ty_ = 2;
    end_g_max_ = 1;
    all16_ = true;
    for (int i = 0; i < n_sims; ++i) {
      SimHost<R> &S = sims_[i];
      max_tx_ = std::max(max_tx_, S.tx);
      max_ty_ = std::max(max_ty_, S.ty);
      all16_ = all16_ && S.tx == 16 && S.ty == 16;
      end_g_max_ = std::max(end_g_max_, S.dev.end_g);
      for (int t = 0; t < S.ntiles; ++t) {
        long long l = 0;
        for (auto &P : S.sp) l += P.h_cnt.empty() ? 0 : P.h_cnt[t];
        load.push_back({l, make_int2(i, t)});
      }
      yee_n += S.ybx * S.yby;
    }
    std::stable_sort(load.begin(), load.end(),
                     [](const std::pair<long long, int2> &a,
                        const std::pair<long long, int2> &b) {
                       return a.first > b.first;
                     });
    std::vector<int2> items(load.size()), yee;
    for (size_t k = 0; k < load.size(); ++k) items[k] = load[k].second;
    yee.reserve(yee_n);
    for (int i = 0; i < n_sims; ++i)
      for (int b = 0; b < sims_[i].ybx * sims_[i].yby; ++b)
        yee.push_back(make_int2(i, b));
    if (!items_.p) {
      if (!dalloc(items_, sizeof(int2) * std::max<size_t>(1, items.size())) ||
          !dalloc(yee_items_, sizeof(int2) * std::max<size_t>(1, yee.size())))
        return fail(ZPIC_ENOMEM, "work lists");
    }
    n_items_ = (int)items.size();
    n_yee_ = (int)yee.size();
    ZP_CU(cudaMemcpyAsync(items_.p, items.data(), sizeof(int2) * items.size(),
                          cudaMemcpyHostToDevice, stream_));
    ZP_CU(cudaMemcpyAsync(yee_items_.p, yee.data(), sizeof(int2) * yee.size(),
                          cudaMemcpyHostToDevice, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  int initial_state(int i) {
    SimHost<R> &S = sims_[i];
    const SimDev<R> *dptr = (const SimDev<R> *)sims_dev_.p + i;
    for (int s = 0; s < (int)S.sp.size(); ++s) {
      const zpic_species &p = S.sp[s].cfg;
      if (p.profile == ZPIC_PROFILE_NONE) continue;
      LoadParams lp{};
      lp.species = s;
      lp.key = sm_out(sm_out(S.cfg.seed, (uint64_t)S.cfg.sim_index + 1),
                      (uint64_t)s + 1);
      lp.ppc_x = p.ppc_x;
      lp.ppc_y = p.ppc_y;
      lp.lattice = p.lattice;
      for (int a = 0; a < 3; ++a) {
        lp.u_th[a] = p.u_th[a];
        lp.u_fl[a] = p.u_fl[a];
      }
      lp.profile = p.profile;
      lp.x0 = p.x0;
      lp.x1 = p.x1;
      lp.n0 = p.n0;
      profile_columns(p, S.nx, S.dx, &lp.col_lo, &lp.col_hi);
      lp.buf = 0;  // step 0 reads copy 0
      ZP_CU(launch_init_load<R>(dptr, S.ntiles, lp, stream_));
    }
    if (S.cfg.laser.enabled) {
      const zpic_laser &l = S.cfg.laser;
      LaserParams lp{l.a0 * l.omega0, l.omega0, l.w0, l.fwhm, l.x0, l.y_center};
      ZP_CU(launch_laser<R>(dptr, S.nx, S.ny, lp, stream_));
    }
    return ZPIC_OK;
  }

  // ---- staging and re-sorting --------------------------------------------------

  int ensure_staging(long long n) {
    if (n <= stg_n_) return ZPIC_OK;
    for (DevMem *m : {&sg_ix_, &sg_iy_, &sg_id_, &sg_tile_, &sg_x_, &sg_y_,
                      &sg_ux_, &sg_uy_, &sg_uz_, &sg_w_})
      dfree(*m);
    n = std::max<long long>(n, 1024);
    if (!dalloc(sg_ix_, 4 * n) || !dalloc(sg_iy_, 4 * n) ||
        !dalloc(sg_id_, 4 * n) || !dalloc(sg_tile_, 4 * n) ||
        !dalloc(sg_x_, sizeof(R) * n) || !dalloc(sg_y_, sizeof(R) * n) ||
        !dalloc(sg_ux_, sizeof(R) * n) || !dalloc(sg_uy_, sizeof(R) * n) ||
        !dalloc(sg_uz_, sizeof(R) * n) || !dalloc(sg_w_, sizeof(R) * n))
      return fail(ZPIC_ENOMEM, "staging buffers");
    stg_n_ = n;
    stg_.ix = (int *)sg_ix_.p;
    stg_.iy = (int *)sg_iy_.p;
    stg_.id = (int *)sg_id_.p;
    stg_.tile = (int *)sg_tile_.p;
    stg_.x = (R *)sg_x_.p;
    stg_.y = (R *)sg_y_.p;
    stg_.ux = (R *)sg_ux_.p;
    stg_.uy = (R *)sg_uy_.p;
    stg_.uz = (R *)sg_uz_.p;
    stg_.w = (R *)sg_w_.p;
    size_t need = 0;
    for (auto &S : sims_) need = std::max<size_t>(need, S.ntiles);
    if (stg_off_.bytes < sizeof(long long) * (need + 1)) {
      dfree(stg_off_);
      if (!dalloc(stg_off_, sizeof(long long) * (need + 1)))
        return fail(ZPIC_ENOMEM, "staging offsets");
    }
    if (!bad_.p && !dalloc(bad_, 4 * 2)) return fail(ZPIC_ENOMEM, "flags");
    return ZPIC_OK;
  }

  // Re-bins n staged particles into species s of sim si (new capacities).
  // Bins n staged particles into the species' tiles.  ready: an event after
  // which every staged plane other than cells and positions has arrived
  // (those two are in place when this is called), or null.
  int rebuild_species(int si, int s, long long n, bool has_w, bool has_id,
                      bool check, cudaEvent_t ready = nullptr) {
    SimHost<R> &S = sims_[si];
    SpeciesHost<R> &P = S.sp[s];
    DevMem counts;
    if (!dalloc(counts, 4 * S.ntiles)) return fail(ZPIC_ENOMEM, "counts");
    ZP_CU(cudaMemsetAsync(counts.p, 0, 4 * S.ntiles, stream_));
    ZP_CU(cudaMemsetAsync(bad_.p, 0, 4, stream_));
    ZP_CU(launch_bin_count<R>(stg_, n, S.nx, S.ny, S.tx, S.ty, S.ntx,
                              (int *)counts.p, (int *)bad_.p, stream_));
    std::vector<int> cnt(S.ntiles);
    int bad = 0;
    ZP_CU(cudaMemcpyAsync(cnt.data(), counts.p, 4 * S.ntiles,
                          cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaMemcpyAsync(&bad, bad_.p, 4, cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    dfree(counts);
    if (bad && check)
      return fail(ZPIC_EINVAL, "particles outside the grid or offsets not in [0,1)");
    const double slack = S.cfg.capacity_slack > 0 ? S.cfg.capacity_slack : 0.25;
    const double nominal = (double)P.cfg.ppc_x * P.cfg.ppc_y * S.tx * S.ty;
    ZP_TRY(alloc_store(si, s, cnt, slack, nominal,
                       full_tile_cap(nominal, slack, window_plasma(S, P))));
    ZP_CU(cudaMemsetAsync(P.cnt.p, 0, 4 * S.ntiles, stream_));
    ZP_CU(cudaMemsetAsync(P.ob_cnt.p, 0, 4 * S.ntiles, stream_));
    ZP_CU(cudaMemsetAsync(P.arr.p, 0, 4 * S.ntiles, stream_));
    if (ready) ZP_CU(cudaStreamWaitEvent(stream_, ready, 0));
    int pc = 0;
    ZP_TRY(particle_copy(si, &pc));
    ZP_CU(launch_bin_scatter<R>(stg_, n, S.dev.sp[s], pc, S.tx,
                                S.ty, has_w ? 1 : 0, has_id ? 1 : 0, stream_));
    P.h_cnt = cnt;
    ZP_TRY(upload_descriptors());
    ZP_TRY(build_items());
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  int read_counts(int si, int s) {
    SimHost<R> &S = sims_[si];
    SpeciesHost<R> &P = S.sp[s];
    P.h_cnt.resize(S.ntiles);
    ZP_CU(cudaMemcpyAsync(P.h_cnt.data(), P.cnt.p, 4 * S.ntiles,
                          cudaMemcpyDeviceToHost, stream_));
    ZP_CU(cudaStreamSynchronize(stream_));
    return ZPIC_OK;
  }

  // After ERR_OVERFLOW: every species of every sim with parked particles is
  // compacted, joined with its overflow entries and re-binned with more room.
  // A tile had more leavers in one step than its outbox holds (the excess
  // went to the overflow buffer): give every tile of the species an outbox
  // of twice that many (the planes are allocated again by alloc_store).
  int grow_outbox(int si, int s) {
    SimHost<R> &S = sims_[si];
    SpeciesHost<R> &P = S.sp[s];
    int need = 0;
    ZP_CU(cudaMemcpy(&need, S.dev.ob_need + s, sizeof(int),
                     cudaMemcpyDeviceToHost));
    if (need <= P.ob_cap) return ZPIC_OK;
    const long long cap = ((2LL * need + 31) / 32) * 32;
    if (cap * S.ntiles >= INT_MAX)
      return fail(ZPIC_EOVERFLOW, "outbox index range exceeded");
    for (DevMem *m : {&P.ob_ix, &P.ob_iy, &P.ob_x, &P.ob_y, &P.ob_ux,
                      &P.ob_uy, &P.ob_uz, &P.ob_w, &P.ob_id})
      dfree(*m);
    P.ob_cap = (int)cap;
    S.dev.sp[s].ob_cap = (int)cap;
    const int zero = 0;
    ZP_CU(cudaMemcpy(S.dev.ob_need + s, &zero, sizeof(int),
                     cudaMemcpyHostToDevice));
    return ZPIC_OK;
  }

  int resort_all() {
    NvtxRange r_("zpic re-sort after tile overflow");
    const int n_ovf = std::min(h_st_->ovf_count, ovf_cap_);
    std::vector<int> osim(n_ovf), osp(n_ovf);
    if (n_ovf > 0) {
      ZP_CU(cudaMemcpy(osim.data(), ovf_.sim, 4 * n_ovf, cudaMemcpyDeviceToHost));
      ZP_CU(cudaMemcpy(osp.data(), ovf_.species, 4 * n_ovf, cudaMemcpyDeviceToHost));
    }
    for (int si = 0; si < n_sims; ++si) {
      SimHost<R> &S = sims_[si];
      for (int s = 0; s < (int)S.sp.size(); ++s) {
        int extra = 0;
        for (int e = 0; e < n_ovf; ++e) extra += osim[e] == si && osp[e] == s;
        if (extra == 0) continue;
        ZP_TRY(read_counts(si, s));
        SpeciesHost<R> &P = S.sp[s];
        std::vector<long long> off(S.ntiles);
        long long n = 0;
        for (int t = 0; t < S.ntiles; ++t) {
          off[t] = n;
          n += P.h_cnt[t];
        }
        ZP_TRY(ensure_staging(n + extra + 1));
        ZP_CU(cudaMemcpyAsync(stg_off_.p, off.data(), sizeof(long long) * S.ntiles,
                              cudaMemcpyHostToDevice, stream_));
        int pc = 0;
        ZP_TRY(particle_copy(si, &pc));
        ZP_CU(launch_compact<R>(S.dev.sp[s], pc, S.tx, S.ty,
                                S.ntx, 0, S.ntiles,
                                (const long long *)stg_off_.p, stg_, stream_));
        ZP_CU(cudaMemsetAsync(bad_.p, 0, 4, stream_));
        ZP_CU(launch_take_overflow<R>(ovf_, n_ovf, si, s, stg_, n,
                                      (int *)bad_.p, stream_));
        ZP_CU(cudaStreamSynchronize(stream_));
        ZP_TRY(grow_outbox(si, s));
        // copies of the compacted store are in staging now; rebuild
        ZP_TRY(rebuild_species(si, s, n + extra, S.sp[s].has_w,
                               S.sp[s].has_id, false));
      }
    }
    ++resorts_;
    ZP_TRY(reset_status());
    return ZPIC_OK;
  }

  // The current copy of simulation si's particle store, (step & 1) ^ pswap
  // (the device flips pswap after a cell-order re-sort); after a sync.
  int particle_copy(int si, int *pc) {
    int p = 0;
    ZP_CU(cudaMemcpy(&p, sims_[si].dev.pswap, sizeof(int),
                     cudaMemcpyDeviceToHost));
    *pc = (h_st_->step & 1) ^ (p & 1);
    return ZPIC_OK;
  }

  // Resident push CTAs per SM of the batch: its first member's setting
  // (0: all that fit), reported as the number in use.
  int resolved_ctas() const {
    const SimHost<R> &S = sims_[0];
    const int fit = push_ctas_fit<R>(max_tx_, max_ty_, ring_wide());
    return S.ctas > 0 && S.ctas < fit ? S.ctas : fit;
  }

  // ---- launch sequence ---------------------------------------------------------

  const SimDev<R> *dsims() const { return (const SimDev<R> *)sims_dev_.p; }
  // some species of some simulation stores weights or ids
  bool ring_wide() const {
    for (const auto &S : sims_)
      for (const auto &P : S.sp)
        if (P.has_w || P.has_id) return true;
    return false;
  }
  BatchStatus *dst() const { return (BatchStatus *)st_mem_.p; }

  // the kernels of one step, in order (the filter only when some
  // simulation of the batch filters its current)
  std::vector<int> stages() const {
    bool filter = false, sort = false;
    for (const auto &S : sims_) {
      filter = filter || S.dev.Jf[0] != nullptr;
      sort = sort || S.dev.sort_every > 0;
    }
    std::vector<int> k = {0};
    if (filter) k.push_back(4);
    k.push_back(1);
    k.push_back(2);
    if (sort) k.push_back(5);
    k.push_back(3);
    return k;
  }

  cudaError_t launch_stage(int k) {
    if (fault("launch")) return cudaErrorLaunchFailure;
    switch (k) {
      case 0:
        return launch_push_deposit<R>(dsims(), n_sims == 1 ? &sims_[0].dev : nullptr,
                                      (const int2 *)items_.p, n_items_,
                                      max_tx_, max_ty_, all16_, ring_wide(),
                                      sims_[0].ctas, dst(), ovf_, stream_);
      case 1:
        return launch_yee<R>(dsims(), (const int2 *)yee_items_.p, n_yee_,
                             dst(), stream_);
      case 2:
        return launch_migrate<R>(dsims(), (const int2 *)items_.p, n_items_,
                                 dst(), ovf_, stream_);
      case 3:
        return launch_end_step<R>(dsims(), n_sims, end_g_max_, dst(), stream_);
      case 5:
        return launch_sort_tiles<R>(dsims(), n_sims, (const int2 *)items_.p,
                                    n_items_, dst(), stream_);
      default:
        return launch_filter<R>(dsims(), (const int2 *)yee_items_.p, n_yee_,
                                dst(), stream_);
    }
  }
  static const char *stage_name(int k) {
    static const char *names[6] = {"push_deposit", "yee", "migrate",
                                   "end_step", "filter_current",
                                   "sort_tiles"};
    return names[k];
  }

  int enqueue(int n) {
    if (n == 0) return ZPIC_OK;
    if (profiling_) {
      ZP_CU(prepare_push_deposit<R>(max_tx_, max_ty_, ring_wide()));
      ZP_CU(prepare_sort_tiles<R>());
      const std::vector<int> order = stages();
      if (timers_.size() != order.size()) {
        timers_.clear();
        for (int k : order) {
          timers_.emplace_back();
          timers_.back().name = stage_name(k);
        }
      }
      for (int i = 0; i < n; ++i)
        for (size_t t = 0; t < order.size(); ++t) {
          cudaEvent_t a, b;
          ZP_CU(cudaEventCreate(&a));
          ZP_CU(cudaEventCreate(&b));
          ZP_CU(cudaEventRecord(a, stream_));
          NvtxRange r_(stage_name(order[t]));
          ZP_CU(launch_stage(order[t]));
          ZP_CU(cudaEventRecord(b, stream_));
          timers_[t].ev.push_back({a, b});
        }
      return ZPIC_OK;
    }
    if (!graph_exec_) ZP_TRY(capture());
    if (fault("launch")) return cuda_fail(cudaErrorLaunchFailure, "graph launch");
    for (int i = 0; i < n; ++i) ZP_CU(cudaGraphLaunch(graph_exec_, stream_));
    return ZPIC_OK;
  }

  int capture() {
    NvtxRange r_("zpic graph capture");
    // kernel attributes are set outside the capture
    ZP_CU(prepare_push_deposit<R>(max_tx_, max_ty_, ring_wide()));
    ZP_CU(prepare_sort_tiles<R>());
    cudaStream_t cs;
    ZP_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t keep = stream_;
    stream_ = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int k : stages())
        if (e == cudaSuccess) e = launch_stage(k);
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      if (e == cudaSuccess) e = e2;
    }
    stream_ = keep;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "graph capture");
    }
    e = cudaGraphInstantiate(&graph_exec_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    return ZPIC_OK;
  }

  void invalidate_graph() {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
  }

  void release() {
    if (stream_) cudaStreamSynchronize(stream_);
    invalidate_graph();
    for (auto &t : timers_)
      for (auto &e : t.ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
    if (alloc_) {
      for (auto &S : sims_) {
        for (auto &P : S.sp)
          for (DevMem *m : {&P.store[0], &P.store[1], &P.off, &P.cap, &P.cnt,
                            &P.ob_cnt, &P.arr, &P.ob_ix,
                            &P.ob_iy, &P.ob_id, &P.ob_x, &P.ob_y, &P.ob_ux,
                            &P.ob_uy, &P.ob_uz, &P.ob_w})
            dfree(*m);
        for (DevMem *m : {&S.fields, &S.part_kin, &S.part_fld, &S.epart,
                          &S.hist, &S.small, &S.energy_rows})
          dfree(*m);
      }
      for (DevMem *m : {&st_mem_, &sims_dev_, &items_, &yee_items_, &ov_sim_,
                        &ov_sp_, &ov_ix_, &ov_iy_, &ov_id_, &ov_x_, &ov_y_,
                        &ov_ux_, &ov_uy_, &ov_uz_, &ov_w_, &sg_ix_, &sg_iy_,
                        &sg_id_, &sg_tile_, &sg_x_, &sg_y_, &sg_ux_, &sg_uy_,
                        &sg_uz_, &sg_w_, &stg_off_, &bad_})
        dfree(*m);
    }
    if (h_st_) cudaFreeHost(h_st_);
    h_st_ = nullptr;
    if (cpy_) {
      cudaStreamSynchronize(cpy_);
      cudaStreamDestroy(cpy_);
    }
    cpy_ = nullptr;
    if (ev_pos_) cudaEventDestroy(ev_pos_);
    if (ev_mom_) cudaEventDestroy(ev_mom_);
    ev_pos_ = ev_mom_ = nullptr;
    if (own_stream_) cudaStreamDestroy(own_stream_);
    own_stream_ = nullptr;
    stream_ = nullptr;
  }

  std::vector<SimHost<R>> sims_;
  std::unique_ptr<Allocator> alloc_;
  cudaStream_t own_stream_ = nullptr, stream_ = nullptr;
  // second stream for host transfers that overlap the library stream's
  // kernels (particle upload and download), with the events that order them
  cudaStream_t cpy_ = nullptr;
  cudaEvent_t ev_pos_ = nullptr, ev_mom_ = nullptr;
  size_t bytes_ = 0;
  DevMem st_mem_, sims_dev_, items_, yee_items_;
  DevMem ov_sim_, ov_sp_, ov_ix_, ov_iy_, ov_id_, ov_x_, ov_y_, ov_ux_, ov_uy_,
      ov_uz_, ov_w_;
  DevMem sg_ix_, sg_iy_, sg_id_, sg_tile_, sg_x_, sg_y_, sg_ux_, sg_uy_, sg_uz_,
      sg_w_, stg_off_, bad_;
  Staging<R> stg_{};
  long long stg_n_ = 0;
  OverflowDev<R> ovf_{};
  int ovf_cap_ = 0;
  int n_items_ = 0, n_yee_ = 0, max_tx_ = 2, max_ty_ = 2;
  bool all16_ = false;
  int end_g_max_ = 1;  // most end-of-step slices of a member
  BatchStatus *h_st_ = nullptr;
  std::vector<SimDev<R>> uploaded_;  // descriptors as last uploaded
  long long target_ = 0;
  int sticky_ = ZPIC_OK;
  int resorts_ = 0;
  bool profiling_ = false;
  std::vector<Timer<R>> timers_;
  cudaGraphExec_t graph_exec_ = nullptr;
};

int make_batch(const zpic_config *cfgs, int n, zpic_batch **out) {
  if (!out) return fail(ZPIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || n < 1) return fail(ZPIC_EINVAL, "no configs");
  for (int i = 0; i < n; ++i) ZP_TRY(validate(&cfgs[i]));
  for (int i = 1; i < n; ++i)
    if (cfgs[i].precision != cfgs[0].precision)
      return fail(ZPIC_EINVAL, "all sims of a batch share one precision");
  // Members of a batch (two or more simulations) that leave a setting at 0
  // take the batch's tuning (zpic_batch_autotune) if it has run, else a
  // 16 x 16 tile (the batched kernel compiled for it) and the other
  // settings as for a single simulation.  The per-class tile sizes of
  // zpic_autotune are not used here: they are chosen for a simulation that
  // has the GPU to itself, and a batch whose members differ in tile size
  // runs the slower generic kernel.
  std::vector<zpic_config> own;
  if (n > 1) {
    own.assign(cfgs, cfgs + n);
    zpic_tuning t{};
    const bool tuned = tuned_batch(cfgs, n, &t);
    for (auto &c : own) {
      if (c.tile_x == 0 && c.tile_y == 0) {
        c.tile_x = tuned ? t.tile_x : 16;
        c.tile_y = tuned ? t.tile_y : 16;
      }
      if (tuned && c.sort_every == 0) c.sort_every = t.sort_every;
      if (tuned && c.push_ctas_per_sm == 0)
        c.push_ctas_per_sm = t.push_ctas_per_sm;
    }
    cfgs = own.data();
  }
  std::unique_ptr<zpic_batch> b(new zpic_batch);
  if (cfgs[0].precision == ZPIC_FP64)
    b->impl.reset(new Batch<double>());
  else
    b->impl.reset(new Batch<float>());
  int r = b->impl->init(cfgs, n);
  if (r != ZPIC_OK) return r;
  for (int i = 0; i < n; ++i) b->views.push_back(new zpic_sim{b.get(), i, false});
  *out = b.release();
  return ZPIC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

#define ZP_SIM(sim)                                               \
  if (!(sim) || !(sim)->b) return fail(ZPIC_EINVAL, "NULL handle"); \
  BatchBase *B = (sim)->b->impl.get();                            \
  const int I = (sim)->index;

extern "C" {

int zpic_create(const zpic_config *cfg, zpic_sim **out) {
  NvtxRange r_("zpic_create");
  if (!out) return fail(ZPIC_EINVAL, "out is NULL");
  *out = nullptr;
  zpic_batch *b = nullptr;
  ZP_TRY(make_batch(cfg, 1, &b));
  zpic_sim *s = b->views[0];
  s->owns = true;
  *out = s;
  return ZPIC_OK;
}

int zpic_destroy(zpic_sim *sim) {
  if (!sim || !sim->b) return fail(ZPIC_EINVAL, "NULL handle");
  if (!sim->owns) return fail(ZPIC_EINVAL, "batch views are freed with the batch");
  return zpic_batch_destroy(sim->b);
}

int zpic_step(zpic_sim *sim, int n) {
  NvtxRange r_("zpic_step");
  ZP_SIM(sim);
  (void)I;
  if (!sim->owns) return fail(ZPIC_EINVAL, "step a batch view with zpic_batch_step");
  return B->step(n);
}

int zpic_sync(zpic_sim *sim) {
  NvtxRange r_("zpic_sync");
  ZP_SIM(sim);
  (void)I;
  return B->sync();
}

int zpic_set_stream(zpic_sim *sim, void *stream) {
  ZP_SIM(sim);
  (void)I;
  return B->set_stream(stream);
}

int zpic_get_fields_f32(zpic_sim *sim, int which, float *dst, size_t cap) {
  ZP_SIM(sim);
  return B->get_fields(I, which, dst, cap, 0);
}

int zpic_get_fields_f64(zpic_sim *sim, int which, double *dst, size_t cap) {
  ZP_SIM(sim);
  return B->get_fields(I, which, dst, cap, 1);
}

int zpic_set_fields_f64(zpic_sim *sim, int which, const double *src, size_t n) {
  ZP_SIM(sim);
  return B->set_fields_f64(I, which, src, n);
}

int zpic_num_particles(zpic_sim *sim, int species, int64_t *n) {
  ZP_SIM(sim);
  return B->num_particles(I, species, n);
}

int zpic_get_particles(zpic_sim *sim, int species, const zpic_particles *dst,
                       size_t *n_written) {
  NvtxRange r_("zpic_get_particles");
  ZP_SIM(sim);
  return B->get_particles(I, species, 0, -1, dst, n_written);
}

int zpic_get_particles_tiles(zpic_sim *sim, int species, int tile_begin,
                             int tile_end, const zpic_particles *dst,
                             size_t *n_written) {
  ZP_SIM(sim);
  if (tile_end < 0) return fail(ZPIC_EINVAL, "tile range");
  return B->get_particles(I, species, tile_begin, tile_end, dst, n_written);
}

int zpic_set_particles(zpic_sim *sim, int species, const zpic_particles *src) {
  NvtxRange r_("zpic_set_particles");
  ZP_SIM(sim);
  return B->set_particles(I, species, src);
}

int zpic_energy(zpic_sim *sim, zpic_energy_rec *dst, size_t cap,
                size_t *n_written) {
  ZP_SIM(sim);
  return B->energy(I, dst, cap, n_written);
}

int zpic_field_energy(zpic_sim *sim, double *wE, double *wB) {
  ZP_SIM(sim);
  return B->field_energy(I, wE, wB);
}

int zpic_get_info(zpic_sim *sim, zpic_info *info) {
  ZP_SIM(sim);
  return B->info(I, info);
}

int zpic_get_tile_counts(zpic_sim *sim, int species, int32_t *dst, size_t cap) {
  ZP_SIM(sim);
  return B->tile_counts(I, species, dst, cap);
}

int zpic_get_state(zpic_sim *sim, zpic_state *out) {
  ZP_SIM(sim);
  return B->get_state(I, out);
}

int zpic_set_state(zpic_sim *sim, const zpic_state *in) {
  ZP_SIM(sim);
  return B->set_state(I, in);
}

int zpic_phasespace(zpic_sim *sim, int species, int qx, int qy,
                    const double range[4], int nbx, int nby, double *dst,
                    size_t cap) {
  ZP_SIM(sim);
  return B->phasespace(I, species, qx, qy, range, nbx, nby, dst, cap);
}

int zpic_profile_enable(zpic_sim *sim, int enable) {
  ZP_SIM(sim);
  (void)I;
  return B->profile_enable(enable);
}

int zpic_profile_read(zpic_sim *sim, char *names, size_t name_len,
                      double *ms_total, int32_t *launches, int cap, int *n,
                      int reset) {
  ZP_SIM(sim);
  (void)I;
  return B->profile_read(names, name_len, ms_total, launches, cap, n, reset);
}

int zpic_batch_create(const zpic_config *cfgs, int n, zpic_batch **out) {
  return make_batch(cfgs, n, out);
}

int zpic_batch_step(zpic_batch *b, int n) {
  NvtxRange r_("zpic_batch_step");
  if (!b) return fail(ZPIC_EINVAL, "NULL batch");
  return b->impl->step(n);
}

int zpic_batch_sync(zpic_batch *b) {
  NvtxRange r_("zpic_batch_sync");
  if (!b) return fail(ZPIC_EINVAL, "NULL batch");
  return b->impl->sync();
}

int zpic_batch_sim(zpic_batch *b, int i, zpic_sim **view) {
  if (!b || !view) return fail(ZPIC_EINVAL, "NULL argument");
  if (i < 0 || i >= (int)b->views.size()) return fail(ZPIC_EINVAL, "index");
  *view = b->views[i];
  return ZPIC_OK;
}

int zpic_batch_set_stream(zpic_batch *b, void *stream) {
  if (!b) return fail(ZPIC_EINVAL, "NULL batch");
  return b->impl->set_stream(stream);
}

int zpic_batch_profile_enable(zpic_batch *b, int enable) {
  if (!b) return fail(ZPIC_EINVAL, "NULL batch");
  return b->impl->profile_enable(enable);
}

int zpic_batch_destroy(zpic_batch *b) {
  if (!b) return fail(ZPIC_EINVAL, "NULL batch");
  for (zpic_sim *v : b->views) delete v;
  b->views.clear();
  b->impl.reset();
  delete b;
  return ZPIC_OK;
}

int zpic_set_allocator(zpic_alloc_fn alloc, zpic_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(ZPIC_EINVAL, "give both hooks or neither");
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return ZPIC_OK;
}

const char *zpic_strerror(int code) {
  switch (code) {
    case ZPIC_OK: return "ok";
    case ZPIC_EINVAL: return "invalid argument";
    case ZPIC_ECFL: return "time step violates the Courant condition";
    case ZPIC_ENOMEM: return "out of memory";
    case ZPIC_ECUDA: return "CUDA error";
    case ZPIC_EOVERFLOW: return "particle storage overflow";
    case ZPIC_ENAN: return "non-finite value";
    case ZPIC_ETIMEOUT: return "device wait timed out";
    case ZPIC_ECAP: return "destination buffer too small";
    case ZPIC_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

const char *zpic_last_error(void) { return g_last_error.c_str(); }

int zpic_version(void) { return ZPIC_VERSION; }

}  // extern "C"
