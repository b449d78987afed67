// zpic_dev.cuh -- device-side data layout of the GB300 PIC library.
//
// One "batch" holds one or more independent simulations that advance in
// lockstep.  Every kernel walks a work list of (simulation, tile) items and
// reads the simulation's SimDev descriptor from device memory, so a single
// simulation is simply a batch of one.
//
// HBM layout per simulation (R = float or double):
//   fields: E[2][3], B[2][3], J[2][3] arrays of ny rows x ld (ld = nx padded
//           to 128 bytes); copy (step & 1) is current, the Yee kernel
//           writes copy (step & 1) ^ 1 (ping-pong, no halo races); J holds
//           8-byte values (int64 fixed point in FP32, double in FP64); with
//           the current filter on, 3 more arrays Jf hold the filtered J;
//   particles, per species: SoA arrays cell (uint16, cell within the tile),
//           x, y, ux, uy, uz (R), optional w (R) and id (int32), one segment per
//           tile [off[t], off[t] + cap[t]) of which cnt[t] are live; two
//           copies (read one, write the other each step; which one is
//           current is (step & 1) ^ *pswap);
//   outbox, per species: ob_cap slots per tile for particles that leave it.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/zpic.h"

namespace zp {

constexpr int kMaxSpecies = ZPIC_MAX_SPECIES;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// CTAs that share the end-of-step energy reduction of one simulation (each
// sums a slice of the partials; the last one to finish combines them): one
// per 640 partial values, at most kEndSlicesMax.  The FP64 sums run on the
// GPU's few FP64 units, so a large grid spreads them over many SMs (64
// slices for a 2048^2 grid: 0.037 ms per step, 0.041 ms with 16), a small
// one keeps the fixed cost of each slice's reduction tree low (the
// 256-simulation batch: 0.008 ms, 0.016 ms with 16 slices each).  The count depends on
// the simulation alone, so it gives the same bits in a batch and alone.
constexpr int kEndSlicesMax = 64;
__host__ __device__ inline int end_slices(int ntiles, int nsp, int nyb) {
  const long long parts = (long long)ntiles * nsp + 2LL * nyb;
  const long long g = (parts + 639) / 640;
  return (int)(g < 1 ? 1 : (g > kEndSlicesMax ? kEndSlicesMax : g));
}
// Values of one slice: kinetic energy per species, E^2, B^2.
constexpr int kEndQ = kMaxSpecies + 2;

// BatchStatus::error bits
constexpr int ERR_OVERFLOW = 1;  // particles parked in the overflow buffer
constexpr int ERR_LOST = 2;      // overflow buffer full: particles dropped
constexpr int ERR_NAN = 4;       // non-finite energy
constexpr int ERR_STORE = 8;     // a stored particle lies outside its tile
constexpr int ERR_TIMEOUT = 16;  // a bounded device wait gave up (reported as
                                 // ZPIC_ETIMEOUT): the re-sort's wait for a
                                 // bulk copy into shared memory

struct BatchStatus {
  int step;         // completed steps
  int error;        // ERR_* bits
  int err_step;     // step that raised the first error (valid if error)
  int ovf_count;    // entries claimed in the overflow buffer
  int lost;         // particles dropped (overflow buffer full)
  int blocks_done;  // ticket counter of the end-of-step kernel
  int push_next;    // next work item of the persistent push kernel
  int pad;
};

// One copy of a species' tile store: SoA planes (w, id may be null).  The
// tile of a particle is implied by the segment it sits in, so only its cell
// within the tile is stored: cell = (ly << 8) | lx (tiles up to 256 x 256).
template <typename R>
struct Planes {
  uint16_t *cell;
  int *id;
  R *x, *y, *ux, *uy, *uz, *w;
};

__host__ __device__ __forceinline__ uint16_t local_cell(int lx, int ly) {
  return (uint16_t)((ly << 8) | lx);
}

template <typename R>
struct SpeciesDev {
  R qm;          // charge-to-mass ratio
  R hq;          // (q/m) dt / 2 : Boris half-kick factor
  R qx, qy;      // q0 dx/dt, q0 dy/dt : Jx, Jy per unit cell displacement
  R q0;          // charge of a weight-1 particle
  R dq[3];       // deposit factors of the shared current tile per component:
                 // FP32: (q0 / Uq) 2^16 (fixed-point units, see SimDev);
                 // FP64: q0 dx/dt, q0 dy/dt, q0 (physical units)
  double kin_scale;  // (q0 / (q/m)) dx dy : mass x cell area, weight 1
  // two copies of the store with one segment layout: the push of step n
  // reads buf[(n & 1) ^ pswap] and writes the other one
  Planes<R> buf[2];
  int *off, *cap, *cnt;            // per tile
  int ob_cap;                      // outbox slots per tile
  int *ob_cnt;                     // per tile
  int *arr;                        // per tile: arrivals claimed this step
  int *ob_ix, *ob_iy, *ob_id;
  R *ob_x, *ob_y, *ob_ux, *ob_uy, *ob_uz, *ob_w;
  // moving-window injection of cold plasma on a lattice
  int inj_ppc_x, inj_ppc_y;        // 0: no injection
  double ramp_x0, ramp_len, n0;
  long long id_base;
};

template <typename R>
struct SimDev {
  int nx, ny, ld;
  int tx, ty, ntx, nty;        // particle tiles
  int ybx, yby;                // Yee blocks in x, y
  int open_x, moving_window;
  int energy_every;
  int nsp;
  R dx, dy, dt;
  R dt_dx, dt_dy;              // dt/dx, dt/dy (cells per unit velocity)
  double dx_d, dy_d, dt_d;     // double values (window schedule, setup)
  R *E[2][3], *B[2][3];
  // deposited current, two copies: FP32 keeps exact fixed-point sums in
  // int64 (units of 2^-30, scaled by jscale when read), so its value does
  // not depend on the order of the tiles' adds; FP64 keeps doubles
  long long *Jq[2][3];         // FP32 (null in FP64)
  R *J[2][3];                  // FP64 (null in FP32)
  R *Jf[3];                    // filtered current (null: no filter)
  // FP32 tiles accumulate J exactly in two-word fixed point with 2^-30 units
  // of Uq dx/dt, Uq dy/dt, Uq (Uq = max |q0| x max weight, so one segment
  // contributes at most one unit) and add it to Jq; a sum v reads as
  // J = float(v) * jscale, two FP32 roundings (no FP64 on the field path).
  float jscale[3];
  // FP64 with ZPIC_DETERMINISTIC: J words hold int64 fixed-point sums
  // (units 2^-47 of Uq dx/dt, Uq dy/dt, Uq), read as value * jscale_d
  int jfixed;
  double jscale_d[3];
  double *part_kin;            // [kMaxSpecies][ntiles] kinetic partials
  double *part_fld;            // [ybx*yby][2] field-energy partials
  double *epart;               // [end_g][kEndQ][2] compensated sums
                               // (sum, error) of the end-of-step slices
  int *eticket;                // slices of this simulation finished
  int end_g;                   // end-of-step slices of this simulation
  zpic_energy_rec *hist;       // energy history
  int hist_cap;
  int hist_skip;               // records before the first one kept (a run
                               // restored at step s keeps those after s)
  int *hist_n;                 // records written
  int *n_shift;                // window shifts done
  int *removed;                // [kMaxSpecies] particles removed at edges
  int *ob_need;                // [kMaxSpecies] most leavers one tile had in
                               // a step when that exceeded its outbox
                               // (0: none); the re-sort grows the outbox
  int *variants;               // [kMaxSpecies] bits of the push-kernel forms
                               // that ran for the species (ZPIC_PUSH_*)
  // Which copy of the particle store is current: copy (step & 1) ^ *pswap.
  // The re-sort after step n (when due) writes the other copy in cell-
  // interleaved order and the end-of-step kernel flips *pswap, so the next
  // push reads the sorted copy.  *sorts counts the re-sorts.
  int *pswap;
  int *sorts;
  int sort_every;              // re-sort interval in steps; <= 0: never
  SpeciesDev<R> sp[kMaxSpecies];
};

// Particles that found no room (outbox or tile full) wait here until the
// host re-sorts the batch.
template <typename R>
struct OverflowDev {
  int cap;
  int *sim, *species, *ix, *iy, *id;
  R *x, *y, *ux, *uy, *uz, *w;
};

// --- small device helpers --------------------------------------------------

__device__ __forceinline__ int wrap1(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Window schedule: shift after step `step` if (step+1) dt >= (n_shift+1) dx.
// Evaluated in double exactly as written so every kernel (and any other
// implementation of the same rule) takes the same decision.
template <typename R>
__device__ __forceinline__ bool shift_due(const SimDev<R> &S, int step,
                                          int n_shift) {
  return S.moving_window &&
         ((double)(step + 1) * S.dt_d >= (double)(n_shift + 1) * S.dx_d);
}

// The particle re-sort runs after step `step` (before the step counter
// advances) every sort_every steps.
template <typename R>
__device__ __forceinline__ bool sort_due(const SimDev<R> &S, int step) {
  return S.sort_every > 0 && ((step + 1) % S.sort_every) == 0;
}

// Float with the bit pattern b (host and device).
__host__ __device__ __forceinline__ float float_of_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// FP32 value of an int64 fixed-point sum v, |v| < 2^54, in FP32 arithmetic
// only (a 64-bit integer conversion would run on the FP64 pipe): v = h 2^32
// + m 2^16 + l with h signed (|h| < 2^22) and m, l in [0, 2^16); each part
// is exact as a float by the add-the-exponent trick (bits of 2^23 (+2^22)
// plus the integer, minus that float), then fmaf(h, 2^32, m 2^16) + l rounds
// twice.  Host and device evaluate the same operations, so the current the
// field solver uses and the one the API reports agree bit for bit.
__host__ __device__ __forceinline__ float fixed_to_float(long long v) {
  const int h = (int)(v >> 32);
  const uint32_t lo = (uint32_t)(unsigned long long)v;
  const float fh = float_of_bits(0x4B400000u + (uint32_t)h) - 12582912.0f;
  const float fm = float_of_bits(0x4B000000u | (lo >> 16)) - 8388608.0f;
  const float fl = float_of_bits(0x4B000000u | (lo & 0xFFFFu)) - 8388608.0f;
  const float hm = fmaf(fh, 4294967296.0f, fm * 65536.0f);
  return hm + fl;
}

// This step's deposited current of component c at array index idx, as R.
template <typename R>
__device__ __forceinline__ R j_value(const SimDev<R> &S, int cur, int c,
                                     size_t idx) {
  if constexpr (sizeof(R) == 4)
    return fixed_to_float(S.Jq[cur][c][idx]) * S.jscale[c];
  else if (S.jfixed)
    return (double)__double_as_longlong(S.J[cur][c][idx]) * S.jscale_d[c];
  else
    return S.J[cur][c][idx];
}

__device__ __forceinline__ bool frozen(const BatchStatus *st, int step) {
  // after an error in an earlier step, later steps are held back until the
  // host has recovered (the step counter stops, the host re-runs them)
  return st->error != 0 && st->err_step < step;
}

// --- SplitMix64 (Steele, Lea & Flood 2014), counter form -------------------

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// k-th output (k >= 1) of a SplitMix64 generator seeded with s
__host__ __device__ __forceinline__ uint64_t sm_out(uint64_t s, uint64_t k) {
  return sm_mix(s + k * 0x9E3779B97F4A7C15ull);
}

}  // namespace zp
