// k_push.cu -- fused particle kernel: interpolation, Boris push, move,
// charge-conserving deposition and in-tile compaction (PIC stages 1-3 of
// Sec. 2.2; the per-region particle advance with local current buffers and
// a ghost-cell reduction of Sec. 3.2, here one CTA per tile at a time).
//
// Persistent: the resident CTAs take (simulation, tile) items, longest
// first, from a device counter.  Per item the CTA
//  1. stages E, B of the tile plus one guard cell on each side and turns
//     them into a coefficient tile (the bilinear interpolant of every cell
//     of every staggered component), and zeroes a shared J tile covering
//     [-1, tx+1] x [-1, ty+1];
//  2. streams the tile's particles in chunks of 32 per warp, the next
//     chunk's records arriving through a per-warp ring of asynchronous
//     copies: bilinear gather from the coefficient tile, relativistic Boris
//     rotation, move by dt u/gamma (at most one cell, CFL), split of the
//     straight path at the cell faces it crosses; the segment in the start
//     cell goes straight into the shared J tile (exact fixed point), the
//     paths of particles that cross a face wait in a per-warp queue and
//     their remaining segments are deposited 32 at a time;
//  3. writes particles that stay in the tile to the tile's segment of the
//     other copy of the store in their input order: each warp owns a
//     contiguous range of the segment and compacts its stayers to the start
//     of that range, and the CTA then moves the last particles into the
//     gaps (close_gaps), so warps never wait for each other and the order of
//     the store (neighbouring slots in neighbouring cells after a re-sort)
//     carries over from step to step; particles that leave go to the tile's
//     outbox, particles leaving an open boundary are dropped;
//  4. adds the shared J tile (interior and guard cells) to the global J,
//     one reduction per cell (periodic images folded here); in FP32 the
//     global J is an int64 fixed-point sum, so the result does not depend
//     on the order of the tiles.
// Traffic per particle: one read and one write of its SoA record (16-bit
// cell within the tile + 5 reals: 22 bytes in FP32).
#include <type_traits>

#include "zpic_dev.cuh"
#include "zpic_kernels.h"

namespace zp {

// CTA shape of the push kernel: kPT threads (kPW warps) per tile, and the
// CTAs per SM that the FP32 register budget is sized for.
constexpr int kPT = 256;
constexpr int kPW = kPT / 32;
constexpr int kPushCtasF32 = 3;
// the batched kernel reads its descriptors from global memory and needs
// more registers
constexpr int kPushCtasF32Batch = 3;
// the batched kernel copies each work item's descriptor into shared memory
// (measured on the 256-simulation sweep: 3.53 ms per push against 3.65 ms
// reading it from global memory)
constexpr bool kBatchDescInSmem = true;

template <typename R>
__device__ __forceinline__ R rsqrt_r(R v);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double v) { return rsqrt(v); }

template <typename R>
__device__ __forceinline__ R fdiv(R a, R b);
template <>
__device__ __forceinline__ float fdiv<float>(float a, float b) {
  return __fdividef(a, b);
}
template <>
__device__ __forceinline__ double fdiv<double>(double a, double b) {
  return a / b;
}

// Crossing decision on one axis: cross iff o1 >= 1 or o1 < 0; a backward
// crossing whose new offset rounds to exactly 1 stays in the cell at offset
// 0.  Returns the cell step; of = stored offset; o1 becomes the path end in
// the start cell's frame (0 after that rounding fix).  Written with selects
// only, so lanes never diverge here.
template <typename R>
__device__ __forceinline__ int axis_cross(R &o1, R &of) {
  const bool fwd = o1 >= R(1), back = o1 < R(0);
  const R t = o1 + R(1);
  const bool fix = back && t == R(1);
  of = fwd ? o1 - R(1) : (back ? (fix ? R(0) : t) : o1);
  o1 = fix ? R(0) : o1;
  return fwd ? 1 : ((back && !fix) ? -1 : 0);
}

// Shared current tile.  FP32: each value is an exact fixed-point sum held
// in two int32 words: a contribution t = c 2^16 (|c| <= 1 unit) is split
// into h = round(t) and l = round((t - h) 2^14) in [-2^13, 2^13], so the
// value is h 2^14 + l in units of 2^-30.  Both roundings use the float
// "add 1.5 2^23" trick (exact for |t| < 2^22): the words receive the bit
// patterns K + h and K + l (K = 0x4B400000) and the bias n K of a word that
// received n adds is removed when the tile is folded, n coming from a count
// of segments per base cell.  Integer shared atomics are native (float ones
// are not) and integer sums do not depend on the order of the adds.  Exact
// while one word receives fewer than 2^18 adds per step and the net sum
// stays below 2^15 units.  FP64: plain double atomics.
template <typename R>
struct TileJ;

template <>
struct TileJ<float> {
  int *hi;   // 3 planes
  int *lo;   // 3 planes
  int *cnt;  // segments per base cell (one plane)
  static constexpr unsigned kBias = 0x4B400000u;  // bits of 1.5 * 2^23
  __device__ __forceinline__ void seg(int b) const { atomicAdd(cnt + b, 1); }
  __device__ __forceinline__ void add(int idx, float t) const {
    const float M = 12582912.0f;                // 1.5 * 2^23
    const float C = 206158430208.0f + M;        // M (1 + 2^14)
    const float th = t + M;                     // M + h
    const float tl = fmaf(t, 16384.0f, fmaf(-th, 16384.0f, C));  // M + l
    atomicAdd(hi + idx, __float_as_int(th));
    atomicAdd(lo + idx, __float_as_int(tl));
  }
  // value of word (plane c, position r in the plane) in 2^-30 units;
  // returns false when it is zero
  __device__ __forceinline__ bool value(int c, int r, int JW, int JP,
                                        long long &v) const {
    unsigned n = (unsigned)cnt[r];
    if (r >= 1 && c != 0) n += (unsigned)cnt[r - 1];
    if (r >= JW && c != 1) n += (unsigned)cnt[r - JW];
    if (r >= JW + 1 && c == 2) n += (unsigned)cnt[r - JW - 1];
    const int h = (int)((unsigned)hi[c * JP + r] - n * kBias);
    const int l = (int)((unsigned)lo[c * JP + r] - n * kBias);
    v = (long long)h * 16384 + l;
    return (h | l) != 0;
  }
  // adds the value of a word to the global fixed-point sum (exact: the sum
  // does not depend on the order in which tiles add)
  __device__ __forceinline__ static void fold(const SimDev<float> &S, int cur,
                                              int c, size_t o, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(S.Jq[cur][c] + o),
              (unsigned long long)v);
  }
  __device__ __forceinline__ void zero(int JP) const {
    for (int k = threadIdx.x; k < 3 * JP; k += blockDim.x) {
      hi[k] = 0;
      lo[k] = 0;
    }
    for (int k = threadIdx.x; k < JP; k += blockDim.x) cnt[k] = 0;
  }
};

template <>
struct TileJ<double> {
  double *v;
  // fixed: the words are int64 fixed-point sums (ZPIC_DETERMINISTIC), the
  // contributions arrive in units of 2^-47 Uq and are rounded to integers
  bool fixed;
  __device__ __forceinline__ void seg(int) const {}
  __device__ __forceinline__ void add(int idx, double t) const {
    if (fixed)
      atomicAdd(reinterpret_cast<unsigned long long *>(v + idx),
                (unsigned long long)__double2ll_rn(t));
    else
      atomicAdd(v + idx, t);
  }
  // the word as stored (a double, or the bits of an int64)
  __device__ __forceinline__ bool value(int c, int r, int, int JP,
                                        double &out) const {
    out = v[c * JP + r];
    return __double_as_longlong(out) != 0;
  }
  __device__ __forceinline__ static void fold(const SimDev<double> &S,
                                              int cur, int c, size_t o,
                                              double v) {
    if (S.jfixed)
      atomicAdd(reinterpret_cast<unsigned long long *>(S.J[cur][c] + o),
                (unsigned long long)__double_as_longlong(v));
    else
      atomicAdd(S.J[cur][c] + o, v);
  }
  __device__ __forceinline__ void zero(int JP) const {
    for (int k = threadIdx.x; k < 3 * JP; k += blockDim.x) v[k] = 0.0;
  }
};

// One straight segment inside tile cell (ci, cj), from (xa, ya) to (xb, yb)
// in that cell's offsets, covering fraction f of the step; qx, qy, qz are
// the particle's deposit factors.  Three planes of JP values, rows of JW,
// origin at cell (-1, -1).
template <typename R>
__device__ __forceinline__ void dep_seg(const TileJ<R> &J, int JW, int JP,
                                        int ci, int cj, R xa, R ya, R xb, R yb,
                                        R f, R qx, R qy, R qz) {
  const R ddx = xb - xa, ddy = yb - ya;
  const R xm = R(0.5) * (xa + xb), ym = R(0.5) * (ya + yb);
  const int b = (cj + 1) * JW + (ci + 1);
  const R ax = qx * ddx, ay = qy * ddy, az = qz * f;
  const R c = ddx * ddy * R(1.0 / 12.0);
  const R axy = ax * ym, ayx = ay * xm;
  J.seg(b);
  // charge flux through the x faces (i+1/2, j), (i+1/2, j+1)
  J.add(b, ax - axy);
  J.add(b + JW, axy);
  // through the y faces (i, j+1/2), (i+1, j+1/2)
  J.add(JP + b, ay - ayx);
  J.add(JP + b + 1, ayx);
  // q vz times the path-averaged bilinear weights of the four nodes
  const R w11 = xm * ym + c, w10 = xm - w11, w01 = ym - w11;
  J.add(2 * JP + b, az * (R(1) - xm - w01));
  J.add(2 * JP + b + 1, az * w10);
  J.add(2 * JP + b + JW, az * w01);
  J.add(2 * JP + b + JW + 1, az * w11);
}

// The path of a particle in its start cell's frame, from (x, y) to
// (x1, y1), split at the cell faces it crosses: cross iff the end lies at or
// beyond a face (axis_cross); sx, sy = path parameters where it meets the x
// face xb and the y face yb (1 when that axis is not crossed, at most 1
// otherwise: the fast division may round a quotient of numbers within an
// ulp of each other above 1).  The order of the crossings is decided only
// between axes that are crossed: a path that crosses one face is cut there
// even when it ends within rounding of it (s = 1), and when both are
// crossed an exact tie counts as x first.  s1 = the first crossing, s2 =
// the second (1 when there is none).  Segment 1 lies in the start cell,
// segment 2 in the cell entered at s1, segment 3 (two crossings) in the
// final cell; each is written in its own cell's frame and the last one ends
// at the stored offsets (xf, yf).  The same code serves the particle loop
// and the deferred segments, so both see the same rounding.
template <typename R>
struct PathSplit {
  int di, dj;     // cell steps
  R xf, yf;       // offsets in the final cell
  R xb, yb;       // crossed faces in the start cell's frame
  R sx, sy, s1, s2;
  R x_sx_y, x_sy;  // y where the path meets the x face, x where it meets y
  bool xfirst, cut, two;
};

template <typename R>
__device__ __forceinline__ PathSplit<R> split_path(R x, R y, R x1, R y1) {
  PathSplit<R> p;
  p.di = axis_cross(x1, p.xf);
  p.dj = axis_cross(y1, p.yf);
  p.xb = p.di > 0 ? R(1) : R(0);
  p.yb = p.dj > 0 ? R(1) : R(0);
  p.sx = p.di ? fmin(fdiv<R>(p.xb - x, x1 - x), R(1)) : R(1);
  p.sy = p.dj ? fmin(fdiv<R>(p.yb - y, y1 - y), R(1)) : R(1);
  p.xfirst = p.di != 0 && (p.dj == 0 || p.sx <= p.sy);
  p.s1 = p.xfirst ? p.sx : p.sy;
  p.s2 = p.xfirst ? p.sy : p.sx;
  p.x_sx_y = y + p.sx * (y1 - y);
  p.x_sy = x + p.sy * (x1 - x);
  p.cut = (p.di | p.dj) != 0;
  p.two = p.di != 0 && p.dj != 0;
  return p;
}

// Per-warp ring of particles whose path crosses a face: the segment in the
// start cell is deposited at once, the one or two segments beyond wait here
// and are deposited 32 particles at a time, one per lane, so that the few
// lanes that need them (a crossing is a few-percent event) do not hold up
// the warp.  Entries keep the raw path (start, end as computed, weight,
// z-deposit factor, start cell) and the split is recomputed when they are
// taken.  SoA, kQ entries; the ring is drained before the species changes.
constexpr int kQ = 64;
constexpr int kQVals = 6;

template <typename R>
struct SegQueue {
  R *v;       // kQVals planes of kQ values: x, y, x1, y1, w, qz
  int *cell;  // kQ packed start cells (lx + 1) | (ly + 1) << 8
};

template <typename R>
__device__ __forceinline__ void queue_put(const SegQueue<R> &q, int slot,
                                          int lx, int ly, R x, R y, R x1, R y1,
                                          R w, R qz) {
  q.v[0 * kQ + slot] = x;
  q.v[1 * kQ + slot] = y;
  q.v[2 * kQ + slot] = x1;
  q.v[3 * kQ + slot] = y1;
  q.v[4 * kQ + slot] = w;
  q.v[5 * kQ + slot] = qz;
  q.cell[slot] = (lx + 1) | ((ly + 1) << 8);
}

// kWhole: the start-cell segment was not deposited in the particle loop
// either (see kWholeQueue), so it is deposited here with the others.
template <typename R, bool kWhole>
__device__ __forceinline__ void queue_take(const SegQueue<R> &q,
                                           const TileJ<R> &J, int JW, int JP,
                                           int slot, R qx0, R qy0) {
  const int pc = q.cell[slot];
  const int lx = (pc & 255) - 1, ly = (pc >> 8) - 1;
  const R x = q.v[0 * kQ + slot], y = q.v[1 * kQ + slot];
  const R w = q.v[4 * kQ + slot], qz = q.v[5 * kQ + slot];
  const PathSplit<R> p =
      split_path(x, y, q.v[2 * kQ + slot], q.v[3 * kQ + slot]);
  const R qx = qx0 * w, qy = qy0 * w;
  if (kWhole)  // segment 1: from the start to the first crossing point
    dep_seg(J, JW, JP, lx, ly, x, y, p.xfirst ? p.xb : p.x_sy,
            p.xfirst ? p.x_sx_y : p.yb, p.s1, qx, qy, qz);
  // segment 2: from the first crossing point into the cell entered there
  const int c2x = p.xfirst ? p.di : 0, c2y = p.xfirst ? 0 : p.dj;
  const R ax2 = p.xfirst ? p.xb - R(p.di) : p.x_sy;
  const R ay2 = p.xfirst ? p.x_sx_y : p.yb - R(p.dj);
  const R bx2 = p.two ? (p.xfirst ? p.x_sy - R(p.di) : p.xb) : p.xf;
  const R by2 = p.two ? (p.xfirst ? p.yb : p.x_sx_y - R(p.dj)) : p.yf;
  dep_seg(J, JW, JP, lx + c2x, ly + c2y, ax2, ay2, bx2, by2, p.s2 - p.s1, qx,
          qy, qz);
  if (p.two) {
    // segment 3: from the second crossing point into the final cell
    const R ax3 = p.xfirst ? p.x_sy - R(p.di) : p.xb - R(p.di);
    const R ay3 = p.xfirst ? p.yb - R(p.dj) : p.x_sx_y - R(p.dj);
    dep_seg(J, JW, JP, lx + p.di, ly + p.dj, ax3, ay3, p.xf, p.yf,
            R(1) - p.s2, qx, qy, qz);
  }
}

// Field tile in coefficient form: for every cell (ci, cj) of a component's
// own (staggered) grid, the bilinear interpolant over that cell written as
// a + b wx + c wy + d wx wy, so a gather is one 16-byte shared load and
// three FMAs.  Grid of (TX + 1) x (TY + 1) cells with origin (-1, -1): a
// half-staggered axis may start one cell left of the particle's cell.
template <typename R>
struct alignas(16) Coef4 {
  R a, b, c, d;
};

template <typename R>
__device__ __forceinline__ R interp(const Coef4<R> *F, int idx, R wx, R wy) {
  const Coef4<R> k = F[idx];
  return fma(fma(k.d, wx, k.c), wy, fma(k.b, wx, k.a));
}

// ---- particle-copy ring: asynchronous 16-byte copies global -> shared ----
// Each warp streams its chunks of 32 particles through kStages stages of its
// own: while a chunk is computed, the copies of the next kStages - 1 chunks
// are in flight (cp.async, tracked per thread in commit groups), without
// holding registers.  A stage holds the chunk's planes back to back: cell
// (32 x 2 bytes), x, y, ux, uy, uz (32 x 4 bytes each), then w and id when
// the species stores them, i.e. 44 to 60 pieces of 16 bytes; lane l copies
// pieces l and l + 32.  FP32 only (FP64 loads directly).
template <typename R>
struct Ring {
  static constexpr int kStages = sizeof(R) == 4 ? 2 : 0;
  static constexpr unsigned kRB = 32 * sizeof(R);  // one real plane
  __host__ __device__ static constexpr unsigned stage_bytes(bool w, bool id) {
    return 64 + 5 * kRB + (w ? kRB : 0) + (id ? 128 : 0);
  }
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One lane's share of a stage: up to two 16-byte pieces.  For piece q the
// source is plane(q) + (p0 << shift(q)) + 16 (q - first piece of the plane),
// p0 being the chunk's first particle (a multiple of 32: segment offsets and
// capacities are multiples of 32, so all 32 slots lie inside the segment).
struct RingLane {
  const char *src[2];
  unsigned sh[2];
  unsigned dst[2];  // shared addresses relative to the stage
  int n;            // pieces of this lane (0..2)
};

template <typename R>
__device__ __forceinline__ RingLane ring_lane(const Planes<R> &I, int lane) {
  RingLane r;
  const int np = (int)Ring<R>::stage_bytes(I.w != nullptr, I.id != nullptr) / 16;
  r.n = 0;
  for (int k = 0; k < 2; ++k) {
    const int q = lane + 32 * k;
    r.src[k] = nullptr;
    r.sh[k] = 0;
    r.dst[k] = 16u * q;
    if (q >= np) continue;
    r.n = k + 1;
    if (q < 4) {
      r.src[k] = reinterpret_cast<const char *>(I.cell) + 16 * q;
      r.sh[k] = 1;
      continue;
    }
    const int pl = (q - 4) >> 3, o = (q - 4) & 7;
    const void *pp = pl == 0   ? (const void *)I.x
                     : pl == 1 ? (const void *)I.y
                     : pl == 2 ? (const void *)I.ux
                     : pl == 3 ? (const void *)I.uy
                     : pl == 4 ? (const void *)I.uz
                     : pl == 5 ? (I.w ? (const void *)I.w : (const void *)I.id)
                               : (const void *)I.id;
    r.src[k] = reinterpret_cast<const char *>(pp) + 16 * o;
    r.sh[k] = 2;
  }
  return r;
}

// A warp takes consecutive chunks: its lanes' sources start at the warp's
// first particle (ring_start) and advance by one chunk per copy.
__device__ __forceinline__ void ring_start(RingLane &r, int p0) {
  r.src[0] += (size_t)p0 << r.sh[0];
  r.src[1] += (size_t)p0 << r.sh[1];
}
__device__ __forceinline__ void ring_issue_next(RingLane &r, unsigned stg) {
  if (r.n > 0) cp_async16(stg + r.dst[0], r.src[0]);
  if (r.n > 1) cp_async16(stg + r.dst[1], r.src[1]);
  r.src[0] += 32u << r.sh[0];
  r.src[1] += 32u << r.sh[1];
}

template <typename R>
__device__ __forceinline__ void block_sum_store(double v, double *dst,
                                                double *red) {
  // deterministic tree: warp shuffle, then warp 0 over the warp sums
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < kPW ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *dst = v;
  }
}

// A particle that leaves its tile goes to the tile's outbox (global cell
// index), or, when the outbox is full, to the overflow buffer that the host
// drains by re-sorting.  Inlined: a call in the particle loop, even one
// that few lanes take, cost 3 % of the kernel's time (measured on the
// 2048^2 plasma: 8.94 against 9.22 ms per launch), and the loop still fits
// its 80 registers without spills.
template <typename R>
__device__ __forceinline__ void park_leaver(const SpeciesDev<R> &P,
                                         const OverflowDev<R> &ovf,
                                         BatchStatus *st, int tile, int slot,
                                         int sim, int s, int step, int nix,
                                         int niy, R xf, R yf, R ux, R uy, R uz,
                                         R w, int pid, bool has_w,
                                         bool has_id) {
  const int ob_cap = P.ob_cap;
  if (slot < ob_cap) {
    const size_t d = (size_t)tile * ob_cap + slot;
    P.ob_ix[d] = nix;
    P.ob_iy[d] = niy;
    P.ob_x[d] = xf;
    P.ob_y[d] = yf;
    P.ob_ux[d] = ux;
    P.ob_uy[d] = uy;
    P.ob_uz[d] = uz;
    if (has_w) P.ob_w[d] = w;
    if (has_id) P.ob_id[d] = pid;
    return;
  }
  const int o = atomicAdd(&st->ovf_count, 1);
  if (o < ovf.cap) {
    ovf.sim[o] = sim;
    ovf.species[o] = s;
    ovf.ix[o] = nix;
    ovf.iy[o] = niy;
    ovf.x[o] = xf;
    ovf.y[o] = yf;
    ovf.ux[o] = ux;
    ovf.uy[o] = uy;
    ovf.uz[o] = uz;
    ovf.w[o] = w;
    ovf.id[o] = pid;
    atomicOr(&st->error, ERR_OVERFLOW);
  } else {
    atomicAdd(&st->lost, 1);
    atomicOr(&st->error, ERR_LOST);
  }
  atomicMin(&st->err_step, step);
}

// After the species' particle loop: warp w kept s_stay[w] particles at the
// start of its range [r0_w, r1_w) of the output segment (the same slot split
// as the loop's), so the tile's kept particles are not yet contiguous.  The
// kept particles that lie at or beyond slot `kept` (their total) move, last
// ones first into the first gaps, into the gaps below `kept`; both lists
// are walked in slot order, so the result does not depend on timing.  Few
// particles leave a tile per step, so few move; they were written moments
// ago by this CTA and are read through L2.  Returns `kept`.
template <typename R>
__device__ __forceinline__ int close_gaps(const Planes<R> &O, int base, int n,
                                          int *sg, bool has_w, bool has_id) {
  // sg[0, kPW): particles kept per warp; sg[kPW, 5 kPW): per range, the
  // first gap slot, the gap slots below `kept`, the first kept particle at
  // or beyond `kept` and their number
  int *gap_lo = sg + kPW, *gap_n = sg + 2 * kPW;
  int *src_lo = sg + 3 * kPW, *src_n = sg + 4 * kPW;
  const int NC = (n + 31) >> 5;
  int kept = 0;
  for (int w = 0; w < kPW; ++w) kept += sg[w];
  if (threadIdx.x < kPW) {
    const int w = threadIdx.x;
    const int r0 = (w * NC / kPW) * 32;
    const int r1 = min(((w + 1) * NC / kPW) * 32, n);
    const int e = r0 + sg[w];
    gap_lo[w] = e;
    gap_n[w] = max(0, min(r1, kept) - e);
    src_lo[w] = max(r0, kept);
    src_n[w] = max(0, e - src_lo[w]);
  }
  __syncthreads();
  int m = 0;
  for (int w = 0; w < kPW; ++w) m += gap_n[w];
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    int kg = k, wg = 0;
    while (kg >= gap_n[wg]) kg -= gap_n[wg++];
    int ks = k, ws = 0;
    while (ks >= src_n[ws]) ks -= src_n[ws++];
    const size_t d = (size_t)base + gap_lo[wg] + kg;
    const size_t q = (size_t)base + src_lo[ws] + ks;
    O.cell[d] = __ldcg(O.cell + q);
    O.x[d] = __ldcg(O.x + q);
    O.y[d] = __ldcg(O.y + q);
    O.ux[d] = __ldcg(O.ux + q);
    O.uy[d] = __ldcg(O.uy + q);
    O.uz[d] = __ldcg(O.uz + q);
    if (has_w) O.w[d] = __ldcg(O.w + q);
    if (has_id) O.id[d] = __ldcg(O.id + q);
  }
  return kept;
}

// Shared-memory layout of the push kernel for tx x ty tiles (byte offsets):
// the coefficient tile (6 components x (tx+1)(ty+1) cells), the current
// tile (3 planes of (tx+3)(ty+3) values, 8 bytes each: two int32 words in
// FP32, one double in FP64), the FP32 segment counts (one int plane), the
// per-warp segment queues, which first serve as the staging area of the
// raw field values (6 planes of (tx+2)(ty+2)), and (FP32) the particle-copy
// ring: kStages stages per warp.
template <typename R>
struct PushSmem {
  size_t coef, j, cnt, q, ring, stages, total;
  __host__ __device__ PushSmem(int tx, int ty, bool wide) {
    const size_t CP = (size_t)(tx + 1) * (ty + 1);
    const size_t JP = (size_t)(tx + 3) * (ty + 3);
    coef = 0;
    j = 6 * CP * sizeof(Coef4<R>);
    cnt = j + 3 * JP * 8;
    const size_t cnt_bytes = sizeof(R) == 4 ? JP * sizeof(int) : 0;
    q = (cnt + cnt_bytes + 15) & ~size_t(15);
    const size_t qbytes =
        (size_t)kPW * kQ * (kQVals * sizeof(R) + sizeof(int));
    const size_t raw = 6 * (size_t)(tx + 2) * (ty + 2) * sizeof(R);
    ring = (q + (qbytes > raw ? qbytes : raw) + 15) & ~size_t(15);
    constexpr int S = Ring<R>::kStages;
    stages = ring;
    total = stages + (size_t)kPW * S * Ring<R>::stage_bytes(wide, wide);
  }
};

// State shared by the chunk loops of one CTA.
template <typename R>
struct TileCtx {
  const Coef4<R> *cf;  // coefficient tile, 6 planes of CP cells
  int CW, CP, JW, JP;
  TileJ<R> jt;
  SegQueue<R> q;
  unsigned char *stages;  // particle-copy ring
  int x0, y0, tw, th, nx, ny;
  int tile, sim, step, shift;
  int pc;  // current copy of the particle store
  R dt_dx, dt_dy;
  bool do_energy;
  int *s_slots;
  int *s_stay;  // particles each warp kept (kPW), then close_gaps scratch
  double *red;
};

// One species of one tile.  kSpec: the species' layout and the boundary are
// compile-time facts (kPlain: no weight or id planes; kOpen: open x boundary
// with a moving window possible); otherwise they are read at run time.
template <typename R, int CUR, bool kSpec, bool kPlain, bool kOpen>
__device__ __forceinline__ void push_species(const SimDev<R> &S, const int s,
                                             TileCtx<R> &T, unsigned &g,
                                             BatchStatus *st,
                                             const OverflowDev<R> &ovf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const SpeciesDev<R> &P = S.sp[s];
  const Planes<R> &I = P.buf[T.pc];
  const Planes<R> &O = P.buf[T.pc ^ 1];
  const bool has_w = kSpec ? !kPlain : I.w != nullptr;
  const bool has_id = kSpec ? !kPlain : I.id != nullptr;
  const bool open_x = kSpec ? kOpen : S.open_x != 0;
  const R hq = P.hq, qx0 = P.dq[0], qy0 = P.dq[1], q00 = P.dq[2];
  const int n = P.cnt[T.tile];
  if (n == 0) {
    // nothing to push: an empty outbox and (on energy steps) no kinetic
    // energy; the species of a tile with particles of other species only
    // (a cloud's tiles in a multi-species batch) cost no barrier
    if (threadIdx.x == 0) {
      P.ob_cnt[T.tile] = 0;
      if (T.do_energy) S.part_kin[(size_t)s * S.ntx * S.nty + T.tile] = 0.0;
    }
    return;
  }
  const int base = P.off[T.tile];
  const int tw = T.tw, th = T.th, CW = T.CW, CP = T.CP, JW = T.JW, JP = T.JP;
  const Coef4<R> *cEx = T.cf, *cEy = T.cf + CP, *cEz = T.cf + 2 * CP;
  const Coef4<R> *cBx = T.cf + 3 * CP, *cBy = T.cf + 4 * CP,
                 *cBz = T.cf + 5 * CP;
  if (threadIdx.x == 0) {
    T.s_slots[1] = 0;
    // report which compiled form pushes this species (read first: the bit
    // is set once, by the first tile that runs it)
    const int form = kSpec ? (kOpen ? ZPIC_PUSH_PLAIN_OPEN
                                    : ZPIC_PUSH_PLAIN_PERIODIC)
                           : ZPIC_PUSH_GENERIC;
    if (!(__ldcg(S.variants + s) & form)) atomicOr(S.variants + s, form);
  }
  __syncthreads();  // also: coefficient tile ready, J tile zeroed
  int n_removed = 0;
  int qhead = 0, qtail = 0;  // warp-uniform ring indices
  R kin = R(0);

  // warps work independently on chunks of 32 particles: no block barrier
  // inside the loop.  Warp `warp` owns the contiguous slots [r0, r1) (its
  // share of the tile's chunks) and writes the particles that stay in the
  // tile to the start of the same range of the other copy, in their input
  // order (no atomic, no wait on other warps); close_gaps then moves the
  // last particles of the tile into the gaps the leavers left.  A store in
  // which neighbouring slots hold neighbouring cells keeps that order from
  // step to step, and so do its bank-conflict-free gathers and deposits.
  constexpr int kS = Ring<R>::kStages;
  // FP64: the split of a crossing path (two divisions, a dozen compares)
  // and all its segments are left to the queue, which takes 32 crossing
  // paths at a time, so the particle loop spends no FP64 work on them (the
  // FP64 form is bound by the FP64 unit).  FP32 splits in the loop: it is
  // bound by issue and shared memory, and the queue would then deposit the
  // start-cell segment as extra atomics.
  constexpr bool kWholeQueue = sizeof(R) == 8;
  const int NC = (n + 31) >> 5;
  const int ca = warp * NC / kPW, cb = (warp + 1) * NC / kPW;
  const int nch = cb - ca;
  const int r0 = ca * 32;
  int n_stay = 0;  // particles this warp has kept (warp-uniform)
  const unsigned sbytes = Ring<R>::stage_bytes(has_w, has_id);
  const unsigned stg0 = smem_addr(T.stages) + warp * kS * sbytes;
  RingLane rl;
  if constexpr (kS > 0) {
    rl = ring_lane(I, lane);
    ring_start(rl, base + r0);
    // prologue: chunks 0 .. kS-2 (one commit group each, empty or not)
    for (int jc = 0; jc < kS - 1; ++jc) {
      if (jc < nch) ring_issue_next(rl, stg0 + ((g + jc) % kS) * sbytes);
      cp_async_commit();
    }
  }
  for (int jc = 0; jc < nch; ++jc, ++g) {
    const int c0 = r0 + jc * 32;
    // lanes past the end repeat the last particle with zero weight: they
    // run the same instructions, deposit nothing and store nothing
    const bool valid = c0 + lane < n;
    const int kk = valid ? lane : n - 1 - c0;  // slot within the chunk
    int lc;
    R x, y, ux, uy, uz, w = R(1);
    int pid = 0;
    if constexpr (kS > 0) {
      // the stage of chunk jc + kS - 1 was read in the previous iteration
      __syncwarp();
      if (jc + kS - 1 < nch)
        ring_issue_next(rl, stg0 + ((g + kS - 1) % kS) * sbytes);
      cp_async_commit();
      cp_async_wait<kS - 1>();  // this lane's pieces of chunk jc landed
      __syncwarp();             // ... and every other lane's
      const unsigned char *stg = T.stages + (warp * kS + g % kS) * sbytes;
      constexpr unsigned RB = Ring<R>::kRB;
      lc = reinterpret_cast<const uint16_t *>(stg)[kk];
      x = reinterpret_cast<const R *>(stg + 64)[kk];
      y = reinterpret_cast<const R *>(stg + 64 + RB)[kk];
      ux = reinterpret_cast<const R *>(stg + 64 + 2 * RB)[kk];
      uy = reinterpret_cast<const R *>(stg + 64 + 3 * RB)[kk];
      uz = reinterpret_cast<const R *>(stg + 64 + 4 * RB)[kk];
      unsigned o = 64 + 5 * RB;
      if (has_w && I.w) {
        w = reinterpret_cast<const R *>(stg + o)[kk];
        o += RB;
      }
      if (has_id && I.id) pid = reinterpret_cast<const int *>(stg + o)[kk];
    } else {
      const int p = base + c0 + kk;
      lc = __ldcs(I.cell + p);
      x = __ldcs(I.x + p);
      y = __ldcs(I.y + p);
      ux = __ldcs(I.ux + p);
      uy = __ldcs(I.uy + p);
      uz = __ldcs(I.uz + p);
      if (has_w && I.w) w = __ldcs(I.w + p);
      if (has_id && I.id) pid = __ldcs(I.id + p);
    }
    const R wd = valid ? w : R(0);
    int lx = lc & 255, ly = lc >> 8;
    // never produced by the library's own kernels: record it and keep
    // the shared-memory accesses inside the tile (a warp-uniform test,
    // then the rare lanes)
    const bool bad = lx >= tw || ly >= th;
    if (__any_sync(0xffffffffu, bad)) {
      if (bad) {
        atomicOr(&st->error, ERR_STORE);
        atomicMin(&st->err_step, T.step);
      }
      lx = min(lx, tw - 1);
      ly = min(ly, th - 1);
    }

    // ---- stage 1: bilinear gather on the staggered grid ----
    // node-centred axis: cell l, weight o; half-staggered axis: cell l-1
    // with weight o+1/2 if o < 1/2, else cell l with weight o-1/2
    const bool xl = x < R(0.5), yl = y < R(0.5);
    const R whx = xl ? x + R(0.5) : x - R(0.5);
    const R why = yl ? y + R(0.5) : y - R(0.5);
    const int i_nn = (ly + 1) * CW + (lx + 1);
    const int i_hn = i_nn - (xl ? 1 : 0);
    const int i_nh = i_nn - (yl ? CW : 0);
    const int i_hh = i_hn - (yl ? CW : 0);
    const R ex = interp(cEx, i_hn, whx, y);
    const R ey = interp(cEy, i_nh, x, why);
    const R ez = interp(cEz, i_nn, x, y);
    const R bx = interp(cBx, i_nh, x, why);
    const R by = interp(cBy, i_hn, whx, y);
    const R bz = interp(cBz, i_hh, whx, why);

    // ---- stage 2: relativistic Boris ----
    const R umx = ux + hq * ex, umy = uy + hq * ey, umz = uz + hq * ez;
    const R rg = rsqrt_r<R>(R(1) + umx * umx + umy * umy + umz * umz);
    const R tx = hq * bx * rg, ty = hq * by * rg, tz = hq * bz * rg;
    const R sf = fdiv<R>(R(2), R(1) + tx * tx + ty * ty + tz * tz);
    const R upx = umx + (umy * tz - umz * ty);
    const R upy = umy + (umz * tx - umx * tz);
    const R upz = umz + (umx * ty - umy * tx);
    ux = umx + sf * (upy * tz - upz * ty) + hq * ex;
    uy = umy + sf * (upz * tx - upx * tz) + hq * ey;
    uz = umz + sf * (upx * ty - upy * tx) + hq * ez;

    // ---- stage 2b: move (at most one cell, CFL) ----
    const R u2 = ux * ux + uy * uy + uz * uz;
    const R rgn = rsqrt_r<R>(R(1) + u2);
    if (T.do_energy) kin += wd * u2 * fdiv<R>(rgn, R(1) + rgn);
    const R x1 = x + T.dt_dx * ux * rgn;
    const R y1 = y + T.dt_dy * uy * rgn;
    PathSplit<R> ps;
    if constexpr (kWholeQueue) {
      // the cell steps and stored offsets only; the split of a crossing
      // path waits for the queue
      R xe = x1, ye = y1;
      ps.di = axis_cross(xe, ps.xf);
      ps.dj = axis_cross(ye, ps.yf);
      ps.cut = (ps.di | ps.dj) != 0;
    } else {
      ps = split_path(x, y, x1, y1);
    }

    // ---- stage 3: charge-conserving deposit, segment in the start cell ----
    const R qz = q00 * wd * uz * rgn;
    if constexpr (kWholeQueue) {
      if (!ps.cut)  // a path inside its cell
        dep_seg(T.jt, JW, JP, lx, ly, x, y, ps.xf, ps.yf, R(1), qx0 * wd,
                qy0 * wd, qz);
    } else {
      const R bx1 = ps.cut ? (ps.xfirst ? ps.xb : ps.x_sy) : ps.xf;
      const R by1 = ps.cut ? (ps.xfirst ? ps.x_sx_y : ps.yb) : ps.yf;
      dep_seg(T.jt, JW, JP, lx, ly, x, y, bx1, by1, ps.s1, qx0 * wd,
              qy0 * wd, qz);
    }
    // the rest of a crossing path waits in the warp's queue
    const bool need = valid && ps.cut;
    const unsigned mq = __ballot_sync(0xffffffffu, need);
    if (mq) {
      if (need)
        queue_put(T.q, (qtail + __popc(mq & lt)) & (kQ - 1), lx, ly, x, y, x1,
                  y1, wd, qz);
      qtail += __popc(mq);
      // the ring holds kQ = 64: before each put at most 31 entries wait,
      // a put adds at most 32, and a full run of 32 is drained at once
      __syncwarp();
      if (qtail - qhead >= 32) {
        queue_take<R, kWholeQueue>(T.q, T.jt, JW, JP,
                                   (qhead + lane) & (kQ - 1), qx0, qy0);
        qhead += 32;
        __syncwarp();
      }
    }

    // ---- new cell: window shift, boundaries, tile membership ----
    int nix, niy, nlx, nly;
    bool removed = false, inside;
    // in the tile's own coordinates first; the global cell, the
    // boundaries and the periodic wrap only for particles that leave the
    // tile's cells (a wrap may bring one back into a tile that spans the
    // box)
    nlx = lx + ps.di - T.shift;
    nly = ly + ps.dj;
    nix = T.x0 + nlx;
    niy = T.y0 + nly;
    if (open_x)  // leaves the window it moved in, or the shifted window
      removed = nix + T.shift >= T.nx || nix < 0;
    inside = !removed && (unsigned)nlx < (unsigned)tw &&
             (unsigned)nly < (unsigned)th;
    if (!inside && !removed) {
      niy = wrap1(niy, T.ny);
      if (!open_x) nix = wrap1(nix, T.nx);
      nlx = nix - T.x0;
      nly = niy - T.y0;
      inside = (unsigned)nlx < (unsigned)tw && (unsigned)nly < (unsigned)th;
    }
    const bool stay = valid && !removed && inside;
    const bool leave = valid && !removed && !inside;
    if (valid && removed) ++n_removed;

    // ---- output: stayers to this warp's range of the other copy, in input
    // order; leavers (global cell) to the tile's outbox ----
    const unsigned bs = __ballot_sync(0xffffffffu, stay);
    const unsigned bl = __ballot_sync(0xffffffffu, leave);
    int lb = 0;
    if (bl) {  // warp-uniform
      if (lane == 0) lb = atomicAdd(&T.s_slots[1], __popc(bl));
      lb = __shfl_sync(0xffffffffu, lb, 0);
    }
    if (stay) {
      const int d = base + r0 + n_stay + __popc(bs & lt);
      __stcs(O.cell + d, local_cell(nlx, nly));
      __stcs(O.x + d, ps.xf);
      __stcs(O.y + d, ps.yf);
      __stcs(O.ux + d, ux);
      __stcs(O.uy + d, uy);
      __stcs(O.uz + d, uz);
      if (has_w && O.w) __stcs(O.w + d, w);
      if (has_id && O.id) __stcs(O.id + d, pid);
    } else if (leave) {
      park_leaver(P, ovf, st, T.tile, lb + __popc(bl & lt), T.sim, s, T.step,
                  nix, niy, ps.xf, ps.yf, ux, uy, uz, w, pid,
                  has_w && O.w != nullptr, has_id && O.id != nullptr);
    }
    n_stay += __popc(bs);
  }
  // segments still waiting in the warp's queue
  __syncwarp();
  if (lane < qtail - qhead)
    queue_take<R, kWholeQueue>(T.q, T.jt, JW, JP,
                               (qhead + lane) & (kQ - 1), qx0, qy0);
  if (lane == 0) T.s_stay[warp] = n_stay;
  if (n_removed) atomicAdd(&S.removed[s], n_removed);
  if (T.do_energy)
    block_sum_store<R>((double)kin,
                       &S.part_kin[(size_t)s * S.ntx * S.nty + T.tile], T.red);
  __syncthreads();  // every warp's stayers written, s_stay complete
  const int kept = close_gaps(O, base, n, T.s_stay, has_w && O.w != nullptr,
                              has_id && O.id != nullptr);
  if (threadIdx.x == 0) {
    P.cnt[T.tile] = kept;
    P.ob_cnt[T.tile] = min(T.s_slots[1], P.ob_cap);
    if (T.s_slots[1] > P.ob_cap) atomicMax(&S.ob_need[s], T.s_slots[1]);
  }
}

// The work of one CTA on one tile; CUR = step & 1 selects the field and
// particle copies, as a compile-time value so that every descriptor access
// has a constant offset.  kSpec: the 16 x 16 FP32 kernels (one simulation
// or a batch), whose species loops are also specialised on layout and
// boundary.
template <typename R, bool kBatch, int TXC, int TYC, int CUR>
__device__ __forceinline__ void push_tile(const SimDev<R> &S, const int sim,
                                          const int tile, const int step,
                                          BatchStatus *st,
                                          const OverflowDev<R> &ovf,
                                          unsigned char *smem_raw,
                                          int *s_slots, int *s_stay,
                                          double *red) {
  constexpr bool kSpec = sizeof(R) == 4 && TXC == 16 && TYC == 16;
  const int nx = S.nx, ny = S.ny, ld = S.ld;
  const int TX = TXC > 0 ? TXC : S.tx, TY = TYC > 0 ? TYC : S.ty;
  const int open_x = S.open_x, nsp = S.nsp;
  const int tcx = tile % S.ntx, tcy = tile / S.ntx;
  const int x0 = tcx * TX, y0 = tcy * TY;

  TileCtx<R> T;
  T.CW = TX + 1;
  T.CP = T.CW * (TY + 1);
  T.JW = TX + 3;
  T.JP = T.JW * (TY + 3);
  const int FW = TX + 2, FP = FW * (TY + 2);
  const int CW = T.CW, CP = T.CP, JW = T.JW, JP = T.JP;
  const PushSmem<R> L(TX, TY, false);  // offsets up to the ring
  Coef4<R> *cf = reinterpret_cast<Coef4<R> *>(smem_raw + L.coef);
  T.cf = cf;
  if constexpr (sizeof(R) == 4) {
    T.jt.hi = reinterpret_cast<int *>(smem_raw + L.j);
    T.jt.lo = T.jt.hi + 3 * JP;
    T.jt.cnt = reinterpret_cast<int *>(smem_raw + L.cnt);
  } else {
    T.jt.v = reinterpret_cast<double *>(smem_raw + L.j);
    T.jt.fixed = S.jfixed != 0;
  }
  const int warp = threadIdx.x >> 5;
  T.q.v = reinterpret_cast<R *>(smem_raw + L.q) + warp * kQVals * kQ;
  T.q.cell = reinterpret_cast<int *>(smem_raw + L.q +
                                     sizeof(R) * kQVals * kQ * kPW) +
             warp * kQ;
  T.stages = smem_raw + L.stages;
  T.x0 = x0;
  T.y0 = y0;
  T.tw = min(TX, nx - x0);
  T.th = min(TY, ny - y0);
  T.nx = nx;
  T.ny = ny;
  T.tile = tile;
  T.sim = sim;
  T.step = step;
  T.pc = CUR ^ *S.pswap;
  T.dt_dx = S.dt_dx;
  T.dt_dy = S.dt_dy;
  T.s_slots = s_slots;
  T.s_stay = s_stay;
  T.red = red;

  // ---- stage 0: fields of the tile + one guard cell, coefficient form ----
  // one cell per thread and pass, the six components inner (index
  // arithmetic and boundary handling shared by the six loads)
  R *raw = reinterpret_cast<R *>(smem_raw + L.q);
  for (int r = threadIdx.x; r < FP; r += blockDim.x) {
    const int lj = r / FW, li = r - lj * FW;
    int gi = x0 - 1 + li;
    const int gj = wrap1(y0 - 1 + lj, ny);
    bool in = true;
    if (open_x)
      in = gi >= 0 && gi < nx;
    else
      gi = wrap1(gi, nx);
    const size_t o = (size_t)gj * ld + (in ? gi : 0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const R *src = c < 3 ? S.E[CUR][c] : S.B[CUR][c - 3];
      raw[c * FP + r] = in ? src[o] : R(0);
    }
  }
  T.jt.zero(JP);
  __syncthreads();
  for (int r = threadIdx.x; r < CP; r += blockDim.x) {
    const int cj = r / CW, ci = r - cj * CW;
    const int b = cj * FW + ci;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const R *f = raw + c * FP + b;
      const R f00 = f[0], f10 = f[1], f01 = f[FW], f11 = f[FW + 1];
      Coef4<R> v;
      v.a = f00;
      v.b = f10 - f00;
      v.c = f01 - f00;
      v.d = (f11 - f10) - v.c;
      cf[c * CP + r] = v;
    }
  }
  // (the species loop's barrier separates these reads of the staging area
  // from the queue writes)
  const int nsh = S.moving_window ? *S.n_shift : 0;
  T.shift = shift_due(S, step, nsh) ? 1 : 0;
  T.do_energy = S.energy_every > 0 && ((step + 1) % S.energy_every) == 0;

  unsigned g = 0;  // chunks this warp has taken through the particle ring
  for (int s = 0; s < nsp; ++s) {
    if constexpr (kSpec) {
      const Planes<R> &I = S.sp[s].buf[T.pc];
      const bool plain = I.w == nullptr && I.id == nullptr;
      if (plain && open_x)
        push_species<R, CUR, true, true, true>(S, s, T, g, st, ovf);
      else if (plain)
        push_species<R, CUR, true, true, false>(S, s, T, g, st, ovf);
      else
        push_species<R, CUR, false, false, false>(S, s, T, g, st, ovf);
    } else {
      push_species<R, CUR, false, false, false>(S, s, T, g, st, ovf);
    }
  }
  __syncthreads();

  // ---- stage 3b: fold the tile's current (with guards) into global J ----
  for (int r = threadIdx.x; r < JP; r += blockDim.x) {
    const int lj = r / JW, li = r - lj * JW;
    int gi = x0 - 1 + li;
    const int gj = wrap1(y0 - 1 + lj, ny);
    if (open_x) {
      if (gi < 0 || gi >= nx) continue;
    } else {
      gi = wrap1(gi, nx);
    }
    const size_t o = (size_t)gj * ld + gi;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      typename std::conditional<sizeof(R) == 4, long long, double>::type v;
      if (T.jt.value(c, r, JW, JP, v)) TileJ<R>::fold(S, CUR, c, o, v);
    }
  }
}

// kBatch = false: one simulation, its descriptor passed as a grid-constant
// kernel parameter; kBatch = true: descriptors of many simulations read from
// device memory.  TXC, TYC > 0: tile size fixed at compile time (shared-
// memory offsets become immediates); 0: taken from the descriptor.
template <typename R, bool kBatch, int TXC, int TYC>
__global__ void __launch_bounds__(
    kPT, sizeof(R) == 4 ? (kBatch ? kPushCtasF32Batch : kPushCtasF32) : 2)
    push_deposit_kernel(const SimDev<R> *__restrict__ sims,
                        const __grid_constant__ SimDev<R> one,
                        const int2 *__restrict__ items, int n_items,
                        BatchStatus *st,
                        const __grid_constant__ OverflowDev<R> ovf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slots[2];  // [1]: leavers written to the outbox
  __shared__ int s_stay[5 * kPW];
  __shared__ double red[kPW];
  __shared__ int s_item;
  // the batch member's descriptor (unused by the one-simulation kernel,
  // which reads its descriptor from the kernel parameters)
  __shared__ SimDev<R> s_desc;
  static_assert(sizeof(SimDev<R>) % 8 == 0, "descriptor copied in 8-byte words");

  const int step = st->step;
  if (frozen(st, step)) return;
  // persistent: as many CTAs as fit on the GPU take the work items (tiles,
  // longest first) from a counter that the end-of-step kernel resets
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&st->push_next, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= n_items) return;
    const int2 it = items[item];
    if constexpr (kBatch && kBatchDescInSmem) {
      // the member's descriptor in shared memory: cheap to reload, so the
      // particle loop need not hold its pointers in registers
      const long long *src = reinterpret_cast<const long long *>(sims + it.x);
      long long *dst = reinterpret_cast<long long *>(&s_desc);
      for (int k = threadIdx.x; k < (int)(sizeof(SimDev<R>) / 8);
           k += blockDim.x)
        dst[k] = src[k];
      __syncthreads();
    }
    const SimDev<R> &S =
        kBatch ? (kBatchDescInSmem ? s_desc : sims[it.x]) : one;
    // a tile without particles deposits nothing and loses nothing: it only
    // reports empty outboxes (and zero kinetic energy on energy steps)
    int n_all = 0;
    for (int s = 0; s < S.nsp; ++s) n_all += S.sp[s].cnt[it.y];
    if (n_all == 0) {
      if (threadIdx.x < S.nsp) {
        S.sp[threadIdx.x].ob_cnt[it.y] = 0;
        if (S.energy_every > 0 && ((step + 1) % S.energy_every) == 0)
          S.part_kin[(size_t)threadIdx.x * S.ntx * S.nty + it.y] = 0.0;
      }
      continue;
    }
    if (step & 1)
      push_tile<R, kBatch, TXC, TYC, 1>(S, it.x, it.y, step, st, ovf,
                                        smem_raw, s_slots, s_stay, red);
    else
      push_tile<R, kBatch, TXC, TYC, 0>(S, it.x, it.y, step, st, ovf,
                                        smem_raw, s_slots, s_stay, red);
    __syncthreads();  // shared memory is reused by the next item
  }
}

template <typename R>
size_t push_smem_bytes(int tx, int ty, bool wide) {
  return PushSmem<R>(tx, ty, wide).total;
}

template <typename R, bool kBatch>
static cudaError_t set_push_smem(int smem) {
  cudaError_t e = cudaFuncSetAttribute(push_deposit_kernel<R, kBatch, 16, 16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(push_deposit_kernel<R, kBatch, 0, 0>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <typename R>
cudaError_t prepare_push_deposit(int max_tx, int max_ty, bool wide) {
  const int smem = (int)push_smem_bytes<R>(max_tx, max_ty, wide);
  cudaError_t e = set_push_smem<R, false>(smem);
  if (e != cudaSuccess) return e;
  return set_push_smem<R, true>(smem);
}

// Resident CTAs of kernel k per SM for `smem` bytes of dynamic shared
// memory, times the SM count: the grid of the persistent push kernel.
// ctas_per_sm > 0 caps the resident CTAs per SM (the tiles in flight per
// SM, which the autotuner chooses); 0 takes all that fit.
template <typename K>
static int persistent_grid(K kernel, size_t smem, int n_items,
                           int ctas_per_sm) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPT,
                                                    smem) != cudaSuccess ||
      per_sm < 1)
    return n_items;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  return n_items < sms * per_sm ? n_items : sms * per_sm;
}

template <typename R>
int push_ctas_fit(int tx, int ty, bool wide) {
  int per_sm = 0;
  const size_t smem = push_smem_bytes<R>(tx, ty, wide);
  if (prepare_push_deposit<R>(tx, ty, wide) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, push_deposit_kernel<R, false, 0, 0>, kPT, smem) !=
      cudaSuccess)
    return 0;
  return per_sm;
}
template int push_ctas_fit<float>(int, int, bool);
template int push_ctas_fit<double>(int, int, bool);

template <typename R>
cudaError_t launch_push_deposit(const SimDev<R> *sims, const SimDev<R> *single,
                                const int2 *items, int n_items, int max_tx,
                                int max_ty, bool all16, bool wide,
                                int ctas_per_sm, BatchStatus *st,
                                const OverflowDev<R> &ovf,
                                cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = push_smem_bytes<R>(max_tx, max_ty, wide);
  // the 16 x 16 kernel needs every simulation of the batch to use 16 x 16
  // tiles (ragged edge tiles are fine)
  const bool t16 = all16;
  if (single) {
    if (t16) {
      auto k = push_deposit_kernel<R, false, 16, 16>;
      k<<<persistent_grid(k, smem, n_items, ctas_per_sm), kPT, smem, stream>>>(
          sims, *single, items, n_items, st, ovf);
    } else {
      auto k = push_deposit_kernel<R, false, 0, 0>;
      k<<<persistent_grid(k, smem, n_items, ctas_per_sm), kPT, smem, stream>>>(
          sims, *single, items, n_items, st, ovf);
    }
  } else {
    if (t16) {
      auto k = push_deposit_kernel<R, true, 16, 16>;
      k<<<persistent_grid(k, smem, n_items, ctas_per_sm), kPT, smem, stream>>>(
          sims, SimDev<R>{}, items, n_items, st, ovf);
    } else {
      auto k = push_deposit_kernel<R, true, 0, 0>;
      k<<<persistent_grid(k, smem, n_items, ctas_per_sm), kPT, smem, stream>>>(
          sims, SimDev<R>{}, items, n_items, st, ovf);
    }
  }
  return cudaGetLastError();
}

template size_t push_smem_bytes<float>(int, int, bool);
template size_t push_smem_bytes<double>(int, int, bool);
template cudaError_t prepare_push_deposit<float>(int, int, bool);
template cudaError_t prepare_push_deposit<double>(int, int, bool);
template cudaError_t launch_push_deposit<float>(const SimDev<float> *,
                                                const SimDev<float> *,
                                                const int2 *, int, int, int,
                                                bool, bool, int, BatchStatus *,
                                                const OverflowDev<float> &,
                                                cudaStream_t);
template cudaError_t launch_push_deposit<double>(const SimDev<double> *,
                                                 const SimDev<double> *,
                                                 const int2 *, int, int, int,
                                                 bool, bool, int,
                                                 BatchStatus *,
                                                 const OverflowDev<double> &,
                                                 cudaStream_t);

}  // namespace zp
