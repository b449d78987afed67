// k_push.cu -- fused particle kernel: interpolation, Boris push, move,
// charge-conserving deposition and in-tile compaction (PIC stages 1-3 of
// Sec. 2.2; the per-region particle advance with local current buffers and
// a ghost-cell reduction of Sec. 3.2, here one CTA per tile).
//
// Per work item (simulation, tile) one CTA:
//  1. stages E, B of the tile plus one guard cell on each side in shared
//     memory ([-1, tx] x [-1, ty]) and zeroes a shared J tile covering
//     [-1, tx+1] x [-1, ty+1];
//  2. streams the tile's particles in chunks of 32 per warp: bilinear
//     gather of the staggered fields from shared memory, relativistic Boris
//     rotation, move by dt u/gamma (at most one cell, CFL), split of the
//     straight path at the cell faces it crosses; the segment in the start
//     cell goes straight into the shared J tile, the segments of particles
//     that cross a face wait in a per-warp queue and are deposited 32 at a
//     time;
//  3. writes particles that stay in the tile to the tile's segment of the
//     other copy of the store (each warp claims a run of slots with one
//     shared-memory atomic, so warps never wait for each other) and
//     particles that leave to the tile's outbox; particles leaving an open
//     boundary are dropped;
//  4. adds the shared J tile (interior and guard cells) to the global J
//     with one reduction per cell (periodic images folded here).
// Traffic per particle: one read and one write of its SoA record (16-bit
// cell within the tile + 5 reals: 22 bytes in FP32).
#include "zpic_dev.cuh"
#include "zpic_kernels.h"

namespace zp {

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
// into hi = round(t) and lo = round((t - hi) 2^14) in [-2^13, 2^13], so the
// value is hi 2^14 + lo in units of 2^-30.  The rounding uses the float
// "add 1.5 2^23" trick (exact for |t| < 2^22) instead of conversion
// instructions.  Integer shared atomics are native (float ones are not) and
// integer sums do not depend on the order of the adds.  Exact while one word
// receives fewer than 2^18 adds per step and the net sum stays below 2^15
// units.  FP64: plain double atomics.
template <typename R>
struct TileJ;

template <>
struct TileJ<float> {
  int *hi;
  int *lo;
  __device__ __forceinline__ void add(int idx, float t) const {
    const float M = 12582912.0f;  // 1.5 * 2^23
    const float th = t + M;
    const int h = __float_as_int(th) - 0x4B400000;
    const float rem = t - (th - M);
    const int l = __float_as_int(fmaf(rem, 16384.0f, M)) - 0x4B400000;
    atomicAdd(hi + idx, h);
    atomicAdd(lo + idx, l);
  }
  __device__ __forceinline__ bool nonzero(int idx) const {
    return (hi[idx] | lo[idx]) != 0;
  }
  __device__ __forceinline__ double value(int idx) const {
    return (double)hi[idx] * 16384.0 + (double)lo[idx];
  }
  __device__ __forceinline__ void zero(int n) const {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      hi[k] = 0;
      lo[k] = 0;
    }
  }
};

template <>
struct TileJ<double> {
  double *v;
  __device__ __forceinline__ void add(int idx, double t) const {
    atomicAdd(v + idx, t);
  }
  __device__ __forceinline__ bool nonzero(int idx) const { return v[idx] != 0.0; }
  __device__ __forceinline__ double value(int idx) const { return v[idx]; }
  __device__ __forceinline__ void zero(int n) const {
    for (int k = threadIdx.x; k < n; k += blockDim.x) v[k] = 0.0;
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

// Per-warp ring of deferred segments: a segment outside the particle's
// start cell exists only for particles that cross a face (a few percent),
// but a warp would run the whole deposit whenever any one of its 32 lanes
// needs it.  Such segments are parked here instead and deposited 32 at a
// time, one per lane.  SoA, kQ entries: offsets, fraction, deposit factors
// and the packed tile cell (ci + 1) | (cj + 1) << 8.
constexpr int kQ = 64;

template <typename R>
struct SegQueue {
  R *v;       // 8 planes of kQ values: xa, ya, xb, yb, f, qx, qy, qz
  int *cell;  // kQ packed cells
};

template <typename R>
__device__ __forceinline__ void queue_put(const SegQueue<R> &q, int slot,
                                          int ci, int cj, R xa, R ya, R xb,
                                          R yb, R f, R qx, R qy, R qz) {
  q.v[0 * kQ + slot] = xa;
  q.v[1 * kQ + slot] = ya;
  q.v[2 * kQ + slot] = xb;
  q.v[3 * kQ + slot] = yb;
  q.v[4 * kQ + slot] = f;
  q.v[5 * kQ + slot] = qx;
  q.v[6 * kQ + slot] = qy;
  q.v[7 * kQ + slot] = qz;
  q.cell[slot] = (ci + 1) | ((cj + 1) << 8);
}

template <typename R>
__device__ __forceinline__ void queue_take(const SegQueue<R> &q,
                                           const TileJ<R> &J, int JW, int JP,
                                           int slot) {
  const int pc = q.cell[slot];
  dep_seg(J, JW, JP, (pc & 255) - 1, (pc >> 8) - 1, q.v[0 * kQ + slot],
          q.v[1 * kQ + slot], q.v[2 * kQ + slot], q.v[3 * kQ + slot],
          q.v[4 * kQ + slot], q.v[5 * kQ + slot], q.v[6 * kQ + slot],
          q.v[7 * kQ + slot]);
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
    v = lane < kWarps ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *dst = v;
  }
}

// kBatch = false: one simulation, its descriptor passed as a grid-constant
// kernel parameter; kBatch = true: descriptors of many simulations read from
// device memory.  TXC, TYC > 0: tile size fixed at compile time (shared-
// memory offsets become immediates); 0: taken from the descriptor.
template <typename R, bool kBatch, int TXC, int TYC>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 4 : 2)
    push_deposit_kernel(const SimDev<R> *__restrict__ sims,
                        const __grid_constant__ SimDev<R> one,
                        const int2 *__restrict__ items, BatchStatus *st,
                        OverflowDev<R> ovf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slots[2];  // stayers written, leavers written
  __shared__ double red[kWarps];

  const int step = st->step;
  if (frozen(st, step)) return;
  const int2 it = items[blockIdx.x];
  const SimDev<R> &S = kBatch ? sims[it.x] : one;
  const int tile = it.y;
  const int nx = S.nx, ny = S.ny, ld = S.ld;
  const int TX = TXC > 0 ? TXC : S.tx, TY = TYC > 0 ? TYC : S.ty;
  const int open_x = S.open_x, nsp = S.nsp;
  const R dt_dx = S.dt_dx, dt_dy = S.dt_dy;
  const int tcx = tile % S.ntx, tcy = tile / S.ntx;
  const int x0 = tcx * TX, y0 = tcy * TY;
  const int tw = min(TX, nx - x0), th = min(TY, ny - y0);
  const int cur = step & 1;

  // shared layout: 6 field planes (FW x FH) then 3 current planes (JW x JH)
  const int FW = TX + 2, FH = TY + 2, FP = FW * FH;
  const int JW = TX + 3, JH = TY + 3, JP = JW * JH;
  R *fs = reinterpret_cast<R *>(smem_raw);
  TileJ<R> jt;
  if constexpr (sizeof(R) == 4) {
    jt.hi = reinterpret_cast<int *>(fs + 6 * FP);
    jt.lo = jt.hi + 3 * JP;
  } else {
    jt.v = reinterpret_cast<double *>(fs + 6 * FP);
  }
  SegQueue<R> q;
  {
    // queues after the current planes (8 bytes per value), 16-byte aligned
    const size_t qoff =
        ((sizeof(R) * 6 * FP + 8 * 3 * (size_t)JP) + 15) & ~size_t(15);
    unsigned char *qb = smem_raw + qoff;
    const int wq = threadIdx.x >> 5;
    q.v = reinterpret_cast<R *>(qb) + wq * 8 * kQ;
    q.cell = reinterpret_cast<int *>(qb + sizeof(R) * 8 * kQ * kWarps) +
             wq * kQ;
  }

  for (int k = threadIdx.x; k < 6 * FP; k += blockDim.x) {
    const int c = k / FP, r = k - c * FP;
    const int lj = r / FW, li = r - lj * FW;
    const R *src = c < 3 ? S.E[cur][c] : S.B[cur][c - 3];
    int gi = x0 - 1 + li;
    const int gj = wrap1(y0 - 1 + lj, ny);
    R v = R(0);
    if (open_x) {
      if (gi >= 0 && gi < nx) v = src[(size_t)gj * ld + gi];
    } else {
      gi = wrap1(gi, nx);
      v = src[(size_t)gj * ld + gi];
    }
    fs[k] = v;
  }
  jt.zero(3 * JP);
  const int nsh = S.moving_window ? *S.n_shift : 0;
  const int shift = shift_due(S, step, nsh) ? 1 : 0;
  const bool do_energy =
      S.energy_every > 0 && ((step + 1) % S.energy_every) == 0;

  const R *Ex = fs, *Ey = fs + FP, *Ez = fs + 2 * FP;
  const R *Bx = fs + 3 * FP, *By = fs + 4 * FP, *Bz = fs + 5 * FP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;

  for (int s = 0; s < nsp; ++s) {
    const SpeciesDev<R> &P = S.sp[s];
    const Planes<R> &I = P.buf[cur];
    const Planes<R> &O = P.buf[cur ^ 1];
    const R hq = P.hq, qx0 = P.dq[0], qy0 = P.dq[1], q00 = P.dq[2];
    const int n = P.cnt[tile];
    const int base = P.off[tile];
    const int ob_cap = P.ob_cap;
    if (threadIdx.x == 0) {
      s_slots[0] = 0;
      s_slots[1] = 0;
    }
    __syncthreads();  // also: fields staged, J tile zeroed
    int n_removed = 0;
    int qhead = 0, qtail = 0;  // warp-uniform ring indices
    R kin = R(0);
    // warps work independently on chunks of 32 particles: no block barrier
    // inside the loop; each warp claims its output slots with one atomic
    for (int c0 = warp * 32; c0 < n; c0 += blockDim.x) {
      const int k = c0 + lane;
      const bool valid = k < n;
      // invalid lanes carry a particle at rest in the tile's first cell and
      // never deposit or store
      int lc = 0, pid = 0;
      R x = R(0.5), y = R(0.5), ux = R(0), uy = R(0), uz = R(0), w = R(1);
      if (valid) {
        const int p = base + k;
        lc = __ldcs(I.cell + p);
        x = __ldcs(I.x + p);
        y = __ldcs(I.y + p);
        ux = __ldcs(I.ux + p);
        uy = __ldcs(I.uy + p);
        uz = __ldcs(I.uz + p);
        if (I.w) w = __ldcs(I.w + p);
        if (I.id) pid = __ldcs(I.id + p);
      }
      int lx = lc & 255, ly = lc >> 8;
      if (lx >= tw || ly >= th) {
        // never produced by the library's own kernels: record it and keep
        // the shared-memory accesses inside the tile
        atomicOr(&st->error, ERR_STORE);
        atomicMin(&st->err_step, step);
        lx = min(lx, tw - 1);
        ly = min(ly, th - 1);
      }

      // ---- stage 1: bilinear gather on the staggered grid ----
      // node-centred axis: cell l, weight o; half-staggered axis: cell l-1
      // with weight o+1/2 if o < 1/2, else cell l with weight o-1/2
      const bool xl = x < R(0.5), yl = y < R(0.5);
      const R whx = xl ? x + R(0.5) : x - R(0.5);
      const R why = yl ? y + R(0.5) : y - R(0.5);
      const int b_nn = (ly + 1) * FW + (lx + 1);
      const int b_hn = b_nn - (xl ? 1 : 0);
      const int b_nh = b_nn - (yl ? FW : 0);
      const int b_hh = b_hn - (yl ? FW : 0);
#define ZP_BILIN(F, b, wx, wy)                                               \
  ((R(1) - (wy)) * ((R(1) - (wx)) * (F)[b] + (wx) * (F)[(b) + 1]) +          \
   (wy) * ((R(1) - (wx)) * (F)[(b) + FW] + (wx) * (F)[(b) + FW + 1]))
      const R ex = ZP_BILIN(Ex, b_hn, whx, y);
      const R ey = ZP_BILIN(Ey, b_nh, x, why);
      const R ez = ZP_BILIN(Ez, b_nn, x, y);
      const R bx = ZP_BILIN(Bx, b_nh, x, why);
      const R by = ZP_BILIN(By, b_hn, whx, y);
      const R bz = ZP_BILIN(Bz, b_hh, whx, why);
#undef ZP_BILIN

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
      if (do_energy && valid) kin += w * u2 * fdiv<R>(rgn, R(1) + rgn);
      R x1 = x + dt_dx * ux * rgn;
      R y1 = y + dt_dy * uy * rgn;
      R xf, yf;
      const int di = axis_cross(x1, xf);
      const int dj = axis_cross(y1, yf);

      // ---- stage 3: charge-conserving deposit ----
      // The straight path from (x, y) to (x1, y1) (start-cell frame) is cut
      // where it meets the x face xb (parameter sx) and the y face yb (sy);
      // s1 = min, s2 = max (an exact tie counts as x first).  Segment 1 lies
      // in the start cell, segment 2 in the cell entered at s1, segment 3 in
      // the final cell; each is written in its own cell's frame and the last
      // one ends at the stored offsets (xf, yf).  Empty segments are skipped
      // per lane; a warp skips a segment that none of its lanes needs.
      const R qx = qx0 * w, qy = qy0 * w, qz = q00 * w * uz * rgn;
      const R xb = di > 0 ? R(1) : R(0);
      const R yb = dj > 0 ? R(1) : R(0);
      const R sx = di ? fdiv<R>(xb - x, x1 - x) : R(1);
      const R sy = dj ? fdiv<R>(yb - y, y1 - y) : R(1);
      const bool xfirst = sx <= sy;
      const R s1 = xfirst ? sx : sy, s2 = xfirst ? sy : sx;
      const R y_sx = y + sx * (y1 - y);  // where the path meets the x face
      const R x_sy = x + sy * (x1 - x);  // where it meets the y face
      const bool cut = (di | dj) != 0;
      const bool two = di != 0 && dj != 0;
      {
        const R bx1 = cut ? (xfirst ? xb : x_sy) : xf;
        const R by1 = cut ? (xfirst ? y_sx : yb) : yf;
        if (valid) dep_seg(jt, JW, JP, lx, ly, x, y, bx1, by1, s1, qx, qy, qz);
      }
      // segments outside the start cell wait in the warp's queue
      const bool need2 = valid && cut, need3 = valid && two;
      const unsigned m2 = __ballot_sync(0xffffffffu, need2);
      if (m2) {
        if (need2) {
          const int c2x = xfirst ? di : 0, c2y = xfirst ? 0 : dj;
          const R ax2 = xfirst ? xb - R(di) : x_sy;
          const R ay2 = xfirst ? y_sx : yb - R(dj);
          const R bx2 = two ? (xfirst ? x_sy - R(di) : xb) : xf;
          const R by2 = two ? (xfirst ? yb : y_sx - R(dj)) : yf;
          queue_put(q, (qtail + __popc(m2 & lt)) & (kQ - 1), lx + c2x,
                    ly + c2y, ax2, ay2, bx2, by2, s2 - s1, qx, qy, qz);
        }
        qtail += __popc(m2);
        // the ring holds kQ = 64: before each put at most 31 entries wait,
        // a put adds at most 32, and a full run of 32 is drained at once
        __syncwarp();
        if (qtail - qhead >= 32) {
          queue_take(q, jt, JW, JP, (qhead + lane) & (kQ - 1));
          qhead += 32;
          __syncwarp();
        }
        const unsigned m3 = __ballot_sync(0xffffffffu, need3);
        if (m3) {
          if (need3) {
            const R ax3 = xfirst ? x_sy - R(di) : xb - R(di);
            const R ay3 = xfirst ? yb - R(dj) : y_sx - R(dj);
            queue_put(q, (qtail + __popc(m3 & lt)) & (kQ - 1), lx + di,
                      ly + dj, ax3, ay3, xf, yf, R(1) - s2, qx, qy, qz);
          }
          qtail += __popc(m3);
          __syncwarp();
          if (qtail - qhead >= 32) {
            queue_take(q, jt, JW, JP, (qhead + lane) & (kQ - 1));
            qhead += 32;
            __syncwarp();
          }
        }
      }

      // ---- new cell: window shift, boundaries, tile membership ----
      int nix = x0 + lx + di - shift;
      const int niy = wrap1(y0 + ly + dj, ny);
      bool removed = false;
      if (open_x)  // leaves the window it moved in, or the shifted window
        removed = nix + shift >= nx || nix < 0;
      else
        nix = wrap1(nix, nx);
      const int nlx = nix - x0, nly = niy - y0;
      const bool inside = (unsigned)nlx < (unsigned)tw && (unsigned)nly < (unsigned)th;
      const bool stay = valid && !removed && inside;
      const bool leave = valid && !removed && !inside;
      if (valid && removed) ++n_removed;

      // ---- output: stayers to this tile's segment of the other copy,
      // leavers (global cell) to the tile's outbox ----
      const unsigned bs = __ballot_sync(0xffffffffu, stay);
      const unsigned bl = __ballot_sync(0xffffffffu, leave);
      int sb = 0, lb = 0;
      if (lane == 0) {
        if (bs) sb = atomicAdd(&s_slots[0], __popc(bs));
        if (bl) lb = atomicAdd(&s_slots[1], __popc(bl));
      }
      sb = __shfl_sync(0xffffffffu, sb, 0);
      lb = __shfl_sync(0xffffffffu, lb, 0);
      if (stay) {
        const int d = base + sb + __popc(bs & lt);
        __stcs(O.cell + d, local_cell(nlx, nly));
        __stcs(O.x + d, xf);
        __stcs(O.y + d, yf);
        __stcs(O.ux + d, ux);
        __stcs(O.uy + d, uy);
        __stcs(O.uz + d, uz);
        if (O.w) __stcs(O.w + d, w);
        if (O.id) __stcs(O.id + d, pid);
      } else if (leave) {
        const int slot = lb + __popc(bl & lt);
        if (slot < ob_cap) {
          const size_t d = (size_t)tile * ob_cap + slot;
          P.ob_ix[d] = nix;
          P.ob_iy[d] = niy;
          P.ob_x[d] = xf;
          P.ob_y[d] = yf;
          P.ob_ux[d] = ux;
          P.ob_uy[d] = uy;
          P.ob_uz[d] = uz;
          if (O.w) P.ob_w[d] = w;
          if (O.id) P.ob_id[d] = pid;
        } else {
          const int o = atomicAdd(&st->ovf_count, 1);
          if (o < ovf.cap) {
            ovf.sim[o] = it.x;
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
      }
    }
    // segments still waiting in the warp's queue
    __syncwarp();
    if (lane < qtail - qhead)
      queue_take(q, jt, JW, JP, (qhead + lane) & (kQ - 1));
    if (n_removed) atomicAdd(&S.removed[s], n_removed);
    if (do_energy)
      block_sum_store<R>((double)kin,
                         &S.part_kin[(size_t)tile * kMaxSpecies + s], red);
    __syncthreads();
    if (threadIdx.x == 0) {
      P.cnt[tile] = s_slots[0];
      P.ob_cnt[tile] = min(s_slots[1], ob_cap);
    }
  }
  __syncthreads();

  // ---- stage 3b: fold the tile's current (with guards) into global J ----
  for (int k = threadIdx.x; k < 3 * JP; k += blockDim.x) {
    if (!jt.nonzero(k)) continue;
    const int c = k / JP, r = k - c * JP;
    const int lj = r / JW, li = r - lj * JW;
    int gi = x0 - 1 + li;
    const int gj = wrap1(y0 - 1 + lj, ny);
    if (open_x) {
      if (gi < 0 || gi >= nx) continue;
    } else {
      gi = wrap1(gi, nx);
    }
    atomicAdd(S.J[cur][c] + (size_t)gj * ld + gi, (R)(jt.value(k) * S.jscale[c]));
  }
}

template <typename R>
size_t push_smem_bytes(int tx, int ty) {
  // 6 field planes of R, then 3 current planes of 8 bytes (two int32 words
  // in FP32, one double in FP64), then (16-byte aligned) per warp a queue of
  // kQ segments of 8 R + 1 int
  const size_t head = sizeof(R) * 6 * (size_t)(tx + 2) * (ty + 2) +
                      8 * 3 * (size_t)(tx + 3) * (ty + 3);
  return ((head + 15) & ~size_t(15)) +
         (size_t)kWarps * kQ * (8 * sizeof(R) + sizeof(int));
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
cudaError_t prepare_push_deposit(int max_tx, int max_ty) {
  const int smem = (int)push_smem_bytes<R>(max_tx, max_ty);
  cudaError_t e = set_push_smem<R, false>(smem);
  if (e != cudaSuccess) return e;
  return set_push_smem<R, true>(smem);
}

template <typename R>
cudaError_t launch_push_deposit(const SimDev<R> *sims, const SimDev<R> *single,
                                const int2 *items, int n_items, int max_tx,
                                int max_ty, bool all16, BatchStatus *st,
                                const OverflowDev<R> &ovf,
                                cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = push_smem_bytes<R>(max_tx, max_ty);
  // the 16 x 16 kernel needs every simulation of the batch to use 16 x 16
  // tiles (ragged edge tiles are fine)
  const bool t16 = all16;
  if (single) {
    if (t16)
      push_deposit_kernel<R, false, 16, 16><<<n_items, kThreads, smem, stream>>>(
          sims, *single, items, st, ovf);
    else
      push_deposit_kernel<R, false, 0, 0><<<n_items, kThreads, smem, stream>>>(
          sims, *single, items, st, ovf);
  } else {
    if (t16)
      push_deposit_kernel<R, true, 16, 16><<<n_items, kThreads, smem, stream>>>(
          sims, SimDev<R>{}, items, st, ovf);
    else
      push_deposit_kernel<R, true, 0, 0><<<n_items, kThreads, smem, stream>>>(
          sims, SimDev<R>{}, items, st, ovf);
  }
  return cudaGetLastError();
}

template size_t push_smem_bytes<float>(int, int);
template size_t push_smem_bytes<double>(int, int);
template cudaError_t prepare_push_deposit<float>(int, int);
template cudaError_t prepare_push_deposit<double>(int, int);
template cudaError_t launch_push_deposit<float>(const SimDev<float> *,
                                                const SimDev<float> *,
                                                const int2 *, int, int, int,
                                                bool, BatchStatus *,
                                                const OverflowDev<float> &,
                                                cudaStream_t);
template cudaError_t launch_push_deposit<double>(const SimDev<double> *,
                                                 const SimDev<double> *,
                                                 const int2 *, int, int, int,
                                                 bool, BatchStatus *,
                                                 const OverflowDev<double> &,
                                                 cudaStream_t);

}  // namespace zp
