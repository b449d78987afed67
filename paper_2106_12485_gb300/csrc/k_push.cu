// k_push.cu -- fused particle kernel: interpolation, Boris push, move,
// charge-conserving deposition and in-tile compaction (PIC stages 1-3 of
// Sec. 2.2; the per-region particle advance with local current buffers and
// a ghost-cell reduction of Sec. 3.2, here one CTA per tile).
//
// Per work item (simulation, tile) one CTA:
//  1. stages E, B of the tile plus one guard cell on each side in shared
//     memory ([-1, tx] x [-1, ty]) and zeroes a shared J tile covering
//     [-1, tx+1] x [-1, ty+1];
//  2. streams the tile's particles in chunks of 256 (one per thread):
//     bilinear gather of the staggered fields from shared memory,
//     relativistic Boris rotation, move by dt u/gamma (at most one cell,
//     CFL), split of the straight path at the cell faces it crosses and
//     accumulation of each segment's current into the shared J tile;
//  3. writes particles that stay in the tile back to the front of the
//     segment (stable in-place compaction: ballot + prefix per warp, warp
//     totals through shared memory) and particles that leave to the tile's
//     outbox; particles leaving an open boundary are dropped;
//  4. adds the shared J tile (interior and guard cells) to the global J
//     with one reduction per cell (periodic images folded here).
// Traffic per particle: one read and one write of its SoA record.
#include "zpic_dev.cuh"
#include "zpic_kernels.h"

namespace zp {

template <typename R>
__device__ __forceinline__ R rsqrt_r(R v);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float v) { return rsqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double v) { return rsqrt(v); }

// Crossing decision on one axis (identical rule to the method's reading:
// cross iff o1 >= 1 or o1 < 0; a backward crossing whose new offset rounds
// to exactly 1 stays in the cell at offset 0).  of = stored offset,
// oe = path end in the start cell's frame.
template <typename R>
__device__ __forceinline__ int axis_cross(R o1, R &of, R &oe) {
  if (o1 >= R(1)) {
    of = o1 - R(1);
    oe = o1;
    return 1;
  }
  if (o1 < R(0)) {
    const R t = o1 + R(1);
    if (t == R(1)) {
      of = R(0);
      oe = R(0);
      return 0;
    }
    of = t;
    oe = o1;
    return -1;
  }
  of = o1;
  oe = o1;
  return 0;
}

// One straight segment inside cell (ci, cj) (tile-local), from (xa, ya) to
// (xb, yb) in that cell's offsets, covering fraction f of the step.
// js: three planes of JP values, row length JW, origin at cell (-1, -1).
template <typename R>
__device__ __forceinline__ void dep_seg(R *js, int JW, int JP, int ci, int cj,
                                        R xa, R ya, R xb, R yb, R f, R qx,
                                        R qy, R qz) {
  const R ddx = xb - xa, ddy = yb - ya;
  const R xm = R(0.5) * (xa + xb), ym = R(0.5) * (ya + yb);
  const int b = (cj + 1) * JW + (ci + 1);
  const R ax = qx * ddx, ay = qy * ddy, az = qz * f;
  const R c = ddx * ddy * R(1.0 / 12.0);
  R *jx = js, *jy = js + JP, *jz = js + 2 * JP;
  atomicAdd(jx + b, ax * (R(1) - ym));
  atomicAdd(jx + b + JW, ax * ym);
  atomicAdd(jy + b, ay * (R(1) - xm));
  atomicAdd(jy + b + 1, ay * xm);
  atomicAdd(jz + b, az * ((R(1) - xm) * (R(1) - ym) + c));
  atomicAdd(jz + b + 1, az * (xm * (R(1) - ym) - c));
  atomicAdd(jz + b + JW, az * ((R(1) - xm) * ym - c));
  atomicAdd(jz + b + JW + 1, az * (xm * ym + c));
}

template <typename R>
__device__ __forceinline__ R field_at(const SimDev<R> &S, const R *f, int gi,
                                      int gj) {
  gj = wrap1(gj, S.ny);
  if (S.open_x) {
    if (gi < 0 || gi >= S.nx) return R(0);
  } else {
    gi = wrap1(gi, S.nx);
  }
  return f[(size_t)gj * S.ld + gi];
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

template <typename R>
__global__ void __launch_bounds__(kThreads, 2)
    push_deposit_kernel(const SimDev<R> *__restrict__ sims,
                        const int2 *__restrict__ items, BatchStatus *st,
                        OverflowDev<R> ovf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int wcnt[2][kWarps][2];
  __shared__ double red[kWarps];

  const int step = st->step;
  if (frozen(st, step)) return;
  const int2 it = items[blockIdx.x];
  const SimDev<R> &S = sims[it.x];
  const int tile = it.y;
  const int tcx = tile % S.ntx, tcy = tile / S.ntx;
  const int x0 = tcx * S.tx, y0 = tcy * S.ty;
  const int tw = min(S.tx, S.nx - x0), th = min(S.ty, S.ny - y0);
  const int cur = step & 1;

  // shared layout: 6 field planes (FW x FH) then 3 current planes (JW x JH)
  const int FW = S.tx + 2, FH = S.ty + 2, FP = FW * FH;
  const int JW = S.tx + 3, JH = S.ty + 3, JP = JW * JH;
  R *fs = reinterpret_cast<R *>(smem_raw);
  R *js = fs + 6 * FP;

  {
    const R *src[6] = {S.E[cur][0], S.E[cur][1], S.E[cur][2],
                       S.B[cur][0], S.B[cur][1], S.B[cur][2]};
    for (int k = threadIdx.x; k < 6 * FP; k += blockDim.x) {
      const int c = k / FP, r = k - c * FP;
      const int lj = r / FW, li = r - lj * FW;
      fs[k] = field_at(S, src[c], x0 - 1 + li, y0 - 1 + lj);
    }
    for (int k = threadIdx.x; k < 3 * JP; k += blockDim.x) js[k] = R(0);
  }
  const int nsh = S.moving_window ? *S.n_shift : 0;
  const int shift = shift_due(S, step, nsh) ? 1 : 0;
  const bool do_energy =
      S.energy_every > 0 && ((step + 1) % S.energy_every) == 0;
  __syncthreads();

  const R *Ex = fs, *Ey = fs + FP, *Ez = fs + 2 * FP;
  const R *Bx = fs + 3 * FP, *By = fs + 4 * FP, *Bz = fs + 5 * FP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int chunk = 0;

  for (int s = 0; s < S.nsp; ++s) {
    const SpeciesDev<R> &P = S.sp[s];
    const int n = P.cnt[tile];
    const size_t base = (size_t)P.off[tile];
    const size_t obase = (size_t)tile * P.ob_cap;
    int n_stay = 0, n_out = 0, n_removed = 0;
    R kin = R(0);
    for (int c0 = 0; c0 < n; c0 += blockDim.x, ++chunk) {
      const int k = c0 + threadIdx.x;
      const bool valid = k < n;
      bool stay = false, leave = false;
      int nix = 0, niy = 0, pid = 0;
      R xf = R(0), yf = R(0), ux = R(0), uy = R(0), uz = R(0), w = R(1);
      if (valid) {
        const size_t p = base + k;
        const int ix = P.ix[p], iy = P.iy[p];
        const R x = P.x[p], y = P.y[p];
        ux = P.ux[p];
        uy = P.uy[p];
        uz = P.uz[p];
        if (P.w) w = P.w[p];
        if (P.id) pid = P.id[p];
        int lx = ix - x0, ly = iy - y0;
        if ((unsigned)lx >= (unsigned)tw || (unsigned)ly >= (unsigned)th) {
          // never produced by the library's own kernels: record and keep
          // the shared-memory accesses inside the tile
          atomicOr(&st->error, ERR_STORE);
          atomicMin(&st->err_step, step);
          lx = min(max(lx, 0), tw - 1);
          ly = min(max(ly, 0), th - 1);
        }

        // ---- stage 1: bilinear gather on the staggered grid ----
        // node-centred axis: cell l, weight o; half-staggered axis: cell
        // l-1 with weight o+1/2 if o < 1/2, else cell l with weight o-1/2
        const bool xl = x < R(0.5), yl = y < R(0.5);
        const int hx = xl ? lx - 1 : lx, hy = yl ? ly - 1 : ly;
        const R whx = xl ? x + R(0.5) : x - R(0.5);
        const R why = yl ? y + R(0.5) : y - R(0.5);
        const int b_nn = (ly + 1) * FW + (lx + 1);
        const int b_hn = (ly + 1) * FW + (hx + 1);
        const int b_nh = (hy + 1) * FW + (lx + 1);
        const int b_hh = (hy + 1) * FW + (hx + 1);
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
        const R h = P.hq;
        const R umx = ux + h * ex, umy = uy + h * ey, umz = uz + h * ez;
        const R rg = rsqrt_r<R>(R(1) + umx * umx + umy * umy + umz * umz);
        const R tx = h * bx * rg, ty = h * by * rg, tz = h * bz * rg;
        const R sf = R(2) / (R(1) + tx * tx + ty * ty + tz * tz);
        const R upx = umx + (umy * tz - umz * ty);
        const R upy = umy + (umz * tx - umx * tz);
        const R upz = umz + (umx * ty - umy * tx);
        ux = umx + sf * (upy * tz - upz * ty) + h * ex;
        uy = umy + sf * (upz * tx - upx * tz) + h * ey;
        uz = umz + sf * (upx * ty - upy * tx) + h * ez;

        // ---- stage 2b: move ----
        const R u2 = ux * ux + uy * uy + uz * uz;
        const R rgn = rsqrt_r<R>(R(1) + u2);
        if (do_energy) kin += w * u2 / (R(1) / rgn + R(1));  // w (gamma-1)
        R x1 = x + S.dt_dx * ux * rgn;
        R y1 = y + S.dt_dy * uy * rgn;
        const int di = axis_cross(x1, xf, x1);
        const int dj = axis_cross(y1, yf, y1);

        // ---- stage 3: charge-conserving deposit, path split at faces ----
        const R qx = P.qx * w, qy = P.qy * w, qz = P.q0 * w * uz * rgn;
        if (di == 0 && dj == 0) {
          dep_seg(js, JW, JP, lx, ly, x, y, xf, yf, R(1), qx, qy, qz);
        } else if (dj == 0) {
          const R xb = di > 0 ? R(1) : R(0);
          const R sx = (xb - x) / (x1 - x);
          const R yc = y + sx * (y1 - y);
          dep_seg(js, JW, JP, lx, ly, x, y, xb, yc, sx, qx, qy, qz);
          dep_seg(js, JW, JP, lx + di, ly, xb - R(di), yc, xf, yf, R(1) - sx,
                  qx, qy, qz);
        } else if (di == 0) {
          const R yb = dj > 0 ? R(1) : R(0);
          const R sy = (yb - y) / (y1 - y);
          const R xc = x + sy * (x1 - x);
          dep_seg(js, JW, JP, lx, ly, x, y, xc, yb, sy, qx, qy, qz);
          dep_seg(js, JW, JP, lx, ly + dj, xc, yb - R(dj), xf, yf, R(1) - sy,
                  qx, qy, qz);
        } else {
          const R xb = di > 0 ? R(1) : R(0);
          const R yb = dj > 0 ? R(1) : R(0);
          const R sx = (xb - x) / (x1 - x);
          const R sy = (yb - y) / (y1 - y);
          const R y_sx = y + sx * (y1 - y);
          const R x_sy = x + sy * (x1 - x);
          if (sx <= sy) {
            dep_seg(js, JW, JP, lx, ly, x, y, xb, y_sx, sx, qx, qy, qz);
            dep_seg(js, JW, JP, lx + di, ly, xb - R(di), y_sx, x_sy - R(di),
                    yb, sy - sx, qx, qy, qz);
            dep_seg(js, JW, JP, lx + di, ly + dj, x_sy - R(di), yb - R(dj), xf,
                    yf, R(1) - sy, qx, qy, qz);
          } else {
            dep_seg(js, JW, JP, lx, ly, x, y, x_sy, yb, sy, qx, qy, qz);
            dep_seg(js, JW, JP, lx, ly + dj, x_sy, yb - R(dj), xb, y_sx - R(dj),
                    sx - sy, qx, qy, qz);
            dep_seg(js, JW, JP, lx + di, ly + dj, xb - R(di), y_sx - R(dj), xf,
                    yf, R(1) - sx, qx, qy, qz);
          }
        }

        // ---- new cell: window shift, boundaries, tile membership ----
        nix = ix + di - shift;
        niy = wrap1(iy + dj, S.ny);
        bool removed = false;
        if (S.open_x) {
          removed = nix < 0 || nix >= S.nx;
        } else {
          nix = wrap1(nix, S.nx);
        }
        if (removed) {
          ++n_removed;
        } else if (nix >= x0 && nix < x0 + tw && niy >= y0 && niy < y0 + th) {
          stay = true;
        } else {
          leave = true;
        }
      }

      // ---- stable compaction of stayers, outbox for leavers ----
      const unsigned bs = __ballot_sync(0xffffffffu, stay);
      const unsigned bl = __ballot_sync(0xffffffffu, leave);
      const int buf = chunk & 1;
      if (lane == 0) {
        wcnt[buf][warp][0] = __popc(bs);
        wcnt[buf][warp][1] = __popc(bl);
      }
      __syncthreads();  // also: every load of this chunk is done
      int os = 0, ol = 0, ts = 0, tl = 0;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) {
        const int a = wcnt[buf][q][0], b = wcnt[buf][q][1];
        if (q < warp) {
          os += a;
          ol += b;
        }
        ts += a;
        tl += b;
      }
      if (stay) {
        const size_t d = base + n_stay + os + __popc(bs & lt);
        P.ix[d] = nix;
        P.iy[d] = niy;
        P.x[d] = xf;
        P.y[d] = yf;
        P.ux[d] = ux;
        P.uy[d] = uy;
        P.uz[d] = uz;
        if (P.w) P.w[d] = w;
        if (P.id) P.id[d] = pid;
      } else if (leave) {
        const int slot = n_out + ol + __popc(bl & lt);
        if (slot < P.ob_cap) {
          const size_t d = obase + slot;
          P.ob_ix[d] = nix;
          P.ob_iy[d] = niy;
          P.ob_x[d] = xf;
          P.ob_y[d] = yf;
          P.ob_ux[d] = ux;
          P.ob_uy[d] = uy;
          P.ob_uz[d] = uz;
          if (P.w) P.ob_w[d] = w;
          if (P.id) P.ob_id[d] = pid;
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
      n_stay += ts;
      n_out += tl;
    }
    if (threadIdx.x == 0) {
      P.cnt[tile] = n_stay;
      P.ob_cnt[tile] = min(n_out, P.ob_cap);
    }
    if (n_removed) atomicAdd(&S.removed[s], n_removed);
    if (do_energy)
      block_sum_store<R>((double)kin,
                         &S.part_kin[(size_t)tile * kMaxSpecies + s], red);
  }
  __syncthreads();

  // ---- stage 3b: fold the tile's current (with guards) into global J ----
  {
    R *J[3] = {S.J[cur][0], S.J[cur][1], S.J[cur][2]};
    for (int k = threadIdx.x; k < 3 * JP; k += blockDim.x) {
      const R v = js[k];
      if (v == R(0)) continue;
      const int c = k / JP, r = k - c * JP;
      const int lj = r / JW, li = r - lj * JW;
      int gi = x0 - 1 + li;
      const int gj = wrap1(y0 - 1 + lj, S.ny);
      if (S.open_x) {
        if (gi < 0 || gi >= S.nx) continue;
      } else {
        gi = wrap1(gi, S.nx);
      }
      atomicAdd(J[c] + (size_t)gj * S.ld + gi, v);
    }
  }
}

template <typename R>
size_t push_smem_bytes(int tx, int ty) {
  return sizeof(R) * (6 * (size_t)(tx + 2) * (ty + 2) +
                      3 * (size_t)(tx + 3) * (ty + 3));
}

template <typename R>
cudaError_t prepare_push_deposit(int max_tx, int max_ty) {
  return cudaFuncSetAttribute(push_deposit_kernel<R>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)push_smem_bytes<R>(max_tx, max_ty));
}

template <typename R>
cudaError_t launch_push_deposit(const SimDev<R> *sims, const int2 *items,
                                int n_items, int max_tx, int max_ty,
                                BatchStatus *st, const OverflowDev<R> &ovf,
                                cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  const size_t smem = push_smem_bytes<R>(max_tx, max_ty);
  push_deposit_kernel<R><<<n_items, kThreads, smem, stream>>>(sims, items, st,
                                                              ovf);
  return cudaGetLastError();
}

template size_t push_smem_bytes<float>(int, int);
template size_t push_smem_bytes<double>(int, int);
template cudaError_t prepare_push_deposit<float>(int, int);
template cudaError_t prepare_push_deposit<double>(int, int);
template cudaError_t launch_push_deposit<float>(const SimDev<float> *,
                                                const int2 *, int, int, int,
                                                BatchStatus *,
                                                const OverflowDev<float> &,
                                                cudaStream_t);
template cudaError_t launch_push_deposit<double>(const SimDev<double> *,
                                                 const int2 *, int, int, int,
                                                 BatchStatus *,
                                                 const OverflowDev<double> &,
                                                 cudaStream_t);

}  // namespace zp
