// k_field.cu -- field kernels: fused Yee step (PIC stage 4 of Sec. 2.2),
// laser initialisation (Sec. 4.1), and the end-of-step bookkeeping
// (energy records, moving-window counter, step counter).
//
// Yee step, one CTA (256 threads) per 32 x Y block of cells (Y = 32 in
// FP32, 16 in FP64), temporal blocking of the three sub-steps inside the
// block:
//   load E^n on [-1, 33] x [-1, Y+1], B^n on [-1, 32] x [-1, Y],
//        J on [0, 32] x [0, Y]
//   B^{n+1/2} = B^n - (dt/2) curl E^n        on [-1, 32] x [-1, Y]
//   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J) on [0, 32] x [0, Y]
//   B^{n+1}   = B^{n+1/2} - (dt/2) curl E^{n+1} on the block's own cells
// and writes E^{n+1}, B^{n+1} of its own cells to the other field copy, one
// cell to the left when the moving window shifts this step.  HBM traffic per
// cell: read E, B, J (9 values), write E, B (6) and zero the other J (3).
#include <math.h>

#include <type_traits>

#include "zpic_dev.cuh"
#include "zpic_kernels.h"

namespace zp {

// periodic index for any i (the 34 x 10 halo can exceed twice a tiny grid);
// indices already in range, nearly all of them, skip the division
__device__ __forceinline__ int wrapg(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  i %= n;
  return i < 0 ? i + n : i;
}

template <typename R>
__device__ __forceinline__ R fld(const SimDev<R> &S, const R *f, int gi,
                                 int gj) {
  gj = wrapg(gj, S.ny);
  if (S.open_x) {
    if (gi < 0 || gi >= S.nx) return R(0);
  } else {
    gi = wrapg(gi, S.nx);
  }
  return f[(size_t)gj * S.ld + gi];
}

// the same boundary rules for this step's deposited current
template <typename R>
__device__ __forceinline__ R fld_j(const SimDev<R> &S, int cur, int c, int gi,
                                   int gj) {
  gj = wrapg(gj, S.ny);
  if (S.open_x) {
    if (gi < 0 || gi >= S.nx) return R(0);
  } else {
    gi = wrapg(gi, S.nx);
  }
  return j_value(S, cur, c, (size_t)gj * S.ld + gi);
}

// The deposited current as stored (FP32: the int64 fixed-point sum; FP64:
// the double), for loads that are scaled only once they have all arrived.
template <typename R>
using JRaw = typename std::conditional<sizeof(R) == 4, long long, R>::type;

template <typename R>
__device__ __forceinline__ const JRaw<R> *j_plane(const SimDev<R> &S, int cur,
                                                  int c) {
  if constexpr (sizeof(R) == 4)
    return S.Jq[cur][c];
  else
    return S.J[cur][c];
}

template <typename R>
__device__ __forceinline__ R j_scale(const SimDev<R> &S, int c, JRaw<R> v) {
  if constexpr (sizeof(R) == 4)
    return fixed_to_float(v) * S.jscale[c];
  else if (S.jfixed)
    return (double)__double_as_longlong(v) * S.jscale_d[c];
  else
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // valid in warp 0 lane 0 (and every warp's lane 0)
}

// Compensated FP64 sum (Kahan-Babuska / Neumaier, with Knuth's branch-free
// TwoSum): s holds the rounded running sum and c the accumulated rounding
// errors, so s + c carries the exact sum's leading digits until c itself
// rounds; the result's error stays near one rounding of the total instead of
// growing with the number of terms.  Used for the energy diagnostics.
struct CSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x, bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ void add(const CSum &o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// CSum over the CTA in a fixed order (shuffle tree, then warp 0 over the
// warp sums); the result is valid in thread 0.
__device__ __forceinline__ CSum block_csum(CSum v, double *red2) {
  for (int o = 16; o > 0; o >>= 1) {
    CSum u;
    u.s = __shfl_down_sync(0xffffffffu, v.s, o);
    u.c = __shfl_down_sync(0xffffffffu, v.c, o);
    v.add(u);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red2[2 * warp] = v.s;
    red2[2 * warp + 1] = v.c;
  }
  __syncthreads();
  CSum w;
  if (lane < (int)(blockDim.x >> 5)) {
    w.s = red2[2 * lane];
    w.c = red2[2 * lane + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    CSum u;
    u.s = __shfl_down_sync(0xffffffffu, w.s, o);
    u.c = __shfl_down_sync(0xffffffffu, w.c, o);
    w.add(u);
  }
  return w;
}

// Sums (e, b) over the CTA and stores the two totals at dst[0], dst[1]:
// each warp adds its 32 values in R (the cells' squares are R already),
// thread 0 adds the warp sums in double, in warp order.  Keeps the FP64 work
// of the field-energy report at one add per warp.
template <typename R>
__device__ __forceinline__ void block_sum2_store(R e, R b, double *red,
                                                 double *dst) {
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[2 * warp] = (double)e;
    red[2 * warp + 1] = (double)b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double se = 0.0, sb = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      se += red[2 * w];
      sb += red[2 * w + 1];
    }
    dst[0] = se;
    dst[1] = sb;
  }
}

// resident Yee CTAs per SM the register budget is sized for (64 registers
// in FP32; on a 2048^2 grid 0.102 ms per step, 0.104 ms at 3 CTAs per SM and
// 0.125 ms at 5, compiled for 48 registers)
constexpr int kYeeCtas = 4;

// Asynchronous copy of one field value (4 or 8 bytes) into shared memory;
// nbytes = 0 writes a zero instead of reading.
template <typename R>
__device__ __forceinline__ void cp_async_val(R *dst, const R *src,
                                             unsigned nbytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d),
                 "l"(src), "r"(nbytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d),
                 "l"(src), "r"(nbytes)
                 : "memory");
}

template <typename R>
__global__ void __launch_bounds__(kThreads, kYeeCtas)
    yee_kernel(const SimDev<R> *__restrict__ sims,
               const int2 *__restrict__ items, BatchStatus *st) {
  constexpr int X = kYeeX, Y = yee_rows<R>();
  constexpr int EW = X + 3, EH = Y + 3;   // E^n on [-1, X+1]
  constexpr int BW = X + 2, BH = Y + 2;   // B on [-1, X]
  constexpr int JW = X + 1, JH = Y + 1;   // J on [0, X]
  __shared__ R se[3][EH][EW];
  __shared__ R sb[3][BH][BW];
  __shared__ R sj[3][JH][JW];
  __shared__ double red[2 * kWarps];

  const int step = st->step;
  if (frozen(st, step)) return;
  const int2 it = items[blockIdx.x];
  const SimDev<R> &S = sims[it.x];
  const int bx = it.y % S.ybx, by = it.y / S.ybx;
  const int x0 = bx * X, y0 = by * Y;
  const int cur = step & 1, nxt = cur ^ 1;
  // the window decision (FP64) once per block, read after the first barrier
  __shared__ int s_shift;
  if (threadIdx.x == 0)
    s_shift = shift_due(S, step, S.moving_window ? *S.n_shift : 0);
  const bool do_energy =
      S.energy_every > 0 && ((step + 1) % S.energy_every) == 0;
  const R dt = S.dt, h = R(0.5) * S.dt;
  const R rdx = R(1) / S.dx, rdy = R(1) / S.dy;

  // The block's halo, cells [x0-1, x0+X+2) x [y0-1, y0+Y+2): E uses all of
  // it, B the first BW x BH, J the part from (x0, y0) on.  Each thread takes
  // halo cells k = tid + u kThreads, works out the cell's address once for
  // all nine arrays, and issues every load before it waits, so a block
  // waits for one memory round trip: E and B go straight into shared memory
  // by asynchronous copies (no registers held), J through registers (it is
  // scaled on the way in).
  constexpr int HN = EH * EW;
  constexpr int UH = (HN + kThreads - 1) / kThreads;
  const bool filtered = S.Jf[0] != nullptr;  // drive E with the filtered J
  const int nx = S.nx, ny = S.ny;
  const bool open_x = S.open_x != 0;
  size_t off[UH];
  bool in[UH];   // inside the halo and not beyond an open x edge
  int hl[UH];    // (lj << 8) | li
#pragma unroll
  for (int u = 0; u < UH; ++u) {
    const int k = threadIdx.x + u * kThreads;
    const int lj = k / EW, li = k - lj * EW;
    int gi = x0 - 1 + li;
    const int gj = wrapg(y0 - 1 + lj, ny);
    bool ok = k < HN;
    if (open_x)
      ok = ok && gi >= 0 && gi < nx;
    else
      gi = wrapg(gi, nx);
    in[u] = ok;
    off[u] = (size_t)gj * S.ld + (ok ? gi : 0);
    hl[u] = (lj << 8) | li;
  }
#pragma unroll
  for (int u = 0; u < UH; ++u) {
    if (threadIdx.x + u * kThreads >= HN) continue;
    const int lj = hl[u] >> 8, li = hl[u] & 255;
    const unsigned nb = in[u] ? (unsigned)sizeof(R) : 0u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cp_async_val<R>(&se[c][lj][li], S.E[cur][c] + off[u], nb);
      if (lj < BH && li < BW)
        cp_async_val<R>(&sb[c][lj][li], S.B[cur][c] + off[u], nb);
    }
  }
  // J on local [0, X] x [0, Y]: halo cells (li, lj) >= (1, 1)
  const auto j_cell = [&](int u) {
    const int lj = hl[u] >> 8, li = hl[u] & 255;
    return lj >= 1 && li >= 1 && lj <= JH && li <= JW;
  };
  if (filtered) {
    R vj[3][UH];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R *__restrict__ pj = S.Jf[c];
#pragma unroll
      for (int u = 0; u < UH; ++u)
        vj[c][u] = in[u] && j_cell(u) ? pj[off[u]] : R(0);
    }
#pragma unroll
    for (int u = 0; u < UH; ++u) {
      if (!j_cell(u) || threadIdx.x + u * kThreads >= HN) continue;
      const int lj = (hl[u] >> 8) - 1, li = (hl[u] & 255) - 1;
#pragma unroll
      for (int c = 0; c < 3; ++c) sj[c][lj][li] = vj[c][u];
    }
  } else {
    // the raw deposit (FP32: int64 fixed point), scaled after the wait
    JRaw<R> vj[3][UH];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const JRaw<R> *__restrict__ pj = j_plane(S, cur, c);
#pragma unroll
      for (int u = 0; u < UH; ++u)
        vj[c][u] = in[u] && j_cell(u) ? pj[off[u]] : JRaw<R>(0);
    }
#pragma unroll
    for (int u = 0; u < UH; ++u) {
      if (!j_cell(u) || threadIdx.x + u * kThreads >= HN) continue;
      const int lj = (hl[u] >> 8) - 1, li = (hl[u] & 255) - 1;
#pragma unroll
      for (int c = 0; c < 3; ++c) sj[c][lj][li] = j_scale(S, c, vj[c][u]);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  const int shift = s_shift;

  // B^{n+1/2} on local [-1, X] x [-1, Y]; sb index = local + 1
  for (int k = threadIdx.x; k < BH * BW; k += blockDim.x) {
    const int lj = k / BW, li = k - lj * BW;  // local (li-1, lj-1)
    // E(i, j) is se[.][lj][li]; E(i+1, j) se[.][lj][li+1]; E(i, j+1) se[.][lj+1][li]
    const R ez = se[2][lj][li];
    const R nbx = sb[0][lj][li] - h * (se[2][lj + 1][li] - ez) * rdy;
    const R nby = sb[1][lj][li] + h * (se[2][lj][li + 1] - ez) * rdx;
    const R nbz = sb[2][lj][li] - h * ((se[1][lj][li + 1] - se[1][lj][li]) * rdx -
                                       (se[0][lj + 1][li] - se[0][lj][li]) * rdy);
    const int gi = x0 - 1 + li;
    const bool out = S.open_x && (gi < 0 || gi >= S.nx);
    sb[0][lj][li] = out ? R(0) : nbx;
    sb[1][lj][li] = out ? R(0) : nby;
    sb[2][lj][li] = out ? R(0) : nbz;
  }
  __syncthreads();

  // E^{n+1} on local [0, X] x [0, Y]: se index = local + 1, sb index = local + 1
  for (int k = threadIdx.x; k < JH * JW; k += blockDim.x) {
    const int j = k / JW, i = k - j * JW;
    const R bzc = sb[2][j + 1][i + 1];
    const R nex = se[0][j + 1][i + 1] +
                  dt * ((bzc - sb[2][j][i + 1]) * rdy - sj[0][j][i]);
    const R ney = se[1][j + 1][i + 1] +
                  dt * (-(bzc - sb[2][j + 1][i]) * rdx - sj[1][j][i]);
    const R nez = se[2][j + 1][i + 1] +
                  dt * ((sb[1][j + 1][i + 1] - sb[1][j + 1][i]) * rdx -
                        (sb[0][j + 1][i + 1] - sb[0][j][i + 1]) * rdy -
                        sj[2][j][i]);
    const int gi = x0 + i;
    const bool out = S.open_x && gi >= S.nx;
    se[0][j + 1][i + 1] = out ? R(0) : nex;
    se[1][j + 1][i + 1] = out ? R(0) : ney;
    se[2][j + 1][i + 1] = out ? R(0) : nez;
  }
  __syncthreads();

  // B^{n+1} on the block's own cells (X * Y / kThreads per thread) and
  // write back
  R e2 = R(0), b2 = R(0);
#pragma unroll
  for (int r = threadIdx.x; r < X * Y; r += kThreads) {
  const int i = r % X, j = r / X;
  const int gi = x0 + i, gj = y0 + j;
  if (gi < S.nx && gj < S.ny) {
    const R ez = se[2][j + 1][i + 1];
    const R nbx = sb[0][j + 1][i + 1] - h * (se[2][j + 2][i + 1] - ez) * rdy;
    const R nby = sb[1][j + 1][i + 1] + h * (se[2][j + 1][i + 2] - ez) * rdx;
    const R nbz = sb[2][j + 1][i + 1] -
                  h * ((se[1][j + 1][i + 2] - se[1][j + 1][i + 1]) * rdx -
                       (se[0][j + 2][i + 1] - se[0][j + 1][i + 1]) * rdy);
    const R ex = se[0][j + 1][i + 1], ey = se[1][j + 1][i + 1];
    if (do_energy) {
      e2 += ex * ex + ey * ey + ez * ez;
      b2 += nbx * nbx + nby * nby + nbz * nbz;
    }
    const size_t row = (size_t)gj * S.ld;
    const int wi = gi - shift;
    if (wi >= 0) {
      S.E[nxt][0][row + wi] = ex;
      S.E[nxt][1][row + wi] = ey;
      S.E[nxt][2][row + wi] = ez;
      S.B[nxt][0][row + wi] = nbx;
      S.B[nxt][1][row + wi] = nby;
      S.B[nxt][2][row + wi] = nbz;
    }
    if (shift && gi == S.nx - 1) {  // the column entering the window
      for (int c = 0; c < 3; ++c) {
        S.E[nxt][c][row + gi] = R(0);
        S.B[nxt][c][row + gi] = R(0);
      }
    }
    for (int c = 0; c < 3; ++c) {
      if constexpr (sizeof(R) == 4)
        S.Jq[nxt][c][row + gi] = 0;
      else
        S.J[nxt][c][row + gi] = R(0);
    }
  }
  }
  if (do_energy)
    block_sum2_store(e2, b2, red, S.part_fld + (size_t)it.y * 2);
}

// Compensated binomial filter of the current (optional; Sec. 2.2 digital
// filter on J, Sec. 4.1 LWFA runs): per component and per axis, x then y,
// one (1, 2, 1)/4 pass and one (-1, 6, -1)/4 pass.  One CTA per Yee
// block (32 x Y): J on [-2, 34) x [-2, Y+2) in shared memory, the two x
// passes on all Y+4 rows, the two y passes on the block's rows; with an open x boundary
// every pass reads zero outside [0, nx), as if each pass were a separate
// sweep over the grid.  Writes Jf, which the Yee kernel then reads.  The
// three components' halos are loaded together (every load issued before
// the first is used), so a block waits for one memory round trip.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    filter_kernel(const SimDev<R> *__restrict__ sims,
                  const int2 *__restrict__ items, BatchStatus *st) {
  constexpr int X = kYeeX, Y = yee_rows<R>();
  constexpr int W = X + 4, H = Y + 4;
  static_assert(X * Y % kThreads == 0, "whole output cells per thread");
  __shared__ R a3[3][H][W];   // J per component, then its compensated x pass
  __shared__ R b[H][W];       // binomial x pass, then binomial y pass
  const int step = st->step;
  if (frozen(st, step)) return;
  const int2 it = items[blockIdx.x];
  const SimDev<R> &S = sims[it.x];
  if (!S.Jf[0]) return;
  const int x0 = (it.y % S.ybx) * X, y0 = (it.y / S.ybx) * Y;
  const int cur = step & 1;
  const bool open_x = S.open_x != 0;
  const R q = R(0.25), h = R(0.5), c15 = R(1.5);
  {
    constexpr int HN = H * W;
    constexpr int UF = (HN + kThreads - 1) / kThreads;
    const int nx = S.nx, ny = S.ny;
    size_t off[UF];
    bool in[UF];  // a halo cell, and not beyond an open x edge
#pragma unroll
    for (int u = 0; u < UF; ++u) {
      const int k = threadIdx.x + u * kThreads;
      const int lj = k / W, li = k - lj * W;
      int gi = x0 - 2 + li;
      const int gj = wrapg(y0 - 2 + lj, ny);
      bool ok = k < HN;
      if (open_x)
        ok = ok && gi >= 0 && gi < nx;
      else
        gi = wrapg(gi, nx);
      in[u] = ok;
      off[u] = (size_t)gj * S.ld + (ok ? gi : 0);
    }
    JRaw<R> v[3][UF];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const JRaw<R> *__restrict__ pj = j_plane(S, cur, c);
#pragma unroll
      for (int u = 0; u < UF; ++u) v[c][u] = in[u] ? pj[off[u]] : JRaw<R>(0);
    }
#pragma unroll
    for (int u = 0; u < UF; ++u) {
      const int k = threadIdx.x + u * kThreads;
      if (k >= HN) continue;
      const int lj = k / W, li = k - lj * W;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        a3[c][lj][li] = in[u] ? j_scale(S, c, v[c][u]) : R(0);
    }
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    R(*a)[W] = a3[c];
    // x binomial on local columns 1..W-2 (global x0 - 1 .. x0 + X)
    for (int k = threadIdx.x; k < H * (W - 2); k += blockDim.x) {
      const int lj = k / (W - 2), li = 1 + k - lj * (W - 2);
      const int gi = x0 - 2 + li;
      const bool out = open_x && (gi < 0 || gi >= S.nx);
      b[lj][li] = out ? R(0)
                      : q * a[lj][li - 1] + h * a[lj][li] + q * a[lj][li + 1];
    }
    __syncthreads();
    // x compensation on local columns 2..W-3 (the block's own columns)
    for (int k = threadIdx.x; k < H * X; k += blockDim.x) {
      const int lj = k / X, li = 2 + k - lj * X;
      a[lj][li] = -q * b[lj][li - 1] + c15 * b[lj][li] - q * b[lj][li + 1];
    }
    __syncthreads();
    // y binomial on local rows 1..H-2 (y is periodic: no edge rule)
    for (int k = threadIdx.x; k < (H - 2) * X; k += blockDim.x) {
      const int lj = 1 + k / X, li = 2 + k % X;
      b[lj][li] = q * a[lj - 1][li] + h * a[lj][li] + q * a[lj + 1][li];
    }
    __syncthreads();
    // y compensation on the block's own rows, written out
    for (int r = threadIdx.x; r < X * Y; r += kThreads) {
      const int i = r % X, j = r / X;
      const int gi = x0 + i, gj = y0 + j;
      const int li = i + 2, lj = j + 2;
      const R v = -q * b[lj - 1][li] + c15 * b[lj][li] - q * b[lj + 1][li];
      if (gi < S.nx && gj < S.ny) S.Jf[c][(size_t)gj * S.ld + gi] = v;
    }
    __syncthreads();
  }
}

template <typename R>
cudaError_t launch_filter(const SimDev<R> *sims, const int2 *items,
                          int n_items, BatchStatus *st, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  filter_kernel<R><<<n_items, kThreads, 0, stream>>>(sims, items, st);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_yee(const SimDev<R> *sims, const int2 *items, int n_items,
                       BatchStatus *st, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  yee_kernel<R><<<n_items, kThreads, 0, stream>>>(sims, items, st);
  return cudaGetLastError();
}

// ---- end of step ----------------------------------------------------------

// g_max CTAs per simulation (blockIdx.x = sim * g_max + slice); slices at
// or beyond the simulation's own count (end_g) only take the step ticket.
// On an energy step each CTA sums its slice of the per-tile kinetic and
// per-Yee-block field partials in compensated FP64 and stores (sum, error)
// per quantity; the last slice of the simulation to finish (ticket)
// combines the slices in slice order and writes the record.  The slicing
// depends on the simulation alone, so a simulation gives the same bits in a
// batch and on its own.  One CTA per simulation (energy steps: that last
// slice; otherwise slice 0) advances the window counter; every CTA takes the
// step ticket (after it has read the step), and the last one advances the
// step.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    end_step_kernel(const SimDev<R> *__restrict__ sims, int g_max,
                    BatchStatus *st) {
  __shared__ double red[kWarps * kEndQ * 2];
  __shared__ double s_part[kEndSlicesMax * kEndQ * 2];
  __shared__ double s_q[kEndQ * 2];
  __shared__ int s_last;
  const int step = st->step;
  if (frozen(st, step)) return;
  const int sim = blockIdx.x / g_max, g = blockIdx.x - sim * g_max;
  const SimDev<R> &S = sims[sim];
  const int G = S.end_g;
  const bool do_energy = g < G && S.energy_every > 0 &&
                         ((step + 1) % S.energy_every) == 0;
  bool owner = g == 0;
  if (do_energy) {
    const int ntiles = S.ntx * S.nty;
    const int nsp = S.nsp;
    // quantity k: kinetic energy of species k (k < nsp), E^2 (kMaxSpecies),
    // B^2 (kMaxSpecies + 1); the others stay zero
    auto used = [&](int k) { return k >= kMaxSpecies || k < nsp; };
    // this slice: tiles [t0, t1), Yee blocks [y0, y1)
    const int t0 = (int)((long long)ntiles * g / G);
    const int t1 = (int)((long long)ntiles * (g + 1) / G);
    const int nyb = S.ybx * S.yby;
    const int y0 = (int)((long long)nyb * g / G);
    const int y1 = (int)((long long)nyb * (g + 1) / G);
    CSum v[kEndQ];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
      if (s >= nsp) continue;
      const double *pk = S.part_kin + (size_t)s * ntiles;
      for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) v[s].add(pk[t]);
    }
    for (int t = y0 + threadIdx.x; t < y1; t += blockDim.x) {
      v[kMaxSpecies].add(S.part_fld[2 * (size_t)t]);
      v[kMaxSpecies + 1].add(S.part_fld[2 * (size_t)t + 1]);
    }
    // all quantities over the CTA at once, in a fixed order: shuffle tree
    // in each warp, then warp 0 over the warp sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < kEndQ; ++k) {
        if (!used(k)) continue;
        CSum u;
        u.s = __shfl_down_sync(0xffffffffu, v[k].s, o);
        u.c = __shfl_down_sync(0xffffffffu, v[k].c, o);
        v[k].add(u);
      }
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < kEndQ; ++k) {
        red[(warp * kEndQ + k) * 2] = v[k].s;
        red[(warp * kEndQ + k) * 2 + 1] = v[k].c;
      }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int k = 0; k < kEndQ; ++k) {
        CSum w;
        if (lane < kWarps) {
          w.s = red[(lane * kEndQ + k) * 2];
          w.c = red[(lane * kEndQ + k) * 2 + 1];
        }
        v[k] = w;
      }
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < kEndQ; ++k) {
          if (!used(k)) continue;
          CSum u;
          u.s = __shfl_down_sync(0xffffffffu, v[k].s, o);
          u.c = __shfl_down_sync(0xffffffffu, v[k].c, o);
          v[k].add(u);
        }
      }
      if (lane == 0) {
        double *slot = S.epart + (size_t)g * kEndQ * 2;
#pragma unroll
        for (int k = 0; k < kEndQ; ++k) {
          slot[2 * k] = v[k].s;
          slot[2 * k + 1] = v[k].c;
        }
        __threadfence();
        s_last = atomicAdd(S.eticket, 1) == G - 1;
      }
    }
    __syncthreads();
    owner = s_last != 0;
    if (owner) {
      // every slice's values, read from L2 by all threads at once; warp w
      // combines quantity k = w, w + kWarps, ... over the slices: lane h
      // adds slices h and h + 32, then a shuffle tree (a fixed order)
      __threadfence();
      for (int k = threadIdx.x; k < G * kEndQ * 2; k += blockDim.x)
        s_part[k] = __ldcg(S.epart + k);
      __syncthreads();
      static_assert(kEndSlicesMax <= 64, "two slices per lane");
      for (int k = warp; k < kEndQ; k += kWarps) {
        CSum q;
        if (used(k)) {
          for (int h = lane; h < G; h += 32) {
            CSum u;
            u.s = s_part[(h * kEndQ + k) * 2];
            u.c = s_part[(h * kEndQ + k) * 2 + 1];
            q.add(u);
          }
          for (int o = 16; o > 0; o >>= 1) {
            CSum u;
            u.s = __shfl_down_sync(0xffffffffu, q.s, o);
            u.c = __shfl_down_sync(0xffffffffu, q.c, o);
            q.add(u);
          }
        }
        if (lane == 0) {
          s_q[2 * k] = q.s;
          s_q[2 * k + 1] = q.c;
        }
      }
      __syncthreads();
    }
    if (owner && threadIdx.x == 0) {
      *S.eticket = 0;  // for the next energy step
      auto total = [&](int k) { return s_q[2 * k] + s_q[2 * k + 1]; };
      const int rec = (step + 1) / S.energy_every - 1 - S.hist_skip;
      const double area = S.dx_d * S.dy_d;
      const double ev = total(kMaxSpecies);
      const double bv = total(kMaxSpecies + 1);
      bool bad = !isfinite(ev) || !isfinite(bv);
      double kin[kMaxSpecies];
      for (int s = 0; s < kMaxSpecies; ++s)
        kin[s] = s < S.nsp ? total(s) * S.sp[s].kin_scale : 0.0;
      if (rec >= 0 && rec < S.hist_cap) {
        zpic_energy_rec &r = S.hist[rec];
        r.step = step + 1;
        r.n_species = S.nsp;
        r.wE = 0.5 * ev * area;
        r.wB = 0.5 * bv * area;
        for (int s = 0; s < kMaxSpecies; ++s) {
          r.kin[s] = kin[s];
          if (s < S.nsp && !isfinite(kin[s])) bad = true;
        }
        *S.hist_n = rec + 1;
      }
      if (bad) {
        atomicOr(&st->error, ERR_NAN);
        atomicMin(&st->err_step, step);
      }
    }
  }
  if (threadIdx.x == 0) {
    if (owner && S.moving_window && shift_due(S, step, *S.n_shift))
      *S.n_shift += 1;
    if (owner && sort_due(S, step)) {
      // the re-sort wrote the other copy of the particle store
      *S.pswap ^= 1;
      *S.sorts += 1;
    }
    __threadfence();
    const int t = atomicAdd(&st->blocks_done, 1);
    if (t == (int)gridDim.x - 1) {
      st->blocks_done = 0;
      st->push_next = 0;  // the next step's push takes items from 0
      __threadfence();
      st->step = step + 1;
    }
  }
}

template <typename R>
cudaError_t launch_end_step(const SimDev<R> *sims, int n_sims, int g_max,
                            BatchStatus *st, cudaStream_t stream) {
  end_step_kernel<R><<<n_sims * g_max, kThreads, 0, stream>>>(sims, g_max,
                                                                st);
  return cudaGetLastError();
}

// ---- field energy of the current fields, on demand ------------------------
//
// One CTA per grid row: sums E^2 and B^2 of the row (FP32/FP64 squares,
// FP64 accumulation, fixed reduction order) and writes the two row sums to
// scratch[2 j], scratch[2 j + 1]; a one-CTA pass adds the rows in order and
// writes 1/2 sum E^2 dx dy and 1/2 sum B^2 dx dy to scratch[2 ny], [2 ny + 1].
// Every scratch value is written before it is read, so the scratch needs no
// clearing between calls.

template <typename R>
__global__ void __launch_bounds__(kThreads)
    field_energy_rows_kernel(FieldPtrs<R> f, int nx, int ld, double *scratch) {
  __shared__ double red[2 * kWarps];
  const size_t row = (size_t)blockIdx.x * ld;
  CSum e, b;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    const R ex = f.e[0][row + i], ey = f.e[1][row + i], ez = f.e[2][row + i];
    const R bx = f.b[0][row + i], by = f.b[1][row + i], bz = f.b[2][row + i];
    e.add((double)ex * ex + (double)ey * ey + (double)ez * ez);
    b.add((double)bx * bx + (double)by * by + (double)bz * bz);
  }
  const double es = block_csum(e, red).value();
  if (threadIdx.x == 0) scratch[2 * (size_t)blockIdx.x] = es;
  const double bs = block_csum(b, red).value();
  if (threadIdx.x == 0) scratch[2 * (size_t)blockIdx.x + 1] = bs;
}

__global__ void __launch_bounds__(kThreads)
    field_energy_final_kernel(double *scratch, int ny, double half_area) {
  __shared__ double red[2 * kWarps];
  CSum es, bs;
  for (int j = threadIdx.x; j < ny; j += blockDim.x) {
    es.add(scratch[2 * (size_t)j]);
    bs.add(scratch[2 * (size_t)j + 1]);
  }
  const double e = block_csum(es, red).value();
  const double b = block_csum(bs, red).value();
  if (threadIdx.x == 0) {
    scratch[2 * (size_t)ny] = half_area * e;
    scratch[2 * (size_t)ny + 1] = half_area * b;
  }
}

template <typename R>
cudaError_t launch_field_energy(FieldPtrs<R> f, int nx, int ny, int ld,
                                double dx, double dy, double *scratch,
                                cudaStream_t stream) {
  if (nx <= 0 || ny <= 0) return cudaErrorInvalidValue;
  field_energy_rows_kernel<R><<<ny, kThreads, 0, stream>>>(f, nx, ld, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  field_energy_final_kernel<<<1, kThreads, 0, stream>>>(scratch, ny,
                                                        0.5 * dx * dy);
  return cudaGetLastError();
}

// ---- laser initialisation ------------------------------------------------

// Gaussian pulse, linear polarisation along y, propagating in +x:
// Ey = E0 exp(-(y-yc)^2/w0^2) exp(-2 ln2 (x-x0)^2/fwhm^2) cos(omega0 (x-x0))
// at the Ey points, and Bz = Ey (a +x wave) at the Bz points.
__device__ __forceinline__ double laser_value(const LaserParams &lp, double X,
                                              double Y) {
  const double dX = X - lp.x0, dY = Y - lp.yc;
  return lp.E0 * exp(-dY * dY / (lp.w0 * lp.w0)) *
         exp(-2.0 * log(2.0) * dX * dX / (lp.fwhm * lp.fwhm)) *
         cos(lp.omega0 * dX);
}

template <typename R>
__global__ void laser_kernel(const SimDev<R> *__restrict__ sim,
                             LaserParams lp) {
  const SimDev<R> &S = *sim;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= S.nx || j >= S.ny) return;
  const double dx = S.dx_d, dy = S.dy_d;
  const size_t k = (size_t)j * S.ld + i;
  S.E[0][1][k] += (R)laser_value(lp, i * dx, (j + 0.5) * dy);
  S.B[0][2][k] += (R)laser_value(lp, (i + 0.5) * dx, (j + 0.5) * dy);
}

template <typename R>
cudaError_t launch_laser(const SimDev<R> *sim_dev, int nx, int ny,
                         LaserParams lp, cudaStream_t stream) {
  dim3 grid((nx + 127) / 128, ny);
  laser_kernel<R><<<grid, 128, 0, stream>>>(sim_dev, lp);
  return cudaGetLastError();
}

#define ZP_INST(R)                                                          \
  template cudaError_t launch_filter<R>(const SimDev<R> *, const int2 *,   \
                                        int, BatchStatus *, cudaStream_t); \
  template cudaError_t launch_yee<R>(const SimDev<R> *, const int2 *, int, \
                                     BatchStatus *, cudaStream_t);          \
  template cudaError_t launch_end_step<R>(const SimDev<R> *, int, int,     \
                                          BatchStatus *, cudaStream_t);     \
  template cudaError_t launch_laser<R>(const SimDev<R> *, int, int,        \
                                       LaserParams, cudaStream_t);          \
  template cudaError_t launch_field_energy<R>(FieldPtrs<R>, int, int, int,  \
                                              double, double, double *,      \
                                              cudaStream_t);
ZP_INST(float)
ZP_INST(double)
#undef ZP_INST

}  // namespace zp
