// k_part.cu -- particle store management: tile migration (the particle
// hand-over between neighbouring regions of Sec. 3.2, at most one cell per
// step so only the 8 neighbour tiles can receive), moving-window injection
// (Sec. 4.1), the initial load, and binning / compaction used by set/get and
// by the overflow re-sort.
#include <math.h>

#include <algorithm>

#include "zpic_dev.cuh"
#include "zpic_kernels.h"

namespace zp {

// ---- migration --------------------------------------------------------------
//
// Two kernels.  migrate_kernel: one warp per tile (four tiles per CTA) reads
// each entry of the tile's outbox once, works out the tile its cell lies in
// (one of the 8 neighbours: particles move at most one cell per step,
// Sec. 3.2) and appends it to that tile's arrivals, behind its stayers: the
// lanes bound for the same tile find each other with __match_any_sync and
// one of them claims their slots with one atomic add on the tile's arrival
// counter.  Tiles in the last column also receive the new plasma column
// when the window shifts, in slots claimed the same way.  Particles that
// find no room go to the overflow buffer and raise ERR_OVERFLOW.
// fold_arrivals_kernel then adds every tile's arrivals to its particle
// count (at most its capacity) and clears the counter.  The order of the
// arrivals within a tile follows the order of the atomic adds; nothing
// computed depends on it (the current is an exact integer sum, and every
// particle is pushed on its own).

template <typename R>
__device__ __forceinline__ void park(OverflowDev<R> &ovf, BatchStatus *st,
                                     int step, int sim, int s, int ix, int iy,
                                     int id, R x, R y, R ux, R uy, R uz, R w) {
  const int o = atomicAdd(&st->ovf_count, 1);
  if (o < ovf.cap) {
    ovf.sim[o] = sim;
    ovf.species[o] = s;
    ovf.ix[o] = ix;
    ovf.iy[o] = iy;
    ovf.id[o] = id;
    ovf.x[o] = x;
    ovf.y[o] = y;
    ovf.ux[o] = ux;
    ovf.uy[o] = uy;
    ovf.uz[o] = uz;
    ovf.w[o] = w;
    atomicOr(&st->error, ERR_OVERFLOW);
  } else {
    atomicAdd(&st->lost, 1);
    atomicOr(&st->error, ERR_LOST);
  }
  atomicMin(&st->err_step, step);
}

template <typename R>
__device__ __forceinline__ double window_density(const SpeciesDev<R> &P,
                                                 double xa) {
  if (xa < P.ramp_x0) return 0.0;
  if (P.ramp_len > 0.0 && xa < P.ramp_x0 + P.ramp_len)
    return P.n0 * (xa - P.ramp_x0) / P.ramp_len;
  return P.n0;
}

// One outbox entry in registers: loaded from the tile's outbox, stored to
// slot d of the destination tile's segment (or parked in the overflow
// buffer when d is beyond the tile's capacity).
template <typename R>
struct OutboxEntry {
  int ix = 0, iy = 0, id = 0;
  R x = R(0), y = R(0), ux = R(0), uy = R(0), uz = R(0), w = R(1);
  __device__ __forceinline__ void load(const SpeciesDev<R> &P, size_t e,
                                       bool has_w, bool has_id) {
    ix = P.ob_ix[e];
    iy = P.ob_iy[e];
    x = P.ob_x[e];
    y = P.ob_y[e];
    ux = P.ob_ux[e];
    uy = P.ob_uy[e];
    uz = P.ob_uz[e];
    if (has_w) w = P.ob_w[e];
    if (has_id) id = P.ob_id[e];
  }
  __device__ __forceinline__ void store(const Planes<R> &O,
                                        const SpeciesDev<R> &P,
                                        OverflowDev<R> &ovf,
                                        BatchStatus *st, int step, int sim,
                                        int s, int dest, int ntx, int tx,
                                        int ty, int d, int cap, int off,
                                        bool has_w, bool has_id) const {
    if (d < cap) {
      const size_t t = (size_t)off + d;
      const int dx0 = (dest % ntx) * tx, dy0 = (dest / ntx) * ty;
      O.cell[t] = local_cell(ix - dx0, iy - dy0);
      O.x[t] = x;
      O.y[t] = y;
      O.ux[t] = ux;
      O.uy[t] = uy;
      O.uz[t] = uz;
      if (has_w) O.w[t] = w;
      if (has_id) O.id[t] = id;
    } else {
      park(ovf, st, step, sim, s, ix, iy, id, x, y, ux, uy, uz, w);
    }
  }
};

constexpr int kPT_MIG = 128;
constexpr int kWarpsMig = kPT_MIG / 32;  // tiles per CTA

// Exclusive prefix sum of v over the CTA (NT threads); total = sum.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int *wsum,
                                                    int &total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < NW ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int before = warp > 0 ? wsum[warp - 1] : 0;
  total = wsum[NW - 1];
  __syncthreads();  // wsum is reused by the next call
  return before + x - v;
}

template <typename R>
__global__ void __launch_bounds__(kPT_MIG)
    migrate_kernel(const SimDev<R> *__restrict__ sims,
                   const int2 *__restrict__ items, int n_items,
                   BatchStatus *st, OverflowDev<R> ovf) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int item = blockIdx.x * kWarpsMig + (threadIdx.x >> 5);
  if (item >= n_items) return;  // warps work alone: no block barrier
  const int step = st->step;
  if (frozen(st, step)) return;
  const int2 it = items[item];
  const SimDev<R> &S = sims[it.x];
  const int tile = it.y;
  const int tx = S.tx, ty = S.ty, ntx = S.ntx;
  const int x0 = (tile % ntx) * tx, y0 = (tile / ntx) * ty;
  const int tw = min(tx, S.nx - x0), th = min(ty, S.ny - y0);
  const int nsh = S.moving_window ? *S.n_shift : 0;
  const bool inject_col = shift_due(S, step, nsh) && (x0 + tw == S.nx);
  // the copy the push kernel just wrote
  const int nxt = ((step + 1) & 1) ^ *S.pswap;
  for (int s = 0; s < S.nsp; ++s) {
    const SpeciesDev<R> &P = S.sp[s];
    const Planes<R> &O = P.buf[nxt];
    const bool has_w = O.w != nullptr, has_id = O.id != nullptr;
    const int n_out = P.ob_cnt[tile];
    const size_t ob0 = (size_t)tile * P.ob_cap;
    // one group of 32 entries per pass; the next group's entries are loaded
    // while this one claims its slots, and the destination's count,
    // capacity and offset (which no lane changes here) before the claim, so
    // a pass waits for about one memory round trip
    OutboxEntry<R> cur;
    bool mine = lane < n_out;
    if (mine) cur.load(P, ob0 + lane, has_w, has_id);
    for (int k0 = 0; k0 < n_out; k0 += 32) {
      OutboxEntry<R> nxt;
      const bool mine_n = k0 + 32 + lane < n_out;
      if (mine_n) nxt.load(P, ob0 + k0 + 32 + lane, has_w, has_id);
      const int ix = cur.ix, iy = cur.iy;
      const int dest = mine ? (iy / ty) * ntx + ix / tx : 0;
      int cnt_d = 0, cap_d = 0, off_d = 0;
      if (mine) {
        cnt_d = P.cnt[dest];
        cap_d = P.cap[dest];
        off_d = P.off[dest];
      }
      // lanes without an entry get keys of their own
      const unsigned peers = __match_any_sync(kAll, mine ? dest : -1 - lane);
      if (mine) {
        const int leader = __ffs(peers) - 1;
        int slot = 0;
        if (lane == leader) slot = atomicAdd(P.arr + dest, __popc(peers));
        slot = __shfl_sync(peers, slot, leader) + __popc(peers & lt);
        cur.store(O, P, ovf, st, step, it.x, s, dest, ntx, tx, ty,
                  cnt_d + slot, cap_d, off_d, has_w, has_id);
      }
      cur = nxt;
      mine = mine_n;
    }
    // moving window: cold plasma on a lattice enters through column nx-1
    if (inject_col && P.inj_ppc_x > 0) {
      const int ppx = P.inj_ppc_x, ppc = ppx * P.inj_ppc_y;
      const int i = S.nx - 1;
      const double xa = (i + nsh + 1 + 0.5) * S.dx_d;  // lab frame
      const double dens = window_density(P, xa);
      if (dens > 0.0) {
        const int total = th * ppc;
        int s0 = 0;
        if (lane == 0) s0 = atomicAdd(P.arr + tile, total);
        s0 = __shfl_sync(kAll, s0, 0);
        const int n_stay = P.cnt[tile], cap = P.cap[tile];
        const size_t base = (size_t)P.off[tile];
        for (int k = lane; k < total; k += 32) {
          const int j = y0 + k / ppc, kk = k % ppc;
          const int kx = kk % ppx, ky = kk / ppx;
          const R px = (R)((kx + 0.5) / ppx);
          const R py = (R)((ky + 0.5) / P.inj_ppc_y);
          const int pid =
              (int)(P.id_base + ((long long)nsh * S.ny + j) * ppc + kk);
          const int d = n_stay + s0 + k;
          if (d < cap) {
            const size_t t = base + d;
            O.cell[t] = local_cell(i - x0, j - y0);
            O.x[t] = px;
            O.y[t] = py;
            O.ux[t] = R(0);
            O.uy[t] = R(0);
            O.uz[t] = R(0);
            if (has_w) O.w[t] = (R)dens;
            if (has_id) O.id[t] = pid;
          } else {
            park(ovf, st, step, it.x, s, i, j, pid, px, py, R(0), R(0), R(0),
                 (R)dens);
          }
        }
      }
    }
  }
}

// Every tile's arrivals join its particle count (those beyond its capacity
// went to the overflow buffer), and the arrival counters start the next
// step at zero.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    fold_arrivals_kernel(const SimDev<R> *__restrict__ sims,
                         const int2 *__restrict__ items, int n_items,
                         BatchStatus *st) {
  const int step = st->step;
  if (frozen(st, step)) return;
  const long long n = (long long)n_items * kMaxSpecies;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q / kMaxSpecies), s = (int)(q - (long long)i * kMaxSpecies);
    const int2 it = items[i];
    const SimDev<R> &S = sims[it.x];
    if (s >= S.nsp) continue;
    const SpeciesDev<R> &P = S.sp[s];
    const int a = P.arr[it.y];
    if (a != 0) {
      P.cnt[it.y] = min(P.cnt[it.y] + a, P.cap[it.y]);
      P.arr[it.y] = 0;
    }
  }
}

template <typename R>
cudaError_t launch_migrate(const SimDev<R> *sims, const int2 *items,
                           int n_items, BatchStatus *st,
                           const OverflowDev<R> &ovf, cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  migrate_kernel<R><<<(n_items + kWarpsMig - 1) / kWarpsMig, kPT_MIG, 0,
                      stream>>>(sims, items, n_items, st, ovf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)n_items * kMaxSpecies;
  const int grid = (int)std::min<long long>((n + kThreads - 1) / kThreads,
                                            152 * 8);
  fold_arrivals_kernel<R><<<grid, kThreads, 0, stream>>>(sims, items, n_items,
                                                          st);
  return cudaGetLastError();
}

// ---- initial load -------------------------------------------------------
//
// One CTA per tile.  The tile's loaded cells are the columns
// [max(x0, col_lo), min(x0+tw, col_hi)) x all its rows; its segment holds
// ppc particles per loaded cell in k-major order (particle q -> k = q / nc,
// local cell q % nc) so neighbouring particles sit in different cells.
// Draw d of particle (cell c, k) is output (c*ppc + k)*8 + d + 1 of the
// SplitMix64 stream `key`: d = 0, 1 offsets, 2..5 Box-Muller normals.

__device__ __forceinline__ double unit53(uint64_t z) {
  return (double)(z >> 11) * 0x1.0p-53;
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    init_load_kernel(const SimDev<R> *__restrict__ sim, LoadParams lp) {
  const SimDev<R> &S = *sim;
  const SpeciesDev<R> &P = S.sp[lp.species];
  const Planes<R> &O = P.buf[lp.buf];
  const int tile = blockIdx.x;
  const int tcx = tile % S.ntx, tcy = tile / S.ntx;
  const int x0 = tcx * S.tx, y0 = tcy * S.ty;
  const int tw = min(S.tx, S.nx - x0), th = min(S.ty, S.ny - y0);
  const int ca = max(x0, lp.col_lo), cb = min(x0 + tw, lp.col_hi);
  if (cb <= ca) return;
  const int nca = cb - ca, nc = nca * th;
  const int ppc = lp.ppc_x * lp.ppc_y;
  const size_t base = (size_t)P.off[tile];
  const bool thermal = lp.u_th[0] != 0.0 || lp.u_th[1] != 0.0 || lp.u_th[2] != 0.0;
  const int total = nc * ppc;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int k = q / nc, lc = q - k * nc;
    const int ix = ca + lc % nca, iy = y0 + lc / nca;
    const long long c = (long long)iy * S.nx + ix;
    const uint64_t ctr = ((uint64_t)c * ppc + k) * 8ull;
    double x, y;
    if (lp.lattice) {
      x = (k % lp.ppc_x + 0.5) / lp.ppc_x;
      y = (k / lp.ppc_x + 0.5) / lp.ppc_y;
    } else {
      x = (double)(sm_out(lp.key, ctr + 1) >> 40) * 0x1.0p-24;
      y = (double)(sm_out(lp.key, ctr + 2) >> 40) * 0x1.0p-24;
    }
    double u[3] = {lp.u_fl[0], lp.u_fl[1], lp.u_fl[2]};
    if (thermal) {
      double nrm[3];
      for (int pr = 0; pr < 2; ++pr) {
        const double u1 =
            ((double)(sm_out(lp.key, ctr + 3 + 2 * pr) >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = unit53(sm_out(lp.key, ctr + 4 + 2 * pr));
        const double r = sqrt(-2.0 * log(u1));
        const double a = 2.0 * M_PI * u2;
        nrm[2 * pr] = r * cos(a);
        if (pr == 0) nrm[1] = r * sin(a);
      }
      for (int a = 0; a < 3; ++a) u[a] += lp.u_th[a] * nrm[a];
    }
    double w = lp.n0;
    if (lp.profile == ZPIC_PROFILE_RAMP) {
      const double xc = (ix + 0.5) * S.dx_d;
      w = xc < lp.x0 + lp.x1 ? lp.n0 * (xc - lp.x0) / lp.x1 : lp.n0;
    }
    const size_t t = base + q;
    O.cell[t] = local_cell(ix - x0, iy - y0);
    O.x[t] = (R)x;
    O.y[t] = (R)y;
    O.ux[t] = (R)u[0];
    O.uy[t] = (R)u[1];
    O.uz[t] = (R)u[2];
    if (O.w) O.w[t] = (R)w;
    if (O.id) O.id[t] = (int)(c * ppc + k);
  }
}

template <typename R>
cudaError_t launch_init_load(const SimDev<R> *sim_dev, int ntiles,
                             LoadParams lp, cudaStream_t stream) {
  if (ntiles == 0) return cudaSuccess;
  init_load_kernel<R><<<ntiles, kThreads, 0, stream>>>(sim_dev, lp);
  return cudaGetLastError();
}

// ---- cell-order re-sort ----------------------------------------------------
//
// Every sort_every steps, after the migration, each tile's particles are
// rewritten into the other copy of the store in cell-interleaved order: the
// first particle of every cell (cells in row-major order within the tile),
// then the second of every cell that holds two or more, and so on.  Thirty-
// two neighbouring slots then hold particles of thirty-two different,
// neighbouring cells, whose coefficient gathers and current atomics in the
// particle kernel fall on different shared-memory banks; that kernel keeps
// the store order from step to step and the order erodes only as particles
// drift between cells.  The end-of-step kernel then makes the sorted copy
// the current one.
//
// Per tile and species: a histogram of the cells; for every rank r a bit
// mask of the cells that hold more than r particles, with prefix counts of
// its 32-cell words; a particle of cell c that takes rank r (in the order
// the slots are read) goes to slot T(r) + (cells before c that hold more
// than r particles), T(r) being the number of particles of rank below r.
// A species of a tile with at most kSortStaged<R> particles is moved plane
// by plane through shared memory: its cells and the permutation (which
// input slot each output slot takes) stay there, each plane arrives by one
// bulk asynchronous copy and is written out in slot order, so every global
// access is coalesced whatever the permutation.  The first plane's copy
// runs while the rank tables are built, and each later one while the plane
// before it is written out (into a second buffer laid over the tables and
// the cells, when a plane fits there: always in FP32).  The particles of
// one cell then take their ranks in any order.  Larger ones are moved
// particle by particle, kSortU chunks of slots per memory round trip, the
// chunks taking their ranks one after the other so that a store close to
// the sorted order is rewritten in long runs.  A tile whose rank table
// exceeds the shared-memory budget keeps its order.
constexpr int kSortThreads = 512;
constexpr int kSortMaxCells = 1024;   // tiles up to 32 x 32
constexpr int kSortMaskWords = 6144;  // ranks x 32-cell words
constexpr int kSortMaxRank = 2048;
constexpr int kSortU = 4;             // chunks of slots per memory round trip
// particles of one species and tile that the staged path takes
template <typename R>
constexpr int kSortStaged = sizeof(R) == 4 ? 20480 : 13312;

__host__ __device__ constexpr size_t sort_tables_bytes() {
  return ((2 * (size_t)kSortMaskWords + kSortMaxRank + 1) * sizeof(unsigned) +
          15) & ~size_t(15);
}
template <typename R>
size_t sort_smem_bytes() {
  // tables, then cells and permutation (16-bit slots), then one plane (the
  // second plane buffer lies over the tables and the cells)
  return sort_tables_bytes() + 4 * (size_t)kSortStaged<R> +
         sizeof(R) * (size_t)kSortStaged<R>;
}

// Bulk asynchronous copies into shared memory, completed on an mbarrier.
// Addresses are 16-byte aligned (segments start at multiples of 32
// particles, planes at 256-byte boundaries) and sizes multiples of 16.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb))
               : "memory");
}
// the calling thread's arrival, expecting `bytes`, then the copy (if any)
__device__ __forceinline__ void bulk_load(void *dst, const void *src,
                                          unsigned bytes,
                                          unsigned long long *mb) {
  // shared memory that threads have read is written by the async proxy next
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_addr(mb)),
      "r"(bytes)
      : "memory");
  if (bytes)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mb))
        : "memory");
}
// Wait for phase `parity` of mb to complete; false if it did not within
// the iteration limit.
constexpr int kBulkWaitLimit = 1 << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long *mb,
                                          unsigned parity) {
  const unsigned a = smem_addr(mb);
  for (int i = 0; i < kBulkWaitLimit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred q;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
        " selp.u32 %0, 1, 0, q;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Plane k of a species' copy (x, y, ux, uy, uz, then w and id if present):
// its address and element size.
template <typename R>
__device__ __forceinline__ int sort_plane_ptr(const Planes<R> &P, int k,
                                              const void *&src) {
  switch (k) {
    case 0: src = P.x; return (int)sizeof(R);
    case 1: src = P.y; return (int)sizeof(R);
    case 2: src = P.ux; return (int)sizeof(R);
    case 3: src = P.uy; return (int)sizeof(R);
    case 4: src = P.uz; return (int)sizeof(R);
    default:
      if (k == 5 && P.w) { src = P.w; return (int)sizeof(R); }
      src = P.id;
      return 4;
  }
}

// dst[d] = buf[pinv[d]] for every output slot d of a plane
template <typename T>
__device__ __forceinline__ void sort_gather(T *__restrict__ dst,
                                            const T *buf,
                                            const uint16_t *pinv, int n) {
#pragma unroll 4
  for (int d = threadIdx.x; d < n; d += blockDim.x)
    __stcs(dst + d, buf[pinv[d]]);
}

template <typename R>
__global__ void __launch_bounds__(kSortThreads, 1)
    sort_tiles_kernel(const SimDev<R> *__restrict__ sims,
                      int n_sims, const int2 *__restrict__ items,
                      int n_items, BatchStatus *st) {
  __shared__ int hist[kSortMaxCells];  // cell counts, then rank cursors
  __shared__ int wsum[kSortThreads / 32];
  __shared__ int s_max;
  extern __shared__ __align__(16) unsigned sort_smem[];
  unsigned *mask = sort_smem;
  unsigned *pre = sort_smem + kSortMaskWords;
  int *T = reinterpret_cast<int *>(sort_smem + 2 * kSortMaskWords);
  constexpr int NS = kSortStaged<R>;
  unsigned char *stage =
      reinterpret_cast<unsigned char *>(sort_smem) + sort_tables_bytes();
  uint16_t *cells_s = reinterpret_cast<uint16_t *>(stage);
  uint16_t *pinv = cells_s + NS;
  // plane buffers: buf0 after the permutation; buf1 over the tables and
  // the cells, which are no longer needed once the permutation is built
  unsigned char *const buf0 = stage + 4 * (size_t)NS;
  unsigned char *const buf1 = reinterpret_cast<unsigned char *>(sort_smem);
  constexpr size_t kBuf1Bytes = sort_tables_bytes() + 2 * (size_t)NS;
  // mbarriers: the cell copy, then one per plane buffer; ph bit i = the
  // parity of mb[i]'s next phase, pend bit i = a copy on mb[i] not waited for
  __shared__ unsigned long long mb[3];
  unsigned ph = 0, pend = 0;
  const int step = st->step;
  if (frozen(st, step)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = kSortThreads / 32;
  // most steps re-sort nothing: leave at once unless some simulation is due
  {
    bool due = false;
    for (int i = threadIdx.x; i < n_sims && !due; i += blockDim.x)
      due = sort_due(sims[i], step);
    if (!__syncthreads_or(due)) return;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&mb[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // copy `bytes` from src into dst on mb[i] (thread 0 issues it; every
  // thread records it)
  auto start_copy = [&](int i, void *dst, const void *src, unsigned bytes) {
    if (threadIdx.x == 0) bulk_load(dst, src, bytes, &mb[i]);
    pend |= 1u << i;
  };
  // wait for the copy on mb[i] and make it (and every thread's plain stores
  // before the call) visible to the CTA.  A copy that does not complete
  // in time is recorded, the copies in flight get one more bounded wait,
  // and every thread leaves (false).
  auto finish_copy = [&](int i) {
    const bool ok = mbar_wait(&mb[i], (ph >> i) & 1u);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&st->error, ERR_TIMEOUT);
        atomicMin(&st->err_step, step);
        for (int j = 0; j < 3; ++j)
          if ((pend >> j) & 1u) mbar_wait(&mb[j], (ph >> j) & 1u);
      }
      return false;
    }
    ph ^= 1u << i;
    pend &= ~(1u << i);
    return true;
  };
  // plane k of a copy of the store at the segment start, its element size,
  // and the bytes of its 16-byte multiple that a bulk copy takes
  auto plane_at = [&](const Planes<R> &Q, int k, size_t base, int n,
                      const char *&ptr, unsigned &bulk) {
    const void *p0;
    const int es = sort_plane_ptr(Q, k, p0);
    ptr = (const char *)p0 + base * es;
    bulk = (unsigned)(n & ~(16 / es - 1)) * es;
    return es;
  };
  for (int ii = blockIdx.x; ii < n_items; ii += gridDim.x) {
    const int2 it = items[ii];
    const SimDev<R> &S = sims[it.x];
    if (!sort_due(S, step)) continue;
    const int tile = it.y;
    const int tcx = tile % S.ntx, tcy = tile / S.ntx;
    const int tw = min(S.tx, S.nx - tcx * S.tx);
    const int th = min(S.ty, S.ny - tcy * S.ty);
    const int nc = tw * th;
    const int W = (nc + 31) >> 5;
    // the copy the push and the migration of this step wrote
    const int src = ((step + 1) & 1) ^ *S.pswap;
    for (int s = 0; s < S.nsp; ++s) {
      const SpeciesDev<R> &P = S.sp[s];
      const Planes<R> &I = P.buf[src];
      const Planes<R> &O = P.buf[src ^ 1];
      const int n = P.cnt[tile];
      const size_t base = (size_t)P.off[tile];
      for (int c = threadIdx.x; c < nc; c += blockDim.x) hist[c] = 0;
      if (threadIdx.x == 0) s_max = 0;
      __syncthreads();
      const bool staged = n <= NS;
      const int np = 5 + (I.w ? 1 : 0) + (I.id ? 1 : 0);
      // two plane buffers when a plane fits over the tables and the cells
      const bool dbl = (size_t)n * sizeof(R) <= kBuf1Bytes;
      if (staged) {
        // the cells, and the first plane while the tables are built
        const char *p0;
        unsigned b0;
        plane_at(I, 0, base, n, p0, b0);
        start_copy(0, cells_s, I.cell + base, (unsigned)(n & ~7) * 2u);
        start_copy(1, buf0, p0, b0);
        for (int p = (n & ~7) + threadIdx.x; p < n; p += blockDim.x)
          cells_s[p] = I.cell[base + p];
        if (!finish_copy(0)) return;
#pragma unroll 4
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          const int lc = cells_s[p];
          atomicAdd(&hist[(lc >> 8) * tw + (lc & 255)], 1);
        }
      } else {
#pragma unroll 4
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          const int lc = I.cell[base + p];
          atomicAdd(&hist[(lc >> 8) * tw + (lc & 255)], 1);
        }
      }
      __syncthreads();
      int m = 0;
      for (int c = threadIdx.x; c < nc; c += blockDim.x) m = max(m, hist[c]);
      for (int o = 16; o > 0; o >>= 1)
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(&s_max, m);
      __syncthreads();
      const int maxc = s_max;
      const bool fits = maxc <= kSortMaxRank &&
                        (long long)maxc * W <= kSortMaskWords;
      if (fits) {
        // bit masks: word (r, j) has bit i set when cell 32 j + i holds
        // more than r particles
        for (int q = warp; q < maxc * W; q += NW) {
          const int r = q / W, c = (q - r * W) * 32 + lane;
          const unsigned b =
              __ballot_sync(0xffffffffu, c < nc && hist[c] > r);
          if (lane == 0) mask[q] = b;
        }
        __syncthreads();
        // prefix counts of the words of each rank (one warp per rank,
        // W <= 32 words), and N(r) = the cells with more than r particles
        for (int r = warp; r < maxc; r += NW) {
          const int v = lane < W ? __popc(mask[r * W + lane]) : 0;
          int x = v;
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
          }
          if (lane < W) pre[r * W + lane] = (unsigned)(x - v);
          if (lane == 31) T[r] = x;
        }
        __syncthreads();
        // T(r) = particles of rank below r: exclusive scan of N over r
        int carry = 0;
        for (int r0 = 0; r0 < maxc; r0 += kSortThreads) {
          const int r = r0 + threadIdx.x;
          const int v = r < maxc ? T[r] : 0;
          int total;
          const int e = block_exclusive_scan<kSortThreads>(v, wsum, total);
          if (r < maxc) T[r] = carry + e;
          carry += total;
        }
      }
      for (int c = threadIdx.x; c < nc; c += blockDim.x) hist[c] = 0;
      __syncthreads();
      if (staged && !fits) {
        // the first plane's copy is not used: let it land before the
        // particle-by-particle path
        if (!finish_copy(1)) return;
      }
      if (fits && staged) {
        // output slot d takes input slot pinv[d]
#pragma unroll 4
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
          const int lc = cells_s[p];
          const int li = (lc >> 8) * tw + (lc & 255);
          const int r = atomicAdd(&hist[li], 1);
          const int wd = r * W + (li >> 5);
          const int d = T[r] + (int)pre[wd] +
                        __popc(mask[wd] & ((1u << (li & 31)) - 1u));
          pinv[d] = (uint16_t)p;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < n; d += blockDim.x)
          O.cell[base + d] = cells_s[pinv[d]];
        const int nb = dbl ? 2 : 1;
        if (dbl && np > 1) {
          __syncthreads();  // the tables and the cells are read
          const char *p1;
          unsigned b1;
          plane_at(I, 1, base, n, p1, b1);
          start_copy(2, buf1, p1, b1);
        }
        // plane k lands in buf0 (k even, or one buffer) or buf1; while it is
        // written out, plane k + 1 is on its way into the other one
        for (int k = 0; k < np; ++k) {
          const int b = nb == 2 ? (k & 1) : 0;
          unsigned char *bk = b ? buf1 : buf0;
          const char *sp;
          unsigned bulk;
          const int es = plane_at(I, k, base, n, sp, bulk);
          const char *dq;
          unsigned dbulk;
          plane_at(O, k, base, n, dq, dbulk);
          char *dp = const_cast<char *>(dq);
          // the ragged end of the plane with plain loads
          for (int p = (int)(bulk / es) + threadIdx.x; p < n; p += blockDim.x) {
            if (es == 8)
              reinterpret_cast<unsigned long long *>(bk)[p] =
                  reinterpret_cast<const unsigned long long *>(sp)[p];
            else
              reinterpret_cast<unsigned *>(bk)[p] =
                  reinterpret_cast<const unsigned *>(sp)[p];
          }
          if (!finish_copy(1 + b)) return;
          if (es == 8)
            sort_gather(reinterpret_cast<unsigned long long *>(dp),
                        reinterpret_cast<const unsigned long long *>(bk),
                        pinv, n);
          else
            sort_gather(reinterpret_cast<unsigned *>(dp),
                        reinterpret_cast<const unsigned *>(bk), pinv, n);
          __syncthreads();  // bk is read: plane k + nb may land there
          if (k + nb < np) {
            const char *pn;
            unsigned bn;
            plane_at(I, k + nb, base, n, pn, bn);
            start_copy(1 + b, bk, pn, bn);
          }
        }
        continue;
      }
      // kSortU chunks of slots per round trip: every thread loads its
      // particle of each chunk first, then the chunks take their ranks one
      // after the other
      constexpr int U = sizeof(R) == 4 ? kSortU : 2;
      for (int p0 = 0; p0 < n; p0 += U * kSortThreads) {
        int lc[U];
        R x[U], y[U], ux[U], uy[U], uz[U], w[U];
        int id[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int p = p0 + k * kSortThreads + threadIdx.x;
          if (p < n) {
            const size_t q = base + p;
            lc[k] = I.cell[q];
            x[k] = I.x[q];
            y[k] = I.y[q];
            ux[k] = I.ux[q];
            uy[k] = I.uy[q];
            uz[k] = I.uz[q];
            w[k] = I.w ? I.w[q] : R(1);
            id[k] = I.id ? I.id[q] : 0;
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int p = p0 + k * kSortThreads + threadIdx.x;
          if (p < n) {
            int d = p;
            if (fits) {
              const int li = (lc[k] >> 8) * tw + (lc[k] & 255);
              const int r = atomicAdd(&hist[li], 1);
              const int wd = r * W + (li >> 5);
              d = T[r] + (int)pre[wd] +
                  __popc(mask[wd] & ((1u << (li & 31)) - 1u));
            }
            const size_t t = base + d;
            O.cell[t] = (uint16_t)lc[k];
            O.x[t] = x[k];
            O.y[t] = y[k];
            O.ux[t] = ux[k];
            O.uy[t] = uy[k];
            O.uz[t] = uz[k];
            if (I.w) O.w[t] = w[k];
            if (I.id) O.id[t] = id[k];
          }
          __syncthreads();  // this chunk's ranks before the next chunk's
        }
      }
    }
  }
}

template <typename R>
cudaError_t prepare_sort_tiles() {
  return cudaFuncSetAttribute(sort_tiles_kernel<R>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sort_smem_bytes<R>());
}

template <typename R>
cudaError_t launch_sort_tiles(const SimDev<R> *sims, int n_sims,
                              const int2 *items, int n_items, BatchStatus *st,
                              cudaStream_t stream) {
  if (n_items == 0) return cudaSuccess;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess)
    sms = 148;
  const int grid = n_items < sms ? n_items : sms;
  sort_tiles_kernel<R><<<grid, kSortThreads, sort_smem_bytes<R>(), stream>>>(
      sims, n_sims, items, n_items, st);
  return cudaGetLastError();
}

template cudaError_t prepare_sort_tiles<float>();
template cudaError_t prepare_sort_tiles<double>();
template cudaError_t launch_sort_tiles<float>(const SimDev<float> *, int,
                                              const int2 *, int,
                                              BatchStatus *, cudaStream_t);
template cudaError_t launch_sort_tiles<double>(const SimDev<double> *, int,
                                               const int2 *, int,
                                               BatchStatus *, cudaStream_t);

// ---- binning ---------------------------------------------------------------

// Both binning kernels walk the particles warp by warp (lane l takes
// particle base + l) and add to a tile's counter once per warp and tile: the
// lanes holding the same tile find each other with __match_any_sync, the
// first of them adds their number, and each takes its rank among them.  A
// tile-ordered input (what get_particles returns) thus costs one atomic per
// warp instead of 32 on the same address.
__device__ __forceinline__ unsigned lanes_before() {
  return (1u << (threadIdx.x & 31)) - 1u;
}

template <typename R>
__global__ void bin_count_kernel(Staging<R> in, long long n, int nx, int ny,
                                 int tx, int ty, int ntx, int *counts,
                                 int *bad) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane);
       base < n; base += stride) {
    const long long p = base + lane;
    int t = -1;
    if (p < n) {
      const int ix = in.ix[p], iy = in.iy[p];
      const R x = in.x[p], y = in.y[p];
      const bool ok = ix >= 0 && ix < nx && iy >= 0 && iy < ny &&
                      x >= R(0) && x < R(1) && y >= R(0) && y < R(1);
      if (ok) {
        t = (iy / ty) * ntx + ix / tx;
      } else {
        atomicAdd(bad, 1);
      }
      in.tile[p] = t;
    }
    // lanes without a tile get keys of their own
    const unsigned peers = __match_any_sync(0xffffffffu, t >= 0 ? t : -1 - lane);
    if (t >= 0 && lane == __ffs(peers) - 1) atomicAdd(&counts[t], __popc(peers));
  }
}

template <typename R>
cudaError_t launch_bin_count(Staging<R> in, long long n, int nx, int ny,
                             int tx, int ty, int ntx, int *counts, int *bad,
                             cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)((n + kThreads - 1) / kThreads < 152 * 16
                             ? (n + kThreads - 1) / kThreads
                             : 152 * 16);
  bin_count_kernel<R><<<grid, kThreads, 0, stream>>>(in, n, nx, ny, tx, ty,
                                                     ntx, counts, bad);
  return cudaGetLastError();
}

template <typename R>
__global__ void bin_scatter_kernel(Staging<R> in, long long n, SpeciesDev<R> P,
                                   int b, int tx, int ty, int has_w,
                                   int has_id) {
  const Planes<R> &O = P.buf[b];
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane);
       base < n; base += stride) {
    const long long p = base + lane;
    const int t = p < n ? in.tile[p] : -1;
    // the record, loaded before the slot is known
    int ix = 0, iy = 0, id = 0;
    R x = R(0), y = R(0), ux = R(0), uy = R(0), uz = R(0), w = R(1);
    if (t >= 0) {
      ix = in.ix[p];
      iy = in.iy[p];
      x = in.x[p];
      y = in.y[p];
      ux = in.ux[p];
      uy = in.uy[p];
      uz = in.uz[p];
      if (has_w) w = in.w[p];
      id = has_id ? in.id[p] : (int)p;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, t >= 0 ? t : -1 - lane);
    if (t < 0) continue;
    const int leader = __ffs(peers) - 1;
    int slot = 0;
    if (lane == leader) slot = atomicAdd(&P.cnt[t], __popc(peers));
    slot = __shfl_sync(peers, slot, leader) + __popc(peers & lanes_before());
    const size_t d = (size_t)P.off[t] + slot;
    O.cell[d] = local_cell(ix % tx, iy % ty);
    O.x[d] = x;
    O.y[d] = y;
    O.ux[d] = ux;
    O.uy[d] = uy;
    O.uz[d] = uz;
    if (O.w) O.w[d] = w;
    if (O.id) O.id[d] = id;
  }
}

template <typename R>
cudaError_t launch_bin_scatter(Staging<R> in, long long n, SpeciesDev<R> sp,
                               int b, int tx, int ty, int has_w, int has_id,
                               cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)((n + kThreads - 1) / kThreads < 152 * 16
                             ? (n + kThreads - 1) / kThreads
                             : 152 * 16);
  bin_scatter_kernel<R><<<grid, kThreads, 0, stream>>>(in, n, sp, b, tx, ty,
                                                       has_w, has_id);
  return cudaGetLastError();
}

// ---- compaction to a contiguous copy ---------------------------------------

template <typename R>
__global__ void __launch_bounds__(kThreads)
    compact_kernel(SpeciesDev<R> P, int b, int tx, int ty, int ntx, int tile0,
                   const long long *dst_off, Staging<R> out) {
  const Planes<R> &I = P.buf[b];
  const int t = tile0 + blockIdx.x;
  const int x0 = (t % ntx) * tx, y0 = (t / ntx) * ty;
  const int n = P.cnt[t];
  const size_t src = (size_t)P.off[t];
  const size_t dst = (size_t)dst_off[blockIdx.x];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int c = I.cell[src + k];
    out.ix[dst + k] = x0 + (c & 255);
    out.iy[dst + k] = y0 + (c >> 8);
    out.x[dst + k] = I.x[src + k];
    out.y[dst + k] = I.y[src + k];
    out.ux[dst + k] = I.ux[src + k];
    out.uy[dst + k] = I.uy[src + k];
    out.uz[dst + k] = I.uz[src + k];
    out.w[dst + k] = I.w ? I.w[src + k] : R(1);
    out.id[dst + k] = I.id ? I.id[src + k] : 0;
  }
}

template <typename R>
cudaError_t launch_compact(SpeciesDev<R> sp, int b, int tx, int ty, int ntx,
                           int tile0, int ntiles, const long long *dst_off,
                           Staging<R> out, cudaStream_t stream) {
  if (ntiles == 0) return cudaSuccess;
  compact_kernel<R><<<ntiles, kThreads, 0, stream>>>(sp, b, tx, ty, ntx, tile0,
                                                     dst_off, out);
  return cudaGetLastError();
}

// Phase-space density of one species (diagnostic report): every particle
// adds |q0| w to the bin (bx, by) of two of its quantities (global position
// in cells ix + x, iy + y, or a momentum component), b = floor((v - lo) *
// nb / (hi - lo)) evaluated in double, kept when 0 <= b < nb.  One CTA per
// tile, double atomics into hist (nby rows of nbx).
template <typename R>
__device__ __forceinline__ double ps_value(int q, int gx, int gy, R x, R y,
                                           R ux, R uy, R uz) {
  switch (q) {
    case ZPIC_PS_X: return (double)gx + (double)x;
    case ZPIC_PS_Y: return (double)gy + (double)y;
    case ZPIC_PS_UX: return (double)ux;
    case ZPIC_PS_UY: return (double)uy;
    default: return (double)uz;
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    phasespace_kernel(SpeciesDev<R> P, int b, int tx, int ty, int ntx,
                      PhaseSpaceSpec ps, double *hist) {
  const Planes<R> &I = P.buf[b];
  const int t = blockIdx.x;
  const int x0 = (t % ntx) * tx, y0 = (t / ntx) * ty;
  const int n = P.cnt[t];
  const size_t src = (size_t)P.off[t];
  const double q0 = ps.q0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int c = I.cell[src + k];
    const int gx = x0 + (c & 255), gy = y0 + (c >> 8);
    const R x = I.x[src + k], y = I.y[src + k];
    const R ux = I.ux[src + k], uy = I.uy[src + k], uz = I.uz[src + k];
    const double tx_ = (ps_value(ps.qx, gx, gy, x, y, ux, uy, uz) - ps.lo[0]) *
                       ps.scale[0];
    const double ty_ = (ps_value(ps.qy, gx, gy, x, y, ux, uy, uz) - ps.lo[1]) *
                       ps.scale[1];
    if (!(tx_ >= 0.0 && tx_ < (double)ps.nbx)) continue;
    if (!(ty_ >= 0.0 && ty_ < (double)ps.nby)) continue;
    const double w = I.w ? (double)I.w[src + k] : 1.0;
    atomicAdd(hist + (size_t)(int)ty_ * ps.nbx + (int)tx_, q0 * w);
  }
}

template <typename R>
cudaError_t launch_phasespace(SpeciesDev<R> sp, int b, int tx, int ty, int ntx,
                              int ntiles, PhaseSpaceSpec ps, double *hist,
                              cudaStream_t stream) {
  if (ntiles == 0) return cudaSuccess;
  phasespace_kernel<R><<<ntiles, kThreads, 0, stream>>>(sp, b, tx, ty, ntx, ps,
                                                        hist);
  return cudaGetLastError();
}

template <typename R>
__global__ void take_overflow_kernel(OverflowDev<R> ovf, int n_entries,
                                     int sim, int species, Staging<R> out,
                                     long long out_base, int *n_taken) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_entries;
       e += gridDim.x * blockDim.x) {
    if (ovf.sim[e] != sim || ovf.species[e] != species) continue;
    const size_t d = (size_t)(out_base + atomicAdd(n_taken, 1));
    out.ix[d] = ovf.ix[e];
    out.iy[d] = ovf.iy[e];
    out.id[d] = ovf.id[e];
    out.x[d] = ovf.x[e];
    out.y[d] = ovf.y[e];
    out.ux[d] = ovf.ux[e];
    out.uy[d] = ovf.uy[e];
    out.uz[d] = ovf.uz[e];
    out.w[d] = ovf.w[e];
  }
}

template <typename R>
cudaError_t launch_take_overflow(OverflowDev<R> ovf, int n_entries, int sim,
                                 int species, Staging<R> out,
                                 long long out_base, int *n_taken,
                                 cudaStream_t stream) {
  if (n_entries <= 0) return cudaSuccess;
  const int grid = (n_entries + kThreads - 1) / kThreads;
  take_overflow_kernel<R><<<grid < 1024 ? grid : 1024, kThreads, 0, stream>>>(
      ovf, n_entries, sim, species, out, out_base, n_taken);
  return cudaGetLastError();
}

#define ZP_INST(R)                                                            \
  template cudaError_t launch_migrate<R>(const SimDev<R> *, const int2 *,    \
                                         int, BatchStatus *,                  \
                                         const OverflowDev<R> &,              \
                                         cudaStream_t);                       \
  template cudaError_t launch_init_load<R>(const SimDev<R> *, int, LoadParams, \
                                           cudaStream_t);                     \
  template cudaError_t launch_bin_count<R>(Staging<R>, long long, int, int,   \
                                           int, int, int, int *, int *,       \
                                           cudaStream_t);                     \
  template cudaError_t launch_bin_scatter<R>(Staging<R>, long long,           \
                                             SpeciesDev<R>, int, int, int,    \
                                             int, int, cudaStream_t);         \
  template cudaError_t launch_compact<R>(SpeciesDev<R>, int, int, int, int,   \
                                         int, int, const long long *,         \
                                         Staging<R>, cudaStream_t);           \
  template cudaError_t launch_phasespace<R>(SpeciesDev<R>, int, int, int, int, \
                                            int, PhaseSpaceSpec, double *,    \
                                            cudaStream_t);                    \
  template cudaError_t launch_take_overflow<R>(OverflowDev<R>, int, int, int, \
                                               Staging<R>, long long, int *,  \
                                               cudaStream_t);
ZP_INST(float)
ZP_INST(double)
#undef ZP_INST

}  // namespace zp
