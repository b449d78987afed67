// zpic_kernels.h -- host-side launchers of the CUDA kernels (all async on
// the given stream).
#pragma once

#include "zpic_dev.cuh"

namespace zp {

// Yee blocks: 32 columns x yee_rows<R>() rows per CTA of 256 threads.
// Larger blocks make the halo a smaller share of the loads and spread each
// block's fixed work over more cells: on a 2048^2 grid 0.16 ms per Yee step
// with 32 x 8, 0.13 ms with 32 x 16, 0.11 ms with 32 x 32 (FP32), 0.10 ms
// once the E and B halo goes straight into shared memory and four CTAs fit
// per SM.  FP64 stays at 32 x 16, whose tiles fill the 48 KB of static
// shared memory.
constexpr int kYeeX = 32;
constexpr int kYeeY = 16;
template <typename R>
__host__ __device__ constexpr int yee_rows() {
  return sizeof(R) == 4 ? 32 : kYeeY;
}

// Dynamic shared memory of the push kernel for tx x ty tiles; wide: some
// species stores weights or ids (larger particle-copy stages).
template <typename R>
size_t push_smem_bytes(int tx, int ty, bool wide);

// Resident push-kernel CTAs per SM for tx x ty tiles (0 on failure).
template <typename R>
int push_ctas_fit(int tx, int ty, bool wide);

// Sets the push kernel's dynamic shared-memory limit (call before launching
// or capturing it).
template <typename R>
cudaError_t prepare_push_deposit(int max_tx, int max_ty, bool wide);

// Stages 1-3 over all (sim, tile) items.  `single` (host copy of the only
// descriptor, or null for a batch) selects the one-simulation kernel that
// takes the descriptor as a kernel parameter.
template <typename R>
cudaError_t launch_push_deposit(const SimDev<R> *sims, const SimDev<R> *single,
                                const int2 *items, int n_items, int max_tx,
                                int max_ty, bool all16, bool wide,
                                int ctas_per_sm, BatchStatus *st,
                                const OverflowDev<R> &ovf,
                                cudaStream_t stream);

// Optional current filter over all (sim, yee block) items: Jf = compensated
// binomial filter of this step's J (simulations without Jf are skipped).
template <typename R>
cudaError_t launch_filter(const SimDev<R> *sims, const int2 *items,
                          int n_items, BatchStatus *st, cudaStream_t stream);

// Stage 4 (B half, E, B half) over all (sim, yee block) items; writes the
// other field copy (shifted one cell when the window moves), zeroes the
// other J copy, field-energy partials on energy steps.
template <typename R>
cudaError_t launch_yee(const SimDev<R> *sims, const int2 *items, int n_items,
                       BatchStatus *st, cudaStream_t stream);

// Moves outbox particles into their new tiles, injects the window column.
template <typename R>
cudaError_t launch_migrate(const SimDev<R> *sims, const int2 *items,
                           int n_items, BatchStatus *st,
                           const OverflowDev<R> &ovf, cudaStream_t stream);

// Cell-order re-sort of every tile of the simulations that are due after
// this step (into the other copy of the store; the end-of-step kernel makes
// it current).  prepare_sort_tiles sets the kernel's shared-memory limit.
template <typename R>
cudaError_t prepare_sort_tiles();
template <typename R>
cudaError_t launch_sort_tiles(const SimDev<R> *sims, int n_sims,
                              const int2 *items, int n_items, BatchStatus *st,
                              cudaStream_t stream);

// Energy records, window counter, step counter.
template <typename R>
cudaError_t launch_end_step(const SimDev<R> *sims, int n_sims, int g_max,
                            BatchStatus *st, cudaStream_t stream);

// Device pointers of the six field components (row length ld).
template <typename R>
struct FieldPtrs {
  const R *e[3], *b[3];
};
// Field energies 1/2 sum E^2 dx dy, 1/2 sum B^2 dx dy of nx*ny cells.
// scratch: 2*ny + 2 doubles of device memory; the results are left in
// scratch[2*ny] (electric) and scratch[2*ny + 1] (magnetic).
template <typename R>
cudaError_t launch_field_energy(FieldPtrs<R> f, int nx, int ny, int ld,
                                double dx, double dy, double *scratch,
                                cudaStream_t stream);

// Laser fields (Sec. 4.1) added to the current E, B copy of one sim.
struct LaserParams {
  double E0, omega0, w0, fwhm, x0, yc;
};
template <typename R>
cudaError_t launch_laser(const SimDev<R> *sim_dev, int nx, int ny,
                         LaserParams lp, cudaStream_t stream);

// Initial load of species s of one sim (counter-based SplitMix64).
struct LoadParams {
  int species;
  uint64_t key;                 // generator key of (seed, sim, species)
  int ppc_x, ppc_y, lattice;
  double u_th[3], u_fl[3];
  int profile;                  // ZPIC_PROFILE_*
  double x0, x1, n0;
  int col_lo, col_hi;           // loaded cell columns [col_lo, col_hi)
  int buf;                      // store copy written
};
template <typename R>
cudaError_t launch_init_load(const SimDev<R> *sim_dev, int ntiles,
                             LoadParams lp, cudaStream_t stream);

// Staging SoA used by set/get particles and re-sorting.
template <typename R>
struct Staging {
  int *ix, *iy, *id, *tile;
  R *x, *y, *ux, *uy, *uz, *w;
};

// tile of each staged particle + per-tile counts; bad[0] counts particles
// outside the grid or with offsets outside [0, 1)
template <typename R>
cudaError_t launch_bin_count(Staging<R> in, long long n, int nx, int ny,
                             int tx, int ty, int ntx, int *counts, int *bad,
                             cudaStream_t stream);
// scatters staged particles into the species' tile store (cnt used as
// cursor, must be zero); ids default to the index when in.id is null
template <typename R>
cudaError_t launch_bin_scatter(Staging<R> in, long long n,
                               SpeciesDev<R> sp_host_copy, int buf, int tx,
                               int ty, int has_w, int has_id,
                               cudaStream_t stream);
// compacts tiles [tile0, tile0 + ntiles) of store copy `buf` into a
// contiguous staging copy, tile tile0 + k from dst_off[k] on (global cells
// rebuilt from the tile index and the local cell)
// Phase-space histogram of one species: quantities qx, qy (ZPIC_PS_*),
// bins over [lo, lo + nb / scale) per axis.
struct PhaseSpaceSpec {
  int qx, qy, nbx, nby;
  double lo[2], scale[2];
  double q0;  // |charge| of a weight-1 particle (double, from the host)
};
template <typename R>
cudaError_t launch_phasespace(SpeciesDev<R> sp_host_copy, int buf, int tx,
                              int ty, int ntx, int ntiles, PhaseSpaceSpec ps,
                              double *hist, cudaStream_t stream);

template <typename R>
cudaError_t launch_compact(SpeciesDev<R> sp_host_copy, int buf, int tx,
                           int ty, int ntx, int tile0, int ntiles,
                           const long long *dst_off, Staging<R> out,
                           cudaStream_t stream);
// appends the overflow entries of (sim, species) to staging at *n_io
template <typename R>
cudaError_t launch_take_overflow(OverflowDev<R> ovf, int n_entries, int sim,
                                 int species, Staging<R> out,
                                 long long out_base, int *n_taken,
                                 cudaStream_t stream);

}  // namespace zp
