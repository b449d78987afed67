/*
 * zpic_oracle.h -- FP64 CPU oracle of the 2D3V electromagnetic PIC time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only tests/, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no header, helper or constant generator
 * with the CUDA path.
 *
 * The method (Guidotti et al., "Particle-In-Cell Simulation using
 * Asynchronous Tasking", arXiv 2106.12485, Sec. 2.2, stages 1-4):
 *   1. bilinear interpolation of E, B (from the previous iteration) at each
 *      particle position,
 *   2. leapfrog + relativistic Boris push of momentum and position,
 *   3. exact charge-conserving (Villasenor-Buneman) current deposition,
 *   4. Yee-mesh FDTD advance of E and B using the current just deposited.
 * Sec. 3.2 adds that a particle moves at most one cell per step; Sec. 4.1
 * adds the laser-initialised fields and the moving window.
 *
 * Units are normalised (c = 1, time in 1/w_p, length in c/w_p, E and B in
 * m c w_p / e, u = p/(m c) = gamma v).  Maxwell: dB/dt = -curl E,
 * dE/dt = curl B - J.
 *
 * Grid layout: nx*ny cells, arrays row-major f[j*nx + i], no guard cells.
 *   Ex(i+1/2, j)  Ey(i, j+1/2)  Ez(i, j)
 *   Bx(i, j+1/2)  By(i+1/2, j)  Bz(i+1/2, j+1/2)
 *   Jx, Jy, Jz co-located with Ex, Ey, Ez.
 * y is always periodic.  x is periodic, or open (moving window): samples
 * outside [0, nx) read as zero and deposits there are dropped.
 *
 * Particle: cell (ix, iy), offsets (x, y) in [0, 1), momentum u, weight w.
 * A particle of weight w carries charge q0*w (density units: a uniform load
 * of ppc particles of weight 1 and q0 = sign(q/m)/ppc gives |rho| = 1) and
 * mass q0*w/(q/m).
 */
#ifndef ZPIC_ORACLE_H
#define ZPIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;            /* cells */
    double dx, dy, dt;     /* cell size, time step */
    int open_x;            /* 0: periodic x; 1: open x (moving window) */
    int filter_j;          /* 1: smooth J with the compensated binomial
                              filter (orc_filter_current) before the field
                              update */
} orc_grid;

typedef struct {
    double *e[3], *b[3], *j[3];   /* each nx*ny */
} orc_fields;

typedef struct {
    long n, cap;
    int *ix, *iy, *id;            /* id may be NULL */
    double *x, *y, *ux, *uy, *uz, *w;
    double qm;                    /* charge-to-mass ratio */
    double q0;                    /* charge of a weight-1 particle */
} orc_species;

/* Moving-window state and plasma injection (Sec. 4.1, LWFA). */
typedef struct {
    int enabled;
    int n_shift;           /* shifts done so far */
    /* injected plasma per species: lattice ppc_x*ppc_y per cell, cold,
     * density profile n(x_abs) = 0 below ramp_x0, linear to n0 over
     * ramp_len, n0 beyond (ramp_len == 0: a step at ramp_x0). */
    int inject_ppc_x[8], inject_ppc_y[8];
    double ramp_x0[8], ramp_len[8], dens_n0[8];
    long id_base[8];       /* id of injected particles: id_base +
                              ((n_shift-1)*ny + j)*ppc + k */
} orc_window;

/* Stage 1: E, B at a particle (bilinear on the staggered grid). */
void orc_gather(const orc_grid *g, const orc_fields *f, int ix, int iy,
                double x, double y, double E[3], double B[3]);

/* Stage 2: relativistic Boris push of u over dt. */
void orc_boris(double qm, double dt, const double E[3], const double B[3],
               double u[3]);

/* Stage 3 for one straight in-cell segment: adds its J to f->j. */
void orc_deposit_segment(const orc_grid *g, const orc_fields *f, int ci,
                         int cj, double xa, double ya, double xb, double yb,
                         double frac, double q, double vz);

/* Stages 2b+3 for one particle: moves it by dt*u/gamma, splits the path at
 * cell faces and deposits each segment.  Updates ix, iy, x, y.  Returns 1 if
 * the particle left an open boundary (to be removed), else 0. */
int orc_move_deposit(const orc_grid *g, const orc_fields *f, int *ix, int *iy,
                     double *x, double *y, const double u[3], double q);

/* Stages 1-3 for a whole species.  J is NOT cleared.  kin (may be NULL)
 * receives sum of m_p (gamma-1) dx dy after the push.  do_deposit = 0
 * moves particles as test particles.  nthreads > 1 splits the particle
 * loop into contiguous ranges, each depositing into a private J copy that
 * is summed in thread order (the particle decomposition of Sec. 3.1). */
void orc_push_deposit(const orc_grid *g, const orc_fields *f, orc_species *s,
                      int do_deposit, int nthreads, double *kin);

/* Optional digital filter of the current (Sec. 2.2: a filter on J against
 * short-wavelength noise; Sec. 4.1: the LWFA runs use a compensated
 * binomial filter).  Per axis, x then y, and per component on its own
 * grid: one binomial pass (1, 2, 1)/4, then one compensation pass
 * (-1, 6, -1)/4, so a mode of wavenumber k is multiplied by
 * (1 - sin^2(k/2)) (1 + sin^2(k/2)) = 1 - sin^4(k/2) per axis.  y is
 * periodic; x is periodic, or open (values outside [0, nx) are zero). */
void orc_filter_current(const orc_grid *g, const orc_fields *f);

/* Stage 4: B -= (dt/2) curl E ; E += dt (curl B - J). */
void orc_yee_b_half(const orc_grid *g, const orc_fields *f);
void orc_yee_e(const orc_grid *g, const orc_fields *f);

/* Field energies 1/2 sum E^2 dx dy and 1/2 sum B^2 dx dy. */
void orc_field_energy(const orc_grid *g, const orc_fields *f, double *wE,
                      double *wB);

/* Gaussian laser pulse, linear polarisation along y, propagating in +x. */
void orc_laser(const orc_grid *g, const orc_fields *f, double a0,
               double omega0, double w0, double fwhm, double x0, double yc);

/* Moving window after step `step` (0-based, fields now at step+1):
 * shifts by one cell if (step+1)*dt >= (n_shift+1)*dx.  Returns 1 if it
 * shifted.  Injects the new right column for each species. */
int orc_window_shift(const orc_grid *g, const orc_fields *f, orc_window *win,
                     int nspecies, orc_species *sp, int step);

/* One full time step: J = 0; stages 1-3 for every species; stage 4;
 * energies; moving window.  energy_out (may be NULL) receives
 * {wE, wB, kin[0..nspecies-1]}.  Returns 0, or -1 if a species ran out of
 * capacity during injection. */
int orc_step(const orc_grid *g, const orc_fields *f, int nspecies,
             orc_species *sp, orc_window *win, int step, int nthreads,
             double *energy_out);

#ifdef __cplusplus
}
#endif
#endif
