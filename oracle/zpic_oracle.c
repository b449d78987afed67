/*
 * zpic_oracle.c -- FP64 CPU oracle of the 2D3V EM-PIC time step.
 *
 * TEST INFRASTRUCTURE ONLY (see zpic_oracle.h).  Plain, slow, written to be
 * checked against the method by eye: every function does one step of the
 * PIC cycle of Sec. 2.2 in the order the paper gives, in double precision,
 * with no blocking, fusion or reordering.
 *
 * Readings where the paper is silent (it prints no equations):
 *  - time centring: x, E, B at integer n, u at n-1/2, J at n+1/2; B is kept
 *    at integer times by two half steps around the E update.
 *  - interpolation: a half-staggered component uses cell i-1 with weight
 *    x+1/2 when the offset x < 1/2, else cell i with weight x-1/2.
 *  - Boris: gamma taken after the first half kick.
 *  - deposit: the straight path is split at the x and y cell faces in the
 *    order they are met (an exact tie counts as x first); each in-cell
 *    segment adds the charge flux of the moving CIC cloud to Jx, Jy and the
 *    exact path average of the bilinear weight times q vz to Jz.
 *  - edge rounding: a crossing happens iff x_new >= 1 or x_new < 0; if a
 *    backward crossing rounds the new offset to exactly 1 the particle stays
 *    in its cell at offset 0.  The deposit ends at the stored position.
 */
#include "zpic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

/* Field sample with the boundary rules of the header. */
static double fld(const orc_grid *g, const double *f, int i, int j) {
    j = wrap(j, g->ny);
    if (g->open_x) {
        if (i < 0 || i >= g->nx) return 0.0;
    } else {
        i = wrap(i, g->nx);
    }
    return f[(long)j * g->nx + i];
}

static void jadd(const orc_grid *g, double *f, int i, int j, double v) {
    j = wrap(j, g->ny);
    if (g->open_x) {
        if (i < 0 || i >= g->nx) return;
    } else {
        i = wrap(i, g->nx);
    }
    f[(long)j * g->nx + i] += v;
}

/* ---- Stage 1: interpolation (Sec. 2.2, "bi-linear interpolation") ---- */

/* Along one axis: a component sampled at integer points (stag = 0) or at
 * half points (stag = 1); returns the lower sample index and the weight of
 * the upper sample for a particle at cell c, offset o. */
static void axis_weight(int c, double o, int stag, int *c0, double *w) {
    if (!stag) {
        *c0 = c;
        *w = o;
    } else if (o < 0.5) {
        *c0 = c - 1;
        *w = o + 0.5;
    } else {
        *c0 = c;
        *w = o - 0.5;
    }
}

static double interp(const orc_grid *g, const double *f, int ix, int iy,
                     double x, double y, int sx, int sy) {
    int i0, j0;
    double wx, wy;
    axis_weight(ix, x, sx, &i0, &wx);
    axis_weight(iy, y, sy, &j0, &wy);
    return (1.0 - wx) * (1.0 - wy) * fld(g, f, i0, j0) +
           wx * (1.0 - wy) * fld(g, f, i0 + 1, j0) +
           (1.0 - wx) * wy * fld(g, f, i0, j0 + 1) +
           wx * wy * fld(g, f, i0 + 1, j0 + 1);
}

void orc_gather(const orc_grid *g, const orc_fields *f, int ix, int iy,
                double x, double y, double E[3], double B[3]) {
    E[0] = interp(g, f->e[0], ix, iy, x, y, 1, 0); /* Ex(i+1/2, j)     */
    E[1] = interp(g, f->e[1], ix, iy, x, y, 0, 1); /* Ey(i, j+1/2)     */
    E[2] = interp(g, f->e[2], ix, iy, x, y, 0, 0); /* Ez(i, j)         */
    B[0] = interp(g, f->b[0], ix, iy, x, y, 0, 1); /* Bx(i, j+1/2)     */
    B[1] = interp(g, f->b[1], ix, iy, x, y, 1, 0); /* By(i+1/2, j)     */
    B[2] = interp(g, f->b[2], ix, iy, x, y, 1, 1); /* Bz(i+1/2, j+1/2) */
}

/* ---- Stage 2: leapfrog + relativistic Boris (Sec. 2.2) ---- */

void orc_boris(double qm, double dt, const double E[3], const double B[3],
               double u[3]) {
    const double h = 0.5 * qm * dt;
    double um[3], t[3], s[3], up[3], upl[3];
    int k;
    /* first half electric kick */
    for (k = 0; k < 3; k++) um[k] = u[k] + h * E[k];
    const double gam = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    /* magnetic rotation */
    for (k = 0; k < 3; k++) t[k] = h * B[k] / gam;
    const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (k = 0; k < 3; k++) s[k] = 2.0 * t[k] / (1.0 + t2);
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    upl[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    upl[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    upl[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    /* second half electric kick */
    for (k = 0; k < 3; k++) u[k] = upl[k] + h * E[k];
}

/* ---- Stage 3: charge-conserving deposition (Sec. 2.2, ref. Villasenor &
 * Buneman 1992) ---- */

void orc_deposit_segment(const orc_grid *g, const orc_fields *f, int ci,
                         int cj, double xa, double ya, double xb, double yb,
                         double frac, double q, double vz) {
    const double ddx = xb - xa, ddy = yb - ya;
    const double xm = 0.5 * (xa + xb), ym = 0.5 * (ya + yb);
    /* charge flux through the x faces (i+1/2, j) and (i+1/2, j+1) */
    const double ax = q * ddx * g->dx / g->dt;
    jadd(g, f->j[0], ci, cj, ax * (1.0 - ym));
    jadd(g, f->j[0], ci, cj + 1, ax * ym);
    /* charge flux through the y faces (i, j+1/2) and (i+1, j+1/2) */
    const double ay = q * ddy * g->dy / g->dt;
    jadd(g, f->j[1], ci, cj, ay * (1.0 - xm));
    jadd(g, f->j[1], ci + 1, cj, ay * xm);
    /* q vz times the path-averaged bilinear node weights */
    const double az = q * vz * frac;
    const double c = ddx * ddy / 12.0;
    jadd(g, f->j[2], ci, cj, az * ((1.0 - xm) * (1.0 - ym) + c));
    jadd(g, f->j[2], ci + 1, cj, az * (xm * (1.0 - ym) - c));
    jadd(g, f->j[2], ci, cj + 1, az * ((1.0 - xm) * ym - c));
    jadd(g, f->j[2], ci + 1, cj + 1, az * (xm * ym + c));
}

/* Crossing decision for one axis: start offset o, unrounded end o1.
 * Returns the cell step d in {-1, 0, 1}; *of = stored new offset, *oe =
 * path end in the start cell's frame (o1, or 0 after the rounding fix). */
static int axis_cross(double o1, double *of, double *oe) {
    if (o1 >= 1.0) {
        *of = o1 - 1.0;
        *oe = o1;
        return 1;
    }
    if (o1 < 0.0) {
        double t = o1 + 1.0;
        if (t == 1.0) { /* rounds back onto the face: stay, offset 0 */
            *of = 0.0;
            *oe = 0.0;
            return 0;
        }
        *of = t;
        *oe = o1;
        return -1;
    }
    *of = o1;
    *oe = o1;
    return 0;
}

int orc_move_deposit(const orc_grid *g, const orc_fields *f, int *ix, int *iy,
                     double *x, double *y, const double u[3], double q) {
    const double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double vz = u[2] / gam;
    const double x0 = *x, y0 = *y;
    const int i = *ix, jj = *iy;
    /* position advance in cell units (at most one cell by the CFL limit,
     * Sec. 3.2) */
    double x1 = x0 + g->dt * u[0] / (gam * g->dx);
    double y1 = y0 + g->dt * u[1] / (gam * g->dy);
    double xf, yf;
    const int di = axis_cross(x1, &xf, &x1);
    const int dj = axis_cross(y1, &yf, &y1);

    if (f) {
        if (di == 0 && dj == 0) {
            orc_deposit_segment(g, f, i, jj, x0, y0, xf, yf, 1.0, q, vz);
        } else if (dj == 0) {
            const double xb = di > 0 ? 1.0 : 0.0;
            const double sx = (xb - x0) / (x1 - x0);
            const double yc = y0 + sx * (y1 - y0);
            orc_deposit_segment(g, f, i, jj, x0, y0, xb, yc, sx, q, vz);
            orc_deposit_segment(g, f, i + di, jj, xb - di, yc, xf, yf,
                                1.0 - sx, q, vz);
        } else if (di == 0) {
            const double yb = dj > 0 ? 1.0 : 0.0;
            const double sy = (yb - y0) / (y1 - y0);
            const double xc = x0 + sy * (x1 - x0);
            orc_deposit_segment(g, f, i, jj, x0, y0, xc, yb, sy, q, vz);
            orc_deposit_segment(g, f, i, jj + dj, xc, yb - dj, xf, yf,
                                1.0 - sy, q, vz);
        } else {
            const double xb = di > 0 ? 1.0 : 0.0;
            const double yb = dj > 0 ? 1.0 : 0.0;
            const double sx = (xb - x0) / (x1 - x0);
            const double sy = (yb - y0) / (y1 - y0);
            const double y_at_sx = y0 + sx * (y1 - y0);
            const double x_at_sy = x0 + sy * (x1 - x0);
            if (sx <= sy) { /* x face first */
                orc_deposit_segment(g, f, i, jj, x0, y0, xb, y_at_sx, sx, q, vz);
                orc_deposit_segment(g, f, i + di, jj, xb - di, y_at_sx,
                                    x_at_sy - di, yb, sy - sx, q, vz);
                orc_deposit_segment(g, f, i + di, jj + dj, x_at_sy - di,
                                    yb - dj, xf, yf, 1.0 - sy, q, vz);
            } else { /* y face first */
                orc_deposit_segment(g, f, i, jj, x0, y0, x_at_sy, yb, sy, q, vz);
                orc_deposit_segment(g, f, i, jj + dj, x_at_sy, yb - dj, xb,
                                    y_at_sx - dj, sx - sy, q, vz);
                orc_deposit_segment(g, f, i + di, jj + dj, xb - di,
                                    y_at_sx - dj, xf, yf, 1.0 - sx, q, vz);
            }
        }
    }

    int ni = i + di, nj = wrap(jj + dj, g->ny);
    *x = xf;
    *y = yf;
    *iy = nj;
    if (g->open_x) {
        *ix = ni;
        return (ni < 0 || ni >= g->nx) ? 1 : 0;
    }
    *ix = wrap(ni, g->nx);
    return 0;
}

/* Advance particles [lo, hi) of species s, depositing into f (may be NULL).
 * removed[p] = 1 marks particles that left an open boundary. */
static double push_range(const orc_grid *g, const orc_fields *fg,
                         const orc_fields *fj, orc_species *s, long lo,
                         long hi, char *removed) {
    double kin = 0.0;
    for (long p = lo; p < hi; p++) {
        double E[3], B[3], u[3] = {s->ux[p], s->uy[p], s->uz[p]};
        orc_gather(g, fg, s->ix[p], s->iy[p], s->x[p], s->y[p], E, B);
        orc_boris(s->qm, g->dt, E, B, u);
        s->ux[p] = u[0];
        s->uy[p] = u[1];
        s->uz[p] = u[2];
        const double q = s->q0 * s->w[p];
        const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double gam = sqrt(1.0 + u2);
        kin += (q / s->qm) * (u2 / (gam + 1.0)); /* m_p (gamma - 1) */
        removed[p] = (char)orc_move_deposit(g, fj, &s->ix[p], &s->iy[p],
                                            &s->x[p], &s->y[p], u, q);
    }
    return kin;
}

static void remove_marked(orc_species *s, const char *removed) {
    long m = 0;
    for (long p = 0; p < s->n; p++) {
        if (removed[p]) continue;
        s->ix[m] = s->ix[p];
        s->iy[m] = s->iy[p];
        if (s->id) s->id[m] = s->id[p];
        s->x[m] = s->x[p];
        s->y[m] = s->y[p];
        s->ux[m] = s->ux[p];
        s->uy[m] = s->uy[p];
        s->uz[m] = s->uz[p];
        s->w[m] = s->w[p];
        m++;
    }
    s->n = m;
}

void orc_push_deposit(const orc_grid *g, const orc_fields *f, orc_species *s,
                      int do_deposit, int nthreads, double *kin) {
    const long ncell = (long)g->nx * g->ny;
    char *removed = (char *)calloc((size_t)(s->n > 0 ? s->n : 1), 1);
    double ktot = 0.0;
    if (nthreads <= 1 || !do_deposit) {
        ktot = push_range(g, f, do_deposit ? f : NULL, s, 0, s->n, removed);
    } else {
        /* Sec. 3.1: particles split evenly over threads, each deposits into
         * its own copy of J; the copies are then summed (here in thread
         * order, so the result is reproducible for a given thread count). */
        double *copies = (double *)calloc((size_t)(3 * ncell * nthreads),
                                          sizeof(double));
        double *kpart = (double *)calloc((size_t)nthreads, sizeof(double));
#pragma omp parallel num_threads(nthreads)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            orc_fields fj = *f;
            for (int c = 0; c < 3; c++) fj.j[c] = copies + (3L * t + c) * ncell;
            const long lo = s->n * t / nthreads, hi = s->n * (t + 1) / nthreads;
            kpart[t] = push_range(g, f, &fj, s, lo, hi, removed);
        }
        for (int t = 0; t < nthreads; t++) {
            ktot += kpart[t];
            for (int c = 0; c < 3; c++) {
                const double *src = copies + (3L * t + c) * ncell;
                for (long k = 0; k < ncell; k++) f->j[c][k] += src[k];
            }
        }
        free(copies);
        free(kpart);
    }
    if (g->open_x) remove_marked(s, removed);
    free(removed);
    if (kin) *kin = ktot * g->dx * g->dy;
}

/* ---- Optional current filter (Sec. 2.2; compensated binomial, Sec. 4.1) ---- */

/* One 3-point pass with weights (a, b, a) along x (dir 0) or y (dir 1). */
static void filter_pass(const orc_grid *g, double *v, int dir, double a,
                        double b) {
    const long n = (long)g->nx * g->ny;
    double *src = malloc(sizeof(double) * n);
    memcpy(src, v, sizeof(double) * n);
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            double lo, hi;
            if (dir == 0) {
                lo = fld(g, src, i - 1, j);
                hi = fld(g, src, i + 1, j);
            } else {
                lo = fld(g, src, i, j - 1);
                hi = fld(g, src, i, j + 1);
            }
            v[(long)j * g->nx + i] = a * lo + b * src[(long)j * g->nx + i] + a * hi;
        }
    free(src);
}

void orc_filter_current(const orc_grid *g, const orc_fields *f) {
    for (int c = 0; c < 3; c++)
        for (int dir = 0; dir < 2; dir++) {
            filter_pass(g, f->j[c], dir, 0.25, 0.5);    /* binomial */
            filter_pass(g, f->j[c], dir, -0.25, 1.5);   /* compensation */
        }
}

/* ---- Stage 4: Yee FDTD field advance (Sec. 2.2) ---- */

void orc_yee_b_half(const orc_grid *g, const orc_fields *f) {
    const double h = 0.5 * g->dt;
    double *bx = f->b[0], *by = f->b[1], *bz = f->b[2];
    const double *ex = f->e[0], *ey = f->e[1], *ez = f->e[2];
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            const long k = (long)j * g->nx + i;
            /* dBx/dt = -dEz/dy at (i, j+1/2) */
            bx[k] -= h * (fld(g, ez, i, j + 1) - fld(g, ez, i, j)) / g->dy;
            /* dBy/dt = +dEz/dx at (i+1/2, j) */
            by[k] += h * (fld(g, ez, i + 1, j) - fld(g, ez, i, j)) / g->dx;
            /* dBz/dt = -(dEy/dx - dEx/dy) at (i+1/2, j+1/2) */
            bz[k] -= h * ((fld(g, ey, i + 1, j) - fld(g, ey, i, j)) / g->dx -
                          (fld(g, ex, i, j + 1) - fld(g, ex, i, j)) / g->dy);
        }
}

void orc_yee_e(const orc_grid *g, const orc_fields *f) {
    const double dt = g->dt;
    double *ex = f->e[0], *ey = f->e[1], *ez = f->e[2];
    const double *bx = f->b[0], *by = f->b[1], *bz = f->b[2];
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            const long k = (long)j * g->nx + i;
            /* dEx/dt = dBz/dy - Jx at (i+1/2, j) */
            ex[k] += dt * ((fld(g, bz, i, j) - fld(g, bz, i, j - 1)) / g->dy -
                           f->j[0][k]);
            /* dEy/dt = -dBz/dx - Jy at (i, j+1/2) */
            ey[k] += dt * (-(fld(g, bz, i, j) - fld(g, bz, i - 1, j)) / g->dx -
                           f->j[1][k]);
            /* dEz/dt = dBy/dx - dBx/dy - Jz at (i, j) */
            ez[k] += dt * ((fld(g, by, i, j) - fld(g, by, i - 1, j)) / g->dx -
                           (fld(g, bx, i, j) - fld(g, bx, i, j - 1)) / g->dy -
                           f->j[2][k]);
        }
}

void orc_field_energy(const orc_grid *g, const orc_fields *f, double *wE,
                      double *wB) {
    const long n = (long)g->nx * g->ny;
    double se = 0.0, sb = 0.0;
    for (int c = 0; c < 3; c++)
        for (long k = 0; k < n; k++) {
            se += f->e[c][k] * f->e[c][k];
            sb += f->b[c][k] * f->b[c][k];
        }
    *wE = 0.5 * se * g->dx * g->dy;
    *wB = 0.5 * sb * g->dx * g->dy;
}

/* ---- Laser initialisation (Sec. 4.1, LWFA: fields start as the laser) ---- */

static double laser_profile(double X, double Y, double E0, double omega0,
                            double w0, double fwhm, double x0, double yc) {
    const double dX = X - x0, dY = Y - yc;
    /* envelope whose intensity (field squared) has full width fwhm in x */
    return E0 * exp(-dY * dY / (w0 * w0)) *
           exp(-2.0 * log(2.0) * dX * dX / (fwhm * fwhm)) * cos(omega0 * dX);
}

void orc_laser(const orc_grid *g, const orc_fields *f, double a0,
               double omega0, double w0, double fwhm, double x0, double yc) {
    const double E0 = a0 * omega0;
    for (int j = 0; j < g->ny; j++)
        for (int i = 0; i < g->nx; i++) {
            const long k = (long)j * g->nx + i;
            /* Ey at (i, j+1/2); Bz = Ey of a +x wave, at (i+1/2, j+1/2) */
            f->e[1][k] += laser_profile(i * g->dx, (j + 0.5) * g->dy, E0,
                                        omega0, w0, fwhm, x0, yc);
            f->b[2][k] += laser_profile((i + 0.5) * g->dx, (j + 0.5) * g->dy,
                                        E0, omega0, w0, fwhm, x0, yc);
        }
}

/* ---- Moving window (Sec. 4.1, LWFA) ---- */

static double ramp_density(const orc_window *win, int s, double xa) {
    if (xa < win->ramp_x0[s]) return 0.0;
    if (win->ramp_len[s] > 0.0 && xa < win->ramp_x0[s] + win->ramp_len[s])
        return win->dens_n0[s] * (xa - win->ramp_x0[s]) / win->ramp_len[s];
    return win->dens_n0[s];
}

int orc_window_shift(const orc_grid *g, const orc_fields *f, orc_window *win,
                     int nspecies, orc_species *sp, int step) {
    if (!win || !win->enabled) return 0;
    if (!((step + 1) * g->dt >= (win->n_shift + 1) * g->dx)) return 0;
    /* fields move one cell towards -x; the new right column is empty */
    for (int c = 0; c < 3; c++) {
        double *fs[2] = {f->e[c], f->b[c]};
        for (int a = 0; a < 2; a++)
            for (int j = 0; j < g->ny; j++) {
                double *row = fs[a] + (long)j * g->nx;
                for (int i = 0; i < g->nx - 1; i++) row[i] = row[i + 1];
                row[g->nx - 1] = 0.0;
            }
    }
    win->n_shift++;
    for (int s = 0; s < nspecies; s++) {
        orc_species *p = &sp[s];
        /* particles follow the window frame; those now left of it leave */
        long m = 0;
        for (long k = 0; k < p->n; k++) {
            if (p->ix[k] - 1 < 0) continue;
            p->ix[m] = p->ix[k] - 1;
            p->iy[m] = p->iy[k];
            if (p->id) p->id[m] = p->id[k];
            p->x[m] = p->x[k];
            p->y[m] = p->y[k];
            p->ux[m] = p->ux[k];
            p->uy[m] = p->uy[k];
            p->uz[m] = p->uz[k];
            p->w[m] = p->w[k];
            m++;
        }
        p->n = m;
        /* cold plasma on a lattice enters through the new right column */
        const int px = win->inject_ppc_x[s], py = win->inject_ppc_y[s];
        if (px <= 0 || py <= 0) continue;
        const int i = g->nx - 1;
        const double xa = (i + win->n_shift + 0.5) * g->dx; /* lab frame */
        const double dens = ramp_density(win, s, xa);
        if (dens <= 0.0) continue;
        for (int j = 0; j < g->ny; j++)
            for (int ky = 0; ky < py; ky++)
                for (int kx = 0; kx < px; kx++) {
                    if (p->n >= p->cap) return -1;
                    const long k = p->n++;
                    const int kk = ky * px + kx;
                    p->ix[k] = i;
                    p->iy[k] = j;
                    p->x[k] = (kx + 0.5) / px;
                    p->y[k] = (ky + 0.5) / py;
                    p->ux[k] = p->uy[k] = p->uz[k] = 0.0;
                    p->w[k] = dens;
                    if (p->id)
                        p->id[k] = (int)(win->id_base[s] +
                                         ((long)(win->n_shift - 1) * g->ny + j) *
                                             (px * py) +
                                         kk);
                }
    }
    return 1;
}

/* ---- The PIC cycle (Sec. 2.2, Fig. 1: stages 1-4 in order) ---- */

int orc_step(const orc_grid *g, const orc_fields *f, int nspecies,
             orc_species *sp, orc_window *win, int step, int nthreads,
             double *energy_out) {
    const long ncell = (long)g->nx * g->ny;
    for (int c = 0; c < 3; c++) memset(f->j[c], 0, sizeof(double) * ncell);
    for (int s = 0; s < nspecies; s++) {
        double kin = 0.0;
        orc_push_deposit(g, f, &sp[s], 1, nthreads, &kin);
        if (energy_out) energy_out[2 + s] = kin;
    }
    if (g->filter_j) orc_filter_current(g, f);
    orc_yee_b_half(g, f);
    orc_yee_e(g, f);
    orc_yee_b_half(g, f);
    if (energy_out) orc_field_energy(g, f, &energy_out[0], &energy_out[1]);
    if (win && win->enabled)
        if (orc_window_shift(g, f, win, nspecies, sp, step) < 0) return -1;
    return 0;
}
