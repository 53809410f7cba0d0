/*
 * rc_oracle.c -- plain, slow, FP64 CPU oracle of the radiance-cascade (RC)
 * formal solution of Osborne & Sannikov, "Radiance Cascades: A Novel
 * High-Resolution Formal Solution for Multidimensional Non-LTE Radiative
 * Transfer" (arXiv 2408.14425).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into librcoracle.so,
 * which only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load.  The CUDA product path never links, calls or includes
 * anything from here, and nothing here comes from the CUDA path: the two
 * share no code, headers, tables or constants.
 *
 * Every routine states the passage of the paper it follows.  The steps run
 * in the paper's order with no blocking, fusion or reordering:
 *
 *   radiance interval R_{a,b}(p,w) = [I_{b->a}, tau_{b->a}]     Sec. 2.2, Eq. 9
 *   piecewise-constant per-cell update, back-to-front march      Sec. 3.2, Eq. 16
 *   merge operator M for contiguous intervals                    Sec. 2.2.1, Eq. 11
 *   cascade scaling law, probe grid, direction set               Sec. 2.3, Eq. 12-13
 *   bilinear interpolation + child-cone averaging, top-down      Sec. 2.3.1
 *   edge clamp of the bilinear lookup                            Sec. 2.5
 *   J as the angular mean                                        Eq. 1
 *   diagonal ALO of the piecewise-constant scheme                Sec. 3.3, Eq. 17
 *
 * Readings taken where the paper is silent or inconsistent (also listed in
 * the design notes):
 *   (R1) Eq. 11 as printed attenuates the nearer interval by the farther one.
 *        Radiation arriving at the probe (what Eq. 1 integrates) is the
 *        nearer interval's own emission plus the farther interval's emission
 *        attenuated by the nearer interval:  I_near + exp(-tau_near) I_far.
 *        That is the form used here; the splitting-invariance test fixes it.
 *   (R2) Interval lengths L0 * g^i with g = 2^alpha = 2^(branching/2)
 *        (rule 0: a_i = sum_{j<i} L0 g^j), or the alternative t_i = L0 g^(i-1)
 *        (rule 1).  The top cascade extends to infinity (Sec. 2.3).
 *   (R3) Cascade-0 probes at cell centres (Sec. 3.2); cascade-i probes at
 *        ((k+1/2) 2^i, (m+1/2) 2^i), P_i = ceil(N / 2^i) per axis.
 *   (R4) Directions theta_{i,k} = 2 pi (k+1/2) / W_i with W_i = W_0 B^i; the
 *        children of k are B k .. B k + B - 1, which tile the parent's cone.
 *   (R5) Outside the domain chi = eta = 0 and nothing enters (Sec. 3.4, free
 *        space).
 *   (R6) Eq. 17 prints Lambda* = exp(-tau_centre->edge); the local operator of
 *        the piecewise-constant update (Eq. 16) is 1 - exp(-tau_centre->edge),
 *        which is the coefficient of the local source function in I at the
 *        cell centre.  The oracle uses 1 - exp(-chi d).
 *
 * Units: positions and interval bounds are in voxel units; chi (m^-1 or
 * voxel^-1) multiplies the physical path length (voxel units x voxel_size).
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC rc_oracle.c -o librcoracle.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define RCO_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Cascade geometry (Sec. 2.3, Eq. 12-13; readings R2-R4)                    */
/* ------------------------------------------------------------------------ */

/* Interval [a_i, b_i] of cascade i (in voxels).  branching = 2 alpha, so the
 * interval lengths grow by 2^alpha per cascade (Eq. 12). */
void rco_interval(int rule, double interval0, int branching, int i,
                  int n_cascades, double* a, double* b)
{
    double g = pow(2.0, 0.5 * (double)branching);
    if (rule == 0) {
        double start = 0.0;
        for (int j = 0; j < i; ++j) start += interval0 * pow(g, (double)j);
        *a = start;
        *b = start + interval0 * pow(g, (double)i);
    } else {
        *a = (i == 0) ? 0.0 : interval0 * pow(g, (double)(i - 1));
        *b = interval0 * pow(g, (double)i);
    }
    if (i == n_cascades - 1) *b = INFINITY; /* top cascade leaves the domain */
}

/* Probes per axis of cascade i for an axis of n cells (reading R3). */
int rco_probes(int n, int i)
{
    int s = 1 << i;
    return (n + s - 1) / s;
}

/* Direction count of cascade i (reading R4). */
long long rco_dirs(int dirs0, int branching, int i)
{
    long long w = dirs0;
    for (int j = 0; j < i; ++j) w *= branching;
    return w;
}

/* Unit vector of direction k of a cascade with W directions (reading R4). */
void rco_direction(long long k, long long W, double* wx, double* wz)
{
    double th = 2.0 * RCO_PI * ((double)k + 0.5) / (double)W;
    *wx = cos(th);
    *wz = sin(th);
}

/* ------------------------------------------------------------------------ */
/* One radiance interval (Sec. 2.2 Eq. 9, Sec. 3.2 Eq. 16)                   */
/* ------------------------------------------------------------------------ */

/* Clip o + t w, t in [*t0,*t1], to the domain box [0,nx] x [0,nz]. */
static int clip_to_box(double ox, double oz, double wx, double wz, int nx, int nz,
                       double* t0, double* t1)
{
    double lo = *t0, hi = *t1;
    if (wx != 0.0) {
        double ta = (0.0 - ox) / wx, tb = ((double)nx - ox) / wx;
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > lo) lo = ta;
        if (tb < hi) hi = tb;
    } else if (ox < 0.0 || ox > (double)nx) {
        return 0;
    }
    if (wz != 0.0) {
        double ta = (0.0 - oz) / wz, tb = ((double)nz - oz) / wz;
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > lo) lo = ta;
        if (tb < hi) hi = tb;
    } else if (oz < 0.0 || oz > (double)nz) {
        return 0;
    }
    if (!(lo < hi)) return 0;
    *t0 = lo;
    *t1 = hi;
    return 1;
}

/* Next grid-plane crossing of one coordinate after parameter t (strictly
 * beyond the plane the point may sit on). */
static double next_plane_t(double o, double w, double t)
{
    if (w == 0.0) return INFINITY;
    double x = o + t * w;
    double m = (w > 0.0) ? floor(x) + 1.0 : ceil(x) - 1.0;
    double tn = (m - o) / w;
    /* guard against rounding that lands on or before t */
    while (!(tn > t)) { m += (w > 0.0) ? 1.0 : -1.0; tn = (m - o) / w; }
    return tn;
}

/*
 * R_{a,b}(o, w) for one wavelength slab (chi, eta: [nz][nx], x fastest).
 * The ray o + t w, t in [a, b], is cut at every cell face it crosses (exact
 * FP64 plane intersections); each piece lies in the cell that holds its
 * midpoint.  Pieces are then integrated back to front, i.e. from t = b
 * towards the probe at t = a (Sec. 3.2), with Eq. 16:
 *     tau += chi ds,   I <- I exp(-chi ds) + (eta/chi)(1 - exp(-chi ds)).
 * A cell with chi = 0 adds eta ds (the chi -> 0 limit of Eq. 16).
 * chi == NULL counts crossings only.  Returns the number of pieces of
 * positive length (the voxel crossings).
 */
long long rco_march(const double* chi, const double* eta, int nx, int nz,
                    double voxel, double ox, double oz, double wx, double wz,
                    double a, double b, double* I_out, double* tau_out)
{
    double t0 = a, t1 = b;
    if (I_out) *I_out = 0.0;
    if (tau_out) *tau_out = 0.0;
    if (!clip_to_box(ox, oz, wx, wz, nx, nz, &t0, &t1)) return 0;

    /* breakpoints in increasing t */
    int cap = nx + nz + 8;
    double* tb = (double*)malloc(sizeof(double) * (size_t)cap);
    int n = 0;
    tb[n++] = t0;
    double tx = next_plane_t(ox, wx, t0), tz = next_plane_t(oz, wz, t0);
    for (;;) {
        double tn = tx < tz ? tx : tz;
        if (!(tn < t1)) break;
        if (n + 1 >= cap) { cap *= 2; tb = (double*)realloc(tb, sizeof(double) * (size_t)cap); }
        tb[n++] = tn;
        if (tx <= tn) tx = next_plane_t(ox, wx, tn);
        if (tz <= tn) tz = next_plane_t(oz, wz, tn);
    }
    tb[n++] = t1;

    long long crossings = 0;
    double I = 0.0, tau = 0.0;
    /* back to front: the piece farthest from the probe first */
    for (int s = n - 2; s >= 0; --s) {
        double ta = tb[s], tbb = tb[s + 1];
        if (!(tbb > ta)) continue;
        double tm = 0.5 * (ta + tbb);
        int ix = (int)floor(ox + tm * wx), iz = (int)floor(oz + tm * wz);
        if (ix < 0) ix = 0;
        if (ix >= nx) ix = nx - 1;
        if (iz < 0) iz = 0;
        if (iz >= nz) iz = nz - 1;
        ++crossings;
        if (!chi) continue;
        double ds = (tbb - ta) * voxel;
        double c = chi[(size_t)iz * nx + ix], e = eta[(size_t)iz * nx + ix];
        double dtau = c * ds;
        if (c > 0.0)
            I = I * exp(-dtau) + (e / c) * (-expm1(-dtau));
        else
            I = I + e * ds;
        tau += dtau;
    }
    free(tb);
    if (I_out) *I_out = I;
    if (tau_out) *tau_out = tau;
    return crossings;
}

/* Merge operator M of two contiguous intervals, near = [a,b], far = [b,c]
 * (Sec. 2.2.1, Eq. 11 under reading R1). */
void rco_merge(double I_near, double tau_near, double I_far, double tau_far,
               double* I_out, double* tau_out)
{
    *I_out = I_near + exp(-tau_near) * I_far;
    *tau_out = tau_near + tau_far;
}

/* ------------------------------------------------------------------------ */
/* Full RC formal solution (Sec. 2.3, 2.3.1, 2.5, Eq. 1)                     */
/* ------------------------------------------------------------------------ */

/* Bilinear lookup coordinate of a cascade-i probe (index m) in cascade i+1's
 * probe index space, clamped to the outermost probes (Sec. 2.5). */
static void upper_weights(int m, int i, int P_up, int* j0, int* j1, double* f)
{
    double pos = ((double)m + 0.5) * (double)(1 << i);        /* voxels */
    double u = pos / (double)(1 << (i + 1)) - 0.5;            /* upper index */
    if (u < 0.0) u = 0.0;
    if (u > (double)(P_up - 1)) u = (double)(P_up - 1);
    int lo = (int)floor(u);
    int hi = lo + 1 < P_up ? lo + 1 : P_up - 1;
    *j0 = lo;
    *j1 = hi;
    *f = u - (double)lo;
}

/*
 * J for n_lambda slabs chi/eta [n_lambda][nz][nx] -> J [n_lambda][nz][nx].
 * alo (nullable) receives the angle-averaged diagonal operator of cascade 0,
 * (1/W0) sum_k (1 - exp(-chi d_k)), d_k the centre-to-edge path (reading R6).
 * crossings_per_level (nullable, n_cascades entries) receives the voxel
 * crossings of one wavelength per cascade.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int rco_rc_solve_fix(const double* chi, const double* eta, int nx, int nz,
                     int n_lambda, double voxel, int n_cascades, int dirs0,
                     int branching, double interval0, int rule, int bilinear_fix,
                     double* J, double* alo, long long* crossings_per_level);

int rco_rc_solve(const double* chi, const double* eta, int nx, int nz,
                 int n_lambda, double voxel, int n_cascades, int dirs0,
                 int branching, double interval0, int rule, double* J,
                 double* alo, long long* crossings_per_level)
{
    return rco_rc_solve_fix(chi, eta, nx, nz, n_lambda, voxel, n_cascades, dirs0, branching,
                            interval0, rule, 0, J, alo, crossings_per_level);
}

/*
 * As rco_rc_solve; with bilinear_fix != 0 every cascade-i ray below the top is traced
 * from its own start p + a_i w to the start of the child interval on each of the four
 * bracketing cascade-(i+1) probes, x_b + a_{i+1} w, merged there with that probe's
 * child-cone average, and the four merged values are averaged with the usual bilinear
 * weights (Sec. 2.5, the bilinear fix).  The diagonal operator (alo) is defined for the
 * basic construction only: with the fix a child interval may start inside the probe's
 * own cell, so alo must be NULL then.
 */
int rco_rc_solve_fix(const double* chi, const double* eta, int nx, int nz,
                     int n_lambda, double voxel, int n_cascades, int dirs0,
                     int branching, double interval0, int rule, int bilinear_fix,
                     double* J, double* alo, long long* crossings_per_level)
{
    if (nx <= 0 || nz <= 0 || n_lambda < 0 || n_cascades < 1 || dirs0 < 1 ||
        branching < 1 || !(interval0 > 0.0) || (bilinear_fix && alo))
        return -1;
    if (crossings_per_level)
        for (int i = 0; i < n_cascades; ++i) crossings_per_level[i] = 0;
    size_t ncell = (size_t)nx * (size_t)nz;

    for (int l = 0; l < n_lambda; ++l) {
        const double* ch = chi + (size_t)l * ncell;
        const double* et = eta + (size_t)l * ncell;
        double* R_up = NULL;          /* merged R of cascade i+1 */
        int Px_up = 0, Pz_up = 0;
        long long W_up = 0;

        for (int i = n_cascades - 1; i >= 0; --i) {
            int Px = rco_probes(nx, i), Pz = rco_probes(nz, i);
            long long W = rco_dirs(dirs0, branching, i);
            double a, b;
            rco_interval(rule, interval0, branching, i, n_cascades, &a, &b);
            double spacing = (double)(1 << i);
            size_t nR = (size_t)Px * (size_t)Pz * (size_t)W;
            double* R = (double*)malloc(sizeof(double) * (nR ? nR : 1));
            if (!R) { free(R_up); return -1; }
            long long lvl_cross = 0;

#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(+ : lvl_cross)
            for (int pz = 0; pz < Pz; ++pz) {
                for (int px = 0; px < Px; ++px) {
                    double ox = ((double)px + 0.5) * spacing;
                    double oz = ((double)pz + 0.5) * spacing;
                    int jx0 = 0, jx1 = 0, jz0 = 0, jz1 = 0;
                    double fx = 0.0, fz = 0.0;
                    if (R_up) {
                        upper_weights(px, i, Px_up, &jx0, &jx1, &fx);
                        upper_weights(pz, i, Pz_up, &jz0, &jz1, &fz);
                    }
                    for (long long k = 0; k < W; ++k) {
                        double wx, wz, I, tau;
                        rco_direction(k, W, &wx, &wz);
                        if (R_up && bilinear_fix) {
                            double a_up, b_up;
                            rco_interval(rule, interval0, branching, i + 1, n_cascades, &a_up, &b_up);
                            const double Ax = ox + a * wx, Az = oz + a * wz;
                            const double up_spacing = (double)(1 << (i + 1));
                            int jz[2] = {jz0, jz1}, jx[2] = {jx0, jx1};
                            double wzz[2] = {1.0 - fz, fz}, wxx[2] = {1.0 - fx, fx};
                            double Rm = 0.0;
                            for (int q = 0; q < 2; ++q)
                                for (int r = 0; r < 2; ++r) {
                                    const double Bx = ((double)jx[r] + 0.5) * up_spacing + a_up * wx;
                                    const double Bz = ((double)jz[q] + 0.5) * up_spacing + a_up * wz;
                                    const double L = hypot(Bx - Ax, Bz - Az);
                                    double Ib = 0.0, tb = 0.0;
                                    if (L > 0.0)
                                        lvl_cross += rco_march(ch, et, nx, nz, voxel, Ax, Az,
                                                               (Bx - Ax) / L, (Bz - Az) / L, 0.0,
                                                               L, &Ib, &tb);
                                    const double* Rp =
                                        R_up + ((size_t)jz[q] * Px_up + jx[r]) * (size_t)W_up;
                                    double avg = 0.0;
                                    for (int c = 0; c < branching; ++c)
                                        avg += Rp[(size_t)(k * branching + c)];
                                    avg /= (double)branching;
                                    double Imerged, taum;
                                    rco_merge(Ib, tb, avg, 0.0, &Imerged, &taum);
                                    Rm += wzz[q] * wxx[r] * Imerged;
                                }
                            R[((size_t)pz * Px + px) * (size_t)W + (size_t)k] = Rm;
                            continue;
                        }
                        lvl_cross += rco_march(ch, et, nx, nz, voxel, ox, oz, wx, wz,
                                               a, b, &I, &tau);
                        double Rm = I;
                        if (R_up) {
                            /* child-cone average on each of the four upper
                             * probes, then bilinear interpolation */
                            int jz[2] = {jz0, jz1}, jx[2] = {jx0, jx1};
                            double wzz[2] = {1.0 - fz, fz}, wxx[2] = {1.0 - fx, fx};
                            double upper = 0.0;
                            for (int q = 0; q < 2; ++q)
                                for (int r = 0; r < 2; ++r) {
                                    const double* Rp =
                                        R_up + ((size_t)jz[q] * Px_up + jx[r]) * (size_t)W_up;
                                    double avg = 0.0;
                                    for (int c = 0; c < branching; ++c)
                                        avg += Rp[(size_t)(k * branching + c)];
                                    avg /= (double)branching;
                                    upper += wzz[q] * wxx[r] * avg;
                                }
                            double tau_far = 0.0, Imerged, taum;
                            rco_merge(I, tau, upper, tau_far, &Imerged, &taum);
                            Rm = Imerged;
                        }
                        R[((size_t)pz * Px + px) * (size_t)W + (size_t)k] = Rm;
                    }
                }
            }
            if (crossings_per_level && l == 0) crossings_per_level[i] = lvl_cross;
            free(R_up);
            R_up = R;
            Px_up = Px;
            Pz_up = Pz;
            W_up = W;
        }

        /* Eq. 1 in flatland: equal-weight mean over the cascade-0 directions */
        double* Jl = J + (size_t)l * ncell;
        for (int iz = 0; iz < nz; ++iz)
            for (int ix = 0; ix < nx; ++ix) {
                double s = 0.0;
                for (long long k = 0; k < W_up; ++k)
                    s += R_up[((size_t)iz * nx + ix) * (size_t)W_up + (size_t)k];
                Jl[(size_t)iz * nx + ix] = s / (double)W_up;
            }
        free(R_up);

        if (alo) {
            double* Al = alo + (size_t)l * ncell;
            for (size_t c = 0; c < ncell; ++c) {
                double s = 0.0;
                for (int k = 0; k < dirs0; ++k) {
                    double wx, wz;
                    rco_direction(k, dirs0, &wx, &wz);
                    double m = fabs(wx) > fabs(wz) ? fabs(wx) : fabs(wz);
                    double d = 0.5 / m * voxel;
                    s += -expm1(-ch[c] * d);
                }
                Al[c] = s / (double)dirs0;
            }
        }
    }
    return 0;
}

/*
 * Sparse RC (Sec. 3.5): only the cells with active[c] != 0 take part.  Inactive cells are
 * transparent with no emission (chi = eta = 0); the cascade-0 probes of active cells are
 * flagged, and every flagged probe flags the (up to four) cascade-(i+1) probes its bilinear
 * lookup brackets, up to the top cascade.  Only flagged probes' intervals are computed
 * (the others are filled with NaN, so a read of one would show); J of inactive cells is 0.
 * rays_per_level (nullable) receives the number of intervals computed per cascade.
 */
int rco_rc_solve_sparse(const double* chi, const double* eta, const unsigned char* active,
                        int nx, int nz, double voxel, int n_cascades, int dirs0, int branching,
                        double interval0, int rule, double* J, long long* rays_per_level)
{
    if (nx <= 0 || nz <= 0 || n_cascades < 1 || dirs0 < 1 || branching < 1 || !active)
        return -1;
    const size_t ncell = (size_t)nx * nz;
    double* mc = (double*)malloc(sizeof(double) * ncell);
    double* me = (double*)malloc(sizeof(double) * ncell);
    for (size_t c = 0; c < ncell; ++c) {
        mc[c] = active[c] ? chi[c] : 0.0;
        me[c] = active[c] ? eta[c] : 0.0;
    }
    /* flags, bottom up */
    unsigned char** F = (unsigned char**)calloc((size_t)n_cascades, sizeof(unsigned char*));
    for (int i = 0; i < n_cascades; ++i)
        F[i] = (unsigned char*)calloc((size_t)rco_probes(nx, i) * rco_probes(nz, i), 1);
    for (size_t c = 0; c < ncell; ++c) F[0][c] = active[c] ? 1 : 0;
    for (int i = 0; i + 1 < n_cascades; ++i) {
        const int Px = rco_probes(nx, i), Pz = rco_probes(nz, i);
        const int Pxu = rco_probes(nx, i + 1), Pzu = rco_probes(nz, i + 1);
        for (int pz = 0; pz < Pz; ++pz)
            for (int px = 0; px < Px; ++px) {
                if (!F[i][(size_t)pz * Px + px]) continue;
                int jx0, jx1, jz0, jz1;
                double fx, fz;
                upper_weights(px, i, Pxu, &jx0, &jx1, &fx);
                upper_weights(pz, i, Pzu, &jz0, &jz1, &fz);
                F[i + 1][(size_t)jz0 * Pxu + jx0] = 1;
                F[i + 1][(size_t)jz0 * Pxu + jx1] = 1;
                F[i + 1][(size_t)jz1 * Pxu + jx0] = 1;
                F[i + 1][(size_t)jz1 * Pxu + jx1] = 1;
            }
    }
    /* top down, flagged probes only */
    double* R_up = NULL;
    int Px_up = 0, Pz_up = 0;
    long long W_up = 0;
    for (int i = n_cascades - 1; i >= 0; --i) {
        const int Px = rco_probes(nx, i), Pz = rco_probes(nz, i);
        const long long W = rco_dirs(dirs0, branching, i);
        double a, b;
        rco_interval(rule, interval0, branching, i, n_cascades, &a, &b);
        const double spacing = (double)(1 << i);
        double* R = (double*)malloc(sizeof(double) * (size_t)Px * Pz * W);
        long long rays = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(+ : rays)
        for (int pz = 0; pz < Pz; ++pz)
            for (int px = 0; px < Px; ++px) {
                double* Rp = R + ((size_t)pz * Px + px) * (size_t)W;
                if (!F[i][(size_t)pz * Px + px]) {
                    for (long long k = 0; k < W; ++k) Rp[k] = NAN;
                    continue;
                }
                const double ox = (px + 0.5) * spacing, oz = (pz + 0.5) * spacing;
                int jx0 = 0, jx1 = 0, jz0 = 0, jz1 = 0;
                double fx = 0.0, fz = 0.0;
                if (R_up) {
                    upper_weights(px, i, Px_up, &jx0, &jx1, &fx);
                    upper_weights(pz, i, Pz_up, &jz0, &jz1, &fz);
                }
                for (long long k = 0; k < W; ++k) {
                    double wx, wz, I, tau;
                    rco_direction(k, W, &wx, &wz);
                    rco_march(mc, me, nx, nz, voxel, ox, oz, wx, wz, a, b, &I, &tau);
                    ++rays;
                    double Rm = I;
                    if (R_up) {
                        int jz[2] = {jz0, jz1}, jx[2] = {jx0, jx1};
                        double wzz[2] = {1.0 - fz, fz}, wxx[2] = {1.0 - fx, fx};
                        double upper = 0.0;
                        for (int q = 0; q < 2; ++q)
                            for (int r = 0; r < 2; ++r) {
                                const double* Ru = R_up + ((size_t)jz[q] * Px_up + jx[r]) * (size_t)W_up;
                                double avg = 0.0;
                                for (int c = 0; c < branching; ++c) avg += Ru[(size_t)(k * branching + c)];
                                upper += wzz[q] * wxx[r] * avg / (double)branching;
                            }
                        double Im, tm;
                        rco_merge(I, tau, upper, 0.0, &Im, &tm);
                        Rm = Im;
                    }
                    Rp[k] = Rm;
                }
            }
        if (rays_per_level) rays_per_level[i] = rays;
        free(R_up);
        R_up = R;
        Px_up = Px;
        Pz_up = Pz;
        W_up = W;
    }
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix) {
            const size_t c = (size_t)iz * nx + ix;
            double s = 0.0;
            if (active[c])
                for (long long k = 0; k < W_up; ++k) s += R_up[c * (size_t)W_up + (size_t)k];
            J[c] = active[c] ? s / (double)W_up : 0.0;
        }
    free(R_up);
    for (int i = 0; i < n_cascades; ++i) free(F[i]);
    free(F);
    free(mc);
    free(me);
    return 0;
}

/*
 * Emergent intensity along one ray, front to back (Sec. 3.9): the ray o + t w, t >= 0, is
 * cut at the cell faces (as in rco_march) and the pieces are taken from the origin outward;
 * each adds exp(-tau_before) S (1 - exp(-chi ds)) (or exp(-tau_before) eta ds where chi = 0),
 * which is also its value of the contribution function.  contrib (nullable, [nz][nx]) receives
 * the contributions per cell.  Returns the intensity reaching the origin.
 */
double rco_emergent(const double* chi, const double* eta, int nx, int nz, double voxel,
                    double ox, double oz, double wx, double wz, double* contrib)
{
    double t0 = 0.0, t1 = INFINITY;
    if (!clip_to_box(ox, oz, wx, wz, nx, nz, &t0, &t1)) return 0.0;
    double I = 0.0, tau = 0.0, t = t0;
    double tx = next_plane_t(ox, wx, t0), tz = next_plane_t(oz, wz, t0);
    for (;;) {
        double tn = tx < tz ? tx : tz;
        if (tn > t1) tn = t1;
        if (tn > t) {
            const double tm = 0.5 * (t + tn);
            int ix = (int)floor(ox + tm * wx), iz = (int)floor(oz + tm * wz);
            if (ix < 0) ix = 0;
            if (ix >= nx) ix = nx - 1;
            if (iz < 0) iz = 0;
            if (iz >= nz) iz = nz - 1;
            const size_t c = (size_t)iz * nx + ix;
            const double ds = (tn - t) * voxel, dtau = chi[c] * ds;
            const double piece = chi[c] > 0.0 ? exp(-tau) * (eta[c] / chi[c]) * (-expm1(-dtau))
                                              : exp(-tau) * eta[c] * ds;
            I += piece;
            if (contrib) contrib[c] += piece;
            tau += dtau;
        }
        if (!(tn < t1)) break;
        if (tx <= tn) tx = next_plane_t(ox, wx, tn);
        if (tz <= tn) tz = next_plane_t(oz, wz, tn);
        t = tn;
    }
    return I;
}

/* Voxel crossings of every cascade of a plan (geometry only). */
long long rco_count_crossings(int nx, int nz, int n_cascades, int dirs0,
                              int branching, double interval0, int rule,
                              long long* per_level)
{
    long long total = 0;
    for (int i = n_cascades - 1; i >= 0; --i) {
        int Px = rco_probes(nx, i), Pz = rco_probes(nz, i);
        long long W = rco_dirs(dirs0, branching, i);
        double a, b, spacing = (double)(1 << i);
        rco_interval(rule, interval0, branching, i, n_cascades, &a, &b);
        long long lvl = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(+ : lvl)
        for (int pz = 0; pz < Pz; ++pz)
            for (int px = 0; px < Px; ++px)
                for (long long k = 0; k < W; ++k) {
                    double wx, wz;
                    rco_direction(k, W, &wx, &wz);
                    lvl += rco_march(NULL, NULL, nx, nz, 1.0, ((double)px + 0.5) * spacing,
                                     ((double)pz + 0.5) * spacing, wx, wz, a, b, NULL, NULL);
                }
        if (per_level) per_level[i] = lvl;
        total += lvl;
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Brute-force long characteristics (the accuracy yardstick for RC)          */
/* ------------------------------------------------------------------------ */

/* J at every cell centre from n_angles equally spaced in-plane rays, each
 * marched from the centre to the domain edge with the same piecewise-constant
 * update (Sec. 1.1 describes long characteristics; Sec. 3.9 the front-to-back
 * single-pass form).  Converges to the exact angular mean of the voxelised
 * model as n_angles grows. */
int rco_lc_solve(const double* chi, const double* eta, int nx, int nz,
                 double voxel, int n_angles, double* J)
{
    if (nx <= 0 || nz <= 0 || n_angles < 1) return -1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix) {
            double s = 0.0;
            for (int k = 0; k < n_angles; ++k) {
                double wx, wz, I, tau;
                rco_direction(k, n_angles, &wx, &wz);
                rco_march(chi, eta, nx, nz, voxel, ix + 0.5, iz + 0.5, wx, wz, 0.0,
                          INFINITY, &I, &tau);
                s += I;
            }
            J[(size_t)iz * nx + ix] = s / (double)n_angles;
        }
    return 0;
}

int rco_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void rco_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
