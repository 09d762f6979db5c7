/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the slip-wall D2Q9 MRT solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant table with the CUDA library; both consume the same
 * seeded inputs (mask, links, per-link parameters) and nothing else.
 *
 * Each step follows the paper's order (Sec. 2 then Sec. 3.A), one node at a
 * time, with no fusion or reordering:
 *   1. rho = sum f, rho u = sum c f + rho a / 2                (Eq. FluidMacr)
 *   2. m = M f; m_eq = M f_eq(rho, u)                          (Eq. LBEequi)
 *      Fbar_i from Eq. LBEforce (with c_i in the first term), F^ = (I - S/2) M Fbar
 *      m' = m - S (m - m_eq) + F^;  f' = M^-1 m'               (Eq. MomentPost)
 *   3. stream: f_i(x + c_i, t+1) = f'_i(x, t)                  (collision/streaming split)
 *   4. every boundary link (x_f, i):                           (Eq. EqNewBDSC)
 *      f_i(x_f,t+1) = r[(1+l-2g)/(1+l) f_ib(x_f,t) + l/(1+l) f'_i(x_f,t)
 *                       + (2g-l)/(1+l) f'_ib(x_f,t) + 2/(1+l) w_i rho_f c_i.u_b / c_s^2]
 *                     + (1-r) f_i^eq(rho_f, u_b)
 *      with f_ib(x_f,t) the pre-collision value at time t and rho_f = sum_i f_i(x_f,t).
 *      The Maxwell part f_i^eq is evaluated at (rho_f, u_d): u_d is the fluid
 *      velocity of x_f at time t (Eq. FluidMacr) in mode 0, under which the
 *      channel analysis of Sec. 3.B (Eq. u1u0Coeff onward) holds exactly, or the
 *      wall velocity u_b as printed in Eq. EqNewBDSC in mode 1.
 * M^-1 is obtained once by Gauss-Jordan elimination of the printed M.
 * Sums over nodes (residual, mass) run serially in a fixed order.
 *
 * The same source builds single-threaded and, with -fopenmp, with the row
 * loops of a step spread over threads: every node's arithmetic is the same
 * and every destination is written by exactly one iteration, so both builds
 * give bitwise the same states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int CXs[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CYs[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPPs[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double Ws[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const double Mprinted[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},  {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

typedef struct {
    int nx, ny, px, py;
    uint8_t *solid;
    double ax, ay;
    double tau[9];
    double M[9][9], Minv[9][9];
    int nl;
    int *lx, *ly, *ld;
    double *lr, *ll, *lg, *lubx, *luby;
    double *f, *fpost, *fnew, *fprev, *rho, *ux, *uy;
    double *snap_ux, *snap_uy; /* velocity at the last interval residual */
    long snap_steps;
    int diffuse_mode;
    long steps;
} olbm;

#define IDX(o, i, x, y) (((size_t)(i) * (o)->ny + (size_t)(y)) * (o)->nx + (size_t)(x))

static int invert9(const double A[9][9], double R[9][9]) {
    double a[9][18];
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 18; j++) a[i][j] = j < 9 ? A[i][j] : (j - 9 == i ? 1.0 : 0.0);
    for (int c = 0; c < 9; c++) {
        int p = c;
        for (int i = c + 1; i < 9; i++)
            if (fabs(a[i][c]) > fabs(a[p][c])) p = i;
        if (a[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < 18; j++) {
                double t = a[c][j]; a[c][j] = a[p][j]; a[p][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 18; j++) a[c][j] /= d;
        for (int i = 0; i < 9; i++) {
            if (i == c) continue;
            double m = a[i][c];
            if (m != 0.0)
                for (int j = 0; j < 18; j++) a[i][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < 9; i++)
        for (int j = 0; j < 9; j++) R[i][j] = a[i][j + 9];
    return 0;
}

/* Eq. LBEequi with c_s^2 = 1/3. */
static double feq(int i, double rho, double ux, double uy) {
    double cu = CXs[i] * ux + CYs[i] * uy;
    double uu = ux * ux + uy * uy;
    return Ws[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* neighbour of (x, y) along (dx, dy); returns 0 when it leaves a
 * non-periodic domain. */
static int neighbour(const olbm *o, int x, int y, int dx, int dy, int *xn, int *yn) {
    int a = x + dx, b = y + dy;
    if (a < 0 || a >= o->nx) {
        if (!o->px) return 0;
        a = (a + o->nx) % o->nx;
    }
    if (b < 0 || b >= o->ny) {
        if (!o->py) return 0;
        b = (b + o->ny) % o->ny;
    }
    *xn = a; *yn = b;
    return 1;
}

void olbm_destroy(olbm *o) {
    if (!o) return;
    free(o->solid); free(o->lx); free(o->ly); free(o->ld);
    free(o->lr); free(o->ll); free(o->lg); free(o->lubx); free(o->luby);
    free(o->f); free(o->fpost); free(o->fnew); free(o->fprev); free(o->rho);
    free(o->ux); free(o->uy); free(o->snap_ux); free(o->snap_uy);
    free(o);
}

static void current_velocity(const olbm *o, double *ux, double *uy);

/* Returns NULL on bad input (a link that is not a fluid node next to a
 * solid one, gamma outside (0, 1], or an unknown direction with no link). */
olbm *olbm_create(int nx, int ny, int periodic_x, int periodic_y, const uint8_t *solid,
                  double ax, double ay, const double *tau9, int n_links, const int32_t *lx,
                  const int32_t *ly, const int32_t *ldir, const double *lr, const double *ll,
                  const double *lg, const double *lubx, const double *luby,
                  int diffuse_mode) {
    if (nx <= 0 || ny <= 0 || n_links < 0 || diffuse_mode < 0 || diffuse_mode > 1) return NULL;
    olbm *o = (olbm *)calloc(1, sizeof(olbm));
    if (!o) return NULL;
    size_t n = (size_t)nx * ny, nf = 9 * n;
    o->nx = nx; o->ny = ny; o->px = periodic_x; o->py = periodic_y;
    o->ax = ax; o->ay = ay;
    o->diffuse_mode = diffuse_mode;
    memcpy(o->tau, tau9, sizeof(o->tau));
    memcpy(o->M, Mprinted, sizeof(o->M));
    if (invert9(o->M, o->Minv)) { olbm_destroy(o); return NULL; }
    o->solid = (uint8_t *)malloc(n);
    o->f = (double *)malloc(nf * sizeof(double));
    o->fpost = (double *)malloc(nf * sizeof(double));
    o->fnew = (double *)malloc(nf * sizeof(double));
    o->fprev = (double *)malloc(nf * sizeof(double));
    o->rho = (double *)malloc(n * sizeof(double));
    o->ux = (double *)calloc(n, sizeof(double));
    o->uy = (double *)calloc(n, sizeof(double));
    o->snap_ux = (double *)calloc(n, sizeof(double));
    o->snap_uy = (double *)calloc(n, sizeof(double));
    size_t nlb = (size_t)(n_links > 0 ? n_links : 1);
    o->nl = n_links;
    o->lx = (int *)malloc(nlb * sizeof(int)); o->ly = (int *)malloc(nlb * sizeof(int));
    o->ld = (int *)malloc(nlb * sizeof(int));
    o->lr = (double *)malloc(nlb * sizeof(double)); o->ll = (double *)malloc(nlb * sizeof(double));
    o->lg = (double *)malloc(nlb * sizeof(double));
    o->lubx = (double *)malloc(nlb * sizeof(double)); o->luby = (double *)malloc(nlb * sizeof(double));
    if (!o->solid || !o->f || !o->fpost || !o->fnew || !o->fprev || !o->rho || !o->ux || !o->uy ||
        !o->snap_ux || !o->snap_uy || !o->lx ||
        !o->ly || !o->ld || !o->lr || !o->ll || !o->lg || !o->lubx || !o->luby) {
        olbm_destroy(o); return NULL;
    }
    memcpy(o->solid, solid, n);
    /* coverage[i][node]: how many links claim unknown (node, i) */
    unsigned char *cover = (unsigned char *)calloc(nf, 1);
    if (!cover) { olbm_destroy(o); return NULL; }
    int bad = 0;
    for (int k = 0; k < n_links; k++) {
        int x = lx[k], y = ly[k], i = ldir[k], xr, yr;
        o->lx[k] = x; o->ly[k] = y; o->ld[k] = i;
        o->lr[k] = lr[k]; o->ll[k] = ll[k]; o->lg[k] = lg[k];
        o->lubx[k] = lubx[k]; o->luby[k] = luby[k];
        if (x < 0 || x >= nx || y < 0 || y >= ny || i < 1 || i > 8) { bad = 1; break; }
        if (!(lg[k] > 0.0 && lg[k] <= 1.0)) { bad = 1; break; }
        if (solid[(size_t)y * nx + x]) { bad = 1; break; }
        if (neighbour(o, x, y, -CXs[i], -CYs[i], &xr, &yr) && !solid[(size_t)yr * nx + xr]) {
            bad = 1; break;
        }
        cover[IDX(o, i, x, y)]++;
    }
    for (int y = 0; y < ny && !bad; y++)
        for (int x = 0; x < nx && !bad; x++) {
            if (solid[(size_t)y * nx + x]) continue;
            for (int i = 1; i < 9; i++) {
                int xr, yr;
                int unknown = !neighbour(o, x, y, -CXs[i], -CYs[i], &xr, &yr) ||
                              solid[(size_t)yr * nx + xr];
                if (unknown != (cover[IDX(o, i, x, y)] == 1)) { bad = 1; break; }
            }
        }
    free(cover);
    if (bad) { olbm_destroy(o); return NULL; }
    /* initial state f = f_eq(1, 0) = w_i everywhere */
    for (int i = 0; i < 9; i++)
        for (size_t p = 0; p < n; p++) o->f[(size_t)i * n + p] = Ws[i];
    memcpy(o->fprev, o->f, nf * sizeof(double));
    memcpy(o->fnew, o->f, nf * sizeof(double));
    memcpy(o->fpost, o->f, nf * sizeof(double));
    for (size_t p = 0; p < n; p++) o->rho[p] = 1.0;
    /* the initial state is the first reference of the interval residual */
    current_velocity(o, o->snap_ux, o->snap_uy);
    return o;
}

static void collide_node(olbm *o, int x, int y) {
    double f[9], m[9], fe[9], me[9], Fb[9], MF[9], mp[9];
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
        f[i] = o->f[IDX(o, i, x, y)];
        rho += f[i];
        jx += CXs[i] * f[i];
        jy += CYs[i] * f[i];
    }
    double ux = (jx + 0.5 * rho * o->ax) / rho;
    double uy = (jy + 0.5 * rho * o->ay) / rho;
    double ua = ux * o->ax + uy * o->ay;
    for (int i = 0; i < 9; i++) {
        fe[i] = feq(i, rho, ux, uy);
        double ca = CXs[i] * o->ax + CYs[i] * o->ay;
        double cu = CXs[i] * ux + CYs[i] * uy;
        /* Eq. LBEforce: w rho [c.a / cs^2 + (u a):(c c - cs^2 I) / cs^4] */
        Fb[i] = Ws[i] * rho * (3.0 * ca + 9.0 * (cu * ca - ua / 3.0));
    }
    for (int k = 0; k < 9; k++) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < 9; i++) {
            a += o->M[k][i] * f[i];
            b += o->M[k][i] * fe[i];
            c += o->M[k][i] * Fb[i];
        }
        m[k] = a; me[k] = b; MF[k] = c;
    }
    for (int k = 0; k < 9; k++) {
        double s = 1.0 / o->tau[k];
        mp[k] = m[k] - s * (m[k] - me[k]) + (1.0 - 0.5 * s) * MF[k];
    }
    for (int i = 0; i < 9; i++) {
        double a = 0.0;
        for (int k = 0; k < 9; k++) a += o->Minv[i][k] * mp[k];
        o->fpost[IDX(o, i, x, y)] = a;
    }
    o->rho[(size_t)y * o->nx + x] = rho;
    o->ux[(size_t)y * o->nx + x] = ux;
    o->uy[(size_t)y * o->nx + x] = uy;
}

void olbm_step(olbm *o, long nsteps) {
    int nx = o->nx, ny = o->ny;
    for (long s = 0; s < nsteps; s++) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                if (!o->solid[(size_t)y * nx + x]) collide_node(o, x, y);
        /* solid nodes keep their values */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                if (o->solid[(size_t)y * nx + x])
                    for (int i = 0; i < 9; i++) o->fnew[IDX(o, i, x, y)] = o->f[IDX(o, i, x, y)];
        /* streaming (each fluid destination has exactly one source) */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                if (o->solid[(size_t)y * nx + x]) continue;
                o->fnew[IDX(o, 0, x, y)] = o->fpost[IDX(o, 0, x, y)];
                for (int i = 1; i < 9; i++) {
                    int xn, yn;
                    if (neighbour(o, x, y, CXs[i], CYs[i], &xn, &yn) &&
                        !o->solid[(size_t)yn * nx + xn])
                        o->fnew[IDX(o, i, xn, yn)] = o->fpost[IDX(o, i, x, y)];
                }
            }
        /* boundary links, Eq. EqNewBDSC (one link per unknown population) */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < o->nl; k++) {
            int x = o->lx[k], y = o->ly[k], i = o->ld[k], ib = OPPs[i];
            double r = o->lr[k], l = o->ll[k], g = o->lg[k];
            double rhof = o->rho[(size_t)y * nx + x];
            double cub = CXs[i] * o->lubx[k] + CYs[i] * o->luby[k];
            double bb = (1.0 + l - 2.0 * g) / (1.0 + l) * o->f[IDX(o, ib, x, y)] +
                        l / (1.0 + l) * o->fpost[IDX(o, i, x, y)] +
                        (2.0 * g - l) / (1.0 + l) * o->fpost[IDX(o, ib, x, y)] +
                        2.0 / (1.0 + l) * Ws[i] * rhof * cub * 3.0;
            double udx = o->lubx[k], udy = o->luby[k];
            if (o->diffuse_mode == 0) {
                udx = o->ux[(size_t)y * nx + x];
                udy = o->uy[(size_t)y * nx + x];
            }
            o->fnew[IDX(o, i, x, y)] = r * bb + (1.0 - r) * feq(i, rhof, udx, udy);
        }
        double *t = o->fprev;
        o->fprev = o->f;
        o->f = o->fnew;
        o->fnew = t;
        o->steps++;
    }
}

/* density and half-force velocity of every node (solid nodes: 0). */
void olbm_fields(const olbm *o, double *rho, double *ux, double *uy) {
    size_t n = (size_t)o->nx * o->ny;
    for (size_t p = 0; p < n; p++) {
        if (o->solid[p]) { rho[p] = ux[p] = uy[p] = 0.0; continue; }
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; i++) {
            double v = o->f[(size_t)i * n + p];
            r += v; jx += CXs[i] * v; jy += CYs[i] * v;
        }
        rho[p] = r;
        ux[p] = (jx + 0.5 * r * o->ax) / r;
        uy[p] = (jy + 0.5 * r * o->ay) / r;
    }
}

/* residual = ||u^n - u^(n-1)||_2 / ||u^n||_2 over fluid nodes; mass = sum of
 * all populations of fluid nodes.  Serial fixed-order sums. */
void olbm_residual(const olbm *o, double *residual, double *mass) {
    size_t n = (size_t)o->nx * o->ny;
    double num = 0.0, den = 0.0, ms = 0.0;
    for (size_t p = 0; p < n; p++) {
        if (o->solid[p]) continue;
        double r1 = 0, x1 = 0, y1 = 0, r0 = 0, x0 = 0, y0 = 0;
        for (int i = 0; i < 9; i++) {
            double a = o->f[(size_t)i * n + p], b = o->fprev[(size_t)i * n + p];
            r1 += a; x1 += CXs[i] * a; y1 += CYs[i] * a;
            r0 += b; x0 += CXs[i] * b; y0 += CYs[i] * b;
        }
        double ux1 = (x1 + 0.5 * r1 * o->ax) / r1, uy1 = (y1 + 0.5 * r1 * o->ay) / r1;
        double ux0 = (x0 + 0.5 * r0 * o->ax) / r0, uy0 = (y0 + 0.5 * r0 * o->ay) / r0;
        num += (ux1 - ux0) * (ux1 - ux0) + (uy1 - uy0) * (uy1 - uy0);
        den += ux1 * ux1 + uy1 * uy1;
        ms += r1;
    }
    if (isnan(num) || isnan(den))
        *residual = NAN;
    else
        *residual = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
    *mass = ms;
}

/* Velocity of every node from the current populations (solid: 0). */
static void current_velocity(const olbm *o, double *ux, double *uy) {
    size_t n = (size_t)o->nx * o->ny;
    for (size_t p = 0; p < n; p++) {
        ux[p] = uy[p] = 0.0;
        if (o->solid[p]) continue;
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; i++) {
            double v = o->f[(size_t)i * n + p];
            r += v; jx += CXs[i] * v; jy += CYs[i] * v;
        }
        ux[p] = (jx + 0.5 * r * o->ax) / r;
        uy[p] = (jy + 0.5 * r * o->ay) / r;
    }
}

/* Interval residual: ||u^n - u^m||_2 / ((n - m) ||u^n||_2) over fluid nodes,
 * u^m the velocity at the previous call (the initial state before the
 * first), then u^n becomes the reference.  0 when no step was taken since.
 * Serial fixed-order sums. */
void olbm_residual_interval(olbm *o, double *residual) {
    size_t n = (size_t)o->nx * o->ny;
    double *ux = (double *)malloc(n * sizeof(double)), *uy = (double *)malloc(n * sizeof(double));
    if (!ux || !uy) { free(ux); free(uy); *residual = NAN; return; }
    current_velocity(o, ux, uy);
    double num = 0.0, den = 0.0;
    for (size_t p = 0; p < n; p++) {
        if (o->solid[p]) continue;
        double dx = ux[p] - o->snap_ux[p], dy = uy[p] - o->snap_uy[p];
        num += dx * dx + dy * dy;
        den += ux[p] * ux[p] + uy[p] * uy[p];
    }
    long span = o->steps - o->snap_steps;
    if (isnan(num) || isnan(den))
        *residual = NAN;
    else if (span <= 0)
        *residual = 0.0;
    else
        *residual = (den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0)) / (double)span;
    memcpy(o->snap_ux, ux, n * sizeof(double));
    memcpy(o->snap_uy, uy, n * sizeof(double));
    o->snap_steps = o->steps;
    free(ux); free(uy);
}

/* f in [9][ny][nx] order. */
void olbm_get_f(const olbm *o, double *f) {
    memcpy(f, o->f, 9 * (size_t)o->nx * o->ny * sizeof(double));
}

void olbm_set_f(olbm *o, const double *f) {
    size_t nf = 9 * (size_t)o->nx * o->ny;
    memcpy(o->f, f, nf * sizeof(double));
    memcpy(o->fprev, f, nf * sizeof(double));
    current_velocity(o, o->snap_ux, o->snap_uy);
    o->snap_steps = o->steps;
}

/* post-collision populations of the last step, [9][ny][nx] */
void olbm_get_fpost(const olbm *o, double *f) {
    memcpy(f, o->fpost, 9 * (size_t)o->nx * o->ny * sizeof(double));
}

void olbm_get_minv(const olbm *o, double *minv) { memcpy(minv, o->Minv, sizeof(o->Minv)); }

long olbm_steps(const olbm *o) { return o->steps; }

/* Threads of the row loops (the OpenMP build; 1 in the single-threaded one). */
void olbm_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int olbm_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
