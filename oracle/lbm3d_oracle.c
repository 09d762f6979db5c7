/*
 * lbm3d_oracle.c -- plain FP64 CPU oracle of the slip-wall D3Q19 MRT solver
 * (the three-dimensional extension the paper names as future work, Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests may load this library.  It shares
 * no code, header or constant table with the CUDA library.
 *
 * The paper derives its scheme in two dimensions only.  This oracle applies
 * the same steps to the D3Q19 lattice, one node at a time, in the same order
 * as the 2-D oracle:
 *   1. rho = sum f, rho u = sum c f + rho a / 2                 (Eq. FluidMacr)
 *   2. m = M f; m_eq = M f_eq(rho, u); Fbar_i of Eq. LBEforce with c_i;
 *      m' = m - S (m - m_eq) + (I - S/2) M Fbar;  f' = M^-1 m'  (Eq. MomentPost)
 *   3. stream: f_i(x + c_i, t+1) = f'_i(x, t)
 *   4. every boundary link (x_f, i), Eq. EqNewBDSC with the D3Q19 weights:
 *      f_i(x_f,t+1) = r[(1+l-2g)/(1+l) f_ib(x_f,t) + l/(1+l) f'_i(x_f,t)
 *                       + (2g-l)/(1+l) f'_ib(x_f,t) + 2/(1+l) w_i rho_f c_i.u_b / c_s^2]
 *                     + (1-r) f_i^eq(rho_f, u_d),
 *      u_d the fluid velocity of x_f (mode 0) or the wall velocity (mode 1).
 * M: the nineteen moments of the D3Q19 MRT basis of d'Humieres et al. (2002),
 * built here by evaluating their defining polynomials at the velocities:
 *   1, 19|c|^2 - 30, (21|c|^4 - 53|c|^2 + 24)/2, c_x, (5|c|^2 - 9) c_x, c_y,
 *   (5|c|^2 - 9) c_y, c_z, (5|c|^2 - 9) c_z, 3 c_x^2 - |c|^2,
 *   (3|c|^2 - 5)(3 c_x^2 - |c|^2), c_y^2 - c_z^2, (3|c|^2 - 5)(c_y^2 - c_z^2),
 *   c_x c_y, c_y c_z, c_x c_z, (c_y^2 - c_z^2) c_x, (c_z^2 - c_x^2) c_y,
 *   (c_x^2 - c_y^2) c_z;
 * M^-1 by Gauss-Jordan elimination.  Sums over nodes run serially in a fixed
 * order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

static int CX[Q], CY[Q], CZ[Q], OPP[Q];
static double WQ[Q];

/* velocities: rest, the six axes (+x, -x, +y, -y, +z, -z), then the twelve
 * diagonals of the xy, xz and yz planes */
static void init_lattice(void) {
    int k = 0;
    CX[k] = CY[k] = CZ[k] = 0; WQ[k] = 1.0 / 3.0; k++;
    for (int a = 0; a < 3; a++)
        for (int s = 1; s >= -1; s -= 2) {
            CX[k] = a == 0 ? s : 0; CY[k] = a == 1 ? s : 0; CZ[k] = a == 2 ? s : 0;
            WQ[k] = 1.0 / 18.0; k++;
        }
    const int pa[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int p = 0; p < 3; p++)
        for (int s1 = 1; s1 >= -1; s1 -= 2)
            for (int s2 = 1; s2 >= -1; s2 -= 2) {
                int v[3] = {0, 0, 0};
                v[pa[p][0]] = s1; v[pa[p][1]] = s2;
                CX[k] = v[0]; CY[k] = v[1]; CZ[k] = v[2]; WQ[k] = 1.0 / 36.0; k++;
            }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++)
            if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) OPP[i] = j;
}

static double basis(int row, double x, double y, double z) {
    double c2 = x * x + y * y + z * z;
    switch (row) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * c2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * c2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * c2 - 9.0) * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}

typedef struct {
    int nx, ny, nz, px, py, pz;
    uint8_t *solid;
    double ax, ay, az;
    double tau[Q];
    double M[Q][Q], Minv[Q][Q];
    int nl;
    int *lx, *ly, *lz, *ld;
    double *lr, *ll, *lg, *lub;
    double *f, *fpost, *fnew, *fprev, *rho, *ux, *uy, *uz;
    int diffuse_mode;
    long steps;
} o3d;

#define NN(o) ((size_t)(o)->nx * (o)->ny * (o)->nz)
#define NODE(o, x, y, z) (((size_t)(z) * (o)->ny + (size_t)(y)) * (o)->nx + (size_t)(x))
#define IDX(o, i, p) ((size_t)(i) * NN(o) + (p))

static int invert(const double A[Q][Q], double R[Q][Q]) {
    double a[Q][2 * Q];
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < 2 * Q; j++) a[i][j] = j < Q ? A[i][j] : (j - Q == i ? 1.0 : 0.0);
    for (int c = 0; c < Q; c++) {
        int p = c;
        for (int i = c + 1; i < Q; i++)
            if (fabs(a[i][c]) > fabs(a[p][c])) p = i;
        if (a[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < 2 * Q; j++) { double t = a[c][j]; a[c][j] = a[p][j]; a[p][j] = t; }
        double d = a[c][c];
        for (int j = 0; j < 2 * Q; j++) a[c][j] /= d;
        for (int i = 0; i < Q; i++) {
            if (i == c) continue;
            double m = a[i][c];
            if (m != 0.0)
                for (int j = 0; j < 2 * Q; j++) a[i][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) R[i][j] = a[i][j + Q];
    return 0;
}

/* Eq. LBEequi with c_s^2 = 1/3 */
static double feq(int i, double rho, double ux, double uy, double uz) {
    double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
    double uu = ux * ux + uy * uy + uz * uz;
    return WQ[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

static int neighbour(const o3d *o, int x, int y, int z, int dx, int dy, int dz, int *xn, int *yn,
                     int *zn) {
    int a = x + dx, b = y + dy, c = z + dz;
    if (a < 0 || a >= o->nx) { if (!o->px) return 0; a = (a + o->nx) % o->nx; }
    if (b < 0 || b >= o->ny) { if (!o->py) return 0; b = (b + o->ny) % o->ny; }
    if (c < 0 || c >= o->nz) { if (!o->pz) return 0; c = (c + o->nz) % o->nz; }
    *xn = a; *yn = b; *zn = c;
    return 1;
}

void o3d_destroy(o3d *o) {
    if (!o) return;
    free(o->solid); free(o->lx); free(o->ly); free(o->lz); free(o->ld);
    free(o->lr); free(o->ll); free(o->lg); free(o->lub);
    free(o->f); free(o->fpost); free(o->fnew); free(o->fprev);
    free(o->rho); free(o->ux); free(o->uy); free(o->uz);
    free(o);
}

/* Links: n_links entries (x, y, z, dir 1..18, r, l, gamma, u_b[3]).  Returns
 * NULL on bad input (a link whose node is solid or whose neighbour x - c_i
 * is fluid, gamma outside (0, 1], an unknown direction with no link). */
o3d *o3d_create(int nx, int ny, int nz, int px, int py, int pz, const uint8_t *solid, double ax,
                double ay, double az, const double *tau19, int n_links, const int32_t *lx,
                const int32_t *ly, const int32_t *lz, const int32_t *ldir, const double *lr,
                const double *ll, const double *lg, const double *lub, int diffuse_mode) {
    init_lattice();
    if (nx <= 0 || ny <= 0 || nz <= 0 || n_links < 0 || diffuse_mode < 0 || diffuse_mode > 1)
        return NULL;
    o3d *o = (o3d *)calloc(1, sizeof(o3d));
    if (!o) return NULL;
    o->nx = nx; o->ny = ny; o->nz = nz; o->px = px; o->py = py; o->pz = pz;
    o->ax = ax; o->ay = ay; o->az = az; o->diffuse_mode = diffuse_mode;
    memcpy(o->tau, tau19, sizeof(o->tau));
    for (int r = 0; r < Q; r++)
        for (int i = 0; i < Q; i++) o->M[r][i] = basis(r, CX[i], CY[i], CZ[i]);
    if (invert(o->M, o->Minv)) { o3d_destroy(o); return NULL; }
    size_t n = NN(o), nf = (size_t)Q * n, nlb = (size_t)(n_links > 0 ? n_links : 1);
    o->solid = (uint8_t *)malloc(n);
    o->f = (double *)malloc(nf * sizeof(double));
    o->fpost = (double *)malloc(nf * sizeof(double));
    o->fnew = (double *)malloc(nf * sizeof(double));
    o->fprev = (double *)malloc(nf * sizeof(double));
    o->rho = (double *)malloc(n * sizeof(double));
    o->ux = (double *)calloc(n, sizeof(double));
    o->uy = (double *)calloc(n, sizeof(double));
    o->uz = (double *)calloc(n, sizeof(double));
    o->nl = n_links;
    o->lx = (int *)malloc(nlb * sizeof(int)); o->ly = (int *)malloc(nlb * sizeof(int));
    o->lz = (int *)malloc(nlb * sizeof(int)); o->ld = (int *)malloc(nlb * sizeof(int));
    o->lr = (double *)malloc(nlb * sizeof(double)); o->ll = (double *)malloc(nlb * sizeof(double));
    o->lg = (double *)malloc(nlb * sizeof(double)); o->lub = (double *)malloc(3 * nlb * sizeof(double));
    if (!o->solid || !o->f || !o->fpost || !o->fnew || !o->fprev || !o->rho || !o->ux || !o->uy ||
        !o->uz || !o->lx || !o->ly || !o->lz || !o->ld || !o->lr || !o->ll || !o->lg || !o->lub) {
        o3d_destroy(o); return NULL;
    }
    memcpy(o->solid, solid, n);
    unsigned char *cover = (unsigned char *)calloc(nf, 1);
    if (!cover) { o3d_destroy(o); return NULL; }
    int bad = 0;
    for (int k = 0; k < n_links && !bad; k++) {
        int x = lx[k], y = ly[k], z = lz[k], i = ldir[k], xr, yr, zr;
        o->lx[k] = x; o->ly[k] = y; o->lz[k] = z; o->ld[k] = i;
        o->lr[k] = lr[k]; o->ll[k] = ll[k]; o->lg[k] = lg[k];
        memcpy(&o->lub[3 * k], &lub[3 * k], 3 * sizeof(double));
        if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz || i < 1 || i >= Q) { bad = 1; break; }
        if (!(lg[k] > 0.0 && lg[k] <= 1.0)) { bad = 1; break; }
        if (solid[NODE(o, x, y, z)]) { bad = 1; break; }
        if (neighbour(o, x, y, z, -CX[i], -CY[i], -CZ[i], &xr, &yr, &zr) &&
            !solid[NODE(o, xr, yr, zr)]) { bad = 1; break; }
        cover[IDX(o, i, NODE(o, x, y, z))]++;
    }
    for (int z = 0; z < nz && !bad; z++)
        for (int y = 0; y < ny && !bad; y++)
            for (int x = 0; x < nx && !bad; x++) {
                size_t p = NODE(o, x, y, z);
                if (solid[p]) continue;
                for (int i = 1; i < Q; i++) {
                    int xr, yr, zr;
                    int unknown = !neighbour(o, x, y, z, -CX[i], -CY[i], -CZ[i], &xr, &yr, &zr) ||
                                  solid[NODE(o, xr, yr, zr)];
                    if (unknown != (cover[IDX(o, i, p)] == 1)) { bad = 1; break; }
                }
            }
    free(cover);
    if (bad) { o3d_destroy(o); return NULL; }
    for (int i = 0; i < Q; i++)
        for (size_t p = 0; p < n; p++) o->f[IDX(o, i, p)] = WQ[i];
    memcpy(o->fprev, o->f, nf * sizeof(double));
    memcpy(o->fnew, o->f, nf * sizeof(double));
    memcpy(o->fpost, o->f, nf * sizeof(double));
    for (size_t p = 0; p < n; p++) o->rho[p] = 1.0;
    return o;
}

static void collide_node(o3d *o, size_t p) {
    double f[Q], m[Q], fe[Q], Fb[Q], me[Q], MF[Q], mp[Q];
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; i++) {
        f[i] = o->f[IDX(o, i, p)];
        rho += f[i]; jx += CX[i] * f[i]; jy += CY[i] * f[i]; jz += CZ[i] * f[i];
    }
    double ux = (jx + 0.5 * rho * o->ax) / rho;
    double uy = (jy + 0.5 * rho * o->ay) / rho;
    double uz = (jz + 0.5 * rho * o->az) / rho;
    double ua = ux * o->ax + uy * o->ay + uz * o->az;
    for (int i = 0; i < Q; i++) {
        fe[i] = feq(i, rho, ux, uy, uz);
        double ca = CX[i] * o->ax + CY[i] * o->ay + CZ[i] * o->az;
        double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
        /* Eq. LBEforce: w rho [c.a / cs^2 + (u a):(c c - cs^2 I) / cs^4] */
        Fb[i] = WQ[i] * rho * (3.0 * ca + 9.0 * (cu * ca - ua / 3.0));
    }
    for (int k = 0; k < Q; k++) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < Q; i++) {
            a += o->M[k][i] * f[i]; b += o->M[k][i] * fe[i]; c += o->M[k][i] * Fb[i];
        }
        m[k] = a; me[k] = b; MF[k] = c;
    }
    for (int k = 0; k < Q; k++) {
        double s = 1.0 / o->tau[k];
        mp[k] = m[k] - s * (m[k] - me[k]) + (1.0 - 0.5 * s) * MF[k];
    }
    for (int i = 0; i < Q; i++) {
        double a = 0.0;
        for (int k = 0; k < Q; k++) a += o->Minv[i][k] * mp[k];
        o->fpost[IDX(o, i, p)] = a;
    }
    o->rho[p] = rho; o->ux[p] = ux; o->uy[p] = uy; o->uz[p] = uz;
}

void o3d_step(o3d *o, long nsteps) {
    size_t n = NN(o);
    for (long s = 0; s < nsteps; s++) {
        for (size_t p = 0; p < n; p++)
            if (!o->solid[p]) collide_node(o, p);
        for (size_t p = 0; p < n; p++)
            if (o->solid[p])
                for (int i = 0; i < Q; i++) o->fnew[IDX(o, i, p)] = o->f[IDX(o, i, p)];
        for (int z = 0; z < o->nz; z++)
            for (int y = 0; y < o->ny; y++)
                for (int x = 0; x < o->nx; x++) {
                    size_t p = NODE(o, x, y, z);
                    if (o->solid[p]) continue;
                    o->fnew[IDX(o, 0, p)] = o->fpost[IDX(o, 0, p)];
                    for (int i = 1; i < Q; i++) {
                        int xn, yn, zn;
                        if (neighbour(o, x, y, z, CX[i], CY[i], CZ[i], &xn, &yn, &zn) &&
                            !o->solid[NODE(o, xn, yn, zn)])
                            o->fnew[IDX(o, i, NODE(o, xn, yn, zn))] = o->fpost[IDX(o, i, p)];
                    }
                }
        for (int k = 0; k < o->nl; k++) {
            size_t p = NODE(o, o->lx[k], o->ly[k], o->lz[k]);
            int i = o->ld[k], ib = OPP[i];
            double r = o->lr[k], l = o->ll[k], g = o->lg[k];
            const double *ub = &o->lub[3 * k];
            double rhof = o->rho[p];
            double cub = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
            double bb = (1.0 + l - 2.0 * g) / (1.0 + l) * o->f[IDX(o, ib, p)] +
                        l / (1.0 + l) * o->fpost[IDX(o, i, p)] +
                        (2.0 * g - l) / (1.0 + l) * o->fpost[IDX(o, ib, p)] +
                        2.0 / (1.0 + l) * WQ[i] * rhof * cub * 3.0;
            double ud[3] = {ub[0], ub[1], ub[2]};
            if (o->diffuse_mode == 0) { ud[0] = o->ux[p]; ud[1] = o->uy[p]; ud[2] = o->uz[p]; }
            o->fnew[IDX(o, i, p)] = r * bb + (1.0 - r) * feq(i, rhof, ud[0], ud[1], ud[2]);
        }
        double *t = o->fprev; o->fprev = o->f; o->f = o->fnew; o->fnew = t;
        o->steps++;
    }
}

void o3d_fields(const o3d *o, double *rho, double *ux, double *uy, double *uz) {
    size_t n = NN(o);
    for (size_t p = 0; p < n; p++) {
        if (o->solid[p]) { rho[p] = ux[p] = uy[p] = uz[p] = 0.0; continue; }
        double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
        for (int i = 0; i < Q; i++) {
            double v = o->f[IDX(o, i, p)];
            r += v; jx += CX[i] * v; jy += CY[i] * v; jz += CZ[i] * v;
        }
        rho[p] = r;
        ux[p] = (jx + 0.5 * r * o->ax) / r;
        uy[p] = (jy + 0.5 * r * o->ay) / r;
        uz[p] = (jz + 0.5 * r * o->az) / r;
    }
}

/* residual = ||u^n - u^(n-1)|| / ||u^n|| over fluid nodes; mass = sum of all
 * populations of fluid nodes.  Serial fixed-order sums. */
void o3d_residual(const o3d *o, double *residual, double *mass) {
    size_t n = NN(o);
    double num = 0.0, den = 0.0, ms = 0.0;
    for (size_t p = 0; p < n; p++) {
        if (o->solid[p]) continue;
        double r1 = 0, r0 = 0, j1[3] = {0, 0, 0}, j0[3] = {0, 0, 0};
        for (int i = 0; i < Q; i++) {
            double a = o->f[IDX(o, i, p)], b = o->fprev[IDX(o, i, p)];
            r1 += a; r0 += b;
            j1[0] += CX[i] * a; j1[1] += CY[i] * a; j1[2] += CZ[i] * a;
            j0[0] += CX[i] * b; j0[1] += CY[i] * b; j0[2] += CZ[i] * b;
        }
        double acc[3] = {o->ax, o->ay, o->az};
        for (int d = 0; d < 3; d++) {
            double u1 = (j1[d] + 0.5 * r1 * acc[d]) / r1, u0 = (j0[d] + 0.5 * r0 * acc[d]) / r0;
            num += (u1 - u0) * (u1 - u0);
            den += u1 * u1;
        }
        ms += r1;
    }
    if (isnan(num) || isnan(den)) *residual = NAN;
    else *residual = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
    *mass = ms;
}

/* f in [19][nz][ny][nx] order */
void o3d_get_f(const o3d *o, double *f) { memcpy(f, o->f, (size_t)Q * NN(o) * sizeof(double)); }

void o3d_set_f(o3d *o, const double *f) {
    memcpy(o->f, f, (size_t)Q * NN(o) * sizeof(double));
    memcpy(o->fprev, f, (size_t)Q * NN(o) * sizeof(double));
}

void o3d_get_m(const o3d *o, double *m) { memcpy(m, o->M, sizeof(o->M)); }

void o3d_lattice(int32_t *c, double *w) {
    init_lattice();
    for (int i = 0; i < Q; i++) {
        c[3 * i] = CX[i]; c[3 * i + 1] = CY[i]; c[3 * i + 2] = CZ[i]; w[i] = WQ[i];
    }
}

long o3d_steps(const o3d *o) { return o->steps; }
