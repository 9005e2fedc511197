/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the D2Q9 Shan-Chen electrowetting
 * update of Li, Li, Chen & Fang, "Lattice Boltzmann simulation of
 * electrowetting-on-dielectric in a rough-wall channel" (arXiv:0708.4182).
 *
 * TEST INFRASTRUCTURE. This file exists to check the CUDA library, not to be
 * used by it. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it. It shares no source, header or helper with the GPU path.
 *
 * Each time step is written as the paper orders it, one lattice-wide phase per
 * function, in double precision, with no blocking or fusion:
 *   1. moments rho, rho*u                      (Eq. 2)
 *   2. pseudopotential psi = rho0(1-exp(-rho/rho0))   (text after Eq. 4)
 *   3. forces  F_sigma (Eq. 5), F_w (Eq. 6), electric force f*n on the
 *      conductive single layer (Eq. 9 and the paragraph that defines rho_c),
 *      plus the channel body force
 *   4. velocity shift  rho*u' = rho*u + tau*F   (Eq. 10)
 *   5. BGK collision towards f_eq(rho, u')     (Eq. 1, Eq. 3)
 *   6. streaming f(x+e_a, t+1) = f*(x, t), periodic in x and y, with half-way
 *      bounce-back where x+e_a is solid      (left side of Eq. 1)
 *
 * Readings where the paper is silent or inconsistent (each is also a parameter
 * or stated here):
 *   - Green-function magnitudes. With the printed weights (2G on axis links, G on
 *     diagonals) the paper's G = -0.52 lies ~3x past the critical strength and
 *     the scheme diverges; Martys & Chen, whom the paper cites for Eq. 6, use G
 *     on axis links and G/2 on diagonals. green = ORC_GREEN_MC (default) takes
 *     that convention for both G_a and W_a; ORC_GREEN_PRINTED takes the printed
 *     one.
 *   - psi of a solid node is 0 in Eq. 5; solids act only through S in Eq. 6.
 *   - The electric force acts on fluid nodes with rho >= rho_c that have at
 *     least one solid axis neighbour; per solid axis face it contributes f
 *     along that face's outward direction towards the wall (the electrode), so
 *     a flat bottom wall gives (0,-f) and a concave corner gets both faces
 *     (normal = ORC_NORMAL_FACES). normal = ORC_NORMAL_UNIT takes the other
 *     reading of "f n" with n a unit vector: the same sum of face directions
 *     scaled to length 1, so a concave corner gets f along the diagonal;
 *     the two readings differ only where two perpendicular faces meet.
 *   - The body force is rho*(body_fx, body_fy) on every fluid node and enters
 *     through the same tau-shift as Eq. 10.
 *   - Walls use half-way link bounce-back (not stated in the paper).
 *   - Observables use the physical velocity u = (sum_a f_a e_a + F/2)/rho and
 *     Q = (1/nx) * sum over fluid nodes of u_x  (Eq. 11 with L = nx).
 *
 * Layout: populations f[a][y][x] (a = 0..8, row-major, x fastest), double.
 * Solid mask solid[y][x], 1 = solid. Solid nodes carry f = 0.
 * Directions (Eq. in the D2Q9 paragraph): e0=(0,0), e1..e4 = (1,0),(0,1),
 * (-1,0),(0,-1), e5..e8 = (1,1),(-1,1),(-1,-1),(1,-1).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q9 9

typedef struct {
    int32_t nx, ny;
    double tau;       /* relaxation time of Eq. 1 */
    double G;         /* fluid-fluid strength, calligraphic G of Eq. 4 */
    double G_wall;    /* fluid-wall strength w of Eq. 6 */
    double rho0;      /* constant of psi */
    double rho_c;     /* critical (conductive) density */
    double f_elec;    /* electric force per wall node f of Eq. 9 */
    double body_fx;   /* body-force acceleration (channel runs) */
    double body_fy;
    int32_t green;    /* ORC_GREEN_MC or ORC_GREEN_PRINTED */
    int32_t normal;   /* ORC_NORMAL_FACES or ORC_NORMAL_UNIT (electric-force direction) */
} orc_params;

enum { ORC_GREEN_MC = 0, ORC_GREEN_PRINTED = 1 };
enum { ORC_NORMAL_FACES = 0, ORC_NORMAL_UNIT = 1 };

static const int EX[Q9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[Q9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WEQ[Q9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* Link weight of the Green function (Eq. 4) or of W_a (Eq. 6) for direction a,
 * given the strength s: axis links |e|=1, diagonal links |e|=sqrt(2). */
static double link_weight(const orc_params *p, double s, int a)
{
    if (a == 0) return 0.0;
    int axis = (a <= 4);
    if (p->green == ORC_GREEN_PRINTED) return axis ? 2.0 * s : s;
    return axis ? s : 0.5 * s;
}

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

static size_t node(const orc_params *p, int x, int y) { return (size_t)y * p->nx + x; }

/* Eq. 3 for one node: equilibrium population a at density rho, velocity u. */
static double feq(int a, double rho, double ux, double uy)
{
    double eu = EX[a] * ux + EY[a] * uy;
    double uu = ux * ux + uy * uy;
    return WEQ[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

int orc_equilibrium(const orc_params *p, const uint8_t *solid, const double *rho,
                    const double *ux, const double *uy, double *f)
{
    size_t n = (size_t)p->nx * p->ny;
    for (size_t i = 0; i < n; ++i)
        for (int a = 0; a < Q9; ++a)
            f[a * n + i] = solid[i] ? 0.0 : feq(a, rho[i], ux[i], uy[i]);
    return 0;
}

/* Phase 1, Eq. 2: rho = sum_a f_a, j = rho*u = sum_a f_a e_a. */
static void moments(const orc_params *p, const uint8_t *solid, const double *f,
                    double *rho, double *jx, double *jy)
{
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n; ++i) {
        double r = 0, mx = 0, my = 0;
        if (!solid[i])
            for (int a = 0; a < Q9; ++a) {
                double fa = f[a * n + i];
                r += fa;
                mx += fa * EX[a];
                my += fa * EY[a];
            }
        rho[i] = r;
        jx[i] = mx;
        jy[i] = my;
    }
}

/* Phase 2: psi(x) = rho0 (1 - exp(-rho/rho0)) on fluid nodes, 0 on solids. */
static void pseudopotential(const orc_params *p, const uint8_t *solid, const double *rho,
                            double *psi)
{
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n; ++i)
        psi[i] = solid[i] ? 0.0 : p->rho0 * (1.0 - exp(-rho[i] / p->rho0));
}

/* Phase 3: the four force terms on every fluid node.
 * F_sigma = -psi(x) sum_a G_a psi(x+e_a) e_a                 (Eq. 5)
 * F_w     = -psi(x) sum_a W_a S(x+e_a) e_a                   (Eq. 6)
 * f_e     = f * sum_{a=1..4, S(x+e_a)=1} e_a  if rho >= rho_c (EWOD layer force)
 * F_b     = rho * (body_fx, body_fy)
 * terms[k*n + i], k = 0..7 : Fs_x, Fs_y, Fw_x, Fw_y, fe_x, fe_y, Fb_x, Fb_y. */
static void forces(const orc_params *p, const uint8_t *solid, const double *rho,
                   const double *psi, double *terms)
{
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            size_t i = node(p, x, y);
            double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (!solid[i]) {
                double sgx = 0, sgy = 0, swx = 0, swy = 0, sex = 0, sey = 0;
                for (int a = 1; a < Q9; ++a) {
                    size_t j = node(p, wrap(x + EX[a], p->nx), wrap(y + EY[a], p->ny));
                    double S = solid[j] ? 1.0 : 0.0;
                    double g = link_weight(p, p->G, a);
                    double w = link_weight(p, p->G_wall, a);
                    sgx += g * psi[j] * EX[a];
                    sgy += g * psi[j] * EY[a];
                    swx += w * S * EX[a];
                    swy += w * S * EY[a];
                    if (a <= 4) {
                        sex += S * EX[a];
                        sey += S * EY[a];
                    }
                }
                t[0] = -psi[i] * sgx;
                t[1] = -psi[i] * sgy;
                t[2] = -psi[i] * swx;
                t[3] = -psi[i] * swy;
                if (rho[i] >= p->rho_c) {
                    double len = 1.0;
                    if (p->normal == ORC_NORMAL_UNIT && (sex != 0.0 || sey != 0.0))
                        len = sqrt(sex * sex + sey * sey);
                    t[4] = p->f_elec * sex / len;
                    t[5] = p->f_elec * sey / len;
                }
                t[6] = rho[i] * p->body_fx;
                t[7] = rho[i] * p->body_fy;
            }
            for (int k = 0; k < 8; ++k) terms[k * n + i] = t[k];
        }
    }
}

static void total_force(size_t n, const double *terms, size_t i, double *Fx, double *Fy)
{
    *Fx = terms[0 * n + i] + terms[2 * n + i] + terms[4 * n + i] + terms[6 * n + i];
    *Fy = terms[1 * n + i] + terms[3 * n + i] + terms[5 * n + i] + terms[7 * n + i];
}

/* Phases 4-5: u' = (j + tau F)/rho (Eq. 10), f* = f - (f - f_eq(rho,u'))/tau (Eq. 1). */
static void collide(const orc_params *p, const uint8_t *solid, const double *f,
                    const double *rho, const double *jx, const double *jy,
                    const double *terms, double *fstar)
{
    size_t n = (size_t)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n; ++i) {
        if (solid[i]) {
            for (int a = 0; a < Q9; ++a) fstar[a * n + i] = 0.0;
            continue;
        }
        double Fx, Fy;
        total_force(n, terms, (size_t)i, &Fx, &Fy);
        double upx = (jx[i] + p->tau * Fx) / rho[i];
        double upy = (jy[i] + p->tau * Fy) / rho[i];
        for (int a = 0; a < Q9; ++a) {
            double fa = f[a * n + i];
            fstar[a * n + i] = fa - (fa - feq(a, rho[i], upx, upy)) / p->tau;
        }
    }
}

/* Phase 6: f_a(x+e_a, t+1) = f*_a(x, t); if x+e_a is solid the population
 * returns along the same link: f_{opp(a)}(x, t+1) = f*_a(x, t). */
static void stream(const orc_params *p, const uint8_t *solid, const double *fstar, double *f)
{
    size_t n = (size_t)p->nx * p->ny;
    memset(f, 0, sizeof(double) * Q9 * n);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; ++y) {
        for (int x = 0; x < p->nx; ++x) {
            size_t i = node(p, x, y);
            if (solid[i]) continue;
            for (int a = 0; a < Q9; ++a) {
                size_t j = node(p, wrap(x + EX[a], p->nx), wrap(y + EY[a], p->ny));
                if (solid[j])
                    f[OPP[a] * n + i] = fstar[a * n + i];
                else
                    f[a * n + j] = fstar[a * n + i];
            }
        }
    }
}

typedef struct {
    double *rho, *jx, *jy, *psi, *terms, *fstar;
} orc_work;

static int work_alloc(const orc_params *p, orc_work *w)
{
    size_t n = (size_t)p->nx * p->ny;
    w->rho = malloc(sizeof(double) * n);
    w->jx = malloc(sizeof(double) * n);
    w->jy = malloc(sizeof(double) * n);
    w->psi = malloc(sizeof(double) * n);
    w->terms = malloc(sizeof(double) * 8 * n);
    w->fstar = malloc(sizeof(double) * Q9 * n);
    return (w->rho && w->jx && w->jy && w->psi && w->terms && w->fstar) ? 0 : -1;
}

static void work_free(orc_work *w)
{
    free(w->rho); free(w->jx); free(w->jy); free(w->psi); free(w->terms); free(w->fstar);
}

static int check(const orc_params *p)
{
    if (p->nx < 1 || p->ny < 1) return -1;
    if (!(p->tau > 0.5) || !(p->rho0 > 0)) return -1;
    if (p->normal != ORC_NORMAL_FACES && p->normal != ORC_NORMAL_UNIT) return -1;
    return 0;
}

/* Phases 1-3 only: moments, psi and the four force terms of the current state. */
int orc_forces(const orc_params *p, const uint8_t *solid, const double *f,
               double *rho, double *jx, double *jy, double *terms)
{
    if (check(p)) return -1;
    size_t n = (size_t)p->nx * p->ny;
    double *psi = malloc(sizeof(double) * n);
    if (!psi) return -2;
    moments(p, solid, f, rho, jx, jy);
    pseudopotential(p, solid, rho, psi);
    forces(p, solid, rho, psi, terms);
    free(psi);
    return 0;
}

/* Advance f (in place) by nsteps time steps. */
int orc_step(const orc_params *p, const uint8_t *solid, double *f, int64_t nsteps)
{
    if (check(p)) return -1;
    orc_work w;
    if (work_alloc(p, &w)) { work_free(&w); return -2; }
    for (int64_t t = 0; t < nsteps; ++t) {
        moments(p, solid, f, w.rho, w.jx, w.jy);
        pseudopotential(p, solid, w.rho, w.psi);
        forces(p, solid, w.rho, w.psi, w.terms);
        collide(p, solid, f, w.rho, w.jx, w.jy, w.terms, w.fstar);
        stream(p, solid, w.fstar, f);
    }
    work_free(&w);
    return 0;
}

/* Per-node density and physical velocity u = (j + F/2)/rho; 0 on solids. */
int orc_fields(const orc_params *p, const uint8_t *solid, const double *f,
               double *rho, double *ux, double *uy)
{
    if (check(p)) return -1;
    size_t n = (size_t)p->nx * p->ny;
    orc_work w;
    if (work_alloc(p, &w)) { work_free(&w); return -2; }
    moments(p, solid, f, w.rho, w.jx, w.jy);
    pseudopotential(p, solid, w.rho, w.psi);
    forces(p, solid, w.rho, w.psi, w.terms);
    for (size_t i = 0; i < n; ++i) {
        rho[i] = w.rho[i];
        ux[i] = uy[i] = 0.0;
        if (solid[i]) continue;
        double Fx, Fy;
        total_force(n, w.terms, i, &Fx, &Fy);
        ux[i] = (w.jx[i] + 0.5 * Fx) / w.rho[i];
        uy[i] = (w.jy[i] + 0.5 * Fy) / w.rho[i];
    }
    work_free(&w);
    return 0;
}

/* Observables of the current state (Eq. 11 and bookkeeping):
 * out[0] mass = sum rho, out[1] Q = (1/nx) sum u_x, out[2..3] momentum
 * sum (j + F/2), out[4] max |u|, out[5] min rho, out[6] count of non-finite
 * rho or u. Sums run over fluid nodes in row-major order. */
int orc_observables(const orc_params *p, const uint8_t *solid, const double *f, double *out)
{
    if (check(p)) return -1;
    size_t n = (size_t)p->nx * p->ny;
    double *rho = malloc(sizeof(double) * n), *ux = malloc(sizeof(double) * n),
           *uy = malloc(sizeof(double) * n);
    if (!rho || !ux || !uy) { free(rho); free(ux); free(uy); return -2; }
    int rc = orc_fields(p, solid, f, rho, ux, uy);
    if (rc == 0) {
        double mass = 0, q = 0, px = 0, py = 0, umax = 0, rmin = INFINITY, bad = 0;
        for (size_t i = 0; i < n; ++i) {
            if (solid[i]) continue;
            if (!isfinite(rho[i]) || !isfinite(ux[i]) || !isfinite(uy[i])) { bad += 1; continue; }
            mass += rho[i];
            q += ux[i];
            px += rho[i] * ux[i];
            py += rho[i] * uy[i];
            double um = sqrt(ux[i] * ux[i] + uy[i] * uy[i]);
            if (um > umax) umax = um;
            if (rho[i] < rmin) rmin = rho[i];
        }
        out[0] = mass;
        out[1] = q / p->nx;
        out[2] = px;
        out[3] = py;
        out[4] = umax;
        out[5] = rmin;
        out[6] = bad;
    }
    free(rho); free(ux); free(uy);
    return rc;
}

/* Threads of the OpenMP loops (n >= 1); returns the count in effect (1
 * without OpenMP). Only timing uses it: results do not depend on it. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
