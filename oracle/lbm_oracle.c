/*
 * lbm_oracle.c -- FP64 CPU oracle of one time step of FishGym's fluid solver
 * (arXiv 2206.01683, Sec. III-B "GPU-accelerated localized fluid-structure
 * interaction"): a D3Q27 lattice Boltzmann step in the robot's accelerating
 * frame (Eq. 3), closed by non-equilibrium extrapolation on the open faces
 * (Sec. III-B "Simulation", Zhao-Li 2002) and two-way coupled to a surface
 * marker set by a direct-forcing immersed boundary.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow definition that the CUDA
 * path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product never links it.  It
 * shares no code, header or table with the CUDA library.
 *
 * Everything is double precision, one loop per step of the method, in the
 * order the method takes them.  The paper names the ingredients but not their
 * formulas; the readings taken where it is silent are stated beside the code
 * that implements them:
 *   - lattice: D3Q27, c_s^2 = 1/3, dx = dt = 1;
 *   - collision: regularized BGK with Guo forcing, i.e. the BGK-Guo
 *     post-collision moments (rho, j, Pi) projected on 2nd-order Hermite space;
 *   - delta kernel: Peskin's 4-point function;
 *   - marker force: direct forcing, F_l = 2 R_l (U_l - U~_l), in M passes
 *     (multi-direct forcing; M = 1 by default), each pass interpolating the
 *     velocity corrected by the force spread so far; optionally only the
 *     normal component of the slip (the paper's slipping wall, Sec. III-B);
 *   - frame force (Eq. 3): dr/dt read as the frame angular velocity omega,
 *     d2r/dt2 as its rate domega, and x' measured from a caller-given origin;
 *     the Coriolis term is solved implicitly together with the Guo half-shift;
 *   - boundary nodes are the outermost cell layer of every non-periodic face.
 *
 * Cell index: c = x + nx*(y + ny*z).  Populations: f[c*27 + i] in this file's
 * own velocity order (rest, 6 faces, 12 edges, 8 corners), see orc_lattice().
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 27
#define CS2 (1.0 / 3.0)

enum { ORC_PERIODIC = 0, ORC_VELOCITY = 1, ORC_OUTFLOW = 2, ORC_FREESLIP = 3 };

static int C[Q][3];
static double W[Q];
static int lattice_ready = 0;

/* D3Q27: every c in {-1,0,1}^3.  The weight depends only on |c|^2:
 * 8/27 (rest), 2/27 (faces), 1/54 (edges), 1/216 (corners). */
static void lattice_init(void) {
    if (lattice_ready) return;
    const double wshell[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    int n = 0;
    for (int shell = 0; shell <= 3; ++shell)
        for (int cz = -1; cz <= 1; ++cz)
            for (int cy = -1; cy <= 1; ++cy)
                for (int cx = -1; cx <= 1; ++cx)
                    if (cx * cx + cy * cy + cz * cz == shell) {
                        C[n][0] = cx; C[n][1] = cy; C[n][2] = cz;
                        W[n] = wshell[shell];
                        ++n;
                    }
    lattice_ready = 1;
}

/* Threads of the OpenMP loops (timing only; results do not depend on it
 * except for the summation order of the mass).  Returns the count in use. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

void orc_lattice(int *c, double *w) {
    lattice_init();
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = C[i][a];
        w[i] = W[i];
    }
}

typedef struct {
    int n[3];            /* nx, ny, nz */
    long ncell;
    double tau;
    int face[6];         /* -x,+x,-y,+y,-z,+z */
    double u_in[3];      /* velocity-inlet value */
    double rho_out;      /* outflow density */
    double *f;           /* post-collision populations f*, [ncell][27] */
    double *fs;          /* post-stream populations, [ncell][27] */
    double *rho, *j, *Pi;/* post-stream moments: rho, j[3], Pi[6] (xx,yy,zz,xy,xz,yz) */
    double *fib;         /* spread IB force density, [ncell][3] */
    double *gext;        /* external body-force density added to fib (pins only), [ncell][3] or NULL */
    int ib_iters;        /* direct-forcing passes M (>= 1) */
    int eq_order;        /* 2, or 3: add the lattice's third-order equilibrium terms */
    int slip;            /* 1: enforce only the normal velocity component */
    double *Nrm;         /* unit marker normals [nm][3] (slip) */
    int nm, nseg;        /* markers */
    double *X, *U, *dV;  /* [nm][3], [nm][3], [nm] */
    int *seg;
    double ref[3];       /* torque reference point of the total row */
    double seg_ref[64][3];   /* torque reference point of each segment row */
    int has_seg_ref;     /* 0: segment rows use ref as well */
    double *Fm;          /* marker force density F_l, [nm][3] */
    double force[64 * 6];/* per segment + total: F(3), T(3) */
    double mass, mass_dev;   /* sum rho and sum (rho - 1) after the last step */
    long step;
} orc_t;

static inline long cidx(const orc_t *o, int x, int y, int z) {
    return (long)x + (long)o->n[0] * ((long)y + (long)o->n[1] * (long)z);
}

static int periodic(const orc_t *o, int axis) { return o->face[2 * axis] == ORC_PERIODIC; }

/* ---------------------------------------------------------------- create */

void *orc_create(int nx, int ny, int nz, double tau, const int *face, const double *u_in,
                 double rho_out) {
    lattice_init();
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5)) return NULL;
    for (int a = 0; a < 3; ++a) {
        int lo = face[2 * a], hi = face[2 * a + 1];
        if ((lo == ORC_PERIODIC) != (hi == ORC_PERIODIC)) return NULL;
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return NULL;
        int na = a == 0 ? nx : a == 1 ? ny : nz;
        if (lo != ORC_PERIODIC && na < 3) return NULL;
    }
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->n[0] = nx; o->n[1] = ny; o->n[2] = nz;
    o->ncell = (long)nx * ny * nz;
    o->tau = tau;
    for (int k = 0; k < 6; ++k) o->face[k] = face[k];
    for (int a = 0; a < 3; ++a) o->u_in[a] = u_in ? u_in[a] : 0.0;
    o->rho_out = rho_out;
    o->ib_iters = 1;
    o->eq_order = 2;
    o->f = (double *)calloc((size_t)o->ncell * Q, sizeof(double));
    o->fs = (double *)calloc((size_t)o->ncell * Q, sizeof(double));
    o->rho = (double *)calloc((size_t)o->ncell, sizeof(double));
    o->j = (double *)calloc((size_t)o->ncell * 3, sizeof(double));
    o->Pi = (double *)calloc((size_t)o->ncell * 6, sizeof(double));
    o->fib = (double *)calloc((size_t)o->ncell * 3, sizeof(double));
    if (!o->f || !o->fs || !o->rho || !o->j || !o->Pi || !o->fib) {
        free(o->f); free(o->fs); free(o->rho); free(o->j); free(o->Pi); free(o->fib);
        free(o);
        return NULL;
    }
    return o;
}

void orc_destroy(void *h) {
    orc_t *o = (orc_t *)h;
    if (!o) return;
    free(o->f); free(o->fs); free(o->rho); free(o->j); free(o->Pi); free(o->fib);
    free(o->X); free(o->U); free(o->dV); free(o->seg); free(o->Fm); free(o->Nrm); free(o->gext);
    free(o);
}

/* ----------------------------------------------------------- equilibrium */

/* Second-order Hermite equilibrium,
 *   f_i^eq = w_i [rho + c_i.(rho u)/cs2 + (c_i c_i - cs2 I):(rho u u)/(2 cs2^2)]. */
static void equilibrium(double rho, const double u[3], double out[Q]) {
    for (int i = 0; i < Q; ++i) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        out[i] = W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* The third-order Hermite terms of the equilibrium that D3Q27 can carry,
 *   f3_i = w_i / (6 cs2^3) sum_abc rho u_a u_b u_c H_abc(c_i),
 *   H_abc(c) = c_a c_b c_c - cs2 (c_a d_bc + c_b d_ac + c_c d_ab),
 * summed over the index triples that are not all equal: on D3Q27
 * c_a^3 = c_a and 3 cs2 = 1, so H_aaa(c) = c_a^3 - 3 cs2 c_a vanishes on every
 * lattice velocity -- the lattice cannot carry rho u_a^3 (the loop skips
 * these terms, which are zero anyway). */
static void hermite3_eq(double rho, const double u[3], double out[Q]) {
    for (int i = 0; i < Q; ++i) {
        const int *c = C[i];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int g = 0; g < 3; ++g) {
                    if (a == b && b == g) continue;
                    double H = c[a] * c[b] * c[g] -
                               CS2 * (c[a] * (b == g) + c[b] * (a == g) + c[g] * (a == b));
                    s += rho * u[a] * u[b] * u[g] * H;
                }
        out[i] = W[i] * s / (6.0 * CS2 * CS2 * CS2);
    }
}

/* Equilibrium of the configured order: second order, plus hermite3_eq. */
static void equilibrium_n(const orc_t *o, double rho, const double u[3], double out[Q]) {
    equilibrium(rho, u, out);
    if (o->eq_order == 3) {
        double t[Q];
        hermite3_eq(rho, u, t);
        for (int i = 0; i < Q; ++i) out[i] += t[i];
    }
}

int orc_set_eq_order(void *h, int order) {
    orc_t *o = (orc_t *)h;
    if (order != 2 && order != 3) return -1;
    o->eq_order = order;
    return 0;
}

/* Rebuild populations from (rho, J, Qt) on the 2nd-order Hermite basis,
 *   f_i = w_i [rho + c_i.J/cs2 + (c_i c_i - cs2 I):Qt/(2 cs2^2)],
 * Qt = Pi - rho cs2 I given as (xx,yy,zz,xy,xz,yz). */
static void hermite2(double rho, const double J[3], const double Qt[6], double out[Q]) {
    for (int i = 0; i < Q; ++i) {
        const int *c = C[i];
        double cJ = c[0] * J[0] + c[1] * J[1] + c[2] * J[2];
        double ccQ = c[0] * c[0] * Qt[0] + c[1] * c[1] * Qt[1] + c[2] * c[2] * Qt[2] +
                     2.0 * (c[0] * c[1] * Qt[3] + c[0] * c[2] * Qt[4] + c[1] * c[2] * Qt[5]);
        double trQ = Qt[0] + Qt[1] + Qt[2];
        out[i] = W[i] * (rho + cJ / CS2 + (ccQ - CS2 * trQ) / (2.0 * CS2 * CS2));
    }
}

void orc_init_fields(void *h, const double *rho, const double *u) {
    orc_t *o = (orc_t *)h;
    for (long c = 0; c < o->ncell; ++c) {
        double r = rho ? rho[c] : 1.0;
        double uu[3] = {0, 0, 0};
        if (u) { uu[0] = u[3 * c]; uu[1] = u[3 * c + 1]; uu[2] = u[3 * c + 2]; }
        equilibrium_n(o, r, uu, o->f + c * Q);
    }
    o->step = 0;
}

/* -------------------------------------------------------------- 1 stream */

/* Pull streaming f_i(x) = f*_i(x - c_i).  Periodic axes wrap; a pull that
 * would cross a non-periodic face can only come from a boundary cell (the
 * outermost layer), whose populations are rebuilt by the boundary rule and
 * never read, so it is marked NaN to make any accidental use visible. */
static void stream(orc_t *o) {
    const int nx = o->n[0], ny = o->n[1], nz = o->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = cidx(o, x, y, z);
                for (int i = 0; i < Q; ++i) {
                    int s[3] = {x - C[i][0], y - C[i][1], z - C[i][2]};
                    int ok = 1;
                    for (int a = 0; a < 3; ++a) {
                        if (s[a] < 0 || s[a] >= o->n[a]) {
                            if (periodic(o, a)) s[a] = (s[a] + o->n[a]) % o->n[a];
                            else ok = 0;
                        }
                    }
                    o->fs[c * Q + i] = ok ? o->f[cidx(o, s[0], s[1], s[2]) * Q + i] : NAN;
                }
            }
}

/* ------------------------------------------------------------- 2 moments */

static void moments(orc_t *o) {
#pragma omp parallel for schedule(static)
    for (long c = 0; c < o->ncell; ++c) {
        const double *f = o->fs + c * Q;
        double r = 0, j[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            r += f[i];
            for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
            P[0] += C[i][0] * C[i][0] * f[i];
            P[1] += C[i][1] * C[i][1] * f[i];
            P[2] += C[i][2] * C[i][2] * f[i];
            P[3] += C[i][0] * C[i][1] * f[i];
            P[4] += C[i][0] * C[i][2] * f[i];
            P[5] += C[i][1] * C[i][2] * f[i];
        }
        o->rho[c] = r;
        for (int a = 0; a < 3; ++a) o->j[3 * c + a] = j[a];
        for (int k = 0; k < 6; ++k) o->Pi[6 * c + k] = P[k];
    }
}

/* ------------------------------------------------------ 3 frame (Eq. 3) */

static void cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* The velocity-independent part of Eq. 3,
 *   a0(x) = -p'' - r'' x x' - r' x (r' x x'),  x' = x - origin,
 * with frame[0..2] = p'', [3..5] = r' (omega), [6..8] = r'' (domega),
 * [9..11] = origin.  The Coriolis term -2 r' x u is handled in collide(). */
static void frame_accel(const double *frame, double x, double y, double z, double a0[3]) {
    const double *acc = frame, *om = frame + 3, *dom = frame + 6, *org = frame + 9;
    double xp[3] = {x - org[0], y - org[1], z - org[2]};
    double t1[3], t2[3], t3[3];
    cross(dom, xp, t1);
    cross(om, xp, t2);
    cross(om, t2, t3);
    for (int a = 0; a < 3; ++a) a0[a] = -acc[a] - t1[a] - t3[a];
}

void orc_frame_accel(const double *frame, double x, double y, double z, double *a0) {
    frame_accel(frame, x, y, z, a0);
}

/* -------------------------------------------------------- delta kernel */

/* Peskin's 4-point function (Peskin 2002, Acta Numerica, Sec. 6). */
double orc_phi(double r) {
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
    if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
    return 0.0;
}

/* The 4 stencil nodes of a marker coordinate X along one axis and their
 * weights: nodes floor(X)-1 .. floor(X)+2, weight phi(X - node); periodic
 * axes wrap the node index. */
static void stencil_axis(const orc_t *o, int axis, double X, int node[4], double wt[4]) {
    int N = o->n[axis];
    if (periodic(o, axis)) X = X - floor(X / N) * N;
    int base = (int)floor(X) - 1;
    for (int k = 0; k < 4; ++k) {
        int m = base + k;
        wt[k] = orc_phi(X - m);
        if (periodic(o, axis)) m = ((m % N) + N) % N;
        node[k] = m;
    }
}

/* Markers must keep their whole stencil off the boundary layer of a
 * non-periodic axis: 2 <= X < N-3. */
static int marker_ok(const orc_t *o, const double *X) {
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(X[a])) return 0;
        if (!periodic(o, a) && !(X[a] >= 2.0 && X[a] < o->n[a] - 3.0)) return 0;
    }
    return 1;
}

/* Interpolation I: out_l = sum_x g(x) delta(x - X_l), for a 3-vector field g. */
static void interp(const orc_t *o, const double *g, int n, const double *X, double *out) {
    for (int l = 0; l < n; ++l) {
        int nd[3][4];
        double wt[3][4];
        for (int a = 0; a < 3; ++a) stencil_axis(o, a, X[3 * l + a], nd[a], wt[a]);
        double s[3] = {0, 0, 0};
        for (int kz = 0; kz < 4; ++kz)
            for (int ky = 0; ky < 4; ++ky)
                for (int kx = 0; kx < 4; ++kx) {
                    double d = wt[0][kx] * wt[1][ky] * wt[2][kz];
                    long c = cidx(o, nd[0][kx], nd[1][ky], nd[2][kz]);
                    for (int a = 0; a < 3; ++a) s[a] += d * g[3 * c + a];
                }
        for (int a = 0; a < 3; ++a) out[3 * l + a] = s[a];
    }
}

/* Spreading S: g(x) += sum_l F_l delta(x - X_l), the transpose of interp(). */
static void spread(const orc_t *o, int n, const double *X, const double *F, double *g) {
    for (int l = 0; l < n; ++l) {
        int nd[3][4];
        double wt[3][4];
        for (int a = 0; a < 3; ++a) stencil_axis(o, a, X[3 * l + a], nd[a], wt[a]);
        for (int kz = 0; kz < 4; ++kz)
            for (int ky = 0; ky < 4; ++ky)
                for (int kx = 0; kx < 4; ++kx) {
                    double d = wt[0][kx] * wt[1][ky] * wt[2][kz];
                    long c = cidx(o, nd[0][kx], nd[1][ky], nd[2][kz]);
                    for (int a = 0; a < 3; ++a) g[3 * c + a] += d * F[3 * l + a];
                }
    }
}

int orc_interp(void *h, const double *g, int n, const double *X, double *out) {
    orc_t *o = (orc_t *)h;
    for (int l = 0; l < n; ++l)
        if (!marker_ok(o, X + 3 * l)) return -1;
    interp(o, g, n, X, out);
    return 0;
}

int orc_spread(void *h, int n, const double *X, const double *F, double *g) {
    orc_t *o = (orc_t *)h;
    for (int l = 0; l < n; ++l)
        if (!marker_ok(o, X + 3 * l)) return -1;
    spread(o, n, X, F, g);
    return 0;
}

int orc_set_markers(void *h, int n, const double *X, const double *U, const double *dV,
                    const int *seg, int nseg, const double *ref) {
    orc_t *o = (orc_t *)h;
    if (n < 0 || nseg < 0 || nseg > 63) return -1;
    for (int l = 0; l < n; ++l) {
        if (!marker_ok(o, X + 3 * l)) return -1;
        if (seg && (seg[l] < 0 || seg[l] >= (nseg > 0 ? nseg : 1))) return -1;
    }
    free(o->X); free(o->U); free(o->dV); free(o->seg); free(o->Fm); free(o->Nrm);
    o->Nrm = NULL;
    if (nseg != o->nseg) o->has_seg_ref = 0;   /* segment points belong to a segmentation */
    o->nm = n;
    o->nseg = nseg;
    o->X = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    o->U = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    o->dV = (double *)malloc(sizeof(double) * (n ? n : 1));
    o->seg = (int *)malloc(sizeof(int) * (n ? n : 1));
    o->Fm = (double *)calloc(3 * (n ? n : 1), sizeof(double));
    memcpy(o->X, X, sizeof(double) * 3 * n);
    memcpy(o->U, U, sizeof(double) * 3 * n);
    memcpy(o->dV, dV, sizeof(double) * n);
    for (int l = 0; l < n; ++l) o->seg[l] = seg ? seg[l] : 0;
    for (int a = 0; a < 3; ++a) o->ref[a] = ref ? ref[a] : 0.0;
    return 0;
}

/* Torque reference points of the segment rows (several bodies in one marker
 * set: each body's segments about that body's own point); NULL returns to
 * the common reference point, and so does a later orc_set_markers with a
 * different segment count.  The total row always uses ref. */
int orc_set_segment_refs(void *h, int nseg, const double *refs) {
    orc_t *o = (orc_t *)h;
    if (!refs) {
        o->has_seg_ref = 0;
        return 0;
    }
    if (nseg != (o->nseg > 0 ? o->nseg : 1) || nseg > 64) return -1;
    for (int s = 0; s < nseg; ++s)
        for (int a = 0; a < 3; ++a) o->seg_ref[s][a] = refs[3 * s + a];
    o->has_seg_ref = 1;
    return 0;
}

/* ------------------------------------------------ 4-5 interpolate, force */

/* Direct forcing.  At every node the pre-IB velocity is
 *   u~(x) = j/rho + a0(x)/2
 * (the Guo half-shift of the frame force; the small Coriolis part is left
 * out).  For each marker R_l = sum delta rho, U~_l = sum delta u~, and the
 * marker force density is F_l = 2 R_l (U_l - U~_l): with Guo's half-shift a
 * force density f moves the fluid velocity by f/(2 rho), so the factor 2
 * brings the interpolated velocity to U_l in one pass when the stencils of
 * different markers do not overlap.
 *
 * Multi-direct forcing repeats the pass M = ib_iters times.  Pass m
 * interpolates the velocity corrected by the force density spread so far,
 *   u~_m(x) = u~(x) + fib_m(x) / (2 rho(x)),
 * forms dF_l = 2 R_l (U_l - U~_m(X_l)) and spreads dF_l dV_l delta into fib;
 * F_l is the sum of the passes' dF_l.  When the passes converge, the
 * interpolated corrected velocity equals U_l at every marker.  M = 1 is the
 * single pass above.  On return o->Fm holds F_l and o->fib the spread force
 * density. */
static void direct_forcing(orc_t *o, const double *frame) {
    const int n = o->nm;
    memset(o->fib, 0, sizeof(double) * 3 * o->ncell);
    if (n == 0) return;
    double *ut = (double *)malloc(sizeof(double) * 3 * o->ncell);
    double *rr = (double *)malloc(sizeof(double) * 3 * o->ncell);
    const int nx = o->n[0], ny = o->n[1], nz = o->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long c = cidx(o, x, y, z);
                double a0[3];
                frame_accel(frame, x, y, z, a0);
                for (int a = 0; a < 3; ++a) {
                    ut[3 * c + a] = o->j[3 * c + a] / o->rho[c] + 0.5 * a0[a];
                    rr[3 * c + a] = o->rho[c];
                }
            }
    double *Ui = (double *)malloc(sizeof(double) * 3 * n);
    double *Ri = (double *)malloc(sizeof(double) * 3 * n);
    double *dF = (double *)malloc(sizeof(double) * 3 * n);
    double *dFdV = (double *)malloc(sizeof(double) * 3 * n);
    double *dfib = (double *)malloc(sizeof(double) * 3 * o->ncell);
    interp(o, rr, n, o->X, Ri);
    memset(o->Fm, 0, sizeof(double) * 3 * n);
    for (int m = 0; m < o->ib_iters; ++m) {
        interp(o, ut, n, o->X, Ui);
        for (int l = 0; l < n; ++l) {
            for (int a = 0; a < 3; ++a) dF[3 * l + a] = 2.0 * Ri[3 * l] * (o->U[3 * l + a] - Ui[3 * l + a]);
            if (o->slip) {   /* keep the normal component: dF <- (dF.n) n */
                const double *nl = o->Nrm + 3 * l;
                const double dn = dF[3 * l] * nl[0] + dF[3 * l + 1] * nl[1] + dF[3 * l + 2] * nl[2];
                for (int a = 0; a < 3; ++a) dF[3 * l + a] = dn * nl[a];
            }
            for (int a = 0; a < 3; ++a) {
                o->Fm[3 * l + a] += dF[3 * l + a];
                dFdV[3 * l + a] = dF[3 * l + a] * o->dV[l];
            }
        }
        memset(dfib, 0, sizeof(double) * 3 * o->ncell);
        spread(o, n, o->X, dFdV, dfib);
        for (long c = 0; c < o->ncell; ++c)
            for (int a = 0; a < 3; ++a) {
                o->fib[3 * c + a] += dfib[3 * c + a];
                ut[3 * c + a] += dfib[3 * c + a] / (2.0 * o->rho[c]);
            }
    }
    free(ut); free(rr); free(Ui); free(Ri); free(dF); free(dFdV); free(dfib);
}

/* Slip (Neumann) direct forcing: only the normal component of the marker
 * slip is enforced, dF_l = 2 R_l ((U_l - U~_l).n_l) n_l, so the fluid may
 * slide along the surface.  N: unit normals [n][3] of the current markers
 * (n must equal their count; normalised here). */
/* External body-force density G[ncell][3] (cell order x fastest), added to
 * the spread IB force density before the collision, so that it enters the
 * Guo forcing exactly as the IB force does; NULL removes it.  Not part of
 * the method: the oracle's pins use it (Kolmogorov flow). */
int orc_set_body_force(void *h, const double *G) {
    orc_t *o = (orc_t *)h;
    if (!G) {
        free(o->gext);
        o->gext = NULL;
        return 0;
    }
    if (!o->gext) o->gext = (double *)malloc(sizeof(double) * 3 * o->ncell);
    if (!o->gext) return -1;
    memcpy(o->gext, G, sizeof(double) * 3 * o->ncell);
    return 0;
}

int orc_set_slip(void *h, int on, int n, const double *N) {
    orc_t *o = (orc_t *)h;
    if (!on) {
        o->slip = 0;
        return 0;
    }
    if (n != o->nm || (n > 0 && !N)) return -1;
    free(o->Nrm);
    o->Nrm = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    for (int l = 0; l < n; ++l) {
        double s = sqrt(N[3 * l] * N[3 * l] + N[3 * l + 1] * N[3 * l + 1] + N[3 * l + 2] * N[3 * l + 2]);
        if (!(s > 0.0)) return -1;
        for (int a = 0; a < 3; ++a) o->Nrm[3 * l + a] = N[3 * l + a] / s;
    }
    o->slip = 1;
    return 0;
}

int orc_set_ib_iters(void *h, int m) {
    orc_t *o = (orc_t *)h;
    if (m < 1 || m > 64) return -1;
    o->ib_iters = m;
    return 0;
}

/* ------------------------------------------------------------ 6 collide */

/* Regularized BGK with Guo forcing at one cell, from its post-stream
 * populations.  a0 is the frame acceleration, fib the spread IB force density,
 * omega the frame angular velocity.
 *   v = j/rho + a0/2 + fib/(2 rho);  u solves u = v - omega x u, i.e.
 *   u = (v - omega x v + (omega.v) omega) / (1 + |omega|^2);
 *   G = rho a0 + fib - 2 rho omega x u        (total force density, Eq. 3)
 *   J  = j + G                                  (post-collision momentum)
 *   Ps = Pi_eq + (1 - 1/tau)(Pi - Pi_eq) + (1 - 1/(2 tau))(u G + G u)
 *   out_i = w_i [rho + c_i.J/cs2 + (c_i c_i - cs2 I):(Ps - rho cs2 I)/(2 cs2^2)]
 * with Pi_eq = rho u u + rho cs2 I.  These are the moments that BGK with
 * Guo's source term produces, rebuilt on the 2nd-order Hermite basis. */
static void collide(const double fs[Q], const double a0[3], const double fib[3],
                    const double om[3], double tau, int eq_order, double out[Q]) {
    double rho = 0, j[3] = {0, 0, 0}, Pi[3][3] = {{0}};
    for (int i = 0; i < Q; ++i) {
        rho += fs[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += C[i][a] * fs[i];
            for (int b = 0; b < 3; ++b) Pi[a][b] += C[i][a] * C[i][b] * fs[i];
        }
    }
    double v[3], u[3], G[3], wv[3], wu[3];
    for (int a = 0; a < 3; ++a) v[a] = j[a] / rho + 0.5 * a0[a] + fib[a] / (2.0 * rho);
    cross(om, v, wv);
    double ov = om[0] * v[0] + om[1] * v[1] + om[2] * v[2];
    double oo = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];
    for (int a = 0; a < 3; ++a) u[a] = (v[a] - wv[a] + ov * om[a]) / (1.0 + oo);
    cross(om, u, wu);
    for (int a = 0; a < 3; ++a) G[a] = rho * a0[a] + fib[a] - 2.0 * rho * wu[a];
    double J[3], Pst[3][3];
    for (int a = 0; a < 3; ++a) J[a] = j[a] + G[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double Peq = rho * u[a] * u[b] + (a == b ? rho * CS2 : 0.0);
            Pst[a][b] = Peq + (1.0 - 1.0 / tau) * (Pi[a][b] - Peq) +
                        (1.0 - 0.5 / tau) * (u[a] * G[b] + G[a] * u[b]);
        }
    double Qt[6] = {Pst[0][0] - rho * CS2, Pst[1][1] - rho * CS2, Pst[2][2] - rho * CS2,
                    Pst[0][1], Pst[0][2], Pst[1][2]};
    hermite2(rho, J, Qt, out);
    if (eq_order == 3) {   /* the post-collision state carries the equilibrium's third moments */
        double t[Q];
        hermite3_eq(rho, u, t);
        for (int i = 0; i < Q; ++i) out[i] += t[i];
    }
}

void orc_collide_cell(const double *fs, const double *a0, const double *fib, const double *om,
                      double tau, int eq_order, double *out) {
    lattice_init();
    collide(fs, a0, fib, om, tau, eq_order == 3 ? 3 : 2, out);
}

/* ------------------------------------------------------ 7 boundary (NEE) */

/* Non-equilibrium extrapolation on a boundary cell x_b (Zhao-Li 2002, the
 * scheme Sec. III-B "Simulation" adopts).  x_f = x_b + n, n the sum of the
 * inward normals of the non-periodic faces that x_b lies on.  From x_f's
 * post-stream moments (rho_f, u_f = j_f/rho_f, Pi_f):
 *   f*_i(x_b) = f_i^eq(rho_b, u_b) + (1 - 1/tau) f_i^neq(x_f),
 * f^neq the Hermite-2 part of Pi_f - Pi_eq(rho_f, u_f).  The face that
 * governs (rho_b, u_b) is the first non-periodic face touched in the order
 * x, y, z (x-faces override side walls):
 *   velocity inlet: u_b = u_in,                rho_b = rho_f
 *   outflow:        u_b = u_f,                 rho_b = rho_out
 *   free slip:      u_b = u_f minus the normal components of every free-slip
 *                   face touched,              rho_b = rho_f
 * No body force acts on boundary cells. */
static void boundary_cell(const orc_t *o, int x, int y, int z, const int side[3]) {
    int xf[3] = {x + side[0], y + side[1], z + side[2]};
    long cf = cidx(o, xf[0], xf[1], xf[2]);
    double rf = o->rho[cf];
    double uf[3] = {o->j[3 * cf] / rf, o->j[3 * cf + 1] / rf, o->j[3 * cf + 2] / rf};
    const double *P = o->Pi + 6 * cf;
    /* Pi_f - Pi_eq(rho_f, u_f), Pi_eq = rho u u + rho cs2 I, as (xx,yy,zz,xy,xz,yz). */
    double Pneq[6] = {P[0] - rf * uf[0] * uf[0] - rf * CS2, P[1] - rf * uf[1] * uf[1] - rf * CS2,
                      P[2] - rf * uf[2] * uf[2] - rf * CS2, P[3] - rf * uf[0] * uf[1],
                      P[4] - rf * uf[0] * uf[2], P[5] - rf * uf[1] * uf[2]};
    int gov = -1;
    for (int a = 0; a < 3 && gov < 0; ++a)
        if (side[a] != 0) gov = a;
    int gface = 2 * gov + (side[gov] < 0 ? 1 : 0); /* side +1 means the low face */
    int type = o->face[gface];
    double rb, ub[3];
    if (type == ORC_VELOCITY) {
        rb = rf;
        for (int a = 0; a < 3; ++a) ub[a] = o->u_in[a];
    } else if (type == ORC_OUTFLOW) {
        rb = o->rho_out;
        for (int a = 0; a < 3; ++a) ub[a] = uf[a];
    } else { /* free slip */
        rb = rf;
        for (int a = 0; a < 3; ++a) ub[a] = uf[a];
        for (int a = 0; a < 3; ++a) {
            if (side[a] == 0) continue;
            int fa = 2 * a + (side[a] < 0 ? 1 : 0);
            if (o->face[fa] == ORC_FREESLIP) ub[a] = 0.0;
        }
    }
    double feq[Q], zero3[3] = {0, 0, 0}, fneq[Q];
    equilibrium_n(o, rb, ub, feq);
    hermite2(0.0, zero3, Pneq, fneq);
    long cb = cidx(o, x, y, z);
    for (int i = 0; i < Q; ++i) o->f[cb * Q + i] = feq[i] + (1.0 - 1.0 / o->tau) * fneq[i];
}

/* -------------------------------------------- 8 body force and torque */

/* F = -sum_l F_l dV_l and T = -sum_l (X_l - X_ref) x F_l dV_l, the force and
 * torque the fluid exerts on the body (the tau_ext of Eq. 1), per segment and
 * in total (last row).  Segment rows take their torque about the segment's
 * reference point when one is set, the total row about ref. */
static void force_torque(orc_t *o) {
    int ns = o->nseg > 0 ? o->nseg : 1;
    memset(o->force, 0, sizeof(o->force));
    for (int l = 0; l < o->nm; ++l) {
        const int sg = o->seg[l];
        const double *rs = o->has_seg_ref ? o->seg_ref[sg] : o->ref;
        double F[3], r[3], rt[3], T[3], Tt[3];
        for (int a = 0; a < 3; ++a) {
            F[a] = -o->Fm[3 * l + a] * o->dV[l];
            r[a] = o->X[3 * l + a] - rs[a];
            rt[a] = o->X[3 * l + a] - o->ref[a];
        }
        cross(r, F, T);
        cross(rt, F, Tt);
        for (int a = 0; a < 3; ++a) {
            o->force[6 * sg + a] += F[a];
            o->force[6 * sg + 3 + a] += T[a];
            o->force[6 * ns + a] += F[a];
            o->force[6 * ns + 3 + a] += Tt[a];
        }
    }
}

/* ----------------------------------------------------------------- step */

/* One time step n -> n+1.  frame: p''[3], omega[3], domega[3], origin[3]. */
int orc_step(void *h, const double *frame) {
    orc_t *o = (orc_t *)h;
    const int nx = o->n[0], ny = o->n[1], nz = o->n[2];
    if (o->slip && o->nm > 0 && !o->Nrm) return -1;   /* normals of the current markers */
    stream(o);                 /* 1 */
    moments(o);                /* 2 */
    direct_forcing(o, frame);  /* 3-5 and 6a: marker forces, spread F_l dV_l */
    if (o->gext)               /* an external force density enters like the IB force */
        for (long c = 0; c < 3 * o->ncell; ++c) o->fib[c] += o->gext[c];
    const double *om = frame + 3;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)   /* 6b collide interior cells, 7 boundary cells */
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int side[3] = {0, 0, 0};
                int p[3] = {x, y, z};
                for (int a = 0; a < 3; ++a) {
                    if (periodic(o, a)) continue;
                    if (p[a] == 0) side[a] = +1;
                    else if (p[a] == o->n[a] - 1) side[a] = -1;
                }
                if (side[0] || side[1] || side[2]) {
                    boundary_cell(o, x, y, z, side);
                } else {
                    long c = cidx(o, x, y, z);
                    double a0[3];
                    frame_accel(frame, x, y, z, a0);
                    collide(o->fs + c * Q, a0, o->fib + 3 * c, om, o->tau, o->eq_order, o->f + c * Q);
                }
            }
    force_torque(o);           /* 8 */
    /* mass = sum_x rho(x), accumulated as ncell + sum_x (rho(x) - 1) so that the
     * sum runs over small numbers and carries no rounding bias */
    double dm = 0.0;
#pragma omp parallel for reduction(+ : dm) schedule(static)
    for (long c = 0; c < o->ncell; ++c) {
        double r = 0.0;
        for (int i = 0; i < Q; ++i) r += o->f[c * Q + i];
        dm += r - 1.0;
    }
    o->mass_dev = dm;
    o->mass = (double)o->ncell + dm;
    o->step += 1;
    return 0;
}

/* ------------------------------------------------------------- getters */

void orc_get_populations(void *h, double *f) {
    orc_t *o = (orc_t *)h;
    memcpy(f, o->f, sizeof(double) * Q * o->ncell);
}

void orc_set_populations(void *h, const double *f) {
    orc_t *o = (orc_t *)h;
    memcpy(o->f, f, sizeof(double) * Q * o->ncell);
}

/* Moments of the stored post-collision state: rho = sum f*, u = sum c f* / rho. */
void orc_get_fields(void *h, double *rho, double *u) {
    orc_t *o = (orc_t *)h;
    for (long c = 0; c < o->ncell; ++c) {
        const double *f = o->f + c * Q;
        double r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            r += f[i];
            for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
        }
        if (rho) rho[c] = r;
        if (u)
            for (int a = 0; a < 3; ++a) u[3 * c + a] = j[a] / r;
    }
}

/* Momentum and angular momentum of the fluid inside a sphere (centre c,
 * radius R) in the stored state: P = sum_x alpha(x) j(x), L = sum_x alpha(x)
 * (x - c) x j(x), j = sum_i c_i f*_i, with the cell's volume fraction
 * approximated by alpha = clamp(R + 1/2 - |x - c|, 0, 1) and x - c the
 * minimal image on periodic axes.  This is the internal-fluid term of a free
 * body's Newton-Euler equations (Kempe & Froehlich 2012, J. Comput. Phys.
 * 231).  out: P[3], L[3]; alpha_sum: sum alpha (the discrete volume). */
void orc_region_momentum(void *h, const double *c, double R, double *out, double *alpha_sum) {
    orc_t *o = (orc_t *)h;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int z = 0; z < o->n[2]; ++z)
        for (int y = 0; y < o->n[1]; ++y)
            for (int x = 0; x < o->n[0]; ++x) {
                int p[3] = {x, y, z};
                double r[3];
                for (int a = 0; a < 3; ++a) {
                    r[a] = p[a] - c[a];
                    if (periodic(o, a)) r[a] -= o->n[a] * floor(r[a] / o->n[a] + 0.5);
                }
                double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                double al = R + 0.5 - d;
                if (al <= 0.0) continue;
                if (al > 1.0) al = 1.0;
                const double *f = o->f + cidx(o, x, y, z) * Q;
                double j[3] = {0, 0, 0};
                for (int i = 0; i < Q; ++i)
                    for (int a = 0; a < 3; ++a) j[a] += C[i][a] * f[i];
                double t[3];
                cross(r, j, t);
                for (int a = 0; a < 3; ++a) {
                    acc[a] += al * j[a];
                    acc[3 + a] += al * t[a];
                }
                acc[6] += al;
            }
    for (int k = 0; k < 6; ++k) out[k] = acc[k];
    if (alpha_sum) *alpha_sum = acc[6];
}

void orc_get_force_torque(void *h, double *out) {
    orc_t *o = (orc_t *)h;
    int ns = o->nseg > 0 ? o->nseg : 1;
    memcpy(out, o->force, sizeof(double) * 6 * (ns + 1));
}

void orc_get_marker_force(void *h, double *F) {
    orc_t *o = (orc_t *)h;
    memcpy(F, o->Fm, sizeof(double) * 3 * o->nm);
}

double orc_mass(void *h) { return ((orc_t *)h)->mass; }

double orc_mass_deviation(void *h) { return ((orc_t *)h)->mass_dev; }

void orc_get_post_stream_moments(void *h, double *rho, double *j, double *Pi) {
    orc_t *o = (orc_t *)h;
    if (rho) memcpy(rho, o->rho, sizeof(double) * o->ncell);
    if (j) memcpy(j, o->j, sizeof(double) * 3 * o->ncell);
    if (Pi) memcpy(Pi, o->Pi, sizeof(double) * 6 * o->ncell);
}

void orc_get_fib(void *h, double *g) {
    orc_t *o = (orc_t *)h;
    memcpy(g, o->fib, sizeof(double) * 3 * o->ncell);
}
