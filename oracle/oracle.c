/*
 * FP64 CPU oracle for the TTI, elastic (3D and 2D) and isotropic acoustic
 * propagators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg load this library.  It shares no code with the
 * CUDA library: it is a plain, slow restatement of the discrete method in
 * double precision, written so that each step can be checked against the
 * paper by eye.  No blocking, no fusion, no reordering: every operator is a
 * loop over its definition, and every adjoint operator is the literal
 * transpose (a scatter loop) of the forward one.
 *
 * Paper: Louboutin et al., "Scaling through abstractions - high-performance
 * vectorial wave simulations for seismic inversion with Devito" (SC20).
 *   - acoustic wave equation, injection dt^2/m, interpolation: Sec. II-A,
 *     Eq. (acou) and the wave-equation listing;
 *   - rotated derivative D_xbar and G_xbarxbar = D_xbar^T D_xbar: Sec. III-A,
 *     Eq. (rot) and the rotated finite-difference listing;
 *   - TTI: 2 wavefields, Thomsen eps/delta, tilt theta, azimuth phi, not
 *     self-adjoint, exact adjoint and gradient required: Sec. III-A;
 *   - zero-lag cross-correlation imaging (adjoint-state gradient): Sec. III;
 *   - elastic velocity-stress system, Eq. (elas1), staggered grids with
 *     half-node averaging and the damp factor: Sec. IV-A, elastic listing;
 *   - Cerjan absorbing layer: Sec. V;
 *   - isotropic acoustic propagator: Eq. (acou) with u.laplace as the sum of
 *     centred second derivatives of the space order, damped like TTI.
 * Readings where the paper is silent (the TTI system of Zhang et al. /
 * Duveneck et al. cited in Sec. III-A, FD weights, damping profiles,
 * staggering, averaging, trilinear interpolation) are listed in the design
 * notes; each is restated where it is used below.
 *
 * Parity status: pinned by the CPU tests (FD weight moment conditions and
 * Fornberg's algorithm, antisymmetry D^T = -D and (D+)^T = -D-, plane-wave
 * dispersion of the TTI operator against the pseudo-acoustic dispersion
 * relation, eps=delta=0 collapse to an isotropic leapfrog, the point-source
 * Green's function, elastic energy conservation, mu=0 invariants, dot tests,
 * assembled-matrix transposes and Taylor tests of the gradients; for the
 * acoustic propagator the second-derivative moment conditions, Green's
 * function convergence, undamped leapfrog energy conservation, the dot test,
 * the assembled step's symmetry and a Taylor test; for the 2D elastic system
 * equality with a y-invariant state of the 3D system, the dot test and the
 * mu = 0 limit; for the sparse points exact reproduction of trilinear
 * functions by the injection/interpolation weights at random off-node
 * fractions and the one-step injection-to-recording product of the weights;
 * for the absorbing layers the first-arrival attenuation into the layer
 * against the WKB prediction of the damping and Cerjan profiles; for TTI
 * the spatial convergence order against the analytic 2D Green's function).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

#define MAXM 8

/* ------------------------------------------------------------------ */
/* descriptor (own definition; the CUDA library has its own)           */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;            /* 1 = TTI, 2 = elastic, 3 = isotropic acoustic,
                            4 = 2D elastic (x-z plane, ny = 1) */
    int nx, ny, nz;      /* PHYSICAL grid points */
    int nbl;             /* absorbing cells added on every face */
    int so;              /* space order (even) */
    int nt;              /* time samples */
    double h;            /* spacing [m] */
    double dt;           /* time step [s] */
    double vdamp;        /* TTI damping reference velocity [m/s];
                            <= 0: max(vp sqrt(1+2 eps)) of the model */
} or_desc;

typedef struct {
    or_desc d;
    int NX, NY, NZ;      /* computational grid */
    int nby;             /* absorbing cells on the y faces (0 in 2D) */
    long N;
    int M;
    double c[MAXM + 1];  /* centred weights c_1..c_M */
    double b[MAXM + 1];  /* staggered weights b_1..b_M */
    double c2[MAXM + 1]; /* second-derivative weights c2_0..c2_M (acoustic) */
    /* TTI */
    double *m, *eps, *del, *th, *ph, *sig;   /* sig: damping rate [1/s] */
    int tti_op;          /* TTI operator: 0 = composed centred first derivatives
                            (Eq. rot), 1 = staggered pair on the diagonal terms */
    /* elastic */
    double *lam, *mu, *bu;                   /* Lame [Pa], buoyancy [m^3/kg] */
    /* forward wavefield store for gradients */
    double *store;       /* TTI: [nt+1][2][N] (p^n, r^n) ; elastic: [nt+1][9][N] ;
                            acoustic: [nt+1][N] */
    int stored;
} or_prob;

/* ------------------------------------------------------------------ */
/* finite-difference weights                                            */
/* ------------------------------------------------------------------ */

/* Centred first derivative of order so (M = so/2), closed form:
 *   c_k = (-1)^(k+1) (M!)^2 / (k (M-k)! (M+k)!),  k = 1..M
 * so that (D u)_i = (1/h) sum_k c_k (u_{i+k} - u_{i-k}). */
int or_weights_centred(int so, double *c)
{
    if (so < 2 || so % 2 || so / 2 > MAXM) return OR_EINVAL;
    int M = so / 2;
    for (int k = 1; k <= M; k++) {
        double num = 1.0, den = (double)k;
        /* (M!)^2 / ((M-k)! (M+k)!) = prod_{j=1..k} (M-k+j)/(M+j) */
        for (int j = 1; j <= k; j++) num *= (double)(M - k + j) / (double)(M + j);
        c[k - 1] = ((k % 2) ? 1.0 : -1.0) * num / den;
    }
    return OR_OK;
}

/* Fornberg (1988), "Generation of finite difference formulas on arbitrarily
 * spaced grids", Math. Comp. 51: weights w[0..n-1] of the derivative of order
 * `order` at z from the nodes x[0..n-1].  Recursion on the number of nodes. */
int or_fornberg(int order, double z, const double *x, int n, double *w)
{
    if (n < 1 || order < 0 || order >= n || n > 64) return OR_EINVAL;
    double C[64][17];
    if (order > 16) return OR_EINVAL;
    for (int i = 0; i < n; i++)
        for (int k = 0; k <= order; k++) C[i][k] = 0.0;
    double c1 = 1.0, c4 = x[0] - z;
    C[0][0] = 1.0;
    for (int i = 1; i < n; i++) {
        int mn = i < order ? i : order;
        double c2 = 1.0, c5 = c4;
        c4 = x[i] - z;
        for (int j = 0; j < i; j++) {
            double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                for (int k = mn; k >= 1; k--)
                    C[i][k] = c1 * (k * C[i - 1][k - 1] - c5 * C[i - 1][k]) / c2;
                C[i][0] = -c1 * c5 * C[i - 1][0] / c2;
            }
            for (int k = mn; k >= 1; k--)
                C[j][k] = (c4 * C[j][k] - k * C[j][k - 1]) / c3;
            C[j][0] = c4 * C[j][0] / c3;
        }
        c1 = c2;
    }
    for (int i = 0; i < n; i++) w[i] = C[i][order];
    return OR_OK;
}

/* Staggered first derivative of order so: Fornberg weights at the half
 * offsets +-1/2, +-3/2, ... ; b_k is the weight of the node at +(k-1/2). */
int or_weights_staggered(int so, double *b)
{
    if (so < 2 || so % 2 || so / 2 > MAXM) return OR_EINVAL;
    int M = so / 2;
    double x[2 * MAXM], w[2 * MAXM];
    for (int k = 1; k <= M; k++) {
        x[2 * (k - 1)] = k - 0.5;
        x[2 * (k - 1) + 1] = -(k - 0.5);
    }
    int rc = or_fornberg(1, 0.0, x, 2 * M, w);
    if (rc) return rc;
    for (int k = 1; k <= M; k++) b[k - 1] = w[2 * (k - 1)];
    return OR_OK;
}

/* Centred second derivative of order so (the u.laplace of the Sec. II-A
 * listing, one axis): Fornberg weights for d^2/dx^2 at 0 on the nodes
 * -M..M; w[k] (k = 0..M) is the weight of the nodes +-k, so that
 *   (D2 u)_i = (1/h^2) (w_0 u_i + sum_k w_k (u_{i+k} + u_{i-k})). */
int or_weights_d2(int so, double *w)
{
    if (so < 2 || so % 2 || so / 2 > MAXM) return OR_EINVAL;
    int M = so / 2;
    double x[2 * MAXM + 1], f[2 * MAXM + 1];
    for (int i = 0; i <= 2 * M; i++) x[i] = i - M;
    int rc = or_fornberg(2, 0.0, x, 2 * M + 1, f);
    if (rc) return rc;
    for (int k = 0; k <= M; k++) w[k] = f[M + k];
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 1D line operators (zero extension outside [0, n))                    */
/* ------------------------------------------------------------------ */
static inline double at(const double *f, long s, int n, int i)
{
    return (i >= 0 && i < n) ? f[(long)i * s] : 0.0;
}

/* centred:  out_i = (1/h) sum_k c_k (f_{i+k} - f_{i-k}) */
static void line_D(const double *f, double *o, long s, int n, const or_prob *P)
{
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int k = 1; k <= P->M; k++)
            acc += P->c[k] * (at(f, s, n, i + k) - at(f, s, n, i - k));
        o[(long)i * s] = acc / P->d.h;
    }
}
/* out += a * D^T w  (literal transpose: scatter of row i of D) */
static void line_DT_add(const double *w, double *o, long s, int n, const or_prob *P, double a)
{
    for (int i = 0; i < n; i++) {
        double wi = a * w[(long)i * s] / P->d.h;
        for (int k = 1; k <= P->M; k++) {
            if (i + k < n) o[(long)(i + k) * s] += P->c[k] * wi;
            if (i - k >= 0) o[(long)(i - k) * s] -= P->c[k] * wi;
        }
    }
}
/* second derivative: out_i = (1/h^2) (c2_0 f_i + sum_k c2_k (f_{i+k} + f_{i-k})) */
static void line_D2(const double *f, double *o, long s, int n, const or_prob *P)
{
    for (int i = 0; i < n; i++) {
        double acc = P->c2[0] * at(f, s, n, i);
        for (int k = 1; k <= P->M; k++)
            acc += P->c2[k] * (at(f, s, n, i + k) + at(f, s, n, i - k));
        o[(long)i * s] = acc / (P->d.h * P->d.h);
    }
}
/* node -> half:  out_{i+1/2} (stored at i) = (1/h) sum_k b_k (f_{i+k} - f_{i-k+1}) */
static void line_Dp(const double *f, double *o, long s, int n, const or_prob *P)
{
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int k = 1; k <= P->M; k++)
            acc += P->b[k] * (at(f, s, n, i + k) - at(f, s, n, i - k + 1));
        o[(long)i * s] = acc / P->d.h;
    }
}
/* half -> node:  out_i = (1/h) sum_k b_k (g_{i+k-1/2} - g_{i-k+1/2}),
 * with g_{j+1/2} stored at j:  = (1/h) sum_k b_k (G_{i+k-1} - G_{i-k}) */
static void line_Dm(const double *f, double *o, long s, int n, const or_prob *P)
{
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int k = 1; k <= P->M; k++)
            acc += P->b[k] * (at(f, s, n, i + k - 1) - at(f, s, n, i - k));
        o[(long)i * s] = acc / P->d.h;
    }
}
/* out += a * (Dp)^T w  (scatter) */
static void line_DpT_add(const double *w, double *o, long s, int n, const or_prob *P, double a)
{
    for (int i = 0; i < n; i++) {
        double wi = a * w[(long)i * s] / P->d.h;
        for (int k = 1; k <= P->M; k++) {
            if (i + k < n) o[(long)(i + k) * s] += P->b[k] * wi;
            if (i - k + 1 >= 0 && i - k + 1 < n) o[(long)(i - k + 1) * s] -= P->b[k] * wi;
        }
    }
}
/* out += a * (Dm)^T w  (scatter) */
static void line_DmT_add(const double *w, double *o, long s, int n, const or_prob *P, double a)
{
    for (int i = 0; i < n; i++) {
        double wi = a * w[(long)i * s] / P->d.h;
        for (int k = 1; k <= P->M; k++) {
            if (i + k - 1 >= 0 && i + k - 1 < n) o[(long)(i + k - 1) * s] += P->b[k] * wi;
            if (i - k >= 0) o[(long)(i - k) * s] -= P->b[k] * wi;
        }
    }
}

typedef void (*line_op)(const double *, double *, long, int, const or_prob *);
typedef void (*line_opT)(const double *, double *, long, int, const or_prob *, double);

/* apply a 1D operator along `axis` (0 = x, 1 = y, 2 = z) to every line */
static void apply_axis(line_op op, const double *f, double *o, int axis, const or_prob *P)
{
    int NX = P->NX, NY = P->NY, NZ = P->NZ;
    if (axis == 2) {
#pragma omp parallel for collapse(2)
        for (int x = 0; x < NX; x++)
            for (int y = 0; y < NY; y++) {
                long base = ((long)x * NY + y) * NZ;
                op(f + base, o + base, 1, NZ, P);
            }
    } else if (axis == 1) {
#pragma omp parallel for collapse(2)
        for (int x = 0; x < NX; x++)
            for (int z = 0; z < NZ; z++) {
                long base = (long)x * NY * NZ + z;
                op(f + base, o + base, NZ, NY, P);
            }
    } else {
#pragma omp parallel for collapse(2)
        for (int y = 0; y < NY; y++)
            for (int z = 0; z < NZ; z++) {
                long base = (long)y * NZ + z;
                op(f + base, o + base, (long)NY * NZ, NX, P);
            }
    }
}
static void apply_axisT(line_opT op, const double *f, double *o, int axis, const or_prob *P, double a)
{
    int NX = P->NX, NY = P->NY, NZ = P->NZ;
    if (axis == 2) {
#pragma omp parallel for collapse(2)
        for (int x = 0; x < NX; x++)
            for (int y = 0; y < NY; y++) {
                long base = ((long)x * NY + y) * NZ;
                op(f + base, o + base, 1, NZ, P, a);
            }
    } else if (axis == 1) {
#pragma omp parallel for collapse(2)
        for (int x = 0; x < NX; x++)
            for (int z = 0; z < NZ; z++) {
                long base = (long)x * NY * NZ + z;
                op(f + base, o + base, NZ, NY, P, a);
            }
    } else {
#pragma omp parallel for collapse(2)
        for (int y = 0; y < NY; y++)
            for (int z = 0; z < NZ; z++) {
                long base = (long)y * NZ + z;
                op(f + base, o + base, (long)NY * NZ, NX, P, a);
            }
    }
}

/* ------------------------------------------------------------------ */
/* grid, model extension, damping                                       */
/* ------------------------------------------------------------------ */
static inline int clampi(int i, int lo, int hi) { return i < lo ? lo : (i > hi ? hi : i); }

/* physical model extended into the absorbing layer by edge replication */
static void extend(const float *phys, double *comp, const or_prob *P, double scale)
{
    const or_desc *d = &P->d;
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                int i = clampi(x - d->nbl, 0, d->nx - 1);
                int j = clampi(y - P->nby, 0, d->ny - 1);
                int k = clampi(z - d->nbl, 0, d->nz - 1);
                comp[((long)x * P->NY + y) * P->NZ + z] =
                    scale * (double)phys[((long)i * d->ny + j) * d->nz + k];
            }
}

/* adjoint of `extend`: every computational point adds into its source */
static void fold(const double *comp, double *phys, const or_prob *P)
{
    const or_desc *d = &P->d;
    memset(phys, 0, sizeof(double) * (size_t)d->nx * d->ny * d->nz);
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                int i = clampi(x - d->nbl, 0, d->nx - 1);
                int j = clampi(y - P->nby, 0, d->ny - 1);
                int k = clampi(z - d->nbl, 0, d->nz - 1);
                phys[((long)i * d->ny + j) * d->nz + k] += comp[((long)x * P->NY + y) * P->NZ + z];
            }
}

/* distance (in cells) of continuous index s from the physical box [nbl, nbl+n-1] */
static double layer_depth(double s, int nbl, int n)
{
    double lo = (double)nbl, hi = (double)(nbl + n - 1);
    if (s < lo) return lo - s;
    if (s > hi) return s - hi;
    return 0.0;
}

/* TTI damping rate sigma [1/s] at a node: sum over axes of
 *   (3 vmax / (2 L)) ln(1/R0) (d/L)^2,  L = nbl*h, R0 = 1e-3, d in metres;
 * the equation is m u_tt + m sigma u_t = ..., so A = m (1 + sigma dt/2). */
static double tti_sigma(const or_prob *P, int x, int y, int z, double vmax)
{
    const or_desc *d = &P->d;
    if (d->nbl <= 0) return 0.0;
    double L = d->nbl * d->h;
    double s0 = 3.0 * vmax / (2.0 * L) * log(1.0 / 1e-3);
    double dx = layer_depth(x, d->nbl, d->nx) * d->h / L;
    double dy = layer_depth(y, d->nbl, d->ny) * d->h / L;
    double dz = layer_depth(z, d->nbl, d->nz) * d->h / L;
    return s0 * (dx * dx + dy * dy + dz * dz);
}

/* Cerjan taper at continuous position (sx, sy, sz):
 *   g = prod_axes exp(-(0.015 d)^2), d = depth into the layer in cells. */
static double cerjan(const or_prob *P, double sx, double sy, double sz)
{
    const or_desc *d = &P->d;
    if (d->nbl <= 0) return 1.0;
    const double a = 0.015;
    double dx = a * layer_depth(sx, d->nbl, d->nx);
    double dy = a * layer_depth(sy, P->nby, d->ny);
    double dz = a * layer_depth(sz, d->nbl, d->nz);
    return exp(-dx * dx) * exp(-dy * dy) * exp(-dz * dz);
}

static long IDX(const or_prob *P, int x, int y, int z) { return ((long)x * P->NY + y) * P->NZ + z; }

static double *dalloc(long n)
{
    double *p = (double *)calloc((size_t)n, sizeof(double));
    return p;
}

/* ------------------------------------------------------------------ */
/* setup / teardown                                                     */
/* ------------------------------------------------------------------ */
void or_destroy(or_prob *P)
{
    if (!P) return;
    free(P->m); free(P->eps); free(P->del); free(P->th); free(P->ph); free(P->sig);
    free(P->lam); free(P->mu); free(P->bu); free(P->store);
    free(P);
}

/* model (physical grid, float32):
 *   TTI:      vp [km/s], eps, delta, theta [rad], phi [rad]
 *   elastic:  vp [km/s], vs [km/s], rho [g/cc]
 *   acoustic: vp [km/s]  (damping as for TTI, vmax = max vp) */
or_prob *or_create(const or_desc *d, const float *const *model)
{
    if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nbl < 0 || d->so < 2 ||
        d->so % 2 || d->so / 2 > MAXM || d->nt < 1 || !(d->h > 0) || !(d->dt > 0))
        return NULL;
    if (d->kind < 1 || d->kind > 4 || (d->kind == 4 && d->ny != 1)) return NULL;
    or_prob *P = (or_prob *)calloc(1, sizeof(or_prob));
    P->d = *d;
    P->NX = d->nx + 2 * d->nbl;
    P->nby = d->kind == 4 ? 0 : d->nbl;
    P->NY = d->ny + 2 * P->nby;
    P->NZ = d->nz + 2 * d->nbl;
    P->N = (long)P->NX * P->NY * P->NZ;
    P->M = d->so / 2;
    double tmp[MAXM];
    or_weights_centred(d->so, tmp);
    for (int k = 1; k <= P->M; k++) P->c[k] = tmp[k - 1];
    or_weights_staggered(d->so, tmp);
    for (int k = 1; k <= P->M; k++) P->b[k] = tmp[k - 1];
    or_weights_d2(d->so, P->c2);
    long N = P->N;
    if (d->kind == 1) {
        double *vp = dalloc(N);
        P->m = dalloc(N); P->eps = dalloc(N); P->del = dalloc(N);
        P->th = dalloc(N); P->ph = dalloc(N); P->sig = dalloc(N);
        if (!vp || !P->m || !P->eps || !P->del || !P->th || !P->ph || !P->sig) {
            free(vp); or_destroy(P); return NULL;
        }
        extend(model[0], vp, P, 1000.0);          /* km/s -> m/s */
        extend(model[1], P->eps, P, 1.0);
        extend(model[2], P->del, P, 1.0);
        extend(model[3], P->th, P, 1.0);
        extend(model[4], P->ph, P, 1.0);
        double vmax = 0.0;
        for (long i = 0; i < N; i++) {
            P->m[i] = 1.0 / (vp[i] * vp[i]);      /* squared slowness [s^2/m^2] */
            double v = vp[i] * sqrt(1.0 + 2.0 * P->eps[i]);
            if (v > vmax) vmax = v;
        }
        if (d->vdamp > 0) vmax = d->vdamp;
        free(vp);
        for (int x = 0; x < P->NX; x++)
            for (int y = 0; y < P->NY; y++)
                for (int z = 0; z < P->NZ; z++)
                    P->sig[IDX(P, x, y, z)] = tti_sigma(P, x, y, z, vmax);
    } else if (d->kind == 3) {
        double *vp = dalloc(N);
        P->m = dalloc(N); P->sig = dalloc(N);
        if (!vp || !P->m || !P->sig) { free(vp); or_destroy(P); return NULL; }
        extend(model[0], vp, P, 1000.0);
        double vmax = 0.0;
        for (long i = 0; i < N; i++) {
            P->m[i] = 1.0 / (vp[i] * vp[i]);
            if (vp[i] > vmax) vmax = vp[i];
        }
        if (d->vdamp > 0) vmax = d->vdamp;
        free(vp);
        for (int x = 0; x < P->NX; x++)
            for (int y = 0; y < P->NY; y++)
                for (int z = 0; z < P->NZ; z++)
                    P->sig[IDX(P, x, y, z)] = tti_sigma(P, x, y, z, vmax);
    } else {
        double *vp = dalloc(N), *vs = dalloc(N), *rho = dalloc(N);
        P->lam = dalloc(N); P->mu = dalloc(N); P->bu = dalloc(N);
        if (!vp || !vs || !rho || !P->lam || !P->mu || !P->bu) {
            free(vp); free(vs); free(rho); or_destroy(P); return NULL;
        }
        extend(model[0], vp, P, 1000.0);
        extend(model[1], vs, P, 1000.0);
        extend(model[2], rho, P, 1000.0);         /* g/cc -> kg/m^3 */
        for (long i = 0; i < N; i++) {
            P->mu[i] = rho[i] * vs[i] * vs[i];
            P->lam[i] = rho[i] * (vp[i] * vp[i] - 2.0 * vs[i] * vs[i]);
            P->bu[i] = 1.0 / rho[i];
        }
        free(vp); free(vs); free(rho);
    }
    return P;
}

long or_npoints(const or_prob *P) { return P->N; }
void or_dims(const or_prob *P, int *dims) { dims[0] = P->NX; dims[1] = P->NY; dims[2] = P->NZ; }
const double *or_param(const or_prob *P, int which)
{
    switch (which) {
    case 0: return P->m; case 1: return P->eps; case 2: return P->del;
    case 3: return P->th; case 4: return P->ph; case 5: return P->sig;
    case 10: return P->lam; case 11: return P->mu; case 12: return P->bu;
    }
    return NULL;
}

/* ------------------------------------------------------------------ */
/* sparse points: trilinear interpolation weights                       */
/* ------------------------------------------------------------------ */
/* Position (metres, origin at the first physical point) -> up to 8
 * (index, weight) pairs on the computational grid; corners whose weight is
 * exactly zero are dropped.  Returns the count, or -1 if out of the grid. */
static int trilinear(const or_prob *P, const float *xyz, long *idx, double *w)
{
    double s[3]; int i0[3]; double f[3];
    int n[3] = {P->NX, P->NY, P->NZ};
    for (int a = 0; a < 3; a++) {
        s[a] = (double)xyz[a] / P->d.h + (a == 1 ? P->nby : P->d.nbl);
        if (!(s[a] >= 0.0) || s[a] > (double)(n[a] - 1)) return -1;
        i0[a] = (int)floor(s[a]);
        f[a] = s[a] - i0[a];
    }
    int cnt = 0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                double wt = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
                if (wt == 0.0) continue;
                idx[cnt] = IDX(P, i0[0] + a, i0[1] + b, i0[2] + c);
                w[cnt] = wt;
                cnt++;
            }
    return cnt;
}

typedef struct { int n; long idx[8]; double w[8]; } pt8;

static pt8 *make_points(const or_prob *P, const float *xyz, int np, int *err)
{
    pt8 *pts = (pt8 *)calloc(np > 0 ? np : 1, sizeof(pt8));
    *err = 0;
    for (int i = 0; i < np; i++) {
        pts[i].n = trilinear(P, xyz + 3 * i, pts[i].idx, pts[i].w);
        if (pts[i].n < 0) *err = 1;
    }
    return pts;
}

static double sample(const pt8 *p, const double *u)
{
    double s = 0.0;
    for (int c = 0; c < p->n; c++) s += p->w[c] * u[p->idx[c]];
    return s;
}

/* ------------------------------------------------------------------ */
/* TTI operator (Sec. III-A, Eq. rot)                                   */
/* ------------------------------------------------------------------ */
/* Rotated frame at a point: x-bar exactly as Eq. (rot),
 *   xb = ( cos th cos ph, cos th sin ph, -sin th ),
 *   yb = ( -sin ph, cos ph, 0 ),
 *   zb = ( sin th cos ph, sin th sin ph, cos th )  (symmetry axis). */
static void frame(double th, double ph, double *xb, double *yb, double *zb)
{
    xb[0] = cos(th) * cos(ph); xb[1] = cos(th) * sin(ph); xb[2] = -sin(th);
    yb[0] = -sin(ph);          yb[1] = cos(ph);           yb[2] = 0.0;
    zb[0] = sin(th) * cos(ph); zb[1] = sin(th) * sin(ph); zb[2] = cos(th);
}

/* H0 p = -(G_xbxb + G_ybyb) p,  Hz r = -G_zbzb r,  G_aa = D_a^T D_a with
 * D_a u = sum_i a_i D_i u (pointwise frame) and D_a^T w = sum_i D_i^T (a_i w).
 * Literal three-axis form with the transposes as scatter loops. */
static void tti_apply_H_sp(const or_prob *P, const double *p, const double *r, double *H0p, double *Hzr);
static void tti_apply_H(const or_prob *P, const double *p, const double *r,
                        double *H0p, double *Hzr)
{
    if (P->tti_op == 1) {
        tti_apply_H_sp(P, p, r, H0p, Hzr);
        return;
    }
    long N = P->N;
    double *gp[3], *gr[3], *ax[3], *ay[3], *az[3];
    for (int i = 0; i < 3; i++) {
        gp[i] = dalloc(N); gr[i] = dalloc(N);
        ax[i] = dalloc(N); ay[i] = dalloc(N); az[i] = dalloc(N);
    }
    for (int i = 0; i < 3; i++) {
        apply_axis(line_D, p, gp[i], i, P);
        apply_axis(line_D, r, gr[i], i, P);
    }
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double xb[3], yb[3], zb[3];
        frame(P->th[q], P->ph[q], xb, yb, zb);
        double Dxp = xb[0] * gp[0][q] + xb[1] * gp[1][q] + xb[2] * gp[2][q];
        double Dyp = yb[0] * gp[0][q] + yb[1] * gp[1][q] + yb[2] * gp[2][q];
        double Dzr = zb[0] * gr[0][q] + zb[1] * gr[1][q] + zb[2] * gr[2][q];
        for (int i = 0; i < 3; i++) {
            ax[i][q] = xb[i] * Dxp;
            ay[i][q] = yb[i] * Dyp;
            az[i][q] = zb[i] * Dzr;
        }
    }
    memset(H0p, 0, sizeof(double) * N);
    memset(Hzr, 0, sizeof(double) * N);
    for (int i = 0; i < 3; i++) {
        apply_axisT(line_DT_add, ax[i], H0p, i, P, -1.0);
        apply_axisT(line_DT_add, ay[i], H0p, i, P, -1.0);
        apply_axisT(line_DT_add, az[i], Hzr, i, P, -1.0);
    }
    for (int i = 0; i < 3; i++) {
        free(gp[i]); free(gr[i]); free(ax[i]); free(ay[i]); free(az[i]);
    }
}

/* Derivatives of the frame of Eq. (rot) with respect to theta and phi. */
static void frame_dth(double th, double ph, double *xb, double *yb, double *zb)
{
    xb[0] = -sin(th) * cos(ph); xb[1] = -sin(th) * sin(ph); xb[2] = -cos(th);
    yb[0] = 0.0;                yb[1] = 0.0;                yb[2] = 0.0;
    zb[0] = cos(th) * cos(ph);  zb[1] = cos(th) * sin(ph);  zb[2] = -sin(th);
}
static void frame_dph(double th, double ph, double *xb, double *yb, double *zb)
{
    xb[0] = -cos(th) * sin(ph); xb[1] = cos(th) * cos(ph);  xb[2] = 0.0;
    yb[0] = -cos(ph);           yb[1] = -sin(ph);           yb[2] = 0.0;
    zb[0] = -sin(th) * sin(ph); zb[1] = sin(th) * cos(ph);  zb[2] = 0.0;
}
static inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Tilt/azimuth imaging of one step: with the bilinear forms
 *   <zp, H0 p> = -sum_{a = xb, yb} <D_a zp, D_a p>,  <zr, Hz r> = -<D_zb zr, D_zb r>
 * (D_a u = sum_i a_i D_i u at each point), the derivative with respect to the
 * angle t at point q is
 *   -sum_{a = xb, yb} [(a_t . D zp)(a . D p) + (a . D zp)(a_t . D p)]
 *   - [(zb_t . D zr)(zb . D r) + (zb . D zr)(zb_t . D r)],
 * all at q; scaled by `scale` and added to gt (t = theta) and gf (t = phi). */
static void tti_frame_image(const or_prob *P, const double *zp, const double *zr, const double *p,
                            const double *r, double scale, double *gt, double *gf, double *at, double *af)
{
    long N = P->N;
    double *Gz[3], *Gr[3], *gp[3], *gr[3];
    for (int i = 0; i < 3; i++) {
        Gz[i] = dalloc(N); Gr[i] = dalloc(N); gp[i] = dalloc(N); gr[i] = dalloc(N);
        apply_axis(line_D, zp, Gz[i], i, P);
        apply_axis(line_D, zr, Gr[i], i, P);
        apply_axis(line_D, p, gp[i], i, P);
        apply_axis(line_D, r, gr[i], i, P);
    }
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double xb[3], yb[3], zb[3], A[3], B[3], C3[3], U[3], V[3], W[3];
        double a[3] = {Gz[0][q], Gz[1][q], Gz[2][q]}, b[3] = {gp[0][q], gp[1][q], gp[2][q]};
        double c[3] = {Gr[0][q], Gr[1][q], Gr[2][q]}, d[3] = {gr[0][q], gr[1][q], gr[2][q]};
        frame(P->th[q], P->ph[q], xb, yb, zb);
        frame_dth(P->th[q], P->ph[q], A, B, C3);
        frame_dph(P->th[q], P->ph[q], U, V, W);
        double t = -(dot3(A, a) * dot3(xb, b) + dot3(xb, a) * dot3(A, b))
                   - (dot3(B, a) * dot3(yb, b) + dot3(yb, a) * dot3(B, b))
                   - (dot3(C3, c) * dot3(zb, d) + dot3(zb, c) * dot3(C3, d));
        double f = -(dot3(U, a) * dot3(xb, b) + dot3(xb, a) * dot3(U, b))
                   - (dot3(V, a) * dot3(yb, b) + dot3(yb, a) * dot3(V, b))
                   - (dot3(W, c) * dot3(zb, d) + dot3(zb, c) * dot3(W, d));
        gt[q] += scale * t;
        gf[q] += scale * f;
        if (at) {
            /* magnitude of the summed terms (for rounding-error bounds of the sum) */
            double u = fabs(dot3(A, a) * dot3(xb, b)) + fabs(dot3(xb, a) * dot3(A, b)) +
                       fabs(dot3(B, a) * dot3(yb, b)) + fabs(dot3(yb, a) * dot3(B, b)) +
                       fabs(dot3(C3, c) * dot3(zb, d)) + fabs(dot3(zb, c) * dot3(C3, d));
            double v = fabs(dot3(U, a) * dot3(xb, b)) + fabs(dot3(xb, a) * dot3(U, b)) +
                       fabs(dot3(V, a) * dot3(yb, b)) + fabs(dot3(yb, a) * dot3(V, b)) +
                       fabs(dot3(W, c) * dot3(zb, d)) + fabs(dot3(zb, c) * dot3(W, d));
            at[q] += fabs(scale) * u;
            af[q] += fabs(scale) * v;
        }
    }
    for (int i = 0; i < 3; i++) { free(Gz[i]); free(Gr[i]); free(gp[i]); free(gr[i]); }
}

/* Tilt/azimuth imaging of one step for the staggered-pair operators
 * (tti_apply_H_sp).  Their bilinear forms differ from the centred ones only
 * in the diagonal terms: with a = D zp, b = D p, c = D zr, d = D r (centred,
 * at the nodes) and the half-point products S0_i(h) = (D+_i zp)(D+_i p)(h),
 * Sz_i(h) = (D+_i zr)(D+_i r)(h) (half point h + 1/2 stored at h),
 *   <zp, H0 p> = -a^T P0 b + sum_i P0_ii a_i b_i - sum_{i,h} P0~_ii(h) S0_i(h)
 * and likewise for Hz with Pz.  P_ii(q) enters P~_ii at the half points
 * q + 1/2 (weight 1/2; 1 at the last node, whose partner is clamped to
 * itself) and q - 1/2 (weight 1/2, none at the first node), so the term at q
 * collects T_i(q) = w+ S_i(q) + w- S_i(q - e_i).  The derivative with
 * respect to an angle t is therefore the centred one (tti_frame_image) plus
 *   sum_i dP0_ii/dt (a_i b_i - T0_i) + sum_i dPz_ii/dt (c_i d_i - Tz_i),
 * dP0_ii/dt = 2 (xb_t,i xb_i + yb_t,i yb_i), dPz_ii/dt = 2 zb_t,i zb_i. */
static void tti_frame_image_sp(const or_prob *P, const double *zp, const double *zr, const double *p,
                               const double *r, double scale, double *gt, double *gf, double *at, double *af)
{
    tti_frame_image(P, zp, zr, p, r, scale, gt, gf, at, af);
    long N = P->N;
    double *a[3], *b[3], *c[3], *d[3], *S0[3], *Sz[3], *t1 = dalloc(N), *t2 = dalloc(N);
    for (int i = 0; i < 3; i++) {
        a[i] = dalloc(N); b[i] = dalloc(N); c[i] = dalloc(N); d[i] = dalloc(N);
        S0[i] = dalloc(N); Sz[i] = dalloc(N);
        apply_axis(line_D, zp, a[i], i, P);
        apply_axis(line_D, p, b[i], i, P);
        apply_axis(line_D, zr, c[i], i, P);
        apply_axis(line_D, r, d[i], i, P);
        apply_axis(line_Dp, zp, t1, i, P);
        apply_axis(line_Dp, p, t2, i, P);
        for (long q = 0; q < N; q++) S0[i][q] = t1[q] * t2[q];
        apply_axis(line_Dp, zr, t1, i, P);
        apply_axis(line_Dp, r, t2, i, P);
        for (long q = 0; q < N; q++) Sz[i][q] = t1[q] * t2[q];
    }
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                const int pos[3] = {x, y, z}, len[3] = {P->NX, P->NY, P->NZ};
                double xb[3], yb[3], zb[3], A[3], B[3], C3[3], U[3], V[3], W[3];
                frame(P->th[q], P->ph[q], xb, yb, zb);
                frame_dth(P->th[q], P->ph[q], A, B, C3);
                frame_dph(P->th[q], P->ph[q], U, V, W);
                double tt = 0.0, ff = 0.0, ta = 0.0, fa = 0.0;
                for (int i = 0; i < 3; i++) {
                    long qm = q - (i == 0 ? (long)P->NY * P->NZ : (i == 1 ? P->NZ : 1));
                    double wp = pos[i] == len[i] - 1 ? 1.0 : 0.5, wm = pos[i] >= 1 ? 0.5 : 0.0;
                    double T0 = wp * S0[i][q] + (wm > 0.0 ? wm * S0[i][qm] : 0.0);
                    double Tz = wp * Sz[i][q] + (wm > 0.0 ? wm * Sz[i][qm] : 0.0);
                    double e0 = a[i][q] * b[i][q] - T0, ez = c[i][q] * d[i][q] - Tz;
                    double d0t = 2.0 * (A[i] * xb[i] + B[i] * yb[i]), dzt = 2.0 * C3[i] * zb[i];
                    double d0f = 2.0 * (U[i] * xb[i] + V[i] * yb[i]), dzf = 2.0 * W[i] * zb[i];
                    tt += d0t * e0 + dzt * ez;
                    ff += d0f * e0 + dzf * ez;
                    ta += fabs(d0t) * (fabs(a[i][q] * b[i][q]) + fabs(T0)) + fabs(dzt) * (fabs(c[i][q] * d[i][q]) + fabs(Tz));
                    fa += fabs(d0f) * (fabs(a[i][q] * b[i][q]) + fabs(T0)) + fabs(dzf) * (fabs(c[i][q] * d[i][q]) + fabs(Tz));
                }
                gt[q] += scale * tt;
                gf[q] += scale * ff;
                if (at) {
                    at[q] += fabs(scale) * ta;
                    af[q] += fabs(scale) * fa;
                }
            }
    for (int i = 0; i < 3; i++) { free(a[i]); free(b[i]); free(c[i]); free(d[i]); free(S0[i]); free(Sz[i]); }
    free(t1); free(t2);
}

/* Staggered-pair variant of the same operators.  With P0 = xb xb^T + yb yb^T
 * and Pz = zb zb^T (pointwise), the centred form above is
 *   H0 u = -sum_{i,j} D_i^T (P0_ij D_j u),  Hz u = -sum_{i,j} D_i^T (Pz_ij D_j u);
 * here each diagonal term i = j uses the staggered pair instead,
 *   -(D+_i)^T (P0_ii~ D+_i u),  P0_ii~ = (P0_ii(q) + P0_ii(q + e_i)) / 2 at the
 * half point (the neighbour clamped at the last node), which has no
 * checkerboard null vector; the cross terms i != j keep the centred D.
 * Both forms are symmetric, so the adjoint machinery is unchanged. */
static void tti_apply_H_sp(const or_prob *P, const double *p, const double *r, double *H0p, double *Hzr)
{
    long N = P->N;
    double *gp[3], *gr[3], *sp[3], *sr[3], *d0[3], *dz[3], *c0[3], *cz[3];
    for (int i = 0; i < 3; i++) {
        gp[i] = dalloc(N); gr[i] = dalloc(N); sp[i] = dalloc(N); sr[i] = dalloc(N);
        d0[i] = dalloc(N); dz[i] = dalloc(N); c0[i] = dalloc(N); cz[i] = dalloc(N);
        apply_axis(line_D, p, gp[i], i, P);
        apply_axis(line_D, r, gr[i], i, P);
        apply_axis(line_Dp, p, sp[i], i, P);
        apply_axis(line_Dp, r, sr[i], i, P);
    }
    /* diagonal entries of P0, Pz at the nodes; cross fluxes sum_{j != i} P_ij D_j u */
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double xb[3], yb[3], zb[3];
        frame(P->th[q], P->ph[q], xb, yb, zb);
        for (int i = 0; i < 3; i++) {
            d0[i][q] = xb[i] * xb[i] + yb[i] * yb[i];
            dz[i][q] = zb[i] * zb[i];
            double a = 0.0, b = 0.0;
            for (int j = 0; j < 3; j++) {
                if (j == i) continue;
                a += (xb[i] * xb[j] + yb[i] * yb[j]) * gp[j][q];
                b += zb[i] * zb[j] * gr[j][q];
            }
            c0[i][q] = a;
            cz[i][q] = b;
        }
    }
    /* diagonal fluxes at the half points: averaged coefficient times D+ u */
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                for (int i = 0; i < 3; i++) {
                    long q1 = IDX(P, clampi(x + (i == 0), 0, P->NX - 1), clampi(y + (i == 1), 0, P->NY - 1),
                                  clampi(z + (i == 2), 0, P->NZ - 1));
                    sp[i][q] *= 0.5 * (d0[i][q] + d0[i][q1]);
                    sr[i][q] *= 0.5 * (dz[i][q] + dz[i][q1]);
                }
            }
    memset(H0p, 0, sizeof(double) * N);
    memset(Hzr, 0, sizeof(double) * N);
    for (int i = 0; i < 3; i++) {
        apply_axisT(line_DT_add, c0[i], H0p, i, P, -1.0);
        apply_axisT(line_DpT_add, sp[i], H0p, i, P, -1.0);
        apply_axisT(line_DT_add, cz[i], Hzr, i, P, -1.0);
        apply_axisT(line_DpT_add, sr[i], Hzr, i, P, -1.0);
    }
    for (int i = 0; i < 3; i++) {
        free(gp[i]); free(gr[i]); free(sp[i]); free(sr[i]);
        free(d0[i]); free(dz[i]); free(c0[i]); free(cz[i]);
    }
}

void or_tti_set_operator(or_prob *P, int op) { P->tti_op = op; }

/* exported for the plane-wave dispersion pin: L u = C [H0 p; Hz r] */
void or_tti_apply_L(const or_prob *P, const double *p, const double *r, double *Lp, double *Lr)
{
    double *H0p = dalloc(P->N), *Hzr = dalloc(P->N);
    tti_apply_H(P, p, r, H0p, Hzr);
    for (long q = 0; q < P->N; q++) {
        double a = 1.0 + 2.0 * P->eps[q], s = sqrt(1.0 + 2.0 * P->del[q]);
        Lp[q] = a * H0p[q] + s * Hzr[q];
        Lr[q] = s * H0p[q] + Hzr[q];
    }
    free(H0p); free(Hzr);
}

/* One leapfrog step (Sec. II-A listing: Eq(u.forward, solve(eq, u.forward))):
 *   A u^{n+1} = dt^2 L u^n + 2 m u^n - B u^{n-1},
 *   A = m (1 + sig dt/2),  B = m (1 - sig dt/2). */
static void tti_step(const or_prob *P, const double *p0, const double *p1,
                     const double *r0, const double *r1, double *p2, double *r2)
{
    long N = P->N;
    double dt = P->d.dt;
    double *H0p = dalloc(N), *Hzr = dalloc(N);
    tti_apply_H(P, p1, r1, H0p, Hzr);
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double a = 1.0 + 2.0 * P->eps[q], s = sqrt(1.0 + 2.0 * P->del[q]);
        double Lp = a * H0p[q] + s * Hzr[q];
        double Lr = s * H0p[q] + Hzr[q];
        double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
        double B = P->m[q] * (1.0 - 0.5 * P->sig[q] * dt);
        p2[q] = (dt * dt * Lp + 2.0 * P->m[q] * p1[q] - B * p0[q]) / A;
        r2[q] = (dt * dt * Lr + 2.0 * P->m[q] * r1[q] - B * r0[q]) / A;
    }
    free(H0p); free(Hzr);
}

/* Adjoint step: A lam^k = dt^2 H (C lam^{k+1}) + 2 m lam^{k+1} - B lam^{k+2}
 * (L^T = H^T C^T = H C: the coupling matrix goes INSIDE the stencil; this
 * is where the TTI system stops being self-adjoint, Sec. III-A).
 * Returns the right-hand side before division by A (receiver injection is
 * added by the caller). */
static void tti_adj_rhs(const or_prob *P, const double *l2, const double *l1,
                        const double *s2, const double *s1, double *rp, double *rr)
{
    long N = P->N;
    double dt = P->d.dt;
    double *zp = dalloc(N), *zr = dalloc(N), *H0 = dalloc(N), *Hz = dalloc(N);
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double a = 1.0 + 2.0 * P->eps[q], s = sqrt(1.0 + 2.0 * P->del[q]);
        zp[q] = a * l1[q] + s * s1[q];
        zr[q] = s * l1[q] + s1[q];
    }
    tti_apply_H(P, zp, zr, H0, Hz);
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double B = P->m[q] * (1.0 - 0.5 * P->sig[q] * dt);
        rp[q] = dt * dt * H0[q] + 2.0 * P->m[q] * l1[q] - B * l2[q];
        rr[q] = dt * dt * Hz[q] + 2.0 * P->m[q] * s1[q] - B * s2[q];
    }
    free(zp); free(zr); free(H0); free(Hz);
}

/* Forward modelling (Sec. II-A listing order, per time step n = 0..nt-1):
 *   d^n = R p^n  (interpolate u, not u.forward);
 *   u^{n+1} from the leapfrog step;
 *   inject q^n into p^{n+1} and r^{n+1} with factor dt^2 / A (= dt^2/m
 *   outside the absorbing layer, as s.inject(u.forward, expr=s*dt**2/m)).
 * traces: [nrec][nt].  store != 0 keeps (p^n, r^n), n = 0..nt, for the
 * gradient. */
int or_tti_forward(or_prob *P, int nsrc, const float *src, const float *wav,
                   int nrec, const float *rec, double *traces, int store)
{
    if (P->d.kind != 1) return OR_EINVAL;
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *p0 = dalloc(N), *p1 = dalloc(N), *p2 = dalloc(N);
    double *r0 = dalloc(N), *r1 = dalloc(N), *r2 = dalloc(N);
    if (store) {
        free(P->store);
        P->store = dalloc((long)(nt + 1) * 2 * N);
        if (!P->store) { free(S); free(R); return OR_ENOMEM; }
        P->stored = 1;
    }
    for (int n = 0; n < nt; n++) {
        for (int i = 0; i < nrec; i++) traces[(long)i * nt + n] = sample(&R[i], p1);
        tti_step(P, p0, p1, r0, r1, p2, r2);
        for (int s = 0; s < nsrc; s++)
            for (int c = 0; c < S[s].n; c++) {
                long q = S[s].idx[c];
                double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
                double v = dt * dt / A * S[s].w[c] * (double)wav[(long)s * nt + n];
                p2[q] += v;
                r2[q] += v;
            }
        if (store) {
            memcpy(P->store + (long)(n + 1) * 2 * N, p2, sizeof(double) * N);
            memcpy(P->store + ((long)(n + 1) * 2 + 1) * N, r2, sizeof(double) * N);
        }
        double *t;
        t = p0; p0 = p1; p1 = p2; p2 = t;
        t = r0; r0 = r1; r1 = r2; r2 = t;
    }
    free(p0); free(p1); free(p2); free(r0); free(r1); free(r2); free(S); free(R);
    return OR_OK;
}

/* Adjoint of or_tti_forward: traces [nrec][nt] -> source side [nsrc][nt].
 * Backward recursion k = nt-1 .. 1 (lam^{nt} = lam^{nt+1} = 0, since the
 * last residual sample r^{nt} does not exist):
 *   A lam^k = dt^2 H C lam^{k+1} + 2 m lam^{k+1} - B lam^{k+2} + R^T r^k,
 *   qbar^{k-1} = dt^2 P lam^k   (P samples p and r at the source).
 * If grad != NULL (computational grid, accumulated) the imaging condition
 *   g -= sum_f lam_f^{n+1} (a u_f^{n+1} - 2 u_f^n + b u_f^{n-1}),
 *   a = 1 + sig dt/2, b = 1 - sig dt/2  (d/dm of A u^{n+1} - 2m u^n + B u^{n-1})
 * is added using the stored forward wavefields. */
static int tti_adjoint_core(or_prob *P, int nrec, const float *rec, const double *res,
                            int nsrc, const float *src, double *qbar, double *grad,
                            double *grad_e, double *grad_d, double *grad_t, double *grad_f,
                            double *abs_tf)
{
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *l2 = dalloc(N), *l1 = dalloc(N), *l0 = dalloc(N);   /* lam^{k+2}, lam^{k+1}, lam^k */
    double *s2 = dalloc(N), *s1 = dalloc(N), *s0 = dalloc(N);
    if (qbar) memset(qbar, 0, sizeof(double) * (size_t)nsrc * nt);
    for (int k = nt - 1; k >= 1; k--) {
        tti_adj_rhs(P, l2, l1, s2, s1, l0, s0);
        for (int i = 0; i < nrec; i++)
            for (int c = 0; c < R[i].n; c++)
                l0[R[i].idx[c]] += R[i].w[c] * res[(long)i * nt + k];
#pragma omp parallel for
        for (long q = 0; q < N; q++) {
            double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
            l0[q] /= A;
            s0[q] /= A;
        }
        if (qbar)
            for (int s = 0; s < nsrc; s++)
                qbar[(long)s * nt + (k - 1)] = dt * dt * (sample(&S[s], l0) + sample(&S[s], s0));
        if (grad) {
            /* lam^k pairs with the forward equation of step n = k-1 */
            const double *up2 = P->store + (long)k * 2 * N, *ur2 = up2 + N;
            const double *up1 = P->store + (long)(k - 1) * 2 * N, *ur1 = up1 + N;
            const double *up0 = k >= 2 ? P->store + (long)(k - 2) * 2 * N : NULL;
            const double *ur0 = k >= 2 ? up0 + N : NULL;
#pragma omp parallel for
            for (long q = 0; q < N; q++) {
                double a = 1.0 + 0.5 * P->sig[q] * dt, b = 1.0 - 0.5 * P->sig[q] * dt;
                double dp = a * up2[q] - 2.0 * up1[q] + (up0 ? b * up0[q] : 0.0);
                double dr = a * ur2[q] - 2.0 * ur1[q] + (ur0 ? b * ur0[q] : 0.0);
                grad[q] -= l0[q] * dp + s0[q] * dr;
            }
        }
        if (grad_e && k >= 2) {
            /* anisotropy: the step n = k-1 depends on eps, delta only through
             * C in dt^2 C [H0 p^n; Hz r^n], with dC/deps = [[2, 0], [0, 0]] and
             * dC/ddelta = [[0, s'], [s', 0]], s' = 1 / sqrt(1 + 2 delta), so
             *   g_eps   += 2 dt^2 lam_p H0 p^n,
             *   g_delta += dt^2 s' (lam_p Hz r^n + lam_r H0 p^n)
             * (p^0 = r^0 = 0: no term for k = 1) */
            const double *up1 = P->store + (long)(k - 1) * 2 * N, *ur1 = up1 + N;
            double *H0 = dalloc(N), *Hz = dalloc(N);
            tti_apply_H(P, up1, ur1, H0, Hz);
#pragma omp parallel for
            for (long q = 0; q < N; q++) {
                grad_e[q] += 2.0 * dt * dt * l0[q] * H0[q];
                grad_d[q] += dt * dt / sqrt(1.0 + 2.0 * P->del[q]) * (l0[q] * Hz[q] + s0[q] * H0[q]);
            }
            free(H0); free(Hz);
        }
        if (grad_t && k >= 2) {
            /* tilt and azimuth: the step n = k-1 depends on theta, phi only
             * through H in dt^2 C H u^n, so the term is dt^2 (C lam)^T dH/dt u^n */
            const double *up1 = P->store + (long)(k - 1) * 2 * N, *ur1 = up1 + N;
            double *zp = dalloc(N), *zr = dalloc(N);
#pragma omp parallel for
            for (long q = 0; q < N; q++) {
                double a = 1.0 + 2.0 * P->eps[q], s = sqrt(1.0 + 2.0 * P->del[q]);
                zp[q] = a * l0[q] + s * s0[q];
                zr[q] = s * l0[q] + s0[q];
            }
            if (P->tti_op == 1)
                tti_frame_image_sp(P, zp, zr, up1, ur1, dt * dt, grad_t, grad_f, abs_tf, abs_tf ? abs_tf + N : NULL);
            else
                tti_frame_image(P, zp, zr, up1, ur1, dt * dt, grad_t, grad_f, abs_tf, abs_tf ? abs_tf + N : NULL);
            free(zp); free(zr);
        }
        double *t;
        t = l2; l2 = l1; l1 = l0; l0 = t;
        t = s2; s2 = s1; s1 = s0; s0 = t;
    }
    free(l0); free(l1); free(l2); free(s0); free(s1); free(s2); free(S); free(R);
    return OR_OK;
}

int or_tti_adjoint(or_prob *P, int nrec, const float *rec, const double *traces,
                   int nsrc, const float *src, double *qbar)
{
    if (P->d.kind != 1) return OR_EINVAL;
    return tti_adjoint_core(P, nrec, rec, traces, nsrc, src, qbar, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* FWI gradient w.r.t. m = 1/vp^2 on the PHYSICAL grid (fold of the
 * computational-grid gradient through the edge-replication extension),
 * J = 1/2 || F(m) q - d_obs ||^2. */
int or_tti_gradient(or_prob *P, int nsrc, const float *src, const float *wav,
                    int nrec, const float *rec, const double *d_obs,
                    double *grad_phys, double *misfit, double *grad_comp)
{
    if (P->d.kind != 1) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_tti_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    if (rc) { free(tr); return rc; }
    double J = 0.0;
    for (long i = 0; i < (long)nrec * nt; i++) {
        tr[i] -= d_obs[i];
        J += 0.5 * tr[i] * tr[i];
    }
    if (misfit) *misfit = J;
    double *g = dalloc(P->N);
    rc = tti_adjoint_core(P, nrec, rec, tr, nsrc, src, NULL, g, NULL, NULL, NULL, NULL, NULL);
    if (!rc) {
        if (grad_comp) memcpy(grad_comp, g, sizeof(double) * P->N);
        if (grad_phys) fold(g, grad_phys, P);
    }
    free(g); free(tr);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* Gradient w.r.t. (m, epsilon, delta, theta, phi) on the physical grid:
 * grad_phys [5][nx][ny][nz] (each folded through the edge replication).
 * abs_phys (may be NULL) [2][nx][ny][nz]: the theta and phi sums taken over
 * the magnitudes of their terms (the scale of their rounding errors). */
int or_tti_gradient_aniso(or_prob *P, int nsrc, const float *src, const float *wav,
                          int nrec, const float *rec, const double *d_obs,
                          double *grad_phys, double *misfit, double *abs_phys)
{
    if (P->d.kind != 1) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_tti_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    if (rc) { free(tr); return rc; }
    double J = 0.0;
    for (long i = 0; i < (long)nrec * nt; i++) {
        tr[i] -= d_obs[i];
        J += 0.5 * tr[i] * tr[i];
    }
    if (misfit) *misfit = J;
    double *g = dalloc(7 * P->N);
    rc = tti_adjoint_core(P, nrec, rec, tr, nsrc, src, NULL, g, g + P->N, g + 2 * P->N, g + 3 * P->N,
                          g + 4 * P->N, g + 5 * P->N);
    const long np = (long)P->d.nx * P->d.ny * P->d.nz;
    if (!rc && grad_phys)
        for (int c = 0; c < 5; c++) fold(g + c * P->N, grad_phys + c * np, P);
    if (!rc && abs_phys)
        for (int c = 0; c < 2; c++) fold(g + (5 + c) * P->N, abs_phys + c * np, P);
    free(g); free(tr);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* Same as or_tti_gradient but with the residual supplied directly (the
 * backward pass of an autograd function with incoming trace gradient). */
int or_tti_backward(or_prob *P, int nsrc, const float *src, const float *wav,
                    int nrec, const float *rec, const double *resid,
                    double *grad_phys, double *qbar)
{
    if (P->d.kind != 1) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_tti_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    free(tr);
    if (rc) return rc;
    double *g = dalloc(P->N);
    rc = tti_adjoint_core(P, nrec, rec, resid, nsrc, src, qbar, g, NULL, NULL, NULL, NULL, NULL);
    if (!rc && grad_phys) fold(g, grad_phys, P);
    free(g);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* One full-grid TTI step from a given state, no sources (float32 state in,
 * double out): p2 = step(p1, p0), r2 = step(r1, r0). adjoint != 0 applies
 * the adjoint step lam^k = (dt^2 H C lam^{k+1} + 2m lam^{k+1} - B lam^{k+2})/A. */
int or_tti_step_state(or_prob *P, const float *p0f, const float *p1f, const float *r0f,
                      const float *r1f, double *p2, double *r2, int adjoint)
{
    long N = P->N;
    double *p0 = dalloc(N), *p1 = dalloc(N), *r0 = dalloc(N), *r1 = dalloc(N);
    for (long q = 0; q < N; q++) { p0[q] = p0f[q]; p1[q] = p1f[q]; r0[q] = r0f[q]; r1[q] = r1f[q]; }
    if (!adjoint) tti_step(P, p0, p1, r0, r1, p2, r2);
    else {
        tti_adj_rhs(P, p0, p1, r0, r1, p2, r2);
        for (long q = 0; q < N; q++) {
            double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * P->d.dt);
            p2[q] /= A; r2[q] /= A;
        }
    }
    free(p0); free(p1); free(r0); free(r1);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Isotropic acoustic propagator (Sec. II-A, Eq. (acou) and the          */
/* wave-equation listing: m u_tt - laplace(u) + damp u_t = q), with the  */
/* damped leapfrog, injection and interpolation of the TTI path on one   */
/* wavefield.  L = sum over axes of the second derivative D2.            */
/* ------------------------------------------------------------------ */
static void ac_apply_L(const or_prob *P, const double *u, double *Lu)
{
    long N = P->N;
    double *t = dalloc(N);
    memset(Lu, 0, sizeof(double) * N);
    for (int a = 0; a < 3; a++) {
        apply_axis(line_D2, u, t, a, P);
        for (long q = 0; q < N; q++) Lu[q] += t[q];
    }
    free(t);
}

/* A u2 = dt^2 L u1 + 2 m u1 - B u0,  A = m (1 + sig dt/2), B = m (1 - sig dt/2).
 * L is symmetric, so the same map advances the adjoint state. */
static void ac_step(const or_prob *P, const double *u0, const double *u1, double *u2)
{
    long N = P->N;
    double dt = P->d.dt;
    double *Lu = dalloc(N);
    ac_apply_L(P, u1, Lu);
#pragma omp parallel for
    for (long q = 0; q < N; q++) {
        double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
        double B = P->m[q] * (1.0 - 0.5 * P->sig[q] * dt);
        u2[q] = (dt * dt * Lu[q] + 2.0 * P->m[q] * u1[q] - B * u0[q]) / A;
    }
    free(Lu);
}

/* Forward modelling, per time step n = 0..nt-1: d^n = R u^n; u^{n+1} from
 * the leapfrog step; q^n injected into u^{n+1} with factor dt^2 / A.
 * traces [nrec][nt]; store != 0 keeps u^n, n = 0..nt. */
int or_ac_forward(or_prob *P, int nsrc, const float *src, const float *wav,
                  int nrec, const float *rec, double *traces, int store)
{
    if (P->d.kind != 3) return OR_EINVAL;
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *u0 = dalloc(N), *u1 = dalloc(N), *u2 = dalloc(N);
    if (store) {
        free(P->store);
        P->store = dalloc((long)(nt + 1) * N);
        if (!P->store) { free(u0); free(u1); free(u2); free(S); free(R); return OR_ENOMEM; }
        P->stored = 1;
    }
    for (int n = 0; n < nt; n++) {
        for (int i = 0; i < nrec; i++) traces[(long)i * nt + n] = sample(&R[i], u1);
        ac_step(P, u0, u1, u2);
        for (int s = 0; s < nsrc; s++)
            for (int c = 0; c < S[s].n; c++) {
                long q = S[s].idx[c];
                double A = P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
                u2[q] += dt * dt / A * S[s].w[c] * (double)wav[(long)s * nt + n];
            }
        if (store) memcpy(P->store + (long)(n + 1) * N, u2, sizeof(double) * N);
        double *t = u0; u0 = u1; u1 = u2; u2 = t;
    }
    free(u0); free(u1); free(u2); free(S); free(R);
    return OR_OK;
}

/* Adjoint of or_ac_forward, k = nt-1 .. 1 (lam^{nt} = lam^{nt+1} = 0):
 *   A lam^k = dt^2 L lam^{k+1} + 2 m lam^{k+1} - B lam^{k+2} + R^T r^k,
 *   qbar^{k-1} = dt^2 (S lam^k);
 * grad != NULL: g -= lam^k (a u^k - 2 u^{k-1} + b u^{k-2}) with the stored
 * forward field (d/dm of the step's A u^{n+1} - 2 m u^n + B u^{n-1}). */
static int ac_adjoint_core(or_prob *P, int nrec, const float *rec, const double *res,
                           int nsrc, const float *src, double *qbar, double *grad)
{
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *l2 = dalloc(N), *l1 = dalloc(N), *l0 = dalloc(N), *Ll = dalloc(N);
    if (qbar) memset(qbar, 0, sizeof(double) * (size_t)nsrc * nt);
    for (int k = nt - 1; k >= 1; k--) {
        ac_apply_L(P, l1, Ll);
#pragma omp parallel for
        for (long q = 0; q < N; q++) {
            double B = P->m[q] * (1.0 - 0.5 * P->sig[q] * dt);
            l0[q] = dt * dt * Ll[q] + 2.0 * P->m[q] * l1[q] - B * l2[q];
        }
        for (int i = 0; i < nrec; i++)
            for (int c = 0; c < R[i].n; c++)
                l0[R[i].idx[c]] += R[i].w[c] * res[(long)i * nt + k];
#pragma omp parallel for
        for (long q = 0; q < N; q++) l0[q] /= P->m[q] * (1.0 + 0.5 * P->sig[q] * dt);
        if (qbar)
            for (int s = 0; s < nsrc; s++)
                qbar[(long)s * nt + (k - 1)] = dt * dt * sample(&S[s], l0);
        if (grad) {
            const double *u2 = P->store + (long)k * N, *u1 = P->store + (long)(k - 1) * N;
            const double *u0 = k >= 2 ? P->store + (long)(k - 2) * N : NULL;
#pragma omp parallel for
            for (long q = 0; q < N; q++) {
                double a = 1.0 + 0.5 * P->sig[q] * dt, b = 1.0 - 0.5 * P->sig[q] * dt;
                grad[q] -= l0[q] * (a * u2[q] - 2.0 * u1[q] + (u0 ? b * u0[q] : 0.0));
            }
        }
        double *t = l2; l2 = l1; l1 = l0; l0 = t;
    }
    free(l0); free(l1); free(l2); free(Ll); free(S); free(R);
    return OR_OK;
}

int or_ac_adjoint(or_prob *P, int nrec, const float *rec, const double *traces,
                  int nsrc, const float *src, double *qbar)
{
    if (P->d.kind != 3) return OR_EINVAL;
    return ac_adjoint_core(P, nrec, rec, traces, nsrc, src, qbar, NULL);
}

/* dJ/dm on the physical grid (fold of the computational gradient),
 * J = 1/2 || F(m) q - d_obs ||^2; grad_comp (may be NULL) the unfolded one. */
int or_ac_gradient(or_prob *P, int nsrc, const float *src, const float *wav,
                   int nrec, const float *rec, const double *d_obs,
                   double *grad_phys, double *misfit, double *grad_comp)
{
    if (P->d.kind != 3) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_ac_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    if (rc) { free(tr); return rc; }
    double J = 0.0;
    for (long i = 0; i < (long)nrec * nt; i++) {
        tr[i] -= d_obs[i];
        J += 0.5 * tr[i] * tr[i];
    }
    if (misfit) *misfit = J;
    double *g = dalloc(P->N);
    rc = ac_adjoint_core(P, nrec, rec, tr, nsrc, src, NULL, g);
    if (!rc) {
        if (grad_comp) memcpy(grad_comp, g, sizeof(double) * P->N);
        if (grad_phys) fold(g, grad_phys, P);
    }
    free(g); free(tr);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* (dJ/dm, dJ/dwavelet) for a given trace residual (autograd backward). */
int or_ac_backward(or_prob *P, int nsrc, const float *src, const float *wav,
                   int nrec, const float *rec, const double *resid,
                   double *grad_phys, double *qbar)
{
    if (P->d.kind != 3) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_ac_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    free(tr);
    if (rc) return rc;
    double *g = dalloc(P->N);
    rc = ac_adjoint_core(P, nrec, rec, resid, nsrc, src, qbar, g);
    if (!rc && grad_phys) fold(g, grad_phys, P);
    free(g);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* nsteps source-free steps of a double state (u0, u1) = (u^{n-1}, u^n) in
 * place: afterwards u1 holds the newest level and u0 the one before. */
int or_ac_step_state_d(or_prob *P, double *u0, double *u1, int nsteps)
{
    if (P->d.kind != 3) return OR_EINVAL;
    double *u2 = dalloc(P->N);
    for (int i = 0; i < nsteps; i++) {
        ac_step(P, u0, u1, u2);
        memcpy(u0, u1, sizeof(double) * P->N);
        memcpy(u1, u2, sizeof(double) * P->N);
    }
    free(u2);
    return OR_OK;
}

/* one step evaluated at npts points idx[] (computational-grid linear
 * indices) from a float32 state (u0, u1); model: the PHYSICAL float32 vp
 * (edge replication by clamped indices); out[i] = u^{n+1} at idx[i]. */
int or_ac_step_points(const or_desc *d, const float *vp, const float *u0, const float *u1,
                      int npts, const long *idx, double *out)
{
    if (d->kind != 3) return OR_EINVAL;
    const int NX = d->nx + 2 * d->nbl, NY = d->ny + 2 * d->nbl, NZ = d->nz + 2 * d->nbl, M = d->so / 2;
    double w[MAXM + 1];
    if (or_weights_d2(d->so, w)) return OR_EINVAL;
    long np = (long)d->nx * d->ny * d->nz;
    double vmax = 0.0;
    for (long q = 0; q < np; q++)
        if (1000.0 * (double)vp[q] > vmax) vmax = 1000.0 * (double)vp[q];
    if (d->vdamp > 0) vmax = d->vdamp;
    or_prob Pd; memset(&Pd, 0, sizeof(Pd)); Pd.d = *d;
    const double dt = d->dt, h2 = d->h * d->h;
#pragma omp parallel for
    for (int i = 0; i < npts; i++) {
        long q = idx[i];
        int z = (int)(q % NZ), y = (int)((q / NZ) % NY), x = (int)(q / ((long)NZ * NY));
        double L = 3.0 * w[0] * u1[q];
        for (int k = 1; k <= M; k++) {
            int c[6][3] = {{x + k, y, z}, {x - k, y, z}, {x, y + k, z}, {x, y - k, z}, {x, y, z + k}, {x, y, z - k}};
            for (int j = 0; j < 6; j++) {
                int a = c[j][0], b = c[j][1], e = c[j][2];
                if (a < 0 || a >= NX || b < 0 || b >= NY || e < 0 || e >= NZ) continue;
                L += w[k] * u1[((long)a * NY + b) * NZ + e];
            }
        }
        L /= h2;
        int pi = clampi(x - d->nbl, 0, d->nx - 1), pj = clampi(y - d->nbl, 0, d->ny - 1),
            pk = clampi(z - d->nbl, 0, d->nz - 1);
        double v = 1000.0 * (double)vp[((long)pi * d->ny + pj) * d->nz + pk];
        double m = 1.0 / (v * v), sg = tti_sigma(&Pd, x, y, z, vmax);
        double A = m * (1.0 + 0.5 * sg * dt), B = m * (1.0 - 0.5 * sg * dt);
        out[i] = (dt * dt * L + 2.0 * m * u1[q] - B * u0[q]) / A;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* TTI at single points (sampled parity at full size)                   */
/* Same definitions evaluated locally; model read from the PHYSICAL     */
/* float32 arrays with clamped indices (= edge-replication extension).  */
/* ------------------------------------------------------------------ */
typedef struct {
    const or_desc *d; int NX, NY, NZ, M; double c[MAXM + 1], b[MAXM + 1];
    const float *vp, *eps, *del, *th, *ph; double vmax;
} pt_ctx;

static double pt_model(const pt_ctx *C, const float *a, int x, int y, int z)
{
    int i = clampi(x - C->d->nbl, 0, C->d->nx - 1);
    int j = clampi(y - C->d->nbl, 0, C->d->ny - 1);
    int k = clampi(z - C->d->nbl, 0, C->d->nz - 1);
    return (double)a[((long)i * C->d->ny + j) * C->d->nz + k];
}
static int pt_in(const pt_ctx *C, int x, int y, int z)
{
    return x >= 0 && x < C->NX && y >= 0 && y < C->NY && z >= 0 && z < C->NZ;
}
static double pt_f(const pt_ctx *C, const float *u, int x, int y, int z)
{
    if (!pt_in(C, x, y, z)) return 0.0;
    return (double)u[((long)x * C->NY + y) * C->NZ + z];
}
/* (D_i u)(x) with zero extension */
static double pt_D(const pt_ctx *C, const float *u, int ax, int x, int y, int z)
{
    double acc = 0.0;
    for (int k = 1; k <= C->M; k++) {
        int xp = x + (ax == 0) * k, yp = y + (ax == 1) * k, zp = z + (ax == 2) * k;
        int xm = x - (ax == 0) * k, ym = y - (ax == 1) * k, zm = z - (ax == 2) * k;
        acc += C->c[k] * (pt_f(C, u, xp, yp, zp) - pt_f(C, u, xm, ym, zm));
    }
    return acc / C->d->h;
}
/* field w_a,i(y) = a_i(y) * D_a u(y) for frame vector a (0: xb, 1: yb, 2: zb), 0 outside */
static double pt_w(const pt_ctx *C, const float *u, int a, int i, int x, int y, int z,
                   const float *pre, double cp, double cr, const float *u2)
{
    if (!pt_in(C, x, y, z)) return 0.0;
    double xb[3], yb[3], zb[3];
    frame(pt_model(C, C->th, x, y, z), pt_model(C, C->ph, x, y, z), xb, yb, zb);
    const double *v = a == 0 ? xb : (a == 1 ? yb : zb);
    double g[3];
    for (int j = 0; j < 3; j++) {
        if (!pre) g[j] = pt_D(C, u, j, x, y, z);
        else {
            /* derivative of the pointwise combination cp*u + cr*u2 with
             * coefficients from C(eps, delta) at each neighbour (adjoint) */
            double acc = 0.0;
            for (int k = 1; k <= C->M; k++) {
                int s[2] = {k, -k};
                for (int t = 0; t < 2; t++) {
                    int xx = x + (j == 0) * s[t], yy = y + (j == 1) * s[t], zz = z + (j == 2) * s[t];
                    if (!pt_in(C, xx, yy, zz)) continue;
                    double e = pt_model(C, C->eps, xx, yy, zz), dl = pt_model(C, C->del, xx, yy, zz);
                    double ca = 1.0 + 2.0 * e, cs = sqrt(1.0 + 2.0 * dl);
                    double val = (cp > 0.5) ? ca * pt_f(C, u, xx, yy, zz) + cs * pt_f(C, u2, xx, yy, zz)
                                            : cs * pt_f(C, u, xx, yy, zz) + pt_f(C, u2, xx, yy, zz);
                    acc += (t == 0 ? 1.0 : -1.0) * C->c[k] * val;
                }
            }
            (void)cr;
            g[j] = acc / C->d->h;
        }
    }
    double Da = v[0] * g[0] + v[1] * g[1] + v[2] * g[2];
    return v[i] * Da;
}
/* (D_i^T w)(x) = (1/h) sum_k c_k (w(x - k e_i) - w(x + k e_i)) */
static double pt_G(const pt_ctx *C, const float *u, int a, int x, int y, int z,
                   const float *pre, double cp, const float *u2)
{
    double acc = 0.0;
    for (int i = 0; i < 3; i++)
        for (int k = 1; k <= C->M; k++) {
            int xm = x - (i == 0) * k, ym = y - (i == 1) * k, zm = z - (i == 2) * k;
            int xp = x + (i == 0) * k, yp = y + (i == 1) * k, zp = z + (i == 2) * k;
            acc += C->c[k] * (pt_w(C, u, a, i, xm, ym, zm, pre, cp, 0, u2) -
                              pt_w(C, u, a, i, xp, yp, zp, pre, cp, 0, u2));
        }
    return acc / C->d->h;
}

/* Staggered-pair operators (the form of tti_apply_H_sp) at one point.  A
 * field accessor gives the differentiated field at a node, zero outside the
 * grid: mode 0 the array u itself; in the transposed step the pointwise
 * combinations zeta = C lam with C from eps, delta at that node (mode 1:
 * (1+2eps) u + sqrt(1+2delta) u2, mode 2: sqrt(1+2delta) u + u2). */
typedef struct { const pt_ctx *C; const float *u, *u2; int mode; } pt_fld;

static double fld_at(const pt_fld *F, int x, int y, int z)
{
    const pt_ctx *C = F->C;
    if (!pt_in(C, x, y, z)) return 0.0;
    double a = pt_f(C, F->u, x, y, z);
    if (F->mode == 0) return a;
    double ca = 1.0 + 2.0 * pt_model(C, C->eps, x, y, z), cs = sqrt(1.0 + 2.0 * pt_model(C, C->del, x, y, z));
    double b = pt_f(C, F->u2, x, y, z);
    return F->mode == 1 ? ca * a + cs * b : cs * a + b;
}
/* centred (D_ax f)(node) and staggered (D+_ax f)(node + 1/2) */
static double fld_D(const pt_fld *F, int ax, int x, int y, int z, int staggered)
{
    const pt_ctx *C = F->C;
    double acc = 0.0;
    for (int k = 1; k <= C->M; k++) {
        int kp = k, km = staggered ? k - 1 : k;
        double fp = fld_at(F, x + (ax == 0) * kp, y + (ax == 1) * kp, z + (ax == 2) * kp);
        double fm = fld_at(F, x - (ax == 0) * km, y - (ax == 1) * km, z - (ax == 2) * km);
        acc += (staggered ? C->b[k] : C->c[k]) * (fp - fm);
    }
    return acc / C->d->h;
}
/* entry (i, j) of P0 = xb xb^T + yb yb^T (which = 0) or Pz = zb zb^T (1) at a node */
static double sp_P(const pt_ctx *C, int which, int i, int j, int x, int y, int z)
{
    double xb[3], yb[3], zb[3];
    frame(pt_model(C, C->th, x, y, z), pt_model(C, C->ph, x, y, z), xb, yb, zb);
    return which ? zb[i] * zb[j] : xb[i] * xb[j] + yb[i] * yb[j];
}
/* cross flux sum_{j != i} P_ij D_j f at a node (0 outside) */
static double sp_cross(const pt_fld *F, int which, int i, int x, int y, int z)
{
    if (!pt_in(F->C, x, y, z)) return 0.0;
    double acc = 0.0;
    for (int j = 0; j < 3; j++)
        if (j != i) acc += sp_P(F->C, which, i, j, x, y, z) * fld_D(F, j, x, y, z, 0);
    return acc;
}
/* diagonal flux at the half point node + e_i/2: the two-node average of
 * P_ii (the neighbour clamped at the last node) times D+_i f (0 outside) */
static double sp_diag(const pt_fld *F, int which, int i, int x, int y, int z)
{
    const pt_ctx *C = F->C;
    if (!pt_in(C, x, y, z)) return 0.0;
    int x1 = clampi(x + (i == 0), 0, C->NX - 1), y1 = clampi(y + (i == 1), 0, C->NY - 1),
        z1 = clampi(z + (i == 2), 0, C->NZ - 1);
    double pa = 0.5 * (sp_P(C, which, i, i, x, y, z) + sp_P(C, which, i, i, x1, y1, z1));
    return pa * fld_D(F, i, x, y, z, 1);
}
/* H u = -sum_i [ D_i^T (cross flux) + (D+_i)^T (diagonal flux) ] at a node, with
 * (D_i^T w)(x) = (1/h) sum_k c_k (w(x - k) - w(x + k)) and
 * ((D+_i)^T s)(x) = (1/h) sum_k b_k (s(x - k) - s(x + k - 1)) */
static double sp_H(const pt_fld *F, int which, int x, int y, int z)
{
    const pt_ctx *C = F->C;
    double acc = 0.0;
    for (int i = 0; i < 3; i++)
        for (int k = 1; k <= C->M; k++) {
            int ex = (i == 0), ey = (i == 1), ez = (i == 2);
            acc += C->c[k] * (sp_cross(F, which, i, x - ex * k, y - ey * k, z - ez * k) -
                              sp_cross(F, which, i, x + ex * k, y + ey * k, z + ez * k));
            acc += C->b[k] * (sp_diag(F, which, i, x - ex * k, y - ey * k, z - ez * k) -
                              sp_diag(F, which, i, x + ex * (k - 1), y + ey * (k - 1), z + ez * (k - 1)));
        }
    return -acc / C->d->h;
}

/* Values of one step (forward, or adjoint if adjoint != 0) at npts points
 * idx[] (computational-grid linear indices).  State arrays are float32 on
 * the computational grid: (p0, p1, r0, r1) = (u^{n-1}, u^n) for p and r
 * (adjoint: lam^{k+2}, lam^{k+1}).  Model arrays are the PHYSICAL float32
 * inputs. out[2*i] = p2, out[2*i+1] = r2. */
int or_tti_step_points_op(const or_desc *d, const float *const *model,
                          const float *p0, const float *p1, const float *r0, const float *r1,
                          int npts, const long *idx, double *out, int adjoint, int op)
{
    pt_ctx C;
    C.d = d; C.NX = d->nx + 2 * d->nbl; C.NY = d->ny + 2 * d->nbl; C.NZ = d->nz + 2 * d->nbl;
    C.M = d->so / 2;
    if (op != 0 && op != 1) return OR_EINVAL;
    double tmp[MAXM];
    if (or_weights_centred(d->so, tmp)) return OR_EINVAL;
    for (int k = 1; k <= C.M; k++) C.c[k] = tmp[k - 1];
    if (or_weights_staggered(d->so, tmp)) return OR_EINVAL;
    for (int k = 1; k <= C.M; k++) C.b[k] = tmp[k - 1];
    C.vp = model[0]; C.eps = model[1]; C.del = model[2]; C.th = model[3]; C.ph = model[4];
    long np = (long)d->nx * d->ny * d->nz;
    double vmax = 0.0;
    for (long q = 0; q < np; q++) {
        double v = 1000.0 * (double)C.vp[q] * sqrt(1.0 + 2.0 * (double)C.eps[q]);
        if (v > vmax) vmax = v;
    }
    if (d->vdamp > 0) vmax = d->vdamp;
    or_prob Pd; memset(&Pd, 0, sizeof(Pd)); Pd.d = *d;
#pragma omp parallel for
    for (int i = 0; i < npts; i++) {
        long q = idx[i];
        int z = (int)(q % C.NZ), y = (int)((q / C.NZ) % C.NY), x = (int)(q / ((long)C.NZ * C.NY));
        double H0, Hz;
        if (op == 1) {                   /* staggered-pair operators */
            pt_fld Fp = {&C, p1, r1, adjoint ? 1 : 0}, Fr = {&C, adjoint ? p1 : r1, r1, adjoint ? 2 : 0};
            H0 = sp_H(&Fp, 0, x, y, z);
            Hz = sp_H(&Fr, 1, x, y, z);
        } else if (!adjoint) {
            H0 = -(pt_G(&C, p1, 0, x, y, z, NULL, 0, NULL) + pt_G(&C, p1, 1, x, y, z, NULL, 0, NULL));
            Hz = -pt_G(&C, r1, 2, x, y, z, NULL, 0, NULL);
        } else {
            H0 = -(pt_G(&C, p1, 0, x, y, z, p1, 1.0, r1) + pt_G(&C, p1, 1, x, y, z, p1, 1.0, r1));
            Hz = -pt_G(&C, p1, 2, x, y, z, p1, 0.0, r1);
        }
        double e = pt_model(&C, C.eps, x, y, z), dl = pt_model(&C, C.del, x, y, z);
        double vp = 1000.0 * pt_model(&C, C.vp, x, y, z);
        double m = 1.0 / (vp * vp);
        double sg = tti_sigma(&Pd, x, y, z, vmax);
        double dt = d->dt;
        double A = m * (1.0 + 0.5 * sg * dt), B = m * (1.0 - 0.5 * sg * dt);
        double Lp, Lr;
        if (!adjoint) {
            double a = 1.0 + 2.0 * e, s = sqrt(1.0 + 2.0 * dl);
            Lp = a * H0 + s * Hz;
            Lr = s * H0 + Hz;
        } else { Lp = H0; Lr = Hz; }
        double P1 = pt_f(&C, p1, x, y, z), P0 = pt_f(&C, p0, x, y, z);
        double R1 = pt_f(&C, r1, x, y, z), R0 = pt_f(&C, r0, x, y, z);
        out[2 * i] = (dt * dt * Lp + 2.0 * m * P1 - B * P0) / A;
        out[2 * i + 1] = (dt * dt * Lr + 2.0 * m * R1 - B * R0) / A;
    }
    return OR_OK;
}

int or_tti_step_points(const or_desc *d, const float *const *model,
                       const float *p0, const float *p1, const float *r0, const float *r1,
                       int npts, const long *idx, double *out, int adjoint)
{
    return or_tti_step_points_op(d, model, p0, p1, r0, r1, npts, idx, out, adjoint, 0);
}

/* ------------------------------------------------------------------ */
/* Elastic (Sec. IV, Eq. elas1, elastic listing)                        */
/* ------------------------------------------------------------------ */
/* Staggering: txx, tyy, tzz, lam, mu, rho at nodes (i,j,k); vx at
 * (i+1/2,j,k), vy at (i,j+1/2,k), vz at (i,j,k+1/2); txy at (i+1/2,j+1/2,k),
 * txz at (i+1/2,j,k+1/2), tyz at (i,j+1/2,k+1/2); half index i+1/2 stored
 * at i.  Half-node averaging: buoyancy = mean of the 2 adjacent nodes,
 * shear modulus = mean of the 4 surrounding nodes (indices clamped to the
 * grid).  State order: vx vy vz txx tyy tzz txy txz tyz. */
enum { VX, VY, VZ, TXX, TYY, TZZ, TXY, TXZ, TYZ };

static double bavg(const or_prob *P, int ax, int x, int y, int z)
{
    int x1 = clampi(x + (ax == 0), 0, P->NX - 1);
    int y1 = clampi(y + (ax == 1), 0, P->NY - 1);
    int z1 = clampi(z + (ax == 2), 0, P->NZ - 1);
    return 0.5 * (P->bu[IDX(P, x, y, z)] + P->bu[IDX(P, x1, y1, z1)]);
}
/* 4 node indices around the edge point of the (a1, a2) plane */
static void edge_nodes(const or_prob *P, int a1, int a2, int x, int y, int z, long *q)
{
    int n = 0;
    for (int s = 0; s < 2; s++)
        for (int t = 0; t < 2; t++) {
            int xx = x + (a1 == 0) * s + (a2 == 0) * t;
            int yy = y + (a1 == 1) * s + (a2 == 1) * t;
            int zz = z + (a1 == 2) * s + (a2 == 2) * t;
            q[n++] = IDX(P, clampi(xx, 0, P->NX - 1), clampi(yy, 0, P->NY - 1), clampi(zz, 0, P->NZ - 1));
        }
}
static double muavg(const or_prob *P, int a1, int a2, int x, int y, int z)
{
    long q[4];
    edge_nodes(P, a1, a2, x, y, z, q);
    return 0.25 * (P->mu[q[0]] + P->mu[q[1]] + P->mu[q[2]] + P->mu[q[3]]);
}
/* taper at the staggered position of a component */
static double gtaper(const or_prob *P, int comp, int x, int y, int z)
{
    double sx = x, sy = y, sz = z;
    switch (comp) {
    case VX: sx += 0.5; break;
    case VY: sy += 0.5; break;
    case VZ: sz += 0.5; break;
    case TXY: sx += 0.5; sy += 0.5; break;
    case TXZ: sx += 0.5; sz += 0.5; break;
    case TYZ: sy += 0.5; sz += 0.5; break;
    default: break;
    }
    return cerjan(P, sx, sy, sz);
}

/* divergence of stress at the velocity positions: Dtau(tau) */
static void el_div_tau(const or_prob *P, double *const *s, double *dv[3])
{
    long N = P->N;
    double *t = dalloc(N);
    for (int c = 0; c < 3; c++) memset(dv[c], 0, sizeof(double) * N);
    /* x: D+x txx + D-y txy + D-z txz */
    apply_axis(line_Dp, s[TXX], t, 0, P); for (long q = 0; q < N; q++) dv[0][q] += t[q];
    apply_axis(line_Dm, s[TXY], t, 1, P); for (long q = 0; q < N; q++) dv[0][q] += t[q];
    apply_axis(line_Dm, s[TXZ], t, 2, P); for (long q = 0; q < N; q++) dv[0][q] += t[q];
    /* y: D-x txy + D+y tyy + D-z tyz */
    apply_axis(line_Dm, s[TXY], t, 0, P); for (long q = 0; q < N; q++) dv[1][q] += t[q];
    apply_axis(line_Dp, s[TYY], t, 1, P); for (long q = 0; q < N; q++) dv[1][q] += t[q];
    apply_axis(line_Dm, s[TYZ], t, 2, P); for (long q = 0; q < N; q++) dv[1][q] += t[q];
    /* z: D-x txz + D-y tyz + D+z tzz */
    apply_axis(line_Dm, s[TXZ], t, 0, P); for (long q = 0; q < N; q++) dv[2][q] += t[q];
    apply_axis(line_Dm, s[TYZ], t, 1, P); for (long q = 0; q < N; q++) dv[2][q] += t[q];
    apply_axis(line_Dp, s[TZZ], t, 2, P); for (long q = 0; q < N; q++) dv[2][q] += t[q];
    free(t);
}

/* strain-like derivatives of velocity: S(v) = (exx, eyy, ezz, gxy, gxz, gyz) */
static void el_strain(const or_prob *P, double *const *s, double *e[6])
{
    long N = P->N;
    double *t = dalloc(N);
    apply_axis(line_Dm, s[VX], e[0], 0, P);
    apply_axis(line_Dm, s[VY], e[1], 1, P);
    apply_axis(line_Dm, s[VZ], e[2], 2, P);
    apply_axis(line_Dp, s[VX], e[3], 1, P); apply_axis(line_Dp, s[VY], t, 0, P);
    for (long q = 0; q < N; q++) e[3][q] += t[q];
    apply_axis(line_Dp, s[VX], e[4], 2, P); apply_axis(line_Dp, s[VZ], t, 0, P);
    for (long q = 0; q < N; q++) e[4][q] += t[q];
    apply_axis(line_Dp, s[VY], e[5], 2, P); apply_axis(line_Dp, s[VZ], t, 1, P);
    for (long q = 0; q < N; q++) e[5][q] += t[q];
    free(t);
}

/* stiffness applied to strain: sigma = C(lam, mu) e */
static void el_stiff(const or_prob *P, double *const *e, double *sg[6])
{
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                double tr = e[0][q] + e[1][q] + e[2][q];
                for (int i = 0; i < 3; i++) sg[i][q] = P->lam[q] * tr + 2.0 * P->mu[q] * e[i][q];
                sg[3][q] = muavg(P, 0, 1, x, y, z) * e[3][q];
                sg[4][q] = muavg(P, 0, 2, x, y, z) * e[4][q];
                sg[5][q] = muavg(P, 1, 2, x, y, z) * e[5][q];
            }
}

/* One forward step in place (elastic listing):
 *   v   <- g (v + dt b div tau)
 *   tau <- g (tau + dt (lam tr(grad v) I + mu (grad v + grad v^T)))   (new v) */
static void el_step(const or_prob *P, double *const *s)
{
    long N = P->N; double dt = P->d.dt;
    double *dv[3], *e[6], *sg[6];
    for (int i = 0; i < 3; i++) dv[i] = dalloc(N);
    for (int i = 0; i < 6; i++) { e[i] = dalloc(N); sg[i] = dalloc(N); }
    el_div_tau(P, s, dv);
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                for (int c = 0; c < 3; c++)
                    s[VX + c][q] = gtaper(P, VX + c, x, y, z) *
                                   (s[VX + c][q] + dt * bavg(P, c, x, y, z) * dv[c][q]);
            }
    el_strain(P, s, e);
    el_stiff(P, e, sg);
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                for (int c = 0; c < 6; c++)
                    s[TXX + c][q] = gtaper(P, TXX + c, x, y, z) * (s[TXX + c][q] + dt * sg[c][q]);
            }
    for (int i = 0; i < 3; i++) free(dv[i]);
    for (int i = 0; i < 6; i++) { free(e[i]); free(sg[i]); }
}

/* Transpose of el_step, in place on the adjoint state (literal transposes):
 *   t = g tau' ;  vbar = v' + dt S^T (C t) ;  tau = t ;
 *   s = g vbar ;  tau += dt Dtau^T (b s) ;  v = s.
 * If gfwd != NULL, accumulates the gradient w.r.t. nodal (lam, mu, b) using
 * the forward state before the step (xf0: tau^n) and after it (xf1: v^{n+1}). */
static void el_step_T(const or_prob *P, double *const *s, double *const *xf0,
                      double *const *xf1, double *const *gfwd)
{
    long N = P->N; double dt = P->d.dt;
    double *t[6], *sg[6], *tmp = dalloc(N);
    for (int i = 0; i < 6; i++) { t[i] = dalloc(N); sg[i] = dalloc(N); }
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                for (int c = 0; c < 6; c++) t[c][q] = gtaper(P, TXX + c, x, y, z) * s[TXX + c][q];
            }
    if (gfwd) {
        /* d/d(lam, mu): dt <t, (dC) S v^{n+1}> */
        double *e[6];
        for (int i = 0; i < 6; i++) e[i] = dalloc(N);
        el_strain(P, xf1, e);
        for (int x = 0; x < P->NX; x++)
            for (int y = 0; y < P->NY; y++)
                for (int z = 0; z < P->NZ; z++) {
                    long q = IDX(P, x, y, z);
                    double tr = e[0][q] + e[1][q] + e[2][q];
                    gfwd[0][q] += dt * (t[0][q] + t[1][q] + t[2][q]) * tr;
                    gfwd[1][q] += dt * 2.0 * (t[0][q] * e[0][q] + t[1][q] * e[1][q] + t[2][q] * e[2][q]);
                    long nq[4];
                    int pl[3][2] = {{0, 1}, {0, 2}, {1, 2}};
                    for (int c = 0; c < 3; c++) {
                        edge_nodes(P, pl[c][0], pl[c][1], x, y, z, nq);
                        double v = 0.25 * dt * t[3 + c][q] * e[3 + c][q];
                        for (int u = 0; u < 4; u++) gfwd[1][nq[u]] += v;
                    }
                }
        for (int i = 0; i < 6; i++) free(e[i]);
    }
    el_stiff(P, t, sg);
    /* v' += dt S^T sigma, S^T written as the scatter transposes of el_strain */
    apply_axisT(line_DmT_add, sg[0], s[VX], 0, P, dt);
    apply_axisT(line_DmT_add, sg[1], s[VY], 1, P, dt);
    apply_axisT(line_DmT_add, sg[2], s[VZ], 2, P, dt);
    apply_axisT(line_DpT_add, sg[3], s[VX], 1, P, dt);
    apply_axisT(line_DpT_add, sg[3], s[VY], 0, P, dt);
    apply_axisT(line_DpT_add, sg[4], s[VX], 2, P, dt);
    apply_axisT(line_DpT_add, sg[4], s[VZ], 0, P, dt);
    apply_axisT(line_DpT_add, sg[5], s[VY], 2, P, dt);
    apply_axisT(line_DpT_add, sg[5], s[VZ], 1, P, dt);
    for (int c = 0; c < 6; c++) memcpy(s[TXX + c], t[c], sizeof(double) * N);
    /* s = g vbar ; w = b s */
    double *w[3];
    for (int c = 0; c < 3; c++) w[c] = dalloc(N);
#pragma omp parallel for collapse(2)
    for (int x = 0; x < P->NX; x++)
        for (int y = 0; y < P->NY; y++)
            for (int z = 0; z < P->NZ; z++) {
                long q = IDX(P, x, y, z);
                for (int c = 0; c < 3; c++) {
                    s[VX + c][q] *= gtaper(P, VX + c, x, y, z);
                    w[c][q] = bavg(P, c, x, y, z) * s[VX + c][q];
                }
            }
    if (gfwd) {
        /* d/db: dt <g vbar, (d b_avg) Dtau tau^n>, b_avg = (b_i + b_{i+1})/2 */
        double *dv[3];
        for (int c = 0; c < 3; c++) dv[c] = dalloc(N);
        el_div_tau(P, xf0, dv);
        for (int x = 0; x < P->NX; x++)
            for (int y = 0; y < P->NY; y++)
                for (int z = 0; z < P->NZ; z++) {
                    long q = IDX(P, x, y, z);
                    for (int c = 0; c < 3; c++) {
                        double v = 0.5 * dt * s[VX + c][q] * dv[c][q];
                        int x1 = clampi(x + (c == 0), 0, P->NX - 1);
                        int y1 = clampi(y + (c == 1), 0, P->NY - 1);
                        int z1 = clampi(z + (c == 2), 0, P->NZ - 1);
                        gfwd[2][q] += v;
                        gfwd[2][IDX(P, x1, y1, z1)] += v;
                    }
                }
        for (int c = 0; c < 3; c++) free(dv[c]);
    }
    /* tau += dt Dtau^T w (scatter transposes of el_div_tau) */
    apply_axisT(line_DpT_add, w[0], s[TXX], 0, P, dt);
    apply_axisT(line_DmT_add, w[0], s[TXY], 1, P, dt);
    apply_axisT(line_DmT_add, w[0], s[TXZ], 2, P, dt);
    apply_axisT(line_DmT_add, w[1], s[TXY], 0, P, dt);
    apply_axisT(line_DpT_add, w[1], s[TYY], 1, P, dt);
    apply_axisT(line_DmT_add, w[1], s[TYZ], 2, P, dt);
    apply_axisT(line_DmT_add, w[2], s[TXZ], 0, P, dt);
    apply_axisT(line_DmT_add, w[2], s[TYZ], 1, P, dt);
    apply_axisT(line_DpT_add, w[2], s[TZZ], 2, P, dt);
    for (int c = 0; c < 3; c++) free(w[c]);
    for (int i = 0; i < 6; i++) { free(t[i]); free(sg[i]); }
    free(tmp);
}

/* Elastic forward: per step n, d^n = R (txx + tyy + tzz)^n (pressure-like
 * trace of stress, Sec. IV-B), then the step, then the explosive source
 * tau_ii^{n+1} += dt w q^n, i = x, y, z. */
int or_el_forward(or_prob *P, int nsrc, const float *src, const float *wav,
                  int nrec, const float *rec, double *traces, int store)
{
    if (P->d.kind != 2) return OR_EINVAL;
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = dalloc(N);
    if (store) {
        free(P->store);
        P->store = dalloc((long)(nt + 1) * 9 * N);
        if (!P->store) { free(S); free(R); for (int c = 0; c < 9; c++) free(s[c]); return OR_ENOMEM; }
        P->stored = 1;
    }
    for (int n = 0; n < nt; n++) {
        for (int i = 0; i < nrec; i++)
            traces[(long)i * nt + n] = sample(&R[i], s[TXX]) + sample(&R[i], s[TYY]) + sample(&R[i], s[TZZ]);
        el_step(P, s);
        for (int j = 0; j < nsrc; j++)
            for (int c = 0; c < S[j].n; c++) {
                double v = dt * S[j].w[c] * (double)wav[(long)j * nt + n];
                s[TXX][S[j].idx[c]] += v;
                s[TYY][S[j].idx[c]] += v;
                s[TZZ][S[j].idx[c]] += v;
            }
        if (store)
            for (int c = 0; c < 9; c++)
                memcpy(P->store + ((long)(n + 1) * 9 + c) * N, s[c], sizeof(double) * N);
    }
    for (int c = 0; c < 9; c++) free(s[c]);
    free(S); free(R);
    return OR_OK;
}

/* Adjoint: Xbar^{nt} = 0; k = nt-1 .. 1: Xbar^k = M^T Xbar^{k+1} + R^T r^k,
 * qbar^{k-1} = dt P (tbar_xx + tbar_yy + tbar_zz)^k.  With grad != NULL,
 * accumulate the (lam, mu, b) gradient of step n = k (forward store). */
static int el_adjoint_core(or_prob *P, int nrec, const float *rec, const double *res,
                           int nsrc, const float *src, double *qbar, double *const *grad)
{
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = dalloc(N);
    if (qbar) memset(qbar, 0, sizeof(double) * (size_t)nsrc * nt);
    for (int k = nt - 1; k >= 1; k--) {
        /* Xbar^k = M_k^T Xbar^{k+1}, M_k = step from X^k to X^{k+1} */
        if (grad) {
            double *x0[9], *x1[9];
            for (int c = 0; c < 9; c++) {
                x0[c] = P->store + ((long)k * 9 + c) * N;
                x1[c] = P->store + ((long)(k + 1) * 9 + c) * N;
            }
            el_step_T(P, s, x0, x1, grad);
        } else {
            el_step_T(P, s, NULL, NULL, NULL);
        }
        for (int i = 0; i < nrec; i++)
            for (int c = 0; c < R[i].n; c++) {
                double v = R[i].w[c] * res[(long)i * nt + k];
                s[TXX][R[i].idx[c]] += v;
                s[TYY][R[i].idx[c]] += v;
                s[TZZ][R[i].idx[c]] += v;
            }
        if (qbar)
            for (int j = 0; j < nsrc; j++)
                qbar[(long)j * nt + (k - 1)] = dt * (sample(&S[j], s[TXX]) + sample(&S[j], s[TYY]) + sample(&S[j], s[TZZ]));
    }
    /* the gradient of the very first step (n = 0) needs Xbar^1 -> step 0 */
    if (grad && nt >= 1) {
        double *x0[9], *x1[9];
        for (int c = 0; c < 9; c++) {
            x0[c] = P->store + ((long)0 * 9 + c) * N;
            x1[c] = P->store + ((long)1 * 9 + c) * N;
        }
        el_step_T(P, s, x0, x1, grad);
    }
    for (int c = 0; c < 9; c++) free(s[c]);
    free(S); free(R);
    return OR_OK;
}

int or_el_adjoint(or_prob *P, int nrec, const float *rec, const double *traces,
                  int nsrc, const float *src, double *qbar)
{
    if (P->d.kind != 2) return OR_EINVAL;
    return el_adjoint_core(P, nrec, rec, traces, nsrc, src, qbar, NULL);
}

/* gradient w.r.t. nodal (lam [Pa], mu [Pa], b = 1/rho [m^3/kg]) on the
 * physical grid: grad = [3][nx][ny][nz] */
int or_el_gradient(or_prob *P, int nsrc, const float *src, const float *wav,
                   int nrec, const float *rec, const double *d_obs,
                   double *grad_phys, double *misfit, double *grad_comp)
{
    if (P->d.kind != 2) return OR_EINVAL;
    int nt = P->d.nt;
    double *tr = dalloc((long)nrec * nt);
    int rc = or_el_forward(P, nsrc, src, wav, nrec, rec, tr, 1);
    if (rc) { free(tr); return rc; }
    double J = 0.0;
    for (long i = 0; i < (long)nrec * nt; i++) {
        tr[i] -= d_obs[i];
        J += 0.5 * tr[i] * tr[i];
    }
    if (misfit) *misfit = J;
    double *g[3];
    for (int c = 0; c < 3; c++) g[c] = dalloc(P->N);
    rc = el_adjoint_core(P, nrec, rec, tr, nsrc, src, NULL, g);
    if (!rc) {
        long np = (long)P->d.nx * P->d.ny * P->d.nz;
        for (int c = 0; c < 3; c++) {
            if (grad_comp) memcpy(grad_comp + c * P->N, g[c], sizeof(double) * P->N);
            if (grad_phys) fold(g[c], grad_phys + c * np, P);
        }
    }
    for (int c = 0; c < 3; c++) free(g[c]);
    free(tr);
    free(P->store); P->store = NULL; P->stored = 0;
    return rc;
}

/* One full-grid elastic step (forward, or transpose if adjoint != 0) from a
 * float32 state [9][N]; result (double) [9][N]. */
int or_el_step_state(or_prob *P, const float *in, double *out, int adjoint, int nsteps)
{
    long N = P->N;
    double *s[9];
    for (int c = 0; c < 9; c++) {
        s[c] = out + (long)c * N;
        for (long q = 0; q < N; q++) s[c][q] = (double)in[(long)c * N + q];
    }
    for (int it = 0; it < nsteps; it++) {
        if (!adjoint) el_step(P, s);
        else el_step_T(P, s, NULL, NULL, NULL);
    }
    return OR_OK;
}

/* Same in double precision (energy tests run many steps in FP64) */
int or_el_step_state_d(or_prob *P, double *state, int adjoint, int nsteps)
{
    long N = P->N;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = state + (long)c * N;
    for (int it = 0; it < nsteps; it++) {
        if (!adjoint) el_step(P, s);
        else el_step_T(P, s, NULL, NULL, NULL);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 2D elastic (x-z plane; Sec. IV-A system, 2D example of Sec. IV-B):  */
/* velocities vx, vz and stresses txx, tzz, txz on the staggered grid   */
/* of the 3D system with every y term dropped (ny = 1, no layer in y).  */
/* The state uses the 3D slots VX, VZ, TXX, TZZ, TXZ; the others stay 0. */
/* ------------------------------------------------------------------ */
static void el2_div_tau(const or_prob *P, double *const *s, double *dvx, double *dvz)
{
    long N = P->N;
    double *t = dalloc(N);
    /* x: D+x txx + D-z txz ;  z: D-x txz + D+z tzz */
    apply_axis(line_Dp, s[TXX], dvx, 0, P);
    apply_axis(line_Dm, s[TXZ], t, 2, P); for (long q = 0; q < N; q++) dvx[q] += t[q];
    apply_axis(line_Dm, s[TXZ], dvz, 0, P);
    apply_axis(line_Dp, s[TZZ], t, 2, P); for (long q = 0; q < N; q++) dvz[q] += t[q];
    free(t);
}

/* strain of v: exx = D-x vx, ezz = D-z vz, gxz = D+z vx + D+x vz */
static void el2_strain(const or_prob *P, double *const *s, double *exx, double *ezz, double *gxz)
{
    long N = P->N;
    double *t = dalloc(N);
    apply_axis(line_Dm, s[VX], exx, 0, P);
    apply_axis(line_Dm, s[VZ], ezz, 2, P);
    apply_axis(line_Dp, s[VX], gxz, 2, P);
    apply_axis(line_Dp, s[VZ], t, 0, P); for (long q = 0; q < N; q++) gxz[q] += t[q];
    free(t);
}

/* 2D stiffness: sxx = lam (exx + ezz) + 2 mu exx, szz = lam (exx + ezz) + 2 mu ezz,
 * sxz = mu_avg gxz (mu averaged over the 4 nodes around the x-z edge point) */
static void el2_stiff(const or_prob *P, const double *exx, const double *ezz, const double *gxz,
                      double *sxx, double *szz, double *sxz)
{
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int z = 0; z < P->NZ; z++) {
            long q = IDX(P, x, 0, z);
            double tr = exx[q] + ezz[q];
            sxx[q] = P->lam[q] * tr + 2.0 * P->mu[q] * exx[q];
            szz[q] = P->lam[q] * tr + 2.0 * P->mu[q] * ezz[q];
            sxz[q] = muavg(P, 0, 2, x, 0, z) * gxz[q];
        }
}

/* one forward step in place: v <- g (v + dt b div tau); tau <- g (tau + dt C S(v)) */
static void el2_step(const or_prob *P, double *const *s)
{
    long N = P->N; double dt = P->d.dt;
    double *dvx = dalloc(N), *dvz = dalloc(N), *e[3], *sg[3];
    for (int i = 0; i < 3; i++) { e[i] = dalloc(N); sg[i] = dalloc(N); }
    el2_div_tau(P, s, dvx, dvz);
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int z = 0; z < P->NZ; z++) {
            long q = IDX(P, x, 0, z);
            s[VX][q] = gtaper(P, VX, x, 0, z) * (s[VX][q] + dt * bavg(P, 0, x, 0, z) * dvx[q]);
            s[VZ][q] = gtaper(P, VZ, x, 0, z) * (s[VZ][q] + dt * bavg(P, 2, x, 0, z) * dvz[q]);
        }
    el2_strain(P, s, e[0], e[1], e[2]);
    el2_stiff(P, e[0], e[1], e[2], sg[0], sg[1], sg[2]);
    const int comp[3] = {TXX, TZZ, TXZ};
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int z = 0; z < P->NZ; z++) {
            long q = IDX(P, x, 0, z);
            for (int c = 0; c < 3; c++)
                s[comp[c]][q] = gtaper(P, comp[c], x, 0, z) * (s[comp[c]][q] + dt * sg[c][q]);
        }
    free(dvx); free(dvz);
    for (int i = 0; i < 3; i++) { free(e[i]); free(sg[i]); }
}

/* transpose of el2_step, in place (literal transposes, as el_step_T):
 *   t = g tau' ; vbar = v' + dt S^T (C t) ; tau = t ; s = g vbar ; tau += dt Dtau^T (b s) ; v = s */
static void el2_step_T(const or_prob *P, double *const *s)
{
    long N = P->N; double dt = P->d.dt;
    const int comp[3] = {TXX, TZZ, TXZ};
    double *t[3], *sg[3], *wx = dalloc(N), *wz = dalloc(N);
    for (int i = 0; i < 3; i++) { t[i] = dalloc(N); sg[i] = dalloc(N); }
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int z = 0; z < P->NZ; z++) {
            long q = IDX(P, x, 0, z);
            for (int c = 0; c < 3; c++) t[c][q] = gtaper(P, comp[c], x, 0, z) * s[comp[c]][q];
        }
    el2_stiff(P, t[0], t[1], t[2], sg[0], sg[1], sg[2]);
    /* S^T: exx = D-x vx, ezz = D-z vz, gxz = D+z vx + D+x vz */
    apply_axisT(line_DmT_add, sg[0], s[VX], 0, P, dt);
    apply_axisT(line_DmT_add, sg[1], s[VZ], 2, P, dt);
    apply_axisT(line_DpT_add, sg[2], s[VX], 2, P, dt);
    apply_axisT(line_DpT_add, sg[2], s[VZ], 0, P, dt);
    for (int c = 0; c < 3; c++) memcpy(s[comp[c]], t[c], sizeof(double) * N);
#pragma omp parallel for
    for (int x = 0; x < P->NX; x++)
        for (int z = 0; z < P->NZ; z++) {
            long q = IDX(P, x, 0, z);
            s[VX][q] *= gtaper(P, VX, x, 0, z);
            s[VZ][q] *= gtaper(P, VZ, x, 0, z);
            wx[q] = bavg(P, 0, x, 0, z) * s[VX][q];
            wz[q] = bavg(P, 2, x, 0, z) * s[VZ][q];
        }
    /* Dtau^T: dvx = D+x txx + D-z txz, dvz = D-x txz + D+z tzz */
    apply_axisT(line_DpT_add, wx, s[TXX], 0, P, dt);
    apply_axisT(line_DmT_add, wx, s[TXZ], 2, P, dt);
    apply_axisT(line_DmT_add, wz, s[TXZ], 0, P, dt);
    apply_axisT(line_DpT_add, wz, s[TZZ], 2, P, dt);
    free(wx); free(wz);
    for (int i = 0; i < 3; i++) { free(t[i]); free(sg[i]); }
}

/* forward modelling: record txx + tzz (2D trace of stress) from X^n, step,
 * inject dt q^n into txx and tzz (explosive source). traces [nrec][nt] */
int or_el2_forward(or_prob *P, int nsrc, const float *src, const float *wav,
                   int nrec, const float *rec, double *traces)
{
    if (P->d.kind != 4) return OR_EINVAL;
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = dalloc(N);
    for (int n = 0; n < nt; n++) {
        for (int i = 0; i < nrec; i++)
            traces[(long)i * nt + n] = sample(&R[i], s[TXX]) + sample(&R[i], s[TZZ]);
        el2_step(P, s);
        for (int j = 0; j < nsrc; j++)
            for (int c = 0; c < S[j].n; c++) {
                double v = dt * S[j].w[c] * (double)wav[(long)j * nt + n];
                s[TXX][S[j].idx[c]] += v;
                s[TZZ][S[j].idx[c]] += v;
            }
    }
    for (int c = 0; c < 9; c++) free(s[c]);
    free(S); free(R);
    return OR_OK;
}

/* adjoint: Xbar^{nt} = 0; k = nt-1 .. 1: Xbar^k = M^T Xbar^{k+1} + R^T r^k,
 * qbar^{k-1} = dt P (tbar_xx + tbar_zz)^k */
int or_el2_adjoint(or_prob *P, int nrec, const float *rec, const double *traces,
                   int nsrc, const float *src, double *qbar)
{
    if (P->d.kind != 4) return OR_EINVAL;
    int e1, e2;
    pt8 *S = make_points(P, src, nsrc, &e1), *R = make_points(P, rec, nrec, &e2);
    if (e1 || e2) { free(S); free(R); return OR_EINVAL; }
    long N = P->N; int nt = P->d.nt; double dt = P->d.dt;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = dalloc(N);
    memset(qbar, 0, sizeof(double) * (size_t)nsrc * nt);
    for (int k = nt - 1; k >= 1; k--) {
        el2_step_T(P, s);
        for (int i = 0; i < nrec; i++)
            for (int c = 0; c < R[i].n; c++) {
                double v = R[i].w[c] * traces[(long)i * nt + k];
                s[TXX][R[i].idx[c]] += v;
                s[TZZ][R[i].idx[c]] += v;
            }
        for (int j = 0; j < nsrc; j++)
            qbar[(long)j * nt + (k - 1)] = dt * (sample(&S[j], s[TXX]) + sample(&S[j], s[TZZ]));
    }
    for (int c = 0; c < 9; c++) free(s[c]);
    free(S); free(R);
    return OR_OK;
}

/* nsteps source-free steps (adjoint != 0: transposed steps) of a double
 * state [9][N] in the 3D slot order (only VX, VZ, TXX, TZZ, TXZ are used) */
int or_el2_step_state_d(or_prob *P, double *state, int adjoint, int nsteps)
{
    if (P->d.kind != 4) return OR_EINVAL;
    long N = P->N;
    double *s[9];
    for (int c = 0; c < 9; c++) s[c] = state + (long)c * N;
    for (int it = 0; it < nsteps; it++) {
        if (!adjoint) el2_step(P, s);
        else el2_step_T(P, s);
    }
    return OR_OK;
}

/* TTI in double precision, many steps, no sources (p0,p1,r0,r1 in/out) */
int or_tti_step_state_d(or_prob *P, double *p0, double *p1, double *r0, double *r1, int nsteps)
{
    long N = P->N;
    double *p2 = dalloc(N), *r2 = dalloc(N);
    for (int it = 0; it < nsteps; it++) {
        tti_step(P, p0, p1, r0, r1, p2, r2);
        memcpy(p0, p1, sizeof(double) * N); memcpy(p1, p2, sizeof(double) * N);
        memcpy(r0, r1, sizeof(double) * N); memcpy(r1, r2, sizeof(double) * N);
    }
    free(p2); free(r2);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Elastic at single points (sampled parity at full size)               */
/* ------------------------------------------------------------------ */
typedef struct {
    const or_desc *d; int NX, NY, NZ, M; double b[MAXM + 1];
    const float *vp, *vs, *rho; const float *const *st; or_prob *P;
} ept_ctx;

static double ep_f(const ept_ctx *C, int comp, int x, int y, int z)
{
    if (x < 0 || x >= C->NX || y < 0 || y >= C->NY || z < 0 || z >= C->NZ) return 0.0;
    return (double)C->st[comp][((long)x * C->NY + y) * C->NZ + z];
}
static void ep_par(const ept_ctx *C, int x, int y, int z, double *lam, double *mu, double *bu)
{
    int i = clampi(x - C->d->nbl, 0, C->d->nx - 1);
    int j = clampi(y - C->d->nbl, 0, C->d->ny - 1);
    int k = clampi(z - C->d->nbl, 0, C->d->nz - 1);
    long q = ((long)i * C->d->ny + j) * C->d->nz + k;
    double vp = 1000.0 * C->vp[q], vs = 1000.0 * C->vs[q], rho = 1000.0 * C->rho[q];
    *mu = rho * vs * vs; *lam = rho * (vp * vp - 2.0 * vs * vs); *bu = 1.0 / rho;
}
/* staggered derivatives of state component `comp` at (x,y,z) along ax */
static double ep_Dp(const ept_ctx *C, int comp, int ax, int x, int y, int z)
{
    double acc = 0.0;
    for (int k = 1; k <= C->M; k++) {
        int dp = k, dm = -k + 1;
        acc += C->b[k] * (ep_f(C, comp, x + (ax == 0) * dp, y + (ax == 1) * dp, z + (ax == 2) * dp) -
                          ep_f(C, comp, x + (ax == 0) * dm, y + (ax == 1) * dm, z + (ax == 2) * dm));
    }
    return acc / C->d->h;
}
static double ep_Dm(const ept_ctx *C, int comp, int ax, int x, int y, int z)
{
    double acc = 0.0;
    for (int k = 1; k <= C->M; k++) {
        int dp = k - 1, dm = -k;
        acc += C->b[k] * (ep_f(C, comp, x + (ax == 0) * dp, y + (ax == 1) * dp, z + (ax == 2) * dp) -
                          ep_f(C, comp, x + (ax == 0) * dm, y + (ax == 1) * dm, z + (ax == 2) * dm));
    }
    return acc / C->d->h;
}
/* new velocity component c at (x,y,z), or 0 outside the grid */
static double ep_vnew(const ept_ctx *C, int c, int x, int y, int z)
{
    if (x < 0 || x >= C->NX || y < 0 || y >= C->NY || z < 0 || z >= C->NZ) return 0.0;
    double dv;
    if (c == 0) dv = ep_Dp(C, TXX, 0, x, y, z) + ep_Dm(C, TXY, 1, x, y, z) + ep_Dm(C, TXZ, 2, x, y, z);
    else if (c == 1) dv = ep_Dm(C, TXY, 0, x, y, z) + ep_Dp(C, TYY, 1, x, y, z) + ep_Dm(C, TYZ, 2, x, y, z);
    else dv = ep_Dm(C, TXZ, 0, x, y, z) + ep_Dm(C, TYZ, 1, x, y, z) + ep_Dp(C, TZZ, 2, x, y, z);
    double l0, m0, b0, l1, m1, b1;
    ep_par(C, x, y, z, &l0, &m0, &b0);
    ep_par(C, clampi(x + (c == 0), 0, C->NX - 1), clampi(y + (c == 1), 0, C->NY - 1),
           clampi(z + (c == 2), 0, C->NZ - 1), &l1, &m1, &b1);
    double bb = 0.5 * (b0 + b1);
    return gtaper(C->P, VX + c, x, y, z) * (ep_f(C, VX + c, x, y, z) + C->d->dt * bb * dv);
}
/* derivative of the NEW velocity component c along ax, staggered kind */
static double ep_Dvnew(const ept_ctx *C, int c, int ax, int plus, int x, int y, int z)
{
    double acc = 0.0;
    for (int k = 1; k <= C->M; k++) {
        int dp = plus ? k : k - 1, dm = plus ? -k + 1 : -k;
        acc += C->b[k] * (ep_vnew(C, c, x + (ax == 0) * dp, y + (ax == 1) * dp, z + (ax == 2) * dp) -
                          ep_vnew(C, c, x + (ax == 0) * dm, y + (ax == 1) * dm, z + (ax == 2) * dm));
    }
    return acc / C->d->h;
}

/* one forward elastic step at sampled points: state float32 [9][N]
 * (computational grid), model = physical (vp, vs, rho) float32;
 * out[9*i + c] = component c of the new state at idx[i]. */
int or_el_step_points(const or_desc *d, const float *const *model, const float *const *state,
                      int npts, const long *idx, double *out)
{
    ept_ctx C;
    C.d = d; C.NX = d->nx + 2 * d->nbl; C.NY = d->ny + 2 * d->nbl; C.NZ = d->nz + 2 * d->nbl;
    C.M = d->so / 2;
    double tmp[MAXM];
    if (or_weights_staggered(d->so, tmp)) return OR_EINVAL;
    for (int k = 1; k <= C.M; k++) C.b[k] = tmp[k - 1];
    C.vp = model[0]; C.vs = model[1]; C.rho = model[2]; C.st = state;
    or_prob Pd; memset(&Pd, 0, sizeof(Pd)); Pd.d = *d; Pd.NX = C.NX; Pd.NY = C.NY; Pd.NZ = C.NZ;
    Pd.nby = d->nbl;
    C.P = &Pd;
#pragma omp parallel for
    for (int i = 0; i < npts; i++) {
        long q = idx[i];
        int z = (int)(q % C.NZ), y = (int)((q / C.NZ) % C.NY), x = (int)(q / ((long)C.NZ * C.NY));
        double dt = d->dt;
        for (int c = 0; c < 3; c++) out[9 * i + c] = ep_vnew(&C, c, x, y, z);
        double exx = ep_Dvnew(&C, 0, 0, 0, x, y, z), eyy = ep_Dvnew(&C, 1, 1, 0, x, y, z);
        double ezz = ep_Dvnew(&C, 2, 2, 0, x, y, z);
        double gxy = ep_Dvnew(&C, 0, 1, 1, x, y, z) + ep_Dvnew(&C, 1, 0, 1, x, y, z);
        double gxz = ep_Dvnew(&C, 0, 2, 1, x, y, z) + ep_Dvnew(&C, 2, 0, 1, x, y, z);
        double gyz = ep_Dvnew(&C, 1, 2, 1, x, y, z) + ep_Dvnew(&C, 2, 1, 1, x, y, z);
        double lam, mu, bu;
        ep_par(&C, x, y, z, &lam, &mu, &bu);
        double tr = exx + eyy + ezz, e3[3] = {exx, eyy, ezz};
        for (int c = 0; c < 3; c++)
            out[9 * i + 3 + c] = gtaper(&Pd, TXX + c, x, y, z) *
                                 (ep_f(&C, TXX + c, x, y, z) + dt * (lam * tr + 2.0 * mu * e3[c]));
        int pl[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        double gam[3] = {gxy, gxz, gyz};
        for (int c = 0; c < 3; c++) {
            double ms = 0.0;
            for (int s = 0; s < 2; s++)
                for (int t = 0; t < 2; t++) {
                    int xx = x + (pl[c][0] == 0) * s + (pl[c][1] == 0) * t;
                    int yy = y + (pl[c][0] == 1) * s + (pl[c][1] == 1) * t;
                    int zz = z + (pl[c][0] == 2) * s + (pl[c][1] == 2) * t;
                    double l_, m_, b_;
                    ep_par(&C, clampi(xx, 0, C.NX - 1), clampi(yy, 0, C.NY - 1), clampi(zz, 0, C.NZ - 1), &l_, &m_, &b_);
                    ms += 0.25 * m_;
                }
            out[9 * i + 6 + c] = gtaper(&Pd, TXY + c, x, y, z) * (ep_f(&C, TXY + c, x, y, z) + dt * ms * gam[c]);
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* helpers exposed for pins                                             */
/* ------------------------------------------------------------------ */
int or_line_op(int which, int so, double h, const double *f, double *out, int n)
{
    or_prob P; memset(&P, 0, sizeof(P));
    P.d.h = h; P.d.so = so; P.M = so / 2;
    double tmp[MAXM];
    if (or_weights_centred(so, tmp)) return OR_EINVAL;
    for (int k = 1; k <= P.M; k++) P.c[k] = tmp[k - 1];
    or_weights_staggered(so, tmp);
    for (int k = 1; k <= P.M; k++) P.b[k] = tmp[k - 1];
    memset(out, 0, sizeof(double) * n);
    switch (which) {
    case 0: line_D(f, out, 1, n, &P); break;
    case 1: line_DT_add(f, out, 1, n, &P, 1.0); break;
    case 2: line_Dp(f, out, 1, n, &P); break;
    case 3: line_Dm(f, out, 1, n, &P); break;
    case 4: line_DpT_add(f, out, 1, n, &P, 1.0); break;
    case 5: line_DmT_add(f, out, 1, n, &P, 1.0); break;
    default: return OR_EINVAL;
    }
    return OR_OK;
}

int or_sparse_weights(const or_prob *P, const float *xyz, long *idx, double *w)
{
    return trilinear(P, xyz, idx, w);
}

void or_fold_grad(const or_prob *P, const double *comp, double *phys) { fold(comp, phys, P); }

double or_tti_sigma_at(const or_prob *P, long q)
{
    return P->sig[q];
}
double or_cerjan_at(const or_prob *P, int comp, int x, int y, int z)
{
    return gtaper(P, comp, x, y, z);
}
