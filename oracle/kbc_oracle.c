/*
 * kbc_oracle.c -- plain, slow FP64 CPU oracle of the D2Q9 KBC / LBGK lattice
 * Boltzmann step (Bosch, Chikatamarla, Karlin, "Entropic multi-relaxation
 * models for simulation of fluid turbulence").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU baseline
 * of the benchmark load this library.  It shares no code, header, table or
 * helper with the CUDA library; nothing in the CUDA library includes or
 * calls anything here.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (fused multiply-add
 * contraction is off so that results are the same on x86-64 and aarch64).
 *
 * Layout of every grid array: SoA, x fastest.  Populations g[9][ny][nx] with
 * the index i = 3(b+1) + (a+1) for the velocity v_i = (a, b); scalar fields
 * [ny][nx].  The stored state is the post-collision field f' of Eq. Egeneral;
 * one step pulls f_i(x) = f'_i(x - v_i) (periodic) and collides at x.
 *
 * Functions whose parity is not pinned by a closed form, an invariant or a
 * brute-force check are listed as such in the test suite; every function
 * below has at least one pin there.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D2Q9 (Sec. 2): tensor product of the 1-D set {-1, 0, 1}. */
#define KBCO_VA(i) ((i) % 3 - 1)
#define KBCO_VB(i) ((i) / 3 - 1)
#define KBCO_IDX(a, b) (3 * ((b) + 1) + ((a) + 1))
/* c_s^2 and W_i are not printed in the paper (Eq. S, Eq. Eq); the standard
 * D2Q9 product weights are used: w_0 = 2/3, w_{+-1} = 1/6, W_(a,b) = w_a w_b,
 * c_s^2 = 1/3.  Tests pin them through the equilibrium moments of Eq. Peq
 * and Eq. Qeq, which hold for no other choice. */
#define KBCO_CS2 (1.0 / 3.0)

enum { KBCO_LBGK = 0, KBCO_A = 1, KBCO_B = 2, KBCO_C = 3, KBCO_D = 4 };

static double kbco_w1(int a) { return a == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
static double kbco_W(int i) { return kbco_w1(KBCO_VA(i)) * kbco_w1(KBCO_VB(i)); }

/* Table 1: A and B use central moments, C and D natural ones. */
static int kbco_variant_central(int variant)
{
    return variant == KBCO_A || variant == KBCO_B;
}

/* Table 1: membership of moment j in (T, N, Pi_xy, Q_xyy, Q_yxx, A) in s. */
static int kbco_in_s(int variant, int j)
{
    switch (variant) {
    case KBCO_LBGK: return 1;                 /* everything in s, h empty */
    case KBCO_A: case KBCO_C: return j <= 2;  /* Pi_xy, N, T */
    case KBCO_B: case KBCO_D: return j == 1 || j == 2; /* Pi_xy, N */
    default: return 0;
    }
}

/* ---- real instance ---------------------------------------------------- */
#define R double
#define FN(x) x##_r
#define RE(x) (x)
#define LOG1P(x) log1p(x)
#include "kbc_oracle_core.inc"
#undef R
#undef FN
#undef RE
#undef LOG1P

/* ---- complex instance (complex-step derivatives) ------------------------ */
#define R double complex
#define FN(x) x##_c
#define RE(x) creal(x)
#define LOG1P(x) clog(1.0 + (x))
#include "kbc_oracle_core.inc"
#undef R
#undef FN
#undef RE
#undef LOG1P

static int valid_variant(int v) { return v >= KBCO_LBGK && v <= KBCO_D; }

static size_t wrap(long i, long n) { return (size_t)(((i % n) + n) % n); }

/* ====================================================================== */
/* Per-node batch entry points (arrays of n nodes, 9 values per node, AoS).  */
/* ====================================================================== */

int kbco_version(void) { return 1; }

double kbco_weight(int i) { return (i >= 0 && i < 9) ? kbco_W(i) : NAN; }

void kbco_feq_batch(int n, const double* rho, const double* ux,
                    const double* uy, double* feq)
{
    for (int p = 0; p < n; ++p) feq_r(rho[p], ux[p], uy[p], feq + 9 * p);
}

/* Higher moments (T, N, Pi_xy, Q_xyy, Q_yxx, A) of each node about its own
 * velocity (central = 1) or about zero (central = 0); also rho and u. */
void kbco_moments_batch(int n, int central, const double* f, double* rho,
                        double* ux, double* uy, double* m6)
{
    for (int p = 0; p < n; ++p) {
        double r, x, y;
        conserved_r(f + 9 * p, &r, &x, &y);
        rho[p] = r; ux[p] = x; uy[p] = y;
        moments_r(f + 9 * p, r, central ? x : 0.0, central ? y : 0.0, m6 + 6 * p);
    }
}

/* Eq. cm for a batch (central -> natural). */
void kbco_natural_from_central_batch(int n, const double* ux, const double* uy,
                                     const double* c6, double* n6)
{
    for (int p = 0; p < n; ++p) natural_from_central_r(ux[p], uy[p], c6 + 6 * p, n6 + 6 * p);
}

/* Eq. momentsD2Q9 (central = 0) or its central form (central = 1). */
void kbco_populations_from_moments_batch(int n, int central, const double* rho,
                                         const double* ux, const double* uy,
                                         const double* m6, double* f)
{
    for (int p = 0; p < n; ++p)
        populations_from_moments_r(central, rho[p], ux[p], uy[p], m6 + 6 * p, f + 9 * p);
}

/* k, s, h of f and the deviations ds, dh (Eq. ksh-representation, Table 1). */
int kbco_split_batch(int n, int variant, const double* f, double* feq,
                     double* ds, double* dh, double* k, double* s, double* h)
{
    if (!valid_variant(variant)) return -1;
    for (int p = 0; p < n; ++p) {
        double seq[9], heq[9];
        split_r(variant, f + 9 * p, feq + 9 * p, ds + 9 * p, dh + 9 * p,
                k ? k + 9 * p : NULL, s ? s + 9 * p : NULL,
                h ? h + 9 * p : NULL, seq, heq);
    }
    return 0;
}

/* One collision per node (see collide_r for the meaning of the flags). */
int kbco_collide_batch(int n, int variant, double beta, int gmode, double gfix,
                       int form, const double* f, double* out, double* gamma)
{
    if (!valid_variant(variant) || !(beta > 0.0 && beta <= 1.0)) return -1;
    for (int p = 0; p < n; ++p)
        collide_r(variant, beta, gmode, gfix, form, f + 9 * p, out + 9 * p,
                  gamma ? gamma + p : NULL);
    return 0;
}

/* Complex-step Jacobian of one collision: J[i*9+k] = d f'_i / d f_k and
 * dbeta[i] = d f'_i / d beta, exact to rounding because the collision is a
 * rational function of f and beta (step 1e-30 on the imaginary axis). */
int kbco_collide_jacobian_batch(int n, int variant, double beta, int gmode,
                                double gfix, const double* f, double* J,
                                double* dbeta)
{
    if (!valid_variant(variant) || !(beta > 0.0 && beta <= 1.0) || gmode == 2) return -1;
    const double hs = 1e-30;
    for (int p = 0; p < n; ++p) {
        double complex fc[9], oc[9];
        for (int k = 0; k < 9; ++k) {
            for (int i = 0; i < 9; ++i) fc[i] = f[9 * p + i];
            fc[k] += I * hs;
            collide_c(variant, beta, gmode, gfix, 0, fc, oc, NULL);
            for (int i = 0; i < 9; ++i) J[81 * p + 9 * i + k] = cimag(oc[i]) / hs;
        }
        if (dbeta) {
            for (int i = 0; i < 9; ++i) fc[i] = f[9 * p + i];
            collide_c(variant, beta + I * hs, gmode, gfix, 0, fc, oc, NULL);
            for (int i = 0; i < 9; ++i) dbeta[9 * p + i] = cimag(oc[i]) / hs;
        }
    }
    return 0;
}

/* ====================================================================== */
/* Grid functions.                                                          */
/* ====================================================================== */

/* g = f^eq(rho, u) at every node (the equilibrium initialisation). */
void kbco_init_feq(int nx, int ny, const double* rho, const double* ux,
                   const double* uy, double* g)
{
    const size_t np = (size_t)nx * ny;
    for (size_t x = 0; x < np; ++x) {
        double fe[9];
        feq_r(rho[x], ux[x], uy[x], fe);
        for (int i = 0; i < 9; ++i) g[i * np + x] = fe[i];
    }
}

/*
 * Grad's approximation (Eq. Grad) with Pi = Pi^eq + Pi^(1) (Eq. Peq,
 * Eq. P1AC); the velocity gradients are periodic central differences of the
 * given field, as the paper does for its turbulence runs.
 */
void kbco_init_grad(int nx, int ny, double beta, const double* rho,
                    const double* ux, const double* uy, double* g)
{
    const size_t np = (size_t)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t c = (size_t)y * nx + x;
            const size_t xp = (size_t)y * nx + wrap(x + 1, nx), xm = (size_t)y * nx + wrap(x - 1, nx);
            const size_t yp = wrap(y + 1, ny) * nx + x, ym = wrap(y - 1, ny) * nx + x;
            /* du[a][b] = d u_b / d x_a */
            const double du[2][2] = {
                {0.5 * (ux[xp] - ux[xm]), 0.5 * (uy[xp] - uy[xm])},
                {0.5 * (ux[yp] - ux[ym]), 0.5 * (uy[yp] - uy[ym])}};
            const double r = rho[c], u[2] = {ux[c], uy[c]};
            double Pi[2][2];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    Pi[a][b] = r * KBCO_CS2 * (a == b) + r * u[a] * u[b]
                             - r * KBCO_CS2 / (2.0 * beta) * (du[a][b] + du[b][a]);
            for (int i = 0; i < 9; ++i) {
                const double v[2] = {KBCO_VA(i), KBCO_VB(i)};
                double lin = 0.0, quad = 0.0;
                for (int a = 0; a < 2; ++a) {
                    lin += r * u[a] * v[a] / KBCO_CS2;
                    for (int b = 0; b < 2; ++b)
                        quad += (Pi[a][b] - r * KBCO_CS2 * (a == b)) *
                                (v[a] * v[b] - KBCO_CS2 * (a == b));
                }
                g[i * np + c] = kbco_W(i) * (r + lin + quad / (2.0 * KBCO_CS2 * KBCO_CS2));
            }
        }
}

/* f_i(x) = g_i((x - v_i) mod (nx, ny)): the streaming of Eq. Egeneral. */
static void pull(int nx, int ny, const double* g, int x, int y, double f[9])
{
    const size_t np = (size_t)nx * ny;
    for (int i = 0; i < 9; ++i) {
        const size_t sx = wrap(x - KBCO_VA(i), nx), sy = wrap(y - KBCO_VB(i), ny);
        f[i] = g[i * np + sy * nx + sx];
    }
}

/*
 * nsteps steps of Eq. Egeneral on a doubly periodic nx x ny grid.  g holds
 * the post-collision state and is updated in place (work is scratch of the
 * same size).  gamma_last, if given, receives the gamma of every node in the
 * last step.  nthreads > 1 splits the rows among OpenMP threads; the
 * arithmetic per node does not depend on it.
 */
int kbco_step(int nx, int ny, int variant, double beta, int gmode, double gfix,
              int nsteps, double* g, double* work, double* gamma_last,
              int nthreads)
{
    if (nx < 1 || ny < 1 || !valid_variant(variant) || !(beta > 0.0 && beta <= 1.0))
        return -1;
    const size_t np = (size_t)nx * ny;
    double* src = g;
    double* dst = work;
    if (nthreads < 1) nthreads = 1;
    for (int t = 0; t < nsteps; ++t) {
        const int last = (t == nsteps - 1);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double f[9], out[9], gm;
                pull(nx, ny, src, x, y, f);
                collide_r(variant, beta, gmode, gfix, 0, f, out, &gm);
                const size_t c = (size_t)y * nx + x;
                for (int i = 0; i < 9; ++i) dst[i * np + c] = out[i];
                if (last && gamma_last) gamma_last[c] = gm;
            }
        double* tmp = src; src = dst; dst = tmp;
    }
    if (src != g) memcpy(g, src, 9 * np * sizeof(double));
    return 0;
}

/* rho and u of every node (identical for the pre- and post-collision field,
 * since the collision conserves them). */
void kbco_macro(int nx, int ny, const double* g, double* rho, double* ux,
                double* uy)
{
    const size_t np = (size_t)nx * ny;
    for (size_t c = 0; c < np; ++c) {
        double f[9], r, x, y;
        for (int i = 0; i < 9; ++i) f[i] = g[i * np + c];
        conserved_r(f, &r, &x, &y);
        rho[c] = r; ux[c] = x; uy[c] = y;
    }
}

/* Mean and standard deviation of n values by the plain two-pass definition:
 * the mean first, then the mean of the squared deviations from it. */
static void mean_std(const double* v, size_t n, double* mean, double* std)
{
    double m = 0.0;
    for (size_t c = 0; c < n; ++c) m += v[c];
    m /= (double)n;
    double q = 0.0;
    for (size_t c = 0; c < n; ++c) q += (v[c] - m) * (v[c] - m);
    *mean = m;
    *std = sqrt(q / (double)n);
}

/*
 * Global diagnostics of the field (the quantities plotted in the paper's
 * shear-layer and turbulence sections), in this order:
 *   [0] mass sum rho        [1] sum rho u_x     [2] sum rho u_y
 *   [3] E = mean |u|^2 / 2  [4] Z = mean w^2 / 2 (w = d_x u_y - d_y u_x by
 *       periodic central differences)
 *   [5] mean gamma  [6] min gamma  [7] max gamma  -- of the collision the next
 *       step performs (pulled populations), 2 for LBGK
 *   [8] spatial std of |u|^2/2   [9] spatial std of w^2/2
 */
int kbco_diagnostics(int nx, int ny, int variant, double beta, int gmode,
                     double gfix, const double* g, double* out)
{
    if (nx < 1 || ny < 1 || !valid_variant(variant)) return -1;
    const size_t np = (size_t)nx * ny;
    double* rho = malloc(np * sizeof(double));
    double* ux = malloc(np * sizeof(double));
    double* uy = malloc(np * sizeof(double));
    double* ke = malloc(np * sizeof(double));
    double* zz = malloc(np * sizeof(double));
    if (!rho || !ux || !uy || !ke || !zz) {
        free(rho); free(ux); free(uy); free(ke); free(zz);
        return -2;
    }
    kbco_macro(nx, ny, g, rho, ux, uy);
    double mass = 0, px = 0, py = 0;
    double gsum = 0, gmin = INFINITY, gmax = -INFINITY;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t c = (size_t)y * nx + x;
            mass += rho[c];
            px += rho[c] * ux[c];
            py += rho[c] * uy[c];
            ke[c] = 0.5 * (ux[c] * ux[c] + uy[c] * uy[c]);
            const double w = 0.5 * (uy[(size_t)y * nx + wrap(x + 1, nx)] - uy[(size_t)y * nx + wrap(x - 1, nx)])
                           - 0.5 * (ux[wrap(y + 1, ny) * nx + x] - ux[wrap(y - 1, ny) * nx + x]);
            zz[c] = 0.5 * w * w;
            double f[9], o[9], gm;
            pull(nx, ny, g, x, y, f);
            collide_r(variant, beta, gmode, gfix, 0, f, o, &gm);
            gsum += gm;
            if (gm < gmin) gmin = gm;
            if (gm > gmax) gmax = gm;
        }
    out[0] = mass; out[1] = px; out[2] = py;
    mean_std(ke, np, &out[3], &out[8]);
    mean_std(zz, np, &out[4], &out[9]);
    out[5] = gsum / (double)np; out[6] = gmin; out[7] = gmax;
    free(rho); free(ux); free(uy); free(ke); free(zz);
    return 0;
}

/*
 * Further diagnostics of the paper's turbulence figures, in this order:
 *   [0] palinstrophy P = mean |grad w|^2 / 2, with w = d_x u_y - d_y u_x and
 *       both derivatives by periodic central differences
 *   [1] spatial std of |grad w|^2 / 2
 *   [2] mean entropy density -sum_i f_i ln(f_i / W_i) (Eq. S)
 *   [3] spatial std of the entropy density
 */
int kbco_diagnostics_ext(int nx, int ny, const double* g, double* out)
{
    if (nx < 1 || ny < 1) return -1;
    const size_t np = (size_t)nx * ny;
    double* rho = malloc(np * sizeof(double));
    double* ux = malloc(np * sizeof(double));
    double* uy = malloc(np * sizeof(double));
    double* w = malloc(np * sizeof(double));
    double* pd = malloc(np * sizeof(double));
    double* sd = malloc(np * sizeof(double));
    if (!rho || !ux || !uy || !w || !pd || !sd) {
        free(rho); free(ux); free(uy); free(w); free(pd); free(sd);
        return -2;
    }
    kbco_macro(nx, ny, g, rho, ux, uy);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            w[(size_t)y * nx + x] =
                0.5 * (uy[(size_t)y * nx + wrap(x + 1, nx)] - uy[(size_t)y * nx + wrap(x - 1, nx)])
              - 0.5 * (ux[wrap(y + 1, ny) * nx + x] - ux[wrap(y - 1, ny) * nx + x]);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t c = (size_t)y * nx + x;
            const double wx = 0.5 * (w[(size_t)y * nx + wrap(x + 1, nx)] - w[(size_t)y * nx + wrap(x - 1, nx)]);
            const double wy = 0.5 * (w[wrap(y + 1, ny) * nx + x] - w[wrap(y - 1, ny) * nx + x]);
            pd[c] = 0.5 * (wx * wx + wy * wy);
            double s = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double f = g[i * np + c];
                s -= f * log(f / kbco_W(i));
            }
            sd[c] = s;
        }
    mean_std(pd, np, &out[0], &out[1]);
    mean_std(sd, np, &out[2], &out[3]);
    free(rho); free(ux); free(uy); free(w); free(pd); free(sd);
    return 0;
}

/* ====================================================================== */
/* Adjoint (discrete reverse sweep; complex-step local derivatives).        */
/* ====================================================================== */

/* Objective density at one node of the final state (per node; J = sum):
 *   objective 0: kinetic energy  rho |u|^2 / 2
 *   objective 1: misfit          |u - u_target|^2 / 2                      */
static double complex node_objective_c(int objective, const double complex f[9],
                                       double tx, double ty)
{
    double complex r, x, y;
    conserved_c(f, &r, &x, &y);
    if (objective == 0) return 0.5 * r * (x * x + y * y);
    return 0.5 * ((x - tx) * (x - tx) + (y - ty) * (y - ty));
}

/*
 * Discrete adjoint of J(g^N) for g^0 = f^eq(rho0, u0), g^{n+1} = C(P g^n):
 *   lambda^N = dJ/dg^N,
 *   lambda^n = P^T (dC/df |_{P g^n})^T lambda^{n+1},
 *   dJ/dbeta = sum_n sum_x lambda^{n+1} . dC/dbeta,
 *   dJ/du0   = (df^eq/du)^T lambda^0.
 * Every local derivative is a complex step of the real arithmetic above.
 * All N+1 states are stored (meant for small grids).
 */
int kbco_adjoint(int nx, int ny, int variant, double beta, int gmode, double gfix,
                 const double* rho0, const double* ux0, const double* uy0,
                 int nsteps, int objective, const double* utx, const double* uty,
                 double* J, double* gux, double* guy, double* gbeta)
{
    if (nx < 1 || ny < 1 || nsteps < 0 || !valid_variant(variant) ||
        !(beta > 0.0 && beta <= 1.0) || (objective != 0 && objective != 1) || gmode == 2)
        return -1;
    const size_t np = (size_t)nx * ny, fs = 9 * np;
    double* states = malloc((size_t)(nsteps + 1) * fs * sizeof(double));
    double* lam = malloc(fs * sizeof(double));
    double* lam2 = malloc(fs * sizeof(double));
    if (!states || !lam || !lam2) { free(states); free(lam); free(lam2); return -2; }
    kbco_init_feq(nx, ny, rho0, ux0, uy0, states);
    for (int n = 0; n < nsteps; ++n) {
        memcpy(states + (size_t)(n + 1) * fs, states + (size_t)n * fs, fs * sizeof(double));
        double* tmp = malloc(fs * sizeof(double));
        if (!tmp) { free(states); free(lam); free(lam2); return -2; }
        kbco_step(nx, ny, variant, beta, gmode, gfix, 1, states + (size_t)(n + 1) * fs, tmp, NULL, 1);
        free(tmp);
    }
    /* J and lambda^N */
    const double hs = 1e-30;
    const double* gN = states + (size_t)nsteps * fs;
    double jsum = 0.0;
    for (size_t c = 0; c < np; ++c) {
        double complex f[9];
        const double tx = objective == 1 ? utx[c] : 0.0, ty = objective == 1 ? uty[c] : 0.0;
        for (int i = 0; i < 9; ++i) f[i] = gN[i * np + c];
        jsum += creal(node_objective_c(objective, f, tx, ty));
        for (int k = 0; k < 9; ++k) {
            for (int i = 0; i < 9; ++i) f[i] = gN[i * np + c];
            f[k] += I * hs;
            lam[k * np + c] = cimag(node_objective_c(objective, f, tx, ty)) / hs;
        }
    }
    *J = jsum;
    double gb = 0.0;
    for (int n = nsteps - 1; n >= 0; --n) {
        const double* gn = states + (size_t)n * fs;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t c = (size_t)y * nx + x;
                double f[9], Jc[81], db[9], mu[9];
                pull(nx, ny, gn, x, y, f);
                kbco_collide_jacobian_batch(1, variant, beta, gmode, gfix, f, Jc, db);
                for (int k = 0; k < 9; ++k) {
                    double acc = 0.0;
                    for (int i = 0; i < 9; ++i) acc += Jc[9 * i + k] * lam[i * np + c];
                    mu[k] = acc;
                }
                for (int i = 0; i < 9; ++i) gb += db[i] * lam[i * np + c];
                /* transpose of the pull: the population pulled from x - v_i
                 * sends its adjoint back there */
                for (int i = 0; i < 9; ++i) {
                    const size_t sx = wrap(x - KBCO_VA(i), nx), sy = wrap(y - KBCO_VB(i), ny);
                    lam2[i * np + sy * nx + sx] = mu[i];
                }
            }
        double* t = lam; lam = lam2; lam2 = t;
    }
    for (size_t c = 0; c < np; ++c) {
        double complex fe[9];
        double ax = 0.0, ay = 0.0;
        feq_c(rho0[c], ux0[c] + I * hs, uy0[c], fe);
        for (int i = 0; i < 9; ++i) ax += cimag(fe[i]) / hs * lam[i * np + c];
        feq_c(rho0[c], ux0[c], uy0[c] + I * hs, fe);
        for (int i = 0; i < 9; ++i) ay += cimag(fe[i]) / hs * lam[i * np + c];
        gux[c] = ax; guy[c] = ay;
    }
    *gbeta = gb;
    free(states); free(lam); free(lam2);
    return 0;
}
