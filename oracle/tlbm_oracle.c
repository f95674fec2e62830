/*
 * FP64 CPU oracle for the double-distribution (DDF) thermal lattice Boltzmann
 * time step of Xu & Li, "Multi-GPU thermal lattice Boltzmann simulations using
 * OpenACC and MPI" (IJHMT 2022).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, by the smoke check and by
 * the benchmark's timed CPU baseline.  The CUDA library never links or calls it,
 * and the two share no code, header, table or generator.
 *
 * Written to be read against the paper, not to be fast:
 *   - moment matrices are built from their defining polynomials evaluated on
 *     the velocity set, and inverted by Gauss-Jordan elimination;
 *   - collision is the literal dense form of Eq. (10a) / Eq. (11a);
 *   - streaming is Eq. (10b) / Eq. (11b) written as a pull, with the half-way
 *     bounce-back and anti-bounce-back rules of §2.2 where the source node lies
 *     outside the cell.
 * Build flags: -O2 -ffp-contract=off (no fused multiply-add anywhere).
 *
 * Readings of points where the paper is silent (each one is pinned by a test):
 *   - velocity ordering of D2Q9 follows the halo sets of §3.1 (f_{2,5,6} move
 *     up, f_{4,7,8} move down); D3Q19 uses rest, +-x, +-y, +-z, then the edges;
 *   - the last entry of the printed D2Q9 forcing vector, Eq. (6a), is read as
 *     u F_y + v F_x (the printed u F_x + v F_y is a typo; M*Ftilde gives the
 *     former and agrees with the D3Q19 entries of Eq. (6b));
 *   - parameter mapping from Eqs. (2)-(4): Delta_T = 1, T0 = 0, H = cell height
 *     in lattice units, U = Ma*c_s, nu = U H sqrt(Pr/Ra), alpha = U H/sqrt(Pr Ra),
 *     g*beta = U^2/H;
 *   - flow rates: s_nu = 1/(3 nu + 1/2) on every even non-conserved moment,
 *     s_q = 8(2 - s_nu)/(8 - s_nu) on every odd non-conserved moment (two-
 *     relaxation-time magic parameter 3/16); conserved rates 1;
 *   - thermal: a_T = -2/3 (D2Q5) or -3/4 (D3Q7); flux-moment rate q_j from
 *     alpha = c_sT^2 (1/q_j - 1/2) with c_sT^2 = omega; even rates from
 *     (1/q_j - 1/2)(1/q_e - 1/2) = 1/4;
 *   - walls sit half-way outside the first and last node; Rayleigh-Benard cell:
 *     hot bottom, cold top, adiabatic sides; side-heated cell (§2.3): hot left,
 *     cold right, adiabatic top/bottom (and front/back);
 *   - Nusselt number (not defined by the paper): 1 + L <u_h T> / (alpha dT),
 *     u_h the velocity along the heat-flux axis and L the cell extent on it.
 */
#include "tlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 19

typedef struct {
    int q;
    int e[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
    double M[QMAX][QMAX];
    double Minv[QMAX][QMAX];
} vset;

struct tlbmo_sim {
    int nx, ny, nz, dim, lattice;
    long N;
    double Ra, Pr, Ma;
    tlbmo_params p;
    double U, H, nu, alpha, gbeta, a_T, omega;
    double S[QMAX], Q[QMAX];
    vset fs, gs;
    double *f, *g, *fp, *gp; /* pre-collision state and post-collision scratch */
    int64_t t;
};

/* ------------------------------------------------------------------------- */
/* Velocity sets (Fig. 1)                                                     */
/* ------------------------------------------------------------------------- */

/* D2Q9 ordering fixed by the halo description of §3.1. */
static const int E_D2Q9[9][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0}};
static const int E_D2Q5[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};
static const int E_D3Q19[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int E_D3Q7[7][3] = {{0, 0, 0}, {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},
                                 {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

/* Rows of the moment matrices as polynomials in the lattice velocity.
 * D2Q9: Lallemand & Luo (2000) basis (rho, e, eps, jx, qx, jy, qy, pxx, pxy). */
static double row_d2q9(int k, int ex, int ey) {
    double e2 = ex * ex + ey * ey;
    switch (k) {
    case 0: return 1.0;
    case 1: return 3.0 * e2 - 4.0;
    case 2: return (9.0 * e2 * e2 - 21.0 * e2) / 2.0 + 4.0;
    case 3: return ex;
    case 4: return (3.0 * e2 - 5.0) * ex;
    case 5: return ey;
    case 6: return (3.0 * e2 - 5.0) * ey;
    case 7: return (double)(ex * ex - ey * ey);
    default: return (double)(ex * ey);
    }
}

/* D3Q19: d'Humieres et al. (2002) basis (rho, e, eps, jx, qx, jy, qy, jz, qz,
 * 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz). */
static double row_d3q19(int k, int ex, int ey, int ez) {
    double e2 = ex * ex + ey * ey + ez * ez;
    double xx = ex * ex, yy = ey * ey, zz = ez * ez;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * e2 - 30.0;
    case 2: return (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
    case 3: return ex;
    case 4: return (5.0 * e2 - 9.0) * ex;
    case 5: return ey;
    case 6: return (5.0 * e2 - 9.0) * ey;
    case 7: return ez;
    case 8: return (5.0 * e2 - 9.0) * ez;
    case 9: return 3.0 * xx - e2;
    case 10: return (3.0 * e2 - 5.0) * (3.0 * xx - e2);
    case 11: return yy - zz;
    case 12: return (3.0 * e2 - 5.0) * (yy - zz);
    case 13: return (double)(ex * ey);
    case 14: return (double)(ey * ez);
    case 15: return (double)(ex * ez);
    case 16: return (yy - zz) * ex;
    case 17: return (zz - xx) * ey;
    default: return (xx - yy) * ez;
    }
}

/* D2Q5 thermal basis: 1, ex, ey, 5|e|^2 - 4, ex^2 - ey^2. */
static double row_d2q5(int k, int ex, int ey) {
    double e2 = ex * ex + ey * ey;
    switch (k) {
    case 0: return 1.0;
    case 1: return ex;
    case 2: return ey;
    case 3: return 5.0 * e2 - 4.0;
    default: return (double)(ex * ex - ey * ey);
    }
}

/* D3Q7 thermal basis: 1, ex, ey, ez, 7|e|^2 - 6, 3ex^2 - |e|^2, ey^2 - ez^2. */
static double row_d3q7(int k, int ex, int ey, int ez) {
    double e2 = ex * ex + ey * ey + ez * ez;
    switch (k) {
    case 0: return 1.0;
    case 1: return ex;
    case 2: return ey;
    case 3: return ez;
    case 4: return 7.0 * e2 - 6.0;
    case 5: return 3.0 * ex * ex - e2;
    default: return (double)(ey * ey - ez * ez);
    }
}

/* Plain Gauss-Jordan inverse with partial pivoting. Returns 0 on success. */
static int invert(int n, double A[QMAX][QMAX], double Ainv[QMAX][QMAX]) {
    double a[QMAX][2 * QMAX];
    for (int r = 0; r < n; r++)
        for (int c = 0; c < 2 * n; c++)
            a[r][c] = c < n ? A[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (a[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int k = 0; k < 2 * n; k++) {
                double t = a[c][k];
                a[c][k] = a[piv][k];
                a[piv][k] = t;
            }
        double d = a[c][c];
        for (int k = 0; k < 2 * n; k++) a[c][k] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double m = a[r][c];
            if (m == 0.0) continue;
            for (int k = 0; k < 2 * n; k++) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) Ainv[r][c] = a[r][n + c];
    return 0;
}

static void build_vset(int which, vset* v) {
    memset(v, 0, sizeof(*v));
    const int(*E)[3];
    switch (which) {
    case 0: v->q = 9; E = E_D2Q9; break;
    case 1: v->q = 5; E = E_D2Q5; break;
    case 2: v->q = 19; E = E_D3Q19; break;
    default: v->q = 7; E = E_D3Q7; break;
    }
    for (int i = 0; i < v->q; i++)
        for (int a = 0; a < 3; a++) v->e[i][a] = E[i][a];
    for (int i = 0; i < v->q; i++) {
        int e2 = v->e[i][0] * v->e[i][0] + v->e[i][1] * v->e[i][1] + v->e[i][2] * v->e[i][2];
        if (which == 0) v->w[i] = e2 == 0 ? 4.0 / 9.0 : (e2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else if (which == 2) v->w[i] = e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        else v->w[i] = 0.0; /* thermal weights follow from a_T, see thermal_geq */
        for (int j = 0; j < v->q; j++)
            if (v->e[j][0] == -v->e[i][0] && v->e[j][1] == -v->e[i][1] &&
                v->e[j][2] == -v->e[i][2])
                v->opp[i] = j;
    }
    for (int k = 0; k < v->q; k++)
        for (int i = 0; i < v->q; i++) {
            int ex = v->e[i][0], ey = v->e[i][1], ez = v->e[i][2];
            double m;
            switch (which) {
            case 0: m = row_d2q9(k, ex, ey); break;
            case 1: m = row_d2q5(k, ex, ey); break;
            case 2: m = row_d3q19(k, ex, ey, ez); break;
            default: m = row_d3q7(k, ex, ey, ez); break;
            }
            v->M[k][i] = m;
        }
    invert(v->q, v->M, v->Minv);
}

/* ------------------------------------------------------------------------- */
/* Equilibria and forcing                                                    */
/* ------------------------------------------------------------------------- */

/* Second-order flow equilibrium, c_s^2 = 1/3. */
static void flow_feq(const vset* v, double rho, const double* u, double* feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < v->q; i++) {
        double eu = v->e[i][0] * u[0] + v->e[i][1] * u[1] + v->e[i][2] * u[2];
        feq[i] = v->w[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Guo et al. (2002) discrete force, Ftilde_i = w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)].
 * The paper gives M*Ftilde in closed form in Eq. (6); the tests check that
 * this product reproduces it. */
static void guo_force(const vset* v, const double* u, const double* F, double* Ft) {
    for (int i = 0; i < v->q; i++) {
        double eu = v->e[i][0] * u[0] + v->e[i][1] * u[1] + v->e[i][2] * u[2];
        double eF = v->e[i][0] * F[0] + v->e[i][1] * F[1] + v->e[i][2] * F[2];
        double emuF = (v->e[i][0] - u[0]) * F[0] + (v->e[i][1] - u[1]) * F[1] +
                      (v->e[i][2] - u[2]) * F[2];
        Ft[i] = v->w[i] * (3.0 * emuF + 9.0 * eu * eF);
    }
}

static void matvec(int q, const double A[QMAX][QMAX], const double* x, double* y) {
    for (int k = 0; k < q; k++) {
        double s = 0.0;
        for (int i = 0; i < q; i++) s += A[k][i] * x[i];
        y[k] = s;
    }
}

/* Thermal equilibrium moments n_eq = [T, uT, vT, (wT), a_T T, 0, (0)]. */
static void thermal_neq(int dim, double a_T, double T, const double* u, double* neq) {
    if (dim == 2) {
        neq[0] = T; neq[1] = u[0] * T; neq[2] = u[1] * T; neq[3] = a_T * T; neq[4] = 0.0;
    } else {
        neq[0] = T; neq[1] = u[0] * T; neq[2] = u[1] * T; neq[3] = u[2] * T;
        neq[4] = a_T * T; neq[5] = 0.0; neq[6] = 0.0;
    }
}

/* g_eq = N^-1 n_eq. */
static void thermal_geq(const vset* v, int dim, double a_T, double T, const double* u,
                        double* geq) {
    double neq[QMAX];
    thermal_neq(dim, a_T, T, u, neq);
    for (int i = 0; i < v->q; i++) {
        double a = 0.0;
        for (int k = 0; k < v->q; k++) a += v->Minv[i][k] * neq[k];
        geq[i] = a;
    }
}

/* ------------------------------------------------------------------------- */
/* Parameters                                                                 */
/* ------------------------------------------------------------------------- */

void tlbmo_default_params(tlbmo_params* p) {
    memset(p, 0, sizeof(*p));
    p->walls = TLBMO_RB;
    p->a_T = p->nu = p->alpha = p->gbeta = NAN;
    p->s_rho = p->s_e = p->s_eps = p->s_j = p->s_q = p->s_pi = p->s_m = NAN;
    p->q_e = p->q_v = NAN;
    p->Th = p->Tc = NAN;
}

static double dflt(double v, double d) { return isnan(v) ? d : v; }

tlbmo_sim* tlbmo_create(int nx, int ny, int nz, int lattice, double Ra, double Pr, double Ma,
                        const tlbmo_params* pin) {
    if (lattice != TLBMO_D2Q9_D2Q5 && lattice != TLBMO_D3Q19_D3Q7) return NULL;
    int dim = lattice == TLBMO_D2Q9_D2Q5 ? 2 : 3;
    if (dim == 2) nz = 1;
    if (nx < 3 || ny < 3 || (dim == 3 && nz < 3)) return NULL;
    if (!(Ra > 0.0) || !(Pr > 0.0) || !(Ma > 0.0)) return NULL;
    tlbmo_sim* s = (tlbmo_sim*)calloc(1, sizeof(tlbmo_sim));
    if (!s) return NULL;
    if (pin) s->p = *pin;
    else tlbmo_default_params(&s->p);
    s->nx = nx; s->ny = ny; s->nz = nz; s->dim = dim; s->lattice = lattice;
    s->N = (long)nx * ny * nz;
    s->Ra = Ra; s->Pr = Pr; s->Ma = Ma;
    build_vset(dim == 2 ? 0 : 2, &s->fs);
    build_vset(dim == 2 ? 1 : 3, &s->gs);

    /* Eqs. (2)-(4): free-fall scaling, Delta_T = 1, H = cell height. */
    s->p.Th = dflt(s->p.Th, 0.5);
    s->p.Tc = dflt(s->p.Tc, -0.5);
    double dT = s->p.Th - s->p.Tc;
    s->U = s->p.u_is_ma ? Ma : Ma / sqrt(3.0);
    s->H = dim == 2 ? ny : nz;
    s->nu = dflt(s->p.nu, s->U * s->H * sqrt(Pr / Ra));
    s->alpha = dflt(s->p.alpha, s->U * s->H / sqrt(Pr * Ra));
    s->gbeta = dflt(s->p.gbeta, s->U * s->U / (s->H * dT));
    s->a_T = dflt(s->p.a_T, dim == 2 ? -2.0 / 3.0 : -0.75);
    /* §2.2: omega = (4 + a_T)/10 (D2Q5), (6 + a_T)/21 (D3Q7). */
    s->omega = dim == 2 ? (4.0 + s->a_T) / 10.0 : (6.0 + s->a_T) / 21.0;
    if (!(3.0 * s->nu > 1e-6) || !(s->alpha > 0.0) || !(s->omega > 0.0)) {
        free(s);
        return NULL;
    }

    double snu = 1.0 / (3.0 * s->nu + 0.5);
    double sq = 8.0 * (2.0 - snu) / (8.0 - snu);
    double s_rho = dflt(s->p.s_rho, 1.0), s_e = dflt(s->p.s_e, snu);
    double s_eps = dflt(s->p.s_eps, snu), s_j = dflt(s->p.s_j, 1.0);
    double s_q = dflt(s->p.s_q, sq), s_pi = dflt(s->p.s_pi, snu), s_m = dflt(s->p.s_m, sq);
    if (dim == 2) {
        double S[9] = {s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, snu, snu};
        memcpy(s->S, S, sizeof(S));
    } else {
        double S[19] = {s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_j, s_q, snu,
                        s_pi,  snu, s_pi,  snu, snu, snu, s_m, s_m, s_m};
        memcpy(s->S, S, sizeof(S));
    }
    /* alpha = c_sT^2 (1/q_j - 1/2), with c_sT^2 = omega for these bases. */
    double qj = 1.0 / (s->alpha / s->omega + 0.5);
    double qeven = 1.0 / (0.5 + 0.25 / (1.0 / qj - 0.5));
    double q_e = dflt(s->p.q_e, qeven), q_v = dflt(s->p.q_v, qeven);
    if (dim == 2) {
        double Q[5] = {1.0, qj, qj, q_e, q_v};
        memcpy(s->Q, Q, sizeof(Q));
    } else {
        double Q[7] = {1.0, qj, qj, qj, q_e, q_v, q_v};
        memcpy(s->Q, Q, sizeof(Q));
    }

    size_t nf = (size_t)s->fs.q * s->N, ng = (size_t)s->gs.q * s->N;
    s->f = (double*)calloc(nf, sizeof(double));
    s->fp = (double*)calloc(nf, sizeof(double));
    s->g = (double*)calloc(ng, sizeof(double));
    s->gp = (double*)calloc(ng, sizeof(double));
    if (!s->f || !s->fp || !s->g || !s->gp) {
        tlbmo_destroy(s);
        return NULL;
    }
    return s;
}

void tlbmo_destroy(tlbmo_sim* s) {
    if (!s) return;
    free(s->f); free(s->fp); free(s->g); free(s->gp);
    free(s);
}

int tlbmo_derived(const tlbmo_sim* s, double* out, int cap) {
    double v[7 + 2 * QMAX];
    int n = 0;
    v[n++] = s->U; v[n++] = s->H; v[n++] = s->nu; v[n++] = s->alpha;
    v[n++] = s->gbeta; v[n++] = s->a_T; v[n++] = s->omega;
    for (int k = 0; k < s->fs.q; k++) v[n++] = s->S[k];
    for (int k = 0; k < s->gs.q; k++) v[n++] = s->Q[k];
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

int64_t tlbmo_time(const tlbmo_sim* s) { return s->t; }

/* ------------------------------------------------------------------------- */
/* Initial state                                                              */
/* ------------------------------------------------------------------------- */

/* splitmix64 output function (Steele, Lea & Flood 2014). */
static uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double tlbmo_uniform(uint64_t seed, uint64_t idx) {
    return (double)(splitmix64(seed ^ splitmix64(idx)) >> 11) * 0x1.0p-53;
}

/* Initial state: fluid at rest, f = f_eq(1, 0); conductive temperature profile
 * between the isothermal walls plus uniform noise amp*(2r - 1); g = g_eq(T, 0). */
void tlbmo_init(tlbmo_sim* s, uint64_t seed, double amp) {
    int heat_axis = s->p.walls == TLBMO_RB ? (s->dim == 2 ? 1 : 2) : 0;
    int L = heat_axis == 0 ? s->nx : (heat_axis == 1 ? s->ny : s->nz);
    const double zero[3] = {0.0, 0.0, 0.0};
    double feq[QMAX], geq[QMAX];
    flow_feq(&s->fs, 1.0, zero, feq);
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long n = x + (long)s->nx * (y + (long)s->ny * z);
                int c = heat_axis == 0 ? x : (heat_axis == 1 ? y : z);
                double r = tlbmo_uniform(seed, (uint64_t)n);
                double T = s->p.Th + (s->p.Tc - s->p.Th) * ((c + 0.5) / L);
                T = T + amp * (2.0 * r - 1.0);
                thermal_geq(&s->gs, s->dim, s->a_T, T, zero, geq);
                for (int i = 0; i < s->fs.q; i++) s->f[i * s->N + n] = feq[i];
                for (int i = 0; i < s->gs.q; i++) s->g[i * s->N + n] = geq[i];
            }
    s->t = 0;
}

void tlbmo_get_populations(const tlbmo_sim* s, double* f, double* g) {
    if (f) memcpy(f, s->f, sizeof(double) * s->fs.q * s->N);
    if (g) memcpy(g, s->g, sizeof(double) * s->gs.q * s->N);
}

void tlbmo_set_populations(tlbmo_sim* s, const double* f, const double* g) {
    if (f) memcpy(s->f, f, sizeof(double) * s->fs.q * s->N);
    if (g) memcpy(s->g, g, sizeof(double) * s->gs.q * s->N);
}

/* ------------------------------------------------------------------------- */
/* Macroscopic quantities (§2.2)                                              */
/* ------------------------------------------------------------------------- */

/* rho = sum f, T = sum g, F = rho g beta (T - T0) ghat + rho a,
 * u = (sum e f + F/2)/rho. */
static void node_macros(const tlbmo_sim* s, const double* f, const double* g, double* rho,
                        double* u, double* T, double* F) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0}, t = 0.0;
    for (int i = 0; i < s->fs.q; i++) {
        r += f[i];
        for (int a = 0; a < 3; a++) m[a] += s->fs.e[i][a] * f[i];
    }
    for (int i = 0; i < s->gs.q; i++) t += g[i];
    int gax = s->dim == 2 ? 1 : 2;
    for (int a = 0; a < 3; a++) F[a] = r * s->p.body_force[a];
    F[gax] += r * s->gbeta * (t - 0.0);
    for (int a = 0; a < 3; a++) u[a] = (m[a] + 0.5 * F[a]) / r;
    *rho = r;
    *T = t;
}

/* ------------------------------------------------------------------------- */
/* Collision, Eq. (10a) and Eq. (11a)                                         */
/* ------------------------------------------------------------------------- */

static void collide(const tlbmo_sim* s, const double* f, const double* g, double* fpost,
                    double* gpost) {
    const vset* fs = &s->fs;
    const vset* gs = &s->gs;
    double rho, u[3], T, F[3];
    node_macros(s, f, g, &rho, u, &T, F);

    double m[QMAX], feq[QMAX], meq[QMAX], Ft[QMAX], MF[QMAX];
    matvec(fs->q, fs->M, f, m);
    flow_feq(fs, rho, u, feq);
    matvec(fs->q, fs->M, feq, meq);
    guo_force(fs, u, F, Ft);
    matvec(fs->q, fs->M, Ft, MF);
    /* f+ = f - M^-1 S (m - m_eq) + M^-1 (I - S/2) M Ftilde */
    double dm[QMAX], src[QMAX];
    for (int k = 0; k < fs->q; k++) {
        dm[k] = s->S[k] * (m[k] - meq[k]);
        src[k] = (1.0 - 0.5 * s->S[k]) * MF[k];
    }
    for (int i = 0; i < fs->q; i++) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < fs->q; k++) {
            a += fs->Minv[i][k] * dm[k];
            b += fs->Minv[i][k] * src[k];
        }
        fpost[i] = f[i] - a + b;
    }

    /* g+ = g - N^-1 Q (n - n_eq) */
    double n[QMAX], neq[QMAX], dn[QMAX];
    matvec(gs->q, gs->M, g, n);
    thermal_neq(s->dim, s->a_T, T, u, neq);
    for (int k = 0; k < gs->q; k++) dn[k] = s->Q[k] * (n[k] - neq[k]);
    for (int i = 0; i < gs->q; i++) {
        double a = 0.0;
        for (int k = 0; k < gs->q; k++) a += gs->Minv[i][k] * dn[k];
        gpost[i] = g[i] - a;
    }
}

void tlbmo_collide_node(const tlbmo_sim* s, const double* f, const double* g, double* fpost,
                        double* gpost) {
    collide(s, f, g, fpost, gpost);
}

/* ------------------------------------------------------------------------- */
/* Streaming with wall rules, Eq. (10b) and Eq. (11b)                         */
/* ------------------------------------------------------------------------- */

/* Temperature of the wall crossed on axis `ax` at side `hi` (0 low, 1 high);
 * returns 1 for an isothermal wall, 0 for an adiabatic one. */
static int wall_temperature(const tlbmo_sim* s, int ax, int hi, double* Tw) {
    int heat_axis = s->p.walls == TLBMO_RB ? (s->dim == 2 ? 1 : 2) : 0;
    if (ax != heat_axis) return 0;
    *Tw = hi ? s->p.Tc : s->p.Th;
    return 1;
}

static void stream(tlbmo_sim* s) {
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const long N = s->N;
    const int dims[3] = {nx, ny, nz};
    long zy;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (zy = 0; zy < (long)nz * ny; zy++) {
        int z = (int)(zy / ny), y = (int)(zy % ny);
        for (int x = 0; x < nx; x++) {
            const int c[3] = {x, y, z};
            long n = x + (long)nx * (y + (long)ny * z);
            /* flow populations: pull from x - e_i, half-way bounce-back otherwise */
            for (int i = 0; i < s->fs.q; i++) {
                int src[3], inside = 1;
                for (int a = 0; a < 3; a++) {
                    src[a] = c[a] - s->fs.e[i][a];
                    if (src[a] < 0 || src[a] >= dims[a]) {
                        if (s->p.periodic_mask & (1 << a)) src[a] = (src[a] + dims[a]) % dims[a];
                        else inside = 0;
                    }
                }
                if (inside) {
                    long sn = src[0] + (long)nx * (src[1] + (long)ny * src[2]);
                    s->f[i * N + n] = s->fp[i * N + sn];
                } else {
                    s->f[i * N + n] = s->fp[s->fs.opp[i] * N + n];
                }
            }
            /* temperature populations: anti-bounce-back on isothermal walls,
             * bounce-back on adiabatic walls */
            for (int i = 0; i < s->gs.q; i++) {
                int src[3], inside = 1, wall_ax = -1, wall_hi = 0;
                for (int a = 0; a < 3; a++) {
                    src[a] = c[a] - s->gs.e[i][a];
                    if (src[a] < 0 || src[a] >= dims[a]) {
                        if (s->p.periodic_mask & (1 << a)) src[a] = (src[a] + dims[a]) % dims[a];
                        else {
                            inside = 0;
                            wall_ax = a;
                            wall_hi = src[a] >= dims[a];
                        }
                    }
                }
                if (inside) {
                    long sn = src[0] + (long)nx * (src[1] + (long)ny * src[2]);
                    s->g[i * N + n] = s->gp[i * N + sn];
                } else {
                    double Tw;
                    double gb = s->gp[s->gs.opp[i] * N + n];
                    if (wall_temperature(s, wall_ax, wall_hi, &Tw))
                        s->g[i * N + n] = -gb + s->omega * Tw;
                    else
                        s->g[i * N + n] = gb;
                }
            }
        }
    }
}

void tlbmo_step(tlbmo_sim* s, int64_t nsteps) {
    const long N = s->N;
    const int qf = s->fs.q, qg = s->gs.q;
    for (int64_t t = 0; t < nsteps; t++) {
        long n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (n = 0; n < N; n++) {
            double f[QMAX], g[QMAX], fo[QMAX], go[QMAX];
            for (int i = 0; i < qf; i++) f[i] = s->f[i * N + n];
            for (int i = 0; i < qg; i++) g[i] = s->g[i * N + n];
            collide(s, f, g, fo, go);
            for (int i = 0; i < qf; i++) s->fp[i * N + n] = fo[i];
            for (int i = 0; i < qg; i++) s->gp[i * N + n] = go[i];
        }
        stream(s);
        s->t++;
    }
}

/* ------------------------------------------------------------------------- */
/* Diagnostics                                                                */
/* ------------------------------------------------------------------------- */

void tlbmo_macros(const tlbmo_sim* s, double* rho, double* ux, double* uy, double* uz,
                  double* T) {
    for (long n = 0; n < s->N; n++) {
        double f[QMAX], g[QMAX], r, u[3], t, F[3];
        for (int i = 0; i < s->fs.q; i++) f[i] = s->f[i * s->N + n];
        for (int i = 0; i < s->gs.q; i++) g[i] = s->g[i * s->N + n];
        node_macros(s, f, g, &r, u, &t, F);
        if (rho) rho[n] = r;
        if (ux) ux[n] = u[0];
        if (uy) uy[n] = u[1];
        if (uz) uz[n] = u[2];
        if (T) T[n] = t;
    }
}

double tlbmo_nusselt(const tlbmo_sim* s) {
    int heat_axis = s->p.walls == TLBMO_RB ? (s->dim == 2 ? 1 : 2) : 0;
    double L = heat_axis == 0 ? s->nx : (heat_axis == 1 ? s->ny : s->nz);
    double sum = 0.0;
    for (long n = 0; n < s->N; n++) {
        double f[QMAX], g[QMAX], r, u[3], t, F[3];
        for (int i = 0; i < s->fs.q; i++) f[i] = s->f[i * s->N + n];
        for (int i = 0; i < s->gs.q; i++) g[i] = s->g[i * s->N + n];
        node_macros(s, f, g, &r, u, &t, F);
        sum += u[heat_axis] * t;
    }
    double dT = s->p.Th - s->p.Tc;
    return 1.0 + L * (sum / (double)s->N) / (s->alpha * dT);
}

void tlbmo_energy(const tlbmo_sim* s, double* ekin, double* mass) {
    double e = 0.0, m = 0.0;
    for (long n = 0; n < s->N; n++) {
        double f[QMAX], g[QMAX], r, u[3], t, F[3];
        for (int i = 0; i < s->fs.q; i++) f[i] = s->f[i * s->N + n];
        for (int i = 0; i < s->gs.q; i++) g[i] = s->g[i * s->N + n];
        node_macros(s, f, g, &r, u, &t, F);
        e += 0.5 * r * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        m += r;
    }
    if (ekin) *ekin = e;
    if (mass) *mass = m;
}

void tlbmo_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int tlbmo_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Accessors for the pins                                                     */
/* ------------------------------------------------------------------------- */

int tlbmo_velocity_set(int which, int* e, double* w, int* opp, double* M, double* Minv) {
    vset v;
    build_vset(which, &v);
    for (int i = 0; i < v.q; i++) {
        if (e)
            for (int a = 0; a < 3; a++) e[i * 3 + a] = v.e[i][a];
        if (w) w[i] = v.w[i];
        if (opp) opp[i] = v.opp[i];
        for (int k = 0; k < v.q; k++) {
            if (M) M[i * v.q + k] = v.M[i][k];
            if (Minv) Minv[i * v.q + k] = v.Minv[i][k];
        }
    }
    return v.q;
}

void tlbmo_forcing_moments(int lattice, const double* u, const double* F, double* out) {
    vset v;
    build_vset(lattice == TLBMO_D2Q9_D2Q5 ? 0 : 2, &v);
    double Ft[QMAX];
    guo_force(&v, u, F, Ft);
    matvec(v.q, v.M, Ft, out);
}

void tlbmo_flow_meq(int lattice, double rho, const double* u, double* out) {
    vset v;
    build_vset(lattice == TLBMO_D2Q9_D2Q5 ? 0 : 2, &v);
    double feq[QMAX];
    flow_feq(&v, rho, u, feq);
    matvec(v.q, v.M, feq, out);
}

void tlbmo_thermal_geq(int lattice, double a_T, double T, const double* u, double* out) {
    vset v;
    int dim = lattice == TLBMO_D2Q9_D2Q5 ? 2 : 3;
    build_vset(dim == 2 ? 1 : 3, &v);
    thermal_geq(&v, dim, a_T, T, u, out);
}
