/*
 * FP64 CPU oracle for the double-distribution thermal lattice Boltzmann step
 * (Xu & Li, "Multi-GPU thermal lattice Boltzmann simulations using OpenACC and
 * MPI", §2.2, Eqs. (5)-(7), (10)-(11)).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this library: only the test suite, the smoke check and the timed CPU baseline
 * of the benchmark use it.  It shares no code, header, table or generator with
 * the CUDA library.
 *
 * Conventions (all arrays dense, x fastest):
 *   node index  n = x + nx*(y + ny*z)          (2D: nz = 1)
 *   population  f[i*N + n], g[i*N + n]          N = nx*ny*nz
 * The state "after t steps" is the PRE-collision population set at time t.
 */
#ifndef TLBM_ORACLE_H
#define TLBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { TLBMO_D2Q9_D2Q5 = 0, TLBMO_D3Q19_D3Q7 = 1 };
enum { TLBMO_RB = 0, TLBMO_SIDE_HEATED = 1 };

/* Every double set to NaN means "derive the default". */
typedef struct {
    int walls;            /* TLBMO_RB or TLBMO_SIDE_HEATED */
    int periodic_mask;    /* bit0 x, bit1 y, bit2 z: periodic axis (test-only) */
    int u_is_ma;          /* 0: U = Ma*c_s (default); 1: U = Ma */
    double a_T;           /* thermal equilibrium constant, default -2/3 (2D), -3/4 (3D) */
    double nu, alpha, gbeta;       /* override the Ra/Pr/Ma mapping */
    double s_rho, s_e, s_eps, s_j, s_q, s_pi, s_m; /* flow rates */
    double q_e, q_v;               /* thermal even-moment rates */
    double body_force[3];          /* constant acceleration, force density rho*a */
    double Th, Tc;                 /* hot / cold wall temperatures (+0.5 / -0.5) */
} tlbmo_params;

typedef struct tlbmo_sim tlbmo_sim;

void tlbmo_default_params(tlbmo_params* p);
/* NULL on invalid arguments (sizes < 3, Ra/Pr/Ma <= 0, tau - 1/2 <= 1e-6). */
tlbmo_sim* tlbmo_create(int nx, int ny, int nz, int lattice, double Ra, double Pr,
                        double Ma, const tlbmo_params* p);
void   tlbmo_destroy(tlbmo_sim* s);
/* out[0..]: U, H, nu, alpha, gbeta, a_T, omega, then S[qf], then Q[qg] */
int    tlbmo_derived(const tlbmo_sim* s, double* out, int cap);
void   tlbmo_init(tlbmo_sim* s, uint64_t seed, double noise_amp);
void   tlbmo_step(tlbmo_sim* s, int64_t n);
int64_t tlbmo_time(const tlbmo_sim* s);
void   tlbmo_get_populations(const tlbmo_sim* s, double* f, double* g);
void   tlbmo_set_populations(tlbmo_sim* s, const double* f, const double* g);
/* any pointer may be NULL */
void   tlbmo_macros(const tlbmo_sim* s, double* rho, double* ux, double* uy,
                    double* uz, double* T);
double tlbmo_nusselt(const tlbmo_sim* s);
void   tlbmo_energy(const tlbmo_sim* s, double* ekin, double* mass);
void   tlbmo_set_threads(int n);
int    tlbmo_get_threads(void);

/* ---- table and single-node accessors used by the pins ---- */
/* which: 0 D2Q9, 1 D2Q5, 2 D3Q19, 3 D3Q7.  Returns q.  Any output may be NULL.
 * e[q*3], w[q] (flow sets only; thermal w depends on a_T), opp[q],
 * M[q*q] row-major (M[k*q+i] = row k evaluated at e_i), Minv[q*q]. */
int    tlbmo_velocity_set(int which, int* e, double* w, int* opp, double* M, double* Minv);
/* Guo source in moment space, M * Ftilde(u, F), for lattice 0/1 (flow set). */
void   tlbmo_forcing_moments(int lattice, const double* u, const double* F, double* out);
/* Moment-space equilibrium M f_eq(rho, u) for the flow set. */
void   tlbmo_flow_meq(int lattice, double rho, const double* u, double* out);
/* Thermal equilibrium populations N^-1 n_eq(T, u). */
void   tlbmo_thermal_geq(int lattice, double a_T, double T, const double* u, double* out);
/* Collide one node with the sim's parameters (no streaming). */
void   tlbmo_collide_node(const tlbmo_sim* s, const double* f, const double* g,
                          double* fpost, double* gpost);
/* The init random number: top 53 bits of splitmix64(seed ^ splitmix64(idx)) * 2^-53. */
double tlbmo_uniform(uint64_t seed, uint64_t idx);

#ifdef __cplusplus
}
#endif
#endif
