/*
 * FP64 CPU oracle of the constraint-penalization lattice Boltzmann method
 * (Millet & Liberge, arXiv 2511.01629).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and lbm_oracle.c are a plain, slow,
 * obviously-correct restatement of the paper's equations, written to check the
 * CUDA library against.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA path (paper_2511_01629_gb300/csrc); the CUDA path never
 * includes or links it.
 *
 * Conventions (lattice units, Section 3 preamble: dx = dt = rho_f = 1):
 *   - node (i, j, k) sits at integer coordinates (i, j, k); flat index
 *     idx = (k * ny + j) * nx + i (x fastest);
 *   - populations are stored [Q][N] (population-major);
 *   - D2Q9 numbering follows the paper's Fig. 1 (1..4 axes, 5..8 diagonals),
 *     D3Q19 numbering: 1..6 = +x,-x,+y,-y,+z,-z, then the 12 edge directions
 *     in opposite pairs;
 *   - walls: halfway bounce-back, wall planes at -1/2 and n-1/2.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int D;                    /* 2 (D2Q9) or 3 (D3Q19) */
    int n[3];                 /* nodes per axis; n[2] = 1 when D = 2 */
    int periodic[3];          /* 1 = periodic axis, 0 = walls on both faces */
    double wall_u[3][2][3];   /* wall velocity of face (axis, 0 = low / 1 = high) */
    double tau;               /* BGK relaxation time, Eq. 10 */
    double alpha;             /* penalty coefficient of E = alpha * Pi_neq, Eq. 17 */
    double rho_f;             /* fluid density (1 in lattice units) */
    double g_drive[3];        /* body acceleration applied on every node */
    double g_grav[3];         /* gravity; acts on solid nodes reduced by buoyancy */
    double delta, eps_p, eps_w; /* collision range and stiffnesses, Eqs. 19-20 */
    int K;                    /* predictor-corrector sub-steps, Algorithm 1 */
} orc_config;

typedef struct orc_sim orc_sim;

/* lattice: fills c (Q*3 ints), w (Q), opp (Q); returns Q or 0 for a bad D */
int orc_lattice(int D, int* c, double* w, int* opp);

/* per-node building blocks (D selects D2Q9 / D3Q19); u, a are 3-vectors */
void orc_feq(int D, const double* u, double p, double* feq);                 /* Eq. 13 */
void orc_force(int D, double tau, const double* u, const double* a, double* F); /* Eq. 14 */
void orc_macro(int D, const double* f, const double* a, double* u, double* p);  /* Eq. 15 */
void orc_source(int D, double alpha, const double* f, const double* feq, double* S); /* Eqs. 16-17 */

/* collision force on every particle at positions X (np*3), Eqs. 19-21 */
void orc_collision_forces(const orc_config* cfg, int np, const double* X, const double* R,
                          const double* ratio, double* F);
/* the same for ellipses (2D): semi-axes a, b, orientation theta (np each) */
void orc_collision_forces_ellipse(const orc_config* cfg, int np, const double* X, const double* a,
                                  const double* b, const double* theta, const double* ratio,
                                  double* F);

/* simulation */
orc_sim* orc_create(const orc_config* cfg);
void     orc_destroy(orc_sim* s);
int      orc_add_particles(orc_sim* s, int n, const double* pos, const double* R,
                           const double* ratio, const double* vel, const double* omega);
/* ellipses (2D, Sec. 3.3): semi-axes a >= b > 0, orientation theta (nullable) */
int      orc_add_ellipses(orc_sim* s, int n, const double* pos, const double* a, const double* b,
                          const double* theta, const double* ratio, const double* vel,
                          const double* omega);
void     orc_set_f(orc_sim* s, const double* f);   /* post-collision state [Q][N] */
void     orc_get_f(const orc_sim* s, double* f);
void     orc_set_static_solid(orc_sim* s, const int* mask); /* test hook, NULL clears */
int      orc_step(orc_sim* s, int nsteps);
void     orc_fields(orc_sim* s, double* u, double* p, int* owner);
void     orc_owner_map(orc_sim* s, int* owner);
int      orc_num_particles(const orc_sim* s);
/* particle state after the last step: X^{n+1}, U^n, omega^n, theta^{n+1},
   A^{n+1} (np*3 each), count^n (np); any pointer may be NULL.  U^n and
   omega^n are also the "previous" velocities the next step averages with. */
void     orc_get_particles(const orc_sim* s, double* X, double* U, double* W, double* theta,
                           double* A, long* count);
void     orc_set_particles(orc_sim* s, const double* X, const double* U, const double* W,
                           const double* theta, const double* A);
/* reductions of Eq. 22 over the current owner map of a given velocity field u (N*3) */
void     orc_rigid_projection(orc_sim* s, const double* u, double* U, double* W, long* count);
long     orc_steps_done(const orc_sim* s);
/* threads of the per-node loops (1 unless built with OpenMP) */
int      orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
