/*
 * FP64 CPU oracle of the constraint-penalization lattice Boltzmann method
 * (Millet & Liberge, arXiv 2511.01629).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the paper used to
 * check the CUDA library.  Only tests/, __graft_entry__.smoke() and the
 * bench's cpu_baseline / reference leg may load it.  It shares no code with
 * the CUDA path.  Build with -ffp-contract=off so no multiply-add is fused
 * (the solid indicator test below must be evaluated with separate roundings).
 *
 * The per-node loops of streaming, the moments and the collision carry
 * OpenMP pragmas.  The parity build ignores them (single-threaded); a second
 * build with -fopenmp runs those loops on all host cores for the timed CPU
 * baseline and long reference runs.  Each node's arithmetic is the same in
 * both builds and every sum over nodes (Eq. 22) stays serial, so the two
 * builds give identical results.
 *
 * One time step (state: post-collision f*, particles X^n, U^{n-1}, w^{n-1}, A^n):
 *   1. solid indicator chi^n / owner map from X^n (Eq. 9, lowest index wins);
 *   2. pull streaming with halfway bounce-back (Eq. 10, left-hand side);
 *   3. acceleration f/rho on each node: drive + on solid nodes the
 *      buoyancy-reduced gravity and the collision acceleration A_i (Sec. 2.4);
 *   4. u and p (Eq. 15);
 *   5. rigid-body projection U^n, w^n over each solid domain (Eq. 22);
 *   6-7. BGK collision with Guo forcing and, on solid nodes, the
 *      penalization source S (Eqs. 10, 13, 14, 17);
 *   8. particle update (Algorithm 1 with the collision forces of Eqs. 19-21).
 * Readings of points where the paper is silent are listed at each function.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0) /* lattice sound speed squared, c_s = c / sqrt(3) (Sec. 2.2) */

/* D2Q9, numbered as in the paper's Fig. 1 (c1..c4 axes, c5..c8 diagonals). */
static const int C9[9][3] = {{0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
/* Eq. 11 gives 1/9 to the velocities of unit length and 1/36 to the
   diagonals; the printed index lists contradict Fig. 1, so the weights are
   assigned by |c| (the only assignment for which Eq. 12 holds). */
static const double W9[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int O9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* D3Q19 (not in the paper): rest, 6 axis and 12 edge velocities. */
static const int C19[19][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                               {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                               {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                               {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const int O19[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

static int lattice_q(int D) { return D == 2 ? 9 : (D == 3 ? 19 : 0); }
static const int (*lattice_c(int D))[3] { return D == 2 ? C9 : C19; }
static const double* lattice_w(int D) { return D == 2 ? W9 : W19; }
static const int* lattice_opp(int D) { return D == 2 ? O9 : O19; }

int orc_lattice(int D, int* c, double* w, int* opp) {
    int Q = lattice_q(D);
    if (!Q) return 0;
    for (int a = 0; a < Q; ++a) {
        for (int d = 0; d < 3; ++d) c[3 * a + d] = lattice_c(D)[a][d];
        w[a] = lattice_w(D)[a];
        opp[a] = lattice_opp(D)[a];
    }
    return Q;
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double cdot(const int* c, const double* v) { return c[0] * v[0] + c[1] * v[1] + c[2] * v[2]; }

/* Eq. 13: zero-shifted incompressible equilibrium; the rest population carries
   -(1-w0) p / cs^2 - w0 u.u / (2 cs^2) so that sum_a feq = 0 (Eq. 12). */
void orc_feq(int D, const double* u, double p, double* feq) {
    int Q = lattice_q(D);
    const int(*c)[3] = lattice_c(D);
    const double* w = lattice_w(D);
    double uu = dot3(u, u);
    feq[0] = -(1.0 - w[0]) * p / CS2 - w[0] * uu / (2.0 * CS2);
    for (int a = 1; a < Q; ++a) {
        double cu = cdot(c[a], u);
        feq[a] = w[a] * (p / CS2 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 14 (Guo forcing) with f/rho = a. */
void orc_force(int D, double tau, const double* u, const double* a, double* F) {
    int Q = lattice_q(D);
    const int(*c)[3] = lattice_c(D);
    const double* w = lattice_w(D);
    double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int q = 0; q < Q; ++q) {
        double cu = cdot(c[q], u);
        double term = 0.0;
        for (int d = 0; d < 3; ++d) term += ((c[q][d] - u[d]) / CS2 + cu * c[q][d] / (CS2 * CS2)) * a[d];
        F[q] = pref * w[q] * term;
    }
}

/* Eq. 15a/b with dt = 1 and f/rho = a. */
void orc_macro(int D, const double* f, const double* a, double* u, double* p) {
    int Q = lattice_q(D);
    const int(*c)[3] = lattice_c(D);
    const double* w = lattice_w(D);
    double m[3] = {0, 0, 0}, s = 0.0;
    for (int q = 0; q < Q; ++q)
        for (int d = 0; d < 3; ++d) m[d] += f[q] * c[q][d];
    for (int d = 0; d < 3; ++d) u[d] = m[d] + 0.5 * a[d];
    for (int q = 1; q < Q; ++q) s += f[q];
    *p = (s * CS2 - 0.5 * w[0] * dot3(u, u)) / (1.0 - w[0]);
}

/* Eqs. 16-17.  The paper prints Pi_neq = sum_a (f_a - feq_a) without the
   dyad; read as the non-equilibrium momentum flux sum_a (f_a - feq_a) c_a c_a.
   S_a = w_a / (2 cs^4) * E : (c_a c_a - cs^2 I), E = alpha Pi_neq. */
void orc_source(int D, double alpha, const double* f, const double* feq, double* S) {
    int Q = lattice_q(D);
    const int(*c)[3] = lattice_c(D);
    const double* w = lattice_w(D);
    double Pi[3][3] = {{0}};
    for (int q = 0; q < Q; ++q)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Pi[i][j] += (f[q] - feq[q]) * c[q][i] * c[q][j];
    for (int q = 0; q < Q; ++q) {
        double contr = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                contr += alpha * Pi[i][j] * (c[q][i] * c[q][j] - (i == j ? CS2 : 0.0));
        S[q] = w[q] / (2.0 * CS2 * CS2) * contr;
    }
}

/* ------------------------------------------------------------------------ */

struct orc_sim {
    orc_config c;
    int Q;
    long N;
    double* f;      /* post-collision populations f* [Q][N] */
    double* fs;     /* populations after streaming, f at time n [Q][N] */
    int* owner;     /* owner[N]: particle index or -1 */
    int* mask;      /* optional static penalized nodes (test hook) */
    double* u;      /* velocity of the last computed time level [N][3] */
    double* a;      /* acceleration f/rho [N][3] */
    int np, cap;
    double *X, *U, *W, *theta, *A; /* [cap][3] */
    double *R, *ratio;             /* [cap]; R = semi-major axis a of an ellipse */
    double* b;                     /* [cap] semi-minor axis; b == R for a disk */
    double *ec, *es;               /* [cap] cos, sin of the orientation theta^n (2D) */
    long* count;                   /* [cap] solid nodes at the last step */
    long steps;
};

static long nidx(const orc_sim* s, int i, int j, int k) {
    return ((long)k * s->c.n[1] + j) * s->c.n[0] + i;
}

/* displacement x_node - X along axis d, minimum image on periodic axes */
static double disp(const orc_config* c, int d, double xnode, double Xp) {
    double dx = xnode - Xp;
    if (c->periodic[d]) {
        double half = 0.5 * c->n[d];
        if (dx > half)
            dx -= c->n[d];
        else if (dx < -half)
            dx += c->n[d];
    }
    return dx;
}

static int is_ellipse(const orc_sim* s, int p) { return s->b[p] != s->R[p]; }

/* Eq. 9 on the lattice: node x is in Omega_s,p iff |x - X_p|^2 <= R_p^2, the
   squared distance summed axis by axis in order x, y, z with separate
   roundings; overlapping particles give the node to the lowest index.
   Ellipse (Sec. 3.3, 2D only): semi-axes a = R_p along the orientation
   e = (cos theta, sin theta) and b_p along e_perp = (-sin theta, cos theta);
   with u = r . e and v = r . e_perp (r = x - X_p, minimum image) the node is
   inside iff b^2 u^2 + a^2 v^2 <= a^2 b^2, i.e. (u/a)^2 + (v/b)^2 <= 1
   without a division, each product and sum rounded separately. */
static int node_inside(const orc_sim* s, int p, const int* xyz) {
    if (is_ellipse(s, p)) {
        double dx = disp(&s->c, 0, (double)xyz[0], s->X[3 * p + 0]);
        double dy = disp(&s->c, 1, (double)xyz[1], s->X[3 * p + 1]);
        double u = dx * s->ec[p] + dy * s->es[p];
        double v = dy * s->ec[p] - dx * s->es[p];
        double a2 = s->R[p] * s->R[p], b2 = s->b[p] * s->b[p];
        return b2 * (u * u) + a2 * (v * v) <= a2 * b2;
    }
    double d2 = 0.0;
    for (int d = 0; d < s->c.D; ++d) {
        double dx = disp(&s->c, d, (double)xyz[d], s->X[3 * p + d]);
        d2 = d2 + dx * dx;
    }
    return d2 <= s->R[p] * s->R[p];
}

/* Particles are visited in index order and a node keeps the first particle
   that contains it, so the lowest index wins.  Only the nodes of each
   particle's bounding box [X - R - 1, X + R + 1] (wrapped on periodic axes)
   are tested; every node outside it is farther than R from the centre (an
   ellipse lies inside the circle of radius a = R).  The orientation of an
   ellipse is theta^n, the z component of theta in 2D. */
static void build_owner(orc_sim* s) {
    int D = s->c.D;
    for (long x = 0; x < s->N; ++x) s->owner[x] = -1;
    for (int p = 0; p < s->np; ++p) {
        s->ec[p] = cos(s->theta[3 * p + 2]);
        s->es[p] = sin(s->theta[3 * p + 2]);
    }
    for (int p = 0; p < s->np; ++p) {
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            if (d >= D) continue;
            lo[d] = (int)floor(s->X[3 * p + d] - s->R[p]) - 1;
            hi[d] = (int)floor(s->X[3 * p + d] + s->R[p]) + 1;
            if (!s->c.periodic[d]) {
                if (lo[d] < 0) lo[d] = 0;
                if (hi[d] > s->c.n[d] - 1) hi[d] = s->c.n[d] - 1;
            } else if (hi[d] - lo[d] + 1 > s->c.n[d]) {
                lo[d] = 0;
                hi[d] = s->c.n[d] - 1;
            }
        }
        for (int k = lo[2]; k <= hi[2]; ++k)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int i = lo[0]; i <= hi[0]; ++i) {
                    int xyz[3] = {i, j, k};
                    for (int d = 0; d < 3; ++d) xyz[d] = ((xyz[d] % s->c.n[d]) + s->c.n[d]) % s->c.n[d];
                    long x = nidx(s, xyz[0], xyz[1], xyz[2]);
                    if (s->owner[x] < 0 && node_inside(s, p, xyz)) s->owner[x] = p;
                }
    }
}

void orc_owner_map(orc_sim* s, int* owner) {
    build_owner(s);
    memcpy(owner, s->owner, sizeof(int) * s->N);
}

orc_sim* orc_create(const orc_config* cfg) {
    if (!cfg || (cfg->D != 2 && cfg->D != 3)) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    if (s->c.D == 2) {
        s->c.n[2] = 1;
        s->c.periodic[2] = 1;
    }
    s->Q = lattice_q(s->c.D);
    s->N = (long)s->c.n[0] * s->c.n[1] * s->c.n[2];
    s->f = (double*)calloc((size_t)s->Q * s->N, sizeof(double));
    s->fs = (double*)calloc((size_t)s->Q * s->N, sizeof(double));
    s->owner = (int*)malloc(sizeof(int) * s->N);
    s->u = (double*)calloc((size_t)3 * s->N, sizeof(double));
    s->a = (double*)calloc((size_t)3 * s->N, sizeof(double));
    for (long x = 0; x < s->N; ++x) s->owner[x] = -1;
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->f); free(s->fs); free(s->owner); free(s->mask); free(s->u); free(s->a);
    free(s->X); free(s->U); free(s->W); free(s->theta); free(s->A);
    free(s->R); free(s->ratio); free(s->count); free(s->b); free(s->ec); free(s->es);
    free(s);
}

int orc_add_particles(orc_sim* s, int n, const double* pos, const double* R, const double* ratio,
                      const double* vel, const double* omega) {
    int D = s->c.D;
    if (s->np + n > s->cap) {
        int cap = s->np + n;
        s->X = (double*)realloc(s->X, sizeof(double) * 3 * cap);
        s->U = (double*)realloc(s->U, sizeof(double) * 3 * cap);
        s->W = (double*)realloc(s->W, sizeof(double) * 3 * cap);
        s->theta = (double*)realloc(s->theta, sizeof(double) * 3 * cap);
        s->A = (double*)realloc(s->A, sizeof(double) * 3 * cap);
        s->R = (double*)realloc(s->R, sizeof(double) * cap);
        s->ratio = (double*)realloc(s->ratio, sizeof(double) * cap);
        s->count = (long*)realloc(s->count, sizeof(long) * cap);
        s->b = (double*)realloc(s->b, sizeof(double) * cap);
        s->ec = (double*)realloc(s->ec, sizeof(double) * cap);
        s->es = (double*)realloc(s->es, sizeof(double) * cap);
        s->cap = cap;
    }
    for (int i = 0; i < n; ++i) {
        int p = s->np + i;
        for (int d = 0; d < 3; ++d) {
            s->X[3 * p + d] = d < D ? pos[D * i + d] : 0.0;
            s->U[3 * p + d] = (vel && d < D) ? vel[D * i + d] : 0.0;
            s->W[3 * p + d] = 0.0;
            s->theta[3 * p + d] = 0.0;
            s->A[3 * p + d] = 0.0;
        }
        if (omega) {
            if (D == 2)
                s->W[3 * p + 2] = omega[i];
            else
                for (int d = 0; d < 3; ++d) s->W[3 * p + d] = omega[3 * i + d];
        }
        s->R[p] = R[i];
        s->b[p] = R[i];
        s->ec[p] = 1.0;
        s->es[p] = 0.0;
        s->ratio[p] = ratio[i];
        s->count[p] = 0;
    }
    s->np += n;
    return 0;
}

/* Ellipses (2D): semi-axes a >= b > 0, orientation theta (angle of the a axis
   from +x, counter-clockwise).  b == a gives a disk.  Returns -1 in 3D or for
   bad axes. */
int orc_add_ellipses(orc_sim* s, int n, const double* pos, const double* a, const double* b,
                     const double* theta, const double* ratio, const double* vel,
                     const double* omega) {
    if (s->c.D != 2) return -1;
    for (int i = 0; i < n; ++i)
        if (!(b[i] > 0.0 && b[i] <= a[i])) return -1;
    int first = s->np;
    orc_add_particles(s, n, pos, a, ratio, vel, omega);
    for (int i = 0; i < n; ++i) {
        s->b[first + i] = b[i];
        s->theta[3 * (first + i) + 2] = theta ? theta[i] : 0.0;
    }
    return 0;
}

void orc_set_f(orc_sim* s, const double* f) { memcpy(s->f, f, sizeof(double) * s->Q * s->N); }
void orc_get_f(const orc_sim* s, double* f) { memcpy(f, s->f, sizeof(double) * s->Q * s->N); }

void orc_set_static_solid(orc_sim* s, const int* mask) {
    free(s->mask);
    s->mask = NULL;
    if (mask) {
        s->mask = (int*)malloc(sizeof(int) * s->N);
        memcpy(s->mask, mask, sizeof(int) * s->N);
    }
}

int orc_num_particles(const orc_sim* s) { return s->np; }
long orc_steps_done(const orc_sim* s) { return s->steps; }

/* Pull streaming: f_a(x) = f*_a(x - c_a).  Where x - c_a lies beyond a wall
   (planes at -1/2 and n - 1/2) the population is the bounced-back
   f*_opp(a)(x) plus 2 w_a (c_a . u_w) / cs^2 for a moving wall (the
   velocity-based model carries no density factor in its first moment). */
static void stream(orc_sim* s) {
    const orc_config* c = &s->c;
    const int(*cv)[3] = lattice_c(c->D);
    const double* w = lattice_w(c->D);
    const int* opp = lattice_opp(c->D);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < c->n[2]; ++k)
        for (int j = 0; j < c->n[1]; ++j)
            for (int i = 0; i < c->n[0]; ++i) {
                int xyz[3] = {i, j, k};
                long x = nidx(s, i, j, k);
                for (int a = 0; a < s->Q; ++a) {
                    int src[3], wall = 0;
                    double uw[3] = {0, 0, 0};
                    for (int d = 0; d < 3; ++d) {
                        src[d] = xyz[d] - cv[a][d];
                        if (src[d] < 0 || src[d] >= c->n[d]) {
                            if (c->periodic[d]) {
                                src[d] = (src[d] + c->n[d]) % c->n[d];
                            } else {
                                int face = src[d] < 0 ? 0 : 1;
                                wall = 1;
                                for (int e = 0; e < 3; ++e) uw[e] += c->wall_u[d][face][e];
                            }
                        }
                    }
                    if (wall)
                        s->fs[a * s->N + x] = s->f[opp[a] * s->N + x] + 2.0 * w[a] * cdot(cv[a], uw) / CS2;
                    else
                        s->fs[a * s->N + x] = s->f[a * s->N + nidx(s, src[0], src[1], src[2])];
                }
            }
}

/* Acceleration f/rho.  The monolithic momentum equation (Eq. 5) carries
   rho(x) g; with one pressure field for fluid and solid the hydrostatic part
   rho_f g is absorbed in p, leaving (1 - rho_f / rho_s) g on solid nodes and
   none on fluid nodes.  Algorithm 1 adds A_i on the nodes of particle i.
   g_drive is a body acceleration on every node (channel driving). */
static void node_accel(const orc_sim* s, long x, double* a) {
    for (int d = 0; d < 3; ++d) a[d] = s->c.g_drive[d];
    int p = s->owner[x];
    if (p >= 0) {
        double red = 1.0 - 1.0 / s->ratio[p]; /* ratio = rho_s / rho_f */
        for (int d = 0; d < 3; ++d) a[d] += red * s->c.g_grav[d] + s->A[3 * p + d];
    }
}

static void node_coords(const orc_sim* s, long x, int* xyz) {
    xyz[0] = (int)(x % s->c.n[0]);
    xyz[1] = (int)((x / s->c.n[0]) % s->c.n[1]);
    xyz[2] = (int)(x / ((long)s->c.n[0] * s->c.n[1]));
}

/* solve the 3x3 system I w = L by Cramer's rule */
static void solve3(const double I[3][3], const double* L, double* w) {
    double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                 I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                 I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
    for (int col = 0; col < 3; ++col) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) M[r][q] = (q == col) ? L[r] : I[r][q];
        double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                    M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                    M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        w[col] = dc / det;
    }
}

/* Eq. 22 on the lattice: U = (1/M) sum rho_s u, I w = sum r x (rho_s u), with
   M = rho_s * (number of solid nodes) and the discrete moment of inertia
   I = rho_s sum (|r|^2 1 - r r^T) (rho_s cancels).  In 2D, w = w_z and
   I reduces to rho_s sum |r|^2. */
static void projection(orc_sim* s, const double* u, double* U, double* W, long* count) {
    int np = s->np, D = s->c.D;
    double* su = (double*)calloc((size_t)3 * np, sizeof(double));
    double* sl = (double*)calloc((size_t)3 * np, sizeof(double));
    double* si = (double*)calloc((size_t)9 * np, sizeof(double));
    long* cnt = (long*)calloc((size_t)np, sizeof(long));
    for (long x = 0; x < s->N; ++x) {
        int p = s->owner[x];
        if (p < 0) continue;
        int xyz[3];
        node_coords(s, x, xyz);
        double r[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) r[d] = disp(&s->c, d, (double)xyz[d], s->X[3 * p + d]);
        const double* ux = u + 3 * x;
        cnt[p] += 1;
        for (int d = 0; d < 3; ++d) su[3 * p + d] += ux[d];
        sl[3 * p + 0] += r[1] * ux[2] - r[2] * ux[1];
        sl[3 * p + 1] += r[2] * ux[0] - r[0] * ux[2];
        sl[3 * p + 2] += r[0] * ux[1] - r[1] * ux[0];
        double rr = dot3(r, r);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) si[9 * p + 3 * i + j] += (i == j ? rr : 0.0) - r[i] * r[j];
    }
    for (int p = 0; p < np; ++p) {
        count[p] = cnt[p];
        for (int d = 0; d < 3; ++d) U[3 * p + d] = su[3 * p + d] / (double)cnt[p];
        if (D == 2) {
            W[3 * p + 0] = 0.0;
            W[3 * p + 1] = 0.0;
            W[3 * p + 2] = sl[3 * p + 2] / si[9 * p + 8]; /* I_zz = sum (rx^2 + ry^2) */
        } else {
            double I[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) I[i][j] = si[9 * p + 3 * i + j];
            solve3(I, sl + 3 * p, W + 3 * p);
        }
    }
    free(su); free(sl); free(si); free(cnt);
}

void orc_rigid_projection(orc_sim* s, const double* u, double* U, double* W, long* count) {
    build_owner(s);
    projection(s, u, U, W, count);
}

/* Extent of particle p along the unit vector (nx, ny): R for a disk; for an
   ellipse its support distance sqrt(a^2 (n.e)^2 + b^2 (n.e_perp)^2), the
   distance from the centre to the tangent line normal to n. */
static double extent(const double* R, const double* b, const double* ec, const double* es, int p,
                     double nx, double ny) {
    if (!b || b[p] == R[p]) return R[p];
    double ne = nx * ec[p] + ny * es[p];
    double np_ = ny * ec[p] - nx * es[p];
    return sqrt(R[p] * R[p] * (ne * ne) + b[p] * b[p] * (np_ * np_));
}

/* Eqs. 19-21.  C = (rho_s - rho_f) |g| of the particle receiving the force;
   the image of particle i behind wall k is its mirror across the wall plane.
   Ellipses (the paper states the forces for disks only): R_i + R_j becomes
   the sum of the two extents along the line of centres, and 2 R_i of a wall
   twice the extent along the wall normal, so that the forces act when the
   gap between the two shapes, measured along that line, is below delta (for
   walls delta / 2, as for disks).  b, ec, es = NULL: all disks. */
static void collision_forces(const orc_config* cfg, int np, const double* X, const double* R,
                             const double* b, const double* ec, const double* es,
                             const double* ratio, double* F) {
    double gmag = sqrt(dot3(cfg->g_grav, cfg->g_grav));
    int D = cfg->D;
    for (int i = 0; i < np; ++i) {
        double C = (ratio[i] - 1.0) * cfg->rho_f * gmag;
        double Fi[3] = {0, 0, 0};
        for (int j = 0; j < np; ++j) {
            if (j == i) continue;
            double dv[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                dv[d] = X[3 * i + d] - X[3 * j + d];
                if (cfg->periodic[d]) {
                    double half = 0.5 * cfg->n[d];
                    if (dv[d] > half)
                        dv[d] -= cfg->n[d];
                    else if (dv[d] < -half)
                        dv[d] += cfg->n[d];
                }
            }
            double dij = sqrt(dot3(dv, dv));
            double range = R[i] + R[j] + cfg->delta;
            if (b && (b[i] != R[i] || b[j] != R[j]) && dij > 0.0)
                range = extent(R, b, ec, es, i, dv[0] / dij, dv[1] / dij) +
                        extent(R, b, ec, es, j, dv[0] / dij, dv[1] / dij) + cfg->delta;
            if (dij <= range) {
                double s = (range - dij) / cfg->delta;
                for (int d = 0; d < 3; ++d) Fi[d] += C / cfg->eps_p * dv[d] * s * s;
            }
        }
        for (int d = 0; d < D; ++d) {
            if (cfg->periodic[d]) continue;
            double walls[2] = {-0.5, cfg->n[d] - 0.5};
            for (int face = 0; face < 2; ++face) {
                double Xim = 2.0 * walls[face] - X[3 * i + d]; /* mirror image */
                double diff = X[3 * i + d] - Xim;
                double dprime = fabs(diff);
                double range = 2.0 * extent(R, b, ec, es, i, d == 0 ? 1.0 : 0.0, d == 1 ? 1.0 : 0.0) +
                               cfg->delta;
                if (dprime <= range) {
                    double s = (range - dprime) / cfg->delta;
                    Fi[d] += C / cfg->eps_w * diff * s * s;
                }
            }
        }
        for (int d = 0; d < 3; ++d) F[3 * i + d] = Fi[d];
    }
}

void orc_collision_forces(const orc_config* cfg, int np, const double* X, const double* R,
                          const double* ratio, double* F) {
    collision_forces(cfg, np, X, R, NULL, NULL, NULL, ratio, F);
}

void orc_collision_forces_ellipse(const orc_config* cfg, int np, const double* X, const double* a,
                                  const double* b, const double* theta, const double* ratio,
                                  double* F) {
    double* ec = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    double* es = (double*)malloc(sizeof(double) * (np > 0 ? np : 1));
    for (int i = 0; i < np; ++i) {
        ec[i] = cos(theta[i]);
        es[i] = sin(theta[i]);
    }
    collision_forces(cfg, np, X, a, b, ec, es, ratio, F);
    free(ec);
    free(es);
}

/* Algorithm 1 (dt = 1) for all particles together, since F_col at each
   sub-step depends on every particle's position at that sub-step.  M is the
   discrete mass rho_s * count^n.  Afterwards A^{n+1} of Algorithm 1:
   (2/dt^2)(X^{n+1} - X^n - dt Ubar) is, in exact arithmetic, twice the sum of
   the K correction displacements dt^2/(2M) (dt/K)^2/2 ... (F1 + F2) that
   Algorithm 1 adds to X^n + dt Ubar, and it is evaluated as that sum: the
   printed difference of positions (~10^3) minus a displacement (~10^-5)
   cancels catastrophically and would leave ulp(X) ~ 2e-13 of rounding noise
   per step in A, which then acts as a force on the solid nodes.  Then
   the orientation theta^{n+1} = theta^n + (w^n + w^{n-1}) / 2 (the paper
   gives no rule; trapezoid like X), and U^{n-1} <- U^n.  Returns -1 when a
   particle centre has left the domain across a wall. */
static int particle_update(orc_sim* s, const double* Un, const double* Wn) {
    int np = s->np, K = s->c.K > 0 ? s->c.K : 1;
    size_t sz = sizeof(double) * 3 * (size_t)np;
    double *Ubar = (double*)malloc(sz), *Xk = (double*)malloc(sz), *Xs = (double*)malloc(sz);
    double *F1 = (double*)malloc(sz), *F2 = (double*)malloc(sz);
    for (int i = 0; i < 3 * np; ++i) {
        Ubar[i] = 0.5 * (Un[i] + s->U[i]);
        Xk[i] = s->X[i];
    }
    double* corr = (double*)calloc((size_t)3 * (np > 0 ? np : 1), sizeof(double));
    double h = 1.0 / K;
    for (int k = 1; k <= K; ++k) {
        collision_forces(&s->c, np, Xk, s->R, s->b, s->ec, s->es, s->ratio, F1);
        for (int i = 0; i < 3 * np; ++i) Xs[i] = Xk[i] + h * Ubar[i];
        collision_forces(&s->c, np, Xs, s->R, s->b, s->ec, s->es, s->ratio, F2);
        for (int p = 0; p < np; ++p) {
            double M = s->ratio[p] * s->c.rho_f * (double)s->count[p];
            for (int d = 0; d < 3; ++d) {
                double c = 1.0 / (2.0 * M) * h * h * 0.5 * (F1[3 * p + d] + F2[3 * p + d]);
                corr[3 * p + d] += c;
                Xk[3 * p + d] = Xs[3 * p + d] + c;
            }
        }
    }
    int status = 0;
    for (int p = 0; p < np; ++p) {
        for (int d = 0; d < 3; ++d) {
            int i = 3 * p + d;
            s->A[i] = 2.0 * corr[i]; /* = 2 (X^{n+1} - X^n - Ubar) in exact arithmetic */
            double xn = Xk[i];
            if (d < s->c.D) {
                if (s->c.periodic[d]) {
                    if (xn >= s->c.n[d]) xn -= s->c.n[d];
                    else if (xn < 0.0) xn += s->c.n[d];
                } else if (xn < -0.5 || xn > s->c.n[d] - 0.5) {
                    status = -1;
                }
            }
            s->X[i] = xn;
            s->theta[i] += 0.5 * (Wn[i] + s->W[i]);
            s->U[i] = Un[i];
            s->W[i] = Wn[i];
        }
    }
    free(Ubar); free(Xk); free(Xs); free(F1); free(F2); free(corr);
    return status;
}

/* steps 1-4 of the time step: owner map, streaming, acceleration, u and p */
static void macroscopic(orc_sim* s, double* p_out) {
    build_owner(s);
    stream(s);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < s->N; ++x) {
        double fl[19];
        for (int q = 0; q < s->Q; ++q) fl[q] = s->fs[q * s->N + x];
        node_accel(s, x, s->a + 3 * x);
        double p;
        orc_macro(s->c.D, fl, s->a + 3 * x, s->u + 3 * x, &p);
        if (p_out) p_out[x] = p;
    }
}

int orc_step(orc_sim* s, int nsteps) {
    int D = s->c.D, Q = s->Q;
    double* Un = (double*)malloc(sizeof(double) * 3 * (s->np > 0 ? s->np : 1));
    double* Wn = (double*)malloc(sizeof(double) * 3 * (s->np > 0 ? s->np : 1));
    int status = 0;
    for (int it = 0; it < nsteps && status == 0; ++it) {
        macroscopic(s, NULL);
        if (s->np > 0) projection(s, s->u, Un, Wn, s->count);
#pragma omp parallel for schedule(static)
        for (long x = 0; x < s->N; ++x) {
            double fl[19], feq[19], F[19], S[19];
            double* ux = s->u + 3 * x;
            double p;
            for (int q = 0; q < Q; ++q) fl[q] = s->fs[q * s->N + x];
            orc_macro(D, fl, s->a + 3 * x, ux, &p);
            orc_feq(D, ux, p, feq);
            orc_force(D, s->c.tau, ux, s->a + 3 * x, F);
            int solid = s->owner[x] >= 0 || (s->mask && s->mask[x]);
            if (solid)
                orc_source(D, s->c.alpha, fl, feq, S);
            else
                for (int q = 0; q < Q; ++q) S[q] = 0.0;
            for (int q = 0; q < Q; ++q)
                s->f[q * s->N + x] = fl[q] - (fl[q] - feq[q]) / s->c.tau + F[q] + S[q];
        }
        if (s->np > 0) status = particle_update(s, Un, Wn);
        s->steps += 1;
    }
    free(Un); free(Wn);
    return status;
}

/* macroscopic fields of the current state (what the next step will see) */
void orc_fields(orc_sim* s, double* u, double* p, int* owner) {
    double* pp = (double*)malloc(sizeof(double) * s->N);
    macroscopic(s, pp);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * s->N);
    if (p) memcpy(p, pp, sizeof(double) * s->N);
    if (owner) memcpy(owner, s->owner, sizeof(int) * s->N);
    free(pp);
}

void orc_get_particles(const orc_sim* s, double* X, double* U, double* W, double* theta, double* A,
                       long* count) {
    size_t sz = sizeof(double) * 3 * s->np;
    if (X) memcpy(X, s->X, sz);
    if (U) memcpy(U, s->U, sz);
    if (W) memcpy(W, s->W, sz);
    if (theta) memcpy(theta, s->theta, sz);
    if (A) memcpy(A, s->A, sz);
    if (count) memcpy(count, s->count, sizeof(long) * s->np);
}

void orc_set_particles(orc_sim* s, const double* X, const double* U, const double* W,
                       const double* theta, const double* A) {
    size_t sz = sizeof(double) * 3 * s->np;
    if (X) memcpy(s->X, X, sz);
    if (U) memcpy(s->U, U, sz);
    if (W) memcpy(s->W, W, sz);
    if (theta) memcpy(s->theta, theta, sz);
    if (A) memcpy(s->A, A, sz);
}

/* threads the per-node loops run on: 1 in the parity build */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
