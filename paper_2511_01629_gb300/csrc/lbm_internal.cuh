// Internal device-side definitions of lbmpen (not part of the C ABI).
//
// Layout in HBM, per instance:
//   populations  f[2][QS][nz][ny][pitch]  (ping-pong; QS = Q - 1 because the
//                rest population is never read back, see lbmpen.h), FP32 or
//                FP16 (scaled by 2^k); pitch = nx rounded up to 32 elements
//                so every row starts on a 128-byte boundary;
//   particles    FP64 state arrays [np][3] plus one PRec per particle that
//                the fluid kernel reads (centre, radius, solid acceleration);
//   tile lists   list_cnt[2][ntiles], list_ent[2][ntiles][cap]: for each
//                tile the particles whose bounding box overlaps it, built by
//                the particle kernel for the next step (no per-node mask);
//   velocity boxes  ubox: per particle a box of (2H + 1)^D entries, H =
//                ceil(R) + 2, centred on floor(X): the fluid kernel stores the
//                velocity of each node the particle owns there (float2 in 2D,
//                float4 in 3D), the particle kernel sums the entries into the
//                exact fixed-point totals of Eq. 22 and resets them to NaN,
//                the mark of an empty entry.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmpen {

// ---------------------------------------------------------------- lattices --
// D2Q9 in the paper's Fig. 1 numbering and D3Q19; q = 0 is the rest velocity.
__host__ __device__ constexpr int d2q9_c(int q, int d) {
    return d == 0 ? (q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0))
         : d == 1 ? (q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0))
                  : 0;
}
__host__ __device__ constexpr int d2q9_opp(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5);
}
__host__ __device__ constexpr float d2q9_w(int q) {
    return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// D3Q19: 1..6 axes (+x,-x,+y,-y,+z,-z), 7..18 edges in opposite pairs
__host__ __device__ constexpr int d3q19_c(int q, int d) {
    // rows: x, y, z components for q = 0..18
    return d == 0 ? (q == 1 || q == 7 || q == 9 || q == 11 || q == 13 ? 1
                     : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14 ? -1 : 0))
         : d == 1 ? (q == 3 || q == 7 || q == 10 || q == 15 || q == 17 ? 1
                     : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18 ? -1 : 0))
                  : (q == 5 || q == 11 || q == 14 || q == 15 || q == 18 ? 1
                     : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17 ? -1 : 0));
}
__host__ __device__ constexpr int d3q19_opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr float d3q19_w(int q) {
    return q == 0 ? 1.0f / 3.0f : (q <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// FP32 coefficients A_q = w_q / cs^2 = 3 w_q.  1/3 and 1/12 are not binary
// fractions, so the nearest floats would give sum_q A_q c_qx^2 = 1 + 7e-9 and
// every collision would scale the momentum of feq by that factor (a drift
// of 1e-5 over 1000 steps).  The pairs below are the closest floats with
// sum_q A_q c_qx^2 = 1 exactly (2 A1 + 4 A2 = 1 in D2Q9, 2 Aa + 8 Ae = 1 in
// D3Q19), so Eqs. 12 and 14 keep u exactly up to the rounding of each operation.
constexpr float D2Q9_A1 = 0x1.555556p-2f;  // axis, ~1/3
constexpr float D2Q9_A2 = 0x1.555554p-4f;  // diagonal, ~1/12
constexpr float D3Q19_AA = 0x1.555554p-3f; // axis, ~1/6
constexpr float D3Q19_AE = 0x1.555556p-4f; // edge, ~1/12

template <int Q> struct Lat;
template <> struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int c(int q, int d) { return d2q9_c(q, d); }
    __host__ __device__ static constexpr int opp(int q) { return d2q9_opp(q); }
    __host__ __device__ static constexpr float w(int q) { return d2q9_w(q); }
    __host__ __device__ static constexpr float A(int q) { return q <= 4 ? D2Q9_A1 : D2Q9_A2; }
    // sum over the stored velocities q >= 1 of A_q
    static constexpr double SUMA = 4.0 * (double)D2Q9_A1 + 4.0 * (double)D2Q9_A2;
};
template <> struct Lat<19> {
    static constexpr int D = 3;
    __host__ __device__ static constexpr int c(int q, int d) { return d3q19_c(q, d); }
    __host__ __device__ static constexpr int opp(int q) { return d3q19_opp(q); }
    __host__ __device__ static constexpr float w(int q) { return d3q19_w(q); }
    __host__ __device__ static constexpr float A(int q) { return q <= 6 ? D3Q19_AA : D3Q19_AE; }
    static constexpr double SUMA = 6.0 * (double)D3Q19_AA + 12.0 * (double)D3Q19_AE;
};

// ------------------------------------------------------------- descriptors --
// Totals of Eq. 22 per particle, all int64:
//   0 count, 1-3 sum d, 4-9 sum d_i d_j (xx, yy, zz, xy, xz, yz),
//   10-12 sum u, 13-15 sum d x u;  d = node - floor(X) (integer offsets),
//   u in fixed point round(u * 2^FXBITS).  Integer sums are exact and do not
//   depend on the order of addition, so the reductions are deterministic;
//   they are converted to FP64 once per particle.  The additions wrap modulo
//   2^64, so a partial or an intermediate total may overflow and the final
//   total is still exact whenever it fits in int64.  It does under these
//   bounds, with |u| < 1/2 (a larger speed stops the run as diverged) and
//   |d| < R + 2 on a particle's n nodes (n < pi (R + 1)^2 in 2D,
//   4/3 pi (R + 1)^3 in 3D): the largest total, a component of sum d x u, is
//   below n (R + 2) 2^(FXBITS - 1), under 2^62 for R <= MAX_RADIUS = 120 in 2D
//   and under 2^63 for R <= MAX_RADIUS_3D = 40 in 3D; a 3D sphere of radius
//   120 (7.2e6 nodes) could reach 2^68, so larger spheres are refused.
constexpr int NPV = 16;
constexpr int CAND_BYTES = 64;  // one candidate record of a tile list (Cand)
constexpr int FXBITS = 40;
constexpr double MAX_RADIUS = 120.0;     // largest disk radius (2D)
constexpr double MAX_RADIUS_3D = 40.0;   // largest sphere radius (3D)
constexpr int LIST_CAP = 64;   // particles listed per tile (overflow -> LBM_ERR_CAPACITY)
constexpr int KBITS = 10;      // list entry = particle << KBITS | slot
constexpr int MAXK = 1 << KBITS;

// Status word bits (device), mapped to lbm_status on the host.
enum { ST_DIVERGED = 1, ST_CAPACITY = 2, ST_PARTICLE = 4, ST_DISPLACEMENT = 8, ST_TIMEOUT = 16 };

// Per-particle constants (host-computed, FP64), stride PCONST_N.
// PC_R is the radius, or the semi-major axis a of an ellipse; PC_B the
// semi-minor axis b (== R for a disk).
enum { PC_GFAC = 0, PC_CPAIR = 1, PC_CWALL = 2, PC_INVDELTA = 3, PC_INVRHOS = 4, PC_R = 5, PC_B = 6,
       PCONST_N = 8 };

// Grid-wide barrier of the particle kernel (all its blocks are resident).
struct GridBar {
    unsigned count;
    unsigned gen;
};

// Particle record read by the fluid kernel; written by the particle kernel
// for the next step.  A disk (sphere) is inside |x - X|^2 <= R^2; an ellipse
// (2D, shape = 1) with semi-axes a = R and b along e = (cos theta, sin theta)
// and e_perp is inside b^2 (r.e)^2 + a^2 (r.e_perp)^2 <= a^2 b^2.
struct __align__(16) PRec {
    double X[3];     // centre X^n (FP64, exact indicator test)
    double R2;       // R * R (a * a of an ellipse)
    int ref[3];      // floor(X) per axis
    int ntiles;      // tiles of the bounding box (slots written this step)
    float frac[3];   // X - floor(X) as float (filter test)
    float R2lo, R2hi;  // float thresholds: d2 < R2lo inside, d2 > R2hi outside
                       //   (an ellipse: only d2 > R2hi, its circumscribed circle)
    float a[3];      // solid-node acceleration (1 - rho_f/rho_s) g + A_i
    int shape;       // 0 disk or sphere, 1 ellipse
    int pad;
    double ec, es;   // cos, sin of theta^n (ellipse; 1, 0 otherwise)
    double b2;       // b * b
    float fc, fs;    // ec, es as float (filter test)
    float ia2, ib2;  // 1 / a^2, 1 / b^2 as float (filter test)
    float qlo, qhi;  // float thresholds of (r.e)^2 / a^2 + (r.e_perp)^2 / b^2
    float pad2[2];
};
static_assert(sizeof(PRec) == 144, "particle record layout");

// The fields of a particle's record that depend only on its size and shape,
// computed on the host when it is added (R2 = R * R and b2 = B * B exactly as
// the exact test needs them) and copied into every new record.
struct RecConst {
    double R2, b2;
    float R2lo, R2hi, ia2, ib2, qlo, qhi;
    int shape, pad;
};
static_assert(sizeof(RecConst) == 48, "record constants layout");

struct InstDesc {
    int n[3];
    int pitch;
    long long qstride;        // elements per stored population
    int periodic[3];
    int ntile[3];             // tiles per axis
    int tile0;                // first global tile of this instance
    int np;                   // particles
    int maxk;                 // most tiles a particle's bounding box may cover (list slot k)
    int part0;                // global index of particle 0 (batched arrays)
    float tau_inv, keep;      // 1/tau and 1 - 1/tau
    float fpref;              // 1 - 1/(2 tau)
    float alpha;
    float gdrive[3];
    float ggrav[3];
    float s_store, s_load;    // FP16 storage scale 2^k and 2^-k (1 for FP32)
    float wterm[3][2][19];    // bounce-back term 2 w_q (c_q . u_wall) / cs^2 per face
    void* f[2];
    PRec* prec;               // [np] records read by this step's fluid kernel
    PRec* prec_out;           // [np] records written for the next step (== prec except
                              //   while the adjoint recomputes a segment into per-step slots)
    int* list_cnt[2];         // [ntiles]
    uint32_t* list_ent[2];    // [ntiles][LIST_CAP]
    void* list_rec[2];        // [ntiles][LIST_CAP] 64-byte candidate records (Cand), same slots
    float* ubox;              // velocity boxes of the particles (see above), NaN when empty
    float* ubox_scratch;      // same shape: sink of launches that do not advance the state
    int2* boxinfo;            // [np] box of particle p: first entry, H
    long long* btot;          // [np][NPV] the box's totals of Eq. 22 (k_box_sums)
    // particle state (FP64), [np][3] unless noted
    double* X;
    double* U;                // U^{n-1} entering the step, U^n after it
    double* W;
    double* Un;               // U^n of the current step (finalised)
    double* Wn;
    double* theta;
    double* A;
    double* R;                // [np]
    double* ratio;            // [np] rho_s / rho_f
    int* count;               // [np]
    double* Xk;               // [2][np][3] Algorithm-1 sub-step positions
    double* Ubar;             // [np][3]
    double* Acor;             // [np][3] sum of the sub-step corrections of Algorithm 1 (K > 1)
    float* Xf;                // [2][np][4] float copy of X^{k} (w = R) for the pair filter
    float* Xsf;               // [2][np][4] float copy of X^{k} + Ubar/K (w = R): predicted positions
    const RecConst* rconst;   // [np] size and shape fields of the records
    double* pconst;           // [np][8]: 1 - rho_f/rho_s, C/eps_p, C/eps_w, 1/delta,
                              //   1/(rho_s rho_f... see PCONST_*), R
    double* invc;             // [np] 1 / (solid nodes at step n)
    double rho_f;
    double gmag;              // |g_grav|
    double delta, eps_p, eps_w;
    double inv_eps_p, inv_eps_w;
    double hK;                // 1 / K
    int K;
    int* status;
    // adjoint recording (null outside the adjoint's segment recomputation):
    double* adj_geo;          // [np][NPV] projection sums of this step about X^n: count,
                              //   sum r (3), sum r r^T (xx yy zz xy xz yz), sum u (3), sum r x u (3)
    double* rec_state;        // [np][16] state after this step: X, U, W, theta, A (3 each), count
};

// Kernel shape of the fused fluid kernel: a tile is (32 * vec) x rows_y x rows_z
// nodes; each warp handles whole x-rows of the tile.
struct Shape {
    int vec;     // register path: nodes per thread along x (vector width)
    int ty, tz;  // tile rows along y and z
    int warps;   // warps per block (consumer warps on the TMA path)
    int persistent;  // register path: blocks pulling tiles from a work counter
    int tma;     // 1: TMA-staged pipeline kernel
    int stages;  // TMA path: shared-memory ring stages
    int tw;      // tile width in nodes (32 * vec, or the TMA box width without halo)
};

// ------------------------------------------------------------- adjoint ---
// One instance's view of one step of the backward sweep (see lbm_adjoint.cu).
struct AdjFluid {
    const void* fin;         // populations entering step n (storage type, population layout)
    const PRec* prec;        // particle records of step n
    const int* lcnt;         // tile lists of step n
    const uint32_t* lent;
    const float* lam_src;    // adjoint of the pre-collision populations of step n + 1
                             //   (population layout, FP32), or the field seed ([Q][N])
    float* lam_dst;          // adjoint of the pre-collision populations of step n
    const float* coef;       // [np][8]: dU^n / count (3), I^-1 dW^n (3)
    double* Abar;            // [np][4]: sums over the particle's nodes of the adjoint
                             //   acceleration (3) and of the alpha derivative (1)
};
struct AdjPart {
    const double* st0;       // [np][16] state entering step n
    const double* st1;       // [np][16] state after step n (U^n, W^n, count^n)
    const double* geo;       // [np][NPV] projection sums of step n
};
// Per-instance adjoint of the particle state and scratch of the particle sweep.
struct AdjBufs {
    double* Xb;              // [np][3] adjoint of X entering the current step
    double* Ub;              // [np][3] ... of U^{n-1}
    double* Wb;              // [np][3] ... of W^{n-1}
    double* Tb;              // [np][3] ... of theta
    double* Ab;              // [np][3] ... of A (seed part; the fluid part is in Abar)
    double* rb;              // [np]    d J / d ratio
    double* alpha_b;         // [1]     d J / d alpha
    double* Abar;            // [np][4] (see AdjFluid)
    float* coef;             // [np][8]
    double* Ubar;            // [np][3] scratch: (U^n + U^{n-1}) / 2
    double* Xk;              // [K+1][np][3] sub-step positions
    double* Xs;              // [K][np][3] predicted positions
    double* F1;              // [K][np][3] collision force at Xk (C = 1: per unit C)
    double* F2;              // [K][np][3] ... at Xs
    double* Xkb;             // [np][3] adjoint of the current sub-step position
    double* Xsb;             // [np][3]
    double* v;               // [np][3] adjoint of the sub-step force sum
    double* Ubb;             // [np][3] adjoint of Ubar
    double* Wnb;             // [np][3] adjoint of W^n
};

// Particle index -> (instance, local index) for the per-particle kernels.
struct PartRef {
    int inst;
    int p;
};

__host__ __device__ inline int tile_w(const Shape& s) { return s.tw; }

}  // namespace lbmpen
