// Per-particle FP64 kernels of lbmpen: the second pass of the rigid-body
// projection (Eq. 22; the per-component finalisation is in lbm_common.cuh),
// the predictor-corrector of Algorithm 1 with the repulsive collision forces
// (Eqs. 19-21), and the rebuild of each particle's record and tile-list
// entries for the next step.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, and an FP64
// instruction occupies a sub-partition's FP64 pipe for ~64 cycles whether one
// lane or 32 are active, so the serial per-particle arithmetic runs one lane
// per (particle, vector component).  The O(N^2) pair search uses a warp per
// particle and filters pairs in FP32 (positions staged in shared memory)
// before the FP64 evaluation of the few pairs in range.
#include "lbm_common.cuh"

namespace lbmpen {

constexpr int PB = 8;         // particles per block (one per warp)
constexpr int XCHUNK = 1024;  // particle positions staged in shared memory at a time

// Extent of a particle along the unit vector (nx, ny): R for a disk; for an
// ellipse (semi-axes R = a and B = b, orientation (ec, es)) the support
// distance sqrt(a^2 (n.e)^2 + b^2 (n.e_perp)^2).  Used in place of the radius
// in Eqs. 19-20, which the paper states for disks.
__device__ __forceinline__ double extent_along(double R, double B, double ec, double es, double nx,
                                               double ny) {
    if (B == R) return R;
    const double ne = __dadd_rn(__dmul_rn(nx, ec), __dmul_rn(ny, es));
    const double np = __dsub_rn(__dmul_rn(ny, ec), __dmul_rn(nx, es));
    return sqrt(__dadd_rn(__dmul_rn(__dmul_rn(R, R), __dmul_rn(ne, ne)),
                          __dmul_rn(__dmul_rn(B, B), __dmul_rn(np, np))));
}

// Pair part of Eq. 21 on particle i at two position sets: Xk[src] (F1) and
// Xk[src] + h Ubar (F2).  The block's particles all belong to one instance;
// its positions are staged in shared memory in chunks and the lanes split
// them.  An FP32 filter with a margin of 2.5 lattice units (a sub-step moves
// a particle by |h Ubar| < 1/2) leaves only pairs near the interaction range
// for the FP64 evaluation, which follows the reference operation order.
__device__ void pair_chunk(const InstDesc& in, int i, int src, double h, int lane, const float4* xs,
                           const float4* xs2, int j0, int nj, float4 xi, float4 xi2, double cp,
                           double inv_delta, double* f1, double* f2) {
    const double* Xb = in.Xk + (long long)src * in.np * 3;
    if (cp == 0.0) return;  // cp = C / eps_p of particle i
    const float reach = xi.w + (float)in.delta + 0.01f;  // FP32 positions carry < 1e-3 error
    const float nf[3] = {(float)in.n[0], (float)in.n[1], (float)in.n[2]};
    const bool per[3] = {in.periodic[0] && in.n[0] > 1, in.periodic[1] && in.n[1] > 1,
                         in.periodic[2] && in.n[2] > 1};
    for (int jj = lane; jj < nj; jj += 32) {
        const int j = j0 + jj;
        if (j == i) continue;
        bool near[2];
        bool far = false;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1 && far) break;
            const float4 a = pass ? xi2 : xi, b = pass ? xs2[jj] : xs[jj];
            float dv[3] = {a.x - b.x, a.y - b.y, a.z - b.z};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (per[d]) dv[d] -= nf[d] * rintf(dv[d] / nf[d]);
            const float lim = reach + b.w;
            const float d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
            near[pass] = d2 <= lim * lim;
            // a predicted position lies within |h Ubar| < sqrt(3)/2 of X^n (a larger
            // step is reported as ST_DISPLACEMENT), so a pair more than 2 beyond
            // range at X^n is out of range at both position sets
            if (pass == 0) far = d2 > (lim + 2.0f) * (lim + 2.0f);
        }
        if (far) continue;
        if (!near[0] && !near[1]) continue;
        const double Bi = in.pconst[PCONST_N * i + PC_B], Bj = in.pconst[PCONST_N * j + PC_B];
        const bool ell = Bi != in.R[i] || Bj != in.R[j];
        for (int pass = 0; pass < 2; ++pass) {
            if (!near[pass]) continue;
            const double sh = pass ? h : 0.0;
            double dd[3];
            for (int d = 0; d < 3; ++d) {
                const double xi_d = Xb[3 * i + d] + sh * in.Ubar[3 * i + d];
                const double xj_d = Xb[3 * j + d] + sh * in.Ubar[3 * j + d];
                dd[d] = xi_d - xj_d;
                if (per[d]) {
                    const double half = 0.5 * in.n[d];
                    if (dd[d] > half) dd[d] -= in.n[d];
                    else if (dd[d] < -half) dd[d] += in.n[d];
                }
            }
            const double dij = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dd[0], dd[0]), __dmul_rn(dd[1], dd[1])),
                                              __dmul_rn(dd[2], dd[2])));
            double range = in.R[i] + in.R[j] + in.delta;
            if (ell && dij > 0.0) {  // ellipses (2D): extents along the line of centres
                const double nx = dd[0] / dij, ny = dd[1] / dij;
                const PRec &ri = in.prec[i], &rj = in.prec[j];
                range = extent_along(in.R[i], Bi, ri.ec, ri.es, nx, ny) +
                        extent_along(in.R[j], Bj, rj.ec, rj.es, nx, ny) + in.delta;
            }
            if (dij <= range) {
                const double sc = (range - dij) * inv_delta;
                double* f = pass ? f2 : f1;
                for (int d = 0; d < 3; ++d) f[d] += cp * dd[d] * sc * sc;
            }
        }
    }
}

// Gather the (few) lanes that found a pair into every lane.
__device__ void gather_pairs(const double* f1, const double* f2, double* F1, double* F2) {
    const unsigned act = __ballot_sync(0xffffffffu, f1[0] != 0 || f1[1] != 0 || f1[2] != 0 ||
                                                        f2[0] != 0 || f2[1] != 0 || f2[2] != 0);
    double g1[3] = {0, 0, 0}, g2[3] = {0, 0, 0};
    for (int l = 0; l < 32; ++l) {
        if (!(act & (1u << l))) continue;
        for (int d = 0; d < 3; ++d) {
            g1[d] += __shfl_sync(0xffffffffu, f1[d], l);
            g2[d] += __shfl_sync(0xffffffffu, f2[d], l);
        }
    }
    for (int d = 0; d < 3; ++d) {
        F1[d] = g1[d];
        F2[d] = g2[d];
    }
}

// Wall part of Eq. 21 (mirror images across the planes -1/2 and n - 1/2),
// component d of the force on a particle at coordinate Xi along axis d; Ri is
// the particle's extent along axis d (its radius, for a disk).
__device__ void wall_force_d(const InstDesc& in, int d, double Xi, double& F, double cw, double inv_delta,
                             double Ri) {
    if (cw == 0.0) return;  // cw = C / eps_w of the particle
    const float reach = 0.5f * (2.0f * (float)Ri + (float)in.delta) + 0.01f;
    if (in.periodic[d] || in.n[d] <= 1) return;
    const float xf = (float)Xi;  // skip walls farther than (2R + delta)/2
    if (xf + 0.5f > reach && (float)in.n[d] - 0.5f - xf > reach) return;
    const double walls[2] = {-0.5, in.n[d] - 0.5};
    for (int face = 0; face < 2; ++face) {
        const double Xim = 2.0 * walls[face] - Xi;
        const double diff = Xi - Xim;
        const double dprime = fabs(diff);
        const double range = 2.0 * Ri + in.delta;
        if (dprime <= range) {
            const double sc = (range - dprime) * inv_delta;
            F += cw * diff * sc * sc;
        }
    }
}

// Tiles along one axis that hold nodes of the node interval [X-R-1, X+R+1]:
// tiles a0 .. a0+na-1 and b0 .. b0+nb-1 (disjoint).  On a periodic axis the
// interval may wrap; it is split at the face before mapping to tiles, since
// the last tile of a ragged axis does not continue into the first one.
struct AxisTiles {
    int a0, na, b0, nb;
};

__device__ AxisTiles axis_tiles_f(float X, float R, int n, int T, int ntile, int periodic) {
    int lo = (int)floorf(X - R) - 1, hi = (int)floorf(X + R) + 1;
    AxisTiles t{0, 1, 0, 0};
    if (!periodic) {
        lo = max(lo, 0);
        hi = max(min(hi, n - 1), lo);
        t.a0 = lo / T;
        t.na = hi / T - t.a0 + 1;
        return t;
    }
    if (hi - lo + 1 >= n) {
        t.a0 = 0;
        t.na = ntile;
        return t;
    }
    int alo, bhi;
    if (lo < 0) {
        alo = lo + n;
        bhi = hi;
    } else if (hi >= n) {
        alo = lo;
        bhi = hi - n;
    } else {
        t.a0 = lo / T;
        t.na = hi / T - t.a0 + 1;
        return t;
    }
    const int ta0 = alo / T, tb1 = bhi / T;
    if (tb1 >= ta0) {  // the two pieces share a tile: take the whole axis
        t.a0 = 0;
        t.na = ntile;
        return t;
    }
    t.a0 = ta0;
    t.na = ntile - ta0;
    t.b0 = 0;
    t.nb = tb1 + 1;
    return t;
}

__device__ __forceinline__ int axis_tile(const AxisTiles& t, int i) {
    return i < t.na ? t.a0 + i : t.b0 + (i - t.na);
}

// Component d of a particle's record for the next fluid step: the reference
// node floor(X), the offset from it, the acceleration term of the penalty
// force, and the tiles of the bounding box [X - R - 1, X + R + 1] along d (its
// one-node margin covers the float rounding).
struct RecComp {
    int ref;
    float frac, a;
    AxisTiles t;
};

__device__ __forceinline__ RecComp record_component(const InstDesc& in, int d, int D, const Shape& sh, double X,
                                                    double A, float Rf, float gfac) {
    const int T = d == 0 ? sh.tw : (d == 1 ? sh.ty : sh.tz);
    RecComp r;
    r.ref = d < D ? __double2int_rd(X) : 0;
    r.frac = (float)(X - (double)r.ref);
    r.a = fmaf(gfac, in.ggrav[d], (float)A);
    r.t = d >= D ? AxisTiles{0, 1, 0, 0}
                 : axis_tiles_f((float)r.ref + r.frac, Rf, in.n[d], T, in.ntile[d], in.periodic[d]);
    return r;
}

// The size and shape fields of particle p's record (host-computed, RecConst)
// and its tile count (nt tiles of the bounding box).
__device__ __forceinline__ void record_radius(const InstDesc& in, PRec& pr, const RecConst& rc, int nt) {
    pr.R2 = rc.R2;
    pr.R2lo = rc.R2lo;
    pr.R2hi = rc.R2hi;
    pr.ntiles = nt;
    pr.shape = rc.shape;
    pr.pad = 0;
    pr.b2 = rc.b2;
    pr.ia2 = rc.ia2;
    pr.ib2 = rc.ib2;
    pr.qlo = rc.qlo;
    pr.qhi = rc.qhi;
    pr.pad2[0] = pr.pad2[1] = 0.f;
    if (nt > in.maxk) atomicOr(in.status, ST_CAPACITY);
}

// Orientation fields of a record: cos and sin of theta (the z component of
// the orientation in 2D) for an ellipse; (1, 0) otherwise.
__device__ __forceinline__ void record_orientation(PRec& pr, bool ellipse, double theta) {
    double c = 1.0, s = 0.0;
    if (ellipse) sincos(theta, &s, &c);
    pr.ec = c;
    pr.es = s;
    pr.fc = (float)c;
    pr.fs = (float)s;
}

// Record of particle p from its state (X, A, theta) and constants (R, B,
// 1 - rho_f/rho_s), with the tiles of its bounding box (slots k enumerate them
// x-fastest; no tile is listed twice).  One thread.
__device__ void make_record_from(const InstDesc& in, int p, int D, const Shape& sh, AxisTiles* at,
                                 const double* Xp, const double* Ap, double R, double B, double theta,
                                 float gfac) {
    PRec pr;
    int nt = 1;
    for (int d = 0; d < 3; ++d) {
        const RecComp r = record_component(in, d, D, sh, Xp[d], Ap[d], (float)R, gfac);
        pr.X[d] = Xp[d];
        pr.ref[d] = r.ref;
        pr.frac[d] = r.frac;
        pr.a[d] = r.a;
        at[d] = r.t;
        nt *= r.t.na + r.t.nb;
    }
    record_radius(in, pr, in.rconst[p], nt);
    record_orientation(pr, B != R, theta);
    in.prec_out[p] = pr;
}

__device__ void make_record(const InstDesc& in, int p, int D, const Shape& sh, AxisTiles* at) {
    double X[3], A[3];
    for (int d = 0; d < 3; ++d) {
        X[d] = in.X[3 * p + d];
        A[d] = in.A[3 * p + d];
    }
    make_record_from(in, p, D, sh, at, X, A, in.pconst[PCONST_N * p + PC_R],
                     in.pconst[PCONST_N * p + PC_B], in.theta[3 * p + 2],
                     (float)in.pconst[PCONST_N * p + PC_GFAC]);
}

// List entries of particle p in the tiles of its bounding box (lanes share),
// from its record for the next step (prec_out[p]): the entry p << KBITS | k
// and, in the same slot, the 64-byte candidate record the TMA kernel copies.
__device__ void append_tiles(const InstDesc& in, int p, const AxisTiles* at, int lpar, int lane,
                             int nl) {
    const int cnt[3] = {at[0].na + at[0].nb, at[1].na + at[1].nb, at[2].na + at[2].nb};
    const int nt = cnt[0] * cnt[1] * cnt[2];
    if (lane >= nt) return;
    const PRec& pr = in.prec_out[p];
    Cand cd;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        cd.ref[d] = pr.ref[d];
        cd.frac[d] = pr.frac[d];
        cd.a[d] = pr.a[d];

    }
    cd.R2lo = pr.R2lo;
    cd.R2hi = pr.R2hi;
    cd.p = p;
    const int2 bi = in.boxinfo[p];
    cd.boff = bi.x;
    cd.bh = bi.y;
    cd.shape = pr.shape;
    Cand* rec = static_cast<Cand*>(in.list_rec[lpar]);
    for (int k = lane; k < nt && k < in.maxk; k += nl) {
        const int kx = k % cnt[0], ky = (k / cnt[0]) % cnt[1], kz = k / (cnt[0] * cnt[1]);
        const int tc[3] = {axis_tile(at[0], kx), axis_tile(at[1], ky), axis_tile(at[2], kz)};
        const int local = (tc[2] * in.ntile[1] + tc[1]) * in.ntile[0] + tc[0];
        const int pos = atomicAdd(&in.list_cnt[lpar][local], 1);
        if (pos < LIST_CAP) {
            // the slot is informational (a particle may cover more than MAXK
            // tiles): only its low KBITS bits go into the entry, below p
            in.list_ent[lpar][(long long)local * LIST_CAP + pos] = ((uint32_t)p << KBITS) | (uint32_t)(k & (MAXK - 1));
            cd.k = k;
            rec[(long long)local * LIST_CAP + pos] = cd;
        } else {
            atomicOr(in.status, ST_CAPACITY);
        }
    }
}

// Algorithm 1 for particle i, component d (one lane per component; the lanes
// of particle slot sl are sl + PB * d, and lanes with valid = false take part
// in the shuffles only): wall forces, the corrected position, and on the last
// sub-step A^{n+1}, theta^{n+1}, U^{n-1} <- U^n and the record for the next
// step.  Each lane evaluates the expressions of a serial loop over d.
// The operands of update_lane, loaded in one batch before the pair search so
// that their latency overlaps it.
struct LaneIn {
    double X0, Ub, Wn, Un, Wo, Th, invrhos, cw, idl, Ri, Bi, gfac, invc, Acor, ec, es;
    int cnt;
    RecConst rc;
};

__device__ __forceinline__ LaneIn load_lane(const InstDesc& in, int i, int d, bool valid, int src, int first) {
    if (!valid) {  // in-range operands for the shuffle-only lanes
        i = 0;
        d = 0;
    }
    const long long j = 3LL * i + d;
    LaneIn L;
    L.X0 = in.Xk[(long long)src * in.np * 3 + j];
    L.Ub = in.Ubar[j];
    L.Wn = in.Wn[j];
    L.Un = in.Un[j];
    L.Wo = in.W[j];
    L.Th = in.theta[j];
    const double* pc = in.pconst + PCONST_N * i;
    L.invrhos = pc[PC_INVRHOS];
    L.cw = pc[PC_CWALL];
    L.idl = pc[PC_INVDELTA];
    L.Ri = pc[PC_R];
    L.Bi = pc[PC_B];
    L.gfac = pc[PC_GFAC];
    L.invc = in.invc[i];
    L.cnt = in.count[i];
    L.Acor = first ? 0.0 : in.Acor[j];
    L.ec = in.prec[i].ec;  // orientation theta^n of this step's record
    L.es = in.prec[i].es;
    L.rc = in.rconst[i];
    return L;
}

__device__ void update_lane(const InstDesc& in, int i, int d, int sl, bool valid, const double* F1in,
                            const double* F2in, int src, double h, int first, int last, int D,
                            const Shape& sh, AxisTiles* at, const LaneIn& L) {
    if (!valid) {  // in-range operands for the shuffle-only lanes; nothing is stored
        i = 0;
        d = 0;
    }
    const int dst = src ^ 1;
    const long long j = 3LL * i + d;
    const double X0 = L.X0, Ub = L.Ub, Wn = L.Wn, Un = L.Un, Wo = L.Wo, Th = L.Th;
    double F1 = F1in[d], F2 = F2in[d];
    const double invrhos = L.invrhos, cw = L.cw, idl = L.idl, Ri = L.Ri, Bi = L.Bi, gfac = L.gfac;
    const double invc = L.invc;
    const int cnt = L.cnt;
    const double invM = invrhos * invc;  // 1 / (rho_s n)
    const double Xst = fma(h, Ub, X0);
    // extent along axis d: the radius, or for an ellipse at theta^n (this
    // step's record) its support distance normal to the walls of axis d
    double Rd = Ri;
    if (Bi != Ri && d < 2)
        Rd = d == 0 ? extent_along(Ri, Bi, L.ec, L.es, 1.0, 0.0) : extent_along(Ri, Bi, L.ec, L.es, 0.0, 1.0);
    wall_force_d(in, d, X0, F1, cw, idl, Rd);
    wall_force_d(in, d, Xst, F2, cw, idl, Rd);
    const double c = 0.25 * h * h * invM;  // (1 / 2M) h^2 / 2
    const double cor = c * (F1 + F2);      // this sub-step's correction
    const double Xn = Xst + cor;
    // A^{n+1} = 2 (X^{n+1} - X^n - Ubar) is twice the sum of the corrections;
    // summed directly, since the difference of positions cancels catastrophically
    const double acc = first ? cor : L.Acor + cor;
    const float Rf = (float)Ri;
    if (!last) {
        if (valid) {
            in.Acor[j] = acc;
            in.Xk[(long long)dst * in.np * 3 + j] = Xn;
            float* xf = in.Xf + ((long long)dst * in.np + i) * 4;
            float* xsf = in.Xsf + ((long long)dst * in.np + i) * 4;
            xf[d] = (float)Xn;
            xsf[d] = (float)fma(h, Ub, Xn);
            if (d == 0) {
                xf[3] = Rf;
                xsf[3] = Rf;
            }
        }
        return;
    }
    bool left = false;
    const double An = 2.0 * acc;
    double xn = Xn;
    if (d < D) {
        if (in.periodic[d]) {
            if (xn >= in.n[d]) xn -= in.n[d];
            else if (xn < 0.0) xn += in.n[d];
        } else if (xn < -0.5 || xn > in.n[d] - 0.5) {
            left = true;
        }
    }
    const double Tn = Th + 0.5 * (Wn + Wo);
    if (valid) {
        in.A[j] = An;
        in.X[j] = xn;
        in.theta[j] = Tn;
        in.U[j] = Un;
        in.W[j] = Wn;
        if (left) atomicOr(in.status, ST_PARTICLE);
        if (in.rec_state) {  // adjoint recording: the state this step hands to the next
            double* r = in.rec_state + 16LL * i;
            r[d] = xn;
            r[3 + d] = Un;
            r[6 + d] = Wn;
            r[9 + d] = Tn;
            r[12 + d] = An;
            if (d == 0) r[15] = (double)cnt;
        }
    }
    const RecComp r = record_component(in, d, D, sh, xn, An, Rf, (float)gfac);
    const int ct = r.t.na + r.t.nb;
    const int nt = __shfl_sync(0xffffffffu, ct, sl) * __shfl_sync(0xffffffffu, ct, sl + PB) *
                   __shfl_sync(0xffffffffu, ct, sl + 2 * PB);
    if (valid) {
        PRec& pr = in.prec_out[i];
        pr.X[d] = xn;
        pr.ref[d] = r.ref;
        pr.frac[d] = r.frac;
        pr.a[d] = r.a;
        at[d] = r.t;
        if (d == 0) record_radius(in, pr, L.rc, nt);
        if (d == 2) record_orientation(pr, Bi != Ri, Tn);
    }
}

// ------------------------------------------------------------- the kernel --
// Default bound on a barrier wait (2 s); a context may set another
// (lbm_set_particle_wait_limit), 0 included: then a block that does not find
// the barrier open on its first look gives up at once.
constexpr unsigned long long PWAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Barrier over all blocks of the particle kernel (launched only when they are
// all resident).  Bounded: after limit_ns it records a timeout and returns
// false, and the kernel stops.  Every block arrives before it waits, so the
// last arrival always resets the count, timeouts included.
__device__ bool grid_sync(GridBar* gb, int* status, unsigned long long limit_ns) {
    if (gridDim.x == 1) {  // one block: the block barrier is the grid barrier
        __syncthreads();
        return true;
    }
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &gb->gen;
        const unsigned g = *vgen;  // generation before this block arrives
        __threadfence();
        if (atomicAdd(&gb->count, 1) == gridDim.x - 1) {
            gb->count = 0;
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (*vgen == g) {
                if (gtimer() - t0 >= limit_ns) {
                    ok = 0;
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// The totals of Eq. 22 of every particle from its velocity box, one block of
// BS_THREADS per particle, launched between the fluid kernel and the particle
// kernel: the threads take the box's entries (3D: only the rows that can reach
// the sphere), turn every filled one (the nodes the particle owned in this
// step's fluid kernel) into exact integer sums, and mark it empty again for
// the next step.  The warps' totals are exact (integer reductions; 64-bit
// sums by limbs) and so is their sum, so the totals do not depend on the order.
constexpr int BS_THREADS = 128;  // 4 blocks per SM: 500 particles in one wave
constexpr int BS_PER = 8;  // entries of a thread in flight at a time

template <int D>
__device__ __forceinline__ void box_block_sums(const InstDesc& in, int p, long long (*red)[NPV]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int2 bi = in.boxinfo[p];
    const int H = bi.y, side = 2 * H + 1;
    const int nent = D == 2 ? side * side : side * side * side;  // < 2^31 for R <= 40
    const int hmax = (H - 1) * (H - 1);  // owned nodes have |d| <= R + 1 <= H - 1
    int icnt = 0, id[3] = {0, 0, 0}, idd[6] = {0, 0, 0, 0, 0, 0};
    long long su[3] = {0, 0, 0}, sl[3] = {0, 0, 0};
    const float nanv = __int_as_float(0x7fffffff);
    for (int e0 = 0; e0 < nent; e0 += BS_THREADS * BS_PER) {
        float4 u[BS_PER];
        int dd[BS_PER][3];
#pragma unroll
        for (int j = 0; j < BS_PER; ++j) {
            const int e = e0 + tid + BS_THREADS * j;
            const int dx = e % side - H, dy = (e / side) % side - H, dz = D == 3 ? e / (side * side) - H : 0;
            dd[j][0] = dx;
            dd[j][1] = dy;
            dd[j][2] = dz;
            u[j] = make_float4(nanv, nanv, nanv, 0.f);
            if (e < nent && (D == 2 || dy * dy + dz * dz <= hmax)) {
                if (D == 2) {
                    const float2 t = __ldcg(reinterpret_cast<const float2*>(in.ubox) + bi.x + e);
                    u[j].x = t.x;
                    u[j].y = t.y;
                } else {
                    u[j] = __ldcg(reinterpret_cast<const float4*>(in.ubox) + bi.x + e);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < BS_PER; ++j) {
            if (!(u[j].x == u[j].x)) continue;  // empty (NaN)
            const int dx = dd[j][0], dy = dd[j][1], dz = dd[j][2];
            const long long ux[3] = {to_fx32(u[j].x), to_fx32(u[j].y), D == 3 ? to_fx32(u[j].z) : 0};
            icnt += 1;
            id[0] += dx; id[1] += dy; id[2] += dz;
            idd[0] += dx * dx; idd[1] += dy * dy; idd[2] += dz * dz;
            idd[3] += dx * dy; idd[4] += dx * dz; idd[5] += dy * dz;
            su[0] += ux[0]; su[1] += ux[1]; su[2] += ux[2];
            sl[2] += (long long)dx * ux[1] - (long long)dy * ux[0];
            if (D == 3) {
                sl[0] += (long long)dy * ux[2] - (long long)dz * ux[1];
                sl[1] += (long long)dz * ux[0] - (long long)dx * ux[2];
            }
            const long long e = bi.x + (long long)(e0 + tid + BS_THREADS * j);
            if (D == 2) reinterpret_cast<float2*>(in.ubox)[e] = make_float2(nanv, nanv);
            else reinterpret_cast<float4*>(in.ubox)[e] = make_float4(nanv, nanv, nanv, 0.f);
        }
    }
    long long v[NPV];
    v[0] = __reduce_add_sync(0xffffffffu, icnt);
#pragma unroll
    for (int k = 0; k < 3; ++k) v[1 + k] = k < D ? (long long)__reduce_add_sync(0xffffffffu, id[k]) : 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool need = D == 3 || k == 0 || k == 1 || k == 3;
        v[4 + k] = need ? (long long)__reduce_add_sync(0xffffffffu, idd[k]) : 0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[10 + k] = k < D ? warp_sum_fx(su[k]) : 0;
        v[13 + k] = (D == 3 || k == 2) ? warp_sum_fx(sl[k]) : 0;
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NPV; ++k) red[warp][k] = v[k];
}

__global__ void __launch_bounds__(BS_THREADS, 4) k_box_sums(const InstDesc* __restrict__ insts,
                                                       const PartRef* __restrict__ refs, int D) {
    __shared__ long long red[BS_THREADS / 32][NPV];
    __shared__ long long tot[NPV];
    const PartRef r = refs[blockIdx.x];
    if (r.inst < 0) return;  // padding entry (block-uniform)
    const InstDesc& in = insts[r.inst];
    if (threadIdx.x >= BS_THREADS - 4) {  // warm L1 with what the second pass reads
        const int k = threadIdx.x - (BS_THREADS - 4);
        const char* a = k < 2 ? reinterpret_cast<const char*>(in.prec + r.p) + 128 * k
                              : (k == 2 ? reinterpret_cast<const char*>(in.U + 3 * r.p)
                                        : reinterpret_cast<const char*>(in.pconst + PCONST_N * r.p));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
    if (D == 2) box_block_sums<2>(in, r.p, red);
    else box_block_sums<3>(in, r.p, red);
    __syncthreads();
    if (threadIdx.x < NPV) {
        long long t = 0;
        for (int w = 0; w < BS_THREADS / 32; ++w) t += red[w][threadIdx.x];
        in.btot[(long long)r.p * NPV + threadIdx.x] = t;
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    // the second pass of Eq. 22 for this particle: translation on warp 0,
    // rotation on warp 1, one lane per component; the kernel boundary after
    // it is the grid-wide barrier Algorithm 1 needs (every particle's U^n)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < 3) {
        if (warp == 0) {
            if (D == 2) finalize_translation<2>(in, r.p, tot, lane);
            else finalize_translation<3>(in, r.p, tot, lane);
        } else if (warp == 1) {
            if (D == 2) finalize_rotation<2>(in, r.p, tot, lane);
            else finalize_rotation<3>(in, r.p, tot, lane);
        }
    }
}

// Phase k (1..K): sub-step k of Algorithm 1, positions Xk[src] -> Xk[src ^ 1];
// the block's warps find the pair forces (one particle each), one thread per
// particle does the FP64 update.
__device__ void phase_substep(const InstDesc& in, const PartRef* refs, int ntotal, int D, int gp0,
                              int src, int K, int first, int last, const Shape& sh, float4* xs, float4* xs2,
                              double (*sF)[6], AxisTiles (*sAT)[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double h = in.hK;
    const int gp = gp0 + warp;
    const bool mine = warp < PB && gp < ntotal && refs[gp].inst >= 0;
    const int i = mine ? refs[gp].p : 0;
    double f1[3] = {0, 0, 0}, f2[3] = {0, 0, 0};
    const float4* Xfb = reinterpret_cast<const float4*>(in.Xf) + (long long)src * in.np;
    const float4* Xsb = reinterpret_cast<const float4*>(in.Xsf) + (long long)src * in.np;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f), xi2 = xi;
    double cp = 0.0, idl = 0.0;
    if (mine) {  // issued before the staging barrier, so the loads overlap it
        xi = Xfb[i];
        xi2 = Xsb[i];
        cp = in.pconst[PCONST_N * i + PC_CPAIR];
        idl = in.pconst[PCONST_N * i + PC_INVDELTA];
    }
    // warp 0: the operands of the update (one lane per particle component)
    const int usl = lane & (PB - 1), ud = lane / PB;
    const bool uvalid = warp == 0 && ud < 3 && gp0 + usl < ntotal && refs[gp0 + usl].inst >= 0;
    LaneIn li;
    if (warp == 0) li = load_lane(in, uvalid ? refs[gp0 + usl].p : 0, ud, uvalid, src, first);
    for (int j0 = 0; j0 < in.np; j0 += XCHUNK) {
        const int nj = min(XCHUNK, in.np - j0);
        // every load of the chunk in flight at once, then the shared stores
        constexpr int PER = XCHUNK / 256;  // blockDim.x == 256
        float4 ra[PER], rb[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + 256 * u;
            if (k < nj) {
                ra[u] = Xfb[j0 + k];
                rb[u] = Xsb[j0 + k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k = threadIdx.x + 256 * u;
            if (k < nj) {
                xs[k] = ra[u];
                xs2[k] = rb[u];
            }
        }
        __syncthreads();
        if (mine) pair_chunk(in, i, src, h, lane, xs, xs2, j0, nj, xi, xi2, cp, idl, f1, f2);
    }
    if (mine) {
        double F1[3], F2[3];
        gather_pairs(f1, f2, F1, F2);
        if (lane == 0)
            for (int d = 0; d < 3; ++d) {
                sF[warp][d] = F1[d];
                sF[warp][3 + d] = F2[d];
            }
    }
    __syncthreads();
    if (warp == 0)  // one lane per (particle, component)
        update_lane(in, uvalid ? refs[gp0 + usl].p : 0, ud, usl, uvalid, sF[usl], sF[usl] + 3, src, h, first, last,
                    D, sh, sAT[usl], li);
}

// Particle part of one time step for the block's 8 particles (one instance),
// phases first..last, phase k = sub-step k of Algorithm 1 (the projection of
// Eq. 22 ran in k_box_sums); after the last sub-step the warps append their
// particle to the next step's tile lists.  With more than one phase (K > 1)
// the blocks meet at grid barriers between phases (the launch guarantees they
// are all resident); with K = 1 there is no barrier.
__global__ void __launch_bounds__(256, 1) k_particles(const InstDesc* __restrict__ insts,
                                                   const PartRef* __restrict__ refs, int ntotal,
                                                   int D, int K, int first, int last, int lpar,
                                                   Shape sh, GridBar* gb, unsigned long long wait_ns) {
    __shared__ double sF[PB][6];
    __shared__ AxisTiles sAT[PB][3];
    __shared__ float4 xs[XCHUNK];
    __shared__ float4 xs2[XCHUNK];
    const int gp0 = blockIdx.x * PB;
    __shared__ __align__(16) InstDesc sdesc;
    stage_desc(&sdesc, insts[refs[gp0].inst]);  // blocks never straddle instances
    const InstDesc& in = sdesc;
    for (int ph = first; ph <= last; ++ph) {
        if (ph > first && !grid_sync(gb, in.status, wait_ns)) return;
        phase_substep(in, refs, ntotal, D, gp0, (ph - 1) & 1, K, ph == 1, ph == K, sh, xs, xs2, sF, sAT);
    }
    if (last == K) {
        __syncthreads();  // records and tile ranges of the block's particles are ready
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int gp = gp0 + warp;
        if (warp < PB && gp < ntotal && refs[gp].inst >= 0)
            append_tiles(in, refs[gp].p, sAT[warp], lpar, lane, 32);
    }
}

// Publish every particle from its current state (after creation, particle
// insertion, a shape change or a state load).  Lists must be zeroed first.
__global__ void k_publish(const InstDesc* __restrict__ insts, const PartRef* __restrict__ refs,
                          int ntotal, int D, int lpar, Shape sh) {
    const int gp = blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= ntotal) return;
    const PartRef r = refs[gp];
    if (r.inst < 0) return;
    AxisTiles at[3];
    make_record(insts[r.inst], r.p, D, sh, at);
    append_tiles(insts[r.inst], r.p, at, lpar, 0, 1);
}

int particle_blocks_resident(int num_sms) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_particles, 256, 0) != cudaSuccess) return 0;
    return nb * num_sms;
}

// The particle part of a step: one launch with grid barriers when all blocks
// fit on the GPU at once, else one launch per phase.
cudaError_t launch_particles(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int K,
                             int lpar, const Shape& sh, GridBar* gb, bool fused, cudaStream_t st,
                             long long wait_ns) {
    const int blocks = (ntotal + PB - 1) / PB;
    const unsigned long long lim = wait_ns < 0 ? PWAIT_NS : (unsigned long long)wait_ns;
    if (fused || K == 1) {
        k_particles<<<blocks, 256, 0, st>>>(insts, refs, ntotal, D, K, 1, K, lpar, sh, gb, lim);
        return cudaGetLastError();
    }
    for (int ph = 1; ph <= K; ++ph)
        k_particles<<<blocks, 256, 0, st>>>(insts, refs, ntotal, D, K, ph, ph, lpar, sh, gb, lim);
    return cudaGetLastError();
}

cudaError_t launch_box_sums(const InstDesc* insts, const PartRef* refs, int ntotal, int D, cudaStream_t st) {
    k_box_sums<<<ntotal, BS_THREADS, 0, st>>>(insts, refs, D);
    return cudaGetLastError();
}

cudaError_t launch_publish(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int lpar,
                           const Shape& sh, cudaStream_t st) {
    k_publish<<<(ntotal + 63) / 64, 64, 0, st>>>(insts, refs, ntotal, D, lpar, sh);
    return cudaGetLastError();
}

}  // namespace lbmpen
