// Discrete adjoint of the penalized LBM step (reverse mode, hand-written).
//
// The forward step n maps the post-collision populations g^{n-1} and the
// particle state P^n = (X^n, U^{n-1}, W^{n-1}, theta^n, A^n) to g^n and P^{n+1}
// (Eqs. 9-17, 22 and Algorithm 1).  With the solid indicator held fixed (it
// is piecewise constant in X, Eq. 9, so its derivative vanishes almost
// everywhere) every stage is differentiable, and the backward sweep applies
// the transposed Jacobians in reverse order:
//
//   k_adj_particles  Algorithm 1 (sub-steps with the collision forces of
//                    Eqs. 19-21, A^{n+1}, theta^{n+1}) and the projection of
//                    Eq. 22 transposed, FP64, one block per instance;
//   k_adj_fluid      the fused collide (Eqs. 10, 13-17) transposed per node
//                    and streaming transposed: the adjoint of f^{n+1}_q at
//                    x + c_q is pulled to x (or the opposite population at x
//                    where x + c_q lies beyond a wall), FP32, one block per tile.
//
// The adjoint fluid kernel reads the populations entering step n (recorded
// by the recomputation of a checkpointed segment) and recomputes the node's
// forward state (u, p, feq, Pi_neq) from them; it writes the adjoint of the
// pre-collision populations of step n and adds, per particle, the sums of the
// adjoint acceleration and of the alpha derivative over the particle's nodes.
#include "lbm_common.cuh"

namespace lbmpen {

namespace {

// ----------------------------------------------------------- node adjoint --
// One node: given the pre-collision populations f (q = 1..Q-1), the local
// acceleration a and lam = d J / d f*, return fb = d J / d f, ab = d J / d a
// and alb = d J / d alpha.  ubp is the part of d J / d u that comes from the
// rigid-body projection (zero on fluid nodes).  The forward map is the one
// of collide():
//   g_q = keep f_q + omk A_q E_q + fA_q G_q + chi S_q,
//   E_q = p - u.u/2 + c.u + 1.5 (c.u)^2,   G_q = c.a (1 + 3 c.u) - u.a,
//   S_q = 1.5 alpha A_q (c_q^T Pi c_q - tr(Pi)/3),  Pi = sum_q (f_q - A_q E_q) c_q c_q^T,
//   u = m + a/2,  p = (s - kuu u.u) / sum A.
template <int Q>
__device__ __forceinline__ void node_adjoint(const float* f, const float* a, const float* lam, bool solid,
                                             bool any_solid, const float* ubp, const CollK& k, float* fb,
                                             float* ab, float* alb) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int QS = Q - 1;
    constexpr float inv_sa = (float)(1.0 / L::SUMA);
    constexpr float kuu = (float)(1.5 - 0.5 * L::SUMA);
    float s, m[3];
    moments<Q>(f, s, m);
    float u[3];
    u[0] = fmaf(0.5f, a[0], m[0]);
    u[1] = fmaf(0.5f, a[1], m[1]);
    u[2] = D == 3 ? fmaf(0.5f, a[2], m[2]) : 0.f;
    const float uu = fmaf(u[2], u[2], fmaf(u[1], u[1], u[0] * u[0]));
    const float p = fmaf(-kuu, uu, s) * inv_sa;
    const float base = fmaf(-0.5f, uu, p);

    float ub[3] = {ubp[0], ubp[1], ubp[2]};
    float ax[3] = {0.f, 0.f, 0.f};
    float Eb[QS], Gb[QS];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int cls = (Q == 9 ? q >= 5 : q >= 7) ? 1 : 0;
        fb[q - 1] = k.keep * lam[q - 1];
        Eb[q - 1] = k.omk * k.A[cls] * lam[q - 1];
        Gb[q - 1] = k.fA[cls] * lam[q - 1];
    }
    *alb = 0.f;
    if (any_solid) {  // warp-uniform: the penalty terms of the solid lanes
        float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // Pi_neq: xx yy zz xy xz yz
        float Pb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // its adjoint
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const float cx = (float)L::c(q, 0), cy = (float)L::c(q, 1), cz = (float)L::c(q, 2);
            const float cu = cx * u[0] + cy * u[1] + cz * u[2];
            const float fn = f[q - 1] - L::A(q) * fmaf(1.5f * cu, cu, base + cu);
            P[0] += cx * cx * fn;
            P[1] += cy * cy * fn;
            P[2] += cz * cz * fn;
            P[3] += cx * cy * fn;
            P[4] += cx * cz * fn;
            P[5] += cy * cz * fn;
            const float wq = solid ? 1.5f * k.alpha * L::A(q) * lam[q - 1] : 0.f;
            Pb[0] += wq * (cx * cx - (1.0f / 3.0f));
            Pb[1] += wq * (cy * cy - (1.0f / 3.0f));
            Pb[2] += wq * (cz * cz - (1.0f / 3.0f));
            Pb[3] += wq * cx * cy;
            Pb[4] += wq * cx * cz;
            Pb[5] += wq * cy * cz;
        }
        const float trP = (P[0] + P[1] + P[2]) * (1.0f / 3.0f);
        float al = 0.f;
#pragma unroll
        for (int q = 1; q < Q; ++q) {
            const float cx = (float)L::c(q, 0), cy = (float)L::c(q, 1), cz = (float)L::c(q, 2);
            const float pcc = cx * cx * P[0] + cy * cy * P[1] + cz * cz * P[2] +
                              2.0f * (cx * cy * P[3] + cx * cz * P[4] + cy * cz * P[5]);
            al = fmaf(solid ? lam[q - 1] * 1.5f * L::A(q) : 0.f, pcc - trP, al);
            const float nu = cx * cx * Pb[0] + cy * cy * Pb[1] + cz * cz * Pb[2] +
                             2.0f * (cx * cy * Pb[3] + cx * cz * Pb[4] + cy * cz * Pb[5]);
            fb[q - 1] += nu;
            Eb[q - 1] -= L::A(q) * nu;
        }
        *alb = al;
    }
    float bb = 0.f, uab = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const float cx = (float)L::c(q, 0), cy = (float)L::c(q, 1), cz = (float)L::c(q, 2);
        const float cu = cx * u[0] + cy * u[1] + cz * u[2];
        const float ca = cx * a[0] + cy * a[1] + cz * a[2];
        const float t = fmaf(3.0f, cu, 1.0f);
        bb += Eb[q - 1];
        const float cub = fmaf(Eb[q - 1], t, 3.0f * ca * Gb[q - 1]);
        const float cab = Gb[q - 1] * t;
        uab -= Gb[q - 1];
        ub[0] = fmaf(cub, cx, ub[0]);
        ub[1] = fmaf(cub, cy, ub[1]);
        ub[2] = fmaf(cub, cz, ub[2]);
        ax[0] = fmaf(cab, cx, ax[0]);
        ax[1] = fmaf(cab, cy, ax[1]);
        ax[2] = fmaf(cab, cz, ax[2]);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ub[d] = fmaf(uab, a[d], ub[d]);
        ax[d] = fmaf(uab, u[d], ax[d]);
    }
    // base = p - u.u/2, p = (s - kuu u.u) / sum A
    const float sb = bb * inv_sa;
    const float uub = -0.5f * bb - kuu * sb;
#pragma unroll
    for (int d = 0; d < 3; ++d) ub[d] = fmaf(2.0f * uub, u[d], ub[d]);
    if (D == 2) ub[2] = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) ab[d] = fmaf(0.5f, ub[d], ax[d]);
    // u = m + a/2 with m = sum_q f_q c_q, s = sum_q f_q
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const float cx = (float)L::c(q, 0), cy = (float)L::c(q, 1), cz = (float)L::c(q, 2);
        fb[q - 1] += sb + cx * ub[0] + cy * ub[1] + cz * ub[2];
    }
}

// Pre-collision population q at node (x, y, z) of step n: pull streaming
// from the recorded populations, with bounce-back and the wall term where
// x - c_q lies beyond a wall (the first such axis names the wall, as in the
// forward kernels).  Selects instead of branches, so that the lanes of a warp
// on a face stay together.
template <int Q, class S, int q>
__device__ __forceinline__ float pull_pre_any(const InstDesc& in, const S* __restrict__ fin, int x, int y, int z,
                                              int qs) {
    using L = Lat<Q>;
    constexpr int c[3] = {L::c(q, 0), L::c(q, 1), L::c(q, 2)};
    int src[3] = {x - c[0], y - c[1], z - c[2]};
    int axis = -1, face = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (c[d] == 0) continue;
        const bool out = src[d] < 0 || src[d] >= in.n[d];
        if (out && in.periodic[d]) src[d] += src[d] < 0 ? in.n[d] : -in.n[d];
        else if (out && axis < 0) {
            axis = d;
            face = src[d] < 0 ? 0 : 1;
        }
    }
    const int node = (z * in.n[1] + y) * in.pitch + x;
    const int off = axis >= 0 ? (L::opp(q) - 1) * qs + node
                              : (q - 1) * qs + (src[2] * in.n[1] + src[1]) * in.pitch + src[0];
    const float v = VecIO<S, 1 + (sizeof(S) == 2)>::load1(fin + off, in.s_load);
    return axis >= 0 ? v + in.wterm[axis][face][q] : v;
}

// Transposed streaming: the adjoint of f*_q at x is the adjoint of f_q at
// x + c_q (wrapped on periodic axes), or of f_opp(q) at x when x + c_q lies
// beyond a wall (the population bounced back at x).
template <int Q, int q>
__device__ __forceinline__ float pull_lam_any(const InstDesc& in, const float* __restrict__ lam, int x, int y, int z,
                                              int qs) {
    using L = Lat<Q>;
    constexpr int c[3] = {L::c(q, 0), L::c(q, 1), L::c(q, 2)};
    int dst[3] = {x + c[0], y + c[1], z + c[2]};
    bool wall = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (c[d] == 0) continue;
        const bool out = dst[d] < 0 || dst[d] >= in.n[d];
        if (out && in.periodic[d]) dst[d] += dst[d] < 0 ? in.n[d] : -in.n[d];
        else if (out) wall = true;
    }
    const int node = (z * in.n[1] + y) * in.pitch + x;
    const int off = wall ? (L::opp(q) - 1) * qs + node : (q - 1) * qs + (dst[2] * in.n[1] + dst[1]) * in.pitch + dst[0];
    return __ldg(lam + off);
}

template <int Q, class S, int q>
struct PullAll {
    static __device__ __forceinline__ void pre(const InstDesc& in, const S* fin, int x, int y, int z, int qs,
                                               float* f) {
        f[q - 1] = pull_pre_any<Q, S, q>(in, fin, x, y, z, qs);
        PullAll<Q, S, q + 1>::pre(in, fin, x, y, z, qs, f);
    }
    static __device__ __forceinline__ void lam(const InstDesc& in, const float* ls, int x, int y, int z, int qs,
                                               float* l) {
        l[q - 1] = pull_lam_any<Q, q>(in, ls, x, y, z, qs);
        PullAll<Q, S, q + 1>::lam(in, ls, x, y, z, qs, l);
    }
};
template <int Q, class S>
struct PullAll<Q, S, Q> {
    static __device__ __forceinline__ void pre(const InstDesc&, const S*, int, int, int, int, float*) {}
    static __device__ __forceinline__ void lam(const InstDesc&, const float*, int, int, int, int, float*) {}
};

}  // namespace

// ------------------------------------------------------------ fluid sweep --
// lam_mode: 0 = pull the adjoint of step n + 1, 1 = read a field seed [Q][N]
// (the adjoint of the final post-collision populations), 2 = zero.
// One block per tile of the forward kernel's shape (its candidate lists are
// per tile); each warp takes whole x-rows of the tile and its lanes stride
// along x, so the loads of a population are coalesced.  Interior nodes use
// per-population element offsets precomputed once per block.
template <int Q, class S>
__global__ void __launch_bounds__(256, Q == 9 ? 3 : 2) k_adj_fluid(const InstDesc* __restrict__ insts,
                                                   const AdjFluid* __restrict__ afs,
                                                   const uint16_t* __restrict__ tile_inst, int lam_mode,
                                                   Shape sh) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int QS = Q - 1;
    __shared__ Cand cand[LIST_CAP];
    __shared__ int offF[QS], offL[QS];  // source offsets of the forward and the transposed pull
    const int t = blockIdx.x;
    const int ii = tile_inst[t];
    const InstDesc& in = insts[ii];
    const AdjFluid& af = afs[ii];
    const int local = t - in.tile0;
    const int tw = sh.tw;
    const int ntx = in.ntile[0], nty = in.ntile[1];
    const int tx = local % ntx, rest = local / ntx;
    const int x0 = tx * tw, y0 = (rest % nty) * sh.ty, z0 = (rest / nty) * sh.tz;
    const int nx = in.n[0], ny = in.n[1], nz = in.n[2];
    const int pitch = in.pitch;
    const int qs = (int)in.qstride;  // (Q - 1) * qstride < 2^31 (validated at creation)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x < QS) {
        const int q = threadIdx.x + 1;
        const int sh_f = (L::c(q, 2) * ny + L::c(q, 1)) * pitch + L::c(q, 0);
        offF[threadIdx.x] = (q - 1) * qs - sh_f;
        offL[threadIdx.x] = (q - 1) * qs + sh_f;
    }
    int ncand = 0;
    if (in.np > 0) {
        ncand = min(af.lcnt[local], LIST_CAP);
        for (int c = threadIdx.x; c < ncand; c += blockDim.x) {
            const uint32_t e = af.lent[(long long)local * LIST_CAP + c];
            const int p = (int)(e >> KBITS);
            const PRec& pr = af.prec[p];
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
            cd.k = (int)(e & (MAXK - 1));
            cd.boff = 0;
            cd.bh = 0;
            cd.shape = pr.shape;
            cand[c] = cd;
        }
    }
    __syncthreads();
    Geo geo = make_geo(in);
    geo.prec = af.prec;
    const CollK ck = make_collk<Q>(make_collp(in));
    const S* __restrict__ fin = static_cast<const S*>(af.fin);
    const float* __restrict__ lsrc = af.lam_src;
    float* __restrict__ ldst = af.lam_dst;
    const float sl = in.s_load;
    const float gd[3] = {in.gdrive[0], in.gdrive[1], in.gdrive[2]};
    const long long N = (long long)nx * ny * nz;
    const int w = min(tw, nx - x0);
    const int wpad = (w + 31) & ~31;
    const int rows = sh.ty * sh.tz;
    for (int r = warp; r < rows; r += nwarps) {
        const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
        if (y >= ny || z >= nz) continue;  // warp-uniform
        const bool row_in = y >= 1 && y + 1 < ny && (D == 2 || (z >= 1 && z + 1 < nz));
        const int rowoff = (z * ny + y) * pitch;
        // D2Q9: two nodes per lane (xo0 and xo0 + 32), both nodes' gathers in
        // flight together before either is computed (D3Q19: one, registers)
        constexpr int NPL = Q == 9 ? 2 : 1;
        for (int xo0 = lane; xo0 < wpad; xo0 += 32 * NPL) {
            float f[NPL][QS], lam[NPL][QS];
            int xsv[NPL], nodev[NPL];
            bool validv[NPL];
#pragma unroll
            for (int h = 0; h < NPL; ++h) {
                const int xo = xo0 + 32 * h;
                validv[h] = xo < w;
                const int xs = validv[h] ? x0 + xo : x0;  // lanes beyond the row compute on a valid node, store nothing
                xsv[h] = xs;
                const int node = rowoff + xs;
                nodev[h] = node;
                // warp-uniform: every lane's stencil stays inside the box
                const bool interior = __all_sync(0xffffffffu, row_in && xs >= 1 && xs + 1 < nx);
                if (interior) {
#pragma unroll
                    for (int q = 0; q < QS; ++q)
                        f[h][q] = VecIO<S, 1 + (sizeof(S) == 2)>::load1(fin + (node + offF[q]), sl);
                } else {
                    PullAll<Q, S, 1>::pre(in, fin, xs, y, z, qs, f[h]);
                }
                if (lam_mode == 0) {
                    if (interior) {
#pragma unroll
                        for (int q = 0; q < QS; ++q) lam[h][q] = __ldg(lsrc + (node + offL[q]));
                    } else {
                        PullAll<Q, S, 1>::lam(in, lsrc, xs, y, z, qs, lam[h]);
                    }
                } else if (lam_mode == 1) {
                    const long long nd = ((long long)z * ny + y) * nx + xs;
#pragma unroll
                    for (int q = 1; q < Q; ++q) lam[h][q - 1] = __ldg(lsrc + (long long)q * N + nd);
                } else {
#pragma unroll
                    for (int q = 0; q < QS; ++q) lam[h][q] = 0.f;
                }
            }
#pragma unroll
            for (int h = 0; h < NPL; ++h) {
                const int xs = xsv[h], node = nodev[h];
                const bool valid = validv[h];
                float a[3] = {gd[0], gd[1], gd[2]};
                float ubp[3] = {0.f, 0.f, 0.f};
                int own = -1;
                if (ncand > 0) {
                    const int xyz[3] = {xs, y, z};
                    int slt = -1;
                    own = owner_of<D>(geo, cand, ncand, xyz, &slt);
                    if (own >= 0) {
                        const Cand& cd = cand[slt];
                        float rr[3] = {0.f, 0.f, 0.f};
#pragma unroll
                        for (int d = 0; d < D; ++d)
                            rr[d] = (float)wrap_int(xyz[d] - cd.ref[d], in.n[d], in.periodic[d]) - cd.frac[d];
                        const float* cf = af.coef + 8LL * own;
#pragma unroll
                        for (int d = 0; d < 3; ++d) a[d] += cd.a[d];
                        // d U / d u = 1 / count, d W / d u: (I^-1 dW) x r
                        ubp[0] = cf[0] + (cf[4] * rr[2] - cf[5] * rr[1]);
                        ubp[1] = cf[1] + (cf[5] * rr[0] - cf[3] * rr[2]);
                        ubp[2] = D == 3 ? cf[2] + (cf[3] * rr[1] - cf[4] * rr[0]) : 0.f;
                    }
                    if (!valid) own = -1;
                }
                float fb[QS], ab[3], alb;
                const bool any_solid = __any_sync(0xffffffffu, own >= 0);
                node_adjoint<Q>(f[h], a, lam[h], own >= 0, any_solid, ubp, ck, fb, ab, &alb);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < QS; ++q) ldst[node + q * qs] = fb[q];
                }
                // per-particle sums of the adjoint acceleration and alpha derivative
                unsigned pend = __ballot_sync(0xffffffffu, own >= 0);
                while (pend) {
                    const int leader = __ffs(pend) - 1;
                    const int p = __shfl_sync(0xffffffffu, own, leader);
                    const bool mine = own == p;
                    float v[4] = {mine ? ab[0] : 0.f, mine ? ab[1] : 0.f, mine ? ab[2] : 0.f, mine ? alb : 0.f};
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
                    if (lane == leader) {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (k < D || k == 3) atomicAdd(af.Abar + 4LL * p + k, (double)v[k]);
                    }
                    pend &= ~__ballot_sync(0xffffffffu, mine);
                }
            }
        }
    }
}

// Adjoint of the initial post-collision populations (transposed streaming of
// the adjoint of step 0), written as [Q][N] with the rest population zero.
template <int Q>
__global__ void k_adj_pull_out(const InstDesc* __restrict__ insts, int inst, const float* __restrict__ lam,
                               float* __restrict__ out) {
    const InstDesc& in = insts[inst];
    const long long N = (long long)in.n[0] * in.n[1] * in.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int x = (int)(i % in.n[0]), y = (int)((i / in.n[0]) % in.n[1]),
              z = (int)(i / ((long long)in.n[0] * in.n[1]));
    float v[Q - 1];
    PullAll<Q, float, 1>::lam(in, lam, x, y, z, (int)in.qstride, v);
    out[i] = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) out[(long long)q * N + i] = v[q - 1];
}

// --------------------------------------------------------- particle sweep --
namespace {

// Whether a particle at coordinate Y (radius R) along wall axis d can be within
// the wall range R + delta/2 of either plane -1/2, n - 1/2: an FP32 test with
// a 0.01 margin (the forward kernel's filter), so that particles far from the
// walls skip the FP64 range tests, whose outcome it cannot change.
__device__ __forceinline__ bool wall_near(const InstDesc& in, int d, double Y, double R) {
    const float reach = 0.5f * (2.0f * (float)R + (float)in.delta) + 0.01f;
    const float yf = (float)Y;
    return !(yf + 0.5f > reach && (float)in.n[d] - 0.5f - yf > reach);
}

// Collision force on particle i per unit C (Eqs. 19-21 with C = 1): pairs
// with the lattice's minimum image, and mirror images across wall planes.
__device__ void unit_force(const InstDesc& in, int D, const double* Y, int i, double* G) {
    G[0] = G[1] = G[2] = 0.0;
    const double idl = in.pconst[PCONST_N * i + PC_INVDELTA];
    for (int j = 0; j < in.np; ++j) {
        if (j == i) continue;
        double dv[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) {
            double x = Y[3 * i + d] - Y[3 * j + d];
            if (in.periodic[d]) {
                const double half = 0.5 * in.n[d];
                if (x > half) x -= in.n[d];
                else if (x < -half) x += in.n[d];
            }
            dv[d] = x;
        }
        const double range = in.R[i] + in.R[j] + in.delta;
        const double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        if (d2 > range * range) continue;
        const double s = (range - sqrt(d2)) * idl;
        for (int d = 0; d < 3; ++d) G[d] += dv[d] * s * s * in.inv_eps_p;
    }
    for (int d = 0; d < D; ++d) {
        if (in.periodic[d] || !wall_near(in, d, Y[3 * i + d], in.R[i])) continue;
        const double walls[2] = {-0.5, in.n[d] - 0.5};
        for (int face = 0; face < 2; ++face) {
            const double diff = 2.0 * (Y[3 * i + d] - walls[face]);
            const double range = 2.0 * in.R[i] + in.delta;
            if (fabs(diff) <= range) {
                const double s = (range - fabs(diff)) * idl;
                G[d] += diff * s * s * in.inv_eps_w;
            }
        }
    }
}

// Transposed Jacobian of the collision forces at positions Y applied to
// their adjoint v: the adjoint of the positions of particle m.  With
// F_i = k_i sum_j phi(d_ij), phi(d) = d s^2, s = (range - |d|)/delta and
// phi'(d) = s^2 1 - (2 s / (delta |d|)) d d^T (even in d):
//   Yb_m = sum_j phi'(d_mj) (k_m v_m - k_j v_j) + walls 2 kw_m psi'(diff) v_m.
__device__ void force_jt(const InstDesc& in, int D, const double* Y, const double* v, int m, double* out) {
    const double idl = in.pconst[PCONST_N * m + PC_INVDELTA];
    const double km = in.pconst[PCONST_N * m + PC_CPAIR];  // C_m / eps_p
    double acc[3] = {0, 0, 0};
    for (int j = 0; j < in.np; ++j) {
        if (j == m) continue;
        double dv[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) {
            double x = Y[3 * m + d] - Y[3 * j + d];
            if (in.periodic[d]) {
                const double half = 0.5 * in.n[d];
                if (x > half) x -= in.n[d];
                else if (x < -half) x += in.n[d];
            }
            dv[d] = x;
        }
        const double range = in.R[m] + in.R[j] + in.delta;
        const double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        if (d2 > range * range || d2 == 0.0) continue;
        const double dist = sqrt(d2);
        const double s = (range - dist) * idl;
        const double kj = in.pconst[PCONST_N * j + PC_CPAIR];
        double w[3];
        for (int d = 0; d < 3; ++d) w[d] = km * v[3 * m + d] - kj * v[3 * j + d];
        const double dw = dv[0] * w[0] + dv[1] * w[1] + dv[2] * w[2];
        const double g = 2.0 * s * idl * rcp64(dist);
        for (int d = 0; d < 3; ++d) acc[d] += s * s * w[d] - g * dv[d] * dw;
    }
    const double kw = in.pconst[PCONST_N * m + PC_CWALL];  // C_m / eps_w
    for (int d = 0; d < D; ++d) {
        if (in.periodic[d] || !wall_near(in, d, Y[3 * m + d], in.R[m])) continue;
        const double walls[2] = {-0.5, in.n[d] - 0.5};
        for (int face = 0; face < 2; ++face) {
            const double diff = 2.0 * (Y[3 * m + d] - walls[face]);
            const double range = 2.0 * in.R[m] + in.delta;
            if (fabs(diff) <= range) {
                const double s = (range - fabs(diff)) * idl;
                acc[d] += 2.0 * kw * (s * s - 2.0 * s * fabs(diff) * idl) * v[3 * m + d];
            }
        }
    }
    for (int d = 0; d < 3; ++d) out[d] = acc[d];
}

}  // namespace

// Backward of the particle part of step n for every instance (block = instance).
template <int D>
__global__ void __launch_bounds__(128) k_adj_particles(const InstDesc* __restrict__ insts,
                                                       const AdjPart* __restrict__ steps,
                                                       const AdjBufs* __restrict__ bufs) {
    const int ii = blockIdx.x;
    __shared__ __align__(16) InstDesc sdesc;
    stage_desc(&sdesc, insts[ii]);
    const InstDesc& in = sdesc;
    const int np = in.np;
    if (np == 0) return;
    const AdjPart sp = steps[ii];
    const AdjBufs b = bufs[ii];
    const int K = in.K;
    const double h = in.hK;
    const double gC = in.rho_f * in.gmag;
    const int tid = threadIdx.x, nt = blockDim.x;
    // 1. fold the fluid sums of step n + 1 into the adjoint of A^{n+1}, of
    //    the density ratios (a = (1 - 1/ratio) g + A on solid nodes) and of alpha
    double al = 0.0;
    for (int p = tid; p < np; p += nt) {
        double Ap[3], gsum = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double fl = b.Abar[4 * p + d];
            Ap[d] = b.Ab[3 * p + d] + fl;
            gsum += fl * (double)in.ggrav[d];
            b.Abar[4 * p + d] = 0.0;
            b.Ab[3 * p + d] = 0.0;
        }
        al += b.Abar[4 * p + 3];
        b.Abar[4 * p + 3] = 0.0;
        const double iratio = in.pconst[PCONST_N * p + PC_INVRHOS] * in.rho_f;
        b.rb[p] += gsum * iratio * iratio;
        // state after step n: X' = Xk_K (wrapped), U' = U^n, W' = W^n,
        // theta' = theta + (W^n + W)/2, A' = 2 (Xk_K - X - Ubar)
        for (int d = 0; d < 3; ++d) {
            const double xb = b.Xb[3 * p + d], tb = b.Tb[3 * p + d];
            b.Xkb[3 * p + d] = xb + 2.0 * Ap[d];
            b.Xb[3 * p + d] = -2.0 * Ap[d];
            b.Ubb[3 * p + d] = -2.0 * Ap[d];
            b.Wnb[3 * p + d] = b.Wb[3 * p + d] + 0.5 * tb;  // adjoint of W^n
            b.Wb[3 * p + d] = 0.5 * tb;                      // adjoint of W^{n-1}
            b.Ubar[3 * p + d] = 0.5 * (sp.st1[16 * p + 3 + d] + sp.st0[16 * p + 3 + d]);
            b.Xk[3 * p + d] = sp.st0[16 * p + d];
        }
    }
    if (al != 0.0) atomicAdd(b.alpha_b, al);
    __syncthreads();
    // 2. forward sub-steps of Algorithm 1 (positions and unit forces)
    const size_t s3 = 3 * (size_t)np;
    for (int j = 1; j <= K; ++j) {
        const double* Xp = b.Xk + (j - 1) * s3;
        double* Xs = b.Xs + (j - 1) * s3;
        for (int p = tid; p < np; p += nt)
            for (int d = 0; d < 3; ++d) Xs[3 * p + d] = Xp[3 * p + d] + h * b.Ubar[3 * p + d];
        __syncthreads();
        for (int p = tid; p < np; p += nt) {
            double G1[3], G2[3];
            unit_force(in, D, Xp, p, G1);
            unit_force(in, D, Xs, p, G2);
            const double Cp = (in.ratio[p] - 1.0) * gC;
            const double c = 0.25 * h * h * in.pconst[PCONST_N * p + PC_INVRHOS] * rcp64(sp.st1[16 * p + 15]);
            for (int d = 0; d < 3; ++d) {
                b.F1[(j - 1) * s3 + 3 * p + d] = G1[d];
                b.F2[(j - 1) * s3 + 3 * p + d] = G2[d];
                b.Xk[j * s3 + 3 * p + d] = Xs[3 * p + d] + c * Cp * (G1[d] + G2[d]);
            }
        }
        __syncthreads();
    }
    // 3. reverse sub-steps: Xk_j = Xs_j + c (F1(Xk_{j-1}) + F2(Xs_j)), Xs_j = Xk_{j-1} + h Ubar
    for (int j = K; j >= 1; --j) {
        for (int p = tid; p < np; p += nt) {
            const double Cp = (in.ratio[p] - 1.0) * gC;
            const double irs = in.pconst[PCONST_N * p + PC_INVRHOS];  // 1 / (rho_s)
            const double c = 0.25 * h * h * irs * rcp64(sp.st1[16 * p + 15]);
            const double iratio = irs * in.rho_f;
            double rbp = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double xkb = b.Xkb[3 * p + d];
                const double Gs = b.F1[(j - 1) * s3 + 3 * p + d] + b.F2[(j - 1) * s3 + 3 * p + d];
                b.v[3 * p + d] = c * xkb;
                // d c / d ratio = -c / ratio, d C / d ratio = rho_f |g|
                rbp += xkb * (-c * iratio * Cp * Gs + c * gC * Gs);
            }
            b.rb[p] += rbp;
        }
        __syncthreads();
        for (int p = tid; p < np; p += nt) {
            double jt[3];
            force_jt(in, D, b.Xs + (j - 1) * s3, b.v, p, jt);
            for (int d = 0; d < 3; ++d) {
                const double xsb = b.Xkb[3 * p + d] + jt[d];
                b.Xsb[3 * p + d] = xsb;
                b.Ubb[3 * p + d] += h * xsb;
            }
        }
        __syncthreads();
        for (int p = tid; p < np; p += nt) {
            double jt[3];
            force_jt(in, D, b.Xk + (j - 1) * s3, b.v, p, jt);
            for (int d = 0; d < 3; ++d) b.Xkb[3 * p + d] = b.Xsb[3 * p + d] + jt[d];
        }
        __syncthreads();
    }
    // 4. Ubar = (U^n + U^{n-1})/2, the projection (Eq. 22) and the outputs
    for (int p = tid; p < np; p += nt) {
        const double* g = sp.geo + (long long)NPV * p;
        const double icnt = rcp64(g[0]);
        double Unb[3], Wnb[3], Xb[3], W[3], Su[3], Sr[3];
        for (int d = 0; d < 3; ++d) {
            Xb[d] = b.Xb[3 * p + d] + b.Xkb[3 * p + d];
            Unb[d] = b.Ub[3 * p + d] + 0.5 * b.Ubb[3 * p + d];
            b.Ub[3 * p + d] = 0.5 * b.Ubb[3 * p + d];
            Wnb[d] = b.Wnb[3 * p + d];
            W[d] = sp.st1[16 * p + 6 + d];
            Su[d] = g[10 + d];
            Sr[d] = g[1 + d];
        }
        double mu[3] = {0, 0, 0};
        if (D == 2) {
            mu[2] = Wnb[2] * rcp64(g[4] + g[5]);
        } else {
            // I = tr(rr) 1 - rr (symmetric); mu = I^-1 Wnb by cofactors
            const double tr = g[4] + g[5] + g[6];
            const double I00 = tr - g[4], I11 = tr - g[5], I22 = tr - g[6];
            const double I01 = -g[7], I02 = -g[8], I12 = -g[9];
            const double c00 = I11 * I22 - I12 * I12, c01 = I02 * I12 - I01 * I22, c02 = I01 * I12 - I02 * I11;
            const double c11 = I00 * I22 - I02 * I02, c12 = I01 * I02 - I00 * I12, c22 = I00 * I11 - I01 * I01;
            const double idet = rcp64(I00 * c00 + I01 * c01 + I02 * c02);
            mu[0] = (c00 * Wnb[0] + c01 * Wnb[1] + c02 * Wnb[2]) * idet;
            mu[1] = (c01 * Wnb[0] + c11 * Wnb[1] + c12 * Wnb[2]) * idet;
            mu[2] = (c02 * Wnb[0] + c12 * Wnb[1] + c22 * Wnb[2]) * idet;
        }
        // d W / d X through r = x - X: mu x Su + 2 (mu.W) Sr - mu (Sr.W) - W (mu.Sr)
        const double muW = mu[0] * W[0] + mu[1] * W[1] + mu[2] * W[2];
        const double SrW = Sr[0] * W[0] + Sr[1] * W[1] + Sr[2] * W[2];
        const double muSr = mu[0] * Sr[0] + mu[1] * Sr[1] + mu[2] * Sr[2];
        const double cx[3] = {mu[1] * Su[2] - mu[2] * Su[1], mu[2] * Su[0] - mu[0] * Su[2],
                              mu[0] * Su[1] - mu[1] * Su[0]};
        for (int d = 0; d < D; ++d) Xb[d] += cx[d] + 2.0 * muW * Sr[d] - mu[d] * SrW - W[d] * muSr;
        for (int d = 0; d < 3; ++d) {
            b.Xb[3 * p + d] = d < D ? Xb[d] : 0.0;
            b.coef[8 * p + d] = (float)(Unb[d] * icnt);
            b.coef[8 * p + 3 + d] = (float)mu[d];
        }
    }
}

// After the sweep: fold the fluid sums of step 0 and write, per instance,
// [d alpha] + per particle [d ratio, d X0 (3), d U0 (3), d W0 (3), d theta0 (3), d A0 (3)].
__global__ void k_adj_finish(const InstDesc* __restrict__ insts, const AdjBufs* __restrict__ bufs,
                             const long long* __restrict__ out_off, double* __restrict__ out) {
    const int ii = blockIdx.x;
    const InstDesc& in = insts[ii];
    const AdjBufs b = bufs[ii];
    double* o = out + out_off[ii];
    double al = 0.0;
    for (int p = threadIdx.x; p < in.np; p += blockDim.x) {
        const double iratio = in.pconst[PCONST_N * p + PC_INVRHOS] * in.rho_f;
        double gsum = 0.0;
        double* r = o + 1 + 16LL * p;
        for (int d = 0; d < 3; ++d) {
            const double fl = b.Abar[4 * p + d];
            gsum += fl * (double)in.ggrav[d];
            r[1 + d] = b.Xb[3 * p + d];
            r[4 + d] = b.Ub[3 * p + d];
            r[7 + d] = b.Wb[3 * p + d];
            r[10 + d] = b.Tb[3 * p + d];
            r[13 + d] = b.Ab[3 * p + d] + fl;
        }
        al += b.Abar[4 * p + 3];
        r[0] = b.rb[p] + gsum * iratio * iratio;
    }
    __shared__ double red[128];
    red[threadIdx.x] = al;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
        o[0] = *b.alpha_b + s;
    }
}

// Copy the particle state between the context arrays and a [np][16] record.
__global__ void k_adj_state(const InstDesc* __restrict__ insts, int inst, double* rec, int to_record) {
    const InstDesc& in = insts[inst];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= in.np) return;
    double* r = rec + 16LL * p;
    double* arr[5] = {in.X, in.U, in.W, in.theta, in.A};
    if (to_record) {
        for (int a = 0; a < 5; ++a)
            for (int d = 0; d < 3; ++d) r[3 * a + d] = arr[a][3 * p + d];
        r[15] = (double)in.count[p];
    } else {
        for (int a = 0; a < 5; ++a)
            for (int d = 0; d < 3; ++d) arr[a][3 * p + d] = r[3 * a + d];
        in.count[p] = (int)r[15];
    }
}

// ------------------------------------------------------------- launchers --
cudaError_t launch_adj_fluid(int Q, int fp16, const InstDesc* insts, const AdjFluid* afs,
                             const uint16_t* tile_inst, int ntiles, int lam_mode, const Shape& sh,
                             cudaStream_t st) {
    // a warp per tile row, up to the 8 warps of the launch bounds
    const int rows = sh.ty * sh.tz;
    const int threads = 32 * (rows < 8 ? rows : 8);
    if (Q == 9) {
        if (fp16) k_adj_fluid<9, __half><<<ntiles, threads, 0, st>>>(insts, afs, tile_inst, lam_mode, sh);
        else k_adj_fluid<9, float><<<ntiles, threads, 0, st>>>(insts, afs, tile_inst, lam_mode, sh);
    } else {
        if (fp16) k_adj_fluid<19, __half><<<ntiles, threads, 0, st>>>(insts, afs, tile_inst, lam_mode, sh);
        else k_adj_fluid<19, float><<<ntiles, threads, 0, st>>>(insts, afs, tile_inst, lam_mode, sh);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_particles(int D, const InstDesc* insts, const AdjPart* steps, const AdjBufs* bufs,
                                 int ninst, cudaStream_t st) {
    if (D == 2) k_adj_particles<2><<<ninst, 128, 0, st>>>(insts, steps, bufs);
    else k_adj_particles<3><<<ninst, 128, 0, st>>>(insts, steps, bufs);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(const InstDesc* insts, const AdjBufs* bufs, const long long* out_off,
                              double* out, int ninst, cudaStream_t st) {
    k_adj_finish<<<ninst, 128, 0, st>>>(insts, bufs, out_off, out);
    return cudaGetLastError();
}

cudaError_t launch_adj_pull_out(int Q, const InstDesc* insts, int inst, long long N, const float* lam,
                                float* out, cudaStream_t st) {
    const unsigned blocks = (unsigned)((N + 255) / 256);
    if (Q == 9) k_adj_pull_out<9><<<blocks, 256, 0, st>>>(insts, inst, lam, out);
    else k_adj_pull_out<19><<<blocks, 256, 0, st>>>(insts, inst, lam, out);
    return cudaGetLastError();
}

cudaError_t launch_adj_state(const InstDesc* insts, int inst, int np, double* rec, int to_record,
                             cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    k_adj_state<<<(np + 127) / 128, 128, 0, st>>>(insts, inst, rec, to_record);
    return cudaGetLastError();
}

}  // namespace lbmpen
