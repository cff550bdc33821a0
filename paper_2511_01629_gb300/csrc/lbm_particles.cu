// Per-particle FP64 kernels of lbmpen: the rigid-body projection (Eq. 22)
// from the fluid kernel's per-tile partial sums, the predictor-corrector of
// Algorithm 1 with the repulsive collision forces (Eqs. 19-21), and the
// rebuild of each particle's record and tile-list entries for the next step.
//
// GB300 runs FP64 at a small fraction of its FP32 rate and the cost of an
// FP64 instruction is paid per warp, so the serial per-particle arithmetic
// runs one particle per thread (32 particles per warp instruction).  Only the
// O(N^2) pair search uses a warp per particle, filtering pairs in FP32 with a
// margin before the FP64 evaluation of the few pairs within range.
#include "lbm_internal.cuh"

namespace lbmpen {

constexpr double FX_SCALE = 1.0 / (double)(1LL << FXBITS);

// Rigid-body projection of particle p (Eq. 22 with rho_s cancelled): the
// tile partials are exact integers, summed exactly, then converted to FP64.
// Moments about the integer reference floor(X) are shifted to the centre:
//   sum r x u = sum d x u - phi x sum u,
//   sum r r^T = sum d d^T - phi sum d^T - sum d phi^T + n phi phi^T.
template <int D>
__device__ void finalize_particle(const InstDesc& in, int p, const long long* v) {
    const double cnt = (double)v[0];
    double phi[3], X[3], Uo[3] = {0, 0, 0}, Wo[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        X[d] = in.X[3 * p + d];
        phi[d] = d < D ? X[d] - (double)in.prec[p].ref[d] : 0.0;
    }
    if (v[0] == 0) {  // no solid node: cannot happen inside the box for R >= 2
        atomicOr(in.status, ST_PARTICLE);
        for (int d = 0; d < 3; ++d) {
            in.Un[3 * p + d] = in.U[3 * p + d];
            in.Wn[3 * p + d] = 0.0;
        }
        in.count[p] = 0;
        return;
    }
    double Sd[3], Su[3], Sl[3];
    for (int d = 0; d < 3; ++d) {
        Sd[d] = (double)v[1 + d];
        Su[d] = (double)v[10 + d] * FX_SCALE;
        Sl[d] = (double)v[13 + d] * FX_SCALE;
    }
    const double inv = 1.0 / cnt;
    for (int d = 0; d < 3; ++d) Uo[d] = Su[d] * inv;
    const double Lv[3] = {Sl[0] - (phi[1] * Su[2] - phi[2] * Su[1]),
                          Sl[1] - (phi[2] * Su[0] - phi[0] * Su[2]),
                          Sl[2] - (phi[0] * Su[1] - phi[1] * Su[0])};
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
    double rr[3][3];
    for (int k = 0; k < 6; ++k) {
        const int i = ii[k], j = jj[k];
        const double val = (double)v[4 + k] - phi[i] * Sd[j] - phi[j] * Sd[i] + cnt * phi[i] * phi[j];
        rr[i][j] = val;
        rr[j][i] = val;
    }
    if (D == 2) {
        Wo[2] = Lv[2] / (rr[0][0] + rr[1][1]);
    } else {
        const double tr = rr[0][0] + rr[1][1] + rr[2][2];
        double I[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) I[i][j] = (i == j ? tr : 0.0) - rr[i][j];
        const double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                           I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                           I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
        const double idet = 1.0 / det;
        for (int col = 0; col < 3; ++col) {
            double M[3][3];
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) M[r][q] = (q == col) ? Lv[r] : I[r][q];
            const double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                              M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                              M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            Wo[col] = dc * idet;
        }
    }
    bool fast = false;
    for (int d = 0; d < 3; ++d) {
        in.Un[3 * p + d] = Uo[d];
        in.Wn[3 * p + d] = Wo[d];
        const double ub = 0.5 * (Uo[d] + in.U[3 * p + d]);
        in.Ubar[3 * p + d] = ub;
        in.Xk[3 * p + d] = X[d];  // sub-step buffer 0 = X^n
        fast |= !(fabs(ub) < 0.5);
    }
    reinterpret_cast<float4*>(in.Xf)[p] =  // float buffer 0 mirrors Xk buffer 0
        make_float4((float)X[0], (float)X[1], (float)X[2], (float)in.R[p]);
    in.count[p] = (int)v[0];
    if (fast) atomicOr(in.status, ST_DISPLACEMENT);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int PB = 8;  // particles per block (one per warp) of the particle kernels
constexpr int XCHUNK = 1024;  // particle positions staged in shared memory at a time

// 32 particles per block: the block's warps sum the slot partials of 4
// particles each (lanes over slots, exact integer tree), then one thread per
// particle does the FP64 part.
__global__ void __launch_bounds__(256) k_finalize(const InstDesc* __restrict__ insts,
                                                  const PartRef* __restrict__ refs, int ntotal,
                                                  int D) {
    __shared__ long long tot[PB][NPV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gp0 = blockIdx.x * PB;
    for (int t = warp; t < PB; t += nwarps) {
        const int gp = gp0 + t;
        if (gp >= ntotal) break;
        const PartRef r = refs[gp];
        if (r.inst < 0) continue;  // padding of the instance's last block
        const InstDesc& in = insts[r.inst];
        const int nt = min(in.prec[r.p].ntiles, in.maxk);  // overflow is flagged at publish
        long long v[NPV];
#pragma unroll
        for (int k = 0; k < NPV; ++k) v[k] = 0;
        for (int s = lane; s < nt; s += 32) {
            longlong2* src = reinterpret_cast<longlong2*>(in.partial + ((long long)r.p * in.maxk + s) * NPV);
#pragma unroll
            for (int k = 0; k < NPV / 2; ++k) {
                const longlong2 a = __ldcg(src + k);
                v[2 * k] += a.x;
                v[2 * k + 1] += a.y;
                src[k] = make_longlong2(0, 0);  // the slot starts the next step at zero
            }
        }
#pragma unroll
        for (int k = 0; k < NPV; ++k) {
            const long long w = warp_sum_ll(v[k]);
            if (lane == 0) tot[t][k] = w;
        }
    }
    __syncthreads();
    if (warp != 0 || lane >= PB) return;
    const int gp = gp0 + lane;
    if (gp >= ntotal) return;
    const PartRef r = refs[gp];
    if (r.inst < 0) return;
    const InstDesc& in = insts[r.inst];
    if (D == 2) finalize_particle<2>(in, r.p, tot[lane]);
    else finalize_particle<3>(in, r.p, tot[lane]);
}

// Pair part of Eq. 21 on particle i at two position sets: Xk[src] (F1) and
// Xk[src] + h Ubar (F2).  The block's particles all belong to one instance;
// its positions are staged in shared memory in chunks and the lanes split
// them.  An FP32 filter with a margin of 2.5 lattice units (a sub-step moves
// a particle by |h Ubar| < 1/2) leaves only pairs near the interaction range
// for the FP64 evaluation, which follows the reference operation order.
__device__ void pair_chunk(const InstDesc& in, int i, int src, double h, int lane, const float4* xs,
                           int j0, int nj, double* f1, double* f2) {
    const double* Xb = in.Xk + (long long)src * in.np * 3;
    const double C = (in.ratio[i] - 1.0) * in.rho_f * in.gmag;
    if (C == 0.0) return;
    const float4 xi = reinterpret_cast<const float4*>(in.Xf)[(long long)src * in.np + i];
    const float reach = xi.w + (float)in.delta + 2.5f;
    const float nf[3] = {(float)in.n[0], (float)in.n[1], (float)in.n[2]};
    const bool per[3] = {in.periodic[0] && in.n[0] > 1, in.periodic[1] && in.n[1] > 1,
                         in.periodic[2] && in.n[2] > 1};
    for (int jj = lane; jj < nj; jj += 32) {
        const int j = j0 + jj;
        if (j == i) continue;
        const float4 xj = xs[jj];
        float dv[3] = {xi.x - xj.x, xi.y - xj.y, xi.z - xj.z};
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (per[d]) dv[d] -= nf[d] * rintf(dv[d] / nf[d]);
        const float lim = reach + xj.w;
        if (dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2] > lim * lim) continue;
        const double range = in.R[i] + in.R[j] + in.delta;
        for (int pass = 0; pass < 2; ++pass) {
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
            if (dij <= range) {
                const double sc = (range - dij) / in.delta;
                double* f = pass ? f2 : f1;
                for (int d = 0; d < 3; ++d) f[d] += C / in.eps_p * dd[d] * sc * sc;
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

// Wall part of Eq. 21 (mirror images across the planes -1/2 and n - 1/2).
__device__ void wall_force(const InstDesc& in, int i, const double* Xi, double* F) {
    const double C = (in.ratio[i] - 1.0) * in.rho_f * in.gmag;
    if (C == 0.0) return;
    for (int d = 0; d < 3; ++d) {
        if (in.periodic[d] || in.n[d] <= 1) continue;
        const double walls[2] = {-0.5, in.n[d] - 0.5};
        for (int face = 0; face < 2; ++face) {
            const double Xim = 2.0 * walls[face] - Xi[d];
            const double diff = Xi[d] - Xim;
            const double dprime = fabs(diff);
            const double range = 2.0 * in.R[i] + in.delta;
            if (dprime <= range) {
                const double sc = (range - dprime) / in.delta;
                F[d] += C / in.eps_w * diff * sc * sc;
            }
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

__device__ AxisTiles axis_tiles(double X, double R, int n, int T, int ntile, int periodic) {
    int lo = (int)floor(X - R) - 1, hi = (int)floor(X + R) + 1;
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

// Record and tile-list entries of particle p at its current X and A for the
// step that reads list parity lpar.  Slots k enumerate the bounding-box tiles
// x-fastest; no tile is listed twice.  The calling warp's lanes (lane0 ..
// lane0 + nl - 1) share the list appends; lane0 writes the record.
__device__ void publish_particle(const InstDesc& in, int p, int lpar, int D, const Shape& sh,
                                 int lane, int nl) {
    const double R = in.R[p];
    const int T[3] = {sh.tw, sh.ty, sh.tz};
    AxisTiles at[3];
    int cnt[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= D) {
            at[d] = AxisTiles{0, 1, 0, 0};
        } else {
            at[d] = axis_tiles(in.X[3 * p + d], R, in.n[d], T[d], in.ntile[d], in.periodic[d]);
        }
        cnt[d] = at[d].na + at[d].nb;
    }
    const int nt = cnt[0] * cnt[1] * cnt[2];
    if (lane == 0) {
        PRec pr;
        const double gfac = 1.0 - 1.0 / in.ratio[p];
        for (int d = 0; d < 3; ++d) {
            const double X = in.X[3 * p + d];
            pr.X[d] = X;
            const double fl = d < D ? floor(X) : 0.0;
            pr.ref[d] = (int)fl;
            pr.frac[d] = (float)(X - fl);
            pr.a[d] = (float)(gfac * (double)in.ggrav[d] + in.A[3 * p + d]);
        }
        pr.R2 = R * R;
        pr.R2lo = (float)(pr.R2 * (1.0 - 1e-5) - 1e-4);
        pr.R2hi = (float)(pr.R2 * (1.0 + 1e-5) + 1e-4);
        pr.ntiles = nt;
        pr.pad = 0;
        in.prec[p] = pr;
        if (nt > in.maxk) atomicOr(in.status, ST_CAPACITY);
    }
    for (int k = lane; k < nt && k < in.maxk; k += nl) {
        const int kx = k % cnt[0], ky = (k / cnt[0]) % cnt[1], kz = k / (cnt[0] * cnt[1]);
        const int tc[3] = {axis_tile(at[0], kx), axis_tile(at[1], ky), axis_tile(at[2], kz)};
        const int local = (tc[2] * in.ntile[1] + tc[1]) * in.ntile[0] + tc[0];
        const int pos = atomicAdd(&in.list_cnt[lpar][local], 1);
        if (pos < LIST_CAP)
            in.list_ent[lpar][(long long)local * LIST_CAP + pos] = ((uint32_t)p << KBITS) | (uint32_t)k;
        else
            atomicOr(in.status, ST_CAPACITY);
    }
}

// Algorithm 1 for particle i (one thread): wall forces, the corrected
// position, and on the last sub-step A^{n+1}, theta^{n+1} and U^{n-1} <- U^n.
__device__ void update_particle(const InstDesc& in, int i, int t, const double (*sF)[6], int src,
                                double h, int last, int D) {
    const int dst = src ^ 1;
    const double* Xs = in.Xk + (long long)src * in.np * 3;
    double X0[3], Xst[3], F1[3], F2[3];
    for (int d = 0; d < 3; ++d) {
        X0[d] = Xs[3 * i + d];
        Xst[d] = X0[d] + h * in.Ubar[3 * i + d];
        F1[d] = sF[t][d];
        F2[d] = sF[t][3 + d];
    }
    wall_force(in, i, X0, F1);
    wall_force(in, i, Xst, F2);
    const double M = in.ratio[i] * in.rho_f * (double)in.count[i];
    double Xn[3];
    for (int d = 0; d < 3; ++d) Xn[d] = Xst[d] + 1.0 / (2.0 * M) * h * h * 0.5 * (F1[d] + F2[d]);
    if (!last) {
        double* Xd = in.Xk + (long long)dst * in.np * 3;
        for (int d = 0; d < 3; ++d) Xd[3 * i + d] = Xn[d];
        reinterpret_cast<float4*>(in.Xf)[(long long)dst * in.np + i] =
            make_float4((float)Xn[0], (float)Xn[1], (float)Xn[2], (float)in.R[i]);
        return;
    }
    bool left = false;
    for (int d = 0; d < 3; ++d) {
        const int j = 3 * i + d;
        in.A[j] = 2.0 * (Xn[d] - in.X[j] - in.Ubar[j]);
        double xn = Xn[d];
        if (d < D) {
            if (in.periodic[d]) {
                if (xn >= in.n[d]) xn -= in.n[d];
                else if (xn < 0.0) xn += in.n[d];
            } else if (xn < -0.5 || xn > in.n[d] - 0.5) {
                left = true;
            }
        }
        in.X[j] = xn;
        in.theta[j] += 0.5 * (in.Wn[j] + in.W[j]);
        in.U[j] = in.Un[j];
        in.W[j] = in.Wn[j];
    }
    if (left) atomicOr(in.status, ST_PARTICLE);
}

// One sub-step k of Algorithm 1 (positions Xk[src] -> Xk[src ^ 1]) for 32
// particles per block: the block's warps find the pair forces (4 particles
// each), one thread per particle does the FP64 update, and after the last
// sub-step the warps publish the particles for the next fluid step.
__global__ void __launch_bounds__(256) k_substep(const InstDesc* __restrict__ insts,
                                                 const PartRef* __restrict__ refs, int ntotal, int D,
                                                 int src, int K, int last, int lpar, Shape sh) {
    __shared__ double sF[PB][6];
    __shared__ float4 xs[XCHUNK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gp0 = blockIdx.x * PB;
    const int inst = refs[gp0].inst;  // blocks never straddle instances
    const InstDesc& in = insts[inst];
    const double h = 1.0 / K;
    const int gp = gp0 + warp;
    const bool mine = warp < PB && gp < ntotal && refs[gp].inst >= 0;
    const int i = mine ? refs[gp].p : 0;
    double f1[3] = {0, 0, 0}, f2[3] = {0, 0, 0};
    const float4* Xfb = reinterpret_cast<const float4*>(in.Xf) + (long long)src * in.np;
    for (int j0 = 0; j0 < in.np; j0 += XCHUNK) {
        const int nj = min(XCHUNK, in.np - j0);
        __syncthreads();
        for (int k = threadIdx.x; k < nj; k += blockDim.x) xs[k] = Xfb[j0 + k];
        __syncthreads();
        if (mine) pair_chunk(in, i, src, h, lane, xs, j0, nj, f1, f2);
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
    if (warp == 0 && lane < PB && gp0 + lane < ntotal && refs[gp0 + lane].inst >= 0)
        update_particle(in, refs[gp0 + lane].p, lane, sF, src, h, last, D);
    if (!last) return;
    __syncthreads();  // new X and A of the block's particles are visible to all warps
    if (mine) publish_particle(in, i, lpar, D, sh, lane, 32);
}

// Publish every particle from its current state (after creation, particle
// insertion, a shape change or a state load).  Lists must be zeroed first.
__global__ void k_publish(const InstDesc* __restrict__ insts, const PartRef* __restrict__ refs,
                          int ntotal, int D, int lpar, Shape sh) {
    const int gp = blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= ntotal) return;
    const PartRef r = refs[gp];
    if (r.inst < 0) return;
    publish_particle(insts[r.inst], r.p, lpar, D, sh, 0, 1);
}

cudaError_t launch_finalize(const InstDesc* insts, const PartRef* refs, int ntotal, int D,
                            cudaStream_t st) {
    k_finalize<<<(ntotal + PB - 1) / PB, 256, 0, st>>>(insts, refs, ntotal, D);
    return cudaGetLastError();
}

cudaError_t launch_substep(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int src,
                           int K, int last, int lpar, const Shape& sh, cudaStream_t st) {
    k_substep<<<(ntotal + PB - 1) / PB, 256, 0, st>>>(insts, refs, ntotal, D, src, K, last, lpar, sh);
    return cudaGetLastError();
}

cudaError_t launch_publish(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int lpar,
                           const Shape& sh, cudaStream_t st) {
    k_publish<<<(ntotal + 63) / 64, 64, 0, st>>>(insts, refs, ntotal, D, lpar, sh);
    return cudaGetLastError();
}

}  // namespace lbmpen
