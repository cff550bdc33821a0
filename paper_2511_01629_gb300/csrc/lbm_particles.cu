// Per-particle FP64 kernels of lbmpen: the rigid-body projection (Eq. 22)
// from the fluid kernel's per-tile partial sums, the predictor-corrector of
// Algorithm 1 with the repulsive collision forces (Eqs. 19-21), and the
// rebuild of each particle's record and tile-list entries for the next step.
//
// One warp per particle.  GB300 runs FP64 at a small fraction of its FP32
// rate, so the pair search filters in FP32 and only pairs within the
// interaction range (plus a margin) are evaluated in FP64.
#include "lbm_internal.cuh"

namespace lbmpen {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rigid-body projection of particle p (Eq. 22 with rho_s cancelled): the sums
// over its bounding-box tiles are added in slot order (lane-strided, then a
// fixed xor tree), so the result does not depend on block scheduling.
// Moments about the integer reference floor(X) are shifted to the centre:
//   sum r x u = sum d x u - phi x sum u,  sum r r = sum d d - phi sum d - sum d phi + n phi phi.
template <int D>
__device__ void finalize_particle(const InstDesc& in, int p, int lane) {
    const int nt = min(in.prec[p].ntiles, in.maxk);  // overflow is flagged at publish
    double v[NPV];
#pragma unroll
    for (int k = 0; k < NPV; ++k) v[k] = 0.0;
    for (int s = lane; s < nt; s += 32) {
        const double* src = in.partial + ((long long)p * in.maxk + s) * NPV;
#pragma unroll
        for (int k = 0; k < NPV; ++k) v[k] += __ldcg(src + k);
    }
#pragma unroll
    for (int k = 0; k < NPV; ++k) v[k] = warp_sum(v[k]);
    if (lane != 0) return;
    const double cnt = v[0];
    double phi[3], X[3], Uo[3], Wo[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        X[d] = in.X[3 * p + d];
        phi[d] = d < D ? X[d] - (double)in.prec[p].ref[d] : 0.0;
    }
    if (cnt < 0.5) {  // no solid node: cannot happen inside the box for R >= 2
        atomicOr(in.status, ST_PARTICLE);
        for (int d = 0; d < 3; ++d) {
            in.Un[3 * p + d] = in.U[3 * p + d];
            in.Wn[3 * p + d] = 0.0;
        }
        in.count[p] = 0;
        return;
    }
    const double* Sd = v + 1;
    const double* Su = v + 10;
    for (int d = 0; d < 3; ++d) Uo[d] = Su[d] / cnt;
    double Lv[3] = {v[13] - (phi[1] * Su[2] - phi[2] * Su[1]),
                    v[14] - (phi[2] * Su[0] - phi[0] * Su[2]),
                    v[15] - (phi[0] * Su[1] - phi[1] * Su[0])};
    // sum r_i r_j
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
    double rr[3][3];
    for (int k = 0; k < 6; ++k) {
        const int i = ii[k], j = jj[k];
        const double val = v[4 + k] - phi[i] * Sd[j] - phi[j] * Sd[i] + cnt * phi[i] * phi[j];
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
        for (int col = 0; col < 3; ++col) {
            double M[3][3];
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) M[r][q] = (q == col) ? Lv[r] : I[r][q];
            const double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                              M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                              M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            Wo[col] = dc / det;
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
    in.Xf[4 * p + 0] = (float)X[0];  // float buffer 0 mirrors Xk buffer 0
    in.Xf[4 * p + 1] = (float)X[1];
    in.Xf[4 * p + 2] = (float)X[2];
    in.count[p] = (int)cnt;
    if (fast) atomicOr(in.status, ST_DISPLACEMENT);
}

__global__ void k_finalize(const InstDesc* __restrict__ insts, const PartRef* __restrict__ refs,
                           int ntotal, int D) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= ntotal) return;
    const PartRef r = refs[gw];
    const InstDesc& in = insts[r.inst];
    if (D == 2) finalize_particle<2>(in, r.p, lane);
    else finalize_particle<3>(in, r.p, lane);
}

// Eqs. 19-21: collision force on particle i with every particle at positions
// Xs = Xk[src] + shift * Ubar, plus its mirror images behind the walls.
// The warp's lanes split the other particles; pairs pass an FP32 distance
// filter with a margin before the FP64 evaluation.
__device__ void collision_force(const InstDesc& in, int i, int src, double shift, int lane,
                                double* F) {
    const double* Xb = in.Xk + (long long)src * in.np * 3;
    const float* Xfb = in.Xf + (long long)src * in.np * 4;
    double Xi[3];
    for (int d = 0; d < 3; ++d) Xi[d] = Xb[3 * i + d] + shift * in.Ubar[3 * i + d];
    const double Ri = in.R[i];
    const double C = (in.ratio[i] - 1.0) * in.rho_f * in.gmag;
    double Fi[3] = {0, 0, 0};
    if (C != 0.0) {
        const float xi0 = Xfb[4 * i], xi1 = Xfb[4 * i + 1], xi2 = Xfb[4 * i + 2];
        const float Rif = (float)Ri;
        for (int j = lane; j < in.np; j += 32) {
            if (j == i) continue;
            float dv0 = xi0 - Xfb[4 * j], dv1 = xi1 - Xfb[4 * j + 1], dv2 = xi2 - Xfb[4 * j + 2];
            if (in.periodic[0]) dv0 -= in.n[0] * rintf(dv0 / in.n[0]);
            if (in.periodic[1]) dv1 -= in.n[1] * rintf(dv1 / in.n[1]);
            if (in.periodic[2] && in.n[2] > 1) dv2 -= in.n[2] * rintf(dv2 / in.n[2]);
            const float lim = Rif + (float)in.R[j] + (float)in.delta + 2.5f;
            if (dv0 * dv0 + dv1 * dv1 + dv2 * dv2 > lim * lim) continue;
            // exact evaluation, operation order of the reference definition
            double dv[3];
            for (int d = 0; d < 3; ++d) {
                const double xj = Xb[3 * j + d] + shift * in.Ubar[3 * j + d];
                dv[d] = Xi[d] - xj;
                if (in.periodic[d] && in.n[d] > 1) {
                    const double half = 0.5 * in.n[d];
                    if (dv[d] > half) dv[d] -= in.n[d];
                    else if (dv[d] < -half) dv[d] += in.n[d];
                }
            }
            const double dij = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dv[0], dv[0]), __dmul_rn(dv[1], dv[1])),
                                              __dmul_rn(dv[2], dv[2])));
            const double range = Ri + in.R[j] + in.delta;
            if (dij <= range) {
                const double s = (range - dij) / in.delta;
                for (int d = 0; d < 3; ++d) Fi[d] += C / in.eps_p * dv[d] * s * s;
            }
        }
        for (int d = 0; d < 3; ++d) Fi[d] = warp_sum(Fi[d]);
        // mirror images across the wall planes -1/2 and n - 1/2
        for (int d = 0; d < 3; ++d) {
            if (in.periodic[d] || in.n[d] <= 1) continue;
            const double walls[2] = {-0.5, in.n[d] - 0.5};
            for (int face = 0; face < 2; ++face) {
                const double Xim = 2.0 * walls[face] - Xi[d];
                const double diff = Xi[d] - Xim;
                const double dprime = fabs(diff);
                const double range = 2.0 * Ri + in.delta;
                if (dprime <= range) {
                    const double s = (range - dprime) / in.delta;
                    Fi[d] += C / in.eps_w * diff * s * s;
                }
            }
        }
    }
    for (int d = 0; d < 3; ++d) F[d] = Fi[d];
}

// Record and tile-list entries of particle p at its current X and A for the
// step that reads list parity lpar.  Slots k enumerate the bounding-box tiles
// x-fastest; a periodic axis never lists the same tile twice.
__device__ void publish_particle(const InstDesc& in, int p, int lpar, int D, const Shape& sh,
                                 int lane) {
    const double R = in.R[p];
    const int T[3] = {32 * sh.vec, sh.ty, sh.tz};
    int t_lo[3], t_n[3];
    for (int d = 0; d < 3; ++d) {
        if (d >= D) {
            t_lo[d] = 0;
            t_n[d] = 1;
            continue;
        }
        const double X = in.X[3 * p + d];
        int lo = (int)floor(X - R) - 1, hi = (int)floor(X + R) + 1;
        if (!in.periodic[d]) {
            lo = max(lo, 0);
            hi = min(hi, in.n[d] - 1);
        }
        int tl = lo >= 0 ? lo / T[d] : -((-lo + T[d] - 1) / T[d]);
        int th = hi >= 0 ? hi / T[d] : -((-hi + T[d] - 1) / T[d]);
        if (th < tl) th = tl;
        int cnt = th - tl + 1;
        if (in.periodic[d] && cnt >= in.ntile[d]) {
            tl = 0;
            cnt = in.ntile[d];
        }
        t_lo[d] = tl;
        t_n[d] = cnt;
    }
    const int nt = t_n[0] * t_n[1] * t_n[2];
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
    for (int k = lane; k < nt && k < in.maxk; k += 32) {
        const int kx = k % t_n[0], ky = (k / t_n[0]) % t_n[1], kz = k / (t_n[0] * t_n[1]);
        int tc[3] = {t_lo[0] + kx, t_lo[1] + ky, t_lo[2] + kz};
        for (int d = 0; d < 3; ++d) {
            if (tc[d] < 0) tc[d] += in.ntile[d];
            if (tc[d] >= in.ntile[d]) tc[d] -= in.ntile[d];
        }
        const int local = (tc[2] * in.ntile[1] + tc[1]) * in.ntile[0] + tc[0];
        const int pos = atomicAdd(&in.list_cnt[lpar][local], 1);
        if (pos < LIST_CAP)
            in.list_ent[lpar][(long long)local * LIST_CAP + pos] = ((uint32_t)p << KBITS) | (uint32_t)k;
        else
            atomicOr(in.status, ST_CAPACITY);
    }
}

// One sub-step k of Algorithm 1 for every particle (positions Xk[src] ->
// Xk[src ^ 1]); the last sub-step also sets A^{n+1}, theta^{n+1}, U^{n-1} <-
// U^n and publishes the particle for the next step's fluid kernel.
__global__ void k_substep(const InstDesc* __restrict__ insts, const PartRef* __restrict__ refs,
                          int ntotal, int D, int src, int K, int last, int lpar, Shape sh) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= ntotal) return;
    const PartRef r = refs[gw];
    const InstDesc& in = insts[r.inst];
    const int i = r.p;
    const double h = 1.0 / K;
    double F1[3], F2[3];
    collision_force(in, i, src, 0.0, lane, F1);
    collision_force(in, i, src, h, lane, F2);
    const int dst = src ^ 1;
    double* Xd = in.Xk + (long long)dst * in.np * 3;
    const double* Xs = in.Xk + (long long)src * in.np * 3;
    const double M = in.ratio[i] * in.rho_f * (double)in.count[i];
    double Xn[3];
    for (int d = 0; d < 3; ++d) {
        const double xs = Xs[3 * i + d] + h * in.Ubar[3 * i + d];
        Xn[d] = xs + 1.0 / (2.0 * M) * h * h * 0.5 * (F1[d] + F2[d]);
    }
    if (!last) {
        if (lane == 0) {
            for (int d = 0; d < 3; ++d) Xd[3 * i + d] = Xn[d];
            float* Xf = in.Xf + (long long)dst * in.np * 4;
            Xf[4 * i] = (float)Xn[0];
            Xf[4 * i + 1] = (float)Xn[1];
            Xf[4 * i + 2] = (float)Xn[2];
        }
        return;
    }
    if (lane == 0) {
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
    __syncwarp();
    publish_particle(in, i, lpar, D, sh, lane);
}

// Publish every particle from its current state (after creation, particle
// insertion, a shape change or a state load).  Lists must be zeroed first.
__global__ void k_publish(const InstDesc* __restrict__ insts, const PartRef* __restrict__ refs,
                          int ntotal, int D, int lpar, Shape sh) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= ntotal) return;
    const PartRef r = refs[gw];
    publish_particle(insts[r.inst], r.p, lpar, D, sh, lane);
}

static unsigned warp_blocks(int n) { return (unsigned)((n + 7) / 8); }

cudaError_t launch_finalize(const InstDesc* insts, const PartRef* refs, int ntotal, int D,
                            cudaStream_t st) {
    k_finalize<<<warp_blocks(ntotal), 256, 0, st>>>(insts, refs, ntotal, D);
    return cudaGetLastError();
}

cudaError_t launch_substep(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int src,
                           int K, int last, int lpar, const Shape& sh, cudaStream_t st) {
    k_substep<<<warp_blocks(ntotal), 256, 0, st>>>(insts, refs, ntotal, D, src, K, last, lpar, sh);
    return cudaGetLastError();
}

cudaError_t launch_publish(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int lpar,
                           const Shape& sh, cudaStream_t st) {
    k_publish<<<warp_blocks(ntotal), 256, 0, st>>>(insts, refs, ntotal, D, lpar, sh);
    return cudaGetLastError();
}

}  // namespace lbmpen
