// Fused pull-scheme stream-collide-penalize kernel of lbmpen (one HBM round
// trip per time step) and the small field / population export kernels.
//
// One tile = (32 * V) x TY x TZ nodes.  Each warp takes whole x-rows of the
// tile; each lane owns V consecutive nodes and moves them with one vector
// load / store per stored population.  The +-1 shifts of pull streaming
// (Eq. 10, left side) are built from the aligned vector of the lane and one
// element passed in from the neighbouring lane by a warp shuffle, so every
// global access stays a coalesced 8/16-byte vector access.
#include "lbm_common.cuh"

namespace lbmpen {

// --------------------------------------------------------------- pulling ---
// Pull streaming of one x-row (Eq. 10, left side) in two halves so that the
// loads of the next row can be in flight while the current row collides:
// issue_q loads the lane's aligned vector of population q from the source
// row (or, on a row whose source lies beyond a wall, the node's own opposite
// population) plus the one edge element the warp cannot get by shuffling;
// assemble_q builds the shifted vector.
template <int Q, int V> struct RowBuf {
    float cur[Q - 1][V];
    float edge[Q - 1];
};

// Source row of population q for row (y, z): -1 if it lies beyond a wall.
template <int Q, int q>
__device__ __forceinline__ int src_row(const InstDesc& in, int y, int z, int* wall_axis,
                                       int* wall_face) {
    using L = Lat<Q>;
    constexpr int cy = L::c(q, 1), cz = L::c(q, 2);
    const int ny = in.n[1], nz = in.n[2];
    int ys = y - cy, zs = z - cz;
    *wall_axis = -1;
    *wall_face = 0;
    if (cy != 0 && (ys < 0 || ys >= ny)) {
        if (in.periodic[1]) ys = ys < 0 ? ys + ny : ys - ny;
        else { *wall_axis = 1; *wall_face = ys < 0 ? 0 : 1; }
    }
    if (cz != 0 && (zs < 0 || zs >= nz)) {
        if (in.periodic[2]) zs = zs < 0 ? zs + nz : zs - nz;
        else if (*wall_axis < 0) { *wall_axis = 2; *wall_face = zs < 0 ? 0 : 1; }
    }
    return *wall_axis >= 0 ? -1 : zs * ny + ys;
}

template <int Q, class S, int V, int q>
__device__ __forceinline__ void issue_q(const InstDesc& in, const S* __restrict__ fin, int xl,
                                        int y, int z, bool active, int lane, RowBuf<Q, V>& rb) {
    using L = Lat<Q>;
    constexpr int cx = L::c(q, 0);
    constexpr int qo = L::opp(q);
    const int nx = in.n[0];
    const float sl = in.s_load;
    int wa, wf;
    const int srow = src_row<Q, q>(in, y, z, &wa, &wf);
    const S* opp_row = fin + (long long)(qo - 1) * in.qstride + ((long long)z * in.n[1] + y) * in.pitch;
    rb.edge[q - 1] = 0.f;
    if (srow < 0) {
        if (active) VecIO<S, V>::load(opp_row + xl, rb.cur[q - 1], sl);
        return;
    }
    const S* row = fin + (long long)(q - 1) * in.qstride + (long long)srow * in.pitch;
    if (active) VecIO<S, V>::load(row + xl, rb.cur[q - 1], sl);
    if constexpr (cx == 1) {
        if (lane == 0 && active) {
            if (xl > 0) rb.edge[q - 1] = VecIO<S, V>::load1(row + xl - 1, sl);
            else if (in.periodic[0]) rb.edge[q - 1] = VecIO<S, V>::load1(row + nx - 1, sl);
            else rb.edge[q - 1] = VecIO<S, V>::load1(opp_row, sl) + in.wterm[0][0][q];
        }
    } else if constexpr (cx == -1) {
        if (active) {
            if (xl + V >= nx) {  // this lane holds x = nx - 1: source beyond the +x face
                if (in.periodic[0]) rb.edge[q - 1] = VecIO<S, V>::load1(row, sl);
                else rb.edge[q - 1] = VecIO<S, V>::load1(opp_row + nx - 1, sl) + in.wterm[0][1][q];
            } else if (lane == 31) {
                rb.edge[q - 1] = VecIO<S, V>::load1(row + xl + V, sl);
            }
        }
    }
}

template <int Q, int V, int q>
__device__ __forceinline__ void assemble_q(const InstDesc& in, int xl, int y, int z, bool active,
                                           int lane, const RowBuf<Q, V>& rb, float (&o)[V]) {
    using L = Lat<Q>;
    constexpr int cx = L::c(q, 0);
    const int nx = in.n[0];
    int wa, wf;
    const int srow = src_row<Q, q>(in, y, z, &wa, &wf);
    const float* cur = rb.cur[q - 1];
    if (srow < 0) {  // the whole row bounces back from a wall plane (warp-uniform)
        const float wt = in.wterm[wa][wf][q];
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = cur[e] + wt;
        return;
    }
    if constexpr (cx == 0) {
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = cur[e];
    } else if constexpr (cx == 1) {
        const float prev = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
        o[0] = lane == 0 ? rb.edge[q - 1] : prev;
#pragma unroll
        for (int e = 1; e < V; ++e) o[e] = cur[e - 1];
    } else {
        const float next = __shfl_down_sync(0xffffffffu, cur[0], 1);
#pragma unroll
        for (int e = 0; e < V - 1; ++e) o[e] = cur[e + 1];
        o[V - 1] = next;
        if (active && xl + V >= nx) {
            const int ef = nx - 1 - xl;
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (e == ef) o[e] = rb.edge[q - 1];
        } else if (lane == 31) {
            o[V - 1] = rb.edge[q - 1];
        }
    }
}

template <int Q, class S, int V, int q>
struct RowOps {
    static __device__ __forceinline__ void issue(const InstDesc& in, const S* fin, int xl, int y,
                                                 int z, bool active, int lane, RowBuf<Q, V>& rb) {
        issue_q<Q, S, V, q>(in, fin, xl, y, z, active, lane, rb);
        RowOps<Q, S, V, q + 1>::issue(in, fin, xl, y, z, active, lane, rb);
    }
    static __device__ __forceinline__ void assemble(const InstDesc& in, int xl, int y, int z,
                                                    bool active, int lane, const RowBuf<Q, V>& rb,
                                                    float (*f)[V]) {
        assemble_q<Q, V, q>(in, xl, y, z, active, lane, rb, f[q - 1]);
        RowOps<Q, S, V, q + 1>::assemble(in, xl, y, z, active, lane, rb, f);
    }
};
template <int Q_, class S, int V>
struct RowOps<Q_, S, V, Q_> {
    static __device__ __forceinline__ void issue(const InstDesc&, const S*, int, int, int, bool, int,
                                                 RowBuf<Q_, V>&) {}
    static __device__ __forceinline__ void assemble(const InstDesc&, int, int, int, bool, int,
                                                    const RowBuf<Q_, V>&, float (*)[V]) {}
};

// ------------------------------------------------------------ fused step ---
// Shared memory of a tile: the candidate particles.
constexpr int SMEM_BYTES = (int)sizeof(Cand) * LIST_CAP;

template <int Q, class S, int V>
__device__ __forceinline__ void fluid_tile(const InstDesc& in, int local, int par, const Shape& sh,
                                           bool commit, unsigned char* smem) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int QS = Q - 1;
    const int tw = 32 * V;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    Cand* cand = reinterpret_cast<Cand*>(smem);
    const Geo geo = make_geo(in);
    const CollK ck = make_collk<Q>(make_collp(in));
    float* const ubox = commit ? in.ubox : in.ubox_scratch;

    const int ntx = in.ntile[0], nty = in.ntile[1];
    const int tx = local % ntx, rest = local / ntx;
    const int x0 = tx * tw, y0 = (rest % nty) * sh.ty, z0 = (rest / nty) * sh.tz;
    const int rows = sh.ty * sh.tz;
    const S* __restrict__ fin = static_cast<const S*>(in.f[par]);
    S* __restrict__ fout = static_cast<S*>(in.f[par ^ 1]);
    const int xl = x0 + lane * V;
    const bool active = xl < in.n[0];

    // 1. loads of this warp's first row go out before the candidate prologue
    RowBuf<Q, V> rb;
    int r = warp;
    {
        const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
        if (r < rows && y < in.n[1] && z < in.n[2])
            RowOps<Q, S, V, 1>::issue(in, fin, xl, y, z, active, lane, rb);
    }
    // 2. candidate particles of the tile
    int ncand = 0;
    if (in.np > 0) {
        ncand = min(in.list_cnt[par][local], LIST_CAP);
        for (int c = tid; c < ncand; c += blockDim.x) {
            const uint32_t e = in.list_ent[par][(long long)local * LIST_CAP + c];
            const int p = (int)(e >> KBITS);
            const PRec& pr = in.prec[p];
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
            const int2 bi = in.boxinfo[p];
            cd.boff = bi.x;
            cd.bh = bi.y;
            cd.shape = pr.shape;
            cand[c] = cd;
        }
        if (commit && tid == 0) in.list_cnt[par ^ 1][local] = 0;
    }
    __syncthreads();

    // 3. rows: assemble, prefetch the next row, collide, store, reduce
    bool bad = false;
    for (; r < rows; r += nwarps) {
        const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
        if (y >= in.n[1] || z >= in.n[2]) continue;
        float f[QS][V];
        RowOps<Q, S, V, 1>::assemble(in, xl, y, z, active, lane, rb, f);
        {
            const int rn = r + nwarps;
            const int yn = y0 + rn % sh.ty, zn = z0 + rn / sh.ty;
            if (rn < rows && yn < in.n[1] && zn < in.n[2])
                RowOps<Q, S, V, 1>::issue(in, fin, xl, yn, zn, active, lane, rb);
        }
        int slot[V];
        float uv[3][V];
        // nodes in pairs: packed FP32x2 collision (same bits as the TMA path)
        constexpr int PAIR = V >= 2 ? 2 : 1;
#pragma unroll
        for (int e = 0; e < V; e += PAIR) {
            int own[2] = {-1, -1}, sl[2] = {-1, -1};
            float2 a2[3], f2v[QS], u2[3], p2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ee = PAIR == 2 ? e + h : e;
                const int xyz[3] = {xl + ee, y, z};
                if (ncand > 0) own[h] = owner_of<D>(geo, cand, ncand, xyz, &sl[h]);
            }
#pragma unroll
            for (int d = 0; d < 3; ++d)
                a2[d] = add2(bc2(in.gdrive[d]), make_float2(own[0] >= 0 ? cand[sl[0]].a[d] : 0.f,
                                                            own[1] >= 0 ? cand[sl[1]].a[d] : 0.f));
#pragma unroll
            for (int q = 0; q < QS; ++q) f2v[q] = make_float2(f[q][e], f[q][PAIR == 2 ? e + 1 : e]);
            collide2<Q>(f2v, a2, own[0] >= 0, own[1] >= 0, ck, u2, &p2);
#pragma unroll
            for (int h = 0; h < PAIR; ++h) {
                const int ee = e + h;
#pragma unroll
                for (int q = 0; q < QS; ++q) f[q][ee] = h ? f2v[q].y : f2v[q].x;
                const float u[3] = {h ? u2[0].y : u2[0].x, h ? u2[1].y : u2[1].x, h ? u2[2].y : u2[2].x};
                float uu = 0.f;
#pragma unroll
                for (int d = 0; d < D; ++d) uu = fmaf(u[d], u[d], uu);
                const bool valid = active && (xl + ee < in.n[0]);
                if (valid && !(uu < 0.25f)) bad = true;
                slot[ee] = valid ? sl[h] : -1;
#pragma unroll
                for (int d = 0; d < 3; ++d) uv[d][ee] = d < D ? u[d] : 0.f;
            }
        }
        if (active) {
            const long long off = ((long long)z * in.n[1] + y) * in.pitch + xl;
#pragma unroll
            for (int q = 0; q < QS; ++q)
                VecIO<S, V>::store(fout + (long long)q * in.qstride + off, f[q], in.s_store);
        }
        if (ncand > 0) {  // the solid nodes' velocities into their particles' boxes (Eq. 22)
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (slot[e] >= 0) box_store<D>(ubox, geo, cand[slot[e]], xl + e, y, z, uv[0][e], uv[1][e], uv[2][e]);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(in.status, ST_DIVERGED);
}

template <int Q, class S, int V>
__global__ void __launch_bounds__(256) k_fluid(const InstDesc* __restrict__ insts,
                                               const uint16_t* __restrict__ tile_inst,
                                               int ntiles, int par, Shape sh, int commit,
                                               int persistent, int* tile_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (!persistent) {
        const int t = blockIdx.x;
        const InstDesc& in = insts[tile_inst[t]];
        fluid_tile<Q, S, V>(in, t - in.tile0, par, sh, commit != 0, smem);
        return;
    }
    __shared__ int s_t;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(&tile_ctr[0], 1);
        __syncthreads();
        const int t = s_t;
        __syncthreads();
        if (t >= ntiles) break;
        const InstDesc& in = insts[tile_inst[t]];
        fluid_tile<Q, S, V>(in, t - in.tile0, par, sh, commit != 0, smem);
        __syncthreads();
    }
    // the last block to leave resets the work counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        const int done = atomicAdd(&tile_ctr[1], 1);
        if (done == (int)gridDim.x - 1) {
            tile_ctr[0] = 0;
            tile_ctr[1] = 0;
        }
    }
}

// u, p, owner of every node of one instance (no collision, state unchanged).
template <int Q, class S>
__global__ void k_fields(const InstDesc* __restrict__ insts, int inst, int par, Shape sh, float* u,
                         float* pout, int* owner) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    const InstDesc& in = insts[inst];
    const long long N = (long long)in.n[0] * in.n[1] * in.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int x = (int)(i % in.n[0]), y = (int)((i / in.n[0]) % in.n[1]),
              z = (int)(i / ((long long)in.n[0] * in.n[1]));
    const S* fin = static_cast<const S*>(in.f[par]);
    float f[Q - 1];
    for (int q = 1; q < Q; ++q) f[q - 1] = pull_scalar<Q, S>(in, fin, q, x, y, z);
    // owner through the same tile candidate lists the fused kernel uses
    int own = -1;
    float a[3] = {in.gdrive[0], in.gdrive[1], in.gdrive[2]};
    if (in.np > 0) {
        const Geo geo = make_geo(in);
        const int tw = sh.tw;
        const int local = (z / sh.tz * in.ntile[1] + y / sh.ty) * in.ntile[0] + x / tw;
        const int nc = min(in.list_cnt[par][local], LIST_CAP);
        const int xyz[3] = {x, y, z};
        for (int c = 0; c < nc; ++c) {
            const uint32_t e = in.list_ent[par][(long long)local * LIST_CAP + c];
            const int p = (int)(e >> KBITS);
            if (own >= 0 && p > own) continue;
            if (inside_exact<D>(geo, in.prec[p], xyz)) own = p;
        }
        if (own >= 0)
            for (int d = 0; d < 3; ++d) a[d] += in.prec[own].a[d];
    }
    float m[3] = {0, 0, 0}, s = 0.f;
    for (int q = 1; q < Q; ++q) {
        s += f[q - 1];
        for (int d = 0; d < D; ++d) m[d] += L::c(q, d) * f[q - 1];
    }
    float uu = 0.f;
    for (int d = 0; d < D; ++d) {
        const float ud = m[d] + 0.5f * a[d];
        uu += ud * ud;
        if (u) u[(long long)d * N + i] = ud;
    }
    if (pout) pout[i] = (s - (float)(1.5 - 0.5 * L::SUMA) * uu) * (float)(1.0 / L::SUMA);
    if (owner) owner[i] = own;
}

// populations between the dense [Q][N] FP32 exchange layout and storage
template <class S>
__global__ void k_pack(const InstDesc* __restrict__ insts, int inst, int par, int Q,
                       const float* __restrict__ src) {
    const InstDesc& in = insts[inst];
    const long long N = (long long)in.n[0] * in.n[1] * in.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * (Q - 1)) return;
    const int q = (int)(i / N) + 1;
    const long long node = i % N;
    const int x = (int)(node % in.n[0]);
    const long long row = node / in.n[0];
    S* f = static_cast<S*>(in.f[par]);
    f[(long long)(q - 1) * in.qstride + row * in.pitch + x] = to_store<S>(src[q * N + node], in.s_store);
}

template <class S>
__global__ void k_unpack(const InstDesc* __restrict__ insts, int inst, int par, int Q,
                         float* __restrict__ dst) {
    const InstDesc& in = insts[inst];
    const long long N = (long long)in.n[0] * in.n[1] * in.n[2];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * Q) return;
    const int q = (int)(i / N);
    const long long node = i % N;
    if (q == 0) {
        dst[i] = 0.f;
        return;
    }
    const int x = (int)(node % in.n[0]);
    const long long row = node / in.n[0];
    const S* f = static_cast<const S*>(in.f[par]);
    dst[i] = VecIO<S, 1 + (sizeof(S) == 2)>::load1(f + (long long)(q - 1) * in.qstride + row * in.pitch + x,
                                                   in.s_load);
}

// ------------------------------------------------------------ host entry ---
template <int Q, class S, int V>
static cudaError_t launch_fluid_v(const InstDesc* insts, const uint16_t* tile_inst, int ntiles,
                                  int par, const Shape& sh, int commit, int persistent, int grid,
                                  int* tile_ctr, cudaStream_t st) {
    auto kern = k_fluid<Q, S, V>;
    const int g = persistent ? grid : ntiles;
    kern<<<g, 32 * sh.warps, SMEM_BYTES, st>>>(insts, tile_inst, ntiles, par, sh, commit, persistent,
                                            tile_ctr);
    return cudaGetLastError();
}

cudaError_t launch_fluid(int Q, int fp16, const InstDesc* insts, const uint16_t* tile_inst,
                         int ntiles, int par, const Shape& sh, int commit, int persistent, int grid,
                         int* tile_ctr, cudaStream_t st) {
#define LBM_CASE(QQ, SS, VV)                                                                    \
    if (Q == QQ && sh.vec == VV)                                                                \
        return launch_fluid_v<QQ, SS, VV>(insts, tile_inst, ntiles, par, sh, commit, persistent, \
                                          grid, tile_ctr, st);
    if (!fp16) {
        LBM_CASE(9, float, 1) LBM_CASE(9, float, 2) LBM_CASE(9, float, 4)
        LBM_CASE(19, float, 1) LBM_CASE(19, float, 2) LBM_CASE(19, float, 4)
    } else {
        LBM_CASE(9, __half, 2) LBM_CASE(9, __half, 4) LBM_CASE(9, __half, 8)
        LBM_CASE(19, __half, 2) LBM_CASE(19, __half, 4) LBM_CASE(19, __half, 8)
    }
#undef LBM_CASE
    return cudaErrorInvalidValue;
}

int fluid_max_blocks_per_sm(int Q, int fp16, const Shape& sh) {
    int nb = 0;
#define LBM_OCC(QQ, SS, VV)                                                                         \
    if (Q == QQ && sh.vec == VV) {                                                                  \
        cudaFuncSetAttribute(k_fluid<QQ, SS, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES); \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fluid<QQ, SS, VV>, 32 * sh.warps, SMEM_BYTES); \
        return nb;                                                                                  \
    }
    if (!fp16) {
        LBM_OCC(9, float, 1) LBM_OCC(9, float, 2) LBM_OCC(9, float, 4)
        LBM_OCC(19, float, 1) LBM_OCC(19, float, 2) LBM_OCC(19, float, 4)
    } else {
        LBM_OCC(9, __half, 2) LBM_OCC(9, __half, 4) LBM_OCC(9, __half, 8)
        LBM_OCC(19, __half, 2) LBM_OCC(19, __half, 4) LBM_OCC(19, __half, 8)
    }
#undef LBM_OCC
    return 0;
}

cudaError_t launch_fields(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                          const Shape& sh, float* u, float* p, int* owner, cudaStream_t st) {
    const int thr = 256;
    const unsigned blocks = (unsigned)((N + thr - 1) / thr);
    if (Q == 9 && !fp16) k_fields<9, float><<<blocks, thr, 0, st>>>(insts, inst, par, sh, u, p, owner);
    else if (Q == 9) k_fields<9, __half><<<blocks, thr, 0, st>>>(insts, inst, par, sh, u, p, owner);
    else if (!fp16) k_fields<19, float><<<blocks, thr, 0, st>>>(insts, inst, par, sh, u, p, owner);
    else k_fields<19, __half><<<blocks, thr, 0, st>>>(insts, inst, par, sh, u, p, owner);
    return cudaGetLastError();
}

cudaError_t launch_pack(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                        const float* src, cudaStream_t st) {
    const int thr = 256;
    const unsigned blocks = (unsigned)((N * (Q - 1) + thr - 1) / thr);
    if (!fp16) k_pack<float><<<blocks, thr, 0, st>>>(insts, inst, par, Q, src);
    else k_pack<__half><<<blocks, thr, 0, st>>>(insts, inst, par, Q, src);
    return cudaGetLastError();
}

cudaError_t launch_unpack(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                          float* dst, cudaStream_t st) {
    const int thr = 256;
    const unsigned blocks = (unsigned)((N * Q + thr - 1) / thr);
    if (!fp16) k_unpack<float><<<blocks, thr, 0, st>>>(insts, inst, par, Q, dst);
    else k_unpack<__half><<<blocks, thr, 0, st>>>(insts, inst, par, Q, dst);
    return cudaGetLastError();
}

}  // namespace lbmpen
