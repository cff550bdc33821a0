// Fused pull-scheme stream-collide-penalize kernel of lbmpen (one HBM round
// trip per time step) and the small field / population export kernels.
//
// One tile = (32 * V) x TY x TZ nodes.  Each warp takes whole x-rows of the
// tile; each lane owns V consecutive nodes and moves them with one vector
// load / store per stored population.  The +-1 shifts of pull streaming
// (Eq. 10, left side) are built from the aligned vector of the lane and one
// element passed in from the neighbouring lane by a warp shuffle, so every
// global access stays a coalesced 8/16-byte vector access.
#include "lbm_internal.cuh"

namespace lbmpen {

// ------------------------------------------------------------ vector I/O ---
template <class S, int V> struct VecIO;

template <int V> struct VecIO<float, V> {
    static __device__ __forceinline__ void load(const float* p, float (&o)[V], float) {
        if constexpr (V == 1) {
            o[0] = __ldg(p);
        } else if constexpr (V == 2) {
            float2 t = __ldg(reinterpret_cast<const float2*>(p));
            o[0] = t.x; o[1] = t.y;
        } else {
            static_assert(V == 4, "fp32 vector width");
            float4 t = __ldg(reinterpret_cast<const float4*>(p));
            o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
        }
    }
    static __device__ __forceinline__ void store(float* p, const float (&v)[V], float) {
        if constexpr (V == 1) {
            p[0] = v[0];
        } else if constexpr (V == 2) {
            *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
        } else {
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
    static __device__ __forceinline__ float load1(const float* p, float) { return __ldg(p); }
};

template <int V> struct VecIO<__half, V> {
    static_assert(V == 2 || V == 4 || V == 8, "fp16 vector width");
    static __device__ __forceinline__ void load(const __half* p, float (&o)[V], float s) {
        if constexpr (V == 2) {
            unsigned int t = __ldg(reinterpret_cast<const unsigned int*>(p));
            float2 a = __half22float2(*reinterpret_cast<__half2*>(&t));
            o[0] = a.x * s; o[1] = a.y * s;
        } else if constexpr (V == 4) {
            uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
            float2 a = __half22float2(*reinterpret_cast<__half2*>(&t.x));
            float2 b = __half22float2(*reinterpret_cast<__half2*>(&t.y));
            o[0] = a.x * s; o[1] = a.y * s; o[2] = b.x * s; o[3] = b.y * s;
        } else {
            uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
            unsigned int w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 a = __half22float2(*reinterpret_cast<__half2*>(&w[i]));
                o[2 * i] = a.x * s; o[2 * i + 1] = a.y * s;
            }
        }
    }
    static __device__ __forceinline__ void store(__half* p, const float (&v)[V], float s) {
        unsigned int w[V / 2];
#pragma unroll
        for (int i = 0; i < V / 2; ++i) {
            __half2 h = __floats2half2_rn(v[2 * i] * s, v[2 * i + 1] * s);
            w[i] = *reinterpret_cast<unsigned int*>(&h);
        }
        if constexpr (V == 2) {
            *reinterpret_cast<unsigned int*>(p) = w[0];
        } else if constexpr (V == 4) {
            *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        } else {
            *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    static __device__ __forceinline__ float load1(const __half* p, float s) {
        return __half2float(p[0]) * s;
    }
};

template <class S> __device__ __forceinline__ S to_store(float v, float s);
template <> __device__ __forceinline__ float to_store<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v, float s) {
    return __float2half_rn(v * s);
}

// -------------------------------------------------------- indicator test ---
// Candidate particle of a tile, staged in shared memory.
struct Cand {
    int ref[3];
    float frac[3];
    float R2lo, R2hi;
    float a[3];
    int p;  // particle index within the instance
    int k;  // partial slot of this tile in the particle's bounding box
};

__device__ __forceinline__ int wrap_int(int d, int n, int per) {
    if (per) {
        int h = n >> 1;
        if (d > h) d -= n;
        else if (d < -h) d += n;
    }
    return d;
}

// Exact FP64 form of Eq. 9 on the lattice, identical operation by operation
// to the reference definition: d2 = ((0 + dx*dx) + dy*dy) + dz*dz with each
// dx = x - X_d taken to the minimum image on periodic axes, then d2 <= R*R.
// Separate roundings (no fused multiply-add) via the _rn intrinsics.
template <int D>
__device__ __noinline__ bool inside_exact(const InstDesc& in, const PRec& pr, const int* xyz) {
    double d2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        double dx = __dsub_rn((double)xyz[d], pr.X[d]);
        if (in.periodic[d]) {
            double half = 0.5 * (double)in.n[d];
            if (dx > half) dx = __dsub_rn(dx, (double)in.n[d]);
            else if (dx < -half) dx = __dadd_rn(dx, (double)in.n[d]);
        }
        d2 = __dadd_rn(d2, __dmul_rn(dx, dx));
    }
    return d2 <= pr.R2;
}

// Owner of a node among the tile's candidates: lowest particle index whose
// solid domain holds the node, or -1.  Float filter with a safety band; nodes
// in the band take the exact FP64 test.
template <int D>
__device__ __forceinline__ int owner_of(const InstDesc& in, const Cand* cand, int ncand,
                                        const int* xyz, int* slot) {
    int best = -1, bslot = -1;
    for (int c = 0; c < ncand; ++c) {
        const Cand& cd = cand[c];
        if (best >= 0 && cd.p > best) continue;
        float d2 = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            int di = wrap_int(xyz[d] - cd.ref[d], in.n[d], in.periodic[d]);
            float dx = (float)di - cd.frac[d];
            d2 = fmaf(dx, dx, d2);
        }
        bool inside;
        if (d2 < cd.R2lo) inside = true;
        else if (d2 > cd.R2hi) inside = false;
        else inside = inside_exact<D>(in, in.prec[cd.p], xyz);
        if (inside && (best < 0 || cd.p < best)) {
            best = cd.p;
            bslot = c;
        }
    }
    *slot = bslot;
    return best;
}

// ------------------------------------------------------------- collision ---
// BGK with Guo forcing (Eqs. 10, 13, 14) and, on solid nodes, the penalty
// source of Eq. 17.  f holds the stored populations q = 1..Q-1 (index q-1)
// of one node after streaming; on return it holds f* of the same node.
template <int Q>
__device__ __forceinline__ void collide(float* f, const float* a, bool solid, const InstDesc& in,
                                        float* u_out, float* p_out) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr float w0 = L::w(0);
    float m[3] = {0.f, 0.f, 0.f}, s = 0.f;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        s += f[q - 1];
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (L::c(q, d) != 0) m[d] += L::c(q, d) > 0 ? f[q - 1] : -f[q - 1];
    }
    float u[3] = {0.f, 0.f, 0.f}, uu = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        u[d] = m[d] + 0.5f * a[d];  // Eq. 15a
        uu = fmaf(u[d], u[d], uu);
    }
    const float p = (s * (1.0f / 3.0f) - 0.5f * w0 * uu) * (1.0f / (1.0f - w0));  // Eq. 15b
#pragma unroll
    for (int d = 0; d < D; ++d) u_out[d] = u[d];
    *p_out = p;
    float ua = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) ua = fmaf(u[d], a[d], ua);

    // Pi_neq = sum (f - feq) c c on solid nodes (Eq. 16 with the dyad)
    float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // xx yy zz xy xz yz
    float feq[Q - 1];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        float cu = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (L::c(q, d) != 0) cu += L::c(q, d) > 0 ? u[d] : -u[d];
        feq[q - 1] = L::w(q) * (3.0f * p + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);  // Eq. 13
        if (solid) {
            const float fn = f[q - 1] - feq[q - 1];
            const int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
            if (cx) P[0] += fn;
            if (cy) P[1] += fn;
            if (cz) P[2] += fn;
            if (cx * cy) P[3] += cx * cy > 0 ? fn : -fn;
            if (cx * cz) P[4] += cx * cz > 0 ? fn : -fn;
            if (cy * cz) P[5] += cy * cz > 0 ? fn : -fn;
        }
    }
    const float trP = (P[0] + P[1] + P[2]) * (1.0f / 3.0f);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
        float cu = 0.f, ca = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            if (L::c(q, d) != 0) {
                cu += L::c(q, d) > 0 ? u[d] : -u[d];
                ca += L::c(q, d) > 0 ? a[d] : -a[d];
            }
        }
        // Eq. 14: (1 - 1/2tau) w [3 (c - u).a + 9 (c.u)(c.a)]
        const float Fq = in.fpref * L::w(q) * (3.0f * (ca - ua) + 9.0f * cu * ca);
        float out = feq[q - 1] + in.keep * (f[q - 1] - feq[q - 1]) + Fq;
        if (solid) {
            // Eq. 17: w/(2 cs^4) alpha Pi:(c c - cs^2 I) = 4.5 w alpha (Pi:cc - tr Pi / 3)
            float pcc = 0.f;
            if (cx) pcc += P[0];
            if (cy) pcc += P[1];
            if (cz) pcc += P[2];
            if (cx * cy) pcc += 2.0f * (cx * cy > 0 ? P[3] : -P[3]);
            if (cx * cz) pcc += 2.0f * (cx * cz > 0 ? P[4] : -P[4]);
            if (cy * cz) pcc += 2.0f * (cy * cz > 0 ? P[5] : -P[5]);
            out += 4.5f * L::w(q) * in.alpha * (pcc - trP);
        }
        f[q - 1] = out;
    }
}

// --------------------------------------------------------------- pulling ---
// Pull population q for the V nodes x = xl .. xl+V-1 of row (y, z).
template <int Q, class S, int V, int q>
__device__ __forceinline__ void pull_q(const InstDesc& in, const S* __restrict__ fin, int xl, int y,
                                       int z, bool active, int lane, float (&o)[V]) {
    using L = Lat<Q>;
    constexpr int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
    constexpr int qo = L::opp(q);
    const int nx = in.n[0], ny = in.n[1], nz = in.n[2];
    const float sl = in.s_load;
    int ys = y - cy, zs = z - cz;
    int wall_axis = -1, wall_face = 0;
    if (cy != 0 && (ys < 0 || ys >= ny)) {
        if (in.periodic[1]) ys = ys < 0 ? ys + ny : ys - ny;
        else { wall_axis = 1; wall_face = ys < 0 ? 0 : 1; }
    }
    if (cz != 0 && (zs < 0 || zs >= nz)) {
        if (in.periodic[2]) zs = zs < 0 ? zs + nz : zs - nz;
        else if (wall_axis < 0) { wall_axis = 2; wall_face = zs < 0 ? 0 : 1; }
    }
    const long long own_row = ((long long)z * ny + y) * in.pitch;
    const S* opp_row = fin + (long long)(qo - 1) * in.qstride + own_row;
    if (wall_axis >= 0) {
        // the whole row bounces back from a wall plane (warp-uniform branch)
        if (active) VecIO<S, V>::load(opp_row + xl, o, sl);
        const float wt = in.wterm[wall_axis][wall_face][q];
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] += wt;
        return;
    }
    const S* row = fin + (long long)(q - 1) * in.qstride + ((long long)zs * ny + ys) * in.pitch;
    float cur[V];
    if (active) VecIO<S, V>::load(row + xl, cur, sl);
    else {
#pragma unroll
        for (int e = 0; e < V; ++e) cur[e] = 0.f;
    }
    if constexpr (cx == 0) {
#pragma unroll
        for (int e = 0; e < V; ++e) o[e] = cur[e];
    } else if constexpr (cx == 1) {
        float prev = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
        if (lane == 0 && active) {
            if (xl > 0) prev = VecIO<S, V>::load1(row + xl - 1, sl);
            else if (in.periodic[0]) prev = VecIO<S, V>::load1(row + nx - 1, sl);
            else prev = VecIO<S, V>::load1(opp_row, sl) + in.wterm[0][0][q];
        }
        o[0] = prev;
#pragma unroll
        for (int e = 1; e < V; ++e) o[e] = cur[e - 1];
    } else {
        float next = __shfl_down_sync(0xffffffffu, cur[0], 1);
#pragma unroll
        for (int e = 0; e < V - 1; ++e) o[e] = cur[e + 1];
        o[V - 1] = next;
        if (active && lane == 31 && xl + V < nx) o[V - 1] = VecIO<S, V>::load1(row + xl + V, sl);
        if (active && xl + V >= nx) {
            // this lane holds x = nx - 1: its source lies beyond the +x face
            const int e = nx - 1 - xl;
            float v;
            if (in.periodic[0]) v = VecIO<S, V>::load1(row, sl);
            else v = VecIO<S, V>::load1(opp_row + nx - 1, sl) + in.wterm[0][1][q];
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (i == e) o[i] = v;
        }
    }
}

template <int Q, class S, int V, int q>
struct PullAll {
    static __device__ __forceinline__ void run(const InstDesc& in, const S* fin, int xl, int y,
                                               int z, bool active, int lane, float (*f)[V]) {
        pull_q<Q, S, V, q>(in, fin, xl, y, z, active, lane, f[q - 1]);
        PullAll<Q, S, V, q + 1>::run(in, fin, xl, y, z, active, lane, f);
    }
};
template <int S_, class S, int V>
struct PullAll<S_, S, V, S_> {
    static __device__ __forceinline__ void run(const InstDesc&, const S*, int, int, int, bool, int,
                                               float (*)[V]) {}
};

// ------------------------------------------------------------ fused step ---
// Shared memory: candidates, then per-node velocity and owner slot for the
// tile reduction, then block-reduction scratch.
struct SmemLayout {
    int cand_off, u_off, slot_off, red_off, bytes;
};

__host__ __device__ inline SmemLayout smem_layout(const Shape& sh, int D, int nwarps) {
    SmemLayout L;
    int nodes = 32 * sh.vec * sh.ty * sh.tz;
    L.cand_off = 0;
    L.u_off = (int)sizeof(Cand) * LIST_CAP;
    L.slot_off = L.u_off + 4 * D * nodes;
    L.red_off = (L.slot_off + nodes + 15) & ~15;
    L.bytes = L.red_off + 8 * NPV * nwarps + 16;
    return L;
}

template <int D>
__device__ void tile_partials(const InstDesc& in, const Cand* cand, int ncand, const float* su,
                              const signed char* sslot, double* red, int nodes, int tw, int ty,
                              int x0, int y0, int z0) {
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthr >> 5;
    for (int c = 0; c < ncand; ++c) {
        const Cand cd = cand[c];
        int icnt = 0, id[3] = {0, 0, 0}, idd[6] = {0, 0, 0, 0, 0, 0};
        double su_[3] = {0, 0, 0}, sl_[3] = {0, 0, 0};
        for (int i = tid; i < nodes; i += nthr) {
            if (sslot[i] != c) continue;
            const int xx = x0 + i % tw, rr = i / tw;
            const int xyz[3] = {xx, y0 + rr % ty, z0 + rr / ty};
            int d[3] = {0, 0, 0};
            double u[3] = {0, 0, 0};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                d[k] = wrap_int(xyz[k] - cd.ref[k], in.n[k], in.periodic[k]);
                u[k] = (double)su[k * nodes + i];
            }
            icnt += 1;
#pragma unroll
            for (int k = 0; k < 3; ++k) id[k] += d[k];
            idd[0] += d[0] * d[0]; idd[1] += d[1] * d[1]; idd[2] += d[2] * d[2];
            idd[3] += d[0] * d[1]; idd[4] += d[0] * d[2]; idd[5] += d[1] * d[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) su_[k] += u[k];
            sl_[0] += (double)d[1] * u[2] - (double)d[2] * u[1];
            sl_[1] += (double)d[2] * u[0] - (double)d[0] * u[2];
            sl_[2] += (double)d[0] * u[1] - (double)d[1] * u[0];
        }
        // fixed-order block reduction: warp tree, then warps in index order
        double v[NPV];
        v[0] = __reduce_add_sync(0xffffffffu, icnt);
#pragma unroll
        for (int k = 0; k < 3; ++k) v[1 + k] = __reduce_add_sync(0xffffffffu, id[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) v[4 + k] = __reduce_add_sync(0xffffffffu, idd[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double a = su_[k], b = sl_[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            }
            v[10 + k] = a;
            v[13 + k] = b;
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NPV; ++k) red[warp * NPV + k] = v[k];
        }
        __syncthreads();
        if (tid < NPV) {
            double acc = 0.0;
            for (int w = 0; w < nwarps; ++w) acc += red[w * NPV + tid];
            in.partial[((long long)cd.p * in.maxk + cd.k) * NPV + tid] = acc;
        }
        __syncthreads();
    }
}

template <int Q, class S, int V>
__device__ __forceinline__ void fluid_tile(const InstDesc& in, int local, int par, const Shape& sh,
                                           bool commit, unsigned char* smem) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int QS = Q - 1;
    const int tw = 32 * V;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const SmemLayout SL = smem_layout(sh, D, nwarps);
    Cand* cand = reinterpret_cast<Cand*>(smem + SL.cand_off);
    float* su = reinterpret_cast<float*>(smem + SL.u_off);
    signed char* sslot = reinterpret_cast<signed char*>(smem + SL.slot_off);
    double* red = reinterpret_cast<double*>(smem + SL.red_off);
    const int nodes = tw * sh.ty * sh.tz;

    const int ntx = in.ntile[0], nty = in.ntile[1];
    const int tx = local % ntx, rest = local / ntx;
    const int x0 = tx * tw, y0 = (rest % nty) * sh.ty, z0 = (rest / nty) * sh.tz;

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
            cand[c] = cd;
        }
        if (commit && tid == 0) in.list_cnt[par ^ 1][local] = 0;
    }
    __syncthreads();

    const S* __restrict__ fin = static_cast<const S*>(in.f[par]);
    S* __restrict__ fout = static_cast<S*>(in.f[par ^ 1]);
    const int rows = sh.ty * sh.tz;
    bool bad = false;
    for (int r = warp; r < rows; r += nwarps) {
        const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
        if (y >= in.n[1] || z >= in.n[2]) {
            if (ncand > 0)
                for (int e = 0; e < V; ++e) sslot[r * tw + lane * V + e] = -1;
            continue;
        }
        const int xl = x0 + lane * V;
        const bool active = xl < in.n[0];
        float f[QS][V];
        PullAll<Q, S, V, 1>::run(in, fin, xl, y, z, active, lane, f);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int xyz[3] = {xl + e, y, z};
            int slot = -1, own = -1;
            if (ncand > 0) own = owner_of<D>(in, cand, ncand, xyz, &slot);
            float a[3] = {in.gdrive[0], in.gdrive[1], in.gdrive[2]};
            if (own >= 0) {
#pragma unroll
                for (int d = 0; d < 3; ++d) a[d] += cand[slot].a[d];
            }
            float fn[QS];
#pragma unroll
            for (int q = 0; q < QS; ++q) fn[q] = f[q][e];
            float u[3], p;
            collide<Q>(fn, a, own >= 0, in, u, &p);
#pragma unroll
            for (int q = 0; q < QS; ++q) f[q][e] = fn[q];
            float uu = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) uu = fmaf(u[d], u[d], uu);
            if (active && xl + e < in.n[0] && !(uu < 0.25f)) bad = true;
            if (ncand > 0) {
                const int i = r * tw + lane * V + e;
                const bool valid = active && (xl + e < in.n[0]);
                sslot[i] = valid ? (signed char)slot : (signed char)-1;
#pragma unroll
                for (int d = 0; d < D; ++d) su[d * nodes + i] = u[d];
            }
        }
        if (active) {
            const long long off = ((long long)z * in.n[1] + y) * in.pitch + xl;
#pragma unroll
            for (int q = 0; q < QS; ++q)
                VecIO<S, V>::store(fout + (long long)q * in.qstride + off, f[q], in.s_store);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(in.status, ST_DIVERGED);
    if (ncand > 0) {
        __syncthreads();
        tile_partials<D>(in, cand, ncand, su, sslot, red, nodes, tw, sh.ty, x0, y0, z0);
    }
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

// ------------------------------------------------------ field export -------
template <int Q, class S>
__device__ float pull_scalar(const InstDesc& in, const S* fin, int q, int x, int y, int z) {
    using L = Lat<Q>;
    const int c[3] = {L::c(q, 0), L::c(q, 1), L::c(q, 2)};
    int src[3] = {x - c[0], y - c[1], z - c[2]};
    int axis = -1, face = 0;
    for (int d = 0; d < 3; ++d) {
        if (src[d] < 0 || src[d] >= in.n[d]) {
            if (in.periodic[d]) src[d] = src[d] < 0 ? src[d] + in.n[d] : src[d] - in.n[d];
            else if (axis < 0) { axis = d; face = src[d] < 0 ? 0 : 1; }
        }
    }
    if (axis >= 0) {
        const int qo = L::opp(q);
        const long long off = ((long long)z * in.n[1] + y) * in.pitch + x;
        return VecIO<S, 1 + (sizeof(S) == 2)>::load1(fin + (long long)(qo - 1) * in.qstride + off,
                                                       in.s_load) + in.wterm[axis][face][q];
    }
    const long long off = ((long long)src[2] * in.n[1] + src[1]) * in.pitch + src[0];
    return VecIO<S, 1 + (sizeof(S) == 2)>::load1(fin + (long long)(q - 1) * in.qstride + off, in.s_load);
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
        const int tw = 32 * sh.vec;
        const int local = (z / sh.tz * in.ntile[1] + y / sh.ty) * in.ntile[0] + x / tw;
        const int nc = min(in.list_cnt[par][local], LIST_CAP);
        const int xyz[3] = {x, y, z};
        for (int c = 0; c < nc; ++c) {
            const uint32_t e = in.list_ent[par][(long long)local * LIST_CAP + c];
            const int p = (int)(e >> KBITS);
            if (own >= 0 && p > own) continue;
            if (inside_exact<D>(in, in.prec[p], xyz)) own = p;
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
    constexpr float w0 = L::w(0);
    if (pout) pout[i] = (s * (1.0f / 3.0f) - 0.5f * w0 * uu) * (1.0f / (1.0f - w0));
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
    const int D = Lat<Q>::D;
    const SmemLayout SL = smem_layout(sh, D, sh.warps);
    auto kern = k_fluid<Q, S, V>;
    const int g = persistent ? grid : ntiles;
    kern<<<g, 32 * sh.warps, SL.bytes, st>>>(insts, tile_inst, ntiles, par, sh, commit, persistent,
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
    const int D = Q == 9 ? 2 : 3;
    const SmemLayout SL = smem_layout(sh, D, sh.warps);
    int nb = 0;
#define LBM_OCC(QQ, SS, VV)                                                                         \
    if (Q == QQ && sh.vec == VV) {                                                                  \
        cudaFuncSetAttribute(k_fluid<QQ, SS, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL.bytes); \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fluid<QQ, SS, VV>, 32 * sh.warps, SL.bytes); \
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
