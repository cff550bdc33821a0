// Device helpers shared by the fused fluid kernels (register path and TMA
// path) and the export kernels of lbmpen.
#pragma once

#include "lbm_internal.cuh"

namespace lbmpen {

// Block-wide copy of an instance descriptor into shared memory: one coalesced
// round trip instead of a dependent global load for every field the serial
// per-particle code touches.  Ends with __syncthreads().
__device__ __forceinline__ void stage_desc(InstDesc* dst, const InstDesc& src) {
    static_assert(sizeof(InstDesc) % 8 == 0, "descriptor copied in 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(&src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(InstDesc) / 8); i += blockDim.x) d[i] = __ldg(s + i);
    __syncthreads();
}

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

__device__ __forceinline__ float to_float_scaled(float v, float) { return v; }
// Two adjacent populations from shared memory (8-byte / 4-byte aligned pair).
__device__ __forceinline__ float2 smem_pair(const float* p, float) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float2 smem_pair(const __half* p, float s) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    return make_float2(v.x * s, v.y * s);
}
// Two adjacent populations to global memory (aligned pair).
__device__ __forceinline__ void store_pair(float* p, float2 v, float) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ void store_pair(__half* p, float2 v, float s) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.x * s, v.y * s);
}
__device__ __forceinline__ float to_float_scaled(__half v, float s) { return __half2float(v) * s; }

template <class S> __device__ __forceinline__ S to_store(float v, float s);
template <> __device__ __forceinline__ float to_store<float>(float v, float) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v, float s) {
    return __float2half_rn(v * s);
}

// -------------------------------------------------------- indicator test ---
// Candidate particle of a tile, staged in shared memory.  The particle kernel
// also writes these records into each tile's list (list_rec), 64 bytes each,
// so that the TMA kernel can fetch a tile's candidates with one bulk copy.
struct __align__(16) Cand {
    int ref[3];
    float frac[3];
    float R2lo, R2hi;
    float a[3];
    int p;     // particle index within the instance
    int k;     // index of this tile among the tiles of the particle's bounding box
    int boff;  // first entry of the particle's velocity box
    int bh;    // H of the box: side 2H + 1, centred on ref
    int shape; // 0 disk or sphere, 1 ellipse (the filter reads its record)
};
static_assert(sizeof(Cand) == CAND_BYTES, "candidate records are copied in 64-byte units");

// Per-tile geometry and collision constants, copied out of the instance
// descriptor into registers: the hot loops must not reload them after every
// population store (the compiler cannot prove the stores do not alias them).
struct Geo {
    int n[3];
    int per[3];
    const PRec* prec;
};
struct CollP {
    float keep, fpref, alpha;
};
__device__ __forceinline__ Geo make_geo(const InstDesc& in) {
    Geo g;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        g.n[d] = in.n[d];
        g.per[d] = in.periodic[d];
    }
    g.prec = in.prec;
    return g;
}
__device__ __forceinline__ CollP make_collp(const InstDesc& in) { return CollP{in.keep, in.fpref, in.alpha}; }

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
// An ellipse (Sec. 3.3, 2D): u = dx cos + dy sin, v = dy cos - dx sin, then
// b^2 (u u) + a^2 (v v) <= a^2 b^2.  Separate roundings (no fused
// multiply-add) via the _rn intrinsics.
template <int D>
__device__ __noinline__ bool inside_exact(const PRec* __restrict__ pr, int x, int y, int z, int nx,
                                          int ny, int nz, int pmask) {
    const int xyz[3] = {x, y, z}, n[3] = {nx, ny, nz};
    double r[3] = {0.0, 0.0, 0.0};
    double d2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        double dx = __dsub_rn((double)xyz[d], pr->X[d]);
        if ((pmask >> d) & 1) {
            double half = 0.5 * (double)n[d];
            if (dx > half) dx = __dsub_rn(dx, (double)n[d]);
            else if (dx < -half) dx = __dadd_rn(dx, (double)n[d]);
        }
        r[d] = dx;
        d2 = __dadd_rn(d2, __dmul_rn(dx, dx));
    }
    if (D == 2 && pr->shape) {
        const double u = __dadd_rn(__dmul_rn(r[0], pr->ec), __dmul_rn(r[1], pr->es));
        const double v = __dsub_rn(__dmul_rn(r[1], pr->ec), __dmul_rn(r[0], pr->es));
        const double lhs = __dadd_rn(__dmul_rn(pr->b2, __dmul_rn(u, u)), __dmul_rn(pr->R2, __dmul_rn(v, v)));
        return lhs <= __dmul_rn(pr->R2, pr->b2);
    }
    return d2 <= pr->R2;
}
template <int D>
__device__ __forceinline__ bool inside_exact(const Geo& g, const PRec& pr, const int* xyz) {
    return inside_exact<D>(&pr, xyz[0], xyz[1], xyz[2], g.n[0], g.n[1], g.n[2],
                           g.per[0] | (g.per[1] << 1) | (g.per[2] << 2));
}

// Float filter of the indicator of candidate cd at a node: the squared
// distance against the band [R2lo, R2hi] of the disk (sphere), or for an
// ellipse inside its circumscribed circle the normalised form
// (r.e / a)^2 + (r.e_perp / b)^2 against the band [qlo, qhi] (its constants
// from the particle's record).  Nodes in a band take the exact FP64 test.
template <int D>
__device__ __forceinline__ bool inside_filtered(const Geo& in, const Cand& cd, const int* xyz) {
    float r[3] = {0.f, 0.f, 0.f};
    float d2 = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        int di = wrap_int(xyz[d] - cd.ref[d], in.n[d], in.per[d]);
        r[d] = (float)di - cd.frac[d];
        d2 = fmaf(r[d], r[d], d2);
    }
    if (d2 > cd.R2hi) return false;
    if (D == 2 && cd.shape) {
        const PRec& pr = in.prec[cd.p];
        const float u = fmaf(r[0], pr.fc, r[1] * pr.fs);
        const float v = fmaf(r[1], pr.fc, -(r[0] * pr.fs));
        const float q = fmaf(u * u, pr.ia2, (v * v) * pr.ib2);
        if (q < pr.qlo) return true;
        if (q > pr.qhi) return false;
        return inside_exact<D>(in, pr, xyz);
    }
    if (d2 < cd.R2lo) return true;
    return inside_exact<D>(in, in.prec[cd.p], xyz);
}

// Owner of a node among the tile's candidates: lowest particle index whose
// solid domain holds the node, or -1 (float filter, exact test in its band).
template <int D>
__device__ __forceinline__ int owner_of(const Geo& in, const Cand* cand, int ncand,
                                        const int* xyz, int* slot) {
    int best = -1, bslot = -1;
    for (int c = 0; c < ncand; ++c) {
        const Cand& cd = cand[c];
        if (best >= 0 && cd.p > best) continue;
        const bool inside = inside_filtered<D>(in, cd, xyz);
        if (inside && (best < 0 || cd.p < best)) {
            best = cd.p;
            bslot = c;
        }
    }
    *slot = bslot;
    return best;
}

// Candidates whose solid domain can reach the row segment of width nodes
// starting at x0 of row (y, z): a uniform test per candidate instead of a test per
// node.  Bit c set = candidate c may own a node of the segment (ncand <= 32).
// Lane c of the (converged) warp tests candidate c; a ballot gathers the bits.
template <int D>
__device__ __forceinline__ unsigned segment_candidates(const Geo& g, const Cand* cand, int ncand, int x0,
                                                       int y, int z, int width, int lane) {
    bool live = false;
    if (lane < ncand) {
        const Cand& cd = cand[lane];
        const float dy = (float)wrap_int(y - cd.ref[1], g.n[1], g.per[1]) - cd.frac[1];
        float rest = cd.R2hi - dy * dy;
        if (D == 3) {
            const float dz = (float)wrap_int(z - cd.ref[2], g.n[2], g.per[2]) - cd.frac[2];
            rest -= dz * dz;
        }
        if (rest >= 0.f) {
            const float hw = sqrtf(rest) + 1.0f;
            // nearest distance along x from the centre to the segment [x0, x0 + width - 1]
            const float dx0 = (float)wrap_int(x0 - cd.ref[0], g.n[0], g.per[0]) - cd.frac[0];
            live = g.per[0] || !(dx0 > hw || dx0 + (float)(width - 1) < -hw);
        }
    }
    return __ballot_sync(0xffffffffu, live);
}

// Owner among the segment's live candidates (bit mask from segment_candidates).
template <int D>
__device__ __forceinline__ int owner_masked(const Geo& in, const Cand* cand, unsigned act,
                                            const int* xyz, int* slot) {
    int best = -1, bslot = -1;
    while (act) {
        const int c = __ffs(act) - 1;
        act &= act - 1;
        const Cand& cd = cand[c];
        if (best >= 0 && cd.p > best) continue;
        const bool inside = inside_filtered<D>(in, cd, xyz);
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
// source of Eq. 17, with A_q = w_q / cs^2:
//   feq_q = A_q (p - u.u/2 + c.u + 1.5 (c.u)^2)                      (Eq. 13)
//   F_q   = (1 - 1/2tau) A_q ((c.a)(1 + 3 c.u) - u.a)                 (Eq. 14)
//   S_q   = 1.5 alpha A_q (Pi_neq : c c - tr(Pi_neq) / 3)             (Eq. 17)
//   f*_q  = (1 - 1/tau) f_q + feq_q / tau + F_q + chi S_q             (Eq. 10)
// and p recovered from the stored populations (Eq. 15b) as
//   p = (sum_{q>=1} f_q - (1.5 - 0.5 sum A) u.u) / sum A,
// the inverse of feq for these coefficients.  Opposite velocities share c.u,
// c.a and p - u.u/2 + 1.5 (c.u)^2, so the work goes pair by pair.
//
// Two nodes at a time: every operation is one packed FP32x2 instruction
// (FFMA2 / FMUL2 / FADD2, each half rounded like its scalar counterpart), so
// a lane collides two nodes for the instruction count of one.  Every product,
// sum and fused multiply-add is written out, so the rounding does not depend
// on the compiler's contraction choices, and the one-node entry point below
// (both halves the same node) gives the same bits as the two-node one.
struct CollK {
    float keep;       // 1 - 1/tau
    float omk;        // 1/tau
    float A[2];       // A for the two weight classes (axis, diagonal/edge)
    float fA[2];      // (1 - 1/2tau) A
    float alpha;
    float sA[2];      // 1.5 alpha A (penalty)
};
template <int Q>
__device__ __forceinline__ CollK make_collk(const CollP& in) {
    using L = Lat<Q>;
    CollK k;
    k.keep = in.keep;
    k.omk = 1.0f - in.keep;
    const float A[2] = {L::A(1), L::A(Q == 9 ? 5 : 7)};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        // A stays exact (sum A c_x^2 = 1): 1/tau multiplies separately, so no
        // rounded product of the two can bias the momentum of feq
        k.A[i] = A[i];
        k.fA[i] = in.fpref * A[i];
        k.sA[i] = (1.5f * in.alpha) * A[i];
    }
    k.alpha = in.alpha;
    return k;
}

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b: b * (-1) is exact, so the fused form rounds once, like FADD
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// c_q . v for a compile-time velocity q, without adding zeros
template <int Q, int q>
__device__ __forceinline__ float2 cdot2(const float2* v) {
    using L = Lat<Q>;
    constexpr int c0 = L::c(q, 0), c1 = L::c(q, 1), c2 = L::c(q, 2);
    float2 r;
    if constexpr (c0 != 0) {
        r = c0 > 0 ? v[0] : mul2(v[0], bc2(-1.0f));
        if constexpr (c1 != 0) r = c1 > 0 ? add2(r, v[1]) : sub2(r, v[1]);
        if constexpr (c2 != 0) r = c2 > 0 ? add2(r, v[2]) : sub2(r, v[2]);
    } else if constexpr (c1 != 0) {
        r = c1 > 0 ? v[1] : mul2(v[1], bc2(-1.0f));
        if constexpr (c2 != 0) r = c2 > 0 ? add2(r, v[2]) : sub2(r, v[2]);
    } else {
        r = c2 > 0 ? v[2] : mul2(v[2], bc2(-1.0f));
    }
    return r;
}

// first velocity of each opposite pair: q odd in both numberings except D2Q9,
// where pairs are (1,3), (2,4), (5,7), (6,8)
template <int Q> __host__ __device__ constexpr bool pair_head(int q) {
    return Q == 9 ? (q == 1 || q == 2 || q == 5 || q == 6) : (q & 1) == 1;
}

template <int Q, int q>
__device__ __forceinline__ void collide_pair2(float2* f, const float2* u, const float2* a, float2 base,
                                              float2 nua, const CollK& k) {
    if constexpr (q < Q) {
        if constexpr (pair_head<Q>(q)) {
            using L = Lat<Q>;
            constexpr int qo = L::opp(q);
            constexpr int cls = (Q == 9 ? q >= 5 : q >= 7) ? 1 : 0;
            const float2 cu = cdot2<Q, q>(u), ca = cdot2<Q, q>(a);
            const float2 t = fma2(mul2(bc2(1.5f), cu), cu, base);
            const float2 eq = add2(t, cu), eo = sub2(t, cu);                    // feq / A
            const float2 Fq = fma2(ca, fma2(bc2(3.0f), cu, bc2(1.0f)), nua);    // F / fA
            const float2 Fo = fma2(ca, fma2(bc2(3.0f), cu, bc2(-1.0f)), nua);   // (-c.a)(1 - 3 c.u) - u.a
            f[q - 1] = fma2(bc2(k.keep), f[q - 1], fma2(bc2(k.omk), mul2(bc2(k.A[cls]), eq), mul2(bc2(k.fA[cls]), Fq)));
            f[qo - 1] = fma2(bc2(k.keep), f[qo - 1], fma2(bc2(k.omk), mul2(bc2(k.A[cls]), eo), mul2(bc2(k.fA[cls]), Fo)));
        }
        collide_pair2<Q, q + 1>(f, u, a, base, nua, k);
    }
}

// tau = 1 (keep = 0, 1/tau = 1): f*_q = feq_q + F_q + chi S_q formed as one
// chain of fused multiply-adds, feq_q = A_q t + A_q (c.u) and the opposite
// feq = A_q t - A_q (c.u), so that the only rounding at the scale of f* is the
// last one (four before).  In the solid, where alpha = 1/tau keeps the
// non-equilibrium stress from step to step, the rounding of every step
// accumulates, so fewer roundings per step is a smaller error.  No constant
// is folded (A_q stays exact), so no momentum bias enters.  P and trP: the
// penalty's Pi_neq and its trace / 3 (PEN only).
template <int Q, int q>
__device__ __forceinline__ float2 pcc2(const float2* P) {  // c_q^T Pi c_q
    using L = Lat<Q>;
    constexpr int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
    float2 r = bc2(0.f);
    bool first = true;
    const int dia[3] = {cx, cy, cz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (!dia[d]) continue;
        r = first ? P[d] : add2(r, P[d]);
        first = false;
    }
    if (cx * cy) r = fma2(bc2(cx * cy > 0 ? 2.0f : -2.0f), P[3], r);
    if (cx * cz) r = fma2(bc2(cx * cz > 0 ? 2.0f : -2.0f), P[4], r);
    if (cy * cz) r = fma2(bc2(cy * cz > 0 ? 2.0f : -2.0f), P[5], r);
    return r;
}

template <int Q, int q, bool PEN>
__device__ __forceinline__ void collide_pair2_t1(float2* f, const float2* u, const float2* a, float2 base,
                                                 float2 nua, const CollK& k, const float2* P, float2 trP,
                                                 bool solid0, bool solid1) {
    if constexpr (q < Q) {
        if constexpr (pair_head<Q>(q)) {
            using L = Lat<Q>;
            constexpr int qo = L::opp(q);
            constexpr int cls = (Q == 9 ? q >= 5 : q >= 7) ? 1 : 0;
            const float2 cu = cdot2<Q, q>(u), ca = cdot2<Q, q>(a);
            const float2 t = fma2(mul2(bc2(1.5f), cu), cu, base);
            const float2 Fq = fma2(ca, fma2(bc2(3.0f), cu, bc2(1.0f)), nua);
            const float2 Fo = fma2(ca, fma2(bc2(3.0f), cu, bc2(-1.0f)), nua);
            float2 gq = mul2(bc2(k.fA[cls]), Fq), go = mul2(bc2(k.fA[cls]), Fo);
            if constexpr (PEN) {  // opposite velocities share c c, so one penalty for both
                const float2 pq = sub2(pcc2<Q, q>(P), trP);
                const float2 sq = fma2(bc2(k.sA[cls]), pq, gq), so = fma2(bc2(k.sA[cls]), pq, go);
                gq = make_float2(solid0 ? sq.x : gq.x, solid1 ? sq.y : gq.y);
                go = make_float2(solid0 ? so.x : go.x, solid1 ? so.y : go.y);
            }
            f[q - 1] = fma2(bc2(k.A[cls]), cu, fma2(bc2(k.A[cls]), t, gq));
            f[qo - 1] = fma2(bc2(-k.A[cls]), cu, fma2(bc2(k.A[cls]), t, go));
        }
        collide_pair2_t1<Q, q + 1, PEN>(f, u, a, base, nua, k, P, trP, solid0, solid1);
    }
}

// Penalty source on solid nodes (Eq. 17) in two parts: the non-equilibrium
// momentum flux Pi_neq = sum_q (f_q - feq_q) c_q c_q of the pre-collision
// populations (xx yy zz xy xz yz), taken before the collision overwrites f,
// and S_q = 1.5 alpha A_q (c_q^T Pi c_q - tr(Pi)/3) added after it.
template <int Q>
__device__ __forceinline__ void pi_neq2(const float2* f, const float2* u, float2 base, float2* P) {
    using L = Lat<Q>;
    bool set[6] = {false, false, false, false, false, false};
#pragma unroll
    for (int i = 0; i < 6; ++i) P[i] = bc2(0.f);
    auto acc = [&](int i, float2 v, bool neg) {
        if (!set[i]) P[i] = neg ? mul2(v, bc2(-1.0f)) : v;
        else P[i] = neg ? sub2(P[i], v) : add2(P[i], v);
        set[i] = true;
    };
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        float2 cu = bc2(0.f);
        bool first = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int c = L::c(q, d);
            if (c == 0) continue;
            if (first) cu = c > 0 ? u[d] : mul2(u[d], bc2(-1.0f));
            else cu = c > 0 ? add2(cu, u[d]) : sub2(cu, u[d]);
            first = false;
        }
        const float2 fn = fma2(bc2(-L::A(q)), fma2(mul2(bc2(1.5f), cu), cu, add2(base, cu)), f[q - 1]);
        const int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
        if (cx) acc(0, fn, false);
        if (cy) acc(1, fn, false);
        if (cz) acc(2, fn, false);
        if (cx * cy) acc(3, fn, cx * cy < 0);
        if (cx * cz) acc(4, fn, cx * cz < 0);
        if (cy * cz) acc(5, fn, cy * cz < 0);
    }
}

template <int Q>
__device__ __forceinline__ void add_penalty2(float2* f, const float2* P, bool solid0, bool solid1, const CollK& k) {
    using L = Lat<Q>;
    const float2 trP = mul2(add2(add2(P[0], P[1]), P[2]), bc2(1.0f / 3.0f));
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int cx = L::c(q, 0), cy = L::c(q, 1), cz = L::c(q, 2);
        float2 pcc = bc2(0.f);
        bool first = true;
        const int dia[3] = {cx, cy, cz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!dia[d]) continue;
            pcc = first ? P[d] : add2(pcc, P[d]);
            first = false;
        }
        if (cx * cy) pcc = fma2(bc2(cx * cy > 0 ? 2.0f : -2.0f), P[3], pcc);
        if (cx * cz) pcc = fma2(bc2(cx * cz > 0 ? 2.0f : -2.0f), P[4], pcc);
        if (cy * cz) pcc = fma2(bc2(cy * cz > 0 ? 2.0f : -2.0f), P[5], pcc);
        const int cls = (Q == 9 ? q >= 5 : q >= 7) ? 1 : 0;
        const float2 fp = fma2(bc2(k.sA[cls]), sub2(pcc, trP), f[q - 1]);
        f[q - 1] = make_float2(solid0 ? fp.x : f[q - 1].x, solid1 ? fp.y : f[q - 1].y);
    }
}

// Moments of the stored populations of two nodes, without adding zeros.
template <int Q>
__device__ __forceinline__ void moments2(const float2* f, float2& s, float2* m) {
    if constexpr (Q == 9) {
        const float2 d13 = sub2(f[0], f[2]), d24 = sub2(f[1], f[3]), d57 = sub2(f[4], f[6]),
                     d68 = sub2(f[5], f[7]);
        s = add2(add2(add2(f[0], f[2]), add2(f[1], f[3])), add2(add2(f[4], f[6]), add2(f[5], f[7])));
        m[0] = add2(d13, sub2(d57, d68));
        m[1] = add2(d24, add2(d57, d68));
        m[2] = bc2(0.f);
    } else {
        // D3Q19 pairs (1,2) x, (3,4) y, (5,6) z, (7,8) xy, (9,10) x-y, (11,12) xz,
        // (13,14) x-z, (15,16) yz, (17,18) y-z; d_k = f_head - f_tail
        const float2 dx = sub2(f[0], f[1]), dy = sub2(f[2], f[3]), dz = sub2(f[4], f[5]);
        const float2 dxy = sub2(f[6], f[7]), dxmy = sub2(f[8], f[9]), dxz = sub2(f[10], f[11]);
        const float2 dxmz = sub2(f[12], f[13]), dyz = sub2(f[14], f[15]), dymz = sub2(f[16], f[17]);
        float2 a0 = f[0], a1 = f[1];
#pragma unroll
        for (int i = 2; i < 18; i += 2) {
            a0 = add2(a0, f[i]);
            a1 = add2(a1, f[i + 1]);
        }
        s = add2(a0, a1);
        m[0] = add2(dx, add2(add2(dxy, dxmy), add2(dxz, dxmz)));
        m[1] = add2(dy, add2(sub2(dxy, dxmy), add2(dyz, dymz)));
        m[2] = add2(dz, add2(sub2(dxz, dxmz), sub2(dyz, dymz)));
    }
}

// Scalar moments (the adjoint's forward recomputation): the same sums.
template <int Q>
__device__ __forceinline__ void moments(const float* f, float& s, float* m) {
    float2 f2v[Q - 1];
#pragma unroll
    for (int q = 0; q < Q - 1; ++q) f2v[q] = bc2(f[q]);
    float2 s2, m2[3];
    moments2<Q>(f2v, s2, m2);
    s = s2.x;
    m[0] = m2[0].x;
    m[1] = m2[1].x;
    m[2] = m2[2].x;
}

// Two nodes: f holds the stored populations q = 1..Q-1 (index q-1) after
// streaming; on return it holds f*.  u and p of Eq. 15 are returned.  solid
// flags the halves on which the penalty acts.
template <int Q>
__device__ __forceinline__ void collide2(float2* f, const float2* a, bool solid0, bool solid1, const CollK& k,
                                         float2* u_out, float2* p_out) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr float inv_sa = (float)(1.0 / L::SUMA);
    constexpr float kuu = (float)(1.5 - 0.5 * L::SUMA);
    float2 s, m[3];
    moments2<Q>(f, s, m);
    float2 u[3];
    u[0] = fma2(bc2(0.5f), a[0], m[0]);  // Eq. 15a
    u[1] = fma2(bc2(0.5f), a[1], m[1]);
    u[2] = D == 3 ? fma2(bc2(0.5f), a[2], m[2]) : bc2(0.f);
    const float2 uu = D == 3 ? fma2(u[2], u[2], fma2(u[1], u[1], mul2(u[0], u[0])))
                             : fma2(u[1], u[1], mul2(u[0], u[0]));
    const float2 p = mul2(fma2(bc2(-kuu), uu, s), bc2(inv_sa));  // Eq. 15b
    const float2 ua = D == 3 ? fma2(u[2], a[2], fma2(u[1], a[1], mul2(u[0], a[0])))
                             : fma2(u[1], a[1], mul2(u[0], a[0]));
    const float2 nua = mul2(ua, bc2(-1.0f));
    const float2 base = fma2(bc2(-0.5f), uu, p);
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[d] = u[d];
    *p_out = p;
    if (k.keep == 0.f) {  // tau = 1: one rounding at the scale of f* (see collide_pair2_t1)
        if (solid0 || solid1) {
            float2 P[6];
            pi_neq2<Q>(f, u, base, P);
            const float2 trP = mul2(add2(add2(P[0], P[1]), P[2]), bc2(1.0f / 3.0f));
            collide_pair2_t1<Q, 1, true>(f, u, a, base, nua, k, P, trP, solid0, solid1);
        } else {
            collide_pair2_t1<Q, 1, false>(f, u, a, base, nua, k, nullptr, bc2(0.f), false, false);
        }
    } else if (solid0 || solid1) {
        float2 P[6];
        pi_neq2<Q>(f, u, base, P);
        collide_pair2<Q, 1>(f, u, a, base, nua, k);
        add_penalty2<Q>(f, P, solid0, solid1, k);
    } else {
        collide_pair2<Q, 1>(f, u, a, base, nua, k);
    }
}

// FP16 storage at tau = 1: f holds the populations at the storage scale
// (2^14 f, as read, without the 2^-14 multiply), and ks is CollK with A, fA
// and sA multiplied by 2^14, so f* comes out at the storage scale too.  The
// moments are linear sums, scaled to lattice units once (sload = 2^-14), and
// a power-of-two scaling commutes with every rounding in the normal range,
// so the stored halves are the same bits as those of collide2 followed by
// the 2^14 multiply; this saves two multiplies per population and node.
template <int Q>
__device__ __forceinline__ void collide2_t1_scaled(float2* f, const float2* a, bool solid0, bool solid1,
                                                   const CollK& ks, float sload, float2* u_out, float2* p_out) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr float inv_sa = (float)(1.0 / L::SUMA);
    constexpr float kuu = (float)(1.5 - 0.5 * L::SUMA);
    float2 s, m[3];
    moments2<Q>(f, s, m);
    s = mul2(s, bc2(sload));
    m[0] = mul2(m[0], bc2(sload));
    m[1] = mul2(m[1], bc2(sload));
    if (D == 3) m[2] = mul2(m[2], bc2(sload));
    float2 u[3];
    u[0] = fma2(bc2(0.5f), a[0], m[0]);  // Eq. 15a
    u[1] = fma2(bc2(0.5f), a[1], m[1]);
    u[2] = D == 3 ? fma2(bc2(0.5f), a[2], m[2]) : bc2(0.f);
    const float2 uu = D == 3 ? fma2(u[2], u[2], fma2(u[1], u[1], mul2(u[0], u[0])))
                             : fma2(u[1], u[1], mul2(u[0], u[0]));
    const float2 p = mul2(fma2(bc2(-kuu), uu, s), bc2(inv_sa));  // Eq. 15b
    const float2 ua = D == 3 ? fma2(u[2], a[2], fma2(u[1], a[1], mul2(u[0], a[0])))
                             : fma2(u[1], a[1], mul2(u[0], a[0]));
    const float2 nua = mul2(ua, bc2(-1.0f));
    const float2 base = fma2(bc2(-0.5f), uu, p);
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[d] = u[d];
    *p_out = p;
    if (solid0 || solid1) {  // Pi_neq of the populations in lattice units
#pragma unroll
        for (int q = 0; q < Q - 1; ++q) f[q] = mul2(f[q], bc2(sload));
        float2 P[6];
        pi_neq2<Q>(f, u, base, P);
        const float2 trP = mul2(add2(add2(P[0], P[1]), P[2]), bc2(1.0f / 3.0f));
        collide_pair2_t1<Q, 1, true>(f, u, a, base, nua, ks, P, trP, solid0, solid1);
    } else {
        collide_pair2_t1<Q, 1, false>(f, u, a, base, nua, ks, nullptr, bc2(0.f), false, false);
    }
}

// One node (both halves of the packed arithmetic carry it): the same bits
// as collide2 gives that node.
template <int Q>
__device__ __forceinline__ void collide(float* f, const float* a, bool solid, const CollK& k, float* u_out,
                                        float* p_out) {
    float2 f2v[Q - 1], a2[3], u2[3], p2;
#pragma unroll
    for (int q = 0; q < Q - 1; ++q) f2v[q] = bc2(f[q]);
#pragma unroll
    for (int d = 0; d < 3; ++d) a2[d] = bc2(a[d]);
    collide2<Q>(f2v, a2, solid, solid, k, u2, &p2);
#pragma unroll
    for (int q = 0; q < Q - 1; ++q) f[q] = f2v[q].x;
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[d] = u2[d].x;
    *p_out = p2.x;
}

// Fixed-point image round(u * 2^FXBITS) of a velocity component, rounded to
// the nearest integer (ties to even): the scaling by a power of two is exact,
// so the conversion is the only rounding.  The value is clamped to |u| < 1/2;
// a larger or non-finite velocity is reported as divergence by the caller.
__device__ __forceinline__ long long to_fx(float u) {
    u = fminf(fmaxf(u, -0.49999997f), 0.49999997f);
    return __float2ll_rn(u * 1099511627776.0f);  // u * 2^40 is exact; round to nearest even
}

// The same round(u * 2^FXBITS) by two 32-bit conversions (the 64-bit one
// issues at the FP64 rate on this GPU): x = u 2^40 is exact, t = trunc(x 2^-20)
// fits in 20 bits, x - t 2^20 is exact (a multiple of ulp(x) below 2^20 in
// magnitude, so at most 24 significant bits), and since t 2^20 is an even
// integer, rne(x) = t 2^20 + rne(x - t 2^20), ties included.
__device__ __forceinline__ long long to_fx32(float u) {
    u = fminf(fmaxf(u, -0.49999997f), 0.49999997f);
    const float x = u * 1099511627776.0f;                  // 2^40, exact
    const int t = __float2int_rz(x * 9.5367431640625e-7f);  // 2^-20, exact scaling
    const float rem = fmaf(-(float)t, 1048576.0f, x);      // exact
    return (long long)t * 1048576LL + (long long)__float2int_rn(rem);
}

// Exact warp sum of 64-bit integers: three 21-bit limbs (the top one signed),
// each summed by one integer reduction (32 lanes keep every limb sum below
// 2^26 in magnitude), recombined modulo 2^64, which is exact whenever the
// total fits in int64.
__device__ __forceinline__ long long warp_sum_fx(long long v) {
    const unsigned l0 = (unsigned)(v & 0x1FFFFF);
    const unsigned l1 = (unsigned)((v >> 21) & 0x1FFFFF);
    const int l2 = (int)(v >> 42);  // arithmetic shift: the signed top limb
    const long long s0 = (long long)__reduce_add_sync(0xffffffffu, l0);
    const long long s1 = (long long)__reduce_add_sync(0xffffffffu, l1);
    const long long s2 = (long long)__reduce_add_sync(0xffffffffu, l2);
    return s0 + s1 * (1LL << 21) + s2 * (1LL << 42);
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Velocity of a node owned by candidate cd into the particle's box: entry
// (d + H) of the offset d = node - floor(X) (minimum image on periodic axes,
// |d| <= R + 1 < H).  The particle kernel takes the sums of Eq. 22 from there.
template <int D>
__device__ __forceinline__ void box_store(float* ubox, const Geo& g, const Cand& cd, int x, int y, int z,
                                          float ux, float uy, float uz) {
    const int side = 2 * cd.bh + 1;
    const int dx = wrap_int(x - cd.ref[0], g.n[0], g.per[0]) + cd.bh;
    const int dy = wrap_int(y - cd.ref[1], g.n[1], g.per[1]) + cd.bh;
    if (D == 2) {
        reinterpret_cast<float2*>(ubox)[cd.boff + dy * side + dx] = make_float2(ux, uy);
    } else {
        const int dz = wrap_int(z - cd.ref[2], g.n[2], g.per[2]) + cd.bh;
        reinterpret_cast<float4*>(ubox)[cd.boff + ((long long)dz * side + dy) * side + dx] =
            make_float4(ux, uy, uz, 0.f);
    }
}

// ----------------------------------------------- per-particle finalisation --
constexpr double FX_SCALE = 1.0 / (double)(1LL << FXBITS);

// 1/x in FP64 for x in the normal FP32 range: an FP32 reciprocal refined by
// two Newton steps (within an ulp of the rounded quotient).  A dependent FP64
// division costs ~10x a fused multiply-add on this GPU.
__device__ __forceinline__ double rcp64(double x) {
    double r = (double)__frcp_rn((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    return fma(r, fma(-x, r, 1.0), r);
}

// Rigid-body projection of particle p (Eq. 22 with rho_s cancelled): the
// box sums are exact integers, summed exactly, then converted to FP64.
// Moments about the integer reference floor(X) are shifted to the centre:
//   sum r x u = sum d x u - phi x sum u,
//   sum r r^T = sum d d^T - phi sum d^T - sum d phi^T + n phi phi^T.
//
// An FP64 instruction takes the FP64 pipe of its SM sub-partition for ~64
// cycles whatever the number of active lanes, so the work is spread over
// lanes by component: the translation (U^n, Ubar, predicted position) runs
// one lane per component d, and the rotation (W^n) one lane per component on
// another warp, concurrently.  Each lane evaluates the same expressions, in
// the same order, as a serial loop over the components would.

// Translational part, component d (0..2) of particle p.
template <int D>
__device__ void finalize_translation(const InstDesc& in, int p, const long long* v, int d) {
    const PRec& pr = in.prec[p];
    // every operand is loaded before the first store, so the loads overlap
    const double X = d < D ? pr.X[d] : 0.0;
    const double Uold = d < D ? in.U[3 * p + d] : 0.0;
    const float Rf = (float)in.pconst[PCONST_N * p + PC_R];
    const double h = in.hK;
    if (v[0] == 0) {  // no solid node: cannot happen inside the box for R >= 2
        if (d == 0) {
            atomicOr(in.status, ST_PARTICLE);
            in.count[p] = 0;
        }
        in.Un[3 * p + d] = in.U[3 * p + d];
        return;
    }
    const double cnt = (double)v[0];
    const double inv = rcp64(cnt);
    double Uo = 0.0, ub = 0.0;
    float Xs = 0.f;
    bool fast = false;
    if (d < D) {
        const double Su = (double)v[10 + d] * FX_SCALE;
        Uo = Su * inv;
        ub = 0.5 * (Uo + Uold);
        fast = !(fabs(ub) < 0.5);
        Xs = (float)(X + h * ub);
    }
    in.Un[3 * p + d] = Uo;
    in.Ubar[3 * p + d] = ub;
    in.Xk[3 * p + d] = X;  // sub-step buffer 0 = X^n
    in.Xf[4 * p + d] = (float)X;
    in.Xsf[4 * p + d] = Xs;
    if (d == 0) {
        in.Xf[4 * p + 3] = Rf;
        in.Xsf[4 * p + 3] = Rf;
        in.count[p] = (int)v[0];
        in.invc[p] = inv;
    }
    if (fast) atomicOr(in.status, ST_DISPLACEMENT);
}

// Rotational part, component c (0..2) of W^n of particle p, and the sums the
// adjoint records (component 0's lane).
template <int D>
__device__ void finalize_rotation(const InstDesc& in, int p, const long long* v, int c) {
    const PRec& pr = in.prec[p];
    double phi[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) phi[d] = pr.X[d] - (double)pr.ref[d];
    if (v[0] == 0) {
        in.Wn[3 * p + c] = 0.0;
        return;
    }
    const double cnt = (double)v[0];
    double Su[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) Su[d] = (double)v[10 + d] * FX_SCALE;
    double Wo = 0.0;
    if (D == 2) {
        if (c == 2) {
            // w_z = sum (r x u)_z / sum |r|^2
            const double Lz = (double)v[15] * FX_SCALE - (phi[0] * Su[1] - phi[1] * Su[0]);
            const double Izz = (double)(v[4] + v[5]) - 2.0 * (phi[0] * (double)v[1] + phi[1] * (double)v[2]) +
                               cnt * (phi[0] * phi[0] + phi[1] * phi[1]);
            Wo = Lz * rcp64(Izz);
        }
    } else {
        const double Sd[3] = {(double)v[1], (double)v[2], (double)v[3]};
        double Sl[3];
        for (int d = 0; d < 3; ++d) Sl[d] = (double)v[13 + d] * FX_SCALE;
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
        const double tr = rr[0][0] + rr[1][1] + rr[2][2];
        double I[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) I[i][j] = (i == j ? tr : 0.0) - rr[i][j];
        const double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                           I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                           I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
        const double idet = rcp64(det);
        // Cramer's rule: column c of I replaced by L
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) M[r][q] = (q == c) ? Lv[r] : I[r][q];
        const double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                          M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        Wo = dc * idet;
    }
    in.Wn[3 * p + c] = Wo;
    if (in.adj_geo && c == 0) {  // adjoint recording: the sums about X^n that the projection used
        double* g = in.adj_geo + (long long)NPV * p;
        const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
        g[0] = cnt;
        for (int d = 0; d < 3; ++d) g[1 + d] = (double)v[1 + d] - cnt * phi[d];
        for (int k = 0; k < 6; ++k) {
            const int i = ii[k], j = jj[k];
            g[4 + k] = (double)v[4 + k] - phi[i] * (double)v[1 + j] - phi[j] * (double)v[1 + i] +
                       cnt * phi[i] * phi[j];
        }
        for (int d = 0; d < 3; ++d) g[10 + d] = Su[d];
        g[13] = (double)v[13] * FX_SCALE - (phi[1] * Su[2] - phi[2] * Su[1]);
        g[14] = (double)v[14] * FX_SCALE - (phi[2] * Su[0] - phi[0] * Su[2]);
        g[15] = (double)v[15] * FX_SCALE - (phi[0] * Su[1] - phi[1] * Su[0]);
    }
}

// Where population q of node (x, y, z) pulls from (Eq. 10, left side): the
// element of the previous post-collision buffer, and the term added to it.
// Across a periodic face the source wraps; across a wall (the first wall axis
// in the order x, y, z) the node's own opposite population bounces back, plus
// the moving-wall term 2 w_q (c_q . u_w) / cs^2.
template <int Q, class S>
__device__ __forceinline__ const S* pull_source(const InstDesc& in, const S* fin, int q, int x, int y, int z,
                                                float* add) {
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
        *add = in.wterm[axis][face][q];
        const long long off = ((long long)z * in.n[1] + y) * in.pitch + x;
        return fin + (long long)(L::opp(q) - 1) * in.qstride + off;
    }
    *add = 0.f;
    const long long off = ((long long)src[2] * in.n[1] + src[1]) * in.pitch + src[0];
    return fin + (long long)(q - 1) * in.qstride + off;
}

template <int Q, class S>
__device__ __noinline__ float pull_scalar(const InstDesc& in, const S* fin, int q, int x, int y, int z) {
    float add;
    const S* p = pull_source<Q, S>(in, fin, q, x, y, z, &add);
    return VecIO<S, 1 + (sizeof(S) == 2)>::load1(p, in.s_load) + add;
}

}  // namespace lbmpen
