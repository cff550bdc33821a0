// TMA-pipelined variant of the fused stream-collide-penalize kernel.
//
// Persistent blocks of one producer warp and NC consumer warps.  The producer
// takes tiles from a work counter (claimed one tile ahead; successive claims
// alternate between the two ends of the tile range) and issues one
// cp.async.bulk.tensor box per stored population: the source rows
// (y - c_y, z - c_z) of the tile, 32*k nodes wide plus a 16-byte halo on both
// sides so that every box starts on a 16-byte boundary; while the copies are
// in flight it stages the tile's header and candidate particles.  The boxes
// of a tile land in one stage of a ring of shared-memory buffers, counted by
// an mbarrier; each consumer lane pulls two adjacent nodes' populations from
// shared memory at x - c_x, collides them with packed FP32x2 arithmetic,
// stores them to HBM with 8-byte coalesced stores, and reduces the
// per-particle sums of Eq. 22.  Bytes in flight live in shared memory instead
// of registers, which keeps HBM busy with few threads.  The populations the
// x-edge node of a tile (x = 0 or nx - 1) pulls across its face (bounce-back
// or periodic wrap) are gathered from HBM by the producer's lanes while the
// copies are in flight, into a small per-stage array, so that the edge rows
// stay on the shared-memory path; rows whose source lies beyond a y or z face
// gather those populations from HBM directly, as the register-path kernel
// does.
//
// Every mbarrier wait is bounded in time; on expiry the kernel records a
// timeout in the status word, waits (bounded) for the copies it issued and
// returns.
#include <cuda.h>

#include "lbm_common.cuh"

namespace lbmpen {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Raise the bytes the current phase waits for, without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity; false once limit_ns has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (now_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// Per-tile record the producer writes next to the staged populations, so
// that consumer warps take the tile's constants from shared memory.
struct StageHdr {
    int tile;   // global tile index, -1 = no more work
    int ncand;
    int inst;
    int x0, y0, z0;
    int n[3];
    int per[3];
    int pitch, maxk;
    long long qstride;
    float gdrive[3];
    float sload, sstore;
    CollK ck;
    const void* fin;
    void* fout;
    long long* partial;
    const PRec* prec;
    int* status;
    int ex;   // x of the tile's edge node whose face values are staged, -1 none,
              //   -2 both edges in one tile (those take the direct gathers)
    int ecx;  // c_x of the staged populations: +1 at x = 0, -1 at x = nx - 1
};

}  // namespace

// Geometry of the shared-memory ring, identical on host and device.
struct TmaLayout {
    int bw;          // box width (nodes) = tile width + 2 halo
    int slab;        // bytes of one population box, rounded to 128
    int stage;       // bytes of all populations of one stage
    int pops_bytes;  // stages * stage
    int hdr_off, cand_off, edge_off, bar_off, bytes;
};

// Populations with c_x = +1 (equally, -1): the ones an x-edge node pulls
// across its face.
__host__ __device__ constexpr int edge_pops(int Q) { return Q == 9 ? 3 : 5; }

__host__ __device__ inline TmaLayout tma_layout(int Q, int ssize, int tw, int rows, int stages) {
    TmaLayout L;
    const int halo = 16 / ssize;
    L.bw = tw + 2 * halo;
    L.slab = ((L.bw * rows * ssize) + 127) & ~127;
    L.stage = (Q - 1) * L.slab;
    L.pops_bytes = stages * L.stage;
    L.hdr_off = L.pops_bytes;
    L.cand_off = L.hdr_off + (int)sizeof(StageHdr) * stages;
    L.edge_off = L.cand_off + (int)sizeof(Cand) * LIST_CAP * stages;
    L.bar_off = (L.edge_off + (int)sizeof(float) * rows * edge_pops(Q) * stages + 15) & ~15;
    L.bytes = L.bar_off + 16 * stages + 128;  // + alignment slack of the base
    return L;
}

// Register budget: two blocks of 9 warps per SM (the shared-memory ring of
// three stages allows no more); each lane collides two nodes at a time.
template <int Q, class S, int TW, int ROWS>
__global__ void __launch_bounds__(288, 2) k_fluid_tma(const InstDesc* __restrict__ insts,
                                                   const CUtensorMap* __restrict__ tmaps,
                                                   const uint16_t* __restrict__ tile_inst, int ntiles,
                                                   int par, Shape sh, int commit, int* tile_ctr,
                                                   int stages, int ninst) {
    using L = Lat<Q>;
    constexpr int D = L::D;
    constexpr int QS = Q - 1;
    constexpr int H = 16 / (int)sizeof(S);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    constexpr int rows = ROWS;  // == sh.ty * sh.tz
    constexpr int BW = TW + 2 * H;
    constexpr int SLAB = ((BW * ROWS * (int)sizeof(S)) + 127) / 128 * 128 / (int)sizeof(S);
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, rows, stages);
    StageHdr* hdr = reinterpret_cast<StageHdr*>(smem + LY.hdr_off);
    Cand* cands = reinterpret_cast<Cand*>(smem + LY.cand_off);
    float* edgev = reinterpret_cast<float*>(smem + LY.edge_off);  // [stages][rows][QE]
    constexpr int QE = edge_pops(Q);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY.bar_off);
    uint64_t* empty = full + stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nc = (blockDim.x >> 5) - 1;  // consumer warps
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nc);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        bool ok = true;
        int issued = 0;
        // tiles from a work counter, claimed one iteration ahead so that the
        // atomic's latency hides behind the current tile's staging
        int t_next = 0;
        if (lane == 0) t_next = atomicAdd(&tile_ctr[0], 1);
        // instance of a tile without a memory round trip: a vote over the
        // instances' first tiles held in the lanes (the table for > 32 instances)
        int tile0_l = 0x7fffffff;
        if (ninst <= 32 && lane < ninst) tile0_l = insts[lane].tile0;
        for (int it = 0;; ++it) {
            const int s = it % stages;
            const uint32_t ph = (uint32_t)(it / stages) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT_NS)) {
                ok = false;
                break;
            }
            const int claim = __shfl_sync(0xffffffffu, t_next, 0);
            // claims alternate between the two ends of the tile range, so the
            // slower boundary rows of both y faces come first, not last
            const int t = (claim & 1) ? ntiles - 1 - (claim >> 1) : (claim >> 1);
            if (claim >= ntiles) {
                if (lane == 0) {
                    hdr[s].tile = -1;
                    mbar_arrive(&full[s]);
                }
                break;
            }
            const int ii = ninst <= 32 ? __popc(__ballot_sync(0xffffffffu, t >= tile0_l)) - 1 : tile_inst[t];
            const InstDesc& in = insts[ii];
            const int local = t - in.tile0;
            const int ntx = in.ntile[0], nty = in.ntile[1];
            const int x0 = (local % ntx) * TW, rest = local / ntx;
            const int y0 = (rest % nty) * sh.ty, z0 = (rest / nty) * sh.tz;
            if (lane == 0) t_next = atomicAdd(&tile_ctr[0], 1);
            // the copies go out first; the tile's header and candidates are
            // staged while they are in flight, and the arrive that completes the
            // phase follows them
            if (lane == 0) {
                const CUtensorMap* map = tmaps + 2 * ii + par;
                mbar_expect_tx(&full[s], (uint32_t)(QS * LY.bw * rows * (int)sizeof(S)));
                unsigned char* dst = smem + s * LY.stage;
#pragma unroll 1
                for (int q = 1; q < Q; ++q) {
                    const int cy = Q == 9 ? d2q9_c(q, 1) : d3q19_c(q, 1);
                    const int cz = Q == 9 ? 0 : d3q19_c(q, 2);
                    if (D == 2)
                        tma_load_3d(dst + (q - 1) * LY.slab, map, x0 - H, y0 - cy, q - 1, &full[s]);
                    else
                        tma_load_4d(dst + (q - 1) * LY.slab, map, x0 - H, y0 - cy, z0 - cz, q - 1, &full[s]);
                }
            }
            // the x-edge node's populations from across its face, one lane per
            // (row, population): independent loads, in the shadow of the copies
            const bool eleft = x0 == 0, eright = x0 + TW >= in.n[0];
            const int ex = eleft && eright ? -2 : eleft ? 0 : eright ? in.n[0] - 1 : -1;
            const int ecx = eleft ? 1 : -1;
            if (ex >= 0) {
                float* ev = edgev + s * rows * QE;
                for (int l = lane; l < rows * QE; l += 32) {
                    const int r = l / QE, k = l % QE;
                    const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
                    int q = 1;  // the k-th population with c_x = ecx
                    for (int m = 0, qq = 1; qq < Q; ++qq)
                        if (L::c(qq, 0) == ecx && m++ == k) q = qq;
                    ev[l] = (y < in.n[1] && z < in.n[2])
                                ? pull_scalar<Q, S>(in, static_cast<const S*>(in.f[par]), q, ex, y, z)
                                : 0.f;
                }
            }
            int ncand = 0;
            if (in.np > 0) {
                ncand = min(in.list_cnt[par][local], LIST_CAP);
                Cand* cs = cands + s * LIST_CAP;
                for (int c = lane; c < ncand; c += 32) {
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
                    cs[c] = cd;
                }
                if (commit && lane == 0) in.list_cnt[par ^ 1][local] = 0;
            }
            if (lane == 0) {
                StageHdr& h = hdr[s];
                h.inst = ii;
                h.x0 = x0;
                h.y0 = y0;
                h.z0 = z0;
                for (int d = 0; d < 3; ++d) {
                    h.n[d] = in.n[d];
                    h.per[d] = in.periodic[d];
                    h.gdrive[d] = in.gdrive[d];
                }
                h.pitch = in.pitch;
                h.maxk = in.maxk;
                h.qstride = in.qstride;
                h.sload = in.s_load;
                h.sstore = in.s_store;
                h.ck = make_collk<Q>(make_collp(in));
                h.fin = in.f[par];
                h.fout = in.f[par ^ 1];
                h.partial = commit ? in.partial : in.partial_scratch;
                h.prec = in.prec;
                h.status = in.status;
                h.tile = t;
                h.ncand = ncand;
                h.ex = ex;
                h.ecx = ecx;
            }
            __syncwarp();  // the lanes' candidate and edge records are visible to lane 0's arrive
            if (lane == 0) mbar_arrive(&full[s]);
            ++issued;
        }
        if (!ok) {
            if (lane == 0) atomicOr(insts[0].status, ST_TIMEOUT);
            // let the copies this warp issued land before the block exits
            for (int k = max(0, issued - stages); k < issued; ++k)
                mbar_wait(&full[k % stages], (uint32_t)(k / stages) & 1u, WAIT_LIMIT_NS);
        }
        if (lane == 0) {  // the last block to leave resets the work counter
            __threadfence();
            if (atomicAdd(&tile_ctr[1], 1) == (int)gridDim.x - 1) {
                tile_ctr[0] = 0;
                tile_ctr[1] = 0;
            }
        }
        return;
    }

    // ------------------------------------------------------------- consumers
    const int cw = warp - 1;
    for (int it = 0;; ++it) {
        const int s = it % stages;
        const uint32_t ph = (uint32_t)(it / stages) & 1u;
        if (!mbar_wait(&full[s], ph, WAIT_LIMIT_NS)) {
            if (lane == 0) atomicOr(insts[0].status, ST_TIMEOUT);
            return;
        }
        const int t = hdr[s].tile;
        if (t < 0) return;
        const StageHdr& h = hdr[s];
        const int ncand = h.ncand;
        const Cand* cand = cands + s * LIST_CAP;
        Geo geo;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            geo.n[d] = h.n[d];
            geo.per[d] = h.per[d];
        }
        geo.prec = h.prec;
        const int nx = h.n[0], ny = h.n[1], nz = h.n[2];
        const int x0 = h.x0, y0 = h.y0, z0 = h.z0;
        const S* stage = reinterpret_cast<const S*>(smem + s * LY.stage);
        const int ex = h.ex, ecx = h.ecx;
        const float* ev = edgev + s * rows * QE;
        bool bad = false;
        for (int r = cw; r < rows; r += nc) {
            const int y = y0 + r % sh.ty, z = z0 + r / sh.ty;
            if (y >= ny || z >= nz) continue;
            // populations whose source row lies inside the staged box
            unsigned rowok = 0;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const int ys = y - L::c(q, 1), zs = z - L::c(q, 2);
                if (ys >= 0 && ys < ny && zs >= 0 && zs < nz) rowok |= 1u << q;
            }
            const bool rowfast = rowok == (((1u << Q) - 1) & ~1u);
            const S* rowbase = stage + r * BW + H;
            S* outrow = static_cast<S*>(h.fout) + ((long long)z * ny + y) * h.pitch;
            // two adjacent nodes per lane: packed FP32x2 arithmetic, 8-byte stores
            for (int j = 0; j < TW / 64; ++j) {
                const int lx = j * 64 + 2 * lane;
                const int x = x0 + lx;
                const bool v0 = x < nx, v1 = x + 1 < nx;
                float2 f[QS];
                if (rowfast && (ex >= 0 || __all_sync(0xffffffffu, x > 0 && x + 1 < nx - 1))) {
#pragma unroll
                    for (int q = 1; q < Q; ++q) {
                        const S* src = rowbase + (q - 1) * SLAB + lx - L::c(q, 0);
                        if (L::c(q, 0) == 0) f[q - 1] = smem_pair(src, h.sload);
                        else f[q - 1] = make_float2(to_float_scaled(src[0], h.sload), to_float_scaled(src[1], h.sload));
                    }
                    // the edge node's populations from across the face (the box
                    // holds zero fill or a neighbour column there); nodes past
                    // nx in a ragged tile are computed but never stored
                    const int e = ex - x;
                    if (ex >= 0 && (e == 0 || e == 1)) {
                        int k = 0;
#pragma unroll
                        for (int q = 1; q < Q; ++q) {
                            if (L::c(q, 0) != 1 && L::c(q, 0) != -1) continue;
                            if (L::c(q, 0) != ecx) continue;
                            const float vv = ev[r * QE + k];
                            ++k;
                            if (e == 0) f[q - 1].x = vv;
                            else f[q - 1].y = vv;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 1; q < Q; ++q) {
                        const int cx = L::c(q, 0);
                        float v[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int xe = x + e;
                            if (((rowok >> q) & 1u) && xe - cx >= 0 && xe - cx < nx)
                                v[e] = to_float_scaled(rowbase[(q - 1) * SLAB + lx + e - cx], h.sload);
                            else
                                v[e] = xe < nx ? pull_scalar<Q, S>(insts[h.inst], static_cast<const S*>(h.fin), q, xe,
                                                                     y, z)
                                               : 0.f;
                        }
                        f[q - 1] = make_float2(v[0], v[1]);
                    }
                }
                const int xyz0[3] = {x, y, z}, xyz1[3] = {x + 1, y, z};
                int own0 = -1, own1 = -1, sl0 = -1, sl1 = -1;
                unsigned act = 0;
                if (ncand > 32) {  // more candidates than mask bits: test them all
                    act = 0xffffffffu;
                    own0 = owner_of<D>(geo, cand, ncand, xyz0, &sl0);
                    own1 = owner_of<D>(geo, cand, ncand, xyz1, &sl1);
                } else if (ncand > 0) {
                    act = segment_candidates<D>(geo, cand, ncand, x0 + j * 64, y, z, 64);
                    if (act) {
                        own0 = owner_masked<D>(geo, cand, act, xyz0, &sl0);
                        own1 = owner_masked<D>(geo, cand, act, xyz1, &sl1);
                    }
                }
                float2 a[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    a[d] = add2(bc2(h.gdrive[d]),
                                make_float2(own0 >= 0 ? cand[sl0].a[d] : 0.f, own1 >= 0 ? cand[sl1].a[d] : 0.f));
                float2 u[3], p;
                collide2<Q>(f, a, own0 >= 0, own1 >= 0, h.ck, u, &p);
                float2 uu = mul2(u[0], u[0]);
#pragma unroll
                for (int d = 1; d < D; ++d) uu = fma2(u[d], u[d], uu);
                bad |= (v0 && !(uu.x < 0.25f)) || (v1 && !(uu.y < 0.25f));
                if (v0) {
                    S* o = outrow + x;
                    const int qs = (int)h.qstride;  // < 2^31 elements per population
                    const float sstore = h.sstore;
                    if (v1) {
#pragma unroll
                        for (int q = 0; q < QS; ++q) {
                            store_pair(o, f[q], sstore);
                            o += qs;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < QS; ++q) {
                            *o = to_store<S>(f[q].x, sstore);
                            o += qs;
                        }
                    }
                }
                if (act) {
                    const int slot[2] = {v0 ? sl0 : -1, v1 ? sl1 : -1};
                    const float uv[3][2] = {{u[0].x, u[0].y}, {u[1].x, u[1].y}, {D == 3 ? u[2].x : 0.f, D == 3 ? u[2].y : 0.f}};
                    row_partials<D, 2>(geo, cand, ncand, h.partial, h.maxk, slot, uv, x, y, z, lane);
                }
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(h.status, ST_DIVERGED);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------- host side ---
template <int Q, class S, int TW, int ROWS>
static cudaError_t launch_tma_t(const InstDesc* insts, const void* tmaps, const uint16_t* tile_inst,
                                int ntiles, int par, const Shape& sh, int commit, int grid,
                                int* tile_ctr, int stages, int ninst, cudaStream_t st) {
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, ROWS, stages);
    k_fluid_tma<Q, S, TW, ROWS><<<grid, 32 * (sh.warps + 1), LY.bytes, st>>>(
        insts, static_cast<const CUtensorMap*>(tmaps), tile_inst, ntiles, par, sh, commit, tile_ctr,
        stages, ninst);
    return cudaGetLastError();
}

int tma_tile_width(int Q) { return Q == 9 ? 128 : 64; }

bool tma_rows_ok(int rows) { return rows == 4 || rows == 8; }

template <int Q, class S, int TW, int ROWS>
static int tma_blocks_t(const Shape& sh, int stages) {
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, ROWS, stages);
    if (cudaFuncSetAttribute(k_fluid_tma<Q, S, TW, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             LY.bytes) != cudaSuccess)
        return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fluid_tma<Q, S, TW, ROWS>, 32 * (sh.warps + 1),
                                                  LY.bytes);
    return nb;
}

#define LBM_TMA_DISPATCH(CALL)                                                          \
    {                                                                                   \
        const int rows = sh.ty * sh.tz;                                                 \
        if (Q == 9 && !fp16 && rows == 4) return CALL(9, float, 128, 4);                \
        if (Q == 9 && !fp16 && rows == 8) return CALL(9, float, 128, 8);                \
        if (Q == 9 && fp16 && rows == 4) return CALL(9, __half, 128, 4);                \
        if (Q == 9 && fp16 && rows == 8) return CALL(9, __half, 128, 8);                \
        if (Q == 19 && !fp16 && rows == 4) return CALL(19, float, 64, 4);               \
        if (Q == 19 && !fp16 && rows == 8) return CALL(19, float, 64, 8);               \
        if (Q == 19 && fp16 && rows == 4) return CALL(19, __half, 64, 4);               \
        if (Q == 19 && fp16 && rows == 8) return CALL(19, __half, 64, 8);               \
    }

int fluid_tma_blocks_per_sm(int Q, int fp16, const Shape& sh, int stages) {
#define LBM_BLK(QQ, SS, TT, RR) tma_blocks_t<QQ, SS, TT, RR>(sh, stages)
    LBM_TMA_DISPATCH(LBM_BLK)
#undef LBM_BLK
    return 0;
}

cudaError_t launch_fluid_tma(int Q, int fp16, const InstDesc* insts, const void* tmaps,
                             const uint16_t* tile_inst, int ntiles, int par, const Shape& sh,
                             int commit, int grid, int* tile_ctr, int stages, int ninst, cudaStream_t st) {
#define LBM_LAUNCH(QQ, SS, TT, RR)                                                                    \
    launch_tma_t<QQ, SS, TT, RR>(insts, tmaps, tile_inst, ntiles, par, sh, commit, grid, tile_ctr, stages, \
                                 ninst, st)
    LBM_TMA_DISPATCH(LBM_LAUNCH)
#undef LBM_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace lbmpen
