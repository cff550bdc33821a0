// TMA-pipelined variant of the fused stream-collide-penalize kernel.
//
// Persistent blocks of one producer warp and NC consumer warps.  The producer
// takes tiles from a work counter (successive claims alternate between the
// two ends of the tile range) and fills a ring of shared-memory stages: the
// tile's populations by cp.async.bulk.tensor (D2Q9: one box of every
// population over the tile rows and one halo row on each side; D3Q19: one
// box per population over its source rows y - c_y, z - c_z), 32*k nodes wide
// plus a 16-byte halo on both sides so that every box starts on a 16-byte
// boundary, and the tile's candidate particles by one bulk copy of the
// records the particle kernel listed for the tile.  Everything else the
// producer needs comes from a per-block shared table of instance constants,
// or was fetched one tile ahead (the next tile's list count and the values
// its x-edge node pulls across the face, by cp.async), so its own path per
// tile touches no global memory.  The copies of a stage are counted by its
// mbarrier; each consumer lane pulls two adjacent nodes' populations from
// shared memory at x - c_x, collides them with packed FP32x2 arithmetic,
// stores them to HBM with 8-byte coalesced stores, and stores the velocity
// of each solid node into its particle's box for the sums of Eq. 22.  Rows whose source lies beyond a y or z face
// gather those populations from HBM directly, as the register-path kernel
// does.
//
// Every mbarrier wait is bounded in time; on expiry the kernel records a
// timeout in the status word, waits (bounded) for the copies it issued and
// returns.
#include <cuda.h>

#include <type_traits>

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

// One bulk copy global -> shared counted by an mbarrier (16-byte aligned
// addresses, a multiple of 16 bytes).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 4-byte asynchronous copy global -> shared (completion: cp_async_wait_all)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// The constants of one instance that a tile needs, copied once per block
// into a shared-memory table (for up to TI_MAX instances) so that neither the
// producer nor the consumers go to global memory for them in the tile loop.
struct __align__(16) TInst {
    const void* f[2];          // population buffers
    float* ubox[2];            // velocity boxes: [0] the state's, [1] scratch
    const PRec* prec;
    int* status;
    int* lcnt[2];              // tile list counts per parity
    const Cand* lrec[2];       // candidate records per parity
    long long qstride;
    int tile0, ntx, nty, pitch, np, maxk;
    int n[3], per[3];
    float gdrive[3], sload, sstore, keep, fpref, alpha;
    float ewt[2][5];           // moving-wall term of the populations an x-edge node pulls
                               //   across the low (0) / high (1) x face
};
constexpr int TI_MAX = 64;
constexpr int TI_WORDS = (int)(sizeof(TInst) / 16);

template <int Q>
__device__ __forceinline__ void make_tinst(TInst& t, const InstDesc& in) {
    for (int b = 0; b < 2; ++b) {
        t.f[b] = in.f[b];
        t.lcnt[b] = in.list_cnt[b];
        t.lrec[b] = static_cast<const Cand*>(in.list_rec[b]);
    }
    t.ubox[0] = in.ubox;
    t.ubox[1] = in.ubox_scratch;
    t.prec = in.prec;
    t.status = in.status;
    t.qstride = in.qstride;
    t.tile0 = in.tile0;
    t.ntx = in.ntile[0];
    t.nty = in.ntile[1];
    t.pitch = in.pitch;
    t.np = in.np;
    t.maxk = in.maxk;
    for (int d = 0; d < 3; ++d) {
        t.n[d] = in.n[d];
        t.per[d] = in.periodic[d];
        t.gdrive[d] = in.gdrive[d];
    }
    t.sload = in.s_load;
    t.sstore = in.s_store;
    t.keep = in.keep;
    t.fpref = in.fpref;
    t.alpha = in.alpha;
    for (int face = 0; face < 2; ++face)
        for (int k = 0; k < 5; ++k) t.ewt[face][k] = 0.f;
    for (int face = 0; face < 2; ++face) {  // face 0 is pulled across by c_x = +1, face 1 by c_x = -1
        const int ecx = face == 0 ? 1 : -1;
        for (int k = 0, q = 1; q < Q; ++q)
            if (Lat<Q>::c(q, 0) == ecx) t.ewt[face][k++] = in.wterm[0][face][q];
    }
}

// Per-tile record the producer writes next to the staged populations.
struct __align__(16) StageHdr {
    TInst ti;   // the tile's instance
    int tile;   // global tile index, -1 = no more work
    int ncand;
    int inst;
    int x0, y0, z0;
    int ex;     // x of the tile's edge node whose face values are staged, -1 none,
                //   -2 both edges in one tile (those take the direct gathers)
    int ecx;    // c_x of the staged populations: +1 at x = 0, -1 at x = nx - 1
};

// The next tile of the producer, prepared one iteration ahead: its place,
// its list count (lane 0) and the values its x-edge node pulls across the face
// (two per lane, loads in flight while the producer waits for a free stage).
// The next tile of the producer, prepared one iteration ahead: its place in
// registers; its list count and the values its x-edge node pulls across the
// face in flight to the shared prefetch buffer (cp.async) while the producer
// waits for a free stage.
struct TileAhead {
    int t, ii, local, x0, y0, z0, ex, ecx, np;
    float sload;
    float add[2];
    int hsel;  // FP16: bit j set = value j is the upper half of its 4-byte word
};
constexpr int PRE_WORDS = 72;  // per prefetch buffer: 64 edge values, the list count

}  // namespace

// Geometry of the shared-memory ring, identical on host and device.
struct TmaLayout {
    int bw;          // box width (nodes) = tile width + 2 halo
    int slab;        // bytes of one population box, rounded to 128
    int stage;       // bytes of all populations of one stage
    int pops_bytes;  // stages * stage
    int hdr_off, cand_off, edge_off, tab_off, pre_off, bar_off, bytes;
};

// Populations with c_x = +1 (equally, -1): the ones an x-edge node pulls
// across its face.
__host__ __device__ constexpr int edge_pops(int Q) { return Q == 9 ? 3 : 5; }

__host__ __device__ inline TmaLayout tma_layout(int Q, int ssize, int tw, int rows, int stages, int ninst) {
    TmaLayout L;
    const int halo = 16 / ssize;
    const int ntab = ninst < TI_MAX ? ninst : TI_MAX;
    L.bw = tw + 2 * halo;
    if (Q == 9) {  // one box per tile: all populations, rows y0 - 1 .. y0 + rows, densely packed
        L.slab = L.bw * (rows + 2) * ssize;
        L.stage = ((Q - 1) * L.slab + 127) & ~127;
    } else {       // one box per population, rows y0 - c_y .., each slab 128-byte aligned
        L.slab = ((L.bw * rows * ssize) + 127) & ~127;
        L.stage = (Q - 1) * L.slab;
    }
    L.pops_bytes = stages * L.stage;
    L.hdr_off = L.pops_bytes;
    L.cand_off = L.hdr_off + (int)sizeof(StageHdr) * stages;  // 16-byte aligned (bulk copies)
    L.edge_off = L.cand_off + CAND_BYTES * LIST_CAP * stages;
    L.tab_off = (L.edge_off + (int)sizeof(float) * rows * edge_pops(Q) * stages + 15) & ~15;
    L.pre_off = L.tab_off + (int)sizeof(TInst) * ntab;
    L.bar_off = L.pre_off + 4 * 2 * PRE_WORDS;
    L.bytes = L.bar_off + 16 * stages + 128;  // + alignment slack of the base
    return L;
}

// The k-th population (0-based) with c_x == ecx.
template <int Q>
__device__ __forceinline__ int edge_pop(int ecx, int k) {
    using L = Lat<Q>;
    int q = 1;
    for (int m = 0, qq = 1; qq < Q; ++qq)
        if (L::c(qq, 0) == ecx && m++ == k) q = qq;
    return q;
}

// Register budget: two blocks of 9 warps per SM; each lane collides two
// nodes at a time.
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
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // Base of the ring rounded up to 128 bytes by an offset from the shared
    // array itself: a pointer rebuilt from an integer would lose its address
    // space, and every access through it would become a generic load.
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    constexpr int rows = ROWS;  // == sh.ty * sh.tz
    constexpr int BW = TW + 2 * H;
    // elements between populations in a stage, and the row offset of population
    // q's source row y - c_y: D2Q9 boxes span rows y0 - 1 .. y0 + rows (one copy
    // per tile), D3Q19 boxes start at the source rows (one copy per population)
    constexpr int SLAB = Q == 9 ? BW * (ROWS + 2)
                                : ((BW * ROWS * (int)sizeof(S)) + 127) / 128 * 128 / (int)sizeof(S);
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, rows, stages, ninst);
    StageHdr* hdr = reinterpret_cast<StageHdr*>(smem + LY.hdr_off);
    Cand* cands = reinterpret_cast<Cand*>(smem + LY.cand_off);
    float* edgev = reinterpret_cast<float*>(smem + LY.edge_off);  // [stages][rows][QE]
    TInst* tab = reinterpret_cast<TInst*>(smem + LY.tab_off);
    uint32_t* pre = reinterpret_cast<uint32_t*>(smem + LY.pre_off);  // [2][PRE_WORDS]
    constexpr int QE = edge_pops(Q);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + LY.bar_off);
    uint64_t* empty = full + stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nc = (blockDim.x >> 5) - 1;  // consumer warps
    const int ntab = ninst < TI_MAX ? ninst : TI_MAX;
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nc);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < ntab; i += blockDim.x) make_tinst<Q>(tab[i], insts[i]);
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        // Tiles come from a work counter; claims alternate between the two
        // ends of the tile range (the slower y-face rows come first).  Two
        // claims are in flight, and everything the next tile needs from
        // global memory is loaded one iteration ahead, so the producer's
        // own path per tile touches only shared memory.
        bool ok = true;
        int issued = 0;
        int c_cur = 0, c_nxt = 0;
        if (lane == 0) {
            c_cur = atomicAdd(&tile_ctr[0], 1);
            c_nxt = atomicAdd(&tile_ctr[0], 1);
        }
        // instance of a tile without a memory round trip: votes over the
        // first tiles of up to TI_MAX instances in the table (lanes hold two)
        const int tf0 = lane < ntab ? tab[lane].tile0 : 0x7fffffff;
        const int tf1 = lane + 32 < ntab ? tab[lane + 32].tile0 : 0x7fffffff;
        auto ahead = [&](int c, int buf) {
            TileAhead a;
            a.t = -1;
            a.np = 0;
            a.ex = -1;
            a.ecx = 1;
            a.sload = 1.f;
            a.add[0] = a.add[1] = 0.f;
            a.hsel = 0;
            uint32_t* pb = pre + buf * PRE_WORDS;
            const int cc = __shfl_sync(0xffffffffu, c, 0);
            if (cc >= ntiles) return a;
            const int t = (cc & 1) ? ntiles - 1 - (cc >> 1) : (cc >> 1);
            a.t = t;
            a.ii = ninst <= TI_MAX ? __popc(__ballot_sync(0xffffffffu, t >= tf0)) +
                                         __popc(__ballot_sync(0xffffffffu, t >= tf1)) - 1
                                   : (int)tile_inst[t];
            const InstDesc& in = insts[a.ii];
            const bool tb = ninst <= TI_MAX;
            const int tile0 = tb ? tab[a.ii].tile0 : in.tile0;
            const int ntx = tb ? tab[a.ii].ntx : in.ntile[0];
            const int nty = tb ? tab[a.ii].nty : in.ntile[1];
            const int n[3] = {tb ? tab[a.ii].n[0] : in.n[0], tb ? tab[a.ii].n[1] : in.n[1],
                              tb ? tab[a.ii].n[2] : in.n[2]};
            a.np = tb ? tab[a.ii].np : in.np;
            a.sload = tb ? tab[a.ii].sload : in.s_load;
            a.local = t - tile0;
            a.x0 = (a.local % ntx) * TW;
            const int rest = a.local / ntx;
            a.y0 = (rest % nty) * sh.ty;
            a.z0 = (rest / nty) * sh.tz;
            if (lane == 0) {
                if (a.np > 0) cp_async4(pb + 64, (tb ? tab[a.ii].lcnt[par] : in.list_cnt[par]) + a.local);
                else pb[64] = 0u;
            }
            const bool eleft = a.x0 == 0, eright = a.x0 + TW >= n[0];
            a.ex = eleft && eright ? -2 : eleft ? 0 : eright ? n[0] - 1 : -1;
            a.ecx = eleft ? 1 : -1;
            if (a.ex >= 0) {
                // the value edge node x = ex pulls across its x face in a row whose
                // other sources lie inside the box (rows that do not use it may
                // get any in-bounds value)
                const S* fin = static_cast<const S*>(tb ? tab[a.ii].f[par] : in.f[par]);
                const long long qstr = tb ? tab[a.ii].qstride : in.qstride;
                const int pitch = tb ? tab[a.ii].pitch : in.pitch;
                const bool xper = (tb ? tab[a.ii].per[0] : in.periodic[0]) != 0;
                const int face = a.ecx > 0 ? 0 : 1;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int l = lane + 32 * j;
                    if (l >= rows * QE) continue;
                    const int r = l / QE, k = l % QE;
                    const int q = edge_pop<Q>(a.ecx, k);
                    const int y = a.y0 + r % sh.ty, z = a.z0 + r / sh.ty;
                    const int ys = y - L::c(q, 1), zs = z - L::c(q, 2);
                    const S* src = nullptr;
                    if (!xper) {  // bounce-back at the x wall
                        if (y < n[1] && z < n[2])
                            src = fin + (long long)(L::opp(q) - 1) * qstr + ((long long)z * n[1] + y) * pitch + a.ex;
                        a.add[j] = tb ? tab[a.ii].ewt[face][k] : in.wterm[0][face][q];
                    } else if (y < n[1] && z < n[2] && ys >= 0 && ys < n[1] && zs >= 0 && zs < n[2]) {
                        const int xs = a.ecx > 0 ? n[0] - 1 : 0;  // periodic wrap
                        src = fin + (long long)(q - 1) * qstr + ((long long)zs * n[1] + ys) * pitch + xs;
                    }
                    if (src) {
                        const uintptr_t ad = reinterpret_cast<uintptr_t>(src);
                        if (sizeof(S) == 2 && (ad & 2)) a.hsel |= 1 << j;
                        cp_async4(pb + l, reinterpret_cast<const void*>(ad & ~(uintptr_t)3));
                    } else {
                        pb[l] = 0u;
                    }
                }
            }
            cp_async_commit();
            return a;
        };
        TileAhead nx_ = ahead(c_cur, 0);
        for (int it = 0;; ++it) {
            const int s = it % stages;
            const uint32_t ph = (uint32_t)(it / stages) & 1u;
            if (!mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT_NS)) {
                ok = false;
                break;
            }
            const TileAhead a = nx_;
            const uint32_t* pb = pre + (it & 1) * PRE_WORDS;
            if (a.t < 0) {
                if (lane == 0) {
                    hdr[s].tile = -1;
                    mbar_arrive(&full[s]);
                }
                break;
            }
            cp_async_wait_all();  // this tile's count and edge values, copied one iteration ago
            __syncwarp();
            const int ncand = min((int)pb[64], LIST_CAP);
            StageHdr& h = hdr[s];
            if (lane == 0) {
                const CUtensorMap* map = tmaps + 2 * a.ii + par;
                unsigned char* dst = smem + s * LY.stage;
                if (Q == 9) {
                    mbar_expect_tx(&full[s], (uint32_t)(QS * LY.bw * (rows + 2) * (int)sizeof(S) + CAND_BYTES * ncand));
                    tma_load_3d(dst, map, a.x0 - H, a.y0 - 1, 0, &full[s]);
                } else {
                    mbar_expect_tx(&full[s], (uint32_t)(QS * LY.bw * rows * (int)sizeof(S) + CAND_BYTES * ncand));
#pragma unroll 1
                    for (int q = 1; q < Q; ++q)
                        tma_load_4d(dst + (q - 1) * LY.slab, map, a.x0 - H, a.y0 - d3q19_c(q, 1),
                                    a.z0 - d3q19_c(q, 2), q - 1, &full[s]);
                }
                if (ncand > 0) {
                    const Cand* lr = ninst <= TI_MAX ? tab[a.ii].lrec[par]
                                                     : static_cast<const Cand*>(insts[a.ii].list_rec[par]);
                    bulk_load(cands + s * LIST_CAP, lr + (long long)a.local * LIST_CAP,
                              (uint32_t)(CAND_BYTES * ncand), &full[s]);
                }
            }
            // the tile's constants, its edge values and its header
            if (ninst <= TI_MAX) {
                if (lane < TI_WORDS)
                    reinterpret_cast<uint4*>(&h.ti)[lane] = reinterpret_cast<const uint4*>(&tab[a.ii])[lane];
            } else if (lane == 0) {
                make_tinst<Q>(h.ti, insts[a.ii]);
            }
            if (a.ex >= 0) {
                float* ev = edgev + s * rows * QE;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int l = lane + 32 * j;
                    if (l < rows * QE) {
                        const uint32_t w = pb[l];
                        float v;
                        if (sizeof(S) == 2) {
                            const unsigned short hb = (unsigned short)(((a.hsel >> j) & 1) ? (w >> 16) : (w & 0xffffu));
                            v = __half2float(__ushort_as_half(hb)) * a.sload;
                        } else {
                            v = __uint_as_float(w);
                        }
                        ev[l] = v + a.add[j];
                    }
                }
            }
            if (lane == 0) {
                h.tile = a.t;
                h.inst = a.ii;
                h.x0 = a.x0;
                h.y0 = a.y0;
                h.z0 = a.z0;
                h.ncand = ncand;
                h.ex = a.ex;
                h.ecx = a.ecx;
                if (commit && a.np > 0)  // this tile's list of the next step starts empty
                    (ninst <= TI_MAX ? tab[a.ii].lcnt[par ^ 1] : insts[a.ii].list_cnt[par ^ 1])[a.local] = 0;
            }
            __syncwarp();  // the lanes' table copy and edge values are visible to lane 0's arrive
            if (lane == 0) mbar_arrive(&full[s]);
            ++issued;
            // the next tile: its claim has been in flight for a whole tile
            if (lane == 0) {
                c_cur = c_nxt;
                c_nxt = atomicAdd(&tile_ctr[0], 1);
            }
            __syncwarp();  // every lane has read this buffer before it is refilled
            nx_ = ahead(c_cur, (it + 1) & 1);
        }
        cp_async_wait_all();  // no copy of this warp outlives it
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
            geo.n[d] = h.ti.n[d];
            geo.per[d] = h.ti.per[d];
        }
        geo.prec = h.ti.prec;
        const int nx = h.ti.n[0], ny = h.ti.n[1], nz = h.ti.n[2];
        const float sload = h.ti.sload;
        const CollK ck = make_collk<Q>(CollP{h.ti.keep, h.ti.fpref, h.ti.alpha});
        float* const ubox = h.ti.ubox[commit ? 0 : 1];
        const int x0 = h.x0, y0 = h.y0, z0 = h.z0;
        const S* stage = reinterpret_cast<const S*>(smem + s * LY.stage);
        const int ex = h.ex, ecx = h.ecx;
        const float* ev = edgev + s * rows * QE;
        bool bad = false;
        const float sstore_t = h.ti.sstore;
        // FOLD (D2Q9, FP16 storage at tau = 1): the populations stay at the
        // storage scale from the stage to the store (collide2_t1_scaled)
        auto tile_rows = [&](auto fold_tag) {
            constexpr bool FOLD = decltype(fold_tag)::value;
            CollK cks = ck;
            if constexpr (FOLD) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    cks.A[i] *= sstore_t;
                    cks.fA[i] *= sstore_t;
                    cks.sA[i] *= sstore_t;
                }
            }
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
                // element of population q's source row in the stage, relative to rowbase
                auto qoff = [&](int q) { return (q - 1) * SLAB + (Q == 9 ? (1 - L::c(q, 1)) * BW : 0); };
                S* outrow = static_cast<S*>(const_cast<void*>(h.ti.f[par ^ 1])) + ((long long)z * ny + y) * h.ti.pitch;
                // two adjacent nodes per lane: packed FP32x2 arithmetic, 8-byte stores
                for (int j = 0; j < TW / 64; ++j) {
                    const int lx = j * 64 + 2 * lane;
                    const int x = x0 + lx;
                    const bool v0 = x < nx, v1 = x + 1 < nx;
                    float2 f[QS];
                    if (rowfast && (ex >= 0 || __all_sync(0xffffffffu, x > 0 && x + 1 < nx - 1))) {
#pragma unroll
                        for (int q = 1; q < Q; ++q) {
                            const S* src = rowbase + qoff(q) + lx - L::c(q, 0);
                            if constexpr (FOLD) {
                                if (L::c(q, 0) == 0) f[q - 1] = __half22float2(*reinterpret_cast<const __half2*>(src));
                                else f[q - 1] = make_float2(__half2float(src[0]), __half2float(src[1]));
                            } else {
                                if (L::c(q, 0) == 0) f[q - 1] = smem_pair(src, sload);
                                else
                                    f[q - 1] = make_float2(to_float_scaled(src[0], sload),
                                                           to_float_scaled(src[1], sload));
                            }
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
                                const float vv = FOLD ? ev[r * QE + k] * sstore_t : ev[r * QE + k];
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
                                if (((rowok >> q) & 1u) && xe - cx >= 0 && xe - cx < nx) {
                                    if constexpr (FOLD) v[e] = __half2float(rowbase[qoff(q) + lx + e - cx]);
                                    else v[e] = to_float_scaled(rowbase[qoff(q) + lx + e - cx], sload);
                                } else {
                                    const S* fin = static_cast<const S*>(h.ti.f[par]);
                                    v[e] = xe < nx ? pull_scalar<Q, S>(insts[h.inst], fin, q, xe, y, z) : 0.f;
                                    if constexpr (FOLD) v[e] *= sstore_t;
                                }
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
                        act = segment_candidates<D>(geo, cand, ncand, x0 + j * 64, y, z, 64, lane);
                        if (act) {
                            own0 = owner_masked<D>(geo, cand, act, xyz0, &sl0);
                            own1 = owner_masked<D>(geo, cand, act, xyz1, &sl1);
                        }
                    }
                    float2 a[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        a[d] = add2(bc2(h.ti.gdrive[d]),
                                    make_float2(own0 >= 0 ? cand[sl0].a[d] : 0.f, own1 >= 0 ? cand[sl1].a[d] : 0.f));
                    float2 u[3], p;
                    if constexpr (FOLD) collide2_t1_scaled<Q>(f, a, own0 >= 0, own1 >= 0, cks, sload, u, &p);
                    else collide2<Q>(f, a, own0 >= 0, own1 >= 0, ck, u, &p);
                    float2 uu = mul2(u[0], u[0]);
#pragma unroll
                    for (int d = 1; d < D; ++d) uu = fma2(u[d], u[d], uu);
                    bad |= (v0 && !(uu.x < 0.25f)) || (v1 && !(uu.y < 0.25f));
                    if (v0) {
                        S* o = outrow + x;
                        const int qs = (int)h.ti.qstride;  // < 2^31 elements per population
                        const float sstore = h.ti.sstore;
                        if (v1) {
#pragma unroll
                            for (int q = 0; q < QS; ++q) {
                                if constexpr (FOLD) *reinterpret_cast<__half2*>(o) = __floats2half2_rn(f[q].x, f[q].y);
                                else store_pair(o, f[q], sstore);
                                o += qs;
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < QS; ++q) {
                                if constexpr (FOLD) *o = __float2half_rn(f[q].x);
                                else *o = to_store<S>(f[q].x, sstore);
                                o += qs;
                            }
                        }
                    }
                    // the solid nodes' velocities into their particles' boxes (Eq. 22)
                    if (v0 && own0 >= 0)
                        box_store<D>(ubox, geo, cand[sl0], x, y, z, u[0].x, u[1].x, D == 3 ? u[2].x : 0.f);
                    if (v1 && own1 >= 0)
                        box_store<D>(ubox, geo, cand[sl1], x + 1, y, z, u[0].y, u[1].y, D == 3 ? u[2].y : 0.f);
                }
            }
        };
        if constexpr (sizeof(S) == 2 && Q == 9) {  // (D3Q19 would spill more)
            if (ck.keep == 0.f) tile_rows(std::true_type{});
            else tile_rows(std::false_type{});
        } else {
            tile_rows(std::false_type{});
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(h.ti.status, ST_DIVERGED);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// ------------------------------------------------------------- host side ---
template <int Q, class S, int TW, int ROWS>
static cudaError_t launch_tma_t(const InstDesc* insts, const void* tmaps, const uint16_t* tile_inst,
                                int ntiles, int par, const Shape& sh, int commit, int grid,
                                int* tile_ctr, int stages, int ninst, cudaStream_t st) {
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, ROWS, stages, ninst);
    k_fluid_tma<Q, S, TW, ROWS><<<grid, 32 * (sh.warps + 1), LY.bytes, st>>>(
        insts, static_cast<const CUtensorMap*>(tmaps), tile_inst, ntiles, par, sh, commit, tile_ctr,
        stages, ninst);
    return cudaGetLastError();
}

int tma_tile_width(int Q) { return Q == 9 ? 128 : 64; }

bool tma_rows_ok(int rows) { return rows == 4 || rows == 8; }

template <int Q, class S, int TW, int ROWS>
static int tma_blocks_t(const Shape& sh, int stages, int ninst) {
    const TmaLayout LY = tma_layout(Q, (int)sizeof(S), TW, ROWS, stages, ninst);
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

int fluid_tma_blocks_per_sm(int Q, int fp16, const Shape& sh, int stages, int ninst) {
#define LBM_BLK(QQ, SS, TT, RR) tma_blocks_t<QQ, SS, TT, RR>(sh, stages, ninst)
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
