// Host side of the lbmpen C ABI (declared in include/lbmpen.h): context and
// device-memory management, launch sequencing, CUDA-graph replay of the step
// loop, the fluid-kernel autotuner and state import/export.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/lbmpen.h"
#include "lbm_internal.cuh"

namespace lbmpen {
cudaError_t launch_fluid(int Q, int fp16, const InstDesc* insts, const uint16_t* tile_inst,
                         int ntiles, int par, const Shape& sh, int commit, int persistent, int grid,
                         int* tile_ctr, cudaStream_t st);
int fluid_max_blocks_per_sm(int Q, int fp16, const Shape& sh);
cudaError_t launch_fields(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                          const Shape& sh, float* u, float* p, int* owner, cudaStream_t st);
cudaError_t launch_pack(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                        const float* src, cudaStream_t st);
cudaError_t launch_unpack(int Q, int fp16, const InstDesc* insts, int inst, long long N, int par,
                          float* dst, cudaStream_t st);
int particle_blocks_resident(int num_sms);
cudaError_t launch_particles(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int K,
                             int lpar, const Shape& sh, GridBar* gb, bool fused, cudaStream_t st,
                             long long wait_ns);
cudaError_t launch_publish(const InstDesc* insts, const PartRef* refs, int ntotal, int D, int lpar,
                           const Shape& sh, cudaStream_t st);
cudaError_t launch_box_sums(const InstDesc* insts, const PartRef* refs, int ntotal, int D, cudaStream_t st);
int tma_tile_width(int Q);
bool tma_rows_ok(int rows);
int fluid_tma_blocks_per_sm(int Q, int fp16, const Shape& sh, int stages, int ninst);
cudaError_t launch_fluid_tma(int Q, int fp16, const InstDesc* insts, const void* tmaps,
                             const uint16_t* tile_inst, int ntiles, int par, const Shape& sh,
                             int commit, int grid, int* tile_ctr, int stages, int ninst, cudaStream_t st);
cudaError_t launch_adj_fluid(int Q, int fp16, const InstDesc* insts, const AdjFluid* afs,
                             const uint16_t* tile_inst, int ntiles, int lam_mode, const Shape& sh,
                             cudaStream_t st);
cudaError_t launch_adj_particles(int D, const InstDesc* insts, const AdjPart* steps, const AdjBufs* bufs,
                                 int ninst, cudaStream_t st);
cudaError_t launch_adj_finish(const InstDesc* insts, const AdjBufs* bufs, const long long* out_off,
                              double* out, int ninst, cudaStream_t st);
cudaError_t launch_adj_pull_out(int Q, const InstDesc* insts, int inst, long long N, const float* lam,
                                float* out, cudaStream_t st);
cudaError_t launch_adj_state(const InstDesc* insts, int inst, int np, double* rec, int to_record,
                             cudaStream_t st);
}  // namespace lbmpen

using namespace lbmpen;

namespace {

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct Instance {
    lbm_config cfg;
    int n[3];
    int pitch = 0;
    long long qstride = 0;
    int np = 0, cap = 0;
    int ntile[3] = {1, 1, 1};
    int ntiles = 0, tile0 = 0;
    int maxk = 0;
    DevBuf f[2], prec, lcnt[2], lent[2], lrec[2], ubox, ubox_scratch, boxinfo, btot, X, U, W, Un, Wn, theta, A, R, ratio, count, Xk, pconst, Xsf, invc,
        Ubar, Xf, Acor, rconst;
    std::vector<double> hR;      // radii, semi-major axes of ellipses (validation)
    std::vector<double> hB;      // semi-minor axes (== hR for disks and spheres)
    std::vector<double> hratio;  // density ratios (per-particle constants)
    std::vector<int> hbox;       // per particle: first entry of its velocity box, H (pairs)
    long long box_entries = 0;   // entries of all velocity boxes
};

// Adjoint recording of one instance: checkpoints of the forward pass and the
// per-step records of the segment being recomputed.
struct AdjInst {
    std::vector<DevBuf> ckpt;   // [nseg] populations at the start of each segment
    DevBuf ckst;                // [nseg + 1][np][16] particle state at segment starts, then the final one
    std::vector<DevBuf> slot;   // [L + 1] populations entering each step of the segment
    DevBuf rprec, rlcnt, rlent, rlrec, rgeo, rstate;  // [L + 1] records of each step
    DevBuf fbar[2];             // adjoint of the pre-collision populations (ping-pong)
    DevBuf pbuf;                // adjoint particle arrays (AdjBufs)
};
struct AdjCtx {
    bool ready = false;         // a recorded forward pass matches the current state
    int nsteps = 0, L = 0, nseg = 0;
    std::vector<AdjInst> ai;
    DevBuf d_rdesc, d_rtmaps, d_afl, d_apt, d_abufs, d_out, d_out_off;
    cudaGraphExec_t seg_exec = nullptr;  // recompute + backward of one full segment
};

}  // namespace

struct lbm_ctx {
    int Q = 9, D = 2, fp16 = 0;
    cudaStream_t st = nullptr;
    lbm_allocator alloc{};
    bool has_alloc = false;
    std::vector<Instance> inst;
    DevBuf d_insts, d_tile_inst, d_tile_ctr, d_status, d_refs, d_tmaps, d_gridbar;
    int ntiles = 0, np_total = 0;
    int par = 0;
    long long steps = 0;
    Shape shape{4, 4, 1, 4, 0, 0, 3, 128};
    int grid = 0, num_sms = 0;
    int graph_steps = 16;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;  // capture stream (capture is not allowed on the legacy stream)
    bool graph_ok[2] = {false, false};
    bool failed = false;
    std::string err;
    AdjCtx adj;
    long long wait_ns = -1;  // bound of the particle kernel's barrier waits; < 0: the default 2 s
};

namespace {

int set_err(lbm_ctx* c, int code, const char* fmt, const char* detail = "") {
    if (c) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, detail);
        c->err = buf;
    }
    return code;
}

int cuda_err(lbm_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBM_OK;
    if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);     \
    } while (0)

int dalloc(lbm_ctx* ctx, DevBuf& b, size_t bytes) {
    if (b.ptr && b.bytes >= bytes) return LBM_OK;
    if (b.ptr) {
        if (ctx->has_alloc) ctx->alloc.free(b.ptr, b.bytes, ctx->st, ctx->alloc.user);
        else cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (ctx->has_alloc) p = ctx->alloc.alloc(bytes, ctx->st, ctx->alloc.user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) return set_err(ctx, LBM_ERR_OOM, "device allocation of %s bytes failed",
                           std::to_string(bytes).c_str());
    b.ptr = p;
    b.bytes = bytes;
    return LBM_OK;
}

void dfree(lbm_ctx* ctx, DevBuf& b) {
    if (!b.ptr) return;
    if (ctx->has_alloc) ctx->alloc.free(b.ptr, b.bytes, ctx->st, ctx->alloc.user);
    else cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

template <class T> T* P(const DevBuf& b) { return static_cast<T*>(b.ptr); }

int validate(const lbm_config* c, char* why, size_t nwhy) {
    auto bad = [&](const char* m) {
        snprintf(why, nwhy, "%s", m);
        return 0;
    };
    if (c->lattice != LBM_D2Q9 && c->lattice != LBM_D3Q19) return bad("lattice must be 9 or 19");
    if (c->storage != LBM_FP32 && c->storage != LBM_FP16) return bad("storage must be FP32 or FP16");
    const int D = c->lattice == LBM_D2Q9 ? 2 : 3;
    for (int d = 0; d < D; ++d)
        if (c->n[d] < 2 || c->n[d] > (1 << 20)) return bad("each axis needs 2 .. 2^20 nodes");
    if (D == 2 && c->n[2] != 1) return bad("D2Q9 needs n[2] = 1");
    if (!(c->tau > 0.5) || !(c->tau < 100.0)) return bad("tau must lie in (0.5, 100)");
    if (!(c->alpha >= 0.0) || c->alpha * c->tau > 1.0 + 1e-12)
        return bad("alpha must lie in [0, 1/tau]");
    if (!(c->rho_f > 0)) return bad("rho_f must be positive");
    if (!(c->delta > 0) || !(c->eps_p > 0) || !(c->eps_w > 0))
        return bad("delta, eps_p and eps_w must be positive");
    if (c->K < 1 || c->K > 64) return bad("K must lie in 1 .. 64");
    if (c->max_particles < 0 || c->max_particles > (1 << 20)) return bad("max_particles out of range");
    if ((double)c->n[0] * c->n[1] * c->n[2] * 19 > 2.0e9)
        return bad("at most 2e9 stored populations per instance");
    if (!(c->max_radius >= 2.0) || c->max_radius > (D == 3 ? MAX_RADIUS_3D : MAX_RADIUS))
        return bad(D == 3 ? "max_radius must lie in [2, 40] for D3Q19" : "max_radius must lie in [2, 120]");
    if (c->fp16_scale_log2 < 0 || c->fp16_scale_log2 > 24) return bad("fp16_scale_log2 in 0 .. 24");
    for (int d = 0; d < 3; ++d) {
        if (c->bc[d] != LBM_PERIODIC && c->bc[d] != LBM_WALL) return bad("bc must be PERIODIC or WALL");
        for (int f = 0; f < 2; ++f) {
            const double* u = c->wall_u[d][f];
            bool moving = u[0] != 0 || u[1] != 0 || u[2] != 0;
            if (!moving) continue;
            if (d >= D || c->bc[d] != LBM_WALL) return bad("wall velocity on a non-wall face");
            if (u[d] != 0) return bad("wall velocity must be tangential");
            for (int e = 0; e < D; ++e)
                if (e != d && c->bc[e] != LBM_PERIODIC)
                    return bad("a moving wall needs every other axis periodic");
        }
    }
    return 1;
}

int max_slots(const Instance& I, int D, const Shape& sh) {
    const int T[3] = {sh.tw, sh.ty, sh.tz};
    int k = 1;
    for (int d = 0; d < D; ++d) {
        const int span = (int)ceil(2 * I.cfg.max_radius) + 4;
        k *= std::min(span / T[d] + 3, I.ntile[d]);  // a wrapped interval splits in two
    }
    return std::max(k, 1);
}

InstDesc make_desc(lbm_ctx* ctx, const Instance& I) {
    InstDesc d{};
    const lbm_config& c = I.cfg;
    for (int a = 0; a < 3; ++a) {
        d.n[a] = I.n[a];
        d.periodic[a] = (a >= ctx->D) ? 1 : (c.bc[a] == LBM_PERIODIC);
        d.ntile[a] = I.ntile[a];
        d.gdrive[a] = (float)c.g_drive[a];
        d.ggrav[a] = (float)c.g_grav[a];
    }
    d.pitch = I.pitch;
    d.qstride = I.qstride;
    d.tile0 = I.tile0;
    d.np = I.np;
    d.maxk = I.maxk;
    d.tau_inv = (float)(1.0 / c.tau);
    d.keep = (float)(1.0 - 1.0 / c.tau);
    d.fpref = (float)(1.0 - 1.0 / (2.0 * c.tau));
    d.alpha = (float)c.alpha;
    if (ctx->fp16) {
        d.s_store = ldexpf(1.0f, c.fp16_scale_log2);
        d.s_load = ldexpf(1.0f, -c.fp16_scale_log2);
    } else {
        d.s_store = d.s_load = 1.0f;
    }
    // bounce-back term 2 w_q (c_q . u_w) / cs^2 for every wall face
    for (int a = 0; a < 3; ++a)
        for (int f = 0; f < 2; ++f)
            for (int q = 0; q < 19; ++q) {
                double cu = 0, w = 0;
                if (q < ctx->Q) {
                    for (int e = 0; e < 3; ++e) {
                        const int cq = ctx->Q == 9 ? d2q9_c(q, e) : d3q19_c(q, e);
                        cu += cq * c.wall_u[a][f][e];
                    }
                    w = ctx->Q == 9 ? d2q9_w(q) : d3q19_w(q);
                }
                d.wterm[a][f][q] = (float)(2.0 * w * cu * 3.0);
            }
    d.f[0] = I.f[0].ptr;
    d.f[1] = I.f[1].ptr;
    d.prec = P<PRec>(I.prec);
    d.prec_out = d.prec;
    d.list_cnt[0] = P<int>(I.lcnt[0]);
    d.list_cnt[1] = P<int>(I.lcnt[1]);
    d.list_ent[0] = P<uint32_t>(I.lent[0]);
    d.list_ent[1] = P<uint32_t>(I.lent[1]);
    d.list_rec[0] = I.lrec[0].ptr;
    d.list_rec[1] = I.lrec[1].ptr;
    d.ubox = P<float>(I.ubox);
    d.ubox_scratch = P<float>(I.ubox_scratch);
    d.boxinfo = P<int2>(I.boxinfo);
    d.btot = P<long long>(I.btot);
    d.X = P<double>(I.X);
    d.U = P<double>(I.U);
    d.W = P<double>(I.W);
    d.Un = P<double>(I.Un);
    d.Wn = P<double>(I.Wn);
    d.theta = P<double>(I.theta);
    d.A = P<double>(I.A);
    d.R = P<double>(I.R);
    d.ratio = P<double>(I.ratio);
    d.count = P<int>(I.count);
    d.Xk = P<double>(I.Xk);
    d.Ubar = P<double>(I.Ubar);
    d.Acor = P<double>(I.Acor);
    d.Xf = P<float>(I.Xf);
    d.pconst = P<double>(I.pconst);
    d.rconst = P<RecConst>(I.rconst);
    d.Xsf = P<float>(I.Xsf);
    d.invc = P<double>(I.invc);
    d.rho_f = c.rho_f;
    d.gmag = sqrt(c.g_grav[0] * c.g_grav[0] + c.g_grav[1] * c.g_grav[1] + c.g_grav[2] * c.g_grav[2]);
    d.delta = c.delta;
    d.eps_p = c.eps_p;
    d.eps_w = c.eps_w;
    d.inv_eps_p = 1.0 / c.eps_p;
    d.inv_eps_w = 1.0 / c.eps_w;
    d.K = c.K;
    d.hK = 1.0 / c.K;
    d.status = P<int>(ctx->d_status);
    d.adj_geo = nullptr;
    d.rec_state = nullptr;
    return d;
}

void invalidate_graphs(lbm_ctx* ctx) {
    for (int i = 0; i < 2; ++i) {
        if (ctx->exec[i]) cudaGraphExecDestroy(ctx->exec[i]);
        ctx->exec[i] = nullptr;
        ctx->graph_ok[i] = false;
    }
}

int upload_descs(lbm_ctx* ctx) {
    std::vector<InstDesc> h;
    for (auto& I : ctx->inst) h.push_back(make_desc(ctx, I));
    int rc = dalloc(ctx, ctx->d_insts, sizeof(InstDesc) * h.size());
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->d_insts.ptr, h.data(), sizeof(InstDesc) * h.size(),
                       cudaMemcpyHostToDevice, ctx->st));
    // particle reference table for the per-particle kernels, padded per
    // instance to whole blocks of 8 so that no block straddles two instances
    std::vector<PartRef> refs;
    for (int i = 0; i < (int)ctx->inst.size(); ++i) {
        for (int p = 0; p < ctx->inst[i].np; ++p) refs.push_back({i, p});
        while (refs.size() % 8) refs.push_back({-1, 0});
    }
    ctx->np_total = (int)refs.size();
    rc = dalloc(ctx, ctx->d_refs, sizeof(PartRef) * std::max<size_t>(refs.size(), 1));
    if (rc) return rc;
    if (!refs.empty())
        CK(cudaMemcpyAsync(ctx->d_refs.ptr, refs.data(), sizeof(PartRef) * refs.size(),
                           cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));  // host vectors go out of scope
    return LBM_OK;
}

// Per-particle constants of the update: 1 - rho_f/rho_s (buoyancy-reduced
// gravity), C/eps_p and C/eps_w with C = (rho_s - rho_f)|g| (Eqs. 19-20),
// 1/delta, 1/rho_s (the mass is rho_s times the node count), R and the
// semi-minor axis B (B == R: disk or sphere).
int upload_pconst(lbm_ctx* ctx, Instance& I) {
    if (I.np == 0) return LBM_OK;
    const lbm_config& c = I.cfg;
    const double g = sqrt(c.g_grav[0] * c.g_grav[0] + c.g_grav[1] * c.g_grav[1] + c.g_grav[2] * c.g_grav[2]);
    std::vector<double> pc(PCONST_N * (size_t)I.np, 0.0);
    for (int p = 0; p < I.np; ++p) {
        const double C = (I.hratio[p] - 1.0) * c.rho_f * g;
        double* q = pc.data() + PCONST_N * p;
        q[PC_GFAC] = 1.0 - 1.0 / I.hratio[p];
        q[PC_CPAIR] = C / c.eps_p;
        q[PC_CWALL] = C / c.eps_w;
        q[PC_INVDELTA] = 1.0 / c.delta;
        q[PC_INVRHOS] = 1.0 / (I.hratio[p] * c.rho_f);
        q[PC_R] = I.hR[p];
        q[PC_B] = I.hB[p];
    }
    CK(cudaMemcpy(I.pconst.ptr, pc.data(), sizeof(double) * pc.size(), cudaMemcpyHostToDevice));
    // record fields that depend only on the size and shape: R^2 and B^2 as the
    // exact test of Eq. 9 takes them, and the float bands of its filter.  The
    // ellipse band: the float form (r.e / a)^2 + (r.e_perp / b)^2 carries a
    // relative error below ~1e-6 (1 + a/b) within the circumscribed circle,
    // and the band is ten times that.
    std::vector<RecConst> rc((size_t)I.np);
    for (int p = 0; p < I.np; ++p) {
        const double R = I.hR[p], B = I.hB[p];
        RecConst& r = rc[p];
        r.R2 = R * R;
        r.b2 = B * B;
        const float Rf = (float)R, R2f = Rf * Rf;
        r.R2lo = R2f * (1.0f - 2e-5f) - 2e-4f;
        r.R2hi = R2f * (1.0f + 2e-5f) + 2e-4f;
        r.ia2 = (float)(1.0 / (R * R));
        r.ib2 = (float)(1.0 / (B * B));
        const float beta = 1e-5f * (1.0f + (float)(R / B));
        r.qlo = 1.0f - beta;
        r.qhi = 1.0f + beta;
        r.shape = B != R;
        r.pad = 0;
    }
    CK(cudaMemcpy(I.rconst.ptr, rc.data(), sizeof(RecConst) * rc.size(), cudaMemcpyHostToDevice));
    return LBM_OK;
}

// Re-publish every particle into the tile lists of the current parity.
int republish(lbm_ctx* ctx) {
    for (auto& I : ctx->inst) {
        if (I.np == 0) continue;
        CK(cudaMemsetAsync(I.lcnt[ctx->par].ptr, 0, sizeof(int) * I.ntiles, ctx->st));
        if (I.ubox.ptr) CK(cudaMemsetAsync(I.ubox.ptr, 0xff, I.ubox.bytes, ctx->st));  // every entry empty (NaN)
    }
    if (ctx->np_total > 0)
        CK(launch_publish(P<InstDesc>(ctx->d_insts), P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D,
                          ctx->par, ctx->shape, ctx->st));
    return LBM_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of one population buffer: the stored populations as a
// [Q-1][nz][ny][pitch] tensor (x innermost, dim = nx so that boxes read
// zeros beyond the last node).  D2Q9 boxes hold every population of a tile
// with one halo row on each side, (tile width + 2 halo) x (ty + 2) x (Q - 1),
// so a tile takes one copy; D3Q19 boxes hold one population's source rows,
// (tile width + 2 halo) x ty x tz.
int encode_pop_map(lbm_ctx* ctx, const Instance& I, void* ptr, CUtensorMap* out) {
    auto enc = tmap_encoder();
    if (!enc) return set_err(ctx, LBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available%s");
    const size_t ss = ctx->fp16 ? 2 : 4;
    const int halo = 16 / (int)ss;
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], es[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    dims[0] = (cuuint64_t)I.n[0];
    dims[1] = (cuuint64_t)I.n[1];
    strides[0] = (cuuint64_t)I.pitch * ss;
    box[0] = (cuuint32_t)(ctx->shape.tw + 2 * halo);
    box[1] = (cuuint32_t)ctx->shape.ty;
    if (ctx->D == 2) {  // one box per tile: every population, rows y0 - 1 .. y0 + ty
        rank = 3;
        dims[2] = (cuuint64_t)(ctx->Q - 1);
        strides[1] = (cuuint64_t)I.pitch * I.n[1] * ss;
        box[1] = (cuuint32_t)(ctx->shape.ty + 2);
        box[2] = (cuuint32_t)(ctx->Q - 1);
    } else {
        rank = 4;
        dims[2] = (cuuint64_t)I.n[2];
        dims[3] = (cuuint64_t)(ctx->Q - 1);
        strides[1] = (cuuint64_t)I.pitch * I.n[1] * ss;
        strides[2] = (cuuint64_t)I.pitch * I.n[1] * I.n[2] * ss;
        box[2] = (cuuint32_t)ctx->shape.tz;
        box[3] = 1;
    }
    CUresult r = enc(out, ctx->fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank,
                     ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(ctx, LBM_ERR_CUDA, "tensor map encoding failed%s");
    return LBM_OK;
}

// One tensor map per instance and population buffer.
int build_tmaps(lbm_ctx* ctx) {
    std::vector<CUtensorMap> maps(2 * ctx->inst.size());
    for (size_t i = 0; i < ctx->inst.size(); ++i)
        for (int b = 0; b < 2; ++b) {
            int rc = encode_pop_map(ctx, ctx->inst[i], ctx->inst[i].f[b].ptr, &maps[2 * i + b]);
            if (rc) return rc;
        }
    int rc = dalloc(ctx, ctx->d_tmaps, sizeof(CUtensorMap) * maps.size());
    if (rc) return rc;
    CK(cudaMemcpy(ctx->d_tmaps.ptr, maps.data(), sizeof(CUtensorMap) * maps.size(),
                  cudaMemcpyHostToDevice));
    return LBM_OK;
}

// Tile grid, tile -> instance table and tile lists for a shape.
int configure_shape(lbm_ctx* ctx, const Shape& sh_in) {
    Shape sh = sh_in;
    if (ctx->D == 2) sh.tz = 1;
    sh.tw = sh.tma ? tma_tile_width(ctx->Q) : 32 * sh.vec;
    ctx->shape = sh;
    const int T[3] = {sh.tw, sh.ty, sh.tz};
    int tile0 = 0;
    std::vector<uint16_t> tab;
    for (int i = 0; i < (int)ctx->inst.size(); ++i) {
        Instance& I = ctx->inst[i];
        I.ntiles = 1;
        for (int d = 0; d < 3; ++d) {
            I.ntile[d] = (I.n[d] + T[d] - 1) / T[d];
            I.ntiles *= I.ntile[d];
        }
        I.tile0 = tile0;
        tile0 += I.ntiles;
        tab.insert(tab.end(), (size_t)I.ntiles, (uint16_t)i);
        I.maxk = max_slots(I, ctx->D, ctx->shape);
        int rc;
        for (int b = 0; b < 2; ++b) {
            if ((rc = dalloc(ctx, I.lcnt[b], sizeof(int) * I.ntiles))) return rc;
            if ((rc = dalloc(ctx, I.lent[b], sizeof(uint32_t) * (size_t)I.ntiles * LIST_CAP))) return rc;
            if ((rc = dalloc(ctx, I.lrec[b], (size_t)CAND_BYTES * I.ntiles * LIST_CAP))) return rc;
            CK(cudaMemsetAsync(I.lcnt[b].ptr, 0, sizeof(int) * I.ntiles, ctx->st));
        }
    }
    ctx->ntiles = tile0;
    int rc = dalloc(ctx, ctx->d_tile_inst, sizeof(uint16_t) * tab.size());
    if (rc) return rc;
    CK(cudaMemcpyAsync(ctx->d_tile_inst.ptr, tab.data(), sizeof(uint16_t) * tab.size(),
                       cudaMemcpyHostToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int occ = sh.tma ? fluid_tma_blocks_per_sm(ctx->Q, ctx->fp16, sh, sh.stages, (int)ctx->inst.size())
                           : fluid_max_blocks_per_sm(ctx->Q, ctx->fp16, sh);
    if (occ < 1) return set_err(ctx, LBM_ERR_INVALID, "kernel shape does not fit on an SM%s");
    ctx->grid = occ * ctx->num_sms;
    if (sh.tma && (rc = build_tmaps(ctx))) return rc;
    if ((rc = upload_descs(ctx))) return rc;
    invalidate_graphs(ctx);
    return republish(ctx);
}

Shape default_shape(int Q, int fp16) {
    // TMA-staged pipeline, 2 stages: D2Q9 FP32 8 rows and 8 consumer warps
    // (one box of all populations per tile, two blocks per SM); D2Q9 FP16 4
    // rows and 4 warps (four blocks per SM: 16 consumer warps, as for FP32,
    // with tiles half as tall); D3Q19 4 warps (four blocks per SM fit in
    // shared memory, against three with 3 stages)
    if (Q == 9) return fp16 ? Shape{8, 4, 1, 4, 1, 1, 2, 128} : Shape{4, 8, 1, 8, 1, 1, 2, 128};
    return Shape{fp16 ? 4 : 2, 2, 2, 4, 1, 1, 2, 64};
}

int enqueue_fluid(lbm_ctx* ctx, int commit, cudaStream_t st) {
    const Shape& sh = ctx->shape;
    if (sh.tma) {
        CK(launch_fluid_tma(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), ctx->d_tmaps.ptr,
                            P<uint16_t>(ctx->d_tile_inst), ctx->ntiles, ctx->par, sh, commit,
                            ctx->grid, P<int>(ctx->d_tile_ctr), sh.stages, (int)ctx->inst.size(), st));
        return LBM_OK;
    }
    CK(launch_fluid(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), P<uint16_t>(ctx->d_tile_inst),
                    ctx->ntiles, ctx->par, sh, commit, sh.persistent, ctx->grid,
                    P<int>(ctx->d_tile_ctr), st));
    return LBM_OK;
}
int enqueue_fluid(lbm_ctx* ctx, int commit) { return enqueue_fluid(ctx, commit, ctx->st); }

// One full time step on stream st (no synchronisation).
int enqueue_step(lbm_ctx* ctx, cudaStream_t st) {
    int rc = enqueue_fluid(ctx, 1, st);
    if (rc) return rc;
    if (ctx->np_total > 0) {
        const int K = ctx->inst[0].cfg.K;
        CK(launch_box_sums(P<InstDesc>(ctx->d_insts), P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D, st));
        const bool fused = (ctx->np_total + 7) / 8 <= particle_blocks_resident(ctx->num_sms);
        CK(launch_particles(P<InstDesc>(ctx->d_insts), P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D,
                            K, ctx->par ^ 1, ctx->shape, P<GridBar>(ctx->d_gridbar), fused, st,
                            ctx->wait_ns));
    }
    ctx->par ^= 1;
    ctx->steps += 1;
    return LBM_OK;
}

int check_ctx(lbm_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID;
    if (ctx->failed) return LBM_ERR_STATE;
    return LBM_OK;
}

int check_inst(lbm_ctx* ctx, int i) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (i < 0 || i >= (int)ctx->inst.size()) return set_err(ctx, LBM_ERR_INVALID, "bad instance index%s");
    return LBM_OK;
}

int read_status(lbm_ctx* ctx) {
    int st = 0;
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(&st, ctx->d_status.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == 0) return LBM_OK;
    ctx->failed = true;
    // a wait that gave up leaves the step half done, so later errors are its consequences
    if (st & ST_TIMEOUT) return set_err(ctx, LBM_ERR_TIMEOUT, "a bounded device wait gave up%s");
    if (st & ST_DIVERGED) return set_err(ctx, LBM_ERR_DIVERGED, "the flow diverged (|u| >= 0.5 or non-finite)%s");
    if (st & ST_PARTICLE) return set_err(ctx, LBM_ERR_PARTICLE, "a particle centre crossed a wall%s");
    if (st & ST_DISPLACEMENT) return set_err(ctx, LBM_ERR_DIVERGED, "a particle moved faster than 0.5 per step%s");
    return set_err(ctx, LBM_ERR_CAPACITY, "a tile overlaps more particles than its list holds%s");
}

void adj_drop_graph(AdjCtx& A) {
    if (A.seg_exec) cudaGraphExecDestroy(A.seg_exec);
    A.seg_exec = nullptr;
}

void adj_release(lbm_ctx* ctx) {
    AdjCtx& A = ctx->adj;
    adj_drop_graph(A);
    for (auto& a : A.ai) {
        for (auto& b : a.ckpt) dfree(ctx, b);
        for (auto& b : a.slot) dfree(ctx, b);
        DevBuf* bufs[] = {&a.ckst, &a.rprec, &a.rlcnt, &a.rlent, &a.rlrec, &a.rgeo, &a.rstate, &a.fbar[0],
                          &a.fbar[1], &a.pbuf};
        for (DevBuf* b : bufs) dfree(ctx, *b);
    }
    A.ai.clear();
    DevBuf* bufs[] = {&A.d_rdesc, &A.d_rtmaps, &A.d_afl, &A.d_apt, &A.d_abufs, &A.d_out, &A.d_out_off};
    for (DevBuf* b : bufs) dfree(ctx, *b);
    A.ready = false;
}

void destroy_all(lbm_ctx* ctx) {
    adj_release(ctx);
    invalidate_graphs(ctx);
    for (auto& I : ctx->inst) {
        DevBuf* bufs[] = {&I.f[0], &I.f[1], &I.prec, &I.lcnt[0], &I.lcnt[1], &I.lent[0], &I.lent[1],
                          &I.lrec[0], &I.lrec[1],
                          &I.ubox, &I.ubox_scratch, &I.boxinfo, &I.btot, &I.X, &I.U, &I.W, &I.Un, &I.Wn, &I.theta, &I.A, &I.R,
                          &I.ratio, &I.count, &I.Xk, &I.Ubar, &I.Xf, &I.pconst, &I.Xsf, &I.invc, &I.Acor, &I.rconst};
        for (DevBuf* b : bufs) dfree(ctx, *b);
    }
    dfree(ctx, ctx->d_insts);
    dfree(ctx, ctx->d_tile_inst);
    dfree(ctx, ctx->d_tile_ctr);
    dfree(ctx, ctx->d_status);
    dfree(ctx, ctx->d_refs);
    dfree(ctx, ctx->d_tmaps);
    dfree(ctx, ctx->d_gridbar);
}

int alloc_particles(lbm_ctx* ctx, Instance& I, int cap) {
    DevBuf* v3[] = {&I.X, &I.U, &I.W, &I.Un, &I.Wn, &I.theta, &I.A, &I.Ubar, &I.Acor};
    int rc;
    const size_t c = (size_t)std::max(cap, 1);
    for (DevBuf* b : v3)
        if ((rc = dalloc(ctx, *b, sizeof(double) * 3 * c))) return rc;
    if ((rc = dalloc(ctx, I.R, sizeof(double) * c))) return rc;
    if ((rc = dalloc(ctx, I.ratio, sizeof(double) * c))) return rc;
    if ((rc = dalloc(ctx, I.count, sizeof(int) * c))) return rc;
    if ((rc = dalloc(ctx, I.prec, sizeof(PRec) * c))) return rc;
    if ((rc = dalloc(ctx, I.Xk, sizeof(double) * 6 * c))) return rc;
    if ((rc = dalloc(ctx, I.Xf, sizeof(float) * 8 * c))) return rc;
    if ((rc = dalloc(ctx, I.pconst, sizeof(double) * PCONST_N * c))) return rc;
    if ((rc = dalloc(ctx, I.rconst, sizeof(RecConst) * c))) return rc;
    if ((rc = dalloc(ctx, I.invc, sizeof(double) * c))) return rc;
    if ((rc = dalloc(ctx, I.Xsf, sizeof(float) * 8 * c))) return rc;
    if ((rc = dalloc(ctx, I.boxinfo, sizeof(int2) * c))) return rc;
    if ((rc = dalloc(ctx, I.btot, sizeof(long long) * NPV * c))) return rc;
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_status_string(int s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA error";
        case LBM_ERR_OOM: return "out of device memory";
        case LBM_ERR_DIVERGED: return "diverged";
        case LBM_ERR_TIMEOUT: return "device wait timed out";
        case LBM_ERR_STATE: return "context unusable";
        case LBM_ERR_CAPACITY: return "tile list capacity exceeded";
        case LBM_ERR_PARTICLE: return "particle left the box";
        default: return "unknown status";
    }
}

int lbm_config_default(lbm_config* cfg, int lattice, int nx, int ny, int nz) {
    if (!cfg) return LBM_ERR_INVALID;
    memset(cfg, 0, sizeof *cfg);
    cfg->lattice = lattice;
    cfg->storage = LBM_FP32;
    cfg->n[0] = nx;
    cfg->n[1] = ny;
    cfg->n[2] = lattice == LBM_D2Q9 ? 1 : nz;
    for (int d = 0; d < 3; ++d) cfg->bc[d] = LBM_WALL;
    if (lattice == LBM_D2Q9) cfg->bc[2] = LBM_PERIODIC;
    cfg->tau = 1.0;
    cfg->alpha = 1.0;
    cfg->rho_f = 1.0;
    cfg->delta = 1.0;
    cfg->eps_p = 2.0;
    cfg->eps_w = 1.0;
    cfg->K = 1;
    cfg->max_particles = 64;
    cfg->max_radius = 16.0;
    cfg->fp16_scale_log2 = 14;
    return (lattice == LBM_D2Q9 || lattice == LBM_D3Q19) ? LBM_OK : LBM_ERR_INVALID;
}

int lbm_create_batch(const lbm_config* cfgs, int n, const lbm_allocator* alloc, void* stream,
                     lbm_ctx** out) {
    if (!cfgs || n < 1 || n > 65535 || !out) return LBM_ERR_INVALID;
    *out = nullptr;
    char why[256];
    for (int i = 0; i < n; ++i) {
        if (!validate(&cfgs[i], why, sizeof why)) return LBM_ERR_INVALID;
        if (cfgs[i].lattice != cfgs[0].lattice || cfgs[i].storage != cfgs[0].storage ||
            cfgs[i].K != cfgs[0].K)
            return LBM_ERR_INVALID;
    }
    lbm_ctx* ctx = new lbm_ctx();
    ctx->Q = cfgs[0].lattice;
    ctx->D = ctx->Q == 9 ? 2 : 3;
    ctx->fp16 = cfgs[0].storage == LBM_FP16;
    ctx->st = static_cast<cudaStream_t>(stream);
    if (alloc && alloc->alloc && alloc->free) {
        ctx->alloc = *alloc;
        ctx->has_alloc = true;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete ctx;
        return LBM_ERR_CUDA;
    }
    ctx->inst.resize(n);
    ctx->shape = default_shape(ctx->Q, ctx->fp16);
    const size_t ssz = ctx->fp16 ? 2 : 4;
    int rc = LBM_OK;
    for (int i = 0; i < n && rc == LBM_OK; ++i) {
        Instance& I = ctx->inst[i];
        I.cfg = cfgs[i];
        for (int d = 0; d < 3; ++d) I.n[d] = cfgs[i].n[d];
        if (ctx->D == 2) I.n[2] = 1;
        I.pitch = (I.n[0] + 31) & ~31;
        I.qstride = (long long)I.pitch * I.n[1] * I.n[2];
        I.cap = cfgs[i].max_particles;
        const size_t fb = ssz * (size_t)(ctx->Q - 1) * (size_t)I.qstride;
        for (int b = 0; b < 2 && rc == LBM_OK; ++b) {
            rc = dalloc(ctx, I.f[b], fb);
            if (rc == LBM_OK && cudaMemsetAsync(I.f[b].ptr, 0, fb, ctx->st) != cudaSuccess)
                rc = LBM_ERR_CUDA;
        }
        if (rc == LBM_OK) rc = alloc_particles(ctx, I, I.cap);
    }
    if (rc == LBM_OK) rc = dalloc(ctx, ctx->d_tile_ctr, sizeof(int) * 2);
    if (rc == LBM_OK) rc = dalloc(ctx, ctx->d_status, sizeof(int) * 4);
    if (rc == LBM_OK) rc = dalloc(ctx, ctx->d_gridbar, sizeof(GridBar));
    if (rc == LBM_OK) cudaMemsetAsync(ctx->d_gridbar.ptr, 0, sizeof(GridBar), ctx->st);
    if (rc == LBM_OK) {
        cudaMemsetAsync(ctx->d_tile_ctr.ptr, 0, sizeof(int) * 2, ctx->st);
        cudaMemsetAsync(ctx->d_status.ptr, 0, sizeof(int) * 4, ctx->st);
        rc = configure_shape(ctx, ctx->shape);
    }
    if (rc == LBM_OK && cudaStreamSynchronize(ctx->st) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (rc != LBM_OK) {
        destroy_all(ctx);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return LBM_OK;
}

int lbm_create(const lbm_config* cfg, const lbm_allocator* alloc, void* stream, lbm_ctx** out) {
    return lbm_create_batch(cfg, 1, alloc, stream, out);
}

int lbm_num_instances(const lbm_ctx* ctx) { return ctx ? (int)ctx->inst.size() : 0; }

int lbm_num_particles(const lbm_ctx* ctx, int i) {
    if (!ctx || i < 0 || i >= (int)ctx->inst.size()) return -1;
    return ctx->inst[i].np;
}

// Velocity boxes of all particles of an instance (side 2H + 1, H = ceil(R) + 2,
// one after another), allocated to fit and marked empty (NaN).
static int layout_boxes(lbm_ctx* ctx, Instance& I) {
    const int D = ctx->D;
    I.hbox.clear();
    I.box_entries = 0;
    for (int k = 0; k < I.np; ++k) {
        const int H = (int)ceil(I.hR[k]) + 2, side = 2 * H + 1;
        I.hbox.push_back((int)I.box_entries);
        I.hbox.push_back(H);
        I.box_entries += D == 2 ? (long long)side * side : (long long)side * side * side;
    }
    if (I.box_entries >= (1LL << 31)) return set_err(ctx, LBM_ERR_INVALID, "velocity boxes exceed 2^31 entries%s");
    if (I.np == 0) return LBM_OK;
    const size_t eb = (size_t)I.box_entries * (D == 2 ? 8 : 16);
    int rc;
    if ((rc = dalloc(ctx, I.ubox, eb)) || (rc = dalloc(ctx, I.ubox_scratch, eb))) return rc;
    CK(cudaMemsetAsync(I.ubox.ptr, 0xff, I.ubox.bytes, ctx->st));  // every entry empty (NaN)
    CK(cudaMemcpyAsync(I.boxinfo.ptr, I.hbox.data(), sizeof(int) * I.hbox.size(), cudaMemcpyHostToDevice,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return LBM_OK;
}

// Disks and spheres (minor == NULL) or ellipses (2D; minor = semi-minor axes,
// theta = orientations or NULL).
static int add_particles_impl(lbm_ctx* ctx, int i, int n, const double* pos, const double* radius,
                              const double* minor, const double* theta, const double* ratio,
                              const double* vel, const double* omega) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    ctx->adj.ready = false;
    if (n < 0 || (n > 0 && (!pos || !radius || !ratio)))
        return set_err(ctx, LBM_ERR_INVALID, "bad particle arrays%s");
    if (n == 0) return LBM_OK;
    Instance& I = ctx->inst[i];
    const int D = ctx->D;
    if (minor && D != 2) return set_err(ctx, LBM_ERR_INVALID, "ellipses need the D2Q9 lattice%s");
    if (I.np + n > I.cap) return set_err(ctx, LBM_ERR_INVALID, "max_particles exceeded%s");
    for (int k = 0; k < n; ++k) {
        if (!(radius[k] >= 2.0) || radius[k] > I.cfg.max_radius)
            return set_err(ctx, LBM_ERR_INVALID, "radius must lie in [2, max_radius]%s");
        if (minor && !(minor[k] >= 1.0 && minor[k] <= radius[k]))
            return set_err(ctx, LBM_ERR_INVALID, "semi-minor axis must lie in [1, a]%s");
        if (theta && !(theta[k] == theta[k] && fabs(theta[k]) < 1e6))
            return set_err(ctx, LBM_ERR_INVALID, "orientation must be finite%s");
        if (!(ratio[k] > 0.0)) return set_err(ctx, LBM_ERR_INVALID, "density ratio must be positive%s");
        for (int d = 0; d < D; ++d) {
            const double x = pos[k * D + d];
            if (!(x == x)) return set_err(ctx, LBM_ERR_INVALID, "non-finite position%s");
            if (I.cfg.bc[d] == LBM_WALL && (x < 0.0 || x > I.n[d] - 1))
                return set_err(ctx, LBM_ERR_INVALID, "particle centre outside the box%s");
            if (I.cfg.bc[d] == LBM_PERIODIC && (x < 0.0 || x >= I.n[d] ||
                                                 radius[k] >= 0.25 * I.n[d]))
                return set_err(ctx, LBM_ERR_INVALID,
                               "periodic axis: need 0 <= x < n and radius < n/4%s");
        }
    }
    // host staging, FP64 [n][3]
    std::vector<double> X(3 * n, 0.0), U(3 * n, 0.0), W(3 * n, 0.0), Z(3 * n, 0.0), T(3 * n, 0.0);
    if (theta)
        for (int k = 0; k < n; ++k) T[3 * k + 2] = theta[k];
    for (int k = 0; k < n; ++k)
        for (int d = 0; d < D; ++d) {
            X[3 * k + d] = pos[k * D + d];
            if (vel) U[3 * k + d] = vel[k * D + d];
        }
    if (omega) {
        for (int k = 0; k < n; ++k) {
            if (D == 2) W[3 * k + 2] = omega[k];
            else
                for (int d = 0; d < 3; ++d) W[3 * k + d] = omega[3 * k + d];
        }
    }
    const size_t o3 = sizeof(double) * 3 * I.np, b3 = sizeof(double) * 3 * n;
    auto up = [&](DevBuf& b, const std::vector<double>& v) {
        return cudaMemcpyAsync(static_cast<char*>(b.ptr) + o3, v.data(), b3, cudaMemcpyHostToDevice,
                               ctx->st);
    };
    CK(up(I.X, X));
    CK(up(I.U, U));
    CK(up(I.W, W));
    CK(up(I.Un, U));
    CK(up(I.Wn, W));
    CK(up(I.theta, T));
    CK(up(I.A, Z));
    CK(cudaMemcpyAsync(P<double>(I.R) + I.np, radius, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(P<double>(I.ratio) + I.np, ratio, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemsetAsync(P<int>(I.count) + I.np, 0, sizeof(int) * n, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    I.np += n;
    I.hR.insert(I.hR.end(), radius, radius + n);
    if (minor) I.hB.insert(I.hB.end(), minor, minor + n);
    else I.hB.insert(I.hB.end(), radius, radius + n);
    I.hratio.insert(I.hratio.end(), ratio, ratio + n);
    if ((rc = layout_boxes(ctx, I))) return rc;
    if ((rc = upload_pconst(ctx, I))) return rc;
    if ((rc = upload_descs(ctx))) return rc;
    invalidate_graphs(ctx);
    return republish(ctx);
}

int lbm_add_particles(lbm_ctx* ctx, int i, int n, const double* pos, const double* radius,
                      const double* ratio, const double* vel, const double* omega) {
    return add_particles_impl(ctx, i, n, pos, radius, nullptr, nullptr, ratio, vel, omega);
}

int lbm_add_ellipses(lbm_ctx* ctx, int i, int n, const double* pos, const double* a, const double* b,
                     const double* theta, const double* ratio, const double* vel, const double* omega) {
    if (n > 0 && !b) return set_err(ctx, LBM_ERR_INVALID, "bad particle arrays%s");
    return add_particles_impl(ctx, i, n, pos, a, b, theta, ratio, vel, omega);
}

static int step_impl(lbm_ctx* ctx, int nsteps) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (nsteps < 0) return set_err(ctx, LBM_ERR_INVALID, "negative step count%s");
    const int G = ctx->graph_steps;
    while (nsteps > 0) {
        if (G > 0 && nsteps >= G) {
            const int p = ctx->par;
            if (!ctx->graph_ok[p]) {
                cudaGraph_t g = nullptr;
                const long long s0 = ctx->steps;
                if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
                CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
                int err = LBM_OK;
                for (int k = 0; k < G && err == LBM_OK; ++k) err = enqueue_step(ctx, ctx->cap);
                cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
                ctx->steps = s0;
                ctx->par = p;
                if (err) return err;
                if (e != cudaSuccess) return cuda_err(ctx, e, "graph capture");
                e = cudaGraphInstantiate(&ctx->exec[p], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_err(ctx, e, "graph instantiate");
                ctx->graph_ok[p] = true;
            }
            CK(cudaGraphLaunch(ctx->exec[p], ctx->st));
            ctx->steps += G;  // G is even: the parity returns to p
            nsteps -= G;
        } else {
            if ((rc = enqueue_step(ctx, ctx->st))) return rc;
            nsteps -= 1;
        }
    }
    return LBM_OK;
}

int lbm_step(lbm_ctx* ctx, int nsteps) {
    if (ctx) ctx->adj.ready = false;
    return step_impl(ctx, nsteps);
}

int lbm_sync(lbm_ctx* ctx) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return read_status(ctx);
}

int lbm_fluid_step_only(lbm_ctx* ctx) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    return enqueue_fluid(ctx, 0);
}

int lbm_step_timed(lbm_ctx* ctx, int nsteps, float* ms_fluid, float* ms_box, float* ms_particles) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (nsteps < 1 || nsteps > 100000) return set_err(ctx, LBM_ERR_INVALID, "nsteps must lie in [1, 100000]%s");
    const int ne = 4 * nsteps;
    std::vector<cudaEvent_t> ev(ne, nullptr);
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < ne && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) --made;
    const bool parts = ctx->np_total > 0;
    double t[3] = {0, 0, 0};
    for (int s = 0; s < nsteps && e == cudaSuccess && rc == LBM_OK; ++s) {
        cudaEvent_t* q = &ev[4 * s];
        e = cudaEventRecord(q[0], ctx->st);
        if (e == cudaSuccess) rc = enqueue_fluid(ctx, 1, ctx->st);
        if (rc == LBM_OK && e == cudaSuccess) e = cudaEventRecord(q[1], ctx->st);
        if (parts && rc == LBM_OK && e == cudaSuccess)
            e = launch_box_sums(P<InstDesc>(ctx->d_insts), P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D, ctx->st);
        if (rc == LBM_OK && e == cudaSuccess) e = cudaEventRecord(q[2], ctx->st);
        if (parts && rc == LBM_OK && e == cudaSuccess) {
            const bool fused = (ctx->np_total + 7) / 8 <= particle_blocks_resident(ctx->num_sms);
            e = launch_particles(P<InstDesc>(ctx->d_insts), P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D,
                                 ctx->inst[0].cfg.K, ctx->par ^ 1, ctx->shape, P<GridBar>(ctx->d_gridbar), fused,
                                 ctx->st, ctx->wait_ns);
        }
        if (rc == LBM_OK && e == cudaSuccess) e = cudaEventRecord(q[3], ctx->st);
        if (rc == LBM_OK && e == cudaSuccess) {
            ctx->par ^= 1;
            ctx->steps += 1;
        }
    }
    if (e == cudaSuccess && rc == LBM_OK) e = cudaStreamSynchronize(ctx->st);
    for (int s = 0; s < nsteps && e == cudaSuccess && rc == LBM_OK; ++s) {
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[4 * s + k], ev[4 * s + k + 1]);
            t[k] += ms;
        }
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    if (rc != LBM_OK) return rc;
    if (e != cudaSuccess) return cuda_err(ctx, e, "lbm_step_timed");
    if (ms_fluid) *ms_fluid = (float)(t[0] / nsteps);
    if (ms_box) *ms_box = (float)(t[1] / nsteps);
    if (ms_particles) *ms_particles = (float)(t[2] / nsteps);
    return read_status(ctx);
}

int lbm_get_fields(lbm_ctx* ctx, int i, float* u, float* p, int* owner, int on_device) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    Instance& I = ctx->inst[i];
    const long long N = (long long)I.n[0] * I.n[1] * I.n[2];
    if (on_device) {
        CK(launch_fields(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), i, N, ctx->par, ctx->shape, u,
                         p, owner, ctx->st));
        return LBM_OK;
    }
    DevBuf du, dp, dow;
    if ((u && (rc = dalloc(ctx, du, sizeof(float) * ctx->D * N))) ||
        (p && (rc = dalloc(ctx, dp, sizeof(float) * N))) ||
        (owner && (rc = dalloc(ctx, dow, sizeof(int) * N)))) {
        dfree(ctx, du); dfree(ctx, dp); dfree(ctx, dow);
        return rc;
    }
    cudaError_t e = launch_fields(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), i, N, ctx->par,
                                  ctx->shape, P<float>(du), P<float>(dp), P<int>(dow), ctx->st);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du.ptr, sizeof(float) * ctx->D * N, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, dp.ptr, sizeof(float) * N, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess && owner) e = cudaMemcpyAsync(owner, dow.ptr, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    dfree(ctx, du); dfree(ctx, dp); dfree(ctx, dow);
    return cuda_err(ctx, e, "lbm_get_fields");
}

int lbm_get_particles(lbm_ctx* ctx, int i, double* pos, double* vel, double* omega, double* theta,
                      double* accel, int* count) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    Instance& I = ctx->inst[i];
    const int n = I.np, D = ctx->D;
    if (n == 0) return LBM_OK;
    std::vector<double> X(3 * n), U(3 * n), W(3 * n), T(3 * n), A(3 * n);
    std::vector<int> C(n);
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(X.data(), I.X.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(U.data(), I.U.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(W.data(), I.W.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(T.data(), I.theta.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(A.data(), I.A.ptr, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(C.data(), I.count.ptr, sizeof(int) * n, cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; ++k) {
        for (int d = 0; d < D; ++d) {
            if (pos) pos[k * D + d] = X[3 * k + d];
            if (vel) vel[k * D + d] = U[3 * k + d];
            if (accel) accel[k * D + d] = A[3 * k + d];
        }
        if (D == 2) {
            if (omega) omega[k] = W[3 * k + 2];
            if (theta) theta[k] = T[3 * k + 2];
        } else {
            for (int d = 0; d < 3; ++d) {
                if (omega) omega[3 * k + d] = W[3 * k + d];
                if (theta) theta[3 * k + d] = T[3 * k + d];
            }
        }
        if (count) count[k] = C[k];
    }
    return LBM_OK;
}

int lbm_get_particles_async(lbm_ctx* ctx, int i, double* pos3, double* vel3, double* omega3, double* theta3,
                            double* accel3, int* count) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    Instance& I = ctx->inst[i];
    const int n = I.np;
    if (n == 0) return LBM_OK;
    const size_t b3 = sizeof(double) * 3 * n;
    const std::pair<double*, DevBuf*> v3[] = {{pos3, &I.X}, {vel3, &I.U}, {omega3, &I.W}, {theta3, &I.theta},
                                              {accel3, &I.A}};
    for (const auto& c : v3)
        if (c.first) CK(cudaMemcpyAsync(c.first, c.second->ptr, b3, cudaMemcpyDeviceToHost, ctx->st));
    if (count) CK(cudaMemcpyAsync(count, I.count.ptr, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->st));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* ctx, int i, const float* f, int on_device) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    ctx->adj.ready = false;
    if (!f) return set_err(ctx, LBM_ERR_INVALID, "null population array%s");
    Instance& I = ctx->inst[i];
    const long long N = (long long)I.n[0] * I.n[1] * I.n[2];
    const float* src = f;
    DevBuf tmp;
    if (!on_device) {
        if ((rc = dalloc(ctx, tmp, sizeof(float) * ctx->Q * N))) return rc;
        CK(cudaMemcpyAsync(tmp.ptr, f, sizeof(float) * ctx->Q * N, cudaMemcpyHostToDevice, ctx->st));
        src = P<float>(tmp);
    }
    cudaError_t e = launch_pack(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), i, N, ctx->par, src, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    dfree(ctx, tmp);
    return cuda_err(ctx, e, "lbm_set_populations");
}

int lbm_get_populations(lbm_ctx* ctx, int i, float* f, int on_device) {
    int rc = check_inst(ctx, i);
    if (rc) return rc;
    if (!f) return set_err(ctx, LBM_ERR_INVALID, "null population array%s");
    Instance& I = ctx->inst[i];
    const long long N = (long long)I.n[0] * I.n[1] * I.n[2];
    if (on_device) {
        CK(launch_unpack(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), i, N, ctx->par, f, ctx->st));
        return LBM_OK;
    }
    DevBuf tmp;
    if ((rc = dalloc(ctx, tmp, sizeof(float) * ctx->Q * N))) return rc;
    cudaError_t e = launch_unpack(ctx->Q, ctx->fp16, P<InstDesc>(ctx->d_insts), i, N, ctx->par,
                                  P<float>(tmp), ctx->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, tmp.ptr, sizeof(float) * ctx->Q * N, cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    dfree(ctx, tmp);
    return cuda_err(ctx, e, "lbm_get_populations");
}

// State blob: header, then per instance the stored populations of the current
// parity followed by the FP64 particle arrays.
int lbm_save_state(lbm_ctx* ctx, void* buf, size_t* bytes) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!bytes) return LBM_ERR_INVALID;
    const size_t ssz = ctx->fp16 ? 2 : 4;
    size_t total = 4 * sizeof(long long);
    for (auto& I : ctx->inst)
        total += sizeof(long long) + ssz * (ctx->Q - 1) * I.qstride +
                 (size_t)I.np * (sizeof(double) * (7 * 3 + 3) + sizeof(int));
    if (!buf) {
        *bytes = total;
        return LBM_OK;
    }
    if (*bytes < total) return set_err(ctx, LBM_ERR_INVALID, "state buffer too small%s");
    CK(cudaStreamSynchronize(ctx->st));
    char* w = static_cast<char*>(buf);
    long long hdr[4] = {0x4c424d50454e32LL, (long long)ctx->inst.size(), ctx->steps, ctx->Q};
    memcpy(w, hdr, sizeof hdr);
    w += sizeof hdr;
    for (auto& I : ctx->inst) {
        long long np = I.np;
        memcpy(w, &np, sizeof np);
        w += sizeof np;
        const size_t fb = ssz * (ctx->Q - 1) * I.qstride;
        CK(cudaMemcpy(w, I.f[ctx->par].ptr, fb, cudaMemcpyDeviceToHost));
        w += fb;
        DevBuf* v3[] = {&I.X, &I.U, &I.W, &I.Un, &I.Wn, &I.theta, &I.A};
        for (DevBuf* b : v3) {
            CK(cudaMemcpy(w, b->ptr, sizeof(double) * 3 * I.np, cudaMemcpyDeviceToHost));
            w += sizeof(double) * 3 * I.np;
        }
        CK(cudaMemcpy(w, I.R.ptr, sizeof(double) * I.np, cudaMemcpyDeviceToHost));
        w += sizeof(double) * I.np;
        memcpy(w, I.hB.data(), sizeof(double) * I.np);
        w += sizeof(double) * I.np;
        CK(cudaMemcpy(w, I.ratio.ptr, sizeof(double) * I.np, cudaMemcpyDeviceToHost));
        w += sizeof(double) * I.np;
        CK(cudaMemcpy(w, I.count.ptr, sizeof(int) * I.np, cudaMemcpyDeviceToHost));
        w += sizeof(int) * I.np;
    }
    *bytes = total;
    return LBM_OK;
}

int lbm_load_state(lbm_ctx* ctx, const void* buf, size_t bytes) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    ctx->adj.ready = false;
    if (!buf || bytes < 4 * sizeof(long long)) return LBM_ERR_INVALID;
    const char* r = static_cast<const char*>(buf);
    long long hdr[4];
    memcpy(hdr, r, sizeof hdr);
    r += sizeof hdr;
    if (hdr[0] != 0x4c424d50454e32LL || hdr[1] != (long long)ctx->inst.size() || hdr[3] != ctx->Q)
        return set_err(ctx, LBM_ERR_INVALID, "state blob does not match this context%s");
    const size_t ssz = ctx->fp16 ? 2 : 4;
    size_t need = sizeof hdr;
    {
        const char* q = r;
        for (auto& I : ctx->inst) {
            if ((size_t)(q - static_cast<const char*>(buf)) + sizeof(long long) > bytes) return LBM_ERR_INVALID;
            long long np;
            memcpy(&np, q, sizeof np);
            if (np < 0 || np > I.cap) return set_err(ctx, LBM_ERR_INVALID, "particle count exceeds capacity%s");
            const size_t add = sizeof(long long) + ssz * (ctx->Q - 1) * I.qstride +
                               (size_t)np * (sizeof(double) * 24 + sizeof(int));
            need += add;
            q += add;
        }
    }
    if (need > bytes) return set_err(ctx, LBM_ERR_INVALID, "state blob truncated%s");
    CK(cudaStreamSynchronize(ctx->st));
    for (auto& I : ctx->inst) {
        long long np;
        memcpy(&np, r, sizeof np);
        r += sizeof np;
        const size_t fb = ssz * (ctx->Q - 1) * I.qstride;
        CK(cudaMemcpy(I.f[ctx->par].ptr, r, fb, cudaMemcpyHostToDevice));
        r += fb;
        I.np = (int)np;
        DevBuf* v3[] = {&I.X, &I.U, &I.W, &I.Un, &I.Wn, &I.theta, &I.A};
        for (DevBuf* b : v3) {
            CK(cudaMemcpy(b->ptr, r, sizeof(double) * 3 * I.np, cudaMemcpyHostToDevice));
            r += sizeof(double) * 3 * I.np;
        }
        I.hR.assign(reinterpret_cast<const double*>(r), reinterpret_cast<const double*>(r) + I.np);
        CK(cudaMemcpy(I.R.ptr, r, sizeof(double) * I.np, cudaMemcpyHostToDevice));
        r += sizeof(double) * I.np;
        I.hB.assign(reinterpret_cast<const double*>(r), reinterpret_cast<const double*>(r) + I.np);
        r += sizeof(double) * I.np;
        CK(cudaMemcpy(I.ratio.ptr, r, sizeof(double) * I.np, cudaMemcpyHostToDevice));
        I.hratio.assign(reinterpret_cast<const double*>(r), reinterpret_cast<const double*>(r) + I.np);
        r += sizeof(double) * I.np;
        if ((rc = layout_boxes(ctx, I))) return rc;
        if ((rc = upload_pconst(ctx, I))) return rc;
        CK(cudaMemcpy(I.count.ptr, r, sizeof(int) * I.np, cudaMemcpyHostToDevice));
        r += sizeof(int) * I.np;
    }
    ctx->steps = hdr[2];
    if ((rc = upload_descs(ctx))) return rc;
    invalidate_graphs(ctx);
    return republish(ctx);
}

int lbm_set_graphs(lbm_ctx* ctx, int steps_per_graph) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (steps_per_graph < 0 || (steps_per_graph & 1))
        return set_err(ctx, LBM_ERR_INVALID, "steps_per_graph must be 0 or a positive even number%s");
    ctx->graph_steps = steps_per_graph;
    invalidate_graphs(ctx);
    return LBM_OK;
}

int lbm_set_particle_wait_limit(lbm_ctx* ctx, double seconds) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (!(seconds >= 0.0) || seconds > 60.0)
        return set_err(ctx, LBM_ERR_INVALID, "the wait limit must lie in [0, 60] s%s");
    ctx->wait_ns = (long long)(seconds * 1e9);
    invalidate_graphs(ctx);  // captured launches carry the old bound
    return LBM_OK;
}

int lbm_kernel_shape(const lbm_ctx* ctx, int* vec, int* tile_rows, int* warps) {
    if (!ctx) return LBM_ERR_INVALID;
    if (vec) *vec = ctx->shape.tma ? 0 : ctx->shape.vec;
    if (tile_rows) *tile_rows = ctx->shape.ty * ctx->shape.tz;
    if (warps) *warps = ctx->shape.warps;
    return LBM_OK;
}

static bool shape_ok(const lbm_ctx* ctx, int vec) {
    return ctx->fp16 ? (vec == 2 || vec == 4 || vec == 8) : (vec == 1 || vec == 2 || vec == 4);
}

int lbm_set_kernel_shape(lbm_ctx* ctx, int vec, int tile_rows, int warps) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if ((vec != 0 && !shape_ok(ctx, vec)) || tile_rows < 1 || tile_rows > 64 || warps < 1 || warps > 8)
        return set_err(ctx, LBM_ERR_INVALID, "unsupported kernel shape%s");
    Shape s = ctx->shape;
    s.tma = vec == 0;
    if (vec) s.vec = vec;
    s.warps = warps;
    if (s.tma && !tma_rows_ok(tile_rows))
        return set_err(ctx, LBM_ERR_INVALID, "TMA tiles hold 4 or 8 rows%s");
    if (ctx->D == 2) {
        s.ty = tile_rows;
        s.tz = 1;
    } else {
        int tz = 1;
        while (tz * tz < tile_rows) tz *= 2;
        if (tile_rows % tz) return set_err(ctx, LBM_ERR_INVALID, "3D tile rows must factor as ty*tz%s");
        s.tz = tz;
        s.ty = tile_rows / tz;
    }
    return configure_shape(ctx, s);
}

int lbm_autotune(lbm_ctx* ctx, int reps) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (reps < 1) reps = 5;
    std::vector<Shape> cand;
    const int vecs32[] = {1, 2, 4}, vecs16[] = {2, 4, 8};
    const int* vecs = ctx->fp16 ? vecs16 : vecs32;
    for (int vi = 0; vi < 3; ++vi)
        for (int rows : {2, 4, 8})
            for (int warps : {2, 4, 8})
                for (int pers : {0, 1}) {
                    if (warps > rows) continue;
                    Shape s{vecs[vi], rows, 1, warps, pers, 0, 0, 0};
                    if (ctx->D == 3) {
                        s.tz = rows >= 4 ? 2 : 1;
                        s.ty = rows / s.tz;
                    }
                    cand.push_back(s);
                }
    for (int rows : {4, 8})
        for (int warps : {4, 8})
            for (int stages : {2, 3, 4}) {
                Shape s{ctx->shape.vec, rows, 1, warps, 1, 1, stages, 0};
                if (ctx->D == 3) {
                    s.tz = rows >= 4 ? 2 : 1;
                    s.ty = rows / s.tz;
                }
                cand.push_back(s);
            }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Shape bests = ctx->shape;
    for (const Shape& s : cand) {
        if ((rc = configure_shape(ctx, s))) {
            if (rc == LBM_ERR_INVALID) {  // does not fit: skip this shape
                rc = LBM_OK;
                continue;
            }
            break;
        }
        for (int w = 0; w < 2; ++w)
            if ((rc = enqueue_fluid(ctx, 0))) break;
        if (rc) break;
        cudaEventRecord(e0, ctx->st);
        for (int k = 0; k < reps && rc == LBM_OK; ++k) rc = enqueue_fluid(ctx, 0);
        cudaEventRecord(e1, ctx->st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = LBM_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bests = ctx->shape;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = configure_shape(ctx, bests);
    return rc ? rc : rc2;
}

int lbm_launches_per_step(const lbm_ctx* ctx) {
    if (!ctx) return 0;
    if (ctx->np_total == 0) return 1;
    const bool fused = (ctx->np_total + 7) / 8 <= particle_blocks_resident(ctx->num_sms);
    return 2 + (fused ? 1 : 1 + ctx->inst[0].cfg.K);  // fluid, box sums, particles
}

long long lbm_steps_done(const lbm_ctx* ctx) { return ctx ? ctx->steps : 0; }

long long lbm_total_nodes(const lbm_ctx* ctx) {
    if (!ctx) return 0;
    long long n = 0;
    for (auto& I : ctx->inst) n += (long long)I.n[0] * I.n[1] * I.n[2];
    return n;
}

// ------------------------------------------------------------- adjoint ---
// Forward pass with checkpoints: the populations and particle state at the
// start of every segment of L steps (L = ceil(sqrt(nsteps)) by default), and
// the final particle state.  The context advances by nsteps like lbm_step.
int lbm_adjoint_forward(lbm_ctx* ctx, int nsteps, int seg_len) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    if (nsteps < 1) return set_err(ctx, LBM_ERR_INVALID, "nsteps must be positive%s");
    if (seg_len < 0) return set_err(ctx, LBM_ERR_INVALID, "negative segment length%s");
    for (const Instance& I : ctx->inst)
        for (int p = 0; p < I.np; ++p)
            if (I.hB[p] != I.hR[p]) return set_err(ctx, LBM_ERR_INVALID, "the adjoint covers disks and spheres only%s");
    AdjCtx& A = ctx->adj;
    A.ready = false;
    // an even segment length keeps the parity of the global step equal to that
    // of the step within its segment, so one set of per-step descriptors (and
    // one captured graph) serves every segment
    int L = seg_len > 0 ? seg_len : std::max(1, (int)ceil(sqrt((double)nsteps)));
    if (L >= nsteps) L = nsteps;
    else if (L & 1) L += 1;
    const int nseg = (nsteps + L - 1) / L;
    const size_t ssz = ctx->fp16 ? 2 : 4;
    const int ni = (int)ctx->inst.size();
    if ((int)A.ai.size() != ni) {
        adj_release(ctx);
        A.ai.resize(ni);
    }
    for (int i = 0; i < ni; ++i) {
        Instance& I = ctx->inst[i];
        AdjInst& a = A.ai[i];
        const size_t fb = ssz * (size_t)(ctx->Q - 1) * (size_t)I.qstride;
        for (size_t s = nseg; s < a.ckpt.size(); ++s) dfree(ctx, a.ckpt[s]);
        a.ckpt.resize(nseg);
        for (int s = 0; s < nseg; ++s)
            if ((rc = dalloc(ctx, a.ckpt[s], fb))) return rc;
        if ((rc = dalloc(ctx, a.ckst, sizeof(double) * 16 * (size_t)std::max(I.np, 1) * (nseg + 1)))) return rc;
    }
    for (int s = 0; s < nseg; ++s) {
        for (int i = 0; i < ni; ++i) {
            Instance& I = ctx->inst[i];
            AdjInst& a = A.ai[i];
            CK(cudaMemcpyAsync(a.ckpt[s].ptr, I.f[ctx->par].ptr, a.ckpt[s].bytes, cudaMemcpyDeviceToDevice,
                               ctx->st));
            CK(launch_adj_state(P<InstDesc>(ctx->d_insts), i, I.np, P<double>(a.ckst) + 16LL * I.np * s, 1,
                                ctx->st));
        }
        if ((rc = step_impl(ctx, std::min(L, nsteps - s * L)))) return rc;
    }
    for (int i = 0; i < ni; ++i) {
        Instance& I = ctx->inst[i];
        CK(launch_adj_state(P<InstDesc>(ctx->d_insts), i, I.np, P<double>(A.ai[i].ckst) + 16LL * I.np * nseg,
                            1, ctx->st));
    }
    A.nsteps = nsteps;
    A.L = L;
    A.nseg = nseg;
    A.ready = true;
    return LBM_OK;
}

namespace {

// Adjoint particle arrays of one instance inside one allocation.
size_t adj_pbuf_doubles(int np, int K) {
    const size_t n3 = 3 * (size_t)std::max(np, 1);
    return 5 * n3 + (size_t)std::max(np, 1) + 1 + 4 * (size_t)std::max(np, 1) + 4 * (size_t)std::max(np, 1) +
           n3 + (size_t)(K + 1) * n3 + 3 * (size_t)K * n3 + 5 * n3 + 8;
}
AdjBufs adj_bufs_layout(void* base, int np, int K) {
    double* q = static_cast<double*>(base);
    const size_t n1 = (size_t)std::max(np, 1), n3 = 3 * n1;
    AdjBufs b;
    b.Xb = q; q += n3;
    b.Ub = q; q += n3;
    b.Wb = q; q += n3;
    b.Tb = q; q += n3;
    b.Ab = q; q += n3;
    b.rb = q; q += n1;
    b.alpha_b = q; q += 1;
    b.Abar = q; q += 4 * n1;
    b.coef = reinterpret_cast<float*>(q); q += 4 * n1;
    b.Ubar = q; q += n3;
    b.Xk = q; q += (size_t)(K + 1) * n3;
    b.Xs = q; q += (size_t)K * n3;
    b.F1 = q; q += (size_t)K * n3;
    b.F2 = q; q += (size_t)K * n3;
    b.Xkb = q; q += n3;
    b.Xsb = q; q += n3;
    b.v = q; q += n3;
    b.Ubb = q; q += n3;
    b.Wnb = q; q += n3;
    return b;
}

}  // namespace

// Backward sweep over the recorded forward pass (see lbmpen.h for layouts).
int lbm_adjoint_backward(lbm_ctx* ctx, const double* seed_particles, const float* seed_field,
                         double* grad_particles, float* grad_field) {
    int rc = check_ctx(ctx);
    if (rc) return rc;
    AdjCtx& A = ctx->adj;
    if (!A.ready) return set_err(ctx, LBM_ERR_STATE, "no recorded forward pass (call lbm_adjoint_forward)%s");
    if (!grad_particles) return set_err(ctx, LBM_ERR_INVALID, "null gradient array%s");
    const int ni = (int)ctx->inst.size(), L = A.L, nseg = A.nseg, N = A.nsteps;
    const int K = ctx->inst[0].cfg.K;
    const size_t ssz = ctx->fp16 ? 2 : 4;
    const Shape& sh = ctx->shape;
    // records, slots and adjoint arrays
    for (int i = 0; i < ni; ++i) {
        Instance& I = ctx->inst[i];
        AdjInst& a = A.ai[i];
        const size_t n1 = (size_t)std::max(I.np, 1);
        const size_t fb = ssz * (size_t)(ctx->Q - 1) * (size_t)I.qstride;
        for (size_t k = L + 1; k < a.slot.size(); ++k) dfree(ctx, a.slot[k]);
        a.slot.resize(L + 1);
        for (int k = 0; k <= L; ++k)
            if ((rc = dalloc(ctx, a.slot[k], fb))) return rc;
        if ((rc = dalloc(ctx, a.rprec, sizeof(PRec) * n1 * (L + 1))) ||
            (rc = dalloc(ctx, a.rlcnt, sizeof(int) * (size_t)I.ntiles * (L + 1))) ||
            (rc = dalloc(ctx, a.rlent, sizeof(uint32_t) * (size_t)I.ntiles * LIST_CAP * (L + 1))) ||
            (rc = dalloc(ctx, a.rlrec, (size_t)CAND_BYTES * I.ntiles * LIST_CAP * (L + 1))) ||
            (rc = dalloc(ctx, a.rgeo, sizeof(double) * NPV * n1 * (L + 1))) ||
            (rc = dalloc(ctx, a.rstate, sizeof(double) * 16 * n1 * (L + 1))) ||
            (rc = dalloc(ctx, a.fbar[0], sizeof(float) * (ctx->Q - 1) * (size_t)I.qstride)) ||
            (rc = dalloc(ctx, a.fbar[1], sizeof(float) * (ctx->Q - 1) * (size_t)I.qstride)) ||
            (rc = dalloc(ctx, a.pbuf, sizeof(double) * adj_pbuf_doubles(I.np, K))))
            return rc;
        CK(cudaMemsetAsync(a.pbuf.ptr, 0, a.pbuf.bytes, ctx->st));
    }
    // descriptors of the recomputation: step k reads slot k and writes slot
    // k + 1, its records go to record k (and k + 1 for the next step's input);
    // entry L is the publish of a segment's first state into record 0
    std::vector<InstDesc> rd((size_t)(L + 1) * ni);
    std::vector<CUtensorMap> tm(sh.tma ? (size_t)L * ni * 2 : 0);
    for (int k = 0; k <= L; ++k)
        for (int i = 0; i < ni; ++i) {
            Instance& I = ctx->inst[i];
            AdjInst& a = A.ai[i];
            const size_t n1 = (size_t)std::max(I.np, 1);
            InstDesc d = make_desc(ctx, I);
            PRec* rp = P<PRec>(a.rprec);
            int* lc = P<int>(a.rlcnt);
            uint32_t* le = P<uint32_t>(a.rlent);
            char* lr = P<char>(a.rlrec);
            if (k == L) {
                d.prec_out = rp;
                d.list_cnt[0] = lc;
                d.list_ent[0] = le;
                d.list_rec[0] = lr;
            } else {
                const int par = k & 1;
                d.f[par] = a.slot[k].ptr;
                d.f[par ^ 1] = a.slot[k + 1].ptr;
                d.prec = rp + n1 * k;
                d.prec_out = rp + n1 * (k + 1);
                d.list_cnt[par] = lc + (size_t)I.ntiles * k;
                d.list_ent[par] = le + (size_t)I.ntiles * LIST_CAP * k;
                d.list_cnt[par ^ 1] = lc + (size_t)I.ntiles * (k + 1);
                d.list_ent[par ^ 1] = le + (size_t)I.ntiles * LIST_CAP * (k + 1);
                d.list_rec[par] = lr + (size_t)CAND_BYTES * I.ntiles * LIST_CAP * k;
                d.list_rec[par ^ 1] = lr + (size_t)CAND_BYTES * I.ntiles * LIST_CAP * (k + 1);
                d.adj_geo = P<double>(a.rgeo) + NPV * n1 * k;
                d.rec_state = P<double>(a.rstate) + 16 * n1 * (k + 1);
                if (sh.tma) {
                    if ((rc = encode_pop_map(ctx, I, a.slot[k].ptr, &tm[(size_t)k * ni * 2 + 2 * i + par]))) return rc;
                    if ((rc = encode_pop_map(ctx, I, a.slot[k + 1].ptr, &tm[(size_t)k * ni * 2 + 2 * i + (par ^ 1)])))
                        return rc;
                }
            }
            rd[(size_t)k * ni + i] = d;
        }
    if ((rc = dalloc(ctx, A.d_rdesc, sizeof(InstDesc) * rd.size()))) return rc;
    CK(cudaMemcpyAsync(A.d_rdesc.ptr, rd.data(), sizeof(InstDesc) * rd.size(), cudaMemcpyHostToDevice, ctx->st));
    if (sh.tma) {
        if ((rc = dalloc(ctx, A.d_rtmaps, sizeof(CUtensorMap) * tm.size()))) return rc;
        CK(cudaMemcpyAsync(A.d_rtmaps.ptr, tm.data(), sizeof(CUtensorMap) * tm.size(), cudaMemcpyHostToDevice,
                           ctx->st));
    }
    // per-step views of the backward sweep, step k of a segment (entry L: the
    // last step of the whole run when it reads a field seed)
    const int len_last = N - (nseg - 1) * L;
    std::vector<AdjFluid> afl((size_t)(L + 1) * ni);
    std::vector<AdjPart> apt((size_t)L * ni);
    std::vector<AdjBufs> ab(ni);
    std::vector<long long> out_off(ni);
    long long nout = 0;
    long long foff = 0;
    std::vector<long long> field_off(ni);
    for (int i = 0; i < ni; ++i) {
        Instance& I = ctx->inst[i];
        ab[i] = adj_bufs_layout(A.ai[i].pbuf.ptr, I.np, K);
        out_off[i] = nout;
        nout += 1 + 16LL * I.np;
        field_off[i] = foff;
        foff += (long long)ctx->Q * I.n[0] * I.n[1] * I.n[2];
    }
    for (int k = 0; k <= L; ++k) {
        const int kk = k == L ? len_last - 1 : k;
        for (int i = 0; i < ni; ++i) {
            Instance& I = ctx->inst[i];
            AdjInst& a = A.ai[i];
            const size_t n1 = (size_t)std::max(I.np, 1);
            AdjFluid f;
            f.fin = a.slot[kk].ptr;
            f.prec = P<PRec>(a.rprec) + n1 * kk;
            f.lcnt = P<int>(a.rlcnt) + (size_t)I.ntiles * kk;
            f.lent = P<uint32_t>(a.rlent) + (size_t)I.ntiles * LIST_CAP * kk;
            f.lam_src = k == L ? (seed_field ? seed_field + field_off[i] : nullptr) : P<float>(a.fbar[(kk + 1) & 1]);
            f.lam_dst = P<float>(a.fbar[kk & 1]);
            f.coef = ab[i].coef;
            f.Abar = ab[i].Abar;
            afl[(size_t)k * ni + i] = f;
            if (k == L) continue;
            AdjPart pp;
            pp.st0 = P<double>(a.rstate) + 16 * n1 * k;
            pp.st1 = P<double>(a.rstate) + 16 * n1 * (k + 1);
            pp.geo = P<double>(a.rgeo) + NPV * n1 * k;
            apt[(size_t)k * ni + i] = pp;
        }
    }
    if ((rc = dalloc(ctx, A.d_afl, sizeof(AdjFluid) * afl.size())) ||
        (rc = dalloc(ctx, A.d_apt, sizeof(AdjPart) * apt.size())) ||
        (rc = dalloc(ctx, A.d_abufs, sizeof(AdjBufs) * ni)) ||
        (rc = dalloc(ctx, A.d_out, sizeof(double) * std::max<long long>(nout, 1))) ||
        (rc = dalloc(ctx, A.d_out_off, sizeof(long long) * ni)))
        return rc;
    CK(cudaMemcpyAsync(A.d_afl.ptr, afl.data(), sizeof(AdjFluid) * afl.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(A.d_apt.ptr, apt.data(), sizeof(AdjPart) * apt.size(), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(A.d_abufs.ptr, ab.data(), sizeof(AdjBufs) * ni, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(A.d_out_off.ptr, out_off.data(), sizeof(long long) * ni, cudaMemcpyHostToDevice, ctx->st));
    // seeds: the adjoint of the final particle state
    std::vector<std::vector<double>> seeds(ni);
    if (seed_particles) {
        const double* sp = seed_particles;
        for (int i = 0; i < ni; ++i) {
            const int np = ctx->inst[i].np;
            std::vector<double>& h = seeds[i];
            h.assign(15 * (size_t)np, 0.0);
            for (int p = 0; p < np; ++p)
                for (int a5 = 0; a5 < 5; ++a5)
                    for (int d = 0; d < 3; ++d) h[(size_t)a5 * 3 * np + 3 * p + d] = sp[15 * p + 3 * a5 + d];
            if (np) CK(cudaMemcpyAsync(ab[i].Xb, h.data(), sizeof(double) * 15 * np, cudaMemcpyHostToDevice, ctx->st));
            sp += 15 * (size_t)np;
        }
    }
    const InstDesc* dI = P<InstDesc>(ctx->d_insts);
    const InstDesc* dR = P<InstDesc>(A.d_rdesc);
    const bool fused = (ctx->np_total + 7) / 8 <= particle_blocks_resident(ctx->num_sms);
    // recomputation of a segment of len steps into the slots and records, then
    // the backward sweep through it (k = len - 1 .. 0); last: the segment holds
    // the final step of the run, whose adjoint comes from the seed
    auto enqueue_segment = [&](cudaStream_t st, int len, bool last) -> int {
        for (int k = 0; k < len; ++k) {
            const int par = k & 1;
            const InstDesc* dk = dR + (size_t)k * ni;
            if (sh.tma)
                CK(launch_fluid_tma(ctx->Q, ctx->fp16, dk, P<CUtensorMap>(A.d_rtmaps) + (size_t)k * ni * 2,
                                    P<uint16_t>(ctx->d_tile_inst), ctx->ntiles, par, sh, 1, ctx->grid,
                                    P<int>(ctx->d_tile_ctr), sh.stages, ni, st));
            else
                CK(launch_fluid(ctx->Q, ctx->fp16, dk, P<uint16_t>(ctx->d_tile_inst), ctx->ntiles, par, sh, 1,
                                sh.persistent, ctx->grid, P<int>(ctx->d_tile_ctr), st));
            if (ctx->np_total > 0) CK(launch_box_sums(dk, P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D, st));
            if (ctx->np_total > 0)
                CK(launch_particles(dk, P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D, K, par ^ 1, sh,
                                    P<GridBar>(ctx->d_gridbar), fused, st, ctx->wait_ns));
        }
        for (int k = len - 1; k >= 0; --k) {
            CK(launch_adj_particles(ctx->D, dI, P<AdjPart>(A.d_apt) + (size_t)k * ni, P<AdjBufs>(A.d_abufs), ni,
                                    st));
            const bool final_step = last && k == len - 1;
            const int mode = final_step ? (seed_field ? 1 : 2) : 0;
            CK(launch_adj_fluid(ctx->Q, ctx->fp16, dI, P<AdjFluid>(A.d_afl) + (size_t)(final_step ? L : k) * ni,
                                P<uint16_t>(ctx->d_tile_inst), ctx->ntiles, mode, sh, st));
        }
        return LBM_OK;
    };
    adj_drop_graph(A);  // descriptors and buffers may have moved since the last capture
    for (int s = nseg - 1; s >= 0; --s) {
        const int len = std::min(L, N - s * L);
        // restore the segment's first state into slot 0, record 0 and the context
        for (int i = 0; i < ni; ++i) {
            Instance& I = ctx->inst[i];
            AdjInst& a = A.ai[i];
            CK(cudaMemcpyAsync(a.slot[0].ptr, a.ckpt[s].ptr, a.ckpt[s].bytes, cudaMemcpyDeviceToDevice, ctx->st));
            double* st = P<double>(a.ckst) + 16LL * I.np * s;
            CK(launch_adj_state(dI, i, I.np, st, 0, ctx->st));
            if (I.np)
                CK(cudaMemcpyAsync(a.rstate.ptr, st, sizeof(double) * 16 * I.np, cudaMemcpyDeviceToDevice, ctx->st));
            CK(cudaMemsetAsync(a.rlcnt.ptr, 0, sizeof(int) * I.ntiles, ctx->st));
            if (I.ubox.ptr) CK(cudaMemsetAsync(I.ubox.ptr, 0xff, I.ubox.bytes, ctx->st));
        }
        if (ctx->np_total > 0)
            CK(launch_publish(dR + (size_t)L * ni, P<PartRef>(ctx->d_refs), ctx->np_total, ctx->D, 0, sh, ctx->st));
        if (s == nseg - 1) {
            if ((rc = enqueue_segment(ctx->st, len, true))) return rc;
            continue;
        }
        // every other segment is a full one: replay one captured graph
        if (!A.seg_exec) {
            cudaGraph_t g = nullptr;
            if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
            const int err = enqueue_segment(ctx->cap, L, false);
            cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
            if (err) return err;
            if (e != cudaSuccess) return cuda_err(ctx, e, "adjoint graph capture");
            e = cudaGraphInstantiate(&A.seg_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_err(ctx, e, "adjoint graph instantiate");
        }
        CK(cudaGraphLaunch(A.seg_exec, ctx->st));
    }
    CK(launch_adj_finish(dI, P<AdjBufs>(A.d_abufs), P<long long>(A.d_out_off), P<double>(A.d_out), ni, ctx->st));
    if (grad_field)
        for (int i = 0; i < ni; ++i) {
            Instance& I = ctx->inst[i];
            const long long Nn = (long long)I.n[0] * I.n[1] * I.n[2];
            CK(launch_adj_pull_out(ctx->Q, dI, i, Nn, P<float>(A.ai[i].fbar[0]), grad_field + field_off[i], ctx->st));
        }
    // the context returns to the state after the forward pass
    for (int i = 0; i < ni; ++i) {
        Instance& I = ctx->inst[i];
        CK(launch_adj_state(dI, i, I.np, P<double>(A.ai[i].ckst) + 16LL * I.np * nseg, 0, ctx->st));
    }
    CK(cudaMemcpyAsync(grad_particles, A.d_out.ptr, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->st));
    return read_status(ctx);
}

int lbm_adjoint_run(lbm_ctx* ctx, int nsteps, int seg_len, const double* seed_particles, const float* seed_field,
                    double* grad_particles, float* grad_field) {
    int rc = lbm_adjoint_forward(ctx, nsteps, seg_len);
    if (rc) return rc;
    return lbm_adjoint_backward(ctx, seed_particles, seed_field, grad_particles, grad_field);
}

int lbm_adjoint_release(lbm_ctx* ctx) {
    if (!ctx) return LBM_ERR_INVALID;
    cudaStreamSynchronize(ctx->st);
    adj_release(ctx);
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    destroy_all(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
}

}  // extern "C"
