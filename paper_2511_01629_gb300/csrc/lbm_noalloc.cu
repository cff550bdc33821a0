// Rigid-body projection (Eq. 22) of a velocity field onto a set of particles,
// in a variant that allocates no memory: its scratch is a fixed array in the
// library's device image instead of memory from cudaMalloc or an allocator.
//
// It exists for callers that cannot allocate device memory at the point where
// they need the projection: a plugin whose host owns all device memory and
// forbids allocation, a frame loop that must not stall on the implicit device
// synchronisation of cudaMalloc/cudaFree, or code holding a stream it may only
// enqueue work on.  The context-based path (lbm_create ... lbm_step) computes
// the same sums inside the fused fluid kernel, with scratch from the caller's
// allocator.
//
// Limits: at most LBM_NOALLOC_MAX_PARTICLES particles, radii <= 120 lattice
// units in 2D and <= 40 in 3D (the bounds under which the exact integer sums
// fit in 64 bits).  Every call uses the same array: calls that overlap on the GPU (on
// different streams, or from several host threads) race and give wrong sums.
// The array stays allocated on every GPU that loads the library until the
// process exits.
#include <mutex>

#include "../../include/lbmpen.h"
#include "lbm_common.cuh"

namespace lbmpen {
namespace {

constexpr int NA_MAXP = LBM_NOALLOC_MAX_PARTICLES;
constexpr int NA_ERR = NA_MAXP * NPV;  // index of the error word after the sums
constexpr int NA_BLOCK = 256;          // nodes of one particle's box per block

// Scratch: int64 sums of Eq. 22 per particle (fixed point, as in the fused
// kernel) followed by one error word.
__device__ __align__(256) long long g_noalloc_scratch[NA_MAXP * NPV + 32];

__global__ void k_na_clear(long long* scratch, int np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np * NPV) scratch[i] = 0;
    if (i == 0) scratch[NA_ERR] = 0;
}

struct NaGrid {
    int n[3];
    int per[3];
    int D;
};

// One block per (particle p, 256-node slice of p's bounding box).  A node is
// counted for p when it lies inside p (exact FP64 form of Eq. 9) and inside
// no particle of lower index, the owner rule of the fused kernel.
__global__ void __launch_bounds__(NA_BLOCK) k_na_accumulate(NaGrid g, const float* __restrict__ u,
                                                            int np, const double* __restrict__ X,
                                                            const double* __restrict__ R,
                                                            double max_radius, long long* scratch) {
    __shared__ int lower[64];  // lower-index particles that overlap p
    __shared__ int nlower;
    const int p = blockIdx.x;
    const int D = g.D;
    double Xp[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) Xp[d] = X[p * D + d];
    const double Rp = R[p];
    if (threadIdx.x == 0) {
        nlower = 0;
        if (!(Rp >= 0.0) || Rp > max_radius) atomicOr(reinterpret_cast<unsigned long long*>(scratch + NA_ERR), 1ull);
    }
    __syncthreads();
    if (!(Rp >= 0.0) || Rp > max_radius) return;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double d2 = 0.0;
        for (int d = 0; d < D; ++d) {
            double dx = X[j * D + d] - Xp[d];
            if (g.per[d]) dx -= g.n[d] * rint(dx / g.n[d]);
            d2 += dx * dx;
        }
        const double reach = R[j] + Rp + 2.0;
        if (d2 <= reach * reach) {
            const int slot = atomicAdd(&nlower, 1);
            if (slot < 64) lower[slot] = j;
            else atomicOr(reinterpret_cast<unsigned long long*>(scratch + NA_ERR), 2ull);
        }
    }
    __syncthreads();
    const int nl = min(nlower, 64);
    // bounding box of p, node range [floor(X - R) - 1, floor(X + R) + 1] per axis
    int lo[3] = {0, 0, 0}, len[3] = {1, 1, 1}, ref[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
        lo[d] = (int)floor(Xp[d] - Rp) - 1;
        len[d] = (int)floor(Xp[d] + Rp) + 1 - lo[d] + 1;
        ref[d] = (int)floor(Xp[d]);
    }
    const long long total = (long long)len[0] * len[1] * len[2];
    const long long k = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
    int icnt = 0, id[3] = {0, 0, 0}, idd[6] = {0, 0, 0, 0, 0, 0};
    long long su[3] = {0, 0, 0}, sl[3] = {0, 0, 0};
    if (k < total) {
        const int off[3] = {(int)(k % len[0]), (int)((k / len[0]) % len[1]), (int)(k / ((long long)len[0] * len[1]))};
        int xyz[3] = {0, 0, 0}, dd[3] = {0, 0, 0};
        bool ok = true;
        for (int d = 0; d < D; ++d) {
            int x = lo[d] + off[d];
            if (g.per[d]) x = ((x % g.n[d]) + g.n[d]) % g.n[d];
            else if (x < 0 || x >= g.n[d]) ok = false;
            xyz[d] = x;
            dd[d] = lo[d] + off[d] - ref[d];  // offset from floor(X), unwrapped
        }
        const int pm = g.per[0] | (g.per[1] << 1) | (g.per[2] << 2);
        PRec pr;
        for (int d = 0; d < 3; ++d) pr.X[d] = Xp[d];
        pr.R2 = Rp * Rp;
        pr.shape = 0;  // disks and spheres only
        if (ok && ((D == 2) ? inside_exact<2>(&pr, xyz[0], xyz[1], 0, g.n[0], g.n[1], 1, pm)
                            : inside_exact<3>(&pr, xyz[0], xyz[1], xyz[2], g.n[0], g.n[1], g.n[2], pm))) {
            bool mine = true;
            for (int i = 0; i < nl && mine; ++i) {
                PRec q;
                const int j = lower[i];
                for (int d = 0; d < 3; ++d) q.X[d] = d < D ? X[j * D + d] : 0.0;
                q.R2 = R[j] * R[j];
                q.shape = 0;
                if ((D == 2) ? inside_exact<2>(&q, xyz[0], xyz[1], 0, g.n[0], g.n[1], 1, pm)
                             : inside_exact<3>(&q, xyz[0], xyz[1], xyz[2], g.n[0], g.n[1], g.n[2], pm))
                    mine = false;
            }
            if (mine) {
                const long long node = ((long long)xyz[2] * g.n[1] + xyz[1]) * g.n[0] + xyz[0];
                long long ux[3] = {0, 0, 0};
                float uu = 0.f;
                for (int d = 0; d < D; ++d) {
                    const float v = u[d * N + node];
                    uu = fmaf(v, v, uu);
                    ux[d] = to_fx(v);
                }
                // the speed bound of the exact sums, as in the fused kernel's
                // divergence test (true for NaN too; to_fx would clamp silently)
                if (!(uu < 0.25f)) atomicOr(reinterpret_cast<unsigned long long*>(scratch + NA_ERR), 4ull);
                icnt = 1;
                for (int d = 0; d < 3; ++d) id[d] = dd[d];
                idd[0] = dd[0] * dd[0]; idd[1] = dd[1] * dd[1]; idd[2] = dd[2] * dd[2];
                idd[3] = dd[0] * dd[1]; idd[4] = dd[0] * dd[2]; idd[5] = dd[1] * dd[2];
                for (int d = 0; d < 3; ++d) su[d] = ux[d];
                sl[0] = (long long)dd[1] * ux[2] - (long long)dd[2] * ux[1];
                sl[1] = (long long)dd[2] * ux[0] - (long long)dd[0] * ux[2];
                sl[2] = (long long)dd[0] * ux[1] - (long long)dd[1] * ux[0];
            }
        }
    }
    long long v[NPV];
    v[0] = __reduce_add_sync(0xffffffffu, icnt);
    for (int d = 0; d < 3; ++d) v[1 + d] = __reduce_add_sync(0xffffffffu, id[d]);
    for (int d = 0; d < 6; ++d) v[4 + d] = __reduce_add_sync(0xffffffffu, idd[d]);
    for (int d = 0; d < 3; ++d) {
        v[10 + d] = warp_sum_ll(su[d]);
        v[13 + d] = warp_sum_ll(sl[d]);
    }
    if ((threadIdx.x & 31) == 0 && v[0] != 0) {
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(scratch + (long long)p * NPV);
        for (int i = 0; i < NPV; ++i)
            if (v[i] != 0) atomicAdd(dst + i, (unsigned long long)v[i]);
    }
}

// U = sum u / n and the angular velocity from the moments about floor(X),
// as in the context path's finalisation.
__global__ void k_na_finalize(int D, int np, const double* __restrict__ X, long long* scratch,
                              double* U, double* W, int* count) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const long long* v = scratch + (long long)p * NPV;
    const double scale = 1.0 / (double)(1LL << FXBITS);
    const double cnt = (double)v[0];
    double phi[3] = {0, 0, 0}, Sd[3], Su[3], Sl[3];
    for (int d = 0; d < 3; ++d) {
        if (d < D) phi[d] = X[p * D + d] - floor(X[p * D + d]);
        Sd[d] = (double)v[1 + d];
        Su[d] = (double)v[10 + d] * scale;
        Sl[d] = (double)v[13 + d] * scale;
    }
    count[p] = (int)v[0];
    auto degenerate = [&]() {  // no node, or a node set without rotational inertia
        atomicOr(reinterpret_cast<unsigned long long*>(scratch + NA_ERR), 8ull);
        for (int d = 0; d < D; ++d) U[p * D + d] = 0.0;
        if (D == 2) W[p] = 0.0;
        else
            for (int d = 0; d < 3; ++d) W[p * 3 + d] = 0.0;
    };
    if (v[0] == 0) {
        degenerate();
        return;
    }
    for (int d = 0; d < D; ++d) U[p * D + d] = Su[d] / cnt;
    const double Lv[3] = {Sl[0] - (phi[1] * Su[2] - phi[2] * Su[1]), Sl[1] - (phi[2] * Su[0] - phi[0] * Su[2]),
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
        const double Izz = rr[0][0] + rr[1][1];
        if (!(Izz > 0.0)) {
            degenerate();
            return;
        }
        W[p] = Lv[2] / Izz;
        return;
    }
    const double tr = rr[0][0] + rr[1][1] + rr[2][2];
    double I[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) I[i][j] = (i == j ? tr : 0.0) - rr[i][j];
    const double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                       I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                       I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
    if (!(det > 0.0)) {  // I is positive semi-definite; singular for collinear node sets
        degenerate();
        return;
    }
    for (int col = 0; col < 3; ++col) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) M[r][q] = (q == col) ? Lv[r] : I[r][q];
        const double dc = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                          M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                          M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        W[p * 3 + col] = dc / det;
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
std::mutex g_na_mutex;
long long* g_na_ptr[256] = {nullptr};

long long* scratch_address(int dev, cudaError_t* err) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (dev < 0 || dev >= 256) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_na_ptr[dev] = static_cast<long long*>(p);
    }
    *err = cudaSuccess;
    return g_na_ptr[dev];
}

}  // namespace
}  // namespace lbmpen

using namespace lbmpen;

extern "C" int lbm_rigid_projection_noalloc(int dim, const int* n, const int* periodic, const float* u,
                                            int np, const double* pos, const double* radius,
                                            double max_radius, double* vel, double* omega,
                                            int* count, void* stream) {
    if ((dim != 2 && dim != 3) || !n || !periodic || np < 0) return LBM_ERR_INVALID;
    if (np > NA_MAXP) return LBM_ERR_INVALID;  // beyond the fixed scratch array
    if (np == 0) return LBM_OK;
    if (!u || !pos || !radius || !vel || !omega || !count) return LBM_ERR_INVALID;
    if (!(max_radius >= 0.0) || max_radius > (dim == 3 ? MAX_RADIUS_3D : MAX_RADIUS)) return LBM_ERR_INVALID;
    NaGrid g;
    g.D = dim;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = d < dim ? n[d] : 1;
        g.per[d] = d < dim ? (periodic[d] != 0) : 1;
        if (g.n[d] < 1) return LBM_ERR_INVALID;
        // a particle's box must not wrap onto itself on a periodic axis
        if (d < dim && g.per[d] && (long long)(2.0 * max_radius) + 4 > g.n[d]) return LBM_ERR_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ERR_CUDA;
    cudaError_t e;
    long long* scratch = scratch_address(dev, &e);
    if (!scratch) return LBM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_na_clear<<<(np * NPV + 255) / 256, 256, 0, st>>>(scratch, np);
    const long long side = (long long)(2.0 * max_radius) + 4;
    const long long box = dim == 2 ? side * side : side * side * side;
    const dim3 grid((unsigned)np, (unsigned)((box + NA_BLOCK - 1) / NA_BLOCK));
    k_na_accumulate<<<grid, NA_BLOCK, 0, st>>>(g, u, np, pos, radius, max_radius, scratch);
    k_na_finalize<<<(np + 127) / 128, 128, 0, st>>>(dim, np, pos, scratch, vel, omega, count);
    if ((e = cudaGetLastError()) != cudaSuccess) return LBM_ERR_CUDA;
    long long err = 0;
    if (cudaMemcpyAsync(&err, scratch + NA_ERR, sizeof err, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (err & 1) return LBM_ERR_INVALID;   // a radius above max_radius
    if (err & 4) return LBM_ERR_DIVERGED;  // a velocity component is non-finite or |u| >= 1/2
    if (err & 2) return LBM_ERR_CAPACITY;  // a particle overlaps more than 64 of lower index
    if (err & 8) return LBM_ERR_PARTICLE;  // a particle owns no node, or its nodes have no inertia
    return LBM_OK;
}
