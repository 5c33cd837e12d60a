// hram_capi.cu -- step engine and C-ABI of the B300 planar WCSPH
// hydrodynamic-ram library (declarations and documentation in hram.h).
//
// A case owns (or borrows) one device workspace carved into the buffers of
// hram_device.cuh.  hr_init_case builds the static ghost geometry on the host
// in FP64, uploads it, evaluates the initial state (a "prime" pass: the step
// kernels with dt = 0), and captures one step as a CUDA graph on a private
// stream; hr_step replays that graph on the caller's stream.
#include "hram_device.cuh"
#include "hram_tangent.cuh"
#include "hram_adjoint.cuh"
#include "hram_n3.cuh"
#include "hram_persist.h"
#include "hram.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace {
// A named NVTX range over one C-ABI call (a profiler's timeline shows the
// library's calls; the kernels inside carry their own names).  Without a
// tool attached the push and pop are no-ops.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

using namespace hr;

namespace {

constexpr int kDiagFields = 19;
constexpr int kDiagThreads = 1024;
constexpr int kTimingEvents = 6;
// steps per graph launch in hr_run: a small case's step is bound by the
// latency of its launches, and one graph of several steps leaves out the gaps
// between graph launches
constexpr int kMultiSteps = 4;
// the split interaction pass: on by default from this many fluid particles
// (below it the step is bound by its kernels' latency, and the boundary
// particles are too large a share to hide); grid of its boundary kernels
// (grid-stride over their lists)
constexpr long long kSplitMinParticles = 262144;
constexpr int kSplitBlocks = 592;
constexpr int kSplitListBlocks = 296;   // extra blocks of the ghost launch

// ------------------------------------------------ auxiliary device kernels

// Specific Tait elastic energy e(rho) (reading R18) divided by B / rho0,
// written in the deviation d without cancellation: for gamma = 7,
// ((1+d)^6 - 1)/6 + 1/(1+d) - 1 = d^2/(1+d) + 5/2 d^2 + 10/3 d^3 + 5/2 d^4 + d^5 + d^6/6.
__device__ __forceinline__ float tait_energy_scaled(const Consts &K, float d)
{
    if (K.gamma7) {
        float poly = fmaf(d, 1.0f / 6.0f, 1.0f);
        poly = fmaf(d, poly, 2.5f);
        poly = fmaf(d, poly, 10.0f / 3.0f);
        poly = fmaf(d, poly, 2.5f);
        return d * d * (poly + 1.0f / (1.0f + d));
    }
    const float g = K.gamma;
    return expm1f((g - 1.0f) * log1pf(d)) / (g - 1.0f) - d / (1.0f + d);
}

// FP64 diagnostics, stage 1: per-particle terms in FP32, sums across a warp
// in FP32 and across the block's warps in FP64 (per-block partial).
// partial layout (16 doubles): px, py, KE, PE, E_el, rho_min, rho_max, p_min,
// p_max, vmax, n_in, penetrated, (unused x4)
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(Consts K, Bufs B, double *part)
{
    __shared__ float sm[kDiagThreads / 32][12];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float v[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 3e38f, -3e38f, 3e38f, -3e38f, 0.f, 0.f, 0.f};
    if (i < K.nf) {
        const float2 r = B.s_pos[i];
        if (!outside_box(K, r.x, r.y)) {
            const float2 u = B.st_vel[i];
            const float d = B.st_rho[i];
            const float v2 = u.x * u.x + u.y * u.y;
            v[0] = K.m * u.x;
            v[1] = K.m * u.y;
            v[2] = 0.5f * K.m * v2;
            v[3] = -K.m * (K.gx * r.x + K.gy * r.y);
            if (K.closure == 1) {
                // the internal energy of the energy equation
                const float e = B.st_D[i].y;
                v[4] = K.m * e;
                v[7] = v[8] = mg_p(K, d, e);
            } else {
                v[4] = K.m * (K.B / K.rho0) * tait_energy_scaled(K, d);
                v[7] = v[8] = tait_p(K, d);
            }
            v[5] = v[6] = K.rho0 * (1.0f + d);
            v[9] = sqrtf(v2);
            v[10] = 1.0f;
            const float dx = r.x - B.S->xc_f, dy = r.y - B.S->yc_f;
            v[11] = (K.ng > 0 && dx * dx + dy * dy < K.R2) ? 1.0f : 0.0f;
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float b = __shfl_xor_sync(0xffffffffu, a, o);
            if (k == 5 || k == 7) a = fminf(a, b);
            else if (k == 6 || k == 8 || k == 9) a = fmaxf(a, b);
            else a += b;
        }
        if (lane == 0) sm[w][k] = a;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        const int k = threadIdx.x;
        double a = sm[0][k];
        for (int q = 1; q < kDiagThreads / 32; ++q) {
            const double b = sm[q][k];
            if (k == 5 || k == 7) a = fmin(a, b);
            else if (k == 6 || k == 8 || k == 9) a = fmax(a, b);
            else a += b;
        }
        part[(size_t)blockIdx.x * 16 + k] = a;
    }
}

// Stage 2 (one block): reduce the partials in block order and write an
// hr_diag record (19 doubles) to out[0] and, when rec >= 0, to hist[rec].
__global__ void k_diag_final(Consts K, Bufs B, const double *part, int nblocks, double *out,
                             double *hist, long long rec, long long hist_cap)
{
    if (threadIdx.x != 0) return;
    double a[12] = {0, 0, 0, 0, 0, 1e300, -1e300, 1e300, -1e300, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 12; ++k) {
            const double x = part[(size_t)b * 16 + k];
            if (k == 5 || k == 7) a[k] = fmin(a[k], x);
            else if (k == 6 || k == 8 || k == 9) a[k] = fmax(a[k], x);
            else a[k] += x;
        }
    const Scalars *S = B.S;
    double d[kDiagFields] = {(double)K.nf * (double)K.m, a[0], a[1], a[2], a[3], a[4], a[5],
                             a[6], a[7], a[8], a[9], a[10], a[11], S->t, S->dt, S->Wb,
                             S->impulse, S->diss, (double)S->step};
    for (int k = 0; k < kDiagFields; ++k) out[k] = d[k];
    if (rec >= 0 && rec < hist_cap)
        for (int k = 0; k < kDiagFields; ++k) hist[(size_t)rec * kDiagFields + k] = d[k];
}

// Uploaded densities -> deviations d = rho / rho0 - 1 (FP64, rounded once),
// and the identity order of the fluid IDs.
__global__ void k_upload_fix(Consts K, Bufs B, const float *rho, double rho0)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    if (rho) B.st_rho[i] = (float)((double)rho[i] / rho0 - 1.0);
    B.s_id[i] = i;
}

// Sorted state -> fluid-ID order.
__global__ void k_unsort(Consts K, Bufs B, float2 *xy, float2 *vel, float *rho, float *p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    const int id = B.s_id[i];
    const float d = B.st_rho[i];
    xy[id] = B.s_pos[i];
    vel[id] = B.st_vel[i];
    rho[id] = K.rho0 * (1.0f + d);
    p[id] = K.closure == 1 ? mg_p(K, d, B.st_D[i].y) : tait_p(K, d);
}

// Sorted internal energy and its rate -> fluid-ID order (closure 1).
__global__ void k_unsort_energy(Consts K, Bufs B, float *e, float *de)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    const int id = B.s_id[i];
    const float2 D = B.st_D[i];
    e[id] = D.y;
    de[id] = D.x;
}

// Debug neighbour enumeration with the same candidate loops and predicate
// as k_ghost and k_pass.  Row r of the output (global point order: fluid by
// slot, then wall ghosts by sorted index, then disk ghosts): count[r] when
// ids == nullptr, else the neighbours' global IDs at off[r].
__global__ void k_neighbors(Consts K, Bufs B, int *count, const long long *off, int *ids)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int npts = K.nf + K.nw + K.ng;
    if (r >= npts) return;
    long long pos = ids ? off[r] : 0;
    int n = 0;
    auto emit = [&](int gid) {
        if (ids) ids[pos + n] = gid;
        ++n;
    };
    if (r < K.nf) {
        const float2 ri = B.s_pos[r];
        if (!outside_box(K, ri.x, ri.y)) {
            const int c = cell_of(K, ri.x, ri.y);
            for_fluid_candidates(K, B.cell_start, c, K.nf, &B.S->status, [&](int j) {
                const float2 rj = B.s_pos[j];
                if (j != r && in_support(ri.x, ri.y, rj.x, rj.y, K.s2)) emit(B.s_id[j]);
            });
            if (K.nw > 0)
                for_fluid_candidates(K, B.wall_start, c, K.nw, &B.S->status, [&](int k) {
                    const float2 rg = B.gw_pos[k];
                    if (in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) emit(K.nf + B.gw_id[k]);
                });
            if (K.ng > 0 && near_disk(K, ri.x, ri.y, (float)B.S->xc, (float)B.S->yc))
                for (int k = 0; k < K.ng; ++k) {
                    const float2 rg = B.gd_pos[k];
                    if (!outside_box(K, rg.x, rg.y) && in_support(ri.x, ri.y, rg.x, rg.y, K.s2))
                        emit(K.nf + K.nw + k);
                }
        }
    } else {
        const int g = r - K.nf;
        const float2 rg = g < K.nw ? B.gw_pos[g] : B.gd_pos[g - K.nw];
        if (!outside_box(K, rg.x, rg.y)) {
            const int c = cell_of(K, rg.x, rg.y);
            for_fluid_candidates(K, B.cell_start, c, K.nf, &B.S->status, [&](int j) {
                const float2 rj = B.s_pos[j];
                if (in_support(rg.x, rg.y, rj.x, rj.y, K.s2)) emit(B.s_id[j]);
            });
        }
    }
    if (!ids) count[r] = n;
}

// Wall-ghost cell keys with the device's own cell arithmetic.
__global__ void k_wall_keys(Consts K, const float2 *pos, int n, int *key)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) key[k] = cell_of(K, pos[k].x, pos[k].y);
}

// Fixed device scratch of hr_neighbor_counts_static: one count per point,
// written by global point index.  Host code must not take its address
// directly; it uses the per-device address from cudaGetSymbolAddress.
__device__ __align__(256) int g_static_neighbor_counts[HR_STATIC_NEIGHBOR_MAX];

// FP32 FMA rate of the device (hr_fp32_rate): every thread runs 16
// independent FMA chains for iters iterations, as scalar fma.rn.f32 or as
// eight packed fma.rn.f32x2 pairs; the chains' sums are stored so none of it
// is dead code.
constexpr int kFmaChains = 16;
__global__ void __launch_bounds__(256) k_fma_rate(float *out, int iters, int packed)
{
    float v[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) v[k] = threadIdx.x * 1e-6f + k * 1e-3f;
    const float b = 0.999999f, c = 1e-7f;
    if (packed) {
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kFmaChains; k += 2) {
                const float2 r = p2_fma(make_float2(v[k], v[k + 1]), make_float2(b, b),
                                        make_float2(c, c));
                v[k] = r.x;
                v[k + 1] = r.y;
            }
        }
    } else {
#pragma unroll 4
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kFmaChains; ++k) v[k] = fmaf(v[k], b, c);
        }
    }
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) sum += v[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// Count-only variant of k_neighbors that writes by global point index (fluid
// ID, then wall-ghost ID, then disk ghost), so no host-side reordering is
// needed.  Same candidate loops and predicate.
__global__ void k_neighbor_counts_static(Consts K, Bufs B, int *counts)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int npts = K.nf + K.nw + K.ng;
    if (r >= npts) return;
    int n = 0;
    int gid;
    if (r < K.nf) {
        gid = B.s_id[r];
        const float2 ri = B.s_pos[r];
        if (!outside_box(K, ri.x, ri.y)) {
            const int c = cell_of(K, ri.x, ri.y);
            for_fluid_candidates(K, B.cell_start, c, K.nf, &B.S->status, [&](int j) {
                const float2 rj = B.s_pos[j];
                if (j != r && in_support(ri.x, ri.y, rj.x, rj.y, K.s2)) ++n;
            });
            if (K.nw > 0)
                for_fluid_candidates(K, B.wall_start, c, K.nw, &B.S->status, [&](int k) {
                    const float2 rg = B.gw_pos[k];
                    if (in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) ++n;
                });
            if (K.ng > 0 && near_disk(K, ri.x, ri.y, (float)B.S->xc, (float)B.S->yc))
                for (int k = 0; k < K.ng; ++k) {
                    const float2 rg = B.gd_pos[k];
                    if (!outside_box(K, rg.x, rg.y) && in_support(ri.x, ri.y, rg.x, rg.y, K.s2))
                        ++n;
                }
        }
    } else {
        const int g = r - K.nf;
        gid = g < K.nw ? K.nf + B.gw_id[g] : r;
        const float2 rg = g < K.nw ? B.gw_pos[g] : B.gd_pos[g - K.nw];
        if (!outside_box(K, rg.x, rg.y)) {
            const int c = cell_of(K, rg.x, rg.y);
            for_fluid_candidates(K, B.cell_start, c, K.nf, &B.S->status, [&](int j) {
                const float2 rj = B.s_pos[j];
                if (in_support(rg.x, rg.y, rj.x, rj.y, K.s2)) ++n;
            });
        }
    }
    counts[gid] = n;
}

constexpr int kMaxDevices = 64;
std::atomic<int *> g_static_counts_ptr[kMaxDevices] = {};
std::mutex g_static_counts_mutex;

// Device address of g_static_neighbor_counts on device dev (which must be
// the current device), looked up once per device.  Two host threads making
// their first call at the same time serialise on the mutex; later calls read
// the published address without locking.
int static_counts_address(int dev, int **out)
{
    if (dev < 0 || dev >= kMaxDevices) return HR_ECUDA;
    int *p = g_static_counts_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_static_counts_mutex);
        p = g_static_counts_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_static_neighbor_counts) != cudaSuccess || !ptr)
                return HR_ECUDA;
            p = static_cast<int *>(ptr);
            g_static_counts_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return HR_OK;
}

// ------------------------------------------------------------ host helpers

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t total = 0;
    size_t add(size_t bytes)
    {
        const size_t off = total;
        total += align256(bytes > 0 ? bytes : 1);
        return off;
    }
};

struct Geometry {
    std::vector<double> wx, wy, wnx, wny;
    std::vector<int> wkind;
};

// Wall ghosts in wall-ID order: lower band (layer-major), upper band, then
// with closed ends the left and right bands.  Layer k at W/2 + (k - 1/2) dx.
Geometry make_walls(const hr_params &P)
{
    Geometry G;
    const int L = P.wall_layers;
    if (L <= 0) return G;
    const long long nx = llround(P.Lx / P.dx), ny = llround(P.W / P.dx);
    const long long i0 = P.end_walls ? -L : 0, i1 = nx + (P.end_walls ? L : 0);
    for (int band = 0; band < 2; ++band)
        for (int k = 1; k <= L; ++k)
            for (long long i = i0; i < i1; ++i) {
                G.wx.push_back(((double)i + 0.5) * P.dx);
                G.wy.push_back(band == 0 ? -0.5 * P.W - ((double)k - 0.5) * P.dx
                                         : 0.5 * P.W + ((double)k - 0.5) * P.dx);
                G.wnx.push_back(0.0);
                G.wny.push_back(band == 0 ? -1.0 : 1.0);
                G.wkind.push_back(KIND_SIDE);
            }
    if (P.end_walls)
        for (int band = 0; band < 2; ++band)
            for (int k = 1; k <= L; ++k)
                for (long long j = 0; j < ny; ++j) {
                    G.wx.push_back(band == 0 ? -((double)k - 0.5) * P.dx
                                             : P.Lx + ((double)k - 0.5) * P.dx);
                    G.wy.push_back(-0.5 * P.W + ((double)j + 0.5) * P.dx);
                    G.wnx.push_back(band == 0 ? -1.0 : 1.0);
                    G.wny.push_back(0.0);
                    G.wkind.push_back(KIND_END);
                }
    return G;
}

int validate(const hr_params *P, long long nf)
{
    if (!P || nf <= 0 || nf > (1LL << 30)) return HR_EINVAL;
    if (!(P->dx > 0) || !(P->h_over_dx > 0) || !(P->Lx > 0) || !(P->W > 0)) return HR_EINVAL;
    if (P->wall_layers < 0 || P->wall_layers > 8 || P->Ng < 0 || P->Ng > 1024) return HR_EINVAL;
    if (P->n_probes < 0 || P->n_probes > HR_MAX_PROBES) return HR_EINVAL;
    if (!(P->rho0 > 0) || !(P->c0 > 0) || !(P->gamma > 1) || !(P->cfl > 0)) return HR_EINVAL;
    if (!(P->rho_lo > 0) || !(P->rho_hi > P->rho_lo)) return HR_EINVAL;
    if (P->motion < 0 || P->motion > 3 || P->dt_mode < 0 || P->dt_mode > 1) return HR_EINVAL;
    if (P->motion == 3 && !(P->disk_density > 0)) return HR_EINVAL;
    if (P->motion == 1 && !(P->drag_M > 0)) return HR_EINVAL;
    if (P->Ng > 0 && !(P->R_disk > 0)) return HR_EINVAL;
    if (!(P->cell_factor >= 0.5)) return HR_EINVAL;
    if ((P->flags & HR_FLAG_STAGE_POS) && (P->flags & HR_FLAG_STAGE_ALL)) return HR_EINVAL;
    // one pass variant at a time
    {
        const int v = P->flags & (HR_FLAG_STAGE_POS | HR_FLAG_STAGE_ALL | HR_FLAG_NEWTON3 |
                                  HR_FLAG_PASS_LANES2 | HR_FLAG_PASS_LANES4);
        if (v & (v - 1)) return HR_EINVAL;
        if ((P->flags & (HR_FLAG_PASS_LANES2 | HR_FLAG_PASS_LANES4)) &&
            (P->cell_factor < 1.0 || (P->flags & HR_FLAG_TANGENT)))
            return HR_EINVAL;
    }
    // the Newton-3 pass: closure 0, the 3 x 3 stencil, no other pass variant
    if ((P->flags & HR_FLAG_NEWTON3) &&
        (P->closure != 0 || P->cell_factor < 1.0 ||
         (P->flags & (HR_FLAG_TANGENT | HR_FLAG_STAGE_POS | HR_FLAG_STAGE_ALL))))
        return HR_EINVAL;
    // cells of side < 2h (5 x 5 stencil): the plain and batched steps only
    if (P->cell_factor < 1.0 &&
        (P->flags & (HR_FLAG_TANGENT | HR_FLAG_STAGE_POS | HR_FLAG_STAGE_ALL)))
        return HR_EINVAL;
    // the split pass: the plain 3 x 3 pass only
    if ((P->flags & HR_FLAG_PASS_SPLIT) &&
        ((P->flags & (HR_FLAG_PASS_FUSED | HR_FLAG_TANGENT | HR_FLAG_STAGE_POS | HR_FLAG_STAGE_ALL |
                      HR_FLAG_NEWTON3 | HR_FLAG_PASS_LANES2 | HR_FLAG_PASS_LANES4)) ||
         P->cell_factor < 1.0))
        return HR_EINVAL;
    // tangent mode: fixed time step (smooth in c0) and a prescribed motion
    if ((P->flags & HR_FLAG_TANGENT) && (P->dt_mode != 1 || P->motion > 2)) return HR_EINVAL;
    if (P->closure < 0 || P->closure > 1) return HR_EINVAL;
    if (P->wall_reflect < 0 || P->wall_reflect > 1) return HR_EINVAL;
    if (P->closure == 1) {
        if ((P->flags & HR_FLAG_TANGENT) || !(P->mg_mu_max > 0)) return HR_EINVAL;
        // the Hugoniot denominator 1 - (S1 - 1) mu must stay positive up to the cap
        if (!((P->mg_S1 - 1.0) * P->mg_mu_max < 1.0)) return HR_EINVAL;
    }
    return HR_OK;
}

}  // namespace

// -------------------------------------------------------------- the case

struct hr_case {
    hr_params P;
    Consts K;
    Bufs B;
    long long nf = 0, nw = 0, ng = 0;
    int device = -1;  // the CUDA device current at hr_init_case
    int n_tiles = 0, pass_blocks = 0, ghost_blocks = 0, drift_blocks = 0, diag_blocks = 0;
    int tghost_blocks = 0;   // blocks of the tangent ghost kernel (one warp per ghost)
    cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // kMultiSteps steps in one graph, for hr_run (absent with HR_FLAG_TIMING)
    cudaGraph_t graph_multi = nullptr;
    cudaGraphExec_t exec_multi = nullptr;
    cudaEvent_t ev[kTimingEvents] = {};
    bool timing = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    // host copies / extra device buffers
    std::vector<int> wall_id_of_sorted;
    std::vector<float> wall_xy_sorted;
    double *diag_part = nullptr, *diag_out = nullptr, *diag_hist = nullptr;
    long long diag_cap = 0, diag_rec = 0;
    float *io = nullptr;  // nf x 6 floats for state transfers
    long long host_step = 0;
    int sticky = 0;
    // reverse mode (hr_adjoint_forward / hr_adjoint_backward)
    struct AdjCtx *adj = nullptr;
    // tangent mode (HR_FLAG_TANGENT)
    bool tangent = false;
    int stage = 0;                // pass variant: 0 global loads, 1/2 staged candidates
    bool n3 = false;              // pass variant: each fluid pair evaluated once
    int lanes = 1;                // pass variant: lanes per particle
    int split_blocks = 0;         // blocks of the split pass's boundary kernels
    cudaEvent_t fork2 = nullptr, join2 = nullptr;   // the split pass's ghost branch
    // the deferred step close: the step graphs leave each step's close to run
    // beside the next step's drift (defer), and the host settles a pending
    // one (settle) before it reads or hands on the case
    bool defer = false;
    bool pending = false;
    int prio_hi = 0;              // the device's greatest stream priority (that branch's)
    TBufs T{};
    int tpass_blocks = 0;
    void *t_base = nullptr;
    size_t t_bytes = 0;
};

struct hr_batch {
    std::vector<hr_case *> cases;
    cudaStream_t stream = nullptr, cap = nullptr, cap2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *mem = nullptr;
    Consts *dK = nullptr;
    Bufs *dB = nullptr;
    int *d_count = nullptr;
    BatchBlock *map[10] = {};
    int nblocks[10] = {};
    int closure = 0;  // shared by every case of the batch
    long long steps = 0;
    // the persistent form (hr_batch_create_persistent): one launch, each case
    // on its own fixed blocks, per-case barriers with bounded waits
    bool persistent = false;
    int2 *blk = nullptr;        // per block: (case, rank in the case)
    int *case_nblk = nullptr;   // per case: blocks
    int *bar = nullptr;         // per case: barrier counter and generation
    int *err = nullptr;         // set by a wait that ran past spin_limit
    int nblk_total = 0;
    long long spin_limit = 0;
};

namespace {

// Derived constants (FP64 on the host, then rounded once).
void make_consts(hr_case *c)
{
    const hr_params &P = c->P;
    Consts &K = c->K;
    std::memset(&K, 0, sizeof K);
    const double h = P.h_over_dx * P.dx;
    const double s = 2.0 * h;
    // cells of side >= 2h take the 3 x 3 stencil; side in [h, 2h) the 5 x 5
    K.sr = P.cell_factor < 1.0 ? 2 : 1;
    const double dc = K.sr == 2 ? s * std::max(P.cell_factor, 0.5005)
                                : s * std::max(P.cell_factor, 1.001);
    double padx, pady;
    if (P.box_pad > 0.0) {
        padx = pady = P.box_pad;
    } else {
        padx = 0.5 * P.Lx;
        pady = P.wall_layers > 0 ? (P.wall_layers + 2) * P.dx + s : 0.5 * P.W;
        if (P.end_walls && P.wall_layers > 0) padx = (P.wall_layers + 2) * P.dx + s;
    }
    const double xlo = -padx, xhi = P.Lx + padx, ylo = -0.5 * P.W - pady, yhi = 0.5 * P.W + pady;
    // sr cells of margin on every side, so a stencil never leaves the grid
    K.x0 = (float)(xlo - K.sr * dc);
    K.y0 = (float)(ylo - K.sr * dc);
    K.inv_dc = (float)(1.0 / dc);
    K.ncx = (int)std::floor((xhi - xlo) / dc) + 1 + 2 * K.sr;
    K.ncy = (int)std::floor((yhi - ylo) / dc) + 1 + 2 * K.sr;
    K.ncell = K.ncx * K.ncy;
    K.xlo = (float)xlo;
    K.xhi = (float)xhi;
    K.ylo = (float)ylo;
    K.yhi = (float)yhi;
    K.W2 = (float)(0.5 * P.W);
    K.Lx = (float)P.Lx;
    K.side_walls = P.wall_layers > 0 || P.wall_reflect == 1;
    K.end_walls = P.end_walls && P.wall_layers > 0;
    const double ad = 7.0 / (4.0 * M_PI * h * h);
    K.h = (float)h;
    K.s2 = (float)(s * s);
    K.half_inv_h = (float)(0.5 / h);
    K.two_inv_h = (float)(2.0 / h);
    K.Wc = (float)ad;
    K.Fc = (float)(-5.0 * ad / (h * h));
    K.m = (float)(P.rho0 * P.dx * P.dx);
    K.rho0 = (float)P.rho0;
    K.inv_rho0 = (float)(1.0 / P.rho0);
    K.B = (float)(P.rho0 * P.c0 * P.c0 / P.gamma);
    K.c0 = (float)P.c0;
    K.p_cav = (float)std::max(P.p_cav, -1e30);
    K.alpha_h = (float)(P.alpha * h);
    K.alpha_f = (float)P.alpha;
    K.eh2 = (float)(P.eta2 * h * h);
    K.nu4 = (float)(4.0 * P.mu_lam / P.rho0);
    K.eps_xsph = (float)P.eps_xsph;
    K.gx = (float)P.gx;
    K.gy = (float)P.gy;
    K.d_lo = (float)(P.rho_lo - 1.0);
    K.d_hi = (float)(P.rho_hi - 1.0);
    K.gamma = (float)P.gamma;
    K.half_gm1 = (float)(0.5 * (P.gamma - 1.0));
    K.inv_rho0c02 = (float)(1.0 / (P.rho0 * P.c0 * P.c0));
    K.gamma7 = P.gamma == 7.0;
    K.nf = (int)c->nf;
    K.nw = (int)c->nw;
    K.ng = (int)c->ng;
    K.m_wall = (float)(P.rho0 * P.dx * P.dx);
    K.m_disk = P.Ng > 0 ? (float)(P.rho0 * P.dx * (2.0 * M_PI * P.R_disk / (double)P.Ng)) : 0.f;
    K.wall_over_m = 1.0f;
    K.disk_over_m = P.Ng > 0 ? (float)(P.dx * (2.0 * M_PI * P.R_disk / (double)P.Ng) /
                                       (P.dx * P.dx))
                             : 0.f;
    K.m_over_rho0 = (float)(P.dx * P.dx);
    K.m2Wc = (float)(-2.0 * ad);
    K.R = (float)P.R_disk;
    K.R2 = (float)(P.R_disk * P.R_disk);
    const double reach = P.R_disk + 1.02 * s;
    K.disk_reach2 = (float)(reach * reach);
    K.ng_over_2pi = (float)((double)c->ng / (2.0 * M_PI));
    K.cfl_h = P.cfl * h;
    K.cfl_h_f = (float)K.cfl_h;
    K.dt_fixed = K.cfl_h / (P.c0 + P.v0);
    K.disk_mass = P.disk_density * M_PI * P.R_disk * P.R_disk;
    K.c0d = P.c0;
    K.v0 = P.v0;
    K.tau = P.tau;
    K.t_ramp = P.t_ramp;
    K.x_c0 = P.x_c0;
    K.y_c0 = P.y_c0;
    K.a_const = P.a_const;
    K.drag_k = P.motion == 1 ? P.drag_Cd * P.rho0 * M_PI * P.drag_R * P.drag_R / (2.0 * P.drag_M)
                             : 0.0;
    K.dt_mode = P.dt_mode;
    K.motion = P.motion;
    // motion 0 (ramp, then exponential decay with tau > 0): after the ramp
    // x(t) = x_c0 + (v0/t_r)(tau^2 - tau (t_r + tau) E) + v0 tau (E - e(t)),
    // E = exp(-t_r/tau), e(t) = exp(-t/tau) (without a ramp: x_c0 + v0 tau (1 - e))
    K.m2d = (double)K.m * (double)K.m;
    K.kin_fast = P.motion == 0 && P.tau > 0.0 ? 1 : 0;
    if (K.kin_fast) {
        const double tr = P.t_ramp > 0.0 ? P.t_ramp : 0.0, tau = P.tau;
        const double E = tr > 0.0 ? std::exp(-tr / tau) : 1.0;
        K.kin_inv_tau = 1.0 / tau;
        K.kin_q = P.v0 * tau;
        K.kin_x1 = P.x_c0 + (tr > 0.0 ? (P.v0 / tr) * (tau * tau - tau * (tr + tau) * E) : 0.0) +
                   K.kin_q * E;
    } else {
        K.kin_inv_tau = K.kin_x1 = K.kin_q = 0.0;
    }
    K.n_probes = P.n_probes;
    for (int k = 0; k < P.n_probes; ++k) {
        K.probe_x[k] = (float)P.probe_xy[2 * k];
        K.probe_y[k] = (float)P.probe_xy[2 * k + 1];
    }
    K.probe_cap = P.probe_capacity > 0 ? P.probe_capacity : (1LL << 16);
    c->drift_blocks = (int)((c->nf + 255) / 256);
    c->pass_blocks = (int)((c->nf + kPassThreads - 1) / kPassThreads);
    c->ghost_blocks =
        (int)std::max<long long>(1, (c->nw + c->ng + kGhostsPerBlock - 1) / kGhostsPerBlock);
    c->tghost_blocks = (int)std::max<long long>(1, (c->nw + c->ng + kGhostWarps - 1) / kGhostWarps);
    c->n_tiles = (K.ncell + 2 + kScanTile - 1) / kScanTile;
    c->diag_blocks = (int)((c->nf + kDiagThreads - 1) / kDiagThreads);
    c->tpass_blocks = (int)((c->nf + kTPassThreads - 1) / kTPassThreads);
    K.n3 = (P.flags & HR_FLAG_NEWTON3) ? 1 : 0;
    c->lanes = (P.flags & HR_FLAG_PASS_LANES4) ? 4 : (P.flags & HR_FLAG_PASS_LANES2) ? 2 : 1;
    if (c->lanes > 1)   // kPassThreads / lanes particles per pass block
        c->pass_blocks = (int)((c->nf * c->lanes + kPassThreads - 1) / kPassThreads);
    if (K.n3) {
        // row chunks of kN3Threads particles: at most one partial chunk per row
        c->pass_blocks = (int)((c->nf + kN3Threads - 1) / kN3Threads) + K.ncy + 1;
        K.n3_tiles_max = c->pass_blocks;
    }
    // the split pass (interior particles beside the ghost pass): large
    // cases with the plain 3 x 3 pass, unless asked for or refused
    {
        const int variants = HR_FLAG_TANGENT | HR_FLAG_STAGE_POS | HR_FLAG_STAGE_ALL | HR_FLAG_NEWTON3 |
                             HR_FLAG_PASS_LANES2 | HR_FLAG_PASS_LANES4 | HR_FLAG_PASS_FUSED;
        const bool plain = K.sr == 1 && !(P.flags & variants) && c->nw + c->ng > 0;
        K.split = plain && ((P.flags & HR_FLAG_PASS_SPLIT) || c->nf >= kSplitMinParticles) ? 1 : 0;
    }
    c->split_blocks = std::max(1, std::min(c->pass_blocks, kSplitBlocks));
    K.n_pass_blocks = c->pass_blocks;
    K.n_ghost_blocks = c->ghost_blocks;
    K.closure = P.closure;
    const double sd = 10.0 / (7.0 * M_PI * h * h);
    K.cub_sd = (float)sd;
    K.cub_Fc = (float)(sd / (h * h));
    K.inv_h = (float)(1.0 / h);
    K.self_w = (float)(P.dx * P.dx * sd);
    K.c_av = (float)(-P.alpha * h * P.c0);
    K.mg_K = (float)(P.rho0 * P.c0 * P.c0);
    K.mg_k1 = (float)(1.0 - 0.5 * P.mg_gamma0);
    K.mg_s1m1 = (float)(P.mg_S1 - 1.0);
    K.mg_g0 = (float)P.mg_gamma0;
    K.mg_a = (float)P.mg_a;
    K.mg_mu_max = (float)P.mg_mu_max;
}

struct Offsets {
    size_t s_pos, s_vel, s_aux, s_rd, s_id, st_vel, st_rho, st_a, st_D, st_X, u_pos, u_vel,
        u_id, u_key, cell_count, cell_start, tile_sum, bucket, ovf, ovf_count, perm_tmp, gw_pos, gw_nrm,
        gw_kind, gw_id, wall_start, disk_off, gd_pos, g_vel, g_aux, ghost_vmax, pass_part,
        probe_now, probe_hist, probe_t, S, diag_part, diag_out, diag_hist, io, part_vmax, part_npen, part_w,
        fin_part, fin_vmax, fin_npen, fin_ticket;
    size_t s_ex;  // closure 1 only
    size_t n3_row_base, n3_tile_row, n3_info, n3_flag, n3_ext_a, n3_ext_b, n3_ctl;  // Newton-3 only
    size_t wall_near;
    size_t split_n, split_pi, split_bi, split_mask, split_pf, split_pv, split_part, split_vmax,
        split_npen;  // the split pass only
    // tangent arrays (zero-sized unless HR_FLAG_TANGENT)
    size_t t_begin, t_s_pos, t_s_vel, t_s_aux, t_s_rd, t_st_vel, t_st_rho, t_st_a, t_st_D, t_st_X,
        t_u_pos, t_u_vel, t_g_vel, t_g_aux, t_perm, t_part, t_sc, t_end;
    size_t total;
};

Offsets plan(const hr_case *c)
{
    const Consts &K = c->K;
    const size_t n = (size_t)c->nf, ng = (size_t)(c->nw + c->ng), nc = (size_t)K.ncell;
    Layout L;
    Offsets o;
    o.s_pos = L.add((n + kPosPad) * 8);  // padded for the predicate's block reads
    o.s_vel = L.add(n * 8);
    o.s_aux = L.add(n * 16);
    o.s_rd = L.add(n * 8);
    o.s_id = L.add(n * 4);
    o.st_vel = L.add(n * 8);
    o.st_rho = L.add(n * 4);
    o.st_a = L.add(n * 8);
    o.st_D = L.add(n * 8);
    o.st_X = L.add(n * 8);
    o.u_pos = L.add(n * 8);
    o.u_vel = L.add(n * 8);
    o.u_id = L.add(n * 4);
    o.u_key = L.add(n * 4);
    o.cell_count = L.add((nc + 1) * 4);
    o.cell_start = L.add((nc + 2) * 4);
    o.tile_sum = L.add((size_t)c->n_tiles * 4);
    o.bucket = L.add((nc + 1) * kBucket * 4);
    o.ovf = L.add(n * 16);
    o.ovf_count = L.add(4);
    o.perm_tmp = L.add(n * 4);
    o.gw_pos = L.add((size_t)c->nw * 8);
    o.gw_nrm = L.add((size_t)c->nw * 8);
    o.gw_kind = L.add((size_t)c->nw * 4);
    o.gw_id = L.add((size_t)c->nw * 4);
    o.wall_start = L.add((nc + 1) * 4);
    o.disk_off = L.add((size_t)c->ng * 16);
    o.gd_pos = L.add((size_t)c->ng * 8);
    o.g_vel = L.add(ng * 8);
    o.g_aux = L.add(ng * 16);
    o.ghost_vmax = L.add((size_t)c->ghost_blocks * 4);
    o.pass_part = L.add((size_t)c->pass_blocks * 16);
    o.part_w = L.add(16);
    o.part_vmax = L.add((size_t)c->pass_blocks * 4);
    o.part_npen = L.add((size_t)c->pass_blocks * 4);
    o.probe_now = L.add(kMaxProbes * 4);
    o.probe_hist = L.add((size_t)K.probe_cap * (size_t)std::max(K.n_probes, 1) * 4);
    o.probe_t = L.add((size_t)K.probe_cap * 8);
    o.S = L.add(sizeof(Scalars));
    o.fin_part = L.add(kFinalizeBlocks * 8 * 4);
    o.fin_vmax = L.add(kFinalizeBlocks * 4);
    o.fin_npen = L.add(kFinalizeBlocks * 4);
    o.fin_ticket = L.add(4);
    o.diag_part = L.add((size_t)c->diag_blocks * 16 * 8);
    o.diag_out = L.add(kDiagFields * 8);
    const long long dcap = c->P.diag_every > 0 ? 4096 : 1;
    o.diag_hist = L.add((size_t)dcap * kDiagFields * 8);
    o.io = L.add(n * 6 * 4);
    o.s_ex = L.add(c->P.closure == 1 ? n * 16 : 0);
    {
        const size_t nt = K.n3 ? (size_t)K.n3_tiles_max : 0;
        o.n3_row_base = L.add(K.n3 ? ((size_t)K.ncy + 1) * 4 : 0);
        o.n3_tile_row = L.add(nt * 4);
        o.n3_info = L.add(nt * 16);
        o.n3_flag = L.add(nt * 4);
        o.n3_ext_a = L.add(nt * kN3ExtCap * 16);
        o.n3_ext_b = L.add(nt * kN3ExtCap * 4);
        o.n3_ctl = L.add(K.n3 ? 8 : 0);
    }
    o.wall_near = L.add(nc);
    {
        const size_t ns = K.split ? n : 0, nb = K.split ? (size_t)c->pass_blocks : 0;
        o.split_n = L.add(K.split ? 8 : 0);
        o.split_pi = L.add(ns * 4);
        o.split_bi = L.add(nb * 4);
        o.split_mask = L.add((nb + 31) / 32 * 4);
        o.split_pf = L.add(ns * 16);
        o.split_pv = L.add(ns * 8);
        o.split_part = L.add(nb * 16);
        o.split_vmax = L.add(nb * 4);
        o.split_npen = L.add(nb * 4);
    }
    const size_t tn = (c->P.flags & HR_FLAG_TANGENT) ? n * kDir : 0;
    const size_t tg = (c->P.flags & HR_FLAG_TANGENT) ? ng * kDir : 0;
    const bool tm = (c->P.flags & HR_FLAG_TANGENT) != 0;
    o.t_begin = L.total;
    o.t_s_pos = L.add(tn * 8);
    o.t_s_vel = L.add(tn * 8);
    o.t_s_aux = L.add(tn * 16);
    o.t_s_rd = L.add(tn * 8);
    o.t_st_vel = L.add(tn * 8);
    o.t_st_rho = L.add(tn * 4);
    o.t_st_a = L.add(tn * 8);
    o.t_st_D = L.add(tn * 8);
    o.t_st_X = L.add(tn * 8);
    o.t_u_pos = L.add(tn * 8);
    o.t_u_vel = L.add(tn * 8);
    o.t_g_vel = L.add(tg * 8);
    o.t_g_aux = L.add(tg * 16);
    o.t_perm = L.add(tm ? n * 4 : 0);
    o.t_part = L.add(tm ? (size_t)c->tpass_blocks * kDir * 4 : 0);
    o.t_sc = L.add(tm ? TSC_N * 8 : 0);
    o.t_end = L.total;
    o.total = L.total;
    return o;
}

template <class T>
T *at(void *base, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

void bind(hr_case *c, const Offsets &o)
{
    void *w = c->ws;
    Bufs &B = c->B;
    B.s_pos = at<float2>(w, o.s_pos);
    B.s_vel = at<float2>(w, o.s_vel);
    B.s_aux = at<float4>(w, o.s_aux);
    B.s_rd = at<float2>(w, o.s_rd);
    B.s_id = at<int>(w, o.s_id);
    B.st_vel = at<float2>(w, o.st_vel);
    B.st_rho = at<float>(w, o.st_rho);
    B.st_a = at<float2>(w, o.st_a);
    B.st_D = at<float2>(w, o.st_D);
    B.st_X = at<float2>(w, o.st_X);
    B.u_pos = at<float2>(w, o.u_pos);
    B.u_vel = at<float2>(w, o.u_vel);
    B.u_id = at<int>(w, o.u_id);
    B.u_key = at<int>(w, o.u_key);
    B.cell_count = at<int>(w, o.cell_count);
    B.cell_start = at<int>(w, o.cell_start);
    B.tile_sum = at<int>(w, o.tile_sum);
    B.bucket = at<int>(w, o.bucket);
    B.ovf = at<int4>(w, o.ovf);
    B.ovf_count = at<int>(w, o.ovf_count);
    B.perm_tmp = at<int>(w, o.perm_tmp);
    B.gw_pos = at<float2>(w, o.gw_pos);
    B.gw_nrm = at<float2>(w, o.gw_nrm);
    B.gw_kind = at<int>(w, o.gw_kind);
    B.gw_id = at<int>(w, o.gw_id);
    B.wall_start = at<int>(w, o.wall_start);
    B.disk_off = at<double2>(w, o.disk_off);
    B.gd_pos = at<float2>(w, o.gd_pos);
    B.g_vel = at<float2>(w, o.g_vel);
    B.g_aux = at<float4>(w, o.g_aux);
    B.ghost_vmax = at<float>(w, o.ghost_vmax);
    B.part.f = at<float4>(w, o.pass_part);
    B.part.vmax = at<float>(w, o.part_vmax);
    B.part.npen = at<int>(w, o.part_npen);
    B.probe_now = at<float>(w, o.probe_now);
    B.probe_hist = at<float>(w, o.probe_hist);
    B.probe_t = at<double>(w, o.probe_t);
    B.S = at<Scalars>(w, o.S);
    B.fin_part = at<float>(w, o.fin_part);
    B.fin_vmax = at<float>(w, o.fin_vmax);
    B.fin_npen = at<int>(w, o.fin_npen);
    B.fin_ticket = at<int>(w, o.fin_ticket);
    c->diag_part = at<double>(w, o.diag_part);
    c->diag_out = at<double>(w, o.diag_out);
    c->diag_hist = at<double>(w, o.diag_hist);
    c->diag_cap = c->P.diag_every > 0 ? 4096 : 1;
    c->io = at<float>(w, o.io);
    c->tangent = (c->P.flags & HR_FLAG_TANGENT) != 0;
    c->stage = (c->P.flags & HR_FLAG_STAGE_POS) ? 1 : (c->P.flags & HR_FLAG_STAGE_ALL) ? 2 : 0;
    // (the two-way coupled disk needs the close's force before its next
    // step; the tangent mode's close carries derivatives of the gate)
    c->defer = !(c->P.flags & HR_FLAG_CLOSE_INLINE) && !c->tangent && c->K.motion != 3;
    B.s_ex = c->P.closure == 1 ? at<float4>(w, o.s_ex) : nullptr;
    B.perm_dst = nullptr;
    c->n3 = c->K.n3 != 0;
    B.n3_row_base = c->n3 ? at<int>(w, o.n3_row_base) : nullptr;
    B.n3_tile_row = c->n3 ? at<int>(w, o.n3_tile_row) : nullptr;
    B.n3_info = c->n3 ? at<int4>(w, o.n3_info) : nullptr;
    B.n3_flag = c->n3 ? at<int>(w, o.n3_flag) : nullptr;
    B.n3_ext_a = c->n3 ? at<float4>(w, o.n3_ext_a) : nullptr;
    B.n3_ext_b = c->n3 ? at<float>(w, o.n3_ext_b) : nullptr;
    B.n3_ctl = c->n3 ? at<int>(w, o.n3_ctl) : nullptr;
    B.wall_near = at<unsigned char>(w, o.wall_near);
    const bool sp = c->K.split != 0;
    B.split_n = sp ? at<int>(w, o.split_n) : nullptr;
    B.split_pi = sp ? at<int>(w, o.split_pi) : nullptr;
    B.split_bi = sp ? at<int>(w, o.split_bi) : nullptr;
    B.split_mask = sp ? at<unsigned>(w, o.split_mask) : nullptr;
    B.split_pf = sp ? at<float4>(w, o.split_pf) : nullptr;
    B.split_pv = sp ? at<int2>(w, o.split_pv) : nullptr;
    B.part_b.f = sp ? at<float4>(w, o.split_part) : nullptr;
    B.part_b.vmax = sp ? at<float>(w, o.split_vmax) : nullptr;
    B.part_b.npen = sp ? at<int>(w, o.split_npen) : nullptr;
    if (c->tangent) {
        TBufs &T = c->T;
        T.n = (int)c->nf;
        T.ngh = (int)(c->nw + c->ng);
        T.s_pos = at<float2>(w, o.t_s_pos);
        T.s_vel = at<float2>(w, o.t_s_vel);
        T.s_aux = at<float4>(w, o.t_s_aux);
        T.s_rd = at<float2>(w, o.t_s_rd);
        T.st_vel = at<float2>(w, o.t_st_vel);
        T.st_rho = at<float>(w, o.t_st_rho);
        T.st_a = at<float2>(w, o.t_st_a);
        T.st_D = at<float2>(w, o.t_st_D);
        T.st_X = at<float2>(w, o.t_st_X);
        T.u_pos = at<float2>(w, o.t_u_pos);
        T.u_vel = at<float2>(w, o.t_u_vel);
        T.g_vel = at<float2>(w, o.t_g_vel);
        T.g_aux = at<float4>(w, o.t_g_aux);
        T.perm_dst = at<int>(w, o.t_perm);
        T.part = at<float>(w, o.t_part);
        T.sc = at<double>(w, o.t_sc);
        B.perm_dst = T.perm_dst;
        c->t_base = at<char>(w, o.t_begin);
        c->t_bytes = o.t_end - o.t_begin;
    }
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) {                                    \
            std::fprintf(stderr, "hram: %s failed: %s\n", #call,    \
                         cudaGetErrorString(e_));                   \
            return HR_ECUDA;                                        \
        }                                                           \
    } while (0)

// A launch at stream priority prio (kept by graph capture as the kernel
// node's priority).
template <typename... KArgs, typename... Args>
cudaError_t launch_prio(void (*kern)(KArgs...), int grid, int block, cudaStream_t s, int prio,
                        Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// The kernels of one step (prime = 1: evaluate without advancing).  An
// extra block of the scan launch evaluates the kinematics; in tangent mode they run,
// with their derivatives, on a side branch that joins before the ghost pass
// (side stream: graph capture), or first on the same stream.  The split
// pass: after the reorder (and the summed density), the boundary lists, the
// ghost pass and the boundary particles' pass and partials run on a
// high-priority branch while the interior particles' pass runs on the main
// stream; both join before the step's close.  (With HR_FLAG_TIMING the
// "ghost" group is then empty and the "pass" group holds both branches.)
// defer: the step's close is left to the next step's drift launch
// (k_close_drift) or to settle(); otherwise k_finalize ends the step.
int launch_step(hr_case *c, cudaStream_t s, int prime, bool with_events, cudaStream_t side,
                bool defer = false)
{
    const Consts &K = c->K;
    const Bufs &B = c->B;
    const int fin_blocks = kFinalizeBlocks + K.n_probes;   // reduction blocks, then one per probe
    if (with_events) CK(cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal));
    // defer (step graphs, never with the tangent mode): the last step's
    // close, if pending, in the first blocks of the drift launch
    // (k_close_drift); this step's close is left pending
    // the kinematics: in an extra block of the scan launch, or (tangent mode, whose
    // kinematics derivatives follow them) on a branch beside the drift and
    // the sort
    const bool kin_branch = c->tangent;
    if (kin_branch && side) {
        CK(cudaEventRecord(c->fork, s));
        CK(cudaStreamWaitEvent(side, c->fork, 0));
        k_kinematics<<<1, 128, 0, side>>>(K, B, prime);
        kt_kinematics<<<1, 32, 0, side>>>(K, B, c->T, prime);
        CK(cudaEventRecord(c->join, side));
    } else if (kin_branch) {
        k_kinematics<<<1, 128, 0, s>>>(K, B, prime);
        kt_kinematics<<<1, 32, 0, s>>>(K, B, c->T, prime);
    }
    if (defer && K.closure == 1)
        k_close_drift<1><<<fin_blocks + c->drift_blocks, 256, 0, s>>>(K, B, fin_blocks, K.split ? 1 : 0);
    else if (defer)
        k_close_drift<0><<<fin_blocks + c->drift_blocks, 256, 0, s>>>(K, B, fin_blocks, K.split ? 1 : 0);
    else
        k_drift_key<<<c->drift_blocks, 256, 0, s>>>(K, B, prime);
    if (c->tangent) kt_drift<<<c->drift_blocks, 256, 0, s>>>(K, B, c->T, prime);
    if (with_events) CK(cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal));
    k_scan_apply<<<c->n_tiles + (kin_branch ? 0 : 1), kScanThreads, 0, s>>>(K, B, prime, kin_branch ? 0 : 1,
                                                                         defer ? 1 : 0);
    const bool paper = K.closure == 1;
    const bool split = K.split != 0;   // (never with the tangent mode)
    if (paper) k_rank_scatter<1><<<c->drift_blocks, 256, 0, s>>>(K, B, prime);
    else k_rank_scatter<0><<<c->drift_blocks, 256, 0, s>>>(K, B, prime);
    if (c->tangent) kt_scatter<<<c->drift_blocks, 256, 0, s>>>(K, B, c->T, prime);
    if (with_events) CK(cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal));
    if (kin_branch && side) CK(cudaStreamWaitEvent(s, c->join, 0));
    // closure 1: the summed density needs the disk ghosts at t^{n+1}
    if (paper) k_density<<<c->drift_blocks, 256, 0, s>>>(K, B, prime);
    if (split) {
        cudaStream_t g = side ? side : s;
        if (side) {
            CK(cudaEventRecord(c->fork2, s));
            CK(cudaStreamWaitEvent(side, c->fork2, 0));
        }
        // the ghost pass, and in its extra blocks the boundary lists
        const int gb = c->ghost_blocks + kSplitListBlocks;
        if (paper) {
            CK(launch_prio(k_ghost<1>, gb, kGhostWarps * 32, g, c->prio_hi, K, B));
            CK(launch_prio(k_pass_boundary<1>, c->split_blocks, kPassThreads, g, c->prio_hi, K, B, prime));
        } else {
            CK(launch_prio(k_ghost<0>, gb, kGhostWarps * 32, g, c->prio_hi, K, B));
            CK(launch_prio(k_pass_boundary<0>, c->split_blocks, kPassThreads, g, c->prio_hi, K, B, prime));
        }
        CK(launch_prio(k_pass_boundary_sums, c->split_blocks, kPassThreads, g, c->prio_hi, K, B));
        if (side) CK(cudaEventRecord(c->join2, side));
        if (with_events) CK(cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal));
        if (paper) k_pass<1, 1, kPassInterior><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
        else k_pass<0, 1, kPassInterior><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
        if (side) CK(cudaStreamWaitEvent(s, c->join2, 0));
    } else {
        if (paper) k_ghost<1><<<c->ghost_blocks, kGhostWarps * 32, 0, s>>>(K, B);
        else k_ghost<0><<<c->ghost_blocks, kGhostWarps * 32, 0, s>>>(K, B);
        if (c->tangent) kt_ghost<<<c->tghost_blocks, kGhostWarps * 32, 0, s>>>(K, B, c->T);
        if (with_events) CK(cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal));
    }
    if (split) {
        // the interior and boundary passes above
    } else if (c->n3) k_pass_n3<<<c->pass_blocks, kN3Threads, 0, s>>>(K, B, prime);
    else if (c->lanes == 2 && paper) k_pass_lanes<1, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->lanes == 2) k_pass_lanes<0, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->lanes == 4 && paper) k_pass_lanes<1, 4><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->lanes == 4) k_pass_lanes<0, 4><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->stage == 1 && paper) k_pass_staged<1, 1><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->stage == 1) k_pass_staged<0, 1><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->stage == 2 && paper) k_pass_staged<1, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (c->stage == 2) k_pass_staged<0, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (K.sr == 2 && paper) k_pass<1, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (K.sr == 2) k_pass<0, 2><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else if (paper) k_pass<1><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    else k_pass<0><<<c->pass_blocks, kPassThreads, 0, s>>>(K, B, prime);
    if (c->tangent) kt_pass<<<c->tpass_blocks, kTPassThreads, 0, s>>>(K, B, c->T, prime);
    if (with_events) CK(cudaEventRecordWithFlags(c->ev[4], s, cudaEventRecordExternal));
    if (defer) {
        // the close runs in the next step's graph (or when the host settles)
    } else if (paper) {
        k_finalize<1><<<fin_blocks, kFinalizeThreads, 0, s>>>(K, B, prime, split ? 1 : 0, 0);
    } else {
        k_finalize<0><<<fin_blocks, kFinalizeThreads, 0, s>>>(K, B, prime, split ? 1 : 0, 0);
    }
    if (c->tangent) kt_finalize<<<1, kTFinThreads, 0, s>>>(K, B, c->T, prime, c->tpass_blocks);
    if (with_events) CK(cudaEventRecordWithFlags(c->ev[5], s, cudaEventRecordExternal));
    CK(cudaGetLastError());
    return HR_OK;
}

int capture(hr_case *c)
{
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = launch_step(c, c->cap, 0, c->timing, c->cap2, c->defer);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
    if (rc != HR_OK) return rc;
    CK(e);
    c->graph = g;
    // the split pass's ghost branch runs at its nodes' priority
    CK(cudaGraphInstantiate(&c->exec, c->graph, cudaGraphInstantiateFlagUseNodePriority));
    if (!c->timing) {
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        int rcm = HR_OK;
        for (int q = 0; q < kMultiSteps && rcm == HR_OK; ++q)
            rcm = launch_step(c, c->cap, 0, false, c->cap2, c->defer);
        cudaGraph_t gm = nullptr;
        const cudaError_t em = cudaStreamEndCapture(c->cap, &gm);
        if (rcm != HR_OK) return rcm;
        CK(em);
        c->graph_multi = gm;
        CK(cudaGraphInstantiate(&c->exec_multi, c->graph_multi, cudaGraphInstantiateFlagUseNodePriority));
    }
    return HR_OK;
}

// Runs the close that the last step graph left pending, then the CFL gate
// (k_finalize mode 2), so the case's scalars, probe records and status are
// those of a close at the end of the step, bit for bit.  Asynchronous.
int settle(hr_case *c)
{
    if (!c->pending) return HR_OK;
    c->pending = false;
    const int fin_blocks = kFinalizeBlocks + c->K.n_probes;
    const int split = c->K.split ? 1 : 0;
    if (c->K.closure == 1)
        k_finalize<1><<<fin_blocks, kFinalizeThreads, 0, c->stream>>>(c->K, c->B, 0, split, 2);
    else
        k_finalize<0><<<fin_blocks, kFinalizeThreads, 0, c->stream>>>(c->K, c->B, 0, split, 2);
    CK(cudaGetLastError());
    return HR_OK;
}

int device_status(hr_case *c)
{
    const int rs = settle(c);
    if (rs != HR_OK) return rs;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    int st = 0;
    CK(cudaMemcpy(&st, &c->B.S->status, sizeof(int), cudaMemcpyDeviceToHost));
    int rc = st & (HR_WPENETRATION | HR_WOUTSIDE | HR_WPROBEFULL);
    if (st & ST_BOUNDS) rc = HR_ECHECK;
    else if (st & ST_N3WAIT) rc = HR_ETIMEOUT;
    else if (st & ST_N3CAP) rc = HR_ERANGE;
    else if (st & ST_NAN) rc = HR_ENAN;
    else if (st & ST_DT) rc = HR_EDT;
    if (rc < 0) c->sticky = rc;
    return c->sticky < 0 ? c->sticky : rc;
}

// Uploads a fluid state in ID order (identity permutation), zero derivatives.
int upload_state(hr_case *c, const float *xy, const float *vel, const float *rho)
{
    // straight from the caller's buffers (pinned ones copy at full speed);
    // the density conversion and the IDs are made on the device
    const size_t n = (size_t)c->nf;
    CK(cudaMemcpyAsync(c->B.s_pos, xy, n * 8, cudaMemcpyHostToDevice, c->stream));
    if (vel) CK(cudaMemcpyAsync(c->B.st_vel, vel, n * 8, cudaMemcpyHostToDevice, c->stream));
    else CK(cudaMemsetAsync(c->B.st_vel, 0, n * 8, c->stream));
    if (rho) CK(cudaMemcpyAsync(c->io, rho, n * 4, cudaMemcpyHostToDevice, c->stream));
    else CK(cudaMemsetAsync(c->B.st_rho, 0, n * 4, c->stream));
    k_upload_fix<<<c->drift_blocks, 256, 0, c->stream>>>(c->K, c->B, rho ? c->io : nullptr,
                                                         c->P.rho0);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->B.st_a, 0, n * 8, c->stream));
    CK(cudaMemsetAsync(c->B.st_D, 0, n * 8, c->stream));
    CK(cudaMemsetAsync(c->B.st_X, 0, n * 8, c->stream));
    CK(cudaMemsetAsync(c->B.cell_count, 0, ((size_t)c->K.ncell + 1) * 4, c->stream));
    CK(cudaMemsetAsync(c->B.tile_sum, 0, (size_t)c->n_tiles * 4, c->stream));
    CK(cudaMemsetAsync(c->B.fin_ticket, 0, 4, c->stream));
    CK(cudaMemsetAsync(c->B.ovf_count, 0, 4, c->stream));
    CK(cudaMemsetAsync(c->B.S, 0, sizeof(Scalars), c->stream));
    if (c->n3) {
        CK(cudaMemsetAsync(c->B.n3_flag, 0, (size_t)c->K.n3_tiles_max * 4, c->stream));
        CK(cudaMemsetAsync(c->B.n3_ctl, 0, 8, c->stream));
    }
    if (c->K.split) {
        CK(cudaMemsetAsync(c->B.split_n, 0, 8, c->stream));
        CK(cudaMemsetAsync(c->B.split_mask, 0, ((size_t)c->pass_blocks + 31) / 32 * 4, c->stream));
    }
    if (c->tangent) {
        // the uploaded state does not depend on the parameters; dt = C h /
        // (c0 + v0) has d dt / d ln c0 = -dt c0 / (c0 + v0)
        CK(cudaMemsetAsync(c->t_base, 0, c->t_bytes, c->stream));
        std::vector<double> sc(TSC_N, 0.0);
        sc[TSC_DT + 1] = -c->K.dt_fixed * c->P.c0 / (c->P.c0 + c->P.v0);
        sc[TSC_PEAK] = -HUGE_VAL;
        sc[TSC_PSTEP] = -1.0;
        CK(cudaMemcpyAsync(c->T.sc, sc.data(), TSC_N * 8, cudaMemcpyHostToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->host_step = 0;
    c->diag_rec = 0;
    c->sticky = 0;
    return HR_OK;
}

int prime(hr_case *c)
{
    const int rc = launch_step(c, c->stream, 1, false, nullptr);
    if (rc != HR_OK) return rc;
    return device_status(c);
}

// Per cell, 1 where the rows of its stencil (reach K.sr; the pass's
// for_fluid_candidates ranges) hold a wall ghost.  start: the wall ghosts'
// cell starts (ncell + 1 entries).
int upload_wall_near(hr_case *c, const std::vector<int> &start)
{
    const Consts &K = c->K;
    const int R = K.sr;
    std::vector<unsigned char> near((size_t)K.ncell, 0);
    for (int cc = 0; cc < K.ncell; ++cc) {
        bool any = false;
        for (int dy = -R; dy <= R && !any; ++dy) {
            const int row = cc + dy * K.ncx;
            const int a = std::min(std::max(row - R, 0), K.ncell);
            const int b = std::min(std::max(row + R + 1, 0), K.ncell);
            any = start[b] > start[a];
        }
        near[cc] = any ? 1 : 0;
    }
    CK(cudaMemcpy(c->B.wall_near, near.data(), near.size(), cudaMemcpyHostToDevice));
    return HR_OK;
}

int build_walls(hr_case *c, const Geometry &G)
{
    const int nw = (int)c->nw;
    if (nw == 0) {
        std::vector<int> ws((size_t)c->K.ncell + 1, 0);
        CK(cudaMemcpy(c->B.wall_start, ws.data(), ws.size() * 4, cudaMemcpyHostToDevice));
        return upload_wall_near(c, ws);
    }
    std::vector<float2> pos(nw);
    for (int k = 0; k < nw; ++k) pos[k] = make_float2((float)G.wx[k], (float)G.wy[k]);
    // keys with the device's cell arithmetic
    int *dkey = nullptr;
    float2 *dpos = nullptr;
    CK(cudaMalloc(&dkey, nw * 4));
    CK(cudaMalloc(&dpos, nw * 8));
    CK(cudaMemcpy(dpos, pos.data(), nw * 8, cudaMemcpyHostToDevice));
    k_wall_keys<<<(nw + 255) / 256, 256>>>(c->K, dpos, nw, dkey);
    std::vector<int> key(nw);
    cudaError_t e = cudaMemcpy(key.data(), dkey, nw * 4, cudaMemcpyDeviceToHost);
    cudaFree(dkey);
    cudaFree(dpos);
    CK(e);
    std::vector<int> order(nw);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<float2> spos(nw), snrm(nw);
    std::vector<int> skind(nw), sid(nw), start((size_t)c->K.ncell + 1, 0);
    for (int k = 0; k < nw; ++k) {
        const int o = order[k];
        spos[k] = pos[o];
        snrm[k] = make_float2((float)G.wnx[o], (float)G.wny[o]);
        skind[k] = G.wkind[o];
        sid[k] = o;
        start[key[o] + 1]++;
    }
    for (int q = 0; q < c->K.ncell; ++q) start[q + 1] += start[q];
    c->wall_id_of_sorted = sid;
    CK(cudaMemcpy(c->B.gw_pos, spos.data(), nw * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.gw_nrm, snrm.data(), nw * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.gw_kind, skind.data(), nw * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.gw_id, sid.data(), nw * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.wall_start, start.data(), start.size() * 4, cudaMemcpyHostToDevice));
    return upload_wall_near(c, start);
}

// ------------------------------------------------------ reverse mode

}  // namespace

// The checkpoint store, the tape of one segment of L steps and the adjoint
// buffers of a case (one device block owned by the case).
struct AdjCtx {
    int L = 0;                    // steps between checkpoints
    long long n_steps = 0;
    void *mem = nullptr;
    size_t bytes = 0;
    std::vector<Slot> tape;       // L slots: the segment being swept
    Slot prime_slot{}, upload{};  // the priming pass and its input (fluid-ID order)
    std::vector<Slot> ckpt;       // ckpt[k]: the state after step k L (ckpt[0] = prime_slot)
    Scalars *S_final = nullptr;   // the scalars after the forward run
    Slot start{};                 // the state a segment starts from (a copy of its checkpoint)
    cudaGraph_t seg_graph[2] = {nullptr, nullptr};        // one full segment, by the parity
    cudaGraphExec_t seg_exec[2] = {nullptr, nullptr};     // of the adjoint buffers at its start
    cudaGraph_t rev_graph[2] = {nullptr, nullptr};        // its reverse half alone (a segment
    cudaGraphExec_t rev_exec[2] = {nullptr, nullptr};     // whose records are on the tape)
    bool taped_last = false;      // the forward run recorded the last segment on the tape
    ABufs A{};
    LState ls[2]{};
    int ep_blocks = 0, bk_blocks = 0, gh_blocks = 0;
    bool forward_done = false;
    double peak = 0.0, impulse = 0.0;
    long long peak_row = -1;
};

namespace {

void adj_free(hr_case *c)
{
    if (!c->adj) return;
    for (int k = 0; k < 2; ++k) {
        if (c->adj->seg_exec[k]) cudaGraphExecDestroy(c->adj->seg_exec[k]);
        if (c->adj->seg_graph[k]) cudaGraphDestroy(c->adj->seg_graph[k]);
        if (c->adj->rev_exec[k]) cudaGraphExecDestroy(c->adj->rev_exec[k]);
        if (c->adj->rev_graph[k]) cudaGraphDestroy(c->adj->rev_graph[k]);
    }
    if (c->adj->mem) cudaFree(c->adj->mem);
    delete c->adj;
    c->adj = nullptr;
}

// Carves the reverse-mode buffers of a run of n_steps steps with a
// checkpoint every L steps.
int adj_alloc(hr_case *c, long long n_steps, int L)
{
    adj_free(c);
    AdjCtx *a = new AdjCtx();
    c->adj = a;
    a->L = L;
    a->n_steps = n_steps;
    const size_t n = (size_t)c->nf, ngh = (size_t)(c->nw + c->ng), nc = (size_t)c->K.ncell;
    const size_t ng = (size_t)c->ng;
    const long long n_ck = (n_steps + L - 1) / L;   // checkpoints 1 .. n_ck - 1 (0 is the prime)
    Layout Lo;
    struct SlotOff {
        size_t s_pos, s_vel, s_aux, s_rd, s_id, st_vel, st_rho, st_a, st_D, st_X, perm, cs, gd, gv,
            ga, S, kin;
    };
    auto full = [&]() {
        SlotOff o;
        o.s_pos = Lo.add((n + kPosPad) * 8);
        o.s_vel = Lo.add(n * 8);
        o.s_aux = Lo.add(n * 16);
        o.s_rd = Lo.add(n * 8);
        o.s_id = Lo.add(n * 4);
        o.st_vel = Lo.add(n * 8);
        o.st_rho = Lo.add(n * 4);
        o.st_a = Lo.add(n * 8);
        o.st_D = Lo.add(n * 8);
        o.st_X = Lo.add(n * 8);
        o.perm = Lo.add(n * 4);
        o.cs = Lo.add((nc + 2) * 4);
        o.gd = Lo.add(std::max<size_t>(ng, 1) * 8);
        o.gv = Lo.add(std::max<size_t>(ngh, 1) * 8);
        o.ga = Lo.add(std::max<size_t>(ngh, 1) * 16);
        o.S = Lo.add(sizeof(Scalars));
        o.kin = Lo.add(6 * 8);
        return o;
    };
    auto state = [&]() {   // a checkpoint: the state a step starts from
        SlotOff o{};
        o.s_pos = Lo.add((n + kPosPad) * 8);
        o.s_id = Lo.add(n * 4);
        o.st_vel = Lo.add(n * 8);
        o.st_rho = Lo.add(n * 4);
        o.st_a = Lo.add(n * 8);
        o.st_D = Lo.add(n * 8);
        o.st_X = Lo.add(n * 8);
        o.S = Lo.add(sizeof(Scalars));
        return o;
    };
    std::vector<SlotOff> tape_o;
    for (long long k = 0; k < std::min<long long>(L, n_steps); ++k) tape_o.push_back(full());
    const SlotOff prime_o = full();
    const SlotOff up_o = state();
    const SlotOff start_o = state();
    std::vector<SlotOff> ck_o;
    for (long long k = 1; k < n_ck; ++k) ck_o.push_back(state());
    const size_t sfin = Lo.add(sizeof(Scalars));
    const size_t nq = n * kOut, gq = std::max<size_t>(ngh, 1) * kOut;
    size_t ls_o[2][7];
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 4; ++k) ls_o[b][k] = Lo.add(nq * 8);
        for (int k = 4; k < 7; ++k) ls_o[b][k] = Lo.add(nq * 4);
    }
    a->ep_blocks = (int)((n + kAThreads - 1) / kAThreads);
    a->bk_blocks = a->ep_blocks;
    a->gh_blocks = (int)std::max<size_t>(1, (ngh + kAGhostWarps - 1) / kAGhostWarps);
    const size_t wA = Lo.add(n * 16), wX = Lo.add(n * 16), wDr = Lo.add(n * 8);
    const size_t lpos = Lo.add(nq * 8), lvh = Lo.add(nq * 8), lrec = Lo.add(nq * 16),
                 lrd = Lo.add(nq * 8);
    const size_t gS1 = Lo.add(gq * 16), gS2 = Lo.add(gq * 8), gpar = Lo.add(gq * 16),
                 grg = Lo.add(gq * 8);
    const size_t ep = Lo.add((size_t)a->ep_blocks * kOut * 4);
    const size_t bk = Lo.add((size_t)a->bk_blocks * kOut * 16);
    const size_t sums = Lo.add((size_t)kAReduceBlocks * kASums * 8);
    const size_t sc = Lo.add(ASC_N * 8);
    const size_t cpart = Lo.add((size_t)(kAReduceBlocks / 32) * kASums * 8);
    const size_t ctick = Lo.add(4);
    a->bytes = Lo.total;
    if (cudaMalloc(&a->mem, a->bytes) != cudaSuccess) {
        cudaGetLastError();
        a->mem = nullptr;
        adj_free(c);
        return HR_ENOMEM;
    }
    void *w = a->mem;
    auto mk = [&](const SlotOff &o, bool isfull) {
        Slot sl{};
        sl.s_pos = at<float2>(w, o.s_pos);
        sl.s_id = at<int>(w, o.s_id);
        sl.st_vel = at<float2>(w, o.st_vel);
        sl.st_rho = at<float>(w, o.st_rho);
        sl.st_a = at<float2>(w, o.st_a);
        sl.st_D = at<float2>(w, o.st_D);
        sl.st_X = at<float2>(w, o.st_X);
        sl.S = at<Scalars>(w, o.S);
        if (isfull) {
            sl.s_vel = at<float2>(w, o.s_vel);
            sl.s_aux = at<float4>(w, o.s_aux);
            sl.s_rd = at<float2>(w, o.s_rd);
            sl.perm_dst = at<int>(w, o.perm);
            sl.cell_start = at<int>(w, o.cs);
            sl.gd_pos = at<float2>(w, o.gd);
            sl.g_vel = at<float2>(w, o.gv);
            sl.g_aux = at<float4>(w, o.ga);
            sl.kin = at<double>(w, o.kin);
        }
        return sl;
    };
    for (auto &o : tape_o) a->tape.push_back(mk(o, true));
    a->prime_slot = mk(prime_o, true);
    a->upload = mk(up_o, false);
    a->start = mk(start_o, false);
    a->ckpt.push_back(a->prime_slot);
    for (auto &o : ck_o) a->ckpt.push_back(mk(o, false));
    a->S_final = at<Scalars>(w, sfin);
    for (int b = 0; b < 2; ++b) {
        LState &l = a->ls[b];
        l.r = at<float2>(w, ls_o[b][0]);
        l.v = at<float2>(w, ls_o[b][1]);
        l.a = at<float2>(w, ls_o[b][2]);
        l.X = at<float2>(w, ls_o[b][3]);
        l.d = at<float>(w, ls_o[b][4]);
        l.D = at<float>(w, ls_o[b][5]);
        l.E = at<float>(w, ls_o[b][6]);
    }
    ABufs &A = a->A;
    A.wA = at<float4>(w, wA);
    A.wX = at<float4>(w, wX);
    A.wDr = at<float2>(w, wDr);
    A.lpos = at<float2>(w, lpos);
    A.lvh = at<float2>(w, lvh);
    A.lrec = at<float4>(w, lrec);
    A.lrd = at<float2>(w, lrd);
    A.gS1 = at<float4>(w, gS1);
    A.gS2 = at<float2>(w, gS2);
    A.gpar = at<float4>(w, gpar);
    A.grg = at<float2>(w, grg);
    A.ep_part = at<float>(w, ep);
    A.bk_part = at<float4>(w, bk);
    A.sums = at<float2>(w, sums);
    A.sc = at<double>(w, sc);
    A.status = &c->B.S->status;
    A.cpart = at<double>(w, cpart);
    A.ctick = at<int>(w, ctick);
    return HR_OK;
}

// The case's buffers with the per-step arrays of slot sl (S: the slot's
// scalars when with_S, else the live ones).
Bufs slot_bufs(const hr_case *c, const Slot &sl, bool with_S)
{
    Bufs B = c->B;
    B.s_pos = sl.s_pos;
    B.s_vel = sl.s_vel;
    B.s_aux = sl.s_aux;
    B.s_rd = sl.s_rd;
    B.s_id = sl.s_id;
    B.st_vel = sl.st_vel;
    B.st_rho = sl.st_rho;
    B.st_a = sl.st_a;
    B.st_D = sl.st_D;
    B.st_X = sl.st_X;
    B.perm_dst = sl.perm_dst;
    B.cell_start = sl.cell_start;
    B.gd_pos = sl.gd_pos;
    B.g_vel = sl.g_vel;
    B.g_aux = sl.g_aux;
    if (with_S) B.S = sl.S;
    return B;
}

// One forward step recorded into slot cur from the state in prev (the
// step's kernels, closure 0, each given the arrays it reads and writes), then
// the scalars snapshot.  The live scalars c->B.S advance as in a plain step.
int launch_tape_step(hr_case *c, cudaStream_t s, const Slot &cur, const Slot &prev, int prime)
{
    Consts K = c->K;
    K.split = 0;   // the one-kernel pass (the same bits as the split one)
    Bufs Bk = c->B;
    Bk.gd_pos = cur.gd_pos;
    Bufs Bd = c->B;   // the drift reads the previous state
    Bd.s_pos = prev.s_pos;
    Bd.s_id = prev.s_id;
    Bd.st_vel = prev.st_vel;
    Bd.st_a = prev.st_a;
    Bd.st_X = prev.st_X;
    Bufs Bs = c->B;   // scan and provisional slots write this step's cell starts
    Bs.cell_start = cur.cell_start;
    Bufs Br = slot_bufs(c, cur, false);   // the reorder writes this step's arrays
    Br.st_rho = prev.st_rho;             // ... from the previous density and rates
    Br.st_D = prev.st_D;
    const Bufs Bc = slot_bufs(c, cur, false);
    // the kinematics (and their derivatives for the reverse sweep) on a side
    // branch beside the drift and the sort, as in the step graph
    CK(cudaEventRecord(c->fork, s));
    CK(cudaStreamWaitEvent(c->cap2, c->fork, 0));
    k_kinematics<<<1, 128, 0, c->cap2>>>(K, Bk, prime);
    ka_kin<<<1, 32, 0, c->cap2>>>(K, c->B.S, cur.kin);
    CK(cudaEventRecord(c->join, c->cap2));
    k_drift_key<<<c->drift_blocks, 256, 0, s>>>(K, Bd, prime);
    k_scan_apply<<<c->n_tiles, kScanThreads, 0, s>>>(K, Bs, prime, 0, 0);
    k_rank_scatter<0><<<c->drift_blocks, 256, 0, s>>>(K, Br, prime);
    CK(cudaStreamWaitEvent(s, c->join, 0));
    k_ghost<0><<<c->ghost_blocks, kGhostWarps * 32, 0, s>>>(K, Bc);
    k_pass<0><<<c->pass_blocks, kPassThreads, 0, s>>>(K, Bc, prime);
    k_finalize<0><<<kFinalizeBlocks + K.n_probes, kFinalizeThreads, 0, s>>>(K, Bc, prime, 0, 0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(cur.S, c->B.S, sizeof(Scalars), cudaMemcpyDeviceToDevice, s));
    return HR_OK;
}

// Copies the case's current state (what the next step starts from) into a
// checkpoint.
int save_ckpt(hr_case *c, const Slot &k, cudaStream_t s)
{
    const size_t n = (size_t)c->nf;
    CK(cudaMemcpyAsync(k.s_pos, c->B.s_pos, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.s_id, c->B.s_id, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.st_vel, c->B.st_vel, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.st_rho, c->B.st_rho, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.st_a, c->B.st_a, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.st_D, c->B.st_D, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.st_X, c->B.st_X, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(k.S, c->B.S, sizeof(Scalars), cudaMemcpyDeviceToDevice, s));
    return HR_OK;
}

// The reverse sweep of one step: slot cur holds the step's record, prev the
// state it started from.  The end-of-step adjoints are in A.cur; the
// adjoints of the start state land in A.prv.
int adjoint_step(hr_case *c, cudaStream_t s, const Slot &cur, const Slot &prev, int prime,
                 bool seed_peak)
{
    AdjCtx *a = c->adj;
    const Consts &K = c->K;
    const Bufs Bc = slot_bufs(c, cur, true);
    Bufs Bp = c->B;
    Bp.s_pos = prev.s_pos;
    Bp.st_vel = prev.st_vel;
    Bp.st_rho = prev.st_rho;
    Bp.st_a = prev.st_a;
    Bp.st_D = prev.st_D;
    Bp.st_X = prev.st_X;
    if (seed_peak && K.n_probes > 0) ka_probe<<<1, 32, 0, s>>>(K, Bc, a->A, a->peak_row);
    ka_epilogue<<<a->ep_blocks, kAThreads, 0, s>>>(K, Bc, a->A, prime);
    ka_ghost<<<a->gh_blocks, kAGhostWarps * 32, 0, s>>>(K, Bc, a->A, prime);
    ka_pass<<<a->ep_blocks, kAThreads, 0, s>>>(K, Bc, a->A, prime);
    ka_back<<<a->bk_blocks, kAThreads, 0, s>>>(K, Bc, Bp, a->A, prime);
    ka_reduce<<<kAReduceBlocks, kAReduceThreads, 0, s>>>(K, a->A, a->ep_blocks, a->bk_blocks,
                                                          a->A.sums);
    ka_close<<<kASums, kAReduceBlocks, 0, s>>>(K, Bc, a->A, prime, a->A.sums, cur.kin);
    CK(cudaGetLastError());
    std::swap(a->A.cur, a->A.prv);
    return HR_OK;
}

// Copies checkpoint k into the segment start state (and its scalars into the
// live ones the recomputation advances).
int load_start(hr_case *c, const Slot &k, cudaStream_t s)
{
    const Slot &d = c->adj->start;
    const size_t n = (size_t)c->nf;
    CK(cudaMemcpyAsync(d.s_pos, k.s_pos, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.s_id, k.s_id, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.st_vel, k.st_vel, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.st_rho, k.st_rho, n * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.st_a, k.st_a, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.st_D, k.st_D, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d.st_X, k.st_X, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->B.S, k.S, sizeof(Scalars), cudaMemcpyDeviceToDevice, s));
    return HR_OK;
}

// One segment of len steps from the start state: the records recomputed
// forwards (unless they are already on the tape), then the reverse sweep
// through them.
int launch_segment(hr_case *c, cudaStream_t s, long long len, bool recompute)
{
    AdjCtx *a = c->adj;
    int rc;
    for (long long k = 0; recompute && k < len; ++k) {
        const Slot &prev = k == 0 ? a->start : a->tape[(size_t)(k - 1)];
        if ((rc = launch_tape_step(c, s, a->tape[(size_t)k], prev, 0)) != HR_OK) return rc;
    }
    for (long long k = len - 1; k >= 0; --k) {
        const Slot &prev = k == 0 ? a->start : a->tape[(size_t)(k - 1)];
        if ((rc = adjoint_step(c, s, a->tape[(size_t)k], prev, 0, true)) != HR_OK) return rc;
    }
    return HR_OK;
}

// A full segment (L steps) as one graph launch: captured once for each
// parity of the adjoint buffers it starts from, with and without the
// recomputation.
int run_full_segment(hr_case *c, cudaStream_t s, bool recompute)
{
    AdjCtx *a = c->adj;
    const int par = a->A.cur.r == a->ls[0].r ? 0 : 1;
    cudaGraph_t &graph = recompute ? a->seg_graph[par] : a->rev_graph[par];
    cudaGraphExec_t &exec = recompute ? a->seg_exec[par] : a->rev_exec[par];
    if (!exec) {
        const ABufs keep = a->A;
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_segment(c, c->cap, a->L, recompute);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        a->A = keep;
        if (rc != HR_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CK(e);
        graph = g;
        CK(cudaGraphInstantiate(&exec, g, 0));
    }
    CK(cudaGraphLaunch(exec, s));
    if (a->L & 1) std::swap(a->A.cur, a->A.prv);
    return HR_OK;
}

// Makes the case's own arrays hold what a plain step would have left in
// them, from the record of the same step (the forward run's last segment
// runs on the tape; the next plain step reads these arrays).
int tape_to_live(hr_case *c, const Slot &sl, cudaStream_t s)
{
    const size_t n = (size_t)c->nf, ngh = (size_t)(c->nw + c->ng), nc = (size_t)c->K.ncell;
    const Bufs &B = c->B;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
    };
    CK(cp(B.s_pos, sl.s_pos, n * 8));
    CK(cp(B.s_vel, sl.s_vel, n * 8));
    CK(cp(B.s_aux, sl.s_aux, n * 16));
    CK(cp(B.s_rd, sl.s_rd, n * 8));
    CK(cp(B.s_id, sl.s_id, n * 4));
    CK(cp(B.st_vel, sl.st_vel, n * 8));
    CK(cp(B.st_rho, sl.st_rho, n * 4));
    CK(cp(B.st_a, sl.st_a, n * 8));
    CK(cp(B.st_D, sl.st_D, n * 8));
    CK(cp(B.st_X, sl.st_X, n * 8));
    CK(cp(B.cell_start, sl.cell_start, (nc + 2) * 4));
    CK(cp(B.gd_pos, sl.gd_pos, (size_t)c->ng * 8));
    CK(cp(B.g_vel, sl.g_vel, ngh * 8));
    CK(cp(B.g_aux, sl.g_aux, ngh * 16));
    return HR_OK;
}

}  // namespace

// ------------------------------------------------------------------ C-ABI

extern "C" {

int hr_workspace_bytes(const hr_params *p, int64_t n_fluid, size_t *bytes)
{
    if (!bytes) return HR_EINVAL;
    const int v = validate(p, n_fluid);
    if (v != HR_OK) return v;
    hr_case tmp;
    tmp.P = *p;
    tmp.nf = n_fluid;
    tmp.nw = (long long)make_walls(*p).wx.size();
    tmp.ng = p->Ng;
    make_consts(&tmp);
    *bytes = plan(&tmp).total;
    return HR_OK;
}

int hr_init_case(const hr_params *p, const float *xy, int64_t n_fluid, const float *vel,
                 const float *rho, void *d_workspace, size_t workspace_bytes, void *cuda_stream,
                 hr_case **out)
{
    const NvtxRange nvtx_range("hr_init_case");
    if (!out) return HR_EINVAL;
    *out = nullptr;
    if (!xy) return HR_EINVAL;
    int rc = validate(p, n_fluid);
    if (rc != HR_OK) return rc;
    hr_case *c = new hr_case();
    c->P = *p;
    c->nf = n_fluid;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return HR_ECUDA;
    }
    const Geometry G = make_walls(*p);
    c->nw = (long long)G.wx.size();
    c->ng = p->Ng;
    make_consts(c);
    const Offsets o = plan(c);
    c->stream = (cudaStream_t)cuda_stream;
    c->timing = (p->flags & HR_FLAG_TIMING) != 0;
    auto fail = [&](int code) {
        hr_destroy(c);
        return code;
    };
    if (d_workspace) {
        // the arrays are carved at 256-byte offsets and read with vector loads
        if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0) return fail(HR_EINVAL);
        if (workspace_bytes < o.total) return fail(HR_ENOMEM);
        c->ws = d_workspace;
        c->ws_bytes = workspace_bytes;
    } else {
        if (cudaMalloc(&c->ws, o.total) != cudaSuccess) {
            cudaGetLastError();
            c->ws = nullptr;
            return fail(HR_ENOMEM);
        }
        c->own_ws = true;
        c->ws_bytes = o.total;
    }
    bind(c, o);
    int prio_lo = 0;
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&prio_lo, &c->prio_hi) != cudaSuccess)
        return fail(HR_ECUDA);
    for (int k = 0; k < kTimingEvents; ++k)
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) return fail(HR_ECUDA);
    if ((rc = build_walls(c, G)) != HR_OK) return fail(rc);
    if (c->ng > 0) {
        std::vector<double2> off((size_t)c->ng);
        for (long long k = 0; k < c->ng; ++k) {
            const double th = 2.0 * M_PI * (double)k / (double)c->ng;
            off[k] = make_double2(p->R_disk * std::cos(th), p->R_disk * std::sin(th));
        }
        if (cudaMemcpy(c->B.disk_off, off.data(), off.size() * 16, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return fail(HR_ECUDA);
    }
    if ((rc = upload_state(c, xy, vel, rho)) != HR_OK) return fail(rc);
    rc = prime(c);
    if (rc < 0) return fail(rc);
    const int rc2 = capture(c);
    if (rc2 != HR_OK) return fail(rc2);
    *out = c;
    return rc;
}

int hr_step(hr_case *c)
{
    const NvtxRange nvtx_range("hr_step");
    if (!c || !c->exec) return HR_EINVAL;
    if (c->sticky < 0) return c->sticky;
    if (cudaGraphLaunch(c->exec, c->stream) != cudaSuccess) return c->sticky = HR_ECUDA;
    c->pending = c->defer;
    c->host_step++;
    if (c->P.diag_every > 0 && c->host_step % c->P.diag_every == 0) {
        const int rs = settle(c);
        if (rs != HR_OK) return c->sticky = rs;
        k_diag_partial<<<c->diag_blocks, kDiagThreads, 0, c->stream>>>(c->K, c->B, c->diag_part);
        k_diag_final<<<1, 32, 0, c->stream>>>(c->K, c->B, c->diag_part, c->diag_blocks,
                                              c->diag_out, c->diag_hist, c->diag_rec,
                                              c->diag_cap);
        c->diag_rec++;
    }
    return HR_OK;
}

int hr_sync(hr_case *c)
{
    if (!c) return HR_EINVAL;
    return device_status(c);
}

// k steps, kMultiSteps per graph launch where no periodic diagnostic falls
// inside a group.
static int run_steps(hr_case *c, int64_t k)
{
    while (k > 0) {
        const bool diag = c->P.diag_every > 0;
        if (c->exec_multi && k >= kMultiSteps && !diag) {
            if (c->sticky < 0) return c->sticky;
            if (cudaGraphLaunch(c->exec_multi, c->stream) != cudaSuccess)
                return c->sticky = HR_ECUDA;
            c->pending = c->defer;
            c->host_step += kMultiSteps;
            k -= kMultiSteps;
        } else {
            const int rc = hr_step(c);
            if (rc < 0) return rc;
            --k;
        }
    }
    return HR_OK;
}

int hr_run(hr_case *c, int64_t n_steps, double t_end)
{
    const NvtxRange nvtx_range("hr_run");
    if (!c) return HR_EINVAL;
    if (!c->exec) return HR_EINVAL;
    if (t_end <= 0.0) {
        const int rc = run_steps(c, n_steps);
        if (rc < 0) return rc;
        return device_status(c);
    }
    int64_t done = 0;
    for (;;) {
        double sc[2];
        if (settle(c) != HR_OK) return HR_ECUDA;
        if (cudaMemcpyAsync(sc, &c->B.S->t, 16, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return HR_ECUDA;
        const int st = device_status(c);
        if (st < 0) return st;
        if (sc[0] >= t_end || (n_steps > 0 && done >= n_steps)) return st;
        // steps that cannot overshoot t_end: dt only shrinks by the CFL gate
        int64_t k = (int64_t)std::floor((t_end - sc[0]) / sc[1]);
        k = std::max<int64_t>(1, std::min<int64_t>(k / 2, 256));
        if (n_steps > 0) k = std::min<int64_t>(k, n_steps - done);
        const int rc = run_steps(c, k);
        if (rc < 0) return rc;
        done += k;
    }
}

int hr_probe_pressure(hr_case *c, float *host_out, int64_t cap_rows, int64_t *n_rows)
{
    if (!c) return HR_EINVAL;
    const int st = device_status(c);
    long long n = 0;
    if (cudaMemcpy(&n, &c->B.S->hist_n, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (n_rows) *n_rows = n;
    if (host_out && c->K.n_probes > 0) {
        if (cap_rows < n) return HR_ERANGE;
        if (n > 0 && cudaMemcpy(host_out, c->B.probe_hist, (size_t)n * c->K.n_probes * 4,
                                cudaMemcpyDeviceToHost) != cudaSuccess)
            return HR_ECUDA;
    }
    return st;
}

int hr_probe_times(hr_case *c, double *host_out, int64_t cap, int64_t *n_out)
{
    if (!c) return HR_EINVAL;
    const int st = device_status(c);
    long long n = 0;
    if (cudaMemcpy(&n, &c->B.S->hist_n, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (n_out) *n_out = n;
    if (host_out) {
        if (cap < n) return HR_ERANGE;
        if (n > 0 &&
            cudaMemcpy(host_out, c->B.probe_t, (size_t)n * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return HR_ECUDA;
    }
    return st;
}

int hr_diagnostics(hr_case *c, hr_diag *out)
{
    if (!c || !out) return HR_EINVAL;
    if (settle(c) != HR_OK) return HR_ECUDA;
    k_diag_partial<<<c->diag_blocks, kDiagThreads, 0, c->stream>>>(c->K, c->B, c->diag_part);
    k_diag_final<<<1, 32, 0, c->stream>>>(c->K, c->B, c->diag_part, c->diag_blocks, c->diag_out,
                                          c->diag_hist, -1, c->diag_cap);
    const int st = device_status(c);
    double d[kDiagFields];
    if (cudaMemcpy(d, c->diag_out, sizeof d, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HR_ECUDA;
    std::memcpy(out, d, sizeof d);
    return st;
}

int hr_diag_history(hr_case *c, double *host_out, int64_t cap_rows, int64_t *n_rows)
{
    if (!c) return HR_EINVAL;
    const int st = device_status(c);
    const long long n = std::min(c->diag_rec, c->diag_cap);
    if (n_rows) *n_rows = n;
    if (host_out) {
        if (cap_rows < n) return HR_ERANGE;
        if (n > 0 && cudaMemcpy(host_out, c->diag_hist, (size_t)n * kDiagFields * 8,
                                cudaMemcpyDeviceToHost) != cudaSuccess)
            return HR_ECUDA;
    }
    return st;
}

int hr_get_state(hr_case *c, float *xy, float *vel, float *rho, float *p, int64_t cap)
{
    const NvtxRange nvtx_range("hr_get_state");
    if (!c) return HR_EINVAL;
    if (cap < c->nf) return HR_ERANGE;
    if (settle(c) != HR_OK) return HR_ECUDA;
    const size_t n = (size_t)c->nf;
    float2 *dxy = reinterpret_cast<float2 *>(c->io);
    float2 *dv = dxy + n;
    float *dr = reinterpret_cast<float *>(dv + n);
    float *dp = dr + n;
    k_unsort<<<c->drift_blocks, 256, 0, c->stream>>>(c->K, c->B, dxy, dv, dr, dp);
    const int st = device_status(c);
    if (st < 0 && st != HR_ENAN) return st;
    if (xy && cudaMemcpy(xy, dxy, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (vel && cudaMemcpy(vel, dv, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (rho && cudaMemcpy(rho, dr, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (p && cudaMemcpy(p, dp, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    return st;
}

int hr_get_energy(hr_case *c, float *e, float *de, int64_t cap)
{
    if (!c || c->K.closure != 1) return HR_EINVAL;
    if (cap < c->nf) return HR_ERANGE;
    if (settle(c) != HR_OK) return HR_ECUDA;
    const size_t n = (size_t)c->nf;
    float *de_ = c->io, *dd = c->io + n;
    k_unsort_energy<<<c->drift_blocks, 256, 0, c->stream>>>(c->K, c->B, de_, dd);
    const int st = device_status(c);
    if (st < 0 && st != HR_ENAN) return st;
    if (e && cudaMemcpy(e, de_, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    if (de && cudaMemcpy(de, dd, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    return st;
}

int hr_set_state(hr_case *c, const float *xy, const float *vel, const float *rho, int64_t n)
{
    const NvtxRange nvtx_range("hr_set_state");
    if (!c || !xy || n != c->nf) return HR_EINVAL;
    const int s0 = device_status(c);
    if (s0 == HR_ECUDA) return s0;
    int rc = upload_state(c, xy, vel, rho);
    if (rc != HR_OK) return rc;
    return prime(c);
}

int hr_get_ghosts(hr_case *c, float *xy, float *p, float *rho, float *vel, int64_t cap)
{
    if (!c) return HR_EINVAL;
    const long long ngh = c->nw + c->ng;
    if (cap < ngh) return HR_ERANGE;
    const int st = device_status(c);
    std::vector<float2> gv((size_t)ngh), gpw((size_t)c->nw), gpd((size_t)c->ng);
    std::vector<float4> ga((size_t)ngh);
    if (ngh > 0) {
        if (cudaMemcpy(gv.data(), c->B.g_vel, ngh * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ga.data(), c->B.g_aux, ngh * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
            return HR_ECUDA;
    }
    if (c->nw > 0 &&
        cudaMemcpy(gpw.data(), c->B.gw_pos, c->nw * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HR_ECUDA;
    if (c->ng > 0 &&
        cudaMemcpy(gpd.data(), c->B.gd_pos, c->ng * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HR_ECUDA;
    for (long long k = 0; k < ngh; ++k) {
        const long long dst = k < c->nw ? c->wall_id_of_sorted[k] : k;
        const float2 pos = k < c->nw ? gpw[k] : gpd[k - c->nw];
        if (xy) { xy[2 * dst] = pos.x; xy[2 * dst + 1] = pos.y; }
        if (p) p[dst] = ga[k].y;
        if (rho) rho[dst] = c->K.rho0 * (1.0f + ga[k].x);
        if (vel) { vel[2 * dst] = gv[k].x; vel[2 * dst + 1] = gv[k].y; }
    }
    return st;
}

int hr_get_scalars(hr_case *c, double *out, int n)
{
    if (!c || !out) return HR_EINVAL;
    const int st = device_status(c);
    Scalars S;
    if (cudaMemcpy(&S, c->B.S, sizeof S, cudaMemcpyDeviceToHost) != cudaSuccess) return HR_ECUDA;
    const double v[14] = {S.t, S.dt, (double)S.step, S.xc, S.yc, S.vproj, S.aproj, S.Fdx,
                          S.Fdy, S.Fwall, S.Wb, S.impulse, S.diss, S.diss_rate};
    for (int k = 0; k < n && k < 14; ++k) out[k] = v[k];
    return st;
}

int hr_case_info(hr_case *c, int64_t *out, int n)
{
    if (!c || !out) return HR_EINVAL;
    const int64_t v[8] = {c->nf, c->nw, c->ng, c->K.ncx, c->K.ncy, c->pass_blocks, c->K.split,
                          c->defer ? 1 : 0};
    for (int k = 0; k < n && k < 8; ++k) out[k] = v[k];
    return HR_OK;
}

int hr_debug_neighbors(hr_case *c, int64_t *offsets, int32_t *ids, int64_t cap, int64_t *n_pairs)
{
    if (!c || !offsets) return HR_EINVAL;
    if (settle(c) != HR_OK) return HR_ECUDA;
    const long long npts = c->nf + c->nw + c->ng;
    int *dcount = nullptr;
    long long *doff = nullptr;
    int *dids = nullptr;
    if (cudaMalloc(&dcount, npts * 4) != cudaSuccess) return HR_ENOMEM;
    const int blocks = (int)((npts + 255) / 256);
    k_neighbors<<<blocks, 256, 0, c->stream>>>(c->K, c->B, dcount, nullptr, nullptr);
    std::vector<int> cnt((size_t)npts);
    std::vector<int> sid((size_t)c->nf);
    int st = device_status(c);
    if (cudaMemcpy(cnt.data(), dcount, npts * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(sid.data(), c->B.s_id, c->nf * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaFree(dcount);
        return HR_ECUDA;
    }
    std::vector<long long> off((size_t)npts + 1, 0);
    for (long long r = 0; r < npts; ++r) off[r + 1] = off[r] + cnt[r];
    const long long total = off[npts];
    if (n_pairs) *n_pairs = total;
    // row index in global point order for each kernel row
    std::vector<long long> grow((size_t)npts);
    for (long long r = 0; r < c->nf; ++r) grow[r] = sid[r];
    for (long long k = 0; k < c->nw; ++k) grow[c->nf + k] = c->nf + c->wall_id_of_sorted[k];
    for (long long k = 0; k < c->ng; ++k) grow[c->nf + c->nw + k] = c->nf + c->nw + k;
    std::vector<long long> goff((size_t)npts + 1, 0);
    for (long long r = 0; r < npts; ++r) goff[grow[r] + 1] = cnt[r];
    for (long long r = 0; r < npts; ++r) goff[r + 1] += goff[r];
    for (long long r = 0; r <= npts; ++r) offsets[r] = goff[r];
    if (!ids) {
        cudaFree(dcount);
        return st;
    }
    if (cap < total) {
        cudaFree(dcount);
        return HR_ERANGE;
    }
    if (cudaMalloc(&doff, (npts + 1) * 8) != cudaSuccess ||
        cudaMalloc(&dids, std::max<long long>(total, 1) * 4) != cudaSuccess) {
        cudaFree(dcount);
        cudaFree(doff);
        return HR_ENOMEM;
    }
    cudaMemcpy(doff, off.data(), (npts + 1) * 8, cudaMemcpyHostToDevice);
    k_neighbors<<<blocks, 256, 0, c->stream>>>(c->K, c->B, dcount, doff, dids);
    st = device_status(c);
    std::vector<int> raw((size_t)std::max<long long>(total, 1));
    const cudaError_t e = cudaMemcpy(raw.data(), dids, total * 4, cudaMemcpyDeviceToHost);
    cudaFree(dcount);
    cudaFree(doff);
    cudaFree(dids);
    if (e != cudaSuccess) return HR_ECUDA;
    for (long long r = 0; r < npts; ++r) {
        int32_t *dst = ids + goff[grow[r]];
        std::memcpy(dst, raw.data() + off[r], (size_t)cnt[r] * 4);
        std::sort(dst, dst + cnt[r]);
    }
    return st;
}

int hr_kernel_times(hr_case *c, float *ms, int n)
{
    if (!c || !ms) return HR_EINVAL;
    if (!c->timing) return HR_EINVAL;
    const int st = device_status(c);
    for (int k = 0; k < n && k < kTimingEvents - 1; ++k)
        if (cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]) != cudaSuccess) return HR_ECUDA;
    return st;
}

// Checkpoint file: magic, counts, params, scalars, state in ID order, probes.
int hr_save_state(hr_case *c, const char *path)
{
    const NvtxRange nvtx_range("hr_save_state");
    if (!c || !path) return HR_EINVAL;
    const int st = device_status(c);
    if (st < 0) return st;
    const size_t n = (size_t)c->nf;
    // ID-order copies through the io buffer
    std::vector<float2> pos(n), vel(n), X(n);
    std::vector<float> d(n);
    std::vector<float4> acc(n);
    std::vector<int> sid(n);
    Scalars S;
    if (cudaMemcpy(sid.data(), c->B.s_id, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pos.data(), c->B.s_pos, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(vel.data(), c->B.st_vel, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(X.data(), c->B.st_X, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(d.data(), c->B.st_rho, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy2D(acc.data(), 16, c->B.st_a, 8, 8, n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy2D(reinterpret_cast<char *>(acc.data()) + 8, 16, c->B.st_D, 8, 8, n,
                     cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&S, c->B.S, sizeof S, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HR_ECUDA;
    std::vector<float2> pos2(n), vel2(n), X2(n);
    std::vector<float> d2(n);
    std::vector<float4> acc2(n);
    for (size_t i = 0; i < n; ++i) {
        const int id = sid[i];
        pos2[id] = pos[i];
        vel2[id] = vel[i];
        X2[id] = X[i];
        d2[id] = d[i];
        acc2[id] = acc[i];
    }
    const long long hn = std::min<long long>(S.hist_n, c->K.probe_cap);
    std::vector<float> ph((size_t)hn * std::max(c->K.n_probes, 1));
    std::vector<double> pt((size_t)hn);
    if (hn > 0 && c->K.n_probes > 0 &&
        (cudaMemcpy(ph.data(), c->B.probe_hist, ph.size() * 4, cudaMemcpyDeviceToHost) !=
             cudaSuccess ||
         cudaMemcpy(pt.data(), c->B.probe_t, pt.size() * 8, cudaMemcpyDeviceToHost) !=
             cudaSuccess))
        return HR_ECUDA;
    FILE *f = std::fopen(path, "wb");
    if (!f) return HR_EIO;
    const char magic[8] = {'H', 'R', 'A', 'M', 'C', 'K', '0', '1'};
    const long long hdr[4] = {c->nf, c->nw, c->ng, hn};
    bool ok = std::fwrite(magic, 8, 1, f) == 1 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(&c->P, sizeof c->P, 1, f) == 1 && std::fwrite(&S, sizeof S, 1, f) == 1 &&
              std::fwrite(pos2.data(), 8, n, f) == n && std::fwrite(vel2.data(), 8, n, f) == n &&
              std::fwrite(d2.data(), 4, n, f) == n && std::fwrite(acc2.data(), 16, n, f) == n &&
              std::fwrite(X2.data(), 8, n, f) == n &&
              std::fwrite(&c->host_step, 8, 1, f) == 1;
    if (ok && hn > 0 && c->K.n_probes > 0)
        ok = std::fwrite(ph.data(), 4, ph.size(), f) == ph.size() &&
             std::fwrite(pt.data(), 8, pt.size(), f) == pt.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? st : HR_EIO;
}

int hr_load_state(hr_case *c, const char *path)
{
    const NvtxRange nvtx_range("hr_load_state");
    if (!c || !path || c->tangent) return HR_EINVAL;
    device_status(c);
    FILE *f = std::fopen(path, "rb");
    if (!f) return HR_EIO;
    char magic[8];
    long long hdr[4];
    hr_params P;
    Scalars S;
    const size_t n = (size_t)c->nf;
    bool ok = std::fread(magic, 8, 1, f) == 1 && std::memcmp(magic, "HRAMCK01", 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, f) == 1 && std::fread(&P, sizeof P, 1, f) == 1 &&
              std::fread(&S, sizeof S, 1, f) == 1;
    ok = ok && hdr[0] == c->nf && hdr[1] == c->nw && hdr[2] == c->ng;
    hr_params a = P, b = c->P;
    a.flags = b.flags = 0;
    a.diag_every = b.diag_every = 0;
    ok = ok && std::memcmp(&a, &b, sizeof a) == 0;
    std::vector<float2> pos(n), vel(n), X(n);
    std::vector<float> d(n);
    std::vector<float4> acc(n);
    long long hstep = 0;
    ok = ok && std::fread(pos.data(), 8, n, f) == n && std::fread(vel.data(), 8, n, f) == n &&
         std::fread(d.data(), 4, n, f) == n && std::fread(acc.data(), 16, n, f) == n &&
         std::fread(X.data(), 8, n, f) == n && std::fread(&hstep, 8, 1, f) == 1;
    const long long hn = ok ? hdr[3] : 0;
    std::vector<float> ph((size_t)hn * std::max(c->K.n_probes, 1));
    std::vector<double> pt((size_t)hn);
    if (ok && hn > 0 && c->K.n_probes > 0)
        ok = std::fread(ph.data(), 4, ph.size(), f) == ph.size() &&
             std::fread(pt.data(), 8, pt.size(), f) == pt.size();
    std::fclose(f);
    if (!ok) return HR_EIO;
    std::vector<int> id(n);
    std::iota(id.begin(), id.end(), 0);
    CK(cudaMemcpy(c->B.s_pos, pos.data(), n * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.st_vel, vel.data(), n * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.st_rho, d.data(), n * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy2D(c->B.st_a, 8, acc.data(), 16, 8, n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy2D(c->B.st_D, 8, reinterpret_cast<const char *>(acc.data()) + 8, 16, 8, n,
                    cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.st_X, X.data(), n * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->B.s_id, id.data(), n * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(c->B.cell_count, 0, ((size_t)c->K.ncell + 1) * 4));
    CK(cudaMemset(c->B.tile_sum, 0, (size_t)c->n_tiles * 4));
    CK(cudaMemset(c->B.fin_ticket, 0, 4));
    CK(cudaMemcpy(c->B.S, &S, sizeof S, cudaMemcpyHostToDevice));
    if (hn > 0 && c->K.n_probes > 0) {
        CK(cudaMemcpy(c->B.probe_hist, ph.data(), ph.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->B.probe_t, pt.data(), pt.size() * 8, cudaMemcpyHostToDevice));
    }
    c->host_step = hstep;
    c->sticky = 0;
    return device_status(c);
}

int hr_tangent_outputs(hr_case *c, double *out, int n)
{
    if (!c || !out || n < 9) return HR_EINVAL;
    if (!c->tangent) return HR_EINVAL;
    const int st = device_status(c);
    if (st < 0) return st;
    double sc[TSC_N];
    Scalars S;
    CK(cudaMemcpy(sc, c->T.sc, sizeof sc, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&S, c->B.S, sizeof S, cudaMemcpyDeviceToHost));
    const bool any = sc[TSC_PSTEP] >= 0.0;
    out[0] = any ? sc[TSC_PEAK] : 0.0;
    for (int k = 0; k < kDir; ++k) out[1 + k] = any ? sc[TSC_DPEAK + k] : 0.0;
    out[4] = S.impulse;
    for (int k = 0; k < kDir; ++k) out[5 + k] = sc[TSC_IMP + k];
    out[8] = any ? sc[TSC_PSTEP] : -1.0;
    return st;
}

int hr_adjoint_forward(hr_case *c, int64_t n_steps, int32_t checkpoint_every, double *out, int n)
{
    const NvtxRange nvtx_range("hr_adjoint_forward");
    if (!c || !out || n < 3 || n_steps < 1 || checkpoint_every < 1) return HR_EINVAL;
    if (c->P.closure != 0 || c->P.dt_mode != 1 || c->P.motion < 0 || c->P.motion > 2 || c->tangent)
        return HR_EINVAL;
    if (c->K.sr != 1 || c->n3 || c->lanes != 1)   // the records take the plain pass's sums
        return HR_EINVAL;
    if (c->K.n_probes < 1 || n_steps > c->K.probe_cap) return HR_EINVAL;
    int st = device_status(c);
    if (st < 0) return st;
    Scalars S0;
    CK(cudaMemcpy(&S0, c->B.S, sizeof S0, cudaMemcpyDeviceToHost));
    if (S0.step != 0) return HR_EINVAL;   // from the uploaded state only
    int rc = adj_alloc(c, n_steps, checkpoint_every);
    if (rc != HR_OK) return rc;
    AdjCtx *a = c->adj;
    cudaStream_t s = c->stream;
    // the uploaded state, and the priming pass recorded from it: checkpoint 0
    ka_to_id_order<<<c->drift_blocks, 256, 0, s>>>(c->K, c->B, a->upload);
    CK(cudaGetLastError());
    if ((rc = launch_tape_step(c, s, a->prime_slot, a->upload, 1)) != HR_OK) return rc;
    // the forward run on the case's own step graph, a checkpoint every L
    // steps; the last segment is recorded on the tape as it runs, so the
    // reverse sweep starts without recomputing it (not with periodic
    // diagnostics, which only the step graph takes)
    const long long last = ((n_steps - 1) / a->L) * a->L;   // the last segment's first step
    a->taped_last = c->P.diag_every <= 0;
    const long long plain_end = a->taped_last ? last : n_steps;
    long long done = 0;
    while (done < plain_end) {
        const long long k = std::min<long long>(a->L, plain_end - done);
        if ((rc = run_steps(c, k)) != HR_OK) return rc;
        if ((rc = settle(c)) != HR_OK) return rc;   // the checkpoint takes the scalars
        done += k;
        if (done < n_steps && (rc = save_ckpt(c, a->ckpt[done / a->L], s)) != HR_OK) return rc;
    }
    if (a->taped_last) {
        const long long len = n_steps - last;
        if ((rc = load_start(c, a->ckpt[(size_t)(last / a->L)], s)) != HR_OK) return rc;
        for (long long k = 0; k < len; ++k) {
            const Slot &prev = k == 0 ? a->start : a->tape[(size_t)(k - 1)];
            if ((rc = launch_tape_step(c, s, a->tape[(size_t)k], prev, 0)) != HR_OK) return rc;
        }
        if ((rc = tape_to_live(c, a->tape[(size_t)(len - 1)], s)) != HR_OK) return rc;
        c->host_step += len;
    }
    if ((rc = settle(c)) != HR_OK) return rc;
    CK(cudaMemcpyAsync(a->S_final, c->B.S, sizeof(Scalars), cudaMemcpyDeviceToDevice, s));
    st = device_status(c);
    if (st < 0) return st;
    // the peak of probe 0 over the run and its row (the first of equal maxima)
    const int np = c->K.n_probes;
    std::vector<float> hist((size_t)n_steps * (size_t)np);
    CK(cudaMemcpy(hist.data(), c->B.probe_hist, hist.size() * 4, cudaMemcpyDeviceToHost));
    double peak = -HUGE_VAL;
    long long row = -1;
    for (long long k = 0; k < n_steps; ++k)
        if ((double)hist[(size_t)k * np] > peak) {
            peak = hist[(size_t)k * np];
            row = k;
        }
    Scalars Sf;
    CK(cudaMemcpy(&Sf, c->B.S, sizeof Sf, cudaMemcpyDeviceToHost));
    a->peak = peak;
    a->peak_row = row;
    a->impulse = Sf.impulse;
    a->forward_done = true;
    out[0] = peak;
    out[1] = Sf.impulse;
    out[2] = (double)row;
    return st;
}

int hr_adjoint_backward(hr_case *c, double *out, int n)
{
    const NvtxRange nvtx_range("hr_adjoint_backward");
    if (!c || !out || n < 6 || !c->adj || !c->adj->forward_done) return HR_EINVAL;
    if (c->sticky < 0) return c->sticky;
    AdjCtx *a = c->adj;
    cudaStream_t s = c->stream;
    const size_t nq = (size_t)c->nf * kOut;
    a->A.cur = a->ls[0];
    a->A.prv = a->ls[1];
    const LState &z = a->A.cur;
    for (float2 *p : {z.r, z.v, z.a, z.X}) CK(cudaMemsetAsync(p, 0, nq * 8, s));
    for (float *p : {z.d, z.D, z.E}) CK(cudaMemsetAsync(p, 0, nq * 4, s));
    CK(cudaMemsetAsync(a->A.sc, 0, ASC_N * 8, s));
    CK(cudaMemsetAsync(a->A.ctick, 0, 4, s));
    const long long N = a->n_steps;
    const int L = a->L;
    int rc;
    for (long long seg = (N + L - 1) / L - 1; seg >= 0; --seg) {
        const long long base = seg * L, len = std::min<long long>(N, base + L) - base;
        // the segment's records recomputed from its checkpoint, then swept
        // backwards (a full segment is one graph launch)
        const bool recompute = !(a->taped_last && base + len == N);
        if (recompute) a->taped_last = false;   // the tape is overwritten from here on
        if ((rc = load_start(c, a->ckpt[(size_t)seg], s)) != HR_OK) return rc;
        rc = len == L ? run_full_segment(c, s, recompute) : launch_segment(c, s, len, recompute);
        if (rc != HR_OK) return rc;
    }
    // the priming pass (a0, D0, X0 of the uploaded state)
    if ((rc = adjoint_step(c, s, a->prime_slot, a->upload, 1, false)) != HR_OK) return rc;
    // the case goes on from the end of the forward run
    CK(cudaMemcpyAsync(c->B.S, a->S_final, sizeof(Scalars), cudaMemcpyDeviceToDevice, s));
    const int st = device_status(c);
    if (st < 0) return st;
    double sc[ASC_N];
    CK(cudaMemcpy(sc, a->A.sc, sizeof sc, cudaMemcpyDeviceToHost));
    // every step's dt = C h / (c0 + v0): d dt / d ln c0 = -dt c0 / (c0 + v0)
    const double dtdc = -c->K.dt_fixed * c->P.c0 / (c->P.c0 + c->P.v0);
    for (int q = 0; q < kOut; ++q) {
        out[3 * q + 0] = sc[ASC_ALPHA + q];
        out[3 * q + 1] = sc[ASC_C0 + q] + sc[ASC_DT + q] * dtdc;
        out[3 * q + 2] = sc[ASC_TAU + q];
    }
    return st;
}

int hr_fp32_rate(int packed, void *cuda_stream, double *tflops)
{
    if (!tflops) return HR_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HR_ECUDA;
    const int threads = 256, blocks = sms * 8, iters = 1 << 14;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HR_OK;
    if (cudaMalloc(&out, (size_t)blocks * threads * 4) != cudaSuccess) {
        cudaGetLastError();
        return HR_ENOMEM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = HR_ECUDA;
    } else {
        k_fma_rate<<<blocks, threads, 0, s>>>(out, iters / 16, packed ? 1 : 0);   // warm-up
        cudaEventRecord(e0, s);
        k_fma_rate<<<blocks, threads, 0, s>>>(out, iters, packed ? 1 : 0);
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f)) {
            rc = HR_ECUDA;
        } else {
            const double flop = 2.0 * kFmaChains * (double)iters * blocks * threads;
            *tflops = flop / (ms * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

int hr_neighbor_counts_static(hr_case *c, int32_t *host_counts, int64_t cap)
{
    if (!c || !host_counts) return HR_EINVAL;
    const long long npts = c->nf + c->nw + c->ng;
    if (npts > HR_STATIC_NEIGHBOR_MAX) return HR_ERANGE;
    if (cap < npts) return HR_ERANGE;
    // the array's address is per device: the case's device must be current
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return HR_ECUDA;
    if (dev != c->device) return HR_EINVAL;
    int *counts = nullptr;
    const int rc = static_counts_address(dev, &counts);
    if (rc != HR_OK) return rc;
    const int blocks = (int)((npts + 255) / 256);
    k_neighbor_counts_static<<<blocks, 256, 0, c->stream>>>(c->K, c->B, counts);
    if (cudaGetLastError() != cudaSuccess) return HR_ECUDA;
    if (cudaMemcpyAsync(host_counts, counts, (size_t)npts * sizeof(int), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess)
        return HR_ECUDA;
    return device_status(c);
}

// ------------------------------------------------------------ batches

namespace {

// BK_PASS maps the cases on the 3 x 3 stencil, BK_PASS5 those on the 5 x 5
enum BatchKernel { BK_KIN, BK_DRIFT, BK_APPLY, BK_SLOT, BK_RANK, BK_GHOST, BK_PASS, BK_FIN, BK_DENS,
                   BK_PASS5 };
constexpr int kBatchKernels = 10;

__global__ void k_batch_count_done(const Bufs *Bs, int n, int *out)
{
    int d = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) d += __ldcg(&Bs[c].S->done);
    d = warp_sum(d);
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        *out = t;
    }
}

// The batch's cases with a step close still pending from their own step
// graphs: settled on their streams and waited for, before the batch reads
// or steps them on its own stream.
int settle_cases(hr_batch *b)
{
    for (hr_case *c : b->cases) {
        if (!c->pending) continue;
        const int rc = settle(c);
        if (rc != HR_OK) return rc;
        CK(cudaStreamSynchronize(c->stream));
    }
    return HR_OK;
}

int batch_launch(hr_batch *b, cudaStream_t s, cudaStream_t side)
{
    const Consts *K = b->dK;
    const Bufs *B = b->dB;
    CK(cudaEventRecord(b->fork, s));
    CK(cudaStreamWaitEvent(side, b->fork, 0));
    kb_kinematics<<<b->nblocks[BK_KIN], 128, 0, side>>>(K, B, b->map[BK_KIN]);
    CK(cudaEventRecord(b->join, side));
    kb_drift_key<<<b->nblocks[BK_DRIFT], 256, 0, s>>>(K, B, b->map[BK_DRIFT]);
    kb_scan_apply<<<b->nblocks[BK_APPLY], kScanThreads, 0, s>>>(K, B, b->map[BK_APPLY]);
    if (b->closure == 1) {
        kb_rank_scatter<1><<<b->nblocks[BK_RANK], 256, 0, s>>>(K, B, b->map[BK_RANK]);
        CK(cudaStreamWaitEvent(s, b->join, 0));
        kb_density<<<b->nblocks[BK_DENS], 256, 0, s>>>(K, B, b->map[BK_DENS]);
        kb_ghost<1><<<b->nblocks[BK_GHOST], kGhostWarps * 32, 0, s>>>(K, B, b->map[BK_GHOST]);
        if (b->nblocks[BK_PASS])
            kb_pass<1, 1><<<b->nblocks[BK_PASS], kPassThreads, 0, s>>>(K, B, b->map[BK_PASS]);
        if (b->nblocks[BK_PASS5])
            kb_pass<1, 2><<<b->nblocks[BK_PASS5], kPassThreads, 0, s>>>(K, B, b->map[BK_PASS5]);
        kb_finalize<1><<<b->nblocks[BK_FIN], kFinalizeThreads, 0, s>>>(K, B, b->map[BK_FIN]);
    } else {
        kb_rank_scatter<0><<<b->nblocks[BK_RANK], 256, 0, s>>>(K, B, b->map[BK_RANK]);
        CK(cudaStreamWaitEvent(s, b->join, 0));
        kb_ghost<0><<<b->nblocks[BK_GHOST], kGhostWarps * 32, 0, s>>>(K, B, b->map[BK_GHOST]);
        if (b->nblocks[BK_PASS])
            kb_pass<0, 1><<<b->nblocks[BK_PASS], kPassThreads, 0, s>>>(K, B, b->map[BK_PASS]);
        if (b->nblocks[BK_PASS5])
            kb_pass<0, 2><<<b->nblocks[BK_PASS5], kPassThreads, 0, s>>>(K, B, b->map[BK_PASS5]);
        kb_finalize<0><<<b->nblocks[BK_FIN], kFinalizeThreads, 0, s>>>(K, B, b->map[BK_FIN]);
    }
    CK(cudaGetLastError());
    return HR_OK;
}

}  // namespace

int hr_batch_create(hr_case *const *cases, int n_cases, double t_end, int schedule,
                    void *cuda_stream, hr_batch **out)
{
    if (!out || !cases || n_cases <= 0 || schedule < 0 || schedule > 2) return HR_EINVAL;
    *out = nullptr;
    hr_batch *b = new hr_batch();
    auto fail = [&](int code) {
        hr_batch_destroy(b);
        return code;
    };
    for (int k = 0; k < n_cases; ++k) {
        // one closure per batch (the kernels are templated on it); no tangents
        if (!cases[k] || cases[k]->sticky < 0 || cases[k]->tangent || cases[k]->n3 ||
            cases[k]->lanes != 1 ||
            cases[k]->K.closure != cases[0]->K.closure)
            return fail(HR_EINVAL);
        b->cases.push_back(cases[k]);
    }
    if (settle_cases(b) != HR_OK) return fail(HR_ECUDA);
    b->stream = (cudaStream_t)cuda_stream;
    // per-kernel block maps: (case, local block, blocks of that case), in the
    // order of the schedule: 0 case after case, 1 round robin over the cases,
    // 2 case after case from the largest case down
    b->closure = cases[0]->K.closure;
    std::vector<BatchBlock> maps[kBatchKernels];
    std::vector<int> order(n_cases);
    std::iota(order.begin(), order.end(), 0);
    if (schedule == 2)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return cases[a]->nf > cases[c]->nf; });
    auto nblk = [&](int k, int q) {
        const hr_case *c = cases[k];
        const int fin = 4 + c->K.n_probes;  // four reduction blocks, one per probe
        const int p3 = c->K.sr == 1 ? c->pass_blocks : 0, p5 = c->K.sr == 2 ? c->pass_blocks : 0;
        const int nb[kBatchKernels] = {1, c->drift_blocks, c->n_tiles, 0 /* no slot kernel */,
                                       c->drift_blocks, c->ghost_blocks, p3, fin,
                                       c->drift_blocks, p5};
        return nb[q];
    };
    for (int q = 0; q < kBatchKernels; ++q) {
        if (schedule == 1) {
            int most = 0;
            for (int k = 0; k < n_cases; ++k) most = std::max(most, nblk(k, q));
            for (int j = 0; j < most; ++j)
                for (int k = 0; k < n_cases; ++k)
                    if (j < nblk(k, q)) maps[q].push_back(BatchBlock{k, j, nblk(k, q), 0});
        } else {
            for (int k : order)
                for (int j = 0; j < nblk(k, q); ++j)
                    maps[q].push_back(BatchBlock{k, j, nblk(k, q), 0});
        }
    }
    size_t bytes = align256(sizeof(Consts) * n_cases) + align256(sizeof(Bufs) * n_cases) + 256;
    size_t off[kBatchKernels];
    for (int q = 0; q < kBatchKernels; ++q) {
        off[q] = bytes;
        bytes += align256(maps[q].size() * sizeof(BatchBlock));
    }
    if (cudaMalloc(&b->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        b->mem = nullptr;
        return fail(HR_ENOMEM);
    }
    b->dK = at<Consts>(b->mem, 0);
    b->dB = at<Bufs>(b->mem, align256(sizeof(Consts) * n_cases));
    b->d_count = at<int>(b->mem, align256(sizeof(Consts) * n_cases) + align256(sizeof(Bufs) * n_cases));
    std::vector<Consts> hk(n_cases);
    std::vector<Bufs> hb(n_cases);
    for (int k = 0; k < n_cases; ++k) {
        hk[k] = cases[k]->K;
        hk[k].split = 0;   // batched steps take the one-kernel pass
        hb[k] = cases[k]->B;
    }
    if (cudaMemcpy(b->dK, hk.data(), sizeof(Consts) * n_cases, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->dB, hb.data(), sizeof(Bufs) * n_cases, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HR_ECUDA);
    for (int q = 0; q < kBatchKernels; ++q) {
        b->map[q] = at<BatchBlock>(b->mem, off[q]);
        b->nblocks[q] = (int)maps[q].size();
        if (cudaMemcpy(b->map[q], maps[q].data(), maps[q].size() * sizeof(BatchBlock),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HR_ECUDA);
    }
    // every case stops at t_end
    for (int k = 0; k < n_cases; ++k) {
        hr_case *c = cases[k];
        if (device_status(c) < 0) return fail(c->sticky);
        Scalars S;
        if (cudaMemcpy(&S, c->B.S, sizeof S, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(HR_ECUDA);
        S.t_end = t_end;
        S.done = (t_end > 0.0 && S.t >= t_end) ? 1 : 0;
        if (cudaMemcpy(c->B.S, &S, sizeof S, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HR_ECUDA);
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(HR_ECUDA);
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(HR_ECUDA);
    const int rc = batch_launch(b, b->cap, b->cap2);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc != HR_OK || e != cudaSuccess) return fail(HR_ECUDA);
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return fail(HR_ECUDA);
    *out = b;
    return HR_OK;
}

int hr_persist_capacity(int closure, int32_t *max_blocks)
{
    if (!max_blocks || closure < 0 || closure > 1) return HR_EINVAL;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    *max_blocks = persist_blocks_per_sm(closure) * sms;
    return *max_blocks > 0 ? HR_OK : HR_ECUDA;
}

int hr_batch_create_persistent(hr_case *const *cases, int n_cases, double t_end,
                               const int32_t *case_blocks, int64_t spin_limit, void *cuda_stream,
                               hr_batch **out)
{
    if (!out || !cases || n_cases <= 0 || !(t_end > 0.0)) return HR_EINVAL;
    *out = nullptr;
    hr_batch *b = new hr_batch();
    auto fail = [&](int code) {
        hr_batch_destroy(b);
        return code;
    };
    for (int k = 0; k < n_cases; ++k) {
        if (!cases[k] || cases[k]->sticky < 0 || cases[k]->tangent || cases[k]->n3 ||
            cases[k]->lanes != 1 ||
            cases[k]->K.closure != cases[0]->K.closure || cases[k]->K.sr != 1)
            return fail(HR_EINVAL);
        b->cases.push_back(cases[k]);
    }
    if (settle_cases(b) != HR_OK) return fail(HR_ECUDA);
    b->stream = (cudaStream_t)cuda_stream;
    b->closure = cases[0]->K.closure;
    b->persistent = true;
    b->spin_limit = spin_limit > 0 ? spin_limit : (1LL << 24);
    int32_t cap = 0;
    int rc = hr_persist_capacity(b->closure, &cap);
    if (rc != HR_OK) return fail(rc);
    // blocks per case: as given, else in proportion to the particle counts
    std::vector<int> nb(n_cases);
    if (case_blocks) {
        for (int k = 0; k < n_cases; ++k) nb[k] = case_blocks[k];
    } else {
        long long tot = 0;
        for (hr_case *c : b->cases) tot += c->nf;
        for (int k = 0; k < n_cases; ++k)
            nb[k] = std::max(1, (int)((double)cap * (double)cases[k]->nf / (double)tot));
    }
    long long total = 0;
    for (int k = 0; k < n_cases; ++k) {
        if (nb[k] < 1) return fail(HR_EINVAL);
        total += nb[k];
    }
    if (total > cap) return fail(HR_EINVAL);   // every block must stay resident
    b->nblk_total = (int)total;
    std::vector<int2> blk;
    for (int k = 0; k < n_cases; ++k)
        for (int r = 0; r < nb[k]; ++r) blk.push_back(make_int2(k, r));
    const size_t bytes = align256(sizeof(Consts) * n_cases) + align256(sizeof(Bufs) * n_cases) +
                         align256(blk.size() * sizeof(int2)) + align256(n_cases * 4) +
                         align256(n_cases * 8) + 256 + 256;
    if (cudaMalloc(&b->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        b->mem = nullptr;
        return fail(HR_ENOMEM);
    }
    size_t off = 0;
    b->dK = at<Consts>(b->mem, off);
    off += align256(sizeof(Consts) * n_cases);
    b->dB = at<Bufs>(b->mem, off);
    off += align256(sizeof(Bufs) * n_cases);
    b->blk = at<int2>(b->mem, off);
    off += align256(blk.size() * sizeof(int2));
    b->case_nblk = at<int>(b->mem, off);
    off += align256(n_cases * 4);
    b->bar = at<int>(b->mem, off);
    off += align256(n_cases * 8);
    b->err = at<int>(b->mem, off);
    off += 256;
    b->d_count = at<int>(b->mem, off);
    std::vector<Consts> hk(n_cases);
    std::vector<Bufs> hb(n_cases);
    for (int k = 0; k < n_cases; ++k) {
        hk[k] = cases[k]->K;
        hk[k].n_probes = cases[k]->K.n_probes;
        hk[k].split = 0;   // the persistent batch takes the one-kernel pass
        hb[k] = cases[k]->B;
    }
    if (cudaMemcpy(b->dK, hk.data(), sizeof(Consts) * n_cases, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->dB, hb.data(), sizeof(Bufs) * n_cases, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->blk, blk.data(), blk.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->case_nblk, nb.data(), n_cases * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->bar, 0, n_cases * 8) != cudaSuccess || cudaMemset(b->err, 0, 4) != cudaSuccess)
        return fail(HR_ECUDA);
    for (int k = 0; k < n_cases; ++k) {
        hr_case *c = cases[k];
        if (device_status(c) < 0) return fail(c->sticky);
        Scalars S;
        if (cudaMemcpy(&S, c->B.S, sizeof S, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(HR_ECUDA);
        S.t_end = t_end;
        S.done = S.t >= t_end ? 1 : 0;
        if (cudaMemcpy(c->B.S, &S, sizeof S, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(HR_ECUDA);
    }
    *out = b;
    return HR_OK;
}

// One persistent launch of up to max_steps steps of every case (<= 0: until
// every case is done).  A wait that ran past the spin limit leaves the cases
// mid-step: they are marked HR_ETIMEOUT.
static int persist_run(hr_batch *b, int64_t max_steps)
{
    for (hr_case *c : b->cases)
        if (c->sticky < 0) return c->sticky;
    if (cudaMemsetAsync(b->err, 0, 4, b->stream) != cudaSuccess) return HR_ECUDA;
    if (persist_launch(b->dK, b->dB, b->blk, b->case_nblk, b->nblk_total, b->bar, b->spin_limit,
                       max_steps > 0 ? max_steps : (1LL << 60), b->err, b->closure, b->stream) != 0) {
        cudaGetLastError();
        return HR_ECUDA;
    }
    int err = 0;
    if (cudaMemcpyAsync(&err, b->err, 4, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return HR_ECUDA;
    if (err) {
        for (hr_case *c : b->cases) c->sticky = HR_ETIMEOUT;
        return HR_ETIMEOUT;
    }
    return HR_OK;
}

int hr_batch_step(hr_batch *b)
{
    const NvtxRange nvtx_range("hr_batch_step");
    if (b && settle_cases(b) != HR_OK) return HR_ECUDA;
    if (b && b->persistent) {
        const int rc = persist_run(b, 1);
        if (rc == HR_OK) b->steps++;
        return rc;
    }
    if (!b || !b->exec) return HR_EINVAL;
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return HR_ECUDA;
    b->steps++;
    return HR_OK;
}

int hr_batch_done(hr_batch *b, int *n_done)
{
    if (!b || !n_done) return HR_EINVAL;
    k_batch_count_done<<<1, 256, 0, b->stream>>>(b->dB, (int)b->cases.size(), b->d_count);
    if (cudaMemcpyAsync(n_done, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return HR_ECUDA;
    return HR_OK;
}

int hr_batch_run(hr_batch *b, int64_t max_steps, int64_t *steps_done)
{
    const NvtxRange nvtx_range("hr_batch_run");
    if (!b) return HR_EINVAL;
    if (settle_cases(b) != HR_OK) return HR_ECUDA;
    const int n = (int)b->cases.size();
    int64_t done_steps = 0;
    int rc = HR_OK;
    if (b->persistent) {
        // the launch runs every case to its stop time (or max_steps steps)
        std::vector<long long> before(n);
        for (int k = 0; k < n; ++k) {
            Scalars S;
            CK(cudaMemcpy(&S, b->cases[k]->B.S, sizeof S, cudaMemcpyDeviceToHost));
            before[k] = S.step;
        }
        rc = persist_run(b, max_steps);
        if (rc != HR_OK) return rc;
        for (int k = 0; k < n; ++k) {
            Scalars S;
            CK(cudaMemcpy(&S, b->cases[k]->B.S, sizeof S, cudaMemcpyDeviceToHost));
            done_steps = std::max<int64_t>(done_steps, S.step - before[k]);
        }
        b->steps += done_steps;
        if (steps_done) *steps_done = done_steps;
        int worst = HR_OK;
        for (hr_case *c : b->cases) {
            const int st = device_status(c);
            if (st < 0) return st;
            worst |= st;
        }
        return worst;
    }
    for (;;) {
        int nd = 0;
        if ((rc = hr_batch_done(b, &nd)) != HR_OK) break;
        if (nd >= n || (max_steps > 0 && done_steps >= max_steps)) break;
        int64_t k = 64;
        if (max_steps > 0) k = std::min<int64_t>(k, max_steps - done_steps);
        for (int64_t q = 0; q < k; ++q)
            if ((rc = hr_batch_step(b)) != HR_OK) break;
        if (rc != HR_OK) break;
        done_steps += k;
    }
    if (steps_done) *steps_done = done_steps;
    if (rc != HR_OK) return rc;
    int worst = HR_OK;
    for (hr_case *c : b->cases) {
        const int st = device_status(c);
        if (st < 0) return st;
        worst |= st;
    }
    return worst;
}

void hr_batch_destroy(hr_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->mem) cudaFree(b->mem);
    delete b;
}

void hr_destroy(hr_case *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->exec_multi) cudaGraphExecDestroy(c->exec_multi);
    if (c->graph_multi) cudaGraphDestroy(c->graph_multi);
    for (int k = 0; k < kTimingEvents; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->fork2) cudaEventDestroy(c->fork2);
    if (c->join2) cudaEventDestroy(c->join2);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    adj_free(c);
    delete c;
}

const char *hr_status_str(int s)
{
    switch (s) {
    case HR_OK: return "ok";
    case HR_EINVAL: return "invalid argument";
    case HR_ENOMEM: return "out of device memory or workspace too small";
    case HR_ECUDA: return "CUDA error";
    case HR_ENAN: return "NaN or Inf in the fluid state";
    case HR_EDT: return "time step underflow";
    case HR_ERANGE: return "buffer too small";
    case HR_EIO: return "checkpoint file error";
    case HR_ECHECK: return "an index check of the bounds-checked build failed";
    case HR_ETIMEOUT: return "a bounded device wait gave up (persistent batch)";
    default: break;
    }
    if (s > 0) return "warning (see HR_W* bits)";
    return "unknown status";
}

}  // extern "C"
