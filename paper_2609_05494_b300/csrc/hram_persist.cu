// hram_persist.cu -- the batched coefficient sweep as one persistent launch.
//
// Every case of a batch gets a fixed set of thread blocks (its share of the
// GPU, chosen by the host's autotuner); all blocks stay resident for the
// whole run (cooperative launch).  A case's blocks advance that case through
// the stages of each step in order -- kinematics and drift, cell scan, stable
// reorder, (summed density,) ghosts, interaction pass, closing reduction --
// and meet at a per-case barrier between stages,
// so cases of different sizes and time steps run at their own pace with no
// grid-wide synchronisation.  A case whose time reaches its stop time leaves
// the loop; the launch ends when every case has.
//
// The stage bodies are the ones of the per-step kernels (hram_device.cuh),
// so a case ends bit for bit where it ends when run alone.  This translation
// unit reads the arrays a step rewrites with plain loads: within one launch
// those arrays change every step, so the read-only data path (which may keep
// a line from an earlier step) must not be used for them.
//
// Every wait is bounded: a block that spins more than spin_limit times at a
// barrier, or that sees another block's failure, records it in *err and
// leaves, so a launch always ends; the host reports HR_ETIMEOUT.
#define HR_DYNAMIC_LOAD(p) (*(p))
#define HR_NO_STEP_KERNELS
#include "hram_device.cuh"
#include "hram_persist.h"

namespace hr {

constexpr int kPersistThreads = 256;

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the nb blocks of one case (cnt, gen: the case's counter and
// generation).  Returns false, for every thread of the block, when the batch
// has failed (a wait ran past spin_limit here or elsewhere).
__device__ __forceinline__ bool case_barrier(int *cnt, int *gen, int nb, long long spin_limit, int *err,
                                             int *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const int g = ld_acquire(gen);
        __threadfence();
        if (atomicAdd(cnt, 1) == nb - 1) {
            atomicExch(cnt, 0);
            __threadfence();
            st_release(gen, g + 1);
        } else {
            long long it = 0;
            while (ld_acquire(gen) == g) {
                if (ld_acquire(err) != 0 || ++it > spin_limit) {
                    atomicOr(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *flag = ok && ld_acquire(err) == 0;
    }
    __syncthreads();
    return *flag != 0;
}

// Cell starts of scan tile bx (kScanTile cells) by one 256-thread block:
// the sums of the tiles before it (counted by the drift) plus an exclusive
// scan of its own cells, which it resets for the next step.  The same
// integers as b_scan_apply (a 1,024-thread block per tile).
__device__ __forceinline__ void scan_tile(const Consts &K, const Bufs &B, int bx)
{
    constexpr int kItems = kScanTile / kPersistThreads;
    __shared__ int wsum[kPersistThreads / 32];
    __shared__ int offset;
    int o = 0;
    for (int t = threadIdx.x; t < bx; t += blockDim.x) o += B.tile_sum[t];
    o = warp_sum(o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = o;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < kPersistThreads / 32; ++k) t += wsum[k];
        offset = t;
    }
    __syncthreads();
    const int n = K.ncell + 1;
    const int base = bx * kScanTile + threadIdx.x * kItems;
    int v[kItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = (base + k < n) ? B.cell_count[base + k] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan(s, wsum, &total) + offset;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) {
            B.cell_start[base + k] = ex;
            B.cell_count[base + k] = 0;
        }
        ex += v[k];
    }
    if (base <= n && n < base + kItems) B.cell_start[n] = K.nf;
    scan_overflow(K, B, bx * kScanTile, min((bx + 1) * kScanTile, n), *B.ovf_count);
    __syncthreads();
}

// Two 128-particle pass blocks (pass block indices 2 q and 2 q + 1) in one
// 256-thread block, with the partials of each half formed as the
// 128-thread kernel forms them (warp sums, then the half's four warps in
// order; the dissipation as its interior and boundary shares).
template <int CL>
__device__ __forceinline__ void pass_pair(const Consts &K, const Bufs &B, int q)
{
    __shared__ float red[kPersistThreads / 32][6];
    __shared__ int redn[kPersistThreads / 32];
    const int i = q * kPersistThreads + threadIdx.x;
    const float dt = B.S->dt_f;
    PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (i < K.nf) pass_single<CL, 1>(K, B, i, dt, 0, P);   // 3 x 3 stencil (cell_factor >= 1)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float da = P.def ? 0.f : P.diss, db = P.def ? P.diss : 0.f;
    if (__any_sync(0xffffffffu, P.fdx != 0.f || P.fdy != 0.f || P.fw != 0.f || P.npen != 0 || P.def)) {
        P.fdx = warp_sum(P.fdx);
        P.fdy = warp_sum(P.fdy);
        P.fw = warp_sum(P.fw);
        P.npen = warp_sum(P.npen);
        db = warp_sum(db);
    }
    da = warp_sum(da);
    P.vmax = warp_max(P.vmax);
    if (lane == 0) {
        red[w][0] = P.fdx;
        red[w][1] = P.fdy;
        red[w][2] = P.fw;
        red[w][3] = da;
        red[w][4] = P.vmax;
        red[w][5] = db;
        redn[w] = P.npen;
    }
    __syncthreads();
    constexpr int NW = kPassThreads / 32;
    if ((threadIdx.x & (kPassThreads - 1)) == 0) {
        const int half = threadIdx.x / kPassThreads;
        const int bx = 2 * q + half;
        if (bx < K.n_pass_blocks) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a5 = 0.f, v = 0.f;
            int np = 0;
            for (int k = half * NW; k < half * NW + NW; ++k) {
                a0 += red[k][0];
                a1 += red[k][1];
                a2 += red[k][2];
                a3 += red[k][3];
                a5 += red[k][5];
                v = fmaxf(v, red[k][4]);
                np += redn[k];
            }
            B.part.f[bx] = make_float4(a0, a1, a2, a3 + a5);
            B.part.vmax[bx] = v;
            B.part.npen[bx] = np;
        }
    }
    __syncthreads();
}

template <int CL>
__global__ void __launch_bounds__(kPersistThreads) kp_batch(const Consts *Ks, const Bufs *Bs,
                                                            const int2 *blk, const int *case_nblk,
                                                            int *bar, long long spin_limit,
                                                            long long max_steps, int *err)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ int flag;
    __shared__ int done;
    const int2 me = blk[blockIdx.x];   // (case, rank in the case)
    const int c = me.x, r = me.y;
    const int nb = case_nblk[c];
    {
        const int *ks = reinterpret_cast<const int *>(Ks + c);
        for (int k = threadIdx.x; k < (int)(sizeof(Consts) / 4); k += blockDim.x)
            reinterpret_cast<int *>(&K)[k] = ks[k];
        const unsigned long long *bs = reinterpret_cast<const unsigned long long *>(Bs + c);
        for (int k = threadIdx.x; k < (int)(sizeof(Bufs) / 8); k += blockDim.x)
            reinterpret_cast<unsigned long long *>(&B)[k] = bs[k];
    }
    __syncthreads();
    int *cnt = bar + 2 * c, *gen = bar + 2 * c + 1;
    const int n256 = (K.nf + kPersistThreads - 1) / kPersistThreads;
    const int nfin = kFinalizeBlocks + K.n_probes;
#pragma unroll 1
    for (long long step = 0; step < max_steps; ++step) {
        if (threadIdx.x == 0) done = ld_acquire(&B.S->done);
        __syncthreads();
        if (done) break;
        for (int vb = r; vb < n256; vb += nb) b_drift_key(K, B, vb, n256, 0);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        // the scan tiles, and the kinematics (needed from the ghost stage on)
        // by a block with no tile, or the last one, off the drift's path
        const int n_tiles = (K.ncell + 2 + kScanTile - 1) / kScanTile;
        for (int vb = r; vb < n_tiles; vb += nb) scan_tile(K, B, vb);
        if (r == (n_tiles < nb ? n_tiles : nb - 1)) b_kinematics(K, B, 0, 1, 0);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        for (int vb = r; vb < n256; vb += nb) b_rank_scatter<CL>(K, B, vb, n256, 0);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        if constexpr (CL == 1) {
            for (int vb = r; vb < n256; vb += nb) b_density(K, B, vb, n256, 0);
            if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        }
        for (int vb = r; vb < K.n_ghost_blocks; vb += nb) b_ghost<CL>(K, B, vb, K.n_ghost_blocks);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        for (int q = r; q < n256; q += nb) pass_pair<CL>(K, B, q);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
        for (int vb = r; vb < nfin; vb += nb) b_finalize<CL, true>(K, B, vb, nfin, 0);
        if (!case_barrier(cnt, gen, nb, spin_limit, err, &flag)) return;
    }
}

int persist_blocks_per_sm(int closure)
{
    int n = 0;
    const cudaError_t e = closure == 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_batch<1>, kPersistThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_batch<0>, kPersistThreads, 0);
    return e == cudaSuccess ? n : 0;
}

int persist_launch(const Consts *dK, const Bufs *dB, const int2 *blk, const int *case_nblk, int nblk,
                   int *bar, long long spin_limit, long long max_steps, int *err, int closure,
                   cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblk);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all blocks resident, or no launch
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        closure == 1 ? cudaLaunchKernelEx(&cfg, kp_batch<1>, dK, dB, blk, case_nblk, bar, spin_limit,
                                          max_steps, err)
                     : cudaLaunchKernelEx(&cfg, kp_batch<0>, dK, dB, blk, case_nblk, bar, spin_limit,
                                          max_steps, err);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace hr
