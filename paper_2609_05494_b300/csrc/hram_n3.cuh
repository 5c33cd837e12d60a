// hram_n3.cuh -- the interaction pass with each fluid pair evaluated once
// (a measured variant, HR_FLAG_NEWTON3; closure 0, single-case steps).
//
// The pair terms of Section 2.2 are antisymmetric (pressure, viscous and
// laminar force, the XSPH sum of eq. xsph) or symmetric (the continuity
// rate) in the pair, so one evaluation serves both particles.  Every pair
// {i, j} is evaluated by the particle that comes first in the half stencil:
// i takes j when j lies later in i's own row of cells (cells c and c + 1,
// j > i in the sorted order) or anywhere in the three cells of the row above
// (c + ncx - 1 .. c + ncx + 1).  Work is split into tiles: runs of up to 128
// consecutive particles of one cell row (the tile table is built from the
// cell starts each step, by the first block of k_rank_scatter).
//
// The sums stay deterministic, with no floating-point atomics:
//  A. each thread evaluates its particle's half-stencil pairs, adds its own
//     side to registers and writes the neighbour's side {f, F v.r, w_X} to
//     the tile's shared pair buffer, at the rank of the pair in the thread's
//     candidate masks (a block scan of the pair counts gives each thread its
//     start);
//  B. every target particle of the tile -- its own particles, the rest of
//     the row up to the last cell + 1, and the three-cell span of the row
//     above -- sums its side of the tile's pairs in ascending order of the
//     evaluating particle, found from the stored masks (a bit test, then a
//     popcount for the rank).  A tile's own particles keep the sums in
//     registers; those of other tiles go to the tile's slab of partials in
//     global memory, then the tile raises its flag (release);
//  C. a tile waits (acquire, bounded) for the flags of the tiles whose slabs
//     hold partials of its particles -- the previous tile of its row and the
//     tiles of the row below under its cells, all with smaller tile numbers
//     (tiles are numbered in row order and taken in that order from a
//     ticket, so a tile only ever waits for tiles that already run) -- adds
//     them in a fixed order and finishes its particles as the plain pass does
//     (ghosts, corrected density, closing kick).
// The summation order differs from the plain pass's, so results agree with
// it to rounding, and two runs agree bit for bit.
//
// Capacities: a candidate row of up to 64 particles per half-stencil range,
// kN3PairCap pairs per tile, kN3ExtCap external targets per tile.  A tile
// beyond one of them (far denser than the density band allows at the usual
// spacing) drops the excess and sets ST_N3CAP (the step reports HR_ERANGE);
// a wait that gives up sets ST_N3WAIT (HR_ETIMEOUT).
#pragma once

namespace hr {

constexpr int kN3PairCap = 2048;
constexpr int kN3ExtCap = 512;
constexpr long long kN3Spin = 1LL << 22;

__device__ __forceinline__ int n3_ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void n3_st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Support mask of up to 64 candidates [base, base + cnt).
__device__ __forceinline__ unsigned long long mask64(const float2 *pos, int base, int cnt, float2 ri,
                                                     float s2)
{
    const unsigned lo = support_mask(pos, base, min(cnt, 32), ri, s2);
    const unsigned hi = cnt > 32 ? support_mask(pos, base + 32, cnt - 32, ri, s2) : 0u;
    return ((unsigned long long)hi << 32) | lo;
}

// pair_terms<0> for a fluid neighbour (m_j = 1, XSPH on), with the viscous
// dissipation of the pair (both particles' shares, Pi F v.r) added to diss;
// returns the neighbour's side: {f, F v.r, w_X} (its force is -f, its
// continuity term F v.r, its XSPH term w_X (v_j - v_i)).
__device__ __forceinline__ float4 pair_terms_n3(const Consts &K, const Self &I, float2 rj, float2 vj,
                                                float rhoj, float Pj, float cj, Acc &A, float &diss)
{
    const float2 d = p2_sub(I.r, rj);
    const float dx = d.x, dy = d.y;
    const float r2 = fmaf(dx, dx, dy * dy);
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    const float t = fmaxf(fmaf(-r, K.half_inv_h, 1.0f), 0.0f);
    const float t3 = t * t * t;
    const float F = K.Fc * t3;
    const float2 v = p2_sub(I.v, vj);
    const float vr = fmaf(v.x, dx, v.y * dy);
    const float Fvr = F * vr;
    A.dr += Fvr;
    const float e = r2 + K.eh2;
    const float inv = __fdividef(1.0f, e * (I.rho + rhoj));
    const float Pi_ij = (I.c + cj) * fminf(vr, 0.0f) * inv;
    const float PF = (I.P + Pj + Pi_ij) * F;
    const float lam = K.nu4 * F * r2 * inv;
    const float2 f = p2_fma(make_float2(-PF, -PF), d, p2_mul(make_float2(lam, lam), v));
    A.a = p2_add(A.a, f);
    diss = fmaf(Pi_ij * F, vr, diss);
    const float wx = K.m2Wc * t3 * t * fmaf(r, K.two_inv_h, 1.0f) * (inv * e);
    A.X = p2_fma(make_float2(wx, wx), v, A.X);
    return make_float4(f.x, f.y, Fvr, wx);
}

// The neighbour's side of one stored pair, added to the target's sums.
__device__ __forceinline__ void n3_take(const float4 e, float2 vj, float2 vi, float2 &a, float &dr,
                                        float2 &X)
{
    a.x -= e.x;
    a.y -= e.y;
    dr += e.z;
    X.x = fmaf(e.w, vj.x - vi.x, X.x);
    X.y = fmaf(e.w, vj.y - vi.y, X.y);
}

__global__ void __launch_bounds__(kN3Threads, 6) k_pass_n3(Consts K, Bufs B, int prime)
{
    __shared__ float4 pb[kN3PairCap];
    __shared__ unsigned long long sm0[kN3Threads], sm1[kN3Threads];
    __shared__ int sb1[kN3Threads], soff[kN3Threads];
    __shared__ float2 sv[kN3Threads];
    __shared__ int s_scan[kN3Threads / 32];
    __shared__ int s_tile, s_cfirst, s_clast, s_ok;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_tile = atomicAdd(&B.n3_ctl[0], 1);
        s_ok = 1;
    }
    __syncthreads();
    const int t = s_tile;
    const int n_tiles = B.n3_row_base[K.ncy];
    PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (t >= n_tiles) {
        // no tile for this ticket: the frozen particles (sorted after every
        // cell) keep their state, and the partials at this index are empty
        const int fz = B.cell_start[K.ncell];
        const int stride = (gridDim.x - n_tiles) * kN3Threads;
        for (int q = fz + (t - n_tiles) * kN3Threads + tid; q < K.nf; q += stride)
            pass_frozen<0>(B, q, B.s_vel[q], B.s_rd[q]);
        pass_block_partials<kN3Threads>(B.part, t, P, &B.S->vmax_bits);
        return;
    }
    const int epoch = B.n3_ctl[1];
    const int row = B.n3_tile_row[t];
    const int chunk = t - B.n3_row_base[row];
    const int rs = B.cell_start[row * K.ncx], re = B.cell_start[(row + 1) * K.ncx];
    const int p0 = rs + chunk * kN3Threads, p1 = min(p0 + kN3Threads, re);
    const int i = p0 + tid;
    const bool act = i < p1;
    const float dt = prime ? 0.0f : B.S->dt_f;
    int *status = &B.S->status;

    // A1: the particle's own data and its half-stencil masks
    float2 ri = make_float2(0.f, 0.f), vi = make_float2(0.f, 0.f), rd = make_float2(0.f, 0.f);
    float4 ai = make_float4(0.f, 0.f, 0.f, 0.f);
    int c = 0, b1 = 0;
    unsigned long long m0 = 0ull, m1 = 0ull;
    if (act) {
        ri = B.s_pos[i];
        vi = B.s_vel[i];
        ai = B.s_aux[i];
        rd = B.s_rd[i];
        c = cell_of(K, ri.x, ri.y);
        const int e0 = B.cell_start[c + 2];
        b1 = B.cell_start[c + K.ncx - 1];
        const int e1 = B.cell_start[c + K.ncx + 2];
        if (kChecked && !hr_ok(e0 >= i + 1 && e1 >= b1 && e1 <= K.nf && e0 <= K.nf, status)) {
            s_ok = 0;
        } else if (e0 - (i + 1) > 64 || e1 - b1 > 64) {
            atomicOr(status, ST_N3CAP);
        } else {
            m0 = mask64(B.s_pos, i + 1, e0 - (i + 1), ri, K.s2);
            m1 = mask64(B.s_pos, b1, e1 - b1, ri, K.s2);
        }
        if (tid == 0) s_cfirst = c;
        if (i == p1 - 1) s_clast = c;
    }
    const int cnt = __popcll(m0) + __popcll(m1);
    int total;
    const int off = block_exclusive_scan(cnt, s_scan, &total);
    sm0[tid] = m0;
    sm1[tid] = m1;
    sb1[tid] = b1;
    soff[tid] = off;
    sv[tid] = vi;
    if (tid == 0 && total > kN3PairCap) atomicOr(status, ST_N3CAP);

    // A2: the half-stencil pairs; own side in registers, the neighbour's in pb
    Acc A{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
    float dissf = 0.0f;
    const Self I{ri, vi, fmaf(K.rho0, ai.x, K.rho0), ai.z, ai.w};
    {
        int slot = off;
        unsigned long long a0 = m0, a1 = m1;
#pragma unroll 1
        while ((a0 | a1) != 0ull) {
            int j;
            if (a0) {
                j = i + __ffsll((long long)a0);
                a0 &= a0 - 1ull;
            } else {
                j = b1 + __ffsll((long long)a1) - 1;
                a1 &= a1 - 1ull;
            }
            const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
            const float2 vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
            const float4 aj = HR_DYNAMIC_LOAD(&B.s_aux[j]);
            const float4 e = pair_terms_n3(K, I, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z, aj.w, A,
                                           dissf);
            if (slot < kN3PairCap) pb[slot] = e;
            ++slot;
        }
    }
    __syncthreads();

    // B1: the tile's own particles take their side of the tile's earlier pairs
    // (same row, cells c - 1 and c, evaluated by particles before them)
    if (act) {
        const int lo = max(p0, B.cell_start[c - 1]);
#pragma unroll 1
        for (int q = lo; q < i; ++q) {
            const int u = q - p0;
            const int bit = i - q - 1;
            if (bit >= 64) continue;
            const unsigned long long mu = sm0[u];
            if (!((mu >> bit) & 1ull)) continue;
            const int slot = soff[u] + __popcll(mu & ((1ull << bit) - 1ull));
            if (slot < kN3PairCap) n3_take(pb[slot], vi, sv[u], A.a, A.dr, A.X);
        }
    }
    // B2: the targets outside the tile -- the rest of the row up to the last
    // cell + 1, then the three-cell span of the row above
    const int c_first = s_cfirst, c_last = s_clast;
    const int n_same = B.cell_start[c_last + 2] - p1;
    const int up_lo = B.cell_start[c_first + K.ncx - 1];
    const int n_up = B.cell_start[c_last + K.ncx + 2] - up_lo;
    const bool fits = n_same <= kN3Threads && n_same + n_up <= kN3ExtCap;
    if (tid == 0 && !fits) atomicOr(status, ST_N3CAP);
    if (fits) {
        float4 *ea = B.n3_ext_a + (size_t)t * kN3ExtCap;
        float *eb = B.n3_ext_b + (size_t)t * kN3ExtCap;
#pragma unroll 1
        for (int q = tid; q < n_same + n_up; q += kN3Threads) {
            const bool same = q < n_same;
            const int j = same ? p1 + q : up_lo + (q - n_same);
            const float2 rj = B.s_pos[j];
            const float2 vj = B.s_vel[j];
            const int cj = cell_of(K, rj.x, rj.y);
            float2 a = make_float2(0.f, 0.f), X = make_float2(0.f, 0.f);
            float dr = 0.0f;
            if (same) {
                const int lo = max(p0, B.cell_start[cj - 1]);
#pragma unroll 1
                for (int g = lo; g < p1; ++g) {
                    const int u = g - p0;
                    const int bit = j - g - 1;
                    if (bit >= 64) continue;
                    const unsigned long long mu = sm0[u];
                    if (!((mu >> bit) & 1ull)) continue;
                    const int slot = soff[u] + __popcll(mu & ((1ull << bit) - 1ull));
                    if (slot < kN3PairCap) n3_take(pb[slot], vj, sv[u], a, dr, X);
                }
            } else {
                const int lo = max(p0, B.cell_start[cj - K.ncx - 1]);
                const int hi = min(p1, B.cell_start[cj - K.ncx + 2]);
#pragma unroll 1
                for (int g = lo; g < hi; ++g) {
                    const int u = g - p0;
                    const int bit = j - sb1[u];
                    if (bit < 0 || bit >= 64) continue;
                    const unsigned long long mu = sm1[u];
                    if (!((mu >> bit) & 1ull)) continue;
                    const int slot =
                        soff[u] + __popcll(sm0[u]) + __popcll(mu & ((1ull << bit) - 1ull));
                    if (slot < kN3PairCap) n3_take(pb[slot], vj, sv[u], a, dr, X);
                }
            }
            ea[q] = make_float4(a.x, a.y, dr, X.x);
            eb[q] = X.y;
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        B.n3_info[t] = make_int4(p1, fits ? n_same : 0, up_lo, fits ? n_up : 0);
        __threadfence();
        n3_st_release(&B.n3_flag[t], epoch);
    }

    // C: the partials of earlier tiles, then the particle's finish
    if (tid == 0) {
        int lo = 0, hi = -1;   // tiles of the row below whose slabs hold our particles
        if (row > 0) {
            const int rb = B.cell_start[(row - 1) * K.ncx];
            const int a = B.cell_start[c_first - K.ncx - 1];
            const int b = B.cell_start[c_last - K.ncx + 2];
            if (b > a) {
                lo = B.n3_row_base[row - 1] + (a - rb) / kN3Threads;
                hi = B.n3_row_base[row - 1] + (b - 1 - rb) / kN3Threads;
            }
        }
        auto wait = [&](int s) {
            long long it = 0;
            while (n3_ld_acquire(&B.n3_flag[s]) != epoch) {
                if (++it > kN3Spin) {
                    atomicOr(status, ST_N3WAIT);
                    s_ok = 0;
                    return;
                }
                __nanosleep(64);
            }
        };
        if (chunk > 0) wait(t - 1);
        for (int s = lo; s <= hi && s_ok; ++s) wait(s);
        __threadfence();
    }
    __syncthreads();
    if (act && s_ok) {
        // the previous tile of the row: the start of this tile is its tail
        if (chunk > 0) {
            const int4 in = B.n3_info[t - 1];
            const int q = i - in.x;
            if (q >= 0 && q < in.y) {
                const size_t o = (size_t)(t - 1) * kN3ExtCap + q;
                const float4 e = B.n3_ext_a[o];
                A.a.x += e.x;
                A.a.y += e.y;
                A.dr += e.z;
                A.X.x += e.w;
                A.X.y += B.n3_ext_b[o];
            }
        }
        // the tiles of the row below, in ascending order
        if (row > 0) {
            const int rb = B.cell_start[(row - 1) * K.ncx];
            const int a = B.cell_start[c - K.ncx - 1];
            const int b = B.cell_start[c - K.ncx + 2];
            if (b > a) {
                const int s0 = B.n3_row_base[row - 1] + (a - rb) / kN3Threads;
                const int s1 = B.n3_row_base[row - 1] + (b - 1 - rb) / kN3Threads;
                for (int s = s0; s <= s1; ++s) {
                    const int4 in = B.n3_info[s];
                    const int q = i - in.z;
                    if (q < 0 || q >= in.w) continue;
                    const size_t o = (size_t)s * kN3ExtCap + in.y + q;
                    const float4 e = B.n3_ext_a[o];
                    A.a.x += e.x;
                    A.a.y += e.y;
                    A.dr += e.z;
                    A.X.x += e.w;
                    A.X.y += B.n3_ext_b[o];
                }
            }
        }
        pass_finish<0>(K, B, i, ri, vi, ai, rd, c, dt, prime, I, A, P);
        P.diss += K.m * K.m * dissf;
    }
    pass_block_partials<kN3Threads>(B.part, t, P, &B.S->vmax_bits);
}

}  // namespace hr
