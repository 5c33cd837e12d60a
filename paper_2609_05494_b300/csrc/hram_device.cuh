// hram_device.cuh -- device data layout and kernels of the planar WCSPH
// hydrodynamic-ram step on B300 (sm_103a).
//
// One step U^{n+1} = T(L(G(U^n))) (Section 4.6) is seven kernels (eight with
// the paper's closure, which adds k_density after the sort):
//   k_drift_key     opening kick, XSPH drift, wall enforcement, cell key,
//                   in-cell slot (atomic count) and the particle's fluid ID
//                   filed in its cell's bucket                 [T, first half]
//   k_kinematics     advances t, projectile kinematics (FP64), disk ghost ring
//                    (a branch of the step graph, beside the drift and sort)
//   k_scan_apply     cell starts (each block scans the tile sums before it;
//                    k_drift_key counts the tile sums beside the cells)
//   k_rank_scatter   stable rank by fluid ID among the cell's bucket, SoA
//                    reorder, Tait pressure of the predicted density
//   k_ghost          Adami ghost extrapolation G (disk ring and wall layers)
//   k_pass           fused interaction sums L + closing kick epilogue
//   k_finalize       probes, FP64 accumulators, CFL gate           [T, gate]
//
// By default a step graph leaves the step's close (b_finalize) pending and
// the next step's graph runs it in the first blocks of its drift launch
// (k_close_drift), the drift taking its dt from the last pass's max |v|;
// k_finalize then only settles a close the host needs before it reads the
// case.
//
// Densities are carried as the relative deviation d = rho/rho0 - 1 in FP32:
// the Tait pressure B((1+d)^7 - 1) = B d (7 + 21 d + ...) then has no
// cancellation and a pressure of 100 Pa is resolved (an FP32 rho near 1000
// kg/m^3 resolves only 134 Pa).  Positions and velocities are FP32; time,
// kinematics and the accumulated diagnostics are FP64, and the step's global
// sums are compensated FP32 (two-float) converted to FP64 once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Loads of the arrays a step rewrites (sorted positions, velocities, EOS
// records, the provisional permutation).  Kernels that see each array's
// values of one step only read them through the read-only data path; the
// persistent batched kernel, which runs many steps in one launch, defines
// this as a plain load before including the header.
#ifndef HR_DYNAMIC_LOAD
#define HR_DYNAMIC_LOAD(p) __ldg(p)
#endif

namespace hr {

constexpr int kMaxProbes = 16;
constexpr int kPassThreads = 128;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kFinalizeThreads = 256;
constexpr int kFinalizeBlocks = 64;
constexpr int kGhostWarps = 8;
constexpr int kGhostLanes = 8;                                  // lanes per ghost in b_ghost
constexpr int kGhostsPerBlock = kGhostWarps * 32 / kGhostLanes;  // ghosts per b_ghost block

// device status bits (warnings share the public HR_W* values)
constexpr int ST_PENETRATION = 1;
constexpr int ST_OUTSIDE = 2;
constexpr int ST_PROBEFULL = 4;
constexpr int ST_NAN = 256;
constexpr int ST_DT = 512;
constexpr int ST_N3CAP = 2048;    // a Newton-3 pass tile went past a capacity
constexpr int kBucket = 16;       // fluid IDs filed per cell by the drift (more go to the overflow list)
constexpr int ST_N3WAIT = 4096;   // a Newton-3 pass tile gave up waiting for another
constexpr int kN3Threads = 128;   // particles per Newton-3 pass tile

enum GhostKind { KIND_SIDE = 1, KIND_END = 2, KIND_DISK = 3 };

// Constants of a case, passed by value (kernel parameter bank).
struct Consts {
    // grid and box
    float x0, y0, inv_dc;
    int ncx, ncy, ncell;
    float xlo, xhi, ylo, yhi;
    float W2, Lx;
    int side_walls, end_walls;
    // kernel
    float h, s2, half_inv_h, two_inv_h, Wc, Fc;
    // fluid
    float m, rho0, inv_rho0, B, c0, p_cav, alpha_h, alpha_f, eh2, nu4, eps_xsph, gx, gy;
    float d_lo, d_hi, gamma, half_gm1, inv_rho0c02;
    int gamma7;
    // ghosts
    int nf, nw, ng;
    float m_wall, m_disk, wall_over_m, disk_over_m, m_over_rho0, m2Wc, R, disk_reach2, R2;
    float ng_over_2pi;  // disk ghosts per radian of the ring
    // CFL and kinematics (FP64)
    double cfl_h, c0d, v0, tau, t_ramp, x_c0, y_c0, a_const, drag_k, dt_fixed, disk_mass;
    float cfl_h_f;
    int dt_mode, motion;
    // probes
    int n_probes;
    float probe_x[kMaxProbes], probe_y[kMaxProbes];
    long long probe_cap;
    int n_pass_blocks, n_ghost_blocks;
    // closure 1 (the paper's): cubic B-spline, summation density,
    // Mie-Grueneisen EOS with the internal-energy equation
    int closure;
    float cub_sd, cub_Fc, inv_h;   // sigma = 10/(7 pi h^2), sigma/h^2, 1/h
    float self_w;                  // (m / rho0) W(0): a particle's own share of its density
    float c_av;                    // -alpha h C: the artificial-viscosity factor of every particle
    float mg_K, mg_k1, mg_s1m1, mg_g0, mg_a, mg_mu_max;  // rho0 C^2, 1 - gamma0/2, S1 - 1, gamma0, a, cap
    // (appended last, so the fields above keep their offsets in the parameter bank)
    int sr;                 // stencil reach in cells: 1 (cells of side >= 2h, 3 x 3) or 2 (side >= h, 5 x 5)
    int n3, n3_tiles_max;   // the Newton-3 pass variant, and its tile capacity
    int split;              // the interaction pass runs split (interior / boundary particles)
    // motion 0 with tau > 0 after the ramp: x(t) = kin_x1 - kin_q e, v = v0 e,
    // a = -v0 e / tau, e = exp(-t kin_inv_tau), the t-independent parts of the
    // closed form formed once on the host (kin_fast)
    int kin_fast;
    double kin_inv_tau, kin_x1, kin_q;
    double m2d;             // (double) m * (double) m, the step close's scale of the force sums
};

// Device-resident scalars of the case.
struct Scalars {
    double t, dt, dt_prev;
    long long step;
    double xc, yc, vproj, aproj;
    double Fdx, Fdy, Fwall, diss_rate;
    double Wb, impulse, diss;
    double probe_imp[kMaxProbes];
    long long hist_n;
    int status;
    int done;          // 1 once t >= t_end (batched runs)
    double t_end;      // stop time of a batched run (<= 0: none)
    // single-precision copies for the per-particle kernels (the FP64 pipe of
    // the B300 is far too slow to convert doubles in every thread)
    float dt_f, ratio_f, xc_f, yc_f, vproj_f, aproj_f;
    // The deferred step close (a step graph whose closing reductions run in
    // the next step, beside its drift): vmax_bits, max |v| over the fluid
    // and the ghosts of the last pass (float bits, atomic max of the block
    // maxima; the graph's kinematics clears it before its pass); close_pending,
    // that step's close has not run yet; dt_stale, dt and its copies still
    // hold that step's step size (the next one follows from vmax_bits).
    unsigned vmax_bits;
    int close_pending, dt_stale, pad_;
};

// Per-block partials of the interaction pass, structure of arrays so the
// finalize kernel streams them with wide independent loads.
struct PassPartials {
    float4 *f;       // {F_disk,x, F_disk,y, F_wall, dissipation rate} / m^2 except the last
    float *vmax;
    int *npen;
};

// Device buffers of a case.  s_* are in the cell order of the current step,
// st_* hold the end-of-step state in that same order, u_* are the drifted
// particles before the sort (previous order).
struct Bufs {
    // sorted (k_rank_scatter)
    float2 *s_pos;   // r^{n+1}
    float2 *s_vel;   // v^{n+1/2}
    float4 *s_aux;   // {d~, p~, p~/rho~^2, -alpha h c~}  predicted density and its EOS
    float2 *s_rd;    // {d^n, D^n}                 for the corrected density
    int *s_id;
    // end-of-step state (k_pass epilogue)
    float2 *st_vel;  // v^{n+1}
    float *st_rho;   // d^{n+1}
    float2 *st_a;    // a^{n+1}
    float2 *st_D;    // {D^{n+1}, D^n}   density rate in units of d per second
    float2 *st_X;    // XSPH sum X^{n+1}
    // drifted, unsorted
    float2 *u_pos, *u_vel;
    int *u_id, *u_key;
    // cell list
    int *cell_count; // ncell + 1 (last = frozen particles)
    int *cell_start; // ncell + 2
    int *tile_sum;
    int *bucket;     // (ncell + 1) x kBucket: the fluid IDs of each cell, in slot order
    int4 *ovf;       // {cell, fluid ID, slot} of the particles past their cell's bucket (nf)
    int *ovf_count;  // entries of ovf this step (reset by k_rank_scatter)
    int *perm_tmp;   // the IDs of slots >= kBucket at cell start + slot (overflowing cells only)
    int *perm_dst;   // previous slot -> slot of this step (tangent mode only, else null)
    float4 *s_ex;    // closure 1: {a^n, e^n, De^n} in this step's cell order (else null)
    // wall ghosts (static, cell order) and disk ghosts
    float2 *gw_pos;
    float2 *gw_nrm;
    int *gw_kind, *gw_id;
    int *wall_start;   // ncell + 1
    double2 *disk_off; // R (cos, sin) theta_k
    float2 *gd_pos;
    // ghost state: walls [0, nw), disk [nw, nw + ng)
    float2 *g_vel;
    float4 *g_aux;     // {d_g, p_g, p_g / rho_g^2, -alpha h c_g}
    float *ghost_vmax; // per ghost block
    PassPartials part;
    float *fin_part;   // kFinalizeBlocks x 4 two-float sums
    float *fin_vmax;
    int *fin_npen;
    int *fin_ticket;
    // probes
    float *probe_now;  // this step's values, one per probe
    float *probe_hist;
    double *probe_t;
    // scalars
    Scalars *S;
    // the Newton-3 pass variant (null otherwise): tile table (per-row first
    // tile, row of each tile), per-tile header {end, same-row targets, first
    // target of the row above, its count}, ready flags, partial slabs, and
    // {ticket, flag value of this step}
    int *n3_row_base, *n3_tile_row;
    int4 *n3_info;
    int *n3_flag;
    float4 *n3_ext_a;
    float *n3_ext_b;
    int *n3_ctl;
    // per cell, nonzero where the cell's stencil holds wall ghosts (static)
    unsigned char *wall_near;
    // the split pass (K.split; null otherwise): the reorder marks in
    // split_mask the pass blocks holding boundary particles (those with
    // ghost candidates); the ghost launch's extra blocks list those blocks and their boundary
    // particles (counts in split_n[0], split_n[1]; any order); the boundary pass leaves each boundary
    // particle's block-partial terms at its sorted index ({F_disk,x,
    // F_disk,y, F_wall, dissipation rate}, {max |v| bits, penetration});
    // the boundary share of each listed block's partials goes to part_b
    int *split_n;
    int *split_pi;
    int *split_bi;
    unsigned *split_mask;
    float4 *split_pf;
    int2 *split_pv;
    PassPartials part_b;
};

// ----------------------------------------------- bounds-checked build

// Built with -DHRAM_CHECKED, every index into the cell lists, the sorted
// arrays and the ghost arrays is checked before it is used: a failed check
// sets ST_BOUNDS in the case's status word and the access is skipped (the
// candidate row or the particle is left out).  Nothing traps.  In the normal
// build the checks compile away.
#ifdef HRAM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
constexpr int ST_BOUNDS = 1024;

__device__ __forceinline__ bool hr_ok(bool cond, int *status)
{
    if constexpr (kChecked) {
        if (!cond) {
            atomicOr(status, ST_BOUNDS);
            return false;
        }
    }
    return true;
}

// A stencil row's candidate range [a, b) of a start array with entries
// [0, ncell] at least (cell_start, wall_start), items [0, limit).
__device__ __forceinline__ bool row_ok(const Consts &K, int row, int a, int b, int limit, int *status)
{
    return hr_ok(row - 1 >= 0 && row + 2 <= K.ncell && 0 <= a && a <= b && b <= limit, status);
}

// ---------------------------------------------------------------- helpers

// Neighbour predicate of the method: FP32, round-to-nearest, no contraction.
__device__ __forceinline__ bool in_support(float xi, float yi, float xj, float yj, float s2)
{
    const float dx = __fsub_rn(xi, xj);
    const float dy = __fsub_rn(yi, yj);
    const float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return r2 < s2;
}

// Packed FP32 pairs: the sm_100-family .f32x2 instructions do two IEEE
// round-to-nearest operations in one issue slot, each lane bit-identical to
// the scalar operation (add/sub/mul rounded once, fma rounded once).
__device__ __forceinline__ float2 p2_add(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 p2_sub(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 p2_mul(float2 a, float2 b)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 p2_fma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// The neighbour predicate on packed pairs: the same three roundings as
// in_support (dx, dy; dx^2, dy^2; their sum).
__device__ __forceinline__ bool in_support2(float2 ri, float2 rj, float s2)
{
    const float2 d = p2_sub(ri, rj);
    const float2 q = p2_mul(d, d);
    return __fadd_rn(q.x, q.y) < s2;
}

// The cell of a point, clamped to keep its stencil inside the grid.  R: the
// stencil reach when the caller knows it at compile time, 0 to read K.sr.
template <int R = 0>
__device__ __forceinline__ int cell_of(const Consts &K, float x, float y)
{
    const int r = R ? R : K.sr;
    int cx = __float2int_rd(__fmul_rn(__fsub_rn(x, K.x0), K.inv_dc));
    int cy = __float2int_rd(__fmul_rn(__fsub_rn(y, K.y0), K.inv_dc));
    cx = min(max(cx, r), K.ncx - 1 - r);
    cy = min(max(cy, r), K.ncy - 1 - r);
    return cy * K.ncx + cx;
}

__device__ __forceinline__ bool outside_box(const Consts &K, float x, float y)
{
    return !(x >= K.xlo && x <= K.xhi && y >= K.ylo && y <= K.yhi);
}

// Tait pressure from the density deviation d, with the cavitation cutoff.
// gamma = 7: (1+d)^7 - 1 = d (7 + 21 d + 35 d^2 + 35 d^3 + 21 d^4 + 7 d^5 + d^6).
__device__ __forceinline__ float tait_p(const Consts &K, float d)
{
    float p;
    if (K.gamma7) {
        float poly = fmaf(d, 1.0f, 7.0f);
        poly = fmaf(d, poly, 21.0f);
        poly = fmaf(d, poly, 35.0f);
        poly = fmaf(d, poly, 35.0f);
        poly = fmaf(d, poly, 21.0f);
        poly = fmaf(d, poly, 7.0f);
        p = K.B * d * poly;
    } else {
        p = K.B * expm1f(K.gamma * log1pf(d));
    }
    return fmaxf(p, K.p_cav);
}

// c = c0 (rho/rho0)^((gamma-1)/2)
__device__ __forceinline__ float sound_speed(const Consts &K, float d)
{
    if (K.gamma7) {
        const float x = 1.0f + d;
        return K.c0 * x * x * x;
    }
    return K.c0 * __powf(1.0f + d, K.half_gm1);
}

// {d, p, p / rho^2, -alpha h c}: what a neighbour contributes to the pair
// terms (the last entry is the artificial-viscosity signal factor).
__device__ __forceinline__ float4 eos_record(const Consts &K, float d)
{
    const float p = tait_p(K, d);
    const float rho = K.rho0 * (1.0f + d);
    return make_float4(d, p, p / (rho * rho), -K.alpha_h * sound_speed(K, d));
}

__device__ __forceinline__ float band(const Consts &K, float d)
{
    return fminf(fmaxf(d, K.d_lo), K.d_hi);
}

// Cubic B-spline of the paper (eq. cubic-kernel), q = r/h:
//   W = sigma (1 - 3/2 q^2 + 3/4 q^3) for q < 1, sigma (2 - q)^3 / 4 for q >= 1,
// and F = (dW/dr)/r = sigma/h^2 (-3 + 9/4 q), resp. -3/4 sigma/h^2 (2 - q)^2 / q.
__device__ __forceinline__ float cubic_w(const Consts &K, float r)
{
    const float q = r * K.inv_h;
    const float u = fmaxf(2.0f - q, 0.0f);
    const float inner = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    return K.cub_sd * (q < 1.0f ? inner : 0.25f * u * u * u);
}

__device__ __forceinline__ float cubic_F(const Consts &K, float r)
{
    const float q = r * K.inv_h;
    const float u = fmaxf(2.0f - q, 0.0f);
    return K.cub_Fc * (q < 1.0f ? fmaf(2.25f, q, -3.0f) : -0.75f * u * u / q);
}

// The closure's smoothing kernel W(r): Wendland C2 (closure 0) or the cubic
// B-spline (closure 1).
template <int CL>
__device__ __forceinline__ float kernel_w(const Consts &K, float r)
{
    if constexpr (CL == 1) {
        return cubic_w(K, r);
    } else {
        const float t = fmaxf(fmaf(-r, K.half_inv_h, 1.0f), 0.0f);
        const float t2 = t * t;
        return K.Wc * t2 * t2 * fmaf(r, K.two_inv_h, 1.0f);
    }
}

// Mie-Grueneisen pressure (eq. eos) of the deviation d = mu and the specific
// internal energy e, with the compression cap mu <= mu_max applied to the
// state and the cavitation cutoff.
__device__ __forceinline__ float mg_p(const Consts &K, float d, float e)
{
    const float mu = fminf(d, K.mg_mu_max);
    const float rho = fmaf(K.rho0, mu, K.rho0);
    float p;
    if (mu >= 0.0f) {
        const float den = fmaf(-K.mg_s1m1, mu, 1.0f);
        p = K.mg_K * mu * fmaf(K.mg_k1, mu, 1.0f) / (den * den) +
            fmaf(K.mg_a, mu, K.mg_g0) * rho * e;
    } else {
        p = fmaf(K.mg_K, mu, K.mg_g0 * rho * e);
    }
    return fmaxf(p, K.p_cav);
}

// {d, p, p / rho^2, e} of closure 1 (its artificial-viscosity factor is the
// constant c_av, so the fourth slot carries the energy the pressure used).
__device__ __forceinline__ float4 mg_record(const Consts &K, float d, float e)
{
    const float p = mg_p(K, d, e);
    const float rho = K.rho0 * (1.0f + d);
    return make_float4(d, p, p / (rho * rho), e);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Compensated single-precision sums ("two-float": hi + lo carries about 48
// bits; Knuth's TwoSum for the error of each addition).  Used for the
// per-step reductions so they keep near-FP64 accuracy on the FP32 pipes; the
// B300's FP64 pipe is slow enough that a warp-wide FP64 reduction costs
// microseconds.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = a.lo + b.lo + err;
    const float hi = s + lo;
    return F2{hi, lo - (hi - s)};
}

__device__ __forceinline__ F2 f2_warp_sum(F2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F2 u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = f2_add(v, u);
    }
    return v;
}

// a6, the CFL gate (eq. cfl): dt = C h / (c0 + max |v|) over fluid and
// ghost velocities, in FP32 (a float ulp of dt is far below every
// tolerance).  dt_mode 1 takes the fixed host value instead.
__device__ __forceinline__ float cfl_dt_f(const Consts &K, float vmax)
{
    return __fdiv_rn(K.cfl_h_f, K.c0 + vmax);
}

// The deferred step close: the next step's size from the last pass's max |v|
// (Scalars::vmax_bits), into the fields the close at the end of a step
// writes (dt_prev, dt, dt_f, ratio_f), with the same arithmetic.  One thread.
// vbits, dtf_old, dt_old: the scalars' vmax_bits, dt_f and dt as read by the
// caller; returns the new dt.
__device__ __forceinline__ double advance_dt(const Consts &K, Scalars *S, unsigned vbits, float dtf_old,
                                             double dt_old)
{
    double dtn;
    float dtf;
    if (K.dt_mode == 1) {
        dtn = K.dt_fixed;
        dtf = (float)dtn;
    } else {
        dtf = cfl_dt_f(K, __uint_as_float(vbits));
        dtn = (double)dtf;
    }
    if (!(dtn > 1e-14)) atomicOr(&S->status, ST_DT);
    S->ratio_f = __fdiv_rn(dtf, dtf_old);
    S->dt_prev = dt_old;
    S->dt = dtn;
    S->dt_f = dtf;
    S->dt_stale = 0;
    return dtn;
}

// Projectile kinematics in closed form (FP64).  Section 2.6.3 ramp,
// exponential decay with time constant tau (motion 0), the paper's quadratic
// drag law after the ramp (motion 1, Section 2.7), constant acceleration
// (motion 2).  Motion 3 uses the ramp here; after it the disk is advanced
// by the fluid force in b_kinematics (two-way coupling).
__device__ inline void kinematics(const Consts &K, double t, double *xo, double *vo, double *ao)
{
    if (K.kin_fast && !(K.t_ramp > 0.0 && t < K.t_ramp)) {
        // motion 0 after the ramp: one exponential per step (an FP64 operation
        // holds a warp's issue for many cycles on this GPU, and this chain is
        // the longest block of the scan launch)
        const double e = exp(-t * K.kin_inv_tau);
        *vo = K.v0 * e;
        *ao = K.v0 * (-e * K.kin_inv_tau);
        *xo = K.kin_x1 - K.kin_q * e;
        return;
    }
    const double v0 = K.v0, tr = K.t_ramp, tau = K.motion == 3 ? 0.0 : K.tau;
    double x = K.x_c0, v, a;
    if (K.motion == 2) {
        v = K.a_const * t;
        a = K.a_const;
        x += 0.5 * K.a_const * t * t;
    } else if (K.motion == 1) {
        if (tr > 0.0 && t < tr) {
            v = v0 * t / tr;
            a = v0 / tr;
            x += 0.5 * v0 * t * t / tr;
        } else {
            const double t1 = tr > 0.0 ? tr : 0.0;
            const double u = 1.0 + K.drag_k * v0 * (t - t1);
            v = v0 / u;
            a = -K.drag_k * v * v;
            x += 0.5 * v0 * t1 + log(u) / K.drag_k;
        }
    } else {
        double f, df, e, de;
        if (tr > 0.0 && t < tr) { f = t / tr; df = 1.0 / tr; }
        else { f = 1.0; df = 0.0; }
        if (tau > 0.0) { e = exp(-t / tau); de = -e / tau; }
        else { e = 1.0; de = 0.0; }
        v = v0 * f * e;
        a = v0 * (df * e + f * de);
        if (tau > 0.0) {
            if (tr > 0.0) {
                const double ta = t < tr ? t : tr;
                x += (v0 / tr) * (tau * tau - tau * (ta + tau) * exp(-ta / tau));
                if (t > tr) x += v0 * tau * (exp(-tr / tau) - exp(-t / tau));
            } else {
                x += v0 * tau * (1.0 - exp(-t / tau));
            }
        } else {
            if (tr > 0.0) {
                const double ta = t < tr ? t : tr;
                x += 0.5 * v0 * ta * ta / tr;
                if (t > tr) x += v0 * (t - tr);
            } else {
                x += v0 * t;
            }
        }
    }
    *xo = x;
    *vo = v;
    *ao = a;
}

// Candidate enumeration shared by every gather (ghost pass, interaction pass,
// probes, debug neighbour lists): the (2R+1) x (2R+1) cell stencil of cell c
// (R = K.sr) is 2R+1 contiguous row ranges [start(row, cx-R),
// start(row, cx+R+1)) of the sorted arrays.  f(j) is called for every
// candidate j.
// (lane, lanes: the candidates lane, lane + lanes, ... of each row, for a
// particle whose work is split over several lanes.  RC: the reach when known
// at compile time, else 0.)
template <int RC = 0, class F>
__device__ __forceinline__ void for_fluid_candidates(const Consts &K, const int *start, int c,
                                                     int limit, int *status, F &&f, int lane = 0,
                                                     int lanes = 1)
{
    const int R = RC ? RC : K.sr;
#pragma unroll 1
    for (int dy = -R; dy <= R; ++dy) {
        const int row = c + dy * K.ncx;
        if (kChecked && !hr_ok(row - R >= 0 && row + R + 1 <= K.ncell, status)) continue;
        const int a = start[row - R], b = start[row + R + 1];
        if (kChecked && !row_ok(K, row, a, b, limit, status)) continue;
        for (int j = a + lane; j < b; j += lanes) f(j);
    }
}

// Disk ghosts are only candidates of fluid within R + 2h (with a margin) of
// the disk centre; the ring is then scanned in full.
__device__ __forceinline__ bool near_disk(const Consts &K, float x, float y, float xc, float yc)
{
    const float dx = x - xc, dy = y - yc;
    return dx * dx + dy * dy < K.disk_reach2;
}

// A boundary particle: one whose interaction pass looks at ghosts, because
// its cell c's stencil holds wall ghosts or it lies near the disk (the
// disk at this step's t^{n+1}).  Every pass form and the reorder decide it
// with this one test on the same FP32 position.
__device__ __forceinline__ bool has_ghost_candidates(const Consts &K, const Bufs &B, float2 r, int c)
{
    return (K.nw > 0 && B.wall_near[c] != 0) ||
           (K.ng > 0 && near_disk(K, r.x, r.y, B.S->xc_f, B.S->yc_f));
}

// The disk ghosts that can lie within the support of a point near the disk.
// Ghost k sits at angle 2 pi k / ng on the circle of radius R about the
// centre, so at distance rho from the centre only ghosts within the angle
// acos((rho^2 + R^2 - (2h)^2) / (2 rho R)) of the point's own angle can (the
// law of cosines); three ghosts on each side are added against rounding.
// The arc is returned as at most two ascending index ranges [a0, a1) and
// [b0, b1), so a loop over them visits its ghosts in the order of a loop over
// the whole ring, and the support test still decides each one.
struct DiskArc {
    int a0, a1, b0, b1;
};

__device__ __forceinline__ DiskArc disk_arc(const Consts &K, float x, float y, float xc, float yc)
{
    const DiskArc all{0, K.ng, 0, 0};
    const float dx = x - xc, dy = y - yc;
    const float rho = sqrtf(dx * dx + dy * dy);
    if (!(rho > 1e-3f * K.R)) return all;
    const float c = (rho * rho + K.R2 - K.s2) / (2.0f * rho * K.R);
    if (!(c > -1.0f)) return all;
    const float half = acosf(fminf(c, 1.0f)) * K.ng_over_2pi + 3.0f;
    if (!(2.0f * half + 3.0f < (float)K.ng)) return all;   // the two ranges never overlap
    float phi = atan2f(dy, dx);
    if (phi < 0.0f) phi += 6.2831853f;
    const float kc = phi * K.ng_over_2pi;
    const int k0 = (int)floorf(kc - half), k1 = (int)ceilf(kc + half);   // inclusive
    if (k0 < 0) return DiskArc{0, k1 + 1, k0 + K.ng, K.ng};
    if (k1 >= K.ng) return DiskArc{0, k1 + 1 - K.ng, k0, K.ng};
    return DiskArc{k0, k1 + 1, 0, 0};
}

// f(k) for the ghosts of the arc, in ascending k.
template <class F>
__device__ __forceinline__ void for_disk_arc(const Consts &K, const DiskArc &A, int *status, F &&f,
                                             int lane = 0, int lanes = 1)
{
    if (kChecked && !hr_ok(0 <= A.a0 && A.a0 <= A.a1 && A.a1 <= K.ng && 0 <= A.b0 &&
                           A.b0 <= A.b1 && A.b1 <= K.ng, status))
        return;
#pragma unroll 1
    for (int k = A.a0 + lane; k < A.a1; k += lanes) f(k);
#pragma unroll 1
    for (int k = A.b0 + lane; k < A.b1; k += lanes) f(k);
}

// ----------------------------------------------------- a2: drift and key

__device__ __forceinline__ int b_drift_one(const Consts &K, const Bufs &B, const int i, float dt);

// Opening kick, XSPH drift, wall enforcement and cell key (the predicted
// density is formed in k_rank_scatter from the same state).  prime = 1
// evaluates the current state without advancing (dt = 0).  The cell
// histogram is counted with one atomic per run of equal keys in consecutive
// lanes: the previous step's cell order keeps most of a warp's particles in
// a few runs.  (Counting the scan's tile sums the same way was slower: a few
// dozen tile counters take every warp's atomic and serialise them.)
// defer: a step graph with the deferred close, where the step size may
// still be the last step's (Scalars::dt_stale): each thread then forms this
// step's from the last pass's max |v|, as the close would have.
__device__ __forceinline__ void b_drift_key(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime,
                                            int defer = 0)
{
    float dt = 0.0f;
    if (!prime) {
        dt = (defer && K.dt_mode == 0 && B.S->dt_stale) ? cfl_dt_f(K, __uint_as_float(B.S->vmax_bits))
                                                        : B.S->dt_f;
    }
    const int i = bx * blockDim.x + threadIdx.x;
    const int key = i < K.nf ? b_drift_one(K, B, i, dt) : -1;
    const int lane = threadIdx.x & 31;
    const unsigned upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;   // lanes 0..lane
    // runs of equal values in consecutive lanes: head lane and length
    auto run = [&](int v, int &head, int &len) {
        const int prev = __shfl_up_sync(0xffffffffu, v, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != v);
        head = 31 - __clz(heads & upto);
        const unsigned after = heads & ~upto;
        len = (after ? __ffs(after) - 1 : 32) - head;
    };
    int head, len;
    run(key, head, len);
    int slot0 = 0;
    if (key >= 0 && lane == head) slot0 = atomicAdd(&B.cell_count[key], len);
    slot0 = __shfl_sync(0xffffffffu, slot0, head);
    if (key >= 0) {
        // the particle's fluid ID in its cell's bucket (past it: the overflow list)
        const int slot = slot0 + (lane - head);
        const int id = B.u_id[i];
        if (slot < kBucket) {
            B.bucket[key * kBucket + slot] = id;
        } else {   // at most nf entries: the list cannot fill
            const int o = atomicAdd(B.ovf_count, 1);
            B.ovf[o] = make_int4(key, id, slot, 0);
        }
    }
    // The scan's tile sums, counted here too.  A block's particles, in the
    // previous step's cell order, almost always fall in one tile: then one
    // atomic adds the block's count.  Otherwise each warp adds its own (one
    // atomic per warp whose keys share a tile, else one per particle).
    __shared__ int t_lo[32], t_hi[32], t_n[32];
    __shared__ int one_tile;
    const int w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    const int tile = key >= 0 ? key / kScanTile : -1;
    const int wlo = __reduce_min_sync(0xffffffffu, key >= 0 ? tile : 0x7fffffff);
    const int whi = __reduce_max_sync(0xffffffffu, tile);
    const int wn = __popc(__ballot_sync(0xffffffffu, key >= 0));
    if (lane == 0) {
        t_lo[w] = wlo;
        t_hi[w] = whi;
        t_n[w] = wn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int lo = 0x7fffffff, hi = -1, n = 0;
        for (int k = 0; k < nw; ++k) {
            lo = min(lo, t_lo[k]);
            hi = max(hi, t_hi[k]);
            n += t_n[k];
        }
        one_tile = lo == hi;
        if (lo == hi && n > 0) atomicAdd(&B.tile_sum[lo], n);
    }
    __syncthreads();
    if (!one_tile) {
        if (wlo == whi) {
            if (lane == 0 && wn > 0) atomicAdd(&B.tile_sum[wlo], wn);
        } else if (key >= 0) {
            atomicAdd(&B.tile_sum[tile], 1);
        }
    }
}

// The per-particle part of b_drift_key (dt: this step's size, 0 when
// priming); returns the cell key.
__device__ __forceinline__ int b_drift_one(const Consts &K, const Bufs &B, const int i, float dt)
{
    float2 r = B.s_pos[i];
    const float2 v = B.st_vel[i];
    const float2 a = B.st_a[i];
    const float2 X = B.st_X[i];
    float2 vh;
    int key;
    if (outside_box(K, r.x, r.y)) {
        vh = v;
        key = K.ncell;
    } else {
        vh.x = fmaf(0.5f * dt, a.x, v.x);
        vh.y = fmaf(0.5f * dt, a.y, v.y);
        r.x = fmaf(dt, fmaf(K.eps_xsph, X.x, vh.x), r.x);
        r.y = fmaf(dt, fmaf(K.eps_xsph, X.y, vh.y), r.y);
        if (K.side_walls) {
            if (r.y > K.W2) { r.y = K.W2 - 1e-6f; vh.y = -vh.y; }
            else if (r.y < -K.W2) { r.y = -K.W2 + 1e-6f; vh.y = -vh.y; }
            if (K.end_walls) {
                if (r.x > K.Lx) { r.x = K.Lx - 1e-6f; vh.x = -vh.x; }
                else if (r.x < 0.0f) { r.x = 1e-6f; vh.x = -vh.x; }
            }
        }
        if (!isfinite(r.x) || !isfinite(r.y) || !isfinite(vh.x) || !isfinite(vh.y))
            atomicOr(&B.S->status, ST_NAN);
        if (outside_box(K, r.x, r.y)) {
            key = K.ncell;
            atomicOr(&B.S->status, ST_OUTSIDE);
        } else {
            key = cell_of(K, r.x, r.y);
        }
    }
    B.u_pos[i] = r;
    B.u_vel[i] = vh;
    B.u_id[i] = B.s_id[i];
    B.u_key[i] = key;
    return key;
}

// ---------------------------------------------------- a3: counting sort

__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) smem_warp[lane] = s;
    }
    __syncthreads();
    const int before = w > 0 ? smem_warp[w - 1] : 0;
    *total = smem_warp[(blockDim.x >> 5) - 1];
    return before + x - v;
}

// a1: advances t by dt (unless priming), evaluates the projectile
// kinematics at t^{n+1} in FP64 and places the disk ghost ring there.  One
// block; in the step graph it runs on a branch beside the drift and the sort.
// defer: a step graph with the deferred close.  The step size is brought
// up to date first if the last step's close has not done it (dt_stale), and
// the fluid and ghost maximum of |v| is cleared for this step's passes; the
// step then leaves its close pending (run beside the next step's drift, or
// by the host before it reads the case).
__device__ __forceinline__ void b_kinematics(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime,
                                             int defer = 0)
{
    __shared__ double kin[2];
    // the ring offsets of the first pass below, loaded before the barrier
    const double2 off0 = (int)threadIdx.x < K.ng ? B.disk_off[threadIdx.x] : make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        Scalars *S = B.S;
        // every scalar read here, loaded before any is written
        const int stale = defer ? S->dt_stale : 0;
        const unsigned vbits = S->vmax_bits;
        const float dtf_old = S->dt_f;
        const double dt_old = S->dt, t_old = S->t;
        const double Fdx = S->Fdx, vproj = S->vproj, xc = S->xc;
        double dt_now = dt_old;
        if (defer) {
            if (stale) dt_now = advance_dt(K, S, vbits, dtf_old, dt_old);
            S->vmax_bits = 0u;
            S->close_pending = 1;
            S->dt_stale = 1;
        }
        const double dt = prime ? 0.0 : dt_now;
        const double t = t_old + dt;
        S->t = t;
        double x, v, a;
        if (K.motion == 3 && !prime && !(K.t_ramp > 0.0 && t <= K.t_ramp)) {
            // two-way coupling (the extension named in the paper's
            // Conclusions): M' dv/dt = -F_x, F the disk ghosts' force on the
            // fluid from the last interaction pass; symplectic Euler in FP64
            a = -Fdx / K.disk_mass;
            v = vproj + dt * a;
            x = xc + dt * v;
        } else {
            kinematics(K, t, &x, &v, &a);
        }
        S->xc = x;
        S->yc = K.y_c0;
        S->vproj = v;
        S->aproj = a;
        S->xc_f = (float)x;
        S->yc_f = (float)K.y_c0;
        S->vproj_f = (float)v;
        S->aproj_f = (float)a;
        kin[0] = x;
        kin[1] = K.y_c0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K.ng; k += blockDim.x) {
        const double2 o = k == (int)threadIdx.x ? off0 : B.disk_off[k];
        B.gd_pos[k] = make_float2((float)(kin[0] + o.x), (float)(kin[1] + o.y));
    }
}

// The particles past their cell's bucket (the drift's overflow list, empty
// unless a cell holds more than kBucket particles), for the cells [c0, c1)
// whose starts this block has just written: each ID goes to perm_tmp at its
// cell's start + its slot, where the reorder reads it.
__device__ __forceinline__ void scan_overflow(const Consts &K, const Bufs &B, int c0, int c1, int no)
{
    __syncthreads();   // this block's cell starts are written
    for (int k = threadIdx.x; k < no; k += blockDim.x) {
        const int4 e = B.ovf[k];
        if (e.x < c0 || e.x >= c1) continue;
        const int dst = B.cell_start[e.x] + e.z;
        if (kChecked && !hr_ok(dst >= 0 && dst < K.nf, &B.S->status)) continue;
        B.perm_tmp[dst] = e.y;
    }
}

// Cell starts: each block adds up the sums of the tiles before it (counted
// by k_drift_key), then an exclusive scan of its own tile, and places its
// cells' overflowing IDs; the counts are reset for the next step (the tile
// sums in k_rank_scatter, once every block here has read them).  The tile's
// counts, the tile sums and the overflow count are all loaded before the
// first barrier, in one round trip.
__device__ __forceinline__ void b_scan_apply(const Consts &K, const Bufs &B, const int bx, const int nbx)
{
    static_assert(kScanItems == 4 && kScanThreads == 1024, "one int4 of counts per thread, 32 warps");
    __shared__ int wsum[32];
    __shared__ int offset;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = K.ncell + 1;
    const int base = bx * kScanTile + threadIdx.x * kScanItems;
    const bool whole = base + kScanItems <= n;   // (the arrays are 16-byte aligned)
    int v[kScanItems];
    if (whole) {
        const int4 q = *reinterpret_cast<const int4 *>(B.cell_count + base);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = (base + k < n) ? B.cell_count[base + k] : 0;
    }
    int o = 0;
    for (int t = threadIdx.x; t < (int)bx; t += blockDim.x) o += B.tile_sum[t];
    const int no = *B.ovf_count;
    // the warp's inclusive scan of the thread sums, and its part of the tile sums
    const int s = v[0] + v[1] + v[2] + v[3];
    int x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    o = warp_sum(o);
    __shared__ int wtile[32];
    if (lane == 31) wsum[w] = x;
    if (lane == 0) wtile[w] = o;
    __syncthreads();
    if (w == 0) {
        // inclusive scan of the warp totals, plus the tiles before this one
        int t = wsum[lane];
        const int tt = warp_sum(wtile[lane]);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        wsum[lane] = t + tt;
        if (lane == 0) offset = tt;
    }
    __syncthreads();
    int ex = (w > 0 ? wsum[w - 1] : offset) + x - s;
    if (whole) {
        const int e0 = ex, e1 = e0 + v[0], e2 = e1 + v[1], e3 = e2 + v[2];
        *reinterpret_cast<int4 *>(B.cell_start + base) = make_int4(e0, e1, e2, e3);
        *reinterpret_cast<int4 *>(B.cell_count + base) = make_int4(0, 0, 0, 0);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < n) {
                B.cell_start[base + k] = ex;
                B.cell_count[base + k] = 0;
            }
            ex += v[k];
        }
    }
    if (base <= n && n < base + kScanItems) B.cell_start[n] = K.nf;
    if (no > 0) scan_overflow(K, B, bx * kScanTile, min((bx + 1) * kScanTile, n), no);
}

// The Newton-3 pass's tile table: chunks of kN3Threads particles of each
// cell row, numbered row by row (the pass takes them in that order from a
// ticket, reset here with the step's flag value advanced).  One block.
__device__ __forceinline__ void n3_table(const Consts &K, const Bufs &B)
{
    __shared__ int wsum[32];
    __shared__ int running;
    if (threadIdx.x == 0) running = 0;
    __syncthreads();
#pragma unroll 1
    for (int r0 = 0; r0 < K.ncy; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        int cnt = 0;
        if (r < K.ncy) cnt = B.cell_start[(r + 1) * K.ncx] - B.cell_start[r * K.ncx];
        const int ch = (cnt + kN3Threads - 1) / kN3Threads;
        int total;
        const int base = running + block_exclusive_scan(ch, wsum, &total);
        if (r < K.ncy) {
            B.n3_row_base[r] = base;
            for (int k = 0; k < ch; ++k)
                if (base + k < K.n3_tiles_max) B.n3_tile_row[base + k] = r;
        }
        __syncthreads();
        if (threadIdx.x == 0) running += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.n3_row_base[K.ncy] = min(running, K.n3_tiles_max);
        B.n3_ctl[0] = 0;
        B.n3_ctl[1] = B.n3_ctl[1] + 1;
    }
}

// Stable order inside a cell: rank by fluid ID among the cell's members
// (its bucket, and for a cell of more than kBucket particles the rest, which
// the scan placed in perm_tmp).  Then the reorder into the SoA arrays of this step.  Block 0
// first clears the tile sums and the overflow count for the next step's
// k_drift_key (and builds the Newton-3 pass's tile table).  Closure 0: with the
// predicted density rho~ = band(rho^n + dt (D^n + (dt^n / dt^{n-1})(D^n -
// D^{n-1}))) and its Tait pressure.  Closure 1: with the predicted velocity
// v* = v^{n+1/2} + dt/2 a^n that the pass sees, and {a^n, e^n, De^n} for the
// closing kick (the density comes from k_density).
// The split pass's marks: the pass block of each boundary particle (bnd;
// dst its sorted index) is marked in split_mask, once per pass block of the
// warp, by an atomic whose result is not waited for.  Every lane of the
// warp takes part.
__device__ __forceinline__ void split_flag(const Bufs &B, int dst, bool bnd)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, bnd);
    if (m == 0u) return;
    if (bnd) {
        const int pb = dst / kPassThreads;
        const unsigned same = __match_any_sync(m, pb);
        if (lane == __ffs(same) - 1) atomicOr(&B.split_mask[pb >> 5], 1u << (pb & 31));
    }
}

// The split pass's lists, from the marks (extra blocks of the ghost pass's
// launch): the marked pass blocks into split_bi, their boundary particles
// into split_pi (one atomic per warp for its slots).  Each NT-thread block
// takes NT / kPassThreads pass blocks at a time (bx, nbx: its index among
// the nbx list blocks, grid-stride); the lists' order varies from run to
// run, what is computed from them does not depend on it.
template <int NT>
__device__ __forceinline__ void b_split_list(const Consts &K, const Bufs &B, const int bx, const int nbx)
{
    constexpr int P = NT / kPassThreads;
    const int lane = threadIdx.x & 31, t = threadIdx.x % kPassThreads, h = threadIdx.x / kPassThreads;
#pragma unroll 1
    for (int b0 = bx * P; b0 < K.n_pass_blocks; b0 += nbx * P) {
        const int b = b0 + h;   // this thread's pass block (uniform in each warp)
        if (b >= K.n_pass_blocks || !((B.split_mask[b >> 5] >> (b & 31)) & 1u)) continue;
        const int i = b * kPassThreads + t;
        bool bnd = false;
        if (i < K.nf) {
            const float2 r = B.s_pos[i];
            bnd = !outside_box(K, r.x, r.y) && has_ghost_candidates(K, B, r, cell_of<1>(K, r.x, r.y));
        }
        const unsigned m = __ballot_sync(0xffffffffu, bnd);
        if (m != 0u) {
            const int leader = __ffs(m) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&B.split_n[0], __popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (bnd) B.split_pi[base + __popc(m & ((1u << lane) - 1u))] = i;
        }
        if (t == 0) B.split_bi[atomicAdd(&B.split_n[1], 1)] = b;
    }
}

template <int CL>
__device__ __forceinline__ int rank_scatter_one(const Consts &K, const Bufs &B, const int i, int prime,
                                                bool &bnd);

template <int CL>
__device__ __forceinline__ void b_rank_scatter(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime)
{
    if (bx == 0) {
        if (K.n3) n3_table(K, B);
        const int n_tiles = (K.ncell + 2 + kScanTile - 1) / kScanTile;
        for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) B.tile_sum[t] = 0;
        if (threadIdx.x == 0) *B.ovf_count = 0;   // the scan has placed the list
    }
    const int i = bx * blockDim.x + threadIdx.x;
    bool bnd = false;
    const int dst = i < K.nf ? rank_scatter_one<CL>(K, B, i, prime, bnd) : -1;
    if (K.split) split_flag(B, dst, bnd && dst >= 0);
}

// Particle i of the previous order: its rank, its reorder; returns its
// sorted index (-1 on a failed bounds check), and with K.split whether it
// is a boundary particle.
template <int CL>
__device__ __forceinline__ int rank_scatter_one(const Consts &K, const Bufs &B, const int i, int prime,
                                                bool &bnd)
{
    // the particle's own data first, so their loads overlap the rank loop's
    const int key = B.u_key[i];
    const int id = B.u_id[i];
    const float d = B.st_rho[i];
    const float2 D = B.st_D[i];
    const float2 up = B.u_pos[i];
    float2 uv = B.u_vel[i];
    if (kChecked && !hr_ok(key >= 0 && key <= K.ncell, &B.S->status)) return -1;
    const int cs = B.cell_start[key], ce = B.cell_start[key + 1];
    // (the split pass's test, its loads issued with the cell starts')
    const bool near = K.split && key != K.ncell && has_ghost_candidates(K, B, up, key);
    if (kChecked && !hr_ok(0 <= cs && cs < ce && ce <= K.nf, &B.S->status)) return -1;
    float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 a = make_float2(0.f, 0.f);
    if constexpr (CL == 1) {
        a = B.st_a[i];
        if (key != K.ncell) {
            const float hdt = prime ? 0.0f : 0.5f * B.S->dt_f;
            uv.x = fmaf(hdt, a.x, uv.x);
            uv.y = fmaf(hdt, a.y, uv.y);
        }
    } else {
        float dp = d;
        if (key != K.ncell) {
            const float dt = prime ? 0.0f : B.S->dt_f;
            const float ratio = prime ? 1.0f : B.S->ratio_f;
            dp = band(K, fmaf(dt, fmaf(ratio, D.x - D.y, D.x), d));
        }
        rec = eos_record(K, dp);
    }
    int rank = 0;
    const int n = ce - cs;
    // the cell's bucket as four 16-byte loads issued together (a bucket row
    // is 64 B, aligned), entries past the cell's count left out
    const int4 *bk = reinterpret_cast<const int4 *>(B.bucket + (size_t)key * kBucket);
    static_assert(kBucket == 16, "four int4 loads per bucket");
    int4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = HR_DYNAMIC_LOAD(&bk[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        rank += (4 * u + 0 < n && q[u].x < id) + (4 * u + 1 < n && q[u].y < id) +
                (4 * u + 2 < n && q[u].z < id) + (4 * u + 3 < n && q[u].w < id);
    }
    // slots kBucket.. of an overflowing cell, placed by the scan
    for (int k = cs + kBucket; k < ce; ++k) rank += HR_DYNAMIC_LOAD(&B.perm_tmp[k]) < id;
    const int dst = cs + rank;
    if (kChecked && !hr_ok(dst < ce, &B.S->status)) return -1;
    B.s_pos[dst] = up;
    B.s_vel[dst] = uv;
    if constexpr (CL == 1) B.s_ex[dst] = make_float4(a.x, a.y, D.y, D.x);
    else B.s_aux[dst] = rec;
    B.s_rd[dst] = make_float2(d, D.x);
    B.s_id[dst] = id;
    if (B.perm_dst) B.perm_dst[i] = dst;
    bnd = near;
    return dst;
}

// Predicate mask of the candidates [base, base + cnt), cnt <= 32, in fixed
// blocks of kMaskChunk candidates: each block is unrolled with constant bit
// positions, and the warp's trip count is the largest ceil(cnt / kMaskChunk)
// of its lanes (rows of 17-24 candidates all take three blocks of 8).  The
// last block reads up to kMaskChunk - 1 entries past the row; the position
// array is padded by kPosPad entries so those reads stay inside it, and
// their bits are masked off.
#ifndef HR_MASK_CHUNK
#define HR_MASK_CHUNK 8
#endif
constexpr int kMaskChunk = HR_MASK_CHUNK;
constexpr int kPosPad = 32;
// (SMEM: pos is a shared-memory array, read with plain loads.)
template <bool SMEM = false>
__device__ __forceinline__ unsigned support_mask(const float2 *pos, int base, int cnt, float2 ri,
                                                 float s2)
{
    unsigned m = 0u;
    const float2 *pp = pos + base;
#pragma unroll 1
    for (int k0 = 0; k0 < cnt; k0 += kMaskChunk) {
        unsigned sub = 0u;
#pragma unroll
        for (int u = 0; u < kMaskChunk; ++u)
            sub |= (unsigned)in_support2(ri, SMEM ? pp[k0 + u] : HR_DYNAMIC_LOAD(pp + k0 + u), s2)
                   << u;
        const int rem = cnt - k0;
        if (rem < kMaskChunk) sub &= (1u << rem) - 1u;
        m |= sub << k0;
    }
    return m;
}

// ------------------------------------- closure 1: summation density

// rho_i = sum_j m_j W_ij over the particle itself, its fluid neighbours and
// the wall and disk ghosts (eq. density-sum; the ghosts complete the sum at
// a boundary), in units of the deviation d = rho/rho0 - 1, then the band.
// The pressure uses the predicted energy e* = e^n + dt De^n.  A particle
// outside the box keeps its density and energy.
__device__ __forceinline__ void b_density(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime)
{
    const int i = bx * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    const float2 ri = B.s_pos[i];
    const float4 ex = B.s_ex[i];
    float d, e;
    if (outside_box(K, ri.x, ri.y)) {
        d = B.s_rd[i].x;
        e = ex.z;
    } else {
        auto w_at = [&](float x, float y) {
            const float dx = ri.x - x, dy = ri.y - y;
            return cubic_w(K, sqrtf(fmaf(dx, dx, dy * dy)));
        };
        float S = K.self_w - 1.0f;
        const int c = cell_of(K, ri.x, ri.y);
        // the stencil rows: predicate masks over blocks of up to 32
        // candidates (unrolled, independent loads), then the set bits in
        // ascending order
        const int R = K.sr;
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            const int row = c + dy * K.ncx;
            if (kChecked && !hr_ok(row - R >= 0 && row + R + 1 <= K.ncell, &B.S->status)) continue;
            const int a = B.cell_start[row - R], b = B.cell_start[row + R + 1];
            if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
#pragma unroll 1
            for (int base = a; base < b; base += 32) {
                unsigned m = support_mask(B.s_pos, base, min(32, b - base), ri, K.s2);
                if (i >= base && i < base + 32) m &= ~(1u << (i - base));
                while (m) {
                    const int j = base + __ffs(m) - 1;
                    m &= m - 1u;
                    const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
                    S = fmaf(K.m_over_rho0, w_at(rj.x, rj.y), S);
                }
            }
        }
        if (K.nw > 0) {
            const float mw = K.m_over_rho0 * K.wall_over_m;
            for_fluid_candidates(K, B.wall_start, c, K.nw, &B.S->status, [&](int k) {
                const float2 rg = __ldg(&B.gw_pos[k]);
                if (in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) S = fmaf(mw, w_at(rg.x, rg.y), S);
            });
        }
        const float xc = B.S->xc_f, yc = B.S->yc_f;
        if (K.ng > 0 && near_disk(K, ri.x, ri.y, xc, yc)) {
            const float md = K.m_over_rho0 * K.disk_over_m;
            for_disk_arc(K, disk_arc(K, ri.x, ri.y, xc, yc), &B.S->status, [&](int k) {
                const float2 rg = B.gd_pos[k];
                if (outside_box(K, rg.x, rg.y) || !in_support(ri.x, ri.y, rg.x, rg.y, K.s2))
                    return;
                S = fmaf(md, w_at(rg.x, rg.y), S);
            });
        }
        d = band(K, S);
        e = fmaf(prime ? 0.0f : B.S->dt_f, ex.w, ex.z);
    }
    B.s_aux[i] = mg_record(K, d, e);
}

// ------------------------------------------------------- a4: ghosts G

// Adami extrapolation (eqs. adami-p, adami-v) for wall ghosts [0, nw) and
// disk ghosts [nw, nw + ng), over fluid neighbours in the 3x3 cell stencil:
//   p_g = max((S_p + (g - a_w) . S_rr) / S_W, p_cav),
//   rho_g = rho0 (1 + p_g / (rho0 c0^2)),  v_g = 2 v_w - S_v / S_W.
// kGhostLanes lanes per ghost (four ghosts per warp): the lanes split the
// stencil's candidates, then the six Shepard sums are combined over the
// ghost's lanes by a butterfly of shuffles.
template <int CL>
__device__ __forceinline__ void b_ghost(const Consts &K, const Bufs &B, const int bx, const int nbx)
{
    __shared__ float red[kGhostWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int sub = lane & (kGhostLanes - 1);
    const int g = bx * kGhostsPerBlock + (int)threadIdx.x / kGhostLanes;
    const bool active = g < K.nw + K.ng;
    const bool disk = g >= K.nw;
    float2 rg = make_float2(0.f, 0.f);
    bool inside = false;
    float SW = 0.f, Sp = 0.f, Srx = 0.f, Sry = 0.f, Svx = 0.f, Svy = 0.f;
    if (active) {
        rg = disk ? B.gd_pos[g - K.nw] : B.gw_pos[g];
        inside = !outside_box(K, rg.x, rg.y);
    }
    if (inside) {
        const int c = cell_of(K, rg.x, rg.y);
        const int R = K.sr;
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            const int row = c + dy * K.ncx;
            if (kChecked && !hr_ok(row - R >= 0 && row + R + 1 <= K.ncell, &B.S->status)) continue;
            const int a = B.cell_start[row - R], b = B.cell_start[row + R + 1];
            if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
            for (int j = a + sub; j < b; j += kGhostLanes) {
                const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
                if (!in_support(rg.x, rg.y, rj.x, rj.y, K.s2)) continue;
                const float dx = rg.x - rj.x, dy2 = rg.y - rj.y;
                const float W = kernel_w<CL>(K, sqrtf(fmaf(dx, dx, dy2 * dy2)));
                const float4 aux = HR_DYNAMIC_LOAD(&B.s_aux[j]);
                const float2 vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
                const float rw = (1.0f + aux.x) * W;
                SW += W;
                Sp = fmaf(aux.y, W, Sp);
                Srx = fmaf(rw, dx, Srx);
                Sry = fmaf(rw, dy2, Sry);
                Svx = fmaf(vj.x, W, Svx);
                Svy = fmaf(vj.y, W, Svy);
            }
        }
    }
    // the ghost's kGhostLanes lanes combine their sums (every lane takes part)
#pragma unroll
    for (int o = kGhostLanes / 2; o > 0; o >>= 1) {
        SW += __shfl_xor_sync(0xffffffffu, SW, o);
        Sp += __shfl_xor_sync(0xffffffffu, Sp, o);
        Srx += __shfl_xor_sync(0xffffffffu, Srx, o);
        Sry += __shfl_xor_sync(0xffffffffu, Sry, o);
        Svx += __shfl_xor_sync(0xffffffffu, Svx, o);
        Svy += __shfl_xor_sync(0xffffffffu, Svy, o);
    }
    float vabs = 0.0f;
    if (active) {
        const float vwx = disk ? B.S->vproj_f : 0.0f;
        const float awx = disk ? B.S->aproj_f : 0.0f;
        float4 aux;
        float2 vg;
        if (SW > 0.0f) {
            const float inv = 1.0f / SW;
            const float bx = K.gx - awx, by = K.gy;
            float pg = (Sp + K.rho0 * (bx * Srx + by * Sry)) * inv;
            pg = fmaxf(pg, K.p_cav);
            const float dg = pg * K.inv_rho0c02;
            const float rho = K.rho0 * (1.0f + dg);
            aux = make_float4(dg, pg, pg / (rho * rho),
                              CL == 1 ? 0.0f : -K.alpha_h * sound_speed(K, dg));
            vg = make_float2(2.0f * vwx - Svx * inv, -Svy * inv);
        } else {
            aux = make_float4(0.0f, 0.0f, 0.0f, CL == 1 ? 0.0f : -K.alpha_h * K.c0);
            vg = make_float2(vwx, 0.0f);
        }
        if (sub == 0) {
            B.g_aux[g] = aux;
            B.g_vel[g] = vg;
        }
        if (inside) vabs = sqrtf(vg.x * vg.x + vg.y * vg.y);
    }
    vabs = warp_max(vabs);
    if (lane == 0) red[w] = vabs;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.0f;
        for (int k = 0; k < kGhostWarps; ++k) v = fmaxf(v, red[k]);
        B.ghost_vmax[bx] = v;
        atomicMax(&B.S->vmax_bits, __float_as_uint(v));   // for the deferred close
    }
}

// --------------------------------------------- a5: fused interaction L

struct Self {
    float2 r, v;
    float rho, P, c;
};

struct Acc {
    float2 a, X, av;
    float dr;
};

// One pair (i, j): continuity, momentum with artificial and laminar
// viscosity (eqs. momentum, artificial-viscosity) and, when xsph, the XSPH
// sum (eq. xsph).  Adds mj times the pair terms (mj = 1 for fluid pairs: the
// uniform fluid mass is applied once per particle) and returns the
// acceleration contribution of j on i per unit mass mj.  I.c and cj hold
// -alpha h c, so Pi_ij = (c'_i + c'_j) min(v_ij . r_ij, 0) / ((r^2 + eta^2 h^2)
// (rho_i + rho_j)) is -alpha cbar mu / rhobar under approach and 0 otherwise.
// Closure 0 accumulates the continuity sum in A.dr; closure 1 the energy
// equation's sum (P_i + P_j + Pi_ij) v_ij . m_j grad_i W_ij (halved and
// scaled by the fluid mass in the epilogue).
// The x and y halves of the vector terms run as packed pairs.
template <int CL>
__device__ __forceinline__ float2 pair_terms(const Consts &K, const Self &I, float2 rj, float2 vj,
                                             float rhoj, float Pj, float cj, float mj, bool xsph,
                                             Acc &A)
{
    const float2 d = p2_sub(I.r, rj);
    const float dx = d.x, dy = d.y;
    const float r2 = fmaf(dx, dx, dy * dy);
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));     // 0 for coincident particles
    float t = 0.0f, t3 = 0.0f, F;
    if constexpr (CL == 1) {
        F = mj * cubic_F(K, r);
    } else {
        t = fmaxf(fmaf(-r, K.half_inv_h, 1.0f), 0.0f);
        t3 = t * t * t;
        F = mj * K.Fc * t3;                             // m_j grad_i W = F r_ij
    }
    const float2 v = p2_sub(I.v, vj);
    const float vr = fmaf(v.x, dx, v.y * dy);
    if constexpr (CL == 0) A.dr = fmaf(F, vr, A.dr);   // continuity
    const float e = r2 + K.eh2;
    const float inv = __fdividef(1.0f, e * (I.rho + rhoj));
    const float Pi_ij = (I.c + cj) * fminf(vr, 0.0f) * inv;
    const float PF = (I.P + Pj + Pi_ij) * F;
    if constexpr (CL == 1) A.dr = fmaf(PF, vr, A.dr);  // internal energy
    const float lam = K.nu4 * F * r2 * inv;             // laminar
    const float2 f = p2_fma(make_float2(-PF, -PF), d, p2_mul(make_float2(lam, lam), v));
    A.a = p2_add(A.a, f);
    const float av = Pi_ij * F;                         // minus the AV acceleration factor
    A.av = p2_fma(make_float2(-av, -av), d, A.av);
    if (xsph) {
        // -(m_j / rhobar) W = -2 W / (rho_i + rho_j) (mj = 1)
        float wx;
        if constexpr (CL == 1) wx = -2.0f * cubic_w(K, r) * (inv * e);
        else wx = K.m2Wc * t3 * t * fmaf(r, K.two_inv_h, 1.0f) * (inv * e);
        A.X = p2_fma(make_float2(wx, wx), v, A.X);
    }
    return f;
}

// The fused interaction pass.  One thread per sorted fluid particle i.
// Phase 1: for each of the three stencil rows, the float predicate of each
// candidate sets one bit of a mask (unrolled loads, no per-candidate
// branching).  Phase 2: one loop over the set bits of all three masks
// evaluates the pair terms, so a warp runs as many iterations as its busiest
// lane has neighbours.  Rows with more than 32 candidates are handled in
// chunks on the spot.  Ghost neighbours follow (static wall lists, then the
// disk ring).  The epilogue applies the uniform fluid mass, the corrected
// density and the closing half kick.  Block partials of the ghost forces,
// the dissipation rate and max |v| are reduced in FP32 per warp and over the
// block's warps in a fixed order; k_finalize sums the block partials in
// compensated FP32.

// Per-thread partials of a pass block (def: the particle is a boundary
// particle, whose dissipation goes to the block's boundary share).
struct PassPart {
    float fdx, fdy, fw, diss, vmax;
    int npen;
    int def;
};

// Phase 1 and 2 of particle i (inside the box): fluid neighbours into A.
template <int CL>
__device__ __forceinline__ void pass_fluid(const Consts &K, const Bufs &B, int i, float2 ri,
                                           int c, const Self &I, Acc &A)
{
    auto fluid_pair = [&](int j) {
        const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
        const float2 vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
        const float4 aj = HR_DYNAMIC_LOAD(&B.s_aux[j]);
        pair_terms<CL>(K, I, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z,
                       CL == 1 ? K.c_av : aj.w, 1.0f, true, A);
    };
    int base0, base1, base2;
    unsigned m0, m1, m2;
    {
        const int r0 = c - K.ncx, r1 = c, r2 = c + K.ncx;
        if (kChecked && !hr_ok(r0 - 1 >= 0 && r2 + 2 <= K.ncell, &B.S->status)) return;
        base0 = B.cell_start[r0 - 1];
        base1 = B.cell_start[r1 - 1];
        base2 = B.cell_start[r2 - 1];
        const int e0 = B.cell_start[r0 + 2], e1 = B.cell_start[r1 + 2],
                  e2 = B.cell_start[r2 + 2];
        if (kChecked && !(row_ok(K, r0, base0, e0, K.nf, &B.S->status) &&
                          row_ok(K, r1, base1, e1, K.nf, &B.S->status) &&
                          row_ok(K, r2, base2, e2, K.nf, &B.S->status)))
            return;
        // rows longer than 32 candidates: chunks evaluated right away
        auto row_mask = [&](int a, int b) -> unsigned {
            if (b - a <= 32) return support_mask(B.s_pos, a, b - a, ri, K.s2);
#pragma unroll 1
            for (int base = a; base < b; base += 32) {
                unsigned m = support_mask(B.s_pos, base, min(32, b - base), ri, K.s2);
                if (i >= base && i < base + 32) m &= ~(1u << (i - base));
                while (m) {
                    const int j = base + __ffs(m) - 1;
                    m &= m - 1u;
                    fluid_pair(j);
                }
            }
            return 0u;
        };
        m0 = row_mask(base0, e0);
        m1 = row_mask(base1, e1);
        m2 = row_mask(base2, e2);
        // the particle itself sits in the middle row
        if (i >= base1 && i < base1 + 32) m1 &= ~(1u << (i - base1));
    }
#pragma unroll 1
    while ((m0 | m1 | m2) != 0u) {
        int j;
        if (m0) {
            j = base0 + __ffs(m0) - 1;
            m0 &= m0 - 1u;
        } else if (m1) {
            j = base1 + __ffs(m1) - 1;
            m1 &= m1 - 1u;
        } else {
            j = base2 + __ffs(m2) - 1;
            m2 &= m2 - 1u;
        }
        fluid_pair(j);
    }
}

// Phases 1 and 2 on cells of side >= h (K.sr = 2): the 5 x 5 stencil as
// five row ranges of five cells each, in the same order (rows from below,
// candidates in sorted order within a row).
template <int CL>
__device__ __forceinline__ void pass_fluid5(const Consts &K, const Bufs &B, int i, float2 ri,
                                            int c, const Self &I, Acc &A)
{
    auto fluid_pair = [&](int j) {
        const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
        const float2 vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
        const float4 aj = HR_DYNAMIC_LOAD(&B.s_aux[j]);
        pair_terms<CL>(K, I, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z,
                       CL == 1 ? K.c_av : aj.w, 1.0f, true, A);
    };
    int base[5];
    unsigned m[5];
    auto row_mask = [&](int a, int b) -> unsigned {
        if (b - a <= 32) return support_mask(B.s_pos, a, b - a, ri, K.s2);
#pragma unroll 1
        for (int bs = a; bs < b; bs += 32) {
            unsigned mm = support_mask(B.s_pos, bs, min(32, b - bs), ri, K.s2);
            if (i >= bs && i < bs + 32) mm &= ~(1u << (i - bs));
            while (mm) {
                const int j = bs + __ffs(mm) - 1;
                mm &= mm - 1u;
                fluid_pair(j);
            }
        }
        return 0u;
    };
    if (kChecked && !hr_ok(c - 2 * K.ncx - 2 >= 0 && c + 2 * K.ncx + 3 <= K.ncell, &B.S->status))
        return;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int row = c + (r - 2) * K.ncx;
        base[r] = B.cell_start[row - 2];
        const int e = B.cell_start[row + 3];
        if (kChecked && !row_ok(K, row, base[r], e, K.nf, &B.S->status)) return;
        m[r] = row_mask(base[r], e);
    }
    if (i >= base[2] && i < base[2] + 32) m[2] &= ~(1u << (i - base[2]));
#pragma unroll 1
    while ((m[0] | m[1] | m[2] | m[3] | m[4]) != 0u) {
        int j;
        if (m[0]) {
            j = base[0] + __ffs(m[0]) - 1;
            m[0] &= m[0] - 1u;
        } else if (m[1]) {
            j = base[1] + __ffs(m[1]) - 1;
            m[1] &= m[1] - 1u;
        } else if (m[2]) {
            j = base[2] + __ffs(m[2]) - 1;
            m[2] &= m[2] - 1u;
        } else if (m[3]) {
            j = base[3] + __ffs(m[3]) - 1;
            m[3] &= m[3] - 1u;
        } else {
            j = base[4] + __ffs(m[4]) - 1;
            m[4] &= m[4] - 1u;
        }
        fluid_pair(j);
    }
}

// The same phases with the block's candidates staged in shared memory (a
// measured variant of the pass, HR_FLAG_STAGE_POS / HR_FLAG_STAGE_ALL).
// When every in-box particle of a pass block lies in one cell row, the three
// stencil rows of all of them are three contiguous ranges of the sorted
// arrays, [start(c_min + dy ncx - 1), start(c_max + dy ncx + 2)) for dy =
// -1, 0, 1 (cell_start is monotone).  The block copies those ranges once --
// the positions (SV = 1), or the positions, velocities and EOS records
// (SV = 2) -- and the predicate (and the pair terms) read them there.  A
// block that spans two cell rows, or whose ranges exceed kStageCap, takes
// the global path.  The candidates, their order and the arithmetic are
// those of pass_fluid, so the results are the same bit for bit.
constexpr int kStageCap = 192;
template <int SV>
struct PassStage {
    int lo[3], n[3];
    int ok;
    float2 pos[3][kStageCap + kMaskChunk];
    float2 vel[SV == 2 ? 3 : 1][SV == 2 ? kStageCap : 1];
    float4 aux[SV == 2 ? 3 : 1][SV == 2 ? kStageCap : 1];
};

template <int SV>
__device__ __forceinline__ void stage_rows(const Consts &K, const Bufs &B, int bx, PassStage<SV> &st)
{
    __shared__ int cmin, cmax;
    if (threadIdx.x == 0) {
        cmin = 0x7fffffff;
        cmax = -1;
    }
    __syncthreads();
    const int i = bx * kPassThreads + threadIdx.x;
    int lo = 0x7fffffff, hi = -1;
    if (i < K.nf) {
        const float2 r = B.s_pos[i];
        if (!outside_box(K, r.x, r.y)) lo = hi = cell_of(K, r.x, r.y);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&cmin, lo);
        atomicMax(&cmax, hi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = cmax >= 0 && cmin / K.ncx == cmax / K.ncx;
        for (int r = 0; r < 3 && ok; ++r) {
            const int a = B.cell_start[cmin + (r - 1) * K.ncx - 1];
            const int b = B.cell_start[cmax + (r - 1) * K.ncx + 2];
            if (kChecked && !hr_ok(a >= 0 && a <= b && b <= K.nf, &B.S->status)) ok = 0;
            st.lo[r] = a;
            st.n[r] = b - a;
            ok = ok && b - a <= kStageCap;
        }
        st.ok = ok;
    }
    __syncthreads();
    if (!st.ok) return;
#pragma unroll 1
    for (int r = 0; r < 3; ++r) {
        const int a = st.lo[r], n = st.n[r];
        for (int k = threadIdx.x; k < n + kMaskChunk; k += kPassThreads) {
            // entries past the range: far away (their bits are masked off too)
            st.pos[r][k] = k < n ? HR_DYNAMIC_LOAD(&B.s_pos[a + k]) : make_float2(3e38f, 3e38f);
            if constexpr (SV == 2) {
                if (k < n) {
                    st.vel[r][k] = HR_DYNAMIC_LOAD(&B.s_vel[a + k]);
                    st.aux[r][k] = HR_DYNAMIC_LOAD(&B.s_aux[a + k]);
                }
            }
        }
    }
    __syncthreads();
}

template <int CL, int SV>
__device__ __forceinline__ void pass_fluid_staged(const Consts &K, const Bufs &B, int i, float2 ri,
                                                  int c, const Self &I, Acc &A,
                                                  const PassStage<SV> &st)
{
    auto fluid_pair = [&](int r, int j) {
        const int k = j - st.lo[r];
        const float2 rj = st.pos[r][k];
        float2 vj;
        float4 aj;
        if constexpr (SV == 2) {
            vj = st.vel[r][k];
            aj = st.aux[r][k];
        } else {
            vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
            aj = HR_DYNAMIC_LOAD(&B.s_aux[j]);
        }
        pair_terms<CL>(K, I, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z,
                       CL == 1 ? K.c_av : aj.w, 1.0f, true, A);
    };
    int base0, base1, base2;
    unsigned m0, m1, m2;
    {
        const int r0 = c - K.ncx, r1 = c, r2 = c + K.ncx;
        base0 = B.cell_start[r0 - 1];
        base1 = B.cell_start[r1 - 1];
        base2 = B.cell_start[r2 - 1];
        const int e0 = B.cell_start[r0 + 2], e1 = B.cell_start[r1 + 2],
                  e2 = B.cell_start[r2 + 2];
        if (kChecked && !(hr_ok(base0 >= st.lo[0] && e0 <= st.lo[0] + st.n[0], &B.S->status) &&
                          hr_ok(base1 >= st.lo[1] && e1 <= st.lo[1] + st.n[1], &B.S->status) &&
                          hr_ok(base2 >= st.lo[2] && e2 <= st.lo[2] + st.n[2], &B.S->status)))
            return;
        auto row_mask = [&](int r, int a, int b) -> unsigned {
            if (b - a <= 32) return support_mask<true>(st.pos[r], a - st.lo[r], b - a, ri, K.s2);
#pragma unroll 1
            for (int base = a; base < b; base += 32) {
                unsigned m = support_mask<true>(st.pos[r], base - st.lo[r], min(32, b - base), ri,
                                                K.s2);
                if (i >= base && i < base + 32) m &= ~(1u << (i - base));
                while (m) {
                    const int j = base + __ffs(m) - 1;
                    m &= m - 1u;
                    fluid_pair(r, j);
                }
            }
            return 0u;
        };
        m0 = row_mask(0, base0, e0);
        m1 = row_mask(1, base1, e1);
        m2 = row_mask(2, base2, e2);
        if (i >= base1 && i < base1 + 32) m1 &= ~(1u << (i - base1));
    }
#pragma unroll 1
    while ((m0 | m1 | m2) != 0u) {
        int j, r;
        if (m0) {
            j = base0 + __ffs(m0) - 1;
            m0 &= m0 - 1u;
            r = 0;
        } else if (m1) {
            j = base1 + __ffs(m1) - 1;
            m1 &= m1 - 1u;
            r = 1;
        } else {
            j = base2 + __ffs(m2) - 1;
            m2 &= m2 - 1u;
            r = 2;
        }
        fluid_pair(r, j);
    }
}

// The wall and disk ghost neighbours of a particle (inside the box) into A,
// their forces into the block partials (split over lanes as
// for_fluid_candidates); P.def is set where there are ghost candidates (the
// test of has_ghost_candidates).
template <int CL, int R = 0>
__device__ __forceinline__ void pass_ghosts(const Consts &K, const Bufs &B, float2 ri, int c,
                                            const Self &I, Acc &A, PassPart &P, int lane = 0,
                                            int lanes = 1)
{
    // wall ghosts (static cell list)
    if (K.nw > 0 && B.wall_near[c] != 0) {
        P.def = 1;
        for_fluid_candidates<R>(K, B.wall_start, c, K.nw, &B.S->status, [&](int k) {
            const float2 rg = __ldg(&B.gw_pos[k]);
            if (!in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) return;
            const float4 ag = B.g_aux[k];
            const float2 vg = B.g_vel[k];
            const float2 f = pair_terms<CL>(K, I, rg, vg, fmaf(K.rho0, ag.x, K.rho0),
                                            ag.z, CL == 1 ? K.c_av : ag.w,
                                            K.wall_over_m, false, A);
            if (__ldg(&B.gw_kind[k]) == KIND_SIDE) {
                const float2 e = __ldg(&B.gw_nrm[k]);
                P.fw -= f.x * e.x + f.y * e.y;
            }
        }, lane, lanes);
    }
    // disk ghosts (the ring, only near the disk)
    if (K.ng > 0) {
        const float xc = B.S->xc_f, yc = B.S->yc_f;
        if (near_disk(K, ri.x, ri.y, xc, yc)) {
            P.def = 1;
            for_disk_arc(K, disk_arc(K, ri.x, ri.y, xc, yc), &B.S->status, [&](int k) {
                const float2 rg = B.gd_pos[k];
                if (outside_box(K, rg.x, rg.y)) return;
                if (!in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) return;
                const float4 ag = B.g_aux[K.nw + k];
                const float2 vg = B.g_vel[K.nw + k];
                const float2 f = pair_terms<CL>(K, I, rg, vg, fmaf(K.rho0, ag.x, K.rho0),
                                                ag.z, CL == 1 ? K.c_av : ag.w,
                                                K.disk_over_m, false, A);
                P.fdx += f.x;
                P.fdy += f.y;
            }, lane, lanes);
            const float ddx = ri.x - xc, ddy = ri.y - yc;
            if (lane == 0) P.npen += ddx * ddx + ddy * ddy < K.R2 ? 1 : 0;
        }
    }
}

// The epilogue of particle i (inside the box), its sums complete in A.
template <int CL>
__device__ __forceinline__ void pass_close(const Consts &K, const Bufs &B, int i, float2 vi,
                                           float4 ai, float2 rd, float dt, int prime, Acc &A,
                                           PassPart &P)
{
    const float ax = fmaf(K.m, A.a.x, K.gx), ay = fmaf(K.m, A.a.y, K.gy);
    float2 vnew;
    if constexpr (CL == 1) {
        // closing kick from the predicted velocity, v^{n+1} = v* +
        // dt/2 (a^{n+1} - a^n); energy e^{n+1} = e^n + dt/2 (De^n + De^{n+1})
        const float4 ex = B.s_ex[i];
        const float De = 0.5f * K.m * A.dr;
        const float hdt = 0.5f * dt;
        vnew = make_float2(fmaf(hdt, ax - ex.x, vi.x), fmaf(hdt, ay - ex.y, vi.y));
        const float enew = fmaf(hdt, ex.w + De, ex.z);
        if (!isfinite(vnew.x) || !isfinite(vnew.y) || !isfinite(enew))
            atomicOr(&B.S->status, ST_NAN);
        B.st_rho[i] = ai.x;
        B.st_D[i] = make_float2(De, enew);
    } else {
        // epilogue: the fluid mass, corrected density, closing half kick (T)
        const float Dd = A.dr * K.m_over_rho0;
        const float dnew = band(K, fmaf(dt, Dd, rd.x));
        vnew = make_float2(fmaf(0.5f * dt, ax, vi.x), fmaf(0.5f * dt, ay, vi.y));
        if (!isfinite(vnew.x) || !isfinite(vnew.y) || !isfinite(dnew))
            atomicOr(&B.S->status, ST_NAN);
        B.st_rho[i] = dnew;
        B.st_D[i] = make_float2(Dd, prime ? Dd : rd.y);
    }
    B.st_vel[i] = vnew;
    B.st_a[i] = make_float2(ax, ay);
    B.st_X[i] = make_float2(K.m * A.X.x, K.m * A.X.y);
    P.vmax = fmaxf(P.vmax, sqrtf(vnew.x * vnew.x + vnew.y * vnew.y));
    P.diss += -K.m * K.m * (vi.x * A.av.x + vi.y * A.av.y);
}

// Ghost neighbours and the epilogue of particle i (inside the box), its
// fluid sums already in A.
template <int CL, int R = 0>
__device__ __forceinline__ void pass_finish(const Consts &K, const Bufs &B, int i, float2 ri,
                                            float2 vi, float4 ai, float2 rd, int c, float dt,
                                            int prime, const Self &I, Acc &A, PassPart &P)
{
    pass_ghosts<CL, R>(K, B, ri, c, I, A, P);
    pass_close<CL>(K, B, i, vi, ai, rd, dt, prime, A, P);
}

// A frozen particle (outside the box) keeps its state, takes part in nothing.
template <int CL>
__device__ __forceinline__ void pass_frozen(const Bufs &B, int i, float2 vi, float2 rd)
{
    B.st_vel[i] = vi;
    B.st_rho[i] = rd.x;
    B.st_a[i] = make_float2(0.f, 0.f);
    B.st_D[i] = make_float2(0.f, CL == 1 ? B.s_ex[i].z : 0.f);
    B.st_X[i] = make_float2(0.f, 0.f);
}

// Which particles a pass launch takes: all of them, only the interior ones
// (no ghost candidates; the split pass's first part, which does not wait for
// the ghost states), or only the boundary ones (its second part).
enum PassMode { kPassAll = 0, kPassInterior = 1, kPassBoundary = 2 };

// R: the stencil reach (1 or 2), or 0 to take it from K.sr (batched and
// persistent kernels, whose cases may differ).  kPassBoundary is handed
// boundary particles only (the reorder's list).
template <int CL, int R = 0, int MODE = kPassAll>
__device__ __forceinline__ void pass_single(const Consts &K, const Bufs &B, int i, float dt,
                                            int prime, PassPart &P)
{
    const float2 ri = B.s_pos[i];
    const float2 vi = B.s_vel[i];
    const float4 ai = B.s_aux[i];
    const float2 rd = B.s_rd[i];
    if (outside_box(K, ri.x, ri.y)) {
        if (MODE != kPassBoundary) pass_frozen<CL>(B, i, vi, rd);
        return;
    }
    const int c = cell_of<R>(K, ri.x, ri.y);
    if (MODE == kPassInterior && has_ghost_candidates(K, B, ri, c)) return;
    const float ci = CL == 1 ? K.c_av : ai.w;
    const Self I{ri, vi, fmaf(K.rho0, ai.x, K.rho0), ai.z, ci};
    Acc A{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
    if (R == 2 || (R == 0 && K.sr == 2)) pass_fluid5<CL>(K, B, i, ri, c, I, A);
    else pass_fluid<CL>(K, B, i, ri, c, I, A);
    if (MODE == kPassInterior) pass_close<CL>(K, B, i, vi, ai, rd, dt, prime, A, P);
    else pass_finish<CL, R>(K, B, i, ri, vi, ai, rd, c, dt, prime, I, A, P);
}

// Block partials of a pass block: FP32 within the warp, then a fixed-order
// sum over the block's warps, into out at index bx.  The dissipation rate is
// summed as two shares, the interior particles' and the boundary particles'
// (P.def), added last: the split pass forms the two shares in separate
// kernels and k_finalize adds them, so every pass form gives the same bits.
template <int NT>
__device__ __forceinline__ void pass_block_partials(const PassPartials &out, const int bx, PassPart P,
                                                    unsigned *vall)
{
    __shared__ float red[NT / 32][6];
    __shared__ int redn[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float da = P.def ? 0.f : P.diss, db = P.def ? P.diss : 0.f;
    // most warps meet no ghost: their ghost sums and boundary share are all
    // zero, and lane 0 already holds the warp's sum
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
    if (threadIdx.x == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a5 = 0.f, v = 0.f;
        int np = 0;
        for (int k = 0; k < NT / 32; ++k) {
            a0 += red[k][0];
            a1 += red[k][1];
            a2 += red[k][2];
            a3 += red[k][3];
            a5 += red[k][5];
            v = fmaxf(v, red[k][4]);
            np += redn[k];
        }
        out.f[bx] = make_float4(a0, a1, a2, a3 + a5);
        out.vmax[bx] = v;
        out.npen[bx] = np;
        // the step's max |v| for the deferred close (v >= 0: its float bits
        // order as the values do)
        atomicMax(vall, __float_as_uint(v));
    }
}

template <int CL, int R = 0, int MODE = kPassAll>
__device__ __forceinline__ void b_pass(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime)
{
    const int i = bx * blockDim.x + threadIdx.x;
    const float dt = prime ? 0.0f : B.S->dt_f;
    PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (i < K.nf) pass_single<CL, R, MODE>(K, B, i, dt, prime, P);
    pass_block_partials<kPassThreads>(B.part, bx, P, &B.S->vmax_bits);
}

// The split pass's boundary part: the listed boundary particles, one per
// thread in list order (grid-stride), each through the whole pass (fluid
// and ghost neighbours, epilogue); its block-partial terms are left at its
// sorted index for b_pass_boundary_sums.
template <int CL>
__device__ __forceinline__ void b_pass_boundary(const Consts &K, const Bufs &B, int prime)
{
    const int n = B.split_n[0];
    const float dt = prime ? 0.0f : B.S->dt_f;
#pragma unroll 1
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = B.split_pi[k];
        if (kChecked && !hr_ok(i >= 0 && i < K.nf, &B.S->status)) continue;
        PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
        pass_single<CL, 1, kPassBoundary>(K, B, i, dt, prime, P);
        B.split_pf[i] = make_float4(P.fdx, P.fdy, P.fw, P.diss);
        B.split_pv[i] = make_int2(__float_as_int(P.vmax), P.npen);
    }
}

// The boundary share of the partials of each listed pass block: the block's
// boundary particles' terms, the others' zero, through the same warp and
// block sums as pass_block_partials (one 128-thread block per listed pass
// block, grid-stride).
__device__ __forceinline__ void b_pass_boundary_sums(const Consts &K, const Bufs &B)
{
    const int n = B.split_n[1];
#pragma unroll 1
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int bx = B.split_bi[k];
        const int i = bx * kPassThreads + threadIdx.x;
        PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
        if (i < K.nf) {
            const float2 ri = B.s_pos[i];
            if (!outside_box(K, ri.x, ri.y) && has_ghost_candidates(K, B, ri, cell_of<1>(K, ri.x, ri.y))) {
                const float4 f = B.split_pf[i];
                const int2 v = B.split_pv[i];
                P = PassPart{f.x, f.y, f.z, f.w, __int_as_float(v.x), v.y, 1};
            }
        }
        pass_block_partials<kPassThreads>(B.part_b, bx, P, &B.S->vmax_bits);
        __syncthreads();   // the reduction's shared arrays, before the next block
    }
}

// The pass block with staged candidates (see PassStage).
template <int CL, int SV>
__device__ __forceinline__ void b_pass_staged(const Consts &K, const Bufs &B, const int bx, int prime)
{
    __shared__ PassStage<SV> st;
    stage_rows<SV>(K, B, bx, st);
    const int i = bx * kPassThreads + threadIdx.x;
    const float dt = prime ? 0.0f : B.S->dt_f;
    PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
    if (i < K.nf) {
        const float2 ri = B.s_pos[i];
        const float2 vi = B.s_vel[i];
        const float4 ai = B.s_aux[i];
        const float2 rd = B.s_rd[i];
        if (outside_box(K, ri.x, ri.y)) {
            pass_frozen<CL>(B, i, vi, rd);
        } else {
            const float ci = CL == 1 ? K.c_av : ai.w;
            const Self I{ri, vi, fmaf(K.rho0, ai.x, K.rho0), ai.z, ci};
            Acc A{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
            const int c = cell_of(K, ri.x, ri.y);
            if (st.ok) pass_fluid_staged<CL, SV>(K, B, i, ri, c, I, A, st);
            else pass_fluid<CL>(K, B, i, ri, c, I, A);
            pass_finish<CL>(K, B, i, ri, vi, ai, rd, c, dt, prime, I, A, P);
        }
    }
    pass_block_partials<kPassThreads>(B.part, bx, P, &B.S->vmax_bits);
}

// The pass with each particle's work split over L consecutive lanes (a
// measured variant for small cases, HR_FLAG_PASS_LANES2 / _LANES4).  The
// candidates of the three stencil rows, in blocks of kMaskChunk taken in
// order, go to the lanes in turn (block g to lane g mod L); each lane
// evaluates the pairs of its blocks, then its share of the wall and disk
// ghosts, and the L partial sums are combined by a butterfly of shuffles
// (every lane ends with the same sums); the first lane closes the particle.
// The candidates and the pair arithmetic are the plain pass's; only the
// order of the sums differs, so results agree with it to rounding and runs
// are reproducible.
template <int L>
__device__ __forceinline__ float lane_group_sum(float v)
{
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int CL, int L>
__global__ void __launch_bounds__(kPassThreads) k_pass_lanes(Consts K, Bufs B, int prime)
{
    constexpr int PPB = kPassThreads / L;
    const int lane = threadIdx.x % L;
    const int i = blockIdx.x * PPB + threadIdx.x / L;
    const float dt = prime ? 0.0f : B.S->dt_f;
    PassPart P{0.f, 0.f, 0.f, 0.f, 0.f, 0};
    Acc A{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), 0.f};
    bool live = false;
    float2 ri = make_float2(0.f, 0.f), vi = make_float2(0.f, 0.f), rd = make_float2(0.f, 0.f);
    float4 ai = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < K.nf) {
        ri = B.s_pos[i];
        vi = B.s_vel[i];
        ai = B.s_aux[i];
        rd = B.s_rd[i];
        if (outside_box(K, ri.x, ri.y)) {
            if (lane == 0) pass_frozen<CL>(B, i, vi, rd);
        } else {
            live = true;
        }
    }
    if (live) {
        const Self I{ri, vi, fmaf(K.rho0, ai.x, K.rho0), ai.z, CL == 1 ? K.c_av : ai.w};
        const int c = cell_of(K, ri.x, ri.y);
        auto fluid_pair = [&](int j) {
            const float2 rj = HR_DYNAMIC_LOAD(&B.s_pos[j]);
            const float2 vj = HR_DYNAMIC_LOAD(&B.s_vel[j]);
            const float4 aj = HR_DYNAMIC_LOAD(&B.s_aux[j]);
            pair_terms<CL>(K, I, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z,
                           CL == 1 ? K.c_av : aj.w, 1.0f, true, A);
        };
        const int base0 = B.cell_start[c - K.ncx - 1], base1 = B.cell_start[c - 1],
                  base2 = B.cell_start[c + K.ncx - 1];
        const int cnt0 = B.cell_start[c - K.ncx + 2] - base0, cnt1 = B.cell_start[c + 2] - base1,
                  cnt2 = B.cell_start[c + K.ncx + 2] - base2;
        bool ok = true;
        if (kChecked)
            ok = row_ok(K, c - K.ncx, base0, base0 + cnt0, K.nf, &B.S->status) &&
                 row_ok(K, c, base1, base1 + cnt1, K.nf, &B.S->status) &&
                 row_ok(K, c + K.ncx, base2, base2 + cnt2, K.nf, &B.S->status);
        const int n0 = (cnt0 + kMaskChunk - 1) / kMaskChunk, n1 = (cnt1 + kMaskChunk - 1) / kMaskChunk,
                  n2 = (cnt2 + kMaskChunk - 1) / kMaskChunk;
#pragma unroll 1
        for (int g = lane; ok && g < n0 + n1 + n2; g += L) {
            const int r = g < n0 ? 0 : (g < n0 + n1 ? 1 : 2);
            const int k = r == 0 ? g : (r == 1 ? g - n0 : g - n0 - n1);
            const int bs = r == 0 ? base0 : (r == 1 ? base1 : base2);
            const int cn = r == 0 ? cnt0 : (r == 1 ? cnt1 : cnt2);
            const int b0 = bs + k * kMaskChunk;
            unsigned m = support_mask(B.s_pos, b0, min(cn - k * kMaskChunk, kMaskChunk), ri, K.s2);
            if (i >= b0 && i < b0 + kMaskChunk) m &= ~(1u << (i - b0));
            while (m) {
                const int j = b0 + __ffs(m) - 1;
                m &= m - 1u;
                fluid_pair(j);
            }
        }
        pass_ghosts<CL>(K, B, ri, c, I, A, P, lane, L);
    }
    A.a.x = lane_group_sum<L>(A.a.x);
    A.a.y = lane_group_sum<L>(A.a.y);
    A.av.x = lane_group_sum<L>(A.av.x);
    A.av.y = lane_group_sum<L>(A.av.y);
    A.X.x = lane_group_sum<L>(A.X.x);
    A.X.y = lane_group_sum<L>(A.X.y);
    A.dr = lane_group_sum<L>(A.dr);
    if (live && lane == 0) pass_close<CL>(K, B, i, vi, ai, rd, dt, prime, A, P);
    pass_block_partials<kPassThreads>(B.part, blockIdx.x, P, &B.S->vmax_bits);
}

// ----------------------------------- a6, a7: probes, accumulators, gate

// Wall-probe value (reading R13: the wall-ghost formula with a = 0, body
// force kept, cutoff applied) at (px, py) over the end-of-step fluid, by one
// warp.  The three stencil rows are flattened into one candidate range so
// the lanes' loads go out together.
template <int CL>
__device__ __forceinline__ float probe_value(const Consts &K, const Bufs &B, float px, float py)
{
    const int lane = threadIdx.x & 31;
    float SW = 0.f, Sp = 0.f, Srx = 0.f, Sry = 0.f;
    auto add = [&](int j) {
        const float2 rj = B.s_pos[j];
        const float d = B.st_rho[j];
        if (!in_support(px, py, rj.x, rj.y, K.s2)) return;
        const float dx = px - rj.x, dy = py - rj.y;
        const float W = kernel_w<CL>(K, sqrtf(fmaf(dx, dx, dy * dy)));
        const float rw = (1.0f + d) * W;
        const float pj = CL == 1 ? mg_p(K, d, B.st_D[j].y) : tait_p(K, d);
        SW += W;
        Sp = fmaf(pj, W, Sp);
        Srx = fmaf(rw, dx, Srx);
        Sry = fmaf(rw, dy, Sry);
    };
    if (!outside_box(K, px, py) && K.sr == 1) {
        const int c = cell_of<1>(K, px, py);
        if (kChecked && !hr_ok(c - K.ncx - 1 >= 0 && c + K.ncx + 2 <= K.ncell, &B.S->status))
            return 0.0f;
        const int a0 = B.cell_start[c - K.ncx - 1], b0 = B.cell_start[c - K.ncx + 2];
        const int a1 = B.cell_start[c - 1], b1 = B.cell_start[c + 2];
        const int a2 = B.cell_start[c + K.ncx - 1], b2 = B.cell_start[c + K.ncx + 2];
        if (kChecked && !(row_ok(K, c - K.ncx, a0, b0, K.nf, &B.S->status) &&
                          row_ok(K, c, a1, b1, K.nf, &B.S->status) &&
                          row_ok(K, c + K.ncx, a2, b2, K.nf, &B.S->status)))
            return 0.0f;
        const int n0 = b0 - a0, n1 = b1 - a1, n = n0 + n1 + (b2 - a2);
        for (int k = lane; k < n; k += 32)
            add(k < n0 ? a0 + k : (k < n0 + n1 ? a1 + (k - n0) : a2 + (k - n0 - n1)));
    } else if (!outside_box(K, px, py)) {
        // 5 x 5 stencil: the rows one after another
        const int c = cell_of<2>(K, px, py);
        for (int dy = -2; dy <= 2; ++dy) {
            const int row = c + dy * K.ncx;
            if (kChecked && !hr_ok(row - 2 >= 0 && row + 3 <= K.ncell, &B.S->status)) continue;
            const int a = B.cell_start[row - 2], b = B.cell_start[row + 3];
            if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
            for (int j = a + lane; j < b; j += 32) add(j);
        }
    }
    SW = warp_sum(SW);
    Sp = warp_sum(Sp);
    Srx = warp_sum(Srx);
    Sry = warp_sum(Sry);
    if (SW > 0.0f) return fmaxf((Sp + K.rho0 * (K.gx * Srx + K.gy * Sry)) / SW, K.p_cav);
    return 0.0f;
}

// Closes the step.  The first nbx - n_probes blocks reduce slices of the
// pass and ghost partials; each of the last n_probes blocks samples one wall
// probe (a7) into probe_now, so the probes and the reduction run side by
// side.  The block that finishes last (atomic ticket) reduces the block
// results, updates the FP64 accumulators and applies the CFL gate (a6); its
// scalar updates are split over three warps.  The sums are compensated FP32
// (two-float) in a fixed tree order, converted to FP64 once at the end.
// SKIP_EMPTY (the persistent batch, where a case's blocks take the virtual
// blocks one after another): a reduction block whose slice holds no partial
// writes its zero sums without the block reduction.  split: the pass ran
// split, and a pass block marked in split_mask has its boundary share in
// part_b, added to its interior share here (the sum pass_block_partials
// forms when one kernel takes the whole block).  With K.split the last block
// also clears the reorder's lists for the next step.
// mode 0: the close at the end of the step, all of the above.  mode 1: the
// deferred close of the last step (Scalars::close_pending; nothing to do
// otherwise), beside the next step's drift: all but the CFL gate, which that
// step's drift and kinematics apply from Scalars::vmax_bits; it writes only
// the scalars it owns (the drift sets status bits meanwhile).  mode 2: as
// mode 1, then the CFL gate as advance_dt, which leaves the scalars as mode 0
// would have (run by the host before it reads the case).
template <int CL, bool SKIP_EMPTY = false>
__device__ __forceinline__ void b_finalize(const Consts &K, const Bufs &B, const int bx, const int nbx, int prime,
                                           int split = 0, int mode = 0)
{
    // (a deferred close returns before its first write when none is pending;
    // the flag is loaded with its first reads, not before them)
    const int pend = mode == 0 ? 1 : __ldcg(&B.S->close_pending);
    constexpr int NW = kFinalizeThreads / 32;
    __shared__ F2 redd[4][NW];
    __shared__ float redv[NW];
    __shared__ int redn[NW];
    __shared__ float probe_p[kMaxProbes];
    __shared__ Scalars S;
    __shared__ int is_last;
    __shared__ F2 tot[4];
    __shared__ float totv;
    __shared__ int totn;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = nbx - K.n_probes;  // reduction blocks
    const bool probe_block = bx >= nb;
    // reduce one (value per thread) set of four sums, max and count over the
    // block; the results land in tot[] (lane 0 of warp 0 writes them)
    auto block_reduce = [&](F2 a0, F2 a1, F2 a2, F2 a3, float v, int np) {
        a0 = f2_warp_sum(a0);
        a1 = f2_warp_sum(a1);
        a2 = f2_warp_sum(a2);
        a3 = f2_warp_sum(a3);
        v = warp_max(v);
        np = warp_sum(np);
        if (lane == 0) {
            redd[0][w] = a0;
            redd[1][w] = a1;
            redd[2][w] = a2;
            redd[3][w] = a3;
            redv[w] = v;
            redn[w] = np;
        }
        __syncthreads();
        if (w == 0) {
            const F2 z{0.f, 0.f};
            F2 b0 = lane < NW ? redd[0][lane] : z, b1 = lane < NW ? redd[1][lane] : z;
            F2 b2 = lane < NW ? redd[2][lane] : z, b3 = lane < NW ? redd[3][lane] : z;
            b0 = f2_warp_sum(b0);
            b1 = f2_warp_sum(b1);
            b2 = f2_warp_sum(b2);
            b3 = f2_warp_sum(b3);
            const float vv = warp_max(lane < NW ? redv[lane] : 0.0f);
            const int nn = warp_sum(lane < NW ? redn[lane] : 0);
            if (lane == 0) {
                tot[0] = b0;
                tot[1] = b1;
                tot[2] = b2;
                tot[3] = b3;
                totv = vv;
                totn = nn;
            }
        }
        __syncthreads();
    };
    if (probe_block) {
        const int q = bx - nb;
        float pv = 0.0f;
        if (w == 0 && !prime) pv = probe_value<CL>(K, B, K.probe_x[q], K.probe_y[q]);
        if (!pend) return;
        if (w == 0 && lane == 0) {
            if (!prime) B.probe_now[q] = pv;
            __threadfence();
            is_last = atomicAdd(B.fin_ticket, 1) == nbx - 1;
        }
    } else if (SKIP_EMPTY && bx * (int)blockDim.x >= max(K.n_pass_blocks, K.n_ghost_blocks)) {
        // a slice past every partial: its sums are zero (what the reduction
        // below would produce), written without the block reduction
        if (threadIdx.x == 0) {
            for (int k = 0; k < 8; ++k) B.fin_part[bx * 8 + k] = 0.0f;
            B.fin_vmax[bx] = 0.0f;
            B.fin_npen[bx] = 0;
            __threadfence();
            is_last = atomicAdd(B.fin_ticket, 1) == nbx - 1;
        }
    } else {
        F2 a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, a3{0.f, 0.f};
        float vmax = 0.0f;
        int npen = 0;
        for (int b = bx * blockDim.x + threadIdx.x; b < K.n_pass_blocks;
             b += nb * blockDim.x) {
            float4 f = B.part.f[b];
            float v = B.part.vmax[b];
            int np = B.part.npen[b];
            if (split) {
                // every load issued before the mark decides (an unlisted
                // block's part_b entry is stale and left unused)
                const unsigned word = B.split_mask[b >> 5];
                const float4 g = B.part_b.f[b];
                const float gv = B.part_b.vmax[b];
                const int gn = B.part_b.npen[b];
                if ((word >> (b & 31)) & 1u) {
                    f = make_float4(f.x + g.x, f.y + g.y, f.z + g.z, f.w + g.w);
                    v = fmaxf(v, gv);
                    np += gn;
                }
            }
            a0 = f2_add(a0, F2{f.x, 0.f});
            a1 = f2_add(a1, F2{f.y, 0.f});
            a2 = f2_add(a2, F2{f.z, 0.f});
            a3 = f2_add(a3, F2{f.w, 0.f});
            vmax = fmaxf(vmax, v);
            npen += np;
        }
        if (mode == 0)   // (the deferred close has no CFL gate to feed)
            for (int b = bx * blockDim.x + threadIdx.x; b < K.n_ghost_blocks;
                 b += nb * blockDim.x)
                vmax = fmaxf(vmax, B.ghost_vmax[b]);
        block_reduce(a0, a1, a2, a3, vmax, npen);
        if (!pend) return;
        if (threadIdx.x == 0) {
            for (int k = 0; k < 4; ++k) {
                B.fin_part[bx * 8 + 2 * k] = tot[k].hi;
                B.fin_part[bx * 8 + 2 * k + 1] = tot[k].lo;
            }
            B.fin_vmax[bx] = totv;
            B.fin_npen[bx] = totn;
            __threadfence();
            is_last = atomicAdd(B.fin_ticket, 1) == nbx - 1;
        }
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    static_assert(sizeof(Scalars) % 8 == 0, "Scalars is copied as doubles");
    for (int k = threadIdx.x; k < (int)(sizeof(Scalars) / 8); k += blockDim.x)
        reinterpret_cast<double *>(&S)[k] = __ldcg(reinterpret_cast<const double *>(B.S) + k);
    {
        const int b = threadIdx.x;
        F2 a[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float v = 0.0f;
        int np = 0;
        if (b < nb) {
            for (int k = 0; k < 4; ++k)
                a[k] = F2{__ldcg(&B.fin_part[b * 8 + 2 * k]), __ldcg(&B.fin_part[b * 8 + 2 * k + 1])};
            v = __ldcg(&B.fin_vmax[b]);
            np = __ldcg(&B.fin_npen[b]);
        }
        block_reduce(a[0], a[1], a[2], a[3], v, np);
    }
    if (threadIdx.x < K.n_probes) probe_p[threadIdx.x] = __ldcg(&B.probe_now[threadIdx.x]);
    __syncthreads();
    // the step's own dt and index, read by every thread before any update
    const double dt = S.dt;
    const long long k = S.step;
    // the four global sums in FP64, one per lane of warp 0 (an FP64
    // operation holds its warp's issue for many cycles on this GPU, so
    // threads 0 and 32 below take them formed)
    __shared__ double sum4[4];
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        const double v = (double)tot[q].hi + (double)tot[q].lo;
        sum4[q] = q < 3 ? K.m2d * v : v;
    }
    __syncthreads();
    if (K.split) {
        // every block has read the marks: clear them and the lists
        for (int k = threadIdx.x; k < (K.n_pass_blocks + 31) / 32; k += blockDim.x) B.split_mask[k] = 0u;
        if (threadIdx.x == 0) {
            B.split_n[0] = 0;
            B.split_n[1] = 0;
        }
    }
    if (threadIdx.x == 0) {
        *B.fin_ticket = 0;
        S.Fdx = sum4[0];
        S.Fdy = sum4[1];
        S.Fwall = sum4[2];
        S.diss_rate = sum4[3];
        if (totn > 0) S.status |= ST_PENETRATION;
        if (!prime) {
            if (k < K.probe_cap) {
                B.probe_t[k] = S.t;
                S.hist_n = k + 1;
            } else if (K.n_probes > 0) {
                S.status |= ST_PROBEFULL;
            }
            S.step = k + 1;
        }
        if (mode == 0) {
            // a6: the CFL gate over fluid and ghost velocities (cfl_dt_f);
            // dt_mode 1 uses the fixed host value
            float dtf;
            double dtn;
            if (K.dt_mode == 1) {
                dtn = K.dt_fixed;
                dtf = (float)dtn;
            } else {
                dtf = cfl_dt_f(K, totv);
                dtn = (double)dtf;
            }
            if (!(dtn > 1e-14)) S.status |= ST_DT;
            S.ratio_f = prime ? 1.0f : __fdiv_rn(dtf, S.dt_f);
            S.done = (S.t_end > 0.0 && S.t >= S.t_end) ? 1 : 0;
            S.dt_prev = prime ? dtn : dt;
            S.dt = dtn;
            S.dt_f = dtf;
        }
    } else if (threadIdx.x == 32) {
        // the FP64 time integrals, beside thread 0 (another warp)
        if (!prime) {
            S.Wb += dt * (sum4[0] * S.vproj);
            S.impulse += dt * sum4[2];
            S.diss += dt * sum4[3];
        }
    } else if (threadIdx.x >= 64 && threadIdx.x < 64 + K.n_probes) {
        // one probe per thread: its history entry and its impulse
        const int q = threadIdx.x - 64;
        if (!prime && k < K.probe_cap) {
            B.probe_hist[k * K.n_probes + q] = probe_p[q];
            S.probe_imp[q] += dt * (double)probe_p[q];
        }
    }
    __syncthreads();
    if (mode == 0) {
        for (int k = threadIdx.x; k < (int)(sizeof(Scalars) / 8); k += blockDim.x)
            reinterpret_cast<double *>(B.S)[k] = reinterpret_cast<const double *>(&S)[k];
        return;
    }
    // the deferred close writes only what it owns
    if (threadIdx.x == 0) {
        Scalars *G = B.S;
        G->Fdx = S.Fdx;
        G->Fdy = S.Fdy;
        G->Fwall = S.Fwall;
        G->diss_rate = S.diss_rate;
        G->Wb = S.Wb;
        G->impulse = S.impulse;
        G->diss = S.diss;
        G->hist_n = S.hist_n;
        G->step = S.step;
        for (int q = 0; q < K.n_probes; ++q) G->probe_imp[q] = S.probe_imp[q];
        const int bits = S.status & (ST_PENETRATION | ST_PROBEFULL);
        if (bits) atomicOr(&G->status, bits);
        G->close_pending = 0;
        if (mode == 2) advance_dt(K, G, G->vmax_bits, G->dt_f, G->dt);
    }
}


// ------------------------------------------------ kernels (one case)

// (A translation unit that only needs the stage bodies defines
// HR_NO_STEP_KERNELS, so the kernels below are defined in one unit only.)
#ifndef HR_NO_STEP_KERNELS

__global__ void __launch_bounds__(256) k_drift_key(Consts K, Bufs B, int prime)
{
    b_drift_key(K, B, blockIdx.x, gridDim.x, prime);
}

// A step graph with the deferred close: its first n_close blocks run the
// last step's close (b_finalize mode 1, nothing if none is pending), the
// rest the drift, which takes this step's dt from the last pass's max |v|
// if that close has not set it.  The close's blocks come first so that they
// start with the drift's first wave; the scan launch that follows (and
// rewrites the cell starts the probes read) waits for both.
static_assert(kFinalizeThreads == 256, "the close's blocks are the drift's size");
template <int CL>
__global__ void __launch_bounds__(256, 8) k_close_drift(Consts K, Bufs B, int n_close, int split)
{
    if ((int)blockIdx.x < n_close) {
        b_finalize<CL>(K, B, blockIdx.x, n_close, 0, split, 1);
        return;
    }
    b_drift_key(K, B, blockIdx.x - n_close, gridDim.x - n_close, 0, 1);
}

__global__ void __launch_bounds__(128) k_kinematics(Consts K, Bufs B, int prime)
{
    b_kinematics(K, B, blockIdx.x, gridDim.x, prime);
}

// kin: one block past the scan tiles advances t and places the disk
// (b_kinematics) on an SM of its own beside the tiles, so the step needs no
// kinematics launch; the reorder that follows sees the disk at t^{n+1}.
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(Consts K, Bufs B, int prime, int kin, int defer)
{
    if (kin && blockIdx.x == gridDim.x - 1) {
        b_kinematics(K, B, 0, 1, prime, defer);
        return;
    }
    b_scan_apply(K, B, blockIdx.x, gridDim.x - kin);
}


template <int CL>
__global__ void __launch_bounds__(256) k_rank_scatter(Consts K, Bufs B, int prime)
{
    b_rank_scatter<CL>(K, B, blockIdx.x, gridDim.x, prime);
}

__global__ void __launch_bounds__(256) k_density(Consts K, Bufs B, int prime)
{
    b_density(K, B, blockIdx.x, gridDim.x, prime);
}

// Blocks past K.n_ghost_blocks (a split-pass step launches them) build the
// split pass's lists.
template <int CL>
__global__ void __launch_bounds__(kGhostWarps * 32) k_ghost(Consts K, Bufs B)
{
    if ((int)blockIdx.x >= K.n_ghost_blocks) {
        b_split_list<kGhostWarps * 32>(K, B, blockIdx.x - K.n_ghost_blocks, gridDim.x - K.n_ghost_blocks);
        return;
    }
    b_ghost<CL>(K, B, blockIdx.x, K.n_ghost_blocks);
}

// 10 resident blocks per SM (48 registers): 40 warps against 36 at the
// compiler's own 54 registers, 3 % faster on the 1.125M workload, no spills
constexpr int kPassMinBlocks = 10;
template <int CL, int R = 1, int MODE = kPassAll>
__global__ void __launch_bounds__(kPassThreads, kPassMinBlocks) k_pass(Consts K, Bufs B, int prime)
{
    b_pass<CL, R, MODE>(K, B, blockIdx.x, gridDim.x, prime);
}

template <int CL>
__global__ void __launch_bounds__(kPassThreads, kPassMinBlocks) k_pass_boundary(Consts K, Bufs B, int prime)
{
    b_pass_boundary<CL>(K, B, prime);
}

__global__ void __launch_bounds__(kPassThreads) k_pass_boundary_sums(Consts K, Bufs B)
{
    b_pass_boundary_sums(K, B);
}

template <int CL, int SV>
__global__ void __launch_bounds__(kPassThreads, kPassMinBlocks) k_pass_staged(Consts K, Bufs B, int prime)
{
    b_pass_staged<CL, SV>(K, B, blockIdx.x, prime);
}

// mode: b_finalize's (0 at the end of the step, 1 deferred to the next
// step's graph, 2 the host's settling of a deferred close)
template <int CL>
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(Consts K, Bufs B, int prime, int split, int mode)
{
    b_finalize<CL>(K, B, blockIdx.x, gridDim.x, prime, split, mode);
}

// --------------------------------------------- kernels (a batch of cases)

// Block b of a batched launch works for case map[b].x as its local block
// map[b].y of map[b].w; the case's constants and buffers are copied to
// shared memory first.  Cases whose run is done (t >= t_end) skip the step.
struct BatchBlock {
    int c, local, nlocal, pad;
};

__device__ __forceinline__ bool batch_enter(const Consts *Ks, const Bufs *Bs, const BatchBlock *map,
                                            Consts &K, Bufs &B, BatchBlock &m)
{
    m = map[blockIdx.x];
    static_assert(sizeof(Consts) % 4 == 0 && sizeof(Bufs) % 8 == 0, "copied as words");
    const int *ks = reinterpret_cast<const int *>(Ks + m.c);
    for (int k = threadIdx.x; k < (int)(sizeof(Consts) / 4); k += blockDim.x)
        reinterpret_cast<int *>(&K)[k] = ks[k];
    const unsigned long long *bs = reinterpret_cast<const unsigned long long *>(Bs + m.c);
    for (int k = threadIdx.x; k < (int)(sizeof(Bufs) / 8); k += blockDim.x)
        reinterpret_cast<unsigned long long *>(&B)[k] = bs[k];
    __syncthreads();
    return !__ldcg(&B.S->done);
}

__global__ void __launch_bounds__(256) kb_drift_key(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_drift_key(K, B, m.local, m.nlocal, 0);
}

__global__ void __launch_bounds__(128) kb_kinematics(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_kinematics(K, B, m.local, m.nlocal, 0);
}

__global__ void __launch_bounds__(kScanThreads) kb_scan_apply(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_scan_apply(K, B, m.local, m.nlocal);
}


template <int CL>
__global__ void __launch_bounds__(256) kb_rank_scatter(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_rank_scatter<CL>(K, B, m.local, m.nlocal, 0);
}

__global__ void __launch_bounds__(256) kb_density(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_density(K, B, m.local, m.nlocal, 0);
}

template <int CL>
__global__ void __launch_bounds__(kGhostWarps * 32) kb_ghost(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_ghost<CL>(K, B, m.local, m.nlocal);
}

// R: the stencil reach of every case on the map (the batch launches one
// map per reach).
template <int CL, int R>
__global__ void __launch_bounds__(kPassThreads) kb_pass(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_pass<CL, R>(K, B, m.local, m.nlocal, 0);
}

template <int CL>
__global__ void __launch_bounds__(kFinalizeThreads) kb_finalize(const Consts *Ks, const Bufs *Bs, const BatchBlock *map)
{
    __shared__ Consts K;
    __shared__ Bufs B;
    __shared__ BatchBlock m;
    if (!batch_enter(Ks, Bs, map, K, B, m)) return;
    b_finalize<CL>(K, B, m.local, m.nlocal, 0);
}

#endif  // HR_NO_STEP_KERNELS

}  // namespace hr
