// hram_adjoint.cuh -- reverse-mode (adjoint) derivatives of the step with
// respect to the artificial-viscosity coefficient alpha, the reference sound
// speed c0 and the disk's deceleration time tau.
//
// The run is swept backwards one step at a time.  Each step's forward record
// (a "slot": its cell order, predicted density and EOS record, ghost state,
// end-of-step state and scalars) is recomputed from a checkpoint of the
// state kept every L steps of the forward run; the adjoint kernels then
// carry lambda, the derivative of the outputs with respect to the state, from
// the end of the step to its start.  Two adjoints are carried at once
// (component 0: the peak probe-0 pressure max_n p(t^n), seeded at the
// forward argmax step; component 1: the wall impulse sum_n dt^n F_wall^{n+1}),
// so one sweep gives the whole 2 x 3 Jacobian.  Every decision of the forward
// step (neighbour sets, cell order, the density band, the cavitation cutoff,
// the artificial-viscosity switch, wall reflections, frozen particles) is held
// as the forward run took it, so the derivative is that of the discrete run,
// the same one the tangent-linear kernels give.
//
// The step's maps and their transposes (closure 0, fixed dt, motions 0-2):
//   drift       vh = v + dt/2 a,  r' = r + dt (vh + eps X),  reflection
//   predictor   d~ = band(d + dt (D + ratio (D - E))),  rec = (d~, p~, p~/rho~^2, -alpha h c~)
//   kinematics  t' = t + dt,  x_c, v_w, a_w at t',  disk ghosts r_g = x_c + R (cos, sin)
//   ghosts      Shepard sums over fluid j, p_g, d_g = p_g / (rho0 c0^2), v_g = 2 v_w - <v>
//   pass        A_i = sum_j f_ij, Dr_i = sum_j F vr, X_i = sum_j wx v_ij
//   epilogue    a' = m A + g, Dd = m/rho0 Dr, d' = band(d + dt Dd), v' = vh + dt/2 a'
//   outputs     J += dt m^2 sum_{i, side-wall g} -f_ig . n_g,  P = probe-0 value at the argmax step
// The pair sums are transposed as gathers: with f_ki = -f_ik, Dr symmetric
// and X antisymmetric, particle k's own inputs receive
//   sum_i d/d(in_k) [ (lA_k - lA_i) . f_ki + (lDr_k + lDr_i) Dr_ki + (lX_k - lX_i) . X_ki ],
// so no particle writes to another's adjoint.  The ghost sums are transposed
// the same way: each ghost first forms the adjoints of its six Shepard sums,
// then each fluid particle gathers its share from the ghosts in its support.
#pragma once
#include "hram_device.cuh"
#include "hram_tangent.cuh"

namespace hr {

constexpr int kOut = 2;          // adjoint components: 0 peak probe-0 pressure, 1 wall impulse
constexpr int kAThreads = 128;   // per-particle adjoint kernels
constexpr int kAGhostWarps = 4;  // ghost adjoint: one warp per ghost
// resident ka_pass blocks per SM: 6 (80 registers, no spills) measured best
// against 7 and 8 (spills) and against two neighbours per loop iteration at
// 4 and 5 (109 and 96 registers): 0.823 against 0.825-0.980 ms per step
constexpr int kAPassMinBlocks = 6;

// One step's forward record.  s_* and st_* are in the step's cell order;
// cell_start, gd_pos, g_* belong to the step; S is the scalars after the step.
struct Slot {
    float2 *s_pos, *s_vel;
    float4 *s_aux;
    float2 *s_rd;
    int *s_id;
    float2 *st_vel;
    float *st_rho;
    float2 *st_a, *st_D, *st_X;
    int *perm_dst, *cell_start;
    float2 *gd_pos, *g_vel;
    float4 *g_aux;
    Scalars *S;
    double *kin;   // dx_c, dv_w, da_w by t, then by ln tau, at the step's time (reverse mode)
};

// Adjoints of the state a step hands to the next: r, v, a, X, d, D (the
// density rate) and E (the previous rate), [i * kOut + c].
struct LState {
    float2 *r, *v, *a, *X;
    float *d, *D, *E;
};

enum {
    ASC_ALPHA = 0,   // d/d ln alpha, both components      [kOut]
    ASC_C0 = 2,      // d/d ln c0 (direct: EOS, sound speed) [kOut]
    ASC_TAU = 4,     // d/d ln tau                           [kOut]
    ASC_DT = 6,      // d/d dt (every step's dt; dt is C h / (c0 + v0))  [kOut]
    ASC_TBAR = 8,    // running adjoint of the time t       [kOut]
    ASC_N = 16
};

struct ABufs {
    LState cur, prv;         // end-of-step adjoints: this step's order / the previous step's
    float4 *wA, *wX;         // pair weights lambda_A, lambda_X of the pass sums, both
                             // components in one vector {x0, y0, x1, y1} per particle
    float2 *wDr;             // pair weights of the continuity sum {c0, c1}
    float2 *lpos, *lvh;      // adjoints of the pass inputs r', vh
    float4 *lrec;            // adjoints of the EOS record {d~ (density), P~, C~, p~}
    float2 *lrd;             // adjoints of {d, D} carried through the sort
    float4 *gS1;             // ghost Shepard-sum adjoints {W, p, rx, ry}  [g * kOut + c]
    float2 *gS2;             // {vx, vy}
    float4 *gpar;            // ghost partials {alpha, c0, v_w, a_w}
    float2 *grg;             // disk ghost position adjoints
    float *ep_part;          // per epilogue block: dt partial [kOut]
    float4 *bk_part;         // per back block: {alpha, c0, dt, 0} [kOut]
    float2 *sums;            // ka_reduce's block sums (two-float) [kAReduceBlocks x kASums]
    double *sc;              // ASC_* accumulators
    int *status;             // the case's status word (bounds-checked build)
    double *cpart;           // ka_close's warp sums [kAReduceBlocks / 32 x kASums]
    int *ctick;              // ka_close's ticket (0 between launches)
};

// ---------------------------------------------------------------- helpers

// Tait pressure without the cutoff, and its slope dp/dd = gamma B (1 + d)^(gamma - 1).
__device__ __forceinline__ float tait_raw(const Consts &K, float d)
{
    if (K.gamma7) {
        float poly = fmaf(d, 1.0f, 7.0f);
        poly = fmaf(d, poly, 21.0f);
        poly = fmaf(d, poly, 35.0f);
        poly = fmaf(d, poly, 35.0f);
        poly = fmaf(d, poly, 21.0f);
        poly = fmaf(d, poly, 7.0f);
        return K.B * d * poly;
    }
    return K.B * expm1f(K.gamma * log1pf(d));
}

__device__ __forceinline__ float tait_slope(const Consts &K, float d)
{
    const float x = 1.0f + d;
    if (K.gamma7) {
        const float x2 = x * x;
        return 7.0f * K.B * x2 * x2 * x2;
    }
    return K.gamma * K.B * __powf(x, K.gamma - 1.0f);
}

// Forward intermediates of one pair as pair_terms forms them, side I = the
// particle whose sums receive the pair (fluid), side J = its neighbour, and
// the local partial derivatives the reverse sweep needs (formed once, shared
// by the adjoint components).
struct PairFwd {
    float dx, dy, vx, vy, vr, F, Q, lam, wx;
    float kFr2, kLamR2, kLamInv, kC, kVr, kInv, kWxT, kWxR, kWxS, kInvR2, kInvS, kFt, kTr, kRr2;
};

__device__ __forceinline__ void pair_fwd(const Consts &K, float2 ri, float2 vi, float rhoi, float Pi,
                                         float Ci, float2 rj, float2 vj, float rhoj, float Pj, float Cj,
                                         float mj, bool xsph, PairFwd &q)
{
    q.dx = ri.x - rj.x;
    q.dy = ri.y - rj.y;
    const float r2 = fmaf(q.dx, q.dx, q.dy * q.dy);
    const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
    const float r = r2 * rinv;
    const float t0 = fmaf(-r, K.half_inv_h, 1.0f);
    const float t = fmaxf(t0, 0.0f);
    const float t2 = t * t, t3 = t2 * t;
    const float mjFc = mj * K.Fc;
    q.F = mjFc * t3;
    q.vx = vi.x - vj.x;
    q.vy = vi.y - vj.y;
    q.vr = fmaf(q.vx, q.dx, q.vy * q.dy);
    const float e = r2 + K.eh2;
    const float S = rhoi + rhoj;
    const float ie = __fdividef(1.0f, e), iS = __fdividef(1.0f, S);
    const float inv = ie * iS;
    const float Csum = Ci + Cj;
    const float mvr = fminf(q.vr, 0.0f);
    q.Q = Pi + Pj + Csum * mvr * inv;
    q.lam = K.nu4 * q.F * r2 * inv;
    // the partials of the reverse sweep
    q.kFr2 = K.nu4 * r2 * inv;          // d lam / dF
    q.kLamR2 = K.nu4 * q.F * inv;       // d lam / d r2 (at fixed inv)
    q.kLamInv = K.nu4 * q.F * r2;       // d lam / d inv
    q.kC = mvr * inv;                   // d Pi / d Csum
    q.kVr = q.vr < 0.0f ? Csum * inv : 0.0f;   // d Pi / d vr (the switch)
    q.kInv = Csum * mvr;                // d Pi / d inv
    if (xsph) {
        const float poly = fmaf(r, K.two_inv_h, 1.0f);
        q.wx = K.m2Wc * t3 * t * poly * iS;
        q.kWxT = K.m2Wc * 4.0f * t3 * poly * iS;
        q.kWxR = K.m2Wc * t3 * t * K.two_inv_h * iS;
        q.kWxS = -q.wx * iS;
    } else {
        q.wx = q.kWxT = q.kWxR = q.kWxS = 0.0f;
    }
    q.kInvR2 = -inv * ie;               // d inv / d r2
    q.kInvS = -inv * iS;                // d inv / d S
    q.kFt = 3.0f * mjFc * t2;           // dF / dt
    q.kTr = t0 > 0.0f ? -K.half_inv_h : 0.0f;   // dt / dr
    q.kRr2 = r2 > 0.0f ? 0.5f * rinv : 0.0f;    // dr / d r2
}

// Adjoint of one pair for the weights (wA on the acceleration sum, wDr on the
// continuity sum, wX on the XSPH sum): the derivatives of
//   wA . f + wDr F vr + wX . (wx v)
// with respect to d = r_I - r_J, v = v_I - v_J, S = rho_I + rho_J, the
// pressure sum Q = P_I + P_J + Pi_ij (its P part) and Csum = C_I + C_J.
struct PairAdj {
    float gdx, gdy, gvx, gvy, gS, gQ, gC;
};

__device__ __forceinline__ PairAdj pair_rev(const PairFwd &q, float wAx, float wAy, float wDr,
                                            float wXx, float wXy)
{
    const float PF = q.Q * q.F;
    // f = -PF d + lam v,  Dr = F vr,  X = wx v
    const float gPF = -fmaf(wAx, q.dx, wAy * q.dy);
    const float glam = fmaf(wAx, q.vx, wAy * q.vy);
    const float gwx = fmaf(wXx, q.vx, wXy * q.vy);
    float gdx = -PF * wAx, gdy = -PF * wAy;
    float gvx = fmaf(q.lam, wAx, q.wx * wXx), gvy = fmaf(q.lam, wAy, q.wx * wXy);
    // PF = Q F; lam = nu4 F r2 inv
    const float gQ = gPF * q.F;
    float gF = fmaf(wDr, q.vr, fmaf(gPF, q.Q, glam * q.kFr2));
    float gr2 = glam * q.kLamR2;
    float ginv = fmaf(gQ, q.kInv, glam * q.kLamInv);
    // Pi_ij = Csum min(vr, 0) inv inside Q; Dr = F vr
    const float gC = gQ * q.kC;
    const float gvr = fmaf(gQ, q.kVr, wDr * q.F);
    // wx = m2Wc t^4 (1 + 2 r / h) / S; inv = 1 / (e S)
    float gt = gwx * q.kWxT;
    float gr = gwx * q.kWxR;
    const float gS = fmaf(gwx, q.kWxS, ginv * q.kInvS);
    gr2 = fmaf(ginv, q.kInvR2, gr2);
    // F = mj Fc t^3, t = max(1 - r / 2h, 0), r = sqrt(r2)
    gt = fmaf(gF, q.kFt, gt);
    gr = fmaf(gt, q.kTr, gr);
    gr2 = fmaf(gr, q.kRr2, gr2);
    // vr = v . d,  r2 = d . d
    gvx = fmaf(gvr, q.dx, gvx);
    gvy = fmaf(gvr, q.dy, gvy);
    gdx = fmaf(gvr, q.vx, fmaf(2.0f * gr2, q.dx, gdx));
    gdy = fmaf(gvr, q.vy, fmaf(2.0f * gr2, q.dy, gdy));
    return PairAdj{gdx, gdy, gvx, gvy, gS, gQ, gC};
}

// Wendland C2 value and gradient factor (grad W = Fw d) at distance r.
__device__ __forceinline__ void w_and_f(const Consts &K, float r, float &W, float &Fw)
{
    const float t = fmaxf(fmaf(-r, K.half_inv_h, 1.0f), 0.0f);
    const float t2 = t * t;
    W = K.Wc * t2 * t2 * fmaf(r, K.two_inv_h, 1.0f);
    Fw = K.Fc * t2 * t;
}

template <typename T>
__device__ __forceinline__ T lane_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// -------------------------------------------------------------- kernels

// Seed of the peak: the probe-0 value of the argmax step, p = max((Sp +
// rho0 g . Sr) / SW, p_cav) over the end-of-step fluid (r', d'); its
// derivative is added to component 0 of the end-of-step adjoints and of the
// c0 accumulator (the Tait pressure of each neighbour depends on c0).  One
// warp; each neighbour is written by one lane.
__global__ void ka_probe(Consts K, Bufs B, ABufs A, long long peak_row)
{
    // the record's scalars count the step it closes: seed only the peak's step
    if (B.S->step - 1 != peak_row) return;
    const int lane = threadIdx.x & 31;
    const float px = K.probe_x[0], py = K.probe_y[0];
    if (outside_box(K, px, py)) return;
    const int c = cell_of(K, px, py);
    float SW = 0.f, Sp = 0.f, Srx = 0.f, Sry = 0.f;
    for (int dy = -1; dy <= 1; ++dy) {
        const int row = c + dy * K.ncx;
        if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, A.status)) continue;
        const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
        if (kChecked && !row_ok(K, row, a, b, K.nf, A.status)) continue;
        for (int j = a + lane; j < b; j += 32) {
            const float2 rj = B.s_pos[j];
            if (!in_support(px, py, rj.x, rj.y, K.s2)) continue;
            const float d = B.st_rho[j];
            const float dx = px - rj.x, dy2 = py - rj.y;
            const float W = kernel_w<0>(K, sqrtf(fmaf(dx, dx, dy2 * dy2)));
            const float rw = (1.0f + d) * W;
            SW += W;
            Sp = fmaf(tait_p(K, d), W, Sp);
            Srx = fmaf(rw, dx, Srx);
            Sry = fmaf(rw, dy2, Sry);
        }
    }
    SW = lane_sum(SW);
    Sp = lane_sum(Sp);
    Srx = lane_sum(Srx);
    Sry = lane_sum(Sry);
    if (!(SW > 0.0f)) return;
    const float inv = 1.0f / SW;
    const float pv = (Sp + K.rho0 * (K.gx * Srx + K.gy * Sry)) * inv;
    if (!(pv > K.p_cav)) return;   // the cutoff holds the value constant
    const float bW = -pv * inv, bp = inv, brx = K.rho0 * K.gx * inv, bry = K.rho0 * K.gy * inv;
    float c0bar = 0.0f;
    for (int dy = -1; dy <= 1; ++dy) {
        const int row = c + dy * K.ncx;
        if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, A.status)) continue;
        const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
        if (kChecked && !row_ok(K, row, a, b, K.nf, A.status)) continue;
        for (int j = a + lane; j < b; j += 32) {
            const float2 rj = B.s_pos[j];
            if (!in_support(px, py, rj.x, rj.y, K.s2)) continue;
            const float d = B.st_rho[j];
            const float dx = px - rj.x, dy2 = py - rj.y;
            float W, Fw;
            w_and_f(K, sqrtf(fmaf(dx, dx, dy2 * dy2)), W, Fw);
            const float praw = tait_raw(K, d);
            const bool cut = !(praw > K.p_cav);
            const float pj = cut ? K.p_cav : praw;
            const float sr = fmaf(brx, dx, bry * dy2);
            const float om = bW + bp * pj + sr * (1.0f + d);
            float dbar = sr * W;
            if (!cut) {
                dbar = fmaf(bp * W, tait_slope(K, d), dbar);
                c0bar = fmaf(bp * W, 2.0f * praw, c0bar);
            }
            // d = p - r_j: the position's adjoint is minus the d-derivative
            const float gx = fmaf(om * Fw, dx, (1.0f + d) * W * brx);
            const float gy = fmaf(om * Fw, dy2, (1.0f + d) * W * bry);
            A.cur.d[j * kOut] += dbar;
            float2 lr = A.cur.r[j * kOut];
            lr.x -= gx;
            lr.y -= gy;
            A.cur.r[j * kOut] = lr;
        }
    }
    c0bar = lane_sum(c0bar);
    if (lane == 0) A.sc[ASC_C0] += (double)c0bar;
}

// Epilogue: the end-of-step adjoints of particle i become the weights of its
// pass sums and the adjoints of its half-step velocity and carried density.
__global__ void __launch_bounds__(kAThreads) ka_epilogue(Consts K, Bufs B, ABufs A, int prime)
{
    __shared__ float red[kAThreads / 32][kOut];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float dtp[kOut] = {0.0f, 0.0f};
    if (i < K.nf) {
        const float dt = prime ? 0.0f : B.S->dt_f;
        const float2 ri = B.s_pos[i];
        const bool frozen = outside_box(K, ri.x, ri.y);
        const float dn = B.st_rho[i];
        const float2 a1 = B.st_a[i];
        const float Dd = B.st_D[i].x;
        const bool clamp = dn <= K.d_lo || dn >= K.d_hi;
        float2 wAc[kOut], wXc[kOut];
        float wDc[kOut];
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const int q = i * kOut + c;
            const float2 lv = A.cur.v[q];
            const float ld = A.cur.d[q];
            float2 wA = make_float2(0.f, 0.f), wX = make_float2(0.f, 0.f);
            float wDr = 0.0f, lrdx = 0.0f, lrdy = 0.0f;
            if (frozen) {
                lrdx = ld;   // d' = d
            } else {
                const float2 la = A.cur.a[q], lX = A.cur.X[q];
                const float lD = A.cur.D[q], lE = A.cur.E[q];
                // v' = vh + dt/2 a'
                const float lax = fmaf(0.5f * dt, lv.x, la.x), lay = fmaf(0.5f * dt, lv.y, la.y);
                dtp[c] += 0.5f * fmaf(a1.x, lv.x, a1.y * lv.y);
                // D' = Dd, d' = band(d + dt Dd)
                float lDd = lD;
                if (!clamp) {
                    lrdx = ld;
                    lDd = fmaf(dt, ld, lDd);
                    dtp[c] = fmaf(Dd, ld, dtp[c]);
                }
                // E' = D (after the priming pass: E' = Dd)
                if (prime) lDd += lE;
                else lrdy = lE;
                wA = make_float2(K.m * lax, K.m * lay);
                wDr = K.m_over_rho0 * lDd;
                wX = make_float2(K.m * lX.x, K.m * lX.y);
            }
            wAc[c] = wA;
            wXc[c] = wX;
            wDc[c] = wDr;
            A.lvh[q] = lv;
            A.lrd[q] = make_float2(lrdx, lrdy);
        }
        A.wA[i] = make_float4(wAc[0].x, wAc[0].y, wAc[1].x, wAc[1].y);
        A.wX[i] = make_float4(wXc[0].x, wXc[0].y, wXc[1].x, wXc[1].y);
        A.wDr[i] = make_float2(wDc[0], wDc[1]);
    }
    // the priming pass runs with the constant dt = 0, not with the case's dt
    if (prime) dtp[0] = dtp[1] = 0.0f;
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        const float s = lane_sum(dtp[c]);
        if (lane == 0) red[w][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < kOut) {
        float s = 0.0f;
        for (int k = 0; k < kAThreads / 32; ++k) s += red[k][threadIdx.x];
        A.ep_part[blockIdx.x * kOut + threadIdx.x] = s;
    }
}

// Ghosts: one warp per ghost.  Loop 1 over its fluid neighbours forms the
// Shepard sums again and gathers the ghost-side adjoint of every pass pair
// (fluid j, ghost g) with the weights of j (plus, for side-wall ghosts, the
// wall impulse's own weight -dt m^2 n on the pair force, component 1).  The
// ghost operator is then transposed to the adjoints of the six Shepard sums
// and of the wall's velocity and acceleration; loop 2 (disk ghosts) adds the
// position adjoint that flows through the sums.
__global__ void __launch_bounds__(kAGhostWarps * 32) ka_ghost(Consts K, Bufs B, ABufs A, int prime)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * kAGhostWarps + w;
    if (g >= K.nw + K.ng) return;
    const bool disk = g >= K.nw;
    const float2 rg = disk ? B.gd_pos[g - K.nw] : B.gw_pos[g];
    float4 S1[kOut], par[kOut];
    float2 S2[kOut], gr[kOut];
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        S1[c] = par[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        S2[c] = gr[c] = make_float2(0.f, 0.f);
    }
    if (!outside_box(K, rg.x, rg.y)) {
        const float aw = disk ? B.S->aproj_f : 0.0f;
        const float4 ag = B.g_aux[g];
        const float2 vg = B.g_vel[g];
        const float rhog = fmaf(K.rho0, ag.x, K.rho0);
        const float mjg = disk ? K.disk_over_m : K.wall_over_m;
        const bool side = !disk && B.gw_kind[g] == KIND_SIDE;
        const float2 nrm = side ? B.gw_nrm[g] : make_float2(0.f, 0.f);
        const float jw = prime ? 0.0f : -B.S->dt_f * K.m * K.m;
        float SW = 0.f, Sp = 0.f, Srx = 0.f, Sry = 0.f, Svx = 0.f, Svy = 0.f;
        float gd[kOut], gP[kOut], gC[kOut];
        float2 gv[kOut];
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            gd[c] = gP[c] = gC[c] = 0.0f;
            gv[c] = make_float2(0.f, 0.f);
        }
        const int cc = cell_of(K, rg.x, rg.y);
        for (int dy = -1; dy <= 1; ++dy) {
            const int row = cc + dy * K.ncx;
            if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, A.status)) continue;
            const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
            if (kChecked && !row_ok(K, row, a, b, K.nf, A.status)) continue;
            for (int j = a + lane; j < b; j += 32) {
                const float2 rj = B.s_pos[j];
                if (!in_support(rg.x, rg.y, rj.x, rj.y, K.s2)) continue;
                const float4 aux = B.s_aux[j];
                const float2 vj = B.s_vel[j];
                const float dx = rg.x - rj.x, dy2 = rg.y - rj.y;
                const float W = kernel_w<0>(K, sqrtf(fmaf(dx, dx, dy2 * dy2)));
                const float rw = (1.0f + aux.x) * W;
                SW += W;
                Sp = fmaf(aux.y, W, Sp);
                Srx = fmaf(rw, dx, Srx);
                Sry = fmaf(rw, dy2, Sry);
                Svx = fmaf(vj.x, W, Svx);
                Svy = fmaf(vj.y, W, Svy);
                PairFwd q;
                pair_fwd(K, rj, vj, fmaf(K.rho0, aux.x, K.rho0), aux.z, aux.w, rg, vg, rhog, ag.z,
                         ag.w, mjg, false, q);
                const float4 wa4 = A.wA[j];
                const float2 wd2 = A.wDr[j];
#pragma unroll
                for (int c = 0; c < kOut; ++c) {
                    float2 wa = c == 0 ? make_float2(wa4.x, wa4.y) : make_float2(wa4.z, wa4.w);
                    if (c == 1 && side) {
                        wa.x = fmaf(jw, nrm.x, wa.x);
                        wa.y = fmaf(jw, nrm.y, wa.y);
                    }
                    const PairAdj p = pair_rev(q, wa.x, wa.y, c == 0 ? wd2.x : wd2.y, 0.f, 0.f);
                    gd[c] = fmaf(K.rho0, p.gS, gd[c]);
                    gP[c] += p.gQ;
                    gC[c] += p.gC;
                    gv[c].x -= p.gvx;
                    gv[c].y -= p.gvy;
                    gr[c].x -= p.gdx;
                    gr[c].y -= p.gdy;
                }
            }
        }
        SW = lane_sum(SW);
        Sp = lane_sum(Sp);
        Srx = lane_sum(Srx);
        Sry = lane_sum(Sry);
        Svx = lane_sum(Svx);
        Svy = lane_sum(Svy);
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            gd[c] = lane_sum(gd[c]);
            gP[c] = lane_sum(gP[c]);
            gC[c] = lane_sum(gC[c]);
            gv[c].x = lane_sum(gv[c].x);
            gv[c].y = lane_sum(gv[c].y);
            gr[c].x = lane_sum(gr[c].x);
            gr[c].y = lane_sum(gr[c].y);
        }
        if (SW > 0.0f) {
            const float inv = 1.0f / SW;
            const float bx = K.gx - aw, by = K.gy;
            const float praw = (Sp + K.rho0 * (bx * Srx + by * Sry)) * inv;
            const bool cut = !(praw > K.p_cav);
            const float pg = cut ? K.p_cav : praw;
            const float dg = pg * K.inv_rho0c02;
            const float x = 1.0f + dg;
            const float rho = K.rho0 * x;
            const float Cg = ag.w;   // -alpha h c0 (1 + d_g)^((gamma - 1) / 2)
#pragma unroll
            for (int c = 0; c < kOut; ++c) {
                float dbar = gd[c];
                // C_g
                dbar = fmaf(gC[c], Cg * K.half_gm1 / x, dbar);
                par[c].x = gC[c] * Cg;
                par[c].y = gC[c] * Cg;
                // P_g = p_g / rho_g^2
                float pbar = gP[c] / (rho * rho);
                dbar = fmaf(gP[c], -2.0f * pg * K.rho0 / (rho * rho * rho), dbar);
                // d_g = p_g / (rho0 c0^2)
                pbar = fmaf(dbar, K.inv_rho0c02, pbar);
                par[c].y = fmaf(dbar, -2.0f * dg, par[c].y);
                if (!cut) {
                    S1[c].y = pbar * inv;
                    S1[c].z = pbar * K.rho0 * bx * inv;
                    S1[c].w = pbar * K.rho0 * by * inv;
                    S1[c].x = -pbar * praw * inv;
                    par[c].w = -pbar * K.rho0 * Srx * inv;   // b_x = g_x - a_w
                }
                // v_g = (2 v_w - Svx / SW, -Svy / SW)
                par[c].z = 2.0f * gv[c].x;
                S2[c] = make_float2(-gv[c].x * inv, -gv[c].y * inv);
                S1[c].x = fmaf(fmaf(gv[c].x, Svx, gv[c].y * Svy), inv * inv, S1[c].x);
            }
            if (disk) {
                // position adjoint through the Shepard sums (d = r_g - r_j)
                float2 hs[kOut];
#pragma unroll
                for (int c = 0; c < kOut; ++c) hs[c] = make_float2(0.f, 0.f);
                for (int dy = -1; dy <= 1; ++dy) {
                    const int row = cc + dy * K.ncx;
                    if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, A.status)) continue;
                    const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
                    if (kChecked && !row_ok(K, row, a, b, K.nf, A.status)) continue;
                    for (int j = a + lane; j < b; j += 32) {
                        const float2 rj = B.s_pos[j];
                        if (!in_support(rg.x, rg.y, rj.x, rj.y, K.s2)) continue;
                        const float4 aux = B.s_aux[j];
                        const float2 vj = B.s_vel[j];
                        const float dx = rg.x - rj.x, dy2 = rg.y - rj.y;
                        float W, Fw;
                        w_and_f(K, sqrtf(fmaf(dx, dx, dy2 * dy2)), W, Fw);
#pragma unroll
                        for (int c = 0; c < kOut; ++c) {
                            const float sr = fmaf(S1[c].z, dx, S1[c].w * dy2);
                            const float om = S1[c].x + S1[c].y * aux.y + sr * (1.0f + aux.x) +
                                             fmaf(S2[c].x, vj.x, S2[c].y * vj.y);
                            hs[c].x += fmaf(om * Fw, dx, (1.0f + aux.x) * W * S1[c].z);
                            hs[c].y += fmaf(om * Fw, dy2, (1.0f + aux.x) * W * S1[c].w);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < kOut; ++c) {
                    gr[c].x += lane_sum(hs[c].x);
                    gr[c].y += lane_sum(hs[c].y);
                }
            }
        } else {
            // no fluid in support: v_g = v_w, rec = (0, 0, 0, -alpha h c0)
#pragma unroll
            for (int c = 0; c < kOut; ++c) {
                par[c].z = gv[c].x;
                par[c].x = par[c].y = gC[c] * ag.w;
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const int q = g * kOut + c;
            A.gS1[q] = S1[c];
            A.gS2[q] = S2[c];
            A.gpar[q] = par[c];
            A.grg[q] = disk ? gr[c] : make_float2(0.f, 0.f);
        }
    }
}

// The ghost Shepard sums' share of a fluid particle k (d = r_g - r_k).
__device__ __forceinline__ void shepard_share(const Consts &K, const ABufs &A, int g, float2 rg,
                                              float2 rk, float2 vk, float4 ak, float2 *gpos,
                                              float2 *gvh, float4 *grec)
{
    const float dx = rg.x - rk.x, dy = rg.y - rk.y;
    float W, Fw;
    w_and_f(K, sqrtf(fmaf(dx, dx, dy * dy)), W, Fw);
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        const float4 s1 = A.gS1[g * kOut + c];
        const float2 s2 = A.gS2[g * kOut + c];
        const float sr = fmaf(s1.z, dx, s1.w * dy);
        const float om = s1.x + s1.y * ak.y + sr * (1.0f + ak.x) + fmaf(s2.x, vk.x, s2.y * vk.y);
        gpos[c].x -= fmaf(om * Fw, dx, (1.0f + ak.x) * W * s1.z);
        gpos[c].y -= fmaf(om * Fw, dy, (1.0f + ak.x) * W * s1.w);
        grec[c].x = fmaf(sr, W, grec[c].x);
        grec[c].w = fmaf(s1.y, W, grec[c].w);
        gvh[c].x = fmaf(s2.x, W, gvh[c].x);
        gvh[c].y = fmaf(s2.y, W, gvh[c].y);
    }
}

// Pass adjoint of fluid particle k (this step's order): its side of every
// fluid pair (both particles' weights), of every ghost pair (its own
// weights), and its share of the ghosts' Shepard sums.  The totals: the
// adjoint of r' (end-of-step position plus pass input), of vh and of the
// EOS record.
__global__ void __launch_bounds__(kAThreads, kAPassMinBlocks) ka_pass(Consts K, Bufs B, ABufs A, int prime)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K.nf) return;
    const float2 rk = B.s_pos[k];
    float2 gpos[kOut], gvh[kOut];
    float4 grec[kOut];
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        gpos[c] = gvh[c] = make_float2(0.f, 0.f);
        grec[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!outside_box(K, rk.x, rk.y)) {
        const float2 vk = B.s_vel[k];
        const float4 ak = B.s_aux[k];
        const float rhok = fmaf(K.rho0, ak.x, K.rho0);
        const float4 wAk = A.wA[k], wXk = A.wX[k];
        const float2 wDk = A.wDr[k];
        const int cc = cell_of(K, rk.x, rk.y);
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            const int row = cc + dy * K.ncx;
            if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, A.status)) continue;
            const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
            if (kChecked && !row_ok(K, row, a, b, K.nf, A.status)) continue;
#pragma unroll 1
            for (int base = a; base < b; base += 32) {
                unsigned m = support_mask(B.s_pos, base, min(32, b - base), rk, K.s2);
                if (k >= base && k < base + 32) m &= ~(1u << (k - base));
                // the pair adjoint of neighbour j (its data loaded by the caller)
                auto fluid_adj = [&](float2 rj, float2 vj, float4 aj, float4 wAj, float4 wXj,
                                     float2 wDj) {
                    PairFwd q;
                    pair_fwd(K, rk, vk, rhok, ak.z, ak.w, rj, vj, fmaf(K.rho0, aj.x, K.rho0), aj.z,
                             aj.w, 1.0f, true, q);
#pragma unroll
                    for (int c = 0; c < kOut; ++c) {
                        const PairAdj p =
                            c == 0 ? pair_rev(q, wAk.x - wAj.x, wAk.y - wAj.y, wDk.x + wDj.x,
                                              wXk.x - wXj.x, wXk.y - wXj.y)
                                   : pair_rev(q, wAk.z - wAj.z, wAk.w - wAj.w, wDk.y + wDj.y,
                                              wXk.z - wXj.z, wXk.w - wXj.w);
                        gpos[c].x += p.gdx;
                        gpos[c].y += p.gdy;
                        gvh[c].x += p.gvx;
                        gvh[c].y += p.gvy;
                        grec[c].x = fmaf(K.rho0, p.gS, grec[c].x);
                        grec[c].y += p.gQ;
                        grec[c].z += p.gC;
                    }
                };
#pragma unroll 1
                while (m) {
                    const int j = base + __ffs(m) - 1;
                    m &= m - 1u;
                    fluid_adj(B.s_pos[j], B.s_vel[j], B.s_aux[j], A.wA[j], A.wX[j], A.wDr[j]);
                }
            }
        }
        const float jw = prime ? 0.0f : -B.S->dt_f * K.m * K.m;
        auto ghost_pair = [&](int g, float2 rg, float mj, bool side) {
            const float4 ag = B.g_aux[g];
            const float2 vg = B.g_vel[g];
            PairFwd q;
            pair_fwd(K, rk, vk, rhok, ak.z, ak.w, rg, vg, fmaf(K.rho0, ag.x, K.rho0), ag.z, ag.w, mj,
                     false, q);
            const float2 nrm = side ? B.gw_nrm[g] : make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < kOut; ++c) {
                float2 wa = c == 0 ? make_float2(wAk.x, wAk.y) : make_float2(wAk.z, wAk.w);
                if (c == 1 && side) {
                    wa.x = fmaf(jw, nrm.x, wa.x);
                    wa.y = fmaf(jw, nrm.y, wa.y);
                }
                const PairAdj p = pair_rev(q, wa.x, wa.y, c == 0 ? wDk.x : wDk.y, 0.f, 0.f);
                gpos[c].x += p.gdx;
                gpos[c].y += p.gdy;
                gvh[c].x += p.gvx;
                gvh[c].y += p.gvy;
                grec[c].x = fmaf(K.rho0, p.gS, grec[c].x);
                grec[c].y += p.gQ;
                grec[c].z += p.gC;
            }
            shepard_share(K, A, g, rg, rk, vk, ak, gpos, gvh, grec);
        };
        if (K.nw > 0)
            for_fluid_candidates(K, B.wall_start, cc, K.nw, A.status, [&](int g) {
                const float2 rg = B.gw_pos[g];
                if (!in_support(rk.x, rk.y, rg.x, rg.y, K.s2)) return;
                ghost_pair(g, rg, K.wall_over_m, B.gw_kind[g] == KIND_SIDE);
            });
        if (K.ng > 0) {
            const float xc = B.S->xc_f, yc = B.S->yc_f;
            if (near_disk(K, rk.x, rk.y, xc, yc))
                for_disk_arc(K, disk_arc(K, rk.x, rk.y, xc, yc), A.status, [&](int kk) {
                    const float2 rg = B.gd_pos[kk];
                    if (outside_box(K, rg.x, rg.y)) return;
                    if (!in_support(rk.x, rk.y, rg.x, rg.y, K.s2)) return;
                    ghost_pair(K.nw + kk, rg, K.disk_over_m, false);
                });
        }
    }
#pragma unroll
    for (int c = 0; c < kOut; ++c) {
        const int q = k * kOut + c;
        const float2 lr = A.cur.r[q];
        A.lpos[q] = make_float2(lr.x + gpos[c].x, lr.y + gpos[c].y);
        const float2 lv = A.lvh[q];
        A.lvh[q] = make_float2(lv.x + gvh[c].x, lv.y + gvh[c].y);
        A.lrec[q] = grec[c];
    }
}

// Back to the previous step's order (particle i there, slot dst here): the
// EOS record and the density predictor, the carried {d, D}, the reorder and
// the drift, transposed.  Bc is this step's record, Bp the previous one (the
// state the step started from).
__global__ void __launch_bounds__(kAThreads) ka_back(Consts K, Bufs Bc, Bufs Bp, ABufs A, int prime)
{
    __shared__ float red[kAThreads / 32][kOut][3];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float part[kOut][3];
#pragma unroll
    for (int c = 0; c < kOut; ++c) part[c][0] = part[c][1] = part[c][2] = 0.0f;
    if (i < K.nf) {
        const int dst = Bc.perm_dst[i];
        const float dt = prime ? 0.0f : Bc.S->dt_f;
        const float ratio = prime ? 1.0f : Bc.S->ratio_f;
        const float2 r = Bp.s_pos[i], v = Bp.st_vel[i], a = Bp.st_a[i], X = Bp.st_X[i];
        const float2 D = Bp.st_D[i];
        const float4 rec = Bc.s_aux[dst];
        const float2 rn = Bc.s_pos[dst];
        const bool keyfrozen = outside_box(K, rn.x, rn.y);
        const bool frozen0 = outside_box(K, r.x, r.y);
        // EOS record of the predicted density
        const float dp = rec.x, x = 1.0f + dp, rho = K.rho0 * x;
        const float praw = tait_raw(K, dp);
        const bool cut = !(praw > K.p_cav);
        const float p = cut ? K.p_cav : praw;
        const float slope = cut ? 0.0f : tait_slope(K, dp);
        const bool clamp = dp <= K.d_lo || dp >= K.d_hi;
        // the drift's wall decisions, repeated with the forward arithmetic
        float2 vh = make_float2(fmaf(0.5f * dt, a.x, v.x), fmaf(0.5f * dt, a.y, v.y));
        bool rx = false, ry = false;
        if (!frozen0 && K.side_walls) {
            const float yy = fmaf(dt, fmaf(K.eps_xsph, X.y, vh.y), r.y);
            const float xx = fmaf(dt, fmaf(K.eps_xsph, X.x, vh.x), r.x);
            ry = yy > K.W2 || yy < -K.W2;
            rx = K.end_walls && (xx > K.Lx || xx < 0.0f);
        }
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const int q = dst * kOut + c;
            const float4 lr4 = A.lrec[q];
            const float2 lrd = A.lrd[q];
            float dbar = lr4.x;
            const float pbar = lr4.w + lr4.y / (rho * rho);
            dbar = fmaf(lr4.y, -2.0f * p * K.rho0 / (rho * rho * rho), dbar);
            if (!cut) {
                dbar = fmaf(pbar, slope, dbar);
                part[c][1] = fmaf(pbar, 2.0f * praw, part[c][1]);
            }
            dbar = fmaf(lr4.z, rec.w * K.half_gm1 / x, dbar);
            part[c][0] = fmaf(lr4.z, rec.w, part[c][0]);
            part[c][1] = fmaf(lr4.z, rec.w, part[c][1]);
            float ld = lrd.x, lD = lrd.y, lE = 0.0f;
            if (keyfrozen) {
                ld += dbar;
            } else if (!clamp) {
                ld += dbar;
                lD = fmaf(dt * (1.0f + ratio), dbar, lD);
                lE = -dt * ratio * dbar;
                part[c][2] = fmaf(fmaf(ratio, D.x - D.y, D.x), dbar, part[c][2]);
            }
            const float2 lpu = A.lpos[q], lvu = A.lvh[q];
            float2 lr_ = lpu, lv_ = lvu, la_ = make_float2(0.f, 0.f), lX_ = make_float2(0.f, 0.f);
            if (!frozen0) {
                // y
                {
                    float lvh = ry ? -lvu.y : lvu.y;
                    if (!ry) {
                        lvh = fmaf(dt, lpu.y, lvh);
                        lX_.y = dt * K.eps_xsph * lpu.y;
                        part[c][2] = fmaf(fmaf(K.eps_xsph, X.y, vh.y), lpu.y, part[c][2]);
                        lr_.y = lpu.y;
                    } else {
                        lr_.y = 0.0f;
                    }
                    lv_.y = lvh;
                    la_.y = 0.5f * dt * lvh;
                    part[c][2] = fmaf(0.5f * a.y, lvh, part[c][2]);
                }
                // x
                {
                    float lvh = rx ? -lvu.x : lvu.x;
                    if (!rx) {
                        lvh = fmaf(dt, lpu.x, lvh);
                        lX_.x = dt * K.eps_xsph * lpu.x;
                        part[c][2] = fmaf(fmaf(K.eps_xsph, X.x, vh.x), lpu.x, part[c][2]);
                        lr_.x = lpu.x;
                    } else {
                        lr_.x = 0.0f;
                    }
                    lv_.x = lvh;
                    la_.x = 0.5f * dt * lvh;
                    part[c][2] = fmaf(0.5f * a.x, lvh, part[c][2]);
                }
            }
            const int o = i * kOut + c;
            A.prv.r[o] = lr_;
            A.prv.v[o] = lv_;
            A.prv.a[o] = la_;
            A.prv.X[o] = lX_;
            A.prv.d[o] = ld;
            A.prv.D[o] = lD;
            A.prv.E[o] = lE;
        }
    }
    if (prime) part[0][2] = part[1][2] = 0.0f;   // dt = 0 is a constant there
#pragma unroll
    for (int c = 0; c < kOut; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float s = lane_sum(part[c][e]);
            if (lane == 0) red[w][c][e] = s;
        }
    __syncthreads();
    if (threadIdx.x < kOut) {
        const int c = threadIdx.x;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int k = 0; k < kAThreads / 32; ++k) {
            s0 += red[k][c][0];
            s1 += red[k][c][1];
            s2 += red[k][c][2];
        }
        A.bk_part[blockIdx.x * kOut + c] = make_float4(s0, s1, s2, 0.0f);
    }
}

// Partial sums of the step's block and ghost partials (the parameters' and
// dt's adjoints, and the disk ghosts' x_c, v_w, a_w adjoints): block r of
// kAReduceBlocks sums slice r of each array in compensated FP32 (two-float)
// and writes its 12 sums; ka_close adds the blocks' sums in block order.
constexpr int kAReduceBlocks = 128;
constexpr int kAReduceThreads = 256;
constexpr int kASums = kOut * 6;   // per component: alpha, c0, dt, x_c, v_w, a_w

__device__ __forceinline__ void slice_of(int n, int r, int &lo, int &hi)
{
    const int per = (n + kAReduceBlocks - 1) / kAReduceBlocks;
    lo = min(n, r * per);
    hi = min(n, lo + per);
}

__global__ void __launch_bounds__(kAReduceThreads) ka_reduce(Consts K, ABufs A, int n_ep, int n_bk,
                                                            float2 *out)
{
    __shared__ F2 red[kAReduceThreads / 32][kASums];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    F2 s[kASums];
#pragma unroll
    for (int e = 0; e < kASums; ++e) s[e] = F2{0.0f, 0.0f};
    int lo, hi;
    slice_of(n_ep, blockIdx.x, lo, hi);
    for (int b = lo + threadIdx.x; b < hi; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < kOut; ++c) s[c * 6 + 2] = f2_add(s[c * 6 + 2], F2{A.ep_part[b * kOut + c], 0.0f});
    slice_of(n_bk, blockIdx.x, lo, hi);
    for (int b = lo + threadIdx.x; b < hi; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const float4 v = A.bk_part[b * kOut + c];
            s[c * 6 + 0] = f2_add(s[c * 6 + 0], F2{v.x, 0.0f});
            s[c * 6 + 1] = f2_add(s[c * 6 + 1], F2{v.y, 0.0f});
            s[c * 6 + 2] = f2_add(s[c * 6 + 2], F2{v.z, 0.0f});
        }
    slice_of(K.nw + K.ng, blockIdx.x, lo, hi);
    for (int g = lo + threadIdx.x; g < hi; g += blockDim.x)
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const float4 v = A.gpar[g * kOut + c];
            s[c * 6 + 0] = f2_add(s[c * 6 + 0], F2{v.x, 0.0f});
            s[c * 6 + 1] = f2_add(s[c * 6 + 1], F2{v.y, 0.0f});
            if (g >= K.nw) {
                s[c * 6 + 3] = f2_add(s[c * 6 + 3], F2{A.grg[g * kOut + c].x, 0.0f});
                s[c * 6 + 4] = f2_add(s[c * 6 + 4], F2{v.z, 0.0f});
                s[c * 6 + 5] = f2_add(s[c * 6 + 5], F2{v.w, 0.0f});
            }
        }
#pragma unroll
    for (int e = 0; e < kASums; ++e) {
        const F2 v = f2_warp_sum(s[e]);
        if (lane == 0) red[w][e] = v;
    }
    __syncthreads();
    if (threadIdx.x < kASums) {
        F2 t{0.0f, 0.0f};
        for (int k = 0; k < kAReduceThreads / 32; ++k) t = f2_add(t, red[k][threadIdx.x]);
        out[blockIdx.x * kASums + threadIdx.x] = make_float2(t.hi, t.lo);
    }
}

// The disk kinematics' derivatives at the time S->t (x_c, v_w, a_w by t and
// by ln tau, FP64 duals), for the reverse sweep of the step; one thread, on
// the recomputed step's side branch beside the drift and the sort.
__global__ void ka_kin(Consts K, const Scalars *S, double *kin)
{
    if (threadIdx.x != 0) return;
    D3d t = dconst(S->t);
    t.d[0] = 1.0;   // direction 0: d/dt; direction 2: d/d ln tau (set by kinematics_T)
    D3d xk, vk, ak;
    kinematics_T(K, t, &xk, &vk, &ak);
    kin[0] = xk.d[0];
    kin[1] = vk.d[0];
    kin[2] = ak.d[0];
    kin[3] = xk.d[2];
    kin[4] = vk.d[2];
    kin[5] = ak.d[2];
}

// Closes the step's reverse sweep (kASums blocks of kAReduceBlocks threads):
// adds the ka_reduce sums in a fixed order (thread b reads block b's sums;
// FP64 across the block), transposes the disk kinematics at t^{n+1} (x_c,
// v_w, a_w as functions of t and tau, from the tangent's FP64 duals),
// carries the adjoint of t (t^{n+1} = t^n + dt) and adds the wall impulse's
// direct dependence on dt (F_wall of the step).
__global__ void __launch_bounds__(kAReduceBlocks) ka_close(Consts K, Bufs B, ABufs A, int prime,
                                                          const float2 *sums, const double *kin)
{
    // One block per sum e (kASums blocks): its warps form the FP64 lane sums
    // of e over the kAReduceBlocks partials; the block that finishes last
    // (atomic ticket) adds them across warps, one lane per sum, and closes
    // the two components on two lanes.  (An FP64 instruction holds its warp
    // for many cycles on this GPU; spread over blocks and lanes the same
    // additions, in the same order, take a fraction of the time.)
    __shared__ int last;
    __shared__ double tot[kASums];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, e = blockIdx.x;
    {
        const float2 v = sums[threadIdx.x * kASums + e];
        const double x = lane_sum((double)v.x + (double)v.y);
        if (lane == 0) A.cpart[w * kASums + e] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(A.ctick, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < kASums) {
        double v = 0.0;
        for (int k = 0; k < kAReduceBlocks / 32; ++k) v += __ldcg(&A.cpart[k * kASums + threadIdx.x]);
        tot[threadIdx.x] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) *A.ctick = 0;
    if (threadIdx.x >= kOut) return;
    double *sc = A.sc;
    // kinematics derivatives at this step's time (t^{n+1}; 0 for the priming
    // pass), formed by ka_kin when the step was recorded; component c on lane c
    const int c = threadIdx.x;
    const double *q = tot + c * 6;
    sc[ASC_ALPHA + c] += q[0];
    sc[ASC_C0 + c] += q[1];
    double dtb = q[2];
    const double xb = q[3], vb = q[4], ab = q[5];
    if (K.ng > 0) sc[ASC_TAU + c] += xb * kin[3] + vb * kin[4] + ab * kin[5];
    if (!prime) {
        if (K.ng > 0) sc[ASC_TBAR + c] += xb * kin[0] + vb * kin[1] + ab * kin[2];
        dtb += sc[ASC_TBAR + c];
        if (c == 1) dtb += B.S->Fwall;   // J = sum_n dt F_wall^{n+1}
    }
    sc[ASC_DT + c] += dtb;
}

// The uploaded state in fluid-ID order, rebuilt from the primed state (the
// priming pass moves nothing: dt = 0): positions, velocities, densities;
// zero rates and accelerations, identity IDs.
__global__ void ka_to_id_order(Consts K, Bufs B, Slot U)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K.nf) return;
    const int id = B.s_id[k];
    U.s_pos[id] = B.s_pos[k];
    U.st_vel[id] = B.st_vel[k];
    U.st_rho[id] = B.st_rho[k];
    U.st_a[id] = make_float2(0.f, 0.f);
    U.st_X[id] = make_float2(0.f, 0.f);
    U.st_D[id] = make_float2(0.f, 0.f);
    U.s_id[id] = id;
}

}  // namespace hr
