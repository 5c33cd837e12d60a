// hram_tangent.cuh -- tangent-linear (forward-mode) derivatives of the step
// with respect to the artificial-viscosity coefficient alpha, the reference
// sound speed c0 and the disk's deceleration time tau.
//
// Every quantity of the step is carried as a dual number: its value and its
// derivatives along three directions, d/d(ln alpha), d/d(ln c0), d/d(ln tau)
// (relative directions keep all derivatives at the scale of the values).
// The tangent kernels run beside the forward kernels inside the same step
// graph; they take the forward step's neighbour sets, cell order and clamp /
// cutoff / switch decisions from the forward values and recompute the pair
// terms on duals, so the derivative is that of the discrete step itself.
// Outputs: the derivatives of the peak probe-0 pressure max_n p(t^n) (taken
// at the argmax step) and of the wall impulse sum_n dt^n F_wall^{n+1}.
// Restricted to a fixed time step (dt_mode 1: dt = C h / (c0 + v0), smooth in
// c0) and the prescribed motions 0-2.
#pragma once
#include "hram_device.cuh"

namespace hr {

constexpr int kDir = 3;
constexpr int kTPassThreads = 128;

template <typename R>
struct Dual {
    R v;
    R d[kDir];
};
using D3 = Dual<float>;
using D3d = Dual<double>;

template <typename R>
__device__ __forceinline__ Dual<R> dconst(R v)
{
    Dual<R> a;
    a.v = v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) a.d[k] = R(0);
    return a;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator+(const Dual<R> &a, const Dual<R> &b)
{
    Dual<R> c;
    c.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = a.d[k] + b.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator-(const Dual<R> &a, const Dual<R> &b)
{
    Dual<R> c;
    c.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = a.d[k] - b.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator-(const Dual<R> &a)
{
    Dual<R> c;
    c.v = -a.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = -a.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator*(const Dual<R> &a, const Dual<R> &b)
{
    Dual<R> c;
    c.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator*(R s, const Dual<R> &a)
{
    Dual<R> c;
    c.v = s * a.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = s * a.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator+(const Dual<R> &a, R s)
{
    Dual<R> c = a;
    c.v += s;
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator+(R s, const Dual<R> &a)
{
    return a + s;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator*(const Dual<R> &a, R s)
{
    return s * a;
}

template <typename R>
__device__ __forceinline__ Dual<R> inv(const Dual<R> &a)
{
    Dual<R> c;
    c.v = R(1) / a.v;
    const R g = -c.v * c.v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = g * a.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> operator/(const Dual<R> &a, const Dual<R> &b)
{
    return a * inv(b);
}

template <typename R>
__device__ __forceinline__ Dual<R> dsqrt(const Dual<R> &a)
{
    Dual<R> c;
    c.v = sqrt(a.v);
    const R g = c.v > R(0) ? R(0.5) / c.v : R(0);
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = g * a.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> dexp(const Dual<R> &a)
{
    Dual<R> c;
    c.v = exp(a.v);
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = c.v * a.d[k];
    return c;
}

template <typename R>
__device__ __forceinline__ Dual<R> dlog(const Dual<R> &a)
{
    Dual<R> c;
    c.v = log(a.v);
#pragma unroll
    for (int k = 0; k < kDir; ++k) c.d[k] = a.d[k] / a.v;
    return c;
}

// max / min: the branch the value takes (derivative of the active argument)
template <typename R>
__device__ __forceinline__ Dual<R> dmax(const Dual<R> &a, const Dual<R> &b)
{
    return a.v >= b.v ? a : b;
}

template <typename R>
__device__ __forceinline__ Dual<R> dmin(const Dual<R> &a, const Dual<R> &b)
{
    return a.v <= b.v ? a : b;
}

__device__ __forceinline__ D3 dwarp_sum(D3 a)
{
    a.v = warp_sum(a.v);
#pragma unroll
    for (int k = 0; k < kDir; ++k) a.d[k] = warp_sum(a.d[k]);
    return a;
}

// Tangent buffers: direction k of particle i at [i * kDir + k] (fluid, current
// cell order; ghosts by ghost index), so that one neighbour's three
// derivatives share cache lines in the gathers.
struct TBufs {
    int n, ngh;
    float2 *s_pos, *s_vel;
    float4 *s_aux;          // tangents of {d~, p~, p~/rho~^2, -alpha h c~}
    float2 *s_rd;           // tangents of {d^n, D^n}
    float2 *st_vel;
    float *st_rho;
    float2 *st_a, *st_D, *st_X;
    float2 *u_pos, *u_vel;
    float2 *g_vel;
    float4 *g_aux;
    int *perm_dst;          // forward sort: previous slot -> this step's slot
    float *part;            // per pass block: wall-force tangents / m^2
    double *sc;             // scalar tangents and the outputs (layout: TSC_*)
};

enum {
    TSC_DT = 0,        // d dt / d ln(theta_k)                         [3]
    TSC_T = 3,         // d t                                          [3]
    TSC_XC = 6,        // d x_c                                        [3]
    TSC_V = 9,         // d v_proj                                     [3]
    TSC_A = 12,        // d a_proj                                     [3]
    TSC_IMP = 15,      // d wall impulse                               [3]
    TSC_PEAK = 18,     // peak probe-0 pressure (value)
    TSC_DPEAK = 19,    // its derivative at the argmax step            [3]
    TSC_PSTEP = 22,    // argmax step
    TSC_FW = 23,       // d F_wall of the last step                    [3]
    TSC_N = 32
};

template <typename R>
__device__ __forceinline__ Dual<R> tload(const float *base, int stride, int i, R v)
{
    Dual<R> a;
    a.v = v;
#pragma unroll
    for (int k = 0; k < kDir; ++k) a.d[k] = R(base[i * kDir + k]);
    return a;
}

__device__ __forceinline__ void tload2(const float2 *base, int stride, int i, float2 v, D3 &x, D3 &y)
{
    x.v = v.x;
    y.v = v.y;
#pragma unroll
    for (int k = 0; k < kDir; ++k) {
        const float2 t = base[i * kDir + k];
        x.d[k] = t.x;
        y.d[k] = t.y;
    }
}

__device__ __forceinline__ void tstore2(float2 *base, int stride, int i, const D3 &x, const D3 &y)
{
#pragma unroll
    for (int k = 0; k < kDir; ++k) base[i * kDir + k] = make_float2(x.d[k], y.d[k]);
}

__device__ __forceinline__ void tstore1(float *base, int stride, int i, const D3 &x)
{
#pragma unroll
    for (int k = 0; k < kDir; ++k) base[i * kDir + k] = x.d[k];
}

// the parameters as duals along their own (relative) directions
__device__ __forceinline__ D3 p_alpha(const Consts &K)
{
    D3 a = dconst(K.alpha_f);
    a.d[0] = K.alpha_f;   // d/d(ln alpha)
    return a;
}

__device__ __forceinline__ D3 p_c0(const Consts &K)
{
    D3 a = dconst(K.c0);
    a.d[1] = K.c0;
    return a;
}

// Tait pressure and its EOS record on duals (B = rho0 c0^2 / gamma).
__device__ __forceinline__ D3 tait_p_T(const Consts &K, const D3 &d)
{
    const D3 c0 = p_c0(K);
    const D3 B = (K.rho0 / K.gamma) * (c0 * c0);
    D3 p;
    if (K.gamma7) {
        D3 poly = d + 7.0f;
        poly = d * poly + 21.0f;
        poly = d * poly + 35.0f;
        poly = d * poly + 35.0f;
        poly = d * poly + 21.0f;
        poly = d * poly + 7.0f;
        p = B * (d * poly);
    } else {
        p = B * (dexp(K.gamma * dlog(d + 1.0f)) + (-1.0f));
    }
    return p.v > K.p_cav ? p : dconst(K.p_cav);
}

__device__ __forceinline__ D3 sound_T(const Consts &K, const D3 &d)
{
    const D3 x = d + 1.0f;
    if (K.gamma7) return p_c0(K) * (x * x * x);
    return p_c0(K) * dexp(K.half_gm1 * dlog(x));
}

// {d, p, p / rho^2, -alpha h c} on duals
__device__ __forceinline__ void eos_record_T(const Consts &K, const D3 &d, D3 *rec)
{
    const D3 p = tait_p_T(K, d);
    const D3 rho = K.rho0 * (d + 1.0f);
    rec[0] = d;
    rec[1] = p;
    rec[2] = p * inv(rho * rho);
    rec[3] = (-K.h) * (p_alpha(K) * sound_T(K, d));
}

struct SelfT {
    D3 x, y, vx, vy, rho, P, c;
};

struct AccT {
    D3 ax, ay, dr, Xx, Xy;
};

// pair_terms on duals (same formula as the float version)
__device__ __forceinline__ void pair_T(const Consts &K, const SelfT &I, const D3 &xj, const D3 &yj,
                                       const D3 &vxj, const D3 &vyj, const D3 &rhoj, const D3 &Pj,
                                       const D3 &cj, float mj, bool xsph, AccT &A, D3 &fx, D3 &fy)
{
    const D3 dx = I.x - xj, dy = I.y - yj;
    const D3 r2 = dx * dx + dy * dy;
    const D3 r = dsqrt(r2);
    const D3 t = dmax(1.0f + (-K.half_inv_h) * r, dconst(0.0f));
    const D3 t3 = t * t * t;
    const D3 F = (mj * K.Fc) * t3;
    const D3 vx = I.vx - vxj, vy = I.vy - vyj;
    const D3 vr = vx * dx + vy * dy;
    A.dr = A.dr + F * vr;
    const D3 e = r2 + K.eh2;
    const D3 iv = inv(e * (I.rho + rhoj));
    const D3 Pi = (I.c + cj) * dmin(vr, dconst(0.0f)) * iv;
    const D3 PF = (I.P + Pj + Pi) * F;
    const D3 lam = K.nu4 * (F * r2 * iv);
    fx = lam * vx - PF * dx;
    fy = lam * vy - PF * dy;
    A.ax = A.ax + fx;
    A.ay = A.ay + fy;
    if (xsph) {
        const D3 wx = K.m2Wc * (t3 * t * (1.0f + K.two_inv_h * r) * (iv * e));
        A.Xx = A.Xx + wx * vx;
        A.Xy = A.Xy + wx * vy;
    }
}

__device__ __forceinline__ D3 kernel_W_T(const Consts &K, const D3 &r)
{
    const D3 t = dmax(1.0f + (-K.half_inv_h) * r, dconst(0.0f));
    const D3 t2 = t * t;
    return K.Wc * (t2 * t2 * (1.0f + K.two_inv_h * r));
}

// Kinematics on FP64 duals: t carries its c0-derivative (through dt), tau
// its own direction.
__device__ inline void kinematics_T(const Consts &K, const D3d &t, D3d *xo, D3d *vo, D3d *ao)
{
    const double v0 = K.v0, tr = K.t_ramp;
    D3d tau = dconst(K.tau);
    tau.d[2] = K.tau;
    D3d x = dconst(K.x_c0), v, a;
    if (K.motion == 2) {
        v = K.a_const * t;
        a = dconst(K.a_const);
        x = x + (0.5 * K.a_const) * (t * t);
    } else if (K.motion == 1) {
        if (tr > 0.0 && t.v < tr) {
            v = (v0 / tr) * t;
            a = dconst(v0 / tr);
            x = x + (0.5 * v0 / tr) * (t * t);
        } else {
            const double t1 = tr > 0.0 ? tr : 0.0;
            const D3d u = 1.0 + (K.drag_k * v0) * (t + (-t1));
            v = v0 * inv(u);
            a = (-K.drag_k) * (v * v);
            x = x + 0.5 * v0 * t1 + (1.0 / K.drag_k) * dlog(u);
        }
    } else {
        D3d f, df, e, de;
        if (tr > 0.0 && t.v < tr) { f = (1.0 / tr) * t; df = dconst(1.0 / tr); }
        else { f = dconst(1.0); df = dconst(0.0); }
        if (K.tau > 0.0) { e = dexp(-(t / tau)); de = -(e / tau); }
        else { e = dconst(1.0); de = dconst(0.0); }
        v = v0 * (f * e);
        a = v0 * (df * e + f * de);
        if (K.tau > 0.0) {
            if (tr > 0.0) {
                const D3d ta = t.v < tr ? t : dconst(tr);
                x = x + (v0 / tr) * (tau * tau - tau * (ta + tau) * dexp(-(ta / tau)));
                if (t.v > tr) x = x + v0 * (tau * (dexp(-(dconst(tr) / tau)) - dexp(-(t / tau))));
            } else {
                x = x + v0 * (tau * (1.0 + (-1.0) * dexp(-(t / tau))));
            }
        } else {
            if (tr > 0.0) {
                const D3d ta = t.v < tr ? t : dconst(tr);
                x = x + (0.5 * v0 / tr) * (ta * ta);
                if (t.v > tr) x = x + v0 * (t + (-tr));
            } else {
                x = x + v0 * t;
            }
        }
    }
    *xo = x;
    *vo = v;
    *ao = a;
}


// ------------------------------------------------------------- kernels

// Kinematics tangents (after k_kinematics, on the same graph branch).
__global__ void kt_kinematics(Consts K, Bufs B, TBufs T, int prime)
{
    if (threadIdx.x != 0) return;
    double *sc = T.sc;
    if (!prime)
        for (int k = 0; k < kDir; ++k) sc[TSC_T + k] += sc[TSC_DT + k];
    D3d t = dconst(B.S->t);
    for (int k = 0; k < kDir; ++k) t.d[k] = sc[TSC_T + k];
    D3d x, v, a;
    kinematics_T(K, t, &x, &v, &a);
    for (int k = 0; k < kDir; ++k) {
        sc[TSC_XC + k] = x.d[k];
        sc[TSC_V + k] = v.d[k];
        sc[TSC_A + k] = a.d[k];
    }
}

__device__ __forceinline__ D3 dual_dt(const Consts &K, const Bufs &B, const TBufs &T, int prime)
{
    D3 dt = dconst(prime ? 0.0f : B.S->dt_f);
    for (int k = 0; k < kDir; ++k) dt.d[k] = prime ? 0.0f : (float)T.sc[TSC_DT + k];
    return dt;
}

// Drift tangents (previous cell order), after k_drift_key and before the
// reorder overwrites the previous positions.  Wall reflections follow the
// forward decision (the same float arithmetic).
__global__ void __launch_bounds__(256) kt_drift(Consts K, Bufs B, TBufs T, int prime)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    const int n = T.n;
    const float2 r = B.s_pos[i], v = B.st_vel[i], a = B.st_a[i], X = B.st_X[i];
    D3 x, y, vx, vy, ax, ay, Xx, Xy;
    tload2(T.s_pos, n, i, r, x, y);
    tload2(T.st_vel, n, i, v, vx, vy);
    if (outside_box(K, r.x, r.y)) {
        tstore2(T.u_pos, n, i, x, y);
        tstore2(T.u_vel, n, i, vx, vy);
        return;
    }
    tload2(T.st_a, n, i, a, ax, ay);
    tload2(T.st_X, n, i, X, Xx, Xy);
    const D3 dt = dual_dt(K, B, T, prime);
    const D3 hdt = 0.5f * dt;
    D3 vhx = vx + hdt * ax, vhy = vy + hdt * ay;
    D3 nx = x + dt * (vhx + K.eps_xsph * Xx), ny = y + dt * (vhy + K.eps_xsph * Xy);
    // the forward step's values, to repeat its wall decisions
    const float fdt = dt.v;
    float2 vh, rr;
    vh.x = fmaf(0.5f * fdt, a.x, v.x);
    vh.y = fmaf(0.5f * fdt, a.y, v.y);
    rr.x = fmaf(fdt, fmaf(K.eps_xsph, X.x, vh.x), r.x);
    rr.y = fmaf(fdt, fmaf(K.eps_xsph, X.y, vh.y), r.y);
    if (K.side_walls) {
        if (rr.y > K.W2 || rr.y < -K.W2) { ny = dconst(ny.v); vhy = -vhy; }
        if (K.end_walls && (rr.x > K.Lx || rr.x < 0.0f)) { nx = dconst(nx.v); vhx = -vhx; }
    }
    tstore2(T.u_pos, n, i, nx, ny);
    tstore2(T.u_vel, n, i, vhx, vhy);
}

// Reorder of the tangents with the forward permutation, predicted density
// and its EOS record on duals (after k_rank_scatter).
__global__ void __launch_bounds__(256) kt_scatter(Consts K, Bufs B, TBufs T, int prime)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K.nf) return;
    const int n = T.n;
    const int dst = T.perm_dst[i];
    const float d = B.st_rho[i];
    const float2 D = B.st_D[i];
    const D3 dd = tload<float>(T.st_rho, n, i, d);
    D3 Dx, Dy;
    tload2(T.st_D, n, i, D, Dx, Dy);
    const float dp_f = B.s_aux[dst].x;   // the forward predicted density
    D3 dp = dd;
    if (B.u_key[i] != K.ncell) {
        const D3 dt = dual_dt(K, B, T, prime);
        const float ratio = prime ? 1.0f : B.S->ratio_f;
        dp = dd + dt * (Dx + ratio * (Dx - Dy));
        if (dp_f <= K.d_lo || dp_f >= K.d_hi) dp = dconst(dp_f);
        dp.v = dp_f;
    }
    D3 rec[4];
    eos_record_T(K, dp, rec);
    for (int k = 0; k < kDir; ++k) {
        T.s_pos[dst * kDir + k] = T.u_pos[i * kDir + k];
        T.s_vel[dst * kDir + k] = T.u_vel[i * kDir + k];
        T.s_aux[dst * kDir + k] = make_float4(rec[0].d[k], rec[1].d[k], rec[2].d[k], rec[3].d[k]);
        T.s_rd[dst * kDir + k] = make_float2(dd.d[k], Dx.d[k]);
    }
}

__device__ __forceinline__ void fluid_dual(const Bufs &B, const TBufs &T, int j, D3 &x, D3 &y,
                                           D3 &vx, D3 &vy, D3 *aux)
{
    const int n = T.n;
    tload2(T.s_pos, n, j, B.s_pos[j], x, y);
    tload2(T.s_vel, n, j, B.s_vel[j], vx, vy);
    const float4 a = B.s_aux[j];
    const float av[4] = {a.x, a.y, a.z, a.w};
    for (int q = 0; q < 4; ++q) aux[q].v = av[q];
    for (int k = 0; k < kDir; ++k) {
        const float4 t = T.s_aux[j * kDir + k];
        aux[0].d[k] = t.x;
        aux[1].d[k] = t.y;
        aux[2].d[k] = t.z;
        aux[3].d[k] = t.w;
    }
}

__device__ __forceinline__ void ghost_dual(const Bufs &B, const TBufs &T, int g, D3 &vx, D3 &vy,
                                           D3 *aux)
{
    const int m = T.ngh;
    tload2(T.g_vel, m, g, B.g_vel[g], vx, vy);
    const float4 a = B.g_aux[g];
    const float av[4] = {a.x, a.y, a.z, a.w};
    for (int q = 0; q < 4; ++q) aux[q].v = av[q];
    for (int k = 0; k < kDir; ++k) {
        const float4 t = T.g_aux[g * kDir + k];
        aux[0].d[k] = t.x;
        aux[1].d[k] = t.y;
        aux[2].d[k] = t.z;
        aux[3].d[k] = t.w;
    }
}

__device__ __forceinline__ D3 disk_coord_dual(const TBufs &T, float v)
{
    D3 a = dconst(v);
    for (int k = 0; k < kDir; ++k) a.d[k] = (float)T.sc[TSC_XC + k];
    return a;
}

// Ghost tangents (after k_ghost): one warp per ghost, same candidates.
__global__ void __launch_bounds__(kGhostWarps * 32) kt_ghost(Consts K, Bufs B, TBufs T)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x * kGhostWarps + w;
    if (g >= K.nw + K.ng) return;
    const bool disk = g >= K.nw;
    const float2 rgf = disk ? B.gd_pos[g - K.nw] : B.gw_pos[g];
    const D3 gx = disk ? disk_coord_dual(T, rgf.x) : dconst(rgf.x);
    const D3 gy = dconst(rgf.y);
    D3 vw = dconst(0.0f), aw = dconst(0.0f);
    if (disk) {
        vw.v = B.S->vproj_f;
        aw.v = B.S->aproj_f;
        for (int k = 0; k < kDir; ++k) {
            vw.d[k] = (float)T.sc[TSC_V + k];
            aw.d[k] = (float)T.sc[TSC_A + k];
        }
    }
    D3 SW = dconst(0.f), Sp = SW, Srx = SW, Sry = SW, Svx = SW, Svy = SW;
    const bool inside = !outside_box(K, rgf.x, rgf.y);
    if (inside) {
        const int c = cell_of(K, rgf.x, rgf.y);
        for (int dy = -1; dy <= 1; ++dy) {
            const int row = c + dy * K.ncx;
            if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, &B.S->status)) continue;
            const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
            if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
            for (int j = a + lane; j < b; j += 32) {
                const float2 rj = B.s_pos[j];
                if (!in_support(rgf.x, rgf.y, rj.x, rj.y, K.s2)) continue;
                D3 x, y, vx, vy, aux[4];
                fluid_dual(B, T, j, x, y, vx, vy, aux);
                const D3 dx = gx - x, dy2 = gy - y;
                const D3 W = kernel_W_T(K, dsqrt(dx * dx + dy2 * dy2));
                const D3 rw = (aux[0] + 1.0f) * W;
                SW = SW + W;
                Sp = Sp + aux[1] * W;
                Srx = Srx + rw * dx;
                Sry = Sry + rw * dy2;
                Svx = Svx + vx * W;
                Svy = Svy + vy * W;
            }
        }
    }
    SW = dwarp_sum(SW);
    Sp = dwarp_sum(Sp);
    Srx = dwarp_sum(Srx);
    Sry = dwarp_sum(Sry);
    Svx = dwarp_sum(Svx);
    Svy = dwarp_sum(Svy);
    if (lane != 0) return;
    const D3 c0 = p_c0(K);
    D3 rec[4], vgx, vgy;
    if (SW.v > 0.0f) {
        const D3 iW = inv(SW);
        const D3 bx = K.gx + (-aw);
        D3 pg = (Sp + K.rho0 * (bx * Srx + K.gy * Sry)) * iW;
        if (!(pg.v > K.p_cav)) pg = dconst(K.p_cav);
        const D3 dg = pg * inv(K.rho0 * (c0 * c0));
        const D3 rho = K.rho0 * (dg + 1.0f);
        rec[0] = dg;
        rec[1] = pg;
        rec[2] = pg * inv(rho * rho);
        rec[3] = (-K.h) * (p_alpha(K) * sound_T(K, dg));
        vgx = 2.0f * vw - Svx * iW;
        vgy = -(Svy * iW);
    } else {
        rec[0] = rec[1] = rec[2] = dconst(0.0f);
        rec[3] = (-K.h) * (p_alpha(K) * c0);
        vgx = vw;
        vgy = dconst(0.0f);
    }
    for (int k = 0; k < kDir; ++k) {
        T.g_aux[g * kDir + k] = make_float4(rec[0].d[k], rec[1].d[k], rec[2].d[k], rec[3].d[k]);
        T.g_vel[g * kDir + k] = make_float2(vgx.d[k], vgy.d[k]);
    }
}

// Interaction-pass tangents (after k_pass): the forward neighbour sets,
// pair terms on duals, the epilogue's derivative.
__global__ void __launch_bounds__(kTPassThreads) kt_pass(Consts K, Bufs B, TBufs T, int prime)
{
    __shared__ float red[kTPassThreads / 32][kDir];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = T.n;
    D3 fw = dconst(0.0f);
    if (i < K.nf) {
        const float2 ri = B.s_pos[i];
        D3 x, y, vx, vy, aux[4];
        fluid_dual(B, T, i, x, y, vx, vy, aux);
        D3 dn, Dn;
        tload2(T.s_rd, n, i, B.s_rd[i], dn, Dn);
        if (outside_box(K, ri.x, ri.y)) {
            tstore2(T.st_vel, n, i, vx, vy);
            tstore1(T.st_rho, n, i, dn);
            const D3 z = dconst(0.0f);
            tstore2(T.st_a, n, i, z, z);
            tstore2(T.st_D, n, i, z, z);
            tstore2(T.st_X, n, i, z, z);
        } else {
            SelfT I{x, y, vx, vy, K.rho0 * (aux[0] + 1.0f), aux[2], aux[3]};
            const D3 z = dconst(0.0f);
            AccT A{z, z, z, z, z};
            D3 fx, fy;
            const int c = cell_of(K, ri.x, ri.y);
            // the forward pass's candidate masks (same predicate, same order), so
            // that a warp evaluates the dual pair terms with all lanes that have
            // a neighbour, not once per candidate under a branch
#pragma unroll 1
            for (int dy = -1; dy <= 1; ++dy) {
                const int row = c + dy * K.ncx;
                if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, &B.S->status)) continue;
                const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
                if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
#pragma unroll 1
                for (int base = a; base < b; base += 32) {
                    unsigned m = support_mask(B.s_pos, base, min(32, b - base), ri, K.s2);
                    if (i >= base && i < base + 32) m &= ~(1u << (i - base));
#pragma unroll 1
                    while (m) {
                        const int j = base + __ffs(m) - 1;
                        m &= m - 1u;
                        D3 xj, yj, vxj, vyj, aj[4];
                        fluid_dual(B, T, j, xj, yj, vxj, vyj, aj);
                        pair_T(K, I, xj, yj, vxj, vyj, K.rho0 * (aj[0] + 1.0f), aj[2], aj[3],
                               1.0f, true, A, fx, fy);
                    }
                }
            }
            if (K.nw > 0)
                for_fluid_candidates(K, B.wall_start, c, K.nw, &B.S->status, [&](int k) {
                    const float2 rg = B.gw_pos[k];
                    if (!in_support(ri.x, ri.y, rg.x, rg.y, K.s2)) return;
                    D3 vgx, vgy, ag[4];
                    ghost_dual(B, T, k, vgx, vgy, ag);
                    pair_T(K, I, dconst(rg.x), dconst(rg.y), vgx, vgy, K.rho0 * (ag[0] + 1.0f), ag[2],
                           ag[3], K.wall_over_m, false, A, fx, fy);
                    if (B.gw_kind[k] == KIND_SIDE) {
                        const float2 e = B.gw_nrm[k];
                        fw = fw - (e.x * fx + e.y * fy);
                    }
                });
            if (K.ng > 0) {
                const float xc = B.S->xc_f, yc = B.S->yc_f;
                if (near_disk(K, ri.x, ri.y, xc, yc))
                    for (int k = 0; k < K.ng; ++k) {
                        const float2 rg = B.gd_pos[k];
                        if (outside_box(K, rg.x, rg.y) || !in_support(ri.x, ri.y, rg.x, rg.y, K.s2))
                            continue;
                        D3 vgx, vgy, ag[4];
                        ghost_dual(B, T, K.nw + k, vgx, vgy, ag);
                        pair_T(K, I, disk_coord_dual(T, rg.x), dconst(rg.y), vgx, vgy,
                               K.rho0 * (ag[0] + 1.0f), ag[2], ag[3], K.disk_over_m, false, A, fx, fy);
                    }
            }
            const D3 dt = dual_dt(K, B, T, prime);
            const D3 ax = K.m * A.ax + K.gx, ay = K.m * A.ay + K.gy;
            const D3 Dd = K.m_over_rho0 * A.dr;
            D3 dnew = dn + dt * Dd;
            const float df = B.st_rho[i];
            if (df <= K.d_lo || df >= K.d_hi) dnew = dconst(df);
            const D3 hdt = 0.5f * dt;
            tstore2(T.st_vel, n, i, vx + hdt * ax, vy + hdt * ay);
            tstore1(T.st_rho, n, i, dnew);
            tstore2(T.st_a, n, i, ax, ay);
            tstore2(T.st_D, n, i, Dd, prime ? Dd : Dn);
            tstore2(T.st_X, n, i, K.m * A.Xx, K.m * A.Xy);
        }
    }
    for (int k = 0; k < kDir; ++k) {
        const float s = warp_sum(fw.d[k]);
        if (lane == 0) red[w][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < kDir) {
        float s = 0.0f;
        for (int q = 0; q < kTPassThreads / 32; ++q) s += red[q][threadIdx.x];
        T.part[blockIdx.x * kDir + threadIdx.x] = s;
    }
}

// Step close of the tangents (after k_finalize): wall-impulse derivative and
// the probe-0 peak's derivative at the argmax step.
constexpr int kTFinThreads = 1024;
__global__ void __launch_bounds__(kTFinThreads) kt_finalize(Consts K, Bufs B, TBufs T, int prime, int nblk)
{
    __shared__ double red[kTFinThreads / 32][kDir];
    __shared__ float probe_d[kDir + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the per-block partials: float sums per thread (loads unrolled so they
    // stay in flight), FP64 from the warp level up
    float s[kDir] = {0.0f, 0.0f, 0.0f};
#pragma unroll 4
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int k = 0; k < kDir; ++k) s[k] += T.part[b * kDir + k];
    for (int k = 0; k < kDir; ++k) {
        const double v = warp_sum((double)s[k]);
        if (lane == 0) red[w][k] = v;
    }
    // probe 0 on duals, one warp
    if (w == 0 && !prime && K.n_probes > 0) {
        const float px = K.probe_x[0], py = K.probe_y[0];
        D3 SW = dconst(0.f), Sp = SW, Srx = SW, Sry = SW;
        if (!outside_box(K, px, py)) {
            const int c = cell_of(K, px, py);
            for (int dy = -1; dy <= 1; ++dy) {
                const int row = c + dy * K.ncx;
                if (kChecked && !hr_ok(row - 1 >= 0 && row + 2 <= K.ncell, &B.S->status)) continue;
                const int a = B.cell_start[row - 1], b = B.cell_start[row + 2];
                if (kChecked && !row_ok(K, row, a, b, K.nf, &B.S->status)) continue;
                for (int j = a + lane; j < b; j += 32) {
                    const float2 rj = B.s_pos[j];
                    if (!in_support(px, py, rj.x, rj.y, K.s2)) continue;
                    D3 x, y;
                    tload2(T.s_pos, T.n, j, rj, x, y);
                    const D3 d = tload<float>(T.st_rho, T.n, j, B.st_rho[j]);
                    const D3 dx = dconst(px) - x, dy2 = dconst(py) - y;
                    const D3 W = kernel_W_T(K, dsqrt(dx * dx + dy2 * dy2));
                    const D3 rw = (d + 1.0f) * W;
                    SW = SW + W;
                    Sp = Sp + tait_p_T(K, d) * W;
                    Srx = Srx + rw * dx;
                    Sry = Sry + rw * dy2;
                }
            }
        }
        SW = dwarp_sum(SW);
        Sp = dwarp_sum(Sp);
        Srx = dwarp_sum(Srx);
        Sry = dwarp_sum(Sry);
        if (lane == 0) {
            D3 p = dconst(0.0f);
            if (SW.v > 0.0f) {
                p = (Sp + K.rho0 * (K.gx * Srx + K.gy * Sry)) * inv(SW);
                if (!(p.v > K.p_cav)) p = dconst(K.p_cav);
            }
            probe_d[0] = p.v;
            for (int k = 0; k < kDir; ++k) probe_d[k + 1] = p.d[k];
        }
    }
    __syncthreads();
    if (threadIdx.x != 0 || prime) return;
    double *sc = T.sc;
    const double m2 = (double)K.m * (double)K.m;
    const double dt = B.S->dt_prev;
    const double Fw = B.S->Fwall;
    for (int k = 0; k < kDir; ++k) {
        double f = 0.0;
        for (int q = 0; q < kTFinThreads / 32; ++q) f += red[q][k];
        sc[TSC_FW + k] = m2 * f;
        sc[TSC_IMP + k] += sc[TSC_DT + k] * Fw + dt * sc[TSC_FW + k];
    }
    // the peak follows the forward probe history (its value and its argmax)
    const float pf = B.probe_now[0];
    if (K.n_probes > 0 && B.S->step <= K.probe_cap && (double)pf > sc[TSC_PEAK]) {
        sc[TSC_PEAK] = pf;
        for (int k = 0; k < kDir; ++k) sc[TSC_DPEAK + k] = probe_d[k + 1];
        sc[TSC_PSTEP] = (double)(B.S->step - 1);
    }
}

}  // namespace hr
