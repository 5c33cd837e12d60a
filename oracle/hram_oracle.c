/*
 * hram_oracle.c -- plain, slow, FP64 CPU oracle of the planar WCSPH
 * hydrodynamic-ram step (Alam, Biswas & Chakraborty, "Verification,
 * Sensitivity, and Operating Limits of a GPU-Accelerated Planar WCSPH Model
 * for Hydrodynamic Ram").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path, and the CUDA path
 * never calls it.  Build:  gcc -O2 -ffp-contract=off -fPIC -shared -lm.
 *
 * Every function follows a passage of the paper or one of the readings that
 * settle what the paper leaves open (listed where they are used, tag "R<n>").
 * The structure is the algorithm in the paper's order; nothing is blocked,
 * fused or reordered beyond what those passages state.
 *
 * Precision: all physics in double.  Only the neighbour *predicate* is done in
 * float, on positions rounded to float, so that neighbour sets are defined
 * bit-for-bit (reading R2): j != i is a neighbour of i iff
 *     fl(fl(dx*dx) + fl(dy*dy)) < s2,  dx = fl(xi - xj), dy = fl(yi - yj),
 * with s2 = fl((2h)^2) and no fused multiply-add (hence -ffp-contract=off).
 *
 * Parity status of each part (what pins it is in the tests):
 *   kernel, predicate, neighbour sets, EOS, pair sums, ghost operator,
 *   kinematics, mass and momentum invariants: pinned.
 *   closure 1 (the paper's closure): cubic kernel by quadrature, summation
 *   density by brute-force lattice sums, Mie-Grueneisen EOS against the
 *   shock Hugoniot of the jump conditions, the energy equation by
 *   conservation of kinetic plus internal energy: pinned.
 *   two-way coupling: the disk's energy loss equals the boundary work.
 *   full multi-step run: no closed form -- pinned only through invariants,
 *   hydrostatic rest, added mass (partially: the planar closed form is the
 *   incompressible limit), reflection and arrival-time checks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ params */

/* Planted-mistake switches.  They exist only so the tests can show that the
 * pins catch a plausible slip; every production use passes 0. */
enum {
    MUT_NONE = 0,
    MUT_GHOST_PRINTED_SIGN = 1,  /* (a - g) instead of (g - a) in the ghost pressure */
    MUT_DROP_PJ = 2,             /* drop p_j / rho_j^2 from the momentum sum */
    MUT_KERNEL_NORM = 4,         /* cubic-spline normalisation 10/(7 pi h^2) on Wendland */
    MUT_AV_SIGN = 8,             /* artificial viscosity switched on under separation */
    MUT_DT_NO_GHOSTS = 16,       /* v_max taken over fluid only */
    MUT_GRAD_SIGN = 32,          /* grad W pointing the wrong way */
    MUT_GHOST_VEL = 64,          /* v_g = v_w + <v>  instead of 2 v_w - <v> */
    MUT_ENERGY_HALF = 128,       /* energy equation without its factor 1/2 */
    MUT_SUM_NO_SELF = 256,       /* summation density without the particle itself */
    MUT_XSPH_GRADW = 512,        /* XSPH weighted by |dW/dr| instead of W */
    MUT_XSPH_RHOJ = 1024,        /* XSPH with m_j / rho_j instead of m_j / rhobar_ij */
    MUT_LAM_HALF = 2048,         /* laminar term with 2 nu instead of 4 nu */
    MUT_AV_CONST_C = 4096        /* artificial viscosity with c0 instead of cbar_ij */
};

typedef struct {
    double dx, h_over_dx, Lx, W;
    int32_t wall_layers, end_walls;
    double R_disk, v0, tau, t_ramp, x_c0, y_c0;
    int32_t Ng, motion;
    double a_const, drag_M, drag_Cd, drag_R;
    double rho0, c0, gamma, p_cav, alpha, eta2, eps_xsph, mu_lam, gx, gy, cfl;
    int32_t dt_mode, n_probes;
    double rho_lo, rho_hi, box_pad;
    double probe_xy[32];
    int32_t mutation, brute;
    double disk_density;
    /* closure 0: the workloads' (Wendland, continuity density, Tait);
     * closure 1: the paper's own (cubic B-spline, summation density,
     * Mie-Grueneisen EOS with the internal-energy equation) */
    int32_t closure;
    double mg_S1, mg_gamma0, mg_a, mg_mu_max;
    /* 1: the side walls reflect particles even without ghost layers (the
     * paper's baseline hard wall, Section "The Channel Walls") */
    int32_t wall_reflect;
} orc_params;

enum { KIND_FLUID = 0, KIND_SIDE = 1, KIND_END = 2, KIND_DISK = 3 };

typedef struct {
    orc_params P;
    /* derived constants */
    double h, s, m, alpha_d, B, nu;
    float s2f;
    double x_lo, x_hi, y_lo, y_hi;
    /* fluid state (ID order) */
    int64_t nf;
    double *x, *y, *vx, *vy, *rho, *ax, *ay, *drho, *Xx, *Xy;
    double *vhx, *vhy, *rhoh, *p, *aavx, *aavy, *drho_prev;
    double *e, *eh, *de;   /* closure 1: specific internal energy, its prediction, rate */
    double *vkx, *vky;     /* closure 1: v^{n+1/2} while the operators see v predicted */
    unsigned char *out;
    /* ghosts: walls first, then disk */
    int64_t nw, nd, ngh;
    double *gx, *gy, *gnx, *gny, *gm;
    int32_t *gkind;
    double *gp, *grho, *gvx, *gvy;
    unsigned char *gout;
    double *doffx, *doffy;
    /* time and projectile */
    double t, dt, dt_prev;
    int64_t step;
    double xc, yc, vproj, aproj;
    /* accumulated diagnostics */
    double Wb, impulse, diss, Fdx, Fdy, Fwall, diss_rate;
    double *probe_hist, *probe_t, *probe_imp;
    int64_t hist_n, hist_cap;
    /* neighbour lists of all points; global index: fluid 0..nf-1, ghosts nf.. */
    int64_t *nb_off;
    int32_t *nb_id;
    int64_t nb_cap;
    int32_t penetrated;
} orc_case;

/* --------------------------------------------------------------- kernel */

/* Cubic B-spline kernel in two dimensions (Section "SPH Fundamentals", eq.
 * cubic-kernel; closure 1):
 *   W(q) = s_d (1 - 3/2 q^2 + 3/4 q^3)  for q <= 1,
 *          s_d (2 - q)^3 / 4            for 1 < q <= 2,  s_d = 10 / (7 pi h^2),
 * and F = (dW/dr) / r:
 *   F = s_d / h^2 (-3 + 9/4 q)          for q <= 1,
 *       s_d / h^2 (-3/4 (2 - q)^2 / q)  for 1 < q < 2. */
static double cubic_W(double h, double r)
{
    double q = r / h, sd = 10.0 / (7.0 * M_PI * h * h);
    if (q >= 2.0) return 0.0;
    if (q <= 1.0) return sd * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    return sd * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
}

static double cubic_F(double h, double r)
{
    double q = r / h, sd = 10.0 / (7.0 * M_PI * h * h);
    if (q >= 2.0) return 0.0;
    if (q <= 1.0) return sd / (h * h) * (-3.0 + 2.25 * q);
    return sd / (h * h) * (-0.75 * (2.0 - q) * (2.0 - q) / q);
}

/* Wendland C2 kernel in two dimensions (reading R1, the workloads' kernel):
 *   W(q) = a_d (1 - q/2)^4 (1 + 2q),  q = r/h in [0, 2],  a_d = 7 / (4 pi h^2).
 * Closure 1 uses the cubic B-spline above instead. */
static double kernel_W(const orc_case *c, double r)
{
    if (c->P.closure == 1) return cubic_W(c->h, r);
    double q = r / c->h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return c->alpha_d * t * t * t * t * (1.0 + 2.0 * q);
}

/* grad_i W_ij = F(r) * (r_i - r_j), F = -5 a_d (1 - q/2)^3 / h^2 (derivative
 * of the kernel above divided by r). */
static double kernel_F(const orc_case *c, double r)
{
    if (c->P.closure == 1) {
        double F = cubic_F(c->h, r);
        return (c->P.mutation & MUT_GRAD_SIGN) ? -F : F;
    }
    double q = r / c->h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    double F = -5.0 * c->alpha_d * t * t * t / (c->h * c->h);
    if (c->P.mutation & MUT_GRAD_SIGN) F = -F;
    return F;
}

/* Stand-alone kernel evaluations for the tests (mutation: planted mistakes). */
static void kernel_only_case(orc_case *c, double h, int32_t mutation)
{
    memset(c, 0, sizeof *c);
    c->h = h;
    c->P.mutation = mutation;
    c->alpha_d = (mutation & MUT_KERNEL_NORM) ? 10.0 / (7.0 * M_PI * h * h)
                                              : 7.0 / (4.0 * M_PI * h * h);
}

double orc_kernel_W(double r, double h, int32_t mutation)
{
    orc_case c;
    kernel_only_case(&c, h, mutation);
    return kernel_W(&c, r);
}

double orc_kernel_F(double r, double h, int32_t mutation)
{
    orc_case c;
    kernel_only_case(&c, h, mutation);
    return kernel_F(&c, r);
}

double orc_cubic_W(double r, double h) { return cubic_W(h, r); }
double orc_cubic_F(double r, double h) { return cubic_F(h, r); }

/* ------------------------------------------------------------ predicate */

/* Neighbour predicate of reading R2, float arithmetic, no contraction. */
static int predicate32(float xi, float yi, float xj, float yj, float s2)
{
    volatile float dx = xi - xj;
    volatile float dy = yi - yj;
    volatile float dx2 = dx * dx;
    volatile float dy2 = dy * dy;
    volatile float r2 = dx2 + dy2;
    return r2 < s2;
}

int orc_predicate32(float xi, float yi, float xj, float yj, float s2)
{
    return predicate32(xi, yi, xj, yj, s2);
}

/* ------------------------------------------------------------------ EOS */

/* Tait equation of state with the cavitation cutoff (reading R4; the cutoff
 * p >= p_cav is the paper's, Section "Closure"):
 *   p = max(B ((rho/rho0)^gamma - 1), p_cav),  B = rho0 c0^2 / gamma. */
static double eos_p(const orc_case *c, double rho)
{
    double p = c->B * (pow(rho / c->P.rho0, c->P.gamma) - 1.0);
    return p > c->P.p_cav ? p : c->P.p_cav;
}

/* Mie-Grueneisen equation of state with a linear Us-Up Hugoniot reference
 * (Section "Closure", eq. eos; closure 1), mu = rho/rho0 - 1, C = c0:
 *   mu >= 0:  p = rho0 C^2 mu [1 + (1 - gamma0/2) mu] / [1 - (S1 - 1) mu]^2
 *                 + (gamma0 + a mu) rho e,
 *   mu <  0:  p = rho0 C^2 mu + gamma0 rho e,
 * then p >= p_cav.  Reading P3: the compression cap mu <= mu_max (0.25) is
 * applied to the state, i.e. the whole formula is evaluated at
 * rho = rho0 (1 + min(mu, mu_max)). */
static double mg_p(const orc_case *c, double rho, double e)
{
    const orc_params *P = &c->P;
    double mu = rho / P->rho0 - 1.0;
    if (mu > P->mg_mu_max) mu = P->mg_mu_max;
    double rc = P->rho0 * (1.0 + mu), K = P->rho0 * P->c0 * P->c0, p;
    if (mu >= 0.0) {
        double den = 1.0 - (P->mg_S1 - 1.0) * mu;
        p = K * mu * (1.0 + (1.0 - 0.5 * P->mg_gamma0) * mu) / (den * den)
            + (P->mg_gamma0 + P->mg_a * mu) * rc * e;
    } else {
        p = K * mu + P->mg_gamma0 * rc * e;
    }
    return p > P->p_cav ? p : P->p_cav;
}

double orc_mg_p(const orc_params *P, double rho, double e)
{
    orc_case c;
    memset(&c, 0, sizeof c);
    c.P = *P;
    return mg_p(&c, rho, e);
}

/* Sound speed c = c0 (rho/rho0)^((gamma-1)/2) (reading R5).  Closure 1
 * (reading P4): the reference celerity c0 = C throughout. */
static double sound_speed(const orc_case *c, double rho)
{
    if (c->P.closure == 1) return c->P.c0;
    return c->P.c0 * pow(rho / c->P.rho0, 0.5 * (c->P.gamma - 1.0));
}

/* Density band [rho_lo, rho_hi] rho0 applied after every density update
 * (Section "Density Summation": clamp to [0.5, 1.5] rho0). */
static double clamp_rho(const orc_case *c, double rho)
{
    double lo = c->P.rho_lo * c->P.rho0, hi = c->P.rho_hi * c->P.rho0;
    return rho < lo ? lo : (rho > hi ? hi : rho);
}

/* Specific elastic energy of the Tait fluid (reading R18):
 *   e(rho) = B [ (rho^(g-1) - rho0^(g-1)) / ((g-1) rho0^g) + 1/rho - 1/rho0 ]. */
static double tait_energy(const orc_case *c, double rho)
{
    double g = c->P.gamma, r0 = c->P.rho0;
    return c->B * ((pow(rho, g - 1.0) - pow(r0, g - 1.0)) / ((g - 1.0) * pow(r0, g))
                   + 1.0 / rho - 1.0 / r0);
}

/* ------------------------------------------------------------ kinematics */

/* Prescribed projectile motion along +x at y = y_c0.
 *  motion 0 (reading R11): v = v0 min(t/t_ramp, 1) exp(-t/tau); the ramp is the
 *           paper's velocity ramp, the exponential the workloads' deceleration.
 *  motion 1: the paper's ramp followed by its quadratic drag law,
 *           M dv/dt = -1/2 Cd rho_f pi R^2 v^2, solved in closed form.
 *  motion 2: constant acceleration from rest (verification case).
 *  motion 3: the ramp (no decay); afterwards the disk is driven by the fluid
 *           force (two-way coupling, advanced in orc_step, not here).
 * Returns centre x, velocity and acceleration, all in closed form. */
void orc_kinematics(const orc_params *P, double t, double *xo, double *vo, double *ao)
{
    double v0 = P->v0, tr = P->t_ramp, tau = P->motion == 3 ? 0.0 : P->tau, x = P->x_c0, v, a;
    if (P->motion == 2) {
        v = P->a_const * t;
        a = P->a_const;
        x += 0.5 * P->a_const * t * t;
    } else if (P->motion == 1) {
        double k = P->drag_Cd * P->rho0 * M_PI * P->drag_R * P->drag_R / (2.0 * P->drag_M);
        if (tr > 0.0 && t < tr) {
            v = v0 * t / tr;
            a = v0 / tr;
            x += 0.5 * v0 * t * t / tr;
        } else {
            double t1 = tr > 0.0 ? tr : 0.0;
            double u = 1.0 + k * v0 * (t - t1);
            v = v0 / u;
            a = -k * v * v;
            x += 0.5 * v0 * t1 + log(u) / k;
        }
    } else {
        double f, df, e, de;
        if (tr > 0.0 && t < tr) { f = t / tr; df = 1.0 / tr; }
        else { f = 1.0; df = 0.0; }
        if (tau > 0.0) { e = exp(-t / tau); de = -e / tau; }
        else { e = 1.0; de = 0.0; }
        v = v0 * f * e;
        a = v0 * (df * e + f * de);
        /* x_c(t) = x_c0 + integral_0^t v */
        if (tau > 0.0) {
            if (tr > 0.0) {
                double ta = t < tr ? t : tr;
                x += (v0 / tr) * (tau * tau - tau * (ta + tau) * exp(-ta / tau));
                if (t > tr) x += v0 * tau * (exp(-tr / tau) - exp(-t / tau));
            } else {
                x += v0 * tau * (1.0 - exp(-t / tau));
            }
        } else {
            if (tr > 0.0) {
                double ta = t < tr ? t : tr;
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

/* ------------------------------------------------------------- geometry */

static int in_box(const orc_case *c, double x, double y)
{
    return x >= c->x_lo && x <= c->x_hi && y >= c->y_lo && y <= c->y_hi;
}

/* Wall ghosts (reading R12; the paper's Section "The Channel Walls" with the
 * workloads' three layers).  Layer k = 1..L of the lower and upper walls sits
 * at y = -/+(W/2 + (k - 1/2) dx), x = (i + 1/2) dx.  With closed ends the side
 * bands extend over the corners and end bands x = -(k - 1/2) dx and
 * Lx + (k - 1/2) dx are added.  Mass rho0 dx^2 each.  Order: lower band
 * (layer-major), upper band, left band, right band. */
static int64_t make_walls(orc_case *c, int count_only)
{
    const orc_params *P = &c->P;
    int64_t n = 0;
    int L = P->wall_layers;
    if (L <= 0) return 0;
    int64_t nx = (int64_t)llround(P->Lx / P->dx), ny = (int64_t)llround(P->W / P->dx);
    int64_t i0 = P->end_walls ? -L : 0, i1 = nx + (P->end_walls ? L : 0);
    for (int band = 0; band < 2; ++band)
        for (int k = 1; k <= L; ++k)
            for (int64_t i = i0; i < i1; ++i) {
                if (!count_only) {
                    double yy = band == 0 ? -0.5 * P->W - ((double)k - 0.5) * P->dx
                                          : 0.5 * P->W + ((double)k - 0.5) * P->dx;
                    c->gx[n] = ((double)i + 0.5) * P->dx;
                    c->gy[n] = yy;
                    c->gnx[n] = 0.0;
                    c->gny[n] = band == 0 ? -1.0 : 1.0;
                    c->gkind[n] = KIND_SIDE;
                    c->gm[n] = P->rho0 * P->dx * P->dx;
                }
                ++n;
            }
    if (P->end_walls)
        for (int band = 0; band < 2; ++band)
            for (int k = 1; k <= L; ++k)
                for (int64_t j = 0; j < ny; ++j) {
                    if (!count_only) {
                        double xx = band == 0 ? -((double)k - 0.5) * P->dx
                                              : P->Lx + ((double)k - 0.5) * P->dx;
                        c->gx[n] = xx;
                        c->gy[n] = -0.5 * P->W + ((double)j + 0.5) * P->dx;
                        c->gnx[n] = band == 0 ? -1.0 : 1.0;
                        c->gny[n] = 0.0;
                        c->gkind[n] = KIND_END;
                        c->gm[n] = P->rho0 * P->dx * P->dx;
                    }
                    ++n;
                }
    return n;
}

/* Disk ghosts (Section "The Projectile"): N_g points at theta_k = 2 pi k / N_g
 * on the circle of radius R about the projectile centre, mass
 * rho0 dx (2 pi R / N_g) each. */
static void place_disk(orc_case *c)
{
    for (int64_t k = 0; k < c->nd; ++k) {
        int64_t g = c->nw + k;
        c->gx[g] = c->xc + c->doffx[k];
        c->gy[g] = c->yc + c->doffy[k];
        c->gout[g] = !in_box(c, c->gx[g], c->gy[g]);
    }
}

/* ----------------------------------------------------------- neighbours */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void nb_push(orc_case *c, int64_t *n, int32_t id)
{
    if (*n >= c->nb_cap) {
        c->nb_cap = c->nb_cap ? 2 * c->nb_cap : 1024;
        c->nb_id = (int32_t *)realloc(c->nb_id, (size_t)c->nb_cap * sizeof(int32_t));
    }
    c->nb_id[(*n)++] = id;
}

/* Builds the neighbour list of every point (fluid: fluid + ghosts; ghost:
 * fluid only), sorted by global index.  Points outside the computational box
 * take part in nothing.  The cell grid is only a search accelerator: cells of
 * side 1.01 * 2h, so every pair passing the predicate lies in adjacent cells;
 * brute mode compares all pairs instead. */
static void build_neighbours(orc_case *c)
{
    int64_t np = c->nf + c->ngh;
    float *xf = (float *)malloc((size_t)np * sizeof(float));
    float *yf = (float *)malloc((size_t)np * sizeof(float));
    unsigned char *act = (unsigned char *)malloc((size_t)np);
    for (int64_t i = 0; i < c->nf; ++i) {
        xf[i] = (float)c->x[i];
        yf[i] = (float)c->y[i];
        act[i] = !c->out[i];
    }
    for (int64_t g = 0; g < c->ngh; ++g) {
        xf[c->nf + g] = (float)c->gx[g];
        yf[c->nf + g] = (float)c->gy[g];
        act[c->nf + g] = !c->gout[g];
    }
    c->nb_off = (int64_t *)realloc(c->nb_off, (size_t)(np + 1) * sizeof(int64_t));
    int64_t n = 0;
    if (c->P.brute) {
        for (int64_t i = 0; i < np; ++i) {
            c->nb_off[i] = n;
            if (!act[i]) continue;
            int64_t jmax = i < c->nf ? np : c->nf;
            for (int64_t j = 0; j < jmax; ++j)
                if (j != i && act[j] && predicate32(xf[i], yf[i], xf[j], yf[j], c->s2f))
                    nb_push(c, &n, (int32_t)j);
        }
        c->nb_off[np] = n;
    } else {
        double dc = 1.01 * c->s;
        double x0 = c->x_lo - dc, y0 = c->y_lo - dc;
        int64_t ncx = (int64_t)floor((c->x_hi - c->x_lo) / dc) + 3;
        int64_t ncy = (int64_t)floor((c->y_hi - c->y_lo) / dc) + 3;
        int64_t ncell = ncx * ncy;
        int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
        int64_t *cell = (int64_t *)malloc((size_t)np * sizeof(int64_t));
        for (int64_t i = 0; i < np; ++i) {
            if (!act[i]) { cell[i] = -1; continue; }
            double xx = i < c->nf ? c->x[i] : c->gx[i - c->nf];
            double yy = i < c->nf ? c->y[i] : c->gy[i - c->nf];
            int64_t cx = (int64_t)floor((xx - x0) / dc), cy = (int64_t)floor((yy - y0) / dc);
            cell[i] = cy * ncx + cx;
            cnt[cell[i] + 1]++;
        }
        for (int64_t k = 0; k < ncell; ++k) cnt[k + 1] += cnt[k];
        int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
        memcpy(fill, cnt, (size_t)ncell * sizeof(int64_t));
        int64_t *item = (int64_t *)malloc((size_t)np * sizeof(int64_t));
        for (int64_t i = 0; i < np; ++i)
            if (cell[i] >= 0) item[fill[cell[i]]++] = i;
        for (int64_t i = 0; i < np; ++i) {
            c->nb_off[i] = n;
            if (cell[i] < 0) continue;
            int64_t cx = cell[i] % ncx, cy = cell[i] / ncx;
            int64_t first = n;
            for (int64_t dy = -1; dy <= 1; ++dy)
                for (int64_t dxc = -1; dxc <= 1; ++dxc) {
                    int64_t k = (cy + dy) * ncx + (cx + dxc);
                    for (int64_t a = cnt[k]; a < cnt[k + 1]; ++a) {
                        int64_t j = item[a];
                        if (j == i) continue;
                        if (i >= c->nf && j >= c->nf) continue; /* ghost-ghost: none */
                        if (predicate32(xf[i], yf[i], xf[j], yf[j], c->s2f))
                            nb_push(c, &n, (int32_t)j);
                    }
                }
            qsort(c->nb_id + first, (size_t)(n - first), sizeof(int32_t), cmp_i32);
        }
        c->nb_off[np] = n;
        free(cnt); free(cell); free(fill); free(item);
    }
    free(xf); free(yf); free(act);
}

/* ------------------------------------------------------------- operators */

static void kinematics_now(orc_case *c)
{
    orc_kinematics(&c->P, c->t, &c->xc, &c->vproj, &c->aproj);
    c->yc = c->P.y_c0;
}

/* Two-way coupling (motion 3; the extension the paper names in its
 * Conclusions): after the ramp the disk is no longer prescribed but obeys
 * M' dv/dt = -F, F the force of the disk ghosts on the fluid from the last
 * interaction sums, M' = rho_disk pi R^2 its mass per unit depth.  Advanced
 * with the step's dt by symplectic Euler in FP64:
 *   a = -F_x / M',  v += dt a,  x += dt v.
 * During the ramp (t <= t_ramp) the ramp's closed form is used. */
static void kinematics_advance(orc_case *c, double dt)
{
    if (c->P.motion != 3 || (c->P.t_ramp > 0.0 && c->t <= c->P.t_ramp)) {
        kinematics_now(c);
        return;
    }
    double M = c->P.disk_density * M_PI * c->P.R_disk * c->P.R_disk;
    c->aproj = -c->Fdx / M;
    c->vproj += dt * c->aproj;
    c->xc += dt * c->vproj;
    c->yc = c->P.y_c0;
}

/* Ghost operator G (Section "The Projectile", equations for p_g, rho_g, v_g;
 * reading R13).  For ghost g over its fluid neighbours j:
 *   S_W = sum W_gj,  S_p = sum p_j W_gj,  S_rr = sum rho_j (r_g - r_j) W_gj,
 *   S_v = sum v_j W_gj,
 *   p_g = max( (S_p + (g - a_w) . S_rr) / S_W , p_cav ),
 *   rho_g = rho0 (1 + p_g / (rho0 c0^2)),   v_g = 2 v_w - S_v / S_W,
 * with (v_w, a_w) the projectile's velocity and acceleration for disk ghosts
 * and zero for wall ghosts.  Reading: the body-force term carries (g - a_w)
 * as in the source the paper follows (Adami, Hu & Adams 2012, hydrostatic
 * balance); the paper's printed (a - g) is selectable only as a planted
 * mistake.  S_W = 0 (no fluid neighbour) gives p_g = 0, rho_g = rho0, v_g = v_w.
 * Fluid enters with the half-step state (r^{n+1}, v^{n+1/2}, p(rho^{n+1/2})). */
static void ghost_operator(orc_case *c)
{
    for (int64_t g = 0; g < c->ngh; ++g) {
        int is_disk = c->gkind[g] == KIND_DISK;
        double vwx = is_disk ? c->vproj : 0.0, vwy = 0.0;
        double awx = is_disk ? c->aproj : 0.0, awy = 0.0;
        double SW = 0, Sp = 0, Srx = 0, Sry = 0, Svx = 0, Svy = 0;
        int64_t gi = c->nf + g;
        for (int64_t a = c->nb_off[gi]; a < c->nb_off[gi + 1]; ++a) {
            int64_t j = c->nb_id[a];
            double rx = c->gx[g] - c->x[j], ry = c->gy[g] - c->y[j];
            double Wgj = kernel_W(c, sqrt(rx * rx + ry * ry));
            SW += Wgj;
            Sp += c->p[j] * Wgj;
            Srx += c->rhoh[j] * rx * Wgj;
            Sry += c->rhoh[j] * ry * Wgj;
            Svx += c->vhx[j] * Wgj;
            Svy += c->vhy[j] * Wgj;
        }
        if (SW > 0.0) {
            double bx = c->P.gx - awx, by = c->P.gy - awy;
            if (c->P.mutation & MUT_GHOST_PRINTED_SIGN) { bx = -bx; by = -by; }
            double pg = (Sp + bx * Srx + by * Sry) / SW;
            if (pg < c->P.p_cav) pg = c->P.p_cav;
            c->gp[g] = pg;
            c->grho[g] = c->P.rho0 * (1.0 + pg / (c->P.rho0 * c->P.c0 * c->P.c0));
            if (c->P.mutation & MUT_GHOST_VEL) {
                c->gvx[g] = vwx + Svx / SW;
                c->gvy[g] = vwy + Svy / SW;
            } else {
                c->gvx[g] = 2.0 * vwx - Svx / SW;
                c->gvy[g] = 2.0 * vwy - Svy / SW;
            }
        } else {
            c->gp[g] = 0.0;
            c->grho[g] = c->P.rho0;
            c->gvx[g] = vwx;
            c->gvy[g] = vwy;
        }
    }
}

/* Interaction operator L (Section "Governing Equations"; continuity route of
 * reading R3).  For fluid i over its neighbours j (fluid or ghost):
 *   D rho_i = sum m_j v_ij . grad_i W_ij                               (R3)
 *   closure 1 instead (reading P5, the internal-energy equation that goes
 *   with the momentum equation's pair terms):
 *   D e_i = 1/2 sum m_j (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) v_ij . grad_i W_ij
 *   a_i = - sum m_j (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) grad_i W_ij    (momentum)
 *         + sum m_j 4 nu (r_ij . grad_i W_ij) / ((rho_i + rho_j)(r^2 + eta^2 h^2)) v_ij
 *                                                    (laminar term, reading R7)
 *         + g                                                       (R8)
 *   Pi_ij = -alpha cbar mu / rhobar if v_ij . r_ij < 0 else 0,
 *   mu = h v_ij . r_ij / (r^2 + eta^2 h^2)            (artificial viscosity, R5-R6)
 *   X_i = sum_{j fluid} (m_j / rhobar_ij) (v_j - v_i) W_ij            (XSPH, R9)
 * Also gathers the pair forces exerted by ghosts for the wall impulse and the
 * boundary work (R16, R17) and the artificial-viscosity power (dissipation). */
static void interaction_operator(orc_case *c)
{
    const double h = c->h, eh2 = c->P.eta2 * h * h;
    double Fdx = 0, Fdy = 0, Fw = 0, diss = 0;
    for (int64_t i = 0; i < c->nf; ++i) {
        c->ax[i] = c->ay[i] = c->drho[i] = c->Xx[i] = c->Xy[i] = 0.0;
        c->aavx[i] = c->aavy[i] = 0.0;
        c->de[i] = 0.0;
        if (c->out[i]) continue;
        double rhoi = c->rhoh[i], Pi_ = c->p[i] / (rhoi * rhoi), ci = sound_speed(c, rhoi);
        double ax = 0, ay = 0, dr = 0, Xx = 0, Xy = 0, avx = 0, avy = 0, de = 0;
        for (int64_t a = c->nb_off[i]; a < c->nb_off[i + 1]; ++a) {
            int64_t j = c->nb_id[a];
            int ghost = j >= c->nf;
            int64_t g = j - c->nf;
            double xj = ghost ? c->gx[g] : c->x[j], yj = ghost ? c->gy[g] : c->y[j];
            double vxj = ghost ? c->gvx[g] : c->vhx[j], vyj = ghost ? c->gvy[g] : c->vhy[j];
            double rhoj = ghost ? c->grho[g] : c->rhoh[j];
            double pj = ghost ? c->gp[g] : c->p[j];
            double mj = ghost ? c->gm[g] : c->m;
            double rx = c->x[i] - xj, ry = c->y[i] - yj;
            double r2 = rx * rx + ry * ry, r = sqrt(r2);
            double F = kernel_F(c, r);
            double vx = c->vhx[i] - vxj, vy = c->vhy[i] - vyj;
            double vr = vx * rx + vy * ry;
            /* continuity */
            dr += mj * vr * F;
            /* artificial viscosity */
            double Pij = 0.0;
            int compress = (c->P.mutation & MUT_AV_SIGN) ? vr > 0.0 : vr < 0.0;
            if (compress) {
                double mu = h * vr / (r2 + eh2);
                double cbar = (c->P.mutation & MUT_AV_CONST_C)
                                  ? c->P.c0 : 0.5 * (ci + sound_speed(c, rhoj));
                double rhobar = 0.5 * (rhoi + rhoj);
                Pij = -c->P.alpha * cbar * mu / rhobar;
            }
            double Pj = (c->P.mutation & MUT_DROP_PJ) ? 0.0 : pj / (rhoj * rhoj);
            /* internal energy (closure 1) */
            double half_e = (c->P.mutation & MUT_ENERGY_HALF) ? 1.0 : 0.5;
            de += half_e * mj * (Pi_ + Pj + Pij) * F * vr;
            double fx = -mj * (Pi_ + Pj + Pij) * F * rx;
            double fy = -mj * (Pi_ + Pj + Pij) * F * ry;
            /* laminar viscosity */
            double lam = mj * ((c->P.mutation & MUT_LAM_HALF) ? 2.0 : 4.0) * c->nu * (F * r2) /
                         ((rhoi + rhoj) * (r2 + eh2));
            fx += lam * vx;
            fy += lam * vy;
            ax += fx;
            ay += fy;
            avx += -mj * Pij * F * rx;
            avy += -mj * Pij * F * ry;
            if (!ghost) {
                double wij = (c->P.mutation & MUT_XSPH_GRADW) ? -F * r : kernel_W(c, r);
                double rhobar = (c->P.mutation & MUT_XSPH_RHOJ) ? rhoj : 0.5 * (rhoi + rhoj);
                Xx += (mj / rhobar) * (vxj - c->vhx[i]) * wij;
                Xy += (mj / rhobar) * (vyj - c->vhy[i]) * wij;
            } else if (c->gkind[g] == KIND_DISK) {
                Fdx += c->m * fx;
                Fdy += c->m * fy;
            } else if (c->gkind[g] == KIND_SIDE) {
                /* force on the wall ghost by particle i is -m_i f; project on
                 * the wall's outward normal */
                Fw += -(c->m * fx) * c->gnx[g] - (c->m * fy) * c->gny[g];
            }
        }
        c->ax[i] = ax + c->P.gx;
        c->ay[i] = ay + c->P.gy;
        c->drho[i] = c->P.closure == 1 ? 0.0 : dr;
        c->de[i] = c->P.closure == 1 ? de : 0.0;
        c->Xx[i] = Xx;
        c->Xy[i] = Xy;
        c->aavx[i] = avx;
        c->aavy[i] = avy;
        diss += -c->m * (c->vhx[i] * avx + c->vhy[i] * avy);
    }
    c->Fdx = Fdx;
    c->Fdy = Fdy;
    c->Fwall = Fw;
    c->diss_rate = diss;
}

/* Summation density (Section "Density Summation", eq. density-sum; closure
 * 1): rho_i = sum_j m_j W_ij over the particle itself and its fluid and ghost
 * neighbours (the ghosts complete the sum near a boundary, Section "The
 * Projectile"), then the band [rho_lo, rho_hi] rho0.  A frozen particle keeps
 * its density. */
static void summation_density(orc_case *c)
{
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) { c->rhoh[i] = c->rho[i]; continue; }
        double rho = (c->P.mutation & MUT_SUM_NO_SELF) ? 0.0 : c->m * kernel_W(c, 0.0);
        for (int64_t a = c->nb_off[i]; a < c->nb_off[i + 1]; ++a) {
            int64_t j = c->nb_id[a];
            int ghost = j >= c->nf;
            double xj = ghost ? c->gx[j - c->nf] : c->x[j];
            double yj = ghost ? c->gy[j - c->nf] : c->y[j];
            double mj = ghost ? c->gm[j - c->nf] : c->m;
            double rx = c->x[i] - xj, ry = c->y[i] - yj;
            rho += mj * kernel_W(c, sqrt(rx * rx + ry * ry));
        }
        c->rho[i] = clamp_rho(c, rho);
        c->rhoh[i] = c->rho[i];
    }
}

/* Pressure of fluid particle i at its end-of-step state. */
static double fluid_p(const orc_case *c, int64_t i)
{
    return c->P.closure == 1 ? mg_p(c, c->rho[i], c->e[i]) : eos_p(c, c->rho[i]);
}

/* Probe value (reading R13): the wall-ghost formula (a = 0, body-force term
 * kept, cutoff applied) evaluated at the probe point over its fluid
 * neighbours with the end-of-step state. */
static double probe_value(orc_case *c, double px, double py)
{
    float pxf = (float)px, pyf = (float)py;
    double SW = 0, Sp = 0, Srx = 0, Sry = 0;
    for (int64_t j = 0; j < c->nf; ++j) {
        if (c->out[j]) continue;
        if (!predicate32(pxf, pyf, (float)c->x[j], (float)c->y[j], c->s2f)) continue;
        double rx = px - c->x[j], ry = py - c->y[j];
        double Wj = kernel_W(c, sqrt(rx * rx + ry * ry));
        SW += Wj;
        Sp += fluid_p(c, j) * Wj;
        Srx += c->rho[j] * rx * Wj;
        Sry += c->rho[j] * ry * Wj;
    }
    if (SW <= 0.0) return 0.0;
    double v = (Sp + c->P.gx * Srx + c->P.gy * Sry) / SW;
    if (c->P.mutation & MUT_GHOST_PRINTED_SIGN) v = (Sp - c->P.gx * Srx - c->P.gy * Sry) / SW;
    return v > c->P.p_cav ? v : c->P.p_cav;
}

/* CFL gate (Section "Time Integration", eq. for Delta t, and Section "GPU
 * Implementation": v_max over all particles including the ghosts):
 *   dt = C h / (c0 + v_max);  dt_mode 1 fixes v_max = v0 (reading R19). */
static double cfl_dt(orc_case *c)
{
    if (c->P.dt_mode == 1) return c->P.cfl * c->h / (c->P.c0 + c->P.v0);
    double vmax = 0.0;
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) continue;
        double v = sqrt(c->vx[i] * c->vx[i] + c->vy[i] * c->vy[i]);
        if (v > vmax) vmax = v;
    }
    if (!(c->P.mutation & MUT_DT_NO_GHOSTS))
        for (int64_t g = 0; g < c->ngh; ++g) {
            if (c->gout[g]) continue;
            double v = sqrt(c->gvx[g] * c->gvx[g] + c->gvy[g] * c->gvy[g]);
            if (v > vmax) vmax = v;
        }
    return c->P.cfl * c->h / (c->P.c0 + vmax);
}

/* p and the half-step copies used by G and L when no drift precedes them. */
static void take_half_state_as_current(orc_case *c)
{
    for (int64_t i = 0; i < c->nf; ++i) {
        c->vhx[i] = c->vx[i];
        c->vhy[i] = c->vy[i];
        c->rhoh[i] = clamp_rho(c, c->rho[i]);
        c->p[i] = eos_p(c, c->rhoh[i]);
    }
}

/* ------------------------------------------------------------- lifecycle */

void orc_destroy(orc_case *c);

orc_case *orc_create(const orc_params *P, int64_t nf, const double *xy, const double *vel,
                     const double *rho)
{
    orc_case *c = (orc_case *)calloc(1, sizeof(orc_case));
    c->P = *P;
    c->h = P->h_over_dx * P->dx;
    c->s = 2.0 * c->h;
    c->s2f = (float)(c->s * c->s);
    c->m = P->rho0 * P->dx * P->dx;
    c->alpha_d = 7.0 / (4.0 * M_PI * c->h * c->h);
    if (P->mutation & MUT_KERNEL_NORM) c->alpha_d = 10.0 / (7.0 * M_PI * c->h * c->h);
    c->B = P->rho0 * P->c0 * P->c0 / P->gamma;
    c->nu = P->mu_lam / P->rho0;
    /* computational box: outside it a point is frozen and takes part in nothing */
    double padx, pady;
    if (P->box_pad > 0.0) padx = pady = P->box_pad;
    else {
        padx = 0.5 * P->Lx;
        pady = P->wall_layers > 0 ? (P->wall_layers + 2) * P->dx + c->s : 0.5 * P->W;
        if (P->end_walls && P->wall_layers > 0) padx = (P->wall_layers + 2) * P->dx + c->s;
    }
    c->x_lo = -padx;
    c->x_hi = P->Lx + padx;
    c->y_lo = -0.5 * P->W - pady;
    c->y_hi = 0.5 * P->W + pady;

    c->nf = nf;
    size_t sz = (size_t)(nf > 0 ? nf : 1) * sizeof(double);
    double **arrs[] = {&c->x, &c->y, &c->vx, &c->vy, &c->rho, &c->ax, &c->ay, &c->drho,
                       &c->Xx, &c->Xy, &c->vhx, &c->vhy, &c->rhoh, &c->p, &c->aavx, &c->aavy,
                       &c->drho_prev, &c->e, &c->eh, &c->de, &c->vkx, &c->vky};
    for (size_t k = 0; k < sizeof arrs / sizeof arrs[0]; ++k) *arrs[k] = (double *)calloc(1, sz);
    c->out = (unsigned char *)calloc((size_t)(nf > 0 ? nf : 1), 1);
    for (int64_t i = 0; i < nf; ++i) {
        c->x[i] = xy[2 * i];
        c->y[i] = xy[2 * i + 1];
        c->vx[i] = vel ? vel[2 * i] : 0.0;
        c->vy[i] = vel ? vel[2 * i + 1] : 0.0;
        c->rho[i] = rho ? rho[i] : P->rho0;
        c->out[i] = !in_box(c, c->x[i], c->y[i]);
    }
    c->nw = make_walls(c, 1);
    c->nd = P->Ng > 0 ? P->Ng : 0;
    c->ngh = c->nw + c->nd;
    size_t gs = (size_t)(c->ngh > 0 ? c->ngh : 1);
    double **garr[] = {&c->gx, &c->gy, &c->gnx, &c->gny, &c->gm, &c->gp, &c->grho, &c->gvx, &c->gvy};
    for (size_t k = 0; k < sizeof garr / sizeof garr[0]; ++k)
        *garr[k] = (double *)calloc(gs, sizeof(double));
    c->gkind = (int32_t *)calloc(gs, sizeof(int32_t));
    c->gout = (unsigned char *)calloc(gs, 1);
    make_walls(c, 0);
    c->doffx = (double *)calloc((size_t)(c->nd > 0 ? c->nd : 1), sizeof(double));
    c->doffy = (double *)calloc((size_t)(c->nd > 0 ? c->nd : 1), sizeof(double));
    for (int64_t k = 0; k < c->nd; ++k) {
        double th = 2.0 * M_PI * (double)k / (double)c->nd;
        c->doffx[k] = P->R_disk * cos(th);
        c->doffy[k] = P->R_disk * sin(th);
        int64_t g = c->nw + k;
        c->gkind[g] = KIND_DISK;
        c->gm[g] = P->rho0 * P->dx * (2.0 * M_PI * P->R_disk / (double)c->nd);
    }
    c->hist_cap = 0;
    c->t = 0.0;
    c->step = 0;
    kinematics_now(c);
    place_disk(c);
    return c;
}

void orc_destroy(orc_case *c)
{
    if (!c) return;
    double *arrs[] = {c->x, c->y, c->vx, c->vy, c->rho, c->ax, c->ay, c->drho, c->Xx, c->Xy,
                      c->vhx, c->vhy, c->rhoh, c->p, c->aavx, c->aavy, c->drho_prev, c->e, c->eh,
                      c->de, c->vkx, c->vky, c->gx, c->gy, c->gnx,
                      c->gny, c->gm, c->gp, c->grho, c->gvx, c->gvy, c->doffx, c->doffy,
                      c->probe_hist, c->probe_t, c->probe_imp};
    for (size_t k = 0; k < sizeof arrs / sizeof arrs[0]; ++k) free(arrs[k]);
    free(c->out); free(c->gkind); free(c->gout); free(c->nb_off); free(c->nb_id);
    free(c);
}

static void record_probes(orc_case *c)
{
    if (c->P.n_probes <= 0) return;
    if (c->hist_n >= c->hist_cap) {
        c->hist_cap = c->hist_cap ? 2 * c->hist_cap : 256;
        c->probe_hist = (double *)realloc(c->probe_hist,
                                          (size_t)(c->hist_cap * c->P.n_probes) * sizeof(double));
        c->probe_t = (double *)realloc(c->probe_t, (size_t)c->hist_cap * sizeof(double));
    }
    if (!c->probe_imp) c->probe_imp = (double *)calloc((size_t)c->P.n_probes, sizeof(double));
    for (int k = 0; k < c->P.n_probes; ++k) {
        double v = probe_value(c, c->P.probe_xy[2 * k], c->P.probe_xy[2 * k + 1]);
        c->probe_hist[c->hist_n * c->P.n_probes + k] = v;
        c->probe_imp[k] += c->dt * v;
    }
    c->probe_t[c->hist_n] = c->t;
    c->hist_n++;
}

/* Evaluates G and L on the current state without advancing time (the
 * initial a^0, D rho^0, X^0 of reading R10) and sets dt from the CFL gate. */
void orc_prime(orc_case *c)
{
    kinematics_now(c);
    place_disk(c);
    for (int64_t i = 0; i < c->nf; ++i) {
        c->rho[i] = clamp_rho(c, c->rho[i]);
        c->out[i] = c->out[i] || !in_box(c, c->x[i], c->y[i]);
    }
    if (c->P.closure == 1) {
        /* the density is a function of the positions: the summation replaces
         * the given density; the internal energy starts at zero */
        for (int64_t i = 0; i < c->nf; ++i) {
            c->vhx[i] = c->vx[i];
            c->vhy[i] = c->vy[i];
            c->eh[i] = c->e[i];
        }
        build_neighbours(c);
        summation_density(c);
        for (int64_t i = 0; i < c->nf; ++i) c->p[i] = mg_p(c, c->rhoh[i], c->eh[i]);
    } else {
        take_half_state_as_current(c);
        build_neighbours(c);
    }
    ghost_operator(c);
    interaction_operator(c);
    for (int64_t i = 0; i < c->nf; ++i) c->drho_prev[i] = c->drho[i];
    c->dt = cfl_dt(c);
    c->dt_prev = c->dt;
}

/* One step U^{n+1} = T(L(G(U^n))) (Section "Numerical Provenance"): the
 * velocity Stormer-Verlet (kick-drift-kick) step of Section "Time
 * Integration" with the continuity density of reading R3.
 *
 * Reading R10 (integrator with a continuity density).  The paper's own
 * density is a function of the positions (summation), so its kick-drift-kick
 * step needs one interaction pass.  With the continuity density a pass gives
 * a (from rho) and D rho (from v) at the same time; half-kicking rho like v
 * would integrate the acoustic pair (rho, v) with forward Euler, which is
 * unstable (amplification sqrt(1 + (omega dt)^2) per step).  Here the density
 * is advanced with the freshly computed D rho (which uses the drift velocity
 * v^{n+1/2}), and the pressure fed to the pass comes from a predicted density
 *     rho~^{n+1} = rho^n + dt^n (D^n + (dt^n / dt^{n-1}) (D^n - D^{n-1})),
 * the linear extrapolation of the two previous D rho.  The scheme is second
 * order and linearly stable for omega dt below about 0.7.
 *   (1) v^{n+1/2} = v^n + dt/2 a^n
 *   (2) r^{n+1} = r^n + dt (v^{n+1/2} + eps X^n); wall enforcement (R14)
 *   (3) t^{n+1} = t^n + dt; projectile kinematics at t^{n+1}
 *   (4) rho~^{n+1} as above (density band applied); ghosts G from
 *       (r^{n+1}, v^{n+1/2}, p(rho~^{n+1}))
 *   (5) interaction sums L on (r^{n+1}, v^{n+1/2}, rho~^{n+1}) -> a, D rho, X
 *   (6) rho^{n+1} = band(rho^n + dt D rho^{n+1}); v^{n+1} = v^{n+1/2} + dt/2 a^{n+1}
 *   (7) dt^{n+1} from the CFL gate over fluid and ghosts. */
static void drift_and_walls(orc_case *c, double dt);
static void close_step(orc_case *c, double dt);

static void step_continuity(orc_case *c)
{
    const double dt = c->dt, half = 0.5 * dt;
    const double ratio = c->dt_prev > 0.0 ? dt / c->dt_prev : 1.0;
    /* (1) opening half kick of the velocity */
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) { c->vhx[i] = c->vx[i]; c->vhy[i] = c->vy[i]; continue; }
        c->vhx[i] = c->vx[i] + half * c->ax[i];
        c->vhy[i] = c->vy[i] + half * c->ay[i];
    }
    /* (2) drift with the XSPH velocity, then wall enforcement (reading R14) */
    drift_and_walls(c, dt);
    /* (3) time and projectile kinematics at t^{n+1} */
    c->t += dt;
    kinematics_advance(c, dt);
    place_disk(c);
    /* (4) predicted density and its pressure, then the ghosts */
    for (int64_t i = 0; i < c->nf; ++i) {
        double Dp = c->drho[i] + ratio * (c->drho[i] - c->drho_prev[i]);
        c->rhoh[i] = c->out[i] ? c->rho[i] : clamp_rho(c, c->rho[i] + dt * Dp);
        c->p[i] = eos_p(c, c->rhoh[i]);
        c->drho_prev[i] = c->drho[i];
    }
    build_neighbours(c);
    ghost_operator(c);
    /* (5) interaction sums */
    interaction_operator(c);
    /* (6) density with the new D rho, closing half kick */
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) {
            c->ax[i] = c->ay[i] = c->drho[i] = c->Xx[i] = c->Xy[i] = 0.0;
            continue;
        }
        c->rho[i] = clamp_rho(c, c->rho[i] + dt * c->drho[i]);
        c->vx[i] = c->vhx[i] + half * c->ax[i];
        c->vy[i] = c->vhy[i] + half * c->ay[i];
    }
    close_step(c, dt);
}

static void drift_and_walls(orc_case *c, double dt)
{
    const double W2 = 0.5 * c->P.W, eps = 1e-6;
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) continue;
        c->x[i] += dt * (c->vhx[i] + c->P.eps_xsph * c->Xx[i]);
        c->y[i] += dt * (c->vhy[i] + c->P.eps_xsph * c->Xy[i]);
        if (c->P.wall_layers > 0 || c->P.wall_reflect) {
            if (c->y[i] > W2) { c->y[i] = W2 - eps; c->vhy[i] = -c->vhy[i]; }
            else if (c->y[i] < -W2) { c->y[i] = -W2 + eps; c->vhy[i] = -c->vhy[i]; }
            if (c->P.end_walls) {
                if (c->x[i] > c->P.Lx) { c->x[i] = c->P.Lx - eps; c->vhx[i] = -c->vhx[i]; }
                else if (c->x[i] < 0.0) { c->x[i] = eps; c->vhx[i] = -c->vhx[i]; }
            }
        }
        if (!in_box(c, c->x[i], c->y[i])) c->out[i] = 1;
    }
}

/* Closure 1 (reading P6): the paper's kick-drift-kick step with the
 * summation density, one interaction pass per step.  The pass sees the state
 * predicted at t^{n+1}: velocities v* = v^{n+1/2} + dt/2 a^n and energies
 * e* = e^n + dt De^n, so that the velocity-dependent terms (artificial
 * viscosity, the energy equation) are centred where the forces are; with
 * v^{n+1/2} instead, the kinetic plus internal energy would drift by
 * dt^2/2 sum m |a|^2 every step (first order overall).
 *   (1) v^{n+1/2} = v^n + dt/2 a^n
 *   (2) r^{n+1} = r^n + dt (v^{n+1/2} + eps X^n); wall enforcement (R14)
 *   (3) t^{n+1}; projectile kinematics at t^{n+1}
 *   (4) rho^{n+1} = band(sum_j m_j W_ij(r^{n+1})); v* and e* as above;
 *       p = MG(rho^{n+1}, e*); ghosts G from (r^{n+1}, v*, p)
 *   (5) interaction sums L on (r^{n+1}, v*, rho^{n+1}, p) -> a^{n+1}, De^{n+1}, X^{n+1}
 *   (6) v^{n+1} = v^{n+1/2} + dt/2 a^{n+1},  e^{n+1} = e^n + dt/2 (De^n + De^{n+1})
 *   (7) dt^{n+1} from the CFL gate. */
static void step_summation(orc_case *c)
{
    const double dt = c->dt, half = 0.5 * dt;
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) {
            c->vhx[i] = c->vx[i];
            c->vhy[i] = c->vy[i];
            continue;
        }
        c->vhx[i] = c->vx[i] + half * c->ax[i];
        c->vhy[i] = c->vy[i] + half * c->ay[i];
    }
    drift_and_walls(c, dt);
    c->t += dt;
    kinematics_advance(c, dt);
    place_disk(c);
    build_neighbours(c);
    summation_density(c);
    for (int64_t i = 0; i < c->nf; ++i) {
        c->vkx[i] = c->vhx[i];
        c->vky[i] = c->vhy[i];
        if (c->out[i]) {
            c->eh[i] = c->e[i];
        } else {
            c->vhx[i] += half * c->ax[i];
            c->vhy[i] += half * c->ay[i];
            c->eh[i] = c->e[i] + dt * c->de[i];
        }
        c->p[i] = mg_p(c, c->rhoh[i], c->eh[i]);
    }
    ghost_operator(c);
    double *de_old = (double *)malloc((size_t)(c->nf > 0 ? c->nf : 1) * sizeof(double));
    memcpy(de_old, c->de, (size_t)c->nf * sizeof(double));
    interaction_operator(c);
    for (int64_t i = 0; i < c->nf; ++i) {
        if (c->out[i]) {
            c->vx[i] = c->vkx[i];
            c->vy[i] = c->vky[i];
            c->ax[i] = c->ay[i] = c->de[i] = c->Xx[i] = c->Xy[i] = 0.0;
            continue;
        }
        c->vx[i] = c->vkx[i] + half * c->ax[i];
        c->vy[i] = c->vky[i] + half * c->ay[i];
        c->e[i] += half * (de_old[i] + c->de[i]);
    }
    free(de_old);
    close_step(c, dt);
}

/* Accumulators, probes and the CFL gate at the end of a step. */
static void close_step(orc_case *c, double dt)
{
    /* accumulated boundary work, wall impulse, dissipation (R16, R17) */
    c->Wb += dt * (c->Fdx * c->vproj);
    c->impulse += dt * c->Fwall;
    c->diss += dt * c->diss_rate;
    c->step++;
    /* probes on the end-of-step state, then (7) the CFL gate */
    record_probes(c);
    c->dt_prev = dt;
    c->dt = cfl_dt(c);
}

void orc_step(orc_case *c)
{
    if (c->P.closure == 1) step_summation(c);
    else step_continuity(c);
}

void orc_run(orc_case *c, int64_t n)
{
    for (int64_t k = 0; k < n; ++k) orc_step(c);
}

/* -------------------------------------------------------------- getters */

int64_t orc_n_fluid(const orc_case *c) { return c->nf; }
int64_t orc_n_wall(const orc_case *c) { return c->nw; }
int64_t orc_n_disk(const orc_case *c) { return c->nd; }

void orc_get_fluid(const orc_case *c, double *xy, double *vel, double *rho, double *p,
                   double *acc, double *drho, double *X, unsigned char *out)
{
    for (int64_t i = 0; i < c->nf; ++i) {
        if (xy) { xy[2 * i] = c->x[i]; xy[2 * i + 1] = c->y[i]; }
        if (vel) { vel[2 * i] = c->vx[i]; vel[2 * i + 1] = c->vy[i]; }
        if (rho) rho[i] = c->rho[i];
        if (p) p[i] = fluid_p(c, i);
        if (acc) { acc[2 * i] = c->ax[i]; acc[2 * i + 1] = c->ay[i]; }
        if (drho) drho[i] = c->drho[i];
        if (X) { X[2 * i] = c->Xx[i]; X[2 * i + 1] = c->Xy[i]; }
        if (out) out[i] = c->out[i];
    }
}

void orc_get_energy(const orc_case *c, double *e, double *de)
{
    for (int64_t i = 0; i < c->nf; ++i) {
        if (e) e[i] = c->e[i];
        if (de) de[i] = c->de[i];
    }
}

void orc_get_ghosts(const orc_case *c, double *xy, double *p, double *rho, double *vel,
                    double *mass, int32_t *kind, unsigned char *out)
{
    for (int64_t g = 0; g < c->ngh; ++g) {
        if (xy) { xy[2 * g] = c->gx[g]; xy[2 * g + 1] = c->gy[g]; }
        if (p) p[g] = c->gp[g];
        if (rho) rho[g] = c->grho[g];
        if (vel) { vel[2 * g] = c->gvx[g]; vel[2 * g + 1] = c->gvy[g]; }
        if (mass) mass[g] = c->gm[g];
        if (kind) kind[g] = c->gkind[g];
        if (out) out[g] = c->gout[g];
    }
}

/* scalars: t, dt, step, xc, yc, vproj, aproj, Fdisk_x, Fdisk_y, Fwall,
 *          Wb, impulse, diss, diss_rate */
void orc_get_scalars(const orc_case *c, double *s)
{
    s[0] = c->t; s[1] = c->dt; s[2] = (double)c->step; s[3] = c->xc; s[4] = c->yc;
    s[5] = c->vproj; s[6] = c->aproj; s[7] = c->Fdx; s[8] = c->Fdy; s[9] = c->Fwall;
    s[10] = c->Wb; s[11] = c->impulse; s[12] = c->diss; s[13] = c->diss_rate;
}

int64_t orc_probe_history(const orc_case *c, double *p, double *t, int64_t cap)
{
    int64_t n = c->hist_n < cap ? c->hist_n : cap;
    if (p) memcpy(p, c->probe_hist, (size_t)(n * c->P.n_probes) * sizeof(double));
    if (t) memcpy(t, c->probe_t, (size_t)n * sizeof(double));
    return c->hist_n;
}

/* Neighbour lists of the current state (as of the last prime/step). */
int64_t orc_neighbours(const orc_case *c, int64_t *off, int32_t *ids, int64_t cap)
{
    int64_t np = c->nf + c->ngh, n = c->nb_off ? c->nb_off[np] : 0;
    if (off && c->nb_off) memcpy(off, c->nb_off, (size_t)(np + 1) * sizeof(int64_t));
    if (ids && n <= cap) memcpy(ids, c->nb_id, (size_t)n * sizeof(int32_t));
    return n;
}

/* Rebuild the neighbour lists for the current positions (no physics). */
void orc_refresh_neighbours(orc_case *c) { build_neighbours(c); }

/* Diagnostics in FP64 (the paper logs mass and mechanical energy; readings
 * R16-R18 add the impulse, boundary work and Tait elastic energy; with
 * closure 1, E_el is the internal energy sum m e of the energy equation):
 *  0 mass  1 px  2 py  3 KE  4 PE  5 E_el  6 rho_min  7 rho_max  8 p_min
 *  9 p_max 10 vmax_fluid 11 n_in 12 penetrated 13 t 14 dt 15 Wb 16 impulse
 * 17 diss 18 step */
void orc_diagnostics(const orc_case *c, double *d)
{
    double mass = 0, px = 0, py = 0, ke = 0, pe = 0, eel = 0, rmin = 1e300, rmax = -1e300;
    double pmin = 1e300, pmax = -1e300, vmax = 0;
    int64_t nin = 0, pen = 0;
    for (int64_t i = 0; i < c->nf; ++i) {
        mass += c->m;
        if (c->out[i]) continue;
        nin++;
        double v2 = c->vx[i] * c->vx[i] + c->vy[i] * c->vy[i];
        px += c->m * c->vx[i];
        py += c->m * c->vy[i];
        ke += 0.5 * c->m * v2;
        pe += -c->m * (c->P.gx * c->x[i] + c->P.gy * c->y[i]);
        eel += c->m * (c->P.closure == 1 ? c->e[i] : tait_energy(c, c->rho[i]));
        double pr = fluid_p(c, i);
        if (c->rho[i] < rmin) rmin = c->rho[i];
        if (c->rho[i] > rmax) rmax = c->rho[i];
        if (pr < pmin) pmin = pr;
        if (pr > pmax) pmax = pr;
        if (sqrt(v2) > vmax) vmax = sqrt(v2);
        if (c->nd > 0) {
            double dx = c->x[i] - c->xc, dy = c->y[i] - c->yc;
            if (dx * dx + dy * dy < c->P.R_disk * c->P.R_disk) pen++;
        }
    }
    d[0] = mass; d[1] = px; d[2] = py; d[3] = ke; d[4] = pe; d[5] = eel;
    d[6] = rmin; d[7] = rmax; d[8] = pmin; d[9] = pmax; d[10] = vmax;
    d[11] = (double)nin; d[12] = (double)pen; d[13] = c->t; d[14] = c->dt;
    d[15] = c->Wb; d[16] = c->impulse; d[17] = c->diss; d[18] = (double)c->step;
}

/* Brute-force neighbour sets of an arbitrary float point set under the R2
 * predicate: CSR over all points, ids ascending.  Returns the pair count;
 * writes ids only when cap suffices. */
int64_t orc_brute_neighbours(int64_t n, const float *xy, float s2, int64_t *off, int32_t *ids,
                             int64_t cap)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        off[i] = k;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (predicate32(xy[2 * i], xy[2 * i + 1], xy[2 * j], xy[2 * j + 1], s2)) {
                if (k < cap) ids[k] = (int32_t)j;
                ++k;
            }
        }
    }
    off[n] = k;
    return k;
}
