/*
 * FP64 CPU oracle for the double-distribution lattice Boltzmann model of two-phase Darcy
 * flow (Chai, Liang, Du, Shi, arXiv 1808.07554).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the GPU solver
 * is checked against.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg may load it; the solver library never does.  It shares no code, header
 * or table with the CUDA sources.
 *
 * Every step is written as a separate plain loop over nodes, in the paper's order and
 * notation, in IEEE double precision (compiled without fast-math and without FMA
 * contraction).  All nine pressure populations are kept, including f_0.
 *
 * Lattice units inside: spacing 1, step 1.  D2Q9 (Eqs. 3-5, 3-5a, 3-6, 3-6a):
 *   c_i = (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)
 *   omega = 4/9, 1/9 (x4), 1/36 (x4);  omega_bar = 0, 1/8 (x8);  c_s^2 = 1/3.
 * Nodes are cell centred; walls lie half-way between a boundary node and its missing
 * neighbour (link-wise boundary rules of Sec. 4).
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - pressure pseudo-time scale s (time/length^2): tau_f = 1/2 + 3 s D_p, source
 *    weight s dx^2 F_p.  PHYSICAL_DT mode: s = dt/dx^2 (pseudo-step = physical step).
 *    REFERENCE mode: s = (tau_p - 1/2) / (3 D_ref), D_ref the geometric mean of D_p
 *    over the grid at t = 0 unless given.
 *  - sub-iteration stop (Sec. 3, "iterated to a steady state"): every m-th sweep k,
 *    r_k = ||dP - mean dP||_2 / ||P^k - mean P^k||_2 with dP = P^k - P^{k-1};
 *    stop when r_k <= tol, or at max_sub_iters (not converged).
 *  - continuation: each physical step starts the pressure iteration from the previous
 *    step's populations; at t = 0 from f = f_eq(P_0).
 *  - wells: a point rate q at one node is a source q/dx^2 there; the producer's
 *    saturation source uses the water fraction at S* = sum_i g_i / phi.
 *  - the initial saturation gradient (Eq. gneq) is a second-order central difference
 *    (mirror at no-flux walls, wrap when periodic, one-sided at Dirichlet walls).
 *  - D2Q5 saturation lattice (Remark V, Eq. 3-4b): weights omega_0 = 1/3, omega_1..4 =
 *    1/6 (c_s^2 = 1/3, the paper gives none); the collision, the walls and Eq. gneq keep
 *    their D2Q9 form with these weights and Gamma_i.
 *  - saturation-dependent D_s (Remark IV): with a linear capillary pressure
 *    P_c = p_e (1 - S), Eq. 2-16 gives D_s = K lambda_n f_w p_e = p_e K lambda_w lambda_n /
 *    lambda_t; the model uses D_s(x, S) = D_s + D_c K lambda_w lambda_n / lambda_t
 *    (D_c = p_e; D_c = 0 is the constant case), so tau_g varies per node (Eq. 3-11b).
 *  - warm start (optional): before a step's pressure solve the equilibrium part of f moves
 *    by f^eq(P^n - P^{n-1}) (Eq. 3-3), i.e. the iteration starts from the pressure
 *    extrapolated linearly in time, 2 P^n - P^{n-1}, with the previous non-equilibrium part
 *    kept; P^n is the pressure of the last pull of step n.  The fixed point of every solve
 *    is unchanged; only the starting iterate moves.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOTCONVERGED 4
#define ORC_ENONFINITE 5

enum { PERIODIC = 0, NOFLUX = 1, DIRICHLET = 2 };
enum { XMIN = 0, XMAX = 1, YMIN = 2, YMAX = 3 };
enum { MOB_QUADRATIC = 0, MOB_DECOUPLED = 1, MOB_RATIONAL = 2 };
enum { TAU_REFERENCE = 0, TAU_PHYSICAL_DT = 1 };

/* D2Q9 velocity set, Eq. 3-6 with c = 1 */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* opposite direction: c_opp(i) = -c_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

typedef struct orc {
    int nx, ny;
    size_t n;
    double dx, dt, phi, beta, mu_w, mu_n, D_s;
    int mobility, tau_mode;
    double tau_p, D_ref, s, tau_g;
    double tol;
    int max_sub, check_every;
    int bc[4];
    double w[9], wbar[9], Gam[9];      /* Eq. 3-5, 3-5a; Gamma_i = g_i^eq / S (Sec. 4) */
    int qs;                            /* saturation lattice: 9 (D2Q9) or 5 (D2Q5) */
    double wg[9];                      /* weights of the saturation lattice */
    double D_c;                        /* capillary part of D_s (Remark IV) */
    double *K;
    double *f[9], *fpre[9];            /* post-collision f_i^+, pulled (pre-collision) f_i */
    double *g[9], *gpre[9];
    double *tauf;                      /* per-node tau_f */
    double *Fp, *Fs;                   /* dense physical sources (may be all zero) */
    double *Fs_t;                      /* dt * F_s at the current step, wells included */
    double *S, *P, *Pprev, *gxX, *gyX; /* S^n, P from the last pull, previous-sweep P, lattice grad P */
    int warm_start;                    /* 1: start each solve from the extrapolated pressure */
    double *Pstep;                     /* P of the last pull of the previous step */
    double *Pb[4], *Sb[4];             /* Dirichlet wall traces, 2n+1 half-spaced values */
    int nw;
    int *wi, *wj, *wprod;
    double *wq;
    int step;
    double last_r;
    int last_k;
} orc;

/* ------------------------------------------------------------------------------------ */
/* constants                                                                            */
/* ------------------------------------------------------------------------------------ */
static void set_constants(orc *o)
{
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < 9; ++i) {
        int e2 = EX[i] * EX[i] + EY[i] * EY[i];
        /* Eq. 3-5 */
        o->w[i] = (i == 0) ? 4.0 / 9.0 : (e2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        /* Eq. 3-5a */
        o->wbar[i] = (i == 0) ? 0.0 : 1.0 / 8.0;
        /* Eq. 3-4: g_i^eq = omega_i S [phi + C:(c_i c_i - cs2 I)/(2 cs2)], C = (beta - phi) I,
           and C:(c_i c_i - cs2 I) = (beta - phi)(|c_i|^2 - 2 cs2) in two dimensions. */
        o->Gam[i] = o->w[i] * (o->phi + (o->beta - o->phi) * ((double)e2 - 2.0 * cs2) / (2.0 * cs2));
        o->wg[i] = o->w[i];
    }
    if (o->qs == 5) {
        /* D2Q5 (Remark V): omega_0 = 1/3, omega_1..4 = 1/6; Eq. 3-4b:
           g_0^eq = [(omega_0 - 1) beta + phi] S, g_i^eq = omega_i beta S */
        for (int i = 0; i < 9; ++i) {
            o->wg[i] = i == 0 ? 1.0 / 3.0 : (i < 5 ? 1.0 / 6.0 : 0.0);
            o->Gam[i] = i == 0 ? (o->wg[0] - 1.0) * o->beta + o->phi : o->wg[i] * o->beta;
        }
    }
}

/* mobilities lambda_w, lambda_t of the chosen law (Eq. 2-9 with k_rw = S^2, k_rn = (1-S)^2
   of Sec. 4.3; the decoupled case lambda_t = lambda_w of Sec. 4.1; Eq. 4-4 of Sec. 4.2) */
static void mobility(const orc *o, double S, double *lw, double *lt)
{
    if (o->mobility == MOB_QUADRATIC) {
        double a = S * S / o->mu_w;
        double b = (1.0 - S) * (1.0 - S) / o->mu_n;
        *lw = a;
        *lt = a + b;
    } else if (o->mobility == MOB_DECOUPLED) {
        *lw = 1.0 / o->mu_w;
        *lt = 1.0 / o->mu_w;
    } else {
        double t = 1.0 / (0.5 - 0.2 * S);
        *lw = S * t;
        *lt = t;
    }
}

static double frac_w(const orc *o, double S)
{
    double lw, lt;
    mobility(o, S, &lw, &lt);
    return lt != 0.0 ? lw / lt : 0.0;
}

/* Eq. 3-11b: D_s = beta c_s^2 (tau_g - 1/2) dt, c_s^2 = (dx/dt)^2 / 3, with
   D_s(x, S) = D_s + D_c K lambda_w lambda_n / lambda_t and lambda_n = lambda_t - lambda_w */
static double tau_g_at(const orc *o, size_t a, double S)
{
    if (o->D_c == 0.0)
        return o->tau_g;
    double lw, lt;
    mobility(o, S, &lw, &lt);
    double Ds = o->D_s + (lt != 0.0 ? o->D_c * o->K[a] * lw * (lt - lw) / lt : 0.0);
    return 0.5 + 3.0 * Ds * o->dt / (o->beta * o->dx * o->dx);
}

/* ------------------------------------------------------------------------------------ */
/* streaming with the boundary rules of Sec. 4                                          */
/* ------------------------------------------------------------------------------------ */
/* Value arriving at node (x, y) along direction i after streaming from the post-collision
   array `post`.  When x - c_i lies outside the domain the link crosses a wall:
     no-flux (bounce-back):       f_i(x_f) = f_opp^+(x_f)
     Dirichlet (anti-bounce-back): f_i(x_f) = -f_opp^+(x_f) + 2 f_opp^eq(value at the wall)
   The x-sides are tested first, so a link leaving through a corner uses the x-side rule.
   `is_g` selects the equilibrium: omega_opp P_b for f, Gamma_opp S_b for g. */
static double pull(const orc *o, double *const *post, int i, int x, int y, int is_g)
{
    int xs = x - EX[i];
    int ys = y - EY[i];
    int side = -1;
    if (xs < 0 || xs >= o->nx) {
        int sd = xs < 0 ? XMIN : XMAX;
        if (o->bc[sd] == PERIODIC)
            xs = (xs + o->nx) % o->nx;
        else
            side = sd;
    }
    if (side < 0 && (ys < 0 || ys >= o->ny)) {
        int sd = ys < 0 ? YMIN : YMAX;
        if (o->bc[sd] == PERIODIC)
            ys = (ys + o->ny) % o->ny;
        else
            side = sd;
    }
    if (side < 0)
        return post[i][(size_t)ys * o->nx + xs];
    double b = post[OPP[i]][(size_t)y * o->nx + x];
    if (o->bc[side] == NOFLUX)
        return b;
    /* half-spaced trace index of the point where the link crosses the wall */
    int k = (side == XMIN || side == XMAX) ? 2 * y + 1 - EY[i] : 2 * x + 1 - EX[i];
    double eq = is_g ? o->Gam[OPP[i]] * o->Sb[side][k] : o->w[OPP[i]] * o->Pb[side][k];
    return -b + 2.0 * eq;
}

/* Streaming of all nine populations.  A node whose eight neighbours are all inside the
   domain copies f_i^+(x - c_i) directly; every other node goes through pull(). */
static void stream(orc *o, double *const *post, double **pre, int is_g)
{
    const int nx = o->nx, ny = o->ny;
    const int q = is_g ? o->qs : 9;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t a = (size_t)y * nx + x;
            int inner = x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2;
            for (int i = 0; i < q; ++i) {
                if (inner)
                    pre[i][a] = post[i][(size_t)(y - EY[i]) * nx + (x - EX[i])];
                else
                    pre[i][a] = pull(o, post, i, x, y, is_g);
            }
        }
    }
}

static void stream_f(orc *o)
{
    stream(o, o->f, o->fpre, 0);
}

static void stream_g(orc *o)
{
    stream(o, o->g, o->gpre, 1);
}

/* ------------------------------------------------------------------------------------ */
/* macroscopic quantities                                                               */
/* ------------------------------------------------------------------------------------ */
/* Eq. 3-9a: P = sum_{i=1..8} f_i / (1 - omega_0)   (f_0 is not part of the sum) */
static void pressure_from_fpre(orc *o, double *P)
{
#pragma omp parallel for schedule(static)
    for (size_t a = 0; a < o->n; ++a) {
        double s = 0.0;
        for (int i = 1; i < 9; ++i)
            s += o->fpre[i][a];
        P[a] = s / (1.0 - o->w[0]);
    }
}

/* Eq. 3-10a in lattice units: grad_X P = -sum_i c_i f_i / (tau_f c_s^2), c_s^2 = 1/3 */
static void gradient_from_fpre(orc *o)
{
#pragma omp parallel for schedule(static)
    for (size_t a = 0; a < o->n; ++a) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < 9; ++i) {
            sx += EX[i] * o->fpre[i][a];
            sy += EY[i] * o->fpre[i][a];
        }
        o->gxX[a] = -3.0 * sx / o->tauf[a];
        o->gyX[a] = -3.0 * sy / o->tauf[a];
    }
}

/* dt * F_s at every node: the dense source plus the wells.  The injector adds q/dx^2;
   the producer removes f_w(S*) q/dx^2 with S* taken from Sstar (per node). */
static void saturation_source(orc *o, const double *Sstar)
{
    for (size_t a = 0; a < o->n; ++a)
        o->Fs_t[a] = o->dt * o->Fs[a];
    for (int m = 0; m < o->nw; ++m) {
        size_t a = (size_t)o->wj[m] * o->nx + o->wi[m];
        double q = o->wq[m] / (o->dx * o->dx);
        if (o->wprod[m])
            o->Fs_t[a] += -o->dt * frac_w(o, Sstar[a]) * q;
        else
            o->Fs_t[a] += o->dt * q;
    }
}

/* Eq. 3-9b: S = (sum_i g_i + dt F_s / 2) / phi, from the pulled g */
static void saturation_from_gpre(orc *o)
{
    double *Sstar = o->S;   /* S* = sum_i g_i / phi, overwritten below */
    for (size_t a = 0; a < o->n; ++a) {
        double s = 0.0;
        for (int i = 0; i < o->qs; ++i)
            s += o->gpre[i][a];
        Sstar[a] = s / o->phi;
    }
    saturation_source(o, Sstar);
    for (size_t a = 0; a < o->n; ++a) {
        double s = 0.0;
        for (int i = 0; i < o->qs; ++i)
            s += o->gpre[i][a];
        o->S[a] = (s + 0.5 * o->Fs_t[a]) / o->phi;
    }
}

/* Eq. 3-11a with D_p = K lambda_t(S) (Eq. 2-16) and the pseudo-time scale s:
   tau_f = 1/2 + 3 s D_p */
static void relaxation_time_f(orc *o)
{
#pragma omp parallel for schedule(static)
    for (size_t a = 0; a < o->n; ++a) {
        double lw, lt;
        mobility(o, o->S[a], &lw, &lt);
        o->tauf[a] = 0.5 + 3.0 * o->s * o->K[a] * lt;
    }
}

/* dense F_p at node a plus the wells (injector +q/dx^2, producer -q/dx^2), scaled by the
   pseudo-step: s dx^2 F_p */
static void pressure_source_field(const orc *o, double *Fp_t)
{
    for (size_t a = 0; a < o->n; ++a)
        Fp_t[a] = o->s * o->dx * o->dx * o->Fp[a];
    for (int m = 0; m < o->nw; ++m) {
        size_t a = (size_t)o->wj[m] * o->nx + o->wi[m];
        double q = o->wq[m] / (o->dx * o->dx);
        Fp_t[a] += o->s * o->dx * o->dx * (o->wprod[m] ? -q : q);
    }
}

/* ------------------------------------------------------------------------------------ */
/* collisions                                                                           */
/* ------------------------------------------------------------------------------------ */
/* Eq. 2-1b (first line) with f_i^eq of Eq. 3-3:
   f_i^+ = f_i - (f_i - f_i^eq)/tau_f + omega_bar_i dt' F_p,
   f_0^eq = (omega_0 - 1) P, f_i^eq = omega_i P (i != 0). */
static void collide_f(orc *o, const double *P, const double *Fp_t)
{
#pragma omp parallel for schedule(static)
    for (size_t a = 0; a < o->n; ++a) {
        for (int i = 0; i < 9; ++i) {
            double feq = (i == 0) ? (o->w[0] - 1.0) * P[a] : o->w[i] * P[a];
            double fi = o->fpre[i][a];
            o->f[i][a] = fi - (fi - feq) / o->tauf[a] + o->wbar[i] * Fp_t[a];
        }
    }
}

/* Eq. 2-1b (second line) with g_i^eq = Gamma_i S (Eq. 3-4) and gamma of Eq. 3-8; in
   lattice units gamma dt c_i.grad P = gamma_t c_i.grad_X P with
   gamma_t = -3 lambda_w K dt / dx^2. */
static void collide_g(orc *o)
{
#pragma omp parallel for schedule(static)
    for (size_t a = 0; a < o->n; ++a) {
        const double tg = tau_g_at(o, a, o->S[a]);
        double lw, lt;
        mobility(o, o->S[a], &lw, &lt);
        double gam_t = -3.0 * lw * o->K[a] * o->dt / (o->dx * o->dx);
        for (int i = 0; i < o->qs; ++i) {
            double geq = o->Gam[i] * o->S[a];
            double gi = o->gpre[i][a];
            double cgrad = EX[i] * o->gxX[a] + EY[i] * o->gyX[a];
            o->g[i][a] = gi - (gi - geq) / tg + o->wg[i] * (1.0 - 1.0 / (2.0 * tg)) * o->Fs_t[a]
                         + gam_t * o->wg[i] * cgrad / tg;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* pressure sub-iteration                                                               */
/* ------------------------------------------------------------------------------------ */
static double residual(const orc *o, const double *P, const double *Pprev)
{
    double md = 0.0, mp = 0.0;
    for (size_t a = 0; a < o->n; ++a) {
        md += P[a] - Pprev[a];
        mp += P[a];
    }
    md /= (double)o->n;
    mp /= (double)o->n;
    double num = 0.0, den = 0.0;
    for (size_t a = 0; a < o->n; ++a) {
        double d = (P[a] - Pprev[a]) - md;
        double p = P[a] - mp;
        num += d * d;
        den += p * p;
    }
    if (den == 0.0)
        return num == 0.0 ? 0.0 : INFINITY;
    return sqrt(num) / sqrt(den);
}

/* one sweep of Eq. 3-1: stream, P (Eq. 3-9a), optional residual, collide */
static double one_sweep(orc *o, int want_r, double *Fp_t, double *Pk)
{
    stream_f(o);
    pressure_from_fpre(o, Pk);
    double r = NAN;
    if (want_r)
        r = residual(o, Pk, o->Pprev);
    collide_f(o, Pk, Fp_t);
    memcpy(o->Pprev, Pk, o->n * sizeof(double));   /* P^{k-1} of the next sweep */
    return r;
}

/* Iterate Eq. 3-1 in pseudo time.  replay < 0: until r <= tol at a check (every
   check_every sweeps) or max_sub sweeps; replay >= 0: exactly that many sweeps (the
   residual is still evaluated on the last one when it is at least the second). */
static int pressure_solve(orc *o, int replay, int *k_out, double *r_out)
{
    double *Fp_t = malloc(o->n * sizeof(double));
    double *Pk = malloc(o->n * sizeof(double));
    if (!Fp_t || !Pk) {
        free(Fp_t);
        free(Pk);
        return ORC_ENOMEM;
    }
    pressure_source_field(o, Fp_t);
    int status = ORC_OK;
    int k = 0;
    double r = NAN;
    if (replay >= 0) {
        for (k = 1; k <= replay; ++k)
            r = one_sweep(o, k == replay && k >= 2, Fp_t, Pk);
        k = replay;
        if (isnan(r) && replay >= 2)
            status = ORC_ENONFINITE;
    } else {
        /* the residual needs a previous sweep of the same step, so checks start at k = 2 */
        for (;;) {
            ++k;
            int at_check = (k % o->check_every == 0) || (k >= o->max_sub);
            int can_r = k >= 2;
            r = one_sweep(o, at_check && can_r, Fp_t, Pk);
            if (!at_check)
                continue;
            if (can_r) {
                if (isnan(r)) {
                    status = ORC_ENONFINITE;
                    break;
                }
                if (r <= o->tol)
                    break;
            }
            if (k >= o->max_sub) {
                status = ORC_ENOTCONVERGED;
                break;
            }
        }
    }
    free(Fp_t);
    free(Pk);
    o->last_k = k;
    o->last_r = r;
    if (k_out)
        *k_out = k;
    if (r_out)
        *r_out = r;
    return status;
}

/* ------------------------------------------------------------------------------------ */
/* initial saturation gradient for Eq. gneq (central differences, lattice units)        */
/* ------------------------------------------------------------------------------------ */
static double fd_axis(const orc *o, const double *S, int x, int y, int axis)
{
    int n = axis == 0 ? o->nx : o->ny;
    int c = axis == 0 ? x : y;
    int lo_side = axis == 0 ? XMIN : YMIN;
    int hi_side = axis == 0 ? XMAX : YMAX;
#define AT(cc) (axis == 0 ? S[(size_t)y * o->nx + (cc)] : S[(size_t)(cc) * o->nx + x])
    if (c == 0 && o->bc[lo_side] == DIRICHLET)
        return (-3.0 * AT(0) + 4.0 * AT(1) - AT(2)) / 2.0;
    if (c == n - 1 && o->bc[hi_side] == DIRICHLET)
        return (3.0 * AT(n - 1) - 4.0 * AT(n - 2) + AT(n - 3)) / 2.0;
    double lo, hi;
    if (c - 1 >= 0)
        lo = AT(c - 1);
    else
        lo = o->bc[lo_side] == PERIODIC ? AT(n - 1) : AT(c);
    if (c + 1 < n)
        hi = AT(c + 1);
    else
        hi = o->bc[hi_side] == PERIODIC ? AT(0) : AT(c);
    return (hi - lo) / 2.0;
#undef AT
}

/* ------------------------------------------------------------------------------------ */
/* public entry points                                                                  */
/* ------------------------------------------------------------------------------------ */
void orc_destroy(orc *o)
{
    if (!o)
        return;
    free(o->K);
    for (int i = 0; i < 9; ++i) {
        free(o->f[i]);
        free(o->fpre[i]);
        free(o->g[i]);
        free(o->gpre[i]);
    }
    free(o->tauf);
    free(o->Fp);
    free(o->Fs);
    free(o->Fs_t);
    free(o->S);
    free(o->P);
    free(o->Pprev);
    free(o->Pstep);
    free(o->gxX);
    free(o->gyX);
    for (int s = 0; s < 4; ++s) {
        free(o->Pb[s]);
        free(o->Sb[s]);
    }
    free(o->wi);
    free(o->wj);
    free(o->wprod);
    free(o->wq);
    free(o);
}

static int trace_len(const orc *o, int side)
{
    return (side == XMIN || side == XMAX) ? 2 * o->ny + 1 : 2 * o->nx + 1;
}

int orc_set_sources(orc *o, const double *Fp, const double *Fs)
{
    for (size_t a = 0; a < o->n; ++a) {
        o->Fp[a] = Fp ? Fp[a] : 0.0;
        o->Fs[a] = Fs ? Fs[a] : 0.0;
    }
    return ORC_OK;
}

int orc_set_dirichlet(orc *o, int side, const double *Pb, const double *Sb)
{
    if (side < 0 || side > 3 || o->bc[side] != DIRICHLET)
        return ORC_EINVAL;
    int L = trace_len(o, side);
    for (int k = 0; k < L; ++k) {
        o->Pb[side][k] = Pb ? Pb[k] : 0.0;
        o->Sb[side][k] = Sb ? Sb[k] : 0.0;
    }
    return ORC_OK;
}

/* Initialisation (Sec. 4, Eqs. gini, gneq): f^+ = f^eq(P_0); tau_f from S_0; pressure
   solve; g(t=0) = Gamma_i S_0 + eps g_i^(1); then the t = 0 collision of g. */
static int initialise(orc *o, const double *P0, const double *S0, int init_replay,
                      int *k_out, double *r_out)
{
    for (size_t a = 0; a < o->n; ++a) {
        double p = P0 ? P0[a] : 0.0;
        for (int i = 0; i < 9; ++i)
            o->f[i][a] = (i == 0) ? (o->w[0] - 1.0) * p : o->w[i] * p;
        o->Pprev[a] = p;
        o->S[a] = S0[a];
    }
    /* D_ref: geometric mean of D_p at t = 0, unless given */
    if (o->tau_mode == TAU_REFERENCE) {
        double D = o->D_ref;
        if (!(D > 0.0)) {
            double acc = 0.0;
            for (size_t a = 0; a < o->n; ++a) {
                double lw, lt;
                mobility(o, S0[a], &lw, &lt);
                acc += log(o->K[a] * lt);
            }
            D = exp(acc / (double)o->n);
        }
        o->D_ref = D;
        o->s = (o->tau_p - 0.5) / (3.0 * D);
    } else {
        o->s = o->dt / (o->dx * o->dx);
    }
    relaxation_time_f(o);
    int st = pressure_solve(o, init_replay, k_out, r_out);
    if (st == ORC_ENOMEM || st == ORC_ENONFINITE)
        return st;
    /* pressure gradient of the converged state (Eq. 3-10a) */
    stream_f(o);
    pressure_from_fpre(o, o->P);
    gradient_from_fpre(o);
    /* dt F_s at t = 0, with S* = S_0 at the producer */
    saturation_source(o, S0);
    for (int y = 0; y < o->ny; ++y) {
        for (int x = 0; x < o->nx; ++x) {
            size_t a = (size_t)y * o->nx + x;
            const double tg = tau_g_at(o, a, S0[a]);
            double sxX = fd_axis(o, S0, x, y, 0);
            double syX = fd_axis(o, S0, x, y, 1);
            double lw, lt;
            mobility(o, S0[a], &lw, &lt);
            double gam_t = -3.0 * lw * o->K[a] * o->dt / (o->dx * o->dx);
            for (int i = 0; i < o->qs; ++i) {
                double cS = EX[i] * sxX + EY[i] * syX;
                double cP = EX[i] * o->gxX[a] + EY[i] * o->gyX[a];
                /* Eq. gneq in lattice units */
                double neq = -tg * ((o->Gam[i] / o->phi - o->wg[i] * (1.0 - 1.0 / (2.0 * tg))) * o->Fs_t[a]
                                    + o->Gam[i] * cS - gam_t * o->wg[i] * cP / tg);
                o->gpre[i][a] = o->Gam[i] * S0[a] + neq;   /* Eq. gini */
            }
        }
    }
    /* S at t = 0 from the initial g (Eq. 3-9b), then the t = 0 collision */
    for (size_t a = 0; a < o->n; ++a) {
        double s = 0.0;
        for (int i = 0; i < o->qs; ++i)
            s += o->gpre[i][a];
        o->S[a] = (s + 0.5 * o->Fs_t[a]) / o->phi;
    }
    collide_g(o);
    memcpy(o->Pstep, o->P, o->n * sizeof(double));
    o->step = 0;
    return st;
}

/* Warm start of a solve: f_i^+ += f_i^eq(P^n - P^{n-1}) (Eq. 3-3: (omega_0 - 1) dP for
   i = 0, omega_i dP otherwise), then remember P^n. */
static void extrapolate_start(orc *o)
{
    for (size_t a = 0; a < o->n; ++a) {
        double dP = o->P[a] - o->Pstep[a];
        for (int i = 0; i < 9; ++i)
            o->f[i][a] += (i == 0 ? o->w[0] - 1.0 : o->w[i]) * dP;
        o->Pstep[a] = o->P[a];
    }
}

/* Create the oracle and run the t = 0 initialisation.
   iparams: nx, ny, mobility, tau_mode, max_sub, check_every, bc[4], init_replay,
            saturation lattice (9 or 5), warm start (0 or 1) (13 ints)
   dparams: dx, dt, phi, beta, mu_w, mu_n, D_s, tau_p, D_ref, tol, D_c (11 doubles)
   wells:   nw entries of (i, j, is_producer) in wint and q in wq. */
orc *orc_create(const int *iparams, const double *dparams, const double *K, const double *S0,
                const double *P0, const double *Fp, const double *Fs, int nw, const int *wint,
                const double *wq, const double *const *Pb, const double *const *Sb, int *status,
                int *k_out, double *r_out)
{
    *status = ORC_EINVAL;
    int nx = iparams[0], ny = iparams[1];
    if (nx < 1 || ny < 1 || !K || !S0)
        return NULL;
    orc *o = calloc(1, sizeof(orc));
    if (!o) {
        *status = ORC_ENOMEM;
        return NULL;
    }
    o->nx = nx;
    o->ny = ny;
    o->n = (size_t)nx * ny;
    o->mobility = iparams[2];
    o->tau_mode = iparams[3];
    o->max_sub = iparams[4];
    o->check_every = iparams[5];
    for (int s = 0; s < 4; ++s)
        o->bc[s] = iparams[6 + s];
    int init_replay = iparams[10];
    o->qs = iparams[11];
    o->warm_start = iparams[12];
    o->dx = dparams[0];
    o->dt = dparams[1];
    o->phi = dparams[2];
    o->beta = dparams[3];
    o->mu_w = dparams[4];
    o->mu_n = dparams[5];
    o->D_s = dparams[6];
    o->tau_p = dparams[7];
    o->D_ref = dparams[8];
    o->tol = dparams[9];
    o->D_c = dparams[10];
    if ((o->qs != 9 && o->qs != 5) || o->check_every < 1 || o->max_sub < 1 || (o->bc[0] == PERIODIC) != (o->bc[1] == PERIODIC) ||
        (o->bc[2] == PERIODIC) != (o->bc[3] == PERIODIC)) {
        free(o);
        return NULL;
    }
    set_constants(o);
    /* Eq. 3-11b: D_s = beta c_s^2 (tau_g - 1/2) dt with c_s^2 = (dx/dt)^2 / 3 */
    o->tau_g = 0.5 + 3.0 * o->D_s * o->dt / (o->beta * o->dx * o->dx);
    size_t bytes = o->n * sizeof(double);
    int ok = 1;
#define ALLOC(p) do { (p) = calloc(o->n, sizeof(double)); ok = ok && (p); } while (0)
    ALLOC(o->K);
    for (int i = 0; i < 9; ++i) {
        ALLOC(o->f[i]);
        ALLOC(o->fpre[i]);
        ALLOC(o->g[i]);
        ALLOC(o->gpre[i]);
    }
    ALLOC(o->tauf);
    ALLOC(o->Fp);
    ALLOC(o->Fs);
    ALLOC(o->Fs_t);
    ALLOC(o->S);
    ALLOC(o->P);
    ALLOC(o->Pprev);
    ALLOC(o->Pstep);
    ALLOC(o->gxX);
    ALLOC(o->gyX);
#undef ALLOC
    for (int s = 0; s < 4; ++s) {
        o->Pb[s] = calloc((size_t)trace_len(o, s), sizeof(double));
        o->Sb[s] = calloc((size_t)trace_len(o, s), sizeof(double));
        ok = ok && o->Pb[s] && o->Sb[s];
    }
    o->nw = nw;
    o->wi = calloc(nw > 0 ? nw : 1, sizeof(int));
    o->wj = calloc(nw > 0 ? nw : 1, sizeof(int));
    o->wprod = calloc(nw > 0 ? nw : 1, sizeof(int));
    o->wq = calloc(nw > 0 ? nw : 1, sizeof(double));
    ok = ok && o->wi && o->wj && o->wprod && o->wq;
    if (!ok) {
        orc_destroy(o);
        *status = ORC_ENOMEM;
        return NULL;
    }
    memcpy(o->K, K, bytes);
    orc_set_sources(o, Fp, Fs);
    for (int m = 0; m < nw; ++m) {
        o->wi[m] = wint[3 * m];
        o->wj[m] = wint[3 * m + 1];
        o->wprod[m] = wint[3 * m + 2];
        o->wq[m] = wq[m];
        if (o->wi[m] < 0 || o->wi[m] >= nx || o->wj[m] < 0 || o->wj[m] >= ny) {
            orc_destroy(o);
            return NULL;
        }
    }
    for (int s = 0; s < 4; ++s)
        if (o->bc[s] == DIRICHLET)
            orc_set_dirichlet(o, s, Pb ? Pb[s] : NULL, Sb ? Sb[s] : NULL);
    *status = initialise(o, P0, S0, init_replay, k_out, r_out);
    if (*status == ORC_ENOMEM || *status == ORC_ENONFINITE) {
        orc_destroy(o);
        return NULL;
    }
    return o;
}

/* a1: stream g, S^n (Eq. 3-9b), tau_f (Eq. 3-11a) */
void orc_refresh(orc *o)
{
    stream_g(o);
    saturation_from_gpre(o);
    relaxation_time_f(o);
}

/* a2/a3: exactly n pressure sweeps (r from the last one when n >= 1 and a previous
   sweep exists), or the sub-iteration to tol when n < 0 */
int orc_pressure(orc *o, int n, int *k_out, double *r_out)
{
    return pressure_solve(o, n, k_out, r_out);
}

/* a4/a5: stream f once more for P and grad P (Eq. 3-10a), stream g, S^n, collide g */
void orc_saturation(orc *o)
{
    stream_f(o);
    pressure_from_fpre(o, o->P);
    gradient_from_fpre(o);
    stream_g(o);
    saturation_from_gpre(o);
    collide_g(o);
}

/* One or more physical steps (Sec. 3 order: S^n, pressure at t_n, grad P^n, g update).
   replay: NULL, or nsteps sweep counts.  k_out/r_out: nsteps entries or NULL. */
int orc_step(orc *o, int nsteps, const int *replay, int *k_out, double *r_out)
{
    int worst = ORC_OK;
    for (int s = 0; s < nsteps; ++s) {
        orc_refresh(o);
        if (o->warm_start)
            extrapolate_start(o);
        int k;
        double r;
        int st = pressure_solve(o, replay ? replay[s] : -1, &k, &r);
        if (k_out)
            k_out[s] = k;
        if (r_out)
            r_out[s] = r;
        if (st == ORC_ENONFINITE || st == ORC_ENOMEM)
            return st;
        if (st != ORC_OK)
            worst = st;
        orc_saturation(o);
        o->step += 1;
    }
    return worst;
}

/* Fields of the current time level: P (Eq. 3-9a), S^n, physical grad P and the Darcy
   velocity u = -K lambda_t grad P (Eq. 3-10b).  Any pointer may be NULL. */
void orc_fields(const orc *o, double *P, double *S, double *gx, double *gy, double *ux, double *uy)
{
    for (size_t a = 0; a < o->n; ++a) {
        double gpx = o->gxX[a] / o->dx, gpy = o->gyX[a] / o->dx;
        double lw, lt;
        mobility(o, o->S[a], &lw, &lt);
        if (P) P[a] = o->P[a];
        if (S) S[a] = o->S[a];
        if (gx) gx[a] = gpx;
        if (gy) gy[a] = gpy;
        if (ux) ux[a] = -o->K[a] * lt * gpx;
        if (uy) uy[a] = -o->K[a] * lt * gpy;
    }
}

/* Raw state: 9 f^+ planes, 9 g^+ planes, tau_f, S (each ny*nx). */
void orc_get_state(const orc *o, double *f, double *g, double *tauf, double *S)
{
    for (int i = 0; i < 9; ++i) {
        if (f) memcpy(f + (size_t)i * o->n, o->f[i], o->n * sizeof(double));
        if (g) memcpy(g + (size_t)i * o->n, o->g[i], o->n * sizeof(double));
    }
    if (tauf) memcpy(tauf, o->tauf, o->n * sizeof(double));
    if (S) memcpy(S, o->S, o->n * sizeof(double));
}

void orc_set_state(orc *o, const double *f, const double *g, const double *tauf, const double *S)
{
    for (int i = 0; i < 9; ++i) {
        if (f) memcpy(o->f[i], f + (size_t)i * o->n, o->n * sizeof(double));
        if (g) memcpy(o->g[i], g + (size_t)i * o->n, o->n * sizeof(double));
    }
    if (tauf) memcpy(o->tauf, tauf, o->n * sizeof(double));
    if (S) memcpy(o->S, S, o->n * sizeof(double));
}

/* The most recent pulled (pre-collision) populations: 9 f planes, 9 g planes.  Right after
   creation the g planes hold g(t = 0) of Eq. gini, before the t = 0 collision. */
void orc_get_pre(const orc *o, double *f, double *g)
{
    for (int i = 0; i < 9; ++i) {
        if (f) memcpy(f + (size_t)i * o->n, o->fpre[i], o->n * sizeof(double));
        if (g) memcpy(g + (size_t)i * o->n, o->gpre[i], o->n * sizeof(double));
    }
}

/* Last-sweep pressure used by the next residual (P^{k-1}). */
void orc_set_prev_pressure(orc *o, const double *P)
{
    memcpy(o->Pprev, P, o->n * sizeof(double));
}

/* Scalars: [s, tau_g (of the constant D_s), D_ref, step, last_r, last_k] */
void orc_scalars(const orc *o, double *out)
{
    out[0] = o->s;
    out[1] = o->tau_g;
    out[2] = o->D_ref;
    out[3] = (double)o->step;
    out[4] = o->last_r;
    out[5] = (double)o->last_k;
}

/* Lattice constants: w[9], wbar[9], Gamma[9], ex[9], ey[9], opp[9], then the saturation
   lattice's weights wg[9] and its size (as doubles). */
void orc_constants(const orc *o, double *out)
{
    for (int i = 0; i < 9; ++i) {
        out[i] = o->w[i];
        out[9 + i] = o->wbar[i];
        out[18 + i] = o->Gam[i];
        out[27 + i] = EX[i];
        out[36 + i] = EY[i];
        out[45 + i] = OPP[i];
        out[54 + i] = o->wg[i];
    }
    out[63] = (double)o->qs;
}

/* sums over all nodes of sum_i f_i^+ and sum_i g_i^+ (conservation checks) */
void orc_sums(const orc *o, double *out)
{
    double sf = 0.0, sg = 0.0;
    for (size_t a = 0; a < o->n; ++a)
        for (int i = 0; i < 9; ++i) {
            sf += o->f[i][a];
            sg += o->g[i][a];
        }
    out[0] = sf;
    out[1] = sg;
}

/* the current dt*F_s plane (wells included) */
void orc_saturation_source(const orc *o, double *out)
{
    memcpy(out, o->Fs_t, o->n * sizeof(double));
}

/* Host threads of the oracle's node loops (OpenMP; 1 when built without it).  Used by the
   timing of the CPU baseline, never by the arithmetic: every loop is over independent nodes,
   so the results do not depend on the thread count. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
