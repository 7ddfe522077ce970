/*
 * FP64 CPU oracle of the two-species lattice Boltzmann model with multirange
 * Shan-Chen interactions (Benzi, Bernaschi, Sbragaglia, Succi, "Herschel-Bulkley
 * rheology from lattice kinetic theory of soft-glassy materials").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain definition the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two only receive the same input
 * arrays.
 *
 * Every step follows the paper's statement of the model, in the paper's order:
 *   Eq. (be)  f_is(r+c_i,t+1) - f_is(r,t) = -(1/tau)[f_is - f^eq_is(rho_s, u + tau F_s/rho_s)]
 *   moments   rho_s = sum_i f_is,  u = sum_s sum_i f_is c_i / sum_s rho_s
 *   f^eq      w_i rho_s (1 + u.c/cs^2 + uu:(cc - cs^2 I)/(2 cs^4)),  cs^2 = 1/3
 *   Eq. (FFF) F_s = F^a_s + F^r_s + F^X_s with
 *             F^{a,r}_s = -G^{a,r}_s psi_s(r) sum_{i in b1,b2} w_i c_i psi_s(r+c_i)
 *             F^X_s     = -(G_AB/rho0) rho_s(r) sum_{i in b1} w_i c_i rho_s'(r+c_i)
 *   psi(rho) = rho0 (1 - exp(-rho/rho0))  (Shan-Chen form, Section "Lattice
 *             Boltzmann with multirange interactions").
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - populations live on D2Q9; the 25 velocities of Fig. 1 are the interaction
 *    stencil only (c_s^2 = 1/3 holds for the D2Q9 weights);
 *  - belt-1 interaction weights are the standard D2Q9 weights the paper names,
 *    1/9 (|c|^2=1) and 1/36 (|c|^2=2); the two-belt weights are the 25-velocity
 *    set 4/63, 4/135, 1/180, 2/945, 1/15120 for |c|^2 = 1,2,4,5,8 (the paper
 *    defers them to its ref. [JCPnoi]).  Both sets have sum w c_x^2 = 1/3 = cs^2,
 *    and their fourth moments sum w c_x^2 c_y^2 are in the ratio 12/7 that the
 *    surface-tension combination G^a + (12/7) G^r of the paper requires;
 *  - G < 0 attracts, G > 0 repels (from the formula; the footnote's wording is
 *    reversed); G_BA = G_AB; the same rho0 enters psi and F^X;
 *  - order inside a step: moments and forces from the post-streaming state,
 *    collision, then streaming;
 *  - Couette walls (not in the paper): halfway bounce-back with a moving-wall
 *    term, walls at y=-1/2 (x-velocity -U) and y=ny-1/2 (+U); the interaction
 *    stencil sees mirror ghosts psi(x,-k) = psi(x,k-1), rho likewise;
 *  - sampled observables: physical velocity (j + F/2)/rho, wall x-momentum
 *    delivered by bounce-back per step (Pi_top, Pi_bot);
 *  - the Kolmogorov forcing of section "Numerical Results", F_x(y) = F0 sin(k_f y),
 *    k_f = 2 pi / L, is a force density shared by the species in proportion to
 *    their density (F_s gains (rho_s / rho) F_x), so it shifts both species'
 *    equilibrium velocities by tau F_x / rho;
 *  - a relaxation time per species (the coupling-dependent relaxation time the
 *    footnote of section "Numerical Results" leaves unexplored; all the paper's
 *    runs share tau = 1): species s relaxes with tau_s, is shifted by
 *    tau_s F_s / rho_s, and u is the common velocity of the two relaxations,
 *    u = (sum_s j_s / tau_s) / (sum_s rho_s / tau_s) (Shan and Doolen, J. Stat.
 *    Phys. 81 (1995) 379), which equals j / rho when the times are equal and
 *    keeps the collision from creating momentum when they are not;
 *  - a multiple-relaxation-time collision (the other form of a relaxation that
 *    depends on more than one time; not in the paper): f* = f - M^-1 S M (f - f^eq)
 *    with M the orthogonal D2Q9 moment basis of Lallemand and Luo (Phys. Rev. E
 *    61 (2000) 6546) and S = diag(s_k).  f^eq is the paper's shifted equilibrium,
 *    so the density and momentum moments relax with 1/tau_s (the rate at which
 *    the shift tau_s F_s / rho_s adds F_s per step); the energy e, its square
 *    eps, the energy flux q and the stress p relax with the cell's s_e, s_eps,
 *    s_q, s_nu, each 0 meaning 1/tau_s.  With all four 0 the collision is the
 *    paper's BGK one (taken on the BGK code path).  The shear viscosity is then
 *    (1/s_nu - 1/2)/3, independent of the forcing time tau.
 *
 * Layout of a population array: [species s=0(A),1(B)][i=0..8][y][x], x fastest.
 * D2Q9 order: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction).
 * Per-site loops may run on several OpenMP threads; every sum over sites is
 * taken in one fixed sequential order, so results do not depend on the thread
 * count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny;
    double tau, rho0;
    double g_aa1, g_aa2, g_bb1, g_bb2, g_ab;
    double u_wall;
    double f0;  /* Kolmogorov body force F_x(y) = f0 sin(2 pi y / ny) */
    int bc;     /* 0: periodic in x and y; 1: Couette (periodic x, walls in y) */
    double tau_b; /* relaxation time of species B; 0: tau (one time for both) */
    /* multiple-relaxation-time rates of the e, eps, q and p moments; 0: 1/tau_s */
    double s_e, s_eps, s_q, s_nu;
} orc_params;

/* Per-step observables of one sampled step (all FP64). */
typedef struct {
    double mass[2];      /* sum over sites of rho_A, rho_B (pre-collision) */
    double mom[2];       /* sum over sites of j_x, j_y (raw, pre-collision) */
    double pi_top;       /* x-momentum delivered by the top wall in this step */
    double pi_bot;       /* x-momentum delivered by the bottom wall in this step */
} orc_obs;

static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* Interaction weights by squared length |c|^2 of the stencil vector. */
static double belt1_weight(int c2)
{
    if (c2 == 1) return 1.0 / 9.0;
    if (c2 == 2) return 1.0 / 36.0;
    return 0.0;
}
static double belt2_weight(int c2)
{
    switch (c2) {
    case 1: return 4.0 / 63.0;
    case 2: return 4.0 / 135.0;
    case 4: return 1.0 / 180.0;
    case 5: return 2.0 / 945.0;
    case 8: return 1.0 / 15120.0;
    default: return 0.0;
    }
}

/* Exposed so tests can check the tables against what the paper fixes. */
double orc_belt_weight(int belt, int cx, int cy)
{
    int c2 = cx * cx + cy * cy;
    return belt == 1 ? belt1_weight(c2) : belt2_weight(c2);
}

#define IDX(p, x, y) ((size_t)(y) * (size_t)(p)->nx + (size_t)(x))
#define FIDX(p, s, i, x, y) ((((size_t)(s) * 9 + (size_t)(i)) * (size_t)(p)->ny + (size_t)(y)) * (size_t)(p)->nx + (size_t)(x))

static int wrap(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Row seen by the interaction stencil at row y+dy: periodic, or mirrored across
 * the walls at y=-1/2 and y=ny-1/2 (Couette). */
static int stencil_row(const orc_params* p, int y)
{
    if (p->bc == 0) return wrap(y, p->ny);
    if (y < 0) return -y - 1;
    if (y >= p->ny) return 2 * p->ny - y - 1;
    return y;
}

/* psi(rho) = rho0 (1 - exp(-rho/rho0)), written as -rho0*expm1(-rho/rho0). */
static double psi_of(double rho, double rho0) { return -rho0 * expm1(-rho / rho0); }

/* psi(rho)/rho with its limit 1 at rho -> 0. */
static double psi_over_rho(double rho, double rho0)
{
    if (rho == 0.0) return 1.0;
    return -rho0 * expm1(-rho / rho0) / rho;
}

static void set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* f_is = f^eq_is(rho_s, u) at every site.  ux/uy may be NULL (u = 0). */
void orc_equilibrium(const orc_params* p, const double* rho_a, const double* rho_b,
                     const double* ux, const double* uy, double* f)
{
    const double* rho[2] = {rho_a, rho_b};
    for (int s = 0; s < 2; ++s)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                size_t k = IDX(p, x, y);
                double u = ux ? ux[k] : 0.0, v = uy ? uy[k] : 0.0;
                double usq = u * u + v * v;
                for (int i = 0; i < 9; ++i) {
                    double cu = CX[i] * u + CY[i] * v;
                    f[FIDX(p, s, i, x, y)] = W[i] * rho[s][k] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                }
            }
}

/* Moments: rho_s = sum_i f_is; j = sum_s sum_i f_is c_i, taken as differences of
 * opposite populations so that a state at rest gives exactly j = 0. */
/* Row k of the orthogonal D2Q9 moment basis of Lallemand and Luo at velocity
 * c_i: the moments rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy are the
 * polynomials 1, 3c^2 - 4, (9c^4 - 21c^2 + 8)/2, c_x, (3c^2 - 5)c_x, c_y,
 * (3c^2 - 5)c_y, c_x^2 - c_y^2, c_x c_y of c = c_i (c^2 = c_x^2 + c_y^2). */
static double mrt_row(int k, int i)
{
    const double cx = CX[i], cy = CY[i], c2 = cx * cx + cy * cy;
    switch (k) {
    case 0: return 1.0;
    case 1: return 3.0 * c2 - 4.0;
    case 2: return (9.0 * c2 * c2 - 21.0 * c2 + 8.0) / 2.0;
    case 3: return cx;
    case 4: return (3.0 * c2 - 5.0) * cx;
    case 5: return cy;
    case 6: return (3.0 * c2 - 5.0) * cy;
    case 7: return cx * cx - cy * cy;
    default: return cx * cy;
    }
}

static int mrt_on(const orc_params* p) { return p->s_e != 0.0 || p->s_eps != 0.0 || p->s_q != 0.0 || p->s_nu != 0.0; }

/* The relaxed populations of one species at one site: BGK, f - (f - f^eq)/tau,
 * or, when the cell sets multiple-relaxation-time rates, f - M^-1 S M (f - f^eq)
 * with M^-1 = M^T D^-1, D = diag(sum_i M_ki^2) (the rows of M are orthogonal). */
static void relax(const orc_params* p, double tau, const double fi[9], const double feq[9], double out[9])
{
    if (!mrt_on(p)) {
        for (int i = 0; i < 9; ++i) out[i] = fi[i] - (fi[i] - feq[i]) / tau;
        return;
    }
    const double om = 1.0 / tau;
    const double s[9] = {om, p->s_e != 0.0 ? p->s_e : om, p->s_eps != 0.0 ? p->s_eps : om, om,
                         p->s_q != 0.0 ? p->s_q : om, om, p->s_q != 0.0 ? p->s_q : om,
                         p->s_nu != 0.0 ? p->s_nu : om, p->s_nu != 0.0 ? p->s_nu : om};
    double n[9];
    for (int k = 0; k < 9; ++k) {
        double m = 0.0, d = 0.0;
        for (int i = 0; i < 9; ++i) {
            m += mrt_row(k, i) * (fi[i] - feq[i]);
            d += mrt_row(k, i) * mrt_row(k, i);
        }
        n[k] = s[k] * m / d;
    }
    for (int i = 0; i < 9; ++i) {
        double c = 0.0;
        for (int k = 0; k < 9; ++k) c += mrt_row(k, i) * n[k];
        out[i] = fi[i] - c;
    }
}

/* Relaxation time of species s: tau for A; tau_b for B, or tau when tau_b is 0. */
static double tau_of(const orc_params* p, int s)
{
    return s == 1 && p->tau_b != 0.0 ? p->tau_b : p->tau;
}

/* The common velocity u = (j_A / tau_A + j_B / tau_B) / (rho_A / tau_A + rho_B / tau_B)
 * multiplied through by tau_A: u = (j_A + r j_B) / (rho_A + r rho_B), r = tau_A / tau_B.
 * With one relaxation time r = 1 and this is u = j / rho bit for bit. */
static double mix_ratio(const orc_params* p)
{
    return tau_of(p, 0) / tau_of(p, 1);
}

static void site_moments(const orc_params* p, const double* f, int x, int y,
                         double rho[2], double j[2], double jw[2])
{
    j[0] = 0.0;
    j[1] = 0.0;
    double jx_s[2], jy_s[2];
    for (int s = 0; s < 2; ++s) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[FIDX(p, s, i, x, y)];
        rho[s] = r;
        double f1 = f[FIDX(p, s, 1, x, y)], f2 = f[FIDX(p, s, 2, x, y)];
        double f3 = f[FIDX(p, s, 3, x, y)], f4 = f[FIDX(p, s, 4, x, y)];
        double f5 = f[FIDX(p, s, 5, x, y)], f6 = f[FIDX(p, s, 6, x, y)];
        double f7 = f[FIDX(p, s, 7, x, y)], f8 = f[FIDX(p, s, 8, x, y)];
        jx_s[s] = (f1 - f3) + (f5 - f7) + (f8 - f6);
        jy_s[s] = (f2 - f4) + (f5 - f7) + (f6 - f8);
    }
    j[0] = jx_s[0] + jx_s[1];
    j[1] = jy_s[0] + jy_s[1];
    if (jw) {
        const double r = mix_ratio(p);
        jw[0] = jx_s[0] + r * jx_s[1];
        jw[1] = jy_s[0] + r * jy_s[1];
    }
}

void orc_moments(const orc_params* p, const double* f, double* rho_a, double* rho_b,
                 double* jx, double* jy)
{
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double rho[2], j[2];
            site_moments(p, f, x, y, rho, j, NULL);
            size_t k = IDX(p, x, y);
            if (rho_a) rho_a[k] = rho[0];
            if (rho_b) rho_b[k] = rho[1];
            if (jx) jx[k] = j[0];
            if (jy) jy[k] = j[1];
        }
}

/* Stencil sums of Eq. (FFF) at one site, for species s, taken over the half
 * stencils b+ (one vector of each +-c pair) as w_c c (g(r+c) - g(r-c)):
 *   S1 = sum_{b1} w c psi_s(r+c),  S2 = sum_{b1+b2} p c psi_s(r+c),
 *   X  = sum_{b1} w c rho_s'(r+c). */
static void stencil_sums(const orc_params* p, const double* psi_s, const double* rho_o,
                         int x, int y, double S1[2], double S2[2], double X[2])
{
    S1[0] = S1[1] = S2[0] = S2[1] = X[0] = X[1] = 0.0;
    for (int dy = 0; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            if (dy == 0 && dx <= 0) continue; /* keep one vector of each pair */
            int c2 = dx * dx + dy * dy;
            int xp = wrap(x + dx, p->nx), yp = stencil_row(p, y + dy);
            int xm = wrap(x - dx, p->nx), ym = stencil_row(p, y - dy);
            double dpsi = psi_s[IDX(p, xp, yp)] - psi_s[IDX(p, xm, ym)];
            double w1 = belt1_weight(c2), w2 = belt2_weight(c2);
            if (w1 != 0.0) {
                double drho = rho_o[IDX(p, xp, yp)] - rho_o[IDX(p, xm, ym)];
                S1[0] += w1 * dx * dpsi;
                S1[1] += w1 * dy * dpsi;
                X[0] += w1 * dx * drho;
                X[1] += w1 * dy * drho;
            }
            S2[0] += w2 * dx * dpsi;
            S2[1] += w2 * dy * dpsi;
        }
}

static void coupling(const orc_params* p, int s, double* ga, double* gr)
{
    *ga = s == 0 ? p->g_aa1 : p->g_bb1;
    *gr = s == 0 ? p->g_aa2 : p->g_bb2;
}

/* Forces of Eq. (FFF) from given density fields (rho_a, rho_b: [ny][nx]).
 * Outputs F_A and F_B components; any output may be NULL. */
void orc_forces(const orc_params* p, const double* rho_a, const double* rho_b,
                double* fax, double* fay, double* fbx, double* fby)
{
    size_t n = (size_t)p->nx * p->ny;
    double* psi = (double*)malloc(2 * n * sizeof(double));
    const double* rho[2] = {rho_a, rho_b};
    for (int s = 0; s < 2; ++s)
        for (size_t k = 0; k < n; ++k) psi[s * n + k] = psi_of(rho[s][k], p->rho0);
    double* out[2][2] = {{fax, fay}, {fbx, fby}};
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t k = IDX(p, x, y);
            for (int s = 0; s < 2; ++s) {
                double S1[2], S2[2], X[2], ga, gr;
                stencil_sums(p, psi + s * n, rho[1 - s], x, y, S1, S2, X);
                coupling(p, s, &ga, &gr);
                for (int a = 0; a < 2; ++a) {
                    double F = -psi[s * n + k] * (ga * S1[a] + gr * S2[a]) - (p->g_ab / p->rho0) * rho[s][k] * X[a];
                    if (out[s][a]) out[s][a][k] = F;
                }
            }
        }
    free(psi);
}

/*
 * One time step of Eq. (be): f_in (post-streaming state at t) -> f_out (t+1).
 * If obs != NULL the step's observables are written to *obs, and profile
 * (length ny, may be NULL) receives sum_x u_phys_x(x, y) with
 * u_phys = (j + (F_A + F_B)/2) / rho at time t.
 */
void orc_step(const orc_params* p, const double* f_in, double* f_out, orc_obs* obs, double* profile)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    const double rho0 = p->rho0, rmix = mix_ratio(p);
    double* rho = (double*)malloc(2 * n * sizeof(double));
    double* psi = (double*)malloc(2 * n * sizeof(double));
    double* jj = (double*)malloc(2 * n * sizeof(double));
    double* jw = (double*)malloc(2 * n * sizeof(double)); /* numerator of the common velocity */
    double* fst = (double*)malloc(18 * n * sizeof(double)); /* post-collision f* */
    double* uphys = (double*)malloc(n * sizeof(double));

    /* 1-2. moments and pseudopotential at every site */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double r[2], j[2], w[2];
            site_moments(p, f_in, x, y, r, j, w);
            size_t k = IDX(p, x, y);
            rho[k] = r[0];
            rho[n + k] = r[1];
            jj[k] = j[0];
            jj[n + k] = j[1];
            jw[k] = w[0];
            jw[n + k] = w[1];
            psi[k] = psi_of(r[0], rho0);
            psi[n + k] = psi_of(r[1], rho0);
        }

    /* 3-6. forces, shifted equilibrium, BGK collision */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t k = IDX(p, x, y);
            double rtot = rho[k] + rho[n + k];
            double rw = rho[k] + rmix * rho[n + k];
            double u[2] = {jw[k] / rw, jw[n + k] / rw}; /* j / rho for one relaxation time */
            double Ftot[2] = {0.0, 0.0};
            const double pi = 3.14159265358979323846;
            const double fx_body = p->f0 == 0.0 ? 0.0 : p->f0 * sin(2.0 * pi * y / p->ny);
            for (int s = 0; s < 2; ++s) {
                double S1[2], S2[2], X[2], ga, gr;
                stencil_sums(p, psi + s * n, rho + (1 - s) * n, x, y, S1, S2, X);
                coupling(p, s, &ga, &gr);
                double rs = rho[s * n + k];
                double por = psi_over_rho(rs, rho0);
                const double tau = tau_of(p, s);
                double us[2];
                for (int a = 0; a < 2; ++a) {
                    /* F_s and the shift tau F_s / rho_s, without dividing by rho_s */
                    double G = ga * S1[a] + gr * S2[a];
                    double F = -psi[s * n + k] * G - (p->g_ab / rho0) * rs * X[a];
                    double body = a == 0 ? fx_body : 0.0;  /* F_x shared as rho_s / rho */
                    Ftot[a] += F + (rs / rtot) * body;
                    us[a] = u[a] - tau * (por * G + (p->g_ab / rho0) * X[a]) + tau * body / rtot;
                }
                double usq = us[0] * us[0] + us[1] * us[1];
                double fi[9], feq[9], fo[9];
                for (int i = 0; i < 9; ++i) {
                    double cu = CX[i] * us[0] + CY[i] * us[1];
                    feq[i] = W[i] * rs * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                    fi[i] = f_in[FIDX(p, s, i, x, y)];
                }
                relax(p, tau, fi, feq, fo);
                for (int i = 0; i < 9; ++i) fst[FIDX(p, s, i, x, y)] = fo[i];
            }
            uphys[k] = (jj[k] + 0.5 * Ftot[0]) / rtot;
        }

    /* 7. streaming; Couette rows use halfway bounce-back with the moving wall term
     *    f_ibar(x_b, t+1) = f*_i(x_b, t) - 2 w_i rho_s(x_b) (c_i . u_w) / cs^2.   */
    double pi_top = 0.0, pi_bot = 0.0;
    const double u_top = p->u_wall, u_bot = -p->u_wall;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 9; ++i)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double v = fst[FIDX(p, s, i, x, y)];
                    int yd = y + CY[i];
                    if (p->bc == 1 && (yd < 0 || yd >= ny)) {
                        double uw = yd < 0 ? u_bot : u_top;
                        double rs = rho[s * n + IDX(p, x, y)];
                        double back = v - 2.0 * W[i] * rs * (CX[i] * uw) * 3.0;
                        f_out[FIDX(p, s, OPP[i], x, y)] = back;
                        /* x-momentum delivered to the fluid by this wall link */
                        double dpx = (double)CX[OPP[i]] * back - (double)CX[i] * v;
                        if (yd < 0) pi_bot += dpx; else pi_top += dpx;
                    } else {
                        int xd = wrap(x + CX[i], nx);
                        yd = wrap(yd, ny);
                        f_out[FIDX(p, s, i, xd, yd)] = v;
                    }
                }

    if (obs) {
        double m[2] = {0.0, 0.0}, mo[2] = {0.0, 0.0};
        for (size_t k = 0; k < n; ++k) {
            m[0] += rho[k];
            m[1] += rho[n + k];
            mo[0] += jj[k];
            mo[1] += jj[n + k];
        }
        obs->mass[0] = m[0];
        obs->mass[1] = m[1];
        obs->mom[0] = mo[0];
        obs->mom[1] = mo[1];
        obs->pi_top = pi_top;
        obs->pi_bot = pi_bot;
    }
    if (profile)
        for (int y = 0; y < ny; ++y) {
            double acc = 0.0;
            for (int x = 0; x < nx; ++x) acc += uphys[IDX(p, x, y)];
            profile[y] = acc;
        }
    free(rho);
    free(psi);
    free(jj);
    free(jw);
    free(fst);
    free(uphys);
}

/*
 * The same time step for one horizontal slab of the cell, rows [y0, y0 + rows),
 * as one rank of a decomposition of the cell over several hosts would take it.
 * It restates orc_step site by site, so a decomposed run equals the whole-cell
 * run bit for bit.
 *
 * Slab arrays hold rows + 4 rows, [s][i][e][x] with slab row e = global row
 * y0 - 2 + e (taken mod ny for a periodic cell).
 *   f_in:  rows y0 .. y0+rows-1 of the post-streaming state at t, and in the two
 *          rows on each side copies of the neighbours' rows y0-2, y0-1 and
 *          y0+rows, y0+rows+1 (at a Couette wall those rows are not read: the
 *          interaction stencil mirrors into the cell).
 *   f_out: the slab's rows of the state at t+1, except the populations that
 *          stream in from the neighbours (c_y = +1 into the first row, c_y = -1
 *          into the last), which it does not write; and in slab rows 1 and rows+2
 *          the populations that stream out of the slab, for the neighbours.
 * obs (nullable) receives the slab's share of the step's observables (its rows'
 * sums; Pi of the walls it holds); profile (nullable, length rows) the row sums
 * of u_phys_x of its rows.  Returns -1 if rows + 4 > ny for a periodic cell or
 * the slab leaves the cell, else 0.
 */
#define SIDX(p, nr, s, i, x, e) ((((size_t)(s) * 9 + (size_t)(i)) * (size_t)(nr) + (size_t)(e)) * (size_t)(p)->nx + (size_t)(x))

/* Slab row of the global row the interaction stencil sees at y. */
static int slab_row(const orc_params* p, int y0, int y)
{
    int g = stencil_row(p, y);
    return p->bc == 0 ? wrap(g - y0 + 2, p->ny) : g - y0 + 2;
}

int orc_step_slab(const orc_params* p, int y0, int rows, const double* f_in, double* f_out,
                  orc_obs* obs, double* profile)
{
    const int nx = p->nx, ny = p->ny, nr = rows + 4;
    if (rows < 1 || y0 < 0 || y0 + rows > ny || (p->bc == 0 && nr > ny)) return -1;
    const size_t n = (size_t)nx * nr;
    const double rho0 = p->rho0, rmix = mix_ratio(p);
    double* rho = (double*)calloc(2 * n, sizeof(double));
    double* psi = (double*)calloc(2 * n, sizeof(double));
    double* jj = (double*)calloc(2 * n, sizeof(double));
    double* jw = (double*)calloc(2 * n, sizeof(double));
    double* fst = (double*)calloc(18 * n, sizeof(double));
    double* uphys = (double*)calloc(n, sizeof(double));

    /* 1-2. moments and pseudopotential on every held row */
    for (int e = 0; e < nr; ++e)
        for (int x = 0; x < nx; ++x) {
            size_t k = (size_t)e * nx + x;
            double jx_s[2], jy_s[2];
            for (int s = 0; s < 2; ++s) {
                double r = 0.0;
                for (int i = 0; i < 9; ++i) r += f_in[SIDX(p, nr, s, i, x, e)];
                rho[s * n + k] = r;
                double f1 = f_in[SIDX(p, nr, s, 1, x, e)], f2 = f_in[SIDX(p, nr, s, 2, x, e)];
                double f3 = f_in[SIDX(p, nr, s, 3, x, e)], f4 = f_in[SIDX(p, nr, s, 4, x, e)];
                double f5 = f_in[SIDX(p, nr, s, 5, x, e)], f6 = f_in[SIDX(p, nr, s, 6, x, e)];
                double f7 = f_in[SIDX(p, nr, s, 7, x, e)], f8 = f_in[SIDX(p, nr, s, 8, x, e)];
                jx_s[s] = (f1 - f3) + (f5 - f7) + (f8 - f6);
                jy_s[s] = (f2 - f4) + (f5 - f7) + (f6 - f8);
                psi[s * n + k] = psi_of(r, rho0);
            }
            jj[k] = jx_s[0] + jx_s[1];
            jj[n + k] = jy_s[0] + jy_s[1];
            jw[k] = jx_s[0] + rmix * jx_s[1];
            jw[n + k] = jy_s[0] + rmix * jy_s[1];
        }

    /* 3-6. forces, shifted equilibrium and collision on the slab's own rows */
    for (int yl = 0; yl < rows; ++yl)
        for (int x = 0; x < nx; ++x) {
            const int y = y0 + yl, e = yl + 2;
            size_t k = (size_t)e * nx + x;
            double rtot = rho[k] + rho[n + k];
            double rw = rho[k] + rmix * rho[n + k];
            double u[2] = {jw[k] / rw, jw[n + k] / rw};
            double Ftot[2] = {0.0, 0.0};
            const double pi = 3.14159265358979323846;
            const double fx_body = p->f0 == 0.0 ? 0.0 : p->f0 * sin(2.0 * pi * y / p->ny);
            for (int s = 0; s < 2; ++s) {
                const double* ps = psi + s * n;
                const double* ro = rho + (1 - s) * n;
                double S1[2] = {0.0, 0.0}, S2[2] = {0.0, 0.0}, X[2] = {0.0, 0.0}, ga, gr;
                for (int dy = 0; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx) {
                        if (dy == 0 && dx <= 0) continue;
                        int c2 = dx * dx + dy * dy;
                        size_t kp = (size_t)slab_row(p, y0, y + dy) * nx + wrap(x + dx, nx);
                        size_t km = (size_t)slab_row(p, y0, y - dy) * nx + wrap(x - dx, nx);
                        double dpsi = ps[kp] - ps[km];
                        double w1 = belt1_weight(c2), w2 = belt2_weight(c2);
                        if (w1 != 0.0) {
                            double drho = ro[kp] - ro[km];
                            S1[0] += w1 * dx * dpsi;
                            S1[1] += w1 * dy * dpsi;
                            X[0] += w1 * dx * drho;
                            X[1] += w1 * dy * drho;
                        }
                        S2[0] += w2 * dx * dpsi;
                        S2[1] += w2 * dy * dpsi;
                    }
                coupling(p, s, &ga, &gr);
                double rs = rho[s * n + k];
                double por = psi_over_rho(rs, rho0);
                const double tau = tau_of(p, s);
                double us[2];
                for (int a = 0; a < 2; ++a) {
                    double G = ga * S1[a] + gr * S2[a];
                    double F = -psi[s * n + k] * G - (p->g_ab / rho0) * rs * X[a];
                    double body = a == 0 ? fx_body : 0.0;
                    Ftot[a] += F + (rs / rtot) * body;
                    us[a] = u[a] - tau * (por * G + (p->g_ab / rho0) * X[a]) + tau * body / rtot;
                }
                double usq = us[0] * us[0] + us[1] * us[1];
                double fi[9], feq[9], fo[9];
                for (int i = 0; i < 9; ++i) {
                    double cu = CX[i] * us[0] + CY[i] * us[1];
                    feq[i] = W[i] * rs * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                    fi[i] = f_in[SIDX(p, nr, s, i, x, e)];
                }
                relax(p, tau, fi, feq, fo);
                for (int i = 0; i < 9; ++i) fst[SIDX(p, nr, s, i, x, e)] = fo[i];
            }
            uphys[k] = (jj[k] + 0.5 * Ftot[0]) / rtot;
        }

    /* 7. streaming inside the slab and into slab rows 1 and rows+2; walls as in orc_step */
    double pi_top = 0.0, pi_bot = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 9; ++i)
            for (int yl = 0; yl < rows; ++yl)
                for (int x = 0; x < nx; ++x) {
                    const int y = y0 + yl, e = yl + 2;
                    double v = fst[SIDX(p, nr, s, i, x, e)];
                    int yd = y + CY[i];
                    if (p->bc == 1 && (yd < 0 || yd >= ny)) {
                        double uw = yd < 0 ? -p->u_wall : p->u_wall;
                        double rs = rho[s * n + (size_t)e * nx + x];
                        double back = v - 2.0 * W[i] * rs * (CX[i] * uw) * 3.0;
                        f_out[SIDX(p, nr, s, OPP[i], x, e)] = back;
                        double dpx = (double)CX[OPP[i]] * back - (double)CX[i] * v;
                        if (yd < 0) pi_bot += dpx; else pi_top += dpx;
                    } else {
                        f_out[SIDX(p, nr, s, i, wrap(x + CX[i], nx), e + CY[i])] = v;
                    }
                }

    if (obs) {
        double m[2] = {0.0, 0.0}, mo[2] = {0.0, 0.0};
        for (int e = 2; e < rows + 2; ++e)
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)e * nx + x;
                m[0] += rho[k];
                m[1] += rho[n + k];
                mo[0] += jj[k];
                mo[1] += jj[n + k];
            }
        obs->mass[0] = m[0];
        obs->mass[1] = m[1];
        obs->mom[0] = mo[0];
        obs->mom[1] = mo[1];
        obs->pi_top = pi_top;
        obs->pi_bot = pi_bot;
    }
    if (profile)
        for (int yl = 0; yl < rows; ++yl) {
            double acc = 0.0;
            for (int x = 0; x < nx; ++x) acc += uphys[(size_t)(yl + 2) * nx + x];
            profile[yl] = acc;
        }
    free(rho);
    free(psi);
    free(jj);
    free(jw);
    free(fst);
    free(uphys);
    return 0;
}

/* Time averages collected over sampled steps. */
typedef struct {
    double sum_pi_top, sum_pi_bot;
    long long n_samples;
} orc_acc;

/*
 * n_steps steps starting at absolute step t0 (f is updated in place).  A step t
 * is sampled if every > 0, t >= start and (t - start) % every == 0: then its
 * Pi_top/Pi_bot are added to acc and its row sums of u_phys_x to prof_acc
 * (length ny).  last_obs receives the observables of the last step (NULL ok).
 * threads <= 0 keeps the OpenMP default.
 */
void orc_run(const orc_params* p, double* f, long long t0, long long n_steps,
             long long start, long long every, orc_acc* acc, double* prof_acc,
             orc_obs* last_obs, int threads)
{
    set_threads(threads);
    size_t nf = (size_t)18 * p->nx * p->ny;
    double* g = (double*)malloc(nf * sizeof(double));
    double* prof = (double*)malloc((size_t)p->ny * sizeof(double));
    for (long long s = 0; s < n_steps; ++s) {
        long long t = t0 + s;
        int sampled = every > 0 && t >= start && (t - start) % every == 0;
        orc_obs o;
        int want_obs = sampled || (last_obs && s == n_steps - 1);
        orc_step(p, f, g, want_obs ? &o : NULL, sampled ? prof : NULL);
        if (sampled && acc) {
            acc->sum_pi_top += o.pi_top;
            acc->sum_pi_bot += o.pi_bot;
            acc->n_samples += 1;
            if (prof_acc)
                for (int y = 0; y < p->ny; ++y) prof_acc[y] += prof[y];
        }
        if (last_obs && s == n_steps - 1) *last_obs = o;
        memcpy(f, g, nf * sizeof(double));
    }
    free(g);
    free(prof);
}
