/*
 * mp_oracle.c -- plain FP64 CPU oracle of the sorption-modified moment-propagation
 * (MP) method of Levesque, Duvail, Pagonabarraga, Frenkel and Rotenberg,
 * "Accounting for adsorption and desorption in Lattice Boltzmann simulations"
 * (arXiv:1303.2470), and of the BGK lattice-Boltzmann fluid solve that feeds it.
 *
 * THIS IS TEST INFRASTRUCTURE. It is the slow, obviously correct statement of what the
 * GPU library computes, used only by tests/, by __graft_entry__.smoke() and by the
 * CPU-baseline / reference legs of bench.py. The product path never loads it, and it
 * shares no code, header, table or helper with the CUDA library.
 *
 * Everything is FP64, one lattice node at a time, in the order the paper states it.
 * Lattice units: dx = dt = 1. D3Q19 velocities (Sec. "Algorithm": the LB distribution is
 * "discretized over 19 values"); the weights are the standard D3Q19 constants.
 *
 * Readings of the paper taken here:
 *  R1  Eq. (newP) as printed adds desorbed mass back into P but never removes the adsorbed
 *      share P*p_a from P, so total mass would grow. At interfacial nodes the adsorption
 *      event competes with the moves: the stay fraction is 1 - sum_i p_i - p_a.
 *  R2  f_i/rho in the link probability p_i is the D3Q19 equilibrium f_i^eq(rho=1, u) of
 *      the steady LB velocity u, so f_i/rho - w_i = w_i [3 c.u + 9/2 (c.u)^2 - 3/2 u^2].
 *  R3  A link whose far end is solid carries no probability (p_i = 0); that share stays.
 *  R4  Interfacial nodes I = fluid nodes with at least one solid D3Q19 neighbour; one
 *      p_a = k_a dt/dx per node, independent of the exposed area.
 *  R5  The VACF uses the displacement of the first step as v(0): the velocity moment
 *      at t = 1 is P_g(r,1) = sum_i pi(r-c_i) p_i(r-c_i) c_ig, with no adsorbed share;
 *      Z(0) = sum_r pi(r) sum_i p_i(r) c_ig^2; D(t) = Z(0)/2 + sum_{m=1..t} Z(m).
 *  R6  Z and D are normalised by the total (free + adsorbed) tracer mass, which the
 *      Boltzmann weights of Sec. "Algorithm" make equal to one.
 *  R15 The LB body force acts on the largest connected cluster of fluid nodes (D3Q19
 *      links). In a sealed pocket a uniform force is balanced by pressure and the steady
 *      velocity is zero; applying it there would only excite the undamped period-2
 *      bounce-back mode of tiny pockets. Ties go to the cluster with the smallest node index.
 *  R16 Steady LB flow: at every residual check that fails, the populations are replaced
 *      by the mean of the last two iterates before stepping on. This leaves the fixed
 *      point of the update unchanged and removes the undamped period-2 modes that
 *      bounce-back sustains at nodes with few open links (for a lone node under a force
 *      the momentum alternates m, -(m + F) forever; the mean is the fixed point u = 0).
 *  Parity of the porous-medium runs is pinned only by invariants (mass, Gamma/rho,
 *  Z(0) closed form): the paper prints no porous-medium numbers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19

/* D3Q19 velocity set: rest, 6 faces, 12 edges; OPP[i] is the link with c = -c_i. */
static const int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const int OPP[NQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static const double WT[NQ] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* exported copies of the table so tests can check it against the lattice identities */
void or_d3q19(int* c /* 19x3 */, double* w /* 19 */, int* opp /* 19 */)
{
    for (int i = 0; i < NQ; ++i) {
        c[3 * i + 0] = CX[i];
        c[3 * i + 1] = CY[i];
        c[3 * i + 2] = CZ[i];
        w[i] = WT[i];
        opp[i] = OPP[i];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Lattice geometry: node n = x + nx*(y + ny*z), periodic on all three axes.             */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
} or_dims;

static int64_t node_of(const or_dims* d, int x, int y, int z)
{
    x = ((x % d->nx) + d->nx) % d->nx;
    y = ((y % d->ny) + d->ny) % d->ny;
    z = ((z % d->nz) + d->nz) % d->nz;
    return (int64_t)x + (int64_t)d->nx * ((int64_t)y + (int64_t)d->ny * z);
}

/* neighbour of node n along +s*c_i (s = +1 or -1) */
static int64_t neighbour(const or_dims* d, int64_t n, int i, int s)
{
    int x = (int)(n % d->nx);
    int y = (int)((n / d->nx) % d->ny);
    int z = (int)(n / ((int64_t)d->nx * d->ny));
    return node_of(d, x + s * CX[i], y + s * CY[i], z + s * CZ[i]);
}

/* Node classes of Sec. "Algorithm" (Boltzmann weights): 0 = solid (S), 1 = fluid not at
 * an interface (F \ I), 2 = interfacial fluid node (I, reading R4). */
int or_classify(int nx, int ny, int nz, const uint8_t* solid, uint8_t* cls,
                int64_t* n_fluid, int64_t* n_iface)
{
    or_dims d = {nx, ny, nz};
    int64_t N = (int64_t)nx * ny * nz, nf = 0, ni = 0;
    for (int64_t n = 0; n < N; ++n) {
        if (solid[n]) {
            cls[n] = 0;
            continue;
        }
        int touches_solid = 0;
        for (int i = 1; i < NQ; ++i)
            if (solid[neighbour(&d, n, i, +1)]) touches_solid = 1;
        cls[n] = touches_solid ? 2 : 1;
        nf += 1;
        ni += touches_solid;
    }
    if (n_fluid) *n_fluid = nf;
    if (n_iface) *n_iface = ni;
    return 0;
}

/* Largest connected cluster of fluid nodes, two fluid nodes being connected when a D3Q19
 * link joins them (periodic). in_cluster[n] = 1 on it, else 0; ties between equally large
 * clusters go to the one holding the smallest node index. Plain breadth-first search. */
int or_largest_cluster(int nx, int ny, int nz, const uint8_t* solid, uint8_t* in_cluster,
                       int64_t* size_out)
{
    or_dims d = {nx, ny, nz};
    int64_t N = (int64_t)nx * ny * nz;
    int64_t* comp = malloc(sizeof(int64_t) * N);
    int64_t* queue = malloc(sizeof(int64_t) * N);
    if (!comp || !queue) {
        free(comp);
        free(queue);
        return -1;
    }
    for (int64_t n = 0; n < N; ++n) comp[n] = -1;
    int64_t best_root = -1, best_size = 0;
    for (int64_t root = 0; root < N; ++root) {
        if (solid[root] || comp[root] >= 0) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = root;
        comp[root] = root;
        while (head < tail) {
            int64_t n = queue[head++];
            for (int i = 1; i < NQ; ++i) {
                int64_t m = neighbour(&d, n, i, +1);
                if (!solid[m] && comp[m] < 0) {
                    comp[m] = root;
                    queue[tail++] = m;
                }
            }
        }
        if (tail > best_size) {
            best_size = tail;
            best_root = root;
        }
    }
    for (int64_t n = 0; n < N; ++n) in_cluster[n] = (best_root >= 0 && comp[n] == best_root) ? 1 : 0;
    if (size_out) *size_out = best_size;
    free(comp);
    free(queue);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Moment propagation with sorption (Sec. "Algorithm").                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    const uint8_t* solid; /* N bytes, nonzero = solid node */
    const double* u;      /* 3*N, SoA: u_x[N], u_y[N], u_z[N]; NULL = fluid at rest */
    double D_b;           /* bulk diffusion coefficient, lattice units */
    double k_a;           /* adsorption rate (length/time), lattice units */
    double k_d;           /* desorption rate (1/time), lattice units */
} or_mp;

/* lambda from D_b = lambda c_s^2 dt / 4 with c_s^2 = 1/3 (Sec. "Algorithm") */
static double lambda_of(const or_mp* m) { return 12.0 * m->D_b; }

/* p_i(r) of Sec. "Algorithm" with Q = 1 (neutral tracers), f_i/rho read as the
 * equilibrium of the local LB velocity (R2), zero for a link into a solid node (R3). */
double or_link_prob(const or_mp* m, int64_t n, int i)
{
    or_dims d = {m->nx, m->ny, m->nz};
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    if (i == 0 || m->solid[n] || m->solid[neighbour(&d, n, i, +1)]) return 0.0;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (m->u) {
        ux = m->u[n];
        uy = m->u[N + n];
        uz = m->u[2 * N + n];
    }
    double cu = CX[i] * ux + CY[i] * uy + CZ[i] * uz;
    double uu = ux * ux + uy * uy + uz * uz;
    double f_over_rho = WT[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    return f_over_rho - WT[i] + WT[i] * lambda_of(m) / 2.0;
}

static int is_interface(const or_mp* m, int64_t n)
{
    or_dims d = {m->nx, m->ny, m->nz};
    if (m->solid[n]) return 0;
    for (int i = 1; i < NQ; ++i)
        if (m->solid[neighbour(&d, n, i, +1)]) return 1;
    return 0;
}

/* sum_i p_i(r) c_ig : mean displacement of a free tracer at r along g (0,1,2) */
double or_mean_step(const or_mp* m, int64_t n, int g)
{
    double s = 0.0;
    for (int i = 1; i < NQ; ++i) {
        int c = g == 0 ? CX[i] : (g == 1 ? CY[i] : CZ[i]);
        s += or_link_prob(m, n, i) * c;
    }
    return s;
}

/* The link probabilities p_i(r) of every node and link, and the interface flags, tabulated
 * once per problem (u is steady, so neither changes from step to step). */
typedef struct {
    int64_t N;
    double* p;      /* p[i*N + n] = p_i(r_n), i = 0..18 (p_0 = 0) */
    uint8_t* iface; /* 1 on I */
} or_tables;

static void tables_free(or_tables* T)
{
    free(T->p);
    free(T->iface);
    T->p = NULL;
    T->iface = NULL;
}

static int tables_make(const or_mp* m, or_tables* T)
{
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    T->N = N;
    T->p = malloc(sizeof(double) * NQ * N);
    T->iface = malloc(N);
    if (!T->p || !T->iface) {
        tables_free(T);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        for (int i = 0; i < NQ; ++i) T->p[(int64_t)i * N + n] = or_link_prob(m, n, i);
        T->iface[n] = (uint8_t)is_interface(m, n);
    }
    return 0;
}

/* One step t -> t+1 of one propagated quantity X with adsorbed partner Xa:
 *   P*(r)       = sum_i X(r-c_i) p_i(r-c_i) + X(r) (1 - sum_i p_i(r) - p_a 1_I(r))
 *                                                       (Eq. propagated_quantity, R1)
 *   Xa(r, t+1)  = X(r) p_a + Xa(r) (1 - p_d)            (Eq. Pads, r in I)
 *   X(r, t+1)   = P*(r) + Xa(r) p_d                     (Eq. newP, r in I)
 * with p_a = k_a dt/dx and p_d = k_d dt. Xa is stored densely (zero off I). */
static void propagate_with(const or_mp* m, const or_tables* T, const double* X, const double* Xa,
                           double* Xn, double* Xan)
{
    or_dims d = {m->nx, m->ny, m->nz};
    int64_t N = T->N;
    double p_a = m->k_a, p_d = m->k_d;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) {
            Xn[n] = 0.0;
            Xan[n] = 0.0;
            continue;
        }
        double inflow = 0.0;
        for (int i = 1; i < NQ; ++i) {
            int64_t src = neighbour(&d, n, i, -1); /* r - c_i */
            inflow += X[src] * T->p[(int64_t)i * N + src];
        }
        double leave = 0.0;
        for (int i = 1; i < NQ; ++i) leave += T->p[(int64_t)i * N + n];
        int iface = T->iface[n];
        double stay = 1.0 - leave - (iface ? p_a : 0.0);
        double pstar = inflow + X[n] * stay;
        if (iface) {
            Xan[n] = X[n] * p_a + Xa[n] * (1.0 - p_d);
            Xn[n] = pstar + Xa[n] * p_d;
        } else {
            Xan[n] = 0.0;
            Xn[n] = pstar;
        }
    }
}

int or_mp_propagate(const or_mp* m, const double* X, const double* Xa, double* Xn, double* Xan)
{
    or_tables T;
    if (tables_make(m, &T) != 0) return -1;
    propagate_with(m, &T, X, Xa, Xn, Xan);
    tables_free(&T);
    return 0;
}

/* Boltzmann weights of Sec. "Algorithm" for a neutral tracer (mu_ex = 0): free part
 * pi(r) = 1/Z on F, adsorbed part pi_ads(r) = K/Z on I with K = exp(-beta dmu_ads)
 * = k_a/(k_d dx); Z makes the total (free + adsorbed) mass one (R6). K = 0 when k_a = 0.
 * Returns -1 when k_a > 0 and k_d = 0 (no equilibrium exists). */
int or_equilibrium(const or_mp* m, double* pi, double* pi_ads)
{
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    double K;
    if (m->k_a == 0.0)
        K = 0.0;
    else if (m->k_d == 0.0)
        return -1;
    else
        K = m->k_a / m->k_d;
    double Zpart = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) continue;
        Zpart += is_interface(m, n) ? 1.0 + K : 1.0;
    }
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) {
            pi[n] = 0.0;
            pi_ads[n] = 0.0;
        } else {
            pi[n] = 1.0 / Zpart;
            pi_ads[n] = is_interface(m, n) ? K / Zpart : 0.0;
        }
    }
    return 0;
}

/* Velocity-weighted propagated quantity at t = 1 (R5): the probability to be at r after
 * the first step, weighted by that step's displacement along g. */
int or_moment_init(const or_mp* m, int g, const double* pi, double* Pg)
{
    or_dims d = {m->nx, m->ny, m->nz};
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    for (int64_t n = 0; n < N; ++n) {
        Pg[n] = 0.0;
        if (m->solid[n]) continue;
        for (int i = 1; i < NQ; ++i) {
            int64_t src = neighbour(&d, n, i, -1);
            if (m->solid[src]) continue;
            int c = g == 0 ? CX[i] : (g == 1 ? CY[i] : CZ[i]);
            Pg[n] += pi[src] * or_link_prob(m, src, i) * c;
        }
    }
    return 0;
}

/* Z_g(0) = <v_g(0)^2> = sum_r pi(r) sum_i p_i(r) c_ig^2 (R5, R6) */
double or_vacf_z0(const or_mp* m, int g, const double* pi)
{
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    double z = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) continue;
        double s = 0.0;
        for (int i = 1; i < NQ; ++i) {
            int c = g == 0 ? CX[i] : (g == 1 ? CY[i] : CZ[i]);
            s += or_link_prob(m, n, i) * c * c;
        }
        z += pi[n] * s;
    }
    return z;
}

/* Z_g(t) = sum_r P_g(r,t) sum_i p_i(r) c_ig (Sec. "Algorithm", last equation). Adsorbed
 * tracers do not move, so only the free moment enters. */
double or_vacf(const or_mp* m, int g, const double* Pg)
{
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    double z = 0.0;
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) continue;
        z += Pg[n] * or_mean_step(m, n, g);
    }
    return z;
}

/* sum over fluid nodes of a dense field */
double or_sum(int64_t N, const uint8_t* solid, const double* X)
{
    double s = 0.0;
    for (int64_t n = 0; n < N; ++n)
        if (!solid[n]) s += X[n];
    return s;
}

/* Full run for one direction g: initialise, then nsteps steps of both the density field
 * (P, Gamma) and the velocity moment (P_g, P_g,ads).
 *   init_mode 0: density starts at the equilibrium (pi, pi_ads);
 *   init_mode 1: density starts uniform over the free fluid, 1/N_f per node, Gamma = 0.
 * Both fields are at t = 1 after initialisation (the density is advanced one step from
 * t = 0). Outputs (each may be NULL):
 *   Z[0..nsteps+1], D[0..nsteps+1]          VACF and D(t) = Z(0)/2 + sum_{m<=t} Z(m)
 *   mass_free[0..nsteps+1], mass_ads[..]    sum_F P and sum_I Gamma of the density field
 *   iface_free[0..nsteps+1]                 sum_I P (for the Gamma/rho ratio at I)
 *   P, Pa, Pg, Pga (N each)                 final fields at t = nsteps+1
 * Returns 0, or -1 on invalid input. */
int or_mp_run(const or_mp* m, int g, int init_mode, int64_t nsteps, double* Z, double* D,
              double* mass_free, double* mass_ads, double* iface_free, double* P_out,
              double* Pa_out, double* Pg_out, double* Pga_out)
{
    int64_t N = (int64_t)m->nx * m->ny * m->nz;
    if (g < 0 || g > 2 || nsteps < 0) return -1;
    double* pi = calloc(N, sizeof(double));
    double* pi_ads = calloc(N, sizeof(double));
    double* X = calloc(N, sizeof(double));
    double* Xa = calloc(N, sizeof(double));
    double* Xn = calloc(N, sizeof(double));
    double* Xan = calloc(N, sizeof(double));
    double* G = calloc(N, sizeof(double));
    double* Ga = calloc(N, sizeof(double));
    double* Gn = calloc(N, sizeof(double));
    double* Gan = calloc(N, sizeof(double));
    int rc = 0;
    if (!pi || !pi_ads || !X || !Xa || !Xn || !Xan || !G || !Ga || !Gn || !Gan) {
        rc = -1;
        goto done;
    }
    if (or_equilibrium(m, pi, pi_ads) != 0) {
        rc = -1;
        goto done;
    }
    or_tables T;
    if (tables_make(m, &T) != 0) {
        rc = -1;
        goto done;
    }
    const uint8_t* iface = T.iface;
    int64_t nf = 0;
    for (int64_t n = 0; n < N; ++n) nf += m->solid[n] ? 0 : 1;
    /* mean displacement sum_i p_i(r) c_ig of a free tracer at each node (the second
     * factor of the VACF sum), from the tabulated p_i */
    double* ustar = calloc(N, sizeof(double));
    if (!ustar) {
        tables_free(&T);
        rc = -1;
        goto done;
    }
    for (int64_t n = 0; n < N; ++n) {
        if (m->solid[n]) continue;
        for (int i = 1; i < NQ; ++i) {
            int c = g == 0 ? CX[i] : (g == 1 ? CY[i] : CZ[i]);
            ustar[n] += T.p[(int64_t)i * N + n] * c;
        }
    }

    /* density field at t = 0 */
    for (int64_t n = 0; n < N; ++n) {
        if (init_mode == 0) {
            X[n] = pi[n];
            Xa[n] = pi_ads[n];
        } else {
            X[n] = m->solid[n] ? 0.0 : 1.0 / (double)nf;
            Xa[n] = 0.0;
        }
    }
#define RECORD_MASS(t)                                                              \
    do {                                                                            \
        double mf = 0.0, ma = 0.0, mi = 0.0;                                        \
        for (int64_t n = 0; n < N; ++n) {                                           \
            if (m->solid[n]) continue;                                              \
            mf += X[n];                                                             \
            ma += Xa[n];                                                            \
            if (iface[n]) mi += X[n];                                               \
        }                                                                           \
        if (mass_free) mass_free[t] = mf;                                           \
        if (mass_ads) mass_ads[t] = ma;                                             \
        if (iface_free) iface_free[t] = mi;                                         \
    } while (0)
    RECORD_MASS(0);
    propagate_with(m, &T, X, Xa, Xn, Xan);
    memcpy(X, Xn, N * sizeof(double));
    memcpy(Xa, Xan, N * sizeof(double));
    RECORD_MASS(1);

    /* velocity moment at t = 1, and Z(0), Z(1) */
    or_moment_init(m, g, pi, G);
    memset(Ga, 0, N * sizeof(double));
    double z0 = or_vacf_z0(m, g, pi);
    double z1 = or_vacf(m, g, G);
    if (Z) {
        Z[0] = z0;
        Z[1] = z1;
    }
    double d = z0 / 2.0;
    if (D) D[0] = d;
    d += z1;
    if (D) D[1] = d;

    for (int64_t t = 1; t <= nsteps; ++t) {
        propagate_with(m, &T, X, Xa, Xn, Xan);
        propagate_with(m, &T, G, Ga, Gn, Gan);
        double* tmp;
        tmp = X; X = Xn; Xn = tmp;
        tmp = Xa; Xa = Xan; Xan = tmp;
        tmp = G; G = Gn; Gn = tmp;
        tmp = Ga; Ga = Gan; Gan = tmp;
        double z = 0.0;
        for (int64_t n = 0; n < N; ++n)
            if (!m->solid[n]) z += G[n] * ustar[n];
        d += z;
        if (Z) Z[t + 1] = z;
        if (D) D[t + 1] = d;
        RECORD_MASS(t + 1);
    }
#undef RECORD_MASS
    if (P_out) memcpy(P_out, X, N * sizeof(double));
    if (Pa_out) memcpy(Pa_out, Xa, N * sizeof(double));
    if (Pg_out) memcpy(Pg_out, G, N * sizeof(double));
    if (Pga_out) memcpy(Pga_out, Ga, N * sizeof(double));
    tables_free(&T);
    free(ustar);
done:
    free(pi);
    free(pi_ads);
    free(X);
    free(Xa);
    free(Xn);
    free(Xan);
    free(G);
    free(Ga);
    free(Gn);
    free(Gan);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* BGK lattice Boltzmann (Eq. lb_evolution) with the Guo body-force term and halfway     */
/* bounce-back at solid links; tau is the BGK relaxation time, F a uniform body force    */
/* acting on fluid nodes. f is stored as f[i*N + n], post-collision.                     */
/* ------------------------------------------------------------------------------------ */

static void lb_equilibrium(double rho, const double u[3], double* feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NQ; ++i) {
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        feq[i] = WT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* f = f^eq(rho = 1, u0) on fluid nodes (u0 = 0 when NULL), f = w_i on solid nodes */
int or_lb_init(int nx, int ny, int nz, const uint8_t* solid, const double* u0, const double* rho0, double* f)
{
    int64_t N = (int64_t)nx * ny * nz;
    for (int64_t n = 0; n < N; ++n) {
        double u[3] = {0.0, 0.0, 0.0}, feq[NQ];
        if (u0 && !solid[n]) {
            u[0] = u0[n];
            u[1] = u0[N + n];
            u[2] = u0[2 * N + n];
        }
        lb_equilibrium((rho0 && !solid[n]) ? rho0[n] : 1.0, u, feq);
        for (int i = 0; i < NQ; ++i) f[(int64_t)i * N + n] = solid[n] ? WT[i] : feq[i];
    }
    return 0;
}

/* One LB step: stream (pull; halfway bounce-back where r - c_i is solid), then
 * rho = sum f, u = (sum f c + F/2)/rho, then BGK collision with the Guo source
 *   f' = f - (f - f^eq(rho,u))/tau + (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i.u) c_i].F
 * Writes the post-collision f_out and the velocity u_out (3*N, zero on solid nodes).
 * The force acts where forced[n] is nonzero (everywhere on the fluid when forced is NULL). */
int or_lb_step(int nx, int ny, int nz, const uint8_t* solid, const uint8_t* forced,
               const double F[3], double tau, const double* f, double* f_out, double* u_out)
{
    or_dims d = {nx, ny, nz};
    int64_t N = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (solid[n]) {
            for (int i = 0; i < NQ; ++i) f_out[(int64_t)i * N + n] = WT[i];
            u_out[n] = u_out[N + n] = u_out[2 * N + n] = 0.0;
            continue;
        }
        double fi[NQ];
        for (int i = 0; i < NQ; ++i) {
            int64_t src = neighbour(&d, n, i, -1);
            if (solid[src])
                fi[i] = f[(int64_t)OPP[i] * N + n];
            else
                fi[i] = f[(int64_t)i * N + src];
        }
        double rho = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
        for (int i = 0; i < NQ; ++i) {
            rho += fi[i];
            mx += fi[i] * CX[i];
            my += fi[i] * CY[i];
            mz += fi[i] * CZ[i];
        }
        double Fn[3] = {0.0, 0.0, 0.0};
        if (!forced || forced[n]) {
            Fn[0] = F[0];
            Fn[1] = F[1];
            Fn[2] = F[2];
        }
        double u[3] = {(mx + 0.5 * Fn[0]) / rho, (my + 0.5 * Fn[1]) / rho, (mz + 0.5 * Fn[2]) / rho};
        double feq[NQ];
        lb_equilibrium(rho, u, feq);
        for (int i = 0; i < NQ; ++i) {
            double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
            double sx = 3.0 * (CX[i] - u[0]) + 9.0 * cu * CX[i];
            double sy = 3.0 * (CY[i] - u[1]) + 9.0 * cu * CY[i];
            double sz = 3.0 * (CZ[i] - u[2]) + 9.0 * cu * CZ[i];
            double Si = (1.0 - 0.5 / tau) * WT[i] * (sx * Fn[0] + sy * Fn[1] + sz * Fn[2]);
            f_out[(int64_t)i * N + n] = fi[i] - (fi[i] - feq[i]) / tau + Si;
        }
        u_out[n] = u[0];
        u_out[N + n] = u[1];
        u_out[2 * N + n] = u[2];
    }
    return 0;
}

/* Runs LB steps from f^eq(1, u_init), with the force on the largest fluid cluster (R15)
 * and the two-iterate mean at failed checks (R16), until the residual
 *   res(t) = max over fluid nodes and components |u(t) - u(t-1)|
 * evaluated at every t that is a multiple of check_every (and at t = max_steps) is below
 * tol. u(0) = u_init (zero when NULL). Returns 0 when converged, 1 when max_steps ran out,
 * -1 on bad input; u_out gets u(steps). */
int or_lb_steady(int nx, int ny, int nz, const uint8_t* solid, const double F[3], double tau,
                 double tol, int64_t max_steps, int64_t check_every, const double* u_init,
                 const double* rho_init, double* u_out, double* rho_out, int64_t* steps_out,
                 double* residual_out, double* f_out)
{
    int64_t N = (int64_t)nx * ny * nz;
    if (tau <= 0.5 || max_steps < 1 || check_every < 1) return -1;
    double* f = malloc(sizeof(double) * NQ * N);
    double* fn = malloc(sizeof(double) * NQ * N);
    double* u = malloc(sizeof(double) * 3 * N);
    double* uprev = malloc(sizeof(double) * 3 * N);
    uint8_t* forced = malloc(N);
    if (!f || !fn || !u || !uprev || !forced ||
        or_largest_cluster(nx, ny, nz, solid, forced, NULL) != 0) {
        free(f); free(fn); free(u); free(uprev); free(forced);
        return -1;
    }
    or_lb_init(nx, ny, nz, solid, u_init, rho_init, f);
    for (int64_t k = 0; k < 3 * N; ++k) uprev[k] = u_init ? u_init[k] : 0.0;
    for (int64_t n = 0; n < N; ++n)
        if (solid[n]) uprev[n] = uprev[N + n] = uprev[2 * N + n] = 0.0;
    int rc = 1;
    int64_t t = 0;
    double res = INFINITY;
    while (t < max_steps) {
        or_lb_step(nx, ny, nz, solid, forced, F, tau, f, fn, u);
        double* tmp = f; f = fn; fn = tmp;
        t += 1;
        if (t % check_every == 0 || t == max_steps) {
            res = 0.0;
            for (int64_t n = 0; n < N; ++n) {
                if (solid[n]) continue;
                for (int c = 0; c < 3; ++c) {
                    double du = fabs(u[c * N + n] - uprev[c * N + n]);
                    if (du > res) res = du;
                }
            }
            if (res < tol) {
                rc = 0;
                break;
            }
            /* R16: replace the state by the mean of the last two iterates (f holds t, fn
             * holds t-1). The fixed point is unchanged; an error mode with eigenvalue lambda
             * is scaled by (1 + lambda)/2, which removes the undamped period-2 modes that
             * bounce-back sustains at strongly confined nodes. */
            if (t < max_steps)
                for (int64_t k = 0; k < (int64_t)NQ * N; ++k) f[k] = 0.5 * (f[k] + fn[k]);
        }
        memcpy(uprev, u, sizeof(double) * 3 * N);
    }
    memcpy(u_out, u, sizeof(double) * 3 * N);
    if (rho_out) /* density of the final state: the collision conserves it, so sum f^post */
        for (int64_t n = 0; n < N; ++n) {
            double r = 0.0;
            if (!solid[n])
                for (int i = 0; i < NQ; ++i) r += f[(int64_t)i * N + n];
            rho_out[n] = r;
        }
    if (steps_out) *steps_out = t;
    if (residual_out) *residual_out = res;
    if (f_out) memcpy(f_out, f, sizeof(double) * NQ * N); /* the final populations */
    free(f); free(fn); free(u); free(uprev); free(forced);
    return rc;
}
